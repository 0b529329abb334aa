"""GB300-native brute-force incoherent de-dispersion and boxcar single-pulse
search (Magro et al. 2011, Section 3.1 and Section 3), with the Section 3.2
subband approximation, behind the C ABI of libdd.so (include/dd.h).  This
package is the thin Python binding; the library is built in-tree by
``paper_1107_2516_gb300.build.build()``.
"""
from .dd import (Batch, CANDIDATE_DTYPE, CHUNK_RESULT_DTYPE, CLUSTER_DTYPE, dd_cluster_candidates, DD_PRIMING, DD_ERR_SEQ, DD_SEQ_GAP, Server, SubbandPlan, SurveyPlan, SurveyPass, DD_F16,
                 DD_F32, DD_U8, DDError, EXPORTS, Plan, dd_execute, dd_last_error, dd_last_stats,
                 dd_plan_autotune, dd_plan_create, dd_plan_destroy, dd_plan_get_kernel,
                 dd_plan_get_tile, dd_plan_info, dd_plan_set_kernel, dd_plan_set_tile, dd_process_host,
                 dd_channelise, dd_search, dd_stats_f32_noalloc, dd_subband_execute, dd_subband_last_stats,
                 dd_subband_plan_create, dd_subband_plan_destroy, dd_subband_plan_info,
                 dd_subband_search, dd_server_ring_schedule, dd_version, load)

__all__ = ["Batch", "CANDIDATE_DTYPE", "CHUNK_RESULT_DTYPE", "CLUSTER_DTYPE", "dd_cluster_candidates", "DD_PRIMING", "DD_ERR_SEQ", "DD_SEQ_GAP", "Server", "SubbandPlan", "SurveyPlan", "SurveyPass",
           "DD_F16", "DD_F32", "DD_U8", "DDError", "EXPORTS", "Plan",
           "dd_execute", "dd_last_error", "dd_last_stats", "dd_plan_autotune", "dd_plan_create",
           "dd_plan_destroy", "dd_plan_get_kernel", "dd_plan_get_tile", "dd_plan_info",
           "dd_plan_set_kernel", "dd_plan_set_tile", "dd_process_host", "dd_search", "dd_channelise",
           "dd_stats_f32_noalloc", "dd_subband_execute", "dd_subband_last_stats",
           "dd_subband_plan_create", "dd_subband_plan_destroy", "dd_subband_plan_info",
           "dd_subband_search", "dd_server_ring_schedule", "dd_version", "load"]
