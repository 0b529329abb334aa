// Register-blocked de-dispersion kernel (kernel 2).
#include "dd_internal.h"

namespace dd {

int fast_configure(dd_plan *p)
{
    p->fast = nullptr;
    return DD_OK;
}

int fast_execute(dd_plan *p, const void *, int64_t, void *, cudaStream_t)
{
    return set_error(DD_ERR_ARG, "kernel 2 unavailable");
}

void fast_release(dd_plan *p) { p->fast = nullptr; }

}  // namespace dd
