"""Candidate clustering (search variant): the library's friends-of-friends
grouping (host code, C ABI) against the oracle's plain all-pairs version, plus
its invariants.  No GPU needed."""
import numpy as np
import pytest

import oracle

dd = pytest.importorskip("paper_1107_2516_gb300")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1107_2516_gb300 import build as ddbuild
    ddbuild.build()
    dd.load()


def _cands(n, seed, ndm=60, nt=5000, blobs=6):
    r = np.random.default_rng(seed)
    c = np.zeros(n, dtype=dd.CANDIDATE_DTYPE)
    centres = [(r.integers(0, ndm), r.integers(0, nt)) for _ in range(blobs)]
    for i in range(n):
        if i % 3 == 0:                                   # scattered points
            c[i]["dm_idx"], c[i]["t"] = r.integers(0, ndm), r.integers(0, nt)
        else:                                            # blobs
            d0, t0 = centres[i % blobs]
            c[i]["dm_idx"], c[i]["t"] = d0 + r.integers(-3, 4), t0 + r.integers(-20, 21)
        c[i]["width_idx"] = r.integers(0, 4)
        c[i]["snr"] = np.float32(6 + r.random() * 10)
    c["snr"][5] = c["snr"][7]                            # a tie
    return c


@pytest.mark.parametrize("dm_link,t_link", [(0, 0), (1, 4), (2, 10), (5, 100)])
def test_matches_all_pairs_oracle(dm_link, t_link):
    c = _cands(900, dm_link * 7 + t_link)
    clusters, labels = dd.dd_cluster_candidates(c, dm_link, t_link)
    ref = oracle.cluster(c, dm_link, t_link)
    assert len(clusters) == len(ref)
    for k, (best, members, (dlo, dhi), (tlo, thi)) in enumerate(ref):
        z = clusters[k]
        assert (int(z["dm_idx"]), int(z["t"]), int(z["width_idx"])) == \
               (int(c[best]["dm_idx"]), int(c[best]["t"]), int(c[best]["width_idx"]))
        assert z["snr"] == c[best]["snr"] and int(z["n_members"]) == len(members)
        assert (int(z["dm_lo"]), int(z["dm_hi"]), int(z["t_lo"]), int(z["t_hi"])) == (dlo, dhi, tlo, thi)
        assert sorted(np.nonzero(labels == k)[0].tolist()) == members


def test_invariants_and_edge_cases():
    c = _cands(400, 3)
    clusters, labels = dd.dd_cluster_candidates(c, 2, 15)
    assert clusters["n_members"].sum() == len(c)
    # members of different clusters are never friends
    for i in range(len(c)):
        for j in range(i + 1, len(c)):
            if labels[i] != labels[j]:
                assert not (abs(int(c[i]["dm_idx"]) - int(c[j]["dm_idx"])) <= 2 and abs(int(c[i]["t"]) - int(c[j]["t"])) <= 15)
    # empty input, one candidate, zero links = one cluster per distinct (dm, t)
    z, l = dd.dd_cluster_candidates(c[:0], 1, 1)
    assert len(z) == 0 and len(l) == 0
    z, l = dd.dd_cluster_candidates(c[:1], 1, 1)
    assert len(z) == 1 and int(z[0]["n_members"]) == 1
    z, _ = dd.dd_cluster_candidates(c, 0, 0)
    assert len(z) == len({(int(a["dm_idx"]), int(a["t"])) for a in c})
    with pytest.raises(dd.DDError):
        dd.dd_cluster_candidates(c, -1, 0)
