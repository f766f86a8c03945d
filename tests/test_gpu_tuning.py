"""Region-I sweep configurations: every wide block variant against the FP64 oracle, the
autotuner's configuration against the untuned run on the same system, and the tuning calls'
argument checks.  All calls go through the C ABI."""
import numpy as np
import pytest

import oracle
import workloads
from _gpuutil import TOL_FP64, TOL_MIXED, check_V, gpu_all, grad_err, rel_max

pytestmark = pytest.mark.gpu

KINDS = {0: (0, 2), 1: (1, 3)}  # precision -> (V sweep kind, adjoint sweep kind)


def _all_wide(precision):
    def setup(h):
        for k in KINDS[precision]:
            t = h.tuning(k)
            h.set_tuning(k, [w if w else 256 for w in t["wide"]])
            assert h.tuning(k)["threads"] == [w if w else 256 for w in t["wide"]]
    return setup


@pytest.fixture(scope="module")
def spdf():
    # every angular class up to (3,3), several tiles in the low classes
    s = workloads.small_system(seed=111, n_atoms=4, lmax=3, nprim=(1, 4), n_waters=14)
    ref = oracle.energy(s)
    ref.update(oracle.forces(s))
    return s, ref


@pytest.mark.parametrize("precision", [0, 1])
def test_wide_blocks_match_oracle(spdf, precision):
    s, ref = spdf
    g = gpu_all(s, precision=precision, screen_tol=0.0, setup=_all_wide(precision))
    tol = TOL_FP64 if precision == 0 else TOL_MIXED
    mixed = precision == 1
    check_V(g["V"], ref["V"], precision)
    for key in ("dE_dRqm", "dE_dRmm", "dE_dq"):
        assert grad_err(g[key], ref, key, mixed) < tol, key


@pytest.fixture(scope="module")
def medium():
    return workloads.small_system(seed=112, n_atoms=8, lmax=2, nprim=(1, 4), n_waters=60)


@pytest.mark.parametrize("precision", [0, 1])
def test_autotune_changes_only_the_schedule(medium, precision):
    import paper_2408_03273_gb300 as q
    plain = gpu_all(medium, precision=precision)
    seen = {}

    def tune(h):
        h.autotune(q.QMMM_TUNE_BOTH_PRECISIONS)
        for k in range(4):
            seen[k] = h.tuning(k)

    tuned = gpu_all(medium, precision=precision, setup=tune)
    nsm = None
    for k, t in seen.items():
        npp = tuned["info"]["n_prim_pairs_class"]
        for c in range(10):
            assert t["threads"][c] in (256, t["wide"][c]), (k, c)
            if npp[c] > 0:
                assert t["share"][c] >= 1, (k, c)
            else:
                assert t["share"][c] == 0, (k, c)
        if t["tuned"]:
            assert all(t["ms"][c] > 0 for c in range(10) if npp[c] > 0)
        nsm = sum(t["share"])
    assert nsm is not None
    # same arithmetic per primitive pair and charge; only the order of atomic additions may differ
    tol = 1e-13 if precision == 0 else 1e-7
    assert rel_max(tuned["V"], plain["V"]) < tol
    assert abs(tuned["E"] - plain["E"]) <= tol * abs(plain["E"])
    for key in ("dE_dRqm", "dE_dRmm", "dE_dq"):
        assert rel_max(tuned[key], plain[key]) < tol, key


def test_set_tuning_rejects_bad_configurations(medium):
    import paper_2408_03273_gb300 as q
    h = q.Handle(medium)
    try:
        with pytest.raises(q.QMMMError):
            h.set_tuning(0, [300] * 10)
        with pytest.raises(q.QMMMError):
            h.set_tuning(0, [256] * 10, [0.0] * 10)
        with pytest.raises(q.QMMMError):
            h.set_tuning(7, [256] * 10)
        t = h.tuning(0)
        assert not t["tuned"] and t["threads"] == [256] * 10
        h.set_tuning(2, [256] * 10, [1.0] * 10)  # equal weights: shares follow the pair counts
        assert h.tuning(2)["threads"] == [256] * 10
    finally:
        h.close()
