"""Structure factor on the tensor cores (QMMM_RECIP_TENSOR): BF16 products of exact 6-bit digit
planes with exact FP32 accumulation of the leading levels.  The region-II potential and everything
downstream against the oracle, on shapes that exercise the tiling: ragged line tiles (128 lines),
one and several blocks of 512 charges, one and two N tiles (2 (2 kz + 1) > 80 rows)."""
import numpy as np
import pytest

import oracle
import workloads
from _gpuutil import TOL_FP64, TOL_MIXED, energy_scale, gpu_all, grad_err, rel_max

pytestmark = pytest.mark.gpu

CASES = {
    # 36 charges, 66 lines, 22 rows
    "tiny": dict(seed=41, n_waters=12, kmax=(5, 5, 5)),
    # two N tiles (86 rows)
    "two_ntiles": dict(seed=42, n_waters=12, kmax=(4, 4, 21)),
    # 1200 charges: three charge blocks, the last one ragged; 3 line tiles
    "three_blocks": dict(seed=43, n_waters=400, box_A=24.0, kmax=(9, 9, 6)),
}


def _system(name):
    kw = dict(CASES[name])
    return workloads.small_system(kw.pop("seed"), n_atoms=3, lmax=2, **kw)


def _tc(h):
    import paper_2408_03273_gb300 as q
    h.set_recip_method(q.QMMM_RECIP_TENSOR)


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("precision", [0, 1])
def test_tensor_core_structure_factor_against_oracle(name, precision):
    s = _system(name)
    ref = oracle.energy(s)
    ref.update(oracle.forces(s))
    g = gpu_all(s, precision=precision, setup=_tc)
    assert rel_max(g["phi"], ref["phi"]) < TOL_FP64
    tol = TOL_FP64 if precision == 0 else TOL_MIXED
    sc = energy_scale(ref)
    assert abs(g["E_II"] - ref["E_II"]) < TOL_FP64 * sc
    assert abs(g["E"] - ref["E"]) < tol * sc
    for k in ("dE_dRqm", "dE_dRmm", "dE_dq"):
        assert grad_err(g[k], ref, k, precision == 1) < tol, k


@pytest.mark.parametrize("name", list(CASES))
def test_tensor_core_matches_cuda_core_reciprocal_part(name):
    # the two methods differ only in the structure factor: their potentials agree to well below
    # the parity tolerance, measured against the size of the reciprocal part alone
    s = _system(name)
    lr = oracle.ewald_phi(s, oracle.EW_LR)
    a = gpu_all(s, precision=0)["phi"]
    b = gpu_all(s, precision=0, setup=_tc)["phi"]
    assert np.max(np.abs(a - b)) < 1e-11 * np.max(np.abs(lr))


def test_tensor_core_water_workload():
    s = workloads.config1_water()
    ref = oracle.energy(s)
    g = gpu_all(s, precision=0, setup=_tc)
    assert rel_max(g["phi"], ref["phi"]) < TOL_FP64
    assert abs(g["E"] - ref["E"]) < TOL_FP64 * energy_scale(ref)


def test_switching_methods_recomputes_potential():
    import paper_2408_03273_gb300 as q
    s = _system("three_blocks")
    h = q.Handle(s)
    try:
        p0 = h.potential()
        h.set_recip_method(q.QMMM_RECIP_TENSOR)
        p1 = h.potential()
        h.set_recip_method(q.QMMM_RECIP_CUDA_CORES)
        p2 = h.potential()
        assert np.array_equal(p0, p2)
        assert rel_max(p1, p0) < 1e-12
        with pytest.raises(q.QMMMError):
            h.set_recip_method(7)
    finally:
        h.close()


def test_auto_selects_tensor_cores_for_the_mixed_path():
    import paper_2408_03273_gb300 as q
    s = _system("three_blocks")
    h = q.Handle(s, precision=q.QMMM_MIXED)  # QMMM_RECIP_AUTO
    try:
        p_auto = h.potential()
        h.set_recip_method(q.QMMM_RECIP_TENSOR)
        assert np.array_equal(h.potential(), p_auto)
        h.set_recip_method(q.QMMM_RECIP_CUDA_CORES)  # double-float on the CUDA cores
        p_df = h.potential()
        assert not np.array_equal(p_df, p_auto)
        assert rel_max(p_df, p_auto) < 1e-11
    finally:
        h.close()
