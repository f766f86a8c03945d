"""Reciprocal sums on the tensor cores (QMMM_RECIP_TENSOR): the structure factor at the QM atoms
and the MM-side sum of the adjoint, as BF16 products of exact 7-bit digit planes with exact FP32
accumulation of the leading levels.  The region-II potential, energies and gradients against the
oracle, on shapes that exercise the tiling: ragged line tiles (128 lines), one and several blocks
of 512 charges, one and two N tiles of the structure factor (2 (2 kz + 1) > 80 rows), ragged
charge tiles of the MM-side sum, its N tiles of unequal size, and its fallback for short n_z rows."""
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
    # 1200 charges: three charge blocks, the last one ragged; 3 line tiles; 10 charge tiles of
    # the MM-side sum, the last one ragged
    "three_blocks": dict(seed=43, n_waters=400, box_A=24.0, kmax=(9, 9, 6)),
    # 2 (2 kz + 1) < 8: the MM-side sum stays on the CUDA cores (a chunk would span three n_y rows)
    "small_kz": dict(seed=44, n_waters=12, kmax=(5, 5, 3)),
    # MM-side N tiles of unequal size: FP64 path 96 + 48 rows (kx 20), mixed path 128 + 64 (kx 30)
    "uneven_ntiles_fp64": dict(seed=48, n_waters=12, kmax=(20, 6, 6)),
    "uneven_ntiles_mixed": dict(seed=49, n_waters=12, kmax=(30, 5, 5)),
}


def _system(name):
    kw = dict(CASES[name])
    return workloads.small_system(kw.pop("seed"), n_atoms=3, lmax=2, **kw)


def _tc(h):
    import paper_2408_03273_gb300 as q
    h.set_recip_method(q.QMMM_RECIP_TENSOR)


def _cuda_cores(h):
    import paper_2408_03273_gb300 as q
    h.set_recip_method(q.QMMM_RECIP_CUDA_CORES)


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
    a = gpu_all(s, precision=0, setup=_cuda_cores)["phi"]
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
        h.set_recip_method(q.QMMM_RECIP_TENSOR)
        p0 = h.potential()
        h.set_recip_method(q.QMMM_RECIP_CUDA_CORES)
        p2 = h.potential()
        assert not np.array_equal(p2, p0)
        assert rel_max(p2, p0) < 1e-12
        h.set_recip_method(q.QMMM_RECIP_TENSOR)
        assert np.array_equal(h.potential(), p0)
        h.set_recip_method(q.QMMM_RECIP_AUTO)  # small: the CUDA cores
        assert np.array_equal(h.potential(), p2)
        with pytest.raises(q.QMMMError):
            h.set_recip_method(7)
    finally:
        h.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_auto_picks_by_size(precision):
    # QMMM_RECIP_AUTO: the CUDA cores for a small reciprocal workload, the tensor cores from
    # 4e7 dense G entries x charges on
    import paper_2408_03273_gb300 as q
    small = _system("three_blocks")                                        # 1.5e6
    large = workloads.small_system(46, n_atoms=3, lmax=2, n_waters=400, box_A=24.0,
                                   kmax=(20, 20, 20))                      # 21 x 41 x 41 x 1194 = 4.2e7
    for s, method in ((small, q.QMMM_RECIP_CUDA_CORES), (large, q.QMMM_RECIP_TENSOR)):
        h = q.Handle(s, precision=precision)
        try:
            p_auto = h.potential()
            h.set_recip_method(method)
            assert np.array_equal(h.potential(), p_auto)
        finally:
            h.close()


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("precision,tol", [(0, 1e-11), (1, 1e-8)])
def test_tensor_core_mm_side_matches_cuda_cores(name, precision, tol):
    # the two methods differ only in the reciprocal sums: dE/dq and dE/dR_MM agree to well below
    # the parity tolerance, measured against the size of the reciprocal part alone.  FP64: seven
    # digit planes, five accumulators (levels 0..3 exact); mixed path: five planes (34-bit
    # operands), three accumulators (levels 2..4 merged in FP32)
    s = _system(name)
    dq_lr, dR_lr = oracle.ewald_mm(s, oracle.multipoles(s), oracle.EW_LR)
    # same precision on both sides (the mixed region-I sweeps differ from FP64 by far more)
    a = gpu_all(s, precision=precision, setup=_cuda_cores)
    b = gpu_all(s, precision=precision, setup=_tc)
    assert np.max(np.abs(a["dE_dq"] - b["dE_dq"])) < tol * np.max(np.abs(dq_lr))
    assert np.max(np.abs(a["dE_dRmm"] - b["dE_dRmm"])) < tol * np.max(np.abs(dR_lr))


def test_tensor_core_active_site_charge_derivatives():
    # the 60-atom active site in 59,463 charges (kmax 16: one N tile of 102 rows, 465 charge
    # tiles) in FP64 with both reciprocal sums on the tensor cores: sampled MM-charge derivatives
    # and the potential against the oracle
    s = workloads.config2_active_site()
    g = gpu_all(s, precision=0, setup=_tc)
    assert rel_max(g["phi"], oracle.ewald_phi(s)) < TOL_FP64
    idx = oracle.region1(s)[0]
    rng = np.random.default_rng(11)
    sub = np.sort(rng.choice(len(idx), 3, replace=False))
    mm = idx[sub]
    ref = oracle.forces(s, charge_subset=sub, mm_subset=mm)
    assert rel_max(g["dE_dq"][mm], ref["dE_dq"][mm]) < TOL_FP64
    assert rel_max(g["dE_dRmm"][mm], ref["dE_dRmm"][mm]) < TOL_FP64


@pytest.mark.parametrize("precision", [0, 1])
def test_tensor_cores_at_large_kmax(precision):
    # kmax 40: the structure factor reads its phase rows from global memory (the staging buffers
    # would not fit in shared memory) over three N tiles and 26 line tiles; the MM-side sum runs
    # one channel per N tile.  Against the CUDA-core kernels of the same precision.
    import paper_2408_03273_gb300 as q
    s = workloads.small_system(45, n_atoms=3, lmax=2, n_waters=12, kmax=(40, 40, 40))
    a = gpu_all(s, precision=precision, setup=_cuda_cores)
    b = gpu_all(s, precision=precision, setup=_tc)
    lr = oracle.ewald_phi(s, oracle.EW_LR)
    dq_lr, dR_lr = oracle.ewald_mm(s, oracle.multipoles(s), oracle.EW_LR)
    tol = 1e-11 if precision == 0 else 1e-8
    assert np.max(np.abs(a["phi"] - b["phi"])) < 1e-11 * np.max(np.abs(lr))
    assert np.max(np.abs(a["dE_dq"] - b["dE_dq"])) < tol * np.max(np.abs(dq_lr))
    assert np.max(np.abs(a["dE_dRmm"] - b["dE_dRmm"])) < tol * np.max(np.abs(dR_lr))
    assert q.QMMM_RECIP_TENSOR == 1


@pytest.mark.parametrize("precision", [0, 1])
def test_tensor_cores_with_three_charges(precision):
    # one water: a charge block of 512 that is almost all padding, one charge tile of 128 with 125
    # empty rows in the MM-side sum; everything against the oracle
    s = workloads.small_system(47, n_atoms=3, lmax=2, n_waters=1, kmax=(5, 5, 5))
    assert s.nmm == 3
    ref = oracle.energy(s)
    ref.update(oracle.forces(s))
    g = gpu_all(s, precision=precision, setup=_tc)
    assert rel_max(g["phi"], ref["phi"]) < TOL_FP64
    tol = TOL_FP64 if precision == 0 else TOL_MIXED
    for k in ("dE_dRqm", "dE_dRmm", "dE_dq"):
        assert grad_err(g[k], ref, k, precision == 1) < tol, k


def test_tensor_cores_with_empty_region1():
    # region I empty: every charge in region II, both tensor-core sums carry all of it
    s = workloads.small_system(seed=107, n_atoms=2, lmax=1, n_waters=6, cutoff_A=0.3)
    ref = oracle.energy(s)
    ref.update(oracle.forces(s))
    g = gpu_all(s, precision=0, setup=_tc)
    assert g["info"]["n_region1"] == 0
    assert abs(g["E"] - ref["E"]) < TOL_FP64 * energy_scale(ref)
    assert rel_max(g["dE_dRmm"], ref["dE_dRmm"]) < TOL_FP64
    assert rel_max(g["dE_dq"], ref["dE_dq"]) < TOL_FP64
