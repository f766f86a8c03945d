"""Large active site with f shells (150 QM atoms, 1500 shells, 5100 AOs, ~200000 MM charges in an
86 A box, kmax 24): sampled V blocks of every angular class up to (f, f) against the oracle, the
charge derivatives of sampled region-I charges against the oracle (the full adjoint launch shape
of every class up to (f, f)), the mixed path against FP64, and invariants of the full gradient."""
import numpy as np
import pytest

import oracle
import workloads
from _gpuutil import TOL_FP64, TOL_MIXED, TOL_MIXED_ELEM, gpu_all, rel_fro, rel_max

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def c4():
    return workloads.config4_large_site()


@pytest.fixture(scope="module")
def c4_gpu(c4):
    return {p: gpu_all(c4, precision=p) for p in (0, 1)}


def test_config4_counts(c4, c4_gpu):
    info = c4_gpu[0]["info"]
    assert info["nao"] == 5100 and info["nshell"] == 1500
    assert info["n_region1"] == len(oracle.region1(c4)[0])
    assert info["n_gvec"] == (49 ** 3 - 1) // 2
    assert all(n > 0 for n in info["n_prim_pairs_class"])  # every class up to (f, f) is present


@pytest.mark.parametrize("precision", [0, 1])
def test_config4_sampled_V_blocks(c4, c4_gpu, precision):
    s = c4
    rng = np.random.default_rng(41)
    off = np.concatenate([[0], np.cumsum([(l + 1) * (l + 2) // 2 for l in s.shell_l])])
    pairs = []
    for la in range(4):
        for lb in range(la + 1):
            A = np.flatnonzero(s.shell_l == la)
            B = np.flatnonzero(s.shell_l == lb)
            for _ in range(3):
                pairs.append((int(rng.choice(A)), int(rng.choice(B))))
    V = c4_gpu[precision]["V"]
    Vref = oracle.vpot(s, pairs=pairs)
    got = np.concatenate([V[off[a]:off[a + 1], off[b]:off[b + 1]].ravel() for a, b in pairs])
    ref = np.concatenate([Vref[off[a]:off[a + 1], off[b]:off[b + 1]].ravel() for a, b in pairs])
    tol = TOL_FP64 if precision == 0 else TOL_MIXED_ELEM
    assert np.max(np.abs(got - ref)) < tol * np.max(np.abs(V))


def test_config4_sampled_charge_derivatives(c4, c4_gpu):
    # dE/dq and dE/dR_MM of two region-I charges: their region-I sums run over every primitive pair
    # of every class (the per-charge sums of the adjoint sweeps at full size) plus the nuclear and
    # MM-side Ewald terms; raw error relative to the largest value of each quantity
    rng = np.random.default_rng(44)
    nI = len(oracle.region1(c4)[0])
    sub = np.sort(rng.choice(nI, 2, replace=False))
    mm, dq, dR = oracle.forces_mm_subset(c4, sub)
    for p, tol in ((0, TOL_FP64), (1, TOL_MIXED)):
        g = c4_gpu[p]
        assert np.max(np.abs(g["dE_dq"][mm] - dq)) < tol * np.max(np.abs(g["dE_dq"])), p
        assert np.max(np.abs(g["dE_dRmm"][mm] - dR)) < tol * np.max(np.abs(g["dE_dRmm"])), p


def test_config4_mixed_vs_fp64(c4_gpu):
    assert rel_fro(c4_gpu[1]["V"], c4_gpu[0]["V"]) < TOL_MIXED
    for k in ("dE_dRqm", "dE_dRmm", "dE_dq"):
        assert rel_max(c4_gpu[1][k], c4_gpu[0][k]) < TOL_MIXED, k
    sc = abs(c4_gpu[0]["E_I_elec"]) + abs(c4_gpu[0]["E_nuc_mm"]) + abs(c4_gpu[0]["E_II"])
    assert abs(c4_gpu[1]["E"] - c4_gpu[0]["E"]) < TOL_MIXED * sc


def test_config4_invariants(c4, c4_gpu):
    for p in (0, 1):
        g = c4_gpu[p]
        tot = g["dE_dRqm"].sum(0) + g["dE_dRmm"].sum(0)
        assert np.max(np.abs(tot)) < (1e-9 if p == 0 else 1e-6) * np.max(np.abs(g["dE_dRqm"]))
        sc = abs(g["E_I_elec"]) + abs(g["E_nuc_mm"]) + abs(g["E_II"])
        assert abs(np.dot(c4.mm_q, g["dE_dq"]) - g["E"]) < (1e-11 if p == 0 else 1e-6) * sc


def test_config4_tensor_core_sums_match_cuda_cores(c4, c4_gpu):
    # kmax 24 takes the tiled shapes of both tensor-core sums (two N tiles of the structure factor,
    # three of the FP64-class MM-side sum): against the FP64 CUDA-core kernels, which the smaller
    # workloads pin to the oracle, relative to the largest value of each quantity
    import paper_2408_03273_gb300 as q
    cc = gpu_all(c4, precision=0, setup=lambda h: h.set_recip_method(q.QMMM_RECIP_CUDA_CORES))
    tc = c4_gpu[0]
    assert rel_max(tc["phi"], cc["phi"]) < 1e-11
    assert rel_max(tc["dE_dq"], cc["dE_dq"]) < 1e-11
    assert rel_max(tc["dE_dRmm"], cc["dE_dRmm"]) < 1e-10
    assert abs(tc["E"] - cc["E"]) < 1e-11 * (abs(cc["E_I_elec"]) + abs(cc["E_nuc_mm"]) + abs(cc["E_II"]))
