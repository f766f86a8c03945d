"""GPU path against the FP64 oracle, element by element, on small seeded systems that still
span several warp tiles and a ragged tail (every angular class l <= 3, Gaussian and point
charges, region-I chunks, screening on and off).  All calls go through the C ABI."""
import numpy as np
import pytest

import oracle
import workloads
from _gpuutil import TOL_FP64, TOL_MIXED, check_V, energy_scale, gpu_all, grad_err, rel_fro, rel_max

pytestmark = pytest.mark.gpu

CASES = {
    # name: small_system kwargs
    "sp_gauss": dict(seed=101, n_atoms=3, lmax=1, nprim=(1, 3), n_waters=10),
    "spd_gauss": dict(seed=102, n_atoms=4, lmax=2, nprim=(1, 4), n_waters=14),
    "spdf_gauss": dict(seed=103, n_atoms=3, lmax=3, nprim=(1, 3), n_waters=8),
    "spd_point": dict(seed=104, n_atoms=3, lmax=2, nprim=(2, 3), n_waters=9, point_charges=True),
    "many_prims": dict(seed=105, n_atoms=2, lmax=2, nprim=(5, 7), n_waters=6),  # > 32 pp per shell pair
}


@pytest.fixture(scope="module", params=list(CASES))
def case(request):
    s = workloads.small_system(**CASES[request.param])
    ref = oracle.energy(s)
    ref.update(oracle.forces(s))
    return request.param, s, ref


@pytest.mark.parametrize("precision", [0, 1])
def test_vpot(case, precision):
    name, s, ref = case
    g = gpu_all(s, precision=precision, screen_tol=0.0)
    check_V(g["V"], ref["V"], precision)
    assert np.array_equal(g["V"], g["V"].T), "V must be exactly symmetric"
    assert abs(g["E_nuc_mm"] - ref["E_nuc_mm"]) < TOL_FP64 * abs(ref["E_nuc_mm"]) + 1e-14


@pytest.mark.parametrize("precision", [0, 1])
def test_energy_and_multipoles(case, precision):
    name, s, ref = case
    g = gpu_all(s, precision=precision, screen_tol=0.0)
    tol = TOL_FP64 if precision == 0 else TOL_MIXED
    sc = energy_scale(ref)
    assert abs(g["E_I_elec"] - ref["E_I_elec"]) < tol * sc
    assert abs(g["E_II"] - ref["E_II"]) < TOL_FP64 * sc   # Ewald part is FP64 on both paths
    assert abs(g["E"] - ref["E"]) < tol * sc
    assert rel_max(g["M"], ref["M"]) < TOL_FP64
    assert rel_max(g["phi"], ref["phi"]) < TOL_FP64


def test_fock_term(case):
    name, s, ref = case
    g = gpu_all(s, precision=0, screen_tol=0.0)
    F = oracle.fock_ii(s, ref["phi"])
    assert rel_max(g["F"], F) < TOL_FP64


def test_density_gradient(case):
    # dE/dgamma = V + F_II (Eqs. 11-14) formed by the library, against the oracle's V and F_II
    import paper_2408_03273_gb300 as q
    name, s, ref = case
    h = q.Handle(s, screen_tol=0.0)
    try:
        with pytest.raises(q.QMMMError):
            h.density_gradient(s.dm)  # V not computed yet at this geometry
        h.vpot()
        G = h.density_gradient(s.dm)
    finally:
        h.close()
    assert rel_max(G, ref["V"] + oracle.fock_ii(s, ref["phi"])) < TOL_FP64


@pytest.mark.parametrize("precision", [0, 1])
def test_forces(case, precision):
    name, s, ref = case
    g = gpu_all(s, precision=precision, screen_tol=0.0)
    tol = TOL_FP64 if precision == 0 else TOL_MIXED
    for k in ("dE_dRqm", "dE_dRmm", "dE_dq"):
        assert grad_err(g[k], ref, k, precision == 1) < tol, (name, k)


def test_screening_default_changes_nothing_visible(case):
    # the default primitive-pair screening (1e-14 relative) stays within FP64 parity
    name, s, ref = case
    g = gpu_all(s, precision=0)
    assert rel_max(g["V"], ref["V"]) < TOL_FP64
    assert rel_max(g["dE_dRqm"], ref["dE_dRqm"]) < TOL_FP64


def test_repeat_is_bitwise_identical():
    # V (at most two additions per element) and the region-II potential (fixed-order sums) are
    # reproducible bit for bit; the multipoles are summed with atomics over shell pairs, so E may
    # differ in the last bits
    s = workloads.small_system(seed=106, n_atoms=3, lmax=2, nprim=(1, 3), n_waters=12)
    a, b = gpu_all(s), gpu_all(s)
    assert np.array_equal(a["V"], b["V"])
    assert np.array_equal(a["phi"], b["phi"])
    assert abs(a["E"] - b["E"]) <= 1e-14 * abs(a["E"])


def test_region1_empty():
    # cutoff smaller than any QM-MM separation: region I holds nothing, V = 0, everything is region II
    s = workloads.small_system(seed=107, n_atoms=2, lmax=1, n_waters=6, cutoff_A=0.3)
    assert len(oracle.region1(s)[0]) == 0
    ref = oracle.energy(s)
    ref.update(oracle.forces(s))
    g = gpu_all(s)
    assert g["info"]["n_region1"] == 0
    assert np.max(np.abs(g["V"])) == 0.0
    assert abs(g["E"] - ref["E"]) < TOL_FP64 * energy_scale(ref)
    assert rel_max(g["dE_dRmm"], ref["dE_dRmm"]) < TOL_FP64


def test_region1_spans_several_chunks():
    # a dense box and a wide cutoff put more charges in region I than one shared-memory chunk holds
    s = workloads.small_system(seed=108, n_atoms=2, lmax=1, nprim=(1, 2), n_waters=5400, box_A=40.0,
                               cutoff_A=19.5, alpha_invA=0.3, kmax=(6, 6, 6))
    nI = len(oracle.region1(s)[0])
    assert nI > 4096 + 2560
    ref_V = oracle.vpot(s)
    g = gpu_all(s, screen_tol=0.0)
    assert g["info"]["n_region1"] == nI
    assert rel_max(g["V"], ref_V) < TOL_FP64
    # the region-I adjoint also runs in several chunks: check the charge derivatives of a sample
    sub = np.arange(0, nI, 97)
    ref = oracle.forces(s, charge_subset=sub)
    idx = oracle.region1(s)[0][sub]
    # images map one-to-one onto MM charges here (box > 2 cutoff), so the sampled charges' dq is complete
    assert len(set(idx)) == len(idx)
    assert rel_max(g["dE_dq"][idx], ref["dE_dq"][idx]) < TOL_FP64
    assert rel_max(g["dE_dRmm"][idx], ref["dE_dRmm"][idx]) < TOL_FP64


def test_small_box_multiple_images():
    # box smaller than twice the cutoffs: several images of a charge in region I and in the
    # Ewald real-space sum
    s = workloads.small_system(seed=109, n_atoms=2, lmax=1, n_waters=8, box_A=9.0, cutoff_A=8.0, alpha_invA=0.5)
    s.ewald_rcut = 7.0 * workloads.ANGSTROM_TO_BOHR
    idx, _ = oracle.region1(s)
    assert len(idx) > len(set(idx))
    ref = oracle.energy(s)
    ref.update(oracle.forces(s))
    g = gpu_all(s, screen_tol=0.0)
    assert rel_max(g["V"], ref["V"]) < TOL_FP64
    assert rel_max(g["phi"], ref["phi"]) < TOL_FP64
    assert rel_max(g["dE_dRmm"], ref["dE_dRmm"]) < TOL_FP64
    assert rel_max(g["dE_dq"], ref["dE_dq"]) < TOL_FP64


def test_no_mm_charges():
    s = workloads.small_system(seed=110, n_atoms=2, lmax=1, n_waters=1)
    s.mm_xyz, s.mm_q, s.mm_sigma = np.zeros((0, 3)), np.zeros(0), np.zeros(0)
    g = gpu_all(s)
    assert np.max(np.abs(g["V"])) == 0.0
    assert g["E"] == 0.0
    assert np.max(np.abs(g["dE_dRqm"])) == 0.0


def test_mixed_region2_potential_keeps_double_float_accuracy(case):
    # the mixed path computes the reciprocal Ewald sums in double-float arithmetic (~47 bits):
    # its region-II potential stays within 1e-12 of the FP64 oracle, far inside the 1e-6 budget
    name, s, ref = case
    g = gpu_all(s, precision=1)
    phi = oracle.ewald_phi(s)
    assert rel_max(g["phi"], phi) < 1e-12, name
