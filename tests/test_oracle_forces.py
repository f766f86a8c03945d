"""Pins of the oracle's gradient of E_QM-MM at fixed density (region-I integral derivatives,
tensor derivatives and the multipole Pulay term of Eq. 15) by finite differences of the oracle
energy, zero net force in a periodic cell and linearity in the MM charges."""
import numpy as np
import pytest

import oracle
import workloads

A2B = workloads.ANGSTROM_TO_BOHR


@pytest.fixture(scope="module")
def case():
    # converged Ewald parameters so that no pair sits on a visible real-space cutoff jump:
    # erfc(alpha rc) ~ 1e-14, exp(-G^2/4 alpha^2) ~ 1e-13 at the cube edge
    s = workloads.small_system(seed=77, n_atoms=3, lmax=2, nprim=(1, 2), n_waters=8, box_A=11.0,
                               cutoff_A=4.5, alpha_invA=1.0, kmax=(19, 19, 19))
    s.ewald_rcut = 5.4 * A2B
    g = oracle.forces(s)
    return s, g


def _E(s):
    return oracle.energy(s)["E"]


def _fd(s, setter, h):
    sp, sm = s.copy(), s.copy()
    setter(sp, +h)
    setter(sm, -h)
    r0 = oracle.region1(s)[0]
    if not (np.array_equal(oracle.region1(sp)[0], r0) and np.array_equal(oracle.region1(sm)[0], r0)):
        return None  # region-I membership changes: the energy is not differentiable there
    return (_E(sp) - _E(sm)) / (2 * h)


def test_qm_gradient_fd(case):
    s, g = case
    h = 1e-4
    scale = np.max(np.abs(g["dE_dRqm"]))
    for j in range(s.natm):
        for x in range(3):
            def setter(t, d, j=j, x=x):
                t.atom_xyz = t.atom_xyz.copy()
                t.atom_xyz[j, x] += d
            fd = _fd(s, setter, h)
            if fd is not None:
                assert abs(fd - g["dE_dRqm"][j, x]) < 2e-7 * scale


def test_mm_gradient_fd(case):
    s, g = case
    h = 1e-4
    scale = np.max(np.abs(g["dE_dRmm"]))
    for i in range(0, s.nmm, 2):
        for x in range(3):
            def setter(t, d, i=i, x=x):
                t.mm_xyz = t.mm_xyz.copy()
                t.mm_xyz[i, x] += d
            fd = _fd(s, setter, h)
            if fd is not None:
                assert abs(fd - g["dE_dRmm"][i, x]) < 2e-7 * scale


def test_charge_gradient_fd(case):
    s, g = case
    scale = np.max(np.abs(g["dE_dq"]))
    for i in range(0, s.nmm, 3):
        def setter(t, d, i=i):
            t.mm_q = t.mm_q.copy()
            t.mm_q[i] += d
        fd = _fd(s, setter, 1e-3)  # E is linear in q: FD is exact up to rounding
        assert abs(fd - g["dE_dq"][i]) < 1e-9 * scale


def test_zero_net_force(case):
    # a rigid translation of every particle leaves the periodic energy unchanged
    s, g = case
    tot = g["dE_dRqm"].sum(0) + g["dE_dRmm"].sum(0)
    assert np.max(np.abs(tot)) < 1e-11 * np.max(np.abs(g["dE_dRqm"]))


def test_charge_linearity(case):
    # E_QM-MM is linear and homogeneous in the MM charges: sum_i q_i dE/dq_i = E - E(q = 0)
    s, g = case
    e = oracle.energy(s)
    t = s.copy()
    t.mm_q = np.zeros_like(s.mm_q)
    e0 = oracle.energy(t)["E"]  # multipoles at q = 0 still carry no MM field: e0 == 0
    assert abs(e0) < 1e-14
    # E is a small residual of O(1) terms here, so the tolerance follows the size of the terms
    scale = abs(e["E_I_elec"]) + abs(e["E_nuc_mm"]) + abs(e["E_II"])
    assert abs(np.dot(s.mm_q, g["dE_dq"]) - e["E"]) < 1e-13 * scale
