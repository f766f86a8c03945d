"""Pins of the oracle's multipolar Ewald potential at the QM sites (SI, "Multipolar Ewald";
Eq. 6 QM-MM lines; Eq. 10) by alpha-invariance, a direct lattice sum of a neutral cell, lattice
shifts and the Gaussian-charge correction."""
import math

import numpy as np
import pytest

import oracle
import workloads

A2B = workloads.ANGSTROM_TO_BOHR
FULL = oracle.EW_SR | oracle.EW_LR | oracle.EW_BG


def _cell(seed, charged=False):
    s = workloads.small_system(seed=seed, n_atoms=3, lmax=0, n_waters=10, box_A=12.0, cutoff_A=5.0)
    if charged:
        s.mm_q = s.mm_q.copy()
        s.mm_q[0] += 0.3  # net MM charge: exercises the neutralising background
    return s


def _phi(s, alpha_invA, kmax, rc_A=5.9, mode=FULL):
    t = s.copy()
    t.ewald_alpha = alpha_invA / A2B
    t.kmax = (kmax, kmax, kmax)
    t.ewald_rcut = rc_A * A2B
    return oracle.ewald_phi(t, mode)


@pytest.mark.parametrize("charged", [False, True])
def test_alpha_invariance(charged):
    # erfc(alpha rc) < 1e-14 and exp(-G^2/4alpha^2) < 1e-14 at the cube edge for every alpha
    s = _cell(31, charged)
    ref = _phi(s, 1.0, 30)
    scale = np.abs(ref).max(axis=0)
    for a in (1.1, 1.2):
        got = _phi(s, a, 30)
        assert np.max(np.abs(got - ref) / scale) < 1e-10


def test_alpha_invariance_needs_background():
    # with a net MM charge the monopole potential depends on alpha unless -pi/(V kappa^2) q_tot is added
    s = _cell(31, True)
    mode = oracle.EW_SR | oracle.EW_LR
    a = _phi(s, 1.0, 30, mode=mode)[:, 0]
    b = _phi(s, 1.2, 30, mode=mode)[:, 0]
    assert np.max(np.abs(a - b)) > 1e-4 * np.max(np.abs(a))


def _octahedral_units(rng, n, box, d=0.8 * A2B, q=0.3):
    pos, chg = [], []
    for _ in range(n):
        c = rng.uniform(-box / 2, box / 2, 3)
        pos.append(c)
        chg.append(-6 * q)
        for ax in range(3):
            for sg in (1, -1):
                e = np.zeros(3)
                e[ax] = sg * d
                pos.append(c + e)
                chg.append(q)
    return np.array(pos), np.array(chg)


def test_direct_lattice_sum_neutral_cell():
    # QM multipoles with zero total charge and dipole; MM made of octahedral units (neutral,
    # dipole-free, isotropic second moment).  The direct spherical lattice sum then converges
    # absolutely to the tin-foil Ewald value (the Bethe constant multiplies sum Q = 0).
    rng = np.random.default_rng(5)
    L = 10.0 * A2B
    qm = rng.uniform(-2, 2, (3, 3))
    M = rng.normal(size=(3, 10))
    M[:, 0] -= M[:, 0].mean()
    M[:, 1:4] -= (M[:, 0:1] * qm + M[:, 1:4]).sum(0) / 3.0  # total dipole zero
    mm, q = _octahedral_units(rng, 2, L)
    s = workloads.small_system(seed=1, n_atoms=3, lmax=0, n_waters=1)
    s.atom_xyz = qm
    s.mm_xyz, s.mm_q, s.mm_sigma = mm, q, np.zeros(len(q))
    s.box = np.full(3, L)
    s.ewald_alpha, s.kmax, s.ewald_rcut = 0.6, (22, 22, 22), 0.5 * L
    e_ewald = oracle.multipole_energy(M, oracle.ewald_phi(s, FULL))

    def direct(N):
        tot = 0.0
        r = np.arange(-N, N + 1)
        ns = np.array([(a, b, c) for a in r for b in r for c in r if a * a + b * b + c * c <= N * N])
        for j in range(3):
            for n in ns:
                for i in range(len(q)):
                    T = oracle.tensor(0, 0.0, qm[j] - mm[i] - n * L)
                    tot += q[i] * np.sum(oracle.W10 * M[j] * T[:10])
        return tot

    d4, d8 = direct(4), direct(8)
    # the direct sum converges onto the Ewald value (measured: 2.6e-8 at N = 4, 3e-10 at N = 8)
    assert abs(d4 - e_ewald) < 1e-7 * abs(e_ewald)
    assert abs(d8 - e_ewald) < 1e-9 * abs(e_ewald)


def test_lattice_shift_invariance():
    s = workloads.small_system(seed=44, n_atoms=3, lmax=0, n_waters=10, box_A=12.0, cutoff_A=5.0)
    p0 = oracle.ewald_phi(s)
    t = s.copy()
    t.mm_xyz[3:6] += s.box * np.array([-1, 0, 1])
    p1 = oracle.ewald_phi(t)
    assert np.max(np.abs(p1 - p0) / (np.abs(p0).max(axis=0) + 1e-300)) < 1e-11


def test_gaussian_charge_correction_region2():
    # A Gaussian charge in region II close to a QM atom interacts as erf(r/sigma)/r:
    # phi_0(sigma) - phi_0(point) = -q erfc(r/sigma)/r for that atom.
    s = workloads.small_system(seed=2, n_atoms=1, lmax=0, n_waters=1, box_A=14.0, cutoff_A=1.0)
    s.atom_xyz = np.array([[0.0, 0.0, 0.0], [6.0, 0.0, 0.0]])
    s.atom_Z = np.array([1.0, 1.0])
    s.shell_atom = np.array([0, 1], dtype=np.int32)
    s.shell_l = np.array([0, 0], dtype=np.int32)
    s.shell_nprim = np.array([1, 1], dtype=np.int32)
    s.shell_prim_offset = np.array([0, 1], dtype=np.int32)
    s.prim_exp, s.prim_coeff = np.array([1.0, 1.0]), np.array([1.0, 1.0])
    sigma = 0.6
    s.mm_xyz = np.array([[6.5, 0.4, 0.0]])  # 0.64 bohr from atom 1, 3.5 bohr from the centre
    s.mm_q, s.mm_sigma = np.array([0.7]), np.array([sigma])
    s.cutoff = 2.0
    g = oracle.ewald_phi(s)
    t = s.copy()
    t.mm_sigma = np.array([0.0])
    p = oracle.ewald_phi(t)
    r = math.hypot(0.5, 0.4)
    assert abs((g[1, 0] - p[1, 0]) - (-0.7 * math.erfc(r / sigma) / r)) < 1e-13
    assert abs(g[0, 0] - p[0, 0]) < 1e-13  # far atom: erfc(6/0.6) is negligible
