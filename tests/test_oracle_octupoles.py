"""Pins of the oracle's Mulliken octupoles (SI, "Multipolar Ewald", fourth definition) and of the
octupole error estimate of the multipole truncation (Sec. "Error Control"): quadrature, the
far-field expansion of the exact region-I energy, and a direct lattice sum of the third-order
region-II potential."""
import numpy as np
import pytest

import oracle
import workloads
from _quad import OPS3, ao_moments

A2B = 1.0 / 0.52917721092


@pytest.fixture(scope="module")
def sysm():
    return workloads.small_system(seed=23, n_atoms=3, lmax=2, nprim=(1, 2), n_waters=6)


def test_octupoles_against_quadrature(sysm):
    s = sysm
    O3 = ao_moments(s, oracle.norm_coeffs(s), OPS3)
    atom_of = np.repeat(s.shell_atom, [(l + 1) * (l + 2) // 2 for l in s.shell_l])
    ref = np.zeros((s.natm, 10))
    for mu in range(s.nao):
        for op in range(10):
            ref[atom_of[mu], op] -= np.dot(s.dm[:, mu], O3[op, mu, :])
    got = oracle.octupoles(s)
    assert np.max(np.abs(got - ref)) < 1e-11 * np.max(np.abs(ref))


def _exact_and_expansion(s, C, q=0.8):
    """Energy of one point charge q at C with the QM system (nuclei + electrons, no periodicity):
    exact (region-I integrals) and its multipole expansion about the atoms up to quadrupole and the
    octupole term alone."""
    chg = (np.asarray(C, dtype=np.float64)[None, :], np.array([q]), np.array([0.0]))
    V = oracle.vpot(s, charges=chg)
    exact = float(np.sum(s.dm * V)) + float(oracle.enucmm(s, charges=chg))
    M, Om = oracle.multipoles(s), oracle.octupoles(s)
    e2 = e3 = 0.0
    for j in range(s.natm):
        T = oracle.tensor(0, 0.0, s.atom_xyz[j] - C)
        e2 += q * np.sum(oracle.W10 * M[j] * T[:10])
        e3 += q * np.sum(oracle.MULT3 * Om[j] * T[10:20])
    return exact, e2, e3


@pytest.mark.parametrize("direction", [(1.0, 0.3, -0.2), (-0.4, 1.0, 0.7), (0.2, -0.5, -1.0)])
def test_octupole_term_is_the_leading_far_field_error(sysm, direction):
    # exact - (l <= 2 expansion) - (octupole term) = O(R^-5): r(R) R^5 tends to a constant.  A
    # wrong sign, index or weight in the octupole term leaves an R^-4 residual, for which
    # r(R) R^5 doubles with R.
    s = sysm
    u = np.asarray(direction) / np.linalg.norm(direction)
    c = s.atom_xyz.mean(0)
    scaled = {}
    for R in (60.0, 120.0):
        ex, e2, e3 = _exact_and_expansion(s, c + R * u)
        scaled[R] = (ex - e2 - e3) * R ** 5
    assert abs(scaled[120.0] / scaled[60.0] - 1.0) < 0.15


def test_octupole_energy_direct_lattice_sum():
    # third-order region-II potential of a neutral, dipole-free MM cell (octahedral units) against
    # the direct spherical lattice sum of q T_abc, contracted with random octupoles
    rng = np.random.default_rng(9)
    L = 10.0 * A2B
    qm = rng.uniform(-2, 2, (2, 3))
    Om = rng.normal(size=(2, 10))
    mm, q = [], []
    for _ in range(2):
        c = rng.uniform(0, L, 3)
        d = rng.uniform(1.0, 1.6)
        for a in range(3):
            for sgn in (1, -1):
                p = c.copy()
                p[a] += sgn * d
                mm.append(p)
                q.append(-0.25)
        mm.append(c)
        q.append(1.5)
    mm, q = np.array(mm), np.array(q)
    s = workloads.small_system(seed=1, n_atoms=2, lmax=0, n_waters=1)
    s.atom_xyz = qm
    s.mm_xyz, s.mm_q, s.mm_sigma = mm, q, np.zeros(len(q))
    s.box = np.full(3, L)
    s.ewald_alpha, s.kmax, s.ewald_rcut = 0.6, (22, 22, 22), 0.5 * L
    phi = oracle.ewald_phi(s, oracle.EW_SR | oracle.EW_LR | oracle.EW_BG)
    e_ewald = float(np.sum(oracle.MULT3 * Om * phi[:, 10:20]))

    def direct(N):
        tot = 0.0
        r = np.arange(-N, N + 1)
        ns = np.array([(a, b, c) for a in r for b in r for c in r if a * a + b * b + c * c <= N * N])
        for j in range(2):
            for n in ns:
                for i in range(len(q)):
                    T = oracle.tensor(0, 0.0, qm[j] - mm[i] - n * L)
                    tot += q[i] * np.sum(oracle.MULT3 * Om[j] * T[10:20])
        return tot

    # the direct sum converges onto the Ewald value (measured: 9.6e-8 at N = 6, 2.1e-8 at N = 8)
    d6, d8 = direct(6), direct(8)
    assert abs(d8 - e_ewald) < 5e-8 * abs(e_ewald)
    assert abs(d8 - e_ewald) < 0.5 * abs(d6 - e_ewald)


def test_octupole_error_depends_on_radius_through_region1_only(sysm):
    # growing region I moves charges from the region-II sum to the exact integrals: the estimate
    # changes by the octupole interaction of exactly those images (point tensors; the Gaussian
    # T-hat correction of region II vanishes for images farther than 9 sigma from every atom)
    s = sysm.copy()
    s.mm_sigma[:] = 0.0  # point charges: no T-hat term
    R1, R2 = 3.5 * A2B, 5.0 * A2B
    e1, e2 = oracle.octupole_error(s, [R1, R2])
    Om = oracle.octupoles(s)
    c = s.atom_xyz.mean(0)
    t = s.copy()
    t.cutoff = R2
    idx2, sh2 = oracle.region1(t)
    shell = 0.0
    for i, shv in zip(idx2, sh2):
        p = s.mm_xyz[i] + shv
        if np.linalg.norm(p - c) < R1:
            continue
        for j in range(s.natm):
            T = oracle.tensor(0, 0.0, s.atom_xyz[j] - p)
            shell += s.mm_q[i] * np.sum(oracle.MULT3 * Om[j] * T[10:20])
    assert abs((e1 - e2) - shell) < 1e-10 * max(abs(shell), abs(e1))
