"""Pins of the oracle's QM-QM periodic-image multipole energy (Eq. 5 in the Ewald form of Eq. 6)
and of its potentials and gradient.

Readings fixed here (each pinned below, not by retyping the formula):
  * the pair energy over ordered pairs carries 2 mu_j Q_i P_a and 2 theta_j Q_i P_ab next to
    Q_j Q_i P (Eq. 5 prints weight 1): only then does 1/2 sum_{j,i} count each dipole-charge and
    quadrupole-charge interaction once -- pinned against the lattice energy of point-charge
    clusters with those moments;
  * the dipole-dipole term is -2 mu_j mu_i P_ab (Eq. 5 prints +2), the physical sign -- same pin;
  * self terms -2 kappa/sqrt(pi) and +(2/3) kappa^3/sqrt(pi) delta_ab (the SI prints -kappa/sqrt(pi)
    and -(2/3) kappa^3/sqrt(pi)) -- pinned by alpha-invariance;
  * a neutralising background -pi/(2 V kappa^2) (sum Q)^2 for a charged QM cell -- alpha-invariance."""
import math

import numpy as np
import pytest
from scipy.special import erfc

import oracle
import workloads

CONV = dict(alpha=0.8, kmax=(22, 22, 22), ewald_rcut=7.5)  # erfc(6) ~ 2e-17, exp(-G^2/4a^2) < 1e-14


def _cell(seed, natm=3, L=15.0, charged=True):
    s = workloads.small_system(seed=seed, n_atoms=natm, lmax=0, n_waters=1)
    rng = np.random.default_rng(seed)
    s.atom_xyz = rng.uniform(0.0, L, (natm, 3))
    s.box = np.full(3, L)
    M = rng.normal(scale=0.3, size=(natm, 10))
    M[:, 0] = rng.normal(size=natm)
    if not charged:
        M[:, 0] -= M[:, 0].mean()
    return s, M


@pytest.mark.parametrize("charged", [False, True])
def test_alpha_invariance(charged):
    s, M = _cell(41, charged=charged)
    E0, u0, g0 = oracle.qmqm(s, M, **CONV)
    for a in (0.9, 1.0):
        E, u, g = oracle.qmqm(s, M, alpha=a, kmax=(26, 26, 26), ewald_rcut=7.5)
        assert abs(E - E0) < 1e-11 * abs(E0)
        assert np.max(np.abs(u - u0)) < 1e-10 * np.max(np.abs(u0))
        assert np.max(np.abs(g - g0)) < 1e-10 * np.max(np.abs(g0))


def _pair_energy_point(M, j, i, d):
    """Pair energy with bare point tensors (for the direct lattice sum)."""
    T = oracle.tensor(0, 0.0, d)
    P2 = [(0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2)]
    Pab = np.zeros((3, 3))
    th = np.zeros((3, 3))
    for k, (a, b) in enumerate(P2):
        Pab[a, b] = Pab[b, a] = T[4 + k]
        th[a, b] = th[b, a] = M[j, 4 + k]
    e = M[j, 0] * M[i, 0] * T[0] + 2.0 * M[i, 0] * np.dot(M[j, 1:4], T[1:4])
    e += 2.0 * M[i, 0] * np.sum(th * Pab) - 2.0 * M[j, 1:4] @ Pab @ M[i, 1:4]
    return e


def test_direct_lattice_sum_neutral_dipole_free():
    # zero total charge and dipole: the spherical direct sum over L != 0 converges absolutely to the
    # tin-foil Ewald value
    s, M = _cell(43, natm=3, charged=False)
    M[:, 1:4] -= (M[:, 0:1] * s.atom_xyz + M[:, 1:4]).sum(0) / 3.0
    E_ew, _, _ = oracle.qmqm(s, M, **CONV)
    L = s.box[0]

    def direct(N):
        r = np.arange(-N, N + 1)
        ns = [np.array(n) for n in ((a, b, c) for a in r for b in r for c in r)
              if 0 < n[0] * n[0] + n[1] * n[1] + n[2] * n[2] <= N * N]
        tot = 0.0
        for j in range(s.natm):
            for i in range(s.natm):
                for n in ns:
                    tot += 0.5 * _pair_energy_point(M, j, i, s.atom_xyz[j] - s.atom_xyz[i] + n * L)
        return tot

    # measured: 6.5e-5 (N = 8), 1.7e-5 (N = 12) relative, shrinking towards the Ewald value
    d8, d12 = direct(8), direct(12)
    assert abs(d12 - E_ew) < 0.5 * abs(d8 - E_ew)
    assert abs(d12 - E_ew) < 3e-5 * abs(E_ew)


def _point_ewald(pos, q, L, kappa=0.8, kmax=22, rc=7.5):
    """Ewald energy of point charges in a cubic box (tin foil, neutralising background), written
    out from the textbook split: erfc real space, reciprocal sum, self and background terms."""
    n = len(q)
    V = L ** 3
    E = 0.0
    m = int(math.ceil(rc / L)) + 1
    shifts = np.array([(a, b, c) for a in range(-m, m + 1) for b in range(-m, m + 1) for c in range(-m, m + 1)]) * L
    for a in range(n):
        d = pos[a] - pos + shifts[:, None, :]  # (images, n, 3)
        r = np.linalg.norm(d, axis=2)
        mask = (r < rc) & (r > 0)
        E += 0.5 * q[a] * np.sum((q[None, :] * erfc(kappa * r) / np.where(mask, r, 1.0))[mask])
    k = np.arange(-kmax, kmax + 1)
    G = 2 * np.pi / L * np.array(np.meshgrid(k, k, k, indexing="ij")).reshape(3, -1).T
    G = G[np.any(G != 0, axis=1)]
    G2 = np.sum(G * G, axis=1)
    S = np.exp(1j * (G @ pos.T)) @ q
    E += 2 * np.pi / V * np.sum(np.exp(-G2 / (4 * kappa ** 2)) / G2 * np.abs(S) ** 2)
    E += -kappa / np.sqrt(np.pi) * np.sum(q * q) - np.pi / (2 * V * kappa ** 2) * np.sum(q) ** 2
    return E


def _cluster_energy_II(centres, charges, offsets, L):
    """Periodic-image energy of charge clusters: all-lattice Ewald energy minus every L = 0 pair
    (the reference cell is the QM calculation's, each cluster's own structure is internal)."""
    pos = np.concatenate([c + o for c, o in zip(centres, offsets)])
    q = np.concatenate(charges)
    E = _point_ewald(pos, q, L)
    for a in range(len(q)):
        for b in range(a + 1, len(q)):
            E -= q[a] * q[b] / np.linalg.norm(pos[a] - pos[b])
    return E


def _moments(charges, offsets):
    M = np.zeros(10)
    M[0] = np.sum(charges)
    M[1:4] = charges @ offsets
    for k, (a, b) in enumerate([(0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2)]):
        M[4 + k] = np.sum(charges * offsets[:, a] * offsets[:, b])
    return M


def test_dipole_charge_and_dipole_dipole_weights_from_point_clusters():
    # sites made of two point charges (charge + dipole; their second moment is O(delta) and kept):
    # the cluster lattice energy equals the multipole formula up to third-order terms
    rng = np.random.default_rng(47)
    L, delta = 15.0, 0.01
    centres = rng.uniform(0, L, (3, 3))
    charges, offsets = [], []
    for Q, mu in ((1.0, 0.25), (-0.6, 0.2), (0.3, 0.3)):
        n = rng.normal(size=3)
        n /= np.linalg.norm(n)
        qp = 0.5 * Q + mu / delta
        charges.append(np.array([qp, Q - qp]))
        offsets.append(np.array([0.5 * delta * n, -0.5 * delta * n]))
    E_cl = _cluster_energy_II(centres, charges, offsets, L)
    s, _ = _cell(1, natm=3, L=L)
    s.atom_xyz = centres
    M = np.array([_moments(c, o) for c, o in zip(charges, offsets)])
    E, _, _ = oracle.qmqm(s, M, **CONV)
    # the energy is bilinear: split it into its charge-charge, dipole-dipole, quadrupole-charge and
    # dipole-charge parts by switching multipoles off
    def part(keep):
        Mk = M * keep
        return oracle.qmqm(s, Mk, **CONV)[0]
    E_qq = part(np.r_[1, 0, 0, 0, np.zeros(6)])
    E_mm = part(np.r_[0, 1, 1, 1, np.zeros(6)])
    E_tq = part(np.r_[1, 0, 0, 0, np.ones(6)]) - E_qq
    E_mq = E - E_qq - E_mm - E_tq
    assert abs(E_cl - E) < 0.01 * min(abs(E_mm), abs(E_mq))
    # the weights as printed in Eq. 5 (dipole-charge 1, dipole-dipole +2) miss the cluster energy
    E_printed = E_qq + 0.5 * E_mq + 0.5 * E_tq - E_mm
    assert abs(E_cl - E_printed) > 0.2 * min(abs(E_mm), abs(E_mq))


def test_quadrupole_charge_weight_from_point_clusters():
    # one site with a quadrupole (three collinear charges plus a net charge), two point charges
    rng = np.random.default_rng(53)
    L, delta, th = 15.0, 0.01, 0.05
    centres = rng.uniform(0, L, (3, 3))
    qq = th / (2 * delta * delta)
    charges = [np.array([qq, qq, -2 * qq + 0.4]), np.array([-0.7]), np.array([0.9])]
    offsets = [np.array([[delta, 0, 0], [-delta, 0, 0], [0, 0, 0]]), np.zeros((1, 3)), np.zeros((1, 3))]
    E_cl = _cluster_energy_II(centres, charges, offsets, L)
    s, _ = _cell(1, natm=3, L=L)
    s.atom_xyz = centres
    M = np.array([_moments(c, o) for c, o in zip(charges, offsets)])
    E, _, _ = oracle.qmqm(s, M, **CONV)
    Mq = M.copy()
    Mq[:, 4:] = 0.0
    E_noquad, _, _ = oracle.qmqm(s, Mq, **CONV)
    theta_term = E - E_noquad
    assert abs(theta_term) > 1e-6
    assert abs(E_cl - E) < 0.01 * abs(theta_term)


def test_gradient_and_potentials_by_finite_differences():
    s, M = _cell(59, natm=3, charged=True)
    E0, u, g = oracle.qmqm(s, M, **CONV)
    h = 1e-4
    for j in range(s.natm):
        for x in range(3):
            t = s.copy()
            t.atom_xyz = s.atom_xyz.copy()
            t.atom_xyz[j, x] += h
            Ep, _, _ = oracle.qmqm(t, M, **CONV)
            t.atom_xyz[j, x] -= 2 * h
            Em, _, _ = oracle.qmqm(t, M, **CONV)
            assert abs((Ep - Em) / (2 * h) - g[j, x]) < 1e-7 * np.max(np.abs(g))
    for j in range(s.natm):
        for c in range(10):
            Mp, Mm = M.copy(), M.copy()
            Mp[j, c] += h
            Mm[j, c] -= h
            dE = (oracle.qmqm(s, Mp, **CONV)[0] - oracle.qmqm(s, Mm, **CONV)[0]) / (2 * h)
            assert abs(dE - oracle.W10[c] * u[j, c]) < 1e-7 * np.max(np.abs(u))


@pytest.fixture(scope="module")
def qsys():
    s = workloads.small_system(seed=61, n_atoms=3, lmax=2, nprim=(1, 2), n_waters=2, box_A=7.0)
    return s


QCONV = dict(alpha=1.4, kmax=(18, 18, 18), ewald_rcut=6.5)


def test_qm_images_gradient_by_finite_differences(qsys):
    # full gradient at fixed density: image tensors plus the multipoles' basis-position dependence
    s = qsys
    ref = oracle.qm_images(s, **QCONV)
    h = 1e-4
    for j in range(s.natm):
        for x in range(3):
            t = s.copy()
            t.atom_xyz = s.atom_xyz.copy()
            t.atom_xyz[j, x] += h
            Ep = oracle.qm_images(t, **QCONV)["E"]
            t.atom_xyz[j, x] -= 2 * h
            Em = oracle.qm_images(t, **QCONV)["E"]
            assert abs((Ep - Em) / (2 * h) - ref["dE_dRqm"][j, x]) < 2e-7 * np.max(np.abs(ref["dE_dRqm"]))


def test_qm_images_fock_is_density_derivative(qsys):
    s = qsys
    ref = oracle.qm_images(s, **QCONV)
    rng = np.random.default_rng(3)
    D = rng.normal(size=(s.nao, s.nao))
    D = D + D.T
    eps = 1e-4
    Ep = oracle.qm_images(s, s.dm + eps * D, **QCONV)["E"]
    Em = oracle.qm_images(s, s.dm - eps * D, **QCONV)["E"]
    assert abs((Ep - Em) / (2 * eps) - np.sum(ref["F"] * D)) < 1e-7 * abs(np.sum(ref["F"] * D))
