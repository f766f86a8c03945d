"""Pins of the oracle's Mulliken multipoles (SI, "Multipolar Ewald" definitions) and of the
region-II Fock term (Eqs. 11-14) against independent quadrature and exact identities."""
import numpy as np
import pytest

import oracle
import workloads
from _quad import ao_moments


@pytest.fixture(scope="module")
def sysm():
    return workloads.small_system(seed=21, n_atoms=3, lmax=2, nprim=(1, 2), n_waters=6)


@pytest.fixture(scope="module")
def moments(sysm):
    return ao_moments(sysm, oracle.norm_coeffs(sysm))


def test_multipoles_against_quadrature(sysm, moments):
    s, O = sysm, moments
    atom_of = np.repeat(s.shell_atom, [(l + 1) * (l + 2) // 2 for l in s.shell_l])
    ref = np.zeros((s.natm, 10))
    ref[:, 0] = s.atom_Z
    for mu in range(s.nao):
        k = atom_of[mu]
        for op in range(10):
            ref[k, op] -= np.dot(s.dm[:, mu], O[op, mu, :])
    got = oracle.multipoles(s)
    assert np.max(np.abs(got - ref)) < 1e-11 * np.max(np.abs(ref))


def test_charge_sum_rule(sysm, moments):
    # sum_j Q_j = sum_j Z_j - tr(gamma S)
    s, O = sysm, moments
    M = oracle.multipoles(s)
    assert abs(M[:, 0].sum() - (s.atom_Z.sum() - np.sum(s.dm * O[0]))) < 1e-11 * s.atom_Z.sum()


def test_total_dipole_identity(sysm, moments):
    # sum_j (mu_j + Q_j R_j) = sum_j Z_j R_j - sum dm <mu| r |nu>: independent of the atom split,
    # so it pins the operator centring and signs
    s, O = sysm, moments
    atom_of = np.repeat(s.shell_atom, [(l + 1) * (l + 2) // 2 for l in s.shell_l])
    Rmu = s.atom_xyz[atom_of]  # centre of each mu
    M = oracle.multipoles(s)
    tot = M[:, 1:4].sum(0) + (M[:, 0:1] * s.atom_xyz).sum(0)
    # <mu|r_a|nu> = <mu|(r-R_mu)_a|nu> + R_mu,a <mu|nu>
    ra = np.stack([O[1 + a] + Rmu[:, a:a + 1] * O[0] for a in range(3)])
    ref = (s.atom_Z[:, None] * s.atom_xyz).sum(0) - np.einsum("nm,amn->a", s.dm, ra)
    assert np.max(np.abs(tot - ref)) < 1e-11 * np.max(np.abs(ref))


def test_fock_is_energy_derivative(sysm):
    # E_II is linear in gamma: E_II(gamma + D) - E_II(gamma) = sum F_II * D for symmetric D
    s = sysm
    phi = np.random.default_rng(3).normal(size=(s.natm, 20))
    F = oracle.fock_ii(s, phi)
    assert np.allclose(F, F.T, atol=1e-14 * np.max(np.abs(F)))
    D = np.random.default_rng(4).normal(size=(s.nao, s.nao))
    D = D + D.T
    e0 = oracle.multipole_energy(oracle.multipoles(s), phi)
    e1 = oracle.multipole_energy(oracle.multipoles(s, s.dm + D), phi)
    assert abs((e1 - e0) - np.sum(F * D)) < 1e-11 * (abs(e1 - e0) + 1)
