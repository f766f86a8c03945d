"""Pins of the oracle's region-I integrals (Eq. 9; point-charge form Eq. 2) and basis
normalisation, against quadrature, closed forms and limits that do not use its recursions."""
import math

import numpy as np
import pytest

import oracle
import workloads
from _quad import cart, int3c_quad, ovl1d

RNG = np.random.default_rng(11)


def _rand_case(rng):
    A = rng.uniform(-1, 1, 3)
    B = A + rng.uniform(-1.2, 1.2, 3)
    C = rng.uniform(-2.5, 2.5, 3)
    a = math.exp(rng.uniform(math.log(0.15), math.log(6.0)))
    b = math.exp(rng.uniform(math.log(0.15), math.log(6.0)))
    return a, A, b, B, C


@pytest.mark.parametrize("la,lb", [(la, lb) for la in range(4) for lb in range(4)])
@pytest.mark.parametrize("kappa", [7.0, 0.9, 0.0])
def test_int3c_against_quadrature(la, lb, kappa):
    rng = np.random.default_rng(100 * la + 10 * lb + int(kappa * 10))
    a, A, b, B, C = _rand_case(rng)
    got = oracle.int3c_prim(la, lb, a, A, b, B, kappa, C)
    ref = int3c_quad(la, lb, a, A, b, B, kappa, C, nodes=160 if kappa == 0 else 96)
    scale = np.max(np.abs(ref))
    assert np.max(np.abs(got - ref)) <= 1e-10 * scale


@pytest.mark.parametrize("kappa", [7.0, 0.3, 40.0])
def test_ss_closed_form(kappa):
    # <s_a s_b | erf(sqrt(kappa) r_C)/r_C> = S_ab erf(sqrt(rho)|PC|)/|PC|,
    # S_ab = (pi/p)^{3/2} K_AB, rho = p kappa/(p + kappa)
    for _ in range(20):
        a, A, b, B, C = _rand_case(RNG)
        p = a + b
        P = (a * A + b * B) / p
        S = (math.pi / p) ** 1.5 * math.exp(-a * b / p * np.sum((A - B) ** 2))
        rho = p * kappa / (p + kappa)
        R = np.linalg.norm(P - C)
        ref = S * math.erf(math.sqrt(rho) * R) / R
        got = oracle.int3c_prim(0, 0, a, A, b, B, kappa, C)[0, 0]
        assert abs(got - ref) <= 1e-14 * abs(ref)
        # point charge: rho -> p
        refp = S * math.erf(math.sqrt(p) * R) / R
        gotp = oracle.int3c_prim(0, 0, a, A, b, B, 0.0, C)[0, 0]
        assert abs(gotp - refp) <= 1e-14 * abs(refp)


@pytest.mark.parametrize("la,lb", [(0, 0), (1, 0), (2, 1), (3, 2), (3, 3)])
def test_point_charge_limit(la, lb):
    # sigma -> 0 (kappa = 1e12) reproduces the point-charge nuclear-attraction integrals
    a, A, b, B, C = _rand_case(np.random.default_rng(la * 7 + lb))
    g = oracle.int3c_prim(la, lb, a, A, b, B, 1e12, C)
    p = oracle.int3c_prim(la, lb, a, A, b, B, 0.0, C)
    assert np.max(np.abs(g - p)) <= 1e-10 * np.max(np.abs(p))


def test_gaussian_charge_far_field():
    # a Gaussian charge far from the pair acts as a point charge (erf -> 1)
    a, A, b, B, _ = _rand_case(RNG)
    C = np.array([40.0, -35.0, 20.0])
    for la, lb in [(1, 1), (2, 2)]:
        g = oracle.int3c_prim(la, lb, a, A, b, B, 7.0, C)
        p = oracle.int3c_prim(la, lb, a, A, b, B, 0.0, C)
        assert np.max(np.abs(g - p)) <= 1e-13 * np.max(np.abs(p))


@pytest.mark.parametrize("l", [0, 1, 2, 3])
def test_contraction_normalisation(l):
    # the contracted x^l component has unit self-overlap (Gauss-Hermite, independent of the C code)
    s = workloads.small_system(seed=3 + l, n_atoms=1, lmax=3, nprim=(3, 4))
    c = oracle.norm_coeffs(s)
    for sh in range(s.nshell):
        if s.shell_l[sh] != l:
            continue
        o, n = s.shell_prim_offset[sh], s.shell_nprim[sh]
        tot = 0.0
        for k in range(n):
            for m in range(n):
                ak, am = s.prim_exp[o + k], s.prim_exp[o + m]
                ox = ovl1d(l, l, 0, ak, 0.0, am, 0.0, 0.0, 0.0)
                oy = ovl1d(0, 0, 0, ak, 0.0, am, 0.0, 0.0, 0.0)
                tot += c[o + k] * c[o + m] * float(ox) * float(oy) ** 2
        assert abs(tot - 1.0) < 1e-13


def test_vpot_matches_quadrature_small_system():
    # whole V over a 2-atom basis with 3 charges, contracted, against the quadrature route
    s = workloads.small_system(seed=5, n_atoms=2, lmax=2, nprim=(1, 2), n_waters=1)
    c = oracle.norm_coeffs(s)
    chg = (np.array([[1.1, -0.4, 0.8], [-1.5, 0.9, 0.2], [0.3, 2.0, -1.0]]), np.array([0.7, -0.4, -0.3]),
           np.array([0.4, 0.0, 0.25]))
    V = oracle.vpot(s, charges=chg)
    off = np.concatenate([[0], np.cumsum([len(cart(l)) for l in s.shell_l])])
    ref = np.zeros_like(V)
    for sa in range(s.nshell):
        for sb in range(s.nshell):
            A, B = s.atom_xyz[s.shell_atom[sa]], s.atom_xyz[s.shell_atom[sb]]
            for ka in range(s.shell_nprim[sa]):
                for kb in range(s.shell_nprim[sb]):
                    pa, pb = s.shell_prim_offset[sa] + ka, s.shell_prim_offset[sb] + kb
                    for C, q, sg in zip(*chg):
                        kap = 1.0 / sg ** 2 if sg > 0 else 0.0
                        ref[off[sa]:off[sa + 1], off[sb]:off[sb + 1]] -= q * c[pa] * c[pb] * int3c_quad(
                            s.shell_l[sa], s.shell_l[sb], s.prim_exp[pa], A, s.prim_exp[pb], B, kap, C,
                            nodes=160 if kap == 0 else 96)
    assert np.max(np.abs(V - ref)) <= 1e-10 * np.max(np.abs(ref))
    assert np.allclose(V, V.T, rtol=0, atol=1e-14 * np.max(np.abs(V)))


def test_vpot_lattice_shift_invariance():
    s = workloads.small_system(seed=8, n_atoms=2, lmax=1, n_waters=8)
    V0 = oracle.vpot(s)
    s2 = s.copy()
    s2.mm_xyz[0:3] += s.box * np.array([1, -1, 2])  # move a whole water by a lattice vector
    V1 = oracle.vpot(s2)
    assert np.max(np.abs(V1 - V0)) <= 1e-12 * np.max(np.abs(V0))
