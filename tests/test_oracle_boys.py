"""Pins of the oracle's Boys function F_n(T) = int_0^1 t^2n exp(-T t^2) dt (used by Eq. 9's
integrals) against results fixed independently of its series/asymptotic code."""
import math

import numpy as np
import pytest

import oracle

scipy_special = pytest.importorskip("scipy.special")

TS = [0.0, 1e-12, 1e-6, 0.05, 0.7, 3.0, 11.0, 24.5, 36.0, 49.9, 50.0, 50.1, 77.0, 300.0, 5e4]


@pytest.mark.parametrize("T", TS)
def test_f0_closed_form(T):
    # F_0(T) = 1/2 sqrt(pi/T) erf(sqrt T), libm erf
    F = oracle.boys(0, T)[0]
    ref = 1.0 if T == 0 else 0.5 * math.sqrt(math.pi / T) * math.erf(math.sqrt(T))
    assert abs(F - ref) <= 2e-15 * ref


def test_value_at_zero():
    F = oracle.boys(12, 0.0)
    assert np.allclose(F, [1.0 / (2 * n + 1) for n in range(13)], rtol=1e-15, atol=0)


@pytest.mark.parametrize("T", TS[1:])
def test_downward_recursion_identity(T):
    # F_n = (2T F_{n+1} + e^{-T}) / (2n+1): ties the orders together in both regimes
    F = oracle.boys(10, T)
    for n in range(10):
        lhs = F[n]
        rhs = (2 * T * F[n + 1] + math.exp(-T)) / (2 * n + 1)
        assert abs(lhs - rhs) <= 2e-13 * lhs


@pytest.mark.parametrize("T", [0.3, 2.0, 9.0, 20.0, 35.0, 49.0, 52.0, 80.0])
def test_against_confluent_hypergeometric(T):
    # F_n(T) = 1F1(n+1/2; n+3/2; -T) / (2n+1), scipy's independent routine
    F = oracle.boys(8, T)
    ref = np.array([scipy_special.hyp1f1(n + 0.5, n + 1.5, -T) / (2 * n + 1) for n in range(9)])
    assert np.max(np.abs(F - ref) / ref) < 1e-12


def test_quadrature_definition():
    # direct Gauss-Legendre quadrature of the defining integral
    x, w = np.polynomial.legendre.leggauss(80)
    t = 0.5 * (x + 1)
    for T in [0.01, 1.0, 7.5, 18.0]:
        F = oracle.boys(6, T)
        for n in range(7):
            ref = 0.5 * np.sum(w * t ** (2 * n) * np.exp(-T * t * t))
            assert abs(F[n] - ref) < 1e-14 * max(ref, 1e-300) + 1e-300


def test_switch_continuity():
    # series (T < 50) and asymptotic (T >= 50) agree at the switch
    d = 1e-7
    a = oracle.boys(10, 50.0 - d)
    b = oracle.boys(10, 50.0)
    # dF_n/dT = -F_{n+1}: F_n(T - d) = F_n(T) + d F_{n+1}(T) + O(d^2)
    pred = b[:10] + d * b[1:11]
    assert np.max(np.abs(a[:10] - pred) / pred) < 1e-13
