"""Pins of the oracle's multipole interaction tensors (SI, "Multipolar Ewald": point tensors T and
Gaussian-screened tensors T-hat) by finite differences, Laplacian traces and limits."""
import math

import numpy as np
import pytest

import oracle

I1 = {0: 1, 1: 2, 2: 3}
I2 = {(0, 0): 4, (0, 1): 5, (0, 2): 6, (1, 1): 7, (1, 2): 8, (2, 2): 9}
I3 = {(0, 0, 0): 10, (0, 0, 1): 11, (0, 0, 2): 12, (0, 1, 1): 13, (0, 1, 2): 14, (0, 2, 2): 15,
      (1, 1, 1): 16, (1, 1, 2): 17, (1, 2, 2): 18, (2, 2, 2): 19}


def i2(a, b):
    return I2[tuple(sorted((a, b)))]


def i3(a, b, c):
    return I3[tuple(sorted((a, b, c)))]


CASES = [(0, 0.0), (1, 0.4), (1, 1.3), (1, 3.0)]
DISP = [np.array([1.3, -0.7, 0.9]), np.array([-0.2, 2.1, 0.35]), np.array([0.6, 0.5, -0.4])]


@pytest.mark.parametrize("kind,beta", CASES)
@pytest.mark.parametrize("d", DISP)
def test_tensor_derivative_chain(kind, beta, d):
    # T_a = d/dR_a T, 2 T_ab = d/dR_b T_a, 3 T_abc = d/dR_c T_ab (central differences, 4th order)
    h = 1e-3 / max(1.0, beta)
    T = oracle.tensor(kind, beta, d)

    def D(comp, c):
        e = np.zeros(3)
        e[c] = h
        f = lambda x: oracle.tensor(kind, beta, d + x * e)[comp]
        return (-f(2) + 8 * f(1) - 8 * f(-1) + f(-2)) / (12 * h)

    scale = np.max(np.abs(T)) + 1e-30
    for a in range(3):
        assert abs(D(0, a) - T[I1[a]]) < 1e-8 * scale
        for b in range(3):
            assert abs(D(I1[a], b) - 2 * T[i2(a, b)]) < 1e-8 * scale
            for c in range(3):
                assert abs(D(i2(a, b), c) - 3 * T[i3(a, b, c)]) < 1e-8 * scale


@pytest.mark.parametrize("d", DISP)
def test_point_tensors_harmonic(d):
    # 1/r is harmonic away from the origin: traces of T_ab and T_abc vanish
    T = oracle.tensor(0, 0.0, d)
    assert abs(sum(T[i2(a, a)] for a in range(3))) < 1e-15 * abs(T[0]) / np.dot(d, d)
    for c in range(3):
        assert abs(sum(T[i3(a, a, c)] for a in range(3))) < 1e-14 * abs(T[0])


@pytest.mark.parametrize("beta", [0.3, 1.0, 2.2])
@pytest.mark.parametrize("d", DISP)
def test_screened_tensor_laplacian(beta, d):
    # Laplacian of erfc(beta r)/r is 4 pi times a normalised Gaussian of width 1/beta:
    # trace(T-hat_ab) = 1/2 lap f = 2 beta^3/sqrt(pi) exp(-beta^2 r^2)
    T = oracle.tensor(1, beta, d)
    r2 = float(np.dot(d, d))
    ref = 2 * beta ** 3 / math.sqrt(math.pi) * math.exp(-beta * beta * r2)
    tr = sum(T[i2(a, a)] for a in range(3))
    assert abs(tr - ref) < 1e-13 * max(abs(ref), 1e-3 * abs(T[0]))


@pytest.mark.parametrize("d", DISP)
def test_screened_tensor_limits(d):
    # beta -> 0: erfc -> 1, T-hat -> T;  beta -> infinity: T-hat -> 0
    T = oracle.tensor(0, 0.0, d)
    small = oracle.tensor(1, 1e-9, d)
    assert np.max(np.abs(small - T)) < 1e-8 * np.max(np.abs(T))
    big = oracle.tensor(1, 40.0, d)
    assert np.max(np.abs(big)) < 1e-100
