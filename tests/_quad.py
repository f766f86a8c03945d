"""Independent numerical quadrature used to pin the oracle's integrals.

The region-I integral of Eq. 9 is evaluated without any Boys function or recursion: the smeared
Coulomb potential is written as erf(s r)/r = 2/sqrt(pi) int_0^s exp(-t^2 r^2) dt, the inner
three-Gaussian overlap factorises into 1-D integrals that Gauss-Hermite quadrature integrates
exactly, and the outer t-integral is done with Gauss-Legendre quadrature.
"""
import math

import numpy as np


def cart(l):
    """Cartesian exponents of shell l, lexicographic (x^l first)."""
    return [(lx, ly, l - lx - ly) for lx in range(l, -1, -1) for ly in range(l - lx, -1, -1)]


def ovl1d(i, j, e, a, A, b, B, c, C, K=None):
    """int (x-A)^i (x-B)^j (x-K)^e exp(-a(x-A)^2 - b(x-B)^2 - c(x-C)^2) dx, exact by Gauss-Hermite.
    a, b, c may be numpy arrays (vectorised over c)."""
    c = np.asarray(c, dtype=float)
    q = a + b + c
    Q = (a * A + b * B + c * C) / q
    pre = np.exp(-(a * b * (A - B) ** 2 + a * c * (A - C) ** 2 + b * c * (B - C) ** 2) / q)
    n = (i + j + e) // 2 + 2
    y, w = np.polynomial.hermite.hermgauss(n)
    K = 0.0 if K is None else K
    x = Q[..., None] + y / np.sqrt(q)[..., None]
    f = (x - A) ** i * (x - B) ** j * (x - K) ** e
    return pre * np.sum(w * f, axis=-1) / np.sqrt(q)


def int3c_quad(la, lb, a, A, b, B, kappa, C, nodes=96):
    """<g_a g_b | erf(sqrt(kappa)|r-C|)/|r-C|> for unnormalised Cartesian primitives; kappa <= 0
    gives the point charge 1/|r-C|."""
    x, w = np.polynomial.legendre.leggauss(nodes)
    if kappa > 0:
        s = math.sqrt(kappa)
        t = 0.5 * s * (x + 1)
        wt = 0.5 * s * w
    else:
        u = 0.5 * (x + 1)
        t = u / (1 - u)
        wt = 0.5 * w / (1 - u) ** 2
    c = t * t
    out = np.zeros((len(cart(la)), len(cart(lb))))
    for ia, ea in enumerate(cart(la)):
        for ib, eb in enumerate(cart(lb)):
            f = np.ones_like(t)
            for d in range(3):
                f = f * ovl1d(ea[d], eb[d], 0, a, A[d], b, B[d], c, C[d])
            out[ia, ib] = 2.0 / math.sqrt(math.pi) * np.sum(wt * f)
    return out


def moment_quad(la, lb, a, A, b, B, K, op):
    """<g_a | (x-K_x)^ox (y-K_y)^oy (z-K_z)^oz | g_b> for unnormalised primitives."""
    out = np.zeros((len(cart(la)), len(cart(lb))))
    for ia, ea in enumerate(cart(la)):
        for ib, eb in enumerate(cart(lb)):
            v = 1.0
            for d in range(3):
                v *= float(ovl1d(ea[d], eb[d], op[d], a, A[d], b, B[d], 0.0, 0.0, K[d]))
            out[ia, ib] = v
    return out


OPS = [(0, 0, 0), (1, 0, 0), (0, 1, 0), (0, 0, 1), (2, 0, 0), (1, 1, 0), (1, 0, 1), (0, 2, 0), (0, 1, 1), (0, 0, 2)]


OPS3 = [(3, 0, 0), (2, 1, 0), (2, 0, 1), (1, 2, 0), (1, 1, 1), (1, 0, 2), (0, 3, 0), (0, 2, 1), (0, 1, 2), (0, 0, 3)]


def ao_moments(s, ncoef, ops=OPS):
    """AO-basis moment matrices O[op][mu,nu] = <mu|(r-R_{atom(mu)})^op|nu> by quadrature."""
    off = np.concatenate([[0], np.cumsum([(l + 1) * (l + 2) // 2 for l in s.shell_l])])
    out = np.zeros((len(ops), s.nao, s.nao))
    for sa in range(s.nshell):
        for sb in range(s.nshell):
            A = s.atom_xyz[s.shell_atom[sa]]
            B = s.atom_xyz[s.shell_atom[sb]]
            la, lb = s.shell_l[sa], s.shell_l[sb]
            for ka in range(s.shell_nprim[sa]):
                for kb in range(s.shell_nprim[sb]):
                    pa, pb = s.shell_prim_offset[sa] + ka, s.shell_prim_offset[sb] + kb
                    cc = ncoef[pa] * ncoef[pb]
                    for k, op in enumerate(ops):
                        out[k, off[sa]:off[sa + 1], off[sb]:off[sb + 1]] += cc * moment_quad(
                            la, lb, s.prim_exp[pa], A, s.prim_exp[pb], B, A, op)
    return out
