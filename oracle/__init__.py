"""Plain FP64 CPU oracle for the periodic QM/MM-Multipole embedding (arXiv 2408.03273).

TEST INFRASTRUCTURE ONLY.  The tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package; the CUDA library and its Python binding never do, and the
two share no code.  The arithmetic lives in ``qmmm_oracle.c`` (Obara-Saika integrals, series /
asymptotic Boys function, literal Ewald loops); this module only compiles it with gcc, marshals
arrays through ctypes and composes the pieces into the energy terms of Eq. 6 / Eq. 10 and their
gradients (Eq. 15 and the region-I integral derivatives).

Parity status: every function here is pinned by a ``-m "not gpu"`` test against an independent
result (closed forms, quadrature, limits, invariances, finite differences, direct lattice sums).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "qmmm_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

# Ewald mode bits (mirrors the C defines)
EW_SR, EW_LR, EW_BG, EW_R1, EW_HAT = 1, 2, 4, 8, 16
EW_ALL = EW_SR | EW_LR | EW_BG | EW_R1 | EW_HAT
# weights of the 10 stored multipole components in a full (a,b) contraction
W10 = np.array([1, 1, 1, 1, 1, 2, 2, 1, 2, 1], dtype=np.float64)


def build(force: bool = False) -> str:
    """Compile the oracle into oracle/_build/liboracle.so (plain gcc, OpenMP, no fast-math)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            dp = ctypes.POINTER(ctypes.c_double)
            ip = ctypes.POINTER(ctypes.c_int)
            i, d = ctypes.c_int, ctypes.c_double
            sig = {
                "oracle_boys": (None, [i, d, dp]),
                "oracle_norm_coeffs": (None, [i, ip, ip, ip, dp, dp, dp]),
                "oracle_int3c_prim": (None, [i, i, d, dp, d, dp, d, dp, dp]),
                "oracle_vpot": (None, [i, ip, ip, ip, ip, dp, dp, dp, i, dp, dp, dp, i, ip, i, dp]),
                "oracle_vgrad": (None, [i, ip, ip, ip, ip, dp, dp, i, dp, i, dp, dp, dp, i, dp, i, ip, dp, dp, dp]),
                "oracle_enucmm": (d, [i, dp, dp, i, dp, dp, dp, dp, dp, dp]),
                "oracle_multipoles": (None, [i, ip, ip, ip, ip, dp, dp, i, dp, dp, i, dp, dp]),
                "oracle_octupoles": (None, [i, ip, ip, ip, ip, dp, dp, i, dp, i, dp, dp]),
                "oracle_qmqm": (None, [i, dp, dp, dp, d, d, ip, dp, dp, dp]),
                "oracle_fock_ii": (None, [i, ip, ip, ip, ip, dp, dp, dp, dp, i, i, dp]),
                "oracle_pulay": (None, [i, ip, ip, ip, ip, dp, dp, dp, dp, i, i, dp, dp]),
                "oracle_tensor": (None, [i, d, dp, dp]),
                "oracle_region1": (i, [i, dp, i, dp, dp, d, i, ip, dp]),
                "oracle_ewald_phi": (None, [i, dp, i, dp, dp, dp, dp, d, d, d, ip, i, dp]),
                "oracle_ewald_mm": (None, [i, dp, dp, i, dp, dp, dp, dp, d, d, d, ip, i, ctypes.c_void_p, dp, dp]),
                "oracle_tensor_grad_qm": (None, [i, dp, dp, dp]),
            }
            for name, (res, args) in sig.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def _d(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _i(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if a is not None else None


def _ip(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int)) if a is not None else None


# ----------------------------------------------------------------------------------------------
# elementary pieces
# ----------------------------------------------------------------------------------------------

def boys(nmax: int, T: float) -> np.ndarray:
    out = np.zeros(nmax + 1)
    lib().oracle_boys(nmax, float(T), _dp(out))
    return out


def tensor(kind: int, beta: float, d) -> np.ndarray:
    """20 Taylor tensor components at displacement d = R_j - R_i (kind 0: 1/r, 1: erfc(beta r)/r)."""
    dd = _d(d)
    out = np.zeros(20)
    lib().oracle_tensor(kind, float(beta), _dp(dd), _dp(out))
    return out


def int3c_prim(la, lb, a, A, b, B, kappa, C) -> np.ndarray:
    out = np.zeros(((la + 1) * (la + 2) // 2) * ((lb + 1) * (lb + 2) // 2))
    A, B, C = _d(A), _d(B), _d(C)
    lib().oracle_int3c_prim(la, lb, a, _dp(A), b, _dp(B), float(kappa), _dp(C), _dp(out))
    return out.reshape((la + 1) * (la + 2) // 2, (lb + 1) * (lb + 2) // 2)


class _Basis:
    def __init__(self, s):
        self.atom, self.l = _i(s.shell_atom), _i(s.shell_l)
        self.nprim, self.off = _i(s.shell_nprim), _i(s.shell_prim_offset)
        self.exps = _d(s.prim_exp)
        self.ncoef = np.zeros_like(self.exps)
        lib().oracle_norm_coeffs(len(self.l), _ip(self.l), _ip(self.nprim), _ip(self.off), _dp(self.exps),
                                 _dp(_d(s.prim_coeff)), _dp(self.ncoef))
        self.n = len(self.l)

    def args(self):
        return (self.n, _ip(self.atom), _ip(self.l), _ip(self.nprim), _ip(self.off), _dp(self.exps), _dp(self.ncoef))


def norm_coeffs(s) -> np.ndarray:
    return _Basis(s).ncoef


def ewald_rc(s) -> float:
    return s.ewald_rcut if s.ewald_rcut > 0 else s.cutoff


def region1(s):
    """Region-I images (charge index, shift) with |R_i + L - c| < cutoff, c = QM mean."""
    qm, mm, box = _d(s.atom_xyz), _d(s.mm_xyz), _d(s.box)
    cap = max(16, s.nmm * 8)
    while True:
        idx = np.zeros(cap, dtype=np.int32)
        sh = np.zeros((cap, 3))
        n = lib().oracle_region1(s.natm, _dp(qm), s.nmm, _dp(mm), _dp(box), float(s.cutoff), cap, _ip(idx), _dp(sh))
        if n <= cap:
            return idx[:n].copy(), sh[:n].copy()
        cap = n


def region1_charges(s):
    idx, sh = region1(s)
    xyz = np.ascontiguousarray(s.mm_xyz[idx] + sh)
    return idx, xyz, _d(s.mm_q[idx]), _d(s.mm_sigma[idx])


def vpot(s, pairs=None, charges=None) -> np.ndarray:
    """Region-I V (Eq. 9) over all ordered shell pairs (or the listed (A,B) pairs only)."""
    b = _Basis(s)
    if charges is None:
        _, cx, cq, cs = region1_charges(s)
    else:
        cx, cq, cs = (_d(c) for c in charges)
    V = np.zeros((s.nao, s.nao))
    pr = None if pairs is None else _i(np.asarray(pairs).reshape(-1, 2))
    npairs = 0 if pr is None else len(pr)
    lib().oracle_vpot(*b.args(), _dp(_d(s.atom_xyz)), len(cq), _dp(cx), _dp(cq), _dp(cs), npairs, _ip(pr),
                      s.nao, _dp(V))
    return V


def enucmm(s, charges=None):
    if charges is None:
        _, cx, cq, cs = region1_charges(s)
    else:
        cx, cq, cs = (_d(c) for c in charges)
    return lib().oracle_enucmm(s.natm, _dp(_d(s.atom_xyz)), _dp(_d(s.atom_Z)), len(cq), _dp(cx), _dp(cq), _dp(cs),
                               None, None, None)


def multipoles(s, dm=None) -> np.ndarray:
    b = _Basis(s)
    dm = _d(s.dm if dm is None else dm)
    out = np.zeros((s.natm, 10))
    lib().oracle_multipoles(*b.args(), s.natm, _dp(_d(s.atom_xyz)), _dp(_d(s.atom_Z)), s.nao, _dp(dm), _dp(out))
    return out


def octupoles(s, dm=None) -> np.ndarray:
    """Mulliken octupoles Omega_j (SI, Multipolar Ewald): natm x 10 (xxx, xxy, xxz, xyy, xyz, xzz,
    yyy, yyz, yzz, zzz)."""
    b = _Basis(s)
    dm = _d(s.dm if dm is None else dm)
    out = np.zeros((s.natm, 10))
    lib().oracle_octupoles(*b.args(), s.natm, _dp(_d(s.atom_xyz)), s.nao, _dp(dm), _dp(out))
    return out


# multiplicity of each unique component of a symmetric rank-3 tensor in the full contraction
MULT3 = np.array([1, 3, 3, 3, 6, 3, 1, 3, 3, 1], dtype=np.float64)


def octupole_error(s, radii, dm=None) -> np.ndarray:
    """Octupole error estimate of the multipole truncation (Sec. "Error Control", the charge-octupole
    sum over region II): for each region-I radius R, sum_j sum_abc Omega_j,abc v_j,abc(R), with
    v_j,abc(R) the third Taylor components (T_abc = 1/6 d^3) of the region-II potential at atom j
    when region I is the sphere of radius R (periodic, as the l <= 2 terms; the Ewald real-space
    cutoff stays the system's).  Region II is recomputed from scratch for every R."""
    Om = octupoles(s, dm)
    out = []
    km = _i(s.kmax)
    for R in radii:
        phi = np.zeros((s.natm, 20))
        lib().oracle_ewald_phi(s.natm, _dp(_d(s.atom_xyz)), s.nmm, _dp(_d(s.mm_xyz)), _dp(_d(s.mm_q)),
                               _dp(_d(s.mm_sigma)), _dp(_d(s.box)), float(R), float(ewald_rc(s)),
                               float(s.ewald_alpha), _ip(km), EW_ALL, _dp(phi))
        out.append(float(np.sum(MULT3[None, :] * Om * phi[:, 10:20])))
    return np.array(out)


def qmqm(s, M=None, alpha=None, kmax=None, ewald_rcut=None):
    """QM-QM periodic-image multipole energy (Eq. 5, in the Ewald form of Eq. 6) for multipoles M
    (natm x 10; default: the Mulliken multipoles of s): (E, u, grad) with u = dE/dM per stored
    component / W10 (natm x 10) and grad = dE/dR_QM at fixed multipoles (natm x 3).  alpha, kmax
    and ewald_rcut default to the system's."""
    M = _d(multipoles(s) if M is None else M)
    E = np.zeros(1)
    u = np.zeros((s.natm, 10))
    g = np.zeros((s.natm, 3))
    km = _i(s.kmax if kmax is None else kmax)
    lib().oracle_qmqm(s.natm, _dp(_d(s.atom_xyz)), _dp(M), _dp(_d(s.box)),
                      float(ewald_rc(s) if ewald_rcut is None else ewald_rcut),
                      float(s.ewald_alpha if alpha is None else alpha), _ip(km), _dp(E), _dp(u), _dp(g))
    return float(E[0]), u, g


def qm_images(s, dm=None, **conv):
    """QM-QM periodic-image term at density dm (Eq. 5 / Eq. 6): E, its gradient dE/dR_QM at fixed
    density (image tensors at fixed multipoles plus the multipoles' dependence on the basis
    positions, the Pulay term of Eq. 15 with the image potential u) and its Fock matrix
    dE/dgamma (Eqs. 11-14 with u in place of the MM potential).  conv: alpha, kmax, ewald_rcut."""
    dm = _d(s.dm if dm is None else dm)
    M = multipoles(s, dm)
    E, u, g = qmqm(s, M, **conv)
    b = _Basis(s)
    lib().oracle_pulay(*b.args(), _dp(_d(s.atom_xyz)), _dp(_d(u)), 10, s.nao, _dp(dm), _dp(g))
    return {"E": E, "dE_dRqm": g, "F": fock_ii(s, u), "u": u, "M": M}


def aspc_coefficients(K: int) -> np.ndarray:
    """Predictor weights of the always-stable predictor-corrector density extrapolation used for
    the MD runs (Sec. "Common Setup", from K+1 previous steps; Kolafa's closed form):
      B_j = (-1)^(j+1) j C(2K+2, K+1-j) / C(2K, K),  j = 1..K+1,
    so that gamma_pred(t) = sum_j B_j gamma(t - j)."""
    from math import comb
    return np.array([(-1) ** (j + 1) * j * comb(2 * K + 2, K + 1 - j) / comb(2 * K, K) for j in range(1, K + 2)])


def aspc_predict(history) -> np.ndarray:
    """history[j-1] = gamma(t - j), most recent first."""
    B = aspc_coefficients(len(history) - 1)
    return sum(b * np.asarray(h, dtype=np.float64) for b, h in zip(B, history))


def ewald_phi(s, mode: int = EW_ALL) -> np.ndarray:
    """Generalised potential (20 components) at each QM atom from all MM charges."""
    out = np.zeros((s.natm, 20))
    km = _i(s.kmax)
    lib().oracle_ewald_phi(s.natm, _dp(_d(s.atom_xyz)), s.nmm, _dp(_d(s.mm_xyz)), _dp(_d(s.mm_q)),
                           _dp(_d(s.mm_sigma)), _dp(_d(s.box)), float(s.cutoff), float(ewald_rc(s)),
                           float(s.ewald_alpha), _ip(km), mode, _dp(out))
    return out


def ewald_mm(s, M, mode: int = EW_ALL, mm_subset=None):
    """MM-side potential (dE/dq) and dE/dR_MM from QM multipoles M[natm,10]; with ``mm_subset``
    only the listed MM charges are evaluated (the rest stay zero)."""
    dq = np.zeros(s.nmm)
    dR = np.zeros((s.nmm, 3))
    km = _i(s.kmax)
    only = None
    if mm_subset is not None:
        only = np.zeros(s.nmm, dtype=np.uint8)
        only[np.asarray(mm_subset)] = 1
    lib().oracle_ewald_mm(s.natm, _dp(_d(s.atom_xyz)), _dp(_d(M)), s.nmm, _dp(_d(s.mm_xyz)), _dp(_d(s.mm_q)),
                          _dp(_d(s.mm_sigma)), _dp(_d(s.box)), float(s.cutoff), float(ewald_rc(s)),
                          float(s.ewald_alpha), _ip(km), mode,
                          None if only is None else ctypes.c_void_p(only.ctypes.data), _dp(dq), _dp(dR))
    return dq, dR


def fock_ii(s, phi) -> np.ndarray:
    b = _Basis(s)
    ph = _d(phi)
    F = np.zeros((s.nao, s.nao))
    lib().oracle_fock_ii(*b.args(), _dp(_d(s.atom_xyz)), _dp(ph), ph.shape[1], s.nao, _dp(F))
    return F


def multipole_energy(M, phi) -> float:
    """E_II = sum_j sum_c W_c M_j,c phi_j,c (first 10 components)."""
    return float(np.sum(W10[None, :] * M * phi[:, :10]))


# ----------------------------------------------------------------------------------------------
# composed energy and gradient
# ----------------------------------------------------------------------------------------------

def pulay_grad(s, phi, dm=None, ncomp: int = 20) -> np.ndarray:
    """The multipoles' dependence on the basis-function centres (the Pulay term of Eq. 15):
    dE/dR_QM of sum_j phi_j . (Q, mu, theta)_j at fixed density, phi[natm, ncomp] the potential
    components the multipoles meet (20: the region-II potential; 10: the QM image potential)."""
    dm = _d(s.dm if dm is None else dm)
    g = np.zeros((s.natm, 3))
    lib().oracle_pulay(*_Basis(s).args(), _dp(_d(s.atom_xyz)), _dp(_d(phi)), ncomp, s.nao, _dp(dm), _dp(g))
    return g


def tensor_grad_qm(s, M, phi) -> np.ndarray:
    """dE/dR_QM from the tensors at fixed multipoles: sum_j (Q, mu, theta)_j . d phi_j / dR_j."""
    g = np.zeros((s.natm, 3))
    lib().oracle_tensor_grad_qm(s.natm, _dp(_d(M)), _dp(_d(phi)), _dp(g))
    return g


def energy(s, dm=None, mode: int = EW_ALL):
    """Energy terms of E_QM-MM at fixed density: region-I electronic and nuclear parts and the
    region-II multipole part (Eq. 6 QM-MM lines + Eq. 10)."""
    dm = s.dm if dm is None else dm
    V = vpot(s)
    En = enucmm(s)
    M = multipoles(s, dm)
    phi = ewald_phi(s, mode)
    EI = float(np.sum(dm * V))
    EII = multipole_energy(M, phi)
    return {"V": V, "E_I_elec": EI, "E_nuc_mm": En, "E_II": EII, "E": EI + En + EII, "M": M, "phi": phi}


def forces(s, dm=None, mode: int = EW_ALL, charge_subset=None, mm_subset=None):
    """dE/dR_QM, dE/dR_MM and dE/dq of E_QM-MM at fixed density (outputs are gradients).

    ``charge_subset`` restricts the region-I integral part to the listed region-I entries
    (indices into the region-I list) and ``mm_subset`` the Ewald MM-side sums to the listed MM
    charges -- used to sample large systems; the QM gradient is then partial and only the listed
    charges' MM gradients are complete."""
    dm = _d(s.dm if dm is None else dm)
    b = _Basis(s)
    idx, cx, cq, cs = region1_charges(s)
    if charge_subset is not None:
        sub = np.asarray(charge_subset)
        idx, cx, cq, cs = idx[sub], np.ascontiguousarray(cx[sub]), cq[sub], cs[sub]
    n = len(cq)
    dRqm = np.zeros((s.natm, 3))
    dC = np.zeros((n, 3))
    dqc = np.zeros(n)
    qm = _d(s.atom_xyz)
    lib().oracle_vgrad(*b.args(), s.natm, _dp(qm), n, _dp(cx), _dp(cq), _dp(cs), s.nao, _dp(dm), 0, None, _dp(dRqm),
                       _dp(dC), _dp(dqc))
    # region-I electronic part alone (the part the mixed-precision path evaluates in FP32)
    elec_qm = dRqm.copy()
    elec_mm, elec_q = np.zeros((s.nmm, 3)), np.zeros(s.nmm)
    np.add.at(elec_mm, idx, dC)
    np.add.at(elec_q, idx, dqc)
    lib().oracle_enucmm(s.natm, _dp(qm), _dp(_d(s.atom_Z)), n, _dp(cx), _dp(cq), _dp(cs), _dp(dRqm), _dp(dC),
                        _dp(dqc))
    dRmm = np.zeros((s.nmm, 3))
    dq = np.zeros(s.nmm)
    np.add.at(dRmm, idx, dC)
    np.add.at(dq, idx, dqc)
    M = multipoles(s, dm)
    phi = ewald_phi(s, mode)
    dRqm += tensor_grad_qm(s, M, phi)
    dRqm += pulay_grad(s, phi, dm)
    dq2, dR2 = ewald_mm(s, M, mode, mm_subset=mm_subset)
    return {"dE_dRqm": dRqm, "dE_dRmm": dRmm + dR2, "dE_dq": dq + dq2, "M": M, "phi": phi,
            "elec": {"dE_dRqm": elec_qm, "dE_dRmm": elec_mm, "dE_dq": elec_q}}


def forces_mm_subset(s, charge_subset, dm=None, mode: int = EW_ALL):
    """dE/dq and dE/dR_MM of the MM charges behind the listed region-I entries (each charge with a
    single image in region I), composed as in ``forces`` without the QM-side terms: the region-I
    electronic and nuclear parts over those entries plus the MM-side Ewald derivatives from the
    multipoles of the full density.  Returns (mm indices, dE_dq[k], dE_dRmm[k, 3])."""
    dm = _d(s.dm if dm is None else dm)
    b = _Basis(s)
    idx, cx, cq, cs = region1_charges(s)
    sub = np.asarray(charge_subset)
    idx, cx, cq, cs = idx[sub], np.ascontiguousarray(cx[sub]), cq[sub], cs[sub]
    n = len(cq)
    dRqm, dC, dqc = np.zeros((s.natm, 3)), np.zeros((n, 3)), np.zeros(n)
    qm = _d(s.atom_xyz)
    lib().oracle_vgrad(*b.args(), s.natm, _dp(qm), n, _dp(cx), _dp(cq), _dp(cs), s.nao, _dp(dm), 0, None, _dp(dRqm),
                       _dp(dC), _dp(dqc))
    lib().oracle_enucmm(s.natm, _dp(qm), _dp(_d(s.atom_Z)), n, _dp(cx), _dp(cq), _dp(cs), _dp(dRqm), _dp(dC),
                        _dp(dqc))
    M = multipoles(s, dm)
    dq2, dR2 = ewald_mm(s, M, mode, mm_subset=idx)
    return idx, dqc + dq2[idx], dC + dR2[idx]


def vgrad_pairs(s, pairs, dm=None):
    """Region-I gradient pieces restricted to the listed ordered shell pairs (timing samples)."""
    dm = _d(s.dm if dm is None else dm)
    b = _Basis(s)
    _, cx, cq, cs = region1_charges(s)
    pr = _i(np.asarray(pairs).reshape(-1, 2))
    n = len(cq)
    dRqm, dC, dqc = np.zeros((s.natm, 3)), np.zeros((n, 3)), np.zeros(n)
    lib().oracle_vgrad(*b.args(), s.natm, _dp(_d(s.atom_xyz)), n, _dp(cx), _dp(cq), _dp(cs), s.nao, _dp(dm), len(pr),
                       _ip(pr), _dp(dRqm), _dp(dC), _dp(dqc))
    return dRqm, dC, dqc
