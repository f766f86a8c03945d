"""ctypes binding of include/qmmm.h: the same entry points, argument marshalling only.

Every array argument may be a numpy array (host) or a torch tensor (host or CUDA); it must be
float64 and C-contiguous.  Outputs that the caller does not pass are allocated here (numpy on
the host by default, or torch tensors on a given device).  The library does all arithmetic on
the GPU; if it cannot be loaded this module raises -- there is no other implementation.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

c_int, c_double, c_void_p, c_ll = ctypes.c_int, ctypes.c_double, ctypes.c_void_p, ctypes.c_longlong

QMMM_FP64, QMMM_MIXED = 0, 1
ERRORS = {0: "QMMM_OK", -1: "QMMM_ERR_ARG", -2: "QMMM_ERR_ALLOC", -3: "QMMM_ERR_CUDA", -4: "QMMM_ERR_TIMEOUT",
          -5: "QMMM_ERR_UNSUPPORTED_L", -6: "QMMM_ERR_STATE"}


class QmmmAtom(ctypes.Structure):
    _fields_ = [("xyz", c_double * 3), ("Z", c_double)]


class QmmmShell(ctypes.Structure):
    _fields_ = [("atom", c_int), ("l", c_int), ("nprim", c_int), ("prim_offset", c_int)]


class QmmmPrimitive(ctypes.Structure):
    _fields_ = [("exponent", c_double), ("coeff", c_double)]


class QmmmCharge(ctypes.Structure):
    _fields_ = [("xyz", c_double * 3), ("q", c_double), ("sigma", c_double)]


class QmmmOptions(ctypes.Structure):
    _fields_ = [("precision", c_int), ("screen_tol", c_double), ("region_mode", c_int), ("ewald_rcut", c_double),
                ("kmax", c_int * 3), ("full_cell_test", c_int)]


class QmmmInfo(ctypes.Structure):
    _fields_ = [("nao", c_int), ("natm", c_int), ("nshell", c_int), ("nmm", c_int), ("n_shell_pairs", c_ll),
                ("n_prim_pairs", c_ll), ("n_region1", c_int), ("n_gvec", c_int), ("n_sigma_classes", c_int),
                ("precision", c_int), ("n_prim_pairs_class", c_ll * 10), ("n_shell_pairs_class", c_ll * 10)]


class QMMMError(RuntimeError):
    def __init__(self, code, where):
        self.code = code
        detail = _L.qmmm_last_error().decode() if _L is not None else ""
        super().__init__(f"{where}: {ERRORS.get(code, code)} ({detail})")


_L = None

EXPORTS = ("qmmm_create", "qmmm_set_stream", "qmmm_set_precision", "qmmm_set_recip_method", "qmmm_set_positions", "qmmm_vpot", "qmmm_ewald",
           "qmmm_energy", "qmmm_density_gradient", "qmmm_forces", "qmmm_get_info", "qmmm_nao", "qmmm_get_potential", "qmmm_last_timing",
           "qmmm_qm_images", "qmmm_aspc_predict", "qmmm_selftest_bounded_wait", "qmmm_octupole_error", "qmmm_rcut_search", "qmmm_autotune", "qmmm_get_tuning", "qmmm_set_tuning", "qmmm_batch_create", "qmmm_batch_run",
           "qmmm_batch_timing", "qmmm_batch_captures", "qmmm_batch_counts", "qmmm_batch_destroy", "qmmm_destroy", "qmmm_strerror", "qmmm_last_error", "qmmm_nuclear_mm_energy_static")


def library_path() -> str:
    return _build.LIB


def load(build_if_needed: bool = True):
    """Load the sm_103a library (building it in-tree first if the sources are newer)."""
    global _L
    if _L is not None:
        return _L
    if build_if_needed and _build.needs_build():
        _build.build()
    if not os.path.exists(_build.LIB):
        raise ImportError(f"CUDA library {_build.LIB} is missing; run paper_2408_03273_gb300.build.build()")
    L = ctypes.CDLL(_build.LIB)
    P = ctypes.POINTER
    sig = {
        "qmmm_create": (c_int, [P(QmmmAtom), c_int, P(QmmmShell), c_int, P(QmmmPrimitive), c_int, P(QmmmCharge), c_int,
                                P(c_double), c_double, c_double, P(QmmmOptions), P(c_void_p)]),
        "qmmm_set_stream": (c_int, [c_void_p, c_void_p]),
        "qmmm_set_precision": (c_int, [c_void_p, c_int]),
        "qmmm_set_recip_method": (c_int, [c_void_p, c_int]),
        "qmmm_set_positions": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p]),
        "qmmm_vpot": (c_int, [c_void_p, c_void_p, c_void_p]),
        "qmmm_ewald": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
        "qmmm_energy": (c_int, [c_void_p, c_void_p, c_void_p]),
        "qmmm_density_gradient": (c_int, [c_void_p, c_void_p, c_void_p]),
        "qmmm_forces": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
        "qmmm_get_info": (c_int, [c_void_p, P(QmmmInfo)]),
        "qmmm_nao": (c_int, [c_void_p]),
        "qmmm_get_potential": (c_int, [c_void_p, c_void_p]),
        "qmmm_last_timing": (c_int, [c_void_p, P(c_double)]),
        "qmmm_qm_images": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
        "qmmm_aspc_predict": (c_int, [c_int, P(c_void_p), ctypes.c_size_t, c_void_p, c_void_p]),
        "qmmm_selftest_bounded_wait": (c_int, [c_void_p]),
        "qmmm_octupole_error": (c_int, [c_void_p, c_void_p, c_double, c_double, c_int, c_void_p, c_void_p]),
        "qmmm_rcut_search": (c_int, [c_void_p, c_void_p, c_double, c_double, c_int, c_double, P(c_double),
                                     P(c_double)]),
        "qmmm_autotune": (c_int, [c_void_p, c_int]),
        "qmmm_get_tuning": (c_int, [c_void_p, c_int, P(c_int), P(c_int), P(c_double), P(c_int), P(c_double)]),
        "qmmm_set_tuning": (c_int, [c_void_p, c_int, P(c_int), P(c_double)]),
        "qmmm_batch_create": (c_int, [P(c_void_p), c_int, c_void_p, P(c_void_p)]),
        "qmmm_batch_run": (c_int, [c_void_p, P(c_void_p), P(c_void_p), P(c_void_p), P(c_void_p), P(c_void_p),
                                   P(c_void_p)]),
        "qmmm_batch_timing": (c_int, [c_void_p, P(c_double)]),
        "qmmm_batch_captures": (c_int, [c_void_p]),
        "qmmm_batch_counts": (c_int, [c_void_p, P(c_int), P(c_int), P(c_int)]),
        "qmmm_batch_destroy": (None, [c_void_p]),
        "qmmm_destroy": (None, [c_void_p]),
        "qmmm_strerror": (ctypes.c_char_p, [c_int]),
        "qmmm_last_error": (ctypes.c_char_p, []),
        "qmmm_nuclear_mm_energy_static": (c_int, [c_int, c_void_p, c_void_p, c_int, c_void_p, c_void_p, c_void_p,
                                                  c_void_p]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _L = L
    return L


def _ptr(x):
    """Address of a float64 C-contiguous numpy array or torch tensor (host or device); None -> NULL."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        if x.dtype != np.float64 or not x.flags["C_CONTIGUOUS"]:
            raise TypeError("arrays must be float64 and C-contiguous")
        return c_void_p(x.ctypes.data)
    try:
        import torch
    except ImportError:  # pragma: no cover
        torch = None
    if torch is not None and isinstance(x, torch.Tensor):
        if x.dtype != torch.float64 or not x.is_contiguous():
            raise TypeError("tensors must be float64 and contiguous")
        return c_void_p(x.data_ptr())
    raise TypeError(f"unsupported array type {type(x)}")


def _check(rc, where):
    if rc != 0:
        raise QMMMError(rc, where)


def _out(x, shape, like):
    if x is not None:
        return x
    if like is not None and not isinstance(like, np.ndarray):
        import torch
        return torch.empty(shape, dtype=torch.float64, device=like.device)
    return np.empty(shape)


# ------------------------------------------------------------------------------------------------
# entry points (names of the C ABI)
# ------------------------------------------------------------------------------------------------

def qmmm_create(atom_xyz, atom_Z, shell_atom, shell_l, shell_nprim, shell_prim_offset, prim_exp, prim_coeff,
                mm_xyz, mm_q, mm_sigma, box, cutoff, ewald_alpha, precision=QMMM_FP64, screen_tol=-1.0,
                ewald_rcut=0.0, kmax=(0, 0, 0)):
    """Create a handle from host arrays (numpy); returns the opaque handle (int)."""
    L = load()
    atom_xyz = np.asarray(atom_xyz, dtype=np.float64).reshape(-1, 3)
    natm = len(atom_xyz)
    atoms = (QmmmAtom * natm)()
    for j in range(natm):
        atoms[j].xyz[:] = [float(v) for v in atom_xyz[j]]
        atoms[j].Z = float(atom_Z[j])
    nshell = len(shell_l)
    shells = (QmmmShell * nshell)()
    for s in range(nshell):
        shells[s].atom, shells[s].l = int(shell_atom[s]), int(shell_l[s])
        shells[s].nprim, shells[s].prim_offset = int(shell_nprim[s]), int(shell_prim_offset[s])
    nprim = len(prim_exp)
    prims = (QmmmPrimitive * nprim)()
    for k in range(nprim):
        prims[k].exponent, prims[k].coeff = float(prim_exp[k]), float(prim_coeff[k])
    mm_xyz = np.asarray(mm_xyz, dtype=np.float64).reshape(-1, 3)
    nmm = len(mm_xyz)
    chg = (QmmmCharge * max(nmm, 1))()
    for i in range(nmm):
        chg[i].xyz[:] = [float(v) for v in mm_xyz[i]]
        chg[i].q, chg[i].sigma = float(mm_q[i]), float(mm_sigma[i])
    opts = QmmmOptions()
    opts.precision, opts.screen_tol, opts.region_mode = int(precision), float(screen_tol), 0
    opts.ewald_rcut = float(ewald_rcut)
    opts.kmax[:] = [int(k) for k in kmax]
    opts.full_cell_test = 0
    bx = (c_double * 3)(*[float(b) for b in box])
    h = c_void_p()
    _check(L.qmmm_create(atoms, natm, shells, nshell, prims, nprim, chg, nmm, bx, float(cutoff), float(ewald_alpha),
                         ctypes.byref(opts), ctypes.byref(h)), "qmmm_create")
    return h.value


def qmmm_set_stream(h, stream):
    """stream: a torch.cuda.Stream, an integer cudaStream_t, or None (legacy stream)."""
    s = getattr(stream, "cuda_stream", stream)
    _check(load().qmmm_set_stream(h, c_void_p(s) if s else None), "qmmm_set_stream")


def qmmm_set_precision(h, precision):
    _check(load().qmmm_set_precision(h, int(precision)), "qmmm_set_precision")


QMMM_RECIP_CUDA_CORES, QMMM_RECIP_TENSOR, QMMM_RECIP_AUTO = 0, 1, 2


def qmmm_set_recip_method(h, method):
    _check(load().qmmm_set_recip_method(h, int(method)), "qmmm_set_recip_method")


def qmmm_set_positions(h, qm_xyz, mm_xyz, mm_q=None):
    _check(load().qmmm_set_positions(h, _ptr(qm_xyz), _ptr(mm_xyz), _ptr(mm_q)), "qmmm_set_positions")


def qmmm_nao(h):
    return load().qmmm_nao(h)


def qmmm_get_info(h):
    info = QmmmInfo()
    _check(load().qmmm_get_info(h, ctypes.byref(info)), "qmmm_get_info")
    out = {}
    for f, _ in QmmmInfo._fields_:
        v = getattr(info, f)
        out[f] = list(v) if f.endswith("_class") else v
    return out


def qmmm_vpot(h, V=None, E_nuc_mm=None, like=None):
    """Region-I V (nao x nao) and the nuclear-MM energy; returns (V, E_nuc_mm)."""
    n = qmmm_nao(h)
    V = _out(V, (n, n), like)
    E = _out(E_nuc_mm, (1,), like)
    _check(load().qmmm_vpot(h, _ptr(V), _ptr(E)), "qmmm_vpot")
    return V, E


def qmmm_ewald(h, dm, E_II=None, multipoles=None, F_II=None, want_F=False):
    info = qmmm_get_info(h)
    E = _out(E_II, (1,), dm)
    M = _out(multipoles, (info["natm"], 10), dm)
    F = F_II if F_II is not None else (_out(None, (info["nao"], info["nao"]), dm) if want_F else None)
    _check(load().qmmm_ewald(h, _ptr(dm), _ptr(E), _ptr(M), _ptr(F)), "qmmm_ewald")
    return E, M, F


def qmmm_density_gradient(h, dm, G=None):
    """G = dE/dgamma = V + F_II (the embedding's Fock contribution, Eqs. 11-14)."""
    info = qmmm_get_info(h)
    G = _out(G, (info["nao"], info["nao"]), dm)
    _check(load().qmmm_density_gradient(h, _ptr(dm), _ptr(G)), "qmmm_density_gradient")
    return G


def qmmm_energy(h, dm, E=None):
    """E = [E_total, E_I_elec, E_nuc_mm, E_II]."""
    E = _out(E, (4,), dm)
    _check(load().qmmm_energy(h, _ptr(dm), _ptr(E)), "qmmm_energy")
    return E


def qmmm_forces(h, dm, dE_dRqm=None, dE_dRmm=None, dE_dq=None):
    info = qmmm_get_info(h)
    gq = _out(dE_dRqm, (info["natm"], 3), dm)
    gm = _out(dE_dRmm, (max(info["nmm"], 0), 3), dm)
    gc = _out(dE_dq, (max(info["nmm"], 0),), dm)
    _check(load().qmmm_forces(h, _ptr(dm), _ptr(gq), _ptr(gm), _ptr(gc)), "qmmm_forces")
    return gq, gm, gc


def qmmm_get_potential(h, v=None, like=None):
    info = qmmm_get_info(h)
    v = _out(v, (info["natm"], 20), like)
    _check(load().qmmm_get_potential(h, _ptr(v)), "qmmm_get_potential")
    return v


def qmmm_last_timing(h):
    out = (c_double * 2)()
    load().qmmm_last_timing(h, out)
    return float(out[0]), float(out[1])


def qmmm_selftest_bounded_wait(stream=None):
    """Return code of the failure-path self-test (QMMM_ERR_TIMEOUT = -4 when it works)."""
    st = stream.cuda_stream if hasattr(stream, "cuda_stream") else stream
    return int(load().qmmm_selftest_bounded_wait(st))


def qmmm_aspc_predict(history, out=None, stream=None):
    """ASPC-predicted density from device tensors history[0] (most recent) .. history[K]."""
    n = history[0].numel()
    out = history[0].new_empty(history[0].shape) if out is None else out
    arr = (c_void_p * len(history))(*[_ptr(x) for x in history])
    st = stream.cuda_stream if hasattr(stream, "cuda_stream") else stream
    _check(load().qmmm_aspc_predict(len(history), arr, n, _ptr(out), st), "qmmm_aspc_predict")
    return out


def qmmm_qm_images(h, dm, want_F=False):
    """QM-QM periodic-image energy, its gradient dE/dR_QM and (optionally) its Fock matrix."""
    info = qmmm_get_info(h)
    E = _out(None, (1,), dm)
    g = _out(None, (info["natm"], 3), dm)
    F = _out(None, (info["nao"], info["nao"]), dm) if want_F else None
    _check(load().qmmm_qm_images(h, _ptr(dm), _ptr(E), _ptr(g), _ptr(F)), "qmmm_qm_images")
    return E, g, F


def qmmm_octupole_error(h, dm, r_lo, dr, n, err=None, octupoles=None, want_octupoles=False):
    """Err(R_k), R_k = r_lo + k dr (bohr), and optionally the Mulliken octupoles (natm x 10)."""
    info = qmmm_get_info(h)
    err = _out(err, (int(n),), dm)
    if want_octupoles:
        octupoles = _out(octupoles, (info["natm"], 10), dm)
    _check(load().qmmm_octupole_error(h, _ptr(dm), float(r_lo), float(dr), int(n), _ptr(err), _ptr(octupoles)),
           "qmmm_octupole_error")
    return (err, octupoles) if want_octupoles else err


def qmmm_rcut_search(h, dm, r_lo, dr, n, eps):
    """(smallest R_k with |Err| < eps or -1, Err there)."""
    r, e = c_double(), c_double()
    _check(load().qmmm_rcut_search(h, _ptr(dm), float(r_lo), float(dr), int(n), float(eps), ctypes.byref(r),
                                   ctypes.byref(e)), "qmmm_rcut_search")
    return r.value, e.value


QMMM_TUNE_V, QMMM_TUNE_FORCES, QMMM_TUNE_BOTH_PRECISIONS = 1, 2, 4
SWEEP_KINDS = ("vpot_f64", "vpot_mixed", "vgrad_f64", "vgrad_mixed")
CLASSES = ((0, 0), (1, 0), (1, 1), (2, 0), (2, 1), (2, 2), (3, 0), (3, 1), (3, 2), (3, 3))


def qmmm_autotune(h, flags=0):
    _check(load().qmmm_autotune(h, int(flags)), "qmmm_autotune")


def qmmm_get_tuning(h, kind):
    """Sweep configuration of one kind (index into SWEEP_KINDS): tuned flag and, per angular class,
    threads per block, SM share, the measured time alone (ms), the wide block size (0: none) and the
    SM-time weight per primitive pair (accepted back by qmmm_set_tuning)."""
    th, sh, ms, wd, wt = (c_int * 10)(), (c_int * 10)(), (c_double * 10)(), (c_int * 10)(), (c_double * 10)()
    rc = load().qmmm_get_tuning(h, int(kind), th, sh, ms, wd, wt)
    _check(min(rc, 0), "qmmm_get_tuning")
    return {"tuned": bool(rc), "threads": list(th), "share": list(sh), "ms": list(ms), "wide": list(wd),
            "weight": list(wt)}


def qmmm_set_tuning(h, kind, threads, weight=None):
    th = (c_int * 10)(*[int(t) for t in threads])
    w = (c_double * 10)(*[float(x) for x in weight]) if weight is not None else None
    _check(load().qmmm_set_tuning(h, int(kind), th, w), "qmmm_set_tuning")


def qmmm_batch_create(handles, stream=None):
    arr = (c_void_p * len(handles))(*handles)
    out = c_void_p()
    st = stream.cuda_stream if hasattr(stream, "cuda_stream") else stream
    _check(load().qmmm_batch_create(arr, len(handles), st, ctypes.byref(out)), "qmmm_batch_create")
    return out.value


def _ptr_array(xs, n):
    if xs is None:
        return None
    return (c_void_p * n)(*[_ptr(x) for x in xs])


def qmmm_batch_run(b, dm, V=None, E=None, dE_dRqm=None, dE_dRmm=None, dE_dq=None):
    """dm and each output: a list with one DEVICE tensor (float64, contiguous) per frame, or None."""
    n = len(dm)
    _check(load().qmmm_batch_run(b, _ptr_array(dm, n), _ptr_array(V, n), _ptr_array(E, n), _ptr_array(dE_dRqm, n),
                                 _ptr_array(dE_dRmm, n), _ptr_array(dE_dq, n)), "qmmm_batch_run")


def qmmm_batch_timing(b, nframes):
    out = (c_double * (nframes + 1))()
    load().qmmm_batch_timing(b, out)
    return float(out[0]), [float(x) for x in out[1:]]


def qmmm_batch_captures(b):
    return int(load().qmmm_batch_captures(b))


def qmmm_batch_counts(b):
    """(recordings, instantiations, in-place updates) of the batch graph."""
    r, i, u = c_int(), c_int(), c_int()
    _check(load().qmmm_batch_counts(b, ctypes.byref(r), ctypes.byref(i), ctypes.byref(u)), "qmmm_batch_counts")
    return r.value, i.value, u.value


def qmmm_batch_destroy(b):
    if b:
        load().qmmm_batch_destroy(b)


def qmmm_destroy(h):
    if h:
        load().qmmm_destroy(h)


def qmmm_strerror(code):
    return load().qmmm_strerror(int(code)).decode()


def qmmm_last_error():
    return load().qmmm_last_error().decode()


def qmmm_nuclear_mm_energy_static(qm_xyz, Z, charges, sigma, E, stream=None):
    """Allocation-free nuclear-MM energy for callers that cannot allocate device memory while
    they run: every argument is a CUDA float64 tensor the caller owns (qm_xyz[natm,3], Z[natm],
    charges[n,4] = x, y, z, q, sigma[n], E[1]); work is queued on ``stream`` and not waited for."""
    s = getattr(stream, "cuda_stream", stream)
    natm = int(qm_xyz.shape[0])
    n = int(charges.shape[0])
    _check(load().qmmm_nuclear_mm_energy_static(natm, _ptr(qm_xyz), _ptr(Z), n, _ptr(charges), _ptr(sigma), _ptr(E),
                                                c_void_p(s) if s else None), "qmmm_nuclear_mm_energy_static")
    return E
