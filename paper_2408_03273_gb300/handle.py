"""Handle wrapper and the autograd Function over the C ABI (marshalling only).

``QMMMEnergy.apply(handle, dm, qm_xyz, mm_xyz, mm_q)`` returns E_QM-MM at fixed density
(Eq. 9 region-I term + nuclear-MM term + region-II multipole terms of Eq. 6/Eq. 10).  Its
backward calls ``qmmm_forces`` -- the hand-written adjoint kernels, which recompute the Boys
R-tensors instead of storing them -- and, when the density needs a gradient, returns
dE/dgamma = V + F_II (Eqs. 11-14).  PyTorch provides device memory and the stream only.
"""
from __future__ import annotations

from . import _lib as L


class Handle:
    """One library handle built from a workload (see ``workloads.System``): lengths in bohr."""

    def __init__(self, s, precision: int = L.QMMM_FP64, screen_tol: float = -1.0):
        self.system = s
        self.h = L.qmmm_create(s.atom_xyz, s.atom_Z, s.shell_atom, s.shell_l, s.shell_nprim, s.shell_prim_offset,
                               s.prim_exp, s.prim_coeff, s.mm_xyz, s.mm_q, s.mm_sigma, s.box, s.cutoff,
                               s.ewald_alpha, precision=precision, screen_tol=screen_tol,
                               ewald_rcut=s.ewald_rcut, kmax=s.kmax)
        self.info = L.qmmm_get_info(self.h)

    # -- marshalling -------------------------------------------------------------------------
    def set_stream(self, stream):
        L.qmmm_set_stream(self.h, stream)

    def set_precision(self, precision: int):
        L.qmmm_set_precision(self.h, precision)
        self.info = L.qmmm_get_info(self.h)

    def set_recip_method(self, method: int):
        """QMMM_RECIP_CUDA_CORES, QMMM_RECIP_TENSOR (structure factor on the tensor cores) or
        QMMM_RECIP_AUTO (tensor cores for the mixed path)."""
        L.qmmm_set_recip_method(self.h, method)

    def set_positions(self, qm_xyz, mm_xyz, mm_q=None):
        L.qmmm_set_positions(self.h, qm_xyz, mm_xyz, mm_q)
        self.info = L.qmmm_get_info(self.h)

    def vpot(self, V=None, E_nuc_mm=None, like=None):
        return L.qmmm_vpot(self.h, V, E_nuc_mm, like=like)

    def ewald(self, dm, want_F=False):
        return L.qmmm_ewald(self.h, dm, want_F=want_F)

    def energy(self, dm, E=None):
        return L.qmmm_energy(self.h, dm, E)

    def density_gradient(self, dm, G=None):
        """dE/dgamma = V + F_II (needs vpot at the current geometry)."""
        return L.qmmm_density_gradient(self.h, dm, G)

    def forces(self, dm, dE_dRqm=None, dE_dRmm=None, dE_dq=None):
        return L.qmmm_forces(self.h, dm, dE_dRqm, dE_dRmm, dE_dq)

    def potential(self, like=None):
        return L.qmmm_get_potential(self.h, like=like)

    def qm_images(self, dm, want_F=False):
        return L.qmmm_qm_images(self.h, dm, want_F=want_F)

    def octupole_error(self, dm, r_lo, dr, n, want_octupoles=False):
        return L.qmmm_octupole_error(self.h, dm, r_lo, dr, n, want_octupoles=want_octupoles)

    def rcut_search(self, dm, r_lo, dr, n, eps):
        return L.qmmm_rcut_search(self.h, dm, r_lo, dr, n, eps)

    def autotune(self, flags: int = 0):
        """Time the region-I class sweeps on this geometry and keep the fastest block shapes and SM
        split (flags: QMMM_TUNE_V / QMMM_TUNE_FORCES / QMMM_TUNE_BOTH_PRECISIONS; 0 = V and forces
        at the current precision)."""
        L.qmmm_autotune(self.h, flags)

    def tuning(self, kind: int):
        return L.qmmm_get_tuning(self.h, kind)

    def set_tuning(self, kind: int, threads, weight=None):
        L.qmmm_set_tuning(self.h, kind, threads, weight)

    def last_timing(self):
        return L.qmmm_last_timing(self.h)

    def close(self):
        if self.h:
            L.qmmm_destroy(self.h)
            self.h = None

    def __del__(self):  # pragma: no cover - interpreter shutdown order
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Several frames (Handles) evaluated together through one recorded CUDA graph: per frame V,
    E[4] and the gradient at that frame's density (see qmmm_batch_run)."""

    def __init__(self, handles, stream=None):
        self.handles = list(handles)  # kept alive: the batch borrows the library handles
        self.b = L.qmmm_batch_create([h.h for h in self.handles], stream)

    def run(self, dm, V=None, E=None, dE_dRqm=None, dE_dRmm=None, dE_dq=None):
        L.qmmm_batch_run(self.b, dm, V, E, dE_dRqm, dE_dRmm, dE_dq)

    def timing(self):
        """(ms of the last run, [ms at which each frame finished])."""
        return L.qmmm_batch_timing(self.b, len(self.handles))

    def captures(self):
        return L.qmmm_batch_captures(self.b)

    def counts(self):
        """(recordings, instantiations, in-place updates)."""
        return L.qmmm_batch_counts(self.b)

    def close(self):
        if self.b:
            L.qmmm_batch_destroy(self.b)
            self.b = None

    def __del__(self):  # pragma: no cover - interpreter shutdown order
        try:
            self.close()
        except Exception:
            pass


def _autograd_function():
    import torch

    class QMMMEnergy(torch.autograd.Function):
        """E_QM-MM(dm, R_QM, R_MM, q) with a hand-written adjoint kernel as backward.

        The backward uses the handle's state from the forward: do not move the handle to another
        geometry between forward and backward."""

        @staticmethod
        def forward(ctx, handle, dm, qm_xyz, mm_xyz, mm_q):
            h = handle.h
            L.qmmm_set_stream(h, torch.cuda.current_stream())
            L.qmmm_set_positions(h, qm_xyz.detach(), mm_xyz.detach(), mm_q.detach())
            L.qmmm_vpot(h, like=dm)  # V stays in the handle for the energy and dE/dgamma
            E = L.qmmm_energy(h, dm.detach())
            ctx.handle = handle
            ctx.save_for_backward(dm)
            return E[0].clone()

        @staticmethod
        def backward(ctx, gE):
            (dm,) = ctx.saved_tensors
            h = ctx.handle.h
            L.qmmm_set_stream(h, torch.cuda.current_stream())
            gq, gm, gc = L.qmmm_forces(h, dm.detach())
            gdm = None
            if ctx.needs_input_grad[1]:
                gdm = gE * L.qmmm_density_gradient(h, dm.detach())  # V + F_II, formed in the library
            return None, gdm, gE * gq, gE * gm, gE * gc

    return QMMMEnergy


class _Lazy:
    _cls = None

    def __getattr__(self, name):
        if _Lazy._cls is None:
            _Lazy._cls = _autograd_function()
        return getattr(_Lazy._cls, name)


QMMMEnergy = _Lazy()
