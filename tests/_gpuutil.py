"""Helpers for the GPU parity tests: build a handle from a workload and compare with the oracle."""
import numpy as np

# tolerances: the FP64 path against the FP64 oracle, and the mixed-precision path
TOL_FP64 = 1e-10
TOL_MIXED = 1e-6
# Mixed path, V element by element (relative to max |V|).  The mixed V is held to TOL_MIXED in
# the relative Frobenius norm; single elements are not: every per-charge term is an FP32 number,
# and the terms of a region-I sum cancel 20-40 fold (neutral waters), so rounding each term once
# to FP32 already leaves 2-5e-7 of max |V| in the s-s elements (CPU emulation with exact F_0), and
# the Hermite recursion adds a small factor for f functions.
TOL_MIXED_ELEM = 3e-6


def check_V(got, ref, precision):
    """V parity: FP64 element by element; mixed in the Frobenius norm plus the element bound."""
    if precision == 0:
        assert rel_max(got, ref) < TOL_FP64
    else:
        assert rel_fro(got, ref) < TOL_MIXED
        assert rel_max(got, ref) < TOL_MIXED_ELEM


def rel_max(got, ref):
    """max |got - ref| / max |ref| (elementwise parity scaled by the largest reference value)."""
    got, ref = np.asarray(got), np.asarray(ref)
    return float(np.max(np.abs(got - ref)) / max(np.max(np.abs(ref)), 1e-300))


def rel_fro(got, ref):
    got, ref = np.asarray(got), np.asarray(ref)
    return float(np.linalg.norm(got - ref) / max(np.linalg.norm(ref), 1e-300))


def energy_scale(e):
    return abs(e["E_I_elec"]) + abs(e["E_nuc_mm"]) + abs(e["E_II"])


def raw_err(got, ref):
    """The raw gradient error: max |got - ref| / max |ref| over the whole array."""
    got, ref = np.asarray(got), np.asarray(ref)
    return float(np.max(np.abs(got - ref)) / max(np.max(np.abs(ref)), 1e-300))


def grad_err(got, ref, key, mixed):
    """Elementwise gradient error on the small stress systems (a few atoms and waters).  FP64 path:
    the raw error.  Mixed path: relative to the larger of the largest reference component and the
    largest component of the region-I electronic term alone -- the only term evaluated in FP32,
    which on these tiny systems nearly cancels against the FP64 nuclear-MM term, so the residual
    total amplifies FP32 rounding by the cancellation ratio (the same normalisation as the
    energy, whose scale is the sum of the magnitudes of its terms).  The named workloads (water,
    active sites, frames) are held to the raw error instead (raw_err)."""
    scale = float(np.max(np.abs(ref[key])))
    if mixed and "elec" in ref:
        scale = max(scale, float(np.max(np.abs(ref["elec"][key]))))
    return float(np.max(np.abs(np.asarray(got) - ref[key]))) / max(scale, 1e-300)


def gpu_all(s, precision=0, screen_tol=-1.0, setup=None):
    """Run the whole path through the C ABI on host arrays; returns a dict like the oracle's.
    setup(handle), if given, runs right after the handle is created (e.g. a sweep configuration)."""
    import paper_2408_03273_gb300 as q
    h = q.Handle(s, precision=precision, screen_tol=screen_tol)
    try:
        if setup is not None:
            setup(h)
        V, En = h.vpot()
        E = h.energy(s.dm)
        EII, M, F = h.ewald(s.dm, want_F=True)
        phi = h.potential()
        gq, gm, gc = h.forces(s.dm)
        return {"V": V, "E_nuc_mm": float(En[0]), "E": float(E[0]), "E_I_elec": float(E[1]), "E_II": float(E[3]),
                "M": M, "F": F, "phi": phi, "dE_dRqm": gq, "dE_dRmm": gm, "dE_dq": gc, "info": h.info,
                "timing": h.last_timing()}
    finally:
        h.close()
