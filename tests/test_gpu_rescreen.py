"""Screening that follows the geometry: the primitive-pair list is screened with a displacement
margin and planned again once a QM atom has moved farther than that margin, so an MD run in which
QM atoms approach keeps every pair that becomes significant.  Two QM atoms start 10 bohr apart with
exponents >= 1 bohr^-2 (their inter-atomic primitive pairs are screened out at 1e-14) and approach to
6 bohr over eight position updates of one handle (K_AB grows to ~1e-8), so the list is planned again on the way; V, the energy and every
gradient stay within 1e-10 of the unscreened FP64 oracle after every update."""
import numpy as np
import pytest

import oracle
import workloads
from _gpuutil import TOL_FP64, energy_scale, rel_max

pytestmark = pytest.mark.gpu


def _two_atoms(sep):
    s = workloads.small_system(seed=3101, n_atoms=2, lmax=1, nprim=(1, 2), n_waters=27, box_A=14.0, cutoff_A=6.0)
    rng = np.random.default_rng(3101)
    s.prim_exp = rng.uniform(1.0, 3.0, size=s.prim_exp.shape)
    c = s.atom_xyz.mean(axis=0)
    s.atom_xyz = np.ascontiguousarray(np.array([c - [sep / 2, 0, 0], c + [sep / 2, 0, 0]]))
    # keep the MM waters away from both QM atoms (whatever their separation below)
    line = lambda p: np.linalg.norm(np.cross(p - c, [1.0, 0.0, 0.0]), axis=-1)  # noqa: E731
    w = s.mm_xyz.reshape(-1, 3, 3)
    keep = np.all((line(w) > 4.0) | (np.abs((w - c)[..., 0]) > sep / 2 + 4.0), axis=1)
    s.mm_xyz = np.ascontiguousarray(w[keep].reshape(-1, 3))
    s.mm_q = np.ascontiguousarray(s.mm_q.reshape(-1, 3)[keep].ravel())
    s.mm_sigma = np.ascontiguousarray(s.mm_sigma.reshape(-1, 3)[keep].ravel())
    return s


def test_pair_list_follows_approaching_atoms():
    import paper_2408_03273_gb300 as q
    s = _two_atoms(10.0)
    h = q.Handle(s)
    try:
        n0 = h.info["n_prim_pairs"]
        c = s.atom_xyz.mean(axis=0)
        for sep in np.arange(9.5, 5.9, -0.5):
            t = s.copy()
            t.atom_xyz = np.ascontiguousarray(np.array([c - [sep / 2, 0, 0], c + [sep / 2, 0, 0]]))
            h.set_positions(t.atom_xyz, t.mm_xyz, t.mm_q)
            V, En = h.vpot()
            E = h.energy(t.dm)
            gq, gm, gc = h.forces(t.dm)
            ref = oracle.energy(t)
            ref.update(oracle.forces(t))
            assert rel_max(V, ref["V"]) < TOL_FP64, sep
            assert abs(E[0] - ref["E"]) < TOL_FP64 * energy_scale(ref), sep
            assert rel_max(gq, ref["dE_dRqm"]) < TOL_FP64, sep
            assert rel_max(gm, ref["dE_dRmm"]) < TOL_FP64, sep
            assert rel_max(gc, ref["dE_dq"]) < TOL_FP64, sep
        # the pairs between the two atoms joined the list on the way
        assert h.info["n_prim_pairs"] > n0
    finally:
        h.close()
