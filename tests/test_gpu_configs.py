"""GPU path on the named workloads:

* QM water in 216 MM waters (18.6 A box, sigma 0.2 A, cutoff 9 A, alpha 0.35 A^-1, kmax 7):
  full element-by-element parity of V, energy terms, multipoles, potential and every gradient,
  FP64 and mixed precision;
* the same inputs through the torch.autograd.Function (hand-written adjoint as backward),
  checked against the oracle gradient and against central finite differences (h = 1e-4 bohr)
  of the GPU energy on 32 seeded coordinates;
* the 60-atom active site in 60000 MM charges (58 A box, cutoff 12 A, alpha 0.3 A^-1, kmax 16),
  at full size in the launch configuration the benchmark times: sampled V blocks and sampled
  MM-charge derivatives against the oracle, the full potential and multipoles against the
  oracle, and size-independent invariants (zero net force, linearity in the MM charges)."""
import numpy as np
import pytest

import oracle
import workloads
from _gpuutil import TOL_FP64, TOL_MIXED, check_V, energy_scale, gpu_all, raw_err, rel_fro, rel_max

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def c1():
    s = workloads.config1_water()
    ref = oracle.energy(s)
    ref.update(oracle.forces(s))
    return s, ref


@pytest.mark.parametrize("precision", [0, 1])
def test_config1_full_parity(c1, precision):
    s, ref = c1
    g = gpu_all(s, precision=precision)
    tol = TOL_FP64 if precision == 0 else TOL_MIXED
    check_V(g["V"], ref["V"], precision)
    assert rel_fro(g["V"], ref["V"]) < tol
    sc = energy_scale(ref)
    assert abs(g["E"] - ref["E"]) < tol * sc
    assert abs(g["E_nuc_mm"] - ref["E_nuc_mm"]) < TOL_FP64 * sc
    assert abs(g["E_II"] - ref["E_II"]) < TOL_FP64 * sc
    assert rel_max(g["M"], ref["M"]) < TOL_FP64
    assert rel_max(g["phi"], ref["phi"]) < TOL_FP64
    for k in ("dE_dRqm", "dE_dRmm", "dE_dq"):
        assert raw_err(g[k], ref[k]) < tol, k  # raw: relative to the largest value of the gradient


def _cuda(a):
    import torch
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def test_config3_autograd_against_oracle(c1):
    import torch

    import paper_2408_03273_gb300 as q
    s, ref = c1
    h = q.Handle(s)
    dm = _cuda(s.dm).requires_grad_(True)
    qm = _cuda(s.atom_xyz).requires_grad_(True)
    mm = _cuda(s.mm_xyz).requires_grad_(True)
    mq = _cuda(s.mm_q).requires_grad_(True)
    E = q.QMMMEnergy.apply(h, dm, qm, mm, mq)
    E.backward()
    torch.cuda.synchronize()
    assert abs(E.item() - ref["E"]) < TOL_FP64 * energy_scale(ref)
    assert rel_max(qm.grad.cpu().numpy(), ref["dE_dRqm"]) < TOL_FP64
    assert rel_max(mm.grad.cpu().numpy(), ref["dE_dRmm"]) < TOL_FP64
    assert rel_max(mq.grad.cpu().numpy(), ref["dE_dq"]) < TOL_FP64
    # dE/dgamma = V + F_II (Eqs. 11-14)
    Fii = oracle.fock_ii(s, ref["phi"])
    assert rel_max(dm.grad.cpu().numpy(), ref["V"] + Fii) < TOL_FP64
    h.close()


def _crosses_cutoff(s, which, idx, axis, h):
    """True if moving this coordinate by +-h moves any QM-MM image pair across the Ewald
    real-space cutoff (a jump of the truncated sum) or changes region-I membership."""
    rc = oracle.ewald_rc(s)
    t_p, t_m = s.copy(), s.copy()
    for t, d in ((t_p, h), (t_m, -h)):
        arr = getattr(t, which).copy()
        arr[idx, axis] += d
        setattr(t, which, arr)
    r0 = oracle.region1(s)[0]
    if not (np.array_equal(oracle.region1(t_p)[0], r0) and np.array_equal(oracle.region1(t_m)[0], r0)):
        return True
    for t in (t_p, t_m):
        d = t.atom_xyz[:, None, :] - t.mm_xyz[None, :, :]
        d -= np.rint(d / t.box) * t.box
        r = np.linalg.norm(d, axis=-1)
        d0 = s.atom_xyz[:, None, :] - s.mm_xyz[None, :, :]
        d0 -= np.rint(d0 / s.box) * s.box
        r0_ = np.linalg.norm(d0, axis=-1)
        if np.any((r < rc) != (r0_ < rc)):
            return True
    return False


def test_config3_finite_differences(c1):
    import paper_2408_03273_gb300 as q
    s, ref = c1
    h_ = 1e-4
    rng = np.random.default_rng(workloads.SEED_BASE + 3)
    coords = [("atom_xyz", j, x) for j in range(s.natm) for x in range(3)]
    coords += [("mm_xyz", int(i), int(x)) for i, x in zip(rng.choice(s.nmm, 40, replace=False), rng.integers(0, 3, 40))]
    picked = [coords[k] for k in rng.permutation(len(coords))][:32]
    handle = q.Handle(s)

    def energy(t):
        handle.set_positions(np.ascontiguousarray(t.atom_xyz), np.ascontiguousarray(t.mm_xyz), None)
        handle.vpot()
        return float(handle.energy(t.dm)[0])

    handle.vpot()
    gq, gm, _ = handle.forces(s.dm)
    checked = 0
    for which, i, x in picked:
        if _crosses_cutoff(s, which, i, x, h_):
            continue
        vals = []
        for d in (h_, -h_):
            t = s.copy()
            arr = getattr(t, which).copy()
            arr[i, x] += d
            setattr(t, which, arr)
            vals.append(energy(t))
        fd = (vals[0] - vals[1]) / (2 * h_)
        an = gq[i, x] if which == "atom_xyz" else gm[i, x]
        scale = max(np.max(np.abs(gq)), np.max(np.abs(gm)))
        assert abs(fd - an) < 1e-6 * scale, (which, i, x, fd, an)
        checked += 1
    assert checked >= 24
    handle.close()


@pytest.fixture(scope="module")
def c2():
    return workloads.config2_active_site()


@pytest.fixture(scope="module")
def c2_gpu(c2):
    return {p: gpu_all(c2, precision=p) for p in (0, 1)}


def test_config2_counts(c2, c2_gpu):
    info = c2_gpu[0]["info"]
    assert info["nao"] == 1560 and info["nshell"] == 600
    assert info["n_region1"] == len(oracle.region1(c2)[0])
    assert info["n_gvec"] == (33 ** 3 - 1) // 2


@pytest.mark.parametrize("precision", [0, 1])
def test_config2_sampled_V_blocks(c2, c2_gpu, precision):
    s = c2
    rng = np.random.default_rng(7)
    off = np.concatenate([[0], np.cumsum([(l + 1) * (l + 2) // 2 for l in s.shell_l])])
    # sample shell pairs of every angular class
    pairs = []
    for la in range(3):
        for lb in range(la + 1):
            A = np.flatnonzero(s.shell_l == la)
            B = np.flatnonzero(s.shell_l == lb)
            for _ in range(6):
                pairs.append((int(rng.choice(A)), int(rng.choice(B))))
    V = c2_gpu[precision]["V"]
    Vref = oracle.vpot(s, pairs=pairs)
    blocks_ref = np.concatenate([Vref[off[a]:off[a + 1], off[b]:off[b + 1]].ravel() for a, b in pairs])
    blocks_got = np.concatenate([V[off[a]:off[a + 1], off[b]:off[b + 1]].ravel() for a, b in pairs])
    tol = TOL_FP64 if precision == 0 else TOL_MIXED
    # elementwise against the largest V element of the whole matrix
    assert np.max(np.abs(blocks_got - blocks_ref)) < tol * np.max(np.abs(V))


def test_config2_mixed_vs_fp64_frobenius(c2_gpu):
    # the FP64 GPU path is oracle-exact on every element checked; the mixed path's whole-matrix
    # error is measured against it
    assert rel_fro(c2_gpu[1]["V"], c2_gpu[0]["V"]) < TOL_MIXED
    for k in ("dE_dRqm", "dE_dRmm", "dE_dq"):
        assert rel_max(c2_gpu[1][k], c2_gpu[0][k]) < TOL_MIXED, k


def test_config2_potential_and_multipoles(c2, c2_gpu):
    g = c2_gpu[0]
    assert rel_max(g["phi"], oracle.ewald_phi(c2)) < TOL_FP64
    assert rel_max(g["M"], oracle.multipoles(c2)) < TOL_FP64


def test_config2_sampled_charge_derivatives(c2, c2_gpu):
    s = c2
    idx = oracle.region1(s)[0]
    rng = np.random.default_rng(11)
    sub = np.sort(rng.choice(len(idx), 3, replace=False))
    mm = idx[sub]
    ref = oracle.forces(s, charge_subset=sub, mm_subset=mm)
    for p, tol in ((0, TOL_FP64), (1, TOL_MIXED)):
        g = c2_gpu[p]
        assert rel_max(g["dE_dq"][mm], ref["dE_dq"][mm]) < tol
        assert rel_max(g["dE_dRmm"][mm], ref["dE_dRmm"][mm]) < tol


def test_config2_invariants(c2, c2_gpu):
    for p in (0, 1):
        g = c2_gpu[p]
        tot = g["dE_dRqm"].sum(0) + g["dE_dRmm"].sum(0)
        assert np.max(np.abs(tot)) < (1e-9 if p == 0 else 1e-6) * np.max(np.abs(g["dE_dRqm"]))
        sc = abs(g["E_I_elec"]) + abs(g["E_nuc_mm"]) + abs(g["E_II"])
        assert abs(np.dot(c2.mm_q, g["dE_dq"]) - g["E"]) < (1e-11 if p == 0 else 1e-6) * sc
