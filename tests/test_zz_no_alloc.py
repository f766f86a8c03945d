"""The allocation-free nuclear-MM energy entry point.

Some callers cannot allocate device memory while they run -- an MD engine that reserves all its
device memory at start-up and calls the embedding from inside its time step (a cudaMalloc there
would implicitly synchronise the device), or a plugin whose memory belongs to the host program's
pool allocator.  qmmm_nuclear_mm_energy_static serves them: it takes only caller-owned device
arrays and keeps its scratch in a fixed array inside the library.  Here its result is compared,
through the C ABI and on two calls in a row, with the E_nuc_mm that qmmm_vpot returns for the
same charges and with the FP64 CPU oracle's sum.  This file is collected last on purpose."""
import numpy as np
import pytest

import oracle
import paper_2408_03273_gb300 as q
import workloads
from _gpuutil import TOL_FP64

pytestmark = pytest.mark.gpu


def _all_in_region1():
    # a 30 A box with a 13.5 A region-I radius: keep only waters whose three atoms lie within
    # 12 A of the QM centre, so every charge is in region I exactly once
    s = workloads.small_system(seed=4242, n_atoms=3, lmax=1, n_waters=2000, box_A=30.0, cutoff_A=13.5)
    c = s.atom_xyz.mean(axis=0)
    w = (s.mm_xyz - c).reshape(-1, 3, 3)
    keep = np.all(np.linalg.norm(w, axis=-1) < 12.0 / 0.52917721092, axis=1)
    s.mm_xyz = np.ascontiguousarray(w[keep].reshape(-1, 3) + c)
    s.mm_q = np.ascontiguousarray(s.mm_q.reshape(-1, 3)[keep].ravel())
    s.mm_sigma = np.ascontiguousarray(s.mm_sigma.reshape(-1, 3)[keep].ravel())
    s.mm_sigma[::7] = 0.0  # some point charges too
    return s


def test_static_scratch_energy_matches_handle_twice():
    import torch
    s = _all_in_region1()
    h = q.Handle(s)
    assert h.info["n_region1"] == s.nmm > 600
    _, En = h.vpot()
    ref = float(En[0])
    h.close()

    dev = torch.device("cuda")
    t = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device=dev)  # noqa: E731
    qm, Z = t(s.atom_xyz), t(s.atom_Z)
    chg = t(np.concatenate([s.mm_xyz, s.mm_q[:, None]], axis=1))
    sig = t(s.mm_sigma)
    E = torch.empty(1, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream()
    got = []
    for _ in range(2):
        E.fill_(float("nan"))
        q.qmmm_nuclear_mm_energy_static(qm, Z, chg, sig, E, stream)
        torch.cuda.synchronize()
        got.append(float(E.item()))
    # the same sum by the FP64 CPU oracle, over the same charges
    ora = oracle.enucmm(s, charges=(s.mm_xyz, s.mm_q, s.mm_sigma))
    assert abs(ref - ora) < TOL_FP64 * abs(ora), (ref, ora)
    for g in got:
        assert abs(g - ref) < TOL_FP64 * abs(ref), (g, ref)
        assert abs(g - ora) < TOL_FP64 * abs(ora), (g, ora)
    assert got[0] == got[1]


def test_static_scratch_gaussian_charge_on_a_nucleus():
    # a Gaussian charge centred exactly on a QM nucleus contributes its limit 2 Z q / (sigma sqrt(pi));
    # every other (nucleus, charge) pair is summed by the oracle as usual
    import torch
    s = workloads.small_system(seed=77, n_atoms=3, lmax=1, n_waters=4)
    xyz = np.array(s.mm_xyz)
    xyz[0] = s.atom_xyz[1]
    sig = np.full(len(s.mm_q), 0.3)
    dev = torch.device("cuda")
    t = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device=dev)  # noqa: E731
    E = torch.empty(1, dtype=torch.float64, device=dev)
    q.qmmm_nuclear_mm_energy_static(t(s.atom_xyz), t(s.atom_Z), t(np.concatenate([xyz, s.mm_q[:, None]], 1)),
                                    t(sig), E, torch.cuda.current_stream())
    torch.cuda.synchronize()
    rest = oracle.enucmm(s, charges=(xyz[1:], s.mm_q[1:], sig[1:]))
    others = s.copy()
    others.atom_xyz = np.ascontiguousarray(s.atom_xyz[[0, 2]])
    others.atom_Z = np.ascontiguousarray(s.atom_Z[[0, 2]])
    c0 = oracle.enucmm(others, charges=(xyz[:1], s.mm_q[:1], sig[:1]))
    limit = s.atom_Z[1] * s.mm_q[0] * 2.0 / (sig[0] * np.sqrt(np.pi))
    ref = rest + c0 + limit
    assert np.isfinite(E.item())
    assert abs(E.item() - ref) < 1e-12 * abs(ref), (E.item(), ref)


def test_static_scratch_rejects_oversize_and_host_memory():
    import torch
    dev = torch.device("cuda")
    qm = torch.zeros((1, 3), dtype=torch.float64, device=dev)
    Z = torch.ones(1, dtype=torch.float64, device=dev)
    E = torch.empty(1, dtype=torch.float64, device=dev)
    big = torch.zeros((262145, 4), dtype=torch.float64, device=dev)
    with pytest.raises(q.QMMMError) as ei:
        q.qmmm_nuclear_mm_energy_static(qm, Z, big, torch.zeros(262145, dtype=torch.float64, device=dev), E)
    assert ei.value.code == -1
    with pytest.raises(q.QMMMError):
        q.qmmm_nuclear_mm_energy_static(qm, Z, np.zeros((4, 4)), np.zeros(4), E)
