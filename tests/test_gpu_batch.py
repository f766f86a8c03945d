"""Batches of frames through one recorded CUDA graph (qmmm_batch_*): every frame's V, energy and
gradient against the same handle's plain calls, frames of the uneven-frames workload (water
clusters of 21 and 45 QM atoms in ~30000 MM charges) inside a recorded graph against the FP64
oracle, graph replay without re-recording, a position update between runs, and the argument
checks."""
import numpy as np
import pytest

import oracle
import workloads
from _gpuutil import TOL_FP64, TOL_MIXED, TOL_MIXED_ELEM, rel_fro

pytestmark = pytest.mark.gpu


def _frames():
    return [workloads.small_system(seed=120 + i, n_atoms=2 + i, lmax=2, nprim=(1, 3), n_waters=10 + 6 * i)
            for i in range(3)]


def _plain(h, s, dm):
    V, _ = h.vpot()
    E = h.energy(dm)
    gq, gm, gc = h.forces(dm)
    return {"V": V, "E": np.asarray(E), "gq": gq, "gm": gm, "gc": gc}


def _dev_outputs(torch, frames):
    dev = torch.device("cuda")
    z = lambda *shape: torch.zeros(shape, dtype=torch.float64, device=dev)  # noqa: E731
    return ([z(s.nao, s.nao) for s in frames], [z(4) for s in frames], [z(s.natm, 3) for s in frames],
            [z(s.nmm, 3) for s in frames], [z(s.nmm) for s in frames])


def _close(a, b, tol):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.max(np.abs(a - b))) <= tol * max(float(np.max(np.abs(b))), 1e-300)


@pytest.fixture(scope="module")
def c5_pair():
    # two frames of the uneven-frames workload (QM water clusters of 21 and 45 atoms, 30666 and
    # 26658 MM charges), with the oracle's V, energy, QM gradient and three sampled MM charges
    frames = workloads.config5_frames(64)
    out = []
    for f in (53, 63):
        s = frames[f]
        idx = oracle.region1(s)[0]
        rng = np.random.default_rng(500 + f)
        mm = idx[np.sort(rng.choice(len(idx), 3, replace=False))]
        ref = oracle.energy(s)
        ref.update(oracle.forces(s, mm_subset=mm))
        out.append((s, mm, ref))
    return out


@pytest.mark.parametrize("precision", [0, 1])
def test_batch_frames_against_oracle(c5_pair, precision):
    torch = pytest.importorskip("torch")
    import paper_2408_03273_gb300 as q
    frames = [s for s, _, _ in c5_pair]
    hs = [q.Handle(s, precision=precision) for s in frames]
    try:
        dev = torch.device("cuda")
        dm = [torch.as_tensor(s.dm, device=dev) for s in frames]
        V, E, gq, gm, gc = _dev_outputs(torch, frames)
        b = q.Batch(hs)
        try:
            for _ in range(2):  # the recording run, then a graph replay
                b.run(dm, V, E, gq, gm, gc)
            assert b.captures() == 1
        finally:
            b.close()
        for i, (s, mm, ref) in enumerate(c5_pair):
            Vi, Ei = V[i].cpu().numpy(), E[i].cpu().numpy()
            sc = abs(ref["E_I_elec"]) + abs(ref["E_nuc_mm"]) + abs(ref["E_II"])
            if precision == 0:
                assert np.max(np.abs(Vi - ref["V"])) < TOL_FP64 * np.max(np.abs(ref["V"])), i
                assert abs(Ei[0] - ref["E"]) < TOL_FP64 * sc, i
            else:
                assert rel_fro(Vi, ref["V"]) < TOL_MIXED, i
                assert np.max(np.abs(Vi - ref["V"])) < TOL_MIXED_ELEM * np.max(np.abs(ref["V"])), i
                assert abs(Ei[0] - ref["E"]) < TOL_MIXED * sc, i
            tol = TOL_FP64 if precision == 0 else TOL_MIXED
            # raw errors: relative to the largest value of each whole gradient
            g = gq[i].cpu().numpy()
            assert np.max(np.abs(g - ref["dE_dRqm"])) < tol * np.max(np.abs(ref["dE_dRqm"])), i
            gmi, gci = gm[i].cpu().numpy(), gc[i].cpu().numpy()
            assert np.max(np.abs(gci[mm] - ref["dE_dq"][mm])) < tol * np.max(np.abs(gci)), i
            assert np.max(np.abs(gmi[mm] - ref["dE_dRmm"][mm])) < tol * np.max(np.abs(gmi)), i
    finally:
        for h in hs:
            h.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_batch_matches_plain_calls_and_replays(precision):
    torch = pytest.importorskip("torch")
    import paper_2408_03273_gb300 as q
    frames = _frames()
    hs = [q.Handle(s, precision=precision) for s in frames]
    try:
        ref = [_plain(h, s, s.dm) for h, s in zip(hs, frames)]
        dev = torch.device("cuda")
        dm = [torch.as_tensor(s.dm, device=dev) for s in frames]
        V, E, gq, gm, gc = _dev_outputs(torch, frames)
        b = q.Batch(hs)
        try:
            tol = 1e-12 if precision == 0 else 1e-7  # same kernels; only atomic addition order differs
            for rep in range(2):
                b.run(dm, V, E, gq, gm, gc)
                assert b.captures() == 1
                for i in range(len(frames)):
                    assert _close(V[i].cpu(), ref[i]["V"], tol), (rep, i)
                    assert _close(E[i].cpu(), ref[i]["E"], tol), (rep, i)
                    for k, out in (("gq", gq), ("gm", gm), ("gc", gc)):
                        assert _close(out[i].cpu(), ref[i][k], tol), (rep, i, k)
            total, per = b.timing()
            assert total > 0 and len(per) == len(frames) and max(per) == pytest.approx(total)
            # new positions for frame 0 (a small shift keeps its region-I size): the graph replays
            s0 = frames[0]
            qm = s0.atom_xyz + 0.01
            n_before = hs[0].info["n_region1"]
            hs[0].set_positions(qm, s0.mm_xyz)
            same_size = hs[0].info["n_region1"] == n_before
            b.run(dm, V, E, gq, gm, gc)
            h_ref = q.Handle(s0, precision=precision)
            try:
                h_ref.set_positions(qm, s0.mm_xyz)
                r0 = _plain(h_ref, s0, s0.dm)
            finally:
                h_ref.close()
            assert b.captures() == (1 if same_size else 2)
            assert _close(V[0].cpu(), r0["V"], tol)
            assert _close(gq[0].cpu(), r0["gq"], tol)
            # a different output array is a different graph
            V2 = [v.clone() for v in V]
            b.run(dm, V2, E, gq, gm, gc)
            assert b.captures() == (2 if same_size else 3)
            assert _close(V2[0].cpu(), r0["V"], tol)
        finally:
            b.close()
    finally:
        for h in hs:
            h.close()


def test_batch_mixes_precisions_and_an_empty_region1():
    # FP64 frames keep their own sweeps inside the graph while the mixed frames' sweeps run
    # batched; a mixed frame whose region I is empty has no sweep to batch.  Against each handle's
    # plain calls, on the recording run and on a replay into cleared outputs.
    torch = pytest.importorskip("torch")
    import paper_2408_03273_gb300 as q
    frames = _frames() + [workloads.small_system(seed=107, n_atoms=2, lmax=1, n_waters=6, cutoff_A=0.3)]
    precs = [1, 0, 1, 1]
    hs = [q.Handle(s, precision=p) for s, p in zip(frames, precs)]
    try:
        assert hs[3].info["n_region1"] == 0 and all(h.info["n_region1"] > 0 for h in hs[:3])
        ref = [_plain(h, s, s.dm) for h, s in zip(hs, frames)]
        dev = torch.device("cuda")
        dm = [torch.as_tensor(s.dm, device=dev) for s in frames]
        V, E, gq, gm, gc = _dev_outputs(torch, frames)
        b = q.Batch(hs)
        try:
            for replay in (False, True):
                if replay:
                    for t in V + E + gq + gm + gc:
                        t.zero_()
                b.run(dm, V, E, gq, gm, gc)
                for i, p in enumerate(precs):
                    tol = 1e-12 if p == 0 else 1e-7
                    for got, key in ((V, "V"), (E, "E"), (gq, "gq"), (gm, "gm"), (gc, "gc")):
                        assert _close(got[i].cpu(), ref[i][key], tol), (replay, i, key)
            assert b.captures() == 1
        finally:
            b.close()
    finally:
        for h in hs:
            h.close()


def test_batch_rejects_host_memory():
    torch = pytest.importorskip("torch")
    import paper_2408_03273_gb300 as q
    frames = _frames()[:2]
    hs = [q.Handle(s) for s in frames]
    try:
        b = q.Batch(hs)
        try:
            with pytest.raises(q.QMMMError):
                b.run([s.dm for s in frames])  # host densities
            dm = [torch.as_tensor(s.dm, device="cuda") for s in frames]
            with pytest.raises(q.QMMMError):
                b.run(dm, V=[np.zeros((s.nao, s.nao)) for s in frames])  # host outputs
        finally:
            b.close()
        with pytest.raises(q.QMMMError):
            q.Batch([hs[0], hs[0]])  # a handle twice
    finally:
        for h in hs:
            h.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_batch_follows_md_steps(precision):
    # new positions every step (region-I sizes change): the batch is recorded again without its
    # plain pass when the buffers suffice, and updated in place when only launch parameters change
    torch = pytest.importorskip("torch")
    import paper_2408_03273_gb300 as q
    frames = _frames()
    hs = [q.Handle(s, precision=precision) for s in frames]
    rng = np.random.default_rng(7)
    try:
        dev = torch.device("cuda")
        dm = [torch.as_tensor(s.dm, device=dev) for s in frames]
        V, E, gq, gm, gc = _dev_outputs(torch, frames)
        b = q.Batch(hs)
        try:
            tol = 1e-12 if precision == 0 else 1e-7
            pos = [(s.atom_xyz.copy(), s.mm_xyz.copy()) for s in frames]
            sizes = []
            for step in range(4):
                if step:
                    for i, h in enumerate(hs):
                        qm, mm = pos[i]
                        qm = qm + rng.normal(scale=0.05, size=qm.shape)
                        mm = mm + rng.normal(scale=0.8, size=mm.shape)  # waters cross the region-I sphere
                        pos[i] = (qm, mm)
                        h.set_positions(qm, mm)
                sizes.append([h.info["n_region1"] for h in hs])
                refs = []
                for i, s in enumerate(frames):
                    r = q.Handle(s, precision=precision)
                    try:
                        r.set_positions(*pos[i])
                        refs.append(_plain(r, s, s.dm))
                    finally:
                        r.close()
                # the run that records the step's graph, then a replay into cleared outputs: every
                # result must come from the graph (a frame left out of the recording would only
                # have been computed once, outside it)
                for replay in (False, True):
                    if replay:
                        for t in V + E + gq + gm + gc:
                            t.zero_()
                    b.run(dm, V, E, gq, gm, gc)
                    for i, ref in enumerate(refs):
                        for got, key in ((V, "V"), (E, "E"), (gq, "gq"), (gm, "gm"), (gc, "gc")):
                            assert _close(got[i].cpu(), ref[key], tol), (step, i, key, replay)
            recorded, inst, upd = b.counts()
            assert 1 <= recorded <= 4 and inst + upd == recorded and inst >= 1
            assert len({tuple(x) for x in sizes}) > 1  # region I did change between steps
        finally:
            b.close()
    finally:
        for h in hs:
            h.close()
