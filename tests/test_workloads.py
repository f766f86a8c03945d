"""The seeded synthetic inputs (workloads/) against the workload recipes they stand in for: QM
regions of the stated size and element mix, rigid TIP3P waters (geometry, charges, neutral
cells), the basis recipe (exponent range, primitive counts, angular momenta), a symmetric
positive semi-definite density of the stated trace, the box/cutoff/Ewald parameters, and
determinism in the seed.  CPU only: the generators hold none of the method's arithmetic."""
import numpy as np
import pytest

import workloads
from workloads.synth import ANGSTROM_TO_BOHR

A = ANGSTROM_TO_BOHR


def waters(s):
    """MM sites as (n, 3, 3) molecules in Angstrom (O, H, H) and their charges."""
    assert s.nmm % 3 == 0
    return s.mm_xyz.reshape(-1, 3, 3) / A, s.mm_q.reshape(-1, 3)


def check_tip3p(s):
    mol, q = waters(s)
    assert np.all(q == np.array([-0.834, 0.417, 0.417]))
    assert abs(s.mm_q.sum()) < 1e-9
    d1 = np.linalg.norm(mol[:, 1] - mol[:, 0], axis=1)
    d2 = np.linalg.norm(mol[:, 2] - mol[:, 0], axis=1)
    assert np.allclose(d1, 0.9572, atol=1e-9) and np.allclose(d2, 0.9572, atol=1e-9)
    cos = np.einsum("ij,ij->i", mol[:, 1] - mol[:, 0], mol[:, 2] - mol[:, 0]) / (d1 * d2)
    assert np.allclose(np.degrees(np.arccos(cos)), 104.52, atol=1e-7)
    # orientations are random: the HOH bisectors spread over the sphere
    bis = (mol[:, 1] + mol[:, 2]) / 2 - mol[:, 0]
    bis /= np.linalg.norm(bis, axis=1)[:, None]
    assert np.linalg.norm(bis.mean(axis=0)) < 0.2


def check_basis(s, lmax, nprim):
    assert s.shell_l.max() <= lmax and s.shell_l.min() == 0
    assert s.shell_nprim.min() >= nprim[0] and s.shell_nprim.max() <= nprim[1]
    assert np.all(s.prim_exp >= 0.1) and np.all(s.prim_exp <= 50.0)
    assert s.nao == int(sum((l + 1) * (l + 2) // 2 for l in s.shell_l))


def check_density(s):
    D = s.dm
    assert D.shape == (s.nao, s.nao)
    assert np.array_equal(D, D.T)
    w = np.linalg.eigvalsh(D)
    assert w.min() > -1e-10 * max(1.0, w.max())
    return float(np.trace(D))


def test_water_cluster_workload():
    s = workloads.config1_water()
    assert s.natm == 3 and sorted(np.asarray(s.atom_Z).astype(int).tolist()) == [1, 1, 8]
    x = s.atom_xyz / A
    o, h1, h2 = x[np.argmax(s.atom_Z)], *x[np.asarray(s.atom_Z) == 1]
    assert np.allclose([np.linalg.norm(h1 - o), np.linalg.norm(h2 - o)], 0.96, atol=1e-9)
    cos = np.dot(h1 - o, h2 - o) / 0.96 ** 2
    assert abs(np.degrees(np.arccos(cos)) - 104.5) < 1e-7
    check_basis(s, 2, (3, 3))
    assert abs(check_density(s) - 10.0) < 1e-9
    check_tip3p(s)
    assert 640 <= s.nmm <= 648  # 216 waters less any that overlapped the QM water
    assert np.allclose(s.box / A, 18.6) and tuple(s.kmax) == (7, 7, 7)
    assert abs(s.cutoff / A - 9.0) < 1e-9 and abs(s.ewald_alpha * A - 0.35) < 1e-9


def test_active_site_workload():
    s = workloads.config2_active_site()
    Z = np.asarray(s.atom_Z).astype(int)
    assert s.natm == 60
    assert {z: int((Z == z).sum()) for z in (6, 7, 8, 1)} == {6: 20, 7: 4, 8: 6, 1: 30}
    x = s.atom_xyz / A
    assert np.linalg.norm(x, axis=1).max() <= 10.0 + 1e-9  # a 10 A sphere about the origin
    d = np.linalg.norm(x[:, None] - x[None], axis=-1) + np.eye(60) * 99
    assert d.min() >= 1.0 - 1e-9
    check_basis(s, 2, (1, 5))
    assert 500 <= s.nshell <= 700
    check_density(s)
    check_tip3p(s)
    assert 59000 <= s.nmm <= 60000
    assert np.allclose(s.box / A, 58.0) and tuple(s.kmax) == (16, 16, 16)
    assert abs(s.cutoff / A - 12.0) < 1e-9 and abs(s.ewald_alpha * A - 0.3) < 1e-9


def test_inputs_are_deterministic_in_the_seed():
    a, b = workloads.config2_active_site(), workloads.config2_active_site()
    for key in ("atom_xyz", "mm_xyz", "mm_q", "prim_exp", "prim_coeff", "dm"):
        assert np.array_equal(getattr(a, key), getattr(b, key)), key
    c = workloads.config2_active_site(seed=a.seed + 1)
    assert not np.array_equal(a.mm_xyz, c.mm_xyz)


@pytest.mark.slow
def test_frames_workload():
    fr = workloads.config5_frames()
    assert len(fr) == 64
    nat = np.array([f.natm for f in fr])
    nmm = np.array([f.nmm for f in fr])
    assert nat.min() >= 20 and nat.max() <= 120 and len(set(nat.tolist())) > 20
    assert nmm.min() >= 20000 * 0.98 and nmm.max() <= 120000
    for f in fr[:4]:
        assert f.shell_l.max() <= 2
        assert abs(f.mm_q.sum()) < 1e-8
