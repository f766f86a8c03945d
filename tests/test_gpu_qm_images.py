"""QM-QM periodic images (Eq. 5 in Ewald form) through the C ABI against the oracle: energy,
gradient at fixed density (image tensors plus the Pulay term) and the Fock matrix."""
import numpy as np
import pytest

import oracle
import workloads
from _gpuutil import TOL_FP64, rel_max

pytestmark = pytest.mark.gpu

CASES = {
    "spd": dict(seed=141, n_atoms=4, lmax=2, nprim=(1, 3), n_waters=6),
    "spdf_small_box": dict(seed=142, n_atoms=3, lmax=3, nprim=(1, 2), n_waters=3, box_A=8.0, cutoff_A=3.9),
}


@pytest.mark.parametrize("name", list(CASES))
def test_qm_images_match_oracle(name):
    import paper_2408_03273_gb300 as q
    s = workloads.small_system(**CASES[name])
    ref = oracle.qm_images(s)
    h = q.Handle(s)
    try:
        E, g, F = h.qm_images(s.dm, want_F=True)
    finally:
        h.close()
    assert abs(float(E[0]) - ref["E"]) < TOL_FP64 * abs(ref["E"])
    assert rel_max(g, ref["dE_dRqm"]) < TOL_FP64
    assert rel_max(F, ref["F"]) < TOL_FP64
    assert np.max(np.abs(g.sum(0))) < 1e-10 * np.max(np.abs(g))  # no net force from images


def test_qm_images_on_device_arrays():
    torch = pytest.importorskip("torch")
    import paper_2408_03273_gb300 as q
    s = workloads.small_system(**CASES["spd"])
    h = q.Handle(s)
    try:
        E_h, g_h, _ = h.qm_images(s.dm)
        E_d, g_d, _ = h.qm_images(torch.as_tensor(s.dm, device="cuda"))
    finally:
        h.close()
    assert abs(float(E_d.cpu()[0]) - float(E_h[0])) <= 1e-14 * abs(float(E_h[0]))
    assert rel_max(g_d.cpu().numpy(), g_h) < 1e-13
