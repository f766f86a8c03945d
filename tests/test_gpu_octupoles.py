"""Octupole error estimate (Sec. "Error Control") through the C ABI against the oracle: the
Mulliken octupoles, Err(R) over radii below and above the handle's region-I radius (the oracle
recomputes region II from scratch for every R, the library moves images between the spheres),
and the R_cut search on that curve."""
import numpy as np
import pytest

import oracle
import workloads
from _gpuutil import TOL_FP64, TOL_MIXED

pytestmark = pytest.mark.gpu

A2B = 1.0 / 0.52917721092
CASES = {
    "gauss": dict(seed=131, n_atoms=3, lmax=2, nprim=(1, 3), n_waters=14),
    "point": dict(seed=132, n_atoms=4, lmax=3, nprim=(1, 2), n_waters=12, point_charges=True),
}


@pytest.fixture(scope="module", params=list(CASES))
def case(request):
    s = workloads.small_system(**CASES[request.param])
    r_lo, dr, n = 3.0 * A2B, 0.25 * A2B, 21  # 3 A .. 8 A; the handle's region I is 5.5 A
    radii = r_lo + dr * np.arange(n)
    return s, (r_lo, dr, n), oracle.octupoles(s), oracle.octupole_error(s, radii)


@pytest.mark.parametrize("precision", [0, 1])
def test_octupole_error_matches_oracle(case, precision):
    import paper_2408_03273_gb300 as q
    s, (r_lo, dr, n), oct_ref, err_ref = case
    h = q.Handle(s, precision=precision)
    try:
        err, oct_ = h.octupole_error(s.dm, r_lo, dr, n, want_octupoles=True)
    finally:
        h.close()
    tol = TOL_FP64 if precision == 0 else TOL_MIXED
    assert np.max(np.abs(oct_ - oct_ref)) < TOL_FP64 * np.max(np.abs(oct_ref))
    assert np.max(np.abs(err - err_ref)) < tol * np.max(np.abs(err_ref))


def test_rcut_search_picks_first_radius_below_eps(case):
    import paper_2408_03273_gb300 as q
    s, (r_lo, dr, n), _, err_ref = case
    h = q.Handle(s)
    try:
        a = np.sort(np.abs(err_ref))
        eps = 0.5 * float(a[len(a) // 2] + a[len(a) // 2 + 1])  # between two values: no tie at eps
        r, e = h.rcut_search(s.dm, r_lo, dr, n, eps)
        k = int(np.argmax(np.abs(err_ref) < eps))
        assert r == pytest.approx(r_lo + k * dr)
        assert e == pytest.approx(err_ref[k], rel=1e-9)
        r_none, _ = h.rcut_search(s.dm, r_lo, dr, n, 1e-300)
        assert r_none == -1.0
    finally:
        h.close()
