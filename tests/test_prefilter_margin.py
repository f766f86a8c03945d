"""The FP32 pre-filter of the real-space Ewald sums never rejects a pair inside the cutoff.

The GPU kernels test every (QM atom, MM charge) pair with FP32 positions (rounded once from FP64)
against the minimum image before the FP64 evaluation, with the squared radius
((max(r_c, 9 sigma)) * 1.001 + 0.05)^2 also rounded to FP32.  This restates that test in numpy
float32 (IEEE single precision: the same subtraction, division, round-half-even and products) and
checks it on pairs placed just inside the cutoff, across the box and at its faces, where the
rounding of the coordinates is largest.
"""
import numpy as np


def lim2_f32(rc, rhat):
    r = max(rc, rhat) * 1.001 + 0.05
    return np.float32(r * r)


def far_min_image_f32(a, c, box, lim2):
    """a, c: float32 positions (n, 3); box: float32 (3,); True where the pair is certainly far."""
    f = a - c
    x = f - np.rint(f / box) * box
    return (x * x).sum(axis=1, dtype=np.float32) > lim2


def _pairs_at_distance(rng, n, box, r):
    a = rng.uniform(-box, 2 * box, size=(n, 3))  # positions anywhere within three box lengths
    u = rng.normal(size=(n, 3))
    u /= np.linalg.norm(u, axis=1)[:, None]
    c = a + r[:, None] * u
    # the charge wrapped into the cell, as the handle stores it (its image is what the filter sees)
    c = c - np.floor(c / box) * box
    return a, c


def test_prefilter_keeps_every_pair_inside_the_cutoff():
    rng = np.random.default_rng(7)
    for box_len, rc in ((35.1, 17.0), (109.6, 22.7), (162.5, 22.7)):  # bohr: water box, active sites
        box = np.full(3, box_len)
        n = 200_000
        r = rc * (1.0 - rng.uniform(0.0, 1e-6, n))  # just inside r_c
        a, c = _pairs_at_distance(rng, n, box, r)
        # the exact minimum-image distance is r (the cutoff is below half the box)
        d = a - c
        d -= np.rint(d / box) * box
        assert np.all(np.linalg.norm(d, axis=1) < rc)
        far = far_min_image_f32(a.astype(np.float32), c.astype(np.float32), box.astype(np.float32),
                                lim2_f32(rc, 0.0))
        assert not far.any()


def test_prefilter_keeps_gaussian_hat_pairs():
    # the T-hat correction reaches 9 sigma; with a wide charge that exceeds the Ewald cutoff
    rng = np.random.default_rng(8)
    box = np.full(3, 60.0)
    rc, rhat = 12.0, 9.0 * 2.5
    n = 100_000
    r = rhat * (1.0 - rng.uniform(0.0, 1e-6, n))
    a, c = _pairs_at_distance(rng, n, box, r)
    far = far_min_image_f32(a.astype(np.float32), c.astype(np.float32), box.astype(np.float32),
                            lim2_f32(rc, rhat))
    assert not far.any()


def test_prefilter_rejects_far_pairs():
    # and it does filter: pairs well beyond the radius plus margin are rejected
    rng = np.random.default_rng(9)
    box = np.full(3, 162.5)
    rc = 22.7
    n = 50_000
    r = rng.uniform(rc * 1.001 + 0.2, 0.5 * 162.5 * 0.99, n)
    a, c = _pairs_at_distance(rng, n, box, r)
    far = far_min_image_f32(a.astype(np.float32), c.astype(np.float32), box.astype(np.float32),
                            lim2_f32(rc, 0.0))
    assert far.all()
