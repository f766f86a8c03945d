"""Host-side scheduling rules of the concurrent class sweeps (csrc/sched.h), compiled with the
host C++ compiler and checked against brute force and the invariants the launcher relies on:
the blocks never exceed the class's share of the SMs or its tile count, the slice count stays
within its bound, the chosen slices are never worse than none, and their busiest-warp work is
within the 2% near-tie margin of the best slicing."""
import os
import shutil
import subprocess

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2408_03273_gb300", "csrc")

DRIVER = r"""
#include <cstdio>
#include "sched.h"
int main()
{
    char op;
    while (std::scanf(" %c", &op) == 1) {
        if (op == 'c') {
            int tiles, nwarp, share, nch, maxsl;
            double setup;
            if (std::scanf("%d %d %d %d %d %lf", &tiles, &nwarp, &share, &nch, &maxsl, &setup) != 6) return 1;
            int gx = 0, ns = 0;
            qmmm::class_slices(tiles, nwarp, share, nch, maxsl, setup, &gx, &ns);
            std::printf("%d %d\n", gx, ns);
        } else if (op == 's') {
            int n, nsm;
            if (std::scanf("%d %d", &n, &nsm) != 2 || n > 64) return 1;
            double w[64];
            int cap[64], share[64], o;
            bool open[64];
            for (int c = 0; c < n; ++c)
                if (std::scanf("%lf %d %d", &w[c], &cap[c], &o) != 3) return 1; else open[c] = o != 0;
            qmmm::split_shares(n, w, cap, open, nsm, share);
            for (int c = 0; c < n; ++c) std::printf("%d ", share[c]);
            std::printf("\n");
        } else if (op == 'v') {
            int nch;
            unsigned long long n2;
            if (std::scanf("%d %llu", &nch, &n2) != 2) return 1;
            std::printf("%d\n", qmmm::vpot_max_slices(nch, (size_t)n2));
        }
    }
    return 0;
}
"""


@pytest.fixture(scope="module")
def sched(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if not cxx:
        pytest.skip("no host C++ compiler")
    d = tmp_path_factory.mktemp("sched")
    src, exe = d / "drv.cpp", d / "drv"
    src.write_text(DRIVER)
    subprocess.run([cxx, "-std=c++17", "-O1", "-I", CSRC, str(src), "-o", str(exe)], check=True)

    def run(lines):
        out = subprocess.run([str(exe)], input="\n".join(lines) + "\n", capture_output=True, text=True,
                             check=True).stdout.split("\n")
        return [tuple(int(x) for x in ln.split()) for ln in out if ln.strip()]

    return run


def busiest(tiles, nwarp, gx, ns, nch, setup):
    per_warp = -(-tiles // (gx * nwarp))
    return per_warp * (setup + -(-nch // ns))


def test_active_site_dd_class(sched):
    # FP64 (d,d) class of the active site: 269 tiles, 8 warps per block, 28 SMs, 1730 charges.
    # One slice leaves 2 tiles on the busiest warp against 1.2 on average; four slices of 7
    # blocks give it 5 tiles of 433 charges (2164 + setup) instead of 2 x 1730.
    (gx, ns), = sched(["c 269 8 28 1730 8 16"])
    assert (gx, ns) == (7, 4)
    assert busiest(269, 8, gx, ns, 1730, 16) < 0.7 * busiest(269, 8, 28, 1, 1730, 16)


def test_many_tiles_need_no_slices(sched):
    # (s,s) class: 1344 tiles on 12 blocks of 8 warps = 14 passes exactly; slices cannot help
    (gx, ns), = sched(["c 1344 8 12 1730 8 16"])
    assert (gx, ns) == (12, 1)


def test_rules_against_brute_force(sched):
    rng = np.random.default_rng(2408)
    cases = []
    for _ in range(400):
        tiles = int(rng.integers(1, 3000))
        nwarp = int(rng.choice([8, 12, 16, 20, 24, 28, 32]))
        share = int(rng.integers(1, 153))
        nch = int(rng.integers(1, 4097))
        maxsl = int(rng.integers(1, 9))
        setup = float(rng.choice([16.0, 64.0]))
        cases.append((tiles, nwarp, share, nch, maxsl, setup))
    res = sched([f"c {t} {w} {s} {n} {m} {u}" for t, w, s, n, m, u in cases])
    for (tiles, nwarp, share, nch, maxsl, setup), (gx, ns) in zip(cases, res):
        assert 1 <= ns <= maxsl
        assert gx >= 1 and gx * ns <= share
        assert gx <= -(-tiles // nwarp)
        chosen = busiest(tiles, nwarp, gx, ns, nch, setup)
        none = busiest(tiles, nwarp, min(share, -(-tiles // nwarp)), 1, nch, setup)
        assert chosen <= none
        best = min(busiest(tiles, nwarp, min(share // s, -(-tiles // nwarp)), s, nch, setup)
                   for s in range(1, maxsl + 1) if share // s >= 1)
        assert chosen <= best / 0.98 + 1e-9


def test_vpot_slice_bound(sched):
    n2_small = 1560 * 1560          # active site: 19.5 MB per partial matrix
    n2_large = 5100 * 5100          # large site: 208 MB per partial matrix
    n2_huge = 9000 * 9000           # 648 MB: no room for two
    res = sched([f"v 1730 {n2_small}", f"v 200 {n2_small}", f"v 100 {n2_small}",
                 f"v 1321 {n2_large}", f"v 4096 {n2_huge}", f"v 4096 1"])
    assert [r[0] for r in res] == [8, 1, 1, 2, 1, 8]


def exact_shares(w, cap, open_, nsm):
    """The proportional split with caps, unrounded (the rule the host code follows)."""
    open_ = list(open_)
    fixed = [0.0] * len(w)
    left = float(nsm)
    while True:
        W = sum(wc for wc, o in zip(w, open_) if o)
        for c, o in enumerate(open_):
            if o and W > 0 and left * w[c] / W >= cap[c]:
                fixed[c] = cap[c]
                left -= cap[c]
                open_[c] = False
                break
        else:
            break
    return [fixed[c] if not open_[c] else (left * w[c] / W if W > 0 else 0.0) for c in range(len(w))], open_


def test_shares_never_oversubscribe(sched):
    # six classes whose proportional shares all end in .5: rounding each to nearest asked for
    # 155 blocks on 152 SMs; the largest-remainder rounding keeps the total at 152
    w = [15.5, 30.5, 16.5, 30.5, 36.5, 22.5]
    line = "s 6 152 " + " ".join(f"{x} 1000 1" for x in w)
    (share,) = sched([line])
    assert sum(share) == 152
    assert all(abs(a - b) < 1.0 for a, b in zip(share, w))


def test_shares_against_exact_split(sched):
    rng = np.random.default_rng(3273)
    cases = []
    for _ in range(300):
        n = 10
        open_ = [bool(x) for x in rng.integers(0, 2, n)]
        if not any(open_):
            open_[0] = True
        w = [float(x) for x in rng.uniform(0.05, 5.0, n)]
        cap = [int(x) for x in rng.integers(1, 80, n)]
        nsm = int(rng.choice([16, 76, 152]))
        cases.append((w, cap, open_, nsm))
    lines = ["s 10 %d " % nsm + " ".join(f"{wc} {cc} {int(o)}" for wc, cc, o in zip(w, cap, open_))
             for w, cap, open_, nsm in cases]
    for (w, cap, open_, nsm), share in zip(cases, sched(lines)):
        exact, still_open = exact_shares(w, cap, open_, nsm)
        for c in range(10):
            if not open_[c]:
                assert share[c] == 0
                continue
            assert 1 <= share[c] <= cap[c]
            if still_open[c]:
                assert abs(share[c] - exact[c]) < 1.0 or (exact[c] < 1.0 and share[c] == 1)
            else:
                assert share[c] == cap[c]
        n_open = sum(open_)
        if all(exact[c] >= 1.0 for c in range(10) if open_[c]):
            # no floor raised to one: the total stays within the SMs, and uses them all when
            # the caps allow
            assert sum(share) <= nsm
            assert sum(share) == min(nsm, sum(cap[c] for c in range(10) if open_[c]))
        else:
            assert sum(share) <= max(nsm, n_open) + n_open
