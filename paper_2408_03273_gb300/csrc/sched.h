// sched.h -- host-side scheduling rules of the concurrent class sweeps that need no device
// state: how many charge slices a class may take, and which slices and blocks per slice it
// takes.  Plain C++ (no CUDA), so the rules are unit-tested on the host.
#pragma once
#include <algorithm>
#include <cstddef>

namespace qmmm {

// Most charge slices per V class: at least 128 charges each, at most 8, and the partial
// matrices (one per slice, each V element written by one class and slice, summed in a fixed
// order) within 512 MB.
inline int vpot_max_slices(int nch, size_t n2)
{
    const size_t cap = ((size_t)512 << 20) / std::max<size_t>(1, n2 * sizeof(double));
    return std::max(1, std::min({8, nch / 128, (int)std::min<size_t>(cap, 8)}));
}

// Charge slices of one class.  The warps of a class sweep take whole 32-pair tiles, so
// the class finishes when its busiest warp does, after ceil(tiles / warps) tiles: a high-l class
// with 1.2 tiles per warp on average runs as long as with 2.  Splitting the charges over ns block
// rows makes the work units ns times finer.  Picks the rows ns <= maxsl and blocks per row gx
// (gx ns <= share) that minimise the busiest warp's work, in charges, with the per-pair setup
// that every row repeats counted as `setup` charges; fewer rows win near-ties.
inline void class_slices(int tiles, int nwarp, int share, int nch, int maxsl, double setup, int *gx, int *ns)
{
    double best = 1e300;
    *gx = std::max(1, share);
    *ns = 1;
    for (int s = 1; s <= maxsl && share / s >= 1; ++s) {
        const int g = std::min(share / s, (tiles + nwarp - 1) / nwarp);
        const int per_warp = (tiles + g * nwarp - 1) / (g * nwarp);
        const double t = per_warp * (setup + (double)((nch + s - 1) / s));
        if (t < 0.98 * best) {
            best = t;
            *gx = g;
            *ns = s;
        }
    }
}

// Shares of nsm SMs for n classes in proportion to their weights w (SM-time: primitive pairs x
// cost), each at most cap[c] blocks; a class whose proportional share reaches its cap is fixed at
// the cap and the rest is shared again.  Rounding keeps the total within nsm (largest remainders
// first, never above a cap) so that one-block-per-SM sweeps are not oversubscribed; every open
// class gets at least one block.  Classes with open[c] false get 0.
inline void split_shares(int n, const double *w, const int *cap, const bool *open_in, int nsm, int *share)
{
    bool open[64];
    double s[64];
    for (int c = 0; c < n; ++c) {
        open[c] = open_in[c];
        share[c] = 0;
        s[c] = 0.0;
    }
    double left = nsm;
    for (bool again = true; again;) {
        again = false;
        double W = 0.0;
        for (int c = 0; c < n; ++c)
            if (open[c]) W += w[c];
        for (int c = 0; c < n; ++c) {
            if (!open[c]) continue;
            s[c] = W > 0.0 ? left * w[c] / W : 0.0;
            if (s[c] >= cap[c]) {  // capped: fix it and share the rest again
                share[c] = cap[c];
                left -= cap[c];
                open[c] = false;
                again = true;
                break;
            }
        }
    }
    int given = 0;
    for (int c = 0; c < n; ++c)
        if (open[c]) {
            share[c] = std::min(cap[c], std::max(1, (int)s[c]));
            given += share[c];
        }
    // the SMs the floors left over, to the largest remainders
    for (int extra = (int)left - given; extra > 0; --extra) {
        int best = -1;
        double frac = -1.0;
        for (int c = 0; c < n; ++c)
            if (open[c] && share[c] < cap[c] && s[c] - share[c] > frac) {
                frac = s[c] - share[c];
                best = c;
            }
        if (best < 0 || frac <= 0.0) break;
        ++share[best];
    }
}

}  // namespace qmmm
