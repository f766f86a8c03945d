// pp_tile.cuh -- one lane per primitive pair: geometry of the Gaussian product and the
// class-template dispatch shared by the V, adjoint and moment kernels.
//
// Work layout: primitive pairs of one angular class (l_A, l_B), sorted by shell pair, are cut
// into tiles of 32; a warp owns a tile (lane = primitive pair) and sweeps region-I charges that
// the block staged into shared memory.  Primitive pairs of one shell pair are contiguous lanes,
// so per-shell-pair sums are segmented warp-shuffle reductions.
#pragma once
#include "device_common.cuh"
#include "qmmm_internal.h"

namespace qmmm {

struct PPLane {
    int s;             // shell-pair index
    SPair sp;
    int atomA, atomB;
    double a, b, p, ip;
    double A[3], B[3], P[3];
    double cab;        // c_a c_b K_AB (normalised contraction coefficients times Gaussian-product factor)
    bool active;
};

__device__ __forceinline__ PPLane load_pp(const BasisDev &bd, int i, int pp_end)
{
    PPLane L;
    L.active = i < pp_end;
    const uint32_t code = __ldg(bd.pp + (L.active ? i : pp_end - 1));
    L.s = (int)(code >> 8);
    const int ka = (code >> 4) & 15, kb = code & 15;
    L.sp = bd.sp[L.s];
    const int pa = __ldg(bd.shell_off + L.sp.shA) + ka, pb = __ldg(bd.shell_off + L.sp.shB) + kb;
    L.atomA = __ldg(bd.shell_atom + L.sp.shA);
    L.atomB = __ldg(bd.shell_atom + L.sp.shB);
    L.a = __ldg(bd.exps + pa);
    L.b = __ldg(bd.exps + pb);
    L.p = L.a + L.b;
    L.ip = 1.0 / L.p;
    double ab2 = 0.0;
#pragma unroll
    for (int x = 0; x < 3; ++x) {
        L.A[x] = bd.qm_xyz[3 * L.atomA + x];
        L.B[x] = bd.qm_xyz[3 * L.atomB + x];
        L.P[x] = (L.a * L.A[x] + L.b * L.B[x]) * L.ip;
        const double d = L.A[x] - L.B[x];
        ab2 += d * d;
    }
    L.cab = L.active ? __ldg(bd.ncoef + pa) * __ldg(bd.ncoef + pb) * exp(-L.a * L.b * L.ip * ab2) : 0.0;
    return L;
}

// Inverse of class_of: the angular momenta of a class index.
__host__ __device__ constexpr int la_of_class(int c)
{
    int la = 0;
    while ((la + 1) * (la + 2) / 2 <= c) ++la;
    return la;
}
__host__ __device__ constexpr int lb_of_class(int c) { return c - la_of_class(c) * (la_of_class(c) + 1) / 2; }
static_assert(la_of_class(class_of(3, 2)) == 3 && lb_of_class(class_of(3, 2)) == 2, "class index inverse");

// The four region-I sweep kernels.
enum SweepKind { SW_VPOT_F64 = 0, SW_VPOT_F32 = 1, SW_VGRAD_F64 = 2, SW_VGRAD_F32 = 3, SW_NKIND = 4 };

// Threads per block of the wide variant of a sweep kernel (0: none).  All warps of a block share
// one staged chunk of charges, and that chunk's shared memory allows one block per SM, so the
// block size sets the warps per SM.  A block of NT threads launched with __launch_bounds__(NT, 1)
// may use 65536 / NT registers per thread, rounded down to a multiple of 8; NT is the widest block
// whose cap stays at or above the kernel's register count at 256 threads, so the wide variant
// holds more warps per SM without spilling.  Classes at 255 registers have no wide variant.
__host__ __device__ constexpr int sweep_wide_threads(int kind, int cls)
{
    // class order: (0,0) (1,0) (1,1) (2,0) (2,1) (2,2) (3,0) (3,1) (3,2) (3,3)
    constexpr int T[SW_NKIND][10] = {
        {1024, 640, 512, 640, 384, 384, 512, 0, 0, 0},  // vpot_f64 : 64 87 105 96 150 158 120 regs
        {896, 768, 512, 512, 384, 0, 384, 0, 0, 0},     // vpot_f32 : 68 80 106 102 154 - 136
        {640, 512, 0, 0, 0, 0, 0, 0, 0, 0},             // vgrad_f64: 93 117
        {768, 640, 384, 384, 0, 0, 0, 0, 0, 0},         // vgrad_f32: 80 96 168 148
    };
    return (kind >= 0 && kind < SW_NKIND && cls >= 0 && cls < 10) ? T[kind][cls] : 0;
}

// Class-split compilation.  A sweep source (vpot_*.cu, vgrad_*.cu) is compiled once per angular
// class with -DQMMM_SPLIT_CLASS=<class index>, which defines that class's kernel and explicitly
// instantiates its launcher, and once without, which compiles only the runtime dispatcher below;
// the launchers are declared (not defined) there and resolved at link time.  The unrolled
// high-l kernels are large, so this keeps every compilation short and lets them run in parallel.
//
// Dispatch a functor templated on (LA, LB) for a runtime class index (l_A >= l_B).
template <template <int, int> class K, typename... Args>
cudaError_t dispatch_class(int cls, Args &&...args)
{
    switch (cls) {
    case class_of(0, 0): return K<0, 0>::run(args...);
    case class_of(1, 0): return K<1, 0>::run(args...);
    case class_of(1, 1): return K<1, 1>::run(args...);
    case class_of(2, 0): return K<2, 0>::run(args...);
    case class_of(2, 1): return K<2, 1>::run(args...);
    case class_of(2, 2): return K<2, 2>::run(args...);
    case class_of(3, 0): return K<3, 0>::run(args...);
    case class_of(3, 1): return K<3, 1>::run(args...);
    case class_of(3, 2): return K<3, 2>::run(args...);
    case class_of(3, 3): return K<3, 3>::run(args...);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace qmmm
