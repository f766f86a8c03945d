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

// Density element of Cartesian components (ia, ib) of a primitive pair, times the pair
// prefactor 2 pi / p c_a c_b K_AB: gamma_{ab} (+ gamma_{ba} for a shell pair off the diagonal,
// whose mirror is not stored).  Zero for an inactive lane.
__device__ __forceinline__ double pair_density(const PPLane &pl, const BasisDev &bd, const double *__restrict__ dm,
                                               int ia, int ib)
{
    if (!pl.active) return 0.0;
    const size_t r = pl.sp.aoA + ia, c = pl.sp.aoB + ib;
    double g = dm[r * bd.nao + c];
    if (pl.sp.shA != pl.sp.shB) g += dm[c * bd.nao + r];
    return g * (TWO_PI * pl.ip * pl.cab);
}

// D0_tuv = sum_ab g_ab E^x_t E^y_u E^z_v: the density folded into the Hermite coefficients of the
// pair (Eq. 9 contracted with the density matrix), once per primitive pair.
template <int LA, int LB>
__device__ __forceinline__ void fold_density(const PPLane &pl, const BasisDev &bd, const double *__restrict__ dm,
                                             double (&D0)[nherm(LA + LB)])
{
    constexpr int L = LA + LB, NA = ncart(LA), NB = ncart(LB);
#pragma unroll
    for (int k = 0; k < nherm(L); ++k) D0[k] = 0.0;
    double Ex[LA + 1][LB + 1][L + 1], Ey[LA + 1][LB + 1][L + 1], Ez[LA + 1][LB + 1][L + 1];
    hermite_E<LA, LB, double>(Ex, pl.P[0] - pl.A[0], pl.P[0] - pl.B[0], 0.5 * pl.ip);
    hermite_E<LA, LB, double>(Ey, pl.P[1] - pl.A[1], pl.P[1] - pl.B[1], 0.5 * pl.ip);
    hermite_E<LA, LB, double>(Ez, pl.P[2] - pl.A[2], pl.P[2] - pl.B[2], 0.5 * pl.ip);
#pragma unroll
    for (int ia = 0; ia < NA; ++ia)
#pragma unroll
        for (int ib = 0; ib < NB; ++ib) {
            const int ax = cart_lx(LA, ia), ay = cart_ly(LA, ia), az = cart_lz(LA, ia);
            const int bx = cart_lx(LB, ib), by = cart_ly(LB, ib), bz = cart_lz(LB, ib);
            const double g = pair_density(pl, bd, dm, ia, ib);
#pragma unroll
            for (int t = 0; t <= ax + bx; ++t)
#pragma unroll
                for (int u = 0; u <= ay + by; ++u) {
                    const double gxy = g * Ex[ax][bx][t] * Ey[ay][by][u];
#pragma unroll
                    for (int w = 0; w <= az + bz; ++w) D0[hidx(t, u, w)] += gxy * Ez[az][bz][w];
                }
        }
}

// The centre-A derivative coefficients themselves, Da_tuv = sum_ab g_ab E'^a_{tuv} (E'^a as in
// contract_dA below), for a sweep that contracts them with partial charge sums.
// With WITH_D0, D0 (as in fold_density) is formed in the same pass.
template <int LA, int LB, bool WITH_D0 = false>
__device__ __forceinline__ void fold_density_dA(const PPLane &pl, const BasisDev &bd, const double *__restrict__ dm,
                                                double (&Dx)[nherm(LA + LB)], double (&Dy)[nherm(LA + LB)],
                                                double (&Dz)[nherm(LA + LB)], double *D0 = nullptr)
{
    constexpr int L = LA + LB, NA = ncart(LA), NB = ncart(LB);
    const double aop = pl.a * pl.ip;
#pragma unroll
    for (int k = 0; k < nherm(L); ++k) {
        Dx[k] = Dy[k] = Dz[k] = 0.0;
        if constexpr (WITH_D0) D0[k] = 0.0;
    }
    double Ex[LA + 2][LB + 1][L + 2], Ey[LA + 2][LB + 1][L + 2], Ez[LA + 2][LB + 1][L + 2];
    hermite_E<LA + 1, LB, double>(Ex, pl.P[0] - pl.A[0], pl.P[0] - pl.B[0], 0.5 * pl.ip);
    hermite_E<LA + 1, LB, double>(Ey, pl.P[1] - pl.A[1], pl.P[1] - pl.B[1], 0.5 * pl.ip);
    hermite_E<LA + 1, LB, double>(Ez, pl.P[2] - pl.A[2], pl.P[2] - pl.B[2], 0.5 * pl.ip);
#pragma unroll
    for (int ia = 0; ia < NA; ++ia)
#pragma unroll
        for (int ib = 0; ib < NB; ++ib) {
            const int ax = cart_lx(LA, ia), ay = cart_ly(LA, ia), az = cart_lz(LA, ia);
            const int bx = cart_lx(LB, ib), by = cart_ly(LB, ib), bz = cart_lz(LB, ib);
            const double g = pair_density(pl, bd, dm, ia, ib);
            double dEx[L + 1], dEy[L + 1], dEz[L + 1];
#pragma unroll
            for (int t = 0; t <= ax + bx; ++t) {
                double e = 2.0 * pl.a * Ex[ax + 1][bx][t];
                if (ax > 0) e -= ax * Ex[ax - 1][bx][t];
                if (t > 0) e -= aop * Ex[ax][bx][t - 1];
                dEx[t] = g * e;
            }
#pragma unroll
            for (int u = 0; u <= ay + by; ++u) {
                double e = 2.0 * pl.a * Ey[ay + 1][by][u];
                if (ay > 0) e -= ay * Ey[ay - 1][by][u];
                if (u > 0) e -= aop * Ey[ay][by][u - 1];
                dEy[u] = e;
            }
#pragma unroll
            for (int w = 0; w <= az + bz; ++w) {
                double e = 2.0 * pl.a * Ez[az + 1][bz][w];
                if (az > 0) e -= az * Ez[az - 1][bz][w];
                if (w > 0) e -= aop * Ez[az][bz][w - 1];
                dEz[w] = e;
            }
#pragma unroll
            for (int t = 0; t <= ax + bx; ++t)
#pragma unroll
                for (int u = 0; u <= ay + by; ++u)
#pragma unroll
                    for (int w = 0; w <= az + bz; ++w) {
                        const int k = hidx(t, u, w);
                        const double gx = g * Ex[ax][bx][t], ey = Ey[ay][by][u], ez = Ez[az][bz][w];
                        Dx[k] += dEx[t] * ey * ez;
                        Dy[k] += gx * dEy[u] * ez;
                        Dz[k] += gx * ey * dEz[w];
                        if constexpr (WITH_D0) D0[k] += gx * ey * ez;
                    }
        }
}

// The centre-A derivative part of the adjoint for one primitive pair, contracted with the
// charge sums S_tuv = sum_C q_C R_tuv(P - C):
//   d_a = sum_ab g_ab sum_tuv E'^a_{tuv} S_tuv,   a = x, y, z,
// where E'^a is the product of Hermite coefficients with the a-factor replaced by
//   E'^{ij}_t = dE^{ij}_t / dX_AB = 2a E^{i+1,j}_t - i E^{i-1,j}_t - (a/p) E^{ij}_{t-1}
// (t <= i + j; E'_{i+j+1} vanishes).  Per-charge terms d_a(C) = sum E' R(C) enter the pair
// gradient only through their q-weighted sum, so summing R over the charges first and
// contracting once per pair gives the same sum.
template <int LA, int LB>
__device__ __forceinline__ void contract_dA(const PPLane &pl, const BasisDev &bd, const double *__restrict__ dm,
                                            const double (&S)[nherm(LA + LB)], double (&d)[3])
{
    constexpr int L = LA + LB, NA = ncart(LA), NB = ncart(LB);
    const double aop = pl.a * pl.ip;
    d[0] = d[1] = d[2] = 0.0;
    double Ex[LA + 2][LB + 1][L + 2], Ey[LA + 2][LB + 1][L + 2], Ez[LA + 2][LB + 1][L + 2];
    hermite_E<LA + 1, LB, double>(Ex, pl.P[0] - pl.A[0], pl.P[0] - pl.B[0], 0.5 * pl.ip);
    hermite_E<LA + 1, LB, double>(Ey, pl.P[1] - pl.A[1], pl.P[1] - pl.B[1], 0.5 * pl.ip);
    hermite_E<LA + 1, LB, double>(Ez, pl.P[2] - pl.A[2], pl.P[2] - pl.B[2], 0.5 * pl.ip);
#pragma unroll
    for (int ia = 0; ia < NA; ++ia)
#pragma unroll
        for (int ib = 0; ib < NB; ++ib) {
            const int ax = cart_lx(LA, ia), ay = cart_ly(LA, ia), az = cart_lz(LA, ia);
            const int bx = cart_lx(LB, ib), by = cart_ly(LB, ib), bz = cart_lz(LB, ib);
            const double g = pair_density(pl, bd, dm, ia, ib);
            double dEx[L + 1], dEy[L + 1], dEz[L + 1];
#pragma unroll
            for (int t = 0; t <= ax + bx; ++t) {
                double e = 2.0 * pl.a * Ex[ax + 1][bx][t];
                if (ax > 0) e -= ax * Ex[ax - 1][bx][t];
                if (t > 0) e -= aop * Ex[ax][bx][t - 1];
                dEx[t] = e;
            }
#pragma unroll
            for (int u = 0; u <= ay + by; ++u) {
                double e = 2.0 * pl.a * Ey[ay + 1][by][u];
                if (ay > 0) e -= ay * Ey[ay - 1][by][u];
                if (u > 0) e -= aop * Ey[ay][by][u - 1];
                dEy[u] = e;
            }
#pragma unroll
            for (int w = 0; w <= az + bz; ++w) {
                double e = 2.0 * pl.a * Ez[az + 1][bz][w];
                if (az > 0) e -= az * Ez[az - 1][bz][w];
                if (w > 0) e -= aop * Ez[az][bz][w - 1];
                dEz[w] = e;
            }
            double sx = 0.0, sy = 0.0, sz = 0.0;
#pragma unroll
            for (int t = 0; t <= ax + bx; ++t)
#pragma unroll
                for (int u = 0; u <= ay + by; ++u)
#pragma unroll
                    for (int w = 0; w <= az + bz; ++w) {
                        const double s = S[hidx(t, u, w)];
                        const double ex = Ex[ax][bx][t], ey = Ey[ay][by][u], ez = Ez[az][bz][w];
                        sx += dEx[t] * ey * ez * s;
                        sy += ex * dEy[u] * ez * s;
                        sz += ex * ey * dEz[w] * s;
                    }
            d[0] += g * sx;
            d[1] += g * sy;
            d[2] += g * sz;
        }
}

// ------------------------------------------------------------------------------------------
// Charge-lane adjoint sweep (mixed precision, every angular class): lanes own region-I charges,
// the primitive pairs' density-folded Hermite coefficients are read from shared memory.  A pair
// record (built once per call in FP64, rounded to FP32) holds, in floats:
//   [0..2] P - centre (hi part, split_grid), [3..5] lo part, [6..7] p (double),
//   then per Hermite index k: (D0_k, Dx_k, Dy_k, Dz_k).
// ------------------------------------------------------------------------------------------
constexpr int CL_NT = 256;    // threads per block
__host__ __device__ constexpr int cl_rec_floats(int L) { return 8 + 4 * nherm(L); }
// primitive pairs per staged batch (two batches of records in shared memory: <= 22 KB)
__host__ __device__ constexpr int cl_batch(int L) { return L <= 4 ? 16 : 8; }
constexpr int CL_BPB = 8;  // batches per block
// Charge-lane variants: (charges per lane, blocks per SM) for variant v of class order L; 0 where
// the class has no such variant.  Charges per lane amortise the per-pair warp reduction and give
// each lane independent chains; the register budget (65536 / (256 x blocks per SM)) bounds them.
__host__ __device__ constexpr int cl_variant(int L, int v, int field)
{
    constexpr int T[7][2][2] = {{{4, 2}, {2, 3}}, {{4, 2}, {2, 3}}, {{2, 2}, {1, 3}}, {{1, 2}, {2, 1}},
                                {{1, 2}, {2, 1}}, {{1, 1}, {0, 0}}, {{1, 1}, {0, 0}}};
    return (L >= 0 && L <= 6) ? T[L][v][field] : 0;
}

// Hermite R tensors as hermite_R, with every loop of constant trip count (bounds as guards) so
// that the nest unrolls completely and R stays in registers.
template <int L, typename T>
__device__ __forceinline__ void hermite_R_u(T (&R)[nherm(L)], const T (&Fn)[L + 1], T X, T Y, T Z)
{
    R[0] = Fn[L];
#pragma unroll
    for (int n = L - 1; n >= 0; --n) {
#pragma unroll
        for (int k = L; k >= 1; --k) {
            if (k > L - n) continue;
#pragma unroll
            for (int t = L; t >= 0; --t) {
                if (t > k) continue;
#pragma unroll
                for (int u = L; u >= 0; --u) {
                    if (u > k - t) continue;
                    const int v = k - t - u;
                    if (t > 0) {
                        T r = X * R[hidx(t - 1, u, v)];
                        if (t > 1) r = fma((T)(t - 1), R[hidx(t - 2, u, v)], r);
                        R[hidx(t, u, v)] = r;
                    } else if (u > 0) {
                        T r = Y * R[hidx(t, u - 1, v)];
                        if (u > 1) r = fma((T)(u - 1), R[hidx(t, u - 2, v)], r);
                        R[hidx(t, u, v)] = r;
                    } else {
                        T r = Z * R[hidx(t, u, v - 1)];
                        if (v > 1) r = fma((T)(v - 1), R[hidx(t, u, v - 2)], r);
                        R[hidx(t, u, v)] = r;
                    }
                }
            }
        }
        R[0] = Fn[n];
    }
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
        {256, 256, 256, 256, 256, 256, 256, 256, 0, 0}, // vgrad_f32: charge lanes, variant 1 as
                                                        // cl_variant (256 threads either way)
    };
    return (kind >= 0 && kind < SW_NKIND && cls >= 0 && cls < 10) ? T[kind][cls] : 0;
}

// Dynamic shared memory of every FP64 sweep block is at least this much: more than half of an
// SM's 228 KB, so no two FP64 sweep blocks share an SM.  The concurrent class sweeps split the
// SMs in shares, one block per SM; with a region I small enough for two charge chunks to fit in
// one SM, the block scheduler would otherwise stack blocks of different classes on some SMs
// (which then share one saturated FP64 pipe) while others stay idle.  The FP32 sweeps are
// latency-bound instead and gain from a second block on an SM, so they are not padded.
constexpr size_t SWEEP_SMEM_MIN = 116 * 1024;

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
