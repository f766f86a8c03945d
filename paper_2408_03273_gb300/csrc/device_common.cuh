// device_common.cuh -- device building blocks shared by the sm_103a kernels.
//
//  * McMurchie-Davidson Hermite machinery for the region-I integrals of Eq. 9:
//      g_a g_b = sum_t E^{ab}_t Lambda_t (per Cartesian direction; Lambda_t = d^t/dP^t of the
//      Gaussian product), and
//      int Lambda_tuv(r) erf(sqrt(kappa)|r-C|)/|r-C| dr = (2 pi/p) sqrt(kappa/(p+kappa)) R_tuv,
//      R^{(n)}_000 = (-2 rho)^n F_n(rho |P-C|^2), rho = p kappa / (p + kappa),
//      R^{(n)}_{t+1,u,v} = t R^{(n+1)}_{t-1,u,v} + X_PC R^{(n+1)}_{t,u,v}  (and for u, v).
//  * Boys function F_m(T): tabulated F_{m+j}(T_k) on a grid (0.1 for FP64, 1/16 for FP32) with a
//    Taylor expansion about
//    the nearest point and downward recursion F_{m-1} = (2T F_m + e^{-T})/(2m-1) for small T;
//    F_0 = sqrt(pi)/2 T^{-1/2} with the upward recursion F_{m+1} = ((2m+1) F_m - e^{-T})/(2T)
//    for large T (the grid-plus-recursion scheme of Helgaker, Jorgensen and Olsen, Molecular
//    Electronic-Structure Theory, Sec. 9.8).  The tables are written by the host planner.
//  * 1-D TMA bulk copies (cp.async.bulk) into shared memory with an mbarrier whose wait is
//    bounded: on time-out the kernel raises an error flag instead of spinning forever.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace qmmm {

constexpr int LMAX = 3;                       // highest shell angular momentum
constexpr int NCLASS = (LMAX + 1) * (LMAX + 2) / 2;
constexpr double PI = 3.14159265358979323846;
constexpr double TWO_PI = 6.28318530717958647692;
constexpr double HALF_SQRT_PI = 0.88622692545275801365;

// Boys tables (rows T_k = k * step; columns m = 0..NCOL-2, last column e^{-T_k})
constexpr double BOYS_STEP = 0.1;
constexpr double BOYS_INV_STEP = 10.0;
constexpr double BOYS_TMAX_D = 60.0;          // FP64 table range; above: asymptotic branch, where
                                              // e^{-T} < 1e-26 is below FP64 resolution of F_m, m <= 8
constexpr int BOYS_NROW_D = 601;
constexpr int BOYS_NCOL_D = 17;               // host table: orders 0..15 + exp column
constexpr int BOYS_TAYLOR_D = 7;              // terms of the FP64 Taylor expansion
constexpr int BOYS_ROW_D = 8;                 // device row for order M: F_{M+j}(T_k) / j!, j = 0..6,
                                              // then e^{-T_k} (64 B: four aligned double2 loads)
constexpr float BOYS_TMAX_F = 20.0f;          // FP32 table range
constexpr double BOYS_STEP_F = 0.0625;        // FP32 grid T_k = k / 16: exact in FP32, so T - T_k is exact
constexpr float BOYS_INV_STEP_F = 16.0f;
constexpr int BOYS_NROW_F = 321;
constexpr int BOYS_NCOL_F = 17;               // host table: orders 0..15 + exp column
constexpr int BOYS_TAYLOR_F = 5;
constexpr int BOYS_ROW_F = 7;                 // device row for order M: F_{M+j}(T_k) / j!, j = 0..4,
                                              // e^{-T_k}, pad (odd stride: lanes on different rows
                                              // read different banks)
constexpr int BOYS_TAB_F = (BOYS_NROW_F * BOYS_ROW_F + 3) / 4 * 4;  // floats per order (16-byte multiple)
constexpr int BOYS_MAXM = 8;                  // highest order any kernel asks for

// ------------------------------------------------------------------------------------------
// index helpers (compile-time)
// ------------------------------------------------------------------------------------------
__host__ __device__ constexpr int nherm(int L) { return (L + 1) * (L + 2) * (L + 3) / 6; }
__host__ __device__ constexpr int ncart(int l) { return (l + 1) * (l + 2) / 2; }
// Hermite (t,u,v) index, ordered by total order then lexicographically (nested over L)
__host__ __device__ constexpr int hidx(int t, int u, int v)
{
    return (t + u + v) * (t + u + v + 1) * (t + u + v + 2) / 6 + (u + v) * (u + v + 1) / 2 + v;
}
// Cartesian component k of shell l (lexicographic: x^l first)
__host__ __device__ constexpr int cart_lx(int l, int k)
{
    int i = 0;
    for (int lx = l; lx >= 0; --lx)
        for (int ly = l - lx; ly >= 0; --ly) {
            if (i == k) return lx;
            ++i;
        }
    return 0;
}
__host__ __device__ constexpr int cart_ly(int l, int k)
{
    int i = 0;
    for (int lx = l; lx >= 0; --lx)
        for (int ly = l - lx; ly >= 0; --ly) {
            if (i == k) return ly;
            ++i;
        }
    return 0;
}
__host__ __device__ constexpr int cart_lz(int l, int k) { return l - cart_lx(l, k) - cart_ly(l, k); }
__host__ __device__ constexpr int class_of(int la, int lb) { return la * (la + 1) / 2 + lb; }

// ------------------------------------------------------------------------------------------
// Boys function
// ------------------------------------------------------------------------------------------
// F_m(T), m = 0..M.  tab holds one table per order M (BOYS_NROW_D rows of BOYS_ROW_D): for
// T < BOYS_TMAX_D a 7-term Taylor expansion about the nearest T_k with the 1/j! folded into the
// table (Horner with one FMA per term), then the stable downward recursion; above, F_0 from its
// asymptotic form and the upward recursion, which is exact there up to e^{-T}.
template <int M>
__device__ __forceinline__ void boys_f64(double T, double (&F)[M + 1], const double *__restrict__ tab)
{
    if (T < BOYS_TMAX_D) {
        const int k = __double2int_rn(T * BOYS_INV_STEP);
        const double x = (double)k * BOYS_STEP - T;  // -(T - T_k)
        const double2 *row =
            reinterpret_cast<const double2 *>(tab + ((size_t)M * BOYS_NROW_D + k) * BOYS_ROW_D);
        const double2 c01 = __ldg(row), c23 = __ldg(row + 1), c45 = __ldg(row + 2), c6e = __ldg(row + 3);
        double f = fma(c6e.x, x, c45.y);
        f = fma(f, x, c45.x);
        f = fma(f, x, c23.y);
        f = fma(f, x, c23.x);
        f = fma(f, x, c01.y);
        f = fma(f, x, c01.x);
        F[M] = f;
        if (M > 0) {
            // e^{-T} = e^{-T_k} e^{x}, |x| <= 0.05: 8-term Taylor of e^x
            double ex = 1.0 + x * (1.0 + x * (0.5 + x * (1.0 / 6.0 + x * (1.0 / 24.0 + x * (1.0 / 120.0 +
                        x * (1.0 / 720.0 + x * (1.0 / 5040.0)))))));
            const double e = c6e.y * ex;
            const double T2 = 2.0 * T;
#pragma unroll
            for (int m = M; m > 0; --m) F[m - 1] = (T2 * F[m] + e) * (1.0 / (2 * m - 1));
        }
    } else {
        const double rs = rsqrt(T);
        F[0] = HALF_SQRT_PI * rs;
        if (M > 0) {
            const double inv2T = 0.5 * rs * rs;
#pragma unroll
            for (int m = 0; m < M; ++m) F[m + 1] = ((2 * m + 1) * inv2T) * F[m];
        }
    }
}

// rho * (X^2 + Y^2 + Z^2) as an unevaluated sum Th + Tl: squares split exactly with FMA and the
// three-term sum and the product by rho carried with two-sum / two-product error terms, so T is
// accurate to about one FP32 rounding of T itself (the per-charge rounding error of r^2 is what
// cancellation between neutral molecules would otherwise amplify).
__device__ __forceinline__ void boys_arg_f32(float rho, float X, float Y, float Z, float &Th, float &Tl)
{
    const float x2 = X * X, y2 = Y * Y, z2 = Z * Z;
    const float ex = fmaf(X, X, -x2), ey = fmaf(Y, Y, -y2), ez = fmaf(Z, Z, -z2);
    float s = x2 + y2;
    float v = s - x2;
    float e = (x2 - (s - v)) + (y2 - v);
    const float s2 = s + z2;
    v = s2 - s;
    e += (s - (s2 - v)) + (z2 - v);
    const float lo = e + (ex + ey + ez);
    Th = rho * s2;
    Tl = fmaf(rho, s2, -Th) + rho * lo;
}

// tab: the order-M FP32 table (BOYS_NROW_F rows of BOYS_ROW_F), staged in shared memory.  The
// argument is the unevaluated sum T + Tlo (boys_arg_f32), and every step keeps the FP32 result
// within about one rounding of F_m:
//  * T < 20: Taylor expansion of F_M about T_k = k/16 (T - T_k exact), e^{-T} = e^{-T_k} e^{x} with
//    e^{-T_k} from the table and a 5-term series of e^{x}, |x| <= 1/32 (no argument-proportional
//    error of a hardware exponential), downward recursion with 2 (T + Tlo);
//  * T >= 20: F_0 = sqrt(pi)/2 (T + Tlo)^{-1/2} (rsqrtf and one Newton step against the full
//    argument), 1/(2 (T + Tlo)) from rs^2 = s2 + s2e (exact product) corrected by the residual
//    g = 1 - (T + Tlo) rs^2, then the upward recursion F_{m+1} = ((2m+1) F_m - e^{-T}) / (2T).
template <int M>
__device__ __forceinline__ void boys_f32(float T, float (&F)[M + 1], const float *__restrict__ tab /* smem */,
                                         float Tlo = 0.0f)
{
    if (T < BOYS_TMAX_F) {
        // nearest grid index without the conversion pipe: adding 1.5 * 2^23 rounds 16 T to an
        // integer held in the low mantissa bits (exact for 16 T < 2^22)
        const float kf = fmaf(T, BOYS_INV_STEP_F, 12582912.0f);
        const int k = __float_as_int(kf) - 0x4B400000;
        const float x = ((kf - 12582912.0f) * (float)BOYS_STEP_F - T) - Tlo;  // -(T + Tlo - T_k)
        const float *row = tab + k * BOYS_ROW_F;  // the order-M table: 1/j! folded in
        float f = fmaf(row[4], x, row[3]);
        f = fmaf(f, x, row[2]);
        f = fmaf(f, x, row[1]);
        f = fmaf(f, x, row[0]);
        F[M] = f;
        if (M > 0) {
            float ex = fmaf(x, 1.0f / 24.0f, 1.0f / 6.0f);
            ex = fmaf(ex, x, 0.5f);
            ex = fmaf(ex, x, 1.0f);
            ex = fmaf(ex, x, 1.0f);
            const float e = row[BOYS_TAYLOR_F] * ex;
            const float T2 = 2.0f * T, T2l = 2.0f * Tlo;
#pragma unroll
            for (int m = M; m > 0; --m) F[m - 1] = fmaf(T2, F[m], fmaf(T2l, F[m], e)) * (1.0f / (2 * m - 1));
        }
    } else {
        // one Newton step on rsqrtf against the full argument T + Tlo: ~1 ulp of T^{-1/2}
        float rs = rsqrtf(T);
        const float r2 = rs * rs;
        const float h = fmaf(-T, r2, 1.0f) - Tlo * r2;  // 1 - (T + Tlo) rs^2
        rs = fmaf(0.5f * rs, h, rs);
        F[0] = (float)HALF_SQRT_PI * rs;
        if (M > 0) {
            const float e = __expf(-T);  // enters only through (2m+1) F_m - e, where it is < 1e-3 of F_m
            const float s2 = rs * rs, s2e = fmaf(rs, rs, -s2);
            const float g = (fmaf(-T, s2, 1.0f) - T * s2e) - Tlo * s2;  // 1 - (T + Tlo)(s2 + s2e)
            const float inv2T = 0.5f * (s2 + fmaf(s2, g, s2e));
#pragma unroll
            for (int m = 0; m < M; ++m) F[m + 1] = fmaf((float)(2 * m + 1), F[m], -e) * inv2T;
        }
    }
}

// ------------------------------------------------------------------------------------------
// Hermite R tensors, in place: on entry Fn[n] = pref * (-2 rho)^n F_n(T) for n = 0..L;
// on exit R[hidx(t,u,v)] = pref * R_tuv for t+u+v <= L.  Each level n is built from level n+1
// in decreasing total order, so entries of order k only read orders k-1 and k-2 that still
// hold level n+1 values.
// ------------------------------------------------------------------------------------------
template <int L, typename T>
__device__ __forceinline__ void hermite_R(T (&R)[nherm(L)], const T (&Fn)[L + 1], T X, T Y, T Z)
{
    R[0] = Fn[L];
#pragma unroll
    for (int n = L - 1; n >= 0; --n) {
#pragma unroll
        for (int k = L - n; k >= 1; --k) {
#pragma unroll
            for (int t = k; t >= 0; --t) {
#pragma unroll
                for (int u = k - t; u >= 0; --u) {
                    const int v = k - t - u;
                    if (t > 0) {
                        T r = X * R[hidx(t - 1, u, v)];
                        if (t > 1) r += (T)(t - 1) * R[hidx(t - 2, u, v)];
                        R[hidx(t, u, v)] = r;
                    } else if (u > 0) {
                        T r = Y * R[hidx(t, u - 1, v)];
                        if (u > 1) r += (T)(u - 1) * R[hidx(t, u - 2, v)];
                        R[hidx(t, u, v)] = r;
                    } else {
                        T r = Z * R[hidx(t, u, v - 1)];
                        if (v > 1) r += (T)(v - 1) * R[hidx(t, u, v - 2)];
                        R[hidx(t, u, v)] = r;
                    }
                }
            }
        }
        R[0] = Fn[n];
    }
}

// ------------------------------------------------------------------------------------------
// Hermite expansion coefficients in one direction, E[i][j][t] for i <= I, j <= J, with
// E^{00}_0 = 1 (the Gaussian-product factor K_AB is carried separately):
//   E^{i+1,j}_t = 1/(2p) E^{ij}_{t-1} + X_PA E^{ij}_t + (t+1) E^{ij}_{t+1}
//   E^{i,j+1}_t = 1/(2p) E^{ij}_{t-1} + X_PB E^{ij}_t + (t+1) E^{ij}_{t+1}
// ------------------------------------------------------------------------------------------
template <int I, int J, typename T>
__device__ __forceinline__ void hermite_E(T (&E)[I + 1][J + 1][I + J + 1], T XPA, T XPB, T inv2p)
{
#pragma unroll
    for (int i = 0; i <= I; ++i)
#pragma unroll
        for (int j = 0; j <= J; ++j)
#pragma unroll
            for (int t = 0; t <= I + J; ++t) E[i][j][t] = (T)0;
    E[0][0][0] = (T)1;
#pragma unroll
    for (int i = 0; i <= I; ++i)
#pragma unroll
        for (int j = 0; j <= J; ++j) {
            if (i == 0 && j == 0) continue;
            const bool up_i = i > 0;
            const int pi = up_i ? i - 1 : i, pj = up_i ? j : j - 1;
            const T X = up_i ? XPA : XPB;
#pragma unroll
            for (int t = 0; t <= i + j; ++t) {
                T e = (T)0;
                if (t > 0) e += inv2p * E[pi][pj][t - 1];
                if (t <= pi + pj) e += X * E[pi][pj][t];
                if (t + 1 <= pi + pj) e += (T)(t + 1) * E[pi][pj][t + 1];
                E[i][j][t] = e;
            }
        }
}

// ------------------------------------------------------------------------------------------
// warp helpers
// ------------------------------------------------------------------------------------------
constexpr unsigned FULL = 0xffffffffu;

// Segmented suffix sum over contiguous segments: after the call, the first lane of every
// segment holds the segment total.  take[k] says whether lane+2^k lies in the same segment.
template <typename T>
__device__ __forceinline__ T seg_reduce(T v, const bool (&take)[5])
{
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        T o = __shfl_down_sync(FULL, v, 1 << k);
        if (take[k]) v += o;
    }
    return v;
}

__device__ __forceinline__ void seg_setup(int key, int lane, bool (&take)[5], bool &head)
{
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        int o = __shfl_down_sync(FULL, key, 1 << k);
        take[k] = (lane + (1 << k) < 32) && (o == key);
    }
    int prev = __shfl_up_sync(FULL, key, 1);
    head = (lane == 0) || (prev != key);
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v)
{
#pragma unroll
    for (int k = 16; k > 0; k >>= 1) v += __shfl_xor_sync(FULL, v, k);
    return v;
}

// ------------------------------------------------------------------------------------------
// TMA bulk copy global -> shared with a bounded mbarrier wait
// ------------------------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, unsigned bytes, uint64_t *bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_addr(dst)),
                 "l"(src), "r"(bytes), "r"(smem_addr(bar))
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, unsigned phase)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(phase)
        : "memory");
    return ok != 0;
}

// Error flags written by kernels (read back by the host after the call).
enum : int { DEVERR_TIMEOUT = 1, DEVERR_BOUNDS = 2 };

__device__ __forceinline__ uint64_t global_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Wait for phase `phase` of an mbarrier, giving up after `limit_ns` nanoseconds of wall time (the
// global timer, read every 32 polls) or 2^24 polls, whichever comes first.  Block-uniform outcome:
// if any thread gave up, every thread gets false and *err records DEVERR_TIMEOUT.
constexpr uint64_t MBAR_LIMIT_NS = 500000000ull;  // 0.5 s: a bulk copy takes microseconds
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, unsigned phase, int *err,
                                                  uint64_t limit_ns = MBAR_LIMIT_NS)
{
    bool done = false;
    const uint64_t t0 = global_ns();
    for (int it = 0; it < (1 << 24); ++it) {
        if (mbar_try_wait(bar, phase)) { done = true; break; }
        if ((it & 31) == 31 && global_ns() - t0 > limit_ns) break;
    }
    const int fail = __syncthreads_or(!done);
    if (fail && threadIdx.x == 0 && err) atomicOr(err, DEVERR_TIMEOUT);
    return !fail;
}

// Stage up to three segments (sizes multiples of 16 bytes, all addresses 16-byte aligned) from
// global to shared memory with the TMA bulk-copy engine, completing on one mbarrier.  Every
// thread of the block must call it.  Returns false on every thread (and sets *err) if the copies
// did not complete within the iteration budget.
struct Seg { void *dst; const void *src; unsigned bytes; };

__device__ __forceinline__ bool stage_segments(const Seg *seg, int nseg, uint64_t *bar, int *err)
{
    if (threadIdx.x == 0) {
        mbar_init(bar, 1);
        fence_mbar_init();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned total = 0;
        for (int k = 0; k < nseg; ++k) total += seg[k].bytes;
        mbar_arrive_expect_tx(bar, total);
        for (int k = 0; k < nseg; ++k) {
            // pieces of at most 64 KiB, one bulk copy each
            const char *s = (const char *)seg[k].src;
            char *d = (char *)seg[k].dst;
            unsigned left = seg[k].bytes;
            while (left) {
                const unsigned n = left > 65536u ? 65536u : left;
                bulk_g2s(d, s, n, bar);
                d += n; s += n; left -= n;
            }
        }
    }
    return mbar_wait_bounded(bar, 0, err);
}

__device__ __forceinline__ bool stage_to_smem(void *dst, const void *src, unsigned bytes, uint64_t *bar, int *err)
{
    Seg s{dst, src, bytes};
    return stage_segments(&s, 1, bar, err);
}

// A coordinate relative to the QM centre as hi + lo floats with hi on a grid of 2^-16 bohr.  For
// |d| < 128 bohr hi is exact in FP32, and the difference of two hi parts (a multiple of 2^-16
// below 256 in magnitude, at most 24 significant bits) is exact too, so a displacement formed as
// (hi_P - hi_C) + (lo_P - lo_C) is rounded once: correctly rounded FP32 (to about 2^-41 bohr).
// A plain split (hi = (float)d) rounds the hi difference as well; in the region-I sums that
// rounding, raised to the tensor order by the Boys argument and the Hermite polynomials, was the
// largest error of the mixed-precision gradient.
__device__ __forceinline__ void split_grid(double d, float &hi, float &lo)
{
    hi = (float)(rint(d * 65536.0) * (1.0 / 65536.0));
    lo = (float)(d - (double)hi);
}

// double-float accumulation: (hi, lo) += x with an error-free two-sum
__device__ __forceinline__ void df_add(float &hi, float &lo, float x)
{
    const float s = hi + x;
    const float v = s - hi;
    const float e = (hi - (s - v)) + (x - v);
    hi = s;
    lo += e;
}

// ------------------------------------------------------------------------------------------
// double-float numbers h + l (|l| <= ulp(h)/2): about 47 significant bits from FP32 pipes.
// Products use the exact FMA residual, sums the two-sum error; a double-float accumulator
// (ah, al) adds exact hi*hi products with a two-sum and lets the small terms collect in al.
// ------------------------------------------------------------------------------------------
struct f2 {
    float h, l;
};

__device__ __forceinline__ f2 f2_from(double x)
{
    const float h = (float)x;
    return f2{h, (float)(x - (double)h)};
}
__device__ __forceinline__ double f2_to(f2 a) { return (double)a.h + (double)a.l; }
__device__ __forceinline__ double f2_to(float h, float l) { return (double)h + (double)l; }

__device__ __forceinline__ f2 f2_fast2sum(float a, float b)
{
    const float s = a + b;
    return f2{s, b - (s - a)};
}
__device__ __forceinline__ f2 f2_add(f2 a, f2 b)
{
    const float s = a.h + b.h;
    const float v = s - a.h;
    float e = (a.h - (s - v)) + (b.h - v);
    e += a.l + b.l;
    return f2_fast2sum(s, e);
}
__device__ __forceinline__ f2 f2_mul(f2 a, f2 b)
{
    const float p = a.h * b.h;
    float e = fmaf(a.h, b.h, -p);
    e = fmaf(a.h, b.l, e);
    e = fmaf(a.l, b.h, e);
    return f2_fast2sum(p, e);
}
__device__ __forceinline__ f2 f2_neg(f2 a) { return f2{-a.h, -a.l}; }

// (ah, al) += a * b
__device__ __forceinline__ void f2_mac(float &ah, float &al, f2 a, f2 b)
{
    const float p = a.h * b.h;
    const float e = fmaf(a.h, b.h, -p);
    const float s = ah + p;
    const float v = s - ah;
    const float t = (ah - (s - v)) + (p - v);
    ah = s;
    al += t + e;
    al = fmaf(a.h, b.l, al);
    al = fmaf(a.l, b.h, al);
}

// complex double-float: (re, im) as f2 pairs, stored as float4 (re.h, re.l, im.h, im.l)
struct c2 {
    f2 re, im;
};
__device__ __forceinline__ c2 c2_from(float4 v) { return c2{f2{v.x, v.y}, f2{v.z, v.w}}; }
__device__ __forceinline__ float4 c2_pack(double re, double im)
{
    const f2 a = f2_from(re), b = f2_from(im);
    return make_float4(a.h, a.l, b.h, b.l);
}
__device__ __forceinline__ c2 c2_mul(c2 a, c2 b)
{
    return c2{f2_add(f2_mul(a.re, b.re), f2_neg(f2_mul(a.im, b.im))), f2_add(f2_mul(a.re, b.im), f2_mul(a.im, b.re))};
}
// complex accumulator (4 floats) += a * b
__device__ __forceinline__ void c2_mac(float (&acc)[4], c2 a, c2 b)
{
    f2_mac(acc[0], acc[1], a.re, b.re);
    f2_mac(acc[0], acc[1], f2_neg(a.im), b.im);
    f2_mac(acc[2], acc[3], a.re, b.im);
    f2_mac(acc[2], acc[3], a.im, b.re);
}

// ------------------------------------------------------------------------------------------
// multipole interaction tensors of a radial function (Ewald kernels, FP64)
//   T = f, T_a = d_a f, T_ab = 1/2 d_ab f, T_abc = 1/6 d_abc f  (derivatives w.r.t. R_j),
//   d_a f = x_a g1, d_ab f = delta_ab g1 + x_a x_b g2,
//   d_abc f = (delta_ab x_c + delta_ac x_b + delta_bc x_a) g2 + x_a x_b x_c g3,
// with g1 = f'/r, g2 = g1'/r, g3 = g2'/r.  For 1/r: g1 = -r^-3, g2 = 3 r^-5, g3 = -15 r^-7.
// For erfc(beta r)/r (SI screened tensors): g1 = -f3, g2 = 3 f5, g3 = -15 f7.
// Component order: 0 | x y z | xx xy xz yy yz zz | xxx xxy xxz xyy xyz xzz yyy yyz yzz zzz.
// ------------------------------------------------------------------------------------------
__device__ __forceinline__ void radial_tensor(double f, double g1, double g2, double g3, double x, double y,
                                              double z, double *T /* [20] */, int order /* 1..3 */)
{
    T[0] = f;
    T[1] = x * g1; T[2] = y * g1; T[3] = z * g1;
    if (order < 2) return;
    T[4] = 0.5 * (g1 + x * x * g2);
    T[5] = 0.5 * (x * y * g2);
    T[6] = 0.5 * (x * z * g2);
    T[7] = 0.5 * (g1 + y * y * g2);
    T[8] = 0.5 * (y * z * g2);
    T[9] = 0.5 * (g1 + z * z * g2);
    if (order < 3) return;
    const double s6 = 1.0 / 6.0;
    T[10] = s6 * (3.0 * x * g2 + x * x * x * g3);       // xxx
    T[11] = s6 * (y * g2 + x * x * y * g3);             // xxy
    T[12] = s6 * (z * g2 + x * x * z * g3);             // xxz
    T[13] = s6 * (x * g2 + x * y * y * g3);             // xyy
    T[14] = s6 * (x * y * z * g3);                      // xyz
    T[15] = s6 * (x * g2 + x * z * z * g3);             // xzz
    T[16] = s6 * (3.0 * y * g2 + y * y * y * g3);       // yyy
    T[17] = s6 * (z * g2 + y * y * z * g3);             // yyz
    T[18] = s6 * (y * g2 + y * z * z * g3);             // yzz
    T[19] = s6 * (3.0 * z * g2 + z * z * z * g3);       // zzz
}

__device__ __forceinline__ void point_radial(double r2, double &f, double &g1, double &g2, double &g3)
{
    const double ri = rsqrt(r2), ri2 = ri * ri;
    f = ri;
    g1 = -f * ri2;
    g2 = -3.0 * g1 * ri2;
    g3 = -5.0 * g2 * ri2;
}

__device__ __forceinline__ void screened_radial(double r2, double beta, double &f, double &g1, double &g2,
                                                double &g3)
{
    const double r = sqrt(r2), ri2 = 1.0 / r2;
    const double e = exp(-beta * beta * r2);
    const double c = beta * (2.0 / 1.7724538509055160273);  // 2 beta / sqrt(pi)
    const double f1 = erfc(beta * r) / r;
    const double f3 = (f1 + c * e) * ri2;
    const double b2 = beta * beta;
    const double f5 = (f3 + (2.0 / 3.0) * b2 * c * e) * ri2;
    const double f7 = (f5 + (4.0 / 15.0) * b2 * b2 * c * e) * ri2;
    f = f1; g1 = -f3; g2 = 3.0 * f5; g3 = -15.0 * f7;
}

// weights of the 10 stored (Q, mu, theta) components in a full (a,b) contraction
__device__ __forceinline__ double w10(int k) { return (k == 5 || k == 6 || k == 8) ? 2.0 : 1.0; }

}  // namespace qmmm
