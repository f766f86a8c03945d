// vgrad_f32.cu -- adjoint of the region-I term, mixed precision (see vgrad_f64.cu for the
// derivative algebra), as a charge-lane sweep: one lane per region-I charge (CPL charges per lane),
// the primitive pairs' density-folded Hermite coefficients (D0, Dx, Dy, Dz, built in FP64 once
// per call and rounded to FP32) read from shared memory batch by batch.  The per-charge Boys/R
// recursion to order L+1 and the seven contractions run in FP32; per-charge sums are kept in
// double-float registers, per-pair sums go through a warp reduce-scatter, compensated FP32
// shared-memory atomics and one FP64 global atomic per block (see the comment above k_vgrad_cl).
#include "pp_tile.cuh"

namespace qmmm {

template <int LA, int LB>
struct VgradF32 {
    static cudaError_t run(const BasisDev &bd, const RegionDev &rg, int pp_begin, int pp_end, int ch_begin,
                           int ch_end, const float *boys, const double *dm, double *gqm, double *gchg, int *err,
                           int nsm, int variant, int nslice, ClScratch cl,
                           cudaStream_t st);
    static cudaError_t run_jobs(const ClJob *jobs, int njob, int nthr, int nitems, int *counter, const float *boys,
                                int variant, int nsm, cudaStream_t st);
};

#ifdef QMMM_SPLIT_CLASS  // one angular class per compilation

// ---------------------------------------------------------------------------------------------
// Charge-lane sweep.  With one lane per primitive pair a lane holds D0, S and R (126 floats for
// (d, d), 288 for (f, f)) and the high-l classes spill to local memory, while every charge needs a
// reduction over the warp's pairs; here a lane owns region-I charges and holds only their R, the
// pairs' density-folded coefficients (D0, Dx, Dy, Dz per Hermite index, one 16-byte broadcast
// load) come from shared memory batch by batch, and the per-pair sums are reduced once per pair
// and warp.  Per (pair, charge), all FP32:
//   e0 = D0.R, e_a = D0.R(+a), h_a = D_a.R                         (7 contractions of nherm(L))
//   charge: dq -= e0, dC_a += q e_a                                 (lane registers, double-float)
//   pair:   sum over the block's charges of q h_a and q e_a        (warp reduce-scatter, then
//           compensated shared-memory atomics, then one FP64 global atomic per block)
// The pair gradient g_A = -(sum q h + a/p sum q e), g_B = sum q h - b/p sum q e is formed in FP64
// by k_cl_pairs once every charge tile has added its sums.
// ---------------------------------------------------------------------------------------------

// ---------------------------------------------------------------------------------------------
// Two charges of a lane at once: Blackwell's packed FP32 pair instructions (add, mul, fma on a
// register pair; each component rounded exactly as the scalar instruction), so the contractions,
// the Hermite recursion and most of the Boys function take half the instructions.
// ---------------------------------------------------------------------------------------------
struct f32x2 {
    float2 v;
    __device__ __forceinline__ f32x2() {}
    __device__ __forceinline__ explicit f32x2(float s) : v(make_float2(s, s)) {}
    __device__ __forceinline__ f32x2(float a, float b) : v(make_float2(a, b)) {}
};
__device__ __forceinline__ f32x2 mk2(float2 x)
{
    f32x2 r;
    r.v = x;
    return r;
}
__device__ __forceinline__ f32x2 operator+(f32x2 a, f32x2 b) { return mk2(__fadd2_rn(a.v, b.v)); }
__device__ __forceinline__ f32x2 operator*(f32x2 a, f32x2 b) { return mk2(__fmul2_rn(a.v, b.v)); }
__device__ __forceinline__ f32x2 fma(f32x2 a, f32x2 b, f32x2 c) { return mk2(__ffma2_rn(a.v, b.v, c.v)); }
__device__ __forceinline__ f32x2 operator-(f32x2 a) { return mk2(__fmul2_rn(a.v, make_float2(-1.0f, -1.0f))); }
__device__ __forceinline__ f32x2 operator-(f32x2 a, f32x2 b) { return fma(b, f32x2(-1.0f), a); }

// boys_arg_f32 for two charges (same operations, componentwise)
__device__ __forceinline__ void boys_arg_x2(f32x2 rho, f32x2 X, f32x2 Y, f32x2 Z, f32x2 &Th, f32x2 &Tl)
{
    const f32x2 x2 = X * X, y2 = Y * Y, z2 = Z * Z;
    const f32x2 ex = fma(X, X, -x2), ey = fma(Y, Y, -y2), ez = fma(Z, Z, -z2);
    const f32x2 s = x2 + y2;
    f32x2 v = s - x2;
    f32x2 e = (x2 - (s - v)) + (y2 - v);
    const f32x2 s2 = s + z2;
    v = s2 - s;
    e = e + ((s - (s2 - v)) + (z2 - v));
    const f32x2 lo = e + ((ex + ey) + ez);
    Th = rho * s2;
    Tl = fma(rho, s2, -Th) + rho * lo;
}

// boys_f32 for two charges: both in the table range or both in the asymptotic range take the
// packed branch; a pair that straddles T = 20 takes the scalar function for each
template <int M>
__device__ __forceinline__ void boys_x2(f32x2 T, f32x2 Tlo, f32x2 (&F)[M + 1], const float *__restrict__ tab)
{
    const bool ta = T.v.x < BOYS_TMAX_F, tb = T.v.y < BOYS_TMAX_F;
    if (ta && tb) {
        const f32x2 kf = fma(T, f32x2(BOYS_INV_STEP_F), f32x2(12582912.0f));
        const int ka = __float_as_int(kf.v.x) - 0x4B400000, kb = __float_as_int(kf.v.y) - 0x4B400000;
        const f32x2 x = ((kf - f32x2(12582912.0f)) * f32x2((float)BOYS_STEP_F) - T) - Tlo;  // -(T + Tlo - T_k)
        const float *ra = tab + ka * BOYS_ROW_F, *rb = tab + kb * BOYS_ROW_F;
        f32x2 f = fma(f32x2(ra[4], rb[4]), x, f32x2(ra[3], rb[3]));
        f = fma(f, x, f32x2(ra[2], rb[2]));
        f = fma(f, x, f32x2(ra[1], rb[1]));
        f = fma(f, x, f32x2(ra[0], rb[0]));
        F[M] = f;
        if (M > 0) {
            f32x2 ex = fma(x, f32x2(1.0f / 24.0f), f32x2(1.0f / 6.0f));
            ex = fma(ex, x, f32x2(0.5f));
            ex = fma(ex, x, f32x2(1.0f));
            ex = fma(ex, x, f32x2(1.0f));
            const f32x2 e = f32x2(ra[BOYS_TAYLOR_F], rb[BOYS_TAYLOR_F]) * ex;
            const f32x2 T2 = f32x2(2.0f) * T, T2l = f32x2(2.0f) * Tlo;
#pragma unroll
            for (int m = M; m > 0; --m) F[m - 1] = fma(T2, F[m], fma(T2l, F[m], e)) * f32x2(1.0f / (2 * m - 1));
        }
    } else if (!ta && !tb) {
        f32x2 rs(rsqrtf(T.v.x), rsqrtf(T.v.y));
        const f32x2 r2 = rs * rs;
        const f32x2 h = fma(-T, r2, f32x2(1.0f)) - Tlo * r2;  // 1 - (T + Tlo) rs^2
        rs = fma(f32x2(0.5f) * rs, h, rs);
        F[0] = f32x2((float)HALF_SQRT_PI) * rs;
        if (M > 0) {
            const f32x2 e(__expf(-T.v.x), __expf(-T.v.y));
            const f32x2 s2 = rs * rs, s2e = fma(rs, rs, -s2);
            const f32x2 g = (fma(-T, s2, f32x2(1.0f)) - T * s2e) - Tlo * s2;
            const f32x2 inv2T = f32x2(0.5f) * (s2 + fma(s2, g, s2e));
#pragma unroll
            for (int m = 0; m < M; ++m) F[m + 1] = fma(f32x2((float)(2 * m + 1)), F[m], -e) * inv2T;
        }
    } else {
        float Fa[M + 1], Fb[M + 1];
        boys_f32<M>(T.v.x, Fa, tab, Tlo.v.x);
        boys_f32<M>(T.v.y, Fb, tab, Tlo.v.y);
#pragma unroll
        for (int m = 0; m <= M; ++m) F[m] = f32x2(Fa[m], Fb[m]);
    }
}

// Every kernel below serves one class over one or many frames ("jobs"): with jobs == nullptr the
// single job `one` (a kernel parameter), otherwise the device array jobs[njob], each job's share of
// the flat thread / item range starting at its thr0 / item0.
__device__ __forceinline__ int cl_job_by_thread(const ClJob *jobs, int njob, int t)
{
    int lo = 0, hi = njob - 1;  // the last job with thr0 <= t
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(&jobs[mid].thr0) <= t) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}
__device__ __forceinline__ int cl_job_by_item(const ClJob *jobs, int njob, int item)
{
    int lo = 0, hi = njob - 1;  // the last job with item0 <= item
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(&jobs[mid].item0) <= item) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Pair records of one class (FP64 Hermite/density algebra, rounded to FP32), once per call; the
// pair's charge sums are cleared here too.  Classes with l_A + l_B <= 3: one thread per pair.
template <int LA, int LB>
__global__ void __launch_bounds__(128)
k_cl_records(ClJob one, const ClJob *__restrict__ jobs, int njob, int nthr)
{
    constexpr int L = LA + LB, NH = nherm(L), R4 = cl_rec_floats(L) / 4;
    const int t = (int)(blockIdx.x * blockDim.x + threadIdx.x);
    if (t >= nthr) return;
    const ClJob &J = jobs ? jobs[cl_job_by_thread(jobs, njob, t)] : one;
    const int i = J.pp_begin + (t - J.thr0);
    if (i >= J.pp_end) return;
    const PPLane pl = load_pp(J.bd, i, J.pp_end);
    float4 *r = J.rec + (size_t)(i - J.pp_begin) * R4;
    float ph[3], pl_[3];
#pragma unroll
    for (int x = 0; x < 3; ++x) split_grid(pl.P[x] - J.rg.centre[x], ph[x], pl_[x]);
    const long long pb = __double_as_longlong(pl.p);
    r[0] = make_float4(ph[0], ph[1], ph[2], pl_[0]);
    r[1] = make_float4(pl_[1], pl_[2], __int_as_float((int)(pb & 0xffffffffll)), __int_as_float((int)(pb >> 32)));
    double D0[NH], Dx[NH], Dy[NH], Dz[NH];
    fold_density_dA<LA, LB, true>(pl, J.bd, J.dm, Dx, Dy, Dz, D0);
#pragma unroll
    for (int k = 0; k < NH; ++k) r[2 + k] = make_float4((float)D0[k], (float)Dx[k], (float)Dy[k], (float)Dz[k]);
    double *ps = J.psum + (size_t)(i - J.pp_begin) * 6;
#pragma unroll
    for (int v = 0; v < 6; ++v) ps[v] = 0.0;
}

// The same records for l_A + l_B >= 4.  One thread per pair kept the four folds and the Hermite
// coefficients in local memory (a 6.7 KB stack frame for (f, f)) and ran a few thousand threads on
// part of the SMs (1.22 ms for the 8657 (f, f) pairs of the large site).  Here a block holds 32
// pairs and four warps (eight when the folds are split): warps 0-2 write the coefficients
// E^{ij}_t (i <= l_A + 1) of their lanes' pairs along x, y, z into shared memory, all warps the
// pair densities, then warp w folds component w % 4 of every lane's record (D0, Dx, Dy, Dz: the
// terms of fold_density_dA in the same order) with its Hermite sums in registers (0.45 ms).  For
// the smaller classes the single thread per pair is faster.
__host__ __device__ constexpr bool rec_tab(int L) { return L >= 4; }
template <int LA, int LB>
__host__ __device__ constexpr int rec_esz()
{
    return (LA + 2) * (LB + 1) * (LA + LB + 2);  // E[i][j][t] of one axis, i <= LA + 1
}
// Hermite-index halves of a record folded by separate warps (f shells with l >= 2 on the other
// centre: 56 or 84 sums per fold do not fit in registers beside the operands)
__host__ __device__ constexpr int rec_split(int L) { return L >= 5 ? 2 : 1; }
template <int LA, int LB>
inline size_t rec_smem()
{
    return ((size_t)3 * rec_esz<LA, LB>() + ncart(LA) * ncart(LB)) * 32 * sizeof(double);
}

// f(Ic<I>{}) for I = B .. E-1: every index a compile-time constant, so that the fold's Hermite sums
// are named registers (pragma unroll left the large classes' loops rolled, the sums in local memory)
template <int I>
struct Ic {
    static constexpr int value = I;
};
template <int B, int E, typename F>
__device__ __forceinline__ void static_for(F &&f)
{
    if constexpr (B < E) {
        f(Ic<B>{});
        static_for<B + 1, E>(f);
    }
}
#define IC_VALUE(x) decltype(x)::value

// es: the lane's column of the block's tables (E along x, y, z, then the pair densities g_ab)
template <int LA, int LB, int C, int K0, int K1>
__device__ __forceinline__ void rec_fold(const PPLane &pl, const double *es, double (&D)[nherm(LA + LB)])
{
    constexpr int L = LA + LB, NA = ncart(LA), NB = ncart(LB), EJ = LB + 1, ET = L + 2, ESZ = rec_esz<LA, LB>();
    const double *ex = es, *ey = es + ESZ * 32, *ez = es + 2 * ESZ * 32, *gs = es + 3 * ESZ * 32;
    // read at each use (volatile): the compiler otherwise keeps hundreds of coefficients of the
    // (f, f) tables live in registers across the unrolled fold
    auto E = [](const double *e, int i, int j, int t) {
        return *reinterpret_cast<const volatile double *>(e + ((i * EJ + j) * ET + t) * 32);
    };
    const double aop = pl.a * pl.ip;
    static_for<K0, K1>([&](auto k_) { D[IC_VALUE(k_)] = 0.0; });
    static_for<0, NA>([&](auto ia_) {
        static_for<0, NB>([&](auto ib_) {
            constexpr int ia = IC_VALUE(ia_), ib = IC_VALUE(ib_);
            constexpr int ax = cart_lx(LA, ia), ay = cart_ly(LA, ia), az = cart_lz(LA, ia);
            constexpr int bx = cart_lx(LB, ib), by = cart_ly(LB, ib), bz = cart_lz(LB, ib);
            const double g = gs[(ia * NB + ib) * 32];
            // E' of the derivative's axis (g folded in along x)
            double dE[L + 1];
            (void)dE;
            if constexpr (C == 1) {
                static_for<0, ax + bx + 1>([&](auto t_) {
                    constexpr int t = IC_VALUE(t_);
                    double e = 2.0 * pl.a * E(ex, ax + 1, bx, t);
                    if constexpr (ax > 0) e -= ax * E(ex, ax - 1, bx, t);
                    if constexpr (t > 0) e -= aop * E(ex, ax, bx, t - 1);
                    dE[t] = g * e;
                });
            } else if constexpr (C == 2) {
                static_for<0, ay + by + 1>([&](auto u_) {
                    constexpr int u = IC_VALUE(u_);
                    double e = 2.0 * pl.a * E(ey, ay + 1, by, u);
                    if constexpr (ay > 0) e -= ay * E(ey, ay - 1, by, u);
                    if constexpr (u > 0) e -= aop * E(ey, ay, by, u - 1);
                    dE[u] = e;
                });
            } else if constexpr (C == 3) {
                static_for<0, az + bz + 1>([&](auto w_) {
                    constexpr int w = IC_VALUE(w_);
                    double e = 2.0 * pl.a * E(ez, az + 1, bz, w);
                    if constexpr (az > 0) e -= az * E(ez, az - 1, bz, w);
                    if constexpr (w > 0) e -= aop * E(ez, az, bz, w - 1);
                    dE[w] = e;
                });
            }
            static_for<0, ax + bx + 1>([&](auto t_) {
                constexpr int t = IC_VALUE(t_);
                const double gx = g * E(ex, ax, bx, t);
                static_for<0, ay + by + 1>([&](auto u_) {
                    constexpr int u = IC_VALUE(u_);
                    const double ey_ = E(ey, ay, by, u);
                    static_for<0, az + bz + 1>([&](auto w_) {
                        constexpr int w = IC_VALUE(w_), k = hidx(t, u, w);
                        if constexpr (k >= K0 && k < K1) {
                            const double ez_ = E(ez, az, bz, w);
                            if constexpr (C == 0) D[k] += gx * ey_ * ez_;
                            else if constexpr (C == 1) D[k] += dE[t] * ey_ * ez_;
                            else if constexpr (C == 2) D[k] += gx * dE[u] * ez_;
                            else D[k] += gx * ey_ * dE[w];
                        }
                    });
                });
            });
        });
    });
}
#undef IC_VALUE

template <int LA, int LB>
__global__ void __launch_bounds__(128 * rec_split(LA + LB), 1)
k_cl_records_tab(ClJob one, const ClJob *__restrict__ jobs, int njob, int nthr)
{
    constexpr int L = LA + LB, NH = nherm(L), R4 = cl_rec_floats(L) / 4, ESZ = rec_esz<LA, LB>();
    constexpr int NAB = ncart(LA) * ncart(LB), NW = 4 * rec_split(L), KH = (NH + 1) / 2;
    extern __shared__ double es_raw[];  // [3 axes][ESZ][32 pairs], then g_ab [NAB][32 pairs]
    // warp w folds component w % 4 (over Hermite half w / 4 when split)
    const int lane = (int)(threadIdx.x & 31), warp = (int)(threadIdx.x >> 5), comp = warp & 3, half = warp >> 2;
    const int t = min((int)blockIdx.x * 32 + lane, nthr - 1);  // the grid covers nthr exactly
    const ClJob &J = jobs ? jobs[cl_job_by_thread(jobs, njob, t)] : one;
    const int i = J.pp_begin + (t - J.thr0);
    const PPLane pl = load_pp(J.bd, i, J.pp_end);  // inactive past pp_end (its density is zero)
    if (warp < 3) {
        // the recursion of hermite_E<LA + 1, LB> (same terms, same order) on the lane's column
        const double pa = comp == 0 ? pl.P[0] - pl.A[0] : comp == 1 ? pl.P[1] - pl.A[1] : pl.P[2] - pl.A[2];
        const double pb = comp == 0 ? pl.P[0] - pl.B[0] : comp == 1 ? pl.P[1] - pl.B[1] : pl.P[2] - pl.B[2];
        const double inv2p = 0.5 * pl.ip;
        double *col = es_raw + warp * ESZ * 32 + lane;
        auto at = [col](int a, int b, int h) -> double & { return col[((a * (LB + 1) + b) * (L + 2) + h) * 32]; };
        for (int q = 0; q < ESZ; ++q) col[q * 32] = 0.0;
        at(0, 0, 0) = 1.0;
#pragma unroll 1
        for (int a = 0; a <= LA + 1; ++a)
#pragma unroll 1
            for (int b = 0; b <= LB; ++b) {
                if (a == 0 && b == 0) continue;
                const bool up_a = a > 0;
                const int pa_ = up_a ? a - 1 : a, pb_ = up_a ? b : b - 1;
                const double X = up_a ? pa : pb;
                for (int h = 0; h <= a + b; ++h) {
                    double e = 0.0;
                    if (h > 0) e += inv2p * at(pa_, pb_, h - 1);
                    if (h <= pa_ + pb_) e += X * at(pa_, pb_, h);
                    if (h + 1 <= pa_ + pb_) e += (double)(h + 1) * at(pa_, pb_, h + 1);
                    at(a, b, h) = e;
                }
            }
    }
    // the pair densities, shared by the four folds (loaded inside the fold, the compiler hoisted
    // them all ahead of the sums: 100 live doubles for (f, f))
    for (int q = warp; q < NAB; q += NW)
        es_raw[(3 * ESZ + q) * 32 + lane] = pair_density(pl, J.bd, J.dm, q / ncart(LB), q % ncart(LB));
    __syncthreads();
    const double *es = es_raw + lane;
    double D[NH];
    constexpr int K1A = rec_split(L) > 1 ? KH : NH;
    if (half == 0) {
        if (comp == 0) rec_fold<LA, LB, 0, 0, K1A>(pl, es, D);
        else if (comp == 1) rec_fold<LA, LB, 1, 0, K1A>(pl, es, D);
        else if (comp == 2) rec_fold<LA, LB, 2, 0, K1A>(pl, es, D);
        else rec_fold<LA, LB, 3, 0, K1A>(pl, es, D);
    } else if constexpr (rec_split(L) > 1) {
        if (comp == 0) rec_fold<LA, LB, 0, KH, NH>(pl, es, D);
        else if (comp == 1) rec_fold<LA, LB, 1, KH, NH>(pl, es, D);
        else if (comp == 2) rec_fold<LA, LB, 2, KH, NH>(pl, es, D);
        else rec_fold<LA, LB, 3, KH, NH>(pl, es, D);
    }
    if (!pl.active) return;
    float4 *r = J.rec + (size_t)(i - J.pp_begin) * R4;
    if (warp == 0) {
        float ph[3], pl_[3];
#pragma unroll
        for (int x = 0; x < 3; ++x) split_grid(pl.P[x] - J.rg.centre[x], ph[x], pl_[x]);
        const long long pb = __double_as_longlong(pl.p);
        r[0] = make_float4(ph[0], ph[1], ph[2], pl_[0]);
        r[1] = make_float4(pl_[1], pl_[2], __int_as_float((int)(pb & 0xffffffffll)), __int_as_float((int)(pb >> 32)));
        double *ps = J.psum + (size_t)(i - J.pp_begin) * 6;
#pragma unroll
        for (int v = 0; v < 6; ++v) ps[v] = 0.0;
    }
    // record entry 2 + k = (D0, Dx, Dy, Dz) of Hermite index k
    float *rf = reinterpret_cast<float *>(r + 2) + comp;
    if (half == 0) {
#pragma unroll
        for (int k = 0; k < K1A; ++k) rf[4 * k] = (float)D[k];
    } else {
#pragma unroll
        for (int k = KH; k < NH; ++k) rf[4 * k] = (float)D[k];
    }
}

// CPL charges per lane (a block's tile holds CL_NT * CPL charges of one width class, lane l the
// entries l, l + CL_NT, ...): the per-pair reduction is paid once per CPL charges and the lane has
// CPL independent chains of Boys/R work, in packed pairs when CPL is even; NB pairs per staged
// batch.  A work item is one (charge tile,
// range of pair batches) of a job.  With counter == nullptr each block does item blockIdx.x;
// otherwise the grid is persistent and its blocks take items from *counter until nitems are done
// (the batched form over many frames).
template <int LA, int LB, int CPL, int MINB>
__global__ void __launch_bounds__(CL_NT, MINB)
k_vgrad_cl(ClJob one, const ClJob *__restrict__ jobs, int njob, int nitems, int *__restrict__ counter,
           const float *__restrict__ boys_g)
{
    constexpr int L = LA + LB, NH1 = nherm(L + 1), R4 = cl_rec_floats(L) / 4, NB = cl_batch(L);
    constexpr int TILE = CL_NT * CPL;
    constexpr int PF = (NB * R4 + CL_NT - 1) / CL_NT;  // float4 per thread of a prefetched batch
    // an even number of charges per lane goes in packed pairs; the coefficients of a record are
    // then held twice in shared memory, (D0, D0, Dx, Dx) and (Dy, Dy, Dz, Dz), so that each
    // operand pair of the packed contractions is one aligned register pair of a 16-byte load
    constexpr bool PACK = CPL % 2 == 0;
    constexpr int RS = PACK ? 2 + 2 * nherm(L) : R4;  // float4 per record in shared memory
    constexpr int CP = PACK ? CPL / 2 : 1;
    __shared__ __align__(16) float tab[BOYS_TAB_F];
    __shared__ __align__(16) float4 buf[2][NB * RS];
    __shared__ float2 rsq[2][NB];  // (rho, sqrt(kappa / (p + kappa))) per pair of a batch
    __shared__ float ps_h[2][NB * 8], ps_l[2][NB * 8];
    __shared__ int s_item;

    for (int k = threadIdx.x; k < BOYS_TAB_F; k += CL_NT) tab[k] = __ldg(boys_g + k);
    for (int k = threadIdx.x; k < 2 * NB * 8; k += CL_NT) {
        (&ps_h[0][0])[k] = 0.0f;  // every batch clears the sums it used, so they stay zero
        (&ps_l[0][0])[k] = 0.0f;
    }
    const int lane = threadIdx.x & 31;
    int item = (int)blockIdx.x;
    for (;;) {
        if (counter) {
            if (threadIdx.x == 0) s_item = atomicAdd(counter, 1);
            __syncthreads();
            item = s_item;
        }
        if (item >= nitems) break;
        const ClJob &J = jobs ? jobs[cl_job_by_item(jobs, njob, item)] : one;
        const int local = item - J.item0, gx = J.gx, npair = J.pp_end - J.pp_begin;
        const RegionDev &rg = J.rg;
        const float4 *__restrict__ rec = J.rec;
        double *__restrict__ psum = J.psum;
        // this item's charge tile: TILE charges of one width class within [ch_begin, ch_end)
        int t = local / gx, cbeg = -1, cend = 0;
        double kap = 0.0;
        for (int c = 0; c < rg.ncls; ++c) {
            const int lo = max(__ldg(rg.cls_off + c), J.ch_begin), hi = min(__ldg(rg.cls_off + c + 1), J.ch_end);
            if (lo >= hi) continue;
            const int nt = (hi - lo + TILE - 1) / TILE;
            if (t < nt) {
                cbeg = lo + t * TILE;
                cend = min(hi, cbeg + TILE);
                kap = __ldg(rg.cls_kappa + c);
                break;
            }
            t -= nt;
        }
        // this item's pair batches
        const int nbatch = (npair + NB - 1) / NB;
        const int bper = (nbatch + gx - 1) / gx;
        const int b0 = (local % gx) * bper, b1 = min(nbatch, b0 + bper);
        if (cbeg >= 0 && b0 < b1) {  // item-uniform
            // this lane's charges: entries lane + i CL_NT of the tile (inactive ones carry q = 0).
            // Consecutive region-I charges (the atoms of one water, whose terms cancel) sit in
            // neighbouring lanes, which the pair-sum reduction combines first; a lane's own charges
            // belong to different waters
            float4 ch[CPL], cl[CPL];
#pragma unroll
            for (int i = 0; i < CPL; ++i) {
                const int j = cbeg + (int)threadIdx.x + i * CL_NT;
                ch[i] = cl[i] = make_float4(0.f, 0.f, 0.f, 0.f);
                if (j < cend) {
                    ch[i] = __ldg(rg.chg_hi + j);
                    cl[i] = __ldg(rg.chg_lo + j);
                }
            }

            // a batch's records: element idx of the batch into smem; the thread holding a record's
            // second float4 (with p) also forms (rho, sq) for the tile's width class, in FP64
            auto put = [&](int s, int idx, float4 v) {
                const int pp = idx / R4, pos = idx - pp * R4;
                if (!PACK || pos < 2) {
                    buf[s][pp * RS + pos] = v;
                } else {
                    buf[s][pp * RS + 2 * pos - 2] = make_float4(v.x, v.x, v.y, v.y);
                    buf[s][pp * RS + 2 * pos - 1] = make_float4(v.z, v.z, v.w, v.w);
                }
                if (pos == 1) {
                    const double p = __longlong_as_double(((long long)__float_as_int(v.w) << 32) |
                                                          (unsigned int)__float_as_int(v.z));
                    const double td = kap > 0.0 ? kap / (p + kap) : 1.0;
                    rsq[s][pp] = make_float2((float)(p * td), (float)sqrt(td));
                }
            };
            // packed charge pairs (2j, 2j + 1): negated coordinates, so that the packed additions
            // form the same correctly rounded displacements as the scalar subtractions
            f32x2 nh[CP][3], nl[CP][3], q2[CP];
            if constexpr (PACK) {
#pragma unroll
                for (int j = 0; j < CP; ++j) {
                    nh[j][0] = f32x2(-ch[2 * j].x, -ch[2 * j + 1].x);
                    nh[j][1] = f32x2(-ch[2 * j].y, -ch[2 * j + 1].y);
                    nh[j][2] = f32x2(-ch[2 * j].z, -ch[2 * j + 1].z);
                    nl[j][0] = f32x2(-cl[2 * j].x, -cl[2 * j + 1].x);
                    nl[j][1] = f32x2(-cl[2 * j].y, -cl[2 * j + 1].y);
                    nl[j][2] = f32x2(-cl[2 * j].z, -cl[2 * j + 1].z);
                    q2[j] = f32x2(ch[2 * j].w, ch[2 * j + 1].w);
                }
            }
            {
                const int nb = min(NB, npair - b0 * NB);
                for (int idx = threadIdx.x; idx < nb * R4; idx += CL_NT)
                    put(0, idx, __ldg(rec + (size_t)b0 * NB * R4 + idx));
            }
            __syncthreads();

            float ah[CPL][4], al[CPL][4];  // per-charge sums (double-float): dC_x, dC_y, dC_z, dq
#pragma unroll
            for (int i = 0; i < CPL; ++i)
#pragma unroll
                for (int c = 0; c < 4; ++c) ah[i][c] = al[i][c] = 0.0f;
            for (int b = b0; b < b1; ++b) {
                const int s = (b - b0) & 1;
                const int nb = min(NB, npair - b * NB);
                // prefetch the next batch into registers while this one is computed
                float4 pf[PF];
                const int nbn = b + 1 < b1 ? min(NB, npair - (b + 1) * NB) : 0;
#pragma unroll
                for (int i = 0; i < PF; ++i) {
                    const int idx = (int)threadIdx.x + i * CL_NT;
                    if (idx < nbn * R4) pf[i] = __ldg(rec + (size_t)(b + 1) * NB * R4 + idx);
                }
                float bp[CPL][4];
#pragma unroll
                for (int i = 0; i < CPL; ++i) bp[i][0] = bp[i][1] = bp[i][2] = bp[i][3] = 0.0f;
                f32x2 bp2[CP][4];
#pragma unroll
                for (int j = 0; j < CP; ++j) bp2[j][0] = bp2[j][1] = bp2[j][2] = bp2[j][3] = f32x2(0.0f);
                for (int p = 0; p < nb; ++p) {
                    const float4 *r = buf[s] + p * RS;
                    const float4 h0 = r[0], h1 = r[1];
                    const float2 rq = rsq[s][p];
                    float v[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};  // this lane's pair sums
                    if constexpr (PACK) {
                        f32x2 vv[6];
#pragma unroll
                        for (int c = 0; c < 6; ++c) vv[c] = f32x2(0.0f);
                        const f32x2 hx(h0.x), hy(h0.y), hz(h0.z), lx(h0.w), ly(h1.x), lz(h1.y);
                        const f32x2 rho(rq.x), m2rho(-2.0f * rq.x);
#pragma unroll
                        for (int j = 0; j < CP; ++j) {
                            const f32x2 X = (hx + nh[j][0]) + (lx + nl[j][0]);
                            const f32x2 Y = (hy + nh[j][1]) + (ly + nl[j][1]);
                            const f32x2 Z = (hz + nh[j][2]) + (lz + nl[j][2]);
                            f32x2 T, Tl;
                            boys_arg_x2(rho, X, Y, Z, T, Tl);
                            f32x2 F[L + 2];
                            boys_x2<L + 1>(T, Tl, F, tab);
                            f32x2 Fn[L + 2];
                            {
                                f32x2 sc(rq.y);
#pragma unroll
                                for (int n = 0; n <= L + 1; ++n) {
                                    Fn[n] = sc * F[n];
                                    sc = sc * m2rho;
                                }
                            }
                            f32x2 R[NH1];
                            hermite_R_u<L + 1, f32x2>(R, Fn, X, Y, Z);
                            f32x2 e0(0.0f), ex(0.0f), ey(0.0f), ez(0.0f), gx(0.0f), gy(0.0f), gz(0.0f);
#pragma unroll
                            for (int tt = 0; tt <= L; ++tt)
#pragma unroll
                                for (int uu = 0; uu <= L; ++uu)
#pragma unroll
                                    for (int ww = 0; ww <= L; ++ww) {
                                        if (tt + uu + ww > L) continue;
                                        const int k = hidx(tt, uu, ww);
                                        const float4 da = r[2 + 2 * k], db = r[3 + 2 * k];
                                        const f32x2 d0(da.x, da.y), dx(da.z, da.w), dy(db.x, db.y), dz(db.z, db.w);
                                        e0 = fma(d0, R[k], e0);
                                        ex = fma(d0, R[hidx(tt + 1, uu, ww)], ex);
                                        ey = fma(d0, R[hidx(tt, uu + 1, ww)], ey);
                                        ez = fma(d0, R[hidx(tt, uu, ww + 1)], ez);
                                        gx = fma(dx, R[k], gx);
                                        gy = fma(dy, R[k], gy);
                                        gz = fma(dz, R[k], gz);
                                    }
                            const f32x2 q = q2[j];
                            bp2[j][0] = fma(q, ex, bp2[j][0]);
                            bp2[j][1] = fma(q, ey, bp2[j][1]);
                            bp2[j][2] = fma(q, ez, bp2[j][2]);
                            bp2[j][3] = bp2[j][3] - e0;
                            vv[0] = fma(q, gx, vv[0]);
                            vv[1] = fma(q, gy, vv[1]);
                            vv[2] = fma(q, gz, vv[2]);
                            vv[3] = fma(q, ex, vv[3]);
                            vv[4] = fma(q, ey, vv[4]);
                            vv[5] = fma(q, ez, vv[5]);
                        }
#pragma unroll
                        for (int c = 0; c < 6; ++c) v[c] = vv[c].v.x + vv[c].v.y;
                    } else {
#pragma unroll
                    for (int i = 0; i < CPL; ++i) {
                        // correctly rounded displacement (grid-split hi parts subtract exactly)
                        const float X = (h0.x - ch[i].x) + (h0.w - cl[i].x);
                        const float Y = (h0.y - ch[i].y) + (h1.x - cl[i].y);
                        const float Z = (h0.z - ch[i].z) + (h1.y - cl[i].z);
                        float T, Tl;
                        boys_arg_f32(rq.x, X, Y, Z, T, Tl);
                        float F[L + 2];
                        boys_f32<L + 1>(T, F, tab, Tl);
                        float Fn[L + 2];
                        {
                            float sc = rq.y;
                            const float m2rho = -2.0f * rq.x;
#pragma unroll
                            for (int n = 0; n <= L + 1; ++n) {
                                Fn[n] = sc * F[n];
                                sc *= m2rho;
                            }
                        }
                        float R[NH1];
                        hermite_R_u<L + 1, float>(R, Fn, X, Y, Z);
                        float e0 = 0.f, ex = 0.f, ey = 0.f, ez = 0.f, hx = 0.f, hy = 0.f, hz = 0.f;
#pragma unroll
                        for (int tt = 0; tt <= L; ++tt)
#pragma unroll
                            for (int uu = 0; uu <= L; ++uu)
#pragma unroll
                                for (int ww = 0; ww <= L; ++ww) {
                                    if (tt + uu + ww > L) continue;
                                    const int k = hidx(tt, uu, ww);
                                    const float4 d = r[2 + k];
                                    e0 = fmaf(d.x, R[k], e0);
                                    ex = fmaf(d.x, R[hidx(tt + 1, uu, ww)], ex);
                                    ey = fmaf(d.x, R[hidx(tt, uu + 1, ww)], ey);
                                    ez = fmaf(d.x, R[hidx(tt, uu, ww + 1)], ez);
                                    hx = fmaf(d.y, R[k], hx);
                                    hy = fmaf(d.z, R[k], hy);
                                    hz = fmaf(d.w, R[k], hz);
                                }
                        const float q = ch[i].w;
                        bp[i][0] = fmaf(q, ex, bp[i][0]);
                        bp[i][1] = fmaf(q, ey, bp[i][1]);
                        bp[i][2] = fmaf(q, ez, bp[i][2]);
                        bp[i][3] -= e0;
                        v[0] = fmaf(q, hx, v[0]);
                        v[1] = fmaf(q, hy, v[1]);
                        v[2] = fmaf(q, hz, v[2]);
                        v[3] = fmaf(q, ex, v[3]);
                        v[4] = fmaf(q, ey, v[4]);
                        v[5] = fmaf(q, ez, v[5]);
                    }
                    }
                    // pair sums over the warp's 32 lanes: reduce-scatter of 8 values (6 used), combining
                    // neighbouring lanes first: consecutive region-I charges are the atoms of one water, so
                    // the partial sums cancel early and stay small (a 16-apart pairing first sums unrelated
                    // monopoles and leaves the FP32 rounding of large partials in the small total).  Lanes
                    // 0..7 end with value vi = bits (0, 1, 2) of the lane number.
                    float w4[4], w2[2], w1;
                    {
                        const bool up = lane & 1;
#pragma unroll
                        for (int i = 0; i < 4; ++i) {
                            const float keep = up ? v[i + 4] : v[i], send = up ? v[i] : v[i + 4];
                            w4[i] = keep + __shfl_xor_sync(FULL, send, 1);
                        }
                        const bool up2 = lane & 2;
#pragma unroll
                        for (int i = 0; i < 2; ++i) {
                            const float keep = up2 ? w4[i + 2] : w4[i], send = up2 ? w4[i] : w4[i + 2];
                            w2[i] = keep + __shfl_xor_sync(FULL, send, 2);
                        }
                        const bool up4 = lane & 4;
                        {
                            const float keep = up4 ? w2[1] : w2[0], send = up4 ? w2[0] : w2[1];
                            w1 = keep + __shfl_xor_sync(FULL, send, 4);
                        }
                        w1 += __shfl_xor_sync(FULL, w1, 8);
                        w1 += __shfl_xor_sync(FULL, w1, 16);
                    }
                    const int vi = (lane & 1) * 4 + ((lane >> 1) & 1) * 2 + ((lane >> 2) & 1);
                    if (lane < 8 && vi < 6) {
                        // compensated shared-memory atomic: the old value gives the rounding error exactly
                        float *hp = &ps_h[s][p * 8 + vi];
                        const float old = atomicAdd(hp, w1);
                        const float sum = old + w1, bv = sum - old;
                        atomicAdd(&ps_l[s][p * 8 + vi], (old - (sum - bv)) + (w1 - bv));
                    }
                }
                if constexpr (PACK) {
#pragma unroll
                    for (int j = 0; j < CP; ++j)
#pragma unroll
                        for (int c = 0; c < 4; ++c) {
                            df_add(ah[2 * j][c], al[2 * j][c], bp2[j][c].v.x);
                            df_add(ah[2 * j + 1][c], al[2 * j + 1][c], bp2[j][c].v.y);
                        }
                } else {
#pragma unroll
                    for (int i = 0; i < CPL; ++i)
#pragma unroll
                        for (int c = 0; c < 4; ++c) df_add(ah[i][c], al[i][c], bp[i][c]);
                }
                __syncthreads();  // batch b read by all warps; its pair sums complete
                if ((int)threadIdx.x < nb * 6) {
                    // each of these threads reads one sum and clears it for batch b + 2 (slots 6, 7 of a
                    // pair are never written)
                    const int pp = (int)threadIdx.x / 6, vv = (int)threadIdx.x % 6, o = pp * 8 + vv;
                    atomicAdd(psum + (size_t)(b * NB + pp) * 6 + vv, (double)ps_h[s][o] + (double)ps_l[s][o]);
                    ps_h[s][o] = ps_l[s][o] = 0.0f;
                }
#pragma unroll
                for (int i = 0; i < PF; ++i) {
                    const int idx = (int)threadIdx.x + i * CL_NT;
                    if (idx < nbn * R4) put(s ^ 1, idx, pf[i]);
                }
                __syncthreads();  // batch b + 1 staged
            }
#pragma unroll
            for (int i = 0; i < CPL; ++i) {
                const int j = cbeg + (int)threadIdx.x + i * CL_NT;
                if (j < cend) {
#pragma unroll
                    for (int c = 0; c < 4; ++c)
                        atomicAdd(J.gchg + 4 * (size_t)j + c, (double)ah[i][c] + (double)al[i][c]);
                }
            }
        }
        if (!counter) break;
        __syncthreads();  // every thread has read s_item and left this item's shared buffers
    }
}

// Pair gradients from the per-pair charge sums (FP64), summed per shell pair and atom.  Each job's
// thread range starts at a multiple of 32, so a warp never mixes jobs.
template <int LA, int LB>
__global__ void __launch_bounds__(128)
k_cl_pairs(ClJob one, const ClJob *__restrict__ jobs, int njob, int nthr)
{
    const int t = (int)(blockIdx.x * blockDim.x + threadIdx.x);
    if (t - (int)(threadIdx.x & 31) >= nthr) return;  // warp-uniform
    const int lane = threadIdx.x & 31;
    const ClJob &J = jobs ? jobs[cl_job_by_thread(jobs, njob, t)] : one;
    const int i = J.pp_begin + (t - J.thr0);
    const PPLane pl = load_pp(J.bd, i, J.pp_end);
    double g[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    if (pl.active) {
        const double *sm = J.psum + (size_t)(i - J.pp_begin) * 6;
        const double aop = pl.a * pl.ip, bop = pl.b * pl.ip;
#pragma unroll
        for (int x = 0; x < 3; ++x) {
            g[x] = -(sm[x] + aop * sm[3 + x]);
            g[3 + x] = sm[x] - bop * sm[3 + x];
        }
    }
    bool take[5], head;
    seg_setup(pl.active ? pl.s : -1 - lane, lane, take, head);
#pragma unroll
    for (int k = 0; k < 6; ++k) g[k] = seg_reduce(g[k], take);
    if (head && pl.active) {
#pragma unroll
        for (int x = 0; x < 3; ++x) {
            atomicAdd(J.gqm + 3 * pl.atomA + x, g[x]);
            atomicAdd(J.gqm + 3 * pl.atomB + x, g[3 + x]);
        }
    }
}

// The three kernels of one class over the jobs (records, sweep, pair gradients); jobs == nullptr:
// the single job `one`, its sweep one block per item (fine-grained blocks of CL_BPB batches: the
// class kernels are launched together, highest class first, and the block scheduler packs their
// blocks onto the SMs as others finish); otherwise a persistent sweep of nsm * MINB blocks taking
// items from *counter (cleared here).
template <int LA, int LB, int CPL, int MINB>
static cudaError_t launch_cl(const ClJob &one, const ClJob *jobs, int njob, int nthr, int nitems, int *counter,
                             const float *boys, int nsm, cudaStream_t st)
{
    if (nthr <= 0 || nitems <= 0) return cudaSuccess;
    cudaError_t e;
    if constexpr (rec_tab(LA + LB)) {
        if (nthr % 32) return cudaErrorInvalidValue;  // every job's pairs are padded to 32
        static bool attr = false;
        if (!attr) {
            if ((e = cudaFuncSetAttribute(k_cl_records_tab<LA, LB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)rec_smem<LA, LB>())) != cudaSuccess)
                return e;
            attr = true;
        }
        k_cl_records_tab<LA, LB>
            <<<nthr / 32, 128 * rec_split(LA + LB), rec_smem<LA, LB>(), st>>>(one, jobs, njob, nthr);
    } else {
        k_cl_records<LA, LB><<<(nthr + 127) / 128, 128, 0, st>>>(one, jobs, njob, nthr);
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const float *tab = boys + (size_t)(LA + LB + 1) * BOYS_TAB_F;
    if (counter) {
        if ((e = cudaMemsetAsync(counter, 0, sizeof(int), st)) != cudaSuccess) return e;
        const int grid = std::min(nitems, MINB * std::max(nsm, 1));
        k_vgrad_cl<LA, LB, CPL, MINB><<<grid, CL_NT, 0, st>>>(one, jobs, njob, nitems, counter, tab);
    } else {
        k_vgrad_cl<LA, LB, CPL, MINB><<<nitems, CL_NT, 0, st>>>(one, jobs, njob, nitems, nullptr, tab);
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    k_cl_pairs<LA, LB><<<(nthr + 127) / 128, 128, 0, st>>>(one, jobs, njob, nthr);
    return cudaGetLastError();
}

template <int LA, int LB>
cudaError_t VgradF32<LA, LB>::run(const BasisDev &bd, const RegionDev &rg, int pp_begin, int pp_end, int ch_begin,
                                  int ch_end, const float *boys, const double *dm, double *gqm, double *gchg,
                                  int *err,
                                  int nsm, int variant, int nslice, ClScratch cl,
                                  cudaStream_t st)
{
    // charge-lane sweep: (charges per lane, blocks per SM) of variant 0 and 1 (cl_variant)
    (void)err;
    (void)nslice;
    if (!cl.rec || !cl.psum) return cudaErrorInvalidValue;
    ClJob one{};
    one.bd = bd;
    one.rg = rg;
    one.dm = dm;
    one.rec = cl.rec;
    one.psum = cl.psum;
    one.gqm = gqm;
    one.gchg = gchg;
    one.pp_begin = pp_begin;
    one.pp_end = pp_end;
    one.ch_begin = ch_begin;
    one.ch_end = ch_end;
    constexpr int L = LA + LB;
    cl_decompose(L, variant, pp_end - pp_begin, ch_end - ch_begin, rg.ncls, one.gx, one.ntile);
    const int nthr = (pp_end - pp_begin + 31) / 32 * 32, nitems = one.gx * one.ntile;
    if (variant == 1) {
        if constexpr (cl_variant(L, 1, 0) > 0)
            return launch_cl<LA, LB, cl_variant(L, 1, 0), cl_variant(L, 1, 1)>(one, nullptr, 1, nthr, nitems,
                                                                               nullptr, boys, nsm, st);
    }
    return launch_cl<LA, LB, cl_variant(L, 0, 0), cl_variant(L, 0, 1)>(one, nullptr, 1, nthr, nitems, nullptr, boys,
                                                                       nsm, st);
}

template <int LA, int LB>
cudaError_t VgradF32<LA, LB>::run_jobs(const ClJob *jobs, int njob, int nthr, int nitems, int *counter,
                                       const float *boys, int variant, int nsm, cudaStream_t st)
{
    constexpr int L = LA + LB;
    const ClJob none{};
    if (variant == 1) {
        if constexpr (cl_variant(L, 1, 0) > 0)
            return launch_cl<LA, LB, cl_variant(L, 1, 0), cl_variant(L, 1, 1)>(none, jobs, njob, nthr, nitems,
                                                                               counter, boys, nsm, st);
    }
    return launch_cl<LA, LB, cl_variant(L, 0, 0), cl_variant(L, 0, 1)>(none, jobs, njob, nthr, nitems, counter, boys,
                                                                       nsm, st);
}

template struct VgradF32<la_of_class(QMMM_SPLIT_CLASS), lb_of_class(QMMM_SPLIT_CLASS)>;

#else  // the dispatcher

void cl_decompose(int L, int variant, int npair, int nch, int ncls, int &gx, int &ntile)
{
    const int cpl = (variant == 1 && cl_variant(L, 1, 0) > 0) ? cl_variant(L, 1, 0) : cl_variant(L, 0, 0);
    const int tile = CL_NT * cpl, nb = cl_batch(L);
    const int nbatch = (npair + nb - 1) / nb;
    gx = std::max(1, (nbatch + CL_BPB - 1) / CL_BPB);
    // a tile never spans two width classes: at most one partial tile per class boundary
    ntile = nch > 0 ? (nch + tile - 1) / tile + std::max(ncls, 1) - 1 : 0;
}

cudaError_t launch_vgrad_f32(const BasisDev &b, const RegionDev &r, int cls, int pp_begin, int pp_end,
                             int ch_begin, int ch_end, const float *boys, const double *dm, double *gqm,
                             double *gchg, int *err, int nsm, int variant, int nslice, ClScratch cl,
                             cudaStream_t st)
{
    if (pp_end <= pp_begin || ch_end <= ch_begin) return cudaSuccess;
    return dispatch_class<VgradF32>(cls, b, r, pp_begin, pp_end, ch_begin, ch_end, boys, dm, gqm, gchg, err, nsm,
                                    variant, nslice, cl, st);
}

namespace {
template <int LA, int LB>
struct VgradJobs {
    static cudaError_t run(const ClJob *jobs, int njob, int nthr, int nitems, int *counter, const float *boys,
                           int variant, int nsm, cudaStream_t st)
    {
        return VgradF32<LA, LB>::run_jobs(jobs, njob, nthr, nitems, counter, boys, variant, nsm, st);
    }
};
}  // namespace

cudaError_t launch_vgrad_cl_jobs(int cls, const ClJob *jobs, int njob, int nthr, int nitems, int *counter,
                                 const float *boys, int variant, int nsm, cudaStream_t st)
{
    if (njob <= 0 || nitems <= 0) return cudaSuccess;
    return dispatch_class<VgradJobs>(cls, jobs, njob, nthr, nitems, counter, boys, variant, nsm, st);
}

#endif

}  // namespace qmmm
