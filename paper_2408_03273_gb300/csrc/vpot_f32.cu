// vpot_f32.cu -- region-I matrix of Eq. 9, mixed precision.
//
// Same tile layout as the FP64 kernel.  The per-(primitive pair, charge) work -- the Boys
// function, the Hermite R recursion and the charge sum -- runs in FP32; everything done once per
// primitive pair (Gaussian product, prefactors, E-contraction, reductions) stays FP64.
//   * Positions enter as FP32 hi/lo pairs relative to the QM centre: X_PC = (P_hi - C_hi) +
//     (P_lo - C_lo), so the difference is accurate to FP32 rounding of X_PC itself.
//   * Charge sums use FP32 partials over 16 charges folded into a double-float (hi, lo) pair by
//     an error-free two-sum, so summation error does not grow with the number of charges.
//   * The FP32 Boys table lives in shared memory (staged with the charges by TMA), with an odd
//     row stride so that lanes reading different rows hit different banks.
#include "pp_tile.cuh"

namespace qmmm {

template <int LA, int LB>
struct VpotF32 {
    static cudaError_t run(const BasisDev &bd, const RegionDev &rg, int pp_begin, int pp_end, int ch_begin,
                           int ch_end, const float *boys, double *V, int *err, int nsm, int variant, int nslice,
                           size_t vstride,
                           cudaStream_t st);
    static cudaError_t run_jobs(const VJob *jobs, int njob, int nblk, int maxch, const float *boys, int *err,
                                int variant, cudaStream_t st);
};

#ifdef QMMM_SPLIT_CLASS  // one angular class per compilation

constexpr int FOLD = 16;

// A block is (bx, slice) of a job: with jobs == nullptr the single job `one` over the grid
// (gx, ns) = (gridDim.x, gridDim.y); otherwise block blockIdx.x of the flat range of all jobs,
// job j owning blocks [blk0, blk0 + gx ns) (the batched form over many frames).
template <int LA, int LB, int NT>
__global__ void __launch_bounds__(NT, 1)
k_vpot_f32(VJob one, const VJob *__restrict__ jobs, int njob, const float *__restrict__ boys_g, unsigned boys_bytes,
           size_t vstride, int *err)
{
    int bx = (int)blockIdx.x, by = (int)blockIdx.y;
    if (jobs) {
        int lo = 0, hi = njob - 1;  // the last job with blk0 <= blockIdx.x
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (__ldg(&jobs[mid].blk0) <= (int)blockIdx.x) lo = mid;
            else hi = mid - 1;
        }
        one = jobs[lo];
        const int local = (int)blockIdx.x - one.blk0;
        bx = local % one.gx;
        by = local / one.gx;
    }
    const BasisDev &bd = one.bd;
    const RegionDev &rg = one.rg;
    const int pp_begin = one.pp_begin, pp_end = one.pp_end, gx = one.gx;
    double *__restrict__ V = one.V + (size_t)by * vstride;  // per-slice partial V when the charges are split
    constexpr int L = LA + LB, NH = nherm(L), NA = ncart(LA), NB = ncart(LB);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ uint64_t bar;
    int ch_begin, ch_end;
    {
        // this block row's slice of the charge chunk (several slices spread small systems over more SMs)
        const int per = (one.ch_end - one.ch_begin + one.ns - 1) / one.ns;
        ch_begin = one.ch_begin + by * per;
        ch_end = min(one.ch_end, ch_begin + per);
    }
    if (ch_begin >= ch_end) return;
    const int nch = ch_end - ch_begin;
    float4 *chi = reinterpret_cast<float4 *>(smem_raw);
    float4 *clo = chi + nch;
    float *tab = reinterpret_cast<float *>(clo + nch);
    {
        Seg s[3] = {{chi, rg.chg_hi + ch_begin, (unsigned)(nch * sizeof(float4))},
                    {clo, rg.chg_lo + ch_begin, (unsigned)(nch * sizeof(float4))},
                    {tab, boys_g, boys_bytes}};
        if (!stage_segments(s, 3, &bar, err)) return;
    }

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    const int ntile = (pp_end - pp_begin + 31) >> 5;
    for (int tile = bx * nwarp + warp; tile < ntile; tile += gx * nwarp) {
        const PPLane pl = load_pp(bd, pp_begin + tile * 32 + lane, pp_end);
        float Ph[3], Plo[3];
#pragma unroll
        for (int x = 0; x < 3; ++x) {
            const double d = pl.P[x] - rg.centre[x];
            split_grid(d, Ph[x], Plo[x]);
        }
        float Wh[NH], Wl[NH];
#pragma unroll
        for (int k = 0; k < NH; ++k) Wh[k] = Wl[k] = 0.0f;

        for (int c = 0; c < rg.ncls; ++c) {
            const int lo = max(__ldg(rg.cls_off + c), ch_begin) - ch_begin;
            const int hi = min(__ldg(rg.cls_off + c + 1), ch_end) - ch_begin;
            if (lo >= hi) continue;
            const double kap = __ldg(rg.cls_kappa + c);
            const double td = kap > 0.0 ? kap / (pl.p + kap) : 1.0;
            const float rho = (float)(pl.p * td), m2rho = -2.0f * rho, sq = (float)sqrt(td);
            for (int j0 = lo; j0 < hi; j0 += FOLD) {
                const int j1 = min(hi, j0 + FOLD);
                float Wt[NH];
#pragma unroll
                for (int k = 0; k < NH; ++k) Wt[k] = 0.0f;
                for (int j = j0; j < j1; ++j) {
                    const float4 ch = chi[j], cl = clo[j];
                    const float X = (Ph[0] - ch.x) + (Plo[0] - cl.x);
                    const float Y = (Ph[1] - ch.y) + (Plo[1] - cl.y);
                    const float Z = (Ph[2] - ch.z) + (Plo[2] - cl.z);
                    float T, Tl;
                    boys_arg_f32(rho, X, Y, Z, T, Tl);
                    float F[L + 1];
                    boys_f32<L>(T, F, tab, Tl);
                    float Fn[L + 1];
                    float sc = ch.w * sq;
#pragma unroll
                    for (int n = 0; n <= L; ++n) {
                        Fn[n] = sc * F[n];
                        sc *= m2rho;
                    }
                    float R[NH];
                    hermite_R_u<L, float>(R, Fn, X, Y, Z);
#pragma unroll
                    for (int k = 0; k < NH; ++k) Wt[k] += R[k];
                }
#pragma unroll
                for (int k = 0; k < NH; ++k) df_add(Wh[k], Wl[k], Wt[k]);
            }
        }
        double W[NH];
#pragma unroll
        for (int k = 0; k < NH; ++k) W[k] = (double)Wh[k] + (double)Wl[k];

        double Ex[LA + 1][LB + 1][L + 1], Ey[LA + 1][LB + 1][L + 1], Ez[LA + 1][LB + 1][L + 1];
        hermite_E<LA, LB, double>(Ex, pl.P[0] - pl.A[0], pl.P[0] - pl.B[0], 0.5 * pl.ip);
        hermite_E<LA, LB, double>(Ey, pl.P[1] - pl.A[1], pl.P[1] - pl.B[1], 0.5 * pl.ip);
        hermite_E<LA, LB, double>(Ez, pl.P[2] - pl.A[2], pl.P[2] - pl.B[2], 0.5 * pl.ip);
        const double coef = -TWO_PI * pl.ip * pl.cab;

        bool take[5], head;
        seg_setup(pl.active ? pl.s : -1 - lane, lane, take, head);
        const bool mirror = pl.sp.shA != pl.sp.shB;
#pragma unroll
        for (int ia = 0; ia < NA; ++ia) {
#pragma unroll
            for (int ib = 0; ib < NB; ++ib) {
                const int ax = cart_lx(LA, ia), ay = cart_ly(LA, ia), az = cart_lz(LA, ia);
                const int bx = cart_lx(LB, ib), by = cart_ly(LB, ib), bz = cart_lz(LB, ib);
                double v = 0.0;
#pragma unroll
                for (int t = 0; t <= ax + bx; ++t)
#pragma unroll
                    for (int u = 0; u <= ay + by; ++u) {
                        const double exy = Ex[ax][bx][t] * Ey[ay][by][u];
#pragma unroll
                        for (int w = 0; w <= az + bz; ++w) v += exy * Ez[az][bz][w] * W[hidx(t, u, w)];
                    }
                v = seg_reduce(coef * v, take);
                if (head && pl.active) {
                    const size_t r = pl.sp.aoA + ia, c = pl.sp.aoB + ib;
                    atomicAdd(V + r * bd.nao + c, v);
                    if (mirror) atomicAdd(V + c * bd.nao + r, v);
                }
            }
        }
    }
}

// bytes of one order's FP32 Boys table (what a block stages)
inline unsigned boys32_bytes() { return (unsigned)(BOYS_TAB_F * sizeof(float)); }

template <int LA, int LB, int NT>
static cudaError_t launch_nt(const BasisDev &bd, const RegionDev &rg, int pp_begin, int pp_end, int ch_begin,
                             int ch_end, const float *boys, double *V, int *err, int nsm, int nslice,
                             size_t vstride, cudaStream_t st)
{
    const unsigned tb = boys32_bytes();
    const int per = (ch_end - ch_begin + nslice - 1) / nslice;
    const size_t smem = (size_t)per * 2 * sizeof(float4) + tb;
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_vpot_f32<LA, LB, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)(CHUNK_F32 * 2 * sizeof(float4) + tb));
        if (e != cudaSuccess) return e;
        attr = true;
    }
    const int ntile = (pp_end - pp_begin + 31) / 32;
    int grid = (ntile + NT / 32 - 1) / (NT / 32);
    if (grid > nsm) grid = nsm;
    if (grid < 1) return cudaSuccess;
    VJob one{};
    one.bd = bd;
    one.rg = rg;
    one.V = V;
    one.pp_begin = pp_begin;
    one.pp_end = pp_end;
    one.ch_begin = ch_begin;
    one.ch_end = ch_end;
    one.gx = grid;
    one.ns = nslice;
    k_vpot_f32<LA, LB, NT><<<dim3(grid, nslice), NT, smem, st>>>(one, nullptr, 0, boys + (size_t)(LA + LB) * BOYS_TAB_F,
                                                                 tb, vstride, err);
    return cudaGetLastError();
}

// every job's blocks in one launch; maxch: the most charges of one block's slice over the jobs
template <int LA, int LB, int NT>
static cudaError_t launch_nt_jobs(const VJob *jobs, int njob, int nblk, int maxch, const float *boys, int *err,
                                  cudaStream_t st)
{
    const unsigned tb = boys32_bytes();
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_vpot_f32<LA, LB, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)(CHUNK_F32 * 2 * sizeof(float4) + tb));
        if (e != cudaSuccess) return e;
        attr = true;
    }
    if (maxch > CHUNK_F32) return cudaErrorInvalidValue;
    const size_t smem = (size_t)maxch * 2 * sizeof(float4) + tb;
    const VJob none{};
    k_vpot_f32<LA, LB, NT><<<nblk, NT, smem, st>>>(none, jobs, njob, boys + (size_t)(LA + LB) * BOYS_TAB_F, tb, 0,
                                                   err);
    return cudaGetLastError();
}

template <int LA, int LB>
cudaError_t VpotF32<LA, LB>::run(const BasisDev &bd, const RegionDev &rg, int pp_begin, int pp_end, int ch_begin,
                                 int ch_end, const float *boys, double *V, int *err, int nsm, int variant,
                                 int nslice, size_t vstride,
                                 cudaStream_t st)
{
    constexpr int W = sweep_wide_threads(SW_VPOT_F32, class_of(LA, LB));
    if constexpr (W > 0)
        if (variant == 1)
            return launch_nt<LA, LB, W>(bd, rg, pp_begin, pp_end, ch_begin, ch_end, boys, V, err, nsm, nslice,
                                        vstride, st);
    return launch_nt<LA, LB, 256>(bd, rg, pp_begin, pp_end, ch_begin, ch_end, boys, V, err, nsm, nslice, vstride, st);
}

template <int LA, int LB>
cudaError_t VpotF32<LA, LB>::run_jobs(const VJob *jobs, int njob, int nblk, int maxch, const float *boys, int *err,
                                      int variant, cudaStream_t st)
{
    constexpr int W = sweep_wide_threads(SW_VPOT_F32, class_of(LA, LB));
    if constexpr (W > 0)
        if (variant == 1) return launch_nt_jobs<LA, LB, W>(jobs, njob, nblk, maxch, boys, err, st);
    return launch_nt_jobs<LA, LB, 256>(jobs, njob, nblk, maxch, boys, err, st);
}

template struct VpotF32<la_of_class(QMMM_SPLIT_CLASS), lb_of_class(QMMM_SPLIT_CLASS)>;

#else  // the dispatcher

cudaError_t launch_vpot_f32(const BasisDev &b, const RegionDev &r, int cls, int pp_begin, int pp_end,
                            int ch_begin, int ch_end, const float *boys, double *V, int *err, int nsm, int variant,
                            int nslice, size_t vstride,
                            cudaStream_t st)
{
    if (pp_end <= pp_begin || ch_end <= ch_begin) return cudaSuccess;
    return dispatch_class<VpotF32>(cls, b, r, pp_begin, pp_end, ch_begin, ch_end, boys, V, err, nsm, variant,
                                   nslice, vstride, st);
}

namespace {
template <int LA, int LB>
struct VpotJobs {
    static cudaError_t run(const VJob *jobs, int njob, int nblk, int maxch, const float *boys, int *err, int variant,
                           cudaStream_t st)
    {
        return VpotF32<LA, LB>::run_jobs(jobs, njob, nblk, maxch, boys, err, variant, st);
    }
};
}  // namespace

cudaError_t launch_vpot_f32_jobs(int cls, const VJob *jobs, int njob, int nblk, int maxch, const float *boys,
                                 int *err, int variant, cudaStream_t st)
{
    if (njob <= 0 || nblk <= 0) return cudaSuccess;
    return dispatch_class<VpotJobs>(cls, jobs, njob, nblk, maxch, boys, err, variant, st);
}

#endif

}  // namespace qmmm
