// vpot_f64.cu -- region-I one-electron matrix of Eq. 9 in FP64 (McMurchie-Davidson).
//
//   V_{ab} = - sum_{C in I} q_C (2 pi/p) sqrt(kappa_C/(p+kappa_C)) c_a c_b K_AB
//            sum_tuv E^x_t E^y_u E^z_v R_tuv(rho_C, P - C)
//
// A warp owns 32 primitive pairs of one angular class; the block stages a chunk of region-I
// charges (x, y, z, q) into shared memory with one TMA bulk copy, every lane sweeps all of them
// (shared-memory broadcast) and accumulates the Hermite sums W_tuv = sum_C q_C s_C R_tuv in
// registers.  Charges are grouped by Gaussian width so that rho and sqrt(kappa/(p+kappa)) are
// computed once per (primitive pair, width class).  The E-contraction runs once per primitive
// pair; primitive pairs of a shell pair are summed by a segmented warp-shuffle reduction and the
// head lane adds the block into V (and its mirror).  A shell pair spans at most two tiles when
// it has at most 32 primitive pairs, so at most two additions reach any element: the result does
// not depend on scheduling.
#include <algorithm>

#include "pp_tile.cuh"

namespace qmmm {

template <int LA, int LB>
struct VpotF64 {
    static cudaError_t run(const BasisDev &bd, const RegionDev &rg, int pp_begin, int pp_end, int ch_begin,
                           int ch_end, const double *boys, double *V, int *err, int nsm, int variant, int nslice,
                           size_t vstride,
                           cudaStream_t st);
};

#ifdef QMMM_SPLIT_CLASS  // one angular class per compilation

template <int LA, int LB, int NT>
__global__ void __launch_bounds__(NT, 1)
k_vpot_f64(BasisDev bd, RegionDev rg, int pp_begin, int pp_end, int ch_begin, int ch_end,
           const double *__restrict__ boys, double *__restrict__ V, size_t vstride, int *err)
{
    V += (size_t)blockIdx.y * vstride;  // per-slice partial V when the charges are split
    constexpr int L = LA + LB, NH = nherm(L), NA = ncart(LA), NB = ncart(LB);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ uint64_t bar;
    double4_32a *chg = reinterpret_cast<double4_32a *>(smem_raw);
    {
        // this block row's slice of the charge chunk (gridDim.y > 1 spreads small systems over more SMs)
        const int per = (ch_end - ch_begin + (int)gridDim.y - 1) / (int)gridDim.y;
        ch_begin += (int)blockIdx.y * per;
        ch_end = min(ch_end, ch_begin + per);
    }
    if (ch_begin >= ch_end) return;
    const int nch = ch_end - ch_begin;
    if (!stage_to_smem(chg, rg.chg + ch_begin, (unsigned)(nch * sizeof(double4_32a)), &bar, err)) return;

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    const int ntile = (pp_end - pp_begin + 31) >> 5;
    for (int tile = blockIdx.x * nwarp + warp; tile < ntile; tile += gridDim.x * nwarp) {
        const PPLane pl = load_pp(bd, pp_begin + tile * 32 + lane, pp_end);
        double W[NH];
#pragma unroll
        for (int k = 0; k < NH; ++k) W[k] = 0.0;

        for (int c = 0; c < rg.ncls; ++c) {
            const int lo = max(__ldg(rg.cls_off + c), ch_begin) - ch_begin;
            const int hi = min(__ldg(rg.cls_off + c + 1), ch_end) - ch_begin;
            if (lo >= hi) continue;
            const double kap = __ldg(rg.cls_kappa + c);
            const double t = kap > 0.0 ? kap / (pl.p + kap) : 1.0;
            const double rho = pl.p * t, m2rho = -2.0 * rho, sq = sqrt(t);
            for (int j = lo; j < hi; ++j) {
                const double4_32a ch = chg[j];
                const double X = pl.P[0] - ch.x, Y = pl.P[1] - ch.y, Z = pl.P[2] - ch.z;
                const double T = rho * (X * X + Y * Y + Z * Z);
                double F[L + 1];
                boys_f64<L>(T, F, boys);
                double Fn[L + 1];
                double sc = ch.w * sq;
#pragma unroll
                for (int n = 0; n <= L; ++n) {
                    Fn[n] = sc * F[n];
                    sc *= m2rho;
                }
                double R[NH];
                hermite_R<L, double>(R, Fn, X, Y, Z);
#pragma unroll
                for (int k = 0; k < NH; ++k) W[k] += R[k];
            }
        }

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

template <int LA, int LB, int NT>
static cudaError_t launch_nt(const BasisDev &bd, const RegionDev &rg, int pp_begin, int pp_end, int ch_begin,
                             int ch_end, const double *boys, double *V, int *err, int nsm, int nslice,
                             size_t vstride, cudaStream_t st)
{
    const int per = (ch_end - ch_begin + nslice - 1) / nslice;
    const size_t smem = std::max((size_t)per * sizeof(double4_32a), SWEEP_SMEM_MIN);
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_vpot_f64<LA, LB, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)(CHUNK_F64 * sizeof(double4_32a)));
        if (e != cudaSuccess) return e;
        attr = true;
    }
    const int ntile = (pp_end - pp_begin + 31) / 32;
    int grid = (ntile + NT / 32 - 1) / (NT / 32);
    if (grid > nsm) grid = nsm;
    if (grid < 1) return cudaSuccess;
    k_vpot_f64<LA, LB, NT><<<dim3(grid, nslice), NT, smem, st>>>(bd, rg, pp_begin, pp_end, ch_begin, ch_end, boys,
                                                                 V, vstride, err);
    return cudaGetLastError();
}

template <int LA, int LB>
cudaError_t VpotF64<LA, LB>::run(const BasisDev &bd, const RegionDev &rg, int pp_begin, int pp_end, int ch_begin,
                                 int ch_end, const double *boys, double *V, int *err, int nsm, int variant,
                                 int nslice, size_t vstride,
                                 cudaStream_t st)
{
    constexpr int W = sweep_wide_threads(SW_VPOT_F64, class_of(LA, LB));
    if constexpr (W > 0)
        if (variant == 1)
            return launch_nt<LA, LB, W>(bd, rg, pp_begin, pp_end, ch_begin, ch_end, boys, V, err, nsm, nslice,
                                        vstride, st);
    return launch_nt<LA, LB, 256>(bd, rg, pp_begin, pp_end, ch_begin, ch_end, boys, V, err, nsm, nslice, vstride, st);
}

template struct VpotF64<la_of_class(QMMM_SPLIT_CLASS), lb_of_class(QMMM_SPLIT_CLASS)>;

#else  // the dispatcher

cudaError_t launch_vpot_f64(const BasisDev &b, const RegionDev &r, int cls, int pp_begin, int pp_end,
                            int ch_begin, int ch_end, const double *boys, double *V, int *err, int nsm,
                            int variant, int nslice, size_t vstride,
                            cudaStream_t st)
{
    if (pp_end <= pp_begin || ch_end <= ch_begin) return cudaSuccess;
    return dispatch_class<VpotF64>(cls, b, r, pp_begin, pp_end, ch_begin, ch_end, boys, V, err, nsm, variant,
                                   nslice, vstride, st);
}

#endif

}  // namespace qmmm
