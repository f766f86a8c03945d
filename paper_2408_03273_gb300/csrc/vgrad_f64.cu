// vgrad_f64.cu -- adjoint of the region-I term: gradient of E_I = sum gamma_{mu nu} V_{mu nu}
// (Eq. 9) with respect to the QM centres, the MM image positions and the MM charges, FP64.
//
// Per primitive pair the density is folded into Hermite coefficients once,
//   D0_tuv = sum_ab g_ab E^x_t E^y_u E^z_v,   Dx_tuv = sum_ab g_ab E'^x_t E^y_u E^z_v, ...
// with g_ab the density element (plus its mirror) times the pair prefactor and
//   E'^{ij}_t = dE^{ij}_t / dX_AB = 2a E^{i+1,j}_t - i E^{i-1,j}_t - (a/p) E^{ij}_{t-1}.
// Moving A shifts P by a/p, so with e_a = sum D0_tuv R_{tuv + 1_a} and d_a = sum Da_tuv R_tuv
// (R recomputed up to L+1 for every charge, never stored):
//   dI/dA_a = d_a + (a/p) e_a,   dI/dB_a = -d_a + (b/p) e_a,   dI/dC_a = -e_a,
// and E contains -q_C I.  The d_a enter only through sum_C q_C d_a(C) = sum Da_tuv S_tuv with
// S_tuv = sum_C q_C R_tuv, so up to L = 4 the sweep accumulates S (NH terms per charge instead
// of the 3 NH of the three contractions) and Da is formed and contracted once per pair after it
// (contract_dA); for L >= 5 the three contractions stay in the loop (see CSUM).
// Per-pair sums over charges stay in registers; per-charge sums over the
// 32 primitive pairs of a tile use a warp butterfly and go to shared-memory accumulators that
// are flushed to global memory once per block.
#include <algorithm>

#include "pp_tile.cuh"

namespace qmmm {

template <int LA, int LB>
struct VgradF64 {
    static cudaError_t run(const BasisDev &bd, const RegionDev &rg, int pp_begin, int pp_end, int ch_begin,
                           int ch_end, const double *boys, const double *dm, double *gqm, double *gchg, int *err,
                           int nsm, int variant, int nslice,
                           cudaStream_t st);
};

#ifdef QMMM_SPLIT_CLASS  // one angular class per compilation

template <int LA, int LB, int NT>
__global__ void __launch_bounds__(NT, 1)
k_vgrad_f64(BasisDev bd, RegionDev rg, int pp_begin, int pp_end, int ch_begin, int ch_end,
            const double *__restrict__ boys, const double *__restrict__ dm, double *__restrict__ gqm,
            double *__restrict__ gchg, int *err)
{
    constexpr int L = LA + LB, NH = nherm(L), NH1 = nherm(L + 1);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ uint64_t bar;
    {
        // this block row's slice of the charge chunk (gridDim.y > 1 spreads small systems over more SMs)
        const int per = (ch_end - ch_begin + (int)gridDim.y - 1) / (int)gridDim.y;
        ch_begin += (int)blockIdx.y * per;
        ch_end = min(ch_end, ch_begin + per);
    }
    if (ch_begin >= ch_end) return;
    const int nch = ch_end - ch_begin;
    double4_32a *chg = reinterpret_cast<double4_32a *>(smem_raw);
    double *acc = reinterpret_cast<double *>(smem_raw + (size_t)nch * sizeof(double4_32a));
    for (int k = threadIdx.x; k < 4 * nch; k += blockDim.x) acc[k] = 0.0;
    if (!stage_to_smem(chg, rg.chg + ch_begin, (unsigned)(nch * sizeof(double4_32a)), &bar, err)) return;

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    const int ntile = (pp_end - pp_begin + 31) >> 5;
    for (int tile = blockIdx.x * nwarp + warp; tile < ntile; tile += gridDim.x * nwarp) {
        const PPLane pl = load_pp(bd, pp_begin + tile * 32 + lane, pp_end);
        const double aop = pl.a * pl.ip, bop = pl.b * pl.ip;
        double D0[NH];
        // L <= 4: S_tuv = sum_C q_C R_tuv(P - C), contracted with the centre-A derivative
        // coefficients once per pair after the charge sweep.  L >= 5 (f shells with d or f): S
        // would be read and written every charge from a register file already full, so there
        // the derivative coefficients are contracted per charge (only read in the loop).
        constexpr bool CSUM = L <= 4;
        double S[CSUM ? NH : 1], Dx[CSUM ? 1 : NH], Dy[CSUM ? 1 : NH], Dz[CSUM ? 1 : NH];
        if constexpr (CSUM) {
            fold_density<LA, LB>(pl, bd, dm, D0);
#pragma unroll
            for (int k = 0; k < NH; ++k) S[k] = 0.0;
        } else {
            fold_density_dA<LA, LB, true>(pl, bd, dm, Dx, Dy, Dz, D0);
        }

        double sex = 0, sey = 0, sez = 0, sdx = 0, sdy = 0, sdz = 0;
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
                double F[L + 2];
                boys_f64<L + 1>(T, F, boys);
                double Fn[L + 2];
                double sc = sq;
#pragma unroll
                for (int n = 0; n <= L + 1; ++n) {
                    Fn[n] = sc * F[n];
                    sc *= m2rho;
                }
                double R[NH1];
                hermite_R<L + 1, double>(R, Fn, X, Y, Z);
                double e0 = 0, ex = 0, ey = 0, ez = 0, dx = 0, dy = 0, dz = 0;
                const double q = ch.w;
#pragma unroll
                for (int t = 0; t <= L; ++t)
#pragma unroll
                    for (int u = 0; u <= L - t; ++u)
#pragma unroll
                        for (int w = 0; w <= L - t - u; ++w) {
                            const int k = hidx(t, u, w);
                            e0 += D0[k] * R[k];
                            ex += D0[k] * R[hidx(t + 1, u, w)];
                            ey += D0[k] * R[hidx(t, u + 1, w)];
                            ez += D0[k] * R[hidx(t, u, w + 1)];
                            if constexpr (CSUM) {
                                S[k] += q * R[k];
                            } else {
                                dx += Dx[k] * R[k];
                                dy += Dy[k] * R[k];
                                dz += Dz[k] * R[k];
                            }
                        }
                sex += q * ex; sey += q * ey; sez += q * ez;
                if constexpr (!CSUM) {
                    sdx += q * dx; sdy += q * dy; sdz += q * dz;
                }
                // per-charge sums over the 32 primitive pairs of (dE/dC_x, dE/dC_y, dE/dC_z, dE/dq) =
                // (q e_x, q e_y, q e_z, -e0): halve the four values twice (each lane keeps one
                // component summed over 4 lanes), then a 3-step butterfly; lane 8c ends with
                // component c.  6 FP64 additions instead of 4 full warp sums (20).
                {
                    const double v0 = q * ex, v1 = q * ey, v2 = q * ez, v3 = -e0;
                    const bool up = lane & 16;
                    double k0 = up ? v2 : v0, k1 = up ? v3 : v1;
                    const double s0 = up ? v0 : v2, s1 = up ? v1 : v3;
                    k0 += __shfl_xor_sync(FULL, s0, 16);
                    k1 += __shfl_xor_sync(FULL, s1, 16);
                    const bool up8 = lane & 8;
                    double k = up8 ? k1 : k0;
                    k += __shfl_xor_sync(FULL, up8 ? k0 : k1, 8);
                    k += __shfl_xor_sync(FULL, k, 4);
                    k += __shfl_xor_sync(FULL, k, 2);
                    k += __shfl_xor_sync(FULL, k, 1);
                    if ((lane & 7) == 0) atomicAdd(acc + 4 * j + (((lane >> 4) << 1) | ((lane >> 3) & 1)), k);
                }
            }
        }
        if constexpr (CSUM) {
            double sd[3];
            contract_dA<LA, LB>(pl, bd, dm, S, sd);
            sdx = sd[0];
            sdy = sd[1];
            sdz = sd[2];
        }
        // dE/dA = -(sd + a/p se), dE/dB = sd - b/p se
        double g[6] = {-(sdx + aop * sex), -(sdy + aop * sey), -(sdz + aop * sez),
                       sdx - bop * sex, sdy - bop * sey, sdz - bop * sez};
        bool take[5], head;
        seg_setup(pl.active ? pl.s : -1 - lane, lane, take, head);
#pragma unroll
        for (int k = 0; k < 6; ++k) g[k] = seg_reduce(g[k], take);
        if (head && pl.active) {
#pragma unroll
            for (int x = 0; x < 3; ++x) {
                atomicAdd(gqm + 3 * pl.atomA + x, g[x]);
                atomicAdd(gqm + 3 * pl.atomB + x, g[3 + x]);
            }
        }
    }
    __syncthreads();
    for (int k = threadIdx.x; k < 4 * nch; k += blockDim.x) {
        const double v = acc[k];
        if (v != 0.0) atomicAdd(gchg + 4 * (size_t)ch_begin + k, v);
    }
}

template <int LA, int LB, int NT>
static cudaError_t launch_nt(const BasisDev &bd, const RegionDev &rg, int pp_begin, int pp_end, int ch_begin,
                             int ch_end, const double *boys, const double *dm, double *gqm, double *gchg, int *err,
                             int nsm, int nslice, cudaStream_t st)
{
    const int nper = (ch_end - ch_begin + nslice - 1) / nslice;  // charges per slice
    const size_t smem = std::max((size_t)nper * (sizeof(double4_32a) + 4 * sizeof(double)), SWEEP_SMEM_MIN);
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_vgrad_f64<LA, LB, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)(CHUNK_GRAD * (sizeof(double4_32a) + 4 * sizeof(double))));
        if (e != cudaSuccess) return e;
        attr = true;
    }
    const int ntile = (pp_end - pp_begin + 31) / 32;
    int grid = (ntile + NT / 32 - 1) / (NT / 32);
    if (grid > nsm) grid = nsm;
    if (grid < 1) return cudaSuccess;
    k_vgrad_f64<LA, LB, NT><<<dim3(grid, nslice), NT, smem, st>>>(bd, rg, pp_begin, pp_end, ch_begin, ch_end, boys,
                                                                  dm, gqm, gchg, err);
    return cudaGetLastError();
}

template <int LA, int LB>
cudaError_t VgradF64<LA, LB>::run(const BasisDev &bd, const RegionDev &rg, int pp_begin, int pp_end, int ch_begin,
                                  int ch_end, const double *boys, const double *dm, double *gqm, double *gchg,
                                  int *err,
                                  int nsm, int variant, int nslice,
                                  cudaStream_t st)
{
    constexpr int W = sweep_wide_threads(SW_VGRAD_F64, class_of(LA, LB));
    if constexpr (W > 0)
        if (variant == 1)
            return launch_nt<LA, LB, W>(bd, rg, pp_begin, pp_end, ch_begin, ch_end, boys, dm, gqm, gchg, err, nsm,
                                        nslice, st);
    return launch_nt<LA, LB, 256>(bd, rg, pp_begin, pp_end, ch_begin, ch_end, boys, dm, gqm, gchg, err, nsm,
                                  nslice, st);
}

template struct VgradF64<la_of_class(QMMM_SPLIT_CLASS), lb_of_class(QMMM_SPLIT_CLASS)>;

#else  // the dispatcher

cudaError_t launch_vgrad_f64(const BasisDev &b, const RegionDev &r, int cls, int pp_begin, int pp_end,
                             int ch_begin, int ch_end, const double *boys, const double *dm, double *gqm,
                             double *gchg, int *err, int nsm, int variant, int nslice, cudaStream_t st)
{
    if (pp_end <= pp_begin || ch_end <= ch_begin) return cudaSuccess;
    return dispatch_class<VgradF64>(cls, b, r, pp_begin, pp_end, ch_begin, ch_end, boys, dm, gqm, gchg, err, nsm,
                                    variant, nslice, st);
}

#endif

}  // namespace qmmm
