// vgrad_f32.cu -- adjoint of the region-I term, mixed precision (see vgrad_f64.cu for the
// derivative algebra).  The density-folded Hermite coefficients D0, Dx, Dy, Dz are built in
// FP64 once per primitive pair and rounded to FP32; the per-charge Boys/R recursion to order L+1
// and the seven contractions run in FP32, with no FP64 instruction inside the charge loop.
// Per-pair sums go through FP32 partials over 16 charges folded into double-float pairs;
// per-charge sums over the warp's 32 primitive pairs use a reduce-scatter (6 shuffles for four
// values) and compensated FP32 shared-memory atomics: the atomic returns the old value, so the
// rounding error of every addition is recovered exactly and kept in a second FP32 word.
#include "pp_tile.cuh"

namespace qmmm {

template <int LA, int LB>
struct VgradF32 {
    static cudaError_t run(const BasisDev &bd, const RegionDev &rg, int pp_begin, int pp_end, int ch_begin,
                           int ch_end, const float *boys, const double *dm, double *gqm, double *gchg, int *err,
                           int nsm, int variant, int nslice,
                           cudaStream_t st);
};

#ifdef QMMM_SPLIT_CLASS  // one angular class per compilation

constexpr int GFOLD = 16;

template <int LA, int LB, int NT>
__global__ void __launch_bounds__(NT, 1)
k_vgrad_f32(BasisDev bd, RegionDev rg, int pp_begin, int pp_end, int ch_begin, int ch_end,
            const float *__restrict__ boys_g, unsigned boys_bytes, const double *__restrict__ dm,
            double *__restrict__ gqm, double *__restrict__ gchg, int *err)
{
    constexpr int L = LA + LB, NH = nherm(L), NH1 = nherm(L + 1), NA = ncart(LA), NB = ncart(LB);
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
    float4 *chi = reinterpret_cast<float4 *>(smem_raw);
    float4 *clo = chi + nch;
    float *tab = reinterpret_cast<float *>(clo + nch);
    // per-charge accumulators as FP32 (hi, lo) pairs: acc_hi[4 nch], acc_lo[4 nch]
    float *acc_hi = reinterpret_cast<float *>(smem_raw + (size_t)nch * 2 * sizeof(float4) + boys_bytes);
    float *acc_lo = acc_hi + 4 * nch;
    for (int k = threadIdx.x; k < 4 * nch; k += blockDim.x) acc_hi[k] = acc_lo[k] = 0.0f;
    {
        Seg s[3] = {{chi, rg.chg_hi + ch_begin, (unsigned)(nch * sizeof(float4))},
                    {clo, rg.chg_lo + ch_begin, (unsigned)(nch * sizeof(float4))},
                    {tab, boys_g, boys_bytes}};
        if (!stage_segments(s, 3, &bar, err)) return;
    }

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    const int ntile = (pp_end - pp_begin + 31) >> 5;
    for (int tile = blockIdx.x * nwarp + warp; tile < ntile; tile += gridDim.x * nwarp) {
        const PPLane pl = load_pp(bd, pp_begin + tile * 32 + lane, pp_end);
        const bool mirror = pl.sp.shA != pl.sp.shB;
        const double coef = TWO_PI * pl.ip * pl.cab;
        const double aop = pl.a * pl.ip, bop = pl.b * pl.ip;
        float Ph[3], Plo[3];
#pragma unroll
        for (int x = 0; x < 3; ++x) {
            const double d = pl.P[x] - rg.centre[x];
            Ph[x] = (float)d;
            Plo[x] = (float)(d - (double)Ph[x]);
        }

        float D0[NH], Dx[NH], Dy[NH], Dz[NH];
        {
            double d0[NH], dx[NH], dy[NH], dz[NH];
#pragma unroll
            for (int k = 0; k < NH; ++k) d0[k] = dx[k] = dy[k] = dz[k] = 0.0;
            double Ex[LA + 2][LB + 1][L + 2], Ey[LA + 2][LB + 1][L + 2], Ez[LA + 2][LB + 1][L + 2];
            hermite_E<LA + 1, LB, double>(Ex, pl.P[0] - pl.A[0], pl.P[0] - pl.B[0], 0.5 * pl.ip);
            hermite_E<LA + 1, LB, double>(Ey, pl.P[1] - pl.A[1], pl.P[1] - pl.B[1], 0.5 * pl.ip);
            hermite_E<LA + 1, LB, double>(Ez, pl.P[2] - pl.A[2], pl.P[2] - pl.B[2], 0.5 * pl.ip);
#pragma unroll
            for (int ia = 0; ia < NA; ++ia) {
#pragma unroll
                for (int ib = 0; ib < NB; ++ib) {
                    const int ax = cart_lx(LA, ia), ay = cart_ly(LA, ia), az = cart_lz(LA, ia);
                    const int bx = cart_lx(LB, ib), by = cart_ly(LB, ib), bz = cart_lz(LB, ib);
                    double g = 0.0;
                    if (pl.active) {
                        const size_t r = pl.sp.aoA + ia, c = pl.sp.aoB + ib;
                        g = dm[r * bd.nao + c];
                        if (mirror) g += dm[c * bd.nao + r];
                        g *= coef;
                    }
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
#pragma unroll
                    for (int t = 0; t <= ax + bx; ++t)
#pragma unroll
                        for (int u = 0; u <= ay + by; ++u)
#pragma unroll
                            for (int w = 0; w <= az + bz; ++w) {
                                const int k = hidx(t, u, w);
                                const double ex = Ex[ax][bx][t], ey = Ey[ay][by][u], ez = Ez[az][bz][w];
                                d0[k] += g * ex * ey * ez;
                                dx[k] += g * dEx[t] * ey * ez;
                                dy[k] += g * ex * dEy[u] * ez;
                                dz[k] += g * ex * ey * dEz[w];
                            }
                }
            }
#pragma unroll
            for (int k = 0; k < NH; ++k) {
                D0[k] = (float)d0[k];
                Dx[k] = (float)dx[k];
                Dy[k] = (float)dy[k];
                Dz[k] = (float)dz[k];
            }
        }

        // per-pair sums over charges as double-float pairs (no FP64 instruction in the charge loop)
        float sh[6] = {0, 0, 0, 0, 0, 0}, sl[6] = {0, 0, 0, 0, 0, 0};
        for (int c = 0; c < rg.ncls; ++c) {
            const int lo = max(__ldg(rg.cls_off + c), ch_begin) - ch_begin;
            const int hi = min(__ldg(rg.cls_off + c + 1), ch_end) - ch_begin;
            if (lo >= hi) continue;
            const double kap = __ldg(rg.cls_kappa + c);
            const double td = kap > 0.0 ? kap / (pl.p + kap) : 1.0;
            const float rho = (float)(pl.p * td), m2rho = -2.0f * rho, sq = (float)sqrt(td);
            for (int j0 = lo; j0 < hi; j0 += GFOLD) {
                const int j1 = min(hi, j0 + GFOLD);
                float tdx = 0, tdy = 0, tdz = 0, tex = 0, tey = 0, tez = 0;
                for (int j = j0; j < j1; ++j) {
                    const float4 ch = chi[j], cl = clo[j];
                    const float X = (Ph[0] - ch.x) + (Plo[0] - cl.x);
                    const float Y = (Ph[1] - ch.y) + (Plo[1] - cl.y);
                    const float Z = (Ph[2] - ch.z) + (Plo[2] - cl.z);
                    float T, Tl;
                    boys_arg_f32(rho, X, Y, Z, T, Tl);
                    float F[L + 2];
                    boys_f32<L + 1>(T, F, tab, Tl);
                    float Fn[L + 2];
                    float sc = sq;
#pragma unroll
                    for (int n = 0; n <= L + 1; ++n) {
                        Fn[n] = sc * F[n];
                        sc *= m2rho;
                    }
                    float R[NH1];
                    hermite_R<L + 1, float>(R, Fn, X, Y, Z);
                    float e0 = 0, ex = 0, ey = 0, ez = 0, dx = 0, dy = 0, dz = 0;
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
                                dx += Dx[k] * R[k];
                                dy += Dy[k] * R[k];
                                dz += Dz[k] * R[k];
                            }
                    const float q = ch.w;
                    tdx += q * dx; tdy += q * dy; tdz += q * dz;
                    tex += q * ex; tey += q * ey; tez += q * ez;
                    // per-charge sums over the 32 primitive pairs: 4 values -> halve twice (each lane
                    // keeps one component summed over 4 lanes), then a 3-step butterfly; lane 8c ends
                    // with component c = (dC_x, dC_y, dC_z, dq)
                    float v0 = q * ex, v1 = q * ey, v2 = q * ez, v3 = -e0;
                    {
                        const bool up = lane & 16;
                        float k0 = up ? v2 : v0, k1 = up ? v3 : v1;
                        const float s0 = up ? v0 : v2, s1 = up ? v1 : v3;
                        k0 += __shfl_xor_sync(FULL, s0, 16);
                        k1 += __shfl_xor_sync(FULL, s1, 16);
                        const bool up8 = lane & 8;
                        float k = up8 ? k1 : k0;
                        k += __shfl_xor_sync(FULL, up8 ? k0 : k1, 8);
                        k += __shfl_xor_sync(FULL, k, 4);
                        k += __shfl_xor_sync(FULL, k, 2);
                        k += __shfl_xor_sync(FULL, k, 1);
                        if ((lane & 7) == 0) {
                            // component index: bit 4 -> (2,3) vs (0,1); bit 3 -> second of the pair
                            const int comp = ((lane >> 4) << 1) | ((lane >> 3) & 1);
                            // compensated atomic: recover the rounding error of the addition exactly
                            float *h = acc_hi + 4 * j + comp;
                            const float old = atomicAdd(h, k);
                            const float sum = old + k, bv = sum - old;
                            atomicAdd(acc_lo + 4 * j + comp, (old - (sum - bv)) + (k - bv));
                        }
                    }
                }
                df_add(sh[0], sl[0], tdx); df_add(sh[1], sl[1], tdy); df_add(sh[2], sl[2], tdz);
                df_add(sh[3], sl[3], tex); df_add(sh[4], sl[4], tey); df_add(sh[5], sl[5], tez);
            }
        }
        const double sdx = (double)sh[0] + sl[0], sdy = (double)sh[1] + sl[1], sdz = (double)sh[2] + sl[2];
        const double sex = (double)sh[3] + sl[3], sey = (double)sh[4] + sl[4], sez = (double)sh[5] + sl[5];
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
        const double v = (double)acc_hi[k] + (double)acc_lo[k];
        if (v != 0.0) atomicAdd(gchg + 4 * (size_t)ch_begin + k, v);
    }
}

// bytes of one order's FP32 Boys table (what a block stages)
inline unsigned boys32_bytes_g() { return (unsigned)(BOYS_TAB_F * sizeof(float)); }

template <int LA, int LB, int NT>
static cudaError_t launch_nt(const BasisDev &bd, const RegionDev &rg, int pp_begin, int pp_end, int ch_begin,
                             int ch_end, const float *boys, const double *dm, double *gqm, double *gchg, int *err,
                             int nsm, int nslice, cudaStream_t st)
{
    const unsigned tb = boys32_bytes_g();
    const size_t per = 2 * sizeof(float4) + 4 * sizeof(double);
    const int nper = (ch_end - ch_begin + nslice - 1) / nslice;  // charges per slice
    const size_t smem = (size_t)nper * per + tb;
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_vgrad_f32<LA, LB, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)(CHUNK_GRAD * per + tb));
        if (e != cudaSuccess) return e;
        attr = true;
    }
    const int ntile = (pp_end - pp_begin + 31) / 32;
    int grid = (ntile + NT / 32 - 1) / (NT / 32);
    if (grid > nsm) grid = nsm;
    if (grid < 1) return cudaSuccess;
    k_vgrad_f32<LA, LB, NT><<<dim3(grid, nslice), NT, smem, st>>>(bd, rg, pp_begin, pp_end, ch_begin, ch_end,
                                                                  boys + (size_t)(LA + LB + 1) * BOYS_TAB_F, tb,
                                                                  dm, gqm, gchg, err);
    return cudaGetLastError();
}

template <int LA, int LB>
cudaError_t VgradF32<LA, LB>::run(const BasisDev &bd, const RegionDev &rg, int pp_begin, int pp_end, int ch_begin,
                                  int ch_end, const float *boys, const double *dm, double *gqm, double *gchg,
                                  int *err,
                                  int nsm, int variant, int nslice,
                                  cudaStream_t st)
{
    constexpr int W = sweep_wide_threads(SW_VGRAD_F32, class_of(LA, LB));
    if constexpr (W > 0)
        if (variant == 1)
            return launch_nt<LA, LB, W>(bd, rg, pp_begin, pp_end, ch_begin, ch_end, boys, dm, gqm, gchg, err, nsm,
                                        nslice, st);
    return launch_nt<LA, LB, 256>(bd, rg, pp_begin, pp_end, ch_begin, ch_end, boys, dm, gqm, gchg, err, nsm,
                                  nslice, st);
}

template struct VgradF32<la_of_class(QMMM_SPLIT_CLASS), lb_of_class(QMMM_SPLIT_CLASS)>;

#else  // the dispatcher

cudaError_t launch_vgrad_f32(const BasisDev &b, const RegionDev &r, int cls, int pp_begin, int pp_end,
                             int ch_begin, int ch_end, const float *boys, const double *dm, double *gqm,
                             double *gchg, int *err, int nsm, int variant, int nslice, cudaStream_t st)
{
    if (pp_end <= pp_begin || ch_end <= ch_begin) return cudaSuccess;
    return dispatch_class<VgradF32>(cls, b, r, pp_begin, pp_end, ch_begin, ch_end, boys, dm, gqm, gchg, err, nsm,
                                    variant, nslice, st);
}

#endif

}  // namespace qmmm
