// vgrad_f32.cu -- adjoint of the region-I term, mixed precision (see vgrad_f64.cu for the
// derivative algebra).  The density-folded Hermite coefficients D0, Dx, Dy, Dz are built in
// FP64 once per primitive pair and rounded to FP32; the per-charge Boys/R recursion to order L+1,
// the four D0 contractions (e_0, e_x, e_y, e_z) and the charge sum S_tuv += q R_tuv run in FP32,
// with no FP64 instruction inside the charge loop.  Every 16 charges the group's S is contracted
// with Dx, Dy, Dz, which wait in the thread's local memory (kept out of the loop's registers).
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

// 16-byte loads and stores of this thread's local memory (an array kept out of registers)
__device__ __forceinline__ void st_local4(uint32_t a, const float (&v)[4])
{
    asm volatile("st.local.v4.f32 [%0], {%1, %2, %3, %4};" ::"r"(a), "f"(v[0]), "f"(v[1]), "f"(v[2]), "f"(v[3])
                 : "memory");
}
__device__ __forceinline__ void ld_local4(uint32_t a, float (&v)[4])
{
    asm volatile("ld.local.v4.f32 {%0, %1, %2, %3}, [%4];" : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3]) : "r"(a)
                 : "memory");
}

template <int LA, int LB, int NT>
__global__ void __launch_bounds__(NT, 1)
k_vgrad_f32(BasisDev bd, RegionDev rg, int pp_begin, int pp_end, int ch_begin, int ch_end,
            const float *__restrict__ boys_g, unsigned boys_bytes, const double *__restrict__ dm,
            double *__restrict__ gqm, double *__restrict__ gchg, int *err)
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
    constexpr int ND4 = (3 * NH + 3) / 4;
    float4 dl[ND4];  // this lane's Dx, Dy, Dz (FP32), accessed only through ld/st.local
    const uint32_t dl_addr = (uint32_t)__cvta_generic_to_local(dl);
    for (int tile = blockIdx.x * nwarp + warp; tile < ntile; tile += gridDim.x * nwarp) {
        const PPLane pl = load_pp(bd, pp_begin + tile * 32 + lane, pp_end);
        const double aop = pl.a * pl.ip, bop = pl.b * pl.ip;
        float Ph[3], Plo[3];
#pragma unroll
        for (int x = 0; x < 3; ++x) {
            const double d = pl.P[x] - rg.centre[x];
            Ph[x] = (float)d;
            Plo[x] = (float)(d - (double)Ph[x]);
        }

        float D0[NH];
        {
            double d0[NH];
            fold_density<LA, LB>(pl, bd, dm, d0);
#pragma unroll
            for (int k = 0; k < NH; ++k) D0[k] = (float)d0[k];
        }
        {
            // Dx, Dy, Dz as FP32 in this thread's local memory: read once per GFOLD charges
            double dx[NH], dy[NH], dz[NH];
            fold_density_dA<LA, LB>(pl, bd, dm, dx, dy, dz);
#pragma unroll
            for (int i = 0; i < ND4; ++i) {
                float v[4];
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    const int e = 4 * i + c;
                    v[c] = e < NH ? (float)dx[e] : e < 2 * NH ? (float)dy[e - NH] : e < 3 * NH ? (float)dz[e - 2 * NH] : 0.0f;
                }
                st_local4(dl_addr + 16u * i, v);
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
                float tex = 0, tey = 0, tez = 0;
                float S[NH];  // sum over this group's charges of q R_tuv (k < NH)
#pragma unroll
                for (int k = 0; k < NH; ++k) S[k] = 0.0f;
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
                    float e0 = 0, ex = 0, ey = 0, ez = 0;
                    const float q = ch.w;
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
                                S[k] += q * R[k];
                            }
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
                // this group's sum_C q_C d_a(C) = sum_k Da_k S_k, Da from local memory
                float tdx = 0, tdy = 0, tdz = 0;
#pragma unroll
                for (int i = 0; i < ND4; ++i) {
                    float v[4];
                    ld_local4(dl_addr + 16u * i, v);
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        const int e = 4 * i + c;
                        if (e < NH) tdx += v[c] * S[e];
                        else if (e < 2 * NH) tdy += v[c] * S[e - NH];
                        else if (e < 3 * NH) tdz += v[c] * S[e - 2 * NH];
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
