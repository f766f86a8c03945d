// mmrecip_tc.cu -- the MM side of the reciprocal Ewald sum (SI, "Multipolar Ewald", long-range
// part, differentiated for the adjoint) on the tensor cores:
//
//   dE/dq_i += sum_G Re[A(G) e^{-iG.R_i}],   dE/dR_i += q_i sum_G G Im[A(G) e^{-iG.R_i}]
//
// over the half space of the kmax cube, with A(G) = 2 g(G) sum_j e^{iG.R_j} (Q_j + i G.mu_j
// - 1/2 G.theta_j.G) from the QM multipoles and the separable phase e^{-iG.R} = X(n_x) Y(n_y) Z(n_z).
// Over K = (n_y, n_z) the sum is a product of two matrices followed by a short contraction:
//
//   T_k[i, n_x] = sum_{n_y, n_z} C_k[n_x, n_y, n_z] Y_i(n_y) Z_i(n_z),   C_0 = A, C_1 = G_y A, C_2 = G_z A,
//   dE/dq_i = Re sum X_i T_0,  f_x = sum G_x Im(X_i T_0),  f_y = sum Im(X_i T_1),  f_z = sum Im(X_i T_2).
//
// A operand (M = 128 charges x K): the outer products Y_i(n_y) Z_i(n_z), digitised on chip from
// fixed-point phase rows staged by TMA; B operand (N = 112 rows (k, n_x, re/im) x K): C_k divided
// by a power of two per (k, n_x) so that |C| <= 1, digitised once per call into the shared-memory
// layout.  Digits as for the structure factor (tc_digits.cuh).  FP64 path: seven planes per operand
// (48-bit fixed point), 28 plane pairs per K-step into FP32 accumulators in tensor memory, five
// accumulators (levels 0..3 kept apart, 4..6 merged), so at most 96 N rows per tile.  Mixed path:
// five planes (34-bit operands, 15 plane pairs) and three accumulators (levels 0 and 1 apart, 2..4
// merged: the merged sum's FP32 rounding is about 2^-31 of level 0's scale), so 160 rows per tile
// and the three channels of kx <= 25 take a single N tile: the A operand is digitised once and no
// N row beyond the 6 (kx + 1) in use is computed.  Against the double-float CUDA-core kernel the
// mixed path's sum differs by 3e-9 (active site, kmax 16) and 1.3e-8 (large site, kmax 24) of the
// largest MM gradient component, a tenth or less of the mixed path's error against FP64.  Level 0
// is exact for any input while 4096 x 2 N_y N_z < 2^24 (kmax <= 20) and beyond that unless the
// row-normalised coefficients, which decay as exp(-G^2/4 alpha^2), sum to more than 2^11 in
// magnitude; levels 1 to 3 are sums of random-sign digit products, typically 2^17 or less.  The epilogue
// (one thread per charge) combines the levels exactly in 64-bit integers, applies the row scales
// and contracts with X_i(n_x) in FP64.
#include <algorithm>

#include "device_common.cuh"
#include "qmmm_internal.h"
#include "tc_common.cuh"
#include "tc_digits.cuh"

namespace qmmm {

namespace {
using namespace tcd;
constexpr int MM = 128;                 // charges per tile (MMA M)
constexpr int NRMAX = 256;              // N rows (channel k, n_x, re/im) of one tile, a multiple of 16
constexpr int KC = 16;                  // K entries per chunk: 8 (n_y, n_z) pairs x re/im
constexpr int PCH = KC / 2;             // pairs per chunk
constexpr int NSTGMAX = 3;              // pipeline depth (2 when three stages do not fit)
constexpr int NACCMAX = 5;              // accumulators: levels 0 .. nacc-2 exact, the rest merged
constexpr int NPROD = 16;               // producer warps
constexpr int NTHR = (NPROD + 2) * 32;  // + MMA warp + loader warp
constexpr uint32_t CMK = 128;                    // byte step between core matrices along K
constexpr uint32_t CMN = (KC / 8) * 128;         // byte step between 8-row groups
constexpr uint32_t APL = MM * KC * 2;            // A plane bytes per chunk
constexpr uint32_t ROWB = MM * 16;               // one staged phase row (128 charges, int4)
constexpr uint32_t PBUF = (2 + PCH) * ROWB;      // Y rows n_y0, n_y0 + 1 and one Z row per pair
constexpr size_t SMEM_MAX = 232448;
__host__ __device__ inline uint32_t mmr_bpl(int nr) { return (uint32_t)nr * KC * 2; }  // B plane bytes
__host__ __device__ inline uint32_t mmr_stage(int nr, int np) { return np * (APL + mmr_bpl(nr)); }
__host__ inline size_t mmr_smem(int nr, int nstg, int np) { return nstg * (size_t)(mmr_stage(nr, np) + PBUF) + 256; }
// fixed-point width of an operand with NP planes, and the balanced input w of a value at 2^(bits + shift)
__host__ __device__ constexpr int mmr_bits(int np) { return 6 + 7 * (np - 1); }
template <int NP>
__device__ __forceinline__ long long fixw_n(long long v, int shift)
{
    return (v + (1ll << (shift - 1)) + (bal<NP>() << shift)) >> shift;
}

struct MmrArgs {
    const int4 *Yt, *Zt;   // [NY][npad], [NZ][npad] split 2^61 fixed point, e^{-2 pi i n u}
    const uint32_t *bpl;   // B planes per chunk (NP * BPL bytes)
    const double *cscale;  // [3][NX] power-of-two row scales
    const double *mm_xyz, *mm_q;
    double *dq, *dR;
    int *err;
    int nmm, npad, NX, NY, NZ, npair, nchunk;
    int nr, nr_last, cpt, nstg;  // N rows of a tile and of the last tile, channels per tile, stages
    int nacc;                  // accumulators (3 or 5)
    double box0;
};
}  // namespace

// Mixed-path epilogue of one charge (row i of the tile) in double-float arithmetic on the FP32
// pipes: the FP64 pipe (2 FMAs per clock and SM) took about a tenth of the kernel's time for the
// level join, the row scales and the contraction with X_i(n_x), while the MMA pipeline of the SM
// stood idle.  The exact levels and the merged one join by error-free two-sums (all terms are
// FP32 values), the row scales are powers of two (exact), the phases X_i(n_x) come from an FP64
// start and step and a double-float recurrence; about 44 significant bits throughout, against
// the 34-bit operands of the sum.
__device__ __forceinline__ void mmr_epilogue_df(const MmrArgs &a, uint32_t tl, int NR, int kfirst, int nk, bool act,
                                                int i)
{
    double sn, cs;
    sincospi(-2.0 * (act ? a.mm_xyz[3 * i] : 0.0) / a.box0, &sn, &cs);
    const c2 step{f2_from(cs), f2_from(sn)};
    c2 X{f2{1.0f, 0.0f}, f2{0.0f, 0.0f}};
    const f2 g1 = f2_from(6.283185307179586476925 / a.box0);  // G_x per unit n_x
    float ph = 0.0f, pl = 0.0f;                               // sum_nx Re(X T_0)
    float fh[3] = {0.0f, 0.0f, 0.0f}, fl[3] = {0.0f, 0.0f, 0.0f};  // sum_nx Im(X T_k), tile channel kl
    for (int nx = 0; nx < a.NX; ++nx) {
#pragma unroll
        for (int kl = 0; kl < 3; ++kl) {
            if (kl >= nk) break;
            const int k = kfirst + kl, col = 2 * (kl * a.NX + nx);
            uint32_t v[NACCMAX][2];
#pragma unroll
            for (int acc = 0; acc < NACCMAX; ++acc) {
                v[acc][0] = v[acc][1] = 0u;
                if (acc < a.nacc)
                    asm volatile("tcgen05.ld.sync.aligned.32x32b.x2.b32 {%0, %1}, [%2];"
                                 : "=r"(v[acc][0]), "=r"(v[acc][1])
                                 : "r"(tl + acc * NR + col)
                                 : "memory");
            }
            tc::tmem_wait_ld();
            const float sc = (float)(__ldg(a.cscale + k * a.NX + nx) * 0x1p-12);  // a power of two
            f2 t[2];
#pragma unroll
            for (int r = 0; r < 2; ++r) {
                float h = __uint_as_float(v[0][r]), l = 0.0f;
#pragma unroll
                for (int acc = 1; acc < NACCMAX; ++acc)
                    if (acc < a.nacc) df_add(h, l, __uint_as_float(v[acc][r]));
                t[r] = f2_fast2sum(h * sc, l * sc);
            }
            if (k == 0) {
                f2_mac(ph, pl, X.re, t[0]);
                f2_mac(ph, pl, f2_neg(X.im), t[1]);
                const f2 u = f2_add(f2_mul(X.re, t[1]), f2_mul(X.im, t[0]));
                f2_mac(fh[kl], fl[kl], f2_mul(g1, f2{(float)nx, 0.0f}), u);
            } else {
                f2_mac(fh[kl], fl[kl], X.re, t[1]);
                f2_mac(fh[kl], fl[kl], X.im, t[0]);
            }
        }
        X = c2_mul(X, step);
    }
    if (act) {
        // each channel belongs to exactly one N tile: no two CTAs write the same output
        const double q = a.mm_q[i];
        if (kfirst == 0) a.dq[i] += f2_to(ph, pl);
#pragma unroll
        for (int kl = 0; kl < 3; ++kl)
            if (kl < nk) a.dR[3 * i + kfirst + kl] += q * f2_to(fh[kl], fl[kl]);
    }
}

// grid (mtiles, N tiles), NTHR threads, mmr_smem() dynamic shared memory; chunk ch uses buffer set
// ch % nstg.  NP digit planes per operand: 7 (48-bit operands, FP64 class) on the FP64 path, 5
// (34-bit) on the mixed path.
template <int NP>
__global__ void __launch_bounds__(NTHR, 1) k_mm_recip_tc(MmrArgs a)
{
    extern __shared__ __align__(1024) unsigned char sm[];
    // the last N tile may hold fewer channels and rows; the smem layout follows its own NR
    const int NSTG = a.nstg, NR = (int)blockIdx.y + 1 == (int)gridDim.y ? a.nr_last : a.nr;
    const uint32_t BPL = mmr_bpl(NR), STG = mmr_stage(NR, NP);
    unsigned char *pbuf0 = sm + NSTG * STG;
    uint64_t *bars = reinterpret_cast<uint64_t *>(pbuf0 + NSTG * PBUF);
    uint64_t *full = bars, *bfull = bars + NSTGMAX, *pfull = bars + 2 * NSTGMAX, *empty = bars + 3 * NSTGMAX;
    uint64_t *done = bars + 4 * NSTGMAX;
    uint32_t *tslot = reinterpret_cast<uint32_t *>(done + 1);
    volatile int *abort = reinterpret_cast<volatile int *>(tslot + 1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.x * MM;
    // N tile blockIdx.y: channels [kfirst, kfirst + nk), its own B planes
    const int kfirst = blockIdx.y * a.cpt, nk = min(a.cpt, 3 - kfirst);
    const uint32_t *bpl = a.bpl + (size_t)blockIdx.y * a.nchunk * (NP * mmr_bpl(a.nr) / 4);

    if (threadIdx.x == 0) {
        for (int k = 0; k < NSTGMAX; ++k) {
            mbar_init(&full[k], NPROD);
            mbar_init(&bfull[k], 1);
            mbar_init(&pfull[k], 1);
            mbar_init(&empty[k], 1);
        }
        mbar_init(done, 1);
        *abort = 0;
        fence_mbar_init();
    }
    if (warp == NPROD) {
        tc::tmem_alloc(tslot, 512);
        tc::tmem_relinquish();
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tbase = *tslot;
    auto give_up = [&]() {
        *abort = 1;
        atomicOr(a.err, DEVERR_TIMEOUT);
    };

    if (warp < NPROD) {
        // ---------------- producers: A planes, 128 charges x 8 pairs per chunk ----------------
        // groups of 8 charges x 4 pairs (32 distinct banks), two per warp
        constexpr int AJ = 2;
        int e_m[AJ], e_j[AJ];
        uint32_t e_off[AJ];
#pragma unroll
        for (int j = 0; j < AJ; ++j) {
            const int combo = warp * AJ + j, rg = combo >> 1, cg = combo & 1;
            e_m[j] = rg * 8 + (lane >> 2);
            e_j[j] = cg * 4 + (lane & 3);
            e_off[j] = rg * CMN + cg * CMK + (lane >> 2) * 16 + (lane & 3) * 4;
        }
        int z0 = 0;  // p0 mod NZ, p0 = ch * PCH (the chunk's first pair)
        for (int ch = 0; ch < a.nchunk; ++ch, z0 = z0 + PCH >= a.NZ ? z0 + PCH - a.NZ : z0 + PCH) {
            const int st = ch % NSTG, u = ch / NSTG;
            if (ch >= NSTG && !tc::mbar_wait_thread(&empty[st], (u - 1) & 1, abort)) {
                give_up();
                break;
            }
            if (!tc::mbar_wait_thread(&pfull[st], u & 1, abort)) {
                give_up();
                break;
            }
            unsigned char *sA = sm + st * STG;
            const int4 *Ys = reinterpret_cast<const int4 *>(pbuf0 + st * PBUF), *Zs = Ys + 2 * MM;
            const int p0 = ch * PCH;
#pragma unroll
            for (int j = 0; j < AJ; ++j) {
                const int m = e_m[j], jp = e_j[j], p = p0 + jp;
                if (m0 + m < a.nmm && p < a.npair) {
                    long long re, im;  // 2^60 scale; the pair lies in row n_y0 + (z0 + jp >= NZ)
                    cmul61(Ys[(z0 + jp >= a.NZ ? MM : 0) + m], Zs[jp * MM + m], re, im);
                    constexpr int SH = 60 - mmr_bits(NP);
                    const PlanesN<NP> pr = planes_n<NP>(fixw_n<NP>(re, SH)), pi = planes_n<NP>(fixw_n<NP>(im, SH));
#pragma unroll
                    for (int s = 0; s < NP; ++s)
                        *reinterpret_cast<uint32_t *>(sA + s * APL + e_off[j]) = pack_bf16(pr.p[s], pi.p[s]);
                } else {
#pragma unroll
                    for (int s = 0; s < NP; ++s) *reinterpret_cast<uint32_t *>(sA + s * APL + e_off[j]) = 0u;
                }
            }
            tc::fence_proxy_async_smem();
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(&full[st]);
        }
    } else if (warp == NPROD) {
        if (lane == 0) {
            // ---------------- MMA issue: NP (NP + 1) / 2 plane pairs per chunk ----------------
            const uint32_t idesc = tc::idesc_bf16_f32(MM, NR);
            for (int ch = 0; ch < a.nchunk; ++ch) {
                const int st = ch % NSTG, u = ch / NSTG;
                if (!tc::mbar_wait_thread(&full[st], u & 1, abort) || !tc::mbar_wait_thread(&bfull[st], u & 1, abort)) {
                    give_up();
                    break;
                }
                tc::fence_after_sync();
                const uint32_t sA = smem_addr(sm + st * STG), sB = sA + NP * APL;
#pragma unroll
                for (int s = 0; s < NP; ++s)
#pragma unroll
                    for (int t = 0; t < NP - s; ++t) {
                        const int acc = s + t < a.nacc - 1 ? s + t : a.nacc - 1;
                        const uint32_t first = (ch == 0 && s == 0 && t == acc);
                        const uint64_t ad = tc::smem_desc(sA + s * APL, CMK, CMN);
                        const uint64_t bd = tc::smem_desc(sB + t * BPL, CMK, CMN);
                        tc::mma_bf16(tbase + acc * NR, ad, bd, idesc, first ? 0u : 1u);
                    }
                tc::commit(&empty[st]);
            }
            tc::commit(done);
        }
    } else {
        // ---------------- loader warp: phase rows and B planes of chunk ch ----------------
        // lane 0 waits and posts the expected bytes; the copies of a chunk (two Y rows, one Z row
        // per pair, the B planes) go out from separate lanes at once
        int issued = 0, pissued = 0;
        for (int ch = 0; ch < a.nchunk; ++ch) {
            const int st = ch % NSTG, u = ch / NSTG;
            int ok = 1;
            if (lane == 0 && ch >= NSTG) ok = tc::mbar_wait_thread(&full[st], (u - 1) & 1, abort);
            if (!__shfl_sync(0xffffffffu, ok, 0)) {
                if (lane == 0) give_up();
                break;
            }
            const int p0 = ch * PCH, iy0 = p0 / a.NZ, iy1 = min(iy0 + 1, a.NY - 1);
            const int nvalid = min(PCH, a.npair - p0);
            unsigned char *dst = pbuf0 + st * PBUF;
            if (lane == 0) mbar_arrive_expect_tx(&pfull[st], (2 + nvalid) * ROWB);
            __syncwarp();
            if (lane < 2) {
                bulk_g2s(dst + lane * ROWB, a.Yt + (size_t)(lane ? iy1 : iy0) * a.npad + m0, ROWB, &pfull[st]);
            } else if (lane < 2 + nvalid) {
                const int iz = (p0 + lane - 2) % a.NZ;
                bulk_g2s(dst + lane * ROWB, a.Zt + (size_t)iz * a.npad + m0, ROWB, &pfull[st]);
            }
            pissued = ch + 1;
            if (lane == 0 && ch >= NSTG) ok = tc::mbar_wait_thread(&empty[st], (u - 1) & 1, abort);
            if (!__shfl_sync(0xffffffffu, ok, 0)) {
                if (lane == 0) give_up();
                break;
            }
            if (lane == 0) {
                mbar_arrive_expect_tx(&bfull[st], NP * BPL);
                bulk_g2s(sm + st * STG + NP * APL, bpl + (size_t)ch * (NP * BPL / 4), NP * BPL, &bfull[st]);
            }
            issued = ch + 1;
        }
        if (lane == 0) {
            // copies possibly still in flight (after a give-up): wait for them to land, bounded in
            // time only (not cut short by the abort flag), before the block may leave
            for (int ch = issued > NSTG ? issued - NSTG : 0; ch < issued; ++ch)
                tc::mbar_drain(&bfull[ch % NSTG], (ch / NSTG) & 1);
            for (int ch = pissued > NSTG ? pissued - NSTG : 0; ch < pissued; ++ch)
                tc::mbar_drain(&pfull[ch % NSTG], (ch / NSTG) & 1);
        }
    }

    // ---------------- epilogue: one thread per charge (warps 0..3) ----------------
    if (warp < 4) {
        if (!tc::mbar_wait_thread(done, 0, abort)) {
            give_up();
            // the MMA thread commits `done` on every path: wait for it (bounded in time only), so
            // that no MMA still writes tensor memory when it is freed below
            tc::mbar_drain(done, 0);
        } else {
            tc::fence_after_sync();
            const int row = 32 * warp + lane, i = m0 + row;
            const uint32_t tl = tbase + ((uint32_t)(32 * warp) << 16);
            const bool act = i < a.nmm;
            if constexpr (NP == MMR_NP_MIXED) {
                mmr_epilogue_df(a, tl, NR, kfirst, nk, act, i);
            } else {
            double sn, cs;
            sincospi(-2.0 * (act ? a.mm_xyz[3 * i] : 0.0) / a.box0, &sn, &cs);
            double xr = 1.0, xi = 0.0;
            double pot = 0.0;
            double f[3] = {0.0, 0.0, 0.0};  // sum_nx Im(X T_k) (channel 0 weighted by G_x)
            for (int nx = 0; nx < a.NX; ++nx) {
                const double gx = 6.283185307179586476925 * nx / a.box0;
                for (int kl = 0; kl < nk; ++kl) {
                    const int k = kfirst + kl, col = 2 * (kl * a.NX + nx);
                    uint32_t v[NACCMAX][2];
#pragma unroll
                    for (int acc = 0; acc < NACCMAX; ++acc) {
                        v[acc][0] = v[acc][1] = 0u;
                        if (acc < a.nacc)
                            asm volatile("tcgen05.ld.sync.aligned.32x32b.x2.b32 {%0, %1}, [%2];"
                                         : "=r"(v[acc][0]), "=r"(v[acc][1])
                                         : "r"(tl + acc * NR + col)
                                         : "memory");
                    }
                    tc::tmem_wait_ld();
                    double t2[2];
#pragma unroll
                    for (int r = 0; r < 2; ++r) {
                        // exact levels 0 .. nacc-2 in units of 2^-21, then the merged rest
                        long long ex = 0;
#pragma unroll
                        for (int l = 0; l < NACCMAX - 1; ++l)
                            if (l < a.nacc - 1)
                                ex += __float2ll_rn(__uint_as_float(v[l][r]) * (float)(1 << (7 * l))) << (21 - 7 * l);
                        t2[r] = fma((double)ex, 0x1p-21, (double)__uint_as_float(v[a.nacc - 1][r]));
                    }
                    const double sc = __ldg(a.cscale + k * a.NX + nx) * 0x1p-12;
                    const double tr = t2[0] * sc, ti = t2[1] * sc;
                    if (k == 0) pot += xr * tr - xi * ti;
                    f[k] += (k == 0 ? gx : 1.0) * (xr * ti + xi * tr);
                }
                const double nr = xr * cs - xi * sn;
                xi = xr * sn + xi * cs;
                xr = nr;
            }
            if (act) {
                // each channel belongs to exactly one N tile: no two CTAs write the same output
                const double q = a.mm_q[i];
                if (kfirst == 0) a.dq[i] += pot;
                for (int kl = 0; kl < nk; ++kl) a.dR[3 * i + kfirst + kl] += q * f[kfirst + kl];
            }
            }
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == NPROD) {
        tc::fence_after_sync();
        tc::tmem_dealloc(tbase, 512);
    }
}

// Y_i(n_y) = e^{-2 pi i n_y u_y}, Z_i(n_z) = e^{-2 pi i n_z u_z} in rows over the charges:
// Yt[iy][i], Zt[iz][i] (index iy = n_y + ky), split 2^61 fixed point.  One thread per (axis,
// charge): the start and the step from FP64 sincospi, the recurrence in fixed point.
__global__ void k_mmr_phases(EwaldDev e, int npad, int4 *Yt, int4 *Zt)
{
    const long long item = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (item >= 2ll * e.nmm) return;
    const int d = 1 + (int)(item / e.nmm), i = (int)(item - (long long)(d - 1) * e.nmm);
    const int k = e.kmax[d], len = 2 * k + 1;
    int4 *col = (d == 1 ? Yt : Zt) + i;
    const double u = e.mm_xyz[3 * i + d] / e.box[d];
    double sn, cs;
    sincospi(-2.0 * u, &sn, &cs);
    const long long sr = fix61(cs), si = fix61(sn);
    sincospi(2.0 * (double)k * u, &sn, &cs);  // index 0 is n = -k
    long long pr = fix61(cs), pi = fix61(sn);
    for (int n = 0; n < len; ++n) {
        col[(size_t)n * npad] = split61(pr, pi);
        const long long nr = (mul61(pr, sr) - mul61(pi, si)) * 2;
        const long long ni = (mul61(pr, si) + mul61(pi, sr)) * 2;
        pr = nr;
        pi = ni;
    }
}

// channel k of the B operand at dense index (n_x, iy, iz): C_0 = A, C_1 = G_y A, C_2 = A_z
__device__ __forceinline__ double2 mmr_channel(const double2 *A, const double2 *Az, int k, size_t idx, double gy)
{
    if (k == 2) return Az[idx];
    const double2 c = A[idx];
    return k == 1 ? make_double2(gy * c.x, gy * c.y) : c;
}

// cscale[k NX + n_x] = 2^e >= max over (n_y, n_z) of |Re C_k|, |Im C_k| (1 where C_k vanishes);
// one block per (k, n_x)
__global__ void __launch_bounds__(256) k_mmr_scale(EwaldDev e, const double2 *A, const double2 *Az, double *cscale)
{
    __shared__ double ws[8];
    const int NX = e.kmax[0] + 1, NY = 2 * e.kmax[1] + 1, NZ = 2 * e.kmax[2] + 1;
    const int k = blockIdx.x / NX, nx = blockIdx.x % NX;
    double m = 0.0;
    for (int t = threadIdx.x; t < NY * NZ; t += 256) {
        const int iy = t / NZ;
        const double gy = 6.283185307179586476925 * (iy - e.kmax[1]) / e.box[1];
        const double2 c = mmr_channel(A, Az, k, (size_t)nx * NY * NZ + t, gy);
        m = fmax(m, fmax(fabs(c.x), fabs(c.y)));
    }
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        double r = 0.0;
        for (int w = 0; w < 8; ++w) r = fmax(r, ws[w]);
        int ex = 0;
        if (r > 0.0) frexp(r, &ex);
        cscale[blockIdx.x] = r > 0.0 ? ldexp(1.0, ex) : 1.0;
    }
}

// B planes of one N tile (channels [kfirst, kfirst + nk)), per chunk of 8 (n_y, n_z) pairs, in the
// shared-memory layout: row (k, n_x, 0) holds (Re C, -Im C), row (k, n_x, 1) holds (Im C, Re C)
// of C_k / cscale.  A warp writes 8 rows x 4 pairs: 128 contiguous bytes of each plane.
template <int NP>
__global__ void k_mmr_bplanes(EwaldDev e, const double2 *A, const double2 *Az, const double *cscale, int kfirst,
                              int nk, int nr, int nchunk, uint32_t *bpl)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long per = (long long)nr * PCH;  // (row, pair) items of one chunk
    if (t >= per * nchunk) return;
    const int ch = (int)(t / per), it = (int)(t - (long long)ch * per);
    const int NX = e.kmax[0] + 1, NY = 2 * e.kmax[1] + 1, NZ = 2 * e.kmax[2] + 1;
    const int lane = it & 31, grp = it >> 5;
    const int j = (grp & 1) * 4 + (lane & 3), n = (grp >> 1) * 8 + (lane >> 2);
    const int p = ch * PCH + j;
    long long w0 = bal<NP>(), w1 = bal<NP>();
    if (n < 2 * nk * NX && p < NY * NZ) {
        const int kl = n / (2 * NX), nx = (n % (2 * NX)) >> 1, r = n & 1, k = kfirst + kl;
        const int iy = p / NZ, iz = p - iy * NZ;
        const double gy = 6.283185307179586476925 * (iy - e.kmax[1]) / e.box[1];
        const double2 c = mmr_channel(A, Az, k, ((size_t)nx * NY + iy) * NZ + iz, gy);
        const double sc = 1.0 / cscale[k * NX + nx];  // a power of two: exact
        const double re = c.x * sc, im = c.y * sc;
        constexpr double SC = (double)(1ll << mmr_bits(NP));
        w0 += __double2ll_rn((r ? im : re) * SC);
        w1 += __double2ll_rn((r ? re : -im) * SC);
    }
    const PlanesN<NP> p0 = planes_n<NP>(w0), p1 = planes_n<NP>(w1);
    const uint32_t words = mmr_bpl(nr) / 4;
    uint32_t *dst = bpl + (size_t)ch * NP * words + ((n >> 3) * CMN + (j >> 2) * CMK + (n & 7) * 16 + (j & 3) * 4) / 4;
#pragma unroll
    for (int s = 0; s < NP; ++s) dst[(size_t)s * words] = pack_bf16(p0.p[s], p1.p[s]);
}

// ---------------------------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------------------------
// nacc accumulators (levels 0 .. nacc-2 exact) of at most 512 / nacc columns each: the channels
// take as few N tiles as fit (FP64 path: 5, 96 rows; mixed path: 3, 160 rows)
void tc_mmr_shape(const EwaldDev &e, int nacc, int np, MmrShape &sh)
{
    sh.np = np;
    const int NX = e.kmax[0] + 1, NY = 2 * e.kmax[1] + 1, NZ = 2 * e.kmax[2] + 1;
    sh.nacc = nacc;
    sh.mtiles = (e.nmm + MM - 1) / MM;
    sh.npad = sh.mtiles * MM;
    sh.npair = NY * NZ;
    sh.nchunk = (sh.npair + PCH - 1) / PCH;
    const int maxr = std::min(NRMAX, 512 / nacc / 16 * 16);  // N rows that fit nacc accumulators
    int cpt = 3;  // channels per N tile: 2 cpt NX rows
    while (cpt > 1 && 2 * cpt * NX > maxr) --cpt;
    sh.cpt = cpt;
    sh.ntiles = (3 + cpt - 1) / cpt;
    sh.nr = (2 * cpt * NX + 15) / 16 * 16;
    sh.nr_last = (2 * (3 - (sh.ntiles - 1) * cpt) * NX + 15) / 16 * 16;
    sh.supported = sh.nr <= maxr && NZ >= PCH;  // a chunk of 8 pairs spans at most two n_y rows
    sh.nstg = mmr_smem(sh.nr, 3, np) <= SMEM_MAX ? 3 : 2;
    sh.phase_rows = (size_t)(NY + NZ) * sh.npad;
    sh.bplane_words = ((size_t)(sh.ntiles - 1) * mmr_bpl(sh.nr) + mmr_bpl(sh.nr_last)) * sh.nchunk * np / 4;
}

template <int NP>
static cudaError_t mm_recip_np(const EwaldDev &e, const MmrShape &sh, const MmrBuf &b, const double2 *A,
                               const double2 *Az, const int4 *Yt, const int4 *Zt, double *dq, double *dR, int *err,
                               cudaStream_t st);

cudaError_t launch_mm_recip_tc(const EwaldDev &e, const MmrShape &sh, const MmrBuf &b, const double2 *A,
                               const double2 *Az, double *dq, double *dR, int *err, cudaStream_t st)
{
    if (e.nmm == 0) return cudaSuccess;
    cudaError_t rc;
    const int NX = e.kmax[0] + 1, NY = 2 * e.kmax[1] + 1;
    int4 *Yt = b.phase, *Zt = Yt + (size_t)NY * sh.npad;
    k_mmr_phases<<<(unsigned)((2ll * e.nmm + 255) / 256), 256, 0, st>>>(e, sh.npad, Yt, Zt);
    if ((rc = cudaGetLastError()) != cudaSuccess) return rc;
    k_mmr_scale<<<3 * NX, 256, 0, st>>>(e, A, Az, b.cscale);
    if ((rc = cudaGetLastError()) != cudaSuccess) return rc;
    if (sh.np == MMR_NP_FP64) return mm_recip_np<MMR_NP_FP64>(e, sh, b, A, Az, Yt, Zt, dq, dR, err, st);
    if (sh.np == MMR_NP_MIXED) return mm_recip_np<MMR_NP_MIXED>(e, sh, b, A, Az, Yt, Zt, dq, dR, err, st);
    return cudaErrorInvalidValue;
}

// B planes and the MMA kernel with NP planes per operand
template <int NP>
static cudaError_t mm_recip_np(const EwaldDev &e, const MmrShape &sh, const MmrBuf &b, const double2 *A,
                               const double2 *Az, const int4 *Yt, const int4 *Zt, double *dq, double *dR, int *err,
                               cudaStream_t st)
{
    cudaError_t rc;
    const int NX = e.kmax[0] + 1, NY = 2 * e.kmax[1] + 1, NZ = 2 * e.kmax[2] + 1;
    const size_t smem = mmr_smem(sh.nr, sh.nstg, NP);
    static size_t at = 0;
    if (smem > at) {
        if ((rc = cudaFuncSetAttribute((const void *)k_mm_recip_tc<NP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem)) != cudaSuccess)
            return rc;
        at = smem;
    }
    const size_t tile_words = (size_t)sh.nchunk * NP * mmr_bpl(sh.nr) / 4;
    for (int tl = 0; tl < sh.ntiles; ++tl) {
        const int kfirst = tl * sh.cpt, nk = std::min(sh.cpt, 3 - kfirst);
        const int nr = tl + 1 == sh.ntiles ? sh.nr_last : sh.nr;
        const long long n = (long long)nr * PCH * sh.nchunk;
        k_mmr_bplanes<NP><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(e, A, Az, b.cscale, kfirst, nk, nr,
                                                                        sh.nchunk, b.bpl + tl * tile_words);
        if ((rc = cudaGetLastError()) != cudaSuccess) return rc;
    }
    MmrArgs a;
    a.Yt = Yt;
    a.Zt = Zt;
    a.bpl = b.bpl;
    a.cscale = b.cscale;
    a.mm_xyz = e.mm_xyz;
    a.mm_q = e.mm_q;
    a.dq = dq;
    a.dR = dR;
    a.err = err;
    a.nmm = e.nmm;
    a.npad = sh.npad;
    a.NX = NX;
    a.NY = NY;
    a.NZ = NZ;
    a.npair = sh.npair;
    a.nchunk = sh.nchunk;
    a.nr = sh.nr;
    a.nr_last = sh.nr_last;
    a.cpt = sh.cpt;
    a.nstg = sh.nstg;
    a.nacc = sh.nacc;
    a.box0 = e.box[0];
    k_mm_recip_tc<NP><<<dim3(sh.mtiles, sh.ntiles), NTHR, smem, st>>>(a);
    if ((rc = cudaGetLastError()) != cudaSuccess) return rc;
    return cudaSuccess;
}

}  // namespace qmmm
