// recip_tc.cu -- the MM structure factor of the reciprocal Ewald sum (SI, "Multipolar Ewald",
// long-range part) on the tensor cores.
//
// S(G) = sum_i q_i exp(i G.R_i) over the half space n_x >= 0 of the cube |n_c| <= kmax, with
// separable phases exp(i G.R) = X(n_x) Y(n_y) Z(n_z), is a product of two matrices:
//
//   S[(n_x, n_y), n_z] = sum_i a_i(n_x, n_y) z_i(n_z),   a_i = q_i X_i(n_x) Y_i(n_y),  z_i = Z_i(n_z)
//
// written in real arithmetic as D[line, (n_z, re/im)] = sum_k A[line, k] B[(n_z, re/im), k] with
// k = (charge, re/im).  The tensor cores multiply BF16 operands exactly and accumulate in FP32, so
// the FP64-class product is built from exact pieces (an Ozaki-type split): every operand element,
// a 48-bit fixed-point number v (|v| <= 2^48, scaled by 1/max|q| for A), is written as seven
// balanced digit planes, a leading one and six of base 128,
//     v 2^-48 = 2^-6 sum_{s<7} p_s,   p_0 in [-64, 64],  p_s in [-64, 63] 2^-7s (s >= 1),
// each p_s exact in BF16 (at most 7 significant bits).  Products of planes with s + t = l carry
// the weight 2^-7l; for l <= 3 each level has its own FP32 accumulator in tensor memory and stays
// an exact integer multiple of 2^-7l over a K block of 1024 terms ((l + 1) 4096 * 1024 <= 2^24),
// levels 4..6 share one accumulator whose FP32 rounding sits near 2^-52 of the leading level, and
// the pairs with s + t >= 7 (weight <= 2^-49) are dropped: 28 plane pairs.  Each CTA (a 128-line
// tile, an N tile and a block of 512 charges) writes its five accumulators; a second kernel sums
// the exact levels over the charge blocks in 64-bit integers and combines them in FP64.
//
// Kernels, in order: per-block max |q|; fixed-point phase rows (one sincospi pair per charge and
// axis, the recurrence in integers); the B digit planes (the n_z phases are shared by every line
// tile, so they are digitised once, straight into the shared-memory layout of the MMA); the MMA
// kernel; the reduction over charge blocks.  In the MMA kernel one thread stages the B planes and
// the phase rows of the next chunk of 16 charges with TMA bulk copies, 16 producer warps build the
// A planes of a chunk (an outer product formed on chip: nothing of it goes to HBM), one thread
// issues the 56 tcgen05.mma of a chunk (2 K-steps x 28 plane pairs), double-buffered through
// mbarriers, and the epilogue reads tensor memory with tcgen05.ld.
#include <algorithm>

#include "device_common.cuh"
#include "qmmm_internal.h"
#include "tc_common.cuh"
#include "tc_digits.cuh"

namespace qmmm {

namespace {
using namespace tcd;
constexpr int TCM = 128;               // lines per tile (MMA M)
constexpr int TCND = tcd::ND;           // digit planes
constexpr int TCKC = 32;               // K entries per chunk (16 charges x re/im): two MMA K-steps
constexpr int TCCH = TCKC / 2;         // charges per chunk
constexpr int TCNCH = 32;              // chunks per charge block
constexpr int NSTAGE = 2;              // pipeline depth (A, B and phase-row buffers)
constexpr int TCCPB = TCCH * TCNCH;    // charges per CTA (512; K block of 1024)
constexpr int TCNACC = 5;              // accumulators: levels 0..3 exact, levels 4..6 merged
constexpr int TCPROD = 16;             // producer warps
constexpr int TCTHREADS = (TCPROD + 2) * 32;  // + the MMA warp + the loader warp
constexpr uint32_t A_PLANE = TCM * TCKC * 2;  // bytes per A digit plane of a chunk
constexpr uint32_t CM_K = 128;                // byte step between core matrices along K
constexpr uint32_t CM_MN = (TCKC / 8) * 128;  // byte step between 8-row groups
constexpr size_t TC_SMEM_MAX = 232448;           // 227 KB per CTA
constexpr int BMAX_CH = 4096;                    // charges per block of the max |q| reduction

__host__ __device__ inline int tc_cstride(int ntr) { return (ntr + 31) / 32 * 32; }
__host__ __device__ inline uint32_t tc_bplane_bytes(int ntr) { return (uint32_t)ntr * TCKC * 2; }
__host__ __device__ inline uint32_t tc_stage_bytes(int ntr) { return TCND * (A_PLANE + tc_bplane_bytes(ntr)); }
// phase rows of one chunk for the A operand: 16 charges x (NX + NY) entries of 16 bytes
__host__ __device__ inline uint32_t tc_pbuf_bytes(int nrow) { return (uint32_t)TCCH * nrow * 16; }
__host__ inline size_t tc_smem_bytes(int ntr, int nrow, bool staged)
{
    return NSTAGE * ((size_t)tc_stage_bytes(ntr) + (staged ? (size_t)tc_pbuf_bytes(nrow) : 0)) + 256;
}

struct TcSfArgs {
    const int4 *qx, *py;  // [npad][NX], [npad][NY] split 2^61 fixed point
    const uint32_t *bpl;  // B planes, per (block, chunk, N tile): TCND * bplane bytes
    int *part;            // per CTA: [5][ntr][128]
    int *err;
    int nmm, NX, NY, NL;
    int ntiles, ntr, mtiles;
};
}  // namespace

// grid (mtiles, nkb * ntiles), TCTHREADS threads, tc_smem_bytes() dynamic shared memory.  STAGED:
// the A phase rows of each chunk come through shared memory (TMA bulk copies); otherwise the
// producers read them from global memory.  The B planes always come by bulk copy.  Chunk ch uses
// buffer set ch % NSTAGE; its barriers complete once per use, phase parity (ch / NSTAGE) & 1.
template <bool STAGED>
__global__ void __launch_bounds__(TCTHREADS, 1) k_sf_tc(TcSfArgs a)
{
    extern __shared__ __align__(1024) unsigned char sm[];
    const int ntr = a.ntr, NX = a.NX, NY = a.NY;
    const uint32_t b_plane = tc_bplane_bytes(ntr), stage = tc_stage_bytes(ntr), bbytes = TCND * b_plane;
    const uint32_t pbytes = STAGED ? tc_pbuf_bytes(NX + NY) : 0;
    unsigned char *pbuf0 = sm + NSTAGE * stage;
    // per stage: full (producers), bfull (B copy), pfull (phase copy), empty (MMA done); then done
    uint64_t *bars = reinterpret_cast<uint64_t *>(pbuf0 + NSTAGE * pbytes);
    uint64_t *full = bars, *bfull = bars + NSTAGE, *pfull = bars + 2 * NSTAGE, *empty = bars + 3 * NSTAGE;
    uint64_t *done = bars + 4 * NSTAGE;
    uint32_t *tslot = reinterpret_cast<uint32_t *>(done + 1);
    volatile int *abort = reinterpret_cast<volatile int *>(tslot + 1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int mt = blockIdx.x, kb = blockIdx.y / a.ntiles, nt = blockIdx.y % a.ntiles;
    const int cstr = tc_cstride(ntr);

    if (threadIdx.x == 0) {
        for (int k = 0; k < NSTAGE; ++k) {
            mbar_init(&full[k], TCPROD);
            mbar_init(&bfull[k], 1);
            mbar_init(&pfull[k], 1);
            mbar_init(&empty[k], 1);
        }
        mbar_init(done, 1);
        *abort = 0;
        fence_mbar_init();
    }
    if (warp == TCPROD) {
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

    if (warp < TCPROD) {
        // ---------------- producers: A digit planes of one chunk ----------------
        // 128 lines x TCCH charges in groups of 8 rows x 4 charges (32 distinct banks); the line
        // indices of a thread are the same for every chunk
        constexpr int NCG = TCCH / 4, AJ = 16 * NCG / TCPROD;
        int a_nx[AJ], a_iy[AJ], a_c[AJ];
        uint32_t a_off[AJ];
#pragma unroll
        for (int j = 0; j < AJ; ++j) {
            const int combo = warp * AJ + j, rg = combo / NCG, cg = combo % NCG;
            const int r = rg * 8 + (lane >> 2), line = mt * TCM + r;
            a_c[j] = cg * 4 + (lane & 3);
            a_nx[j] = line < a.NL ? line / NY : -1;
            a_iy[j] = line < a.NL ? line - a_nx[j] * NY : 0;
            a_off[j] = rg * CM_MN + cg * CM_K + (lane >> 2) * 16 + (lane & 3) * 4;
        }
        for (int ch = 0; ch < TCNCH; ++ch) {
            const int st = ch % NSTAGE, u = ch / NSTAGE;
            if (ch >= NSTAGE && !tc::mbar_wait_thread(&empty[st], (u - 1) & 1, abort)) {
                give_up();
                break;
            }
            if (STAGED && !tc::mbar_wait_thread(&pfull[st], u & 1, abort)) {
                give_up();
                break;
            }
            unsigned char *sA = sm + st * stage;
            const int c0 = kb * TCCPB + ch * TCCH, cmax = a.nmm - c0;
            const int4 *qx, *py;
            if (STAGED) {
                qx = reinterpret_cast<const int4 *>(pbuf0 + st * pbytes);
                py = qx + TCCH * NX;
            } else {
                qx = a.qx + (size_t)c0 * NX;
                py = a.py + (size_t)c0 * NY;
            }
#pragma unroll
            for (int j = 0; j < AJ; ++j) {
                const int c = a_c[j];
                if (a_nx[j] >= 0 && c < cmax) {
                    long long re, im;  // 2^60 scale
                    cmul61(qx[c * NX + a_nx[j]], py[c * NY + a_iy[j]], re, im);
                    const Planes pr = planes(fixw(re, 12)), pi = planes(fixw(im, 12));
#pragma unroll
                    for (int s = 0; s < TCND; ++s)
                        *reinterpret_cast<uint32_t *>(sA + s * A_PLANE + a_off[j]) = pack_bf16(pr.p[s], pi.p[s]);
                } else {
#pragma unroll
                    for (int s = 0; s < TCND; ++s) *reinterpret_cast<uint32_t *>(sA + s * A_PLANE + a_off[j]) = 0u;
                }
            }
            tc::fence_proxy_async_smem();
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(&full[st]);
        }
    } else if (warp == TCPROD) {
        if (lane == 0) {
            // ---------------- MMA issue: one thread, 28 plane pairs per K-step ----------------
            const uint32_t idesc = tc::idesc_bf16_f32(TCM, ntr);
            for (int ch = 0; ch < TCNCH; ++ch) {
                const int st = ch % NSTAGE, u = ch / NSTAGE;
                if (!tc::mbar_wait_thread(&full[st], u & 1, abort) || !tc::mbar_wait_thread(&bfull[st], u & 1, abort)) {
                    give_up();
                    break;
                }
                tc::fence_after_sync();
                const uint32_t sA = smem_addr(sm + st * stage), sB = sA + TCND * A_PLANE;
#pragma unroll 1
                for (int kk = 0; kk < TCKC / 16; ++kk)
#pragma unroll
                    for (int s = 0; s < TCND; ++s)
#pragma unroll
                        for (int t = 0; t < TCND - s; ++t) {
                            const int acc = s + t < TCNACC - 1 ? s + t : TCNACC - 1;
                            const uint32_t first = (ch == 0 && kk == 0 && s == 0 && t == acc);
                            const uint64_t ad = tc::smem_desc(sA + s * A_PLANE + kk * 2 * CM_K, CM_K, CM_MN);
                            const uint64_t bd = tc::smem_desc(sB + t * b_plane + kk * 2 * CM_K, CM_K, CM_MN);
                            tc::mma_bf16(tbase + acc * cstr, ad, bd, idesc, first ? 0u : 1u);
                        }
                tc::commit(&empty[st]);
            }
            tc::commit(done);
        }
    } else if (lane == 0) {
        // ---------------- loader: phase rows and B planes of chunk ch ----------------
        int issued = 0, pissued = 0;
        for (int ch = 0; ch < TCNCH; ++ch) {
            const int st = ch % NSTAGE, u = ch / NSTAGE;
            const size_t c0 = (size_t)kb * TCCPB + (size_t)ch * TCCH;
            if (STAGED) {
                // the producers have finished chunk ch - NSTAGE: its phase rows are no longer read
                if (ch >= NSTAGE && !tc::mbar_wait_thread(&full[st], (u - 1) & 1, abort)) {
                    give_up();
                    break;
                }
                unsigned char *dst = pbuf0 + st * pbytes;
                mbar_arrive_expect_tx(&pfull[st], pbytes);
                bulk_g2s(dst, a.qx + c0 * NX, TCCH * NX * 16, &pfull[st]);
                bulk_g2s(dst + TCCH * NX * 16, a.py + c0 * NY, TCCH * NY * 16, &pfull[st]);
                pissued = ch + 1;
            }
            // the MMA has finished chunk ch - NSTAGE: the B area of the buffer set is free
            if (ch >= NSTAGE && !tc::mbar_wait_thread(&empty[st], (u - 1) & 1, abort)) {
                give_up();
                break;
            }
            const uint32_t *src = a.bpl + ((size_t)(kb * TCNCH + ch) * a.ntiles + nt) * (bbytes / 4);
            mbar_arrive_expect_tx(&bfull[st], bbytes);
            bulk_g2s(sm + st * stage + TCND * A_PLANE, src, bbytes, &bfull[st]);
            issued = ch + 1;
        }
        // copies possibly still in flight (after a give-up): wait for them to land, bounded in time
        // only (not cut short by the abort flag), before the block may leave
        for (int ch = issued > NSTAGE ? issued - NSTAGE : 0; ch < issued; ++ch)
            tc::mbar_drain(&bfull[ch % NSTAGE], (ch / NSTAGE) & 1);
        for (int ch = pissued > NSTAGE ? pissued - NSTAGE : 0; ch < pissued; ++ch)
            tc::mbar_drain(&pfull[ch % NSTAGE], (ch / NSTAGE) & 1);
    }

    // ---------------- epilogue: tensor memory -> per-CTA partials (warps 0..7) ----------------
    if (warp < 8) {
        if (!tc::mbar_wait_thread(done, 0, abort)) {
            give_up();
            // the MMA thread commits `done` on every path: wait for it (bounded in time only), so
            // that no MMA still writes tensor memory when it is freed below
            tc::mbar_drain(done, 0);
        } else {
            tc::fence_after_sync();
            const int q = warp & 3, half = warp >> 2, row = 32 * q + lane;
            int *dst = a.part + (size_t)((kb * a.ntiles + nt) * a.mtiles + mt) * (TCNACC * ntr * TCM);
            const int cw = ntr / 2;
            for (int acc = 0; acc < TCNACC; ++acc)
                for (int cb = half * cw; cb < half * cw + cw; cb += 8) {
                    float v[8];
                    tc::tmem_ld8(tbase + ((uint32_t)(32 * q) << 16) + acc * cstr + cb, v);
                    tc::tmem_wait_ld();
                    const float sc = acc < TCNACC - 1 ? (float)(1 << (7 * acc)) : 1.0f;
#pragma unroll
                    for (int k = 0; k < 8; ++k) {
                        const int w = acc < TCNACC - 1 ? __float2int_rn(v[k] * sc) : __float_as_int(v[k]);
                        dst[((size_t)acc * ntr + cb + k) * TCM + row] = w;
                    }
                }
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == TCPROD) {
        tc::fence_after_sync();
        tc::tmem_dealloc(tbase, 512);
    }
}

// B digit planes of every (charge block, chunk, N tile), in the shared-memory layout of one stage:
// row (n_z, re) holds (z_re, -z_im), row (n_z, im) holds (z_im, z_re) per charge.  One thread per
// (row, charge); a warp covers 8 rows x 4 charges, i.e. 128 contiguous bytes of each plane.
__global__ void k_tc_bplanes(const int4 *pz, int nmm, int NZ, int ntiles, int ntr, long long nitems, uint32_t *bpl)
{
    const long long item = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (item >= nitems) return;
    const int per = ntr * TCCH;  // items of one (block, chunk, N tile)
    const long long grp = item / per;
    const int it = (int)(item - grp * per);
    const int nt = (int)(grp % ntiles), chunk = (int)(grp / ntiles);  // chunk over all blocks
    constexpr int NCG = TCCH / 4;  // groups of 4 charges
    const int ln = it & 31, combo = it >> 5;
    const int c = (combo % NCG) * 4 + (ln & 3);
    const int izl = (combo / NCG) * 4 + ((ln >> 2) & 3), rr = ln >> 4;
    const int iz = nt * (ntr / 2) + izl, n = 2 * izl + rr;
    const int ci = chunk * TCCH + c;
    long long w0 = BAL, w1 = BAL;
    if (iz < NZ && ci < nmm) {
        const int4 z = pz[(size_t)ci * NZ + iz];
        const long long r48 = fixw(join61(z.x, z.y), 13) - BAL, i48 = fixw(join61(z.z, z.w), 13) - BAL;
        w0 += rr ? i48 : r48;
        w1 += rr ? r48 : -i48;
    }
    const Planes p0 = planes(w0), p1 = planes(w1);
    const uint32_t b_words = tc_bplane_bytes(ntr) / 4;
    uint32_t *dst = bpl + (size_t)grp * (TCND * b_words) +
                    ((n >> 3) * CM_MN + (c >> 2) * CM_K + (n & 7) * 16 + (c & 3) * 4) / 4;
#pragma unroll
    for (int s = 0; s < TCND; ++s) dst[(size_t)s * b_words] = pack_bf16(p0.p[s], p1.p[s]);
}

// S[line * NZ + iz] from the partials: grid (mtiles, NZ), 4 x 128 threads: a row of the line tile
// per thread, the charge blocks split over the four thread groups and added in a fixed order
constexpr int RED_G = 4;
__device__ __forceinline__ double max_of(const double *bmax, int n)
{
    double m = 0.0;
    for (int k = 0; k < n; ++k) m = fmax(m, bmax[k]);
    return m > 0.0 ? m : 1.0;
}
__global__ void __launch_bounds__(TCM *RED_G) k_sf_tc_reduce(const int *part, int nkb, int ntiles, int ntr,
                                                            int mtiles, int NL, int NZ, const double *bmax,
                                                            int nbmax, double2 *S)
{
    __shared__ long long sI[RED_G - 1][2][TCNACC - 1][TCM];
    __shared__ double sF[RED_G - 1][2][TCM];
    const int mt = blockIdx.x, iz = blockIdx.y, row = threadIdx.x & (TCM - 1), g = threadIdx.x / TCM;
    const int line = mt * TCM + row;
    const int half = ntr / 2, nt = iz / half, nl = 2 * (iz - nt * half);
    long long I[2][TCNACC - 1] = {};
    double F[2] = {0.0, 0.0};
    if (line < NL)
        for (int kb = g; kb < nkb; kb += RED_G) {
            const int *p = part + (size_t)((kb * ntiles + nt) * mtiles + mt) * (TCNACC * ntr * TCM);
#pragma unroll
            for (int r = 0; r < 2; ++r) {
#pragma unroll
                for (int acc = 0; acc < TCNACC - 1; ++acc) I[r][acc] += p[((size_t)acc * ntr + nl + r) * TCM + row];
                F[r] += (double)__int_as_float(p[((size_t)(TCNACC - 1) * ntr + nl + r) * TCM + row]);
            }
        }
    if (g > 0) {
        for (int r = 0; r < 2; ++r) {
            for (int acc = 0; acc < TCNACC - 1; ++acc) sI[g - 1][r][acc][row] = I[r][acc];
            sF[g - 1][r][row] = F[r];
        }
    }
    __syncthreads();
    if (g > 0 || line >= NL) return;
    for (int h = 0; h < RED_G - 1; ++h)
        for (int r = 0; r < 2; ++r) {
            for (int acc = 0; acc < TCNACC - 1; ++acc) I[r][acc] += sI[h][r][acc][row];
            F[r] += sF[h][r][row];
        }
    const double sc = max_of(bmax, nbmax) * 0x1p-12;
    double v[2];
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        double t = F[r];
        for (int acc = TCNACC - 2; acc >= 0; --acc) t += ldexp((double)I[r][acc], -7 * acc);
        v[r] = sc * t;
    }
    S[(size_t)line * NZ + iz] = make_double2(v[0], v[1]);
}

// bmax[b] = max |q_i| over charges [b BMAX_CH, (b + 1) BMAX_CH)
__global__ void __launch_bounds__(256) k_absmax(const double *q, int n, double *bmax)
{
    __shared__ double ws[8];
    const int i0 = blockIdx.x * BMAX_CH;
    double m = 0.0;
#pragma unroll 4
    for (int k = threadIdx.x; k < BMAX_CH; k += 256)
        if (i0 + k < n) m = fmax(m, fabs(q[i0 + k]));
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        double r = 0.0;
        for (int w = 0; w < 8; ++w) r = fmax(r, ws[w]);
        bmax[blockIdx.x] = r;
    }
}

// fixed-point phase rows: qx = (q_i / max|q|) X_i(n_x), py = Y_i(n_y), pz = Z_i(n_z), split 2^61;
// one thread per (axis, charge): the start and the step from FP64 sincospi, the recurrence in
// 2^61 fixed point (each step rounds within 2^-60; at most 2 kmax + 1 steps)
__global__ void k_tc_phases(EwaldDev e, const double *bmax, int nbmax, int4 *qx, int4 *py, int4 *pz)
{
    const long long item = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (item >= 3ll * e.nmm) return;
    const int d = (int)(item / e.nmm), i = (int)(item - (long long)d * e.nmm);
    const int len = d == 0 ? e.kmax[0] + 1 : 2 * e.kmax[d] + 1, off = d == 0 ? 0 : e.kmax[d];
    int4 *row = (d == 0 ? qx : d == 1 ? py : pz) + (size_t)i * len;
    const double u = e.mm_xyz[3 * i + d] / e.box[d];
    const double scale = d == 0 ? e.mm_q[i] / max_of(bmax, nbmax) : 1.0;
    double sn, cs;
    sincospi(2.0 * u, &sn, &cs);
    const long long sr = fix61(cs), si = fix61(sn);
    sincospi(-2.0 * (double)off * u, &sn, &cs);
    long long pr = fix61(cs * scale), pi = fix61(sn * scale);
    for (int n = 0; n < len; ++n) {
        row[n] = split61(pr, pi);
        const long long nr = (mul61(pr, sr) - mul61(pi, si)) * 2;  // 2^60 -> 2^61
        const long long ni = (mul61(pr, si) + mul61(pi, sr)) * 2;
        pr = nr;
        pi = ni;
    }
}

// ---------------------------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------------------------
void tc_sf_shape(const EwaldDev &e, TcShape &sh)
{
    const int NX = e.kmax[0] + 1, NY = 2 * e.kmax[1] + 1, NZ = 2 * e.kmax[2] + 1;
    sh.NL = NX * NY;
    sh.mtiles = (sh.NL + TCM - 1) / TCM;
    const int rows = 2 * NZ;
    sh.ntiles = (rows + 79) / 80;
    int per = (rows + sh.ntiles - 1) / sh.ntiles;  // rows per N tile, even
    per += per & 1;
    sh.ntr = (per + 15) / 16 * 16;                  // <= 80: 5 accumulators fit in 512 TMEM columns
    sh.nkb = (e.nmm + TCCPB - 1) / TCCPB;
    sh.nbmax = (e.nmm + BMAX_CH - 1) / BMAX_CH;
    sh.part_ints = (size_t)sh.nkb * sh.ntiles * sh.mtiles * TCNACC * sh.ntr * TCM;
    // phase rows for whole charge blocks (the bulk copies of the last block stay in bounds)
    sh.phase_rows = (size_t)sh.nkb * TCCPB * (NX + NY + NZ);
    sh.bplane_words = (size_t)sh.nkb * TCNCH * sh.ntiles * TCND * tc_bplane_bytes(sh.ntr) / 4;
    sh.staged = tc_smem_bytes(sh.ntr, NX + NY, true) <= TC_SMEM_MAX;
}

cudaError_t launch_structure_factor_tc(const EwaldDev &e, const TcShape &sh, const TcBuf &b, double2 *S, int *err,
                                       cudaStream_t st)
{
    if (e.nmm == 0) return cudaMemsetAsync(S, 0, sizeof(double2) * (size_t)ewald_dense_size(e), st);
    cudaError_t rc;
    const int NX = e.kmax[0] + 1, NY = 2 * e.kmax[1] + 1, NZ = 2 * e.kmax[2] + 1;
    k_absmax<<<sh.nbmax, 256, 0, st>>>(e.mm_q, e.nmm, b.bmax);
    if ((rc = cudaGetLastError()) != cudaSuccess) return rc;
    const size_t npad = (size_t)sh.nkb * TCCPB;
    int4 *qx = b.phase, *py = qx + npad * NX, *pz = py + npad * NY;
    {
        const long long n = 3ll * e.nmm;
        k_tc_phases<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(e, b.bmax, sh.nbmax, qx, py, pz);
        if ((rc = cudaGetLastError()) != cudaSuccess) return rc;
    }
    {
        const long long n = (long long)sh.nkb * TCNCH * sh.ntiles * sh.ntr * TCCH;
        k_tc_bplanes<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(pz, e.nmm, NZ, sh.ntiles, sh.ntr, n, b.bpl);
        if ((rc = cudaGetLastError()) != cudaSuccess) return rc;
    }
    {
        const size_t smem = tc_smem_bytes(sh.ntr, NX + NY, sh.staged);
        const void *fn = sh.staged ? (const void *)k_sf_tc<true> : (const void *)k_sf_tc<false>;
        static size_t attr[2] = {0, 0};
        if (smem > attr[sh.staged]) {
            if ((rc = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess)
                return rc;
            attr[sh.staged] = smem;
        }
        TcSfArgs a;
        a.qx = qx;
        a.py = py;
        a.bpl = b.bpl;
        a.part = b.part;
        a.err = err;
        a.nmm = e.nmm;
        a.NX = NX;
        a.NY = NY;
        a.NL = sh.NL;
        a.ntiles = sh.ntiles;
        a.ntr = sh.ntr;
        a.mtiles = sh.mtiles;
        const dim3 grid(sh.mtiles, sh.nkb * sh.ntiles);
        if (sh.staged)
            k_sf_tc<true><<<grid, TCTHREADS, smem, st>>>(a);
        else
            k_sf_tc<false><<<grid, TCTHREADS, smem, st>>>(a);
        if ((rc = cudaGetLastError()) != cudaSuccess) return rc;
    }
    k_sf_tc_reduce<<<dim3(sh.mtiles, NZ), TCM * RED_G, 0, st>>>(b.part, sh.nkb, sh.ntiles, sh.ntr, sh.mtiles, sh.NL,
                                                               NZ, b.bmax, sh.nbmax, S);
    return cudaGetLastError();
}

}  // namespace qmmm
