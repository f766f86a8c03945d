// ewald.cu -- region I and the multipolar Ewald interaction between QM multipoles and MM charges
// (Eq. 6, QM-MM lines; Eq. 10; SI "Multipolar Ewald"), FP64 throughout.
//
// Region-II potential at QM atom j (20 Taylor components c):
//   v_j,c = sum_i q_i [ psi_c(R_j - R_i) - sum_{L: i+L in I} T_c - sum_{L: i+L not in I} That_c(1/sigma_i) ]
//   psi = psi_SR (erfc(alpha r)/r tensors over images within the Ewald cutoff)
//       + psi_LR ((4 pi / V) sum_{G != 0} exp(-G^2/4alpha^2)/G^2 cos(G.(R_j - R_i)) and its
//         derivatives, prefactors (iG)^n / n!)
//       - pi/(V alpha^2) on the monopole (neutralising background).
// The reciprocal part uses the structure factor S(G) = sum_i q_i exp(i G.R_i), evaluated over the
// half space of the cube |n_c| <= kmax (the -G partner is its conjugate) with separable phases
// exp(i G.R) = X(n_x) Y(n_y) Z(n_z): a thread owns one (n_x, n_y) line and eight n_z values, so each
// (G, charge) term costs one complex multiply-add.
// The adjoint needs the same tensors contracted with the multipoles, at every MM site:
//   dE/dq_i = sum_j sum_c w_c M_j,c Psi_c(j,i),  dE/dR_i = -q_i sum_j sum_c w_c M_j,c dPsi_c/dR_j.
#include <algorithm>

#include "device_common.cuh"
#include "qmmm_internal.h"

namespace qmmm {

// ---------------------------------------------------------------------------------------------
// region I
// ---------------------------------------------------------------------------------------------
__device__ __forceinline__ bool in_region1(const EwaldDev &e, double x, double y, double z)
{
    const double dx = x - e.centre[0], dy = y - e.centre[1], dz = z - e.centre[2];
    return dx * dx + dy * dy + dz * dz < e.rcut * e.rcut;
}

// Images of MM charge i that lie in region I, in (nx, ny, nz) order; calls f(pos, n) for each.
template <typename Fn>
__device__ __forceinline__ int region1_images(const EwaldDev &e, int i, Fn f)
{
    const double x = e.mm_xyz[3 * i], y = e.mm_xyz[3 * i + 1], z = e.mm_xyz[3 * i + 2];
    const double n0x = -rint((x - e.centre[0]) / e.box[0]);
    const double n0y = -rint((y - e.centre[1]) / e.box[1]);
    const double n0z = -rint((z - e.centre[2]) / e.box[2]);
    const int mx = (int)ceil(e.rcut / e.box[0]), my = (int)ceil(e.rcut / e.box[1]), mz = (int)ceil(e.rcut / e.box[2]);
    int cnt = 0;
    for (int a = -mx; a <= mx; ++a)
        for (int b = -my; b <= my; ++b)
            for (int c = -mz; c <= mz; ++c) {
                const double px = x + (n0x + a) * e.box[0];
                const double py = y + (n0y + b) * e.box[1];
                const double pz = z + (n0z + c) * e.box[2];
                if (in_region1(e, px, py, pz)) {
                    f(px, py, pz, cnt);
                    ++cnt;
                }
            }
    return cnt;
}

__global__ void k_region1_count(EwaldDev e, int *blk_count, int *cls_count)
{
    __shared__ int ws[32];
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    int cnt = 0;
    if (i < e.nmm) {
        cnt = region1_images(e, i, [](double, double, double, int) {});
        if (cnt) atomicAdd(cls_count + e.mm_cls[i], cnt);
    }
    int s = cnt;
#pragma unroll
    for (int k = 16; k > 0; k >>= 1) s += __shfl_xor_sync(FULL, s, k);
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        int t = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += ws[w];
        blk_count[blockIdx.x] = t;
    }
}

// exclusive scan of nblk counts in place; blk[nblk] receives the total (single block)
__global__ void k_scan_blocks(int *blk, int nblk)
{
    __shared__ int carry;
    __shared__ int ws[32];
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int base = 0; base < nblk; base += blockDim.x) {
        const int i = base + threadIdx.x;
        const int v = i < nblk ? blk[i] : 0;
        // inclusive warp scan
        int x = v;
#pragma unroll
        for (int k = 1; k < 32; k <<= 1) {
            const int o = __shfl_up_sync(FULL, x, k);
            if ((threadIdx.x & 31) >= k) x += o;
        }
        if ((threadIdx.x & 31) == 31) ws[threadIdx.x >> 5] = x;
        __syncthreads();
        if (threadIdx.x < 32) {
            int y = threadIdx.x < (blockDim.x >> 5) ? ws[threadIdx.x] : 0;
#pragma unroll
            for (int k = 1; k < 32; k <<= 1) {
                const int o = __shfl_up_sync(FULL, y, k);
                if (threadIdx.x >= k) y += o;
            }
            ws[threadIdx.x] = y;
        }
        __syncthreads();
        const int wpre = (threadIdx.x >> 5) ? ws[(threadIdx.x >> 5) - 1] : 0;
        const int excl = carry + wpre + x - v;
        const int tot = ws[(blockDim.x >> 5) - 1];
        __syncthreads();
        if (i < nblk) blk[i] = excl;
        if (threadIdx.x == 0) carry += tot;
        __syncthreads();
    }
    if (threadIdx.x == 0) blk[nblk] = carry;
}

__global__ void k_region1_fill(EwaldDev e, const int *blk_off, double4_32a *chg, float4 *hi, float4 *lo, int *idx)
{
    __shared__ int ws[32];
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    int cnt = 0;
    if (i < e.nmm) cnt = region1_images(e, i, [](double, double, double, int) {});
    // block exclusive scan of cnt
    int x = cnt;
#pragma unroll
    for (int k = 1; k < 32; k <<= 1) {
        const int o = __shfl_up_sync(FULL, x, k);
        if ((threadIdx.x & 31) >= k) x += o;
    }
    if ((threadIdx.x & 31) == 31) ws[threadIdx.x >> 5] = x;
    __syncthreads();
    if (threadIdx.x < 32) {
        int y = threadIdx.x < (blockDim.x >> 5) ? ws[threadIdx.x] : 0;
#pragma unroll
        for (int k = 1; k < 32; k <<= 1) {
            const int o = __shfl_up_sync(FULL, y, k);
            if (threadIdx.x >= k) y += o;
        }
        ws[threadIdx.x] = y;
    }
    __syncthreads();
    const int wpre = (threadIdx.x >> 5) ? ws[(threadIdx.x >> 5) - 1] : 0;
    const int base = blk_off[blockIdx.x] + wpre + x - cnt;
    if (i < e.nmm && cnt) {
        const double q = e.mm_q[i];
        region1_images(e, i, [&](double px, double py, double pz, int k) {
            const int o = base + k;
            double4_32a c;
            c.x = px; c.y = py; c.z = pz; c.w = q;
            chg[o] = c;
            float hx, hy, hz, lx, ly, lz;  // grid-split hi/lo about the QM centre (split_grid)
            split_grid(px - e.centre[0], hx, lx);
            split_grid(py - e.centre[1], hy, ly);
            split_grid(pz - e.centre[2], hz, lz);
            hi[o] = make_float4(hx, hy, hz, (float)q);
            lo[o] = make_float4(lx, ly, lz, 0.0f);
            idx[o] = i;
        });
    }
}

cudaError_t launch_region1_count(const EwaldDev &e, int *blk_count, int *cls_count, int nblk, cudaStream_t st)
{
    k_region1_count<<<nblk, 256, 0, st>>>(e, blk_count, cls_count);
    return cudaGetLastError();
}
cudaError_t launch_scan_blocks(int *blk, int nblk, cudaStream_t st)
{
    k_scan_blocks<<<1, 1024, 0, st>>>(blk, nblk);
    return cudaGetLastError();
}
cudaError_t launch_region1_fill(const EwaldDev &e, const int *blk_off, double4_32a *chg, float4 *hi, float4 *lo,
                                int *idx, int nblk, cudaStream_t st)
{
    k_region1_fill<<<nblk, 256, 0, st>>>(e, blk_off, chg, hi, lo, idx);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------------
// block reduction of NV doubles into out[] (deterministic: fixed tree)
// ---------------------------------------------------------------------------------------------
template <int NV>
__device__ __forceinline__ void block_reduce_store(double (&v)[NV], double *out, double *scratch /* 32*NV */)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int k = 0; k < NV; ++k) v[k] = warp_sum(v[k]);
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < NV; ++k) scratch[w * NV + k] = v[k];
    __syncthreads();
    if (threadIdx.x < NV) {
        double s = 0.0;
        for (int ww = 0; ww < nw; ++ww) s += scratch[ww * NV + threadIdx.x];
        out[threadIdx.x] = s;
    }
    __syncthreads();
}

// The FP32 check in front of the FP64 evaluation of the real-space sums: with the minimum image
// only (no further images searched), a pair farther apart than sqrt(lim2) is certainly outside
// both ranges.  lim2 carries a margin (relative 1e-3 and 0.05 bohr) far above the FP32 rounding
// of the positions and the displacement, so no pair the FP64 test accepts is dropped; with images
// beyond the minimum one it never filters.
__device__ __forceinline__ float filter_lim2(double rc, double rhat)
{
    const double r = fmax(rc, rhat) * 1.001 + 0.05;
    return (float)(r * r);
}
// The same test from the FP32 positions of a QM atom (a) and a charge (c, with its squared filter
// radius in c.w): rounding the positions to FP32 moves a displacement by a few 1e-5 bohr at most,
// far inside the margin of filter_lim2
__device__ __forceinline__ bool far_min_image_f(const EwaldDev &e, float4 a, float4 c)
{
    if (e.img[0] | e.img[1] | e.img[2]) return false;
    const float bx = (float)e.box[0], by = (float)e.box[1], bz = (float)e.box[2];
    const float fx = a.x - c.x, fy = a.y - c.y, fz = a.z - c.z;
    const float x = fx - rintf(fx / bx) * bx, y = fy - rintf(fy / by) * by, z = fz - rintf(fz / bz) * bz;
    return x * x + y * y + z * z > c.w;
}

// FP32 inputs of the real-space pre-filter, written with the positions: per MM charge its
// position and squared filter radius (the Ewald cutoff or the Gaussian-hat range 9 sigma, with the
// margin of filter_lim2), per QM atom its position.  The filter formed these in FP64 for every
// (atom, charge) pair, an FP64 division among them, which made the real-space sums FP64-bound
// over all pairs rather than over the few within the cutoff.
__global__ void k_filter_prep(EwaldDev e, float4 *mmf, float4 *qmf)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < e.nmm) {
        const double beta = e.mm_beta[t];
        mmf[t] = make_float4((float)e.mm_xyz[3 * t], (float)e.mm_xyz[3 * t + 1], (float)e.mm_xyz[3 * t + 2],
                             filter_lim2(e.ewald_rc, beta > 0.0 ? 9.0 / beta : 0.0));
    } else if (t < e.nmm + e.natm) {
        const int j = t - e.nmm;
        qmf[j] = make_float4((float)e.qm_xyz[3 * j], (float)e.qm_xyz[3 * j + 1], (float)e.qm_xyz[3 * j + 2], 0.0f);
    }
}

// ---------------------------------------------------------------------------------------------
// QM-site potential: real space (psi_SR and the T-hat correction of Eq. 10)
// grid (nslice, natm); partial[(j*nslice + slice)*20 + c]
// ---------------------------------------------------------------------------------------------
// The charges of a slice are scanned 256 at a time with the FP32 filter; the survivors are
// compacted into a shared queue in charge order (warp ballots and a block scan, so the order and
// hence the sums are the same on every run) and evaluated in FP64 by all threads once 256 have
// gathered, so the FP64 pipe runs full warps instead of one or two lanes of each.
constexpr int PR_Q = 512;
__global__ void __launch_bounds__(256) k_phi_real(EwaldDev e, double *partial)
{
    __shared__ double scratch[8 * 20];
    __shared__ int queue[PR_Q];
    __shared__ int wcnt[8];
    const int j = blockIdx.y, nslice = gridDim.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const double Rx = e.qm_xyz[3 * j], Ry = e.qm_xyz[3 * j + 1], Rz = e.qm_xyz[3 * j + 2];
    const float4 aj = e.qm_filt[j];
    const double rc2 = e.ewald_rc * e.ewald_rc;
    const int per = (e.nmm + nslice - 1) / nslice, i0 = blockIdx.x * per, i1 = min(e.nmm, i0 + per);
    double acc[20];
#pragma unroll
    for (int k = 0; k < 20; ++k) acc[k] = 0.0;
    double T[20];
    int count = 0;  // block-uniform
    for (int base = i0; base < i1; base += 256) {
        const int i = base + threadIdx.x;
        bool cand = false;
        if (i < i1) cand = !far_min_image_f(e, aj, __ldg(e.mm_filt + i));
        const unsigned bal = __ballot_sync(0xffffffffu, cand);
        if (lane == 0) wcnt[warp] = __popc(bal);
        __syncthreads();
        int off = count, tot = 0;
        for (int w = 0; w < 8; ++w) {
            if (w < warp) off += wcnt[w];
            tot += wcnt[w];
        }
        if (cand) queue[off + __popc(bal & ((1u << lane) - 1u))] = i;
        count += tot;
        __syncthreads();
        if (count < 256 && base + 256 < i1) continue;
        // FP64 evaluation of the queued charges, entry q by thread q mod 256
        for (int qi = threadIdx.x; qi < count; qi += 256) {
            const int ic = queue[qi];
            const double q = e.mm_q[ic], beta = e.mm_beta[ic];
            const double xi = e.mm_xyz[3 * ic], yi = e.mm_xyz[3 * ic + 1], zi = e.mm_xyz[3 * ic + 2];
            const double dx0 = Rx - xi, dy0 = Ry - yi, dz0 = Rz - zi;
            const double nx0 = rint(dx0 / e.box[0]), ny0 = rint(dy0 / e.box[1]), nz0 = rint(dz0 / e.box[2]);
            const double rhat2 = beta > 0.0 ? (9.0 / beta) * (9.0 / beta) : -1.0;
            for (int a = -e.img[0]; a <= e.img[0]; ++a)
                for (int b = -e.img[1]; b <= e.img[1]; ++b)
                    for (int c = -e.img[2]; c <= e.img[2]; ++c) {
                        const double sx = (nx0 + a) * e.box[0], sy = (ny0 + b) * e.box[1], sz = (nz0 + c) * e.box[2];
                        const double x = dx0 - sx, y = dy0 - sy, z = dz0 - sz;
                        const double r2 = x * x + y * y + z * z;
                        if (r2 < rc2) {
                            double f, g1, g2, g3;
                            screened_radial(r2, e.alpha, f, g1, g2, g3);
                            radial_tensor(f, g1, g2, g3, x, y, z, T, 3);
#pragma unroll
                            for (int k = 0; k < 20; ++k) acc[k] += q * T[k];
                        }
                        if (r2 < rhat2 && !in_region1(e, xi + sx, yi + sy, zi + sz)) {
                            double f, g1, g2, g3;
                            screened_radial(r2, beta, f, g1, g2, g3);
                            radial_tensor(f, g1, g2, g3, x, y, z, T, 3);
#pragma unroll
                            for (int k = 0; k < 20; ++k) acc[k] -= q * T[k];
                        }
                    }
        }
        count = 0;
        __syncthreads();
    }
    block_reduce_store<20>(acc, partial + ((size_t)j * nslice + blockIdx.x) * 20, scratch);
}

// region-I point tensors: grid natm; out[j*20 + c]
__global__ void __launch_bounds__(256) k_phi_region1(EwaldDev e, const double4_32a *rI, int nI, double *out)
{
    __shared__ double scratch[8 * 20];
    const int j = blockIdx.x;
    const double Rx = e.qm_xyz[3 * j], Ry = e.qm_xyz[3 * j + 1], Rz = e.qm_xyz[3 * j + 2];
    double acc[20], T[20];
#pragma unroll
    for (int k = 0; k < 20; ++k) acc[k] = 0.0;
    for (int k = threadIdx.x; k < nI; k += blockDim.x) {
        const double4_32a c = rI[k];
        const double x = Rx - c.x, y = Ry - c.y, z = Rz - c.z;
        double f, g1, g2, g3;
        point_radial(x * x + y * y + z * z, f, g1, g2, g3);
        radial_tensor(f, g1, g2, g3, x, y, z, T, 3);
#pragma unroll
        for (int m = 0; m < 20; ++m) acc[m] -= c.w * T[m];
    }
    block_reduce_store<20>(acc, out + (size_t)j * 20, scratch);
}

// ---------------------------------------------------------------------------------------------
// reciprocal space: structure factor over the dense box nx in [0,kx], ny in [-ky,ky], nz in [-kz,kz]
// ---------------------------------------------------------------------------------------------
constexpr int SF_TILE = 32;  // charges per shared-memory phase tile
constexpr int SF_NZ = 8;     // nz values per thread

__device__ __forceinline__ double2 cmul(double2 a, double2 b)
{
    return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}

// Phase tables e^{i 2 pi n x / L} for n = 0..nmax by repeated multiplication (relative error
// grows by about one rounding per step).
__device__ __forceinline__ void phase_row(double2 *dst, double frac /* x/L */, int nmax, int stride)
{
    double s, c;
    sincospi(2.0 * frac, &s, &c);
    const double2 e1 = make_double2(c, s);
    double2 z = make_double2(1.0, 0.0);
    for (int n = 0; n <= nmax; ++n) {
        dst[n * stride] = z;
        z = cmul(z, e1);
    }
}

// grid (ceil(items/256), nslice); items = NL * NZC; partial[slice][NL][2kz+1]; `tile` charges
// (<= SF_TILE) per shared-memory phase tile
__global__ void __launch_bounds__(256) k_structure_factor(EwaldDev e, double2 *partial, int tile)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int kx = e.kmax[0], ky = e.kmax[1], kz = e.kmax[2];
    const int NX = kx + 1, NY = 2 * ky + 1, NZ = 2 * kz + 1;
    const int NZC = (NZ + SF_NZ - 1) / SF_NZ;
    const int NZP = NZC * SF_NZ;                             // z rows padded with zeros to a multiple of 8
    const int NL = NX * NY;
    double2 *px = reinterpret_cast<double2 *>(smem_raw);   // [tile][NX]
    double2 *py = px + tile * NX;                            // [tile][NY] (index n+ky)
    double2 *pz = py + tile * NY;                            // [tile][NZP]
    const int item = blockIdx.x * blockDim.x + threadIdx.x;
    const bool active = item < NL * NZC;
    // z chunk outermost: the threads of a warp share zc, so their z-phase reads are broadcasts
    const int line = active ? item % NL : 0, zc = active ? item / NL : 0;
    const int nx = line / NY, iy = line % NY, iz0 = zc * SF_NZ;
    double2 acc[SF_NZ];
#pragma unroll
    for (int k = 0; k < SF_NZ; ++k) acc[k] = make_double2(0.0, 0.0);

    const int nslice = gridDim.y;
    const int per = (e.nmm + nslice - 1) / nslice;
    const int i0 = blockIdx.y * per, i1 = min(e.nmm, i0 + per);
    for (int t0 = i0; t0 < i1; t0 += tile) {
        const int nt = min(tile, i1 - t0);
        __syncthreads();
        // 3 * nt rows of phases; negative n from the conjugate of positive n
        for (int r = threadIdx.x; r < 3 * tile; r += blockDim.x) {
            const int c = r / 3, d = r % 3;
            if (c >= nt) continue;
            const double x = e.mm_xyz[3 * (t0 + c) + d] / e.box[d];
            if (d == 0) {
                phase_row(px + c * NX, x, kx, 1);
                const double q = e.mm_q[t0 + c];
                for (int n = 0; n < NX; ++n) px[c * NX + n] = make_double2(q * px[c * NX + n].x, q * px[c * NX + n].y);
            } else if (d == 1) {
                phase_row(py + c * NY + ky, x, ky, 1);
                for (int n = 1; n <= ky; ++n) {
                    const double2 v = py[c * NY + ky + n];
                    py[c * NY + ky - n] = make_double2(v.x, -v.y);
                }
            } else {
                phase_row(pz + c * NZP + kz, x, kz, 1);
                for (int n = 1; n <= kz; ++n) {
                    const double2 v = pz[c * NZP + kz + n];
                    pz[c * NZP + kz - n] = make_double2(v.x, -v.y);
                }
                for (int n = NZ; n < NZP; ++n) pz[c * NZP + n] = make_double2(0.0, 0.0);
            }
        }
        __syncthreads();
        if (active) {
            for (int c = 0; c < nt; ++c) {
                const double2 a = cmul(px[c * NX + nx], py[c * NY + iy]);
                const double nay = -a.y;
                const double2 *zr = pz + c * NZP + iz0;
#pragma unroll
                for (int k = 0; k < SF_NZ; ++k) {
                    const double2 b = zr[k];  // rows are padded by SF_NZ - 1 entries
                    acc[k].x = fma(a.x, b.x, fma(nay, b.y, acc[k].x));
                    acc[k].y = fma(a.x, b.y, fma(a.y, b.x, acc[k].y));
                }
            }
        }
    }
    if (active) {
        double2 *dst = partial + ((size_t)blockIdx.y * NL + line) * NZ;
#pragma unroll
        for (int k = 0; k < SF_NZ; ++k)
            if (iz0 + k < NZ) dst[iz0 + k] = acc[k];
    }
}

// Double-float variant (mixed-precision path): the same tiling, with phases and the eight
// accumulators as FP32 (hi, lo) pairs -- each (G, charge) term is an error-free complex
// multiply-add of about 48 FP32 operations instead of 4 FP64 FMAs (~47-bit accuracy per term).
__device__ __forceinline__ void phase_row_df(float4 *dst, double frac, int nmax, double scale)
{
    // start and step in FP64 (one sincospi), the recurrence itself in double-float arithmetic
    double s, c;
    sincospi(2.0 * frac, &s, &c);
    const c2 e1{f2_from(c), f2_from(s)};
    c2 z{f2_from(scale), f2{0.f, 0.f}};
    for (int n = 0; n <= nmax; ++n) {
        dst[n] = make_float4(z.re.h, z.re.l, z.im.h, z.im.l);
        z = c2_mul(z, e1);
    }
}

__global__ void __launch_bounds__(256, 3) k_structure_factor_df(EwaldDev e, double2 *partial, int tile)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int kx = e.kmax[0], ky = e.kmax[1], kz = e.kmax[2];
    const int NX = kx + 1, NY = 2 * ky + 1, NZ = 2 * kz + 1;
    const int NZC = (NZ + SF_NZ - 1) / SF_NZ;
    const int NZP = NZC * SF_NZ;
    const int NL = NX * NY;
    float4 *px = reinterpret_cast<float4 *>(smem_raw);  // [tile][NX]
    float4 *py = px + tile * NX;                          // [tile][NY]
    float4 *pz = py + tile * NY;                          // [tile][NZP]
    const int item = blockIdx.x * blockDim.x + threadIdx.x;
    const bool active = item < NL * NZC;
    // z chunk outermost: the threads of a warp share zc, so their z-phase reads are broadcasts
    const int line = active ? item % NL : 0, zc = active ? item / NL : 0;
    const int nx = line / NY, iy = line % NY, iz0 = zc * SF_NZ;
    float acc[SF_NZ][4];
#pragma unroll
    for (int k = 0; k < SF_NZ; ++k) acc[k][0] = acc[k][1] = acc[k][2] = acc[k][3] = 0.0f;

    const int nslice = gridDim.y;
    const int per = (e.nmm + nslice - 1) / nslice;
    const int i0 = blockIdx.y * per, i1 = min(e.nmm, i0 + per);
    for (int t0 = i0; t0 < i1; t0 += tile) {
        const int nt = min(tile, i1 - t0);
        __syncthreads();
        for (int r = threadIdx.x; r < 3 * tile; r += blockDim.x) {
            const int c = r / 3, d = r % 3;
            if (c >= nt) continue;
            const double x = e.mm_xyz[3 * (t0 + c) + d] / e.box[d];
            if (d == 0) {
                phase_row_df(px + c * NX, x, kx, e.mm_q[t0 + c]);
            } else if (d == 1) {
                phase_row_df(py + c * NY + ky, x, ky, 1.0);
                for (int n = 1; n <= ky; ++n) {
                    const float4 v = py[c * NY + ky + n];
                    py[c * NY + ky - n] = make_float4(v.x, v.y, -v.z, -v.w);
                }
            } else {
                phase_row_df(pz + c * NZP + kz, x, kz, 1.0);
                for (int n = 1; n <= kz; ++n) {
                    const float4 v = pz[c * NZP + kz + n];
                    pz[c * NZP + kz - n] = make_float4(v.x, v.y, -v.z, -v.w);
                }
                for (int n = NZ; n < NZP; ++n) pz[c * NZP + n] = make_float4(0.f, 0.f, 0.f, 0.f);
            }
        }
        __syncthreads();
        if (active) {
            for (int c = 0; c < nt; ++c) {
                const c2 a = c2_mul(c2_from(px[c * NX + nx]), c2_from(py[c * NY + iy]));
                const float4 *zr = pz + c * NZP + iz0;
#pragma unroll
                for (int k = 0; k < SF_NZ; ++k) c2_mac(acc[k], a, c2_from(zr[k]));
            }
        }
    }
    if (active) {
        double2 *dst = partial + ((size_t)blockIdx.y * NL + line) * NZ;
#pragma unroll
        for (int k = 0; k < SF_NZ; ++k)
            if (iz0 + k < NZ) dst[iz0 + k] = make_double2(f2_to(acc[k][0], acc[k][1]), f2_to(acc[k][2], acc[k][3]));
    }
}

__global__ void k_sum_slices(const double2 *partial, int nslice, int n, double2 *out)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    double2 s = make_double2(0.0, 0.0);
    for (int sl = 0; sl < nslice; ++sl) {
        const double2 v = partial[(size_t)sl * n + k];
        s.x += v.x; s.y += v.y;
    }
    out[k] = s;
}

// reciprocal factor of a dense index: 2 g(G) on the half space (n_x > 0, or n_x = 0 and
// (n_y > 0 or (n_y = 0 and n_z > 0))), zero elsewhere; written at plan time.
__global__ void k_gfac(EwaldDev e, double *gfac)
{
    const int kx = e.kmax[0], ky = e.kmax[1], kz = e.kmax[2];
    const int NY = 2 * ky + 1, NZ = 2 * kz + 1, n = (kx + 1) * NY * NZ;
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int nx = k / (NY * NZ), ny = (k / NZ) % NY - ky, nz = k % NZ - kz;
    const bool half = nx > 0 || (nx == 0 && (ny > 0 || (ny == 0 && nz > 0)));
    if (!half) { gfac[k] = 0.0; return; }
    const double V = e.box[0] * e.box[1] * e.box[2];
    const double Gx = TWO_PI * nx / e.box[0], Gy = TWO_PI * ny / e.box[1], Gz = TWO_PI * nz / e.box[2];
    const double G2 = Gx * Gx + Gy * Gy + Gz * Gz;
    gfac[k] = 2.0 * 4.0 * PI / V * exp(-G2 / (4.0 * e.alpha * e.alpha)) / G2;
}

// QM-site reciprocal part: grid (natm, nslice); block (j, sl) sums the dense entries of slice sl
// for QM atom j into part[(j nslice + sl) 20 + c].  The phase exp(iG.R_j) = X(n_x) Y(n_y) Z(n_z)
// comes from the atom's three phase rows in shared memory (one sincospi per entry), so a
// (G, atom) term costs two complex multiplies instead of a sincos.
constexpr int PHR_MAXN = 2 * 56 + 1;
__global__ void __launch_bounds__(256) k_phi_recip(EwaldDev e, const double2 *S, const double *gfac, double *part)
{
    __shared__ double scratch[8 * 20];
    __shared__ double2 ph[3][PHR_MAXN];
    const int j = blockIdx.x, sl = blockIdx.y, ns = gridDim.y;
    const int kx = e.kmax[0], ky = e.kmax[1], kz = e.kmax[2];
    const int NY = 2 * ky + 1, NZ = 2 * kz + 1, n = (kx + 1) * NY * NZ;
    // rows: X(n_x) n_x = 0..kx; Y(n_y), Z(n_z) indexed n + k
    for (int t = threadIdx.x; t < (kx + 1) + NY + NZ; t += blockDim.x) {
        const int d = t <= kx ? 0 : t <= kx + NY ? 1 : 2;
        const int idx = d == 0 ? t : d == 1 ? t - (kx + 1) : t - (kx + 1) - NY;
        const int nn = d == 0 ? idx : idx - e.kmax[d];
        double sn, cs;
        sincospi(2.0 * nn * (e.qm_xyz[3 * j + d] / e.box[d]), &sn, &cs);
        ph[d][idx] = make_double2(cs, sn);
    }
    __syncthreads();
    const int per = (n + ns - 1) / ns, k0 = sl * per, k1 = min(n, k0 + per);
    double acc[20];
#pragma unroll
    for (int k = 0; k < 20; ++k) acc[k] = 0.0;
    for (int k = k0 + threadIdx.x; k < k1; k += blockDim.x) {
        const double g = gfac[k];
        if (g == 0.0) continue;
        const int nx = k / (NY * NZ), iy = (k / NZ) % NY, iz = k % NZ;
        const double Gx = TWO_PI * nx / e.box[0], Gy = TWO_PI * (iy - ky) / e.box[1],
                     Gz = TWO_PI * (iz - kz) / e.box[2];
        const double2 p = cmul(cmul(ph[0][nx], ph[1][iy]), ph[2][iz]);
        const double c = p.x, s = p.y;
        const double2 Sk = S[k];
        // exp(i G.R_j) conj(S)
        const double re = g * (c * Sk.x + s * Sk.y);
        const double im = g * (s * Sk.x - c * Sk.y);
        const double G[3] = {Gx, Gy, Gz};
        acc[0] += re;
        acc[1] -= Gx * im; acc[2] -= Gy * im; acc[3] -= Gz * im;
        acc[4] -= 0.5 * Gx * Gx * re; acc[5] -= 0.5 * Gx * Gy * re; acc[6] -= 0.5 * Gx * Gz * re;
        acc[7] -= 0.5 * Gy * Gy * re; acc[8] -= 0.5 * Gy * Gz * re; acc[9] -= 0.5 * Gz * Gz * re;
        const double s6 = im / 6.0;
        acc[10] += s6 * G[0] * G[0] * G[0]; acc[11] += s6 * G[0] * G[0] * G[1]; acc[12] += s6 * G[0] * G[0] * G[2];
        acc[13] += s6 * G[0] * G[1] * G[1]; acc[14] += s6 * G[0] * G[1] * G[2]; acc[15] += s6 * G[0] * G[2] * G[2];
        acc[16] += s6 * G[1] * G[1] * G[1]; acc[17] += s6 * G[1] * G[1] * G[2]; acc[18] += s6 * G[1] * G[2] * G[2];
        acc[19] += s6 * G[2] * G[2] * G[2];
    }
    block_reduce_store<20>(acc, part + ((size_t)j * ns + sl) * 20, scratch);
}

// Mixed path: the reciprocal factor times S(G) as double-float (re.h, re.l, im.h, im.l), once per
// call for all QM atoms
__global__ void k_gs_df(int n, const double2 *S, const double *gfac, float4 *gS)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const double g = gfac[k];
    const double2 v = S[k];
    gS[k] = c2_pack(g * v.x, g * v.y);
}

// k_phi_recip in double-float arithmetic on the FP32 pipes (mixed path): the same terms, about 44
// significant bits per operation (the region-II potential stays within 1e-10 of the FP64 one),
// where the FP64 kernel spent about 60 FP64 instructions per (G, atom) on an FP64 pipe that
// executes 2 of them per clock and SM.
__global__ void __launch_bounds__(256) k_phi_recip_df(EwaldDev e, const float4 *gS, double *part)
{
    __shared__ double scratch[8 * 20];
    __shared__ float4 ph[3][PHR_MAXN];
    const int j = blockIdx.x, sl = blockIdx.y, ns = gridDim.y;
    const int kx = e.kmax[0], ky = e.kmax[1], kz = e.kmax[2];
    const int NY = 2 * ky + 1, NZ = 2 * kz + 1, n = (kx + 1) * NY * NZ;
    for (int t = threadIdx.x; t < (kx + 1) + NY + NZ; t += blockDim.x) {
        const int d = t <= kx ? 0 : t <= kx + NY ? 1 : 2;
        const int idx = d == 0 ? t : d == 1 ? t - (kx + 1) : t - (kx + 1) - NY;
        const int nn = d == 0 ? idx : idx - e.kmax[d];
        double sn, cs;
        sincospi(2.0 * nn * (e.qm_xyz[3 * j + d] / e.box[d]), &sn, &cs);
        ph[d][idx] = c2_pack(cs, sn);
    }
    __syncthreads();
    const f2 g1[3] = {f2_from(TWO_PI / e.box[0]), f2_from(TWO_PI / e.box[1]), f2_from(TWO_PI / e.box[2])};
    const f2 sixth = f2_from(1.0 / 6.0);
    const int per = (n + ns - 1) / ns, k0 = sl * per, k1 = min(n, k0 + per);
    float ah[20], al[20];
#pragma unroll
    for (int c = 0; c < 20; ++c) ah[c] = al[c] = 0.0f;
    const f2 one{1.0f, 0.0f};
    for (int k = k0 + threadIdx.x; k < k1; k += blockDim.x) {
        const float4 w = gS[k];
        if (w.x == 0.0f && w.z == 0.0f) continue;  // outside the half space (g = 0), or S = 0
        const int nx = k / (NY * NZ), iy = (k / NZ) % NY, iz = k % NZ;
        const c2 p = c2_mul(c2_mul(c2_from(ph[0][nx]), c2_from(ph[1][iy])), c2_from(ph[2][iz]));
        const c2 q = c2_from(w);
        // exp(i G.R_j) conj(g S): re = c Sr + s Si, im = s Sr - c Si
        const f2 re = f2_add(f2_mul(p.re, q.re), f2_mul(p.im, q.im));
        const f2 im = f2_add(f2_mul(p.im, q.re), f2_neg(f2_mul(p.re, q.im)));
        const f2 G[3] = {f2_mul(g1[0], f2{(float)nx, 0.0f}), f2_mul(g1[1], f2{(float)(iy - ky), 0.0f}),
                         f2_mul(g1[2], f2{(float)(iz - kz), 0.0f})};
        f2_mac(ah[0], al[0], re, one);
        const f2 mim = f2_neg(im), mhre{-0.5f * re.h, -0.5f * re.l};
        f2 t6[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            f2_mac(ah[1 + a], al[1 + a], G[a], mim);
            t6[a] = f2_mul(f2_mul(G[a], im), sixth);
        }
        // u_ab = G_a G_b in the order xx xy xz yy yz zz
        const f2 u[6] = {f2_mul(G[0], G[0]), f2_mul(G[0], G[1]), f2_mul(G[0], G[2]),
                         f2_mul(G[1], G[1]), f2_mul(G[1], G[2]), f2_mul(G[2], G[2])};
#pragma unroll
        for (int c = 0; c < 6; ++c) f2_mac(ah[4 + c], al[4 + c], u[c], mhre);
        // xxx xxy xxz xyy xyz xzz yyy yyz yzz zzz = u_ab t_c / 6
        f2_mac(ah[10], al[10], u[0], t6[0]);
        f2_mac(ah[11], al[11], u[0], t6[1]);
        f2_mac(ah[12], al[12], u[0], t6[2]);
        f2_mac(ah[13], al[13], u[1], t6[1]);
        f2_mac(ah[14], al[14], u[1], t6[2]);
        f2_mac(ah[15], al[15], u[2], t6[2]);
        f2_mac(ah[16], al[16], u[3], t6[1]);
        f2_mac(ah[17], al[17], u[3], t6[2]);
        f2_mac(ah[18], al[18], u[4], t6[2]);
        f2_mac(ah[19], al[19], u[5], t6[2]);
    }
    double acc[20];
#pragma unroll
    for (int c = 0; c < 20; ++c) acc[c] = f2_to(ah[c], al[c]);
    block_reduce_store<20>(acc, part + ((size_t)j * ns + sl) * 20, scratch);
}

// G slices per QM atom of the reciprocal part: two blocks per SM in all
int ewald_recip_nslice(const EwaldDev &e, int nsm)
{
    int ns = (2 * nsm + e.natm - 1) / (e.natm > 0 ? e.natm : 1);
    const int n = ewald_dense_size(e);
    if (ns > (n + 1023) / 1024) ns = (n + 1023) / 1024;
    if (ns < 1) ns = 1;
    return ns;
}

int ewald_dense_size(const EwaldDev &e)
{
    return (e.kmax[0] + 1) * (2 * e.kmax[1] + 1) * (2 * e.kmax[2] + 1);
}
static int sf_items(const EwaldDev &e)
{
    const int NZ = 2 * e.kmax[2] + 1;
    return (e.kmax[0] + 1) * (2 * e.kmax[1] + 1) * ((NZ + SF_NZ - 1) / SF_NZ);
}
// shared memory of one structure-factor block and its phase-tile depth
static size_t sf_smem(const EwaldDev &e, int *tile_out)
{
    const int NX = e.kmax[0] + 1, NY = 2 * e.kmax[1] + 1, NZ = 2 * e.kmax[2] + 1;
    const int NZP = (NZ + SF_NZ - 1) / SF_NZ * SF_NZ;
    const size_t row = (size_t)(NX + NY + NZP) * sizeof(double2);
    int tile = (int)std::min<size_t>(SF_TILE, (200u * 1024u) / row);
    if (tile < 1) tile = 1;
    if (tile_out) *tile_out = tile;
    return (size_t)tile * row;
}

// Charge slices of the structure factor: the grid (line blocks x slices) is sized to one full
// wave of resident blocks, so no partial last wave leaves most SMs idle.
int ewald_sf_nslice(const EwaldDev &e, int nsm, bool df)
{
    const size_t smem = sf_smem(e, nullptr);
    const void *fn = df ? (const void *)k_structure_factor_df : (const void *)k_structure_factor;
    if (smem > 48 * 1024) cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int per_sm = 1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, 256, smem) != cudaSuccess || per_sm < 1) {
        cudaGetLastError();
        per_sm = 1;
    }
    const int bx = (sf_items(e) + 255) / 256;
    int ns = (nsm * per_sm) / bx;
    if (ns > 256) ns = 256;
    if (ns > e.nmm / SF_TILE + 1) ns = e.nmm / SF_TILE + 1;
    if (ns < 1) ns = 1;
    return ns;
}
int ewald_real_nslice(const EwaldDev &e, int nsm)
{
    int ns = (2 * nsm + e.natm - 1) / (e.natm > 0 ? e.natm : 1);
    if (ns > (e.nmm + 255) / 256) ns = (e.nmm + 255) / 256;
    if (ns < 1) ns = 1;
    return ns;
}
cudaError_t launch_gfac(const EwaldDev &e, double *gfac, cudaStream_t st)
{
    const int n = ewald_dense_size(e);
    k_gfac<<<(n + 255) / 256, 256, 0, st>>>(e, gfac);
    return cudaGetLastError();
}

__global__ void k_sum1(const double *x, int n, int stride, double *out)
{
    __shared__ double ws[32];
    double s = 0.0;
    for (int k = threadIdx.x; k < n; k += blockDim.x) s += x[(size_t)k * stride];
    s = warp_sum(s);
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += ws[w];
        out[0] = t;
    }
}
cudaError_t launch_sum(const double *x, int n, double *out, cudaStream_t st)
{
    k_sum1<<<1, 1024, 0, st>>>(x, n, 1, out);
    return cudaGetLastError();
}
cudaError_t launch_sum_strided(const double *x, int n, int stride, double *out, cudaStream_t st)
{
    k_sum1<<<1, 1024, 0, st>>>(x, n, stride, out);
    return cudaGetLastError();
}

__global__ void k_phi_final(EwaldDev e, const double *precip, int rslice, const double *preal, int nslice,
                            const double *pr1, const double *sums, double *phi)
{
    const int j = blockIdx.x, k = threadIdx.x;
    if (k >= 20) return;
    double v = 0.0;
    for (int sl = 0; sl < rslice; ++sl) v += precip[((size_t)j * rslice + sl) * 20 + k];
    for (int sl = 0; sl < nslice; ++sl) v += preal[((size_t)j * nslice + sl) * 20 + k];
    v += pr1[(size_t)j * 20 + k];
    if (k == 0) v += -PI / (e.box[0] * e.box[1] * e.box[2] * e.alpha * e.alpha) * sums[0];
    phi[(size_t)j * 20 + k] = v;
}

cudaError_t launch_ewald_phi(const EwaldDev &e, const double4_32a *rI, int nI, const EwaldBuf &w, double *phi,
                             bool df, cudaStream_t st)
{
    cudaError_t err;
    // FP32 inputs of the real-space pre-filters (here and in the forces' MM-side sum)
    if (e.nmm + e.natm > 0) {
        k_filter_prep<<<(e.nmm + e.natm + 255) / 256, 256, 0, st>>>(e, w.mm_filt, w.qm_filt);
        if ((err = cudaGetLastError()) != cudaSuccess) return err;
    }
    // sum of MM charges (background)
    if ((err = launch_sum(e.mm_q, e.nmm, w.sums, st)) != cudaSuccess) return err;
    // real space
    {
        dim3 grid(w.real_nslice, e.natm);
        k_phi_real<<<grid, 256, 0, st>>>(e, w.preal);
        if ((err = cudaGetLastError()) != cudaSuccess) return err;
    }
    k_phi_region1<<<e.natm, 256, 0, st>>>(e, rI, nI, w.pr1);
    if ((err = cudaGetLastError()) != cudaSuccess) return err;
    // structure factor
    if (w.recip == 1) {
        if ((err = launch_structure_factor_tc(e, w.tcs, w.tcb, w.S, w.err, st)) != cudaSuccess) return err;
    } else {
        int tile = 1;
        const size_t smem = sf_smem(e, &tile);
        static size_t attr = 0, attr_df = 0;
        size_t &a = df ? attr_df : attr;
        if (smem > 48 * 1024 && smem > a) {
            if ((err = cudaFuncSetAttribute(df ? (const void *)k_structure_factor_df : (const void *)k_structure_factor,
                                            cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess)
                return err;
            a = smem;
        }
        const int nslice = df ? w.sf_nslice_df : w.sf_nslice;
        dim3 grid((sf_items(e) + 255) / 256, nslice);
        if (df)
            k_structure_factor_df<<<grid, 256, smem, st>>>(e, w.Spart, tile);
        else
            k_structure_factor<<<grid, 256, smem, st>>>(e, w.Spart, tile);
        if ((err = cudaGetLastError()) != cudaSuccess) return err;
        const int n = ewald_dense_size(e);
        k_sum_slices<<<(n + 255) / 256, 256, 0, st>>>(w.Spart, nslice, n, w.S);
        if ((err = cudaGetLastError()) != cudaSuccess) return err;
    }
    // reciprocal part at the QM sites (G slices), then the final combination in a fixed order
    if (df && w.gSdf) {
        const int n = ewald_dense_size(e);
        k_gs_df<<<(n + 255) / 256, 256, 0, st>>>(n, w.S, w.gfac, w.gSdf);
        if ((err = cudaGetLastError()) != cudaSuccess) return err;
        k_phi_recip_df<<<dim3(e.natm, w.recip_nslice), 256, 0, st>>>(e, w.gSdf, w.precip);
    } else {
        k_phi_recip<<<dim3(e.natm, w.recip_nslice), 256, 0, st>>>(e, w.S, w.gfac, w.precip);
    }
    if ((err = cudaGetLastError()) != cudaSuccess) return err;
    k_phi_final<<<e.natm, 32, 0, st>>>(e, w.precip, w.recip_nslice, w.preal, w.real_nslice, w.pr1, w.sums, phi);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------------
// MM-side adjoint
// ---------------------------------------------------------------------------------------------
// contraction helpers: potential sum_c w_c M_c T_c and field d/dR_j of it
__device__ __forceinline__ void contract_pot_field(const double *M, const double *T, double &pot, double (&fld)[3])
{
    pot = M[0] * T[0] + M[1] * T[1] + M[2] * T[2] + M[3] * T[3] + M[4] * T[4] + 2.0 * M[5] * T[5] +
          2.0 * M[6] * T[6] + M[7] * T[7] + 2.0 * M[8] * T[8] + M[9] * T[9];
    // d_x T_0 = T_x; d_x T_a = 2 T_ax; d_x T_ab = 3 T_abx   (index tables of the symmetric tensors)
    const int I2[3][3] = {{4, 5, 6}, {5, 7, 8}, {6, 8, 9}};
    const int I3[3][3][3] = {{{10, 11, 12}, {11, 13, 14}, {12, 14, 15}},
                             {{11, 13, 14}, {13, 16, 17}, {14, 17, 18}},
                             {{12, 14, 15}, {14, 17, 18}, {15, 18, 19}}};
    const int P2[6][2] = {{0, 0}, {0, 1}, {0, 2}, {1, 1}, {1, 2}, {2, 2}};
#pragma unroll
    for (int x = 0; x < 3; ++x) {
        double g = M[0] * T[1 + x];
#pragma unroll
        for (int a = 0; a < 3; ++a) g += 2.0 * M[1 + a] * T[I2[a][x]];
#pragma unroll
        for (int k = 0; k < 6; ++k) g += 3.0 * w10(4 + k) * M[4 + k] * T[I3[P2[k][0]][P2[k][1]][x]];
        fld[x] = g;
    }
}

// Blocks of 32 MM charges (one per lane) x 8 warps; warp w takes the QM atoms j = w, w + 8, ...
// and the 8 partial sums per charge are added in a fixed order (as in the nuclear-MM kernel), so
// small N_MM still fills the GPU and the result is reproducible.
constexpr int MMQ_CH = 32, MMQ_WARPS = 8;

// per-charge reduction over the 8 warps: red[4][8][32]; returns the sums in lane order on warp 0
__device__ __forceinline__ void mmq_reduce(double (&red)[4][MMQ_WARPS][MMQ_CH], double pot, const double (&fld)[3],
                                           double (&out)[4])
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    red[0][warp][lane] = pot;
    red[1][warp][lane] = fld[0];
    red[2][warp][lane] = fld[1];
    red[3][warp][lane] = fld[2];
    __syncthreads();
    out[0] = out[1] = out[2] = out[3] = 0.0;
    if (warp == 0)
        for (int w = 0; w < MMQ_WARPS; ++w)
#pragma unroll
            for (int v = 0; v < 4; ++v) out[v] += red[v][w][lane];
}

// Blocks of 32 MM charges.  The (charge, QM atom) pairs of a block are scanned 256 at a time with
// the FP32 filter and the survivors compacted in pair order (charge-major) into a shared queue;
// all threads then evaluate the queued pairs in FP64, and each charge's owner thread adds its
// pairs' contributions in queue order (the same order on every run).
constexpr int MR_Q = 1024;
__global__ void __launch_bounds__(256) k_mm_real(EwaldDev e, const double *mult, double *dq, double *dR)
{
    __shared__ int queue[MR_Q];
    __shared__ double contrib[MR_Q][4];
    __shared__ int wcnt[8];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int c0 = blockIdx.x * MMQ_CH, nch = min(MMQ_CH, e.nmm - c0), natm = e.natm;
    const int npairs = nch * natm;
    const double rc2 = e.ewald_rc * e.ewald_rc;
    double sum[4] = {0.0, 0.0, 0.0, 0.0};  // charge threadIdx.x (< nch)
    double T[20];
    int count = 0;  // block-uniform
    for (int base = 0; base < npairs; base += 256) {
        const int t = base + threadIdx.x;
        bool cand = false;
        if (t < npairs) {
            const int il = t / natm, j = t - il * natm;
            cand = !far_min_image_f(e, __ldg(e.qm_filt + j), __ldg(e.mm_filt + c0 + il));
        }
        const unsigned bal = __ballot_sync(0xffffffffu, cand);
        if (lane == 0) wcnt[warp] = __popc(bal);
        __syncthreads();
        int off = count, tot = 0;
        for (int w = 0; w < 8; ++w) {
            if (w < warp) off += wcnt[w];
            tot += wcnt[w];
        }
        if (cand) queue[off + __popc(bal & ((1u << lane) - 1u))] = t;
        count += tot;
        __syncthreads();
        if (count <= MR_Q - 256 && base + 256 < npairs) continue;
        for (int qi = threadIdx.x; qi < count; qi += 256) {
            const int tq = queue[qi], il = tq / natm, j = tq - il * natm, i = c0 + il;
            const double beta = e.mm_beta[i];
            const double xi = e.mm_xyz[3 * i], yi = e.mm_xyz[3 * i + 1], zi = e.mm_xyz[3 * i + 2];
            const double rhat2 = beta > 0.0 ? (9.0 / beta) * (9.0 / beta) : -1.0;
            const double dx0 = __ldg(e.qm_xyz + 3 * j) - xi, dy0 = __ldg(e.qm_xyz + 3 * j + 1) - yi,
                         dz0 = __ldg(e.qm_xyz + 3 * j + 2) - zi;
            const double nx0 = rint(dx0 / e.box[0]), ny0 = rint(dy0 / e.box[1]), nz0 = rint(dz0 / e.box[2]);
            double pot = 0.0, fld[3] = {0.0, 0.0, 0.0};
            for (int a = -e.img[0]; a <= e.img[0]; ++a)
                for (int b = -e.img[1]; b <= e.img[1]; ++b)
                    for (int c = -e.img[2]; c <= e.img[2]; ++c) {
                        const double sx = (nx0 + a) * e.box[0], sy = (ny0 + b) * e.box[1], sz = (nz0 + c) * e.box[2];
                        const double x = dx0 - sx, y = dy0 - sy, z = dz0 - sz;
                        const double r2 = x * x + y * y + z * z;
                        const bool sr = r2 < rc2;
                        const bool hat = r2 < rhat2 && !in_region1(e, xi + sx, yi + sy, zi + sz);
                        if (!sr && !hat) continue;
                        double Mj[10];
#pragma unroll
                        for (int k = 0; k < 10; ++k) Mj[k] = __ldg(mult + 10 * j + k);
                        double f, g1, g2, g3, p, fl[3];
                        if (sr) {
                            screened_radial(r2, e.alpha, f, g1, g2, g3);
                            radial_tensor(f, g1, g2, g3, x, y, z, T, 3);
                            contract_pot_field(Mj, T, p, fl);
                            pot += p; fld[0] += fl[0]; fld[1] += fl[1]; fld[2] += fl[2];
                        }
                        if (hat) {
                            screened_radial(r2, beta, f, g1, g2, g3);
                            radial_tensor(f, g1, g2, g3, x, y, z, T, 3);
                            contract_pot_field(Mj, T, p, fl);
                            pot -= p; fld[0] -= fl[0]; fld[1] -= fl[1]; fld[2] -= fl[2];
                        }
                    }
            contrib[qi][0] = pot;
            contrib[qi][1] = fld[0];
            contrib[qi][2] = fld[1];
            contrib[qi][3] = fld[2];
        }
        __syncthreads();
        if (threadIdx.x < nch)
            for (int qi = 0; qi < count; ++qi)
                if (queue[qi] / natm == (int)threadIdx.x)
#pragma unroll
                    for (int v = 0; v < 4; ++v) sum[v] += contrib[qi][v];
        count = 0;
        __syncthreads();
    }
    if (threadIdx.x < nch) {
        const int i = c0 + threadIdx.x;
        const double q = e.mm_q[i];
        dq[i] += sum[0];
        dR[3 * i] += -q * sum[1];
        dR[3 * i + 1] += -q * sum[2];
        dR[3 * i + 2] += -q * sum[3];
    }
}

// minus the point tensors over region I, per region-I image (gchg += : [dC_x, dC_y, dC_z, dq])
__global__ void __launch_bounds__(MMQ_CH *MMQ_WARPS) k_mm_region1(EwaldDev e, const double4_32a *rI, int nI,
                                                                   const double *mult, double *gchg)
{
    __shared__ double red[4][MMQ_WARPS][MMQ_CH];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int k = blockIdx.x * MMQ_CH + lane;
    const bool act = k < nI;
    double4_32a c;
    c.x = c.y = c.z = c.w = 0.0;
    if (act) c = rI[k];
    double pot = 0.0, fld[3] = {0.0, 0.0, 0.0}, T[20];
    for (int j = warp; act && j < e.natm; j += MMQ_WARPS) {
        const double x = __ldg(e.qm_xyz + 3 * j) - c.x, y = __ldg(e.qm_xyz + 3 * j + 1) - c.y,
                     z = __ldg(e.qm_xyz + 3 * j + 2) - c.z;
        double f, g1, g2, g3, p, fl[3], Mj[10];
#pragma unroll
        for (int m = 0; m < 10; ++m) Mj[m] = __ldg(mult + 10 * j + m);
        point_radial(x * x + y * y + z * z, f, g1, g2, g3);
        radial_tensor(f, g1, g2, g3, x, y, z, T, 3);
        contract_pot_field(Mj, T, p, fl);
        pot += p; fld[0] += fl[0]; fld[1] += fl[1]; fld[2] += fl[2];
    }
    double t[4];
    mmq_reduce(red, pot, fld, t);
    if (warp == 0 && act) {  // atomics: the region-I adjoint sweep may add to gchg at the same time
        atomicAdd(gchg + 4 * (size_t)k + 0, c.w * t[1]);
        atomicAdd(gchg + 4 * (size_t)k + 1, c.w * t[2]);
        atomicAdd(gchg + 4 * (size_t)k + 2, c.w * t[3]);
        atomicAdd(gchg + 4 * (size_t)k + 3, -t[0]);
    }
}

// Phase rows of the QM atoms: ph[(j 3 + d) PHR_MAXN + idx] = exp(2 pi i n u_jd), idx = n for
// d = 0 (n = 0..kx) and n + k_d for d = 1, 2 (n = -k_d..k_d); one sincospi per entry
__global__ void k_atom_phases(EwaldDev e, double2 *ph, float4 *phdf)
{
    const int j = blockIdx.x;
    const int kx = e.kmax[0], NY = 2 * e.kmax[1] + 1, NZ = 2 * e.kmax[2] + 1;
    for (int t = threadIdx.x; t < (kx + 1) + NY + NZ; t += blockDim.x) {
        const int d = t <= kx ? 0 : t <= kx + NY ? 1 : 2;
        const int idx = d == 0 ? t : d == 1 ? t - (kx + 1) : t - (kx + 1) - NY;
        const int nn = d == 0 ? idx : idx - e.kmax[d];
        double sn, cs;
        sincospi(2.0 * nn * (e.qm_xyz[3 * j + d] / e.box[d]), &sn, &cs);
        ph[((size_t)j * 3 + d) * PHR_MAXN + idx] = make_double2(cs, sn);
        if (phdf) phdf[((size_t)j * 3 + d) * PHR_MAXN + idx] = c2_pack(cs, sn);  // mixed path
    }
}

// A(G) = 2 g(G) sum_j exp(i G.R_j) (Q_j + i G.mu_j - 1/2 G.theta_j.G) on the dense box, and
// Az(G) = G_z A(G) (the z-field channel of the MM-side sum); exp(i G.R_j) from the atom's phase
// rows (two complex multiplies)
__global__ void __launch_bounds__(256) k_multipole_sf(EwaldDev e, const double *gfac, const double *mult,
                                                      const double2 *ph, double2 *A, double2 *Az, float4 *Adf,
                                                      float4 *Azdf)
{
    const int kx = e.kmax[0], ky = e.kmax[1], kz = e.kmax[2];
    const int NY = 2 * ky + 1, NZ = 2 * kz + 1, n = (kx + 1) * NY * NZ;
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const double g = gfac[k];
    if (g == 0.0) {
        A[k] = make_double2(0.0, 0.0);
        Az[k] = make_double2(0.0, 0.0);
        if (Adf) {
            Adf[k] = make_float4(0.f, 0.f, 0.f, 0.f);
            Azdf[k] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
        return;
    }
    const int nx = k / (NY * NZ), ny = (k / NZ) % NY - ky, nz = k % NZ - kz;
    const double Gx = TWO_PI * nx / e.box[0], Gy = TWO_PI * ny / e.box[1], Gz = TWO_PI * nz / e.box[2];
    double re = 0.0, im = 0.0;
    for (int j = 0; j < e.natm; ++j) {
        const double *M = mult + 10 * j;
        const double mr = M[0] - 0.5 * (M[4] * Gx * Gx + 2.0 * M[5] * Gx * Gy + 2.0 * M[6] * Gx * Gz + M[7] * Gy * Gy +
                                        2.0 * M[8] * Gy * Gz + M[9] * Gz * Gz);
        const double mi = Gx * M[1] + Gy * M[2] + Gz * M[3];
        const double2 *pj = ph + (size_t)j * 3 * PHR_MAXN;
        const double2 p = cmul(cmul(__ldg(pj + nx), __ldg(pj + PHR_MAXN + ny + ky)), __ldg(pj + 2 * PHR_MAXN + nz + kz));
        const double s = p.y, c = p.x;
        re += c * mr - s * mi;
        im += s * mr + c * mi;
    }
    A[k] = make_double2(g * re, g * im);
    Az[k] = make_double2(Gz * g * re, Gz * g * im);
    if (Adf) {
        Adf[k] = c2_pack(g * re, g * im);
        Azdf[k] = c2_pack(Gz * g * re, Gz * g * im);
    }
}

// Mixed path: A(G) and Az(G) as k_multipole_sf, the sum over the QM atoms in double-float
// arithmetic on the FP32 pipes (about 44 significant bits; the mixed MM-side sum takes 34-bit
// operands), where the FP64 kernel issues about 30 FP64 instructions per (G, atom).  The
// multipoles of a chunk of atoms are staged in shared memory, pre-scaled by exact powers of two so
// that Q - 1/2 G.theta.G = Q + sum_{a <= b} m_ab G_a G_b (m_aa = -theta_aa / 2, m_ab = -theta_ab).
constexpr int MSF_CH = 64;
__global__ void __launch_bounds__(256) k_multipole_sf_df(EwaldDev e, const double *gfac, const double *mult,
                                                         const float4 *phdf, double2 *A, double2 *Az, float4 *Adf,
                                                         float4 *Azdf)
{
    __shared__ float2 msh[MSF_CH][10];
    const int kx = e.kmax[0], ky = e.kmax[1], kz = e.kmax[2];
    const int NY = 2 * ky + 1, NZ = 2 * kz + 1, n = (kx + 1) * NY * NZ;
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    const bool act = k < n && gfac[k] != 0.0;
    const int kk = min(k, n - 1);
    const int nx = kk / (NY * NZ), iy = (kk / NZ) % NY, iz = kk % NZ;
    const f2 G[3] = {f2_mul(f2_from(TWO_PI / e.box[0]), f2{(float)nx, 0.0f}),
                     f2_mul(f2_from(TWO_PI / e.box[1]), f2{(float)(iy - ky), 0.0f}),
                     f2_mul(f2_from(TWO_PI / e.box[2]), f2{(float)(iz - kz), 0.0f})};
    const f2 u[6] = {f2_mul(G[0], G[0]), f2_mul(G[0], G[1]), f2_mul(G[0], G[2]),
                     f2_mul(G[1], G[1]), f2_mul(G[1], G[2]), f2_mul(G[2], G[2])};
    // normalised double-float from an accumulator (two-sum)
    auto norm = [](float h, float l) {
        const float s = h + l, v = s - h;
        return f2{s, (h - (s - v)) + (l - v)};
    };
    float rh = 0.0f, rl = 0.0f, ih = 0.0f, il = 0.0f;
    for (int j0 = 0; j0 < e.natm; j0 += MSF_CH) {
        const int nj = min(MSF_CH, e.natm - j0);
        __syncthreads();
        for (int t = threadIdx.x; t < nj * 10; t += blockDim.x) {
            const int jj = t / 10, c = t - jj * 10;
            double v = mult[10 * (size_t)(j0 + jj) + c];
            if (c >= 4) v *= (c == 4 || c == 7 || c == 9) ? -0.5 : -1.0;
            const f2 f = f2_from(v);
            msh[jj][c] = make_float2(f.h, f.l);
        }
        __syncthreads();
        if (!act) continue;
        for (int jj = 0; jj < nj; ++jj) {
            const float2 *M = msh[jj];
            float mh = M[0].x, ml = M[0].y;  // Q + sum m_ab G_a G_b
#pragma unroll
            for (int c = 0; c < 6; ++c) f2_mac(mh, ml, f2{M[4 + c].x, M[4 + c].y}, u[c]);
            float qh = 0.0f, ql = 0.0f;  // G.mu
#pragma unroll
            for (int a = 0; a < 3; ++a) f2_mac(qh, ql, f2{M[1 + a].x, M[1 + a].y}, G[a]);
            const f2 mr = norm(mh, ml), mi = norm(qh, ql);
            const float4 *pj = phdf + (size_t)(j0 + jj) * 3 * PHR_MAXN;
            const c2 p = c2_mul(c2_mul(c2_from(__ldg(pj + nx)), c2_from(__ldg(pj + PHR_MAXN + iy))),
                                c2_from(__ldg(pj + 2 * PHR_MAXN + iz)));
            // re += c mr - s mi, im += s mr + c mi
            f2_mac(rh, rl, p.re, mr);
            f2_mac(rh, rl, f2_neg(p.im), mi);
            f2_mac(ih, il, p.im, mr);
            f2_mac(ih, il, p.re, mi);
        }
    }
    if (k >= n) return;
    if (!act) {
        A[k] = make_double2(0.0, 0.0);
        Az[k] = make_double2(0.0, 0.0);
        Adf[k] = make_float4(0.f, 0.f, 0.f, 0.f);
        Azdf[k] = make_float4(0.f, 0.f, 0.f, 0.f);
        return;
    }
    const double g = gfac[k], re = f2_to(rh, rl), im = f2_to(ih, il);
    const double Gz = TWO_PI * (iz - kz) / e.box[2];
    A[k] = make_double2(g * re, g * im);
    Az[k] = make_double2(Gz * g * re, Gz * g * im);
    Adf[k] = c2_pack(g * re, g * im);
    Azdf[k] = c2_pack(Gz * g * re, Gz * g * im);
}

// dq_i += sum_G Re[A(G) exp(-iG.R_i)],  dR_i += q_i sum_G G Im[A(G) exp(-iG.R_i)].
// exp(-iG.R) = X(n_x) Y(n_y) Z(n_z).  A block takes 32 MM charges (one per lane) and its 8 warps
// share the half-space (n_x, n_y) lines round-robin: for each line a warp stages the line's A and
// Az rows in shared memory, forms B = sum_nz A Z and Bz = sum_nz Az Z per lane (Z rows of the
// block's charges in shared memory, one row per lane), then applies X(n_x) Y(n_y) from per-charge
// phase tables.  The 8 warps' partial sums are added in a fixed order at the end.  Small blocks
// (32 charges) make a grid of many waves, so the last one leaves little of the GPU idle.
constexpr int MMR_CH = 32, MMR_WARPS = 8, MMR_SEG = 8;

// shared memory of one block: phase tables Z[NZ][32], X[NX][32], Y[NY][32] (16 B entries), the
// per-warp A/Az line buffers [8][2][NZ] (16 B) and the reduction area [8 values][8 warps][32]
// (4 B, double-float) / [4][8][32] (8 B, FP64) -- 8 KiB either way.
size_t mm_recip_smem(const EwaldDev &e)
{
    const int NX = e.kmax[0] + 1, NY = 2 * e.kmax[1] + 1, NZ = 2 * e.kmax[2] + 1;
    return (size_t)(NZ + NX + NY) * MMR_CH * 16 + (size_t)MMR_WARPS * 2 * NZ * 16 + 8 * MMR_WARPS * MMR_CH * 4;
}

// line index -> (n_x, row of n_y): n_x = 0 keeps n_y >= 0 (the half space), n_x > 0 all n_y
__device__ __forceinline__ void mm_line(int L, int ky, int NY, int &nx, int &iy)
{
    if (L <= ky) {
        nx = 0;
        iy = ky + L;
    } else {
        const int r = L - ky - 1;
        nx = 1 + r / NY;
        iy = r % NY;
    }
}

__global__ void __launch_bounds__(MMR_CH *MMR_WARPS, 2) k_mm_recip(EwaldDev e, const double2 *__restrict__ A,
                                                                 const double2 *__restrict__ Az, double *dq,
                                                                 double *dR)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int kx = e.kmax[0], ky = e.kmax[1], kz = e.kmax[2];
    const int NX = kx + 1, NY = 2 * ky + 1, NZ = 2 * kz + 1;
    double2 *zs = reinterpret_cast<double2 *>(smem_raw);  // [NZ][32]
    double2 *xs = zs + NZ * MMR_CH;                        // [NX][32]
    double2 *ys = xs + NX * MMR_CH;                        // [NY][32]
    double2 *wab = ys + NY * MMR_CH;                       // [8][2][NZ]
    double *red = reinterpret_cast<double *>(wab + MMR_WARPS * 2 * NZ);  // [4][8][32]
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int i = blockIdx.x * MMR_CH + lane;
    const bool act = i < e.nmm;
    const int ii = act ? i : 0;
    // fractional coordinates
    const double u0 = e.mm_xyz[3 * ii] / e.box[0], u1 = e.mm_xyz[3 * ii + 1] / e.box[1],
                 u2 = e.mm_xyz[3 * ii + 2] / e.box[2];
    // phase rows in segments of 8 (one sincospi each, then the recurrence), segments over warps
    {
        const int sx = (NX + MMR_SEG - 1) / MMR_SEG, sy = (NY + MMR_SEG - 1) / MMR_SEG,
                  sz = (NZ + MMR_SEG - 1) / MMR_SEG;
        for (int sg = warp; sg < sx + sy + sz; sg += MMR_WARPS) {
            const int d = sg < sx ? 0 : sg < sx + sy ? 1 : 2;
            const int s = sg - (d == 0 ? 0 : d == 1 ? sx : sx + sy);
            const int len = d == 0 ? NX : d == 1 ? NY : NZ, off = d == 0 ? 0 : d == 1 ? ky : kz;
            const double fd = d == 0 ? u0 : d == 1 ? u1 : u2;
            double2 *row = d == 0 ? xs : d == 1 ? ys : zs;
            double sn, cs;
            sincospi(-2.0 * fd, &sn, &cs);
            const double2 step = make_double2(cs, sn);
            const int n0 = s * MMR_SEG;
            sincospi(-2.0 * (n0 - off) * fd, &sn, &cs);
            double2 p = make_double2(cs, sn);
            for (int n = n0; n < min(len, n0 + MMR_SEG); ++n) {
                row[n * MMR_CH + lane] = p;
                p = cmul(p, step);
            }
        }
    }
    __syncthreads();
    double pot = 0.0, fx = 0.0, fy = 0.0, fz = 0.0;
    double2 *wa = wab + warp * 2 * NZ, *waz = wa + NZ;
    const int nlines = kx * NY + ky + 1;
    for (int L = warp; L < nlines; L += MMR_WARPS) {
        int nx, iy;
        mm_line(L, ky, NY, nx, iy);
        const size_t base = ((size_t)nx * NY + iy) * NZ;
        __syncwarp();
        for (int k = lane; k < NZ; k += 32) {
            wa[k] = __ldg(A + base + k);
            waz[k] = __ldg(Az + base + k);
        }
        __syncwarp();
        double br = 0.0, bi = 0.0, bzr = 0.0, bzi = 0.0;
        for (int iz = 0; iz < NZ; ++iz) {
            const double2 a = wa[iz], az = waz[iz], z = zs[iz * MMR_CH + lane];
            br = fma(a.x, z.x, br);
            br = fma(-a.y, z.y, br);
            bi = fma(a.x, z.y, bi);
            bi = fma(a.y, z.x, bi);
            bzr = fma(az.x, z.x, bzr);
            bzr = fma(-az.y, z.y, bzr);
            bzi = fma(az.x, z.y, bzi);
            bzi = fma(az.y, z.x, bzi);
        }
        const double2 pxy = cmul(xs[nx * MMR_CH + lane], ys[iy * MMR_CH + lane]);
        const double re = pxy.x * br - pxy.y * bi;
        const double im = pxy.x * bi + pxy.y * br;
        pot += re;
        fx += TWO_PI * nx / e.box[0] * im;
        fy += TWO_PI * (iy - ky) / e.box[1] * im;
        fz += pxy.x * bzi + pxy.y * bzr;
    }
    red[(0 * MMR_WARPS + warp) * MMR_CH + lane] = pot;
    red[(1 * MMR_WARPS + warp) * MMR_CH + lane] = fx;
    red[(2 * MMR_WARPS + warp) * MMR_CH + lane] = fy;
    red[(3 * MMR_WARPS + warp) * MMR_CH + lane] = fz;
    __syncthreads();
    if (warp == 0 && act) {
        double t[4] = {0.0, 0.0, 0.0, 0.0};
        for (int w = 0; w < MMR_WARPS; ++w)
#pragma unroll
            for (int v = 0; v < 4; ++v) t[v] += red[(v * MMR_WARPS + w) * MMR_CH + lane];
        const double q = e.mm_q[i];
        dq[i] += t[0];
        dR[3 * i] += q * t[1];
        dR[3 * i + 1] += q * t[2];
        dR[3 * i + 2] += q * t[3];
    }
}

// Double-float variant (mixed-precision path): A, Az and the phase tables as FP32 (hi, lo)
// pairs; the dot products along n_z are error-free multiply-adds, the per-line combination runs
// in double-float arithmetic, and the phase rows start from one FP64 sincospi per segment.
__global__ void __launch_bounds__(MMR_CH *MMR_WARPS, 3) k_mm_recip_df(EwaldDev e, const float4 *__restrict__ A,
                                                                    const float4 *__restrict__ Az, double *dq,
                                                                    double *dR)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int kx = e.kmax[0], ky = e.kmax[1], kz = e.kmax[2];
    const int NX = kx + 1, NY = 2 * ky + 1, NZ = 2 * kz + 1;
    float4 *zs = reinterpret_cast<float4 *>(smem_raw);  // [NZ][32]
    float4 *xs = zs + NZ * MMR_CH;                       // [NX][32]
    float4 *ys = xs + NX * MMR_CH;                       // [NY][32]
    float4 *wab = ys + NY * MMR_CH;                      // [8][2][NZ]
    float *red = reinterpret_cast<float *>(wab + MMR_WARPS * 2 * NZ);  // [8][8][32]
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int i = blockIdx.x * MMR_CH + lane;
    const bool act = i < e.nmm;
    const int ii = act ? i : 0;
    // fractional coordinates
    const double u0 = e.mm_xyz[3 * ii] / e.box[0], u1 = e.mm_xyz[3 * ii + 1] / e.box[1],
                 u2 = e.mm_xyz[3 * ii + 2] / e.box[2];
    {
        const int sx = (NX + MMR_SEG - 1) / MMR_SEG, sy = (NY + MMR_SEG - 1) / MMR_SEG,
                  sz = (NZ + MMR_SEG - 1) / MMR_SEG;
        for (int sg = warp; sg < sx + sy + sz; sg += MMR_WARPS) {
            const int d = sg < sx ? 0 : sg < sx + sy ? 1 : 2;
            const int s = sg - (d == 0 ? 0 : d == 1 ? sx : sx + sy);
            const int len = d == 0 ? NX : d == 1 ? NY : NZ, off = d == 0 ? 0 : d == 1 ? ky : kz;
            const double fd = d == 0 ? u0 : d == 1 ? u1 : u2;
            float4 *row = d == 0 ? xs : d == 1 ? ys : zs;
            double sn, cs;
            sincospi(-2.0 * fd, &sn, &cs);
            const c2 step{f2_from(cs), f2_from(sn)};
            const int n0 = s * MMR_SEG;
            sincospi(-2.0 * (n0 - off) * fd, &sn, &cs);
            c2 p{f2_from(cs), f2_from(sn)};
            for (int n = n0; n < min(len, n0 + MMR_SEG); ++n) {
                row[n * MMR_CH + lane] = make_float4(p.re.h, p.re.l, p.im.h, p.im.l);
                p = c2_mul(p, step);
            }
        }
    }
    __syncthreads();
    f2 pot{0.f, 0.f}, fx{0.f, 0.f}, fy{0.f, 0.f}, fz{0.f, 0.f};
    float4 *wa = wab + warp * 2 * NZ, *waz = wa + NZ;
    const f2 gx1 = f2_from(TWO_PI / e.box[0]), gy1 = f2_from(TWO_PI / e.box[1]);
    const int nlines = kx * NY + ky + 1;
    for (int L = warp; L < nlines; L += MMR_WARPS) {
        int nx, iy;
        mm_line(L, ky, NY, nx, iy);
        const size_t base = ((size_t)nx * NY + iy) * NZ;
        __syncwarp();
        for (int k = lane; k < NZ; k += 32) {
            wa[k] = __ldg(A + base + k);
            waz[k] = __ldg(Az + base + k);
        }
        __syncwarp();
        // two independent accumulator sets (even / odd n_z) for instruction-level parallelism
        float B[4] = {0.f, 0.f, 0.f, 0.f}, Bz[4] = {0.f, 0.f, 0.f, 0.f};
        float C[4] = {0.f, 0.f, 0.f, 0.f}, Cz[4] = {0.f, 0.f, 0.f, 0.f};
        int iz = 0;
        for (; iz + 1 < NZ; iz += 2) {
            const c2 z0 = c2_from(zs[iz * MMR_CH + lane]), z1 = c2_from(zs[(iz + 1) * MMR_CH + lane]);
            c2_mac(B, c2_from(wa[iz]), z0);
            c2_mac(C, c2_from(wa[iz + 1]), z1);
            c2_mac(Bz, c2_from(waz[iz]), z0);
            c2_mac(Cz, c2_from(waz[iz + 1]), z1);
        }
        if (iz < NZ) {
            const c2 z0 = c2_from(zs[iz * MMR_CH + lane]);
            c2_mac(B, c2_from(wa[iz]), z0);
            c2_mac(Bz, c2_from(waz[iz]), z0);
        }
        const c2 pxy = c2_mul(c2_from(xs[nx * MMR_CH + lane]), c2_from(ys[iy * MMR_CH + lane]));
        const c2 b{f2_add(f2_add(f2{B[0], 0.f}, f2{B[1], 0.f}), f2_add(f2{C[0], 0.f}, f2{C[1], 0.f})),
                   f2_add(f2_add(f2{B[2], 0.f}, f2{B[3], 0.f}), f2_add(f2{C[2], 0.f}, f2{C[3], 0.f}))};
        const f2 bzr = f2_add(f2_add(f2{Bz[0], 0.f}, f2{Bz[1], 0.f}), f2_add(f2{Cz[0], 0.f}, f2{Cz[1], 0.f}));
        const f2 bzi = f2_add(f2_add(f2{Bz[2], 0.f}, f2{Bz[3], 0.f}), f2_add(f2{Cz[2], 0.f}, f2{Cz[3], 0.f}));
        const c2 pr = c2_mul(pxy, b);
        pot = f2_add(pot, pr.re);
        // G_x = (2 pi / L_x) n_x and G_y = (2 pi / L_y) n_y: small integers times a double-float
        fx = f2_add(fx, f2_mul(f2_mul(gx1, f2{(float)nx, 0.f}), pr.im));
        fy = f2_add(fy, f2_mul(f2_mul(gy1, f2{(float)(iy - ky), 0.f}), pr.im));
        fz = f2_add(fz, f2_add(f2_mul(pxy.re, bzi), f2_mul(pxy.im, bzr)));
    }
    const f2 vals[4] = {pot, fx, fy, fz};
#pragma unroll
    for (int v = 0; v < 4; ++v) {
        red[((2 * v) * MMR_WARPS + warp) * MMR_CH + lane] = vals[v].h;
        red[((2 * v + 1) * MMR_WARPS + warp) * MMR_CH + lane] = vals[v].l;
    }
    __syncthreads();
    if (warp == 0 && act) {
        f2 t[4] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
        for (int w = 0; w < MMR_WARPS; ++w)
#pragma unroll
            for (int v = 0; v < 4; ++v)
                t[v] = f2_add(t[v], f2{red[((2 * v) * MMR_WARPS + w) * MMR_CH + lane],
                                       red[((2 * v + 1) * MMR_WARPS + w) * MMR_CH + lane]});
        const double q = e.mm_q[i];
        dq[i] += f2_to(t[0]);
        dR[3 * i] += q * f2_to(t[1]);
        dR[3 * i + 1] += q * f2_to(t[2]);
        dR[3 * i + 2] += q * f2_to(t[3]);
    }
}

__global__ void k_mm_background(EwaldDev e, const double *sums, double *dq)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= e.nmm) return;
    dq[i] += -PI / (e.box[0] * e.box[1] * e.box[2] * e.alpha * e.alpha) * sums[1];
}

// QM tensor gradient: dE/dR_j,x = sum_c w_c M_j,c d_x v_j,c (d_x v_0 = v_x, d_x v_a = 2 v_ax, d_x v_ab = 3 v_abx)
__global__ void k_qm_tensor_grad(int natm, const double *mult, const double *phi, double *gqm)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= natm) return;
    double p, fl[3];
    contract_pot_field(mult + 10 * j, phi + 20 * j, p, fl);
    atomicAdd(gqm + 3 * j, fl[0]);  // atomics: the region-I adjoint sweep may run at the same time
    atomicAdd(gqm + 3 * j + 1, fl[1]);
    atomicAdd(gqm + 3 * j + 2, fl[2]);
}

cudaError_t launch_ewald_mm(const EwaldDev &e, const double4_32a *rI, int nI, const double *mult, const double *phi,
                            const EwaldBuf &w, double *dq_int, double *dR_int, double *gchg, double *gqm, bool df,
                            cudaStream_t st)
{
    cudaError_t err;
    if ((err = launch_sum_strided(mult, e.natm, 10, w.sums + 1, st)) != cudaSuccess) return err;
    if (e.nmm > 0) {
        k_mm_real<<<(e.nmm + MMQ_CH - 1) / MMQ_CH, 256, 0, st>>>(e, mult, dq_int, dR_int);
        if ((err = cudaGetLastError()) != cudaSuccess) return err;
    }
    if (nI > 0) {
        k_mm_region1<<<(nI + MMQ_CH - 1) / MMQ_CH, MMQ_CH * MMQ_WARPS, 0, st>>>(e, rI, nI, mult, gchg);
        if ((err = cudaGetLastError()) != cudaSuccess) return err;
    }
    if (e.nmm > 0) {
        const int n = ewald_dense_size(e);
        const bool sfdf = df && w.atom_phdf && w.Adf && w.Azdf;
        k_atom_phases<<<e.natm, 128, 0, st>>>(e, w.atom_ph, sfdf ? w.atom_phdf : nullptr);
        if ((err = cudaGetLastError()) != cudaSuccess) return err;
        if (sfdf)
            k_multipole_sf_df<<<(n + 255) / 256, 256, 0, st>>>(e, w.gfac, mult, w.atom_phdf, w.A, w.Az, w.Adf,
                                                                w.Azdf);
        else
            k_multipole_sf<<<(n + 255) / 256, 256, 0, st>>>(e, w.gfac, mult, w.atom_ph, w.A, w.Az,
                                                             df ? w.Adf : nullptr, df ? w.Azdf : nullptr);
        if ((err = cudaGetLastError()) != cudaSuccess) return err;
        const MmrShape &ms = w.mms[df ? 1 : 0];
        if (w.recip == 1 && ms.supported) {
            if ((err = launch_mm_recip_tc(e, ms, w.mmb, w.A, w.Az, dq_int, dR_int, w.err, st)) != cudaSuccess)
                return err;
            k_mm_background<<<(e.nmm + 255) / 256, 256, 0, st>>>(e, w.sums, dq_int);
            if ((err = cudaGetLastError()) != cudaSuccess) return err;
            k_qm_tensor_grad<<<(e.natm + 63) / 64, 64, 0, st>>>(e.natm, mult, phi, gqm);
            return cudaGetLastError();
        }
        const size_t smem = mm_recip_smem(e);
        static size_t attr = 0, attr_df = 0;
        size_t &a = df ? attr_df : attr;
        if (smem > 48 * 1024 && smem > a) {
            if ((err = cudaFuncSetAttribute(df ? (const void *)k_mm_recip_df : (const void *)k_mm_recip,
                                            cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess)
                return err;
            a = smem;
        }
        const int nb = (e.nmm + MMR_CH - 1) / MMR_CH;
        if (df)
            k_mm_recip_df<<<nb, MMR_CH * MMR_WARPS, smem, st>>>(e, w.Adf, w.Azdf, dq_int, dR_int);
        else
            k_mm_recip<<<nb, MMR_CH * MMR_WARPS, smem, st>>>(e, w.A, w.Az, dq_int, dR_int);
        if ((err = cudaGetLastError()) != cudaSuccess) return err;
        k_mm_background<<<(e.nmm + 255) / 256, 256, 0, st>>>(e, w.sums, dq_int);
        if ((err = cudaGetLastError()) != cudaSuccess) return err;
    }
    k_qm_tensor_grad<<<(e.natm + 63) / 64, 64, 0, st>>>(e.natm, mult, phi, gqm);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------------
// region-I nuclear-MM term  sum_j Z_j q_C erf(r/sigma_C)/r  (1/r for point charges)
// ---------------------------------------------------------------------------------------------
// Block = 32 charges x 8 warps; warp w takes the QM atoms j = w, w + 8, ...  Per-charge values
// are summed over the 8 warps in shared memory in a fixed order, so E and dE/dq are reproducible.
constexpr int ENUC_CH = 32, ENUC_WARPS = 8;
int enucmm_nblk(int nI) { return nI > 0 ? (nI + ENUC_CH - 1) / ENUC_CH : 1; }

__global__ void __launch_bounds__(ENUC_CH * ENUC_WARPS)
k_enucmm(const double *qm_xyz, const double *Z, int natm, const double4_32a *rI, const int *rI_idx, int nI,
         const double *mm_beta, double *Epart, double *gqm, double *gchg, int want_grad)
{
    __shared__ double red[5][ENUC_WARPS][ENUC_CH];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int k = blockIdx.x * ENUC_CH + lane;
    const bool act = k < nI;
    double4_32a c;
    c.x = c.y = c.z = c.w = 0.0;
    double beta = 0.0;
    if (act) {
        c = rI[k];
        beta = mm_beta[rI_idx[k]];
    }
    double E = 0.0, dq = 0.0, dC[3] = {0.0, 0.0, 0.0};
    for (int j = warp; j < natm; j += ENUC_WARPS) {
        double g[3] = {0.0, 0.0, 0.0};
        if (act) {
            const double x = qm_xyz[3 * j] - c.x, y = qm_xyz[3 * j + 1] - c.y, z = qm_xyz[3 * j + 2] - c.z;
            const double r2 = x * x + y * y + z * z, r = sqrt(r2);
            double f, fpr;  // f(r) and f'(r)/r
            if (beta > 0.0) {
                const double c2 = beta * (2.0 / 1.7724538509055160273), br2 = beta * beta * r2;
                if (br2 < 1e-8) {
                    // charge centre on (or next to) the nucleus: series of erf(beta r)/r about r = 0
                    f = c2 * (1.0 - br2 * (1.0 / 3.0));
                    fpr = -(2.0 / 3.0) * c2 * beta * beta * (1.0 - 0.6 * br2);
                } else {
                    f = erf(beta * r) / r;
                    fpr = (c2 * exp(-br2) - f) / r2;
                }
            } else {
                f = 1.0 / r;
                fpr = -f / r2;
            }
            const double Zj = Z[j];
            E += Zj * c.w * f;
            dq += Zj * f;
            const double s = Zj * c.w * fpr;
            g[0] = s * x; g[1] = s * y; g[2] = s * z;
            dC[0] -= g[0]; dC[1] -= g[1]; dC[2] -= g[2];
        }
        if (want_grad) {
#pragma unroll
            for (int x = 0; x < 3; ++x) {
                const double v = warp_sum(g[x]);
                if (lane == 0 && v != 0.0) atomicAdd(gqm + 3 * j + x, v);
            }
        }
    }
    red[0][warp][lane] = E;
    red[1][warp][lane] = dq;
    red[2][warp][lane] = dC[0];
    red[3][warp][lane] = dC[1];
    red[4][warp][lane] = dC[2];
    __syncthreads();
    if (warp == 0) {
        double t[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
        for (int w = 0; w < ENUC_WARPS; ++w)
#pragma unroll
            for (int v = 0; v < 5; ++v) t[v] += red[v][w][lane];
        if (want_grad && act) {  // atomics: the region-I adjoint sweep may add at the same time
            atomicAdd(gchg + 4 * (size_t)k + 0, t[2]);
            atomicAdd(gchg + 4 * (size_t)k + 1, t[3]);
            atomicAdd(gchg + 4 * (size_t)k + 2, t[4]);
            atomicAdd(gchg + 4 * (size_t)k + 3, t[1]);
        }
        const double e = warp_sum(t[0]);
        if (lane == 0) Epart[blockIdx.x] = e;
    }
}

cudaError_t launch_enucmm(const double *qm_xyz, const double *Z, int natm, const double4_32a *rI, const int *rI_idx,
                          int nI, const double *mm_beta, double *Epart, double *gqm, double *gchg, int want_grad,
                          cudaStream_t st)
{
    k_enucmm<<<enucmm_nblk(nI), ENUC_CH * ENUC_WARPS, 0, st>>>(qm_xyz, Z, natm, rI, rI_idx, nI, mm_beta, Epart, gqm,
                                                               gchg, want_grad);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------------
// Octupole error estimate of the multipole truncation (Sec. "Error Control")
//   Err(R) = sum_j sum_abc Omega_j,abc v_j,abc(R),
// v_j,abc(R) the third Taylor components of the region-II potential with region I of radius R.
// From the handle's v (region I of radius rc) it follows for any R by moving the images between
// the two spheres:  Err(R) = E0 + F(rc) - F(R),  F(R) = sum over images with r_min <= d < R of
//   e_i = q_i sum_j Omega_j : (T_ji - [r_ji < 9 sigma_i] T-hat_ji)   (third-order parts),
// d = |image - centre|, since an image entering region I adds -q T (the region-I subtraction) and
// drops -q T-hat (the Gaussian correction of region II).
// ---------------------------------------------------------------------------------------------
__constant__ double c_mult3[10] = {1, 3, 3, 3, 6, 3, 1, 3, 3, 1};  // multiplicity of each unique component

// bins[k], k < nbin - 1: images with r_lo + k dr <= d < r_lo + (k + 1) dr;  bins[nbin - 1]: images
// with r_min <= d < r_lo;  bins[nbin]: images with r_min <= d < rc.  e.rcut must be r_max.
__global__ void __launch_bounds__(256) k_oct_shell(EwaldDev e, const double *oct, double r_min, double r_lo,
                                                   double dr, int nbin, double rc, double *bins)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= e.nmm) return;
    const double q = e.mm_q[i], beta = e.mm_beta[i];
    const double rhat2 = beta > 0.0 ? (9.0 / beta) * (9.0 / beta) : -1.0;
    region1_images(e, i, [&](double px, double py, double pz, int) {
        const double cx = px - e.centre[0], cy = py - e.centre[1], cz = pz - e.centre[2];
        const double d = sqrt(cx * cx + cy * cy + cz * cz);
        if (d < r_min) return;
        double ei = 0.0, T[20], Th[20];
        for (int j = 0; j < e.natm; ++j) {
            const double x = __ldg(e.qm_xyz + 3 * j) - px, y = __ldg(e.qm_xyz + 3 * j + 1) - py,
                         z = __ldg(e.qm_xyz + 3 * j + 2) - pz;
            const double r2 = x * x + y * y + z * z;
            double f, g1, g2, g3;
            point_radial(r2, f, g1, g2, g3);
            radial_tensor(f, g1, g2, g3, x, y, z, T, 3);
            if (r2 < rhat2) {
                screened_radial(r2, beta, f, g1, g2, g3);
                radial_tensor(f, g1, g2, g3, x, y, z, Th, 3);
#pragma unroll
                for (int c = 10; c < 20; ++c) T[c] -= Th[c];
            }
#pragma unroll
            for (int c = 0; c < 10; ++c) ei += c_mult3[c] * __ldg(oct + 10 * j + c) * T[10 + c];
        }
        ei *= q;
        if (d < r_lo) atomicAdd(bins + nbin - 1, ei);
        else {
            const int k = (int)floor((d - r_lo) / dr);
            if (k < nbin - 1) atomicAdd(bins + k, ei);
        }
        if (d < rc) atomicAdd(bins + nbin, ei);
    });
}

// E0 = sum_j Omega_j : v_j(rc) and err[k] = E0 + F(rc) - F(R_k); one block
__global__ void k_oct_finish(const double *oct, const double *phi, int natm, const double *bins, int nbin,
                             double *err)
{
    __shared__ double ws[32];
    double s = 0.0;
    for (int t = threadIdx.x; t < 10 * natm; t += blockDim.x) s += c_mult3[t % 10] * oct[t] * phi[20 * (t / 10) + 10 + t % 10];
    s = warp_sum(s);
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double e0 = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) e0 += ws[w];
        double F = bins[nbin - 1];  // F(r_lo)
        for (int k = 0; k < nbin; ++k) {
            err[k] = e0 + bins[nbin] - F;
            if (k < nbin - 1) F += bins[k];
        }
    }
}

cudaError_t launch_octupole_error(const EwaldDev &e0, const double *oct, const double *phi, double r_lo, double dr,
                                  int n, double *bins, double *err, cudaStream_t st)
{
    EwaldDev e = e0;
    const double rc = e0.rcut, r_hi = r_lo + (n - 1) * dr;
    const double r_min = fmin(r_lo, rc);
    e.rcut = fmax(r_hi, rc);  // candidate images: r_min <= d < r_max
    cudaError_t err_ = cudaMemsetAsync(bins, 0, (n + 1) * sizeof(double), st);
    if (err_ != cudaSuccess) return err_;
    if (e.nmm > 0) {
        k_oct_shell<<<(e.nmm + 255) / 256, 256, 0, st>>>(e, oct, r_min, r_lo, dr, n, rc, bins);
        if ((err_ = cudaGetLastError()) != cudaSuccess) return err_;
    }
    k_oct_finish<<<1, 256, 0, st>>>(oct, phi, e.natm, bins, n, err);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------------
// QM-QM periodic images (Eq. 5 in the Ewald form of Eq. 6)
//   P_ji = sum_{L != 0} T(R_j - R_i + L) (20 Taylor components), by Ewald: erfc real space over
//   images within the Ewald cutoff, reciprocal sum over the half space (2 g(G) weights), self
//   terms -2 kappa/sqrt(pi) and +(2/3) kappa^3/sqrt(pi) delta_ab for i = j, minus the L = 0 point
//   tensor for i != j (the reference-cell pair belongs to the QM calculation).
//   E = 1/2 sum_{j,i} [Q_j Q_i P + 2 mu_j.Q_i P_a + 2 theta_j:Q_i P_ab - 2 mu_j mu_i : P_ab]
//       - pi/(2 V kappa^2) (sum Q)^2.
// ---------------------------------------------------------------------------------------------
__constant__ int c_p2[6][2] = {{0, 0}, {0, 1}, {0, 2}, {1, 1}, {1, 2}, {2, 2}};
__constant__ int c_p3[10][3] = {{0, 0, 0}, {0, 0, 1}, {0, 0, 2}, {0, 1, 1}, {0, 1, 2},
                                {0, 2, 2}, {1, 1, 1}, {1, 1, 2}, {1, 2, 2}, {2, 2, 2}};

// one block per ordered pair (i = blockIdx.x, j = blockIdx.y); P[(j*natm + i)*20 + c]
__global__ void __launch_bounds__(128) k_qmqm_pairs(EwaldDev e, const double *gfac, double *P)
{
    __shared__ double scratch[4 * 20];
    const int i = blockIdx.x, j = blockIdx.y;
    const double d0[3] = {e.qm_xyz[3 * j] - e.qm_xyz[3 * i], e.qm_xyz[3 * j + 1] - e.qm_xyz[3 * i + 1],
                          e.qm_xyz[3 * j + 2] - e.qm_xyz[3 * i + 2]};
    double acc[20];
#pragma unroll
    for (int c = 0; c < 20; ++c) acc[c] = 0.0;
    const int kx = e.kmax[0], ky = e.kmax[1], kz = e.kmax[2];
    const int NY = 2 * ky + 1, NZ = 2 * kz + 1, n = (kx + 1) * NY * NZ;
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
        const double w = gfac[k];
        if (w == 0.0) continue;
        const double G[3] = {TWO_PI * (k / (NY * NZ)) / e.box[0], TWO_PI * ((k / NZ) % NY - ky) / e.box[1],
                             TWO_PI * (k % NZ - kz) / e.box[2]};
        double sn, cs;
        sincos(G[0] * d0[0] + G[1] * d0[1] + G[2] * d0[2], &sn, &cs);
        acc[0] += w * cs;
#pragma unroll
        for (int a = 0; a < 3; ++a) acc[1 + a] -= w * G[a] * sn;
#pragma unroll
        for (int c = 0; c < 6; ++c) acc[4 + c] -= 0.5 * w * G[c_p2[c][0]] * G[c_p2[c][1]] * cs;
#pragma unroll
        for (int c = 0; c < 10; ++c)
            acc[10 + c] += w * G[c_p3[c][0]] * G[c_p3[c][1]] * G[c_p3[c][2]] * sn * (1.0 / 6.0);
    }
    if (threadIdx.x == 0) {
        double T[20];
        const double rc2 = e.ewald_rc * e.ewald_rc;
        double n0[3];
#pragma unroll
        for (int x = 0; x < 3; ++x) n0[x] = rint(d0[x] / e.box[x]);
        for (int a = -e.img[0] - 1; a <= e.img[0] + 1; ++a)
            for (int b = -e.img[1] - 1; b <= e.img[1] + 1; ++b)
                for (int c = -e.img[2] - 1; c <= e.img[2] + 1; ++c) {
                    const double L[3] = {(n0[0] + a) * e.box[0], (n0[1] + b) * e.box[1], (n0[2] + c) * e.box[2]};
                    if (i == j && L[0] == 0.0 && L[1] == 0.0 && L[2] == 0.0) continue;
                    const double x = d0[0] - L[0], y = d0[1] - L[1], z = d0[2] - L[2];
                    const double r2 = x * x + y * y + z * z;
                    if (r2 >= rc2) continue;
                    double f, g1, g2, g3;
                    screened_radial(r2, e.alpha, f, g1, g2, g3);
                    radial_tensor(f, g1, g2, g3, x, y, z, T, 3);
#pragma unroll
                    for (int k = 0; k < 20; ++k) acc[k] += T[k];
                }
        if (i == j) {
            const double k1 = 2.0 * e.alpha / 1.7724538509055160273, k3 = k1 * e.alpha * e.alpha / 3.0;
            acc[0] -= k1;
            acc[4] += k3;
            acc[7] += k3;
            acc[9] += k3;
        } else {
            double f, g1, g2, g3;
            point_radial(d0[0] * d0[0] + d0[1] * d0[1] + d0[2] * d0[2], f, g1, g2, g3);
            radial_tensor(f, g1, g2, g3, d0[0], d0[1], d0[2], T, 3);
#pragma unroll
            for (int k = 0; k < 20; ++k) acc[k] -= T[k];
        }
    }
    block_reduce_store<20>(acc, P + ((size_t)j * gridDim.x + i) * 20, scratch);
}

// Energy, image potentials u (dE/dM per stored component / W10, 20-stride like phi) and the
// gradient at fixed multipoles, from the pair tensors.  One block; each atom's sums in a fixed order.
__global__ void k_qmqm_contract(int natm, const double *P, const double *M, double bg, double *E, double *u20,
                                double *grad)
{
    __shared__ double ws[32];
    double esum = 0.0;
    for (int k = threadIdx.x; k < natm; k += blockDim.x) {
        double uk[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0}, gk[3] = {0.0, 0.0, 0.0};
        for (int o = 0; o < natm; ++o) {
            // (j, i) = (k, o): first slot is k
            for (int pass = 0; pass < 2; ++pass) {
                const int j = pass == 0 ? k : o, i = pass == 0 ? o : k;
                const double *p = P + ((size_t)j * natm + i) * 20;
                double Pab[3][3], thj[3][3];
                for (int c = 0; c < 6; ++c) {
                    const int a = c_p2[c][0], b = c_p2[c][1];
                    Pab[a][b] = Pab[b][a] = p[4 + c];
                    thj[a][b] = thj[b][a] = M[10 * j + 4 + c];
                }
                const double Qj = M[10 * j], Qi = M[10 * i];
                const double *mj = M + 10 * j + 1, *mi = M + 10 * i + 1;
                if (pass == 0) {
                    // the pair energy, counted once per ordered pair
                    double e2 = Qj * Qi * p[0];
                    for (int a = 0; a < 3; ++a) e2 += 2.0 * mj[a] * Qi * p[1 + a];
                    for (int a = 0; a < 3; ++a)
                        for (int b = 0; b < 3; ++b)
                            e2 += 2.0 * thj[a][b] * Qi * Pab[a][b] - 2.0 * mj[a] * mi[b] * Pab[a][b];
                    esum += 0.5 * e2;
                    // k in the first slot
                    uk[0] += 0.5 * Qi * p[0];
                    for (int a = 0; a < 3; ++a) {
                        double t = 2.0 * Qi * p[1 + a];
                        for (int b = 0; b < 3; ++b) t -= 2.0 * mi[b] * Pab[a][b];
                        uk[1 + a] += 0.5 * t;
                    }
                    for (int c = 0; c < 6; ++c) uk[4 + c] += Qi * p[4 + c];
                    // gradient: d/dR_j of e(j, i) with R_i fixed, for i != j
                    if (i != j)
                        for (int c = 0; c < 3; ++c) {
                            double g = Qj * Qi * p[1 + c];
                            for (int a = 0; a < 3; ++a) g += 4.0 * mj[a] * Qi * Pab[a][c];
                            for (int a = 0; a < 3; ++a)
                                for (int b = 0; b < 3; ++b) {
                                    // P_abc from the 10 stored components
                                    int s3[3] = {a, b, c};
                                    // sort the three indices
                                    if (s3[0] > s3[1]) { int t = s3[0]; s3[0] = s3[1]; s3[1] = t; }
                                    if (s3[1] > s3[2]) { int t = s3[1]; s3[1] = s3[2]; s3[2] = t; }
                                    if (s3[0] > s3[1]) { int t = s3[0]; s3[0] = s3[1]; s3[1] = t; }
                                    int idx = 0;
                                    for (int q = 0; q < 10; ++q)
                                        if (c_p3[q][0] == s3[0] && c_p3[q][1] == s3[1] && c_p3[q][2] == s3[2]) idx = q;
                                    g += (6.0 * thj[a][b] * Qi - 6.0 * mj[a] * mi[b]) * p[10 + idx];
                                }
                            gk[c] += 0.5 * g;
                        }
                } else {
                    // k in the second slot of e(j = o, i = k)
                    double t = Qj * p[0];
                    for (int a = 0; a < 3; ++a) t += 2.0 * mj[a] * p[1 + a];
                    for (int a = 0; a < 3; ++a)
                        for (int b = 0; b < 3; ++b) t += 2.0 * thj[a][b] * Pab[a][b];
                    uk[0] += 0.5 * t;
                    for (int b = 0; b < 3; ++b) {
                        double s2 = 0.0;
                        for (int a = 0; a < 3; ++a) s2 -= 2.0 * mj[a] * Pab[a][b];
                        uk[1 + b] += 0.5 * s2;
                    }
                    // gradient: d/dR_i of e(j, i) = -d/dd
                    if (i != j)
                        for (int c = 0; c < 3; ++c) {
                            double g = Qj * Qi * p[1 + c];
                            for (int a = 0; a < 3; ++a) g += 4.0 * mj[a] * Qi * Pab[a][c];
                            for (int a = 0; a < 3; ++a)
                                for (int b = 0; b < 3; ++b) {
                                    int s3[3] = {a, b, c};
                                    if (s3[0] > s3[1]) { int t2 = s3[0]; s3[0] = s3[1]; s3[1] = t2; }
                                    if (s3[1] > s3[2]) { int t2 = s3[1]; s3[1] = s3[2]; s3[2] = t2; }
                                    if (s3[0] > s3[1]) { int t2 = s3[0]; s3[0] = s3[1]; s3[1] = t2; }
                                    int idx = 0;
                                    for (int q = 0; q < 10; ++q)
                                        if (c_p3[q][0] == s3[0] && c_p3[q][1] == s3[1] && c_p3[q][2] == s3[2]) idx = q;
                                    g += (6.0 * thj[a][b] * Qi - 6.0 * mj[a] * mi[b]) * p[10 + idx];
                                }
                            gk[c] -= 0.5 * g;
                        }
                }
            }
        }
        double qsum = 0.0;
        for (int o = 0; o < natm; ++o) qsum += M[10 * o];
        uk[0] += 2.0 * bg * qsum;
        for (int c = 0; c < 10; ++c) u20[20 * k + c] = uk[c];
        for (int c = 10; c < 20; ++c) u20[20 * k + c] = 0.0;
        for (int c = 0; c < 3; ++c) grad[3 * k + c] = gk[c];
    }
    esum = warp_sum(esum);
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = esum;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0, qsum = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += ws[w];
        for (int o = 0; o < natm; ++o) qsum += M[10 * o];
        E[0] = t + bg * qsum * qsum;
    }
}

cudaError_t launch_qm_images(const EwaldDev &e, const double *gfac, const double *mult, double *P, double *E,
                             double *u20, double *grad, cudaStream_t st)
{
    if (e.natm <= 0) return cudaSuccess;
    k_qmqm_pairs<<<dim3(e.natm, e.natm), 128, 0, st>>>(e, gfac, P);
    cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess) return err;
    const double V = e.box[0] * e.box[1] * e.box[2];
    k_qmqm_contract<<<1, 256, 0, st>>>(e.natm, P, mult, -PI / (2.0 * V * e.alpha * e.alpha), E, u20, grad);
    return cudaGetLastError();
}

__global__ void k_scatter_region(const int *rI_idx, int nI, const double *gchg, double *dq, double *dR)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nI) return;
    const int i = rI_idx[k];
    atomicAdd(dR + 3 * i, gchg[4 * (size_t)k]);
    atomicAdd(dR + 3 * i + 1, gchg[4 * (size_t)k + 1]);
    atomicAdd(dR + 3 * i + 2, gchg[4 * (size_t)k + 2]);
    atomicAdd(dq + i, gchg[4 * (size_t)k + 3]);
}

cudaError_t launch_scatter_region(const int *rI_idx, int nI, const double *gchg, double *dq_int, double *dR_int,
                                  cudaStream_t st)
{
    if (nI <= 0) return cudaSuccess;
    k_scatter_region<<<(nI + 255) / 256, 256, 0, st>>>(rI_idx, nI, gchg, dq_int, dR_int);
    return cudaGetLastError();
}

}  // namespace qmmm
