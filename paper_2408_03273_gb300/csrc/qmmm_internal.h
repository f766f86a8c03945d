// qmmm_internal.h -- handle layout and kernel-launcher declarations of the GB300 library.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/qmmm.h"

namespace qmmm {

constexpr int MAX_SIGMA_CLASSES = 64;
constexpr int MAX_NPRIM = 16;
constexpr int CHUNK_F64 = 4096;  // region-I charges per V-forward launch (FP64: 32 B each)
constexpr int CHUNK_GRAD = 2560; // per adjoint launch (charge + per-charge accumulators)
constexpr int CHUNK_F32 = 4096;  // mixed path

// Per shell pair: shells (A, B) with l_A >= l_B, their AO offsets.
struct SPair { int shA, shB, aoA, aoB; };

// Everything a pp-tile kernel needs (device pointers).
struct BasisDev {
    const int *shell_atom, *shell_off, *shell_ao;
    const double *exps, *ncoef;
    const double *qm_xyz;   // natm*3
    const SPair *sp;
    const uint32_t *pp;     // packed (sp << 8) | (ka << 4) | kb, class-sorted
    int nao, natm;
};

struct RegionDev {
    const double4_32a *chg;         // region-I images (x, y, z, q), class-major
    const float4 *chg_hi;       // FP32 coordinates relative to the QM centre (hi part), w = q
    const float4 *chg_lo;       // lo parts (x, y, z), w = 0
    const int *idx;             // internal MM index of each image
    const int *cls_off;         // [ncls+1] class offsets in the list
    const double *cls_kappa;    // [ncls] exponent 1/sigma^2 (<= 0: point charge)
    int ncls;
    int n;
    const double *centre;       // [3] the QM centre, in device memory (read at run time, so a
                                // recorded graph sees the current geometry)
};

struct qmmm_handle_impl;

// launchers (defined in the .cu files); all return a cudaError_t of the last launch
// Region-I sweeps.  `nsm` caps the grid (the class's share of the SMs); `variant` picks the block
// shape: 0 = 256 threads, 1 = the class's wide block (sweep_wide_threads), where one exists;
// `nslice` splits the charge chunk over that many block rows (small systems), the V kernels then
// writing slice s into V + s * vstride.
// dst[k] = sum_s src[s*n + k], s < nslice, in order (the V slices)
cudaError_t launch_sum_slices_d(const double *src, int nslice, size_t n, double *dst, cudaStream_t st);
cudaError_t launch_vpot_f64(const BasisDev &b, const RegionDev &r, int cls, int pp_begin, int pp_end,
                            int ch_begin, int ch_end, const double *boys, double *V, int *err, int nsm, int variant,
                            int nslice, size_t vstride, cudaStream_t st);
cudaError_t launch_vpot_f32(const BasisDev &b, const RegionDev &r, int cls, int pp_begin, int pp_end,
                            int ch_begin, int ch_end, const float *boys, double *V, int *err, int nsm, int variant,
                            int nslice, size_t vstride, cudaStream_t st);
// One frame's share of a class's mixed V sweep: its basis, region I and V, the primitive pairs
// [pp_begin, pp_end) and region-I charges [ch_begin, ch_end) in ns slices of gx blocks each, its
// blocks [blk0, blk0 + gx ns) of a batched launch.
struct VJob {
    BasisDev bd;
    RegionDev rg;
    double *V;
    int pp_begin, pp_end, ch_begin, ch_end;
    int gx, ns, blk0;
};
// The mixed V sweep of class cls over njob frames in one launch of nblk blocks, every block adding
// into its frame's V; maxch: the most charges of one slice (<= CHUNK_F32).
cudaError_t launch_vpot_f32_jobs(int cls, const VJob *jobs, int njob, int nblk, int maxch, const float *boys,
                                 int *err, int variant, cudaStream_t st);
cudaError_t launch_vgrad_f64(const BasisDev &b, const RegionDev &r, int cls, int pp_begin, int pp_end,
                             int ch_begin, int ch_end, const double *boys, const double *dm, double *gqm,
                             double *gchg /* n*4: dC xyz, dq */, int *err, int nsm, int variant, int nslice,
                             cudaStream_t st);
// Scratch of one class's charge-lane adjoint sweep (mixed path): pair
// records (cl_rec_floats(L) floats per primitive pair) and per-pair charge sums (6 doubles).
struct ClScratch {
    float4 *rec = nullptr;
    double *psum = nullptr;
};
cudaError_t launch_vgrad_f32(const BasisDev &b, const RegionDev &r, int cls, int pp_begin, int pp_end,
                             int ch_begin, int ch_end, const float *boys, const double *dm, double *gqm,
                             double *gchg, int *err, int nsm, int variant, int nslice, ClScratch cl,
                             cudaStream_t st);
// One frame's share of a class's charge-lane adjoint: its basis, region I, density and outputs,
// the primitive pairs [pp_begin, pp_end) and region-I charges [ch_begin, ch_end), its work items
// (ntile charge tiles x gx ranges of pair batches, from cl_decompose) and where its items and
// threads start in the flat ranges of a batched launch (item0, thr0; thr0 a multiple of 32).
struct ClJob {
    BasisDev bd;
    RegionDev rg;
    const double *dm;
    float4 *rec;
    double *psum;
    double *gqm, *gchg;
    int pp_begin, pp_end, ch_begin, ch_end;
    int gx, ntile;
    int item0, thr0;
};
// work items of one class's charge-lane sweep: gx ranges of pair batches x ntile charge tiles
void cl_decompose(int L, int variant, int npair, int nch, int ncls, int &gx, int &ntile);
// The charge-lane adjoint of class cls over njob frames with one launch of each of its kernels
// (records, a persistent sweep over nitems items, pair gradients); jobs is a device array,
// counter a device int (cleared here).
cudaError_t launch_vgrad_cl_jobs(int cls, const ClJob *jobs, int njob, int nthr, int nitems, int *counter,
                                 const float *boys, int variant, int nsm, cudaStream_t st);

// moments / multipoles / Fock / Pulay (mode bits below)
enum { MOM_MULT = 1, MOM_FOCK = 2, MOM_PULAY = 4 };
// Mulliken octupoles: oct[natm*10] -= (accumulated; the caller zeroes it)
cudaError_t launch_octupoles(const BasisDev &b, int cls, int pp_begin, int pp_end, const double *dm, double *oct,
                             cudaStream_t st);
cudaError_t launch_moments(const BasisDev &b, int cls, int pp_begin, int pp_end, const double *dm,
                           const double *phi /* natm*20 */, double *mult /* natm*10 */, double *F,
                           double *gqm, int mode, cudaStream_t st);

// region I and Ewald
struct EwaldDev {
    const double *qm_xyz;       // natm*3
    const double *mm_xyz;       // nmm*3 (internal order)
    const double *mm_q;         // nmm
    const double *mm_beta;      // nmm: 1/sigma (0: point charge)
    const int *mm_cls;          // nmm: sigma class
    const float4 *mm_filt;      // nmm: FP32 position and squared pre-filter radius (real-space sums)
    const float4 *qm_filt;      // natm: FP32 position
    int natm, nmm;
    double box[3];
    double centre[3];
    double rcut;                // region-I radius
    double ewald_rc;
    double alpha;
    int img[3];                 // image search half-width beyond the minimum image
    const double4_32a *G;           // (Gx, Gy, Gz, 2 g(G)) half space
    int nG;
    int kmax[3];
};
// Octupole error estimate: err[k] for region-I radii r_lo + k dr, k < n (bins: n + 1 doubles)
cudaError_t launch_octupole_error(const EwaldDev &e, const double *oct, const double *phi, double r_lo, double dr,
                                  int n, double *bins, double *err, cudaStream_t st);
// QM-QM periodic images: pair tensors P[natm*natm*20] (scratch), energy E[1], image potentials
// u20[natm*20] (components 10..19 zero), gradient at fixed multipoles grad[natm*3]
cudaError_t launch_qm_images(const EwaldDev &e, const double *gfac, const double *mult, double *P, double *E,
                             double *u20, double *grad, cudaStream_t st);
cudaError_t launch_region1_count(const EwaldDev &e, int *blk_count, int *cls_count, int nblk, cudaStream_t st);
cudaError_t launch_region1_fill(const EwaldDev &e, const int *blk_off, double4_32a *chg, float4 *hi, float4 *lo,
                                int *idx, int nblk, cudaStream_t st);
cudaError_t launch_scan_blocks(int *blk_count, int nblk, cudaStream_t st);

// Tensor-core structure factor (recip_tc.cu): tile shape and scratch.
struct TcShape {
    int NL = 0, mtiles = 0, ntiles = 0, ntr = 0, nkb = 0;  // lines, line tiles, N tiles (rows each), charge blocks
    int nbmax = 0;           // blocks of the max|q| reduction
    size_t part_ints = 0;    // per-CTA accumulator partials, int32 words
    size_t phase_rows = 0;   // fixed-point phase entries (int4: re hi/lo, im hi/lo), whole charge blocks
    size_t bplane_words = 0; // digit planes of the B operand (32-bit words), in shared-memory layout
    bool staged = false;     // phase rows of each chunk staged in shared memory by TMA bulk copies
};
struct TcBuf {
    int4 *phase = nullptr;      // qX [npad][NX], Y [npad][NY], Z [npad][NZ] (2^61 fixed point, split)
    uint32_t *bpl = nullptr;    // B digit planes per (charge block, chunk, N tile)
    int *part = nullptr;
    double *bmax = nullptr;     // per-block max |q|
};
void tc_sf_shape(const EwaldDev &e, TcShape &sh);
// S (dense, as the FP64 kernel writes it) by BF16 tensor-core products of exact digit planes
cudaError_t launch_structure_factor_tc(const EwaldDev &e, const TcShape &sh, const TcBuf &b, double2 *S, int *err,
                                       cudaStream_t st);

// Tensor-core MM-side reciprocal sum (mmrecip_tc.cu): tiling and scratch.
// digit planes per operand of the MM-side tensor-core sum: 7 (48-bit fixed point) on the FP64
// path, 5 (34-bit, 15 plane pairs instead of 28) on the mixed path, whose error is set by its FP32
// region-I sweeps (about 1e-7 of the largest gradient; the 5-plane sum adds about 1e-8 at most)
constexpr int MMR_NP_FP64 = 7, MMR_NP_MIXED = 5;
struct MmrShape {
    int mtiles = 0, npad = 0, npair = 0, nchunk = 0;  // charge tiles (128), padded charges, (n_y, n_z) pairs, chunks of 8
    int cpt = 3, ntiles = 1, nr = 0, nstg = 3;        // channels per N tile, N tiles, N rows, stages
    int nr_last = 0;                                  // N rows of the last N tile (fewer channels)
    int nacc = 4;                                     // accumulators (exact levels + 1)
    int np = 7;                                       // digit planes per operand (5 or 7)
    bool supported = false;                           // kx small enough for one channel per tile
    size_t phase_rows = 0;                            // Y and Z phase rows (int4)
    size_t bplane_words = 0;                          // B digit planes of all N tiles (32-bit words)
};
struct MmrBuf {
    int4 *phase = nullptr;     // Yt [NY][npad], Zt [NZ][npad]
    uint32_t *bpl = nullptr;   // B planes per N tile and chunk
    double *cscale = nullptr;  // [3][NX] power-of-two row scales
};
void tc_mmr_shape(const EwaldDev &e, int nacc, int np, MmrShape &sh);
// dq[i] += sum_G Re[A e^{-iG.R_i}], dR[i] += q_i sum_G G Im[A e^{-iG.R_i}] (internal order), from the
// dense A and A_z = G_z A of k_multipole_sf, on the BF16 tensor cores (exact digit planes)
cudaError_t launch_mm_recip_tc(const EwaldDev &e, const MmrShape &sh, const MmrBuf &b, const double2 *A,
                               const double2 *Az, double *dq, double *dR, int *err, cudaStream_t st);

// Scratch of the Ewald kernels (device buffers owned by the handle).
struct EwaldBuf {
    double *gfac = nullptr;      // dense (kx+1)(2ky+1)(2kz+1): 2 g(G) on the half space, else 0
    double2 *S = nullptr;        // dense MM structure factor
    double2 *Spart = nullptr;    // per-slice partial structure factors
    int sf_nslice = 1;     // charge slices of the FP64 structure-factor grid
    int sf_nslice_df = 1;  // the same for the double-float kernel
    double *preal = nullptr;     // natm * real_nslice * 20
    int real_nslice = 1;
    double *precip = nullptr;    // natm * recip_nslice * 20 (reciprocal part per G slice)
    double2 *atom_ph = nullptr;  // natm * 3 * (2 * 56 + 1) phase rows of the QM atoms
    float4 *atom_phdf = nullptr; // the same rows as double-float (re.h, re.l, im.h, im.l), mixed path
    float4 *mm_filt = nullptr, *qm_filt = nullptr;  // written with the positions (EwaldDev copies)
    int recip_nslice = 1;
    double *pr1 = nullptr;       // natm * 20
    double2 *A = nullptr;        // dense multipole structure factor times 2 g(G)
    double2 *Az = nullptr;       // G_z times A
    float4 *Adf = nullptr;       // A and Az as double-float (re.h, re.l, im.h, im.l), mixed path
    float4 *gSdf = nullptr;      // 2 g(G) S(G) as double-float, mixed path (region-II potential)
    float4 *Azdf = nullptr;
    double *sums = nullptr;      // [0] sum q_MM, [1] sum Q_QM
    int recip = 0;               // reciprocal sums: 0 CUDA cores (FP64 / double-float), 1 tensor cores
    TcShape tcs;
    TcBuf tcb;
    MmrShape mms[2];             // MM-side sum: [0] FP64 path (7 planes, 5 accumulators: levels 0-3
                                 // exact), [1] mixed path (5 planes, 3: levels 0-1 exact, 2-4 merged)
    MmrBuf mmb;
    int *err = nullptr;          // device error word of the handle
};
int ewald_dense_size(const EwaldDev &e);
int ewald_sf_nslice(const EwaldDev &e, int nsm, bool df);
int ewald_real_nslice(const EwaldDev &e, int nsm);
int ewald_recip_nslice(const EwaldDev &e, int nsm);
cudaError_t launch_gfac(const EwaldDev &e, double *gfac, cudaStream_t st);
// v_j,c (natm*20) at the current geometry
// df: double-float reciprocal sums (mixed-precision path) instead of FP64
cudaError_t launch_ewald_phi(const EwaldDev &e, const double4_32a *rI, int nI, const EwaldBuf &w, double *phi,
                             bool df, cudaStream_t st);
// MM-side adjoint of the multipole energy and the QM tensor gradient:
//   dq_int[nmm] +=, dR_int[nmm*3] += (internal order), gchg[nI*4] += (region-I T part), gqm[natm*3] +=
cudaError_t launch_ewald_mm(const EwaldDev &e, const double4_32a *rI, int nI, const double *mult, const double *phi,
                            const EwaldBuf &w, double *dq_int, double *dR_int, double *gchg, double *gqm, bool df,
                            cudaStream_t st);
// region-I nuclear-MM term: Epart[nblk] partial energies (nblk = ceil(nI/256)); optional gradients
int enucmm_nblk(int nI);
cudaError_t launch_enucmm(const double *qm_xyz, const double *Z, int natm, const double4_32a *rI, const int *rI_idx,
                          int nI, const double *mm_beta, double *Epart, double *gqm, double *gchg, int want_grad,
                          cudaStream_t st);
cudaError_t launch_scatter_region(const int *rI_idx, int nI, const double *gchg, double *dq_int, double *dR_int,
                                  cudaStream_t st);
// out4 = {total, E_I = sum dm V (if have_V), E_nuc (sum of Epart), E_II = sum w M v}; partials: scratch[npart]
cudaError_t launch_energy_terms(const double *dm, const double *V, int nao, int have_V, const double *mult,
                                const double *phi, int natm, const double *Epart, int nEpart, double *partials,
                                int npart, double *out4, cudaStream_t st);
cudaError_t launch_gather_mm(const double *xyz_user, const double *q_user, const int *perm, int nmm, double *xyz,
                             double *q, cudaStream_t st);
cudaError_t launch_unpermute(const double *dq_int, const double *dR_int, const int *perm, int nmm, double *dq,
                             double *dR, cudaStream_t st);
cudaError_t launch_sum(const double *x, int n, double *out, cudaStream_t st);  // out[0] = sum x (one block)
cudaError_t launch_sum_strided(const double *x, int n, int stride, double *out, cudaStream_t st);

// record the detail message returned by qmmm_last_error()
void set_last_error(const std::string &msg);

}  // namespace qmmm
