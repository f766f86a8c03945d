// api.cu -- host planner and the C ABI of include/qmmm.h.
//
// Planner (qmmm_create): normalise the contracted Cartesian basis, build the shell-pair list
// (l_A >= l_B) sorted by angular class and screened at the primitive-pair level by
// |c_a c_b| K_AB (pi/p)^{3/2}, order the MM charges by Gaussian width and spatial cell (so
// region-I images come out grouped by width, which lets the kernels hoist
// sqrt(kappa/(p+kappa)) out of the charge loop), tabulate the Boys function for the FP64 and
// FP32 kernels, and write the reciprocal prefactors 2 g(G) = 2 (4 pi/V) exp(-G^2/4 alpha^2)/G^2.
// Per geometry (qmmm_set_positions): region I by an order-preserving device compaction, then the
// region-II potential v (20 components per QM atom).  All arithmetic on the path runs in the
// kernels; the host only plans, copies and launches.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <memory>
#include <string>
#include <vector>

#include "device_common.cuh"
#include "pp_tile.cuh"
#include "qmmm_internal.h"
#include "sched.h"

using namespace qmmm;

namespace {

thread_local std::string g_last_error;

int fail(int code, const std::string &msg)
{
    g_last_error = msg;
    return code;
}

}  // namespace

void qmmm::set_last_error(const std::string &msg) { g_last_error = msg; }

namespace {

#define CUDA_TRY(call)                                                                          \
    do {                                                                                        \
        cudaError_t _e = (call);                                                                \
        if (_e != cudaSuccess)                                                                  \
            return fail(QMMM_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(_e));    \
    } while (0)

template <typename T>
struct DBuf {
    T *p = nullptr;
    size_t n = 0;
    int ensure(size_t count)
    {
        if (count <= n && p) return QMMM_OK;
        if (p) cudaFree(p);
        p = nullptr;
        n = 0;
        size_t c = count ? count : 1;
        if (cudaMalloc((void **)&p, c * sizeof(T)) != cudaSuccess) {
            cudaGetLastError();
            return fail(QMMM_ERR_ALLOC, "cudaMalloc failed");
        }
        n = c;
        return QMMM_OK;
    }
    void release()
    {
        if (p) cudaFree(p);
        p = nullptr;
        n = 0;
    }
};

bool is_device_ptr(const void *ptr)
{
    if (!ptr) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

double dfact_odd(int n)  // (2n-1)!!
{
    double r = 1.0;
    for (int k = 2 * n - 1; k > 1; k -= 2) r *= k;
    return r;
}

// Boys table: F_m(T_k) for m = 0..nm-1 by the convergent series of the highest order (all terms
// positive) followed by the stable downward recursion, in long double; last column e^{-T_k}.
void boys_table(int nrow, int ncol, double step, std::vector<double> &out)
{
    out.assign((size_t)nrow * ncol, 0.0);
    const int mtop = ncol - 2;
    for (int k = 0; k < nrow; ++k) {
        const long double T = (long double)k * step;
        const long double eT = expl(-T);
        long double term = 1.0L / (2 * mtop + 1), sum = term;
        for (int i = 1; i < 4000; ++i) {
            term *= 2.0L * T / (2 * mtop + 2 * i + 1);
            sum += term;
            if (term < 1e-22L * sum) break;
        }
        std::vector<long double> F(mtop + 1);
        F[mtop] = eT * sum;
        for (int m = mtop; m > 0; --m) F[m - 1] = (2.0L * T * F[m] + eT) / (2 * m - 1);
        for (int m = 0; m <= mtop; ++m) out[(size_t)k * ncol + m] = (double)F[m];
        out[(size_t)k * ncol + ncol - 1] = (double)eT;
    }
}

// Size estimate of a primitive pair's charge distribution g_a g_b used for screening:
// |c_a c_b| K_AB (pi/p)^{3/2} (|PA| + p^{-1/2})^{l_a} (|PB| + p^{-1/2})^{l_b}; the polynomial
// factor bounds (x-A)^i (x-B)^j over the bulk of the product Gaussian.
double pair_bound(double a, double b, double ca, double cb, double ab2, int la, int lb)
{
    const double p = a + b, r = 1.0 / std::sqrt(p), ab = std::sqrt(ab2);
    const double pa = b / p * ab + r, pb = a / p * ab + r;
    return std::fabs(ca * cb) * std::exp(-a * b / p * ab2) * std::pow(PI / p, 1.5) * std::pow(pa, la) * std::pow(pb, lb);
}

// The largest pair_bound over every distance in [|AB| - 2 margin, |AB| + 2 margin]: the Gaussian
// factor at the shortest distance, the polynomial factors at the longest.  A pair kept by this
// bound stays kept while no QM atom moves farther than `margin` from where the list was planned.
double pair_bound_margin(double a, double b, double ca, double cb, double ab2, int la, int lb, double margin)
{
    const double p = a + b, r = 1.0 / std::sqrt(p), ab = std::sqrt(ab2);
    const double lo = std::max(0.0, ab - 2.0 * margin), hi = ab + 2.0 * margin;
    const double pa = b / p * hi + r, pb = a / p * hi + r;
    return std::fabs(ca * cb) * std::exp(-a * b / p * lo * lo) * std::pow(PI / p, 1.5) * std::pow(pa, la) *
           std::pow(pb, lb);
}

// QM displacement (bohr) the screened pair list tolerates before it is planned again
constexpr double SCREEN_MARGIN = 0.1;

}  // namespace

struct qmmm_handle {
    int device = 0, nsm = 152;
    cudaStream_t stream = nullptr;
    int natm = 0, nshell = 0, nprim = 0, nmm = 0, nao = 0;
    int precision = QMMM_FP64;
    int recip_mode = QMMM_RECIP_AUTO;  // structure-factor method requested (see select_recip)
    double box[3] = {0, 0, 0}, cutoff = 0, alpha = 0, ewald_rc = 0;
    int kmax[3] = {0, 0, 0};
    double screen_tol = 1e-14;
    double centre[3] = {0, 0, 0};
    // host copies
    std::vector<double> Z, qm_xyz, exps, ncoef;
    std::vector<int> shell_atom, shell_l, shell_nprim, shell_off, shell_ao;
    std::vector<int> perm;  // internal MM index -> user index
    std::vector<double> cls_kappa;
    int ncls = 0;
    long long n_sp = 0, n_pp = 0;
    int class_off[NCLASS + 1] = {0};
    std::vector<double> screen_xyz;  // QM positions the pair list was screened at
    long long plan_gen = 0;          // incremented whenever the pair list is planned again
    long long sp_class[NCLASS] = {0};
    int nI = 0;
    std::vector<int> cls_off_I;
    bool V_valid = false;
    float t_sweep = 0.f, t_other = 0.f;
    bool quiet = false;  // inside a batch graph capture: no host synchronisation, no timing events
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
    cudaStream_t side[NCLASS] = {};   // one stream per angular class (concurrent class sweeps)
    cudaEvent_t fork = nullptr, join[NCLASS] = {};
    // the moment kernels' class streams (fork_classes), apart from the sweeps' so that the two can
    // run at the same time, and a stream that only records the end of a sweep for its timing
    cudaStream_t mside[NCLASS] = {}, tstream = nullptr;
    cudaEvent_t mfork = nullptr, mjoin[NCLASS] = {};
    // region-I sweep configuration per kernel kind (SweepKind) and angular class: SM-time weight
    // per primitive pair (flop model, or measured by qmmm_autotune), block variant, measured time
    double cls_cost[SW_NKIND][NCLASS] = {};
    int cls_variant[SW_NKIND][NCLASS] = {};
    double cls_ms[SW_NKIND][NCLASS] = {};
    int tuned_mask = 0, tuned_nI = 0;
    DBuf<double> tune_V, tune_dm, tune_gqm, tune_gchg;  // autotuner scratch
    DBuf<double> oct, oct_bins, oct_err;                  // octupole error estimate
    DBuf<double> qmq_P, qmq_u, qmq_g, qmq_E, qmq_F;       // QM-QM periodic images
    DBuf<double> Vslices;                                 // per-slice partial V (small systems)
    EwaldBuf ew;
    int nblk_mm = 1;

    // device buffers
    DBuf<double> qm, Zd, dexps, dncoef, mm_xyz, mm_q, mm_beta, user_xyz, user_q;
    DBuf<int> dshell_atom, dshell_off, dshell_ao, dperm, mm_cls, blk, cls_count, rI_idx, dcls_off;
    DBuf<SPair> sp;
    DBuf<uint32_t> pp;
    DBuf<double4_32a> rI;
    DBuf<float4> rI_hi, rI_lo;
    DBuf<double> dcls_kappa, gfac, preal, precip, pr1, sums, phi, boys64, V, dm, F, mult, mult_init, gqm, gchg, dq_int,
        dR_int, dq_out, dR_out, Epart, partials, out4;
    DBuf<float> boys32;
    DBuf<double> centre_d;  // [3] QM centre for the kernels
    DBuf<double2> S, Spart, A, Az, atom_ph;
    DBuf<float4> Adf, Azdf, gSdf, atom_phdf, mm_filt, qm_filt;
    DBuf<int> err;
    DBuf<int4> tc_phase;  // tensor-core structure factor scratch (allocated on first use)
    DBuf<uint32_t> tc_bpl;
    DBuf<int> tc_part;
    DBuf<double> tc_bmax;
    DBuf<int4> mmr_phase;  // tensor-core MM-side reciprocal sum scratch
    DBuf<uint32_t> mmr_bpl;
    DBuf<double> mmr_cscale;
    // charge-lane adjoint sweep (mixed path): pair records and per-pair charge sums, one region
    // per class (classes run concurrently)
    DBuf<float4> cl_rec;
    DBuf<double> cl_psum;
    size_t cl_rec_off[NCLASS] = {}, cl_psum_off[NCLASS] = {};

    BasisDev basis() const
    {
        BasisDev b;
        b.shell_atom = dshell_atom.p;
        b.shell_off = dshell_off.p;
        b.shell_ao = dshell_ao.p;
        b.exps = dexps.p;
        b.ncoef = dncoef.p;
        b.qm_xyz = qm.p;
        b.sp = sp.p;
        b.pp = pp.p;
        b.nao = nao;
        b.natm = natm;
        return b;
    }
    RegionDev region() const
    {
        RegionDev r;
        r.chg = rI.p;
        r.chg_hi = rI_hi.p;
        r.chg_lo = rI_lo.p;
        r.idx = rI_idx.p;
        r.cls_off = dcls_off.p;
        r.cls_kappa = dcls_kappa.p;
        r.ncls = ncls;
        r.n = nI;
        r.centre = centre_d.p;
        return r;
    }
    EwaldDev ewald() const
    {
        EwaldDev e;
        e.qm_xyz = qm.p;
        e.mm_xyz = mm_xyz.p;
        e.mm_q = mm_q.p;
        e.mm_beta = mm_beta.p;
        e.mm_cls = mm_cls.p;
        e.mm_filt = mm_filt.p;
        e.qm_filt = qm_filt.p;
        e.natm = natm;
        e.nmm = nmm;
        for (int x = 0; x < 3; ++x) {
            e.box[x] = box[x];
            e.centre[x] = centre[x];
            e.kmax[x] = kmax[x];
            // images beyond the minimum image are needed only when a cutoff exceeds half the box
            const double rmax = std::max(ewald_rc, 9.0 * max_sigma);
            e.img[x] = rmax > 0.5 * box[x] ? (int)std::ceil(rmax / box[x] - 0.5) : 0;
        }
        e.rcut = cutoff;
        e.ewald_rc = ewald_rc;
        e.alpha = alpha;
        e.G = nullptr;
        e.nG = ewald_dense_size(e);
        return e;
    }
    double max_sigma = 0.0;

    ~qmmm_handle()
    {
        for (auto &e : ev)
            if (e) cudaEventDestroy(e);
        for (int c = 0; c < NCLASS; ++c) {
            if (side[c]) cudaStreamDestroy(side[c]);
            if (join[c]) cudaEventDestroy(join[c]);
            if (mside[c]) cudaStreamDestroy(mside[c]);
            if (mjoin[c]) cudaEventDestroy(mjoin[c]);
        }
        if (fork) cudaEventDestroy(fork);
        if (mfork) cudaEventDestroy(mfork);
        if (tstream) cudaStreamDestroy(tstream);
        qm.release(); Zd.release(); dexps.release(); dncoef.release(); mm_xyz.release(); mm_q.release();
        mm_beta.release(); user_xyz.release(); user_q.release(); dshell_atom.release(); dshell_off.release();
        dshell_ao.release(); dperm.release(); mm_cls.release(); blk.release(); cls_count.release();
        rI_idx.release(); dcls_off.release(); sp.release(); pp.release(); rI.release(); rI_hi.release();
        rI_lo.release(); dcls_kappa.release(); gfac.release(); preal.release(); precip.release(); pr1.release(); sums.release();
        phi.release(); boys64.release(); V.release(); dm.release(); F.release(); mult.release();
        mult_init.release(); gqm.release(); gchg.release(); dq_int.release(); dR_int.release();
        dq_out.release(); dR_out.release(); Epart.release(); partials.release(); out4.release();
        boys32.release(); S.release(); Spart.release(); A.release(); Az.release(); atom_ph.release(); err.release();
        tc_phase.release(); tc_bpl.release(); tc_part.release(); tc_bmax.release();
        mmr_phase.release(); mmr_bpl.release(); mmr_cscale.release();
        Adf.release(); Azdf.release(); gSdf.release(); atom_phdf.release(); mm_filt.release(); qm_filt.release();
        tune_V.release(); tune_dm.release(); tune_gqm.release(); tune_gchg.release();
        oct.release(); oct_bins.release(); oct_err.release();
        qmq_P.release(); qmq_u.release(); qmq_g.release(); qmq_E.release(); qmq_F.release();
        Vslices.release(); centre_d.release(); cl_rec.release(); cl_psum.release();
    }
};

namespace {

constexpr int NPART = 256;

void reset_tuning(qmmm_handle *h, int kind);

int check_device_errors(qmmm_handle *h)
{
    CUDA_TRY(cudaStreamSynchronize(h->stream));
    CUDA_TRY(cudaGetLastError());
    int e = 0;
    CUDA_TRY(cudaMemcpy(&e, h->err.p, sizeof(int), cudaMemcpyDeviceToHost));
    if (e) {
        CUDA_TRY(cudaMemset(h->err.p, 0, sizeof(int)));
        if (e & DEVERR_TIMEOUT) return fail(QMMM_ERR_TIMEOUT, "a bounded device wait ran out");
        return fail(QMMM_ERR_CUDA, "device bounds check failed");
    }
    return QMMM_OK;
}

// Timing mark k of the current call (skipped while a batch graph is being captured).
cudaError_t mark(qmmm_handle *h, int k) { return h->quiet ? cudaSuccess : cudaEventRecord(h->ev[k], h->stream); }

// End of a call: wait for the device, check its error flag and read the `nmarks` timing marks
// (3: sweep = mark 0..1, rest = 1..2; 4: sweep = mark 0..1 with mark 1 on the timing stream after
// the class streams, rest = the span 3..2 less the sweep; 2: everything = 0..1).  Inside a batch
// capture nothing waits: the batch checks every frame after the graph has run.
int finish(qmmm_handle *h, int nmarks)
{
    if (h->quiet) return QMMM_OK;
    const int rc = check_device_errors(h);
    if (rc) return rc;
    if (nmarks == 3) {
        cudaEventElapsedTime(&h->t_sweep, h->ev[0], h->ev[1]);
        cudaEventElapsedTime(&h->t_other, h->ev[1], h->ev[2]);
    } else if (nmarks == 4) {
        float all = 0.f;
        cudaEventElapsedTime(&h->t_sweep, h->ev[0], h->ev[1]);
        cudaEventElapsedTime(&all, h->ev[3], h->ev[2]);
        h->t_other = all - h->t_sweep;
    } else if (nmarks == 2) {
        h->t_sweep = 0.f;
        cudaEventElapsedTime(&h->t_other, h->ev[0], h->ev[1]);
    }
    return QMMM_OK;
}

// copy an input array to a device buffer unless it already lives on the device
int stage_input(qmmm_handle *h, const double *src, size_t n, DBuf<double> &buf, const double **out)
{
    if (is_device_ptr(src)) {
        *out = src;
        return QMMM_OK;
    }
    int rc = buf.ensure(n);
    if (rc) return rc;
    CUDA_TRY(cudaMemcpyAsync(buf.p, src, n * sizeof(double), cudaMemcpyHostToDevice, h->stream));
    *out = buf.p;
    return QMMM_OK;
}

int copy_out(qmmm_handle *h, double *dst, const double *src, size_t n)
{
    if (!dst) return QMMM_OK;
    CUDA_TRY(cudaMemcpyAsync(dst, src, n * sizeof(double), cudaMemcpyDefault, h->stream));
    return QMMM_OK;
}

// The reciprocal-sum method in effect; allocates the tensor-core scratch the first time it is
// needed.  QMMM_RECIP_AUTO: the tensor cores once the reciprocal work is large enough to outweigh
// the five extra launches of each tensor-core sum (the CUDA-core kernels win below ~4e7 dense G
// entries x charges: on the 645-charge water workload, 1.2e6, by 0.14 ms per mixed step).
constexpr double RECIP_TC_MIN_WORK = 4e7;
int select_recip(qmmm_handle *h)
{
    int m = h->recip_mode;
    if (m == QMMM_RECIP_AUTO) {
        const double work = (double)ewald_dense_size(h->ewald()) * (double)h->nmm;
        m = work >= RECIP_TC_MIN_WORK ? QMMM_RECIP_TENSOR : QMMM_RECIP_CUDA_CORES;
    }
    if (m == QMMM_RECIP_TENSOR && !h->tc_part.p) {
        const TcShape &sh = h->ew.tcs;
        int rc;
        if ((rc = h->tc_phase.ensure(sh.phase_rows)) || (rc = h->tc_bpl.ensure(sh.bplane_words)) ||
            (rc = h->tc_part.ensure(sh.part_ints)) || (rc = h->tc_bmax.ensure(sh.nbmax)))
            return rc;
        // the padding beyond the last charge is copied but never used; keep it defined
        CUDA_TRY(cudaMemset(h->tc_phase.p, 0, sh.phase_rows * sizeof(int4)));
        h->ew.tcb.phase = h->tc_phase.p;
        h->ew.tcb.bpl = h->tc_bpl.p;
        h->ew.tcb.part = h->tc_part.p;
        h->ew.tcb.bmax = h->tc_bmax.p;
        const MmrShape &m0 = h->ew.mms[0], &m1 = h->ew.mms[1];
        if (m0.supported || m1.supported) {
            if ((rc = h->mmr_phase.ensure(m0.phase_rows)) ||
                (rc = h->mmr_bpl.ensure(std::max(m0.bplane_words, m1.bplane_words))) ||
                (rc = h->mmr_cscale.ensure(3 * (h->kmax[0] + 1))))
                return rc;
            // the rows of padding charges are copied but never used; keep them defined
            CUDA_TRY(cudaMemset(h->mmr_phase.p, 0, m0.phase_rows * sizeof(int4)));
            h->ew.mmb.phase = h->mmr_phase.p;
            h->ew.mmb.bpl = h->mmr_bpl.p;
            h->ew.mmb.cscale = h->mmr_cscale.p;
        }
    }
    h->ew.recip = m;
    return QMMM_OK;
}

// Shell pairs (l_A >= l_B) sorted by angular class, primitive pairs screened (R16, with the
// margin of pair_bound_margin), uploaded; the QM positions used are kept so that
// qmmm_set_positions plans again once a QM atom has moved farther than SCREEN_MARGIN.
int plan_pairs(qmmm_handle *h)
{
    const int nshell = h->nshell;
    std::vector<std::vector<SPair>> sp_cls(NCLASS);
    std::vector<std::vector<uint32_t>> pp_cls(NCLASS);
    auto ab2_of = [&](int i, int j) {
        const double *A = &h->qm_xyz[3 * h->shell_atom[i]], *B = &h->qm_xyz[3 * h->shell_atom[j]];
        return (A[0] - B[0]) * (A[0] - B[0]) + (A[1] - B[1]) * (A[1] - B[1]) + (A[2] - B[2]) * (A[2] - B[2]);
    };
    // pass 1: largest screening value
    double vmax = 0.0;
    for (int i = 0; i < nshell; ++i)
        for (int j = i; j < nshell; ++j) {
            const double ab2 = ab2_of(i, j);
            for (int ka = 0; ka < h->shell_nprim[i]; ++ka)
                for (int kb = 0; kb < h->shell_nprim[j]; ++kb) {
                    const double a = h->exps[h->shell_off[i] + ka], b = h->exps[h->shell_off[j] + kb];
                    const double v = pair_bound(a, b, h->ncoef[h->shell_off[i] + ka], h->ncoef[h->shell_off[j] + kb],
                                                ab2, h->shell_l[i], h->shell_l[j]);
                    vmax = std::max(vmax, v);
                }
        }
    // pass 2: the pairs kept, with the displacement margin
    const double thr = h->screen_tol * vmax;
    long long nsp = 0;
    for (int i = 0; i < nshell; ++i)
        for (int j = i; j < nshell; ++j) {
            int sA = i, sB = j;
            if (h->shell_l[j] > h->shell_l[i]) std::swap(sA, sB);
            const int cls = class_of(h->shell_l[sA], h->shell_l[sB]);
            const double ab2 = ab2_of(sA, sB);
            std::vector<uint32_t> kept;
            for (int ka = 0; ka < h->shell_nprim[sA]; ++ka)
                for (int kb = 0; kb < h->shell_nprim[sB]; ++kb) {
                    const double a = h->exps[h->shell_off[sA] + ka], b = h->exps[h->shell_off[sB] + kb];
                    const double v = pair_bound_margin(a, b, h->ncoef[h->shell_off[sA] + ka],
                                                       h->ncoef[h->shell_off[sB] + kb], ab2, h->shell_l[sA],
                                                       h->shell_l[sB], SCREEN_MARGIN);
                    if (h->screen_tol == 0.0 || v >= thr) kept.push_back((uint32_t)((ka << 4) | kb));
                }
            if (kept.empty()) continue;
            const int sidx = (int)sp_cls[cls].size();
            sp_cls[cls].push_back(SPair{sA, sB, h->shell_ao[sA], h->shell_ao[sB]});
            for (uint32_t c : kept) pp_cls[cls].push_back(((uint32_t)sidx << 8) | c);  // re-based below
            ++nsp;
        }
    if (nsp >= (1LL << 24)) return fail(QMMM_ERR_ARG, "too many shell pairs (>= 2^24)");
    std::vector<SPair> sp_all;
    std::vector<uint32_t> pp_all;
    h->class_off[0] = 0;
    for (int c = 0; c < NCLASS; ++c) {
        const uint32_t base = (uint32_t)sp_all.size();
        for (const SPair &sp : sp_cls[c]) sp_all.push_back(sp);
        for (uint32_t code : pp_cls[c]) pp_all.push_back(((((code >> 8) + base)) << 8) | (code & 0xff));
        h->class_off[c + 1] = (int)pp_all.size();
        h->sp_class[c] = (long long)sp_cls[c].size();
    }
    h->n_sp = (long long)sp_all.size();
    h->n_pp = (long long)pp_all.size();
    int rc;
    if ((rc = h->sp.ensure(std::max<size_t>(sp_all.size(), 1))) || (rc = h->pp.ensure(std::max<size_t>(pp_all.size(), 1))))
        return rc;
    if (!sp_all.empty())
        CUDA_TRY(cudaMemcpy(h->sp.p, sp_all.data(), sp_all.size() * sizeof(SPair), cudaMemcpyHostToDevice));
    if (!pp_all.empty())
        CUDA_TRY(cudaMemcpy(h->pp.p, pp_all.data(), pp_all.size() * sizeof(uint32_t), cudaMemcpyHostToDevice));
    h->screen_xyz = h->qm_xyz;
    ++h->plan_gen;
    h->V_valid = false;
    return QMMM_OK;
}

// Plan the pair list again if a QM atom moved farther than SCREEN_MARGIN since it was planned.
int replan_if_moved(qmmm_handle *h)
{
    if (h->screen_tol == 0.0 || h->screen_xyz.size() != h->qm_xyz.size()) return QMMM_OK;
    double d2max = 0.0;
    for (int j = 0; j < h->natm; ++j) {
        double d2 = 0.0;
        for (int x = 0; x < 3; ++x) {
            const double d = h->qm_xyz[3 * j + x] - h->screen_xyz[3 * j + x];
            d2 += d * d;
        }
        d2max = std::max(d2max, d2);
    }
    if (d2max <= SCREEN_MARGIN * SCREEN_MARGIN) return QMMM_OK;
    CUDA_TRY(cudaStreamSynchronize(h->stream));  // kernels in flight may still read the old list
    return plan_pairs(h);
}

int run_positions(qmmm_handle *h, const double *qm_xyz, const double *mm_xyz, const double *mm_q)
{
    cudaStream_t st = h->stream;
    // QM positions: host copy (centre) and device copy
    if (qm_xyz) {
        if (is_device_ptr(qm_xyz)) {
            CUDA_TRY(cudaMemcpyAsync(h->qm.p, qm_xyz, 3 * h->natm * sizeof(double), cudaMemcpyDeviceToDevice, st));
            CUDA_TRY(cudaMemcpyAsync(h->qm_xyz.data(), qm_xyz, 3 * h->natm * sizeof(double), cudaMemcpyDeviceToHost, st));
            CUDA_TRY(cudaStreamSynchronize(st));
        } else {
            std::memcpy(h->qm_xyz.data(), qm_xyz, 3 * h->natm * sizeof(double));
            CUDA_TRY(cudaMemcpyAsync(h->qm.p, h->qm_xyz.data(), 3 * h->natm * sizeof(double), cudaMemcpyHostToDevice, st));
        }
    }
    if (qm_xyz) {
        int rc = replan_if_moved(h);
        if (rc) return rc;
    }
    for (int x = 0; x < 3; ++x) {
        double c = 0.0;
        for (int j = 0; j < h->natm; ++j) c += h->qm_xyz[3 * j + x];
        h->centre[x] = c / h->natm;
    }
    {
        int rc;
        if ((rc = h->centre_d.ensure(3))) return rc;
        CUDA_TRY(cudaMemcpyAsync(h->centre_d.p, h->centre, 3 * sizeof(double), cudaMemcpyHostToDevice, st));
    }
    // MM positions/charges: user order -> internal order
    if (h->nmm > 0 && (mm_xyz || mm_q)) {
        const double *ux = nullptr, *uq = nullptr;
        int rc;
        if (mm_xyz && (rc = stage_input(h, mm_xyz, 3 * (size_t)h->nmm, h->user_xyz, &ux))) return rc;
        if (mm_q && (rc = stage_input(h, mm_q, (size_t)h->nmm, h->user_q, &uq))) return rc;
        CUDA_TRY(launch_gather_mm(ux, uq, h->dperm.p, h->nmm, h->mm_xyz.p, h->mm_q.p, st));
    }
    EwaldDev e = h->ewald();
    // region I: count, scan, fill (order preserving, grouped by width class)
    h->nI = 0;
    if (h->nmm > 0) {
        CUDA_TRY(cudaMemsetAsync(h->cls_count.p, 0, h->ncls * sizeof(int), st));
        CUDA_TRY(launch_region1_count(e, h->blk.p, h->cls_count.p, h->nblk_mm, st));
        CUDA_TRY(launch_scan_blocks(h->blk.p, h->nblk_mm, st));
        std::vector<int> cnt(h->ncls + 1);
        CUDA_TRY(cudaMemcpyAsync(cnt.data(), h->blk.p + h->nblk_mm, sizeof(int), cudaMemcpyDeviceToHost, st));
        CUDA_TRY(cudaMemcpyAsync(cnt.data() + 1, h->cls_count.p, h->ncls * sizeof(int), cudaMemcpyDeviceToHost, st));
        CUDA_TRY(cudaStreamSynchronize(st));
        h->nI = cnt[0];
        // a tuned sweep configuration holds while region I keeps roughly its size
        if (h->tuned_mask && 4 * (long long)std::abs(h->nI - h->tuned_nI) > h->tuned_nI)
            for (int k = 0; k < SW_NKIND; ++k) reset_tuning(h, k);
        h->cls_off_I.assign(h->ncls + 1, 0);
        for (int c = 0; c < h->ncls; ++c) h->cls_off_I[c + 1] = h->cls_off_I[c] + cnt[1 + c];
        if (h->cls_off_I[h->ncls] != h->nI) return fail(QMMM_ERR_CUDA, "region-I class counts inconsistent");
        int rc;
        if ((rc = h->rI.ensure(h->nI)) || (rc = h->rI_hi.ensure(h->nI)) || (rc = h->rI_lo.ensure(h->nI)) ||
            (rc = h->rI_idx.ensure(h->nI)) || (rc = h->gchg.ensure(4 * (size_t)std::max(h->nI, 1))) ||
            (rc = h->Epart.ensure(enucmm_nblk(h->nI))))
            return rc;
        CUDA_TRY(cudaMemcpyAsync(h->dcls_off.p, h->cls_off_I.data(), (h->ncls + 1) * sizeof(int),
                                 cudaMemcpyHostToDevice, st));
        if (h->nI > 0)
            CUDA_TRY(launch_region1_fill(e, h->blk.p, h->rI.p, h->rI_hi.p, h->rI_lo.p, h->rI_idx.p, h->nblk_mm, st));
    } else {
        h->cls_off_I.assign(h->ncls + 1, 0);
    }
    // region-II potential at the QM sites
    {
        int rc = select_recip(h);
        if (rc) return rc;
    }
    CUDA_TRY(launch_ewald_phi(e, h->rI.p, h->nI, h->ew, h->phi.p, h->precision == QMMM_MIXED, st));
    h->V_valid = false;
    return check_device_errors(h);
}

bool kind_is_grad(int kind) { return kind == SW_VGRAD_F64 || kind == SW_VGRAD_F32; }
bool kind_is_mixed(int kind) { return kind == SW_VPOT_F32 || kind == SW_VGRAD_F32; }

// Region-I charges per sweep launch (what one block stages into shared memory).
int chunk_for_kind(int kind)
{
    if (kind_is_grad(kind)) return CHUNK_GRAD;
    return kind_is_mixed(kind) ? CHUNK_F32 : CHUNK_F64;
}

// Work per (primitive pair, charge) of a class with L = l_A + l_B: the flop model that splits the
// SMs between the concurrent class sweeps until qmmm_autotune measures the real costs.
double class_weight(int L, bool grad)
{
    auto c4 = [](int n) { return n >= 4 ? (double)n * (n - 1) * (n - 2) * (n - 3) / 24.0 : 0.0; };
    auto c3 = [](int n) { return n >= 3 ? (double)n * (n - 1) * (n - 2) / 6.0 : 0.0; };
    return grad ? 75 + 3 * L + 2 * c4(L + 5) + 14 * c3(L + 3) : 40 + 3 * L + 2 * c4(L + 4) + 2 * c3(L + 3);
}

int sweep_kind(const qmmm_handle *h, bool grad)
{
    const bool mixed = h->precision == QMMM_MIXED;
    return grad ? (mixed ? SW_VGRAD_F32 : SW_VGRAD_F64) : (mixed ? SW_VPOT_F32 : SW_VPOT_F64);
}

void reset_tuning(qmmm_handle *h, int kind)
{
    for (int c = 0; c < NCLASS; ++c) {
        h->cls_cost[kind][c] = class_weight(la_of_class(c) + lb_of_class(c), kind_is_grad(kind));
        h->cls_variant[kind][c] = 0;
        h->cls_ms[kind][c] = 0.0;
    }
    h->tuned_mask &= ~(1 << kind);
}

int variant_threads(int kind, int cls, int variant)
{
    const int w = sweep_wide_threads(kind, cls);
    return (variant == 1 && w > 0) ? w : 256;
}

// Blocks a class sweep can fill with one charge slice: one 32-pair tile per warp.
int tile_cap(const qmmm_handle *h, int kind, int cls, int variant)
{
    const int npp = h->class_off[cls + 1] - h->class_off[cls];
    const int nwarp = variant_threads(kind, cls, variant) / 32;
    return std::max(1, ((npp + 31) / 32 + nwarp - 1) / nwarp);
}

// Grid caps of the concurrent class sweeps: shares of the SMs in proportion to each class's
// SM-time (primitive pairs x cost), but never more blocks than the class has warps' worth of
// 32-pair tiles for (times maxsl, when a class may split its charges over maxsl block rows);
// what a capped class cannot use goes to the others.  Returns false when no class has work.
bool split_sms(const qmmm_handle *h, int kind, const int *variant, int *share, int maxsl = 1)
{
    double w[NCLASS];
    int cap[NCLASS];
    bool open[NCLASS];
    int nopen = 0;
    for (int c = 0; c < NCLASS; ++c) {
        const int npp = h->class_off[c + 1] - h->class_off[c];
        open[c] = npp > 0;
        cap[c] = 0;
        w[c] = 0.0;
        if (!open[c]) continue;
        cap[c] = tile_cap(h, kind, c, variant[c]) * maxsl;
        w[c] = npp * std::max(h->cls_cost[kind][c], 1e-30);
        ++nopen;
    }
    if (!nopen) {
        for (int c = 0; c < NCLASS; ++c) share[c] = 0;
        return false;
    }
    split_shares(NCLASS, w, cap, open, h->nsm, share);
    return true;
}

// Launch the sweep of every non-empty angular class concurrently: each class on its own stream,
// forked from and joined back into the handle's stream, its grid capped at its share of the SMs
// (so small classes do not leave most SMs idle while they run alone).  With maxsl > 1 (sweeps
// over nch charges; V sweeps then write slice s of a class into partial matrix s) every class
// picks its own charge slices (class_slices), and a class with fewer tiles than its share of the
// SMs may take up to maxsl times its tile count in blocks.
template <typename F>
int run_classes(qmmm_handle *h, int kind, F launch, int nslice = 1, int maxsl = 1, int nch = 0, bool join = true)
{
    int share[NCLASS];
    if (!split_sms(h, kind, h->cls_variant[kind], share, nslice == 1 ? maxsl : 1)) return QMMM_OK;
    CUDA_TRY(cudaEventRecord(h->fork, h->stream));
    // the charge-lane sweeps (mixed adjoint) size their own fine-grained grids and are launched
    // highest class first (their blocks are the longest), so that the short low-l blocks fill the tail
    const bool cl = kind == SW_VGRAD_F32;
    for (int i = 0; i < NCLASS; ++i) {
        const int c = cl ? NCLASS - 1 - i : i;
        const int p0 = h->class_off[c], p1 = h->class_off[c + 1];
        if (p1 <= p0) continue;
        int sh = share[c], ns = nslice;
        if (nslice == 1 && maxsl > 1) {
            const int nwarp = variant_threads(kind, c, h->cls_variant[kind][c]) / 32;
            // per-pair setup in charges of sweep work: FP64 Hermite/density setup against an FP64
            // charge loop (~1%), or against an FP32 one (several percent)
            const double setup = kind_is_mixed(kind) ? 64.0 : 16.0;
            class_slices((p1 - p0 + 31) / 32, nwarp, sh, nch, maxsl, setup, &sh, &ns);
        }
        CUDA_TRY(cudaStreamWaitEvent(h->side[c], h->fork, 0));
        CUDA_TRY(launch(c, p0, p1, sh, h->cls_variant[kind][c], ns, h->side[c]));
        CUDA_TRY(cudaEventRecord(h->join[c], h->side[c]));
    }
    if (join)
        for (int c = 0; c < NCLASS; ++c)
            if (h->class_off[c + 1] > h->class_off[c]) CUDA_TRY(cudaStreamWaitEvent(h->stream, h->join[c], 0));
    return QMMM_OK;
}

// Make `s` wait for every class sweep launched by run_classes(..., join = false).
int join_classes(qmmm_handle *h, cudaStream_t s)
{
    for (int c = 0; c < NCLASS; ++c)
        if (h->class_off[c + 1] > h->class_off[c]) CUDA_TRY(cudaStreamWaitEvent(s, h->join[c], 0));
    return QMMM_OK;
}

// One kernel per non-empty angular class, all classes concurrently on the moment kernels' class
// streams (forked from and joined back into the handle's stream), each with its full grid.
template <typename F>
int fork_classes(qmmm_handle *h, F launch)
{
    CUDA_TRY(cudaEventRecord(h->mfork, h->stream));
    for (int c = 0; c < NCLASS; ++c) {
        const int p0 = h->class_off[c], p1 = h->class_off[c + 1];
        if (p1 <= p0) continue;
        CUDA_TRY(cudaStreamWaitEvent(h->mside[c], h->mfork, 0));
        CUDA_TRY(launch(c, p0, p1, h->mside[c]));
        CUDA_TRY(cudaEventRecord(h->mjoin[c], h->mside[c]));
    }
    for (int c = 0; c < NCLASS; ++c)
        if (h->class_off[c + 1] > h->class_off[c]) CUDA_TRY(cudaStreamWaitEvent(h->stream, h->mjoin[c], 0));
    return QMMM_OK;
}

// Charge slices of a sweep: when the classes together ask for fewer than half the SMs (a small
// QM region: few 32-pair tiles), the charge chunk is split over up to 8 block rows so that the
// work spreads over more SMs (at least 64 charges per slice).
int sweep_slices(const qmmm_handle *h, int kind, int nch)
{
    int share[NCLASS];
    if (!split_sms(h, kind, h->cls_variant[kind], share)) return 1;
    int blocks = 0;
    for (int c = 0; c < NCLASS; ++c) blocks += share[c];
    int ns = blocks > 0 ? h->nsm / blocks : 1;
    ns = std::min(ns, std::min(8, nch / 64));
    return std::max(ns, 1);
}

// One class sweep of the given kind over region-I charges [c0, c1), split into nslice block rows;
// V kernels write slice s into V + s * vstride.
// Scratch of the charge-lane adjoint sweep for every class that takes it (allocated on first use).
int ensure_cl(qmmm_handle *h)
{
    size_t nrec = 0, nps = 0;
    for (int c = 0; c < NCLASS; ++c) {
        const int L = la_of_class(c) + lb_of_class(c);
        const size_t npp = (size_t)(h->class_off[c + 1] - h->class_off[c]);
        h->cl_rec_off[c] = nrec;
        h->cl_psum_off[c] = nps;
        nrec += npp * (cl_rec_floats(L) / 4);
        nps += npp * 6;
    }
    int rc;
    if ((rc = h->cl_rec.ensure(std::max<size_t>(nrec, 1))) || (rc = h->cl_psum.ensure(std::max<size_t>(nps, 1))))
        return rc;
    return QMMM_OK;
}

cudaError_t launch_sweep(const qmmm_handle *h, int kind, int cls, int p0, int p1, int c0, int c1, int share,
                         int variant, int nslice, size_t vstride, const double *ddm, double *V, double *gqm,
                         double *gchg, cudaStream_t cs)
{
    const BasisDev b = h->basis();
    const RegionDev r = h->region();
    switch (kind) {
    case SW_VPOT_F64:
        return launch_vpot_f64(b, r, cls, p0, p1, c0, c1, h->boys64.p, V, h->err.p, share, variant, nslice, vstride,
                               cs);
    case SW_VPOT_F32:
        return launch_vpot_f32(b, r, cls, p0, p1, c0, c1, h->boys32.p, V, h->err.p, share, variant, nslice, vstride,
                               cs);
    case SW_VGRAD_F64:
        return launch_vgrad_f64(b, r, cls, p0, p1, c0, c1, h->boys64.p, ddm, gqm, gchg, h->err.p, share, variant,
                                nslice, cs);
    case SW_VGRAD_F32: {
        ClScratch cl;
        if (h->cl_rec.p && h->cl_psum.p) {
            cl.rec = h->cl_rec.p + h->cl_rec_off[cls];
            cl.psum = h->cl_psum.p + h->cl_psum_off[cls];
        }
        return launch_vgrad_f32(b, r, cls, p0, p1, c0, c1, h->boys32.p, ddm, gqm, gchg, h->err.p, share, variant,
                                nslice, cl, cs);
    }
    default: return cudaErrorInvalidValue;
    }
}

// Charges per autotuner timing run: the class kernels sweep every staged charge per pair, so
// their times scale with the count; a few hundred keep tuning short and the ratios intact.
constexpr int TUNE_CHARGES = 512;

// Best of three timed runs after a warm-up, on the handle's stream.
template <typename F>
int time_best(qmmm_handle *h, cudaEvent_t e0, cudaEvent_t e1, F run, float *ms)
{
    float best = 1e30f;
    for (int rep = 0; rep < 4; ++rep) {
        CUDA_TRY(cudaEventRecord(e0, h->stream));
        const int rc = run();
        if (rc) return rc;
        CUDA_TRY(cudaEventRecord(e1, h->stream));
        CUDA_TRY(cudaEventSynchronize(e1));
        float t = 0.f;
        CUDA_TRY(cudaEventElapsedTime(&t, e0, e1));
        if (rep > 0) best = std::min(best, t);
    }
    *ms = best;
    return check_device_errors(h);
}

// The class sweeps of one kind, alone (cls >= 0) or all concurrently (cls < 0), over the first
// charges of region I, in the autotuner's scratch buffers.
int tune_launch(qmmm_handle *h, int kind, int cls, int share, int variant)
{
    const int c1 = std::min(h->nI, std::min(chunk_for_kind(kind), TUNE_CHARGES));
    auto one = [&](int c, int p0, int p1, int s, int v, int ns, cudaStream_t cs) {
        return launch_sweep(h, kind, c, p0, p1, 0, c1, s, v, ns, 0, h->tune_dm.p, h->tune_V.p, h->tune_gqm.p,
                            h->tune_gchg.p, cs);
    };
    if (cls < 0) {
        // the slices of the real sweep (V slices all add into the one scratch matrix here)
        const int maxsl = kind_is_grad(kind) ? std::max(1, std::min(8, c1 / 128))
                                             : vpot_max_slices(c1, (size_t)h->nao * h->nao);
        return run_classes(h, kind, one, 1, maxsl, c1);
    }
    CUDA_TRY(one(cls, h->class_off[cls], h->class_off[cls + 1], share, variant, 1, h->stream));
    return QMMM_OK;
}

// Tune one sweep kind: two rounds of timing every class alone, in each block variant, at its
// current share; the SM-time (time x blocks) per primitive pair becomes the class's cost, which
// sets the next shares.  The result is kept only if the concurrent sweep beats the model's.
int tune_kind(qmmm_handle *h, int kind, cudaEvent_t e0, cudaEvent_t e1)
{
    reset_tuning(h, kind);
    int share[NCLASS];
    if (!split_sms(h, kind, h->cls_variant[kind], share)) return QMMM_OK;
    int rc;
    float t_model = 0.f, t_tuned = 0.f;
    if ((rc = time_best(h, e0, e1, [&] { return tune_launch(h, kind, -1, 0, 0); }, &t_model))) return rc;
    double ms[NCLASS] = {}, ms0[NCLASS] = {}, cost0[NCLASS] = {};
    for (int round = 0; round < 2; ++round) {
        split_sms(h, kind, h->cls_variant[kind], share);
        double cost[NCLASS];
        int var[NCLASS];
        for (int c = 0; c < NCLASS; ++c) {
            cost[c] = cost0[c] = h->cls_cost[kind][c];
            var[c] = h->cls_variant[kind][c];
            const int npp = h->class_off[c + 1] - h->class_off[c];
            if (npp <= 0) continue;
            double best = 1e300;
            const int nvar = sweep_wide_threads(kind, c) > 0 ? 2 : 1;
            for (int v = 0; v < nvar; ++v) {
                float t = 0.f;
                if ((rc = time_best(h, e0, e1, [&] { return tune_launch(h, kind, c, share[c], v); }, &t))) return rc;
                // SM-time with every warp equally loaded: the kernel ran ceil(tiles / warps)
                // tile passes, so its time per pass times tiles / warps per block is the class's
                // work free of the tile quantisation, which the per-class charge slices remove
                const int nwarp = variant_threads(kind, c, v) / 32, tiles = (npp + 31) / 32;
                const int blocks = std::min(share[c], (tiles + nwarp - 1) / nwarp);
                const int passes = (tiles + blocks * nwarp - 1) / (blocks * nwarp);
                double smt = (double)t / passes * tiles / nwarp;
                // the charge-lane sweep runs its fine-grained grid on the whole GPU: SM-time
                if (kind == SW_VGRAD_F32) smt = (double)t * h->nsm;
                if (v == 0) {
                    cost0[c] = smt / npp;
                    ms0[c] = t;
                }
                if (smt < best) {
                    best = smt;
                    var[c] = v;
                    ms[c] = t;
                }
            }
            cost[c] = best / npp;
        }
        for (int c = 0; c < NCLASS; ++c) {
            h->cls_cost[kind][c] = cost[c];
            h->cls_variant[kind][c] = var[c];
        }
    }
    if ((rc = time_best(h, e0, e1, [&] { return tune_launch(h, kind, -1, 0, 0); }, &t_tuned))) return rc;
    // A wide block that wins alone can lose in the concurrent sweep (its lower register cap
    // spills, and the spill traffic of all classes meets in L2): also try the measured split with
    // 256-thread blocks only, and keep the fastest of the three schedules.
    double tc[NCLASS];
    int tv[NCLASS];
    for (int c = 0; c < NCLASS; ++c) {
        tc[c] = h->cls_cost[kind][c];
        tv[c] = h->cls_variant[kind][c];
        h->cls_cost[kind][c] = cost0[c];
        h->cls_variant[kind][c] = 0;
    }
    float t_narrow = 0.f;
    if ((rc = time_best(h, e0, e1, [&] { return tune_launch(h, kind, -1, 0, 0); }, &t_narrow))) return rc;
    if (t_narrow < t_model && t_narrow <= t_tuned) {
        for (int c = 0; c < NCLASS; ++c) h->cls_ms[kind][c] = ms0[c];
        h->tuned_mask |= 1 << kind;
    } else if (t_tuned < t_model) {
        for (int c = 0; c < NCLASS; ++c) {
            h->cls_cost[kind][c] = tc[c];
            h->cls_variant[kind][c] = tv[c];
            h->cls_ms[kind][c] = ms[c];
        }
        h->tuned_mask |= 1 << kind;
    } else {
        reset_tuning(h, kind);
    }
    return QMMM_OK;
}

}  // namespace

extern "C" {

const char *qmmm_strerror(int code)
{
    switch (code) {
    case QMMM_OK: return "ok";
    case QMMM_ERR_ARG: return "invalid argument";
    case QMMM_ERR_ALLOC: return "allocation failed";
    case QMMM_ERR_CUDA: return "CUDA error";
    case QMMM_ERR_TIMEOUT: return "bounded device wait timed out";
    case QMMM_ERR_UNSUPPORTED_L: return "unsupported shell (l > 3 or more than 16 primitives)";
    case QMMM_ERR_STATE: return "call order violated";
    default: return "unknown error";
    }
}

const char *qmmm_last_error(void) { return g_last_error.c_str(); }

int qmmm_create(const qmmm_atom *atoms, int natm, const qmmm_shell *shells, int nshell, const qmmm_primitive *prims,
                int nprim, const qmmm_charge *charges, int nmm, const double box[3], double cutoff,
                double ewald_alpha, const qmmm_options *opts, qmmm_handle **out)
{
    if (!out) return fail(QMMM_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (!atoms || natm <= 0 || !shells || nshell <= 0 || !prims || nprim <= 0 || nmm < 0 || (nmm > 0 && !charges) ||
        !box)
        return fail(QMMM_ERR_ARG, "null array or non-positive size");
    if (!(box[0] > 0 && box[1] > 0 && box[2] > 0) || !(cutoff > 0) || !(ewald_alpha > 0))
        return fail(QMMM_ERR_ARG, "box, cutoff and ewald_alpha must be positive");
    if (opts && opts->full_cell_test) return fail(QMMM_ERR_ARG, "full_cell_test is reserved");
    if (opts && opts->region_mode != 0) return fail(QMMM_ERR_ARG, "only region_mode 0 (sphere) is supported");
    if (opts && opts->precision != QMMM_FP64 && opts->precision != QMMM_MIXED)
        return fail(QMMM_ERR_ARG, "precision must be QMMM_FP64 or QMMM_MIXED");

    // host-side validation first: no CUDA call happens for invalid input
    for (int s = 0; s < nshell; ++s) {
        const qmmm_shell &sh = shells[s];
        if (sh.l < 0 || sh.l > LMAX || sh.nprim < 1 || sh.nprim > MAX_NPRIM)
            return fail(QMMM_ERR_UNSUPPORTED_L, "shell " + std::to_string(s) + ": l or nprim out of range");
        if (sh.atom < 0 || sh.atom >= natm || sh.prim_offset < 0 || sh.prim_offset + sh.nprim > nprim)
            return fail(QMMM_ERR_ARG, "shell " + std::to_string(s) + ": atom or primitive range invalid");
    }
    for (int k = 0; k < nprim; ++k)
        if (!(prims[k].exponent > 0) || !std::isfinite(prims[k].exponent) || !std::isfinite(prims[k].coeff))
            return fail(QMMM_ERR_ARG, "primitive " + std::to_string(k) + ": exponent must be positive and finite");
    for (int j = 0; j < natm; ++j)
        if (!std::isfinite(atoms[j].xyz[0]) || !std::isfinite(atoms[j].xyz[1]) || !std::isfinite(atoms[j].xyz[2]) ||
            !std::isfinite(atoms[j].Z))
            return fail(QMMM_ERR_ARG, "QM atom " + std::to_string(j) + ": non-finite data");
    for (int i = 0; i < nmm; ++i)
        if (!std::isfinite(charges[i].xyz[0]) || !std::isfinite(charges[i].xyz[1]) || !std::isfinite(charges[i].xyz[2]) ||
            !std::isfinite(charges[i].q) || !std::isfinite(charges[i].sigma))
            return fail(QMMM_ERR_ARG, "MM charge " + std::to_string(i) + ": non-finite data");
    {
        std::map<double, int> w;
        for (int i = 0; i < nmm && (int)w.size() <= MAX_SIGMA_CLASSES; ++i)
            w.emplace(charges[i].sigma > 0 ? charges[i].sigma : 0.0, 0);
        if ((int)w.size() > MAX_SIGMA_CLASSES) return fail(QMMM_ERR_ARG, "more than 64 distinct Gaussian widths");
    }
    for (int x = 0; x < 3; ++x)
        if (opts && opts->kmax[x] > 56) return fail(QMMM_ERR_ARG, "kmax too large (> 56)");

    auto h = new qmmm_handle();
    std::unique_ptr<qmmm_handle> guard(h);
    CUDA_TRY(cudaGetDevice(&h->device));
    CUDA_TRY(cudaDeviceGetAttribute(&h->nsm, cudaDevAttrMultiProcessorCount, h->device));
    h->natm = natm;
    h->nshell = nshell;
    h->nprim = nprim;
    h->nmm = nmm;
    for (int x = 0; x < 3; ++x) h->box[x] = box[x];
    h->cutoff = cutoff;
    h->alpha = ewald_alpha;
    h->precision = opts ? opts->precision : QMMM_FP64;
    h->screen_tol = (opts && opts->screen_tol >= 0) ? opts->screen_tol : 1e-14;
    h->ewald_rc = (opts && opts->ewald_rcut > 0) ? opts->ewald_rcut : cutoff;
    for (int x = 0; x < 3; ++x) {
        int k = opts ? opts->kmax[x] : 0;
        if (k <= 0) {
            // exp(-G^2 / 4 alpha^2) < 1e-8 at the cube edge
            const double gmax = 2.0 * ewald_alpha * std::sqrt(std::log(1e8));
            k = (int)std::ceil(gmax * box[x] / (2.0 * PI));
        }
        if (k > 56) return fail(QMMM_ERR_ARG, "kmax too large (> 56)");
        h->kmax[x] = k;
    }

    // QM atoms and basis
    h->Z.resize(natm);
    h->qm_xyz.resize(3 * natm);
    for (int j = 0; j < natm; ++j) {
        h->Z[j] = atoms[j].Z;
        for (int x = 0; x < 3; ++x) h->qm_xyz[3 * j + x] = atoms[j].xyz[x];
    }
    h->shell_atom.resize(nshell);
    h->shell_l.resize(nshell);
    h->shell_nprim.resize(nshell);
    h->shell_off.resize(nshell);
    h->shell_ao.resize(nshell);
    int ao = 0;
    for (int s = 0; s < nshell; ++s) {
        const qmmm_shell &sh = shells[s];
        if (sh.l < 0 || sh.l > LMAX || sh.nprim < 1 || sh.nprim > MAX_NPRIM)
            return fail(QMMM_ERR_UNSUPPORTED_L, "shell " + std::to_string(s) + ": l or nprim out of range");
        if (sh.atom < 0 || sh.atom >= natm || sh.prim_offset < 0 || sh.prim_offset + sh.nprim > nprim)
            return fail(QMMM_ERR_ARG, "shell " + std::to_string(s) + ": atom or primitive range invalid");
        h->shell_atom[s] = sh.atom;
        h->shell_l[s] = sh.l;
        h->shell_nprim[s] = sh.nprim;
        h->shell_off[s] = sh.prim_offset;
        h->shell_ao[s] = ao;
        ao += ncart(sh.l);
    }
    h->nao = ao;
    h->exps.resize(nprim);
    h->ncoef.assign(nprim, 0.0);
    for (int k = 0; k < nprim; ++k) {
        if (!(prims[k].exponent > 0) || !std::isfinite(prims[k].coeff))
            return fail(QMMM_ERR_ARG, "primitive " + std::to_string(k) + ": exponent must be positive");
        h->exps[k] = prims[k].exponent;
    }
    // normalisation: x^l component of each primitive, then the contraction
    for (int s = 0; s < nshell; ++s) {
        const int l = h->shell_l[s], o = h->shell_off[s], n = h->shell_nprim[s];
        for (int k = 0; k < n; ++k) {
            const double a = h->exps[o + k];
            h->ncoef[o + k] = prims[o + k].coeff * std::pow(2.0 * a / PI, 0.75) * std::pow(4.0 * a, 0.5 * l) /
                              std::sqrt(dfact_odd(l));
        }
        double ss = 0.0;
        for (int k = 0; k < n; ++k)
            for (int m = 0; m < n; ++m) {
                const double p = h->exps[o + k] + h->exps[o + m];
                ss += h->ncoef[o + k] * h->ncoef[o + m] * dfact_odd(l) / std::pow(2.0 * p, l) * std::pow(PI / p, 1.5);
            }
        if (!(ss > 0)) return fail(QMMM_ERR_ARG, "shell " + std::to_string(s) + " has zero norm");
        for (int k = 0; k < n; ++k) h->ncoef[o + k] /= std::sqrt(ss);
    }

    {
        int rc = plan_pairs(h);
        if (rc) return rc;
    }

    // MM charges: width classes, internal order by (class, cell)
    std::vector<double> sig(nmm), uq(nmm), ux(3 * (size_t)nmm);
    for (int i = 0; i < nmm; ++i) {
        sig[i] = charges[i].sigma > 0 ? charges[i].sigma : 0.0;
        uq[i] = charges[i].q;
        for (int x = 0; x < 3; ++x) ux[3 * (size_t)i + x] = charges[i].xyz[x];
        if (!std::isfinite(sig[i]) || !std::isfinite(uq[i])) return fail(QMMM_ERR_ARG, "non-finite MM charge data");
    }
    std::map<double, int> wcls;
    for (double s : sig) wcls.emplace(s, 0);
    if ((int)wcls.size() > MAX_SIGMA_CLASSES) return fail(QMMM_ERR_ARG, "more than 64 distinct Gaussian widths");
    {
        int c = 0;
        for (auto &kv : wcls) {
            kv.second = c++;
            h->cls_kappa.push_back(kv.first > 0 ? 1.0 / (kv.first * kv.first) : 0.0);
            h->max_sigma = std::max(h->max_sigma, kv.first);
        }
        h->ncls = c > 0 ? c : 1;
        if (h->cls_kappa.empty()) h->cls_kappa.push_back(0.0);
    }
    std::vector<int> cls_user(nmm);
    std::vector<long long> key(nmm);
    const double cell = 8.0 / 0.52917721092;  // 8 Angstrom bins
    int ncx[3];
    for (int x = 0; x < 3; ++x) ncx[x] = std::max(1, (int)(box[x] / cell));
    for (int i = 0; i < nmm; ++i) {
        cls_user[i] = wcls[sig[i]];
        long long cid = 0;
        for (int x = 0; x < 3; ++x) {
            double f = ux[3 * (size_t)i + x] / box[x];
            f -= std::floor(f);
            int b = std::min(ncx[x] - 1, (int)(f * ncx[x]));
            cid = cid * ncx[x] + b;
        }
        key[i] = (long long)cls_user[i] * (1LL << 40) + cid;
    }
    h->perm.resize(nmm);
    for (int i = 0; i < nmm; ++i) h->perm[i] = i;
    std::stable_sort(h->perm.begin(), h->perm.end(), [&](int a, int b) { return key[a] < key[b]; });
    std::vector<int> cls_int(nmm);
    std::vector<double> beta_int(nmm);
    for (int i = 0; i < nmm; ++i) {
        cls_int[i] = cls_user[h->perm[i]];
        beta_int[i] = sig[h->perm[i]] > 0 ? 1.0 / sig[h->perm[i]] : 0.0;
    }

    // allocations and uploads
    {
        int rc;
        const size_t nm = std::max(nmm, 1);
        h->nblk_mm = std::max(1, (nmm + 255) / 256);
        if ((rc = h->qm.ensure(3 * natm)) || (rc = h->Zd.ensure(natm)) || (rc = h->dexps.ensure(nprim)) ||
            (rc = h->dncoef.ensure(nprim)) || (rc = h->dshell_atom.ensure(nshell)) || (rc = h->dshell_off.ensure(nshell)) ||
            (rc = h->dshell_ao.ensure(nshell)) || (rc = h->mm_xyz.ensure(3 * nm)) || (rc = h->mm_q.ensure(nm)) ||
            (rc = h->mm_beta.ensure(nm)) || (rc = h->mm_cls.ensure(nm)) || (rc = h->dperm.ensure(nm)) ||
            (rc = h->blk.ensure(h->nblk_mm + 1)) || (rc = h->cls_count.ensure(h->ncls)) ||
            (rc = h->dcls_off.ensure(h->ncls + 1)) || (rc = h->dcls_kappa.ensure(h->ncls)) ||
            (rc = h->phi.ensure(20 * (size_t)natm)) || (rc = h->mult.ensure(10 * (size_t)natm)) ||
            (rc = h->mult_init.ensure(10 * (size_t)natm)) || (rc = h->gqm.ensure(3 * (size_t)natm)) ||
            (rc = h->dq_int.ensure(nm)) || (rc = h->dR_int.ensure(3 * nm)) || (rc = h->dq_out.ensure(nm)) ||
            (rc = h->dR_out.ensure(3 * nm)) || (rc = h->partials.ensure(NPART)) || (rc = h->out4.ensure(8)) ||
            (rc = h->err.ensure(1)) || (rc = h->sums.ensure(2)) || (rc = h->Epart.ensure(1)) ||
            (rc = h->rI.ensure(1)) || (rc = h->rI_hi.ensure(1)) || (rc = h->rI_lo.ensure(1)) ||
            (rc = h->rI_idx.ensure(1)) || (rc = h->gchg.ensure(4)) || (rc = h->mm_filt.ensure(nm)) ||
            (rc = h->qm_filt.ensure((size_t)std::max(natm, 1))))
            return rc;
        CUDA_TRY(cudaMemset(h->err.p, 0, sizeof(int)));
        CUDA_TRY(cudaMemcpy(h->Zd.p, h->Z.data(), natm * sizeof(double), cudaMemcpyHostToDevice));
        CUDA_TRY(cudaMemcpy(h->dexps.p, h->exps.data(), nprim * sizeof(double), cudaMemcpyHostToDevice));
        CUDA_TRY(cudaMemcpy(h->dncoef.p, h->ncoef.data(), nprim * sizeof(double), cudaMemcpyHostToDevice));
        CUDA_TRY(cudaMemcpy(h->dshell_atom.p, h->shell_atom.data(), nshell * sizeof(int), cudaMemcpyHostToDevice));
        CUDA_TRY(cudaMemcpy(h->dshell_off.p, h->shell_off.data(), nshell * sizeof(int), cudaMemcpyHostToDevice));
        CUDA_TRY(cudaMemcpy(h->dshell_ao.p, h->shell_ao.data(), nshell * sizeof(int), cudaMemcpyHostToDevice));
        if (nmm > 0) {
            CUDA_TRY(cudaMemcpy(h->dperm.p, h->perm.data(), nmm * sizeof(int), cudaMemcpyHostToDevice));
            CUDA_TRY(cudaMemcpy(h->mm_cls.p, cls_int.data(), nmm * sizeof(int), cudaMemcpyHostToDevice));
            CUDA_TRY(cudaMemcpy(h->mm_beta.p, beta_int.data(), nmm * sizeof(double), cudaMemcpyHostToDevice));
        }
        CUDA_TRY(cudaMemcpy(h->dcls_kappa.p, h->cls_kappa.data(), h->ncls * sizeof(double), cudaMemcpyHostToDevice));
        std::vector<double> minit(10 * (size_t)natm, 0.0);
        for (int j = 0; j < natm; ++j) minit[10 * j] = h->Z[j];
        CUDA_TRY(cudaMemcpy(h->mult_init.p, minit.data(), minit.size() * sizeof(double), cudaMemcpyHostToDevice));
        // Boys tables
        std::vector<double> raw, t64((size_t)BOYS_MAXM * BOYS_NROW_D * BOYS_ROW_D);
        boys_table(BOYS_NROW_D, BOYS_NCOL_D, BOYS_STEP, raw);
        // one table per order M: F_{M+j}(T_k) / j!, j = 0..6, then e^{-T_k}
        for (int M = 0; M < BOYS_MAXM; ++M)
            for (int k = 0; k < BOYS_NROW_D; ++k) {
                double *row = &t64[((size_t)M * BOYS_NROW_D + k) * BOYS_ROW_D];
                double fact = 1.0;
                for (int j = 0; j < BOYS_TAYLOR_D; ++j) {
                    if (j > 0) fact *= j;
                    row[j] = raw[(size_t)k * BOYS_NCOL_D + M + j] / fact;
                }
                row[BOYS_ROW_D - 1] = raw[(size_t)k * BOYS_NCOL_D + BOYS_NCOL_D - 1];
            }
        if ((rc = h->boys64.ensure(t64.size()))) return rc;
        CUDA_TRY(cudaMemcpy(h->boys64.p, t64.data(), t64.size() * sizeof(double), cudaMemcpyHostToDevice));
        std::vector<double> t32d;
        boys_table(BOYS_NROW_F, BOYS_NCOL_F, BOYS_STEP_F, t32d);
        // one table per order M: F_{M+j}(T_k) / j!, j = 0..4, then e^{-T_k}
        std::vector<float> t32((size_t)BOYS_MAXM * BOYS_TAB_F, 0.0f);
        for (int M = 0; M < BOYS_MAXM; ++M)
            for (int k = 0; k < BOYS_NROW_F; ++k) {
                float *row = &t32[(size_t)M * BOYS_TAB_F + (size_t)k * BOYS_ROW_F];
                double fact = 1.0;
                for (int j = 0; j < BOYS_TAYLOR_F; ++j) {
                    if (j > 0) fact *= j;
                    row[j] = (float)(t32d[(size_t)k * BOYS_NCOL_F + M + j] / fact);
                }
                row[BOYS_TAYLOR_F] = (float)t32d[(size_t)k * BOYS_NCOL_F + BOYS_NCOL_F - 1];
            }
        if ((rc = h->boys32.ensure(t32.size()))) return rc;
        CUDA_TRY(cudaMemcpy(h->boys32.p, t32.data(), t32.size() * sizeof(float), cudaMemcpyHostToDevice));
        // Ewald buffers
        EwaldDev e = h->ewald();
        const int nd = ewald_dense_size(e);
        h->ew.sf_nslice = ewald_sf_nslice(e, h->nsm, false);
        h->ew.sf_nslice_df = ewald_sf_nslice(e, h->nsm, true);
        h->ew.real_nslice = ewald_real_nslice(e, h->nsm);
        h->ew.recip_nslice = ewald_recip_nslice(e, h->nsm);
        if ((rc = h->gfac.ensure(nd)) || (rc = h->S.ensure(nd)) || (rc = h->A.ensure(nd)) || (rc = h->Az.ensure(nd)) ||
            (rc = h->Adf.ensure(nd)) || (rc = h->Azdf.ensure(nd)) || (rc = h->gSdf.ensure(nd)) ||
            (rc = h->Spart.ensure((size_t)nd * std::max(h->ew.sf_nslice, h->ew.sf_nslice_df))) ||
            (rc = h->preal.ensure((size_t)natm * h->ew.real_nslice * 20)) ||
            (rc = h->precip.ensure((size_t)natm * h->ew.recip_nslice * 20)) || (rc = h->pr1.ensure(20 * (size_t)natm)) ||
            (rc = h->atom_ph.ensure((size_t)natm * 3 * (2 * 56 + 1))) ||
            (rc = h->atom_phdf.ensure((size_t)natm * 3 * (2 * 56 + 1))))
            return rc;
        h->ew.gfac = h->gfac.p;
        h->ew.S = h->S.p;
        h->ew.Spart = h->Spart.p;
        h->ew.preal = h->preal.p;
        h->ew.precip = h->precip.p;
        h->ew.atom_ph = h->atom_ph.p;
        h->ew.atom_phdf = h->atom_phdf.p;
        h->ew.mm_filt = h->mm_filt.p;
        h->ew.qm_filt = h->qm_filt.p;
        h->ew.pr1 = h->pr1.p;
        h->ew.A = h->A.p;
        h->ew.Az = h->Az.p;
        h->ew.Adf = h->Adf.p;
        h->ew.gSdf = h->gSdf.p;
        h->ew.Azdf = h->Azdf.p;
        h->ew.sums = h->sums.p;
        h->ew.err = h->err.p;
        tc_sf_shape(e, h->ew.tcs);
        tc_mmr_shape(e, 5, MMR_NP_FP64, h->ew.mms[0]);
        tc_mmr_shape(e, 3, MMR_NP_MIXED, h->ew.mms[1]);
        CUDA_TRY(launch_gfac(e, h->gfac.p, nullptr));
        for (int k = 0; k < 4; ++k) CUDA_TRY(cudaEventCreate(&h->ev[k]));
        CUDA_TRY(cudaEventCreateWithFlags(&h->fork, cudaEventDisableTiming));
        CUDA_TRY(cudaEventCreateWithFlags(&h->mfork, cudaEventDisableTiming));
        CUDA_TRY(cudaStreamCreateWithFlags(&h->tstream, cudaStreamNonBlocking));
        for (int c = 0; c < NCLASS; ++c) {
            CUDA_TRY(cudaStreamCreateWithFlags(&h->side[c], cudaStreamNonBlocking));
            CUDA_TRY(cudaEventCreateWithFlags(&h->join[c], cudaEventDisableTiming));
            CUDA_TRY(cudaStreamCreateWithFlags(&h->mside[c], cudaStreamNonBlocking));
            CUDA_TRY(cudaEventCreateWithFlags(&h->mjoin[c], cudaEventDisableTiming));
        }
    }
    for (int k = 0; k < SW_NKIND; ++k) reset_tuning(h, k);
    // initial geometry
    std::vector<double> qm0 = h->qm_xyz;
    int rc = run_positions(h, qm0.data(), nmm ? ux.data() : nullptr, nmm ? uq.data() : nullptr);
    if (rc) return rc;
    *out = guard.release();
    return QMMM_OK;
}

int qmmm_set_stream(qmmm_handle *h, void *stream)
{
    if (!h) return fail(QMMM_ERR_ARG, "null handle");
    h->stream = (cudaStream_t)stream;
    return QMMM_OK;
}

int qmmm_set_precision(qmmm_handle *h, int precision)
{
    if (!h) return fail(QMMM_ERR_ARG, "null handle");
    if (precision != QMMM_FP64 && precision != QMMM_MIXED) return fail(QMMM_ERR_ARG, "bad precision");
    if (precision != h->precision) h->V_valid = false;
    h->precision = precision;
    return QMMM_OK;
}

int qmmm_set_recip_method(qmmm_handle *h, int method)
{
    if (!h) return fail(QMMM_ERR_ARG, "null handle");
    if (method != QMMM_RECIP_CUDA_CORES && method != QMMM_RECIP_TENSOR && method != QMMM_RECIP_AUTO)
        return fail(QMMM_ERR_ARG, "bad method");
    const int before = h->ew.recip;
    h->recip_mode = method;
    int rc = select_recip(h);
    if (rc) return rc;
    if (h->ew.recip == before) return QMMM_OK;
    // the region-II potential at the current geometry, by the selected method
    CUDA_TRY(launch_ewald_phi(h->ewald(), h->rI.p, h->nI, h->ew, h->phi.p, h->precision == QMMM_MIXED, h->stream));
    h->V_valid = false;
    return check_device_errors(h);
}

int qmmm_set_positions(qmmm_handle *h, const double *qm_xyz, const double *mm_xyz, const double *mm_q)
{
    if (!h) return fail(QMMM_ERR_ARG, "null handle");
    return run_positions(h, qm_xyz, mm_xyz, mm_q);
}

// qmmm_vpot in parts (a batch runs the mixed V sweeps of all its frames together):
// vpot_prep clears V, or the per-slice partial matrices when slices is set (then *Vdst points at
// them and *nbuf is their count); vpot_sweep runs the class sweeps; vpot_end sums the slices, adds
// the nuclear-MM energy and copies out.
static int vpot_prep(qmmm_handle *h, bool slices, double **Vdst, int *nbuf)
{
    cudaStream_t st = h->stream;
    int rc;
    const size_t n2 = (size_t)h->nao * h->nao;
    if ((rc = h->V.ensure(n2))) return rc;
    CUDA_TRY(cudaMemsetAsync(h->V.p, 0, n2 * sizeof(double), st));
    *Vdst = h->V.p;
    *nbuf = 1;
    if (!slices) return QMMM_OK;
    const int kind = sweep_kind(h, false), ch = chunk_for_kind(kind);
    const int ns = sweep_slices(h, kind, std::min(h->nI, ch));
    // otherwise per-class charge slices (class_slices), as many as the per-slice partial
    // matrices' memory allows
    const int maxsl = ns > 1 ? 1 : vpot_max_slices(std::min(h->nI, ch), n2);
    *nbuf = std::max(ns, maxsl);
    if (*nbuf > 1) {  // per-slice partial V, summed in a fixed order afterwards
        if ((rc = h->Vslices.ensure((size_t)*nbuf * n2))) return rc;
        CUDA_TRY(cudaMemsetAsync(h->Vslices.p, 0, (size_t)*nbuf * n2 * sizeof(double), st));
        *Vdst = h->Vslices.p;
    }
    CUDA_TRY(mark(h, 0));
    return QMMM_OK;
}

static int vpot_sweep(qmmm_handle *h, double *Vdst, int nbuf)
{
    int rc;
    const int kind = sweep_kind(h, false), ch = chunk_for_kind(kind);
    const size_t n2 = (size_t)h->nao * h->nao;
    const int ns = sweep_slices(h, kind, std::min(h->nI, ch));
    const int maxsl = ns > 1 ? 1 : vpot_max_slices(std::min(h->nI, ch), n2);
    for (int c0 = 0; c0 < h->nI; c0 += ch) {
        const int c1 = std::min(h->nI, c0 + ch);
        rc = run_classes(
            h, kind,
            [&](int cls, int p0, int p1, int share, int variant, int nsl, cudaStream_t cs) {
                return launch_sweep(h, kind, cls, p0, p1, c0, c1, share, variant, nsl, nbuf > 1 ? n2 : 0, nullptr,
                                    Vdst, nullptr, nullptr, cs);
            },
            ns, maxsl, c1 - c0);
        if (rc) return rc;
    }
    return QMMM_OK;
}

// enuc == false (a batch frame, whose forces have already formed the nuclear-MM partials): no
// E_nuc_mm output
static int vpot_end(qmmm_handle *h, int nbuf, double *Vout, double *E_nuc_mm, bool enuc = true)
{
    cudaStream_t st = h->stream;
    int rc;
    const size_t n2 = (size_t)h->nao * h->nao;
    if (nbuf > 1) CUDA_TRY(launch_sum_slices_d(h->Vslices.p, nbuf, n2, h->V.p, st));
    CUDA_TRY(mark(h, 1));
    if (enuc) {
        CUDA_TRY(launch_enucmm(h->qm.p, h->Zd.p, h->natm, h->rI.p, h->rI_idx.p, h->nI, h->mm_beta.p, h->Epart.p,
                               nullptr, nullptr, 0, st));
        CUDA_TRY(launch_sum(h->Epart.p, enucmm_nblk(h->nI), h->out4.p + 4, st));
    } else {
        E_nuc_mm = nullptr;
    }
    if ((rc = copy_out(h, Vout, h->V.p, n2))) return rc;
    if ((rc = copy_out(h, E_nuc_mm, h->out4.p + 4, 1))) return rc;
    CUDA_TRY(mark(h, 2));
    if ((rc = finish(h, 3))) return rc;
    h->V_valid = true;
    return QMMM_OK;
}

int qmmm_vpot(qmmm_handle *h, double *Vout, double *E_nuc_mm)
{
    if (!h) return fail(QMMM_ERR_ARG, "null handle");
    int rc, nbuf;
    double *Vdst;
    if ((rc = vpot_prep(h, true, &Vdst, &nbuf))) return rc;
    if ((rc = vpot_sweep(h, Vdst, nbuf))) return rc;
    return vpot_end(h, nbuf, Vout, E_nuc_mm);
}

static int compute_multipoles(qmmm_handle *h, const double *ddm, double *F, int extra_mode)
{
    cudaStream_t st = h->stream;
    CUDA_TRY(cudaMemcpyAsync(h->mult.p, h->mult_init.p, 10 * (size_t)h->natm * sizeof(double), cudaMemcpyDeviceToDevice, st));
    const BasisDev b = h->basis();
    const int mode = MOM_MULT | (F ? MOM_FOCK : 0) | extra_mode;
    // the classes are small kernels (one lane per primitive pair): run them concurrently
    return fork_classes(h, [&](int cls, int p0, int p1, cudaStream_t cs) {
        return launch_moments(b, cls, p0, p1, ddm, h->phi.p, h->mult.p, F, h->gqm.p, mode, cs);
    });
}

int qmmm_ewald(qmmm_handle *h, const double *dmat, double *E_II, double *multipoles, double *F_II)
{
    if (!h || !dmat) return fail(QMMM_ERR_ARG, "null handle or density");
    cudaStream_t st = h->stream;
    int rc;
    const double *ddm;
    const size_t n2 = (size_t)h->nao * h->nao;
    CUDA_TRY(mark(h, 0));
    if ((rc = stage_input(h, dmat, n2, h->dm, &ddm))) return rc;
    double *Fd = nullptr;
    if (F_II) {
        if ((rc = h->F.ensure(n2))) return rc;
        CUDA_TRY(cudaMemsetAsync(h->F.p, 0, n2 * sizeof(double), st));
        Fd = h->F.p;
    }
    if ((rc = compute_multipoles(h, ddm, Fd, 0))) return rc;
    CUDA_TRY(launch_energy_terms(ddm, nullptr, h->nao, 0, h->mult.p, h->phi.p, h->natm, h->Epart.p, 0, h->partials.p,
                                 NPART, h->out4.p, st));
    if ((rc = copy_out(h, E_II, h->out4.p + 3, 1))) return rc;
    if ((rc = copy_out(h, multipoles, h->mult.p, 10 * (size_t)h->natm))) return rc;
    if (F_II && (rc = copy_out(h, F_II, h->F.p, n2))) return rc;
    CUDA_TRY(mark(h, 1));
    if ((rc = finish(h, 2))) return rc;
    return QMMM_OK;
}

int qmmm_density_gradient(qmmm_handle *h, const double *dmat, double *G)
{
    if (!h || !dmat || !G) return fail(QMMM_ERR_ARG, "null argument");
    if (!h->V_valid) return fail(QMMM_ERR_STATE, "qmmm_vpot must run at the current geometry first");
    cudaStream_t st = h->stream;
    int rc;
    const double *ddm;
    const size_t n2 = (size_t)h->nao * h->nao;
    if ((rc = stage_input(h, dmat, n2, h->dm, &ddm))) return rc;
    if ((rc = h->F.ensure(n2))) return rc;
    // start from V; the moment kernels add the region-II Fock term into it
    CUDA_TRY(cudaMemcpyAsync(h->F.p, h->V.p, n2 * sizeof(double), cudaMemcpyDeviceToDevice, st));
    if ((rc = compute_multipoles(h, ddm, h->F.p, 0))) return rc;
    if ((rc = copy_out(h, G, h->F.p, n2))) return rc;
    return finish(h, 0);
}

// E from V, the multipoles already in h->mult and the nuclear-MM partials (no multipole pass:
// a batch frame's forces have just formed the same multipoles from the same density)
static int energy_terms(qmmm_handle *h, const double *ddm, double *E)
{
    CUDA_TRY(launch_energy_terms(ddm, h->V.p, h->nao, 1, h->mult.p, h->phi.p, h->natm, h->Epart.p,
                                 enucmm_nblk(h->nI), h->partials.p, NPART, h->out4.p, h->stream));
    return copy_out(h, E, h->out4.p, 4);
}

int qmmm_energy(qmmm_handle *h, const double *dmat, double *E)
{
    if (!h || !dmat || !E) return fail(QMMM_ERR_ARG, "null argument");
    if (!h->V_valid) return fail(QMMM_ERR_STATE, "qmmm_vpot must run at the current geometry first");
    int rc;
    const double *ddm;
    const size_t n2 = (size_t)h->nao * h->nao;
    if ((rc = stage_input(h, dmat, n2, h->dm, &ddm))) return rc;
    if ((rc = compute_multipoles(h, ddm, nullptr, 0))) return rc;
    if ((rc = energy_terms(h, ddm, E))) return rc;
    return finish(h, 0);
}

// The forces in parts.  forces_prep: the density and the cleared outputs.  forces_sweep: the
// region-I adjoint sweep (all classes on the class streams, left unjoined).  forces_rest:
// multipoles with the Pulay term, the nuclear-MM region-I term and the multipolar Ewald sums.  The
// sweep needs only the density and the cleared outputs, and every kernel adds to the gradients
// atomically, so the sweep may run beside the rest (a batch runs the sweeps of all its frames
// together).  forces_end: region-I charge gradients to the MM atoms, the user's order, copies out.
static int forces_prep(qmmm_handle *h, const double *dmat, const double **ddm)
{
    cudaStream_t st = h->stream;
    int rc;
    const size_t n2 = (size_t)h->nao * h->nao;
    CUDA_TRY(mark(h, 3));
    if ((rc = stage_input(h, dmat, n2, h->dm, ddm))) return rc;
    CUDA_TRY(cudaMemsetAsync(h->gqm.p, 0, 3 * (size_t)h->natm * sizeof(double), st));
    CUDA_TRY(cudaMemsetAsync(h->gchg.p, 0, 4 * (size_t)std::max(h->nI, 1) * sizeof(double), st));
    CUDA_TRY(cudaMemsetAsync(h->dq_int.p, 0, (size_t)std::max(h->nmm, 1) * sizeof(double), st));
    CUDA_TRY(cudaMemsetAsync(h->dR_int.p, 0, 3 * (size_t)std::max(h->nmm, 1) * sizeof(double), st));
    return QMMM_OK;
}

static int forces_sweep(qmmm_handle *h, const double *ddm)
{
    int rc;
    const int kind = sweep_kind(h, true), ch = chunk_for_kind(kind);
    if (kind == SW_VGRAD_F32 && (rc = ensure_cl(h))) return rc;
    const int ns = sweep_slices(h, kind, std::min(h->nI, ch));
    for (int c0 = 0; c0 < h->nI; c0 += ch) {
        const int c1 = std::min(h->nI, c0 + ch);
        rc = run_classes(
            h, kind,
            [&](int cls, int p0, int p1, int share, int variant, int nsl, cudaStream_t cs) {
                return launch_sweep(h, kind, cls, p0, p1, c0, c1, share, variant, nsl, 0, ddm, nullptr, h->gqm.p,
                                    h->gchg.p, cs);
            },
            ns, std::max(1, std::min(8, (c1 - c0) / 128)), c1 - c0, false);
        if (rc) return rc;
    }
    return QMMM_OK;
}

static int forces_rest(qmmm_handle *h, const double *ddm)
{
    cudaStream_t st = h->stream;
    int rc;
    if ((rc = compute_multipoles(h, ddm, nullptr, MOM_PULAY))) return rc;
    CUDA_TRY(launch_enucmm(h->qm.p, h->Zd.p, h->natm, h->rI.p, h->rI_idx.p, h->nI, h->mm_beta.p, h->Epart.p, h->gqm.p,
                           h->gchg.p, 1, st));
    const EwaldDev e = h->ewald();
    CUDA_TRY(launch_ewald_mm(e, h->rI.p, h->nmm > 0 ? h->nI : 0, h->mult.p, h->phi.p, h->ew, h->dq_int.p,
                             h->dR_int.p, h->gchg.p, h->gqm.p, h->precision == QMMM_MIXED, st));
    return QMMM_OK;
}

static int forces_end(qmmm_handle *h, double *dE_dRqm, double *dE_dRmm, double *dE_dq)
{
    cudaStream_t st = h->stream;
    int rc;
    if (h->nmm > 0) {
        CUDA_TRY(launch_scatter_region(h->rI_idx.p, h->nI, h->gchg.p, h->dq_int.p, h->dR_int.p, st));
        CUDA_TRY(launch_unpermute(h->dq_int.p, h->dR_int.p, h->dperm.p, h->nmm, h->dq_out.p, h->dR_out.p, st));
    }
    if ((rc = copy_out(h, dE_dRqm, h->gqm.p, 3 * (size_t)h->natm))) return rc;
    if (h->nmm > 0) {
        if ((rc = copy_out(h, dE_dRmm, h->dR_out.p, 3 * (size_t)h->nmm))) return rc;
        if ((rc = copy_out(h, dE_dq, h->dq_out.p, (size_t)h->nmm))) return rc;
    }
    return QMMM_OK;
}

int qmmm_forces(qmmm_handle *h, const double *dmat, double *dE_dRqm, double *dE_dRmm, double *dE_dq)
{
    if (!h || !dmat) return fail(QMMM_ERR_ARG, "null handle or density");
    int rc;
    const double *ddm;
    if ((rc = forces_prep(h, dmat, &ddm))) return rc;
    CUDA_TRY(mark(h, 0));
    if ((rc = forces_sweep(h, ddm))) return rc;
    if (!h->quiet) {  // the sweep's own end, for its timing
        if ((rc = join_classes(h, h->tstream))) return rc;
        CUDA_TRY(cudaEventRecord(h->ev[1], h->tstream));
    }
    // The rest follows the sweep: run beside it, it delayed the FP64 classes, which hold their
    // shares of the SMs for the whole sweep (large site: FP64 step 461 -> 496 ms), and on the mixed
    // path it saved 2.6 of 49.6 ms but left the sweep's own duration unmeasurable
    if ((rc = join_classes(h, h->stream))) return rc;
    if ((rc = forces_rest(h, ddm))) return rc;
    if ((rc = forces_end(h, dE_dRqm, dE_dRmm, dE_dq))) return rc;
    CUDA_TRY(mark(h, 2));
    return finish(h, 4);
}

int qmmm_get_info(const qmmm_handle *h, qmmm_info_t *info)
{
    if (!h || !info) return fail(QMMM_ERR_ARG, "null argument");
    info->nao = h->nao;
    info->natm = h->natm;
    info->nshell = h->nshell;
    info->nmm = h->nmm;
    info->n_shell_pairs = h->n_sp;
    info->n_prim_pairs = h->n_pp;
    info->n_region1 = h->nI;
    EwaldDev e = h->ewald();
    info->n_gvec = ((2 * e.kmax[0] + 1) * (2 * e.kmax[1] + 1) * (2 * e.kmax[2] + 1) - 1) / 2;
    info->n_sigma_classes = h->ncls;
    info->precision = h->precision;
    for (int c = 0; c < NCLASS; ++c) {
        info->n_prim_pairs_class[c] = h->class_off[c + 1] - h->class_off[c];
        info->n_shell_pairs_class[c] = h->sp_class[c];
    }
    return QMMM_OK;
}

int qmmm_nao(const qmmm_handle *h) { return h ? h->nao : fail(QMMM_ERR_ARG, "null handle"); }

int qmmm_get_potential(qmmm_handle *h, double *v)
{
    if (!h || !v) return fail(QMMM_ERR_ARG, "null argument");
    int rc;
    if ((rc = copy_out(h, v, h->phi.p, 20 * (size_t)h->natm))) return rc;
    return check_device_errors(h);
}

int qmmm_qm_images(qmmm_handle *h, const double *dmat, double *E, double *dE_dRqm, double *F)
{
    if (!h || !dmat) return fail(QMMM_ERR_ARG, "null handle or density");
    cudaStream_t st = h->stream;
    int rc;
    const double *ddm;
    const size_t n2 = (size_t)h->nao * h->nao, na = (size_t)h->natm;
    if ((rc = stage_input(h, dmat, n2, h->dm, &ddm))) return rc;
    if ((rc = h->qmq_P.ensure(na * na * 20)) || (rc = h->qmq_u.ensure(na * 20)) || (rc = h->qmq_g.ensure(na * 3)) ||
        (rc = h->qmq_E.ensure(1)))
        return rc;
    double *Fd = nullptr;
    if (F) {
        if ((rc = h->qmq_F.ensure(n2))) return rc;
        CUDA_TRY(cudaMemsetAsync(h->qmq_F.p, 0, n2 * sizeof(double), st));
        Fd = h->qmq_F.p;
    }
    // Mulliken multipoles at this density, then the image tensors, energy, potentials, gradient
    if ((rc = compute_multipoles(h, ddm, nullptr, 0))) return rc;
    CUDA_TRY(launch_qm_images(h->ewald(), h->gfac.p, h->mult.p, h->qmq_P.p, h->qmq_E.p, h->qmq_u.p, h->qmq_g.p, st));
    // the multipoles move with the basis (Pulay) and depend on gamma (Fock): the moment kernels
    // with the image potential in place of the MM one
    const BasisDev b = h->basis();
    const int mode = MOM_PULAY | (Fd ? MOM_FOCK : 0);
    if ((rc = fork_classes(h, [&](int cls, int p0, int p1, cudaStream_t cs) {
             return launch_moments(b, cls, p0, p1, ddm, h->qmq_u.p, h->mult.p, Fd, h->qmq_g.p, mode, cs);
         })))
        return rc;
    if ((rc = copy_out(h, E, h->qmq_E.p, 1))) return rc;
    if ((rc = copy_out(h, dE_dRqm, h->qmq_g.p, 3 * na))) return rc;
    if (F && (rc = copy_out(h, F, h->qmq_F.p, n2))) return rc;
    return finish(h, 0);
}

int qmmm_octupole_error(qmmm_handle *h, const double *dmat, double r_lo, double dr, int n, double *err,
                        double *octupoles)
{
    if (!h || !dmat || !err) return fail(QMMM_ERR_ARG, "null argument");
    if (n < 1 || n > 65536 || !(dr > 0.0) || !(r_lo >= 0.0))
        return fail(QMMM_ERR_ARG, "need 1 <= n <= 65536, dr > 0, r_lo >= 0");
    cudaStream_t st = h->stream;
    int rc;
    const double *ddm;
    const size_t n2 = (size_t)h->nao * h->nao;
    if ((rc = stage_input(h, dmat, n2, h->dm, &ddm))) return rc;
    if ((rc = h->oct.ensure(10 * (size_t)h->natm)) || (rc = h->oct_bins.ensure((size_t)n + 1)) ||
        (rc = h->oct_err.ensure((size_t)n)))
        return rc;
    CUDA_TRY(cudaMemsetAsync(h->oct.p, 0, 10 * (size_t)h->natm * sizeof(double), st));
    const BasisDev b = h->basis();
    if ((rc = fork_classes(h, [&](int cls, int p0, int p1, cudaStream_t cs) {
             return launch_octupoles(b, cls, p0, p1, ddm, h->oct.p, cs);
         })))
        return rc;
    CUDA_TRY(launch_octupole_error(h->ewald(), h->oct.p, h->phi.p, r_lo, dr, n, h->oct_bins.p, h->oct_err.p, st));
    if ((rc = copy_out(h, err, h->oct_err.p, (size_t)n))) return rc;
    if ((rc = copy_out(h, octupoles, h->oct.p, 10 * (size_t)h->natm))) return rc;
    return finish(h, 0);
}

int qmmm_rcut_search(qmmm_handle *h, const double *dm, double r_lo, double dr, int n, double eps, double *rcut,
                     double *err_at)
{
    if (!rcut || !(eps > 0.0)) return fail(QMMM_ERR_ARG, "null output or eps <= 0");
    std::vector<double> err(std::max(n, 1));
    const int rc = qmmm_octupole_error(h, dm, r_lo, dr, n, err.data(), nullptr);
    if (rc) return rc;
    *rcut = -1.0;
    if (err_at) *err_at = 0.0;
    for (int k = 0; k < n; ++k)
        if (std::fabs(err[k]) < eps) {
            *rcut = r_lo + k * dr;
            if (err_at) *err_at = err[k];
            break;
        }
    return QMMM_OK;
}

int qmmm_autotune(qmmm_handle *h, int flags)
{
    if (!h) return fail(QMMM_ERR_ARG, "null handle");
    if (flags & ~(QMMM_TUNE_V | QMMM_TUNE_FORCES | QMMM_TUNE_BOTH_PRECISIONS))
        return fail(QMMM_ERR_ARG, "unknown autotune flags");
    int which = flags & (QMMM_TUNE_V | QMMM_TUNE_FORCES);
    if (!which) which = QMMM_TUNE_V | QMMM_TUNE_FORCES;
    int kinds[SW_NKIND], nk = 0;
    for (int k = 0; k < SW_NKIND; ++k) {
        const bool grad = kind_is_grad(k), mixed = kind_is_mixed(k);
        if (!(which & (grad ? QMMM_TUNE_FORCES : QMMM_TUNE_V))) continue;
        if (!(flags & QMMM_TUNE_BOTH_PRECISIONS) && mixed != (h->precision == QMMM_MIXED)) continue;
        kinds[nk++] = k;
    }
    if (h->nI == 0 || h->n_pp == 0) return QMMM_OK;
    const size_t n2 = (size_t)h->nao * h->nao;
    const int nch = std::min(h->nI, TUNE_CHARGES);
    int rc;
    if ((rc = h->tune_V.ensure(n2)) || (rc = h->tune_dm.ensure(n2)) || (rc = h->tune_gqm.ensure(3 * (size_t)h->natm)) ||
        (rc = h->tune_gchg.ensure(4 * (size_t)nch)) || (rc = ensure_cl(h)))
        return rc;
    // a zero density: the sweeps' work does not depend on its values
    CUDA_TRY(cudaMemsetAsync(h->tune_dm.p, 0, n2 * sizeof(double), h->stream));
    cudaEvent_t e[2] = {nullptr, nullptr};
    CUDA_TRY(cudaEventCreate(&e[0]));
    if (cudaEventCreate(&e[1]) != cudaSuccess) {
        cudaEventDestroy(e[0]);
        return fail(QMMM_ERR_CUDA, "cudaEventCreate");
    }
    for (int i = 0; i < nk && !rc; ++i) rc = tune_kind(h, kinds[i], e[0], e[1]);
    cudaEventDestroy(e[0]);
    cudaEventDestroy(e[1]);
    if (rc) return rc;
    h->tuned_nI = h->nI;
    return QMMM_OK;
}

int qmmm_get_tuning(const qmmm_handle *h, int kind, int *threads, int *share, double *ms, int *wide,
                    double *weight)
{
    if (!h || kind < 0 || kind >= SW_NKIND) return fail(QMMM_ERR_ARG, "null handle or unknown sweep kind");
    int sh[NCLASS];
    if (!split_sms(h, kind, h->cls_variant[kind], sh))
        for (int c = 0; c < NCLASS; ++c) sh[c] = 0;
    for (int c = 0; c < NCLASS; ++c) {
        if (threads) threads[c] = variant_threads(kind, c, h->cls_variant[kind][c]);
        if (share) share[c] = sh[c];
        if (ms) ms[c] = h->cls_ms[kind][c];
        if (wide) wide[c] = sweep_wide_threads(kind, c);
        if (weight) weight[c] = h->cls_cost[kind][c];
    }
    return (h->tuned_mask >> kind) & 1;
}

int qmmm_set_tuning(qmmm_handle *h, int kind, const int *threads, const double *weight)
{
    if (!h || kind < 0 || kind >= SW_NKIND || !threads) return fail(QMMM_ERR_ARG, "null argument or unknown kind");
    int var[NCLASS];
    for (int c = 0; c < NCLASS; ++c) {
        const int w = sweep_wide_threads(kind, c);
        if (threads[c] == 256) var[c] = 0;
        else if (w > 0 && threads[c] == w) var[c] = 1;
        else return fail(QMMM_ERR_ARG, "block size " + std::to_string(threads[c]) + " not available for class " +
                                           std::to_string(c));
        if (weight && !(weight[c] > 0.0)) return fail(QMMM_ERR_ARG, "weights must be positive");
    }
    reset_tuning(h, kind);
    for (int c = 0; c < NCLASS; ++c) {
        h->cls_variant[kind][c] = var[c];
        if (weight) h->cls_cost[kind][c] = weight[c];
    }
    h->tuned_nI = h->nI;
    return QMMM_OK;
}

int qmmm_last_timing(const qmmm_handle *h, double *out)
{
    if (!h || !out) return fail(QMMM_ERR_ARG, "null argument");
    out[0] = h->t_sweep;
    out[1] = h->t_other;
    return 2;
}

void qmmm_destroy(qmmm_handle *h) { delete h; }

}  // extern "C"

// ---------------------------------------------------------------------------------------------
// Batches of frames: one CUDA graph over every frame's V, energy and gradient
// ---------------------------------------------------------------------------------------------
struct qmmm_batch {
    std::vector<qmmm_handle *> f;
    cudaStream_t stream = nullptr;
    bool own_stream = false;        // created here: the legacy stream cannot be captured
    std::vector<cudaStream_t> fst;  // one stream per frame
    std::vector<cudaEvent_t> done;  // frame f complete (recorded by the graph, for timing)
    std::vector<cudaEvent_t> join;  // frame f joins the batch stream
    cudaEvent_t start = nullptr, fork = nullptr;
    // batched region-I adjoint of the mixed frames: frame f reached its sweep (adone), all did
    // (all_a), class c's sweep over every frame done (cjoin), all classes done (sweeps); per class
    // a stream, a device job table region (jobs + job_off[c]) and a work counter
    std::vector<cudaEvent_t> adone;
    cudaEvent_t all_a = nullptr, sweeps = nullptr, cjoin[NCLASS] = {};
    cudaStream_t cst[NCLASS] = {};
    DBuf<ClJob> jobs;
    DBuf<int> counter;
    int job_off[NCLASS] = {}, njob[NCLASS] = {}, nthr[NCLASS] = {}, nitems[NCLASS] = {}, variant[NCLASS] = {};
    // the batched mixed V sweep: per class a job table region (vjobs + vjob_off[c]), its blocks,
    // the most charges of one block's slice and the block variant; V of every frame done (vdone)
    DBuf<VJob> vjobs;
    int vjob_off[NCLASS] = {}, nvjob[NCLASS] = {}, vblk[NCLASS] = {}, vmaxch[NCLASS] = {}, vvariant[NCLASS] = {};
    cudaEvent_t vdone = nullptr, vjoin[NCLASS] = {};
    cudaGraphExec_t exec = nullptr;
    std::vector<long long> key;  // what the graph was recorded for
    std::vector<int> planned_nI; // each frame's region-I size at the last plain pass (buffer sizes)
    int captures = 0, instantiations = 0, updates = 0;
    std::vector<double> ms;  // last run: total, then per frame
    ~qmmm_batch()
    {
        if (exec) cudaGraphExecDestroy(exec);
        for (cudaEvent_t e : done)
            if (e) cudaEventDestroy(e);
        for (cudaEvent_t e : join)
            if (e) cudaEventDestroy(e);
        for (cudaStream_t s : fst)
            if (s) cudaStreamDestroy(s);
        if (start) cudaEventDestroy(start);
        if (fork) cudaEventDestroy(fork);
        for (cudaEvent_t e : adone)
            if (e) cudaEventDestroy(e);
        if (all_a) cudaEventDestroy(all_a);
        if (sweeps) cudaEventDestroy(sweeps);
        if (vdone) cudaEventDestroy(vdone);
        for (int c = 0; c < NCLASS; ++c) {
            if (cjoin[c]) cudaEventDestroy(cjoin[c]);
            if (vjoin[c]) cudaEventDestroy(vjoin[c]);
            if (cst[c]) cudaStreamDestroy(cst[c]);
        }
        jobs.release();
        counter.release();
        vjobs.release();
        if (own_stream && stream) cudaStreamDestroy(stream);
    }
};

namespace {

// Everything a recorded batch graph depends on: per frame its region-I size, precision, sweep
// configuration and the arrays it reads and writes.
std::vector<long long> batch_key(const qmmm_batch *b, const double *const *dm, double *const *V, double *const *E,
                                 double *const *gq, double *const *gm, double *const *gc)
{
    std::vector<long long> k;
    auto ptr = [](const void *p) { return (long long)(uintptr_t)p; };
    for (size_t i = 0; i < b->f.size(); ++i) {
        const qmmm_handle *h = b->f[i];
        k.push_back(h->nI);
        k.push_back(h->plan_gen);
        k.push_back(h->precision);
        for (int kind = 0; kind < SW_NKIND; ++kind)
            for (int c = 0; c < NCLASS; ++c) {
                long long bits;
                std::memcpy(&bits, &h->cls_cost[kind][c], sizeof(bits));
                k.push_back(bits);
                k.push_back(h->cls_variant[kind][c]);
            }
        k.push_back(ptr(dm[i]));
        k.push_back(ptr(V ? V[i] : nullptr));
        k.push_back(ptr(E ? E[i] : nullptr));
        k.push_back(ptr(gq ? gq[i] : nullptr));
        k.push_back(ptr(gm ? gm[i] : nullptr));
        k.push_back(ptr(gc ? gc[i] : nullptr));
    }
    return k;
}

// One frame's work through the public calls, on the handle's current stream.
int batch_frame(qmmm_handle *h, const double *dm, double *V, double *E, double *gq, double *gm, double *gc)
{
    int rc;
    if ((rc = qmmm_vpot(h, V, nullptr))) return rc;
    if (E && (rc = qmmm_energy(h, dm, E))) return rc;
    return qmmm_forces(h, dm, gq, gm, gc);
}

// Frames whose region-I adjoint the batch runs for all of them at once: the charge-lane sweep
// (mixed precision) over a non-empty region I.
bool batch_defers(const qmmm_handle *h) { return sweep_kind(h, true) == SW_VGRAD_F32 && h->nI > 0; }

// The job tables of the batched adjoint: per class, one job per deferring frame with pairs in
// that class, in descending order of the pair batches per item (the longest items are taken
// first), uploaded to b->jobs.  Every class takes one block variant: that of the frame with the
// most pair x charge work in the class.
int batch_build_jobs(qmmm_batch *b, const double *const *dm)
{
    std::vector<ClJob> all;
    for (int c = 0; c < NCLASS; ++c) {
        b->job_off[c] = (int)all.size();
        b->njob[c] = b->nthr[c] = b->nitems[c] = 0;
        const int L = la_of_class(c) + lb_of_class(c);
        double best = -1.0;
        b->variant[c] = 0;
        for (qmmm_handle *h : b->f) {
            if (!batch_defers(h)) continue;
            const double w = (double)(h->class_off[c + 1] - h->class_off[c]) * h->nI;
            if (w > best) {
                best = w;
                b->variant[c] = h->cls_variant[SW_VGRAD_F32][c];
            }
        }
        std::vector<ClJob> cj;
        for (size_t i = 0; i < b->f.size(); ++i) {
            qmmm_handle *h = b->f[i];
            const int p0 = h->class_off[c], p1 = h->class_off[c + 1];
            if (!batch_defers(h) || p1 <= p0) continue;
            ClJob J{};
            J.bd = h->basis();
            J.rg = h->region();
            J.dm = dm[i];
            J.rec = h->cl_rec.p + h->cl_rec_off[c];
            J.psum = h->cl_psum.p + h->cl_psum_off[c];
            J.gqm = h->gqm.p;
            J.gchg = h->gchg.p;
            J.pp_begin = p0;
            J.pp_end = p1;
            J.ch_begin = 0;
            J.ch_end = h->nI;
            cl_decompose(L, b->variant[c], p1 - p0, h->nI, h->ncls, J.gx, J.ntile);
            cj.push_back(J);
        }
        const int nb = cl_batch(L);
        auto bper = [nb](const ClJob &J) { return ((J.pp_end - J.pp_begin + nb - 1) / nb + J.gx - 1) / J.gx; };
        std::stable_sort(cj.begin(), cj.end(), [&](const ClJob &x, const ClJob &y) { return bper(x) > bper(y); });
        int item = 0, thr = 0;
        for (ClJob &J : cj) {
            J.item0 = item;
            J.thr0 = thr;
            item += J.gx * J.ntile;
            thr += (J.pp_end - J.pp_begin + 31) / 32 * 32;
        }
        b->njob[c] = (int)cj.size();
        b->nitems[c] = item;
        b->nthr[c] = thr;
        all.insert(all.end(), cj.begin(), cj.end());
    }
    int rc;
    if ((rc = b->jobs.ensure(std::max<size_t>(all.size(), 1))) || (rc = b->counter.ensure(NCLASS))) return rc;
    if (!all.empty())
        CUDA_TRY(cudaMemcpy(b->jobs.p, all.data(), all.size() * sizeof(ClJob), cudaMemcpyHostToDevice));

    // the V sweep: per class one job per deferring frame, each charge slice (at most CHUNK_F32
    // charges) in blocks of one 32-pair tile per warp; the block variant of the frame with the
    // most work in the class
    std::vector<VJob> vall;
    for (int c = 0; c < NCLASS; ++c) {
        b->vjob_off[c] = (int)vall.size();
        b->nvjob[c] = b->vblk[c] = b->vmaxch[c] = 0;
        double best = -1.0;
        b->vvariant[c] = 0;
        for (qmmm_handle *h : b->f) {
            if (!batch_defers(h)) continue;
            const double w = (double)(h->class_off[c + 1] - h->class_off[c]) * h->nI;
            if (w > best) {
                best = w;
                b->vvariant[c] = h->cls_variant[SW_VPOT_F32][c];
            }
        }
        const int nwarp = variant_threads(SW_VPOT_F32, c, b->vvariant[c]) / 32;
        int blk = 0;
        for (size_t i = 0; i < b->f.size(); ++i) {
            qmmm_handle *h = b->f[i];
            const int p0 = h->class_off[c], p1 = h->class_off[c + 1];
            if (!batch_defers(h) || p1 <= p0) continue;
            VJob J{};
            J.bd = h->basis();
            J.rg = h->region();
            J.V = h->V.p;
            J.pp_begin = p0;
            J.pp_end = p1;
            J.ch_begin = 0;
            J.ch_end = h->nI;
            J.ns = (h->nI + CHUNK_F32 - 1) / CHUNK_F32;
            J.gx = ((p1 - p0 + 31) / 32 + nwarp - 1) / nwarp;
            J.blk0 = blk;
            blk += J.gx * J.ns;
            b->vmaxch[c] = std::max(b->vmaxch[c], (h->nI + J.ns - 1) / J.ns);
            vall.push_back(J);
            ++b->nvjob[c];
        }
        b->vblk[c] = blk;
    }
    if ((rc = b->vjobs.ensure(std::max<size_t>(vall.size(), 1)))) return rc;
    if (!vall.empty())
        CUDA_TRY(cudaMemcpy(b->vjobs.p, vall.data(), vall.size() * sizeof(VJob), cudaMemcpyHostToDevice));
    return QMMM_OK;
}

// The batched adjoint inside the capture: every class over the deferring frames once all of them
// have cleared their gradients (one launch of each of the class's three kernels), highest class
// first, beside the frames' other work.
int batch_sweeps(qmmm_batch *b, const std::vector<int> &deferred)
{
    for (int i : deferred) CUDA_TRY(cudaStreamWaitEvent(b->stream, b->adone[i], 0));
    CUDA_TRY(cudaEventRecord(b->all_a, b->stream));
    const qmmm_handle *h0 = b->f[deferred[0]];
    for (int i = 0; i < NCLASS; ++i) {
        const int c = NCLASS - 1 - i;
        if (!b->njob[c] && !b->nvjob[c]) continue;
        CUDA_TRY(cudaStreamWaitEvent(b->cst[c], b->all_a, 0));
        CUDA_TRY(launch_vpot_f32_jobs(c, b->vjobs.p + b->vjob_off[c], b->nvjob[c], b->vblk[c], b->vmaxch[c],
                                      h0->boys32.p, h0->err.p, b->vvariant[c], b->cst[c]));
        CUDA_TRY(cudaEventRecord(b->vjoin[c], b->cst[c]));
        CUDA_TRY(launch_vgrad_cl_jobs(c, b->jobs.p + b->job_off[c], b->njob[c], b->nthr[c], b->nitems[c],
                                      b->counter.p + c, h0->boys32.p, b->variant[c], h0->nsm, b->cst[c]));
        CUDA_TRY(cudaEventRecord(b->cjoin[c], b->cst[c]));
    }
    for (int c = 0; c < NCLASS; ++c)
        if (b->njob[c] || b->nvjob[c]) CUDA_TRY(cudaStreamWaitEvent(b->stream, b->vjoin[c], 0));
    CUDA_TRY(cudaEventRecord(b->vdone, b->stream));
    for (int c = 0; c < NCLASS; ++c)
        if (b->njob[c] || b->nvjob[c]) CUDA_TRY(cudaStreamWaitEvent(b->stream, b->cjoin[c], 0));
    CUDA_TRY(cudaEventRecord(b->sweeps, b->stream));
    return QMMM_OK;
}

}  // namespace

extern "C" {

int qmmm_batch_create(qmmm_handle *const *frames, int nframes, void *stream, qmmm_batch **out)
{
    if (!out || !frames || nframes <= 0) return fail(QMMM_ERR_ARG, "null argument or no frames");
    *out = nullptr;
    std::unique_ptr<qmmm_batch> b(new qmmm_batch());
    b->stream = (cudaStream_t)stream;
    if (!b->stream) {
        CUDA_TRY(cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking));
        b->own_stream = true;
    }
    for (int i = 0; i < nframes; ++i) {
        if (!frames[i]) return fail(QMMM_ERR_ARG, "null frame handle");
        for (int j = 0; j < i; ++j)
            if (frames[j] == frames[i]) return fail(QMMM_ERR_ARG, "a handle appears twice in the batch");
        b->f.push_back(frames[i]);
    }
    b->fst.assign(nframes, nullptr);
    b->done.assign(nframes, nullptr);
    b->join.assign(nframes, nullptr);
    CUDA_TRY(cudaEventCreate(&b->start));
    CUDA_TRY(cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming));
    b->adone.assign(nframes, nullptr);
    for (int i = 0; i < nframes; ++i) {
        CUDA_TRY(cudaStreamCreateWithFlags(&b->fst[i], cudaStreamNonBlocking));
        CUDA_TRY(cudaEventCreate(&b->done[i]));
        CUDA_TRY(cudaEventCreateWithFlags(&b->join[i], cudaEventDisableTiming));
        CUDA_TRY(cudaEventCreateWithFlags(&b->adone[i], cudaEventDisableTiming));
    }
    CUDA_TRY(cudaEventCreateWithFlags(&b->all_a, cudaEventDisableTiming));
    CUDA_TRY(cudaEventCreateWithFlags(&b->sweeps, cudaEventDisableTiming));
    CUDA_TRY(cudaEventCreateWithFlags(&b->vdone, cudaEventDisableTiming));
    for (int c = 0; c < NCLASS; ++c) {
        CUDA_TRY(cudaStreamCreateWithFlags(&b->cst[c], cudaStreamNonBlocking));
        CUDA_TRY(cudaEventCreateWithFlags(&b->cjoin[c], cudaEventDisableTiming));
        CUDA_TRY(cudaEventCreateWithFlags(&b->vjoin[c], cudaEventDisableTiming));
    }
    b->ms.assign(nframes + 1, 0.0);
    *out = b.release();
    return QMMM_OK;
}

int qmmm_batch_run(qmmm_batch *b, const double *const *dm, double *const *V, double *const *E,
                   double *const *dE_dRqm, double *const *dE_dRmm, double *const *dE_dq)
{
    if (!b || !dm) return fail(QMMM_ERR_ARG, "null batch or density array");
    const int n = (int)b->f.size();
    auto at = [](double *const *a, int i) { return a ? a[i] : nullptr; };
    for (int i = 0; i < n; ++i) {
        if (!dm[i] || !is_device_ptr(dm[i])) return fail(QMMM_ERR_ARG, "every density must be device memory");
        const void *o[5] = {at(V, i), at(E, i), at(dE_dRqm, i), at(dE_dRmm, i), at(dE_dq, i)};
        for (const void *p : o)
            if (p && !is_device_ptr(p)) return fail(QMMM_ERR_ARG, "batch outputs must be device memory");
    }
    std::vector<cudaStream_t> own(n);
    for (int i = 0; i < n; ++i) own[i] = b->f[i]->stream;
    auto restore = [&] {
        for (int i = 0; i < n; ++i) {
            b->f[i]->stream = own[i];
            b->f[i]->quiet = false;
        }
    };
    int rc = QMMM_OK;
    std::vector<long long> key = batch_key(b, dm, V, E, dE_dRqm, dE_dRmm, dE_dq);
    if (!b->exec || key != b->key) {
        // plain pass, which sizes every buffer and sets every kernel attribute, before the first
        // recording and whenever a frame's region I outgrew its buffers; otherwise (new positions
        // of the same frames, as in MD) only the recording is repeated
        bool plain = !b->exec || (int)b->planned_nI.size() != n;
        for (int i = 0; i < n && !plain; ++i) plain = b->f[i]->nI > b->planned_nI[i];
        if (plain) {
            for (int i = 0; i < n && !rc; ++i) {
                b->f[i]->stream = b->fst[i];
                rc = batch_frame(b->f[i], dm[i], at(V, i), at(E, i), at(dE_dRqm, i), at(dE_dRmm, i), at(dE_dq, i));
            }
            if (rc) {
                restore();
                return rc;
            }
            b->planned_nI.assign(n, 0);
            for (int i = 0; i < n; ++i) b->planned_nI[i] = b->f[i]->nI;
        }
        // the frames whose adjoint sweeps run batched: their scratch sized and their job tables
        // written before the capture (nothing is allocated or copied synchronously inside it)
        std::vector<int> deferred;
        for (int i = 0; i < n; ++i)
            if (batch_defers(b->f[i])) deferred.push_back(i);
        for (int i : deferred)
            if ((rc = ensure_cl(b->f[i]))) break;
        if (!rc && !deferred.empty()) rc = batch_build_jobs(b, dm);
        if (rc) {
            restore();
            return rc;
        }
        std::vector<char> defer(n, 0);
        for (int i : deferred) defer[i] = 1;
        // every frame issues its work on its batch stream, which joins the capture (a frame left on
        // its own stream would run at once, outside the graph)
        for (int i = 0; i < n; ++i) b->f[i]->stream = b->fst[i];
        cudaGraph_t graph = nullptr;
        cudaError_t e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeRelaxed);
        if (e == cudaSuccess) e = cudaEventRecordWithFlags(b->start, b->stream, cudaEventRecordExternal);
        if (e == cudaSuccess) e = cudaEventRecord(b->fork, b->stream);
        // each frame up to its sweep (the whole frame where it is not deferred)
        for (int i = 0; i < n && e == cudaSuccess && !rc; ++i) {
            qmmm_handle *h = b->f[i];
            if ((e = cudaStreamWaitEvent(b->fst[i], b->fork, 0)) != cudaSuccess) break;
            h->quiet = true;
            if (defer[i]) {
                // cleared V and gradients (the batched sweeps wait for these of every frame), then
                // the forces' other parts beside the sweeps; V and the energy follow below
                const double *ddm = nullptr;
                double *Vdst;
                int nbuf;
                rc = vpot_prep(h, false, &Vdst, &nbuf);
                if (!rc) rc = forces_prep(h, dm[i], &ddm);
                if (!rc && (e = cudaEventRecord(b->adone[i], b->fst[i])) == cudaSuccess) rc = forces_rest(h, ddm);
                h->quiet = false;
                if (rc) break;
                continue;  // the loop condition stops on a failed record
            }
            rc = batch_frame(h, dm[i], at(V, i), at(E, i), at(dE_dRqm, i), at(dE_dRmm, i), at(dE_dq, i));
            h->quiet = false;
            if (rc) break;
            if ((e = cudaEventRecordWithFlags(b->done[i], b->fst[i], cudaEventRecordExternal)) != cudaSuccess) break;
            if ((e = cudaEventRecord(b->join[i], b->fst[i])) != cudaSuccess) break;
            e = cudaStreamWaitEvent(b->stream, b->join[i], 0);
        }
        // the deferred frames' sweeps, all classes over all of them, then each frame's last part
        if (e == cudaSuccess && !rc && !deferred.empty()) rc = batch_sweeps(b, deferred);
        for (size_t k = 0; k < deferred.size() && e == cudaSuccess && !rc; ++k) {
            const int i = deferred[k];
            qmmm_handle *h = b->f[i];
            if ((e = cudaStreamWaitEvent(b->fst[i], b->vdone, 0)) != cudaSuccess) break;
            h->quiet = true;
            rc = vpot_end(h, 1, at(V, i), nullptr, false);
            // the energy from the multipoles and nuclear-MM partials the frame's forces formed
            if (!rc && at(E, i)) rc = energy_terms(h, dm[i], at(E, i));
            if (!rc && (e = cudaStreamWaitEvent(b->fst[i], b->sweeps, 0)) == cudaSuccess)
                rc = forces_end(h, at(dE_dRqm, i), at(dE_dRmm, i), at(dE_dq, i));
            h->quiet = false;
            if (rc || e != cudaSuccess) break;
            if ((e = cudaEventRecordWithFlags(b->done[i], b->fst[i], cudaEventRecordExternal)) != cudaSuccess) break;
            if ((e = cudaEventRecord(b->join[i], b->fst[i])) != cudaSuccess) break;
            e = cudaStreamWaitEvent(b->stream, b->join[i], 0);
        }
        // always end the capture, so the stream leaves capture mode even after a failure
        const cudaError_t e_end = cudaStreamEndCapture(b->stream, &graph);
        restore();
        if (rc || e != cudaSuccess || e_end != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            cudaGetLastError();
            if (rc) return rc;
            return fail(QMMM_ERR_CUDA, std::string("batch graph capture: ") +
                                           cudaGetErrorString(e != cudaSuccess ? e : e_end));
        }
        // same topology with new launch parameters (region-I sizes, pointers): update in place
        bool updated = false;
        if (b->exec) {
            cudaGraphExecUpdateResultInfo info;
            if (cudaGraphExecUpdate(b->exec, graph, &info) == cudaSuccess) {
                updated = true;
                ++b->updates;
            } else {
                cudaGetLastError();
                cudaGraphExecDestroy(b->exec);
                b->exec = nullptr;
            }
        }
        if (!updated) {
            e = cudaGraphInstantiate(&b->exec, graph, 0);
            if (e != cudaSuccess) {
                cudaGraphDestroy(graph);
                b->exec = nullptr;
                return fail(QMMM_ERR_CUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e));
            }
            ++b->instantiations;
        }
        cudaGraphDestroy(graph);
        b->key = key;
        ++b->captures;
    }
    CUDA_TRY(cudaGraphLaunch(b->exec, b->stream));
    CUDA_TRY(cudaStreamSynchronize(b->stream));
    double total = 0.0;
    for (int i = 0; i < n; ++i) {
        float t = 0.f;
        CUDA_TRY(cudaEventElapsedTime(&t, b->start, b->done[i]));
        b->ms[1 + i] = t;
        total = std::max(total, (double)t);
        if ((rc = check_device_errors(b->f[i]))) return rc;
        b->f[i]->V_valid = true;
    }
    b->ms[0] = total;
    return QMMM_OK;
}

int qmmm_batch_timing(const qmmm_batch *b, double *ms)
{
    if (!b || !ms) return fail(QMMM_ERR_ARG, "null argument");
    for (size_t i = 0; i < b->ms.size(); ++i) ms[i] = b->ms[i];
    return (int)b->ms.size();
}

int qmmm_batch_captures(const qmmm_batch *b) { return b ? b->captures : fail(QMMM_ERR_ARG, "null batch"); }

int qmmm_batch_counts(const qmmm_batch *b, int *recorded, int *instantiated, int *updated)
{
    if (!b) return fail(QMMM_ERR_ARG, "null batch");
    if (recorded) *recorded = b->captures;
    if (instantiated) *instantiated = b->instantiations;
    if (updated) *updated = b->updates;
    return QMMM_OK;
}

void qmmm_batch_destroy(qmmm_batch *b) { delete b; }

}  // extern "C"
