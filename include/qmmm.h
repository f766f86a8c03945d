/*
 * qmmm.h -- C ABI of the GB300 (sm_103a) implementation of the data-parallel hot path of the
 * periodic QM/MM-Multipole electrostatic embedding (arXiv 2408.03273).
 *
 * The calls follow the energy partition of Eq. 1, E = E_QM + E_QM-MM + E_MM; this library owns
 * E_QM-MM at a fixed one-body density matrix gamma and its gradient:
 *
 *   E_QM-MM = sum_{mu nu} gamma_{mu nu} V_{mu nu}          region-I electronic term, Eq. 9
 *           + E_nuc_mm                                     region-I nuclear-MM term
 *           + E_II                                         multipole terms of Eq. 6 (QM-MM
 *                                                          lines) plus the Gaussian-charge
 *                                                          correction of Eq. 10
 *
 *   V_{mu nu} = - sum_{i in I} q_i <mu nu | phi_i>,  phi_i a normalised Gaussian of exponent
 *   1/sigma_i^2 (sigma_i <= 0: point charge, Eq. 2).
 *   E_II = sum_j [Q_j v_j + mu_j . v_j,a + theta_j : v_j,ab] with Mulliken multipoles (SI,
 *   "Multipolar Ewald") and the potential v of region II built from the Ewald tensors psi, minus
 *   the point tensors T over region I, minus the screened tensors T-hat over region II.
 *
 * Region I (Sec. "Error Control via Charge-Octupole Estimation") is the set of MM images with
 * |R_i + L - c| < cutoff, c the unweighted mean of the QM positions.  Ewald (SI): real-space
 * erfc sum over images within ewald_rcut, reciprocal sum over the cube max|n_c| <= kmax_c,
 * n != 0, G = 2 pi n / box, tin-foil boundary, neutralising background -pi/(V alpha^2).
 *
 * Conventions
 *   - Atomic units (bohr, hartree, elementary charge).  Orthorhombic box.
 *   - Cartesian Gaussian shells, l <= 3, 1..16 primitives; raw coefficients are normalised by
 *     the library (each primitive normalises its x^l component; the contraction is
 *     renormalised; the same factor multiplies every Cartesian component).  AO order: shells
 *     in input order, components lexicographic (xx, xy, xz, yy, yz, zz).
 *   - Matrices are nao x nao, row-major, FP64.  Gradients are dE/dX (not forces).
 *   - Multipoles per atom (10): Q, mu_x, mu_y, mu_z, theta_xx, theta_xy, theta_xz, theta_yy,
 *     theta_yz, theta_zz (theta is the non-traceless second moment).
 *   - Pointers: every array argument may be host or device memory (detected per call with
 *     cudaPointerGetAttributes).  Host outputs are written before the call returns; device
 *     outputs are written on the handle's stream (the call still synchronises that stream
 *     before returning).  Inputs are copied; the caller keeps ownership of everything it
 *     passes.  Outputs are caller-allocated.
 *   - Errors: every call returns QMMM_OK (0) or a negative QMMM_ERR_* code; on error, outputs
 *     are left untouched or partially written and the handle stays usable unless the code is
 *     QMMM_ERR_CUDA.  qmmm_strerror() gives a message, qmmm_last_error() the last detail.
 *   - Threading: a handle is not thread-safe; distinct handles are independent.
 */
#ifndef QMMM_H
#define QMMM_H

#ifdef __cplusplus
extern "C" {
#endif

/* QM nucleus: position (bohr) and nuclear charge (enters Q_j, SI first equation). */
typedef struct { double xyz[3]; double Z; } qmmm_atom;
/* Cartesian shell on atom `atom` with angular momentum l and primitives
 * [prim_offset, prim_offset + nprim) of the primitive array. */
typedef struct { int atom; int l; int nprim; int prim_offset; } qmmm_shell;
/* Primitive Gaussian: exponent (bohr^-2) and raw contraction coefficient. */
typedef struct { double exponent; double coeff; } qmmm_primitive;
/* MM charge: position (bohr), charge (e) and Gaussian width sigma (bohr); exponent 1/sigma^2. */
typedef struct { double xyz[3]; double q; double sigma; } qmmm_charge;

enum {
    QMMM_OK = 0,
    QMMM_ERR_ARG = -1,           /* invalid argument (null handle, sizes, unsupported option) */
    QMMM_ERR_ALLOC = -2,         /* device or host allocation failed */
    QMMM_ERR_CUDA = -3,          /* a CUDA call failed; see qmmm_last_error() */
    QMMM_ERR_TIMEOUT = -4,       /* a bounded device-side wait ran out */
    QMMM_ERR_UNSUPPORTED_L = -5, /* a shell with l > 3 or more than 16 primitives */
    QMMM_ERR_STATE = -6          /* call order violated (e.g. E_I requested before qmmm_vpot) */
};

enum { QMMM_FP64 = 0, QMMM_MIXED = 1 };

/* Create-time options.  A NULL pointer selects the defaults in brackets. */
typedef struct {
    int precision;      /* QMMM_FP64 or QMMM_MIXED [QMMM_FP64]                                 */
    double screen_tol;  /* primitive pairs with |c_a c_b| K_AB (pi/p)^{3/2} below screen_tol
                           times the largest value are dropped; 0 disables; < 0: [1e-14]       */
    int region_mode;    /* 0: sphere of radius cutoff about the QM centre [0]                  */
    double ewald_rcut;  /* Ewald real-space cutoff (bohr); <= 0: equal to cutoff [cutoff]       */
    int kmax[3];        /* reciprocal cube half-widths (<= 56); 0: chosen so that
                           exp(-G^2/4alpha^2) < 1e-8 at the edge                               */
    int full_cell_test; /* reserved, must be 0                                                 */
} qmmm_options;

typedef struct qmmm_handle qmmm_handle;

/* Counts describing the plan of a handle (after the last qmmm_set_positions). */
typedef struct {
    int nao, natm, nshell, nmm;
    long long n_shell_pairs;    /* screened shell pairs (i <= j)                               */
    long long n_prim_pairs;     /* screened primitive pairs                                    */
    int n_region1;              /* region-I MM images                                          */
    int n_gvec;                 /* reciprocal vectors in the half space (each stands for +-G) */
    int n_sigma_classes;        /* distinct Gaussian widths                                   */
    int precision;
    long long n_prim_pairs_class[10]; /* screened primitive pairs per angular class (l_A >= l_B),
                                         class index l_A (l_A + 1)/2 + l_B                        */
    long long n_shell_pairs_class[10];
} qmmm_info_t;

/* Copies the inputs, normalises the basis, builds the angular-class-sorted, overlap-screened
 * shell-pair list, the reciprocal vectors and the Boys tables, uploads everything to the
 * current CUDA device and runs qmmm_set_positions with the given positions.
 *   atoms[natm], shells[nshell], prims[nprim], charges[nmm] (host memory),
 *   box[3] (bohr), cutoff = region-I radius R_cut (bohr), ewald_alpha (bohr^-1, the erfc
 *   splitting parameter), opts may be NULL.  *out receives the handle. */
int qmmm_create(const qmmm_atom *atoms, int natm, const qmmm_shell *shells, int nshell,
                const qmmm_primitive *prims, int nprim, const qmmm_charge *charges, int nmm,
                const double box[3], double cutoff, double ewald_alpha,
                const qmmm_options *opts, qmmm_handle **out);

/* Stream for all later work of the handle (a cudaStream_t passed as void*; NULL = legacy). */
int qmmm_set_stream(qmmm_handle *h, void *stream);

/* Switch the region-I V / adjoint arithmetic: QMMM_FP64, or QMMM_MIXED.  On the mixed path the
 * per-(primitive pair, charge) work of Eq. 9 and its derivatives runs in FP32: correctly rounded
 * FP32 displacements (coordinates split into hi parts on a 2^-16 bohr grid and lo parts), the
 * Boys function from an FP32 table with its argument carried as an unevaluated FP32 pair, the
 * Hermite recursion and the contractions with the density-folded coefficients (built per pair
 * in FP64, rounded to FP32).  Per-pair and per-charge sums are carried in double-float (FP32
 * pairs) and finished in FP64.  Everything else stays FP64-class on both paths: the per-pair
 * Hermite/density algebra, the nuclear-MM term, the real-space Ewald sums, the multipoles and
 * moment integrals.  The two reciprocal Ewald sums are, on the tensor cores, exact products of
 * BF16 digit planes of fixed-point operands (QMMM_RECIP_TENSOR: 48-bit, except the mixed path's
 * MM-side sum, 34-bit, within about 1e-8 of the largest MM gradient) and on the CUDA cores FP64
 * (double-float on the mixed path, about 47 bits).  On the mixed path the two G sums around
 * them, the region-II potential's reciprocal part at the QM atoms and the multipole structure
 * factor A(G) of the MM-side sum, run in double-float arithmetic (about 44 bits; the region-II
 * potential stays within 1e-12 of FP64).  Measured error of the mixed path against
 * FP64: 1e-7 to 8e-7 in V (relative Frobenius norm) and up to 8e-7 in the gradients
 * (max |error| / max |gradient|) on the benchmark workloads. */
int qmmm_set_precision(qmmm_handle *h, int precision);

/* Method of the two reciprocal Ewald sums (SI, "Multipolar Ewald", long-range part): the MM
 * structure factor S(G) = sum_i q_i exp(iG.R_i) behind the region-II potential at the QM atoms,
 * and the MM-side sum of the adjoint (dE/dq_i, dE/dR_i from the QM multipoles):
 *   QMMM_RECIP_CUDA_CORES: FP64 (double-float for QMMM_MIXED) on the CUDA cores;
 *   QMMM_RECIP_TENSOR: each sum as a product of two matrices on the BF16 tensor cores, every
 *     operand split exactly into seven digit planes (a leading one and six of 7 bits, 48-bit
 *     fixed point) with exact FP32 accumulation of the leading digit levels: FP64 class (about
 *     1e-12 relative on the region-II potential and the MM gradients).  The mixed path's MM-side
 *     sum takes five planes (34-bit fixed point) and two exact levels instead of seven and four
 *     (within about 1e-8 of the largest MM gradient; 15 plane products instead of 28, and a
 *     single N tile up to kx = 25); the MM-side sum stays on the CUDA cores when 2 kz + 1 < 8;
 *   QMMM_RECIP_AUTO [default]: QMMM_RECIP_TENSOR when (kx + 1)(2 ky + 1)(2 kz + 1) N_MM >= 4e7,
 *     else QMMM_RECIP_CUDA_CORES (small systems, where the extra launches outweigh the work).
 * The tensor-core scratch is allocated the first time the method is in effect: fixed-point
 * phase rows (16 (kx + 4 ky + 4 kz + 5) bytes per charge), the B-operand digit planes and the
 * structure factor's partial sums (about 3 KB per charge at kmax 16 in all).
 * Recomputes the region-II potential at the current geometry if the method in effect changes.
 * QMMM_ERR_ARG for another value. */
enum { QMMM_RECIP_CUDA_CORES = 0, QMMM_RECIP_TENSOR = 1, QMMM_RECIP_AUTO = 2 };
int qmmm_set_recip_method(qmmm_handle *h, int method);

/* New geometry (MD step): qm_xyz[natm*3], mm_xyz[nmm*3] (bohr), mm_q[nmm] (NULL keeps the
 * charges).  Rebuilds region I and the gamma-independent region-II potential v (20 Taylor
 * components per QM atom, Eq. 6 QM-MM lines + Eq. 10). */
int qmmm_set_positions(qmmm_handle *h, const double *qm_xyz, const double *mm_xyz, const double *mm_q);

/* Region-I one-electron matrix V[nao*nao] of Eq. 9 (symmetric) and, if E_nuc_mm != NULL, the
 * region-I nuclear-MM energy sum_j sum_{i in I} Z_j q_i erf(r/sigma_i)/r.  V stays cached in
 * the handle for qmmm_energy. */
int qmmm_vpot(qmmm_handle *h, double *V, double *E_nuc_mm);

/* Multipole part at density dm[nao*nao] (symmetric): E_II (scalar), optionally the Mulliken
 * multipoles multipoles[natm*10] and the region-II Fock term F_II[nao*nao] of Eqs. 11-14,
 * F_{mu nu} = -1/2 sum_j sum_c v_j,c [d_{mu in j} + d_{nu in j}] <mu|O_c(r - R_j)|nu>. */
int qmmm_ewald(qmmm_handle *h, const double *dm, double *E_II, double *multipoles, double *F_II);

/* Total E_QM-MM at dm: E[4] = {E_total, E_I_elec = sum gamma V, E_nuc_mm, E_II}.  Needs a
 * prior qmmm_vpot at the current geometry (QMMM_ERR_STATE otherwise). */
int qmmm_energy(qmmm_handle *h, const double *dm, double *E);

/* Derivative of E_QM-MM with respect to the density matrix, the embedding's contribution to the
 * Fock/KS matrix (Eqs. 11-14): G[nao*nao] = dE/dgamma = V + F_II, V the region-I matrix of the
 * last qmmm_vpot (Eq. 9) and F_II the region-II multipole term as in qmmm_ewald at density dm.
 * Needs a prior qmmm_vpot at the current geometry (QMMM_ERR_STATE otherwise).  dm and G: host or
 * device memory. */
int qmmm_density_gradient(qmmm_handle *h, const double *dm, double *G);

/* Gradient of E_QM-MM at fixed dm (region-I integral derivatives, nuclear-MM term, tensor
 * derivatives, and the multipole Pulay term of Eq. 15): dE_dRqm[natm*3], dE_dRmm[nmm*3],
 * dE_dq[nmm].  Any output may be NULL. */
int qmmm_forces(qmmm_handle *h, const double *dm, double *dE_dRqm, double *dE_dRmm, double *dE_dq);

/* Plan counts. */
int qmmm_get_info(const qmmm_handle *h, qmmm_info_t *info);
int qmmm_nao(const qmmm_handle *h);

/* Region-II potential v[natm*20] at the current geometry (components: scalar, 3 first, 6
 * second and 10 third derivatives in the order xxx,xxy,xxz,xyy,xyz,xzz,yyy,yyz,yzz,zzz). */
int qmmm_get_potential(qmmm_handle *h, double *v);

/* Timing of the kernels launched by the last call (milliseconds, CUDA events on the handle's
 * stream): out[0] region-I V or its adjoint sweep, out[1] everything else in the call.
 * Returns the number of values written (2). */
int qmmm_last_timing(const qmmm_handle *h, double *out);

/* QM-QM periodic images (Eq. 5, summed by Ewald as in Eq. 6): the interaction of the QM
 * Mulliken multipoles at density dm with all their periodic images, minus the reference-cell
 * pairs (the QM calculation's own), with the tin-foil boundary and, for a charged QM cell, the
 * neutralising background -pi/(2 V kappa^2) (sum Q)^2:
 *   E = 1/2 sum_{j,i} sum_{L != 0} [Q_j Q_i T + 2 mu_j.Q_i T_a + 2 theta_j:Q_i T_ab - 2 mu_j mu_i:T_ab]
 * at R_j - R_i + L (readings: the dipole-charge and quadrupole-charge weights 2 and the
 * dipole-dipole sign follow from the lattice energy of point multipoles; Eq. 5 prints 1, 1, +2).
 * E[1]; dE_dRqm[natm*3], its gradient at fixed density (image tensors and the Pulay term of the
 * moving basis); F[nao*nao], dE/dgamma (nullable).  Not part of E from qmmm_energy: add it when the
 * QM cell's images are to be included.  Arrays: host or device memory. */
int qmmm_qm_images(qmmm_handle *h, const double *dm, double *E, double *dE_dRqm, double *F);

/* Density predictor for MD (Sec. "Common Setup": the always-stable predictor-corrector of the
 * one-particle density matrix from the K+1 preceding steps, used as the SCF guess and to set
 * region I on the fly):  out = sum_{j=1}^{K+1} B_j hist[j-1],
 *   B_j = (-1)^(j+1) j C(2K+2, K+1-j) / C(2K, K),  K = nhist - 1, 1 <= nhist <= 9
 * (nhist = 4 as in the paper: B = 2.8, -2.8, 1.2, -0.2).  hist[0] is the most recent density.
 * hist[*] and out: DEVICE arrays of n doubles; queued on `stream`, returns without waiting. */
int qmmm_aspc_predict(int nhist, const double *const *hist, size_t n, double *out, void *stream);

/* Octupole error estimate of the multipole truncation (Sec. "Error Control"): the leading error
 * of keeping region-II interactions to quadrupole order is the charge-octupole interaction
 *   Err(R) = sum_{i in II} sum_j sum_abc Omega_j,abc q_i T_ji,abc,
 * Omega_j the Mulliken octupoles (SI, fourth multipole definition) at density dm.  The sum over
 * region II is taken in the same periodic (Ewald) form as the l <= 2 terms: Err(R) = sum_j
 * Omega_j : v_j^(3)(R), with v^(3) the third Taylor components of the region-II potential (T_abc =
 * 1/6 d^3) when region I is the sphere of radius R about the QM centre; the Ewald real-space cutoff
 * stays the handle's.  err[k] = Err(r_lo + k dr), k = 0..n-1 (1 <= n <= 65536, dr > 0, bohr),
 * obtained from the handle's current region-II potential by moving the images between radius R
 * and the handle's cutoff.  octupoles[natm*10] (NULL: not returned) in the order xxx, xxy, xxz,
 * xyy, xyz, xzz, yyy, yyz, yzz, zzz.  dm[nao*nao], err, octupoles: host or device memory. */
int qmmm_octupole_error(qmmm_handle *h, const double *dm, double r_lo, double dr, int n, double *err,
                        double *octupoles);

/* On-the-fly region-I radius (same section): the smallest R_k = r_lo + k dr, k < n, with
 * |Err(R_k)| < eps; *rcut = R_k (or -1 if none), *err_at = Err(R_k) (nullable).  The handle's own
 * cutoff is not changed: create a handle with the new radius to use it. */
int qmmm_rcut_search(qmmm_handle *h, const double *dm, double r_lo, double dr, int n, double eps, double *rcut,
                     double *err_at);

/* Autotuner (the paper has no counterpart: its integrals come from a library).  The region-I
 * sweeps run one kernel per angular class (l_A, l_B), all classes at once on their own streams,
 * each with a cap on its grid -- its share of the SMs -- and a block shape.  By default the
 * shares follow a flop model of each class's work and every class uses 256-thread blocks.
 * qmmm_autotune times each class kernel alone on this handle's geometry, in each block shape
 * it has (256 threads, or a wider block where registers allow: more pair tiles per CTA on the
 * same staged charges), keeps the faster shape, sets each class's share in proportion to its
 * measured SM-time so that the classes finish together, and keeps the tuned configuration only
 * if the concurrent sweep is faster than the untuned one.
 *   flags: QMMM_TUNE_V and/or QMMM_TUNE_FORCES select the V and adjoint sweeps (0 = both);
 *   QMMM_TUNE_BOTH_PRECISIONS tunes the FP64 and the mixed kernels, else the current precision.
 * Needs a geometry (qmmm_create / qmmm_set_positions).  It works in scratch buffers with a zero
 * density: results of earlier calls stay valid, and results of later calls are unchanged apart
 * from the order of floating-point atomic additions.  It synchronises the handle's stream and
 * takes of the order of 20 sweep launches per tuned kernel.  The tuning is kept until
 * qmmm_set_positions changes region I's size by more than a quarter, when it resets to the model. */
enum { QMMM_TUNE_V = 1, QMMM_TUNE_FORCES = 2, QMMM_TUNE_BOTH_PRECISIONS = 4 };
int qmmm_autotune(qmmm_handle *h, int flags);

/* The sweep configuration in use for one kernel kind (0 V FP64, 1 V mixed, 2 adjoint FP64,
 * 3 adjoint mixed), per angular class in the order (0,0) (1,0) (1,1) (2,0) (2,1) (2,2) (3,0)
 * (3,1) (3,2) (3,3): threads[10] per block, share[10] = grid cap (SMs; 0 for an empty class),
 * ms[10] = the class's measured time alone at that share (0 if not measured), wide[10] = the
 * class's wide block size (0: it has only 256-thread blocks), weight[10] = the SM-time per
 * primitive pair that sets the shares (ms x blocks / pairs when tuned, the flop model if not;
 * qmmm_set_tuning accepts it back, e.g. to share one frame's tuning with similar frames).  Any
 * array may be NULL.  Returns 1 if the kind was tuned, 0 if it runs the model configuration, <0
 * on error. */
int qmmm_get_tuning(const qmmm_handle *h, int kind, int *threads, int *share, double *ms, int *wide,
                    double *weight);

/* Install a sweep configuration (e.g. one saved from qmmm_get_tuning on an earlier run of the
 * same system): threads[10] per class must be 256 or that class's wide block size (the values
 * qmmm_get_tuning can report); weight[10] (NULL = the flop model) is each class's SM-time per
 * primitive pair, in any common unit, from which the SM shares follow.  QMMM_ERR_ARG if a block
 * size is not available for its class or a weight is not positive. */
int qmmm_set_tuning(qmmm_handle *h, int kind, const int *threads, const double *weight);

/* ---------------------------------------------------------------------------------------------
 * Batches of independent systems (MD frames or sampling replicas of uneven sizes).  The paper
 * runs one system per process; this groups F handles (each from qmmm_create, each with its own
 * geometry, basis and charges) so that one call evaluates, for every frame, V (Eq. 9), the
 * energy E[4] as qmmm_energy, and the gradient as qmmm_forces, at that frame's density.
 *
 * qmmm_batch_run records the whole batch once into a CUDA graph -- every frame on its own stream
 * -- and from then on launches the graph: one launch per call, no host work per kernel.  The
 * region-I sweeps of the mixed-precision frames are batched: per angular class one launch of the
 * V sweep and one of each adjoint kernel over all those frames (job tables in device memory,
 * written before the recording), beside the frames' multipole and Ewald work; FP64 frames run
 * their own sweeps on their class streams.  Before recording it runs the batch once through the plain calls (which
 * sizes every buffer and sets every kernel attribute); the graph is recorded again when a frame's
 * region-I size, precision, sweep configuration or any array pointer differs from the recorded
 * one (see qmmm_batch_counts).  Positions change through qmmm_set_positions on the frame's
 * handle between runs.
 *
 * qmmm_batch_create: frames[nframes] (borrowed: they must outlive the batch and must not be used
 * on their own while the batch runs), stream = cudaStream_t as void* (NULL: the batch creates its
 * own stream, since the legacy stream cannot be recorded).
 * qmmm_batch_run: per frame f, DEVICE pointers dm[f] (nao_f^2, input), V[f] (nao_f^2),
 * E[f] (4 doubles), dE_dRqm[f] (natm_f*3), dE_dRmm[f] (nmm_f*3), dE_dq[f] (nmm_f); each of the
 * output pointer arrays may be NULL (that output is not written) and so may single entries.
 * Host memory is rejected (QMMM_ERR_ARG): a recorded graph cannot copy to pageable memory.  The
 * call returns after the graph has finished and every frame's device error flag is checked.
 * qmmm_batch_timing: ms[0] = the last run (graph launch to last frame done), ms[1 + f] = the time
 * at which frame f's outputs were complete, measured from the same start; returns nframes + 1. */
typedef struct qmmm_batch qmmm_batch;
int qmmm_batch_create(qmmm_handle *const *frames, int nframes, void *stream, qmmm_batch **out);
int qmmm_batch_run(qmmm_batch *b, const double *const *dm, double *const *V, double *const *E,
                   double *const *dE_dRqm, double *const *dE_dRmm, double *const *dE_dq);
int qmmm_batch_timing(const qmmm_batch *b, double *ms);
/* Number of graph recordings so far (1 after the first run when nothing changes). */
int qmmm_batch_captures(const qmmm_batch *b);
/* Recordings, instantiations and in-place updates of the batch graph so far.  After new
 * positions (an MD step) the batch is recorded again without the plain pass -- unless a frame's
 * region I outgrew its buffers -- and, when only launch parameters changed (sizes, grids,
 * pointers), the instantiated graph is updated in place instead of instantiated anew. */
int qmmm_batch_counts(const qmmm_batch *b, int *recorded, int *instantiated, int *updated);
void qmmm_batch_destroy(qmmm_batch *b);

/* Self-test of the failure path (no counterpart in the paper).  Every wait in the kernels (the
 * mbarrier that completes a TMA bulk copy) gives up after 0.5 s of wall time and then records a
 * device error flag and returns, which the call reports as QMMM_ERR_TIMEOUT with the CUDA context
 * still usable.  This launches one block that waits on an mbarrier nothing completes; it returns
 * QMMM_ERR_TIMEOUT when the failure path works (after a 20 ms wait); it never faults or hangs.
 * stream: a cudaStream_t as void* (NULL = legacy stream). */
int qmmm_selftest_bounded_wait(void *stream);

void qmmm_destroy(qmmm_handle *h);
const char *qmmm_strerror(int code);
const char *qmmm_last_error(void);

/* Allocation-free nuclear-MM energy, for callers that must not allocate device memory while
 * they run (an MD engine that reserves all its device memory at start-up and calls this from its
 * time step, where a cudaMalloc would implicitly synchronise the device; a plugin whose memory
 * belongs to the host program's pool allocator).  The paper has no counterpart: it is a variant
 * of the kernel behind qmmm_vpot's E_nuc_mm, taking the charges directly instead of a handle.
 *   E[0] = sum_j sum_i Z[j] q_i erf(r_ij / sigma[i]) / r_ij  (1/r_ij where sigma[i] <= 0),
 *   with the limit 2 / (sigma[i] sqrt(pi)) for a Gaussian charge centred on a nucleus; a point
 *   charge on a nucleus makes E non-finite (+-inf or NaN), as the energy is;
 *   qm_xyz[natm*3], Z[natm], charges[ncharge*4] = (x, y, z, q) per charge (bohr, e),
 *   sigma[ncharge] (bohr), E[1]: all DEVICE memory owned by the caller.  Work is queued on
 *   `stream` (a cudaStream_t; NULL = legacy stream) and the call returns without waiting.
 * Scratch is a fixed array inside the library (one double per 256 charges, at most 262144
 * charges per call: larger ncharge returns QMMM_ERR_ARG); every GPU that loads the library holds
 * it until the process exits.  The first call on each device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current; make that first call before any stream
 * capture.  All calls on a device share the array, so calls whose work overlaps on the GPU race
 * and give wrong results: serialise them (one stream, or events).  Nothing is allocated or freed.
 * Errors: QMMM_ERR_ARG (null/host pointer, negative or too large size), QMMM_ERR_CUDA. */
int qmmm_nuclear_mm_energy_static(int natm, const double *qm_xyz, const double *Z, int ncharge,
                                  const double *charges, const double *sigma, double *E, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* QMMM_H */
