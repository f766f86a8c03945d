/*
 * qmmm_oracle.c -- plain, slow, FP64 CPU oracle for the periodic QM/MM-Multipole embedding
 * (arXiv 2408.03273).  TEST INFRASTRUCTURE ONLY: the tests, the package smoke check and the
 * CPU-baseline leg of the benchmark call it; the CUDA library never links or calls it, and it
 * shares no code, header or table with the CUDA path.
 *
 * What it computes, each piece citing the passage it follows:
 *   - Boys function F_n(T) by its power series and its large-T asymptotic form.
 *   - Region-I one-electron integrals over Gaussian-smeared MM charges, Eq. 9 (point-charge
 *     form Eq. 2), by Obara-Saika vertical recursion on (e0|s) and the Head-Gordon-Pople
 *     horizontal recursion.  The Gaussian charge is a normalised s function of exponent
 *     kappa = 1/sigma^2; sigma <= 0 is the point-charge limit.
 *   - Mulliken charge / dipole / (non-traceless) quadrupole, SI Sec. "Multipolar Ewald"
 *     (first equations), with moment integrals from the Obara-Saika three-centre overlap
 *     recursion (operator centre treated as a zero-exponent Gaussian).
 *   - Multipole interaction tensors T (SI, point tensors), T-hat (SI, Gaussian-screened
 *     tensors built from f1..f7) and the Ewald tensors psi = psi_SR + psi_LR (SI, Ewald for
 *     multipoles) with a neutralising background.
 *   - The QM-MM part of Eq. 6 plus the Gaussian correction Eq. 10, the Fock term Eqs. 11-14 and
 *     the nuclear gradient (region-I integral derivatives, tensor derivatives, and the
 *     multipole Pulay term Eq. 15).
 *
 * Readings of the paper taken here (all listed in the design notes of the repository):
 *   psi_LR_ab uses prefactor 2*pi/V and exp(-G^2/(4 kappa^2)) (the printed 4*pi/V and
 *   exp(-G^2/(2 kappa^2)) contradict the derivative of psi_LR_a);  the Gaussian width enters
 *   T-hat as erfc(r/sigma)/r;  the neutralising background adds -pi/(V kappa^2) to psi;  the
 *   region-I nuclear-MM term sum_j Z_j q_i erf(r/sigma)/r is part of the exact region-I energy;
 *   region I is the set of MM images with |R_i + L - c| < R_cut, c the unweighted mean of the QM
 *   positions.
 *
 * Units: atomic units.  Cartesian order inside a shell: lexicographic (xx,xy,xz,yy,yz,zz).
 * Tensor component order (20): [0] scalar, [1..3] x,y,z, [4..9] xx,xy,xz,yy,yz,zz,
 * [10..19] xxx,xxy,xxz,xyy,xyz,xzz,yyy,yyz,yzz,zzz.  Multipoles (10): Q, mu_xyz, theta_(6).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_PI 3.14159265358979323846
#define LMAXT 9 /* highest total angular momentum handled by the recursions */

/* ------------------------------------------------------------------------------------------ */
/* Boys function                                                                                */
/* ------------------------------------------------------------------------------------------ */

/* F_n(T) = int_0^1 t^{2n} exp(-T t^2) dt.
 * Small T (< 50): F_n(T) = exp(-T) sum_k (2T)^k / [(2n+1)(2n+3)...(2n+2k+1)]  (all terms
 * positive, no cancellation).
 * Large T: F_0(T) = 1/2 sqrt(pi/T) erf(sqrt T) (the asymptotic form, erfc(sqrt T) < 1e-22 there)
 * and the exact upward relation F_{n+1} = ((2n+1) F_n - exp(-T)) / (2T), stable for large T. */
void oracle_boys(int nmax, double T, double *F)
{
    if (T < 50.0) {
        for (int n = 0; n <= nmax; n++) {
            double term = 1.0 / (2.0 * n + 1.0), sum = term;
            for (int k = 1; k < 2000; k++) {
                term *= 2.0 * T / (2.0 * n + 2.0 * k + 1.0);
                sum += term;
                if (term < 1e-18 * sum) break;
            }
            F[n] = exp(-T) * sum;
        }
    } else {
        double e = exp(-T);
        F[0] = 0.5 * sqrt(OR_PI / T);
        for (int n = 0; n < nmax; n++) F[n + 1] = ((2.0 * n + 1.0) * F[n] - e) / (2.0 * T);
    }
}

/* ------------------------------------------------------------------------------------------ */
/* basis helpers                                                                                */
/* ------------------------------------------------------------------------------------------ */

static int ncart(int l) { return (l + 1) * (l + 2) / 2; }

/* Cartesian exponents of shell l in lexicographic order. */
static void cart_comp(int l, int (*c)[3])
{
    int k = 0;
    for (int lx = l; lx >= 0; lx--)
        for (int ly = l - lx; ly >= 0; ly--) {
            c[k][0] = lx; c[k][1] = ly; c[k][2] = l - lx - ly; k++;
        }
}

static double dfact_odd(int n) /* (2n-1)!!, with (-1)!! = 1 */
{
    double r = 1.0;
    for (int k = 2 * n - 1; k > 1; k -= 2) r *= k;
    return r;
}

/* Normalised contraction coefficients: each primitive carries the factor that normalises its
 * x^l component, (2a/pi)^{3/4} (4a)^{l/2} / sqrt((2l-1)!!), and the contracted x^l function is
 * renormalised to one.  The same factor multiplies every Cartesian component. */
void oracle_norm_coeffs(int nshell, const int *shell_l, const int *shell_nprim, const int *shell_off,
                        const double *exps, const double *coeffs, double *out)
{
    for (int s = 0; s < nshell; s++) {
        int l = shell_l[s], n = shell_nprim[s], o = shell_off[s];
        for (int k = 0; k < n; k++) {
            double a = exps[o + k];
            out[o + k] = coeffs[o + k] * pow(2.0 * a / OR_PI, 0.75) * pow(4.0 * a, 0.5 * l) / sqrt(dfact_odd(l));
        }
        double ss = 0.0;
        for (int k = 0; k < n; k++)
            for (int m = 0; m < n; m++) {
                double p = exps[o + k] + exps[o + m];
                ss += out[o + k] * out[o + m] * dfact_odd(l) / pow(2.0 * p, l) * pow(OR_PI / p, 1.5);
            }
        for (int k = 0; k < n; k++) out[o + k] /= sqrt(ss);
    }
}

/* ------------------------------------------------------------------------------------------ */
/* three-centre integral (a b | Gaussian charge) by Obara-Saika + HRR                           */
/* ------------------------------------------------------------------------------------------ */

typedef struct {
    double v[LMAXT + 1][LMAXT + 1][LMAXT + 1][LMAXT + 1]; /* [m][ex][ey][ez] */
    double AB[3];
} os_work;

/* Vertical recursion (Obara-Saika) for [e 0 | s]^(m), |e| <= ltot, Gaussian-charge ket.
 *   [e+1_i]^(m) = PA_i [e]^(m) + WP_i [e]^(m+1) + e_i/(2p) ([e-1_i]^(m) - rho/p [e-1_i]^(m+1))
 * base [0]^(m) = (2 pi / p) sqrt(kappa/(p+kappa)) K_AB F_m(rho |PC|^2), rho = p kappa/(p+kappa),
 * W = (p P + kappa C)/(p + kappa).  kappa <= 0 selects the point charge (rho = p, W = C). */
static void os_vrr(os_work *w, int ltot, double a, const double *A, double b, const double *B,
                   double kappa, const double *C)
{
    double p = a + b, P[3], PA[3], WP[3], rho, pref, F[LMAXT + 2];
    double AB2 = 0.0;
    for (int i = 0; i < 3; i++) {
        P[i] = (a * A[i] + b * B[i]) / p;
        PA[i] = P[i] - A[i];
        w->AB[i] = A[i] - B[i];
        AB2 += w->AB[i] * w->AB[i];
    }
    double KAB = exp(-a * b / p * AB2);
    if (kappa > 0.0) {
        rho = p * kappa / (p + kappa);
        pref = 2.0 * OR_PI / p * sqrt(kappa / (p + kappa)) * KAB;
        for (int i = 0; i < 3; i++) WP[i] = (p * P[i] + kappa * C[i]) / (p + kappa) - P[i];
    } else {
        rho = p;
        pref = 2.0 * OR_PI / p * KAB;
        for (int i = 0; i < 3; i++) WP[i] = C[i] - P[i];
    }
    double PC2 = 0.0;
    for (int i = 0; i < 3; i++) PC2 += (P[i] - C[i]) * (P[i] - C[i]);
    oracle_boys(ltot, rho * PC2, F);
    for (int m = 0; m <= ltot; m++) w->v[m][0][0][0] = pref * F[m];
    for (int n = 1; n <= ltot; n++) {
        for (int ex = n; ex >= 0; ex--)
            for (int ey = n - ex; ey >= 0; ey--) {
                int ez = n - ex - ey, e[3] = {ex, ey, ez};
                int i = ex > 0 ? 0 : (ey > 0 ? 1 : 2);
                int e1[3] = {ex, ey, ez}, e2[3] = {ex, ey, ez};
                e1[i] -= 1; e2[i] -= 2;
                for (int m = 0; m <= ltot - n; m++) {
                    double val = PA[i] * w->v[m][e1[0]][e1[1]][e1[2]] + WP[i] * w->v[m + 1][e1[0]][e1[1]][e1[2]];
                    if (e[i] >= 2)
                        val += (e[i] - 1) / (2.0 * p) *
                               (w->v[m][e2[0]][e2[1]][e2[2]] - rho / p * w->v[m + 1][e2[0]][e2[1]][e2[2]]);
                    w->v[m][ex][ey][ez] = val;
                }
            }
    }
}

/* Horizontal recursion (Head-Gordon-Pople): [a, b+1_i| = [a+1_i, b| + AB_i [a, b|. */
static double os_hrr(const os_work *w, const int *a, const int *b)
{
    int i = b[0] > 0 ? 0 : (b[1] > 0 ? 1 : (b[2] > 0 ? 2 : -1));
    if (i < 0) return w->v[0][a[0]][a[1]][a[2]];
    int a1[3] = {a[0], a[1], a[2]}, b1[3] = {b[0], b[1], b[2]};
    a1[i] += 1; b1[i] -= 1;
    return os_hrr(w, a1, b1) + w->AB[i] * os_hrr(w, a, b1);
}

/* Unnormalised primitive block out[ncart(la)][ncart(lb)] = <g_a g_b | phi_C> (Gaussian charge of
 * exponent kappa, normalised; kappa <= 0: point charge 1/|r-C|). */
void oracle_int3c_prim(int la, int lb, double a, const double *A, double b, const double *B,
                       double kappa, const double *C, double *out)
{
    os_work *w = (os_work *)malloc(sizeof(os_work));
    os_vrr(w, la + lb, a, A, b, B, kappa, C);
    int ca[36][3], cb[36][3];
    cart_comp(la, ca); cart_comp(lb, cb);
    for (int i = 0; i < ncart(la); i++)
        for (int j = 0; j < ncart(lb); j++) out[i * ncart(lb) + j] = os_hrr(w, ca[i], cb[j]);
    free(w);
}

/* ------------------------------------------------------------------------------------------ */
/* region-I V matrix (Eq. 9), electronic gradient, nuclear-MM region-I term                     */
/* ------------------------------------------------------------------------------------------ */

static void ao_offsets(int nshell, const int *shell_l, int *off)
{
    int o = 0;
    for (int s = 0; s < nshell; s++) { off[s] = o; o += ncart(shell_l[s]); }
}

static double charge_kappa(double sigma) { return sigma > 0.0 ? 1.0 / (sigma * sigma) : 0.0; }

/* V[mu,nu] = - sum_C q_C <mu nu | phi_C> over the given charges (positions already imaged).
 * If pairs != NULL only the ordered shell pairs (pairs[2k], pairs[2k+1]) are evaluated and only
 * their blocks of V are written (the rest is left untouched); otherwise every ordered pair.
 * ncoef are normalised coefficients from oracle_norm_coeffs. */
void oracle_vpot(int nshell, const int *shell_atom, const int *shell_l, const int *shell_nprim,
                 const int *shell_off, const double *exps, const double *ncoef, const double *qm_xyz,
                 int nchg, const double *c_xyz, const double *c_q, const double *c_sigma,
                 int npairs, const int *pairs, int nao, double *V)
{
    int *aoff = (int *)malloc(sizeof(int) * nshell);
    ao_offsets(nshell, shell_l, aoff);
    long ntask = pairs ? npairs : (long)nshell * nshell;
#pragma omp parallel
    {
        os_work *w = (os_work *)malloc(sizeof(os_work));
#pragma omp for schedule(dynamic, 1)
        for (long t = 0; t < ntask; t++) {
            int sA = pairs ? pairs[2 * t] : (int)(t / nshell);
            int sB = pairs ? pairs[2 * t + 1] : (int)(t % nshell);
            int la = shell_l[sA], lb = shell_l[sB], na = ncart(la), nb = ncart(lb);
            int ca[36][3], cb[36][3];
            cart_comp(la, ca); cart_comp(lb, cb);
            const double *A = qm_xyz + 3 * shell_atom[sA], *B = qm_xyz + 3 * shell_atom[sB];
            double blk[100];
            memset(blk, 0, sizeof(blk));
            for (int ka = 0; ka < shell_nprim[sA]; ka++)
                for (int kb = 0; kb < shell_nprim[sB]; kb++) {
                    double a = exps[shell_off[sA] + ka], b = exps[shell_off[sB] + kb];
                    double cc = ncoef[shell_off[sA] + ka] * ncoef[shell_off[sB] + kb];
                    for (int c = 0; c < nchg; c++) {
                        os_vrr(w, la + lb, a, A, b, B, charge_kappa(c_sigma[c]), c_xyz + 3 * c);
                        for (int i = 0; i < na; i++)
                            for (int j = 0; j < nb; j++) blk[i * nb + j] -= c_q[c] * cc * os_hrr(w, ca[i], cb[j]);
                    }
                }
            for (int i = 0; i < na; i++)
                for (int j = 0; j < nb; j++) V[(long)(aoff[sA] + i) * nao + aoff[sB] + j] = blk[i * nb + j];
        }
        free(w);
    }
    free(aoff);
}

/* Electronic region-I gradient at fixed density for the given charges.
 *   E = sum_{mu nu} dm[mu,nu] V[mu,nu].
 * d/dA of a primitive: 2a [a+1_i| - a_i [a-1_i|;  d/dC = -(d/dA + d/dB) (translation).
 * Outputs are accumulated (+=): dRqm[natm*3], dC[nchg*3], dq[nchg].  Ordered shell pairs. */
void oracle_vgrad(int nshell, const int *shell_atom, const int *shell_l, const int *shell_nprim,
                  const int *shell_off, const double *exps, const double *ncoef, int natm,
                  const double *qm_xyz, int nchg, const double *c_xyz, const double *c_q,
                  const double *c_sigma, int nao, const double *dm, int npairs, const int *pairs,
                  double *dRqm, double *dC, double *dq)
{
    /* pairs != NULL: only the listed ordered shell pairs contribute (a sampling convenience;
     * the full gradient sums every ordered pair). */
    int *aoff = (int *)malloc(sizeof(int) * nshell);
    ao_offsets(nshell, shell_l, aoff);
    int nthr = 1;
#ifdef _OPENMP
    nthr = omp_get_max_threads();
#endif
    double *accR = (double *)calloc((size_t)nthr * natm * 3, sizeof(double));
    double *accC = (double *)calloc((size_t)nthr * nchg * 4, sizeof(double));
#pragma omp parallel
    {
        int tid = 0;
#ifdef _OPENMP
        tid = omp_get_thread_num();
#endif
        double *myR = accR + (size_t)tid * natm * 3, *myC = accC + (size_t)tid * nchg * 4;
        os_work *w = (os_work *)malloc(sizeof(os_work));
        long ntask = pairs ? npairs : (long)nshell * nshell;
#pragma omp for schedule(dynamic, 1)
        for (long t = 0; t < ntask; t++) {
            int sA = pairs ? pairs[2 * t] : (int)(t / nshell);
            int sB = pairs ? pairs[2 * t + 1] : (int)(t % nshell);
            int la = shell_l[sA], lb = shell_l[sB];
            int ca[36][3], cb[36][3];
            cart_comp(la, ca); cart_comp(lb, cb);
            const double *A = qm_xyz + 3 * shell_atom[sA], *B = qm_xyz + 3 * shell_atom[sB];
            for (int ka = 0; ka < shell_nprim[sA]; ka++)
                for (int kb = 0; kb < shell_nprim[sB]; kb++) {
                    double a = exps[shell_off[sA] + ka], b = exps[shell_off[sB] + kb];
                    double cc = ncoef[shell_off[sA] + ka] * ncoef[shell_off[sB] + kb];
                    for (int c = 0; c < nchg; c++) {
                        os_vrr(w, la + lb + 1, a, A, b, B, charge_kappa(c_sigma[c]), c_xyz + 3 * c);
                        double e0 = 0.0, gA[3] = {0, 0, 0}, gB[3] = {0, 0, 0};
                        for (int i = 0; i < ncart(la); i++)
                            for (int j = 0; j < ncart(lb); j++) {
                                double d = dm[(long)(aoff[sA] + i) * nao + aoff[sB] + j] * cc;
                                if (d == 0.0) continue;
                                e0 += d * os_hrr(w, ca[i], cb[j]);
                                for (int x = 0; x < 3; x++) {
                                    int ap[3] = {ca[i][0], ca[i][1], ca[i][2]}, am[3] = {ca[i][0], ca[i][1], ca[i][2]};
                                    int bp[3] = {cb[j][0], cb[j][1], cb[j][2]}, bm[3] = {cb[j][0], cb[j][1], cb[j][2]};
                                    ap[x]++; am[x]--; bp[x]++; bm[x]--;
                                    double da = 2.0 * a * os_hrr(w, ap, cb[j]);
                                    if (ca[i][x] > 0) da -= ca[i][x] * os_hrr(w, am, cb[j]);
                                    double db = 2.0 * b * os_hrr(w, ca[i], bp);
                                    if (cb[j][x] > 0) db -= cb[j][x] * os_hrr(w, ca[i], bm);
                                    gA[x] += d * da;
                                    gB[x] += d * db;
                                }
                            }
                        /* V = -q <..>, so every term carries -q */
                        double q = c_q[c];
                        myC[4 * c + 3] -= e0;
                        for (int x = 0; x < 3; x++) {
                            myR[3 * shell_atom[sA] + x] -= q * gA[x];
                            myR[3 * shell_atom[sB] + x] -= q * gB[x];
                            myC[4 * c + x] += q * (gA[x] + gB[x]);
                        }
                    }
                }
        }
        free(w);
    }
    for (int t = 0; t < nthr; t++) {
        for (int i = 0; i < natm * 3; i++) dRqm[i] += accR[(size_t)t * natm * 3 + i];
        for (int c = 0; c < nchg; c++) {
            for (int x = 0; x < 3; x++) dC[3 * c + x] += accC[(size_t)t * nchg * 4 + 4 * c + x];
            dq[c] += accC[(size_t)t * nchg * 4 + 4 * c + 3];
        }
    }
    free(accR); free(accC); free(aoff);
}

/* Region-I nuclear-MM energy sum_j sum_C Z_j q_C erf(r/sigma_C)/r (1/r for point charges) and
 * its derivatives (accumulated).  Returns the energy. */
double oracle_enucmm(int natm, const double *qm_xyz, const double *Z, int nchg, const double *c_xyz,
                     const double *c_q, const double *c_sigma, double *dRqm, double *dC, double *dq)
{
    double E = 0.0;
    for (int j = 0; j < natm; j++)
        for (int c = 0; c < nchg; c++) {
            double d[3], r2 = 0.0;
            for (int x = 0; x < 3; x++) { d[x] = qm_xyz[3 * j + x] - c_xyz[3 * c + x]; r2 += d[x] * d[x]; }
            double r = sqrt(r2), f, fp; /* f(r) and f'(r) */
            if (c_sigma[c] > 0.0) {
                double s = 1.0 / c_sigma[c];
                f = erf(s * r) / r;
                fp = (2.0 * s / sqrt(OR_PI) * exp(-s * s * r2) - f) / r;
            } else {
                f = 1.0 / r;
                fp = -1.0 / r2;
            }
            E += Z[j] * c_q[c] * f;
            if (dq) dq[c] += Z[j] * f;
            for (int x = 0; x < 3; x++) {
                double g = Z[j] * c_q[c] * fp * d[x] / r;
                if (dRqm) dRqm[3 * j + x] += g;
                if (dC) dC[3 * c + x] -= g;
            }
        }
    return E;
}

/* ------------------------------------------------------------------------------------------ */
/* moment integrals, Mulliken multipoles, Fock term, Pulay gradient                            */
/* ------------------------------------------------------------------------------------------ */

/* 1-D Obara-Saika overlap with a zero-exponent third factor (x-K)^e:
 *   S[i][j][e] = int (x-A)^i (x-B)^j (x-K)^e exp(-a(x-A)^2 - b(x-B)^2) dx. */
static void os_overlap1d(int imax, int jmax, int emax, double a, double Ax, double b, double Bx, double Kx,
                         double S[LMAXT + 2][LMAXT + 2][4])
{
    double p = a + b, Px = (a * Ax + b * Bx) / p, XAB = Ax - Bx;
    double XPA = Px - Ax, XPB = Px - Bx, XPK = Px - Kx;
    memset(S, 0, sizeof(double) * (LMAXT + 2) * (LMAXT + 2) * 4);
    for (int e = 0; e <= emax; e++)
        for (int i = 0; i <= imax; i++)
            for (int j = 0; j <= jmax; j++) {
                double v;
                if (i == 0 && j == 0 && e == 0) v = sqrt(OR_PI / p) * exp(-a * b / p * XAB * XAB);
                else if (i > 0) {
                    v = XPA * S[i - 1][j][e];
                    double t = 0.0;
                    if (i > 1) t += (i - 1) * S[i - 2][j][e];
                    if (j > 0) t += j * S[i - 1][j - 1][e];
                    if (e > 0) t += e * S[i - 1][j][e - 1];
                    v += t / (2.0 * p);
                } else if (j > 0) {
                    v = XPB * S[i][j - 1][e];
                    double t = 0.0;
                    if (j > 1) t += (j - 1) * S[i][j - 2][e];
                    if (e > 0) t += e * S[i][j - 1][e - 1];
                    v += t / (2.0 * p);
                } else {
                    v = XPK * S[i][j][e - 1];
                    if (e > 1) v += (e - 1) * S[i][j][e - 2] / (2.0 * p);
                }
                S[i][j][e] = v;
            }
}

/* operator exponent table for the 10 multipole operators 1, x, y, z, xx, xy, xz, yy, yz, zz */
static const int OPX[10][3] = {{0, 0, 0}, {1, 0, 0}, {0, 1, 0}, {0, 0, 1}, {2, 0, 0},
                               {1, 1, 0}, {1, 0, 1}, {0, 2, 0}, {0, 1, 1}, {0, 0, 2}};

/* Contracted moment block <mu| (r-K)^op |nu> for shells sA, sB, all 10 operators, optionally with
 * nu's angular momentum shifted: out[op][i][j] with j over ncart(lb + dlb) (dlb in {-1,0,1}) and
 * the primitive factor (2b)^{dlb==1} for derivative use handled by the caller. */
static void moment_block(int la, int lb_eff, const double *A, const double *B, const double *K,
                         int nA, const double *expA, const double *cA, int nB, const double *expB,
                         const double *cB, double bscale_pow, double *out /* [10][36][36] */)
{
    int ca[36][3], cb[66][3];
    cart_comp(la, ca);
    if (lb_eff >= 0) cart_comp(lb_eff, cb);
    int na = ncart(la), nb = lb_eff >= 0 ? ncart(lb_eff) : 0;
    memset(out, 0, sizeof(double) * 10 * 36 * 36);
    if (lb_eff < 0) return;
    static double Sx[LMAXT + 2][LMAXT + 2][4], Sy[LMAXT + 2][LMAXT + 2][4], Sz[LMAXT + 2][LMAXT + 2][4];
#pragma omp threadprivate(Sx, Sy, Sz)
    for (int ka = 0; ka < nA; ka++)
        for (int kb = 0; kb < nB; kb++) {
            double a = expA[ka], b = expB[kb];
            double cc = cA[ka] * cB[kb] * pow(2.0 * b, bscale_pow);
            os_overlap1d(la, lb_eff, 2, a, A[0], b, B[0], K[0], Sx);
            os_overlap1d(la, lb_eff, 2, a, A[1], b, B[1], K[1], Sy);
            os_overlap1d(la, lb_eff, 2, a, A[2], b, B[2], K[2], Sz);
            for (int op = 0; op < 10; op++)
                for (int i = 0; i < na; i++)
                    for (int j = 0; j < nb; j++)
                        out[(op * 36 + i) * 36 + j] += cc * Sx[ca[i][0]][cb[j][0]][OPX[op][0]] *
                                                       Sy[ca[i][1]][cb[j][1]][OPX[op][1]] *
                                                       Sz[ca[i][2]][cb[j][2]][OPX[op][2]];
        }
}

/* Mulliken multipoles (SI, Multipolar Ewald):
 *   Q_k = Z_k - sum_{mu in k, nu} dm[nu,mu] <mu|nu>
 *   mu_k,a = - sum dm[nu,mu] <mu|(r-R_k)_a|nu>,  theta_k,ab = - sum dm[nu,mu] <mu|(r-R_k)_a (r-R_k)_b|nu>
 * out[natm*10]. */
void oracle_multipoles(int nshell, const int *shell_atom, const int *shell_l, const int *shell_nprim,
                       const int *shell_off, const double *exps, const double *ncoef, int natm,
                       const double *qm_xyz, const double *Z, int nao, const double *dm, double *out)
{
    int *aoff = (int *)malloc(sizeof(int) * nshell);
    ao_offsets(nshell, shell_l, aoff);
    double *blk = (double *)malloc(sizeof(double) * 10 * 36 * 36);
    for (int k = 0; k < natm; k++) {
        for (int c = 0; c < 10; c++) out[10 * k + c] = 0.0;
        out[10 * k] = Z[k];
    }
    for (int sA = 0; sA < nshell; sA++)
        for (int sB = 0; sB < nshell; sB++) {
            int k = shell_atom[sA];
            moment_block(shell_l[sA], shell_l[sB], qm_xyz + 3 * k, qm_xyz + 3 * shell_atom[sB], qm_xyz + 3 * k,
                         shell_nprim[sA], exps + shell_off[sA], ncoef + shell_off[sA], shell_nprim[sB],
                         exps + shell_off[sB], ncoef + shell_off[sB], 0.0, blk);
            for (int op = 0; op < 10; op++)
                for (int i = 0; i < ncart(shell_l[sA]); i++)
                    for (int j = 0; j < ncart(shell_l[sB]); j++)
                        out[10 * k + op] -= dm[(long)(aoff[sB] + j) * nao + aoff[sA] + i] * blk[(op * 36 + i) * 36 + j];
        }
    free(blk); free(aoff);
}

/* Mulliken octupoles (SI, Multipolar Ewald, fourth definition):
 *   Omega_k,abc = - sum_{mu in k, nu} dm[nu,mu] <mu|(r-R_k)_a (r-R_k)_b (r-R_k)_c|nu>
 * for the 10 unique components xxx, xxy, xxz, xyy, xyz, xzz, yyy, yyz, yzz, zzz; out[natm*10].
 * The moments are products of three 1-D Obara-Saika overlaps with the (x-K)^e factor, e <= 3. */
static const int OPX3[10][3] = {{3, 0, 0}, {2, 1, 0}, {2, 0, 1}, {1, 2, 0}, {1, 1, 1},
                                {1, 0, 2}, {0, 3, 0}, {0, 2, 1}, {0, 1, 2}, {0, 0, 3}};

void oracle_octupoles(int nshell, const int *shell_atom, const int *shell_l, const int *shell_nprim,
                      const int *shell_off, const double *exps, const double *ncoef, int natm,
                      const double *qm_xyz, int nao, const double *dm, double *out)
{
    int *aoff = (int *)malloc(sizeof(int) * nshell);
    ao_offsets(nshell, shell_l, aoff);
    for (int c = 0; c < 10 * natm; c++) out[c] = 0.0;
    static double Sx[LMAXT + 2][LMAXT + 2][4], Sy[LMAXT + 2][LMAXT + 2][4], Sz[LMAXT + 2][LMAXT + 2][4];
    for (int sA = 0; sA < nshell; sA++)
        for (int sB = 0; sB < nshell; sB++) {
            const int k = shell_atom[sA], la = shell_l[sA], lb = shell_l[sB];
            const double *A = qm_xyz + 3 * k, *B = qm_xyz + 3 * shell_atom[sB];
            int ca[36][3], cb[36][3];
            cart_comp(la, ca);
            cart_comp(lb, cb);
            for (int ka = 0; ka < shell_nprim[sA]; ka++)
                for (int kb = 0; kb < shell_nprim[sB]; kb++) {
                    const double a = exps[shell_off[sA] + ka], b = exps[shell_off[sB] + kb];
                    const double cc = ncoef[shell_off[sA] + ka] * ncoef[shell_off[sB] + kb];
                    os_overlap1d(la, lb, 3, a, A[0], b, B[0], A[0], Sx);
                    os_overlap1d(la, lb, 3, a, A[1], b, B[1], A[1], Sy);
                    os_overlap1d(la, lb, 3, a, A[2], b, B[2], A[2], Sz);
                    for (int i = 0; i < ncart(la); i++)
                        for (int j = 0; j < ncart(lb); j++) {
                            const double g = dm[(long)(aoff[sB] + j) * nao + aoff[sA] + i];
                            for (int op = 0; op < 10; op++)
                                out[10 * k + op] -= g * cc * Sx[ca[i][0]][cb[j][0]][OPX3[op][0]] *
                                                    Sy[ca[i][1]][cb[j][1]][OPX3[op][1]] *
                                                    Sz[ca[i][2]][cb[j][2]][OPX3[op][2]];
                        }
                }
        }
    free(aoff);
}

/* weight of the 10 stored components in a full (a,b) contraction: off-diagonal theta counts twice */
static const double W10[10] = {1, 1, 1, 1, 1, 2, 2, 1, 2, 1};

/* Fock contribution of region II, Eqs. 11-14:
 *   F[mu,nu] = -1/2 [ sum_c W_c phi_{k(mu)},c <mu|O_c^{k(mu)}|nu> + (mu<->nu) ]
 * phi[natm*10] holds (v, v_a, v_ab) per atom (the 10 first components of the potential). */
void oracle_fock_ii(int nshell, const int *shell_atom, const int *shell_l, const int *shell_nprim,
                    const int *shell_off, const double *exps, const double *ncoef, const double *qm_xyz,
                    const double *phi, int phi_stride, int nao, double *F)
{
    int *aoff = (int *)malloc(sizeof(int) * nshell);
    ao_offsets(nshell, shell_l, aoff);
    double *blk = (double *)malloc(sizeof(double) * 10 * 36 * 36);
    memset(F, 0, sizeof(double) * nao * nao);
    for (int sA = 0; sA < nshell; sA++)
        for (int sB = 0; sB < nshell; sB++) {
            int k = shell_atom[sA];
            moment_block(shell_l[sA], shell_l[sB], qm_xyz + 3 * k, qm_xyz + 3 * shell_atom[sB], qm_xyz + 3 * k,
                         shell_nprim[sA], exps + shell_off[sA], ncoef + shell_off[sA], shell_nprim[sB],
                         exps + shell_off[sB], ncoef + shell_off[sB], 0.0, blk);
            for (int i = 0; i < ncart(shell_l[sA]); i++)
                for (int j = 0; j < ncart(shell_l[sB]); j++) {
                    double v = 0.0;
                    for (int op = 0; op < 10; op++) v += W10[op] * phi[phi_stride * k + op] * blk[(op * 36 + i) * 36 + j];
                    long mu = aoff[sA] + i, nu = aoff[sB] + j;
                    F[mu * nao + nu] -= 0.5 * v;
                    F[nu * nao + mu] -= 0.5 * v;
                }
        }
    free(blk); free(aoff);
}

/* Multipole Pulay gradient, Eq. 15, written with the local potential polynomial
 * W_k(r) = sum_c W_c phi_k,c O_c(r - R_k):
 *   E_mult = sum_k Z_k phi_k,0 - sum_{mu in k, nu} dm[nu,mu] <mu|W_k|nu>.
 * Moving nu's centre B changes <mu|W_k|nu> by <mu|W_k|d nu/dB> with d g_b/dB_x =
 * 2b g_{b+1x} - b_x g_{b-1x}; translating atom k (mu and the operator centre) gives the
 * opposite change.  Accumulates into dRqm[natm*3]. */
void oracle_pulay(int nshell, const int *shell_atom, const int *shell_l, const int *shell_nprim,
                  const int *shell_off, const double *exps, const double *ncoef, const double *qm_xyz,
                  const double *phi, int phi_stride, int nao, const double *dm, double *dRqm)
{
    int *aoff = (int *)malloc(sizeof(int) * nshell);
    ao_offsets(nshell, shell_l, aoff);
    double *bp = (double *)malloc(sizeof(double) * 10 * 36 * 36);
    double *bm = (double *)malloc(sizeof(double) * 10 * 36 * 36);
    for (int sA = 0; sA < nshell; sA++)
        for (int sB = 0; sB < nshell; sB++) {
            int k = shell_atom[sA], kB = shell_atom[sB], la = shell_l[sA], lb = shell_l[sB];
            if (k == kB) continue; /* joint translation: no change */
            int ca[36][3], cb[36][3], cbp[36][3], cbm[36][3];
            cart_comp(la, ca); cart_comp(lb, cb); cart_comp(lb + 1, cbp);
            if (lb > 0) cart_comp(lb - 1, cbm);
            /* b+1 block carries the factor 2b per primitive; b-1 block plain */
            moment_block(la, lb + 1, qm_xyz + 3 * k, qm_xyz + 3 * kB, qm_xyz + 3 * k, shell_nprim[sA],
                         exps + shell_off[sA], ncoef + shell_off[sA], shell_nprim[sB], exps + shell_off[sB],
                         ncoef + shell_off[sB], 1.0, bp);
            moment_block(la, lb - 1, qm_xyz + 3 * k, qm_xyz + 3 * kB, qm_xyz + 3 * k, shell_nprim[sA],
                         exps + shell_off[sA], ncoef + shell_off[sA], shell_nprim[sB], exps + shell_off[sB],
                         ncoef + shell_off[sB], 0.0, bm);
            for (int i = 0; i < ncart(la); i++)
                for (int j = 0; j < ncart(lb); j++) {
                    double d = dm[(long)(aoff[sB] + j) * nao + aoff[sA] + i];
                    for (int x = 0; x < 3; x++) {
                        int up[3] = {cb[j][0], cb[j][1], cb[j][2]}, dn[3] = {cb[j][0], cb[j][1], cb[j][2]};
                        up[x]++; dn[x]--;
                        int jp = -1, jm = -1;
                        for (int t = 0; t < ncart(lb + 1); t++)
                            if (cbp[t][0] == up[0] && cbp[t][1] == up[1] && cbp[t][2] == up[2]) jp = t;
                        if (cb[j][x] > 0)
                            for (int t = 0; t < ncart(lb - 1); t++)
                                if (cbm[t][0] == dn[0] && cbm[t][1] == dn[1] && cbm[t][2] == dn[2]) jm = t;
                        double g = 0.0;
                        for (int op = 0; op < 10; op++) {
                            double dint = bp[(op * 36 + i) * 36 + jp];
                            if (jm >= 0) dint -= cb[j][x] * bm[(op * 36 + i) * 36 + jm];
                            g += W10[op] * phi[phi_stride * k + op] * dint;
                        }
                        /* dE/dB = -dm * <mu|W|dnu/dB>;  dE/dR_k = +dm * <mu|W|dnu/dB> */
                        dRqm[3 * kB + x] -= d * g;
                        dRqm[3 * k + x] += d * g;
                    }
                }
        }
    free(bp); free(bm); free(aoff);
}

/* ------------------------------------------------------------------------------------------ */
/* interaction tensors                                                                          */
/* ------------------------------------------------------------------------------------------ */

/* Taylor tensors of a radial potential f at displacement d = R_j - R_i, in the paper's
 * convention T = f, T_a = d_a f, T_ab = 1/2 d_ab f, T_abc = 1/6 d_abc f (derivatives w.r.t.
 * R_j).  With g1 = f'/r, g2 = g1'/r, g3 = g2'/r:
 *   d_a f = x_a g1;  d_ab f = delta_ab g1 + x_a x_b g2;
 *   d_abc f = (delta_ab x_c + delta_ac x_b + delta_bc x_a) g2 + x_a x_b x_c g3.
 * kind 0: f = 1/r (SI point tensors).  kind 1: f = erfc(beta r)/r, for which g1 = -f3,
 * g2 = 3 f5, g3 = -15 f7 with f1..f7 from the SI (Gaussian-screened tensors). */
void oracle_tensor(int kind, double beta, const double *d, double *T)
{
    double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2], r = sqrt(r2);
    double f, g1, g2, g3;
    if (kind == 0) {
        f = 1.0 / r;
        g1 = -f / r2;
        g2 = 3.0 * f / (r2 * r2);
        g3 = -15.0 * f / (r2 * r2 * r2);
    } else {
        double e = exp(-beta * beta * r2), sp = sqrt(OR_PI);
        double f1 = erfc(beta * r) / r;
        double f3 = (f1 + 2.0 * beta / sp * e) / r2;
        double f5 = (f3 + 4.0 / 3.0 * beta * beta * beta / sp * e) / r2;
        double f7 = (f5 + 8.0 / 15.0 * pow(beta, 5) / sp * e) / r2;
        f = f1; g1 = -f3; g2 = 3.0 * f5; g3 = -15.0 * f7;
    }
    static const int P2[6][2] = {{0, 0}, {0, 1}, {0, 2}, {1, 1}, {1, 2}, {2, 2}};
    static const int P3[10][3] = {{0, 0, 0}, {0, 0, 1}, {0, 0, 2}, {0, 1, 1}, {0, 1, 2},
                                  {0, 2, 2}, {1, 1, 1}, {1, 1, 2}, {1, 2, 2}, {2, 2, 2}};
    T[0] = f;
    for (int a = 0; a < 3; a++) T[1 + a] = d[a] * g1;
    for (int k = 0; k < 6; k++) {
        int a = P2[k][0], b = P2[k][1];
        T[4 + k] = 0.5 * ((a == b ? g1 : 0.0) + d[a] * d[b] * g2);
    }
    for (int k = 0; k < 10; k++) {
        int a = P3[k][0], b = P3[k][1], c = P3[k][2];
        double s = (a == b ? d[c] : 0.0) + (a == c ? d[b] : 0.0) + (b == c ? d[a] : 0.0);
        T[10 + k] = (s * g2 + d[a] * d[b] * d[c] * g3) / 6.0;
    }
}

/* ------------------------------------------------------------------------------------------ */
/* region I, Ewald potentials at the QM sites and at the MM sites                             */
/* ------------------------------------------------------------------------------------------ */

static void qm_centre(int natm, const double *qm_xyz, double *c)
{
    c[0] = c[1] = c[2] = 0.0;
    for (int j = 0; j < natm; j++)
        for (int x = 0; x < 3; x++) c[x] += qm_xyz[3 * j + x];
    for (int x = 0; x < 3; x++) c[x] /= natm;
}

static int in_region1(const double *c, const double *pos, double rcut)
{
    double r2 = 0.0;
    for (int x = 0; x < 3; x++) r2 += (pos[x] - c[x]) * (pos[x] - c[x]);
    return r2 < rcut * rcut;
}

/* Region I (Sec. "Error Control", sphere about the QM geometric centre): all images
 * (i, n) with |R_i + n*box - c| < rcut, in order of i then (nx, ny, nz).  Writes up to cap
 * entries (idx[k], shift[3k..3k+2] = n*box) and returns the total count. */
int oracle_region1(int natm, const double *qm_xyz, int nmm, const double *mm_xyz, const double *box,
                   double rcut, int cap, int *idx, double *shift)
{
    double c[3];
    qm_centre(natm, qm_xyz, c);
    int m[3], cnt = 0;
    for (int x = 0; x < 3; x++) m[x] = (int)ceil(rcut / box[x]) + 2;
    for (int i = 0; i < nmm; i++)
        for (int nx = -m[0]; nx <= m[0]; nx++)
            for (int ny = -m[1]; ny <= m[1]; ny++)
                for (int nz = -m[2]; nz <= m[2]; nz++) {
                    double s[3] = {nx * box[0], ny * box[1], nz * box[2]};
                    double pos[3] = {mm_xyz[3 * i] + s[0], mm_xyz[3 * i + 1] + s[1], mm_xyz[3 * i + 2] + s[2]};
                    if (in_region1(c, pos, rcut)) {
                        if (cnt < cap) {
                            idx[cnt] = i;
                            for (int x = 0; x < 3; x++) shift[3 * cnt + x] = s[x];
                        }
                        cnt++;
                    }
                }
    return cnt;
}

/* mode bits for the Ewald pieces */
#define EW_SR 1   /* psi_SR: erfc-screened real-space sum over images within the Ewald cutoff */
#define EW_LR 2   /* psi_LR: reciprocal sum over G != 0 in the cube max|n_c| <= kmax */
#define EW_BG 4   /* neutralising background -pi/(V kappa^2) on the monopole */
#define EW_R1 8   /* minus point tensors T over region I */
#define EW_HAT 16 /* minus T-hat(1/sigma) over region-II images close enough to matter */

static void ew_images(const double *box, double rc, int *m)
{
    for (int x = 0; x < 3; x++) m[x] = (int)ceil(rc / box[x]) + 1;
}

/* Generalised potential at every QM site j (Eq. 6 QM-MM terms + Eq. 10):
 *   phi_j,c = sum_i q_i [ psi_c(R_j - R_i) - sum_{L: i+L in I} T_c(R_j-R_i-L)
 *                          - sum_{L: i+L not in I} That_c(1/sigma_i; R_j-R_i-L) ]
 * for the 20 tensor components c.  Energy: E_II = sum_j sum_c W_c M_j,c phi_j,c (c < 10). */
void oracle_ewald_phi(int natm, const double *qm_xyz, int nmm, const double *mm_xyz, const double *q,
                      const double *sigma, const double *box, double rcut, double ewald_rc, double kappa,
                      const int *kmax, int mode, double *phi)
{
    double c[3], V = box[0] * box[1] * box[2];
    qm_centre(natm, qm_xyz, c);
    memset(phi, 0, sizeof(double) * natm * 20);
    int mrc[3], mr1[3];
    ew_images(box, ewald_rc, mrc);
    for (int x = 0; x < 3; x++) mr1[x] = (int)ceil(rcut / box[x]) + 2;
#pragma omp parallel for schedule(dynamic, 1)
    for (int j = 0; j < natm; j++) {
        double T[20], acc[20];
        memset(acc, 0, sizeof(acc));
        for (int i = 0; i < nmm; i++) {
            double d0[3];
            for (int x = 0; x < 3; x++) d0[x] = qm_xyz[3 * j + x] - mm_xyz[3 * i + x];
            if (mode & EW_SR) {
                for (int nx = -mrc[0]; nx <= mrc[0]; nx++)
                    for (int ny = -mrc[1]; ny <= mrc[1]; ny++)
                        for (int nz = -mrc[2]; nz <= mrc[2]; nz++) {
                            double d[3] = {d0[0] - nx * box[0], d0[1] - ny * box[1], d0[2] - nz * box[2]};
                            if (d[0] * d[0] + d[1] * d[1] + d[2] * d[2] >= ewald_rc * ewald_rc) continue;
                            oracle_tensor(1, kappa, d, T);
                            for (int k = 0; k < 20; k++) acc[k] += q[i] * T[k];
                        }
            }
            if (mode & (EW_R1 | EW_HAT)) {
                double rhat = sigma[i] > 0.0 ? 9.0 * sigma[i] : 0.0;
                for (int nx = -mr1[0]; nx <= mr1[0]; nx++)
                    for (int ny = -mr1[1]; ny <= mr1[1]; ny++)
                        for (int nz = -mr1[2]; nz <= mr1[2]; nz++) {
                            double s[3] = {nx * box[0], ny * box[1], nz * box[2]};
                            double pos[3] = {mm_xyz[3 * i] + s[0], mm_xyz[3 * i + 1] + s[1], mm_xyz[3 * i + 2] + s[2]};
                            double d[3] = {d0[0] - s[0], d0[1] - s[1], d0[2] - s[2]};
                            int inI = in_region1(c, pos, rcut);
                            if (inI && (mode & EW_R1)) {
                                oracle_tensor(0, 0.0, d, T);
                                for (int k = 0; k < 20; k++) acc[k] -= q[i] * T[k];
                            } else if (!inI && (mode & EW_HAT) && rhat > 0.0 &&
                                       d[0] * d[0] + d[1] * d[1] + d[2] * d[2] < rhat * rhat) {
                                oracle_tensor(1, 1.0 / sigma[i], d, T);
                                for (int k = 0; k < 20; k++) acc[k] -= q[i] * T[k];
                            }
                        }
            }
        }
        for (int k = 0; k < 20; k++) phi[20 * j + k] = acc[k];
    }
    if (mode & EW_BG) {
        double qt = 0.0;
        for (int i = 0; i < nmm; i++) qt += q[i];
        for (int j = 0; j < natm; j++) phi[20 * j] += -OR_PI / (V * kappa * kappa) * qt;
    }
    if (mode & EW_LR) {
        /* structure factor S(G) = sum_i q_i exp(i G.R_i), then for each QM site
         * Re/Im of exp(i G.R_j) conj(S(G)) with the derivative factors (i G)^n / n! */
        int nG = (2 * kmax[0] + 1) * (2 * kmax[1] + 1) * (2 * kmax[2] + 1);
#pragma omp parallel
        {
            double local[20 * 512];
            double *acc = natm <= 512 ? local : (double *)malloc(sizeof(double) * 20 * natm);
            memset(acc, 0, sizeof(double) * 20 * natm);
#pragma omp for schedule(dynamic, 16)
            for (int g = 0; g < nG; g++) {
                int nx = g / ((2 * kmax[1] + 1) * (2 * kmax[2] + 1)) - kmax[0];
                int ny = (g / (2 * kmax[2] + 1)) % (2 * kmax[1] + 1) - kmax[1];
                int nz = g % (2 * kmax[2] + 1) - kmax[2];
                if (nx == 0 && ny == 0 && nz == 0) continue;
                double G[3] = {2.0 * OR_PI * nx / box[0], 2.0 * OR_PI * ny / box[1], 2.0 * OR_PI * nz / box[2]};
                double G2 = G[0] * G[0] + G[1] * G[1] + G[2] * G[2];
                double gf = 4.0 * OR_PI / V * exp(-G2 / (4.0 * kappa * kappa)) / G2;
                double Sre = 0.0, Sim = 0.0;
                for (int i = 0; i < nmm; i++) {
                    double th = G[0] * mm_xyz[3 * i] + G[1] * mm_xyz[3 * i + 1] + G[2] * mm_xyz[3 * i + 2];
                    Sre += q[i] * cos(th);
                    Sim += q[i] * sin(th);
                }
                for (int j = 0; j < natm; j++) {
                    double th = G[0] * qm_xyz[3 * j] + G[1] * qm_xyz[3 * j + 1] + G[2] * qm_xyz[3 * j + 2];
                    /* exp(i th) * conj(S) */
                    double re = cos(th) * Sre + sin(th) * Sim;
                    double im = sin(th) * Sre - cos(th) * Sim;
                    double *a = acc + 20 * j;
                    a[0] += gf * re;
                    for (int x = 0; x < 3; x++) a[1 + x] += -gf * G[x] * im;
                    static const int P2[6][2] = {{0, 0}, {0, 1}, {0, 2}, {1, 1}, {1, 2}, {2, 2}};
                    static const int P3[10][3] = {{0, 0, 0}, {0, 0, 1}, {0, 0, 2}, {0, 1, 1}, {0, 1, 2},
                                                  {0, 2, 2}, {1, 1, 1}, {1, 1, 2}, {1, 2, 2}, {2, 2, 2}};
                    for (int k = 0; k < 6; k++) a[4 + k] += -0.5 * gf * G[P2[k][0]] * G[P2[k][1]] * re;
                    for (int k = 0; k < 10; k++)
                        a[10 + k] += gf / 6.0 * G[P3[k][0]] * G[P3[k][1]] * G[P3[k][2]] * im;
                }
            }
#pragma omp critical
            for (int k = 0; k < 20 * natm; k++) phi[k] += acc[k];
            if (acc != local) free(acc);
        }
    }
}

/* MM-side potential and field from the QM multipoles M[natm*10] (same pieces as above):
 *   dq[i]  += sum_j sum_c W_c M_j,c Psi_c(j,i)             (dE/dq_i)
 *   dR[i]  += - q_i sum_j sum_{c} W_c M_j,c d/dR_j Psi_c    (dE/dR_i; Psi depends on R_j - R_i)
 * where Psi is the same combination of psi, T and T-hat as in oracle_ewald_phi. */
void oracle_ewald_mm(int natm, const double *qm_xyz, const double *M, int nmm, const double *mm_xyz,
                     const double *q, const double *sigma, const double *box, double rcut, double ewald_rc,
                     double kappa, const int *kmax, int mode, const unsigned char *only, double *dq, double *dR)
{
    /* only != NULL: evaluate the MM side for the charges with only[i] != 0 (the others are left
     * untouched); a sampling convenience for large systems, same arithmetic. */
    double c[3], V = box[0] * box[1] * box[2];
    qm_centre(natm, qm_xyz, c);
    int mrc[3], mr1[3];
    ew_images(box, ewald_rc, mrc);
    for (int x = 0; x < 3; x++) mr1[x] = (int)ceil(rcut / box[x]) + 2;
    /* dE/dR_j of psi_c: d_x T_0 = T_x; d_x T_a = 2 T_ax; d_x T_ab = 3 T_abx.  Index helpers. */
    static const int I2[3][3] = {{4, 5, 6}, {5, 7, 8}, {6, 8, 9}};
    static const int I3[3][3][3] = {{{10, 11, 12}, {11, 13, 14}, {12, 14, 15}},
                                    {{11, 13, 14}, {13, 16, 17}, {14, 17, 18}},
                                    {{12, 14, 15}, {14, 17, 18}, {15, 18, 19}}};
    static const int P2[6][2] = {{0, 0}, {0, 1}, {0, 2}, {1, 1}, {1, 2}, {2, 2}};
#pragma omp parallel for schedule(dynamic, 64)
    for (int i = 0; i < nmm; i++) {
        if (only && !only[i]) continue;
        double T[20], pot = 0.0, fld[3] = {0, 0, 0};
        for (int j = 0; j < natm; j++) {
            const double *Mj = M + 10 * j;
            double d0[3];
            for (int x = 0; x < 3; x++) d0[x] = qm_xyz[3 * j + x] - mm_xyz[3 * i + x];
            for (int pass = 0; pass < 2; pass++) {
                int *mm_ = pass == 0 ? mrc : mr1;
                if (pass == 0 && !(mode & EW_SR)) continue;
                if (pass == 1 && !(mode & (EW_R1 | EW_HAT))) continue;
                for (int nx = -mm_[0]; nx <= mm_[0]; nx++)
                    for (int ny = -mm_[1]; ny <= mm_[1]; ny++)
                        for (int nz = -mm_[2]; nz <= mm_[2]; nz++) {
                            double s[3] = {nx * box[0], ny * box[1], nz * box[2]};
                            double d[3] = {d0[0] - s[0], d0[1] - s[1], d0[2] - s[2]};
                            double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2], sgn;
                            if (pass == 0) {
                                if (r2 >= ewald_rc * ewald_rc) continue;
                                oracle_tensor(1, kappa, d, T);
                                sgn = 1.0;
                            } else {
                                double pos[3] = {mm_xyz[3 * i] + s[0], mm_xyz[3 * i + 1] + s[1], mm_xyz[3 * i + 2] + s[2]};
                                int inI = in_region1(c, pos, rcut);
                                double rhat = sigma[i] > 0.0 ? 9.0 * sigma[i] : 0.0;
                                if (inI && (mode & EW_R1)) oracle_tensor(0, 0.0, d, T);
                                else if (!inI && (mode & EW_HAT) && rhat > 0.0 && r2 < rhat * rhat)
                                    oracle_tensor(1, 1.0 / sigma[i], d, T);
                                else continue;
                                sgn = -1.0;
                            }
                            for (int k = 0; k < 10; k++) pot += sgn * W10[k] * Mj[k] * T[k];
                            for (int x = 0; x < 3; x++) {
                                double g = Mj[0] * T[1 + x];
                                for (int a = 0; a < 3; a++) g += 2.0 * Mj[1 + a] * T[I2[a][x]];
                                for (int k = 0; k < 6; k++)
                                    g += 3.0 * W10[4 + k] * Mj[4 + k] * T[I3[P2[k][0]][P2[k][1]][x]];
                                fld[x] += sgn * g; /* d/dR_j */
                            }
                        }
            }
        }
        dq[i] += pot;
        for (int x = 0; x < 3; x++) dR[3 * i + x] += -q[i] * fld[x];
    }
    if (mode & EW_BG) {
        double Qt = 0.0;
        for (int j = 0; j < natm; j++) Qt += M[10 * j];
        for (int i = 0; i < nmm; i++)
            if (!only || only[i]) dq[i] += -OR_PI / (V * kappa * kappa) * Qt;
    }
    if (mode & EW_LR) {
        /* A(G) = sum_j exp(i G.R_j) (Q_j + i G.mu_j - 1/2 G.theta_j.G);
         * dq_i += (4 pi/V) sum_G g(G) Re[A(G) exp(-i G.R_i)],  dR_i += q_i (4 pi/V) sum_G g Re[A (-iG) exp(-iG.R_i)] */
        int nG = (2 * kmax[0] + 1) * (2 * kmax[1] + 1) * (2 * kmax[2] + 1);
        double *Are = (double *)malloc(sizeof(double) * nG), *Aim = (double *)malloc(sizeof(double) * nG);
        double *Gv = (double *)malloc(sizeof(double) * nG * 4);
        for (int g = 0; g < nG; g++) {
            int nx = g / ((2 * kmax[1] + 1) * (2 * kmax[2] + 1)) - kmax[0];
            int ny = (g / (2 * kmax[2] + 1)) % (2 * kmax[1] + 1) - kmax[1];
            int nz = g % (2 * kmax[2] + 1) - kmax[2];
            double G[3] = {2.0 * OR_PI * nx / box[0], 2.0 * OR_PI * ny / box[1], 2.0 * OR_PI * nz / box[2]};
            double G2 = G[0] * G[0] + G[1] * G[1] + G[2] * G[2];
            Gv[4 * g] = G[0]; Gv[4 * g + 1] = G[1]; Gv[4 * g + 2] = G[2];
            Gv[4 * g + 3] = (G2 == 0.0) ? 0.0 : 4.0 * OR_PI / V * exp(-G2 / (4.0 * kappa * kappa)) / G2;
            double re = 0.0, im = 0.0;
            for (int j = 0; j < natm; j++) {
                const double *Mj = M + 10 * j;
                double th = G[0] * qm_xyz[3 * j] + G[1] * qm_xyz[3 * j + 1] + G[2] * qm_xyz[3 * j + 2];
                double mr = Mj[0], mi = G[0] * Mj[1] + G[1] * Mj[2] + G[2] * Mj[3];
                for (int k = 0; k < 6; k++) mr -= 0.5 * W10[4 + k] * Mj[4 + k] * G[P2[k][0]] * G[P2[k][1]];
                re += cos(th) * mr - sin(th) * mi;
                im += sin(th) * mr + cos(th) * mi;
            }
            Are[g] = re; Aim[g] = im;
        }
#pragma omp parallel for schedule(dynamic, 64)
        for (int i = 0; i < nmm; i++) {
            if (only && !only[i]) continue;
            double pot = 0.0, fr[3] = {0, 0, 0};
            for (int g = 0; g < nG; g++) {
                if (Gv[4 * g + 3] == 0.0) continue;
                double th = Gv[4 * g] * mm_xyz[3 * i] + Gv[4 * g + 1] * mm_xyz[3 * i + 1] + Gv[4 * g + 2] * mm_xyz[3 * i + 2];
                /* A * exp(-i th) */
                double re = Are[g] * cos(th) + Aim[g] * sin(th);
                double im = Aim[g] * cos(th) - Are[g] * sin(th);
                pot += Gv[4 * g + 3] * re;
                /* Re[(-i G_x)(re + i im)] = G_x im */
                for (int x = 0; x < 3; x++) fr[x] += Gv[4 * g + 3] * Gv[4 * g + x] * im;
            }
            dq[i] += pot;
            for (int x = 0; x < 3; x++) dR[3 * i + x] += q[i] * fr[x];
        }
        free(Are); free(Aim); free(Gv);
    }
}

/* Tensor part of dE/dR_QM: dE/dR_j,x = sum_c W_c M_j,c d_x phi_j,c with d_x phi_0 = phi_x,
 * d_x phi_a = 2 phi_ax, d_x phi_ab = 3 phi_abx (phi from oracle_ewald_phi).  Accumulates. */
/* QM-QM periodic-image multipole energy (Eq. 5 and its Ewald form in Eq. 6, readings in the test
 * file): with the image tensor P_ji = sum_{L != 0} T(R_j - R_i + L), evaluated as the Ewald sum
 * (erfc real space over images within ewald_rc, reciprocal sum over the kmax cube, self terms
 * -2 kappa/sqrt(pi) and +(2/3) kappa^3/sqrt(pi) delta_ab for i = j) minus the L = 0 point tensor
 * for i != j, and the pair energy
 *   e(j,i) = Q_j Q_i P + 2 mu_j.Q_i P_a + 2 theta_j:Q_i P_ab - 2 mu_j mu_i : P_ab,
 * E = 1/2 sum_{j,i} e(j,i) - pi/(2 V kappa^2) (sum_j Q_j)^2.  Outputs: E[0]; u[natm*10], the
 * derivative of E with respect to each stored multipole component divided by its weight W10 (the
 * potential that plays the role of phi for the Fock and Pulay terms); grad[natm*3], dE/dR at fixed
 * multipoles.  M[natm*10] in the stored order (Q, mu xyz, theta xx xy xz yy yz zz). */
void oracle_qmqm(int natm, const double *qm_xyz, const double *M, const double *box, double ewald_rc, double kappa,
                 const int *kmax, double *E, double *u, double *grad)
{
    const double V = box[0] * box[1] * box[2], sp = sqrt(OR_PI);
    static const int P2[6][2] = {{0, 0}, {0, 1}, {0, 2}, {1, 1}, {1, 2}, {2, 2}};
    int mrc[3];
    ew_images(box, ewald_rc, mrc);
    double etot = 0.0, qsum = 0.0;
    memset(u, 0, sizeof(double) * natm * 10);
    memset(grad, 0, sizeof(double) * natm * 3);
    for (int j = 0; j < natm; j++) qsum += M[10 * j];
    for (int j = 0; j < natm; j++)
        for (int i = 0; i < natm; i++) {
            double P[20], T[20];
            memset(P, 0, sizeof(P));
            double d0[3];
            for (int x = 0; x < 3; x++) d0[x] = qm_xyz[3 * j + x] - qm_xyz[3 * i + x];
            /* real space: erfc-screened tensors over images within the Ewald cutoff */
            for (int nx = -mrc[0]; nx <= mrc[0]; nx++)
                for (int ny = -mrc[1]; ny <= mrc[1]; ny++)
                    for (int nz = -mrc[2]; nz <= mrc[2]; nz++) {
                        if (i == j && nx == 0 && ny == 0 && nz == 0) continue;
                        double d[3] = {d0[0] - nx * box[0], d0[1] - ny * box[1], d0[2] - nz * box[2]};
                        if (d[0] * d[0] + d[1] * d[1] + d[2] * d[2] >= ewald_rc * ewald_rc) continue;
                        oracle_tensor(1, kappa, d, T);
                        for (int k = 0; k < 20; k++) P[k] += T[k];
                    }
            /* reciprocal space: T = f, f_a, 1/2 f_ab, 1/6 f_abc of (4 pi / V) sum g(G) cos(G.d) */
            for (int nx = -kmax[0]; nx <= kmax[0]; nx++)
                for (int ny = -kmax[1]; ny <= kmax[1]; ny++)
                    for (int nz = -kmax[2]; nz <= kmax[2]; nz++) {
                        if (nx == 0 && ny == 0 && nz == 0) continue;
                        double G[3] = {2.0 * OR_PI * nx / box[0], 2.0 * OR_PI * ny / box[1], 2.0 * OR_PI * nz / box[2]};
                        double G2 = G[0] * G[0] + G[1] * G[1] + G[2] * G[2];
                        double g = 4.0 * OR_PI / V * exp(-G2 / (4.0 * kappa * kappa)) / G2;
                        double ph = G[0] * d0[0] + G[1] * d0[1] + G[2] * d0[2], cs = cos(ph), sn = sin(ph);
                        P[0] += g * cs;
                        for (int a = 0; a < 3; a++) P[1 + a] -= g * G[a] * sn;
                        for (int k = 0; k < 6; k++) P[4 + k] -= 0.5 * g * G[P2[k][0]] * G[P2[k][1]] * cs;
                        static const int P3[10][3] = {{0, 0, 0}, {0, 0, 1}, {0, 0, 2}, {0, 1, 1}, {0, 1, 2},
                                                      {0, 2, 2}, {1, 1, 1}, {1, 1, 2}, {1, 2, 2}, {2, 2, 2}};
                        for (int k = 0; k < 10; k++)
                            P[10 + k] += g * G[P3[k][0]] * G[P3[k][1]] * G[P3[k][2]] * sn / 6.0;
                    }
            if (i == j) {
                /* self terms: Taylor coefficients of -erf(kappa r)/r at r = 0 */
                P[0] += -2.0 * kappa / sp;
                P[4] += 2.0 / 3.0 * kappa * kappa * kappa / sp;
                P[7] += 2.0 / 3.0 * kappa * kappa * kappa / sp;
                P[9] += 2.0 / 3.0 * kappa * kappa * kappa / sp;
            } else {
                /* the reference-cell pair is the QM calculation's: remove its point interaction */
                oracle_tensor(0, 0.0, d0, T);
                for (int k = 0; k < 20; k++) P[k] -= T[k];
            }
            /* full symmetric 3x3 views of P_ab and theta, 3x3x3 of P_abc */
            double Pab[3][3], thj[3][3], Pabc[3][3][3];
            for (int k = 0; k < 6; k++) {
                int a = P2[k][0], b = P2[k][1];
                Pab[a][b] = Pab[b][a] = P[4 + k];
                thj[a][b] = thj[b][a] = M[10 * j + 4 + k];
            }
            {
                static const int P3[10][3] = {{0, 0, 0}, {0, 0, 1}, {0, 0, 2}, {0, 1, 1}, {0, 1, 2},
                                              {0, 2, 2}, {1, 1, 1}, {1, 1, 2}, {1, 2, 2}, {2, 2, 2}};
                for (int k = 0; k < 10; k++) {
                    int a = P3[k][0], b = P3[k][1], c = P3[k][2];
                    Pabc[a][b][c] = Pabc[a][c][b] = Pabc[b][a][c] = Pabc[b][c][a] = Pabc[c][a][b] = Pabc[c][b][a] = P[10 + k];
                }
            }
            const double Qj = M[10 * j], Qi = M[10 * i];
            const double *mj = M + 10 * j + 1, *mi = M + 10 * i + 1;
            double e = Qj * Qi * P[0];
            for (int a = 0; a < 3; a++) e += 2.0 * mj[a] * Qi * P[1 + a];
            for (int a = 0; a < 3; a++)
                for (int b = 0; b < 3; b++) e += 2.0 * thj[a][b] * Qi * Pab[a][b] - 2.0 * mj[a] * mi[b] * Pab[a][b];
            etot += 0.5 * e;
            /* conjugate potentials: 1/2 de/dM_j (first slot) and 1/2 de/dM_i (second slot) */
            u[10 * j] += 0.5 * Qi * P[0];
            for (int a = 0; a < 3; a++) {
                double t = 2.0 * Qi * P[1 + a];
                for (int b = 0; b < 3; b++) t -= 2.0 * mi[b] * Pab[a][b];
                u[10 * j + 1 + a] += 0.5 * t;
            }
            for (int k = 0; k < 6; k++) u[10 * j + 4 + k] += 0.5 * 2.0 * Qi * P[4 + k];
            {
                double t = Qj * P[0];
                for (int a = 0; a < 3; a++) t += 2.0 * mj[a] * P[1 + a];
                for (int a = 0; a < 3; a++)
                    for (int b = 0; b < 3; b++) t += 2.0 * thj[a][b] * Pab[a][b];
                u[10 * i] += 0.5 * t;
                for (int b = 0; b < 3; b++) {
                    double s2 = 0.0;
                    for (int a = 0; a < 3; a++) s2 -= 2.0 * mj[a] * Pab[a][b];
                    u[10 * i + 1 + b] += 0.5 * s2;
                }
            }
            /* gradient at fixed multipoles: d/dd of e, d = R_j - R_i (i = j terms do not move) */
            if (i != j)
                for (int c = 0; c < 3; c++) {
                    double g = Qj * Qi * P[1 + c];
                    for (int a = 0; a < 3; a++) g += 2.0 * mj[a] * Qi * 2.0 * Pab[a][c];
                    for (int a = 0; a < 3; a++)
                        for (int b = 0; b < 3; b++)
                            g += 2.0 * thj[a][b] * Qi * 3.0 * Pabc[a][b][c] - 2.0 * mj[a] * mi[b] * 3.0 * Pabc[a][b][c];
                    grad[3 * j + c] += 0.5 * g;
                    grad[3 * i + c] -= 0.5 * g;
                }
        }
    /* neutralising background for a charged QM cell */
    etot += -OR_PI / (2.0 * V * kappa * kappa) * qsum * qsum;
    for (int j = 0; j < natm; j++) u[10 * j] += -OR_PI / (V * kappa * kappa) * qsum;
    E[0] = etot;
}

void oracle_tensor_grad_qm(int natm, const double *M, const double *phi, double *dRqm)
{
    static const int I2[3][3] = {{4, 5, 6}, {5, 7, 8}, {6, 8, 9}};
    static const int I3[3][3][3] = {{{10, 11, 12}, {11, 13, 14}, {12, 14, 15}},
                                    {{11, 13, 14}, {13, 16, 17}, {14, 17, 18}},
                                    {{12, 14, 15}, {14, 17, 18}, {15, 18, 19}}};
    static const int P2[6][2] = {{0, 0}, {0, 1}, {0, 2}, {1, 1}, {1, 2}, {2, 2}};
    for (int j = 0; j < natm; j++) {
        const double *Mj = M + 10 * j, *p = phi + 20 * j;
        for (int x = 0; x < 3; x++) {
            double g = Mj[0] * p[1 + x];
            for (int a = 0; a < 3; a++) g += 2.0 * Mj[1 + a] * p[I2[a][x]];
            for (int k = 0; k < 6; k++) g += 3.0 * W10[4 + k] * Mj[4 + k] * p[I3[P2[k][0]][P2[k][1]][x]];
            dRqm[3 * j + x] += g;
        }
    }
}
