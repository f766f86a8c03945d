// moments.cu -- overlap-type moment integrals about the atom centres and what is built from
// them: Mulliken charge/dipole/quadrupole (SI, "Multipolar Ewald"), the region-II Fock term of
// Eqs. 11-14 and the multipole Pulay gradient of Eq. 15.
//
// Multipoles and the Fock term: one lane per primitive pair.  With the Pulay gradient: two kernels
// per angular class, one thread per (primitive pair, Cartesian component of shell A) for everything
// about centre A and one per (primitive pair, component of shell B) for centre B, so each thread
// keeps one row (column) of the 1-D moment tables in registers with static indexing.
// In one direction the moment about a centre K is
//   <i| (x-K)^e |j> = sum_t E^{ij}_t M^e_t,  M^0 = (1), M^1 = (X_PK, 1),
//   M^2 = (X_PK^2 + 1/(2p), 2 X_PK, 2)   (times sqrt(pi/p), folded into the prefactor).
// With the local potential polynomial W_k(r) = sum_c w_c v_k,c O_c(r - R_k) of atom k
// (w = 1, or 2 for the off-diagonal theta components), the multipole energy is
// E_II = sum_k Z_k v_k,0 - sum_{mu in k, nu} gamma_{nu mu} <mu|W_k|nu>, hence
//   F_{mu nu} = -1/2 (<mu|W_{k(mu)}|nu> + <mu|W_{k(nu)}|nu>),
// and moving the centre B of nu by d changes <mu|W_k|nu> by <mu|W_k|d nu/dB> with
// d g_b/dB_x = 2b g_{b+1x} - b_x g_{b-1x}; moving atom k (mu and the operator) gives minus that.
#include "pp_tile.cuh"

namespace qmmm {

__constant__ int c_opx[10] = {0, 1, 0, 0, 2, 1, 1, 0, 0, 0};
__constant__ int c_opy[10] = {0, 0, 1, 0, 0, 1, 0, 2, 1, 0};
__constant__ int c_opz[10] = {0, 0, 0, 1, 0, 0, 1, 0, 1, 2};
__constant__ double c_w10[10] = {1, 1, 1, 1, 1, 2, 2, 1, 2, 1};

// One thread per primitive pair with the full 1-D moment tables (multipoles and the Fock term:
// the tables are small there, and one Hermite setup per pair serves all components).
template <int LA, int LB>
__global__ void __launch_bounds__(128)
k_moments(BasisDev bd, int pp_begin, int pp_end, const double *__restrict__ dm, const double *__restrict__ phi,
          double *__restrict__ mult, double *__restrict__ F, double *__restrict__ gqm, int mode)
{
    constexpr int L = LA + LB, NA = ncart(LA), NB = ncart(LB);
    constexpr int I = LA + 1, J = LB + 1;
    const int lane = threadIdx.x & 31;
    const int i = pp_begin + (blockIdx.x * blockDim.x + threadIdx.x);
    if (pp_begin + (int)((blockIdx.x * blockDim.x + (threadIdx.x & ~31))) >= pp_end) return;  // whole warp out
    const PPLane pl = load_pp(bd, i, pp_end);
    const bool mirror = pl.sp.shA != pl.sp.shB;
    const bool pulay = (mode & MOM_PULAY) && pl.atomA != pl.atomB;

    // 1-D moment tables about centre A (atom of shell A) and centre B, per direction
    double SA[3][I + 1][J + 1][3], SB[3][I + 1][J + 1][3];
    {
        double E[I + 1][J + 1][I + J + 1];
        const double h = 0.5 * pl.ip;
#pragma unroll 1
        for (int d = 0; d < 3; ++d) {
            hermite_E<I, J, double>(E, pl.P[d] - pl.A[d], pl.P[d] - pl.B[d], h);
            const double XA = pl.P[d] - pl.A[d], XB = pl.P[d] - pl.B[d];
#pragma unroll
            for (int a = 0; a <= I; ++a)
#pragma unroll
                for (int b = 0; b <= J; ++b) {
                    const double e0 = E[a][b][0], e1 = (a + b >= 1) ? E[a][b][1] : 0.0,
                                 e2 = (a + b >= 2) ? E[a][b][2] : 0.0;
                    SA[d][a][b][0] = e0;
                    SA[d][a][b][1] = XA * e0 + e1;
                    SA[d][a][b][2] = (XA * XA + h) * e0 + 2.0 * XA * e1 + 2.0 * e2;
                    SB[d][a][b][0] = e0;
                    SB[d][a][b][1] = XB * e0 + e1;
                    SB[d][a][b][2] = (XB * XB + h) * e0 + 2.0 * XB * e1 + 2.0 * e2;
                }
        }
    }
    const double spp = PI * pl.ip;
    const double coef = pl.active ? pl.cab * spp * sqrt(spp) : 0.0;
    double wA[10], wB[10];
#pragma unroll
    for (int k = 0; k < 10; ++k) {
        wA[k] = c_w10[k] * phi[20 * pl.atomA + k];
        wB[k] = c_w10[k] * phi[20 * pl.atomB + k];
    }

    bool take[5], head;
    seg_setup(pl.active ? pl.s : -1 - lane, lane, take, head);

    double mA[10], mB[10], g[3] = {0.0, 0.0, 0.0};
#pragma unroll
    for (int k = 0; k < 10; ++k) mA[k] = mB[k] = 0.0;

#pragma unroll 1
    for (int ia = 0; ia < NA; ++ia) {
#pragma unroll 1
        for (int ib = 0; ib < NB; ++ib) {
            const int ax = cart_lx(LA, ia), ay = cart_ly(LA, ia), az = cart_lz(LA, ia);
            const int bx = cart_lx(LB, ib), by = cart_ly(LB, ib), bz = cart_lz(LB, ib);
            const size_t r = pl.sp.aoA + ia, c = pl.sp.aoB + ib;
            double g_ba = 0.0, g_ab = 0.0;
            if (pl.active && (mode & (MOM_MULT | MOM_PULAY))) {
                g_ba = dm[c * bd.nao + r];
                g_ab = dm[r * bd.nao + c];
            }
            double fA = 0.0, fB = 0.0;
#pragma unroll
            for (int op = 0; op < 10; ++op) {
                const int ox = c_opx[op], oy = c_opy[op], oz = c_opz[op];
                const double sa = SA[0][ax][bx][ox] * SA[1][ay][by][oy] * SA[2][az][bz][oz];
                const double sb = SB[0][ax][bx][ox] * SB[1][ay][by][oy] * SB[2][az][bz][oz];
                mA[op] -= g_ba * sa;
                mB[op] -= g_ab * sb;
                fA += wA[op] * sa;
                fB += wB[op] * sb;
                if (pulay) {
                    // G1: d/dB of <a|W_A|b>;  G2: d/dA of <a|W_B|b>
                    const double dBx = 2.0 * pl.b * SA[0][ax][bx + 1][ox] - (bx > 0 ? bx * SA[0][ax][bx - 1][ox] : 0.0);
                    const double dBy = 2.0 * pl.b * SA[1][ay][by + 1][oy] - (by > 0 ? by * SA[1][ay][by - 1][oy] : 0.0);
                    const double dBz = 2.0 * pl.b * SA[2][az][bz + 1][oz] - (bz > 0 ? bz * SA[2][az][bz - 1][oz] : 0.0);
                    const double dAx = 2.0 * pl.a * SB[0][ax + 1][bx][ox] - (ax > 0 ? ax * SB[0][ax - 1][bx][ox] : 0.0);
                    const double dAy = 2.0 * pl.a * SB[1][ay + 1][by][oy] - (ay > 0 ? ay * SB[1][ay - 1][by][oy] : 0.0);
                    const double dAz = 2.0 * pl.a * SB[2][az + 1][bz][oz] - (az > 0 ? az * SB[2][az - 1][bz][oz] : 0.0);
                    const double ga = g_ba * wA[op], gb = g_ab * wB[op];
                    const double sAy = SA[1][ay][by][oy], sAz = SA[2][az][bz][oz], sAx = SA[0][ax][bx][ox];
                    const double sBy = SB[1][ay][by][oy], sBz = SB[2][az][bz][oz], sBx = SB[0][ax][bx][ox];
                    g[0] += ga * dBx * sAy * sAz - gb * dAx * sBy * sBz;
                    g[1] += ga * sAx * dBy * sAz - gb * sBx * dAy * sBz;
                    g[2] += ga * sAx * sAy * dBz - gb * sBx * sBy * dAz;
                }
            }
            if (mode & MOM_FOCK) {
                const double f = seg_reduce(-0.5 * coef * (fA + fB), take);
                if (head && pl.active) {
                    atomicAdd(F + r * bd.nao + c, f);
                    if (mirror) atomicAdd(F + c * bd.nao + r, f);
                }
            }
        }
    }
    if (mode & MOM_MULT) {
#pragma unroll
        for (int k = 0; k < 10; ++k) {
            const double va = seg_reduce(coef * mA[k], take);
            const double vb = seg_reduce(mirror ? coef * mB[k] : 0.0, take);
            if (head && pl.active) {
                atomicAdd(mult + 10 * pl.atomA + k, va);
                if (mirror) atomicAdd(mult + 10 * pl.atomB + k, vb);
            }
        }
    }
    if (mode & MOM_PULAY) {
#pragma unroll
        for (int x = 0; x < 3; ++x) {
            const double v = seg_reduce(pulay ? coef * g[x] : 0.0, take);
            if (head && pl.active && pl.atomA != pl.atomB) {
                atomicAdd(gqm + 3 * pl.atomA + x, v);
                atomicAdd(gqm + 3 * pl.atomB + x, -v);
            }
        }
    }
}

// Operator O_c = (x-K)^ox (y-K)^oy (z-K)^oz of the ten multipole components c (charge, dipole,
// quadrupole in the order 1, x, y, z, xx, xy, xz, yy, yz, zz); weight 2 for the off-diagonal
// quadrupole components.  constexpr, so that unrolled loops index the moment tables statically.
__host__ __device__ constexpr int op_x(int c) { return c == 1 ? 1 : c == 4 ? 2 : (c == 5 || c == 6) ? 1 : 0; }
__host__ __device__ constexpr int op_y(int c) { return c == 2 ? 1 : c == 7 ? 2 : (c == 5 || c == 8) ? 1 : 0; }
__host__ __device__ constexpr int op_z(int c) { return c == 3 ? 1 : c == 9 ? 2 : (c == 6 || c == 8) ? 1 : 0; }
__host__ __device__ constexpr double op_w(int c) { return (c == 5 || c == 6 || c == 8) ? 2.0 : 1.0; }

// The 1-D moments of orders 0..2 about centre K from one Hermite row: (e0, X e0 + e1,
// (X^2 + h) e0 + 2 X e1 + 2 e2), X = P - K, h = 1/(2p).
__device__ __forceinline__ void moments3(double e0, double e1, double e2, double X, double h, double (&m)[3])
{
    m[0] = e0;
    m[1] = X * e0 + e1;
    m[2] = (X * X + h) * e0 + 2.0 * X * e1 + 2.0 * e2;
}

// E^{r,k}_t, t = 0..2, for one fixed index r of the first kind (runtime, 0..NR) and every k = 0..NK
// of the second: the recursion runs first in the fixed direction up to r (a short vector, the
// entry r selected by predicate, so all indexing stays static), then along k.  X1, X2: the
// displacements P - (centre of the first / second kind); h = 1/(2p).
template <int NR, int NK>
__device__ __forceinline__ void hermite_line(double X1, double X2, double h, int r, double (&out)[NK + 1][3])
{
    constexpr int T = NR + NK + 1;  // largest t reached
    double v[T + 1], sel[T + 1];
#pragma unroll
    for (int t = 0; t <= T; ++t) v[t] = sel[t] = 0.0;
    v[0] = 1.0;
#pragma unroll
    for (int a = 0; a <= NR; ++a) {
        if (a == r)
#pragma unroll
            for (int t = 0; t <= T; ++t) sel[t] = v[t];
        if (a < NR) {
            double w[T + 1];
#pragma unroll
            for (int t = 0; t <= T; ++t)
                w[t] = (t > 0 ? h * v[t - 1] : 0.0) + X1 * v[t] + (t < T ? (t + 1) * v[t + 1] : 0.0);
#pragma unroll
            for (int t = 0; t <= T; ++t) v[t] = w[t];
        }
    }
#pragma unroll
    for (int k = 0; k <= NK; ++k) {
        out[k][0] = sel[0];
        out[k][1] = sel[1];
        out[k][2] = T >= 2 ? sel[T >= 2 ? 2 : 0] : 0.0;
        if (k < NK) {
            double w[T + 1];
#pragma unroll
            for (int t = 0; t <= T; ++t)
                w[t] = (t > 0 ? h * sel[t - 1] : 0.0) + X2 * sel[t] + (t < T ? (t + 1) * sel[t + 1] : 0.0);
#pragma unroll
            for (int t = 0; t <= T; ++t) sel[t] = w[t];
        }
    }
}

// A side: one thread per (primitive pair, Cartesian component ia of shell A): the moments about
// A (multipoles of atom A, the Fock term with W_A, and the Pulay term d/dB <a|W_A|b>).  grid
// (ceil(n/128), NA); the lanes of a warp share ia, so primitive pairs of one shell pair are
// contiguous lanes and reduce before their atomics.
template <int LA, int LB>
__global__ void __launch_bounds__(128) k_mom_a(BasisDev bd, int pp_begin, int pp_end, const double *__restrict__ dm,
                                               const double *__restrict__ phi, double *__restrict__ mult,
                                               double *__restrict__ F, double *__restrict__ gqm, int mode)
{
    constexpr int NB = ncart(LB);
    const int lane = threadIdx.x & 31, ia = blockIdx.y;
    const int i = pp_begin + (blockIdx.x * blockDim.x + threadIdx.x);
    if (pp_begin + (int)((blockIdx.x * blockDim.x + (threadIdx.x & ~31))) >= pp_end) return;  // whole warp out
    const PPLane pl = load_pp(bd, i, pp_end);
    const bool mirror = pl.sp.shA != pl.sp.shB;
    const bool pulay = (mode & MOM_PULAY) && pl.atomA != pl.atomB;
    int a3[3];
    {
        // the Cartesian exponents of component ia
        int k = 0;
        a3[0] = a3[1] = a3[2] = 0;
#pragma unroll
        for (int x = LA; x >= 0; --x)
#pragma unroll
            for (int y = LA - x; y >= 0; --y) {
                if (k == ia) {
                    a3[0] = x;
                    a3[1] = y;
                    a3[2] = LA - x - y;
                }
                ++k;
            }
    }
    // SA[d][b][o]: moments about A of order o for the row a = a3[d], b <= LB + 1
    double SA[3][LB + 2][3];
    const double h = 0.5 * pl.ip;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        double e[LB + 2][3];
        hermite_line<LA, LB + 1>(pl.P[d] - pl.A[d], pl.P[d] - pl.B[d], h, a3[d], e);
#pragma unroll
        for (int b = 0; b <= LB + 1; ++b) moments3(e[b][0], e[b][1], e[b][2], pl.P[d] - pl.A[d], h, SA[d][b]);
    }
    const double spp = PI * pl.ip;
    const double coef = pl.active ? pl.cab * spp * sqrt(spp) : 0.0;
    double wA[10];
#pragma unroll
    for (int c = 0; c < 10; ++c) wA[c] = op_w(c) * phi[20 * pl.atomA + c];
    bool take[5], head;
    seg_setup(pl.active ? pl.s : -1 - lane, lane, take, head);
    double mA[10], g[3] = {0.0, 0.0, 0.0};
#pragma unroll
    for (int c = 0; c < 10; ++c) mA[c] = 0.0;
    const size_t r = pl.sp.aoA + ia;
#pragma unroll
    for (int ib = 0; ib < NB; ++ib) {
        const int bx = cart_lx(LB, ib), by = cart_ly(LB, ib), bz = cart_lz(LB, ib);
        const size_t c = pl.sp.aoB + ib;
        const double g_ba = (pl.active && (mode & (MOM_MULT | MOM_PULAY))) ? dm[c * bd.nao + r] : 0.0;
        double fA = 0.0;
#pragma unroll
        for (int op = 0; op < 10; ++op) {
            const int ox = op_x(op), oy = op_y(op), oz = op_z(op);
            const double sx = SA[0][bx][ox], sy = SA[1][by][oy], sz = SA[2][bz][oz];
            const double sa = sx * sy * sz;
            mA[op] -= g_ba * sa;
            fA += wA[op] * sa;
            if (pulay) {
                // d/dB of <a|W_A|b>: d g_b/dB_x = 2b g_{b+1x} - b_x g_{b-1x}
                const double dBx = 2.0 * pl.b * SA[0][bx + 1][ox] - (bx > 0 ? bx * SA[0][bx > 0 ? bx - 1 : 0][ox] : 0.0);
                const double dBy = 2.0 * pl.b * SA[1][by + 1][oy] - (by > 0 ? by * SA[1][by > 0 ? by - 1 : 0][oy] : 0.0);
                const double dBz = 2.0 * pl.b * SA[2][bz + 1][oz] - (bz > 0 ? bz * SA[2][bz > 0 ? bz - 1 : 0][oz] : 0.0);
                const double ga = g_ba * wA[op];
                g[0] += ga * dBx * sy * sz;
                g[1] += ga * sx * dBy * sz;
                g[2] += ga * sx * sy * dBz;
            }
        }
        if (mode & MOM_FOCK) {
            const double f = seg_reduce(-0.5 * coef * fA, take);
            if (head && pl.active) {
                atomicAdd(F + r * bd.nao + c, f);
                if (mirror) atomicAdd(F + c * bd.nao + r, f);
            }
        }
    }
    if (mode & MOM_MULT) {
#pragma unroll
        for (int k = 0; k < 10; ++k) {
            const double va = seg_reduce(coef * mA[k], take);
            if (head && pl.active) atomicAdd(mult + 10 * pl.atomA + k, va);
        }
    }
    if (mode & MOM_PULAY) {
#pragma unroll
        for (int x = 0; x < 3; ++x) {
            const double v = seg_reduce(pulay ? coef * g[x] : 0.0, take);
            if (head && pl.active && pl.atomA != pl.atomB) {
                atomicAdd(gqm + 3 * pl.atomA + x, v);
                atomicAdd(gqm + 3 * pl.atomB + x, -v);
            }
        }
    }
}

// B side: one thread per (primitive pair, Cartesian component ib of shell B): the moments about
// B (multipoles of atom B for off-diagonal shell pairs, the Fock term with W_B, and the Pulay
// term d/dA <a|W_B|b>).  grid (ceil(n/128), NB).
template <int LA, int LB>
__global__ void __launch_bounds__(128) k_mom_b(BasisDev bd, int pp_begin, int pp_end, const double *__restrict__ dm,
                                               const double *__restrict__ phi, double *__restrict__ mult,
                                               double *__restrict__ F, double *__restrict__ gqm, int mode)
{
    constexpr int NA = ncart(LA);
    const int lane = threadIdx.x & 31, ib = blockIdx.y;
    const int i = pp_begin + (blockIdx.x * blockDim.x + threadIdx.x);
    if (pp_begin + (int)((blockIdx.x * blockDim.x + (threadIdx.x & ~31))) >= pp_end) return;  // whole warp out
    const PPLane pl = load_pp(bd, i, pp_end);
    const bool mirror = pl.sp.shA != pl.sp.shB;
    const bool pulay = (mode & MOM_PULAY) && pl.atomA != pl.atomB;
    int b3[3];
    {
        int k = 0;
        b3[0] = b3[1] = b3[2] = 0;
#pragma unroll
        for (int x = LB; x >= 0; --x)
#pragma unroll
            for (int y = LB - x; y >= 0; --y) {
                if (k == ib) {
                    b3[0] = x;
                    b3[1] = y;
                    b3[2] = LB - x - y;
                }
                ++k;
            }
    }
    // SB[d][a][o]: moments about B of order o for the column b = b3[d], a <= LA + 1
    double SB[3][LA + 2][3];
    const double h = 0.5 * pl.ip;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        double e[LA + 2][3];
        hermite_line<LB, LA + 1>(pl.P[d] - pl.B[d], pl.P[d] - pl.A[d], h, b3[d], e);
#pragma unroll
        for (int a = 0; a <= LA + 1; ++a) moments3(e[a][0], e[a][1], e[a][2], pl.P[d] - pl.B[d], h, SB[d][a]);
    }
    const double spp = PI * pl.ip;
    const double coef = pl.active ? pl.cab * spp * sqrt(spp) : 0.0;
    double wB[10];
#pragma unroll
    for (int c = 0; c < 10; ++c) wB[c] = op_w(c) * phi[20 * pl.atomB + c];
    bool take[5], head;
    seg_setup(pl.active ? pl.s : -1 - lane, lane, take, head);
    double mB[10], g[3] = {0.0, 0.0, 0.0};
#pragma unroll
    for (int c = 0; c < 10; ++c) mB[c] = 0.0;
    const size_t c = pl.sp.aoB + ib;
#pragma unroll
    for (int ia = 0; ia < NA; ++ia) {
        const int ax = cart_lx(LA, ia), ay = cart_ly(LA, ia), az = cart_lz(LA, ia);
        const size_t r = pl.sp.aoA + ia;
        const double g_ab = (pl.active && (mode & (MOM_MULT | MOM_PULAY))) ? dm[r * bd.nao + c] : 0.0;
        double fB = 0.0;
#pragma unroll
        for (int op = 0; op < 10; ++op) {
            const int ox = op_x(op), oy = op_y(op), oz = op_z(op);
            const double sx = SB[0][ax][ox], sy = SB[1][ay][oy], sz = SB[2][az][oz];
            const double sb = sx * sy * sz;
            mB[op] -= g_ab * sb;
            fB += wB[op] * sb;
            if (pulay) {
                // d/dA of <a|W_B|b>
                const double dAx = 2.0 * pl.a * SB[0][ax + 1][ox] - (ax > 0 ? ax * SB[0][ax > 0 ? ax - 1 : 0][ox] : 0.0);
                const double dAy = 2.0 * pl.a * SB[1][ay + 1][oy] - (ay > 0 ? ay * SB[1][ay > 0 ? ay - 1 : 0][oy] : 0.0);
                const double dAz = 2.0 * pl.a * SB[2][az + 1][oz] - (az > 0 ? az * SB[2][az > 0 ? az - 1 : 0][oz] : 0.0);
                const double gb = g_ab * wB[op];
                g[0] -= gb * dAx * sy * sz;
                g[1] -= gb * sx * dAy * sz;
                g[2] -= gb * sx * sy * dAz;
            }
        }
        if (mode & MOM_FOCK) {
            const double f = seg_reduce(-0.5 * coef * fB, take);
            if (head && pl.active) {
                atomicAdd(F + r * bd.nao + c, f);
                if (mirror) atomicAdd(F + c * bd.nao + r, f);
            }
        }
    }
    if (mode & MOM_MULT) {
#pragma unroll
        for (int k = 0; k < 10; ++k) {
            const double vb = seg_reduce(mirror ? coef * mB[k] : 0.0, take);
            if (head && pl.active && mirror) atomicAdd(mult + 10 * pl.atomB + k, vb);
        }
    }
    if (mode & MOM_PULAY) {
#pragma unroll
        for (int x = 0; x < 3; ++x) {
            const double v = seg_reduce(pulay ? coef * g[x] : 0.0, take);
            if (head && pl.active && pl.atomA != pl.atomB) {
                atomicAdd(gqm + 3 * pl.atomA + x, v);
                atomicAdd(gqm + 3 * pl.atomB + x, -v);
            }
        }
    }
}

// Mulliken octupoles (SI, fourth multipole definition):
//   Omega_k,abc = - sum_{mu in k, nu} gamma_{nu mu} <mu|(r-R_k)_a (r-R_k)_b (r-R_k)_c|nu>.
// Third 1-D moment about K from the Hermite expansion:
//   M^3 = (X^3 + 3hX, 3X^2 + 3h, 6X, 6), h = 1/(2p), X = P - K.
__constant__ int c_o3x[10] = {3, 2, 2, 1, 1, 1, 0, 0, 0, 0};
__constant__ int c_o3y[10] = {0, 1, 0, 2, 1, 0, 3, 2, 1, 0};
__constant__ int c_o3z[10] = {0, 0, 1, 0, 1, 2, 0, 1, 2, 3};

template <int LA, int LB>
__global__ void __launch_bounds__(128)
k_octupoles(BasisDev bd, int pp_begin, int pp_end, const double *__restrict__ dm, double *__restrict__ oct)
{
    constexpr int NA = ncart(LA), NB = ncart(LB);
    const int lane = threadIdx.x & 31;
    const int i = pp_begin + (blockIdx.x * blockDim.x + threadIdx.x);
    if (pp_begin + (int)((blockIdx.x * blockDim.x + (threadIdx.x & ~31))) >= pp_end) return;  // whole warp out
    const PPLane pl = load_pp(bd, i, pp_end);
    const bool mirror = pl.sp.shA != pl.sp.shB;
    // 1-D moments of order 0 and 3 about A and B, per direction (orders 1, 2 are not needed)
    double SA[3][LA + 1][LB + 1][4], SB[3][LA + 1][LB + 1][4];
    {
        double E[LA + 1][LB + 1][LA + LB + 1];
        const double h = 0.5 * pl.ip;
#pragma unroll 1
        for (int d = 0; d < 3; ++d) {
            hermite_E<LA, LB, double>(E, pl.P[d] - pl.A[d], pl.P[d] - pl.B[d], h);
            const double XA = pl.P[d] - pl.A[d], XB = pl.P[d] - pl.B[d];
#pragma unroll
            for (int a = 0; a <= LA; ++a)
#pragma unroll
                for (int b = 0; b <= LB; ++b) {
                    // E^{ab}_t vanishes for t > a + b; the array holds t <= LA + LB only
                    const double e0 = E[a][b][0];
                    double e1 = 0.0, e2 = 0.0, e3 = 0.0;
                    if constexpr (LA + LB >= 1) e1 = (a + b >= 1) ? E[a][b][1] : 0.0;
                    if constexpr (LA + LB >= 2) e2 = (a + b >= 2) ? E[a][b][2] : 0.0;
                    if constexpr (LA + LB >= 3) e3 = (a + b >= 3) ? E[a][b][3] : 0.0;
                    SA[d][a][b][0] = e0;
                    SA[d][a][b][1] = XA * e0 + e1;
                    SA[d][a][b][2] = (XA * XA + h) * e0 + 2.0 * XA * e1 + 2.0 * e2;
                    SA[d][a][b][3] = (XA * XA + 3.0 * h) * XA * e0 + 3.0 * (XA * XA + h) * e1 + 6.0 * XA * e2 + 6.0 * e3;
                    SB[d][a][b][0] = e0;
                    SB[d][a][b][1] = XB * e0 + e1;
                    SB[d][a][b][2] = (XB * XB + h) * e0 + 2.0 * XB * e1 + 2.0 * e2;
                    SB[d][a][b][3] = (XB * XB + 3.0 * h) * XB * e0 + 3.0 * (XB * XB + h) * e1 + 6.0 * XB * e2 + 6.0 * e3;
                }
        }
    }
    const double spp = PI * pl.ip;
    const double coef = pl.active ? pl.cab * spp * sqrt(spp) : 0.0;
    bool take[5], head;
    seg_setup(pl.active ? pl.s : -1 - lane, lane, take, head);
    double mA[10], mB[10];
#pragma unroll
    for (int k = 0; k < 10; ++k) mA[k] = mB[k] = 0.0;
#pragma unroll 1
    for (int ia = 0; ia < NA; ++ia) {
#pragma unroll 1
        for (int ib = 0; ib < NB; ++ib) {
            const int ax = cart_lx(LA, ia), ay = cart_ly(LA, ia), az = cart_lz(LA, ia);
            const int bx = cart_lx(LB, ib), by = cart_ly(LB, ib), bz = cart_lz(LB, ib);
            const size_t r = pl.sp.aoA + ia, c = pl.sp.aoB + ib;
            const double g_ba = pl.active ? dm[c * bd.nao + r] : 0.0;
            const double g_ab = pl.active ? dm[r * bd.nao + c] : 0.0;
#pragma unroll
            for (int op = 0; op < 10; ++op) {
                const int ox = c_o3x[op], oy = c_o3y[op], oz = c_o3z[op];
                mA[op] -= g_ba * SA[0][ax][bx][ox] * SA[1][ay][by][oy] * SA[2][az][bz][oz];
                mB[op] -= g_ab * SB[0][ax][bx][ox] * SB[1][ay][by][oy] * SB[2][az][bz][oz];
            }
        }
    }
#pragma unroll
    for (int k = 0; k < 10; ++k) {
        const double va = seg_reduce(coef * mA[k], take);
        const double vb = seg_reduce(mirror ? coef * mB[k] : 0.0, take);
        if (head && pl.active) {
            atomicAdd(oct + 10 * pl.atomA + k, va);
            if (mirror) atomicAdd(oct + 10 * pl.atomB + k, vb);
        }
    }
}

template <int LA, int LB>
struct Octupoles {
    static cudaError_t run(const BasisDev &bd, int pp_begin, int pp_end, const double *dm, double *oct,
                           cudaStream_t st)
    {
        const int grid = (pp_end - pp_begin + 127) / 128;
        k_octupoles<LA, LB><<<grid, 128, 0, st>>>(bd, pp_begin, pp_end, dm, oct);
        return cudaGetLastError();
    }
};

cudaError_t launch_octupoles(const BasisDev &b, int cls, int pp_begin, int pp_end, const double *dm, double *oct,
                             cudaStream_t st)
{
    if (pp_end <= pp_begin) return cudaSuccess;
    return dispatch_class<Octupoles>(cls, b, pp_begin, pp_end, dm, oct, st);
}

template <int LA, int LB>
struct Moments {
    static cudaError_t run(const BasisDev &bd, int pp_begin, int pp_end, const double *dm, const double *phi,
                           double *mult, double *F, double *gqm, int mode, cudaStream_t st)
    {
        const int n = pp_end - pp_begin;
        const int gx = (n + 127) / 128;
        if (!(mode & MOM_PULAY)) {
            k_moments<LA, LB><<<gx, 128, 0, st>>>(bd, pp_begin, pp_end, dm, phi, mult, F, gqm, mode);
            return cudaGetLastError();
        }
        k_mom_a<LA, LB><<<dim3(gx, ncart(LA)), 128, 0, st>>>(bd, pp_begin, pp_end, dm, phi, mult, F, gqm, mode);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        k_mom_b<LA, LB><<<dim3(gx, ncart(LB)), 128, 0, st>>>(bd, pp_begin, pp_end, dm, phi, mult, F, gqm, mode);
        return cudaGetLastError();
    }
};

cudaError_t launch_moments(const BasisDev &b, int cls, int pp_begin, int pp_end, const double *dm,
                           const double *phi, double *mult, double *F, double *gqm, int mode, cudaStream_t st)
{
    if (pp_end <= pp_begin) return cudaSuccess;
    return dispatch_class<Moments>(cls, b, pp_begin, pp_end, dm, phi, mult, F, gqm, mode, st);
}

}  // namespace qmmm
