// misc.cu -- deterministic energy reductions and MM reordering.
//
// E_QM-MM = sum gamma V (region-I electronic, Eq. 9) + E_nuc_mm + E_II, with
// E_II = sum_j sum_c w_c M_j,c v_j,c (Eq. 6 QM-MM lines + Eq. 10); every sum here runs in a fixed
// order so repeated calls give identical bits.
#include <algorithm>
#include <string>

#include "device_common.cuh"
#include "qmmm_internal.h"

namespace qmmm {

__global__ void k_dot_partials(const double *a, const double *b, size_t n, double *partials)
{
    __shared__ double ws[32];
    double s = 0.0;
    for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (size_t)gridDim.x * blockDim.x)
        s += a[k] * b[k];
    s = warp_sum(s);
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += ws[w];
        partials[blockIdx.x] = t;
    }
}

__global__ void k_energy_final(const double *partials, int npart, const double *Epart, int nE, const double *mult,
                               const double *phi, int natm, int have_V, double *out4)
{
    __shared__ double ws[3][32];
    double eI = 0.0, en = 0.0, e2 = 0.0;
    if (have_V)
        for (int k = threadIdx.x; k < npart; k += blockDim.x) eI += partials[k];
    for (int k = threadIdx.x; k < nE; k += blockDim.x) en += Epart[k];
    for (int k = threadIdx.x; k < natm * 10; k += blockDim.x) {
        const int j = k / 10, c = k % 10;
        e2 += w10(c) * mult[k] * phi[20 * j + c];
    }
    eI = warp_sum(eI);
    en = warp_sum(en);
    e2 = warp_sum(e2);
    if ((threadIdx.x & 31) == 0) {
        ws[0][threadIdx.x >> 5] = eI;
        ws[1][threadIdx.x >> 5] = en;
        ws[2][threadIdx.x >> 5] = e2;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, b = 0.0, c = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            a += ws[0][w];
            b += ws[1][w];
            c += ws[2][w];
        }
        out4[0] = a + b + c;
        out4[1] = a;
        out4[2] = b;
        out4[3] = c;
    }
}

cudaError_t launch_energy_terms(const double *dm, const double *V, int nao, int have_V, const double *mult,
                                const double *phi, int natm, const double *Epart, int nEpart, double *partials,
                                int npart, double *out4, cudaStream_t st)
{
    if (have_V) {
        k_dot_partials<<<npart, 256, 0, st>>>(dm, V, (size_t)nao * nao, partials);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    k_energy_final<<<1, 512, 0, st>>>(partials, npart, Epart, nEpart, mult, phi, natm, have_V, out4);
    return cudaGetLastError();
}

__global__ void k_gather_mm(const double *xyz_user, const double *q_user, const int *perm, int nmm, double *xyz,
                            double *q)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nmm) return;
    const int u = perm[i];
    if (xyz_user) {
        xyz[3 * i] = xyz_user[3 * u];
        xyz[3 * i + 1] = xyz_user[3 * u + 1];
        xyz[3 * i + 2] = xyz_user[3 * u + 2];
    }
    if (q_user) q[i] = q_user[u];
}

cudaError_t launch_gather_mm(const double *xyz_user, const double *q_user, const int *perm, int nmm, double *xyz,
                             double *q, cudaStream_t st)
{
    k_gather_mm<<<(nmm + 255) / 256, 256, 0, st>>>(xyz_user, q_user, perm, nmm, xyz, q);
    return cudaGetLastError();
}

__global__ void k_unpermute(const double *dq_int, const double *dR_int, const int *perm, int nmm, double *dq,
                            double *dR)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nmm) return;
    const int u = perm[i];
    if (dq) dq[u] = dq_int[i];
    if (dR) {
        dR[3 * u] = dR_int[3 * i];
        dR[3 * u + 1] = dR_int[3 * i + 1];
        dR[3 * u + 2] = dR_int[3 * i + 2];
    }
}

cudaError_t launch_unpermute(const double *dq_int, const double *dR_int, const int *perm, int nmm, double *dq,
                             double *dR, cudaStream_t st)
{
    k_unpermute<<<(nmm + 255) / 256, 256, 0, st>>>(dq_int, dR_int, perm, nmm, dq, dR);
    return cudaGetLastError();
}

__global__ void k_sum_slices_d(const double *src, int nslice, size_t n, double *dst)
{
    for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (size_t)gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int sl = 0; sl < nslice; ++sl) s += src[(size_t)sl * n + k];
        dst[k] = s;
    }
}

cudaError_t launch_sum_slices_d(const double *src, int nslice, size_t n, double *dst, cudaStream_t st)
{
    if (n == 0) return cudaSuccess;
    const int grid = (int)std::min<size_t>((n + 255) / 256, 8192);
    k_sum_slices_d<<<grid, 256, 0, st>>>(src, nslice, n, dst);
    return cudaGetLastError();
}

// ASPC density predictor: out = sum_j B_j hist_j (the weights come from the host)
struct AspcArgs {
    const double *h[9];
    double B[9];
    int m;
};

__global__ void k_aspc(AspcArgs a, size_t n, double *out)
{
    for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (size_t)gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int j = 0; j < a.m; ++j) s += a.B[j] * a.h[j][k];
        out[k] = s;
    }
}

}  // namespace qmmm

namespace {
bool dev_ptr(const void *p)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}
}  // namespace

extern "C" int qmmm_aspc_predict(int nhist, const double *const *hist, size_t n, double *out, void *stream)
{
    if (nhist < 1 || nhist > 9 || !hist || !out) {
        qmmm::set_last_error("need 1 <= nhist <= 9 and non-null arrays");
        return QMMM_ERR_ARG;
    }
    qmmm::AspcArgs a;
    a.m = nhist;
    const int K = nhist - 1;
    auto comb = [](int N, int k) {
        if (k < 0 || k > N) return 0.0;
        double c = 1.0;
        for (int t = 1; t <= k; ++t) c = c * (N - k + t) / t;
        return c;
    };
    for (int j = 1; j <= nhist; ++j) {
        if (!hist[j - 1] || !dev_ptr(hist[j - 1])) {
            qmmm::set_last_error("history arrays must be device memory");
            return QMMM_ERR_ARG;
        }
        a.h[j - 1] = hist[j - 1];
        a.B[j - 1] = ((j % 2) ? 1.0 : -1.0) * j * comb(2 * K + 2, K + 1 - j) / comb(2 * K, K);
    }
    if (!dev_ptr(out)) {
        qmmm::set_last_error("output must be device memory");
        return QMMM_ERR_ARG;
    }
    if (n == 0) return QMMM_OK;
    const int grid = (int)std::min<size_t>((n + 255) / 256, 4096);
    qmmm::k_aspc<<<grid, 256, 0, static_cast<cudaStream_t>(stream)>>>(a, n, out);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        qmmm::set_last_error(std::string("k_aspc: ") + cudaGetErrorString(e));
        return QMMM_ERR_CUDA;
    }
    return QMMM_OK;
}
