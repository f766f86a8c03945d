// noalloc.cu -- an entry point that allocates nothing: the region-I nuclear-MM energy
//   E = sum_j sum_i Z_j q_i erf(r_ij / sigma_i) / r_ij   (1/r_ij for sigma_i <= 0)
// over caller-provided charges, with its per-block partial sums kept in a fixed file-scope
// device array instead of memory obtained from cudaMalloc.
//
// Who needs it: callers that must not allocate while they run -- an MD engine that reserves all
// device memory when it starts and calls the embedding from inside its time step (a cudaMalloc
// there would implicitly synchronise the device and stall its other streams), or a plugin whose
// device memory is owned by the host program's own pool allocator.  Everything they pass is
// device memory they already own; the only extra memory is the static array below, which every
// GPU that loads this library keeps until the process exits.
#include <mutex>
#include <string>

#include "device_common.cuh"
#include "qmmm_internal.h"

namespace {

constexpr int NOALLOC_THREADS = 256;
constexpr int NOALLOC_MAX_BLOCKS = 1024;  // 1024 * 256 = 262144 charges at most per call

// Scratch: one partial energy per block of the first kernel.  Shared by every call on a device;
// it keeps the last call's values, and each call overwrites exactly the slots it later reads.
static __device__ __align__(256) double g_noalloc_partial[NOALLOC_MAX_BLOCKS];

__global__ void __launch_bounds__(NOALLOC_THREADS)
k_enucmm_static(const double *__restrict__ qm_xyz, const double *__restrict__ Z, int natm,
                const double *__restrict__ chg /* n*4: x, y, z, q */, const double *__restrict__ sigma, int n,
                double *__restrict__ partial)
{
    __shared__ double ws[NOALLOC_THREADS / 32];
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    double E = 0.0;
    if (k < n) {
        const double cx = chg[4 * (size_t)k], cy = chg[4 * (size_t)k + 1], cz = chg[4 * (size_t)k + 2],
                     q = chg[4 * (size_t)k + 3];
        const double s = sigma[k];
        const double beta = s > 0.0 ? 1.0 / s : 0.0;
        for (int j = 0; j < natm; ++j) {
            const double x = qm_xyz[3 * j] - cx, y = qm_xyz[3 * j + 1] - cy, z = qm_xyz[3 * j + 2] - cz;
            const double r = sqrt(x * x + y * y + z * z);
            double f;
            if (beta > 0.0) {
                // a Gaussian charge on (or next to) the nucleus: erf(beta r)/r tends to 2 beta/sqrt(pi);
                // the two-term series is exact to rounding for beta r < 1e-4
                const double br = beta * r;
                f = br < 1e-4 ? beta * (2.0 / 1.7724538509055160273) * (1.0 - br * br * (1.0 / 3.0)) : erf(br) / r;
            } else {
                f = 1.0 / r;  // a point charge on a nucleus gives an infinite energy (+-inf or NaN in E)
            }
            E += Z[j] * q * f;
        }
    }
    E = qmmm::warp_sum(E);
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = E;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < NOALLOC_THREADS / 32; ++w) t += ws[w];
        partial[blockIdx.x] = t;  // every slot this call reads is written here first
    }
}

__global__ void k_enucmm_static_sum(const double *__restrict__ partial, int nblk, double *__restrict__ E)
{
    __shared__ double ws[32];
    double s = 0.0;
    for (int k = threadIdx.x; k < nblk; k += blockDim.x) s += partial[k];
    s = qmmm::warp_sum(s);
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += ws[w];
        E[0] = t;
    }
}

std::mutex g_noalloc_mutex;
double *g_noalloc_ptr[64] = {nullptr};  // device address of the scratch, per device ordinal

bool on_device(const void *p)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace

extern "C" int qmmm_nuclear_mm_energy_static(int natm, const double *qm_xyz, const double *Z, int ncharge,
                                             const double *charges, const double *sigma, double *E, void *stream)
{
    if (natm <= 0 || ncharge < 0 || !qm_xyz || !Z || !E || (ncharge > 0 && (!charges || !sigma))) {
        qmmm::set_last_error("null pointer or negative size");
        return QMMM_ERR_ARG;
    }
    const int nblk = ncharge > 0 ? (ncharge + NOALLOC_THREADS - 1) / NOALLOC_THREADS : 1;
    if (nblk > NOALLOC_MAX_BLOCKS) {
        qmmm::set_last_error("ncharge " + std::to_string(ncharge) + " exceeds the static scratch limit of " +
                          std::to_string(NOALLOC_MAX_BLOCKS * NOALLOC_THREADS) + " charges");
        return QMMM_ERR_ARG;
    }
    if (!on_device(qm_xyz) || !on_device(Z) || !on_device(E) || (ncharge > 0 && (!on_device(charges) || !on_device(sigma)))) {
        qmmm::set_last_error("every array must be device memory");
        return QMMM_ERR_ARG;
    }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
        cudaGetLastError();
        qmmm::set_last_error("no usable current device");
        return QMMM_ERR_CUDA;
    }
    double *scratch;
    {
        // set-up, once per device and with that device current: the array's name is a host-side
        // stand-in, the kernels need its device address
        std::lock_guard<std::mutex> lock(g_noalloc_mutex);
        if (!g_noalloc_ptr[dev]) {
            void *p = nullptr;
            const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_partial);
            if (e != cudaSuccess) {
                qmmm::set_last_error(std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
                return QMMM_ERR_CUDA;
            }
            g_noalloc_ptr[dev] = static_cast<double *>(p);
        }
        scratch = g_noalloc_ptr[dev];
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    k_enucmm_static<<<nblk, NOALLOC_THREADS, 0, st>>>(qm_xyz, Z, natm, charges, sigma, ncharge, scratch);
    k_enucmm_static_sum<<<1, 256, 0, st>>>(scratch, ncharge > 0 ? nblk : 0, E);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        qmmm::set_last_error(std::string("launch: ") + cudaGetErrorString(e));
        return QMMM_ERR_CUDA;
    }
    return QMMM_OK;
}

// ---------------------------------------------------------------------------------------------
// Self-test of the failure path: one block waits on an mbarrier that nothing completes (no copy
// is issued), so the bounded wait gives up after 20 ms, the kernel records DEVERR_TIMEOUT and
// returns.
// ---------------------------------------------------------------------------------------------
namespace {
__global__ void k_wait_for_nothing(int *err)
{
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) {
        qmmm::mbar_init(&bar, 1);
        qmmm::fence_mbar_init();
    }
    __syncthreads();
    qmmm::mbar_wait_bounded(&bar, 0, err, 20000000ull);  // 20 ms
}
}  // namespace

extern "C" int qmmm_selftest_bounded_wait(void *stream)
{
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int *err = nullptr;
    if (cudaMalloc(&err, sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        qmmm::set_last_error("cudaMalloc");
        return QMMM_ERR_ALLOC;
    }
    int flag = 0;
    cudaError_t e = cudaMemsetAsync(err, 0, sizeof(int), st);
    if (e == cudaSuccess) {
        k_wait_for_nothing<<<1, 64, 0, st>>>(err);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(&flag, err, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(err);
    if (e != cudaSuccess) {
        qmmm::set_last_error(std::string("self-test: ") + cudaGetErrorString(e));
        return QMMM_ERR_CUDA;
    }
    if (flag & qmmm::DEVERR_TIMEOUT) {
        qmmm::set_last_error("the bounded wait ran out, as intended");
        return QMMM_ERR_TIMEOUT;
    }
    qmmm::set_last_error("the wait completed although nothing could complete it");
    return QMMM_ERR_CUDA;
}
