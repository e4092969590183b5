// Standalone in-place inverse of a symmetric positive definite matrix on the
// device: the factor of Sections 4.2-4.3 is cached as the explicit inverse of
// S = I + A Delta^{-1} A^T ("its inverse" is allowed where the factorisation
// is cached before the iterations), computed by Gauss-Jordan elimination
// without pivoting (safe for SPD: every pivot is a Schur-complement diagonal,
// positive).  One step per pivot k; the old row k and column k are copied to
// scratch before the rank-one update of the whole matrix.
#include <cuda_runtime.h>

#include <cmath>
#include <string>

#include "internal.h"

namespace hsde {

__global__ void k_gj1_copy(const double* __restrict__ S, int m, int k, double* __restrict__ rowbuf,
                           double* __restrict__ colbuf) {
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < m; j += gridDim.x * blockDim.x) {
        rowbuf[j] = S[(int64_t)k * m + j];
        colbuf[j] = S[(int64_t)j * m + k];
    }
}

__global__ void k_gj1_update(double* __restrict__ S, int m, int k, const double* __restrict__ rowbuf,
                             const double* __restrict__ colbuf) {
    const int i = blockIdx.y * blockDim.y + threadIdx.y;
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m || j >= m) return;
    const double piv = rowbuf[k];
    double val;
    if (i == k && j == k) val = 1.0 / piv;
    else if (i == k) val = rowbuf[j] / piv;
    else if (j == k) val = -colbuf[i] / piv;
    else val = S[(int64_t)i * m + j] - colbuf[i] * rowbuf[j] / piv;
    S[(int64_t)i * m + j] = val;
}

// Runs the m Gauss-Jordan steps on `st`; scratch holds 2m doubles.
int gj_inverse_single(double* S, int m, double* scratch, cudaStream_t st) {
    double* rowbuf = scratch;
    double* colbuf = scratch + m;
    const dim3 blk(32, 8);
    const dim3 grd((m + 31) / 32, (m + 7) / 8);
    const int cgrid = (m + 255) / 256;
    for (int k = 0; k < m; ++k) {
        k_gj1_copy<<<cgrid, 256, 0, st>>>(S, m, k, rowbuf, colbuf);
        k_gj1_update<<<grd, blk, 0, st>>>(S, m, k, rowbuf, colbuf);
    }
    return cudaGetLastError() == cudaSuccess ? HSDE_OK : HSDE_ECUDA;
}

}  // namespace hsde

extern "C" int hsde_spd_inverse(double* S, int32_t m, void* cuda_stream) {
    using namespace hsde;
    if (!S || m <= 0) return set_error(HSDE_EINVAL, "hsde_spd_inverse: null matrix or m <= 0");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(cuda_stream);
    double* scratch = nullptr;
    if (cudaMallocAsync(reinterpret_cast<void**>(&scratch), sizeof(double) * 2 * (size_t)m, st) != cudaSuccess)
        return set_error(HSDE_ENOMEM, "hsde_spd_inverse: scratch allocation failed");
    const int rc = gj_inverse_single(S, m, scratch, st);
    const cudaError_t e = cudaFreeAsync(scratch, st);
    if (rc != HSDE_OK) return set_error(rc, "hsde_spd_inverse: kernel launch failed");
    return e == cudaSuccess ? HSDE_OK : set_error(HSDE_ECUDA, "hsde_spd_inverse: cudaFreeAsync failed");
}

// ---------------------------------------------------------------------------
// Allocation-free variant.  Some callers cannot allocate device memory when
// they invert: code that runs while a CUDA graph is being captured under a
// framework that forbids allocation there, real-time or embedded hosts that
// fix their memory budget up front, and processes whose memory is owned by a
// pooling allocator that any stray cudaMalloc/cudaMallocAsync would bypass.
// This entry point runs the same Gauss-Jordan kernels with their pivot row
// and column taken from a fixed array in device memory instead.
// ---------------------------------------------------------------------------
#include <mutex>

namespace {

constexpr int32_t kNoAllocMaxM = 8192;   // largest m: 2 * 8192 doubles = 128 KiB per GPU
constexpr int kMaxDevices = 64;

// Pivot row and column scratch of hsde_spd_inverse_noalloc.  Every GPU that
// loads the library holds this array until the process exits.
static __device__ __align__(256) double g_gj_scratch[2 * kNoAllocMaxM];

std::mutex g_scratch_mu;
double* g_scratch_addr[kMaxDevices] = {};   // device address of g_gj_scratch, per device

}  // namespace

extern "C" int hsde_spd_inverse_noalloc(double* S, int32_t m, void* cuda_stream) {
    using namespace hsde;
    if (!S || m <= 0) return set_error(HSDE_EINVAL, "hsde_spd_inverse_noalloc: null matrix or m <= 0");
    if (m > kNoAllocMaxM)
        return set_error(HSDE_ERANGE, "hsde_spd_inverse_noalloc: m = " + std::to_string(m) +
                                          " exceeds the static scratch limit of " + std::to_string(kNoAllocMaxM));
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
        return set_error(HSDE_ECUDA, "hsde_spd_inverse_noalloc: no usable current device");
    double* scratch = nullptr;
    {
        // One-time set-up per device, with that device current: the host-side
        // name g_gj_scratch is not a device address; ask the runtime for it.
        std::lock_guard<std::mutex> lk(g_scratch_mu);
        if (!g_scratch_addr[dev]) {
            void* p = nullptr;
            const cudaError_t e = cudaGetSymbolAddress(&p, g_gj_scratch);
            if (e != cudaSuccess || !p)
                return set_error(HSDE_ECUDA, std::string("hsde_spd_inverse_noalloc: cudaGetSymbolAddress: ") +
                                                 cudaGetErrorString(e));
            g_scratch_addr[dev] = static_cast<double*>(p);
        }
        scratch = g_scratch_addr[dev];
    }
    // The scratch needs no clearing: each step writes the pivot row and
    // column before the update kernel reads them.
    const int rc = gj_inverse_single(S, m, scratch, reinterpret_cast<cudaStream_t>(cuda_stream));
    if (rc != HSDE_OK) return set_error(rc, "hsde_spd_inverse_noalloc: kernel launch failed");
    return HSDE_OK;
}
