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
