// Cone projection of the clique blocks (Eq. Step2 on S = S_1 x ... x S_p)
// fused with the gather x_k = H_k x (Section 3.1), the rank-one correction of
// Eq. MatrixInverseResult on the s and v blocks, and the nu update of
// Eq. Step3 (z <- z - s_hat + s).
//
// For clique k, with xh = x_w - eta x_p gathered through H_k (the corrected
// x_hat of the affine step):
//   s_hat = (s + z - v + H_k xh)/2,  v_hat = (s + z + v - H_k xh)/2
//   a     = s_hat - z                  (the point projected in Eq. Step2)
//   s     = Pi_psd(a) = V max(Lambda, 0) V^T
//   z     = s - a,   v = v_hat
// and the stopping-rule partial ||H_k xh - s||^2 (full-vec weights).
//
// Eigensolver: cyclic two-sided Jacobi (Golub & Van Loan, symmetric Schur
// decomposition by 2x2 rotations) in shared memory, parallel ordering by the
// round-robin ("circle") tournament so that the c/2 rotations of a round are
// disjoint.  A rotation pair (kr, kc) updates the 2x2 block of rows
// {p_kr, q_kr} x columns {p_kc, q_kc} as J_kr^T X J_kc in place, so one pass
// applies the whole round to A; V <- V J in the same pass.  Odd sizes are
// padded with a zero row/column that is never rotated.  A group of G threads
// owns one clique (G = 8, 16 or 32 lanes of a warp, or a whole CTA for larger
// cliques); groups never wait on each other.
#include <cuda_runtime.h>

#include <cmath>

#include "internal.h"

namespace hsde {

template <typename T, int CMAX, int G>
struct ConeCfg {
    static constexpr int LD = CMAX + 1;
    static constexpr int K = CMAX / 2;
    static constexpr int NTH = (G >= 128) ? G : 128;
    static constexpr int GPB = NTH / G;
    // per group: A, V, rot cos/sin/tan, lambda, reduction scratch (T), then rot p/q (int)
    static constexpr size_t t_elems = 2 * CMAX * LD + 3 * K + CMAX + 32;
    static constexpr size_t bytes = t_elems * sizeof(T) + 2 * K * sizeof(int);
    static constexpr size_t group_bytes = (bytes + 15) / 16 * 16;
    static constexpr size_t smem = GPB * group_bytes;
};

template <int G>
__device__ __forceinline__ unsigned gmask() {
    if constexpr (G >= 32) {
        return 0xffffffffu;
    } else {
        const int base = (threadIdx.x & 31) & ~(G - 1);
        return ((1u << G) - 1u) << base;
    }
}

template <int G>
__device__ __forceinline__ void gsync() {
    if constexpr (G <= 32) __syncwarp(gmask<G>());
    else __syncthreads();
}

template <int G, typename T>
__device__ __forceinline__ T gsum(T v, T* red) {
    if constexpr (G <= 32) {
        const unsigned mask = gmask<G>();
#pragma unroll
        for (int o = G / 2; o > 0; o >>= 1) v += __shfl_xor_sync(mask, v, o, G);
        return v;
    } else {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        __syncthreads();
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
        __syncthreads();
        T t = 0;
#pragma unroll
        for (int i = 0; i < G / 32; ++i) t += red[i];
        __syncthreads();
        return t;
    }
}

__device__ __forceinline__ void rr_pair(int r, int k, int cp, int& p, int& q) {
    const int mm = cp - 1;
    if (k == 0) {
        p = mm;
        q = r;
    } else {
        p = (r + k) % mm;
        q = (r - k + mm) % mm;
    }
}

template <typename T>
__device__ __forceinline__ T t_sqrt(T x);
template <>
__device__ __forceinline__ float t_sqrt<float>(float x) { return sqrtf(x); }
template <>
__device__ __forceinline__ double t_sqrt<double>(double x) { return sqrt(x); }

template <typename T, int CMAX, int G>
__global__ void __launch_bounds__(ConeCfg<T, CMAX, G>::NTH)
k_cone(DevView V, const int32_t* __restrict__ list, int nlist, int max_sweeps, T tol2) {
    using C = ConeCfg<T, CMAX, G>;
    constexpr int LD = C::LD;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int g = threadIdx.x / G, lane = threadIdx.x % G;
    const int li = blockIdx.x * C::GPB + g;
    if (li >= nlist) return;
    const int k = list[li];
    const InstDev& I = V.inst[V.cl_inst[k]];
    if (I.status != HSDE_RUNNING) return;

    unsigned char* base = smem_raw + (size_t)g * C::group_bytes;
    T* A = reinterpret_cast<T*>(base);
    T* Vm = A + CMAX * LD;
    T* rc = Vm + CMAX * LD;
    T* rs = rc + C::K;
    T* rt = rs + C::K;
    T* lam = rt + C::K;
    T* red = lam + CMAX;
    int* rp = reinterpret_cast<int*>(red + 32);
    int* rq = rp + C::K;

    T* s = reinterpret_cast<T*>(V.s);
    T* z = reinterpret_cast<T*>(V.z);
    T* v = reinterpret_cast<T*>(V.v);
    const int c = V.cl_size[k];
    const int cp = (c + 1) & ~1;
    const int K = cp >> 1;
    const int64_t off = V.cl_off[k];
    const double eta = I.eta;

    for (int idx = lane; idx < cp * cp; idx += G) {
        const int i = idx / cp, j = idx - (idx / cp) * cp;
        A[i * LD + j] = T(0);
        Vm[i * LD + j] = (i == j) ? T(1) : T(0);
    }
    gsync<G>();
    // gather + rank-one correction: a = s_hat - z
    for (int b = 0, colbase = 0; b < c; colbase += c - b, ++b) {
        for (int a = b + lane; a < c; a += G) {
            const int64_t j = off + colbase + (a - b);
            const int gi = V.gmap[j];
            const double gx = V.xw[gi] - eta * V.xp[gi];
            const double av = 0.5 * ((double)s[j] - (double)z[j] - (double)v[j] + gx);
            A[a * LD + b] = (T)av;
            A[b * LD + a] = (T)av;
        }
    }
    gsync<G>();

    for (int sweep = 0; sweep <= max_sweeps; ++sweep) {
        // convergence test on the off-diagonal mass
        T offd = 0, tot = 0;
        for (int idx = lane; idx < c * c; idx += G) {
            const int i = idx / c, j = idx - (idx / c) * c;
            const T a = A[i * LD + j];
            tot += a * a;
            if (i != j) offd += a * a;
        }
        offd = gsum<G>(offd, red);
        tot = gsum<G>(tot, red);
        if (offd <= tol2 * tot || sweep == max_sweeps) break;
        for (int r = 0; r < cp - 1; ++r) {
            if (lane < K) {
                int p, q;
                rr_pair(r, lane, cp, p, q);
                const T app = A[p * LD + p], aqq = A[q * LD + q], apq = A[p * LD + q];
                T cs = 1, sn = 0, t = 0;
                if (apq != T(0)) {
                    const T theta = (aqq - app) / (T(2) * apq);
                    const T at = fabs(theta);
                    t = T(1) / (at + t_sqrt<T>(T(1) + theta * theta));
                    if (theta < T(0)) t = -t;
                    cs = T(1) / t_sqrt<T>(T(1) + t * t);
                    sn = t * cs;
                }
                rp[lane] = p; rq[lane] = q;
                rc[lane] = cs; rs[lane] = sn; rt[lane] = t;
            }
            gsync<G>();
            for (int idx = lane; idx < K * K; idx += G) {
                const int kr = idx / K, kc = idx - (idx / K) * K;
                const int pr = rp[kr], qr = rq[kr];
                if (kr == kc) {
                    const T t = rt[kr];
                    if (t != T(0)) {
                        const T apq = A[pr * LD + qr];
                        A[pr * LD + pr] -= t * apq;
                        A[qr * LD + qr] += t * apq;
                        A[pr * LD + qr] = T(0);
                        A[qr * LD + pr] = T(0);
                    }
                } else {
                    const int pc = rp[kc], qc = rq[kc];
                    const T cr = rc[kr], sr = rs[kr], cc = rc[kc], sc = rs[kc];
                    const T x00 = A[pr * LD + pc], x01 = A[pr * LD + qc];
                    const T x10 = A[qr * LD + pc], x11 = A[qr * LD + qc];
                    const T y00 = cr * x00 - sr * x10, y01 = cr * x01 - sr * x11;
                    const T y10 = sr * x00 + cr * x10, y11 = sr * x01 + cr * x11;
                    A[pr * LD + pc] = cc * y00 - sc * y01;
                    A[pr * LD + qc] = sc * y00 + cc * y01;
                    A[qr * LD + pc] = cc * y10 - sc * y11;
                    A[qr * LD + qc] = sc * y10 + cc * y11;
                }
            }
            for (int idx = lane; idx < cp * K; idx += G) {
                const int i = idx / K, kc = idx - (idx / K) * K;
                const int pc = rp[kc], qc = rq[kc];
                const T cc = rc[kc], sc = rs[kc];
                const T vp = Vm[i * LD + pc], vq = Vm[i * LD + qc];
                Vm[i * LD + pc] = cc * vp - sc * vq;
                Vm[i * LD + qc] = sc * vp + cc * vq;
            }
            gsync<G>();
        }
    }
    for (int i = lane; i < cp; i += G) lam[i] = fmax(A[i * LD + i], T(0));
    gsync<G>();

    double res = 0.0;
    for (int b = 0, colbase = 0; b < c; colbase += c - b, ++b) {
        for (int a = b + lane; a < c; a += G) {
            T acc = 0;
            for (int q = 0; q < c; ++q) acc += Vm[a * LD + q] * lam[q] * Vm[b * LD + q];
            const int64_t j = off + colbase + (a - b);
            const int gi = V.gmap[j];
            const double gx = V.xw[gi] - eta * V.xp[gi];
            const double so = s[j], zo = z[j], vo = v[j];
            const double av = 0.5 * (so - zo - vo + gx);
            const double vn = 0.5 * (so + zo + vo - gx);
            const double sn = (double)acc;
            s[j] = (T)sn;
            z[j] = (T)(sn - av);
            v[j] = (T)vn;
            const double d = gx - sn;
            res += (a == b ? 1.0 : 2.0) * d * d;
        }
    }
    // fixed-order group reduction in double
    if constexpr (G <= 32) {
        const unsigned mask = gmask<G>();
#pragma unroll
        for (int o = G / 2; o > 0; o >>= 1) res += __shfl_xor_sync(mask, res, o, G);
        if (lane == 0) V.cl_part[k] = res;
    } else {
        double* dred = reinterpret_cast<double*>(A);   // A is no longer needed
        __syncthreads();
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) res += __shfl_xor_sync(0xffffffffu, res, o);
        if ((threadIdx.x & 31) == 0) dred[threadIdx.x >> 5] = res;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0;
            for (int i = 0; i < G / 32; ++i) t += dred[i];
            V.cl_part[k] = t;
        }
    }
}

template <typename T, int CMAX, int G>
static int launch_one(const DevView& V, const Bucket& bk, int max_sweeps, double tol, cudaStream_t st) {
    using C = ConeCfg<T, CMAX, G>;
    auto kern = k_cone<T, CMAX, G>;
    const int grid = (bk.count + C::GPB - 1) / C::GPB;
    kern<<<grid, C::NTH, C::smem, st>>>(V, bk.list, bk.count, max_sweeps, (T)(tol * tol));
    return HSDE_OK;
}

template <typename T, int CMAX, int G>
static int prepare_one() {
    using C = ConeCfg<T, CMAX, G>;
    if (C::smem > 48 * 1024) {
        if (cudaFuncSetAttribute(k_cone<T, CMAX, G>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)C::smem) != cudaSuccess)
            return HSDE_ECUDA;
    }
    return HSDE_OK;
}

// Opt every variant into its dynamic shared memory size (outside any capture).
int cone_prepare(bool mixed) {
    int rc = HSDE_OK;
    if (mixed) {
        rc |= prepare_one<float, 8, 8>();
        rc |= prepare_one<float, 16, 16>();
        rc |= prepare_one<float, 32, 32>();
        rc |= prepare_one<float, 64, 128>();
        rc |= prepare_one<float, 128, 256>();
    } else {
        rc |= prepare_one<double, 8, 8>();
        rc |= prepare_one<double, 16, 16>();
        rc |= prepare_one<double, 32, 32>();
        rc |= prepare_one<double, 64, 128>();
    }
    return rc == HSDE_OK ? HSDE_OK : HSDE_ECUDA;
}

int cone_smem_bytes(int cmax, bool mixed) {
    if (mixed) {
        switch (cmax) {
            case 8: return (int)ConeCfg<float, 8, 8>::smem;
            case 16: return (int)ConeCfg<float, 16, 16>::smem;
            case 32: return (int)ConeCfg<float, 32, 32>::smem;
            case 64: return (int)ConeCfg<float, 64, 128>::smem;
            case 128: return (int)ConeCfg<float, 128, 256>::smem;
        }
    } else {
        switch (cmax) {
            case 8: return (int)ConeCfg<double, 8, 8>::smem;
            case 16: return (int)ConeCfg<double, 16, 16>::smem;
            case 32: return (int)ConeCfg<double, 32, 32>::smem;
            case 64: return (int)ConeCfg<double, 64, 128>::smem;
        }
    }
    return -1;
}

int launch_cone(const DevView& V, const Bucket& bk, bool mixed, int max_sweeps, double tol, void* stp) {
    if (bk.count == 0) return HSDE_OK;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stp);
    if (mixed) {
        switch (bk.cmax) {
            case 8: return launch_one<float, 8, 8>(V, bk, max_sweeps, tol, st);
            case 16: return launch_one<float, 16, 16>(V, bk, max_sweeps, tol, st);
            case 32: return launch_one<float, 32, 32>(V, bk, max_sweeps, tol, st);
            case 64: return launch_one<float, 64, 128>(V, bk, max_sweeps, tol, st);
            case 128: return launch_one<float, 128, 256>(V, bk, max_sweeps, tol, st);
        }
    } else {
        switch (bk.cmax) {
            case 8: return launch_one<double, 8, 8>(V, bk, max_sweeps, tol, st);
            case 16: return launch_one<double, 16, 16>(V, bk, max_sweeps, tol, st);
            case 32: return launch_one<double, 32, 32>(V, bk, max_sweeps, tol, st);
            case 64: return launch_one<double, 64, 128>(V, bk, max_sweeps, tol, st);
        }
    }
    return HSDE_ERANGE;
}

}  // namespace hsde
