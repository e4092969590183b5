// Cone projections by tridiagonalisation + implicit QR (Eq. Step2 on
// S = S_1 x ... x S_p), fused with the gather, the rank-one correction of
// Eq. MatrixInverseResult and the nu update of Eq. Step3 exactly as the
// Jacobi kernel in cone.cu does (same per-entry arithmetic, cone_common.cuh).
// Two kernels:
//
// k_cone_big<T>: the cliques above the Jacobi bucket sizes (the large cliques
// of Table 1, e.g. the 304-vertex clique of qpG51), up to CONE_BIG.  One CTA
// of 512 threads per clique; the c x c matrix and Q^T live in a per-clique
// workspace in global memory (L2-resident: 2 ld^2 elements, ld = c rounded
// up to 16), the tridiagonal and the rotations in shared memory.
//  1. Householder tridiagonalisation (Golub & Van Loan, symmetric
//     Householder tridiagonalisation): for j = 0 .. c-3 the reflection
//     H_j = I - beta v v^T that zeroes row j beyond j+1 is applied to the
//     trailing block as B <- B - v w^T - w v^T with p = beta B v,
//     w = p - (beta p^T v / 2) v.  v is kept in row j of the workspace.
//     From the first step whose trailing block fits the shared memory left
//     over, that block is copied there and the steps continue on it.
//  2. Q = H_0 H_1 ... H_{c-3}, accumulated backwards on Q^T (row k of QT is
//     eigenvector k): QT_sub <- QT_sub - beta (QT_sub v) v^T, in shared
//     memory while the growing block fits.
//  3. Implicit symmetric QR with the Wilkinson shift on the tridiagonal
//     (d, e), scaled by a power of two to norm [1, 2), deflating from the
//     bottom.  Lane 0 of warp 0 chases the bulge of each step and writes its
//     rotations into a ring of QR_SLOTS slots; warps 1 .. apply them to the
//     rows of QT (each thread carries whole columns through the chain,
//     coalesced over the threads), meeting the chase on mbarriers whose
//     waits are bounded.  A step that would exceed 30 c steps in total stops
//     the solve; the clique is then counted as unconverged.
//  4. Rebuild s = Q max(Lambda, 0) Q^T on the lower triangle: in FP32 with
//     tensor cores as split-precision TF32 (each operand a = a_hi + a_lo,
//     both TF32; a_hi b_hi + a_hi b_lo + a_lo b_hi accumulated in FP32,
//     which keeps FP32 accuracy), in FP64 by FMA loops.
//  5. s, z, v and the clique's stopping-rule partials as in cone.cu.
//
// k_cone_qrw<CP>: many cliques of 33 to 64 in the mixed form (on request,
// options.eigensolver): one warp per clique with everything in shared
// memory (see the comment above it).
//
// A clique's workspace is private to its CTA; nothing waits on another CTA.
#include <cuda_runtime.h>

#include <cstdint>
#include <type_traits>

#include "cone_common.cuh"
#include "internal.h"

namespace hsde {

namespace {

constexpr int BIG_NT = 512;
constexpr int BIG_WARPS = BIG_NT / 32;
constexpr int BIG_CHASERS = 32;   // warp 0 chases; the other warps apply rotations
constexpr int QR_SLOTS = 4;       // QR steps the chase may run ahead of their application

template <typename T> struct QrEps;
template <> struct QrEps<float> { static constexpr float value = 1.1920929e-7f; };     // 2^-23
template <> struct QrEps<double> { static constexpr double value = 2.220446049250313e-16; };   // 2^-52

// Sum over the CTA, in an order fixed by the thread count: a shuffle tree in
// each warp, then warp 0 combines the warp sums by a shuffle tree and
// publishes the total.  Every thread gets the result.  red holds
// BIG_WARPS + 1 values of S.
template <typename S>
__device__ __forceinline__ S block_sum(S v, S* red) {
    static_assert(BIG_WARPS <= 32, "one warp combines the warp sums");
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();   // red is free (an earlier block_sum has been read)
    if (lane == 0) red[warp] = v;
    __syncthreads();
    if (warp == 0) {
        S t = lane < BIG_WARPS ? red[lane] : S(0);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if (lane == 0) red[BIG_WARPS] = t;
    }
    __syncthreads();
    return red[BIG_WARPS];
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ float qr_hypot(float a, float b) { return hypotf(a, b); }
__device__ __forceinline__ double qr_hypot(double a, double b) { return hypot(a, b); }

// Rotation (cs, sn, r) with cs x + sn z = r = sqrt(x^2 + z^2), -sn x + cs z = 0,
// on the chase's critical path.  The tridiagonal is scaled before the QR
// steps so that |x|, |z| <= 4, so x^2 + z^2 cannot overflow; a sum below
// 1e-30 (FP32) or 1e-36 (FP64), both entries negligible against the matrix
// norm 1, gives the identity rotation.  FP32: the hardware reciprocal square root (no
// branch); FP64: its FP32 value refined by two Newton steps
// y <- y (3 - q y^2) / 2 (each doubles the correct digits: ~2^-22 -> 2^-44
// -> below 2^-53).
__device__ __forceinline__ float rsqrt_hw(float q) {
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(q));
    return y;
}
__device__ __forceinline__ void givens(float x, float z, float& cs, float& sn, float& r) {
    const float q = fmaf(x, x, z * z);
    const bool ok = q > 1e-30f;
    const float iq = rsqrt_hw(ok ? q : 1.f);
    cs = ok ? x * iq : 1.f;
    sn = ok ? z * iq : 0.f;
    r = ok ? q * iq : 0.f;
}
__device__ __forceinline__ void givens(double x, double z, double& cs, double& sn, double& r) {
    const double q = fma(x, x, z * z);
    const bool ok = q > 1e-36;   // (float)q stays a normal number
    const double qq = ok ? q : 1.0;
    double y = (double)rsqrt_hw((float)qq);
    y = y * fma(-0.5 * qq, y * y, 1.5);
    y = y * fma(-0.5 * qq, y * y, 1.5);
    cs = ok ? x * y : 1.0;
    sn = ok ? z * y : 0.0;
    r = ok ? q * y : 0.0;
}

__device__ __forceinline__ float fma_t(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double fma_t(double a, double b, double c) { return fma(a, b, c); }

// mbarrier helpers (CTA scope) for the chase / apply pipeline.  A wait
// polls at most QR_WAIT_LIMIT times and reports failure instead of
// waiting on.
constexpr int QR_WAIT_LIMIT = 1 << 22;

__device__ __forceinline__ void mbar_init(uint64_t* b, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"((unsigned)__cvta_generic_to_shared(b)), "r"(count)
                 : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* b) {
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(
                     (unsigned)__cvta_generic_to_shared(b))
                 : "memory");
}
// true once the phase of the given parity has completed
__device__ __forceinline__ bool mbar_wait(uint64_t* b, unsigned parity) {
    const unsigned a = (unsigned)__cvta_generic_to_shared(b);
    for (int it = 0; it < QR_WAIT_LIMIT; ++it) {
        unsigned done;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

// out[r] = scale * sum_i M[r][i] vec[i] for rows r < L of the block at M
// (row stride ld), columns i < L: a warp per group of RG rows, so that a
// lane has the loads of RG rows in flight.
constexpr int RG = 8;

template <typename T>
__device__ __forceinline__ void rows_matvec(const T* __restrict__ M, int ld, int L, const T* __restrict__ vec,
                                            T scale, T* __restrict__ out) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int r0 = RG * warp; r0 < L; r0 += RG * BIG_WARPS) {
        const int nr = L - r0 < RG ? L - r0 : RG;
        const T* mr[RG];
        T a[RG];
#pragma unroll
        for (int q = 0; q < RG; ++q) {
            mr[q] = M + (size_t)(r0 + (q < nr ? q : 0)) * ld;
            a[q] = T(0);
        }
        for (int i = lane; i < L; i += 32) {
            T x[RG];
#pragma unroll
            for (int q = 0; q < RG; ++q) x[q] = mr[q][i];
            const T vi = vec[i];
#pragma unroll
            for (int q = 0; q < RG; ++q) a[q] += x[q] * vi;
        }
#pragma unroll
        for (int q = 0; q < RG; ++q) a[q] = warp_sum(a[q]);
        if (lane < nr) {
            T o = a[0];
#pragma unroll
            for (int q = 1; q < RG; ++q) o = lane == q ? a[q] : o;
            out[r0 + lane] = scale * o;
        }
    }
}

// M[r][i] -= u[r] v[i] + (w ? w[r] x[i] : 0) for r, i < L: RG rows of a
// warp at a time, loads first.
template <typename T>
__device__ __forceinline__ void rows_update(T* __restrict__ M, int ld, int L, const T* __restrict__ u,
                                            const T* __restrict__ vv, const T* __restrict__ w,
                                            const T* __restrict__ xv) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int r0 = RG * warp; r0 < L; r0 += RG * BIG_WARPS) {
        const int nr = L - r0 < RG ? L - r0 : RG;
        T* mr[RG];
        T ur[RG], wr[RG];
#pragma unroll
        for (int q = 0; q < RG; ++q) {
            const int r = r0 + (q < nr ? q : 0);
            mr[q] = M + (size_t)r * ld;
            ur[q] = u[r];
            wr[q] = w ? w[r] : T(0);
        }
        for (int i = lane; i < L; i += 32) {
            T x[RG];
#pragma unroll
            for (int q = 0; q < RG; ++q) x[q] = mr[q][i];
            const T vi = vv[i], xi = w ? xv[i] : T(0);
#pragma unroll
            for (int q = 0; q < RG; ++q)
                if (q < nr) mr[q][i] = x[q] - (ur[q] * vi + wr[q] * xi);
        }
    }
}

// FP32 -> TF32 (round to nearest, ties away), as a 32-bit pattern.
__device__ __forceinline__ uint32_t to_tf32(float a) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(a));
    return r;
}

// D += A B for one 16 x 8 x 8 TF32 tile (warp-wide; FP32 accumulators).
__device__ __forceinline__ void mma_tf32(float (&d)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
    asm volatile(
        "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// Split-precision TF32 rebuild of the lower triangle of QT^T diag(lam) QT
// into W (row-major, stride ld).  Tiles of 16 x 8 on or below the diagonal,
// one warp per tile; A(m, k) = lam_k QT[k][m], B(k, n) = QT[k][n].  Blocks of
// 8 eigenvalues that are all clamped to zero are skipped (warp-uniform).
// Fragment layout of m16n8k8 (TF32): with g = lane / 4, t = lane % 4,
// a0 (g, t), a1 (g + 8, t), a2 (g, t + 4), a3 (g + 8, t + 4); b0 (t, g),
// b1 (t + 4, g); d0 (g, 2t), d1 (g, 2t + 1), d2 (g + 8, 2t), d3 (g + 8, 2t + 1).
__device__ void rebuild_tf32x3(const float* __restrict__ QT, const float* __restrict__ lam, float* __restrict__ W,
                               int c, int ld) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int g = lane >> 2, t = lane & 3;
    const int mtiles = ld / 16;
    const int ntile_total = mtiles * (mtiles + 1);   // row block mt has 2 mt + 2 column tiles of 8
    for (int tile = warp; tile < ntile_total; tile += BIG_WARPS) {
        int mt = (int)((sqrtf(4.f * tile + 1.f) - 1.f) * 0.5f);
        while (mt > 0 && mt * (mt + 1) > tile) --mt;
        while ((mt + 1) * (mt + 2) <= tile) ++mt;
        const int nt = tile - mt * (mt + 1);
        const int m0 = mt * 16, n0 = nt * 8;
        if (m0 >= c || n0 >= c) continue;   // warp-uniform
        float acc[4] = {0.f, 0.f, 0.f, 0.f};
        for (int k0 = 0; k0 < c; k0 += 8) {
            const float l0 = lam[k0 + t], l1 = lam[k0 + t + 4];
            if (__all_sync(0xffffffffu, l0 == 0.f && l1 == 0.f)) continue;
            const float* r0 = QT + (size_t)(k0 + t) * ld;
            const float* r1 = QT + (size_t)(k0 + t + 4) * ld;
            const float av[4] = {l0 * r0[m0 + g], l0 * r0[m0 + g + 8], l1 * r1[m0 + g], l1 * r1[m0 + g + 8]};
            const float bv[2] = {r0[n0 + g], r1[n0 + g]};
            uint32_t ah[4], al[4], bh[2], bl[2];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                ah[q] = to_tf32(av[q]);
                al[q] = to_tf32(av[q] - __uint_as_float(ah[q]));
            }
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                bh[q] = to_tf32(bv[q]);
                bl[q] = to_tf32(bv[q] - __uint_as_float(bh[q]));
            }
            mma_tf32(acc, al, bh);   // small terms first
            mma_tf32(acc, ah, bl);
            mma_tf32(acc, ah, bh);
        }
        const int rr[4] = {m0 + g, m0 + g, m0 + g + 8, m0 + g + 8};
        const int cc[4] = {n0 + 2 * t, n0 + 2 * t + 1, n0 + 2 * t, n0 + 2 * t + 1};
#pragma unroll
        for (int q = 0; q < 4; ++q)
            if (rr[q] < c && cc[q] <= rr[q]) W[(size_t)rr[q] * ld + cc[q]] = acc[q];
    }
}

// FP64 rebuild: a warp per row m, lanes over the columns n <= m, summing over
// the eigenvalues that stay positive (pos[0 .. npos)).
__device__ void rebuild_fp64(const double* __restrict__ QT, const double* __restrict__ lam,
                             const int* __restrict__ pos, int npos, double* __restrict__ W, int c, int ld) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int m = warp; m < c; m += BIG_WARPS) {
        for (int n = lane; n <= m; n += 32) {
            double a = 0.0;
            for (int q = 0; q < npos; ++q) {
                const int k = pos[q];
                const double* r = QT + (size_t)k * ld;
                a = fma(lam[k] * r[m], r[n], a);
            }
            W[(size_t)m * ld + n] = a;
        }
    }
}

// Bytes of the per-clique arrays in shared memory for cliques up to ld
// (rounded up to 16), 16-byte aligned; the trailing-block buffer follows.
template <typename T>
__host__ __device__ constexpr size_t big_smem_base(int ld) {
    return ((size_t)(6 + 2 * QR_SLOTS) * ld * sizeof(T) + (BIG_WARPS + 2) * sizeof(double) +
            (size_t)ld * sizeof(int) + 15) /
           16 * 16;
}

template <typename T>
__global__ void __launch_bounds__(BIG_NT, 1)
k_cone_big(DevView V, const int32_t* __restrict__ list, int nlist, int ldmax, int cap) {
    static_assert(BIG_CHASERS == 32, "warp 0 is the chaser warp");
    const int li = blockIdx.x;
    if (li >= nlist) return;
    const int k = list[li];
    const InstDev& I = V.inst[V.cl_inst[k]];
    if (I.status != HSDE_RUNNING) return;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int c = V.cl_size[k];
    const int ld = (c + 15) / 16 * 16;
    T* W = reinterpret_cast<T*>(V.big_ws) + V.big_off[k];   // ld x ld
    T* QT = W + (size_t)ld * ld;                             // ld x ld

    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* d = reinterpret_cast<T*>(smem_raw);   // [ld] diagonal of the tridiagonal, then eigenvalues
    T* e = d + ld;                           // [ld] its off-diagonal
    T* hv = e + ld;                          // [ld] Householder vector of the current step
    T* pw = hv + ld;                         // [ld] p, then w; products QT_sub v
    T* beta = pw + ld;                       // [ld] beta_j of every reflection
    T* lam = beta + ld;                      // [ld] max(lambda, 0) (0 beyond c)
    T* ring = lam + ld;                      // [QR_SLOTS][2 ld] (cs, sn) of the QR steps in flight
    double* red = reinterpret_cast<double*>(ring + QR_SLOTS * 2 * ld);   // [BIG_WARPS + 2]
    T* redT = reinterpret_cast<T*>(red);                 // the same space, as T
    int* pos = reinterpret_cast<int*>(red + BIG_WARPS + 2);  // [ld] eigenvalues kept (FP64 rebuild)
    // the trailing blocks of the tridiagonalisation and of the accumulation
    // of Q move here once they fit (cap elements; the layout above is sized
    // for the bucket's largest clique, ldmax)
    T* Sb = reinterpret_cast<T*>(smem_raw + big_smem_base<T>(ldmax));
    __shared__ int s_lo[QR_SLOTS], s_hi[QR_SLOTS], s_steps, s_fail, s_npos;
    __shared__ uint64_t full_bar[QR_SLOTS], empty_bar[QR_SLOTS];

    T* s = reinterpret_cast<T*>(V.s);
    T* z = reinterpret_cast<T*>(V.z);
    T* v = reinterpret_cast<T*>(V.v);
    const int nlow = c * (c + 1) / 2;
    const int64_t off = V.cl_off[k];
    const double eta = I.eta;
    const double al = V.alpha;

    // ---- workspace: W = 0, QT = I (padding zero) ----
    for (int64_t idx = tid; idx < (int64_t)ld * ld; idx += BIG_NT) {
        const int i = (int)(idx / ld), j = (int)(idx - (int64_t)(idx / ld) * ld);
        W[idx] = T(0);
        QT[idx] = (i == j && i < c) ? T(1) : T(0);
    }
    __syncthreads();
    // ---- gather + rank-one correction: the point a to project, both triangles ----
    for (int en = tid; en < nlow; en += BIG_NT) {
        const int b = packed_column(en, c);
        const int arow = b + (en - (b * c - b * (b - 1) / 2));
        const int gi = V.gmap[off + en];
        const double gx = V.xw[gi] - eta * V.xp[gi];
        T av, vn, hx;
        cone_inputs<T>(s[off + en], z[off + en], v[off + en], (T)gx, (T)al, V.x, gi, av, vn, hx);
        W[(size_t)arow * ld + b] = av;
        W[(size_t)b * ld + arow] = av;
    }
    __syncthreads();

    // ---- 1. Householder tridiagonalisation ----
    // The active matrix is M(i, k) = Mb[(i - mo) ms + (k - mo)]: the
    // workspace W, then, from the first step whose block (rows and columns
    // j .. c-1) fits the shared-memory buffer, a copy of that block there.
    // The Householder vectors also go to their rows of W (the accumulation
    // reads them from there).
    T* Mb = W;
    int ms = ld, mo = 0;
    for (int j = 0; j + 2 < c; ++j) {
        const int L = c - j - 1;
        if (Mb == W && (L + 1) * (L + 1) <= cap) {
            const int n = L + 1;
            for (int idx = tid; idx < n * n; idx += BIG_NT) {
                const int r = idx / n, k2 = idx - (idx / n) * n;
                Sb[idx] = W[(size_t)(j + r) * ld + j + k2];
            }
            __syncthreads();
            Mb = Sb;
            ms = n;
            mo = j;
        }
        T* rowj = Mb + (size_t)(j - mo) * ms + (j + 1 - mo);   // x = A(j, j+1 ..)
        T ss = T(0);
        for (int i = tid; i < L; i += BIG_NT) {
            const T xi = rowj[i];
            hv[i] = xi;
            ss += xi * xi;
        }
        const T nx2 = block_sum<T>(ss, redT);
        if (nx2 == T(0)) {   // uniform: nothing to annihilate
            if (tid == 0) { beta[j] = T(0); e[j] = T(0); d[j] = Mb[(size_t)(j - mo) * ms + (j - mo)]; }
            __syncthreads();
            continue;
        }
        const T x0 = hv[0];
        const T nx = sqrt(nx2);
        const T alpha = x0 >= T(0) ? -nx : nx;           // H x = alpha e_1
        const T bj = T(1) / (nx * (nx + (x0 >= T(0) ? x0 : -x0)));   // 2 / v^T v
        __syncthreads();                                 // every thread has read hv[0]
        if (tid == 0) hv[0] = x0 - alpha;
        __syncthreads();
        // p = beta B v, B = A(j+1 .., j+1 ..)
        T* B0 = Mb + (size_t)(j + 1 - mo) * ms + (j + 1 - mo);
        rows_matvec<T>(B0, ms, L, hv, bj, pw);
        __syncthreads();
        T pv = T(0);
        for (int i = tid; i < L; i += BIG_NT) pv += pw[i] * hv[i];
        const T Kc = T(0.5) * bj * block_sum<T>(pv, redT);
        for (int i = tid; i < L; i += BIG_NT) pw[i] -= Kc * hv[i];   // w
        __syncthreads();
        // B <- B - v w^T - w v^T; row j keeps v
        rows_update<T>(B0, ms, L, hv, pw, pw, hv);
        T* wj = W + (size_t)j * ld + j + 1;
        for (int i = tid; i < L; i += BIG_NT) wj[i] = hv[i];
        if (tid == 0) { beta[j] = bj; e[j] = alpha; d[j] = Mb[(size_t)(j - mo) * ms + (j - mo)]; }
        __syncthreads();
    }
    if (tid == 0) {
        auto M = [&](int i, int k2) { return Mb[(size_t)(i - mo) * ms + (k2 - mo)]; };
        if (c >= 2) {
            d[c - 2] = M(c - 2, c - 2);
            e[c - 2] = M(c - 1, c - 2);
        }
        d[c - 1] = M(c - 1, c - 1);
    }
    __syncthreads();

    // ---- 2. QT <- QT H_j for j = c-3 .. 0 (rows and columns j+1 .. of QT) ----
    // The block grows from the bottom-right corner: rows and columns
    // qa .. c-1 (the largest block that fits, n = c - qa) are accumulated in
    // shared memory, then written to QT before the first larger step.
    int qn = 0;
    while ((qn + 1) * (qn + 1) <= cap && qn + 1 <= c) ++qn;
    const int qa = c - qn;
    for (int idx = tid; idx < qn * qn; idx += BIG_NT) {
        const int r = idx / qn, k2 = idx - (idx / qn) * qn;
        Sb[idx] = r == k2 ? T(1) : T(0);
    }
    bool flushed = qn == 0;
    __syncthreads();
    for (int j = c - 3; j >= 0; --j) {
        const T bj = beta[j];
        if (bj == T(0)) continue;   // uniform
        const int L = c - j - 1;
        T* Q0;
        int qs;
        if (j + 1 >= qa) {
            Q0 = Sb + (size_t)(j + 1 - qa) * qn + (j + 1 - qa);
            qs = qn;
        } else {
            if (!flushed) {
                for (int idx = tid; idx < qn * qn; idx += BIG_NT) {
                    const int r = idx / qn, k2 = idx - (idx / qn) * qn;
                    QT[(size_t)(qa + r) * ld + qa + k2] = Sb[idx];
                }
                flushed = true;
                __syncthreads();
            }
            Q0 = QT + (size_t)(j + 1) * ld + j + 1;
            qs = ld;
        }
        const T* vj = W + (size_t)j * ld + j + 1;
        for (int i = tid; i < L; i += BIG_NT) hv[i] = vj[i];
        __syncthreads();
        rows_matvec<T>(Q0, qs, L, hv, bj, pw);
        __syncthreads();
        rows_update<T>(Q0, qs, L, pw, hv, (const T*)nullptr, (const T*)nullptr);
        __syncthreads();
    }
    if (!flushed) {
        for (int idx = tid; idx < qn * qn; idx += BIG_NT) {
            const int r = idx / qn, k2 = idx - (idx / qn) * qn;
            QT[(size_t)(qa + r) * ld + qa + k2] = Sb[idx];
        }
    }
    __syncthreads();

    // ---- 3. implicit QR steps (Wilkinson shift) on (d, e) ----
    // Lane 0 of warp 0 chases the bulge of each step and writes its
    // rotations to a ring of QR_SLOTS slots; warps 1 .. apply them to the rows
    // of QT as they come (each thread owns whole columns of QT, so the
    // appliers never wait on each other).  full_bar[s]: the slot's step is
    // written (one arrival, the chaser); empty_bar[s]: every applier warp is
    // done with it.  Every wait is bounded; one that gives up marks the
    // clique unconverged and leaves the loop.
    if (tid == 0) {
        s_steps = 0;
        s_fail = 0;
        for (int q = 0; q < QR_SLOTS; ++q) {
            mbar_init(&full_bar[q], 1);
            mbar_init(&empty_bar[q], BIG_WARPS - 1);
        }
    }
    __syncthreads();
    if (warp == 0) {
        if (tid == 0) {
            const T eps = QrEps<T>::value;
            T tnorm = T(0);   // max_k |d_k| + |e_k| + |e_{k-1}| (the absolute floor of the deflation test)
            int hi = c - 1;
            bool finite = true;
            for (int q = 0; q < c; ++q) {
                const T a = (d[q] < T(0) ? -d[q] : d[q]) + (q + 1 < c ? (e[q] < T(0) ? -e[q] : e[q]) : T(0)) +
                            (q > 0 ? (e[q - 1] < T(0) ? -e[q - 1] : e[q - 1]) : T(0));
                finite = finite && isfinite(a);
                tnorm = a > tnorm ? a : tnorm;
            }
            if (!finite) {   // a non-finite input: no QR steps (the verdict reports it)
                hi = 0;
                s_fail = 1;
            }
            // scale (d, e) by a power of two to max_k |d_k| + |e_k| + |e_{k-1}|
            // in [1, 2) (exact; the eigenvectors do not change, the
            // eigenvalues are scaled back after the steps)
            T tsc = T(1);
            if (finite && tnorm > T(0)) {
                int ex;
                frexp(tnorm, &ex);
                tsc = ldexp(T(1), ex - 1);
                const T inv = T(1) / tsc;
                for (int q = 0; q < c; ++q) {
                    d[q] *= inv;
                    if (q + 1 < c) e[q] *= inv;
                }
                tnorm *= inv;
            }
            int steps = 0;
            const int max_steps = 30 * c;
            int lo_cur = -1;   // start of the unreduced block being reduced (-1: none yet)
            for (int t = 0;; ++t) {
                const int slot = t % QR_SLOTS, use = t / QR_SLOTS;
                if (use > 0 && !mbar_wait(&empty_bar[slot], (use - 1) & 1)) {
                    s_fail = 1;
                    break;
                }
                int lo = 0;
                bool step = false;
                while (hi > 0) {
                    const T ad = (d[hi - 1] < T(0) ? -d[hi - 1] : d[hi - 1]) + (d[hi] < T(0) ? -d[hi] : d[hi]);
                    const T ae = e[hi - 1] < T(0) ? -e[hi - 1] : e[hi - 1];
                    if (ae <= eps * ad || ae <= eps * tnorm) {
                        e[hi - 1] = T(0);
                        --hi;
                        continue;
                    }
                    step = true;
                    break;
                }
                if (step && steps >= max_steps) {
                    step = false;
                    s_fail = 1;
                }
                if (step) {
                    // the block's start: scanned when a new block begins; within
                    // a block only the chase changes e, and it reports the
                    // largest negligible e it leaves (split below)
                    if (lo_cur < 0 || lo_cur >= hi) {
                        lo = hi - 1;
                        while (lo > 0) {
                            const T ad = (d[lo - 1] < T(0) ? -d[lo - 1] : d[lo - 1]) + (d[lo] < T(0) ? -d[lo] : d[lo]);
                            const T ae = e[lo - 1] < T(0) ? -e[lo - 1] : e[lo - 1];
                            if (ae <= eps * ad || ae <= eps * tnorm) break;
                            --lo;
                        }
                        if (lo > 0) e[lo - 1] = T(0);
                        lo_cur = lo;
                    }
                    lo = lo_cur;
                    int split = lo;   // largest q in (lo, hi) whose final e[q-1] is negligible
                    T dprev = T(0);   // final d[q-1]
                    // Wilkinson shift: the eigenvalue of the trailing 2 x 2
                    // block closer to d[hi]
                    const T dl = (d[hi - 1] - d[hi]) * T(0.5);
                    const T eh = e[hi - 1];
                    const T hy = qr_hypot(dl, eh);
                    const T mu = d[hi] - eh * (eh / (dl + (dl >= T(0) ? hy : -hy)));
                    T x = d[lo] - mu, zb = e[lo];
                    T* rt = ring + (size_t)slot * 2 * ld;
                    // the rotated d[q], e[q] are carried in registers; d[q+1],
                    // e[q+1] are still the step's inputs and are loaded ahead
                    T dq = d[lo], eq = e[lo];
                    T dn = d[lo + 1], en = lo + 1 < hi ? e[lo + 1] : T(0);
                    for (int q = lo; q < hi; ++q) {
                        const T dn2 = q + 2 <= hi ? d[q + 2] : T(0);
                        const T en2 = q + 2 < hi ? e[q + 2] : T(0);
                        T cs, sn, r;
                        givens(x, zb, cs, sn, r);
                        if (q > lo) e[q - 1] = r;
                        // J^T [[a, b], [b, g]] J with a = dq, b = eq, g = dn:
                        // d'_q = a + s^2 (g - a) + 2 c s b, d'_{q+1} = a + g - d'_q,
                        // e'_q = c s (g - a) + (c^2 - s^2) b
                        const T ga = dn - dq, csn = cs * sn;
                        const T nd0 = dq + fma_t(sn * sn, ga, T(2) * csn * eq);
                        const T nd1 = (dq + dn) - nd0;
                        const T ne = fma_t(csn, ga, (cs - sn) * (cs + sn) * eq);
                        if (q > lo) {
                            const T ar = r < T(0) ? -r : r;
                            const T ad = (dprev < T(0) ? -dprev : dprev) + (nd0 < T(0) ? -nd0 : nd0);
                            if (ar <= eps * ad || ar <= eps * tnorm) split = q;
                        }
                        dprev = nd0;
                        d[q] = nd0;
                        e[q] = ne;
                        rt[2 * q] = cs;
                        rt[2 * q + 1] = sn;
                        x = ne;
                        zb = sn * en;      // the bulge at (q + 2, q)
                        eq = cs * en;      // e[q + 1] after the row rotation
                        dq = nd1;
                        dn = dn2;
                        en = en2;
                    }
                    d[hi] = dq;
                    if (split > lo) {
                        e[split - 1] = T(0);
                        lo_cur = split;
                    }
                    ++steps;
                }
                s_lo[slot] = lo;
                s_hi[slot] = step ? hi : -1;   // -1: no more steps
                mbar_arrive(&full_bar[slot]);  // release: the slot's writes are visible to the waiters
                if (!step) break;
            }
            s_steps = steps;
            for (int q = 0; q < c; ++q) d[q] *= tsc;
        }
        __syncwarp();
    } else {
        using T2 = typename std::conditional<sizeof(T) == 4, float2, double2>::type;
        constexpr int R = 16;   // rows of a column loaded together
        for (int t = 0;; ++t) {
            const int slot = t % QR_SLOTS, use = t / QR_SLOTS;
            if (!mbar_wait(&full_bar[slot], use & 1)) {
                s_fail = 1;
                break;
            }
            const int lo = s_lo[slot], h1 = s_hi[slot];
            if (h1 < 0) break;
            const T2* rt = reinterpret_cast<const T2*>(ring + (size_t)slot * 2 * ld);
            for (int i = tid - 32; i < c; i += BIG_NT - 32) {
                T* col = QT + i;
                T q = col[(size_t)lo * ld];
                // rows r0 + 1 .. r0 + R in nx; the next chunk's rows are
                // loaded before this chunk's rotations
                T nx[R];
#pragma unroll
                for (int u = 0; u < R; ++u) nx[u] = lo + 1 + u <= h1 ? col[(size_t)(lo + 1 + u) * ld] : T(0);
                for (int r0 = lo; r0 < h1; r0 += R) {
                    const int n = h1 - r0 < R ? h1 - r0 : R;
                    T nn[R];
#pragma unroll
                    for (int u = 0; u < R; ++u) nn[u] = r0 + R + 1 + u <= h1 ? col[(size_t)(r0 + R + 1 + u) * ld] : T(0);
#pragma unroll
                    for (int u = 0; u < R; ++u) {
                        if (u < n) {
                            const T2 g = rt[r0 + u];
                            col[(size_t)(r0 + u) * ld] = g.x * q + g.y * nx[u];
                            q = g.x * nx[u] - g.y * q;
                        }
                    }
#pragma unroll
                    for (int u = 0; u < R; ++u) nx[u] = nn[u];
                }
                col[(size_t)h1 * ld] = q;
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&empty_bar[slot]);
        }
    }
    __syncthreads();

    // ---- 4. rebuild s = Q max(Lambda, 0) Q^T (lower triangle into W) ----
    for (int q = tid; q < ld; q += BIG_NT) lam[q] = (q < c && d[q] > T(0)) ? d[q] : T(0);
    if (warp == 0) {
        int base = 0;
        for (int c0 = 0; c0 < c; c0 += 32) {
            const int q = c0 + lane;
            const bool pp = q < c && d[q] > T(0);
            const unsigned m = __ballot_sync(0xffffffffu, pp);
            if (pp) pos[base + __popc(m & ((1u << lane) - 1u))] = q;
            base += __popc(m);
        }
        if (lane == 0) s_npos = base;
    }
    __syncthreads();
    if constexpr (sizeof(T) == 4) {
        rebuild_tf32x3(reinterpret_cast<const float*>(QT), reinterpret_cast<const float*>(lam),
                       reinterpret_cast<float*>(W), c, ld);
    } else {
        rebuild_fp64(reinterpret_cast<const double*>(QT), reinterpret_cast<const double*>(lam), pos, s_npos,
                     reinterpret_cast<double*>(W), c, ld);
    }
    __syncthreads();

    // ---- 5. s, z, v and the stopping-rule partials ----
    T res = T(0), sres = T(0);
    for (int en = tid; en < nlow; en += BIG_NT) {
        const int b = packed_column(en, c);
        const int arow = b + (en - (b * c - b * (b - 1) / 2));
        const int64_t jj = off + en;
        const T sn = W[(size_t)arow * ld + b];
        const int gi = V.gmap[jj];
        const double gx = V.xw[gi] - eta * V.xp[gi];
        T av, vn, hx;
        cone_inputs<T>(s[jj], z[jj], v[jj], (T)gx, (T)al, V.x, gi, av, vn, hx);
        s[jj] = sn;
        z[jj] = sn - av;
        v[jj] = vn;
        const T dd = hx - sn;
        const T w = arow == b ? T(1) : T(2);
        res += w * dd * dd;
        sres += w * sn * sn;
    }
    const double rsum = block_sum<double>((double)res, red);
    const double ssum = block_sum<double>((double)sres, red);
    if (tid == 0) {
        V.cl_part[2 * k] = rsum;
        V.cl_part[2 * k + 1] = ssum;
        // QR steps per eigenvalue, rounded up (about 2 with the Wilkinson shift)
        V.cl_sweeps[k] = (s_steps + c - 1) / c;
        if (s_fail) atomicAdd(&V.inst[V.cl_inst[k]].unconv, 1);
    }
}

// Dynamic shared memory a CTA of the kernel may take in each precision (the
// opt-in maximum less the kernel's static shared memory; set up once).
int g_big_dyn[2] = {0, 0};



// ---------------------------------------------------------------------------
// Tridiagonal QR with one warp per clique, all in shared memory (FP32, the
// mixed form), for the throughput case: many cliques of 33 to 64.  The
// serial part of the method (each QR step's bulge chase, one lane) is
// hidden by the other cliques' warps on the same SM (about fourteen per
// SM), where the Jacobi sweeps move the whole matrix through shared memory
// every round.
//  - the clique matrix in a CP x (CP + 1) buffer (odd stride: a lane per
//    row or per column is conflict-free);
//  - Householder tridiagonalisation, a lane per row of the trailing block;
//  - Q^T formed in place of the reflectors (backward accumulation: before
//    the step of reflector j, rows and columns j+1 .. hold the product of
//    the later reflectors, bordered by a unit row and column);
//  - QR steps as in k_cone_big (lane 0 chases, then every lane applies the
//    step's rotations to its columns of Q^T);
//  - the rebuild s = Q max(Lambda, 0) Q^T fused with the scatter: each lane
//    forms its packed entries from the positive eigenpairs.
// ---------------------------------------------------------------------------
template <int CP>
constexpr size_t qrw_smem() {
    return (size_t)CP * sizeof(float2) + ((size_t)CP * (CP + 1) + 5 * CP) * sizeof(float);
}

template <int CP>
__global__ void __launch_bounds__(32, 16)
k_cone_qrw(DevView V, const int32_t* __restrict__ list, int nlist) {
    constexpr int LDA = CP + 1;
    const int li = blockIdx.x;
    if (li >= nlist) return;
    const int k = list[li];
    const InstDev& I = V.inst[V.cl_inst[k]];
    if (I.status != HSDE_RUNNING) return;
    const int lane = threadIdx.x;
    const int c = V.cl_size[k];
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2* rot = reinterpret_cast<float2*>(smem_raw);          // [CP] (cs, sn) of the current QR step
    float* A = reinterpret_cast<float*>(rot + CP);               // [CP x LDA]
    float* d = A + CP * LDA;                                     // [CP]
    float* e = d + CP;                                           // [CP]
    float* beta = e + CP;                                        // [CP]
    float* hv = beta + CP;                                       // [CP]
    float* pw = hv + CP;                                         // [CP]
    int* pos = reinterpret_cast<int*>(hv);                       // eigenvalues kept (after the QR steps)
    __shared__ int s_lo, s_hi, s_steps, s_fail, s_npos;

    float* s = reinterpret_cast<float*>(V.s);
    float* z = reinterpret_cast<float*>(V.z);
    float* v = reinterpret_cast<float*>(V.v);
    const int nlow = c * (c + 1) / 2;
    const int64_t off = V.cl_off[k];
    const double eta = I.eta;
    const double al = V.alpha;

    // ---- gather + rank-one correction, both triangles ----
    for (int en = lane; en < nlow; en += 32) {
        const int b = packed_column(en, c);
        const int arow = b + (en - (b * c - b * (b - 1) / 2));
        const int gi = V.gmap[off + en];
        const double gx = V.xw[gi] - eta * V.xp[gi];
        float av, vn, hx;
        cone_inputs<float>(s[off + en], z[off + en], v[off + en], (float)gx, (float)al, V.x, gi, av, vn, hx);
        A[arow * LDA + b] = av;
        A[b * LDA + arow] = av;
    }
    __syncwarp();

    // ---- Householder tridiagonalisation ----
    for (int j = 0; j + 2 < c; ++j) {
        const int L = c - j - 1;
        const float* rowj = A + j * LDA + j + 1;
        float ss = 0.f;
        for (int i = lane; i < L; i += 32) {
            const float xi = rowj[i];
            hv[i] = xi;
            ss = fmaf(xi, xi, ss);
        }
        const float nx2 = warp_sum(ss);
        __syncwarp();
        if (nx2 == 0.f) {
            if (lane == 0) { beta[j] = 0.f; e[j] = 0.f; d[j] = A[j * LDA + j]; }
            __syncwarp();
            continue;
        }
        const float x0 = hv[0];
        const float nx = sqrtf(nx2);
        const float alpha = x0 >= 0.f ? -nx : nx;
        const float bj = 1.f / (nx * (nx + fabsf(x0)));
        __syncwarp();
        if (lane == 0) hv[0] = x0 - alpha;
        __syncwarp();
        float* B0 = A + (j + 1) * LDA + j + 1;
        for (int r = lane; r < L; r += 32) {
            const float* br = B0 + r * LDA;
            float a = 0.f;
            for (int i = 0; i < L; ++i) a = fmaf(br[i], hv[i], a);
            pw[r] = bj * a;
        }
        __syncwarp();
        float pv = 0.f;
        for (int i = lane; i < L; i += 32) pv = fmaf(pw[i], hv[i], pv);
        const float Kc = 0.5f * bj * warp_sum(pv);
        for (int i = lane; i < L; i += 32) pw[i] = fmaf(-Kc, hv[i], pw[i]);
        __syncwarp();
        for (int r = lane; r < L; r += 32) {
            float* br = B0 + r * LDA;
            const float vr = hv[r], wr = pw[r];
            for (int i = 0; i < L; ++i) br[i] -= vr * pw[i] + wr * hv[i];
        }
        for (int i = lane; i < L; i += 32) A[j * LDA + j + 1 + i] = hv[i];
        if (lane == 0) { beta[j] = bj; e[j] = alpha; d[j] = A[j * LDA + j]; }
        __syncwarp();
    }
    if (lane == 0) {
        if (c >= 2) {
            d[c - 2] = A[(c - 2) * LDA + c - 2];
            e[c - 2] = A[(c - 1) * LDA + c - 2];
        }
        d[c - 1] = A[(c - 1) * LDA + c - 1];
    }
    __syncwarp();

    // ---- Q^T in place of the reflectors ----
    {
        const int t0 = c >= 2 ? c - 2 : 0, tn = c - t0;
        for (int idx = lane; idx < tn * tn; idx += 32) {
            const int r = idx / tn, q = idx - (idx / tn) * tn;
            A[(t0 + r) * LDA + t0 + q] = r == q ? 1.f : 0.f;
        }
        __syncwarp();
    }
    for (int j = c - 3; j >= 0; --j) {
        const int L = c - j - 1;
        float* Q0 = A + (j + 1) * LDA + j + 1;
        for (int i = lane; i < L; i += 32) hv[i] = A[j * LDA + j + 1 + i];
        __syncwarp();
        for (int i = lane; i < L; i += 32) {
            Q0[i] = i == 0 ? 1.f : 0.f;
            Q0[i * LDA] = i == 0 ? 1.f : 0.f;
        }
        __syncwarp();
        const float bj = beta[j];
        if (bj != 0.f) {
            for (int r = lane; r < L; r += 32) {
                const float* qr = Q0 + r * LDA;
                float a = 0.f;
                for (int i = 0; i < L; ++i) a = fmaf(qr[i], hv[i], a);
                pw[r] = bj * a;
            }
            __syncwarp();
            for (int r = lane; r < L; r += 32) {
                float* qr = Q0 + r * LDA;
                const float u = pw[r];
                for (int i = 0; i < L; ++i) qr[i] = fmaf(-u, hv[i], qr[i]);
            }
            __syncwarp();
        }
    }
    for (int i = lane; i < c; i += 32) {
        A[i] = i == 0 ? 1.f : 0.f;
        A[i * LDA] = i == 0 ? 1.f : 0.f;
    }
    if (lane == 0) { s_fail = 0; s_steps = 0; }
    __syncwarp();

    // ---- implicit QR steps (Wilkinson shift): lane 0 chases, all apply ----
    const float eps = QrEps<float>::value;
    float tnorm = 0.f, tsc = 1.f;
    int hi = c - 1, steps = 0, lo_cur = -1;
    const int max_steps = 30 * c;
    if (lane == 0) {
        bool finite = true;
        for (int q = 0; q < c; ++q) {
            const float a = fabsf(d[q]) + (q + 1 < c ? fabsf(e[q]) : 0.f) + (q > 0 ? fabsf(e[q - 1]) : 0.f);
            finite = finite && isfinite(a);
            tnorm = fmaxf(tnorm, a);
        }
        if (!finite) {
            hi = 0;
            s_fail = 1;
        } else if (tnorm > 0.f) {
            int ex;
            frexpf(tnorm, &ex);
            tsc = ldexpf(1.f, ex - 1);
            const float inv = 1.f / tsc;
            for (int q = 0; q < c; ++q) {
                d[q] *= inv;
                if (q + 1 < c) e[q] *= inv;
            }
            tnorm *= inv;
        }
    }
    for (;;) {
        if (lane == 0) {
            int lo = 0;
            bool step = false;
            while (hi > 0) {
                const float ae = fabsf(e[hi - 1]);
                if (ae <= eps * (fabsf(d[hi - 1]) + fabsf(d[hi])) || ae <= eps * tnorm) {
                    e[hi - 1] = 0.f;
                    --hi;
                    continue;
                }
                step = true;
                break;
            }
            if (step && steps >= max_steps) {
                step = false;
                s_fail = 1;
            }
            if (step) {
                if (lo_cur < 0 || lo_cur >= hi) {
                    lo = hi - 1;
                    while (lo > 0) {
                        const float ae = fabsf(e[lo - 1]);
                        if (ae <= eps * (fabsf(d[lo - 1]) + fabsf(d[lo])) || ae <= eps * tnorm) break;
                        --lo;
                    }
                    if (lo > 0) e[lo - 1] = 0.f;
                    lo_cur = lo;
                }
                lo = lo_cur;
                int split = lo;
                float dprev = 0.f;
                const float dl = (d[hi - 1] - d[hi]) * 0.5f;
                const float eh = e[hi - 1];
                const float hy = hypotf(dl, eh);
                const float mu = d[hi] - eh * (eh / (dl + (dl >= 0.f ? hy : -hy)));
                float x = d[lo] - mu, zb = e[lo];
                float dq = d[lo], eq = e[lo];
                float dn = d[lo + 1], en = lo + 1 < hi ? e[lo + 1] : 0.f;
                for (int q = lo; q < hi; ++q) {
                    const float dn2 = q + 2 <= hi ? d[q + 2] : 0.f;
                    const float en2 = q + 2 < hi ? e[q + 2] : 0.f;
                    float cs, sn, r;
                    givens(x, zb, cs, sn, r);
                    if (q > lo) e[q - 1] = r;
                    const float ga = dn - dq, csn = cs * sn;
                    const float nd0 = dq + fmaf(sn * sn, ga, 2.f * csn * eq);
                    const float nd1 = (dq + dn) - nd0;
                    const float ne = fmaf(csn, ga, (cs - sn) * (cs + sn) * eq);
                    if (q > lo && (fabsf(r) <= eps * (fabsf(dprev) + fabsf(nd0)) || fabsf(r) <= eps * tnorm))
                        split = q;
                    dprev = nd0;
                    d[q] = nd0;
                    e[q] = ne;
                    rot[q] = make_float2(cs, sn);
                    x = ne;
                    zb = sn * en;
                    eq = cs * en;
                    dq = nd1;
                    dn = dn2;
                    en = en2;
                }
                d[hi] = dq;
                if (split > lo) {
                    e[split - 1] = 0.f;
                    lo_cur = split;
                }
                ++steps;
            }
            s_lo = lo;
            s_hi = step ? hi : -1;
        }
        __syncwarp();
        const int lo = s_lo, h1 = s_hi;
        if (h1 < 0) break;
        for (int i = lane; i < c; i += 32) {
            float q = A[lo * LDA + i];
            for (int r = lo; r < h1; ++r) {
                const float nx = A[(r + 1) * LDA + i];
                const float2 g = rot[r];
                A[r * LDA + i] = fmaf(g.x, q, g.y * nx);
                q = fmaf(g.x, nx, -g.y * q);
            }
            A[h1 * LDA + i] = q;
        }
        __syncwarp();
    }
    if (lane == 0) {
        s_steps = steps;
        for (int q = 0; q < c; ++q) d[q] *= tsc;
    }
    __syncwarp();

    // ---- rebuild with the scatter, s, z, v and the stopping-rule partials ----
    {
        int base = 0;
        for (int c0 = 0; c0 < c; c0 += 32) {
            const int q = c0 + lane;
            const bool pp = q < c && d[q] > 0.f;
            const unsigned m = __ballot_sync(0xffffffffu, pp);
            if (pp) pos[base + __popc(m & ((1u << lane) - 1u))] = q;
            base += __popc(m);
        }
        if (lane == 0) s_npos = base;
    }
    __syncwarp();
    const int npos = s_npos;
    float res = 0.f, sres = 0.f;
    for (int en = lane; en < nlow; en += 32) {
        const int b = packed_column(en, c);
        const int arow = b + (en - (b * c - b * (b - 1) / 2));
        float sn = 0.f;
        for (int t = 0; t < npos; ++t) {
            const int q = pos[t];
            const float* qr = A + q * LDA;
            sn = fmaf(d[q] * qr[arow], qr[b], sn);
        }
        const int64_t jj = off + en;
        const int gi = V.gmap[jj];
        const double gx = V.xw[gi] - eta * V.xp[gi];
        float av, vn, hx;
        cone_inputs<float>(s[jj], z[jj], v[jj], (float)gx, (float)al, V.x, gi, av, vn, hx);
        s[jj] = sn;
        z[jj] = sn - av;
        v[jj] = vn;
        const float dd = hx - sn;
        const float w = arow == b ? 1.f : 2.f;
        res = fmaf(w * dd, dd, res);
        sres = fmaf(w * sn, sn, sres);
    }
    const double rsum = (double)warp_sum(res);
    const double ssum = (double)warp_sum(sres);
    if (lane == 0) {
        V.cl_part[2 * k] = rsum;
        V.cl_part[2 * k + 1] = ssum;
        V.cl_sweeps[k] = (s_steps + c - 1) / c;
        if (s_fail) atomicAdd(&V.inst[V.cl_inst[k]].unconv, 1);
    }
}

}  // namespace

int64_t cone_big_ws_elems(int c) {
    const int64_t ld = (c + 15) / 16 * 16;
    return 2 * ld * ld;
}

template <typename T>
static int prepare_big() {
    int dev = 0, optin = 0;
    cudaFuncAttributes fa{};
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess ||
        cudaFuncGetAttributes(&fa, k_cone_big<T>) != cudaSuccess)
        return HSDE_ECUDA;
    const int dyn = optin - (int)fa.sharedSizeBytes;
    if (dyn <= 0 || cudaFuncSetAttribute(k_cone_big<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn) != cudaSuccess)
        return HSDE_ECUDA;
    g_big_dyn[sizeof(T) == 4 ? 0 : 1] = dyn;
    return HSDE_OK;
}

int cone_big_prepare(bool mixed) { return mixed ? prepare_big<float>() : prepare_big<double>(); }

template <typename T>
static int launch_big(const DevView& V, const Bucket& bk, cudaStream_t st) {
    // every CTA takes the whole opt-in shared memory (one clique per SM):
    // the per-clique arrays for the bucket's largest clique, the rest for
    // the trailing blocks
    const int ldmax = (bk.csize_max + 15) / 16 * 16;
    const size_t base = big_smem_base<T>(ldmax);
    const int dyn = g_big_dyn[sizeof(T) == 4 ? 0 : 1];
    if (dyn <= 0 || base > (size_t)dyn) return HSDE_ECUDA;
    const int cap = (int)(((size_t)dyn - base) / sizeof(T));
    k_cone_big<T><<<bk.count, BIG_NT, (size_t)dyn, st>>>(V, bk.list, bk.count, ldmax, cap);
    return HSDE_OK;
}

int launch_cone_big(const DevView& V, const Bucket& bk, bool mixed, void* stp) {
    if (bk.count == 0) return HSDE_OK;
    if (V.big_ws == nullptr || V.big_off == nullptr) return HSDE_ECUDA;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stp);
    return mixed ? launch_big<float>(V, bk, st) : launch_big<double>(V, bk, st);
}

bool cone_qrw_has(int cp) { return cp == 36 || cp == 40 || cp == 44 || cp == 48 || cp == 56 || cp == 64; }

int launch_cone_qrw(const DevView& V, const Bucket& bk, void* stp) {
    if (bk.count == 0) return HSDE_OK;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stp);
    switch (bk.cmax) {
#define QRW(cp)                                                                                     \
    case cp:                                                                                        \
        k_cone_qrw<cp><<<bk.count, 32, qrw_smem<cp>(), st>>>(V, bk.list, bk.count);                \
        return HSDE_OK;
        QRW(36) QRW(40) QRW(44) QRW(48) QRW(56) QRW(64)
#undef QRW
        default:
            return HSDE_ERANGE;
    }
}

}  // namespace hsde
