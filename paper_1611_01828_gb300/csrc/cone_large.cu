// Cone projection of the cliques above the Jacobi bucket sizes (Eq. Step2 on
// S = S_1 x ... x S_p for the large cliques of Table 1, e.g. the 304-vertex
// clique of qpG51), fused with the gather, the rank-one correction of
// Eq. MatrixInverseResult and the nu update of Eq. Step3 exactly as the
// Jacobi kernel in cone.cu does (same per-entry arithmetic, cone_common.cuh).
//
// One CTA per clique; the c x c matrix and its eigenvectors live in a
// per-clique workspace in global memory (L2-resident: 2 ld^2 elements, ld = c
// rounded up to 16), the tridiagonal and the rotations in shared memory.
//
//  1. Householder tridiagonalisation (Golub & Van Loan, symmetric
//     Householder tridiagonalisation): for j = 0 .. c-3 the reflection
//     H_j = I - beta v v^T that zeroes row j beyond j+1 is applied to the
//     trailing block as B <- B - v w^T - w v^T with p = beta B v,
//     w = p - (beta p^T v / 2) v.  v is kept in row j of the workspace.
//  2. Q = H_0 H_1 ... H_{c-3}, accumulated backwards on Q^T (row k of QT is
//     eigenvector k): QT_sub <- QT_sub - beta (QT_sub v) v^T.
//  3. Implicit symmetric QR with the Wilkinson shift on the tridiagonal
//     (d, e), deflating from the bottom.  One lane chases the bulge of a
//     step and records its rotations; the other warps apply the previous
//     step's rotations to the rows of QT (each thread carries one column
//     through the chain, coalesced over the threads), so chase and
//     application overlap.  A step that would exceed 30 c steps in total
//     stops the solve; the clique is then counted as unconverged.
//  4. Rebuild s = Q max(Lambda, 0) Q^T on the lower triangle: in FP32 with
//     tensor cores as split-precision TF32 (each operand a = a_hi + a_lo,
//     both TF32; a_hi b_hi + a_hi b_lo + a_lo b_hi accumulated in FP32,
//     which keeps FP32 accuracy), in FP64 by FMA loops.
//  5. s, z, v and the clique's stopping-rule partials as in cone.cu.
//
// The workspace of a clique is private to its CTA; nothing waits on another
// CTA.
#include <cuda_runtime.h>

#include <cstdint>

#include "cone_common.cuh"
#include "internal.h"

namespace hsde {

namespace {

constexpr int BIG_NT = 512;
constexpr int BIG_WARPS = BIG_NT / 32;
constexpr int BIG_CHASERS = 32;   // warp 0 chases; the other warps apply rotations

template <typename T> struct QrEps;
template <> struct QrEps<float> { static constexpr float value = 1.1920929e-7f; };     // 2^-23
template <> struct QrEps<double> { static constexpr double value = 2.220446049250313e-16; };   // 2^-52

// Sum over the CTA, in an order fixed by the thread count: a shuffle tree in
// each warp, then the warp sums in warp order.  Every thread gets the result.
template <typename S>
__device__ __forceinline__ S block_sum(S v, S* red) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();   // red is free (an earlier block_sum has been read)
    if (lane == 0) red[warp] = v;
    __syncthreads();
    S t = S(0);
#pragma unroll
    for (int w = 0; w < BIG_WARPS; ++w) t += red[w];
    return t;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ float qr_hypot(float a, float b) { return hypotf(a, b); }
__device__ __forceinline__ double qr_hypot(double a, double b) { return hypot(a, b); }

// Rotation (cs, sn, r) with cs x + sn z = r = sqrt(x^2 + z^2), -sn x + cs z = 0.
// FP32: from the reciprocal square root of x^2 + z^2 when that sum is a
// normal number well inside the range (the chase's critical path), else by
// hypot; FP64 by hypot and division.
__device__ __forceinline__ void givens(float x, float z, float& cs, float& sn, float& r) {
    const float q = fmaf(x, x, z * z);
    if (q > 1e-30f && q < 1e30f) {
        const float iq = rsqrtf(q);
        cs = x * iq;
        sn = z * iq;
        r = q * iq;
    } else {
        r = hypotf(x, z);
        cs = 1.f;
        sn = 0.f;
        if (r != 0.f) {
            cs = x / r;
            sn = z / r;
        }
    }
}
__device__ __forceinline__ void givens(double x, double z, double& cs, double& sn, double& r) {
    r = hypot(x, z);
    cs = 1.0;
    sn = 0.0;
    if (r != 0.0) {
        cs = x / r;
        sn = z / r;
    }
}

// out[r] = scale * sum_i M[r][i] vec[i] for rows r < L of the block at M
// (row stride ld), columns i < L: a warp per group of four rows, so that a
// lane has the loads of four rows in flight.
template <typename T>
__device__ __forceinline__ void rows_matvec(const T* __restrict__ M, int ld, int L, const T* __restrict__ vec,
                                            T scale, T* __restrict__ out) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int r0 = 4 * warp; r0 < L; r0 += 4 * BIG_WARPS) {
        const int nr = L - r0 < 4 ? L - r0 : 4;
        const T* m0 = M + (size_t)r0 * ld;
        const T* m1 = m0 + (nr > 1 ? ld : 0);
        const T* m2 = m0 + (nr > 2 ? 2 * (size_t)ld : 0);
        const T* m3 = m0 + (nr > 3 ? 3 * (size_t)ld : 0);
        T a0 = T(0), a1 = T(0), a2 = T(0), a3 = T(0);
#pragma unroll 2
        for (int i = lane; i < L; i += 32) {
            const T x0 = m0[i], x1 = m1[i], x2 = m2[i], x3 = m3[i];
            const T vi = vec[i];
            a0 += x0 * vi;
            a1 += x1 * vi;
            a2 += x2 * vi;
            a3 += x3 * vi;
        }
        a0 = warp_sum(a0);
        a1 = warp_sum(a1);
        a2 = warp_sum(a2);
        a3 = warp_sum(a3);
        if (lane == 0) {
            out[r0] = scale * a0;
            if (nr > 1) out[r0 + 1] = scale * a1;
            if (nr > 2) out[r0 + 2] = scale * a2;
            if (nr > 3) out[r0 + 3] = scale * a3;
        }
    }
}

// M[r][i] -= u[r] v[i] + (w ? w[r] x[i] : 0) for r, i < L: four rows of a
// warp at a time, loads first.
template <typename T>
__device__ __forceinline__ void rows_update(T* __restrict__ M, int ld, int L, const T* __restrict__ u,
                                            const T* __restrict__ vv, const T* __restrict__ w,
                                            const T* __restrict__ xv) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int r0 = 4 * warp; r0 < L; r0 += 4 * BIG_WARPS) {
        const int nr = L - r0 < 4 ? L - r0 : 4;
        T* mr[4];
        T ur[4], wr[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int r = r0 + (q < nr ? q : 0);
            mr[q] = M + (size_t)r * ld;
            ur[q] = u[r];
            wr[q] = w ? w[r] : T(0);
        }
        for (int i = lane; i < L; i += 32) {
            T x[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) x[q] = mr[q][i];
            const T vi = vv[i], xi = w ? xv[i] : T(0);
#pragma unroll
            for (int q = 0; q < 4; ++q)
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

template <typename T>
__global__ void __launch_bounds__(BIG_NT, 1)
k_cone_big(DevView V, const int32_t* __restrict__ list, int nlist) {
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
    T* rc = beta + ld;                       // [2 ld] rotation cosines (two steps in flight)
    T* rs = rc + 2 * ld;                     // [2 ld] rotation sines
    T* lam = rs + 2 * ld;                    // [ld] max(lambda, 0) (0 beyond c)
    double* red = reinterpret_cast<double*>(lam + ld);   // [BIG_WARPS] (8-byte aligned: 9 ld T's)
    int* pos = reinterpret_cast<int*>(red + BIG_WARPS);  // [ld] eigenvalues kept (FP64 rebuild)
    __shared__ int s_lo[2], s_hi[2], s_more, s_steps, s_fail, s_npos;

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
    for (int j = 0; j + 2 < c; ++j) {
        const int L = c - j - 1;
        T* rowj = W + (size_t)j * ld + j + 1;   // x = A(j, j+1 ..)
        T ss = T(0);
        for (int i = tid; i < L; i += BIG_NT) {
            const T xi = rowj[i];
            hv[i] = xi;
            ss += xi * xi;
        }
        const double nx2 = block_sum<double>((double)ss, red);
        if (nx2 == 0.0) {   // uniform: nothing to annihilate
            if (tid == 0) { beta[j] = T(0); e[j] = T(0); d[j] = W[(size_t)j * ld + j]; }
            __syncthreads();
            continue;
        }
        const T x0 = hv[0];
        const T nx = (T)sqrt(nx2);
        const T alpha = x0 >= T(0) ? -nx : nx;           // H x = alpha e_1
        const T bj = T(1) / (nx * (nx + (x0 >= T(0) ? x0 : -x0)));   // 2 / v^T v
        __syncthreads();                                 // every thread has read hv[0]
        if (tid == 0) hv[0] = x0 - alpha;
        __syncthreads();
        // p = beta B v, B = A(j+1 .., j+1 ..)
        T* B0 = W + (size_t)(j + 1) * ld + j + 1;
        rows_matvec<T>(B0, ld, L, hv, bj, pw);
        __syncthreads();
        T pv = T(0);
        for (int i = tid; i < L; i += BIG_NT) pv += pw[i] * hv[i];
        const T Kc = T(0.5) * bj * (T)block_sum<double>((double)pv, red);
        for (int i = tid; i < L; i += BIG_NT) pw[i] -= Kc * hv[i];   // w
        __syncthreads();
        // B <- B - v w^T - w v^T; row j keeps v
        rows_update<T>(B0, ld, L, hv, pw, pw, hv);
        for (int i = tid; i < L; i += BIG_NT) rowj[i] = hv[i];
        if (tid == 0) { beta[j] = bj; e[j] = alpha; d[j] = W[(size_t)j * ld + j]; }
        __syncthreads();
    }
    if (tid == 0) {
        if (c >= 2) {
            d[c - 2] = W[(size_t)(c - 2) * ld + c - 2];
            e[c - 2] = W[(size_t)(c - 1) * ld + c - 2];
        }
        d[c - 1] = W[(size_t)(c - 1) * ld + c - 1];
    }
    __syncthreads();

    // ---- 2. QT <- QT H_j for j = c-3 .. 0 (rows and columns j+1 .. of QT) ----
    for (int j = c - 3; j >= 0; --j) {
        const T bj = beta[j];
        if (bj == T(0)) continue;   // uniform
        const int L = c - j - 1;
        const T* vj = W + (size_t)j * ld + j + 1;
        for (int i = tid; i < L; i += BIG_NT) hv[i] = vj[i];
        __syncthreads();
        T* Q0 = QT + (size_t)(j + 1) * ld + j + 1;
        rows_matvec<T>(Q0, ld, L, hv, bj, pw);
        __syncthreads();
        rows_update<T>(Q0, ld, L, pw, hv, (const T*)nullptr, (const T*)nullptr);
        __syncthreads();
    }

    // ---- 3. implicit QR steps (Wilkinson shift) on (d, e) ----
    // Phase p: lane 0 of warp 0 chases step p into buffer p & 1 while warps
    // 1 .. apply step p - 1 from the other buffer to the rows of QT.
    if (tid == 0) {
        s_more = 1;
        s_steps = 0;
        s_fail = 0;
        s_lo[0] = s_lo[1] = 0;
        s_hi[0] = s_hi[1] = -1;   // nothing to apply
    }
    __syncthreads();
    const T eps = QrEps<T>::value;
    T tnorm = T(0);   // max_k |d_k| + |e_k| + |e_{k-1}| (the absolute floor of the deflation test)
    int hi = c - 1;        // chaser state (tid 0)
    if (tid == 0) {
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
    }
    int steps = 0;
    const int max_steps = 30 * c;
    for (int p = 0;; ++p) {
        const int buf = p & 1;
        if (warp == 0) {
            if (tid == 0) {
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
                    lo = hi - 1;
                    while (lo > 0) {
                        const T ad = (d[lo - 1] < T(0) ? -d[lo - 1] : d[lo - 1]) + (d[lo] < T(0) ? -d[lo] : d[lo]);
                        const T ae = e[lo - 1] < T(0) ? -e[lo - 1] : e[lo - 1];
                        if (ae <= eps * ad || ae <= eps * tnorm) break;
                        --lo;
                    }
                    if (lo > 0) e[lo - 1] = T(0);
                    // Wilkinson shift: the eigenvalue of the trailing 2 x 2
                    // block closer to d[hi]
                    const T dl = (d[hi - 1] - d[hi]) * T(0.5);
                    const T eh = e[hi - 1];
                    const T hy = qr_hypot(dl, eh);
                    const T mu = d[hi] - eh * (eh / (dl + (dl >= T(0) ? hy : -hy)));
                    T x = d[lo] - mu, zb = e[lo];
                    T* cb = rc + buf * ld;
                    T* sb = rs + buf * ld;
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
                        const T c2 = cs * cs, s2 = sn * sn, csb = T(2) * cs * sn * eq;
                        const T nd0 = c2 * dq + csb + s2 * dn;
                        const T nd1 = s2 * dq - csb + c2 * dn;
                        const T ne = cs * sn * (dn - dq) + (c2 - s2) * eq;
                        d[q] = nd0;
                        e[q] = ne;
                        cb[q] = cs;
                        sb[q] = sn;
                        x = ne;
                        zb = sn * en;      // the bulge at (q + 2, q)
                        eq = cs * en;      // e[q + 1] after the row rotation
                        dq = nd1;
                        dn = dn2;
                        en = en2;
                    }
                    d[hi] = dq;
                    ++steps;
                }
                s_lo[buf] = lo;
                s_hi[buf] = step ? hi : -1;
                s_more = step ? 1 : 0;
            }
        } else {
            // apply step p - 1 (buffer buf ^ 1) to rows lo .. hi of QT
            const int ob = buf ^ 1;
            const int lo = s_lo[ob], h1 = s_hi[ob];
            if (p > 0 && h1 >= 0) {
                const T* cb = rc + ob * ld;
                const T* sb = rs + ob * ld;
                constexpr int R = 16;   // rows of a column loaded together
                for (int i = tid - 32; i < c; i += BIG_NT - 32) {
                    T* col = QT + i;
                    T q = col[(size_t)lo * ld];
                    for (int r0 = lo; r0 < h1; r0 += R) {
                        const int n = h1 - r0 < R ? h1 - r0 : R;
                        T nx[R];
#pragma unroll
                        for (int u = 0; u < R; ++u) nx[u] = u < n ? col[(size_t)(r0 + 1 + u) * ld] : T(0);
#pragma unroll
                        for (int u = 0; u < R; ++u) {
                            if (u < n) {
                                const T cs = cb[r0 + u], sn = sb[r0 + u];
                                col[(size_t)(r0 + u) * ld] = cs * q + sn * nx[u];
                                q = cs * nx[u] - sn * q;
                            }
                        }
                    }
                    col[(size_t)h1 * ld] = q;
                }
            }
        }
        __syncthreads();
        if (!s_more) {
            // the step of this phase was empty; the previous one has been applied
            break;
        }
        __syncthreads();   // s_more read by all before the chaser writes it again
    }
    if (tid == 0) s_steps = steps;

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

template <typename T>
size_t big_smem(int cmax) {
    const int ld = (cmax + 15) / 16 * 16;
    return (size_t)9 * ld * sizeof(T) + BIG_WARPS * sizeof(double) + (size_t)ld * sizeof(int);
}

}  // namespace

int64_t cone_big_ws_elems(int c) {
    const int64_t ld = (c + 15) / 16 * 16;
    return 2 * ld * ld;
}

int cone_big_prepare(bool mixed) {
    const size_t sm = mixed ? big_smem<float>(CONE_BIG) : big_smem<double>(CONE_BIG);
    const cudaError_t e = mixed ? cudaFuncSetAttribute(k_cone_big<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                       (int)sm)
                                : cudaFuncSetAttribute(k_cone_big<double>,
                                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    return e == cudaSuccess ? HSDE_OK : HSDE_ECUDA;
}

int launch_cone_big(const DevView& V, const Bucket& bk, bool mixed, void* stp) {
    if (bk.count == 0) return HSDE_OK;
    if (V.big_ws == nullptr || V.big_off == nullptr) return HSDE_ECUDA;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stp);
    // shared memory sized for the largest clique the path takes
    if (mixed) k_cone_big<float><<<bk.count, BIG_NT, big_smem<float>(CONE_BIG), st>>>(V, bk.list, bk.count);
    else k_cone_big<double><<<bk.count, BIG_NT, big_smem<double>(CONE_BIG), st>>>(V, bk.list, bk.count);
    return HSDE_OK;
}

}  // namespace hsde
