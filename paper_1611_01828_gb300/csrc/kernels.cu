// Per-iteration kernels of the block-eliminated affine projection (Eq. Step1
// via Sections 4.2-4.3), the scalar tau/kappa updates of Eqs. Step2-Step3,
// the stopping-rule reductions, and the one-time setup kernels.
//
// Fused form of the affine step used here (algebraically equal to the
// paper's chain of eliminations; the oracle follows the printed order):
//   omega_tau = tau + kappa
//   g0 = x - omega_tau c + 1/2 H^T (s + z + v)          (N space)
//   f  = Delta^{-1} g0,  Delta = I + D/2
//   q  = y + omega_tau b - A f                           (m space)
//   y_w = S^{-1} q,      S = I + A Delta^{-1} A^T        (cached inverse)
//   x_w = f + Delta^{-1} A^T y_w
//   eta = (c^T x_w - b^T y_w) / (1 + zeta^T M^{-1} zeta) (Eq. MatrixInverseResult)
//   x_hat = x_w - eta x_p,  y_hat = y_w - eta y_p,
//   tau_hat = omega_tau + c^T x_hat - b^T y_hat          (Eq. FirstBlockElimination)
// then the cone step on the relaxed point u_rel = alpha u_hat + (1 - alpha) u
// (alpha = 1: the literal Eqs. Step2-Step3):
//   x = x_rel,  y = y_rel,
//   tau = max(0, tau_rel - kappa), kappa += tau - tau_rel
// The clique part (s_hat, v_hat, the PSD projection and z) is in cone.cu.
// All of it runs on the scaled data (A~ = D A, b~ = sigma D b, c~ = rho c,
// or the data as given); the stopping rule unscales (readings P5-P7).
//
// Every reduction is a fixed-order tree (no float atomics): results are
// bitwise reproducible for a given launch configuration.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include "internal.h"

namespace hsde {

static constexpr int NT = 256;   // threads per CTA for N-space tiles and m rows
static_assert(TILE_N == NT, "one pattern entry per thread in the N-space kernels");

template <typename S>
__device__ __forceinline__ S warp_sum(S v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Sum over the CTA (blockDim.x == NT); result valid in every thread.
__device__ __forceinline__ double block_sum(double v, double* sh) {
    v = warp_sum(v);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) sh[w] = v;
    __syncthreads();
    double t = (threadIdx.x < NT / 32) ? sh[threadIdx.x] : 0.0;
    if (w == 0) t = warp_sum(t);
    if (threadIdx.x == 0) sh[0] = t;
    __syncthreads();
    const double r = sh[0];
    __syncthreads();
    return r;
}

// NV block sums at once (one set of barriers); each value is summed in the
// same order as block_sum.  sh holds NV * NT / 32 doubles.
template <int NV>
__device__ __forceinline__ void block_sum_n(double (&v)[NV], double* sh) {
    constexpr int W = NT / 32;
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
#pragma unroll
    for (int i = 0; i < NV; ++i) v[i] = warp_sum(v[i]);
    __syncthreads();
    if (l == 0) {
#pragma unroll
        for (int i = 0; i < NV; ++i) sh[i * W + w] = v[i];
    }
    __syncthreads();
    if (w == 0) {
#pragma unroll
        for (int i = 0; i < NV; ++i) {
            double t = (l < W) ? sh[i * W + l] : 0.0;
            t = warp_sum(t);
            if (l == 0) sh[i * W] = t;
        }
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < NV; ++i) v[i] = sh[i * W];
    __syncthreads();
}

__device__ __forceinline__ bool is_check_iter(const DevView& V, int iter) {
    return (iter % V.check_every) == 0 || iter >= V.max_iter;
}

template <typename T>
__device__ __forceinline__ double ld(const void* p, int64_t i) {
    return (double)reinterpret_cast<const T*>(p)[i];
}

// s + z + v of one packed copy, added in the precision of the clique arrays
// (in FP32 for the mixed form: one conversion instead of three, and no FP64
// additions, which run at a small fraction of the FP32 rate on this GPU).
// k_post, k_rhs and k_long all use it, so they agree bit for bit.
template <typename T>
__device__ __forceinline__ double copy_szv(const DevView& V, int64_t p) {
    const T* s = reinterpret_cast<const T*>(V.s);
    const T* z = reinterpret_cast<const T*>(V.z);
    const T* v = reinterpret_cast<const T*>(V.v);
    return (double)(s[p] + z[p] + v[p]);
}

// NV block sums (blockDim.x == NT) through shared memory: every value is
// summed by one warp in a fixed order (strided lanes, then a butterfly), so
// each double is added about 12 times per warp instead of 5 times by every
// thread.  buf holds NV * NT doubles; the result is valid in every thread.
template <int NV, typename S>
__device__ __forceinline__ void block_sum_t(S (&v)[NV], S* buf) {
    __syncthreads();
#pragma unroll
    for (int i = 0; i < NV; ++i) buf[i * NT + threadIdx.x] = v[i];
    __syncthreads();
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    for (int i = w; i < NV; i += NT / 32) {
        S s = S(0);
#pragma unroll
        for (int k = 0; k < NT / 32; ++k) s += buf[i * NT + l + 32 * k];
        s = warp_sum(s);
        if (l == 0) buf[i * NT] = s;
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < NV; ++i) v[i] = buf[i * NT];
    __syncthreads();
}

// ---------------------------------------------------------------------------
// g0, f = Delta^{-1} g0 ; Setup mode: f = Delta^{-1} c
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(NT) k_rhs(DevView V, int mode) {
    const int4 t = V.tiles[blockIdx.x];
    const InstDev& I = V.inst[t.x];
    if (mode == (int)Mode::Setup) {
        for (int e = t.y + threadIdx.x; e < t.z; e += NT) V.f[e] = V.c[e] * V.inv_delta[e];
        return;
    }
    if (I.status != HSDE_RUNNING) return;
    const double ot = I.tau + I.kappa;
    for (int e = t.y + threadIdx.x; e < t.z; e += NT) {
        double acc = 0.0;
        const int li = V.long_id[e];
        if (li >= 0) {
            acc = V.lall[li];                       // k_long, launched just before
        } else {
            const int j1 = V.ssc_ptr[e + 1];
            for (int j = V.ssc_ptr[e]; j < j1; ++j) acc += copy_szv<T>(V, V.ssc_idx[j]);
        }
        V.f[e] = (V.x[e] - ot * V.c[e] + 0.5 * acc) * V.inv_delta[e];
    }
}

// H^T z and H^T (s + z + v) of each long entry: one CTA per entry, the
// copies strided over the threads and summed in a fixed tree (the same
// values as a sequential sum up to rounding, and the same bits every run).
template <typename T>
__global__ void __launch_bounds__(NT) k_long(DevView V) {
    __shared__ double sh[2 * NT / 32];
    const int l = blockIdx.x;
    if (V.inst[V.long_inst[l]].status != HSDE_RUNNING) return;
    const int e = V.long_e[l];
    double v2[2] = {0.0, 0.0};
    const int k1 = V.sc_ptr[e + 1];
    for (int k = V.sc_ptr[e] + threadIdx.x; k < k1; k += NT) {
        const int p = V.sc_idx[k];
        v2[0] += ld<T>(V.z, p);
        v2[1] += copy_szv<T>(V, p);
    }
    block_sum_n<2>(v2, sh);
    if (threadIdx.x == 0) {
        V.lhz[l] = v2[0];
        V.lall[l] = v2[1];
    }
}

// q = y + omega_tau b - A f  (Setup: q = -b - A f).  One warp per row.
__global__ void __launch_bounds__(NT) k_spmv_A(DevView V, int mode) {
    const int row = (blockIdx.x * NT + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (row >= V.Mtot) return;
    const InstDev& I = V.inst[V.row_inst[row]];
    if (mode == (int)Mode::Iter && I.status != HSDE_RUNNING) return;
    double acc = 0.0;
    const int j1 = V.A_ptr[row + 1];
    for (int j = V.A_ptr[row] + lane; j < j1; j += 32) acc += V.A_val[j] * V.f[V.A_col[j]];
    acc = warp_sum(acc);
    if (lane == 0) {
        const double base = (mode == (int)Mode::Iter) ? V.y[row] + (I.tau + I.kappa) * V.b[row]
                                                      : -V.b[row];
        V.q[row] = base - acc;
    }
}

// y_w = S^{-1} q (dense row dot products or a diagonal scale).  One warp per row.
__global__ void __launch_bounds__(NT) k_solve(DevView V, int mode) {
    const int row = (blockIdx.x * NT + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (row >= V.Mtot) return;
    const InstDev& I = V.inst[V.row_inst[row]];
    if (mode == (int)Mode::Iter && I.status != HSDE_RUNNING) return;
    double* out = (mode == (int)Mode::Iter) ? V.yw : V.yp;
    if (!I.dense) {
        if (lane == 0) out[row] = V.sdiag[row] * V.q[row];
        return;
    }
    if (I.dense != 1) return;      // structured S: launch_lr_solve
    const int i = row - I.m_off;
    const double* Srow = V.sinv + I.sinv_off + (int64_t)i * I.m;
    const double* qq = V.q + I.m_off;
    double acc = 0.0;
    for (int j = lane; j < I.m; j += 32) acc += Srow[j] * qq[j];
    acc = warp_sum(acc);
    if (lane == 0) out[row] = acc;
}

// x_w = f + Delta^{-1} A^T y_w (Setup: x_p = f + Delta^{-1} A^T y_p),
// and the tile partial of c^T x_w (off-diagonal entries weighted 2).
__global__ void __launch_bounds__(NT) k_spmv_At(DevView V, int mode) {
    __shared__ double sh[32];
    const int4 t = V.tiles[blockIdx.x];
    const InstDev& I = V.inst[t.x];
    if (mode == (int)Mode::Iter && I.status != HSDE_RUNNING) return;
    const double* yin = (mode == (int)Mode::Iter) ? V.yw : V.yp;
    double* out = (mode == (int)Mode::Iter) ? V.xw : V.xp;
    double part = 0.0;
    for (int e = t.y + threadIdx.x; e < t.z; e += NT) {
        double acc = 0.0;
        const int j1 = V.At_ptr[e + 1];
        for (int j = V.At_ptr[e]; j < j1; ++j) acc += V.At_val[j] * yin[V.At_col[j]];
        const double xv = V.f[e] + V.inv_delta[e] * acc;
        out[e] = xv;
        if (mode == (int)Mode::Setup) V.atyp[e] = acc;     // A^T y_p, cached
        part += (V.diag[e] ? 1.0 : 2.0) * V.c[e] * xv;
    }
    part = block_sum(part, sh);
    if (threadIdx.x == 0) V.part[(int64_t)blockIdx.x * KPART + 0] = part;
}


// ===========================================================================
// Fused iteration kernels.  Per iteration (after the cone projections of the
// previous one have produced s, z, v and k_post has produced f):
//   k_fwd          q = y + omega_tau b - A f; diagonal S: y_w = S^{-1} q
//   k_solve_dense  dense S: y_w = S^{-1} q                 (only if any S is dense)
//   k_bwd_eta      x_w = f + Delta^{-1} A^T y_w over nonzero-balanced A^T
//                  tiles; the last CTA of each instance computes eta, tau
//                  and kappa
//   k_cone ...     per clique bucket, in parallel
//   k_post         x = x_w - eta x_p and y = y_w - eta y_p (a slice of the
//                  constraints per CTA); all stopping-rule sums; the last CTA
//                  of each instance takes the verdict; f of the next iteration
// "Last CTA" is the usual completion-counter pattern: every CTA publishes its
// partial sums, fences, and increments a per-instance counter; the CTA that
// sees the final count reduces the partials in tile order.  Nothing waits.
// ===========================================================================

__device__ __forceinline__ bool last_cta(int* counter, int total, int* flag_sh) {
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        const int prev = atomicAdd(counter, 1);
        *flag_sh = (prev == total - 1);
    }
    __syncthreads();
    const bool last = *flag_sh != 0;
    if (last) __threadfence();
    return last;
}

// q and, for diagonal S, y_w and b_i y_w,i.  One warp per row.
__global__ void __launch_bounds__(NT) k_fwd(DevView V) {
    const int row = (blockIdx.x * NT + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (row >= V.Mtot) return;
    const InstDev& I = V.inst[V.row_inst[row]];
    if (I.status != HSDE_RUNNING) return;
    double acc = 0.0;
    const int j1 = V.A_ptr[row + 1];
    for (int j = V.A_ptr[row] + lane; j < j1; j += 32) acc += V.A_val[j] * V.f[V.A_col[j]];
    acc = warp_sum(acc);
    if (lane == 0) {
        V.af[row] = acc;
        const double q = V.y[row] + (I.tau + I.kappa) * V.b[row] - acc;
        if (I.dense) {
            V.q[row] = q;
        } else {
            const double yw = V.sdiag[row] * q;
            V.yw[row] = yw;
            V.rowb[row] = V.b[row] * yw;
        }
    }
}

// dense S: y_w = S^{-1} q and b_i y_w,i.  One warp per row.
__global__ void __launch_bounds__(NT) k_solve_dense(DevView V) {
    const int row = (blockIdx.x * NT + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (row >= V.Mtot) return;
    const InstDev& I = V.inst[V.row_inst[row]];
    if (I.status != HSDE_RUNNING || I.dense != 1) return;
    const int i = row - I.m_off;
    const double* Srow = V.sinv + I.sinv_off + (int64_t)i * I.m;
    const double* qq = V.q + I.m_off;
    double acc = 0.0;
    for (int j = lane; j < I.m; j += 32) acc += Srow[j] * qq[j];
    acc = warp_sum(acc);
    if (lane == 0) {
        V.yw[row] = acc;
        V.rowb[row] = V.b[row] * acc;
    }
}

// x_w = f + Delta^{-1} A^T y_w; last CTA per instance: eta, tau, kappa, y.
__global__ void __launch_bounds__(NT) k_bwd_eta(DevView V) {
    __shared__ double sh[32];
    __shared__ int flag;
    const int4 t = V.at_tiles[blockIdx.x];   // (inst, first entry, end, lanes per row)
    InstDev& I = V.inst[t.x];
    if (I.status != HSDE_RUNNING) return;
    double part = 0.0;
    const int G = t.w;
    if (G >= NT) {
        // one long row of A^T: the whole CTA, coalesced strides
        const int e = t.y;
        double acc = 0.0;
        const int j1 = V.At_ptr[e + 1];
        for (int j = V.At_ptr[e] + threadIdx.x; j < j1; j += NT) acc += V.At_val[j] * V.yw[V.At_col[j]];
        acc = block_sum(acc, sh);
        if (threadIdx.x == 0) {
            const double xv = V.f[e] + V.inv_delta[e] * acc;
            V.xw[e] = xv;
            V.atyw[e] = acc;
            part = (V.diag[e] ? 1.0 : 2.0) * V.c[e] * xv;
        }
    } else {
        // Groups of G lanes (a power of two <= 32, aligned in the warp) take
        // one row at a time: each lane accumulates its strided share of the
        // row with FMAs (four independent loads and gathers in flight), then
        // the group combines by a butterfly and its first lane finishes the
        // row.  One FP64 operation per nonzero plus G log2 G per row: on this
        // GPU the FP64 pipe, not DRAM, sets the time of this kernel, so the
        // tiles give each lane about a dozen nonzeros of a row (the butterfly
        // of a 32-lane group per row cost more than the products).  The loop
        // bound is uniform over the CTA, so every lane reaches each shuffle.
        const int nrow = t.z - t.y;      // <= TILE_N == NT
        const int grp = threadIdx.x / G, lane = threadIdx.x & (G - 1), ngrp = NT / G;
        for (int base = 0; base < nrow; base += ngrp) {
            const int r = base + grp;
            const bool valid = r < nrow;
            const int e = t.y + r;
            double acc = 0.0;
            if (valid) {
                const int j0 = V.At_ptr[e], j1 = V.At_ptr[e + 1];
                int j = j0 + lane;
                double a0 = 0.0, a1 = 0.0;
                for (; j + 3 * G < j1; j += 4 * G) {
                    const int c0 = V.At_col[j], c1 = V.At_col[j + G], c2 = V.At_col[j + 2 * G],
                              c3 = V.At_col[j + 3 * G];
                    const double v0 = V.At_val[j], v1 = V.At_val[j + G], v2 = V.At_val[j + 2 * G],
                                 v3 = V.At_val[j + 3 * G];
                    const double y0 = V.yw[c0], y1 = V.yw[c1], y2 = V.yw[c2], y3 = V.yw[c3];
                    a0 = fma(v0, y0, a0);
                    a1 = fma(v1, y1, a1);
                    a0 = fma(v2, y2, a0);
                    a1 = fma(v3, y3, a1);
                }
                for (; j < j1; j += G) a0 = fma(V.At_val[j], V.yw[V.At_col[j]], a0);
                acc = a0 + a1;
            }
            for (int o = G >> 1; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
            if (valid && lane == 0) {
                const double xv = V.f[e] + V.inv_delta[e] * acc;
                V.xw[e] = xv;
                V.atyw[e] = acc;
                part += (V.diag[e] ? 1.0 : 2.0) * V.c[e] * xv;
            }
        }
    }
    part = block_sum(part, sh);
    if (threadIdx.x == 0) V.at_part[blockIdx.x] = part;
    if (!last_cta(V.counters + 2 * t.x, I.at_end - I.at_begin, &flag)) return;
    // ---- last CTA of this instance ----
    double cb[2] = {0.0, 0.0};   // c^T x_w, b^T y_w
    for (int tt = I.at_begin + threadIdx.x; tt < I.at_end; tt += NT) cb[0] += __ldcg(V.at_part + tt);
    for (int i = threadIdx.x; i < I.m; i += NT) cb[1] += __ldcg(V.rowb + I.m_off + i);
    block_sum_n<2>(cb, sh);
    const double sw = cb[0] - cb[1];
    const double eta = sw / I.den;
    const double tau = I.tau, kappa = I.kappa;
    const double ot = tau + kappa;
    const double tau_hat = ot + sw - eta * I.ctp;
    const double al = V.alpha;
    const double tau_rel = (al == 1.0) ? tau_hat : al * tau_hat + (1.0 - al) * tau;
    const double tau_new = fmax(0.0, tau_rel - kappa);
    const double kappa_new = kappa - tau_rel + tau_new;
    // y = y_w - eta y_p and the constraint-space sums of the stopping rule
    // follow in k_post, spread over all of its CTAs.
    if (threadIdx.x == 0) {
        if (V.tape_scal) {
            V.tape_scal[2 * t.x] = tau_hat;
            V.tape_scal[2 * t.x + 1] = tau_hat - kappa;
        }
        I.ot_prev = ot;
        I.eta = eta;
        I.tau = tau_new;
        I.kappa = kappa_new;
        I.iter += 1;
        if (!isfinite(eta) || !isfinite(tau_new) || !isfinite(kappa_new)) I.status = HSDE_NUMERICAL_ERROR;
        V.counters[2 * t.x] = 0;
    }
}

// x = alpha (x_w - eta x_p) + (1 - alpha) x; stopping-rule partials over N
// (r = A^T y + H^T z):
//   ||r - tau c||^2, ||r||^2, c^T x  (full-vec weights), on check iterations;
// f = Delta^{-1}(x - omega_tau' c + 1/2 H^T (s+z+v)) for the next iteration;
// y = alpha (y_w - eta y_p) + (1 - alpha) y over a slice of the constraints
// per CTA, with the constraint-space partials ||D^{-1}(A x - tau b)||^2,
// ||D^{-1} A x||^2, b^T y; the last CTA of each instance takes the verdict
// (readings P5/P6) on the unscaled values (reading P7).
// With alpha != 1 the new A x and A^T y need those of the previous iterate:
// they are kept in V.ax and V.aty (A x_hat and A^T y_hat come from the
// affine step's own vectors, see below).
// Copies of pattern entries (H^T) staged per pass of k_post.
constexpr int POST_STAGE = 2048;

template <typename T>
__global__ void __launch_bounds__(NT) k_post(DevView V) {
    __shared__ int flag;
    // per staged copy: z, and s + z + v; afterwards the reductions' buffer
    __shared__ double stage[2 * POST_STAGE];
    double* cz = stage;
    double* call = stage + POST_STAGE;
    static_assert(2 * POST_STAGE >= 11 * NT, "the reductions reuse the staging buffer");
    const int4 t = V.tiles[blockIdx.x];
    InstDev& I = V.inst[t.x];
    if (I.status != HSDE_RUNNING) return;
    const bool check = is_check_iter(V, I.iter);
    const double eta = I.eta, tau = I.tau;
    const double ot = I.tau + I.kappa;            // omega_tau of the next iteration
    const double al = V.alpha;
    const bool relax = al != 1.0;
    // Stopping-rule partial sums of this tile in PS: FP32 in the mixed form
    // (each is tested to ~1e-4 and the differences inside them, r - tau c and
    // A x - tau b, are formed in FP64 first), FP64 in the FP64 form; the
    // tiles' partials are added in FP64 by the last CTA.
    using PS = T;
    PS a1 = PS(0), a2 = PS(0), a3 = PS(0);
    // ||A^T y||^2, ||H^T z||^2, ||H x||^2 for the certificate cancellation
    // test, which compares them with 1e-2 only: accumulated in FP32
    float a4 = 0.f, a5 = 0.f, a6 = 0.f;
    // one pattern entry per thread (TILE_N == NT)
    const int e = t.y + threadIdx.x;
    const bool has = e < t.z;
    double x = 0.0;
    int k0 = 0, k1 = 0, ncopy = 0;
    if (has) {
        const double xh = V.xw[e] - eta * V.xp[e];
        x = relax ? al * xh + (1.0 - al) * V.x[e] : xh;
        V.x[e] = x;
        k0 = V.ssc_ptr[e];
        k1 = V.ssc_ptr[e + 1];
        ncopy = V.sc_ptr[e + 1] - V.sc_ptr[e];
    }
    // H^T z and H^T (s + z + v): the tile's short copies are one contiguous
    // range; the CTA loads them together (coalesced indices, one gather per
    // copy) into shared memory, then each entry sums its own copies in
    // order.  A long entry takes the sums k_long formed.
    double hz = 0.0, hall = 0.0;
    const int c0 = V.ssc_ptr[t.y], c1 = V.ssc_ptr[t.z];
    for (int cb = c0; cb < c1; cb += POST_STAGE) {
        const int ce = min(c1, cb + POST_STAGE);
        __syncthreads();
        for (int c = cb + threadIdx.x; c < ce; c += NT) {
            const int p = V.ssc_idx[c];
            cz[c - cb] = ld<T>(V.z, p);
            call[c - cb] = copy_szv<T>(V, p);
        }
        __syncthreads();
        const int a = max(k0, cb), b = min(k1, ce);
        for (int k = a; k < b; ++k) {
            hz += cz[k - cb];
            hall += call[k - cb];
        }
    }
    if (has) {
        const int li = V.long_id[e];
        if (li >= 0) {
            hz = V.lhz[li];
            hall = V.lall[li];
        }
        const double ce = V.c[e];
        V.f[e] = (x - ot * ce + 0.5 * hall) * V.inv_delta[e];
        // A^T y_hat = A^T y_w - eta A^T y_p (both kept from this iteration / setup)
        double aty = V.atyw[e] - eta * V.atyp[e];
        if (relax) {
            aty = al * aty + (1.0 - al) * V.aty[e];
            V.aty[e] = aty;
        }
        if (check) {
            const double r = hz + aty;
            const double d = r - tau * ce;
            const PS w = V.diag[e] ? PS(1) : PS(2);
            const PS pd = (PS)d, pr = (PS)r;
            a1 += w * pd * pd;
            a2 += w * pr * pr;
            a3 += w * (PS)ce * (PS)x;
            const float fw = (float)w, fa = (float)aty, fh = (float)hz, fx = (float)x;
            a4 += fw * fa * fa;
            a5 += fw * fh * fh;
            a6 += fw * (float)ncopy * fx * fx;    // x repeated in each clique containing it
        }
    }
    // This CTA's slice of the constraints.  A x is not formed by an SpMV:
    // with S y_w = q,
    //   A x_w = A f + A Delta^{-1} A^T y_w = A f + (S - I) y_w = A f + q - y_w,
    //   A x_p = -b - y_p  (the same identity on the setup solve),
    // so A x_hat = A x_w - eta A x_p from values this step already has.
    PS b1 = PS(0), b2 = PS(0), b3 = PS(0);
    bool has_rows;
    {
        const int nt = I.tile_end - I.tile_begin, ti = blockIdx.x - I.tile_begin;
        const int i0 = (int)((int64_t)I.m * ti / nt), i1 = (int)((int64_t)I.m * (ti + 1) / nt);
        has_rows = i1 > i0;
        const double otp = I.ot_prev;
        for (int i = i0 + threadIdx.x; i < i1; i += NT) {
            const int row = I.m_off + i;
            const double bi = V.b[row], yw = V.yw[row], yp = V.yp[row];
            const double yold = V.y[row];
            double ynew = yw - eta * yp;
            if (relax) ynew = al * ynew + (1.0 - al) * yold;
            if (check || relax) {
                const double afr = V.af[row];
                const double q = yold + otp * bi - afr;
                double ax = (afr + q - yw) - eta * (-bi - yp);
                if (relax) {
                    ax = al * ax + (1.0 - al) * V.ax[row];
                    V.ax[row] = ax;
                }
                if (check) {
                    const PS w2 = (PS)V.dinv2[row];
                    const PS pd = (PS)(ax - tau * bi), pa = (PS)ax;
                    b1 += w2 * pd * pd;
                    b2 += w2 * pa * pa;
                    b3 += (PS)bi * (PS)ynew;
                }
            }
            V.y[row] = ynew;
        }
    }
    if (check) {
        double* pp = V.part + (int64_t)blockIdx.x * KPART;
        if constexpr (sizeof(PS) == 4) {
            // the mixed form: one FP32 reduction of all nine
            float v9[9] = {a1, a2, a3, b1, b2, b3, a4, a5, a6};
            block_sum_t<9>(v9, reinterpret_cast<float*>(stage));
            if (threadIdx.x == 0) {
#pragma unroll
                for (int i = 0; i < 9; ++i) pp[1 + i] = (double)v9[i];
            }
        } else {
            // FP64 pipe time is what this kernel spends: the three N-space
            // sums in FP64, the cancellation sums (compared with 1e-2 only)
            // in FP32, and the constraint-space sums only in tiles that hold
            // constraints
            double v3[3] = {a1, a2, a3};
            block_sum_t<3>(v3, stage);
            float f3[3] = {a4, a5, a6};
            block_sum_t<3>(f3, reinterpret_cast<float*>(stage));
            double w3[3] = {b1, b2, b3};
            if (has_rows) block_sum_t<3>(w3, stage);
            if (threadIdx.x == 0) {
                const double out9[9] = {v3[0], v3[1], v3[2], w3[0], w3[1], w3[2],
                                        (double)f3[0], (double)f3[1], (double)f3[2]};
#pragma unroll
                for (int i = 0; i < 9; ++i) pp[1 + i] = out9[i];
            }
        }
    }
    if (!last_cta(V.counters + 2 * t.x + 1, I.tile_end - I.tile_begin, &flag)) return;
    // ---- last CTA of this instance ----
    if (threadIdx.x == 0) {
        V.counters[2 * t.x + 1] = 0;
        I.vcold = 0;                                // stored eigenbases are valid from now on
        const int uc = atomicExch(&I.unconv, 0);    // every k_cone of this iteration is done
        I.unconv_last = uc;
        if (uc > 0) I.unconv_iters += 1;
    }
    if (!check) return;
    double v11[11] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
    for (int tt = I.tile_begin + threadIdx.x; tt < I.tile_end; tt += NT) {
        const double* pp = V.part + (int64_t)tt * KPART;
#pragma unroll
        for (int i = 0; i < 9; ++i) v11[i] += __ldcg(pp + 1 + i);
    }
    for (int k = I.cl_begin + threadIdx.x; k < I.cl_end; k += NT) {
        v11[9] += __ldcg(V.cl_part + 2 * k);
        v11[10] += __ldcg(V.cl_part + 2 * k + 1);
    }
    block_sum_t<11>(v11, stage);
    a1 = v11[0]; a2 = v11[1]; a3 = v11[2];
    const double r0 = v11[3], r1 = v11[4], r2 = v11[5], hs = v11[9];
    const double aty2 = v11[6], hz2 = v11[7], hx2 = v11[8], ss2 = v11[10];
    if (threadIdx.x != 0) return;
    // unscaled values (reading P7): x = x~/sigma, s = s~/sigma, y = D y~/rho,
    // z = z~/rho, so c^T x = c~^T x~/(rho sigma), b^T y = b~^T y~/(sigma rho),
    // A x - tau b = D^{-1}(A~ x~ - tau b~)/sigma, A^T y + H^T z = r~/rho
    const double sg = I.sigma, rh = I.rho;
    const double ctx = a3 / (rh * sg), bty = r2 / (sg * rh);
    double pres = INFINITY, dres = INFINITY, gap = INFINITY, pobj = NAN, dobj = NAN;
    if (tau > 0) {
        pres = sqrt(r0 + hs) / (sg * tau) / (1.0 + I.bnorm);
        dres = sqrt(a1) / (rh * tau) / (1.0 + I.cnorm);
        pobj = ctx / tau;
        dobj = bty / tau;
        gap = fabs(pobj - dobj) / (1.0 + fabs(pobj) + fabs(dobj));
    }
    const double pinf = bty > 0 ? sqrt(a2) / rh / bty : INFINITY;
    const double dinf = ctx < 0 ? sqrt(r1 + hs) / sg / (-ctx) : INFINITY;
    // reading P6: a certificate's two terms must also cancel (scale-free, so
    // the scaled sums serve as they are)
    const double pden = sqrt(aty2) + sqrt(hz2), dden = sqrt(hx2) + sqrt(ss2);
    const double pcan = pden > 0 ? sqrt(a2) / pden : INFINITY;
    const double dcan = dden > 0 ? sqrt(r1 + hs) / dden : INFINITY;
    I.pres = pres; I.dres = dres; I.gap = gap; I.pobj = pobj; I.dobj = dobj;
    I.pinf = pinf; I.dinf = dinf; I.ctx = ctx; I.bty = bty;
    int st = HSDE_RUNNING;
    if (!isfinite(a1) || !isfinite(a2) || !isfinite(r0) || !isfinite(hs) || !isfinite(ctx) || !isfinite(bty)) {
        st = HSDE_NUMERICAL_ERROR;
    } else if (tau > 0 && pres <= V.eps && dres <= V.eps && gap <= V.eps) {
        st = HSDE_SOLVED;
    } else if (bty > 0 && pinf <= V.eps && pcan <= CERT_CANCEL) {
        st = HSDE_PRIMAL_INFEASIBLE;
    } else if (ctx < 0 && dinf <= V.eps && dcan <= CERT_CANCEL) {
        st = HSDE_DUAL_INFEASIBLE;
    } else if (I.iter >= V.max_iter) {
        st = HSDE_MAX_ITER;
    }
    I.status = st;
}

// den = 1 + c^T x_p - b^T y_p, ctp = den - 1.  One CTA per instance.  (The
// norms of the original b and c used by the stopping rule are set on the host.)
__global__ void __launch_bounds__(NT) k_setup_den(DevView V) {
    __shared__ double sh[32];
    InstDev& I = V.inst[blockIdx.x];
    double ctp = 0.0;
    for (int t = I.tile_begin + threadIdx.x; t < I.tile_end; t += NT) ctp += V.part[(int64_t)t * KPART];
    ctp = block_sum(ctp, sh);
    double btp = 0.0;
    for (int i = threadIdx.x; i < I.m; i += NT) btp += V.b[I.m_off + i] * V.yp[I.m_off + i];
    btp = block_sum(btp, sh);
    if (threadIdx.x == 0) {
        I.ctp = ctp - btp;
        I.den = 1.0 + I.ctp;
    }
}

// A x and A^T y of the stored iterate (rows [r0, r1) and entries [e0, e1) of
// one instance), for the over-relaxation after a state is loaded.
__global__ void __launch_bounds__(NT) k_state_ax(DevView V, int r0, int r1) {
    const int row = r0 + (int)(((int64_t)blockIdx.x * NT + threadIdx.x) >> 5), lane = threadIdx.x & 31;
    if (row >= r1) return;
    double acc = 0.0;
    const int j1 = V.A_ptr[row + 1];
    for (int j = V.A_ptr[row] + lane; j < j1; j += 32) acc += V.A_val[j] * V.x[V.A_col[j]];
    acc = warp_sum(acc);
    if (lane == 0) V.ax[row] = acc;
}

__global__ void __launch_bounds__(NT) k_state_aty(DevView V, int64_t e0, int64_t e1) {
    const int64_t e = e0 + (int64_t)blockIdx.x * NT + threadIdx.x;
    if (e >= e1) return;
    double acc = 0.0;
    const int j1 = V.At_ptr[e + 1];
    for (int j = V.At_ptr[e]; j < j1; ++j) acc += V.At_val[j] * V.y[V.At_col[j]];
    V.aty[e] = acc;
}

// One in-place Gauss-Jordan step (pivot k) on every dense S with m > k.
// S is symmetric positive definite with eigenvalues >= 1, so no pivoting is
// needed.  rowbuf/colbuf hold row k and column k before the step.  The dense
// instances are sorted by m (descending) so the ones still active at step k
// are a prefix; their 32 x 8 tiles are numbered consecutively (tile_pre) and
// one CTA handles one tile, so no CTA is launched for a finished instance.
__global__ void k_gj_copy(double* pool, const int64_t* offs, const int32_t* ms, int nact, int k,
                          double* rowbuf, double* colbuf, const int64_t* boff) {
    const int d = blockIdx.y;
    if (d >= nact) return;
    const int m = ms[d];
    double* S = pool + offs[d];
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < m; j += gridDim.x * blockDim.x) {
        rowbuf[boff[d] + j] = S[(int64_t)k * m + j];
        colbuf[boff[d] + j] = S[(int64_t)j * m + k];
    }
}

__global__ void k_gj_update(double* pool, const int64_t* offs, const int32_t* ms, const int64_t* tile_pre,
                            int nact, int k, const double* rowbuf, const double* colbuf, const int64_t* boff) {
    // find the instance of this tile (tile_pre is the exclusive prefix of tile counts)
    const int64_t tile = blockIdx.x;
    int lo = 0, hi = nact - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (tile_pre[mid] <= tile) lo = mid; else hi = mid - 1;
    }
    const int d = lo;
    const int m = ms[d];
    const int tx = (m + 31) / 32;
    const int64_t local = tile - tile_pre[d];
    const int ti = (int)(local / tx), tj = (int)(local - (local / tx) * tx);
    const int i = ti * 8 + threadIdx.y;
    const int j = tj * 32 + threadIdx.x;
    if (i >= m || j >= m) return;
    double* S = pool + offs[d];
    const double* rk = rowbuf + boff[d];
    const double* ck = colbuf + boff[d];
    const double piv = rk[k];
    double val;
    if (i == k && j == k) val = 1.0 / piv;
    else if (i == k) val = rk[j] / piv;
    else if (j == k) val = -ck[i] / piv;
    else val = S[(int64_t)i * m + j] - ck[i] * rk[j] / piv;
    S[(int64_t)i * m + j] = val;
}

// ---------------------------------------------------------------------------
// Dense S = I + A Delta^{-1} A^T (Section 4.3, the matrix of Eq.
// FactorizationMatrix) formed on the device, one warp per constraint row i of
// the dense instances:  S_ij = delta_ij + sum_{e in A_i} A_ie Delta_e^{-1}
// a_je, with A_ie the weighted value of row i (off-diagonal entries count
// twice) and a_je the raw values of column e of A^T.  The warp walks row i's
// entries in order and its lanes spread over each entry's constraints, which
// are distinct, so every S_ij receives its terms in a fixed order
// (deterministic); the row is built in shared memory (SMEM) or in place in
// the pool row, which the warp owns.
// ---------------------------------------------------------------------------
template <bool SMEM>
__global__ void k_form_S(DevView V, const int32_t* rows, int32_t nrows, int warps, int32_t stride) {
    extern __shared__ double srow[];
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    const int32_t r = blockIdx.x * warps + w;
    if (r >= nrows) return;
    const int32_t i = rows[r];
    const InstDev& I = V.inst[V.row_inst[i]];
    const int32_t m = I.m, mo = I.m_off;
    double* out = V.sinv + I.sinv_off + (int64_t)(i - mo) * m;
    // each warp's row buffer: stride = the largest m of the launch (the
    // warps of one CTA can serve instances of different m)
    double* acc = SMEM ? srow + (size_t)w * stride : out;
    for (int32_t j = l; j < m; j += 32) acc[j] = (j == i - mo) ? 1.0 : 0.0;
    __syncwarp();
    for (int32_t k = V.A_ptr[i]; k < V.A_ptr[i + 1]; ++k) {
        const int32_t e = V.A_col[k];
        const double we = V.A_val[k] * V.inv_delta[e];
        for (int32_t t = V.At_ptr[e] + l; t < V.At_ptr[e + 1]; t += 32)
            acc[V.At_col[t] - mo] += we * V.At_val[t];
        __syncwarp();
    }
    if (SMEM)
        for (int32_t j = l; j < m; j += 32) out[j] = acc[j];
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
static inline cudaStream_t S_(void* st) { return reinterpret_cast<cudaStream_t>(st); }
// one warp per row; rows < 2^31 / 32 is guaranteed by the setup limits
static inline int rows_grid(int rows) { return (int)(((int64_t)rows * 32 + NT - 1) / NT); }

void launch_long(const DevView& V, bool mixed, void* st) {
    if (V.nlong <= 0) return;
    if (mixed) k_long<float><<<V.nlong, NT, 0, S_(st)>>>(V);
    else k_long<double><<<V.nlong, NT, 0, S_(st)>>>(V);
}

void launch_rhs(const DevView& V, bool mixed, Mode mode, void* st) {
    if (V.ntiles == 0) return;
    if (mode == Mode::Iter) launch_long(V, mixed, st);
    if (mixed) k_rhs<float><<<V.ntiles, NT, 0, S_(st)>>>(V, (int)mode);
    else k_rhs<double><<<V.ntiles, NT, 0, S_(st)>>>(V, (int)mode);
}
void launch_spmv_A(const DevView& V, Mode mode, void* st) {
    if (V.Mtot == 0) return;
    k_spmv_A<<<rows_grid(V.Mtot), NT, 0, S_(st)>>>(V, (int)mode);
}
void launch_solve(const DevView& V, Mode mode, void* st) {
    if (V.Mtot == 0) return;
    k_solve<<<rows_grid(V.Mtot), NT, 0, S_(st)>>>(V, (int)mode);
    if (mode == Mode::Iter) launch_lr_solve(V, V.q, V.yw, V.rowb, true, st);
    else launch_lr_solve(V, V.q, V.yp, nullptr, false, st);
}
void launch_spmv_At(const DevView& V, Mode mode, void* st) {
    if (V.ntiles == 0) return;
    k_spmv_At<<<V.ntiles, NT, 0, S_(st)>>>(V, (int)mode);
}
void launch_setup_den(const DevView& V, void* st) { k_setup_den<<<V.B, NT, 0, S_(st)>>>(V); }

void launch_state_products(const DevView& V, int r0, int r1, int64_t e0, int64_t e1, void* st) {
    if (r1 > r0) k_state_ax<<<rows_grid(r1 - r0), NT, 0, S_(st)>>>(V, r0, r1);
    if (e1 > e0) k_state_aty<<<(unsigned)((e1 - e0 + NT - 1) / NT), NT, 0, S_(st)>>>(V, e0, e1);
}

void launch_fwd(const DevView& V, void* st) {
    if (V.Mtot > 0) k_fwd<<<rows_grid(V.Mtot), NT, 0, S_(st)>>>(V);
}
void launch_solve_dense(const DevView& V, void* st) {
    if (V.Mtot > 0) k_solve_dense<<<rows_grid(V.Mtot), NT, 0, S_(st)>>>(V);
}
void launch_bwd_eta(const DevView& V, void* st) {
    if (V.nat > 0) k_bwd_eta<<<V.nat, NT, 0, S_(st)>>>(V);
}
void launch_post(const DevView& V, bool mixed, void* st) {
    if (V.ntiles == 0) return;
    if (mixed) k_post<float><<<V.ntiles, NT, 0, S_(st)>>>(V);
    else k_post<double><<<V.ntiles, NT, 0, S_(st)>>>(V);
}

// ---------------------------------------------------------------------------
// New data (c, b) given in device memory (hsde_set_data).  k_data_sums forms,
// per CTA, the count of non-finite values, sum (d_i b_i)^2, sum b_i^2 and the
// full-vec sum of c_e^2 that the scaling of reading P7 needs; the host adds
// the CTAs' partials in order.  k_data_apply writes c~ = rho c and
// b~ = sigma D b into the instance's slices.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(NT) k_data_sums(const double* c, int64_t N, const uint8_t* diag,
                                                  const double* b, int32_t m, const double* dscale,
                                                  const int32_t* perm, double* part) {
    __shared__ double sh[4 * (NT / 32)];
    double v[4] = {0.0, 0.0, 0.0, 0.0};
    const int64_t stride = (int64_t)gridDim.x * NT;
    for (int64_t e = (int64_t)blockIdx.x * NT + threadIdx.x; e < N; e += stride) {
        const double ce = c[e];
        if (!isfinite(ce)) v[0] += 1.0;
        else v[3] += (diag[e] ? 1.0 : 2.0) * ce * ce;
    }
    for (int64_t i = (int64_t)blockIdx.x * NT + threadIdx.x; i < m; i += stride) {
        const double bi = b[perm ? perm[i] : i];
        if (!isfinite(bi)) {
            v[0] += 1.0;
        } else {
            const double db = dscale[i] * bi;
            v[1] += db * db;
            v[2] += bi * bi;
        }
    }
    block_sum_n<4>(v, sh);
    if (threadIdx.x == 0)
        for (int k = 0; k < 4; ++k) part[4 * blockIdx.x + k] = v[k];
}

__global__ void __launch_bounds__(NT) k_data_apply(const double* c, int64_t N, double rho, const double* b,
                                                   int32_t m, double sigma, const double* dscale,
                                                   const int32_t* perm, double* cdst, double* bdst) {
    const int64_t stride = (int64_t)gridDim.x * NT;
    for (int64_t e = (int64_t)blockIdx.x * NT + threadIdx.x; e < N; e += stride) cdst[e] = rho * c[e];
    for (int64_t i = (int64_t)blockIdx.x * NT + threadIdx.x; i < m; i += stride)
        bdst[i] = sigma * dscale[i] * b[perm ? perm[i] : i];
}

// m-vectors between the caller's constraint order and the internal one:
// gather dst[i] = src[perm[i]], scatter dst[perm[i]] = src[i].
__global__ void __launch_bounds__(NT) k_perm_move(double* dst, const double* src, const int32_t* perm, int32_t m,
                                                  int scatter) {
    for (int64_t i = (int64_t)blockIdx.x * NT + threadIdx.x; i < m; i += (int64_t)gridDim.x * NT) {
        if (scatter) dst[perm[i]] = src[i];
        else dst[i] = src[perm[i]];
    }
}

int data_grid(int64_t N, int32_t m) {
    const int64_t n = std::max<int64_t>(N, m);
    return (int)std::max<int64_t>(1, std::min<int64_t>((n + NT - 1) / NT, DATA_MAX_CTAS));
}
void launch_data_sums(const double* c, int64_t N, const uint8_t* diag, const double* b, int32_t m,
                      const double* dscale, const int32_t* perm, double* part, void* st) {
    k_data_sums<<<data_grid(N, m), NT, 0, S_(st)>>>(c, N, diag, b, m, dscale, perm, part);
}
void launch_data_apply(const double* c, int64_t N, double rho, const double* b, int32_t m, double sigma,
                       const double* dscale, const int32_t* perm, double* cdst, double* bdst, void* st) {
    k_data_apply<<<data_grid(N, m), NT, 0, S_(st)>>>(c, N, rho, b, m, sigma, dscale, perm, cdst, bdst);
}
void launch_perm_move(double* dst, const double* src, const int32_t* perm, int32_t m, bool scatter, void* st) {
    if (m <= 0) return;
    k_perm_move<<<data_grid(0, m), NT, 0, S_(st)>>>(dst, src, perm, m, scatter ? 1 : 0);
}

void launch_gj_step(double* pool, const int64_t* offs, const int32_t* ms, const int64_t* tile_pre, int nact,
                    int64_t ntiles, int32_t k, int32_t mmax, double* rowbuf, double* colbuf, const int64_t* boff,
                    void* st) {
    if (nact <= 0 || ntiles <= 0) return;
    dim3 gc((mmax + 255) / 256, nact);
    k_gj_copy<<<gc, 256, 0, S_(st)>>>(pool, offs, ms, nact, k, rowbuf, colbuf, boff);
    k_gj_update<<<(unsigned)ntiles, dim3(32, 8), 0, S_(st)>>>(pool, offs, ms, tile_pre, nact, k, rowbuf, colbuf,
                                                             boff);
}

void launch_form_S(const DevView& V, const int32_t* rows, int32_t nrows, int32_t mmax, void* st) {
    if (nrows <= 0) return;
    const size_t per_warp = sizeof(double) * (size_t)mmax;
    if (per_warp <= FORM_S_SMEM / 2) {
        const int warps = (int)std::min<size_t>(8, FORM_S_SMEM / per_warp);
        const size_t sm = per_warp * warps;
        cudaFuncSetAttribute(k_form_S<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        k_form_S<true><<<(nrows + warps - 1) / warps, 32 * warps, sm, S_(st)>>>(V, rows, nrows, warps, mmax);
    } else {
        k_form_S<false><<<(nrows + 7) / 8, 256, 0, S_(st)>>>(V, rows, nrows, 8, mmax);
    }
}

}  // namespace hsde
