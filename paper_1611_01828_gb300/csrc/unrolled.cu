// Reverse mode through unrolled ADMM iterations (Eqs. Step1-Step3).
//
// * k_rev_clique: vector-Jacobian product of the psd projection of every
//   clique block (Daleckii-Krein): for a = V diag(l) V^T and an upstream
//   symmetric gradient G,  a_bar = V (Gamma o (V^T G V)) V^T  with
//   Gamma_ij = (max(l_i,0) - max(l_j,0)) / (l_i - l_j) for l_i != l_j and
//   1, 1/2, 0 for l_i == l_j > 0, = 0, < 0 (1/2 is what a central difference
//   sees at an exactly-zero eigenvalue; eigenvalues below 1e-10 (FP64) or
//   1e-5 (FP32) of the block's largest are taken as zero).  V and l come from the forward
//   Jacobi solve of the same iteration (the tape).
// * k_ap_*: u_hat = (I + Q(c, sb*b))^{-1} omega for any omega, by the same
//   eliminations as the iteration (Sections 4.2-4.3) with the sign of b as a
//   parameter.  Q is skew-symmetric, so the adjoint solve is
//   (I+Q)^{-T} = (I - Q)^{-1} = D (I + Q(c, -b))^{-1} D,
//   D = diag(I_x, I_s, -I_y, -I_v, -1): the same cached factor S serves both.
// * k_rev_*: the remaining linear adjoints (tau step, nu update) and the
//   accumulation of the gradients with respect to c and b through Q.
// All adjoint vectors use the full-vec component convention (the adjoint of a
// lower pattern entry equals the adjoint of each of its two vec positions).
#include <cuda_runtime.h>

#include <cmath>

#include "internal.h"

namespace hsde {

static constexpr int NT = 256;

__device__ __forceinline__ double u_warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ double u_block_sum(double v, double* sh) {
    v = u_warp_sum(v);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) sh[w] = v;
    __syncthreads();
    double t = (threadIdx.x < NT / 32) ? sh[threadIdx.x] : 0.0;
    if (w == 0) t = u_warp_sum(t);
    if (threadIdx.x == 0) sh[0] = t;
    __syncthreads();
    const double r = sh[0];
    __syncthreads();
    return r;
}

template <typename T>
__device__ __forceinline__ double ldT(const void* p, int64_t i) {
    return p ? (double)reinterpret_cast<const T*>(p)[i] : 0.0;
}

// ---------------------------------------------------------------------------
// affine apply: u_hat = (I + Q(c, sb b))^{-1} omega
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(NT) k_ap_g0(DevView V, ApplyArgs A) {
    const int4 t = V.tiles[blockIdx.x];
    const double wt = A.wtau ? A.wtau[t.x] : 0.0;
    for (int e = t.y + threadIdx.x; e < t.z; e += NT) {
        double acc = 0.0;
        if (A.ws || A.wv) {
            const int k1 = V.sc_ptr[e + 1];
            for (int k = V.sc_ptr[e]; k < k1; ++k) {
                const int p = V.sc_idx[k];
                acc += ldT<T>(A.ws, p) + ldT<T>(A.wv, p);
            }
        }
        A.f[e] = (A.wx[e] - wt * V.c[e] + 0.5 * acc) * V.inv_delta[e];
    }
}

__global__ void __launch_bounds__(NT) k_ap_q(DevView V, ApplyArgs A) {
    const int row = (blockIdx.x * NT + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (row >= V.Mtot) return;
    const int b = V.row_inst[row];
    const InstDev& I = V.inst[b];
    double acc = 0.0;
    const int j1 = V.A_ptr[row + 1];
    for (int j = V.A_ptr[row] + lane; j < j1; j += 32) acc += V.A_val[j] * A.f[V.A_col[j]];
    acc = u_warp_sum(acc);
    if (lane == 0) {
        const double wt = A.wtau ? A.wtau[b] : 0.0;
        const double q = A.wy_sign * A.wy[row] + wt * A.sb * V.b[row] - acc;
        if (I.dense) A.q[row] = q;
        else A.yw[row] = V.sdiag[row] * q;
    }
}

__global__ void __launch_bounds__(NT) k_ap_solve(DevView V, ApplyArgs A) {
    const int row = (blockIdx.x * NT + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (row >= V.Mtot) return;
    const InstDev& I = V.inst[V.row_inst[row]];
    if (I.dense != 1) return;      // diagonal: done in k_ap_q; structured: launch_lr_solve
    const int i = row - I.m_off;
    const double* Srow = V.sinv + I.sinv_off + (int64_t)i * I.m;
    const double* qq = A.q + I.m_off;
    double acc = 0.0;
    for (int j = lane; j < I.m; j += 32) acc += Srow[j] * qq[j];
    acc = u_warp_sum(acc);
    if (lane == 0) A.yw[row] = acc;
}

__global__ void __launch_bounds__(NT) k_ap_xw(DevView V, ApplyArgs A) {
    __shared__ double sh[32];
    const int4 t = V.tiles[blockIdx.x];
    double part = 0.0;
    for (int e = t.y + threadIdx.x; e < t.z; e += NT) {
        double acc = 0.0;
        const int j1 = V.At_ptr[e + 1];
        for (int j = V.At_ptr[e]; j < j1; ++j) acc += V.At_val[j] * A.yw[V.At_col[j]];
        const double xv = A.f[e] + V.inv_delta[e] * acc;
        A.xw[e] = xv;
        part += (V.diag[e] ? 1.0 : 2.0) * V.c[e] * xv;
    }
    part = u_block_sum(part, sh);
    if (threadIdx.x == 0) A.part[blockIdx.x] = part;
}

// eta, tau_hat and y_hat per instance (one CTA each); setup mode (den == null)
// stores den' = 1 + c^T x_p' - sb b^T y_p' instead.
__global__ void __launch_bounds__(NT) k_ap_eta(DevView V, ApplyArgs A) {
    __shared__ double sh[32];
    const InstDev& I = V.inst[blockIdx.x];
    double ctw = 0.0;
    for (int t = I.tile_begin + threadIdx.x; t < I.tile_end; t += NT) ctw += A.part[t];
    ctw = u_block_sum(ctw, sh);
    double byw = 0.0;
    for (int i = threadIdx.x; i < I.m; i += NT) byw += V.b[I.m_off + i] * A.yw[I.m_off + i];
    byw = u_block_sum(byw, sh);
    const double sw = ctw - A.sb * byw;
    if (!A.den) {
        if (threadIdx.x == 0) {
            A.den_out[blockIdx.x] = 1.0 + sw;
            A.ctp_out[blockIdx.x] = sw;
        }
        return;
    }
    const double eta = sw / A.den[blockIdx.x];
    const double wt = A.wtau ? A.wtau[blockIdx.x] : 0.0;
    for (int i = threadIdx.x; i < I.m; i += NT)
        A.oy[I.m_off + i] = A.yw[I.m_off + i] - eta * A.yp[I.m_off + i];
    if (threadIdx.x == 0) {
        A.eta[blockIdx.x] = eta;
        A.otau[blockIdx.x] = wt + sw - eta * A.ctp[blockIdx.x];
    }
}

__global__ void __launch_bounds__(NT) k_ap_outx(DevView V, ApplyArgs A) {
    const int4 t = V.tiles[blockIdx.x];
    const double eta = A.eta[t.x];
    for (int e = t.y + threadIdx.x; e < t.z; e += NT) A.ox[e] = A.xw[e] - eta * A.xp[e];
}

// clique blocks of u_hat: s_hat = (w_s - w_v + H x_hat)/2, v_hat = (w_s + w_v - H x_hat)/2.
template <typename T>
__global__ void __launch_bounds__(NT) k_ap_outs(DevView V, ApplyArgs A) {
    const int k = (blockIdx.x * NT + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (k >= V.ncl) return;
    const double eta = A.eta[V.cl_inst[k]];
    const int c = V.cl_size[k];
    const int64_t off = V.cl_off[k];
    const int P = c * (c + 1) / 2;
    T* os = reinterpret_cast<T*>(A.os);
    T* ov = reinterpret_cast<T*>(A.ov);
    for (int t = lane; t < P; t += 32) {
        const int64_t j = off + t;
        const int gi = V.gmap[j];
        const double gx = A.xw[gi] - eta * A.xp[gi];
        const double ws = ldT<T>(A.ws, j), wv = ldT<T>(A.wv, j);
        os[j] = (T)(0.5 * (ws - wv + gx));
        ov[j] = (T)(0.5 * (ws + wv - gx));
    }
}

// ---------------------------------------------------------------------------
// Daleckii-Krein backward of the clique projections
// ---------------------------------------------------------------------------
template <typename T, int CP, int G>
struct RevCfg {
    static constexpr int LD = CP + 2;
    static constexpr int NTH = (G >= 128) ? G : 128;
    static constexpr int GPB = NTH / G;
    static constexpr size_t group_bytes = ((3 * CP * LD + CP) * sizeof(T) + 15) / 16 * 16;
    static constexpr size_t smem = GPB * group_bytes;
};

template <int G>
__device__ __forceinline__ void rsync(int gid) {
    if constexpr (G < 32) {
        const int base = (threadIdx.x & 31) & ~(G - 1);
        __syncwarp(((1u << G) - 1u) << base);
    } else if constexpr (G == 32) {
        __syncwarp();
    } else {
        asm volatile("bar.sync %0, %1;" ::"r"(gid + 1), "r"(G) : "memory");
    }
}

template <typename T>
__device__ __forceinline__ T dk_gamma(T li, T lj) {
    if (li == lj) return li > T(0) ? T(1) : (li < T(0) ? T(0) : T(0.5));
    const T pi = li > T(0) ? li : T(0), pj = lj > T(0) ? lj : T(0);
    return (pi - pj) / (li - lj);
}

// For every clique of one bucket: G = s_bar + z_bar (upstream adjoint of the
// projected block), a_bar = DK(G); writes the D-flipped adjoint inputs of
// the affine solve, w_s = a_bar - z_bar and w_v = -v_bar, and z_bar -= a_bar.
template <typename T, int CP, int G>
__global__ void __launch_bounds__(RevCfg<T, CP, G>::NTH)
k_rev_clique(DevView V, RevArgs R, const int32_t* __restrict__ list, int nlist) {
    using Cfg = RevCfg<T, CP, G>;
    constexpr int LD = Cfg::LD;
    extern __shared__ __align__(16) unsigned char smem_u[];
    const int gid = threadIdx.x / G, lane = threadIdx.x % G;
    const int li = blockIdx.x * Cfg::GPB + gid;
    if (li >= nlist) return;
    const int k = list[li];
    T* Vm = reinterpret_cast<T*>(smem_u + (size_t)gid * Cfg::group_bytes);
    T* Gm = Vm + CP * LD;
    T* Tm = Gm + CP * LD;
    T* lam = Tm + CP * LD;
    const T* tv = reinterpret_cast<const T*>(R.tape_v) + R.tv_off[k];
    const int c = V.cl_size[k];
    const int64_t off = V.cl_off[k];
    T* sbar = reinterpret_cast<T*>(R.sbar);
    T* zbar = reinterpret_cast<T*>(R.zbar);
    const T* vbar = reinterpret_cast<const T*>(R.vbar);
    T* aws = reinterpret_cast<T*>(R.aw_s);
    T* awv = reinterpret_cast<T*>(R.aw_v);
    for (int idx = lane; idx < CP * CP; idx += G) {
        const int i = idx / CP, j = idx - (idx / CP) * CP;
        Vm[i * LD + j] = tv[idx];
        Gm[i * LD + j] = T(0);
    }
    for (int i = lane; i < CP; i += G) lam[i] = tv[CP * CP + i];
    rsync<G>(gid);
    // eigenvalues below a fraction of the block's largest count as exactly 0
    // (1e-10 in FP64, 1e-5 in FP32), so rounding does not pick the derivative
    {
        T mx = 0;
        for (int i = 0; i < CP; ++i) mx = fmax(mx, fabs(lam[i]));
        const T thr = mx * (sizeof(T) == 8 ? T(1e-10) : T(1e-5));
        rsync<G>(gid);
        for (int i = lane; i < CP; i += G)
            if (fabs(lam[i]) <= thr) lam[i] = T(0);
        rsync<G>(gid);
    }
    for (int idx = lane; idx < c * c; idx += G) {
        const int bcol = idx / c, arow = idx - bcol * c;
        if (arow < bcol) continue;
        const int64_t j = off + (int64_t)bcol * c - (bcol * (bcol - 1)) / 2 + (arow - bcol);
        const T g = sbar[j] + zbar[j];
        Gm[arow * LD + bcol] = g;
        Gm[bcol * LD + arow] = g;
    }
    rsync<G>(gid);
    // Tm = G V
    for (int idx = lane; idx < CP * CP; idx += G) {
        const int i = idx / CP, j = idx - (idx / CP) * CP;
        T acc = 0;
        for (int q = 0; q < CP; ++q) acc += Gm[i * LD + q] * Vm[q * LD + j];
        Tm[i * LD + j] = acc;
    }
    rsync<G>(gid);
    // Gm = Gamma o (V^T Tm)
    for (int idx = lane; idx < CP * CP; idx += G) {
        const int i = idx / CP, j = idx - (idx / CP) * CP;
        T acc = 0;
        for (int q = 0; q < CP; ++q) acc += Vm[q * LD + i] * Tm[q * LD + j];
        Gm[i * LD + j] = acc * dk_gamma<T>(lam[i], lam[j]);
    }
    rsync<G>(gid);
    // Tm = V Gm
    for (int idx = lane; idx < CP * CP; idx += G) {
        const int i = idx / CP, j = idx - (idx / CP) * CP;
        T acc = 0;
        for (int q = 0; q < CP; ++q) acc += Vm[i * LD + q] * Gm[q * LD + j];
        Tm[i * LD + j] = acc;
    }
    rsync<G>(gid);
    // a_bar = Tm V^T (lower entries of the real block)
    for (int idx = lane; idx < c * c; idx += G) {
        const int bcol = idx / c, arow = idx - bcol * c;
        if (arow < bcol) continue;
        T acc = 0;
        for (int q = 0; q < CP; ++q) acc += Tm[arow * LD + q] * Vm[bcol * LD + q];
        const int64_t j = off + (int64_t)bcol * c - (bcol * (bcol - 1)) / 2 + (arow - bcol);
        const T zb = zbar[j];
        aws[j] = acc - zb;
        awv[j] = -vbar[j];
        zbar[j] = zb - acc;
    }
}

// ---------------------------------------------------------------------------
// scalar and vector adjoint updates
// ---------------------------------------------------------------------------
// tau' = max(0, tau_hat - kappa), kappa' = kappa - tau_hat + tau':
// input adjoints (taubar, kappabar) of (tau', kappa'); output the D-flipped
// w_tau = -tau_hat_bar for the affine solve and the partial kappa adjoint.
__global__ void k_rev_scal_pre(RevArgs R, int slot, int B) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    const double tb = R.adj_scal[2 * b], kb = R.adj_scal[2 * b + 1];
    const double pos = R.tape_scal[(size_t)slot * 2 * B + 2 * b + 1] > 0.0 ? 1.0 : 0.0;
    const double tt = tb + kb;
    const double that_bar = -kb + pos * tt;
    R.wtau[b] = -that_bar;
    R.kpart[b] = kb - pos * tt;
}

__global__ void k_rev_scal_post(RevArgs R, int B) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    const double om_tau = -R.otau[b];
    R.adj_scal[2 * b] = om_tau;
    R.adj_scal[2 * b + 1] = R.kpart[b] + om_tau;
}

// x_bar <- omega_bar_x;  g_c += -(omega_bar_x tau_hat - omega_bar_tau x_hat)
__global__ void __launch_bounds__(NT) k_rev_upd_n(DevView V, RevArgs R, int slot) {
    const int4 t = V.tiles[blockIdx.x];
    const int B = V.B;
    const double that = R.tape_scal[(size_t)slot * 2 * B + 2 * t.x];
    const double om_tau = -R.otau[t.x];
    const double* xh = R.tape_x + (size_t)slot * V.Ntot;
    for (int e = t.y + threadIdx.x; e < t.z; e += NT) {
        const double ox = R.ox[e];
        R.gc[e] += -(ox * that - om_tau * xh[e]);
        R.xbar[e] = ox;
    }
}

// y_bar <- omega_bar_y = -o_y;  g_b += omega_bar_y tau_hat - omega_bar_tau y_hat
__global__ void __launch_bounds__(NT) k_rev_upd_m(DevView V, RevArgs R, int slot) {
    const int row = blockIdx.x * NT + threadIdx.x;
    if (row >= V.Mtot) return;
    const int b = V.row_inst[row];
    const int B = V.B;
    const double that = R.tape_scal[(size_t)slot * 2 * B + 2 * b];
    const double om_tau = -R.otau[b];
    const double om_y = -R.oy[row];
    const double yh = R.tape_y[(size_t)slot * V.Mtot + row];
    R.gb[row] += om_y * that - om_tau * yh;
    R.ybar[row] = om_y;
}

// s_bar <- o_s, v_bar <- -o_v, z_bar += o_s
template <typename T>
__global__ void __launch_bounds__(NT) k_rev_upd_p(DevView V, RevArgs R) {
    const int64_t j = (int64_t)blockIdx.x * NT + threadIdx.x;
    if (j >= V.Ptot) return;
    const T os = reinterpret_cast<const T*>(R.os)[j];
    reinterpret_cast<T*>(R.sbar)[j] = os;
    reinterpret_cast<T*>(R.vbar)[j] = -reinterpret_cast<const T*>(R.ov)[j];
    reinterpret_cast<T*>(R.zbar)[j] += os;
}

// seeds given per lower pattern entry (gradient with respect to the stored
// value) -> full-vec component adjoint: divide off-diagonal entries by 2
__global__ void __launch_bounds__(NT) k_rev_seed(DevView V, RevArgs R) {
    const int64_t e = (int64_t)blockIdx.x * NT + threadIdx.x;
    if (e >= V.Ntot) return;
    R.xbar[e] = R.xbar[e] * (V.diag[e] ? 1.0 : 0.5);
}

// gradient per stored lower value of C: off-diagonal entries count twice
__global__ void __launch_bounds__(NT) k_rev_finish(DevView V, RevArgs R) {
    const int64_t e = (int64_t)blockIdx.x * NT + threadIdx.x;
    if (e >= V.Ntot) return;
    R.gc[e] = R.gc[e] * (V.diag[e] ? 1.0 : 2.0);
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
static inline cudaStream_t Su(void* st) { return reinterpret_cast<cudaStream_t>(st); }

void launch_apply(const DevView& V, const ApplyArgs& A, bool mixed, bool setup_only, void* st) {
    if (V.ntiles > 0) {
        if (mixed) k_ap_g0<float><<<V.ntiles, NT, 0, Su(st)>>>(V, A);
        else k_ap_g0<double><<<V.ntiles, NT, 0, Su(st)>>>(V, A);
    }
    if (V.Mtot > 0) {
        const int rg = (V.Mtot * 32 + NT - 1) / NT;
        k_ap_q<<<rg, NT, 0, Su(st)>>>(V, A);
        k_ap_solve<<<rg, NT, 0, Su(st)>>>(V, A);
        launch_lr_solve(V, A.q, A.yw, nullptr, false, st);
    }
    if (V.ntiles > 0) k_ap_xw<<<V.ntiles, NT, 0, Su(st)>>>(V, A);
    k_ap_eta<<<V.B, NT, 0, Su(st)>>>(V, A);
    if (setup_only) return;
    if (V.ntiles > 0) k_ap_outx<<<V.ntiles, NT, 0, Su(st)>>>(V, A);
    if (V.ncl > 0) {
        const int cg = (V.ncl * 32 + NT - 1) / NT;
        if (mixed) k_ap_outs<float><<<cg, NT, 0, Su(st)>>>(V, A);
        else k_ap_outs<double><<<cg, NT, 0, Su(st)>>>(V, A);
    }
}

// the same padded sizes as the forward eigensolver's buckets (cone.cu)
#define HSDE_REV_BUCKETS(X)                                                                     \
    X(4, 4) X(8, 8) X(12, 16) X(16, 32) X(20, 64) X(24, 64) X(28, 128) X(32, 128) X(36, 256)   \
    X(40, 256) X(44, 512) X(48, 512) X(56, 512) X(64, 512) X(80, 512) X(96, 1024) X(112, 1024)

// a size exists for a precision only if its CTA fits the opt-in shared memory
template <typename T, int CP, int G>
constexpr bool rev_fits() {
    return RevCfg<T, CP, G>::smem <= 232448;
}

template <typename T, int CP, int G>
static int rev_prepare_one() {
    if constexpr (!rev_fits<T, CP, G>()) return HSDE_OK;
    using Cfg = RevCfg<T, CP, G>;
    if (Cfg::smem > 48 * 1024 &&
        cudaFuncSetAttribute(k_rev_clique<T, CP, G>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Cfg::smem) !=
            cudaSuccess)
        return HSDE_ECUDA;
    return HSDE_OK;
}

int rev_prepare(bool mixed) {
    int rc = HSDE_OK;
#define X(cp, g) rc |= mixed ? rev_prepare_one<float, cp, g>() : rev_prepare_one<double, cp, g>();
    HSDE_REV_BUCKETS(X)
#undef X
    return rc == HSDE_OK ? HSDE_OK : HSDE_ECUDA;
}

template <typename T, int CP, int G>
static int rev_launch_one(const DevView& V, const RevArgs& R, const Bucket& bk, void* st) {
    if constexpr (!rev_fits<T, CP, G>()) {
        return HSDE_ERANGE;
    } else {
        using C = RevCfg<T, CP, G>;
        k_rev_clique<T, CP, G><<<(bk.count + C::GPB - 1) / C::GPB, C::NTH, C::smem, Su(st)>>>(V, R, bk.list,
                                                                                             bk.count);
        return HSDE_OK;
    }
}

int launch_rev_clique(const DevView& V, const RevArgs& R, const Bucket& bk, bool mixed, void* st) {
    if (bk.count == 0) return HSDE_OK;
#define X(cp, g)                                                                  \
    if (bk.cmax == cp) return mixed ? rev_launch_one<float, cp, g>(V, R, bk, st)   \
                                    : rev_launch_one<double, cp, g>(V, R, bk, st);
    HSDE_REV_BUCKETS(X)
#undef X
    return HSDE_ERANGE;
}

void launch_rev_scal_pre(const RevArgs& R, int slot, int B, void* st) {
    k_rev_scal_pre<<<(B + 127) / 128, 128, 0, Su(st)>>>(R, slot, B);
}
void launch_rev_scal_post(const RevArgs& R, int B, void* st) {
    k_rev_scal_post<<<(B + 127) / 128, 128, 0, Su(st)>>>(R, B);
}
void launch_rev_update(const DevView& V, const RevArgs& R, int slot, bool mixed, void* st) {
    if (V.ntiles > 0) k_rev_upd_n<<<V.ntiles, NT, 0, Su(st)>>>(V, R, slot);
    if (V.Mtot > 0) k_rev_upd_m<<<(V.Mtot + NT - 1) / NT, NT, 0, Su(st)>>>(V, R, slot);
    if (V.Ptot > 0) {
        const unsigned g = (unsigned)((V.Ptot + NT - 1) / NT);
        if (mixed) k_rev_upd_p<float><<<g, NT, 0, Su(st)>>>(V, R);
        else k_rev_upd_p<double><<<g, NT, 0, Su(st)>>>(V, R);
    }
}
void launch_rev_seed(const DevView& V, const RevArgs& R, void* st) {
    if (V.Ntot > 0) k_rev_seed<<<(unsigned)((V.Ntot + NT - 1) / NT), NT, 0, Su(st)>>>(V, R);
}
void launch_rev_finish(const DevView& V, const RevArgs& R, void* st) {
    if (V.Ntot > 0) k_rev_finish<<<(unsigned)((V.Ntot + NT - 1) / NT), NT, 0, Su(st)>>>(V, R);
}

}  // namespace hsde
