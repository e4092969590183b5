// Cone projection of the clique blocks (Eq. Step2 on S = S_1 x ... x S_p)
// fused with the gather x_k = H_k x (Section 3.1), the rank-one correction of
// Eq. MatrixInverseResult on the s and v blocks, and the nu update of
// Eq. Step3 (z <- z - s_hat + s).
//
// For clique k, with xh = x_w - eta x_p gathered through H_k (the corrected
// x_hat of the affine step) and the over-relaxation alpha (1: the literal
// Eqs. Step2-Step3):
//   s_hat = (s + z - v + H_k xh)/2,  v_hat = (s + z + v - H_k xh)/2
//   a     = alpha s_hat + (1 - alpha) s - z   (the point projected in Eq. Step2)
//   s     = Pi_psd(a) = V max(Lambda, 0) V^T
//   z     = s - a,   v = alpha v_hat + (1 - alpha) v
// and the stopping-rule partial ||H_k x_new - s||^2 (full-vec weights), with
// x_new = alpha xh + (1 - alpha) x (x is still the previous iterate here).
//
// Eigensolver: two-sided cyclic Jacobi (symmetric Schur decomposition by 2x2
// rotations, Golub & Van Loan) with a parallel round-robin ordering.  The
// matrix is padded to CP (the bucket's size, a compile-time constant) with
// zero rows/columns that are never rotated.  Rows and columns live in "slots":
// in every round slot pair (2k, 2k+1) is rotated, and the result of each 2x2
// block J_r^T X J_c is written straight to the slots those indices occupy in
// the next round (ping-pong buffers), following the circle tournament
// (slot 0 fixed, the others advance one place), so every index pair meets
// once per sweep.  Only the lower triangle of A is kept: the blocks with
// row pair >= column pair are rotated, and each result goes to its lower
// position in the next round's slots.  V is stored slot-major (row = slot,
// column = original index), so a rotation mixes two rows and every access
// is a coalesced 2-vector; no permutation has to be tracked:
// s = V max(diag A, 0) V^T with V(i, slot) = Vs[slot][i].
// Warm start: V of the previous iteration (per clique, FP32/FP64 as the
// clique arrays) seeds the next solve through A <- V^T A V; every `refresh`
// iterations one Newton-Schulz step V <- V (3I - V^T V)/2 first restores the
// orthogonality that rounding erodes from one iteration to the next.
//
// A group of G threads owns one clique; groups never wait on each other
// (sub-warp shuffles for G < 32, named barriers for G > 32).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include "cone_common.cuh"
#include "internal.h"

namespace hsde {

// Row stride of the CP x LD buffers: even (2-vector accesses stay aligned),
// chosen per bucket size to spread a round's accesses over the 32 banks.  A
// warp's items run along a row and then jump by two rows, so 2 LD mod 32
// decides the conflicts between rows; the values below minimise the
// wavefronts of a whole round (A loads and scattered stores, V loads and
// stores) in a count over every warp's addresses.  Small buckets (several
// cliques per warp) keep CP + 2.
constexpr int cone_ld_spread(int cp) {
    switch (cp) {
        case 20: return 26;
        case 24: return 28;
        case 32: return 44;
        case 36: return 50;
        case 40: return 52;
        case 44: return 54;
        case 48: return 56;
        case 56: return 60;
        case 64: return 76;
        case 80: return 88;
        case 96: return 108;
        case 112: return 120;
        default: return cp + 2;
    }
}

template <typename T>
constexpr size_t cone_group_bytes(int cp, int ld) {
    // per group: A0, A1, V0, V1 (CP x LD), rot (cs,sn) K, tan K, lambda CP, red
    // (one double per warp of the group, whatever T is: 64 elements), and
    // the list of slots with a positive eigenvalue (CP + 1 ints)
    return ((4 * (size_t)cp * ld + 2 * (cp / 2) + cp / 2 + cp + 64 + (cp + 2)) * sizeof(T) + 15) / 16 * 16;
}

// Half the opt-in shared memory: two one-clique CTAs still share an SM.
constexpr size_t CONE_SMEM_HALF = 232448 / 2;

template <typename T, int CP, int G>
constexpr int cone_ld() {
    const int nth = (G > 32) ? G : 128;
    const size_t base = (size_t)(nth / G) * cone_group_bytes<T>(CP, CP + 2);
    const size_t spread = (size_t)(nth / G) * cone_group_bytes<T>(CP, cone_ld_spread(CP));
    // keep CP + 2 where the wider rows would lose the bucket its second
    // resident CTA or no longer fit
    if (spread > 232448 || (base <= CONE_SMEM_HALF && spread > CONE_SMEM_HALF)) return CP + 2;
    return cone_ld_spread(CP);
}

template <typename T, int CP_, int G_>
struct ConeCfg {
    static constexpr int CP = CP_;
    static constexpr int G = G_;
    static constexpr int K = CP / 2;
    static constexpr int LD = cone_ld<T, CP_, G_>();
    static_assert(LD % 2 == 0 && LD >= CP + 2, "even row stride beyond the padded size");
    static constexpr int NTH = (G > 32) ? G : 128;    // threads per CTA
    static constexpr int GPB = NTH / G;               // groups (cliques) per CTA
    static constexpr int NBLK = K * (K + 1) / 2;      // lower 2x2 blocks (row pair >= column pair)
    static constexpr int BPL = (NBLK + G - 1) / G;    // 2x2 blocks per thread per round
    static constexpr int NVP = K * K;                 // V items: slot pair x column pair
    static constexpr int VPL = (NVP + G - 1) / G;     // V items per thread per round
    static_assert(G <= 32 ? (32 % G == 0) : (G % 32 == 0), "group: a power of two <= 32 or whole warps");
    static_assert(BPL <= 32 && VPL <= 32, "per-thread masks are 32 bits");
    static_assert((G + 31) / 32 * sizeof(double) <= 64 * sizeof(T), "red holds one double per warp");
    static_assert((4 * CP * LD + 3 * K + CP) % 2 == 0, "red is 8-byte aligned");
    static constexpr size_t group_bytes = cone_group_bytes<T>(CP, LD);
    static constexpr size_t smem = GPB * group_bytes;
    // resident CTAs the register budget is sized for: many-clique CTAs 8;
    // one clique per CTA 2 where two fit the shared memory (the kernel waits
    // on barriers and shared memory, so a second CTA hides that latency),
    // else 1
    static constexpr int MINB = GPB > 1 ? 8 : (2 * smem <= 232448 && NTH <= 512 ? 2 : 1);
};

template <typename T> struct Vec2;
template <> struct Vec2<float> { using type = float2; };
template <> struct Vec2<double> { using type = double2; };

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
__device__ __forceinline__ void gsync(int gid) {
    if constexpr (G <= 32) {
        __syncwarp(gmask<G>());
    } else {
        asm volatile("bar.sync %0, %1;" ::"r"(gid + 1), "r"(G) : "memory");
    }
}

// Lanes of the fixed-order sums: a bucket's variants (different group sizes
// G) must give bitwise the same results, so the reductions whose rounding
// reaches the output (the convergence test, the clique's residual partials)
// run in an order set by the bucket size alone.
template <int CP>
struct FixedLanes {
    static constexpr int value = CP >= 20 ? 32 : 4;
};

// Sum of vals[0..n) (shared memory) in an order independent of G: lane
// l < RW adds vals[l], vals[l + RW], ... in turn, then the RW lanes combine
// by a butterfly.  Every thread of the group gets the result.  RW <= G.
template <int G, int RW, typename S>
__device__ __forceinline__ S fixed_sum(const S* vals, int n, S* red, int gid) {
    static_assert(RW <= 32 && (RW & (RW - 1)) == 0, "RW: a power of two <= 32");
    static_assert(G >= RW, "the group has the RW lanes");
    const int lane = threadIdx.x % G;
    const int base = (G >= 32) ? 0 : ((threadIdx.x & 31) & ~(G - 1));
    S v = S(0);
    if (lane < RW) {
        for (int i = lane; i < n; i += RW) v += vals[i];
        const unsigned m = (RW == 32) ? 0xffffffffu : (((1u << RW) - 1u) << base);
#pragma unroll
        for (int o = RW / 2; o > 0; o >>= 1) v += __shfl_xor_sync(m, v, o);
    }
    if constexpr (G <= 32) {
        return __shfl_sync(gmask<G>(), v, base);
    } else {
        gsync<G>(gid);
        if (lane == 0) red[0] = v;
        gsync<G>(gid);
        const S t = red[0];
        gsync<G>(gid);
        return t;
    }
}

// Circle-tournament slot map: slot 0 stays, the others advance along
// T1 -> T2 -> ... -> T(K-1) -> B(K-1) -> ... -> B0 -> T1  (Tk = 2k, Bk = 2k+1).
template <int CP>
__device__ __forceinline__ int sigma(int j) {
    constexpr int K = CP / 2;
    if (j == 0) return 0;
    const int k = j >> 1;
    if (j & 1) return k == 0 ? 2 : j - 2;
    return k == K - 1 ? j + 1 : j + 2;
}

// Jacobi rotation (c, s, t = s/c) that zeroes a_pq of the 2x2 block
// [[a_pp, a_pq], [a_pq, a_qq]] (Golub & Van Loan, symmetric Schur 2x2):
// theta = (a_qq - a_pp) / (2 a_pq), t = sign(theta) / (|theta| + sqrt(1 + theta^2)).
// FP32 uses the approximate divide, reciprocal and reciprocal square root
// instructions for t: the update applies c = 1/sqrt(1 + t^2) and s = t c as
// computed, so their error only perturbs the angle (a_pq is zeroed to
// ~1e-7 relative, which the update drops), not the orthogonality of the
// rotation.  For |theta| > 1e18, sqrt(1 + theta^2) = |theta| in FP32.
__device__ __forceinline__ void rotation(float app, float aqq, float apq, float& cs, float& sn, float& t) {
    cs = 1.f; sn = 0.f; t = 0.f;
    if (apq != 0.f) {
        const float theta = __fdividef(aqq - app, 2.f * apq);
        const float at = fabsf(theta);
        const float q = fmaf(theta, theta, 1.f);
        const float r = at < 1e18f ? q * rsqrtf(q) : at;
        t = __fdividef(1.f, at + r);
        if (theta < 0.f) t = -t;
        cs = rsqrtf(fmaf(t, t, 1.f));
        sn = t * cs;
    }
}
__device__ __forceinline__ void rotation(double app, double aqq, double apq, double& cs, double& sn, double& t) {
    cs = 1.0; sn = 0.0; t = 0.0;
    if (apq != 0.0) {
        const double theta = (aqq - app) / (2.0 * apq);
        t = 1.0 / (fabs(theta) + sqrt(1.0 + theta * theta));
        if (theta < 0.0) t = -t;
        cs = 1.0 / sqrt(1.0 + t * t);
        sn = t * cs;
    }
}

// Products and FMAs with the rounding fixed by the source (no contraction
// left to the compiler), so that the register-V and shared-memory variants
// of a bucket update V with bitwise the same arithmetic.
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float fma_rn(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fma_rn(double a, double b, double c) { return __fma_rn(a, b, c); }

// The rotation (c, s) of one slot pair applied to the pair's entries (v0, v1)
// of one column of V: (c v0 - s v1, s v0 + c v1).
template <typename T>
__device__ __forceinline__ void rot_pair(T c, T s, T v0, T v1, T& n0, T& n1) {
    n0 = fma_rn(-s, v1, mul_rn(c, v0));
    n1 = fma_rn(s, v0, mul_rn(c, v1));
}

// Offsets (in elements of one CP x LD buffer) a thread uses in every round.
// The thread-to-block assignment does not change between rounds, so the
// tournament map is evaluated once per solve, not once per round.
template <int LD>
__device__ __forceinline__ int lower_pos(int r, int c) {
    return r >= c ? r * LD + c : c * LD + r;
}

template <typename Cfg>
struct RoundPlan {
    int a_src[Cfg::BPL];       // top-left of the 2x2 block (rows 2kr, 2kr+1; cols 2kc, 2kc+1), kr >= kc
    int a_dst[Cfg::BPL][4];    // lower positions of (r0,c0) (r0,c1) (r1,c0) (r1,c1) in the next slots
    int rot_r[Cfg::BPL], rot_c[Cfg::BPL];
    int v_src[Cfg::VPL], v_dst0[Cfg::VPL], v_dst1[Cfg::VPL], v_rot[Cfg::VPL];
    unsigned diag_mask, a_valid, v_valid;

    __device__ __forceinline__ void build(int lane) {
        constexpr int CP = Cfg::CP, K = Cfg::K, LD = Cfg::LD, G = Cfg::G;
        diag_mask = 0u; a_valid = 0u; v_valid = 0u;
#pragma unroll
        for (int i = 0; i < Cfg::BPL; ++i) {
            int b = lane + i * G;
            if (b < Cfg::NBLK) a_valid |= 1u << i;
            else b = 0;
            int kr = 0;
            while ((kr + 1) * (kr + 2) / 2 <= b) ++kr;
            const int kc = b - kr * (kr + 1) / 2;
            const int r0 = sigma<CP>(2 * kr), r1 = sigma<CP>(2 * kr + 1);
            const int c0 = sigma<CP>(2 * kc), c1 = sigma<CP>(2 * kc + 1);
            a_src[i] = (2 * kr) * LD + 2 * kc;
            a_dst[i][0] = lower_pos<LD>(r0, c0);
            a_dst[i][1] = lower_pos<LD>(r0, c1);
            a_dst[i][2] = lower_pos<LD>(r1, c0);
            a_dst[i][3] = lower_pos<LD>(r1, c1);
            rot_r[i] = 2 * kr;
            rot_c[i] = 2 * kc;
            if (kr == kc) diag_mask |= 1u << i;
        }
#pragma unroll
        for (int i = 0; i < Cfg::VPL; ++i) {
            int b = lane + i * G;
            if (b < Cfg::NVP) v_valid |= 1u << i;
            else b = 0;
            const int kp = b / K, col = 2 * (b - (b / K) * K);
            v_src[i] = (2 * kp) * LD + col;
            v_dst0[i] = sigma<CP>(2 * kp) * LD + col;
            v_dst1[i] = sigma<CP>(2 * kp + 1) * LD + col;
            v_rot[i] = 2 * kp;
        }
    }
};

// Block i of a thread's round plan: J_r^T X J_c of the 2 x 2 block X (rows
// 2kr, 2kr+1; columns 2kc, 2kc+1), written to its slots of the next round.
// A diagonal block keeps its lower triangle: a_pp - t a_pq, 0, a_qq + t a_pq.
template <typename Cfg, typename T>
__device__ __forceinline__ void update_block(const RoundPlan<Cfg>& pl, int i, const T* __restrict__ A,
                                             T* __restrict__ An, const T* __restrict__ rot,
                                             const T* __restrict__ tan_) {
    constexpr int LD = Cfg::LD;
    using V2 = typename Vec2<T>::type;
    const V2 top = *reinterpret_cast<const V2*>(A + pl.a_src[i]);
    const V2 bot = *reinterpret_cast<const V2*>(A + pl.a_src[i] + LD);
    if (pl.diag_mask & (1u << i)) {
        // top.y lies above the diagonal (not kept); a_pq = bot.x
        const T t = tan_[pl.rot_r[i] >> 1];
        const T apq = bot.x;
        An[pl.a_dst[i][0]] = fma_rn(-t, apq, top.x);
        An[pl.a_dst[i][1]] = (t == T(0)) ? apq : T(0);
        An[pl.a_dst[i][3]] = fma_rn(t, apq, bot.y);
    } else {
        const V2 rr = *reinterpret_cast<const V2*>(rot + pl.rot_r[i]);
        const V2 rc = *reinterpret_cast<const V2*>(rot + pl.rot_c[i]);
        T y00, y01, y10, y11, d0, d1, d2, d3;
        rot_pair(rr.x, rr.y, top.x, bot.x, y00, y10);    // J_r^T X, first column
        rot_pair(rr.x, rr.y, top.y, bot.y, y01, y11);    // second column
        rot_pair(rc.x, rc.y, y00, y01, d0, d1);          // (.) J_c, first row
        rot_pair(rc.x, rc.y, y10, y11, d2, d3);          // second row
        An[pl.a_dst[i][0]] = d0;
        An[pl.a_dst[i][1]] = d1;
        An[pl.a_dst[i][2]] = d2;
        An[pl.a_dst[i][3]] = d3;
    }
}

template <typename Cfg, typename T>
__device__ __forceinline__ void jacobi_round(const RoundPlan<Cfg>& pl, const T* __restrict__ A,
                                             T* __restrict__ An, const T* __restrict__ Vc, T* __restrict__ Vn,
                                             T* __restrict__ rot, T* __restrict__ tan_, int lane, int gid) {
    constexpr int K = Cfg::K, LD = Cfg::LD, G = Cfg::G;
    using V2 = typename Vec2<T>::type;
    // rotation of every slot pair (2k, 2k+1), from the lower triangle
    if (lane < K) {
        const int k = lane;
        const T app = A[(2 * k) * LD + 2 * k];
        const V2 qrow = *reinterpret_cast<const V2*>(A + (2 * k + 1) * LD + 2 * k);   // (a_qp, a_qq)
        T cs, sn, t;
        rotation(app, qrow.y, qrow.x, cs, sn, t);
        V2 cssn;
        cssn.x = cs;
        cssn.y = sn;
        *reinterpret_cast<V2*>(rot + 2 * k) = cssn;
        tan_[k] = t;
    }
    gsync<G>(gid);
#pragma unroll
    for (int i = 0; i < Cfg::BPL; ++i) {
        if ((Cfg::NBLK % G != 0) && !(pl.a_valid & (1u << i))) continue;
        update_block(pl, i, A, An, rot, tan_);
    }
#pragma unroll
    for (int i = 0; i < Cfg::VPL; ++i) {
        if ((Cfg::NVP % G != 0) && !(pl.v_valid & (1u << i))) continue;
        const V2 rc = *reinterpret_cast<const V2*>(rot + pl.v_rot[i]);
        const V2 v0 = *reinterpret_cast<const V2*>(Vc + pl.v_src[i]);
        const V2 v1 = *reinterpret_cast<const V2*>(Vc + pl.v_src[i] + LD);
        V2 n0, n1;
        rot_pair(rc.x, rc.y, v0.x, v1.x, n0.x, n1.x);
        rot_pair(rc.x, rc.y, v0.y, v1.y, n0.y, n1.y);
        *reinterpret_cast<V2*>(Vn + pl.v_dst0[i]) = n0;
        *reinterpret_cast<V2*>(Vn + pl.v_dst1[i]) = n1;
    }
    gsync<G>(gid);
}

// Slot c_i of the circle-tournament cycle: 1 -> 2 -> 4 -> ... -> CP-2 ->
// CP-1 -> CP-3 -> ... -> 3 -> 1 (slot 0 stays), so sigma(c_i) = c_(i+1).
template <int CP>
__device__ __forceinline__ int cycle_slot(int i) {
    constexpr int K = CP / 2;
    return i == 0 ? 1 : (i < K ? 2 * i : 4 * K - 1 - 2 * i);
}

// One round of the register-V variant.  The A-threads (is_a; the plan is
// theirs) compute the rotations and update A as in jacobi_round; each
// V-thread holds one column of V (all CP slots) in registers, applies the
// round's K rotations and then the slot permutation sigma, moving values
// along the one cycle of sigma (register moves, no shared memory).
template <typename PCfg, int GT, typename T>
__device__ __forceinline__ void jacobi_round_rv(const RoundPlan<PCfg>& pl, const T* __restrict__ A,
                                                T* __restrict__ An, T* __restrict__ rot, T* __restrict__ tan_,
                                                int alane, bool is_a, T (&vr)[PCfg::CP], int gid) {
    constexpr int CP = PCfg::CP, K = PCfg::K, LD = PCfg::LD, G = PCfg::G;
    using V2 = typename Vec2<T>::type;
    if (is_a && alane < K) {
        const int k = alane;
        const T app = A[(2 * k) * LD + 2 * k];
        const V2 qrow = *reinterpret_cast<const V2*>(A + (2 * k + 1) * LD + 2 * k);
        T cs, sn, t;
        rotation(app, qrow.y, qrow.x, cs, sn, t);
        V2 cssn;
        cssn.x = cs;
        cssn.y = sn;
        *reinterpret_cast<V2*>(rot + 2 * k) = cssn;
        tan_[k] = t;
    }
    gsync<GT>(gid);
    if (is_a) {
#pragma unroll
        for (int i = 0; i < PCfg::BPL; ++i) {
            if ((PCfg::NBLK % G != 0) && !(pl.a_valid & (1u << i))) continue;
            update_block(pl, i, A, An, rot, tan_);
        }
    } else {
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const V2 cs = *reinterpret_cast<const V2*>(rot + 2 * k);
            T n0, n1;
            rot_pair(cs.x, cs.y, vr[2 * k], vr[2 * k + 1], n0, n1);
            vr[2 * k] = n0;
            vr[2 * k + 1] = n1;
        }
        const T last = vr[cycle_slot<CP>(CP - 2)];
#pragma unroll
        for (int i = CP - 2; i >= 1; --i) vr[cycle_slot<CP>(i)] = vr[cycle_slot<CP>(i - 1)];
        vr[cycle_slot<CP>(0)] = last;
    }
    gsync<GT>(gid);
}

// Entry (i, j), i >= j, of the synthetic symmetric matrix of clique k that
// the autotuner's dry runs diagonalise: a hash of (k, i, j) mapped to
// [-1, 1], the diagonal shifted by i / c so that the spectrum is spread.
template <typename T>
__device__ __forceinline__ T dry_entry(int k, int i, int j) {
    uint32_t h = (uint32_t)k * 0x9E3779B1u ^ (uint32_t)(i * 0x85EBCA77u) ^ (uint32_t)(j * 0xC2B2AE3Du);
    h ^= h >> 16;
    h *= 0x7FEB352Du;
    h ^= h >> 15;
    h *= 0x846CA68Bu;
    h ^= h >> 16;
    const T u = T((double)(h >> 8) * (2.0 / 16777216.0) - 1.0);
    return i == j ? u + T(i) * T(0.05) : u;
}

// MB: resident CTAs the registers are sized for (ConeCfg::MINB, or 1 for a
// bucket whose CTAs each have an SM to themselves); ST: one-clique CTAs may
// keep the gathered values in registers until the rebuild (the latency
// variants) instead of re-reading them (the throughput variants, whose
// registers go to more resident CTAs).  dry != 0 (autotuning): a
// deterministic synthetic matrix instead of the gather, a cold start,
// exactly max_sweeps sweeps, and no global writes.
// Register-V variant (VR): of the G threads, the last GV = 32 ceil(CP / 32)
// each hold one column of V in registers through the sweeps (no shared-
// memory traffic for V), the first G - GV (the A-threads) update A; every
// other phase runs on all G threads as in the other variants.
template <int CP, int G, bool VR>
struct RegV {
    static constexpr int GV = VR ? (CP + 31) / 32 * 32 : 0;
    static constexpr int GA = G - GV;
};

template <typename T, int CP, int G, int MB, bool ST, bool VR>
__global__ void __launch_bounds__(ConeCfg<T, CP, G>::NTH, MB)
k_cone(DevView V, const int32_t* __restrict__ list, int nlist, int max_sweeps, T tol2, int warm, int refresh,
       int dry) {
    using Cfg = ConeCfg<T, CP, G>;
    constexpr int GA = RegV<CP, G, VR>::GA;
    static_assert(!VR || (G > 32 && GA >= 32 && GA % 32 == 0), "register-V: whole warps of each kind");
    // the round plan's configuration: the A-threads' (all threads without VR)
    using PCfg = ConeCfg<T, CP, VR ? GA : G>;
    static_assert(PCfg::LD == Cfg::LD, "the plan indexes the buffers with their row stride");
    using V2 = typename Vec2<T>::type;
    constexpr int LD = Cfg::LD, K = Cfg::K;
    constexpr int EPT = (CP * (CP + 1) / 2 + G - 1) / G;   // lower entries per thread
    // One clique per CTA: the gathered values stay in registers until the
    // rebuild.  Groups of <= 32 lanes (many cliques per CTA) re-read them
    // instead, keeping registers, and so resident CTAs, as they were.
    constexpr bool STASH = ST && G > 32;
    constexpr int RW = FixedLanes<CP>::value;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int gid = threadIdx.x / G, lane = threadIdx.x % G;
    const int li = blockIdx.x * Cfg::GPB + gid;
    if (li >= nlist) return;
    const int k = list[li];
    const InstDev& I = V.inst[V.cl_inst[k]];
    if (I.status != HSDE_RUNNING) return;

    T* A0 = reinterpret_cast<T*>(smem_raw + (size_t)gid * Cfg::group_bytes);
    T* A1 = A0 + CP * LD;
    T* V0 = A1 + CP * LD;
    T* V1 = V0 + CP * LD;
    T* rot = V1 + CP * LD;
    T* tan_ = rot + 2 * K;
    T* lam = tan_ + K;
    T* red = lam + CP;
    int* pos = reinterpret_cast<int*>(red + 64);   // positive eigenvalues (slots), count at [CP]

    T* s = reinterpret_cast<T*>(V.s);
    T* z = reinterpret_cast<T*>(V.z);
    T* v = reinterpret_cast<T*>(V.v);
    const int c = V.cl_size[k];
    const int nlow = c * (c + 1) / 2;
    const int64_t off = V.cl_off[k];
    const double eta = I.eta;
    const double al = V.alpha;
    T* Vst = V.vstore ? reinterpret_cast<T*>(V.vstore) + V.vs_off[k] : nullptr;
    const bool use_warm = !dry && warm && Vst != nullptr && !I.vcold;
    // every refresh-th iteration the stored basis, whose orthogonality
    // drifts by rounding from one iteration to the next, gets one
    // Newton-Schulz step V <- V (3I - V^T V) / 2 before use
    const bool reorth = use_warm && refresh > 0 && (I.iter % refresh) == (1 % refresh);

    // The stored basis is read with all of a thread's loads in flight at
    // once (they are issued before any shared-memory store); zero A0
    // (padding included) and set V0 = I or the stored basis (slot-major).
    constexpr int IPT = (CP * CP + G - 1) / G;
    T vst[IPT];
#pragma unroll
    for (int q = 0; q < IPT; ++q) {
        const int idx = lane + q * G;
        vst[q] = (use_warm && idx < CP * CP) ? Vst[idx] : T(0);
    }
    // With STASH each thread keeps its lower entries' a, H_k xh and v_hat in
    // registers until the rebuild writes s, z, v; their first loads are
    // issued here too.
    int apos[STASH ? EPT : 1];   // arow * LD + bcol; -1: no entry
    unsigned diag_bits = 0u;
    T avs[STASH ? EPT : 1], gxs[STASH ? EPT : 1];
    T vns[STASH ? EPT : 1];
    int gi[STASH ? EPT : 1];
    T so[STASH ? EPT : 1], zo[STASH ? EPT : 1], vo[STASH ? EPT : 1];
    if constexpr (STASH) {
#pragma unroll
        for (int q = 0; q < EPT; ++q) {
            const int e = lane + q * G;
            apos[q] = -1;
            if (e < nlow) {
                const int b = packed_column(e, c);
                const int arow = b + (e - (b * c - b * (b - 1) / 2));
                apos[q] = arow * LD + b;
                if (arow == b) diag_bits |= 1u << q;
                gi[q] = V.gmap[off + e];
                so[q] = s[off + e];
                zo[q] = z[off + e];
                vo[q] = v[off + e];
            }
        }
    }
#pragma unroll
    for (int q = 0; q < IPT; ++q) {
        const int idx = lane + q * G;
        if (idx < CP * CP) {
            const int i = idx / CP, j = idx - (idx / CP) * CP;
            A0[i * LD + j] = T(0);
            V0[i * LD + j] = use_warm ? vst[q] : ((i == j) ? T(1) : T(0));
        }
    }
    // Gather + rank-one correction, a = s_hat - z, over the lower entries
    // (packed order e = j - off).
    if constexpr (STASH) {
        gsync<G>(gid);   // A0 zeroed
#pragma unroll
        for (int q = 0; q < EPT; ++q) {
            if (apos[q] < 0) continue;
            const double gx = V.xw[gi[q]] - eta * V.xp[gi[q]];
            T av, vn, hx;
            cone_inputs<T>(so[q], zo[q], vo[q], (T)gx, (T)al, V.x, gi[q], av, vn, hx);
            gxs[q] = hx;
            avs[q] = av;
            vns[q] = vn;
            const int arow = apos[q] / LD, b = apos[q] - (apos[q] / LD) * LD;
            const T a = dry ? dry_entry<T>(k, arow, b) : (T)av;
            A0[apos[q]] = a;
            A0[b * LD + arow] = a;
        }
    } else {
        gsync<G>(gid);   // A0 zeroed
        for (int e = lane; e < nlow; e += G) {
            const int b = packed_column(e, c);
            const int arow = b + (e - (b * c - b * (b - 1) / 2));
            const int gi = V.gmap[off + e];
            const double gx = V.xw[gi] - eta * V.xp[gi];
            T av, vn, hx;
            cone_inputs<T>(s[off + e], z[off + e], v[off + e], (T)gx, (T)al, V.x, gi, av, vn, hx);
            const T a = dry ? dry_entry<T>(k, arow, b) : (T)av;
            A0[arow * LD + b] = a;
            A0[b * LD + arow] = a;
        }
    }
    gsync<G>(gid);
    T* A = A0;
    T* An = A1;
    T* Vc = V0;
    T* Vn = V1;
    const bool is_a = !VR || lane < GA;
    RoundPlan<PCfg> plan;
    plan.build(is_a ? lane : 0);
    const int cq = (c + 1) & ~1;   // A and its products vanish beyond c
    if (reorth) {
        // Gram matrix G = V^T V (slot x slot) into An, 2 x 2 tiles over all CP
        // rows (the padding slots' unit vectors included)
        for (int tix = lane; tix < K * K; tix += G) {
            const int ts = tix / K, tt = tix - (tix / K) * K;
            T g00 = 0, g01 = 0, g10 = 0, g11 = 0;
            for (int q = 0; q < CP; q += 2) {
                const V2 a0 = *reinterpret_cast<const V2*>(Vc + (2 * ts) * LD + q);
                const V2 a1 = *reinterpret_cast<const V2*>(Vc + (2 * ts + 1) * LD + q);
                const V2 b0 = *reinterpret_cast<const V2*>(Vc + (2 * tt) * LD + q);
                const V2 b1 = *reinterpret_cast<const V2*>(Vc + (2 * tt + 1) * LD + q);
                g00 += a0.x * b0.x + a0.y * b0.y;
                g01 += a0.x * b1.x + a0.y * b1.y;
                g10 += a1.x * b0.x + a1.y * b0.y;
                g11 += a1.x * b1.x + a1.y * b1.y;
            }
            V2 r0, r1;
            r0.x = g00; r0.y = g01; r1.x = g10; r1.y = g11;
            *reinterpret_cast<V2*>(An + (2 * ts) * LD + 2 * tt) = r0;
            *reinterpret_cast<V2*>(An + (2 * ts + 1) * LD + 2 * tt) = r1;
        }
        gsync<G>(gid);
        // slot-major: V_s <- 1.5 V_s - 0.5 G V_s
        for (int tix = lane; tix < K * K; tix += G) {
            const int ts = tix / K, ti = tix - (tix / K) * K;
            T p00 = 0, p01 = 0, p10 = 0, p11 = 0;
            for (int j = 0; j < CP; j += 2) {
                const V2 g0 = *reinterpret_cast<const V2*>(An + (2 * ts) * LD + j);
                const V2 g1 = *reinterpret_cast<const V2*>(An + (2 * ts + 1) * LD + j);
                const V2 v0 = *reinterpret_cast<const V2*>(Vc + j * LD + 2 * ti);
                const V2 v1 = *reinterpret_cast<const V2*>(Vc + (j + 1) * LD + 2 * ti);
                p00 += g0.x * v0.x + g0.y * v1.x;
                p01 += g0.x * v0.y + g0.y * v1.y;
                p10 += g1.x * v0.x + g1.y * v1.x;
                p11 += g1.x * v0.y + g1.y * v1.y;
            }
            const V2 c0 = *reinterpret_cast<const V2*>(Vc + (2 * ts) * LD + 2 * ti);
            const V2 c1 = *reinterpret_cast<const V2*>(Vc + (2 * ts + 1) * LD + 2 * ti);
            V2 n0, n1;
            n0.x = T(1.5) * c0.x - T(0.5) * p00;
            n0.y = T(1.5) * c0.y - T(0.5) * p01;
            n1.x = T(1.5) * c1.x - T(0.5) * p10;
            n1.y = T(1.5) * c1.y - T(0.5) * p11;
            *reinterpret_cast<V2*>(Vn + (2 * ts) * LD + 2 * ti) = n0;
            *reinterpret_cast<V2*>(Vn + (2 * ts + 1) * LD + 2 * ti) = n1;
        }
        gsync<G>(gid);
        T* t2 = Vc; Vc = Vn; Vn = t2;
    }
    if (use_warm) {
        // An = V^T A (slot x original; A symmetric and full), 2 x 2 tiles
        for (int tix = lane; tix < K * K; tix += G) {
            const int ts = tix / K, ti = tix - (tix / K) * K;
            T a00 = 0, a01 = 0, a10 = 0, a11 = 0;
            for (int q = 0; q < cq; q += 2) {
                const V2 v0 = *reinterpret_cast<const V2*>(Vc + (2 * ts) * LD + q);
                const V2 v1 = *reinterpret_cast<const V2*>(Vc + (2 * ts + 1) * LD + q);
                const V2 x0 = *reinterpret_cast<const V2*>(A + (2 * ti) * LD + q);
                const V2 x1 = *reinterpret_cast<const V2*>(A + (2 * ti + 1) * LD + q);
                a00 += v0.x * x0.x + v0.y * x0.y;
                a01 += v0.x * x1.x + v0.y * x1.y;
                a10 += v1.x * x0.x + v1.y * x0.y;
                a11 += v1.x * x1.x + v1.y * x1.y;
            }
            V2 r0, r1;
            r0.x = a00; r0.y = a01; r1.x = a10; r1.y = a11;
            *reinterpret_cast<V2*>(An + (2 * ts) * LD + 2 * ti) = r0;
            *reinterpret_cast<V2*>(An + (2 * ts + 1) * LD + 2 * ti) = r1;
        }
        gsync<G>(gid);
        // lower triangle of A = An V, 2 x 2 tiles (the round plan's blocks)
#pragma unroll
        for (int i = 0; i < PCfg::BPL; ++i) {
            if (!is_a || ((PCfg::NBLK % PCfg::G != 0) && !(plan.a_valid & (1u << i)))) continue;
            const int r = plan.rot_r[i], cl = plan.rot_c[i];
            T a00 = 0, a01 = 0, a10 = 0, a11 = 0;
            for (int q = 0; q < cq; q += 2) {
                const V2 x0 = *reinterpret_cast<const V2*>(An + r * LD + q);
                const V2 x1 = *reinterpret_cast<const V2*>(An + (r + 1) * LD + q);
                const V2 v0 = *reinterpret_cast<const V2*>(Vc + cl * LD + q);
                const V2 v1 = *reinterpret_cast<const V2*>(Vc + (cl + 1) * LD + q);
                a00 += x0.x * v0.x + x0.y * v0.y;
                a01 += x0.x * v1.x + x0.y * v1.y;
                a10 += x1.x * v0.x + x1.y * v0.y;
                a11 += x1.x * v1.x + x1.y * v1.y;
            }
            A[r * LD + cl] = a00;
            A[(r + 1) * LD + cl] = a10;
            A[(r + 1) * LD + cl + 1] = a11;
            if (r != cl) A[r * LD + cl + 1] = a01;
        }
        gsync<G>(gid);
    }

    // register-V: each V-thread takes its column of V (slot-major in Vc)
    T vr[VR ? CP : 1];
    if constexpr (VR) {
        const int col = lane - GA;
#pragma unroll
        for (int q = 0; q < CP; ++q) vr[q] = (!is_a && col < CP) ? Vc[q * LD + col] : T(0);
    }
    int sweeps_done = 0;
    bool converged = false;
    for (int sweep = 0; sweep <= max_sweeps; ++sweep) {
        sweeps_done = sweep;
        // per-row sums (row r: 2 sum_{j<r} a_rj^2 and a_rr^2) into the free
        // buffer An, then fixed-order sums over the rows
        for (int r = lane; r < CP; r += G) {
            T o = T(0);
            for (int j = 0; j < r; ++j) {
                const T a = A[r * LD + j];
                o += a * a;
            }
            const T d = A[r * LD + r];
            An[r] = T(2) * o;
            An[CP + r] = d * d;
        }
        gsync<G>(gid);
        const T offd = fixed_sum<G, RW>(An, CP, red, gid);
        const T tot = fixed_sum<G, RW>(An + CP, CP, red, gid) + offd;
        converged = offd <= tol2 * tot;
        if ((converged && !dry) || sweep == max_sweeps) break;
        for (int r = 0; r < CP - 1; ++r) {
            if constexpr (VR) {
                jacobi_round_rv<PCfg, G>(plan, A, An, rot, tan_, lane, is_a, vr, gid);
            } else {
                jacobi_round<Cfg>(plan, A, An, Vc, Vn, rot, tan_, lane, gid);
                T* t2 = Vc; Vc = Vn; Vn = t2;
            }
            T* t1 = A; A = An; An = t1;
        }
    }
    if constexpr (VR) {
        // the V columns back to shared memory (slot-major) for what follows
        const int col = lane - GA;
        if (!is_a && col < CP) {
#pragma unroll
            for (int q = 0; q < CP; ++q) Vc[q * LD + col] = vr[q];
        }
        gsync<G>(gid);
    }
    if (V.tape_v && !dry) {
        // reverse-mode tape: eigenvectors (original index x slot) and raw eigenvalues
        T* tv = reinterpret_cast<T*>(V.tape_v) + V.tv_off[k];
        for (int idx = lane; idx < CP * CP; idx += G) {
            const int i = idx / CP, j = idx - (idx / CP) * CP;
            tv[idx] = Vc[j * LD + i];   // (original index i, slot j)
        }
        for (int i = lane; i < CP; i += G) tv[CP * CP + i] = A[i * LD + i];
    }
    for (int i = lane; i < CP; i += G) lam[i] = fmax(A[i * LD + i], T(0));
    if (Vst != nullptr && warm && !dry) {
        for (int idx = lane; idx < CP * CP; idx += G) {
            const int i = idx / CP, j = idx - (idx / CP) * CP;
            Vst[idx] = Vc[i * LD + j];
        }
    }
    // slots with a positive eigenvalue, in slot order (one warp, or the group)
    if constexpr (G >= 32) {
        if (lane < 32) {
            int base = 0;
            for (int c0 = 0; c0 < CP; c0 += 32) {
                const int i = c0 + lane;
                const bool pp = i < CP && A[i * LD + i] > T(0);
                const unsigned m = __ballot_sync(0xffffffffu, pp);
                if (pp) pos[base + __popc(m & ((1u << lane) - 1u))] = i;
                base += __popc(m);
            }
            if (lane == 0) pos[CP] = base;
        }
    } else {
        const unsigned gm = gmask<G>();
        const int sh = (threadIdx.x & 31) & ~(G - 1);
        int base = 0;
        for (int c0 = 0; c0 < CP; c0 += G) {
            const int i = c0 + lane;
            const bool pp = i < CP && A[i * LD + i] > T(0);
            const unsigned m = (__ballot_sync(gm, pp) & gm) >> sh;
            if (pp) pos[base + __popc(m & ((1u << lane) - 1u))] = i;
            base += __popc(m);
        }
        if (lane == 0) pos[CP] = base;
    }
    gsync<G>(gid);

    // s = V max(Lambda, 0) V^T on the lower triangle (2 x 2 tiles, positive
    // eigenvalues only), into the free buffer An
    const int npos = pos[CP];
#pragma unroll
    for (int i = 0; i < PCfg::BPL; ++i) {
        if (!is_a || ((PCfg::NBLK % PCfg::G != 0) && !(plan.a_valid & (1u << i)))) continue;
        const int r = plan.rot_r[i], cl = plan.rot_c[i];
        if (cl >= c) continue;
        T a00 = 0, a01 = 0, a10 = 0, a11 = 0;
        for (int t = 0; t < npos; ++t) {
            const int q = pos[t];
            const T w = lam[q];
            const V2 x = *reinterpret_cast<const V2*>(Vc + q * LD + r);
            const V2 y = *reinterpret_cast<const V2*>(Vc + q * LD + cl);
            const T wx0 = w * x.x, wx1 = w * x.y;
            a00 += wx0 * y.x;
            a01 += wx0 * y.y;
            a10 += wx1 * y.x;
            a11 += wx1 * y.y;
        }
        An[r * LD + cl] = a00;
        An[(r + 1) * LD + cl] = a10;
        An[(r + 1) * LD + cl + 1] = a11;
        if (r != cl) An[r * LD + cl + 1] = a01;
    }
    gsync<G>(gid);

    // each lower entry's contributions to ||H_k x - s_k||^2 and ||s_k||^2 go
    // to the free buffers A and Vn (nlow values each fit: LD > c) and are
    // summed in a fixed order
    T* cres = A;
    T* csres = Vn;
    if constexpr (STASH) {
#pragma unroll
        for (int q = 0; q < EPT; ++q) {
            if (apos[q] < 0) continue;
            const int e = lane + q * G;
            const int64_t j = off + e;
            const T sn = An[apos[q]];
            if (!dry) {
                s[j] = sn;
                z[j] = sn - avs[q];
                v[j] = vns[q];
            }
            const T d = gxs[q] - sn;
            const T w = (diag_bits >> q) & 1u ? T(1) : T(2);
            cres[e] = w * d * d;
            csres[e] = w * sn * sn;
        }
    } else {
        for (int e = lane; e < nlow; e += G) {
            const int b = packed_column(e, c);
            const int arow = b + (e - (b * c - b * (b - 1) / 2));
            const int64_t j = off + e;
            const T sn = An[arow * LD + b];
            const int gi = V.gmap[j];
            const double gx = V.xw[gi] - eta * V.xp[gi];
            T av, vn, hx;
            cone_inputs<T>(s[j], z[j], v[j], (T)gx, (T)al, V.x, gi, av, vn, hx);
            if (!dry) {
                s[j] = sn;
                z[j] = sn - av;
                v[j] = vn;
            }
            const T d = hx - sn;
            const T w = arow == b ? T(1) : T(2);
            cres[e] = w * d * d;
            csres[e] = w * sn * sn;
        }
    }
    gsync<G>(gid);
    const double res = (double)fixed_sum<G, RW>(cres, nlow, red, gid);
    const double sres = (double)fixed_sum<G, RW>(csres, nlow, red, gid);
    if (lane == 0 && !dry) {
        V.cl_part[2 * k] = res;
        V.cl_part[2 * k + 1] = sres;
        V.cl_sweeps[k] = sweeps_done;
        // an eigensolve that ran out of sweeps is counted, not hidden (the
        // projection is then only as accurate as its last sweep)
        if (!converged) atomicAdd(&V.inst[V.cl_inst[k]].unconv, 1);
    }
}

// ---------------------------------------------------------------------------
// buckets: padded size CP; threads per clique G of the latency variant, GT of
// the throughput variant and GR of the register-V variant (0: none)
// ---------------------------------------------------------------------------
// (padding a clique of c to CP costs about (CP/c)^3 of the work, so the
// sizes are spaced by 4 above 16.)  The latency variant gives about one 2x2
// block per thread and round (K(K+1)/2 blocks, K = CP/2) and keeps the
// gathered values in registers: the fastest solve of one clique.  The
// throughput variant gives about two blocks per thread, re-reads the
// gathered values, and is compiled for as many resident CTAs as the shared
// memory allows with ~72 registers a thread: more cliques per SM.  The
// register-V variant (FP32) adds a warp or two that hold V in registers
// through the sweeps, about three blocks per A-thread.  All give bitwise the
// same results (the same per-element arithmetic with its rounding fixed in
// the source, and sums in a fixed order).  Sizes above 64 hold one clique per
// CTA of up to 1024 threads; a size exists for a precision only if its CTA
// fits the opt-in shared memory (FP32 up to 112, FP64 up to 80).
#define HSDE_CONE_BUCKETS(X)                                                                          \
    X(4, 4, 0, 0) X(8, 8, 0, 0) X(12, 16, 0, 0) X(16, 32, 0, 0) X(20, 64, 32, 0) X(24, 96, 64, 64)   \
    X(28, 128, 64, 96) X(32, 160, 96, 96) X(36, 192, 96, 128) X(40, 224, 128, 160)                  \
    X(44, 256, 128, 160) X(48, 320, 160, 192) X(56, 416, 224, 224) X(64, 544, 288, 256)             \
    X(80, 832, 416, 0) X(96, 1024, 0, 0) X(112, 1024, 0, 0)

// Opt-in shared memory per CTA on this architecture (227 KB).
constexpr size_t CONE_SMEM_MAX = 232448;

template <typename T, int CP, int G>
constexpr bool cone_fits() {
    return ConeCfg<T, CP, G>::smem <= CONE_SMEM_MAX;
}

// Resident CTAs of a throughput variant: as many as the shared memory holds,
// at most 896 threads an SM (about 72 registers a thread).
template <typename T, int CP, int G>
constexpr int thr_minb() {
    using Cfg = ConeCfg<T, CP, G>;
    if (Cfg::GPB > 1) return 8;
    const int by_smem = (int)(CONE_SMEM_MAX / Cfg::smem);
    const int by_thr = 896 / Cfg::NTH;
    const int m = by_smem < by_thr ? by_smem : by_thr;
    return m < 1 ? 1 : (m > 16 ? 16 : m);
}

// Resident CTAs of a register-V variant: as many as the shared memory holds
// while every thread keeps CP + 48 registers (the V column or the A-thread's
// round plan, both live through the sweeps).  Each of the four SM
// sub-partitions has 16384 registers for the warps it holds.
template <typename T, int CP, int G>
constexpr int rv_minb() {
    using Cfg = ConeCfg<T, CP, G>;
    const int regs = (CP + 48 + 7) / 8 * 8;
    const int warps_per_smsp = 16384 / (32 * regs);
    const int by_regs = 4 * warps_per_smsp / (Cfg::NTH / 32);
    const int by_smem = (int)(CONE_SMEM_MAX / Cfg::smem);
    const int m = by_smem < by_regs ? by_smem : by_regs;
    return m < 1 ? 1 : (m > 16 ? 16 : m);
}

template <typename T, int GR>
constexpr bool has_rv() {
    return GR > 0 && sizeof(T) == 4;
}

// Device limits read by cone_prepare: opt-in shared memory per CTA, SMs.
static int g_smem_optin = 0;
static int g_num_sms = 0;

template <typename T, int CP, int G, int MB, bool ST, bool VR>
static cudaError_t allow_smem(int bytes) {
    if (bytes <= 48 * 1024) return cudaSuccess;
    return cudaFuncSetAttribute(k_cone<T, CP, G, MB, ST, VR>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

template <typename T, int CP, int G, int GT, int GR>
static int prepare_one() {
    if constexpr (!cone_fits<T, CP, G>()) {
        return HSDE_OK;                                          // never used in this precision
    } else {
        using Cfg = ConeCfg<T, CP, G>;
        // one clique per CTA: allowed the whole opt-in shared memory, which a
        // launch asks for when the bucket has few cliques (a CTA alone on its SM)
        const int want = Cfg::GPB == 1 ? std::max<int>(g_smem_optin, (int)Cfg::smem) : (int)Cfg::smem;
        if (allow_smem<T, CP, G, Cfg::MINB, true, false>(want) != cudaSuccess) return HSDE_ECUDA;
        if constexpr (Cfg::GPB == 1 && CP >= 32 && Cfg::MINB != 1) {
            if (allow_smem<T, CP, G, 1, true, false>(want) != cudaSuccess) return HSDE_ECUDA;
        }
        if constexpr (GT > 0) {
            if constexpr (cone_fits<T, CP, GT>()) {
                if (allow_smem<T, CP, GT, thr_minb<T, CP, GT>(), false, false>((int)ConeCfg<T, CP, GT>::smem) !=
                    cudaSuccess)
                    return HSDE_ECUDA;
            }
        }
        if constexpr (has_rv<T, GR>()) {
            if constexpr (cone_fits<T, CP, GR>()) {
                if (allow_smem<T, CP, GR, rv_minb<T, CP, GR>(), false, true>((int)ConeCfg<T, CP, GR>::smem) !=
                    cudaSuccess)
                    return HSDE_ECUDA;
            }
        }
        return HSDE_OK;
    }
}

// A bucket of few large cliques sets the latency of the whole cone phase:
// each of its CTAs takes a whole SM (no small-clique CTA shares its
// shared-memory bandwidth or issue slots).
template <typename T, int CP, int G>
static bool alone_one(const Bucket& bk) {
    if constexpr (!cone_fits<T, CP, G>()) {
        return false;
    } else {
        using Cfg = ConeCfg<T, CP, G>;
        const int grid = (bk.count + Cfg::GPB - 1) / Cfg::GPB;
        return Cfg::GPB == 1 && CP >= 32 && 3 * grid <= g_num_sms && g_smem_optin >= (int)Cfg::smem;
    }
}

template <typename T, int CP, int G, int GT, int GR>
static bool has_variant(int v) {
    if constexpr (!cone_fits<T, CP, G>()) {
        return false;
    } else {
        if (v == 0) return true;
        if (v == 1) return GT > 0 && cone_fits<T, CP, (GT > 0 ? GT : G)>();
        if (v == 2) return has_rv<T, GR>() && cone_fits<T, CP, (GR > 0 ? GR : G)>();
        return false;
    }
}

template <typename T, int CP, int G, int GT, int GR>
static int launch_one(const DevView& V, const Bucket& bk, int max_sweeps, double tol, int warm, int refresh,
                      int dry, cudaStream_t st) {
    if constexpr (!cone_fits<T, CP, G>()) {
        return HSDE_ERANGE;
    } else {
        using Cfg = ConeCfg<T, CP, G>;
        const T tol2 = (T)(tol * tol);
        if constexpr (GT > 0) {
            if constexpr (cone_fits<T, CP, GT>()) {
                if (bk.variant == 1) {
                    using CT = ConeCfg<T, CP, GT>;
                    const int grid = (bk.count + CT::GPB - 1) / CT::GPB;
                    k_cone<T, CP, GT, thr_minb<T, CP, GT>(), false, false><<<grid, CT::NTH, CT::smem, st>>>(
                        V, bk.list, bk.count, max_sweeps, tol2, warm, refresh, dry);
                    return HSDE_OK;
                }
            }
        }
        if constexpr (has_rv<T, GR>()) {
            if constexpr (cone_fits<T, CP, GR>()) {
                if (bk.variant == 2) {
                    using CR = ConeCfg<T, CP, GR>;
                    k_cone<T, CP, GR, rv_minb<T, CP, GR>(), false, true><<<bk.count, CR::NTH, CR::smem, st>>>(
                        V, bk.list, bk.count, max_sweeps, tol2, warm, refresh, dry);
                    return HSDE_OK;
                }
            }
        }
        const int grid = (bk.count + Cfg::GPB - 1) / Cfg::GPB;
        if constexpr (Cfg::GPB == 1 && CP >= 32 && Cfg::MINB != 1) {
            // a CTA alone on its SM: the variant with the full register budget
            if (alone_one<T, CP, G>(bk)) {
                k_cone<T, CP, G, 1, true, false><<<grid, Cfg::NTH, (size_t)g_smem_optin, st>>>(
                    V, bk.list, bk.count, max_sweeps, tol2, warm, refresh, dry);
                return HSDE_OK;
            }
        }
        const size_t smem = alone_one<T, CP, G>(bk) ? (size_t)g_smem_optin : Cfg::smem;
        k_cone<T, CP, G, Cfg::MINB, true, false><<<grid, Cfg::NTH, smem, st>>>(V, bk.list, bk.count, max_sweeps,
                                                                                tol2, warm, refresh, dry);
        return HSDE_OK;
    }
}

// Cliques above the largest Jacobi bucket of a precision (and up to
// CONE_BIG) go to the tridiagonal QR path of cone_large.cu.
int cone_bucket_of(int c, bool mixed) {
#define X(cp, g, gt, gr) \
    if (c <= cp && (mixed ? cone_fits<float, cp, g>() : cone_fits<double, cp, g>())) return cp;
    HSDE_CONE_BUCKETS(X)
#undef X
    return c <= CONE_BIG ? CONE_BIG : -1;
}

int cone_max_clique(bool) { return CONE_BIG; }

int cone_jacobi_max(bool mixed) {
    int mx = 0;
#define X(cp, g, gt, gr) \
    if (mixed ? cone_fits<float, cp, g>() : cone_fits<double, cp, g>()) mx = cp;
    HSDE_CONE_BUCKETS(X)
#undef X
    return mx;
}

void cone_bucket_sizes(std::vector<int>& out, bool mixed) {
    out.clear();
#define X(cp, g, gt, gr) \
    if (mixed ? cone_fits<float, cp, g>() : cone_fits<double, cp, g>()) out.push_back(cp);
    HSDE_CONE_BUCKETS(X)
#undef X
    out.push_back(CONE_BIG);
}

bool cone_has_variant(int cmax, bool mixed, int variant) {
    if (cmax == CONE_BIG) return variant == 0;
#define X(cp, g, gt, gr)                                                                            \
    if (cmax == cp)                                                                                 \
        return mixed ? has_variant<float, cp, g, gt, gr>(variant) : has_variant<double, cp, g, gt, gr>(variant);
    HSDE_CONE_BUCKETS(X)
#undef X
    return false;
}

int cone_vstore_elems(int c, bool mixed) {
    const int cp = cone_bucket_of(c, mixed);
    if (cp == CONE_BIG) return 0;   // the QR path keeps no basis from one iteration to the next
    return cp < 0 ? -1 : cp * cp;
}

int cone_prepare(bool mixed) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&g_smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return HSDE_ECUDA;
    int rc = HSDE_OK;
#define X(cp, g, gt, gr) \
    rc |= mixed ? prepare_one<float, cp, g, gt, gr>() : prepare_one<double, cp, g, gt, gr>();
    HSDE_CONE_BUCKETS(X)
#undef X
    rc |= cone_big_prepare(mixed);
    return rc == HSDE_OK ? HSDE_OK : HSDE_ECUDA;
}

int cone_smem_bytes(int cmax, bool mixed) {
#define X(cp, g, gt, gr) \
    if (cmax == cp) return mixed ? (int)ConeCfg<float, cp, g>::smem : (int)ConeCfg<double, cp, g>::smem;
    HSDE_CONE_BUCKETS(X)
#undef X
    return -1;
}

bool cone_bucket_alone(const Bucket& bk, bool mixed) {
    if (bk.cmax == CONE_BIG) return true;   // one CTA per clique, launched first
#define X(cp, g, gt, gr) \
    if (bk.cmax == cp) return mixed ? alone_one<float, cp, g>(bk) : alone_one<double, cp, g>(bk);
    HSDE_CONE_BUCKETS(X)
#undef X
    return false;
}

int launch_cone(const DevView& V, const Bucket& bk, bool mixed, int max_sweeps, double tol, int warm, int refresh,
                void* stp, int dry) {
    if (bk.count == 0) return HSDE_OK;
    if (bk.cmax == CONE_BIG) return dry ? HSDE_OK : launch_cone_big(V, bk, mixed, stp);
    if (bk.variant == 3) return dry ? HSDE_OK : (mixed ? launch_cone_qrw(V, bk, stp) : HSDE_ERANGE);
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stp);
#define X(cp, g, gt, gr)                                                                                   \
    if (bk.cmax == cp) {                                                                                   \
        return mixed ? launch_one<float, cp, g, gt, gr>(V, bk, max_sweeps, tol, warm, refresh, dry, st)   \
                     : launch_one<double, cp, g, gt, gr>(V, bk, max_sweeps, tol, warm, refresh, dry, st); \
    }
    HSDE_CONE_BUCKETS(X)
#undef X
    return HSDE_ERANGE;
}

}  // namespace hsde
