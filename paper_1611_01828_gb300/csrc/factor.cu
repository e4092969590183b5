// Structured form of the cached factor (Sections 4.2-4.3): the only matrix
// the method factors is S = I + A Delta^{-1} A^T (m x m).  With the
// constraints of a chordally decomposed problem local to cliques, S is
//     S = B + U U^T,
//     B = I + sum over "local" pattern entries e of w_e Delta_e^{-1} a_e a_e^T
//         (block-diagonal after grouping the constraints that share such an
//          entry: connected components, found by union-find),
//     U = [ sqrt(w_e Delta_e^{-1}) a_e ]  over the r "long" entries
//         (a_e: column e of A, w_e the full-vec weight 1 or 2),
// where an entry is long when more constraints touch it than a block may
// hold (the arrow corner of a block-arrow, which every constraint touches).
// The matrix inversion lemma then gives
//     S^{-1} q = t - W h,  t = B^{-1} q,  W = B^{-1} U,
//     h = K^{-1} U^T t,    K = I_r + U^T W,
// so an iteration reads the block inverses and U, W (about m (b + 2r)
// values) instead of a dense m x m inverse, and the setup inverts small
// blocks and one r x r matrix instead of an m x m one.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <numeric>

#include "internal.h"

namespace hsde {

// In-place inverse of a symmetric positive definite n x n row-major matrix
// by Gauss-Jordan elimination without pivoting (every pivot of an SPD matrix
// is a positive Schur-complement diagonal).
static void gj_inverse_host(double* M, int n) {
    std::vector<double> row(n), col(n);
    for (int k = 0; k < n; ++k) {
        for (int j = 0; j < n; ++j) {
            row[j] = M[(size_t)k * n + j];
            col[j] = M[(size_t)j * n + k];
        }
        const double piv = row[k];
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j) {
                double v;
                if (i == k && j == k) v = 1.0 / piv;
                else if (i == k) v = row[j] / piv;
                else if (j == k) v = -col[i] / piv;
                else v = M[(size_t)i * n + j] - col[i] * row[j] / piv;
                M[(size_t)i * n + j] = v;
            }
    }
}

bool build_lowrank(int32_t m, int64_t N, const int32_t* At_ptr, const int32_t* At_col, const double* At_val,
                   const uint8_t* diag, const double* inv_delta, LowRankHost& L) {
    L = LowRankHost();
    if (m <= 0) return false;
    // long entries and the union-find of constraints over the local ones
    std::vector<int32_t> parent(m);
    std::iota(parent.begin(), parent.end(), 0);
    auto find = [&](int32_t a) {
        while (parent[a] != a) {
            parent[a] = parent[parent[a]];
            a = parent[a];
        }
        return a;
    };
    std::vector<int64_t> long_e;
    for (int64_t e = 0; e < N; ++e) {
        const int32_t j0 = At_ptr[e], j1 = At_ptr[e + 1];
        if (j1 - j0 > LR_BMAX) {
            long_e.push_back(e);
            if ((int)long_e.size() > LR_RMAX) return false;
            continue;
        }
        for (int32_t j = j0 + 1; j < j1; ++j) {
            const int32_t a = find(At_col[j0]), b = find(At_col[j]);
            if (a != b) parent[std::max(a, b)] = std::min(a, b);
        }
    }
    const int r = (int)long_e.size();
    // blocks in order of their smallest constraint; members ascending
    std::vector<int32_t> bid(m, -1), root_bid(m, -1);
    int32_t nb = 0;
    for (int32_t i = 0; i < m; ++i) {
        const int32_t ro = find(i);
        if (root_bid[ro] < 0) root_bid[ro] = nb++;
        bid[i] = root_bid[ro];
    }
    std::vector<int32_t> bsz(nb, 0);
    for (int32_t i = 0; i < m; ++i) bsz[bid[i]]++;
    int64_t cost = 2LL * m * r;
    for (int32_t k = 0; k < nb; ++k) {
        if (bsz[k] > LR_BMAX) return false;
        cost += (int64_t)bsz[k] * bsz[k];
    }
    // worth it only if an iteration reads well under the dense inverse
    if (2 * cost >= (int64_t)m * m) return false;
    L.r = r;
    L.blk_ptr.assign(nb + 1, 0);
    for (int32_t k = 0; k < nb; ++k) L.blk_ptr[k + 1] = L.blk_ptr[k] + bsz[k];
    L.members.resize(m);
    L.row_blk.resize(m);
    L.row_pos.resize(m);
    {
        std::vector<int32_t> fill(L.blk_ptr.begin(), L.blk_ptr.end() - 1);
        for (int32_t i = 0; i < m; ++i) {
            const int32_t k = bid[i];
            L.row_blk[i] = k;
            L.row_pos[i] = fill[k] - L.blk_ptr[k];
            L.members[fill[k]++] = i;
        }
    }
    L.blk_off.resize(nb);
    int64_t tot = 0;
    for (int32_t k = 0; k < nb; ++k) {
        L.blk_off[k] = tot;
        tot += (int64_t)bsz[k] * bsz[k];
    }
    // B = I + local terms, block by block (row-major, both triangles).  The
    // local entries of a block are gathered into a dense b x n_e matrix G
    // (row p: constraint p's values times sqrt(w_e Delta_e^{-1})), and
    // B = I + G G^T is formed by dot products over contiguous rows (the lower
    // triangle, mirrored: B is exactly symmetric).  A block whose entries
    // touch few of its constraints (G mostly zero) is scattered entry by
    // entry instead.
    L.binv.assign(tot, 0.0);
    for (int32_t k = 0; k < nb; ++k)
        for (int32_t p = 0; p < bsz[k]; ++p) L.binv[L.blk_off[k] + (int64_t)p * bsz[k] + p] = 1.0;
    std::vector<int64_t> bent_ptr(nb + 1, 0), pairs(nb, 0);
    for (int64_t e = 0; e < N; ++e) {
        const int32_t j0 = At_ptr[e], j1 = At_ptr[e + 1];
        if (j1 - j0 > LR_BMAX || j1 == j0) continue;
        const int32_t k = L.row_blk[At_col[j0]];
        bent_ptr[k + 1] += 1;
        pairs[k] += (int64_t)(j1 - j0) * (j1 - j0);
    }
    for (int32_t k = 0; k < nb; ++k) bent_ptr[k + 1] += bent_ptr[k];
    std::vector<int64_t> bent(bent_ptr[nb]);
    {
        std::vector<int64_t> fill(bent_ptr.begin(), bent_ptr.end() - 1);
        for (int64_t e = 0; e < N; ++e) {
            const int32_t j0 = At_ptr[e], j1 = At_ptr[e + 1];
            if (j1 - j0 > LR_BMAX || j1 == j0) continue;
            bent[fill[L.row_blk[At_col[j0]]]++] = e;
        }
    }
    std::vector<double> G;
    std::vector<int32_t> pos;
    std::vector<double> val;
    for (int32_t k = 0; k < nb; ++k) {
        const int32_t b = bsz[k];
        const int64_t ne = bent_ptr[k + 1] - bent_ptr[k];
        double* Bk = L.binv.data() + L.blk_off[k];
        if (ne == 0) continue;
        if (4 * pairs[k] >= (int64_t)b * b * ne) {
            G.assign((size_t)b * ne, 0.0);
            for (int64_t q = 0; q < ne; ++q) {
                const int64_t e = bent[bent_ptr[k] + q];
                const double sw = std::sqrt((diag[e] ? 1.0 : 2.0) * inv_delta[e]);
                for (int32_t j = At_ptr[e]; j < At_ptr[e + 1]; ++j)
                    G[(size_t)L.row_pos[At_col[j]] * ne + q] = sw * At_val[j];
            }
            // lower triangle in 4 x 4 tiles of (pa, pb), 16 running sums each
            for (int32_t pa0 = 0; pa0 < b; pa0 += 4)
                for (int32_t pb0 = 0; pb0 <= pa0; pb0 += 4) {
                    double acc[4][4] = {};
                    const double* ga[4];
                    const double* gb[4];
                    for (int u = 0; u < 4; ++u) {
                        ga[u] = G.data() + (size_t)std::min(pa0 + u, b - 1) * ne;
                        gb[u] = G.data() + (size_t)std::min(pb0 + u, b - 1) * ne;
                    }
                    for (int64_t q = 0; q < ne; ++q) {
                        const double a0 = ga[0][q], a1 = ga[1][q], a2 = ga[2][q], a3 = ga[3][q];
                        const double b0 = gb[0][q], b1 = gb[1][q], b2 = gb[2][q], b3 = gb[3][q];
                        acc[0][0] += a0 * b0; acc[0][1] += a0 * b1; acc[0][2] += a0 * b2; acc[0][3] += a0 * b3;
                        acc[1][0] += a1 * b0; acc[1][1] += a1 * b1; acc[1][2] += a1 * b2; acc[1][3] += a1 * b3;
                        acc[2][0] += a2 * b0; acc[2][1] += a2 * b1; acc[2][2] += a2 * b2; acc[2][3] += a2 * b3;
                        acc[3][0] += a3 * b0; acc[3][1] += a3 * b1; acc[3][2] += a3 * b2; acc[3][3] += a3 * b3;
                    }
                    for (int u = 0; u < 4; ++u)
                        for (int v = 0; v < 4; ++v) {
                            const int32_t pa = pa0 + u, pb = pb0 + v;
                            if (pa >= b || pb > pa) continue;
                            Bk[(int64_t)pa * b + pb] += acc[u][v];
                            if (pb != pa) Bk[(int64_t)pb * b + pa] += acc[u][v];
                        }
                }
        } else {
            for (int64_t q = 0; q < ne; ++q) {
                const int64_t e = bent[bent_ptr[k] + q];
                const int32_t j0 = At_ptr[e], j1 = At_ptr[e + 1];
                const double w = (diag[e] ? 1.0 : 2.0) * inv_delta[e];
                pos.resize(j1 - j0);
                val.resize(j1 - j0);
                for (int32_t j = j0; j < j1; ++j) {
                    pos[j - j0] = L.row_pos[At_col[j]];
                    val[j - j0] = At_val[j];
                }
                for (int32_t a = 0; a < j1 - j0; ++a) {
                    double* Brow = Bk + (int64_t)pos[a] * b;
                    const double wa = w * val[a];
                    for (int32_t c = 0; c < j1 - j0; ++c) Brow[pos[c]] += wa * val[c];
                }
            }
        }
    }
    for (int32_t k = 0; k < nb; ++k) gj_inverse_host(L.binv.data() + L.blk_off[k], bsz[k]);
    if (r == 0) return true;
    // U (m x r) and W = B^{-1} U
    L.U.assign((size_t)m * r, 0.0);
    for (int c = 0; c < r; ++c) {
        const int64_t e = long_e[c];
        const double s = std::sqrt((diag[e] ? 1.0 : 2.0) * inv_delta[e]);
        for (int32_t j = At_ptr[e]; j < At_ptr[e + 1]; ++j) L.U[(size_t)At_col[j] * r + c] = s * At_val[j];
    }
    L.W.assign((size_t)m * r, 0.0);
    for (int32_t i = 0; i < m; ++i) {
        const int32_t k = L.row_blk[i], b = bsz[k], p = L.row_pos[i];
        const double* Bi = L.binv.data() + L.blk_off[k] + (int64_t)p * b;
        const int32_t* mem = L.members.data() + L.blk_ptr[k];
        for (int c = 0; c < r; ++c) {
            double acc = 0.0;
            for (int32_t q = 0; q < b; ++q) acc += Bi[q] * L.U[(size_t)mem[q] * r + c];
            L.W[(size_t)i * r + c] = acc;
        }
    }
    // K = I + U^T W (symmetric in exact arithmetic; symmetrised), then K^{-1}
    L.kinv.assign((size_t)r * r, 0.0);
    for (int a = 0; a < r; ++a)
        for (int c = 0; c < r; ++c) {
            double acc = 0.0;
            for (int32_t i = 0; i < m; ++i) acc += L.U[(size_t)i * r + a] * L.W[(size_t)i * r + c];
            L.kinv[(size_t)a * r + c] = acc + (a == c ? 1.0 : 0.0);
        }
    for (int a = 0; a < r; ++a)
        for (int c = 0; c < a; ++c) {
            const double s = 0.5 * (L.kinv[(size_t)a * r + c] + L.kinv[(size_t)c * r + a]);
            L.kinv[(size_t)a * r + c] = L.kinv[(size_t)c * r + a] = s;
        }
    gj_inverse_host(L.kinv.data(), r);
    return true;
}

// ---------------------------------------------------------------------------
// Device solve y = S^{-1} q for the instances in structured form, over tiles
// of LR_TILE constraint rows of one instance (one CTA, 8 warps, a row per
// warp at a time).  k_lr_t: t = B^{-1} q (a row of its block's inverse
// against the block's q), written to y, and the tile's partial of U^T t;
// the last CTA of an instance sums the partials in tile order and forms
// h = K^{-1} U^T t.  k_lr_y: y = t - W h and, on iterations, b_i y_i.
// Fixed-order sums only: bitwise reproducible.
// ---------------------------------------------------------------------------
namespace {

constexpr int LNT = 256;

__device__ __forceinline__ double lr_warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__global__ void __launch_bounds__(LNT) k_lr_t(DevView V, const double* __restrict__ qin, double* __restrict__ yout,
                                              int iter) {
    __shared__ double gw[LNT / 32][LR_RMAX];
    __shared__ double g[LR_RMAX];
    __shared__ int flag;
    const int4 t = V.lr_tiles[blockIdx.x];   // (instance, first row, end row, -)
    InstDev& I = V.inst[t.x];
    if (iter && I.status != HSDE_RUNNING) return;
    const int r = I.lr_r;
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    double g0 = 0.0, g1 = 0.0;
    for (int row = t.y + w; row < t.z; row += LNT / 32) {
        const int b = V.lr_bsz[row];
        const double* Br = V.lr_binv + V.lr_binv_row[row];
        const int32_t* mem = V.lr_members + V.lr_mem[row];
        double acc = 0.0;
        for (int p = l; p < b; p += 32) acc += Br[p] * qin[mem[p]];
        acc = lr_warp_sum(acc);
        if (l == 0) yout[row] = acc;
        const double* Ui = V.lr_U + I.lr_off + (int64_t)(row - I.m_off) * r;
        if (l < r) g0 += Ui[l] * acc;
        if (l + 32 < r) g1 += Ui[l + 32] * acc;
    }
    gw[w][l] = g0;
    gw[w][l + 32] = g1;
    __syncthreads();
    if (threadIdx.x < LR_RMAX) {
        double s = 0.0;
#pragma unroll
        for (int k = 0; k < LNT / 32; ++k) s += gw[k][threadIdx.x];
        V.lr_part[(int64_t)blockIdx.x * LR_RMAX + threadIdx.x] = s;
    }
    // last CTA of this instance: h = K^{-1} (sum of the tile partials)
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) flag = (atomicAdd(V.counters + 2 * V.B + t.x, 1) == I.lr_tile_end - I.lr_tile_begin - 1);
    __syncthreads();
    if (!flag) return;
    __threadfence();
    if (threadIdx.x < LR_RMAX) {
        double s = 0.0;
        for (int tt = I.lr_tile_begin; tt < I.lr_tile_end; ++tt) s += __ldcg(V.lr_part + (int64_t)tt * LR_RMAX + threadIdx.x);
        g[threadIdx.x] = s;
    }
    __syncthreads();
    if ((int)threadIdx.x < r) {
        const double* Kr = V.lr_kinv + I.kinv_off + (int64_t)threadIdx.x * r;
        double s = 0.0;
        for (int c = 0; c < r; ++c) s += Kr[c] * g[c];
        V.lr_h[I.h_off + threadIdx.x] = s;
    }
    if (threadIdx.x == 0) V.counters[2 * V.B + t.x] = 0;
}

__global__ void __launch_bounds__(LNT) k_lr_y(DevView V, double* __restrict__ yout, double* __restrict__ rowb,
                                              int iter) {
    const int4 t = V.lr_tiles[blockIdx.x];
    const InstDev& I = V.inst[t.x];
    if (iter && I.status != HSDE_RUNNING) return;
    const int r = I.lr_r;
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    const double* h = V.lr_h + I.h_off;
    for (int row = t.y + w; row < t.z; row += LNT / 32) {
        const double* Wi = V.lr_W + I.lr_off + (int64_t)(row - I.m_off) * r;
        double acc = 0.0;
        for (int c = l; c < r; c += 32) acc += Wi[c] * h[c];
        acc = lr_warp_sum(acc);
        if (l == 0) {
            const double y = yout[row] - acc;
            yout[row] = y;
            if (rowb) rowb[row] = V.b[row] * y;
        }
    }
}

}  // namespace

void launch_lr_solve(const DevView& V, const double* qin, double* yout, double* rowb, bool iter, void* st) {
    if (V.nlr <= 0) return;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(st);
    k_lr_t<<<V.nlr, LNT, 0, s>>>(V, qin, yout, iter ? 1 : 0);
    k_lr_y<<<V.nlr, LNT, 0, s>>>(V, yout, rowb, iter ? 1 : 0);
}

}  // namespace hsde
