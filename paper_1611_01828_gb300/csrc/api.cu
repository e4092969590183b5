// C-ABI of libhsde (include/hsde.h): setup, iterate, queries.
//
// Device memory: one arena per handle (cudaMalloc once at setup), carved
// into the concatenated per-instance arrays; nothing is allocated while
// iterating.  One iteration is a fixed launch sequence (affine step, eta,
// clique cone projections in parallel graph branches, stopping rule) that is
// captured once into a CUDA graph and replayed.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <thread>
#include <chrono>
#include <climits>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <numeric>
#include <string>
#include <tuple>
#include <vector>

#include "internal.h"

using namespace hsde;

namespace {

thread_local std::string g_err;

int fail(int code, const std::string& msg) {
    g_err = msg;
    return code;
}

}  // namespace

int hsde::set_error(int code, const std::string& msg) { return fail(code, msg); }

namespace {

#define CK(call)                                                                        \
    do {                                                                                \
        cudaError_t e_ = (call);                                                        \
        if (e_ != cudaSuccess) {                                                        \
            return fail(HSDE_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
        }                                                                               \
    } while (0)

double now_ms() {
    return std::chrono::duration<double, std::milli>(
               std::chrono::steady_clock::now().time_since_epoch()).count();
}

// Host preparation of one instance.
struct HostPrep {
    Symbolic S;
    int32_t n = 0, m = 0, cmax = 0;
    std::vector<double> cvec, inv_delta;
    std::vector<uint8_t> diag;
    std::vector<int32_t> sc_ptr, sc_idx;      // local packed indices
    std::vector<int32_t> A_ptr, A_col;        // local entry indices
    std::vector<double> A_val;                // off-diagonal weight 2 applied
    std::vector<int32_t> At_ptr, At_col;      // local constraint indices
    std::vector<double> At_val;
    std::vector<double> b;
    // internal constraint order: row i of A, b, y is the caller's row perm[i]
    // (empty: the caller's order).  Constraints are ordered by the first
    // pattern entry they touch, so that the constraints of one clique are
    // neighbours and the gathers of A^T y read contiguous runs.
    std::vector<int32_t> perm;
    // data scaling (hsde_options.scaling): A~ = D A, b~ = sigma D b, c~ = rho c
    std::vector<double> dscale;               // d_i (1 when not scaling)
    double sigma = 1.0, rho = 1.0;
    double bnorm = 0.0, cnorm = 0.0;          // ||b||, ||c|| of the original data
    bool dense = false;                       // two constraints share an entry
    bool lowrank = false;                     // dense S kept as B + U U^T (factor.cu)
    LowRankHost lr;
    std::vector<double> Sdiag_inv;            // m (diagonal case)
};

// Scaling factors of one instance from its ORIGINAL data (the practical form
// of the cited ADMM; the paper applies it without saying how): sigma and rho
// from max(||D b||, ||c||), where D b is the row-normalised b.
// sigma, rho and the original norms from the sums sum (d_i b_i)^2, sum b_i^2
// and the full-vec sum c_e^2 (reading P7).
void scale_from_sums(double nb, double bb, double cc, const hsde_options& O, double& sigma, double& rho,
                     double& bnorm, double& cnorm) {
    bnorm = std::sqrt(bb);
    cnorm = std::sqrt(cc);
    sigma = rho = 1.0;
    if (!O.scaling) return;
    const double mx = std::max(std::sqrt(nb), cnorm);
    if (mx > 0.0) {
        sigma = O.scale_norm / mx;
        rho = O.dual_weight * O.scale_norm / mx;
    }
}

void scale_factors(const HostPrep& H, const double* b, const double* c, const hsde_options& O, double& sigma,
                   double& rho, double& bnorm, double& cnorm) {
    double nb = 0.0, bb = 0.0, cc = 0.0;
    for (int32_t i = 0; i < H.m; ++i) {
        const double db = H.dscale[i] * b[i];
        nb += db * db;
        bb += b[i] * b[i];
    }
    for (size_t e = 0; e < H.diag.size(); ++e) cc += (H.diag[e] ? 1.0 : 2.0) * c[e] * c[e];
    scale_from_sums(nb, bb, cc, O, sigma, rho, bnorm, cnorm);
}

int prepare(const hsde_problem* P, const hsde_options& O, HostPrep& H, std::string& err) {
    int rc = build_symbolic(P, H.S, err);
    if (rc != HSDE_OK) return rc;
    const Symbolic& S = H.S;
    H.n = P->n;
    H.m = P->m;
    const int64_t N = S.N();
    const int32_t p = S.p();
    H.cmax = 0;
    for (int32_t k = 0; k < p; ++k) H.cmax = std::max(H.cmax, S.clique_ptr[k + 1] - S.clique_ptr[k]);
    H.diag.resize(N);
    H.inv_delta.resize(N);
    for (int64_t e = 0; e < N; ++e) {
        H.diag[e] = (S.pat_row[e] == S.pat_col[e]) ? 1 : 0;
        H.inv_delta[e] = 1.0 / (1.0 + 0.5 * (double)S.D[e]);
    }
    H.cvec.assign(N, 0.0);
    for (int64_t k = 0; k < P->C_nnz; ++k) {
        const int32_t e = S.pos(P->C_row[k], P->C_col[k]);
        H.cvec[e] = P->C_val[k];
    }
    // H^T as CSR over entries (packed positions ascending within an entry)
    H.sc_ptr.assign(N + 1, 0);
    for (int32_t e : S.gather) H.sc_ptr[e + 1] += 1;
    for (int64_t e = 0; e < N; ++e) H.sc_ptr[e + 1] += H.sc_ptr[e];
    H.sc_idx.resize(S.gather.size());
    {
        std::vector<int32_t> fill(H.sc_ptr.begin(), H.sc_ptr.end() - 1);
        for (size_t j = 0; j < S.gather.size(); ++j) H.sc_idx[fill[S.gather[j]]++] = (int32_t)j;
    }
    // A (rows = constraints) with full-vec weights, and A^T (rows = entries);
    // with scaling, every row i is multiplied by d_i = 1 / ||A_i|| (full-vec)
    const int32_t m = P->m;
    H.A_ptr.assign(m + 1, 0);
    H.dscale.assign(m, 1.0);
    const int64_t a0 = m > 0 ? P->A_ptr[0] : 0;
    std::vector<std::pair<int32_t, double>> row;
    H.A_col.reserve(m > 0 ? (size_t)(P->A_ptr[m] - a0) : 0);
    H.A_val.reserve(H.A_col.capacity());
    // pattern position of each entry: a binary search in its column, or,
    // for the next row of the same column (entries given column by column,
    // rows ascending), a galloping search on from the previous position
    const int32_t* pcol = S.pat_colptr.data();
    const int32_t* prow = S.pat_row.data();
    for (int32_t i = 0; i < m; ++i) {
        const size_t base = H.A_col.size();
        double nrm = 0.0;
        bool sorted = true;   // entries given in (column, row) order are already in pattern order
        int32_t cur_c = -1, cur_r = -1, cp = 0, ce = 0, prev_e = INT32_MIN;
        for (int64_t k = P->A_ptr[i] - a0; k < P->A_ptr[i + 1] - a0; ++k) {
            const int32_t r = P->A_row[k], c = P->A_col[k];
            if (c == cur_c && r > cur_r) {
                if (cp < ce && prow[cp] < r) {
                    int32_t lo = cp, step = 1;
                    while (lo + step < ce && prow[lo + step] < r) {
                        lo += step;
                        step <<= 1;
                    }
                    const int32_t hi = std::min(lo + step, ce);
                    cp = (int32_t)(std::lower_bound(prow + lo + 1, prow + hi, r) - prow);
                }
            } else {
                cur_c = c;
                ce = pcol[c + 1];
                cp = (int32_t)(std::lower_bound(prow + pcol[c], prow + ce, r) - prow);
            }
            cur_r = r;
            const int32_t e = (cp < ce && prow[cp] == r) ? cp : -1;
            sorted = sorted && e >= prev_e;
            prev_e = e;
            H.A_col.push_back(e);
            H.A_val.push_back(P->A_val[k]);
            nrm += (r == c ? 1.0 : 2.0) * P->A_val[k] * P->A_val[k];
        }
        if (O.scaling && nrm > 0.0) H.dscale[i] = 1.0 / std::sqrt(nrm);
        const double di = H.dscale[i];
        const size_t end_i = H.A_col.size();
        if (!sorted) {
            row.clear();
            for (size_t j = base; j < end_i; ++j) row.push_back({H.A_col[j], H.A_val[j]});
            std::sort(row.begin(), row.end(),
                      [](const std::pair<int32_t, double>& a, const std::pair<int32_t, double>& b) {
                          return a.first < b.first;
                      });
            for (size_t j = base; j < end_i; ++j) {
                H.A_col[j] = row[j - base].first;
                H.A_val[j] = row[j - base].second;
            }
        }
        for (size_t j = base; j < end_i; ++j) {
            const double v = H.A_val[j] * di;
            H.A_val[j] = H.diag[H.A_col[j]] ? v : 2.0 * v;
        }
        H.A_ptr[i + 1] = (int32_t)end_i;
    }
    // internal order of the constraints: by the first pattern entry of each
    // row (stable, so an already ordered problem keeps the identity)
    std::vector<double> bp(P->b, P->b + m);
    {
        std::vector<int32_t> order(m);
        std::iota(order.begin(), order.end(), 0);
        auto first = [&](int32_t i) { return H.A_ptr[i + 1] > H.A_ptr[i] ? H.A_col[H.A_ptr[i]] : INT32_MAX; };
        std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) { return first(a) < first(b); });
        bool ident = true;
        for (int32_t i = 0; i < m; ++i) ident = ident && order[i] == i;
        if (!ident) {
            std::vector<int32_t> ptr(m + 1, 0), col;
            std::vector<double> val, dsc(m);
            col.reserve(H.A_col.size());
            val.reserve(H.A_val.size());
            for (int32_t i = 0; i < m; ++i) {
                const int32_t o = order[i];
                col.insert(col.end(), H.A_col.begin() + H.A_ptr[o], H.A_col.begin() + H.A_ptr[o + 1]);
                val.insert(val.end(), H.A_val.begin() + H.A_ptr[o], H.A_val.begin() + H.A_ptr[o + 1]);
                ptr[i + 1] = (int32_t)col.size();
                dsc[i] = H.dscale[o];
                bp[i] = P->b[o];
            }
            H.A_ptr.swap(ptr);
            H.A_col.swap(col);
            H.A_val.swap(val);
            H.dscale.swap(dsc);
            H.perm.swap(order);
        }
    }
    H.At_ptr.assign(N + 1, 0);
    for (int32_t e : H.A_col) H.At_ptr[e + 1] += 1;
    for (int64_t e = 0; e < N; ++e) H.At_ptr[e + 1] += H.At_ptr[e];
    H.At_col.resize(H.A_col.size());
    H.At_val.resize(H.A_col.size());
    int32_t max_at = 0;
    {
        std::vector<int32_t> fill(H.At_ptr.begin(), H.At_ptr.end() - 1);
        for (int32_t i = 0; i < m; ++i)
            for (int32_t j = H.A_ptr[i]; j < H.A_ptr[i + 1]; ++j) {
                const int32_t e = H.A_col[j];
                const double raw = H.diag[e] ? H.A_val[j] : 0.5 * H.A_val[j];
                H.At_col[fill[e]] = i;
                H.At_val[fill[e]] = raw;
                fill[e]++;
            }
        for (int64_t e = 0; e < N; ++e) max_at = std::max(max_at, H.At_ptr[e + 1] - H.At_ptr[e]);
    }
    // b~ = sigma D b, c~ = rho c (the factors from the original data)
    scale_factors(H, bp.data(), H.cvec.data(), O, H.sigma, H.rho, H.bnorm, H.cnorm);
    H.b.resize(m);
    for (int32_t i = 0; i < m; ++i) H.b[i] = H.sigma * H.dscale[i] * bp[i];
    for (double& cv : H.cvec) cv *= H.rho;
    // S = I + A Delta^{-1} A^T (full-vec inner products); diagonal if no two
    // constraints share a pattern entry.
    H.dense = max_at > 1;
    if (H.dense && O.structured_factor)
        H.lowrank = build_lowrank(m, N, H.At_ptr.data(), H.At_col.data(), H.At_val.data(), H.diag.data(),
                                  H.inv_delta.data(), H.lr);
    if (H.lowrank) {
        // nothing more: the structured factor replaces the dense S
    } else if (!H.dense) {
        std::vector<double> d(m, 1.0);
        for (int64_t e = 0; e < N; ++e)
            for (int32_t j = H.At_ptr[e]; j < H.At_ptr[e + 1]; ++j) {
                const double a = H.At_val[j];
                d[H.At_col[j]] += (H.diag[e] ? 1.0 : 2.0) * a * a * H.inv_delta[e];
            }
        H.Sdiag_inv.resize(m);
        for (int32_t i = 0; i < m; ++i) H.Sdiag_inv[i] = 1.0 / d[i];
    }
    // otherwise S is dense: formed on the device (k_form_S) and inverted there
    return HSDE_OK;
}


}  // namespace

struct hsde_symbolic {
    Symbolic S;
};

// Buffers of the reverse sweep through unrolled iterations (allocated on the
// first hsde_unrolled_forward, outside the iteration hot path).
struct UnrollWS {
    void* mem = nullptr;
    size_t bytes = 0;
    int K = 0, ckpt = 0, nseg = 0;
    size_t cp_stride = 0;
    char* cp = nullptr;
    int64_t tv_total = 0;
    void* tape_v = nullptr;
    double *tape_scal = nullptr, *tape_x = nullptr, *tape_y = nullptr;
    double *xbar = nullptr, *ybar = nullptr, *adj_scal = nullptr, *wtau = nullptr, *kpart = nullptr;
    void *sbar = nullptr, *zbar = nullptr, *vbar = nullptr, *aw_s = nullptr, *aw_v = nullptr;
    double *f2 = nullptr, *q2 = nullptr, *yw2 = nullptr, *xw2 = nullptr, *part2 = nullptr, *eta2 = nullptr;
    double *otau = nullptr, *ox = nullptr, *oy = nullptr;
    void *os = nullptr, *ov = nullptr;
    double *xp_neg = nullptr, *yp_neg = nullptr, *den_neg = nullptr, *ctp_neg = nullptr;
    double *gc = nullptr, *gb = nullptr;
    int64_t* tv_off = nullptr;
    bool neg_ready = false;
    bool forward_done = false;
};

struct hsde_handle {
    int32_t B = 0;
    hsde_options opt{};
    bool mixed = true;
    int device = 0;
    std::vector<HostPrep> prep;
    std::vector<int64_t> x_off, p_off;
    std::vector<int32_t> m_off;
    cudaStream_t st = nullptr;
    bool own_stream = false;
    cudaStream_t side[MAX_BUCKETS] = {};
    cudaEvent_t ev_fork = nullptr, ev_join[MAX_BUCKETS] = {};
    void* arena = nullptr;
    size_t arena_bytes = 0;
    DevView V{};
    std::vector<Bucket> buckets;
    InstDev* host_inst = nullptr;       // pinned mirror
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    double setup_ms = 0, iterate_ms = 0;
    int max_sweeps = 12;
    double jtol = 1e-6;
    int warm = 1, refresh = 32;
    // phase timing (options.profile)
    bool profile = false;
    bool capturing = false;
    cudaEvent_t ev_it0 = nullptr, ev_aff = nullptr, ev_chk = nullptr, ev_it1 = nullptr;
    cudaEvent_t ev_cs[MAX_BUCKETS] = {}, ev_ce[MAX_BUCKETS] = {};
    std::vector<int64_t> bucket_c3;
    std::vector<std::vector<int32_t>> bucket_ids;   // host copy of each bucket's clique list
    int kernels_per_iter = 0;
    int64_t launched = 0;      // iterations enqueued since setup
    bool any_dense = false;
    bool need_rhs = true;      // f must be formed before the next iteration (after setup / set_state)
    UnrollWS uw;
    // hsde_set_data from device memory: d_i of every instance and the
    // per-CTA sums (allocated on first use)
    double* dscale_dev = nullptr;
    double* data_part = nullptr;
    int32_t* perm_dev = nullptr;        // [Mtot] caller index of each internal row (null: all identity)
    double* data_part_host = nullptr;   // pinned
};

namespace {

cudaError_t rec(hsde_handle* h, cudaEvent_t ev, cudaStream_t s) {
    if (!h->profile) return cudaSuccess;
    return h->capturing ? cudaEventRecordWithFlags(ev, s, cudaEventRecordExternal) : cudaEventRecord(ev, s);
}

int enqueue_iteration_v(hsde_handle* h, const DevView& V, int warm, bool events);

int enqueue_iteration(hsde_handle* h) { return enqueue_iteration_v(h, h->V, h->warm, true); }

int enqueue_iteration_v(hsde_handle* h, const DevView& V, int warm, bool events) {
    const bool prof = h->profile;
    if (!events) h->profile = false;
    struct Restore { hsde_handle* h; bool p; ~Restore() { h->profile = p; } } restore{h, prof};
    CK(rec(h, h->ev_it0, h->st));
    launch_fwd(V, h->st);
    if (h->any_dense) launch_solve_dense(V, h->st);
    launch_lr_solve(V, V.q, V.yw, V.rowb, true, h->st);
    launch_bwd_eta(V, h->st);
    CK(rec(h, h->ev_aff, h->st));
    // fork: every clique bucket on its own branch; buckets whose CTAs each
    // take a whole SM go first, largest cliques first (their CTAs are placed
    // while SMs are still empty), then the others by total work sum c^3,
    // largest first (the longest branch starts first)
    CK(cudaEventRecord(h->ev_fork, h->st));
    const size_t nb = h->buckets.size();
    std::vector<size_t> order, rest;
    for (size_t i = nb; i-- > 0;)
        (cone_bucket_alone(h->buckets[i], h->mixed) ? order : rest).push_back(i);
    std::stable_sort(rest.begin(), rest.end(), [&](size_t a, size_t b) { return h->bucket_c3[a] > h->bucket_c3[b]; });
    order.insert(order.end(), rest.begin(), rest.end());
    for (size_t i : order) {
        CK(cudaStreamWaitEvent(h->side[i], h->ev_fork, 0));
        CK(rec(h, h->ev_cs[i], h->side[i]));
        int rc = launch_cone(V, h->buckets[i], h->mixed, h->max_sweeps, h->jtol, warm, h->refresh,
                             h->side[i]);
        if (rc != HSDE_OK) return fail(rc, "cone launch failed");
        CK(rec(h, h->ev_ce[i], h->side[i]));
        CK(cudaEventRecord(h->ev_join[i], h->side[i]));
    }
    for (size_t i = 0; i < nb; ++i) CK(cudaStreamWaitEvent(h->st, h->ev_join[i], 0));
    CK(rec(h, h->ev_chk, h->st));
    launch_long(V, h->mixed, h->st);
    launch_post(V, h->mixed, h->st);
    CK(rec(h, h->ev_it1, h->st));
    CK(cudaGetLastError());
    return HSDE_OK;
}

int count_kernels(const hsde_handle* h) {
    const DevView& V = h->V;
    int k = 0;
    if (V.ntiles > 0) k += 2;          // bwd_eta, post
    if (V.nlong > 0) k += 1;           // long entries' H^T sums
    if (V.Mtot > 0) k += 1;            // fwd
    if (h->any_dense) k += 1;          // solve_dense
    if (V.nlr > 0) k += 2;             // structured solve
    for (const auto& b : h->buckets) k += b.count > 0 ? 1 : 0;
    return k;
}

int sync_inst(hsde_handle* h) {
    CK(cudaMemcpyAsync(h->host_inst, h->V.inst, sizeof(InstDev) * h->B, cudaMemcpyDeviceToHost, h->st));
    CK(cudaStreamSynchronize(h->st));
    return HSDE_OK;
}

void free_handle(hsde_handle* h) {
    if (!h) return;
    if (h->exec) cudaGraphExecDestroy(h->exec);
    if (h->graph) cudaGraphDestroy(h->graph);
    if (h->st) cudaStreamSynchronize(h->st);
    for (auto& s : h->side) if (s) cudaStreamDestroy(s);
    for (auto& e : h->ev_join) if (e) cudaEventDestroy(e);
    if (h->ev_fork) cudaEventDestroy(h->ev_fork);
    for (cudaEvent_t e : {h->ev_it0, h->ev_aff, h->ev_chk, h->ev_it1}) if (e) cudaEventDestroy(e);
    for (auto& e : h->ev_cs) if (e) cudaEventDestroy(e);
    for (auto& e : h->ev_ce) if (e) cudaEventDestroy(e);
    if (h->arena) cudaFree(h->arena);
    if (h->uw.mem) cudaFree(h->uw.mem);
    if (h->dscale_dev) cudaFree(h->dscale_dev);
    if (h->perm_dev) cudaFree(h->perm_dev);
    if (h->data_part) cudaFree(h->data_part);
    if (h->data_part_host) cudaFreeHost(h->data_part_host);
    if (h->host_inst) cudaFreeHost(h->host_inst);
    if (h->own_stream && h->st) cudaStreamDestroy(h->st);
    delete h;
}

struct Carver {
    size_t off = 0;
    template <typename T>
    size_t take(size_t count) {
        off = (off + 255) / 256 * 256;
        const size_t o = off;
        off += count * sizeof(T);
        return o;
    }
};

template <typename T>
int upload(void* dst, const std::vector<T>& v, cudaStream_t st) {
    if (v.empty()) return HSDE_OK;
    CK(cudaMemcpyAsync(dst, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, st));
    return HSDE_OK;
}

// A^T tiles of one instance for k_bwd_eta: runs of whole rows (pattern
// entries) with at most TILE_N rows and AT_TILE_NNZ nonzeros, so that every
// CTA gets about the same number of nonzeros whatever the row lengths.  Each
// row of a tile is reduced by a group of lanes, the power of two (1 ... 32)
// that gives each lane at most AT_LANE_NNZ of the tile's mean row; a row
// longer than AT_TILE_NNZ is a tile alone, reduced by the whole CTA
// (lanes = TILE_N).
void append_at_tiles(const HostPrep& H, int32_t b, int64_t xo, std::vector<int4>& out) {
    const int64_t N = H.S.N();
    int64_t e0 = 0, nnz = 0;
    auto close = [&](int64_t e1) {
        const int64_t rows = e1 - e0;
        int lanes = 1;
        if (rows == 1 && nnz > AT_TILE_NNZ) lanes = TILE_N;
        else
            while (lanes < 32 && (int64_t)lanes * AT_LANE_NNZ * rows < nnz) lanes *= 2;
        out.push_back(make_int4(b, (int)(xo + e0), (int)(xo + e1), lanes));
        e0 = e1;
        nnz = 0;
    };
    for (int64_t e = 0; e < N; ++e) {
        const int64_t len = H.At_ptr[e + 1] - H.At_ptr[e];
        if (e > e0 && (e - e0 >= TILE_N || nnz + len > AT_TILE_NNZ)) close(e);
        nnz += len;
    }
    if (N > e0) close(N);
}

// ---- eigensolver variant per bucket (the autotuner) ----
// A bucket of few large cliques (each CTA alone on its SM) runs the latency
// variant.  Any other bucket with more than one variant gets the fastest for
// its clique count on this GPU, timed once per (precision, size, count, SMs)
// in dry runs (synthetic matrices, two sweeps, no writes) and cached for the
// process.  All variants give bitwise the same results, so the choice
// changes only the time.  options.autotune: 1 time them (default); 0 the
// throughput variant unless alone; 2 always latency; 3 always throughput;
// 4 register-V where a bucket has it (else throughput, else latency).
std::mutex g_tune_mu;
std::map<std::tuple<int, int, int, int>, int> g_tune_cache;

int time_variant(hsde_handle* h, Bucket& bk, int variant, float& ms) {
    bk.variant = variant;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    struct Ev { cudaEvent_t a, b; ~Ev() { cudaEventDestroy(a); cudaEventDestroy(b); } } ev{e0, e1};
    constexpr int REPS = 3;
    int rc = launch_cone(h->V, bk, h->mixed, 2, 1e-6, 0, 0, h->st, 1);   // warm-up
    CK(cudaEventRecord(e0, h->st));
    for (int r = 0; r < REPS && rc == HSDE_OK; ++r) rc = launch_cone(h->V, bk, h->mixed, 2, 1e-6, 0, 0, h->st, 1);
    CK(cudaEventRecord(e1, h->st));
    if (rc != HSDE_OK) return fail(rc, "eigensolver variant launch");
    CK(cudaGetLastError());
    CK(cudaEventSynchronize(e1));
    CK(cudaEventElapsedTime(&ms, e0, e1));
    ms /= REPS;
    return HSDE_OK;
}

int choose_variants(hsde_handle* h) {
    int nsm = 0;
    CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, h->device));
    for (Bucket& bk : h->buckets) {
        bk.variant = 0;
        // mixed cliques of 33 to 64: the warp tridiagonal QR when asked for
        // (options.eigensolver = 1)
        if (h->mixed && cone_qrw_has(bk.cmax) && h->opt.eigensolver == 1) {
            bk.variant = 3;
            continue;
        }
        bool has[3];
        int nv = 0;
        for (int v = 0; v < 3; ++v) nv += (has[v] = cone_has_variant(bk.cmax, h->mixed, v)) ? 1 : 0;
        if (nv < 2 || cone_bucket_alone(bk, h->mixed)) continue;
        const int mode = h->opt.autotune;
        if (mode == 2) continue;
        if (mode == 0 || mode == 3) {
            bk.variant = has[1] ? 1 : 0;
            continue;
        }
        if (mode == 4) {
            bk.variant = has[2] ? 2 : (has[1] ? 1 : 0);
            continue;
        }
        const auto key = std::make_tuple((int)h->mixed, (int)bk.cmax, (int)bk.count, nsm);
        {
            std::lock_guard<std::mutex> lk(g_tune_mu);
            auto it = g_tune_cache.find(key);
            if (it != g_tune_cache.end()) {
                bk.variant = it->second;
                continue;
            }
        }
        // candidates in the order throughput, latency, register-V; a later
        // one replaces the best so far only if its dry runs are 5% faster
        // (they run alone, while the iteration runs the buckets side by side)
        int best = -1;
        float tbest = 0.f;
        for (int v : {1, 0, 2}) {
            if (!has[v]) continue;
            float t = 0.f;
            int rc;
            if ((rc = time_variant(h, bk, v, t)) != HSDE_OK) return rc;
            if (best < 0 || t < 0.95f * tbest) { best = v; tbest = t; }
        }
        bk.variant = best;
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tune_cache[key] = best;
    }
    return HSDE_OK;
}

int setup_impl(const hsde_problem* P, int32_t B, const hsde_options* O, hsde_handle** out) {
    const double t0 = now_ms();
    if (!out) return fail(HSDE_EINVAL, "out is null");
    *out = nullptr;
    if (!P || B <= 0) return fail(HSDE_EINVAL, "null problem or B <= 0");
    hsde_options opt;
    hsde_default_options(&opt);
    if (O) opt = *O;
    if (!(opt.eps_tol > 0) || opt.max_iter <= 0 || opt.check_every <= 0 ||
        (opt.precision != HSDE_FP64 && opt.precision != HSDE_MIXED) || opt.jacobi_max_sweeps < 0 ||
        opt.jacobi_tol < 0 || opt.warm_start < -1 || opt.warm_start > 1 || opt.warm_refresh < 0 ||
        (opt.scaling != 0 && opt.scaling != 1) || (opt.structured_factor != 0 && opt.structured_factor != 1) || !(opt.alpha > 0.0 && opt.alpha < 2.0) ||
        !(opt.scale_norm > 0.0) || !(opt.dual_weight > 0.0) || !std::isfinite(opt.scale_norm) ||
        !std::isfinite(opt.dual_weight) || opt.autotune < 0 || opt.autotune > 4 || opt.eigensolver < 0 ||
        opt.eigensolver > 1)
        return fail(HSDE_EINVAL, "invalid options");

    auto* h = new hsde_handle();
    struct Guard {
        hsde_handle*& h;
        ~Guard() { if (h) free_handle(h); }
    } guard{h};
    h->B = B;
    h->opt = opt;
    h->mixed = opt.precision == HSDE_MIXED;
    h->device = opt.device;
    h->max_sweeps = opt.jacobi_max_sweeps > 0 ? opt.jacobi_max_sweeps : (h->mixed ? 12 : 16);
    h->jtol = opt.jacobi_tol > 0 ? opt.jacobi_tol : (h->mixed ? 1e-6 : 1e-14);
    h->warm = opt.warm_start == -1 ? (h->mixed ? 1 : 0) : opt.warm_start;
    h->refresh = opt.warm_refresh > 0 ? opt.warm_refresh : 32;

    // ---- host analysis and preparation (instances in parallel) ----
    h->prep.resize(B);
    {
        std::vector<int> rcs(B, HSDE_OK);
        std::vector<std::string> errs(B);
        std::atomic<int32_t> next{0};
        const unsigned hw = std::max(1u, std::thread::hardware_concurrency());
        const int nth = (int)std::min<unsigned>(hw, (unsigned)B);
        auto work = [&]() {
            for (;;) {
                const int32_t b = next.fetch_add(1);
                if (b >= B) return;
                try {
                    rcs[b] = prepare(&P[b], opt, h->prep[b], errs[b]);
                } catch (const std::bad_alloc&) {
                    rcs[b] = HSDE_ENOMEM;
                    errs[b] = "host allocation failed";
                }
            }
        };
        std::vector<std::thread> pool;
        for (int t = 1; t < nth; ++t) pool.emplace_back(work);
        work();
        for (auto& t : pool) t.join();
        for (int32_t b = 0; b < B; ++b) {
            if (rcs[b] != HSDE_OK) return fail(rcs[b], "instance " + std::to_string(b) + ": " + errs[b]);
            if (cone_bucket_of(h->prep[b].cmax, h->mixed) < 0)
                return fail(HSDE_ERANGE, "instance " + std::to_string(b) + ": clique of size " +
                                              std::to_string(h->prep[b].cmax) + " exceeds " +
                                              std::to_string(cone_max_clique(h->mixed)) + " (" +
                                              (h->mixed ? "mixed" : "FP64") + " eigensolvers)");
        }
    }
    // ---- totals and offsets ----
    int64_t Ntot = 0, Ptot = 0, nnzA = 0, Mtot = 0, ncl = 0, ntiles = 0, sinv = 0, scn = 0;
    int64_t lr_uw = 0, lr_k = 0, lr_hh = 0, lr_bi = 0;   // structured factor pools
    int64_t nlong = 0, sscn = 0;                          // long entries, short copies
    std::vector<int4> lr_tiles;
    h->x_off.resize(B); h->p_off.resize(B); h->m_off.resize(B);
    std::vector<InstDev> inst(B);
    std::vector<int4> hat;   // A^T tiles
    for (int32_t b = 0; b < B; ++b) {
        const HostPrep& H = h->prep[b];
        InstDev& I = inst[b];
        std::memset(&I, 0, sizeof(I));
        I.x_off = Ntot; I.N = H.S.N();
        I.p_off = Ptot; I.P = H.S.P();
        I.m_off = (int32_t)Mtot; I.m = H.m;
        I.cl_begin = (int32_t)ncl; I.cl_end = (int32_t)(ncl + H.S.p());
        I.tile_begin = (int32_t)ntiles;
        ntiles += (I.N + TILE_N - 1) / TILE_N;
        I.tile_end = (int32_t)ntiles;
        I.at_begin = (int32_t)hat.size();
        append_at_tiles(H, b, Ntot, hat);
        I.at_end = (int32_t)hat.size();
        I.dense = H.dense ? (H.lowrank ? 2 : 1) : 0;
        I.sinv_off = sinv;
        if (I.dense == 1) sinv += (int64_t)H.m * H.m;
        if (I.dense == 2) {
            I.lr_r = H.lr.r;
            I.lr_off = lr_uw; I.kinv_off = lr_k; I.h_off = lr_hh;
            lr_uw += (int64_t)H.m * H.lr.r;
            lr_k += (int64_t)H.lr.r * H.lr.r;
            lr_hh += H.lr.r;
            lr_bi += (int64_t)H.lr.binv.size();
            I.lr_tile_begin = (int32_t)lr_tiles.size();
            for (int32_t r0 = 0; r0 < H.m; r0 += LR_TILE)
                lr_tiles.push_back(make_int4(b, (int)(Mtot + r0), (int)(Mtot + std::min(H.m, r0 + LR_TILE)), 0));
            I.lr_tile_end = (int32_t)lr_tiles.size();
        }
        I.status = HSDE_RUNNING;
        I.vcold = 1;
        I.tau = 1.0; I.kappa = 1.0;
        I.sigma = H.sigma; I.rho = H.rho; I.bnorm = H.bnorm; I.cnorm = H.cnorm;
        h->x_off[b] = Ntot; h->p_off[b] = Ptot; h->m_off[b] = (int32_t)Mtot;
        Ntot += I.N; Ptot += I.P; Mtot += H.m; ncl += H.S.p(); nnzA += (int64_t)H.A_col.size();
        scn += (int64_t)H.sc_idx.size();
        for (int64_t e = 0; e < H.S.N(); ++e) {
            const int32_t d = H.sc_ptr[e + 1] - H.sc_ptr[e];
            if (d > LONG_COPIES) ++nlong;
            else sscn += d;
        }
    }
    // the device index arrays (pattern entries, packed positions, constraint
    // rows and the CSR offsets of A and A^T) are 32-bit over the whole batch;
    // the warp-per-row kernels index rows * 32 threads in 32 bits
    {
        constexpr int64_t lim = INT32_MAX;
        if (Ntot > lim || Ptot > lim || Mtot > lim / 32 || nnzA > lim || scn > lim || ncl > lim / 32)
            return fail(HSDE_ERANGE, "batch too large for 32-bit indices: N = " + std::to_string(Ntot) +
                                         ", P = " + std::to_string(Ptot) + ", m = " + std::to_string(Mtot) +
                                         ", nnz(A) = " + std::to_string(nnzA));
    }
    std::vector<int64_t> hvso;
    int64_t vsn = 0;
    if (h->warm) {
        for (int32_t b = 0; b < B; ++b) {
            const Symbolic& S = h->prep[b].S;
            for (int32_t k = 0; k < S.p(); ++k) {
                hvso.push_back(vsn);
                vsn += cone_vstore_elems(S.clique_ptr[k + 1] - S.clique_ptr[k], h->mixed);
            }
        }
    }
    // workspaces of the cliques on the tridiagonal QR path (cone_large.cu)
    std::vector<int64_t> hbigo;
    int64_t bign = 0;
    for (int32_t b = 0; b < B; ++b) {
        const Symbolic& S = h->prep[b].S;
        for (int32_t k = 0; k < S.p(); ++k) {
            const int c = S.clique_ptr[k + 1] - S.clique_ptr[k];
            if (cone_bucket_of(c, h->mixed) == CONE_BIG) {
                hbigo.push_back(bign);
                bign += cone_big_ws_elems(c);
            } else {
                hbigo.push_back(-1);
            }
        }
    }
    const int64_t LIM = (int64_t)1 << 31;
    if (Ntot >= LIM || Ptot >= LIM || nnzA >= LIM || Mtot >= LIM || scn >= LIM)
        return fail(HSDE_ERANGE, "problem totals exceed int32 indexing");

    // ---- device, streams ----
    CK(cudaSetDevice(h->device));
    if (opt.cuda_stream) {
        h->st = reinterpret_cast<cudaStream_t>(opt.cuda_stream);
    } else {
        CK(cudaStreamCreateWithFlags(&h->st, cudaStreamNonBlocking));
        h->own_stream = true;
    }
    for (auto& s : h->side) CK(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    CK(cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming));
    for (auto& e : h->ev_join) CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    CK(cudaMallocHost(&h->host_inst, sizeof(InstDev) * B));
    h->profile = opt.profile != 0;
    if (h->profile) {
        for (cudaEvent_t* e : {&h->ev_it0, &h->ev_aff, &h->ev_chk, &h->ev_it1}) CK(cudaEventCreate(e));
        for (auto& e : h->ev_cs) CK(cudaEventCreate(&e));
        for (auto& e : h->ev_ce) CK(cudaEventCreate(&e));
    }

    // ---- arena layout ----
    const size_t Tsz = h->mixed ? sizeof(float) : sizeof(double);
    Carver cv;
    const size_t o_x = cv.take<double>(Ntot), o_c = cv.take<double>(Ntot), o_id = cv.take<double>(Ntot),
                 o_xp = cv.take<double>(Ntot), o_f = cv.take<double>(Ntot), o_xw = cv.take<double>(Ntot),
                 o_diag = cv.take<uint8_t>(Ntot), o_scp = cv.take<int32_t>(Ntot + 1),
                 o_sci = cv.take<int32_t>(scn), o_atp = cv.take<int32_t>(Ntot + 1),
                 o_atc = cv.take<int32_t>(nnzA), o_atv = cv.take<double>(nnzA);
    const size_t o_y = cv.take<double>(Mtot), o_b = cv.take<double>(Mtot), o_yp = cv.take<double>(Mtot),
                 o_q = cv.take<double>(Mtot), o_yw = cv.take<double>(Mtot),
                 o_ap = cv.take<int32_t>(Mtot + 1), o_ac = cv.take<int32_t>(nnzA),
                 o_av = cv.take<double>(nnzA), o_ri = cv.take<int32_t>(Mtot),
                 o_sd = cv.take<double>(Mtot), o_sinv = cv.take<double>(sinv);
    size_t o_s = cv.take<char>(Ptot * Tsz), o_z = cv.take<char>(Ptot * Tsz), o_v = cv.take<char>(Ptot * Tsz);
    const size_t o_vst = cv.take<char>(vsn * Tsz), o_vso = cv.take<int64_t>(hvso.size());
    const size_t o_bigws = cv.take<char>(bign * Tsz), o_bigo = cv.take<int64_t>(hbigo.size());
    const size_t o_g = cv.take<int32_t>(Ptot), o_clo = cv.take<int32_t>(ncl), o_cls = cv.take<int32_t>(ncl),
                 o_cli = cv.take<int32_t>(ncl), o_inst = cv.take<InstDev>(B), o_tiles = cv.take<int4>(ntiles),
                 o_part = cv.take<double>(ntiles * KPART), o_clp = cv.take<double>(2 * ncl),
                 o_att = cv.take<int4>(hat.size()), o_atpart = cv.take<double>(hat.size()),
                 o_clsw = cv.take<int32_t>(ncl),
                 o_blist = cv.take<int32_t>(ncl),
                 o_rowb = cv.take<double>(Mtot), o_cnt = cv.take<int>(3 * (size_t)B),
                 o_af = cv.take<double>(Mtot), o_atyw = cv.take<double>(Ntot), o_atyp = cv.take<double>(Ntot),
                 o_dinv2 = cv.take<double>(Mtot), o_ax = cv.take<double>(Mtot), o_aty = cv.take<double>(Ntot);
    const size_t o_lrbr = cv.take<int64_t>(Mtot), o_lrmem = cv.take<int32_t>(Mtot), o_lrbsz = cv.take<int32_t>(Mtot),
                 o_lrmembers = cv.take<int32_t>(Mtot), o_lrbinv = cv.take<double>(lr_bi),
                 o_lrU = cv.take<double>(lr_uw), o_lrW = cv.take<double>(lr_uw), o_lrk = cv.take<double>(lr_k),
                 o_lrh = cv.take<double>(lr_hh + 1), o_lrpart = cv.take<double>(lr_tiles.size() * (size_t)LR_RMAX),
                 o_lrtiles = cv.take<int4>(lr_tiles.size());
    const size_t o_sscp = cv.take<int32_t>(Ntot + 1), o_ssci = cv.take<int32_t>(sscn),
                 o_lid = cv.take<int32_t>(Ntot), o_le = cv.take<int32_t>(nlong), o_linst = cv.take<int32_t>(nlong),
                 o_lhz = cv.take<double>(nlong), o_lall = cv.take<double>(nlong);
    // Gauss-Jordan scratch and per-dense-instance tables
    int ndense = 0;
    int32_t mmax = 0;
    for (int32_t b = 0; b < B; ++b)
        if (h->prep[b].dense && !h->prep[b].lowrank) { ++ndense; mmax = std::max(mmax, h->prep[b].m); }
    h->any_dense = ndense > 0;
    const size_t o_gjrow = cv.take<double>(Mtot), o_gjcol = cv.take<double>(Mtot),
                 o_gjoff = cv.take<int64_t>(ndense), o_gjm = cv.take<int32_t>(ndense),
                 o_gjb = cv.take<int64_t>(ndense), o_gjtp = cv.take<int64_t>(ndense + 1);
    h->arena_bytes = cv.off + 256;
    CK(cudaMalloc(&h->arena, h->arena_bytes));
    char* ar = reinterpret_cast<char*>(h->arena);
    DevView& V = h->V;
    V.B = B; V.Ntot = Ntot; V.Ptot = Ptot; V.Mtot = (int32_t)Mtot; V.ntiles = (int32_t)ntiles;
    V.nat = (int32_t)hat.size();
    V.at_tiles = (const int4*)(ar + o_att); V.at_part = (double*)(ar + o_atpart);
    V.ncl = (int32_t)ncl;
    V.x = (double*)(ar + o_x); V.c = (const double*)(ar + o_c); V.inv_delta = (const double*)(ar + o_id);
    V.xp = (double*)(ar + o_xp); V.f = (double*)(ar + o_f); V.xw = (double*)(ar + o_xw);
    V.diag = (const uint8_t*)(ar + o_diag); V.sc_ptr = (const int32_t*)(ar + o_scp);
    V.sc_idx = (const int32_t*)(ar + o_sci); V.At_ptr = (const int32_t*)(ar + o_atp);
    V.At_col = (const int32_t*)(ar + o_atc); V.At_val = (const double*)(ar + o_atv);
    V.y = (double*)(ar + o_y); V.b = (const double*)(ar + o_b); V.yp = (double*)(ar + o_yp);
    V.q = (double*)(ar + o_q); V.yw = (double*)(ar + o_yw); V.A_ptr = (const int32_t*)(ar + o_ap);
    V.A_col = (const int32_t*)(ar + o_ac); V.A_val = (const double*)(ar + o_av);
    V.row_inst = (const int32_t*)(ar + o_ri); V.sdiag = (const double*)(ar + o_sd);
    V.sinv = (double*)(ar + o_sinv);
    V.s = ar + o_s; V.z = ar + o_z; V.v = ar + o_v;
    V.vstore = h->warm ? (void*)(ar + o_vst) : nullptr;
    V.vs_off = (const int64_t*)(ar + o_vso);
    V.big_ws = bign > 0 ? (void*)(ar + o_bigws) : nullptr;
    V.big_off = (const int64_t*)(ar + o_bigo);
    V.gmap = (const int32_t*)(ar + o_g); V.cl_off = (const int32_t*)(ar + o_clo);
    V.cl_size = (const int32_t*)(ar + o_cls); V.cl_inst = (const int32_t*)(ar + o_cli);
    V.inst = (InstDev*)(ar + o_inst); V.tiles = (const int4*)(ar + o_tiles);
    V.part = (double*)(ar + o_part); V.cl_part = (double*)(ar + o_clp);
    V.cl_sweeps = (int32_t*)(ar + o_clsw);
    V.rowb = (double*)(ar + o_rowb);
    V.af = (double*)(ar + o_af);
    V.atyw = (double*)(ar + o_atyw);
    V.atyp = (double*)(ar + o_atyp);
    V.counters = (int*)(ar + o_cnt);
    V.dinv2 = (const double*)(ar + o_dinv2);
    V.lr_binv_row = (const int64_t*)(ar + o_lrbr); V.lr_mem = (const int32_t*)(ar + o_lrmem);
    V.lr_bsz = (const int32_t*)(ar + o_lrbsz); V.lr_members = (const int32_t*)(ar + o_lrmembers);
    V.lr_binv = (const double*)(ar + o_lrbinv); V.lr_U = (const double*)(ar + o_lrU);
    V.lr_W = (const double*)(ar + o_lrW); V.lr_kinv = (const double*)(ar + o_lrk);
    V.lr_h = (double*)(ar + o_lrh); V.lr_part = (double*)(ar + o_lrpart);
    V.lr_tiles = (const int4*)(ar + o_lrtiles); V.nlr = (int32_t)lr_tiles.size();
    V.ssc_ptr = (const int32_t*)(ar + o_sscp); V.ssc_idx = (const int32_t*)(ar + o_ssci);
    V.long_id = (const int32_t*)(ar + o_lid); V.long_e = (const int32_t*)(ar + o_le);
    V.long_inst = (const int32_t*)(ar + o_linst); V.lhz = (double*)(ar + o_lhz); V.lall = (double*)(ar + o_lall);
    V.nlong = (int32_t)nlong;
    V.ax = (double*)(ar + o_ax);
    V.aty = (double*)(ar + o_aty);
    V.eps = opt.eps_tol; V.max_iter = opt.max_iter; V.check_every = opt.check_every;
    V.alpha = opt.alpha;

    // ---- concatenated host buffers with absolute indices ----
    std::vector<double> hc, hid, hAtv, hb, hAv, hsd, hdinv2;
    std::vector<uint8_t> hdiag;
    std::vector<int32_t> hscp, hsci, hatp, hatc, hap, hac, hri, hg, hclo, hcls, hcli;
    std::vector<int32_t> hsscp, hssci, hlid, hle, hlinst;   // short H^T CSR and the long entries
    hsscp.reserve(Ntot + 1); hssci.reserve(sscn); hlid.reserve(Ntot);
    std::vector<int4> htiles;
    hc.reserve(Ntot); hid.reserve(Ntot); hdiag.reserve(Ntot);
    hscp.reserve(Ntot + 1); hatp.reserve(Ntot + 1); hap.reserve(Mtot + 1);
    hsd.assign(Mtot, 0.0);
    for (int32_t b = 0; b < B; ++b) {
        const HostPrep& H = h->prep[b];
        const int64_t xo = h->x_off[b], po = h->p_off[b];
        const int32_t mo = h->m_off[b];
        hc.insert(hc.end(), H.cvec.begin(), H.cvec.end());
        hid.insert(hid.end(), H.inv_delta.begin(), H.inv_delta.end());
        hdiag.insert(hdiag.end(), H.diag.begin(), H.diag.end());
        const int32_t scbase = (int32_t)hsci.size(), atbase = (int32_t)hatc.size(), abase = (int32_t)hac.size();
        for (int64_t e = 0; e < H.S.N(); ++e) {
            hscp.push_back(scbase + H.sc_ptr[e]);
            hatp.push_back(atbase + H.At_ptr[e]);
        }
        for (int32_t j : H.sc_idx) hsci.push_back((int32_t)(po + j));
        for (int64_t e = 0; e < H.S.N(); ++e) {
            hsscp.push_back((int32_t)hssci.size());
            const int32_t j0 = H.sc_ptr[e], j1 = H.sc_ptr[e + 1];
            if (j1 - j0 > LONG_COPIES) {
                hlid.push_back((int32_t)hle.size());
                hle.push_back((int32_t)(xo + e));
                hlinst.push_back(b);
            } else {
                hlid.push_back(-1);
                for (int32_t j = j0; j < j1; ++j) hssci.push_back((int32_t)(po + H.sc_idx[j]));
            }
        }
        for (size_t j = 0; j < H.At_col.size(); ++j) hatc.push_back(mo + H.At_col[j]);
        hAtv.insert(hAtv.end(), H.At_val.begin(), H.At_val.end());
        for (int32_t i = 0; i < H.m; ++i) {
            hap.push_back(abase + H.A_ptr[i]);
            hri.push_back(b);
        }
        for (int32_t e : H.A_col) hac.push_back((int32_t)(xo + e));
        hAv.insert(hAv.end(), H.A_val.begin(), H.A_val.end());
        hb.insert(hb.end(), H.b.begin(), H.b.end());
        for (int32_t i = 0; i < H.m; ++i) hdinv2.push_back(1.0 / (H.dscale[i] * H.dscale[i]));
        if (!H.dense)
            for (int32_t i = 0; i < H.m; ++i) hsd[mo + i] = H.Sdiag_inv[i];
        for (int32_t e : H.S.gather) hg.push_back((int32_t)(xo + e));
        for (int32_t k = 0; k < H.S.p(); ++k) {
            hclo.push_back((int32_t)(po + H.S.packed_ptr[k]));
            hcls.push_back(H.S.clique_ptr[k + 1] - H.S.clique_ptr[k]);
            hcli.push_back(b);
        }
        for (int64_t s0 = 0; s0 < H.S.N(); s0 += TILE_N)
            htiles.push_back(make_int4(b, (int)(xo + s0), (int)(xo + std::min<int64_t>(H.S.N(), s0 + TILE_N)), 0));
    }
    hscp.push_back((int32_t)hsci.size());
    hsscp.push_back((int32_t)hssci.size());
    hatp.push_back((int32_t)hatc.size());
    hap.push_back((int32_t)hac.size());

    cudaStream_t st = h->st;
    CK(cudaMemsetAsync(h->arena, 0, h->arena_bytes, st));
    int rc;
#define UP(off, vec) if ((rc = upload(ar + (off), vec, st)) != HSDE_OK) return rc
    UP(o_c, hc); UP(o_id, hid); UP(o_diag, hdiag); UP(o_scp, hscp); UP(o_sci, hsci);
    UP(o_sscp, hsscp); UP(o_ssci, hssci); UP(o_lid, hlid); UP(o_le, hle); UP(o_linst, hlinst);
    UP(o_atp, hatp); UP(o_atc, hatc); UP(o_atv, hAtv); UP(o_b, hb); UP(o_ap, hap); UP(o_ac, hac);
    UP(o_av, hAv); UP(o_ri, hri); UP(o_sd, hsd); UP(o_g, hg); UP(o_clo, hclo); UP(o_cls, hcls);
    UP(o_cli, hcli); UP(o_vso, hvso); UP(o_bigo, hbigo); UP(o_dinv2, hdinv2);
    {
        // structured factors: per-row block data with absolute indices, pools
        std::vector<int64_t> hbr(Mtot, 0);
        std::vector<int32_t> hmem(Mtot, 0), hbsz(Mtot, 0), hmembers(Mtot, 0);
        std::vector<double> hbinv, hU, hW, hK;
        hbinv.reserve(lr_bi); hU.reserve(lr_uw); hW.reserve(lr_uw); hK.reserve(lr_k);
        for (int32_t b = 0; b < B; ++b) {
            const HostPrep& H = h->prep[b];
            if (!H.lowrank) continue;
            const LowRankHost& L = H.lr;
            const int32_t mo = h->m_off[b];
            const int64_t bo = (int64_t)hbinv.size();
            for (int32_t i = 0; i < H.m; ++i) {
                const int32_t k = L.row_blk[i], bs = L.blk_ptr[k + 1] - L.blk_ptr[k];
                hbr[mo + i] = bo + L.blk_off[k] + (int64_t)L.row_pos[i] * bs;
                hmem[mo + i] = mo + L.blk_ptr[k];
                hbsz[mo + i] = bs;
                hmembers[mo + i] = mo + L.members[i];
            }
            hbinv.insert(hbinv.end(), L.binv.begin(), L.binv.end());
            hU.insert(hU.end(), L.U.begin(), L.U.end());
            hW.insert(hW.end(), L.W.begin(), L.W.end());
            hK.insert(hK.end(), L.kinv.begin(), L.kinv.end());
        }
        UP(o_lrbr, hbr); UP(o_lrmem, hmem); UP(o_lrbsz, hbsz); UP(o_lrmembers, hmembers);
        UP(o_lrbinv, hbinv); UP(o_lrU, hU); UP(o_lrW, hW); UP(o_lrk, hK); UP(o_lrtiles, lr_tiles);
        CK(cudaStreamSynchronize(st));
        for (auto& H : h->prep) H.lr = LowRankHost();
    }
    {
        std::vector<InstDev> iv(inst);
        CK(cudaMemcpyAsync(ar + o_inst, iv.data(), sizeof(InstDev) * B, cudaMemcpyHostToDevice, st));
        CK(cudaMemcpyAsync(ar + o_tiles, htiles.data(), sizeof(int4) * htiles.size(), cudaMemcpyHostToDevice, st));
        if (!hat.empty())
            CK(cudaMemcpyAsync(ar + o_att, hat.data(), sizeof(int4) * hat.size(), cudaMemcpyHostToDevice, st));
        CK(cudaStreamSynchronize(st));
    }
    // ---- dense S: upload and invert in place (Gauss-Jordan, SPD) ----
    if (ndense > 0) {
        // dense instances sorted by m, descending: the active ones at step k are a prefix
        std::vector<int32_t> ord;
        for (int32_t b = 0; b < B; ++b)
            if (h->prep[b].dense && !h->prep[b].lowrank) ord.push_back(b);
        std::stable_sort(ord.begin(), ord.end(), [&](int32_t a, int32_t b) { return h->prep[a].m > h->prep[b].m; });
        std::vector<int64_t> offs, boffs, tpre;
        std::vector<int32_t> ms, rows;
        int64_t acc_tiles = 0;
        for (int32_t b : ord) {
            const HostPrep& H = h->prep[b];
            for (int32_t i = 0; i < H.m; ++i) rows.push_back(inst[b].m_off + i);
            offs.push_back(inst[b].sinv_off);
            ms.push_back(H.m);
            boffs.push_back(inst[b].m_off);
            tpre.push_back(acc_tiles);
            acc_tiles += (int64_t)((H.m + 31) / 32) * ((H.m + 7) / 8);
        }
        tpre.push_back(acc_tiles);
        UP(o_gjoff, offs); UP(o_gjm, ms); UP(o_gjb, boffs); UP(o_gjtp, tpre);
        {
            // S = I + A Delta^{-1} A^T of every dense instance, in the pool
            int32_t* drows = nullptr;
            CK(cudaMalloc(&drows, sizeof(int32_t) * rows.size()));
            const cudaError_t e1 =
                cudaMemcpyAsync(drows, rows.data(), sizeof(int32_t) * rows.size(), cudaMemcpyHostToDevice, st);
            if (e1 == cudaSuccess) launch_form_S(V, drows, (int32_t)rows.size(), mmax, st);
            const cudaError_t e2 = cudaGetLastError();
            const cudaError_t e3 = cudaStreamSynchronize(st);
            cudaFree(drows);
            CK(e1); CK(e2); CK(e3);
        }
        int nact = (int)ord.size();
        for (int32_t k = 0; k < mmax; ++k) {
            while (nact > 0 && ms[nact - 1] <= k) --nact;
            launch_gj_step(V.sinv, (const int64_t*)(ar + o_gjoff), (const int32_t*)(ar + o_gjm),
                           (const int64_t*)(ar + o_gjtp), nact, tpre[nact], k, ms[0],
                           (double*)(ar + o_gjrow), (double*)(ar + o_gjcol), (const int64_t*)(ar + o_gjb), st);
        }
        CK(cudaGetLastError());
        CK(cudaStreamSynchronize(st));
    }
#undef UP
    // ---- the caller's index of every internal constraint row (device copy,
    // for the device-pointer paths), when some instance was reordered ----
    {
        bool any = false;
        for (const HostPrep& H : h->prep) any = any || !H.perm.empty();
        if (any && Mtot > 0) {
            std::vector<int32_t> pm;
            pm.reserve(Mtot);
            for (const HostPrep& H : h->prep)
                for (int32_t j = 0; j < H.m; ++j) pm.push_back(H.perm.empty() ? j : H.perm[j]);
            CK(cudaMalloc(&h->perm_dev, sizeof(int32_t) * pm.size()));
            CK(cudaMemcpy(h->perm_dev, pm.data(), sizeof(int32_t) * pm.size(), cudaMemcpyHostToDevice));
        }
    }
    // ---- cached M^{-1} zeta = (x_p, ., y_p, .) and 1 + zeta^T M^{-1} zeta ----
    launch_rhs(V, h->mixed, Mode::Setup, st);
    launch_spmv_A(V, Mode::Setup, st);
    launch_solve(V, Mode::Setup, st);
    launch_spmv_At(V, Mode::Setup, st);
    launch_setup_den(V, st);
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(st));

    // ---- clique buckets (largest cliques first) ----
    {
        std::vector<int> caps;
        cone_bucket_sizes(caps, h->mixed);
        const int NB = (int)caps.size();
        if (NB > MAX_BUCKETS) return fail(HSDE_ECUDA, "internal: more eigensolver buckets than graph branches");
        std::vector<std::vector<int32_t>> lists(NB);
        std::vector<int32_t> ids(ncl);
        for (int64_t k = 0; k < ncl; ++k) ids[k] = (int32_t)k;
        std::stable_sort(ids.begin(), ids.end(), [&](int32_t a, int32_t b) { return hcls[a] > hcls[b]; });
        std::vector<int64_t> c3(NB, 0);
        for (int32_t k : ids) {
            const int bk = cone_bucket_of(hcls[k], h->mixed);
            for (int t = 0; t < NB; ++t)
                if (caps[t] == bk) { lists[t].push_back(k); c3[t] += (int64_t)hcls[k] * hcls[k] * hcls[k]; }
        }
        int32_t* dl = (int32_t*)(ar + o_blist);
        size_t used = 0;
        for (int t = 0; t < NB; ++t) {
            if (lists[t].empty()) continue;
            CK(cudaMemcpyAsync(dl + used, lists[t].data(), sizeof(int32_t) * lists[t].size(),
                               cudaMemcpyHostToDevice, st));
            h->buckets.push_back(Bucket{caps[t], (int32_t)lists[t].size(), 0, dl + used, hcls[lists[t][0]]});
            h->bucket_c3.push_back(c3[t]);
            h->bucket_ids.push_back(lists[t]);
            used += lists[t].size();
        }
        CK(cudaStreamSynchronize(st));
    }
    if (cone_prepare(h->mixed) != HSDE_OK || rev_prepare(h->mixed) != HSDE_OK)
        return fail(HSDE_ECUDA, "cudaFuncSetAttribute failed");
    if ((rc = choose_variants(h)) != HSDE_OK) return rc;

    // ---- capture one iteration into a graph ----
    h->kernels_per_iter = count_kernels(h);
    if (opt.use_graph) {
        CK(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
        h->capturing = true;
        int rc2 = enqueue_iteration(h);
        h->capturing = false;
        cudaGraph_t g = nullptr;
        cudaError_t e2 = cudaStreamEndCapture(st, &g);
        if (rc2 != HSDE_OK) { if (g) cudaGraphDestroy(g); return rc2; }
        if (e2 != cudaSuccess) return fail(HSDE_ECUDA, std::string("graph capture: ") + cudaGetErrorString(e2));
        h->graph = g;
        CK(cudaGraphInstantiate(&h->exec, g, 0));
    }
    CK(cudaStreamSynchronize(st));
    h->setup_ms = now_ms() - t0;
    *out = h;
    h = nullptr;   // release guard
    return HSDE_OK;
}

int check_handle(const hsde_handle* h, int32_t i) {
    if (!h) return fail(HSDE_EINVAL, "null handle");
    if (i < 0 || i >= h->B) return fail(HSDE_EINVAL, "instance index out of range");
    return HSDE_OK;
}

// An m-vector of one instance from the internal constraint order to the
// caller's (out[perm[i]] = in[i]) and back (out[i] = in[perm[i]]).
void to_caller(const HostPrep& H, const double* in, double* out) {
    for (int32_t i = 0; i < H.m; ++i) out[H.perm[i]] = in[i];
}
void to_internal(const HostPrep& H, const double* in, double* out) {
    for (int32_t i = 0; i < H.m; ++i) out[i] = in[H.perm[i]];
}

// kind = 1 for device (or managed) memory of the handle's GPU, 0 for host
// memory; a pointer into another GPU's memory is refused.
int pointer_kind(const hsde_handle* h, const void* p, int& kind) {
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        kind = 0;
        return HSDE_OK;
    }
    kind = (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) ? 1 : 0;
    if (a.type == cudaMemoryTypeDevice && a.device != h->device)
        return fail(HSDE_EINVAL, "device pointer of another GPU");
    return HSDE_OK;
}

// The m-vector of a single-instance handle between the device (internal
// constraint order) and a caller buffer (host or device memory, the
// caller's order).  Both return with the copy done.
int m_out(hsde_handle* h, double* dst, const double* src) {
    const HostPrep& H = h->prep[0];
    const int32_t m = H.m;
    if (m == 0) return HSDE_OK;
    if (H.perm.empty()) {
        CK(cudaMemcpy(dst, src, sizeof(double) * m, cudaMemcpyDefault));
        return HSDE_OK;
    }
    int kind = 0, rc;
    if ((rc = pointer_kind(h, dst, kind)) != HSDE_OK) return rc;
    if (kind) {
        launch_perm_move(dst, src, h->perm_dev, m, true, h->st);
        CK(cudaGetLastError());
        CK(cudaStreamSynchronize(h->st));
    } else {
        std::vector<double> t(m);
        CK(cudaMemcpy(t.data(), src, sizeof(double) * m, cudaMemcpyDeviceToHost));
        to_caller(H, t.data(), dst);
    }
    return HSDE_OK;
}

int m_in(hsde_handle* h, double* dst, const double* src) {
    const HostPrep& H = h->prep[0];
    const int32_t m = H.m;
    if (m == 0) return HSDE_OK;
    CK(cudaStreamSynchronize(h->st));
    if (H.perm.empty()) {
        CK(cudaMemcpy(dst, src, sizeof(double) * m, cudaMemcpyDefault));
        return HSDE_OK;
    }
    int kind = 0, rc;
    if ((rc = pointer_kind(h, src, kind)) != HSDE_OK) return rc;
    if (kind) {
        launch_perm_move(dst, src, h->perm_dev, m, false, h->st);
        CK(cudaGetLastError());
        CK(cudaStreamSynchronize(h->st));
    } else {
        std::vector<double> t(m);
        to_internal(H, src, t.data());
        CK(cudaMemcpy(dst, t.data(), sizeof(double) * m, cudaMemcpyHostToDevice));
    }
    return HSDE_OK;
}

}  // namespace

extern "C" {

void hsde_default_options(hsde_options* o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->eps_tol = 1e-4;
    o->max_iter = 2000;
    o->check_every = 1;
    o->precision = HSDE_MIXED;
    o->device = 0;
    o->cuda_stream = nullptr;
    o->jacobi_max_sweeps = 0;
    o->use_graph = 1;
    o->jacobi_tol = 0.0;
    o->profile = 0;
    o->warm_start = -1;
    o->warm_refresh = 0;
    o->scaling = 1;
    o->structured_factor = 1;
    o->alpha = 1.8;
    o->scale_norm = 10.0;
    o->dual_weight = 1.5;
    o->autotune = 1;
    o->eigensolver = 0;
}

const char* hsde_last_error(void) { return g_err.c_str(); }

int hsde_analyze(const hsde_problem* P, hsde_symbolic** out) {
    try {
        if (!out) return fail(HSDE_EINVAL, "out is null");
        *out = nullptr;
        auto* s = new hsde_symbolic();
        std::string err;
        int rc = build_symbolic(P, s->S, err);
        if (rc != HSDE_OK) { delete s; return fail(rc, err); }
        *out = s;
        return HSDE_OK;
    } catch (const std::bad_alloc&) {
        return fail(HSDE_ENOMEM, "host allocation failed");
    } catch (...) {
        return fail(HSDE_EINVAL, "unexpected error");
    }
}

static void fill_sizes(const Symbolic& S, int32_t m, int dense, hsde_sizes* o) {
    std::memset(o, 0, sizeof(*o));
    o->n = S.n; o->m = m; o->p = S.p();
    o->N = S.N(); o->P = S.P();
    int64_t nd = 0;
    int32_t cmax = 0;
    for (int32_t k = 0; k < S.p(); ++k) {
        const int64_t c = S.clique_ptr[k + 1] - S.clique_ptr[k];
        nd += c * c;
        cmax = std::max<int32_t>(cmax, (int32_t)c);
    }
    o->n_d = nd; o->c_max = cmax;
    o->state_len = o->N + 3 * o->P + m + 2;
    o->S_dense = dense;
}

int hsde_symbolic_sizes(const hsde_symbolic* s, hsde_sizes* out) {
    if (!s || !out) return fail(HSDE_EINVAL, "null argument");
    fill_sizes(s->S, 0, false, out);
    out->state_len = 0;
    return HSDE_OK;
}

static void copy_structure(const Symbolic& S, int32_t* order, int32_t* clique_ptr, int32_t* clique_idx,
                           int32_t* pat_colptr, int32_t* pat_row, int32_t* gather, int32_t* D) {
    auto cp = [](int32_t* dst, const std::vector<int32_t>& v) {
        if (dst && !v.empty()) std::memcpy(dst, v.data(), v.size() * sizeof(int32_t));
    };
    cp(order, S.order); cp(clique_ptr, S.clique_ptr); cp(clique_idx, S.clique_idx);
    cp(pat_colptr, S.pat_colptr); cp(pat_row, S.pat_row); cp(gather, S.gather); cp(D, S.D);
}

int hsde_symbolic_get(const hsde_symbolic* s, int32_t* order, int32_t* clique_ptr, int32_t* clique_idx,
                      int32_t* pat_colptr, int32_t* pat_row, int32_t* gather, int32_t* D) {
    if (!s) return fail(HSDE_EINVAL, "null symbolic");
    copy_structure(s->S, order, clique_ptr, clique_idx, pat_colptr, pat_row, gather, D);
    return HSDE_OK;
}

void hsde_symbolic_free(hsde_symbolic* s) { delete s; }

int hsde_setup(const hsde_problem* P, const hsde_options* O, hsde_handle** out) {
    return hsde_setup_batch(P, 1, O, out);
}

int hsde_setup_batch(const hsde_problem* P, int32_t B, const hsde_options* O, hsde_handle** out) {
    try {
        return setup_impl(P, B, O, out);
    } catch (const std::bad_alloc&) {
        return fail(HSDE_ENOMEM, "host allocation failed");
    } catch (...) {
        return fail(HSDE_EINVAL, "unexpected error");
    }
}

int hsde_iterate(hsde_handle* h, int32_t k, int32_t* status_out) {
    if (!h) return fail(HSDE_EINVAL, "null handle");
    if (k < 0) return fail(HSDE_EINVAL, "k < 0");
    const double t0 = now_ms();
    CK(cudaSetDevice(h->device));
    if (k > 0 && h->need_rhs) {
        // f of the first iteration (later iterations get it from the previous one)
        launch_rhs(h->V, h->mixed, Mode::Iter, h->st);
        CK(cudaGetLastError());
        h->need_rhs = false;
    }
    for (int32_t it = 0; it < k; ++it) {
        h->launched++;
        if (h->exec) {
            CK(cudaGraphLaunch(h->exec, h->st));
        } else {
            int rc = enqueue_iteration(h);
            if (rc != HSDE_OK) return rc;
        }
    }
    if (status_out) {
        int rc = sync_inst(h);
        if (rc != HSDE_OK) return rc;
        for (int32_t b = 0; b < h->B; ++b) status_out[b] = h->host_inst[b].status;
        h->iterate_ms += now_ms() - t0;
    }
    return HSDE_OK;
}

int hsde_sync(hsde_handle* h) {
    if (!h) return fail(HSDE_EINVAL, "null handle");
    CK(cudaStreamSynchronize(h->st));
    return HSDE_OK;
}

int hsde_num_instances(const hsde_handle* h) { return h ? h->B : 0; }

int hsde_get_sizes(const hsde_handle* h, int32_t i, hsde_sizes* out) {
    int rc = check_handle(h, i);
    if (rc != HSDE_OK) return rc;
    if (!out) return fail(HSDE_EINVAL, "null output");
    fill_sizes(h->prep[i].S, h->prep[i].m, h->prep[i].dense ? (h->prep[i].lowrank ? 2 : 1) : 0, out);
    return HSDE_OK;
}

int hsde_get_structure(const hsde_handle* h, int32_t i, int32_t* order, int32_t* clique_ptr,
                       int32_t* clique_idx, int32_t* pat_colptr, int32_t* pat_row, int32_t* gather,
                       int32_t* D) {
    int rc = check_handle(h, i);
    if (rc != HSDE_OK) return rc;
    copy_structure(h->prep[i].S, order, clique_ptr, clique_idx, pat_colptr, pat_row, gather, D);
    return HSDE_OK;
}

int hsde_get_info(hsde_handle* h, int32_t i, hsde_info* out) {
    int rc = check_handle(h, i);
    if (rc != HSDE_OK) return rc;
    if (!out) return fail(HSDE_EINVAL, "null output");
    if ((rc = sync_inst(h)) != HSDE_OK) return rc;
    const InstDev& I = h->host_inst[i];
    std::memset(out, 0, sizeof(*out));
    out->status = I.status; out->iterations = I.iter;
    out->pres = I.pres; out->dres = I.dres; out->gap = I.gap;
    out->pobj = I.pobj; out->dobj = I.dobj; out->tau = I.tau; out->kappa = I.kappa;
    out->pinf_ratio = I.pinf; out->dinf_ratio = I.dinf;
    out->setup_ms = h->setup_ms; out->iterate_ms = h->iterate_ms;
    out->jacobi_unconverged = I.unconv_last;
    out->jacobi_unconverged_iterations = I.unconv_iters;
    return HSDE_OK;
}

}  // extern "C"

namespace {

// download s/z/v of instance i as doubles
int get_packed(hsde_handle* h, const void* base, int32_t i, double* dst) {
    const int64_t P = h->prep[i].S.P();
    const int64_t po = h->p_off[i];
    if (P == 0) return HSDE_OK;
    if (h->mixed) {
        std::vector<float> tmp(P);
        CK(cudaMemcpy(tmp.data(), (const float*)base + po, sizeof(float) * P, cudaMemcpyDeviceToHost));
        for (int64_t j = 0; j < P; ++j) dst[j] = tmp[j];
    } else {
        CK(cudaMemcpy(dst, (const double*)base + po, sizeof(double) * P, cudaMemcpyDeviceToHost));
    }
    return HSDE_OK;
}

int set_packed(hsde_handle* h, void* base, int32_t i, const double* src) {
    const int64_t P = h->prep[i].S.P();
    const int64_t po = h->p_off[i];
    if (P == 0) return HSDE_OK;
    if (h->mixed) {
        std::vector<float> tmp(P);
        for (int64_t j = 0; j < P; ++j) tmp[j] = (float)src[j];
        CK(cudaMemcpy((float*)base + po, tmp.data(), sizeof(float) * P, cudaMemcpyHostToDevice));
    } else {
        CK(cudaMemcpy((double*)base + po, src, sizeof(double) * P, cudaMemcpyHostToDevice));
    }
    return HSDE_OK;
}

// H^T z for instance i (host scatter over the gather map)
void scatter_host(const HostPrep& H, const double* zp, double* out) {
    const int64_t N = H.S.N();
    std::fill(out, out + N, 0.0);
    for (size_t j = 0; j < H.S.gather.size(); ++j) out[H.S.gather[j]] += zp[j];
}

}  // namespace

extern "C" {

int hsde_get_state(hsde_handle* h, int32_t i, double* state) {
    int rc = check_handle(h, i);
    if (rc != HSDE_OK) return rc;
    if (!state) return fail(HSDE_EINVAL, "null state");
    CK(cudaSetDevice(h->device));
    if ((rc = sync_inst(h)) != HSDE_OK) return rc;
    const HostPrep& H = h->prep[i];
    const int64_t N = H.S.N(), P = H.S.P();
    const int32_t m = H.m;
    double* p = state;
    CK(cudaMemcpy(p, h->V.x + h->x_off[i], sizeof(double) * N, cudaMemcpyDeviceToHost)); p += N;
    if ((rc = get_packed(h, h->V.s, i, p)) != HSDE_OK) return rc; p += P;
    if (m && H.perm.empty()) {
        CK(cudaMemcpy(p, h->V.y + h->m_off[i], sizeof(double) * m, cudaMemcpyDeviceToHost));
    } else if (m) {
        std::vector<double> yi(m);
        CK(cudaMemcpy(yi.data(), h->V.y + h->m_off[i], sizeof(double) * m, cudaMemcpyDeviceToHost));
        to_caller(H, yi.data(), p);
    }
    p += m;
    if ((rc = get_packed(h, h->V.v, i, p)) != HSDE_OK) return rc; p += P;
    *p++ = h->host_inst[i].tau;
    if ((rc = get_packed(h, h->V.z, i, p)) != HSDE_OK) return rc; p += P;
    *p++ = h->host_inst[i].kappa;
    return HSDE_OK;
}

int hsde_set_state(hsde_handle* h, int32_t i, const double* state, int32_t iterations) {
    int rc = check_handle(h, i);
    if (rc != HSDE_OK) return rc;
    if (!state || iterations < 0) return fail(HSDE_EINVAL, "null state or negative iteration count");
    CK(cudaSetDevice(h->device));
    if ((rc = sync_inst(h)) != HSDE_OK) return rc;
    const HostPrep& H = h->prep[i];
    const int64_t N = H.S.N(), P = H.S.P();
    const int32_t m = H.m;
    const double* p = state;
    CK(cudaMemcpy(h->V.x + h->x_off[i], p, sizeof(double) * N, cudaMemcpyHostToDevice)); p += N;
    if ((rc = set_packed(h, h->V.s, i, p)) != HSDE_OK) return rc; p += P;
    if (m && H.perm.empty()) {
        CK(cudaMemcpy(h->V.y + h->m_off[i], p, sizeof(double) * m, cudaMemcpyHostToDevice));
    } else if (m) {
        std::vector<double> yi(m);
        to_internal(H, p, yi.data());
        CK(cudaMemcpy(h->V.y + h->m_off[i], yi.data(), sizeof(double) * m, cudaMemcpyHostToDevice));
    }
    p += m;
    if ((rc = set_packed(h, h->V.v, i, p)) != HSDE_OK) return rc; p += P;
    const double tau = *p++;
    if ((rc = set_packed(h, h->V.z, i, p)) != HSDE_OK) return rc; p += P;
    const double kappa = *p++;
    InstDev I = h->host_inst[i];
    I.tau = tau; I.kappa = kappa; I.status = HSDE_RUNNING; I.iter = iterations; I.eta = 0.0;
    I.vcold = 1;
    h->need_rhs = true;
    CK(cudaMemcpy(h->V.inst + i, &I, sizeof(InstDev), cudaMemcpyHostToDevice));
    h->host_inst[i] = I;
    // the over-relaxation carries A x and A^T y of the iterate from one
    // iteration to the next; form them for the loaded one
    if (h->V.alpha != 1.0) {
        launch_state_products(h->V, h->m_off[i], h->m_off[i] + m, h->x_off[i], h->x_off[i] + N, h->st);
        CK(cudaGetLastError());
        CK(cudaStreamSynchronize(h->st));
    }
    return HSDE_OK;
}

int hsde_get_solution(hsde_handle* h, int32_t i, double* X, double* y, double* Z, double* pobj,
                      double* dobj) {
    int rc = check_handle(h, i);
    if (rc != HSDE_OK) return rc;
    CK(cudaSetDevice(h->device));
    if ((rc = sync_inst(h)) != HSDE_OK) return rc;
    const InstDev& I = h->host_inst[i];
    if (I.status != HSDE_SOLVED) return fail(HSDE_ESTATE, "instance is not solved");
    const HostPrep& H = h->prep[i];
    const int64_t N = H.S.N(), P = H.S.P();
    const double tau = I.tau;
    // unscaled: X = x~/(sigma tau), y = D y~/(rho tau), Z = H^T z~/(rho tau)
    if (X) {
        CK(cudaMemcpy(X, h->V.x + h->x_off[i], sizeof(double) * N, cudaMemcpyDeviceToHost));
        for (int64_t e = 0; e < N; ++e) X[e] /= I.sigma * tau;
    }
    if (y && H.m) {
        std::vector<double> yi(H.m);
        CK(cudaMemcpy(yi.data(), h->V.y + h->m_off[i], sizeof(double) * H.m, cudaMemcpyDeviceToHost));
        for (int32_t j = 0; j < H.m; ++j) yi[j] = H.dscale[j] * yi[j] / (I.rho * tau);
        if (H.perm.empty()) std::copy(yi.begin(), yi.end(), y);
        else to_caller(H, yi.data(), y);
    }
    if (Z) {
        std::vector<double> zp(P);
        if ((rc = get_packed(h, h->V.z, i, zp.data())) != HSDE_OK) return rc;
        scatter_host(H, zp.data(), Z);
        for (int64_t e = 0; e < N; ++e) Z[e] /= I.rho * tau;
    }
    if (pobj) *pobj = I.pobj;
    if (dobj) *dobj = I.dobj;
    return HSDE_OK;
}

int hsde_get_certificate(hsde_handle* h, int32_t i, int32_t kind, double* y, double* Z, double* X) {
    int rc = check_handle(h, i);
    if (rc != HSDE_OK) return rc;
    CK(cudaSetDevice(h->device));
    if ((rc = sync_inst(h)) != HSDE_OK) return rc;
    const InstDev& I = h->host_inst[i];
    if (kind != I.status || (kind != HSDE_PRIMAL_INFEASIBLE && kind != HSDE_DUAL_INFEASIBLE))
        return fail(HSDE_ESTATE, "instance verdict does not match the certificate kind");
    const HostPrep& H = h->prep[i];
    const int64_t N = H.S.N(), P = H.S.P();
    // I.bty = b^T y and I.ctx = c^T x of the unscaled homogeneous iterate
    // (y = D y~/rho, z = z~/rho, x = x~/sigma)
    if (kind == HSDE_PRIMAL_INFEASIBLE) {
        const double bty = I.bty;
        if (y && H.m) {
            std::vector<double> yi(H.m);
            CK(cudaMemcpy(yi.data(), h->V.y + h->m_off[i], sizeof(double) * H.m, cudaMemcpyDeviceToHost));
            for (int32_t j = 0; j < H.m; ++j) yi[j] = H.dscale[j] * yi[j] / I.rho / bty;
            if (H.perm.empty()) std::copy(yi.begin(), yi.end(), y);
            else to_caller(H, yi.data(), y);
        }
        if (Z) {
            std::vector<double> zp(P);
            if ((rc = get_packed(h, h->V.z, i, zp.data())) != HSDE_OK) return rc;
            scatter_host(H, zp.data(), Z);
            for (int64_t e = 0; e < N; ++e) Z[e] = Z[e] / I.rho / bty;
        }
    } else {
        const double nctx = -I.ctx;
        if (X) {
            CK(cudaMemcpy(X, h->V.x + h->x_off[i], sizeof(double) * N, cudaMemcpyDeviceToHost));
            for (int64_t e = 0; e < N; ++e) X[e] = X[e] / I.sigma / nctx;
        }
    }
    return HSDE_OK;
}

int hsde_get_profile(hsde_handle* h, hsde_profile* out) {
    if (!h || !out) return fail(HSDE_EINVAL, "null argument");
    std::memset(out, 0, sizeof(*out));
    out->kernels_per_iteration = h->kernels_per_iter;
    if (h->launched == 0) return HSDE_OK;
    CK(cudaSetDevice(h->device));
    CK(cudaStreamSynchronize(h->st));
    // Jacobi sweeps of the last solve of every clique (with or without the
    // phase events)
    std::vector<int32_t> sw(h->V.ncl);
    if (h->V.ncl > 0)
        CK(cudaMemcpy(sw.data(), h->V.cl_sweeps, sizeof(int32_t) * sw.size(), cudaMemcpyDeviceToHost));
    int64_t tot = 0;
    int32_t mx = 0;
    for (int32_t v : sw) { tot += v; mx = std::max(mx, v); }
    out->sweeps_mean = sw.empty() ? 0.0 : (double)tot / (double)sw.size();
    out->sweeps_max = mx;
    if (!h->profile) return HSDE_OK;
    int np = 0;
    auto put = [&](const char* name, cudaEvent_t a, cudaEvent_t b, int64_t units) -> int {
        if (np >= HSDE_MAX_PHASES) return HSDE_OK;
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, a, b));
        out->phase_ms[np] = ms;
        std::snprintf(out->phase_name[np], sizeof(out->phase_name[np]), "%s", name);
        out->phase_units[np] = units;
        ++np;
        return HSDE_OK;
    };
    int rc;
    if ((rc = put("affine", h->ev_it0, h->ev_aff, h->V.Ntot)) != HSDE_OK) return rc;
    for (size_t i = 0; i < h->buckets.size(); ++i) {
        char nm[24];
        if (h->buckets[i].cmax == CONE_BIG) std::snprintf(nm, sizeof(nm), "cone_qr");
        else std::snprintf(nm, sizeof(nm), "cone_c%d", h->buckets[i].cmax);
        if ((rc = put(nm, h->ev_cs[i], h->ev_ce[i], h->bucket_c3[i])) != HSDE_OK) return rc;
    }
    if ((rc = put("post", h->ev_chk, h->ev_it1, h->V.Ntot)) != HSDE_OK) return rc;
    if ((rc = put("iteration", h->ev_it0, h->ev_it1, h->V.Ntot)) != HSDE_OK) return rc;
    out->nphases = np;
    // cone phases follow "affine" in bucket order
    for (size_t i = 0; i < h->buckets.size() && 1 + i < (size_t)HSDE_MAX_PHASES; ++i) {
        int32_t bm = 0;
        for (int32_t k : h->bucket_ids[i]) bm = std::max(bm, sw[k]);
        out->phase_sweeps_max[1 + i] = bm;
        out->phase_variant[1 + i] = h->buckets[i].variant;
    }
    return HSDE_OK;
}

}  // extern "C"

namespace {

// Allocate (or grow) the reverse-mode workspace for K iterations with a
// checkpoint every ckpt iterations.
int ensure_unroll_ws(hsde_handle* h, int K, int ckpt) {
    UnrollWS& w = h->uw;
    const DevView& V = h->V;
    const size_t T = h->mixed ? sizeof(float) : sizeof(double);
    const int nseg = (K + ckpt - 1) / ckpt;
    const int64_t N = V.Ntot, P = V.Ptot, M = V.Mtot, B = V.B;
    // per-clique tape offsets (CP*CP + CP elements each)
    std::vector<int64_t> tvo;
    int64_t tv = 0;
    for (const auto& H : h->prep)
        for (int32_t k = 0; k < H.S.p(); ++k) {
            const int cp = cone_bucket_of(H.S.clique_ptr[k + 1] - H.S.clique_ptr[k], h->mixed);
            tvo.push_back(tv);
            tv += (int64_t)cp * cp + cp;
        }
    Carver cv;
    const size_t cp_stride = ((N * 8 + 3 * P * T + M * 8 + sizeof(InstDev) * B) + 255) / 256 * 256;
    const size_t o_cp = cv.take<char>(cp_stride * (size_t)nseg);
    const size_t o_tv = cv.take<char>((size_t)tv * T * ckpt), o_ts = cv.take<double>(2 * B * (size_t)ckpt),
                 o_tx = cv.take<double>(N * (size_t)ckpt), o_ty = cv.take<double>(M * (size_t)ckpt);
    const size_t o_xb = cv.take<double>(N), o_yb = cv.take<double>(M), o_as = cv.take<double>(2 * B),
                 o_wt = cv.take<double>(B), o_kp = cv.take<double>(B);
    const size_t o_sb = cv.take<char>(P * T), o_zb = cv.take<char>(P * T), o_vb = cv.take<char>(P * T),
                 o_aws = cv.take<char>(P * T), o_awv = cv.take<char>(P * T);
    const size_t o_f2 = cv.take<double>(N), o_q2 = cv.take<double>(M), o_yw2 = cv.take<double>(M),
                 o_xw2 = cv.take<double>(N), o_p2 = cv.take<double>(V.ntiles), o_e2 = cv.take<double>(B),
                 o_ot = cv.take<double>(B), o_ox = cv.take<double>(N), o_oy = cv.take<double>(M);
    const size_t o_os = cv.take<char>(P * T), o_ov = cv.take<char>(P * T);
    const size_t o_xpn = cv.take<double>(N), o_ypn = cv.take<double>(M), o_dn = cv.take<double>(B),
                 o_cn = cv.take<double>(B), o_gc = cv.take<double>(N), o_gb = cv.take<double>(M),
                 o_tvo = cv.take<int64_t>(tvo.size());
    const size_t bytes = cv.off + 256;
    if (bytes > w.bytes) {
        if (w.mem) CK(cudaFree(w.mem));
        w.mem = nullptr;
        w.bytes = 0;
        CK(cudaMalloc(&w.mem, bytes));
        w.bytes = bytes;
        w.neg_ready = false;
    }
    char* m = reinterpret_cast<char*>(w.mem);
    w.K = K; w.ckpt = ckpt; w.nseg = nseg; w.cp_stride = cp_stride; w.tv_total = tv;
    w.cp = m + o_cp; w.tape_v = m + o_tv; w.tape_scal = (double*)(m + o_ts);
    w.tape_x = (double*)(m + o_tx); w.tape_y = (double*)(m + o_ty);
    w.xbar = (double*)(m + o_xb); w.ybar = (double*)(m + o_yb); w.adj_scal = (double*)(m + o_as);
    w.wtau = (double*)(m + o_wt); w.kpart = (double*)(m + o_kp);
    w.sbar = m + o_sb; w.zbar = m + o_zb; w.vbar = m + o_vb; w.aw_s = m + o_aws; w.aw_v = m + o_awv;
    w.f2 = (double*)(m + o_f2); w.q2 = (double*)(m + o_q2); w.yw2 = (double*)(m + o_yw2);
    w.xw2 = (double*)(m + o_xw2); w.part2 = (double*)(m + o_p2); w.eta2 = (double*)(m + o_e2);
    w.otau = (double*)(m + o_ot); w.ox = (double*)(m + o_ox); w.oy = (double*)(m + o_oy);
    w.os = m + o_os; w.ov = m + o_ov;
    w.xp_neg = (double*)(m + o_xpn); w.yp_neg = (double*)(m + o_ypn);
    w.den_neg = (double*)(m + o_dn); w.ctp_neg = (double*)(m + o_cn);
    w.gc = (double*)(m + o_gc); w.gb = (double*)(m + o_gb);
    w.tv_off = (int64_t*)(m + o_tvo);
    if (!tvo.empty())
        CK(cudaMemcpyAsync(w.tv_off, tvo.data(), sizeof(int64_t) * tvo.size(), cudaMemcpyHostToDevice, h->st));
    return HSDE_OK;
}

// M^{-1} zeta' for the adjoint solve, zeta' = (c, 0, b, 0) (Q with b negated).
int ensure_neg_zeta(hsde_handle* h) {
    UnrollWS& w = h->uw;
    if (w.neg_ready) return HSDE_OK;
    ApplyArgs A{};
    A.wx = h->V.c; A.ws = nullptr; A.wv = nullptr; A.wy = h->V.b; A.wy_sign = 1.0; A.wtau = nullptr; A.sb = -1.0;
    A.den = nullptr; A.f = w.f2; A.q = w.q2; A.yw = w.yp_neg; A.xw = w.xp_neg; A.part = w.part2;
    A.den_out = w.den_neg; A.ctp_out = w.ctp_neg;
    launch_apply(h->V, A, h->mixed, true, h->st);
    CK(cudaGetLastError());
    w.neg_ready = true;
    return HSDE_OK;
}

// The view used while unrolling: no stopping, no warm start, optional tape.
DevView unroll_view(const hsde_handle* h) {
    DevView V = h->V;
    V.eps = -1.0;
    V.max_iter = 0x7fffffff;
    V.vstore = nullptr;
    V.tv_off = h->uw.tv_off;
    V.tape_v = nullptr;
    V.tape_scal = nullptr;
    return V;
}

int reset_standard_start(hsde_handle* h) {
    const DevView& V = h->V;
    const size_t T = h->mixed ? sizeof(float) : sizeof(double);
    CK(cudaMemsetAsync(V.x, 0, sizeof(double) * V.Ntot, h->st));
    CK(cudaMemsetAsync(V.s, 0, T * V.Ptot, h->st));
    CK(cudaMemsetAsync(V.z, 0, T * V.Ptot, h->st));
    CK(cudaMemsetAsync(V.v, 0, T * V.Ptot, h->st));
    if (V.Mtot) CK(cudaMemsetAsync(V.y, 0, sizeof(double) * V.Mtot, h->st));
    if (V.Mtot) CK(cudaMemsetAsync(V.ax, 0, sizeof(double) * V.Mtot, h->st));
    CK(cudaMemsetAsync(V.aty, 0, sizeof(double) * V.Ntot, h->st));
    int rc = sync_inst(h);
    if (rc != HSDE_OK) return rc;
    for (int32_t b = 0; b < h->B; ++b) {
        InstDev& I = h->host_inst[b];
        I.tau = 1.0; I.kappa = 1.0; I.eta = 0.0; I.iter = 0; I.status = HSDE_RUNNING; I.vcold = 1;
    }
    CK(cudaMemcpyAsync(V.inst, h->host_inst, sizeof(InstDev) * h->B, cudaMemcpyHostToDevice, h->st));
    h->need_rhs = true;
    return HSDE_OK;
}

int copy_state(hsde_handle* h, char* dst, bool save) {
    const DevView& V = h->V;
    const size_t T = h->mixed ? sizeof(float) : sizeof(double);
    struct Part { void* dev; size_t n; } parts[] = {
        {V.x, sizeof(double) * V.Ntot}, {V.s, T * V.Ptot}, {V.z, T * V.Ptot}, {V.v, T * V.Ptot},
        {V.y, sizeof(double) * V.Mtot}, {V.inst, sizeof(InstDev) * V.B}};
    size_t off = 0;
    for (auto& p : parts) {
        if (p.n) {
            if (save) CK(cudaMemcpyAsync(dst + off, p.dev, p.n, cudaMemcpyDeviceToDevice, h->st));
            else CK(cudaMemcpyAsync(p.dev, dst + off, p.n, cudaMemcpyDeviceToDevice, h->st));
        }
        off += p.n;
    }
    return HSDE_OK;
}

}  // namespace

extern "C" {

int hsde_set_data(hsde_handle* h, int32_t i, const double* c, const double* b) {
    int rc = check_handle(h, i);
    if (rc != HSDE_OK) return rc;
    if (!c || (!b && h->prep[i].m > 0)) return fail(HSDE_EINVAL, "null data");
    CK(cudaSetDevice(h->device));
    HostPrep& H = h->prep[i];
    const int64_t N = H.S.N();
    int kc, kb = 0;
    if ((rc = pointer_kind(h, c, kc)) != HSDE_OK) return rc;
    if (H.m && (rc = pointer_kind(h, b, kb)) != HSDE_OK) return rc;
    if (H.m && kc != kb) return fail(HSDE_EINVAL, "c and b must both be host or both device pointers");
    double* cdst = const_cast<double*>(h->V.c) + h->x_off[i];
    double* bdst = const_cast<double*>(h->V.b) + h->m_off[i];
    if (kc) {
        // device data: sums and scaled copies by kernels, only 4 doubles per
        // CTA come back to the host
        if (!h->dscale_dev) {
            std::vector<double> d;
            for (const HostPrep& Hb : h->prep) d.insert(d.end(), Hb.dscale.begin(), Hb.dscale.end());
            CK(cudaMalloc(&h->dscale_dev, sizeof(double) * std::max<size_t>(1, d.size())));
            CK(cudaMalloc(&h->data_part, sizeof(double) * 4 * DATA_MAX_CTAS));
            CK(cudaMallocHost(&h->data_part_host, sizeof(double) * 4 * DATA_MAX_CTAS));
            if (!d.empty())
                CK(cudaMemcpy(h->dscale_dev, d.data(), sizeof(double) * d.size(), cudaMemcpyHostToDevice));
        }
        const double* dsc = h->dscale_dev + h->m_off[i];
        const uint8_t* dg = h->V.diag + h->x_off[i];
        const int32_t* pm = H.perm.empty() ? nullptr : h->perm_dev + h->m_off[i];
        launch_data_sums(c, N, dg, b, H.m, dsc, pm, h->data_part, h->st);
        const int nb = data_grid(N, H.m);
        CK(cudaMemcpyAsync(h->data_part_host, h->data_part, sizeof(double) * 4 * nb, cudaMemcpyDeviceToHost,
                           h->st));
        CK(cudaStreamSynchronize(h->st));
        double sm[4] = {0.0, 0.0, 0.0, 0.0};
        for (int k = 0; k < nb; ++k)
            for (int j = 0; j < 4; ++j) sm[j] += h->data_part_host[4 * k + j];
        if (sm[0] != 0.0) return fail(HSDE_EINVAL, "non-finite c or b");
        scale_from_sums(sm[1], sm[2], sm[3], h->opt, H.sigma, H.rho, H.bnorm, H.cnorm);
        launch_data_apply(c, N, H.rho, b, H.m, H.sigma, dsc, pm, cdst, bdst, h->st);
        CK(cudaGetLastError());
    } else {
        for (int64_t e = 0; e < N; ++e)
            if (!std::isfinite(c[e])) return fail(HSDE_EINVAL, "non-finite c");
        for (int32_t j = 0; j < H.m; ++j)
            if (!std::isfinite(b[j])) return fail(HSDE_EINVAL, "non-finite b");
        std::vector<double> bi;
        if (!H.perm.empty()) {
            bi.resize(H.m);
            to_internal(H, b, bi.data());
            b = bi.data();
        }
        // new scaling factors from the new data (D depends on A only)
        scale_factors(H, b, c, h->opt, H.sigma, H.rho, H.bnorm, H.cnorm);
        H.cvec.resize(N);
        for (int64_t e = 0; e < N; ++e) H.cvec[e] = H.rho * c[e];
        H.b.resize(H.m);
        for (int32_t j = 0; j < H.m; ++j) H.b[j] = H.sigma * H.dscale[j] * b[j];
        CK(cudaMemcpy(cdst, H.cvec.data(), sizeof(double) * N, cudaMemcpyHostToDevice));
        if (H.m) CK(cudaMemcpy(bdst, H.b.data(), sizeof(double) * H.m, cudaMemcpyHostToDevice));
    }
    if ((rc = sync_inst(h)) != HSDE_OK) return rc;
    InstDev I = h->host_inst[i];
    I.sigma = H.sigma; I.rho = H.rho; I.bnorm = H.bnorm; I.cnorm = H.cnorm;
    h->host_inst[i] = I;
    CK(cudaMemcpy(h->V.inst + i, &I, sizeof(InstDev), cudaMemcpyHostToDevice));
    // S does not depend on (c, b); M^{-1} zeta and 1 + zeta^T M^{-1} zeta do
    launch_rhs(h->V, h->mixed, Mode::Setup, h->st);
    launch_spmv_A(h->V, Mode::Setup, h->st);
    launch_solve(h->V, Mode::Setup, h->st);
    launch_spmv_At(h->V, Mode::Setup, h->st);
    launch_setup_den(h->V, h->st);
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(h->st));
    h->uw.neg_ready = false;
    h->uw.forward_done = false;
    h->need_rhs = true;
    return HSDE_OK;
}

int hsde_unrolled_forward(hsde_handle* h, int32_t K, int32_t ckpt, double* x, double* y, double* tau,
                          double* kappa) {
    if (!h) return fail(HSDE_EINVAL, "null handle");
    if (h->B != 1) return fail(HSDE_EINVAL, "unrolled differentiation needs a single-instance handle");
    if (K < 1 || ckpt < 1) return fail(HSDE_EINVAL, "K and ckpt must be positive");
    if (h->opt.alpha != 1.0 || h->opt.scaling != 0)
        return fail(HSDE_EINVAL, "unrolled differentiation needs options alpha = 1 and scaling = 0");
    for (const auto& bk : h->buckets)
        if (bk.cmax == CONE_BIG)
            return fail(HSDE_ERANGE, "unrolled differentiation takes cliques up to " +
                                         std::to_string(cone_jacobi_max(h->mixed)) +
                                         " (the Jacobi eigensolvers); this problem has larger ones");
    CK(cudaSetDevice(h->device));
    int rc;
    if ((rc = ensure_unroll_ws(h, K, ckpt)) != HSDE_OK) return rc;
    if ((rc = ensure_neg_zeta(h)) != HSDE_OK) return rc;
    if ((rc = reset_standard_start(h)) != HSDE_OK) return rc;
    UnrollWS& w = h->uw;
    const DevView Vu = unroll_view(h);
    launch_rhs(Vu, h->mixed, Mode::Iter, h->st);
    h->need_rhs = false;
    for (int32_t k = 0; k < K; ++k) {
        if (k % ckpt == 0 && (rc = copy_state(h, w.cp + (size_t)(k / ckpt) * w.cp_stride, true)) != HSDE_OK)
            return rc;
        if ((rc = enqueue_iteration_v(h, Vu, 0, false)) != HSDE_OK) return rc;
    }
    if ((rc = sync_inst(h)) != HSDE_OK) return rc;
    const InstDev& I = h->host_inst[0];
    // caller buffers: host or device memory (unified addressing)
    if (x) CK(cudaMemcpy(x, h->V.x, sizeof(double) * h->V.Ntot, cudaMemcpyDefault));
    if (y && (rc = m_out(h, y, h->V.y)) != HSDE_OK) return rc;
    if (tau) *tau = I.tau;
    if (kappa) *kappa = I.kappa;
    w.forward_done = true;
    return HSDE_OK;
}

int hsde_unrolled_backward(hsde_handle* h, const double* xbar, const double* ybar, double taubar, double kappabar,
                           double* gC, double* gb) {
    if (!h) return fail(HSDE_EINVAL, "null handle");
    UnrollWS& w = h->uw;
    if (!w.forward_done) return fail(HSDE_ESTATE, "hsde_unrolled_forward must run first");
    CK(cudaSetDevice(h->device));
    const DevView& V = h->V;
    const size_t T = h->mixed ? sizeof(float) : sizeof(double);
    cudaStream_t st = h->st;
    // seeds
    // caller buffers: host or device memory (unified addressing)
    if (xbar) CK(cudaMemcpyAsync(w.xbar, xbar, sizeof(double) * V.Ntot, cudaMemcpyDefault, st));
    else CK(cudaMemsetAsync(w.xbar, 0, sizeof(double) * V.Ntot, st));
    if (V.Mtot) {
        if (ybar) {
            int rc0;
            if ((rc0 = m_in(h, w.ybar, ybar)) != HSDE_OK) return rc0;
        }
        else CK(cudaMemsetAsync(w.ybar, 0, sizeof(double) * V.Mtot, st));
    }
    const double sc[2] = {taubar, kappabar};
    CK(cudaMemcpyAsync(w.adj_scal, sc, sizeof(sc), cudaMemcpyHostToDevice, st));
    CK(cudaMemsetAsync(w.sbar, 0, T * V.Ptot, st));
    CK(cudaMemsetAsync(w.zbar, 0, T * V.Ptot, st));
    CK(cudaMemsetAsync(w.vbar, 0, T * V.Ptot, st));
    CK(cudaMemsetAsync(w.gc, 0, sizeof(double) * V.Ntot, st));
    if (V.Mtot) CK(cudaMemsetAsync(w.gb, 0, sizeof(double) * V.Mtot, st));
    RevArgs R{};
    R.tv_off = w.tv_off; R.tape_scal = w.tape_scal; R.tape_x = w.tape_x; R.tape_y = w.tape_y;
    R.xbar = w.xbar; R.ybar = w.ybar; R.sbar = w.sbar; R.zbar = w.zbar; R.vbar = w.vbar;
    R.adj_scal = w.adj_scal; R.wtau = w.wtau; R.kpart = w.kpart; R.aw_s = w.aw_s; R.aw_v = w.aw_v;
    R.otau = w.otau; R.ox = w.ox; R.oy = w.oy; R.os = w.os; R.ov = w.ov; R.gc = w.gc; R.gb = w.gb;
    launch_rev_seed(V, R, st);
    ApplyArgs A{};
    A.wx = w.xbar; A.ws = w.aw_s; A.wv = w.aw_v; A.wy = w.ybar; A.wy_sign = -1.0; A.wtau = w.wtau; A.sb = -1.0;
    A.xp = w.xp_neg; A.yp = w.yp_neg; A.den = w.den_neg; A.ctp = w.ctp_neg;
    A.f = w.f2; A.q = w.q2; A.yw = w.yw2; A.xw = w.xw2; A.part = w.part2; A.eta = w.eta2;
    A.ox = w.ox; A.os = w.os; A.ov = w.ov; A.oy = w.oy; A.otau = w.otau;
    const DevView Vu = unroll_view(h);
    const size_t tvT = (size_t)w.tv_total * T;
    int rc;
    for (int seg = w.nseg - 1; seg >= 0; --seg) {
        const int k0 = seg * w.ckpt;
        const int len = std::min(w.ckpt, w.K - k0);
        if ((rc = copy_state(h, w.cp + (size_t)seg * w.cp_stride, false)) != HSDE_OK) return rc;
        launch_rhs(Vu, h->mixed, Mode::Iter, st);
        for (int j = 0; j < len; ++j) {
            DevView Vt = Vu;
            Vt.tape_v = reinterpret_cast<char*>(w.tape_v) + (size_t)j * tvT;
            Vt.tape_scal = w.tape_scal + (size_t)j * 2 * V.B;
            if ((rc = enqueue_iteration_v(h, Vt, 0, false)) != HSDE_OK) return rc;
            CK(cudaMemcpyAsync(w.tape_x + (size_t)j * V.Ntot, V.x, sizeof(double) * V.Ntot,
                               cudaMemcpyDeviceToDevice, st));
            if (V.Mtot)
                CK(cudaMemcpyAsync(w.tape_y + (size_t)j * V.Mtot, V.y, sizeof(double) * V.Mtot,
                                   cudaMemcpyDeviceToDevice, st));
        }
        for (int j = len - 1; j >= 0; --j) {
            R.tape_v = reinterpret_cast<char*>(w.tape_v) + (size_t)j * tvT;
            launch_rev_scal_pre(R, j, V.B, st);
            for (const auto& bk : h->buckets) {
                rc = launch_rev_clique(Vu, R, bk, h->mixed, st);
                if (rc != HSDE_OK) return fail(rc, "reverse clique launch failed");
            }
            launch_apply(Vu, A, h->mixed, false, st);
            launch_rev_update(Vu, R, j, h->mixed, st);
            launch_rev_scal_post(R, V.B, st);
        }
    }
    launch_rev_finish(V, R, st);
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(st));
    if (gC) CK(cudaMemcpy(gC, w.gc, sizeof(double) * V.Ntot, cudaMemcpyDefault));
    if (gb && V.Mtot && (rc = m_out(h, gb, w.gb)) != HSDE_OK) return rc;
    h->need_rhs = true;
    return HSDE_OK;
}

void hsde_destroy(hsde_handle* h) {
    if (!h) return;
    cudaSetDevice(h->device);
    free_handle(h);
}

}  // extern "C"
