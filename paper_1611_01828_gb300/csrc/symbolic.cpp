// Host symbolic analysis (Section 2.1-2.2 and the selectors of Section 3.1):
// aggregate pattern, chordal extension by exact minimum degree, maximal
// cliques in natural order, the gather map of H_k = E_Ck (x) E_Ck and
// D = H^T H (Section 4.3).  Integer work, deterministic.
//
// Rules (the paper names no extension method):
//  * eliminate the alive vertex of smallest degree in the elimination graph,
//    ties to the smallest index; its alive neighbourhood becomes a clique;
//  * candidate K_v = {v} U N(v); maximal cliques are the candidates contained
//    in no other candidate, ordered by elimination step, members ascending;
//  * E' (lower, CSC order) = the edges {v, u}, u in N(v), plus the diagonal;
//  * packed clique order: (a,b), b = 0..c-1, a = b..c-1.
#include <algorithm>
#include <cstdint>
#include <cmath>
#include <functional>
#include <queue>
#include <utility>

#include "internal.h"

namespace hsde {

namespace {

// Set of vertex indices with O(1) insert / erase / membership (open
// addressing, linear probing, tombstones).  Used for the neighbourhoods of
// high-degree vertices during the elimination, where a sorted-vector union
// would cost the whole neighbourhood per update (an arrow vertex adjacent to
// every other vertex made the analysis quadratic in n).
class VSet {
  public:
    size_t size() const { return live_; }
    bool insert(int32_t k) {
        if ((used_ + 1) * 2 > slots_.size()) {
            size_t n = 64;
            while (n < 4 * (live_ + 1)) n *= 2;      // tombstones are dropped by the rehash
            rehash(n);
        }
        size_t i = slot(k), tomb = SIZE_MAX;
        while (slots_[i] != EMPTY) {
            if (slots_[i] == k) return false;
            if (slots_[i] == TOMB && tomb == SIZE_MAX) tomb = i;
            i = (i + 1) & (slots_.size() - 1);
        }
        if (tomb != SIZE_MAX) {
            slots_[tomb] = k;
        } else {
            slots_[i] = k;
            ++used_;
        }
        ++live_;
        return true;
    }
    void erase(int32_t k) {
        if (slots_.empty()) return;
        size_t i = slot(k);
        while (slots_[i] != EMPTY) {
            if (slots_[i] == k) {
                slots_[i] = TOMB;
                --live_;
                return;
            }
            i = (i + 1) & (slots_.size() - 1);
        }
    }
    void to_sorted(std::vector<int32_t>& out) const {
        out.clear();
        out.reserve(live_);
        for (int32_t k : slots_)
            if (k >= 0) out.push_back(k);
        std::sort(out.begin(), out.end());
    }

  private:
    static constexpr int32_t EMPTY = -1, TOMB = -2;
    std::vector<int32_t> slots_;
    size_t used_ = 0, live_ = 0;
    size_t slot(int32_t k) const { return ((uint32_t)k * 2654435761u) & (slots_.size() - 1); }
    void rehash(size_t n) {
        std::vector<int32_t> old;
        old.swap(slots_);
        slots_.assign(n, EMPTY);
        used_ = live_ = 0;
        for (int32_t k : old)
            if (k >= 0) insert(k);
    }
};

// Neighbourhoods above this size live in a VSet instead of a sorted vector.
constexpr size_t BIG_DEGREE = 256;

}  // namespace

int32_t Symbolic::pos(int32_t r, int32_t c) const {
    if (c < 0 || c >= n) return -1;
    auto b = pat_row.begin() + pat_colptr[c];
    auto e = pat_row.begin() + pat_colptr[c + 1];
    auto it = std::lower_bound(b, e, r);
    if (it == e || *it != r) return -1;
    return (int32_t)(it - pat_row.begin());
}

static bool check_coo(int32_t n, int64_t nnz, const int32_t* r, const int32_t* c, const double* v,
                      const char* what, std::string& err) {
    if (nnz < 0 || (nnz > 0 && (!r || !c || !v))) {
        err = std::string(what) + ": null pointer or negative count";
        return false;
    }
    // entries given in (column, row) order, the usual case, need no sort:
    // strictly increasing keys have no duplicate
    bool increasing = true;
    int64_t prev = -1;
    for (int64_t k = 0; k < nnz; ++k) {
        if (r[k] < 0 || r[k] >= n || c[k] < 0 || c[k] >= n) {
            err = std::string(what) + ": index out of range";
            return false;
        }
        const int64_t key = (int64_t)c[k] * n + r[k];
        if (key <= prev) {
            increasing = false;
            break;
        }
        prev = key;
    }
    std::vector<int64_t> keys;
    if (!increasing) keys.reserve((size_t)nnz);
    for (int64_t k = 0; k < nnz; ++k) {
        if (r[k] < 0 || r[k] >= n || c[k] < 0 || c[k] >= n) {
            err = std::string(what) + ": index out of range";
            return false;
        }
        if (r[k] < c[k]) {
            err = std::string(what) + ": upper-triangle entry (row < col)";
            return false;
        }
        if (v && !std::isfinite(v[k])) {
            err = std::string(what) + ": non-finite value";
            return false;
        }
        if (!increasing) keys.push_back((int64_t)c[k] * n + r[k]);
    }
    std::sort(keys.begin(), keys.end());
    if (std::adjacent_find(keys.begin(), keys.end()) != keys.end()) {
        err = std::string(what) + ": duplicate entry";
        return false;
    }
    return true;
}

int build_symbolic(const hsde_problem* P, Symbolic& S, std::string& err) {
    if (!P) { err = "null problem"; return HSDE_EINVAL; }
    const int32_t n = P->n, m = P->m;
    if (n <= 0) { err = "n must be positive"; return HSDE_EINVAL; }
    if (m < 0) { err = "m must be non-negative"; return HSDE_EINVAL; }
    if (!check_coo(n, P->C_nnz, P->C_row, P->C_col, P->C_val, "C", err)) return HSDE_EINVAL;
    if (m > 0 && (!P->A_ptr || !P->b)) { err = "A_ptr or b is null"; return HSDE_EINVAL; }
    if (m > 0) {
        if (P->A_ptr[0] != 0) { err = "A_ptr[0] must be 0"; return HSDE_EINVAL; }
        for (int32_t i = 0; i < m; ++i) {
            if (P->A_ptr[i + 1] < P->A_ptr[i]) { err = "A_ptr not monotone"; return HSDE_EINVAL; }
            if (!std::isfinite(P->b[i])) { err = "b: non-finite value"; return HSDE_EINVAL; }
        }
        const int64_t a0 = P->A_ptr[0];
        for (int32_t i = 0; i < m; ++i) {
            const int64_t s = P->A_ptr[i] - a0, e = P->A_ptr[i + 1] - a0;
            if (!check_coo(n, e - s, P->A_row + s, P->A_col + s, P->A_val + s, "A_i", err))
                return HSDE_EINVAL;
        }
    }
    if (P->pattern_nnz > 0 &&
        !check_coo(n, P->pattern_nnz, P->pattern_row, P->pattern_col, nullptr, "pattern", err)) {
        // duplicates in the optional pattern are harmless; re-check without them
        if (err.find("duplicate") == std::string::npos) return HSDE_EINVAL;
        err.clear();
    }

    // ---- aggregate pattern: adjacency (off-diagonal) as sorted lists ----
    // The constraint matrices of clique-local problems repeat the same
    // entries many times (5M entries for 30k distinct ones on a block-arrow
    // with d = 50), so the entries are bucketed by column (counting sort)
    // and de-duplicated with a stamp per row, in time linear in the input.
    const int64_t annz = m > 0 ? P->A_ptr[m] - P->A_ptr[0] : 0;
    const int32_t* Ar = m > 0 ? P->A_row : nullptr;
    const int32_t* Ac = m > 0 ? P->A_col : nullptr;
    std::vector<int64_t> cptr(n + 1, 0);
    auto each_entry = [&](auto&& fn) {
        for (int64_t k = 0; k < P->C_nnz; ++k) fn(P->C_row[k], P->C_col[k]);
        for (int64_t k = 0; k < annz; ++k) fn(Ar[k], Ac[k]);
        for (int64_t k = 0; k < P->pattern_nnz; ++k) fn(P->pattern_row[k], P->pattern_col[k]);
    };
    each_entry([&](int32_t r, int32_t c) { if (r != c) ++cptr[c + 1]; });
    for (int32_t j = 0; j < n; ++j) cptr[j + 1] += cptr[j];
    std::vector<int32_t> rows_by_col((size_t)cptr[n]);
    {
        std::vector<int64_t> fill(cptr.begin(), cptr.end() - 1);
        each_entry([&](int32_t r, int32_t c) { if (r != c) rows_by_col[(size_t)fill[c]++] = r; });
    }
    std::vector<std::vector<int32_t>> adj(n);
    {
        std::vector<int32_t> stamp(n, -1);
        for (int32_t j = 0; j < n; ++j)
            for (int64_t k = cptr[j]; k < cptr[j + 1]; ++k) {
                const int32_t r = rows_by_col[(size_t)k];
                if (stamp[r] == j) continue;
                stamp[r] = j;
                adj[r].push_back(j);
                adj[j].push_back(r);
            }
    }
    std::vector<int32_t>().swap(rows_by_col);
    for (auto& a : adj) std::sort(a.begin(), a.end());

    // ---- exact minimum degree ----
    S.n = n;
    S.order.clear();
    S.order.reserve(n);
    std::vector<std::vector<int32_t>> cand;     // K_v in elimination order (sorted)
    cand.reserve(n);
    std::vector<char> alive(n, 1);
    // a vertex's neighbourhood is the sorted vector adj[v] or, once it is
    // large, the hash set big[v] (is_big[v]); the sets are the same either way
    std::vector<VSet> big(n);
    std::vector<char> is_big(n, 0);
    auto degree = [&](int32_t v) -> int64_t { return is_big[v] ? (int64_t)big[v].size() : (int64_t)adj[v].size(); };
    using QE = std::pair<int64_t, int32_t>;
    std::priority_queue<QE, std::vector<QE>, std::greater<QE>> heap;
    for (int32_t v = 0; v < n; ++v) heap.push({(int64_t)adj[v].size(), v});
    std::vector<int32_t> merged;
    while (!heap.empty()) {
        const QE top = heap.top();
        heap.pop();
        const int32_t v = top.second;
        if (!alive[v] || top.first != degree(v)) continue;
        std::vector<int32_t> nb;
        if (is_big[v]) {
            big[v].to_sorted(nb);
            big[v] = VSet();
        } else {
            nb = std::move(adj[v]);
        }
        adj[v].clear();
        S.order.push_back(v);
        std::vector<int32_t> K = nb;
        K.insert(std::upper_bound(K.begin(), K.end(), v), v);
        cand.push_back(std::move(K));
        alive[v] = 0;
        for (int32_t u : nb) {
            // N(u) <- (N(u) U N(v)) minus {u, v}
            if (is_big[u]) {
                for (int32_t w : nb)
                    if (w != u) big[u].insert(w);
                big[u].erase(v);
                continue;
            }
            auto& au = adj[u];
            merged.clear();
            merged.reserve(au.size() + nb.size());
            std::set_union(au.begin(), au.end(), nb.begin(), nb.end(), std::back_inserter(merged));
            merged.erase(std::remove_if(merged.begin(), merged.end(),
                                        [&](int32_t w) { return w == u || w == v; }),
                         merged.end());
            au.swap(merged);
            if (au.size() > BIG_DEGREE) {
                for (int32_t w : au) big[u].insert(w);
                is_big[u] = 1;
                std::vector<int32_t>().swap(au);
            }
        }
        for (int32_t u : nb) heap.push({degree(u), u});
    }

    // ---- maximal cliques ----
    std::vector<int32_t> step(n);
    for (int32_t t = 0; t < n; ++t) step[S.order[t]] = t;
    std::vector<std::vector<int32_t>> earlier(n);
    for (int32_t t = 0; t < n; ++t) {
        const int32_t v = S.order[t];
        for (int32_t u : cand[t])
            if (u != v) earlier[step[u]].push_back(t);
    }
    S.clique_ptr.assign(1, 0);
    S.clique_idx.clear();
    for (int32_t t = 0; t < n; ++t) {
        bool maximal = true;
        for (int32_t s : earlier[t]) {
            if (std::includes(cand[s].begin(), cand[s].end(), cand[t].begin(), cand[t].end())) {
                maximal = false;
                break;
            }
        }
        if (!maximal) continue;
        S.clique_idx.insert(S.clique_idx.end(), cand[t].begin(), cand[t].end());
        S.clique_ptr.push_back((int32_t)S.clique_idx.size());
    }

    // ---- chordal pattern E' in CSC-lower order ----
    std::vector<std::vector<int32_t>> col(n);
    for (int32_t j = 0; j < n; ++j) col[j].push_back(j);
    for (int32_t t = 0; t < n; ++t) {
        const int32_t v = S.order[t];
        for (int32_t u : cand[t]) {
            if (u == v) continue;
            col[std::min(u, v)].push_back(std::max(u, v));
        }
    }
    S.pat_colptr.assign(n + 1, 0);
    S.pat_row.clear();
    S.pat_col.clear();
    for (int32_t j = 0; j < n; ++j) {
        auto& cj = col[j];
        std::sort(cj.begin(), cj.end());
        cj.erase(std::unique(cj.begin(), cj.end()), cj.end());
        S.pat_row.insert(S.pat_row.end(), cj.begin(), cj.end());
        S.pat_col.insert(S.pat_col.end(), cj.size(), j);
        S.pat_colptr[j + 1] = (int32_t)S.pat_row.size();
    }

    // ---- gather map (H) and D = H^T H ----
    const int32_t p = S.p();
    S.packed_ptr.assign(p + 1, 0);
    S.gather.clear();
    for (int32_t k = 0; k < p; ++k) {
        const int32_t* mem = S.clique_idx.data() + S.clique_ptr[k];
        const int32_t c = S.clique_ptr[k + 1] - S.clique_ptr[k];
        for (int32_t b = 0; b < c; ++b)
            for (int32_t a = b; a < c; ++a) {
                const int32_t e = S.pos(mem[a], mem[b]);
                if (e < 0) { err = "internal: clique entry missing from E'"; return HSDE_EINVAL; }
                S.gather.push_back(e);
            }
        S.packed_ptr[k + 1] = (int64_t)S.gather.size();
    }
    S.D.assign(S.N(), 0);
    for (int32_t e : S.gather) S.D[e] += 1;
    return HSDE_OK;
}

}  // namespace hsde
