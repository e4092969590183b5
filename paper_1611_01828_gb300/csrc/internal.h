// Internal declarations shared by the translation units of libhsde.
// Not part of the public ABI (see include/hsde.h).
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "hsde.h"

namespace hsde {

// ---------------------------------------------------------------------------
// Host-side symbolic analysis of one instance (Section 2.1-2.2, Section 4.3)
// ---------------------------------------------------------------------------
struct Symbolic {
    int32_t n = 0;
    std::vector<int32_t> order;        // vertex eliminated at each step
    std::vector<int32_t> clique_ptr;   // [p+1]
    std::vector<int32_t> clique_idx;   // members, ascending within a clique
    std::vector<int32_t> pat_colptr;   // [n+1]  CSC lower pattern E'
    std::vector<int32_t> pat_row;      // [N]
    std::vector<int32_t> pat_col;      // [N]
    std::vector<int64_t> packed_ptr;   // [p+1]
    std::vector<int32_t> gather;       // [P] packed clique entry -> pattern position
    std::vector<int32_t> D;            // [N] cliques containing each entry

    int64_t N() const { return (int64_t)pat_row.size(); }
    int32_t p() const { return (int32_t)clique_ptr.size() - 1; }
    int64_t P() const { return packed_ptr.empty() ? 0 : packed_ptr.back(); }
    int32_t pos(int32_t r, int32_t c) const;   // -1 if (r,c) not in E'
};

// Records the message returned by hsde_last_error() on this thread; returns code.
int set_error(int code, const std::string& msg);

// Validates the problem and runs the analysis; returns HSDE_OK or HSDE_EINVAL.
int build_symbolic(const hsde_problem* P, Symbolic& S, std::string& err);

// ---------------------------------------------------------------------------
// Per-instance scalars that live on the device (one record per instance).
// ---------------------------------------------------------------------------
struct InstDev {
    // offsets into the concatenated arrays
    int64_t x_off, N;        // pattern entries
    int64_t p_off, P;        // packed clique entries
    int64_t sinv_off;        // dense S^{-1} offset in the pool (doubles)
    int64_t lr_off;          // offset of this instance's U and W (m x r each) in their pools
    int64_t kinv_off;        // offset of K^{-1} (r x r)
    int64_t h_off;           // offset of the r-vector h of the current solve
    int32_t m_off, m;        // constraints
    int32_t cl_begin, cl_end;      // cliques
    int32_t tile_begin, tile_end;  // N-space tiles
    int32_t at_begin, at_end;      // A^T tiles (nonzero-balanced, k_bwd_eta)
    int32_t dense;           // S stored diagonal (0), as a dense inverse (1), or as
                             // block-diagonal plus low rank (2, factor.cu)
    int32_t lr_r;            // rank of the low-rank part (dense == 2)
    int32_t lr_tile_begin, lr_tile_end;   // its row tiles (k_lr_t / k_lr_y)
    int32_t status;          // HSDE_RUNNING ...
    int32_t iter;            // iterations done
    int32_t vcold;           // 1: the stored eigenbases are not valid (cold start next)
    int32_t unconv;          // cliques whose eigensolve stopped at max_sweeps above the
                             // tolerance in the current iteration (k_cone counts)
    int32_t unconv_last;     // the same count for the last completed iteration
    int32_t unconv_iters;    // iterations with at least one such clique
    // cached by setup
    double den;              // 1 + zeta^T M^{-1} zeta
    double ctp;              // c^T x_p - b^T y_p
    double bnorm, cnorm;     // ||b||, ||c|| of the original data (full-vec norms)
    double sigma, rho;       // data scaling: b~ = sigma D b, c~ = rho c (1, 1 unscaled)
    // iterate scalars
    double tau, kappa, eta;
    // last check
    double pres, dres, gap, pobj, dobj, pinf, dinf, ctx, bty;
    // omega_tau = tau + kappa of the current iteration (before the update),
    // from k_bwd_eta to k_post
    double ot_prev;
};

// Number of partial sums stored per N-space tile.
constexpr int KPART = 10;
// A certificate's two terms must cancel to this fraction of their size
// (reading P6: the ratio to b^T y or -c^T x alone is not scale-invariant).
constexpr double CERT_CANCEL = 1e-2;
// Entries per N-space tile (one CTA of 256 threads each).
constexpr int TILE_N = 256;
// Copies above which an entry's H^T sums are formed by a CTA of its own.
constexpr int LONG_COPIES = 32;
// Nonzeros of A^T per A^T tile (whole rows; a longer row is a tile alone).
constexpr int AT_TILE_NNZ = 4096;
// Nonzeros of one A^T row per lane of its reducing group (k_bwd_eta).
constexpr int AT_LANE_NNZ = 12;

// Device view of the whole batch (plain pointers into one arena).
struct DevView {
    int32_t B;
    int64_t Ntot, Ptot;
    int32_t Mtot, ntiles, ncl, nat;
    // N space
    double* x; const double* c; const double* inv_delta; double* xp;
    double* f; double* xw;
    const uint8_t* diag;
    const int32_t* sc_ptr; const int32_t* sc_idx;        // H^T as CSR over entries
    // entries in more than LONG_COPIES cliques (the arrow corner of a
    // block-arrow is in every clique) are summed by k_long, a CTA each; the
    // other copies form the short CSR that k_post stages tile by tile
    const int32_t* ssc_ptr; const int32_t* ssc_idx;      // H^T without the long entries
    const int32_t* long_id;  // [Ntot] index of a long entry, -1 otherwise
    const int32_t* long_e;   // [nlong] its pattern entry
    const int32_t* long_inst;   // [nlong] its instance
    double* lhz;             // [nlong] (H^T z) of the long entry
    double* lall;            // [nlong] (H^T (s + z + v)) of the long entry
    int32_t nlong;
    const int32_t* At_ptr; const int32_t* At_col; const double* At_val;
    // m space
    double* y; const double* b; double* yp; double* q; double* yw;
    const int32_t* A_ptr; const int32_t* A_col; const double* A_val;   // weighted
    const int32_t* row_inst;
    const double* sdiag;     // diagonal S^{-1}
    double* sinv;            // dense S^{-1} pool
    // packed clique space (float or double)
    void* s; void* z; void* v;
    const int32_t* gmap;     // absolute x index per packed entry
    void* vstore;            // per-clique eigenbasis of the last solve (warm start), or null
    void* big_ws;            // workspaces of the cliques on the tridiagonal QR path (cone_large.cu)
    const int64_t* big_off;  // [ncl] offset of each such clique's workspace (elements), -1 otherwise
    const int64_t* vs_off;   // [ncl] offset of each clique's CP x CP basis in vstore
    const int32_t* cl_off; const int32_t* cl_size; const int32_t* cl_inst;
    // instances and tiles
    InstDev* inst;
    const int4* tiles;       // (inst, begin, end, 0)
    double* part;            // [ntiles * KPART]
    const int4* at_tiles;    // (inst, begin, end, lanes per row; NT: whole CTA on one row)
    double* at_part;         // [nat] c^T x_w partial of each A^T tile
    double* cl_part;         // [2 ncl]: per clique ||H_k x - s_k||^2 and ||s_k||^2 (full-vec)
    int32_t* cl_sweeps;      // [ncl] Jacobi sweeps used by each clique in its last solve
    double* rowb;            // [Mtot] b_i (y_w)_i
    double* af;              // [Mtot] A f of the current iteration
    const double* dinv2;     // [Mtot] 1 / d_i^2 (row scaling D; 1 unscaled)
    double* ax;              // [Mtot] A x of the current iterate (over-relaxation)
    double* aty;             // [Ntot] A^T y of the current iterate (over-relaxation)
    // structured S = B + U U^T (instances with dense == 2; factor.cu)
    const int64_t* lr_binv_row;  // [Mtot] offset of the row's row of its block inverse
    const int32_t* lr_mem;       // [Mtot] offset of the row's block members in lr_members
    const int32_t* lr_bsz;       // [Mtot] size of the row's block (0: not structured)
    const int32_t* lr_members;   // absolute constraint rows of every block
    const double* lr_binv;       // block inverses, row-major, concatenated
    const double* lr_U;          // U, m x r row-major per instance
    const double* lr_W;          // W = B^{-1} U, same layout
    const double* lr_kinv;       // K^{-1}, r x r per instance
    double* lr_h;                // h of the current solve, r per instance
    double* lr_part;             // [nlr * LR_RMAX] tile partials of U^T t
    const int4* lr_tiles;        // (instance, first row, end row, 0)
    int32_t nlr;                 // number of row tiles of structured instances
    // reverse-mode tape of one iteration (null when not recording)
    void* tape_v;            // per clique: CP x CP eigenvectors, then CP eigenvalues
    const int64_t* tv_off;   // [ncl] offset of each clique's tape block (elements)
    double* tape_scal;       // [2B] tau_hat and tau_hat - kappa
    double* atyw;            // [Ntot] A^T y_w of the current iteration
    double* atyp;            // [Ntot] A^T y_p (setup)
    int* counters;           // [3B] completion counters of k_bwd_eta, k_post and k_lr_t
    // options
    double eps;
    double alpha;            // over-relaxation (1: the literal Eqs. Step1-Step3)
    int32_t max_iter, check_every;
};

// Arguments of one affine apply u_hat = (I + Q(c, sb*b))^{-1} omega.
struct ApplyArgs {
    const double* wx; const void* ws; const void* wv; const double* wy; double wy_sign;
    const double* wtau;      // [B] omega_tau (null: 0)
    double sb;               // sign of b in Q
    const double* xp; const double* yp; const double* den; const double* ctp;   // M^{-1} zeta for sb
    double* f; double* q; double* yw; double* xw; double* part; double* eta;    // scratch
    double* ox; void* os; void* ov; double* oy; double* otau;                    // u_hat
    double* den_out; double* ctp_out;    // setup mode (den == null)
};

// Reverse-mode buffers.
struct RevArgs {
    void* tape_v; const int64_t* tv_off; double* tape_scal; double* tape_x; double* tape_y;
    double* xbar; double* ybar; void* sbar; void* zbar; void* vbar;
    double* adj_scal;        // [2B] (tau_bar, kappa_bar)
    double* wtau;            // [B]
    double* kpart;           // [B]
    void* aw_s; void* aw_v;
    const double* otau; const double* ox; const double* oy; const void* os; const void* ov;
    double* gc; double* gb;
};

// Structured factor limits: blocks of at most LR_BMAX constraints, at most
// LR_RMAX low-rank columns, LR_TILE rows per tile of the structured solve.
constexpr int LR_BMAX = 128;
constexpr int LR_RMAX = 64;
constexpr int LR_TILE = 64;

// Host-built structured form of S for one instance (factor.cu).
struct LowRankHost {
    int32_t r = 0;
    std::vector<int32_t> blk_ptr;   // [nb+1] into members
    std::vector<int32_t> members;   // constraints grouped by block, ascending within
    std::vector<int32_t> row_blk;   // [m] block of each constraint
    std::vector<int32_t> row_pos;   // [m] its position in the block
    std::vector<int64_t> blk_off;   // [nb] offset of each block's inverse in binv
    std::vector<double> binv;       // block inverses, row-major
    std::vector<double> U, W;       // [m r] row-major
    std::vector<double> kinv;       // [r r]
};
// Builds B, U, W, K^{-1} from A^T (CSR over pattern entries, raw values), the
// diagonal flags and Delta^{-1}; false if the structure does not pay (a block
// above LR_BMAX, more than LR_RMAX long entries, or no saving over a dense
// inverse), in which case S stays dense.
bool build_lowrank(int32_t m, int64_t N, const int32_t* At_ptr, const int32_t* At_col, const double* At_val,
                   const uint8_t* diag, const double* inv_delta, LowRankHost& L);
// y = S^{-1} q for the structured instances (rowb: b_i y_i on iterations, or null)
void launch_lr_solve(const DevView& V, const double* qin, double* yout, double* rowb, bool iter, void* st);

// Most eigensolver buckets (graph branches, side streams) of one handle.
constexpr int MAX_BUCKETS = 20;
// Bucket id (and largest clique) of the tridiagonal QR path that takes the
// cliques above the Jacobi bucket sizes (cone_large.cu).
constexpr int CONE_BIG = 1024;

// Bucket of cliques handled by one eigensolver variant.
struct Bucket {
    int32_t cmax;            // padded size CP of the bucket (4 ... 112), CONE_BIG for the QR path
    int32_t count;
    int32_t variant;         // 0 latency, 1 throughput, 2 register-V variant (cone.cu),
                             // 3 warp tridiagonal QR (cone_large.cu)
    int32_t* list;           // device array of clique ids (largest first)
    int32_t csize_max;       // size of the bucket's largest clique
};

// ---------------------------------------------------------------------------
// Launchers (defined in the .cu files).  All enqueue on `st`.
// ---------------------------------------------------------------------------
enum class Mode : int { Iter = 0, Setup = 1 };

void launch_rhs(const DevView& V, bool mixed, Mode mode, void* st);
void launch_spmv_A(const DevView& V, Mode mode, void* st);
void launch_solve(const DevView& V, Mode mode, void* st);
void launch_spmv_At(const DevView& V, Mode mode, void* st);
void launch_fwd(const DevView& V, void* st);
void launch_solve_dense(const DevView& V, void* st);
void launch_bwd_eta(const DevView& V, void* st);
void launch_post(const DevView& V, bool mixed, void* st);
// H^T sums of the long entries (before k_post, and inside launch_rhs in Iter mode)
void launch_long(const DevView& V, bool mixed, void* st);
void launch_setup_den(const DevView& V, void* st);
// Dense S = I + A Delta^{-1} A^T into the S^{-1} pool (before its in-place
// inversion), one warp per listed constraint row (absolute indices, rows of
// instances with dense == 1); mmax = the largest m among them.
constexpr size_t FORM_S_SMEM = 200 * 1024;
void launch_form_S(const DevView& V, const int32_t* rows, int32_t nrows, int32_t mmax, void* st);
// New data from device memory: per-CTA sums (non-finite count, ||D b||^2,
// ||b||^2, full-vec ||c||^2; 4 per CTA, data_grid(N, m) CTAs), then the
// scaled copies c~ = rho c, b~ = sigma D b.
constexpr int DATA_MAX_CTAS = 304;
int data_grid(int64_t N, int32_t m);
void launch_data_sums(const double* c, int64_t N, const uint8_t* diag, const double* b, int32_t m,
                      const double* dscale, const int32_t* perm, double* part, void* st);
void launch_data_apply(const double* c, int64_t N, double rho, const double* b, int32_t m, double sigma,
                       const double* dscale, const int32_t* perm, double* cdst, double* bdst, void* st);
// m-vector of one instance between the caller's constraint order and the
// internal one (perm[i]: the caller's index of internal row i): scatter
// dst[perm[i]] = src[i], else gather dst[i] = src[perm[i]]
void launch_perm_move(double* dst, const double* src, const int32_t* perm, int32_t m, bool scatter, void* st);
// A x and A^T y of the stored iterate into V.ax, V.aty for the constraint
// rows [r0, r1) and pattern entries [e0, e1) (after hsde_set_state)
void launch_state_products(const DevView& V, int r0, int r1, int64_t e0, int64_t e1, void* st);
// cone projection of every clique in one bucket (Eq. Step2 on S, fused with
// the H gather, the rank-one correction and the nu update of Eq. Step3)
// dry != 0: the autotuner's timing run (synthetic matrices, exactly
// max_sweeps sweeps, no global writes)
int  launch_cone(const DevView& V, const Bucket& bk, bool mixed, int max_sweeps, double tol,
                 int warm, int refresh, void* st, int dry = 0);
// whether a bucket size has eigensolver variant 0 (latency), 1 (throughput)
// or 2 (register-V) in a precision
bool cone_has_variant(int cmax, bool mixed, int variant);
int  cone_smem_bytes(int cmax, bool mixed);
// padded size of the bucket of a clique of size c in a precision, -1 if none
int  cone_bucket_of(int c, bool mixed);
int  cone_max_clique(bool mixed);    // largest clique the eigensolvers of a precision take
int  cone_jacobi_max(bool mixed);    // largest clique of the Jacobi buckets (above: the QR path)
void cone_bucket_sizes(std::vector<int>& out, bool mixed);   // the precision's buckets, ascending
int  cone_vstore_elems(int c, bool mixed);   // stored basis size for a clique of size c
bool cone_bucket_alone(const Bucket& bk, bool mixed);   // its CTAs each take a whole SM (launched first)
int  cone_prepare(bool mixed);
// tridiagonal QR path (cone_large.cu): workspace elements of a clique of
// size c, kernel attributes, and the launch of a CONE_BIG bucket
int64_t cone_big_ws_elems(int c);
int  cone_big_prepare(bool mixed);
int  launch_cone_big(const DevView& V, const Bucket& bk, bool mixed, void* st);
// tridiagonal QR with one warp per clique (cone_large.cu; FP32, padded
// sizes 36 ... 64): whether a bucket size has it, and its launch (variant 3)
bool cone_qrw_has(int cp);
int  launch_cone_qrw(const DevView& V, const Bucket& bk, void* st);
// reverse mode (unrolled.cu)
void launch_apply(const DevView& V, const ApplyArgs& A, bool mixed, bool setup_only, void* st);
int  rev_prepare(bool mixed);
int  launch_rev_clique(const DevView& V, const RevArgs& R, const Bucket& bk, bool mixed, void* st);
void launch_rev_scal_pre(const RevArgs& R, int slot, int B, void* st);
void launch_rev_scal_post(const RevArgs& R, int B, void* st);
void launch_rev_update(const DevView& V, const RevArgs& R, int slot, bool mixed, void* st);
void launch_rev_seed(const DevView& V, const RevArgs& R, void* st);
void launch_rev_finish(const DevView& V, const RevArgs& R, void* st);
// Gauss-Jordan inversion of the dense S matrices (setup)
void launch_gj_step(double* pool, const int64_t* offs, const int32_t* ms, const int64_t* tile_pre,
                    int nact, int64_t ntiles, int32_t k, int32_t mmax, double* rowbuf, double* colbuf,
                    const int64_t* boff, void* st);

}  // namespace hsde
