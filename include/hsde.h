/*
 * hsde.h -- C-ABI of libhsde: ADMM for the homogeneous self-dual embedding of
 * chordally sparse SDPs on one GB300 (sm_103a).
 *
 * Method: Zheng, Fantuzzi, Papachristodoulou, Goulart, Wynn, "Fast ADMM for
 * homogeneous self-dual embedding of sparse SDPs" (arXiv:1611.01828).
 *
 * Problem (Section 3, Eqs. PrimalSDP / DualSDP):
 *     min <C, X>  s.t.  <A_i, X> = b_i (i = 1..m),  X psd
 *     max <b, y>  s.t.  sum_i y_i A_i + Z = C,       Z psd
 * C and every A_i are symmetric n x n matrices given by their LOWER triangle
 * (row >= col, diagonal included where nonzero) in COO form.
 *
 * Layouts used by the queries (all 0-based, int32 indices, FP64 values):
 *   pattern   the chordal extension E' of the aggregate sparsity pattern,
 *             lower triangle in CSC order (by column, then row): N entries.
 *   x, X, Z   one value per pattern entry (the lower triangle of a symmetric
 *             matrix restricted to E').
 *   cliques   p maximal cliques C_1..C_p of E', members ascending.
 *   packed    clique block k stored as its lower triangle column-major:
 *             (a,b) for b = 0..c_k-1, a = b..c_k-1; blocks concatenated
 *             (P = sum_k c_k (c_k+1)/2 values).
 *   state     [x (N) | s (P) | y (m) | v (P) | tau | z (P) | kappa]
 *             = (x, s, y, v, tau) of u and (z, kappa) of nu (Section 3.2;
 *             the free-cone parts h, r, w of nu are identically zero from the
 *             standard start, Eq. Step3, and are not stored).  With data
 *             scaling on (hsde_options.scaling) the state is that of the
 *             scaled problem: x~ = sigma x, s~ = sigma s, y~ = rho D^{-1} y,
 *             v~ = rho v, z~ = rho z; the solution and certificate queries
 *             return unscaled values.
 * Inner products and norms are those of the full column-stack vec: entries
 * off the diagonal count twice.
 *
 * Errors: every int-returning call returns HSDE_OK (0) or a negative code;
 * hsde_last_error() gives a message for the calling thread.  No call throws
 * across the ABI.  A handle is not thread-safe: one host thread per handle.
 */
#ifndef HSDE_H
#define HSDE_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define HSDE_API __attribute__((visibility("default")))
#else
#define HSDE_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* return codes */
#define HSDE_OK        0
#define HSDE_EINVAL   (-1)   /* invalid argument or problem data            */
#define HSDE_ENOMEM   (-2)   /* host or device allocation failed            */
#define HSDE_ECUDA    (-3)   /* CUDA runtime error (no device, launch, ...)  */
#define HSDE_ESTATE   (-4)   /* query does not match the instance's verdict */
#define HSDE_ERANGE   (-5)   /* size beyond what this build supports (cliques
                                larger than 1024; cliques above 112 in
                                HSDE_MIXED or 80 in HSDE_FP64 in
                                hsde_unrolled_forward; totals beyond int32
                                indexing) */

/* per-instance iteration status (readings of the paper's stopping rule) */
#define HSDE_RUNNING            0
#define HSDE_SOLVED             1
#define HSDE_PRIMAL_INFEASIBLE  2
#define HSDE_DUAL_INFEASIBLE    3
#define HSDE_MAX_ITER           4
#define HSDE_NUMERICAL_ERROR    5

/* arithmetic of the clique arrays and cone projections */
#define HSDE_FP64   0   /* FP64 everywhere                                      */
#define HSDE_MIXED  1   /* FP32 clique arrays, gather/scatter and eigensolves;
                           FP64 for x, y, A, the cached factor, solves and all
                           reductions                                           */

typedef struct hsde_problem {
    int32_t n;                 /* matrix size, > 0                               */
    int32_t m;                 /* number of equality constraints, >= 0           */
    int64_t C_nnz;
    const int32_t* C_row;      /* [C_nnz], row >= col                             */
    const int32_t* C_col;
    const double*  C_val;
    const int64_t* A_ptr;      /* [m+1]: entries of A_i are A_ptr[i]..A_ptr[i+1]-1 */
    const int32_t* A_row;      /* [A_ptr[m]], row >= col                          */
    const int32_t* A_col;
    const double*  A_val;
    const double*  b;          /* [m]                                             */
    int64_t pattern_nnz;       /* optional extra lower-triangle pattern; may be 0 */
    const int32_t* pattern_row;
    const int32_t* pattern_col;
} hsde_problem;

typedef struct hsde_options {
    double  eps_tol;      /* stopping tolerance, default 1e-4 (Section 5)          */
    int32_t max_iter;     /* default 2000 (Section 5)                              */
    int32_t check_every;  /* test the stopping rule every k-th iteration, default 1 */
    int32_t precision;    /* HSDE_FP64 or HSDE_MIXED, default HSDE_MIXED           */
    int32_t device;       /* CUDA device ordinal, default 0                        */
    void*   cuda_stream;  /* cudaStream_t to run on; NULL: the library creates one */
    int32_t jacobi_max_sweeps;   /* 0: default (FP32 12, FP64 16)                */
    int32_t use_graph;    /* 1 (default): replay iterations through a CUDA graph   */
    double  jacobi_tol;   /* 0: default relative off-diagonal tolerance           */
    int32_t profile;      /* 1: record CUDA events around each phase of every
                             iteration (read back with hsde_get_profile)        */
    int32_t warm_start;   /* eigensolver warm start from the previous iteration's
                             eigenbasis of each clique: -1 default (on in
                             HSDE_MIXED, off in HSDE_FP64), 0 off,
                             1 on.  Results then depend on the solve history, so
                             a resumed run (hsde_set_state) matches a straight
                             run to rounding, not bitwise.                      */
    int32_t warm_refresh; /* every k-th iteration the stored bases get one
                             Newton-Schulz step V <- V (3I - V^T V)/2 against
                             the rounding drift of their orthogonality,
                             default 32                                        */
    int32_t scaling;      /* data scaling (the practical form of the cited
                             ADMM, not specified by the paper): 1 (default) runs
                             on A~ = D A (unit-norm constraint rows),
                             b~ = sigma D b, c~ = rho c with one factor
                             sigma = scale_norm / max(||D b||, ||c||) and
                             rho = dual_weight * sigma; 0 runs on the data as
                             given.  The stopping rule is always evaluated on
                             the unscaled iterate against the original data. */
    int32_t structured_factor;   /* 1 (default): when the constraints are local to
                             cliques, keep S = I + A Delta^{-1} A^T as
                             block-diagonal plus low rank, S = B + U U^T, and
                             solve with the matrix inversion lemma (blocks of at
                             most 128 constraints, rank at most 64, used only when
                             it reads less than half of a dense inverse); 0: a
                             dense inverse whenever S is not diagonal          */
    double  alpha;        /* over-relaxation: the cone step projects
                             alpha u_hat + (1 - alpha) u - nu; in (0, 2),
                             default 1.8; 1 is the literal Eqs. Step1-Step3   */
    double  scale_norm;   /* target norm of the scaled b~ and c~, default 10   */
    double  dual_weight;  /* extra factor of rho over sigma, default 1.5       */
    int32_t autotune;     /* eigensolver variant of each clique bucket (the
                             latency variant: about one 2x2 block per thread;
                             the throughput variant: fewer threads a clique,
                             more cliques per SM; the register-V variant,
                             FP32 sizes 24-64: V held in registers through
                             the sweeps).  All give bitwise the same results.
                             1 (default): time them once per (precision,
                             bucket size, clique count, SM count) at setup
                             and keep the fastest (cached for the process);
                             0: throughput unless the bucket's CTAs each have
                             an SM to themselves; 2: always latency;
                             3: always throughput; 4: register-V where the
                             bucket has it.  A bucket of few large cliques
                             always runs the latency variant.               */
    int32_t eigensolver;  /* HSDE_MIXED cliques of 33 to 64: 0 (default) the
                             warm-started Jacobi; 1 the tridiagonal QR with
                             one warp per clique, all in shared memory (a
                             constant cost per iteration: faster than the
                             Jacobi while the warm start still needs ~3
                             sweeps a clique, slower once it settles to ~1).
                             The two agree to FP32 rounding, not bitwise.    */
} hsde_options;

typedef struct hsde_sizes {
    int32_t n, m, p;      /* matrix size, constraints, cliques                    */
    int32_t c_max;        /* largest clique                                       */
    int64_t N;            /* pattern entries (lower, diagonal included)          */
    int64_t P;            /* packed clique storage sum_k c_k(c_k+1)/2             */
    int64_t n_d;          /* sum_k c_k^2 (Section 3.2)                            */
    int64_t state_len;    /* N + 3P + m + 2                                       */
    int32_t S_dense;      /* how S = I + A Delta^{-1} A^T is kept: 0 diagonal, 1 dense
                             inverse, 2 block-diagonal plus low rank           */
    int32_t _pad;
} hsde_sizes;

typedef struct hsde_info {
    int32_t status;       /* HSDE_RUNNING ...                                     */
    int32_t iterations;   /* ADMM iterations performed on this instance           */
    double  pres, dres, gap;      /* at the last check (readings P5)             */
    double  pobj, dobj;           /* c^T x / tau, b^T y / tau                     */
    double  tau, kappa;
    double  pinf_ratio, dinf_ratio;  /* certificate ratios (reading P6)          */
    double  setup_ms;     /* host + device setup ("Pre- time" of Tables 2-4)    */
    double  iterate_ms;   /* wall time spent inside hsde_iterate               */
    int32_t jacobi_unconverged;  /* cliques whose eigensolve stopped at
                                    jacobi_max_sweeps above jacobi_tol in the
                                    last iteration (0 in a healthy run)      */
    int32_t jacobi_unconverged_iterations;  /* iterations with at least one  */
} hsde_info;

#define HSDE_MAX_PHASES 24
typedef struct hsde_profile {
    int32_t kernels_per_iteration;   /* kernel launches in one iteration          */
    int32_t nphases;
    double  phase_ms[HSDE_MAX_PHASES];   /* device time of each phase in the last
                                            iteration launched (profile = 1)    */
    char    phase_name[HSDE_MAX_PHASES][24];
    int64_t phase_units[HSDE_MAX_PHASES];  /* work units of the phase: pattern
                                              entries (affine, check) or
                                              sum_k c_k^3 (cone buckets)        */
    double  sweeps_mean;  /* Jacobi sweeps per clique in the last iteration (QR
                             path: QR steps per eigenvalue, rounded up)        */
    int32_t sweeps_max;
    int32_t _pad;
    int32_t phase_sweeps_max[HSDE_MAX_PHASES];  /* cone phases: most sweeps any
                                                   clique of the bucket took
                                                   (it sets the phase's time); 0
                                                   for the other phases       */
    int32_t phase_variant[HSDE_MAX_PHASES];  /* cone phases: the eigensolver
                                                variant the bucket runs (0
                                                latency, 1 throughput, 2
                                                register-V; see
                                                options.autotune; 3 the
                                                warp tridiagonal QR, see
                                                options.eigensolver)        */
} hsde_profile;

typedef struct hsde_handle hsde_handle;
typedef struct hsde_symbolic hsde_symbolic;

/* Fill *o with the defaults listed above. */
HSDE_API void hsde_default_options(hsde_options* o);

/* Message of the last failing call on this thread ("" if none). */
HSDE_API const char* hsde_last_error(void);

/* ------------------------------------------------------------------------
 * Host-only symbolic analysis (Section 2.1-2.2; no GPU is touched).
 * Aggregate pattern supp(C) U supp(A_i) U diag U extra pattern, chordal
 * extension by exact minimum degree (ties to the smallest vertex index),
 * maximal cliques ordered by the elimination step of their defining vertex,
 * members ascending; H_k as the gather map, D = H^T H (Section 4.3).
 * Inputs are copied; *out must be released with hsde_symbolic_free.
 * Errors: HSDE_EINVAL for out-of-range or upper-triangle indices, duplicate
 * entries inside C or inside one A_i, non-finite values, n <= 0, m < 0.
 * ---------------------------------------------------------------------- */
HSDE_API int  hsde_analyze(const hsde_problem* P, hsde_symbolic** out);
HSDE_API int  hsde_symbolic_sizes(const hsde_symbolic* s, hsde_sizes* out);
/* Any output pointer may be NULL.  Sizes: order[n] (vertex eliminated at
 * each step), clique_ptr[p+1], clique_idx[sum c_k], pat_colptr[n+1],
 * pat_row[N], gather[P] (packed clique entry -> pattern position), D[N]. */
HSDE_API int  hsde_symbolic_get(const hsde_symbolic* s, int32_t* order, int32_t* clique_ptr,
                       int32_t* clique_idx, int32_t* pat_colptr, int32_t* pat_row,
                       int32_t* gather, int32_t* D);
HSDE_API void hsde_symbolic_free(hsde_symbolic* s);

/* ------------------------------------------------------------------------
 * Setup (Section 4.2-4.3 "cached before starting the iterations"): symbolic
 * analysis, upload, S = I + A Delta^{-1} A^T with Delta = I + D/2 and its
 * FP64 inverse (diagonal when no two constraints share a pattern entry),
 * the cached M^{-1} zeta and 1 + zeta^T M^{-1} zeta, and the starting point
 * u0 = (0,0,0,0,1), nu0 = (0,0,0,0,1).  All inputs are copied; the caller may
 * free them on return.  *out is NULL on error.  hsde_setup_batch sets up B
 * independent instances behind one handle; they iterate in the same launches
 * and each stops on its own verdict.
 * Errors: HSDE_EINVAL (see hsde_analyze; also B <= 0, bad options),
 * HSDE_ENOMEM, HSDE_ECUDA (no device / CUDA failure), HSDE_ERANGE (a clique
 * larger than this build's eigensolvers or totals beyond int32 indexing).
 * ---------------------------------------------------------------------- */
HSDE_API int  hsde_setup(const hsde_problem* P, const hsde_options* O, hsde_handle** out);
HSDE_API int  hsde_setup_batch(const hsde_problem* P, int32_t B, const hsde_options* O,
                      hsde_handle** out);

/* Run up to k more ADMM iterations (Eqs. Step1-Step3) on every instance
 * that is still HSDE_RUNNING; an instance freezes on its verdict.  Work is
 * enqueued on the handle's stream.  If status_out is non-NULL the call
 * waits for the work and writes one status per instance (B entries). */
HSDE_API int  hsde_iterate(hsde_handle* h, int32_t k, int32_t* status_out);
/* Wait for all work enqueued on the handle's stream. */
HSDE_API int  hsde_sync(hsde_handle* h);

HSDE_API int  hsde_num_instances(const hsde_handle* h);
HSDE_API int  hsde_get_sizes(const hsde_handle* h, int32_t i, hsde_sizes* out);
/* Same layout as hsde_symbolic_get, for instance i of a handle. */
HSDE_API int  hsde_get_structure(const hsde_handle* h, int32_t i, int32_t* order, int32_t* clique_ptr,
                        int32_t* clique_idx, int32_t* pat_colptr, int32_t* pat_row,
                        int32_t* gather, int32_t* D);
HSDE_API int  hsde_get_info(hsde_handle* h, int32_t i, hsde_info* out);

/* Checkpoint / resume: copy the state (layout above, state_len doubles) of
 * instance i to or from host memory.  In HSDE_MIXED mode s, v, z are rounded
 * to FP32 on set.  set_state also resets the instance to HSDE_RUNNING with
 * the given iteration counter. */
HSDE_API int  hsde_get_state(hsde_handle* h, int32_t i, double* state);
HSDE_API int  hsde_set_state(hsde_handle* h, int32_t i, const double* state, int32_t iterations);

/* Solution of a SOLVED instance (reading P5): X = x/tau and Z = H^T z / tau
 * (the Agler sum of the clique blocks, Theorem 2) as N pattern values, y/tau,
 * and the objectives.  Any output pointer may be NULL.  HSDE_ESTATE if the
 * instance is not SOLVED. */
HSDE_API int  hsde_get_solution(hsde_handle* h, int32_t i, double* X, double* y, double* Z,
                       double* pobj, double* dobj);
/* Certificate of an infeasible instance (reading P6).  PRIMAL_INFEASIBLE:
 * y/(b^T y) (m values) and Z = H^T z/(b^T y) (N values), with
 * A^T y + Z ~ 0, b^T y = 1 and every clique block of z psd.
 * DUAL_INFEASIBLE: X = x/(-c^T x) (N values) with A(X) ~ 0, <C, X> = -1 and
 * every clique block of X psd; y and Z are left untouched.  HSDE_ESTATE if
 * the verdict does not match the certificate asked for (kind =
 * HSDE_PRIMAL_INFEASIBLE or HSDE_DUAL_INFEASIBLE). */
HSDE_API int  hsde_get_certificate(hsde_handle* h, int32_t i, int32_t kind, double* y, double* Z,
                          double* X);

/* Launch count of one iteration, the Jacobi sweeps of the last iteration
 * (mean per clique and most) and, if the handle was set up with
 * profile = 1, the device time of each phase of the last iteration (waits
 * for the handle's stream).  Phases: "affine" (A f, S^{-1}, A^T y_w, eta),
 * one "cone_cK" per clique bucket (cliques of size <= K, each on its own
 * graph branch), "cone_qr" for the cliques above the Jacobi sizes (112 in
 * HSDE_MIXED, 80 in HSDE_FP64; up to 1024): Householder tridiagonalisation,
 * implicit QR with the Wilkinson shift and a split-precision TF32
 * tensor-core rebuild in HSDE_MIXED, one CTA per clique; its sweeps count
 * QR steps per eigenvalue, rounded up), "post" (x update, stopping rule,
 * verdict and the next right-hand side) and "iteration" (all of it). */
HSDE_API int  hsde_get_profile(hsde_handle* h, hsde_profile* out);

/* In-place inverse of a dense m x m symmetric positive definite matrix held
 * in DEVICE memory (row-major, m*m doubles): the cached factor of Sections
 * 4.2-4.3, kept as the explicit inverse of S = I + A Delta^{-1} A^T.
 * Gauss-Jordan elimination without pivoting (every pivot of an SPD matrix is
 * positive).  2m doubles of device scratch are allocated with
 * cudaMallocAsync on the stream and released with cudaFreeAsync once the
 * work is enqueued.  Asynchronous on cuda_stream (NULL: legacy default
 * stream); the caller keeps ownership of S.  A matrix that is not SPD gives
 * a meaningless result (no error is detected).
 * Errors: HSDE_EINVAL (null S, m <= 0), HSDE_ENOMEM, HSDE_ECUDA. */
HSDE_API int  hsde_spd_inverse(double* S, int32_t m, void* cuda_stream);

/* Same inverse as hsde_spd_inverse, for callers that must not allocate
 * device memory during the call (for example code running under CUDA graph
 * capture in a framework that forbids allocation there, real-time hosts with
 * a fixed memory budget, or processes whose device memory is managed by a
 * pooling allocator).  The paper has no counterpart: this is a deployment
 * variant.  It allocates nothing: the 2m-double pivot scratch lives in a
 * fixed array in device memory (limit m <= 8192, i.e. 128 KiB that every GPU
 * loading the library keeps until the process exits).  The first call on a
 * device looks up that array's device address (cudaGetSymbolAddress) and
 * caches it; make that first call before any stream capture.  All calls on a
 * device share the one scratch array, which keeps the last call's contents
 * (nothing in it needs to start at zero): calls whose work overlaps on the
 * GPU (different streams, or concurrent host threads) race and give wrong
 * results; serialise them on one stream.  Asynchronous on cuda_stream.
 * Errors: HSDE_EINVAL (null S, m <= 0), HSDE_ERANGE (m > 8192),
 * HSDE_ECUDA (no current device, symbol lookup or launch failure). */
HSDE_API int  hsde_spd_inverse_noalloc(double* S, int32_t m, void* cuda_stream);

/* Replace the data c = C (N pattern values, lower CSC order) and b (m values)
 * of instance i, keeping the pattern, the constraint matrices and the cached
 * factor S (which does not depend on c or b); the scaling factors sigma and
 * rho, M^{-1} zeta and 1 + zeta^T M^{-1} zeta (Eq. MatrixInverseResult) are
 * recomputed.  The iterate is left as it is.  c and b are both host memory
 * or both device memory of the handle's GPU (unified addressing tells them
 * apart).  Device data never passes through the host: kernels check it and
 * form the sums of the scaling, whose partials the host adds in a fixed
 * order (the norms, sigma and rho can differ from the host path's in the
 * last bit; unscaled handles upload c and b unchanged either way).  The
 * caller's writes to device c and b must be complete (synchronise the
 * producing stream) before the call; the call returns after its own work
 * is done.  Errors: HSDE_EINVAL (null, non-finite, a mix of host and device
 * pointers, or a pointer into another GPU). */
HSDE_API int  hsde_set_data(hsde_handle* h, int32_t i, const double* c, const double* b);

/* Unrolled differentiation (single-instance handles).  hsde_unrolled_forward
 * runs exactly K iterations of Eqs. Step1-Step3 from the standard start
 * u0 = (0,0,0,0,1), nu0 = (0,0,0,0,1), with the stopping rule and the
 * eigensolver warm start disabled, keeping the iterate every ckpt iterations,
 * and returns x_K (N), y_K (m), tau_K and kappa_K.
 * hsde_unrolled_backward then returns the gradient of
 *     L = sum_e xbar_e x_K,e + ybar^T y_K + taubar tau_K + kappabar kappa_K
 * with respect to the stored lower values of C (gC, N values; an entry off
 * the diagonal stands for both (i,j) and (j,i)) and b (gb, m values), through
 * every iteration: the psd projections by the Daleckii-Krein formula (1/2 at
 * coinciding zero eigenvalues), the tau step, and the affine step by the
 * adjoint solve (I+Q)^{-T} = (I-Q)^{-1} with the same cached factor.  Each
 * checkpoint segment is recomputed once to record its eigendecompositions.
 * Not in the paper.  Afterwards the handle's iterate is undefined (use
 * hsde_set_state).  The handle must run the literal iteration on the data
 * as given (options alpha = 1 and scaling = 0): the scaling factors depend
 * on c and b.  Errors: HSDE_EINVAL (B != 1, K or ckpt < 1, alpha != 1 or
 * scaling on),
 * HSDE_ESTATE (backward without forward), HSDE_ENOMEM, HSDE_ECUDA.
 * Every array argument (x, y, xbar, ybar, gC, gb) may be host memory or
 * device memory of the handle's GPU; device seeds must be complete before
 * the call, and both calls return with their outputs written. */
HSDE_API int  hsde_unrolled_forward(hsde_handle* h, int32_t K, int32_t ckpt, double* x, double* y,
                                    double* tau, double* kappa);
HSDE_API int  hsde_unrolled_backward(hsde_handle* h, const double* xbar, const double* ybar,
                                     double taubar, double kappabar, double* gC, double* gb);

/* Free all device and host memory of the handle.  NULL-safe. */
HSDE_API void hsde_destroy(hsde_handle* h);

#ifdef __cplusplus
}
#endif
#endif /* HSDE_H */
