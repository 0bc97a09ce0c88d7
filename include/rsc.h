/*
 * rsc.h -- C ABI of a GB300 (sm_103a) implementation of the rank-structured
 * supernodal Cholesky preconditioner of Chadwick & Bindel, "An efficient solver
 * for sparse linear systems based on rank-structured Cholesky factorization"
 * (arXiv 1507.05593).
 *
 * The problem is A x = b with A symmetric positive definite (Section 1, Eq. "main").
 * rsc_analyze orders A by nested dissection and computes the supernodal structure
 * (Sections 2.1, 2.2, 3.1, 4.1); rsc_factor builds the approximate factor
 * L ~ chol(P A P^T) with compressed off-diagonal and diagonal blocks (Algorithms
 * 1-6, Sections 3-5); rsc_solve runs PCG preconditioned by the two triangular
 * solves with L (Section 1; Section 6.1 uses PCG to a relative residual).
 *
 * Conventions for every call:
 *  - indices are 0-based; the matrix is the FULL symmetric CSR (both triangles),
 *    column indices sorted and unique within each row, the diagonal present;
 *  - pointers named d_* are device pointers of the current CUDA device, all
 *    others are host pointers; the caller owns every buffer it passes and the
 *    library copies what it keeps;
 *  - no C++ exception crosses this boundary; a failing call returns a status
 *    and rsc_last_error(handle) describes it (NULL handle: last global error);
 *  - a handle is not thread safe and issues its GPU work on one stream.
 */
#ifndef RSC_H
#define RSC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rsc_handle rsc_handle;

typedef enum {
    RSC_OK = 0,
    RSC_ERR_INVALID_ARG = 1,    /* malformed input (sizes, pattern, NaN, NULL) */
    RSC_ERR_NOT_SPD = 2,        /* a pivot <= 0 after every restart (Section 5.3) */
    RSC_ERR_NO_CONVERGENCE = 3, /* PCG hit max_iter; x holds the last iterate */
    RSC_ERR_OOM = 4,            /* device or host allocation failed */
    RSC_ERR_CUDA = 5,           /* a CUDA runtime error (no device, launch failure) */
    RSC_ERR_TIMEOUT = 6,        /* a bounded device wait gave up */
    RSC_ERR_STATE = 7           /* call order: factor before analyze, solve before factor */
} rsc_status;

typedef enum {
    RSC_PREC_FP64 = 0,   /* every step in FP64 */
    RSC_PREC_FP32 = 1,   /* factor, Schur updates, diagonal Cholesky tiles, sampling and the
                            preconditioner apply in FP32 (FP64 kept for PCG) */
    RSC_PREC_TF32 = 2,   /* as FP32, Schur-update GEMMs on tensor cores in TF32 */
    RSC_PREC_BF16 = 3    /* as FP32, Schur-update GEMMs on tensor cores in BF16 */
} rsc_precision;

/* Parameters of the method (Sections 3.1, 4.1, 5.2, 5.3). */
typedef struct {
    int32_t tau_O;         /* separators with >= tau_O unknowns are compressed (Section 3.1); 256 */
    int32_t tau_D;         /* largest dense diagonal block (Section 4.1); 256 */
    int32_t leaf_size;     /* nested-dissection leaf: at most this many nodes; 64 */
    int32_t sample_block;  /* columns per randomized sampling pass; 16 (only 16 supported) */
    int32_t power_iters;   /* power iterations in Alg. 3; 0 */
    int32_t dof_per_node;  /* unknowns per node kept adjacent (3 for elasticity); 1 */
    int32_t max_restarts;  /* indefinite restarts before diagonal compression is switched off; 8 */
    int32_t precision;     /* rsc_precision; RSC_PREC_FP64 */
    int32_t diag_compress; /* 1: compress diagonal blocks hierarchically (Section 4); 1 */
    int32_t ordering;      /* 0: nested dissection by lattice bisection (coords = integer lattice
                              positions); 1: graph nested dissection for general sparsity, guided by
                              coords (any real positions).  coords == NULL selects 1 with spectral
                              positions (Section 4.3); 0 */
    uint64_t seed;         /* key of the Philox4x32-10 stream of the random test matrices; 0 */
    int32_t amalgamate;    /* 1: relaxed amalgamation of small supernodes (Section 3.1's grouping "as in
                              CHOLMOD"): a supernode's last child merges into it while the merged
                              block has at most 4 columns, or at most 16 / 48 columns with at most
                              80% / 10% entries new to both blocks, or at most 5% new entries at any
                              size; compressed separators (>= tau_O columns) are never merged; 0 */
    int32_t interior_blocks; /* 1: interior blocks (Section 5.1): for every maximal subtree B of the
                              supernodal tree without a compressed supernode, L(R_B, C_B) is not kept
                              after the factorization; the solves use A(R_B, C_B) L_B^{-T} instead
                              (Eq. interiorBlockClosedForm).  The allocation-free apply does not
                              support it (RSC_ERR_INVALID_ARG); 0 */
} rsc_options;

typedef struct {
    double factor_bytes;      /* bytes of the stored factor (dense blocks + V, U) */
    double factor_flops;      /* algorithmic flops of the last rsc_factor */
    double factor_seconds;    /* device time of the last rsc_factor (CUDA events) */
    double solve_seconds;     /* device time of the last solve */
    int32_t restarts;         /* restarts taken by the last rsc_factor (Section 5.3) */
    int32_t n_supernodes;
    int32_t n_compressed;     /* supernodes with compressed blocks */
    int32_t n_levels;         /* levels of the supernodal elimination tree */
    int32_t max_rank;         /* largest off-diagonal rank */
    int32_t last_iters;       /* PCG iterations of the last solve */
    double last_relres;       /* true relative residual of the last solve */
    int64_t gpu_launches;     /* kernels launched by the last factor + solve */
} rsc_stats_t;

/* Fill *opts with the defaults listed above.  Returns RSC_INVALID_ARG on NULL. */
rsc_status rsc_options_default(rsc_options* opts);

/*
 * Symbolic analysis on the host (Sections 2.1, 2.2, 3.1, 4.1): nested-dissection
 * ordering of the nodes by recursive coordinate bisection, one supernode per
 * nested-dissection leaf or separator, supernodal row structures R_j, the
 * supernodal elimination tree and its levels, and the within-separator
 * geometric ordering and block tree of every separator with more than tau_D
 * unknowns that is large enough to be compressed.
 *   n        unknowns; row_ptr[n+1] (int64), col_idx[nnz] (int32), val[nnz] (FP64);
 *   coords   n x 3 row-major positions of each unknown (unknowns of one node repeat
 *            the node's position): integer lattice positions for opts->ordering = 0,
 *            any real positions for 1; NULL: positions from the three lowest
 *            non-constant eigenvectors of the node graph's Laplacian (Section 4.3,
 *            Lanczos on the host) and the graph ordering;
 *   opts     NULL for defaults.
 * The values are copied and used by rsc_factor.  No GPU work is done here.
 * Errors: RSC_ERR_INVALID_ARG (pattern not symmetric, unsorted, missing
 * diagonal, non-finite value, n not a multiple of dof_per_node, ordering not 0 or 1).
 */
rsc_status rsc_analyze(int64_t n, const int64_t* row_ptr, const int32_t* col_idx, const double* val,
                       const double* coords, const rsc_options* opts, rsc_handle** out);

/* perm[n]: perm[new] = old unknown; *n_snodes = M; snode_ptr[M+1] column boundaries
 * (each output may be NULL). */
rsc_status rsc_get_ordering(const rsc_handle* h, int32_t* perm, int32_t* n_snodes, int64_t* snode_ptr);

/* Node positions the ordering used (Section 4.3): pos[3 * node + axis] for the n / dof_per_node
 * nodes, the given coordinates or the spectral ones (rounded lattice positions for
 * ordering 0).  Errors: RSC_ERR_INVALID_ARG (NULL). */
rsc_status rsc_get_coordinates(const rsc_handle* h, double* pos);

/* Supernodal structure: rows_ptr[M+1] and rows[rows_ptr[M]] hold R_j (sorted
 * permuted row indices after C_j); parent[M] (-1 for roots); level[M]; kind[M]
 * (0 leaf, 1 separator).  Pass rows == NULL to query rows_ptr only. */
rsc_status rsc_get_structure(const rsc_handle* h, int64_t* rows_ptr, int32_t* rows, int32_t* parent,
                             int32_t* level, int32_t* kind);

/*
 * Numeric factorization on the GPU (Algorithms 1-6).  tol <= 0: compression off,
 * the exact supernodal Cholesky factor (Alg. 1).  tol > 0: supernodes that are
 * separators with >= tau_O unknowns get off-diagonal blocks L^O_j ~ V_j U_j^T
 * (Alg. 2, 3; adaptive: stop when the sampled residual falls to tol relative)
 * and, above tau_D unknowns, hierarchically compressed diagonal blocks (Alg. 4-6)
 * at tolerance tol_D = tol / 1.25^restart.  On an indefinite diagonal block the
 * factorization restarts (Section 5.3); after max_restarts restarts diagonal
 * compression is switched off.  Errors: RSC_ERR_STATE, RSC_ERR_NOT_SPD,
 * RSC_ERR_OOM, RSC_ERR_CUDA, RSC_ERR_TIMEOUT.  Synchronous.
 */
rsc_status rsc_factor(rsc_handle* h, double tol);

/*
 * Numeric factorization in the fixed-rank form of Section 5.2: the same supernodes
 * as rsc_factor with tol > 0 are compressed, but each block B (m x n) gets the rank
 * of Eq. rankFunction, ceil(alpha sqrt(k) log2 k) + p with k = min(m, n), capped at
 * k: alpha_O for off-diagonal blocks L^O_j (Alg. 3), alpha_D for the internal
 * blocks of hierarchical diagonal blocks (Section 4.2).  The samples are drawn in
 * 16-column passes from the same Philox stream as rsc_factor, with
 * opts.power_iters power iterations (Alg. 3); the adaptive stopping test is off, so
 * a block stops early only when its sampled columns are numerically dependent.
 * On an indefinite diagonal block the factorization restarts with
 * alpha_D <- 1.25 alpha_D (Section 5.3, which starts from alpha_D = 0.5); after
 * max_restarts restarts diagonal compression is switched off.
 * Errors: RSC_ERR_INVALID_ARG (alpha_O, alpha_D negative or not finite, p < 0), and
 * those of rsc_factor.  Synchronous.
 */
rsc_status rsc_factor_fixed_rank(rsc_handle* h, double alpha_O, double alpha_D, int32_t p);

/* New values for the same pattern (val[nnz] as in rsc_analyze); the next
 * rsc_factor uses them. */
rsc_status rsc_refactor_values(rsc_handle* h, const double* val);

/* As rsc_refactor_values with the values on the device: d_val[nnz] (FP64, the order of the CSR
 * given to rsc_analyze), read on cuda_stream (a cudaStream_t, NULL = the handle's stream); the
 * call returns after the library holds its own copy.  Until the next rsc_refactor_values the
 * factorization and the SpMV of the solves use these values (no host copy is made).  Errors:
 * RSC_ERR_INVALID_ARG (NULL, a non-finite value). */
rsc_status rsc_refactor_values_device(rsc_handle* h, const double* d_val, void* cuda_stream);

/*
 * PCG from x0 = 0 on the original (unpermuted) system, preconditioned by
 * M^{-1} = P (L L^T)^{-1} P^T, until ||r||/||b|| <= rtol (recursive residual,
 * confirmed by the true residual).  b[n], x[n] host FP64.  *iters = CG steps;
 * *final_relres = true relative residual.  RSC_ERR_NO_CONVERGENCE leaves the
 * last iterate in x.  Synchronous.
 */
rsc_status rsc_solve(rsc_handle* h, const double* b, double* x, double rtol, int32_t max_iter,
                     int32_t* iters, double* final_relres);

/* As rsc_solve with device vectors d_b[n], d_x[n] (FP64) on cuda_stream
 * (a cudaStream_t, NULL = the handle's stream). */
rsc_status rsc_solve_device(rsc_handle* h, const double* d_b, double* d_x, double rtol, int32_t max_iter,
                            int32_t* iters, double* final_relres, void* cuda_stream);

/* One application of the preconditioner: d_z = P (L L^T)^{-1} P^T d_r (device FP64, n). */
rsc_status rsc_apply_preconditioner_device(rsc_handle* h, const double* d_r, double* d_z, void* cuda_stream);

/*
 * Independent systems (batching form; the paper solves one system at a time): a
 * matrix that is block diagonal up to ordering -- several systems stacked, each a
 * connected component of A's graph -- is analysed one component at a time, so the
 * supernodal elimination tree is a forest and every level of the factorization runs
 * the supernodes of all systems together.  *n_systems = number of components;
 * sys_ptr[n_systems+1] (may be NULL) their row ranges.  RSC_ERR_INVALID_ARG if the
 * components are not contiguous row ranges of the original numbering.
 */
rsc_status rsc_get_systems(const rsc_handle* h, int32_t* n_systems, int64_t* sys_ptr);

/*
 * Batched PCG: every (system, right-hand side) pair runs its own PCG recurrence
 * (own alpha, beta and stopping test, Section 6.1's relative residual) on the
 * stacked system, preconditioned by the factor of the stacked matrix (which does
 * not couple systems).  d_B, d_X: n x nrhs column-major device FP64.  iters[q],
 * final_relres[q] for pair q = column * n_systems + system.  RSC_ERR_NO_CONVERGENCE
 * if some pair did not reach rtol within max_iter (X holds the last iterates).
 */
rsc_status rsc_solve_batch_device(rsc_handle* h, int32_t nrhs, const double* d_B, double* d_X, double rtol,
                                  int32_t max_iter, int32_t* iters, double* final_relres, void* cuda_stream);

/*
 * Sparse outer product over A's pattern (the paper has no counterpart; it serves
 * the adjoint gradient of x = A^{-1} b): d_out[e] = alpha * d_u[i] * d_v[j] for every
 * stored entry e = (i, j) of the CSR given to rsc_analyze, in its order.  With
 * u = lambda (the adjoint solution of A lambda = dL/dx), v = x and alpha = -1 this is
 * dL/dA restricted to the pattern.  d_u[n], d_v[n], d_out[nnz] device FP64.
 */
rsc_status rsc_pattern_outer_device(rsc_handle* h, const double* d_u, const double* d_v, double alpha,
                                    double* d_out, void* cuda_stream);

/*
 * Allocation-free variant of rsc_apply_preconditioner_device (the paper has no
 * counterpart; this is an interface convenience).  For callers that cannot call
 * cudaMalloc while they apply the preconditioner: frameworks whose device memory
 * is owned by their own allocator or held to a fixed budget, and latency-bound
 * loops that cannot afford the implicit device synchronisation of cudaMalloc and
 * cudaFree.  It computes the same d_z = P (L L^T)^{-1} P^T d_r and allocates no
 * device memory: its work vector, low-rank temporaries and task records live in
 * one file-scope static device array of 64 MiB, which every GPU that loads the
 * library holds until the process exits.
 *  - The first call on a device looks up the array's address (cudaGetSymbolAddress,
 *    with that device current); the first call after each rsc_factor (or with
 *    another handle) copies its task records into the array on cuda_stream.  Make
 *    such a first call before any stream capture.
 *  - Every call synchronises cuda_stream before it returns: d_z holds the result and
 *    a failure of the call's kernels is reported by the call itself.
 *  - Every call, from every handle, shares the one array and it keeps the last
 *    call's contents; calls whose GPU work overlaps (other streams, other host
 *    threads) race with each other.
 *  - Returns RSC_ERR_INVALID_ARG when the problem needs more than the 64 MiB
 *    (about n * sizeof(factor element) plus the task records), RSC_ERR_STATE
 *    before rsc_factor or when the current CUDA device is not the one the handle
 *    was factored on.
 */
rsc_status rsc_apply_preconditioner_device_noalloc(rsc_handle* h, const double* d_r, double* d_z, void* cuda_stream);

/* Per-supernode results of the last factor.  info[8] = {c_j, |R_j|, compressed,
 * rank of L^O_j (0 if uncompressed), hierarchical diagonal, blocks in L^D_j,
 * level, kind}. */
rsc_status rsc_get_supernode_info(const rsc_handle* h, int32_t j, int32_t* info);

/* Dense blocks of supernode j (FP64, column-major): LD[c*c] the diagonal block
 * (hierarchical blocks expanded, V_s U_s^T in the off-diagonal blocks), LO[r*c]
 * L^O_j or V_j U_j^T (either may be NULL), r = |R_j|.  With interior_blocks = 1 the
 * rows of R_j after an interior block's columns are not stored and come back as NaN. */
rsc_status rsc_get_supernode_blocks(const rsc_handle* h, int32_t j, double* LD, double* LO);

rsc_status rsc_get_stats(const rsc_handle* h, rsc_stats_t* out);

/* Kernel profiler (measurement aid, not part of the method): enable != 0 turns on
 * CUDA-event timing around the launches of the listed kernel classes
 * (comma-separated names, e.g. "push,tn,nn"; NULL or "" = all) and clears the
 * accumulated counts.  Classes: push (extend-add), potrf, trsm, panel_gemm, tn,
 * nn, trsv, spmv, dot, axpy. */
rsc_status rsc_profile(rsc_handle* h, int32_t enable, const char* kernels);

/* JSON object {class: {launches, ms, flops, bytes}} of the profiled launches since
 * the last rsc_profile call (algorithmic flops and bytes).  json[len] host buffer. */
rsc_status rsc_get_kernel_profile(rsc_handle* h, char* json, int64_t len);

/* Failure detection (the paper has no counterpart).  The cooperative kernel of the range finder
 * (Alg. 3, one launch per sampling pass) separates its phases by grid barriers whose waits are
 * bounded: after `polls` polls (about 64 ns apart) a waiting block gives up, the kernel records
 * the expiry and returns, the following passes of that factorization do no work, and rsc_factor
 * returns RSC_ERR_TIMEOUT; the handle stays usable (rsc_refactor_values, rsc_factor).
 * polls = 0 restores the default (2^22 polls, about a quarter of a second).  Errors:
 * RSC_ERR_INVALID_ARG (polls < 0). */
rsc_status rsc_set_wait_limit(rsc_handle* h, int64_t polls);

/* Kernel-variant tuning of the BF16 / TF32 forms (the paper has no counterpart): the thin
 * products of the implicit sampling (Alg. 2, Alg. 5 and their transposes) have a SIMT kernel
 * and a tcgen05 tensor-core kernel with different tiles.  During a handle's first rsc_factor
 * in those forms the launches alternate between the two, timed with CUDA events, per (product
 * class, sample-column width, log2 of the launch's flops); later factorizations use the faster
 * one per key.  json[len] receives {key: {choice (0 SIMT, 1 tensor cores), simt_ns_per_mflop,
 * tensor_ns_per_mflop, launches: [simt, tensor]}}; {} before the first factorization.
 * Errors: RSC_ERR_INVALID_ARG (NULL, or len too small). */
rsc_status rsc_get_autotune(const rsc_handle* h, char* json, int64_t len);

/* Message of the last error on h (or of the last failed rsc_analyze if h is NULL). */
const char* rsc_last_error(const rsc_handle* h);

void rsc_destroy(rsc_handle* h);

#ifdef __cplusplus
}
#endif

#endif /* RSC_H */
