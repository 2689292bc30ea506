/*
 * lair.h -- C ABI of the GB300 lAIR library (liblair.so).
 *
 * lAIR: algebraic multigrid with local approximate ideal restriction and
 * F-relaxation (Manteuffel, Ruge, Southworth, "Nonsymmetric algebraic multigrid
 * based on local approximate ideal restriction (lAIR)"). The library builds a
 * multigrid hierarchy on one GPU and solves A x = b with V-cycles as the
 * preconditioner of an FP64 outer iteration.
 *
 * Conventions that hold for every call:
 *  - Matrices are CSR: int64 row pointers, int32 column indices sorted
 *    ascending within each row, no duplicates, diagonal stored, float64 values.
 *  - The caller owns every buffer it passes. The library copies what it keeps
 *    (the matrix) and never retains a caller pointer after a call returns.
 *  - Vectors may live in host memory (pageable or pinned) or device memory; the
 *    library checks each pointer and copies host data itself.
 *  - Device work is ordered on the stream given in lair_options.stream; with
 *    NULL the handle creates its own blocking stream (ordered with the legacy
 *    default stream). Calls return after their device work has finished.
 *  - Failures come back as a lair_status, never as an abort or exception;
 *    lair_last_error() gives a one-line description.
 *  - No call is thread-safe with respect to the same handle.
 */
#ifndef LAIR_H
#define LAIR_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    LAIR_OK = 0,
    LAIR_ERR_INVALID_ARG = 1,       /* a NULL pointer, a negative size, an unknown option value */
    LAIR_ERR_NOT_SQUARE = 2,        /* row pointers inconsistent with n / nnz */
    LAIR_ERR_UNSORTED_CSR = 3,      /* columns not strictly ascending or out of range */
    LAIR_ERR_DUPLICATE_ENTRY = 4,
    LAIR_ERR_ZERO_DIAGONAL = 5,     /* missing or zero diagonal (or singular DG block) */
    LAIR_ERR_COARSENING_STALLED = 6,/* no coarse points and the level is too large for a direct solve */
    LAIR_ERR_NOT_CONVERGED = 7,     /* max_iter reached above tol (x holds the last iterate) */
    LAIR_ERR_NAN = 8,               /* a residual norm became NaN or Inf */
    LAIR_ERR_OOM = 9,               /* device allocation failed */
    LAIR_ERR_ARENA_OVERFLOW = 10,   /* a size bound of a fixed device buffer was exceeded */
    LAIR_ERR_DEVICE_TIMEOUT = 11,   /* a bounded device-side wait gave up */
    LAIR_ERR_CUDA = 12,             /* any other CUDA runtime error */
    LAIR_ERR_UNSUPPORTED = 13       /* an input beyond a documented limit */
} lair_status;

/* C/F splitting: classical Ruge-Stueben first pass, no second pass (Sec. 4), on the
 * whole level (RS, at most 32768 points); PMIS (hashed-weight parallel independent
 * set); a user array on level 0; AUTO = the first pass run independently on
 * consecutive index blocks of rs_block points (exactly RS on levels that fit in one
 * block), in parallel over blocks. */
typedef enum { LAIR_CF_RS = 0, LAIR_CF_PMIS = 1, LAIR_CF_USER = 2, LAIR_CF_AUTO = 3 } lair_cf_mode;

/* Interpolation P = [W; I] (Eq. (2.2)): approximate ideal interpolation
 * (W ~ -A_ff^{-1} A_fc, Eq. (2.6), by local solves on the transposed
 * neighbourhoods) or one-point interpolation (Sec. 4). */
typedef enum { LAIR_P_LAIP = 0, LAIR_P_ONEPOINT = 1 } lair_interp;

/* Restriction R = [Z I]: lAIR (Sec. 3.1: Z from the local systems of Eq. (3.2) on the
 * strong F-neighbourhoods) or the Neumann approximation nAIR (Sec. 3.2) that the paper
 * compares it with: Z = -A_cf sum_{m=0}^{k} (D_ff^{-1} E_ff)^m D_ff^{-1} with E_ff = D_ff - A_ff
 * and degree k = distance - 1 (the printed -A_cf sum L_ff^m once A has a unit diagonal),
 * supported on the F points within `distance` edges of the C point in the graph of all
 * nonzeros of A. */
typedef enum { LAIR_R_LAIR = 0, LAIR_R_NEUMANN = 1 } lair_restriction;

/* Post-relaxation after coarse-grid correction (Sec. 4): Jacobi sweeps over
 * F, F, C points (the paper's choice), F, C, F, or F, F only. */
typedef enum { LAIR_RELAX_FFC = 0, LAIR_RELAX_FCF = 1, LAIR_RELAX_FF = 2 } lair_relax;

/* LAIR_FP64: everything in double. LAIR_MIXED: local solves, relaxation, the
 * cycle's residuals and transfers in float; the outer residual, Krylov
 * orthogonalisation, Galerkin products, all structural decisions and the
 * coarsest direct solve stay in double. */
typedef enum { LAIR_FP64 = 0, LAIR_MIXED = 1 } lair_precision;

/* Outer iteration: stationary (iterative refinement x += M^{-1}(b - A x)) or
 * right-preconditioned flexible GMRES with restart (Sec. 4: V-cycles as a
 * GMRES preconditioner). */
typedef enum { LAIR_CYCLE_STATIONARY = 0, LAIR_CYCLE_FGMRES = 1 } lair_cycle;

typedef struct {
    int64_t n;
    int64_t nnz;
    const int64_t *row_ptr;   /* n+1 */
    const int32_t *col;       /* nnz, ascending per row */
    const double *val;        /* nnz */
    int on_device;            /* 1: the three arrays are device pointers */
} lair_csr;

typedef struct {
    int cf_mode;              /* lair_cf_mode (default AUTO) */
    const int8_t *cf_user;    /* LAIR_CF_USER: host array of n entries, nonzero = C, 0 = F; with nodal = k
                                 the k entries of every node must agree (else LAIR_ERR_INVALID_ARG) */
    int distance;             /* restriction/interpolation neighbourhood distance, 1 to 4 (Sec. 3.1, Sec. 4:
                                 each step adds the strong F neighbours of the previous set) */
    double theta;             /* strength threshold for the neighbourhoods (Sec. 4, N_i) */
    double theta_cf;          /* strength threshold for the splitting */
    int strength_abs;         /* 1: compare |a_ij| instead of -a_ij */
    int interp;               /* lair_interp */
    int relax;                /* lair_relax */
    double lump_tol;          /* lumping threshold theta_D on coarse levels (Sec. 3.3), 0 = off */
    int lump_level0;          /* 1: lump the finest operator as well */
    int precision;            /* lair_precision */
    int coarse_max;           /* direct solve once a level has <= coarse_max unknowns */
    int max_levels;
    int block_size;           /* > 1: scale A and b by the inverse block diagonal first (DG, Sec. 4.2.1) */
    int rs_block;             /* AUTO: index-block size of the blocked first pass (1..32768) */
    uint64_t pmis_seed;
    int fgmres_restart;
    void *stream;             /* cudaStream_t, or NULL (see above); never the legacy default stream itself */
    int timing;               /* 1: record CUDA-event timings of the main kernels and set-up phases
                                 (lair_kernel_timers); 2: also one timer per set-up phase and level */
    int restriction;          /* lair_restriction (default lAIR) */
    int nodal;                /* 2..8: nodal (block) hierarchy on nodes of that many consecutive unknowns
                                 (Sec. 3.1 with k x k blocks; Sec. 4.2.1, approach (iii)): strength of
                                 connection on the block Frobenius norms, C/F splitting by node, R from the
                                 block local systems of the node neighbourhoods, one-point P as k x k
                                 identity blocks, lumping by whole blocks, block Jacobi relaxation.
                                 n must be a multiple of it; not with block_size, the Neumann restriction or
                                 batched systems. 0 or 1: off (default). */
    int autotune;             /* 1 (default): before the cycle is captured, time the launch schedules (threads
                                 per block, grid cap) of the restriction, interpolation and sweep views of at
                                 least 65,536 rows and keep the fastest when it beats the default by 5 %;
                                 choices are cached for the process by view shape, so later hierarchies of
                                 similar levels reuse them. Results do not depend on it. 0: the fixed default
                                 schedule everywhere. */
    int wait_polls;           /* bound on the polls of every device-side wait (the grid barriers of the
                                 cooperative PMIS kernel, levels above 8192 points); 0 (default): 4,194,304
                                 polls of the barrier word. A wait that runs out makes the call return
                                 LAIR_ERR_DEVICE_TIMEOUT; every block of the kernel returns and the CUDA
                                 context stays usable. Small values exist to test that path. */
} lair_options;

typedef struct {
    int iters;                /* preconditioner applications (V-cycles) */
    double final_rel;         /* ||b - A x|| / ||b|| of the system solved (scaled one with block_size) */
    double setup_ms;          /* of the handle (filled by every call that reports) */
    double solve_ms;
    int nlevels;
    int64_t singular_R;       /* local systems that took the least-squares branch */
    int64_t singular_P;
    double op_complexity;     /* sum nnz(A_l) / nnz(A_0) */
    double cycle_complexity;  /* nonzeros touched per cycle / nnz(A_0) */
    double *hist;             /* optional, caller-owned: residual history */
    int hist_cap;
    int hist_len;
} lair_report;

typedef struct {
    int64_t n, nnz, nc, nnz_R, nnz_P;
    int is_coarsest;
} lair_level_info;

typedef struct lair_handle lair_handle;

/* Fill *o with the defaults (AUTO splitting, distance 1, theta 0.25, lAIP, F-F-C,
 * lumping 1e-3 on coarse levels, FP64, coarse_max 128, 25 levels, rs_block 4096,
 * FGMRES restart 30). */
lair_status lair_options_default(lair_options *o);

/* Build the hierarchy for A (Sec. 2.1 set-up: strength, splitting, lAIR
 * restriction by the local systems of Eq. (3.2), interpolation, Galerkin
 * product R A P, lumping; recursively). A is copied; *h receives a new handle
 * that the caller releases with lair_free(). On failure *h may still hold a
 * handle (for lair_last_error) that must be freed. */
lair_status lair_setup(const lair_csr *A, const lair_options *o, lair_handle **h);

/* New values for the matrix the hierarchy was built for, on the same pattern: the
 * backward Euler matrix I + dt S of Sec. 4.1.1 when dt or the coefficients change
 * between time steps. val holds A's nnz values in the order of the set-up's CSR (host
 * or device; read before the call returns). The C/F splittings, the neighbourhoods of
 * the local systems (Sec. 3.1), the patterns of R, P and every coarse operator (after
 * lumping, Sec. 3.3), every allocation and the captured cycle are kept; every value is
 * recomputed in the set-up's arithmetic: block scaling, R and lAIP by their local
 * systems on the kept sets, one-point P unchanged (all ones), R A P, the entries of the
 * product outside the kept coarse pattern lumped to the diagonal in ascending column
 * order, Jacobi diagonals, FP32 copies, the coarsest factorisation. An adjoint
 * hierarchy, if built, is refreshed too. With the set-up's own values the result is
 * the set-up's, bit for bit. Errors: LAIR_ERR_INVALID_ARG (NULL arguments, a handle
 * without a complete hierarchy), LAIR_ERR_ZERO_DIAGONAL (a zero pivot on some level);
 * after an error the hierarchy's values are unspecified until a successful refresh. */
lair_status lair_refresh(lair_handle *h, const double *val);

/* Solve A x = b to ||b - A x||/||b|| <= tol. x holds the initial guess on entry
 * (host or device, n doubles) and the result on return. cycle is a lair_cycle;
 * max_iter bounds the V-cycles. rep may be NULL. Returns LAIR_ERR_NOT_CONVERGED
 * if max_iter is reached first. */
lair_status lair_solve(lair_handle *h, const double *b, double *x, double tol, int cycle,
                       int max_iter, lair_report *rep);

/* Batched independent systems. A is the block-diagonal matrix of
 * nsys systems; sys_offsets (host, nsys + 1 entries, from 0 to n) gives each system's first
 * row. One hierarchy is built for the whole batch, so every set-up and cycle step is one
 * launch over all systems of all sizes; nothing couples the systems (the C/F splitting
 * blocks never span two systems), so each system gets the hierarchy it would get alone,
 * apart from the common number of levels. User splittings and block scaling are not
 * available here (LAIR_ERR_INVALID_ARG / LAIR_ERR_UNSUPPORTED). */
lair_status lair_setup_batched(const lair_csr *A, int nsys, const int64_t *sys_offsets, const lair_options *o,
                               lair_handle **h);

/* Solve every system of a batched handle to its own relative residual
 * ||b_q - A_q x_q|| / ||b_q|| <= tol. cycle: LAIR_CYCLE_STATIONARY (FP64 refinement; a system
 * is no longer updated once it has converged) or LAIR_CYCLE_FGMRES (FGMRES per system, all
 * systems stepping together, each with its own rotations, stopping test and restarts).
 * b, x: n doubles (host or device; x holds the initial guess). iters and rel (host, nsys
 * entries, may be NULL) receive per-system cycle counts and final relative residuals.
 * Returns LAIR_ERR_NOT_CONVERGED if some system is still above tol after max_iter cycles. */
lair_status lair_solve_batched(lair_handle *h, const double *b, double *x, double tol, int cycle, int max_iter,
                               int *iters, double *rel);

/* Convenience: set up and solve nsys separate systems in one batch. A[q] (host or device
 * arrays, per A[q].on_device), b[q] and x[q] (host or device, x[q] holds the initial guess
 * and receives the solution) describe system q. The systems are concatenated on the host,
 * solved with lair_setup_batched + lair_solve_batched, and the handle is released. */
lair_status lair_batch_setup_solve(int nsys, const lair_csr *A, const double *const *b, double *const *x,
                                   const lair_options *o, double tol, int cycle, int max_iter, int *iters, double *rel);

/* x = M^{-1} b: one V-cycle with zero initial guess (Sec. 4 cycle), in the
 * handle's precision. b, x: n doubles, host or device. */
lair_status lair_precond_apply(lair_handle *h, const double *b, double *x);

/* Adjoint solve A^T lambda = g (for gradients). The first call builds a second
 * hierarchy on A^T with the same options (C/F splitting of A^T is computed,
 * never taken from cf_user) and keeps it in the handle. */
lair_status lair_adjoint(lair_handle *h, const double *g, double *lambda, double tol, int cycle,
                         int max_iter, lair_report *rep);

/* grad_vals[k] = -lambda[i] * x[j] for every stored entry k = (i, j) of A:
 * the gradient of a scalar loss through x = A^{-1} b with respect to the
 * nonzeros of A, given lambda = A^{-T} dL/dx. All three pointers are of the same
 * kind (host or device); grad_vals has nnz entries. With block scaling the
 * gradient is with respect to the unscaled A. */
lair_status lair_grad_A(lair_handle *h, const double *lambda, const double *x, double *grad_vals);

/* Level sizes. out may hold max_levels entries; *nlevels receives the count. */
lair_status lair_hierarchy_info(const lair_handle *h, lair_level_info *out, int max_levels, int *nlevels);

/* Host copies of one level's CSR (which: 0 = A_l, 1 = R_l, 2 = P_l). Sizes from
 * lair_hierarchy_info (rows + 1, nnz). Any of the three pointers may be NULL. */
lair_status lair_export_csr(const lair_handle *h, int level, int which, int64_t *row_ptr,
                            int32_t *col, double *val);

/* Host copies of one level's splitting (n entries, 1 = C, 0 = F), strength mask
 * over A_l's pattern (nnz entries), and the per-C-point least-squares flags of
 * the restriction and interpolation solves (nc entries each). NULL skips. */
lair_status lair_export_cf(const lair_handle *h, int level, int8_t *cf, uint8_t *strong,
                           uint8_t *ls_R, uint8_t *ls_P);

/* Timing of one kind of kernel launch, accumulated since the handle was created:
 * CUDA events recorded on the launching stream immediately before and after each
 * launch (inside the captured cycle graph for cycle kernels). bytes_per_launch is
 * the algorithmic byte count of one launch (matrix entries read once, vectors read
 * or written once). Filled only when lair_options.timing was set at set-up. */
typedef struct {
    char name[40];
    int64_t launches;
    double total_ms;
    double bytes_per_launch;
} lair_kernel_timer;

/* Copy up to cap timers into out; *count receives the number available. */
lair_status lair_kernel_timers(const lair_handle *h, lair_kernel_timer *out, int cap, int *count);

/* Solve nsys independent dense local systems M_k z_k = rhs_k of one size s without
 * allocating any memory. The paper has no counterpart to this entry point: it exists for
 * callers that cannot call cudaMalloc at the point where they need the solve (code running
 * while a CUDA graph is captured or replayed, processes whose device memory is already
 * handed out to other pools, or latency-critical threads that must stay off the allocator).
 * The solve is the one lair_setup uses for the rows of R (LU with partial pivoting, the
 * minimum-norm least-squares branch for singular systems), so results are bit-identical.
 *   M:       nsys * s * s doubles, row-major per system, device memory (not modified)
 *   rhs:     nsys * s doubles, device memory
 *   z:       nsys * s doubles, device memory, receives the solutions
 *   ls_flag: nsys bytes of device memory or NULL; 1 where the least-squares branch was used
 *   stream:  cudaStream_t (NULL = legacy default stream); the call only enqueues the work
 * Limits: 1 <= s <= 64 (LAIR_ERR_UNSUPPORTED above). Working storage is one fixed device
 * array of 10,194,944 bytes (152 slots of 64*64*2 + 3*64 doubles) that every GPU loading
 * the library holds until the process exits; every call writes what it reads, so nothing
 * of an earlier call leaks in, but all calls share the array: calls that may overlap on the
 * GPU (different streams, or different host threads) race and must be serialised by the
 * caller. The first call on a device looks up the array's device address; make that first
 * call before any stream capture. The address is kept for the life of the process: after
 * cudaDeviceReset() of a device the entry point must not be used on that device again.
 * Returns LAIR_ERR_INVALID_ARG for NULL pointers or s < 1, and LAIR_ERR_CUDA, without
 * launching, if an earlier CUDA error is still pending on the calling thread. */
lair_status lair_local_solve_noalloc(int64_t nsys, int32_t s, const double *M, const double *rhs, double *z,
                                     uint8_t *ls_flag, void *stream);

/* Number of device kernels the library has launched since the handle was created. */
int64_t lair_kernel_launches(const lair_handle *h);

void lair_free(lair_handle *h);
const char *lair_status_string(lair_status s);
const char *lair_last_error(const lair_handle *h);

#ifdef __cplusplus
}
#endif
#endif /* LAIR_H */
