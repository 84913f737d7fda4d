/*
 * dfc_lrr.h -- C ABI of the GB300 (sm_103a) DFC-LRR solver.
 *
 * Problem (eq. (1), Section 1; eq. (2), Section 2.2):
 *   LRR       min ||Z||_* + lambda ||S||_{2,1}   s.t.  M = M Z + S
 *   block i   min ||Z_i||_* + lambda ||S_i||_{2,1} s.t. C_i = M Z_i + S_i
 * with ||.||_* the nuclear norm and ||.||_{2,1} the sum of column 2-norms.
 * DFC-LRR (Algorithm 1, Section 2.2): D step = random column partition of M
 * into t blocks C_i (passed in as `perm` + `offsets`, or drawn by the library
 * from `seed`, see dfc_partition); F step = the t block
 * problems, each solved by the inexact augmented-Lagrangian iteration named as
 * the base solver in Section 4; C step = column projection of
 * [Z_1 ... Z_t] onto the column space of Z_1.
 *
 * Memory: every array argument marked (device) is a device pointer that the
 * caller allocates and owns; (host) arrays are ordinary host memory.  Matrices
 * are column-major.  The library never frees caller memory.  Work memory is a
 * single caller-provided device buffer of at least lrr_workspace_bytes() bytes
 * (256-byte aligned); with workspace == NULL the library allocates it with
 * cudaMallocAsync on `stream` and frees it before returning.
 *
 * Streams: all device work is queued on `stream`; the call returns after the
 * stream has drained the solve (it reads convergence flags and the per-block
 * counters back to the host).
 *
 * Errors: every entry point returns an lrr_status.  Negative values are
 * failures (nothing in `result` is valid); LRR_NOT_CONVERGED (> 0) means all
 * outputs are written but at least one block stopped at max_iter.  No entry
 * point aborts, traps or prints.
 */
#ifndef DFC_LRR_H
#define DFC_LRR_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define LRR_API __attribute__((visibility("default")))
#else
#define LRR_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    LRR_OK = 0,
    LRR_NOT_CONVERGED = 1,      /* outputs valid, some block hit max_iter            */
    LRR_ERR_INVALID = -1,       /* bad size, pointer, option or partition            */
    LRR_ERR_NONFINITE = -2,     /* M holds NaN or Inf                                */
    LRR_ERR_CUDA = -3,          /* a CUDA runtime call failed                        */
    LRR_ERR_WORKSPACE = -4,     /* workspace too small or misaligned                 */
    LRR_ERR_RANK = -5,          /* M is numerically zero                             */
    LRR_ERR_UNSUPPORTED = -6,   /* option combination not built: MIXED needs n <= 8388480
                                   (65535 tensor-core column tiles)                      */
    LRR_ERR_TOO_LARGE = -7      /* problem exceeds lrr_svt_noalloc's fixed scratch array */
} lrr_status;

typedef enum {
    LRR_PREC_F64 = 0,    /* every step in float64                                     */
    LRR_PREC_F32 = 1,    /* iteration in float32, one-time factor in float64          */
    LRR_PREC_MIXED = 2   /* bf16 tensor-core products with float32 accumulation in the
                            iteration bulk, float32 refinement phase to convergence    */
} lrr_precision;

typedef struct {
    const void* M;              /* (device) m x n, column-major, leading dim ldm >= m;
                                   float for F32/MIXED, double for F64                  */
    int64_t m, n, ldm;
    int32_t t;                  /* number of column blocks, 1 <= t <= n                  */
    const int64_t* perm;        /* (host) n: block i observes the original columns
                                   perm[offsets[i] .. offsets[i+1]-1]; a permutation.
                                   NULL: the permutation dfc_partition draws from seed    */
    const int64_t* offsets;     /* (host) t+1, offsets[0] = 0, offsets[t] = n, strictly
                                   increasing.  NULL: the even split of dfc_partition     */
    uint64_t seed;              /* used only when perm is NULL                           */
} lrr_problem;

typedef struct {
    double lambda;              /* > 0                                                   */
    double rho;                 /* penalty growth, > 1 (1.1)                             */
    double mu0;                 /* initial penalty, > 0 (1e-6)                           */
    double mu_max;              /* penalty cap (1e10)                                    */
    double eps;                 /* stop when ||C-MZ-S||_inf < eps and ||Z-J||_inf < eps  */
    int32_t max_iter;           /* >= 1 (1000)                                           */
    int32_t precision;          /* lrr_precision                                         */
    int32_t batched;            /* 1: all blocks advance together in every launch;
                                   0: blocks are solved one after another                */
    int32_t jacobi_sweeps;      /* max Jacobi sweeps per SVT (0 -> default 12)           */
    double rank_tol;            /* rank(M) = #{sigma > rank_tol * sigma_max} (0 -> 1e-6)  */
    double mixed_switch;        /* MIXED: a block leaves the bf16 products for good once
                                   ||Z + Y2/mu||_F > mixed_switch / mu, i.e. just before
                                   its SVT first keeps a direction (0 -> 0.5)            */
    int32_t profile;            /* 1: record per-phase CUDA-event times into stats     */
} lrr_options;

/* Per-phase device time of one solve, measured with CUDA events recorded on
 * the solve's stream around each phase (only when lrr_options.profile != 0),
 * and kernel-launch counts (always). */
#define LRR_NPHASE 12
enum {
    LRR_PH_SETUP = 0,       /* checks, M M^T, its eigendecomposition, V          */
    LRR_PH_GRAM = 1,        /* SVT Gram products A^T A / A A^T                    */
    LRR_PH_WARM = 2,        /* (unused: the warm start is folded into GRAM)       */
    LRR_PH_JACOBI = 3,      /* block-Jacobi sweeps                                */
    LRR_PH_SVT_APPLY = 4,   /* H = W h W^T and J = A H (or H A), gate, weights   */
    LRR_PH_ZGEMM = 5,       /* U^T P                                              */
    LRR_PH_ZUPDATE = 6,     /* Z-step, Y2 step, next SVT input                    */
    LRR_PH_MZGEMM = 7,      /* U diag(sigma) Z                                    */
    LRR_PH_EUPDATE = 8,     /* E-step, Y1 step, residual                          */
    LRR_PH_STOP = 9,        /* stop test: bounds, bf16 tensor-core ||Z-J||_inf
                               stage, float32 products for undecided blocks       */
    LRR_PH_COMBINE = 10,    /* C step and output scatter                          */
    LRR_PH_HOST = 11        /* host synchronisation points (flag read-back)       */
};
typedef struct {
    double phase_ms[LRR_NPHASE];
    int64_t phase_launches[LRR_NPHASE];
    int64_t launches;           /* kernels launched by the call                       */
    int64_t iterations;         /* ALM iterations launched (all blocks together)      */
    int64_t svt_sweeps;         /* Jacobi sweeps run, summed over blocks and iterations */
    int64_t svt_calls;          /* SVTs that needed an SVD, summed over blocks          */
} lrr_stats;

typedef struct {
    void* Z;                    /* (device, may be NULL) n x n, ld n, original column
                                   order: the combined estimate (Algorithm 1 output)      */
    void* S;                    /* (device, may be NULL) m x n, ld m, original order      */
    int32_t* iters;             /* (host, may be NULL) t: ALM iterations per block        */
    double* resid;              /* (host, may be NULL) t x 2: final ||C_i-MZ_i-S_i||_inf,
                                   ||Z_i-J_i||_inf per block                              */
    int32_t* ranks;             /* (host, may be NULL) t+2: [rank(M), k1, SVT rank of each
                                   block at its final iteration]                          */
    double* timings_ms;         /* (host, may be NULL) 3: setup, iteration, combine        */
    lrr_stats* stats;           /* (host, may be NULL) per-phase times and launch counts  */
} lrr_result;

/* D step of Algorithm 1 (Section 2.2), on the host: a uniformly random
 * permutation of 0..n-1 into perm (n entries, may be NULL) and the even split
 * offsets[i] = floor(i n / t) into offsets (t+1 entries, may be NULL).  The
 * permutation is Durstenfeld's Fisher-Yates shuffle of the identity driven by
 * SplitMix64 seeded with `seed` (uniform integers by rejection), so a seed
 * fixes it on every platform.  The solve calls this when lrr_problem.perm or
 * .offsets is NULL.  Returns LRR_ERR_INVALID unless 1 <= t <= n and at least
 * one output is given.  Needs no GPU. */
LRR_API int dfc_partition(int64_t n, int32_t t, uint64_t seed, int64_t* perm, int64_t* offsets);

/* Bytes of device workspace a solve of `p` with options `o` needs (0 on invalid
 * arguments). */
LRR_API size_t lrr_workspace_bytes(const lrr_problem* p, const lrr_options* o);

/* Plain LRR, eq. (1): requires p->t == 1 (the one block is all of M, in the
 * order given by perm).  No C step.  Returns an lrr_status. */
LRR_API int lrr_solve(const lrr_problem* p, const lrr_options* o, void* workspace, size_t workspace_bytes,
              lrr_result* r, void* stream);

/* DFC-LRR, Algorithm 1: the t block problems of eq. (2) (F step), then the
 * column projection onto the column space of Z_1 (C step; skipped for t == 1,
 * where it is the identity).  Returns an lrr_status. */
LRR_API int dfc_lrr_solve(const lrr_problem* p, const lrr_options* o, void* workspace, size_t workspace_bytes,
                  lrr_result* r, void* stream);

/* Singular-value thresholding, the proximal map of tau ||.||_* that forms the
 * J-step of every ALM iteration: for A = U diag(s) V^T,
 *   J = U diag(max(s - tau, 0)) V^T.
 * A (device, rows x cols, ld lda) and J (device, rows x cols, ld ldj) are
 * column-major float (precision LRR_PREC_F32) or double (LRR_PREC_F64); J may
 * not alias A.  *rank (host, may be NULL) receives #{s > tau}.  Computed as in
 * the solver: one-sided block Jacobi on the columns of A (tall) or A^T (wide),
 * from a cold start.  Scratch memory is taken with cudaMallocAsync on `stream`
 * and released before returning; the call synchronises `stream`.
 * rows, cols <= 65536. */
LRR_API int lrr_svt(const void* A, int64_t rows, int64_t cols, int64_t lda, double tau, void* J, int64_t ldj,
                    int32_t precision, int32_t* rank, void* stream);

/* lrr_svt without any memory allocation.  Same operation, arguments and
 * result as lrr_svt; the paper has no counterpart.  It serves callers that
 * cannot call cudaMalloc (or any allocator) at the point where they need an
 * SVT: code whose device memory is owned by another allocator that must not
 * be bypassed (a framework's caching pool, a fixed arena reserved at start-up),
 * and code on a latency-critical path where a pool that grows on demand could
 * stall it.  The caller still owns A and J.
 * Scratch: one file-scope device array of lrr_svt_noalloc_capacity() bytes
 * (32 MiB), present on every device that loads the library until the process
 * exits.  A problem whose scratch would exceed it (float32 square matrices up
 * to about 1400 x 1400, float64 about 1000 x 1000) returns LRR_ERR_TOO_LARGE.
 * The first call on a device looks up the array's device address (with that
 * device current); make that first call before any stream capture.  Every
 * call uses the same array and writes everything it reads, so calls are
 * independent when they run one after another; calls that overlap on the GPU
 * (several streams or host threads at once) race on the array and must not be
 * issued.  The call copies a few scalars from host memory to the array and
 * synchronises `stream` before it returns. */
LRR_API int lrr_svt_noalloc(const void* A, int64_t rows, int64_t cols, int64_t lda, double tau, void* J, int64_t ldj,
                            int32_t precision, int32_t* rank, void* stream);

/* Size in bytes of lrr_svt_noalloc's fixed scratch array. */
LRR_API size_t lrr_svt_noalloc_capacity(void);

/* The tensor-core product of the mixed-precision iteration on its own:
 * C = A B with A (M x K) and B (K x N) bf16, both stored K-major (element
 * (m, k) at A[k + m lda], element (k, n) at B[k + n ldb]), lda and ldb
 * multiples of 8, A and B 16-byte aligned; C float, column-major, ldc >= M;
 * N <= 8388480 (65535 column tiles of 128; larger N is LRR_ERR_INVALID).
 * All device pointers; the call
 * synchronises `stream` and returns LRR_ERR_CUDA if a launch failed or a wait
 * inside the kernel timed out.
 * Scratch: one int taken with cudaMallocAsync. */
LRR_API int lrr_gemm_bf16(const void* A, int64_t lda, const void* B, int64_t ldb, float* C, int64_t ldc, int64_t M,
                          int64_t N, int64_t K, void* stream);

/* Fill `o` with the defaults above (lambda = 0.1). */
LRR_API void lrr_default_options(lrr_options* o);

/* Static description of a status code. */
LRR_API const char* lrr_status_string(int status);

#ifdef __cplusplus
}
#endif
#endif /* DFC_LRR_H */
