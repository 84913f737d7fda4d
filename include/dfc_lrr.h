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
                            iteration bulk (split bf16: hi and lo parts of each
                            float32 operand, three bf16 MMAs per product), float32
                            refinement phase to convergence                           */
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
    int32_t tc_products;        /* F32/MIXED: 1 = the float32 products of the iteration on
                                   the tensor cores in split TF32 (each product float32-
                                   accurate, see lrr_gemm_f32); 0 (default) = on the CUDA
                                   cores.  Over a whole solve the split-TF32 iterate drifts
                                   further from the float64 oracle (3.1e-5 against 1.5e-6
                                   relative in block 1 of the 1000 x 20000 workload), so
                                   it is not the default                                 */
    int32_t autotune;           /* 1: pick the launch shapes of the Jacobi and of the
                                   products by timing the candidates on the first solve
                                   of each problem shape (cached per process and device);
                                   0: fixed defaults                                     */
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
    /* Factored form of the combined estimate (Section 2.2: the column
     * projection is cheap because the block solutions come in factored form;
     * Z = F G costs (n + n) k values instead of n^2):  Z = F[:, :k] G[:k, :]
     * with F orthonormal.  kmax = lrr_factor_max_rank(p); k <= kmax is
     * returned in *factor_k.  For t > 1, F spans the column space of Z_1 (the
     * C step's basis, k = k1) and G = F^T [Z_1 ... Z_t]; for t = 1, F is the
     * right singular basis V of M (k = rank(M)) and G = V^T Z. */
    void* F;                    /* (device, may be NULL) n x kmax, ld n                   */
    void* G;                    /* (device, may be NULL) kmax x n, ld kmax, original
                                   column order                                          */
    int32_t* factor_k;          /* (host, may be NULL) 1: k                               */
    int32_t* sweeps;            /* (host, may be NULL) t: Jacobi sweeps run per block,
                                   summed over its iterations                            */
} lrr_result;

/* Largest k the factored output (lrr_result.F / .G) can have: min(m, l_1)
 * for t > 1 (l_1 = offsets[1], the first block's width), min(m, n) for t = 1.
 * 0 for an invalid problem. */
LRR_API int64_t lrr_factor_max_rank(const lrr_problem* p);

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

/* The alternative formulation of the footnote to eq. (2): both instances of
 * M become C_i, so block i solves
 *   min ||Z_i||_* + lambda ||S_i||_{2,1}  s.t.  C_i = C_i Z_i + S_i   (Z_i: l_i x l_i),
 * and the C step is a low-rank approximation of diag(Z_1, ..., Z_t): its
 * truncated SVD at rank `rank` (<= 0: k1, the SVT rank of block 1 at its final
 * iteration; the footnote leaves the rank open).  The block problems have
 * different dictionaries and run as independent problems on `streams`
 * concurrent streams (lrr_solve_batch).  r->Z (device, n x n, original order;
 * zero outside the diagonal blocks) and r->S as for dfc_lrr_solve; r->F/G are
 * not produced (LRR_ERR_UNSUPPORTED if given); r->ranks = [largest rank(C_i),
 * rank used, SVT rank of each block].  Scratch via cudaMallocAsync.
 * Returns an lrr_status. */
LRR_API int dfc_lrr_solve_local(const lrr_problem* p, const lrr_options* o, int64_t rank, lrr_result* r,
                                int32_t streams, void* stream);

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

/* The float32-accurate tensor-core product of the iteration on its own:
 * C = A B with A (M x K) and B (K x N) float32, both stored K-major (element
 * (m, k) at A[k + m lda], element (k, n) at B[k + n ldb]); C float,
 * column-major, ldc >= M; N <= 8388480.  Every operand is split into a TF32
 * part and a float32 remainder and three TF32 tensor-core products are summed
 * in float32 (error near that of a float32 product; the remainders' product,
 * below 2^-20 |a||b| per term, is dropped).  All device pointers; scratch (the
 * split operands, 8 (M + N) K bytes) is taken with cudaMallocAsync; the call
 * synchronises `stream`. */
LRR_API int lrr_gemm_f32(const float* A, int64_t lda, const float* B, int64_t ldb, float* C, int64_t ldc, int64_t M,
                         int64_t N, int64_t K, void* stream);

/* Device time of the iteration's tensor-core product alone, for measuring
 * it: kind 0 = the bf16 product (lrr_gemm_bf16), kind 1 = the split-TF32
 * product (lrr_gemm_f32) on operands already split, kind 2 = the split-bf16
 * product of the mixed form's bf16 phase (three bf16 MMAs, operands already
 * split).  Fills synthetic M x K and K x N operands in scratch taken with cudaMallocAsync, launches the
 * kernel once untimed and `repeat` times back to back between two CUDA
 * events on `stream`, and stores the mean time per launch (ms). */
LRR_API int lrr_gemm_timing(int32_t kind, int64_t M, int64_t N, int64_t K, int32_t repeat, double* ms_per_launch,
                            void* stream);

/* Differentiable unrolled LRR.  The map (M, lambda) -> Z_K: plain LRR
 * (eq. (1), t = 1, the observations are the dictionary) run for exactly K
 * iterations of the inexact ALM the solver uses (Section 4's base solver),
 * from the zero start, the K-th iteration without its dual step; the penalty
 * follows the fixed schedule mu_k = min(rho^(k-1) mu0, mu_max).
 * lrr_unrolled_backward returns the gradients of a loss L(Z_K) given
 * Zbar = dL/dZ_K: dL/dM (both the dictionary's and the observations' part)
 * and dL/dlambda, by a hand-written reverse pass (the SVT derivative through
 * the singular triplets, the column-shrink Jacobian, the Z-update solve, the
 * dual steps) that recomputes the iterates from states kept every
 * `checkpoint` iterations. */
typedef struct {
    double lambda;          /* > 0                                                    */
    double rho;             /* >= 1                                                   */
    double mu0;             /* > 0                                                    */
    double mu_max;          /* >= mu0                                                 */
    double rank_tol;        /* rank(M) threshold relative to sigma_max (0 -> 1e-6)    */
    int32_t K;              /* iterations, >= 1                                       */
    int32_t checkpoint;     /* iterations between kept states (0 -> 5)                */
    int32_t precision;      /* LRR_PREC_F32 or LRR_PREC_F64                           */
} lrr_unrolled_options;

/* Device workspace for a forward (with_grad = 0) or backward (with_grad = 1)
 * call of an m x n problem (0 on invalid arguments); m <= 4096, n <= 16384. */
LRR_API size_t lrr_unrolled_workspace_bytes(int64_t m, int64_t n, const lrr_unrolled_options* o, int32_t with_grad);

/* Z (device, n x n, ld ldz >= n) = Z_K(M, lambda).  M (device) m x n, ld ldm,
 * float or double as o->precision.  workspace NULL: cudaMallocAsync on
 * stream.  Synchronises stream.  Returns an lrr_status. */
LRR_API int lrr_unrolled_forward(const void* M, int64_t m, int64_t n, int64_t ldm, const lrr_unrolled_options* o,
                                 void* Z, int64_t ldz, void* workspace, size_t workspace_bytes, void* stream);

/* Mbar (device, m x n, ld ldmb) = dL/dM and *lambar (host) = dL/dlambda for
 * Zbar = dL/dZ_K (device, n x n, ld ldzb).  Synchronises stream. */
LRR_API int lrr_unrolled_backward(const void* M, int64_t m, int64_t n, int64_t ldm, const lrr_unrolled_options* o,
                                  const void* Zbar, int64_t ldzb, void* Mbar, int64_t ldmb, double* lambar,
                                  void* workspace, size_t workspace_bytes, void* stream);

/* Segmentation of an estimate Z (Section 4.1.2's post-processing), on the
 * GPU, from its factored form Z = F[:, :k] G[:k, :] (lrr_result.F / .G):
 * U = the left singular vectors of Z with singular value > rel_tol * s_max
 * (the paper's "top" singular vectors; reading: rel_tol = 1e-6), affinity
 * |U U^T|, the `clusters` leading eigenvectors of the normalised affinity
 * D^-1/2 |U U^T| D^-1/2 (the smallest of the normalised Laplacian; subspace
 * iteration, power_iters steps), rows scaled to unit norm, then k-means
 * (k-means++ seeding from SplitMix64 of seed, `restarts` restarts, the lowest
 * cost wins).  F (device, n x k, ld ldf), G (device, k x n, ld ldg) float;
 * labels (host, n) receives cluster indices 0..clusters-1.  The n x n
 * affinity lives in the workspace (lrr_segment_workspace_bytes; NULL:
 * cudaMallocAsync).  clusters <= 64.  Synchronises stream. */
LRR_API size_t lrr_segment_workspace_bytes(int64_t n, int64_t k, int32_t clusters, int32_t restarts);
LRR_API int lrr_segment(const float* F, int64_t ldf, const float* G, int64_t ldg, int64_t n, int64_t k,
                        int32_t clusters, double rel_tol, uint64_t seed, int32_t restarts, int32_t power_iters,
                        int32_t* labels, void* workspace, size_t workspace_bytes, void* stream);

/* `count` independent problems (each its own M, sizes and partition) solved
 * with dfc_lrr_solve under the same options, concurrently: `streams` host
 * threads (0 -> 8) each drive their own CUDA stream and take the next problem
 * when one is done; every problem's scratch is stream-ordered on its stream
 * (so the options' workspace is not used).  The call first synchronises
 * `stream` (inputs ready), returns after every problem is solved, writes each
 * problem's status into status[i] (host, may be NULL) and returns the worst
 * (a failure before LRR_NOT_CONVERGED before LRR_OK).  results (host, count
 * entries, may be NULL) as for dfc_lrr_solve. */
LRR_API int lrr_solve_batch(const lrr_problem* problems, int32_t count, const lrr_options* o, lrr_result* results,
                            int32_t* status, int32_t streams, void* stream);

/* Fill `o` with the defaults above (lambda = 0.1). */
LRR_API void lrr_default_options(lrr_options* o);

/* Static description of a status code. */
LRR_API const char* lrr_status_string(int status);

#ifdef __cplusplus
}
#endif
#endif /* DFC_LRR_H */
