// Launchers of the DFC-LRR kernels (one translation unit per family).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <cstring>

namespace lrr {

// ---------------------------------------------------------------- grouped GEMM
// C_g = alpha * op(A_g) * op(B_g) + beta * C_g for every group g whose flag is
// nonzero (flag == nullptr: always).  Column-major, op = transpose if trans*.
// ccol (optional, device, int64): column j of the product is stored at column
// ccol[j] of C (used to undo the D-step permutation).
template <typename T>
struct GemmDesc {
    const T* A;
    const T* B;
    T* C;
    const int* flag;
    const int64_t* ccol;
    const T* kscale;      // optional: op(A)(i,k) is multiplied by kscale[k]
    T* absmax;            // optional: store nothing, atomically max |alpha op(A) op(B)| here
    int64_t lda, ldb, ldc;
    int m, n, k;
    T alpha, beta;
};

template <typename T>
cudaError_t gemm_grouped(const GemmDesc<T>* d_desc, int groups, bool transA, bool transB, int max_m, int max_n,
                         cudaStream_t s);

// ---------------------------------------------------------- batched Jacobi eig
// Symmetric matrices G_i (pp_i x pp_i, ld pp_i, pp_i a multiple of 2*bs) are
// reduced to diagonal form in place by block Jacobi rotations, accumulated into
// W_i (pp_i x pp_i, ld pp_i): on exit G_in = W diag(G_out) W^T.
template <typename T>
struct JacDesc {
    T* G;
    T* W;
    T* R;          // rotation scratch: (pp/(2bs)) * (2bs)^2 values
    int* rot;      // per pivot pair of the current round: 1 if its rotation is not the identity
    int* done;     // per matrix: 1 when converged (checked before each sweep)
    T* off;        // per matrix: max scaled off-diagonal seen in the current sweep
    const int* active;  // optional: skip when *active == 0
    const T* scale;     // per matrix: max |G_ii| at entry (off-diagonals below eps*scale are zero)
    int pp;        // padded order (multiple of 2*bs)
};

// Runs up to `sweeps` cyclic block-Jacobi sweeps (round-robin pairing of the
// pp/bs diagonal blocks) on every matrix; a matrix stops once a whole sweep
// saw no scaled off-diagonal |G_ij|/sqrt(G_ii G_jj) above tol.  bs = 16 for
// double, 32 for float.  `done` and `off` are reset at entry.
// With done_dev (the `done` word of a single matrix) the host reads it after
// every sweep and stops launching once it is set; sweeps_run (host) receives
// the sweeps launched.
template <typename T>
cudaError_t jacobi_sweeps(const JacDesc<T>* d_desc, int nmat, int max_pp, int sweeps, T tol, cudaStream_t s,
                         const int* done_dev = nullptr, int* sweeps_run = nullptr);
// One-sided block Jacobi (osj.cu): X (L x p, ld ldx) is rotated to orthogonal
// columns together with W (p x p, ld ldw); pp = p rounded up to the pivot
// width.  off points at three slots (the per-sweep convergence maxima).
template <typename T>
struct OsjDesc {
    T* X;
    T* W;
    int* done;
    T* off;
    const int* active;
    const T* scale;     // largest squared column norm of X
    const double* mu;   // SVT threshold is 1/mu (nullptr: measure every pair)
    int64_t ldx, ldw;
    int L, p, pp;
    int strict;         // 1: resolve pairs straddling tau to angle tol (C-step block)
    int* ctr;           // optional: two ints of scratch; the cluster's CTAs then take the
                        // pivots of a round from a shared counter instead of a fixed share
};

// One launch: every block is a thread-block cluster of `cluster` CTAs (0:
// one per pivot of a round, up to osj_max_cluster()) that runs its sweeps
// until converged or `sweeps` are done.  `quad_exit`: stop one sweep early
// once quadratic convergence guarantees the tolerance (see osj_svd).
template <typename T>
cudaError_t osj_sweeps(const OsjDesc<T>* d_desc, int nmat, int max_pp, int sweeps, T tol, int* sweeps_run,
                       cudaStream_t s, int cluster = 0, int quad_exit = 0);
// largest cluster size osj_sweeps uses on the current device (16 or 8)
template <typename T>
int osj_max_cluster();

template <typename T> constexpr int jacobi_bs() { return sizeof(T) == 8 ? 16 : 32; }
// pivot width of the one-sided Jacobi (two column blocks of 16); the column
// count p of its matrices is padded to a multiple of it
constexpr int osj_pivot_width() { return 32; }

// D step (partition.cu, host): perm and/or offsets of dfc_partition
void draw_partition(int64_t n, int t, uint64_t seed, int64_t* perm, int64_t* offsets);

// ------------------------------------------------------ tensor-core product
// C (M x N, column-major, float) = A B, A and B bf16 and K-major (tc_gemm.cu).
cudaError_t tc_gemm_bf16(const void* A, int64_t lda, const void* B, int64_t ldb, float* C, int64_t ldc, int M, int N,
                         int K, int* err, cudaStream_t s);

// Float32-accurate product on the tensor cores (split TF32): C (M x N,
// column-major, float) = A B from A = Ahi + Alo and B = Bhi + Blo, all four
// float32, K-major, 16-byte aligned, lda and ldb multiples of 4, hi the
// nearest TF32 value and lo the nearest TF32 value to the rest (split_tf32
// below).
// With flag != nullptr, 128-column tiles of C whose columns all belong to
// blocks b (colblk) with flag[b] == 0 are left untouched.
cudaError_t tc_gemm_3xtf32(const float* Ahi, const float* Alo, int64_t lda, const float* Bhi, const float* Blo,
                           int64_t ldb, float* C, int64_t ldc, int M, int N, int K, const int* colblk,
                           const int* flag, int* err, cudaStream_t s);

// The same from split bf16 operands ("bf16x3"): A = Ahi + Alo, B = Bhi + Blo,
// all four bf16, K-major, 16-byte aligned, lda and ldb multiples of 8, hi the
// nearest bf16 value and lo the nearest bf16 value to the rest (split_bf16).
// Relative error per product term about 2^-16, against 2^-8 for tc_gemm_bf16.
cudaError_t tc_gemm_bf16x3(const void* Ahi, const void* Alo, int64_t lda, const void* Bhi, const void* Blo,
                           int64_t ldb, float* C, int64_t ldc, int M, int N, int K, int* err, cudaStream_t s);

// Split of x into hi + lo for the split-TF32 product: hi = x rounded to the
// nearest TF32 value (10 explicit mantissa bits), lo = (x - hi) rounded to
// the nearest TF32 value.  Both are exact TF32 numbers, so the tensor cores
// use them without further rounding; |x - hi - lo| <= 2^-22 |x|, with
// unbiased signs (truncation would bias every product the same way).
__host__ __device__ __forceinline__ float tf32_rn(float x) {
    uint32_t u;
#ifdef __CUDA_ARCH__
    u = __float_as_uint(x);
#else
    memcpy(&u, &x, 4);
#endif
    if ((u & 0x7F800000u) != 0x7F800000u) u = (u + 0x1000u) & 0xFFFFE000u;   // finite: round half away
    float r;
#ifdef __CUDA_ARCH__
    r = __uint_as_float(u);
#else
    memcpy(&r, &u, 4);
#endif
    return r;
}
__host__ __device__ __forceinline__ void split_tf32(float x, float& hi, float& lo) {
    hi = tf32_rn(x);
    lo = tf32_rn(x - hi);
}

// Reduction form of the same product: C is not stored; for every column block b
// (colblk maps a column of C to its block) with need[b] != 0 the largest |C_ij|
// over its columns is folded into bmax[b] (float bits, atomicMax; bmax must hold
// nonnegative values on entry).  Tiles whose columns belong to no such block,
// and the whole launch when *run == 0 (run may be null), do nothing.
struct TcAbsmax {
    const int* run;
    const int* colblk;
    const int* need;
    unsigned* bmax;
};
cudaError_t tc_gemm_bf16_absmax(const void* A, int64_t lda, const void* B, int64_t ldb, int M, int N, int K,
                                TcAbsmax am, int* err, cudaStream_t s);

}  // namespace lrr
