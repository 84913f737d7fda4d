// Grouped general matrix product on the CUDA cores (float32 / float64).
// This is the accurate product of the plain-precision path: every group is an
// independent column-major product C = alpha op(A) op(B) + beta C.
#include "common.cuh"
#include "kernels.cuh"

namespace lrr {
namespace {

constexpr int BM = 64, BN = 64, BK = 16, NT = 256;

template <typename T, bool TA, bool TB>
__global__ void __launch_bounds__(NT) gemm_kernel(const GemmDesc<T>* __restrict__ descs, int tiles_m) {
    const GemmDesc<T> d = descs[blockIdx.z];
    if (d.flag && *d.flag == 0) return;
    const int tm = blockIdx.x % tiles_m, tn = blockIdx.x / tiles_m;
    const int m0 = tm * BM, n0 = tn * BN;
    if (m0 >= d.m || n0 >= d.n) return;

    __shared__ T As[BK][BM + 1];
    __shared__ T Bs[BK][BN + 1];
    const int t = threadIdx.x;
    const int tx = t % 16, ty = t / 16;
    T acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = T(0);

    for (int k0 = 0; k0 < d.k; k0 += BK) {
        // A tile: element (i, kk) of op(A)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            int i, kk;
            if (!TA) { i = t % BM; kk = t / BM + 4 * q; }
            else     { kk = t % BK; i = t / BK + 16 * q; }
            const int gi = m0 + i, gk = k0 + kk;
            T v = T(0);
            if (gi < d.m && gk < d.k) {
                v = TA ? d.A[gk + (int64_t)gi * d.lda] : d.A[gi + (int64_t)gk * d.lda];
                if (d.kscale) v *= d.kscale[gk];
            }
            As[kk][i] = v;
        }
        // B tile: element (kk, j) of op(B)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            int j, kk;
            if (!TB) { kk = t % BK; j = t / BK + 16 * q; }
            else     { j = t % BN; kk = t / BN + 4 * q; }
            const int gj = n0 + j, gk = k0 + kk;
            T v = T(0);
            if (gj < d.n && gk < d.k) v = TB ? d.B[gj + (int64_t)gk * d.ldb] : d.B[gk + (int64_t)gj * d.ldb];
            Bs[kk][j] = v;
        }
        __syncthreads();
        // each BK-long slab of the sum is formed in a fresh partial and then
        // added to the accumulator: one long chain of FMAs into a single
        // register lets rounding grow with K (with K in the thousands it
        // doubled the float32 error of the iterate on face-like data), while
        // slab partials keep it near that of a blocked sum
        T part[4][4];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) part[i][j] = T(0);
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            T a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[kk][tx + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = Bs[kk][ty + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) part[i][j] = fma(a[i], b[j], part[i][j]);
        }
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[i][j] += part[i][j];
        __syncthreads();
    }
    if (d.absmax) {
        T mx = T(0);
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int i = 0; i < 4; ++i)
                if (n0 + ty + 16 * j < d.n && m0 + tx + 16 * i < d.m) mx = fmax(mx, fabs(d.alpha * acc[i][j]));
        mx = warp_max(mx);
        if ((t & 31) == 0) atomic_max_nonneg(d.absmax, mx);
        return;
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int gj = n0 + ty + 16 * j;
        if (gj >= d.n) continue;
        const int64_t cj = d.ccol ? d.ccol[gj] : gj;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int gi = m0 + tx + 16 * i;
            if (gi >= d.m) continue;
            T* c = d.C + gi + cj * d.ldc;
            T v = d.alpha * acc[i][j];
            if (d.beta != T(0)) v = fma(d.beta, *c, v);
            *c = v;
        }
    }
}

}  // namespace

template <typename T>
cudaError_t gemm_grouped(const GemmDesc<T>* d_desc, int groups, bool transA, bool transB, int max_m, int max_n,
                         cudaStream_t s) {
    if (groups <= 0 || max_m <= 0 || max_n <= 0) return cudaSuccess;
    const int tiles_m = (int)ceil_div(max_m, BM), tiles_n = (int)ceil_div(max_n, BN);
    dim3 grid((unsigned)(tiles_m * tiles_n), 1, (unsigned)groups);
    if (!transA && !transB) gemm_kernel<T, false, false><<<grid, NT, 0, s>>>(d_desc, tiles_m);
    else if (transA && !transB) gemm_kernel<T, true, false><<<grid, NT, 0, s>>>(d_desc, tiles_m);
    else if (!transA && transB) gemm_kernel<T, false, true><<<grid, NT, 0, s>>>(d_desc, tiles_m);
    else gemm_kernel<T, true, true><<<grid, NT, 0, s>>>(d_desc, tiles_m);
    return cudaGetLastError();
}

template cudaError_t gemm_grouped<float>(const GemmDesc<float>*, int, bool, bool, int, int, cudaStream_t);
template cudaError_t gemm_grouped<double>(const GemmDesc<double>*, int, bool, bool, int, int, cudaStream_t);

}  // namespace lrr
