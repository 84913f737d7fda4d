// Segmentation of the combined estimate on the GPU (Section 4.1.2's
// post-processing): affinity |U U^T| from the left singular vectors U of Z with
// singular values above rel_tol * sigma_max, normalised spectral embedding in
// K dimensions, k-means.
//
// Z arrives in the factored form the solver returns (Z = F G, F orthonormal,
// n x k, and G, k x n), so its left singular vectors are F times those of G:
// the one-sided Jacobi on G^T gives G^T W with orthogonal columns, i.e.
// G = W diag(s) Vg^T, and U = F W restricted to the kept columns.
//   affinity     A = |U U^T| (n x n, float32, materialised), degrees d = A 1
//   embedding    the K leading eigenvectors of D^-1/2 A D^-1/2 (the K smallest
//                of the normalised Laplacian) by subspace iteration on
//                (I + D^-1/2 A D^-1/2)/2 with Cholesky re-orthonormalisation,
//                rows scaled to unit norm
//   k-means      one CTA per restart: k-means++ seeding from a counter-based
//                generator (SplitMix64 of seed, restart, step), Lloyd
//                iterations to a fixed point; every sum is taken in a fixed
//                order, so labels do not depend on scheduling; the restart
//                with the smallest cost wins (ties: the lowest index).
#include <algorithm>
#include <cstring>
#include <vector>

#include "dfc_lrr.h"
#include "alm_kernels.cuh"
#include "common.cuh"
#include "kernels.cuh"

namespace lrr {
namespace {

constexpr int KMAX = 64;          // largest number of clusters
constexpr int KNT = 1024;         // threads of a k-means CTA
constexpr int KW = KNT / 32;

inline unsigned gs(int64_t count) { return (unsigned)std::min<int64_t>((count + 255) / 256, 152 * 32); }

__device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
    x += 0x9E3779B97F4A7C15ull;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    return x ^ (x >> 31);
}

// |A|, row sums (A symmetric, column-major: column sums), one warp per column
__global__ void abs_colsum(float* __restrict__ A, int64_t n, double* __restrict__ d) {
    const int64_t j = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (j >= n) return;
    double acc = 0.0;
    for (int64_t i = lane; i < n; i += 32) {
        const float v = fabsf(A[i + j * n]);
        A[i + j * n] = v;
        acc += v;
    }
    acc = warp_sum(acc);
    if (lane == 0) d[j] = acc;
}

// A_ij <- (A_ij dinv_i dinv_j + delta_ij) / 2: the shifted normalised affinity
__global__ void normalise_shift(float* __restrict__ A, int64_t n, const double* __restrict__ d) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n * n; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e % n, j = e / n;
        const double di = d[i] > 0 ? 1.0 / sqrt(d[i]) : 0.0, dj = d[j] > 0 ? 1.0 / sqrt(d[j]) : 0.0;
        A[e] = (float)(0.5 * ((double)A[e] * di * dj + (i == j ? 1.0 : 0.0)));
    }
}

// Y <- Y R^-1 for the Cholesky factor R of G = Y^T Y (K x K, K <= KMAX), in
// float64 in one CTA; G is given (column-major, K x K).  A non-positive pivot
// (rank-deficient Y) leaves that column unscaled.
__global__ void chol_inv(const float* __restrict__ G, int K, float* __restrict__ Rinv) {
    __shared__ double L[KMAX][KMAX + 1];
    __shared__ double Li[KMAX][KMAX + 1];
    const int t = threadIdx.x;
    for (int e = t; e < K * K; e += blockDim.x) L[e % K][e / K] = (double)G[e];
    __syncthreads();
    if (t == 0) {
        // R^T R = G with R upper triangular, column by column
        for (int j = 0; j < K; ++j) {
            for (int i = 0; i < j; ++i) {
                double s = L[i][j];
                for (int q = 0; q < i; ++q) s -= L[q][i] * L[q][j];
                L[i][j] = s / L[i][i];
            }
            double s = L[j][j];
            for (int q = 0; q < j; ++q) s -= L[q][j] * L[q][j];
            L[j][j] = s > 0 ? sqrt(s) : 1.0;
        }
        // inverse of the upper-triangular R
        for (int j = 0; j < K; ++j) {
            for (int i = j + 1; i < K; ++i) Li[i][j] = 0.0;
            Li[j][j] = 1.0 / L[j][j];
            for (int i = j - 1; i >= 0; --i) {
                double s = 0.0;
                for (int q = i + 1; q <= j; ++q) s += L[i][q] * Li[q][j];
                Li[i][j] = -s / L[i][i];
            }
        }
    }
    __syncthreads();
    for (int e = t; e < K * K; e += blockDim.x) Rinv[e] = (float)Li[e % K][e / K];
}

// rows of Y (n x K) scaled to unit norm; one thread per row
__global__ void row_normalise(float* __restrict__ Y, int64_t n, int K) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    double s = 0.0;
    for (int c = 0; c < K; ++c) s += (double)Y[i + c * n] * Y[i + c * n];
    const double inv = s > 0 ? 1.0 / sqrt(s) : 1.0;
    for (int c = 0; c < K; ++c) Y[i + c * n] = (float)(Y[i + c * n] * inv);
}

// gathers the columns of X (rows x p) whose weight w > thr into Out (rows x q)
__global__ void gather_kept(const float* __restrict__ X, int64_t rows, const int* __restrict__ idx, int q,
                            float* __restrict__ Out) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < rows * q; e += (int64_t)gridDim.x * blockDim.x)
        Out[e] = X[e % rows + (int64_t)idx[e / rows] * rows];
}

// One k-means restart per CTA on the embedding Y (n x K, column-major): k-means++
// seeding, then Lloyd iterations until the labels stop changing (at most
// max_iter).  Writes labels (n per restart) and the final cost.  Every sum
// runs over the points in index order, so the result does not depend on
// scheduling.
__global__ void __launch_bounds__(KNT) kmeans_restart(const float* __restrict__ Y, int64_t n, int K, uint64_t seed,
                                                      int max_iter, int* __restrict__ labels_all,
                                                      float* __restrict__ d2_all, double* __restrict__ cost) {
    const int r = blockIdx.x;
    int* lab = labels_all + (int64_t)r * n;
    float* d2 = d2_all + (int64_t)r * n;
    __shared__ float C[KMAX][KMAX];
    __shared__ double red[KW];
    __shared__ int cnt[KMAX];
    __shared__ int pick;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int64_t per = (n + KW - 1) / KW;            // points of a warp, contiguous
    const int64_t p0 = warp * per, p1 = min((int64_t)n, p0 + per);
    auto dist2 = [&](int64_t p, int c) {
        float s = 0.f;
        for (int q = 0; q < K; ++q) {
            const float v = Y[p + q * n] - C[c][q];
            s = fmaf(v, v, s);
        }
        return s;
    };
    // ---- k-means++: the first center uniform, then with probability
    //      proportional to the squared distance to the nearest chosen center
    for (int c = 0; c < K; ++c) {
        if (c == 0) {
            if (t == 0) pick = (int)(splitmix64(seed ^ ((uint64_t)r << 32)) % (uint64_t)n);
        } else {
            double s = 0.0;
            for (int64_t p = p0 + lane; p < p1; p += 32) s += d2[p];
            s = warp_sum(s);
            if (lane == 0) red[warp] = s;
            __syncthreads();
            if (t == 0) {
                double tot = 0.0;
                for (int w = 0; w < KW; ++w) tot += red[w];
                const uint64_t h = splitmix64(seed ^ ((uint64_t)r << 32) ^ (uint64_t)c * 0x100000001B3ull);
                const double target = (double)(h >> 11) * (1.0 / 9007199254740992.0) * tot;
                double acc = 0.0;
                int w = 0;
                while (w < KW - 1 && acc + red[w] <= target) acc += red[w++];
                int chosen = (int)min((int64_t)w * per, n - 1);
                for (int64_t p = w * per, pe = min(n, (int64_t)(w + 1) * per); p < pe; ++p) {
                    acc += d2[p];
                    chosen = (int)p;
                    if (acc > target) break;
                }
                pick = chosen;
            }
        }
        __syncthreads();
        for (int q = t; q < K; q += KNT) C[c][q] = Y[pick + q * n];
        __syncthreads();
        for (int64_t p = t; p < n; p += KNT) {
            const float dd = dist2(p, c);
            d2[p] = c == 0 ? dd : fminf(d2[p], dd);
        }
        __syncthreads();
    }
    // ---- Lloyd iterations
    for (int it = 0; it < max_iter; ++it) {
        int changed = 0;
        for (int64_t p = t; p < n; p += KNT) {
            float best = 3.4e38f;
            int bi = 0;
            for (int c = 0; c < K; ++c) {
                const float dd = dist2(p, c);
                if (dd < best) { best = dd; bi = c; }
            }
            if (it == 0 || lab[p] != bi) changed = 1;
            lab[p] = bi;
        }
        if (__syncthreads_or(changed) == 0) break;
        // new centers: thread (c, q) sums dimension q over cluster c's points
        // in index order
        double sum = 0.0;
        int count = 0;
        const int c = t / K, q = t % K;
        if (t < K * K) {
            for (int64_t p = 0; p < n; ++p)
                if (lab[p] == c) { sum += Y[p + q * n]; ++count; }
            if (q == 0) cnt[c] = count;
        }
        __syncthreads();
        if (t < K * K && cnt[c] > 0) C[c][q] = (float)(sum / cnt[c]);
        __syncthreads();
    }
    // cost
    double s = 0.0;
    for (int64_t p = t; p < n; p += KNT) s += dist2(p, lab[p]);
    s = warp_sum(s);
    if (lane == 0) red[warp] = s;
    __syncthreads();
    if (t == 0) {
        double tot = 0.0;
        for (int w = 0; w < KW; ++w) tot += red[w];
        cost[r] = tot;
    }
}

// column 2-norms of X (rows x p), one warp per column
__global__ void col_norms(const float* __restrict__ X, int64_t rows, int p, double* __restrict__ out) {
    const int j = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (j >= p) return;
    double a = 0.0;
    for (int64_t i = lane; i < rows; i += 32) a += (double)X[i + j * rows] * X[i + j * rows];
    a = warp_sum(a);
    if (lane == 0) out[j] = sqrt(a);
}

#define STRY(x)                                   \
    do {                                          \
        cudaError_t _e = (x);                     \
        if (_e != cudaSuccess) return LRR_ERR_CUDA; \
    } while (0)

struct SegBuf {
    float *X, *W, *U, *Uk, *A, *Y, *Y2, *G, *Ri;
    double *d, *cost;
    float *sc, *of3, *d2;
    int *done, *on, *idx, *labels;
    OsjDesc<float>* od;
    GemmDesc<float>* gd;
};

size_t seg_layout(SegBuf& b, char* base, int64_t n, int k, int K, int restarts) {
    size_t off = 0;
    auto take = [&](size_t bytes) -> char* {
        off = (off + 255) / 256 * 256;
        char* p = base ? base + off : nullptr;
        off += std::max<size_t>(bytes, 1);
        return p;
    };
    const int pp = (k + 31) / 32 * 32;
    b.X = (float*)take(sizeof(float) * n * k);
    b.W = (float*)take(sizeof(float) * pp * pp);
    b.U = (float*)take(sizeof(float) * n * k);
    b.Uk = (float*)take(sizeof(float) * n * k);
    b.A = (float*)take(sizeof(float) * n * n);
    b.Y = (float*)take(sizeof(float) * n * K);
    b.Y2 = (float*)take(sizeof(float) * n * K);
    b.G = (float*)take(sizeof(float) * K * K);
    b.Ri = (float*)take(sizeof(float) * K * K);
    b.d = (double*)take(sizeof(double) * std::max<int64_t>(n, k));
    b.cost = (double*)take(sizeof(double) * restarts);
    b.sc = (float*)take(sizeof(float));
    b.of3 = (float*)take(sizeof(float) * 3);
    b.d2 = (float*)take(sizeof(float) * n * restarts);
    b.done = (int*)take(sizeof(int));
    b.on = (int*)take(sizeof(int));
    b.idx = (int*)take(sizeof(int) * k);
    b.labels = (int*)take(sizeof(int) * n * restarts);
    b.od = (OsjDesc<float>*)take(sizeof(OsjDesc<float>));
    b.gd = (GemmDesc<float>*)take(sizeof(GemmDesc<float>) * 16);
    return off + 256;
}

int gemm1(SegBuf& b, int slot, bool ta, bool tb, int M, int N, int K, const float* A, int64_t lda, const float* B,
          int64_t ldb, float* C, int64_t ldc, cudaStream_t s) {
    GemmDesc<float> d{};
    d.A = A; d.B = B; d.C = C; d.lda = lda; d.ldb = ldb; d.ldc = ldc; d.m = M; d.n = N; d.k = K;
    d.alpha = 1.f; d.beta = 0.f;
    STRY(cudaMemcpyAsync(b.gd + slot, &d, sizeof(d), cudaMemcpyHostToDevice, s));
    STRY(gemm_grouped<float>(b.gd + slot, 1, ta, tb, M, N, s));
    return LRR_OK;
}

}  // namespace
}  // namespace lrr

extern "C" {

size_t lrr_segment_workspace_bytes(int64_t n, int64_t k, int32_t clusters, int32_t restarts) {
    if (n < 2 || k < 1 || k > n || clusters < 1 || clusters > lrr::KMAX || clusters > n || restarts < 1) return 0;
    lrr::SegBuf b{};
    return lrr::seg_layout(b, nullptr, n, (int)k, clusters, restarts);
}

int lrr_segment(const float* F, int64_t ldf, const float* G, int64_t ldg, int64_t n, int64_t k, int32_t clusters,
                double rel_tol, uint64_t seed, int32_t restarts, int32_t power_iters, int32_t* labels, void* workspace,
                size_t workspace_bytes, void* stream) {
    using namespace lrr;
    if (!F || !G || !labels || n < 2 || k < 1 || k > n || ldf < n || ldg < k || clusters < 1 ||
        clusters > KMAX || clusters > n || restarts < 1 || restarts > 1024 || power_iters < 1 || !(rel_tol >= 0) ||
        n > 46340)
        return LRR_ERR_INVALID;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int K = clusters, kk = (int)k;
    SegBuf b{};
    const size_t need = seg_layout(b, nullptr, n, kk, K, restarts);
    void* own = nullptr;
    if (!workspace) {
        if (cudaMallocAsync(&own, need, s) != cudaSuccess) return LRR_ERR_CUDA;
        workspace = own;
        workspace_bytes = need;
    }
    struct Free {
        void* p; cudaStream_t s;
        ~Free() { if (p) cudaFreeAsync(p, s); }
    } guard{own, s};
    if (workspace_bytes < need - 256 || reinterpret_cast<uintptr_t>(workspace) % 256) return LRR_ERR_WORKSPACE;
    seg_layout(b, static_cast<char*>(workspace), n, kk, K, restarts);
    const int pp = (kk + 31) / 32 * 32;
    // ---- left singular vectors: X = G^T W (n x k), W = I, one-sided Jacobi
    k::init_padded<float><<<gs((int64_t)pp * pp), 256, 0, s>>>(b.W, kk, pp, 1.f, 1);
    k::gather_cols<float, float><<<dim3(gs(k), (unsigned)std::min<int64_t>(n, 65535)), 256, 0, s>>>(G, ldg, nullptr, k,
                                                                                                   n, b.U);
    // b.U holds G (k x n, ld k); X = G^T
    {
        const int r = gemm1(b, 0, true, false, (int)n, kk, kk, b.U, k, b.W, pp, b.X, n, s);
        if (r != LRR_OK) return r;
    }
    OsjDesc<float> od{};
    const int one = 1;
    od.X = b.X; od.W = b.W; od.done = b.done; od.off = b.of3; od.active = b.on; od.scale = b.sc; od.mu = nullptr;
    od.ldx = n; od.ldw = pp; od.L = (int)n; od.p = kk; od.pp = pp; od.strict = 1;
    STRY(cudaMemcpyAsync(b.od, &od, sizeof(od), cudaMemcpyHostToDevice, s));
    STRY(cudaMemcpyAsync(b.on, &one, sizeof(int), cudaMemcpyHostToDevice, s));
    k::col_norm_max<float><<<1, 256, 0, s>>>(b.od, b.on, b.sc, 1);
    STRY(osj_sweeps<float>(b.od, 1, pp, 40, 2e-6f, nullptr, s, 0));
    // kept directions: singular values s_j = ||x_j|| above rel_tol * max
    col_norms<<<(unsigned)(((int64_t)kk * 32 + 255) / 256), 256, 0, s>>>(b.X, n, kk, b.d);
    std::vector<double> sv((size_t)kk, 0.0);
    STRY(cudaMemcpyAsync(sv.data(), b.d, sizeof(double) * kk, cudaMemcpyDeviceToHost, s));
    STRY(cudaStreamSynchronize(s));
    const double smax = *std::max_element(sv.begin(), sv.end());
    std::vector<int> idx;
    for (int j = 0; j < kk; ++j)
        if (sv[j] > rel_tol * smax && sv[j] > 0) idx.push_back(j);
    const int q = (int)idx.size();
    if (q == 0) return LRR_ERR_RANK;
    STRY(cudaMemcpyAsync(b.idx, idx.data(), sizeof(int) * q, cudaMemcpyHostToDevice, s));
    // U = F W (n x k), then the kept columns
    {
        const int r = gemm1(b, 1, false, false, (int)n, kk, kk, F, ldf, b.W, pp, b.U, n, s);
        if (r != LRR_OK) return r;
    }
    gather_kept<<<gs(n * q), 256, 0, s>>>(b.U, n, b.idx, q, b.Uk);
    // ---- affinity and its normalisation
    {
        const int r = gemm1(b, 2, false, true, (int)n, (int)n, q, b.Uk, n, b.Uk, n, b.A, n, s);
        if (r != LRR_OK) return r;
    }
    abs_colsum<<<(unsigned)((n * 32 + 255) / 256), 256, 0, s>>>(b.A, n, b.d);
    normalise_shift<<<gs(n * n), 256, 0, s>>>(b.A, n, b.d);
    // ---- subspace iteration for the K leading eigenvectors
    k::fill_hash<float><<<gs(n * K), 256, 0, s>>>(b.Y, n * K, (uint32_t)(seed * 2654435761u + 7u));
    for (int it = 0; it < power_iters; ++it) {
        int r = gemm1(b, 3, false, false, (int)n, K, (int)n, b.A, n, b.Y, n, b.Y2, n, s);
        if (r != LRR_OK) return r;
        r = gemm1(b, 4, true, false, K, K, (int)n, b.Y2, n, b.Y2, n, b.G, K, s);
        if (r != LRR_OK) return r;
        chol_inv<<<1, 256, 0, s>>>(b.G, K, b.Ri);
        r = gemm1(b, 5, false, false, (int)n, K, K, b.Y2, n, b.Ri, K, b.Y, n, s);
        if (r != LRR_OK) return r;
    }
    // (the basis of the leading eigenspace is used as it is: the rows' mutual
    // distances, and so k-means, do not change under an orthogonal rotation
    // of the embedding's columns)
    row_normalise<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(b.Y, n, K);
    // ---- k-means, one CTA per restart
    kmeans_restart<<<restarts, KNT, 0, s>>>(b.Y, n, K, seed, 300, b.labels, b.d2, b.cost);
    STRY(cudaGetLastError());
    std::vector<double> cost((size_t)restarts);
    STRY(cudaMemcpyAsync(cost.data(), b.cost, sizeof(double) * restarts, cudaMemcpyDeviceToHost, s));
    STRY(cudaStreamSynchronize(s));
    int best = 0;
    for (int r = 1; r < restarts; ++r)
        if (cost[r] < cost[best] - 1e-12) best = r;
    STRY(cudaMemcpyAsync(labels, b.labels + (int64_t)best * n, sizeof(int) * n, cudaMemcpyDeviceToHost, s));
    STRY(cudaStreamSynchronize(s));
    return LRR_OK;
}

}  // extern "C"
