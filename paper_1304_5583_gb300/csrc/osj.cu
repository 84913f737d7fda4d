// Batched one-sided block-Jacobi SVD for the singular-value thresholding step.
//
// For every block the L x p matrix X (X = A W for a tall A, X = A^T W for a
// wide one, W the previous iteration's right basis) is driven to orthogonal
// columns by rotations X <- X R, W <- W R.  In each round the p/b column
// blocks are paired round-robin and one CTA per pair
//   1. forms the 2b x 2b Gram S = X_P^T X_P afresh from the columns of X
//      (so each entry carries only the rounding of its own two columns),
//   2. diagonalises S in shared memory (inner cyclic Jacobi),
//   3. applies the accumulated rotation to X_P and W_P in row chunks.
// Pairs of a round touch disjoint columns, so one launch per round suffices.
// A matrix is converged once a whole sweep saw every pivot Gram with
// max |s_ij| / sqrt(s_ii s_jj) <= tol; then the squared column norms of X are
// the eigenvalues of the Gram A^T A (or A A^T) and W holds its eigenvectors.
#include <type_traits>

#include "common.cuh"
#include "inner_jacobi.cuh"
#include "kernels.cuh"

namespace lrr {
namespace {

constexpr int NT = 256;
// pivot Gram chunk sums accumulated in float64 (measured: no accuracy gain over
// float32 once the block rotations are re-orthonormalised, so off)
constexpr bool kGramF64 = false;

__device__ __forceinline__ int pcol(int i, int a, int c, int b) { return i < b ? a * b + i : c * b + (i - b); }

// 16-byte vector of TI = 16 / sizeof(T) elements (float4 / double2)
template <typename T> struct Vec16;
template <> struct Vec16<float> { using type = float4; };
template <> struct Vec16<double> { using type = double2; };

__device__ __forceinline__ void unpack(const float4& v, float (&x)[4]) { x[0] = v.x; x[1] = v.y; x[2] = v.z; x[3] = v.w; }
__device__ __forceinline__ void unpack(const double2& v, double (&x)[2]) { x[0] = v.x; x[1] = v.y; }

// Copies rows r0 .. r0+B2-1 of the pivot columns of a column-major matrix into
// a B2 x LD row-major shared tile (zero outside); consecutive threads read
// consecutive rows of a column.
template <typename T, int B2, int LD>
__device__ __forceinline__ void load_chunk(T* tile, const T* __restrict__ base, int64_t ld, int rows, int ncol, int r0,
                                           int a, int c, int b) {
    for (int e = threadIdx.x; e < B2 * B2; e += NT) {
        const int rr = e % B2, cc = e / B2;
        const int gr = r0 + rr, gc = pcol(cc, a, c, b);
        tile[rr * LD + cc] = (gr < rows && gc < ncol) ? base[gr + (int64_t)gc * ld] : T(0);
    }
}

template <typename T, int B2>
__global__ void __launch_bounds__(NT) osj_round(const OsjDesc<T>* __restrict__ descs, int round) {
    constexpr int b = B2 / 2;
    constexpr int TI = B2 / 16;        // each thread owns a TI x TI tile of the B2 x B2 products
    constexpr int LD = B2 + 4;         // padded row stride of the shared tiles (16-byte rows)
    using V = typename Vec16<T>::type;
    static_assert(sizeof(V) == TI * sizeof(T), "tile width must match the 16-byte vector");
    const OsjDesc<T> d = descs[blockIdx.y];
    if (d.active && *d.active == 0) return;
    if (*d.done) return;
    const int nb = d.pp / b, npairs = nb / 2;
    const int P = blockIdx.x;
    if (P >= npairs) return;
    const int a = circle_item(P, round, nb), c = circle_item(nb - 1 - P, round, nb);

    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* const X0 = reinterpret_cast<T*>(smem_raw);   // one B2 x LD chunk tile
    auto Xb = [&](int) { return X0; };
    // S and R use an odd row stride (conflict-free for the inner Jacobi's
    // scattered row/column pairs); after the rotation is final it is copied
    // into R4 (stride LD, 16-byte rows, over S's space) for vector reads
    constexpr int LO = B2 + 1;
    T(*S)[LO] = reinterpret_cast<T(*)[LO]>(X0 + B2 * LD);
    T(*R4)[LD] = reinterpret_cast<T(*)[LD]>(X0 + B2 * LD);
    T(*R)[LO] = reinterpret_cast<T(*)[LO]>(X0 + 2 * B2 * LD);
    __shared__ T cs[b], sn[b];
    __shared__ int pi[b], qi[b];
    __shared__ T red[NT / 32];
    const int t = threadIdx.x;
    const int ti = t % 16, tj = t / 16;     // tile coordinates: rows ti*TI.., cols tj*TI..
    // columns whose norm is below ~4 eps times the largest column are rounding
    // noise of earlier rotations: their mutual angles carry no information
    const T noise = T(4) * num<T>::eps();
    const T floor2 = noise * noise * (*d.scale) + num<T>::tiny();

    // 1. pivot Gram S = X_P^T X_P from the columns of X, in B2-row chunks
    //    (next chunk in flight while the current one is multiplied)
    using Acc = typename std::conditional<kGramF64, double, T>::type;
    Acc acc[TI][TI];
#pragma unroll
    for (int u = 0; u < TI; ++u)
#pragma unroll
        for (int v = 0; v < TI; ++v) acc[u][v] = Acc(0);
    const int nchunk = (d.L + B2 - 1) / B2;
    for (int ch = 0; ch < nchunk; ++ch) {
        load_chunk<T, B2, LD>(Xb(ch), d.X, d.ldx, d.L, d.p, ch * B2, a, c, b);
        __syncthreads();
        const T* Xs = Xb(ch);
        T part[TI][TI];
#pragma unroll
        for (int u = 0; u < TI; ++u)
#pragma unroll
            for (int v = 0; v < TI; ++v) part[u][v] = T(0);
#pragma unroll 4
        for (int rr = 0; rr < B2; ++rr) {
            T xi[TI], xj[TI];
            unpack(*reinterpret_cast<const V*>(Xs + rr * LD + ti * TI), xi);
            unpack(*reinterpret_cast<const V*>(Xs + rr * LD + tj * TI), xj);
#pragma unroll
            for (int u = 0; u < TI; ++u)
#pragma unroll
                for (int v = 0; v < TI; ++v) part[u][v] = fma(xi[u], xj[v], part[u][v]);
        }
#pragma unroll
        for (int u = 0; u < TI; ++u)
#pragma unroll
            for (int v = 0; v < TI; ++v) acc[u][v] += (Acc)part[u][v];
        __syncthreads();
    }
#pragma unroll
    for (int u = 0; u < TI; ++u)
#pragma unroll
        for (int v = 0; v < TI; ++v) {
            const int i = ti * TI + u, j = tj * TI + v;
            S[i][j] = (T)acc[u][v];
            R[i][j] = (i == j) ? T(1) : T(0);
        }
    __syncthreads();

    // 2. convergence measure before rotating: how much the rotation this pair
    //    still needs could change J = U max(Sigma - tau, 0) V^T, relative to
    //    the largest singular value.  For columns of norms a, b, an unresolved
    //    rotation of tangent t moves J by about t |f(a) - f(b)| (f(s) =
    //    max(s - tau, 0) is 1-Lipschitz, so |a - b| bounds it), plus tau theta
    //    when both lie above tau (the pair then enters J as A - tau U V^T and
    //    theta = |s_ij| / (a b) is its angle defect).  Pairs whose norms
    //    satisfy a^2 + b^2 <= tau^2 have every singular value below tau and
    //    are removed by the SVT whatever their rotation; noise columns (below
    //    the rounding floor) are skipped.  A `strict` matrix (the block whose
    //    kept left singular subspace the C step projects onto) also needs that
    //    subspace itself: pairs straddling tau are measured by t alone.
    const T tau = d.mu ? (T)(1.0 / *d.mu) : T(0);
    const T tau2 = tau * tau;
    const T inv_smax = T(1) / (sqrt(*d.scale) + num<T>::tiny());
    T offm = T(0);
    for (int e = t; e < B2 * B2; e += NT) {
        const int i = e % B2, j = e / B2;
        const T sii = S[i][i], sjj = S[j][j];
        if (i < j && sii > floor2 && sjj > floor2 && sii + sjj > tau2) {
            const T sij = fabs(S[i][j]);
            const T a = sqrt(sii), bb = sqrt(sjj);
            const T hd = T(0.5) * fabs(sii - sjj);
            const T tn = sij / (hd + sqrt(hd * hd + sij * sij) + num<T>::tiny());
            T mm;
            if (a > tau && bb > tau) mm = tn * fabs(a - bb) + tau * sij / (a * bb);
            else if (a > tau || bb > tau) mm = d.strict ? tn * (*d.scale > 0 ? sqrt(*d.scale) : T(1)) : tn * fabs(a - bb);
            else mm = tn * (sqrt(sii + sjj) - tau);
            offm = fmax(offm, mm * inv_smax);
        }
    }
    offm = warp_max(offm);
    if ((t & 31) == 0) red[t >> 5] = offm;
    __syncthreads();
    T mx = T(0);
    for (int w = 0; w < NT / 32; ++w) mx = fmax(mx, red[w]);
    if (t == 0) atomic_max_nonneg(d.off, mx);
    // a pivot already orthogonal to a few eps needs no rotation.  The measure
    // is relative to the largest column, so on data with one dominant
    // singular value (nonnegative data) a pair can sit below a loose skip
    // threshold while its rotation still matters relative to the rest of J:
    // in float32 the threshold is 4 eps (16 eps cost a 5x larger error in Z on
    // face-like data, and 1-2 eps gain nothing more)
    if (mx <= (sizeof(T) == 4 ? T(4) : T(16)) * num<T>::eps()) return;

    // 3. rotate the pivot Gram to diagonal form; rotations that only mix noise
    //    columns (|s_pq| below floor2) do not keep the inner sweeps going, and
    //    in float32 neither do rotations with tan < 3e-4: after such a sweep
    //    the remaining off-diagonal part is second order in those angles,
    //    below the sweep tolerance (this drops the confirming inner sweep)
    const int rot = inner_jacobi<T, B2, NT, LO>(S, R, cs, sn, pi, qi, num<T>::tiny(), floor2, 4,
                                                sizeof(T) == 4 ? T(3e-4) : T(0));
    if (!rot) return;

    // R is a product of some thousand plane rotations, orthogonal only to
    // ~sqrt(count) eps.  Applied to graded columns that defect would mix
    // eps-sized parts of the large columns into the small ones and cap the
    // attainable orthogonality, so one Newton-Schulz step R <- R (3I - R^T R)/2
    // restores orthogonality to ~eps^2 before R touches X and W.
    {
        T g[TI][TI];
#pragma unroll
        for (int u = 0; u < TI; ++u)
#pragma unroll
            for (int v = 0; v < TI; ++v) g[u][v] = T(0);
        for (int k = 0; k < B2; ++k) {
            T ri[TI], rj[TI];
#pragma unroll
            for (int u = 0; u < TI; ++u) { ri[u] = R[k][ti * TI + u]; rj[u] = R[k][tj * TI + u]; }
#pragma unroll
            for (int u = 0; u < TI; ++u)
#pragma unroll
                for (int v = 0; v < TI; ++v) g[u][v] = fma(ri[u], rj[v], g[u][v]);
        }
        // the first chunk buffer (free here) holds R^T R
        T* Xs = Xb(0);
#pragma unroll
        for (int u = 0; u < TI; ++u)
#pragma unroll
            for (int v = 0; v < TI; ++v) Xs[(ti * TI + u) * LD + tj * TI + v] = g[u][v];
        __syncthreads();
        T y[TI][TI];
#pragma unroll
        for (int u = 0; u < TI; ++u)
#pragma unroll
            for (int v = 0; v < TI; ++v) y[u][v] = T(0);
        for (int k = 0; k < B2; ++k) {
            T ri[TI], gk[TI];
#pragma unroll
            for (int u = 0; u < TI; ++u) { ri[u] = R[ti + 16 * u][k]; gk[u] = Xs[k * LD + tj * TI + u]; }
#pragma unroll
            for (int u = 0; u < TI; ++u)
#pragma unroll
                for (int v = 0; v < TI; ++v) y[u][v] = fma(ri[u], gk[v], y[u][v]);
        }
        __syncthreads();
#pragma unroll
        for (int u = 0; u < TI; ++u)
#pragma unroll
            for (int v = 0; v < TI; ++v) {
                const int i = ti + 16 * u, j = tj * TI + v;
                R[i][j] = T(1.5) * R[i][j] - T(0.5) * y[u][v];
            }
        __syncthreads();
    }

    // the rotation is applied in update form, x_j <- x_j + sum_k x_k (R - I)_kj:
    // once the sweeps have converged R - I is tiny and so is the rounding it
    // adds, instead of a fresh eps |x| at every application
    for (int e = t; e < B2 * B2; e += NT) {
        const int i = e / B2, j = e % B2;
        R4[i][j] = R[i][j] - (i == j ? T(1) : T(0));
    }
    __syncthreads();

    // 4. X_P <- X_P R and W_P <- W_P R, row chunk by row chunk (double-buffered)
    for (int pass = 0; pass < 2; ++pass) {
        T* base = pass == 0 ? d.X : d.W;
        const int64_t ld = pass == 0 ? d.ldx : d.ldw;
        const int rows = pass == 0 ? d.L : d.p;
        const int nch = (rows + B2 - 1) / B2;
        for (int ch = 0; ch < nch; ++ch) {
            load_chunk<T, B2, LO>(Xb(ch), base, ld, rows, d.p, ch * B2, a, c, b);
            __syncthreads();
            const T* Xs = Xb(ch);
            const int r0 = ch * B2;
            T out[TI][TI];
#pragma unroll
            for (int u = 0; u < TI; ++u)
#pragma unroll
                for (int v = 0; v < TI; ++v) out[u][v] = T(0);
#pragma unroll 4
            for (int k = 0; k < B2; ++k) {
                T xr[TI];
#pragma unroll
                for (int u = 0; u < TI; ++u) xr[u] = Xs[(ti + 16 * u) * LO + k];
                T rk[TI];
                unpack(*reinterpret_cast<const V*>(&R4[k][tj * TI]), rk);
#pragma unroll
                for (int u = 0; u < TI; ++u)
#pragma unroll
                    for (int v = 0; v < TI; ++v) out[u][v] = fma(xr[u], rk[v], out[u][v]);
            }
#pragma unroll
            for (int u = 0; u < TI; ++u)
#pragma unroll
                for (int v = 0; v < TI; ++v) {
                    const int gr = r0 + ti + 16 * u, gc = pcol(tj * TI + v, a, c, b);
                    if (gr < rows && gc < d.p)
                        base[gr + (int64_t)gc * ld] = Xs[(ti + 16 * u) * LO + tj * TI + v] + out[u][v];
                }
            __syncthreads();
        }
    }
}

template <typename T>
__global__ void osj_reset(const OsjDesc<T>* __restrict__ descs, int nmat) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nmat) return;
    *descs[i].done = 0;
    *descs[i].off = T(0);
}

template <typename T>
__global__ void osj_check(const OsjDesc<T>* __restrict__ descs, int nmat, T tol, int* __restrict__ sweeps_run) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nmat) return;
    const OsjDesc<T> d = descs[i];
    if (d.active && *d.active == 0) return;
    if (*d.done == 0) {
        if (sweeps_run) sweeps_run[i] += 1;
        // scaled off-diagonals below ~64 eps are at the rounding level of the
        // fresh pivot Grams
        const T t_eff = fmax(tol, T(64) * num<T>::eps());
        if (*d.off <= t_eff) *d.done = 1;
    }
    *d.off = T(0);
}

}  // namespace

template <typename T>
cudaError_t osj_sweeps(const OsjDesc<T>* d_desc, int nmat, int max_pp, int sweeps, T tol, int* sweeps_run,
                       cudaStream_t s) {
    constexpr int b = jacobi_bs<T>();
    constexpr int B2 = 2 * b;
    if (nmat <= 0 || max_pp <= 0) return cudaSuccess;
    const int nb = max_pp / b, npairs = nb / 2;
    const size_t smem = sizeof(T) * (2 * B2 * (B2 + 4) + B2 * (B2 + 1));
    static std::atomic<uint64_t> smem_set{0};
    const cudaError_t ea = ensure_smem_limit(osj_round<T, B2>, (int)smem, smem_set);
    if (ea != cudaSuccess) return ea;
    osj_reset<T><<<ceil_div(nmat, 128), 128, 0, s>>>(d_desc, nmat);
    const dim3 g((unsigned)npairs, (unsigned)nmat);
    for (int sw = 0; sw < sweeps; ++sw) {
        for (int r = 0; r < nb - 1; ++r) osj_round<T, B2><<<g, NT, smem, s>>>(d_desc, r);
        osj_check<T><<<ceil_div(nmat, 128), 128, 0, s>>>(d_desc, nmat, tol, sweeps_run);
    }
    return cudaGetLastError();
}

template cudaError_t osj_sweeps<float>(const OsjDesc<float>*, int, int, int, float, int*, cudaStream_t);
template cudaError_t osj_sweeps<double>(const OsjDesc<double>*, int, int, int, double, int*, cudaStream_t);

}  // namespace lrr
