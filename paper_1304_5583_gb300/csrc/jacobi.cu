// Batched block-Jacobi eigensolver for symmetric matrices (float32 / float64).
//
// The SVT of every ALM iteration needs the eigendecomposition of a Gram
// matrix, and the one-time factor needs that of M M^T.  Cyclic block Jacobi
// keeps the work in dense 2b x 2b tiles: in every round the diagonal blocks
// are paired round-robin, each CTA diagonalises one 2b x 2b pivot submatrix
// in shared memory (inner cyclic Jacobi with the classical rotation angle),
// and a second kernel applies the accumulated rotations R_P to the
// off-diagonal tiles (G <- R^T G R) and to the eigenvector matrix (W <- W R).
#include "common.cuh"
#include "inner_jacobi.cuh"
#include "kernels.cuh"

namespace lrr {
namespace {

constexpr int NT = 256;


// global row of local index i (0..2b-1) of the pivot pair (a, c)
__device__ __forceinline__ int pair_row(int i, int a, int c, int b) { return i < b ? a * b + i : c * b + (i - b); }

template <typename T, int B2>
__global__ void __launch_bounds__(NT) jac_solve(const JacDesc<T>* __restrict__ descs, int round, T tol) {
    constexpr int b = B2 / 2;
    const JacDesc<T> d = descs[blockIdx.y];
    if (d.active && *d.active == 0) return;
    if (*d.done) return;
    const int nb = d.pp / b, npairs = nb / 2;
    const int P = blockIdx.x;
    if (P >= npairs) return;
    const int a = circle_item(P, round, nb), c = circle_item(nb - 1 - P, round, nb);

    __shared__ T S[B2][B2 + 1];
    __shared__ T R[B2][B2 + 1];
    __shared__ T cs[b], sn[b];
    __shared__ int pi[b], qi[b];
    __shared__ T red[NT / 32];
    const int t = threadIdx.x;
    // Off-diagonal entries below the rounding noise of the Gram products
    // (~sqrt(order) * eps * max|G_ii|) carry no information and do not count
    // towards the convergence measure; they are still rotated away like any
    // other entry above eps * sqrt(G_ii G_jj), so a converged sweep leaves the
    // resolved part of the spectrum at working accuracy.
    const T floor_abs = T(4) * sqrt(T(d.pp)) * num<T>::eps() * (*d.scale) + num<T>::tiny();
    const T floor_rot = num<T>::eps() * num<T>::eps() * (*d.scale) + num<T>::tiny();

    for (int e = t; e < B2 * B2; e += NT) {
        const int i = e % B2, j = e / B2;
        S[i][j] = d.G[pair_row(i, a, c, b) + (int64_t)pair_row(j, a, c, b) * d.pp];
        R[i][j] = (i == j) ? T(1) : T(0);
    }
    __syncthreads();

    // convergence measure of this pivot block before rotating it, and whether
    // any entry is large enough to rotate at all
    T offm = T(0);
    int any = 0;
    for (int e = t; e < B2 * B2; e += NT) {
        const int i = e % B2, j = e / B2;
        if (i < j) {
            const T v = fabs(S[i][j]);
            const T sc = sqrt(fabs(S[i][i] * S[j][j]));
            if (v > floor_abs) offm = fmax(offm, v / (sc + num<T>::tiny()));
            if (v > floor_rot && v > num<T>::eps() * sc) any = 1;
        }
    }
    offm = warp_max(offm);
    if ((t & 31) == 0) red[t >> 5] = offm;
    __syncthreads();
    if (t == 0) {
        T mx = T(0);
        for (int w = 0; w < NT / 32; ++w) mx = fmax(mx, red[w]);
        atomic_max_nonneg(d.off, mx);
    }
    const bool need = __syncthreads_or(any) != 0;

    // float32 (the start of the setup's eigendecomposition): one inner sweep
    // per pivot, the outer sweeps continue from there; float64: up to six
    const int any_rot =
        need ? inner_jacobi<T, B2, NT>(S, R, cs, sn, pi, qi, floor_rot, floor_abs, sizeof(T) == 4 ? 1 : 6) : 0;
    // diagonalised pivot block back into G, rotation out for the apply kernel
    if (t == 0) d.rot[P] = any_rot;
    if (any_rot) {
        T* Rg = d.R + (int64_t)P * B2 * B2;
        for (int e = t; e < B2 * B2; e += NT) {
            const int i = e % B2, j = e / B2;
            d.G[pair_row(i, a, c, b) + (int64_t)pair_row(j, a, c, b) * d.pp] = S[i][j];
            Rg[e] = R[i][j];
        }
    }
}

template <typename T, int B2>
__global__ void __launch_bounds__(NT) jac_apply(const JacDesc<T>* __restrict__ descs, int round) {
    constexpr int b = B2 / 2;
    const JacDesc<T> d = descs[blockIdx.y];
    if (d.active && *d.active == 0) return;
    if (*d.done) return;
    const int nb = d.pp / b, npairs = nb / 2;
    const int ntile_g = npairs * (npairs - 1) / 2;
    int tile = blockIdx.x;
    if (tile >= ntile_g + npairs * npairs) return;

    __shared__ T X[B2][B2 + 1];
    __shared__ T Q[B2][B2 + 1];
    const int t = threadIdx.x;
    // each thread owns 16 (B2=64) or 4 (B2=32) output entries: rows i0 + 16*ii, cols tj
    constexpr int PER = B2 * B2 / NT;

    if (tile < ntile_g) {
        // off-diagonal tile (P, Q), P < Q:  G[I_P, I_Q] <- R_P^T G[I_P, I_Q] R_Q
        int P = 0, rem = tile;
        while (rem >= npairs - 1 - P) { rem -= npairs - 1 - P; ++P; }
        const int Qp = P + 1 + rem;
        const int rP = d.rot[P], rQ = d.rot[Qp];
        if (!rP && !rQ) return;
        const int a = circle_item(P, round, nb), c = circle_item(nb - 1 - P, round, nb);
        const int a2 = circle_item(Qp, round, nb), c2 = circle_item(nb - 1 - Qp, round, nb);
        const T* RP = d.R + (int64_t)P * B2 * B2;
        const T* RQ = d.R + (int64_t)Qp * B2 * B2;
        for (int e = t; e < B2 * B2; e += NT) {
            const int i = e % B2, j = e / B2;
            X[i][j] = d.G[pair_row(i, a, c, b) + (int64_t)pair_row(j, a2, c2, b) * d.pp];
            Q[i][j] = rQ ? RQ[e] : (i == j ? T(1) : T(0));
        }
        __syncthreads();
        T acc[PER];
#pragma unroll
        for (int u = 0; u < PER; ++u) {
            const int e = t + u * NT, i = e % B2, j = e / B2;
            T s = T(0);
#pragma unroll 8
            for (int k = 0; k < B2; ++k) s = fma(X[i][k], Q[k][j], s);
            acc[u] = s;
        }
        __syncthreads();
#pragma unroll
        for (int u = 0; u < PER; ++u) {
            const int e = t + u * NT, i = e % B2, j = e / B2;
            X[i][j] = acc[u];
            Q[i][j] = rP ? RP[e] : (i == j ? T(1) : T(0));
        }
        __syncthreads();
#pragma unroll
        for (int u = 0; u < PER; ++u) {
            const int e = t + u * NT, i = e % B2, j = e / B2;
            T s = T(0);
#pragma unroll 8
            for (int k = 0; k < B2; ++k) s = fma(Q[k][i], X[k][j], s);
            const int gi = pair_row(i, a, c, b), gj = pair_row(j, a2, c2, b);
            d.G[gi + (int64_t)gj * d.pp] = s;
            d.G[gj + (int64_t)gi * d.pp] = s;
        }
    } else {
        // eigenvector tile: rows chunk ch, columns I_P:  W[ch, I_P] <- W[ch, I_P] R_P
        tile -= ntile_g;
        const int P = tile % npairs, ch = tile / npairs;
        if (!d.rot[P]) return;
        const int a = circle_item(P, round, nb), c = circle_item(nb - 1 - P, round, nb);
        const T* RP = d.R + (int64_t)P * B2 * B2;
        for (int e = t; e < B2 * B2; e += NT) {
            const int i = e % B2, j = e / B2;
            X[i][j] = d.W[(ch * B2 + i) + (int64_t)pair_row(j, a, c, b) * d.pp];
            Q[i][j] = RP[e];
        }
        __syncthreads();
#pragma unroll
        for (int u = 0; u < PER; ++u) {
            const int e = t + u * NT, i = e % B2, j = e / B2;
            T s = T(0);
#pragma unroll 8
            for (int k = 0; k < B2; ++k) s = fma(X[i][k], Q[k][j], s);
            d.W[(ch * B2 + i) + (int64_t)pair_row(j, a, c, b) * d.pp] = s;
        }
    }
}

template <typename T>
__global__ void jac_reset(const JacDesc<T>* __restrict__ descs, int nmat) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nmat) return;
    *descs[i].done = 0;
    *descs[i].off = T(0);
}

template <typename T>
__global__ void jac_check(const JacDesc<T>* __restrict__ descs, int nmat, T tol) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nmat) return;
    const JacDesc<T> d = descs[i];
    if (*d.done == 0 && *d.off <= tol) *d.done = 1;
    *d.off = T(0);
}

}  // namespace

template <typename T>
cudaError_t jacobi_sweeps(const JacDesc<T>* d_desc, int nmat, int max_pp, int sweeps, T tol, cudaStream_t s,
                         const int* done_dev, int* sweeps_run) {
    constexpr int b = jacobi_bs<T>();
    constexpr int B2 = 2 * b;
    if (sweeps_run) *sweeps_run = 0;
    if (nmat <= 0 || max_pp <= 0) return cudaSuccess;
    const int nb = max_pp / b, npairs = nb / 2;
    jac_reset<T><<<ceil_div(nmat, 128), 128, 0, s>>>(d_desc, nmat);
    const dim3 gs((unsigned)npairs, (unsigned)nmat);
    const dim3 ga((unsigned)(npairs * (npairs - 1) / 2 + npairs * npairs), (unsigned)nmat);
    for (int sw = 0; sw < sweeps; ++sw) {
        for (int r = 0; r < nb - 1; ++r) {
            jac_solve<T, B2><<<gs, NT, 0, s>>>(d_desc, r, tol);
            jac_apply<T, B2><<<ga, NT, 0, s>>>(d_desc, r);
        }
        jac_check<T><<<ceil_div(nmat, 128), 128, 0, s>>>(d_desc, nmat, tol);
        if (sweeps_run) *sweeps_run = sw + 1;
        if (done_dev) {
            // one matrix: stop launching once it has converged
            int done = 0;
            cudaError_t e = cudaMemcpyAsync(&done, done_dev, sizeof(int), cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
            if (e != cudaSuccess) return e;
            if (done) break;
        }
    }
    return cudaGetLastError();
}

template cudaError_t jacobi_sweeps<float>(const JacDesc<float>*, int, int, int, float, cudaStream_t, const int*,
                                          int*);
template cudaError_t jacobi_sweeps<double>(const JacDesc<double>*, int, int, int, double, cudaStream_t, const int*,
                                           int*);

}  // namespace lrr
