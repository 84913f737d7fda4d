// Element-wise and per-block kernels of the inexact ALM iteration (reduced
// coordinates).  Included by solver.cu only.
//
// Reduced coordinates: with M = U diag(sigma) V^T (compact, rank r) every ALM
// iterate starting from zero keeps its columns in range(M^T) = range(V)
// (the SVT, (I + M^T M)^{-1} and the dual steps all map range(V) into
// itself), so Z = V Zt, J = V Jt, Y2 = V Y2t with r x l blocks Zt, Jt, Y2t:
//   SVT:      Jt = SVT_{1/mu}(Zt + Y2t/mu)         (SVT commutes with V)
//   Z-step:   Zt = (sigma (U^T P) + Jt - Y2t/mu) / (1 + sigma^2),  P = C - E + Y1/mu
//   M Z   =   U diag(sigma) Zt
// E, Y1 and the residual C - M Z - E stay in the m-dimensional data space.
#pragma once
#include <cuda_bf16.h>

#include "common.cuh"
#include "kernels.cuh"

namespace lrr {
namespace k {

template <typename T, typename Tin>
__global__ void gather_cols(const Tin* __restrict__ M, int64_t ldm, const int64_t* __restrict__ perm, int64_t m,
                            int64_t n, T* __restrict__ C) {
    for (int64_t j = blockIdx.y; j < n; j += gridDim.y) {
        const Tin* src = M + (perm ? perm[j] : j) * ldm;
        T* dst = C + j * m;
        for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x)
            dst[i] = (T)src[i];
    }
}

template <typename Tin>
__global__ void nonfinite_check(const Tin* __restrict__ M, int64_t ldm, int64_t m, int64_t n, int* flag) {
    for (int64_t j = blockIdx.y; j < n; j += gridDim.y)
        for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
            const Tin v = M[i + j * ldm];
            if (!isfinite(v)) *flag = 1;
        }
}

template <typename T>
__global__ void fill(T* __restrict__ x, int64_t count, T v) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x)
        x[i] = v;
}

template <typename T>
__global__ void copy_convert_f64(const double* __restrict__ src, T* __restrict__ dst, int64_t count) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = (T)src[i];
}

template <typename T>
__global__ void copy_convert_to_f64(const T* __restrict__ src, double* __restrict__ dst, int64_t count) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = (double)src[i];
}

// x[i] = a uniform value in [-0.5, 0.5) from a hash of i (synthetic input for
// timing launch shapes; its statistics do not matter)
template <typename T>
__global__ void fill_hash(T* __restrict__ x, int64_t count, uint32_t seed) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
        uint32_t h = (uint32_t)i * 0x9E3779B1u ^ seed;
        h ^= h >> 16; h *= 0x85EBCA6Bu; h ^= h >> 13; h *= 0xC2B2AE35u; h ^= h >> 16;
        x[i] = (T)((double)h * (1.0 / 4294967296.0) - 0.5);
    }
}

// split of x for the bf16x3 product: hi = x rounded to the nearest bf16,
// lo = (x - hi) rounded to the nearest bf16 (x - hi is exact in float32)
__device__ __forceinline__ void split_bf16(float x, uint16_t& hi, uint16_t& lo) {
    const __nv_bfloat16 h = __float2bfloat16(x);
    hi = __bfloat16_as_ushort(h);
    lo = __bfloat16_as_ushort(__float2bfloat16(x - __bfloat162float(h)));
}

// bf16 bit patterns of the same hashed values
static __global__ void fill_hash_bf16(uint16_t* __restrict__ x, int64_t count, uint32_t seed) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
        uint32_t h = (uint32_t)i * 0x9E3779B1u ^ seed;
        h ^= h >> 16; h *= 0x85EBCA6Bu; h ^= h >> 13; h *= 0xC2B2AE35u; h ^= h >> 16;
        x[i] = __bfloat16_as_ushort(__float2bfloat16((float)((double)h * (1.0 / 4294967296.0) - 0.5)));
    }
}

// square pp x pp matrix, ld pp: real part p x p is left alone; padding gets
// `diag` on the diagonal and zeros elsewhere.  With eye != 0 the real part is
// set to the identity too (eigenvector matrices).
template <typename T>
__global__ void init_padded(T* __restrict__ G, int p, int pp, T diag, int eye) {
    const int64_t count = (int64_t)pp * pp;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < count; e += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(e % pp), j = (int)(e / pp);
        if (i < p && j < p) {
            if (eye) G[e] = (i == j) ? T(1) : T(0);
        } else {
            G[e] = (i == j) ? diag : T(0);
        }
    }
}

// Per-block SVT gate: ||A||_F^2 <= tau^2 means every singular value of A is
// <= tau, so the threshold removes all of them and J = 0 with no SVD.
// The Z-step kernel of the same iteration then accumulates the next value.
template <typename T>
__global__ void svt_gate(const int* __restrict__ act, double* __restrict__ afro, const double* __restrict__ mu,
                         int* __restrict__ svt_on, T* __restrict__ scale, int* __restrict__ calls,
                         int* __restrict__ fp32_on, int* __restrict__ gemm32, double margin, int nblk) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nblk) return;
    const double tau = 1.0 / mu[b];
    svt_on[b] = (act[b] && afro[b] > tau * tau) ? 1 : 0;
    if (svt_on[b]) calls[b] += 1;
    // mixed precision: float32 products from the first iteration in which
    // ||A||_F exceeds margin * tau (sticky); before that J = 0 and the bf16
    // rounding of the products is forgotten by the iteration
    if (afro[b] > margin * margin * tau * tau) fp32_on[b] = 1;
    gemm32[b] = (act[b] && fp32_on[b]) ? 1 : 0;
    if (act[b]) {
        scale[b] = (T)afro[b];
        afro[b] = 0.0;
    }
}

// Largest squared column norm of X (the Jacobi noise scale): one CTA per block.
template <typename T>
__global__ void col_norm_max(const OsjDesc<T>* __restrict__ descs, const int* __restrict__ on, T* __restrict__ scale,
                             int nblk) {
    const int b = blockIdx.x;
    if (b >= nblk || !on[b]) return;
    const OsjDesc<T> d = descs[b];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    T mx = T(0);
    for (int j = warp; j < d.p; j += nw) {
        const T* x = d.X + (int64_t)j * d.ldx;
        T acc = T(0);
        for (int i = lane; i < d.L; i += 32) acc += x[i] * x[i];
        mx = fmax(mx, warp_sum(acc));
    }
    __shared__ T s_m[32];
    if (lane == 0) s_m[warp] = mx;
    __syncthreads();
    if (threadIdx.x == 0) {
        T m2 = T(0);
        for (int w = 0; w < nw; ++w) m2 = fmax(m2, s_m[w]);
        scale[b] = m2;
    }
}

// After the one-sided Jacobi the columns x_j of X are orthogonal and
// ||x_j||^2 are the eigenvalues lambda_j of the Gram; the singular values of A
// are sqrt(lambda_j).  h_j = max(1 - tau/||x_j||, 0), so that
// J = X diag(h) W^T (tall) or W diag(h) X^T (wide) = U max(Sigma - tau, 0) V^T.
// Also counts the SVT rank.  One CTA per block.
template <typename T>
__global__ void svt_weights(const OsjDesc<T>* __restrict__ descs, T* const* __restrict__ h,
                            const int* __restrict__ act, const int* __restrict__ svt_on,
                            const double* __restrict__ mu, int* __restrict__ rank, int nblk) {
    const int b = blockIdx.x;
    if (b >= nblk || !act[b]) return;
    const OsjDesc<T> d = descs[b];
    T* hb = h[b];
    const double tau = 1.0 / mu[b];
    const T tau_t = (T)tau;
    const int on = svt_on[b];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    int cnt = 0;
    for (int j = warp; j < d.pp; j += nw) {
        T w = T(0);
        if (on && j < d.p) {
            const T* x = d.X + (int64_t)j * d.ldx;
            T acc = T(0);
            for (int i = lane; i < d.L; i += 32) acc += x[i] * x[i];
            const T nrm = sqrt(warp_sum(acc));
            if (nrm > tau_t) w = T(1) - tau_t / nrm;
        }
        if (lane == 0) {
            hb[j] = w;
            if (w > T(0)) ++cnt;
        }
    }
    __shared__ int s_c[32];
    if (lane == 0) s_c[warp] = cnt;
    __syncthreads();
    if (threadIdx.x == 0) {
        int a2 = 0;
        for (int w2 = 0; w2 < nw; ++w2) a2 += s_c[w2];
        rank[b] = a2;
    }
}

// Z-step in reduced coordinates, fused with the Y2 dual step and the next
// SVT input; one warp per column.  With T = U^T (Y1/mu - E) on entry:
//   Zt = (sigma (Theta + T) + Jt - Y2t/mu) / (1 + sigma^2)
//   T <- Delta = Theta - sigma Zt   (so that C - M Z = C_perp + U Delta)
template <typename T>
__global__ void z_update(int r, int64_t n, const int* __restrict__ colblk, const int* __restrict__ act,
                         const double* __restrict__ mu, double rho, double mu_max, T* __restrict__ Tt,
                         const T* __restrict__ Theta, const T* __restrict__ Jt, T* __restrict__ Y2t,
                         T* __restrict__ Zt, T* __restrict__ D, T* __restrict__ A, const T* __restrict__ sig,
                         const T* __restrict__ dinv, T* __restrict__ dmax, double* __restrict__ afro,
                         uint16_t* __restrict__ dbf, uint16_t* __restrict__ dbf_lo, int64_t ldd,
                         float* __restrict__ dhi, float* __restrict__ dlo, int64_t lds) {
    const int64_t j = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (j >= n) return;
    const int b = colblk[j];
    if (!act[b]) return;
    const double mud = mu[b];
    const double mun = fmin(rho * mud, mu_max);
    const T imu = (T)(1.0 / mud), muT = (T)mud, imun = (T)(1.0 / mun);
    const int64_t o = j * r;
    T acc = T(0), aacc = T(0);
    for (int i = lane; i < r; i += 32) {
        const T th = Theta[o + i], jv = Jt[o + i], y2 = Y2t[o + i];
        const T z = dinv[i] * (sig[i] * (th + Tt[o + i]) + jv - y2 * imu);
        const T dl = th - sig[i] * z;
        const T dd = z - jv;
        const T y2n = y2 + muT * dd;
        const T av = z + y2n * imun;
        Zt[o + i] = z;
        Tt[o + i] = dl;
        if (dbf) split_bf16((float)dl, dbf[i + j * ldd], dbf_lo[i + j * ldd]);
        if (dhi) split_tf32((float)dl, dhi[i + j * lds], dlo[i + j * lds]);
        D[o + i] = dd;
        Y2t[o + i] = y2n;
        A[o + i] = av;
        acc += dd * dd;
        aacc += av * av;
    }
    acc = warp_sum(acc);
    aacc = warp_sum(aacc);
    if (lane == 0) {
        atomic_max_nonneg(&dmax[b], sqrt(acc));
        atomicAdd(&afro[b], (double)aacc);   // ||A||_F^2 of the next SVT input
    }
}

// E-step (column shrinkage), primal residual, Y1 dual step and the next
// Z-step right-hand side Q = Y1/mu' - E; one warp per column.  The residual
// C - M Z arrives as C_perp + U Delta (Cp may be null when C_perp = 0).
template <typename T>
__global__ void e_update(int64_t m, int64_t n, const int* __restrict__ colblk, const int* __restrict__ act,
                         const double* __restrict__ mu, double rho, double mu_max, double lam,
                         const T* __restrict__ Cp, const T* __restrict__ UD, T* __restrict__ Y1, T* __restrict__ E,
                         T* __restrict__ Q, T* __restrict__ r1max, uint16_t* __restrict__ qbf,
                         uint16_t* __restrict__ qbf_lo, int64_t ldq, float* __restrict__ qhi,
                         float* __restrict__ qlo, int64_t lds) {
    const int64_t j = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (j >= n) return;
    const int b = colblk[j];
    if (!act[b]) return;
    const double mud = mu[b];
    const double mun = fmin(rho * mud, mu_max);
    const T imu = (T)(1.0 / mud), muT = (T)mud, imun = (T)(1.0 / mun);
    const T thr = (T)(lam / mud);
    const int64_t o = j * m;
    T acc = T(0);
    for (int64_t i = lane; i < m; i += 32) {
        const T res = (Cp ? Cp[o + i] : T(0)) + UD[o + i];
        const T x = res + Y1[o + i] * imu;
        acc += x * x;
    }
    const T nrm = sqrt(warp_sum(acc));
    const T sc = nrm > thr ? T(1) - thr / nrm : T(0);
    T amax = T(0);
    for (int64_t i = lane; i < m; i += 32) {
        const T res = (Cp ? Cp[o + i] : T(0)) + UD[o + i];
        const T y1 = Y1[o + i];
        const T x = res + y1 * imu;
        const T e = sc * x;
        const T l1 = res - e;
        const T y1n = y1 + muT * l1;
        E[o + i] = e;
        Y1[o + i] = y1n;
        const T qv = y1n * imun - e;
        Q[o + i] = qv;
        if (qbf) split_bf16((float)qv, qbf[i + j * ldq], qbf_lo[i + j * ldq]);
        if (qhi) split_tf32((float)qv, qhi[i + j * lds], qlo[i + j * lds]);
        amax = fmax(amax, fabs(l1));
    }
    amax = warp_max(amax);
    if (lane == 0) atomic_max_nonneg(&r1max[b], amax);
}

// Stop test, part 1: ||C - M Z - E||_inf < eps is necessary.  ||Z - J||_inf =
// max |V D| <= nu * max_j ||D_j|| (nu = largest row norm of V) decides
// convergence when that bound is already below eps; otherwise the exact value
// is needed (a product with V).
// ||V d||_inf >= ||V d||_2 / sqrt(n) = ||d||_2 / sqrt(n) (V has orthonormal
// columns), so max_j ||D_j|| / sqrt(n) >= eps already rules convergence out.
template <typename T>
__global__ void stop_part1(int nblk, const int* __restrict__ act, const T* __restrict__ r1, const T* __restrict__ dmax,
                           T nu, double inv_sqrt_n, double eps, int* __restrict__ need_exact,
                           int* __restrict__ conv_bound, int* __restrict__ any_need, int* __restrict__ need_cnt) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nblk) return;
    int ne = 0, cb = 0;
    if (act[b] && (double)r1[b] < eps && (double)dmax[b] * inv_sqrt_n < eps) {
        if ((double)(nu * dmax[b]) < eps) cb = 1; else ne = 1;
    }
    need_exact[b] = ne;
    conv_bound[b] = cb;
    if (ne && any_need) *any_need = 1;
    if (ne && need_cnt) atomicAdd(need_cnt, 1);
}

// bf16 copy (K-major, leading dimension ldo) of the columns of D = Zt - Jt
// whose block still needs the value of ||V D||_inf
template <typename T>
__global__ void d_to_bf16_needed(const T* __restrict__ D, int64_t ld, int r, int64_t n, const int* __restrict__ colblk,
                                 const int* __restrict__ need, const int* __restrict__ any_need,
                                 uint16_t* __restrict__ dst, int64_t ldo) {
    if (*any_need == 0) return;
    for (int64_t j = blockIdx.y; j < n; j += gridDim.y) {
        if (!need[colblk[j]]) continue;
        for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < r; i += gridDim.x * blockDim.x)
            dst[i + j * ldo] = __bfloat16_as_ushort(__float2bfloat16((float)D[i + j * ld]));
    }
}

// Stop test, tensor-core stage.  bmax[b] = max |V D| over block b computed from
// bf16-rounded V and D.  Rounding each operand to bf16 (unit roundoff u = 2^-8)
// changes every product by at most (2u + u^2) |v_jk d_k|, and float32
// accumulation over K terms adds at most ~K 2^-24 sum |v_jk d_k|; with
// sum_k |v_jk d_k| <= ||v_j|| ||d|| <= nu max_j ||D_j|| the bf16 maximum is
// within err = rel * nu * dmax of the exact one (rel carries a factor-2
// margin).  Where that settles the comparison with eps the block needs no
// float32 product: converged (bound below eps) or not (value above eps).
template <typename T>
__global__ void stop_tc_decide(int nblk, int* __restrict__ need_exact, int* __restrict__ conv_bound,
                               const unsigned* __restrict__ bmax, const T* __restrict__ dmax, T nu, double eps,
                               double rel, int* __restrict__ tc_dec, T* __restrict__ r2x) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nblk || !need_exact[b]) return;
    const double mh = (double)__uint_as_float(bmax[b]);
    const double e = rel * (double)nu * (double)dmax[b];
    if (mh + e < eps) {
        conv_bound[b] = 1;
        need_exact[b] = 0;
        tc_dec[b] = 1;
        r2x[b] = (T)(mh + e);
    } else if (mh - e >= eps) {
        need_exact[b] = 0;
        tc_dec[b] = 1;
        r2x[b] = (T)mh;
    }
}

template <typename T>
__global__ void stop_part2(int nblk, int* __restrict__ act, int* __restrict__ iters, double* __restrict__ mu,
                           double rho, double mu_max, double eps, int max_iter, T* __restrict__ r1,
                           T* __restrict__ dmax, T* __restrict__ r2x, const int* __restrict__ need_exact,
                           const int* __restrict__ conv_bound, T nu, double* __restrict__ resid,
                           const int* __restrict__ rank_cur, int* __restrict__ rank_fin, int* __restrict__ conv,
                           double* __restrict__ mu_fin, double* __restrict__ afro, int* __restrict__ tc_dec,
                           unsigned* __restrict__ bmax, int* __restrict__ any_need) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nblk) return;
    if (act[b]) {
        const int it = ++iters[b];
        const bool ok = conv_bound[b] || (need_exact[b] && (double)r2x[b] < eps);
        const bool have = need_exact[b] || (tc_dec && tc_dec[b]);
        const double rz = have ? (double)r2x[b] : (double)(nu * dmax[b]);
        resid[2 * b] = (double)r1[b];
        resid[2 * b + 1] = rz;
        rank_fin[b] = rank_cur[b];
        mu_fin[b] = mu[b];
        if (ok || it >= max_iter) {
            act[b] = 0;
            conv[b] = ok ? 1 : 0;
        } else {
            mu[b] = fmin(rho * mu[b], mu_max);
        }
    }
    r1[b] = T(0);
    dmax[b] = T(0);
    r2x[b] = T(0);
    if (tc_dec) tc_dec[b] = 0;
    if (bmax) bmax[b] = 0u;
    if (any_need && b == 0) *any_need = 0;
}

// one-time factor M M^T = W diag(lam) W^T (columns of W in `order`, the r
// kept ones): U (float64), U diag(1/sigma) (for V = M^T U diag(1/sigma))
static __global__ void setup_factors(const double* __restrict__ W, int64_t ldw, int64_t m, int r,
                              const int* __restrict__ order, const double* __restrict__ lam, double* __restrict__ Ud,
                              double* __restrict__ Usd) {
    const int k = blockIdx.y;
    if (k >= r) return;
    const int src = order[k];
    const double s = sqrt(fmax(lam[k], 0.0));
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
        const double u = W[i + (int64_t)src * ldw];
        Ud[i + k * m] = u;
        Usd[i + k * m] = u / s;
    }
}

// bf16 copy of a column-major rows x cols matrix, same orientation, leading
// dimension ldo (padding rows untouched): the K-major operand layout when the
// contraction runs over the rows
template <typename T>
__global__ void to_bf16_km(const T* __restrict__ src, int64_t ld, int64_t rows, int64_t cols,
                           uint16_t* __restrict__ dst, int64_t ldo) {
    for (int64_t j = blockIdx.y; j < cols; j += gridDim.y)
        for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < rows; i += (int64_t)gridDim.x * blockDim.x)
            dst[i + j * ldo] = __bfloat16_as_ushort(__float2bfloat16((float)src[i + j * ld]));
}

// bf16 transpose of a column-major rows x cols matrix: dst[j + i * ldo] = src(i, j)
// (the K-major operand layout when the contraction runs over the columns)
template <typename T>
__global__ void to_bf16_transposed(const T* __restrict__ src, int64_t ld, int64_t rows, int64_t cols,
                                   uint16_t* __restrict__ dst, int64_t ldo) {
    for (int64_t i = blockIdx.y; i < rows; i += gridDim.y)
        for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < cols; j += (int64_t)gridDim.x * blockDim.x)
            dst[j + i * ldo] = __bfloat16_as_ushort(__float2bfloat16((float)src[i + j * ld]));
}

// split bf16 copies (hi, lo) of a column-major rows x cols matrix, same
// orientation (as to_bf16_km)
template <typename T>
__global__ void to_bf16_split_km(const T* __restrict__ src, int64_t ld, int64_t rows, int64_t cols,
                                 uint16_t* __restrict__ hi, uint16_t* __restrict__ lo, int64_t ldo) {
    for (int64_t j = blockIdx.y; j < cols; j += gridDim.y)
        for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < rows; i += (int64_t)gridDim.x * blockDim.x)
            split_bf16((float)src[i + j * ld], hi[i + j * ldo], lo[i + j * ldo]);
}

// split bf16 copies of the transpose (as to_bf16_transposed)
template <typename T>
__global__ void to_bf16_split_transposed(const T* __restrict__ src, int64_t ld, int64_t rows, int64_t cols,
                                         uint16_t* __restrict__ hi, uint16_t* __restrict__ lo, int64_t ldo) {
    for (int64_t i = blockIdx.y; i < rows; i += gridDim.y)
        for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < cols; j += (int64_t)gridDim.x * blockDim.x)
            split_bf16((float)src[i + j * ld], hi[j + i * ldo], lo[j + i * ldo]);
}

// split TF32 copy of a column-major rows x cols float32 matrix (same
// orientation, leading dimension ldo, padding rows zero): hi + lo = src with
// hi exact in TF32 (operands of tc_gemm_3xtf32)
template <typename T>
__global__ void split_tf32_km(const T* __restrict__ src, int64_t ld, int64_t rows, int64_t cols,
                              float* __restrict__ hi, float* __restrict__ lo, int64_t ldo) {
    for (int64_t j = blockIdx.y; j < cols; j += gridDim.y)
        for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < ldo; i += (int64_t)gridDim.x * blockDim.x) {
            float h = 0.f, l = 0.f;
            if (i < rows) split_tf32((float)src[i + j * ld], h, l);
            hi[i + j * ldo] = h;
            lo[i + j * ldo] = l;
        }
}

// the same for the transpose: dst(j, i) = src(i, j), dst with leading
// dimension ldo >= cols (padding zero)
template <typename T>
__global__ void split_tf32_transposed(const T* __restrict__ src, int64_t ld, int64_t rows, int64_t cols,
                                      float* __restrict__ hi, float* __restrict__ lo, int64_t ldo) {
    for (int64_t i = blockIdx.y; i < rows; i += gridDim.y)
        for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < ldo; j += (int64_t)gridDim.x * blockDim.x) {
            float h = 0.f, l = 0.f;
            if (j < cols) split_tf32((float)src[i + j * ld], h, l);
            hi[j + i * ldo] = h;
            lo[j + i * ldo] = l;
        }
}

// Theta(k, j) = sigma_k V(perm_j, k) in the iteration precision and in float64
template <typename T>
__global__ void theta_from_v(const double* __restrict__ Vd, int64_t n, const double* __restrict__ lam,
                             const int64_t* __restrict__ perm, int r, T* __restrict__ Th, double* __restrict__ Thd) {
    const int k = blockIdx.y;
    if (k >= r) return;
    const double s = sqrt(fmax(lam[k], 0.0));
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
        const double v = s * Vd[perm[j] + (int64_t)k * n];
        Th[k + j * r] = (T)v;
        Thd[k + j * r] = v;
    }
}

template <typename T>
__global__ void diag_of(const T* __restrict__ G, int64_t ld, int64_t count, double* __restrict__ out) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < count) out[i] = (double)G[i + i * ld];
}

// sigma, 1/(1+sigma^2), U and U diag(sigma) in the iteration's precision
template <typename T>
__global__ void setup_scalars(const double* __restrict__ lam, int r, const double* __restrict__ Ud, int64_t m,
                              T* __restrict__ sig, T* __restrict__ dinv, T* __restrict__ U, T* __restrict__ US) {
    const int k = blockIdx.y;
    if (k >= r) return;
    const double s = sqrt(fmax(lam[k], 0.0));
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        sig[k] = (T)s;
        dinv[k] = (T)(1.0 / (1.0 + s * s));
    }
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
        const double u = Ud[i + k * m];
        U[i + k * m] = (T)u;
        US[i + k * m] = (T)(u * s);
    }
}

// largest row 2-norm of V (n x r): nu in the bound |v_i . d| <= ||v_i|| ||d||
template <typename T>
__global__ void row_norm_max(const T* __restrict__ V, int64_t n, int r, T* __restrict__ out) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    double acc = 0.0;
    for (int k = 0; k < r; ++k) {
        const double v = (double)V[i + k * n];
        acc += v * v;
    }
    atomic_max_nonneg(out, (T)(sqrt(acc) * (1.0 + 1e-6)));
}

// dst[:, perm[j]] = src[:, j] for the m x n column-major src (ld lds) and dst (ld ldd)
template <typename T>
__global__ void scatter_cols(const T* __restrict__ src, int64_t m, int64_t n, const int64_t* __restrict__ perm,
                             T* __restrict__ dst, int64_t lds, int64_t ldd) {
    for (int64_t j = blockIdx.y; j < n; j += gridDim.y)
        for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x)
            dst[i + perm[j] * ldd] = src[i + j * lds];
}

// C-step helpers -----------------------------------------------------------
// keep-list of the kept SVT directions (h > 0) of block 0
template <typename T>
__global__ void kept_columns(const T* __restrict__ h, int p, int* __restrict__ idx, int* __restrict__ count) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    int c = 0;
    for (int i = 0; i < p; ++i)
        if (h[i] > T(0)) idx[c++] = i;
    *count = c;
}

// F64 copy of selected columns of a (rows x ?) matrix, normalised to unit norm
template <typename T>
__global__ void gather_normalise_f64(const T* __restrict__ src, int64_t ld, int64_t rows, const int* __restrict__ idx,
                                     const int* __restrict__ count, double* __restrict__ dst) {
    const int k = blockIdx.x;
    if (k >= *count) return;
    const T* s = src + (int64_t)idx[k] * ld;
    double acc = 0.0;
    for (int64_t i = threadIdx.x; i < rows; i += blockDim.x) {
        const double v = (double)s[i];
        acc += v * v;
    }
    __shared__ double red[32];
    acc = warp_sum(acc);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        double v = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
        v = warp_sum(v);
        if (threadIdx.x == 0) red[0] = v;
    }
    __syncthreads();
    const double inv = red[0] > 0.0 ? 1.0 / sqrt(red[0]) : 0.0;
    for (int64_t i = threadIdx.x; i < rows; i += blockDim.x) dst[i + (int64_t)k * rows] = (double)s[i] * inv;
}

// X <- 1.5 X - 0.5 Y  (Newton-Schulz step for the polar factor, Y = X X^T X)
static __global__ void ns_combine(double* __restrict__ X, const double* __restrict__ Y, int64_t count) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x)
        X[i] = 1.5 * X[i] - 0.5 * Y[i];
}

// Given Y = W (W^T W): Wi <- 2 W - Y (= W (2I - W^T W), the first-order
// inverse transpose W^{-T}) and W <- 1.5 W - 0.5 Y (one Newton-Schulz step
// towards orthogonality).  Rotations accumulated in float32 drift from
// orthogonal by ~eps per round; with Wi in the SVT reconstruction the drift
// enters J only at second order, and the Newton-Schulz step keeps the warm
// start of the next iteration orthogonal.
template <typename T>
__global__ void ns_orth(T* const* __restrict__ W, T* const* __restrict__ Y, T* const* __restrict__ Wi,
                        const int* __restrict__ p, const int* __restrict__ pp, const int* __restrict__ on, int nblk) {
    const int b = blockIdx.y;
    if (b >= nblk || !on[b]) return;
    const int n = p[b], ld = pp[b];
    T* w = W[b];
    T* wi = Wi[b];
    const T* y = Y[b];
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)n * n;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(e % n), j = (int)(e / n);
        const int64_t o = i + (int64_t)j * ld;
        const T wv = w[o], yv = y[o];
        wi[o] = T(2) * wv - yv;
        w[o] = T(1.5) * wv - T(0.5) * yv;
    }
}

}  // namespace k
}  // namespace lrr
