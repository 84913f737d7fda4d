// K unrolled inexact-ALM iterations of plain LRR (eq. (1), the observations
// are the dictionary, C = M) and their reverse-mode derivative: the map
// (M, lambda) -> Z_K and the pull-back of dL/dZ_K to dL/dM and dL/dlambda.
//
// Forward iteration (the iteration of the solver, from the zero start, the
// K-th one without its dual step), in the n-dimensional space of Z:
//   A  = Z + Y2/mu,            J = SVT_{1/mu}(A)
//   R  = M^T (C - E + Y1/mu) + J - Y2/mu,   Z' = (I + M^T M)^{-1} R
//   E' = shrink(C - M Z' + Y1/mu, lambda/mu)
//   Y1' = Y1 + mu (C - M Z' - E'),  Y2' = Y2 + mu (Z' - J)
// (I + M^T M)^{-1} R = R - M^T Wm diag(1/(1+l)) Wm^T M R with M M^T = Wm diag(l) Wm^T
// (float64 eigendecomposition, once).  A stays in range(M^T) = range(V), V
// the right singular vectors of M, so its SVD is that of the r x n matrix
// V^T A, computed by the batched one-sided Jacobi warm-started from the
// previous iteration's basis.
//
// Backward (derived from the steps above; mu is a fixed schedule): see the
// comments of backward_step.  The SVT derivative uses the singular triplets
// of A = U diag(s) Vr^T (U = V W, Vr = X diag(1/s)):
//   Abar = U (core - P F - F P) Vr^T + (Jbar Vr) F Vr^T + U F (U^T Jbar)
//   P = U^T Jbar Vr,  F = diag(f(s)/s),  f(s) = max(s - tau, 0),
//   core = diag(f'(s_i) P_ii) + G+ o sym(P) + G- o skew(P) off the diagonal,
//   G+_ij = (f_i - f_j)/(s_i - s_j),  G-_ij = (f_i + f_j)/(s_i + s_j).
// The states (Z, E, Y1, Y2 and the Jacobi warm start) are kept every
// `checkpoint` iterations; the backward pass recomputes each segment from its
// checkpoint and then reverses it.
#include <algorithm>
#include <cstring>
#include <numeric>
#include <vector>

#include "dfc_lrr.h"
#include "alm_kernels.cuh"
#include "common.cuh"
#include "kernels.cuh"

namespace lrr {
namespace {

constexpr size_t kAl = 256;

struct Bump {
    char* base;
    size_t off = 0;
    explicit Bump(void* b) : base(static_cast<char*>(b)) {}
    template <typename X>
    X* take(size_t count) {
        off = (off + kAl - 1) / kAl * kAl;
        X* p = base ? reinterpret_cast<X*>(base + off) : nullptr;
        off += std::max<size_t>(count, 1) * sizeof(X);
        return p;
    }
};

inline unsigned g1(int64_t count) { return (unsigned)std::min<int64_t>((count + 255) / 256, 152 * 32); }
inline int rup(int x, int q) { return (x + q - 1) / q * q; }

// ------------------------------------------------------------------ kernels
namespace u {

// y = a x + b y  (element-wise, count entries)
template <typename T>
__global__ void axpby(int64_t count, T a, const T* __restrict__ x, T b, T* __restrict__ y) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x)
        y[i] = a * x[i] + b * y[i];
}
// z = a x + b y
template <typename T>
__global__ void lincomb(int64_t count, T a, const T* __restrict__ x, T b, const T* __restrict__ y, T* __restrict__ z) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x)
        z[i] = a * x[i] + b * y[i];
}
// z = x + a y + b w
template <typename T>
__global__ void lincomb3(int64_t count, const T* __restrict__ x, T a, const T* __restrict__ y, T b,
                         const T* __restrict__ w, T* __restrict__ z) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x)
        z[i] = x[i] + a * y[i] + b * w[i];
}
// rows of X (rows x cols, ld rows) scaled by d[row]
template <typename T>
__global__ void scale_rows(T* __restrict__ X, int64_t rows, int64_t cols, const T* __restrict__ d) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < rows * cols; e += (int64_t)gridDim.x * blockDim.x)
        X[e] *= d[e % rows];
}
// out(:, j) = X(:, j) * d[j]  (rows x cols, ld rows)
template <typename T>
__global__ void scale_cols(const T* __restrict__ X, int64_t rows, int64_t cols, const T* __restrict__ d,
                           T* __restrict__ out) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < rows * cols; e += (int64_t)gridDim.x * blockDim.x)
        out[e] = X[e] * d[e / rows];
}

// Column shrinkage E = shrink(X, theta), X = C - MZ + Y1/mu formed here and
// kept (one warp per column); also the primal part of the dual step when
// `dual`: Y1 <- Y1 + mu (C - MZ - E).
template <typename T>
__global__ void shrink_fwd(int64_t m, int64_t n, const T* __restrict__ C, int64_t ldc, const T* __restrict__ MZ,
                           T* __restrict__ Y1, T* __restrict__ E, T* __restrict__ X, T mu, T theta, int dual) {
    const int64_t j = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (j >= n) return;
    const T imu = T(1) / mu;
    T acc = T(0);
    for (int64_t i = lane; i < m; i += 32) {
        const T x = C[i + j * ldc] - MZ[i + j * m] + Y1[i + j * m] * imu;
        X[i + j * m] = x;
        acc += x * x;
    }
    const T nrm = sqrt(warp_sum(acc));
    const T sc = nrm > theta ? T(1) - theta / nrm : T(0);
    for (int64_t i = lane; i < m; i += 32) {
        const T e = sc * X[i + j * m];
        E[i + j * m] = e;
        if (dual) Y1[i + j * m] += mu * (C[i + j * ldc] - MZ[i + j * m] - e);
    }
}

// Adjoint of the column shrinkage: Xbar = (1 - theta/r) ebar + theta (x.ebar) x / r^3
// on columns with r = ||x|| > theta (zero elsewhere); dtheta += -(x.ebar)/r.
template <typename T>
__global__ void shrink_adj(int64_t m, int64_t n, const T* __restrict__ X, const T* __restrict__ Eb,
                           T* __restrict__ Xb, T theta, double dscale, double* __restrict__ dtheta) {
    const int64_t j = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (j >= n) return;
    T xx = T(0), xe = T(0);
    for (int64_t i = lane; i < m; i += 32) {
        const T x = X[i + j * m], e = Eb[i + j * m];
        xx += x * x;
        xe += x * e;
    }
    xx = warp_sum(xx);
    xe = warp_sum(xe);
    const T r = sqrt(xx);
    const bool act = r > theta;
    const T a = act ? T(1) - theta / r : T(0), b = act ? theta * xe / (r * r * r) : T(0);
    for (int64_t i = lane; i < m; i += 32) Xb[i + j * m] = a * Eb[i + j * m] + b * X[i + j * m];
    if (lane == 0 && act) atomicAdd(dtheta, -dscale * (double)(xe / r));
}

// SVT weights from the orthogonalised columns of X (n x p): s_i = ||x_i||,
// h_i = f(s_i)/s_i (the reconstruction weight), fs = f/s, inv_s = 1/s (0 for
// a zero column); one warp per column.
template <typename T>
__global__ void svt_svals(const T* __restrict__ X, int64_t ld, int64_t L, int p, T tau, T* __restrict__ s,
                          T* __restrict__ fs, T* __restrict__ inv_s, int* __restrict__ rank) {
    const int j = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (j >= p) return;
    T acc = T(0);
    for (int64_t i = lane; i < L; i += 32) acc += X[i + j * ld] * X[i + j * ld];
    const T nrm = sqrt(warp_sum(acc));
    if (lane == 0) {
        s[j] = nrm;
        fs[j] = nrm > tau ? T(1) - tau / nrm : T(0);
        inv_s[j] = nrm > T(0) ? T(1) / nrm : T(0);
        if (nrm > tau) atomicAdd(rank, 1);
    }
}

// F_i = f(s_i)/s_i (0 for a zero singular value)
template <typename T>
__global__ void f_over_s(const T* __restrict__ s, int p, T tau, T* __restrict__ F) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < p) F[i] = (s[i] > tau && s[i] > T(0)) ? (s[i] - tau) / s[i] : T(0);
}

// C2 = core(P) - P F - F P for the SVT adjoint (p x p, ld p); F = diag(f/s)
template <typename T>
__global__ void svt_core(const T* __restrict__ P, int p, const T* __restrict__ s, T tau, T* __restrict__ C2) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < p * p; e += gridDim.x * blockDim.x) {
        const int i = e % p, j = e / p;
        const T si = s[i], sj = s[j];
        const T fi = si > tau ? si - tau : T(0), fj = sj > tau ? sj - tau : T(0);
        const T Fi = si > T(0) ? fi / si : T(0), Fj = sj > T(0) ? fj / sj : T(0);
        const T pij = P[i + j * p], pji = P[j + i * p];
        T core;
        if (i == j) {
            core = (si > tau ? T(1) : T(0)) * pij;
        } else {
            const T gp = si != sj ? (fi - fj) / (si - sj) : (si > tau ? T(1) : T(0));
            const T gm = si + sj > T(0) ? (fi + fj) / (si + sj) : T(0);
            core = gp * T(0.5) * (pij + pji) + gm * T(0.5) * (pij - pji);
        }
        C2[e] = core - pij * Fj - Fi * pij;
    }
}

}  // namespace u

// ------------------------------------------------------------------ engine
template <typename T>
struct Engine {
    int64_t m, n, ldm;
    int r, p, pp, K, cp, nseg;
    const T* M;
    double lam;
    std::vector<double> mu;
    cudaStream_t s;
    // one-time factor
    double *Md, *Kd, *Wd, *Rd, *lam_d, *Ud, *Usd, *Vd;
    double *joff_d, *jscale_d;
    int *jdone_d, *rot_d, *order_d;
    JacDesc<double>* jdesc;
    int mpp;
    T *Wm, *dinv, *V;            // Wm (m x m) eigenvectors of M M^T, dinv = 1/(1+l), V (n x r)
    // iteration state and scratch
    T *Z, *E, *Y1, *Y2, *Wj;     // Wj: Jacobi basis (pp x pp)
    T *A, *At, *X, *J, *R, *T1, *T2, *MZ, *Xe, *H, *T1b;
    T *sv, *fs, *invs;
    int* rank_d;
    T *Wh, *Wg, *Wt;             // W^T W, W (W^T W), first-order inverse
    OsjDesc<T>* od;
    T *oscale, *ooff;
    int *odone, *oon;
    T **pW, **pH, **pT;
    int *pv, *ppv;
    GemmDesc<T>* gd;
    int gslot = 0;
    // checkpoints and saved iterates of one segment
    std::vector<T*> cpZ, cpE, cpY1, cpY2, cpW;
    std::vector<T*> svZ, svMZ, svXe, svEin, svY1in, svU, svVr, svS;
    // adjoints
    T *Zb, *Eb, *Y1b, *Y2b, *Cb, *MZb, *Jb, *Xb, *Q, *MQ, *Ab, *Y1ib, *Y2ib, *Eib, *B1, *B2, *Pm, *C2, *L1, *FB2, *Fv;
    T *Mb;
    double* dth;

    cudaError_t gemm(bool ta, bool tb, int M_, int N_, int K_, T alpha, const T* A_, int64_t lda, const T* B_,
                     int64_t ldb, T beta, T* C_, int64_t ldc) {
        GemmDesc<T> d{};
        d.A = A_; d.B = B_; d.C = C_; d.flag = nullptr; d.ccol = nullptr; d.kscale = nullptr; d.absmax = nullptr;
        d.lda = lda; d.ldb = ldb; d.ldc = ldc; d.m = M_; d.n = N_; d.k = K_; d.alpha = alpha; d.beta = beta;
        GemmDesc<T>* slot = gd + (gslot++ % 64);
        cudaError_t e = cudaMemcpyAsync(slot, &d, sizeof(d), cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) return e;
        return gemm_grouped<T>(slot, 1, ta, tb, M_, N_, s);
    }
};

template <typename T>
size_t carve_engine(Engine<T>& g, Bump& b) {
    const int64_t m = g.m, n = g.n, mm = m * n, nn = n * n;
    const int r = g.r, pp = g.pp;
    g.Md = b.take<double>(mm);
    g.Kd = b.take<double>((size_t)g.mpp * g.mpp);
    g.Wd = b.take<double>((size_t)g.mpp * g.mpp);
    g.Rd = b.take<double>((size_t)g.mpp * 32);
    g.lam_d = b.take<double>(m);
    g.Ud = b.take<double>(m * m);
    g.Usd = b.take<double>(m * m);
    g.Vd = b.take<double>(n * m);
    g.joff_d = b.take<double>(1);
    g.jscale_d = b.take<double>(1);
    g.jdone_d = b.take<int>(1);
    g.rot_d = b.take<int>(g.mpp / 32);
    g.order_d = b.take<int>(m);
    g.jdesc = b.take<JacDesc<double>>(1);
    g.Wm = b.take<T>(m * m);
    g.dinv = b.take<T>(m);
    g.V = b.take<T>(n * (int64_t)r);
    g.Z = b.take<T>(nn); g.E = b.take<T>(mm); g.Y1 = b.take<T>(mm); g.Y2 = b.take<T>(nn);
    g.Wj = b.take<T>((size_t)pp * pp);
    g.A = b.take<T>(nn); g.At = b.take<T>(n * (int64_t)r); g.X = b.take<T>(n * (int64_t)r); g.J = b.take<T>(nn);
    g.R = b.take<T>(nn); g.T1 = b.take<T>(mm); g.T2 = b.take<T>(mm); g.MZ = b.take<T>(mm); g.Xe = b.take<T>(mm);
    g.H = b.take<T>(n * (int64_t)r); g.T1b = b.take<T>(nn);
    g.sv = b.take<T>(pp); g.fs = b.take<T>(pp); g.invs = b.take<T>(pp);
    g.rank_d = b.take<int>(1);
    g.Wh = b.take<T>((size_t)pp * pp); g.Wg = b.take<T>((size_t)pp * pp); g.Wt = b.take<T>((size_t)pp * pp);
    g.od = b.take<OsjDesc<T>>(1);
    g.oscale = b.take<T>(1); g.ooff = b.take<T>(3);
    g.odone = b.take<int>(1); g.oon = b.take<int>(1);
    g.pW = b.take<T*>(1); g.pH = b.take<T*>(1); g.pT = b.take<T*>(1);
    g.pv = b.take<int>(1); g.ppv = b.take<int>(1);
    g.gd = b.take<GemmDesc<T>>(64);
    g.cpZ.resize(g.nseg); g.cpE.resize(g.nseg); g.cpY1.resize(g.nseg); g.cpY2.resize(g.nseg); g.cpW.resize(g.nseg);
    for (int i = 0; i < g.nseg; ++i) {
        g.cpZ[i] = b.take<T>(nn); g.cpE[i] = b.take<T>(mm); g.cpY1[i] = b.take<T>(mm); g.cpY2[i] = b.take<T>(nn);
        g.cpW[i] = b.take<T>((size_t)pp * pp);
    }
    const int cp = g.cp;
    g.svZ.resize(cp); g.svMZ.resize(cp); g.svXe.resize(cp); g.svEin.resize(cp); g.svY1in.resize(cp);
    g.svU.resize(cp); g.svVr.resize(cp); g.svS.resize(cp);
    for (int i = 0; i < cp; ++i) {
        g.svZ[i] = b.take<T>(nn); g.svMZ[i] = b.take<T>(mm); g.svXe[i] = b.take<T>(mm);
        g.svEin[i] = b.take<T>(mm); g.svY1in[i] = b.take<T>(mm);
        g.svU[i] = b.take<T>(n * (int64_t)r); g.svVr[i] = b.take<T>(n * (int64_t)r); g.svS[i] = b.take<T>(pp);
    }
    g.Zb = b.take<T>(nn); g.Eb = b.take<T>(mm); g.Y1b = b.take<T>(mm); g.Y2b = b.take<T>(nn);
    g.Cb = b.take<T>(mm); g.MZb = b.take<T>(mm); g.Jb = b.take<T>(nn); g.Xb = b.take<T>(mm); g.Q = b.take<T>(nn);
    g.MQ = b.take<T>(mm); g.Ab = b.take<T>(nn); g.Y1ib = b.take<T>(mm); g.Y2ib = b.take<T>(nn); g.Eib = b.take<T>(mm);
    g.B1 = b.take<T>(n * (int64_t)r); g.B2 = b.take<T>(n * (int64_t)r); g.Pm = b.take<T>((size_t)r * r);
    g.C2 = b.take<T>((size_t)r * r); g.L1 = b.take<T>(n * (int64_t)r); g.FB2 = b.take<T>(n * (int64_t)r);
    g.Fv = b.take<T>(pp);
    g.Mb = b.take<T>(mm);
    g.dth = b.take<double>(1);
    return b.off + kAl;
}

#define UTRY(x)                                   \
    do {                                          \
        cudaError_t _e = (x);                     \
        if (_e != cudaSuccess) return LRR_ERR_CUDA; \
    } while (0)

// the one-time factor: M M^T = Wm diag(l) Wm^T (float64 block Jacobi), rank r,
// V = M^T U diag(1/sigma) for the r eigenvalues above rank_tol
template <typename T>
int setup(Engine<T>& g, double rank_tol) {
    const int64_t m = g.m, n = g.n;
    cudaStream_t s = g.s;
    lrr::k::gather_cols<double, T><<<dim3(g1(m), (unsigned)std::min<int64_t>(n, 65535)), 256, 0, s>>>(
        g.M, g.ldm, nullptr, m, n, g.Md);
    lrr::k::init_padded<double><<<g1((int64_t)g.mpp * g.mpp), 256, 0, s>>>(g.Kd, (int)m, g.mpp, -1.0, 0);
    lrr::k::init_padded<double><<<g1((int64_t)g.mpp * g.mpp), 256, 0, s>>>(g.Wd, (int)m, g.mpp, 1.0, 1);
    {
        GemmDesc<double> d{};
        d.A = g.Md; d.B = g.Md; d.C = g.Kd; d.lda = m; d.ldb = m; d.ldc = g.mpp;
        d.m = (int)m; d.n = (int)m; d.k = (int)n; d.alpha = 1.0; d.beta = 0.0;
        GemmDesc<double>* dd = reinterpret_cast<GemmDesc<double>*>(g.gd);
        UTRY(cudaMemcpyAsync(dd, &d, sizeof(d), cudaMemcpyHostToDevice, s));
        UTRY(gemm_grouped<double>(dd, 1, false, true, (int)m, (int)m, s));
    }
    lrr::k::diag_of<double><<<ceil_div(m, 256), 256, 0, s>>>(g.Kd, g.mpp, m, g.lam_d);
    std::vector<double> dg((size_t)m);
    UTRY(cudaMemcpyAsync(dg.data(), g.lam_d, sizeof(double) * m, cudaMemcpyDeviceToHost, s));
    UTRY(cudaStreamSynchronize(s));
    double sc = 0;
    for (double v : dg) sc = std::max(sc, std::fabs(v));
    if (!(sc > 0)) return LRR_ERR_RANK;
    JacDesc<double> jd{};
    jd.G = g.Kd; jd.W = g.Wd; jd.R = g.Rd; jd.rot = g.rot_d; jd.done = g.jdone_d; jd.off = g.joff_d;
    jd.active = nullptr; jd.scale = g.jscale_d; jd.pp = g.mpp;
    UTRY(cudaMemcpyAsync(g.jscale_d, &sc, sizeof(double), cudaMemcpyHostToDevice, s));
    UTRY(cudaMemcpyAsync(g.jdesc, &jd, sizeof(jd), cudaMemcpyHostToDevice, s));
    UTRY(jacobi_sweeps<double>(g.jdesc, 1, g.mpp, 40, 1e-13, s, g.jdone_d));
    lrr::k::diag_of<double><<<ceil_div(m, 256), 256, 0, s>>>(g.Kd, g.mpp, m, g.lam_d);
    std::vector<double> ev((size_t)m);
    UTRY(cudaMemcpyAsync(ev.data(), g.lam_d, sizeof(double) * m, cudaMemcpyDeviceToHost, s));
    UTRY(cudaStreamSynchronize(s));
    std::vector<int> order((size_t)m);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return ev[a] > ev[b]; });
    const double smax = std::sqrt(std::max(ev[order[0]], 0.0));
    int r = 0;
    while (r < (int)m && std::sqrt(std::max(ev[order[r]], 0.0)) > rank_tol * smax) ++r;
    if (r == 0) return LRR_ERR_RANK;
    g.r = r;                                  // buffers were sized for min(m, n)
    g.p = r;
    g.pp = rup(r, osj_pivot_width());
    // all m eigenpairs, sorted, for (I + M M^T)^{-1}; the first r for V
    std::vector<double> lam_sorted((size_t)m);
    for (int i = 0; i < (int)m; ++i) lam_sorted[i] = std::max(ev[order[i]], 0.0);
    UTRY(cudaMemcpyAsync(g.order_d, order.data(), sizeof(int) * m, cudaMemcpyHostToDevice, s));
    UTRY(cudaMemcpyAsync(g.lam_d, lam_sorted.data(), sizeof(double) * m, cudaMemcpyHostToDevice, s));
    lrr::k::setup_factors<<<dim3(g1(m), (unsigned)m), 256, 0, s>>>(g.Wd, g.mpp, m, (int)m, g.order_d, g.lam_d,
                                                                    g.Ud, g.Usd);
    lrr::k::copy_convert_f64<T><<<g1(m * m), 256, 0, s>>>(g.Ud, g.Wm, m * m);
    std::vector<T> dinv((size_t)m);
    for (int i = 0; i < (int)m; ++i) dinv[i] = (T)(1.0 / (1.0 + lam_sorted[i]));
    UTRY(cudaMemcpyAsync(g.dinv, dinv.data(), sizeof(T) * m, cudaMemcpyHostToDevice, s));
    {
        GemmDesc<double> d{};
        d.A = g.Md; d.B = g.Usd; d.C = g.Vd; d.lda = m; d.ldb = m; d.ldc = n;
        d.m = (int)n; d.n = r; d.k = (int)m; d.alpha = 1.0; d.beta = 0.0;
        GemmDesc<double>* dd = reinterpret_cast<GemmDesc<double>*>(g.gd);
        UTRY(cudaMemcpyAsync(dd, &d, sizeof(d), cudaMemcpyHostToDevice, s));
        UTRY(gemm_grouped<double>(dd, 1, true, false, (int)n, r, s));
    }
    lrr::k::copy_convert_f64<T><<<g1(n * (int64_t)r), 256, 0, s>>>(g.Vd, g.V, n * (int64_t)r);
    return LRR_OK;
}

// Zout = (I + M^T M)^{-1} Rin = Rin - M^T Wm diag(dinv) Wm^T M Rin  (n x n)
template <typename T>
int solve_S(Engine<T>& g, const T* Rin, T* Zout) {
    const int64_t m = g.m, n = g.n;
    UTRY(g.gemm(false, false, (int)m, (int)n, (int)n, T(1), g.M, g.ldm, Rin, n, T(0), g.T1, m));
    UTRY(g.gemm(true, false, (int)m, (int)n, (int)m, T(1), g.Wm, m, g.T1, m, T(0), g.T2, m));
    u::scale_rows<T><<<g1(m * n), 256, 0, g.s>>>(g.T2, m, n, g.dinv);
    UTRY(g.gemm(false, false, (int)m, (int)n, (int)m, T(1), g.Wm, m, g.T2, m, T(0), g.T1, m));
    if (Zout != Rin) UTRY(cudaMemcpyAsync(Zout, Rin, sizeof(T) * n * n, cudaMemcpyDeviceToDevice, g.s));
    UTRY(g.gemm(true, false, (int)n, (int)n, (int)m, T(-1), g.M, g.ldm, g.T1, m, T(1), Zout, n));
    return LRR_OK;
}

// SVT of A (n x n, in range(V)): At = (V^T A)^T = A^T V (n x r), X = At Wj, one-sided
// Jacobi (warm start Wj), then J = V Wt diag(h) X^T with Wt the first-order inverse
// transpose of Wj; returns the triplets U = V Wj (n x r), s, Vr = X diag(1/s) when asked.
template <typename T>
int svt(Engine<T>& g, double mu, T* Uout, T* Vrout, T* Sout) {
    const int64_t n = g.n;
    const int r = g.r, pp = g.pp;
    cudaStream_t s = g.s;
    UTRY(g.gemm(true, false, (int)n, r, (int)n, T(1), g.A, n, g.V, n, T(0), g.At, n));
    UTRY(g.gemm(false, false, (int)n, r, r, T(1), g.At, n, g.Wj, pp, T(0), g.X, n));
    const int one = 1;
    UTRY(cudaMemcpyAsync(g.oon, &one, sizeof(int), cudaMemcpyHostToDevice, s));
    lrr::k::col_norm_max<T><<<1, 256, 0, s>>>(g.od, g.oon, g.oscale, 1);
    UTRY(osj_sweeps<T>(g.od, 1, pp, 40, sizeof(T) == 8 ? T(1e-13) : T(2e-6), nullptr, s, 0));
    const T tau = (T)(1.0 / mu);
    UTRY(cudaMemsetAsync(g.rank_d, 0, sizeof(int), s));
    u::svt_svals<T><<<ceil_div((int64_t)r * 32, 256), 256, 0, s>>>(g.X, n, n, r, tau, g.sv, g.fs, g.invs, g.rank_d);
    // W^T W, W (W^T W): Wt = 2W - W W^T W (first-order inverse transpose), W <- 1.5 W - 0.5 W W^T W
    UTRY(g.gemm(true, false, r, r, r, T(1), g.Wj, pp, g.Wj, pp, T(0), g.Wh, pp));
    UTRY(g.gemm(false, false, r, r, r, T(1), g.Wj, pp, g.Wh, pp, T(0), g.Wg, pp));
    if (Uout) {
        // triplets from the orthogonalised columns, before the warm start is polished
        UTRY(g.gemm(false, false, (int)n, r, r, T(1), g.V, n, g.Wj, pp, T(0), Uout, n));
        u::scale_cols<T><<<g1(n * (int64_t)r), 256, 0, s>>>(g.X, n, r, g.invs, Vrout);
        UTRY(cudaMemcpyAsync(Sout, g.sv, sizeof(T) * r, cudaMemcpyDeviceToDevice, s));
    }
    lrr::k::ns_orth<T><<<dim3(64, 1), 256, 0, s>>>(g.pW, g.pH, g.pT, g.pv, g.ppv, g.oon, 1);
    // J = V (Wt diag(h) X^T): H = X diag(h) (n x r), Jr^T = H Wt^T -> J = V (Wt H^T)
    u::scale_cols<T><<<g1(n * (int64_t)r), 256, 0, s>>>(g.X, n, r, g.fs, g.H);
    UTRY(g.gemm(false, true, (int)n, r, r, T(1), g.H, n, g.Wt, pp, T(0), g.At, n));       // At = H Wt^T (n x r)
    UTRY(g.gemm(false, true, (int)n, (int)n, r, T(1), g.V, n, g.At, n, T(0), g.J, n));    // J = V At^T
    return LRR_OK;
}

// one forward iteration k on the engine's state; saves the backward's
// intermediates into slot `sv` (-1: none)
template <typename T>
int forward_step(Engine<T>& g, int k, int sv) {
    const int64_t m = g.m, n = g.n, mm = m * n, nn = n * n;
    cudaStream_t s = g.s;
    const double mu = g.mu[k];
    const T muT = (T)mu, imu = (T)(1.0 / mu);
    const bool last = k == g.K - 1;
    if (sv >= 0) {
        UTRY(cudaMemcpyAsync(g.svEin[sv], g.E, sizeof(T) * mm, cudaMemcpyDeviceToDevice, s));
        UTRY(cudaMemcpyAsync(g.svY1in[sv], g.Y1, sizeof(T) * mm, cudaMemcpyDeviceToDevice, s));
    }
    u::lincomb<T><<<g1(nn), 256, 0, s>>>(nn, T(1), g.Z, imu, g.Y2, g.A);
    int rc = svt<T>(g, mu, sv >= 0 ? g.svU[sv] : nullptr, sv >= 0 ? g.svVr[sv] : nullptr,
                    sv >= 0 ? g.svS[sv] : nullptr);
    if (rc != LRR_OK) return rc;
    // R = M^T (C - E + Y1/mu) + J - Y2/mu
    lrr::k::gather_cols<T, T><<<dim3(g1(m), (unsigned)std::min<int64_t>(n, 65535)), 256, 0, s>>>(g.M, g.ldm, nullptr,
                                                                                                 m, n, g.T2);
    u::lincomb3<T><<<g1(mm), 256, 0, s>>>(mm, g.T2, T(-1), g.E, imu, g.Y1, g.T2);
    u::lincomb<T><<<g1(nn), 256, 0, s>>>(nn, T(1), g.J, -imu, g.Y2, g.R);
    UTRY(g.gemm(true, false, (int)n, (int)n, (int)m, T(1), g.M, g.ldm, g.T2, m, T(1), g.R, n));
    // Z = S^-1 R
    rc = solve_S<T>(g, g.R, g.Z);
    if (rc != LRR_OK) return rc;
    UTRY(g.gemm(false, false, (int)m, (int)n, (int)n, T(1), g.M, g.ldm, g.Z, n, T(0), g.MZ, m));
    u::shrink_fwd<T><<<ceil_div(n * 32, 256), 256, 0, s>>>(m, n, g.M, g.ldm, g.MZ, g.Y1, g.E, g.Xe, muT,
                                                          (T)(g.lam / mu), last ? 0 : 1);
    if (!last) {
        u::axpby<T><<<g1(nn), 256, 0, s>>>(nn, muT, g.Z, T(1), g.Y2);
        u::axpby<T><<<g1(nn), 256, 0, s>>>(nn, -muT, g.J, T(1), g.Y2);
    }
    if (sv >= 0) {
        UTRY(cudaMemcpyAsync(g.svZ[sv], g.Z, sizeof(T) * nn, cudaMemcpyDeviceToDevice, s));
        UTRY(cudaMemcpyAsync(g.svMZ[sv], g.MZ, sizeof(T) * mm, cudaMemcpyDeviceToDevice, s));
        UTRY(cudaMemcpyAsync(g.svXe[sv], g.Xe, sizeof(T) * mm, cudaMemcpyDeviceToDevice, s));
    }
    return LRR_OK;
}

// one backward iteration k (its intermediates in slot sv): pulls the adjoints
// of the iterate after step k (Zb, Eb, Y1b, Y2b) back to the iterate before
// it, accumulating dL/dM into Mb and dL/dlambda into *dth.
template <typename T>
int backward_step(Engine<T>& g, int k, int sv) {
    const int64_t m = g.m, n = g.n, mm = m * n, nn = n * n;
    const int r = g.r;
    cudaStream_t s = g.s;
    const double mu = g.mu[k];
    const T muT = (T)mu, imu = (T)(1.0 / mu);
    const bool last = k == g.K - 1;
    // dual step Y1' = Y1 + mu (C - MZ - E), Y2' = Y2 + mu (Z - J)
    if (!last) {
        u::lincomb<T><<<g1(mm), 256, 0, s>>>(mm, muT, g.Y1b, T(0), g.Y1b, g.Cb);
        u::lincomb<T><<<g1(mm), 256, 0, s>>>(mm, -muT, g.Y1b, T(0), g.Y1b, g.MZb);
        u::axpby<T><<<g1(mm), 256, 0, s>>>(mm, -muT, g.Y1b, T(1), g.Eb);
        u::axpby<T><<<g1(nn), 256, 0, s>>>(nn, muT, g.Y2b, T(1), g.Zb);
        u::lincomb<T><<<g1(nn), 256, 0, s>>>(nn, -muT, g.Y2b, T(0), g.Y2b, g.Jb);
    } else {
        UTRY(cudaMemsetAsync(g.Cb, 0, sizeof(T) * mm, s));
        UTRY(cudaMemsetAsync(g.MZb, 0, sizeof(T) * mm, s));
        UTRY(cudaMemsetAsync(g.Jb, 0, sizeof(T) * nn, s));
    }
    UTRY(cudaMemcpyAsync(g.Y1ib, g.Y1b, sizeof(T) * mm, cudaMemcpyDeviceToDevice, s));
    UTRY(cudaMemcpyAsync(g.Y2ib, g.Y2b, sizeof(T) * nn, cudaMemcpyDeviceToDevice, s));
    // E-step E = shrink(X, lambda/mu), X = C - MZ + Y1/mu
    u::shrink_adj<T><<<ceil_div(n * 32, 256), 256, 0, s>>>(m, n, g.svXe[sv], g.Eb, g.Xb, (T)(g.lam / mu), 1.0 / mu,
                                                          g.dth);
    u::axpby<T><<<g1(mm), 256, 0, s>>>(mm, T(1), g.Xb, T(1), g.Cb);
    u::axpby<T><<<g1(mm), 256, 0, s>>>(mm, T(-1), g.Xb, T(1), g.MZb);
    u::axpby<T><<<g1(mm), 256, 0, s>>>(mm, imu, g.Xb, T(1), g.Y1ib);
    // MZ = M Z
    UTRY(g.gemm(false, true, (int)m, (int)n, (int)n, T(1), g.MZb, m, g.svZ[sv], n, T(1), g.Mb, m));
    UTRY(g.gemm(true, false, (int)n, (int)n, (int)m, T(1), g.M, g.ldm, g.MZb, m, T(1), g.Zb, n));
    // Z = S^-1 R:  Q = S^-1 Zbar,  Mbar -= (M Z) Q^T + (M Q) Z^T
    int rc = solve_S<T>(g, g.Zb, g.Q);
    if (rc != LRR_OK) return rc;
    UTRY(g.gemm(false, false, (int)m, (int)n, (int)n, T(1), g.M, g.ldm, g.Q, n, T(0), g.MQ, m));
    UTRY(g.gemm(false, true, (int)m, (int)n, (int)n, T(-1), g.svMZ[sv], m, g.Q, n, T(1), g.Mb, m));
    UTRY(g.gemm(false, true, (int)m, (int)n, (int)n, T(-1), g.MQ, m, g.svZ[sv], n, T(1), g.Mb, m));
    // R = M^T (C - E + Y1/mu) + J - Y2/mu with Rbar = Q
    lrr::k::gather_cols<T, T><<<dim3(g1(m), (unsigned)std::min<int64_t>(n, 65535)), 256, 0, s>>>(g.M, g.ldm, nullptr,
                                                                                                 m, n, g.T2);
    u::lincomb3<T><<<g1(mm), 256, 0, s>>>(mm, g.T2, T(-1), g.svEin[sv], imu, g.svY1in[sv], g.T2);
    UTRY(g.gemm(false, true, (int)m, (int)n, (int)n, T(1), g.T2, m, g.Q, n, T(1), g.Mb, m));
    u::axpby<T><<<g1(mm), 256, 0, s>>>(mm, T(1), g.MQ, T(1), g.Cb);
    u::lincomb<T><<<g1(mm), 256, 0, s>>>(mm, T(-1), g.MQ, T(0), g.MQ, g.Eib);
    u::axpby<T><<<g1(nn), 256, 0, s>>>(nn, T(1), g.Q, T(1), g.Jb);
    u::axpby<T><<<g1(mm), 256, 0, s>>>(mm, imu, g.MQ, T(1), g.Y1ib);
    u::axpby<T><<<g1(nn), 256, 0, s>>>(nn, -imu, g.Q, T(1), g.Y2ib);
    // J = SVT(A), A = Z + Y2/mu:  Abar from Jbar through the singular triplets
    const T tau = (T)(1.0 / mu);
    T* U = g.svU[sv];
    T* Vr = g.svVr[sv];
    UTRY(g.gemm(false, false, (int)n, r, (int)n, T(1), g.Jb, n, Vr, n, T(0), g.B1, n));     // Jbar Vr
    UTRY(g.gemm(true, false, (int)n, r, (int)n, T(1), g.Jb, n, U, n, T(0), g.B2, n));       // (U^T Jbar)^T
    UTRY(g.gemm(true, false, r, r, (int)n, T(1), U, n, g.B1, n, T(0), g.Pm, r));           // P = U^T Jbar Vr
    u::svt_core<T><<<g1((int64_t)r * r), 256, 0, s>>>(g.Pm, r, g.svS[sv], tau, g.C2);
    u::f_over_s<T><<<ceil_div(r, 256), 256, 0, s>>>(g.svS[sv], r, tau, g.Fv);
    u::scale_cols<T><<<g1(n * (int64_t)r), 256, 0, s>>>(g.B1, n, r, g.Fv, g.L1);
    UTRY(g.gemm(false, false, (int)n, r, r, T(1), U, n, g.C2, r, T(1), g.L1, n));           // L1 = U C2 + B1 F
    u::scale_cols<T><<<g1(n * (int64_t)r), 256, 0, s>>>(g.B2, n, r, g.Fv, g.FB2);          // (F U^T Jbar)^T
    UTRY(g.gemm(false, true, (int)n, (int)n, r, T(1), g.L1, n, Vr, n, T(0), g.Ab, n));
    UTRY(g.gemm(false, true, (int)n, (int)n, r, T(1), U, n, g.FB2, n, T(1), g.Ab, n));
    u::axpby<T><<<g1(nn), 256, 0, s>>>(nn, imu, g.Ab, T(1), g.Y2ib);
    // observations are the dictionary
    u::axpby<T><<<g1(mm), 256, 0, s>>>(mm, T(1), g.Cb, T(1), g.Mb);
    std::swap(g.Zb, g.Ab);
    std::swap(g.Eb, g.Eib);
    std::swap(g.Y1b, g.Y1ib);
    std::swap(g.Y2b, g.Y2ib);
    return LRR_OK;
}

template <typename T>
int reset_state(Engine<T>& g) {
    const int64_t m = g.m, n = g.n;
    cudaStream_t s = g.s;
    UTRY(cudaMemsetAsync(g.Z, 0, sizeof(T) * n * n, s));
    UTRY(cudaMemsetAsync(g.Y2, 0, sizeof(T) * n * n, s));
    UTRY(cudaMemsetAsync(g.E, 0, sizeof(T) * m * n, s));
    UTRY(cudaMemsetAsync(g.Y1, 0, sizeof(T) * m * n, s));
    lrr::k::init_padded<T><<<g1((int64_t)g.pp * g.pp), 256, 0, s>>>(g.Wj, g.r, g.pp, T(1), 1);
    return LRR_OK;
}

template <typename T>
int copy_state(Engine<T>& g, int seg, bool save) {
    const int64_t m = g.m, n = g.n;
    cudaStream_t s = g.s;
    auto cp = [&](T* a, T* b, size_t count) {
        return cudaMemcpyAsync(save ? b : a, save ? a : b, sizeof(T) * count, cudaMemcpyDeviceToDevice, s);
    };
    UTRY(cp(g.Z, g.cpZ[seg], n * n));
    UTRY(cp(g.Y2, g.cpY2[seg], n * n));
    UTRY(cp(g.E, g.cpE[seg], m * n));
    UTRY(cp(g.Y1, g.cpY1[seg], m * n));
    UTRY(cp(g.Wj, g.cpW[seg], (size_t)g.pp * g.pp));
    return LRR_OK;
}

template <typename T>
int engine_init(Engine<T>& g) {
    cudaStream_t s = g.s;
    OsjDesc<T> d{};
    d.X = g.X; d.W = g.Wj; d.done = g.odone; d.off = g.ooff; d.active = g.oon; d.scale = g.oscale;
    // no threshold in the measure (d.mu null): the reverse pass needs every
    // singular pair resolved, including the ones the SVT removes
    d.mu = nullptr;
    d.ldx = g.n; d.ldw = g.pp; d.L = (int)g.n; d.p = g.r; d.pp = g.pp; d.strict = 1;
    UTRY(cudaMemcpyAsync(g.od, &d, sizeof(d), cudaMemcpyHostToDevice, s));
    T* ptrs[3] = {g.Wj, g.Wg, g.Wt};
    UTRY(cudaMemcpyAsync(g.pW, &ptrs[0], sizeof(T*), cudaMemcpyHostToDevice, s));
    UTRY(cudaMemcpyAsync(g.pH, &ptrs[1], sizeof(T*), cudaMemcpyHostToDevice, s));
    UTRY(cudaMemcpyAsync(g.pT, &ptrs[2], sizeof(T*), cudaMemcpyHostToDevice, s));
    const int pv[2] = {g.r, g.pp};
    UTRY(cudaMemcpyAsync(g.pv, &pv[0], sizeof(int), cudaMemcpyHostToDevice, s));
    UTRY(cudaMemcpyAsync(g.ppv, &pv[1], sizeof(int), cudaMemcpyHostToDevice, s));
    UTRY(cudaMemsetAsync(g.Wt, 0, sizeof(T) * g.pp * g.pp, s));
    UTRY(cudaMemsetAsync(g.Wg, 0, sizeof(T) * g.pp * g.pp, s));
    return LRR_OK;
}

bool valid_unrolled(int64_t m, int64_t n, int64_t ldm, const lrr_unrolled_options* o) {
    if (!o || m < 1 || n < 1 || ldm < m || m > 4096 || n > 16384) return false;
    if (!(o->lambda > 0) || !(o->rho >= 1) || !(o->mu0 > 0) || !(o->mu_max >= o->mu0)) return false;
    if (o->K < 1 || o->K > 100000 || o->checkpoint < 0) return false;
    return o->precision == LRR_PREC_F32 || o->precision == LRR_PREC_F64;
}

template <typename T>
Engine<T> make_engine(const void* M, int64_t m, int64_t n, int64_t ldm, const lrr_unrolled_options* o, bool grad) {
    Engine<T> g{};
    g.m = m; g.n = n; g.ldm = ldm;
    g.M = static_cast<const T*>(M);
    g.lam = o->lambda;
    g.K = o->K;
    g.cp = grad ? std::max(1, std::min(o->checkpoint > 0 ? o->checkpoint : 5, o->K)) : 1;
    g.nseg = grad ? (g.K + g.cp - 1) / g.cp : 0;
    g.r = (int)std::min(m, n);
    g.p = g.r;
    g.pp = rup(g.r, osj_pivot_width());
    g.mpp = rup((int)m, 2 * jacobi_bs<double>());
    double mu = o->mu0;
    for (int k = 0; k < g.K; ++k) {
        g.mu.push_back(mu);
        mu = std::min(o->rho * mu, o->mu_max);
    }
    return g;
}

template <typename T>
size_t unrolled_ws(int64_t m, int64_t n, const lrr_unrolled_options* o, bool grad) {
    Engine<T> g = make_engine<T>(nullptr, m, n, std::max<int64_t>(m, 1), o, grad);
    if (!grad) g.cp = 0;
    Bump b(nullptr);
    return carve_engine<T>(g, b);
}

template <typename T>
int unrolled_run(const void* M, int64_t m, int64_t n, int64_t ldm, const lrr_unrolled_options* o, void* Zout,
                 int64_t ldz, const void* Zbar, int64_t ldzb, void* Mbar, int64_t ldmb, double* lambar, void* ws,
                 size_t wsb, cudaStream_t s) {
    const bool grad = Zbar != nullptr;
    Engine<T> g = make_engine<T>(M, m, n, ldm, o, grad);
    if (!grad) g.cp = 0;
    g.s = s;
    Bump probe(nullptr);
    const size_t need = carve_engine<T>(g, probe);
    void* own = nullptr;
    if (!ws) {
        if (cudaMallocAsync(&own, need, s) != cudaSuccess) return LRR_ERR_CUDA;
        ws = own;
        wsb = need;
    }
    struct Free {
        void* p; cudaStream_t s;
        ~Free() { if (p) cudaFreeAsync(p, s); }
    } guard{own, s};
    if (wsb < need - kAl || (reinterpret_cast<uintptr_t>(ws) % kAl) != 0) return LRR_ERR_WORKSPACE;
    Bump b(ws);
    carve_engine<T>(g, b);
    int rc = setup<T>(g, o->rank_tol > 0 ? o->rank_tol : 1e-6);
    if (rc != LRR_OK) return rc;
    rc = engine_init<T>(g);
    if (rc != LRR_OK) return rc;
    rc = reset_state<T>(g);
    if (rc != LRR_OK) return rc;
    for (int k = 0; k < g.K; ++k) {
        if (grad && k % g.cp == 0) {
            rc = copy_state<T>(g, k / g.cp, true);
            if (rc != LRR_OK) return rc;
        }
        rc = forward_step<T>(g, k, -1);
        if (rc != LRR_OK) return rc;
    }
    if (Zout)
        UTRY(cudaMemcpy2DAsync(Zout, sizeof(T) * ldz, g.Z, sizeof(T) * n, sizeof(T) * n, (size_t)n,
                               cudaMemcpyDeviceToDevice, s));
    if (grad) {
        UTRY(cudaMemcpy2DAsync(g.Zb, sizeof(T) * n, Zbar, sizeof(T) * ldzb, sizeof(T) * n, (size_t)n,
                               cudaMemcpyDeviceToDevice, s));
        UTRY(cudaMemsetAsync(g.Eb, 0, sizeof(T) * m * n, s));
        UTRY(cudaMemsetAsync(g.Y1b, 0, sizeof(T) * m * n, s));
        UTRY(cudaMemsetAsync(g.Y2b, 0, sizeof(T) * n * n, s));
        UTRY(cudaMemsetAsync(g.Mb, 0, sizeof(T) * m * n, s));
        UTRY(cudaMemsetAsync(g.dth, 0, sizeof(double), s));
        for (int seg = g.nseg - 1; seg >= 0; --seg) {
            const int k0 = seg * g.cp, k1 = std::min(g.K, k0 + g.cp);
            rc = copy_state<T>(g, seg, false);
            if (rc != LRR_OK) return rc;
            for (int k = k0; k < k1; ++k) {
                rc = forward_step<T>(g, k, k - k0);
                if (rc != LRR_OK) return rc;
            }
            for (int k = k1 - 1; k >= k0; --k) {
                rc = backward_step<T>(g, k, k - k0);
                if (rc != LRR_OK) return rc;
            }
        }
        if (Mbar)
            UTRY(cudaMemcpy2DAsync(Mbar, sizeof(T) * ldmb, g.Mb, sizeof(T) * m, sizeof(T) * m, (size_t)n,
                                   cudaMemcpyDeviceToDevice, s));
        double lb = 0.0;
        UTRY(cudaMemcpyAsync(&lb, g.dth, sizeof(double), cudaMemcpyDeviceToHost, s));
        UTRY(cudaStreamSynchronize(s));
        if (lambar) *lambar = lb;
    }
    UTRY(cudaStreamSynchronize(s));
    return LRR_OK;
}

}  // namespace
}  // namespace lrr

extern "C" {

size_t lrr_unrolled_workspace_bytes(int64_t m, int64_t n, const lrr_unrolled_options* o, int32_t with_grad) {
    if (!lrr::valid_unrolled(m, n, m, o)) return 0;
    return o->precision == LRR_PREC_F64 ? lrr::unrolled_ws<double>(m, n, o, with_grad != 0)
                                        : lrr::unrolled_ws<float>(m, n, o, with_grad != 0);
}

int lrr_unrolled_forward(const void* M, int64_t m, int64_t n, int64_t ldm, const lrr_unrolled_options* o, void* Z,
                         int64_t ldz, void* workspace, size_t workspace_bytes, void* stream) {
    if (!M || !Z || !lrr::valid_unrolled(m, n, ldm, o) || ldz < n) return LRR_ERR_INVALID;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (o->precision == LRR_PREC_F64)
        return lrr::unrolled_run<double>(M, m, n, ldm, o, Z, ldz, nullptr, 0, nullptr, 0, nullptr, workspace,
                                         workspace_bytes, s);
    return lrr::unrolled_run<float>(M, m, n, ldm, o, Z, ldz, nullptr, 0, nullptr, 0, nullptr, workspace,
                                    workspace_bytes, s);
}

int lrr_unrolled_backward(const void* M, int64_t m, int64_t n, int64_t ldm, const lrr_unrolled_options* o,
                          const void* Zbar, int64_t ldzb, void* Mbar, int64_t ldmb, double* lambar, void* workspace,
                          size_t workspace_bytes, void* stream) {
    if (!M || !Zbar || !Mbar || !lambar || !lrr::valid_unrolled(m, n, ldm, o) || ldzb < n || ldmb < m)
        return LRR_ERR_INVALID;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (o->precision == LRR_PREC_F64)
        return lrr::unrolled_run<double>(M, m, n, ldm, o, nullptr, 0, Zbar, ldzb, Mbar, ldmb, lambar, workspace,
                                         workspace_bytes, s);
    return lrr::unrolled_run<float>(M, m, n, ldm, o, nullptr, 0, Zbar, ldzb, Mbar, ldmb, lambar, workspace,
                                    workspace_bytes, s);
}

}  // extern "C"
