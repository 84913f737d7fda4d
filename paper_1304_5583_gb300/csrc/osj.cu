// Batched one-sided block-Jacobi SVD for the singular-value thresholding step.
//
// For every block the L x p matrix X (X = A W for a tall A, X = A^T W for a
// wide one, W the previous iteration's right basis) is driven to orthogonal
// columns by rotations X <- X R, W <- W R.  The p columns are split into
// column blocks of b = 16; in each round the pp/b column blocks are paired
// round-robin (circle method) and every pair (a pivot of 2b = 32 columns)
//   1. forms the 32 x 32 Gram S = X_P^T X_P afresh from the columns of X
//      (each entry carries only the rounding of its own two columns),
//   2. rotates S towards diagonal form in shared memory (one inner cyclic
//      Jacobi sweep in float32, up to four in float64),
//   3. re-orthonormalises the accumulated rotation R and applies it to X_P
//      and W_P in update form.
// Pairs of a round touch disjoint columns.
//
// One launch runs every sweep of every block: each block is a thread-block
// cluster whose CTAs share the pairs of a round (a free CTA takes the next
// pair from a per-block counter) and meet at a cluster barrier between rounds
// (the barrier's release/acquire makes one round's column updates visible to
// the next).  After each sweep the cluster reduces the
// largest convergence measure seen in it and stops once that is below the
// tolerance, so a converged block costs nothing further and the others are
// not held to a common sweep count.
#include <cooperative_groups.h>

#include <type_traits>

#include "common.cuh"
#include "inner_jacobi.cuh"
#include "kernels.cuh"

namespace cg = cooperative_groups;

namespace lrr {
namespace {

constexpr int OB = 16;            // column-block width b
constexpr int B2 = 2 * OB;        // pivot width
constexpr int NT = 128;           // threads per CTA (one pivot at a time)
constexpr int NW = NT / 32;
constexpr int CH = 64;            // rows per staged chunk of the pivot columns
constexpr int LDX = B2 + 4;       // row stride of the staged chunk (16-byte rows)
constexpr int LO = B2 + 1;        // odd row stride of S and R (conflict-free scattered access)
constexpr int WORK = NW * B2 * B2;   // scratch: chunk tile, then per-warp partial Grams, then R^T R and R - I
static_assert(CH * LDX <= WORK && LO * B2 + B2 * B2 <= WORK, "scratch too small");

// Inner sweeps per pivot, at most.  float32 runs one: the pivot need not be
// diagonalised exactly, the next outer sweep continues from where one inner
// sweep leaves it.  On the 1000 x 20000 solve this took 10 881 outer sweeps
// against 11 126 with up to four inner sweeps, and 2.64 s of Jacobi time
// against 3.20 s.  float64 keeps up to four.
template <typename T> __host__ __device__ constexpr int inner_sweeps() { return sizeof(T) == 4 ? 1 : 4; }

__device__ __forceinline__ int pcol(int i, int a, int c) { return i < OB ? a * OB + i : c * OB + (i - OB); }

template <typename T>
struct Smem {
    T work[WORK];
    T S[B2][LO];
    T R[B2][LO];
    T cs[OB], sn[OB];
    int pi[OB], qi[OB];
    T red[NW];
    int pick;
};

// 16-byte vector loads from shared memory
__device__ __forceinline__ void lds4(const float* p, float (&v)[4]) {
    const float4 x = *reinterpret_cast<const float4*>(p);
    v[0] = x.x; v[1] = x.y; v[2] = x.z; v[3] = x.w;
}
__device__ __forceinline__ void lds4(const double* p, double (&v)[4]) {
    const double2 x = *reinterpret_cast<const double2*>(p);
    const double2 y = *reinterpret_cast<const double2*>(p + 2);
    v[0] = x.x; v[1] = x.y; v[2] = y.x; v[3] = y.y;
}

// One pivot (column blocks a and c) of one round: Gram, measure, rotation.
// Returns the convergence measure of the pivot (block-uniform).
template <typename T>
__device__ T osj_pivot(const OsjDesc<T>& d, Smem<T>& sm, int a, int c) {
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;

    // ---- 1. Gram S = X_P^T X_P over the L rows, in CH-row chunks staged in
    //      shared memory (the next chunk is fetched into registers while the
    //      current one is multiplied).  Warp w sums rows w*16 .. w*16+15 of a
    //      chunk into a fresh partial (4 x 8 entries per lane); the warps'
    //      totals are added in a fixed order at the end.
    T* const Xs = sm.work;
    constexpr int PER = CH * B2 / NT;           // chunk elements loaded per thread
    const int ti = lane & 7, tj = lane >> 3;     // S rows 4ti.., cols 8tj..
    T acc[4][8];
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 8; ++v) acc[u][v] = T(0);
    // thread t fetches row t % CH of the chunk in columns t / CH + 2u (u < PER):
    // the first PER/2 lie in column block a, the rest in column block c
    static_assert(NT == 2 * CH && PER == B2 / 2, "fetch mapping");
    T pre[PER];
    const int frow = t % CH, fcol = t / CH;
    const T* const pa = d.X + (int64_t)(a * OB + fcol) * d.ldx + frow;
    const T* const pc = d.X + (int64_t)(c * OB + fcol) * d.ldx + frow;
    const int64_t fst = 2 * d.ldx;
    auto fetch = [&](int ch) {
        const bool rok = ch * CH + frow < d.L;
        const int64_t ro = (int64_t)ch * CH;
#pragma unroll
        for (int u = 0; u < PER / 2; ++u) {
            pre[u] = (rok && a * OB + fcol + 2 * u < d.p) ? __ldcg(pa + ro + u * fst) : T(0);
            pre[u + PER / 2] = (rok && c * OB + fcol + 2 * u < d.p) ? __ldcg(pc + ro + u * fst) : T(0);
        }
    };
    const int nchunk = (d.L + CH - 1) / CH;
    fetch(0);
    for (int ch = 0; ch < nchunk; ++ch) {
#pragma unroll
        for (int u = 0; u < PER / 2; ++u) {
            Xs[frow * LDX + fcol + 2 * u] = pre[u];
            Xs[frow * LDX + OB + fcol + 2 * u] = pre[u + PER / 2];
        }
        __syncthreads();
        if (ch + 1 < nchunk) fetch(ch + 1);
        T part[4][8];
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int v = 0; v < 8; ++v) part[u][v] = T(0);
#pragma unroll 4
        for (int rr = warp * (CH / NW); rr < (warp + 1) * (CH / NW); ++rr) {
            T xi[4], xj0[4], xj1[4];
            lds4(Xs + rr * LDX + ti * 4, xi);
            lds4(Xs + rr * LDX + tj * 8, xj0);
            lds4(Xs + rr * LDX + tj * 8 + 4, xj1);
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int v = 0; v < 4; ++v) {
                    part[u][v] = fma(xi[u], xj0[v], part[u][v]);
                    part[u][v + 4] = fma(xi[u], xj1[v], part[u][v + 4]);
                }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int v = 0; v < 8; ++v) acc[u][v] += part[u][v];
        __syncthreads();
    }
    // per-warp partials -> S (fixed order), R = I
    T* const Pw = sm.work + warp * B2 * B2;
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 8; ++v) Pw[(ti * 4 + u) * B2 + tj * 8 + v] = acc[u][v];
    __syncthreads();
    for (int e = t; e < B2 * B2; e += NT) {
        const int i = e / B2, j = e % B2;
        T s = sm.work[e];
#pragma unroll
        for (int w = 1; w < NW; ++w) s += sm.work[w * B2 * B2 + e];
        sm.S[i][j] = s;
        sm.R[i][j] = (i == j) ? T(1) : T(0);
    }
    __syncthreads();

    // ---- 2. convergence measure before rotating: how much the rotation this
    //      pair still needs could change J = U max(Sigma - tau, 0) V^T,
    //      relative to the largest singular value.  For columns of norms a, b
    //      an unresolved rotation of tangent t moves J by about t |f(a) - f(b)|
    //      (f(s) = max(s - tau, 0) is 1-Lipschitz, so |a - b| bounds it), plus
    //      tau theta when both lie above tau (the pair then enters J as
    //      A - tau U V^T and theta = |s_ij| / (a b) is its angle defect).
    //      Pairs with a^2 + b^2 <= tau^2 have every singular value below tau
    //      and are removed by the SVT whatever their rotation; columns below
    //      the rounding floor (~4 eps of the largest) are noise and skipped.  A
    //      `strict` matrix (the block whose kept left singular subspace the C
    //      step projects onto) also needs that subspace itself: pairs that
    //      straddle tau are measured by t alone.
    const T noise = T(4) * num<T>::eps();
    const T floor2 = noise * noise * (*d.scale) + num<T>::tiny();
    const T tau = d.mu ? (T)(1.0 / *d.mu) : T(0);
    const T tau2 = tau * tau;
    const T smax = sqrt(*d.scale);
    const T inv_smax = T(1) / (smax + num<T>::tiny());
    T offm = T(0);
    for (int e = t; e < B2 * B2; e += NT) {
        const int i = e % B2, j = e / B2;
        const T sii = sm.S[i][i], sjj = sm.S[j][j];
        if (i < j && sii > floor2 && sjj > floor2 && sii + sjj > tau2) {
            const T sij = fabs(sm.S[i][j]);
            const T na = sqrt(sii), nb = sqrt(sjj);
            const T hd = T(0.5) * fabs(sii - sjj);
            const T tn = sij / (hd + sqrt(hd * hd + sij * sij) + num<T>::tiny());
            T mm;
            if (na > tau && nb > tau) mm = tn * fabs(na - nb) + tau * sij / (na * nb);
            else if (na > tau || nb > tau) mm = d.strict ? tn * (*d.scale > 0 ? smax : T(1)) : tn * fabs(na - nb);
            else mm = tn * (sqrt(sii + sjj) - tau);
            offm = fmax(offm, mm * inv_smax);
        }
    }
    offm = warp_max(offm);
    if (lane == 0) sm.red[warp] = offm;
    __syncthreads();
    T mx = T(0);
#pragma unroll
    for (int w = 0; w < NW; ++w) mx = fmax(mx, sm.red[w]);
    // a pivot already orthogonal to a few eps needs no rotation (4 eps in
    // float32: on data with one dominant singular value the measure, relative
    // to the largest column, must resolve pairs well below it)
    if (mx <= (sizeof(T) == 4 ? T(4) : T(16)) * num<T>::eps()) return mx;

    // ---- 3. rotate the pivot Gram towards diagonal form (all threads of the
    //      CTA): one inner sweep in float32; in float64 up to four, where
    //      rotations that only mix noise columns do not keep the sweeps going
    const int rot = inner_jacobi<T, B2, NT, LO>(sm.S, sm.R, sm.cs, sm.sn, sm.pi, sm.qi, num<T>::tiny(), floor2,
                                                inner_sweeps<T>(),
                                                sizeof(T) == 4 ? T(3e-4) : T(0));
    if (!rot) return mx;

    // R is a product of some hundred plane rotations, orthogonal only to
    // ~sqrt(count) eps; one Newton-Schulz step R <- R (3I - R^T R)/2 restores
    // orthogonality to ~eps^2 before R touches X and W (applied to graded
    // columns the defect would mix eps-sized parts of the large columns into
    // the small ones)
    T* const G = sm.work;                     // R^T R, stride LO
    T* const R4 = sm.work + LO * B2;          // R - I, stride B2 (16-byte rows)
    constexpr int PE = B2 * B2 / NT;
#pragma unroll
    for (int u = 0; u < PE; ++u) {
        const int e = t + u * NT, i = e % B2, j = e / B2;
        T g = T(0);
#pragma unroll 8
        for (int k = 0; k < B2; ++k) g = fma(sm.R[k][i], sm.R[k][j], g);
        G[i * LO + j] = g;
    }
    __syncthreads();
    T y[PE];
#pragma unroll
    for (int u = 0; u < PE; ++u) {
        const int e = t + u * NT, i = e % B2, j = e / B2;
        T s = T(0);
#pragma unroll 8
        for (int k = 0; k < B2; ++k) s = fma(sm.R[i][k], G[k * LO + j], s);
        y[u] = s;
    }
    __syncthreads();
    // the rotation is applied in update form, x_j <- x_j + sum_k x_k (R - I)_kj:
    // once the sweeps have converged R - I is tiny and so is the rounding it
    // adds, instead of a fresh eps |x| at every application
#pragma unroll
    for (int u = 0; u < PE; ++u) {
        const int e = t + u * NT, i = e % B2, j = e / B2;
        const T rn = T(1.5) * sm.R[i][j] - T(0.5) * y[u];
        R4[i * B2 + j] = rn - (i == j ? T(1) : T(0));
    }
    __syncthreads();

    // ---- 4. X_P <- X_P R and W_P <- W_P R: one row per lane, the 32 pivot
    //      columns of that row in registers, rows of R - I read by broadcast
    for (int pass = 0; pass < 2; ++pass) {
        T* base = pass == 0 ? d.X : d.W;
        const int64_t ld = pass == 0 ? d.ldx : d.ldw;
        const int rows = pass == 0 ? d.L : d.p;
        for (int r0 = warp * 32; r0 < rows; r0 += NT) {
            const int row = r0 + lane;
            const bool ok = row < rows;
            T x[B2];
#pragma unroll
            for (int k = 0; k < B2; ++k) {
                const int gc = pcol(k, a, c);
                x[k] = (ok && gc < d.p) ? __ldcg(base + row + (int64_t)gc * ld) : T(0);
            }
            // outputs in groups of OW columns (fewer live registers for float64)
            constexpr int OW = 8;
#pragma unroll
            for (int half = 0; half < B2 / OW; ++half) {
                T o[OW];
#pragma unroll
                for (int v = 0; v < OW; ++v) o[v] = T(0);
#pragma unroll
                for (int k = 0; k < B2; ++k) {
                    T rk[OW];
#pragma unroll
                    for (int q = 0; q < OW / 4; ++q) {
                        T v4[4];
                        lds4(R4 + k * B2 + half * OW + q * 4, v4);
#pragma unroll
                        for (int z = 0; z < 4; ++z) rk[q * 4 + z] = v4[z];
                    }
#pragma unroll
                    for (int v = 0; v < OW; ++v) o[v] = fma(x[k], rk[v], o[v]);
                }
#pragma unroll
                for (int v = 0; v < OW; ++v) {
                    const int j = half * OW + v;
                    const int gc = pcol(j, a, c);
                    if (ok && gc < d.p) base[row + (int64_t)gc * ld] = x[j] + o[v];
                }
            }
        }
    }
    __syncthreads();
    return mx;
}

// One cluster per matrix (blockIdx.y); the cluster's CTAs share the pivots of
// each round.  `off` holds three slots per matrix (one per sweep, reused every
// third sweep), `done` is set when the matrix converged.
// With `quad_exit`, a sweep whose measure o (taken before its rotations)
// satisfies 16 o^2 <= tol ends the loop without a confirming sweep: cyclic
// Jacobi converges quadratically near the end (the off-diagonal part after a
// sweep is O(o^2)), so the rotations of that sweep already bring the matrix
// below the tolerance.
template <typename T>
__global__ void __launch_bounds__(NT, 5) osj_svd(const OsjDesc<T>* __restrict__ descs, int sweeps, T tol,
                                              int* __restrict__ sweeps_run, int quad_exit) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Smem<T>& sm = *reinterpret_cast<Smem<T>*>(smem_raw);
    const int mat = blockIdx.y;
    const OsjDesc<T> d = descs[mat];
    if (d.active && *d.active == 0) return;     // uniform over the cluster
    cg::cluster_group cl = cg::this_cluster();
    const int rank = (int)cl.block_rank(), csize = (int)cl.num_blocks();
    const int nb = d.pp / OB, npairs = nb / 2;
    const int t = threadIdx.x;
    if (rank == 0 && t == 0) {
        d.off[0] = T(0); d.off[1] = T(0); d.off[2] = T(0);
        *d.done = 0;
        if (d.ctr) { atomicExch(d.ctr, 0); atomicExch(d.ctr + 1, 0); }
    }
    // scaled off-diagonals below ~64 eps are at the rounding level of the
    // fresh pivot Grams
    const T t_eff = fmax(tol, T(64) * num<T>::eps());
    cl.sync();
    int R = 0;        // rounds run so far (selects the counter of the round)
    for (int sw = 0; sw < sweeps; ++sw) {
        T mine = T(0);
        for (int r = 0; r < nb - 1; ++r, ++R) {
            if (d.ctr) {
                // pivots go to whichever CTA of the cluster is free: a pivot
                // that rotates costs several times one that is already
                // orthogonal.  Counter R & 1 serves this round; the other one,
                // last used in the previous round (finished at the cluster
                // barrier), is reset for the next.
                if (rank == 0 && t == 0) {
                    atomicExch(d.ctr + ((R + 1) & 1), 0);
                    __threadfence();
                }
            }
            for (int k = 0;; ++k) {
                int P = rank + k * csize;          // fixed share without a counter
                if (d.ctr) {
                    if (t == 0) sm.pick = atomicAdd(d.ctr + (R & 1), 1);
                    __syncthreads();
                    P = sm.pick;
                    __syncthreads();
                }
                if (P >= npairs) break;
                const int a = circle_item(P, r, nb), c = circle_item(nb - 1 - P, r, nb);
                mine = fmax(mine, osj_pivot<T>(d, sm, a, c));
            }
            cl.sync();
        }
        if (t == 0) {
            atomic_max_nonneg(d.off + sw % 3, mine);
            if (rank == 0) d.off[(sw + 1) % 3] = T(0);
        }
        cl.sync();
        const T o = __ldcg(d.off + sw % 3);
        if (rank == 0 && t == 0 && sweeps_run) sweeps_run[mat] += 1;
        if (o <= t_eff || (quad_exit && T(16) * o * o <= t_eff)) {
            if (rank == 0 && t == 0) *d.done = 1;
            break;
        }
    }
}

}  // namespace

template <typename T>
int osj_max_cluster() {
    // 16 (the non-portable limit) when the device schedules clusters that
    // large for this kernel, else 8
    static std::atomic<int> big_ok{-1};
    if (big_ok.load() < 0) {
        int ok = 0;
        const size_t smem = sizeof(Smem<T>);
        static std::atomic<uint64_t> smem_set{0};
        if (ensure_smem_limit(osj_svd<T>, (int)smem, smem_set) == cudaSuccess &&
            cudaFuncSetAttribute(osj_svd<T>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) == cudaSuccess) {
            cudaLaunchConfig_t cfg = {};
            cfg.gridDim = dim3(16, 1, 1);
            cfg.blockDim = dim3(NT, 1, 1);
            cfg.dynamicSmemBytes = smem;
            cudaLaunchAttribute at;
            at.id = cudaLaunchAttributeClusterDimension;
            at.val.clusterDim.x = 16; at.val.clusterDim.y = 1; at.val.clusterDim.z = 1;
            cfg.attrs = &at;
            cfg.numAttrs = 1;
            int nclus = 0;
            if (cudaOccupancyMaxActiveClusters(&nclus, osj_svd<T>, &cfg) == cudaSuccess && nclus > 0) ok = 1;
        }
        (void)cudaGetLastError();
        big_ok.store(ok);
    }
    return big_ok.load() ? 16 : 8;
}

template <typename T>
int default_cluster(int nmat, int max_pairs, int cmax, size_t smem) {
    int best = 1;
    for (int c = std::min(cmax, std::max(1, max_pairs)); c >= 1; c /= 2) {
        if (c > 8 && cudaFuncSetAttribute(osj_svd<T>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess)
            continue;
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((unsigned)c, 1, 1);
        cfg.blockDim = dim3(NT, 1, 1);
        cfg.dynamicSmemBytes = smem;
        cudaLaunchAttribute at;
        at.id = cudaLaunchAttributeClusterDimension;
        at.val.clusterDim.x = (unsigned)c; at.val.clusterDim.y = 1; at.val.clusterDim.z = 1;
        cfg.attrs = &at;
        cfg.numAttrs = 1;
        int nclus = 0;
        if (cudaOccupancyMaxActiveClusters(&nclus, osj_svd<T>, &cfg) == cudaSuccess && nclus >= nmat) {
            best = c;
            break;
        }
        best = c;
    }
    (void)cudaGetLastError();
    return best;
}

template <typename T>
cudaError_t osj_sweeps(const OsjDesc<T>* d_desc, int nmat, int max_pp, int sweeps, T tol, int* sweeps_run,
                       cudaStream_t s, int cluster, int quad_exit) {
    if (nmat <= 0 || max_pp <= 0 || sweeps <= 0) return cudaSuccess;
    const int max_pairs = max_pp / B2;
    const size_t smem = sizeof(Smem<T>);
    static std::atomic<uint64_t> smem_set{0};
    cudaError_t e = ensure_smem_limit(osj_svd<T>, (int)smem, smem_set);
    if (e != cudaSuccess) return e;
    // cluster size: the caller's choice (autotuned), else the largest (up to
    // one CTA per pivot of a round) at which every block's cluster can be
    // resident at once -- a block waiting for a second wave would double the
    // time of the whole batch
    const int cmax = osj_max_cluster<T>();
    int csize = cluster > 0 ? std::min(cluster, cmax) : default_cluster<T>(nmat, max_pairs, cmax, smem);
    csize = std::max(1, std::min(csize, max_pairs));
    if (csize > 8) {
        e = cudaFuncSetAttribute(osj_svd<T>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (e != cudaSuccess) return e;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)csize, (unsigned)nmat, 1);
    cfg.blockDim = dim3(NT, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at;
    at.id = cudaLaunchAttributeClusterDimension;
    at.val.clusterDim.x = (unsigned)csize; at.val.clusterDim.y = 1; at.val.clusterDim.z = 1;
    cfg.attrs = &at;
    cfg.numAttrs = 1;
    e = cudaLaunchKernelEx(&cfg, osj_svd<T>, d_desc, sweeps, tol, sweeps_run, quad_exit);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

template cudaError_t osj_sweeps<float>(const OsjDesc<float>*, int, int, int, float, int*, cudaStream_t, int, int);
template cudaError_t osj_sweeps<double>(const OsjDesc<double>*, int, int, int, double, int*, cudaStream_t, int, int);
template int osj_max_cluster<float>();
template int osj_max_cluster<double>();

}  // namespace lrr
