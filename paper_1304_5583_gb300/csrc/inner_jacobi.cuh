// Cyclic Jacobi on one small symmetric matrix held in shared memory, shared by
// the two-sided eigensolver (jacobi.cu) and the one-sided SVT solver (osj.cu).
#pragma once
#include "common.cuh"

namespace lrr {

// item at position `pos` of round `r` in the circle-method schedule of N items:
// every round pairs position k with N-1-k, and N-1 rounds pair every two items once
__device__ __forceinline__ int circle_item(int pos, int r, int N) {
    return pos == 0 ? 0 : 1 + ((pos - 1 + r) % (N - 1));
}

// Tangent of the classical Jacobi rotation that annihilates s_pq:
// tan(2 theta) = 2 s_pq / (s_qq - s_pp), the root of smaller magnitude.
template <typename T>
__device__ __forceinline__ void jacobi_rotation(T app, T aqq, T apq, T& cc, T& ss) {
    const T theta = (aqq - app) / (T(2) * apq);
    T tt;
    if (fabs(theta) > T(1) / num<T>::eps()) tt = T(0.5) / theta;
    else tt = (theta >= T(0) ? T(1) : T(-1)) / (fabs(theta) + sqrt(theta * theta + T(1)));
    cc = T(1) / sqrt(tt * tt + T(1));
    ss = tt * cc;
}
// float: the hardware reciprocal and reciprocal square root.  The rotations
// only steer the pivot towards diagonal form: the accumulated rotation is
// re-orthonormalised before it touches the columns, and the next sweep forms
// its Grams afresh, so a few ulps in c and s cost no accuracy, while the
// shorter dependent chain shortens every step of the inner sweep.
template <>
__device__ __forceinline__ void jacobi_rotation<float>(float app, float aqq, float apq, float& cc, float& ss) {
    const float theta = __fdividef(aqq - app, 2.f * apq);
    float tt;
    if (fabsf(theta) > 1.f / FLT_EPSILON) {
        tt = __fdividef(0.5f, theta);
    } else {
        const float h = fmaf(theta, theta, 1.f);
        tt = copysignf(__fdividef(1.f, fabsf(theta) + h * rsqrtf(h)), theta);
    }
    cc = rsqrtf(fmaf(tt, tt, 1.f));
    ss = tt * cc;
}

// Diagonalises S (B2 x B2, row stride LDS) in place by classical Jacobi
// rotations (angle from tan(2 theta) = 2 s_pq / (s_qq - s_pp)), B2/2 disjoint
// rotations per parallel step, accumulating the rotations into R (R <- R J, R
// must hold the identity on entry).  An entry is rotated while
// |s_pq| > eps * sqrt(|s_pp s_qq|) and |s_pq| > floor_rot; sweeps stop after one
// in which no rotation of an entry above floor_sig had |tan| > exit_tan, or
// after max_sweeps.  Returns nonzero (block-uniform) if any rotation was applied.
template <typename T, int B2, int NT, int LDS = B2 + 1>
__device__ int inner_jacobi(T (*S)[LDS], T (*R)[LDS], T* cs, T* sn, int* pi, int* qi, T floor_rot,
                            T floor_sig, int max_sweeps, T exit_tan = T(0)) {
    constexpr int b = B2 / 2;
    const int t = threadIdx.x;
    int rotated_total = 0;
    for (int sweep = 0; sweep < max_sweeps; ++sweep) {
        int rotated = 0, rotated_sig = 0;
        for (int r = 0; r < B2 - 1; ++r) {
            if (t < b) {
                const int p = circle_item(t, r, B2), q = circle_item(B2 - 1 - t, r, B2);
                const T app = S[p][p], aqq = S[q][q], apq = S[p][q];
                T cc = T(1), ss = T(0);
                if (fabs(apq) > floor_rot && fabs(apq) > num<T>::eps() * sqrt(fabs(app * aqq))) {
                    jacobi_rotation<T>(app, aqq, apq, cc, ss);
                    rotated = 1;
                    if (fabs(apq) > floor_sig && fabs(ss) > exit_tan * cc) rotated_sig = 1;
                }
                cs[t] = cc; sn[t] = ss; pi[t] = p; qi[t] = q;
            }
            __syncthreads();
            // S <- J^T S J on every 2x2 sub-block (p_k,q_k) x (p_l,q_l) at once
            for (int e = t; e < b * b; e += NT) {
                const int k = e % b, l = e / b;
                const int p = pi[k], q = qi[k], u = pi[l], v = qi[l];
                const T ck = cs[k], sk = sn[k], cl = cs[l], sl = sn[l];
                const T s_pu = S[p][u], s_pv = S[p][v], s_qu = S[q][u], s_qv = S[q][v];
                const T r_pu = ck * s_pu - sk * s_qu, r_pv = ck * s_pv - sk * s_qv;
                const T r_qu = sk * s_pu + ck * s_qu, r_qv = sk * s_pv + ck * s_qv;
                // the rotated pair's own off-diagonal entries are zero by
                // construction (k == l: u = p, v = q); only this thread
                // touches them in this step
                const bool own = k == l && sk != T(0);
                S[p][u] = cl * r_pu - sl * r_pv;
                S[p][v] = own ? T(0) : sl * r_pu + cl * r_pv;
                S[q][u] = own ? T(0) : cl * r_qu - sl * r_qv;
                S[q][v] = sl * r_qu + cl * r_qv;
            }
            // R <- R J
            for (int e = t; e < B2 * b; e += NT) {
                const int i = e % B2, l = e / B2;
                const int u = pi[l], v = qi[l];
                const T cl = cs[l], sl = sn[l];
                const T x = R[i][u], y = R[i][v];
                R[i][u] = cl * x - sl * y;
                R[i][v] = sl * x + cl * y;
            }
            __syncthreads();
        }
        rotated_total |= rotated;
        if (!__syncthreads_or(rotated_sig)) break;
    }
    return __syncthreads_or(rotated_total);
}

}  // namespace lrr
