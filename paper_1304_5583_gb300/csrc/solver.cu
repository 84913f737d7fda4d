// DFC-LRR solver: host orchestration and the C ABI declared in dfc_lrr.h.
//
// Flow of one call (Algorithm 1, Section 2.2):
//   checks            -> non-finite scan of M, partition validation
//   one-time factor   -> K = M M^T (float64), block-Jacobi eigendecomposition
//                        K = U diag(sigma^2) U^T, rank r, V = M^T U diag(1/sigma).
//                        This factors I + M^T M = V diag(1+sigma^2) V^T + (I - V V^T)
//                        once for every block, because all blocks share the
//                        dictionary M (eq. (2)).
//   F step            -> the t block problems advance together: every launch
//                        covers all still-active blocks (per-block penalty mu_i,
//                        stop flag and iteration count); `batched = 0` runs the
//                        same kernels on one block at a time.
//   C step            -> column projection onto the column space of Z_1
//                        (orthonormal basis of J_1's factored form), then the
//                        D-step permutation is undone while writing Z and S.
#include <algorithm>
#include <chrono>
#include <cstring>
#include <numeric>
#include <type_traits>
#include <map>
#include <mutex>
#include <numeric>
#include <tuple>
#include <vector>

#include "dfc_lrr.h"
#include "alm_kernels.cuh"
#include "common.cuh"
#include "kernels.cuh"

namespace lrr {
namespace {

constexpr size_t kAlign = 256;

struct Arena {
    char* base;
    size_t off = 0;
    explicit Arena(void* b) : base(static_cast<char*>(b)) {}
    template <typename X>
    X* take(size_t count) {
        off = (off + kAlign - 1) / kAlign * kAlign;
        X* p = base ? reinterpret_cast<X*>(base + off) : nullptr;
        off += std::max<size_t>(count, 1) * sizeof(X);
        return p;
    }
};

inline int round_up(int x, int q) { return (x + q - 1) / q * q; }

// widest n the tensor-core products take (65535 column tiles of 128)
constexpr int64_t kTcMaxN = 65535LL * 128;

bool valid_problem(const lrr_problem* p, const lrr_options* o) {
    if (!p || !o || !p->M || !p->perm || !p->offsets) return false;
    if (p->m < 1 || p->n < 1 || p->ldm < p->m || p->t < 1 || p->t > p->n) return false;
    if (p->m > (1 << 20) || p->n > (1 << 24)) return false;
    if (p->offsets[0] != 0 || p->offsets[p->t] != p->n) return false;
    for (int i = 0; i < p->t; ++i)
        if (p->offsets[i + 1] <= p->offsets[i]) return false;
    std::vector<char> seen((size_t)p->n, 0);
    for (int64_t j = 0; j < p->n; ++j) {
        const int64_t c = p->perm[j];
        if (c < 0 || c >= p->n || seen[(size_t)c]) return false;
        seen[(size_t)c] = 1;
    }
    if (!(o->lambda > 0) || !(o->rho > 1) || !(o->mu0 > 0) || !(o->mu_max >= o->mu0) || !(o->eps > 0)) return false;
    if (o->max_iter < 1) return false;
    if (o->precision < LRR_PREC_F64 || o->precision > LRR_PREC_MIXED) return false;
    return true;
}

template <typename T>
struct BlockInfo {
    int64_t col0;
    int l, pmax, ppmax;
};

// Every device array of one solve, carved from the workspace.
template <typename T>
struct Buffers {
    int64_t m, n;
    int t, rmax, mpp;
    // one-time factor (float64)
    double *Md, *Kd, *Wd, *Rd, *Dd, *lam_raw, *lam, *Ud, *Usd, *Vd;
    double *jac_off_d, *jac_scale_d;
    int *jac_done_d, *order;
    JacDesc<double>* jac_setup;
    // float32 start of the factor: K and its eigenvectors in float32, then
    // float64 scratch for the polish from that basis
    float *Kf, *Wf, *Rf, *jac_off_f, *jac_scale_f;
    int *rot_f, *jac_done_f;
    JacDesc<float>* jac_setup_f;
    double *T1d, *T2d;
    // factor in the iteration precision
    T *U, *US, *sig, *dinv, *V, *nu;
    // state (m x n) and reduced state (rmax x n)
    T *C, *P, *MZ, *E, *Y1;       // C holds C_perp = C - U U^T C; P holds Q = Y1/mu - E; MZ holds U (Theta - sigma Z)
    T *Zt, *Jt, *Y2t, *A, *D, *Tt, *Theta;
    double *Thd, *Cpd;
    // per block
    std::vector<T*> G, W, H, R, h, T1;
    std::vector<int*> rot;
    int* rot_d;
    double *mu, *mu_fin, *resid;
    int *act, *iters, *svt_on, *rank_cur, *rank_fin, *need_exact, *conv_bound, *conv, *jdone, *jctr, *colblk, *flag;
    T *r1, *dmax, *r2x, *jscale, *joff;
    int64_t* perm;
    // descriptor / pointer tables
    GemmDesc<T>* gd;       // 12 * t descriptors
    OsjDesc<T>* jd;
    double* afro;
    int* jsweeps;
    int* svtcalls;
    T** Gp;
    T** hp;
    T** Wp;
    T** Hp;
    T** T1p;
    int *pv, *ppv;
    // mixed precision: split bf16 (hi, lo) K-major operands of the
    // tensor-core products
    int64_t ldm8, ldr8;
    uint16_t *Ubf, *USbf, *Pbf, *Zbf, *Ubf_lo, *USbf_lo, *Pbf_lo, *Zbf_lo;
    int *fp32_on, *gemm32, *tc_err;
    // float32 products on the tensor cores (split TF32): U and U^T split once,
    // P = Y1/mu - E and Delta split by the kernels that produce them
    int64_t m4, r4;
    float *Uh, *Ul, *UTh, *UTl, *Ph, *Pl, *Dh, *Dl;
    // float32 iteration: bf16 V (K-major) and D for the tensor-core stage of the stop test
    uint16_t *Vbf, *Dbf;
    unsigned* bmax;
    int *tc_dec, *any_need, *need_cnt;
    // C step
    int *kept, *kept_n;
    double *Fd, *Gk, *Yd;
    T *Q, *Wc;
};

template <typename T>
Buffers<T> carve(Arena& a, const lrr_problem* p, bool need_md, const std::vector<BlockInfo<T>>& blk, bool mixed,
                 bool tc32) {
    Buffers<T> b{};
    b.m = p->m;
    b.n = p->n;
    b.t = p->t;
    b.rmax = (int)std::min<int64_t>(p->m, p->n);
    constexpr int B2d = 2 * jacobi_bs<double>();
    constexpr int B2f = 2 * jacobi_bs<float>();
    static_assert(B2f % B2d == 0, "padding serves both precisions");
    constexpr int B2 = osj_pivot_width();
    b.mpp = round_up((int)p->m, B2f);
    const int64_t m = p->m, n = p->n, r = b.rmax, mpp = b.mpp;
    b.Md = need_md ? a.take<double>(m * n) : nullptr;
    b.Kd = a.take<double>(mpp * mpp);
    b.Wd = a.take<double>(mpp * mpp);
    b.Rd = a.take<double>(mpp * B2d);
    b.lam_raw = a.take<double>(m);
    b.lam = a.take<double>(m);
    b.order = a.take<int>(m);
    b.Ud = a.take<double>(m * r);
    b.Usd = a.take<double>(m * r);
    b.Vd = a.take<double>(n * r);
    b.jac_off_d = a.take<double>(1);
    b.jac_scale_d = a.take<double>(1);
    b.jac_done_d = a.take<int>(1);
    b.jac_setup = a.take<JacDesc<double>>(1);
    b.Kf = a.take<float>(mpp * mpp);
    b.Wf = a.take<float>(mpp * mpp);
    b.Rf = a.take<float>(mpp * B2f);
    b.rot_f = a.take<int>(mpp / B2f);
    b.jac_off_f = a.take<float>(1);
    b.jac_scale_f = a.take<float>(1);
    b.jac_done_f = a.take<int>(1);
    b.jac_setup_f = a.take<JacDesc<float>>(1);
    b.T1d = a.take<double>(mpp * mpp);
    b.T2d = a.take<double>(mpp * mpp);
    b.U = a.take<T>(m * r);
    b.US = a.take<T>(m * r);
    b.sig = a.take<T>(r);
    b.dinv = a.take<T>(r);
    b.V = a.take<T>(n * r);
    b.nu = a.take<T>(1);
    b.C = a.take<T>(m * n);
    b.P = a.take<T>(m * n);
    b.MZ = a.take<T>(m * n);
    b.E = a.take<T>(m * n);
    b.Y1 = a.take<T>(m * n);
    b.Zt = a.take<T>(r * n);
    b.Jt = a.take<T>(r * n);
    b.Y2t = a.take<T>(r * n);
    b.A = a.take<T>(r * n);
    b.D = a.take<T>(r * n);
    b.Tt = a.take<T>(r * n);
    b.Theta = a.take<T>(r * n);
    b.Thd = a.take<double>(r * n);
    b.Cpd = a.take<double>(m * n);
    const int t = p->t;
    b.G.resize(t); b.W.resize(t); b.H.resize(t); b.R.resize(t); b.h.resize(t); b.T1.resize(t); b.rot.resize(t);
    b.rot_d = a.take<int>(mpp / B2d);
    for (int i = 0; i < t; ++i) {
        const int64_t pp = blk[i].ppmax;
        b.W[i] = a.take<T>(pp * pp);
        b.H[i] = a.take<T>(pp * pp);
        b.T1[i] = a.take<T>(pp * pp);
        b.R[i] = a.take<T>(pp * B2);
        b.h[i] = a.take<T>(pp);
        b.rot[i] = a.take<int>(pp / B2);
    }
    b.mu = a.take<double>(t);
    b.mu_fin = a.take<double>(t);
    b.resid = a.take<double>(2 * t);
    b.act = a.take<int>(t);
    b.iters = a.take<int>(t);
    b.svt_on = a.take<int>(t);
    b.rank_cur = a.take<int>(t);
    b.rank_fin = a.take<int>(t);
    b.need_exact = a.take<int>(t);
    b.conv_bound = a.take<int>(t);
    b.conv = a.take<int>(t);
    b.jdone = a.take<int>(t);
    b.jctr = a.take<int>(2 * (size_t)t);
    b.colblk = a.take<int>(n);
    b.flag = a.take<int>(4);
    b.r1 = a.take<T>(t);
    b.dmax = a.take<T>(t);
    b.r2x = a.take<T>(t);
    b.jscale = a.take<T>(t);
    b.joff = a.take<T>(3 * (size_t)t);   // three convergence slots per block
    b.perm = a.take<int64_t>(n);
    b.gd = a.take<GemmDesc<T>>(16 * (size_t)t + 16);
    b.jd = a.take<OsjDesc<T>>(t);
    b.afro = a.take<double>(t);
    b.jsweeps = a.take<int>(t);
    b.svtcalls = a.take<int>(t);
    b.Gp = a.take<T*>(t);
    b.hp = a.take<T*>(t);
    b.Wp = a.take<T*>(t);
    b.Hp = a.take<T*>(t);
    b.T1p = a.take<T*>(t);
    b.pv = a.take<int>(t);
    b.ppv = a.take<int>(t);
    const int64_t p0 = blk[0].ppmax;
    b.kept = a.take<int>(p0);
    b.kept_n = a.take<int>(1);
    b.Fd = a.take<double>(r * p0);
    b.Gk = a.take<double>(p0 * p0);
    b.Yd = a.take<double>(r * p0);
    b.Q = a.take<T>(r * p0);
    b.Wc = a.take<T>(p0 * n);
    b.ldm8 = (m + 7) / 8 * 8;
    b.ldr8 = (r + 7) / 8 * 8;
    b.Ubf = mixed ? a.take<uint16_t>(r * b.ldm8) : nullptr;
    b.USbf = mixed ? a.take<uint16_t>(m * b.ldr8) : nullptr;
    b.Pbf = mixed ? a.take<uint16_t>(n * b.ldm8) : nullptr;
    b.Zbf = mixed ? a.take<uint16_t>(n * b.ldr8) : nullptr;
    b.Ubf_lo = mixed ? a.take<uint16_t>(r * b.ldm8) : nullptr;
    b.USbf_lo = mixed ? a.take<uint16_t>(m * b.ldr8) : nullptr;
    b.Pbf_lo = mixed ? a.take<uint16_t>(n * b.ldm8) : nullptr;
    b.Zbf_lo = mixed ? a.take<uint16_t>(n * b.ldr8) : nullptr;
    b.m4 = (m + 3) / 4 * 4;
    b.r4 = (r + 3) / 4 * 4;
    b.Uh = tc32 ? a.take<float>(b.m4 * r) : nullptr;
    b.Ul = tc32 ? a.take<float>(b.m4 * r) : nullptr;
    b.UTh = tc32 ? a.take<float>(b.r4 * m) : nullptr;
    b.UTl = tc32 ? a.take<float>(b.r4 * m) : nullptr;
    b.Ph = tc32 ? a.take<float>(b.m4 * n) : nullptr;
    b.Pl = tc32 ? a.take<float>(b.m4 * n) : nullptr;
    b.Dh = tc32 ? a.take<float>(b.r4 * n) : nullptr;
    b.Dl = tc32 ? a.take<float>(b.r4 * n) : nullptr;
    b.fp32_on = a.take<int>(t);
    b.gemm32 = a.take<int>(t);
    b.tc_err = a.take<int>(1);
    // (the tensor-core product's grid covers n in 128-column tiles, at most 65535 of them)
    const bool tc_stop = std::is_same<T, float>::value && n <= kTcMaxN;
    b.Vbf = tc_stop ? a.take<uint16_t>(n * b.ldr8) : nullptr;
    b.Dbf = tc_stop ? a.take<uint16_t>(n * b.ldr8) : nullptr;
    b.bmax = tc_stop ? a.take<unsigned>(t) : nullptr;
    b.tc_dec = tc_stop ? a.take<int>(t) : nullptr;
    b.any_need = tc_stop ? a.take<int>(1) : nullptr;
    b.need_cnt = tc_stop ? a.take<int>(1) : nullptr;
    return b;
}

template <typename T>
std::vector<BlockInfo<T>> block_info(const lrr_problem* p) {
    constexpr int B2 = osj_pivot_width();
    const int rmax = (int)std::min<int64_t>(p->m, p->n);
    std::vector<BlockInfo<T>> v((size_t)p->t);
    for (int i = 0; i < p->t; ++i) {
        v[i].col0 = p->offsets[i];
        v[i].l = (int)(p->offsets[i + 1] - p->offsets[i]);
        v[i].pmax = std::min(rmax, v[i].l);
        v[i].ppmax = round_up(v[i].pmax, B2);
    }
    return v;
}

inline unsigned grid1(int64_t count, int threads = 256) {
    return (unsigned)std::min<int64_t>((count + threads - 1) / threads, 152 * 32);
}

// Per-phase CUDA-event timing on the solve's stream plus launch counting.
struct Prof {
    bool on = false;
    cudaStream_t s = nullptr;
    double ms[LRR_NPHASE] = {};
    int64_t calls[LRR_NPHASE] = {};
    int64_t launches = 0, iterations = 0;
    std::vector<cudaEvent_t> free_ev;
    std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> pending;
    cudaEvent_t open_ev = nullptr;
    cudaEvent_t get() {
        if (!free_ev.empty()) { cudaEvent_t e = free_ev.back(); free_ev.pop_back(); return e; }
        cudaEvent_t e = nullptr;
        cudaEventCreate(&e);
        return e;
    }
    void begin() {
        if (!on) return;
        open_ev = get();
        cudaEventRecord(open_ev, s);
    }
    void end(int ph, int64_t nlaunch) {
        launches += nlaunch;
        calls[ph] += nlaunch;
        if (!on || !open_ev) return;
        cudaEvent_t e = get();
        cudaEventRecord(e, s);
        pending.push_back({ph, {open_ev, e}});
        open_ev = nullptr;
    }
    // after a stream synchronisation: fold the recorded pairs into ms[]
    void flush() {
        for (auto& p : pending) {
            float t = 0.f;
            if (cudaEventElapsedTime(&t, p.second.first, p.second.second) == cudaSuccess) ms[p.first] += t;
            free_ev.push_back(p.second.first);
            free_ev.push_back(p.second.second);
        }
        pending.clear();
    }
    ~Prof() {
        for (auto& p : pending) { cudaEventDestroy(p.second.first); cudaEventDestroy(p.second.second); }
        for (auto e : free_ev) cudaEventDestroy(e);
    }
};

template <typename T>
GemmDesc<T> gdesc(const T* A, int64_t lda, const T* B, int64_t ldb, T* C, int64_t ldc, int m, int n, int k,
                  const int* flag, T alpha = T(1), T beta = T(0)) {
    GemmDesc<T> d{};
    d.A = A; d.B = B; d.C = C; d.flag = flag; d.ccol = nullptr; d.kscale = nullptr; d.absmax = nullptr;
    d.lda = lda; d.ldb = ldb; d.ldc = ldc; d.m = m; d.n = n; d.k = k; d.alpha = alpha; d.beta = beta;
    return d;
}

// A set of grouped-GEMM launches prepared once per solve.
template <typename T>
struct GemmSet {
    int first = 0, count = 0, max_m = 0, max_n = 0;
    bool ta = false, tb = false;
};

// ---- autotuner: launch shape of the batched Jacobi (cluster size per block),
// picked by timing the candidates on synthetic input of the problem's block
// shapes the first time a shape is solved; cached per process and device.
struct TuneKey {
    int dev, prec;
    int64_t m, n, r;
    int t, max_pp;
    bool operator<(const TuneKey& o) const {
        return std::tie(dev, prec, m, n, r, t, max_pp) < std::tie(o.dev, o.prec, o.m, o.n, o.r, o.t, o.max_pp);
    }
};
std::mutex g_tune_mutex;
std::map<TuneKey, int> g_tune_cluster;

// Jacobi sweep tolerance of the iteration (scaled off-diagonal)
template <typename T>
constexpr T jtol_of() { return sizeof(T) == 8 ? T(1e-13) : T(2e-6); }

// float32 products on the tensor cores in split TF32, on request only
// (lrr_options.tc_products; float32 iteration; the grid covers n in 128-column
// tiles, at most 65535 of them)
template <typename T>
bool use_tc32(const lrr_problem* p, const lrr_options* o) {
    return std::is_same<T, float>::value && o->precision != LRR_PREC_F64 && o->tc_products && p->n <= kTcMaxN;
}

template <typename T, typename Tin>
int solve_impl(const lrr_problem* p, const lrr_options* o, void* ws, size_t ws_bytes, lrr_result* res,
               cudaStream_t s, bool dfc) {
    const auto blk = block_info<T>(p);
    const bool need_md = !std::is_same<Tin, double>::value;
    Arena probe(nullptr);
    const bool mixed = o->precision == LRR_PREC_MIXED;
    if (mixed && p->n > kTcMaxN) return LRR_ERR_UNSUPPORTED;
    const bool tc32 = use_tc32<T>(p, o);
    carve<T>(probe, p, need_md, blk, mixed, tc32);
    const size_t need = probe.off + kAlign;
    void* own = nullptr;
    if (!ws) {
        if (cudaMallocAsync(&own, need, s) != cudaSuccess) return LRR_ERR_CUDA;
        ws = own;
        ws_bytes = need;
    }
    struct Free {
        void* p; cudaStream_t s;
        ~Free() { if (p) cudaFreeAsync(p, s); }
    } guard{own, s};
    if (ws_bytes < need - kAlign || (reinterpret_cast<uintptr_t>(ws) % kAlign) != 0) return LRR_ERR_WORKSPACE;
    Arena arena(ws);
    Buffers<T> B = carve<T>(arena, p, need_md, blk, mixed, tc32);
    const int64_t m = p->m, n = p->n;
    const int t = p->t;
    const Tin* M = static_cast<const Tin*>(p->M);

    Prof prof;
    prof.on = o->profile != 0;
    prof.s = s;
    cudaEvent_t ev[4];
    for (auto& e : ev) LRR_CUDA_TRY(cudaEventCreate(&e));
    struct EvFree {
        cudaEvent_t* e;
        ~EvFree() { for (int i = 0; i < 4; ++i) cudaEventDestroy(e[i]); }
    } evguard{ev};
    LRR_CUDA_TRY(cudaEventRecord(ev[0], s));

    // ---- checks: non-finite entries
    int hflag = 0;
    LRR_CUDA_TRY(cudaMemsetAsync(B.flag, 0, sizeof(int) * 4, s));
    k::nonfinite_check<Tin><<<dim3(grid1(m), (unsigned)std::min<int64_t>(n, 65535)), 256, 0, s>>>(M, p->ldm, m, n, B.flag);
    LRR_CUDA_TRY(cudaMemcpyAsync(&hflag, B.flag, sizeof(int), cudaMemcpyDeviceToHost, s));
    LRR_CUDA_TRY(cudaStreamSynchronize(s));
    if (hflag) return LRR_ERR_NONFINITE;

    // ---- D step inputs
    std::vector<int> colblk((size_t)n);
    for (int i = 0; i < t; ++i)
        for (int64_t j = p->offsets[i]; j < p->offsets[i + 1]; ++j) colblk[(size_t)j] = i;
    LRR_CUDA_TRY(cudaMemcpyAsync(B.perm, p->perm, sizeof(int64_t) * n, cudaMemcpyHostToDevice, s));
    LRR_CUDA_TRY(cudaMemcpyAsync(B.colblk, colblk.data(), sizeof(int) * n, cudaMemcpyHostToDevice, s));

    // ---- one-time factor in float64
    const double* Md = nullptr;
    int64_t ldmd = p->ldm;
    if (need_md) {
        k::gather_cols<double, Tin><<<dim3(grid1(m), (unsigned)std::min<int64_t>(n, 65535)), 256, 0, s>>>(M, p->ldm, nullptr, m, n, B.Md);
        Md = B.Md;
        ldmd = m;
    } else {
        Md = reinterpret_cast<const double*>(M);
    }
    std::vector<GemmDesc<double>> hd(3);
    int setup_sweeps[2] = {0, 0};     // float32 and float64 Jacobi sweeps of the factor
    hd[0] = gdesc<double>(Md, ldmd, Md, ldmd, B.Kd, B.mpp, (int)m, (int)m, (int)n, nullptr);
    GemmDesc<double>* dd = reinterpret_cast<GemmDesc<double>*>(B.gd);  // scratch slot, reused below
    LRR_CUDA_TRY(cudaMemcpyAsync(dd, hd.data(), sizeof(GemmDesc<double>), cudaMemcpyHostToDevice, s));
    k::init_padded<double><<<grid1((int64_t)B.mpp * B.mpp), 256, 0, s>>>(B.Kd, (int)m, B.mpp, -1.0, 0);
    k::init_padded<double><<<grid1((int64_t)B.mpp * B.mpp), 256, 0, s>>>(B.Wd, (int)m, B.mpp, 1.0, 1);
    LRR_CUDA_TRY(gemm_grouped<double>(dd, 1, false, true, (int)m, (int)m, s));
    {
        // scale for the Jacobi noise floor: max diagonal of K
        k::diag_of<double><<<ceil_div(m, 256), 256, 0, s>>>(B.Kd, B.mpp, m, B.lam_raw);
        std::vector<double> dg((size_t)m);
        LRR_CUDA_TRY(cudaMemcpyAsync(dg.data(), B.lam_raw, sizeof(double) * m, cudaMemcpyDeviceToHost, s));
        LRR_CUDA_TRY(cudaStreamSynchronize(s));
        double sc = 0;
        for (double v : dg) sc = std::max(sc, std::fabs(v));
        if (!(sc > 0)) return LRR_ERR_RANK;
        // The eigendecomposition starts in float32 and is finished in float64:
        //   1. K_f = float(K), block Jacobi in float32 -> eigenvectors U0
        //      (orthogonal to ~1e-6, the large eigenpairs already resolved);
        //   2. U0 in float64, made orthonormal to float64 rounding by two
        //      Newton-Schulz steps U0 <- U0 (3I - U0^T U0)/2 (quadratic from a
        //      1e-6 defect);
        //   3. K' = U0^T K U0 in float64 is nearly diagonal; the float64 block
        //      Jacobi on K' converges in a few sweeps to K' = W diag(lambda) W^T;
        //   4. the eigenvectors of K are U0 W.
        // The float64 sweeps decide the accuracy (same tolerance as a float64
        // start); the float32 start only removes the sweeps that float64 would
        // spend on the large rotations.
        const int64_t mp = B.mpp, mm = mp * mp;
        k::copy_convert_f64<float><<<grid1(mm), 256, 0, s>>>(B.Kd, B.Kf, mm);
        k::init_padded<float><<<grid1(mm), 256, 0, s>>>(B.Wf, (int)m, (int)mp, 1.f, 1);
        const float scf = (float)sc;
        JacDesc<float> jf{};
        jf.G = B.Kf; jf.W = B.Wf; jf.R = B.Rf; jf.rot = B.rot_f; jf.done = B.jac_done_f; jf.off = B.jac_off_f;
        jf.active = nullptr; jf.scale = B.jac_scale_f; jf.pp = (int)mp;
        LRR_CUDA_TRY(cudaMemcpyAsync(B.jac_scale_f, &scf, sizeof(float), cudaMemcpyHostToDevice, s));
        LRR_CUDA_TRY(cudaMemcpyAsync(B.jac_setup_f, &jf, sizeof(jf), cudaMemcpyHostToDevice, s));
        LRR_CUDA_TRY(jacobi_sweeps<float>(B.jac_setup_f, 1, (int)mp, 40, 1e-5f, s, B.jac_done_f, &setup_sweeps[0]));
        double* U0 = B.T2d;
        double* G1 = B.T1d;
        k::copy_convert_to_f64<float><<<grid1(mm), 256, 0, s>>>(B.Wf, U0, mm);
        auto gemm1 = [&](const double* A, const double* Bm, double* C, bool ta, double alpha, double beta) {
            GemmDesc<double> g = gdesc<double>(A, mp, Bm, mp, C, mp, (int)mp, (int)mp, (int)mp, nullptr, alpha, beta);
            cudaError_t e = cudaMemcpyAsync(dd, &g, sizeof(g), cudaMemcpyHostToDevice, s);
            if (e == cudaSuccess) e = gemm_grouped<double>(dd, 1, ta, false, (int)mp, (int)mp, s);
            return e;
        };
        for (int it = 0; it < 2; ++it) {
            // G1 = U0^T U0;  Wd = 1.5 U0 - 0.5 U0 G1;  U0 <- Wd
            LRR_CUDA_TRY(gemm1(U0, U0, G1, true, 1.0, 0.0));
            LRR_CUDA_TRY(cudaMemcpyAsync(B.Wd, U0, sizeof(double) * mm, cudaMemcpyDeviceToDevice, s));
            LRR_CUDA_TRY(gemm1(U0, G1, B.Wd, false, -0.5, 1.5));
            LRR_CUDA_TRY(cudaMemcpyAsync(U0, B.Wd, sizeof(double) * mm, cudaMemcpyDeviceToDevice, s));
        }
        // K' = U0^T (K U0), in place of K
        LRR_CUDA_TRY(gemm1(B.Kd, U0, G1, false, 1.0, 0.0));
        LRR_CUDA_TRY(gemm1(U0, G1, B.Kd, true, 1.0, 0.0));
        k::init_padded<double><<<grid1(mm), 256, 0, s>>>(B.Wd, (int)m, (int)mp, 1.0, 1);
        JacDesc<double> jd{};
        jd.G = B.Kd; jd.W = B.Wd; jd.R = B.Rd; jd.rot = B.rot_d; jd.done = B.jac_done_d; jd.off = B.jac_off_d;
        jd.active = nullptr; jd.scale = B.jac_scale_d; jd.pp = (int)mp;
        LRR_CUDA_TRY(cudaMemcpyAsync(B.jac_scale_d, &sc, sizeof(double), cudaMemcpyHostToDevice, s));
        LRR_CUDA_TRY(cudaMemcpyAsync(B.jac_setup, &jd, sizeof(jd), cudaMemcpyHostToDevice, s));
        LRR_CUDA_TRY(jacobi_sweeps<double>(B.jac_setup, 1, (int)mp, 40, 1e-13, s, B.jac_done_d, &setup_sweeps[1]));
        // eigenvectors of K: U0 W
        LRR_CUDA_TRY(gemm1(U0, B.Wd, G1, false, 1.0, 0.0));
        LRR_CUDA_TRY(cudaMemcpyAsync(B.Wd, G1, sizeof(double) * mm, cudaMemcpyDeviceToDevice, s));
    }
    k::diag_of<double><<<ceil_div(m, 256), 256, 0, s>>>(B.Kd, B.mpp, m, B.lam_raw);
    std::vector<double> ev_h((size_t)m);
    LRR_CUDA_TRY(cudaMemcpyAsync(ev_h.data(), B.lam_raw, sizeof(double) * m, cudaMemcpyDeviceToHost, s));
    LRR_CUDA_TRY(cudaStreamSynchronize(s));
    std::vector<int> order((size_t)m);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return ev_h[a] > ev_h[b]; });
    const double smax = std::sqrt(std::max(ev_h[order[0]], 0.0));
    const double rtol = o->rank_tol > 0 ? o->rank_tol : 1e-6;
    int r = 0;
    while (r < (int)m && r < B.rmax && std::sqrt(std::max(ev_h[order[r]], 0.0)) > rtol * smax) ++r;
    if (r == 0 || !(smax > 0)) return LRR_ERR_RANK;
    std::vector<double> lam_sorted((size_t)r);
    for (int k2 = 0; k2 < r; ++k2) lam_sorted[k2] = ev_h[order[k2]];
    LRR_CUDA_TRY(cudaMemcpyAsync(B.order, order.data(), sizeof(int) * r, cudaMemcpyHostToDevice, s));
    LRR_CUDA_TRY(cudaMemcpyAsync(B.lam, lam_sorted.data(), sizeof(double) * r, cudaMemcpyHostToDevice, s));
    k::setup_factors<<<dim3(grid1(m), (unsigned)r), 256, 0, s>>>(B.Wd, B.mpp, m, r, B.order, B.lam, B.Ud, B.Usd);
    k::setup_scalars<T><<<dim3(grid1(m), (unsigned)r), 256, 0, s>>>(B.lam, r, B.Ud, m, B.sig, B.dinv, B.U, B.US);
    if (mixed) {
        k::to_bf16_split_km<T><<<dim3(grid1(B.ldm8), (unsigned)r), 256, 0, s>>>(B.U, m, m, r, B.Ubf, B.Ubf_lo,
                                                                               B.ldm8);
        k::to_bf16_split_transposed<T><<<dim3(grid1(B.ldr8), (unsigned)std::min<int64_t>(m, 65535)), 256, 0, s>>>(
            B.U, m, m, r, B.USbf, B.USbf_lo, B.ldr8);
    }
    if constexpr (std::is_same<T, float>::value) {
        if (tc32) {
            // A operands of U^T P (U itself, K = m) and of U Delta (U^T, K = r)
            k::split_tf32_km<T><<<dim3(grid1(B.m4), (unsigned)r), 256, 0, s>>>(B.U, m, m, r, B.Uh, B.Ul, B.m4);
            k::split_tf32_transposed<T><<<dim3(grid1(B.r4), (unsigned)std::min<int64_t>(m, 65535)), 256, 0, s>>>(
                B.U, m, m, r, B.UTh, B.UTl, B.r4);
            LRR_CUDA_TRY(cudaMemsetAsync(B.Ph, 0, sizeof(float) * B.m4 * n, s));
            LRR_CUDA_TRY(cudaMemsetAsync(B.Pl, 0, sizeof(float) * B.m4 * n, s));
        }
    }
    hd[1] = gdesc<double>(Md, ldmd, B.Usd, m, B.Vd, n, (int)n, r, (int)m, nullptr);
    LRR_CUDA_TRY(cudaMemcpyAsync(dd + 1, &hd[1], sizeof(GemmDesc<double>), cudaMemcpyHostToDevice, s));
    LRR_CUDA_TRY(gemm_grouped<double>(dd + 1, 1, true, false, (int)n, r, s));
    k::copy_convert_f64<T><<<grid1(n * r), 256, 0, s>>>(B.Vd, B.V, n * r);
    if (B.Vbf)
        k::to_bf16_transposed<T><<<dim3(grid1(B.ldr8), (unsigned)std::min<int64_t>(n, 65535)), 256, 0, s>>>(
            B.V, n, n, r, B.Vbf, B.ldr8);
    // reduced coordinates of the observations, Theta = U^T C = diag(sigma) V[perm, :]^T,
    // and the part of C outside range(U), C_perp = C - U Theta (zero when r = m):
    // the iteration then forms U^T (Y1/mu - E) and C - M Z = C_perp + U (Theta - sigma Z)
    // as products of small differences instead of differences of large products
    LRR_CUDA_TRY(cudaMemcpyAsync(B.perm, p->perm, sizeof(int64_t) * n, cudaMemcpyHostToDevice, s));
    k::theta_from_v<T><<<dim3(grid1(n), (unsigned)r), 256, 0, s>>>(B.Vd, n, B.lam, B.perm, r, B.Theta, B.Thd);
    const bool has_perp = r < (int)m;
    if (has_perp) {
        // C_perp = M[:, perm] - U Theta in float64, then to the iteration precision
        k::gather_cols<double, Tin><<<dim3(grid1(m), (unsigned)std::min<int64_t>(n, 65535)), 256, 0, s>>>(
            M, p->ldm, B.perm, m, n, B.Cpd);
        hd[2] = gdesc<double>(B.Ud, m, B.Thd, r, B.Cpd, m, (int)m, (int)n, r, nullptr, -1.0, 1.0);
        LRR_CUDA_TRY(cudaMemcpyAsync(dd + 2, &hd[2], sizeof(GemmDesc<double>), cudaMemcpyHostToDevice, s));
        LRR_CUDA_TRY(gemm_grouped<double>(dd + 2, 1, false, false, (int)m, (int)n, s));
        k::copy_convert_f64<T><<<grid1(m * n), 256, 0, s>>>(B.Cpd, B.C, m * n);
    }
    LRR_CUDA_TRY(cudaMemsetAsync(B.nu, 0, sizeof(T), s));
    k::row_norm_max<T><<<ceil_div(n, 256), 256, 0, s>>>(B.V, n, r, B.nu);
    T nu_h = T(0);
    LRR_CUDA_TRY(cudaMemcpyAsync(&nu_h, B.nu, sizeof(T), cudaMemcpyDeviceToHost, s));
    LRR_CUDA_TRY(cudaStreamSynchronize(s));
    LRR_CUDA_TRY(cudaEventRecord(ev[1], s));
    {
        const int64_t nbd = B.mpp / jacobi_bs<double>(), nbf = B.mpp / jacobi_bs<float>();
        const int64_t jac_launches_setup = (1 + setup_sweeps[0] * (2 * (nbf - 1) + 1)) +
                                           (1 + setup_sweeps[1] * (2 * (nbd - 1) + 1));
        // checks, gather, K, init x2, diag, float32 start (convert, init, copy
        // back), 2 x 2 Newton-Schulz products, K' (2), init, U0 W, diag, factors
        const int64_t setup_launches = 1 + (need_md ? 1 : 0) + 1 + 2 + 1 + 3 + 4 + 2 + 1 + 1 + 1 + 2 +
                                       jac_launches_setup + 1 + 1 + 1;
        prof.launches += setup_launches;
        prof.calls[LRR_PH_SETUP] += setup_launches;
    }

    // ---- per-block tables (sizes now known: p_i = min(r, l_i))
    constexpr int B2 = osj_pivot_width();
    std::vector<int> pv((size_t)t), ppv((size_t)t);
    std::vector<char> tall((size_t)t);
    int max_p = 0, max_pp = 0, max_l = 0;
    for (int i = 0; i < t; ++i) {
        tall[i] = blk[i].l <= r;
        pv[i] = std::min(r, blk[i].l);
        ppv[i] = round_up(pv[i], B2);
        max_p = std::max(max_p, pv[i]);
        max_pp = std::max(max_pp, ppv[i]);
        max_l = std::max(max_l, blk[i].l);
    }
    LRR_CUDA_TRY(cudaMemcpyAsync(B.hp, B.h.data(), sizeof(T*) * t, cudaMemcpyHostToDevice, s));
    LRR_CUDA_TRY(cudaMemcpyAsync(B.Wp, B.W.data(), sizeof(T*) * t, cudaMemcpyHostToDevice, s));
    LRR_CUDA_TRY(cudaMemcpyAsync(B.Hp, B.H.data(), sizeof(T*) * t, cudaMemcpyHostToDevice, s));
    LRR_CUDA_TRY(cudaMemcpyAsync(B.T1p, B.T1.data(), sizeof(T*) * t, cudaMemcpyHostToDevice, s));
    LRR_CUDA_TRY(cudaMemcpyAsync(B.pv, pv.data(), sizeof(int) * t, cudaMemcpyHostToDevice, s));
    LRR_CUDA_TRY(cudaMemcpyAsync(B.ppv, ppv.data(), sizeof(int) * t, cudaMemcpyHostToDevice, s));
    std::vector<OsjDesc<T>> jdh((size_t)t);
    for (int i = 0; i < t; ++i) {
        OsjDesc<T>& j = jdh[i];
        j.X = B.D + blk[i].col0 * r;
        j.ldx = tall[i] ? r : blk[i].l;
        j.L = tall[i] ? r : blk[i].l;
        j.W = B.W[i]; j.ldw = ppv[i]; j.p = pv[i]; j.pp = ppv[i];
        j.done = B.jdone + i; j.off = B.joff + 3 * i; j.active = B.svt_on + i; j.scale = B.jscale + i;
        j.ctr = B.jctr + 2 * i;
        j.mu = B.mu + i;
        j.strict = (dfc && t > 1 && i == 0) ? 1 : 0;
    }
    LRR_CUDA_TRY(cudaMemcpyAsync(B.jd, jdh.data(), sizeof(OsjDesc<T>) * t, cudaMemcpyHostToDevice, s));
    // the float32 Jacobi stops without its confirming sweep once quadratic
    // convergence guarantees the tolerance; float64 keeps the confirming sweep
    const int quad_exit = sizeof(T) == 4 ? 1 : 0;

    // ---- autotune the Jacobi's cluster size (before the state is initialised:
    //      it runs on synthetic columns in the SVT buffers, then clears them)
    int jcluster = 0;
    if (o->autotune) {
        int dev = 0;
        LRR_CUDA_TRY(cudaGetDevice(&dev));
        const TuneKey key{dev, o->precision, m, n, r, t, max_pp};
        bool have = false;
        {
            std::lock_guard<std::mutex> lk(g_tune_mutex);
            auto it = g_tune_cluster.find(key);
            if (it != g_tune_cluster.end()) { jcluster = it->second; have = true; }
        }
        if (!have) {
            std::vector<int> cand;
            const int max_pairs = max_pp / B2, cmax = osj_max_cluster<T>();
            for (int c : {4, 8, 16})
                if (c <= cmax && (c <= max_pairs || cand.empty())) cand.push_back(std::min(c, max_pairs));
            std::vector<int> on((size_t)t, 1);
            std::vector<double> mu_t((size_t)t, 1e10);
            LRR_CUDA_TRY(cudaMemcpyAsync(B.svt_on, on.data(), sizeof(int) * t, cudaMemcpyHostToDevice, s));
            LRR_CUDA_TRY(cudaMemcpyAsync(B.mu, mu_t.data(), sizeof(double) * t, cudaMemcpyHostToDevice, s));
            cudaEvent_t ta, tb;
            LRR_CUDA_TRY(cudaEventCreate(&ta));
            LRR_CUDA_TRY(cudaEventCreate(&tb));
            float best = 1e30f;
            for (int c : cand) {
                k::fill_hash<T><<<grid1(r * n), 256, 0, s>>>(B.D, r * n, 12345u);
                for (int i = 0; i < t; ++i)
                    k::init_padded<T><<<grid1((int64_t)ppv[i] * ppv[i]), 256, 0, s>>>(B.W[i], pv[i], ppv[i], T(1), 1);
                k::col_norm_max<T><<<t, 256, 0, s>>>(B.jd, B.svt_on, B.jscale, t);
                cudaEventRecord(ta, s);
                const cudaError_t e = osj_sweeps<T>(B.jd, t, max_pp, 2, jtol_of<T>(), nullptr, s, c, quad_exit);
                cudaEventRecord(tb, s);
                if (e != cudaSuccess || cudaEventSynchronize(tb) != cudaSuccess) {
                    cudaEventDestroy(ta); cudaEventDestroy(tb);
                    return LRR_ERR_CUDA;
                }
                float ms = 0.f;
                cudaEventElapsedTime(&ms, ta, tb);
                if (ms < best) { best = ms; jcluster = c; }
            }
            cudaEventDestroy(ta);
            cudaEventDestroy(tb);
            std::lock_guard<std::mutex> lk(g_tune_mutex);
            g_tune_cluster[key] = jcluster;
        }
    }

    // grouped GEMM descriptor sets
    std::vector<GemmDesc<T>> gh;
    std::vector<GemmSet<T>> sets;
    auto add_set = [&](bool ta, bool tb, const std::vector<GemmDesc<T>>& ds) {
        GemmSet<T> g;
        g.first = (int)gh.size(); g.count = (int)ds.size(); g.ta = ta; g.tb = tb;
        for (auto& d : ds) { g.max_m = std::max(g.max_m, d.m); g.max_n = std::max(g.max_n, d.n); gh.push_back(d); }
        sets.push_back(g);
        return (int)sets.size() - 1;
    };
    std::vector<GemmDesc<T>> xw_tall, xw_wide, jmul, tmul, mzmul, exact, orth1, orth2;
    for (int i = 0; i < t; ++i) {
        const int64_t c0 = blk[i].col0;
        const int l = blk[i].l, pp_ = ppv[i], pi = pv[i];
        T* Ai = B.A + c0 * r;
        // X = A W (tall) or A^T W (wide): A rotated into the previous right
        // basis; the one-sided Jacobi then finishes orthogonalising its columns
        T* Xi = B.D + c0 * r;
        if (tall[i]) {
            xw_tall.push_back(gdesc<T>(Ai, r, B.W[i], pp_, Xi, r, r, l, l, B.svt_on + i));
            // J = X diag(h) W^{-1}:  A = X W^{-1}, so this keeps the kept directions only
            GemmDesc<T> jd_ = gdesc<T>(Xi, r, B.T1[i], pp_, B.Jt + c0 * r, r, r, l, l, B.act + i);
            jd_.kscale = B.h[i];
            jmul.push_back(jd_);
        } else {
            xw_wide.push_back(gdesc<T>(Ai, r, B.W[i], pp_, Xi, l, l, r, r, B.svt_on + i));
            // J = W^{-T} diag(h) X^T:  A^T = X W^{-1}
            GemmDesc<T> jd_ = gdesc<T>(B.T1[i], pp_, Xi, l, B.Jt + c0 * r, r, r, l, r, B.act + i);
            jd_.kscale = B.h[i];
            jmul.push_back(jd_);
        }
        orth1.push_back(gdesc<T>(B.W[i], pp_, B.W[i], pp_, B.T1[i], pp_, pi, pi, pi, B.svt_on + i));
        orth2.push_back(gdesc<T>(B.W[i], pp_, B.T1[i], pp_, B.H[i], pp_, pi, pi, pi, B.svt_on + i));
        tmul.push_back(gdesc<T>(B.U, m, B.P + c0 * m, m, B.Tt + c0 * r, r, r, l, (int)m, B.gemm32 + i));
        mzmul.push_back(gdesc<T>(B.U, m, B.Tt + c0 * r, r, B.MZ + c0 * m, m, (int)m, l, r, B.gemm32 + i));
        GemmDesc<T> ex = gdesc<T>(B.V, n, B.D + c0 * r, r, nullptr, 0, (int)n, l, r, B.need_exact + i);
        ex.absmax = B.r2x + i;
        exact.push_back(ex);
    }
    const int S_XT = xw_tall.empty() ? -1 : add_set(false, false, xw_tall);
    const int S_XW = xw_wide.empty() ? -1 : add_set(true, false, xw_wide);
    const int S_J = add_set(false, true, jmul);
    const int S_T = add_set(true, false, tmul);
    const int S_MZ = add_set(false, false, mzmul);
    const int S_EX = add_set(false, false, exact);
    const int S_O1 = add_set(true, false, orth1);
    const int S_O2 = add_set(false, false, orth2);
    if (gh.size() + 10 > 16 * (size_t)t + 16) return LRR_ERR_INVALID;
    LRR_CUDA_TRY(cudaMemcpyAsync(B.gd, gh.data(), sizeof(GemmDesc<T>) * gh.size(), cudaMemcpyHostToDevice, s));
    auto run_set = [&](int si) -> cudaError_t {
        if (si < 0) return cudaSuccess;
        const GemmSet<T>& g = sets[si];
        return gemm_grouped<T>(B.gd + g.first, g.count, g.ta, g.tb, g.max_m, g.max_n, s);
    };

    // ---- state
    prof.launches += 1 + (int64_t)t;
    prof.calls[LRR_PH_SETUP] += 1 + (int64_t)t;
    LRR_CUDA_TRY(cudaMemsetAsync(B.P, 0, sizeof(T) * m * n, s));
    LRR_CUDA_TRY(cudaMemsetAsync(B.E, 0, sizeof(T) * m * n, s));
    LRR_CUDA_TRY(cudaMemsetAsync(B.Y1, 0, sizeof(T) * m * n, s));
    {
        T* zs[5] = {B.Zt, B.Jt, B.Y2t, B.A, B.D};
        for (T* x : zs) { LRR_CUDA_TRY(cudaMemsetAsync(x, 0, sizeof(T) * r * n, s)); }
    }
    for (int i = 0; i < t; ++i)
        k::init_padded<T><<<grid1((int64_t)ppv[i] * ppv[i]), 256, 0, s>>>(B.W[i], pv[i], ppv[i], T(1), 1);
    LRR_CUDA_TRY(cudaMemsetAsync(B.afro, 0, sizeof(double) * t, s));
    if (B.bmax) {
        LRR_CUDA_TRY(cudaMemsetAsync(B.bmax, 0, sizeof(unsigned) * t, s));
        LRR_CUDA_TRY(cudaMemsetAsync(B.tc_dec, 0, sizeof(int) * t, s));
        LRR_CUDA_TRY(cudaMemsetAsync(B.any_need, 0, sizeof(int), s));
        LRR_CUDA_TRY(cudaMemsetAsync(B.need_cnt, 0, sizeof(int), s));
    }
    {
        // mixed: every block starts on the bf16 tensor-core products (fp32_on = 0)
        std::vector<int> f32init((size_t)t, mixed ? 0 : 1);
        LRR_CUDA_TRY(cudaMemcpyAsync(B.fp32_on, f32init.data(), sizeof(int) * t, cudaMemcpyHostToDevice, s));
        LRR_CUDA_TRY(cudaMemsetAsync(B.tc_err, 0, sizeof(int), s));
        if (mixed) {
            LRR_CUDA_TRY(cudaMemsetAsync(B.Pbf, 0, sizeof(uint16_t) * n * B.ldm8, s));
            LRR_CUDA_TRY(cudaMemsetAsync(B.Zbf, 0, sizeof(uint16_t) * n * B.ldr8, s));
            LRR_CUDA_TRY(cudaMemsetAsync(B.Pbf_lo, 0, sizeof(uint16_t) * n * B.ldm8, s));
            LRR_CUDA_TRY(cudaMemsetAsync(B.Zbf_lo, 0, sizeof(uint16_t) * n * B.ldr8, s));
        }
    }
    for (int i = 0; i < t; ++i)   // the SVT reconstruction reads it with zero weights before the first SVD
        LRR_CUDA_TRY(cudaMemsetAsync(B.T1[i], 0, sizeof(T) * (size_t)ppv[i] * ppv[i], s));
    LRR_CUDA_TRY(cudaMemsetAsync(B.jsweeps, 0, sizeof(int) * t, s));
    LRR_CUDA_TRY(cudaMemsetAsync(B.svtcalls, 0, sizeof(int) * t, s));
    std::vector<double> mu0((size_t)t, o->mu0);
    LRR_CUDA_TRY(cudaMemcpyAsync(B.mu, mu0.data(), sizeof(double) * t, cudaMemcpyHostToDevice, s));
    LRR_CUDA_TRY(cudaMemcpyAsync(B.mu_fin, mu0.data(), sizeof(double) * t, cudaMemcpyHostToDevice, s));
    {
        int* zi[7] = {B.iters, B.conv, B.rank_cur, B.rank_fin, B.svt_on, B.need_exact, B.conv_bound};
        for (int* x : zi) { LRR_CUDA_TRY(cudaMemsetAsync(x, 0, sizeof(int) * t, s)); }
        T* zt[3] = {B.r1, B.dmax, B.r2x};
        for (T* x : zt) { LRR_CUDA_TRY(cudaMemsetAsync(x, 0, sizeof(T) * t, s)); }
    }
    LRR_CUDA_TRY(cudaMemsetAsync(B.resid, 0, sizeof(double) * 2 * t, s));

    const int sweeps = o->jacobi_sweeps > 0 ? o->jacobi_sweeps : 12;
    // mixed: a block leaves the bf16 products once ||A||_F > margin * tau, i.e.
    // just before its SVT starts to act (J = 0 up to then)
    const double switch_margin = mixed ? (o->mixed_switch > 0 ? o->mixed_switch : 0.5) : 0.0;
    bool bf16_phase = mixed;
    const T jtol = jtol_of<T>();
    const unsigned wgrid_n = (unsigned)((n * 32 + 255) / 256);
    auto nl = [&](int si) -> int64_t { return si < 0 ? 0 : 1; };
    const int64_t jac_launches = 1;   // every sweep of every block in one launch
    // relative error bound of the bf16 stop-test product (stop_tc_decide), with a factor-2 margin
    const double tc_rel = 2.0 * (2.0 / 256.0 + 1.0 / 65536.0 + (double)r / 16777216.0);
    // the tensor-core stage of the stop test runs in chunks that follow one in
    // which some block needed ||V D||_inf (its empty launches are not free)
    bool tc_window = false;
    auto iteration = [&]() -> int {
        prof.iterations += 1;
        // J-step: SVT of A = Zt + Y2t/mu through the Gram eigendecomposition
        prof.begin();
        k::svt_gate<T><<<ceil_div(t, 128), 128, 0, s>>>(B.act, B.afro, B.mu, B.svt_on, B.jscale, B.svtcalls,
                                                         B.fp32_on, B.gemm32, switch_margin, t);
        LRR_CUDA_TRY(run_set(S_XT));
        LRR_CUDA_TRY(run_set(S_XW));
        prof.end(LRR_PH_GRAM, 1 + nl(S_XT) + nl(S_XW));
        prof.begin();
        k::col_norm_max<T><<<t, 256, 0, s>>>(B.jd, B.svt_on, B.jscale, t);
        LRR_CUDA_TRY(osj_sweeps<T>(B.jd, t, max_pp, sweeps, jtol, B.jsweeps, s, jcluster, quad_exit));
        prof.end(LRR_PH_JACOBI, jac_launches + 1);
        prof.begin();
        k::svt_weights<T><<<t, 256, 0, s>>>(B.jd, B.hp, B.act, B.svt_on, B.mu, B.rank_cur, t);
        // W^T W and W (W^T W): first-order inverse for J, Newton-Schulz for the warm start
        LRR_CUDA_TRY(run_set(S_O1));
        LRR_CUDA_TRY(run_set(S_O2));
        k::ns_orth<T><<<dim3(64, (unsigned)t), 256, 0, s>>>(B.Wp, B.Hp, B.T1p, B.pv, B.ppv, B.svt_on, t);
        LRR_CUDA_TRY(run_set(S_J));
        prof.end(LRR_PH_SVT_APPLY, 5);
        // Z-step
        prof.begin();
        if constexpr (std::is_same<T, float>::value) {
            if (bf16_phase) {
                // all columns at once; blocks already in float32 are recomputed below
                LRR_CUDA_TRY(tc_gemm_bf16x3(B.Ubf, B.Ubf_lo, B.ldm8, B.Pbf, B.Pbf_lo, B.ldm8, B.Tt, r, r, (int)n,
                                            (int)m, B.tc_err, s));
            }
        }
        if (tc32) {
            // float32-accurate U^T P on the tensor cores for the blocks past the bf16 phase
            LRR_CUDA_TRY(tc_gemm_3xtf32(B.Uh, B.Ul, B.m4, B.Ph, B.Pl, B.m4, reinterpret_cast<float*>(B.Tt), r, r,
                                        (int)n, (int)m, B.colblk, B.gemm32, B.tc_err, s));
        } else {
            LRR_CUDA_TRY(run_set(S_T));
        }
        prof.end(LRR_PH_ZGEMM, bf16_phase ? 2 : 1);
        prof.begin();
        k::z_update<T><<<wgrid_n, 256, 0, s>>>(r, n, B.colblk, B.act, B.mu, o->rho, o->mu_max, B.Tt, B.Theta, B.Jt,
                                               B.Y2t, B.Zt, B.D, B.A, B.sig, B.dinv, B.dmax, B.afro,
                                               bf16_phase ? B.Zbf : nullptr, B.Zbf_lo, B.ldr8, tc32 ? B.Dh : nullptr,
                                               tc32 ? B.Dl : nullptr, B.r4);
        prof.end(LRR_PH_ZUPDATE, 1);
        // E-step, residuals, duals
        prof.begin();
        if constexpr (std::is_same<T, float>::value) {
            if (bf16_phase)
                LRR_CUDA_TRY(tc_gemm_bf16x3(B.USbf, B.USbf_lo, B.ldr8, B.Zbf, B.Zbf_lo, B.ldr8, B.MZ, m, (int)m,
                                            (int)n, r, B.tc_err, s));
        }
        if (tc32) {
            LRR_CUDA_TRY(tc_gemm_3xtf32(B.UTh, B.UTl, B.r4, B.Dh, B.Dl, B.r4, reinterpret_cast<float*>(B.MZ), m,
                                        (int)m, (int)n, r, B.colblk, B.gemm32, B.tc_err, s));
        } else {
            LRR_CUDA_TRY(run_set(S_MZ));
        }
        prof.end(LRR_PH_MZGEMM, bf16_phase ? 2 : 1);
        prof.begin();
        k::e_update<T><<<wgrid_n, 256, 0, s>>>(m, n, B.colblk, B.act, B.mu, o->rho, o->mu_max, o->lambda,
                                               has_perp ? B.C : nullptr, B.MZ, B.Y1, B.E, B.P, B.r1,
                                               bf16_phase ? B.Pbf : nullptr, B.Pbf_lo, B.ldm8, tc32 ? B.Ph : nullptr,
                                               tc32 ? B.Pl : nullptr, B.m4);
        prof.end(LRR_PH_EUPDATE, 1);
        prof.begin();
        k::stop_part1<T><<<ceil_div(t, 128), 128, 0, s>>>(t, B.act, B.r1, B.dmax, nu_h, 1.0 / std::sqrt((double)n), o->eps, B.need_exact,
                                                          B.conv_bound, B.any_need, B.need_cnt);
        const bool tc_stage = B.bmax && tc_window;
        if (tc_stage) {
            // ||V D||_inf from bf16 operands on the tensor cores first; the float32
            // product below then runs only for blocks that value cannot decide
            k::d_to_bf16_needed<T><<<dim3(grid1(r), (unsigned)std::min<int64_t>(n, 4096)), 256, 0, s>>>(
                B.D, r, r, n, B.colblk, B.need_exact, B.any_need, B.Dbf, B.ldr8);
            LRR_CUDA_TRY(tc_gemm_bf16_absmax(B.Vbf, B.ldr8, B.Dbf, B.ldr8, (int)n, (int)n, r,
                                             TcAbsmax{B.any_need, B.colblk, B.need_exact, B.bmax}, B.tc_err, s));
            k::stop_tc_decide<T><<<ceil_div(t, 128), 128, 0, s>>>(t, B.need_exact, B.conv_bound, B.bmax, B.dmax, nu_h,
                                                                 o->eps, tc_rel, B.tc_dec, B.r2x);
        }
        LRR_CUDA_TRY(run_set(S_EX));
        k::stop_part2<T><<<ceil_div(t, 128), 128, 0, s>>>(t, B.act, B.iters, B.mu, o->rho, o->mu_max, o->eps,
                                                          o->max_iter, B.r1, B.dmax, B.r2x, B.need_exact,
                                                          B.conv_bound, nu_h, B.resid, B.rank_cur, B.rank_fin,
                                                          B.conv, B.mu_fin, B.afro, B.tc_dec, B.bmax, B.any_need);
        prof.end(LRR_PH_STOP, tc_stage ? 6 : 3);
        LRR_CUDA_TRY(cudaGetLastError());
        return LRR_OK;
    };
    auto run_loop = [&](const std::vector<int>& act0) -> int {
        LRR_CUDA_TRY(cudaMemcpyAsync(B.act, act0.data(), sizeof(int) * t, cudaMemcpyHostToDevice, s));
        std::vector<int> ah((size_t)t), fh((size_t)t);
        int done_it = 0, nneed = 0;
        const int chunk = 4;
        tc_window = false;
        while (done_it < o->max_iter) {
            for (int c = 0; c < chunk && done_it < o->max_iter; ++c, ++done_it) {
                const int rc = iteration();
                if (rc != LRR_OK) return rc;
            }
            prof.begin();
            LRR_CUDA_TRY(cudaMemcpyAsync(ah.data(), B.act, sizeof(int) * t, cudaMemcpyDeviceToHost, s));
            if (bf16_phase) LRR_CUDA_TRY(cudaMemcpyAsync(fh.data(), B.fp32_on, sizeof(int) * t, cudaMemcpyDeviceToHost, s));
            if (B.need_cnt) LRR_CUDA_TRY(cudaMemcpyAsync(&nneed, B.need_cnt, sizeof(int), cudaMemcpyDeviceToHost, s));
            prof.end(LRR_PH_HOST, 0);
            LRR_CUDA_TRY(cudaStreamSynchronize(s));
            prof.flush();
            if (B.need_cnt) {
                tc_window = nneed > 0;
                LRR_CUDA_TRY(cudaMemsetAsync(B.need_cnt, 0, sizeof(int), s));
            }
            if (bf16_phase) {
                bool any16 = false;
                for (int i = 0; i < t; ++i) any16 |= (ah[i] != 0 && fh[i] == 0);
                if (!any16) bf16_phase = false;
            }
            if (std::none_of(ah.begin(), ah.end(), [](int v) { return v != 0; })) break;
        }
        return LRR_OK;
    };
    if (o->batched) {
        const int rc = run_loop(std::vector<int>((size_t)t, 1));
        if (rc != LRR_OK) return rc;
    } else {
        for (int i = 0; i < t; ++i) {
            std::vector<int> a0((size_t)t, 0);
            a0[i] = 1;
            const int rc = run_loop(a0);
            if (rc != LRR_OK) return rc;
        }
    }
    LRR_CUDA_TRY(cudaEventRecord(ev[2], s));

    // ---- C step
    int k1 = 0;
    std::vector<int> rank_fin((size_t)t);
    LRR_CUDA_TRY(cudaMemcpyAsync(rank_fin.data(), B.rank_fin, sizeof(int) * t, cudaMemcpyDeviceToHost, s));
    T* Zfinal = B.Zt;
    if (dfc && t > 1) {
        const int p0 = pv[0], pp0 = ppv[0];
        // keep-list of block 1's SVT directions with h > 0 (final iteration)
        k::kept_columns<T><<<1, 32, 0, s>>>(B.h[0], p0, B.kept, B.kept_n);
        const T* src;
        int64_t ldsrc;
        if (tall[0]) {
            // left factor of J_1 = A W h W^T:  J_1 W = (A W) h  -> columns with h > 0
            std::vector<GemmDesc<T>> fd{gdesc<T>(B.Jt, r, B.W[0], pp0, B.Tt, r, r, p0, p0, nullptr)};
            LRR_CUDA_TRY(cudaMemcpyAsync(B.gd + gh.size(), fd.data(), sizeof(GemmDesc<T>), cudaMemcpyHostToDevice, s));
            LRR_CUDA_TRY(gemm_grouped<T>(B.gd + gh.size(), 1, false, false, r, p0, s));
            src = B.Tt;
            ldsrc = r;
        } else {
            // J_1 = W h W^T A: column space spanned by the kept eigenvectors
            src = B.W[0];
            ldsrc = pp0;
        }
        k::gather_normalise_f64<T><<<p0, 256, 0, s>>>(src, ldsrc, r, B.kept, B.kept_n, B.Fd);
        LRR_CUDA_TRY(cudaMemcpyAsync(&k1, B.kept_n, sizeof(int), cudaMemcpyDeviceToHost, s));
        LRR_CUDA_TRY(cudaStreamSynchronize(s));
        if (k1 > 0) {
            // orthonormal basis of span(F) in float64: the columns are already
            // orthogonal up to the Jacobi tolerance, so Newton-Schulz steps
            // X <- X (3I - X^T X)/2 converge quadratically to the polar factor
            GemmDesc<double>* d64 = reinterpret_cast<GemmDesc<double>*>(B.gd + gh.size());
            std::vector<GemmDesc<double>> nd{gdesc<double>(B.Fd, r, B.Fd, r, B.Gk, k1, k1, k1, r, nullptr),
                                             gdesc<double>(B.Fd, r, B.Gk, k1, B.Yd, r, r, k1, k1, nullptr)};
            LRR_CUDA_TRY(cudaMemcpyAsync(d64, nd.data(), sizeof(GemmDesc<double>) * 2, cudaMemcpyHostToDevice, s));
            for (int it = 0; it < 3; ++it) {
                LRR_CUDA_TRY(gemm_grouped<double>(d64, 1, true, false, k1, k1, s));
                LRR_CUDA_TRY(gemm_grouped<double>(d64 + 1, 1, false, false, r, k1, s));
                k::ns_combine<<<grid1((int64_t)r * k1), 256, 0, s>>>(B.Fd, B.Yd, (int64_t)r * k1);
            }
            k::copy_convert_f64<T><<<grid1((int64_t)r * k1), 256, 0, s>>>(B.Fd, B.Q, (int64_t)r * k1);
            std::vector<GemmDesc<T>> cd{gdesc<T>(B.Q, r, B.Zt, r, B.Wc, k1, k1, (int)n, r, nullptr),
                                        gdesc<T>(B.Q, r, B.Wc, k1, B.Tt, r, r, (int)n, k1, nullptr)};
            GemmDesc<T>* dT = B.gd + gh.size() + 4;
            LRR_CUDA_TRY(cudaMemcpyAsync(dT, cd.data(), sizeof(GemmDesc<T>) * 2, cudaMemcpyHostToDevice, s));
            LRR_CUDA_TRY(gemm_grouped<T>(dT, 1, true, false, k1, (int)n, s));
            LRR_CUDA_TRY(gemm_grouped<T>(dT + 1, 1, false, false, r, (int)n, s));
        } else {
            LRR_CUDA_TRY(cudaMemsetAsync(B.Tt, 0, sizeof(T) * r * n, s));
        }
        Zfinal = B.Tt;
    } else {
        k1 = rank_fin[0];
    }
    if (res && res->Z) {
        GemmDesc<T> zd = gdesc<T>(B.V, n, Zfinal, r, static_cast<T*>(res->Z), n, (int)n, (int)n, r, nullptr);
        zd.ccol = B.perm;
        GemmDesc<T>* dz = B.gd + gh.size() + 8;
        LRR_CUDA_TRY(cudaMemcpyAsync(dz, &zd, sizeof(zd), cudaMemcpyHostToDevice, s));
        LRR_CUDA_TRY(gemm_grouped<T>(dz, 1, false, false, (int)n, (int)n, s));
    }
    if (res && res->S)
        k::scatter_cols<T><<<dim3(grid1(m), (unsigned)std::min<int64_t>(n, 65535)), 256, 0, s>>>(
            B.E, m, n, B.perm, static_cast<T*>(res->S), m, m);
    // factored output: Z = F G with F = V Q (t > 1) or V (t = 1)
    int fk = 0;
    int64_t fcl = 0;
    if (res && (res->F || res->G)) {
        const bool comb = dfc && t > 1;
        fk = comb ? k1 : r;
        const int64_t kmax = comb ? std::min<int64_t>(m, blk[0].l) : std::min<int64_t>(m, n);
        if (fk > 0 && res->F) {
            if (comb) {
                GemmDesc<T> fd = gdesc<T>(B.V, n, B.Q, r, static_cast<T*>(res->F), n, (int)n, fk, r, nullptr);
                GemmDesc<T>* df = B.gd + gh.size() + 9;
                LRR_CUDA_TRY(cudaMemcpyAsync(df, &fd, sizeof(fd), cudaMemcpyHostToDevice, s));
                LRR_CUDA_TRY(gemm_grouped<T>(df, 1, false, false, (int)n, fk, s));
            } else {
                LRR_CUDA_TRY(cudaMemcpy2DAsync(res->F, sizeof(T) * n, B.V, sizeof(T) * n, sizeof(T) * n, (size_t)r,
                                               cudaMemcpyDeviceToDevice, s));
            }
            ++fcl;
        }
        if (fk > 0 && res->G) {
            k::scatter_cols<T><<<dim3(grid1(fk), (unsigned)std::min<int64_t>(n, 65535)), 256, 0, s>>>(
                comb ? B.Wc : B.Zt, fk, n, B.perm, static_cast<T*>(res->G), comb ? k1 : r, kmax);
            ++fcl;
        }
    }
    LRR_CUDA_TRY(cudaEventRecord(ev[3], s));
    {
        int64_t cl = (res && res->Z ? 1 : 0) + (res && res->S ? 1 : 0) + fcl;
        if (dfc && t > 1) cl += 2 + (tall[0] ? 1 : 0) + (k1 > 0 ? 3 * 3 + 3 : 0);
        prof.launches += cl;
        prof.calls[LRR_PH_COMBINE] += cl;
    }

    int tc_err_h = 0;
    LRR_CUDA_TRY(cudaMemcpyAsync(&tc_err_h, B.tc_err, sizeof(int), cudaMemcpyDeviceToHost, s));
    std::vector<int> iters_h((size_t)t), conv_h((size_t)t);
    std::vector<double> resid_h((size_t)2 * t);
    LRR_CUDA_TRY(cudaMemcpyAsync(iters_h.data(), B.iters, sizeof(int) * t, cudaMemcpyDeviceToHost, s));
    LRR_CUDA_TRY(cudaMemcpyAsync(conv_h.data(), B.conv, sizeof(int) * t, cudaMemcpyDeviceToHost, s));
    LRR_CUDA_TRY(cudaMemcpyAsync(resid_h.data(), B.resid, sizeof(double) * 2 * t, cudaMemcpyDeviceToHost, s));
    LRR_CUDA_TRY(cudaStreamSynchronize(s));
    if (res) {
        if (res->iters) std::copy(iters_h.begin(), iters_h.end(), res->iters);
        if (res->resid) std::copy(resid_h.begin(), resid_h.end(), res->resid);
        if (res->ranks) {
            res->ranks[0] = r;
            res->ranks[1] = k1;
            for (int i = 0; i < t; ++i) res->ranks[2 + i] = rank_fin[i];
        }
        if (res->stats) {
            lrr_stats& st = *res->stats;
            std::memset(&st, 0, sizeof(st));
            prof.flush();
            for (int i = 0; i < LRR_NPHASE; ++i) { st.phase_ms[i] = prof.ms[i]; st.phase_launches[i] = prof.calls[i]; }
            float a = 0, c = 0;
            cudaEventElapsedTime(&a, ev[0], ev[1]);
            cudaEventElapsedTime(&c, ev[2], ev[3]);
            st.phase_ms[LRR_PH_SETUP] = a;
            st.phase_ms[LRR_PH_COMBINE] = c;
            st.launches = prof.launches;
            st.iterations = prof.iterations;
            std::vector<int> sw((size_t)t), sc((size_t)t);
            cudaMemcpy(sw.data(), B.jsweeps, sizeof(int) * t, cudaMemcpyDeviceToHost);
            cudaMemcpy(sc.data(), B.svtcalls, sizeof(int) * t, cudaMemcpyDeviceToHost);
            for (int i = 0; i < t; ++i) { st.svt_sweeps += sw[i]; st.svt_calls += sc[i]; }
        }
        if (res->factor_k) *res->factor_k = fk;
        if (res->sweeps) {
            LRR_CUDA_TRY(cudaMemcpy(res->sweeps, B.jsweeps, sizeof(int) * t, cudaMemcpyDeviceToHost));
        }
        if (res->timings_ms) {
            float a = 0, b2 = 0, c = 0;
            cudaEventElapsedTime(&a, ev[0], ev[1]);
            cudaEventElapsedTime(&b2, ev[1], ev[2]);
            cudaEventElapsedTime(&c, ev[2], ev[3]);
            res->timings_ms[0] = a; res->timings_ms[1] = b2; res->timings_ms[2] = c;
        }
    }
    if (tc_err_h) return LRR_ERR_CUDA;   // a tensor-core product timed out
    for (int i = 0; i < t; ++i)
        if (!conv_h[i]) return LRR_NOT_CONVERGED;
    return LRR_OK;
}


// Stand-alone singular-value thresholding with the solver's own SVT kernels
// (cold start W = I).  Scratch is taken with cudaMallocAsync on the stream.
template <typename T>
int svt_impl(const T* A, int64_t rows, int64_t cols, int64_t lda, double tau, T* J, int64_t ldj, int32_t* rank_out,
             cudaStream_t s) {
    constexpr int B2 = osj_pivot_width();
    const bool tall = cols <= rows;
    const int p = (int)std::min(rows, cols);
    const int L = (int)(tall ? rows : cols);
    const int pp = round_up(p, B2);
    Arena sz(nullptr);
    auto lay = [&](Arena& a, T** X, T** W, T** H, T** T1, T** h, int** ints, double** dbl, OsjDesc<T>** od,
                   GemmDesc<T>** gd, T** Wp, T** Hp, T** hp, T** scl, T** off, T** T1p) {
        *X = a.take<T>((size_t)L * p);
        *W = a.take<T>((size_t)pp * pp);
        *H = a.take<T>((size_t)pp * pp);
        *T1 = a.take<T>((size_t)pp * pp);
        *h = a.take<T>(pp);
        *ints = a.take<int>(16);
        *dbl = a.take<double>(4);
        *od = a.take<OsjDesc<T>>(1);
        *gd = a.take<GemmDesc<T>>(8);
        *Wp = reinterpret_cast<T*>(a.take<T*>(1));
        *Hp = reinterpret_cast<T*>(a.take<T*>(1));
        *hp = reinterpret_cast<T*>(a.take<T*>(1));
        *scl = a.take<T>(1);
        *off = a.take<T>(3);
        *T1p = reinterpret_cast<T*>(a.take<T*>(1));
    };
    T *X, *W, *H, *T1, *h, *Wp, *Hp, *hp, *scl, *off, *T1p;
    int* ints;
    double* dbl;
    OsjDesc<T>* od;
    GemmDesc<T>* gd;
    lay(sz, &X, &W, &H, &T1, &h, &ints, &dbl, &od, &gd, &Wp, &Hp, &hp, &scl, &off, &T1p);
    void* mem = nullptr;
    if (cudaMallocAsync(&mem, sz.off + kAlign, s) != cudaSuccess) return LRR_ERR_CUDA;
    struct Free {
        void* p; cudaStream_t s;
        ~Free() { if (p) cudaFreeAsync(p, s); }
    } guard{mem, s};
    Arena a(mem);
    lay(a, &X, &W, &H, &T1, &h, &ints, &dbl, &od, &gd, &Wp, &Hp, &hp, &scl, &off, &T1p);
    int* act = ints;          // [0]
    int* on = ints + 1;       // [1]
    int* rk = ints + 2;       // [2]
    int* done = ints + 3;     // [3]
    int* swp = ints + 4;      // [4]
    double* mu = dbl;
    const int one[2] = {1, 1};
    const double mud = 1.0 / tau;
    LRR_CUDA_TRY(cudaMemcpyAsync(act, one, sizeof(int) * 2, cudaMemcpyHostToDevice, s));
    LRR_CUDA_TRY(cudaMemsetAsync(swp, 0, sizeof(int), s));
    LRR_CUDA_TRY(cudaMemcpyAsync(mu, &mud, sizeof(double), cudaMemcpyHostToDevice, s));
    k::init_padded<T><<<grid1((int64_t)pp * pp), 256, 0, s>>>(W, p, pp, T(1), 1);
    T* ptrs[4] = {W, H, h, T1};
    LRR_CUDA_TRY(cudaMemcpyAsync(T1p, &ptrs[3], sizeof(T*), cudaMemcpyHostToDevice, s));
    LRR_CUDA_TRY(cudaMemcpyAsync(Wp, &ptrs[0], sizeof(T*), cudaMemcpyHostToDevice, s));
    LRR_CUDA_TRY(cudaMemcpyAsync(Hp, &ptrs[1], sizeof(T*), cudaMemcpyHostToDevice, s));
    LRR_CUDA_TRY(cudaMemcpyAsync(hp, &ptrs[2], sizeof(T*), cudaMemcpyHostToDevice, s));
    const int pvals[2] = {p, pp};
    int* pv = ints + 8;
    int* ppv = ints + 9;
    LRR_CUDA_TRY(cudaMemcpyAsync(pv, &pvals[0], sizeof(int), cudaMemcpyHostToDevice, s));
    LRR_CUDA_TRY(cudaMemcpyAsync(ppv, &pvals[1], sizeof(int), cudaMemcpyHostToDevice, s));
    OsjDesc<T> d{};
    d.X = X; d.W = W; d.done = done; d.off = off; d.active = on; d.scale = scl; d.mu = mu;
    d.ldx = L; d.ldw = pp; d.L = L; d.p = p; d.pp = pp; d.strict = 1;
    LRR_CUDA_TRY(cudaMemcpyAsync(od, &d, sizeof(d), cudaMemcpyHostToDevice, s));
    GemmDesc<T> g[5];
    if (tall) g[0] = gdesc<T>(A, lda, W, pp, X, L, L, p, p, nullptr);          // X = A W
    else g[0] = gdesc<T>(A, lda, W, pp, X, L, L, p, p, nullptr);               // X = A^T W
    g[1] = gdesc<T>(W, pp, W, pp, T1, pp, p, p, p, nullptr);                   // W^T W
    g[2] = gdesc<T>(W, pp, T1, pp, H, pp, p, p, p, nullptr);                   // W (W^T W)
    if (tall) g[3] = gdesc<T>(X, L, T1, pp, J, ldj, (int)rows, (int)cols, p, nullptr);   // J = X h W^{-1}
    else g[3] = gdesc<T>(T1, pp, X, L, J, ldj, (int)rows, (int)cols, p, nullptr);        // J = W^{-T} h X^T
    g[3].kscale = h;
    LRR_CUDA_TRY(cudaMemcpyAsync(gd, g, sizeof(g), cudaMemcpyHostToDevice, s));
    LRR_CUDA_TRY(gemm_grouped<T>(gd, 1, !tall, false, L, p, s));
    k::col_norm_max<T><<<1, 256, 0, s>>>(od, on, scl, 1);
    LRR_CUDA_TRY(osj_sweeps<T>(od, 1, pp, 40, sizeof(T) == 8 ? T(1e-13) : T(2e-6), swp, s));
    k::svt_weights<T><<<1, 256, 0, s>>>(od, reinterpret_cast<T* const*>(hp), act, on, mu, rk, 1);
    LRR_CUDA_TRY(gemm_grouped<T>(gd + 1, 1, true, false, p, p, s));
    LRR_CUDA_TRY(gemm_grouped<T>(gd + 2, 1, false, false, p, p, s));
    k::ns_orth<T><<<dim3(64, 1), 256, 0, s>>>(reinterpret_cast<T* const*>(Wp), reinterpret_cast<T* const*>(Hp),
                                              reinterpret_cast<T* const*>(T1p), pv, ppv, on, 1);
    LRR_CUDA_TRY(gemm_grouped<T>(gd + 3, 1, false, true, (int)rows, (int)cols, s));
    int rk_h = 0;
    LRR_CUDA_TRY(cudaMemcpyAsync(&rk_h, rk, sizeof(int), cudaMemcpyDeviceToHost, s));
    LRR_CUDA_TRY(cudaStreamSynchronize(s));
    if (rank_out) *rank_out = rk_h;
    return LRR_OK;
}


// ---------------------------------------------------------------------------
// lrr_svt_noalloc: the stand-alone SVT with all of its scratch in one
// file-scope device array instead of a stream-ordered allocation.
//
// Capacity: kNoAllocScratchBytes (32 MiB) on every device that loads this
// library, held until the process exits.  The device address of the array is
// looked up once per device (cudaGetSymbolAddress, with that device current)
// by the first call made on it; make that first call before capturing the
// stream into a CUDA graph.  All calls share the array: every value a call
// reads is written by the same call first, and calls whose work overlaps on
// the GPU (two streams, two host threads) race on it.
constexpr size_t kNoAllocScratchBytes = size_t(32) << 20;
static __device__ __align__(256) unsigned char g_svt_scratch[kNoAllocScratchBytes];

std::mutex g_scratch_mutex;
void* g_scratch_ptr[64] = {};

// device address of g_svt_scratch on the current device (nullptr on failure)
void* svt_scratch_address() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_svt_scratch) != cudaSuccess) return nullptr;
        g_scratch_ptr[dev] = p;
    }
    return g_scratch_ptr[dev];
}

template <typename T>
int svt_noalloc_impl(const T* A, int64_t rows, int64_t cols, int64_t lda, double tau, T* J, int64_t ldj,
                     int32_t* rank_out, cudaStream_t s) {
    constexpr int B2 = osj_pivot_width();
    const bool tall = cols <= rows;
    const int p = (int)std::min(rows, cols);
    const int L = (int)(tall ? rows : cols);
    const int pp = round_up(p, B2);
    struct Parts {
        T *X, *W, *H, *T1, *h, *scl, *off;
        T **Wp, **Hp, **hp, **T1p;
        int* ints;
        double* dbl;
        OsjDesc<T>* od;
        GemmDesc<T>* gd;
    };
    auto lay = [&](Arena& a) {
        Parts q;
        q.X = a.take<T>((size_t)L * p);
        q.W = a.take<T>((size_t)pp * pp);
        q.H = a.take<T>((size_t)pp * pp);
        q.T1 = a.take<T>((size_t)pp * pp);
        q.h = a.take<T>(pp);
        q.ints = a.take<int>(16);
        q.dbl = a.take<double>(4);
        q.od = a.take<OsjDesc<T>>(1);
        q.gd = a.take<GemmDesc<T>>(8);
        q.Wp = a.take<T*>(1);
        q.Hp = a.take<T*>(1);
        q.hp = a.take<T*>(1);
        q.T1p = a.take<T*>(1);
        q.scl = a.take<T>(1);
        q.off = a.take<T>(3);
        return q;
    };
    Arena sz(nullptr);
    lay(sz);
    if (sz.off > kNoAllocScratchBytes) return LRR_ERR_TOO_LARGE;
    void* base = svt_scratch_address();
    if (!base) return LRR_ERR_CUDA;
    Arena a(base);
    const Parts q = lay(a);
    int* act = q.ints;
    int* on = q.ints + 1;
    int* rk = q.ints + 2;
    int* done = q.ints + 3;
    int* swp = q.ints + 4;
    int* pv = q.ints + 8;
    int* ppv = q.ints + 9;
    double* mu = q.dbl;
    const int one[2] = {1, 1};
    const double mud = 1.0 / tau;
    const int pvals[2] = {p, pp};
    T* ptrs[4] = {q.W, q.H, q.h, q.T1};
    LRR_CUDA_TRY(cudaMemcpyAsync(act, one, sizeof(int) * 2, cudaMemcpyHostToDevice, s));
    LRR_CUDA_TRY(cudaMemsetAsync(swp, 0, sizeof(int), s));
    LRR_CUDA_TRY(cudaMemcpyAsync(mu, &mud, sizeof(double), cudaMemcpyHostToDevice, s));
    LRR_CUDA_TRY(cudaMemcpyAsync(pv, pvals, sizeof(int) * 2, cudaMemcpyHostToDevice, s));
    LRR_CUDA_TRY(cudaMemcpyAsync(q.Wp, &ptrs[0], sizeof(T*), cudaMemcpyHostToDevice, s));
    LRR_CUDA_TRY(cudaMemcpyAsync(q.Hp, &ptrs[1], sizeof(T*), cudaMemcpyHostToDevice, s));
    LRR_CUDA_TRY(cudaMemcpyAsync(q.hp, &ptrs[2], sizeof(T*), cudaMemcpyHostToDevice, s));
    LRR_CUDA_TRY(cudaMemcpyAsync(q.T1p, &ptrs[3], sizeof(T*), cudaMemcpyHostToDevice, s));
    k::init_padded<T><<<grid1((int64_t)pp * pp), 256, 0, s>>>(q.W, p, pp, T(1), 1);
    OsjDesc<T> d{};
    d.X = q.X; d.W = q.W; d.done = done; d.off = q.off; d.active = on; d.scale = q.scl; d.mu = mu;
    d.ldx = L; d.ldw = pp; d.L = L; d.p = p; d.pp = pp; d.strict = 1;
    LRR_CUDA_TRY(cudaMemcpyAsync(q.od, &d, sizeof(d), cudaMemcpyHostToDevice, s));
    GemmDesc<T> g[4];
    g[0] = gdesc<T>(A, lda, q.W, pp, q.X, L, L, p, p, nullptr);                         // X = A W or A^T W
    g[1] = gdesc<T>(q.W, pp, q.W, pp, q.T1, pp, p, p, p, nullptr);                      // W^T W
    g[2] = gdesc<T>(q.W, pp, q.T1, pp, q.H, pp, p, p, p, nullptr);                      // W (W^T W)
    if (tall) g[3] = gdesc<T>(q.X, L, q.T1, pp, J, ldj, (int)rows, (int)cols, p, nullptr);
    else g[3] = gdesc<T>(q.T1, pp, q.X, L, J, ldj, (int)rows, (int)cols, p, nullptr);
    g[3].kscale = q.h;
    LRR_CUDA_TRY(cudaMemcpyAsync(q.gd, g, sizeof(g), cudaMemcpyHostToDevice, s));
    LRR_CUDA_TRY(gemm_grouped<T>(q.gd, 1, !tall, false, L, p, s));
    k::col_norm_max<T><<<1, 256, 0, s>>>(q.od, on, q.scl, 1);
    LRR_CUDA_TRY(osj_sweeps<T>(q.od, 1, pp, 40, sizeof(T) == 8 ? T(1e-13) : T(2e-6), swp, s));
    k::svt_weights<T><<<1, 256, 0, s>>>(q.od, q.hp, act, on, mu, rk, 1);
    LRR_CUDA_TRY(gemm_grouped<T>(q.gd + 1, 1, true, false, p, p, s));
    LRR_CUDA_TRY(gemm_grouped<T>(q.gd + 2, 1, false, false, p, p, s));
    k::ns_orth<T><<<dim3(64, 1), 256, 0, s>>>(q.Wp, q.Hp, q.T1p, pv, ppv, on, 1);
    LRR_CUDA_TRY(gemm_grouped<T>(q.gd + 3, 1, false, true, (int)rows, (int)cols, s));
    int rk_h = 0;
    LRR_CUDA_TRY(cudaMemcpyAsync(&rk_h, rk, sizeof(int), cudaMemcpyDeviceToHost, s));
    LRR_CUDA_TRY(cudaStreamSynchronize(s));
    if (rank_out) *rank_out = rk_h;
    return LRR_OK;
}

template <typename T, typename Tin>
size_t workspace_impl(const lrr_problem* p, const lrr_options* o, bool mixed) {
    const auto blk = block_info<T>(p);
    Arena probe(nullptr);
    carve<T>(probe, p, !std::is_same<Tin, double>::value, blk, mixed, use_tc32<T>(p, o));
    return probe.off + kAlign;
}

// The problem with a NULL perm / offsets replaced by the D step's defaults
// (dfc_partition); the vectors own the drawn arrays.
struct Resolved {
    lrr_problem q{};
    std::vector<int64_t> perm, off;
};
const lrr_problem* resolve(const lrr_problem* p, Resolved& r) {
    if (!p || (p->perm && p->offsets)) return p;
    if (p->n < 1 || p->t < 1 || p->t > p->n || p->n > (1 << 24)) return nullptr;
    r.q = *p;
    if (!p->perm) {
        r.perm.resize((size_t)p->n);
        draw_partition(p->n, p->t, p->seed, r.perm.data(), nullptr);
        r.q.perm = r.perm.data();
    }
    if (!p->offsets) {
        r.off.resize((size_t)p->t + 1);
        draw_partition(p->n, p->t, p->seed, nullptr, r.off.data());
        r.q.offsets = r.off.data();
    }
    return &r.q;
}

int dispatch(const lrr_problem* p0, const lrr_options* o, void* ws, size_t wsb, lrr_result* r, void* stream, bool dfc) {
    Resolved rs;
    const lrr_problem* p = resolve(p0, rs);
    if (!valid_problem(p, o)) return LRR_ERR_INVALID;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    switch (o->precision) {
        case LRR_PREC_F64: return solve_impl<double, double>(p, o, ws, wsb, r, s, dfc);
        case LRR_PREC_F32:
        case LRR_PREC_MIXED: return solve_impl<float, float>(p, o, ws, wsb, r, s, dfc);
        default: return LRR_ERR_UNSUPPORTED;
    }
}

// scatter of a block's l x l estimate to rows and columns perm[off .. off+l-1]
template <typename T>
__global__ void scatter_block(const T* __restrict__ src, int64_t l, const int64_t* __restrict__ perm, int64_t off,
                              T* __restrict__ Z, int64_t n) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < l * l; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t a = e % l, b = e / l;
        Z[perm[off + a] + perm[off + b] * n] = src[e];
    }
}

// The footnote variant of Algorithm 1: every block problem uses its own
// observations C_i as the dictionary (l_i x l_i solutions, solved as t
// independent LRR problems on concurrent streams), and the C step keeps the
// `rank` largest singular triplets of diag(Z_1, ..., Z_t).
template <typename T>
int local_impl(const lrr_problem* p, const lrr_options* o, int64_t rank, lrr_result* res, int32_t streams,
               cudaStream_t s) {
    const int64_t m = p->m, n = p->n;
    const int t = p->t;
    const T* M = static_cast<const T*>(p->M);
    std::vector<int64_t> l((size_t)t), kmax((size_t)t), off((size_t)t + 1);
    int64_t lmax = 0, words = m * n + m * n + n * n;   // C (block order), S (block order), scratch
    for (int i = 0; i < t; ++i) {
        off[i] = p->offsets[i];
        l[i] = p->offsets[i + 1] - p->offsets[i];
        kmax[i] = std::min<int64_t>(m, l[i]);
        lmax = std::max(lmax, l[i]);
    }
    off[t] = n;
    int64_t fwords = 0;
    for (int i = 0; i < t; ++i) fwords += 2 * l[i] * kmax[i];   // F_i, G_i
    const int B2 = osj_pivot_width();
    int64_t wwords = 0;
    std::vector<int> kp((size_t)t);
    for (int i = 0; i < t; ++i) {
        kp[i] = round_up((int)kmax[i], B2);
        wwords += (int64_t)kp[i] * kp[i] + l[i] * kmax[i] + l[i] * kmax[i];   // W_i, X_i, T_i
    }
    const size_t bytes = sizeof(T) * (size_t)(words + fwords + wwords) + sizeof(int64_t) * n +
                         (sizeof(OsjDesc<T>) + sizeof(GemmDesc<T>) * 2 + 64 * sizeof(T) + 64) * (size_t)t + 4096 * 4;
    void* mem = nullptr;
    if (cudaMallocAsync(&mem, bytes, s) != cudaSuccess) return LRR_ERR_CUDA;
    struct Free {
        void* p; cudaStream_t s;
        ~Free() { if (p) cudaFreeAsync(p, s); }
    } guard{mem, s};
    Arena a(mem);
    T* Cb = a.take<T>(m * n);
    T* Sb = a.take<T>(m * n);
    T* Zs = a.take<T>(lmax * lmax);
    int64_t* perm_d = a.take<int64_t>(n);
    std::vector<T*> F((size_t)t), G((size_t)t), W((size_t)t), X((size_t)t), Tm((size_t)t);
    for (int i = 0; i < t; ++i) {
        F[i] = a.take<T>(l[i] * kmax[i]);
        G[i] = a.take<T>(kmax[i] * l[i]);
        W[i] = a.take<T>((size_t)kp[i] * kp[i]);
        X[i] = a.take<T>(l[i] * kmax[i]);
        Tm[i] = a.take<T>(l[i] * kmax[i]);
    }
    OsjDesc<T>* od = a.take<OsjDesc<T>>(t);
    GemmDesc<T>* gd = a.take<GemmDesc<T>>(2 * (size_t)t);
    T* scl = a.take<T>(t);
    T* off3 = a.take<T>(3 * (size_t)t);
    int* done = a.take<int>(t);
    int* on = a.take<int>(t);
    T* hk = a.take<T>((size_t)t * 1);   // placeholder (per-block masks follow)
    (void)hk;
    std::vector<T*> H((size_t)t);
    for (int i = 0; i < t; ++i) H[i] = a.take<T>(kp[i]);
    if (a.off > bytes) return LRR_ERR_WORKSPACE;
    LRR_CUDA_TRY(cudaMemcpyAsync(perm_d, p->perm, sizeof(int64_t) * n, cudaMemcpyHostToDevice, s));
    k::gather_cols<T, T><<<dim3(grid1(m), (unsigned)std::min<int64_t>(n, 65535)), 256, 0, s>>>(M, p->ldm, perm_d, m, n,
                                                                                               Cb);
    // ---- F step: t independent LRR problems C_i = C_i Z_i + S_i
    std::vector<std::vector<int64_t>> ids((size_t)t), offs((size_t)t);
    std::vector<lrr_problem> probs((size_t)t);
    std::vector<lrr_result> rs((size_t)t);
    std::vector<int32_t> its((size_t)t), fk((size_t)t), st((size_t)t), sw((size_t)t);
    std::vector<double> rsd((size_t)2 * t);
    std::vector<std::vector<int32_t>> rk((size_t)t, std::vector<int32_t>(3));
    for (int i = 0; i < t; ++i) {
        ids[i].resize((size_t)l[i]);
        std::iota(ids[i].begin(), ids[i].end(), 0);
        offs[i] = {0, l[i]};
        lrr_problem& q = probs[i];
        q = lrr_problem{};
        q.M = Cb + off[i] * m; q.m = m; q.n = l[i]; q.ldm = m; q.t = 1;
        q.perm = ids[i].data(); q.offsets = offs[i].data();
        lrr_result& r = rs[i];
        r = lrr_result{};
        r.S = Sb + off[i] * m; r.F = F[i]; r.G = G[i]; r.factor_k = &fk[i]; r.iters = &its[i];
        r.resid = &rsd[2 * i]; r.ranks = rk[i].data(); r.sweeps = &sw[i];
    }
    LRR_CUDA_TRY(cudaStreamSynchronize(s));
    int rc = lrr_solve_batch(probs.data(), t, o, rs.data(), st.data(), streams, s);
    if (rc < 0) return rc;
    // ---- C step: singular values of every Z_i = F_i G_i are those of G_i
    //      (F_i orthonormal); one-sided Jacobi on X_i = G_i^T W_i for all blocks
    std::vector<OsjDesc<T>> dh((size_t)t);
    std::vector<GemmDesc<T>> g1v((size_t)t);
    int max_kp = 0;
    for (int i = 0; i < t; ++i) {
        const int ki = std::max(1, fk[i]);
        k::init_padded<T><<<grid1((int64_t)kp[i] * kp[i]), 256, 0, s>>>(W[i], ki, kp[i], T(1), 1);
        GemmDesc<T> g = gdesc<T>(G[i], kmax[i], W[i], kp[i], X[i], l[i], (int)l[i], ki, ki, nullptr);
        g1v[i] = g;
        OsjDesc<T>& d = dh[i];
        d = OsjDesc<T>{};
        d.X = X[i]; d.W = W[i]; d.done = done + i; d.off = off3 + 3 * i; d.active = on + i; d.scale = scl + i;
        d.mu = nullptr; d.ldx = l[i]; d.ldw = kp[i]; d.L = (int)l[i]; d.p = ki; d.pp = round_up(ki, B2);
        d.strict = 1;
        max_kp = std::max(max_kp, d.pp);
    }
    std::vector<int> onh((size_t)t);
    for (int i = 0; i < t; ++i) onh[i] = fk[i] > 0 ? 1 : 0;
    LRR_CUDA_TRY(cudaMemcpyAsync(on, onh.data(), sizeof(int) * t, cudaMemcpyHostToDevice, s));
    LRR_CUDA_TRY(cudaMemcpyAsync(gd, g1v.data(), sizeof(GemmDesc<T>) * t, cudaMemcpyHostToDevice, s));
    LRR_CUDA_TRY(gemm_grouped<T>(gd, t, true, false, (int)lmax, max_kp, s));
    LRR_CUDA_TRY(cudaMemcpyAsync(od, dh.data(), sizeof(OsjDesc<T>) * t, cudaMemcpyHostToDevice, s));
    k::col_norm_max<T><<<t, 256, 0, s>>>(od, on, scl, t);
    LRR_CUDA_TRY(osj_sweeps<T>(od, t, max_kp, 40, sizeof(T) == 8 ? T(1e-13) : T(2e-6), nullptr, s, 0));
    // singular values to the host; the global top `rank`
    std::vector<std::vector<T>> xs((size_t)t);
    std::vector<std::tuple<double, int, int>> all;
    for (int i = 0; i < t; ++i) {
        if (fk[i] <= 0) continue;
        xs[i].resize((size_t)(l[i] * fk[i]));
        LRR_CUDA_TRY(cudaMemcpyAsync(xs[i].data(), X[i], sizeof(T) * l[i] * fk[i], cudaMemcpyDeviceToHost, s));
    }
    LRR_CUDA_TRY(cudaStreamSynchronize(s));
    for (int i = 0; i < t; ++i)
        for (int j = 0; j < fk[i]; ++j) {
            double q = 0;
            for (int64_t r0 = 0; r0 < l[i]; ++r0) q += (double)xs[i][r0 + j * l[i]] * xs[i][r0 + j * l[i]];
            all.emplace_back(-std::sqrt(q), i, j);
        }
    std::sort(all.begin(), all.end());
    const int64_t kk = rank > 0 ? rank : (int64_t)rk[0][1];
    std::vector<std::vector<T>> hh((size_t)t);
    for (int i = 0; i < t; ++i) hh[i].assign((size_t)kp[i], T(0));
    for (int64_t q = 0; q < std::min<int64_t>(kk, (int64_t)all.size()); ++q)
        if (-std::get<0>(all[(size_t)q]) > 0) hh[std::get<1>(all[(size_t)q])][std::get<2>(all[(size_t)q])] = T(1);
    // Z_i,k = F_i W_i diag(h_i) X_i^T, scattered to the original rows and columns
    if (res && res->Z) {
        LRR_CUDA_TRY(cudaMemsetAsync(res->Z, 0, sizeof(T) * n * n, s));
        for (int i = 0; i < t; ++i) {
            const int ki = fk[i];
            if (ki <= 0) continue;
            LRR_CUDA_TRY(cudaMemcpyAsync(H[i], hh[i].data(), sizeof(T) * kp[i], cudaMemcpyHostToDevice, s));
            GemmDesc<T> ga = gdesc<T>(F[i], l[i], W[i], kp[i], Tm[i], l[i], (int)l[i], ki, ki, nullptr);
            GemmDesc<T> gb = gdesc<T>(Tm[i], l[i], X[i], l[i], Zs, l[i], (int)l[i], (int)l[i], ki, nullptr);
            gb.kscale = H[i];
            LRR_CUDA_TRY(cudaMemcpyAsync(gd + 2 * i, &ga, sizeof(ga), cudaMemcpyHostToDevice, s));
            LRR_CUDA_TRY(cudaMemcpyAsync(gd + 2 * i + 1, &gb, sizeof(gb), cudaMemcpyHostToDevice, s));
            LRR_CUDA_TRY(gemm_grouped<T>(gd + 2 * i, 1, false, false, (int)l[i], ki, s));
            LRR_CUDA_TRY(gemm_grouped<T>(gd + 2 * i + 1, 1, false, true, (int)l[i], (int)l[i], s));
            scatter_block<T><<<grid1(l[i] * l[i]), 256, 0, s>>>(Zs, l[i], perm_d, off[i], static_cast<T*>(res->Z), n);
        }
    }
    if (res && res->S)
        k::scatter_cols<T><<<dim3(grid1(m), (unsigned)std::min<int64_t>(n, 65535)), 256, 0, s>>>(
            Sb, m, n, perm_d, static_cast<T*>(res->S), m, m);
    LRR_CUDA_TRY(cudaStreamSynchronize(s));
    if (res) {
        if (res->iters) for (int i = 0; i < t; ++i) res->iters[i] = its[i];
        if (res->resid) for (int i = 0; i < 2 * t; ++i) res->resid[i] = rsd[i];
        if (res->ranks) {
            int rmax = 0;
            for (int i = 0; i < t; ++i) rmax = std::max(rmax, rk[i][0]);
            res->ranks[0] = rmax;
            res->ranks[1] = (int32_t)std::min<int64_t>(kk, (int64_t)all.size());
            for (int i = 0; i < t; ++i) res->ranks[2 + i] = rk[i][1];
        }
        if (res->sweeps) for (int i = 0; i < t; ++i) res->sweeps[i] = sw[i];
        if (res->factor_k) *res->factor_k = 0;
    }
    return rc;
}

}  // namespace
}  // namespace lrr

extern "C" {

int dfc_lrr_solve_local(const lrr_problem* p0, const lrr_options* o, int64_t rank, lrr_result* r, int32_t streams,
                        void* stream) {
    lrr::Resolved rsv;
    const lrr_problem* p = lrr::resolve(p0, rsv);
    if (!lrr::valid_problem(p, o) || streams < 0) return LRR_ERR_INVALID;
    if (r && (r->F || r->G)) return LRR_ERR_UNSUPPORTED;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (o->precision == LRR_PREC_F64) return lrr::local_impl<double>(p, o, rank, r, streams, s);
    return lrr::local_impl<float>(p, o, rank, r, streams, s);
}

size_t lrr_workspace_bytes(const lrr_problem* p0, const lrr_options* o) {
    lrr::Resolved rs;
    const lrr_problem* p = lrr::resolve(p0, rs);
    if (!lrr::valid_problem(p, o)) return 0;
    switch (o->precision) {
        case LRR_PREC_F64: return lrr::workspace_impl<double, double>(p, o, false);
        case LRR_PREC_F32: return lrr::workspace_impl<float, float>(p, o, false);
        case LRR_PREC_MIXED: return lrr::workspace_impl<float, float>(p, o, true);
        default: return 0;
    }
}

int lrr_solve(const lrr_problem* p, const lrr_options* o, void* ws, size_t wsb, lrr_result* r, void* stream) {
    if (!p || p->t != 1) return LRR_ERR_INVALID;
    return lrr::dispatch(p, o, ws, wsb, r, stream, false);
}

int dfc_lrr_solve(const lrr_problem* p, const lrr_options* o, void* ws, size_t wsb, lrr_result* r, void* stream) {
    return lrr::dispatch(p, o, ws, wsb, r, stream, true);
}

int lrr_svt(const void* A, int64_t rows, int64_t cols, int64_t lda, double tau, void* J, int64_t ldj,
            int32_t precision, int32_t* rank, void* stream) {
    if (!A || !J || rows < 1 || cols < 1 || lda < rows || ldj < rows || !(tau > 0)) return LRR_ERR_INVALID;
    if (rows > (1 << 16) || cols > (1 << 16)) return LRR_ERR_INVALID;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (precision == LRR_PREC_F64)
        return lrr::svt_impl<double>(static_cast<const double*>(A), rows, cols, lda, tau, static_cast<double*>(J), ldj,
                                     rank, s);
    if (precision == LRR_PREC_F32)
        return lrr::svt_impl<float>(static_cast<const float*>(A), rows, cols, lda, tau, static_cast<float*>(J), ldj,
                                    rank, s);
    return LRR_ERR_UNSUPPORTED;
}

int lrr_gemm_bf16(const void* A, int64_t lda, const void* B, int64_t ldb, float* C, int64_t ldc, int64_t M, int64_t N,
                  int64_t K, void* stream) {
    if (!A || !B || !C || M < 1 || N < 1 || K < 1 || lda < K || ldb < K || ldc < M) return LRR_ERR_INVALID;
    if (M > (1 << 30) || N > lrr::kTcMaxN || K > (1 << 30)) return LRR_ERR_INVALID;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int* err = nullptr;
    if (cudaMallocAsync(&err, sizeof(int), s) != cudaSuccess) return LRR_ERR_CUDA;
    int rc = LRR_OK;
    if (cudaMemsetAsync(err, 0, sizeof(int), s) != cudaSuccess ||
        lrr::tc_gemm_bf16(A, lda, B, ldb, C, ldc, (int)M, (int)N, (int)K, err, s) != cudaSuccess)
        rc = LRR_ERR_CUDA;
    int h = 0;
    if (cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess) rc = LRR_ERR_CUDA;
    cudaFreeAsync(err, s);
    if (cudaStreamSynchronize(s) != cudaSuccess) rc = LRR_ERR_CUDA;
    if (h) rc = LRR_ERR_CUDA;
    return rc;
}

int lrr_gemm_f32(const float* A, int64_t lda, const float* B, int64_t ldb, float* C, int64_t ldc, int64_t M,
                 int64_t N, int64_t K, void* stream) {
    if (!A || !B || !C || M < 1 || N < 1 || K < 1 || lda < K || ldb < K || ldc < M) return LRR_ERR_INVALID;
    if (M > (1 << 30) || N > lrr::kTcMaxN || K > (1 << 30)) return LRR_ERR_INVALID;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int64_t k4 = (K + 3) / 4 * 4;
    const size_t words = (size_t)k4 * (size_t)(M + N) * 2;
    void* mem = nullptr;
    if (cudaMallocAsync(&mem, words * sizeof(float) + 256, s) != cudaSuccess) return LRR_ERR_CUDA;
    float* ah = static_cast<float*>(mem);
    float* al = ah + (size_t)k4 * M;
    float* bh = al + (size_t)k4 * M;
    float* bl = bh + (size_t)k4 * N;
    int* err = reinterpret_cast<int*>(bl + (size_t)k4 * N);
    int rc = LRR_OK;
    lrr::k::split_tf32_km<float><<<dim3(lrr::grid1(k4), (unsigned)std::min<int64_t>(M, 65535)), 256, 0, s>>>(
        A, lda, K, M, ah, al, k4);
    lrr::k::split_tf32_km<float><<<dim3(lrr::grid1(k4), (unsigned)std::min<int64_t>(N, 65535)), 256, 0, s>>>(
        B, ldb, K, N, bh, bl, k4);
    if (cudaMemsetAsync(err, 0, sizeof(int), s) != cudaSuccess ||
        lrr::tc_gemm_3xtf32(ah, al, k4, bh, bl, k4, C, ldc, (int)M, (int)N, (int)K, nullptr, nullptr, err, s) !=
            cudaSuccess)
        rc = LRR_ERR_CUDA;
    int h = 0;
    if (cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess) rc = LRR_ERR_CUDA;
    cudaFreeAsync(mem, s);
    if (cudaStreamSynchronize(s) != cudaSuccess) rc = LRR_ERR_CUDA;
    if (h) rc = LRR_ERR_CUDA;
    return rc;
}

int lrr_gemm_timing(int32_t kind, int64_t M, int64_t N, int64_t K, int32_t repeat, double* ms_per_launch,
                    void* stream) {
    if (!ms_per_launch || M < 1 || N < 1 || K < 1 || repeat < 1 || kind < 0 || kind > 2) return LRR_ERR_INVALID;
    if (M > (1 << 20) || N > lrr::kTcMaxN || K > (1 << 20)) return LRR_ERR_INVALID;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const bool bf = kind != 1;
    const int64_t kp = bf ? (K + 7) / 8 * 8 : (K + 3) / 4 * 4;
    const size_t esz = bf ? 2 : 4;
    const size_t nops = kind == 0 ? 1 : 2;          // split forms: hi and lo
    const size_t abytes = ((size_t)kp * M * esz + 255) / 256 * 256, bbytes = ((size_t)kp * N * esz + 255) / 256 * 256;
    const size_t total = nops * (abytes + bbytes) + sizeof(float) * (size_t)M * N + 256;
    void* mem = nullptr;
    if (cudaMallocAsync(&mem, total, s) != cudaSuccess) return LRR_ERR_CUDA;
    char* p = static_cast<char*>(mem);
    void* A0 = p; p += abytes;
    void* A1 = p; p += nops > 1 ? abytes : 0;
    void* B0 = p; p += bbytes;
    void* B1 = p; p += nops > 1 ? bbytes : 0;
    float* C = reinterpret_cast<float*>(p); p += sizeof(float) * (size_t)M * N;
    int* err = reinterpret_cast<int*>((reinterpret_cast<uintptr_t>(p) + 15) / 16 * 16);
    int rc = LRR_OK;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (kind == 0) {
        lrr::k::fill_hash_bf16<<<lrr::grid1(kp * M), 256, 0, s>>>(static_cast<uint16_t*>(A0), kp * M, 1u);
        lrr::k::fill_hash_bf16<<<lrr::grid1(kp * N), 256, 0, s>>>(static_cast<uint16_t*>(B0), kp * N, 2u);
    } else if (kind == 2) {
        lrr::k::fill_hash_bf16<<<lrr::grid1(kp * M), 256, 0, s>>>(static_cast<uint16_t*>(A0), kp * M, 1u);
        lrr::k::fill_hash_bf16<<<lrr::grid1(kp * M), 256, 0, s>>>(static_cast<uint16_t*>(A1), kp * M, 3u);
        lrr::k::fill_hash_bf16<<<lrr::grid1(kp * N), 256, 0, s>>>(static_cast<uint16_t*>(B0), kp * N, 2u);
        lrr::k::fill_hash_bf16<<<lrr::grid1(kp * N), 256, 0, s>>>(static_cast<uint16_t*>(B1), kp * N, 4u);
    } else {
        lrr::k::fill_hash<float><<<lrr::grid1(kp * M), 256, 0, s>>>(static_cast<float*>(A0), kp * M, 1u);
        lrr::k::fill_hash<float><<<lrr::grid1(kp * M), 256, 0, s>>>(static_cast<float*>(A1), kp * M, 3u);
        lrr::k::fill_hash<float><<<lrr::grid1(kp * N), 256, 0, s>>>(static_cast<float*>(B0), kp * N, 2u);
        lrr::k::fill_hash<float><<<lrr::grid1(kp * N), 256, 0, s>>>(static_cast<float*>(B1), kp * N, 4u);
    }
    auto launch = [&]() {
        if (kind == 2) return lrr::tc_gemm_bf16x3(A0, A1, kp, B0, B1, kp, C, M, (int)M, (int)N, (int)K, err, s);
        return kind == 0 ? lrr::tc_gemm_bf16(A0, kp, B0, kp, C, M, (int)M, (int)N, (int)K, err, s)
                         : lrr::tc_gemm_3xtf32(static_cast<float*>(A0), static_cast<float*>(A1), kp,
                                               static_cast<float*>(B0), static_cast<float*>(B1), kp, C, M, (int)M,
                                               (int)N, (int)K, nullptr, nullptr, err, s);
    };
    if (cudaMemsetAsync(err, 0, sizeof(int), s) != cudaSuccess || launch() != cudaSuccess ||
        cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
        rc = LRR_ERR_CUDA;
    if (rc == LRR_OK) {
        cudaEventRecord(e0, s);
        for (int i = 0; i < repeat && rc == LRR_OK; ++i)
            if (launch() != cudaSuccess) rc = LRR_ERR_CUDA;
        cudaEventRecord(e1, s);
    }
    int h = 0;
    if (cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess) rc = LRR_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) rc = LRR_ERR_CUDA;
    float ms = 0.f;
    if (rc == LRR_OK && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess) *ms_per_launch = ms / repeat;
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFreeAsync(mem, s);
    cudaStreamSynchronize(s);
    if (h) rc = LRR_ERR_CUDA;
    return rc;
}

int lrr_svt_noalloc(const void* A, int64_t rows, int64_t cols, int64_t lda, double tau, void* J, int64_t ldj,
                    int32_t precision, int32_t* rank, void* stream) {
    if (!A || !J || rows < 1 || cols < 1 || lda < rows || ldj < rows || !(tau > 0)) return LRR_ERR_INVALID;
    if (rows > (1 << 16) || cols > (1 << 16)) return LRR_ERR_TOO_LARGE;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (precision == LRR_PREC_F64)
        return lrr::svt_noalloc_impl<double>(static_cast<const double*>(A), rows, cols, lda, tau,
                                             static_cast<double*>(J), ldj, rank, s);
    if (precision == LRR_PREC_F32)
        return lrr::svt_noalloc_impl<float>(static_cast<const float*>(A), rows, cols, lda, tau, static_cast<float*>(J),
                                            ldj, rank, s);
    return LRR_ERR_UNSUPPORTED;
}

size_t lrr_svt_noalloc_capacity(void) { return lrr::kNoAllocScratchBytes; }

int64_t lrr_factor_max_rank(const lrr_problem* p) {
    if (!p || p->m < 1 || p->n < 1 || p->t < 1 || p->t > p->n) return 0;
    if (p->t == 1) return std::min(p->m, p->n);
    const int64_t l1 = p->offsets ? p->offsets[1] - p->offsets[0] : p->n / p->t;
    return l1 > 0 ? std::min(p->m, l1) : 0;
}

void lrr_default_options(lrr_options* o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->lambda = 0.1;
    o->rho = 1.1;
    o->mu0 = 1e-6;
    o->mu_max = 1e10;
    o->eps = 1e-6;
    o->max_iter = 1000;
    o->precision = LRR_PREC_F32;
    o->batched = 1;
    o->jacobi_sweeps = 0;
    o->rank_tol = 0.0;
    o->mixed_switch = 0.0;
}

const char* lrr_status_string(int s) {
    switch (s) {
        case LRR_OK: return "ok";
        case LRR_NOT_CONVERGED: return "not converged: at least one block reached max_iter";
        case LRR_ERR_INVALID: return "invalid argument";
        case LRR_ERR_NONFINITE: return "M contains NaN or Inf";
        case LRR_ERR_CUDA: return "CUDA runtime error";
        case LRR_ERR_WORKSPACE: return "workspace too small or not 256-byte aligned";
        case LRR_ERR_RANK: return "M is numerically zero";
        case LRR_ERR_UNSUPPORTED: return "option combination not available (unknown precision, or mixed precision with n > 8388480)";
        case LRR_ERR_TOO_LARGE: return "problem does not fit the fixed scratch array of lrr_svt_noalloc";
        default: return "unknown status";
    }
}

}  // extern "C"
