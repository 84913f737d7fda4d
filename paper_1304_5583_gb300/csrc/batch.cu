// Many independent problems at once: a pool of host threads, each with its
// own CUDA stream, takes problems from a shared counter and solves each with
// dfc_lrr_solve (its scratch stream-ordered on that stream).  Problems whose
// dictionaries differ cannot share one batched launch (the batched solver
// shares the factor of M between blocks), so they overlap on the GPU through
// concurrent streams instead: the footnote variant's per-block problems and
// the many small problems of a phase-transition sweep.
#include <algorithm>
#include <atomic>
#include <thread>
#include <vector>

#include "dfc_lrr.h"
#include "common.cuh"

namespace lrr {
namespace {

int worse(int a, int b) {
    // failures (negative) dominate, then "not converged"
    if (a < 0 || b < 0) return std::min(a, b);
    return std::max(a, b);
}

}  // namespace
}  // namespace lrr

extern "C" {

int lrr_solve_batch(const lrr_problem* problems, int32_t count, const lrr_options* o, lrr_result* results,
                    int32_t* status, int32_t streams, void* stream) {
    if (!problems || !o || count < 0 || streams < 0) return LRR_ERR_INVALID;
    if (count == 0) return LRR_OK;
    cudaStream_t s0 = static_cast<cudaStream_t>(stream);
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return LRR_ERR_CUDA;
    // inputs written on the caller's stream must be complete
    if (cudaStreamSynchronize(s0) != cudaSuccess) return LRR_ERR_CUDA;
    const int nw = std::max(1, std::min<int>(streams > 0 ? streams : 8, count));
    std::atomic<int> next{0};
    std::vector<int> st((size_t)count, LRR_OK);
    std::vector<int> werr((size_t)nw, LRR_OK);
    auto worker = [&](int w) {
        if (cudaSetDevice(dev) != cudaSuccess) { werr[w] = LRR_ERR_CUDA; return; }
        cudaStream_t s = nullptr;
        if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) { werr[w] = LRR_ERR_CUDA; return; }
        for (int i = next.fetch_add(1); i < count; i = next.fetch_add(1))
            st[(size_t)i] = dfc_lrr_solve(problems + i, o, nullptr, 0, results ? results + i : nullptr, s);
        if (cudaStreamSynchronize(s) != cudaSuccess) werr[w] = LRR_ERR_CUDA;
        cudaStreamDestroy(s);
    };
    std::vector<std::thread> pool;
    for (int w = 1; w < nw; ++w) pool.emplace_back(worker, w);
    worker(0);
    for (auto& th : pool) th.join();
    int rc = LRR_OK;
    for (int i = 0; i < count; ++i) {
        if (status) status[i] = st[(size_t)i];
        rc = lrr::worse(rc, st[(size_t)i]);
    }
    for (int e : werr) rc = lrr::worse(rc, e);
    return rc;
}

}  // extern "C"
