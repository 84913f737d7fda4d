// Shared device helpers for the DFC-LRR kernels (sm_103a).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>

#include <cfloat>
#include <cmath>

#define LRR_CUDA_TRY(expr)                       \
    do {                                         \
        cudaError_t _e = (expr);                 \
        if (_e != cudaSuccess) return LRR_ERR_CUDA; \
    } while (0)

namespace lrr {

template <typename T> struct num;
template <> struct num<float> {
    static __host__ __device__ constexpr float eps() { return FLT_EPSILON; }
    static __host__ __device__ constexpr float tiny() { return FLT_MIN; }
};
template <> struct num<double> {
    static __host__ __device__ constexpr double eps() { return DBL_EPSILON; }
    static __host__ __device__ constexpr double tiny() { return DBL_MIN; }
};

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
template <typename T>
__device__ __forceinline__ T warp_max(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// atomic max of a non-negative floating value, stored as its bit pattern
// (non-negative IEEE values order like their unsigned bit patterns)
__device__ __forceinline__ void atomic_max_nonneg(float* addr, float v) {
    atomicMax(reinterpret_cast<unsigned int*>(addr), __float_as_uint(v));
}
__device__ __forceinline__ void atomic_max_nonneg(double* addr, double v) {
    atomicMax(reinterpret_cast<unsigned long long*>(addr), (unsigned long long)__double_as_longlong(v));
}

inline unsigned ceil_div(int64_t a, int64_t b) { return (unsigned)((a + b - 1) / b); }

// Raises a kernel's dynamic shared-memory limit once per device (the attribute
// belongs to the device's context); `done` holds one bit per device id.
template <typename K>
inline cudaError_t ensure_smem_limit(K kernel, int bytes, std::atomic<uint64_t>& done) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const uint64_t bit = (dev >= 0 && dev < 64) ? (uint64_t(1) << dev) : 0;
    if (bit && (done.load(std::memory_order_acquire) & bit)) return cudaSuccess;
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess && bit) done.fetch_or(bit, std::memory_order_acq_rel);
    return e;
}

}  // namespace lrr
