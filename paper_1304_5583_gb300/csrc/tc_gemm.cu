// bf16 x bf16 -> fp32 matrix products on the 5th-generation tensor cores
// (tcgen05.mma) with TMA-fed shared-memory tiles and the accumulator in
// tensor memory.  Used by the mixed-precision iteration (U^T P and
// U diag(sigma) Z over all blocks at once, from split operands), by the stop
// test (V D with a max-abs epilogue) and on request for the float32 products.
//
// C (M x N, column-major, ldc) = A * B with A given K-major (element (m, k) at
// A[k + m * lda]) and B given K-major (element (k, n) at B[k + n * ldb]); both
// bf16 with lda, ldb multiples of 8.
// tc_gemm_kernel (plain bf16): persistent, one CTA per SM over 128 x 256
// tiles of C:
//   warp 0      TMA producer: 64-wide K slabs of A (128 rows) and B (256
//               rows) into a 4-stage ring (128-byte swizzle), completion
//               tracked by mbarriers; the ring runs on from tile to tile;
//   warp 1      allocates 2 x 256 TMEM columns (two accumulators), one
//               elected lane issues four 128x256x16 MMAs per slab and commits
//               each slab back to the ring and each finished tile to the
//               epilogue;
//   warps 2..5  epilogue: tcgen05.ld of their 32-lane quadrant of the
//               accumulator, float32 stores (rows contiguous in C), or, in
//               the reduction form, a per-column-block max |C_ij| (warp
//               reduction, one atomic per warp and block) without storing C;
//               the drained accumulator is handed back to warp 1, so tile
//               i + 1's MMAs overlap tile i's epilogue.
// tc_gemm_split_kernel (split operands, float32 accuracy): one 128 x 128
// tile per CTA, see below.
// Every wait is bounded (about one second of spinning); a timeout sets *err,
// drains the copies and MMAs already issued and frees TMEM before returning.
#include <algorithm>
#include <atomic>

#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include "common.cuh"
#include "kernels.cuh"

namespace lrr {
namespace {

constexpr int BM = 128, BN = 128, BK = 64;
constexpr int NT = 192;
constexpr uint32_t TILE_BYTES = BM * BK * 2;            // 128-row slab of 64 bf16: 16 KB
// persistent bf16 product: 128 x 256 tiles, 4-stage ring of 48 KB stages
constexpr int PBN = 256, PSTAGES = 4;
constexpr uint32_t TILE_A_BYTES = BM * BK * 2;          // 16 KB
constexpr uint32_t TILE_B_BYTES = PBN * BK * 2;         // 32 KB
constexpr uint32_t PSTAGE_BYTES = TILE_A_BYTES + TILE_B_BYTES;
constexpr long long WAIT_CYCLES = 2000000000LL;          // ~1 s at 2 GHz

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count));
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(smem_u32(bar)) : "memory");
}
// bounded wait: false (and *err set) after WAIT_CYCLES
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, int* err) {
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (clock64() - t0 > WAIT_CYCLES) {
            atomicExch(err, 1);
            return false;
        }
    }
    return true;
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int c0, int c1, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];\n" ::"r"(
            smem_u32(dst)),
        "l"(map), "r"(c0), "r"(c1), "r"(smem_u32(bar))
        : "memory");
}

// shared-memory matrix descriptor: K-major tile of 8-row x 128-byte swizzle
// atoms (stride between 8-row groups 1024 bytes), descriptor version 1
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
    uint64_t d = 0;
    d |= (uint64_t)((addr >> 4) & 0x3FFF);
    d |= (uint64_t)1 << 16;                 // leading-byte offset (unused with 128B swizzle)
    d |= (uint64_t)(1024 >> 4) << 32;       // stride-byte offset
    d |= (uint64_t)1 << 46;                 // descriptor version
    d |= (uint64_t)2 << 61;                 // 128-byte swizzle
    return d;
}

// instruction descriptor, kind::f16: fp32 accumulate, bf16 A and B, both K-major
__host__ __device__ constexpr uint32_t idesc_bf16(int m, int n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

// Persistent form: one CTA per SM walks the 128 x 256 tiles of C (tile index
// blockIdx.x, then every gridDim.x-th; tiles in M fastest, so the CTAs working
// at the same time share the B slabs in L2).  The producer's stage ring and
// the k-block counter run on across tiles; the accumulator is double-buffered
// in TMEM (2 x 256 columns), so the MMAs of tile i + 1 run while the epilogue
// drains tile i.
__global__ void __launch_bounds__(NT, 1) tc_gemm_kernel(const __grid_constant__ CUtensorMap mapA,
                                                        const __grid_constant__ CUtensorMap mapB, float* __restrict__ C,
                                                        int64_t ldc, int M, int N, int K, int* __restrict__ err,
                                                        const TcAbsmax am) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    // 1024-byte alignment for the swizzled tiles
    unsigned char* base = reinterpret_cast<unsigned char*>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    __shared__ __align__(8) uint64_t full_bar[PSTAGES], empty_bar[PSTAGES], accf[2], acce[2], drain_bar;
    __shared__ uint32_t tmem_slot;
    __shared__ int abort_flag;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int tiles_m = (M + BM - 1) / BM;
    const int ntiles = tiles_m * ((N + PBN - 1) / PBN);
    const int nk = (K + BK - 1) / BK;

    // reduction form: the whole launch does nothing when *run == 0
    // (uniform, before any barrier or TMEM use)
    if (am.bmax && am.run && *am.run == 0) return;
    // reduction form: a tile none of whose columns belongs to a block that
    // asks for the maximum is skipped by every role alike
    auto skip = [&](int tile) -> bool {
        if (!am.bmax) return false;
        const int n0 = (tile / tiles_m) * PBN;
        const int b_lo = am.colblk[n0], b_hi = am.colblk[min(n0 + PBN, N) - 1];
        for (int b = b_lo; b <= b_hi; ++b)
            if (am.need[b] != 0) return false;
        return true;
    };

    if (threadIdx.x == 0) {
        for (int s = 0; s < PSTAGES; ++s) {
            mbar_init(&full_bar[s], 1);
            mbar_init(&empty_bar[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&accf[b], 1);
            mbar_init(&acce[b], 4);
        }
        mbar_init(&drain_bar, 1);
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(&tmem_slot)),
                     "r"(2 * PBN));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n");
    const uint32_t tmem = tmem_slot;

    if (warp == 0) {
        if (lane == 0) {
            int64_t g = 0;     // k-blocks issued over all tiles of this CTA
            bool ok = true;
            for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
                if (skip(tile)) continue;
                const int m0 = (tile % tiles_m) * BM, n0 = (tile / tiles_m) * PBN;
                for (int kb = 0; kb < nk; ++kb, ++g) {
                    const int s = (int)(g % PSTAGES);
                    if (g >= PSTAGES && !mbar_wait(&empty_bar[s], (uint32_t)((g / PSTAGES) - 1) & 1, err)) ok = false;
                    if (!ok || abort_flag) {
                        ok = false;
                        break;
                    }
                    unsigned char* st = base + s * PSTAGE_BYTES;
                    mbar_expect_tx(&full_bar[s], PSTAGE_BYTES);
                    tma_load_2d(st, &mapA, kb * BK, m0, &full_bar[s]);
                    tma_load_2d(st + TILE_A_BYTES, &mapB, kb * BK, n0, &full_bar[s]);
                }
            }
            if (!ok) {
                abort_flag = 1;
                // let the copies already in flight land before the CTA exits
                for (int64_t j = g - PSTAGES < 0 ? 0 : g - PSTAGES; j < g; ++j)
                    mbar_wait(&full_bar[j % PSTAGES], (uint32_t)(j / PSTAGES) & 1, err);
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            constexpr uint32_t idesc = idesc_bf16(BM, PBN);
            int64_t g = 0;
            int i = 0;         // tiles computed by this CTA
            bool ok = true;
            for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
                if (skip(tile)) continue;
                const int buf = i & 1;
                // the epilogue must have drained this accumulator (tile i - 2)
                if (i >= 2 && !mbar_wait(&acce[buf], (uint32_t)((i >> 1) - 1) & 1, err)) {
                    ok = false;
                    break;
                }
                const uint32_t acc = tmem + (uint32_t)(buf * PBN);
                for (int kb = 0; kb < nk; ++kb, ++g) {
                    const int s = (int)(g % PSTAGES);
                    if (!mbar_wait(&full_bar[s], (uint32_t)(g / PSTAGES) & 1, err) || abort_flag) {
                        ok = false;
                        break;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;\n");
                    const uint32_t a_addr = smem_u32(base + s * PSTAGE_BYTES);
                    const uint32_t b_addr = a_addr + TILE_A_BYTES;
#pragma unroll
                    for (int k = 0; k < BK / 16; ++k) {
                        const uint64_t da = smem_desc(a_addr + k * 32);
                        const uint64_t db = smem_desc(b_addr + k * 32);
                        const uint32_t accum = (kb > 0 || k > 0) ? 1u : 0u;
                        asm volatile(
                            "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
                            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(acc),
                            "l"(da), "l"(db), "r"(idesc), "r"(accum));
                    }
                    asm volatile(
                        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                            smem_u32(&empty_bar[s]))
                        : "memory");
                }
                if (!ok) break;
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                                 smem_u32(&accf[buf]))
                             : "memory");
                ++i;
            }
            if (!ok) {
                abort_flag = 1;
                // every MMA issued so far completes before TMEM is released
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                                 smem_u32(&drain_bar))
                             : "memory");
                mbar_wait(&drain_bar, 0, err);
            }
        }
    } else {
        // epilogue warps 2..5 own TMEM lane quadrants (warp % 4)
        const int q = warp & 3;
        int i = 0;
        bool ok = true;
        for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
            if (skip(tile)) continue;
            const int buf = i & 1;
            ok = __all_sync(0xffffffffu, ok && mbar_wait(&accf[buf], (uint32_t)(i >> 1) & 1, err) && !abort_flag);
            if (!ok) break;
            asm volatile("tcgen05.fence::after_thread_sync;\n");
            const int m0 = (tile % tiles_m) * BM, n0 = (tile / tiles_m) * PBN;
            const int row = m0 + q * 32 + lane;
            // reduction form: running max of the current column block; the
            // block changes at the same column for every lane of the warp
            int cur_b = -1;
            float cur_m = 0.f;
            auto flush = [&]() {
                if (cur_b >= 0 && am.need[cur_b]) {
                    const unsigned u = __reduce_max_sync(0xffffffffu, __float_as_uint(cur_m));
                    if (lane == 0) atomicMax(am.bmax + cur_b, u);
                }
            };
#pragma unroll 1
            for (int c0 = 0; c0 < PBN; c0 += 16) {
                if (n0 + c0 >= N) break;      // warp-uniform
                uint32_t v[16];
                const uint32_t taddr = tmem + (uint32_t)(buf * PBN) + ((uint32_t)(q * 32) << 16) + (uint32_t)c0;
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, "
                    "%13, %14, %15}, [%16];\n"
                    : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                      "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]),
                      "=r"(v[15])
                    : "r"(taddr));
                asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
                if (am.bmax) {
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        const int col = n0 + c0 + j;
                        if (col < N) {
                            const int b = am.colblk[col];
                            if (b != cur_b) {
                                flush();
                                cur_b = b;
                                cur_m = 0.f;
                            }
                            if (row < M) {
                                // NaN wins (its bits exceed every finite |x|)
                                const float a = fabsf(__uint_as_float(v[j]));
                                if (a > cur_m || a != a) cur_m = a;
                            }
                        }
                    }
                } else if (row < M) {
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        const int col = n0 + c0 + j;
                        if (col < N) C[row + (int64_t)col * ldc] = __uint_as_float(v[j]);
                    }
                }
            }
            if (am.bmax) flush();
            // accumulator drained: the MMA warp may reuse it for tile i + 2
            asm volatile("tcgen05.fence::before_thread_sync;\n");
            __syncwarp();
            if (lane == 0) mbar_arrive(&acce[buf]);
            ++i;
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n");
    __syncthreads();
    if (warp == 1) {
        asm volatile("tcgen05.fence::after_thread_sync;\n");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(2 * PBN));
    }
}

// ---------------------------------------------------------------------------
// Float32-accurate products on the tensor cores from split operands: every
// float32 operand x is given as x ~ hi + lo, hi and lo both exact in the
// tensor-core input type (hi the nearest value to x, lo the nearest to x - hi),
// and
//   a b ~ a_hi b_hi + a_hi b_lo + a_lo b_hi     (a_lo b_lo dropped)
// runs as three MMAs into one float32 accumulator.
//   split TF32 ("3xTF32", kind::tf32): the dropped term is below 2^-22 |a b|
//     and the split error below 2^-21 |a b| (split_tf32);
//   split bf16 ("bf16x3", the three-product form of Henry, Tang and Heinecke,
//     "Leveraging the bfloat16 artificial intelligence datatype for
//     higher-precision computations", ARITH 2019; kind::f16): hi and lo carry
//     8 significant bits each, so the dropped term is below 2^-16 |a b| and
//     the split error below 2^-17 |a b| -- about 2^7 below the bf16 product.
// Same CTA structure as tc_gemm_kernel; a stage holds A_hi, A_lo, B_hi, B_lo
// slabs of 128 bytes along K (32 float32 or 64 bf16 values).  With
// `tile_flag` set, a 128-column tile whose columns all belong to blocks whose
// flag is zero is skipped.
constexpr int BK32 = 32, STAGES32 = 3;
constexpr uint32_t STAGE_BYTES32 = 4 * TILE_BYTES;

// instruction descriptor, kind::tf32: fp32 accumulate, TF32 A and B, both K-major
__host__ __device__ constexpr uint32_t idesc_tf32(int m, int n) {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

struct TileSkip {
    const int* colblk;   // block of each column of C
    const int* flag;     // per block: nonzero = compute its columns
};


// The accumulator is drained into float32 registers every SLAB k-blocks: the
// tensor cores add each MMA's products to the accumulator with a truncating
// alignment, an error that grows with the magnitude the accumulator has
// reached, so a long K is summed as short tensor-core slabs (each into a fresh
// accumulator) added in float32 on the CUDA cores.  Two TMEM accumulators
// (128 columns each) alternate: the MMAs of one slab overlap the draining of
// the previous one.
constexpr int SLAB = 2;

template <bool BF>
__global__ void __launch_bounds__(NT, 1) tc_gemm_split_kernel(
    const __grid_constant__ CUtensorMap mapAh, const __grid_constant__ CUtensorMap mapAl,
    const __grid_constant__ CUtensorMap mapBh, const __grid_constant__ CUtensorMap mapBl, float* __restrict__ C,
    int64_t ldc, int M, int N, int K, int* __restrict__ err, const TileSkip sk) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* base = reinterpret_cast<unsigned char*>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    __shared__ __align__(8) uint64_t full_bar[STAGES32], empty_bar[STAGES32], accf[2], acce[2], drain_bar;
    __shared__ uint32_t tmem_slot;
    __shared__ int abort_flag;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.x * BM, n0 = blockIdx.y * BN;
    constexpr int KB = BF ? BK : BK32;           // K values per 128-byte slab
    const int nk = (K + KB - 1) / KB;
    const int nslab = (nk + SLAB - 1) / SLAB;

    // leave (uniformly, before any barrier or TMEM use) when no column of
    // this tile belongs to a block that needs the product
    if (sk.flag) {
        const int b_lo = sk.colblk[n0], b_hi = sk.colblk[min(n0 + BN, N) - 1];
        bool any = false;
        for (int b = b_lo; b <= b_hi; ++b) any |= sk.flag[b] != 0;
        if (!any) return;
    }

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES32; ++s) {
            mbar_init(&full_bar[s], 1);
            mbar_init(&empty_bar[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&accf[b], 1);
            mbar_init(&acce[b], 4);
        }
        mbar_init(&drain_bar, 1);
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(&tmem_slot)),
                     "r"(2 * BN));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n");
    const uint32_t tmem = tmem_slot;

    if (warp == 0) {
        if (lane == 0) {
            int issued = 0;
            for (int kb = 0; kb < nk; ++kb) {
                const int s = kb % STAGES32;
                if (kb >= STAGES32 && !mbar_wait(&empty_bar[s], ((kb / STAGES32) - 1) & 1, err)) {
                    abort_flag = 1;
                    break;
                }
                if (abort_flag) break;
                unsigned char* st = base + s * STAGE_BYTES32;
                mbar_expect_tx(&full_bar[s], STAGE_BYTES32);
                tma_load_2d(st, &mapAh, kb * KB, m0, &full_bar[s]);
                tma_load_2d(st + TILE_BYTES, &mapAl, kb * KB, m0, &full_bar[s]);
                tma_load_2d(st + 2 * TILE_BYTES, &mapBh, kb * KB, n0, &full_bar[s]);
                tma_load_2d(st + 3 * TILE_BYTES, &mapBl, kb * KB, n0, &full_bar[s]);
                issued = kb + 1;
            }
            if (abort_flag) {
                for (int kb = issued - STAGES32 < 0 ? 0 : issued - STAGES32; kb < issued; ++kb)
                    mbar_wait(&full_bar[kb % STAGES32], (kb / STAGES32) & 1, err);
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            constexpr uint32_t idesc = BF ? idesc_bf16(BM, BN) : idesc_tf32(BM, BN);
            bool ok = true;
            for (int kb = 0; kb < nk && ok; ++kb) {
                const int s = kb % STAGES32;
                const int slab = kb / SLAB, buf = slab & 1, in_slab = kb % SLAB;
                // the epilogue must have drained this accumulator (slab - 2)
                if (in_slab == 0 && slab >= 2 && !mbar_wait(&acce[buf], ((slab >> 1) - 1) & 1, err)) ok = false;
                if (ok && (!mbar_wait(&full_bar[s], (kb / STAGES32) & 1, err) || abort_flag)) ok = false;
                if (!ok) break;
                asm volatile("tcgen05.fence::after_thread_sync;\n");
                const uint32_t acc = tmem + (uint32_t)(buf * BN);
                const uint32_t ah = smem_u32(base + s * STAGE_BYTES32);
                const uint32_t al = ah + TILE_BYTES, bh = ah + 2 * TILE_BYTES, bl = ah + 3 * TILE_BYTES;
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const uint32_t off = k * 32;    // 32 bytes along K: 8 float32 or 16 bf16
                    const uint64_t dah = smem_desc(ah + off), dal = smem_desc(al + off);
                    const uint64_t dbh = smem_desc(bh + off), dbl = smem_desc(bl + off);
                    const uint32_t accum = (in_slab > 0 || k > 0) ? 1u : 0u;
                    // small terms first, the hi x hi term last
                    if constexpr (BF) {
                        asm volatile(
                            "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
                            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(acc),
                            "l"(dal), "l"(dbh), "r"(idesc), "r"(accum));
                        asm volatile("tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, 1;\n" ::"r"(acc),
                                     "l"(dah), "l"(dbl), "r"(idesc));
                        asm volatile("tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, 1;\n" ::"r"(acc),
                                     "l"(dah), "l"(dbh), "r"(idesc));
                    } else {
                        asm volatile(
                            "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
                            " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(acc),
                            "l"(dal), "l"(dbh), "r"(idesc), "r"(accum));
                        asm volatile("tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, 1;\n" ::"r"(acc),
                                     "l"(dah), "l"(dbl), "r"(idesc));
                        asm volatile("tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, 1;\n" ::"r"(acc),
                                     "l"(dah), "l"(dbh), "r"(idesc));
                    }
                }
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                                 smem_u32(&empty_bar[s]))
                             : "memory");
                if (in_slab == SLAB - 1 || kb == nk - 1)
                    asm volatile(
                        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                            smem_u32(&accf[buf]))
                        : "memory");
            }
            if (!ok) {
                abort_flag = 1;
                // every MMA issued so far completes before TMEM is released
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                                 smem_u32(&drain_bar))
                             : "memory");
                mbar_wait(&drain_bar, 0, err);
            }
        }
    } else {
        // epilogue warps 2..5 own TMEM lane quadrants (warp % 4): one row of
        // the tile per thread, its 128 columns summed slab by slab in float32
        const int q = warp & 3;
        float sum[BN];
#pragma unroll
        for (int j = 0; j < BN; ++j) sum[j] = 0.f;
        bool ok = true;
        for (int slab = 0; slab < nslab; ++slab) {
            const int buf = slab & 1;
            ok = __all_sync(0xffffffffu, ok && mbar_wait(&accf[buf], (slab >> 1) & 1, err) && !abort_flag);
            if (!ok) break;
            asm volatile("tcgen05.fence::after_thread_sync;\n");
#pragma unroll
            for (int c0 = 0; c0 < BN; c0 += 16) {
                uint32_t v[16];
                const uint32_t taddr = tmem + (uint32_t)(buf * BN) + ((uint32_t)(q * 32) << 16) + (uint32_t)c0;
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, "
                    "%13, %14, %15}, [%16];\n"
                    : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                      "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]),
                      "=r"(v[15])
                    : "r"(taddr));
                asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
                for (int j = 0; j < 16; ++j) sum[c0 + j] += __uint_as_float(v[j]);
            }
            asm volatile("tcgen05.fence::before_thread_sync;\n");
            __syncwarp();
            if (lane == 0) mbar_arrive(&acce[buf]);
        }
        const int row = m0 + q * 32 + lane;
        if (ok && row < M) {
#pragma unroll
            for (int j = 0; j < BN; ++j) {
                const int col = n0 + j;
                if (col < N) C[row + (int64_t)col * ldc] = sum[j];
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n");
    __syncthreads();
    if (warp == 1) {
        asm volatile("tcgen05.fence::after_thread_sync;\n");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(2 * BN));
    }
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    // looked up once (thread-safe static initialisation: solves may run on
    // several host threads at once)
    static const PFN_cuTensorMapEncodeTiled_v12000 fn = []() -> PFN_cuTensorMapEncodeTiled_v12000 {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
        return nullptr;
    }();
    return fn;
}

// 2-D bf16 tensor map over a K-major operand: inner dimension K (ld elements
// per row), outer dimension `rows`; 64 x 128 boxes, 128-byte swizzle, zero fill
bool make_map(CUtensorMap* map, const void* ptr, int64_t K, int64_t rows, int64_t ld, bool f32 = false,
              int box_rows = BM) {
    auto fn = encode_fn();
    if (!fn) return false;
    const int esz = f32 ? 4 : 2;
    cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)(ld * esz)};
    cuuint32_t box[2] = {(cuuint32_t)(f32 ? BK32 : BK), (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    return fn(map, f32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(ptr),
              dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
              CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

size_t tc_gemm_smem_bytes() { return (size_t)PSTAGES * PSTAGE_BYTES + 1024; }

namespace {
cudaError_t tc_launch(const void* A, int64_t lda, const void* B, int64_t ldb, float* C, int64_t ldc, int M, int N,
                      int K, int* err, const TcAbsmax& am, cudaStream_t s) {
    if (M <= 0 || N <= 0 || K <= 0) return cudaSuccess;
    if ((lda % 8) || (ldb % 8) || (reinterpret_cast<uintptr_t>(A) % 16) || (reinterpret_cast<uintptr_t>(B) % 16))
        return cudaErrorInvalidValue;
    CUtensorMap ma, mb;
    if (!make_map(&ma, A, K, M, lda) || !make_map(&mb, B, K, N, ldb, false, PBN)) return cudaErrorInvalidValue;
    const int64_t ntiles = (int64_t)ceil_div(M, BM) * ceil_div(N, PBN);
    if (ntiles > (1LL << 30)) return cudaErrorInvalidValue;
    static std::atomic<uint64_t> smem_set{0};
    const cudaError_t ea = ensure_smem_limit(tc_gemm_kernel, (int)tc_gemm_smem_bytes(), smem_set);
    if (ea != cudaSuccess) return ea;
    int dev = 0, nsm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    // one CTA per SM (the 193 KB ring admits no second one)
    const unsigned grid = (unsigned)std::min<int64_t>(ntiles, std::max(1, nsm));
    tc_gemm_kernel<<<grid, NT, tc_gemm_smem_bytes(), s>>>(ma, mb, C, ldc, M, N, K, err, am);
    return cudaGetLastError();
}
}  // namespace

namespace {
template <bool BF>
cudaError_t split_launch(const void* Ahi, const void* Alo, int64_t lda, const void* Bhi, const void* Blo, int64_t ldb,
                         float* C, int64_t ldc, int M, int N, int K, const int* colblk, const int* flag, int* err,
                         cudaStream_t s) {
    if (M <= 0 || N <= 0 || K <= 0) return cudaSuccess;
    const int64_t align = BF ? 8 : 4;               // 16-byte row strides
    if ((lda % align) || (ldb % align)) return cudaErrorInvalidValue;
    for (const void* p : {Ahi, Alo, Bhi, Blo})
        if (reinterpret_cast<uintptr_t>(p) % 16) return cudaErrorInvalidValue;
    if (flag && !colblk) return cudaErrorInvalidValue;
    CUtensorMap mah, mal, mbh, mbl;
    if (!make_map(&mah, Ahi, K, M, lda, !BF) || !make_map(&mal, Alo, K, M, lda, !BF) ||
        !make_map(&mbh, Bhi, K, N, ldb, !BF) || !make_map(&mbl, Blo, K, N, ldb, !BF))
        return cudaErrorInvalidValue;
    if (ceil_div(N, BN) > 65535) return cudaErrorInvalidValue;
    const size_t smem = (size_t)STAGES32 * STAGE_BYTES32 + 1024;
    static std::atomic<uint64_t> smem_set{0};
    const cudaError_t ea = ensure_smem_limit(tc_gemm_split_kernel<BF>, (int)smem, smem_set);
    if (ea != cudaSuccess) return ea;
    const dim3 grid((unsigned)ceil_div(M, BM), (unsigned)ceil_div(N, BN));
    tc_gemm_split_kernel<BF><<<grid, NT, smem, s>>>(mah, mal, mbh, mbl, C, ldc, M, N, K, err, TileSkip{colblk, flag});
    return cudaGetLastError();
}
}  // namespace

cudaError_t tc_gemm_3xtf32(const float* Ahi, const float* Alo, int64_t lda, const float* Bhi, const float* Blo,
                           int64_t ldb, float* C, int64_t ldc, int M, int N, int K, const int* colblk,
                           const int* flag, int* err, cudaStream_t s) {
    return split_launch<false>(Ahi, Alo, lda, Bhi, Blo, ldb, C, ldc, M, N, K, colblk, flag, err, s);
}

cudaError_t tc_gemm_bf16x3(const void* Ahi, const void* Alo, int64_t lda, const void* Bhi, const void* Blo,
                           int64_t ldb, float* C, int64_t ldc, int M, int N, int K, int* err, cudaStream_t s) {
    return split_launch<true>(Ahi, Alo, lda, Bhi, Blo, ldb, C, ldc, M, N, K, nullptr, nullptr, err, s);
}

cudaError_t tc_gemm_bf16(const void* A, int64_t lda, const void* B, int64_t ldb, float* C, int64_t ldc, int M, int N,
                         int K, int* err, cudaStream_t s) {
    return tc_launch(A, lda, B, ldb, C, ldc, M, N, K, err, TcAbsmax{nullptr, nullptr, nullptr, nullptr}, s);
}

cudaError_t tc_gemm_bf16_absmax(const void* A, int64_t lda, const void* B, int64_t ldb, int M, int N, int K,
                                TcAbsmax am, int* err, cudaStream_t s) {
    if (!am.colblk || !am.need || !am.bmax) return cudaErrorInvalidValue;
    return tc_launch(A, lda, B, ldb, nullptr, 0, M, N, K, err, am, s);
}

}  // namespace lrr
