// common.cuh -- shared device helpers of the sm_103a library.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>

#include "rbfgs.h"

// Device status word bits (rb_ctx::d_status).  Kernels that modify the
// iterate return early when any bit is set, so a failed step and every later
// step leave X / L untouched.
enum : int {
    ST_NOTSPD = 1,     // Cholesky pivot <= 0 or non-finite
    ST_NONFINITE = 2,  // non-finite value in a q x q core
    ST_TIMEOUT = 4,    // a bounded device-side wait gave up
};

#define RB_CUDA(call)                                   \
    do {                                                \
        cudaError_t e_ = (call);                        \
        if (e_ != cudaSuccess) return RB_ECUDA;         \
    } while (0)

#define RB_TRY(call)                                    \
    do {                                                \
        rb_status s_ = (call);                          \
        if (s_ != RB_OK) return s_;                     \
    } while (0)

__device__ __forceinline__ bool status_bad(const int *st) { return st != nullptr && *(volatile const int *)st != 0; }

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11): ten rounds of two
// 32x32 -> 64 multiplies per 4-word block, key bumped by the Weyl increments
// between rounds.  Counter words: (w0, w1, k_lo, stream_lo); key = seed.
// ---------------------------------------------------------------------------
struct u32x4 {
    uint32_t x, y, z, w;
};

__host__ __device__ __forceinline__ u32x4 philox10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                                   uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        const uint64_t m0 = (uint64_t)0xD2511F53u * c0;
        const uint64_t m1 = (uint64_t)0xCD9E8D57u * c2;
        const uint32_t n0 = (uint32_t)(m1 >> 32) ^ c1 ^ k0;
        const uint32_t n2 = (uint32_t)(m0 >> 32) ^ c3 ^ k1;
        c1 = (uint32_t)m1;
        c3 = (uint32_t)m0;
        c0 = n0;
        c2 = n2;
    }
    return u32x4{c0, c1, c2, c3};
}

// Counter-word tags separating the draws of one (seed, stream, step).
constexpr uint32_t TAG_COORD = 0xC0000000u;  // coordinate-block / Floyd draws
constexpr uint32_t TAG_COLS = 0xD0000000u;   // residual column sample

// 24-bit uniform in (0,1): ((x >> 8) + 1/2) 2^-24 -- exact in FP32 and FP64.
__host__ __device__ __forceinline__ float u24f(uint32_t x) { return ((float)(x >> 8) + 0.5f) * (1.0f / 16777216.0f); }
__host__ __device__ __forceinline__ double u24d(uint32_t x) { return ((double)(x >> 8) + 0.5) * (1.0 / 16777216.0); }

inline int ceil_div(long long a, long long b) { return (int)((a + b - 1) / b); }

// Kernels launched by this library since load (host-side count, one per launch).
extern std::atomic<unsigned long long> g_rb_launches;
inline void rb_count_launch() { g_rb_launches.fetch_add(1, std::memory_order_relaxed); }
