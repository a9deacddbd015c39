// tc_update.cu -- persistent tcgen05 kernel for the AdaRBFGS factor update
//   L += S^ V      (Eq. (Cholimprov): S^ = S C^-T is n x q, V is q x n)
// with single-pass TF32 products: the correction vanishes at the fixed point
// (V = 0 when L L^T = A^-1), so its rounding shrinks with the error.
//
// The pass is bound by HBM (read L once, write L once).  Each CTA owns a
// contiguous run of 128 x 64 output tiles, row block by row block:
//   warp 0     TMA: the S^ row block (128 x q, K-major, 128-byte swizzle) once
//              per row block; per tile a V tile (64 x q) and the L tile
//              (128 x 64, column-major) into a two-deep ring;
//   warp 1     tcgen05.mma kind::tf32, K = q, into one of two TMEM
//              accumulators (64 columns each), so the MMA of tile i+1 runs
//              while tile i drains;
//   warps 4-7  drain the accumulator (thread = row), add it to the L tile in
//              shared memory and TMA-store the tile back.
// All mbarrier waits are bounded; a wait that gives up records ST_TIMEOUT
// in the caller's status word and the CTA winds down.
#include <algorithm>

#include "tc.cuh"
#include "tc_ptx.cuh"

using namespace tcx;

namespace {

constexpr int UBN = 64;                      // tile columns
constexpr int L_TILE_BYTES = 128 * UBN * 4;  // 32 KB, column-major

template <int KC>  // K = q padded to KC x 32
struct UCfg {
    static constexpr int SH_BYTES = KC * 128 * 128;  // KC chunks of 128 rows x 128 B
    static constexpr int V_BYTES = KC * UBN * 128;   // KC chunks of 64 rows x 128 B
    static constexpr int STAGE_BYTES = V_BYTES + L_TILE_BYTES;
    static constexpr int SMEM = SH_BYTES + 2 * STAGE_BYTES + 1024 + 256;
};

template <int KC>
__global__ void __launch_bounds__(256, 1)
k_tc_update(const __grid_constant__ CUtensorMap tmSh, const __grid_constant__ CUtensorMap tmV,
            const __grid_constant__ CUtensorMap tmL, int ncb, int ntiles, const int *status, int *err)
{
    using CF = UCfg<KC>;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    if (status_bad(status)) return;  // uniform across the CTA
    unsigned char *smem = (unsigned char *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    unsigned char *sh = smem;
    unsigned char *stg = smem + CF::SH_BYTES;
    uint64_t *bars = (uint64_t *)(stg + 2 * CF::STAGE_BYTES);
    uint64_t *full = bars;        // [2] V + L tile landed
    uint64_t *sempty = bars + 2;  // [2] stage released (tile stored)
    uint64_t *afull = bars + 4;   // [2] accumulator written
    uint64_t *aempty = bars + 6;  // [2] accumulator drained
    uint64_t *shfull = bars + 8;  // S^ row block landed
    uint64_t *shfree = bars + 9;  // MMAs reading the previous S^ block done
    uint32_t *tmem_slot = (uint32_t *)(bars + 10);
    volatile int *abort_flag = (volatile int *)(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int tb = (int)((long long)ntiles * blockIdx.x / gridDim.x);
    const int te = (int)((long long)ntiles * (blockIdx.x + 1) / gridDim.x);
    const int nt = te - tb;

    if (threadIdx.x == 0) {
        for (int s = 0; s < 2; ++s) {
            mbar_init(smem_u32(&full[s]), 1);
            mbar_init(smem_u32(&sempty[s]), 1);
            mbar_init(smem_u32(&afull[s]), 1);
            mbar_init(smem_u32(&aempty[s]), 128);
        }
        mbar_init(smem_u32(shfull), 1);
        mbar_init(smem_u32(shfree), 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(128u)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        if (lane == 0) {
            int cur_rb = -1, sh_loads = 0;
            for (int i = 0; i < nt; ++i) {
                const int t = tb + i, rb = t / ncb, cb = t - rb * ncb, s = i & 1;
                if (rb != cur_rb) {
                    if (sh_loads > 0 && !mbar_wait(smem_u32(shfree), (sh_loads - 1) & 1, err, abort_flag)) break;
                    const uint32_t fb = smem_u32(shfull);
                    mbar_expect_tx(fb, CF::SH_BYTES);
                    for (int kc = 0; kc < KC; ++kc) tma_load_2d(smem_u32(sh + kc * 16384), &tmSh, 32 * kc, rb * 128, fb);
                    cur_rb = rb;
                    ++sh_loads;
                }
                if (i >= 2 && !mbar_wait(smem_u32(&sempty[s]), ((i >> 1) - 1) & 1, err, abort_flag)) break;
                unsigned char *st = stg + s * CF::STAGE_BYTES;
                const uint32_t fb = smem_u32(&full[s]);
                mbar_expect_tx(fb, CF::STAGE_BYTES);
                for (int kc = 0; kc < KC; ++kc) tma_load_2d(smem_u32(st + kc * 8192), &tmV, 32 * kc, cb * UBN, fb);
                tma_load_2d(smem_u32(st + CF::V_BYTES), &tmL, rb * 128, cb * UBN, fb);
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            const uint32_t idesc = idesc_tf32(UBN, 0);
            const uint32_t sh_u = smem_u32(sh);
            int cur_rb = -1, sh_loads = 0;
            for (int i = 0; i < nt; ++i) {
                const int t = tb + i, rb = t / ncb, s = i & 1, b = i & 1;
                if (rb != cur_rb) {
                    if (!mbar_wait(smem_u32(shfull), sh_loads & 1, err, abort_flag)) break;
                    ++sh_loads;
                    cur_rb = rb;
                }
                if (!mbar_wait(smem_u32(&full[s]), (i >> 1) & 1, err, abort_flag)) break;
                if (i >= 2 && !mbar_wait(smem_u32(&aempty[b]), ((i >> 1) - 1) & 1, err, abort_flag)) break;
                tc_fence_after();
                const uint32_t v_u = smem_u32(stg + s * CF::STAGE_BYTES);
#pragma unroll
                for (int kc = 0; kc < KC; ++kc)
#pragma unroll
                    for (int k8 = 0; k8 < 4; ++k8) {
                        const uint64_t da = umma_desc(sh_u + kc * 16384 + k8 * 32, 16, 1024);
                        const uint64_t db = umma_desc(v_u + kc * 8192 + k8 * 32, 16, 1024);
                        mma_tf32(tmem + (uint32_t)(b * UBN), da, db, idesc, (kc | k8) ? 1u : 0u);
                    }
                mma_commit(smem_u32(&afull[b]));
                const bool last_of_rb = (i == nt - 1) || ((t + 1) / ncb != rb);
                if (last_of_rb) mma_commit(smem_u32(shfree));
            }
        }
    } else if (warp >= 4) {
        const int r = threadIdx.x - 128;  // tile row = TMEM lane
        const int wq = warp & 3;
        for (int i = 0; i < nt; ++i) {
            const int t = tb + i, rb = t / ncb, cb = t - rb * ncb, s = i & 1, b = i & 1;
            if (!mbar_wait(smem_u32(&afull[b]), (i >> 1) & 1, err, abort_flag)) break;
            if (!mbar_wait(smem_u32(&full[s]), (i >> 1) & 1, err, abort_flag)) break;
            tc_fence_after();
            float *Ls = (float *)(stg + s * CF::STAGE_BYTES + CF::V_BYTES);  // [64 cols][128 rows]
#pragma unroll
            for (int c0 = 0; c0 < UBN; c0 += 16) {
                uint32_t v[16];
                tmem_ld16(tmem + ((uint32_t)(32 * wq) << 16) + (uint32_t)(b * UBN + c0), v);
#pragma unroll
                for (int j = 0; j < 16; ++j) Ls[(c0 + j) * 128 + r] += __uint_as_float(v[j]);
            }
            tc_fence_before();
            mbar_arrive(smem_u32(&aempty[b]));
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            named_bar(1, 128);
            if (r == 0) {
                tma_store_2d(&tmL, smem_u32(Ls), rb * 128, cb * UBN);
                bulk_commit();
                bulk_wait_read0();
                mbar_arrive(smem_u32(&sempty[s]));
            }
        }
        if (r == 0) bulk_wait0();
    }
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(128u) : "memory");
    }
}

template <int KC>
int launch_update(cudaStream_t st, const CUtensorMap &ms, const CUtensorMap &mv, const CUtensorMap &ml, int n,
                  const int *status, int *err)
{
    using CF = UCfg<KC>;
    static bool attr = false;
    if (!attr) {
        if (cudaFuncSetAttribute(k_tc_update<KC>, cudaFuncAttributeMaxDynamicSharedMemorySize, CF::SMEM) !=
            cudaSuccess)
            return -1;
        attr = true;
    }
    const int nrb = (n + 127) / 128, ncb = (n + UBN - 1) / UBN;
    const int ntiles = nrb * ncb;
    const int grid = std::min(ntiles, tc_num_sms());
    rb_count_launch();
    k_tc_update<KC><<<grid, 256, CF::SMEM, st>>>(ms, mv, ml, ncb, ntiles, status, err);
    return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

}  // namespace

int tc_update_persistent(tc_plan *p, cudaStream_t st, int n, int q, const float *ShT, const float *V, float *L,
                         int64_t ldl, const int *status)
{
    (void)p;
    if (q < 1 || q > 128 || (q % 4) || (ldl % 4) || ((uintptr_t)ShT % 16) || ((uintptr_t)V % 16) ||
        ((uintptr_t)L % 16))
        return 1;
    CUtensorMap ms, mv, ml;
    if (!tc_make_map(&ms, ShT, q, n, q, 32, 128, 1) || !tc_make_map(&mv, V, q, n, q, 32, UBN, 1) ||
        !tc_make_map(&ml, L, n, n, ldl, 128, UBN, 0))
        return -4;
    int *err = const_cast<int *>(status);
    switch ((q + 31) / 32) {
    case 1: return launch_update<1>(st, ms, mv, ml, n, status, err);
    case 2: return launch_update<2>(st, ms, mv, ml, n, status, err);
    case 3: return launch_update<3>(st, ms, mv, ml, n, status, err);
    default: return launch_update<4>(st, ms, mv, ml, n, status, err);
    }
}
