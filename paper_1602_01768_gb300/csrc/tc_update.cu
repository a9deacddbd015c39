// tc_update.cu -- persistent tcgen05 kernel for the AdaRBFGS factor update
//   L += S^ V      (Eq. (Cholimprov): S^ = S C^-T is n x q, V is q x n)
// with single-pass TF32 products: the correction vanishes at the fixed point
// (V = 0 when L L^T = A^-1), so its rounding shrinks with the error.
//
// The pass is bound by HBM (read L once, write L once).  Each CTA owns a
// contiguous run of 128 x 64 output tiles, row block by row block:
//   warp 0     TMA: per tile a V tile (64 x q, K-major, 128-byte swizzle) and
//              the L tile (128 x 64, column-major) into a three-deep ring;
//   warp 1     tcgen05.mma kind::tf32, K = q, A = the S^ row block from TMEM,
//              into one of two TMEM accumulators (64 columns each), so the MMA
//              of tile i+1 runs while tile i drains;
//   warps 4-7  write the S^ row blocks into TMEM (two buffers, thread = row),
//              drain the accumulator, add it to the L tile in shared memory
//              and TMA-store the tile back.
// With S^ in TMEM the MMAs read only V from shared memory, which leaves room
// for the third stage of L tiles in flight.
// All mbarrier waits are bounded; a wait that gives up records ST_TIMEOUT
// in the caller's status word and the CTA winds down.
#include <algorithm>

#include "tc.cuh"
#include "tc_ptx.cuh"

using namespace tcx;

namespace {

constexpr int UBN = 64;                      // tile columns
constexpr int L_TILE_BYTES = 128 * UBN * 4;  // 32 KB, column-major
constexpr int USTAGES = 3;

template <int KC>  // K = q padded to KC x 32
struct UCfg {
    static constexpr int V_BYTES = KC * UBN * 128;  // KC chunks of 64 rows x 128 B
    static constexpr int STAGE_BYTES = V_BYTES + L_TILE_BYTES;
    static constexpr int SMEM = USTAGES * STAGE_BYTES + 1024 + 256;
    static constexpr int SH_COLS = KC * 32;  // TMEM columns of one S^ buffer
};

// 32 lanes x 16 columns of 32-bit values from registers into TMEM.
__device__ __forceinline__ void tmem_st16u(uint32_t taddr, const uint32_t (&r)[16])
{
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16};" ::"r"(taddr),
        "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]), "r"(r[8]), "r"(r[9]),
        "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15])
        : "memory");
}

__device__ __forceinline__ void mma_tf32_tsu(uint32_t d_tmem, uint32_t a_tmem, uint64_t b, uint32_t idesc,
                                             uint32_t acc)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n\t}\n" ::"r"(d_tmem),
        "r"(a_tmem), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}

template <int KC>
__global__ void __launch_bounds__(256, 1)
k_tc_update(const float *__restrict__ ShT, int n, int q, const __grid_constant__ CUtensorMap tmV,
            const __grid_constant__ CUtensorMap tmL, int ncb, int ntiles, const int *status, int *err)
{
    using CF = UCfg<KC>;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    if (status_bad(status)) return;  // uniform across the CTA
    unsigned char *smem = (unsigned char *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    unsigned char *stg = smem;
    uint64_t *bars = (uint64_t *)(stg + USTAGES * CF::STAGE_BYTES);
    uint64_t *full = bars;                  // [3] V + L tile landed
    uint64_t *sempty = bars + USTAGES;      // [3] stage released (tile stored)
    uint64_t *afull = bars + 2 * USTAGES;   // [2] accumulator written
    uint64_t *aempty = afull + 2;           // [2] accumulator drained
    uint64_t *shfull = aempty + 2;          // [2] S^ buffer written
    uint64_t *shfree = shfull + 2;          // [2] MMAs reading the S^ buffer done
    uint32_t *tmem_slot = (uint32_t *)(shfree + 2);
    volatile int *abort_flag = (volatile int *)(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int tb = (int)((long long)ntiles * blockIdx.x / gridDim.x);
    const int te = (int)((long long)ntiles * (blockIdx.x + 1) / gridDim.x);
    const int nt = te - tb;

    if (threadIdx.x == 0) {
        for (int s = 0; s < USTAGES; ++s) {
            mbar_init(smem_u32(&full[s]), 1);
            mbar_init(smem_u32(&sempty[s]), 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(smem_u32(&afull[b]), 1);
            mbar_init(smem_u32(&aempty[b]), 128);
            mbar_init(smem_u32(&shfull[b]), 128);
            mbar_init(smem_u32(&shfree[b]), 1);
        }
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(512u)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;  // accumulators: columns [0, 2 UBN); S^ buffers after them
    auto sh_col = [&](int sb) { return (uint32_t)(2 * UBN + sb * CF::SH_COLS); };

    if (warp == 0) {
        if (lane == 0) {
            for (int i = 0; i < nt; ++i) {
                const int t = tb + i, rb = t / ncb, cb = t - rb * ncb, s = i % USTAGES;
                if (i >= USTAGES &&
                    !mbar_wait(smem_u32(&sempty[s]), ((i / USTAGES) - 1) & 1, err, abort_flag))
                    break;
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
            int cur_rb = -1, ord = -1;  // row block and its ordinal in this CTA's run
            for (int i = 0; i < nt; ++i) {
                const int t = tb + i, rb = t / ncb, s = i % USTAGES, b = i & 1;
                if (rb != cur_rb) {
                    cur_rb = rb;
                    ++ord;
                    if (!mbar_wait(smem_u32(&shfull[ord & 1]), (ord >> 1) & 1, err, abort_flag)) break;
                }
                if (!mbar_wait(smem_u32(&full[s]), (i / USTAGES) & 1, err, abort_flag)) break;
                if (i >= 2 && !mbar_wait(smem_u32(&aempty[b]), ((i >> 1) - 1) & 1, err, abort_flag)) break;
                tc_fence_after();
                const uint32_t v_u = smem_u32(stg + s * CF::STAGE_BYTES);
                const uint32_t ta = tmem + sh_col(ord & 1);
#pragma unroll
                for (int kc = 0; kc < KC; ++kc)
#pragma unroll
                    for (int k8 = 0; k8 < 4; ++k8) {
                        const uint64_t db = umma_desc(v_u + kc * 8192 + k8 * 32, 16, 1024);
                        mma_tf32_tsu(tmem + (uint32_t)(b * UBN), ta + 32 * kc + 8 * k8, db, idesc,
                                     (kc | k8) ? 1u : 0u);
                    }
                mma_commit(smem_u32(&afull[b]));
                const bool last_of_rb = (i == nt - 1) || ((t + 1) / ncb != rb);
                if (last_of_rb) mma_commit(smem_u32(&shfree[ord & 1]));
            }
        }
    } else if (warp >= 4) {
        const int r = threadIdx.x - 128;  // tile row = TMEM lane
        const int wq = warp & 3;
        const uint32_t lane_base = tmem + ((uint32_t)(32 * wq) << 16);
        bool ok = true;
        // row block of ordinal k of this CTA's run (-1 past the end)
        const int rb_first = nt > 0 ? tb / ncb : 0, rb_last = nt > 0 ? (te - 1) / ncb : -1;
        auto load_sh = [&](int k) {  // S^ rows of that row block into buffer k & 1 (rows past n are zero)
            const int rb = rb_first + k;
            if (rb > rb_last) return;
            if (k >= 2 && !mbar_wait(smem_u32(&shfree[k & 1]), ((k >> 1) - 1) & 1, err, abort_flag)) {
                ok = false;
                return;
            }
            tc_fence_after();
            const int row = rb * 128 + r;
            const float4 *src = (const float4 *)(ShT + (size_t)row * q);
#pragma unroll
            for (int c0 = 0; c0 < KC * 32; c0 += 16) {
                uint32_t w[16];
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int c = c0 + 4 * j;
                    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
                    if (row < n && c < q) v = src[c >> 2];  // q % 4 == 0
                    w[4 * j] = __float_as_uint(v.x);
                    w[4 * j + 1] = __float_as_uint(v.y);
                    w[4 * j + 2] = __float_as_uint(v.z);
                    w[4 * j + 3] = __float_as_uint(v.w);
                }
                tmem_st16u(lane_base + sh_col(k & 1) + c0, w);
            }
            asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
            tc_fence_before();
            mbar_arrive(smem_u32(&shfull[k & 1]));
        };
        load_sh(0);
        load_sh(1);
        int ord = 0, cur_rb = rb_first;
        for (int i = 0; i < nt && ok; ++i) {
            const int t = tb + i, rb = t / ncb, cb = t - rb * ncb, s = i % USTAGES, b = i & 1;
            if (rb != cur_rb) {
                cur_rb = rb;
                ++ord;
            }
            if (!mbar_wait(smem_u32(&afull[b]), (i >> 1) & 1, err, abort_flag)) break;
            if (!mbar_wait(smem_u32(&full[s]), (i / USTAGES) & 1, err, abort_flag)) break;
            tc_fence_after();
            float *Ls = (float *)(stg + s * CF::STAGE_BYTES + CF::V_BYTES);  // [64 cols][128 rows]
#pragma unroll
            for (int c0 = 0; c0 < UBN; c0 += 16) {
                uint32_t v[16];
                tmem_ld16(lane_base + (uint32_t)(b * UBN + c0), v);
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
            // after the last tile of a row block its MMAs are complete: refill that buffer
            const bool last_of_rb = (i == nt - 1) || ((t + 1) / ncb != rb);
            if (last_of_rb) load_sh(ord + 2);
        }
        if (r == 0) bulk_wait0();
    }
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512u) : "memory");
    }
}

template <int KC>
int launch_update(cudaStream_t st, const float *ShT, int n, int q, const CUtensorMap &mv, const CUtensorMap &ml,
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
    k_tc_update<KC><<<grid, 256, CF::SMEM, st>>>(ShT, n, q, mv, ml, ncb, ntiles, status, err);
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
    CUtensorMap mv, ml;
    if (!tc_make_map(&mv, V, q, n, q, 32, UBN, 1) || !tc_make_map(&ml, L, n, n, ldl, 128, UBN, 0)) return -4;
    int *err = const_cast<int *>(status);
    switch ((q + 31) / 32) {
    case 1: return launch_update<1>(st, ShT, n, q, mv, ml, status, err);
    case 2: return launch_update<2>(st, ShT, n, q, mv, ml, status, err);
    case 3: return launch_update<3>(st, ShT, n, q, mv, ml, status, err);
    default: return launch_update<4>(st, ShT, n, q, mv, ml, status, err);
    }
}
