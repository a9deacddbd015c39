// tc_update_s.cu -- AdaRBFGS factor update fused with the next step's sketch
// product (Eq. (Cholimprov) and the first line of Algorithm 4):
//
//   L+ = L + S^ V               (optional: do_update = 0 only forms S)
//   S_next = L+ S~_next         (S~_next exact in TF32: two products, L+ = hi + lo)
//
// Every L tile that the update streams through HBM is also the A operand of
// its share of S_next = sum over column tiles of L+(rows, cols) S~_next(cols, :),
// so the next step needs no separate pass over L.  Each CTA owns a contiguous
// run of 128 x 64 tiles of L, row block by row block (as in tc_update.cu):
//   warp 0      TMA: L tile (128 x 64) into the L half of a two-deep ring (released
//               as soon as the epilogue has read it);
//   warp 2      TMA: V tile (64 x q) into the V half of the ring (released by the
//               update MMAs) and the S~_next tile (64 rows x q) into its own slot;
//   warp 1      tcgen05.mma: L-tile update (A = S^ row block in TMEM, B = V) into
//               one of two accumulators;
//   warp 3      tcgen05.mma: the S_next product of each tile as soon as its L+ is
//               in TMEM (A = L+ hi / lo, B = S~_next), chunked every 8 tiles
//               (a thread's commits track its own MMAs, so the two streams of
//               MMAs are ordered independently);
//   warps 4-7   per tile: read the L rows (which frees the L half of the slot),
//               add the update accumulator and write L+ into TMEM, as hi (the FP32
//               value, which the MMA truncates) and lo = L+ - hi, for the S_next
//               MMA; refill S^ in TMEM when the row block changes;
//   warps 8-11  per tile: read L+ back from TMEM, stage it in the warp's own
//               32-row output buffer and TMA-store it from there; per chunk: drain
//               the S_next accumulator, keep running sums (FP32, round-to-nearest),
//               and write one partial 128 x q block per row block that the CTA
//               touches; the warp that is last to finish its quarter of a row block
//               (an atomic count per row block and quarter) adds the partials of the
//               CTAs that share the row block in CTA order and writes S_next (and its
//               lo part when asked); these warps take registers from warps 0-3
//               (setmaxnreg) for the q running sums.
// TMEM: update accumulators [0, 128), S^ [128, 256), L+ hi [256, 320),
// L+ lo [320, 384), S_next accumulator [384, 512).
// All mbarrier waits are bounded; a wait that gives up records ST_TIMEOUT and
// the CTA winds down.
#include <cuda_bf16.h>

#include <algorithm>

#include "tc.cuh"
#include "tc_ptx.cuh"

using namespace tcx;

namespace {

constexpr int UBN = 64;                      // tile columns
constexpr int L_TILE_BYTES = 128 * UBN * 4;  // 32 KB, column-major
constexpr int NSTAGES = 2;
constexpr int TSLOTS = 2;                    // S~_next tiles in flight
constexpr int SCHUNK = 8;                    // tiles per S_next accumulation chunk (512 of K)
constexpr uint32_t COL_SH = 128, COL_LHI = 256, COL_LLO = 320, COL_SACC = 384;
// Registers per thread: 168 at launch (384 threads); warps 0-3 drop to REG_ISSUE and warps 8-11
// (running sums of S_next, NQ per thread) rise to REG_DRAIN: 128 x (128 + 168 + 192) <= 384 x 168.
constexpr int REG_ISSUE = 128, REG_DRAIN = 192;
static_assert(128 * (REG_ISSUE + 168 + REG_DRAIN) <= 384 * 168, "register split");

template <int KC>  // q padded to NQ = 32 KC
struct SCfg {
    static constexpr int NQ = KC * 32;
    static constexpr int V_BYTES = KC * UBN * 128;  // KC chunks of 64 rows x 128 B
    static constexpr int STAGE_BYTES = V_BYTES + L_TILE_BYTES;
    static constexpr int T_BYTES = 2 * NQ * 128;     // two 32-wide K chunks of NQ rows x 128 B
    static constexpr int OUT_BYTES = 4 * 32 * UBN * 4;  // one 32-row L+ block per epilogue warp
    static constexpr int SMEM = NSTAGES * STAGE_BYTES + TSLOTS * T_BYTES + OUT_BYTES + 1024 + 256;
    static_assert(SMEM <= 227 * 1024, "shared memory");
};

__device__ __forceinline__ void st16(uint32_t taddr, const uint32_t (&r)[16])
{
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16};" ::"r"(taddr),
        "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]), "r"(r[8]), "r"(r[9]),
        "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15])
        : "memory");
}

__device__ __forceinline__ void mma_ts(uint32_t d_tmem, uint32_t a_tmem, uint64_t b, uint32_t idesc, uint32_t acc)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n\t}\n" ::"r"(d_tmem),
        "r"(a_tmem), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}

__device__ __forceinline__ float hi_tf32(float x) { return __uint_as_float(__float_as_uint(x) & 0xFFFFE000u); }

template <int KC>
__global__ void __launch_bounds__(384, 1)
k_tc_update_s(const float *__restrict__ ShT, int n, int q, const __grid_constant__ CUtensorMap tmV,
              const __grid_constant__ CUtensorMap tmL, const __grid_constant__ CUtensorMap tmLo,
              const __grid_constant__ CUtensorMap tmT, int ncb, int ntiles,
              int do_update, float *Spart, int *rb_cnt, int maxseg, float *S, float *Slo, int64_t lds,
              const int *status, int *err, __nv_bfloat16 *Sbf, int64_t ldbf)
{
    using CF = SCfg<KC>;
    constexpr int NQ = CF::NQ;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    if (status_bad(status)) return;  // uniform across the CTA
    unsigned char *smem = (unsigned char *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    unsigned char *stg = smem;
    unsigned char *tsl = smem + NSTAGES * CF::STAGE_BYTES;  // S~_next tile
    float *outb = (float *)(tsl + TSLOTS * CF::T_BYTES);  // [4 warps][64 cols][32 rows]
    uint64_t *bars = (uint64_t *)((unsigned char *)outb + CF::OUT_BYTES);
    uint64_t *lfull_s = bars;                // [2] L tile landed
    uint64_t *lempty_s = bars + NSTAGES;     // [2] L tile read by the epilogue
    uint64_t *vfull = bars + 2 * NSTAGES;    // [2] V tile landed
    uint64_t *vempty = bars + 3 * NSTAGES;   // [2] V tile read by the update MMAs
    uint64_t *afull = bars + 4 * NSTAGES;    // [2] update accumulator written
    uint64_t *aempty = afull + 2;            // [2] update accumulator drained
    uint64_t *tfull = aempty + 2;            // [TSLOTS] S~_next tile landed
    uint64_t *tempty = tfull + TSLOTS;       // [TSLOTS] S~_next tile read (S_next MMA done)
    uint64_t *lfull = tempty + TSLOTS;       // L+ hi / lo written to TMEM
    uint64_t *lempty = lfull + 1;            // L+ read (S_next MMA done, L+ staged for the store)
    uint64_t *shfull = lempty + 1;           // S^ written to TMEM
    uint64_t *shfree = shfull + 1;           // update MMAs reading S^ done
    uint64_t *sfull = shfree + 1;            // S_next chunk accumulated
    uint64_t *sfree = sfull + 1;             // S_next chunk drained
    uint32_t *tmem_slot = (uint32_t *)(sfree + 1);
    volatile int *abort_flag = (volatile int *)(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int tb = (int)((long long)ntiles * blockIdx.x / gridDim.x);
    const int te = (int)((long long)ntiles * (blockIdx.x + 1) / gridDim.x);
    const int nt = te - tb;
    const int rb_first = tb / ncb;

    if (threadIdx.x == 0) {
        for (int s = 0; s < NSTAGES; ++s) {
            mbar_init(smem_u32(&lfull_s[s]), 1);
            mbar_init(smem_u32(&lempty_s[s]), 4);  // one arrival per epilogue warp
            mbar_init(smem_u32(&vfull[s]), 1);
            mbar_init(smem_u32(&vempty[s]), 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(smem_u32(&afull[b]), 1);
            mbar_init(smem_u32(&aempty[b]), 128);
        }
        for (int s = 0; s < TSLOTS; ++s) {
            mbar_init(smem_u32(&tfull[s]), 1);
            mbar_init(smem_u32(&tempty[s]), 1);
        }
        mbar_init(smem_u32(lfull), 128);
        mbar_init(smem_u32(lempty), 1 + 4);  // the S_next MMA commit and one arrival per store warp
        mbar_init(smem_u32(shfull), 128);
        mbar_init(smem_u32(shfree), 1);
        mbar_init(smem_u32(sfull), 1);
        mbar_init(smem_u32(sfree), 128);
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
    const uint32_t tmem = *tmem_slot;
    // Tile i of this CTA's run is (row block rb, column block cb); every role advances the pair
    // with its loop index instead of dividing by ncb per tile.
    const int cb_first = tb - rb_first * ncb;
    auto next_tile = [&](int &rb, int &cb) {
        if (++cb == ncb) {
            cb = 0;
            ++rb;
        }
    };
    // S_next chunking: a tile's position in this CTA's run of its row block, and whether it ends it
    auto seg_pos = [&](int i, int rb, int cb) { return rb == rb_first ? i : cb; };
    auto last_of_rb = [&](int i, int cb) { return i + 1 == nt || cb + 1 == ncb; };

    if (warp < 4) {
        // single-thread roles: give registers to the S_next drain warps
        asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;" ::"n"(REG_ISSUE));
        if (warp == 0) {
            // ---------------- TMA: L tiles ----------------
            if (lane == 0) {
                int rb = rb_first, cb = cb_first;
                for (int i = 0; i < nt; ++i, next_tile(rb, cb)) {
                    const int s = i % NSTAGES;
                    if (i >= NSTAGES && !mbar_wait(smem_u32(&lempty_s[s]), ((i / NSTAGES) - 1) & 1, err, abort_flag))
                        break;
                    const uint32_t fb = smem_u32(&lfull_s[s]);
                    mbar_expect_tx(fb, L_TILE_BYTES);
                    tma_load_2d(smem_u32(stg + s * CF::STAGE_BYTES + CF::V_BYTES), &tmL, rb * 128, cb * UBN, fb);
                }
            }
        } else if (warp == 2) {
            // ---------------- TMA: V tiles and S~_next tiles (rows cb * 64 .. + 63) ----------------
            if (lane == 0) {
                int rb = rb_first, cb = cb_first;
                for (int i = 0; i < nt; ++i, next_tile(rb, cb)) {
                    const int ts = i % TSLOTS, s = i % NSTAGES;
                    if (do_update) {
                        if (i >= NSTAGES && !mbar_wait(smem_u32(&vempty[s]), ((i / NSTAGES) - 1) & 1, err, abort_flag))
                            break;
                        const uint32_t vb = smem_u32(&vfull[s]);
                        mbar_expect_tx(vb, CF::V_BYTES);
                        for (int kc = 0; kc < KC; ++kc)
                            tma_load_2d(smem_u32(stg + s * CF::STAGE_BYTES + kc * 8192), &tmV, 32 * kc, cb * UBN, vb);
                    }
                    if (i >= TSLOTS && !mbar_wait(smem_u32(&tempty[ts]), ((i / TSLOTS) - 1) & 1, err, abort_flag)) break;
                    const uint32_t fb = smem_u32(&tfull[ts]);
                    unsigned char *tp = tsl + ts * CF::T_BYTES;
                    mbar_expect_tx(fb, CF::T_BYTES);
                    tma_load_2d(smem_u32(tp), &tmT, cb * UBN, 0, fb);
                    tma_load_2d(smem_u32(tp + NQ * 128), &tmT, cb * UBN + 32, 0, fb);
                }
            }
        } else if (warp == 3) {
            // ---------------- MMA issuer for the S_next products (own thread, own commits) ----------------
            if (lane == 0) {
                const uint32_t idesc_s = idesc_tf32(NQ, 0);
                int chunk = -1;  // S_next chunk being accumulated
                bool ok = true;
                // S_next product of tile j (L+ of tile j in TMEM, S~_next tile j in smem)
                auto s_mma = [&](int j, int rb, int cb) {
                    const int p = seg_pos(j, rb, cb);
                    const bool cstart = (p % SCHUNK) == 0;
                    const bool cend = ((p + 1) % SCHUNK) == 0 || last_of_rb(j, cb);
                    if (cstart) {
                        ++chunk;
                        if (chunk >= 1 && !mbar_wait(smem_u32(sfree), (chunk - 1) & 1, err, abort_flag)) {
                            ok = false;
                            return;
                        }
                    }
                    const int ts = j % TSLOTS;
                    if (!mbar_wait(smem_u32(lfull), j & 1, err, abort_flag) ||
                        !mbar_wait(smem_u32(&tfull[ts]), (j / TSLOTS) & 1, err, abort_flag)) {
                        ok = false;
                        return;
                    }
                    tc_fence_after();
                    const uint32_t t_u = smem_u32(tsl + ts * CF::T_BYTES);
    #pragma unroll
                    for (int kk = 0; kk < UBN / 8; ++kk) {
                        const uint64_t db = umma_desc(t_u + (kk >> 2) * (NQ * 128) + (kk & 3) * 32, 16, 1024);
                        mma_ts(tmem + COL_SACC, tmem + COL_LLO + 8 * kk, db, idesc_s, (cstart && kk == 0) ? 0u : 1u);
                        mma_ts(tmem + COL_SACC, tmem + COL_LHI + 8 * kk, db, idesc_s, 1u);
                    }
                    mma_commit(smem_u32(lempty));
                    mma_commit(smem_u32(&tempty[ts]));
                    if (cend) mma_commit(smem_u32(sfull));
                };
                int rb = rb_first, cb = cb_first;
                for (int j = 0; j < nt && ok; ++j, next_tile(rb, cb)) s_mma(j, rb, cb);
            }
        } else if (warp == 1) {
            // ---------------- MMA issuer for the L-tile update ----------------
            if (lane == 0 && do_update) {
                const uint32_t idesc_u = idesc_tf32(UBN, 0);
                int cur_rb = -1;
                int rb = rb_first, cb = cb_first;
                for (int i = 0; i < nt; ++i, next_tile(rb, cb)) {
                    const int s = i % NSTAGES, b = i & 1;
                    {
                        if (rb != cur_rb) {
                            const int k = rb - rb_first;  // S^ refills of this CTA
                            if (!mbar_wait(smem_u32(shfull), k & 1, err, abort_flag)) break;
                            cur_rb = rb;
                        }
                        if (!mbar_wait(smem_u32(&vfull[s]), (i / NSTAGES) & 1, err, abort_flag)) break;
                        if (i >= 2 && !mbar_wait(smem_u32(&aempty[b]), ((i >> 1) - 1) & 1, err, abort_flag)) break;
                        tc_fence_after();
                        const uint32_t v_u = smem_u32(stg + s * CF::STAGE_BYTES);
    #pragma unroll
                        for (int kc = 0; kc < KC; ++kc)
    #pragma unroll
                            for (int k8 = 0; k8 < 4; ++k8) {
                                const uint64_t db = umma_desc(v_u + kc * 8192 + k8 * 32, 16, 1024);
                                mma_ts(tmem + (uint32_t)(b * UBN), tmem + COL_SH + 32 * kc + 8 * k8, db, idesc_u,
                                       (kc | k8) ? 1u : 0u);
                            }
                        mma_commit(smem_u32(&afull[b]));
                        mma_commit(smem_u32(&vempty[s]));
                        if (last_of_rb(i, cb)) mma_commit(smem_u32(shfree));
                    }
                }
            }
        }
    } else if (warp < 8) {
        // ---------------- L tile epilogue, L+ into TMEM, S^ refills ----------------
        const int r = threadIdx.x - 128;  // tile row = TMEM lane
        const uint32_t lane_base = tmem + ((uint32_t)(32 * (warp & 3)) << 16);
        bool ok = true;
        // waits agree across the warp (the TMEM accesses and the stage release are warp-wide)
        auto wwait = [&](uint64_t *bar, uint32_t par) {
            return __all_sync(0xffffffffu, mbar_wait(smem_u32(bar), par, err, abort_flag));
        };
        auto load_sh = [&](int rb) {  // S^ rows of row block rb into TMEM (rows past n are zero)
            const int k = rb - rb_first;
            if (k >= 1 && !wwait(shfree, (k - 1) & 1)) {
                ok = false;
                return;
            }
            tc_fence_after();
            const int row = rb * 128 + r;
            const float4 *src = (const float4 *)(ShT + (size_t)row * q);
            // 32 columns per batch: all loads of a batch are in flight together
#pragma unroll
            for (int b0 = 0; b0 < KC * 32; b0 += 32) {
                float4 v[8];
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const int c = b0 + 4 * j;
                    v[j] = make_float4(0.f, 0.f, 0.f, 0.f);
                    if (row < n && c < q) v[j] = src[c >> 2];  // q % 4 == 0
                }
#pragma unroll
                for (int c0 = 0; c0 < 32; c0 += 16) {
                    uint32_t w[16];
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        const float4 x = v[(c0 >> 2) + j];
                        w[4 * j] = __float_as_uint(x.x);
                        w[4 * j + 1] = __float_as_uint(x.y);
                        w[4 * j + 2] = __float_as_uint(x.z);
                        w[4 * j + 3] = __float_as_uint(x.w);
                    }
                    st16(lane_base + COL_SH + b0 + c0, w);
                }
            }
            asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
            tc_fence_before();
            mbar_arrive(smem_u32(shfull));
        };
        if (do_update && nt > 0) load_sh(rb_first);
        int rb = rb_first, cb = cb_first;
        for (int i = 0; i < nt && ok; ++i, next_tile(rb, cb)) {
            const int s = i % NSTAGES, b = i & 1;
            // the L row first (shared memory), then the accumulator (TMEM, one wait for all loads)
            if (!wwait(&lfull_s[s], (i / NSTAGES) & 1)) break;
            const float *Ls = (const float *)(stg + s * CF::STAGE_BYTES + CF::V_BYTES);  // [64 cols][128 rows]
            float lp[UBN];
#pragma unroll
            for (int c = 0; c < UBN; ++c) lp[c] = Ls[c * 128 + r];
            // The stage is released before the values are used, so make every lane wait for its loads
            // first: an instruction that reads all 64 registers cannot issue until they have arrived
            // (an arrival right after the loads were issued let the next TMA load overwrite rows still
            // being read in the BF16 GEMM's converter).
            uint32_t dep = 0;
#pragma unroll
            for (int c = 0; c < UBN; ++c) dep |= __float_as_uint(lp[c]);
            asm volatile("" ::"r"(dep));
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_u32(&lempty_s[s]));  // the L tile is in registers
            if (do_update) {
                if (!wwait(&afull[b], (i >> 1) & 1)) break;
                tc_fence_after();
                const uint32_t ta = lane_base + (uint32_t)(b * UBN);
                // the accumulator in two 32-column halves (one wait each)
#pragma unroll
                for (int hc = 0; hc < UBN; hc += 32) {
                    uint32_t v[32];
#pragma unroll
                    for (int c0 = 0; c0 < 32; c0 += 16)
                        asm volatile(
                            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
                            "%11, %12, %13, %14, %15}, [%16];"
                            : "=r"(v[c0]), "=r"(v[c0 + 1]), "=r"(v[c0 + 2]), "=r"(v[c0 + 3]), "=r"(v[c0 + 4]),
                              "=r"(v[c0 + 5]), "=r"(v[c0 + 6]), "=r"(v[c0 + 7]), "=r"(v[c0 + 8]), "=r"(v[c0 + 9]),
                              "=r"(v[c0 + 10]), "=r"(v[c0 + 11]), "=r"(v[c0 + 12]), "=r"(v[c0 + 13]),
                              "=r"(v[c0 + 14]), "=r"(v[c0 + 15])
                            : "r"(ta + hc + c0));
                    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
                    for (int c = 0; c < 32; ++c) lp[hc + c] += __uint_as_float(v[c]);
                }
                tc_fence_before();
                mbar_arrive(smem_u32(&aempty[b]));
            }
            // L+ of this tile as the A operand of its S_next product (after the previous one is read)
            if (i >= 1 && !wwait(lempty, (i - 1) & 1)) break;
            tc_fence_after();
#pragma unroll
            for (int c0 = 0; c0 < UBN; c0 += 16) {
                uint32_t w[16];
#pragma unroll
                for (int j = 0; j < 16; ++j) w[j] = __float_as_uint(lp[c0 + j]);
                st16(lane_base + COL_LHI + c0, w);
#pragma unroll
                for (int j = 0; j < 16; ++j) w[j] = __float_as_uint(lp[c0 + j] - hi_tf32(lp[c0 + j]));
                st16(lane_base + COL_LLO + c0, w);
            }
            asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
            tc_fence_before();
            mbar_arrive(smem_u32(lfull));
            // the update MMAs of this row block are done once its last tile drained: refill S^
            if (do_update && last_of_rb(i, cb) && i + 1 < nt) load_sh(rb + 1);
        }
    } else {
        asm volatile("setmaxnreg.inc.sync.aligned.u32 %0;" ::"n"(REG_DRAIN));
        // ---------------- L+ stores and S_next chunks ----------------
        const int wq = warp & 3;
        const uint32_t lane_base = tmem + ((uint32_t)(32 * wq) << 16);
        float *ow = outb + wq * (32 * UBN);  // [64 cols][32 rows]
        auto wwait = [&](uint64_t *bar, uint32_t par) {
            return __all_sync(0xffffffffu, mbar_wait(smem_u32(bar), par, err, abort_flag));
        };
        float run[NQ];
#pragma unroll
        for (int j = 0; j < NQ; ++j) run[j] = 0.f;
        int c = 0;
        int rb = rb_first, cb = cb_first;
        for (int i = 0; i < nt; ++i, next_tile(rb, cb)) {
            const int p = seg_pos(i, rb, cb);
            // L+ of tile i (the hi slot holds the FP32 value) to the output buffer, then one TMA store
            if (!wwait(lfull, i & 1)) break;
            tc_fence_after();
            if (do_update) {
                if (lane == 0) bulk_wait_read0();  // the previous store has read the buffer
                __syncwarp();
#pragma unroll
                for (int c0 = 0; c0 < UBN; c0 += 32) {
#pragma unroll
                    for (int c1 = c0; c1 < c0 + 32; c1 += 16) {
                        uint32_t v0[16];
                        tmem_ld16(lane_base + COL_LHI + c1, v0);
#pragma unroll
                        for (int j = 0; j < 16; ++j) ow[(c1 + j) * 32 + lane] = __uint_as_float(v0[j]);
                    }
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_u32(lempty));
            if (do_update) {
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                __syncwarp();
                if (lane == 0 && rb * 128 + 32 * wq < n) {  // a block wholly past row n stores nothing
                    tma_store_2d(&tmLo, smem_u32(ow), rb * 128 + 32 * wq, cb * UBN);
                    bulk_commit();
                }
            }
            // S_next chunk ends with tile i: running sums; a row block's last chunk writes its partial block
            if (((p + 1) % SCHUNK) == 0 || last_of_rb(i, cb)) {
                if (!wwait(sfull, c & 1)) break;
                tc_fence_after();
                const uint32_t keep = (p < SCHUNK) ? 0u : 0xFFFFFFFFu;  // a row block starts a fresh sum
#pragma unroll
                for (int c0 = 0; c0 < NQ; c0 += 16) {
                    uint32_t v[16];
                    tmem_ld16(lane_base + COL_SACC + c0, v);
#pragma unroll
                    for (int j = 0; j < 16; ++j)
                        run[c0 + j] = __uint_as_float(__float_as_uint(run[c0 + j]) & keep) + __uint_as_float(v[j]);
                }
                tc_fence_before();
                mbar_arrive(smem_u32(sfree));
                ++c;
                if (last_of_rb(i, cb)) {  // partial block (rows x NQ, column-major, ld 128)
                    const int seg = rb - rb_first;
                    float *dst = Spart + ((size_t)blockIdx.x * maxseg + seg) * (128 * NQ) + 32 * wq + lane;
#pragma unroll
                    for (int j = 0; j < NQ; ++j) dst[j * 128] = run[j];
                    // CTAs whose tile runs meet the row block: b0 .. b1
                    auto cta_of = [&](int tile) {
                        int cb = (int)((long long)tile * gridDim.x / ntiles);
                        while (cb + 1 < (int)gridDim.x && (long long)ntiles * (cb + 1) / gridDim.x <= tile) ++cb;
                        while (cb > 0 && (long long)ntiles * cb / gridDim.x > tile) --cb;
                        return cb;
                    };
                    const int b0 = cta_of(rb * ncb), b1 = cta_of(min(rb * ncb + ncb, ntiles) - 1);
                    __threadfence();
                    __syncwarp();
                    int old = 0;
                    if (lane == 0) old = atomicAdd(&rb_cnt[4 * rb + wq], 1);
                    old = __shfl_sync(0xffffffffu, old, 0);
                    if (old == b1 - b0) {  // every other partial of this quarter is written: S_next rows
                        if (lane == 0) rb_cnt[4 * rb + wq] = 0;  // ready for the next launch
                        __threadfence();
#pragma unroll
                        for (int j = 0; j < NQ; ++j) run[j] = 0.f;
                        for (int bb = b0; bb <= b1; ++bb) {
                            const int sg = rb - (int)((long long)ntiles * bb / gridDim.x) / ncb;
                            const float *pp = Spart + ((size_t)bb * maxseg + sg) * (128 * NQ) + 32 * wq + lane;
#pragma unroll
                            for (int j = 0; j < NQ; ++j) run[j] += __ldcg(pp + j * 128);
                        }
                        const int row = rb * 128 + 32 * wq + lane;
                        if (row < n)
#pragma unroll
                            for (int j = 0; j < NQ; ++j)
                                if (j < q) {
                                    S[row + (int64_t)j * lds] = run[j];
                                    if (Slo) Slo[row + (int64_t)j * lds] = run[j] - hi_tf32(run[j]);  // for a 3-term product
                                    if (Sbf) {  // BF16 hi and lo, for a BF16-split product
                                        const __nv_bfloat16 hb = __float2bfloat16_rn(run[j]);
                                        Sbf[row + (int64_t)j * ldbf] = hb;
                                        Sbf[(int64_t)q * ldbf + row + (int64_t)j * ldbf] =
                                            __float2bfloat16_rn(run[j] - __bfloat162float(hb));
                                    }
                                }
                    }
                }
            }
        }
        if (lane == 0) bulk_wait0();
        tc_fence_before();
    }
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512u) : "memory");
    }
}

template <int KC>
int launch_update_s(cudaStream_t st, const float *ShT, int n, int q, const CUtensorMap &mv, const CUtensorMap &ml,
                    const CUtensorMap &mlo,
                    const CUtensorMap &mt, int do_update, float *Spart, size_t spart_elems, float *S, float *Slo,
                    int64_t lds, const int *status, int *err, void *Sbf, int64_t ldbf, int reserve_sms)
{
    using CF = SCfg<KC>;
    static bool attr = false;
    if (!attr) {
        if (cudaFuncSetAttribute(k_tc_update_s<KC>, cudaFuncAttributeMaxDynamicSharedMemorySize, CF::SMEM) !=
            cudaSuccess)
            return -1;
        // the register split raises warps 8-11 out of what the CTA holds: refuse a
        // build whose launch count leaves too few (setmaxnreg.inc would never return)
        cudaFuncAttributes fa;
        if (cudaFuncGetAttributes(&fa, k_tc_update_s<KC>) != cudaSuccess ||
            384 * fa.numRegs < 128 * (REG_ISSUE + 168 + REG_DRAIN))
            return -1;
        attr = true;
    }
    const int nrb = (n + 127) / 128, ncb = (n + UBN - 1) / UBN;
    const int ntiles = nrb * ncb;
    // reserve_sms SMs stay free for work on other streams
    const int grid = std::min(ntiles, std::max(1, tc_num_sms() - std::max(0, std::min(reserve_sms, 8))));
    int maxseg = 1;
    for (int b = 0; b < grid; ++b) {
        const long long t0 = (long long)ntiles * b / grid, t1 = (long long)ntiles * (b + 1) / grid;
        if (t1 > t0) maxseg = std::max(maxseg, (int)((t1 - 1) / ncb - t0 / ncb + 1));
    }
    // workspace: arrival counts (4 per row block, zero between launches) then the partial blocks
    const size_t cnt_floats = ((size_t)4 * nrb + 31) / 32 * 32;
    if (cnt_floats + (size_t)grid * maxseg * 128 * CF::NQ > spart_elems) return -2;
    rb_count_launch();
    k_tc_update_s<KC><<<grid, 384, CF::SMEM, st>>>(ShT, n, q, mv, ml, mlo, mt, ncb, ntiles, do_update,
                                                   Spart + cnt_floats, (int *)Spart, maxseg, S, Slo, lds, status,
                                                   err, (__nv_bfloat16 *)Sbf, ldbf);
    return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

}  // namespace

size_t tc_update_s_workspace(int n, int q)
{
    // the partial blocks of every grid a launch may use (all SMs but 0 .. 8 reserved): the
    // largest CTAs x (row blocks a CTA's tile run meets)
    const int nrb = (n + 127) / 128, ncb = (n + UBN - 1) / UBN, ntiles = nrb * ncb;
    size_t blocks = 0;
    for (int r = 0; r <= 8; ++r) {
        const int grid = std::min(ntiles, std::max(1, tc_num_sms() - r));
        int maxseg = 1;
        for (int b = 0; b < grid; ++b) {
            const long long t0 = (long long)ntiles * b / grid, t1 = (long long)ntiles * (b + 1) / grid;
            if (t1 > t0) maxseg = std::max(maxseg, (int)((t1 - 1) / ncb - t0 / ncb + 1));
        }
        blocks = std::max(blocks, (size_t)grid * maxseg);
    }
    const size_t cnt_floats = ((size_t)4 * nrb + 31) / 32 * 32;  // arrival counts (as int)
    return cnt_floats + blocks * 128 * (size_t)(((q + 31) / 32) * 32);
}

int tc_update_next_s(cudaStream_t st, int n, int q, const float *ShT, const float *V, float *L, int64_t ldl,
                     const float *St_next, float *S_out, int do_update, float *Spart, size_t spart_elems,
                     const int *status, float *S_lo, void *S_bf, int64_t ld_bf, int reserve_sms)
{
    if (S_bf && (ld_bf < n || ld_bf % 8)) return 1;
    if (q < 1 || q > 128 || (q % 4) || (ldl % 4) || (n % 4) || ((uintptr_t)ShT % 16) || ((uintptr_t)V % 16) ||
        ((uintptr_t)L % 16) || ((uintptr_t)St_next % 16) || ((uintptr_t)S_lo % 16))
        return 1;
    CUtensorMap mv, ml, mlo, mt;
    const int nq = ((q + 31) / 32) * 32;
    if (!tc_make_map(&mv, V, q, n, q, 32, UBN, 1) || !tc_make_map(&ml, L, n, n, ldl, 128, UBN, 0) ||
        !tc_make_map(&mlo, L, n, n, ldl, 32, UBN, 0) ||
        !tc_make_map(&mt, St_next, n, q, n, 32, nq, 1))
        return -4;
    int *err = const_cast<int *>(status);
    switch (nq / 32) {
    case 1: return launch_update_s<1>(st, ShT, n, q, mv, ml, mlo, mt, do_update, Spart, spart_elems, S_out, S_lo, n, status, err, S_bf, ld_bf, reserve_sms);
    case 2: return launch_update_s<2>(st, ShT, n, q, mv, ml, mlo, mt, do_update, Spart, spart_elems, S_out, S_lo, n, status, err, S_bf, ld_bf, reserve_sms);
    case 3: return launch_update_s<3>(st, ShT, n, q, mv, ml, mlo, mt, do_update, Spart, spart_elems, S_out, S_lo, n, status, err, S_bf, ld_bf, reserve_sms);
    default:
        return launch_update_s<4>(st, ShT, n, q, mv, ml, mlo, mt, do_update, Spart, spart_elems, S_out, S_lo, n, status, err, S_bf, ld_bf, reserve_sms);
    }
}
