// tc.cu -- tcgen05 / TMA GEMM for sm_103a (see tc.cuh for the contract).
//
// Work is cut into units of one 128 x 32 k-block of one 128 x BN output tile.
// When the output has fewer tiles than the GPU has SMs the launch is
// stream-K: one CTA per SM, each taking an equal contiguous run of units in
// (tile, k-block) order; every piece of a tile that a CTA covers (a segment)
// is written as a partial tile, and the CTA that finishes a tile's last piece
// (an atomic count per tile and 32-row quarter tells it so) sums the pieces in
// CTA order and writes the output, so results are deterministic and no second
// kernel runs.  Otherwise each CTA owns one tile.
// Warp roles, 384 threads:
//   warp 0      TMA producer: streams 128 x 32 tiles of op(A) and BN x 32
//               tiles of B (and of B's lo part) with 128-byte swizzle into a
//               STAGES-deep ring;
//   warp 1      allocates TMEM and issues tcgen05.mma kind::tf32 from one
//               elected thread, B from shared memory (K-major);
//   warps 4-7   converter: each thread takes one row of the landed A tile and
//               writes to TMEM what the MMA reads from there: lo = x - hi(x)
//               for split products (hi = x itself: the MMA keeps the top 11
//               significand bits) and hi too for 3-term products and for an
//               M-contiguous op(A); a K-contiguous 2-term hi is read from
//               shared memory directly;
//   warps 8-11  drain the chunk accumulators (tcgen05.ld), keep the running
//               sums and write the output (and, on request, its lo part for a
//               later 3-term product) or stream-K partial tiles, and add the
//               pieces of a tile when they finish it; they take registers from
//               the other warps (setmaxnreg) for the BN running sums.
// A 3-term k-step issues two MMAs: hi x [B | B lo] of width 2 BN and lo x B
// (the MMA issue rate, not the arithmetic, bounds these products).
// Every mbarrier wait is bounded (about two seconds of SM clock); a wait
// that gives up records ST_TIMEOUT in the caller's status word and the CTA
// winds down instead of hanging.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <mutex>

#include "kernels.cuh"
#include "tc.cuh"
#include "tc_ptx.cuh"

namespace {
using namespace tcx;

// BF = 1: kind::f16 products on BF16 parts of the FP32 operands.  The A tile
// (FP32, K-contiguous) lands as two 128 x 32 boxes per 64-wide k-block and the
// converter writes its BF16 parts into TMEM, two K-consecutive values per
// 32-bit column (the lower K index in the low half); B comes pre-split as BF16
// hi and lo panels (64 BF16 = one 128-byte swizzle row).  x = hi + lo with
// hi = bf16(x), lo = bf16(x - hi) (round to nearest; A's lo rounds ties away
// from zero, B's to even): the 3-term product hi hi + hi lo + lo hi carries
// ~16 bits, each MMA covers K = 16.
template <int BN, int TERMS, int AMN, int BF = 0>
struct Cfg {
    // The A tile lands in shared memory by TMA; the converter warps write the
    // lo part (2 and 3 terms) into TMEM, and the hi part too for an
    // M-contiguous tile (transposed to lanes = rows) and for 3-term products.
    // With A in TMEM an MMA reads only B from shared memory: for 3 terms that
    // cuts the tensor core's shared-memory reads per k-block from 80 to 48 KB,
    // which is what held the two shared-memory-operand MMAs back (measured on
    // GB300: 0.31 against 0.36 ms for a 16384 x 16384 x 128 product).
    static constexpr bool HI_TMEM = AMN != 0 || TERMS == 3 || BF != 0;
    // A k-step of a 3-term product issues two MMAs instead of three: hi x [B | B lo]
    // is one MMA of width 2 BN (B lo follows B in the stage, so the two form one
    // K-major operand of 2 BN rows) and lo x B the other.  The MMA issue rate, not
    // the arithmetic, bounds these products on GB300 (halving N leaves the time of
    // a 16384 x 16384 x 128 product unchanged), so fewer, wider MMAs are faster.
    // The accumulator is then 2 BN columns wide ([hi B + lo B | hi B lo], summed by
    // the drain) and single-buffered.
    static constexpr bool PACK = TERMS == 3 && 2 * BN <= 256;
    static constexpr int ACC_COLS = PACK ? 2 * BN : BN;  // one accumulator
    static constexpr int NACC = PACK ? 1 : 2;            // accumulators (chunks alternate when 2)
    static constexpr bool LO_TMEM = TERMS >= 2;
    static constexpr bool CONVERT = HI_TMEM || LO_TMEM;
    static constexpr int LO_OFF = HI_TMEM ? 32 : 0;  // TMEM column of lo within a stage
    static constexpr int BKE = BF ? 64 : BK;          // K elements per k-block
    // k-blocks per accumulation chunk: 64 MMA steps either way (512 of K at K = 8 per TF32 MMA,
    // 1024 of K at K = 16 per BF16 MMA), so the drift each chunk bounds is the same
    static constexpr int CHUNK = BF ? 2 * CHUNK_KB * BK / BKE : CHUNK_KB * BK / BKE;
    static constexpr int A_BYTES = BM * BKE * 4;
    static constexpr int B_BYTES = BN * BKE * (BF ? 2 : 4);
    static constexpr int STAGE_BYTES = A_BYTES + B_BYTES * (TERMS == 3 ? 2 : 1);  // [A | B | B lo]
    static constexpr int A_TMEM_COLS = 32 * ((HI_TMEM ? 1 : 0) + (LO_TMEM ? 1 : 0));
    // TMEM: two chunk accumulators (2 BN columns), then the A stages
    static constexpr int STAGES_SMEM = (200 * 1024) / STAGE_BYTES;
    static constexpr int STAGES_TMEM = CONVERT ? (512 - NACC * ACC_COLS) / A_TMEM_COLS : 8;
    static constexpr int STAGES_A = STAGES_SMEM < STAGES_TMEM ? STAGES_SMEM : STAGES_TMEM;
    static constexpr int STAGES = STAGES_A > 8 ? 8 : STAGES_A;
    static constexpr int TMEM_COLS = CONVERT ? 512 : (2 * BN < 32 ? 32 : 2 * BN);
    // BF16 products run three decoupled rings: NA FP32 A slots in shared memory, freed by the
    // converter as soon as it has written the tile's BF16 parts into TMEM (so A streams NA
    // k-blocks deep), NBS slots of B's BF16 parts, freed when their MMAs complete, and NT TMEM
    // stages of A, freed when their MMAs complete.  Otherwise one ring of STAGES [A | B | B lo]
    // stages, each freed when its MMAs complete.
    static constexpr bool SPLIT = BF != 0;
    static constexpr int NA = SPLIT ? 3 : 0;
    static constexpr int NBS = SPLIT ? 4 : 0;  // B waits on the MMAs: one slot more than A (measured)
    static constexpr int NT = SPLIT ? (STAGES_TMEM < 4 ? STAGES_TMEM : 4) : 0;
    static constexpr int B2_BYTES = B_BYTES * (TERMS == 3 ? 2 : 1);  // B and its lo part
    static constexpr int RING_BYTES = SPLIT ? NA * A_BYTES + NBS * B2_BYTES : STAGES * STAGE_BYTES;
    static constexpr int SMEM = RING_BYTES + 1024 /*align*/ + 512 /*barriers*/;
    static_assert(STAGES >= 2, "pipeline needs two stages");
    static_assert(!SPLIT || (NT >= 2 && RING_BYTES <= 224 * 1024), "BF16 rings");
    static_assert(!BF || (AMN == 0 && TERMS != 2), "BF16 products: K-contiguous A, 1 or 3 terms");
};

__device__ __forceinline__ float tf32_hi(float x) { return __uint_as_float(__float_as_uint(x) & 0xFFFFE000u); }

// Register split of the GEMM CTA (setmaxnreg): warps 0-7 drop to GEMM_REG_LOW,
// the drain warps 8-11 rise to GEMM_REG_DRAIN.
constexpr int GEMM_REG_LOW = 120, GEMM_REG_DRAIN = 208;
static_assert(128 * (2 * GEMM_REG_LOW + GEMM_REG_DRAIN) <= 384 * 168, "register split");

// lo = x - hi(x), elementwise over a column-major rows x cols panel (ld).  The
// tensor core reads an FP32 operand of kind::tf32 as its top 19 bits (the low
// 13 mantissa bits are dropped, not rounded), so x itself serves as the hi part.
__global__ void k_split_lo(int rows, int cols, const float *X, int64_t ldx, float *L, int64_t ldl)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y;
    if (i < rows) {
        const float v = X[i + (int64_t)j * ldx];
        L[i + (int64_t)j * ldl] = v - tf32_hi(v);
    }
}

// 32 lanes x 16 columns of 32-bit values from registers into TMEM.
__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t (&r)[16])
{
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16};" ::"r"(taddr),
        "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]), "r"(r[8]), "r"(r[9]),
        "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15])
        : "memory");
}

// Instruction descriptor, kind::f16 with BF16 A and B (both the same type), D F32,
// A and B K-major, N = n, M = 128.
__host__ __device__ constexpr uint32_t idesc_bf16(int n)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
}

// D (TMEM) += A (TMEM, BF16 pairs: M rows on lanes, K/2 on columns) x B (smem descriptor, BF16).
__device__ __forceinline__ void mma_bf16_ts(uint32_t d_tmem, uint32_t a_tmem, uint64_t b, uint32_t idesc,
                                            uint32_t acc)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n\t}\n" ::"r"(d_tmem),
        "r"(a_tmem), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}

// D (TMEM) += A (TMEM, M rows on lanes, K on columns) x B (smem descriptor).
__device__ __forceinline__ void mma_tf32_ts(uint32_t d_tmem, uint32_t a_tmem, uint64_t b, uint32_t idesc,
                                            uint32_t acc)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n\t}\n" ::"r"(d_tmem),
        "r"(a_tmem), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}

// Half h (K columns 16h .. 16h + 15) of row m of the stage's raw A tile.
// K-contiguous tile: row m is 128 bytes with 16-byte chunk j stored at chunk
// j ^ (m & 7).  M-contiguous tile: four 32-row boxes 4 KB apart; element
// (m, k) in 16-byte chunk ((m & 31) / 4) ^ (k & 7) of the box's K-row k.
template <int AMN>
__device__ __forceinline__ void load_a_half(const unsigned char *raw, int m, int h, float (&v)[16])
{
    if (AMN) {
        const int mi = m & 31;
        const unsigned char *src = raw + (m >> 5) * 4096 + ((mi & 3) << 2);
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) {
            const int k = 16 * h + kk;
            v[kk] = *(const float *)(src + k * 128 + (((mi >> 2) ^ (k & 7)) << 4));
        }
    } else {
#pragma unroll
        for (int jj = 0; jj < 4; ++jj) {
            const int j = 4 * h + jj;
            const float4 f = *(const float4 *)(raw + m * 128 + ((j ^ (m & 7)) << 4));
            v[4 * jj] = f.x;
            v[4 * jj + 1] = f.y;
            v[4 * jj + 2] = f.z;
            v[4 * jj + 3] = f.w;
        }
    }
}

template <int BN, int TERMS, int AMN, int BF>
__global__ void __launch_bounds__(384, 1)
k_tc_gemm(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
          const __grid_constant__ CUtensorMap tmBlo, int M, int N, int mt, int nkb, long long U, int maxseg,
          float alpha, float beta, const float *Cin, int64_t ldcin, float *C, float *Clo, int64_t ldc, int ctrans,
          float *part, int *tile_cnt, const int *status, int *err, __nv_bfloat16 *Cbf, int64_t ldbf,
          long long bfhalf)
{
    using CF = Cfg<BN, TERMS, AMN, BF>;
    constexpr int STAGES = CF::STAGES;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    if (status_bad(status)) return;  // uniform: every thread reads the same word

    unsigned char *smem = (unsigned char *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    unsigned char *bar_area = smem + CF::RING_BYTES;
    // one ring: full / conv / empty per stage.  BF16 rings: full / empty per A slot (NA), conv /
    // tempty per TMEM stage (NT), bfull / bempty per B slot (NBS)
    constexpr int NFULL = CF::SPLIT ? CF::NA : STAGES, NCONV = CF::SPLIT ? CF::NT : STAGES;
    uint64_t *full = (uint64_t *)bar_area;
    uint64_t *conv = full + NFULL;
    uint64_t *empty = conv + NCONV;
    uint64_t *bfull = empty + NFULL;
    uint64_t *bempty = bfull + CF::NBS;
    uint64_t *tempty = bempty + CF::NBS;
    uint64_t *chunk_full = tempty + CF::NT;  // [2] accumulator b holds a finished K chunk
    uint64_t *chunk_free = chunk_full + 2;  // [2] accumulator b drained
    uint32_t *tmem_slot = (uint32_t *)(chunk_free + 2);
    volatile int *abort_flag = (volatile int *)(tmem_slot + 1);

    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    // This CTA's units [u_b, u_e): unit u is k-block u % nkb of tile u / nkb;
    // tile t covers rows (t % mt) BM and columns (t / mt) BN.  A segment is the
    // run of this CTA's units inside one tile; a chunk is at most CHUNK_KB
    // units of a segment, counted from the segment start.
    const int u_b = (int)(U * blockIdx.x / gridDim.x), u_e = (int)(U * (blockIdx.x + 1) / gridDim.x);
    const int nk = u_e - u_b;
    const int t_b = u_b / nkb, kb_b = u_b - t_b * nkb;

    if (threadIdx.x == 0) {
        for (int s = 0; s < NFULL; ++s) {
            mbar_init(smem_u32(&full[s]), 1);
            mbar_init(smem_u32(&empty[s]), CF::SPLIT ? 128 : 1);  // BF16: freed by the 128 converter threads
        }
        for (int s = 0; s < NCONV; ++s) mbar_init(smem_u32(&conv[s]), 128);
        for (int s = 0; s < CF::NBS; ++s) {
            mbar_init(smem_u32(&bfull[s]), 1);
            mbar_init(smem_u32(&bempty[s]), 1);
        }
        for (int s = 0; s < CF::NT; ++s) mbar_init(smem_u32(&tempty[s]), 1);
        for (int b = 0; b < 2; ++b) {
            mbar_init(smem_u32(&chunk_full[b]), 1);
            mbar_init(smem_u32(&chunk_free[b]), 128);
        }
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"((uint32_t)CF::TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;  // accumulators: columns [0, 2 BN); A stages after them

    auto stage_a = [&](int s) { return CF::SPLIT ? smem + s * CF::A_BYTES : smem + s * CF::STAGE_BYTES; };
    auto stage_b = [&](int s) {
        return CF::SPLIT ? smem + CF::NA * CF::A_BYTES + s * CF::B2_BYTES : smem + s * CF::STAGE_BYTES + CF::A_BYTES;
    };
    auto stage_blo = [&](int s) { return stage_b(s) + CF::B_BYTES; };
    auto a_col = [&](int s) { return (uint32_t)(CF::NACC * CF::ACC_COLS + s * CF::A_TMEM_COLS); };

    // registers: the drain warps keep BN running sums per thread; the single-thread
    // roles and the converter need far fewer.  The split must fit in what the CTA
    // was launched with (384 x 168; launch_bn checks the compiled count).
    constexpr int REG_LOW = GEMM_REG_LOW, REG_DRAIN = GEMM_REG_DRAIN;
    if (warp < 4) {
        asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;" ::"n"(REG_LOW));
        if (CF::SPLIT && (warp == 0 || warp == 2)) {
            // ---------------- TMA producers: A ring (warp 0), B ring (warp 2) ----------------
            if (lane == 0) {
                const bool ring_a = warp == 0;
                const int nslot = ring_a ? CF::NA : CF::NBS;
                uint64_t *f = ring_a ? full : bfull, *e = ring_a ? empty : bempty;
                int t = t_b, kb = kb_b, m0 = (t % mt) * BM, n0 = (t / mt) * BN;
                for (int i = 0; i < nk; ++i) {
                    const int s = i % nslot;
                    if (i >= nslot && !mbar_wait(smem_u32(&e[s]), ((i / nslot) - 1) & 1, err, abort_flag)) break;
                    const uint32_t fb = smem_u32(&f[s]);
                    const int k = kb * CF::BKE;
                    if (ring_a) {  // two 128 x 32 FP32 boxes per 64-wide k-block
                        mbar_expect_tx(fb, CF::A_BYTES);
                        tma_load_2d(smem_u32(stage_a(s)), &tmA, k, m0, fb);
                        tma_load_2d(smem_u32(stage_a(s) + A_TILE_BYTES), &tmA, k + BK, m0, fb);
                    } else {
                        mbar_expect_tx(fb, CF::B2_BYTES);
                        tma_load_2d(smem_u32(stage_b(s)), &tmB, k, n0, fb);
                        if (TERMS == 3) tma_load_2d(smem_u32(stage_blo(s)), &tmBlo, k, n0, fb);
                    }
                    if (++kb == nkb) {
                        kb = 0;
                        ++t;
                        m0 = (t % mt) * BM;
                        n0 = (t / mt) * BN;
                    }
                }
            }
        } else if (warp == 0) {
            // ---------------- TMA producer (warp 0) ----------------
            if (lane == 0) {
                int t = t_b, kb = kb_b, m0 = (t % mt) * BM, n0 = (t / mt) * BN;
                for (int i = 0; i < nk; ++i) {
                    const int s = i % STAGES;
                    if (i >= STAGES && !mbar_wait(smem_u32(&empty[s]), ((i / STAGES) - 1) & 1, err, abort_flag)) break;
                    const uint32_t fb = smem_u32(&full[s]);
                    mbar_expect_tx(fb, CF::STAGE_BYTES);
                    const int k = kb * CF::BKE;
                    if (BF) {  // two 128 x 32 FP32 boxes per 64-wide k-block
                        tma_load_2d(smem_u32(stage_a(s)), &tmA, k, m0, fb);
                        tma_load_2d(smem_u32(stage_a(s) + A_TILE_BYTES), &tmA, k + BK, m0, fb);
                    } else if (AMN) {
    #pragma unroll
                        for (int c = 0; c < BM / 32; ++c)
                            tma_load_2d(smem_u32(stage_a(s) + c * 4096), &tmA, m0 + 32 * c, k, fb);
                    } else {
                        tma_load_2d(smem_u32(stage_a(s)), &tmA, k, m0, fb);
                    }
                    tma_load_2d(smem_u32(stage_b(s)), &tmB, k, n0, fb);
                    if (TERMS == 3) tma_load_2d(smem_u32(stage_blo(s)), &tmBlo, k, n0, fb);  // B lo, split once per call
                    if (++kb == nkb) {
                        kb = 0;
                        ++t;
                        m0 = (t % mt) * BM;
                        n0 = (t / mt) * BN;
                    }
                }
            }
        } else if (warp == 1) {
            // ---------------- MMA issuer (warp 1) ----------------
            if (lane == 0) {
                const uint32_t idesc = idesc_tf32(BN, 0);
                const uint32_t idesc2 = idesc_tf32(CF::PACK ? 2 * BN : BN, 0);  // hi x [B | B lo]
                int c = -1;           // chunk being accumulated
                int kb = kb_b, p = 0;  // k-block in the tile, position in the segment
                for (int i = 0; i < nk; ++i) {
                    const int s = i % STAGES;
                    const bool cstart = (p % CF::CHUNK) == 0;
                    const bool cend = ((p + 1) % CF::CHUNK) == 0 || kb + 1 == nkb || i + 1 == nk;
                    if (cstart) ++c;
                    const int b = CF::NACC == 2 ? (c & 1) : 0;
                    if (CF::NACC == 2) {
                        if (cstart && c >= 2 && !mbar_wait(smem_u32(&chunk_free[b]), ((c >> 1) - 1) & 1, err, abort_flag))
                            break;
                    } else {
                        if (cstart && c >= 1 && !mbar_wait(smem_u32(&chunk_free[0]), (c - 1) & 1, err, abort_flag)) break;
                    }
                    // BF16 rings: the TMEM stage of A (converted) and the B slot; else the stage
                    const int st = CF::SPLIT ? i % CF::NT : s, sb = CF::SPLIT ? i % CF::NBS : s;
                    if (CF::SPLIT) {
                        if (!mbar_wait(smem_u32(&conv[st]), (i / CF::NT) & 1, err, abort_flag)) break;
                        if (!mbar_wait(smem_u32(&bfull[sb]), (i / CF::NBS) & 1, err, abort_flag)) break;
                    } else {
                        const uint32_t wb = CF::CONVERT ? smem_u32(&conv[s]) : smem_u32(&full[s]);
                        if (!mbar_wait(wb, (i / STAGES) & 1, err, abort_flag)) break;
                    }
                    tc_fence_after();
                    const uint32_t dacc = tmem + (uint32_t)(b * CF::ACC_COLS);
                    const uint32_t a_s = smem_u32(stage_a(s)), b_hi = smem_u32(stage_b(sb)), b_lo = smem_u32(stage_blo(sb));
                    const uint32_t ta = tmem + a_col(st);
                    if (BF) {
                        // K = 16 BF16 per MMA: 32 bytes along a 128-byte swizzle row of B, 8 TMEM columns of A
    #pragma unroll
                        for (int kk = 0; kk < CF::BKE / 16; ++kk) {
                            const uint64_t db = umma_desc(b_hi + kk * 32, 16, 1024);
                            const uint32_t first = (cstart && kk == 0) ? 0u : 1u;
                            if (CF::PACK) {
                                mma_bf16_ts(dacc, ta + 8 * kk, db, idesc_bf16(2 * BN), first);              // hi x [hi | lo]
                                mma_bf16_ts(dacc, ta + CF::LO_OFF + 8 * kk, db, idesc_bf16(BN), 1u);        // lo x hi
                            } else if (TERMS == 3) {
                                mma_bf16_ts(dacc, ta + CF::LO_OFF + 8 * kk, db, idesc_bf16(BN), first);     // lo x hi
                                mma_bf16_ts(dacc, ta + 8 * kk, umma_desc(b_lo + kk * 32, 16, 1024), idesc_bf16(BN),
                                            1u);                                                            // hi x lo
                                mma_bf16_ts(dacc, ta + 8 * kk, db, idesc_bf16(BN), 1u);                     // hi x hi
                            } else {
                                mma_bf16_ts(dacc, ta + 8 * kk, db, idesc_bf16(BN), first);
                            }
                        }
                    } else {
    #pragma unroll
                    for (int kk = 0; kk < BK / 8; ++kk) {
                        // K = 8 TF32 per MMA: 32 bytes along a 128-byte swizzle row, 8 TMEM columns
                        const uint64_t db_hi = umma_desc(b_hi + kk * 32, 16, 1024);
                        const uint32_t first = (cstart && kk == 0) ? 0u : 1u;  // each chunk starts a fresh sum
                        auto mma_hi = [&](uint64_t db, uint32_t accum, uint32_t id) {  // A hi x db
                            if (CF::HI_TMEM)
                                mma_tf32_ts(dacc, ta + 8 * kk, db, id, accum);
                            else
                                mma_tf32(dacc, umma_desc(a_s + kk * 32, 16, 1024), db, id, accum);
                        };
                        if (CF::PACK) {
                            mma_hi(db_hi, first, idesc2);                                      // hi x [hi | lo]
                            mma_tf32_ts(dacc, ta + CF::LO_OFF + 8 * kk, db_hi, idesc, 1u);     // lo x hi
                        } else if (TERMS == 3) {
                            mma_tf32_ts(dacc, ta + CF::LO_OFF + 8 * kk, db_hi, idesc, first);  // lo x hi
                            mma_hi(umma_desc(b_lo + kk * 32, 16, 1024), 1u, idesc);           // hi x lo
                            mma_hi(db_hi, 1u, idesc);                                          // hi x hi
                        } else if (TERMS == 2) {  // B exact in TF32
                            mma_tf32_ts(dacc, ta + CF::LO_OFF + 8 * kk, db_hi, idesc, first);  // lo x B
                            mma_hi(db_hi, 1u, idesc);                                          // hi x B
                        } else {
                            mma_hi(db_hi, first, idesc);
                        }
                    }
                    }
                    if (CF::SPLIT) {  // B slot and TMEM stage free once these MMAs complete
                        mma_commit(smem_u32(&bempty[sb]));
                        mma_commit(smem_u32(&tempty[st]));
                    } else {
                        mma_commit(smem_u32(&empty[s]));
                    }
                    if (cend) mma_commit(smem_u32(&chunk_full[b]));
                    ++p;
                    if (++kb == nkb) {
                        kb = 0;
                        p = 0;
                    }
                }
            }
        }
    } else if (warp < 8) {
        asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;" ::"n"(REG_LOW));
        // ---------------- converter (warps 4-7): A lo [and hi] into TMEM ----------------
        if (CF::CONVERT) {
            const int r = threadIdx.x - 128;  // tile row = TMEM lane
            const uint32_t lane_base = tmem + ((uint32_t)(32 * (warp & 3)) << 16);
            for (int i = 0; i < nk; ++i) {
                // BF16 rings: A slot s (NA deep) into TMEM stage st (NT deep, free once the MMAs of
                // k-block i - NT complete); else one stage index for both
                const int s = CF::SPLIT ? i % CF::NA : i % STAGES, st = CF::SPLIT ? i % CF::NT : s;
                if (!mbar_wait(smem_u32(&full[s]), (i / (CF::SPLIT ? CF::NA : STAGES)) & 1, err, abort_flag)) break;
                if (BF) {
                    // Row r's 64 FP32 values into registers.  The A slot is released only after they
                    // have been converted and stored: releasing it right after the loads (before the
                    // values were used) let the next TMA load overwrite rows still being read, and
                    // the products came out different from run to run.
                    float v[4][16];
#pragma unroll
                    for (int g = 0; g < 2; ++g)
#pragma unroll
                        for (int h = 0; h < 2; ++h) load_a_half<0>(stage_a(s) + g * A_TILE_BYTES, r, h, v[2 * g + h]);
                    if (CF::SPLIT && i >= CF::NT &&
                        !mbar_wait(smem_u32(&tempty[st]), ((i / CF::NT) - 1) & 1, err, abort_flag))
                        break;
                    const uint32_t taddr = lane_base + a_col(st);
                    // -> 32 columns of BF16 hi pairs (and 32 of lo pairs).  hi is rounded to nearest
                    // even by the conversion unit; lo = x - hi (exact in FP32) is rounded to nearest,
                    // ties away from zero, on the integer pipe (add half an ulp of BF16 to the bit
                    // pattern, keep the top 16 bits): the conversion unit runs at a fraction of the
                    // ALU rate, and one conversion per pair instead of two halves the converter's time.
#pragma unroll
                    for (int g = 0; g < 2; ++g) {  // one 128 x 32 box each
                        uint32_t wh[16], wl[16];
#pragma unroll
                        for (int h = 0; h < 2; ++h) {
#pragma unroll
                            for (int k = 0; k < 8; ++k) {
                                const float x0 = v[2 * g + h][2 * k], x1 = v[2 * g + h][2 * k + 1];
                                const __nv_bfloat162 hi = __floats2bfloat162_rn(x0, x1);
                                const uint32_t hb = *reinterpret_cast<const uint32_t *>(&hi);
                                const uint32_t l0 = __float_as_uint(x0 - __uint_as_float(hb << 16)) + 0x8000u;
                                const uint32_t l1 = __float_as_uint(x1 - __uint_as_float(hb & 0xFFFF0000u)) + 0x8000u;
                                wh[8 * h + k] = hb;
                                wl[8 * h + k] = __byte_perm(l0, l1, 0x7632);  // top halves: l0 low, l1 high
                            }
                        }
                        tmem_st16(taddr + 16 * g, wh);
                        if (CF::LO_TMEM) tmem_st16(taddr + CF::LO_OFF + 16 * g, wl);
                    }
                } else {
                if (CF::SPLIT && i >= CF::NT &&
                    !mbar_wait(smem_u32(&tempty[st]), ((i / CF::NT) - 1) & 1, err, abort_flag))
                    break;
                const uint32_t taddr = lane_base + a_col(st);
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    float v[16];
                    load_a_half<AMN>(stage_a(s), r, h, v);
                    uint32_t w[16];
                    if (CF::HI_TMEM) {
#pragma unroll
                        for (int k = 0; k < 16; ++k) w[k] = __float_as_uint(v[k]);
                        tmem_st16(taddr + 16 * h, w);
                    }
                    if (CF::LO_TMEM) {
#pragma unroll
                        for (int k = 0; k < 16; ++k) w[k] = __float_as_uint(v[k] - tf32_hi(v[k]));
                        tmem_st16(taddr + CF::LO_OFF + 16 * h, w);
                    }
                }
                }
                asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
                tc_fence_before();
                mbar_arrive(smem_u32(&conv[st]));
                if (CF::SPLIT) mbar_arrive(smem_u32(&empty[s]));  // A slot read: the producer may refill it
            }
        }
    } else {
        asm volatile("setmaxnreg.inc.sync.aligned.u32 %0;" ::"n"(REG_DRAIN));
        // ---------------- drain and epilogue (warps 8-11) ----------------
        // Running sum of the finished K chunks, one tile row per thread, added on
        // the CUDA cores with round-to-nearest.  The tensor core's FP32 accumulation
        // drifts toward zero over long K (about one truncation per MMA step, relative
        // to the growing sum); restarting it every CHUNK_KB k-blocks bounds that drift.
        const int wq = warp & 3;  // this warp's TMEM lane quarter
        float run[BN];
#pragma unroll
        for (int j = 0; j < BN; ++j) run[j] = 0.f;
        int u = u_b, t = t_b, kb = kb_b, c = 0;
        bool fresh = true;  // next chunk starts a segment
        while (u < u_e) {
            const int len = min(CF::CHUNK, min(nkb - kb, u_e - u));
            const int b = CF::NACC == 2 ? (c & 1) : 0;
            const uint32_t ph = CF::NACC == 2 ? ((c >> 1) & 1) : (c & 1);
            if (!__all_sync(0xffffffffu, mbar_wait(smem_u32(&chunk_full[b]), ph, err, abort_flag))) break;
            tc_fence_after();
            // the first chunk of a segment starts the sum: clear the running value by mask
            const uint32_t keep = fresh ? 0u : 0xFFFFFFFFu;
#pragma unroll
            for (int c0 = 0; c0 < BN; c0 += 16) {
                uint32_t rr[16];
                const uint32_t ta = tmem + ((uint32_t)(32 * wq) << 16) + (uint32_t)(b * CF::ACC_COLS + c0);
                if (CF::PACK) {  // both halves of the accumulator ([.. | hi x B lo]), one wait
                    uint32_t r2[16];
                    tmem_ld16_async(ta, rr);
                    tmem_ld16_async(ta + BN, r2);
                    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
                    for (int j = 0; j < 16; ++j) rr[j] = __float_as_uint(__uint_as_float(rr[j]) + __uint_as_float(r2[j]));
                } else {
                    tmem_ld16(ta, rr);
                }
#pragma unroll
                for (int j = 0; j < 16; ++j)
                    run[c0 + j] = __uint_as_float(__float_as_uint(run[c0 + j]) & keep) + __uint_as_float(rr[j]);
            }
            tc_fence_before();
            mbar_arrive(smem_u32(&chunk_free[b]));
            u += len;
            kb += len;
            ++c;
            fresh = (kb == nkb || u == u_e);
            if (fresh) {
                // segment finished.  Stream-K: write the partial tile into slot (CTA,
                // segment index) of the workspace; the warp whose quarter of the tile
                // is the last to arrive sums all pieces in CTA order and writes C.
                bool write_c = (part == nullptr);
                if (part != nullptr) {
                    float *dst = part + ((size_t)blockIdx.x * maxseg + (t - t_b)) * (BM * BN) + 32 * wq + lane;
#pragma unroll
                    for (int j = 0; j < BN; ++j) dst[j * BM] = run[j];
                    // CTAs whose units meet the tile: b0 (holds its first unit) .. b1 (its last)
                    const long long t0 = (long long)t * nkb, t1 = t0 + nkb;
                    auto cta_of = [&](long long unit) {
                        int cb = (int)(unit * gridDim.x / U);
                        while (cb + 1 < (int)gridDim.x && U * (cb + 1) / gridDim.x <= unit) ++cb;
                        while (cb > 0 && U * cb / gridDim.x > unit) --cb;
                        return cb;
                    };
                    const int b0 = cta_of(t0), b1 = cta_of(t1 - 1);
                    __threadfence();
                    __syncwarp();
                    int old = -1;  // split-K launch (no counts): a separate kernel adds the pieces
                    if (tile_cnt) {
                        if (lane == 0) old = atomicAdd(&tile_cnt[4 * t + wq], 1);
                        old = __shfl_sync(0xffffffffu, old, 0);
                    }
                    if (old == b1 - b0) {  // every other piece is written
                        if (lane == 0) tile_cnt[4 * t + wq] = 0;  // ready for the next launch
                        __threadfence();
#pragma unroll
                        for (int j = 0; j < BN; ++j) run[j] = 0.f;
                        for (int bb = b0; bb <= b1; ++bb) {
                            const float *pp = part + ((size_t)bb * maxseg + (size_t)(t - (U * bb / gridDim.x) / nkb)) *
                                                         (BM * BN) + 32 * wq + lane;
#pragma unroll
                            for (int j = 0; j < BN; ++j) run[j] += __ldcg(pp + j * BM);
                        }
                        write_c = true;
                    }
                }
                // Transposed output of a one-tile-per-CTA launch: the tile's MMAs are complete, so
                // the ring is idle; each warp stages its 32 rows x BN block there and writes every
                // output row (BN contiguous floats) with 16-byte stores across the warp, instead of
                // one 4-byte store per row per column.
                const bool staged = write_c && ctrans && part == nullptr && beta == 0.f && Clo == nullptr &&
                                    Cbf == nullptr && (ldc & 3) == 0 && ((uintptr_t)C & 15) == 0 &&
                                    (size_t)4 * 32 * (BN + 4) * 4 <= (size_t)CF::RING_BYTES;
                if (staged) {
                    float *stg = (float *)smem + wq * 32 * (BN + 4);  // [32 rows][BN + 4], 16-byte rows
#pragma unroll
                    for (int j = 0; j < BN; j += 4)
                        *(float4 *)(stg + lane * (BN + 4) + j) =
                            make_float4(alpha * run[j], alpha * run[j + 1], alpha * run[j + 2], alpha * run[j + 3]);
                    __syncwarp();
                    const int mrow0 = (t % mt) * BM + 32 * wq, n0 = (t / mt) * BN;
                    for (int rr = 0; rr < 32; ++rr) {
                        const int m = mrow0 + rr;
                        if (m >= M) break;
                        float *crow = C + (int64_t)m * ldc + n0;
#pragma unroll
                        for (int j0 = 0; j0 < BN; j0 += 128) {
                            const int j = j0 + 4 * lane;
                            if (j < BN) {
                                const float4 v = *(const float4 *)(stg + rr * (BN + 4) + j);
                                if (n0 + j + 3 < N) {
                                    *(float4 *)(crow + j) = v;
                                } else {
                                    if (n0 + j < N) crow[j] = v.x;
                                    if (n0 + j + 1 < N) crow[j + 1] = v.y;
                                    if (n0 + j + 2 < N) crow[j + 2] = v.z;
                                }
                            }
                        }
                    }
                    __syncwarp();
                    write_c = false;
                }
                if (write_c) {
                    const int m = (t % mt) * BM + 32 * wq + lane, n0 = (t / mt) * BN;
                    if (m < M) {
                        // element (m, n) at C[m + n ldc], or at C[n + m ldc] when ctrans
                        const int64_t sm = ctrans ? ldc : 1, sn = ctrans ? 1 : ldc;
                        const int64_t si = ctrans ? ldcin : 1, sj = ctrans ? 1 : ldcin;
                        float *cp = C + m * sm + (int64_t)n0 * sn;
                        const float *ci = Cin + m * si + (int64_t)n0 * sj;
                        // C's lo part (x - hi(x)) beside C when a later product takes C as its B
                        float *cl = Clo ? Clo + m * sm + (int64_t)n0 * sn : nullptr;
                        // and its BF16 parts (hi, then lo bfhalf elements later) for a later BF16-split product
                        __nv_bfloat16 *cb = Cbf ? Cbf + m + (int64_t)n0 * ldbf : nullptr;
#pragma unroll
                        for (int j = 0; j < BN; ++j) {
                            if (n0 + j < N) {
                                float o = alpha * run[j];
                                if (beta != 0.f) o = fmaf(beta, *ci, o);
                                *cp = o;
                                if (cl) cl[j * sn] = o - tf32_hi(o);
                                if (cb) {
                                    const __nv_bfloat16 hb = __float2bfloat16_rn(o);
                                    cb[j * ldbf] = hb;
                                    cb[bfhalf + j * ldbf] = __float2bfloat16_rn(o - __bfloat162float(hb));
                                }
                            }
                            cp += sn;
                            ci += sj;
                        }
                    }
                }
                if (kb == nkb) {
                    kb = 0;
                    ++t;
                }
            }
        }
        tc_fence_before();
    }
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"((uint32_t)CF::TMEM_COLS)
                     : "memory");
    }
}

// Split-K sum: C (M x N, M, N <= one tile) = alpha sum_b part[b] in CTA order b = 0, 1, ..,
// each piece a BM x BN tile (element (m, n) at m + n BM).
__global__ void k_splitk_sum(const float *part, int nparts, int tile, int M, int N, float alpha, float *C, int64_t ldc,
                             const int *status)
{
    if (status_bad(status)) return;
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= tile) return;
    const int m = e % BM, n = e / BM;
    if (m >= M || n >= N) return;
    float acc = 0.f;
    for (int b = 0; b < nparts; ++b) acc += __ldcg(part + (size_t)b * tile + e);
    C[m + (int64_t)n * ldc] = alpha * acc;
}

PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
std::once_flag g_encode_once;

bool get_encoder()
{
    std::call_once(g_encode_once, [] {
        cudaDriverEntryPointQueryResult q;
        void *fn = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            g_encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
    });
    return g_encode != nullptr;
}

// 2-D FP32 tensor map: inner extent `inner` (contiguous), outer extent
// `outer` with row pitch ld elements; box {32, box_rows}; 128-byte swizzle;
// out-of-range elements read as zero.
bool make_map(CUtensorMap *map, const float *ptr, int inner, int outer, int64_t ld, int box_rows)
{
    cuuint64_t dims[2] = {(cuuint64_t)inner, (cuuint64_t)outer};
    cuuint64_t strides[1] = {(cuuint64_t)ld * 4};
    cuuint32_t box[2] = {32, (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = g_encode(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, (void *)ptr, dims, strides, box, estr,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

int g_num_sms = 0;

}  // namespace

bool tc_make_map(CUtensorMap *map, const float *ptr, int inner, int outer, int64_t ld, int box_inner, int box_outer,
                 int swizzle128)
{
    if (!get_encoder()) return false;
    cuuint64_t dims[2] = {(cuuint64_t)inner, (cuuint64_t)outer};
    cuuint64_t strides[1] = {(cuuint64_t)ld * 4};
    cuuint32_t box[2] = {(cuuint32_t)box_inner, (cuuint32_t)box_outer};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = g_encode(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, (void *)ptr, dims, strides, box, estr,
                          CU_TENSOR_MAP_INTERLEAVE_NONE,
                          swizzle128 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_NONE,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

int tc_num_sms()
{
    if (!g_num_sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev);
        if (g_num_sms <= 0) g_num_sms = 148;
    }
    return g_num_sms;
}

struct tc_plan {
    int prec = 0;
    float *part = nullptr;
    size_t part_cap = 0;
    float *blo = nullptr;  // lo part of the B operand (3-term products)
    size_t blo_cap = 0;
    int *cnt = nullptr;  // stream-K arrival counts, 4 per tile, zero between launches
    size_t cnt_cap = 0;
    int *err = nullptr;
};

tc_plan *tc_plan_create(int n, int q, int prec)
{
    (void)n;
    (void)q;
    if (!get_encoder()) return nullptr;
    tc_plan *p = new tc_plan();
    p->prec = prec;
    if (cudaMalloc(&p->err, sizeof(int)) != cudaSuccess) {
        delete p;
        return nullptr;
    }
    cudaMemset(p->err, 0, sizeof(int));
    if (!g_num_sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev);
        if (g_num_sms <= 0) g_num_sms = 148;
    }
    return p;
}

void tc_plan_destroy(tc_plan *p)
{
    if (!p) return;
    if (p->part) cudaFree(p->part);
    if (p->blo) cudaFree(p->blo);
    if (p->cnt) cudaFree(p->cnt);
    if (p->err) cudaFree(p->err);
    delete p;
}

int tc_plan_error(tc_plan *p, cudaStream_t st)
{
    int e = 0;
    if (!p) return 0;
    cudaMemcpyAsync(&e, p->err, sizeof(int), cudaMemcpyDeviceToHost, st);
    cudaStreamSynchronize(st);
    return e;
}

template <int BN, int TERMS, int AMN, int BF = 0>
static int launch_bn(tc_plan *p, cudaStream_t st, const CUtensorMap &ma, const CUtensorMap &mb,
                     const CUtensorMap &mblo, int M, int N, int K,
                     float alpha, float beta, const float *Cin, int64_t ldcin, float *C, float *Clo, int64_t ldc,
                     const int *status, int *err, int reserve, int ctrans, void *Cbf = nullptr, int64_t ldbf = 0,
                     long long bfhalf = 0, int splitk = 0)
{
    using CF = Cfg<BN, TERMS, AMN, BF>;
    static bool attr = false;
    if (!attr) {
        if (cudaFuncSetAttribute(k_tc_gemm<BN, TERMS, AMN, BF>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 CF::SMEM) != cudaSuccess)
            return -1;
        // the register split raises warps 8-11 out of what the CTA holds: refuse a
        // build whose launch count leaves too few (setmaxnreg.inc would never return)
        cudaFuncAttributes fa;
        if (cudaFuncGetAttributes(&fa, k_tc_gemm<BN, TERMS, AMN, BF>) != cudaSuccess ||
            384 * fa.numRegs < 128 * (2 * GEMM_REG_LOW + GEMM_REG_DRAIN))
            return -1;
        attr = true;
    }
    const int mt = (M + BM - 1) / BM, nt = (N + BN - 1) / BN;
    const int nkb = (K + CF::BKE - 1) / CF::BKE;
    const int tiles = mt * nt;
    const long long U = (long long)tiles * nkb;
    // stream-K when the tiles alone leave SMs idle and each SM still gets a few
    // k-blocks; `reserve` SMs are left free for work on other streams
    const int sms = std::max(1, g_num_sms - std::max(0, reserve));
    // split-K (one output tile, splitk CTAs): every CTA writes its piece and k_splitk_sum adds them
    const bool streamk = splitk > 0 || (tiles < sms && U >= 4LL * sms && nkb >= 4 * CF::CHUNK);  // short K: one tile per CTA
    const int G = splitk > 0 ? (int)std::min<long long>(splitk, U) : streamk ? sms : tiles;
    int maxseg = 1;
    float *part = nullptr;
    if (streamk) {
        for (int b = 0; b < G; ++b) {
            const long long u0 = U * b / G, u1 = U * (b + 1) / G;
            if (u1 > u0) maxseg = std::max(maxseg, (int)((u1 - 1) / nkb - u0 / nkb + 1));
        }
        const size_t need = (size_t)G * maxseg * BM * BN;
        if (need > p->part_cap) {
            if (p->part) cudaFree(p->part);
            p->part = nullptr;
            p->part_cap = 0;
            if (cudaMalloc(&p->part, need * sizeof(float)) != cudaSuccess) return -2;
            p->part_cap = need;
        }
        part = p->part;
        if ((size_t)4 * tiles > p->cnt_cap) {
            if (p->cnt) cudaFree(p->cnt);
            p->cnt = nullptr;
            p->cnt_cap = 0;
            if (cudaMalloc(&p->cnt, sizeof(int) * 4 * tiles) != cudaSuccess) return -2;
            if (cudaMemsetAsync(p->cnt, 0, sizeof(int) * 4 * tiles, st) != cudaSuccess) return -2;
            p->cnt_cap = (size_t)4 * tiles;
        }
    }
    rb_count_launch();
    k_tc_gemm<BN, TERMS, AMN, BF><<<G, 384, CF::SMEM, st>>>(ma, mb, mblo, M, N, mt, nkb, U, maxseg, alpha, beta, Cin,
                                                        ldcin, C, Clo, ldc, ctrans, part, splitk > 0 ? nullptr : p->cnt,
                                                        status, err, (__nv_bfloat16 *)Cbf, ldbf, bfhalf);
    if (splitk > 0) {
        rb_count_launch();
        k_splitk_sum<<<(BM * BN + 255) / 256, 256, 0, st>>>(part, G, BM * BN, M, N, alpha, C, ldc, status);
    }
    return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

template <int TERMS>
static int launch_terms(tc_plan *p, cudaStream_t st, int a_layout, int M, int N, int K, float alpha, const float *A,
                        int64_t lda, const float *B, const float *Blo, int64_t ldb, float beta, const float *Cin,
                        int64_t ldcin, float *C, float *Clo, int64_t ldc, const int *status, int *err, int reserve,
                        int ctrans, int splitk = 0)
{
    const int a_mn = (a_layout == TC_A_MN);
    const int bn = N <= 32 ? 32 : N <= 64 ? 64 : 128;
    CUtensorMap ma, mb;
    bool ok = a_mn ? make_map(&ma, A, M, K, lda, 32) : make_map(&ma, A, K, M, lda, BM);
    ok = ok && make_map(&mb, B, K, N, ldb, bn);
    CUtensorMap mblo = mb;
    if (TERMS == 3 && Blo) {
        ok = ok && make_map(&mblo, Blo, K, N, ldb, bn);  // lo part of B supplied by the caller
    } else if (TERMS == 3) {
        // lo part of B, split once here rather than in every CTA (B is shared by all M tiles)
        const int ldlo = (K + 3) & ~3;  // 16-byte rows for TMA
        const size_t need = (size_t)ldlo * N;
        if (need > p->blo_cap) {
            if (p->blo) cudaFree(p->blo);
            p->blo = nullptr;
            p->blo_cap = 0;
            if (cudaMalloc(&p->blo, need * sizeof(float)) != cudaSuccess) return -2;
            p->blo_cap = need;
        }
        dim3 g((K + 255) / 256, N);
        rb_count_launch();
        k_split_lo<<<g, 256, 0, st>>>(K, N, B, ldb, p->blo, ldlo);
        ok = ok && make_map(&mblo, p->blo, K, N, ldlo, bn);
    }
    if (!ok) return -4;
#define RB_TC_CASE(BNV)                                                                                     \
    case BNV:                                                                                                  \
        return a_mn ? launch_bn<BNV, TERMS, 1>(p, st, ma, mb, mblo, M, N, K, alpha, beta, Cin, ldcin, C, Clo, ldc, \
                                               status, err, reserve, ctrans, nullptr, 0, 0, splitk)             \
                    : launch_bn<BNV, TERMS, 0>(p, st, ma, mb, mblo, M, N, K, alpha, beta, Cin, ldcin, C, Clo, ldc, \
                                               status, err, reserve, ctrans, nullptr, 0, 0, splitk);
    switch (bn) {
        RB_TC_CASE(32)
        RB_TC_CASE(64)
        RB_TC_CASE(128)
    default: return -5;
    }
#undef RB_TC_CASE
}

static bool tma_ok(const void *ptr, int64_t ld) { return ((uintptr_t)ptr % 16 == 0) && (ld % 4 == 0); }

// C's lo part after a CUDA-core product (the tensor-core epilogue writes it itself)
static void split_after_simt(cudaStream_t st, int M, int N, const float *C, float *Clo, int64_t ldc)
{
    if (!Clo) return;
    rb_count_launch();
    k_split_lo<<<dim3((M + 255) / 256, N), 256, 0, st>>>(M, N, C, ldc, Clo, ldc);
}

static int tc_run(tc_plan *p, cudaStream_t st, int terms, int a_layout, int M, int N, int K, float alpha,
                  const float *A, int64_t lda, const float *B, int64_t ldb, float beta, const float *Cin,
                  int64_t ldcin, float *C, int64_t ldc, const int *status, int reserve = 0, int ctrans = 0,
                  const float *Blo = nullptr, float *Clo = nullptr)
{
    if (M <= 0 || N <= 0) return 0;
    if (Clo && (ctrans || terms == 1)) return -7;  // C's lo part: plain output of a split product only
    const bool ok = p && K > 0 && tma_ok(A, lda) && tma_ok(B, ldb) && (!Blo || tma_ok(Blo, ldb));
    if (!ok && ctrans) return -6;  // the SIMT kernels have no transposed output
    if (!ok) {
        // SIMT fallback: alpha op(A) B + beta Cin (Cin copied to C first when distinct)
        if (beta != 0.f && Cin != C) launch_copy2d<float, float>(st, M, N, Cin, ldcin, C, ldc, 1.0);
        gemm_simt<float>(st, a_layout == TC_A_K, false, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, status);
        split_after_simt(st, M, N, C, Clo, ldc);
        return 1;
    }
    int *err = status ? const_cast<int *>(status) : p->err;
    const int rc =
        (terms == 3)   ? launch_terms<3>(p, st, a_layout, M, N, K, alpha, A, lda, B, Blo, ldb, beta, Cin, ldcin, C,
                                         Clo, ldc, status, err, reserve, ctrans)
        : (terms == 2) ? launch_terms<2>(p, st, a_layout, M, N, K, alpha, A, lda, B, nullptr, ldb, beta, Cin, ldcin,
                                         C, Clo, ldc, status, err, reserve, ctrans)
                       : launch_terms<1>(p, st, a_layout, M, N, K, alpha, A, lda, B, nullptr, ldb, beta, Cin, ldcin,
                                         C, nullptr, ldc, status, err, reserve, ctrans);
    if (rc == 0) return 0;
    if (ctrans) return rc;
    // the tensor-core launch could not be set up (tensor map or workspace): run the same product on CUDA cores
    if (beta != 0.f && Cin != C) launch_copy2d<float, float>(st, M, N, Cin, ldcin, C, ldc, 1.0);
    gemm_simt<float>(st, a_layout == TC_A_K, false, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, status);
    split_after_simt(st, M, N, C, Clo, ldc);
    return 1;
}

int tc_gemm_nk(tc_plan *p, cudaStream_t st, int terms, int a_layout, int M, int N, int K, const float *A, int64_t lda,
               const float *B, int64_t ldb, float *C, int64_t ldc, const int *status, int reserve_sms)
{
    return tc_run(p, st, terms, a_layout, M, N, K, 1.f, A, lda, B, ldb, 0.f, nullptr, 0, C, ldc, status, reserve_sms);
}

int tc_gemm_nk_t(tc_plan *p, cudaStream_t st, int terms, int a_layout, int M, int N, int K, const float *A,
                 int64_t lda, const float *B, int64_t ldb, float *C, int64_t ldc, const int *status, int reserve_sms,
                 const float *Blo)
{
    return tc_run(p, st, terms, a_layout, M, N, K, 1.f, A, lda, B, ldb, 0.f, nullptr, 0, C, ldc, status, reserve_sms,
                  1, Blo);
}

void tc_split_lo(cudaStream_t st, int rows, int cols, const float *X, int64_t ldx, float *Lo, int64_t ldl)
{
    if (rows <= 0 || cols <= 0) return;
    rb_count_launch();
    k_split_lo<<<dim3((rows + 255) / 256, cols), 256, 0, st>>>(rows, cols, X, ldx, Lo, ldl);
}

int tc_gemm_nk_axpby(tc_plan *p, cudaStream_t st, int terms, int a_layout, int M, int N, int K, float alpha,
                     const float *A, int64_t lda, const float *B, int64_t ldb, float beta, const float *Cin,
                     int64_t ldcin, float *C, int64_t ldc)
{
    return tc_run(p, st, terms, a_layout, M, N, K, alpha, A, lda, B, ldb, beta, Cin, ldcin, C, ldc, nullptr);
}

int tc_update(tc_plan *p, cudaStream_t st, int terms, int n, int q, const float *ShT, const float *V, float *L,
              int64_t ldl, const int *status)
{
    // L (n x n) += op(A) B with op(A)(i, c) = ShT[c + i q] (K-major, K = q), B(c, j) = V[c + j q]
    return tc_run(p, st, terms, TC_A_K, n, n, q, 1.f, ShT, q, V, q, 1.f, L, ldl, L, ldl, status);
}

int tc_gemm_nk_lo(tc_plan *p, cudaStream_t st, int terms, int a_layout, int M, int N, int K, const float *A,
                  int64_t lda, const float *B, const float *Blo, int64_t ldb, float *C, float *Clo, int64_t ldc,
                  const int *status, int reserve_sms)
{
    return tc_run(p, st, terms, a_layout, M, N, K, 1.f, A, lda, B, ldb, 0.f, nullptr, 0, C, ldc, status, reserve_sms,
                  0, Blo, Clo);
}

// ---------------------------------------------------------------------------
// BF16-split products (kind::f16).
// ---------------------------------------------------------------------------
namespace {

// hi = bf16(x), lo = bf16(x - hi) (round to nearest) of a column-major rows x cols panel
__global__ void k_split_bf16(int rows, int cols, const float *X, int64_t ldx, __nv_bfloat16 *H, __nv_bfloat16 *L,
                             int64_t ldo)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y;
    if (i < rows) {
        const float v = X[i + (int64_t)j * ldx];
        const __nv_bfloat16 h = __float2bfloat16_rn(v);
        H[i + (int64_t)j * ldo] = h;
        if (L) L[i + (int64_t)j * ldo] = __float2bfloat16_rn(v - __bfloat162float(h));
    }
}

// 2-D BF16 tensor map: inner extent `inner` (contiguous), row pitch ld elements;
// box {64, box_rows} (one 128-byte swizzle row); out-of-range elements read as zero.
bool make_map_bf16(CUtensorMap *map, const void *ptr, int inner, int outer, int64_t ld, int box_rows)
{
    cuuint64_t dims[2] = {(cuuint64_t)inner, (cuuint64_t)outer};
    cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
    cuuint32_t box[2] = {64, (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = g_encode(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(ptr), dims, strides, box, estr,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

}  // namespace

void tc_split_bf16(cudaStream_t st, int rows, int cols, const float *X, int64_t ldx, void *Xh, void *Xl, int64_t ldo)
{
    if (rows <= 0 || cols <= 0) return;
    rb_count_launch();
    k_split_bf16<<<dim3((rows + 255) / 256, cols), 256, 0, st>>>(rows, cols, X, ldx, (__nv_bfloat16 *)Xh,
                                                                   (__nv_bfloat16 *)Xl, ldo);
}

int tc_gemm_bf(tc_plan *p, cudaStream_t st, int terms, int M, int N, int K, const float *A, int64_t lda,
               const void *Bh, const void *Bl, int64_t ldb, float *C, float *Clo, int64_t ldc, const int *status,
               int reserve_sms, void *Cbf, int64_t ldcbf)
{
    if (M <= 0 || N <= 0) return 0;
    if (!p || K <= 0 || (terms != 1 && terms != 3) || (terms == 3 && !Bl)) return -1;
    if (!tma_ok(A, lda) || (uintptr_t)Bh % 16 || (Bl && (uintptr_t)Bl % 16) || ldb % 8) return -6;
    if (Clo && terms == 1) return -7;
    const int bn = N <= 32 ? 32 : N <= 64 ? 64 : 128;
    CUtensorMap ma, mb, mblo;
    bool ok = get_encoder() && make_map(&ma, A, K, M, lda, BM) && make_map_bf16(&mb, Bh, K, N, ldb, bn);
    mblo = mb;
    if (terms == 3) ok = ok && make_map_bf16(&mblo, Bl, K, N, ldb, bn);
    if (!ok) return -4;
    int *err = status ? const_cast<int *>(status) : p->err;
#define RB_BF_CASE(BNV)                                                                                          \
    case BNV:                                                                                                       \
        return terms == 3 ? launch_bn<BNV, 3, 0, 1>(p, st, ma, mb, mblo, M, N, K, 1.f, 0.f, nullptr, 0, C, Clo, ldc, \
                                                    status, err, reserve_sms, 0, Cbf, ldcbf,                       \
                                                    (long long)ldcbf * N)                                          \
                          : launch_bn<BNV, 1, 0, 1>(p, st, ma, mb, mblo, M, N, K, 1.f, 0.f, nullptr, 0, C, nullptr,  \
                                                    ldc, status, err, reserve_sms, 0, Cbf, ldcbf,                  \
                                                    (long long)ldcbf * N);
    switch (bn) {
        RB_BF_CASE(32)
        RB_BF_CASE(64)
        RB_BF_CASE(128)
    default: return -5;
    }
#undef RB_BF_CASE
}

int tc_gemm_splitk(tc_plan *p, cudaStream_t st, int terms, int a_layout, int M, int N, int K, const float *A,
                   int64_t lda, const float *B, const float *Blo, int64_t ldb, float *C, int64_t ldc, const int *status,
                   int nctas)
{
    if (M <= 0 || N <= 0) return 0;
    if (!p || K <= 0 || M > BM || N > 128 || nctas < 1 || !tma_ok(A, lda) || !tma_ok(B, ldb) ||
        (Blo && !tma_ok(Blo, ldb)) || (terms == 3 && !Blo))
        return -6;
    int *err = status ? const_cast<int *>(status) : p->err;
    CUtensorMap ma, mb, mblo;
    const int bn = N <= 32 ? 32 : N <= 64 ? 64 : 128;
    const int a_mn = (a_layout == TC_A_MN);
    bool ok = get_encoder() && (a_mn ? make_map(&ma, A, M, K, lda, 32) : make_map(&ma, A, K, M, lda, BM)) &&
              make_map(&mb, B, K, N, ldb, bn);
    mblo = mb;
    if (terms == 3) ok = ok && make_map(&mblo, Blo, K, N, ldb, bn);
    if (!ok) return -4;
#define RB_SK_CASE(BNV, TT)                                                                                          \
    if (bn == BNV && terms == TT)                                                                                       \
        return a_mn ? launch_bn<BNV, TT, 1>(p, st, ma, mb, mblo, M, N, K, 1.f, 0.f, nullptr, 0, C, nullptr, ldc, status, \
                                            err, 0, 0, nullptr, 0, 0, nctas)                                            \
                    : launch_bn<BNV, TT, 0>(p, st, ma, mb, mblo, M, N, K, 1.f, 0.f, nullptr, 0, C, nullptr, ldc, status, \
                                            err, 0, 0, nullptr, 0, 0, nctas);
    RB_SK_CASE(128, 1)
    RB_SK_CASE(128, 3)
    RB_SK_CASE(64, 1)
    RB_SK_CASE(64, 3)
    RB_SK_CASE(32, 1)
    RB_SK_CASE(32, 3)
#undef RB_SK_CASE
    return -5;
}
