// tc.cuh -- tensor-core (tcgen05 + TMA) GEMMs on FP32-stored operands.
//
//   C = alpha op(A) B + beta Cin        (column-major C, M x N)
//   op(A) M x K: TC_A_K  -> element (m, k) at A[k + m lda]  (K contiguous)
//                TC_A_MN -> element (m, k) at A[m + k lda]  (M contiguous)
//   B K x N:     element (k, n) at B[k + n ldb]             (K contiguous)
//
// terms = 1: single-pass TF32 products (FP32 accumulate).
// terms = 2: B already exact in TF32 (e.g. the TF32-rounded Gaussian sketch):
//            A = hi + lo, C accumulates hi*B + lo*B.
// terms = 3: each operand split x = hi + lo with hi = x truncated to the
//            11 leading significand bits (exact in TF32) and lo = x - hi;
//            C accumulates hi*hi + hi*lo + lo*hi, which carries ~22 bits.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

enum { TC_A_K = 0, TC_A_MN = 1 };

struct tc_plan;

tc_plan *tc_plan_create(int n, int q, int prec);
void tc_plan_destroy(tc_plan *p);

// Returns 0 when launched on the tensor cores, 1 when it fell back to the
// SIMT kernel (shape or alignment outside what TMA accepts), <0 on error.
// A stream-K launch (fewer output tiles than SMs) uses all SMs but
// reserve_sms, which stay free for kernels on other streams.
int tc_gemm_nk(tc_plan *p, cudaStream_t st, int terms, int a_layout, int M, int N, int K, const float *A,
               int64_t lda, const float *B, int64_t ldb, float *C, int64_t ldc, const int *status,
               int reserve_sms = 0);
// Same product with C written transposed: element (m, n) at C[n + m ldc]
// (C^T column-major).  Tensor cores only: returns <0 where that is not possible.
// Blo (may be null): B's lo part, as for tc_gemm_nk_lo.
int tc_gemm_nk_t(tc_plan *p, cudaStream_t st, int terms, int a_layout, int M, int N, int K, const float *A,
                 int64_t lda, const float *B, int64_t ldb, float *C, int64_t ldc, const int *status,
                 int reserve_sms = 0, const float *Blo = nullptr);
// Lo = X - hi(X) elementwise (hi = the top 11 significand bits that a TF32 MMA reads), rows x cols
// column-major panels; the Blo operand of a 3-term product.
void tc_split_lo(cudaStream_t st, int rows, int cols, const float *X, int64_t ldx, float *Lo, int64_t ldl);
// As tc_gemm_nk, with two hand-offs between products.  Blo (may be null): the
// lo part of B (element-wise x - hi(x), K x N, ld ldb, 16-byte aligned), already
// formed by the kernel that wrote B, so this call does not split B itself.  Clo
// (may be null; terms >= 2): C's lo part, written beside C (same layout and ld)
// for a later product that takes C as its B.
int tc_gemm_nk_lo(tc_plan *p, cudaStream_t st, int terms, int a_layout, int M, int N, int K, const float *A,
                  int64_t lda, const float *B, const float *Blo, int64_t ldb, float *C, float *Clo, int64_t ldc,
                  const int *status, int reserve_sms = 0);
int tc_gemm_nk_axpby(tc_plan *p, cudaStream_t st, int terms, int a_layout, int M, int N, int K, float alpha,
                     const float *A, int64_t lda, const float *B, int64_t ldb, float beta, const float *Cin,
                     int64_t ldcin, float *C, int64_t ldc);
// BF16-split products (kind::f16): C = op(A) B with op(A) K-contiguous FP32
// (element (m, k) at A[k + m lda]) and B given as its BF16 parts Bh (hi) and Bl
// (lo, needed for terms = 3), K x N, K contiguous, ld ldb (a multiple of 8),
// 16-byte aligned.  terms = 1: hi(A) hi(B); terms = 3: hi hi + hi lo + lo hi
// (~16 significant bits).  FP32 accumulation restarted every 1024 of K (64 MMA steps).  Clo
// (terms = 3, may be null): C's TF32 lo part beside C, as tc_gemm_nk_lo writes
// it.  Returns 0 when launched, < 0 when the shape or alignment is outside the
// kernel.  Cbf (may be null): C's own BF16 parts written beside C, hi at
// Cbf[m + n ldcbf] and lo ldcbf N elements later (ldcbf a multiple of 8), for a
// later BF16-split product that takes C as its B.
int tc_gemm_bf(tc_plan *p, cudaStream_t st, int terms, int M, int N, int K, const float *A, int64_t lda,
               const void *Bh, const void *Bl, int64_t ldb, float *C, float *Clo, int64_t ldc, const int *status,
               int reserve_sms = 0, void *Cbf = nullptr, int64_t ldcbf = 0);
// One-tile products (M <= 128, N <= 128) split over K on nctas CTAs: each CTA
// writes its partial tile and a second kernel adds them in CTA order (every SM
// takes part in the sum; no CTA waits for the others).  terms 1 or 3 (3 needs
// Blo, B's lo part).  Returns 0 when launched, < 0 when outside the kernel.
int tc_gemm_splitk(tc_plan *p, cudaStream_t st, int terms, int a_layout, int M, int N, int K, const float *A,
                   int64_t lda, const float *B, const float *Blo, int64_t ldb, float *C, int64_t ldc, const int *status,
                   int nctas);
// Xh = bf16(X), Xl = bf16(X - Xh) (Xl may be null), column-major rows x cols, ld ldo.
void tc_split_bf16(cudaStream_t st, int rows, int cols, const float *X, int64_t ldx, void *Xh, void *Xl, int64_t ldo);
// L += S^ V with S^ given row-major (element (i, c) at ShT[c + i q]) and V
// q x n column-major (ld q).
int tc_update(tc_plan *p, cudaStream_t st, int terms, int n, int q, const float *ShT, const float *V, float *L,
              int64_t ldl, const int *status);

// Device error word of the plan's kernels (bounded waits that gave up).
int tc_plan_error(tc_plan *p, cudaStream_t st);

// Host helpers shared by the tensor-core kernels.
struct CUtensorMap_st;
bool tc_make_map(CUtensorMap_st *map, const float *ptr, int inner, int outer, int64_t ld, int box_inner,
                 int box_outer, int swizzle128);
int tc_num_sms();

// Persistent rank-q update L += S^ V (see tc_update.cu); returns 0 when it
// ran on the tensor cores, 1 when the shape needs the generic kernel.
int tc_update_persistent(tc_plan *p, cudaStream_t st, int n, int q, const float *ShT, const float *V, float *L,
                         int64_t ldl, const int *status);

// Fused update and next sketch product (see tc_update_s.cu):
//   L += S^ V (when do_update), then S_out = L S~_next (n x q, ld n)
// with S~_next exact in TF32.  Spart is a workspace of at least
// tc_update_s_workspace(n, q) floats, zeroed once before its first use (its
// head holds arrival counts that every complete launch leaves at zero).  S_lo (may be null, 16-byte aligned):
// S_out's lo part x - hi(x), same layout, for the 3-term product that takes S
// as its B.  Returns 0 when it ran on the tensor cores, 1 when the shape is
// outside the kernel (q > 128, q or n not a multiple of 4, unaligned
// pointers), < 0 on error.
size_t tc_update_s_workspace(int n, int q);
// S_bf (may be null): S_out's BF16 parts, hi at S_bf[i + j ld_bf] and lo ld_bf q
// elements later, for the BF16-split product that takes S as its B.  reserve_sms
// (at most 8) SMs are left free for work on other streams.
int tc_update_next_s(cudaStream_t st, int n, int q, const float *ShT, const float *V, float *L, int64_t ldl,
                     const float *St_next, float *S_out, int do_update, float *Spart, size_t spart_elems,
                     const int *status, float *S_lo = nullptr, void *S_bf = nullptr, int64_t ld_bf = 0,
                     int reserve_sms = 0);
