// gemm_simt.cu -- SIMT (CUDA-core) GEMM, FP32 and FP64, column-major:
//   C = alpha op(A) op(B) + beta C,   op(A) M x K, op(B) K x N.
// The plain-precision path of every product of the method (FP64 parity mode
// and the plain FP32 form) and the fallback for shapes the tensor-core
// kernels do not take.  Each thread owns a TM x TN sub-tile with rows strided
// by BM/TM and columns strided by BN/TN, which keeps shared-memory reads
// conflict free; tiles of A and B are staged through shared memory with
// loads laid out along each operand's contiguous dimension.
#include "kernels.cuh"

template <typename T, int BM, int BN, int BK, int TM, int TN, bool TA, bool TB>
__global__ void __launch_bounds__((BM / TM) * (BN / TN))
k_gemm(int M, int N, int K, T alpha, const T *__restrict__ A, int64_t lda, const T *__restrict__ B, int64_t ldb,
       T beta, T *__restrict__ C, int64_t ldc, const int *status)
{
    constexpr int NT = (BM / TM) * (BN / TN);
    constexpr int RM = BM / TM;  // thread-grid rows
    constexpr int RN = BN / TN;
    __shared__ T As[BK][BM + 1];
    __shared__ T Bs[BK][BN + 1];
    if (status_bad(status)) return;

    const int tid = threadIdx.x;
    const int m0 = blockIdx.x * BM;
    const int n0 = blockIdx.y * BN;
    const int tm = tid % RM;
    const int tn = tid / RM;

    T acc[TM][TN];
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = T(0);

    for (int k0 = 0; k0 < K; k0 += BK) {
        // op(A)(m, k): A[m + k lda] (contiguous in m) or A[k + m lda] (contiguous in k)
#pragma unroll 4
        for (int e = tid; e < BM * BK; e += NT) {
            int mm, kk;
            if (!TA) {
                mm = e % BM;
                kk = e / BM;
            } else {
                kk = e % BK;
                mm = e / BK;
            }
            const int gm = m0 + mm, gk = k0 + kk;
            T v = T(0);
            if (gm < M && gk < K) v = TA ? A[gk + (int64_t)gm * lda] : A[gm + (int64_t)gk * lda];
            As[kk][mm] = v;
        }
        // op(B)(k, n): B[k + n ldb] (contiguous in k) or B[n + k ldb] (contiguous in n)
#pragma unroll 4
        for (int e = tid; e < BN * BK; e += NT) {
            int nn, kk;
            if (!TB) {
                kk = e % BK;
                nn = e / BK;
            } else {
                nn = e % BN;
                kk = e / BN;
            }
            const int gn = n0 + nn, gk = k0 + kk;
            T v = T(0);
            if (gn < N && gk < K) v = TB ? B[gn + (int64_t)gk * ldb] : B[gk + (int64_t)gn * ldb];
            Bs[kk][nn] = v;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            T a[TM], b[TN];
#pragma unroll
            for (int i = 0; i < TM; ++i) a[i] = As[kk][tm + i * RM];
#pragma unroll
            for (int j = 0; j < TN; ++j) b[j] = Bs[kk][tn + j * RN];
#pragma unroll
            for (int i = 0; i < TM; ++i)
#pragma unroll
                for (int j = 0; j < TN; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int j = 0; j < TN; ++j) {
        const int gn = n0 + tn + j * RN;
        if (gn >= N) continue;
#pragma unroll
        for (int i = 0; i < TM; ++i) {
            const int gm = m0 + tm + i * RM;
            if (gm >= M) continue;
            T *c = C + gm + (int64_t)gn * ldc;
            *c = (beta == T(0)) ? alpha * acc[i][j] : fma(alpha, acc[i][j], beta * *c);
        }
    }
}

// FP32 SGEMM for aligned operands (ld a multiple of 4, 16-byte aligned bases): 128 x 128
// tiles, 256 threads, 8 x 8 outputs per thread as 2 x 2 blocks of 4 x 4 (rows tm*4 and
// 64 + tm*4, columns tn*4 and 64 + tn*4, tm = thread % 16: 128-bit shared loads without bank
// conflicts, and consecutive threads own consecutive rows, so C moves as float4 columns),
// BK = 8, tiles double-buffered in shared memory with the next tile's global loads
// (float4 along each operand's contiguous dimension) issued before the current tile's
// FMAs.  Every output is summed over k in ascending order with one fma per term, as in
// k_gemm, so both kernels give the same bits.
constexpr int SG_BM = 128, SG_BN = 128, SG_BK = 8, SG_NT = 256;

template <bool TA, bool TB>
__global__ void __launch_bounds__(SG_NT, 2)
k_sgemm(int M, int N, int K, float alpha, const float *__restrict__ A, int64_t lda, const float *__restrict__ B,
        int64_t ldb, float beta, float *__restrict__ C, int64_t ldc, const int *status)
{
    __shared__ __align__(16) float As[2][SG_BK][SG_BM];
    __shared__ __align__(16) float Bs[2][SG_BK][SG_BN];
    if (status_bad(status)) return;
    const int tid = threadIdx.x, tm = tid % 16, tn = tid / 16;
    const int m0 = blockIdx.x * SG_BM, n0 = blockIdx.y * SG_BN;
    // one float4 of A and one of B per thread per tile (128 x 8 = 256 float4 each)
    // !TA: A(m, k) = A[m + k lda], a float4 along m: (m = 4 (tid % 32), k = tid / 32)
    //  TA: A(m, k) = A[k + m lda], a float4 along k: (m = tid / 2, k = 4 (tid % 2))
    const int am = TA ? tid / 2 : 4 * (tid % 32), ak = TA ? 4 * (tid % 2) : tid / 32;
    // !TB: B(k, n) = B[k + n ldb], a float4 along k: (n = tid / 2, k = 4 (tid % 2))
    //  TB: B(k, n) = B[n + k ldb], a float4 along n: (n = 4 (tid % 32), k = tid / 32)
    const int bn = TB ? 4 * (tid % 32) : tid / 2, bk = TB ? tid / 32 : 4 * (tid % 2);
    auto load_a = [&](int k0, float4 &v) {
        const int gm = m0 + am, gk = k0 + ak;
        float e[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int mm = TA ? gm : gm + u, kk = TA ? gk + u : gk;
            e[u] = (mm < M && kk < K) ? (TA ? A[kk + (int64_t)mm * lda] : A[mm + (int64_t)kk * lda]) : 0.f;
        }
        const bool full = TA ? (gm < M && gk + 3 < K) : (gm + 3 < M && gk < K);
        v = full ? (TA ? *(const float4 *)(A + gk + (int64_t)gm * lda) : *(const float4 *)(A + gm + (int64_t)gk * lda))
                 : make_float4(e[0], e[1], e[2], e[3]);
    };
    auto load_b = [&](int k0, float4 &v) {
        const int gn = n0 + bn, gk = k0 + bk;
        float e[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int nn = TB ? gn + u : gn, kk = TB ? gk : gk + u;
            e[u] = (nn < N && kk < K) ? (TB ? B[nn + (int64_t)kk * ldb] : B[kk + (int64_t)nn * ldb]) : 0.f;
        }
        const bool full = TB ? (gn + 3 < N && gk < K) : (gn < N && gk + 3 < K);
        v = full ? (TB ? *(const float4 *)(B + gn + (int64_t)gk * ldb) : *(const float4 *)(B + gk + (int64_t)gn * ldb))
                 : make_float4(e[0], e[1], e[2], e[3]);
    };
    auto store_a = [&](int buf, const float4 &v) {
        if (TA) {  // four k of one m
            As[buf][ak][am] = v.x;
            As[buf][ak + 1][am] = v.y;
            As[buf][ak + 2][am] = v.z;
            As[buf][ak + 3][am] = v.w;
        } else {
            *(float4 *)&As[buf][ak][am] = v;
        }
    };
    auto store_b = [&](int buf, const float4 &v) {
        if (TB) {
            *(float4 *)&Bs[buf][bk][bn] = v;
        } else {  // four k of one n
            Bs[buf][bk][bn] = v.x;
            Bs[buf][bk + 1][bn] = v.y;
            Bs[buf][bk + 2][bn] = v.z;
            Bs[buf][bk + 3][bn] = v.w;
        }
    };
    float acc[8][8];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;
    float4 ra, rb;
    load_a(0, ra);
    load_b(0, rb);
    store_a(0, ra);
    store_b(0, rb);
    __syncthreads();
    int buf = 0;
    for (int k0 = 0; k0 < K; k0 += SG_BK) {
        const bool more = k0 + SG_BK < K;
        if (more) {  // the next tile's global loads, in flight during this tile's FMAs
            load_a(k0 + SG_BK, ra);
            load_b(k0 + SG_BK, rb);
        }
#pragma unroll
        for (int kk = 0; kk < SG_BK; ++kk) {
            const float4 a0 = *(const float4 *)&As[buf][kk][tm * 4], a1 = *(const float4 *)&As[buf][kk][64 + tm * 4];
            const float4 b0 = *(const float4 *)&Bs[buf][kk][tn * 4], b1 = *(const float4 *)&Bs[buf][kk][64 + tn * 4];
            const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
            const float b[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
        }
        if (more) {
            store_a(buf ^ 1, ra);
            store_b(buf ^ 1, rb);
        }
        __syncthreads();
        buf ^= 1;
    }
    const bool cvec = ldc % 4 == 0 && (uintptr_t)C % 16 == 0;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const int gn = n0 + (j < 4 ? tn * 4 + j : 64 + tn * 4 + j - 4);
        if (gn >= N) continue;
#pragma unroll
        for (int h = 0; h < 2; ++h) {  // rows m0 + tm*4 .. + 3, then m0 + 64 + tm*4 .. + 3
            const int gm = m0 + 64 * h + tm * 4;
            float *c = C + gm + (int64_t)gn * ldc;
            if (cvec && gm + 3 < M) {
                float4 o = make_float4(alpha * acc[4 * h][j], alpha * acc[4 * h + 1][j], alpha * acc[4 * h + 2][j],
                                       alpha * acc[4 * h + 3][j]);
                if (beta != 0.f) {
                    const float4 ci = *(const float4 *)c;
                    o = make_float4(fmaf(alpha, acc[4 * h][j], beta * ci.x), fmaf(alpha, acc[4 * h + 1][j], beta * ci.y),
                                    fmaf(alpha, acc[4 * h + 2][j], beta * ci.z),
                                    fmaf(alpha, acc[4 * h + 3][j], beta * ci.w));
                }
                *(float4 *)c = o;
            } else {
#pragma unroll
                for (int i = 0; i < 4; ++i)
                    if (gm + i < M)
                        c[i] = (beta == 0.f) ? alpha * acc[4 * h + i][j] : fmaf(alpha, acc[4 * h + i][j], beta * c[i]);
            }
        }
    }
}

template <typename T, bool TA, bool TB>
static void gemm_dispatch(cudaStream_t st, int M, int N, int K, T alpha, const T *A, int64_t lda, const T *B,
                          int64_t ldb, T beta, T *C, int64_t ldc, const int *status)
{
    if constexpr (sizeof(T) == 4) {
        const bool aligned = lda % 4 == 0 && ldb % 4 == 0 && (uintptr_t)A % 16 == 0 && (uintptr_t)B % 16 == 0;
        // the register-blocked kernel where a 128 x 128 tile is filled enough to pay
        if (aligned && (int64_t)M * N >= (int64_t)64 * SG_BM * SG_BN && M >= 64 && N >= 64) {
            dim3 grid(ceil_div(M, SG_BM), ceil_div(N, SG_BN));
            rb_count_launch();
            k_sgemm<TA, TB><<<grid, SG_NT, 0, st>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, status);
            return;
        }
        if (N <= 32) {
            constexpr int BM = 128, BN = 32, BK = 16, TM = 8, TN = 2;
            dim3 grid(ceil_div(M, BM), ceil_div(N, BN));
            rb_count_launch();
            k_gemm<T, BM, BN, BK, TM, TN, TA, TB>
                <<<grid, (BM / TM) * (BN / TN), 0, st>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, status);
        } else {
            constexpr int BM = 128, BN = 64, BK = 16, TM = 8, TN = 4;
            dim3 grid(ceil_div(M, BM), ceil_div(N, BN));
            rb_count_launch();
            k_gemm<T, BM, BN, BK, TM, TN, TA, TB>
                <<<grid, (BM / TM) * (BN / TN), 0, st>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, status);
        }
    } else {
        if (N <= 16) {
            constexpr int BM = 64, BN = 16, BK = 16, TM = 4, TN = 1;
            dim3 grid(ceil_div(M, BM), ceil_div(N, BN));
            rb_count_launch();
            k_gemm<T, BM, BN, BK, TM, TN, TA, TB>
                <<<grid, (BM / TM) * (BN / TN), 0, st>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, status);
        } else {
            constexpr int BM = 64, BN = 64, BK = 16, TM = 4, TN = 4;
            dim3 grid(ceil_div(M, BM), ceil_div(N, BN));
            rb_count_launch();
            k_gemm<T, BM, BN, BK, TM, TN, TA, TB>
                <<<grid, (BM / TM) * (BN / TN), 0, st>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, status);
        }
    }
}

template <typename T>
void gemm_simt(cudaStream_t st, bool ta, bool tb, int M, int N, int K, T alpha, const T *A, int64_t lda,
               const T *B, int64_t ldb, T beta, T *C, int64_t ldc, const int *status)
{
    if (M <= 0 || N <= 0) return;
    if (!ta && !tb) gemm_dispatch<T, false, false>(st, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, status);
    if (!ta && tb) gemm_dispatch<T, false, true>(st, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, status);
    if (ta && !tb) gemm_dispatch<T, true, false>(st, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, status);
    if (ta && tb) gemm_dispatch<T, true, true>(st, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, status);
}

template void gemm_simt<float>(cudaStream_t, bool, bool, int, int, int, float, const float *, int64_t,
                               const float *, int64_t, float, float *, int64_t, const int *);
template void gemm_simt<double>(cudaStream_t, bool, bool, int, int, int, double, const double *, int64_t,
                                const double *, int64_t, double, double *, int64_t, const int *);
