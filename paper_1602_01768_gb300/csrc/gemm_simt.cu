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

template <typename T, bool TA, bool TB>
static void gemm_dispatch(cudaStream_t st, int M, int N, int K, T alpha, const T *A, int64_t lda, const T *B,
                          int64_t ldb, T beta, T *C, int64_t ldc, const int *status)
{
    if constexpr (sizeof(T) == 4) {
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
