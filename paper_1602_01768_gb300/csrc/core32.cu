// core32.cu -- blocked FP32 q x q core of AdaRBFGS for the FP32-storage
// modes: lower Cholesky C C^T = S^T A S (and D D^T = S~^T S~) and the
// inverse of each factor, one CTA per matrix, everything in shared memory.
//
// Cholesky: 32-column panels; the 32 x 32 diagonal block is factored by one
// warp (row per lane, warp-synchronous), the rows below it are solved in
// parallel (row per thread), then the trailing lower triangle is updated in
// parallel.  Inverse: the 32 x 32 diagonal blocks are inverted by one warp
// each (column per lane); pairs of inverted blocks are then merged,
// [[A, 0], [B, C]]^-1 = [[A^-1, 0], [-C^-1 B A^-1, C^-1]], doubling the block
// size until it covers q.  A pivot that is not positive and finite records
// ST_NOTSPD and leaves the outputs untouched.
#include "kernels.cuh"

namespace {

constexpr int CT = 256;  // threads (register arrays of 32 need the 255-register budget)

__device__ void chol_blocked(float *a, int QP, int *fail)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int c0 = 0; c0 < QP; c0 += 32) {
        if (warp == 0) {
            // diagonal block: lane i holds row i in registers, columns via shuffles
            float r[32];
#pragma unroll
            for (int c = 0; c < 32; ++c) r[c] = a[(c0 + lane) + (c0 + c) * QP];
            bool bad = false;
#pragma unroll
            for (int j = 0; j < 32; ++j) {
                const float d = __shfl_sync(0xffffffffu, r[j], j);
                if (!(d > 0.f) || !isfinite(d)) {
                    bad = true;
                    break;
                }
                const float sd = sqrtf(d);
                if (lane == j)
                    r[j] = sd;
                else if (lane > j)
                    r[j] = r[j] / sd;
#pragma unroll
                for (int c = j + 1; c < 32; ++c) {
                    const float lcj = __shfl_sync(0xffffffffu, r[j], c);
                    if (lane >= c) r[c] -= r[j] * lcj;
                }
            }
            if (bad) {
                if (lane == 0) *fail = 1;
            } else {
#pragma unroll
                for (int c = 0; c < 32; ++c)
                    if (c <= lane) a[(c0 + lane) + (c0 + c) * QP] = r[c];
            }
        }
        __syncthreads();
        if (*fail) return;
        // rows below the diagonal block: x D^T = a[r, c0:c0+32], row in registers
        for (int row = c0 + 32 + threadIdx.x; row < QP; row += CT) {
            float x[32];
#pragma unroll
            for (int j = 0; j < 32; ++j) x[j] = a[row + (c0 + j) * QP];
#pragma unroll
            for (int j = 0; j < 32; ++j) {
                float s = x[j];
#pragma unroll
                for (int k = 0; k < j; ++k) s -= x[k] * a[(c0 + j) + (c0 + k) * QP];
                x[j] = s / a[(c0 + j) + (c0 + j) * QP];
            }
#pragma unroll
            for (int j = 0; j < 32; ++j) a[row + (c0 + j) * QP] = x[j];
        }
        __syncthreads();
        // trailing lower triangle
        const int m = QP - c0 - 32;
        for (int e = threadIdx.x; e < m * m; e += CT) {
            const int rr = e % m, cc = e / m;
            if (rr < cc) continue;
            const int r = c0 + 32 + rr, c = c0 + 32 + cc;
            float s = 0.f;
#pragma unroll 8
            for (int k = 0; k < 32; ++k) s += a[r + (c0 + k) * QP] * a[c + (c0 + k) * QP];
            a[r + c * QP] -= s;
        }
        __syncthreads();
    }
}

// x = inverse of the lower-triangular a (both QP x QP, column-major); t is
// scratch of QP * QP / 4 floats.
__device__ void tri_inverse_blocked(const float *a, float *x, float *t, int QP)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int e = threadIdx.x; e < QP * QP; e += CT) x[e] = 0.f;
    __syncthreads();
    const int NB = QP / 32;
    if (warp < NB) {  // diagonal blocks, column per lane, column kept in registers
        const int o = 32 * warp, c = lane;
        float xc[32];
#pragma unroll
        for (int i = 0; i < 32; ++i) {
            float s = 0.f;
#pragma unroll
            for (int k = 0; k < i; ++k) s += a[(o + i) + (o + k) * QP] * xc[k];  // xc[k] = 0 for k < c
            const float inv = 1.f / a[(o + i) + (o + i) * QP];
            xc[i] = (i == c) ? inv : ((i > c) ? -s * inv : 0.f);
        }
#pragma unroll
        for (int i = 0; i < 32; ++i) x[(o + i) + (o + c) * QP] = xc[i];
    }
    __syncthreads();
    for (int b = 32; b < QP; b *= 2) {
        const int pairs = QP / (2 * b);
        // T_g = B_g X11_g  (B = a[o+b : o+2b, o : o+b], X11 lower)
        for (int e = threadIdx.x; e < pairs * b * b; e += CT) {
            const int g = e / (b * b), ij = e % (b * b), i = ij % b, j = ij / b, o = 2 * b * g;
            float s = 0.f;
            for (int k = j; k < b; ++k) s += a[(o + b + i) + (o + k) * QP] * x[(o + k) + (o + j) * QP];
            t[e] = s;
        }
        __syncthreads();
        // X21_g = -X22_g T_g  (X22 lower)
        for (int e = threadIdx.x; e < pairs * b * b; e += CT) {
            const int g = e / (b * b), ij = e % (b * b), i = ij % b, j = ij / b, o = 2 * b * g;
            float s = 0.f;
            for (int k = 0; k <= i; ++k) s += x[(o + b + i) + (o + b + k) * QP] * t[g * b * b + k + j * b];
            x[(o + b + i) + (o + j) * QP] = -s;
        }
        __syncthreads();
    }
}

__global__ void __launch_bounds__(CT, 1) k_core32(int q, const double *M, const double *N, float *Cinv, float *Dinv,
                                                  int *status)
{
    // blockIdx.x = 0 handles M -> Cinv, 1 handles N -> Dinv; a launch of one
    // block with M == N handles a single matrix.
    extern __shared__ float sm32[];
    __shared__ int fail;
    if (status_bad(status)) return;
    const int QP = ((q + 31) / 32) * 32;
    float *a = sm32, *x = sm32 + QP * QP, *t = sm32 + 2 * QP * QP;
    const double *src = blockIdx.x == 0 ? M : N;
    float *dst = blockIdx.x == 0 ? Cinv : Dinv;
    if (threadIdx.x == 0) fail = 0;
    for (int e = threadIdx.x; e < QP * QP; e += CT) {
        const int i = e % QP, j = e / QP;
        float v;
        if (i < q && j < q)
            v = (float)(0.5 * (src[i + j * q] + src[j + i * q]));
        else
            v = (i == j) ? 1.f : 0.f;  // pad with the identity: its factor is the identity
        a[e] = v;
    }
    __syncthreads();
    chol_blocked(a, QP, &fail);
    if (fail) {
        if (threadIdx.x == 0) atomicOr(status, ST_NOTSPD);
        return;
    }
    tri_inverse_blocked(a, x, t, QP);
    for (int e = threadIdx.x; e < q * q; e += CT) {
        const int i = e % q, j = e / q;
        const float v = (i >= j) ? x[i + j * QP] : 0.f;
        if (!isfinite(v)) atomicOr(status, ST_NONFINITE);
        dst[e] = v;
    }
}

}  // namespace

void launch_core_ada32(cudaStream_t st, int q, const double *M, const double *N, float *Cinv, float *Dinv,
                       int *status)
{
    const int QP = ((q + 31) / 32) * 32;
    const size_t smem = sizeof(float) * (2 * QP * QP + QP * QP / 4 + 32);
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(k_core32, cudaFuncAttributeMaxDynamicSharedMemorySize, 160 * 1024);
        attr = true;
    }
    rb_count_launch();
    k_core32<<<(N && Dinv) ? 2 : 1, CT, smem, st>>>(q, M, N, Cinv, Dinv, status);
}
