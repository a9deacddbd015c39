// core64.cu -- FP64 q x q core of AdaRBFGS for the FP32-storage tensor-core
// forms: the lower Cholesky factor of one symmetric q x q matrix
// (C C^T = S^T A S or D D^T = S~^T S~, Algorithm 4) and the inverse of that
// factor, factored and inverted in FP64 in one CTA, written out in FP32 the
// way the tensor-core GEMMs read it (scaled transposes into their B operands).
//
// The algorithm is the blocked right-looking one of k_core_blk in core32.cu
// (32 x 32 blocks, q padded to 32 nb with the identity): per block column p,
// warp 0 factors and inverts the diagonal block, all threads form the panel
// L_ip = A_ip X_pp^T and the trailing update A_ij -= L_ip L_jp^T; then the
// off-diagonal blocks of X = L^-1 follow by block diagonals d,
// T = sum_{k=j}^{i-1} L_ik X_kj, X_ij = -X_ii T (i = j + d).
// In FP64 the unpacked 128 x 129 layout of two matrices would not fit in
// shared memory, so both A (overwritten by L) and X keep only their lower
// block triangle, each block 32 x 33 (padded rows), and T has a scratch of
// its own.  A pivot that is not positive and finite records ST_NOTSPD and
// writes nothing.
#include "kernels.cuh"

namespace {

constexpr int KT64 = 512;  // threads
constexpr int NBMAX = 4;   // q <= 128
constexpr int BLD = 33;    // padded leading dimension of a 32 x 32 block
constexpr int BLK = 32 * BLD;
constexpr int NPACK = NBMAX * (NBMAX + 1) / 2;  // blocks of the lower block triangle

// Element (i, j) of a block-lower-packed matrix (block row of i >= block column of j):
// blocks packed column after column, block column c holding blocks c .. nb - 1.
__device__ __forceinline__ double &pk(double *m, int nb, int i, int j)
{
    const int bi = i >> 5, bj = j >> 5;
    const int b = bj * nb - (bj * (bj - 1)) / 2 + (bi - bj);
    return m[b * BLK + (i & 31) + (j & 31) * BLD];
}

struct Core64Out {
    const float *src;  // symmetric q x q input (ld q); its symmetric part is factored
    float *xt1;        // s1 X^T (ld1), or null
    int ld1;
    float s1;
    float *xt2;        // s2 X^T (ld2), or null
    int ld2;
    float s2;
};

__global__ void __launch_bounds__(KT64, 1) k_core_blk64(int q, Core64Out out, int *status)
{
    extern __shared__ double smd[];
    const int nb = (q + 31) / 32, QP = 32 * nb;
    double *a = smd;                 // A, overwritten by L
    double *x = smd + NPACK * BLK;   // X = L^-1
    double *t = smd + 2 * NPACK * BLK;  // T blocks of the current block diagonal
    __shared__ int fail;
    if (status_bad(status)) return;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (tid == 0) fail = 0;
    // symmetric part of the padded matrix, lower block triangle only (identity padding)
    for (int e = tid; e < QP * QP; e += KT64) {
        const int i = e % QP, j = e / QP;
        if ((i >> 5) < (j >> 5)) continue;
        double v;
        if (i < q && j < q)
            v = 0.5 * ((double)out.src[i + (size_t)j * q] + (double)out.src[j + (size_t)i * q]);
        else
            v = (i == j) ? 1.0 : 0.0;
        pk(a, nb, i, j) = v;
    }
    __syncthreads();
    for (int p = 0; p < nb; ++p) {
        const int o = 32 * p;
        if (warp == 0) {
            // diagonal block: L_pp in place (lane = row)
            bool bad = false;
            for (int j = 0; j < 32; ++j) {
                const double d = pk(a, nb, o + j, o + j);
                bad = bad || !(d > 0.0) || !isfinite(d);
                const double sd = sqrt(d), inv = 1.0 / sd;
                double lij = 0.0;
                if (lane > j) {
                    lij = pk(a, nb, o + lane, o + j) * inv;
                    pk(a, nb, o + lane, o + j) = lij;
                } else if (lane == j) {
                    pk(a, nb, o + j, o + j) = sd;
                }
                __syncwarp();
                for (int c = j + 1; c <= lane; ++c) pk(a, nb, o + lane, o + c) -= lij * pk(a, nb, o + c, o + j);
                __syncwarp();
            }
            if (bad) {
                if (lane == 0) fail = 1;
            } else {
                // X_pp = L_pp^-1 (lane = column), zeros above the diagonal of the block
                for (int i = 0; i < 32; ++i) {
                    double s = (i == lane) ? 1.0 : 0.0;
                    for (int k = lane; k < i; ++k) s -= pk(a, nb, o + i, o + k) * pk(x, nb, o + k, o + lane);
                    pk(x, nb, o + i, o + lane) = (i >= lane) ? s / pk(a, nb, o + i, o + i) : 0.0;
                }
            }
        }
        __syncthreads();
        if (fail) {
            if (tid == 0) atomicOr(status, ST_NOTSPD);
            return;
        }
        // panel: L_ip = A_ip X_pp^T, i > p (all values computed before any is stored)
        const int npanel = (nb - 1 - p) * 1024;
        double pv[6];
#pragma unroll
        for (int u = 0; u < 6; ++u) {
            const int e = tid + u * KT64;
            pv[u] = 0.0;
            if (e < npanel) {
                const int blk = e >> 10, w = e & 1023, r = w & 31, c = w >> 5;
                const int i = o + 32 * (blk + 1) + r;
                double s = 0.0;
                for (int k = 0; k <= c; ++k) s += pk(a, nb, i, o + k) * pk(x, nb, o + c, o + k);
                pv[u] = s;
            }
        }
        __syncthreads();
#pragma unroll
        for (int u = 0; u < 6; ++u) {
            const int e = tid + u * KT64;
            if (e < npanel) {
                const int blk = e >> 10, w = e & 1023, r = w & 31, c = w >> 5;
                pk(a, nb, o + 32 * (blk + 1) + r, o + c) = pv[u];
            }
        }
        __syncthreads();
        // trailing update: A_ij -= L_ip L_jp^T over the lower block triangle p < bj <= bi
        const int m = nb - 1 - p;
        const int ntr = m * (m + 1) / 2 * 1024;
        for (int e = tid; e < ntr; e += KT64) {
            int blk = e >> 10, bj = 0;
            while (blk >= m - bj) {
                blk -= m - bj;
                ++bj;
            }
            const int bi = bj + blk, w = e & 1023, r = w & 31, c = w >> 5;
            const int i = o + 32 * (bi + 1) + r, j = o + 32 * (bj + 1) + c;
            double s = 0.0;
            for (int k = 0; k < 32; ++k) s += pk(a, nb, i, o + k) * pk(a, nb, j, o + k);
            pk(a, nb, i, j) -= s;
        }
        __syncthreads();
    }
    // off-diagonal blocks of X by block diagonals
    for (int d = 1; d < nb; ++d) {
        const int nt = (nb - d) * 1024;
        for (int e = tid; e < nt; e += KT64) {  // T_j = sum_{k=j}^{j+d-1} L_(j+d, k) X_(k, j)
            const int bj = e >> 10, w = e & 1023, r = w & 31, c = w >> 5, bi = bj + d;
            double s = 0.0;
            for (int bk = bj; bk < bi; ++bk)
                for (int k = 0; k < 32; ++k) s += pk(a, nb, 32 * bi + r, 32 * bk + k) * pk(x, nb, 32 * bk + k, 32 * bj + c);
            t[bj * BLK + r + c * BLD] = s;
        }
        __syncthreads();
        for (int e = tid; e < nt; e += KT64) {  // X_(j+d, j) = -X_(j+d, j+d) T_j
            const int bj = e >> 10, w = e & 1023, r = w & 31, c = w >> 5, bi = bj + d;
            double s = 0.0;
            for (int k = 0; k <= r; ++k) s += pk(x, nb, 32 * bi + r, 32 * bi + k) * t[bj * BLK + k + c * BLD];
            pk(x, nb, 32 * bi + r, 32 * bj + c) = -s;
        }
        __syncthreads();
    }
    // scaled transposes s X^T (entry (r, c) of X^T is X(c, r), zero above X's diagonal)
    for (int e = tid; e < q * q; e += KT64) {
        const int r = e % q, c = e / q;
        const double w = (c >= r) ? pk(x, nb, c, r) : 0.0;
        if (!isfinite(w)) atomicOr(status, ST_NONFINITE);
        if (out.xt1) out.xt1[r + (size_t)c * out.ld1] = (float)(out.s1 * w);
        if (out.xt2) out.xt2[r + (size_t)c * out.ld2] = (float)(out.s2 * w);
    }
}

}  // namespace

bool launch_core_tr64(cudaStream_t st, int q, const float *M, float *xt1, int ld1, float s1, float *xt2, int ld2,
                      float s2, int *status)
{
    if (q > 32 * NBMAX) return false;
    static bool attr = false;
    const size_t smem = sizeof(double) * (2 * NPACK + (NBMAX - 1)) * BLK;
    if (!attr) {
        if (cudaFuncSetAttribute(k_core_blk64, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
            return false;
        attr = true;
    }
    rb_count_launch();
    k_core_blk64<<<1, KT64, smem, st>>>(q, Core64Out{M, xt1, ld1, s1, xt2, ld2, s2}, status);
    return true;
}
