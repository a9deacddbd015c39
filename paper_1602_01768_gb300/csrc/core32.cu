// core32.cu -- FP32 q x q core of AdaRBFGS for the FP32-storage modes:
// lower Cholesky C C^T = S^T A S (and D D^T = S~^T S~) and the inverse of
// each factor, one CTA per matrix.  q <= 128 takes k_core_blk (32 x 32 blocks,
// block GEMMs between a few barriers); larger q the older blocked kernel:
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

// q <= 128: blocked right-looking factorisation on 32 x 32 blocks (q padded
// to 32 nb with the identity, whose factor and inverse are the identity).
// Per block column p:
//   warp 0       factors the diagonal block (row per lane, shuffles) and
//                inverts it (column per lane, forward substitution);
//   all threads  panel L_ip = A_ip X_pp^T, then the trailing update
//                A_ij -= L_ip L_jp^T of the lower block triangle;
// then the off-diagonal blocks of X = L^-1 by block diagonals d = 1, 2, ..:
//   T = sum_{k=j}^{i-1} L_ik X_kj,  X_ij = -X_ii T   (i = j + d).
// Every phase but the diagonal block is a set of small GEMMs, so the kernel
// needs a handful of barriers instead of one per column.
// One matrix of a core launch: the Gram matrix it factors (FP64, q x q) and
// where X = L^-1 goes: plainly (dst, lower, ld q) and as up to two scaled
// transposes s X^T (xt1 / xt2 with their leading dimensions); null skips.
struct CoreOut {
    const double *src;
    const float *srcf;  // FP32 Gram matrix instead of src when not null
    float *dst;
    float *xt1;
    int ld1;
    float s1;
    float *xt2;
    int ld2;
    float s2;
};

constexpr int KT = 512;   // threads
constexpr int LDK = 129;  // padded leading dimension: row and column walks are conflict-free

__device__ __forceinline__ float &ak(float *m, int i, int j) { return m[i + j * LDK]; }

__global__ void __launch_bounds__(KT, 1) k_core_blk(int q, CoreOut o0, CoreOut o1, int *status)
{
    extern __shared__ float smk[];
    float *a = smk;               // A, overwritten by L (lower blocks)
    float *x = smk + 128 * LDK;   // X = L^-1 (lower blocks); upper blocks hold T
    __shared__ int fail;
    if (status_bad(status)) return;
    const CoreOut &out = blockIdx.x == 0 ? o0 : o1;
    const double *src = out.src;
    const int nb = (q + 31) / 32, QP = 32 * nb;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (tid == 0) fail = 0;
    // coalesced load of the padded matrix (thread: one row, every fourth column) ...
    {
        const int i = tid & 127, j0 = tid >> 7;
        float v[32];
#pragma unroll
        for (int u = 0; u < 32; ++u) {
            const int j = j0 + 4 * u;
            v[u] = (i < q && j < q) ? (out.srcf ? out.srcf[i + (size_t)j * q] : (float)src[i + (size_t)j * q])
                                    : (i == j ? 1.f : 0.f);
        }
#pragma unroll
        for (int u = 0; u < 32; ++u) ak(a, i, j0 + 4 * u) = v[u];
    }
    __syncthreads();
    // ... then the lower triangle takes the symmetric part 0.5 (a_ij + a_ji) (upper left as it is)
    {
        const int i = tid & 127;
        if (i < QP)
            for (int j = tid >> 7; j < i; j += 4) ak(a, i, j) = 0.5f * (ak(a, i, j) + ak(a, j, i));
    }
    __syncthreads();
    for (int p = 0; p < nb; ++p) {
        const int o = 32 * p;
        if (warp == 0) {
            // ---- diagonal block: L_pp in place (lane = row); compact loops keep the
            // code small (this runs once per block column, mostly alone on the SM) ----
            // column j of L travels by warp shuffle (l_cj is lane c's lij), so the row
            // updates below read nothing another lane writes and go 8 at a time
            bool bad = false;
            for (int j = 0; j < 32; ++j) {
                const float d = ak(a, o + j, o + j);
                bad = bad || !(d > 0.f) || !isfinite(d);
                const float sd = sqrtf(d), inv = 1.f / sd;
                float lij = 0.f;
                if (lane > j) {
                    lij = ak(a, o + lane, o + j) * inv;
                    ak(a, o + lane, o + j) = lij;
                } else if (lane == j) {
                    ak(a, o + j, o + j) = sd;
                }
                for (int c = j + 1; c < 32; c += 8) {  // the same trip count on every lane
                    float lc[8];
#pragma unroll
                    for (int u = 0; u < 8; ++u) lc[u] = __shfl_sync(0xffffffffu, lij, (c + u) & 31);
#pragma unroll
                    for (int u = 0; u < 8; ++u)
                        if (c + u <= lane) ak(a, o + lane, o + c + u) -= lij * lc[u];
                }
                __syncwarp();
            }
            if (bad) {
                if (lane == 0) fail = 1;
            } else {
                // ---- X_pp = L_pp^-1 (lane = column, kept in its column of x) ----
                // rows i in order; x above the diagonal is written as zero first, so every
                // lane sums k from 0 with four independent partial sums
                for (int i = 0; i < 32; ++i) {
                    float s0 = (i == lane) ? 1.f : 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
                    int k = 0;
                    for (; k + 3 < i; k += 4) {
                        s0 -= ak(a, o + i, o + k) * ak(x, o + k, o + lane);
                        s1 -= ak(a, o + i, o + k + 1) * ak(x, o + k + 1, o + lane);
                        s2 -= ak(a, o + i, o + k + 2) * ak(x, o + k + 2, o + lane);
                        s3 -= ak(a, o + i, o + k + 3) * ak(x, o + k + 3, o + lane);
                    }
                    for (; k < i; ++k) s0 -= ak(a, o + i, o + k) * ak(x, o + k, o + lane);
                    ak(x, o + i, o + lane) = (i >= lane) ? ((s0 + s1) + (s2 + s3)) / ak(a, o + i, o + i) : 0.f;
                }
            }
        }
        __syncthreads();
        if (fail) {
            if (tid == 0) atomicOr(status, ST_NOTSPD);
            return;
        }
        // ---- panel: L_ip = A_ip X_pp^T, i > p (into registers, then stored) ----
        const int npanel = (nb - 1 - p) * 1024;
        float pv[6];
#pragma unroll
        for (int u = 0; u < 6; ++u) {
            const int e = tid + u * KT;
            pv[u] = 0.f;
            if (e < npanel) {
                const int blk = e >> 10, w = e & 1023, r = w & 31, c = w >> 5;  // row r, column c of block
                const int i = o + 32 * (blk + 1) + r;
                float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
                int k = 0;
                for (; k + 3 <= c; k += 4) {  // X_pp lower: k <= c
                    s0 += ak(a, i, o + k) * ak(x, o + c, o + k);
                    s1 += ak(a, i, o + k + 1) * ak(x, o + c, o + k + 1);
                    s2 += ak(a, i, o + k + 2) * ak(x, o + c, o + k + 2);
                    s3 += ak(a, i, o + k + 3) * ak(x, o + c, o + k + 3);
                }
                for (; k <= c; ++k) s0 += ak(a, i, o + k) * ak(x, o + c, o + k);
                pv[u] = (s0 + s1) + (s2 + s3);
            }
        }
        __syncthreads();
#pragma unroll
        for (int u = 0; u < 6; ++u) {
            const int e = tid + u * KT;
            if (e < npanel) {
                const int blk = e >> 10, w = e & 1023, r = w & 31, c = w >> 5;
                ak(a, o + 32 * (blk + 1) + r, o + c) = pv[u];
            }
        }
        __syncthreads();
        // ---- trailing update: A_ij -= L_ip L_jp^T, p < j <= i ----
        const int m = nb - 1 - p;            // trailing blocks per side
        const int ntr = m * (m + 1) / 2 * 1024;  // lower block triangle incl. diagonal blocks
        for (int e = tid; e < ntr; e += KT) {
            int blk = e >> 10, bj = 0;
            while (blk >= m - bj) {  // column-major packing of the lower block triangle
                blk -= m - bj;
                ++bj;
            }
            const int bi = bj + blk, w = e & 1023, r = w & 31, c = w >> 5;
            const int i = o + 32 * (bi + 1) + r, j = o + 32 * (bj + 1) + c;
            float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
#pragma unroll 2
            for (int k = 0; k < 32; k += 4) {
                s0 += ak(a, i, o + k) * ak(a, j, o + k);
                s1 += ak(a, i, o + k + 1) * ak(a, j, o + k + 1);
                s2 += ak(a, i, o + k + 2) * ak(a, j, o + k + 2);
                s3 += ak(a, i, o + k + 3) * ak(a, j, o + k + 3);
            }
            ak(a, i, j) -= (s0 + s1) + (s2 + s3);
        }
        __syncthreads();
    }
    // ---- off-diagonal blocks of X by block diagonals ----
    for (int d = 1; d < nb; ++d) {
        const int nt = (nb - d) * 1024;
        // T_(j+d, j) = sum_{k=j}^{j+d-1} L_(j+d, k) X_(k, j), stored in the upper block (j, j+d) of x
        for (int e = tid; e < nt; e += KT) {
            const int bj = e >> 10, w = e & 1023, r = w & 31, c = w >> 5, bi = bj + d;
            float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
            for (int bk = bj; bk < bi; ++bk) {
#pragma unroll 2
                for (int k = 0; k < 32; k += 4) {
                    s0 += ak(a, 32 * bi + r, 32 * bk + k) * ak(x, 32 * bk + k, 32 * bj + c);
                    s1 += ak(a, 32 * bi + r, 32 * bk + k + 1) * ak(x, 32 * bk + k + 1, 32 * bj + c);
                    s2 += ak(a, 32 * bi + r, 32 * bk + k + 2) * ak(x, 32 * bk + k + 2, 32 * bj + c);
                    s3 += ak(a, 32 * bi + r, 32 * bk + k + 3) * ak(x, 32 * bk + k + 3, 32 * bj + c);
                }
            }
            ak(x, 32 * bj + r, 32 * bi + c) = (s0 + s1) + (s2 + s3);  // transposed slot: row r of T at (bj, bi)
        }
        __syncthreads();
        // X_(i, j) = -X_ii T,  X_ii lower
        for (int e = tid; e < nt; e += KT) {
            const int bj = e >> 10, w = e & 1023, r = w & 31, c = w >> 5, bi = bj + d;
            float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
            int k = 0;
            for (; k + 3 <= r; k += 4) {
                s0 += ak(x, 32 * bi + r, 32 * bi + k) * ak(x, 32 * bj + k, 32 * bi + c);
                s1 += ak(x, 32 * bi + r, 32 * bi + k + 1) * ak(x, 32 * bj + k + 1, 32 * bi + c);
                s2 += ak(x, 32 * bi + r, 32 * bi + k + 2) * ak(x, 32 * bj + k + 2, 32 * bi + c);
                s3 += ak(x, 32 * bi + r, 32 * bi + k + 3) * ak(x, 32 * bj + k + 3, 32 * bi + c);
            }
            for (; k <= r; ++k) s0 += ak(x, 32 * bi + r, 32 * bi + k) * ak(x, 32 * bj + k, 32 * bi + c);
            ak(x, 32 * bi + r, 32 * bj + c) = -((s0 + s1) + (s2 + s3));
        }
        __syncthreads();
    }
    // ---- write X (lower; the upper triangle is zero) and the scaled transposes ----
    const int r = tid & 127;  // thread: row r, every fourth column
    if (r < q) {
        for (int c = tid >> 7; c < q; c += 4) {
            const float v = (r >= c) ? ak(x, r, c) : 0.f;
            if (!isfinite(v)) atomicOr(status, ST_NONFINITE);
            if (out.dst) out.dst[r + (size_t)c * q] = v;
            // the transposes walk r fastest over their own columns: entry (r, c) of X^T is X(c, r)
            const float w = (c >= r) ? ak(x, c, r) : 0.f;
            if (out.xt1) out.xt1[r + (size_t)c * out.ld1] = out.s1 * w;
            if (out.xt2) out.xt2[r + (size_t)c * out.ld2] = out.s2 * w;
        }
    }
}

void launch_core_blk(cudaStream_t st, int q, const CoreOut &o0, const CoreOut *o1, int *status)
{
    static bool fattr = false;
    const size_t fsm = sizeof(float) * (2 * 128 * LDK);
    if (!fattr) {
        cudaFuncSetAttribute(k_core_blk, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fsm);
        fattr = true;
    }
    rb_count_launch();
    k_core_blk<<<o1 ? 2 : 1, KT, fsm, st>>>(q, o0, o1 ? *o1 : o0, status);
}

}  // namespace

bool launch_core_tr32(cudaStream_t st, int q, const float *M, float *Xinv, float *xt1, int ld1, float s1,
                      float *xt2, int ld2, float s2, int *status)
{
    if (q > 128) return false;
    launch_core_blk(st, q, CoreOut{nullptr, M, Xinv, xt1, ld1, s1, xt2, ld2, s2}, nullptr, status);
    return true;
}

void launch_core_ada32(cudaStream_t st, int q, const double *M, const double *N, float *Cinv, float *Dinv,
                       int *status)
{
    if (q <= 128) {
        CoreOut o0{M, nullptr, Cinv, nullptr, 0, 0.f, nullptr, 0, 0.f},
            o1{N, nullptr, Dinv, nullptr, 0, 0.f, nullptr, 0, 0.f};
        launch_core_blk(st, q, o0, (N && Dinv) ? &o1 : nullptr, status);
        return;
    }
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
