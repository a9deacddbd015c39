// core64.cu -- FP64 q x q core of AdaRBFGS for the FP32-storage tensor-core
// forms: the lower Cholesky factor of one symmetric q x q matrix
// (C C^T = S^T A S or D D^T = S~^T S~, Algorithm 4) and the inverse of that
// factor, factored and inverted in FP64 in one CTA, written out in FP32 the
// way the tensor-core GEMMs read it (scaled transposes into their B operands).
//
// The algorithm is the blocked right-looking one of k_core_blk in core32.cu
// (32 x 32 blocks, q padded to 32 nb with the identity): per block column p,
// the CTA factors and inverts the diagonal block (diag_block), all threads form the panel
// L_ip = A_ip X_pp^T and the trailing update A_ij -= L_ip L_jp^T; then the
// off-diagonal blocks of X = L^-1 follow by block diagonals d,
// T = sum_{k=j}^{i-1} L_ik X_kj, X_ij = -X_ii T (i = j + d).
// k_core_cl64 below spreads the same work over a cluster of CTAs.
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

// 1 / sqrt(d) in FP64 for a pivot d > 0: an FP32 estimate y refined by one step of cubic
// convergence from the series (1 - r)^(-1/2) = 1 + r/2 + 3 r^2/8 + ..., r = 1 - d y^2:
// y <- y + y r (1/2 + 3 r/8).  The estimate is good to ~2^-22, so the omitted r^3 term is ~2^-66,
// below FP64 rounding; the step is four dependent FP64 operations (GB300's FP64 units are few, and
// every one on this chain is paid for each of the q pivots in turn).  Outside [1e-30, 1e30] (or not
// finite) it takes sqrt and a division instead.
__device__ __forceinline__ double rsqrt_nr(double d)
{
    if (!(d > 1e-30 && d < 1e30)) return 1.0 / sqrt(d);
    const double y = (double)rsqrtf((float)d);
    const double t = d * y;
    const double r = fma(-t, y, 1.0);
    const double c = fma(0.375, r, 0.5);
    const double yr = y * r;
    return fma(yr, c, y);
}

// Dot product of len terms ab(k) = (u_k, v_k) in four partial sums (term k into sum k mod 4, each
// ascending, then (s0 + s1) + (s2 + s3)): four independent FMA chains instead of one.  Both FP64
// kernels use it for every element, so they agree bit for bit.
template <typename F>
__device__ __forceinline__ double dot4(int len, F ab)
{
    double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
    int k = 0;
    for (; k + 4 <= len; k += 4) {
        double u, v;
        ab(k, u, v);
        s0 = fma(u, v, s0);
        ab(k + 1, u, v);
        s1 = fma(u, v, s1);
        ab(k + 2, u, v);
        s2 = fma(u, v, s2);
        ab(k + 3, u, v);
        s3 = fma(u, v, s3);
    }
    double u, v;
    if (k < len) {
        ab(k, u, v);
        s0 = fma(u, v, s0);
    }
    if (k + 1 < len) {
        ab(k + 1, u, v);
        s1 = fma(u, v, s1);
    }
    if (k + 2 < len) {
        ab(k + 2, u, v);
        s2 = fma(u, v, s2);
    }
    return (s0 + s1) + (s2 + s3);
}

// The symmetric part of the q x q FP32 input, padded with the identity to 32 nb, into the lower
// block triangle of a.  M is first copied into xs (at least q (q + 1) floats) with coalesced reads
// and a padded pitch, so that both M_ij and M_ji are then read from shared memory without conflicts.
__device__ void load_sym(double *a, float *xs, int q, int nb, const float *src)
{
    const int tid = threadIdx.x, QP = 32 * nb, ps = q + 1;
    for (int e = tid; e < q * q; e += KT64) xs[(e % q) + (e / q) * ps] = src[e];
    __syncthreads();
    for (int e = tid; e < QP * QP; e += KT64) {
        const int i = e % QP, j = e / QP;
        if ((i >> 5) < (j >> 5)) continue;
        double v;
        if (i < q && j < q)
            v = 0.5 * ((double)xs[i + j * ps] + (double)xs[j + i * ps]);
        else
            v = (i == j) ? 1.0 : 0.0;
        pk(a, nb, i, j) = v;
    }
    __syncthreads();
}

// Panel element L_ip(r, c) = sum_{k <= c} A_ip(r, k) X_pp(c, k) (row i of the matrix, block column o).
__device__ __forceinline__ double panel_val(double *a, double *x, int nb, int i, int o, int c)
{
    return dot4(c + 1, [&](int k, double &u, double &v) {
        u = pk(a, nb, i, o + k);
        v = pk(x, nb, o + c, o + k);
    });
}

// Trailing-update term sum_{k < 32} L_ip(i, k) L_jp(j, k).
__device__ __forceinline__ double trail_val(double *a, int nb, int i, int j, int o)
{
    return dot4(32, [&](int k, double &u, double &v) {
        u = pk(a, nb, i, o + k);
        v = pk(a, nb, j, o + k);
    });
}

// T_j(r, c) = sum_{k = 32 bj}^{32 bi - 1} L(32 bi + r, k) X(k, 32 bj + c).
__device__ __forceinline__ double t_val(double *a, double *x, int nb, int bi, int bj, int r, int c)
{
    return dot4(32 * (bi - bj), [&](int kk, double &u, double &v) {
        const int k = 32 * bj + kk;
        u = pk(a, nb, 32 * bi + r, k);
        v = pk(x, nb, k, 32 * bj + c);
    });
}

// X_(bi, bj)(r, c) = -sum_{k <= r} X_(bi, bi)(r, k) T_bj(k, c).
__device__ __forceinline__ double x_val(double *x, const double *t, int nb, int bi, int bj, int r, int c)
{
    return -dot4(r + 1, [&](int k, double &u, double &v) {
        u = pk(x, nb, 32 * bi + r, 32 * bi + k);
        v = t[bj * BLK + k + c * BLD];
    });
}

// Pivot j of the diagonal block (warp 0): lane 0 takes the reciprocal square root of A_jj (stored
// as invd[j], L_jj = d / sqrt(d)), and every lane below the diagonal scales its element of column j.
__device__ __forceinline__ void pivot_col(double *a, int nb, int o, int j, double *invd, int *bad)
{
    const int lane = threadIdx.x & 31;
    double inv = 0.0;
    if (lane == 0) {
        const double d = pk(a, nb, o + j, o + j);
        if (!(d > 0.0) || !isfinite(d)) *bad = 1;
        inv = rsqrt_nr(d);
        invd[j] = inv;
        pk(a, nb, o + j, o + j) = d * inv;
    }
    inv = __shfl_sync(0xffffffffu, inv, 0);
    if (lane > j) pk(a, nb, o + lane, o + j) = pk(a, nb, o + lane, o + j) * inv;
}

// Diagonal block p (rows and columns o .. o + 31, o = 32 p) of the block-packed matrices:
// L_pp in place of A_pp (lower Cholesky) and X_pp = L_pp^-1, by all KT64 threads of the CTA.
// Cholesky with one pivot of look-ahead: while warps 1 .. 15 update columns j + 2 .. 31 with
// column j, warp 0 updates column j + 1, takes its pivot (one thread: GB300 runs FP64 at a small
// fraction of its FP32 rate, so the other warps do not repeat it) and scales it, so one barrier
// separates the steps.  X_pp right-looking: at step k every later row subtracts L_ik X_kc, X_kc
// taken as the unscaled row times the stored 1 / L_kk, and the rows are scaled once at the end.
// Each element sees the same operations in the same order as a textbook right-looking Cholesky and
// a forward substitution down each column of the inverse, whatever the warp that runs them.
// Sets *bad when a pivot is not positive and finite (the same in every thread).  invd: 32 doubles.
__device__ void diag_block(double *a, double *x, int nb, int o, double *invd, int *bad)
{
    const int tid = threadIdx.x;
    if (tid < 32) pivot_col(a, nb, o, 0, invd, bad);
    __syncthreads();
    for (int j = 0; j < 32; ++j) {
        // column j is final; update the block's trailing elements (r, c), j < c <= r, with it
        if (tid < 32) {
            if (j + 1 < 32) {
                const int r = tid;  // column j + 1, by warp 0, then its pivot
                if (r > j) pk(a, nb, o + r, o + j + 1) -= pk(a, nb, o + r, o + j) * pk(a, nb, o + j + 1, o + j);
                __syncwarp();
                pivot_col(a, nb, o, j + 1, invd, bad);
            }
        } else {
            for (int e = tid - 32; e < 1024; e += KT64 - 32) {  // columns j + 2 .. 31
                const int r = e >> 5, c = e & 31;
                if (c > j + 1 && c <= r) {
                    const double lij = pk(a, nb, o + r, o + j);
                    pk(a, nb, o + r, o + c) -= lij * pk(a, nb, o + c, o + j);
                }
            }
        }
        __syncthreads();
    }
    if (*bad) return;  // read after the last barrier: the same in every thread
    for (int e = tid; e < 1024; e += KT64) {
        const int r = e & 31, c = e >> 5;
        pk(x, nb, o + r, o + c) = (r == c) ? 1.0 : 0.0;
    }
    __syncthreads();
    for (int k = 0; k < 31; ++k) {
        for (int e = tid; e < 1024; e += KT64) {  // X_ic -= L_ik X_kc, i > k >= c
            const int i = e >> 5, c = e & 31;
            if (i > k && c <= k) {
                const double xkc = pk(x, nb, o + k, o + c) * invd[k];
                pk(x, nb, o + i, o + c) -= pk(a, nb, o + i, o + k) * xkc;
            }
        }
        __syncthreads();
    }
    for (int e = tid; e < 1024; e += KT64) {
        const int k = e >> 5, c = e & 31;
        if (c <= k) pk(x, nb, o + k, o + c) = pk(x, nb, o + k, o + c) * invd[k];
    }
    __syncthreads();
}

__global__ void __launch_bounds__(KT64, 1) k_core_blk64(int q, Core64Out out, int *status)
{
    extern __shared__ double smd[];
    const int nb = (q + 31) / 32;
    double *a = smd;                 // A, overwritten by L
    double *x = smd + NPACK * BLK;   // X = L^-1
    double *t = smd + 2 * NPACK * BLK;  // T blocks of the current block diagonal
    __shared__ int fail;
    __shared__ double invd[32];
    if (status_bad(status)) return;
    const int tid = threadIdx.x;
    if (tid == 0) fail = 0;
    // symmetric part of the padded matrix, lower block triangle only (identity padding); X's space
    // stages the FP32 input
    load_sym(a, (float *)x, q, nb, out.src);
    for (int p = 0; p < nb; ++p) {
        const int o = 32 * p;
        diag_block(a, x, nb, o, invd, &fail);
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
                pv[u] = panel_val(a, x, nb, o + 32 * (blk + 1) + r, o, c);
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
            pk(a, nb, i, j) -= trail_val(a, nb, i, j, o);
        }
        __syncthreads();
    }
    // off-diagonal blocks of X by block diagonals
    for (int d = 1; d < nb; ++d) {
        const int nt = (nb - d) * 1024;
        for (int e = tid; e < nt; e += KT64) {  // T_j = sum_{k=j}^{j+d-1} L_(j+d, k) X_(k, j)
            const int bj = e >> 10, w = e & 1023, r = w & 31, c = w >> 5, bi = bj + d;
            t[bj * BLK + r + c * BLD] = t_val(a, x, nb, bi, bj, r, c);
        }
        __syncthreads();
        for (int e = tid; e < nt; e += KT64) {  // X_(j+d, j) = -X_(j+d, j+d) T_j
            const int bj = e >> 10, w = e & 1023, r = w & 31, c = w >> 5, bi = bj + d;
            pk(x, nb, 32 * bi + r, 32 * bj + c) = x_val(x, t, nb, bi, bj, r, c);
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

// The same factorisation and inverse on a cluster of CL CTAs (q <= 128).  Every CTA keeps a
// full copy of A (-> L), X and T in its shared memory.  The diagonal blocks are factored and
// inverted by every CTA alike (identical work on identical copies, so every CTA takes the same
// branch on a failed pivot); the panel, the trailing update and the off-diagonal blocks of X are
// split over the cluster's threads, and each element, computed by one thread exactly as in
// k_core_blk64, is written to every CTA's copy through distributed shared memory before a
// cluster barrier.  The results are bit-identical to k_core_blk64; the FP64 work of the panels,
// updates and off-diagonal blocks is spread over CL SMs.
__device__ __forceinline__ void cl_sync()
{
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

__device__ __forceinline__ uint32_t cl_rank()
{
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

__device__ __forceinline__ uint32_t cl_nrank()
{
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
    return r;
}

// Shared-memory address of `local` in the CTA of cluster rank r.
__device__ __forceinline__ uint32_t cl_map(const void *local, uint32_t r)
{
    uint32_t out;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(out) : "r"((uint32_t)__cvta_generic_to_shared(local)), "r"(r));
    return out;
}

__device__ __forceinline__ void cl_st(uint32_t addr, double v)
{
    asm volatile("st.shared::cluster.f64 [%0], %1;" ::"r"(addr), "d"(v) : "memory");
}

// *p = v in every CTA of the cluster (p points into this CTA's shared memory)
__device__ __forceinline__ void put_all(double *p, double v, uint32_t ncl)
{
    for (uint32_t r = 0; r < ncl; ++r) cl_st(cl_map(p, r), v);
}

__global__ void __launch_bounds__(KT64, 1) k_core_cl64(int q, Core64Out out, int *status)
{
    extern __shared__ double smd[];
    const int nb = (q + 31) / 32;
    double *a = smd;
    double *x = smd + NPACK * BLK;
    double *t = smd + 2 * NPACK * BLK;
    __shared__ int flag;
    __shared__ double invd[32];
    const int tid = threadIdx.x;
    const uint32_t rank = cl_rank(), ncl = cl_nrank();
    const int gt = (int)rank * KT64 + tid, gstride = (int)ncl * KT64;  // this thread's share of the cluster's work
    // one reading of the status word for the whole cluster (rank 0's), so that every CTA takes
    // the same path through the cluster barriers below
    if (tid == 0) flag = (rank == 0 && status_bad(status)) ? 1 : 0;
    cl_sync();
    if (tid == 0 && rank != 0) {
        int v;
        asm volatile("ld.shared::cluster.s32 %0, [%1];" : "=r"(v) : "r"(cl_map(&flag, 0)) : "memory");
        flag = v;
    }
    cl_sync();  // rank 0's flag read everywhere before any CTA may leave
    if (flag) return;
    if (tid == 0) flag = 0;
    load_sym(a, (float *)x, q, nb, out.src);  // every copy loads the same symmetric part
    for (int p = 0; p < nb; ++p) {
        const int o = 32 * p;
        diag_block(a, x, nb, o, invd, &flag);  // in every CTA alike
        if (flag) {  // the same in every CTA (same data, same operations)
            if (tid == 0 && rank == 0) atomicOr(status, ST_NOTSPD);
            return;
        }
        // panel: L_ip = A_ip X_pp^T, i > p (every value computed before any copy is written)
        const int npanel = (nb - 1 - p) * 1024;
        constexpr int PV = (3 * 1024 + KT64 * 2 - 1) / (KT64 * 2);  // values per thread (clusters of >= 2 CTAs)
        double pv[PV];
#pragma unroll
        for (int u = 0; u < PV; ++u) {
            const int e = gt + u * gstride;
            pv[u] = 0.0;
            if (e < npanel) {
                const int blk = e >> 10, w = e & 1023, r = w & 31, c = w >> 5;
                pv[u] = panel_val(a, x, nb, o + 32 * (blk + 1) + r, o, c);
            }
        }
        cl_sync();
#pragma unroll
        for (int u = 0; u < PV; ++u) {
            const int e = gt + u * gstride;
            if (e < npanel) {
                const int blk = e >> 10, w = e & 1023, r = w & 31, c = w >> 5;
                put_all(&pk(a, nb, o + 32 * (blk + 1) + r, o + c), pv[u], ncl);
            }
        }
        cl_sync();
        // trailing update: A_ij -= L_ip L_jp^T over the lower block triangle p < bj <= bi
        const int m = nb - 1 - p;
        const int ntr = m * (m + 1) / 2 * 1024;
        for (int e = gt; e < ntr; e += gstride) {
            int blk = e >> 10, bj = 0;
            while (blk >= m - bj) {
                blk -= m - bj;
                ++bj;
            }
            const int bi = bj + blk, w = e & 1023, r = w & 31, c = w >> 5;
            const int i = o + 32 * (bi + 1) + r, j = o + 32 * (bj + 1) + c;
            double &dst = pk(a, nb, i, j);
            put_all(&dst, dst - trail_val(a, nb, i, j, o), ncl);
        }
        cl_sync();
    }
    // off-diagonal blocks of X by block diagonals
    for (int d = 1; d < nb; ++d) {
        const int nt = (nb - d) * 1024;
        for (int e = gt; e < nt; e += gstride) {  // T_j = sum_{k=j}^{j+d-1} L_(j+d, k) X_(k, j)
            const int bj = e >> 10, w = e & 1023, r = w & 31, c = w >> 5, bi = bj + d;
            put_all(&t[bj * BLK + r + c * BLD], t_val(a, x, nb, bi, bj, r, c), ncl);
        }
        cl_sync();
        for (int e = gt; e < nt; e += gstride) {  // X_(j+d, j) = -X_(j+d, j+d) T_j
            const int bj = e >> 10, w = e & 1023, r = w & 31, c = w >> 5, bi = bj + d;
            put_all(&pk(x, nb, 32 * bi + r, 32 * bj + c), x_val(x, t, nb, bi, bj, r, c), ncl);
        }
        cl_sync();
    }
    for (int e = gt; e < q * q; e += gstride) {
        const int r = e % q, c = e / q;
        const double w = (c >= r) ? pk(x, nb, c, r) : 0.0;
        if (!isfinite(w)) atomicOr(status, ST_NONFINITE);
        if (out.xt1) out.xt1[r + (size_t)c * out.ld1] = (float)(out.s1 * w);
        if (out.xt2) out.xt2[r + (size_t)c * out.ld2] = (float)(out.s2 * w);
    }
}

}  // namespace

int launch_core_tr64(cudaStream_t st, int q, const float *M, float *xt1, int ld1, float s1, float *xt2, int ld2,
                     float s2, int *status, int cluster)
{
    if (q > 32 * NBMAX) return 0;
    static bool attr = false;
    const size_t smem = sizeof(double) * (2 * NPACK + (NBMAX - 1)) * BLK;
    const Core64Out o{M, xt1, ld1, s1, xt2, ld2, s2};
    static int cl_ok = -1;  // 1 when a cluster of `cluster` CTAs of this kernel can be resident at all
    if (cluster > 1 && cl_ok != 0) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(cluster, 1, 1);
        cfg.blockDim = dim3(KT64, 1, 1);
        cfg.dynamicSmemBytes = smem;
        cfg.stream = st;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = cluster;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        if (cl_ok < 0) {
            int nclus = 0;
            cl_ok = cudaFuncSetAttribute(k_core_cl64, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) ==
                            cudaSuccess &&
                        cudaOccupancyMaxActiveClusters(&nclus, k_core_cl64, &cfg) == cudaSuccess && nclus > 0
                    ? 1
                    : 0;
            cudaGetLastError();
        }
        if (cl_ok == 1) {
            rb_count_launch();
            if (cudaLaunchKernelEx(&cfg, k_core_cl64, q, o, status) == cudaSuccess) return cluster;
            cudaGetLastError();  // not launched: one CTA below
        }
    }
    if (!attr) {
        if (cudaFuncSetAttribute(k_core_blk64, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
            return 0;
        attr = true;
    }
    rb_count_launch();
    k_core_blk64<<<1, KT64, smem, st>>>(q, o, status);
    return 1;
}
