// batch.cu -- many RBFGS problems of uneven size in one persistent launch.
//
// Each problem i is an SPD A_i (n_i x n_i, FP32) with iterate X_i (X0 = I)
// and a coordinate sketch: a contiguous block C of q_i coordinates drawn with
// probability proportional to its diagonal trace (the convenient
// probabilities of Sec. 7.2 with W = A^-1; Philox key = seed, counter stream
// = the problem's stream id).  One step is Eq. (qunac) with S = I[:, C]:
//   G = A[:, C], M = A[C, C], Y = X G, T = G^T Y, C C^T = M (FP64 Cholesky),
//   Lam = M^-1, W = S (Lam + Lam T Lam)/2 - Y Lam,
//   X[:, C] += W + (W[C, :])^T restricted to rows C, X[C, j] += W[j, :]^T (j not in C).
// The blocks are a fixed partition of [n], so M, its Cholesky factor and Lam
// depend only on the block: they are formed once per block when the batch is
// created (FP64 factorisation, Lam stored FP32) and a step reads the drawn
// block's Lam; a block whose Cholesky broke down makes the step that draws it
// fail with ST_NOTSPD, exactly as a factorisation inside the step would.
// A persistent grid pulls problems from an atomic work queue (largest n
// first); a CTA runs `steps` steps on its problem before taking the next.
// Every step of a problem runs in one CTA in a fixed order, so a problem's
// iterates do not depend on what else is in the batch.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <numeric>
#include <vector>

#include "kernels.cuh"

namespace {

constexpr int BT = 256;     // threads per CTA of the residual kernel
constexpr int QMAX = 32;    // largest block
constexpr int NMAX = 1024;  // largest problem
constexpr int YK = 128;           // columns of X (rows of G) per staged block of the Y pass
constexpr int GLD = QMAX + 4;     // row pitch of a staged G block (16-byte rows, 4-way bank spread)
constexpr int GT_FLOATS = YK * GLD;  // staged G: YK x GLD (Y), q x 32 or q x 32 cpw <= 4096 (T waves)
constexpr int PRE_WARPS = 2;     // warps (blocks) per CTA of the per-block factorisation

struct BatchDev {
    const float *A;
    float *X;
    const int64_t *off;  // element offset of problem i in A and X (a multiple of 4)
    const int *n, *q;
    const int *ld;       // leading dimension of A_i and X_i: n_i rounded up to a multiple of 4
    const uint64_t *P;  // trace-weight prefix sums, nb_i + 1 entries each
    const int64_t *offP;
    const int *nb;
    float *Lam;          // per block b of problem i: Lam_b = A[C_b, C_b]^-1, q x q (ld q)
    const int64_t *offL; // element offset of problem i's blocks in Lam
    int *bad;            // per block (offset offP[i]): 1 = its Cholesky broke down
    const uint64_t *stream;
    uint64_t *k;       // steps done
    const int *active; // 0 = skip
    int *status;       // per problem: ST_* bits
    const int *order;  // work order (largest n first)
    int *queue;
    int count;
    uint64_t seed;
};

__device__ void draw_block(const BatchDev &d, int p, int n, int q, uint64_t k, int &first, int &size, int &blk)
{
    const uint64_t *P = d.P + d.offP[p];
    const int nb = d.nb[p];
    const u32x4 w = philox10(0u, TAG_COORD, (uint32_t)k, (uint32_t)d.stream[p], (uint32_t)d.seed,
                             (uint32_t)(d.seed >> 32));
    const uint64_t r = (uint64_t)w.x | ((uint64_t)w.y << 32);
    const uint64_t t = __umul64hi(r, P[nb]);
    int lo = 0, hi = nb - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (P[mid] <= t)
            lo = mid;
        else
            hi = mid - 1;
    }
    blk = lo;
    first = lo * q;
    size = ((lo + 1) * q <= n) ? q : n - lo * q;
}

// One warp per (problem, block): M = A[C, C] padded with I to q x q (FP64), lower
// Cholesky M = C C^T (row per lane), C^-1 (column per lane), Lam = C^-T C^-1 (FP64 sums,
// stored FP32, ld q).  A pivot <= 0 or non-finite marks the block bad.
__global__ void __launch_bounds__(32 * PRE_WARPS) k_batch_blocks(BatchDev d, const int2 *items, int nitems)
{
    __shared__ double Ms[PRE_WARPS][QMAX * QMAX];
    __shared__ double Cs[PRE_WARPS][QMAX * QMAX];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int it = blockIdx.x * PRE_WARPS + w;
    if (it >= nitems) return;  // the whole warp: only warp-level syncs below
    const int p = items[it].x, blk = items[it].y;
    const int n = d.n[p], q = d.q[p], ld = d.ld[p];
    const int first = blk * q, size = min(q, n - first);
    const float *A = d.A + d.off[p];
    double *M = Ms[w], *Ci = Cs[w];
    for (int e = lane; e < q * q; e += 32) {
        const int a = e % q, b = e / q;
        M[a + b * QMAX] = (a < size && b < size) ? (double)A[(first + a) + (int64_t)(first + b) * ld]
                                                 : (a == b ? 1.0 : 0.0);
    }
    __syncwarp();
    bool fail = false;
    for (int j = 0; j < q; ++j) {
        const double dj = M[j + j * QMAX];  // the same value in every lane
        if (!(dj > 0.0) || !isfinite(dj)) {
            fail = true;
            break;
        }
        const double sd = sqrt(dj);
        __syncwarp();
        if (lane == j) M[j + j * QMAX] = sd;
        if (lane > j && lane < q) M[lane + j * QMAX] /= sd;
        __syncwarp();
        if (lane > j && lane < q) {
            const double lij = M[lane + j * QMAX];
            for (int c = j + 1; c <= lane; ++c) M[lane + c * QMAX] -= lij * M[c + j * QMAX];
        }
        __syncwarp();
    }
    if (fail) {
        if (lane == 0) d.bad[d.offP[p] + blk] = 1;
        return;
    }
    if (lane < q) {
        const int c = lane;
        Ci[c + c * QMAX] = 1.0 / M[c + c * QMAX];
        for (int i = c + 1; i < q; ++i) {
            double t = 0.0;
            for (int k = c; k < i; ++k) t += M[i + k * QMAX] * Ci[k + c * QMAX];
            Ci[i + c * QMAX] = -t / M[i + i * QMAX];
        }
    }
    __syncwarp();
    float *L = d.Lam + d.offL[p] + (int64_t)blk * q * q;
    for (int e = lane; e < q * q; e += 32) {
        const int a = e % q, b = e / q;
        double t = 0.0;
        for (int k = max(a, b); k < q; ++k) t += Ci[k + a * QMAX] * Ci[k + b * QMAX];
        L[a + b * q] = (float)t;
    }
}

// TB threads per CTA (the tile shape the autotuner picks: 256 or 512), RPT = NMAX / TB
// consecutive rows of every problem per thread (rows RPT t .. RPT t + RPT - 1), read from X
// as one 16- or 8-byte vector per column.  The order of every sum does not depend on TB, so the
// iterates are the same for every shape:
//   Y = X G     row by row, k ascending;
//   T = G^T Y   per (a, b): 32-row chunks summed k ascending, chunks added in ascending
//               order to a running total (a wave of chunks is computed in parallel when
//               q^2 < TB, but always added in chunk order);
//   q x q products and W = S B1 - Y Lam element by element, inner index ascending.
template <int TB>
__global__ void __launch_bounds__(TB, 1) k_batch_rbfgs(BatchDev d, int steps)
{
    constexpr int RPT = NMAX / TB;  // consecutive rows per thread
    constexpr int KU = 8;           // columns of X loaded ahead per thread
    constexpr int NPM = (QMAX * QMAX + TB - 1) / TB;
    extern __shared__ float bsm[];
    float *Ys = bsm;                     // n x q, ld ldy = ld + 4 (Y, then W); rows n .. ld - 1 are zero
    float *Gt = Ys + (NMAX + 4) * QMAX;  // staged rows of G = A[:, C]
    float *Lam = Gt + GT_FLOATS;         // QMAX x QMAX
    float *Tm = Lam + QMAX * QMAX;       // T, then sym(T) Lam
    float *B1 = Tm + QMAX * QMAX;        // (Lam + Lam T Lam) / 2
    float *part = B1 + QMAX * QMAX;      // TB chunk sums of T (one wave)
    __shared__ int s_item, s_first, s_size, s_blk, s_bad;

    const int tid = threadIdx.x;
    for (;;) {
        if (tid == 0) s_item = atomicAdd(d.queue, 1);
        __syncthreads();
        const int item = s_item;
        __syncthreads();
        if (item >= d.count) break;
        const int p = d.order[item];
        if (!d.active[p] || d.status[p]) continue;
        const int n = d.n[p], q = d.q[p], ld = d.ld[p];
        const float *A = d.A + d.off[p];
        float *X = d.X + d.off[p];
        const int ldy = ld + 4;  // 16-byte columns
        for (int s = 0; s < steps; ++s) {
            if (tid == 0) {
                int f, z, b;
                draw_block(d, p, n, q, d.k[p], f, z, b);
                s_first = f;
                s_size = z;
                s_blk = b;
                s_bad = d.bad[d.offP[p] + b];
            }
            __syncthreads();
            const int first = s_first, size = s_size;
            if (s_bad) {  // the drawn block's Cholesky broke down at creation: A is not SPD
                if (tid == 0) atomicOr(&d.status[p], ST_NOTSPD);
                __syncthreads();
                break;
            }
            {
                const float *Lg = d.Lam + d.offL[p] + (int64_t)s_blk * q * q;
                for (int e = tid; e < q * q; e += TB) Lam[(e % q) + (e / q) * QMAX] = Lg[e];
            }
            // Y = X G, G = A[:, C]: rows i0 .. i0 + RPT - 1; KU columns of X in flight per thread
            const int i0 = RPT * tid;
            float acc[RPT][QMAX];
#pragma unroll
            for (int r = 0; r < RPT; ++r)
#pragma unroll
                for (int c = 0; c < QMAX; ++c) acc[r][c] = 0.f;
            auto load_x = [&](float (&xv)[KU][RPT], int k0, int kb, int kend) {
#pragma unroll
                for (int u = 0; u < KU; ++u) {
                    const float *xp = X + i0 + (int64_t)(k0 + kb + u) * ld;
                    const bool ok = i0 < n && kb + u < kend;
                    if constexpr (RPT == 4) {
                        const float4 v = ok ? *(const float4 *)xp : make_float4(0.f, 0.f, 0.f, 0.f);
                        xv[u][0] = v.x;
                        xv[u][1] = v.y;
                        xv[u][2] = v.z;
                        xv[u][3] = v.w;
                    } else {
                        const float2 v = ok ? *(const float2 *)xp : make_float2(0.f, 0.f);
                        xv[u][0] = v.x;
                        xv[u][1] = v.y;
                    }
                }
            };
            for (int k0 = 0; k0 < n; k0 += YK) {
                const int kend = min(YK, n - k0);
                float xv[KU][RPT];
                load_x(xv, k0, 0, kend);  // in flight across the staging below
                __syncthreads();
                for (int e = tid; e < YK * QMAX; e += TB) {
                    const int kk = e % YK, c = e / YK;
                    Gt[kk * GLD + c] = (kk < kend && c < size) ? A[(k0 + kk) + (int64_t)(first + c) * ld] : 0.f;
                }
                __syncthreads();
                for (int kb = 0; kb < kend; kb += KU) {
                    float xn[KU][RPT];  // next columns, loaded while these are used
                    load_x(xn, k0, kb + KU, kend);
#pragma unroll
                    for (int u = 0; u < KU; ++u) {
                        const float4 *g4 = (const float4 *)(Gt + (kb + u) * GLD);
#pragma unroll
                        for (int c4 = 0; c4 < QMAX / 4; ++c4) {
                            if (4 * c4 >= q) break;
                            const float4 g = g4[c4];
#pragma unroll
                            for (int r = 0; r < RPT; ++r) {
                                acc[r][4 * c4] = fmaf(xv[u][r], g.x, acc[r][4 * c4]);
                                acc[r][4 * c4 + 1] = fmaf(xv[u][r], g.y, acc[r][4 * c4 + 1]);
                                acc[r][4 * c4 + 2] = fmaf(xv[u][r], g.z, acc[r][4 * c4 + 2]);
                                acc[r][4 * c4 + 3] = fmaf(xv[u][r], g.w, acc[r][4 * c4 + 3]);
                            }
                        }
                    }
#pragma unroll
                    for (int u = 0; u < KU; ++u)
#pragma unroll
                        for (int r = 0; r < RPT; ++r) xv[u][r] = xn[u][r];
                }
            }
            // Y rows i0 .. i0 + RPT - 1 as one vector per column; rows n .. ld - 1 get 0 (X's zero
            // rows, or no loads at all), which the T pass below reads
            if (i0 < ld) {
#pragma unroll
                for (int c = 0; c < QMAX; ++c) {
                    if (c >= q) break;
                    float *yp = Ys + i0 + c * ldy;
                    if constexpr (RPT == 4)
                        *(float4 *)yp = make_float4(acc[0][c], acc[1][c], acc[2][c], acc[3][c]);
                    else
                        *(float2 *)yp = make_float2(acc[0][c], acc[1][c]);
                }
            }
            __syncthreads();
            // T = G^T Y in 32-row chunks (see above); a staged chunk holds G's columns
            // contiguously (rows within a column), so both operands are read 4 rows at a time
            {
                const int P = q * q, nch = (n + 31) >> 5;
                if (P >= TB) {  // one chunk per wave, ceil(P / TB) pairs per thread
                    float tr[NPM];
#pragma unroll
                    for (int u = 0; u < NPM; ++u) tr[u] = 0.f;
                    for (int c = 0; c < nch; ++c) {
                        const int r0 = c * 32;
                        __syncthreads();
                        for (int e = tid; e < 32 * q; e += TB) {
                            const int kk = e % 32, a = e / 32;
                            Gt[a * 32 + kk] = (r0 + kk < n && a < size) ? A[(r0 + kk) + (int64_t)(first + a) * ld] : 0.f;
                        }
                        __syncthreads();
                        const int k4 = (min(32, n - r0) + 3) >> 2;  // rows up to ld - 1: Y and G are zero there
#pragma unroll
                        for (int u = 0; u < NPM; ++u) {
                            const int e = tid + u * TB;
                            if (e < P) {
                                const int a = e % q, b = e / q;
                                const float4 *y4 = (const float4 *)(Ys + r0 + b * ldy);
                                const float4 *g4 = (const float4 *)(Gt + a * 32);
                                float in = 0.f;
                                for (int kk = 0; kk < k4; ++kk) {
                                    const float4 g = g4[kk], y = y4[kk];
                                    in = fmaf(g.x, y.x, in);
                                    in = fmaf(g.y, y.y, in);
                                    in = fmaf(g.z, y.z, in);
                                    in = fmaf(g.w, y.w, in);
                                }
                                tr[u] += in;
                            }
                        }
                    }
#pragma unroll
                    for (int u = 0; u < NPM; ++u) {
                        const int e = tid + u * TB;
                        if (e < P) Tm[(e % q) + (e / q) * QMAX] = tr[u];
                    }
                } else {  // cpw chunks per wave, one pair per thread, added in chunk order by the pair's owner
                    const int cpw = TB / P, cr = 32 * cpw;
                    const int j = tid / P, e = tid % P, a = e % q, b = e / q;
                    const bool act = j < cpw;
                    float tr = 0.f;
                    for (int c0 = 0; c0 < nch; c0 += cpw) {
                        __syncthreads();
                        for (int f = tid; f < cr * q; f += TB) {
                            const int row = f % cr, aa = f / cr;
                            const int i = c0 * 32 + row;
                            Gt[aa * cr + row] = (i < n && aa < size) ? A[i + (int64_t)(first + aa) * ld] : 0.f;
                        }
                        __syncthreads();
                        if (act) {
                            float in = 0.f;
                            if (c0 + j < nch) {
                                const int r0 = (c0 + j) * 32, k4 = (min(32, n - r0) + 3) >> 2;
                                const float4 *y4 = (const float4 *)(Ys + r0 + b * ldy);
                                const float4 *g4 = (const float4 *)(Gt + a * cr + j * 32);
                                for (int kk = 0; kk < k4; ++kk) {
                                    const float4 g = g4[kk], y = y4[kk];
                                    in = fmaf(g.x, y.x, in);
                                    in = fmaf(g.y, y.y, in);
                                    in = fmaf(g.z, y.z, in);
                                    in = fmaf(g.w, y.w, in);
                                }
                            }
                            part[tid] = in;
                        }
                        __syncthreads();
                        if (tid < P)
                            for (int jj = 0; jj < cpw && c0 + jj < nch; ++jj) tr += part[jj * P + tid];
                    }
                    if (tid < P) Tm[a + b * QMAX] = tr;
                }
            }
            __syncthreads();
            // B1 = (Lam + Lam T Lam) / 2: first Tm <- sym(T) Lam (via registers), then Lam (Tm)
            float tl[NPM];
#pragma unroll
            for (int u = 0; u < NPM; ++u) {
                const int e = tid + u * TB;
                float t = 0.f;
                if (e < q * q) {
                    const int a = e % q, b = e / q;
                    for (int k = 0; k < q; ++k)
                        t = fmaf(0.5f * (Tm[a + k * QMAX] + Tm[k + a * QMAX]), Lam[k + b * QMAX], t);
                }
                tl[u] = t;
            }
            __syncthreads();
#pragma unroll
            for (int u = 0; u < NPM; ++u) {
                const int e = tid + u * TB;
                if (e < q * q) Tm[(e % q) + (e / q) * QMAX] = tl[u];
            }
            __syncthreads();
            for (int e = tid; e < q * q; e += TB) {
                const int a = e % q, b = e / q;
                float t = 0.f;
                for (int k = 0; k < q; ++k) t = fmaf(Lam[a + k * QMAX], Tm[k + b * QMAX], t);
                B1[a + b * QMAX] = 0.5f * (Lam[a + b * QMAX] + t);
            }
            __syncthreads();
            // W = -Y Lam + S B1, in place of Y (each thread its own rows, one vector per column)
            if (i0 < n) {
                float y[RPT][QMAX];
#pragma unroll
                for (int c = 0; c < QMAX; ++c) {
                    if constexpr (RPT == 4) {
                        const float4 v = c < q ? *(const float4 *)(Ys + i0 + c * ldy) : make_float4(0.f, 0.f, 0.f, 0.f);
                        y[0][c] = v.x;
                        y[1][c] = v.y;
                        y[2][c] = v.z;
                        y[3][c] = v.w;
                    } else {
                        const float2 v = c < q ? *(const float2 *)(Ys + i0 + c * ldy) : make_float2(0.f, 0.f);
                        y[0][c] = v.x;
                        y[1][c] = v.y;
                    }
                }
                for (int c = 0; c < q; ++c) {
                    float w[RPT];
#pragma unroll
                    for (int r = 0; r < RPT; ++r) w[r] = 0.f;
                    const float4 *l4 = (const float4 *)(Lam + c * QMAX);
#pragma unroll
                    for (int b4 = 0; b4 < QMAX / 4; ++b4) {
                        if (4 * b4 >= q) break;
                        const float4 l = l4[b4];
#pragma unroll
                        for (int r = 0; r < RPT; ++r) {
                            w[r] = fmaf(y[r][4 * b4], l.x, w[r]);
                            w[r] = fmaf(y[r][4 * b4 + 1], l.y, w[r]);
                            w[r] = fmaf(y[r][4 * b4 + 2], l.z, w[r]);
                            w[r] = fmaf(y[r][4 * b4 + 3], l.w, w[r]);
                        }
                    }
#pragma unroll
                    for (int r = 0; r < RPT; ++r) {
                        w[r] = -w[r];
                        const int ri = i0 + r - first;
                        if (ri >= 0 && ri < size) w[r] += B1[ri + c * QMAX];
                    }
                    float *wp = Ys + i0 + c * ldy;
                    if constexpr (RPT == 4)
                        *(float4 *)wp = make_float4(w[0], w[1], w[2], w[3]);
                    else
                        *(float2 *)wp = make_float2(w[0], w[1]);
                }
            }
            __syncthreads();
            // X[:, C] += W + (W[C, :])^T on rows C: all rows, consecutive rows across a warp
            for (int e = tid; e < n * size; e += TB) {
                const int i = e % n, c = e / n;
                const int ri = i - first;
                float dlt = Ys[i + c * ldy];
                if (ri >= 0 && ri < size) dlt += Ys[(first + c) + ri * ldy];
                X[i + (int64_t)(first + c) * ld] += dlt;
            }
            // X[C, j] += W[j, :]^T for columns j outside C: the q rows of a column across
            // consecutive threads
            for (int e = tid; e < q * n; e += TB) {
                const int c = e % q, j = e / q;
                if (c < size && (j < first || j >= first + size)) X[(first + c) + (int64_t)j * ld] += Ys[j + c * ldy];
            }
            __syncthreads();
            if (tid == 0) d.k[p] += 1;
            __syncthreads();
        }
    }
}

// Per-problem sampled residual: J = m distinct columns (Floyd with key col_seed,
// counter (t, TAG_COLS, 0, problem)), r_i^2 = (1/m) sum_{j in J} ||e_j - X A e_j||^2
// summed in FP64.  One CTA per problem.
__global__ void __launch_bounds__(BT) k_batch_resid(BatchDev d, int mcols, uint64_t col_seed, double *resid)
{
    __shared__ int J[64];
    __shared__ double red[BT];
    const int p = blockIdx.x;
    const int n = d.n[p], ld = d.ld[p];
    const int m = min(mcols, n);
    const float *A = d.A + d.off[p];
    const float *X = d.X + d.off[p];
    if (threadIdx.x == 0) {
        for (int i = 0; i < m; ++i) {
            const uint32_t t = (uint32_t)(n - m + i);
            const u32x4 w = philox10((uint32_t)i, TAG_COLS, 0u, (uint32_t)p, (uint32_t)col_seed,
                                     (uint32_t)(col_seed >> 32));
            const int dd = (int)(((uint64_t)w.x * (uint64_t)(t + 1u)) >> 32);
            bool seen = false;
            for (int a = 0; a < i; ++a) seen |= (J[a] == dd);
            J[i] = seen ? (int)t : dd;
        }
    }
    __syncthreads();
    double s = 0.0;
    for (int jj = 0; jj < m; ++jj) {
        const int j = J[jj];
        for (int i = threadIdx.x; i < n; i += BT) {
            float z = 0.f;
            for (int k = 0; k < n; ++k) z = fmaf(X[i + (int64_t)k * ld], A[k + (int64_t)j * ld], z);
            const double e = ((i == j) ? 1.0 : 0.0) - (double)z;
            s += e * e;
        }
    }
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = BT / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) resid[p] = sqrt(red[0] / m);
}

__global__ void k_batch_identity(BatchDev d)
{
    const int p = blockIdx.y;
    const int n = d.n[p], ld = d.ld[p];
    float *X = d.X + d.off[p];
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < (int64_t)ld * n;
         e += (int64_t)gridDim.x * blockDim.x)
        X[e] = ((e % ld) == (e / ld)) ? 1.f : 0.f;  // rows n .. ld - 1 stay zero
}

constexpr size_t batch_smem(int tb)
{
    return sizeof(float) * ((NMAX + 4) * QMAX + GT_FLOATS + 3 * QMAX * QMAX + tb);
}

}  // namespace

struct rb_batch {
    int count = 0;
    cudaStream_t st = nullptr;
    std::vector<int> n, q, nb, order, ld;
    std::vector<int64_t> off, offP, offL;
    float *A = nullptr, *X = nullptr, *Lam = nullptr;
    uint64_t *P = nullptr, *k = nullptr, *stream = nullptr;
    int64_t *d_off = nullptr, *d_offP = nullptr, *d_offL = nullptr;
    int *d_bad = nullptr;
    int *d_n = nullptr, *d_q = nullptr, *d_ld = nullptr, *d_nb = nullptr, *d_order = nullptr, *d_active = nullptr,
        *d_status = nullptr, *d_queue = nullptr;
    double *d_resid = nullptr;
    int tb = 256;                // threads per CTA of the step kernel (picked by the autotuner)
    int *h_active = nullptr;     // pinned
    double *h_resid = nullptr;   // pinned
    int *h_status = nullptr;     // pinned
    uint64_t seed = 0;
    int grid = 0;
    cudaGraphExec_t gexec = nullptr;
    int g_steps = -1, g_cols = -1;
    uint64_t g_seed = 0;

    BatchDev dev() const
    {
        BatchDev d;
        d.A = A;
        d.X = X;
        d.off = d_off;
        d.n = d_n;
        d.q = d_q;
        d.ld = d_ld;
        d.P = P;
        d.offP = d_offP;
        d.nb = d_nb;
        d.Lam = Lam;
        d.offL = d_offL;
        d.bad = d_bad;
        d.stream = stream;
        d.k = k;
        d.active = d_active;
        d.status = d_status;
        d.order = d_order;
        d.queue = d_queue;
        d.count = count;
        d.seed = seed;
        return d;
    }
};

static void batch_free(rb_batch *b)
{
    if (!b) return;
    if (b->gexec) cudaGraphExecDestroy(b->gexec);
    void *ptrs[] = {b->A, b->X, b->Lam, b->P, b->k, b->stream, b->d_off, b->d_offP, b->d_offL, b->d_bad, b->d_n,
                    b->d_q, b->d_ld, b->d_nb, b->d_order, b->d_active, b->d_status, b->d_queue, b->d_resid};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    if (b->h_active) cudaFreeHost(b->h_active);
    if (b->h_resid) cudaFreeHost(b->h_resid);
    if (b->h_status) cudaFreeHost(b->h_status);
    delete b;
}

static void launch_batch_step(rb_batch *b, cudaStream_t st, int steps)
{
    if (b->tb == 512)
        k_batch_rbfgs<512><<<b->grid, 512, batch_smem(512), st>>>(b->dev(), steps);
    else
        k_batch_rbfgs<256><<<b->grid, 256, batch_smem(256), st>>>(b->dev(), steps);
}

// Tile-shape autotuner.  Candidates: 256 or 512 threads per CTA (4 or 2 rows of each
// problem per thread).  Keyed by the batch's largest n (rounded up to a power of two),
// its largest q and the precision (FP32): the first batch of a key times two steps of
// every problem with each shape and keeps the faster; later batches of the key reuse it.
// The iterates do not depend on the shape, so the choice changes only the speed.  The
// trial steps are undone (X = I, k = 0, status cleared) before the batch is returned.
std::mutex g_tune_mu;
std::map<uint64_t, int> g_tune;

static rb_status batch_autotune(rb_batch *b)
{
    int nmax = 1, qmax = 1;
    for (int i = 0; i < b->count; ++i) {
        nmax = std::max(nmax, b->n[i]);
        qmax = std::max(qmax, b->q[i]);
    }
    int nb2 = 1;
    while (nb2 < nmax) nb2 <<= 1;
    const uint64_t key = ((uint64_t)nb2 << 32) | ((uint64_t)qmax << 8) | (uint64_t)RB_FP32;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tune.find(key);
        if (it != g_tune.end()) {
            b->tb = it->second;
            return RB_OK;
        }
    }
    cudaStream_t st = b->st;
    cudaEvent_t e0, e1;
    RB_CUDA(cudaEventCreate(&e0));
    RB_CUDA(cudaEventCreate(&e1));
    float best = INFINITY;
    int best_tb = 256;
    for (int tb : {256, 512}) {
        b->tb = tb;
        cudaMemsetAsync(b->d_queue, 0, sizeof(int), st);
        cudaEventRecord(e0, st);
        rb_count_launch();
        launch_batch_step(b, st, 2);
        cudaEventRecord(e1, st);
        if (cudaEventSynchronize(e1) != cudaSuccess) {
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            return RB_ECUDA;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best) {
            best = ms;
            best_tb = tb;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    b->tb = best_tb;
    // undo the trial steps
    rb_count_launch();
    k_batch_identity<<<dim3(64, b->count), 256, 0, st>>>(b->dev());
    RB_CUDA(cudaMemsetAsync(b->k, 0, sizeof(uint64_t) * b->count, st));
    RB_CUDA(cudaMemsetAsync(b->d_status, 0, sizeof(int) * b->count, st));
    RB_CUDA(cudaStreamSynchronize(st));
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune[key] = best_tb;
    return RB_OK;
}

extern "C" rb_status rb_batch_tile(rb_batch_t b, int *threads_per_cta)
{
    if (!b || !threads_per_cta) return RB_EINVAL;
    *threads_per_cta = b->tb;
    return RB_OK;
}

extern "C" rb_status rb_batch_set_tile(rb_batch_t b, int threads_per_cta)
{
    if (!b || (threads_per_cta != 256 && threads_per_cta != 512)) return RB_EINVAL;
    if (threads_per_cta != b->tb && b->gexec) {  // the captured round launches the old shape
        cudaGraphExecDestroy(b->gexec);
        b->gexec = nullptr;
    }
    b->tb = threads_per_cta;
    return RB_OK;
}

template <typename P>
static bool dalloc(P **p, size_t bytes)
{
    return cudaMalloc((void **)p, bytes ? bytes : 16) == cudaSuccess;
}

extern "C" rb_status rb_batch_create(rb_batch_t *out, int count, const int *n, const void *const *A_dev,
                                     const int64_t *lda, int a_is_fp64, const int *q, const uint64_t *stream_ids,
                                     uint64_t seed, void *stream)
{
    if (!out || count < 1 || !n || !A_dev || !lda || !q) return RB_EINVAL;
    *out = nullptr;
    for (int i = 0; i < count; ++i) {
        if (n[i] < 1 || n[i] > NMAX || q[i] < 1 || q[i] > QMAX || q[i] > n[i] || lda[i] < n[i] || !A_dev[i])
            return RB_EINVAL;
        if (q[i] % 4) return RB_EUNSUPPORTED;  // blocks of whole float4 columns
    }
    rb_batch *b = new rb_batch();
    b->count = count;
    b->st = (cudaStream_t)stream;
    b->seed = seed;
    b->n.assign(n, n + count);
    b->q.assign(q, q + count);
    b->off.resize(count);
    b->offP.resize(count);
    b->offL.resize(count);
    b->nb.resize(count);
    b->ld.resize(count);
    int64_t tot = 0, totP = 0, totL = 0;
    std::vector<int2> items;  // (problem, block) pairs of the per-block factorisation
    for (int i = 0; i < count; ++i) {
        b->ld[i] = (n[i] + 3) & ~3;  // 16-byte columns: rows RPT t .. are read as one vector
        b->off[i] = tot;
        tot += (int64_t)b->ld[i] * n[i];
        b->nb[i] = (n[i] + q[i] - 1) / q[i];
        b->offP[i] = totP;
        totP += b->nb[i] + 1;
        b->offL[i] = totL;
        totL += (int64_t)b->nb[i] * q[i] * q[i];
        for (int c = 0; c < b->nb[i]; ++c) items.push_back(make_int2(i, c));
    }
    b->order.resize(count);
    std::iota(b->order.begin(), b->order.end(), 0);
    std::stable_sort(b->order.begin(), b->order.end(), [&](int x, int y) { return n[x] > n[y]; });
    int2 *d_items = nullptr;
    bool ok = dalloc(&b->A, sizeof(float) * tot) && dalloc(&b->X, sizeof(float) * tot) &&
              dalloc(&b->Lam, sizeof(float) * totL) && dalloc(&b->d_offL, sizeof(int64_t) * count) &&
              dalloc(&b->d_bad, sizeof(int) * totP) && dalloc(&d_items, sizeof(int2) * items.size()) &&
              dalloc(&b->P, sizeof(uint64_t) * totP) && dalloc(&b->k, sizeof(uint64_t) * count) &&
              dalloc(&b->stream, sizeof(uint64_t) * count) && dalloc(&b->d_off, sizeof(int64_t) * count) &&
              dalloc(&b->d_offP, sizeof(int64_t) * count) && dalloc(&b->d_n, sizeof(int) * count) &&
              dalloc(&b->d_q, sizeof(int) * count) && dalloc(&b->d_ld, sizeof(int) * count) && dalloc(&b->d_nb, sizeof(int) * count) &&
              dalloc(&b->d_order, sizeof(int) * count) && dalloc(&b->d_active, sizeof(int) * count) &&
              dalloc(&b->d_status, sizeof(int) * count) && dalloc(&b->d_queue, sizeof(int)) &&
              dalloc(&b->d_resid, sizeof(double) * count) &&
              cudaMallocHost(&b->h_active, sizeof(int) * count) == cudaSuccess &&
              cudaMallocHost(&b->h_resid, sizeof(double) * count) == cudaSuccess &&
              cudaMallocHost(&b->h_status, sizeof(int) * count) == cudaSuccess;
    struct ItemsFree {
        int2 *p;
        ~ItemsFree()
        {
            if (p) cudaFree(p);
        }
    } items_guard{d_items};  // the block list is needed only while the batch is created
    if (!ok) {
        cudaGetLastError();
        batch_free(b);
        return RB_ENOMEM;
    }
    cudaStream_t st = b->st;
    // pack A (FP32) and compute the trace weights of every problem's blocks
    std::vector<uint64_t> hP(totP);
    std::vector<double> diag;
    if (cudaMemsetAsync(b->A, 0, sizeof(float) * tot, st) != cudaSuccess) {  // rows n .. ld - 1 stay zero
        batch_free(b);
        return RB_ECUDA;
    }
    for (int i = 0; i < count; ++i) {
        if (a_is_fp64)
            launch_copy2d<double, float>(st, n[i], n[i], (const double *)A_dev[i], lda[i], b->A + b->off[i], b->ld[i],
                                         1.0);
        else
            launch_copy2d<float, float>(st, n[i], n[i], (const float *)A_dev[i], lda[i], b->A + b->off[i], b->ld[i],
                                        1.0);
    }
    // diagonals of the packed FP32 A (the values the kernels use)
    std::vector<float> hd;
    for (int i = 0; i < count; ++i) {
        hd.resize(n[i]);
        if (cudaMemcpy2DAsync(hd.data(), sizeof(float), b->A + b->off[i], sizeof(float) * (b->ld[i] + 1), sizeof(float),
                              n[i], cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess) {
            batch_free(b);
            return RB_ECUDA;
        }
        const int nbi = b->nb[i], qi = q[i];
        std::vector<double> s(nbi);
        double T = 0.0;
        for (int c = 0; c < nbi; ++c) {
            double acc = 0.0;
            for (int r = c * qi; r < n[i] && r < (c + 1) * qi; ++r) acc += (double)hd[r];
            s[c] = acc;
        }
        for (int c = 0; c < nbi; ++c) T += s[c];
        uint64_t *Pi = hP.data() + b->offP[i];
        Pi[0] = 0;
        for (int c = 0; c < nbi; ++c) {
            if (!(s[c] > 0.0) || !(T > 0.0)) {
                batch_free(b);
                return RB_ENOTSPD;
            }
            uint64_t w = (uint64_t)floor(ldexp(s[c] / T, 52));
            if (w == 0) w = 1;
            Pi[c + 1] = Pi[c] + w;
        }
    }
    std::vector<uint64_t> sid(count);
    for (int i = 0; i < count; ++i) sid[i] = stream_ids ? stream_ids[i] : (uint64_t)i;
    for (int i = 0; i < count; ++i) b->h_active[i] = 1;
    bool cp = cudaMemcpyAsync(b->P, hP.data(), sizeof(uint64_t) * totP, cudaMemcpyHostToDevice, st) == cudaSuccess &&
              cudaMemcpyAsync(b->stream, sid.data(), sizeof(uint64_t) * count, cudaMemcpyHostToDevice, st) ==
                  cudaSuccess &&
              cudaMemcpyAsync(b->d_off, b->off.data(), sizeof(int64_t) * count, cudaMemcpyHostToDevice, st) ==
                  cudaSuccess &&
              cudaMemcpyAsync(b->d_offP, b->offP.data(), sizeof(int64_t) * count, cudaMemcpyHostToDevice, st) ==
                  cudaSuccess &&
              cudaMemcpyAsync(b->d_offL, b->offL.data(), sizeof(int64_t) * count, cudaMemcpyHostToDevice, st) ==
                  cudaSuccess &&
              cudaMemcpyAsync(d_items, items.data(), sizeof(int2) * items.size(), cudaMemcpyHostToDevice, st) ==
                  cudaSuccess &&
              cudaMemsetAsync(b->d_bad, 0, sizeof(int) * totP, st) == cudaSuccess &&
              cudaMemcpyAsync(b->d_n, n, sizeof(int) * count, cudaMemcpyHostToDevice, st) == cudaSuccess &&
              cudaMemcpyAsync(b->d_q, q, sizeof(int) * count, cudaMemcpyHostToDevice, st) == cudaSuccess &&
              cudaMemcpyAsync(b->d_ld, b->ld.data(), sizeof(int) * count, cudaMemcpyHostToDevice, st) ==
                  cudaSuccess &&
              cudaMemcpyAsync(b->d_nb, b->nb.data(), sizeof(int) * count, cudaMemcpyHostToDevice, st) ==
                  cudaSuccess &&
              cudaMemcpyAsync(b->d_order, b->order.data(), sizeof(int) * count, cudaMemcpyHostToDevice, st) ==
                  cudaSuccess &&
              cudaMemcpyAsync(b->d_active, b->h_active, sizeof(int) * count, cudaMemcpyHostToDevice, st) ==
                  cudaSuccess &&
              cudaMemsetAsync(b->k, 0, sizeof(uint64_t) * count, st) == cudaSuccess &&
              cudaMemsetAsync(b->d_status, 0, sizeof(int) * count, st) == cudaSuccess;
    if (cp) {
        dim3 g(64, count);
        rb_count_launch();
        k_batch_identity<<<g, 256, 0, st>>>(b->dev());
        const int nit = (int)items.size();
        rb_count_launch();
        k_batch_blocks<<<(nit + PRE_WARPS - 1) / PRE_WARPS, 32 * PRE_WARPS, 0, st>>>(b->dev(), d_items, nit);
        cp = cudaStreamSynchronize(st) == cudaSuccess;
    }
    if (!cp) {
        batch_free(b);
        return RB_ECUDA;
    }
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(k_batch_rbfgs<256>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)batch_smem(256));
        cudaFuncSetAttribute(k_batch_rbfgs<512>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)batch_smem(512));
        attr = true;
    }
    int sms = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    b->grid = std::max(1, std::min(count, sms > 0 ? sms : 148));
    const rb_status ts = batch_autotune(b);
    if (ts != RB_OK) {
        batch_free(b);
        return ts;
    }
    *out = b;
    return RB_OK;
}

// One round: reset the queue, `steps` steps on every active problem (one
// persistent launch), then the sampled residual of every problem and its
// copy to pinned host memory.  Captured once per (steps, ncols, col_seed)
// as a CUDA graph and replayed.
static rb_status batch_round(rb_batch *b, int steps, int ncols, uint64_t col_seed)
{
    cudaStream_t st = b->st;
    if (!b->gexec || b->g_steps != steps || b->g_cols != ncols || b->g_seed != col_seed) {
        if (b->gexec) {
            cudaGraphExecDestroy(b->gexec);
            b->gexec = nullptr;
        }
        cudaStream_t cs;
        if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) return RB_ECUDA;
        cudaGraph_t g = nullptr;
        bool ok = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
        if (ok) {
            cudaMemcpyAsync(b->d_active, b->h_active, sizeof(int) * b->count, cudaMemcpyHostToDevice, cs);
            cudaMemsetAsync(b->d_queue, 0, sizeof(int), cs);
            if (steps > 0) launch_batch_step(b, cs, steps);
            if (ncols > 0) {
                k_batch_resid<<<b->count, BT, 0, cs>>>(b->dev(), ncols, col_seed, b->d_resid);
                cudaMemcpyAsync(b->h_resid, b->d_resid, sizeof(double) * b->count, cudaMemcpyDeviceToHost, cs);
            }
            cudaMemcpyAsync(b->h_status, b->d_status, sizeof(int) * b->count, cudaMemcpyDeviceToHost, cs);
            ok = cudaStreamEndCapture(cs, &g) == cudaSuccess;
        }
        if (ok) ok = cudaGraphInstantiate(&b->gexec, g, 0) == cudaSuccess;
        if (g) cudaGraphDestroy(g);
        cudaStreamDestroy(cs);
        if (!ok) {
            cudaGetLastError();
            return RB_ECUDA;
        }
        b->g_steps = steps;
        b->g_cols = ncols;
        b->g_seed = col_seed;
    }
    RB_CUDA(cudaGraphLaunch(b->gexec, st));
    if (steps > 0) rb_count_launch();  // kernels in the graph replay
    if (ncols > 0) rb_count_launch();
    RB_CUDA(cudaStreamSynchronize(st));
    return RB_OK;
}

extern "C" rb_status rb_batch_step(rb_batch_t b, int steps)
{
    if (!b || steps < 0) return RB_EINVAL;
    return batch_round(b, steps, 0, 0);
}

extern "C" rb_status rb_batch_residual(rb_batch_t b, int ncols, uint64_t col_seed, double *out)
{
    if (!b || !out || ncols < 1 || ncols > 64) return RB_EINVAL;
    RB_TRY(batch_round(b, 0, ncols, col_seed));
    memcpy(out, b->h_resid, sizeof(double) * b->count);
    return RB_OK;
}

extern "C" rb_status rb_batch_solve(rb_batch_t b, double tol, int max_iter, int check_every, int ncols, int *iters,
                                    double *resid, int *status, int *nconverged)
{
    if (!b || check_every < 1 || max_iter < 0 || ncols < 1 || ncols > 64) return RB_EINVAL;
    const int count = b->count;
    std::vector<int> it(count, 0);
    std::vector<double> r(count, INFINITY);
    int done = 0, conv = 0;
    for (int i = 0; i < count; ++i) b->h_active[i] = 1;
    const uint64_t col_seed = 0xba7c4000ull;  // fixed: one graph for the whole solve
    while (done < max_iter) {
        const int chunk = std::min(check_every, max_iter - done);
        RB_TRY(batch_round(b, chunk, ncols, col_seed));
        done += chunk;
        int active = 0;
        for (int i = 0; i < count; ++i) {
            if (!b->h_active[i]) continue;
            it[i] = done;
            r[i] = b->h_resid[i];
            if (b->h_status[i] != 0 || r[i] <= tol || !isfinite(r[i])) {
                b->h_active[i] = 0;
                if (b->h_status[i] == 0 && r[i] <= tol) ++conv;
            } else {
                ++active;
            }
        }
        if (!active) break;
    }
    for (int i = 0; i < count; ++i) {
        if (iters) iters[i] = it[i];
        if (resid) resid[i] = r[i];
        if (status) status[i] = (b->h_status[i] & ST_NOTSPD) ? RB_ENOTSPD : (r[i] <= tol ? RB_OK : RB_NOTCONV);
    }
    if (nconverged) *nconverged = conv;
    return conv == count ? RB_OK : RB_NOTCONV;
}

extern "C" rb_status rb_batch_export(rb_batch_t b, int i, void *out_dev, int64_t ld)
{
    if (!b || i < 0 || i >= b->count || !out_dev || ld < b->n[i]) return RB_EINVAL;
    launch_copy2d<float, float>(b->st, b->n[i], b->n[i], b->X + b->off[i], b->ld[i], (float *)out_dev, ld, 1.0);
    RB_CUDA(cudaGetLastError());
    return RB_OK;
}

extern "C" rb_status rb_batch_destroy(rb_batch_t b)
{
    if (!b) return RB_EINVAL;
    cudaStreamSynchronize(b->st);
    batch_free(b);
    return RB_OK;
}
