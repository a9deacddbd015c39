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

struct BatchDev {
    const float *A;
    float *X;
    const int64_t *off;  // element offset of problem i in A and X
    const int *n, *q;
    const uint64_t *P;  // trace-weight prefix sums, nb_i + 1 entries each
    const int64_t *offP;
    const int *nb;
    const uint64_t *stream;
    uint64_t *k;       // steps done
    const int *active; // 0 = skip
    int *status;       // per problem: ST_* bits
    const int *order;  // work order (largest n first)
    int *queue;
    int count;
    uint64_t seed;
};

__device__ void draw_block(const BatchDev &d, int p, int n, int q, uint64_t k, int &first, int &size)
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
    first = lo * q;
    size = ((lo + 1) * q <= n) ? q : n - lo * q;
}

// TB threads per CTA (the tile shape the autotuner picks: 256 or 512), NMAX / TB rows of
// every problem per thread.  The order of every sum (Y row by row over k, T element by
// element over i, the q x q products element by element) does not depend on TB, so
// the iterates are the same for every shape.
template <int TB>
__global__ void __launch_bounds__(TB, 1) k_batch_rbfgs(BatchDev d, int steps)
{
    constexpr int BT = TB;
    constexpr int RPT = NMAX / TB;  // rows per thread
    extern __shared__ float bsm[];
    float *Ys = bsm;                                  // n x q, ld n + 1 (Y, then W)
    float *Gt = Ys + (NMAX + 1) * QMAX;               // 32 x QMAX tile of G rows
    double *Md = (double *)(Gt + 32 * QMAX);          // QMAX x QMAX (M, then C)
    float *Lam = (float *)(Md + QMAX * QMAX);         // QMAX x QMAX
    float *Tm = Lam + QMAX * QMAX;                    // T, then Lam T
    float *B1 = Tm + QMAX * QMAX;                     // (Lam + Lam T Lam) / 2
    float *Ci = B1 + QMAX * QMAX;                     // C^-1
    __shared__ int s_item, s_first, s_size, s_fail;

    const int tid = threadIdx.x;
    for (;;) {
        if (tid == 0) s_item = atomicAdd(d.queue, 1);
        __syncthreads();
        const int item = s_item;
        __syncthreads();
        if (item >= d.count) break;
        const int p = d.order[item];
        if (!d.active[p] || d.status[p]) continue;
        const int n = d.n[p], q = d.q[p];
        const float *A = d.A + d.off[p];
        float *X = d.X + d.off[p];
        const int ldy = n + 1;
        for (int s = 0; s < steps; ++s) {
            if (tid == 0) {
                int f, z;
                draw_block(d, p, n, q, d.k[p], f, z);
                s_first = f;
                s_size = z;
                s_fail = 0;
            }
            __syncthreads();
            const int first = s_first, size = s_size;
            // M = A[C, C] padded with I (FP64)
            for (int e = tid; e < q * q; e += BT) {
                const int a = e % q, b = e / q;
                Md[a + b * QMAX] = (a < size && b < size) ? (double)A[(first + a) + (int64_t)(first + b) * n]
                                                          : (a == b ? 1.0 : 0.0);
            }
            // Y = X G, G = A[:, C]: rows i = tid + BT r
            float acc[RPT][QMAX];
#pragma unroll
            for (int r = 0; r < RPT; ++r)
#pragma unroll
                for (int c = 0; c < QMAX; ++c) acc[r][c] = 0.f;
            for (int k0 = 0; k0 < n; k0 += 32) {
                __syncthreads();
                for (int e = tid; e < 32 * QMAX; e += BT) {
                    const int kk = e % 32, c = e / 32;
                    Gt[kk * QMAX + c] = (k0 + kk < n && c < size) ? A[(k0 + kk) + (int64_t)(first + c) * n] : 0.f;
                }
                __syncthreads();
                const int kend = min(32, n - k0);
                for (int kk = 0; kk < kend; ++kk) {
                    const float4 *g4 = (const float4 *)(Gt + kk * QMAX);
#pragma unroll
                    for (int r = 0; r < RPT; ++r) {
                        const int i = tid + BT * r;
                        if (i >= n) break;
                        const float x = X[i + (int64_t)(k0 + kk) * n];
#pragma unroll
                        for (int c4 = 0; c4 < QMAX / 4; ++c4) {
                            if (4 * c4 >= q) break;
                            const float4 g = g4[c4];
                            acc[r][4 * c4] = fmaf(x, g.x, acc[r][4 * c4]);
                            acc[r][4 * c4 + 1] = fmaf(x, g.y, acc[r][4 * c4 + 1]);
                            acc[r][4 * c4 + 2] = fmaf(x, g.z, acc[r][4 * c4 + 2]);
                            acc[r][4 * c4 + 3] = fmaf(x, g.w, acc[r][4 * c4 + 3]);
                        }
                    }
                }
            }
#pragma unroll
            for (int r = 0; r < RPT; ++r) {
                const int i = tid + BT * r;
                if (i >= n) break;
#pragma unroll
                for (int c = 0; c < QMAX; ++c)
                    if (c < q) Ys[i + c * ldy] = acc[r][c];
            }
            __syncthreads();
            // T = G^T Y (FP32 over n rows, i ascending): G's rows staged 32 at a time like the
            // Y pass, each (a, b) summed by one thread
            {
                constexpr int NP = (QMAX * QMAX + BT - 1) / BT;
                float t[NP];
#pragma unroll
                for (int u = 0; u < NP; ++u) t[u] = 0.f;
                for (int i0 = 0; i0 < n; i0 += 32) {
                    __syncthreads();
                    for (int e = tid; e < 32 * QMAX; e += BT) {
                        const int kk = e % 32, c = e / 32;
                        Gt[kk * QMAX + c] = (i0 + kk < n && c < size) ? A[(i0 + kk) + (int64_t)(first + c) * n] : 0.f;
                    }
                    __syncthreads();
                    const int kend = min(32, n - i0);
#pragma unroll
                    for (int u = 0; u < NP; ++u) {
                        const int e = tid + u * BT;
                        if (e < q * q) {
                            const int a = e % q, b = e / q;
                            const float *yb = Ys + i0 + b * ldy;
                            for (int kk = 0; kk < kend; ++kk) t[u] = fmaf(Gt[kk * QMAX + a], yb[kk], t[u]);
                        }
                    }
                }
#pragma unroll
                for (int u = 0; u < NP; ++u) {
                    const int e = tid + u * BT;
                    if (e < q * q) Tm[(e % q) + (e / q) * QMAX] = t[u];
                }
            }
            // FP64 Cholesky of M (warp 0, row per lane)
            if (tid < 32) {
                const int lane = tid;
                for (int j = 0; j < q; ++j) {
                    const double dj = Md[j + j * QMAX];
                    if (!(dj > 0.0) || !isfinite(dj)) {
                        if (lane == 0) s_fail = 1;
                        break;
                    }
                    const double sd = sqrt(dj);
                    __syncwarp();
                    if (lane == j) Md[j + j * QMAX] = sd;
                    if (lane > j && lane < q) Md[lane + j * QMAX] /= sd;
                    __syncwarp();
                    if (lane > j && lane < q) {
                        const double lij = Md[lane + j * QMAX];
                        for (int c = j + 1; c <= lane; ++c) Md[lane + c * QMAX] -= lij * Md[c + j * QMAX];
                    }
                    __syncwarp();
                }
            }
            __syncthreads();
            if (s_fail) {
                if (tid == 0) atomicOr(&d.status[p], ST_NOTSPD);
                __syncthreads();
                break;
            }
            // C^-1 (FP32, column per lane of warp 0)
            if (tid < 32) {
                const int c = tid;
                for (int i = 0; i < QMAX; ++i) Ci[i + c * QMAX] = 0.f;
                if (c < q) {
                    Ci[c + c * QMAX] = (float)(1.0 / Md[c + c * QMAX]);
                    for (int i = c + 1; i < q; ++i) {
                        double t = 0.0;
                        for (int k = c; k < i; ++k) t += Md[i + k * QMAX] * (double)Ci[k + c * QMAX];
                        Ci[i + c * QMAX] = (float)(-t / Md[i + i * QMAX]);
                    }
                }
            }
            __syncthreads();
            // Lam = C^-T C^-1
            for (int e = tid; e < q * q; e += BT) {
                const int a = e % q, b = e / q;
                float t = 0.f;
                for (int k = max(a, b); k < q; ++k) t = fmaf(Ci[k + a * QMAX], Ci[k + b * QMAX], t);
                Lam[a + b * QMAX] = t;
            }
            __syncthreads();
            // B1 = (Lam + Lam T Lam) / 2: first Tm <- T Lam (in place via registers), then Lam (T Lam)
            float tl[(QMAX * QMAX + BT - 1) / BT];
            int ne = 0;
            for (int e = tid; e < q * q; e += BT, ++ne) {
                const int a = e % q, b = e / q;
                float t = 0.f;
                for (int k = 0; k < q; ++k) t = fmaf(0.5f * (Tm[a + k * QMAX] + Tm[k + a * QMAX]), Lam[k + b * QMAX], t);
                tl[ne] = t;
            }
            __syncthreads();
            ne = 0;
            for (int e = tid; e < q * q; e += BT, ++ne) Tm[(e % q) + (e / q) * QMAX] = tl[ne];
            __syncthreads();
            for (int e = tid; e < q * q; e += BT) {
                const int a = e % q, b = e / q;
                float t = 0.f;
                for (int k = 0; k < q; ++k) t = fmaf(Lam[a + k * QMAX], Tm[k + b * QMAX], t);
                B1[a + b * QMAX] = 0.5f * (Lam[a + b * QMAX] + t);
            }
            __syncthreads();
            // W = -Y Lam + S B1, in place of Y (row-wise)
#pragma unroll
            for (int r = 0; r < RPT; ++r) {
                const int i = tid + BT * r;
                if (i >= n) break;
                float y[QMAX];
#pragma unroll
                for (int c = 0; c < QMAX; ++c) y[c] = (c < q) ? Ys[i + c * ldy] : 0.f;
                const int ri = i - first;
#pragma unroll 4
                for (int c = 0; c < q; ++c) {
                    float w = 0.f;
#pragma unroll
                    for (int b = 0; b < QMAX; ++b) w = fmaf(y[b], (b < q) ? Lam[b + c * QMAX] : 0.f, w);
                    w = -w;
                    if (ri >= 0 && ri < size) w += B1[ri + c * QMAX];
                    Ys[i + c * ldy] = w;
                }
            }
            __syncthreads();
            // X update: columns C (all rows) and rows C (columns outside C)
#pragma unroll
            for (int r = 0; r < RPT; ++r) {
                const int i = tid + BT * r;
                if (i >= n) break;
                const int ri = i - first;
                for (int c = 0; c < size; ++c) {
                    float dlt = Ys[i + c * ldy];
                    if (ri >= 0 && ri < size) dlt += Ys[(first + c) + ri * ldy];
                    X[i + (int64_t)(first + c) * n] += dlt;
                }
                if (ri < 0 || ri >= size)
                    for (int c = 0; c < size; ++c) X[(first + c) + (int64_t)i * n] += Ys[i + c * ldy];
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
    const int n = d.n[p];
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
            for (int k = 0; k < n; ++k) z = fmaf(X[i + (int64_t)k * n], A[k + (int64_t)j * n], z);
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
    const int n = d.n[p];
    float *X = d.X + d.off[p];
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < (int64_t)n * n;
         e += (int64_t)gridDim.x * blockDim.x)
        X[e] = ((e % n) == (e / n)) ? 1.f : 0.f;
}

constexpr size_t batch_smem()
{
    return sizeof(float) * ((NMAX + 1) * QMAX + 32 * QMAX) + sizeof(double) * QMAX * QMAX +
           sizeof(float) * 4 * QMAX * QMAX;
}

}  // namespace

struct rb_batch {
    int count = 0;
    cudaStream_t st = nullptr;
    std::vector<int> n, q, nb, order;
    std::vector<int64_t> off, offP;
    float *A = nullptr, *X = nullptr;
    uint64_t *P = nullptr, *k = nullptr, *stream = nullptr;
    int64_t *d_off = nullptr, *d_offP = nullptr;
    int *d_n = nullptr, *d_q = nullptr, *d_nb = nullptr, *d_order = nullptr, *d_active = nullptr,
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
        d.P = P;
        d.offP = d_offP;
        d.nb = d_nb;
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
    void *ptrs[] = {b->A, b->X, b->P, b->k, b->stream, b->d_off, b->d_offP, b->d_n, b->d_q, b->d_nb,
                    b->d_order, b->d_active, b->d_status, b->d_queue, b->d_resid};
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
        k_batch_rbfgs<512><<<b->grid, 512, batch_smem(), st>>>(b->dev(), steps);
    else
        k_batch_rbfgs<256><<<b->grid, 256, batch_smem(), st>>>(b->dev(), steps);
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
    b->nb.resize(count);
    int64_t tot = 0, totP = 0;
    for (int i = 0; i < count; ++i) {
        b->off[i] = tot;
        tot += (int64_t)n[i] * n[i];
        b->nb[i] = (n[i] + q[i] - 1) / q[i];
        b->offP[i] = totP;
        totP += b->nb[i] + 1;
    }
    b->order.resize(count);
    std::iota(b->order.begin(), b->order.end(), 0);
    std::stable_sort(b->order.begin(), b->order.end(), [&](int x, int y) { return n[x] > n[y]; });
    bool ok = dalloc(&b->A, sizeof(float) * tot) && dalloc(&b->X, sizeof(float) * tot) &&
              dalloc(&b->P, sizeof(uint64_t) * totP) && dalloc(&b->k, sizeof(uint64_t) * count) &&
              dalloc(&b->stream, sizeof(uint64_t) * count) && dalloc(&b->d_off, sizeof(int64_t) * count) &&
              dalloc(&b->d_offP, sizeof(int64_t) * count) && dalloc(&b->d_n, sizeof(int) * count) &&
              dalloc(&b->d_q, sizeof(int) * count) && dalloc(&b->d_nb, sizeof(int) * count) &&
              dalloc(&b->d_order, sizeof(int) * count) && dalloc(&b->d_active, sizeof(int) * count) &&
              dalloc(&b->d_status, sizeof(int) * count) && dalloc(&b->d_queue, sizeof(int)) &&
              dalloc(&b->d_resid, sizeof(double) * count) &&
              cudaMallocHost(&b->h_active, sizeof(int) * count) == cudaSuccess &&
              cudaMallocHost(&b->h_resid, sizeof(double) * count) == cudaSuccess &&
              cudaMallocHost(&b->h_status, sizeof(int) * count) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        batch_free(b);
        return RB_ENOMEM;
    }
    cudaStream_t st = b->st;
    // pack A (FP32) and compute the trace weights of every problem's blocks
    std::vector<uint64_t> hP(totP);
    std::vector<double> diag;
    for (int i = 0; i < count; ++i) {
        if (a_is_fp64)
            launch_copy2d<double, float>(st, n[i], n[i], (const double *)A_dev[i], lda[i], b->A + b->off[i], n[i], 1.0);
        else
            launch_copy2d<float, float>(st, n[i], n[i], (const float *)A_dev[i], lda[i], b->A + b->off[i], n[i], 1.0);
    }
    // diagonals of the packed FP32 A (the values the kernels use)
    std::vector<float> hd;
    for (int i = 0; i < count; ++i) {
        hd.resize(n[i]);
        if (cudaMemcpy2DAsync(hd.data(), sizeof(float), b->A + b->off[i], sizeof(float) * (n[i] + 1), sizeof(float),
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
              cudaMemcpyAsync(b->d_n, n, sizeof(int) * count, cudaMemcpyHostToDevice, st) == cudaSuccess &&
              cudaMemcpyAsync(b->d_q, q, sizeof(int) * count, cudaMemcpyHostToDevice, st) == cudaSuccess &&
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
        cp = cudaStreamSynchronize(st) == cudaSuccess;
    }
    if (!cp) {
        batch_free(b);
        return RB_ECUDA;
    }
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(k_batch_rbfgs<256>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)batch_smem());
        cudaFuncSetAttribute(k_batch_rbfgs<512>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)batch_smem());
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
    launch_copy2d<float, float>(b->st, b->n[i], b->n[i], b->X + b->off[i], b->n[i], (float *)out_dev, ld, 1.0);
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
