// api.cu -- the C ABI of include/rbfgs.h: handles, step drivers, residual
// monitor and solve loop.  Every arithmetic step runs in the kernels of this
// library; the host only sequences launches and reads back scalars.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include <cuda_bf16.h>

#include "kernels.cuh"
#include "tc.cuh"

struct rb_ctx {
    int method = 0, sketch = 0, prec = 0, core_fp64 = 0;
    int c_core64 = 0;  // the C core (S^T A S) in FP64 even when core_fp64 is 0 (the tensor forms' default)
    int n = 0, q = 0;
    bool f64 = false;
    uint64_t seed = 0, stream_id = 0, k = 0;
    cudaStream_t st = nullptr;
    size_t esz = 4;

    void *A = nullptr;  // own copy of A, ld n
    void *X = nullptr;  // iterate: X (RBFGS/NS/MR) or L (AdaRBFGS), ld n
    void *X2 = nullptr, *X3 = nullptr;  // n x n scratch (NS/MR/exact residual)

    // n x q panels (ld n) and q x n panels (ld q)
    void *St = nullptr, *S = nullptr, *G = nullptr, *Y = nullptr, *Sh = nullptr;
    void *W = nullptr, *V = nullptr;  // W and Stb share St's allocation (see alloc_sketch_workspace)
    void *Stb = nullptr;              // second sketch buffer: step k uses St (k even) or Stb (k odd)
    bool s_valid = false;             // S holds L_k S~_k from the previous fused update
    float *Spart = nullptr;           // partial S blocks of the fused update
    size_t spart_cap = 0;
    float *Slo = nullptr, *Glo = nullptr;  // lo parts (x - hi(x)) of S and G for the 3-term products
    bool slo_valid = false;                // Slo belongs to the S in place
    bool sbf_valid = false;                // Sbf holds the BF16 parts of the S in place
    float *Bv = nullptr, *Bs = nullptr;  // tensor-core V and S^: [D^-T; -C^-T] (2q x q) and C^-T (q x q)
    float *Bvlo = nullptr;               // lo part of Bv, split by the streams that write each half
    float *Mf = nullptr, *Nf = nullptr;  // FP32 Gram products S^T A S and S~^T S~ (tensor-core path)
    void *Sbf = nullptr, *Gbf = nullptr;  // BF16 forms: [hi | lo] BF16 parts of S and G (n x q each, ld ldbf)
    int64_t ldbf = 0;
    tc_plan *tc2 = nullptr;              // plan (own workspace) for the side stream's tensor-core GEMMs
    void *P3 = nullptr;  // RBFGS: [S | W | S], n x 3q; tensor-core RBFGS [S | Y | -], AIP [S | W^T | -]
    float *PQ = nullptr;   // tensor-core RBFGS: the update's row-major panels [S W] and [W S] (n x 2q each);
                           // AIP: S row-major (n x q)
    float *Ylo = nullptr;  // tensor-core RBFGS: Y's lo part
    void *Cinv = nullptr, *Dinv = nullptr, *Lam = nullptr, *B1 = nullptr;  // q x q
    double *part = nullptr, *M = nullptr, *N = nullptr, *Tm = nullptr;
    double *dots = nullptr, *dpart = nullptr;
    double *pv = nullptr, *pw = nullptr, *sigma = nullptr;
    int *d_status = nullptr;
    int *blk = nullptr, *idx = nullptr;
    uint64_t *P = nullptr;
    int nb = 0;
    double host_sigma = 0.0;

    // residual workspace (grown on demand)
    int *J = nullptr;
    int rcap = 0;
    void *R1 = nullptr, *R2 = nullptr, *R3 = nullptr;
    double *rpart = nullptr, *rsum = nullptr;

    tc_plan *tc = nullptr;  // tensor-core plan (FP32 storage, TF32 modes)

    // Tensor-core step: the n x n passes run on a high-priority internal stream
    // st1 and the q x q work on a low-priority side stream st2 (fork/join by
    // events, joined back into the handle's stream at the end of each step).
    cudaStream_t st1 = nullptr, st2 = nullptr;
    cudaEvent_t ev_sk = nullptr, ev_g = nullptr, ev_core = nullptr, ev_in = nullptr, ev_out = nullptr;
    // the D chain (S~^T S~ and its core) on a low-priority stream of its own, with its own
    // tensor-core plan, so the C chain after G never queues behind it
    cudaStream_t st3 = nullptr;
    cudaEvent_t ev_d = nullptr, ev_v = nullptr;
    tc_plan *tc3 = nullptr;
    // fused steps: the next step's D^-T (its sketch does not depend on the iterate) is formed
    // during this step's update; d_ready says it is in Bv for the step about to run
    bool d_ready = false;

    // asynchronous residual check (rbfgs_residual_start / _poll)
    int *h_J = nullptr;           // pinned column sample
    int h_J_cap = 0;
    double *h_rsum = nullptr;     // pinned sum of squares
    int *h_status = nullptr;      // pinned copy of the status word
    cudaEvent_t ev_res = nullptr;
    int res_m = 0, res_pending = 0;

    // phase profiling (rbfgs_profile_step): events recorded between phases on the handle's
    // stream, and side-stream marks (time from the step start)
    int prof_on = 0, prof_n = 0, prof_ns = 0;
    cudaEvent_t prof_ev[24], prof_side_ev[8];
    const char *prof_name[24], *prof_side_name[8];
};

std::atomic<unsigned long long> g_rb_launches{0};

// Phase boundary: when profiling, record an event on the handle's stream
// closing the phase that just ended.
static inline void mark(rb_ctx *h, const char *ended)
{
    if (!h->prof_on || h->prof_n >= 23) return;
    h->prof_name[h->prof_n] = ended;
    cudaEventRecord(h->prof_ev[++h->prof_n], h->st);
}

// Side-stream mark: when profiling, record an event on stream s at the end of the named work.
static inline void mark_side(rb_ctx *h, cudaStream_t s, const char *name)
{
    if (!h->prof_on || h->prof_ns >= 8) return;
    h->prof_side_name[h->prof_ns] = name;
    cudaEventRecord(h->prof_side_ev[h->prof_ns++], s);
}

static void rb_free(void *&p)
{
    if (p) cudaFree(p);
    p = nullptr;
}
template <typename T>
static void rb_freet(T *&p)
{
    if (p) cudaFree(p);
    p = nullptr;
}

template <typename P>
static rb_status rb_alloc(P **p, size_t bytes)
{
    if (bytes == 0) bytes = 16;
    if (cudaMalloc((void **)p, bytes) != cudaSuccess) {
        *p = nullptr;
        cudaGetLastError();
        return RB_ENOMEM;
    }
    return RB_OK;
}

extern "C" void rbfgs_default_opts(rb_opts *o)
{
    if (!o) return;
    memset(o, 0, sizeof(*o));
    o->method = RB_METHOD_RBFGS;
    o->sketch = RB_SKETCH_GAUSS;
    o->q = 8;
    o->prec = RB_FP64;
}

extern "C" const char *rbfgs_status_string(int s)
{
    switch (s) {
    case RB_OK: return "ok";
    case RB_NOTCONV: return "not converged within max_iter";
    case RB_EINVAL: return "invalid argument";
    case RB_ENOMEM: return "device allocation failed";
    case RB_ECUDA: return "CUDA runtime error";
    case RB_ENOTSPD: return "Cholesky breakdown: A not SPD or sketch rank deficient";
    case RB_ENONFINITE: return "non-finite value";
    case RB_ETIMEOUT: return "device wait timed out";
    case RB_EUNSUPPORTED: return "unsupported combination";
    default: return "unknown status";
    }
}

static void destroy_ctx(rb_ctx *h)
{
    if (!h) return;
    h->W = nullptr;  // parts of St's allocation
    h->Stb = nullptr;
    void **bufs[] = {&h->A, &h->X, &h->X2, &h->X3, &h->St, &h->S, &h->G, &h->Y, &h->Sh,
                     &h->V, &h->P3, &h->Cinv, &h->Dinv, &h->Lam, &h->B1, &h->R1, &h->R2, &h->R3};
    for (void **b : bufs) rb_free(*b);
    rb_freet(h->Bv);
    rb_freet(h->Bvlo);
    rb_freet(h->Bs);
    rb_freet(h->Spart);
    rb_freet(h->Slo);
    rb_freet(h->Glo);
    rb_freet(h->PQ);
    rb_freet(h->Ylo);
    rb_freet(h->Mf);
    rb_freet(h->Nf);
    rb_free(h->Sbf);
    rb_free(h->Gbf);
    if (h->tc2) tc_plan_destroy(h->tc2);
    h->tc2 = nullptr;
    rb_freet(h->part);
    rb_freet(h->M);
    rb_freet(h->N);
    rb_freet(h->Tm);
    rb_freet(h->dots);
    rb_freet(h->dpart);
    rb_freet(h->pv);
    rb_freet(h->pw);
    rb_freet(h->sigma);
    rb_freet(h->d_status);
    rb_freet(h->blk);
    rb_freet(h->idx);
    rb_freet(h->P);
    rb_freet(h->J);
    rb_freet(h->rpart);
    rb_freet(h->rsum);
    tc_plan_destroy(h->tc);
    if (h->h_J) cudaFreeHost(h->h_J);
    if (h->h_rsum) cudaFreeHost(h->h_rsum);
    if (h->h_status) cudaFreeHost(h->h_status);
    if (h->ev_res) cudaEventDestroy(h->ev_res);
    if (h->ev_sk) cudaEventDestroy(h->ev_sk);
    if (h->ev_g) cudaEventDestroy(h->ev_g);
    if (h->ev_core) cudaEventDestroy(h->ev_core);
    if (h->ev_in) cudaEventDestroy(h->ev_in);
    if (h->ev_out) cudaEventDestroy(h->ev_out);
    if (h->st1) cudaStreamDestroy(h->st1);
    if (h->st2) cudaStreamDestroy(h->st2);
    if (h->st3) cudaStreamDestroy(h->st3);
    if (h->ev_d) cudaEventDestroy(h->ev_d);
    if (h->ev_v) cudaEventDestroy(h->ev_v);
    if (h->tc3) tc_plan_destroy(h->tc3);
    delete h;
}

static rb_status status_from_device(rb_ctx *h)
{
    int s = 0;
    RB_CUDA(cudaMemcpyAsync(&s, h->d_status, sizeof(int), cudaMemcpyDeviceToHost, h->st));
    RB_CUDA(cudaStreamSynchronize(h->st));
    if (s & ST_NOTSPD) return RB_ENOTSPD;
    if (s & ST_NONFINITE) return RB_ENONFINITE;
    if (s & ST_TIMEOUT) return RB_ETIMEOUT;
    return RB_OK;
}

// Copy the caller's A into the handle's storage type (ld n).
static rb_status copy_in_A(rb_ctx *h, const void *A, int64_t lda, int a_is_fp64)
{
    const int n = h->n;
    RB_TRY(rb_alloc(&h->A, h->esz * (size_t)n * n));
    if (h->f64) {
        if (a_is_fp64)
            launch_copy2d<double, double>(h->st, n, n, (const double *)A, lda, (double *)h->A, n, 1.0);
        else
            launch_copy2d<float, double>(h->st, n, n, (const float *)A, lda, (double *)h->A, n, 1.0);
    } else {
        if (a_is_fp64)
            launch_copy2d<double, float>(h->st, n, n, (const double *)A, lda, (float *)h->A, n, 1.0);
        else
            launch_copy2d<float, float>(h->st, n, n, (const float *)A, lda, (float *)h->A, n, 1.0);
    }
    RB_CUDA(cudaGetLastError());
    return RB_OK;
}

// Trace weights of the contiguous coordinate blocks (exact integers, computed
// on the host in the order s_b = sum_{i in C_b} A_ii ascending i, T = sum_b s_b
// ascending b, w_b = max(1, floor(2^52 s_b / T)), prefix sums P).
static rb_status build_trace_weights(rb_ctx *h)
{
    const int n = h->n, q = h->q;
    double *dd = nullptr;
    RB_TRY(rb_alloc(&dd, sizeof(double) * n));
    if (h->f64)
        launch_diag<double>(h->st, n, (const double *)h->A, n, dd);
    else
        launch_diag<float>(h->st, n, (const float *)h->A, n, dd);
    std::vector<double> d(n);
    cudaError_t e1 = cudaMemcpyAsync(d.data(), dd, sizeof(double) * n, cudaMemcpyDeviceToHost, h->st);
    cudaError_t e2 = cudaStreamSynchronize(h->st);
    cudaFree(dd);
    if (e1 != cudaSuccess || e2 != cudaSuccess) return RB_ECUDA;
    const int nb = (n + q - 1) / q;
    std::vector<double> s(nb);
    double T = 0.0;
    for (int b = 0; b < nb; ++b) {
        double acc = 0.0;
        for (int i = b * q; i < n && i < (b + 1) * q; ++i) acc += d[i];
        s[b] = acc;
    }
    for (int b = 0; b < nb; ++b) T += s[b];
    if (!(T > 0.0)) return RB_ENOTSPD;
    std::vector<uint64_t> P(nb + 1, 0);
    for (int b = 0; b < nb; ++b) {
        if (!(s[b] > 0.0)) return RB_ENOTSPD;
        uint64_t w = (uint64_t)floor(ldexp(s[b] / T, 52));
        if (w == 0) w = 1;
        P[b + 1] = P[b] + w;
    }
    RB_TRY(rb_alloc(&h->P, sizeof(uint64_t) * (nb + 1)));
    RB_CUDA(cudaMemcpyAsync(h->P, P.data(), sizeof(uint64_t) * (nb + 1), cudaMemcpyHostToDevice, h->st));
    RB_CUDA(cudaStreamSynchronize(h->st));
    h->nb = nb;
    return RB_OK;
}

static rb_status alloc_common(rb_ctx *h)
{
    RB_TRY(rb_alloc(&h->d_status, sizeof(int)));
    RB_CUDA(cudaMemsetAsync(h->d_status, 0, sizeof(int), h->st));
    RB_TRY(rb_alloc(&h->rsum, sizeof(double) * 2));
    RB_TRY(rb_alloc(&h->dots, sizeof(double) * 2));
    RB_TRY(rb_alloc(&h->dpart, sizeof(double) * 2 * 512));
    return RB_OK;
}

// methods that iterate on X with the RBFGS sketches (Gaussian or trace-weighted blocks)
static bool x_sketch_method(int m) { return m == RB_METHOD_RBFGS || m == RB_METHOD_AIP; }

static rb_status alloc_sketch_workspace(rb_ctx *h)
{
    const size_t n = h->n, q = h->q, e = h->esz;
    const size_t nq = n * q * e, qq = q * q * e;
    const int nch = ceil_div(h->n, GRAM_CHUNK);
    // [S~_a | W^T | S~_b] side by side: [S~_a | W^T] or [W^T | S~_b] is the n x 2q
    // M-contiguous operand of V^T, whichever sketch buffer the step uses
    RB_TRY(rb_alloc(&h->St, 3 * nq));
    h->W = (char *)h->St + nq;
    h->Stb = (char *)h->St + 2 * nq;
    RB_TRY(rb_alloc(&h->S, nq));
    RB_TRY(rb_alloc(&h->G, nq));
    RB_TRY(rb_alloc(&h->Y, nq));
    RB_TRY(rb_alloc(&h->Sh, nq));
    if (!h->f64) {
        RB_TRY(rb_alloc(&h->Bv, 2 * q * q * sizeof(float)));
        RB_TRY(rb_alloc(&h->Bvlo, 2 * q * q * sizeof(float)));
        RB_TRY(rb_alloc(&h->Bs, q * q * sizeof(float)));
        RB_TRY(rb_alloc(&h->Mf, q * q * sizeof(float)));
        RB_TRY(rb_alloc(&h->Nf, q * q * sizeof(float)));
        if (h->method == RB_METHOD_ADARBFGS && q <= 128) {
            h->spart_cap = tc_update_s_workspace(h->n, (int)q);
            RB_TRY(rb_alloc(&h->Spart, h->spart_cap * sizeof(float)));
            // the fused kernel's arrival counts live at the head of this workspace and must start at zero
            RB_CUDA(cudaMemsetAsync(h->Spart, 0, h->spart_cap * sizeof(float), h->st));
            RB_TRY(rb_alloc(&h->Slo, nq));
            RB_TRY(rb_alloc(&h->Glo, nq));
        }
        if (h->prec == RB_BF16 || h->prec == RB_BF16X3) {
            h->ldbf = (h->n + 7) & ~(int64_t)7;  // 16-byte rows for TMA
            const size_t half = (size_t)h->ldbf * q * 2;  // bytes of one BF16 n x q panel
            RB_TRY(rb_alloc(&h->Sbf, 2 * half));
            RB_TRY(rb_alloc(&h->Gbf, 2 * half));
        }
    }
    RB_TRY(rb_alloc(&h->V, nq));
    RB_TRY(rb_alloc(&h->Cinv, qq));
    RB_TRY(rb_alloc(&h->Dinv, qq));
    RB_TRY(rb_alloc(&h->Lam, qq));
    RB_TRY(rb_alloc(&h->B1, qq));
    // FP64 Gram partials (one q x q block per chunk of rows); also the RBFGS / AIP packed core's scratch (3 q x q)
    RB_TRY(rb_alloc(&h->part, sizeof(double) * q * q * std::max(nch, 3)));
    RB_TRY(rb_alloc(&h->M, sizeof(double) * q * q));
    RB_TRY(rb_alloc(&h->N, sizeof(double) * q * q));
    RB_TRY(rb_alloc(&h->Tm, sizeof(double) * q * q));
    RB_TRY(rb_alloc(&h->blk, sizeof(int) * 2));
    RB_TRY(rb_alloc(&h->idx, sizeof(int) * q));
    if (x_sketch_method(h->method)) RB_TRY(rb_alloc(&h->P3, 3 * nq));
    if (x_sketch_method(h->method) && !h->f64 && h->prec != RB_FP32) {  // tensor-core RBFGS / AIP
        RB_TRY(rb_alloc(&h->PQ, 4 * n * q * sizeof(float)));
        RB_TRY(rb_alloc(&h->Glo, nq));
        RB_TRY(rb_alloc(&h->Ylo, nq));
    }
    return RB_OK;
}

static bool prec_ok(int prec) { return prec >= RB_FP64 && prec <= RB_BF16X3; }
static bool prec_bf16(int prec) { return prec == RB_BF16 || prec == RB_BF16X3; }

// Default precision of the AdaRBFGS q x q core for each storage/product form.
static int default_core_fp64(int prec) { return prec == RB_FP64 ? 1 : 0; }

extern "C" rb_status rbfgs_init(rbfgs_t *out, int n, const void *A_dev, int64_t lda, int a_is_fp64,
                                const rb_opts *opts, void *stream)
{
    if (!out || !A_dev || !opts || n < 1 || lda < n) return RB_EINVAL;
    *out = nullptr;
    const int method = opts->method, sketch = opts->sketch, q = opts->q, prec = opts->prec;
    if (!x_sketch_method(method) && method != RB_METHOD_ADARBFGS) return RB_EINVAL;
    if (!prec_ok(prec)) return RB_EINVAL;
    if (q < 1 || q > n || q > 128) return RB_EINVAL;
    if (x_sketch_method(method) && q > 64) return RB_EUNSUPPORTED;  // the RBFGS core holds 3 q x q in smem
    if (x_sketch_method(method) && sketch != RB_SKETCH_GAUSS && sketch != RB_SKETCH_COORD_TRACE)
        return RB_EUNSUPPORTED;
    if (method == RB_METHOD_ADARBFGS && sketch != RB_SKETCH_GAUSS && sketch != RB_SKETCH_COORD_UNIFORM)
        return RB_EUNSUPPORTED;
    if (prec_bf16(prec) && method != RB_METHOD_ADARBFGS) return RB_EUNSUPPORTED;
    rb_ctx *h = new rb_ctx();
    h->method = method;
    h->sketch = sketch;
    h->prec = prec;
    h->n = n;
    h->q = q;
    h->f64 = (prec == RB_FP64);
    h->esz = h->f64 ? 8 : 4;
    h->seed = opts->seed;
    h->stream_id = opts->stream_id;
    // q x q core precision with FP32 storage: FP64 when asked (> 0), FP32 when asked (< 0),
    // else the form's default
    h->core_fp64 = opts->core_fp64 > 0 ? 1 : opts->core_fp64 < 0 ? 0 : default_core_fp64(prec);
    // by default the tensor-core forms factor S^T A S in FP64 (on a CTA cluster, beside W = G^T L)
    // and S~^T S~, a Gaussian Gram with condition number near 1, in FP32
    h->c_core64 = h->core_fp64 || (opts->core_fp64 == 0 && prec != RB_FP32 && prec != RB_FP64);
    h->st = (cudaStream_t)stream;
    rb_status s = RB_OK;
    do {
        if ((s = alloc_common(h)) != RB_OK) break;
        if ((s = copy_in_A(h, A_dev, lda, a_is_fp64)) != RB_OK) break;
        if ((s = rb_alloc(&h->X, h->esz * (size_t)n * n)) != RB_OK) break;
        if (h->f64)
            launch_set_identity<double>(h->st, n, (double *)h->X, n, 1.0);
        else
            launch_set_identity<float>(h->st, n, (float *)h->X, n, 1.0f);
        if ((s = alloc_sketch_workspace(h)) != RB_OK) break;
        if (x_sketch_method(method) && sketch == RB_SKETCH_COORD_TRACE)
            if ((s = build_trace_weights(h)) != RB_OK) break;
        if (!h->f64 && prec != RB_FP32) {
            h->tc = tc_plan_create(n, q, prec);
            if (!h->tc) {
                s = RB_ENOMEM;
                break;
            }
        }
        if (cudaGetLastError() != cudaSuccess) {
            s = RB_ECUDA;
            break;
        }
    } while (0);
    if (s != RB_OK) {
        destroy_ctx(h);
        return s;
    }
    *out = h;
    return RB_OK;
}

// ---------------------------------------------------------------------------
// One RBFGS step (Algorithm 3 with W = A^-1, Eq. (qunac) in its expanded
// rank-2q form).
// ---------------------------------------------------------------------------
template <typename T>
static void rbfgs_step_gauss(rb_ctx *h)
{
    const int n = h->n, q = h->q;
    cudaStream_t st = h->st;
    const int *stp = h->d_status;
    T *A = (T *)h->A, *X = (T *)h->X;
    T *S = (T *)h->P3, *Wp = S + (size_t)n * q, *S2 = S + 2 * (size_t)n * q;
    T *G = (T *)h->G, *Y = (T *)h->Y;
    launch_gauss_sketch<T>(st, n, q, h->seed, h->stream_id, h->k, S, n);
    launch_copy2d<T, T>(st, n, q, S, n, S2, n, 1.0);
    mark(h, "sketch");
    gemm_simt<T>(st, false, false, n, q, n, T(1), A, n, S, n, T(0), G, n, stp);   // G = A S
    mark(h, "G=AS");
    launch_gram<T>(st, n, q, q, S, n, G, n, h->part, h->M);                        // M = S^T A S
    mark(h, "gram S^TAS");
    gemm_simt<T>(st, false, false, n, q, n, T(1), X, n, G, n, T(0), Y, n, stp);   // Y = X G
    mark(h, "Y=XG");
    launch_gram<T>(st, n, q, q, G, n, Y, n, h->part, h->Tm);                       // T = G^T X G
    launch_core_rbfgs<T>(st, q, h->M, h->Tm, (T *)h->Lam, (T *)h->B1, h->d_status);
    mark(h, "gram T + core");
    gemm_simt<T>(st, false, false, n, q, q, T(1), S, n, (T *)h->B1, q, T(0), Wp, n, stp);  // W = S B1
    gemm_simt<T>(st, false, false, n, q, q, T(-1), Y, n, (T *)h->Lam, q, T(1), Wp, n, stp); //   - Y Lam
    mark(h, "W");
    gemm_simt<T>(st, false, true, n, n, 2 * q, T(1), S, n, Wp, n, T(1), X, n, stp);         // X += [S W][W S]^T
    mark(h, "update X");
}

template <typename T>
static void rbfgs_step_coord(rb_ctx *h)
{
    const int n = h->n, q = h->q;
    cudaStream_t st = h->st;
    const int *stp = h->d_status;
    T *A = (T *)h->A, *X = (T *)h->X, *G = (T *)h->G, *Y = (T *)h->Y, *W = (T *)h->W;
    launch_coord_trace_draw(st, n, q, h->nb, h->P, h->seed, h->stream_id, h->k, h->blk);
    launch_coord_gather<T>(st, n, q, A, n, h->blk, G, n, h->M, stp);               // G = A[:, C], M = A[C, C]
    mark(h, "draw + gather");
    bool ytc = false;  // Y = X G, the one pass over X: on the tensor cores in the FP32-storage tensor forms
    if constexpr (sizeof(T) == 4)
        if (h->tc && h->prec != RB_FP32)
            ytc = tc_gemm_nk(h->tc, st, h->prec == RB_TF32 ? 1 : 3, TC_A_K, n, q, n, X, n, G, n, Y, n, stp) >= 0;
    if (!ytc) gemm_simt<T>(st, false, false, n, q, n, T(1), X, n, G, n, T(0), Y, n, stp);  // Y = X G
    mark(h, "Y=XG");
    launch_gram<T>(st, n, q, q, G, n, Y, n, h->part, h->Tm);                       // T = G^T X G
    launch_core_rbfgs<T>(st, q, h->M, h->Tm, (T *)h->Lam, (T *)h->B1, h->d_status);
    mark(h, "gram T + core");
    gemm_simt<T>(st, false, false, n, q, q, T(-1), Y, n, (T *)h->Lam, q, T(0), W, n, stp);  // W = -Y Lam
    launch_coord_add_b1<T>(st, q, h->blk, (const T *)h->B1, W, n, stp);                     //   + S B1
    launch_coord_update<T>(st, n, q, h->blk, W, n, X, n, stp);                               // rows/cols C
    mark(h, "update rows/cols");
}

// ---------------------------------------------------------------------------
// Tensor-core RBFGS and AIP steps (FP32 storage; Gaussian sketch, exact in TF32).
// ---------------------------------------------------------------------------
// CTAs of a q x q Gram product when it runs split over K
constexpr int GRAM_CTAS = 64;

// q x q Gram product X1^T X2 (K = n) into out (ld q): split over K on the tensor cores
// (3 terms with X2's lo part, else 1), any other shape by the general product.
static void tc_gram(rb_ctx *h, int terms, const float *X1, const float *X2, const float *X2lo, float *out)
{
    const int n = h->n, q = h->q;
    if (tc_gemm_splitk(h->tc, h->st, terms, TC_A_K, q, q, n, X1, n, X2, terms == 3 ? X2lo : nullptr, n, out, q,
                       h->d_status, GRAM_CTAS) != 0)
        tc_gemm_nk(h->tc, h->st, terms, TC_A_K, q, q, n, X1, n, X2, n, out, q, h->d_status);
}

// shapes the tensor-core RBFGS / AIP steps take: 16-byte rows of X and of the 2q-wide panels
static bool x_tc_shape(rb_ctx *h)
{
    return !h->f64 && h->tc && h->PQ && h->n % 4 == 0 && h->q % 4 == 0 && h->q <= 64;
}

// RBFGS, Eq. (qunac) in its expanded form:
//   G = A S, M = S^T G, Y = X G, T = G^T Y, [B1; -Lam] from the core,
//   W = [S | Y] [B1; -Lam] = S B1 - Y Lam,  X += S W^T + W S^T.
// The rank-2q update is one pass over X: X += P Q^T with the row-major panels P = [S W]
// and Q = [W S] (W written into both, transposed, by its product's epilogue).
static void rbfgs_step_tc(rb_ctx *h)
{
    const int n = h->n, q = h->q;
    cudaStream_t st = h->st;
    const int *stp = h->d_status;
    float *A = (float *)h->A, *X = (float *)h->X, *G = (float *)h->G;
    float *S = (float *)h->P3, *Y = S + (size_t)n * q;  // [S | Y]: W's M-contiguous A operand
    float *P = h->PQ, *Q = h->PQ + 2 * (size_t)n * q;
    const int acc = (h->prec == RB_TF32) ? 1 : 3, upd = (h->prec == RB_TF32X3) ? 3 : 1;
    float *Glo = acc == 3 ? h->Glo : nullptr, *Ylo = acc == 3 ? h->Ylo : nullptr;
    launch_gauss_sketch<float>(st, n, q, h->seed, h->stream_id, h->k, S, n);
    mark(h, "sketch");
    // G = A S: S is exact in TF32, so A's two parts carry the product; G's lo part beside G
    tc_gemm_nk_lo(h->tc, st, acc == 3 ? 2 : 1, TC_A_K, n, q, n, A, n, S, nullptr, n, G, Glo, n, stp);
    mark(h, "G=AS");
    tc_gram(h, acc, S, G, Glo, h->Mf);  // M = S^T A S
    // Y = X G (X symmetric: its columns are its rows), Y's lo part beside Y
    tc_gemm_nk_lo(h->tc, st, acc, TC_A_K, n, q, n, X, n, G, Glo, n, Y, Ylo, n, stp);
    mark(h, "Y=XG");
    tc_gram(h, acc, G, Y, Ylo, h->Nf);  // T = G^T X G
    launch_core_pack(st, q, h->Mf, h->Nf, h->Bv, h->part, h->d_status);
    mark(h, "grams + core");
    // W = [S | Y] [B1; -Lam], transposed into columns q .. 2q-1 of P's rows and 0 .. q-1 of Q's
    tc_gemm_nk_t(h->tc, st, acc, TC_A_MN, n, q, 2 * q, S, n, h->Bv, 2 * q, P + q, 2 * q, stp);
    tc_gemm_nk_t(h->tc, st, acc, TC_A_MN, n, q, 2 * q, S, n, h->Bv, 2 * q, Q, 2 * q, stp);
    launch_rows_from_cols(st, n, q, S, n, P, 2 * q, 0);
    launch_rows_from_cols(st, n, q, S, n, Q, 2 * q, q);
    mark(h, "W");
    // X += [S W][W S]^T: W -> 0 at the fixed point, so the mixed form takes one TF32 pass
    if (upd != 1 || tc_update_persistent(h->tc, st, n, 2 * q, P, Q, X, n, stp) != 0)
        tc_update(h->tc, st, upd, n, 2 * q, P, Q, X, n, stp);
    mark(h, "update X");
}

// AIP, Eq. (BFGSas): G = A S, Lam = (S^T G)^-1, W^T = X^T G,
//   V^T = [S | W^T] [Lam; -Lam] = (S - W^T) Lam,  X += S V  (one pass over X).
static void aip_step_tc(rb_ctx *h)
{
    const int n = h->n, q = h->q;
    cudaStream_t st = h->st;
    const int *stp = h->d_status;
    float *A = (float *)h->A, *X = (float *)h->X, *G = (float *)h->G, *V = (float *)h->V;
    float *S = (float *)h->P3, *Wt = S + (size_t)n * q;  // [S | W^T]: V^T's M-contiguous A operand
    float *Srow = h->PQ;
    const int acc = (h->prec == RB_TF32) ? 1 : 3, upd = (h->prec == RB_TF32X3) ? 3 : 1;
    float *Glo = acc == 3 ? h->Glo : nullptr;
    launch_gauss_sketch<float>(st, n, q, h->seed, h->stream_id, h->k, S, n);
    mark(h, "sketch");
    tc_gemm_nk_lo(h->tc, st, acc == 3 ? 2 : 1, TC_A_K, n, q, n, A, n, S, nullptr, n, G, Glo, n, stp);  // G = A S
    mark(h, "G=AS");
    tc_gram(h, acc, S, G, Glo, h->Mf);
    launch_core_pack(st, q, h->Mf, nullptr, h->Bv, h->part, h->d_status);  // [Lam; -Lam]
    mark(h, "gram + core");
    // W^T = X^T G (element (m, k) of X^T at X[k + m n])
    tc_gemm_nk_lo(h->tc, st, acc, TC_A_K, n, q, n, X, n, G, Glo, n, Wt, nullptr, n, stp);
    mark(h, "W=G^TX");
    tc_gemm_nk_t(h->tc, st, acc, TC_A_MN, n, q, 2 * q, S, n, h->Bv, 2 * q, V, q, stp);  // V (q x n, ld q)
    launch_rows_from_cols(st, n, q, S, n, Srow, q, 0);
    mark(h, "V");
    // X += S V: V -> 0 at the fixed point, so the mixed form takes one TF32 pass
    if (upd != 1 || tc_update_persistent(h->tc, st, n, q, Srow, V, X, n, stp) != 0)
        tc_update(h->tc, st, upd, n, q, Srow, V, X, n, stp);
    mark(h, "update X");
}

extern "C" rb_status rbfgs_step(rbfgs_t h, int nsteps)
{
    if (!h || nsteps < 0 || h->method != RB_METHOD_RBFGS) return RB_EINVAL;
    for (int s = 0; s < nsteps; ++s) {
        if (h->sketch == RB_SKETCH_COORD_TRACE) {
            if (h->f64)
                rbfgs_step_coord<double>(h);
            else
                rbfgs_step_coord<float>(h);
        } else {
            if (h->f64)
                rbfgs_step_gauss<double>(h);
            else if (x_tc_shape(h))
                rbfgs_step_tc(h);
            else
                rbfgs_step_gauss<float>(h);
        }
        ++h->k;
    }
    RB_CUDA(cudaGetLastError());
    return RB_OK;
}

// Approximate inverse preconditioning, Eq. (BFGSas) (Sec. 8; Algorithm 1 with
// W = A^-1): X+ = X + S Lambda (S^T - G^T X), G = A S, Lambda = (S^T G)^-1.
template <typename T>
static void aip_step_gauss(rb_ctx *h)
{
    const int n = h->n, q = h->q;
    cudaStream_t st = h->st;
    const int *stp = h->d_status;
    T *A = (T *)h->A, *X = (T *)h->X, *S = (T *)h->P3, *G = (T *)h->G;
    T *W = (T *)h->Y, *V = (T *)h->V, *Lam = (T *)h->Lam;  // W, V: q x n (ld q)
    launch_gauss_sketch<T>(st, n, q, h->seed, h->stream_id, h->k, S, n);
    mark(h, "sketch");
    gemm_simt<T>(st, false, false, n, q, n, T(1), A, n, S, n, T(0), G, n, stp);   // G = A S
    mark(h, "G=AS");
    launch_gram<T>(st, n, q, q, S, n, G, n, h->part, h->M);                        // M = S^T A S
    launch_core_rbfgs<T>(st, q, h->M, h->M, Lam, (T *)h->B1, h->d_status);        // Lambda = M^-1
    mark(h, "gram + core");
    gemm_simt<T>(st, true, false, q, n, n, T(1), G, n, X, n, T(0), W, q, stp);    // W = G^T X
    mark(h, "W=G^TX");
    gemm_simt<T>(st, false, true, q, n, q, T(1), Lam, q, S, n, T(0), V, q, stp);  // V = Lambda S^T
    gemm_simt<T>(st, false, false, q, n, q, T(-1), Lam, q, W, q, T(1), V, q, stp);  //   - Lambda W
    mark(h, "V");
    gemm_simt<T>(st, false, false, n, n, q, T(1), S, n, V, q, T(1), X, n, stp);   // X += S V
    mark(h, "update X");
}

template <typename T>
static void aip_step_coord(rb_ctx *h)
{
    const int n = h->n, q = h->q;
    cudaStream_t st = h->st;
    const int *stp = h->d_status;
    T *A = (T *)h->A, *X = (T *)h->X, *G = (T *)h->G;
    T *W = (T *)h->Y, *V = (T *)h->V, *Lam = (T *)h->Lam;
    launch_coord_trace_draw(st, n, q, h->nb, h->P, h->seed, h->stream_id, h->k, h->blk);
    launch_coord_gather<T>(st, n, q, A, n, h->blk, G, n, h->M, stp);               // G = A[:, C], M = A[C, C]
    launch_core_rbfgs<T>(st, q, h->M, h->M, Lam, (T *)h->B1, h->d_status);        // Lambda = M^-1 (padded)
    mark(h, "draw + gather + core");
    bool wtc = false;  // W = G^T X, the one pass over X, as W^T = X^T G with a transposed output (q x n, ld q)
    if constexpr (sizeof(T) == 4)
        if (h->tc && h->prec != RB_FP32)
            wtc = tc_gemm_nk_t(h->tc, st, h->prec == RB_TF32 ? 1 : 3, TC_A_K, n, q, n, X, n, G, n, W, q, stp) == 0;
    if (!wtc) gemm_simt<T>(st, true, false, q, n, n, T(1), G, n, X, n, T(0), W, q, stp);  // W = G^T X
    mark(h, "W=G^TX");
    gemm_simt<T>(st, false, false, q, n, q, T(-1), Lam, q, W, q, T(0), V, q, stp); // V = -Lambda W
    launch_aip_coord<T>(st, n, q, h->blk, Lam, V, q, X, n, stp);                  // + Lambda I[C,:]; X[C,:] += V
    mark(h, "update rows");
}

extern "C" rb_status aip_step(rbfgs_t h, int nsteps)
{
    if (!h || nsteps < 0 || h->method != RB_METHOD_AIP) return RB_EINVAL;
    for (int s = 0; s < nsteps; ++s) {
        if (h->sketch == RB_SKETCH_COORD_TRACE) {
            if (h->f64)
                aip_step_coord<double>(h);
            else
                aip_step_coord<float>(h);
        } else {
            if (h->f64)
                aip_step_gauss<double>(h);
            else if (x_tc_shape(h))
                aip_step_tc(h);
            else
                aip_step_gauss<float>(h);
        }
        ++h->k;
    }
    RB_CUDA(cudaGetLastError());
    return RB_OK;
}

// ---------------------------------------------------------------------------
// One AdaRBFGS step (Algorithm 4, Eq. (Cholimprov) with lower Cholesky
// factors: L+ = L + (S C^-T)(D^-1 S~^T - C^-1 (A S)^T L)).
// ---------------------------------------------------------------------------
template <typename T>
static void ada_draw(rb_ctx *h, T *St, uint64_t k, cudaStream_t s = nullptr)
{
    cudaStream_t st = s ? s : h->st;
    if (h->sketch == RB_SKETCH_COORD_UNIFORM) {
        launch_floyd_draw(st, h->n, h->q, h->seed, h->stream_id, k, h->idx);
        launch_coord_matrix<T>(st, h->n, h->q, h->idx, St, h->n);
    } else {
        launch_gauss_sketch<T>(st, h->n, h->q, h->seed, h->stream_id, k, St, h->n);
    }
}

template <typename T>
static void ada_step_simt(rb_ctx *h)
{
    const int n = h->n, q = h->q;
    cudaStream_t st = h->st;
    const int *stp = h->d_status;
    T *A = (T *)h->A, *L = (T *)h->X, *St = (T *)h->St, *S = (T *)h->S, *G = (T *)h->G;
    T *W = (T *)h->W, *V = (T *)h->V, *Sh = (T *)h->Sh, *Ci = (T *)h->Cinv, *Di = (T *)h->Dinv;
    ada_draw<T>(h, St, h->k);
    mark(h, "sketch");
    gemm_simt<T>(st, false, false, n, q, n, T(1), L, n, St, n, T(0), S, n, stp);   // S = L S~
    mark(h, "S=LS~");
    gemm_simt<T>(st, false, false, n, q, n, T(1), A, n, S, n, T(0), G, n, stp);    // G = A S
    mark(h, "G=AS");
    launch_gram<T>(st, n, q, q, S, n, G, n, h->part, h->M);                         // S^T A S
    launch_gram<T>(st, n, q, q, St, n, St, n, h->part, h->N);                       // S~^T S~
    mark(h, "grams");
    if constexpr (sizeof(T) == 4) {
        if (!h->core_fp64)
            launch_core_ada32(st, q, h->M, h->N, Ci, Di, h->d_status);                  // C^-1, D^-1 (FP32)
        else
            launch_core_ada<T>(st, q, h->M, h->N, Ci, Di, h->d_status);
    } else {
        launch_core_ada<T>(st, q, h->M, h->N, Ci, Di, h->d_status);                 // C^-1, D^-1 (FP64)
    }
    mark(h, "q x q core");
    gemm_simt<T>(st, true, false, q, n, n, T(1), G, n, L, n, T(0), W, q, stp);     // W = G^T L
    mark(h, "W=G^TL");
    gemm_simt<T>(st, false, true, q, n, q, T(1), Di, q, St, n, T(0), V, q, stp);   // V = D^-1 S~^T
    gemm_simt<T>(st, false, false, q, n, q, T(-1), Ci, q, W, q, T(1), V, q, stp);  //   - C^-1 W
    gemm_simt<T>(st, false, true, n, q, q, T(1), S, n, Ci, q, T(0), Sh, n, stp);   // S^ = S C^-T
    mark(h, "V, S^");
    gemm_simt<T>(st, false, false, n, n, q, T(1), Sh, n, V, q, T(1), L, n, stp);   // L += S^ V
    mark(h, "update L");
}

static bool ensure_side_stream(rb_ctx *h)
{
    if (h->st1 && h->st2 && h->st3 && h->ev_v) return true;
    int least = 0, greatest = 0;
    cudaDeviceGetStreamPriorityRange(&least, &greatest);
    if (!h->st1 && cudaStreamCreateWithPriority(&h->st1, cudaStreamNonBlocking, greatest) != cudaSuccess) return false;
    if (!h->st2 && cudaStreamCreateWithPriority(&h->st2, cudaStreamNonBlocking, least) != cudaSuccess) return false;
    if (!h->st3 && cudaStreamCreateWithPriority(&h->st3, cudaStreamNonBlocking, least) != cudaSuccess) return false;
    const unsigned fl = cudaEventDisableTiming;
    for (cudaEvent_t *e : {&h->ev_sk, &h->ev_g, &h->ev_core, &h->ev_in, &h->ev_out, &h->ev_d, &h->ev_v})
        if (!*e && cudaEventCreateWithFlags(e, fl) != cudaSuccess) return false;
    return true;
}

// SMs that the stream-K GEMMs leave to the side stream while it runs the
// Gram products and the q x q core: W = L^T G overlaps S^T G (three passes) and
// C^-1 and needs 8 (with 4 the chain outlasted W); G = A S overlaps only the
// one-pass S~^T S~ and D^-1, for which 4 suffice.
constexpr int SIDE_SMS = 8;
constexpr int SIDE_SMS_G = 4;
// SMs the fused update leaves to the next step's D chain (S~^T S~ and its core)
constexpr int SIDE_SMS_UPD = 4;


// V^T = [S~ | W^T] Bv is a 3-term product in the 3-term forms: each stream that writes a half of Bv
// also writes that half's lo part into Bvlo, so that V's launch splits nothing.
static bool bv_split(const rb_ctx *h) { return h->prec != RB_TF32 && h->prec != RB_BF16 && h->Bvlo != nullptr; }

// D chain on the handle's D stream: S~^T S~ (one exact pass: S~ is TF32) on the SMs other
// work leaves free, then its core, D^-T written as rows dofs .. dofs + q - 1 of Bv.
static void ada_d_chain(rb_ctx *h, const float *St, int dofs, int reserve)
{
    const int n = h->n, q = h->q;
    tc_gemm_nk(h->tc3, h->st3, 1, TC_A_K, q, q, n, St, n, St, n, h->Nf, q, h->d_status, reserve);
    if (h->core_fp64)
        launch_core_tr64(h->st3, q, h->Nf, h->Bv + dofs, 2 * q, 1.f, nullptr, 0, 0.f, h->d_status);
    else
        launch_core_tr32(h->st3, q, h->Nf, nullptr, h->Bv + dofs, 2 * q, 1.f, nullptr, 0, 0.f, h->d_status);
    if (bv_split(h)) tc_split_lo(h->st3, q, q, h->Bv + dofs, 2 * q, h->Bvlo + dofs, 2 * q);
    cudaEventRecord(h->ev_d, h->st3);
}

// Tensor-core step.  The q x q work runs on a low-priority side stream while
// the n x n passes run on a high-priority one; the GEMMs that overlap side
// work leave SIDE_SMS SMs free for it.  With the fused update (single-pass
// correction, q <= 128) the step is
//   main:  [S = L S~ once, after init / reset / import]  G = A S -> W^T = L^T G
//          -> [join] -> V, S^ -> draw S~_{k+1} -> L += S^ V and S = L S~_{k+1}
//   side:  S~^T S~, D^-1 (from the step start)   [after G]  S^T G, C^-1
// so every step streams A once and L three times (read for W, read + write).
// Otherwise S = L S~ is its own GEMM at the start of the step.
static void ada_step_tc(rb_ctx *h)
{
    const int n = h->n, q = h->q;
    // the side-stream core writes its inverses straight into the tensor-core B operands, which
    // needs q <= 128 and 16-byte rows; the FP64 core exists only in that form
    const bool tcv_shape = q <= 128 && q % 4 == 0 && n % 4 == 0;
    const bool fork = (!h->core_fp64 || tcv_shape) && ensure_side_stream(h);
    cudaStream_t user = h->st;
    if (fork) {  // run the step on st1 (every helper launches on h->st), joined to the caller's stream
        cudaEventRecord(h->ev_in, user);
        cudaStreamWaitEvent(h->st1, h->ev_in, 0);
        h->st = h->st1;
    }
    cudaStream_t st = h->st;
    const int *stp = h->d_status;
    float *A = (float *)h->A, *L = (float *)h->X, *S = (float *)h->S, *G = (float *)h->G;
    float *W = (float *)h->W, *V = (float *)h->V, *Sh = (float *)h->Sh, *Ci = (float *)h->Cinv,
          *Di = (float *)h->Dinv;
    const int acc = (h->prec == RB_TF32 || h->prec == RB_BF16) ? 1 : 3;  // split terms, accuracy-critical products
    const int upd = (h->prec == RB_TF32X3) ? 3 : 1;
    // BF16 forms: G = A S and W^T = L^T G as BF16-split products (1 or 3 terms)
    const int bfterms = h->prec == RB_BF16X3 ? 3 : h->prec == RB_BF16 ? 1 : 0;
    const size_t bfhalf = (size_t)h->ldbf * q;  // elements of one BF16 panel
    const int side_sms = SIDE_SMS;
    const int rsv = fork ? side_sms : 0;
    cudaStream_t side = fork ? h->st2 : st;
    // V and S^ on the tensor cores: the cores write their inverses transposed
    // straight into the B operands (needs q <= 128 and 16-byte rows)
    bool tcv = fork && tcv_shape;
    if (tcv && !h->tc2) tcv = (h->tc2 = tc_plan_create(n, q, h->prec)) != nullptr;
    if (tcv && !h->tc3) tcv = (h->tc3 = tc_plan_create(n, q, h->prec)) != nullptr;
    // AdaRBFGS_cols: S = L[:, C] is a gather of q columns and S~^T S~ = I (distinct coordinates),
    // so there is no product to fuse into the update and the D chain writes D^-T = I
    const bool cols = h->sketch == RB_SKETCH_COORD_UNIFORM;
    const bool fuse = tcv && upd == 1 && h->Spart && !cols;
    // the next step's D chain runs during this step's fused update
    const bool dpipe = fuse;
    bool core_first = false;  // FP64 C core on a cluster before W (W then runs on the side stream)
    const bool d_now = tcv && !(dpipe && h->d_ready);  // this step's D chain still to run (during G)
    const int rsv_g = (fork && ((d_now && !cols) || !tcv)) ? SIDE_SMS_G : 0;
    // the side stream's Gram products run stream-K on the SIDE_SMS SMs the main GEMMs leave free
    const int side_rsv = std::max(0, tc_num_sms() - side_sms), side_rsv_g = std::max(0, tc_num_sms() - SIDE_SMS_G);
    // sketch buffers: [S~_a | W^T | S~_b]; step k uses S~_a (k even) or S~_b (k odd) when fused
    const bool odd = fuse && (h->k & 1);
    float *St = odd ? (float *)h->Stb : (float *)h->St;
    float *St_next = odd ? (float *)h->St : (float *)h->Stb;
    float *SW = odd ? W : St;          // V^T's A operand: [S~ | W^T] or [W^T | S~]
    const int dofs = odd ? q : 0;      // rows of D^-T in Bv (the -C^-T rows take the other half)
    const int cofs = odd ? 0 : q;
    if (!fuse || !h->s_valid) {
        ada_draw<float>(h, St, h->k);
        mark(h, "sketch");
        h->slo_valid = false;
        h->sbf_valid = false;
        if (fuse) {  // S = L S~ from the fused kernel without the update, so every S comes from one path
            // (the same grid as the fused updates, so S's partial sums are added in the same order)
            const int rc = tc_update_next_s(st, n, q, Sh, V, L, n, St, S, 0, h->Spart, h->spart_cap, stp, h->Slo,
                                            bfterms ? h->Sbf : nullptr, h->ldbf, dpipe ? SIDE_SMS_UPD : 0);
            if (rc != 0) {
                tc_gemm_nk(h->tc, st, acc == 3 ? 2 : acc, TC_A_MN, n, q, n, L, n, St, n, S, n, stp);
            } else {
                h->slo_valid = h->Slo != nullptr;
                h->sbf_valid = bfterms != 0;
            }
        } else if (cols) {
            launch_gather_cols<float>(st, n, q, L, n, h->idx, S, n);  // S = L[:, C] (C ascending, as S~'s columns)
        } else {
            // S = L S~ (A = L, M-contiguous); S~ is exact in TF32, so the split needs only L's two parts
            tc_gemm_nk(h->tc, st, acc == 3 ? 2 : acc, TC_A_MN, n, q, n, L, n, St, n, S, n, stp);
        }
        mark(h, "S=LS~");
    }
    if (fork) {
        cudaEventRecord(h->ev_sk, st);
        if (tcv) {  // S~^T S~ -> D^-T into Bv, on the D chain's own stream (unless the previous step did it)
            if (d_now) {
                cudaStreamWaitEvent(h->st3, h->ev_sk, 0);
                if (cols) {  // D = I
                    launch_set_identity<float>(h->st3, q, h->Bv + dofs, 2 * q, 1.f);
                    if (bv_split(h)) tc_split_lo(h->st3, q, q, h->Bv + dofs, 2 * q, h->Bvlo + dofs, 2 * q);
                    cudaEventRecord(h->ev_d, h->st3);
                } else {
                    ada_d_chain(h, St, dofs, side_rsv_g);
                }
                mark_side(h, h->st3, "@D core done");
            }
        } else {
            cudaStreamWaitEvent(side, h->ev_sk, 0);
            launch_gram<float>(side, n, q, q, St, n, St, n, h->part, h->N);  // S~^T S~ -> D^-1
            launch_core_ada32(side, q, h->N, nullptr, Di, nullptr, h->d_status);
        }
    }
    // G = A S (A symmetric); S's lo part comes from the kernel that formed S, and G's is
    // written beside G for the two products that take G as their B (W and S^T G)
    const bool glo = acc == 3 && h->Glo != nullptr;
    bool gbf = false;
    if (bfterms) {  // S's BF16 parts come from the kernel that formed S (else split here); G's are written beside G
        __nv_bfloat16_raw *sb = (__nv_bfloat16_raw *)h->Sbf;
        if (!h->sbf_valid) tc_split_bf16(st, n, q, S, n, sb, sb + bfhalf, h->ldbf);
        gbf = tc_gemm_bf(h->tc, st, bfterms, n, q, n, A, n, sb, sb + bfhalf, h->ldbf, G, glo ? h->Glo : nullptr, n,
                         stp, rsv_g, h->Gbf, h->ldbf) == 0;
    }
    if (!gbf)
        tc_gemm_nk_lo(h->tc, st, acc, TC_A_K, n, q, n, A, n, S, (acc == 3 && h->slo_valid) ? h->Slo : nullptr, n, G,
                      glo ? h->Glo : nullptr, n, stp, rsv_g);
    mark(h, fork ? "G=AS | D core" : "G=AS");
    if (fork) {
        // S^T G (3 x TF32) on the main stream right after G, split over K on GRAM_CTAS CTAs with the
        // whole GPU free, so that only the C core overlaps W (3-term forms, whose G carries its lo part)
        const bool gram_main = tcv && glo &&
                               tc_gemm_splitk(h->tc, st, 3, TC_A_K, q, q, n, S, n, G, h->Glo, n, h->Mf, q, stp,
                                              GRAM_CTAS) == 0;
        if (gram_main) mark(h, "S^T G");
        cudaEventRecord(h->ev_g, st);
        cudaStreamWaitEvent(side, h->ev_g, 0);
        core_first = tcv && gram_main && h->c_core64;
        if (core_first) {
            // FP64 C core on a cluster of SIDE_SMS CTAs.  A cluster needs all its SMs in one GPC: it
            // is launched in stream order right after S^T G, so it is placed while the GPU is idle,
            // and W = G^T L, on the low-priority side stream behind an event, takes the other SMs.
            launch_core_tr64(st, q, h->Mf, h->Bv + cofs, 2 * q, -1.f, h->Bs, q, 1.f, h->d_status, SIDE_SMS);
            if (bv_split(h)) tc_split_lo(st, q, q, h->Bv + cofs, 2 * q, h->Bvlo + cofs, 2 * q);
            mark_side(h, st, "@C core done");
            bool wbf_s = false;
            if (bfterms) {
                __nv_bfloat16_raw *gb = (__nv_bfloat16_raw *)h->Gbf;
                if (!gbf) tc_split_bf16(side, n, q, G, n, gb, gb + bfhalf, h->ldbf);
                wbf_s = tc_gemm_bf(h->tc, side, bfterms, n, q, n, L, n, gb, gb + bfhalf, h->ldbf, W, nullptr, n, stp,
                                   rsv) == 0;
            }
            if (!wbf_s)
                tc_gemm_nk_lo(h->tc, side, acc, TC_A_K, n, q, n, L, n, G, glo ? h->Glo : nullptr, n, W, nullptr, n,
                              stp, rsv);
            cudaEventRecord(h->ev_core, side);  // W done
            mark_side(h, side, "@W done");
            if (fuse) {  // on the SMs the core frees while W runs: S^ = S C^-T and the next step's sketch
                tc_gemm_nk_t(h->tc2, st, upd, TC_A_MN, n, q, q, S, n, h->Bs, q, Sh, q, stp);
                ada_draw<float>(h, St_next, h->k + 1, st);
            }
        } else if (tcv) {  // S^T A S = S^T G (3 x TF32) -> -C^-T into Bv, C^-T into Bs
            if (!gram_main) {
                tc_gemm_nk_lo(h->tc2, side, 3, TC_A_K, q, q, n, S, n, G, glo ? h->Glo : nullptr, n, h->Mf, nullptr,
                              q, stp, side_rsv);
                mark_side(h, side, "@S^T G done");
            }
            if (h->c_core64)  // C C^T = S^T A S in FP64, spread over a cluster of the SIDE_SMS SMs W leaves free
                launch_core_tr64(side, q, h->Mf, h->Bv + cofs, 2 * q, -1.f, h->Bs, q, 1.f, h->d_status, SIDE_SMS);
            else
                launch_core_tr32(side, q, h->Mf, nullptr, h->Bv + cofs, 2 * q, -1.f, h->Bs, q, 1.f, h->d_status);
            if (bv_split(h)) tc_split_lo(side, q, q, h->Bv + cofs, 2 * q, h->Bvlo + cofs, 2 * q);
        } else {
            launch_gram<float>(side, n, q, q, S, n, G, n, h->part, h->M);    // S^T A S -> C^-1
            launch_core_ada32(side, q, h->M, nullptr, Ci, nullptr, h->d_status);
        }
        if (!core_first) {
            cudaEventRecord(h->ev_core, side);
            mark_side(h, side, "@C core done");
        }
        // off the main stream while it runs W's tail and V: S^ = S C^-T (it needs only S and the C
        // core) and the next step's sketch (its buffer is free: nothing of this step reads it); only
        // the fused update waits for them
        if (fuse && !core_first) {
            tc_gemm_nk_t(h->tc2, side, upd, TC_A_MN, n, q, q, S, n, h->Bs, q, Sh, q, stp);
            ada_draw<float>(h, St_next, h->k + 1, side);
            cudaEventRecord(h->ev_g, side);
        }
    } else {
        launch_gram<float>(st, n, q, q, S, n, G, n, h->part, h->M);
        launch_gram<float>(st, n, q, q, St, n, St, n, h->part, h->N);
        mark(h, "grams");
        if (!h->core_fp64)
            launch_core_ada32(st, q, h->M, h->N, Ci, Di, h->d_status);
        else
            launch_core_ada<float>(st, q, h->M, h->N, Ci, Di, h->d_status);
        mark(h, "q x q core");
    }
    bool wbf = core_first;  // W already launched on the side stream
    if (bfterms && !core_first) {  // W^T = L^T G on G's BF16 parts (written by G's epilogue unless G fell back)
        __nv_bfloat16_raw *gb = (__nv_bfloat16_raw *)h->Gbf;
        if (!gbf) tc_split_bf16(st, n, q, G, n, gb, gb + bfhalf, h->ldbf);
        wbf = tc_gemm_bf(h->tc, st, bfterms, n, q, n, L, n, gb, gb + bfhalf, h->ldbf, W, nullptr, n, stp, rsv) == 0;
    }
    if (!wbf)
        tc_gemm_nk_lo(h->tc, st, acc, TC_A_K, n, q, n, L, n, G, glo ? h->Glo : nullptr, n, W, nullptr, n, stp,
                      rsv);  // W^T = L^T G (n x q)
    if (fork) {  // join: C^-1 (or, with the core first, W) and D^-1 ready
        cudaStreamWaitEvent(st, h->ev_core, 0);
        if (tcv) cudaStreamWaitEvent(st, h->ev_d, 0);
    }
    mark(h, fork ? "W=G^TL | C core" : "W=G^TL");
    if (tcv) {
        // V^T = [S~ | W^T] [D^-T; -C^-T] (or both halves swapped), written transposed: V is q x n (ld q)
        tc_gemm_nk_t(h->tc, st, acc, TC_A_MN, n, q, 2 * q, SW, n, h->Bv, 2 * q, V, q, stp, 0,
                     (acc == 3 && bv_split(h)) ? h->Bvlo : nullptr);
        // S^ = S C^-T, written transposed (row-major n x q) for the K-major update operand (side stream
        // when the update is fused)
        if (!fuse) tc_gemm_nk_t(h->tc, st, upd, TC_A_MN, n, q, q, S, n, h->Bs, q, Sh, q, stp);
    } else {
        // V = D^-1 S~^T - C^-1 W, stored q x n (ld q); W^T is n x q (ld n)
        gemm_simt<float>(st, false, true, q, n, q, 1.f, Di, q, St, n, 0.f, V, q, stp);
        gemm_simt<float>(st, false, true, q, n, q, -1.f, Ci, q, W, n, 1.f, V, q, stp);
        // S^ = S C^-T stored row-major (n x q with q contiguous) for the K-major update operand
        gemm_simt<float>(st, false, true, q, n, q, 1.f, Ci, q, S, n, 0.f, Sh, q, stp);  // S^^T = C^-1 S^T (q x n)
    }
    mark(h, "V, S^");
    if (fuse) {
        // L += S^ V fused with S = L S~_{k+1} (the sketch was drawn on the side stream)
        if (fork)
            cudaStreamWaitEvent(st, h->ev_g, 0);
        else
            ada_draw<float>(h, St_next, h->k + 1);
        if (dpipe) {  // V has read Bv and S~_{k+1} is drawn: the next step's D chain, beside the update
            cudaEventRecord(h->ev_v, st);
            cudaStreamWaitEvent(h->st3, h->ev_v, 0);
            ada_d_chain(h, St_next, odd ? 0 : q, std::max(0, tc_num_sms() - SIDE_SMS_UPD));
            mark_side(h, h->st3, "@next D core done");
        }
        const int rc = tc_update_next_s(st, n, q, Sh, V, L, n, St_next, S, 1, h->Spart, h->spart_cap, stp, h->Slo,
                                        bfterms ? h->Sbf : nullptr, h->ldbf, dpipe ? SIDE_SMS_UPD : 0);
        h->d_ready = dpipe && rc == 0;
        if (rc == 0) {
            h->s_valid = true;
            h->slo_valid = h->Slo != nullptr;
            h->sbf_valid = bfterms != 0;
        } else {
            h->s_valid = false;
            h->slo_valid = false;
            h->sbf_valid = false;
            if (tc_update_persistent(h->tc, st, n, q, Sh, V, L, n, stp) != 0)
                tc_update(h->tc, st, upd, n, q, Sh, V, L, n, stp);
        }
        mark(h, "update L + next S");
    } else {
        // L += S^ V: persistent HBM-streaming kernel for the single-pass form
        if (upd != 1 || tc_update_persistent(h->tc, st, n, q, Sh, V, L, n, stp) != 0)
            tc_update(h->tc, st, upd, n, q, Sh, V, L, n, stp);
        mark(h, "update L");
    }
    if (fork) {
        cudaEventRecord(h->ev_out, h->st1);
        h->st = user;
        cudaStreamWaitEvent(user, h->ev_out, 0);
    }
}

extern "C" rb_status adarbfgs_step(rbfgs_t h, int nsteps)
{
    if (!h || nsteps < 0 || h->method != RB_METHOD_ADARBFGS) return RB_EINVAL;
    for (int s = 0; s < nsteps; ++s) {
        if (h->f64)
            ada_step_simt<double>(h);
        else if (h->prec == RB_FP32 || !h->tc)
            ada_step_simt<float>(h);
        else
            ada_step_tc(h);
        ++h->k;
    }
    RB_CUDA(cudaGetLastError());
    return RB_OK;
}

// ---------------------------------------------------------------------------
// Residual monitor.
// ---------------------------------------------------------------------------
static void host_floyd(uint64_t seed, int n, int m, std::vector<int> &out)
{
    out.assign(m, 0);
    for (int i = 0; i < m; ++i) {
        const uint32_t t = (uint32_t)(n - m + i);
        const u32x4 w = philox10((uint32_t)i, TAG_COLS, 0u, 0u, (uint32_t)seed, (uint32_t)(seed >> 32));
        const int d = (int)(((uint64_t)w.x * (uint64_t)(t + 1u)) >> 32);
        bool seen = false;
        for (int a = 0; a < i; ++a) seen |= (out[a] == d);
        out[i] = seen ? (int)t : d;
    }
    std::sort(out.begin(), out.end());
}

static rb_status ensure_resid_ws(rb_ctx *h, int m)
{
    if (m <= h->rcap) return RB_OK;
    rb_free(h->R1);
    rb_free(h->R2);
    rb_free(h->R3);
    rb_freet(h->J);
    rb_freet(h->rpart);
    h->rcap = 0;
    const size_t bytes = h->esz * (size_t)h->n * m;
    RB_TRY(rb_alloc(&h->R1, bytes));
    RB_TRY(rb_alloc(&h->R2, bytes));
    RB_TRY(rb_alloc(&h->R3, bytes));
    RB_TRY(rb_alloc(&h->J, sizeof(int) * m));
    RB_TRY(rb_alloc(&h->rpart, sizeof(double) * 32 * (size_t)m));
    h->rcap = m;
    return RB_OK;
}

template <typename T>
static void resid_products(rb_ctx *h, int m, const T *Y, T *Z1, T *Z)
{
    const int n = h->n;
    cudaStream_t st = h->st;
    const T *X = (const T *)h->X;
    const bool tc = (!h->f64 && h->tc && h->prec != RB_FP32);
    if (h->method == RB_METHOD_ADARBFGS) {
        if constexpr (sizeof(T) == 4) {
            if (tc) {
                // residual products always at ~FP32 accuracy (3-term split)
                tc_gemm_nk(h->tc, st, 3, TC_A_K, n, m, n, (const float *)X, n, (const float *)Y, n, (float *)Z1, n,
                           nullptr);
                tc_gemm_nk(h->tc, st, 3, TC_A_MN, n, m, n, (const float *)X, n, (const float *)Z1, n, (float *)Z, n,
                           nullptr);
                return;
            }
        }
        gemm_simt<T>(st, true, false, n, m, n, T(1), X, n, Y, n, T(0), Z1, n, nullptr);  // L^T A e_J
        gemm_simt<T>(st, false, false, n, m, n, T(1), X, n, Z1, n, T(0), Z, n, nullptr); // L L^T A e_J
    } else {
        gemm_simt<T>(st, false, false, n, m, n, T(1), X, n, Y, n, T(0), Z, n, nullptr);  // X A e_J
    }
}

template <typename T>
static void resid_launch(rb_ctx *h, bool exact, int m, const int *J)
{
    const int n = h->n;
    const T *Y = (const T *)h->A;  // exact: Y = A (all columns)
    if (!exact) {
        launch_gather_cols<T>(h->st, n, m, (const T *)h->A, n, J, (T *)h->R1, n);
        Y = (const T *)h->R1;
    }
    T *Z1 = (T *)h->R3, *Z = (T *)h->R2;
    resid_products<T>(h, m, Y, Z1, Z);
    launch_resid_sumsq<T>(h->st, n, m, Z, n, J, h->rpart, h->rsum);
}

extern "C" rb_status rbfgs_residual(rbfgs_t h, int ncols, uint64_t col_seed, double *out)
{
    if (!h || !out || ncols < 0) return RB_EINVAL;
    const int n = h->n;
    const bool exact = (ncols == 0 || ncols >= n);
    const int m = exact ? n : ncols;
    RB_TRY(ensure_resid_ws(h, m));
    cudaStream_t st = h->st;
    const int *J = nullptr;
    std::vector<int> hj;
    if (!exact) {
        host_floyd(col_seed, n, m, hj);
        RB_CUDA(cudaMemcpyAsync(h->J, hj.data(), sizeof(int) * m, cudaMemcpyHostToDevice, st));
        J = h->J;
    }
    if (h->f64)
        resid_launch<double>(h, exact, m, J);
    else
        resid_launch<float>(h, exact, m, J);
    RB_CUDA(cudaGetLastError());
    double sum = 0.0;
    RB_CUDA(cudaMemcpyAsync(&sum, h->rsum, sizeof(double), cudaMemcpyDeviceToHost, st));
    RB_CUDA(cudaStreamSynchronize(st));
    RB_TRY(status_from_device(h));
    const double r = sqrt(sum / m);
    if (!isfinite(r)) return RB_ENONFINITE;
    *out = r;
    return RB_OK;
}

extern "C" rb_status rbfgs_residual_start(rbfgs_t h, int ncols, uint64_t col_seed)
{
    if (!h || ncols < 0) return RB_EINVAL;
    const int n = h->n;
    const bool exact = (ncols == 0 || ncols >= n);
    const int m = exact ? n : ncols;
    RB_TRY(ensure_resid_ws(h, m));
    if (!h->ev_res) {
        RB_CUDA(cudaEventCreateWithFlags(&h->ev_res, cudaEventDisableTiming));
        RB_CUDA(cudaMallocHost(&h->h_rsum, sizeof(double)));
        RB_CUDA(cudaMallocHost(&h->h_status, sizeof(int)));
    }
    cudaStream_t st = h->st;
    const int *J = nullptr;
    if (!exact) {
        if (m > h->h_J_cap) {  // grown once; reused while no check is in flight
            if (h->h_J) cudaFreeHost(h->h_J);
            h->h_J = nullptr;
            h->h_J_cap = 0;
            RB_CUDA(cudaMallocHost(&h->h_J, sizeof(int) * m));
            h->h_J_cap = m;
        }
        std::vector<int> hj;
        host_floyd(col_seed, n, m, hj);
        memcpy(h->h_J, hj.data(), sizeof(int) * m);
        RB_CUDA(cudaMemcpyAsync(h->J, h->h_J, sizeof(int) * m, cudaMemcpyHostToDevice, st));
        J = h->J;
    }
    if (h->f64)
        resid_launch<double>(h, exact, m, J);
    else
        resid_launch<float>(h, exact, m, J);
    RB_CUDA(cudaMemcpyAsync(h->h_rsum, h->rsum, sizeof(double), cudaMemcpyDeviceToHost, st));
    RB_CUDA(cudaMemcpyAsync(h->h_status, h->d_status, sizeof(int), cudaMemcpyDeviceToHost, st));
    RB_CUDA(cudaEventRecord(h->ev_res, st));
    h->res_m = m;
    h->res_pending = 1;
    return RB_OK;
}

extern "C" rb_status rbfgs_residual_poll(rbfgs_t h, int *ready, double *out)
{
    if (!h || !ready || !out || !h->res_pending) return RB_EINVAL;
    const cudaError_t q = cudaEventQuery(h->ev_res);
    if (q == cudaErrorNotReady) {
        *ready = 0;
        return RB_OK;
    }
    if (q != cudaSuccess) return RB_ECUDA;
    *ready = 1;
    h->res_pending = 0;
    const int s = *h->h_status;
    if (s & ST_NOTSPD) return RB_ENOTSPD;
    if (s & ST_NONFINITE) return RB_ENONFINITE;
    if (s & ST_TIMEOUT) return RB_ETIMEOUT;
    const double r = sqrt(*h->h_rsum / h->res_m);
    if (!isfinite(r)) return RB_ENONFINITE;
    *out = r;
    return RB_OK;
}

extern "C" rb_status rbfgs_footprint(int n, const rb_opts *opts, size_t *bytes)
{
    if (n < 1 || !opts || !bytes) return RB_EINVAL;
    const size_t e = (opts->prec == RB_FP64) ? 8 : 4, q = (size_t)opts->q, nn = (size_t)n * n;
    size_t b = 2 * nn * e;                                // A and the iterate
    b += 10 * (size_t)n * q * e + 4 * q * q * 8;          // panels and q x q matrices
    b += (size_t)((n + 127) / 128) * q * q * 8;           // Gram chunk partials
    b += 3 * (size_t)n * 1024 * e;                        // residual workspace (<= 1024 columns)
    if (x_sketch_method(opts->method)) b += 3 * (size_t)n * q * e;
    b += 2 * (size_t)n * q * e;                           // tensor-core operand splits
    if (opts->prec == RB_BF16 || opts->prec == RB_BF16X3) b += 4 * (size_t)(n + 8) * q * 2;  // BF16 parts of S, G
    *bytes = b + (1u << 20);
    return RB_OK;
}

// Predicted spacing of residual checks: the residual falls about geometrically (the linear rate of
// Sec. 6; Sec. 9's one-step bound for AdaRBFGS improves as the iterate does), so from two checks
// (r0 after k0 steps, r1 after k1) the rate is log rho = log(r1 / r0) / (k1 - k0) and the steps
// left to tol are d = log(tol / r1) / log rho; the next check comes after d / 2 steps, at least e
// and at most 8 e (8 e while the residual is not falling).  Halving the predicted distance keeps
// the overshoot past the crossing at most e steps while the rate holds or improves, as it does
// for AdaRBFGS.
extern "C" int rb_next_check_gap(int e, int k0, double r0, int k1, double r1, double tol)
{
    if (e < 1) return 1;
    if (k0 < 0 || k1 <= k0 || !(r0 > 0) || !(r1 > tol) || !(tol > 0)) return e;
    const double lr = log(r1 / r0) / (double)(k1 - k0);
    if (!(lr < 0)) return 8 * e;
    const double half = 0.5 * log(tol / r1) / lr;
    return (int)std::max((double)e, std::min(8.0 * e, floor(half)));
}

extern "C" rb_status rbfgs_solve(rbfgs_t h, double tol, int max_iter, int check_every, int check_cols,
                                 int confirm_cols, int *iters, double *resid)
{
    if (!h || max_iter < 0 || check_every == 0 || check_cols < 0) return RB_EINVAL;
    const bool predicted = check_every < 0;
    const int e = predicted ? -check_every : check_every;
    int done = 0;
    double r = INFINITY;
    uint64_t col_seed = 0x5eed0000ull;
    int k0 = -1;  // the check before the last one: steps and residual
    double r0 = 0.0;
    int gap = e;
    while (done < max_iter) {
        const int chunk = std::min(gap, max_iter - done);
        rb_status s = RB_OK;
        if (h->method == RB_METHOD_RBFGS)
            s = rbfgs_step(h, chunk);
        else if (h->method == RB_METHOD_AIP)
            s = aip_step(h, chunk);
        else if (h->method == RB_METHOD_ADARBFGS)
            s = adarbfgs_step(h, chunk);
        else if (h->method == RB_METHOD_NS)
            s = newton_schulz_step(h, chunk);
        else
            s = mr_step(h, chunk);
        if (s != RB_OK) return s;
        done += chunk;
        RB_TRY(rbfgs_residual(h, check_cols, col_seed++, &r));
        double rk = r;
        if (r <= tol) {
            double rc = r;
            if (confirm_cols != check_cols) RB_TRY(rbfgs_residual(h, confirm_cols, col_seed++, &rc));
            r = rc;
            if (rc <= tol) break;
            rk = rc;
        }
        gap = predicted ? rb_next_check_gap(e, k0, r0, done, rk, tol) : e;
        k0 = done;
        r0 = rk;
    }
    if (iters) *iters = done;
    if (resid) *resid = r;
    return (r <= tol) ? RB_OK : RB_NOTCONV;
}

extern "C" rb_status rbfgs_export(rbfgs_t h, int what, void *out, int64_t ld)
{
    if (!h || !out || ld < h->n) return RB_EINVAL;
    const int n = h->n;
    if (what == RB_WHAT_L) {
        if (h->method != RB_METHOD_ADARBFGS) return RB_EINVAL;
    } else if (what != RB_WHAT_X) {
        return RB_EINVAL;
    }
    if (what == RB_WHAT_X && h->method == RB_METHOD_ADARBFGS) {
        if (h->f64)
            gemm_simt<double>(h->st, false, true, n, n, n, 1.0, (const double *)h->X, n, (const double *)h->X, n,
                              0.0, (double *)out, ld, nullptr);
        else
            gemm_simt<float>(h->st, false, true, n, n, n, 1.f, (const float *)h->X, n, (const float *)h->X, n, 0.f,
                             (float *)out, ld, nullptr);
    } else {
        if (h->f64)
            launch_copy2d<double, double>(h->st, n, n, (const double *)h->X, n, (double *)out, ld, 1.0);
        else
            launch_copy2d<float, float>(h->st, n, n, (const float *)h->X, n, (float *)out, ld, 1.0);
    }
    RB_CUDA(cudaGetLastError());
    return RB_OK;
}

extern "C" rb_status rbfgs_import(rbfgs_t h, int what, const void *in, int64_t ld)
{
    if (!h || !in || ld < h->n) return RB_EINVAL;
    const bool want_l = (h->method == RB_METHOD_ADARBFGS);
    if ((what == RB_WHAT_L) != want_l) return RB_EINVAL;
    const int n = h->n;
    if (h->f64)
        launch_copy2d<double, double>(h->st, n, n, (const double *)in, ld, (double *)h->X, n, 1.0);
    else
        launch_copy2d<float, float>(h->st, n, n, (const float *)in, ld, (float *)h->X, n, 1.0);
    RB_CUDA(cudaMemsetAsync(h->d_status, 0, sizeof(int), h->st));
    h->s_valid = false;
    h->d_ready = false;
    RB_CUDA(cudaGetLastError());
    return RB_OK;
}

extern "C" rb_status rbfgs_set_step(rbfgs_t h, uint64_t k)
{
    if (!h) return RB_EINVAL;
    h->k = k;
    h->s_valid = false;
    h->d_ready = false;
    return RB_OK;
}

extern "C" rb_status rbfgs_get_step(rbfgs_t h, uint64_t *k)
{
    if (!h || !k) return RB_EINVAL;
    *k = h->k;
    return RB_OK;
}

template <typename T>
static void coord_block_matrix(rb_ctx *h, uint64_t k, T *out, int64_t ld);

extern "C" rb_status rbfgs_draw_sketch(rbfgs_t h, uint64_t k, void *out, int64_t ld)
{
    if (!h || !out || ld < h->n || h->q < 1) return RB_EINVAL;
    const int n = h->n, q = h->q;
    if (x_sketch_method(h->method) && h->sketch == RB_SKETCH_COORD_TRACE) {
        if (h->f64)
            coord_block_matrix<double>(h, k, (double *)out, ld);
        else
            coord_block_matrix<float>(h, k, (float *)out, ld);
    } else if (h->sketch == RB_SKETCH_COORD_UNIFORM) {
        launch_floyd_draw(h->st, n, q, h->seed, h->stream_id, k, h->idx);
        if (h->f64)
            launch_coord_matrix<double>(h->st, n, q, h->idx, (double *)out, ld);
        else
            launch_coord_matrix<float>(h->st, n, q, h->idx, (float *)out, ld);
    } else {
        if (h->f64)
            launch_gauss_sketch<double>(h->st, n, q, h->seed, h->stream_id, k, (double *)out, ld);
        else
            launch_gauss_sketch<float>(h->st, n, q, h->seed, h->stream_id, k, (float *)out, ld);
    }
    RB_CUDA(cudaGetLastError());
    return RB_OK;
}

template <typename T>
static void coord_block_matrix(rb_ctx *h, uint64_t k, T *out, int64_t ld)
{
    const int n = h->n, q = h->q;
    launch_coord_trace_draw(h->st, n, q, h->nb, h->P, h->seed, h->stream_id, k, h->blk);
    // 0/1 matrix from the block: column c has a one in row first + c (c < size)
    launch_block_matrix<T>(h->st, n, q, h->blk, out, ld);
}

void rb_handle_status(rbfgs_t h, int **status, cudaStream_t *st)
{
    *status = h->d_status;
    *st = h->st;
}

extern "C" rb_status rbfgs_sync(rbfgs_t h)
{
    if (!h) return RB_EINVAL;
    return status_from_device(h);
}

// ---------------------------------------------------------------------------
// Comparison methods (Sec. 10).
// ---------------------------------------------------------------------------
static rb_status init_dense_method(rbfgs_t *out, int method, int n, const void *A_dev, int64_t lda, int a_is_fp64,
                                   int prec, void *stream, rb_ctx **hp)
{
    if (!out || !A_dev || n < 1 || lda < n || !prec_ok(prec)) return RB_EINVAL;
    *out = nullptr;
    if (prec_bf16(prec)) return RB_EUNSUPPORTED;
    rb_ctx *h = new rb_ctx();
    h->method = method;
    h->prec = prec;
    h->n = n;
    h->q = 0;
    h->f64 = (prec == RB_FP64);
    h->esz = h->f64 ? 8 : 4;
    h->st = (cudaStream_t)stream;
    rb_status s = RB_OK;
    do {
        if ((s = alloc_common(h)) != RB_OK) break;
        if ((s = copy_in_A(h, A_dev, lda, a_is_fp64)) != RB_OK) break;
        const size_t nn = h->esz * (size_t)n * n;
        if ((s = rb_alloc(&h->X, nn)) != RB_OK) break;
        if ((s = rb_alloc(&h->X2, nn)) != RB_OK) break;
        if ((s = rb_alloc(&h->X3, nn)) != RB_OK) break;
        if ((s = rb_alloc(&h->pv, sizeof(double) * n)) != RB_OK) break;
        if ((s = rb_alloc(&h->pw, sizeof(double) * n)) != RB_OK) break;
        if ((s = rb_alloc(&h->sigma, sizeof(double))) != RB_OK) break;
        if (!h->f64 && prec != RB_FP32) {
            h->tc = tc_plan_create(n, 0, prec);
            if (!h->tc) {
                s = RB_ENOMEM;
                break;
            }
        }
    } while (0);
    if (s != RB_OK) {
        destroy_ctx(h);
        return s;
    }
    *hp = h;
    return RB_OK;
}

extern "C" rb_status newton_schulz_init(rbfgs_t *out, int n, const void *A_dev, int64_t lda, int a_is_fp64,
                                        int prec, int power_iters, double sigma_override, void *stream)
{
    rb_ctx *h = nullptr;
    RB_TRY(init_dense_method(out, RB_METHOD_NS, n, A_dev, lda, a_is_fp64, prec, stream, &h));
    double sigma = sigma_override;
    if (!(sigma > 0.0)) {
        const int iters = power_iters > 0 ? power_iters : 100;
        if (h->f64)
            launch_power_iteration<double>(h->st, n, (const double *)h->A, n, iters, h->pv, h->pw, h->sigma);
        else
            launch_power_iteration<float>(h->st, n, (const float *)h->A, n, iters, h->pv, h->pw, h->sigma);
        if (cudaMemcpyAsync(&sigma, h->sigma, sizeof(double), cudaMemcpyDeviceToHost, h->st) != cudaSuccess ||
            cudaStreamSynchronize(h->st) != cudaSuccess) {
            destroy_ctx(h);
            return RB_ECUDA;
        }
    }
    h->host_sigma = sigma;
    const double scale = 0.99 / (sigma * sigma);
    // X0 = 0.99 A^T / sigma^2 (A symmetric)
    if (h->f64)
        launch_copy2d<double, double>(h->st, n, n, (const double *)h->A, n, (double *)h->X, n, scale);
    else
        launch_copy2d<float, float>(h->st, n, n, (const float *)h->A, n, (float *)h->X, n, scale);
    if (cudaGetLastError() != cudaSuccess) {
        destroy_ctx(h);
        return RB_ECUDA;
    }
    *out = h;
    return RB_OK;
}

template <typename T>
static void ns_step_impl(rb_ctx *h)
{
    const int n = h->n;
    cudaStream_t st = h->st;
    T *A = (T *)h->A, *X = (T *)h->X, *P = (T *)h->X2, *Xn = (T *)h->X3;
    if constexpr (sizeof(T) == 4) {
        if (h->tc) {
            const int terms = (h->prec == RB_TF32) ? 1 : 3;
            tc_gemm_nk(h->tc, st, terms, TC_A_K, n, n, n, (const float *)A, n, (const float *)X, n, (float *)P, n,
                       nullptr);                                                                   // P = A X
            mark(h, "P=AX");
            tc_gemm_nk_axpby(h->tc, st, terms, TC_A_MN, n, n, n, -1.f, (const float *)X, n, (const float *)P, n, 2.f,
                             (const float *)X, n, (float *)Xn, n);                                 // 2X - X P
            mark(h, "X=2X-XP");
            std::swap(h->X, h->X3);
            return;
        }
    }
    gemm_simt<T>(st, false, false, n, n, n, T(1), A, n, X, n, T(0), P, n, nullptr);      // P = A X
    mark(h, "P=AX");
    launch_copy2d<T, T>(st, n, n, X, n, Xn, n, 2.0);                                       // Xn = 2 X
    gemm_simt<T>(st, false, false, n, n, n, T(-1), X, n, P, n, T(1), Xn, n, nullptr);    // Xn -= X P
    mark(h, "X=2X-XP");
    std::swap(h->X, h->X3);
}

extern "C" rb_status newton_schulz_step(rbfgs_t h, int nsteps)
{
    if (!h || nsteps < 0 || h->method != RB_METHOD_NS) return RB_EINVAL;
    for (int s = 0; s < nsteps; ++s) {
        if (h->f64)
            ns_step_impl<double>(h);
        else
            ns_step_impl<float>(h);
        ++h->k;
    }
    RB_CUDA(cudaGetLastError());
    return RB_OK;
}

extern "C" rb_status rbfgs_sigma(rbfgs_t h, double *sigma)
{
    if (!h || !sigma || h->method != RB_METHOD_NS) return RB_EINVAL;
    *sigma = h->host_sigma;
    return RB_OK;
}

extern "C" rb_status rbfgs_core64(int q, const float *M_dev, float s, float *out_dev, int64_t ldo, int *cluster,
                                void *stream)
{
    if (q < 1 || q > 128 || !M_dev || !out_dev || ldo < q || ldo > INT32_MAX || !cluster || *cluster < 1 ||
        *cluster > 8)
        return RB_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    int *d_st = nullptr;
    if (cudaMalloc(&d_st, sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        return RB_ENOMEM;
    }
    int used = 0, hs = 0;
    rb_status r = RB_OK;
    if (cudaMemsetAsync(d_st, 0, sizeof(int), st) != cudaSuccess ||
        (used = launch_core_tr64(st, q, M_dev, out_dev, (int)ldo, s, nullptr, 0, 0.f, d_st, *cluster)) == 0 ||
        cudaMemcpyAsync(&hs, d_st, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        r = RB_ECUDA;
    cudaFree(d_st);
    if (r != RB_OK) return r;
    *cluster = used;
    return (hs & ST_NOTSPD) ? RB_ENOTSPD : (hs & ST_NONFINITE) ? RB_ENONFINITE : RB_OK;
}

extern "C" rb_status mr_init(rbfgs_t *out, int n, const void *A_dev, int64_t lda, int a_is_fp64, int prec,
                             void *stream)
{
    rb_ctx *h = nullptr;
    RB_TRY(init_dense_method(out, RB_METHOD_MR, n, A_dev, lda, a_is_fp64, prec, stream, &h));
    // X0 = (Tr A / Tr A A^T) I: Tr A and ||A||_F^2 summed in FP64 on the device
    if (h->f64) {
        launch_set_identity<double>(h->st, n, (double *)h->X2, n, 1.0);
        launch_mr_dots<double>(h->st, n, (const double *)h->X2, n, (const double *)h->A, n, h->dpart, h->dots);
    } else {
        launch_set_identity<float>(h->st, n, (float *)h->X2, n, 1.0f);
        launch_mr_dots<float>(h->st, n, (const float *)h->X2, n, (const float *)h->A, n, h->dpart, h->dots);
    }
    double d[2] = {0, 0};
    if (cudaMemcpyAsync(d, h->dots, sizeof(d), cudaMemcpyDeviceToHost, h->st) != cudaSuccess ||
        cudaStreamSynchronize(h->st) != cudaSuccess || !(d[1] > 0.0)) {
        destroy_ctx(h);
        return RB_ECUDA;
    }
    if (h->f64)
        launch_set_identity<double>(h->st, n, (double *)h->X, n, d[0] / d[1]);
    else
        launch_set_identity<float>(h->st, n, (float *)h->X, n, (float)(d[0] / d[1]));
    *out = h;
    return RB_OK;
}

template <typename T>
static void mr_step_impl(rb_ctx *h)
{
    const int n = h->n;
    cudaStream_t st = h->st;
    T *A = (T *)h->A, *X = (T *)h->X, *R = (T *)h->X2, *Q = (T *)h->X3;
    gemm_simt<T>(st, false, false, n, n, n, T(1), A, n, X, n, T(0), R, n, nullptr);   // A X
    launch_i_minus<T>(st, n, R, n);                                                      // R = I - A X
    gemm_simt<T>(st, false, false, n, n, n, T(1), X, n, R, n, T(0), Q, n, nullptr);   // X R
    T *AQ = (T *)h->R1;
    gemm_simt<T>(st, false, false, n, n, n, T(1), A, n, Q, n, T(0), AQ, n, nullptr);  // A X R
    launch_mr_dots<T>(st, n, R, n, AQ, n, h->dpart, h->dots);                          // <R, AXR>, ||AXR||^2
    launch_axpy_dev<T>(st, n, h->dots, Q, n, X, n);                                    // X += alpha X R
}

extern "C" rb_status mr_step(rbfgs_t h, int nsteps)
{
    if (!h || nsteps < 0 || h->method != RB_METHOD_MR) return RB_EINVAL;
    RB_TRY(ensure_resid_ws(h, h->n));
    for (int s = 0; s < nsteps; ++s) {
        if (h->f64)
            mr_step_impl<double>(h);
        else
            mr_step_impl<float>(h);
        ++h->k;
    }
    RB_CUDA(cudaGetLastError());
    return RB_OK;
}

extern "C" rb_status rbfgs_reset(rbfgs_t h, uint64_t seed, uint64_t stream_id)
{
    if (!h || (!x_sketch_method(h->method) && h->method != RB_METHOD_ADARBFGS)) return RB_EINVAL;
    if (h->f64)
        launch_set_identity<double>(h->st, h->n, (double *)h->X, h->n, 1.0);
    else
        launch_set_identity<float>(h->st, h->n, (float *)h->X, h->n, 1.0f);
    RB_CUDA(cudaMemsetAsync(h->d_status, 0, sizeof(int), h->st));
    h->k = 0;
    h->seed = seed;
    h->stream_id = stream_id;
    h->s_valid = false;
    h->d_ready = false;
    RB_CUDA(cudaGetLastError());
    return RB_OK;
}

extern "C" rb_status rbfgs_launch_count(uint64_t *count)
{
    if (!count) return RB_EINVAL;
    *count = g_rb_launches.load();
    return RB_OK;
}

extern "C" rb_status rbfgs_profile_step(rbfgs_t h, double *ms, const char **names, int cap, int *nphases)
{
    if (!h || !ms || !nphases || cap < 1) return RB_EINVAL;
    for (int i = 0; i < 24; ++i) RB_CUDA(cudaEventCreate(&h->prof_ev[i]));
    for (int i = 0; i < 8; ++i) RB_CUDA(cudaEventCreate(&h->prof_side_ev[i]));
    h->prof_on = 1;
    h->prof_n = 0;
    h->prof_ns = 0;
    cudaEventRecord(h->prof_ev[0], h->st);
    rb_status s;
    if (h->method == RB_METHOD_RBFGS)
        s = rbfgs_step(h, 1);
    else if (h->method == RB_METHOD_AIP)
        s = aip_step(h, 1);
    else if (h->method == RB_METHOD_ADARBFGS)
        s = adarbfgs_step(h, 1);
    else if (h->method == RB_METHOD_NS)
        s = newton_schulz_step(h, 1);
    else
        s = mr_step(h, 1);
    h->prof_on = 0;
    cudaError_t e = cudaEventSynchronize(h->prof_ev[h->prof_n]);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();  // the side-stream marks too
    int np = std::min(h->prof_n, cap);
    for (int i = 0; i < np && e == cudaSuccess; ++i) {
        float t = 0.f;
        cudaEventElapsedTime(&t, h->prof_ev[i], h->prof_ev[i + 1]);
        ms[i] = t;
        if (names) names[i] = h->prof_name[i];
    }
    // side-stream marks (names start with '@'): time from the step start, not a phase length
    for (int i = 0; i < h->prof_ns && np < cap && e == cudaSuccess; ++i, ++np) {
        float t = 0.f;
        cudaEventElapsedTime(&t, h->prof_ev[0], h->prof_side_ev[i]);
        ms[np] = t;
        if (names) names[np] = h->prof_side_name[i];
    }
    for (int i = 0; i < 24; ++i) cudaEventDestroy(h->prof_ev[i]);
    for (int i = 0; i < 8; ++i) cudaEventDestroy(h->prof_side_ev[i]);
    *nphases = np;
    if (s != RB_OK) return s;
    return e == cudaSuccess ? RB_OK : RB_ECUDA;
}

extern "C" rb_status rbfgs_load_host(rbfgs_t h, const void *A_host, int64_t lda, int a_is_fp64)
{
    if (!h || !A_host || lda < h->n || (!x_sketch_method(h->method) && h->method != RB_METHOD_ADARBFGS))
        return RB_EINVAL;
    const int n = h->n;
    const size_t in_esz = a_is_fp64 ? 8 : 4;
    if (in_esz == h->esz) {
        RB_CUDA(cudaMemcpy2DAsync(h->A, h->esz * n, A_host, in_esz * lda, in_esz * n, n, cudaMemcpyHostToDevice,
                                  h->st));
    } else {
        void *tmp = nullptr;
        RB_TRY(rb_alloc(&tmp, in_esz * (size_t)n * n));
        cudaMemcpy2DAsync(tmp, in_esz * n, A_host, in_esz * lda, in_esz * n, n, cudaMemcpyHostToDevice, h->st);
        if (a_is_fp64)
            launch_copy2d<double, float>(h->st, n, n, (const double *)tmp, n, (float *)h->A, n, 1.0);
        else
            launch_copy2d<float, double>(h->st, n, n, (const float *)tmp, n, (double *)h->A, n, 1.0);
        cudaStreamSynchronize(h->st);
        cudaFree(tmp);
    }
    if (h->f64)
        launch_set_identity<double>(h->st, n, (double *)h->X, n, 1.0);
    else
        launch_set_identity<float>(h->st, n, (float *)h->X, n, 1.0f);
    h->s_valid = false;
    h->d_ready = false;
    RB_CUDA(cudaMemsetAsync(h->d_status, 0, sizeof(int), h->st));
    h->k = 0;
    if (x_sketch_method(h->method) && h->sketch == RB_SKETCH_COORD_TRACE) {
        rb_freet(h->P);
        RB_TRY(build_trace_weights(h));
    }
    RB_CUDA(cudaGetLastError());
    return RB_OK;
}

extern "C" rb_status rbfgs_export_host(rbfgs_t h, int what, void *out_host, int64_t ld)
{
    if (!h || !out_host || ld < h->n) return RB_EINVAL;
    const int n = h->n;
    const void *src = h->X;
    if (what == RB_WHAT_X && h->method == RB_METHOD_ADARBFGS) {
        RB_TRY(h->X2 ? RB_OK : rb_alloc(&h->X2, h->esz * (size_t)n * n));
        RB_TRY(rbfgs_export(h, what, h->X2, n));
        src = h->X2;
    } else if (what == RB_WHAT_L && h->method != RB_METHOD_ADARBFGS) {
        return RB_EINVAL;
    }
    RB_CUDA(cudaMemcpy2DAsync(out_host, h->esz * ld, src, h->esz * n, h->esz * n, n, cudaMemcpyDeviceToHost, h->st));
    RB_CUDA(cudaStreamSynchronize(h->st));
    return RB_OK;
}

extern "C" rb_status rbfgs_destroy(rbfgs_t h)
{
    if (!h) return RB_EINVAL;
    cudaStreamSynchronize(h->st);
    destroy_ctx(h);
    return RB_OK;
}
