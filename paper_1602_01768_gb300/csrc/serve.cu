// serve.cu -- continuous-batching server for AdaRBFGS inversion requests.
//
// Requests (an SPD A, a tolerance, a seed) are queued on submit.  A
// scheduler thread admits them first-come-first-served while the HBM budget
// (the handles' footprint, rbfgs_footprint) and the live-request cap allow,
// gives each admitted request its own handle and CUDA stream, and keeps
// every live request moving: `check_every` AdaRBFGS steps, then a
// non-blocking residual check, polled without waiting.  (A fixed, short chunk:
// a request's chunk is enqueued on its stream in one go, and a chunk of a few
// hundred steps would fill the stream's launch queue and block the scheduler
// thread, starving the other requests.)  Requests that reach
// their tolerance (or fail, or hit max_iter) write their factor L to the
// caller's output, release their memory and wake waiters, so queued
// requests are admitted as soon as room frees up.  Work of different
// requests overlaps on the device through their streams; each request's
// arithmetic is that of a lone handle with the same seed, so its result
// does not depend on what else is running.
#include <math.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include <cuda_runtime.h>

#include "rbfgs.h"

namespace {

enum { Q_QUEUED = 0, Q_RUNNING = 1, Q_DONE = 2 };

struct Req {
    int64_t id = 0;
    int n = 0, q = 0;
    double tol = 0;
    uint64_t seed = 0;
    const void *A = nullptr;
    int a_on_device = 0, a_is_fp64 = 0;
    int64_t lda = 0;
    void *out = nullptr;
    int out_on_device = 0;
    int64_t ldo = 0;
    size_t bytes = 0;
    double t_submit = 0, t_admit = 0, t_done = 0;
    int state = Q_QUEUED;
    rbfgs_t h = nullptr;
    cudaStream_t st = nullptr;
    void *staging = nullptr;
    int steps = 0;
    double resid = INFINITY;
    int status = RB_OK;
    uint64_t col_seed = 0;
    int prec = RB_MIXED;     // the form this request runs in (chosen from its tolerance)
    double best = INFINITY;  // smallest residual seen (updated on a 10 % fall) and the steps then
    int best_steps = 0;
    int floor_limited = 0;
};

// Form of a request: the server's form, except that a BF16 form serves only tolerances down to
// 1e-4 (the 3-term BF16 products leave a residual floor near 2e-5 on the request matrices; the
// 3xTF32 mixed form's is near 7e-6 at n / q = 64).
int request_prec(int server_prec, double tol)
{
    if ((server_prec == RB_BF16X3 || server_prec == RB_BF16) && tol < 1e-4) return RB_MIXED;
    return server_prec;
}

// Steps without a 10 % fall of the residual, in units of the check spacing, after which a
// request is finished as floor-limited: the residual then sits at the floor of the request's
// arithmetic, above its tolerance.
constexpr int STALL_CHECKS = 8;

double now_s(const std::chrono::steady_clock::time_point &t0)
{
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
}

}  // namespace

struct rb_srv {
    size_t budget = 0, used = 0;
    int max_live = 0, prec = RB_MIXED, check_every = 32, check_cols = 256, max_iter = 20000;
    int device = 0;
    std::mutex mu;
    std::condition_variable cv;
    std::deque<int64_t> queue;
    std::map<int64_t, Req *> reqs;
    std::vector<Req *> live;
    std::thread worker;
    bool stop = false;
    int64_t next_id = 1;
    std::chrono::steady_clock::time_point t0;
    std::vector<double> latencies;
    int completed = 0, failed = 0;
    double first_submit = -1, last_done = 0;
};

static void release(rb_srv *s, Req *r)
{
    if (r->h) rbfgs_destroy(r->h);
    r->h = nullptr;
    if (r->staging) cudaFree(r->staging);
    r->staging = nullptr;
    if (r->st) cudaStreamDestroy(r->st);
    r->st = nullptr;
}

// Admission work for one request (outside the lock): stream, handle, first chunk.
static void start_request(rb_srv *s, Req *r)
{
    rb_opts o;
    rbfgs_default_opts(&o);
    o.method = RB_METHOD_ADARBFGS;
    o.sketch = RB_SKETCH_GAUSS;
    o.q = r->q;
    o.prec = r->prec;
    o.seed = r->seed;
    rb_status st = RB_OK;
    if (cudaStreamCreateWithFlags(&r->st, cudaStreamNonBlocking) != cudaSuccess) st = RB_ECUDA;
    const void *Adev = r->A;
    int64_t lda = r->lda;
    if (st == RB_OK && !r->a_on_device) {
        const size_t esz = r->a_is_fp64 ? 8 : 4;
        if (cudaMalloc(&r->staging, esz * (size_t)r->n * r->n) != cudaSuccess) {
            st = RB_ENOMEM;
        } else if (cudaMemcpy2DAsync(r->staging, esz * r->n, r->A, esz * r->lda, esz * r->n, r->n,
                                     cudaMemcpyHostToDevice, r->st) != cudaSuccess) {
            st = RB_ECUDA;
        }
        Adev = r->staging;
        lda = r->n;
    }
    if (st == RB_OK) st = rbfgs_init(&r->h, r->n, Adev, lda, r->a_is_fp64, &o, r->st);
    if (st == RB_OK && r->staging) {  // init copied A into the handle
        cudaStreamSynchronize(r->st);
        cudaFree(r->staging);
        r->staging = nullptr;
    }
    if (st == RB_OK) st = adarbfgs_step(r->h, s->check_every);
    if (st == RB_OK) {
        r->steps = s->check_every;
        st = rbfgs_residual_start(r->h, s->check_cols, r->col_seed++);
    }
    r->status = st;
}

// Completion work (outside the lock): copy L out, free the request's memory.
static void finish_request(rb_srv *s, Req *r)
{
    if (r->h && r->out && r->status != RB_ENOTSPD && r->status >= 0) {
        rb_status st;
        if (r->out_on_device) {
            st = rbfgs_export(r->h, RB_WHAT_L, r->out, r->ldo);
            if (st == RB_OK && cudaStreamSynchronize(r->st) != cudaSuccess) st = RB_ECUDA;
        } else {
            st = rbfgs_export_host(r->h, RB_WHAT_L, r->out, r->ldo);
        }
        if (st != RB_OK) r->status = st;
    }
    release(s, r);
}

static void worker_loop(rb_srv *s)
{
    cudaSetDevice(s->device);
    std::vector<Req *> admitted, finished;
    for (;;) {
        admitted.clear();
        {
            std::unique_lock<std::mutex> lk(s->mu);
            if (s->stop && s->queue.empty() && s->live.empty()) break;
            if (s->queue.empty() && s->live.empty()) {
                s->cv.wait_for(lk, std::chrono::milliseconds(50));
                continue;
            }
            while (!s->queue.empty() && (int)s->live.size() < s->max_live) {
                Req *r = s->reqs[s->queue.front()];
                if (s->used + r->bytes > s->budget) break;  // first come, first served
                s->queue.pop_front();
                s->used += r->bytes;
                r->state = Q_RUNNING;
                r->t_admit = now_s(s->t0);
                s->live.push_back(r);
                admitted.push_back(r);
            }
        }
        for (Req *r : admitted) start_request(s, r);
        // progress every live request whose residual check has landed
        finished.clear();
        std::vector<Req *> live;
        {
            std::lock_guard<std::mutex> lk(s->mu);
            live = s->live;
        }
        bool progressed = !admitted.empty();
        for (Req *r : live) {
            bool done = false;
            if (r->status != RB_OK) {
                done = true;
            } else {
                int ready = 0;
                double res = 0;
                rb_status st = rbfgs_residual_poll(r->h, &ready, &res);
                if (st != RB_OK) {
                    r->status = st;
                    done = true;
                } else if (ready) {
                    progressed = true;
                    r->resid = res;
                    if (res < 0.9 * r->best) {
                        r->best = res;
                        r->best_steps = r->steps;
                    }
                    if (res <= r->tol) {
                        done = true;
                    } else if (r->steps >= s->max_iter) {
                        r->status = RB_NOTCONV;
                        done = true;
                    } else if (r->steps - r->best_steps >= STALL_CHECKS * s->check_every) {  // at its floor
                        r->status = RB_NOTCONV;
                        r->floor_limited = 1;
                        r->resid = r->best;
                        done = true;
                    } else {
                        const int chunk = std::min(s->check_every, s->max_iter - r->steps);
                        st = adarbfgs_step(r->h, chunk);
                        if (st == RB_OK) st = rbfgs_residual_start(r->h, s->check_cols, r->col_seed++);
                        r->steps += chunk;
                        if (st != RB_OK) {
                            r->status = st;
                            done = true;
                        }
                    }
                }
            }
            if (done) finished.push_back(r);
        }
        for (Req *r : finished) finish_request(s, r);
        if (!finished.empty()) {
            std::lock_guard<std::mutex> lk(s->mu);
            const double t = now_s(s->t0);
            for (Req *r : finished) {
                r->t_done = t;
                r->state = Q_DONE;
                s->used -= r->bytes;
                s->live.erase(std::find(s->live.begin(), s->live.end(), r));
                s->latencies.push_back(r->t_done - r->t_submit);
                if (r->status == RB_OK)
                    ++s->completed;
                else
                    ++s->failed;
                s->last_done = t;
            }
            s->cv.notify_all();
        }
        if (!progressed && finished.empty()) std::this_thread::sleep_for(std::chrono::microseconds(20));
    }
}

extern "C" rb_status rb_srv_create(rb_srv_t *out, size_t hbm_budget_bytes, int max_live, int prec, int check_every,
                                   int check_cols, int max_iter)
{
    if (!out || hbm_budget_bytes == 0 || max_live < 1 || check_every < 1 || check_cols < 1 || max_iter < 1)
        return RB_EINVAL;
    if (prec != RB_FP32 && prec != RB_TF32 && prec != RB_TF32X3 && prec != RB_MIXED && prec != RB_FP64 &&
        prec != RB_BF16 && prec != RB_BF16X3)
        return RB_EINVAL;
    rb_srv *s = new rb_srv();
    s->budget = hbm_budget_bytes;
    s->max_live = max_live;
    s->prec = prec;
    s->check_every = check_every;
    s->check_cols = check_cols;
    s->max_iter = max_iter;
    s->t0 = std::chrono::steady_clock::now();
    if (cudaGetDevice(&s->device) != cudaSuccess) {
        delete s;
        return RB_ECUDA;
    }
    s->worker = std::thread(worker_loop, s);
    *out = s;
    return RB_OK;
}

extern "C" rb_status rb_srv_submit(rb_srv_t s, int n, const void *A, int a_on_device, int64_t lda, int a_is_fp64,
                                   double tol, uint64_t seed, int q, void *out, int out_on_device, int64_t ldo,
                                   int64_t *ticket)
{
    if (!s || !A || n < 1 || lda < n || !(tol > 0) || !ticket || (out && ldo < n)) return RB_EINVAL;
    if (q <= 0) q = std::max(32, 32 * (int)lround(sqrt((double)n) / 32.0));
    q = std::min(q, std::min(n, 128));
    rb_opts o;
    rbfgs_default_opts(&o);
    o.method = RB_METHOD_ADARBFGS;
    o.q = q;
    o.prec = request_prec(s->prec, tol);
    size_t bytes = 0;
    if (rbfgs_footprint(n, &o, &bytes) != RB_OK) return RB_EINVAL;
    if (!a_on_device) bytes += (size_t)n * n * (a_is_fp64 ? 8 : 4);  // staging copy at admission
    if (bytes > s->budget) return RB_ENOMEM;                           // could never be admitted
    Req *r = new Req();
    r->n = n;
    r->q = q;
    r->tol = tol;
    r->seed = seed;
    r->A = A;
    r->a_on_device = a_on_device;
    r->a_is_fp64 = a_is_fp64;
    r->lda = lda;
    r->out = out;
    r->out_on_device = out_on_device;
    r->ldo = ldo;
    r->bytes = bytes;
    r->col_seed = seed ^ 0x9e3779b97f4a7c15ull;
    r->prec = o.prec;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->stop) {
            delete r;
            return RB_EINVAL;
        }
        r->id = s->next_id++;
        r->t_submit = now_s(s->t0);
        if (s->first_submit < 0) s->first_submit = r->t_submit;
        s->reqs[r->id] = r;
        s->queue.push_back(r->id);
        *ticket = r->id;
    }
    s->cv.notify_all();
    return RB_OK;
}

extern "C" rb_status rb_srv_poll(rb_srv_t s, int64_t ticket, int *done)
{
    if (!s || !done) return RB_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return RB_EINVAL;
    *done = it->second->state == Q_DONE;
    return RB_OK;
}

extern "C" rb_status rb_srv_wait(rb_srv_t s, int64_t ticket, double timeout_s, rb_srv_result *res)
{
    if (!s || !res) return RB_EINVAL;
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return RB_EINVAL;
    Req *r = it->second;
    const auto deadline = std::chrono::steady_clock::now() + std::chrono::duration<double>(timeout_s);
    while (r->state != Q_DONE) {
        if (s->cv.wait_until(lk, deadline) == std::cv_status::timeout && r->state != Q_DONE) return RB_ETIMEOUT;
    }
    res->ticket = r->id;
    res->status = r->status;
    res->iters = r->steps;
    res->resid = r->resid;
    res->latency_s = r->t_done - r->t_submit;
    res->queue_s = r->t_admit - r->t_submit;
    res->n = r->n;
    res->q = r->q;
    res->prec = r->prec;
    res->floor_limited = r->floor_limited;
    s->reqs.erase(it);
    delete r;
    return RB_OK;
}

extern "C" rb_status rb_srv_stats(rb_srv_t s, rb_srv_summary *st)
{
    if (!s || !st) return RB_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    std::vector<double> lat = s->latencies;
    std::sort(lat.begin(), lat.end());
    auto pct = [&](double p) {
        if (lat.empty()) return 0.0;
        size_t i = (size_t)ceil(p * lat.size());
        if (i > 0) --i;
        return lat[std::min(i, lat.size() - 1)];
    };
    st->completed = s->completed;
    st->failed = s->failed;
    st->queued = (int)s->queue.size();
    st->live = (int)s->live.size();
    st->p50_s = pct(0.50);
    st->p99_s = pct(0.99);
    const double span = s->last_done - (s->first_submit < 0 ? 0 : s->first_submit);
    st->solves_per_s = span > 0 ? s->completed / span : 0.0;
    st->hbm_in_use = s->used;
    return RB_OK;
}

extern "C" rb_status rb_srv_destroy(rb_srv_t s)
{
    if (!s) return RB_EINVAL;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv.notify_all();
    if (s->worker.joinable()) s->worker.join();
    for (auto &kv : s->reqs) delete kv.second;
    delete s;
    return RB_OK;
}
