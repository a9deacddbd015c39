/*
 * rbfgs.h -- C ABI of the GB300 (sm_103a) library for randomized quasi-Newton
 * matrix inversion (Gower & Richtarik, "Randomized Quasi-Newton Updates are
 * Linearly Convergent Matrix Inversion Algorithms", arXiv:1602.01768).
 *
 * The problem (Sec. 5 and Sec. 9): given a dense symmetric positive definite
 * A (n x n), iterate towards X = A^-1 with
 *   - RBFGS (Algorithm 3 with W = A^-1, the block BFGS update Eq. (qunac),
 *     Sec. 8.8):  X+ = S L S^T + (I - S L S^T A) X (I - A S L S^T),
 *     L = (S^T A S)^-1, S drawn i.i.d. each step (Gaussian or a coordinate
 *     block);
 *   - AdaRBFGS (Algorithm 4, factored update Eq. (Cholimprov), Sec. 9.3):
 *     X = L L^T kept as its factor, S = L S~ with S~ drawn i.i.d.;
 *   - Newton-Schulz, Eq. (Newton-Schulz), and MR, Eq. (MRiter), the
 *     comparison methods of Sec. 10.
 *
 * Conventions shared by every entry point
 *   - Matrices are column-major with an explicit leading dimension (ld >= n),
 *     element type FP32 or FP64 as stated per call.
 *   - Pointers named *_dev are device pointers of the current CUDA device;
 *     pointers named *_host are host pointers (pinned or pageable).
 *   - A handle owns every device buffer it allocates (its copy of A, the
 *     iterate X or its factor L, workspaces); the caller owns everything it
 *     passes in and may free it as soon as the call returns.
 *   - All work is queued on the CUDA stream given at creation (a cudaStream_t
 *     passed as void*; NULL = legacy default stream).  Step calls are
 *     asynchronous; calls documented as "synchronises" wait for the stream.
 *   - Every call returns an rb_status and never aborts the process.  Device
 *     side failures (a Cholesky breakdown, a non-finite value) are recorded
 *     in a device status word; the step that hits one and every later step
 *     leave the iterate untouched, and the next synchronising call returns
 *     the failure.
 *   - A handle is used from one host thread at a time; distinct handles are
 *     independent.
 */
#ifndef RBFGS_H
#define RBFGS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rb_ctx *rbfgs_t;

typedef enum {
    RB_OK = 0,
    RB_NOTCONV = 1,        /* solve stopped at max_iter above the tolerance (not an error) */
    RB_EINVAL = -1,        /* bad argument (null pointer, n < 1, q out of range, ld < n) */
    RB_ENOMEM = -2,        /* device allocation failed */
    RB_ECUDA = -3,         /* a CUDA runtime call failed */
    RB_ENOTSPD = -4,       /* Cholesky of S^T A S or S~^T S~ met a pivot <= 0 / non-finite:
                              A is not SPD or S is rank deficient (Thm 5.1 needs full rank) */
    RB_ENONFINITE = -5,    /* a non-finite residual */
    RB_ETIMEOUT = -6,      /* a bounded device-side wait gave up */
    RB_EUNSUPPORTED = -7   /* combination not built (method/precision/sketch) */
} rb_status;

typedef enum {
    RB_FP64 = 0,    /* FP64 storage and arithmetic (the parity mode) */
    RB_FP32 = 1,    /* FP32 storage, FP32 SIMT products (q x q core: see rb_opts.core_fp64) */
    RB_TF32 = 2,    /* FP32 storage, single-pass TF32 tensor-core products */
    RB_TF32X3 = 3,  /* FP32 storage, 3-term split TF32 tensor-core products (~FP32 accuracy) */
    RB_MIXED = 4,   /* FP32 storage, 3xTF32 where accuracy needs it, 1xTF32 for the
                       rank-q correction whose size vanishes at the fixed point */
    RB_BF16 = 5,    /* AdaRBFGS only: as RB_TF32, with the two n x n-streaming products
                       G = A S and W^T = L^T G in one BF16 pass (8 significant bits) */
    RB_BF16X3 = 6   /* AdaRBFGS only: as RB_MIXED, with G = A S and W^T = L^T G as 3-term
                       BF16 splits (hi hi + hi lo + lo hi, ~16 significant bits): half the
                       tensor-core work of 3xTF32 for the two passes that stream A and L */
} rb_prec;

typedef enum {
    RB_SKETCH_GAUSS = 0,          /* S (RBFGS) or S~ (AdaRBFGS) i.i.d. N(0,1), n x q */
    RB_SKETCH_COORD_TRACE = 1,    /* RBFGS: contiguous block of q coordinates, drawn with
                                     probability proportional to its diagonal trace
                                     (Sec. 7.2, Eq. (convprob) with W = A^-1) */
    RB_SKETCH_COORD_UNIFORM = 2   /* AdaRBFGS_cols: q distinct coordinates, uniform (Sec. 10) */
} rb_sketch;

typedef enum {
    RB_METHOD_RBFGS = 0,
    RB_METHOD_ADARBFGS = 1,
    RB_METHOD_NS = 2,
    RB_METHOD_MR = 3,
    RB_METHOD_AIP = 4 /* approximate inverse preconditioning, Eq. (BFGSas) */
} rb_method;

typedef enum { RB_WHAT_X = 0, RB_WHAT_L = 1 } rb_what;

typedef struct {
    int32_t method;     /* rb_method */
    int32_t sketch;     /* rb_sketch */
    int32_t q;          /* sketch width, 1 <= q <= min(n, 128) */
    int32_t prec;       /* rb_prec */
    uint64_t seed;      /* Philox key of the sketch stream */
    uint64_t stream_id; /* Philox counter word 3: independent streams for one seed */
    int32_t power_iters;/* Newton-Schulz: power iterations for ||A||_2 (0 = 100) */
    int32_t core_fp64;  /* AdaRBFGS with FP32 storage, precision of the q x q Cholesky factors and
                           their inverses: 1 = FP64 (both), -1 = FP32 (both), 0 = the form's
                           default: the tensor-core forms factor C C^T = S^T A S in FP64 (with
                           q <= 128 and n a multiple of 4) and D D^T = S~^T S~ (a Gaussian Gram,
                           condition number near 1) in FP32; RB_FP32 factors both in FP32; FP64
                           storage always factors in FP64 */
    int32_t reserved[6];
} rb_opts;

/* Fill *opts with defaults: RBFGS, Gaussian sketch, q = 8, FP64, seed 0, stream 0. */
void rbfgs_default_opts(rb_opts *opts);

/*
 * Create a solver for the n x n SPD matrix A_dev (ld lda, a_is_fp64 selects
 * FP64 or FP32 elements).  A is copied into the handle's storage type (FP64
 * for RB_FP64, FP32 otherwise).  The iterate starts at X0 = I (RBFGS) or
 * L0 = I (AdaRBFGS), the starts of Sec. 10; Newton-Schulz and MR use
 * newton_schulz_init / mr_init.  The step counter k starts at 0.
 * Errors: RB_EINVAL, RB_ENOMEM, RB_ECUDA, RB_EUNSUPPORTED.
 */
rb_status rbfgs_init(rbfgs_t *h, int n, const void *A_dev, int64_t lda, int a_is_fp64,
                     const rb_opts *opts, void *stream);

/*
 * nsteps RBFGS steps (Algorithm 3, W = A^-1): draw S_k, G = A S, the q x q
 * core (Cholesky of S^T A S in FP64 in every form), Y = X G, T = G^T Y and the symmetric
 * rank-2q update X += S W^T + W S^T, W = S (Lam + Lam T Lam)/2 - Y Lam, which
 * equals Eq. (qunac).  Asynchronous.  The handle must be an RBFGS handle.
 */
rb_status rbfgs_step(rbfgs_t h, int nsteps);

/*
 * nsteps steps of the approximate inverse preconditioning update, Eq.
 * (BFGSas) of Sec. 8 (the nonsymmetric row variant, Algorithm 1, with
 * W = A^-1 for SPD A):  X+ = X + S (S^T A S)^-1 S^T (I - A X),  computed as
 * G = A S, Lambda = (S^T G)^-1 (Cholesky in FP64), W = G^T X,
 * X += S Lambda (S^T - W).  The iterate is not symmetric in general; with a
 * coordinate block C only the rows C of X change.  Sketches as for RBFGS
 * (RB_SKETCH_GAUSS or RB_SKETCH_COORD_TRACE, q <= 64); all precisions run
 * on CUDA cores (FP64 for RB_FP64, FP32 otherwise).  Asynchronous.  The
 * handle must be created with opts.method = RB_METHOD_AIP (X0 = I).
 * Errors: RB_EINVAL; a breakdown of S^T A S is reported as RB_ENOTSPD by the
 * next synchronising call.
 */
rb_status aip_step(rbfgs_t h, int nsteps);

/*
 * nsteps AdaRBFGS steps (Algorithm 4, Eq. (Cholimprov)): draw S~_k,
 * S = L S~, G = A S, C C^T = S^T A S and D D^T = S~^T S~ (lower Cholesky in
 * the precision opts.core_fp64 selects), W = G^T L,
 * V = D^-1 S~^T - C^-1 W, L += S C^-T V.  Asynchronous.
 */
rb_status adarbfgs_step(rbfgs_t h, int nsteps);

/*
 * The q x q core of Algorithm 4 on its own, in FP64: the lower Cholesky
 * factor C of the symmetric part of M (C C^T = (M + M^T) / 2; M is q x q FP32,
 * column-major, ld q, device memory, q <= 128) and its inverse, written as
 * s C^-T (FP32, ld ldo >= q, device memory): R = C^-T of Eq. (Cholimprov),
 * scaled.  *cluster in 1 .. 8 asks for the CTAs to spread the FP64 work over
 * (a thread-block cluster when it is more than 1); on return it holds the CTAs
 * that ran (1 when no such cluster fits).  Every cluster size gives the same
 * bits.  A pivot <= 0 or non-finite returns RB_ENOTSPD and leaves out_dev
 * untouched.  Allocates one status word; synchronises the stream.
 */
rb_status rbfgs_core64(int q, const float *M_dev, float s, float *out_dev, int64_t ldo, int *cluster,
                       void *stream);

/*
 * Residual ||I - X A||_F / sqrt(n) of the current iterate (X = L L^T for
 * AdaRBFGS), the stopping quantity of Sec. 10 without its normalisation by
 * ||I - A X0||_F.  ncols = 0 evaluates it exactly (cost O(n^3)); ncols = m > 0
 * estimates it from m distinct columns J (Floyd sampling on Philox with key
 * col_seed): sqrt(sum_{j in J} ||e_j - X A e_j||^2 / m).  Sums in FP64.
 * Synchronises; returns the first recorded device failure, if any.
 */
rb_status rbfgs_residual(rbfgs_t h, int ncols, uint64_t col_seed, double *out);

/*
 * Non-blocking form of rbfgs_residual: rbfgs_residual_start queues the
 * residual kernels and the copy of its sum (and of the status word) to
 * pinned host memory on the handle's stream; rbfgs_residual_poll sets
 * *ready = 0 while that is in flight, else *ready = 1 and *out (or the
 * recorded device failure).  One check in flight per handle.
 */
rb_status rbfgs_residual_start(rbfgs_t h, int ncols, uint64_t col_seed);
rb_status rbfgs_residual_poll(rbfgs_t h, int *ready, double *out);

/* Device bytes rbfgs_init (plus a residual check of up to 1024 columns) allocates
 * for an n x n problem with these options -- the admission test of the server. */
rb_status rbfgs_footprint(int n, const rb_opts *opts, size_t *bytes);

/*
 * Run steps until the sampled residual (check_cols columns; a final exact or
 * sampled confirmation with confirm_cols, 0 = exact) is <= tol, or max_iter
 * steps are done.  check_every > 0: a check every check_every steps.
 * check_every = -e < 0: predicted spacing -- e steps to the first two checks,
 * then half the steps that the geometric rate seen between the last two
 * checks predicts to reach tol, at least e and at most 8 e (the residual
 * decays linearly in expectation, Sec. 6).  Each check draws a fresh column
 * sample.  *iters gets the steps taken, *resid the last confirmed residual.
 * Returns RB_OK, RB_NOTCONV or an error (RB_EINVAL for check_every = 0).
 * Synchronises.
 */
rb_status rbfgs_solve(rbfgs_t h, double tol, int max_iter, int check_every, int check_cols,
                      int confirm_cols, int *iters, double *resid);

/*
 * The predicted check spacing of rbfgs_solve, for callers that run their own
 * loop on one handle: steps to the next check after checks with residuals r0 (after k0
 * steps) and r1 (after k1 > k0 steps), minimum spacing e >= 1.  Returns e when
 * k0 < 0 (no earlier check), r1 <= tol or an argument is not positive; 8 e when
 * r1 >= r0; else floor(log(tol / r1) / (2 log rho)) with
 * log rho = log(r1 / r0) / (k1 - k0), clamped to [e, 8 e].  Host only.
 */
int rb_next_check_gap(int e, int k0, double r0, int k1, double r1, double tol);

/*
 * Copy the iterate out: what = RB_WHAT_X (X; for AdaRBFGS X = L L^T is formed)
 * or RB_WHAT_L (AdaRBFGS factor).  out_dev has the handle's storage type
 * (FP64 for RB_FP64, else FP32) and leading dimension ld.  Asynchronous.
 */
rb_status rbfgs_export(rbfgs_t h, int what, void *out_dev, int64_t ld);

/*
 * Replace the iterate (X for RBFGS/NS/MR, L for AdaRBFGS) by in_dev (storage
 * type, ld).  With rbfgs_set_step this resumes a run from a checkpoint: the
 * sketch stream is counter based, so the resumed run draws exactly the
 * sketches of the uninterrupted one.  Asynchronous.
 */
rb_status rbfgs_import(rbfgs_t h, int what, const void *in_dev, int64_t ld);
rb_status rbfgs_set_step(rbfgs_t h, uint64_t k);
rb_status rbfgs_get_step(rbfgs_t h, uint64_t *k);

/*
 * Write the sketch of step k into out_dev (n x q, storage type, ld >= n):
 * the Gaussian S_k (RBFGS) or S~_k (AdaRBFGS), or the 0/1 coordinate matrix
 * I[:, C_k] (columns beyond a ragged last block are zero).  The draw is a pure
 * function of (seed, stream_id, k), so this reproduces exactly what step k
 * uses.  Asynchronous.
 */
rb_status rbfgs_draw_sketch(rbfgs_t h, uint64_t k, void *out_dev, int64_t ld);

/* Device status word (0 = fine); synchronises. */
rb_status rbfgs_sync(rbfgs_t h);

/*
 * Newton-Schulz (Sec. 10): X0 = 0.99 A / sigma^2, sigma = ||A||_2 from
 * power_iters steps of the power iteration started at 1/sqrt(n) (standing in
 * for MATLAB normest); sigma_override > 0 skips the estimate.  Steps:
 * X+ = 2 X - X (A X), Eq. (Newton-Schulz).  Use rbfgs_residual / export /
 * destroy on the handle.
 */
rb_status newton_schulz_init(rbfgs_t *h, int n, const void *A_dev, int64_t lda, int a_is_fp64,
                             int prec, int power_iters, double sigma_override, void *stream);
rb_status newton_schulz_step(rbfgs_t h, int nsteps);

/*
 * Minimal residual (Sec. 10, Eq. (MRiter)): X0 = (Tr A / Tr A A^T) I;
 * R = I - A X, X+ = X + alpha X R, alpha = <R, A X R> / ||A X R||_F^2.
 */
rb_status mr_init(rbfgs_t *h, int n, const void *A_dev, int64_t lda, int a_is_fp64, int prec,
                  void *stream);
rb_status mr_step(rbfgs_t h, int nsteps);

/* Spectral-norm estimate sigma used by newton_schulz_init (synchronises). */
rb_status rbfgs_sigma(rbfgs_t h, double *sigma);

/*
 * The same power-iteration estimate of ||A||_2 as newton_schulz_init, for
 * callers that cannot allocate device memory: services that fix their
 * device-memory plan at start-up (cudaMalloc can synchronise the device and
 * fragment a pool an outer allocator owns) or code whose framework allocator
 * must own every byte.  The paper has no counterpart; this is a library
 * convenience.  Allocates nothing: its scratch (two n-vectors and a scalar)
 * lives in a static device array of the library, 1 MiB per device that loads
 * the library, held until the process exits.
 *   n, A_dev, lda, a_is_fp64: the SPD matrix (device pointer, column-major).
 *   power_iters: iterations from v0 = 1/sqrt(n) (0 = 100), as for
 *   newton_schulz_init.  *sigma_out receives ||A v|| after the last one.
 * n > 65536 is rejected with RB_EINVAL.  Every call looks up the scratch's
 * device address (cudaGetSymbolAddress) in the context current on the calling
 * thread, so a device reset or a switch of context is safe; the first call in
 * a context also loads the library's device code there, so make it before any
 * stream capture.  All calls share the one scratch array: calls that overlap
 * on the GPU (other streams, other host threads) race.  Synchronises the
 * stream.
 */
rb_status rbfgs_sigma_noalloc(int n, const void *A_dev, int64_t lda, int a_is_fp64, int power_iters,
                              double *sigma_out, void *stream);

/*
 * Host-buffer entry points (the end-to-end path of a caller whose data is in
 * host memory).  rbfgs_load_host copies a new A from A_host (ld lda, FP32 or
 * FP64 elements) into an existing RBFGS/AdaRBFGS handle of the same n and
 * restarts it (X0 = I or L0 = I, k = 0, status cleared); asynchronous, so
 * A_host must stay valid until the next synchronising call.
 * rbfgs_export_host copies X (X = L L^T for AdaRBFGS) or L into out_host
 * (storage type, ld); synchronises.
 */
rb_status rbfgs_load_host(rbfgs_t h, const void *A_host, int64_t lda, int a_is_fp64);
rb_status rbfgs_export_host(rbfgs_t h, int what, void *out_host, int64_t ld);

/*
 * Run ONE step of the handle's method with a CUDA event recorded on its
 * stream at every phase boundary (sketch draw, each n x n pass, q x q core,
 * update).  ms[i] gets the device time of phase i and names[i] (if names is
 * not NULL) its name, for i < *nphases <= cap.  Entries whose name starts
 * with '@' follow the phases: they mark the end of work on the internal side
 * streams (the q x q cores) as the time from the start of the step.  The
 * step is a real step: it advances the iterate and k.  Synchronises.
 */
rb_status rbfgs_profile_step(rbfgs_t h, double *ms, const char **names, int cap, int *nphases);

/*
 * Restart an RBFGS/AdaRBFGS handle on the same A: X0 = I or L0 = I, k = 0,
 * status cleared, new sketch seed and stream.  Asynchronous.
 */
rb_status rbfgs_reset(rbfgs_t h, uint64_t seed, uint64_t stream_id);

/*
 * Failure-path check of the bounded device-side waits (no counterpart in the
 * paper).  Every mbarrier wait in this library's tensor-core kernels gives up
 * after a fixed number of SM cycles (about two seconds), records the failure
 * in the handle's device status word and lets the kernel return instead of
 * hanging the GPU.  This call queues, on the handle's stream, one small kernel
 * that waits on a barrier nothing ever completes (it issues no copy and no
 * MMA, so nothing is left in flight) with a limit of limit_cycles SM cycles
 * (1 .. 2^32).  The wait runs out and marks the handle failed: later steps
 * leave the iterate untouched and the next synchronising call returns
 * RB_ETIMEOUT.  Asynchronous.  Errors: RB_EINVAL.
 */
rb_status rbfgs_wait_selftest(rbfgs_t h, int64_t limit_cycles);

/* Number of kernels this library has launched since it was loaded. */
rb_status rbfgs_launch_count(uint64_t *count);

rb_status rbfgs_destroy(rbfgs_t h);

/*
 * Batched RBFGS: many SPD problems of uneven size (n_i <= 1024), each with
 * X0 = I and the trace-weighted coordinate-block sketch of q_i coordinates
 * (q_i in {4, 8, ..., 32}, a multiple of 4), Philox key `seed` and counter
 * stream stream_ids[i] (NULL: i), exactly as an rbfgs_init handle with
 * RB_SKETCH_COORD_TRACE would draw them.  Storage FP32, the q x q Cholesky in
 * FP64.  The blocks are a fixed partition, so every block's Cholesky factor and
 * Lambda = A[C, C]^-1 are formed once, at creation (FP64, Lambda kept in FP32);
 * a step that draws a block whose factorisation broke down (pivot <= 0 or
 * non-finite) fails its problem with RB_ENOTSPD and leaves its iterate
 * untouched.  All problems advance in one persistent launch: CTAs pull problems
 * from a device work queue (largest n first) and run the requested steps
 * on each; every problem is processed by one CTA in a fixed order, so its
 * iterates do not depend on the rest of the batch.  The round (steps, then a
 * sampled residual per problem) is captured as a CUDA graph and replayed.
 * A_dev[i] are device pointers (ld lda[i]) copied at creation.
 */
typedef struct rb_batch *rb_batch_t;
rb_status rb_batch_create(rb_batch_t *b, int count, const int *n, const void *const *A_dev, const int64_t *lda,
                          int a_is_fp64, const int *q, const uint64_t *stream_ids, uint64_t seed, void *stream);
/* `steps` steps on every active problem (synchronises). */
rb_status rb_batch_step(rb_batch_t b, int steps);
/* Sampled residual ||I - X_i A_i||_F / sqrt(n_i) of every problem from ncols <= 64
 * Floyd-sampled columns (key col_seed, counter stream i); out has count entries. */
rb_status rb_batch_residual(rb_batch_t b, int ncols, uint64_t col_seed, double *out);
/* Steps in rounds of check_every until each problem's sampled residual is <= tol (it
 * then stops), it fails (RB_ENOTSPD in status[i]) or max_iter steps are done.
 * iters/resid/status have count entries; returns RB_OK when all converged. */
rb_status rb_batch_solve(rb_batch_t b, double tol, int max_iter, int check_every, int ncols, int *iters,
                         double *resid, int *status, int *nconverged);
/* X_i into out_dev (FP32, ld >= n_i); asynchronous. */
rb_status rb_batch_export(rb_batch_t b, int i, void *out_dev, int64_t ld);
/* Tile shape of the step kernel: threads per CTA, 256 or 512 (NMAX / threads rows of
 * a problem per thread).  rb_batch_create picks it with an autotuner: the first batch
 * for a key (largest n rounded up to a power of two, largest q, precision) times two
 * steps of its problems with each shape, keeps the faster (the trial steps are undone)
 * and caches the choice for later batches of the same key.  Every sum runs in an order
 * that does not depend on the shape, so the iterates are the same for either;
 * rb_batch_set_tile overrides the choice. */
rb_status rb_batch_tile(rb_batch_t b, int *threads_per_cta);
rb_status rb_batch_set_tile(rb_batch_t b, int threads_per_cta);
rb_status rb_batch_destroy(rb_batch_t b);

/*
 * Serving loop with continuous batching (AdaRBFGS, Gaussian sketch).
 * rb_srv_create starts a scheduler thread on the current device.  Each request
 * runs in the server's form `prec`, except that a BF16 form serves only
 * tolerances >= 1e-4 (smaller ones run in RB_MIXED): its products leave a
 * residual floor near 2e-5.  A request whose sampled residual has not fallen
 * by 10 % over 8 check_every steps is finished as floor-limited (RB_NOTCONV with
 * floor_limited = 1): every FP32-storage form stops falling near a floor set by
 * its rounding (measured: ~3e-6 FP32, ~7e-6 3xTF32 at n / q = 64), so smaller
 * tolerances are not reachable in them.  Each
 * submitted request (an SPD A, tol, seed; q = 0 picks 32 round(sqrt(n)/32),
 * at least 32) waits in a FIFO queue until its device footprint
 * (rbfgs_footprint, plus a staging copy when A is in host memory) fits in
 * hbm_budget_bytes and fewer than max_live requests are running; it then
 * gets its own handle and stream, advances check_every steps at a time with
 * non-blocking residual checks of check_cols sampled columns, and finishes
 * when the residual is <= tol, after max_iter steps (RB_NOTCONV) or on a
 * failure.  At the finish its factor L (FP32, ld ldo) is copied to `out`
 * (device or host per out_on_device; NULL = discard) and its memory is
 * released, which admits the next queued requests.  A and out must stay
 * valid until the request is reported done.  A request's iterates depend
 * only on its own (A, q, seed), not on the other requests in flight.
 */
typedef struct rb_srv *rb_srv_t;
typedef struct {
    int64_t ticket;
    int32_t status;   /* RB_OK, RB_NOTCONV or an error */
    int32_t iters;
    double resid;     /* last sampled residual */
    double latency_s; /* submit -> done */
    double queue_s;   /* submit -> admitted */
    int32_t n, q;
    int32_t prec;          /* the form the request ran in */
    int32_t floor_limited; /* 1: stopped above tol because the residual stopped falling (RB_NOTCONV;
                              resid is then the floor its arithmetic reached) */
} rb_srv_result;
typedef struct {
    int32_t completed, failed, queued, live;
    double p50_s, p99_s;  /* latency percentiles of finished requests */
    double solves_per_s;  /* completed / (last finish - first submit) */
    uint64_t hbm_in_use;  /* admitted footprint */
} rb_srv_summary;
rb_status rb_srv_create(rb_srv_t *s, size_t hbm_budget_bytes, int max_live, int prec, int check_every,
                        int check_cols, int max_iter);
/* RB_ENOMEM when the request alone exceeds the budget. */
rb_status rb_srv_submit(rb_srv_t s, int n, const void *A, int a_on_device, int64_t lda, int a_is_fp64, double tol,
                        uint64_t seed, int q, void *out, int out_on_device, int64_t ldo, int64_t *ticket);
rb_status rb_srv_poll(rb_srv_t s, int64_t ticket, int *done);
/* Blocks until the request is done (RB_ETIMEOUT after timeout_s), fills *res and
 * retires the ticket. */
rb_status rb_srv_wait(rb_srv_t s, int64_t ticket, double timeout_s, rb_srv_result *res);
rb_status rb_srv_stats(rb_srv_t s, rb_srv_summary *stats);
/* Finishes every submitted request, then stops the scheduler. */
rb_status rb_srv_destroy(rb_srv_t s);

const char *rbfgs_status_string(int status);

#ifdef __cplusplus
}
#endif

#endif /* RBFGS_H */
