// noalloc.cu -- spectral-norm estimate for callers that must not allocate
// device memory.
//
// newton_schulz_init estimates sigma = ||A||_2 with scratch it allocates
// (two n-vectors and one scalar).  Some callers cannot allocate: services
// that fix their device-memory plan at start-up (cudaMalloc can synchronise
// the whole device and fragment a pool that an outer allocator owns), or
// code running under a framework whose allocator must own every byte.
// rbfgs_sigma_noalloc runs the same power iteration with its scratch in the
// file-scope array below instead.  That array is part of the library image:
// every GPU that loads this library holds it until the process exits.
#include "kernels.cuh"

// Largest n accepted by rbfgs_sigma_noalloc.
constexpr int RB_NOALLOC_MAX_N = 65536;

// Scratch of the power iteration: v (n doubles), w (n doubles), sigma (1).
// 2 * 65536 * 8 + 8 bytes = 1 MiB + 8 B on every device that loads the library.
static __device__ __align__(256) double g_noalloc_scratch[2 * RB_NOALLOC_MAX_N + 2];

namespace {

// Device address of g_noalloc_scratch in the CUDA context current on this
// thread.  A __device__ array belongs to a context, not to a device ordinal:
// after cudaDeviceReset, or under a non-primary context, an address cached per
// device could point into memory that is no longer this array.  So it is
// looked up on every call; cudaGetSymbolAddress allocates nothing.
rb_status scratch_for_current_context(double **out)
{
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || p == nullptr) {
        cudaGetLastError();
        return RB_ECUDA;
    }
    *out = (double *)p;
    return RB_OK;
}

}  // namespace

extern "C" rb_status rbfgs_sigma_noalloc(int n, const void *A_dev, int64_t lda, int a_is_fp64, int power_iters,
                                         double *sigma_out, void *stream)
{
    if (!A_dev || !sigma_out || n < 1 || lda < n) return RB_EINVAL;
    if (n > RB_NOALLOC_MAX_N) return RB_EINVAL;  // beyond the static scratch
    double *scratch = nullptr;
    RB_TRY(scratch_for_current_context(&scratch));
    double *v = scratch, *w = scratch + RB_NOALLOC_MAX_N, *sig = scratch + 2 * RB_NOALLOC_MAX_N;
    cudaStream_t st = (cudaStream_t)stream;
    const int iters = power_iters > 0 ? power_iters : 100;
    // v is re-initialised and w, sigma fully rewritten by the iteration, so no
    // state from an earlier call is read.
    if (a_is_fp64)
        launch_power_iteration<double>(st, n, (const double *)A_dev, lda, iters, v, w, sig);
    else
        launch_power_iteration<float>(st, n, (const float *)A_dev, lda, iters, v, w, sig);
    RB_CUDA(cudaGetLastError());
    double s = 0.0;
    RB_CUDA(cudaMemcpyAsync(&s, sig, sizeof(double), cudaMemcpyDeviceToHost, st));
    RB_CUDA(cudaStreamSynchronize(st));
    *sigma_out = s;
    return RB_OK;
}
