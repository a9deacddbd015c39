// selftest.cu -- failure-path check of the bounded mbarrier waits that every
// tcgen05 / TMA kernel of this library uses.
//
// k_wait_selftest runs the same bounded wait on an mbarrier that nothing ever
// completes: it has issued no TMA copy and no MMA and holds no tensor memory,
// so when the wait gives up there is nothing in flight to drain.  The wait
// records ST_TIMEOUT in the status word it is given and the kernel returns,
// exactly as a real kernel's timed-out wait does; the context stays usable.
#include "kernels.cuh"
#include "tc_ptx.cuh"

namespace {

__global__ void k_wait_selftest(long long limit_cycles, int *status)
{
    __shared__ __align__(8) uint64_t bar;
    __shared__ int abort_flag;
    using namespace tcx;
    if (threadIdx.x == 0) {
        mbar_init(smem_u32(&bar), 1);
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    // one expected arrival that never comes: phase 0 never completes
    mbar_wait_for(smem_u32(&bar), 0, status, (volatile int *)&abort_flag, limit_cycles);
}

}  // namespace

extern "C" rb_status rbfgs_wait_selftest(rbfgs_t h, int64_t limit_cycles)
{
    if (!h || limit_cycles < 1 || limit_cycles > (1ll << 32)) return RB_EINVAL;
    int *status = nullptr;
    cudaStream_t st = nullptr;
    rb_handle_status(h, &status, &st);
    rb_count_launch();
    k_wait_selftest<<<1, 32, 0, st>>>((long long)limit_cycles, status);
    RB_CUDA(cudaGetLastError());
    return RB_OK;
}
