// Self-test of the bounded waits that every TMA kernel of the library uses:
// a wait whose completion never comes must run out, set the error word and
// let the kernel return, so that the host sees DDCC_ERR_TIMEOUT instead of a
// hung GPU.  The test kernel arms an mbarrier for bytes that no copy will
// deliver (nothing is in flight, so nothing can land after the kernel ends)
// and waits on it with a short poll limit; its control case arrives without
// expecting bytes and completes at once.
#include "ddcc.h"
#include "ddcc_tma.cuh"

namespace ddcc {
namespace {

__global__ void k_wait_selftest(int* __restrict__ err, int deliver, unsigned limit) {
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) {
        tma::mbar_init(&bar, 1);
        tma::mbar_init_fence();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        if (deliver)
            asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tma::smem_u32(&bar)) : "memory");
        else
            tma::mbar_expect_tx(&bar, 16);   // 16 bytes that no copy will bring
    }
    const bool ok = tma::mbar_wait_bounded(&bar, 0, limit);
    if (!__syncthreads_and(ok) && threadIdx.x == 0) atomicOr(err, 1);
}

}  // namespace
}  // namespace ddcc

extern "C" int ddcc_selftest_bounded_wait(void* cuda_stream, int* dev_flag, int deliver) {
    if (!dev_flag) return DDCC_ERR_PARAM;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    int host = 0;
    if (cudaMemsetAsync(dev_flag, 0, sizeof(int), s) != cudaSuccess) return DDCC_ERR_CUDA;
    ddcc::k_wait_selftest<<<1, 64, 0, s>>>(dev_flag, deliver ? 1 : 0, 4096u);
    if (cudaGetLastError() != cudaSuccess) return DDCC_ERR_CUDA;
    if (cudaMemcpyAsync(&host, dev_flag, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return DDCC_ERR_CUDA;
    return host ? DDCC_ERR_TIMEOUT : DDCC_OK;
}
