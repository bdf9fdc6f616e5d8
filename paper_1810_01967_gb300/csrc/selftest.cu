// Self-test of the bounded device-side waits: a wait that nothing will ever satisfy gives up
// after its time bound, the kernel raises MRF_DERR_TIMEOUT and the host reports MRF_ETIMEOUT.
// Nothing else is in flight when the wait expires, so the context stays usable.
#include <string>

#include "mrf_internal.cuh"
#include "ptx.cuh"

namespace {

__global__ void k_wait_nobody(uint64_t timeout_ns, uint32_t* err) {
    __shared__ uint64_t bar;
    mrfk::mbar_init(&bar, 1);
    mrfk::fence_mbar_init();
    // phase 0 completes only when one thread arrives; none does
    if (!mrfk::mbar_wait(&bar, 0, timeout_ns)) atomicOr(err, MRF_DERR_TIMEOUT);
}

}  // namespace

extern "C" mrf_status mrf_selftest_wait_timeout(int64_t timeout_ns, void* stream) {
    if (timeout_ns < 1 || timeout_ns > 1000000000) {
        mrf_set_error("timeout_ns must be in 1 .. 1e9");
        return MRF_EINVAL;
    }
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    uint32_t* err = nullptr;
    MRF_CUDA_TRY(cudaMalloc(&err, sizeof(uint32_t)));
    uint32_t e = 0;
    cudaError_t c = cudaMemsetAsync(err, 0, sizeof(uint32_t), st);
    if (c == cudaSuccess) {
        k_wait_nobody<<<1, 1, 0, st>>>(static_cast<uint64_t>(timeout_ns), err);
        c = cudaGetLastError();
    }
    if (c == cudaSuccess) c = cudaMemcpyAsync(&e, err, sizeof(e), cudaMemcpyDeviceToHost, st);
    if (c == cudaSuccess) c = cudaStreamSynchronize(st);
    cudaFree(err);
    if (c != cudaSuccess) {
        mrf_set_error(std::string("wait self-test: ") + cudaGetErrorString(c));
        return MRF_ECUDA;
    }
    if (e & MRF_DERR_TIMEOUT) {
        mrf_set_error("a device-side wait bound expired (self-test)");
        return MRF_ETIMEOUT;
    }
    mrf_set_error("the wait self-test did not time out");
    return MRF_EINTERNAL;
}
