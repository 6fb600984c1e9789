// Failure-detection self-test on the device. The bounded mbarrier waits of the
// tensor-core SDNet kernel (mf_wait.cuh) run here against a phase that nothing ever
// completes: every wait must give up after its limit, record the timeout in the device
// status word and return, and the host must read MF_ERR_TIMEOUT from that word exactly
// as mf_sweep does, with the CUDA context left usable. Nothing traps, asserts or faults.
#include <cuda_runtime.h>

#include <string>

#include "../../include/mosaicflow.h"
#include "mf_internal.cuh"
#include "mf_wait.cuh"

namespace mf {
void set_last_error(const std::string& msg);
}

namespace {

// 64 threads: in warp 0, lanes 0-15 use the spinning wait and lanes 16-31 the spinning
// wait that sleeps between polls (both also stop on the CTA abort flag); warp 1 uses the
// try_wait form that ignores the abort flag and runs to its own limit.
__global__ void wait_timeout_kernel(unsigned long long limit_ns, int* status, int* gave_up) {
  __shared__ __align__(8) unsigned long long bar_word;
  __shared__ int abort_word;
  const uint32_t bar = (uint32_t)__cvta_generic_to_shared(&bar_word);
  if (threadIdx.x == 0) {
    mf::mbar_init(bar, 1);  // one expected arrival, which never comes
    abort_word = 0;
  }
  __syncthreads();
  volatile int* abort_flag = &abort_word;
  bool ok;
  if (threadIdx.x < 16) ok = mf::wait_spin(bar, 0, abort_flag, status, limit_ns);
  else if (threadIdx.x < 32) ok = mf::wait_nap_inl(bar, 0, abort_flag, status, limit_ns);
  else ok = mf::wait_bounded(bar, 0, abort_flag, status, false, limit_ns);
  if (!ok) atomicAdd(gave_up, 1);
}

}  // namespace

extern "C" mf_status mf_check_wait_timeout(double limit_ms, int* waits_gave_up) {
  if (!(limit_ms > 0.0 && limit_ms <= 1000.0)) {
    mf::set_last_error("mf_check_wait_timeout: limit_ms must be in (0, 1000]");
    return MF_ERR_INVALID_ARG;
  }
  int* d = nullptr;
  cudaError_t e = cudaMalloc(&d, 2 * sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(d, 0, 2 * sizeof(int));
  if (e == cudaSuccess) {
    wait_timeout_kernel<<<1, 64>>>((unsigned long long)(limit_ms * 1e6), d, d + 1);
    e = cudaGetLastError();
  }
  int h[2] = {0, 0};
  if (e == cudaSuccess) e = cudaMemcpy(h, d, sizeof(h), cudaMemcpyDeviceToHost);
  if (d) cudaFree(d);
  if (e != cudaSuccess) {
    mf::set_last_error(std::string("mf_check_wait_timeout: ") + cudaGetErrorString(e));
    return MF_ERR_CUDA;
  }
  if (waits_gave_up) *waits_gave_up = h[1];
  if (h[0] != mf::kDevErrNone) {
    mf::set_last_error("mf_check_wait_timeout: a kernel wait timed out (expected)");
    return MF_ERR_TIMEOUT;
  }
  return MF_OK;
}
