// selftest.cu -- a self-test of the bounded device waits the rollouts and
// the tensor-core contraction use: one warp waits on an mbarrier whose
// expected bytes never arrive (nothing copies into it), so the wait can only
// end by giving up at its time limit; the kernel then reports that and
// returns, and the context stays usable.
#include <chrono>

#include "rollout_common.cuh"

namespace mtp {
namespace {

__global__ void k_wait_selftest(uint64_t limit_ns, uint32_t* out) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) {
    const unsigned b = (unsigned)__cvta_generic_to_shared(&bar);
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(b) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    // the one arrival, expecting 16 bytes that no copy will deliver
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], 16;" ::"r"(b) : "memory");
  }
  __syncwarp();
  const bool done = mbar_wait_bounded(&bar, 0u, limit_ns);
  if (threadIdx.x == 0) out[0] = done ? 1u : 2u;
}

}  // namespace
}  // namespace mtp

extern "C" mtp_status mtp_selftest_bounded_wait(double limit_s, double* waited_s) {
  if (!(limit_s > 0.0) || limit_s > 10.0)
    return MTP_ERR_INVALID_ARG;
  uint32_t* d_out = nullptr;
  if (cudaMalloc(&d_out, sizeof(uint32_t)) != cudaSuccess) return MTP_ERR_OUT_OF_MEMORY;
  cudaMemset(d_out, 0, sizeof(uint32_t));
  const auto t0 = std::chrono::steady_clock::now();
  mtp::k_wait_selftest<<<1, 32>>>((uint64_t)(limit_s * 1e9), d_out);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  const auto t1 = std::chrono::steady_clock::now();
  uint32_t out = 0;
  if (e == cudaSuccess) e = cudaMemcpy(&out, d_out, sizeof(uint32_t), cudaMemcpyDeviceToHost);
  cudaFree(d_out);
  if (waited_s) *waited_s = std::chrono::duration<double>(t1 - t0).count();
  if (e != cudaSuccess) return MTP_ERR_CUDA;
  return out == 2u ? MTP_ERR_TIMEOUT : (out == 1u ? MTP_OK : MTP_ERR_CUDA);
}
