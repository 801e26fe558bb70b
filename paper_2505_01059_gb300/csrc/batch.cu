// batch.cu -- packing kernels of the batched planner: the packed start
// states are scattered to each instance's x0 buffer before an iteration and
// every instance's u* is gathered into one packed output after it.
#include "mtp_device.cuh"

namespace mtp {
namespace {

// one block per instance; off has count + 1 entries
__global__ void k_scatter(const float* __restrict__ packed, float* const* __restrict__ dst,
                          const int* __restrict__ off) {
  const int i = blockIdx.x;
  const int n = off[i + 1] - off[i];
  for (int e = threadIdx.x; e < n; e += blockDim.x) dst[i][e] = packed[off[i] + e];
}

__global__ void k_gather(const float* const* __restrict__ src, const int* __restrict__ off,
                         float* __restrict__ packed) {
  const int i = blockIdx.x;
  const int n = off[i + 1] - off[i];
  for (int e = threadIdx.x; e < n; e += blockDim.x) packed[off[i] + e] = src[i][e];
}

}  // namespace

cudaError_t launch_scatter(const float* packed, float* const* d_dst, const int* d_off, int count,
                           cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  k_scatter<<<count, 64, 0, s>>>(packed, d_dst, d_off);
  return cudaGetLastError();
}

cudaError_t launch_gather(const float* const* d_src, const int* d_off, float* packed, int count,
                          cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  k_gather<<<count, 64, 0, s>>>(d_src, d_off, packed);
  return cudaGetLastError();
}

}  // namespace mtp
