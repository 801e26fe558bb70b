// rollout_pm_batch.cu -- launcher of the batched k-D point-mass rollout (one
// launch over many instances of one dimension), with direct or staged control
// loads (rollout_kernels.cuh).
#include "rollout_kernels.cuh"

namespace mtp {
namespace {

constexpr int kMaxPmAxes = 16;

template <int K, int T>
cudaError_t pm_batch_launch(const RolloutArgs* ra, const PointMassModel* pm, const int* row_start,
                            int count, int total_rows, int block, cudaStream_t s) {
  k_rollout_pm_batch<K, T><<<(total_rows + block - 1) / block, block, staged_smem<K, T>(block), s>>>(
      ra, pm, row_start, count);
  return cudaGetLastError();
}

template <int K>
cudaError_t pm_batch_dispatch(const RolloutArgs* ra, const PointMassModel* pm, const int* row_start,
                              int count, int total_rows, int k, int block, int chunk, int samples,
                              cudaStream_t s) {
  if constexpr (K <= kMaxPmAxes) {
    if (k == K) {
      if (samples == 2) {
        const int threads = total_rows / 2;  // rows are padded to 64 per instance
        k_rollout_pm_batch2<K><<<(threads + block - 1) / block, block, 0, s>>>(ra, pm, row_start, count);
        return cudaGetLastError();
      }
      if (chunk == 8) return pm_batch_launch<K, 8>(ra, pm, row_start, count, total_rows, block, s);
      if (chunk == 4) return pm_batch_launch<K, 4>(ra, pm, row_start, count, total_rows, block, s);
      return pm_batch_launch<K, 0>(ra, pm, row_start, count, total_rows, block, s);
    }
    return pm_batch_dispatch<K + 1>(ra, pm, row_start, count, total_rows, k, block, chunk, samples, s);
  } else {
    return cudaErrorInvalidValue;
  }
}

template <int K>
cudaError_t pm_batch_attributes() {
  if constexpr (K <= kMaxPmAxes) {
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(k_rollout_pm_batch<K, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)staged_smem<K, 4>(kThreads))) ||
        (e = cudaFuncSetAttribute(k_rollout_pm_batch<K, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)staged_smem<K, 8>(kThreads))))
      return e;
    return pm_batch_attributes<K + 1>();
  } else {
    return cudaSuccess;
  }
}

}  // namespace

cudaError_t init_rollout_pm_batch_attributes() { return pm_batch_attributes<1>(); }

cudaError_t launch_rollout_pointmass_batch(const RolloutArgs* d_ra, const PointMassModel* d_pm,
                                           const int* d_row_start, int count, int total_rows,
                                           int k, int block, int chunk, int samples, cudaStream_t s) {
  if (total_rows <= 0) return cudaSuccess;
  return pm_batch_dispatch<1>(d_ra, d_pm, d_row_start, count, total_rows, k, block, chunk, samples, s);
}

}  // namespace mtp
