// rollout_pm.cu -- launcher of the standalone k-D point-mass rollout, with
// direct or staged control loads (rollout_kernels.cuh).
#include "rollout_kernels.cuh"

namespace mtp {
namespace {

constexpr int kMaxPmAxes = 16;

template <int K, int T>
cudaError_t pm_launch(const RolloutArgs& a, const PointMassModel& m, cudaStream_t s) {
  const int bd = rollout_block(a.rows);
  k_rollout_pm<K, T><<<(a.rows + bd - 1) / bd, bd, staged_smem<K, T>(bd), s>>>(a, m);
  return cudaGetLastError();
}

template <int K>
cudaError_t pm_dispatch(const RolloutArgs& a, const PointMassModel& m, int k, int chunk,
                        cudaStream_t s) {
  if constexpr (K <= kMaxPmAxes) {
    if (k == K) {
      if (chunk == 8) return pm_launch<K, 8>(a, m, s);
      if (chunk == 4) return pm_launch<K, 4>(a, m, s);
      return pm_launch<K, 0>(a, m, s);
    }
    return pm_dispatch<K + 1>(a, m, k, chunk, s);
  } else {
    return cudaErrorInvalidValue;
  }
}

template <int K>
cudaError_t pm_attributes() {
  if constexpr (K <= kMaxPmAxes) {
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(k_rollout_pm<K, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)staged_smem<K, 4>(kThreads))) ||
        (e = cudaFuncSetAttribute(k_rollout_pm<K, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)staged_smem<K, 8>(kThreads))))
      return e;
    return pm_attributes<K + 1>();
  } else {
    return cudaSuccess;
  }
}

}  // namespace

cudaError_t init_rollout_pm_attributes() { return pm_attributes<1>(); }

cudaError_t launch_rollout_pointmass(const RolloutArgs& a, const PointMassModel& m, int chunk,
                                     cudaStream_t s) {
  if (a.rows <= 0) return cudaSuccess;
  if (!can_stage(a, a.n)) chunk = 0;
  return pm_dispatch<1>(a, m, a.n, chunk, s);
}

}  // namespace mtp
