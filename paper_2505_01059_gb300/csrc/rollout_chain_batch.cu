// rollout_chain_batch.cu -- launcher of the batched planar-chain rollout (one
// launch over many instances of one link count), with direct or staged
// control loads (rollout_kernels.cuh; chains stage 4 steps at a time).
#include "rollout_kernels.cuh"

namespace mtp {
namespace {

constexpr int kMaxChainLinks = 12;

template <int NL, int T>
cudaError_t chain_batch_launch(const RolloutArgs* ra, const ChainModel* cm, const int* row_start,
                               int count, int total_rows, int block, cudaStream_t s) {
  k_rollout_chain_batch<NL, T><<<(total_rows + block - 1) / block, block, staged_smem<NL, T>(block),
                                 s>>>(ra, cm, row_start, count);
  return cudaGetLastError();
}

template <int NL>
cudaError_t chain_batch_dispatch(const RolloutArgs* ra, const ChainModel* cm, const int* row_start,
                                 int count, int total_rows, int links, int block, int chunk,
                                 cudaStream_t s) {
  if constexpr (NL <= kMaxChainLinks) {
    if (links == NL)
      return chunk ? chain_batch_launch<NL, 4>(ra, cm, row_start, count, total_rows, block, s)
                   : chain_batch_launch<NL, 0>(ra, cm, row_start, count, total_rows, block, s);
    return chain_batch_dispatch<NL + 1>(ra, cm, row_start, count, total_rows, links, block, chunk, s);
  } else {
    return cudaErrorInvalidValue;
  }
}

template <int NL>
cudaError_t chain_batch_attributes() {
  if constexpr (NL <= kMaxChainLinks) {
    cudaError_t e = cudaFuncSetAttribute(k_rollout_chain_batch<NL, 4>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)staged_smem<NL, 4>(kThreads));
    if (e != cudaSuccess) return e;
    return chain_batch_attributes<NL + 1>();
  } else {
    return cudaSuccess;
  }
}

}  // namespace

cudaError_t init_rollout_chain_batch_attributes() { return chain_batch_attributes<1>(); }

cudaError_t launch_rollout_chain_batch(const RolloutArgs* d_ra, const ChainModel* d_cm,
                                       const int* d_row_start, int count, int total_rows,
                                       int links, int block, int chunk, cudaStream_t s) {
  if (total_rows <= 0) return cudaSuccess;
  return chain_batch_dispatch<1>(d_ra, d_cm, d_row_start, count, total_rows, links, block, chunk, s);
}

}  // namespace mtp
