// rollout_chain.cu -- launcher of the standalone planar-chain rollout, with
// direct or staged control loads (rollout_kernels.cuh).  Chains stage 4
// steps at a time: their long step bodies need no longer chunks to hide the
// copies.
#include "rollout_kernels.cuh"

namespace mtp {
namespace {

constexpr int kMaxChainLinks = 12;

template <int NL, int T>
cudaError_t chain_launch(const RolloutArgs& a, const ChainModel& m, cudaStream_t s) {
  const int bd = rollout_block(a.rows);
  k_rollout_chain<NL, T><<<(a.rows + bd - 1) / bd, bd, staged_smem<NL, T>(bd), s>>>(a, m);
  return cudaGetLastError();
}

template <int NL>
cudaError_t chain_dispatch(const RolloutArgs& a, const ChainModel& m, int links, int chunk,
                           cudaStream_t s) {
  if constexpr (NL <= kMaxChainLinks) {
    if (links == NL) return chunk ? chain_launch<NL, 4>(a, m, s) : chain_launch<NL, 0>(a, m, s);
    return chain_dispatch<NL + 1>(a, m, links, chunk, s);
  } else {
    return cudaErrorInvalidValue;
  }
}

template <int NL>
cudaError_t chain_attributes() {
  if constexpr (NL <= kMaxChainLinks) {
    cudaError_t e = cudaFuncSetAttribute(k_rollout_chain<NL, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)staged_smem<NL, 4>(kThreads));
    if (e != cudaSuccess) return e;
    return chain_attributes<NL + 1>();
  } else {
    return cudaSuccess;
  }
}

}  // namespace

cudaError_t init_rollout_chain_attributes() { return chain_attributes<1>(); }

cudaError_t launch_rollout_chain(const RolloutArgs& a, const ChainModel& m, int links, int chunk,
                                 cudaStream_t s) {
  if (a.rows <= 0) return cudaSuccess;
  if (!can_stage(a, links)) chunk = 0;
  return chain_dispatch<1>(a, m, links, chunk, s);
}

int rollout_blocks(int rows) {
  if (rows <= 0) return 0;
  const int bd = rollout_block(rows);
  return (rows + bd - 1) / bd;
}

}  // namespace mtp
