// rollout_persist.cu -- the rollouts of a whole batch in one persistent
// launch, or two (Alg. 2 rollout fused with the Eq. 2 cost, the bodies of
// rollout_kernels.cuh).
//
// Work items are warp tiles: 32 consecutive candidates of one instance.  The
// instances are listed group by group, the longest group first and within a
// group the longest expected rollout first (H times the time per step of the
// group's dynamics and dimension), and numbered by a prefix of their warp
// tiles, so item w belongs to the instance whose range holds w.  Each warp of
// the launch repeatedly takes the next item from a device counter (one
// atomic add per item), looks its instance up by binary search, and runs
// that tile's rollout: a point mass of K axes or a planar chain of L links,
// with direct control loads or staged 4 steps at a time.  A warp therefore
// moves between instances of different sizes and dynamics, while the warps
// running at one time mostly run the same body.  The bodies are the
// per-candidate rollouts of the other kernels (the same templates), so every
// cost is the same bits as in a per-group or standalone launch.  The
// two-launch mode of the batch runs the same kernel over two ranges of the
// entries (w_base numbers the second range's tiles).
//
// The warps never wait on one another: an item, once taken, depends only on
// the candidates generated before the launch.  A staged tile's waits are the
// bounded waits of StagedRows; a warp whose wait gave up scores its tile
// +inf, marks the instance's status word and leaves the loop.
//
// The bodies are inlined into the kernel: as separate functions their
// arguments went through a 240-byte stack frame and the launch was 7-8 %
// slower on the batch of 256.  The launch is bounded at three 128-thread
// CTAs per SM, i.e. at most 170 registers per thread (168 used, no spills).
//
// Measured on GB300 on the 256-instance batch (the bench's timed region):
// 2.68 ms per iteration with two launches, against 2.79-2.91 ms with each
// group's rollout launched in its own stream's chain.  The order of the
// tiles matters: sorted by length alone across all groups, the warps of an
// SM ran different bodies at once, half of their stall samples were
// instruction fetches, and the iteration took 3.5 ms; tiles are therefore
// taken group by group (longest group first, longest tiles first within it).
#include <map>
#include <mutex>

#include "rollout_kernels.cuh"

namespace mtp {
namespace {

constexpr int kPersistThreads = 128;
constexpr int kPersistChunk = 4;  // horizon chunk of a staged tile

// Point masses evaluate every obstacle slot without a branch (ALL): the
// slots past n_obs add exactly +0, so the bits are those of the guarded loop
// of the per-group kernel, and mixed with the chains' tiles the branch-free
// form is faster (256-instance batch 2.73 -> 2.68 ms per iteration).
template <int K, int T>
__device__ __forceinline__ bool persist_pm(const RolloutArgs& a, const PointMassModel& m, int r, bool live,
                                        uint64_t* bars, float* buf, int& seq) {
  if constexpr (T == 0) {
    (void)bars;
    (void)buf;
    (void)seq;
    if (!live) return true;
    return rollout_pm_body<K, kPrefetchBatch, true, 0>(a, m, r, true, nullptr);
  } else {
    StagedRows<K, T> st;
    st.attach(bars, buf, live ? a.U + (size_t)r * a.H * K : nullptr, a.H, seq);
    const bool ok = rollout_pm_body<K, kPrefetchBatch, true, T>(a, m, r, live, &st);
    seq = st.seq;
    return __all_sync(0xffffffffu, ok);
  }
}

template <int NL, int T>
__device__ __forceinline__ bool persist_chain(const RolloutArgs& a, const ChainModel& m, int r, bool live,
                                           uint64_t* bars, float* buf, int& seq) {
  if constexpr (T == 0) {
    (void)bars;
    (void)buf;
    (void)seq;
    if (!live) return true;
    return rollout_chain_body<NL, kPrefetchBatch, 0>(a, m, r, true, nullptr);
  } else {
    StagedRows<NL, T> st;
    st.attach(bars, buf, live ? a.U + (size_t)r * a.H * NL : nullptr, a.H, seq);
    const bool ok = rollout_chain_body<NL, kPrefetchBatch, T>(a, m, r, live, &st);
    seq = st.seq;
    return __all_sync(0xffffffffu, ok);
  }
}

template <int K>
__device__ __forceinline__ bool pm_tile(int k, bool staged, const RolloutArgs& a, const PointMassModel& m,
                                        int r, bool live, uint64_t* bars, float* buf, int& seq) {
  if constexpr (K <= kPersistMaxAxes) {
    if (k == K)
      return staged ? persist_pm<K, kPersistChunk>(a, m, r, live, bars, buf, seq)
                    : persist_pm<K, 0>(a, m, r, live, bars, buf, seq);
    return pm_tile<K + 1>(k, staged, a, m, r, live, bars, buf, seq);
  } else {
    return false;
  }
}

template <int NL>
__device__ __forceinline__ bool chain_tile(int links, bool staged, const RolloutArgs& a, const ChainModel& m,
                                           int r, bool live, uint64_t* bars, float* buf, int& seq) {
  if constexpr (NL <= kPersistMaxLinks) {
    if (links == NL)
      return staged ? persist_chain<NL, kPersistChunk>(a, m, r, live, bars, buf, seq)
                    : persist_chain<NL, 0>(a, m, r, live, bars, buf, seq);
    return chain_tile<NL + 1>(links, staged, a, m, r, live, bars, buf, seq);
  } else {
    return false;
  }
}

__global__ void __launch_bounds__(kPersistThreads, 3) k_rollout_persistent(const PersistArgs p) {
  __shared__ PointMassModel models[kPersistThreads / 32];
  extern __shared__ __align__(16) unsigned char persist_smem[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  unsigned char* area = persist_smem + (size_t)warp * p.warp_bytes;
  uint64_t* bars = reinterpret_cast<uint64_t*>(area);
  float* buf = reinterpret_cast<float*>(area + 16);
  if (p.warp_bytes > 0) init_stage_bars(bars);
  int seq = 0;
  for (;;) {
    int w = 0;
    if (lane == 0) w = (int)atomicAdd(p.head, 1u);
    w = __shfl_sync(0xffffffffu, w, 0);
    if (w >= p.total_warps) break;
    w += p.w_base;
    // the instance whose warp range holds w: the last k with wstart[k] <= w
    int lo = 0, hi = p.count;
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (__ldg(p.wstart + mid) <= w) lo = mid;
      else hi = mid;
    }
    const int code = __ldg(p.code + lo);
    const int model = __ldg(p.model + lo);
    const RolloutArgs a = p.ra[__ldg(p.order + lo)];
    const int r = (w - __ldg(p.wstart + lo)) * 32 + lane;
    const bool live = r < a.rows;
    const int dim = (code >> 8) & 0xff;
    // staged only where the instance's rows allow it and this launch has
    // staging buffers (a direct-load launch has none)
    const bool staged = p.warp_bytes > 0 && (code >> 16) != 0;
    bool ok;
    if ((code & 0xff) == MTP_DYN_POINTMASS) {
      PointMassModel& m = models[warp];
      const int* src = reinterpret_cast<const int*>(p.pm + model);
      int* dst = reinterpret_cast<int*>(&m);
      for (int q = lane; q < (int)(sizeof(PointMassModel) / sizeof(int)); q += 32) dst[q] = __ldg(src + q);
      __syncwarp();
      ok = pm_tile<1>(dim, staged, a, m, r, live, bars, buf, seq);
    } else {
      const ChainModel cm = p.cm[model];
      ok = chain_tile<1>(dim, staged, a, cm, r, live, bars, buf, seq);
    }
    // the model slot and the staging buffers are reused by the next item
    __syncwarp();
    if (!__all_sync(0xffffffffu, ok)) break;
  }
}

}  // namespace

size_t persist_warp_bytes(int max_pm_axes_staged, int max_links_staged) {
  size_t f = 0;
  auto need = [&](int k) {
    const int quads = (kPersistChunk * k + 3) / 4;
    const int stride = 4 * (quads % 2 ? quads : quads + 1);
    f = std::max(f, (size_t)2 * 32 * stride);
  };
  if (max_pm_axes_staged > 0) need(max_pm_axes_staged);
  if (max_links_staged > 0) need(max_links_staged);
  return f ? 16 + f * sizeof(float) : 0;
}

int persist_blocks_per_sm(size_t warp_bytes) {
  // per device and shared-memory size, computed once: a batch refilled every
  // serving cycle asks again each time
  static std::mutex mu;
  static std::map<std::pair<int, size_t>, int> cache;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  std::lock_guard<std::mutex> lock(mu);
  auto it = cache.find({dev, warp_bytes});
  if (it != cache.end()) return it->second;
  // the attribute is the ceiling of every launch's shared memory: the
  // largest staged tile any batch can have
  const int warps = kPersistThreads / 32;
  const size_t ceiling = persist_warp_bytes(kPersistMaxAxes, kPersistMaxLinks) * warps;
  if (cudaFuncSetAttribute(k_rollout_persistent, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ceiling) !=
      cudaSuccess)
    return 0;
  int blocks = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, k_rollout_persistent, kPersistThreads,
                                                    warp_bytes * warps) != cudaSuccess)
    return 0;
  cache[{dev, warp_bytes}] = blocks;
  return blocks;
}

cudaError_t launch_rollout_persistent(const PersistArgs& p, int blocks_per_sm, cudaStream_t s) {
  if (p.total_warps <= 0) return cudaSuccess;
  const int warps_per_block = kPersistThreads / 32;
  const int grid = std::max(1, std::min(blocks_per_sm * device_sms(),
                                        (p.total_warps + warps_per_block - 1) / warps_per_block));
  cudaError_t e = cudaMemsetAsync(p.head, 0, sizeof(unsigned), s);
  if (e != cudaSuccess) return e;
  k_rollout_persistent<<<grid, kPersistThreads, p.warp_bytes * warps_per_block, s>>>(p);
  return cudaGetLastError();
}

}  // namespace mtp
