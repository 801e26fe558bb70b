// rollout_common.cuh -- helpers shared by the rollout kernels: compile-time
// loops, packed lower-triangle indexing, the per-model randomisation scales,
// reduced-range sine / cosine and the batch row -> instance lookup.
#pragma once

#include "mtp_device.cuh"

namespace mtp {
namespace {

// Control steps requested ahead of use by the point-mass and chain rollouts.
// Measured on GB300 (depths 1 / 2 / 3 / 4): a lone instance, which has one
// warp per SM sub-partition at most, is fastest at 2 (7-link arm 118 / 105 /
// 105 / 109 us per step); a batch, where registers set how many warps are
// resident, at 1 (256 instances 4.06 / 4.16 / 4.25 / 4.37 ms per iteration).
constexpr int kPrefetchAlone = 2;
constexpr int kPrefetchBatch = 1;

// Compile-time loop: calls f(IC<i>) for i in [B, E), so every array index
// derived from i is a constant and the arrays stay in registers.
template <int V>
struct IC {
  static constexpr int value = V;
};
template <int B, int E>
struct Unroll {
  template <class F>
  static __device__ __forceinline__ void run(F&& f) {
    if constexpr (B < E) {
      f(IC<B>{});
      Unroll<B + 1, E>::run(f);
    }
  }
};

// Model scales of slots 0..S-1 for one model unit, four slots per generator
// call (the same words draw() returns one at a time).
template <int S>
__device__ __forceinline__ void dr_scales(const RolloutArgs& a, uint32_t iter, uint32_t unit,
                                          float (&out)[S]) {
  if (a.dr_mode == MTP_DR_NONE) {
#pragma unroll
    for (int j = 0; j < S; ++j) out[j] = 1.f;
    return;
  }
  const uint32_t tag = (a.dr_mode == MTP_DR_SHARED) ? kTagParamModel : kTagParamSample;
  const float span = a.dr_hi - a.dr_lo;
#pragma unroll
  for (int g = 0; g < (S + 3) / 4; ++g) {
    const uint4 r = philox(make_uint4(unit, (uint32_t)g, iter, tag), a.key);
    const uint32_t w[4] = {r.x, r.y, r.z, r.w};
#pragma unroll
    for (int q = 0; q < 4; ++q)
      if (4 * g + q < S) out[4 * g + q] = fmaf(span, unit24(w[q]), a.dr_lo);
  }
}

// sin and cos of an absolute link angle: Cody-Waite reduction of x by 2 pi
// (a two-term split of 2 pi) to [-pi, pi], then the SFU sine / cosine, whose
// absolute error on that interval is about 4e-7.
__device__ __forceinline__ void sincos_reduced(float x, float* s, float* c) {
  const float k = rintf(x * 0.15915494309189535f);
  float r = fmaf(-k, 6.28318548202514648f, x);
  r = fmaf(-k, -1.7484556e-07f, r);
  __sincosf(r, s, c);
}

// Asynchronous 4-byte global-to-shared copy (cp.async, cached at L1), its
// commit, and the wait for all of the thread's committed copies.
__device__ __forceinline__ void copy_async_f32(float* smem_dst, const float* gmem_src) {
  const unsigned dst = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(dst), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void copy_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void copy_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

template <int NL>
struct Tri {
  static constexpr int size = NL * (NL + 1) / 2;
  static __device__ __forceinline__ constexpr int at(int i, int j) { return i * (i + 1) / 2 + j; }
};

// Instance of global row g in a batch: row_start (count + 1 entries) holds
// each instance's first row, rows padded to whole warps.
__device__ __forceinline__ int batch_instance(const int* __restrict__ row_start, int count, int g) {
  int lo = 0, hi = count;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (__ldg(row_start + mid) <= g) lo = mid;
    else hi = mid;
  }
  return lo;
}

}  // namespace
}  // namespace mtp
