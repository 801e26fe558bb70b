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

// ---------------------------------------------------------------------------
// Staged control rows.  A rollout thread reads its candidate's controls one
// step after another; a warp's 32 lanes read 32 different rows, H * n floats
// apart, so each direct warp load touches 32 cache lines (measured: 31
// sectors per request and the L1 at 83-93 % of its throughput in the batched
// 7-link and 9-axis rollouts, whose issue slots were 44 % and 22 % busy).
// Staged instead, each warp's rows pass through shared memory a horizon
// chunk of T steps at a time: lane l issues one bulk copy (cp.async.bulk,
// the TMA engine's untiled form) of row l's next T * K floats, an mbarrier
// per buffer counts the bytes, and two buffers alternate so that chunk c + 1
// arrives while chunk c is used.  A bulk copy needs 16-byte aligned source,
// destination and size: the host stages only rows whose base is 16-byte
// aligned and whose length H * K is a multiple of 4 floats, with T a
// multiple of 4, so every chunk start and length is a multiple of 16 bytes.
// The row stride in shared memory is a multiple of 4 floats with an odd
// quotient, so that the lanes' 16-byte row starts fall in distinct bank
// quads (a scalar read is then a 4-way conflict, against 32 lines per direct
// warp load).
// ---------------------------------------------------------------------------
template <int K, int T>
struct StageShape {
  static_assert(T % 4 == 0, "chunks must be whole 16-byte units");
  static constexpr int kRow = T * K;
  static constexpr int kQuads = (kRow + 3) / 4;
  static constexpr int kStride = 4 * (kQuads % 2 ? kQuads : kQuads + 1);  // floats
  static constexpr int kBuf = 32 * kStride;                                 // floats per buffer
  static constexpr size_t kWarpBytes = 2 * kBuf * sizeof(float) + 16;       // + two mbarriers
};

// Bounded mbarrier wait: try_wait on the phase with the given parity for at
// most limit_ns of the global timer (about two seconds by default), then
// give up (returns false).
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity,
                                                  uint64_t limit_ns = 2000000000ull) {
  const unsigned addr = (unsigned)__cvta_generic_to_shared(bar);
  uint64_t t_start = 0;
  for (int spin = 0;; ++spin) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n"
        " mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(addr), "r"(parity)
        : "memory");
    if (done) return true;
    uint64_t now;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(now));
    if (spin == 0) t_start = now;
    else if (now - t_start > limit_ns) return false;
  }
}

// The two mbarriers of a warp's staging, initialised by one lane.
__device__ __forceinline__ void init_stage_bars(uint64_t* bars) {
  if ((threadIdx.x & 31) == 0) {
    const unsigned b0 = (unsigned)__cvta_generic_to_shared(bars);
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(b0) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(b0 + 8) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncwarp();
}

template <int K, int T>
struct StagedRows {
  using Shape = StageShape<K, T>;
  float* buf;        // [2][32][kStride]
  uint64_t* bar;     // [2]
  const float* row;  // this lane's row (null when the lane has no candidate)
  int H, chunks;
  int seq;           // chunks consumed so far (buffer and phase of the next one)
  uint32_t live;     // lanes with a candidate
  int lane;

  // `smem` is this warp's kWarpBytes of shared memory (16-byte aligned).
  // Every lane of the warp calls it.
  __device__ __forceinline__ void init(unsigned char* smem, const float* my_row, int H_) {
    buf = reinterpret_cast<float*>(smem);
    bar = reinterpret_cast<uint64_t*>(smem + 2 * Shape::kBuf * sizeof(float));
    row = my_row;
    H = H_;
    chunks = (H + T - 1) / T;
    seq = 0;
    lane = threadIdx.x & 31;
    live = __ballot_sync(0xffffffffu, my_row != nullptr);
    if (lane == 0) {
      const unsigned b0 = (unsigned)__cvta_generic_to_shared(bar);
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(b0) : "memory");
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(b0 + 8) : "memory");
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncwarp();
  }

  // Binds this warp's next row set to barriers and buffers that the warp
  // keeps across rows of different widths: `bars` holds two mbarriers
  // initialised once (init_bars), `buffer` two buffers of at least kBuf
  // floats, and `seq_` counts the chunks this warp has consumed on those
  // barriers so far (it sets their phases).  Every lane calls it.
  __device__ __forceinline__ void attach(uint64_t* bars, float* buffer, const float* my_row, int H_,
                                         int seq_) {
    buf = buffer;
    bar = bars;
    row = my_row;
    H = H_;
    chunks = (H + T - 1) / T;
    seq = seq_;
    lane = threadIdx.x & 31;
    live = __ballot_sync(0xffffffffu, my_row != nullptr);
  }

  // Data chunk c (steps c*T ..) as the g-th chunk of this warp's sequence,
  // into buffer g & 1.  Every lane of the warp calls it; the lanes' reads of
  // that buffer's previous chunk have been consumed by then.
  __device__ __forceinline__ void issue(int c, int g) {
    __syncwarp();
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    const int t0 = c * T;
    const int steps = min(T, H - t0);
    const uint32_t bytes = (uint32_t)(steps * K * sizeof(float));
    const unsigned b = (unsigned)__cvta_generic_to_shared(bar + (g & 1));
    if (lane == 0) {
      const uint32_t total = bytes * (uint32_t)__popc(live);
      asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(b), "r"(total)
                   : "memory");
    }
    __syncwarp();
    if (row) {
      const unsigned dst = (unsigned)__cvta_generic_to_shared(buf + (g & 1) * Shape::kBuf +
                                                              lane * Shape::kStride);
      asm volatile(
          "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
          ::"r"(dst), "l"(row + (size_t)t0 * K), "r"(bytes), "r"(b)
          : "memory");
    }
  }

  // Waits for the g-th chunk (bounded); false, on every lane, when the wait
  // gave up.
  __device__ __forceinline__ bool wait(int g) {
    const bool ok = mbar_wait_bounded(bar + (g & 1), (uint32_t)((g >> 1) & 1));
    return __all_sync(0xffffffffu, ok);
  }

  // This lane's floats of the g-th chunk.
  __device__ __forceinline__ const float* chunk(int g) const {
    return buf + (g & 1) * Shape::kBuf + lane * Shape::kStride;
  }

  // After a failed wait on the g-th chunk: waits (again bounded) for the
  // copies still in flight into this warp's buffers (the g-th and, when it
  // was issued, the next) before the warp may leave.
  __device__ __forceinline__ void drain(int g, bool next_issued) {
    mbar_wait_bounded(bar + (g & 1), (uint32_t)((g >> 1) & 1));
    if (next_issued) mbar_wait_bounded(bar + ((g + 1) & 1), (uint32_t)(((g + 1) >> 1) & 1));
  }
};

// Feeds step(t, u) the K controls of every step t = 0 .. H-1 of this lane's
// candidate row Ub.  T == 0: direct loads PF steps ahead into a rotating
// register buffer (the loop is unrolled by PF so its slots are constants).
// T > 0: the warp's rows staged through shared memory by `st` (initialised
// by the caller on every lane of the warp).  Returns false when a staged wait
// gave up; the remaining steps are then skipped.
template <int K, int PF, int T, class Step>
__device__ __forceinline__ bool for_each_step(const float* Ub, int H, StagedRows<K, T>* st,
                                              Step&& step) {
  if constexpr (T == 0) {
    (void)st;
    float ubuf[PF][K];
#pragma unroll
    for (int q = 0; q < PF; ++q)
#pragma unroll
      for (int k = 0; k < K; ++k) ubuf[q][k] = __ldg(Ub + min(q, H - 1) * K + k);
    for (int t0 = 0; t0 < H; t0 += PF) {
      Unroll<0, PF>::run([&](auto Q) {
        constexpr int q = decltype(Q)::value;
        const int t = t0 + q;
        if (t < H) {
          float u[K];
          const int tn = min(t + PF, H - 1);
#pragma unroll
          for (int k = 0; k < K; ++k) {
            u[k] = ubuf[q][k];
            ubuf[q][k] = __ldg(Ub + tn * K + k);  // PF steps ahead
          }
          step(t, u);
        }
      });
    }
    return true;
  } else {
    const int chunks = st->chunks;
    const int g0 = st->seq;
    st->issue(0, g0);
    for (int c = 0; c < chunks; ++c) {
      const bool next = c + 1 < chunks;
      if (next) st->issue(c + 1, g0 + c + 1);
      if (!st->wait(g0 + c)) {
        st->drain(g0 + c, next);
        st->seq = g0 + c + 1 + (next ? 1 : 0);
        return false;
      }
      // a rolled loop over the chunk's steps: its reads need no constant
      // slots, and the step body stays one copy
      const float* src = st->chunk(g0 + c);
      const int steps = min(T, H - c * T);
#pragma unroll 1
      for (int q = 0; q < steps; ++q) {
        float u[K];
#pragma unroll
        for (int k = 0; k < K; ++k) u[k] = src[q * K + k];
        step(c * T + q, u);
      }
    }
    st->seq = g0 + chunks;
    return true;
  }
}

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
