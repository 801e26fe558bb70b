// candidates.cu -- Alg. 2 sampling: the random multipartite graph (Def. 1),
// path sampling (Alg. 1), interpolation (Def. 2 / Def. 3 / straight lines),
// local Gaussian samples and the nominal-mean row, all written into the
// (B, H, n) candidate tensor in one launch.
//
// Blocks [0, graph_blocks) each produce `paths_per_block` graph paths: the
// block regenerates the whole graph Z in shared memory from Philox (it is a
// pure function of (seed, iteration), a few KB, cheaper to recompute than to
// synchronise across blocks), draws its paths' layer indices, gathers the
// waypoints and interpolates them with coalesced row-major stores.  The other
// blocks stream the local Gaussian rows and the mean row, four elements per
// generator call.
#include <cuda_bf16.h>

#include "mtp_device.cuh"

namespace mtp {
namespace {

constexpr int kThreads = 256;
constexpr int kPrepThreads = 1024;

// Eq. 6 with the end rules stated under it, 0-based knot a of M knots.
// slope(j) is the slope of piece j (between knots j and j+1).
template <class SlopeFn>
__device__ __forceinline__ float akima_knot_slope(int a, int M, SlopeFn slope) {
  if (M == 2) return slope(0);
  if (a == 0) return slope(0);
  if (a == M - 1) return slope(M - 2);
  if (a == 1) return 0.5f * (slope(0) + slope(1));
  if (a == M - 2) return 0.5f * (slope(M - 2) + slope(M - 3));
  const float mm2 = slope(a - 2), mm1 = slope(a - 1), m0 = slope(a), mp1 = slope(a + 1);
  const float w1 = fabsf(mp1 - m0), w2 = fabsf(mm1 - mm2);
  if (w1 + w2 == 0.f) return 0.5f * (mm1 + m0);
  return (w1 * mm1 + w2 * m0) / (w1 + w2);
}

// Standard normal pair by Box-Muller from two 32-bit words.  The angle
// 2 pi u2 is evaluated as pi + x with x = 2 pi (u2 - 1/2) in [-pi, pi), where
// the SFU sine / cosine have absolute error about 4e-7; the radius keeps the
// accurate logarithm because it is ill-conditioned for u1 near 1.  Its
// square root is r2 * rsqrt(r2) (a few ulp; r2 = 0 when u1 = 1).
__device__ __forceinline__ void box_muller(uint32_t w0, uint32_t w1, float& e0, float& e1) {
  const float u1 = (float)((w0 >> 8) + 1u) * 5.9604644775390625e-8f;  // (0, 1]
  const float u2 = (float)(w1 >> 8) * 5.9604644775390625e-8f;         // [0, 1)
  const float r2 = -2.f * logf(u1);
  const float radius = r2 > 0.f ? r2 * rsqrtf(r2) : 0.f;
  float sn, cs;
  __sincosf(6.28318530717958648f * (u2 - 0.5f), &sn, &cs);
  e0 = -radius * cs;
  e1 = -radius * sn;
}

// The control box copied to shared memory once per block: reading it from
// the kernel parameters with a run-time dimension index goes through the
// constant cache's indexed path, whose throughput bounded the whole kernel.
__device__ __forceinline__ void stage_box(const CandArgs& a, float* lo, float* hi) {
  for (int i = threadIdx.x; i < a.dm.n; i += blockDim.x) {
    lo[i] = a.umin[i];
    hi[i] = a.umax[i];
  }
  __syncthreads();
}

// Local rows (Alg. 2 local sampling) and the mean row: block `lb` of
// `nlb` blocks given to them; mu + sigma * eps, four elements of a row per
// generator call.  MODE (LocalMode) selects whether the draws, the finished
// samples from stored draws, or both in one pass are made.  Each thread
// keeps one group q of four consecutive (t, i) elements and walks rows
// q-group by q-group with a fixed row stride, so the group's mean, spread
// and box bounds are loaded once.
template <int MODE>
__device__ __forceinline__ void local_rows_body(const CandArgs& a, int lb, int nlb) {
  __shared__ float box_lo[MTP_MAX_CTRL], box_hi[MTP_MAX_CTRL];
  stage_box(a, box_lo, box_hi);
  const Dims dm = a.dm;
  const uint32_t iter = (a.d_iter ? *a.d_iter : a.iter) + a.iter_offset;
  const int n = dm.n;
  const int Hn = dm.H * n;
  const int G = (Hn + 3) >> 2;
  // the arguments read once into registers: the loops' stores would
  // otherwise make the compiler reload them (they may alias the arguments)
  const int local_rows = a.local_rows;
  float* __restrict__ const U_local = a.U_local;
  float* __restrict__ const U_mean = a.U_mean;
  const float* __restrict__ const mu = a.mu;
  const float* __restrict__ const sigma = a.sigma;
  const Key key = a.key;
  const int rows = local_rows + ((MODE != kLocalNoise && U_mean) ? 1 : 0);  // + the mean row
  // whole 16-byte groups: one vector load of mu and sigma and one vector
  // store per generator call (rows of a 16-byte aligned tensor stay aligned)
  const bool vec = (Hn & 3) == 0 &&
                   ((reinterpret_cast<uintptr_t>(U_local) | reinterpret_cast<uintptr_t>(mu) |
                     reinterpret_cast<uintptr_t>(sigma)) & 15) == 0;
  // threads [0, RS * QS): q-groups t % QS, t % QS + QS, ...; rows t / QS,
  // t / QS + RS, ... (QS = G when there are at least G threads)
  const int T = nlb * blockDim.x;
  const int t = lb * blockDim.x + threadIdx.x;
  const int QS = T >= G ? G : T;
  const int RS = T / QS;
  if (t >= RS * QS) return;
  for (int q = t % QS; q < G; q += QS) {
    float mv[4], sv[4], lo[4], hi[4];
    int i = (4 * q) % n;  // dimension of the group's first element; the next ones step from it
#pragma unroll
    for (int w = 0; w < 4; ++w) {
      const int el = 4 * q + w;
      lo[w] = box_lo[i];
      hi[w] = box_hi[i];
      i = i + 1 == n ? 0 : i + 1;
      mv[w] = el < Hn ? mu[el] : 0.f;
      sv[w] = el < Hn ? sigma[el] : 0.f;
    }
    for (int row = t / QS; row < rows; row += RS) {
      if (row < local_rows) {
        float* dst = U_local + (size_t)row * Hn;
        float eps[4];
        if constexpr (MODE == kLocalFinish) {
          if (vec) {
            const float4 e4 = reinterpret_cast<const float4*>(dst)[q];
            eps[0] = e4.x;
            eps[1] = e4.y;
            eps[2] = e4.z;
            eps[3] = e4.w;
          } else {
#pragma unroll
            for (int w = 0; w < 4; ++w) eps[w] = (4 * q + w < Hn) ? dst[4 * q + w] : 0.f;
          }
        } else {
          const uint4 r = philox(make_uint4((uint32_t)row, (uint32_t)q, iter, kTagLocal), key);
          box_muller(r.x, r.y, eps[0], eps[1]);
          box_muller(r.z, r.w, eps[2], eps[3]);
        }
        float o[4];
#pragma unroll
        for (int w = 0; w < 4; ++w)
          o[w] = MODE == kLocalNoise ? eps[w] : clamp_box(fmaf(sv[w], eps[w], mv[w]), lo[w], hi[w]);
        if (vec) {
          reinterpret_cast<float4*>(dst)[q] = make_float4(o[0], o[1], o[2], o[3]);
        } else {
#pragma unroll
          for (int w = 0; w < 4; ++w)
            if (4 * q + w < Hn) dst[4 * q + w] = o[w];
        }
      } else {
#pragma unroll
        for (int w = 0; w < 4; ++w) {
          const int el = 4 * q + w;
          if (el < Hn) U_mean[el] = clamp_box(mv[w], lo[w], hi[w]);
        }
      }
    }
  }
}

// Def. 1: Z[m][j][:] uniform over the box, four dimensions per call, written
// by the whole block into Z (shared memory).
__device__ __forceinline__ void regenerate_Z(const CandArgs& a, float* Z, uint32_t iter,
                                             const float* box_lo, const float* box_hi) {
  const int M = a.dm.M, N = a.dm.N, n = a.dm.n;
  const int ng = (n + 3) >> 2;
  for (int e = threadIdx.x; e < M * N * ng; e += blockDim.x) {
    const int node = e / ng, g = e - node * ng;
    const uint4 r = philox(make_uint4((uint32_t)node, (uint32_t)g, iter, kTagGraph), a.key);
#pragma unroll
    for (int w = 0; w < 4; ++w) {
      const int i = 4 * g + w;
      if (i < n) Z[node * n + i] = fmaf(box_hi[i] - box_lo[i], unit24(pick(r, w)), box_lo[i]);
    }
  }
}

template <int V>
struct Int {
  static constexpr int value = V;
};

// Clamped stores of `total` interpolated elements of consecutive rows,
// u = f(path, t, i), coalesced over (t, i); each thread's (path, t, i)
// position advances by a fixed stride, so it is carried along instead of
// divided out.
template <class F>
__device__ __forceinline__ void store_rows(const CandArgs& a, float* __restrict__ out, int total, const float* box_lo,
                                           const float* box_hi, F f) {
  const int H = a.dm.H, n = a.dm.n, Hn = H * n;
  int e = threadIdx.x;
  int sp = e / Hn, rem = e - sp * Hn;
  int t = rem / n, i = rem - t * n;
  const int ds = blockDim.x / Hn, drem = blockDim.x - ds * Hn;
  const int dt = drem / n, di = drem - dt * n;
  for (; e < total; e += blockDim.x) {
    out[e] = clamp_box(f(sp, t, i), box_lo[i], box_hi[i]);
    sp += ds;
    t += dt;
    i += di;
    if (i >= n) {
      i -= n;
      ++t;
    }
    if (t >= H) {
      t -= H;
      ++sp;
    }
  }
}

// Graph rows of graph block `bid` (Alg. 1 and the interpolation): its paths'
// layer indices, their waypoints gathered from the graph Zs (shared or
// global memory) into C (shared memory, followed by the Akima scratch), and
// the interpolated, clamped rows.  Every path is computed on its own, so the
// grouping of paths into blocks does not change any value.
__device__ __forceinline__ void graph_paths_body(const CandArgs& a, const float* Zs, float* C,
                                                 int bid, uint32_t iter, const float* box_lo,
                                                 const float* box_hi) {
  const Dims dm = a.dm;
  const int H = dm.H, n = dm.n, M = dm.M, N = dm.N;
  const int Hn = H * n;
  const int SPB = a.paths_per_block;
  const int b0 = bid * SPB;
  const int nb = min(SPB, a.graph_rows - b0);
  float* coef = C + SPB * M * n;
  if (a.C_in == nullptr) {
    // Alg. 1: layer indices with replacement, then C = Z[m][I[b][m]][:].
    const int mg = (M + 3) >> 2;
    for (int e = threadIdx.x; e < nb * mg; e += blockDim.x) {
      const int s = e / mg, g = e - s * mg;
      const uint4 r = philox(make_uint4((uint32_t)(b0 + s), (uint32_t)g, iter, kTagPath), a.key);
#pragma unroll
      for (int w = 0; w < 4; ++w) {
        const int m = 4 * g + w;
        if (m < M) {
          const int j = index_of(pick(r, w), (uint32_t)N);
          const float* src = Zs + (m * N + j) * n;
          float* dst = C + (s * M + m) * n;
          for (int i = 0; i < n; ++i) dst[i] = src[i];
        }
      }
    }
  } else {
    const float* src = a.C_in + (size_t)b0 * M * n;
    for (int e = threadIdx.x; e < nb * M * n; e += blockDim.x) C[e] = src[e];
  }
  __syncthreads();
  if (a.bf16 && a.interp == MTP_INTERP_BSPLINE) {
    // BF16 operands: each knot rounded to the nearest bfloat16 (ties to
    // even); its products with the BF16 basis are exact in FP32
    for (int e = threadIdx.x; e < nb * M * n; e += blockDim.x)
      C[e] = __bfloat162float(__float2bfloat16_rn(C[e]));
    __syncthreads();
  }

  if (a.interp == MTP_INTERP_AKIMA) {
    // Eqs. 6-7, one thread per (path, dimension) row walking its knots in
    // order: piece slopes m, knot slopes s, then piece coefficients
    // (a, b, c, d).  The row's slopes are its own thread's, so the passes
    // need no barrier between them (and no division of a flat index).
    const float inv_h = a.inv_h;
    const int K1 = M - 1;
    float* mslope = coef + (size_t)SPB * n * K1 * 4;  // (nb, n, M-1)
    float* kslope = mslope + (size_t)SPB * n * K1;    // (nb, n, M)
    int sp = threadIdx.x / n;
    const int i = threadIdx.x - sp * n;
    const int rows_per_pass = blockDim.x / n;  // whole paths per pass of the block
    for (; sp < nb && threadIdx.x < rows_per_pass * n; sp += rows_per_pass) {
      const int si = sp * n + i;
      const float* z = C + sp * M * n + i;
      float* m = mslope + si * K1;
      float* ks = kslope + si * M;
      for (int k = 0; k < K1; ++k) m[k] = (z[(k + 1) * n] - z[k * n]) * inv_h;
      for (int k = 0; k < M; ++k) ks[k] = akima_knot_slope(k, M, [&](int j) { return m[j]; });
      for (int k = 0; k < K1; ++k) {
        const float mk = m[k];
        const float s_left = ks[k], s_right = ks[k + 1];
        float* cf = coef + ((size_t)si * K1 + k) * 4;
        cf[0] = z[k * n];
        cf[1] = s_left;
        cf[2] = (3.f * mk - 2.f * s_left - s_right) * inv_h;
        cf[3] = (s_left + s_right - 2.f * mk) * (inv_h * inv_h);
      }
    }
    __syncthreads();
  }

  // Interpolate and store rows b0 .. b0+nb-1 (coalesced over (t, i)),
  // with the interpolation kind (and the B-spline degree) fixed at compile
  // time so the per-element sum is unrolled.  The tables' addresses are
  // read into registers first: the stores would otherwise make the compiler
  // reload them from the arguments for every element.
  float* __restrict__ const out = a.U_graph + (size_t)b0 * Hn;
  const int32_t* __restrict__ const bfirst = a.bfirst;
  const float* __restrict__ const basis = a.basis;
  const int32_t* __restrict__ const seg = a.seg;
  const float* __restrict__ const delta = a.delta;
  const float inv_h_t = a.inv_h;
  const int total = nb * Hn;
  if (a.interp == MTP_INTERP_BSPLINE) {
    // Def. 2: sum over the (p+1)-wide non-zero window of basis row t.
    auto bspline = [&](auto D) {
      store_rows(a, out, total, box_lo, box_hi, [&](int sp, int t, int i) {
        constexpr int deg = decltype(D)::value;
        const int f = bfirst[t];
        const float* brow = basis + (size_t)t * M;
        const float* zc = C + sp * M * n + i;
        float u = 0.f;
#pragma unroll
        for (int q = 0; q <= deg; ++q) {
          const int m = f + q;
          if (m < M) u = fmaf(brow[m], zc[m * n], u);
        }
        return u;
      });
    };
    switch (a.degree) {
      case 0: bspline(Int<0>{}); break;
      case 1: bspline(Int<1>{}); break;
      case 2: bspline(Int<2>{}); break;
      case 3: bspline(Int<3>{}); break;
      case 4: bspline(Int<4>{}); break;
      case 5: bspline(Int<5>{}); break;
      case 6: bspline(Int<6>{}); break;
      default: bspline(Int<7>{}); break;
    }
  } else if (a.interp == MTP_INTERP_AKIMA) {
    store_rows(a, out, total, box_lo, box_hi, [&](int sp, int t, int i) {
      const int k = seg[t];
      const float dl = delta[t];
      const float* cf = coef + ((size_t)(sp * n + i) * (M - 1) + k) * 4;
      return fmaf(fmaf(fmaf(cf[3], dl, cf[2]), dl, cf[1]), dl, cf[0]);
    });
  } else {
    store_rows(a, out, total, box_lo, box_hi, [&](int sp, int t, int i) {
      const int k = seg[t];
      const float w = fminf(delta[t] * inv_h_t, 1.f);
      const float z0 = C[(sp * M + k) * n + i], z1 = C[(sp * M + k + 1) * n + i];
      return fmaf(w, z1 - z0, z0);
    });
  }
}

// One block of candidate generation for one planning problem: block `bid`
// of `nblocks` blocks that instance is given (graph blocks first).
__device__ __forceinline__ void candidates_body(const CandArgs& a, float* smem, int bid,
                                                int nblocks) {
  if (bid < a.graph_blocks) {
    __shared__ float box_lo[MTP_MAX_CTRL], box_hi[MTP_MAX_CTRL];
    stage_box(a, box_lo, box_hi);
    const uint32_t iter = (a.d_iter ? *a.d_iter : a.iter) + a.iter_offset;
    float* Z = smem;
    float* C = Z + ((a.C_in || a.Z_global) ? 0 : a.dm.M * a.dm.N * a.dm.n);
    const float* Zs = a.Z_global;
    if (a.C_in == nullptr && Zs == nullptr) {
      regenerate_Z(a, Z, iter, box_lo, box_hi);
      __syncthreads();
      Zs = Z;
    }
    graph_paths_body(a, Zs, C, bid, iter, box_lo, box_hi);
    return;
  }
  local_rows_body<kLocalFull>(a, bid - a.graph_blocks, nblocks - a.graph_blocks);
}

__global__ void __launch_bounds__(kThreads, 5) k_candidates(const CandArgs a) {
  extern __shared__ float smem[];
  candidates_body(a, smem, blockIdx.x, gridDim.x);
}

// Many planning problems in one launch: block_start (count + 1 entries)
// gives each instance's first block; each block copies its instance's
// arguments into shared memory and runs the same body.
__global__ void __launch_bounds__(kThreads) k_candidates_batch(const CandArgs* __restrict__ args,
                                                               const int* __restrict__ block_start,
                                                               int count) {
  extern __shared__ float smem[];
  __shared__ CandArgs sa;
  const int blk = block_start[0] + (int)blockIdx.x;  // block_start holds absolute block numbers
  int lo = 0, hi = count;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (block_start[mid] <= blk) lo = mid;
    else hi = mid;
  }
  const int* src = reinterpret_cast<const int*>(args + lo);
  int* dst = reinterpret_cast<int*>(&sa);
  for (int w = threadIdx.x; w < (int)(sizeof(CandArgs) / sizeof(int)); w += blockDim.x) dst[w] = src[w];
  __syncthreads();
  candidates_body(sa, smem, blk - block_start[lo], block_start[lo + 1] - block_start[lo]);
}

// Local rows of many planning problems (no shared memory, so the blocks
// pack densely); local_start (count + 1 entries) gives each instance's
// first local block.
__global__ void __launch_bounds__(kThreads) k_local_batch(const CandArgs* __restrict__ args,
                                                          const int* __restrict__ local_start,
                                                          int count) {
  const int blk = local_start[0] + (int)blockIdx.x;  // local_start holds absolute block numbers
  int lo = 0, hi = count;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (local_start[mid] <= blk) lo = mid;
    else hi = mid;
  }
  local_rows_body<kLocalFull>(args[lo], blk - local_start[lo], local_start[lo + 1] - local_start[lo]);
}

// Def. 1: the graph Z of the current iteration written to global memory,
// block `blk` of `nblk` given to it, four dimensions per generator call.
__device__ __forceinline__ void graph_Z_body(const CandArgs& a, float* Z, int blk, int nblk) {
  __shared__ float box_lo[MTP_MAX_CTRL], box_hi[MTP_MAX_CTRL];
  stage_box(a, box_lo, box_hi);
  const int M = a.dm.M, N = a.dm.N, n = a.dm.n;
  const uint32_t iter = (a.d_iter ? *a.d_iter : a.iter) + a.iter_offset;
  const int ng = (n + 3) >> 2;
  for (int e = blk * blockDim.x + threadIdx.x; e < M * N * ng; e += nblk * blockDim.x) {
    const int node = e / ng, g = e - node * ng;
    const uint4 r = philox(make_uint4((uint32_t)node, (uint32_t)g, iter, kTagGraph), a.key);
#pragma unroll
    for (int w = 0; w < 4; ++w) {
      const int i = 4 * g + w;
      if (i < n) Z[node * n + i] = fmaf(box_hi[i] - box_lo[i], unit24(pick(r, w)), box_lo[i]);
    }
  }
}

// One planning problem whose graph is too large to regenerate in every
// block's shared memory: Z once per iteration, its graph blocks gather from it.
__global__ void __launch_bounds__(kThreads) k_graph_Z(const CandArgs a, float* Z) {
  graph_Z_body(a, Z, blockIdx.x, gridDim.x);
}

// Def. 1 for many planning problems: each instance's graph Z for its
// current iteration, written once to global memory so that its graph
// blocks gather from it instead of regenerating it.
__global__ void __launch_bounds__(kThreads) k_graph_Z_batch(const CandArgs* __restrict__ args,
                                                            float* const* __restrict__ Zs,
                                                            const int* __restrict__ block_start,
                                                            int count) {
  const int blk = block_start[0] + (int)blockIdx.x;  // block_start holds absolute block numbers
  int lo = 0, hi = count;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (block_start[mid] <= blk) lo = mid;
    else hi = mid;
  }
  graph_Z_body(args[lo], Zs[lo], blk - block_start[lo], block_start[lo + 1] - block_start[lo]);
}

// The next iteration's candidates, made while the current iteration's
// rollout runs: `gridDim.x` persistent blocks, each on an SM of its own (the
// launch asks for the whole of an SM's shared memory, so no block of another
// kernel can share the SM and slow that kernel's warps).  Each block makes
// the graph Z of iteration d_iter + iter_offset once in shared memory, then
// the graph rows of graph blocks blockIdx.x, blockIdx.x + gridDim.x, ...,
// then (when U_local is set) its grid-stride share of the local rows'
// standard normal draws.  The mean and spread are not read: the finishing
// pass applies them once they are known.
__global__ void __launch_bounds__(kPrepThreads, 1) k_prepare(const CandArgs a) {
  extern __shared__ float smem[];
  if (a.graph_blocks > 0) {
    __shared__ float box_lo[MTP_MAX_CTRL], box_hi[MTP_MAX_CTRL];
    stage_box(a, box_lo, box_hi);
    const uint32_t iter = (a.d_iter ? *a.d_iter : a.iter) + a.iter_offset;
    float* Z = smem;
    regenerate_Z(a, Z, iter, box_lo, box_hi);
    float* C = Z + a.dm.M * a.dm.N * a.dm.n;
    for (int vb = blockIdx.x; vb < a.graph_blocks; vb += gridDim.x) {
      __syncthreads();  // Z complete; the previous paths' scratch no longer read
      graph_paths_body(a, Z, C, vb, iter, box_lo, box_hi);
    }
  }
  if (a.U_local && a.local_rows > 0) local_rows_body<kLocalNoise>(a, blockIdx.x, gridDim.x);
}

// Asks the L2 to fetch [p, p + bytes) from device memory; no data comes back
// to the SM.  p and bytes are multiples of 16.
__device__ __forceinline__ void prefetch_l2_bulk(const void* p, uint32_t bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

// The local rows and the mean row of an iteration whose graph rows were
// made during the previous one: from their stored draws, clamp(mu + sigma *
// eps) (local_mode kLocalFinish), or drawn here (kLocalFull).  The graph
// rows, possibly evicted from L2 since they were made, are prefetched back
// into L2 for the rollout that follows (16 KB per request, the 16-byte
// aligned interior of the rows).
__global__ void __launch_bounds__(kThreads) k_finish(const CandArgs a) {
  if (threadIdx.x == 0 && a.U_graph && a.graph_rows > 0) {
    const uintptr_t b = reinterpret_cast<uintptr_t>(a.U_graph);
    const uintptr_t lo = (b + 15) & ~uintptr_t(15);
    const uintptr_t hi = (b + (size_t)a.graph_rows * a.dm.H * a.dm.n * sizeof(float)) & ~uintptr_t(15);
    constexpr uintptr_t kChunk = 16384;
    for (uintptr_t p = lo + (uintptr_t)blockIdx.x * kChunk; p < hi; p += (uintptr_t)gridDim.x * kChunk)
      prefetch_l2_bulk(reinterpret_cast<const void*>(p), (uint32_t)(hi - p < kChunk ? hi - p : kChunk));
  }
  if (a.local_mode == kLocalFinish) local_rows_body<kLocalFinish>(a, blockIdx.x, gridDim.x);
  else local_rows_body<kLocalFull>(a, blockIdx.x, gridDim.x);
}

// Def. 1 / Alg. 1 outputs for inspection: Z, I and C written to global memory.
__global__ void k_sample_tensor(Dims dm, Key key, uint32_t iter, CandArgs box, float* Z,
                                int32_t* I, float* C) {
  const int n = dm.n, M = dm.M, N = dm.N, P = dm.P;
  const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long stride = (long long)gridDim.x * blockDim.x;
  if (Z)
    for (long long e = tid; e < (long long)M * N * n; e += stride) {
      const int node = (int)(e / n), i = (int)(e - (long long)node * n);
      Z[e] = fmaf(box.umax[i] - box.umin[i], unit24(draw(key, node, i, iter, kTagGraph)),
                  box.umin[i]);
    }
  if (I)
    for (long long e = tid; e < (long long)P * M; e += stride) {
      const int b = (int)(e / M), m = (int)(e - (long long)b * M);
      I[e] = index_of(draw(key, b, m, iter, kTagPath), (uint32_t)N);
    }
  if (C)
    for (long long e = tid; e < (long long)P * M * n; e += stride) {
      const int bm = (int)(e / n), i = (int)(e - (long long)bm * n);
      const int b = bm / M, m = bm - b * M;
      const int j = index_of(draw(key, b, m, iter, kTagPath), (uint32_t)N);
      C[e] = fmaf(box.umax[i] - box.umin[i], unit24(draw(key, m * N + j, i, iter, kTagGraph)),
                  box.umin[i]);
    }
}

}  // namespace

size_t candidates_smem_bytes(const CandArgs& a) {
  const Dims& d = a.dm;
  size_t f = 0;
  if (a.graph_blocks > 0) {
    if (!a.C_in && !a.Z_global) f += (size_t)d.M * d.N * d.n;
    f += (size_t)a.paths_per_block * d.M * d.n;
    if (a.interp == MTP_INTERP_AKIMA)  // coefficients, piece slopes, knot slopes
      f += (size_t)a.paths_per_block * d.n * ((d.M - 1) * 5 + d.M);
  }
  return f * sizeof(float);
}

// Opt in to large dynamic shared memory on the current device (called by
// mtp_create, outside any stream capture).
cudaError_t init_candidate_attributes() {
  cudaError_t e = cudaFuncSetAttribute(k_candidates, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       200 * 1024);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_candidates_batch, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              200 * 1024);
}

cudaError_t launch_candidates_batch(const CandArgs* d_args, const int* d_block_start, int count,
                                    int total_blocks, size_t smem, cudaStream_t s) {
  if (total_blocks <= 0) return cudaSuccess;
  k_candidates_batch<<<total_blocks, kThreads, smem, s>>>(d_args, d_block_start, count);
  return cudaGetLastError();
}

cudaError_t launch_candidates(const CandArgs& a, int local_blocks, cudaStream_t s) {
  const int grid = a.graph_blocks + local_blocks;
  if (grid <= 0) return cudaSuccess;
  k_candidates<<<grid, kThreads, candidates_smem_bytes(a), s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_graph_Z(const CandArgs& a, float* Z, cudaStream_t s) {
  const int items = a.dm.M * a.dm.N * ((a.dm.n + 3) / 4);
  int blocks = (items + kThreads - 1) / kThreads;
  if (blocks > device_sms()) blocks = device_sms();
  if (blocks <= 0) return cudaSuccess;
  k_graph_Z<<<blocks, kThreads, 0, s>>>(a, Z);
  return cudaGetLastError();
}

size_t prepare_smem_need(const CandArgs& a) {
  const Dims& d = a.dm;
  size_t f = 0;
  if (a.graph_blocks > 0) {
    f += (size_t)d.M * d.N * d.n + (size_t)a.paths_per_block * d.M * d.n;
    if (a.interp == MTP_INTERP_AKIMA)
      f += (size_t)a.paths_per_block * d.n * ((d.M - 1) * 5 + d.M);
  }
  return f * sizeof(float);
}

// The dynamic shared memory that makes one k_prepare block fill an SM: the
// per-block opt-in limit less the kernel's static shared memory.
cudaError_t init_prepare_attributes(size_t* dyn_smem) {
  int dev = 0, optin = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev)) != cudaSuccess)
    return e;
  cudaFuncAttributes fa{};
  if ((e = cudaFuncGetAttributes(&fa, k_prepare)) != cudaSuccess) return e;
  const size_t dyn = (size_t)optin > fa.sharedSizeBytes ? (size_t)optin - fa.sharedSizeBytes : 0;
  if ((e = cudaFuncSetAttribute(k_prepare, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn)) !=
      cudaSuccess)
    return e;
  *dyn_smem = dyn;
  return cudaSuccess;
}

cudaError_t launch_prepare(const CandArgs& a, int grid, size_t dyn_smem, cudaStream_t s) {
  if (grid <= 0) return cudaSuccess;
  k_prepare<<<grid, kPrepThreads, dyn_smem, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_finish(const CandArgs& a, int blocks, cudaStream_t s) {
  if (blocks <= 0) return cudaSuccess;
  k_finish<<<blocks, kThreads, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_local_batch(const CandArgs* d_args, const int* d_local_start, int count,
                               int total_blocks, cudaStream_t s) {
  if (total_blocks <= 0) return cudaSuccess;
  k_local_batch<<<total_blocks, kThreads, 0, s>>>(d_args, d_local_start, count);
  return cudaGetLastError();
}

cudaError_t launch_graph_Z_batch(const CandArgs* d_args, float* const* d_Z, const int* d_block_start,
                                 int count, int total_blocks, cudaStream_t s) {
  if (total_blocks <= 0) return cudaSuccess;
  k_graph_Z_batch<<<total_blocks, kThreads, 0, s>>>(d_args, d_Z, d_block_start, count);
  return cudaGetLastError();
}

cudaError_t launch_sample_tensor(const Dims& dm, Key key, uint32_t iter, const float* umin,
                                 const float* umax, float* Z, int32_t* I, float* C,
                                 cudaStream_t s) {
  CandArgs box{};
  for (int i = 0; i < dm.n; ++i) {
    box.umin[i] = umin[i];
    box.umax[i] = umax[i];
  }
  long long work = (long long)dm.M * dm.N * dm.n;
  work = work > (long long)dm.P * dm.M * dm.n ? work : (long long)dm.P * dm.M * dm.n;
  int grid = (int)((work + 255) / 256);
  if (grid > 4096) grid = 4096;
  if (grid < 1) grid = 1;
  k_sample_tensor<<<grid, 256, 0, s>>>(dm, key, iter, box, Z, I, C);
  return cudaGetLastError();
}

}  // namespace mtp
