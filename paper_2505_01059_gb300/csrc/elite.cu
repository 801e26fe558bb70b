// elite.cu -- Alg. 2 elite selection and the modified CEM update.
//
// k_select (one CTA): turns the B costs into order-preserving 32-bit keys
// (NaN -> +inf, -0 -> +0), finds the E-th smallest key by a 4-pass 8-bit
// radix select over shared memory, collects the keys below it plus the
// lowest-index ties (a block scan in index order), sorts those E (key, index)
// pairs with a bitonic network and computes the softmax weights in FP64.
// k_update (many CTAs): one warp per (t, i) element reduces the weighted
// FP64 mean and spread over the elites, applies the floor and the smoothing.
#include "mtp_device.cuh"

namespace mtp {
namespace {

constexpr int kSelThreads = 1024;
constexpr size_t kSelSmemMax = 200 * 1024;  // dynamic shared memory of one selection block
constexpr int kOneBlockMax = 32768;         // above this, two stages (measured below)
constexpr int kChunkKeys = 16384;           // first-stage chunk length

__device__ __forceinline__ uint32_t order_key(float f) {
  if (isnan(f)) f = __int_as_float(0x7f800000);
  f = f + 0.f;  // -0 -> +0
  const uint32_t b = __float_as_uint(f);
  return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}

// The cost an order key stands for (NaN costs come back as +inf, -0 as +0,
// as the selection and the softmax treat them).
__device__ __forceinline__ float key_cost(uint32_t k) {
  return __uint_as_float((k & 0x80000000u) ? (k & 0x7fffffffu) : ~k);
}

__device__ __forceinline__ int next_pow2(int v) {
  int p = 1;
  while (p < v) p <<= 1;
  return p;
}

// Bins with at most this many keys end the radix passes early.
constexpr int kBoundaryMax = 64;

// Keys a thread loads together in the selection's first pass over the costs
// and in the collection of the selected keys (the histogram passes keep a
// plain loop: batched, the 7-link arm's two passes took 3.0 us instead of 2.3).
constexpr int kSelBatch = 8;

// Ascending bitonic sort of 64 values held two per lane (v0 = element lane,
// v1 = element lane + 32) in one warp.
__device__ __forceinline__ void warp_sort64(unsigned long long& v0, unsigned long long& v1, int lane) {
  for (int k = 2; k <= 64; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      if (j == 32) {  // partner is the lane's other element (k == 64, ascending)
        const unsigned long long lo = v0 < v1 ? v0 : v1, hi = v0 < v1 ? v1 : v0;
        v0 = lo;
        v1 = hi;
      } else {
        const bool lower = (lane & j) == 0;
        const unsigned long long o0 = __shfl_xor_sync(0xffffffffu, v0, j);
        const unsigned long long o1 = __shfl_xor_sync(0xffffffffu, v1, j);
        const bool up0 = (lane & k) == 0, up1 = ((lane + 32) & k) == 0;
        v0 = (lower == up0) ? (v0 < o0 ? v0 : o0) : (v0 < o0 ? o0 : v0);
        v1 = (lower == up1) ? (v1 < o1 ? v1 : o1) : (v1 < o1 ? o1 : v1);
      }
    }
  }
}

// Selection modes: kSelAll takes the B costs to the elites, weights and u*;
// kSelChunk (block c of many) takes costs [c chunk, (c+1) chunk) to their own
// top min(E, chunk) (key, index) pairs, sorted, written to pairs[c E ..]
// (the rest of its E slots padded with all-ones); kSelMerge takes those pairs
// (B = chunks * E of them) to the elites, weights and u*.  Chunks cover the
// indices in order and each chunk's pairs are sorted by (key, index), so
// among equal keys the merge's position order is the index order: the two
// stages give exactly the one-block result.
enum SelMode { kSelAll = 0, kSelChunk = 1, kSelMerge = 2 };

template <int MODE>
__device__ __forceinline__ void select_body(const SelectArgs& a, unsigned char* sm_raw) {
  const int base = MODE == kSelChunk ? (int)blockIdx.x * a.chunk : 0;
  const int B = MODE == kSelChunk ? min(a.chunk, a.B - base) : a.B;
  const int E = MODE == kSelChunk ? min(a.E, B) : a.E;
  const float* costs = a.cost + base;
  const int Bp = (B + 1) & ~1;
  uint32_t* keys = reinterpret_cast<uint32_t*>(sm_raw);
  unsigned long long* sel = reinterpret_cast<unsigned long long*>(keys + Bp);
  __shared__ uint32_t hist[512];
  __shared__ uint32_t warp_tot[32];
  __shared__ uint32_t s_digit, s_below, s_lt, s_cnt, s_nb;
  __shared__ double s_red[32];

  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  __shared__ uint32_t s_kmin[32], s_kmax[32];
  uint32_t kmin = 0xffffffffu, kmax = 0u;
  // kSelBatch costs per thread requested together: a plain loop issued one
  // L2 round trip after the other (measured on the legged workload, 16
  // costs per thread: 4.4 us for this phase)
  for (int b0 = tid; b0 < B; b0 += kSelBatch * blockDim.x) {
    uint32_t kv[kSelBatch];
    if constexpr (MODE == kSelMerge) {
#pragma unroll
      for (int j = 0; j < kSelBatch; ++j) {
        const int b = b0 + j * blockDim.x;
        kv[j] = b < B ? (uint32_t)(a.pairs[b] >> 32) : 0u;
      }
    } else {
      float cv[kSelBatch];
#pragma unroll
      for (int j = 0; j < kSelBatch; ++j) {
        const int b = b0 + j * blockDim.x;
        cv[j] = b < B ? costs[b] : 0.f;
      }
#pragma unroll
      for (int j = 0; j < kSelBatch; ++j) kv[j] = order_key(cv[j]);
    }
#pragma unroll
    for (int j = 0; j < kSelBatch; ++j) {
      const int b = b0 + j * blockDim.x;
      if (b < B) {
        const uint32_t k = kv[j];
        keys[b] = k;
        kmin = min(kmin, k);
        kmax = max(kmax, k);
      }
    }
  }
  for (int i = tid; i < 512; i += blockDim.x) hist[i] = 0;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    kmin = min(kmin, __shfl_xor_sync(0xffffffffu, kmin, o));
    kmax = max(kmax, __shfl_xor_sync(0xffffffffu, kmax, o));
  }
  if (lane == 0) {
    s_kmin[wid] = kmin;
    s_kmax[wid] = kmax;
  }
  __syncthreads();
  // every warp reduces the per-warp extremes itself (no second barrier)
  kmin = lane < (int)(blockDim.x >> 5) ? s_kmin[lane] : 0xffffffffu;
  kmax = lane < (int)(blockDim.x >> 5) ? s_kmax[lane] : 0u;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    kmin = min(kmin, __shfl_xor_sync(0xffffffffu, kmin, o));
    kmax = max(kmax, __shfl_xor_sync(0xffffffffu, kmax, o));
  }

  // Sec. 4.1 cost entropy, read as the entropy of p_b = exp(-J_b / lambda) / Z
  // over all B candidates: with d_b = J_b - J_min and w_b = exp(-d_b / lambda),
  // H = -sum_b p_b log p_b = log Z + sum_b w_b d_b / (lambda Z).  The weights
  // in FP32, their sums in FP64.
  if (MODE == kSelAll && a.entropy) {
    const float cmin = key_cost(kmin);
    const float inv_l = (float)a.inv_lambda;
    double z = 0.0, sd = 0.0;
    if (cmin < INFINITY) {
      for (int b = tid; b < B; b += blockDim.x) {
        const float d = key_cost(keys[b]) - cmin;
        const float w = expf(-d * inv_l);
        if (w > 0.f) {
          z += (double)w;
          sd += (double)w * (double)d;
        }
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      z += __shfl_xor_sync(0xffffffffu, z, o);
      sd += __shfl_xor_sync(0xffffffffu, sd, o);
    }
    __shared__ double s_z[32], s_sd[32];
    if (lane == 0) {
      s_z[wid] = z;
      s_sd[wid] = sd;
    }
    __syncthreads();
    if (tid == 0) {
      double Z = 0.0, SD = 0.0;
      for (int q = 0; q < (int)(blockDim.x >> 5); ++q) {
        Z += s_z[q];
        SD += s_sd[q];
      }
      *a.entropy = Z > 0.0 ? log(Z) + SD * a.inv_lambda / Z : (double)NAN;
    }
  }

  // radix select of the E-th smallest key (rank 1-based), 8-bit digits from
  // the highest bit where the keys differ down (the bits above it are
  // common to all keys, and a digit over them would put every key in one
  // histogram bin); two histogram buffers alternate so each pass needs only
  // two block barriers
  const int top = kmin == kmax ? 0 : 32 - __clz(kmin ^ kmax);  // bits that still differ
  const int passes = (top + 7) >> 3;
  uint32_t mask = top >= 32 ? 0u : ~((1u << top) - 1u);
  uint32_t prefix = kmin & mask;
  uint32_t rank = (uint32_t)E;
  bool boundary = false;
  for (int pass = 0; pass < passes; ++pass) {
    const int shift = max(top - 8 * (pass + 1), 0);
    const uint32_t dmask = (1u << (top - 8 * pass - shift)) - 1u;  // 8 bits, fewer at the bottom
    uint32_t* cur = hist + 256 * (pass & 1);
    uint32_t* nxt = hist + 256 * ((pass + 1) & 1);
    for (int b = tid; b < B; b += blockDim.x) {
      const uint32_t k = keys[b];
      if ((k & mask) == prefix) atomicAdd(&cur[(k >> shift) & dmask], 1u);
    }
    for (int i = tid; i < 256; i += blockDim.x) nxt[i] = 0;
    __syncthreads();
    if (wid == 0) {
      // lane l owns digits 8l .. 8l+7
      uint32_t c[8], sum = 0;
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        c[q] = cur[lane * 8 + q];
        sum += c[q];
      }
      uint32_t incl = sum;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
      }
      uint32_t run = incl - sum;
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        if (run < rank && rank <= run + c[q]) {
          s_digit = (uint32_t)(lane * 8 + q);
          s_below = run;
          s_cnt = c[q];
        }
        run += c[q];
      }
    }
    __syncthreads();
    prefix |= s_digit << shift;
    mask |= dmask << shift;
    rank -= s_below;
    if (s_cnt <= kBoundaryMax) {  // block-uniform: read after the barrier
      boundary = true;
      break;
    }
  }
  const int Ep = next_pow2(E);
  if (boundary) {
    // The bin holding the E-th key has at most kBoundaryMax keys: every key
    // below the bin is an elite, and the bin's keys are sorted by
    // (key, index) in one warp to take the `rank` still needed.
    unsigned long long* bnd = sel + Ep;
    if (tid == 0) {
      s_lt = 0;
      s_nb = 0;
    }
    __syncthreads();
    for (int b0 = tid; b0 < B; b0 += kSelBatch * blockDim.x) {
      uint32_t kv[kSelBatch];
#pragma unroll
      for (int j = 0; j < kSelBatch; ++j) {
        const int b = b0 + j * blockDim.x;
        kv[j] = b < B ? keys[b] : 0xffffffffu;
      }
#pragma unroll
      for (int j = 0; j < kSelBatch; ++j) {
        const int b = b0 + j * blockDim.x;
        if (b >= B) continue;
        const uint32_t km = kv[j] & mask;
        if (km < prefix) sel[atomicAdd(&s_lt, 1u)] = ((unsigned long long)kv[j] << 32) | (uint32_t)b;
        else if (km == prefix) bnd[atomicAdd(&s_nb, 1u)] = ((unsigned long long)kv[j] << 32) | (uint32_t)b;
      }
    }
    __syncthreads();
    if (wid == 0) {
      const int nb = (int)s_nb;
      unsigned long long v0 = lane < nb ? bnd[lane] : ~0ull;
      unsigned long long v1 = lane + 32 < nb ? bnd[lane + 32] : ~0ull;
      warp_sort64(v0, v1, lane);
      const uint32_t base = (uint32_t)E - rank;  // == s_lt
      if ((uint32_t)lane < rank) sel[base + lane] = v0;
      if ((uint32_t)(lane + 32) < rank) sel[base + lane + 32] = v1;
    }
    for (int i = E + tid; i < Ep; i += blockDim.x) sel[i] = ~0ull;
    __syncthreads();
  } else {
  const uint32_t T = prefix;       // the E-th smallest key
  const uint32_t need_eq = rank;   // how many keys equal to T are taken

  // ties at T are taken in index order: block scan of per-thread tie counts
  const int chunk = (B + blockDim.x - 1) / blockDim.x;
  const int lo = tid * chunk, hi = min(B, lo + chunk);
  uint32_t eq = 0;
  for (int b = lo; b < hi; ++b) eq += (keys[b] == T);
  uint32_t incl = eq;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t v = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += v;
  }
  if (lane == 31) warp_tot[wid] = incl;
  if (tid == 0) s_lt = 0;
  __syncthreads();
  if (wid == 0) {
    const int nw = blockDim.x >> 5;
    uint32_t v = lane < nw ? warp_tot[lane] : 0u, x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane < nw) warp_tot[lane] = x - v;  // exclusive warp offsets
  }
  __syncthreads();
  uint32_t eq_rank = warp_tot[wid] + incl - eq;
  const uint32_t n_lt = (uint32_t)E - need_eq;
  for (int b = lo; b < hi; ++b) {
    const uint32_t k = keys[b];
    if (k < T) {
      const uint32_t slot = atomicAdd(&s_lt, 1u);
      sel[slot] = ((unsigned long long)k << 32) | (uint32_t)b;
    } else if (k == T) {
      if (eq_rank < need_eq) sel[n_lt + eq_rank] = ((unsigned long long)k << 32) | (uint32_t)b;
      ++eq_rank;
    }
  }
  for (int i = E + tid; i < Ep; i += blockDim.x) sel[i] = ~0ull;
  __syncthreads();
  }

  // bitonic sort of the E selected (key, index) pairs, ascending: in the
  // registers of one warp for E <= 64, through shared memory otherwise
  if (Ep <= 64) {
    if (wid == 0) {
      unsigned long long v0 = lane < Ep ? sel[lane] : ~0ull;
      unsigned long long v1 = lane + 32 < Ep ? sel[lane + 32] : ~0ull;
      warp_sort64(v0, v1, lane);
      if (lane < Ep) sel[lane] = v0;
      if (lane + 32 < Ep) sel[lane + 32] = v1;
    }
  } else {
    for (int k = 2; k <= Ep; k <<= 1) {
      for (int j = k >> 1; j > 0; j >>= 1) {
        for (int i = tid; i < Ep; i += blockDim.x) {
          const int ixj = i ^ j;
          if (ixj > i) {
            const unsigned long long x = sel[i], y = sel[ixj];
            const bool up = (i & k) == 0;
            if ((x > y) == up) {
              sel[i] = y;
              sel[ixj] = x;
            }
          }
        }
        __syncthreads();
      }
    }
  }
  __syncthreads();

  if constexpr (MODE == kSelChunk) {
    unsigned long long* out = a.pairs + (size_t)blockIdx.x * a.E;
    for (int k = tid; k < a.E; k += blockDim.x)
      out[k] = k < E ? ((sel[k] & 0xffffffff00000000ull) | (unsigned long long)(uint32_t)(base + (int)(sel[k] & 0xffffffffu)))
                     : ~0ull;
    return;
  }
  // the candidate index of sorted entry k (a position among the pairs when merging)
  auto index_of_sel = [&](unsigned long long e) -> int {
    const int j = (int)(e & 0xffffffffu);
    if constexpr (MODE == kSelMerge) return (int)(a.pairs[j] & 0xffffffffu);
    else return j;
  };
  // u* = U[elite[0], 0, :], requested before the softmax so the load
  // overlaps it
  const int best_row = index_of_sel(sel[0]);
  if (E <= 64) {
    // One warp, elites lane and lane + 32, their costs decoded from the
    // sorted order keys (no global reload), no block barrier.  The two
    // halves are reduced separately and then added, which is the order of
    // the block-wide reduction below for the same E, so the weights are the
    // same bits either way.
    if (wid != 0) return;
    const float u_best = lane < a.n ? a.U[(size_t)best_row * a.H * a.n + lane] : 0.f;
    const double best = (double)key_cost((uint32_t)(sel[0] >> 32));
    const bool uniform = (a.update_rule == MTP_UPDATE_PLAIN_CEM) || !(best < INFINITY);
    double w[2] = {0.0, 0.0};
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int k = lane + 32 * h;
      if (k < E) {
        const unsigned long long e = sel[k];
        const int idx = index_of_sel(e);
        a.elite[k] = idx;
        if (a.elite_out) a.elite_out[k] = idx;
        const double c = (double)key_cost((uint32_t)(e >> 32));
        w[h] = uniform ? 1.0 : exp(-(c - best) * a.inv_lambda);
      }
    }
    double s0 = w[0], s1 = w[1];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      s0 += __shfl_xor_sync(0xffffffffu, s0, o);
      s1 += __shfl_xor_sync(0xffffffffu, s1, o);
    }
    const double inv_total = 1.0 / (s0 + s1);
    if (lane < E) a.weight[lane] = w[0] * inv_total;
    if (lane + 32 < E) a.weight[lane + 32] = w[1] * inv_total;
    if (lane < a.n) {
      a.ustar[lane] = u_best;
      if (a.ustar_out) a.ustar_out[lane] = u_best;
    }
    return;
  }
  const float u_best = tid < a.n ? a.U[(size_t)best_row * a.H * a.n + tid] : 0.f;
  // softmax weights over the elites (FP64), shifted by the best cost
  const double best = (double)a.cost[best_row];
  const bool uniform = (a.update_rule == MTP_UPDATE_PLAIN_CEM) || !(best < INFINITY);
  double part = 0.0;
  // elites on consecutive threads: the FP64 pipe is occupied per warp
  // instruction, so full warps do the exponentials at the least cost.  A
  // thread keeps its first weight for the normalisation (the launch gives at
  // least min(E, 1024) threads, so with E <= 1024 that is its only one).
  const int nw = blockDim.x >> 5;
  const int k0 = tid;
  double w_first = 0.0;
  for (int k = k0; k < E; k += blockDim.x) {
    const int idx = index_of_sel(sel[k]);
    a.elite[k] = idx;
    if (a.elite_out) a.elite_out[k] = idx;
    double c = (double)a.cost[idx];
    if (isnan(c)) c = INFINITY;
    const double w = uniform ? 1.0 : exp(-(c - best) * a.inv_lambda);
    if (k == k0) w_first = w;
    else a.weight[k] = w;
    part += w;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
  if (lane == 0) s_red[wid] = part;
  __syncthreads();
  if (wid == 0) {
    double v = lane < nw ? s_red[lane] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) s_red[0] = 1.0 / v;
  }
  __syncthreads();
  const double inv_total = s_red[0];
  for (int k = k0; k < E; k += blockDim.x) a.weight[k] = (k == k0 ? w_first : a.weight[k]) * inv_total;
  if (tid < a.n) {
    a.ustar[tid] = u_best;
    if (a.ustar_out) a.ustar_out[tid] = u_best;
  }
}

__global__ void __launch_bounds__(kSelThreads) k_select(const SelectArgs a) {
  extern __shared__ __align__(16) unsigned char sm_raw[];
  select_body<kSelAll>(a, sm_raw);
}

// First stage of the selection over many CTAs: block c, chunk c of the costs.
__global__ void __launch_bounds__(kSelThreads) k_select_chunks(const SelectArgs a) {
  extern __shared__ __align__(16) unsigned char sm_raw[];
  select_body<kSelChunk>(a, sm_raw);
}

// Second stage: one CTA over the chunks' pairs (a.B = chunks * E).
__global__ void __launch_bounds__(kSelThreads) k_select_merge(const SelectArgs a) {
  extern __shared__ __align__(16) unsigned char sm_raw[];
  select_body<kSelMerge>(a, sm_raw);
}

// One block per planning problem.
__global__ void __launch_bounds__(kSelThreads) k_select_batch(const SelectArgs* __restrict__ args) {
  extern __shared__ __align__(16) unsigned char sm_raw[];
  const SelectArgs a = args[blockIdx.x];
  select_body<kSelAll>(a, sm_raw);
}

// The FP64 sums over elites follow one canonical order for every launch
// shape: elite k feeds virtual lane k mod 32 (in increasing k), and the 32
// virtual lanes are combined by the butterfly o = 16, 8, 4, 2, 1.  A group of
// G physical lanes gives each lane the 32 / G virtual lanes v = sub + G j; the
// butterfly steps o >= G pair virtual lanes held by the same lane and run in
// registers, the steps o < G run as shuffles.  Every pairwise add is the same
// (a + b == b + a), so the result is bit-identical for any G.
template <int G>
__device__ __forceinline__ double canonical_sum(double (&part)[32 / G]) {
  constexpr int P = 32 / G;
#pragma unroll
  for (int o = 16; o >= G && o >= 1; o >>= 1) {
    constexpr int dummy = 0;
    (void)dummy;
    const int sj = o / G;
#pragma unroll
    for (int j = 0; j < P; ++j)
      if ((j & sj) == 0) part[j] = part[j] + part[j ^ sj];
  }
  double v = part[0];
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) v = v + __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Rounds of 32 elites whose loads the update issues together (measured on
// the C1 point mass, E 32: 1 or 2 rounds 46.1 us per plan step, 4 rounds
// 47.7; the 7-link arm, E 64, the same within 1 us for 1, 2 and 4).
constexpr int kUpdRounds = 2;

// Threads per block of the update launches.
constexpr int kUpdThreads = 128;

// The new mean and spread of element e from the sums over the elites of
// d = u - c and w d^2 (shift c), then the floor and the smoothing.
__device__ __forceinline__ void finish_element(const UpdateArgs& a, int e, double c, double S1,
                                               double S2, bool cem) {
  if (cem) {
    // Sec. 2.1 CEM update: mean and unbiased variance of the elites
    const double E = (double)a.E;
    const double m1 = c + S1 / E;
    const double ss = fmax(S2 - S1 * (S1 / E), 0.0);
    const double s1 = a.E > 1 ? sqrt(ss / (E - 1.0)) : 0.0;
    const double mn = a.alpha * a.mu[e] + (1.0 - a.alpha) * m1;
    const double sn = a.alpha * a.sigma[e] + (1.0 - a.alpha) * s1;
    a.mu[e] = mn;
    a.sigma[e] = sn;
    a.mu_f[e] = (float)mn;
    a.sigma_f[e] = (float)sn;
  } else {
    // Alg. 2: weighted mean and standard deviation (weights sum to one)
    const double m1 = c + S1;
    double s1 = sqrt(fmax(S2 - S1 * S1, 0.0));
    if (s1 < a.sigma_min) s1 = a.sigma_min;
    const double mn = m1 + a.alpha * (a.mu[e] - m1);
    const double sn = s1 + a.alpha * (a.sigma[e] - s1);
    a.mu[e] = mn;
    a.sigma[e] = sn;
    a.mu_f[e] = (float)mn;
    a.sigma_f[e] = (float)sn;
  }
}

// Groups of G lanes each own one (t, i) element.  Thread `gt` of `threads`
// threads given to one planning problem.
template <int G>
__device__ __forceinline__ void update_body(const UpdateArgs& a, int gt, int threads) {
  constexpr int P = 32 / G;
  const int sub = threadIdx.x & (G - 1);
  const int Hn = a.H * a.n;
  const bool cem = a.update_rule == MTP_UPDATE_PLAIN_CEM;
  // G == 1: thread gt owns elements gt, gt + threads, ... (no shuffles).
  // G > 1: the loop runs block-uniformly (as many sweeps as the block's first
  // group needs; groups past the end idle through the shuffles), so that
  // each sweep ends with the block's elements finished together: lane 0 of
  // each group leaves its sums in shared memory and thread s finishes group
  // s's element.  That is one stream of FP64 instructions for all of the
  // block's elements instead of one per element, with the same arithmetic.
  const int per_sweep = (G == 1) ? threads : (threads / 32) * (32 / G);
  const int first = (G == 1) ? gt : (gt / 32) * (32 / G) + (threadIdx.x & 31) / G;
  const int block_first = ((gt - (int)threadIdx.x) / 32) * (32 / G);
  const int sweeps = (G == 1) ? 0 : (Hn - block_first + per_sweep - 1) / per_sweep;
  constexpr int kGroups = G > 1 ? kUpdThreads / G : 1;
  __shared__ double sh_S1[kGroups], sh_S2[kGroups], sh_c[kGroups];
  __shared__ int sh_e[kGroups];
  for (int it = 0, e = first; (G == 1) ? (e < Hn) : (it < sweeps); ++it, e += per_sweep) {
    const bool valid = e < Hn;
    // one pass over the elites: sums of d = u - c and d^2 with the shift c =
    // the best elite's value, so that the variance S2 - S1^2 does not cancel
    // (the spread of the elites is small next to their mean late in a run)
    const double c = valid ? (double)__ldg(a.U + (size_t)__ldg(a.elite) * Hn + e) : 0.0;
    double p1[P], p2[P];
#pragma unroll
    for (int j = 0; j < P; ++j) {
      p1[j] = 0.0;
      p2[j] = 0.0;
    }
    // virtual lane v = sub + G j takes elites v, v + 32, ... in that order.
    // With few virtual lanes per thread, R rounds of 32 elites are gathered
    // at once: first all their indices, then all their rows' values and
    // weights, so a pass over the elites waits for two dependent loads
    // rather than two per round.  With many, the P gathers of one round are
    // already independent and issued together (R = 1).
    constexpr int R = P == 1 ? kUpdRounds : (P == 2 ? kUpdRounds / 2 : 1);
    if (valid) {
      if constexpr (R > 1) {
        for (int k0 = 0; k0 < a.E; k0 += 32 * R) {
          int idx[R][P];
#pragma unroll
          for (int r = 0; r < R; ++r)
#pragma unroll
            for (int j = 0; j < P; ++j) {
              const int k = k0 + 32 * r + sub + G * j;
              idx[r][j] = k < a.E ? __ldg(a.elite + k) : 0;
            }
          float uv[R][P];
          double wv[R][P];
#pragma unroll
          for (int r = 0; r < R; ++r)
#pragma unroll
            for (int j = 0; j < P; ++j) {
              const int k = k0 + 32 * r + sub + G * j;
              uv[r][j] = k < a.E ? __ldg(a.U + (size_t)idx[r][j] * Hn + e) : 0.f;
              wv[r][j] = (k < a.E && !cem) ? a.weight[k] : 1.0;
            }
#pragma unroll
          for (int r = 0; r < R; ++r)
#pragma unroll
            for (int j = 0; j < P; ++j) {
              const int k = k0 + 32 * r + sub + G * j;
              if (k < a.E) {
                const double d = (double)uv[r][j] - c;
                const double wd = cem ? d : wv[r][j] * d;
                p1[j] = p1[j] + wd;
                p2[j] = fma(wd, d, p2[j]);
              }
            }
        }
      } else {
        for (int k0 = 0; k0 < a.E; k0 += 32) {
#pragma unroll
          for (int j = 0; j < P; ++j) {
            const int k = k0 + sub + G * j;
            if (k < a.E) {
              const double d = (double)__ldg(a.U + (size_t)__ldg(a.elite + k) * Hn + e) - c;
              const double wd = cem ? d : a.weight[k] * d;
              p1[j] = p1[j] + wd;
              p2[j] = fma(wd, d, p2[j]);
            }
          }
        }
      }
    }
    const double S1 = canonical_sum<G>(p1);
    const double S2 = canonical_sum<G>(p2);
    if constexpr (G == 1) {
      if (valid) finish_element(a, e, c, S1, S2, cem);
    } else {
      const int slot = threadIdx.x / G;
      if (sub == 0) {
        sh_S1[slot] = S1;
        sh_S2[slot] = S2;
        sh_c[slot] = c;
        sh_e[slot] = valid ? e : -1;
      }
      __syncthreads();
      if (threadIdx.x < kGroups && sh_e[threadIdx.x] >= 0)
        finish_element(a, sh_e[threadIdx.x], sh_c[threadIdx.x], sh_S1[threadIdx.x], sh_S2[threadIdx.x], cem);
      __syncthreads();  // the next sweep rewrites the slots
    }
  }
  if (a.d_iter && gt == 0) *a.d_iter += 1u;
}

template <int G>
__global__ void __launch_bounds__(kUpdThreads) k_update(const UpdateArgs a) {
  update_body<G>(a, blockIdx.x * blockDim.x + threadIdx.x, gridDim.x * blockDim.x);
}

// Many planning problems: thread_start (count + 1 entries) holds each
// instance's first thread.
template <int G>
__global__ void __launch_bounds__(kUpdThreads) k_update_batch(const UpdateArgs* __restrict__ args,
                                                      const int* __restrict__ thread_start,
                                                      int count) {
  // thread_start holds absolute thread numbers; this launch starts at thread_start[0]
  const int gt = __ldg(thread_start) + (int)(blockIdx.x * blockDim.x + threadIdx.x);
  if (gt >= __ldg(thread_start + count)) return;
  int lo = 0, hi = count;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (__ldg(thread_start + mid) <= gt) lo = mid;
    else hi = mid;
  }
  const UpdateArgs a = args[lo];
  update_body<G>(a, gt - __ldg(thread_start + lo),
                 __ldg(thread_start + lo + 1) - __ldg(thread_start + lo));
}

// Warm start: one thread per control dimension walks the horizon forward (in
// place is safe: row t reads row t+k >= t); the last row repeats.
__device__ __forceinline__ void shift_body(double* mu, double* sigma, float* mu_f, float* sigma_f,
                                           int H, int n, int k, int i) {
  for (int t = 0; t < H; ++t) {
    const int src = t + k < H ? t + k : H - 1;
    mu[t * n + i] = mu[src * n + i];
    sigma[t * n + i] = sigma[src * n + i];
    mu_f[t * n + i] = (float)mu[t * n + i];
    sigma_f[t * n + i] = (float)sigma[t * n + i];
  }
}

__global__ void k_shift(double* mu, double* sigma, float* mu_f, float* sigma_f, int H, int n,
                        int k) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) shift_body(mu, sigma, mu_f, sigma_f, H, n, k, i);
}

// one block per instance of a batch
__global__ void k_shift_batch(const UpdateArgs* __restrict__ args, int k) {
  const UpdateArgs& a = args[blockIdx.x];
  for (int i = threadIdx.x; i < a.n; i += blockDim.x)
    shift_body(a.mu, a.sigma, a.mu_f, a.sigma_f, a.H, a.n, k, i);
}

}  // namespace

size_t select_smem_bytes(int B, int E) {
  int Ep = 1;
  while (Ep < E) Ep <<= 1;
  // keys, the selected pairs, the boundary bin's pairs
  return (size_t)((B + 1) & ~1) * 4 + (size_t)Ep * 8 + (size_t)kBoundaryMax * 8;
}

cudaError_t init_select_attributes() {
  cudaError_t e;
  if ((e = cudaFuncSetAttribute(k_select, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024)) ||
      (e = cudaFuncSetAttribute(k_select_chunks, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024)) ||
      (e = cudaFuncSetAttribute(k_select_merge, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024)))
    return e;
  return cudaFuncSetAttribute(k_select_batch, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              200 * 1024);
}

cudaError_t launch_select_batch(const SelectArgs* d_args, int count, size_t smem, cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  k_select_batch<<<count, kSelThreads, smem, s>>>(d_args);
  return cudaGetLastError();
}

// Batches have many (t, i) elements: one lane each, no cross-lane sums.
cudaError_t launch_update_batch(const UpdateArgs* d_args, const int* d_thread_start, int count,
                                int total_threads, cudaStream_t s) {
  if (total_threads <= 0) return cudaSuccess;
  k_update_batch<1><<<(total_threads + kUpdThreads - 1) / kUpdThreads, kUpdThreads, 0, s>>>(d_args, d_thread_start, count);
  return cudaGetLastError();
}

int update_threads(int H, int n) { return H * n; }

// Threads of the single-instance selection block: about kSelKeys keys per
// thread, at least 128 and at least E (up to 1024), so that with E <= 1024
// every elite's weight has a thread of its own, as in the batched launch,
// and both give the same sums.  Measured: on the C1 point mass (B 512) the
// 128-thread block selects in 10.8-11.3 us against 12.2-12.6 with 1024
// threads; on the 7-link arm (B 4096) 4 and 8 keys per thread tie and 16
// are 3 us slower.
constexpr int kSelKeys = 4;

int select_threads(int B, int E) {
  int t = (B + kSelKeys - 1) / kSelKeys;
  if (t < E) t = E;
  t = (t + 31) & ~31;
  if (t < 128) t = 128;
  if (t > kSelThreads) t = kSelThreads;
  return t;
}

cudaError_t launch_select(const SelectArgs& a, cudaStream_t s) {
  k_select<<<1, select_threads(a.B, a.E), select_smem_bytes(a.B, a.E), s>>>(a);
  return cudaGetLastError();
}

// Two-stage selection plan for B candidates and E elites: the chunk length
// and chunk count, or chunks = 0 when one block selects them (its keys fit
// its shared memory and B is at most kOneBlockMax).  Chunks are as long as
// one block's shared memory allows, and their E-pair outputs must fit the
// merging block; infeasible sizes return chunks = -1.
void select_plan(int B, int E, int* chunk, int* chunks) {
  *chunk = B;
  *chunks = 0;
  if (select_smem_bytes(B, E) <= kSelSmemMax && B <= kOneBlockMax) return;
  int c = kChunkKeys;
  while (c > E && select_smem_bytes(c, E) > kSelSmemMax) c >>= 1;
  if (c < E) c = E;
  const long long n = ((long long)B + c - 1) / c;
  if (select_smem_bytes(c, E) > kSelSmemMax || select_smem_bytes((int)std::min<long long>(n * E, 1 << 30), E) > kSelSmemMax) {
    *chunks = -1;
    return;
  }
  *chunk = c;
  *chunks = (int)n;
}

cudaError_t launch_select_two_stage(const SelectArgs& a, int chunk, int chunks, cudaStream_t s) {
  SelectArgs c1 = a;
  c1.chunk = chunk;
  k_select_chunks<<<chunks, select_threads(chunk, a.E), select_smem_bytes(chunk, a.E), s>>>(c1);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  SelectArgs c2 = a;
  c2.B = chunks * a.E;
  k_select_merge<<<1, select_threads(c2.B, a.E), select_smem_bytes(c2.B, a.E), s>>>(c2);
  return cudaGetLastError();
}

// Lanes per element: as many as keep about 256 threads per SM busy, up to a warp.
cudaError_t launch_update(const UpdateArgs& a, cudaStream_t s) {
  const int Hn = a.H * a.n;
  // lanes per element: enough threads to spread the gathers over the GPU.
  // The kernel is latency-bound (elite index, then row gather), so more
  // lanes win even though each lane repeats the FP64 butterfly (8 lanes per
  // element measured slower than 32 on the 7-link arm workload)
  int G = 1;
  const long long want = (long long)device_sms() * 256;
  while (G < 32 && (long long)Hn * G < want) G <<= 1;
  const long long threads = (long long)Hn * G;
  const int blocks = (int)((threads + kUpdThreads - 1) / kUpdThreads);
  switch (G) {
    case 1: k_update<1><<<blocks, kUpdThreads, 0, s>>>(a); break;
    case 2: k_update<2><<<blocks, kUpdThreads, 0, s>>>(a); break;
    case 4: k_update<4><<<blocks, kUpdThreads, 0, s>>>(a); break;
    case 8: k_update<8><<<blocks, kUpdThreads, 0, s>>>(a); break;
    case 16: k_update<16><<<blocks, kUpdThreads, 0, s>>>(a); break;
    default: k_update<32><<<blocks, kUpdThreads, 0, s>>>(a); break;
  }
  return cudaGetLastError();
}

cudaError_t launch_shift_batch(const UpdateArgs* d_args, int count, int k, cudaStream_t s) {
  if (count <= 0 || k <= 0) return cudaSuccess;
  k_shift_batch<<<count, 32, 0, s>>>(d_args, k);
  return cudaGetLastError();
}

cudaError_t launch_shift(double* mu, double* sigma, float* mu_f, float* sigma_f, int H, int n, int k,
                         cudaStream_t s) {
  k_shift<<<(n + 63) / 64, 64, 0, s>>>(mu, sigma, mu_f, sigma_f, H, n, k);
  return cudaGetLastError();
}

}  // namespace mtp
