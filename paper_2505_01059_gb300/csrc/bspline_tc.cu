// bspline_tc.cu -- Def. 2 B-spline interpolation of the graph paths as a
// dense contraction on the 5th-generation tensor cores (tcgen05), for the
// BF16-operand mode (MTP_FLAG_BF16_BASIS).
//
// The graph rows of an iteration are U[b, t, i] = sum_m B[t, m] C[b, m, i]
// (Def. 2 with the basis B_p sampled at the H evaluation times and the
// waypoints C of path b, Alg. 1).  Seen as one GEMM,
// D[(b, i), t] = sum_m W[(b, i), m] B[t, m] with W the gathered waypoints
// (one row per path and control dimension) and B the (H x M) basis table,
// K = M.  A tile is up to 128 (path, dimension) rows by one 128-step slice
// of the horizon: warp w's 32 accumulator lanes hold floor(32 / n) whole
// paths (rows 32 w + n p + i), so a path never straddles two warps and the
// rows are dense for any n.  Each CTA (one warpgroup) loops over tiles: it
// draws the paths' layer indices (Alg. 1, four layers per generator call),
// copies their waypoints, already rounded to bfloat16, from the instance's
// graph (staged in shared memory once per instance) into the A operand, and
// one thread issues tcgen05.mma.cta_group::1.kind::f16 (BF16 x BF16 -> FP32,
// M = 128 rows, N = 128 steps, K = 16 per instruction) into tensor memory.
// The products of two bfloat16 values are exact in FP32; the sums are FP32.
// The epilogue reads 16 steps of its row at a time with tcgen05.ld, clamps
// them to the control box and writes them through a per-warp shared-memory
// transpose: for each of the warp's paths, 16 steps x n controls are one
// contiguous block of U, stored with 16-byte vector stores.
//
// Shared-memory operands use the canonical K-major layout without swizzle:
// 8-row x 16-byte core matrices, the two (or more) core matrices of a row
// group along K 128 bytes apart (leading byte offset) and consecutive row
// groups 16 K bytes apart (stride byte offset).  Each CTA allocates 128
// tensor-memory columns (its accumulator) and asks for enough shared memory
// that at most four CTAs share an SM, so their allocations always fit the
// SM's 512 columns.
#include <algorithm>

#include <cuda_bf16.h>

#include "mtp_device.cuh"

namespace mtp {
namespace {

constexpr int kTcThreads = 128;
constexpr int kMaxK = 64;            // layers (M) padded to a multiple of 16
constexpr int kMaxSlices = 2;        // 128-step horizon slices (H <= 256)
constexpr int kZsMax = 12288;        // graph elements (M N n) staged in shared memory
constexpr uint32_t kTmemCols = 128;
constexpr size_t kMinSmem = 50 * 1024;  // at most four CTAs per SM (their TMEM fits)
constexpr int kBatchTilesPerCta = 8;

struct TcSmem {
  __nv_bfloat16 W[128 * kMaxK];   // A operand: waypoints, row 32 w + n p + i, K-major
  __nv_bfloat16 Bs[128 * kMaxK];  // B operand: basis of one slice, row t, K-major
  __nv_bfloat16 Zs[kZsMax];       // the instance's graph in bfloat16, when it fits
  // per warp: 16 steps of its paths' rows, path by path in the order of U
  float stage[kTcThreads / 32][32 * 16];
  float lo[MTP_MAX_CTRL], hi[MTP_MAX_CTRL];
  uint64_t mma_bar;
  uint32_t tmem_base;
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// Byte offset of element (row, k) in a K-major, unswizzled canonical layout
// with K columns: core matrix (row / 8, k / 8), row (row % 8) of 16 bytes.
__device__ __forceinline__ int kmajor_offset(int row, int k, int K) {
  return (row >> 3) * (16 * K) + (k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2;
}

// tcgen05 shared-memory matrix descriptor: start address, leading and stride
// byte offsets (all in 16-byte units), the fixed version field (bits 46-48 =
// 0b001), no base offset, no swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | ((uint64_t)1 << 46);
}

// Instruction descriptor of kind::f16: FP32 accumulator (bits 4-5 = 1),
// BF16 A and B (bits 7-9, 10-12 = 1), both K-major, N >> 3 at bit 17,
// M >> 4 at bit 24.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}

// Paths per warp and per tile for n control dimensions (n <= 16).
__host__ __device__ constexpr int tc_paths_per_warp(int n) { return 32 / n; }
__host__ __device__ constexpr int tc_paths_per_tile(int n) {
  return (kTcThreads / 32) * tc_paths_per_warp(n);
}

// Waits for the MMA's commit, bounded by 2 s of global time; backs off
// between polls so that the waiting warps leave the issue slots to the
// co-resident CTAs' epilogues.
__device__ __forceinline__ bool mbar_wait_bounded_tc(uint64_t* bar, uint32_t parity) {
  const unsigned addr = smem_u32(bar);
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
    else if (now - t_start > 2000000000ull) return false;
    if (spin >= 4) __nanosleep(64);
  }
}

// The basis of one horizon slice s as the B operand:
// Bs[r][k] = basis[(128 s + r) * M + k], zero past H and past M.
__device__ void load_basis(TcSmem& S, const CandArgs& a, int K, int s) {
  const int H = a.dm.H, M = a.dm.M;
  unsigned char* base = reinterpret_cast<unsigned char*>(&S.Bs[0]);
  for (int e = threadIdx.x; e < 128 * K; e += blockDim.x) {
    const int r = e / K, k = e - r * K;
    const int t = 128 * s + r;
    const float v = (t < H && k < M) ? a.basis[(size_t)t * M + k] : 0.f;
    *reinterpret_cast<__nv_bfloat16*>(base + kmajor_offset(r, k, K)) = __float2bfloat16_rn(v);
  }
}

__device__ __forceinline__ bool graph_staged(const CandArgs& a) {
  return a.C_in == nullptr && a.dm.M * a.dm.N * a.dm.n <= kZsMax;
}

// Path group g of one instance's graph rows, horizon slice s (the B operand
// holds that slice's basis).  Returns false when the bounded wait for the
// MMA gave up.
__device__ __forceinline__ bool tc_tile(TcSmem& S, const CandArgs& a, int g, int s, int K, uint32_t iter,
                        uint32_t& phase) {
  const Dims dm = a.dm;
  const int H = dm.H, n = dm.n, M = dm.M, N = dm.N;
  const int ppw = tc_paths_per_warp(n);
  const int b0 = g * tc_paths_per_tile(n);
  const int nb = min(tc_paths_per_tile(n), a.graph_rows - b0);
  unsigned char* Wb = reinterpret_cast<unsigned char*>(S.W);
  const bool staged = graph_staged(a);
  // Alg. 1 for the tile's paths (one generator call per four layers) and
  // the copy of their waypoints, in bfloat16, into the A operand: row
  // 32 (q / ppw) + n (q % ppw) + i for the tile's path q, column m.
  const int quads = (M + 3) >> 2;
  for (int e = threadIdx.x; e < nb * quads; e += blockDim.x) {
    const int q = e / quads, mq = e - q * quads;
    const int row0 = 32 * (q / ppw) + n * (q % ppw);
    uint4 r = make_uint4(0u, 0u, 0u, 0u);
    if (a.C_in == nullptr)
      r = philox(make_uint4((uint32_t)(b0 + q), (uint32_t)mq, iter, kTagPath), a.key);
#pragma unroll
    for (int w = 0; w < 4; ++w) {
      const int m = 4 * mq + w;
      if (m < M) {
        if (a.C_in) {
          const float* z = a.C_in + ((size_t)(b0 + q) * M + m) * n;
          for (int i = 0; i < n; ++i)
            *reinterpret_cast<__nv_bfloat16*>(Wb + kmajor_offset(row0 + i, m, K)) = __float2bfloat16_rn(z[i]);
        } else {
          const int j = index_of(pick(r, (uint32_t)w), (uint32_t)N);
          if (staged) {
            const __nv_bfloat16* z = S.Zs + (m * N + j) * n;
            for (int i = 0; i < n; ++i)
              *reinterpret_cast<__nv_bfloat16*>(Wb + kmajor_offset(row0 + i, m, K)) = z[i];
          } else {
            const float* z = a.Z_global + ((size_t)m * N + j) * n;
            for (int i = 0; i < n; ++i)
              *reinterpret_cast<__nv_bfloat16*>(Wb + kmajor_offset(row0 + i, m, K)) = __float2bfloat16_rn(z[i]);
          }
        }
      }
    }
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  __syncthreads();
  if (threadIdx.x == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t idesc = idesc_bf16(128, 128);
    const uint32_t sbo = 16u * (uint32_t)K;
    const uint32_t d_tmem = S.tmem_base;
    for (int ks = 0; ks < K / 16; ++ks) {
      const uint64_t ad = smem_desc(smem_u32(&S.W[0]) + 256u * ks, 128u, sbo);
      const uint64_t bd = smem_desc(smem_u32(&S.Bs[0]) + 256u * ks, 128u, sbo);
      const uint32_t acc = ks > 0 ? 1u : 0u;
      asm volatile(
          "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
          " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
          "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
          : "memory");
    }
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_u32(&S.mma_bar))
                 : "memory");
  }
  const bool ok = mbar_wait_bounded_tc(&S.mma_bar, phase);
  phase ^= 1u;
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (!__syncthreads_and(ok)) return false;
  // epilogue: warp w reads accumulator lanes 32 w .. 32 w + 31, 16 steps
  // (columns) at a time; lane l holds row (path l / n, dimension l % n) of
  // the warp's paths.  Clamped values go to the warp's staging area in the
  // order of U (path-major, then step, then dimension), from which each
  // path's 16 n contiguous floats of U are written.
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int p = lane / n, i = lane - p * n;
  const int wb0 = b0 + w * ppw;                          // the warp's first path
  const int wpaths = max(0, min(ppw, a.graph_rows - wb0));  // its paths in this tile
  const float lo = i < n ? S.lo[i] : 0.f, hi = i < n ? S.hi[i] : 0.f;
  const bool vec = ((reinterpret_cast<uintptr_t>(a.U_graph) & 15) == 0) && ((H * n) & 3) == 0;
  const int t_end = min(128 * (s + 1), H);
  float* st = S.stage[w];
  for (int t0 = 128 * s; t0 < t_end; t0 += 16) {
    const uint32_t taddr = S.tmem_base + ((uint32_t)(32 * w) << 16) + (uint32_t)(t0 - 128 * s);
    uint32_t v[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
          "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
          "=r"(v[14]), "=r"(v[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
    if (wpaths == 0) continue;
    const int steps = min(16, H - t0);  // steps of this chunk inside the horizon
    __syncwarp();                        // the previous chunk's reads of st are done
    if (p < wpaths) {
      float* sp = st + p * 16 * n + i;
#pragma unroll
      for (int tt = 0; tt < 16; ++tt) {
        if (tt < steps) *sp = clamp_box(__uint_as_float(v[tt]), lo, hi);
        sp += n;
      }
    }
    __syncwarp();
    const int piece = steps * n;  // floats of one path in this chunk
    // flat over the warp's pieces; the piece index e / len is taken as
    // (e + 1/2) * (1 / len) rounded down, exact here (e < 2^12, len <= 256:
    // the product's rounding error stays far below the 1/(2 len) margin)
    const size_t Hn = (size_t)H * n;
    if (vec && (piece & 3) == 0) {
      const int q4 = piece >> 2;
      const float inv = 1.f / (float)q4;
      for (int e = lane; e < wpaths * q4; e += 32) {
        const int pp = __float2int_rz(((float)e + 0.5f) * inv), o = e - pp * q4;
        reinterpret_cast<float4*>(a.U_graph + (wb0 + pp) * Hn + (size_t)t0 * n)[o] =
            reinterpret_cast<const float4*>(st + pp * 16 * n)[o];
      }
    } else {
      const float inv = 1.f / (float)piece;
      for (int e = lane; e < wpaths * piece; e += 32) {
        const int pp = __float2int_rz(((float)e + 0.5f) * inv), o = e - pp * piece;
        a.U_graph[(wb0 + pp) * Hn + (size_t)t0 * n + o] = st[pp * 16 * n + o];
      }
    }
  }
  __syncwarp();
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  return true;
}

// Per-CTA set-up for one instance: box, a zeroed A operand (its columns
// past M stay zero) and the instance's graph in bfloat16 (when it fits).
__device__ void tc_instance_setup(TcSmem& S, const CandArgs& a) {
  for (int i = threadIdx.x; i < a.dm.n; i += blockDim.x) {
    S.lo[i] = a.umin[i];
    S.hi[i] = a.umax[i];
  }
  uint32_t* Ww = reinterpret_cast<uint32_t*>(S.W);
  for (int e = threadIdx.x; e < (int)(sizeof(S.W) / 4); e += blockDim.x) Ww[e] = 0u;
  if (graph_staged(a)) {
    const int total = a.dm.M * a.dm.N * a.dm.n;
    for (int e = threadIdx.x; e < total; e += blockDim.x) S.Zs[e] = __float2bfloat16_rn(a.Z_global[e]);
  }
  __syncthreads();
}

__device__ void tc_begin(TcSmem& S) {
  if (threadIdx.x < 32) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&S.tmem_base)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&S.mma_bar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// Releases the tensor memory.  After a failed wait, first waits (bounded)
// for the MMA still in flight.
__device__ void tc_end(TcSmem& S, bool failed, uint32_t phase, uint32_t* status) {
  // every bulk copy of rows has landed before the CTA leaves
  if ((threadIdx.x & 31) == 0) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
  if (failed) {
    mbar_wait_bounded_tc(&S.mma_bar, phase ^ 1u);
    if (threadIdx.x == 0 && status) atomicOr(status, kStatusTcTimeout);
  }
  __syncthreads();
  if (threadIdx.x < 32)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(S.tmem_base),
                 "r"(kTmemCols)
                 : "memory");
}

__device__ __forceinline__ TcSmem& tc_smem() {
  extern __shared__ __align__(1024) unsigned char tc_dyn_smem[];
  return *reinterpret_cast<TcSmem*>(tc_dyn_smem);
}

// One instance: CTAs loop over its tiles, slice-major (tile = s * groups + g),
// so that a CTA changes slice, and reloads the basis, rarely.
__global__ void __launch_bounds__(kTcThreads) k_bspline_tc(const CandArgs a) {
  TcSmem& S = tc_smem();
  const int K = ((a.dm.M + 15) / 16) * 16;
  const int groups = (a.graph_rows + tc_paths_per_tile(a.dm.n) - 1) / tc_paths_per_tile(a.dm.n);
  const int tiles = groups * ((a.dm.H + 127) / 128);
  const uint32_t iter = (a.d_iter ? *a.d_iter : a.iter) + a.iter_offset;
  tc_begin(S);
  tc_instance_setup(S, a);
  uint32_t phase = 0;
  bool failed = false;
  int cur_s = -1;
  for (int tile = blockIdx.x; tile < tiles && !failed; tile += gridDim.x) {
    const int s = tile / groups, g = tile - s * groups;
    if (s != cur_s) {
      load_basis(S, a, K, s);
      __syncthreads();
      cur_s = s;
    }
    failed = !tc_tile(S, a, g, s, K, iter, phase);
  }
  tc_end(S, failed, phase, a.status);
}

// Many instances: tile_start (count + 1 entries) numbers each instance's
// first tile; each CTA takes a contiguous range of the global tile list (so
// it changes instance, and reloads its set-up, rarely) and sets up again
// whenever the instance or the slice changes.
__global__ void __launch_bounds__(kTcThreads) k_bspline_tc_batch(const CandArgs* __restrict__ args,
                                                                 const int* __restrict__ tile_start,
                                                                 int count) {
  TcSmem& S = tc_smem();
  __shared__ CandArgs sa;
  tc_begin(S);
  const int total = tile_start[count];
  int cur = -1, cur_s = -1, K = 16;
  uint32_t iter = 0, phase = 0;
  bool failed = false;
  const int per = (total + gridDim.x - 1) / gridDim.x;
  const int g_end = min(total, ((int)blockIdx.x + 1) * per);
  for (int g = (int)blockIdx.x * per; g < g_end && !failed; ++g) {
    int lo = 0, hi = count;
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (tile_start[mid] <= g) lo = mid;
      else hi = mid;
    }
    if (lo != cur) {
      __syncthreads();
      const int* src = reinterpret_cast<const int*>(args + lo);
      int* dst = reinterpret_cast<int*>(&sa);
      for (int q = threadIdx.x; q < (int)(sizeof(CandArgs) / sizeof(int)); q += blockDim.x) dst[q] = src[q];
      __syncthreads();
      cur = lo;
      cur_s = -1;
      K = ((sa.dm.M + 15) / 16) * 16;
      iter = (sa.d_iter ? *sa.d_iter : sa.iter) + sa.iter_offset;
      tc_instance_setup(S, sa);
    }
    // the instance's tiles slice-major, as in the single-instance kernel
    const int groups = (sa.graph_rows + tc_paths_per_tile(sa.dm.n) - 1) / tc_paths_per_tile(sa.dm.n);
    const int tile = g - tile_start[lo];
    const int s = tile / groups, pg = tile - s * groups;
    if (s != cur_s) {
      load_basis(S, sa, K, s);
      __syncthreads();
      cur_s = s;
    }
    failed = !tc_tile(S, sa, pg, s, K, iter, phase);
  }
  tc_end(S, failed, phase, cur >= 0 ? sa.status : nullptr);
}

size_t tc_smem_bytes() { return sizeof(TcSmem) > kMinSmem ? sizeof(TcSmem) : kMinSmem; }
static_assert(sizeof(TcSmem) >= kMinSmem, "at most four CTAs per SM keep their TMEM allocations within 512 columns");

}  // namespace

bool bspline_tc_eligible(const CandArgs& a) {
  return a.bf16 && a.interp == MTP_INTERP_BSPLINE && a.dm.H <= 128 * kMaxSlices &&
         a.dm.M <= kMaxK && a.dm.n <= 16 && a.graph_rows > 0;
}

int bspline_tc_tiles(const CandArgs& a) {
  const int per = tc_paths_per_tile(a.dm.n);
  return ((a.graph_rows + per - 1) / per) * ((a.dm.H + 127) / 128);
}

// CTAs of the contraction kernels resident on one SM (set with their
// attributes; shared memory bounds it)
static int g_tc_blocks_per_sm = 1;

cudaError_t init_bspline_tc_attributes() {
  cudaError_t e = cudaFuncSetAttribute(k_bspline_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)tc_smem_bytes());
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_bspline_tc_batch, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)tc_smem_bytes());
  if (e != cudaSuccess) return e;
  // the largest shared-memory carveout, so that several CTAs fit an SM
  for (const void* k : {(const void*)k_bspline_tc, (const void*)k_bspline_tc_batch}) {
    e = cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return e;
  }
  // CTAs per SM from the SM's shared memory (the occupancy query answered 1
  // for these kernels, while ncu's launch statistics, with the maximum
  // carveout, showed room for 3; at 1 CTA per SM the legged workload's 1230
  // tiles ran 8 to a CTA, one after another)
  int dev = 0, smem_sm = 0, reserved = 0;
  if ((e = cudaGetDevice(&dev)) ||
      (e = cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev)) ||
      (e = cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev)))
    return e;
  cudaFuncAttributes fa{};
  if ((e = cudaFuncGetAttributes(&fa, k_bspline_tc_batch))) return e;
  const size_t per_cta = tc_smem_bytes() + fa.sharedSizeBytes + (size_t)reserved;
  const int blocks = (int)((size_t)smem_sm / per_cta);
  g_tc_blocks_per_sm = std::max(1, std::min(blocks, 4));
  return cudaSuccess;
}

cudaError_t launch_bspline_tc(const CandArgs& a, cudaStream_t s) {
  const int tiles = bspline_tc_tiles(a);
  if (tiles <= 0) return cudaSuccess;
  const int grid = std::min(tiles, g_tc_blocks_per_sm * device_sms());
  k_bspline_tc<<<grid, kTcThreads, tc_smem_bytes(), s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_bspline_tc_batch(const CandArgs* d_args, const int* d_tile_start, int count,
                                    int total_tiles, cudaStream_t s) {
  if (total_tiles <= 0) return cudaSuccess;
  // at least kBatchTilesPerCta tiles per CTA: in a batch the launches of
  // other groups run beside this one, and each CTA's set-up (tensor memory,
  // operands) is paid once for its whole range
  const int grid = std::min((total_tiles + kBatchTilesPerCta - 1) / kBatchTilesPerCta,
                            g_tc_blocks_per_sm * device_sms());
  k_bspline_tc_batch<<<grid, kTcThreads, tc_smem_bytes(), s>>>(d_args, d_tile_start, count);
  return cudaGetLastError();
}

}  // namespace mtp
