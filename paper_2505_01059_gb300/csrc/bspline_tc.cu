// bspline_tc.cu -- Def. 2 B-spline interpolation of the graph paths as a
// dense contraction on the 5th-generation tensor cores (tcgen05), for the
// BF16-operand mode (MTP_FLAG_BF16_BASIS).
//
// The graph rows of an iteration are U[b, t, i] = sum_m B[t, m] C[b, m, i]
// (Def. 2 with the basis B_p sampled at the H evaluation times and the
// waypoints C of path b, Alg. 1).  Seen as one GEMM, D[t, (b, i)] =
// sum_m A[t, m] B[m, (b, i)] with A the (H x M) basis table and B the
// gathered waypoints, K = M.  A tile is one 128-step slice of the horizon
// for up to kPaths paths; each CTA (one warpgroup) loops over tiles: it
// draws the paths' layer indices (Alg. 1), gathers their waypoints from the
// iteration's graph Z, rounds them to bfloat16 into the B operand (K-major,
// 16 columns per path, the columns past n zero), and one thread issues
// tcgen05.mma.cta_group::1.kind::f16 (BF16 x BF16 -> FP32, M = 128 steps,
// N = 128, K = 16 per instruction) into tensor memory.  The products of two
// bfloat16 values are exact in FP32; the sums are FP32.
// The epilogue reads each path's columns back with tcgen05.ld, clamps them
// to the control box and writes them through a per-warp shared-memory
// transpose as contiguous, coalesced rows of U.
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
constexpr int kPaths = 8;            // paths per tile, 16 accumulator columns each
constexpr int kNTile = kPaths * 16;  // MMA N
constexpr int kMaxK = 64;            // layers (M) padded to a multiple of 16
constexpr int kMaxSlices = 2;        // 128-step horizon slices (H <= 256)
constexpr uint32_t kTmemCols = 128;
constexpr size_t kMinSmem = 50 * 1024;  // at most four CTAs per SM (their TMEM fits)
constexpr int kBatchTilesPerCta = 8;

struct TcSmem {
  __nv_bfloat16 A[128 * kMaxK];              // basis of one slice, K-major canonical layout
  __nv_bfloat16 B[kNTile * kMaxK];           // waypoints, K-major canonical layout
  // per warp, two buffers of one path's 32 rows x n controls in the order
  // they take in U (a contiguous block there), written out by bulk copies
  float stage[kTcThreads / 32][2][32 * 16];
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
  }
}

// The basis of one horizon slice s as the A operand:
// A[r][k] = basis[(128 s + r) * M + k], zero past H and past M.
__device__ void load_basis(TcSmem& S, const CandArgs& a, int K, int s) {
  const int H = a.dm.H, M = a.dm.M;
  unsigned char* base = reinterpret_cast<unsigned char*>(&S.A[0]);
  for (int e = threadIdx.x; e < 128 * K; e += blockDim.x) {
    const int r = e / K, k = e - r * K;
    const int t = 128 * s + r;
    const float v = (t < H && k < M) ? a.basis[(size_t)t * M + k] : 0.f;
    *reinterpret_cast<__nv_bfloat16*>(base + kmajor_offset(r, k, K)) = __float2bfloat16_rn(v);
  }
}

// Path group g of one instance's graph rows, horizon slice s (the A operand
// holds that slice's basis).  Returns false when the bounded wait for the
// MMA gave up.
__device__ bool tc_tile(TcSmem& S, const CandArgs& a, int g, int s, int K, uint32_t iter,
                        uint32_t& phase) {
  const Dims dm = a.dm;
  const int H = dm.H, n = dm.n, M = dm.M, N = dm.N;
  const int b0 = g * kPaths;
  const int nb = min(kPaths, a.graph_rows - b0);
  unsigned char* Bb = reinterpret_cast<unsigned char*>(S.B);
  // Alg. 1 for the tile's paths and the gather of their waypoints, rounded
  // to bfloat16, into the B operand: column 16 p + i, row m.
  for (int e = threadIdx.x; e < nb * M; e += blockDim.x) {
    const int p = e / M, m = e - p * M;
    const float* z;
    if (a.C_in) {
      z = a.C_in + ((size_t)(b0 + p) * M + m) * n;
    } else {
      const uint4 r = philox(make_uint4((uint32_t)(b0 + p), (uint32_t)(m >> 2), iter, kTagPath), a.key);
      const int j = index_of(pick(r, (uint32_t)(m & 3)), (uint32_t)N);
      z = a.Z_global + ((size_t)m * N + j) * n;
    }
    for (int i = 0; i < n; ++i)
      *reinterpret_cast<__nv_bfloat16*>(Bb + kmajor_offset(16 * p + i, m, K)) = __float2bfloat16_rn(z[i]);
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  __syncthreads();
  if (threadIdx.x == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t idesc = idesc_bf16(128, kNTile);
    const uint32_t sbo = 16u * (uint32_t)K;
    const uint32_t d_tmem = S.tmem_base;
    for (int ks = 0; ks < K / 16; ++ks) {
      const uint64_t ad = smem_desc(smem_u32(&S.A[0]) + 256u * ks, 128u, sbo);
      const uint64_t bd = smem_desc(smem_u32(&S.B[0]) + 256u * ks, 128u, sbo);
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
  // epilogue: warp w reads accumulator lanes 32 w .. 32 w + 31 (steps
  // t0 .. t0 + 31 of each slice) path by path, clamps them to the box (kept
  // in registers) and writes the path's rows t0 .. t0 + 31, a contiguous
  // block of U, from shared memory: one bulk copy when its start and length
  // are whole 16-byte units, else coalesced stores
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float lo[16], hi[16];
#pragma unroll
  for (int i = 0; i < 16; ++i) {
    lo[i] = i < n ? S.lo[i] : 0.f;
    hi[i] = i < n ? S.hi[i] : 0.f;
  }
  const bool bulk_ok = ((reinterpret_cast<uintptr_t>(a.U_graph) & 15) == 0) && ((H * n) & 3) == 0;
  int buf = 0;
  {
    const int t0 = 128 * s + 32 * w;
    const int rows = min(32, H - t0);
    for (int p = 0; p < nb; ++p) {
      const uint32_t taddr = S.tmem_base + ((uint32_t)(32 * w) << 16) + (uint32_t)(16 * p);
      uint32_t v[16];
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
          : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
            "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
            "=r"(v[14]), "=r"(v[15])
          : "r"(taddr));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      if (rows <= 0) continue;
      float* st = S.stage[w][buf];
      // the bulk copy that last read this buffer (two paths ago) must be done
      if (lane == 0) asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory");
      __syncwarp();
#pragma unroll
      for (int i = 0; i < 16; ++i)
        if (i < n) st[lane * n + i] = clamp_box(__uint_as_float(v[i]), lo[i], hi[i]);
      float* out = a.U_graph + ((size_t)(b0 + p) * H + t0) * n;
      const int count = rows * n;
      if (bulk_ok && (count & 3) == 0) {
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncwarp();
        if (lane == 0) {
          asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(out),
                       "r"(smem_u32(st)), "r"((uint32_t)(count * 4))
                       : "memory");
          asm volatile("cp.async.bulk.commit_group;" ::: "memory");
        }
        buf ^= 1;
      } else {
        __syncwarp();
        for (int e = lane; e < count; e += 32) out[e] = st[e];
        __syncwarp();
      }
    }
  }
  // the warp's bulk copies have read their sources before the next tile
  // refills the buffers
  if (lane == 0) asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
  __syncwarp();
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  return true;
}

// Per-CTA set-up for one instance: box and a zeroed B operand.
__device__ void tc_instance_setup(TcSmem& S, const CandArgs& a) {
  for (int i = threadIdx.x; i < a.dm.n; i += blockDim.x) {
    S.lo[i] = a.umin[i];
    S.hi[i] = a.umax[i];
  }
  uint32_t* Bw = reinterpret_cast<uint32_t*>(S.B);
  for (int e = threadIdx.x; e < (int)(sizeof(S.B) / 4); e += blockDim.x) Bw[e] = 0u;
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
  const int groups = (a.graph_rows + kPaths - 1) / kPaths;
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
    const int groups = (sa.graph_rows + kPaths - 1) / kPaths;
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

}  // namespace

bool bspline_tc_eligible(const CandArgs& a) {
  return a.bf16 && a.interp == MTP_INTERP_BSPLINE && a.dm.H <= 128 * kMaxSlices &&
         a.dm.M <= kMaxK && a.dm.n <= 16 && a.graph_rows > 0;
}

int bspline_tc_tiles(const CandArgs& a) {
  return ((a.graph_rows + kPaths - 1) / kPaths) * ((a.dm.H + 127) / 128);
}

cudaError_t init_bspline_tc_attributes() {
  cudaError_t e = cudaFuncSetAttribute(k_bspline_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)tc_smem_bytes());
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_bspline_tc_batch, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)tc_smem_bytes());
}

cudaError_t launch_bspline_tc(const CandArgs& a, cudaStream_t s) {
  const int tiles = bspline_tc_tiles(a);
  if (tiles <= 0) return cudaSuccess;
  const int grid = std::min(tiles, 4 * device_sms());
  k_bspline_tc<<<grid, kTcThreads, tc_smem_bytes(), s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_bspline_tc_batch(const CandArgs* d_args, const int* d_tile_start, int count,
                                    int total_tiles, cudaStream_t s) {
  if (total_tiles <= 0) return cudaSuccess;
  // at least kBatchTilesPerCta tiles per CTA: in a batch the launches of
  // other groups run beside this one, and each CTA's set-up (tensor memory,
  // operands) is paid once for its whole range
  const int grid = std::min((total_tiles + kBatchTilesPerCta - 1) / kBatchTilesPerCta, 4 * device_sms());
  k_bspline_tc_batch<<<grid, kTcThreads, tc_smem_bytes(), s>>>(d_args, d_tile_start, count);
  return cudaGetLastError();
}

}  // namespace mtp
