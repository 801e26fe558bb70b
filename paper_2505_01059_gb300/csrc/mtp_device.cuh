// mtp_device.cuh -- device-side building blocks shared by the MTP kernels:
// the counter-based generator, launch argument blocks and small helpers.
#pragma once

#include <cstdint>
#include <string>

#include <cuda_runtime.h>

#include "mtp.h"

namespace mtp {

// Stream tags of the Philox counter (word 3): one independent stream per kind
// of random draw of Alg. 2.
enum : uint32_t {
  kTagGraph = 1,        // Def. 1 graph waypoints
  kTagPath = 2,         // Alg. 1 path indices
  kTagLocal = 3,        // Alg. 2 local Gaussian samples
  kTagParamSample = 4,  // per-candidate model scales
  kTagParamModel = 5,   // shared randomised models
};

struct Key {
  uint32_t k0, k1;
};

// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of two 32x32
// multiplies with the published multipliers, key bumped by the Weyl constants.
__device__ __forceinline__ uint4 philox(uint4 c, Key key) {
  uint32_t k0 = key.k0, k1 = key.k1;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    // one 32 x 32 -> 64-bit product per multiplier, split into its halves
    // (measured 5 % faster on the 7-link arm step than a separate low
    // product and __umulhi)
    const unsigned long long p0 = 0xD2511F53ull * c.x, p1 = 0xCD9E8D57ull * c.z;
    const uint32_t lo0 = (uint32_t)p0, hi0 = (uint32_t)(p0 >> 32);
    const uint32_t lo1 = (uint32_t)p1, hi1 = (uint32_t)(p1 >> 32);
    c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return c;
}

__device__ __forceinline__ uint32_t pick(uint4 v, uint32_t w) {
  return w == 0 ? v.x : (w == 1 ? v.y : (w == 2 ? v.z : v.w));
}

// Word (b & 3) of the generator call at counter (a, b / 4, iter, tag).
__device__ __forceinline__ uint32_t draw(Key key, uint32_t a, uint32_t b, uint32_t iter,
                                         uint32_t tag) {
  return pick(philox(make_uint4(a, b >> 2, iter, tag), key), b & 3u);
}

// Uniform in [0, 1) from the top 24 bits (exact in FP32).
__device__ __forceinline__ float unit24(uint32_t r) {
  return (float)(r >> 8) * 5.9604644775390625e-8f;
}

// Uniform index in [0, N): high word of r * N (multiply-high mapping).
__device__ __forceinline__ int32_t index_of(uint32_t r, uint32_t N) {
  return (int32_t)__umulhi(r, N);
}

__device__ __forceinline__ float clamp_box(float v, float lo, float hi) {
  return v < lo ? lo : (v > hi ? hi : v);
}

// Compensated (Kahan) accumulation in FP32.
struct KahanSum {
  float s = 0.f, c = 0.f;
  __device__ __forceinline__ void add(float x, bool kahan) {
    if (kahan) {
      const float y = x - c;
      const float t = s + y;
      c = (t - s) - y;
      s = t;
    } else {
      s += x;
    }
  }
  // The same sums without a branch (the compensation stays zero when off).
  // Measured: 3 % faster in the legged rollout, 2-3 % slower in the chain
  // and point-mass rollouts, so only the legged rollout uses it.
  __device__ __forceinline__ void add_branch_free(float x, bool kahan) {
    const float y = x - c;
    const float t = s + y;
    c = kahan ? (t - s) - y : 0.f;
    s = t;
  }
};

struct Dims {
  int32_t B, P, L, E, H, n, d, M, N;
};

// What the local-row pass writes into rows [0, local_rows): the finished
// samples clamp(mu + sigma * eps) (kLocalFull), the standard normal draws eps
// alone (kLocalNoise, which depend only on the key and the iteration and so
// can be made ahead of the iteration's mean and spread), or the finished
// samples from draws already stored there (kLocalFinish).  The arithmetic of
// a finished sample is the same single fused multiply-add and clamp in every
// mode, so the three routes give the same bits.
enum LocalMode : int32_t { kLocalFull = 0, kLocalNoise = 1, kLocalFinish = 2 };

// Candidate generation (Def. 1, Alg. 1, interpolation, local sampling).
struct CandArgs {
  Dims dm;
  Key key;
  uint32_t iter;
  const uint32_t* d_iter;  // when set, the iteration is read from here
  uint32_t iter_offset;    // added to that iteration (1: the next iteration's draws)
  int32_t local_mode;      // LocalMode
  int32_t interp;          // mtp_interp
  int32_t degree;          // B-spline degree p
  int32_t bf16;            // B-spline contraction with BF16 operands (the basis table is
                           // rounded on the host, the knots as they are gathered)
  float inv_h;             // reciprocal knot spacing of the Akima / linear knots
  const float* basis;      // (H, M) B-spline basis, row t
  const int32_t* bfirst;   // (H) first non-zero basis column of row t
  const int32_t* seg;      // (H) Akima / linear piece of step t
  const float* delta;      // (H) offset of step t from the piece's left knot
  // graph rows
  const float* C_in;       // (P, M, n) given waypoints, or null to sample them
  const float* Z_global;   // (M, N, n) graph already in global memory, or null to
                           // regenerate it in each block's shared memory
  float* U_graph;          // output rows of the graph paths (graph_rows, H, n)
  int32_t graph_rows;
  int32_t graph_blocks;    // blocks [0, graph_blocks) make graph rows
  int32_t paths_per_block;
  // local rows and the mean row
  float* U_local;          // rows [0, local_rows) or null
  int32_t local_rows;
  float* U_mean;           // the mean row or null
  const float* mu;         // (H, n) FP32 copy of the FP64 mean
  const float* sigma;      // (H, n) FP32 copy of the FP64 spread
  float umin[MTP_MAX_CTRL], umax[MTP_MAX_CTRL];
  uint32_t* status;        // the handle's device status word (bounded waits that gave up)
};

struct RolloutArgs {
  int32_t H, n, d;
  float dt;
  Key key;
  uint32_t iter;
  const uint32_t* d_iter;
  int32_t dr_mode, R;
  float dr_lo, dr_hi;
  const float* x0;   // (d)
  const float* U;    // (rows, H, n), row r is candidate row0 + r
  int32_t row0, rows;
  float* cost;       // (rows)
  float* X;          // (H+1, d) states of the single requested row, or null
  int32_t kahan;
  uint32_t* status;  // device status word of the handle (bits set by a rollout), or null
};

// Bits of a handle's device status word, set when a bounded wait gave up:
// a rollout's wait for its staged controls (those candidates cost +inf), or
// the tensor-core contraction's wait for its MMA (those graph rows are not
// written).
constexpr uint32_t kStatusStageTimeout = 1u;
constexpr uint32_t kStatusTcTimeout = 2u;

// Whether a rollout launch may stage its controls through shared memory with
// bulk copies (see StagedRows): 16-byte aligned rows of a multiple of 4
// floats, one model per candidate, no state output.
inline bool can_stage(const RolloutArgs& a, int k) {
  return a.X == nullptr && a.dr_mode != MTP_DR_SHARED &&
         ((uintptr_t)a.U % 16u) == 0 && ((long long)a.H * k) % 4 == 0;
}

// The obstacle centres first and the struct 16-byte aligned: each centre
// row starts on a 16-byte boundary, so a rollout reads it (from shared
// memory in the batched kernel) with 16-byte vector loads.
struct alignas(16) PointMassModel {
  float obs_c[MTP_MAX_OBSTACLES][16];
  float target[16];
  float obs_r[MTP_MAX_OBSTACLES];
  float w_target, w_obs, w_ctrl, w_term;
  int32_t n_obs;
};

struct ChainModel {
  float mass[12], length[12];
  float gravity;
  float target[2];
  float w_target, w_ctrl, w_term;
};

struct LeggedModel {
  float mass[16], length[16];
  float gravity;
  float k_contact, c_contact, mu_friction, inv_v_slip;
  float target[3];  // height, forward velocity, pitch
  float w_height, w_vel, w_pitch, w_ctrl, w_term;
};

struct SelectArgs {
  const float* cost;  // (B)
  const float* U;     // (B, H, n)
  int32_t B, E, H, n;
  double inv_lambda;  // 1 / lambda
  int32_t update_rule;
  int32_t* elite;     // (E) internal
  double* weight;     // (E) internal
  float* ustar;       // (n) internal
  int32_t* elite_out; // optional copy
  float* ustar_out;   // optional copy
  double* entropy;    // optional: the cost entropy of all B costs (Sec. 4.1 diagnostic)
  // two-stage selection (B beyond one block): scratch of chunks * E
  // (key, index) pairs and the first stage's chunk length
  unsigned long long* pairs;
  int32_t chunk;
};

struct UpdateArgs {
  const float* U;       // (B, H, n)
  const int32_t* elite; // (E)
  const double* weight; // (E)
  int32_t E, H, n;
  double alpha, sigma_min;
  int32_t update_rule;
  double* mu;           // (H, n) in/out
  double* sigma;        // (H, n) in/out
  float* mu_f;          // (H, n) FP32 copies written alongside
  float* sigma_f;
  uint32_t* d_iter;     // incremented once when set
};

// host-side launchers (defined in the .cu files)
void set_thread_error(const std::string& msg);  // text for mtp_last_error(NULL)
// Streaming multiprocessors of the current device, queried once per device
// and cached (launch shapes are sized from it, never from a fixed count).
int device_sms();
size_t candidates_smem_bytes(const CandArgs& a);
cudaError_t init_candidate_attributes();
cudaError_t init_select_attributes();
cudaError_t launch_candidates(const CandArgs& a, int local_blocks, cudaStream_t s);
cudaError_t launch_sample_tensor(const Dims& dm, Key key, uint32_t iter, const float* umin,
                                 const float* umax, float* Z, int32_t* I, float* C,
                                 cudaStream_t s);
// Rollouts: `chunk` is the horizon chunk of staged control loads (4 or 8
// steps; 0, or a launch that cannot stage, loads directly).
cudaError_t init_rollout_pm_attributes();
cudaError_t init_rollout_chain_attributes();
cudaError_t init_rollout_pm_batch_attributes();
cudaError_t init_rollout_chain_batch_attributes();
cudaError_t launch_rollout_pointmass(const RolloutArgs& a, const PointMassModel& m, int chunk,
                                     cudaStream_t s);
cudaError_t launch_rollout_chain(const RolloutArgs& a, const ChainModel& m, int links, int chunk,
                                 cudaStream_t s);
cudaError_t launch_rollout_legged(const RolloutArgs& a, const LeggedModel& m, int links,
                                  cudaStream_t s);
cudaError_t launch_rollout_legged_batch(const RolloutArgs* d_ra, const LeggedModel* d_lm,
                                        const int* d_row_start, int count, int total_rows,
                                        int links, cudaStream_t s);
// The rollouts of many instances in one persistent launch
// (rollout_persist.cu): warp tiles of 32 candidates, taken in order from a
// device counter by every warp of the launch.  Entry k of the tables is one
// instance, group by group and within a group longest expected rollout
// first: its position in the batch's
// RolloutArgs, its model, its code (dynamics | dimension << 8 | staged << 16)
// and its first warp tile wstart[k] (count + 1 entries).  Point masses of up
// to kPersistMaxAxes axes and chains of up to kPersistMaxLinks links.
constexpr int kPersistMaxAxes = 16;
constexpr int kPersistMaxLinks = 9;
struct PersistArgs {
  const RolloutArgs* ra;
  const PointMassModel* pm;
  const ChainModel* cm;
  const int* order;
  const int* wstart;
  const int* code;
  const int* model;
  unsigned* head;     // the tile counter, zeroed by the launch
  int count, total_warps;
  int w_base;         // wstart[0]: the first tile of these entries in the batch's numbering
  size_t warp_bytes;  // shared memory per warp: two mbarriers and two staging buffers (0: no staging)
};
// Shared memory per warp for staged tiles of at most these widths (0: none).
size_t persist_warp_bytes(int max_pm_axes_staged, int max_links_staged);
// Resident 128-thread CTAs per SM of the persistent launch with that much
// shared memory per warp (0 on error); also sets the launch's shared-memory
// attribute.
int persist_blocks_per_sm(size_t warp_bytes);
cudaError_t launch_rollout_persistent(const PersistArgs& p, int blocks_per_sm, cudaStream_t s);
// Def. 2 graph rows on the tensor cores (BF16 operands, FP32 sums): whether a
// generation's graph part goes there (BF16 B-spline, H <= 256, M <= 64,
// n <= 16), its tile count, and the launches (standalone and over many
// instances, tile_start numbering each instance's first tile).  The graph Z
// must be in global memory (Z_global) unless C_in is given.
bool bspline_tc_eligible(const CandArgs& a);
int bspline_tc_tiles(const CandArgs& a);
cudaError_t init_bspline_tc_attributes();
cudaError_t launch_bspline_tc(const CandArgs& a, cudaStream_t s);
cudaError_t launch_bspline_tc_batch(const CandArgs* d_args, const int* d_tile_start, int count,
                                    int total_tiles, cudaStream_t s);
cudaError_t launch_select(const SelectArgs& a, cudaStream_t s);
// Two-stage selection for B beyond one block: chunks > 0 stages of `chunk`
// costs each (select_plan; chunks = 0: one block suffices, -1: too large).
void select_plan(int B, int E, int* chunk, int* chunks);
cudaError_t launch_select_two_stage(const SelectArgs& a, int chunk, int chunks, cudaStream_t s);
size_t select_smem_bytes(int B, int E);
cudaError_t launch_update(const UpdateArgs& a, cudaStream_t s);
// batched forms: one launch over many planning problems
cudaError_t launch_graph_Z(const CandArgs& a, float* Z, cudaStream_t s);
// Pipelined generation of the next iteration (graph rows and local draws of
// iteration d_iter + iter_offset) by `grid` persistent blocks that each take
// a whole SM's shared memory, so that they only run on SMs no other kernel
// occupies; and the finishing pass of the local rows and the mean row.
cudaError_t init_prepare_attributes(size_t* dyn_smem);
size_t prepare_smem_need(const CandArgs& a);
cudaError_t launch_prepare(const CandArgs& a, int grid, size_t dyn_smem, cudaStream_t s);
cudaError_t launch_finish(const CandArgs& a, int blocks, cudaStream_t s);
// Blocks of the standalone rollout launch for `rows` candidates (point mass
// and chain; the legged rollout is not counted here).
int rollout_blocks(int rows);
cudaError_t launch_local_batch(const CandArgs* d_args, const int* d_local_start, int count,
                               int total_blocks, cudaStream_t s);
cudaError_t launch_graph_Z_batch(const CandArgs* d_args, float* const* d_Z, const int* d_block_start,
                                 int count, int total_blocks, cudaStream_t s);
cudaError_t launch_candidates_batch(const CandArgs* d_args, const int* d_block_start, int count,
                                    int total_blocks, size_t smem, cudaStream_t s);
cudaError_t launch_rollout_pointmass_batch(const RolloutArgs* d_ra, const PointMassModel* d_pm,
                                           const int* d_row_start, int count, int total_rows,
                                           int k, int block, int chunk, int samples,
                                           cudaStream_t s);
cudaError_t launch_rollout_chain_batch(const RolloutArgs* d_ra, const ChainModel* d_cm,
                                       const int* d_row_start, int count, int total_rows,
                                       int links, int block, int chunk, cudaStream_t s);
cudaError_t launch_select_batch(const SelectArgs* d_args, int count, size_t smem, cudaStream_t s);
cudaError_t launch_update_batch(const UpdateArgs* d_args, const int* d_thread_start, int count,
                                int total_threads, cudaStream_t s);
int update_threads(int H, int n);  // threads one instance's update gets in a batch
cudaError_t launch_scatter(const float* packed, float* const* d_dst, const int* d_off, int count,
                           cudaStream_t s);
cudaError_t launch_gather(const float* const* d_src, const int* d_off, float* packed, int count,
                          cudaStream_t s);
cudaError_t launch_shift_batch(const UpdateArgs* d_args, int count, int k, cudaStream_t s);
cudaError_t launch_shift(double* mu, double* sigma, float* mu_f, float* sigma_f, int H, int n, int k,
                         cudaStream_t s);

}  // namespace mtp
