// handle.cuh -- the planner handle shared by the C ABI's single-instance
// (mtp_abi.cu) and batched (batch_abi.cu) parts: its device state and the
// argument builders of its kernels.  Internal to the library.
#pragma once

#include <map>
#include <string>
#include <vector>

#include "mtp_device.cuh"

struct mtp_handle {
  mtp_problem pr{};
  mtp::Dims dm{};
  int device = 0;
  mtp::Key key{};
  // interpolation tables
  float* basis = nullptr;
  int32_t* bfirst = nullptr;
  int32_t* seg = nullptr;
  float* delta = nullptr;
  float inv_h = 1.f;
  int paths_per_block = 1;
  bool global_Z = false;  // Z written once per iteration instead of per graph block
  // planner state
  double* mu = nullptr;
  double* sigma = nullptr;
  float* mu_f = nullptr;     // FP32 copies read by the samplers
  float* sigma_f = nullptr;
  uint32_t* iter_dev = nullptr;
  uint32_t iter_host = 0;
  // scratch of one iteration
  float* U = nullptr;  // candidates of the latest iteration: Ubuf[cur]
  // Pipelined generation.  Everything costly in an iteration's candidates
  // (the graph rows and the local rows' standard normal draws) depends only
  // on the key and the iteration number, not on the mean and spread.  When
  // the rollout leaves SMs idle, a single-instance iteration therefore
  // makes the next iteration's graph rows (and, with many idle SMs, its
  // draws) on those SMs while its rollout runs (on `side`), into the other
  // candidate buffer; the next iteration then only makes (or finishes) its
  // local rows and mean row.
  bool pipeline = false;
  bool prep_local = false;    // the local draws are prepared too (else only the graph rows)
  float* Ubuf[2] = {nullptr, nullptr};
  int cur = 0;                // Ubuf[cur] holds the latest iteration's candidates
  bool prep_valid = false;    // Ubuf[cur ^ 1] holds the draws and graph rows of prep_iter
  uint32_t prep_iter = 0;
  int prep_grid = 0;          // SMs the rollout leaves free
  int prep_spb = 1;           // graph paths per pass of a k_prepare block
  size_t prep_smem = 0;       // dynamic shared memory of a k_prepare block (a whole SM)
  cudaStream_t side = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  float* cost = nullptr;
  int32_t* elite = nullptr;
  double* weight = nullptr;
  float* ustar = nullptr;
  float* x0 = nullptr;
  float* Z = nullptr;  // (M, N, n) graph of the current iteration (batched planning)
  uint32_t* status = nullptr;  // device status word: bits a rollout sets when a bounded wait gave up
  int rollout_chunk = 0;       // horizon chunk of the staged control loads of a lone rollout (0: direct)
  bool tc_graph = false;       // graph rows contracted on the tensor cores (BF16 B-spline)
  double* entropy = nullptr;   // last iteration's cost entropy (MTP_FLAG_COST_ENTROPY)
  // two-stage elite selection (B beyond one block): chunk length, chunk
  // count (0: one block) and the chunks' (key, index) pairs
  int sel_chunk = 0, sel_chunks = 0;
  unsigned long long* sel_pairs = nullptr;
  // replay
  cudaStream_t cap_stream = nullptr;
  std::map<int, cudaGraphExec_t> graphs;   // key: (iterations, cur, first prepared)
  std::map<int, cudaGraphExec_t> hgraphs;  // the same with the host-pointer step's copies
  float* x0_pin = nullptr;                 // pinned staging of mtp_plan_step_host: start state
  float* ustar_pin = nullptr;              // and u*, written by the selection kernel
  // profiling
  bool profiling = false;
  std::vector<cudaEvent_t> events;  // eager launches: kEvPerIter per iteration, read by mtp_stage_times
  size_t ev_used = 0;
  std::vector<cudaEvent_t> gevents;            // inside profiled graphs: kEvPerIter per iteration
  std::map<int, cudaGraphExec_t> pgraphs;      // graphs with the stage events captured
  double stage_acc[5] = {0, 0, 0, 0, 0};       // read from gevents after each profiled replay
  int64_t stage_iters = 0;
  std::string err;
};

namespace mtp {

// Makes `dev` current for the scope and restores the previous device.
struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
    else prev = -1;
  }
  ~DeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

// Akima paths per block where blocks do not end the critical path: the
// persistent preparation and the batched launch (measured on the 7-link arm:
// 8 / 16 / 32 paths prepare an iteration's graph rows in 57 / 45 / 37 us; the
// batch of 256 instances takes 3.78 / 3.72 / 3.70 ms; a lone unpipelined arm
// generates in 16.4 / 18.4 / 25 us, where the last blocks set the time).
constexpr int kWideAkimaPaths = 32;

// Kernel arguments of a handle's iteration (the iteration from d_iter when set).
CandArgs cand_args(const mtp_handle* h, uint32_t iter, const uint32_t* d_iter);
RolloutArgs rollout_args(const mtp_handle* h, uint32_t iter, const uint32_t* d_iter,
                         const float* x0, const float* U, int row0, int rows, float* cost);
PointMassModel pointmass_model(const mtp_problem& p);
ChainModel chain_model(const mtp_problem& p);
LeggedModel legged_model(const mtp_problem& p);

}  // namespace mtp
