// batch_abi.cu -- batched planning over many handles (the mtp_batch_* calls
// of include/mtp.h): device tables of all instances, one CUDA graph per
// iteration, rollouts grouped by (dynamics, control dimension) on their own
// streams, and the rollout-tile autotuner.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "handle.cuh"

using namespace mtp;

// ---------------------------------------------------------------------------
// Batched planning over many handles
// ---------------------------------------------------------------------------

namespace {

struct BatchGroup {
  int dyn = 0, n = 0;
  int first = 0, count = 0;   // instances [first, first + count) of the sorted order
  int model_first = 0;        // first model of this group in its dynamics' table
  int rows_first = 0;         // offset of this group's row_start segment
  int total_rows = 0;
  int block = 128;
  int chunk = 0;              // horizon chunk of staged control loads (0: direct loads)
  int samples = 1;            // candidates per thread (point masses: 1 or 2, direct loads)
  bool stageable = false;     // every member's rows can be staged (see can_stage)
  bool pairable = false;      // point masses with one model per candidate: 2 per thread allowed
  // this group's share of the generation, selection and update launches
  int z_blocks = 0, cand_blocks = 0, local_blocks = 0, upd_threads = 0;
  // members whose graph rows are contracted on the tensor cores (BF16 basis):
  // entries [tc_first, tc_first + tc_count) of the tensor-core argument list,
  // their tile numbering at tc_start_first of d_tc_start
  int tc_first = 0, tc_count = 0, tc_start_first = 0, tc_tiles = 0;
  size_t cand_smem = 0, sel_smem = 0;
  double est = 0.0;  // expected rollout time (ms): sets the groups' launch order
};

constexpr int kMaxGroups = 64;
// Two-launch persistent mode: the first launch takes the groups that make up
// this fraction of the expected rollout work, and runs this many CTAs per SM
// fewer than the second, leaving them to the second part's generation.
// Measured on the batch of 256 (ms per iteration): fraction 0.35 / 0.5 /
// 0.65 / 0.75 / 0.85: 2.84 / 2.74-2.75 / 2.73 / 2.77 / 2.98 (0.65 measured
// again with the later point-mass change: 2.69 against 2.77 / 2.98); the
// first launch with as many CTAs as the second: 2.81.
#ifndef MTP_PERSIST_SPLIT_FRACTION
#define MTP_PERSIST_SPLIT_FRACTION 0.65
#endif
#ifndef MTP_PERSIST_FIRST_FEWER
#define MTP_PERSIST_FIRST_FEWER 1
#endif
constexpr double kPersistSplitFraction = MTP_PERSIST_SPLIT_FRACTION;
constexpr int kPersistFirstFewer = MTP_PERSIST_FIRST_FEWER;
// Horizon chunk of staged control loads before the autotuner has run.
constexpr int kDefaultChunk = 4;
constexpr size_t kBatchGraphSmem = 40 * 1024;  // four graph blocks per SM
constexpr int kLocalRowsPerThreadBatch = 16;

// Device tables of a batch, packed into one device block that is refilled in
// place from a pinned host mirror with one copy.  The layout depends on the
// instance count, so the pointers are set on every fill.
struct BatchTables {
  int cap = 0;
  size_t block_bytes = 0;
  unsigned char* d_block = nullptr;
  unsigned char* h_block = nullptr;  // pinned mirror
  cudaEvent_t copied = nullptr;      // the mirror's last copy has been read
  CandArgs* d_cand = nullptr;
  int* d_cand_start = nullptr;
  int* d_local_start = nullptr;
  CandArgs* d_tc = nullptr;     // graph parts contracted on the tensor cores, in group order
  int* d_tc_start = nullptr;    // one segment of (members + 1) tile offsets per group
  float** d_Z = nullptr;
  int* d_z_start = nullptr;
  RolloutArgs* d_ra = nullptr;  // in group order
  PointMassModel* d_pm = nullptr;
  ChainModel* d_cm = nullptr;
  LeggedModel* d_lm = nullptr;
  int* d_row_start = nullptr;  // one segment of (members + 1) entries per group
  SelectArgs* d_sel = nullptr;
  UpdateArgs* d_upd = nullptr;
  int* d_warp_start = nullptr;
  float** d_x0_dst = nullptr;
  float** d_ustar_src = nullptr;
  int* d_x0_off = nullptr;
  int* d_us_off = nullptr;
  // the persistent rollout launch: one entry per instance it covers, group
  // by group, longest expected rollout first within a group (PersistArgs)
  int* d_p_order = nullptr;
  int* d_p_wstart = nullptr;
  int* d_p_code = nullptr;
  int* d_p_model = nullptr;
  unsigned* d_p_head = nullptr;
};

// Packs the tables of `count` instances (n_pm point masses, n_cm chains,
// n_lm legged robots, `groups` rollout groups) at 64-byte boundaries; with
// `base` null it only returns the size.
size_t layout_tables(BatchTables* t, unsigned char* base, int count, int n_pm, int n_cm, int n_lm,
                     int groups) {
  size_t off = 0;
  auto take = [&](auto** field, size_t n) {
    using T = std::remove_pointer_t<std::remove_reference_t<decltype(*field)>>;
    off = (off + 63) & ~size_t(63);
    if (base) *field = reinterpret_cast<T*>(base + off);
    off += sizeof(T) * n;
  };
  BatchTables dummy;
  BatchTables* d = t ? t : &dummy;
  take(&d->d_cand, count);
  take(&d->d_cand_start, count + 1);
  take(&d->d_local_start, count + 1);
  take(&d->d_tc, count);
  take(&d->d_tc_start, count + groups);
  take(&d->d_Z, count);
  take(&d->d_z_start, count + 1);
  take(&d->d_ra, count);
  take(&d->d_pm, n_pm);
  take(&d->d_cm, n_cm);
  take(&d->d_lm, n_lm);
  take(&d->d_row_start, count + groups);
  take(&d->d_sel, count);
  take(&d->d_upd, count);
  take(&d->d_warp_start, count + 1);
  take(&d->d_x0_dst, count);
  take(&d->d_ustar_src, count);
  take(&d->d_x0_off, count + 1);
  take(&d->d_us_off, count + 1);
  take(&d->d_p_order, count);
  take(&d->d_p_wstart, count + 1);
  take(&d->d_p_code, count);
  take(&d->d_p_model, count);
  take(&d->d_p_head, 2);
  return off;
}

}  // namespace

struct mtp_batch {
  std::vector<mtp_handle*> hs;         // in the caller's order
  std::vector<mtp_handle*> hs_sorted;  // in group order (groups[g].first indexes it)
  int device = 0;
  BatchTables t;
  int count = 0;
  std::vector<BatchGroup> groups;
  // (dyn, n) -> rollout tile chosen by the autotuner: (candidates per block, horizon chunk,
  // candidates per thread)
  std::map<std::pair<int, int>, std::array<int, 3>> tuned;
  // (dyn, n) -> the autotuner's rollout time of the group (ms) per rollout step
  std::map<std::pair<int, int>, double> tuned_ms_per_step;
  // groups in launch order: longest expected rollout first
  std::vector<int> launch_order;
  std::vector<int> x0_off, us_off;
  cudaStream_t cap_stream = nullptr;
  cudaEvent_t fork_ev = nullptr;
  cudaStream_t group_stream[kMaxGroups] = {};
  cudaEvent_t group_done[kMaxGroups] = {};
  std::map<int, cudaGraphExec_t> graphs;  // key: graph_key(iterations, cur, first prepared)
  int runs_since_fill = 0;
  // How the rollouts run (MTP_BATCH_ROLLOUT_*): one launch per group on its
  // stream, or the point-mass and chain groups (up to kPersistMaxAxes axes,
  // kPersistMaxLinks links) in one persistent launch, their tiles staged or
  // loaded directly.
  int rollout_mode = MTP_BATCH_ROLLOUT_GROUPS;
  std::vector<char> covered;    // per group: its rollouts are in the persistent launch
  int p_count = 0, p_total_warps = 0;
  // the two-launch persistent mode: entries [0, p_split) and [p_split,
  // p_count), split at a group boundary near half of the expected work;
  // groups of launch rank < p_split_rank are in the first launch
  int p_split = 0, p_split_warps = 0, p_split_rank = 0;
  cudaStream_t persist_stream[2] = {nullptr, nullptr};
  cudaEvent_t persist_ev2 = nullptr;
  cudaStream_t group_stream_hi[kMaxGroups] = {};  // high priority: the first launch's generation
  size_t p_warp_bytes = 0;      // staged tiles' shared memory per warp (0: none stageable)
  int p_blocks[2] = {0, 0};     // resident CTAs per SM: staged mode, direct mode
  cudaEvent_t persist_ev = nullptr;
  double mode_ms[4] = {0, 0, 0, 0};  // the autotuner's iteration time per mode (0: not timed)
  std::string err;
};

namespace {

// Groups are launched longest first.  The GPU takes a launch's blocks in
// the order the launches arrive, and the groups' rollouts are long,
// latency-bound launches: enqueued last, the longest groups would start
// only when the earlier ones had drained and end the iteration alone
// (measured on the batch of 256: the 9-link chains started 2.4 ms into a
// 3.3 ms iteration).  A group's expected time is its rollout steps times the
// autotuner's time per step for its (dynamics, dimension), or before
// tuning a per-step cost model: the chains' step grows with the square of
// the link count (the mass matrix and its factorisation), the point mass
// step with its axes.
template <class StepsFn>
void set_launch_order(mtp_batch* b, StepsFn steps_of) {
  for (auto& g : b->groups) {
    const double steps = (double)steps_of(g);
    auto it = b->tuned_ms_per_step.find({g.dyn, g.n});
    if (it != b->tuned_ms_per_step.end()) {
      g.est = steps * it->second;
    } else {
      const double w = g.dyn == MTP_DYN_POINTMASS ? 40.0 * g.n : 12.0 * g.n * g.n;  // instructions per step
      g.est = steps * w * 1e-9;
    }
  }
  b->launch_order.resize(b->groups.size());
  for (size_t i = 0; i < b->groups.size(); ++i) b->launch_order[i] = (int)i;
  std::stable_sort(b->launch_order.begin(), b->launch_order.end(),
                   [&](int x, int y) { return b->groups[x].est > b->groups[y].est; });
}

mtp_status batch_fail(mtp_batch* b, mtp_status st, const std::string& msg) {
  if (b) b->err = msg;
  mtp::set_thread_error(msg);
  return st;
}

void drop_graphs(mtp_batch* b) {
  for (auto& kv : b->graphs) cudaGraphExecDestroy(kv.second);
  b->graphs.clear();
}

void free_batch(mtp_batch* b) {
  drop_graphs(b);
  if (b->t.d_block) cudaFree(b->t.d_block);
  if (b->t.h_block) cudaFreeHost(b->t.h_block);
  if (b->t.copied) cudaEventDestroy(b->t.copied);
  for (int g = 0; g < kMaxGroups; ++g) {
    if (b->group_stream[g]) cudaStreamDestroy(b->group_stream[g]);
    if (b->group_done[g]) cudaEventDestroy(b->group_done[g]);
  }
  if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
  if (b->fork_ev) cudaEventDestroy(b->fork_ev);
  if (b->persist_ev) cudaEventDestroy(b->persist_ev);
  if (b->persist_ev2) cudaEventDestroy(b->persist_ev2);
  for (int k = 0; k < 2; ++k)
    if (b->persist_stream[k]) cudaStreamDestroy(b->persist_stream[k]);
  for (int g = 0; g < kMaxGroups; ++g)
    if (b->group_stream_hi[g]) cudaStreamDestroy(b->group_stream_hi[g]);
  delete b;
}

cudaError_t alloc_batch(mtp_batch* b, int cap) {
  BatchTables& t = b->t;
  t.cap = cap;
  // every instance could be of any dynamics and every one its own group
  t.block_bytes = layout_tables(nullptr, nullptr, cap, cap, cap, cap, std::min(cap, kMaxGroups));
  cudaError_t e;
  if ((e = cudaMalloc((void**)&t.d_block, t.block_bytes)) ||
      (e = cudaMallocHost((void**)&t.h_block, t.block_bytes)) ||
      (e = cudaEventCreateWithFlags(&t.copied, cudaEventDisableTiming)) ||
      (e = cudaEventRecord(t.copied, 0)) ||
      (e = cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking)) ||
      (e = cudaEventCreateWithFlags(&b->fork_ev, cudaEventDisableTiming)) ||
      (e = cudaEventCreateWithFlags(&b->persist_ev, cudaEventDisableTiming)) ||
      (e = cudaEventCreateWithFlags(&b->persist_ev2, cudaEventDisableTiming)) ||
      (e = cudaStreamCreateWithFlags(&b->persist_stream[0], cudaStreamNonBlocking)) ||
      (e = cudaStreamCreateWithFlags(&b->persist_stream[1], cudaStreamNonBlocking)))
    return e;
  return cudaSuccess;
}

int group_key_n(const mtp_handle* h) {
  return h->pr.dyn == MTP_DYN_POINTMASS ? h->dm.n : h->pr.n_links;
}

// Fills the batch's tables for `handles` (at most the capacity, distinct,
// on the batch's device) with one host-to-device copy on `s`.  Instances are
// grouped by (dynamics, dimension) for the rollouts; everything else keeps
// the caller's order.  Captured graphs are dropped: their launches baked in
// the previous layout.
cudaError_t fill_batch(mtp_batch* b, mtp_handle* const* handles, int count, cudaStream_t s) {
  BatchTables& t = b->t;
  cudaError_t e;
  if ((e = cudaEventSynchronize(t.copied))) return e;  // the mirror is free again
  drop_graphs(b);
  b->runs_since_fill = 0;
  b->count = 0;  // unusable until this fill has succeeded
  b->hs.clear();
  // rollout groups: sorted by (dynamics, dimension), stable in the caller's order
  std::vector<int> order(count);
  for (int i = 0; i < count; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
    const int dx = handles[x]->pr.dyn, dy = handles[y]->pr.dyn;
    if (dx != dy) return dx < dy;
    return group_key_n(handles[x]) < group_key_n(handles[y]);
  });
  b->groups.clear();
  int n_dyn[3] = {0, 0, 0};
  for (int pos = 0; pos < count; ++pos) {
    const mtp_handle* h = handles[order[pos]];
    const int dyn = h->pr.dyn, n = group_key_n(h);
    if (b->groups.empty() || b->groups.back().dyn != dyn || b->groups.back().n != n) {
      if ((int)b->groups.size() == kMaxGroups) return cudaErrorInvalidValue;
      BatchGroup g;
      g.dyn = dyn;
      g.n = n;
      g.first = pos;
      g.model_first = n_dyn[dyn];
      auto it = b->tuned.find({dyn, n});
      g.block = it != b->tuned.end() ? it->second[0] : 128;
      g.chunk = it != b->tuned.end() ? it->second[1] : kDefaultChunk;
      g.samples = it != b->tuned.end() ? it->second[2] : 1;
      b->groups.push_back(g);
    }
    ++b->groups.back().count;
    ++n_dyn[dyn];
  }
  layout_tables(&t, t.h_block, count, n_dyn[MTP_DYN_POINTMASS], n_dyn[MTP_DYN_CHAIN],
                n_dyn[MTP_DYN_LEGGED], (int)b->groups.size());
  // host views of the mirror (same offsets as the device block)
  BatchTables hv = t;
  const size_t used = layout_tables(&t, t.d_block, count, n_dyn[MTP_DYN_POINTMASS],
                                    n_dyn[MTP_DYN_CHAIN], n_dyn[MTP_DYN_LEGGED], (int)b->groups.size());
  // candidate generation, selection and update tables in group order, so
  // that each group's stream launches them over a contiguous range
  hv.d_cand_start[0] = hv.d_z_start[0] = hv.d_local_start[0] = hv.d_warp_start[0] = 0;
  std::vector<CandArgs> tc_args(count);
  std::vector<char> is_tc(count, 0);
  for (int pos = 0; pos < count; ++pos) {
    mtp_handle* h = handles[order[pos]];
    // a batch makes every iteration's candidates in full, in the first buffer
    h->cur = 0;
    h->U = h->Ubuf[0];
    h->prep_valid = false;
    const Dims& dm = h->dm;
    const size_t Hn = (size_t)dm.H * dm.n;
    CandArgs c = cand_args(h, 0, h->iter_dev);
    c.U_graph = h->U + Hn * dm.L;
    c.graph_rows = dm.P;
    c.U_local = h->U;
    c.local_rows = dm.L;
    c.U_mean = h->U + Hn * (dm.B - 1);
    c.Z_global = h->Z;
    // one launch gives every block the largest instance's shared memory, so
    // paths per block shrink until the instance fits kBatchGraphSmem (a
    // path's values do not depend on how paths are grouped into blocks)
    c.paths_per_block = std::max(h->paths_per_block, kWideAkimaPaths * (h->pr.interp == MTP_INTERP_AKIMA));
    c.graph_blocks = 1;  // counts the graph part in candidates_smem_bytes
    while (c.paths_per_block > 1 && candidates_smem_bytes(c) > kBatchGraphSmem) c.paths_per_block /= 2;
    c.graph_blocks = (dm.P + c.paths_per_block - 1) / c.paths_per_block;
    if (h->tc_graph && bspline_tc_eligible(c)) {
      tc_args[pos] = c;     // its graph rows go to the tensor cores
      is_tc[pos] = 1;
      c.graph_blocks = 0;
      c.paths_per_block = 1;
    }
    hv.d_Z[pos] = h->Z;
    hv.d_z_start[pos + 1] = hv.d_z_start[pos] + (dm.M * dm.N * ((dm.n + 3) / 4) + 255) / 256;
    const long long items = ((long long)dm.L + 1) * (((long long)Hn + 3) / 4);
    hv.d_cand[pos] = c;
    hv.d_cand_start[pos + 1] = hv.d_cand_start[pos] + c.graph_blocks;  // local rows run apart
    // 16 groups of four elements per thread: each thread's set-up (instance
    // search, box, its group's mean and spread) is paid once for 16 rows
    hv.d_local_start[pos + 1] =
        hv.d_local_start[pos] + (int)std::max<long long>(1, (items + 256 * kLocalRowsPerThreadBatch - 1) /
                                                                (256 * kLocalRowsPerThreadBatch));
    hv.d_sel[pos] = SelectArgs{h->cost, h->U, dm.B, dm.E, dm.H, dm.n, 1.0 / h->pr.lambda, h->pr.update_rule,
                               h->elite, h->weight, h->ustar, nullptr, nullptr, h->entropy};
    hv.d_upd[pos] = UpdateArgs{h->U, h->elite, h->weight, dm.E, dm.H, dm.n, h->pr.alpha, h->pr.sigma_min,
                               h->pr.update_rule, h->mu, h->sigma, h->mu_f, h->sigma_f, h->iter_dev};
    hv.d_warp_start[pos + 1] = hv.d_warp_start[pos] + update_threads(dm.H, dm.n);
  }
  // tensor-core members, group by group
  {
    int tc_pos = 0, seg = 0;
    for (auto& g : b->groups) {
      g.tc_first = tc_pos;
      g.tc_start_first = seg;
      int tiles = 0;
      hv.d_tc_start[seg] = 0;
      for (int pos = g.first; pos < g.first + g.count; ++pos) {
        if (!is_tc[pos]) continue;
        hv.d_tc[tc_pos++] = tc_args[pos];
        tiles += bspline_tc_tiles(tc_args[pos]);
        hv.d_tc_start[seg + (tc_pos - g.tc_first)] = tiles;
      }
      g.tc_count = tc_pos - g.tc_first;
      g.tc_tiles = tiles;
      seg += g.tc_count + 1;
    }
  }
  for (auto& g : b->groups) {
    const int a0 = g.first, a1 = g.first + g.count;
    g.z_blocks = hv.d_z_start[a1] - hv.d_z_start[a0];
    g.cand_blocks = hv.d_cand_start[a1] - hv.d_cand_start[a0];
    g.local_blocks = hv.d_local_start[a1] - hv.d_local_start[a0];
    g.upd_threads = hv.d_warp_start[a1] - hv.d_warp_start[a0];
    g.cand_smem = g.sel_smem = 0;
    for (int pos = a0; pos < a1; ++pos) {
      g.cand_smem = std::max(g.cand_smem, candidates_smem_bytes(hv.d_cand[pos]));
      g.sel_smem = std::max(g.sel_smem, select_smem_bytes(hv.d_sel[pos].B, hv.d_sel[pos].E));
    }
  }
  // rollouts, in group order; whole warps per instance
  int rs = 0;
  for (auto& g : b->groups) {
    g.rows_first = rs;
    int* row = hv.d_row_start + rs;
    row[0] = 0;
    for (int j = 0; j < g.count; ++j) {
      mtp_handle* h = handles[order[g.first + j]];
      hv.d_ra[g.first + j] = rollout_args(h, 0, h->iter_dev, h->x0, h->U, 0, h->dm.B, h->cost);
      const int m = g.model_first + j;
      if (g.dyn == MTP_DYN_POINTMASS) hv.d_pm[m] = pointmass_model(h->pr);
      else if (g.dyn == MTP_DYN_LEGGED) hv.d_lm[m] = legged_model(h->pr);
      else hv.d_cm[m] = chain_model(h->pr);
      // whole warps per instance; point masses whole pairs of warps (two
      // candidates per thread take rows 32 apart)
      const int pad = g.dyn == MTP_DYN_POINTMASS ? 64 : 32;
      row[j + 1] = row[j] + ((h->dm.B + pad - 1) / pad) * pad;
    }
    g.total_rows = row[g.count];
    g.stageable = g.dyn != MTP_DYN_LEGGED;
    for (int j = 0; j < g.count; ++j)
      g.stageable = g.stageable && can_stage(hv.d_ra[g.first + j], group_key_n(handles[order[g.first + j]]));
    if (!g.stageable) g.chunk = 0;
    g.pairable = g.dyn == MTP_DYN_POINTMASS;
    for (int j = 0; j < g.count; ++j)
      g.pairable = g.pairable && hv.d_ra[g.first + j].dr_mode != MTP_DR_SHARED;
    if (!g.pairable) g.samples = 1;
    if (g.samples == 2) g.chunk = 0;
    rs += g.count + 1;
  }
  set_launch_order(b, [&](const BatchGroup& g) {
    long long steps = 0;
    for (int j = 0; j < g.count; ++j) {
      const mtp_handle* h = handles[order[g.first + j]];
      steps += (long long)h->dm.B * h->dm.H;
    }
    return steps;
  });
  // the persistent launch's entries: every instance of a covered group,
  // ordered below (H steps at the group's time per step sets a tile's length)
  {
    b->covered.assign(b->groups.size(), 0);
    struct Entry {
      double est;
      int pos, code, model, warps;
    };
    std::vector<Entry> ent;
    int max_pm = 0, max_links = 0;
    for (size_t gi = 0; gi < b->groups.size(); ++gi) {
      const BatchGroup& g = b->groups[gi];
      const bool cov = (g.dyn == MTP_DYN_POINTMASS && g.n <= kPersistMaxAxes) ||
                       (g.dyn == MTP_DYN_CHAIN && g.n <= kPersistMaxLinks);
      if (!cov || g.total_rows <= 0) continue;
      b->covered[gi] = 1;
      auto it = b->tuned_ms_per_step.find({g.dyn, g.n});
      const double per_step = it != b->tuned_ms_per_step.end()
                                  ? it->second
                                  : (g.dyn == MTP_DYN_POINTMASS ? 40.0 * g.n : 12.0 * g.n * g.n) * 1e-9;
      for (int j = 0; j < g.count; ++j) {
        const int pos = g.first + j;
        const mtp_handle* h = handles[order[pos]];
        const bool stage = can_stage(hv.d_ra[pos], g.n);
        if (stage) (g.dyn == MTP_DYN_POINTMASS ? max_pm : max_links) = std::max(
                       g.dyn == MTP_DYN_POINTMASS ? max_pm : max_links, g.n);
        ent.push_back({per_step * h->dm.H, pos, g.dyn | (g.n << 8) | (stage ? 1 << 16 : 0),
                       g.model_first + j, (h->dm.B + 31) / 32});
      }
    }
    // groups in their launch order (longest group first), and within a group
    // the longest tiles first: warps that run at the same time then mostly
    // run the same body, which keeps the instruction cache warm (with every
    // tile ordered by length alone, warps of one SM ran different bodies and
    // half of their stall samples were instruction fetches)
    std::vector<int> group_rank(b->groups.size(), 0);
    for (size_t r = 0; r < b->launch_order.size(); ++r) group_rank[b->launch_order[r]] = (int)r;
    std::vector<int> entry_group;
    for (const Entry& en : ent) {
      int gi = 0;
      while (!(en.pos >= b->groups[gi].first && en.pos < b->groups[gi].first + b->groups[gi].count)) ++gi;
      entry_group.push_back(group_rank[gi]);
    }
    std::vector<int> idx(ent.size());
    for (size_t k = 0; k < idx.size(); ++k) idx[k] = (int)k;
    std::stable_sort(idx.begin(), idx.end(), [&](int x, int y) {
      if (entry_group[x] != entry_group[y]) return entry_group[x] < entry_group[y];
      return ent[x].est > ent[y].est;
    });
    std::vector<Entry> sorted;
    std::vector<int> sorted_group;
    for (int k : idx) {
      sorted.push_back(ent[k]);
      sorted_group.push_back(entry_group[k]);
    }
    ent.swap(sorted);
    int w = 0;
    for (size_t k = 0; k < ent.size(); ++k) {
      hv.d_p_order[k] = ent[k].pos;
      hv.d_p_code[k] = ent[k].code;
      hv.d_p_model[k] = ent[k].model;
      hv.d_p_wstart[k] = w;
      w += ent[k].warps;
    }
    hv.d_p_wstart[ent.size()] = w;
    hv.d_p_head[0] = hv.d_p_head[1] = 0u;
    {
      double total = 0.0, acc = 0.0;
      for (const Entry& en : ent) total += en.est * en.warps;
      b->p_split = (int)ent.size();
      b->p_split_rank = (int)b->groups.size();
      for (size_t k = 0; k < ent.size(); ++k) {
        if (k > 0 && sorted_group[k] != sorted_group[k - 1] && acc >= kPersistSplitFraction * total) {
          b->p_split = (int)k;
          b->p_split_rank = sorted_group[k];
          break;
        }
        acc += ent[k].est * ent[k].warps;
      }
      b->p_split_warps = hv.d_p_wstart[b->p_split];
    }
    b->p_count = (int)ent.size();
    b->p_total_warps = w;
    b->p_warp_bytes = persist_warp_bytes(max_pm, max_links);
    b->p_blocks[0] = persist_blocks_per_sm(b->p_warp_bytes);
    b->p_blocks[1] = persist_blocks_per_sm(0);
    if (b->p_count > 0 && (b->p_blocks[0] < 1 || b->p_blocks[1] < 1)) return cudaErrorInvalidConfiguration;
  }
  // packing of x0 and u*, in the caller's order
  b->x0_off.assign(count + 1, 0);
  b->us_off.assign(count + 1, 0);
  hv.d_x0_off[0] = hv.d_us_off[0] = 0;
  for (int i = 0; i < count; ++i) {
    mtp_handle* h = handles[i];
    hv.d_x0_dst[i] = h->x0;
    hv.d_ustar_src[i] = h->ustar;
    b->x0_off[i + 1] = b->x0_off[i] + h->dm.d;
    b->us_off[i + 1] = b->us_off[i] + h->dm.n;
    hv.d_x0_off[i + 1] = b->x0_off[i + 1];
    hv.d_us_off[i + 1] = b->us_off[i + 1];
  }
  if ((e = cudaMemcpyAsync(t.d_block, t.h_block, used, cudaMemcpyHostToDevice, s)) ||
      (e = cudaEventRecord(t.copied, s)))
    return e;
  b->hs.assign(handles, handles + count);
  b->hs_sorted.resize(count);
  for (int pos = 0; pos < count; ++pos) b->hs_sorted[pos] = handles[order[pos]];
  b->count = count;
  for (size_t g = 0; g < b->groups.size(); ++g) {
    if (!b->group_stream[g]) {
      int lo = 0, hi = 0;
      if ((e = cudaStreamCreateWithFlags(&b->group_stream[g], cudaStreamNonBlocking)) ||
          (e = cudaEventCreateWithFlags(&b->group_done[g], cudaEventDisableTiming)) ||
          (e = cudaDeviceGetStreamPriorityRange(&lo, &hi)) ||
          (e = cudaStreamCreateWithPriority(&b->group_stream_hi[g], cudaStreamNonBlocking, hi)))
        return e;
    }
  }
  return cudaSuccess;
}

cudaError_t launch_group(const mtp_batch* b, const BatchGroup& g, int block, int chunk, int samples,
                         cudaStream_t s) {
  const BatchTables& t = b->t;
  const RolloutArgs* ra = t.d_ra + g.first;
  const int* rs = t.d_row_start + g.rows_first;
  if (!g.stageable) chunk = 0;
  if (!g.pairable) samples = 1;
  if (samples == 2) chunk = 0;
  if (g.dyn == MTP_DYN_POINTMASS)
    return launch_rollout_pointmass_batch(ra, t.d_pm + g.model_first, rs, g.count, g.total_rows, g.n,
                                          block, chunk, samples, s);
  if (g.dyn == MTP_DYN_LEGGED)  // fixed 64-thread blocks (shared-memory staging)
    return launch_rollout_legged_batch(ra, t.d_lm + g.model_first, rs, g.count, g.total_rows, g.n, s);
  return launch_rollout_chain_batch(ra, t.d_cm + g.model_first, rs, g.count, g.total_rows, g.n, block,
                                    chunk, s);
}

// One batched Alg. 2 iteration.  Each (dynamics, dimension) group runs its
// whole iteration on its own stream: graphs, graph paths and local rows of
// its instances, its rollouts, one selection block per instance, the update.
// Groups overlap one another (one group's generation fills the issue slots
// that the others' latency-bound rollouts leave idle).
// part 0: every entry; part 1 / 2: the first / second launch of the
// two-launch mode
PersistArgs persist_args(const mtp_batch* b, bool staged, int part = 0) {
  const BatchTables& t = b->t;
  PersistArgs p{};
  p.ra = t.d_ra;
  p.pm = t.d_pm;
  p.cm = t.d_cm;
  p.order = t.d_p_order;
  p.wstart = t.d_p_wstart;
  p.code = t.d_p_code;
  p.model = t.d_p_model;
  p.head = t.d_p_head;
  p.count = b->p_count;
  p.total_warps = b->p_total_warps;
  p.w_base = 0;
  p.warp_bytes = staged ? b->p_warp_bytes : 0;
  if (part == 1) {
    p.count = b->p_split;
    p.total_warps = b->p_split_warps;
  } else if (part == 2) {
    const int k = b->p_split;
    p.order += k;
    p.wstart += k;
    p.code += k;
    p.model += k;
    p.head += 1;
    p.count = b->p_count - k;
    p.total_warps = b->p_total_warps - b->p_split_warps;
    p.w_base = b->p_split_warps;
  }
  return p;
}

cudaError_t enqueue_batch_iteration(mtp_batch* b, cudaStream_t s);

// One batched iteration with the covered groups' rollouts in one persistent
// launch: every group generates its candidates on its own stream; the
// persistent launch starts when the covered groups' candidates are all made
// (the groups it does not cover keep their own rollout launch); then each
// covered group selects and updates on its stream.  Staged tiles, or every
// tile with direct loads (`staged` false).
cudaError_t enqueue_batch_iteration_persistent(mtp_batch* b, cudaStream_t s, bool staged, bool split) {
  cudaError_t e;
  const BatchTables& t = b->t;
  split = split && b->p_split > 0 && b->p_split < b->p_count;
  std::vector<int> rank(b->groups.size(), 0);
  for (size_t r = 0; r < b->launch_order.size(); ++r) rank[b->launch_order[r]] = (int)r;
  auto first_part = [&](int gi) { return split && rank[gi] < b->p_split_rank; };
  if ((e = cudaEventRecord(b->fork_ev, s))) return e;
  for (const int gi : b->launch_order) {
    const BatchGroup& g = b->groups[gi];
    cudaStream_t gs = first_part(gi) ? b->group_stream_hi[gi] : b->group_stream[gi];
    const int f = g.first;
    if ((e = cudaStreamWaitEvent(gs, b->fork_ev, 0))) return e;
    if ((e = launch_graph_Z_batch(t.d_cand + f, t.d_Z + f, t.d_z_start + f, g.count, g.z_blocks, gs))) return e;
    if ((e = launch_candidates_batch(t.d_cand + f, t.d_cand_start + f, g.count, g.cand_blocks, g.cand_smem, gs)))
      return e;
    if (g.tc_count > 0 &&
        (e = launch_bspline_tc_batch(t.d_tc + g.tc_first, t.d_tc_start + g.tc_start_first, g.tc_count,
                                     g.tc_tiles, gs)))
      return e;
    if ((e = launch_local_batch(t.d_cand + f, t.d_local_start + f, g.count, g.local_blocks, gs))) return e;
    if (!b->covered[gi]) {
      if ((e = launch_group(b, g, g.block, g.chunk, g.samples, gs))) return e;
      if ((e = launch_select_batch(t.d_sel + f, g.count, g.sel_smem, gs))) return e;
      if ((e = launch_update_batch(t.d_upd + f, t.d_warp_start + f, g.count, g.upd_threads, gs))) return e;
    }
    if ((e = cudaEventRecord(b->group_done[gi], gs))) return e;
  }
  if (!split) {
    for (size_t gi = 0; gi < b->groups.size(); ++gi)
      if (b->covered[gi] && (e = cudaStreamWaitEvent(s, b->group_done[gi], 0))) return e;
    if ((e = launch_rollout_persistent(persist_args(b, staged), b->p_blocks[staged ? 0 : 1], s))) return e;
    if ((e = cudaEventRecord(b->persist_ev, s))) return e;
  } else {
    // the first launch starts when the first part's candidates are made and
    // keeps one CTA per SM free for the second part's generation; the second
    // starts when its own candidates are made
    cudaStream_t ps[2] = {b->persist_stream[0], b->persist_stream[1]};
    cudaEvent_t pev[2] = {b->persist_ev, b->persist_ev2};
    for (int part = 0; part < 2; ++part) {
      if ((e = cudaStreamWaitEvent(ps[part], b->fork_ev, 0))) return e;
      for (size_t gi = 0; gi < b->groups.size(); ++gi)
        if (b->covered[gi] && first_part((int)gi) == (part == 0) &&
            (e = cudaStreamWaitEvent(ps[part], b->group_done[gi], 0)))
          return e;
      const int blocks = part == 0 ? std::max(1, b->p_blocks[staged ? 0 : 1] - kPersistFirstFewer)
                                   : b->p_blocks[staged ? 0 : 1];
      if ((e = launch_rollout_persistent(persist_args(b, staged, part + 1), blocks, ps[part]))) return e;
      if ((e = cudaEventRecord(pev[part], ps[part]))) return e;
    }
  }
  for (const int gi : b->launch_order) {
    if (!b->covered[gi]) continue;
    const BatchGroup& g = b->groups[gi];
    cudaStream_t gs = first_part(gi) ? b->group_stream_hi[gi] : b->group_stream[gi];
    const int f = g.first;
    if ((e = cudaStreamWaitEvent(gs, split && !first_part(gi) ? b->persist_ev2 : b->persist_ev, 0))) return e;
    if ((e = launch_select_batch(t.d_sel + f, g.count, g.sel_smem, gs))) return e;
    if ((e = launch_update_batch(t.d_upd + f, t.d_warp_start + f, g.count, g.upd_threads, gs))) return e;
    if ((e = cudaEventRecord(b->group_done[gi], gs))) return e;
  }
  for (size_t gi = 0; gi < b->groups.size(); ++gi)
    if ((e = cudaStreamWaitEvent(s, b->group_done[gi], 0))) return e;
  return cudaSuccess;
}

cudaError_t enqueue_batch_iteration(mtp_batch* b, cudaStream_t s) {
  cudaError_t e;
  const BatchTables& t = b->t;
  if (b->rollout_mode != MTP_BATCH_ROLLOUT_GROUPS && b->p_total_warps > 0)
    return enqueue_batch_iteration_persistent(b, s, b->rollout_mode != MTP_BATCH_ROLLOUT_PERSISTENT_DIRECT,
                                              b->rollout_mode == MTP_BATCH_ROLLOUT_PERSISTENT_SPLIT);
  if ((e = cudaEventRecord(b->fork_ev, s))) return e;
  for (const int gi : b->launch_order) {
    const BatchGroup& g = b->groups[gi];
    cudaStream_t gs = b->group_stream[gi];
    const int f = g.first;
    if ((e = cudaStreamWaitEvent(gs, b->fork_ev, 0))) return e;
    if ((e = launch_graph_Z_batch(t.d_cand + f, t.d_Z + f, t.d_z_start + f, g.count, g.z_blocks, gs))) return e;
    if ((e = launch_candidates_batch(t.d_cand + f, t.d_cand_start + f, g.count, g.cand_blocks, g.cand_smem, gs)))
      return e;
    if (g.tc_count > 0 &&
        (e = launch_bspline_tc_batch(t.d_tc + g.tc_first, t.d_tc_start + g.tc_start_first, g.tc_count,
                                     g.tc_tiles, gs)))
      return e;
    if ((e = launch_local_batch(t.d_cand + f, t.d_local_start + f, g.count, g.local_blocks, gs))) return e;
    if ((e = launch_group(b, g, g.block, g.chunk, g.samples, gs))) return e;
    if ((e = launch_select_batch(t.d_sel + f, g.count, g.sel_smem, gs))) return e;
    if ((e = launch_update_batch(t.d_upd + f, t.d_warp_start + f, g.count, g.upd_threads, gs))) return e;
    if ((e = cudaEventRecord(b->group_done[gi], gs))) return e;
  }
  for (size_t gi = 0; gi < b->groups.size(); ++gi)
    if ((e = cudaStreamWaitEvent(s, b->group_done[gi], 0))) return e;
  return cudaSuccess;
}

// scatter x0 -> iterations -> gather u*.  The first run after a fill
// launches eagerly; later runs over the same layout replay captured graphs.
cudaError_t run_batch(mtp_batch* b, const float* d_x0, int iters, float* d_ustar, cudaStream_t s) {
  const bool graphs = b->runs_since_fill++ > 0;
  cudaError_t e = launch_scatter(d_x0, b->t.d_x0_dst, b->t.d_x0_off, b->count, s);
  if (e != cudaSuccess) return e;
  if (!graphs) {
    for (int k = 0; k < iters; ++k)
      if ((e = enqueue_batch_iteration(b, s))) return e;
  } else {
    int left = iters;
    while (left > 0) {
      const int chunk = left > 64 ? 64 : left;
      auto it = b->graphs.find(chunk);
      if (it == b->graphs.end()) {
        cudaGraph_t graph;
        if ((e = cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal))) return e;
        for (int k = 0; k < chunk && e == cudaSuccess; ++k) e = enqueue_batch_iteration(b, b->cap_stream);
        cudaError_t e2 = cudaStreamEndCapture(b->cap_stream, &graph);
        if (e != cudaSuccess) return e;
        if (e2 != cudaSuccess) return e2;
        cudaGraphExec_t exec;
        // kernel nodes keep the priority of the stream they were captured
        // from (the two-launch persistent mode's first-part generation)
        e = cudaGraphInstantiate(&exec, graph, cudaGraphInstantiateFlagUseNodePriority);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) return e;
        it = b->graphs.emplace(chunk, exec).first;
      }
      if ((e = cudaGraphLaunch(it->second, s))) return e;
      left -= chunk;
    }
  }
  e = launch_gather(b->t.d_ustar_src, b->t.d_us_off, d_ustar, b->count, s);
  if (e != cudaSuccess) return e;
  for (mtp_handle* h : b->hs) {
    h->iter_host += (uint32_t)iters;
    h->cur = 0;  // the tables point at the first buffer (set when they were filled)
    h->U = h->Ubuf[0];
    h->prep_valid = false;
  }
  return cudaSuccess;
}

}  // namespace

extern "C" {

namespace {

// Planner state of every instance of the batch (mean, spread, their FP32
// copies, the iteration counter), saved to one device buffer so that timing
// runs of whole iterations can be undone.
struct SavedStates {
  unsigned char* d = nullptr;
  std::vector<size_t> off;
  cudaError_t save(const mtp_batch* b, cudaStream_t s) {
    size_t bytes = 0;
    off.clear();
    for (const mtp_handle* h : b->hs) {
      off.push_back(bytes);
      const size_t hn = (size_t)h->dm.H * h->dm.n;
      bytes += ((2 * hn * sizeof(double) + 2 * hn * sizeof(float) + sizeof(uint32_t)) + 255) & ~size_t(255);
    }
    cudaError_t e = cudaMalloc((void**)&d, std::max<size_t>(bytes, 256));
    if (e != cudaSuccess) return e;
    return copy(b, s, true);
  }
  cudaError_t copy(const mtp_batch* b, cudaStream_t s, bool to_saved) {
    cudaError_t e = cudaSuccess;
    for (size_t i = 0; i < b->hs.size() && e == cudaSuccess; ++i) {
      const mtp_handle* h = b->hs[i];
      const size_t hn = (size_t)h->dm.H * h->dm.n;
      unsigned char* p = d + off[i];
      void* live[5] = {h->mu, h->sigma, h->mu_f, h->sigma_f, h->iter_dev};
      const size_t len[5] = {hn * sizeof(double), hn * sizeof(double), hn * sizeof(float), hn * sizeof(float),
                             sizeof(uint32_t)};
      for (int k = 0; k < 5 && e == cudaSuccess; ++k) {
        e = to_saved ? cudaMemcpyAsync(p, live[k], len[k], cudaMemcpyDeviceToDevice, s)
                     : cudaMemcpyAsync(live[k], p, len[k], cudaMemcpyDeviceToDevice, s);
        p += len[k];
      }
    }
    return e;
  }
  ~SavedStates() {
    if (d) cudaFree(d);
  }
};

// Times one iteration in each rollout mode as a captured graph, the form
// mtp_batch_plan_step replays (best of three after one untimed replay, every
// replay from the saved states), and keeps the fastest; the states are
// restored afterwards.
cudaError_t tune_rollout_mode(mtp_batch* b) {
  cudaStream_t s = b->cap_stream;
  SavedStates st;
  cudaError_t e = st.save(b, s);
  cudaEvent_t t0 = nullptr, t1 = nullptr;
  if (e == cudaSuccess) e = cudaEventCreate(&t0);
  if (e == cudaSuccess) e = cudaEventCreate(&t1);
  int best_mode = MTP_BATCH_ROLLOUT_GROUPS;
  double best = 1e30;
  for (int mode = 0; mode < 4 && e == cudaSuccess; ++mode) {
    b->mode_ms[mode] = 0.0;
    if (mode != MTP_BATCH_ROLLOUT_GROUPS && b->p_total_warps <= 0) continue;
    b->rollout_mode = mode;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    if ((e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal))) break;
    e = enqueue_batch_iteration(b, s);
    const cudaError_t e2 = cudaStreamEndCapture(s, &graph);
    if (e == cudaSuccess) e = e2;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, cudaGraphInstantiateFlagUseNodePriority);
    if (graph) cudaGraphDestroy(graph);
    float ms_min = 1e30f;
    for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {
      if ((e = st.copy(b, s, false))) break;
      if ((e = cudaEventRecord(t0, s))) break;
      if ((e = cudaGraphLaunch(exec, s))) break;
      if ((e = cudaEventRecord(t1, s))) break;
      if ((e = cudaEventSynchronize(t1))) break;
      float ms = 0.f;
      if ((e = cudaEventElapsedTime(&ms, t0, t1))) break;
      if (rep > 0) ms_min = std::min(ms_min, ms);
    }
    if (exec) cudaGraphExecDestroy(exec);
    b->mode_ms[mode] = ms_min;
    if (ms_min < best) {
      best = ms_min;
      best_mode = mode;
    }
  }
  b->rollout_mode = best_mode;
  if (e == cudaSuccess) e = st.copy(b, s, false);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (t0) cudaEventDestroy(t0);
  if (t1) cudaEventDestroy(t1);
  return e;
}

}  // namespace

static mtp_status check_batch_handles(mtp_handle* const* handles, int32_t count, int dev) {
  for (int i = 0; i < count; ++i) {
    if (!handles[i]) return batch_fail(nullptr, MTP_ERR_INVALID_ARG, "batch: null handle");
    if (handles[i]->sel_chunks > 0)
      return batch_fail(nullptr, MTP_ERR_UNSUPPORTED,
                        "batch: B too large for the one-block selection a batch gives each instance");
    if (handles[i]->device != dev)
      return batch_fail(nullptr, MTP_ERR_INVALID_ARG, "batch: handles must live on the batch's device");
    for (int j = 0; j < i; ++j)
      if (handles[j] == handles[i]) return batch_fail(nullptr, MTP_ERR_INVALID_ARG, "batch: repeated handle");
  }
  return MTP_OK;
}

mtp_status mtp_batch_reserve(int32_t capacity, mtp_batch** out) {
  if (!out || capacity < 1) return batch_fail(nullptr, MTP_ERR_INVALID_ARG, "batch_reserve: bad argument");
  *out = nullptr;
  mtp_batch* b = new mtp_batch();
  cudaGetDevice(&b->device);
  cudaError_t e = init_candidate_attributes();
  if (e == cudaSuccess) e = init_select_attributes();
  if (e == cudaSuccess) e = init_rollout_pm_batch_attributes();
  if (e == cudaSuccess) e = init_bspline_tc_attributes();
  if (e == cudaSuccess) e = init_rollout_chain_batch_attributes();
  if (e == cudaSuccess) e = alloc_batch(b, capacity);
  if (e != cudaSuccess) {
    mtp_status st = batch_fail(nullptr, e == cudaErrorMemoryAllocation ? MTP_ERR_OUT_OF_MEMORY : MTP_ERR_CUDA,
                               std::string("batch_reserve: ") + cudaGetErrorString(e));
    free_batch(b);
    return st;
  }
  *out = b;
  return MTP_OK;
}

mtp_status mtp_batch_fill(mtp_batch* b, mtp_handle* const* handles, int32_t count, void* stream) {
  if (!b || !handles || count < 1 || count > b->t.cap)
    return batch_fail(b, MTP_ERR_INVALID_ARG, "batch_fill: bad argument (count must be 1 .. capacity)");
  mtp_status st = check_batch_handles(handles, count, b->device);
  if (st != MTP_OK) return batch_fail(b, st, mtp_last_error(nullptr));
  DeviceGuard guard(b->device);
  cudaError_t e = fill_batch(b, handles, count, (cudaStream_t)stream);
  if (e == cudaErrorInvalidValue)
    return batch_fail(b, MTP_ERR_INVALID_ARG, "batch_fill: more than 64 (dynamics, dimension) groups");
  if (e != cudaSuccess) return batch_fail(b, MTP_ERR_CUDA, std::string("batch_fill: ") + cudaGetErrorString(e));
  return MTP_OK;
}

mtp_status mtp_batch_create(mtp_handle* const* handles, int32_t count, mtp_batch** out) {
  if (!handles || !out || count < 1) return batch_fail(nullptr, MTP_ERR_INVALID_ARG, "batch_create: bad argument");
  *out = nullptr;
  int dev = 0;
  cudaGetDevice(&dev);
  mtp_status st = check_batch_handles(handles, count, dev);
  if (st != MTP_OK) return st;
  mtp_batch* b = nullptr;
  if ((st = mtp_batch_reserve(count, &b)) != MTP_OK) return st;
  if ((st = mtp_batch_fill(b, handles, count, b->cap_stream)) != MTP_OK) {
    mtp::set_thread_error(b->err);
    free_batch(b);
    return st;
  }
  cudaError_t e = cudaStreamSynchronize(b->cap_stream);
  if (e != cudaSuccess) {
    free_batch(b);
    return batch_fail(nullptr, MTP_ERR_CUDA, std::string("batch_create: ") + cudaGetErrorString(e));
  }
  *out = b;
  return MTP_OK;
}

mtp_status mtp_batch_destroy(mtp_batch* b) {
  if (!b) return MTP_ERR_INVALID_ARG;
  DeviceGuard g(b->device);
  cudaDeviceSynchronize();
  free_batch(b);
  return MTP_OK;
}

mtp_status mtp_batch_layout(const mtp_batch* b, int32_t* x0_offset, int32_t* ustar_offset) {
  if (!b || b->count < 1) return MTP_ERR_INVALID_ARG;
  const size_t c = b->hs.size() + 1;
  if (x0_offset) std::copy(b->x0_off.begin(), b->x0_off.begin() + c, x0_offset);
  if (ustar_offset) std::copy(b->us_off.begin(), b->us_off.begin() + c, ustar_offset);
  return MTP_OK;
}

mtp_status mtp_batch_plan_step(mtp_batch* b, const float* d_x0, int32_t iters, float* d_ustar,
                               void* stream) {
  if (!b || !d_x0 || !d_ustar || iters < 1 || b->count < 1)
    return batch_fail(b, MTP_ERR_INVALID_ARG, "batch_plan_step: bad argument (or batch never filled)");
  DeviceGuard guard(b->device);
  cudaError_t e = run_batch(b, d_x0, iters, d_ustar, (cudaStream_t)stream);
  if (e != cudaSuccess) return batch_fail(b, MTP_ERR_CUDA, std::string("batch_plan_step: ") + cudaGetErrorString(e));
  return MTP_OK;
}

mtp_status mtp_batch_shift(mtp_batch* b, int32_t k, void* stream) {
  if (!b || k < 0 || b->count < 1) return batch_fail(b, MTP_ERR_INVALID_ARG, "batch_shift: bad argument");
  DeviceGuard guard(b->device);
  cudaError_t e = launch_shift_batch(b->t.d_upd, b->count, k, (cudaStream_t)stream);
  if (e != cudaSuccess) return batch_fail(b, MTP_ERR_CUDA, std::string("batch_shift: ") + cudaGetErrorString(e));
  return MTP_OK;
}

mtp_status mtp_batch_autotune(mtp_batch* b, int32_t* tiles_out, int32_t* n_groups, void* stream) {
  if (!b) return MTP_ERR_INVALID_ARG;
  if (b->count < 1) return batch_fail(b, MTP_ERR_INVALID_ARG, "autotune: batch never filled");
  DeviceGuard guard(b->device);
  (void)stream;
  cudaEventSynchronize(b->t.copied);  // the tables may have been filled on another stream
  // rollout tiles: candidates per block (the kernels are bounded at 128
  // threads) x horizon chunk of the staged control loads (0: direct loads)
  const int blocks[3] = {32, 64, 128};
  const int chunks[3] = {0, 4, 8};  // chains stage 4 steps at a time (8 is not tried)
  cudaEvent_t t0, t1;
  cudaEventCreate(&t0);
  cudaEventCreate(&t1);
  cudaError_t e = cudaSuccess;
  // tiles: (candidates per block, horizon chunk, candidates per thread)
  struct Tile {
    int block, chunk, samples;
  };
  std::vector<Tile> tiles;
  for (int chunk : chunks)
    for (int block : blocks) tiles.push_back({block, chunk, 1});
  for (int block : blocks) tiles.push_back({block, 0, 2});
  auto group_steps = [&](const BatchGroup& g) {
    long long steps = 0;
    for (int j = 0; j < g.count; ++j) steps += (long long)b->hs_sorted[g.first + j]->dm.B * b->hs_sorted[g.first + j]->dm.H;
    return steps;
  };
  for (auto& g : b->groups) {
    float best = 1e30f;
    Tile best_tile{g.block, g.chunk, g.samples};
    for (const Tile& tl : tiles) {
      // the legged rollout has one fixed tile: timed once, for the launch order
      if (g.dyn == MTP_DYN_LEGGED && (tl.block != blocks[0] || tl.chunk || tl.samples != 1)) continue;
      if (tl.chunk && !g.stageable) continue;
      if (tl.chunk == 8 && g.dyn == MTP_DYN_CHAIN) continue;
      if (tl.samples == 2 && !g.pairable) continue;
      float ms_min = 1e30f;
      for (int rep = 0; rep < 3 && e == cudaSuccess; ++rep) {
        cudaEventRecord(t0, b->cap_stream);
        e = launch_group(b, g, tl.block, tl.chunk, tl.samples, b->cap_stream);
        cudaEventRecord(t1, b->cap_stream);
        cudaEventSynchronize(t1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, t0, t1);
        ms_min = std::min(ms_min, ms);
      }
      if (ms_min < best) {
        best = ms_min;
        best_tile = tl;
      }
    }
    if (e == cudaSuccess && best < 1e30f)
      b->tuned_ms_per_step[{g.dyn, g.n}] = (double)best / (double)std::max(1LL, (long long)group_steps(g));
    if (g.dyn == MTP_DYN_LEGGED) continue;
    g.block = best_tile.block;
    g.chunk = best_tile.chunk;
    g.samples = best_tile.samples;
    b->tuned[{g.dyn, g.n}] = {g.block, g.chunk, g.samples};
  }
  set_launch_order(b, group_steps);
  cudaEventDestroy(t0);
  cudaEventDestroy(t1);
  // refill with the tuned tiles and times per step (the persistent launch's
  // longest-first order uses them), then time the rollout modes
  if (e == cudaSuccess) {
    std::vector<mtp_handle*> hs = b->hs;
    e = fill_batch(b, hs.data(), (int)hs.size(), b->cap_stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->cap_stream);
  }
  if (e == cudaSuccess) e = tune_rollout_mode(b);
  if (e != cudaSuccess) return batch_fail(b, MTP_ERR_CUDA, std::string("autotune: ") + cudaGetErrorString(e));
  for (auto& kv : b->graphs) cudaGraphExecDestroy(kv.second);  // tiles changed: recapture
  b->graphs.clear();
  if (n_groups) *n_groups = (int32_t)b->groups.size();
  if (tiles_out)
    for (size_t i = 0; i < b->groups.size(); ++i) {
      tiles_out[5 * i + 0] = b->groups[i].dyn;
      tiles_out[5 * i + 1] = b->groups[i].n;
      tiles_out[5 * i + 2] = b->groups[i].block;
      tiles_out[5 * i + 3] = b->groups[i].chunk;
      tiles_out[5 * i + 4] = b->groups[i].samples;
    }
  return MTP_OK;
}

mtp_status mtp_batch_launches(const mtp_batch* b, int32_t iters, int32_t* launches) {
  if (!b || !launches || iters < 1 || b->count < 1) return MTP_ERR_INVALID_ARG;
  const bool persistent = b->rollout_mode != MTP_BATCH_ROLLOUT_GROUPS && b->p_total_warps > 0;
  const bool split = b->rollout_mode == MTP_BATCH_ROLLOUT_PERSISTENT_SPLIT && b->p_split > 0 &&
                     b->p_split < b->p_count;
  long long per_iter = persistent ? (split ? 2 : 1) : 0;
  for (size_t gi = 0; gi < b->groups.size(); ++gi) {
    const BatchGroup& g = b->groups[gi];
    per_iter += (g.z_blocks > 0) + (g.cand_blocks > 0) + (g.local_blocks > 0) + (g.tc_count > 0);
    per_iter += (g.total_rows > 0 && !(persistent && b->covered[gi])) + (g.count > 0) + (g.upd_threads > 0);
  }
  *launches = (int32_t)(2 + per_iter * iters);  // scatter of x0 and gather of u* once per call
  return MTP_OK;
}

mtp_status mtp_batch_set_rollout_mode(mtp_batch* b, int32_t mode) {
  if (!b || mode < MTP_BATCH_ROLLOUT_GROUPS || mode > MTP_BATCH_ROLLOUT_PERSISTENT_SPLIT)
    return batch_fail(b, MTP_ERR_INVALID_ARG, "batch_set_rollout_mode: unknown mode");
  if (b->rollout_mode != mode) {
    b->rollout_mode = mode;
    drop_graphs(b);
    b->runs_since_fill = 0;
  }
  return MTP_OK;
}

mtp_status mtp_batch_rollout_mode(const mtp_batch* b, int32_t* mode, double* ms4) {
  if (!b || !mode) return MTP_ERR_INVALID_ARG;
  *mode = b->rollout_mode;
  if (ms4)
    for (int k = 0; k < 4; ++k) ms4[k] = b->mode_ms[k];
  return MTP_OK;
}

mtp_status mtp_batch_persistent_time(mtp_batch* b, int32_t reps, double* ms, int64_t* steps, void* stream) {
  if (!b || reps < 1 || !ms) return batch_fail(b, MTP_ERR_INVALID_ARG, "persistent_time: bad argument");
  if (b->count < 1) return batch_fail(b, MTP_ERR_INVALID_ARG, "persistent_time: batch never filled");
  DeviceGuard guard(b->device);
  cudaStream_t s = (cudaStream_t)stream;
  *ms = 0.0;
  long long covered_steps = 0;
  for (size_t gi = 0; gi < b->groups.size(); ++gi) {
    if (!b->covered[gi]) continue;
    const BatchGroup& g = b->groups[gi];
    for (int j = 0; j < g.count; ++j)
      covered_steps += (long long)b->hs_sorted[g.first + j]->dm.B * b->hs_sorted[g.first + j]->dm.H;
  }
  if (steps) *steps = covered_steps;
  if (b->p_total_warps <= 0) return MTP_OK;
  const bool staged = b->rollout_mode != MTP_BATCH_ROLLOUT_PERSISTENT_DIRECT;
  cudaEvent_t t0 = nullptr, t1 = nullptr;
  cudaError_t e = cudaEventCreate(&t0);
  if (e == cudaSuccess) e = cudaEventCreate(&t1);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(s, b->t.copied, 0);
  double sum = 0.0;
  for (int rep = 0; rep < reps && e == cudaSuccess; ++rep) {
    if ((e = cudaEventRecord(t0, s))) break;
    if ((e = launch_rollout_persistent(persist_args(b, staged), b->p_blocks[staged ? 0 : 1], s))) break;
    if ((e = cudaEventRecord(t1, s))) break;
    if ((e = cudaEventSynchronize(t1))) break;
    float v = 0.f;
    if ((e = cudaEventElapsedTime(&v, t0, t1))) break;
    sum += v;
  }
  if (t0) cudaEventDestroy(t0);
  if (t1) cudaEventDestroy(t1);
  if (e != cudaSuccess) return batch_fail(b, MTP_ERR_CUDA, std::string("persistent_time: ") + cudaGetErrorString(e));
  *ms = sum / reps;
  return MTP_OK;
}

mtp_status mtp_batch_rollout_times(mtp_batch* b, int32_t reps, double* ms_out, int32_t* info_out,
                                   int32_t max_groups, int32_t* n_groups, void* stream) {
  if (!b || reps < 1 || !n_groups) return MTP_ERR_INVALID_ARG;
  if (b->count < 1) return batch_fail(b, MTP_ERR_INVALID_ARG, "rollout_times: batch never filled");
  DeviceGuard guard(b->device);
  cudaStream_t s = (cudaStream_t)stream;
  *n_groups = (int32_t)b->groups.size();
  if ((ms_out || info_out) && max_groups < (int32_t)b->groups.size())
    return batch_fail(b, MTP_ERR_INVALID_ARG, "rollout_times: max_groups below the group count");
  cudaEvent_t t0, t1;
  cudaError_t e = cudaEventCreate(&t0);
  if (e == cudaSuccess) e = cudaEventCreate(&t1);
  if (e != cudaSuccess) return batch_fail(b, MTP_ERR_CUDA, std::string("rollout_times: ") + cudaGetErrorString(e));
  if (e == cudaSuccess) e = cudaStreamWaitEvent(s, b->t.copied, 0);  // tables filled on another stream
  for (size_t gi = 0; gi < b->groups.size() && e == cudaSuccess; ++gi) {
    const BatchGroup& g = b->groups[gi];
    double sum = 0.0;
    for (int rep = 0; rep < reps && e == cudaSuccess; ++rep) {
      if ((e = cudaEventRecord(t0, s))) break;
      if ((e = launch_group(b, g, g.block, g.chunk, g.samples, s))) break;
      if ((e = cudaEventRecord(t1, s))) break;
      if ((e = cudaEventSynchronize(t1))) break;
      float ms = 0.f;
      if ((e = cudaEventElapsedTime(&ms, t0, t1))) break;
      sum += ms;
    }
    if (ms_out) ms_out[gi] = sum / reps;
    if (info_out) {
      long long rows = 0, steps = 0;
      for (int j = 0; j < g.count; ++j) {
        const mtp_handle* h = b->hs_sorted[g.first + j];
        rows += h->dm.B;
        steps += (long long)h->dm.B * h->dm.H;
      }
      int32_t* o = info_out + 8 * gi;
      o[0] = g.dyn;
      o[1] = g.n;
      o[2] = g.block;
      o[3] = g.count;
      o[4] = (int32_t)rows;
      o[5] = (int32_t)std::min<long long>(steps, 0x7fffffff);
      o[6] = g.stageable ? g.chunk : 0;
      o[7] = g.pairable ? g.samples : 1;
    }
  }
  cudaEventDestroy(t0);
  cudaEventDestroy(t1);
  if (e != cudaSuccess) return batch_fail(b, MTP_ERR_CUDA, std::string("rollout_times: ") + cudaGetErrorString(e));
  return MTP_OK;
}

}  // extern "C"
