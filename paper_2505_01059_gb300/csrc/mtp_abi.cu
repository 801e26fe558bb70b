// mtp_abi.cu -- the single-instance part of the C ABI of include/mtp.h:
// problem validation, the handle's device state, host precompute of the
// interpolation tables (the B-spline basis of Def. 2 by the closed-form
// cardinal B-spline, the Akima / straight-line piece table of Def. 3), and
// the launch sequence of one planner iteration (Alg. 2), pipelined when the
// rollout leaves SMs idle and replayed as a CUDA graph.  Batched planning is
// in batch_abi.cu, serving in server.cu.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <type_traits>
#include <vector>

#include "handle.cuh"

using namespace mtp;

namespace {

thread_local std::string g_create_error;

constexpr size_t kMaxSmem = 200 * 1024;

}  // namespace

void mtp::set_thread_error(const std::string& msg) { g_create_error = msg; }


namespace {

mtp_status fail(mtp_handle* h, mtp_status st, const std::string& msg) {
  if (h) h->err = msg;
  else g_create_error = msg;
  return st;
}

mtp_status cuda_fail(mtp_handle* h, cudaError_t e, const char* where) {
  std::string msg = std::string(where) + ": " + cudaGetErrorString(e);
  return fail(h, e == cudaErrorMemoryAllocation ? MTP_ERR_OUT_OF_MEMORY : MTP_ERR_CUDA, msg);
}

#define MTP_CUDA(h, call)                                   \
  do {                                                      \
    cudaError_t e_ = (call);                                \
    if (e_ != cudaSuccess) return cuda_fail((h), e_, #call); \
  } while (0)

int32_t num_graph_samples(double beta, int32_t B) {
  int32_t P = (int32_t)std::floor(beta * (double)B);
  if (P > B - 1) P = B - 1;
  if (P < 0) P = 0;
  return P;
}

// Cardinal B-spline of degree p on the integer knots 0..p+1 by the truncated
// power form N_p(y) = 1/p! sum_k (-1)^k C(p+1, k) (y - k)_+^p, evaluated only
// inside its support and on the nearer half (N_p(y) = N_p(p+1-y)) to keep the
// alternating sum short.  The indicator of degree 0 is half-open; `left`
// takes the left limit (the closed right end of the valid span).
double cardinal_bspline(int p, double y, bool left) {
  const double end = (double)(p + 1);
  if (y < 0.0 || y > end) return 0.0;
  if (y == end) return (left && p == 0) ? 1.0 : 0.0;
  if (y == 0.0) return (!left && p == 0) ? 1.0 : 0.0;
  if (p == 0) return 1.0;  // interior of [0, 1)
  if (y > 0.5 * end) y = end - y;  // continuous for p >= 1: no knot-side question
  double acc = 0.0, binom = 1.0, fact = 1.0;
  for (int k = 2; k <= p; ++k) fact *= k;
  for (int k = 0; k <= p + 1 && y - k > 0.0; ++k) {
    acc += ((k & 1) ? -binom : binom) * std::pow(y - k, p);
    binom = binom * (p + 1 - k) / (k + 1);
  }
  return acc / fact;
}

mtp_status validate(const mtp_problem& p) {
  auto bad = [](const std::string& m) { return fail(nullptr, MTP_ERR_INVALID_ARG, m); };
  if (p.dyn == MTP_DYN_POINTMASS) {
    if (p.ctrl_dim < 1 || p.ctrl_dim > 16) return bad("point mass: ctrl_dim must be in 1..16");
    if (p.state_dim != 2 * p.ctrl_dim) return bad("point mass: state_dim must be 2*ctrl_dim");
    if (p.n_obstacles < 0 || p.n_obstacles > MTP_MAX_OBSTACLES) return bad("n_obstacles out of range");
  } else if (p.dyn == MTP_DYN_CHAIN) {
    if (p.n_links < 1 || p.n_links > 12) return bad("chain: n_links must be in 1..12");
    if (p.ctrl_dim != p.n_links || p.state_dim != 2 * p.n_links)
      return bad("chain: ctrl_dim must be n_links and state_dim 2*n_links");
    for (int j = 0; j < p.n_links; ++j)
      if (!(p.link_mass[j] > 0.f) || !(p.link_length[j] > 0.f)) return bad("chain: link mass/length must be > 0");
  } else if (p.dyn == MTP_DYN_LEGGED) {
    if (p.n_links < 2 || p.n_links > 16) return bad("legged: n_links must be in 2..16");
    if (p.ctrl_dim != p.n_links - 1 || p.state_dim != 2 * (p.n_links + 2))
      return bad("legged: ctrl_dim must be n_links-1 and state_dim 2*(n_links+2)");
    for (int j = 0; j < p.n_links; ++j)
      if (!(p.link_mass[j] > 0.f) || !(p.link_length[j] > 0.f)) return bad("legged: link mass/length must be > 0");
    if (!(p.k_contact >= 0.f) || !(p.c_contact >= 0.f) || !(p.mu_friction >= 0.f) || !(p.v_slip > 0.f))
      return bad("legged: need k, c, friction >= 0 and v_slip > 0");
  } else {
    return bad("unknown dyn");
  }
  if (p.horizon < 1) return bad("horizon must be >= 1");
  if (!(p.dt > 0.f)) return bad("dt must be > 0");
  for (int i = 0; i < p.ctrl_dim; ++i)
    if (!(p.u_min[i] < p.u_max[i]) || !std::isfinite(p.u_min[i]) || !std::isfinite(p.u_max[i]))
      return bad("control box: need finite u_min < u_max");
  if (p.M < 1 || p.M > 64) return bad("M must be in 1..64");
  if (p.N < 1) return bad("N must be >= 1");
  if (p.B < 1 || p.B > (1 << 24)) return bad("B must be in 1..2^24");
  if (p.E < 1 || p.E > p.B) return bad("E must be in 1..B");
  if (!(p.beta >= 0.0 && p.beta <= 1.0)) return bad("beta must be in [0, 1]");
  if (!(p.lambda > 0.0)) return bad("lambda must be > 0");
  if (!(p.alpha >= 0.0 && p.alpha < 1.0)) return bad("alpha must be in [0, 1)");
  if (!(p.sigma_min > 0.0)) return bad("sigma_min must be > 0");
  if (!(p.sigma_init >= 0.0) || !std::isfinite(p.mu_init)) return bad("bad mu_init / sigma_init");
  if (p.interp < 0 || p.interp > 2) return bad("unknown interp");
  if (p.interp == MTP_INTERP_BSPLINE && (p.bspline_degree < 0 || p.bspline_degree > 7 || p.M < p.bspline_degree + 1))
    return bad("B-spline: need 0 <= degree <= 7 and M >= degree + 1");
  if (p.time_mapping < 0 || p.time_mapping > 1) return bad("unknown time_mapping");
  if (p.update_rule < 0 || p.update_rule > 1) return bad("unknown update_rule");
  if (p.dr_mode < 0 || p.dr_mode > 2) return bad("unknown dr_mode");
  if (p.dr_mode == MTP_DR_SHARED && (p.R < 1 || p.R > 64)) return bad("R must be in 1..64");
  if (p.dr_mode != MTP_DR_NONE && !(p.dr_lo > 0.f && p.dr_lo <= p.dr_hi)) return bad("need 0 < dr_lo <= dr_hi");
  if ((size_t)p.M * p.N * p.ctrl_dim * 4 > 160 * 1024) return bad("graph M*N*n too large for one block's shared memory");
  {
    int chunk = 0, chunks = 0;
    select_plan(p.B, p.E, &chunk, &chunks);
    if (chunks < 0) return bad("B and E too large for the two-stage elite selection");
  }
  if ((p.flags & MTP_FLAG_BF16_BASIS) && p.interp != MTP_INTERP_BSPLINE)
    return fail(nullptr, MTP_ERR_UNSUPPORTED, "the BF16 basis applies to B-spline interpolation only");
  return MTP_OK;
}

// A one-layer graph (M = 1) makes constant paths whatever the interpolation
// (each path is its single waypoint held over the horizon).  The handle runs
// that as the degree-0 B-spline over one basis function, which is 1 at every
// step of its valid span (the span then covers the whole horizon, so the
// time reading does not matter); no contraction rounds the waypoint, so BF16
// operands do not apply.
mtp_problem normalized(const mtp_problem& in) {
  mtp_problem p = in;
  if (p.M == 1) {
    p.interp = MTP_INTERP_BSPLINE;
    p.bspline_degree = 0;
    p.time_mapping = MTP_TIME_VALID_SPAN;
    p.flags &= ~MTP_FLAG_BF16_BASIS;
  }
  return p;
}

template <class T>
cudaError_t dalloc(T** p, size_t count) {
  return cudaMalloc((void**)p, sizeof(T) * (count ? count : 1));
}

// Nearest bfloat16 of a finite float, ties to even, as a float: the low 16
// bits of the IEEE-754 encoding are rounded away (adding 0x7fff plus the
// lowest kept bit carries into the kept bits exactly when the dropped part
// is above one half, or exactly one half with an odd kept part).
float round_bf16(float x) {
  uint32_t u;
  std::memcpy(&u, &x, 4);
  u += 0x7fffu + ((u >> 16) & 1u);
  u &= 0xffff0000u;
  float r;
  std::memcpy(&r, &u, 4);
  return r;
}

mtp_status build_tables(mtp_handle* h) {
  const mtp_problem& p = h->pr;
  const bool bf16 = (p.flags & MTP_FLAG_BF16_BASIS) != 0;
  const int H = p.horizon, M = p.M;
  std::vector<float> basis((size_t)H * M, 0.f);
  std::vector<int32_t> bfirst(H, 0), seg(H, 0);
  std::vector<float> delta(H, 0.f);
  if (p.interp == MTP_INTERP_BSPLINE) {
    const int deg = p.bspline_degree;
    for (int j = 0; j < H; ++j) {
      // evaluation point in knot units (knot i at i): Def. 2 with the chosen reading
      double x;
      bool left = false;
      if (p.time_mapping == MTP_TIME_PAPER_LITERAL) {
        x = (double)((M + deg + 1) * j) / (double)H;
      } else {
        x = H > 1 ? (double)deg + (double)((M - deg) * j) / (double)(H - 1) : (double)deg;
        left = (H > 1 && j == H - 1);
      }
      int first = -1;
      for (int m = 0; m < M; ++m) {
        const double v = cardinal_bspline(deg, x - m, left);
        basis[(size_t)j * M + m] = bf16 ? round_bf16((float)v) : (float)v;
        if (v != 0.0 && first < 0) first = m;
      }
      if (first < 0) first = 0;
      if (first > M - 1 - deg) first = M - 1 - deg;
      bfirst[j] = first;
    }
  } else {
    // Def. 3 knots: i/(M-1) (valid span) or i/M (paper literal); piece of step t
    const bool lit = p.time_mapping == MTP_TIME_PAPER_LITERAL;
    h->inv_h = lit ? (float)M : (float)(M - 1);
    for (int j = 0; j < H; ++j) {
      long long k = lit ? ((long long)j * M) / H : (H > 1 ? ((long long)j * (M - 1)) / (H - 1) : 0);
      if (k > M - 2) k = M - 2;
      const double t = lit ? (double)j / (double)H : (H > 1 ? (double)j / (double)(H - 1) : 0.0);
      const double tk = lit ? (double)k / (double)M : (double)k / (double)(M - 1);
      seg[j] = (int32_t)k;
      delta[j] = (float)(t - tk);
    }
  }
  MTP_CUDA(h, dalloc(&h->basis, basis.size()));
  MTP_CUDA(h, dalloc(&h->bfirst, H));
  MTP_CUDA(h, dalloc(&h->seg, H));
  MTP_CUDA(h, dalloc(&h->delta, H));
  MTP_CUDA(h, cudaMemcpy(h->basis, basis.data(), basis.size() * 4, cudaMemcpyHostToDevice));
  MTP_CUDA(h, cudaMemcpy(h->bfirst, bfirst.data(), H * 4, cudaMemcpyHostToDevice));
  MTP_CUDA(h, cudaMemcpy(h->seg, seg.data(), H * 4, cudaMemcpyHostToDevice));
  MTP_CUDA(h, cudaMemcpy(h->delta, delta.data(), H * 4, cudaMemcpyHostToDevice));
  return MTP_OK;
}

}  // namespace

namespace mtp {
int device_sms() {
  constexpr int kMaxDevices = 64;
  static std::atomic<int> cache[kMaxDevices];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0) return 1;
  if (dev < kMaxDevices) {
    const int v = cache[dev].load(std::memory_order_relaxed);
    if (v > 0) return v;
  }
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0)
    sms = 1;
  if (dev < kMaxDevices) cache[dev].store(sms, std::memory_order_relaxed);
  return sms;
}

CandArgs cand_args(const mtp_handle* h, uint32_t iter, const uint32_t* d_iter) {
  CandArgs a{};
  a.dm = h->dm;
  a.key = h->key;
  a.iter = iter;
  a.d_iter = d_iter;
  a.interp = h->pr.interp;
  a.degree = h->pr.bspline_degree;
  a.bf16 = (h->pr.flags & MTP_FLAG_BF16_BASIS) ? 1 : 0;
  a.inv_h = h->inv_h;
  a.basis = h->basis;
  a.bfirst = h->bfirst;
  a.seg = h->seg;
  a.delta = h->delta;
  a.paths_per_block = h->paths_per_block;
  a.mu = h->mu_f;
  a.sigma = h->sigma_f;
  a.status = h->status;
  for (int i = 0; i < h->dm.n; ++i) {
    a.umin[i] = h->pr.u_min[i];
    a.umax[i] = h->pr.u_max[i];
  }
  return a;
}
}  // namespace mtp

namespace {

// Blocks of 256 threads for the local rows: about `rows_per_thread` rows
// per thread, each thread on one group of four elements, at most 8 blocks
// per SM.  Generating them, 4 rows per thread (measured on the 7-link arm:
// 1, 4 and 16 rows per thread generate in 17.7-18.1, 16.7 and 17.0 us; the
// legged workload, capped at 8 blocks per SM, does not change).  Finishing
// stored draws, one row per thread: that pass only waits for its loads.
constexpr int kLocalRowsPerThread = 4;
constexpr int kFinishRowsPerThread = 1;

int local_blocks_for(const mtp_handle* h, long long rows_plus_mean,
                     int rows_per_thread = kLocalRowsPerThread) {
  const long long G = ((long long)h->dm.H * h->dm.n + 3) / 4;
  long long items = rows_plus_mean * G;
  long long blocks = (items + 256LL * rows_per_thread - 1) / (256LL * rows_per_thread);
  const long long cap = (long long)mtp::device_sms() * 8;
  if (blocks > cap) blocks = cap;
  if (blocks < 1) blocks = 1;
  return (int)blocks;
}

}  // namespace

namespace mtp {
RolloutArgs rollout_args(const mtp_handle* h, uint32_t iter, const uint32_t* d_iter,
                         const float* x0, const float* U, int row0, int rows, float* cost) {
  RolloutArgs a{};
  a.H = h->dm.H;
  a.n = h->dm.n;
  a.d = h->dm.d;
  a.dt = h->pr.dt;
  a.key = h->key;
  a.iter = iter;
  a.d_iter = d_iter;
  a.dr_mode = h->pr.dr_mode;
  a.R = h->pr.R;
  a.dr_lo = h->pr.dr_lo;
  a.dr_hi = h->pr.dr_hi;
  a.x0 = x0;
  a.U = U;
  a.row0 = row0;
  a.rows = rows;
  a.cost = cost;
  a.kahan = (h->pr.flags & MTP_FLAG_NO_KAHAN) ? 0 : 1;
  a.status = h->status;
  return a;
}

PointMassModel pointmass_model(const mtp_problem& p) {
  PointMassModel m{};
  for (int k = 0; k < p.ctrl_dim; ++k) m.target[k] = p.target[k];
  m.w_target = p.w_target;
  m.w_obs = p.w_obs;
  m.w_ctrl = p.w_ctrl;
  m.w_term = p.w_term;
  m.n_obs = p.n_obstacles;
  for (int o = 0; o < p.n_obstacles; ++o) {
    for (int k = 0; k < p.ctrl_dim; ++k) m.obs_c[o][k] = p.obs_center[o][k];
    m.obs_r[o] = p.obs_radius[o];
  }
  return m;
}

ChainModel chain_model(const mtp_problem& p) {
  ChainModel m{};
  for (int j = 0; j < p.n_links; ++j) {
    m.mass[j] = p.link_mass[j];
    m.length[j] = p.link_length[j];
  }
  m.gravity = p.gravity;
  m.target[0] = p.target[0];
  m.target[1] = p.target[1];
  m.w_target = p.w_target;
  m.w_ctrl = p.w_ctrl;
  m.w_term = p.w_term;
  return m;
}

LeggedModel legged_model(const mtp_problem& p) {
  LeggedModel m{};
  for (int j = 0; j < p.n_links; ++j) {
    m.mass[j] = p.link_mass[j];
    m.length[j] = p.link_length[j];
  }
  m.gravity = p.gravity;
  m.k_contact = p.k_contact;
  m.c_contact = p.c_contact;
  m.mu_friction = p.mu_friction;
  m.inv_v_slip = 1.f / p.v_slip;
  for (int i = 0; i < 3; ++i) m.target[i] = p.target[i];
  m.w_height = p.w_height;
  m.w_vel = p.w_vel;
  m.w_pitch = p.w_pitch;
  m.w_ctrl = p.w_ctrl;
  m.w_term = p.w_term;
  return m;
}
}  // namespace mtp

namespace {

// Candidate generation of one handle (graph rows, local rows, mean row as
// `c` asks), with the graph written first when it is not regenerated per block.
cudaError_t launch_generate(const mtp_handle* h, CandArgs& c, cudaStream_t s) {
  const bool tc = c.graph_blocks > 0 && h->tc_graph && bspline_tc_eligible(c);
  const int local_blocks = c.U_local ? local_blocks_for(h, (long long)c.local_rows + 1) : 0;
  if (tc && h->side && !h->pipeline && local_blocks > 0) {
    // the graph (its Z, then the tensor-core rows) on the side stream beside
    // the local rows and the mean row: they write disjoint rows of U.  On the
    // 16-link legged workload this took generation from 183 to about 120 us
    // (the serial launches left the tensor-core rows on the critical path)
    cudaError_t e;
    if ((e = cudaEventRecord(h->ev_fork, s)) || (e = cudaStreamWaitEvent(h->side, h->ev_fork, 0))) return e;
    if (!c.C_in) {
      c.Z_global = h->Z;
      if ((e = launch_graph_Z(c, h->Z, h->side))) return e;
    }
    if ((e = launch_bspline_tc(c, h->side)) || (e = cudaEventRecord(h->ev_join, h->side))) return e;
    CandArgs local = c;
    local.graph_blocks = 0;
    if ((e = launch_candidates(local, local_blocks, s))) return e;
    return cudaStreamWaitEvent(s, h->ev_join, 0);
  }
  if (c.graph_blocks > 0 && (h->global_Z || tc) && !c.C_in) {
    c.Z_global = h->Z;
    cudaError_t e = launch_graph_Z(c, h->Z, s);
    if (e != cudaSuccess) return e;
  }
  if (!tc) return launch_candidates(c, local_blocks, s);
  // graph rows on the tensor cores; local rows and the mean row as usual
  CandArgs local = c;
  local.graph_blocks = 0;
  cudaError_t e = launch_candidates(local, local_blocks, s);
  if (e != cudaSuccess) return e;
  return launch_bspline_tc(c, s);
}

// Alg. 2 elite selection of a handle: one block, or two stages when its B
// is beyond one block (many blocks select their chunks, one merges).
cudaError_t launch_selection(const mtp_handle* h, const SelectArgs& a, cudaStream_t s) {
  if (h->sel_chunks > 0) return launch_select_two_stage(a, h->sel_chunk, h->sel_chunks, s);
  return launch_select(a, s);
}

cudaError_t launch_rollout(const mtp_handle* h, const RolloutArgs& a, cudaStream_t s) {
  const mtp_problem& p = h->pr;
  if (p.dyn == MTP_DYN_POINTMASS) return launch_rollout_pointmass(a, pointmass_model(p), h->rollout_chunk, s);
  if (p.dyn == MTP_DYN_LEGGED) return launch_rollout_legged(a, legged_model(p), p.n_links, s);
  return launch_rollout_chain(a, chain_model(p), p.n_links, h->rollout_chunk, s);
}

// Stage event: inside a stream capture it must be an external event record
// node to be timed afterwards (a plain record there only orders streams).
inline void stage_event(cudaEvent_t ev, cudaStream_t s, bool captured) {
  if (captured) cudaEventRecordWithFlags(ev, s, cudaEventRecordExternal);
  else cudaEventRecord(ev, s);
}

// Stage events per iteration: generate, rollout, select, update on the
// launch stream (five marks), and the overlapped preparation on the side
// stream (two marks).
constexpr int kEvPerIter = 7;

// The candidate-generation arguments of the handle's own iteration, writing
// the (B, H, n) tensor U.
CandArgs own_cand_args(const mtp_handle* h, float* U) {
  const Dims& dm = h->dm;
  const size_t Hn = (size_t)dm.H * dm.n;
  CandArgs c = cand_args(h, 0, h->iter_dev);
  c.U_graph = U + Hn * dm.L;
  c.graph_rows = dm.P;
  c.graph_blocks = (dm.P + h->paths_per_block - 1) / h->paths_per_block;
  c.U_local = U;
  c.local_rows = dm.L;
  c.U_mean = U + Hn * (dm.B - 1);
  return c;
}

// How an iteration gets its candidates.
enum class Gen { kFull, kFinish };

// One Alg. 2 iteration on the handle's own buffers, iteration from iter_dev,
// candidates in Ubuf[work].  kFinish: Ubuf[work] already holds this
// iteration's graph rows and local draws.  With the pipeline on, the next
// iteration's graph rows and draws are made into Ubuf[work ^ 1] on the side
// stream while this iteration's rollout runs; the update, which advances
// iter_dev, waits for them.
cudaError_t enqueue_iteration(mtp_handle* h, cudaStream_t s, int work, Gen gen, cudaEvent_t* ev,
                              bool captured = false, float* ustar_out = nullptr) {
  cudaError_t e;
  const Dims& dm = h->dm;
  float* U = h->Ubuf[work];
  if (ev) stage_event(ev[0], s, captured);
  CandArgs c = own_cand_args(h, U);
  if (gen == Gen::kFinish) {
    c.local_mode = h->prep_local ? kLocalFinish : kLocalFull;
    e = launch_finish(c, local_blocks_for(h, (long long)dm.L + 1,
                                          h->prep_local ? kFinishRowsPerThread : kLocalRowsPerThread),
                      s);
  } else {
    e = launch_generate(h, c, s);
  }
  if (e != cudaSuccess) return e;
  if (ev) stage_event(ev[1], s, captured);
  if (h->pipeline) {
    if ((e = cudaEventRecord(h->ev_fork, s)) != cudaSuccess) return e;
    if ((e = cudaStreamWaitEvent(h->side, h->ev_fork, 0)) != cudaSuccess) return e;
    if (ev) stage_event(ev[5], h->side, captured);
    CandArgs nx = own_cand_args(h, h->Ubuf[work ^ 1]);
    nx.iter_offset = 1;
    nx.local_mode = kLocalNoise;
    nx.U_mean = nullptr;
    if (!h->prep_local) nx.U_local = nullptr;
    nx.paths_per_block = h->prep_spb;
    nx.graph_blocks = (dm.P + h->prep_spb - 1) / h->prep_spb;
    if ((e = launch_prepare(nx, h->prep_grid, h->prep_smem, h->side)) != cudaSuccess) return e;
    if (ev) stage_event(ev[6], h->side, captured);
    if ((e = cudaEventRecord(h->ev_join, h->side)) != cudaSuccess) return e;
  }
  RolloutArgs r = rollout_args(h, 0, h->iter_dev, h->x0, U, 0, dm.B, h->cost);
  if ((e = launch_rollout(h, r, s)) != cudaSuccess) return e;
  if (ev) stage_event(ev[2], s, captured);
  SelectArgs sa{h->cost, U, dm.B, dm.E, dm.H, dm.n, 1.0 / h->pr.lambda, h->pr.update_rule,
                h->elite, h->weight, h->ustar, nullptr, ustar_out, h->entropy, h->sel_pairs, 0};
  if ((e = launch_selection(h, sa, s)) != cudaSuccess) return e;
  if (ev) stage_event(ev[3], s, captured);
  if (h->pipeline && (e = cudaStreamWaitEvent(s, h->ev_join, 0)) != cudaSuccess) return e;
  UpdateArgs ua{U, h->elite, h->weight, dm.E, dm.H, dm.n, h->pr.alpha, h->pr.sigma_min,
                h->pr.update_rule, h->mu, h->sigma, h->mu_f, h->sigma_f, h->iter_dev};
  if ((e = launch_update(ua, s)) != cudaSuccess) return e;
  if (ev) stage_event(ev[4], s, captured);
  return cudaSuccess;
}

// Host bookkeeping of one enqueued iteration: which buffer it used, whether
// its successor's draws are prepared.
void after_iteration(mtp_handle* h, int work) {
  h->cur = work;
  h->U = h->Ubuf[work];
  if (h->pipeline) {
    h->prep_valid = true;
    h->prep_iter = h->iter_host + 1;
  }
  h->iter_host += 1;
}

// Sizes of a problem: P graph rows (floor(beta B), at most B - 1), L local
// rows, and the mean row.
Dims dims_of(const mtp_problem& p) {
  Dims dm{};
  dm.B = p.B;
  dm.P = num_graph_samples(p.beta, p.B);
  dm.L = p.B - dm.P - 1;
  dm.E = p.E;
  dm.H = p.horizon;
  dm.n = p.ctrl_dim;
  dm.d = p.state_dim;
  dm.M = p.M;
  dm.N = p.N;
  return dm;
}

// A graph larger than 16 KB is written once per iteration rather than
// regenerated in every graph block's shared memory.
bool global_graph(const Dims& dm) { return (long long)dm.M * dm.N * dm.n > 4096; }

// Graph paths per block, at most 32: about 64K output elements per block for
// B-spline rows, whose blocks otherwise repeat their fixed costs (two
// barriers, the gather of the waypoints) for little work (measured on the
// legged workload, 3,840 elements per row: 4K / 8K / 16K / 32K / 64K / 128K
// elements per block generate in 140.9 / 136.0 / 131.7 / 123.5 / 120.4 /
// 128.2 us); about 4K for Akima and straight lines, and at least 8 paths
// for Akima so its per-(path, dimension) coefficient pass is wide; shrunk
// until the block's shared memory fits.
int paths_per_block_for(const Dims& dm, int32_t interp, bool global_Z) {
  const long long Hn = (long long)dm.H * dm.n;
  const long long target = interp == MTP_INTERP_BSPLINE ? 65536 : 4096;
  int spb = (int)std::min<long long>((target + Hn - 1) / Hn, 32);
  if (interp == MTP_INTERP_AKIMA && spb < 8) spb = 8;
  if (spb < 1) spb = 1;
  if (spb > 32) spb = 32;
  for (;;) {
    CandArgs probe{};
    probe.dm = dm;
    probe.interp = interp;
    probe.graph_blocks = 1;
    probe.paths_per_block = spb;
    probe.Z_global = global_Z ? reinterpret_cast<float*>(16) : nullptr;  // only tested for null
    if (candidates_smem_bytes(probe) <= kMaxSmem || spb == 1) break;
    spb /= 2;
  }
  return spb;
}

// Idle SMs for the pipeline.  From kMinPrepareSMs the next iteration's
// graph rows are prepared beside the rollout and the local rows are drawn
// on the critical path; from kFullPrepareSMs the local rows' draws are
// prepared too and only finished on the critical path.  Measured with L2
// flushed between plan steps, as the bench does:
//  - 7-link arm, B 4096 (24 idle SMs): preparing the draws too lost
//    1.5-13 us per step (their finishing pass reads them back from DRAM,
//    and 24 SMs prepare both in 80 us, longer than the rollout);
//  - 2-D point mass, B 512 (136 idle SMs): preparing the draws too gains
//    4-7 us per step.
constexpr int kMinPrepareSMs = 16;
constexpr int kFullPrepareSMs = 64;

// Whether a single-instance plan step pipelines its generation (see
// mtp_handle::pipeline), whether the local draws are prepared too, on how
// many SMs, with how much shared memory per block.  The point-mass and
// chain rollouts take one block per 32-128 candidates; the legged rollout
// fills the GPU and is not pipelined.
// Whether a problem's graph rows go to the tensor cores: BF16-basis
// B-splines of a shape the contraction takes (H <= 256, M <= 64, n <= 16).
// Other BF16-basis problems use the FP32-pipe window sum with the same BF16
// operands.  (A size threshold, the window sum below 1 M graph outputs, was
// measured and not kept: on the batch of 256 it changed nothing, 2.75 against
// 2.74-2.83 ms.)
bool tc_graph_rule(const mtp_problem& p, const Dims& dm) {
  CandArgs probe{};
  probe.dm = dm;
  probe.bf16 = (p.flags & MTP_FLAG_BF16_BASIS) ? 1 : 0;
  probe.interp = p.interp;
  probe.graph_rows = dm.P;
  return bspline_tc_eligible(probe);
}

cudaError_t pipeline_plan(const mtp_problem& p, const Dims& dm, int paths_per_block, bool* on,
                          bool* local, int* grid, size_t* smem, int* prep_spb) {
  *on = false;
  *local = false;
  *grid = 0;
  *smem = 0;
  *prep_spb = paths_per_block;
  int dev = 0, sms = 0;
  cudaError_t e;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  if ((e = init_prepare_attributes(smem)) != cudaSuccess) return e;
  // graph rows contracted on the tensor cores sum in the tensor cores' order,
  // which the persistent preparation (an FP32-pipe sum) does not reproduce:
  // not pipelined
  if ((p.flags & MTP_FLAG_NO_PIPELINE) || tc_graph_rule(p, dm) || p.dyn == MTP_DYN_LEGGED)
    return cudaSuccess;
  const int free_sms = sms - rollout_blocks(dm.B);
  if (free_sms < kMinPrepareSMs) return cudaSuccess;
  const bool draws = free_sms >= kFullPrepareSMs && dm.L > 0;
  if (!draws && dm.P <= 0) return cudaSuccess;  // nothing to prepare
  CandArgs probe{};
  probe.dm = dm;
  probe.interp = p.interp;
  probe.graph_blocks = dm.P > 0 ? 1 : 0;
  probe.paths_per_block = paths_per_block;
  if (prepare_smem_need(probe) > *smem) return cudaSuccess;
  // a persistent block passes over many paths: wider Akima passes there
  probe.paths_per_block = std::max(paths_per_block, kWideAkimaPaths * (p.interp == MTP_INTERP_AKIMA));
  while (probe.paths_per_block > paths_per_block && prepare_smem_need(probe) > *smem) probe.paths_per_block /= 2;
  *prep_spb = std::max(probe.paths_per_block, paths_per_block);
  *on = true;
  *local = draws;
  *grid = free_sms;
  return cudaSuccess;
}

void free_handle(mtp_handle* h) {
  for (auto& kv : h->graphs) cudaGraphExecDestroy(kv.second);
  for (cudaEvent_t e : h->events) cudaEventDestroy(e);
  for (cudaEvent_t e : h->gevents) cudaEventDestroy(e);
  for (auto& kv : h->pgraphs) cudaGraphExecDestroy(kv.second);
  for (auto& kv : h->hgraphs) cudaGraphExecDestroy(kv.second);
  if (h->x0_pin) cudaFreeHost(h->x0_pin);
  if (h->ustar_pin) cudaFreeHost(h->ustar_pin);
  if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
  if (h->side) cudaStreamDestroy(h->side);
  if (h->ev_fork) cudaEventDestroy(h->ev_fork);
  if (h->ev_join) cudaEventDestroy(h->ev_join);
  void* ptrs[] = {h->basis, h->bfirst, h->seg, h->delta, h->mu, h->sigma, h->mu_f, h->sigma_f,
                  h->iter_dev,
                  h->Ubuf[0], h->Ubuf[1], h->cost, h->elite, h->weight, h->ustar, h->x0, h->Z,
                  h->status, h->entropy, h->sel_pairs};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  delete h;
}

}  // namespace

extern "C" {

size_t mtp_problem_bytes(void) { return sizeof(mtp_problem); }

mtp_status mtp_create(const mtp_problem* problem, mtp_handle** out) {
  if (!problem || !out) return fail(nullptr, MTP_ERR_INVALID_ARG, "null argument");
  *out = nullptr;
  mtp_status st = validate(*problem);
  if (st != MTP_OK) return st;
  mtp_handle* h = new mtp_handle();
  h->pr = normalized(*problem);
  const mtp_problem& p = h->pr;
  cudaGetDevice(&h->device);
  Dims& dm = h->dm;
  dm = dims_of(p);
  h->key.k0 = (uint32_t)(p.seed & 0xffffffffu);
  h->key.k1 = (uint32_t)(p.seed >> 32);
  h->global_Z = global_graph(dm);
  h->paths_per_block = paths_per_block_for(dm, p.interp, h->global_Z);
  h->tc_graph = tc_graph_rule(p, dm);
  select_plan(dm.B, dm.E, &h->sel_chunk, &h->sel_chunks);
  auto err = [&](mtp_status s) {
    g_create_error = h->err;
    free_handle(h);
    return s;
  };
  cudaError_t e;
  if ((e = init_candidate_attributes()) != cudaSuccess) return err(cuda_fail(h, e, "attributes"));
  if ((e = init_select_attributes()) != cudaSuccess) return err(cuda_fail(h, e, "attributes"));
  if ((e = init_rollout_pm_attributes()) != cudaSuccess) return err(cuda_fail(h, e, "attributes"));
  if ((e = init_rollout_chain_attributes()) != cudaSuccess) return err(cuda_fail(h, e, "attributes"));
  if ((e = init_bspline_tc_attributes()) != cudaSuccess) return err(cuda_fail(h, e, "attributes"));
  if ((e = pipeline_plan(p, dm, h->paths_per_block, &h->pipeline, &h->prep_local, &h->prep_grid,
                         &h->prep_smem, &h->prep_spb)) !=
      cudaSuccess)
    return err(cuda_fail(h, e, "attributes"));
  if ((st = build_tables(h)) != MTP_OK) return err(st);
  const size_t rowsz = (size_t)dm.H * dm.n;
  if ((e = dalloc(&h->mu, rowsz)) || (e = dalloc(&h->sigma, rowsz)) ||
      (e = dalloc(&h->mu_f, rowsz)) || (e = dalloc(&h->sigma_f, rowsz)) ||
      (e = dalloc(&h->iter_dev, 1)) || (e = dalloc(&h->Ubuf[0], rowsz * dm.B)) ||
      (e = dalloc(&h->cost, dm.B)) || (e = dalloc(&h->elite, dm.E)) ||
      (e = dalloc(&h->weight, dm.E)) || (e = dalloc(&h->ustar, dm.n)) ||
      (e = dalloc(&h->x0, dm.d)) || (e = dalloc(&h->Z, (size_t)dm.M * dm.N * dm.n)) ||
      (e = dalloc(&h->status, 1)) ||
      ((p.flags & MTP_FLAG_COST_ENTROPY) && (e = dalloc(&h->entropy, 1))) ||
      (h->sel_chunks > 0 && (e = dalloc(&h->sel_pairs, (size_t)h->sel_chunks * dm.E))))
    return err(cuda_fail(h, e, "cudaMalloc"));
  std::vector<double> mu(rowsz, p.mu_init), sg(rowsz, p.sigma_init);
  std::vector<float> muf(rowsz, (float)p.mu_init), sgf(rowsz, (float)p.sigma_init);
  uint32_t zero = 0;
  if ((e = cudaMemcpy(h->mu, mu.data(), rowsz * 8, cudaMemcpyHostToDevice)) ||
      (e = cudaMemcpy(h->sigma, sg.data(), rowsz * 8, cudaMemcpyHostToDevice)) ||
      (e = cudaMemcpy(h->mu_f, muf.data(), rowsz * 4, cudaMemcpyHostToDevice)) ||
      (e = cudaMemcpy(h->sigma_f, sgf.data(), rowsz * 4, cudaMemcpyHostToDevice)) ||
      (e = cudaMemcpy(h->iter_dev, &zero, 4, cudaMemcpyHostToDevice)) ||
      (e = cudaMemset(h->ustar, 0, dm.n * 4)) || (e = cudaMemset(h->status, 0, 4)))
    return err(cuda_fail(h, e, "cudaMemcpy"));
  h->U = h->Ubuf[0];
  if ((e = cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking)) != cudaSuccess)
    return err(cuda_fail(h, e, "cudaStreamCreate"));
  *out = h;
  return MTP_OK;
}

mtp_status mtp_problem_device_bytes(const mtp_problem* problem, uint64_t* bytes) {
  if (!problem || !bytes) return fail(nullptr, MTP_ERR_INVALID_ARG, "null argument");
  mtp_status st = validate(*problem);
  if (st != MTP_OK) return st;
  const mtp_problem p = normalized(*problem);
  const uint64_t rowsz = (uint64_t)p.horizon * p.ctrl_dim;
  auto r = [](uint64_t b) { return (b + 511) & ~uint64_t(511); };  // allocation granularity
  *bytes = r((uint64_t)p.horizon * p.M * 4) + 3 * r((uint64_t)p.horizon * 4)  // tables
           + 2 * r(rowsz * 8) + 2 * r(rowsz * 4) + r(4)                       // mean, spread
           + r(rowsz * p.B * 4) + r((uint64_t)p.B * 4)                        // U, cost
           + r((uint64_t)p.E * 4) + r((uint64_t)p.E * 8)                      // elites, weights
           + r((uint64_t)p.ctrl_dim * 4) + r((uint64_t)p.state_dim * 4)
           + r((uint64_t)p.M * p.N * p.ctrl_dim * 4)                          // graph Z
           + r(4)                                                             // status word
           + ((p.flags & MTP_FLAG_COST_ENTROPY) ? r(8) : 0);                  // entropy
  {
    int chunk = 0, chunks = 0;
    select_plan(p.B, p.E, &chunk, &chunks);
    if (chunks > 0) *bytes += r((uint64_t)chunks * p.E * 8);          // selection pairs
  }
  const Dims dm = dims_of(p);
  bool on = false, local = false;
  int grid = 0;
  size_t smem = 0;
  int spb = 1;
  cudaError_t e = pipeline_plan(p, dm, paths_per_block_for(dm, p.interp, global_graph(dm)), &on, &local,
                                &grid, &smem, &spb);
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "device query");
  if (on) *bytes += r(rowsz * p.B * 4);  // the second candidate buffer of the pipelined plan step
  return MTP_OK;
}

mtp_status mtp_destroy(mtp_handle* h) {
  if (!h) return MTP_ERR_INVALID_ARG;
  DeviceGuard g(h->device);
  cudaDeviceSynchronize();
  free_handle(h);
  return MTP_OK;
}

const char* mtp_last_error(const mtp_handle* h) {
  return h ? h->err.c_str() : g_create_error.c_str();
}

mtp_status mtp_get_sizes(const mtp_handle* h, mtp_sizes* out) {
  if (!h || !out) return MTP_ERR_INVALID_ARG;
  const Dims& d = h->dm;
  // candidates (+ graph when written once), rollout, select, update; when
  // pipelined: finish, prepare (graph in its shared memory), rollout, select, update
  // (tensor-core graph rows: graph, local rows, contraction, rollout, select, update)
  const int kpi = (h->pipeline ? 5 : (h->tc_graph ? 6 : (h->global_Z && d.P > 0 ? 5 : 4))) +
                  (h->sel_chunks > 0 ? 1 : 0);  // the two-stage selection's second launch
  *out = mtp_sizes{d.B, d.P, d.L, d.E, d.H, d.n, d.d, d.M, d.N, kpi,
                   h->pipeline ? (h->prep_local ? 2 : 1) : 0};
  return MTP_OK;
}

mtp_status mtp_get_buffers(const mtp_handle* h, mtp_buffers* out) {
  if (!h || !out) return MTP_ERR_INVALID_ARG;
  *out = mtp_buffers{h->U, h->cost, h->elite, h->weight, h->mu, h->sigma, h->ustar, h->iter_dev};
  return MTP_OK;
}

mtp_status mtp_sample_tensor(mtp_handle* h, uint32_t iter, float* d_Z, int32_t* d_idx,
                             float* d_C, void* stream) {
  if (!h) return MTP_ERR_INVALID_ARG;
  DeviceGuard g(h->device);
  cudaError_t e = launch_sample_tensor(h->dm, h->key, iter, h->pr.u_min, h->pr.u_max, d_Z, d_idx,
                                       d_C, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "sample_tensor");
  return MTP_OK;
}

mtp_status mtp_interpolate(mtp_handle* h, const float* d_C, int32_t P, float* d_U, void* stream) {
  if (!h || !d_C || !d_U || P < 0) return fail(h, MTP_ERR_INVALID_ARG, "interpolate: bad argument");
  if (P == 0) return MTP_OK;
  DeviceGuard g(h->device);
  CandArgs c = cand_args(h, 0, nullptr);
  c.C_in = d_C;
  c.U_graph = d_U;
  c.graph_rows = P;
  c.graph_blocks = (P + h->paths_per_block - 1) / h->paths_per_block;
  cudaError_t e = (h->tc_graph && bspline_tc_eligible(c))
                      ? launch_bspline_tc(c, (cudaStream_t)stream)
                      : launch_candidates(c, 0, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "interpolate");
  return MTP_OK;
}

mtp_status mtp_sample_local(mtp_handle* h, uint32_t iter, float* d_U, void* stream) {
  if (!h || !d_U) return fail(h, MTP_ERR_INVALID_ARG, "sample_local: bad argument");
  DeviceGuard g(h->device);
  const size_t Hn = (size_t)h->dm.H * h->dm.n;
  CandArgs c = cand_args(h, iter, nullptr);
  c.U_local = d_U;
  c.local_rows = h->dm.L;
  c.U_mean = d_U + Hn * (h->dm.B - 1);
  cudaError_t e = launch_generate(h, c, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "sample_local");
  return MTP_OK;
}

mtp_status mtp_generate_candidates(mtp_handle* h, uint32_t iter, float* d_U, void* stream) {
  if (!h || !d_U) return fail(h, MTP_ERR_INVALID_ARG, "generate_candidates: bad argument");
  DeviceGuard g(h->device);
  const Dims& dm = h->dm;
  const size_t Hn = (size_t)dm.H * dm.n;
  CandArgs c = cand_args(h, iter, nullptr);
  c.U_graph = d_U + Hn * dm.L;
  c.graph_rows = dm.P;
  c.graph_blocks = (dm.P + h->paths_per_block - 1) / h->paths_per_block;
  c.U_local = d_U;
  c.local_rows = dm.L;
  c.U_mean = d_U + Hn * (dm.B - 1);
  cudaError_t e = launch_generate(h, c, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "generate_candidates");
  return MTP_OK;
}

mtp_status mtp_rollout_cost(mtp_handle* h, uint32_t iter, const float* d_x0, const float* d_U,
                            int32_t row0, int32_t rows, float* d_cost, void* stream) {
  if (!h || !d_x0 || !d_U || !d_cost || row0 < 0 || rows < 0 || row0 + rows > h->dm.B)
    return fail(h, MTP_ERR_INVALID_ARG, "rollout_cost: bad argument");
  DeviceGuard g(h->device);
  RolloutArgs a = rollout_args(h, iter, nullptr, d_x0, d_U, row0, rows, d_cost);
  cudaError_t e = launch_rollout(h, a, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "rollout_cost");
  return MTP_OK;
}

mtp_status mtp_rollout_states(mtp_handle* h, uint32_t iter, const float* d_x0, const float* d_Urow,
                              int32_t row, float* d_X, float* d_cost, void* stream) {
  if (!h || !d_x0 || !d_Urow || !d_X || !d_cost || row < 0 || row >= h->dm.B)
    return fail(h, MTP_ERR_INVALID_ARG, "rollout_states: bad argument");
  if (h->pr.dr_mode == MTP_DR_SHARED)
    return fail(h, MTP_ERR_INVALID_ARG, "rollout_states: one trajectory per model is ambiguous with shared models");
  DeviceGuard g(h->device);
  RolloutArgs a = rollout_args(h, iter, nullptr, d_x0, d_Urow, row, 1, d_cost);
  a.X = d_X;
  cudaError_t e = launch_rollout(h, a, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "rollout_states");
  return MTP_OK;
}

mtp_status mtp_elite_update(mtp_handle* h, const float* d_cost, const float* d_U, int32_t* d_elite,
                            float* d_ustar, void* stream) {
  if (!h || !d_cost || !d_U) return fail(h, MTP_ERR_INVALID_ARG, "elite_update: bad argument");
  DeviceGuard g(h->device);
  const Dims& dm = h->dm;
  cudaStream_t s = (cudaStream_t)stream;
  SelectArgs sa{d_cost, d_U, dm.B, dm.E, dm.H, dm.n, 1.0 / h->pr.lambda, h->pr.update_rule,
                h->elite, h->weight, h->ustar, d_elite, d_ustar, h->entropy, h->sel_pairs, 0};
  cudaError_t e = launch_selection(h, sa, s);
  if (e != cudaSuccess) return cuda_fail(h, e, "select");
  UpdateArgs ua{d_U, h->elite, h->weight, dm.E, dm.H, dm.n, h->pr.alpha, h->pr.sigma_min,
                h->pr.update_rule, h->mu, h->sigma, h->mu_f, h->sigma_f, nullptr};
  e = launch_update(ua, s);
  if (e != cudaSuccess) return cuda_fail(h, e, "update");
  return MTP_OK;
}

// Candidate buffer and generation route of iteration j of a run of
// iterations that starts from the handle's current state.
static void iteration_plan(const mtp_handle* h, int c0, bool first_prepared, int j, int* work, Gen* gen) {
  if (!h->pipeline) {
    *work = 0;
    *gen = Gen::kFull;
    return;
  }
  *work = c0 ^ ((j + 1) & 1);
  *gen = (j > 0 || first_prepared) ? Gen::kFinish : Gen::kFull;
}

static mtp_status read_stage_events(mtp_handle* h, const cudaEvent_t* ev, double* acc) {
  cudaError_t e;
  for (int st = 0; st < 4; ++st) {
    float ms = 0.f;
    if ((e = cudaEventElapsedTime(&ms, ev[st], ev[st + 1])) != cudaSuccess)
      return cuda_fail(h, e, "cudaEventElapsedTime");
    acc[st] += ms;
  }
  if (h->pipeline) {
    float ms = 0.f;
    if ((e = cudaEventElapsedTime(&ms, ev[5], ev[6])) != cudaSuccess)
      return cuda_fail(h, e, "cudaEventElapsedTime");
    acc[4] += ms;
  }
  return MTP_OK;
}

// The pipeline's second candidate buffer, stream and events, made by the
// first single-instance plan step that uses them (a handle planned only in
// batches never needs them).  If they cannot be made the handle plans
// without the pipeline, which gives the same results.
static void ensure_pipeline(mtp_handle* h) {
  if (h->tc_graph && !h->pipeline && !h->side) {
    // a tensor-core handle's side stream for its graph rows (launch_generate);
    // without it the rows are made after the local rows, with the same bits
    if (cudaStreamCreateWithFlags(&h->side, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming) != cudaSuccess) {
      cudaGetLastError();
      if (h->side) cudaStreamDestroy(h->side);
      if (h->ev_fork) cudaEventDestroy(h->ev_fork);
      if (h->ev_join) cudaEventDestroy(h->ev_join);
      h->side = nullptr;
      h->ev_fork = h->ev_join = nullptr;
    }
    return;
  }
  if (!h->pipeline || h->side) return;
  const size_t n = (size_t)h->dm.H * h->dm.n * h->dm.B;
  if (dalloc(&h->Ubuf[1], n) != cudaSuccess ||
      cudaStreamCreateWithFlags(&h->side, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();  // clear the failure: the plain path needs none of these
    if (h->Ubuf[1]) cudaFree(h->Ubuf[1]);
    if (h->side) cudaStreamDestroy(h->side);
    if (h->ev_fork) cudaEventDestroy(h->ev_fork);
    if (h->ev_join) cudaEventDestroy(h->ev_join);
    h->Ubuf[1] = nullptr;
    h->side = nullptr;
    h->ev_fork = h->ev_join = nullptr;
    h->pipeline = false;
    h->prep_local = false;
    h->prep_valid = false;
    h->cur = 0;
    h->U = h->Ubuf[0];
  }
}

// The CUDA graph of `chunk` iterations starting from buffer c0 (the first
// iteration's draws prepared or not), captured on first use into `cache`.
// With `events` (profiling) each iteration records its stage events; with
// `x0_src` (pinned) the graph first uploads the start state from it, and the
// last iteration's selection also writes u* to `ustar_dst` (pinned).
static mtp_status chunk_graph(mtp_handle* h, std::map<int, cudaGraphExec_t>& cache, int chunk, int c0,
                              bool prepared, bool events, const float* x0_src, float* ustar_dst,
                              cudaGraphExec_t* out) {
  const int key = chunk * 4 + c0 * 2 + (prepared ? 1 : 0);
  auto it = cache.find(key);
  if (it != cache.end()) {
    *out = it->second;
    return MTP_OK;
  }
  cudaError_t e;
  cudaGraph_t graph;
  if ((e = cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal)) != cudaSuccess)
    return cuda_fail(h, e, "cudaStreamBeginCapture");
  if (x0_src)
    e = cudaMemcpyAsync(h->x0, x0_src, (size_t)h->dm.d * 4, cudaMemcpyHostToDevice, h->cap_stream);
  for (int k = 0; k < chunk && e == cudaSuccess; ++k) {
    cudaEvent_t* ev = events ? h->gevents.data() + kEvPerIter * k : nullptr;
    int work;
    Gen gen;
    iteration_plan(h, c0, prepared, k, &work, &gen);
    e = enqueue_iteration(h, h->cap_stream, work, gen, ev, true, k == chunk - 1 ? ustar_dst : nullptr);
  }
  if (e != cudaSuccess) {
    cudaStreamEndCapture(h->cap_stream, &graph);
    if (graph) cudaGraphDestroy(graph);
    return cuda_fail(h, e, "capture");
  }
  if ((e = cudaStreamEndCapture(h->cap_stream, &graph)) != cudaSuccess)
    return cuda_fail(h, e, "cudaStreamEndCapture");
  cudaGraphExec_t exec;
  e = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) return cuda_fail(h, e, "cudaGraphInstantiate");
  cache.emplace(key, exec);
  *out = exec;
  return MTP_OK;
}

// Host bookkeeping of a launched chunk (see after_iteration).
static void after_chunk(mtp_handle* h, int chunk, int c0, bool prepared) {
  for (int k = 0; k < chunk; ++k) {
    int work;
    Gen gen;
    iteration_plan(h, c0, prepared, k, &work, &gen);
    after_iteration(h, work);
  }
}

static mtp_status plan_device(mtp_handle* h, int32_t iters, cudaStream_t s) {
  cudaError_t e;
  ensure_pipeline(h);
  const bool use_graph = !(h->pr.flags & MTP_FLAG_NO_GRAPH);
  if (!use_graph) {
    for (int k = 0; k < iters; ++k) {
      cudaEvent_t* ev = nullptr;
      if (h->profiling) {
        while (h->events.size() < h->ev_used + kEvPerIter) {
          cudaEvent_t x;
          if ((e = cudaEventCreate(&x)) != cudaSuccess) return cuda_fail(h, e, "cudaEventCreate");
          h->events.push_back(x);
        }
        ev = h->events.data() + h->ev_used;
        h->ev_used += kEvPerIter;
      }
      const bool prepared = h->pipeline && h->prep_valid && h->prep_iter == h->iter_host;
      int work;
      Gen gen;
      iteration_plan(h, h->cur, prepared, 0, &work, &gen);
      if ((e = enqueue_iteration(h, s, work, gen, ev)) != cudaSuccess) return cuda_fail(h, e, "plan_step");
      after_iteration(h, work);
    }
    return MTP_OK;
  }
  // one captured graph per distinct (iteration count, starting buffer,
  // whether the first iteration's draws are prepared), at most 64
  // iterations each; with profiling on, a second set of graphs also records
  // the stage events, and each replay is waited for and its stage times
  // accumulated
  constexpr int kChunk = 64;
  if (h->profiling) {
    while (h->gevents.size() < (size_t)kEvPerIter * kChunk) {
      cudaEvent_t x;
      if ((e = cudaEventCreate(&x)) != cudaSuccess) return cuda_fail(h, e, "cudaEventCreate");
      h->gevents.push_back(x);
    }
  }
  auto& cache = h->profiling ? h->pgraphs : h->graphs;
  int left = iters;
  while (left > 0) {
    const int chunk = left > kChunk ? kChunk : left;
    const int c0 = h->cur;
    const bool prepared = h->pipeline && h->prep_valid && h->prep_iter == h->iter_host;
    cudaGraphExec_t exec;
    mtp_status st = chunk_graph(h, cache, chunk, c0, prepared, h->profiling, nullptr, nullptr, &exec);
    if (st != MTP_OK) return st;
    if ((e = cudaGraphLaunch(exec, s)) != cudaSuccess) return cuda_fail(h, e, "cudaGraphLaunch");
    after_chunk(h, chunk, c0, prepared);
    if (h->profiling) {
      if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return cuda_fail(h, e, "profiled replay");
      for (int k = 0; k < chunk; ++k) {
        const mtp_status rs = read_stage_events(h, h->gevents.data() + kEvPerIter * k, h->stage_acc);
        if (rs != MTP_OK) return rs;
      }
      h->stage_iters += chunk;
    }
    left -= chunk;
  }
  return MTP_OK;
}

mtp_status mtp_plan_step(mtp_handle* h, const float* d_x0, int32_t iters, float* d_ustar, void* stream) {
  if (!h || !d_x0 || !d_ustar || iters < 1) return fail(h, MTP_ERR_INVALID_ARG, "plan_step: bad argument");
  DeviceGuard g(h->device);
  cudaStream_t s = (cudaStream_t)stream;
  MTP_CUDA(h, cudaMemcpyAsync(h->x0, d_x0, h->dm.d * 4, cudaMemcpyDeviceToDevice, s));
  mtp_status st = plan_device(h, iters, s);
  if (st != MTP_OK) return st;
  MTP_CUDA(h, cudaMemcpyAsync(d_ustar, h->ustar, h->dm.n * 4, cudaMemcpyDeviceToDevice, s));
  return MTP_OK;
}

// mtp_plan_step_host in one graph launch: the start state is staged in
// pinned memory and its upload is the graph's first node, and the last
// iteration's selection kernel writes u* straight into pinned memory, so a
// call is one graph launch and one synchronisation.  Up to 64 iterations,
// graph mode, profiling off; otherwise the caller takes the general path.
static bool plan_host_graph(mtp_handle* h, const float* h_x0, int32_t iters, float* h_ustar,
                            cudaStream_t s, mtp_status* st) {
  constexpr int kChunk = 64;
  if ((h->pr.flags & MTP_FLAG_NO_GRAPH) || h->profiling || iters > kChunk) return false;
  cudaError_t e;
  if (!h->x0_pin) {
    if (cudaMallocHost(&h->x0_pin, (size_t)h->dm.d * 4) != cudaSuccess ||
        cudaMallocHost(&h->ustar_pin, (size_t)h->dm.n * 4) != cudaSuccess) {
      cudaGetLastError();
      if (h->x0_pin) cudaFreeHost(h->x0_pin);
      h->x0_pin = nullptr;
      h->ustar_pin = nullptr;
      return false;
    }
  }
  ensure_pipeline(h);
  std::memcpy(h->x0_pin, h_x0, (size_t)h->dm.d * 4);
  const int c0 = h->cur;
  const bool prepared = h->pipeline && h->prep_valid && h->prep_iter == h->iter_host;
  cudaGraphExec_t exec;
  *st = chunk_graph(h, h->hgraphs, iters, c0, prepared, false, h->x0_pin, h->ustar_pin, &exec);
  if (*st != MTP_OK) return true;
  if ((e = cudaGraphLaunch(exec, s)) != cudaSuccess) {
    *st = cuda_fail(h, e, "cudaGraphLaunch");
    return true;
  }
  after_chunk(h, iters, c0, prepared);
  if ((e = cudaStreamSynchronize(s)) != cudaSuccess) {
    *st = cuda_fail(h, e, "cudaStreamSynchronize");
    return true;
  }
  std::memcpy(h_ustar, h->ustar_pin, (size_t)h->dm.n * 4);
  *st = MTP_OK;
  return true;
}

mtp_status mtp_plan_step_host(mtp_handle* h, const float* h_x0, int32_t iters, float* h_ustar,
                              void* stream) {
  if (!h || !h_x0 || !h_ustar || iters < 1) return fail(h, MTP_ERR_INVALID_ARG, "plan_step_host: bad argument");
  DeviceGuard g(h->device);
  cudaStream_t s = (cudaStream_t)stream;
  mtp_status hs = MTP_OK;
  if (plan_host_graph(h, h_x0, iters, h_ustar, s, &hs)) return hs;
  MTP_CUDA(h, cudaMemcpyAsync(h->x0, h_x0, h->dm.d * 4, cudaMemcpyHostToDevice, s));
  mtp_status st = plan_device(h, iters, s);
  if (st != MTP_OK) return st;
  MTP_CUDA(h, cudaMemcpyAsync(h_ustar, h->ustar, h->dm.n * 4, cudaMemcpyDeviceToHost, s));
  MTP_CUDA(h, cudaStreamSynchronize(s));
  return MTP_OK;
}

mtp_status mtp_shift(mtp_handle* h, int32_t k, void* stream) {
  if (!h || k < 0) return fail(h, MTP_ERR_INVALID_ARG, "shift: bad argument");
  if (k == 0) return MTP_OK;
  DeviceGuard g(h->device);
  cudaError_t e = launch_shift(h->mu, h->sigma, h->mu_f, h->sigma_f, h->dm.H, h->dm.n, k,
                               (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "shift");
  return MTP_OK;
}

mtp_status mtp_cost_entropy(mtp_handle* h, double* h_entropy) {
  if (!h || !h_entropy) return fail(h, MTP_ERR_INVALID_ARG, "cost_entropy: bad argument");
  if (!h->entropy)
    return fail(h, MTP_ERR_INVALID_ARG, "cost_entropy: create the problem with MTP_FLAG_COST_ENTROPY");
  DeviceGuard g(h->device);
  MTP_CUDA(h, cudaDeviceSynchronize());
  MTP_CUDA(h, cudaMemcpy(h_entropy, h->entropy, 8, cudaMemcpyDeviceToHost));
  return MTP_OK;
}

mtp_status mtp_device_status(mtp_handle* h) {
  if (!h) return MTP_ERR_INVALID_ARG;
  DeviceGuard g(h->device);
  uint32_t word = 0;
  MTP_CUDA(h, cudaDeviceSynchronize());
  MTP_CUDA(h, cudaMemcpy(&word, h->status, 4, cudaMemcpyDeviceToHost));
  if (word == 0) return MTP_OK;
  MTP_CUDA(h, cudaMemset(h->status, 0, 4));
  return fail(h, MTP_ERR_TIMEOUT,
              "a rollout's bounded wait for its staged controls gave up (those candidates cost +inf)");
}

mtp_status mtp_get_state(mtp_handle* h, double* h_mu, double* h_sigma, uint32_t* h_iter) {
  if (!h) return MTP_ERR_INVALID_ARG;
  DeviceGuard g(h->device);
  const size_t bytes = (size_t)h->dm.H * h->dm.n * 8;
  MTP_CUDA(h, cudaDeviceSynchronize());
  if (h_mu) MTP_CUDA(h, cudaMemcpy(h_mu, h->mu, bytes, cudaMemcpyDeviceToHost));
  if (h_sigma) MTP_CUDA(h, cudaMemcpy(h_sigma, h->sigma, bytes, cudaMemcpyDeviceToHost));
  if (h_iter) MTP_CUDA(h, cudaMemcpy(h_iter, h->iter_dev, 4, cudaMemcpyDeviceToHost));
  return MTP_OK;
}

mtp_status mtp_set_state(mtp_handle* h, const double* h_mu, const double* h_sigma, uint32_t iter) {
  if (!h || !h_mu || !h_sigma) return MTP_ERR_INVALID_ARG;
  DeviceGuard g(h->device);
  const size_t bytes = (size_t)h->dm.H * h->dm.n * 8;
  MTP_CUDA(h, cudaDeviceSynchronize());
  MTP_CUDA(h, cudaMemcpy(h->mu, h_mu, bytes, cudaMemcpyHostToDevice));
  MTP_CUDA(h, cudaMemcpy(h->sigma, h_sigma, bytes, cudaMemcpyHostToDevice));
  const size_t cnt = (size_t)h->dm.H * h->dm.n;
  std::vector<float> muf(cnt), sgf(cnt);
  for (size_t i = 0; i < cnt; ++i) {
    muf[i] = (float)h_mu[i];
    sgf[i] = (float)h_sigma[i];
  }
  MTP_CUDA(h, cudaMemcpy(h->mu_f, muf.data(), cnt * 4, cudaMemcpyHostToDevice));
  MTP_CUDA(h, cudaMemcpy(h->sigma_f, sgf.data(), cnt * 4, cudaMemcpyHostToDevice));
  MTP_CUDA(h, cudaMemcpy(h->iter_dev, &iter, 4, cudaMemcpyHostToDevice));
  h->iter_host = iter;
  return MTP_OK;
}

mtp_status mtp_set_profiling(mtp_handle* h, int32_t enable) {
  if (!h) return MTP_ERR_INVALID_ARG;
  h->profiling = enable != 0;
  h->ev_used = 0;
  for (int i = 0; i < 5; ++i) h->stage_acc[i] = 0.0;
  h->stage_iters = 0;
  return MTP_OK;
}

static mtp_status stage_times(mtp_handle* h, double* ms5, int32_t* iterations) {
  DeviceGuard g(h->device);
  for (int i = 0; i < 5; ++i) ms5[i] = h->stage_acc[i];
  const int64_t g_it = h->stage_iters;
  for (int i = 0; i < 5; ++i) h->stage_acc[i] = 0.0;
  h->stage_iters = 0;
  const size_t n_it = h->ev_used / kEvPerIter;
  // the update's end mark follows the side stream's work (the update waits for it)
  if (n_it > 0) MTP_CUDA(h, cudaEventSynchronize(h->events[h->ev_used - kEvPerIter + 4]));
  for (size_t k = 0; k < n_it; ++k) {
    mtp_status st = read_stage_events(h, h->events.data() + kEvPerIter * k, ms5);
    if (st != MTP_OK) return st;
  }
  if (iterations) *iterations = (int32_t)(n_it + g_it);
  h->ev_used = 0;
  return MTP_OK;
}

mtp_status mtp_stage_times(mtp_handle* h, double* ms4, int32_t* iterations) {
  if (!h || !ms4) return MTP_ERR_INVALID_ARG;
  double ms5[5];
  mtp_status st = stage_times(h, ms5, iterations);
  for (int i = 0; i < 4; ++i) ms4[i] = ms5[i];
  return st;
}

mtp_status mtp_stage_times5(mtp_handle* h, double* ms5, int32_t* iterations) {
  if (!h || !ms5) return MTP_ERR_INVALID_ARG;
  return stage_times(h, ms5, iterations);
}

}  // extern "C"
