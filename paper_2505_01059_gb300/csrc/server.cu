// server.cu -- the re-plan server: continuous batching of many robots'
// receding-horizon planning requests onto batched planner cycles.
//
// Built on the public batch API only.  A worker thread owns two cycle slots,
// each a batch workspace with its own stream, pinned staging and device
// buffers, all allocated when the server is created.  A cycle takes the
// requests the scheduler hands out, refills its slot's batch tables (one
// copy), uploads the start states, runs the planner iterations (Alg. 2 loop
// body, batched as in Sec. 3.3 / Sec. 4), applies the warm-start shift and
// copies u* back; while it runs the worker can start the other slot on
// robots that are not in flight.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cstring>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "../../include/mtp.h"
#include "scheduler.h"

namespace mtp {
void set_thread_error(const std::string& msg);  // text of mtp_last_error(NULL)
}

namespace {

constexpr int kSlots = 2;
constexpr int kMaxState = 2 * MTP_MAX_CTRL;  // point mass, k = 32, is the widest state
constexpr double kIdleWait = 0.005;          // worker's wait for work when nothing is in flight
constexpr double kBusyWait = 50e-6;          // ... and between checks of a cycle in flight

struct Slot {
  mtp_batch* b = nullptr;
  cudaStream_t s = nullptr;
  cudaEvent_t done = nullptr;
  float* h_x0 = nullptr;  // pinned
  float* h_us = nullptr;  // pinned
  float* d_x0 = nullptr;
  float* d_us = nullptr;
  std::vector<mtp_sched::Request> reqs;
  std::vector<int32_t> us_off;
  bool busy = false;
  uint64_t seq = 0;  // launch order of the cycle in the slot
};

}  // namespace

struct mtp_server {
  mtp_server_config cfg{};
  int device = 0;
  uint64_t budget = 0;
  mtp_sched::Scheduler sched;
  std::mutex reg_mu;  // guards the robot tables and the admitted bytes
  std::vector<mtp_handle*> robots;
  std::vector<int32_t> robot_d, robot_n;
  uint64_t bytes_admitted = 0;  // robots admitted, and registrations in progress
  int registering = 0;          // registrations between admission and their handle
  Slot slots[kSlots];
  std::thread worker;
  std::atomic<bool> stop{false};
  std::atomic<int> failed{0};
  std::atomic<uint64_t> cycles{0}, planned{0};
  uint64_t seq = 0;
  mutable std::mutex err_mu;
  std::string err;

  mtp_server(const mtp_server_config& c) : cfg(c), sched(c.max_batch, c.max_queue) {}

  void set_error(const std::string& msg) {
    std::lock_guard<std::mutex> lock(err_mu);
    err = msg;
  }
};

namespace {

struct DeviceScope {
  int prev = -1;
  explicit DeviceScope(int dev) {
    if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
    else prev = -1;
  }
  ~DeviceScope() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

void free_slot(Slot& sl) {
  if (sl.b) mtp_batch_destroy(sl.b);
  if (sl.s) cudaStreamDestroy(sl.s);
  if (sl.done) cudaEventDestroy(sl.done);
  if (sl.h_x0) cudaFreeHost(sl.h_x0);
  if (sl.h_us) cudaFreeHost(sl.h_us);
  if (sl.d_x0) cudaFree(sl.d_x0);
  if (sl.d_us) cudaFree(sl.d_us);
  sl = Slot();
}

cudaError_t alloc_slot(Slot& sl, int cap) {
  const size_t xb = sizeof(float) * (size_t)cap * kMaxState, ub = sizeof(float) * (size_t)cap * MTP_MAX_CTRL;
  cudaError_t e;
  if ((e = cudaStreamCreateWithFlags(&sl.s, cudaStreamNonBlocking)) ||
      (e = cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming)) ||
      (e = cudaMallocHost((void**)&sl.h_x0, xb)) || (e = cudaMallocHost((void**)&sl.h_us, ub)) ||
      (e = cudaMalloc((void**)&sl.d_x0, xb)) || (e = cudaMalloc((void**)&sl.d_us, ub)))
    return e;
  sl.reqs.reserve(cap);
  sl.us_off.assign(cap + 1, 0);
  return cudaSuccess;
}

// Waits for the slot's cycle and hands its results to the scheduler.
bool finish(mtp_server* S, Slot& sl) {
  cudaError_t e = cudaEventSynchronize(sl.done);
  sl.busy = false;
  if (e != cudaSuccess) {
    S->set_error(std::string("server cycle: ") + cudaGetErrorString(e));
    return false;
  }
  const double now = mtp_sched::now_seconds();
  for (size_t i = 0; i < sl.reqs.size(); ++i)
    S->sched.complete(sl.reqs[i], sl.h_us + sl.us_off[i], sl.us_off[i + 1] - sl.us_off[i], now);
  sl.reqs.clear();
  return true;
}

// Enqueues one cycle over `reqs` in an idle slot.
bool launch(mtp_server* S, Slot& sl, std::vector<mtp_sched::Request>&& reqs) {
  const int count = (int)reqs.size();
  std::vector<mtp_handle*> hs(count);
  {
    std::lock_guard<std::mutex> lock(S->reg_mu);
    for (int i = 0; i < count; ++i) hs[i] = S->robots[reqs[i].robot];
  }
  sl.reqs = std::move(reqs);
  std::vector<int32_t> x0_off(count + 1);
  mtp_status st;
  auto bail = [&](const char* where) {
    S->set_error(std::string(where) + ": " + mtp_last_error(nullptr));
    return false;
  };
  if ((st = mtp_batch_fill(sl.b, hs.data(), count, sl.s)) != MTP_OK) return bail("server fill");
  if ((st = mtp_batch_layout(sl.b, x0_off.data(), sl.us_off.data())) != MTP_OK) return bail("server layout");
  for (int i = 0; i < count; ++i)
    std::memcpy(sl.h_x0 + x0_off[i], sl.reqs[i].x0.data(), sizeof(float) * (x0_off[i + 1] - x0_off[i]));
  cudaError_t e = cudaMemcpyAsync(sl.d_x0, sl.h_x0, sizeof(float) * x0_off[count], cudaMemcpyHostToDevice, sl.s);
  if (e != cudaSuccess) {
    S->set_error(std::string("server upload: ") + cudaGetErrorString(e));
    return false;
  }
  if ((st = mtp_batch_plan_step(sl.b, sl.d_x0, S->cfg.iters_per_request, sl.d_us, sl.s)) != MTP_OK)
    return bail("server plan");
  if (S->cfg.shift_after > 0 && (st = mtp_batch_shift(sl.b, S->cfg.shift_after, sl.s)) != MTP_OK)
    return bail("server shift");
  if ((e = cudaMemcpyAsync(sl.h_us, sl.d_us, sizeof(float) * sl.us_off[count], cudaMemcpyDeviceToHost, sl.s)) ||
      (e = cudaEventRecord(sl.done, sl.s))) {
    S->set_error(std::string("server download: ") + cudaGetErrorString(e));
    return false;
  }
  sl.busy = true;
  sl.seq = ++S->seq;
  S->cycles.fetch_add(1);
  S->planned.fetch_add((uint64_t)count);
  return true;
}

Slot* oldest_busy(mtp_server* S) {
  Slot* o = nullptr;
  for (Slot& sl : S->slots)
    if (sl.busy && (!o || sl.seq < o->seq)) o = &sl;
  return o;
}

void worker_main(mtp_server* S) {
  cudaSetDevice(S->device);
  bool ok = true;
  while (ok && !S->stop.load()) {
    Slot* busy = oldest_busy(S);
    std::vector<mtp_sched::Request> reqs = S->sched.next_cycle(busy ? kBusyWait : kIdleWait);
    if (reqs.empty()) {
      // no new work: collect the oldest cycle once it is done
      if (busy) {
        const cudaError_t q = cudaEventQuery(busy->done);
        if (q == cudaSuccess) ok = finish(S, *busy);
        else if (q != cudaErrorNotReady) ok = finish(S, *busy);  // reports the error
      }
      continue;
    }
    Slot* free_sl = nullptr;
    for (Slot& sl : S->slots)
      if (!sl.busy) free_sl = &sl;
    if (!free_sl) {
      free_sl = oldest_busy(S);
      ok = finish(S, *free_sl);
      if (!ok) break;
    }
    ok = launch(S, *free_sl, std::move(reqs));
  }
  for (Slot& sl : S->slots)  // cycles in flight end normally
    if (sl.busy) ok = finish(S, sl) && ok;
  if (!ok) S->failed.store(1);
}

mtp_status server_fail(mtp_server* S, mtp_status st, const std::string& msg) {
  if (S) S->set_error(msg);
  return st;
}

// One ticket: at most n_max values of its u* go to `out`.
mtp_status poll_one(mtp_server* S, uint64_t ticket, float* out, int n_max, double wait_s) {
  switch (S->sched.poll(ticket, out, n_max, wait_s)) {
    case mtp_sched::kReady:
      return MTP_OK;
    case mtp_sched::kUnknown:
      return server_fail(S, MTP_ERR_INVALID_ARG, "poll: unknown or already collected ticket");
    default:
      if (S->failed.load()) return server_fail(S, MTP_ERR_CUDA, "poll: the server failed");
      return wait_s == 0.0 ? MTP_ERR_NOT_READY : MTP_ERR_TIMEOUT;
  }
}

}  // namespace

extern "C" {

mtp_status mtp_server_create(const mtp_server_config* cfg, mtp_server** out) {
  if (!cfg || !out) return MTP_ERR_INVALID_ARG;
  *out = nullptr;
  if (cfg->max_batch < 1 || cfg->iters_per_request < 1 || cfg->shift_after < 0 || cfg->max_queue < 1 ||
      cfg->max_robots < 1) {
    mtp::set_thread_error("server_create: max_batch, iters_per_request, max_queue and max_robots must be >= 1, "
                          "shift_after >= 0");
    return MTP_ERR_INVALID_ARG;
  }
  mtp_server* S = new mtp_server(*cfg);
  cudaGetDevice(&S->device);
  S->robots.reserve(cfg->max_robots);
  mtp_status st = MTP_OK;
  for (Slot& sl : S->slots) {
    if ((st = mtp_batch_reserve(cfg->max_batch, &sl.b)) != MTP_OK) break;
    cudaError_t e = alloc_slot(sl, cfg->max_batch);
    if (e != cudaSuccess) {
      st = e == cudaErrorMemoryAllocation ? MTP_ERR_OUT_OF_MEMORY : MTP_ERR_CUDA;
      break;
    }
  }
  if (st == MTP_OK) {
    S->budget = cfg->memory_budget;
    if (S->budget == 0) {
      size_t free_b = 0, total_b = 0;
      if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) st = MTP_ERR_CUDA;
      S->budget = (uint64_t)(0.9 * (double)free_b);
    }
  }
  if (st != MTP_OK) {
    if (st != MTP_ERR_INVALID_ARG) mtp::set_thread_error("server_create: could not allocate the cycle slots");
    for (Slot& sl : S->slots) free_slot(sl);
    delete S;
    return st;
  }
  S->worker = std::thread(worker_main, S);
  *out = S;
  return MTP_OK;
}

mtp_status mtp_server_destroy(mtp_server* S) {
  if (!S) return MTP_ERR_INVALID_ARG;
  S->stop.store(true);
  S->sched.close();
  if (S->worker.joinable()) S->worker.join();
  DeviceScope g(S->device);
  for (Slot& sl : S->slots) free_slot(sl);
  for (mtp_handle* h : S->robots) mtp_destroy(h);
  delete S;
  return MTP_OK;
}

mtp_status mtp_server_register(mtp_server* S, const mtp_problem* problem, int32_t* robot) {
  if (!S || !problem || !robot) return server_fail(S, MTP_ERR_INVALID_ARG, "register: null argument");
  // served robots are planned in batches only: no single-instance pipeline
  // (and so no second candidate buffer in the footprint)
  mtp_problem pr = *problem;
  pr.flags |= MTP_FLAG_NO_PIPELINE;
  uint64_t bytes = 0;
  mtp_status st = mtp_problem_device_bytes(&pr, &bytes);
  if (st != MTP_OK) return server_fail(S, st, std::string("register: ") + mtp_last_error(nullptr));
  // admission is decided and reserved under the lock; the handle (device
  // allocations, synchronous copies) is created outside it, so cycles that
  // start meanwhile are not held up
  {
    std::lock_guard<std::mutex> lock(S->reg_mu);
    if ((int)S->robots.size() + S->registering >= S->cfg.max_robots)
      return server_fail(S, MTP_ERR_ADMISSION, "register: max_robots reached");
    if (S->bytes_admitted + bytes > S->budget)
      return server_fail(S, MTP_ERR_ADMISSION,
                         "register: " + std::to_string(bytes) + " bytes do not fit the remaining budget of " +
                             std::to_string(S->budget - S->bytes_admitted));
    S->bytes_admitted += bytes;
    ++S->registering;
  }
  mtp_handle* h = nullptr;
  {
    DeviceScope g(S->device);
    st = mtp_create(&pr, &h);
  }
  std::lock_guard<std::mutex> lock(S->reg_mu);
  --S->registering;
  if (st != MTP_OK) {
    S->bytes_admitted -= bytes;  // the reservation is returned
    return server_fail(S, st, std::string("register: ") + mtp_last_error(nullptr));
  }
  *robot = (int32_t)S->robots.size();
  S->robots.push_back(h);
  S->robot_d.push_back(problem->state_dim);
  S->robot_n.push_back(problem->ctrl_dim);
  return MTP_OK;
}

mtp_status mtp_submit(mtp_server* S, int32_t robot, const float* h_x0, uint64_t* ticket) {
  if (!S || !h_x0 || !ticket) return server_fail(S, MTP_ERR_INVALID_ARG, "submit: null argument");
  if (S->failed.load()) return server_fail(S, MTP_ERR_CUDA, "submit: the server failed");
  int d = 0;
  {
    std::lock_guard<std::mutex> lock(S->reg_mu);
    if (robot < 0 || robot >= (int32_t)S->robots.size())
      return server_fail(S, MTP_ERR_INVALID_ARG, "submit: unknown robot");
    d = S->robot_d[robot];
  }
  const uint64_t t = S->sched.submit(robot, h_x0, d, mtp_sched::now_seconds());
  if (t == 0) return server_fail(S, MTP_ERR_ADMISSION, "submit: the robot's queue is full");
  *ticket = t;
  return MTP_OK;
}

mtp_status mtp_poll(mtp_server* S, uint64_t ticket, float* h_ustar, double timeout_s) {
  if (!S || !h_ustar || !(timeout_s >= 0.0)) return server_fail(S, MTP_ERR_INVALID_ARG, "poll: bad argument");
  return poll_one(S, ticket, h_ustar, MTP_MAX_CTRL, timeout_s);
}

mtp_status mtp_submit_many(mtp_server* S, int32_t count, const int32_t* robots, const float* h_x0,
                           uint64_t* tickets, int32_t* accepted) {
  if (accepted) *accepted = 0;
  if (!S || count < 0 || (count > 0 && (!robots || !h_x0 || !tickets)))
    return server_fail(S, MTP_ERR_INVALID_ARG, "submit_many: bad argument");
  size_t off = 0;
  for (int32_t i = 0; i < count; ++i) {
    int d = 0;
    {
      std::lock_guard<std::mutex> lock(S->reg_mu);
      if (robots[i] < 0 || robots[i] >= (int32_t)S->robots.size())
        return server_fail(S, MTP_ERR_INVALID_ARG, "submit_many: unknown robot");
      d = S->robot_d[robots[i]];
    }
    const mtp_status st = mtp_submit(S, robots[i], h_x0 + off, tickets + i);
    if (st != MTP_OK) return st;
    off += (size_t)d;
    if (accepted) *accepted = i + 1;
  }
  return MTP_OK;
}

mtp_status mtp_poll_many(mtp_server* S, int32_t count, const uint64_t* tickets, float* h_ustar,
                         int32_t stride, double timeout_s, int32_t* status, int32_t* ready) {
  if (ready) *ready = 0;
  if (!S || count < 0 || stride < 1 || !(timeout_s >= 0.0) ||
      (count > 0 && (!tickets || !h_ustar || !status)))
    return server_fail(S, MTP_ERR_INVALID_ARG, "poll_many: bad argument");
  const double deadline = mtp_sched::now_seconds() + timeout_s;
  int32_t n_ok = 0;
  for (int32_t i = 0; i < count; ++i) {
    const double left = timeout_s > 0.0 ? std::max(0.0, deadline - mtp_sched::now_seconds()) : 0.0;
    mtp_status st = poll_one(S, tickets[i], h_ustar + (size_t)i * stride, stride, left);
    if (st == MTP_ERR_NOT_READY && timeout_s > 0.0) st = MTP_ERR_TIMEOUT;  // the shared deadline passed
    status[i] = st;
    if (st == MTP_OK) ++n_ok;
  }
  if (ready) *ready = n_ok;
  return MTP_OK;
}

mtp_status mtp_server_get_stats(mtp_server* S, mtp_server_stats* out) {
  if (!S || !out) return MTP_ERR_INVALID_ARG;
  const auto c = S->sched.counters();
  std::memset(out, 0, sizeof(*out));
  out->submitted = c.submitted;
  out->completed = c.completed;
  out->queued = c.queued;
  out->in_flight = c.in_flight;
  out->cycles = S->cycles.load();
  out->planned = S->planned.load();
  out->failed = S->failed.load();
  {
    std::lock_guard<std::mutex> lock(S->reg_mu);
    out->robots = (int32_t)S->robots.size();
    out->bytes_admitted = S->bytes_admitted;
  }
  out->p50_latency_s = S->sched.latency_percentile(50.0);
  out->p99_latency_s = S->sched.latency_percentile(99.0);
  return MTP_OK;
}

const char* mtp_server_last_error(const mtp_server* S) {
  if (!S) return "null server";
  std::lock_guard<std::mutex> lock(S->err_mu);
  thread_local std::string copy;
  copy = S->err;
  return copy.c_str();
}

}  // extern "C"
