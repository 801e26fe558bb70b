// scheduler.h -- host-side request scheduling of the re-plan server
// (continuous batching).  Plain C++17, no CUDA: the server drives it from its
// worker thread, and the CPU tests drive it directly.
//
// Every robot has a FIFO of requests.  A cycle takes up to `max_batch`
// robots that have a queued request and no request in flight (a robot's
// next plan starts from the planner state its previous one left), oldest
// request first.  Completed results wait for poll; latency is submit ->
// completion.  Memory stays bounded by the outstanding requests: a ticket is
// forgotten once its result has been polled.
#pragma once

#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstdint>
#include <deque>
#include <map>
#include <mutex>
#include <set>
#include <unordered_map>
#include <unordered_set>
#include <vector>

namespace mtp_sched {

struct Request {
  uint64_t ticket = 0;
  int robot = -1;
  std::vector<float> x0;
  double t_submit = 0.0;
};

enum PollStatus { kReady = 0, kPending = 1, kUnknown = 2 };

inline double now_seconds() {
  using namespace std::chrono;
  return duration<double>(steady_clock::now().time_since_epoch()).count();
}

class Scheduler {
 public:
  static constexpr size_t kLatencyWindow = 1 << 16;  // percentiles over the latest completions

  explicit Scheduler(int max_batch, int max_queue = 1 << 30)
      : max_batch_(max_batch < 1 ? 1 : max_batch), max_queue_(max_queue < 1 ? 1 : max_queue) {}

  // Queues a request; returns its ticket, or 0 when the robot already has
  // max_queue requests queued.
  uint64_t submit(int robot, const float* x0, int d, double now) {
    std::lock_guard<std::mutex> lock(mu_);
    auto& q = queues_[robot];
    if ((int)q.size() >= max_queue_) return 0;
    Request r;
    r.ticket = ++last_ticket_;
    r.robot = robot;
    r.x0.assign(x0, x0 + d);
    r.t_submit = now;
    q.push_back(std::move(r));
    outstanding_.insert(last_ticket_);
    ++queued_;
    ++submitted_;
    if (!in_flight_.count(robot) && q.size() == 1) ready_.insert({now, robot});
    cv_.notify_all();
    return last_ticket_;
  }

  // Up to max_batch requests of idle robots, oldest first; their robots are
  // marked in flight.  Waits up to `wait_s` for work when there is none.
  std::vector<Request> next_cycle(double wait_s) {
    std::unique_lock<std::mutex> lock(mu_);
    if (ready_.empty() && wait_s > 0 && !closing_)
      cv_.wait_for(lock, std::chrono::duration<double>(wait_s), [&] { return !ready_.empty() || closing_; });
    std::vector<Request> out;
    while (!ready_.empty() && (int)out.size() < max_batch_) {
      const int robot = ready_.begin()->second;
      ready_.erase(ready_.begin());
      auto& q = queues_[robot];
      out.push_back(std::move(q.front()));
      q.pop_front();
      in_flight_.insert(robot);
      --queued_;
    }
    return out;
  }

  // Records the result of an in-flight request and frees its robot.
  void complete(const Request& r, const float* ustar, int n, double now) {
    std::lock_guard<std::mutex> lock(mu_);
    done_[r.ticket].assign(ustar, ustar + n);
    const double lat = now - r.t_submit;
    if (latencies_.size() < kLatencyWindow) latencies_.push_back(lat);
    else latencies_[lat_next_] = lat;
    lat_next_ = (lat_next_ + 1) % kLatencyWindow;
    in_flight_.erase(r.robot);
    auto& q = queues_[r.robot];
    if (!q.empty()) ready_.insert({q.front().t_submit, r.robot});
    ++completed_;
    cv_.notify_all();
  }

  // kReady: the result (at most `n` values) is copied to `out` and the
  // ticket forgotten.  kPending after waiting up to `wait_s` seconds.
  // kUnknown: never issued, or already collected.
  PollStatus poll(uint64_t ticket, float* out, int n, double wait_s) {
    std::unique_lock<std::mutex> lock(mu_);
    if (!outstanding_.count(ticket)) return kUnknown;
    auto ready = [&] { return done_.count(ticket) > 0; };
    if (!ready() && wait_s > 0) cv_.wait_for(lock, std::chrono::duration<double>(wait_s), ready);
    auto it = done_.find(ticket);
    if (it == done_.end()) return kPending;
    std::copy(it->second.begin(), it->second.begin() + std::min<size_t>((size_t)n, it->second.size()), out);
    done_.erase(it);
    outstanding_.erase(ticket);
    return kReady;
  }

  // Wakes every waiter; next_cycle stops waiting for work.
  void close() {
    std::lock_guard<std::mutex> lock(mu_);
    closing_ = true;
    cv_.notify_all();
  }

  // latency percentile p (0..100) over the latest completions, seconds
  // (nearest rank)
  double latency_percentile(double p) const {
    std::lock_guard<std::mutex> lock(mu_);
    if (latencies_.empty()) return 0.0;
    std::vector<double> v(latencies_);
    std::sort(v.begin(), v.end());
    double rank = p / 100.0 * (double)v.size();
    size_t k = rank <= 1.0 ? 0 : (size_t)std::ceil(rank - 1e-9) - 1;
    return v[std::min(k, v.size() - 1)];
  }

  struct Counters {
    uint64_t submitted, completed;
    int queued, in_flight;
  };
  Counters counters() const {
    std::lock_guard<std::mutex> lock(mu_);
    return Counters{submitted_, completed_, queued_, (int)in_flight_.size()};
  }

 private:
  mutable std::mutex mu_;
  std::condition_variable cv_;
  int max_batch_, max_queue_;
  uint64_t last_ticket_ = 0, submitted_ = 0, completed_ = 0;
  int queued_ = 0;
  bool closing_ = false;
  std::map<int, std::deque<Request>> queues_;
  std::set<std::pair<double, int>> ready_;  // (oldest queued submit time, robot) of idle robots
  std::unordered_set<int> in_flight_;
  std::unordered_map<uint64_t, std::vector<float>> done_;
  std::unordered_set<uint64_t> outstanding_;  // issued and not yet collected
  std::vector<double> latencies_;
  size_t lat_next_ = 0;
};

}  // namespace mtp_sched
