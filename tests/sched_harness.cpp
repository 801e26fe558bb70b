// CPU checks of the re-plan server's request scheduler (scheduler.h), built
// and run by tests/test_scheduler_cpu.py.  Prints "OK <case>" per passing
// case; any failed check prints "FAIL ..." and exits 1.
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <mutex>
#include <set>
#include <thread>
#include <vector>

#include "../paper_2505_01059_gb300/csrc/scheduler.h"

using mtp_sched::Request;
using mtp_sched::Scheduler;

#define CHECK(c)                                                  \
  do {                                                            \
    if (!(c)) {                                                   \
      std::printf("FAIL %s:%d %s\n", __FILE__, __LINE__, #c);     \
      std::exit(1);                                               \
    }                                                             \
  } while (0)

static void fifo_and_one_in_flight() {
  Scheduler s(8);
  float x[2] = {1.f, 2.f};
  const uint64_t t1 = s.submit(0, x, 2, 1.0), t2 = s.submit(0, x, 2, 2.0), t3 = s.submit(1, x, 2, 3.0);
  CHECK(t1 == 1 && t2 == 2 && t3 == 3);
  auto c1 = s.next_cycle(0.0);
  CHECK(c1.size() == 2 && c1[0].ticket == t1 && c1[1].ticket == t3);  // t2: robot 0 is in flight
  CHECK(s.next_cycle(0.0).empty());
  float u = 7.f;
  s.complete(c1[0], &u, 1, 4.0);
  auto c2 = s.next_cycle(0.0);
  CHECK(c2.size() == 1 && c2[0].ticket == t2 && c2[0].x0.size() == 2 && c2[0].x0[1] == 2.f);
  auto k = s.counters();
  CHECK(k.submitted == 3 && k.completed == 1 && k.queued == 0 && k.in_flight == 2);
  std::printf("OK fifo_and_one_in_flight\n");
}

static void oldest_first_up_to_max_batch() {
  Scheduler s(3);
  float x = 0.f;
  const double times[5] = {5.0, 1.0, 3.0, 2.0, 4.0};
  for (int r = 0; r < 5; ++r) s.submit(r, &x, 1, times[r]);
  auto c = s.next_cycle(0.0);
  CHECK(c.size() == 3 && c[0].robot == 1 && c[1].robot == 3 && c[2].robot == 2);
  auto c2 = s.next_cycle(0.0);
  CHECK(c2.size() == 2 && c2[0].robot == 4 && c2[1].robot == 0);
  std::printf("OK oldest_first_up_to_max_batch\n");
}

static void queue_limit() {
  Scheduler s(4, 2);
  float x = 0.f;
  CHECK(s.submit(0, &x, 1, 0.0) != 0);
  CHECK(s.submit(0, &x, 1, 0.0) != 0);
  CHECK(s.submit(0, &x, 1, 0.0) == 0);  // refused
  CHECK(s.submit(1, &x, 1, 0.0) != 0);  // other robots are unaffected
  auto c = s.next_cycle(0.0);           // one of robot 0's requests leaves the queue
  CHECK(c.size() == 2);
  CHECK(s.submit(0, &x, 1, 0.0) != 0);
  std::printf("OK queue_limit\n");
}

static void poll_states() {
  Scheduler s(4);
  float x = 0.f, out[3] = {0, 0, 0};
  CHECK(s.poll(1, out, 3, 0.0) == mtp_sched::kUnknown);  // never issued
  const uint64_t t = s.submit(2, &x, 1, 0.0);
  CHECK(s.poll(t, out, 3, 0.0) == mtp_sched::kPending);
  CHECK(s.poll(t, out, 3, 0.01) == mtp_sched::kPending);  // bounded wait ran out
  auto c = s.next_cycle(0.0);
  const float u[3] = {1.f, -2.f, 3.5f};
  s.complete(c[0], u, 3, 1.0);
  CHECK(s.poll(t, out, 3, 0.0) == mtp_sched::kReady);
  CHECK(out[0] == 1.f && out[1] == -2.f && out[2] == 3.5f);
  CHECK(s.poll(t, out, 3, 0.0) == mtp_sched::kUnknown);  // already collected
  std::printf("OK poll_states\n");
}

static void latency_percentiles() {
  Scheduler s(1000);
  float x = 0.f;
  for (int i = 0; i < 100; ++i) s.submit(i, &x, 1, 0.0);
  auto c = s.next_cycle(0.0);
  CHECK(c.size() == 100);
  for (int i = 0; i < 100; ++i) s.complete(c[i], &x, 1, (double)(i + 1));  // latencies 1..100
  CHECK(s.latency_percentile(50.0) == 50.0);
  CHECK(s.latency_percentile(99.0) == 99.0);
  CHECK(s.latency_percentile(100.0) == 100.0);
  CHECK(s.latency_percentile(0.0) == 1.0);
  std::printf("OK latency_percentiles\n");
}

// Closed-loop clients on several threads against a worker thread that runs
// cycles; each result must be its own request's (x0 doubled), and no robot
// may ever be in two cycles at once.
static void threaded_closed_loop() {
  const int robots = 16, per_robot = 200, clients = 4;
  Scheduler s(5);
  std::atomic<bool> stop{false};
  std::atomic<int> violations{0}, cycles{0};
  std::thread worker([&] {
    std::set<int> busy;
    while (!stop.load()) {
      auto c = s.next_cycle(0.002);
      if (c.empty()) continue;
      ++cycles;
      for (auto& r : c)
        if (!busy.insert(r.robot).second) ++violations;
      CHECK((int)c.size() <= 5);
      std::this_thread::sleep_for(std::chrono::microseconds(100));
      for (auto& r : c) {
        float u = 2.f * r.x0[0];
        busy.erase(r.robot);
        s.complete(r, &u, 1, mtp_sched::now_seconds());
      }
    }
  });
  std::atomic<int> wrong{0};
  std::vector<std::thread> cl;
  for (int c = 0; c < clients; ++c)
    cl.emplace_back([&, c] {
      for (int k = 0; k < per_robot; ++k)
        for (int r = c; r < robots; r += clients) {
          float x = (float)(r * 1000 + k), out = -1.f;
          const uint64_t t = s.submit(r, &x, 1, mtp_sched::now_seconds());
          if (t == 0) {
            ++wrong;
            continue;
          }
          int tries = 0;
          while (s.poll(t, &out, 1, 0.05) != mtp_sched::kReady && ++tries < 200) {
          }
          if (out != 2.f * x) ++wrong;
        }
    });
  for (auto& t : cl) t.join();
  stop.store(true);
  s.close();
  worker.join();
  auto k = s.counters();
  CHECK(wrong.load() == 0 && violations.load() == 0);
  CHECK(k.submitted == (uint64_t)robots * per_robot && k.completed == k.submitted);
  CHECK(k.queued == 0 && k.in_flight == 0);
  CHECK(cycles.load() < robots * per_robot);  // requests were batched
  std::printf("OK threaded_closed_loop cycles=%d\n", cycles.load());
}

int main() {
  fifo_and_one_in_flight();
  oldest_first_up_to_max_batch();
  queue_limit();
  poll_states();
  latency_percentiles();
  threaded_closed_loop();
  std::printf("ALL OK\n");
  return 0;
}
