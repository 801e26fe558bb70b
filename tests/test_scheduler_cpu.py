"""CPU tests of the re-plan server's request scheduler.

The scheduler is plain C++ (no CUDA); tests/sched_harness.cpp drives it
directly: per-robot FIFO with one request in flight per robot, oldest
request first up to the batch limit, queue limit, poll states, latency
percentiles, and a multi-threaded closed loop where every result must be the
request's own.
"""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    exe = str(tmp_path_factory.mktemp("sched") / "sched_harness")
    subprocess.run([gxx, "-std=c++17", "-O1", "-Wall", "-Werror", "-pthread",
                    os.path.join(HERE, "sched_harness.cpp"), "-o", exe], check=True)
    return exe


def test_scheduler_cases(harness):
    r = subprocess.run([harness], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stdout + r.stderr
    for case in ("fifo_and_one_in_flight", "oldest_first_up_to_max_batch", "queue_limit",
                 "poll_states", "latency_percentiles", "threaded_closed_loop"):
        assert f"OK {case}" in r.stdout
    assert "ALL OK" in r.stdout
