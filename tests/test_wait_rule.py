"""The kernels' bounded-wait rule on the host (no GPU).

The persistent tensor-core kernel bounds every wait on a pipeline barrier: a
wait gives up (and the call then reports FE_ERR_TIMEOUT) only when its phase
has made no progress for the plan's limit, counted from the start of that
wait.  tests/wait_rule_model.cpp replays the device loop with the library's
own decision rule (csrc/fe_wait.h) on a modelled clock: a launch lasting tens
of thousands of limits whose waits each complete within the limit never gives
up, a wait that never completes gives up within three limits, and a phase
that completes later than that is given up on.
"""
import os
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def model(tmp_path_factory):
    exe = str(tmp_path_factory.mktemp("wait") / "wait_rule_model")
    subprocess.check_call(["g++", "-O1", "-std=c++17", "-o", exe, os.path.join(ROOT, "tests", "wait_rule_model.cpp")])
    return exe


def _run(exe, scenario, limit):
    out = subprocess.check_output([exe, scenario, str(limit)], text=True)
    kv = dict(line.split() for line in out.strip().splitlines())
    return int(kv["gave_up"]), int(kv["elapsed"])


@pytest.mark.parametrize("limit", [1000, 100000, 2000000000])
def test_long_launch_never_gives_up(model, limit):
    gave_up, elapsed = _run(model, "long", limit)
    assert gave_up == 0
    assert elapsed > 1000 * limit or limit == 2000000000 and elapsed > 40000 * limit


@pytest.mark.parametrize("limit", [1000, 100000, 2000000000])
def test_stalled_wait_gives_up_within_three_limits(model, limit):
    gave_up, elapsed = _run(model, "stall", limit)
    assert gave_up == 1
    assert limit < elapsed <= 3 * limit


@pytest.mark.parametrize("limit", [1000, 2000000000])
def test_late_phase_is_given_up_on(model, limit):
    gave_up, _ = _run(model, "late", limit)
    assert gave_up == 1
