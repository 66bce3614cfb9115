"""The benchmark's N > 1 path on the CPU: world-size-2 ``gloo`` process groups.

The training step has no exchange step, so N GPUs run N independent replicas;
the only cross-rank work is in the timing (barrier on both sides of the timed
region, the slowest rank's time, units of all ranks over it, rank 0 prints).
These tests run that code (``bench.Replicas``) as two real processes with the
``gloo`` backend, each rank timing a host "step" of a different length.
"""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

WORKER = r"""
import json, os, sys, time
sys.path.insert(0, sys.argv[1])
import bench

reps = bench.Replicas("gloo")
time.sleep(float(os.environ.get("LATE_S", "0")))  # a rank that reaches the first barrier late
steps = 4
step_s = 0.05 * (1 + reps.rank)          # rank 1 is twice as slow as rank 0
t_enter = time.time()
reps.barrier()
t_start = time.time()
t0 = time.perf_counter()
for _ in range(steps):
    time.sleep(step_s)
own_ms = (time.perf_counter() - t0) * 1e3
ms = reps.slowest_ms(own_ms)
reps.barrier()
t_leave = time.time()
out = dict(rank=reps.rank, world=reps.world, printer=reps.printer, own_ms=own_ms, ms=ms,
           rate=reps.rate(steps, ms), t_enter=t_enter, t_start=t_start, t_leave=t_leave, steps=steps)
reps.close()
with open(os.path.join(sys.argv[2], "rank%d.json" % out["rank"]), "w") as f:
    json.dump(out, f)
if out["printer"]:
    print(json.dumps(dict(value=out["rate"], n_gpus=out["world"])))
"""


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _launch(world: int, tmp_path, delay_rank=None):
    port = _free_port()
    procs = []
    for r in range(world):
        env = dict(os.environ, RANK=str(r), LOCAL_RANK=str(r), WORLD_SIZE=str(world), LOCAL_WORLD_SIZE=str(world),
                   MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
        if delay_rank == r:
            env["LATE_S"] = "0.5"
        procs.append(subprocess.Popen([sys.executable, "-c", WORKER, ROOT, str(tmp_path)], env=env,
                                      stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        try:
            so, se = p.communicate(timeout=120)
        except subprocess.TimeoutExpired:
            for q in procs:
                q.kill()
            raise
        outs.append((p.returncode, so, se))
    for rc, so, se in outs:
        assert rc == 0, se[-2000:]
    recs = [json.load(open(tmp_path / f"rank{r}.json")) for r in range(world)]
    return recs, [so for _, so, _ in outs]


def test_two_replicas_slowest_rank_and_whole_job_rate(tmp_path):
    recs, stdout = _launch(2, tmp_path)
    own = [r["own_ms"] for r in recs]
    assert own[1] > own[0]  # rank 1 slept twice as long
    for r in recs:
        assert r["world"] == 2
        assert r["ms"] == pytest.approx(max(own), rel=1e-12)  # every rank sees the slowest time
        assert r["rate"] == pytest.approx(r["steps"] * 2 / (max(own) / 1e3), rel=1e-12)
    # whole-job rate: both ranks' steps over the slowest rank's time, below twice the fast rank's own rate
    assert recs[0]["rate"] < 2 * recs[0]["steps"] / (own[0] / 1e3)
    # rank 0 alone prints, and prints one line
    assert [r["printer"] for r in recs] == [True, False]
    assert stdout[1].strip() == ""
    lines = stdout[0].strip().splitlines()
    assert len(lines) == 1
    line = json.loads(lines[0])
    assert line["n_gpus"] == 2 and line["value"] == pytest.approx(recs[0]["rate"])


def test_barrier_holds_timed_region_until_all_ranks_arrive(tmp_path):
    recs, _ = _launch(2, tmp_path, delay_rank=1)
    # rank 0 starts timing only after the late rank reached the barrier
    assert recs[0]["t_start"] >= recs[1]["t_enter"] - 0.01
    assert recs[0]["t_start"] - recs[0]["t_enter"] > 0.3
    # and leaves the timed region only after the slow rank finished its steps
    assert recs[0]["t_leave"] >= recs[1]["t_start"] + recs[1]["own_ms"] / 1e3 - 0.01


def test_single_process_needs_no_process_group(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench

    for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    reps = bench.Replicas("gloo")
    assert reps.world == 1 and reps.printer and reps.dist is None
    reps.barrier()
    assert reps.slowest_ms(12.5) == 12.5
    assert reps.rate(10, 500.0) == pytest.approx(20.0)
    reps.close()


def test_reference_arm_other_ranks_exit_without_work():
    env = dict(os.environ, RANK="1", LOCAL_RANK="1", WORLD_SIZE="2", MASTER_ADDR="127.0.0.1", MASTER_PORT="1")
    p = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                        "--steps", "1", "--warmup", "3"], env=env, capture_output=True, text=True, timeout=120)
    assert p.returncode == 0, p.stderr[-2000:]
    assert p.stdout.strip() == ""
