"""CPU checks of bench.py's reporting: the reference arm's JSON line (the FP64 oracle on
the host, no GPU), silence on ranks other than 0, the clock record's throttle reasons,
and the algorithmic bytes behind the roofline figures."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def run_bench(args, env_extra=None):
    env = dict(os.environ)
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        env.pop(k, None)
    env.update(env_extra or {})
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], capture_output=True, text=True,
                          env=env, cwd=ROOT, timeout=600)


def test_reference_arm_json_line():
    r = run_bench(["--impl", "reference", "--steps", "1", "--warmup", "0"])
    assert r.returncode == 0, r.stderr
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == bench.UNIT
    assert d["value"] > 0 and d["higher_is_better"] is True and d["steps"] == 1
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] == bench.CPU_SAMPLE_SLICES
    assert d["cpu_baseline"]["value"] == d["value"] and d["cpu_baseline"]["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert "workload" in d["config"] and d["vs_baseline"] is None


def test_reference_arm_other_ranks_print_nothing():
    r = run_bench(["--impl", "reference", "--steps", "1", "--warmup", "0"], {"RANK": "1", "WORLD_SIZE": "2"})
    assert r.returncode == 0 and r.stdout.strip() == ""


def test_clock_record_reasons():
    c = bench.Clocks(0)
    idle = "0, 1005, 2070, 160.0, 0x0, Not Active, Not Active, Not Active, Not Active"
    load = ["0, 2070, 2070, 990.0, 0x0, Not Active, Not Active, Not Active, Not Active",
            "0, 2055, 2070, 1010.0, 0x4, Not Active, Not Active, Not Active, Active",
            "0, 1900, 2070, 1000.0, 0x8, Active, Not Active, Not Active, Not Active"]
    c.out = "\n".join([idle] + load)
    s = c.summary()
    assert s["samples"] == 3 and s["sm_mhz"] == 2055 and s["sm_max_mhz"] == 2070
    assert s["reasons"] == ["hw_slowdown", "sw_power_cap"]
    c.out = ""
    assert c.summary()["reasons"] == ["nvidia-smi unavailable"]


def test_algorithmic_bytes_of_the_knee_scan():
    """Bytes per launch on the knee scan (S=320, C=12, M=1, K=4, N=256x160), as the kernel
    table states them: row passes 6.71 GB, column pass 10.07 GB, LLR + FISTA 2.52 GB."""
    ab = bench.algorithmic_bytes(320, 12, 1, 4, 256 * 160)
    assert ab["row_fwd"] == ab["row_adj"] == pytest.approx(6.71e9, rel=2e-3)
    assert ab["col"] == pytest.approx(10.07e9, rel=2e-3)
    assert ab["llr"] == pytest.approx(2.52e9, rel=2e-3)


def test_cpu_sample_is_seeded_distinct_and_stable():
    """The oracle's timing sample: 8 distinct slices of the scan, the same every run."""
    import t2sh_synth as synth
    a = bench.sample_slices(synth.KNEE_320x256x160)
    b = bench.sample_slices(synth.KNEE_320x256x160)
    assert a == b and len(a) == bench.CPU_SAMPLE_SLICES == len(set(a))
    assert a == sorted(a) and 0 <= a[0] and a[-1] < 320
    assert bench.sample_slices(synth.PAPER_288x260x240) != a
    assert bench.shape_by_name(bench.shape_name(synth.PAPER_288x260x240)) is synth.PAPER_288x260x240


def test_batch3_config_names_the_three_scans():
    import t2sh_synth as synth
    c = bench.batch3_config(1)
    assert c["slices"] == sum(sh.nslices for sh in synth.BATCH_SCANS) == 864
    assert len(c["scans"]) == 3 and "256x160 C=12" in c["workload"] and "192x192 C=16" in c["workload"]


class _FakePlan:
    def __init__(self, i, log):
        self.i, self.log, self.closed = i, log, False

    def close(self):
        assert not self.closed
        self.closed = True
        self.log.append(("close", self.i))


def test_pipelined_steps_overlap_the_next_plan_with_the_solve():
    """The end-to-end leg's pipelining: plan i+1 is being made on another thread while solve
    i runs (the solve waits for it to start), every plan is solved once in order and closed
    after its solve, and the phase times add up."""
    import threading
    n = 4
    log, lock = [], threading.Lock()
    begun = [threading.Event() for _ in range(n)]
    threads = {}

    def make(i):
        begun[i].set()
        threads[i] = threading.current_thread().ident
        with lock:
            log.append(("make", i))
        return _FakePlan(i, log), 0.001 * (i + 1)

    def solve(p):
        if p.i + 1 < n:
            assert begun[p.i + 1].wait(timeout=10), "the next plan was not requested before this solve"
        with lock:
            log.append(("solve", p.i))

    t = bench.pipelined_steps(make, solve, n)
    assert [e[1] for e in log if e[0] == "solve"] == list(range(n))
    assert [e[1] for e in log if e[0] == "close"] == list(range(n))
    for i in range(n):
        assert log.index(("solve", i)) < log.index(("close", i))
    assert threading.current_thread().ident not in threads.values()
    assert abs(t["plan"] - 0.010) < 1e-12 and min(t.values()) >= 0
    assert bench.pipelined_steps(make, solve, 0) == {"plan": 0.0, "wait": 0.0, "solve": 0.0, "destroy": 0.0}


def test_pipelined_steps_close_a_plan_whose_solve_fails():
    log = []

    def make(i):
        return _FakePlan(i, log), 0.0

    def solve(p):
        if p.i == 1:
            raise RuntimeError("solve failed")

    with pytest.raises(RuntimeError):
        bench.pipelined_steps(make, solve, 3)
    assert ("close", 0) in log and ("close", 1) in log
