"""Host-side logic of the benchmark, without a GPU: the reference arm (the
oracle timed on the host cores) prints the contract's JSON line, also when
fewer steps are asked for than its phase cycle has phases, and only on rank
0; the clock record summarises nvidia-smi samples (median SM clock, throttle
reasons)."""

import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.parametrize("steps,warmup", [(1, 1), (2, 3)])
def test_reference_arm_prints_one_contract_line(steps, warmup):
    env = dict(os.environ, CUDA_VISIBLE_DEVICES="")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--grid", "8",
                        "--nrhs", "2", "--steps", str(steps), "--warmup", str(warmup)],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0 and line["steps"] == steps
    assert line["warmup"] == warmup and line["higher_is_better"] is True and line["dtype"] == "f64"
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == line["value"] and cb["cores"] == 2
    assert line["e2e"] == {"value": line["value"], "unit": line["unit"], "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}


def test_reference_arm_other_ranks_exit_without_work():
    env = dict(os.environ, CUDA_VISIBLE_DEVICES="", RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--grid", "8",
                        "--nrhs", "2", "--steps", "1", "--warmup", "1"],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0 and r.stdout.strip() == "", (r.stdout[-500:], r.stderr[-500:])


def test_clock_summary_of_nvidia_smi_lines():
    sys.path.insert(0, ROOT)
    import bench

    lines = [
        "0, 2070, 2070, 900.12, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active\n",
        "0, 1965, 2070, 1390.50, 0x0000000000000004, Not Active, Not Active, Not Active, Active\n",
        "0, 2070, 2070, 1200.00, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active\n",
        "0, [N/A], 2070, [N/A], [N/A], [N/A], [N/A], [N/A], [N/A]\n",  # a sample the tool could not read
        "garbled\n",
    ]
    c = bench.ClockSampler.summarise(lines)
    assert c == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 4}
    hot = lines[:1] + ["0, 1500, 2070, 1000, 0x48, Not Active, Active, Not Active, Not Active\n"]
    assert bench.ClockSampler.summarise(hot)["reasons"] == ["hw_thermal_slowdown"]
    assert bench.ClockSampler.summarise(["garbled\n"]) is None


def test_clock_sampler_stop_reads_and_removes_its_file(tmp_path):
    sys.path.insert(0, ROOT)
    import bench

    class _Done:  # a sampler process that has already exited
        def terminate(self):
            pass

        def wait(self, timeout=None):
            return 0

    path = tmp_path / "clocks.csv"
    path.write_text("0, 2070, 2070, 900, 0x0, Not Active, Not Active, Not Active, Not Active\n")
    s = bench.ClockSampler(0)
    s.proc, s.path = _Done(), str(path)
    assert s.stop() == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": [], "samples": 1}
    assert not path.exists()
    assert bench.ClockSampler(0).stop() is None  # never started


def test_recorded_traffic_holds_only_while_the_source_is_unchanged(tmp_path, monkeypatch):
    sys.path.insert(0, ROOT)
    import hashlib

    import bench

    src = tmp_path / "k.cu"
    src.write_text("__global__ void k() {}\n")
    h = hashlib.sha256(src.read_bytes()).hexdigest()[:16]
    (tmp_path / "profiles").mkdir()
    (tmp_path / "profiles" / "dram_traffic.md").write_text(
        "| kernel | workload | source | sha256[:16] | DRAM bytes per launch |\n|---|---|---|---|---:|\n"
        f"| k | w1 | k.cu | {h} | 1234 |\n| k | w2 | k.cu | 0000000000000000 | 99 |\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.recorded_traffic("k", "w1") == 1234.0
    assert bench.recorded_traffic("k", "w2") is None  # recorded for another version of the source
    assert bench.recorded_traffic("k", "w3") is None  # never captured
    src.write_text("__global__ void k() { }\n")  # the kernel changed since the capture
    assert bench.recorded_traffic("k", "w1") is None
