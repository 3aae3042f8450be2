"""bench.py's reference arm (the FP64 oracle timed on the host cores) prints
one JSON line with the contract's keys; it needs no GPU."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "2",
                        "--warmup", "1"], capture_output=True, text=True, cwd=ROOT, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "impl", "cpu_baseline", "e2e"):
        assert k in line, k
    assert line["impl"] == "reference" and line["value"] > 0 and line["steps"] == 2
    assert line["unit"] == "atom-steps/s" and line["higher_is_better"] is True
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["value"] == line["value"]
    assert line["cpu_baseline"]["cores"] == len(os.sched_getaffinity(0))      # one oracle process per core
    assert line["e2e"] == {"value": line["value"], "unit": line["unit"], "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}


def test_clock_sampler_summary(tmp_path):
    """The clocks object of the bench line from nvidia-smi CSV samples: the
    median SM clock of the loaded three quarters of the samples, the maximum,
    and every throttle reason seen Active at least once."""
    import importlib.util
    spec = importlib.util.spec_from_file_location("_bench", os.path.join(ROOT, "bench.py"))
    bench = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(bench)

    class Done:
        def terminate(self):
            pass

        def wait(self):
            return 0

    rows = ["0, 600, 2070, 120.5, 0x0, Not Active, Not Active, Not Active, Not Active"]
    rows += [f"0, {1900 + 10 * k}, 2070, 900.0, 0x4, Not Active, Not Active, Not Active, Active" for k in range(7)]
    rows += ["0, [N/A], 2070, [N/A], 0x0, Not Active, Not Active, Not Active, Not Active", "garbled"]
    path = tmp_path / "clocks.csv"
    path.write_text("\n".join(rows) + "\n")
    cs = bench.ClockSampler(0)
    cs.proc, cs.path = Done(), str(path)
    out = cs.stop()
    assert out["samples"] == 9 and out["sm_max_mhz"] == 2070.0 and out["power_w_max"] == 900.0
    assert out["sm_mhz"] == 1935.0     # the lowest quarter (600 and 1900 MHz) dropped, median of 1910..1960
    assert out["reasons"] == ["sw_power_cap"]
    assert not path.exists()

    rows = ["0, 1500, 2070, 1000, 0x8, Active, Not Active, Active, Not Active"] * 4
    path.write_text("\n".join(rows) + "\n")
    cs.proc, cs.path = Done(), str(path)
    assert cs.stop()["reasons"] == ["hw_slowdown", "sw_thermal_slowdown"]

    cs.proc = None
    assert cs.stop()["reasons"] == ["nvidia-smi unavailable"]
