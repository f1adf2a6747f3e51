"""The benchmark's reference arm (the oracle, timed on the host cores) keeps
the JSON-line contract: one line, on rank 0 only, with the same metric, unit
and direction as the GPU arm, a cpu_baseline and a zero-copy e2e entry.  Runs
on the CPU with the small 32x32 workload."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _lines(cmd):
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1")
    out = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    return [json.loads(l) for l in out.stdout.splitlines() if l.startswith("{")]


def _check(line):
    sys.path.insert(0, ROOT)
    import bench
    assert line["impl"] == "reference"
    assert line["metric"] == bench.METRIC and line["unit"] == "solves/s" and line["higher_is_better"] is True
    assert line["value"] > 0 and line["steps"] == 2 and line["warmup"] == 1
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == line["value"] and cb["sample"]
    e2e = line["e2e"]
    assert e2e["value"] == line["value"] and e2e["unit"] == line["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0
    assert line["config"]["name"] == "C1" and line["config"]["workload"].startswith("C1: 32x32 lattice")


def test_reference_arm_single_process():
    lines = _lines([sys.executable, "bench.py", "--impl", "reference", "--workload", "C1",
                    "--steps", "2", "--warmup", "1"])
    assert len(lines) == 1
    _check(lines[0])


def test_reference_arm_under_torchrun_prints_once():
    pytest.importorskip("torch")
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    lines = _lines([sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
                    "--master-addr", "127.0.0.1", "--master-port", str(port), "bench.py", "--impl", "reference",
                    "--workload", "C1", "--gpus", "2", "--steps", "2", "--warmup", "1"])
    assert len(lines) == 1
    _check(lines[0])
    assert lines[0]["n_gpus"] == 2


def test_sweep_forms_option_pins_each_level():
    """--sweep-forms 'form,param;...' pins level 0, 1, ... in order."""
    sys.path.insert(0, ROOT)
    import bench
    calls = []

    class FakeW:
        @staticmethod
        def amg_pin_sweep_form(amg, level, nrhs, prec, form, param):
            calls.append((amg, level, nrhs, prec, form, param))

    bench.pin_sweep_forms(FakeW, "h", "2,2080;2,2064;3,2", 64, 1)
    assert calls == [("h", 0, 64, 1, 2, 2080), ("h", 1, 64, 1, 2, 2064), ("h", 2, 64, 1, 3, 2)]
    calls.clear()
    bench.pin_sweep_forms(FakeW, "h", "", 64, 1)
    assert calls == []
