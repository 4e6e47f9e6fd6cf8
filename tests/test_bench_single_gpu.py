"""bench.py has no multi-GPU form: it refuses --gpus > 1 and a torchrun world before it
touches CUDA (the sigma kernels share tiles inside clusters by TMA multicast, which this
library only issues in single-GPU processes)."""
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(args, env_extra):
    env = dict(os.environ, **env_extra)
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], env=env,
                          capture_output=True, text=True, timeout=120)


def test_bench_refuses_more_than_one_gpu():
    r = _run(["--gpus", "2"], {})
    assert r.returncode != 0
    assert "one GPU only" in r.stderr
    assert "Traceback" not in r.stderr


def test_bench_refuses_a_torchrun_world():
    r = _run([], {"WORLD_SIZE": "2", "RANK": "0", "LOCAL_RANK": "0"})
    assert r.returncode != 0
    assert "one GPU only" in r.stderr
