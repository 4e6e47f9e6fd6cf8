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


def test_roofline_traffic_follows_the_committed_capture():
    """The roofline `traffic` comes from the committed ncu summary while the sigma kernel's
    source is the one that summary was captured from, and is withheld otherwise."""
    import hashlib

    sys.path.insert(0, ROOT)
    import bench
    import synth

    text = open(bench.TRAFFIC_PROFILE).read()
    src = hashlib.sha256(open(bench.KERNEL_SOURCE, "rb").read()).hexdigest()
    per, note = bench.measured_traffic(synth.CONFIGS["c2"], "bf16")
    if src in text:
        assert per is not None and per > 0, note
        assert per > 1e9  # a full c2 launch moves GBs (T round trip between the stages)
    else:
        assert per is None and "changed" in note
