"""The benchmark's reference arm on the CPU: one JSON line with the keys of the
benchmark contract, timed on the FP64 oracle over bounded samples of the c3
workload (the headline), and sample windows that stay inside the workload
however many steps are asked for.  Also the paper-style NumPy FP32 baseline
the benchmark reports beside the oracle: it must compute the channeliser."""

import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(*args):
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", *args],
                         cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, out.stdout
    return json.loads(lines[0])


def test_reference_arm_line():
    d = _run("--steps", "3", "--warmup", "3")
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "impl", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference"
    assert d["steps"] == 3 and d["warmup"] == 3 and d["n_gpus"] == 1
    assert d["value"] > 0 and d["higher_is_better"] is True
    assert d["config"]["workload"].startswith("c3")
    # the GPU arm prints this same dict for its default run (64 streams, FFT path)
    sys.path.insert(0, ROOT)
    import bench
    assert d["config"] == bench.c3_config("fft", 4096, 16, 64, 64 << 20, 64 * 241)
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    e = d["e2e"]
    assert e["value"] == d["value"] and e["unit"] == d["unit"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0


def test_reference_arm_other_ranks_print_nothing():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "3",
                          "--warmup", "3"], cwd=ROOT, capture_output=True, text=True, timeout=600, env=env)
    assert out.returncode == 0
    assert not [l for l in out.stdout.splitlines() if l.startswith("{")]


def test_reference_arm_long_runs_wrap():
    # 100 samples of 16 spectra run past the 241 spectra of a stream
    d = _run("--steps", "100", "--warmup", "3")
    assert d["steps"] == 100 and d["value"] > 0


def test_numpy_paper_style_baseline_is_the_channeliser():
    """bench.numpy_pfb_f32 (the CPU comparison program) against the FP64
    oracle: FP32 accuracy on a ragged c3-like stream, every spectrum."""
    import numpy as np
    sys.path.insert(0, ROOT)
    import bench
    import oracle
    from paper_2408_16551_gb300 import synth
    P, T = 512, 16
    x = synth.small_stream(P, T, P * 80 + 13, seed=3, window=synth.WIN_BLACKMAN).generate()
    h = oracle.prototype(P, T, oracle.WIN_BLACKMAN)
    got = bench.numpy_pfb_f32(x, P, T, h.astype(np.float32))
    ref = oracle.pfb(oracle.dequant(x, oracle.IN_C64), P, T, h)
    assert got.shape == ref.shape and got.dtype == np.complex64
    assert oracle.rel_l2(got, ref) < 2e-6
