"""pfb_execute_host_noalloc: the host-buffer entry point that allocates no
device memory.

It is meant for callers that must not allocate device memory (a process whose
device memory belongs to another allocator, or a latency-critical thread that
cannot take the synchronisation cudaMalloc/cudaFree may imply).  It stages
through a fixed static device area instead of plan-owned cudaMalloc buffers.
Its results are checked against the existing pfb_execute_host, through the
C ABI, on two calls in a row (the second call must not see the first call's
leftovers in the shared area).  Both run the same kernel on the same input,
so the results must be equal bit for bit.  On a fresh plan, a no-alloc call
made before any pfb_execute_host must leave the device's free memory
unchanged, and an input too large for the area must be rejected before
anything runs.

This file is named so that pytest collects it last.
"""

import numpy as np
import pytest

import paper_2408_16551_gb300 as pkg
from paper_2408_16551_gb300 import synth

from gpu_common import TOL_F32, TOL_MAX_F32, assert_close, reference

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2408_16551_gb300 import build
    build.build()
    torch.cuda.set_device(0)


@pytest.mark.parametrize("P,T,dt,n1,n2", [
    (1024, 16, synth.IN_C64, 1024 * 700 + 5, 1024 * 333 + 17),   # second call smaller: stale rows would show
    (256, 8, synth.IN_CI8, 256 * 2000 + 3, 256 * 4100 + 255),
    (4096, 16, synth.IN_R32, 4096 * 300 + 1, 4096 * 40 + 4000),
])
def test_noalloc_matches_execute_host_twice(P, T, dt, n1, n2):
    plan = pkg.Plan(P, T, dt, pkg.PFB_WIN_HAMMING)
    for call, (n, seed) in enumerate(((n1, 31), (n2, 32))):
        x = synth.small_stream(P, T, n, in_dtype=dt, seed=seed).generate()
        want = plan.execute_host(x)
        got = plan.execute_host_noalloc(x)
        assert got.shape == want.shape == (n // P - T + 1, P), call
        assert np.array_equal(got, want), f"call {call}"
    # and both against the FP64 oracle on the last input
    assert_close(got, reference(x, dt, P, T, pkg.PFB_WIN_HAMMING), TOL_F32, TOL_MAX_F32, what="oracle")
    plan.close()


def test_noalloc_first_calls_allocate_nothing():
    """A fresh plan whose first host-buffer calls are no-alloc calls: after one
    warm-up call, a second call leaves cudaMemGetInfo's free bytes unchanged;
    pfb_execute_host (which does allocate staging buffers) runs only
    afterwards, and the two results are equal bit for bit."""
    import torch
    P, T = 1024, 16
    plan = pkg.Plan(P, T, pkg.PFB_IN_C64, pkg.PFB_WIN_HANN)
    x0 = synth.small_stream(P, T, P * 400 + 11, seed=45).generate()
    x1 = synth.small_stream(P, T, P * 900 + 3, seed=46).generate()
    plan.execute_host_noalloc(x0)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    got = plan.execute_host_noalloc(x1)
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, (free0, free1)
    want = plan.execute_host(x1)
    assert np.array_equal(got, want)
    plan.close()


def test_noalloc_split_bf16_path_twice():
    P, T = 1024, 16
    plan = pkg.Plan(P, T, pkg.PFB_IN_C64, pkg.PFB_WIN_BLACKMAN, pkg.PFB_DFT_GEMM_BF16X3)
    for seed, n in ((41, P * 500 + 9), (42, P * 120)):
        x = synth.small_stream(P, T, n, seed=seed).generate()
        want = plan.execute_host(x)
        got = plan.execute_host_noalloc(x)
        assert np.array_equal(got, want), f"seed {seed}"
    plan.close()


def test_noalloc_rejects_inputs_beyond_the_area():
    P, T = 1024, 16
    plan = pkg.Plan(P, T)
    # complex64 in and out: about 8 + 8 bytes per sample, so 2^21 + P*T samples
    # need more than the 32 MiB area
    n = (1 << 21) + P * T
    x = np.zeros(n, dtype=np.complex64)
    out = np.full((n // P - T + 1, P), 7 + 7j, dtype=np.complex64)
    with pytest.raises(pkg.PFBError) as e:
        plan.execute_host_noalloc(x, out)
    assert e.value.status == pkg.PFB_ERR_INVALID
    assert "staging area" in str(e.value)
    assert np.all(out == 7 + 7j)  # nothing was written
    # the largest input that fits still runs and matches
    S_max = 0
    for S in range((pkg.NOALLOC_SCRATCH_BYTES // (16 * P)) + 8, 0, -1):
        frames = S + T - 1
        if (frames * P * 8 + 255) // 256 * 256 + S * P * 8 <= pkg.NOALLOC_SCRATCH_BYTES:
            S_max = S
            break
    n_max = (S_max + T - 1) * P
    x = synth.small_stream(P, T, n_max, seed=43).generate()
    assert np.array_equal(plan.execute_host_noalloc(x), plan.execute_host(x))
    with pytest.raises(pkg.PFBError):
        plan.execute_host_noalloc(synth.small_stream(P, T, n_max + P, seed=44).generate())
    plan.close()
