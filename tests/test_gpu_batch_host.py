"""pfb_execute_batch_host: uneven streams from and to host memory (GPU).

The streams are staged through the library's device buffers in chunks of
about 32 MB of input, three chunks in flight, so the case below spans more
chunks than slots (slot reuse) and mixes plans, dtypes, streams with zero
spectra and a stream larger than one chunk.  Results must equal
pfb_execute_batch on device copies bit for bit, and sampled streams the FP64
oracle."""

import numpy as np
import pytest

import paper_2408_16551_gb300 as pkg
from paper_2408_16551_gb300 import synth

from gpu_common import TOL_F32, TOL_MAX_F32, assert_close, reference, to_device

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2408_16551_gb300 import build
    build.build()
    torch.cuda.set_device(0)


def test_batch_host_equals_device_batch_and_oracle():
    import torch
    shapes = [(1024, 16, synth.IN_C64), (4096, 16, synth.IN_C64), (256, 8, synth.IN_CI8), (512, 4, synth.IN_R32)]
    plans = {s: pkg.Plan(s[0], s[1], s[2], synth.WIN_HAMMING) for s in shapes}
    rng = np.random.default_rng(61)
    cases = []
    for i in range(14):
        P, T, dt = shapes[i % len(shapes)]
        if i == 3:
            n = P * (T - 1) - 5                       # no spectra
        elif i == 5:
            n = (5 << 20) + 123                       # larger than one 32 MB chunk (complex64)
        else:
            n = int(P * (T - 1) + rng.integers(P, 1 << 20))
        x = synth.small_stream(P, T, n, in_dtype=dt, seed=100 + i).generate()
        cases.append((plans[(P, T, dt)], x))
    outs_h = [np.full((max(p.out_spectra(x.size // 2 if p.in_dtype == pkg.PFB_IN_CI8 else x.size), 1), p.P), 7 + 7j,
                      dtype=np.complex64) for p, x in cases]
    pkg.pfb_execute_batch_host([(p, x, o) for (p, x), o in zip(cases, outs_h)])
    xs_d = [to_device(x) for _, x in cases]
    outs_d = [torch.zeros(o.shape, dtype=torch.complex64, device="cuda") for o in outs_h]
    pkg.pfb_execute_batch([(p, xd, od) for (p, _), xd, od in zip(cases, xs_d, outs_d)])
    torch.cuda.synchronize()
    for i, ((p, x), oh, od) in enumerate(zip(cases, outs_h, outs_d)):
        n = x.size // 2 if p.in_dtype == pkg.PFB_IN_CI8 else x.size
        S = p.out_spectra(n)
        if S == 0:
            assert np.all(oh == 7 + 7j), i  # untouched
            continue
        assert np.array_equal(oh[:S], od[:S].cpu().numpy()), i
    for i in (0, 2, 5, 7):
        p, x = cases[i]
        n = x.size // 2 if p.in_dtype == pkg.PFB_IN_CI8 else x.size
        S = p.out_spectra(n)
        rows = [0, S // 2, S - 1]
        ref = np.concatenate([reference(x, p.in_dtype, p.P, p.T, synth.WIN_HAMMING, s0=r, ns=1) for r in rows])
        assert_close(outs_h[i][rows], ref, TOL_F32, TOL_MAX_F32, what=f"stream {i}")
    for p in plans.values():
        assert p.status() == pkg.PFB_OK
        p.close()


def test_batch_host_rejects_before_copying():
    plan = pkg.Plan(1024, 16)
    x = np.zeros(1024 * 40, dtype=np.complex64)
    out = np.full((10, 1024), 7 + 7j, dtype=np.complex64)   # 25 spectra needed
    with pytest.raises(pkg.PFBError) as e:
        pkg.pfb_execute_batch_host([(plan, x, out)])
    assert e.value.status == pkg.PFB_ERR_INVALID
    assert np.all(out == 7 + 7j)
    over = pkg.Plan(1024, 16, hop=512)
    with pytest.raises(pkg.PFBError) as e:
        pkg.pfb_execute_batch_host([(over, x, np.empty((60, 1024), np.complex64))])
    assert e.value.status == pkg.PFB_ERR_UNSUPPORTED
    plan.close(); over.close()
