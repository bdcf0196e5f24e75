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
    assert pkg.last_host_route() == "staged"   # pageable buffers
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


def _pinned_copy(x, offset_elems=0):
    """x copied into page-locked host memory (torch pin_memory), as a numpy
    view starting offset_elems elements into the allocation."""
    import torch
    tdt = {np.complex64: torch.complex64, np.float32: torch.float32, np.int8: torch.int8}[x.dtype.type]
    buf = torch.empty(x.size + offset_elems, dtype=tdt).pin_memory()
    v = buf.numpy()[offset_elems:].reshape(x.shape)
    v[...] = x
    return buf, v


def _host_case(shapes, seed, n_streams):
    rng = np.random.default_rng(seed)
    plans = {s: pkg.Plan(s[0], s[1], s[2], synth.WIN_BLACKMAN) for s in shapes}
    cases = []
    for i in range(n_streams):
        P, T, dt = shapes[i % len(shapes)]
        n = P * (T - 1) - 3 if i == 2 else int(P * (T - 1) + rng.integers(1, 40) * P + rng.integers(0, P))
        x = synth.small_stream(P, T, n, in_dtype=dt, seed=seed + i).generate()
        cases.append((plans[(P, T, dt)], x))
    return plans, cases


def _n(p, x):
    return x.size // 2 if p.in_dtype == pkg.PFB_IN_CI8 else x.size


def _device_reference(cases):
    import torch
    outs_d = [torch.zeros((max(p.out_spectra(_n(p, x)), 1), p.P), dtype=torch.complex64, device="cuda")
              for p, x in cases]
    pkg.pfb_execute_batch([(p, to_device(x), od) for (p, x), od in zip(cases, outs_d)])
    torch.cuda.synchronize()
    return [od.cpu().numpy() for od in outs_d]


def test_mapped_route_pinned_buffers_equal_device_path():
    """Page-locked buffers and the four-step cluster kernel (P = 4096): the
    kernels read and write host memory in place; the result equals the
    device path bit for bit, and forcing the staged route gives it again."""
    shapes = [(4096, 16, synth.IN_C64), (4096, 16, synth.IN_CI8), (4096, 8, synth.IN_R32)]
    plans, cases = _host_case(shapes, 300, 7)
    for p in plans.values():
        assert p.variant == 3, p.kernel_name
    ref = _device_reference(cases)
    keep, entries, outs = [], [], []
    for p, x in cases:
        bx, vx = _pinned_copy(x)
        bo, vo = _pinned_copy(np.full((max(p.out_spectra(_n(p, x)), 1), p.P), 7 + 7j, np.complex64))
        keep += [bx, bo]
        entries.append((p, vx, vo))
        outs.append(vo)
    try:
        for route, name in ((pkg.PFB_HOST_ROUTE_AUTO, "mapped"), (pkg.PFB_HOST_ROUTE_STAGED, "staged")):
            pkg.set_host_route(route)
            for o in outs:
                o[...] = 7 + 7j
            pkg.pfb_execute_batch_host(entries)
            assert pkg.last_host_route() == name
            for i, ((p, x), o, r) in enumerate(zip(cases, outs, ref)):
                S = p.out_spectra(_n(p, x))
                if S == 0:
                    assert np.all(o == 7 + 7j), (name, i)
                    continue
                assert np.array_equal(o[:S], r[:S]), (name, i)
    finally:
        pkg.set_host_route(pkg.PFB_HOST_ROUTE_AUTO)
    p, x = cases[0]
    S = p.out_spectra(_n(p, x))
    rows = [0, S // 2, S - 1]
    want = np.concatenate([reference(x, p.in_dtype, p.P, p.T, synth.WIN_BLACKMAN, s0=r, ns=1) for r in rows])
    assert_close(outs[0][rows], want, TOL_F32, TOL_MAX_F32, what="mapped stream 0")
    for p in plans.values():
        assert p.status() == pkg.PFB_OK
        p.close()


def test_mapped_route_falls_back_to_staged():
    """The mapped route needs every buffer page-locked, 16-byte aligned and
    every plan on a kernel that reads per thread: pageable memory, an
    8-byte-aligned pinned view and a batch mixing in another P each take the
    staged route, with the same results."""
    shapes = [(4096, 16, synth.IN_C64)]
    plans, cases = _host_case(shapes, 400, 3)
    ref = _device_reference(cases)

    def run(entries, outs, want):
        for o in outs:
            o[...] = 7 + 7j
        pkg.pfb_execute_batch_host(entries)
        assert pkg.last_host_route() == want
        for (p, x), o, r in zip(cases, outs, ref):
            S = p.out_spectra(_n(p, x))
            if S:
                assert np.array_equal(o[:S], r[:S])

    # pageable
    outs = [np.empty_like(r) for r in ref]
    run([(p, x, o) for (p, x), o in zip(cases, outs)], outs, "staged")
    # pinned but 8-byte aligned input
    keep, entries, outs = [], [], []
    for p, x in cases:
        bx, vx = _pinned_copy(x, offset_elems=1)
        bo, vo = _pinned_copy(np.empty((max(p.out_spectra(x.size), 1), p.P), np.complex64))
        keep += [bx, bo]
        entries.append((p, vx, vo))
        outs.append(vo)
    assert vx.ctypes.data % 16 == 8
    run(entries, outs, "staged")
    # pinned and aligned: mapped
    keep2, entries2, outs2 = [], [], []
    for p, x in cases:
        bx, vx = _pinned_copy(x)
        bo, vo = _pinned_copy(np.empty((max(p.out_spectra(x.size), 1), p.P), np.complex64))
        keep2 += [bx, bo]
        entries2.append((p, vx, vo))
        outs2.append(vo)
    run(entries2, outs2, "mapped")
    # the same plus a P = 1024 stream (a kernel that moves its input with bulk copies)
    other = pkg.Plan(1024, 16, synth.IN_C64, synth.WIN_BLACKMAN)
    y = synth.small_stream(1024, 16, 1024 * 40, in_dtype=synth.IN_C64, seed=401).generate()
    by, vy = _pinned_copy(y)
    bq, vq = _pinned_copy(np.empty((other.out_spectra(y.size), 1024), np.complex64))
    pkg.pfb_execute_batch_host(entries2 + [(other, vy, vq)])
    assert pkg.last_host_route() == "staged"
    assert np.array_equal(vq, _device_reference([(other, y)])[0])
    with pytest.raises(pkg.PFBError):
        pkg.set_host_route(5)
    for p in list(plans.values()) + [other]:
        assert p.status() == pkg.PFB_OK
        p.close()


@pytest.mark.parametrize("T,dt", [(16, synth.IN_C64), (8, synth.IN_CI8), (4, synth.IN_R32)])
def test_execute_host_mapped_route(T, dt):
    """pfb_execute_host with page-locked buffers on the four-step kernel
    (P = 4096): the mapped route, bitwise equal to the device path and to the
    staged route; the oracle on sampled rows.  A P = 1024 plan on the same
    kind of buffers stays staged."""
    import torch
    P = 4096
    plan = pkg.Plan(P, T, dt, synth.WIN_HAMMING)
    assert plan.variant == 3
    n = P * (T - 1 + 333) + 13
    x = synth.small_stream(P, T, n, in_dtype=dt, seed=T + 900).generate()
    S = plan.out_spectra(_n(plan, x))
    ref = plan.execute(to_device(x)).cpu().numpy()
    torch.cuda.synchronize()
    bx, vx = _pinned_copy(x)
    bo, vo = _pinned_copy(np.zeros((S, P), np.complex64))
    try:
        for route, name in ((pkg.PFB_HOST_ROUTE_AUTO, "mapped"), (pkg.PFB_HOST_ROUTE_STAGED, "staged")):
            pkg.set_host_route(route)
            vo[...] = 7 + 7j
            plan.execute_host(vx, vo)
            assert pkg.last_host_route() == name
            assert np.array_equal(vo, ref), name
    finally:
        pkg.set_host_route(pkg.PFB_HOST_ROUTE_AUTO)
    rows = [0, S // 2, S - 1]
    want = np.concatenate([reference(x, dt, P, T, synth.WIN_HAMMING, s0=r, ns=1) for r in rows])
    assert_close(vo[rows], want, TOL_F32, TOL_MAX_F32, what=f"mapped pfb_execute_host T={T}")
    assert plan.status() == pkg.PFB_OK
    plan.close()
    small = pkg.Plan(1024, 16, synth.IN_C64, synth.WIN_HAMMING)
    y = synth.small_stream(1024, 16, 1024 * 60, seed=901).generate()
    by, vy = _pinned_copy(y)
    bq, vq = _pinned_copy(np.zeros((small.out_spectra(y.size), 1024), np.complex64))
    small.execute_host(vy, vq)
    assert pkg.last_host_route() == "staged"
    assert np.array_equal(vq, small.execute(to_device(y)).cpu().numpy())
    small.close()
