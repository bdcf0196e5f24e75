"""Parity of the FFT path (fused FIR + radix FFT, FP32) with the FP64 oracle,
through the C ABI.  Sizes span several work units and a ragged tail."""

import numpy as np
import pytest

import oracle
import paper_2408_16551_gb300 as pkg
from paper_2408_16551_gb300 import synth

from gpu_common import TOL_F32, assert_close, reference, to_device

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2408_16551_gb300 import build
    build.build()
    torch.cuda.set_device(0)


def _run(P, T, in_dtype, n, window=synth.WIN_HANN, seed=0, scale=1.0):
    import torch
    spec = synth.small_stream(P, T, n, in_dtype=in_dtype, seed=seed, window=window)
    x = spec.generate()
    plan = pkg.Plan(P, T, in_dtype, window, pkg.PFB_DFT_FFT_F32, in_scale=scale)
    X = plan.execute(to_device(x))
    torch.cuda.synchronize()
    return plan, x, X.cpu().numpy()


FAST = [(P, T, dt) for P in (64, 128, 256, 512, 1024)
        for (T, dt) in ((16, synth.IN_C64), (8, synth.IN_R32), (4, synth.IN_CI8), (3, synth.IN_C64),
                        (1, synth.IN_C64), (12, synth.IN_CI8))]
GENERIC = [(4, 2, synth.IN_C64), (8, 3, synth.IN_R32), (16, 4, synth.IN_R32), (32, 16, synth.IN_CI8),
           (64, 17, synth.IN_C64), (1024, 64, synth.IN_C64), (4096, 20, synth.IN_C64), (2048, 33, synth.IN_CI8)]
CLUSTER = [(2048, 16, synth.IN_C64), (4096, 16, synth.IN_CI8), (4096, 8, synth.IN_C64), (4096, 16, synth.IN_C64),
           (2048, 4, synth.IN_R32), (4096, 3, synth.IN_C64), (4096, 12, synth.IN_R32)]


@pytest.mark.parametrize("P,T,dt", FAST + GENERIC + CLUSTER)
def test_fft_path_parity(P, T, dt):
    n = P * (T - 1 + 8 * 5 + 3) + 7          # 5 full units + 3 spectra + a partial frame
    plan, x, got = _run(P, T, dt, n, seed=P + T)
    ref = reference(x, dt, P, T, synth.WIN_HANN)
    assert got.shape == (plan.out_spectra(n), P)
    assert_close(got, ref, what=f"{plan.kernel_name} P={P} T={T} dt={dt}")


def test_fast_family_is_selected():
    for P, T in ((64, 16), (1024, 16), (256, 8)):
        assert pkg.Plan(P, T).kernel_name == "pfb_fir_fft_f32"
    assert pkg.Plan(4096, 16).kernel_name == "pfb_fir_fft_f32_cluster"
    assert pkg.Plan(2048, 8).kernel_name == "pfb_fir_fft_f32_cluster"
    assert pkg.Plan(4096, 20).kernel_name == "pfb_fir_fft_f32_generic"
    assert pkg.Plan(32, 16).kernel_name == "pfb_fir_fft_f32_generic"


@pytest.mark.parametrize("P,T", [(64, 4), (1024, 16), (4096, 16), (16, 4)])
def test_zero_spectra_is_a_noop(P, T):
    import torch
    plan = pkg.Plan(P, T)
    for n in (0, P - 1, P * T - 1):
        assert plan.out_spectra(n) == 0
        x = torch.zeros(max(n, 1), dtype=torch.complex64, device="cuda")[:n]
        out = torch.full((2, P), 7.0, dtype=torch.complex64, device="cuda")
        plan.execute(x, out=out)
        torch.cuda.synchronize()
        assert torch.all(out == 7.0)


@pytest.mark.parametrize("P,T", [(64, 4), (1024, 16), (4096, 16)])
def test_exactly_one_spectrum_and_output_capacity(P, T):
    import torch
    n = P * T
    plan, x, got = _run(P, T, synth.IN_C64, n, seed=5)
    assert got.shape == (1, P)
    assert_close(got, reference(x, synth.IN_C64, P, T, synth.WIN_HANN))
    small = torch.empty((0, P), dtype=torch.complex64, device="cuda")
    with pytest.raises(pkg.PFBError) as ei:
        plan.execute(to_device(x), out=small)
    assert ei.value.status == pkg.PFB_ERR_INVALID


def test_config1_real_input():
    spec = synth.config_c1()
    x = spec.generate()
    plan = pkg.Plan(spec.P, spec.T, pkg.PFB_IN_R32, spec.window)
    got = plan.execute(to_device(x)).cpu().numpy()
    ref = reference(x, synth.IN_R32, spec.P, spec.T, spec.window)
    assert got.shape == (1021, 16)
    assert_close(got, ref, what="c1")
    assert_close(got[:253], ref[:253], what="c1 first 253 rows")


def test_config2_full_size_sampled():
    """2^24 complex samples, P=1024, T=16: compare sampled spectra one by one."""
    import torch
    spec = synth.config_c2()
    x = spec.generate()
    plan = pkg.Plan(spec.P, spec.T, pkg.PFB_IN_C64, spec.window)
    X = plan.execute(to_device(x))
    torch.cuda.synchronize()
    S = plan.out_spectra(x.size)
    assert X.shape == (S, spec.P) == (16369, 1024)
    rng = np.random.default_rng(99)
    rows = sorted(set([0, 1, 7, 8, S // 2, S - 9, S - 2, S - 1] + list(rng.integers(0, S, 24))))
    h = oracle.prototype(spec.P, spec.T, spec.window)
    xs = oracle.dequant(x, oracle.IN_C64)
    got = X[rows].cpu().numpy()
    ref = np.concatenate([oracle.pfb(xs, spec.P, spec.T, h, s0=int(r), ns=1) for r in rows])
    assert_close(got, ref, what="c2 sampled")
    # every spectrum is finite and the tones sit in their channels
    Xa = X.abs().mean(dim=0).cpu().numpy()
    tone_bins = [c for (c, _, _) in spec.tones]
    assert set(np.argsort(Xa)[-len(tone_bins):]) == set(tone_bins)
    assert torch.isfinite(X.view(torch.float32)).all()


def test_deterministic_bitwise():
    import torch
    P, T = 1024, 16
    spec = synth.small_stream(P, T, P * 200, seed=1)
    xd = to_device(spec.generate())
    plan = pkg.Plan(P, T)
    a = plan.execute(xd).clone()
    b = plan.execute(xd)
    torch.cuda.synchronize()
    assert torch.equal(a, b)


def test_taps_generated_on_gpu_match_oracle():
    for (P, T, w) in ((16, 4, pkg.PFB_WIN_HANN), (1024, 16, pkg.PFB_WIN_HAMMING), (4096, 16, pkg.PFB_WIN_BLACKMAN),
                      (256, 8, pkg.PFB_WIN_HANN)):
        h_gpu = pkg.Plan(P, T, window=w).taps()
        h_ref = oracle.prototype(P, T, w)
        assert np.max(np.abs(h_gpu - h_ref)) <= 1e-14 * np.max(np.abs(h_ref)) * 10


def test_user_taps():
    P, T = 256, 8
    rng = np.random.default_rng(4)
    taps = rng.standard_normal(P * T)
    spec = synth.small_stream(P, T, P * 60, seed=8)
    x = spec.generate()
    plan = pkg.Plan(P, T, window=pkg.PFB_WIN_USER, user_taps=taps)
    assert np.array_equal(plan.taps(), taps)
    got = plan.execute(to_device(x)).cpu().numpy()
    ref = reference(x, synth.IN_C64, P, T, synth.WIN_USER, user_taps=taps)
    assert_close(got, ref, what="user taps")


def test_int8_scale():
    P, T = 512, 16
    spec = synth.small_stream(P, T, P * 70, in_dtype=synth.IN_CI8, seed=2)
    x = spec.generate()
    plan = pkg.Plan(P, T, pkg.PFB_IN_CI8, in_scale=0.125)
    got = plan.execute(to_device(x)).cpu().numpy()
    ref = reference(x, synth.IN_CI8, P, T, synth.WIN_HANN, scale=0.125)
    assert_close(got, ref, what="int8 scaled")


def test_batch_equals_single_bitwise():
    import torch
    shapes = [(256, 8, synth.IN_C64, 256 * 300 + 5), (1024, 16, synth.IN_C64, 1024 * 100),
              (1024, 16, synth.IN_C64, 1024 * 15), (4096, 16, synth.IN_C64, 4096 * 40),
              (512, 16, synth.IN_CI8, 512 * 77), (16, 4, synth.IN_R32, 16 * 999), (256, 8, synth.IN_C64, 256 * 33)]
    entries, singles = [], []
    for i, (P, T, dt, n) in enumerate(shapes):
        x = to_device(synth.small_stream(P, T, n, in_dtype=dt, seed=30 + i).generate())
        plan = pkg.Plan(P, T, dt, window=i % 3)
        S = plan.out_spectra(n)
        out = torch.zeros((max(S, 1), P), dtype=torch.complex64, device="cuda")
        entries.append((plan, x, out))
        singles.append(plan.execute(x).clone() if S > 0 else None)
    pkg.pfb_execute_batch(entries)
    torch.cuda.synchronize()
    for (plan, x, out), ref in zip(entries, singles):
        if ref is not None:
            assert torch.equal(out[:ref.shape[0]], ref)
    for (_, _, out) in entries:
        out.zero_()
    b = pkg.Batch(entries)
    b.launch()
    b.launch()
    torch.cuda.synchronize()
    for (plan, x, out), ref in zip(entries, singles):
        if ref is not None:
            assert torch.equal(out[:ref.shape[0]], ref)


def test_execute_host_matches_device():
    import torch
    P, T = 1024, 16
    x = synth.small_stream(P, T, P * 90 + 3, seed=6).generate()
    plan = pkg.Plan(P, T)
    dev = plan.execute(to_device(x)).cpu().numpy()
    host = plan.execute_host(x)
    assert np.array_equal(dev, host)


@pytest.mark.parametrize("P,T,dt,n", [(1024, 16, synth.IN_C64, (5 << 22) + 3 * 1024 + 5),
                                      (256, 8, synth.IN_CI8, (9 << 23) + 77),
                                      (4096, 16, synth.IN_R32, (3 << 22) + 4096 * 7 + 1)])
def test_execute_host_chunked_matches_device(P, T, dt, n):
    """Host-buffer path over several pipeline chunks (input > 16 MB), ragged tail:
    identical to the device-resident launch."""
    import torch
    x = synth.small_stream(P, T, n, in_dtype=dt, seed=12).generate()
    plan = pkg.Plan(P, T, dt, pkg.PFB_WIN_HAMMING)
    dev = plan.execute(to_device(x)).cpu().numpy()
    host = plan.execute_host(x)
    assert host.shape == dev.shape == (n // P - T + 1, P)
    assert np.array_equal(dev, host)
    xp = torch.from_numpy(x).pin_memory()
    outp = torch.empty((n // P - T + 1, P), dtype=torch.complex64).pin_memory()
    plan.execute_host(xp.numpy(), outp.numpy())
    assert np.array_equal(dev, outp.numpy())


@pytest.mark.parametrize("P,T,dt", [(1024, 16, synth.IN_C64), (512, 8, synth.IN_CI8), (256, 16, synth.IN_R32),
                                    (128, 4, synth.IN_C64), (64, 12, synth.IN_C64), (1024, 8, synth.IN_CI8),
                                    (1024, 4, synth.IN_R32), (512, 16, synth.IN_C64), (1024, 12, synth.IN_C64)])
def test_every_fast_variant_matches_oracle(P, T, dt):
    import torch
    n = P * (T - 1 + 8 * 7 + 5) + 3
    x = synth.small_stream(P, T, n, in_dtype=dt, seed=77).generate()
    ref = reference(x, dt, P, T, synth.WIN_HAMMING)
    plan = pkg.Plan(P, T, dt, pkg.PFB_WIN_HAMMING)
    assert plan.num_variants == 6
    xd = to_device(x)
    outs = []
    for v in range(plan.num_variants):
        try:
            plan.variant = v
        except pkg.PFBError as e:      # variant 5 needs P >= 128 and T in {4, 8, 16}
            assert e.status == pkg.PFB_ERR_UNSUPPORTED and v == 5 and (P < 128 or T not in (4, 8, 16))
            continue
        assert plan.variant == v
        got = plan.execute(xd).cpu().numpy()
        assert_close(got, ref, what=f"variant {v} P={P} T={T}")
        outs.append(got)


def test_autotune_picks_a_variant_and_keeps_results():
    P, T = 1024, 16
    n = P * 4000
    plan = pkg.Plan(P, T, pkg.PFB_IN_C64, pkg.PFB_WIN_HANN)
    ms = plan.autotune(n)
    assert ms > 0 and 0 <= plan.variant < plan.num_variants
    x = synth.small_stream(P, T, P * 100, seed=5).generate()
    got = plan.execute(to_device(x)).cpu().numpy()
    assert_close(got, reference(x, synth.IN_C64, P, T, synth.WIN_HANN))
    with pytest.raises(pkg.PFBError):
        plan.variant = 9


@pytest.mark.parametrize("P,T", [(1024, 16), (256, 8)])
def test_ws_variant_streams_and_batches(P, T):
    """Warp-specialised variant: several streams in one launch (segments that
    start mid-range), chunked serving with resident state, bitwise equality."""
    import torch
    shapes = [P * 300 + 17, P * (T + 1), P * 40, P * (T - 1)]     # the last one gives 0 spectra
    plans, xs, singles = [], [], []
    for i, n in enumerate(shapes):
        plan = pkg.Plan(P, T, pkg.PFB_IN_C64, pkg.PFB_WIN_BLACKMAN)
        plan.variant = 5
        x = synth.small_stream(P, T, n, seed=60 + i).generate()
        xd = to_device(x)
        plans.append(plan); xs.append((x, xd))
        if plan.out_spectra(n) > 0:
            got = plan.execute(xd)
            assert_close(got.cpu().numpy(), reference(x, synth.IN_C64, P, T, synth.WIN_BLACKMAN), what=f"ws {i}")
            singles.append(got.clone())
        else:
            singles.append(None)
    entries = []
    for plan, (x, xd), n in zip(plans, xs, shapes):
        S = plan.out_spectra(n)
        entries.append((plan, xd, torch.zeros((max(S, 1), P), dtype=torch.complex64, device="cuda")))
    pkg.pfb_execute_batch(entries)
    torch.cuda.synchronize()
    for (plan, xd, out), ref in zip(entries, singles):
        if ref is not None:
            assert torch.equal(out[:ref.shape[0]], ref)


WS_CLUSTER = [(4096, 16, synth.IN_C64, 43), (2048, 16, synth.IN_CI8, 43), (4096, 8, synth.IN_R32, 301),
              (2048, 4, synth.IN_C64, 1000), (4096, 4, synth.IN_CI8, 7), (4096, 16, synth.IN_C64, 1001),
              (2048, 8, synth.IN_R32, 1)]


@pytest.mark.parametrize("P,T,dt,S", WS_CLUSTER)
def test_cluster_variants_match_oracle(P, T, dt, S):
    """P = 2048 / 4096 on a CTA cluster: variant 0 (synchronous), variant 1
    (warp-specialised, cross-CTA step in the FFT warps), variant 2
    (warp-specialised, one exchange from the FIR warps' radix-4 step to the
    receiving FFT warps' radix-CS step) and, for P = 4096, variant 3 (four-step
    64 x 64: contiguous input and output runs per CTA) against the oracle;
    every warp-specialised variant is bitwise reproducible."""
    import torch
    n = P * (S + T - 1) + 5
    x = synth.small_stream(P, T, n, in_dtype=dt, seed=P + S).generate()
    ref = reference(x, dt, P, T, synth.WIN_BLACKMAN)
    plan = pkg.Plan(P, T, dt, pkg.PFB_WIN_BLACKMAN)
    assert plan.num_variants == 4 and plan.variant == (3 if P == 4096 else 2)
    xd = to_device(x)
    outs = {}
    ws = (1, 2, 3) if P == 4096 else (1, 2)
    if P != 4096:
        with pytest.raises(pkg.PFBError):
            plan.variant = 3
    for v in (0,) + ws:
        plan.variant = v
        X = plan.execute(xd)
        torch.cuda.synchronize()
        outs[v] = X.cpu().numpy()
        assert plan.status() == pkg.PFB_OK
        assert_close(outs[v], ref, what=f"cluster variant {v} P={P} T={T} dt={dt} S={S}")
    for v in ws:
        plan.variant = v
        for _ in range(3):  # a ring or receive slot reused too early shows up as wrong spectra
            again = plan.execute(xd).cpu().numpy()
            assert np.array_equal(again, outs[v]), v


@pytest.mark.parametrize("variant", [1, 2, 3])
def test_cluster_ws_batch_equals_single(variant):
    """Uneven streams (some with 0 spectra) of one P = 4096 plan in one batched
    launch of a warp-specialised cluster kernel: identical to per-stream runs."""
    import torch
    P, T = 4096, 16
    plan = pkg.Plan(P, T, pkg.PFB_IN_C64, pkg.PFB_WIN_HANN)
    plan.variant = variant
    lens = [P * 20 + 3, P * 3, P * 15, P * 97 + 11, P * 16, P * 300, P * 41]
    xs = [to_device(synth.small_stream(P, T, n, seed=70 + i).generate()) for i, n in enumerate(lens)]
    singles = [plan.execute(x).clone() if plan.out_spectra(x.numel()) > 0 else None for x in xs]
    outs = [torch.full((max(plan.out_spectra(x.numel()), 1), P), 9.0, dtype=torch.complex64, device="cuda")
            for x in xs]
    pkg.pfb_execute_batch([(plan, x, o) for x, o in zip(xs, outs)])
    torch.cuda.synchronize()
    for s, o in zip(singles, outs):
        if s is not None:
            assert torch.equal(o[:s.shape[0]], s)
        else:
            assert torch.all(o == 9.0)


@pytest.mark.parametrize("P,variant", [(1024, 5), (4096, 1), (4096, 2), (2048, 2), (4096, 3)])
def test_ws_repeatable_at_scale(P, variant):
    """A warp-specialised kernel over 4096 spectra (P = 1024: one stream; P =
    2048, 4096: 16 streams of 256 spectra in one launch, every cluster with
    several segments), run six times: bitwise identical (a race on the TMA
    ring or a receive slot would corrupt runs of spectra); sampled rows
    against the oracle."""
    import torch
    T = 16
    plan = pkg.Plan(P, T, pkg.PFB_IN_C64, pkg.PFB_WIN_HAMMING)
    plan.variant = variant
    if P == 1024:
        xs = [synth.small_stream(P, T, P * (4096 + T - 1), seed=17).generate()]
    else:
        xs = [synth.small_stream(P, T, P * (256 + T - 1) + 9, seed=17 + i).generate() for i in range(16)]
    xd = [to_device(x) for x in xs]
    outs = [torch.empty((plan.out_spectra(x.size), P), dtype=torch.complex64, device="cuda") for x in xs]

    def run():
        pkg.pfb_execute_batch([(plan, x, o) for x, o in zip(xd, outs)])
        torch.cuda.synchronize()
        return [o.clone() for o in outs]

    a = run()
    for _ in range(5):
        b = run()
        assert all(torch.equal(u, v) for u, v in zip(a, b))
    assert plan.status() == pkg.PFB_OK
    for i in (0, len(xs) - 1):
        S = a[i].shape[0]
        rows = [0, S // 2, S - 1]
        ref = np.concatenate([reference(xs[i], synth.IN_C64, P, T, synth.WIN_HAMMING, s0=r, ns=1) for r in rows])
        assert_close(a[i][rows].cpu().numpy(), ref, what=f"P={P} variant {variant} stream {i}")


HOP = [(1024, 16, synth.IN_C64, 512, 0), (1024, 16, synth.IN_C64, 256, 1), (256, 8, synth.IN_R32, 64, 0),
       (64, 4, synth.IN_CI8, 16, 1), (4096, 16, synth.IN_C64, 2048, 0), (2048, 8, synth.IN_CI8, 512, 1),
       (512, 16, synth.IN_C64, 128, 0), (32, 4, synth.IN_C64, 16, 1), (4096, 12, synth.IN_R32, 1024, 1)]


@pytest.mark.parametrize("P,T,dt,D,rev", HOP)
def test_oversampled_and_tap_order_match_oracle(P, T, dt, D, rev):
    """Hop D < P (oversampled channeliser) and the convolution tap order, every
    kernel variant of the plan's family, against the FP64 oracle."""
    import torch
    from gpu_common import reference_hop
    S_want = 3 * (P // D) + 7
    n = P * T + D * (S_want - 1) + D // 2 + 1      # ragged tail shorter than the hop
    x = synth.small_stream(P, T, n, in_dtype=dt, seed=P + D + rev).generate()
    order = pkg.PFB_TAPS_CONVOLUTION if rev else pkg.PFB_TAPS_CORRELATION
    plan = pkg.Plan(P, T, dt, pkg.PFB_WIN_HAMMING, hop=D, tap_order=order)
    assert plan.out_spectra(n) == S_want
    ref = reference_hop(x, dt, P, T, synth.WIN_HAMMING, D, reverse=bool(rev))
    assert ref.shape[0] == S_want
    xd = to_device(x)
    for v in range(plan.num_variants):
        try:
            plan.variant = v
        except pkg.PFBError:
            continue
        X = plan.execute(xd)
        torch.cuda.synchronize()
        assert_close(X.cpu().numpy(), ref, what=f"hop {D} rev {rev} {plan.kernel_name} variant {v}")


@pytest.mark.parametrize("path,P,T,D", [(pkg.PFB_DFT_GEMM_BF16X3, 1024, 16, 512), (pkg.PFB_DFT_GEMM_F32, 256, 8, 128),
                                        (pkg.PFB_DFT_GEMM_BF16X3, 4096, 16, 2048)])
def test_oversampled_gemm_paths(path, P, T, D):
    import torch
    from gpu_common import TOL_BF16X3, TOL_MAX_BF16X3, TOL_MAX_F32, reference_hop
    n = P * T + D * 20 + 3
    x = synth.small_stream(P, T, n, seed=D).generate()
    plan = pkg.Plan(P, T, pkg.PFB_IN_C64, pkg.PFB_WIN_BLACKMAN, path, hop=D)
    ref = reference_hop(x, synth.IN_C64, P, T, synth.WIN_BLACKMAN, D)
    X = plan.execute(to_device(x))
    torch.cuda.synchronize()
    if path == pkg.PFB_DFT_GEMM_BF16X3:
        assert_close(X.cpu().numpy(), ref, TOL_BF16X3, TOL_MAX_BF16X3, what="bf16x3 hop")
    else:
        assert_close(X.cpu().numpy(), ref, TOL_F32, TOL_MAX_F32, what="gemm f32 hop")


def test_oversampled_batch_equals_single():
    import torch
    P, T, D = 1024, 16, 256
    plan = pkg.Plan(P, T, pkg.PFB_IN_C64, pkg.PFB_WIN_HANN, hop=D)
    lens = [P * T + D * 50 + 3, P * T - 1, P * T + D * 5, P * 40 + 17]
    xs = [to_device(synth.small_stream(P, T, n, seed=90 + i).generate()) for i, n in enumerate(lens)]
    singles = [plan.execute(x).clone() if plan.out_spectra(x.numel()) > 0 else None for x in xs]
    outs = [torch.full((max(plan.out_spectra(x.numel()), 1), P), 5.0, dtype=torch.complex64, device="cuda")
            for x in xs]
    pkg.pfb_execute_batch([(plan, x, o) for x, o in zip(xs, outs)])
    torch.cuda.synchronize()
    for s, o in zip(singles, outs):
        if s is not None:
            assert torch.equal(o[:s.shape[0]], s)
        else:
            assert torch.all(o == 5.0)
    with pytest.raises(pkg.PFBError) as e:
        plan.execute_host(np.zeros(P * T * 2, dtype=np.complex64))
    assert e.value.status == pkg.PFB_ERR_UNSUPPORTED
