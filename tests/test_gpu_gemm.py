"""Parity of the two DFT-as-matrix-product paths with the FP64 oracle:
FP32 on the SIMT cores (rel. L2 <= 2e-6) and split-bf16 on the tensor cores
(rel. L2 <= 1e-5), through the C ABI."""

import numpy as np
import pytest

import oracle
import paper_2408_16551_gb300 as pkg
from paper_2408_16551_gb300 import synth

from gpu_common import TOL_BF16X3, TOL_MAX_BF16X3, assert_close, reference, to_device
from split_models import factored_dft_model, split_bf16x3_model

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2408_16551_gb300 import build
    build.build()
    torch.cuda.set_device(0)


def _run(path, P, T, dt, n, seed=0, window=synth.WIN_HANN):
    import torch
    x = synth.small_stream(P, T, n, in_dtype=dt, seed=seed, window=window).generate()
    plan = pkg.Plan(P, T, dt, window, path)
    X = plan.execute(to_device(x))
    torch.cuda.synchronize()
    return plan, x, X.cpu().numpy()


@pytest.mark.parametrize("P,T,dt", [(64, 4, synth.IN_C64), (128, 16, synth.IN_R32), (256, 8, synth.IN_CI8),
                                    (1024, 16, synth.IN_C64), (64, 20, synth.IN_C64)])
def test_gemm_f32_parity(P, T, dt):
    n = P * (T - 1 + 64 * 2 + 37) + 5
    plan, x, got = _run(pkg.PFB_DFT_GEMM_F32, P, T, dt, n, seed=P + T)
    assert plan.kernel_name == "pfb_fir_dftgemm_f32"
    assert_close(got, reference(x, dt, P, T, synth.WIN_HANN), what=f"gemm_f32 P={P} T={T}")


BF16 = [(128, 16, synth.IN_C64), (256, 8, synth.IN_C64), (256, 4, synth.IN_R32), (512, 16, synth.IN_CI8),
        (1024, 16, synth.IN_C64), (4096, 16, synth.IN_C64), (256, 3, synth.IN_C64)]


@pytest.mark.parametrize("P,T,dt", BF16)
def test_gemm_bf16x3_parity(P, T, dt):
    rows = 128 * 2 + 45 if P <= 1024 else 128 + 9
    n = P * (T - 1 + rows) + 3
    plan, x, got = _run(pkg.PFB_DFT_GEMM_BF16X3, P, T, dt, n, seed=2 * P + T)
    assert plan.kernel_name == "pfb_fir_dftgemm_bf16x3"
    ref = reference(x, dt, P, T, synth.WIN_HANN)
    e2, em = assert_close(got, ref, TOL_BF16X3, TOL_MAX_BF16X3, what=f"bf16x3 P={P} T={T}")
    assert e2 > 1e-8          # split arithmetic is not exact: the kernel really ran the bf16 path


def _run_variant(variant, P, T, dt, n, seed=0, window=synth.WIN_HANN):
    import torch
    x = synth.small_stream(P, T, n, in_dtype=dt, seed=seed, window=window).generate()
    plan = pkg.Plan(P, T, dt, window, pkg.PFB_DFT_GEMM_BF16X3)
    plan.variant = variant
    X = plan.execute(to_device(x))
    torch.cuda.synchronize()
    return plan, x, X.cpu().numpy()


@pytest.mark.parametrize("P,T", [(256, 8), (1024, 16)])
def test_gemm_bf16x3_matches_split_model(P, T):
    """Dense DFT-matrix product (variant 0) against the FP64 model of the split
    arithmetic (hi*hi + hi*lo + lo*hi): agreement to FP32-accumulation error
    separates split error from indexing."""
    n = P * (T - 1 + 200)
    plan, x, got = _run_variant(0, P, T, synth.IN_C64, n, seed=9)
    h = oracle.prototype(P, T, oracle.WIN_HANN)
    y = oracle.fir(oracle.dequant(x, oracle.IN_C64), P, T, h)
    model = split_bf16x3_model(y.astype(np.complex64), P)
    exact = oracle.dft(y)
    e_model = oracle.rel_l2(got, model)
    e_exact = oracle.rel_l2(got, exact)
    # The tensor core's FP32 accumulation adds ~1.8e-8 of the result per MMA
    # step; the kernel accumulates chunks of 8 K blocks (96 MMA steps) in TMEM
    # and sums the chunks in FP32 on the CUDA cores, so the distance to the
    # exact-split model is bounded near 96 * 1.8e-8 = 1.7e-6 for every P.
    # An indexing or split bug would show up as an O(1) error here.
    assert e_model < 3e-6, e_model
    assert e_exact < 1e-5


def test_gemm_bf16x3_deterministic_and_chunked():
    import torch
    P, T, chunk = 1024, 16, 1024 * 64
    x = to_device(synth.small_stream(P, T, chunk * 5, seed=12).generate())
    plan = pkg.Plan(P, T, pkg.PFB_IN_C64, pkg.PFB_WIN_HANN, pkg.PFB_DFT_GEMM_BF16X3)
    a = plan.execute(x).clone()
    b = plan.execute(x)
    torch.cuda.synchronize()
    assert torch.equal(a, b)
    srv = pkg.Server(hbm_budget_bytes=1 << 32, max_slots=4)
    sid = srv.open_stream(plan)
    outs, tickets = [], []
    for c in range(5):
        S = srv.next_spectra(sid, chunk)
        o = torch.empty((S, P), dtype=torch.complex64, device="cuda")
        tickets.append(srv.submit(sid, x[c * chunk:(c + 1) * chunk], chunk, o))
        outs.append(o)
    for t in tickets:
        assert srv.wait(t, 20000) == pkg.PFB_OK
    assert torch.equal(torch.cat(outs), a)
    srv.close()


def test_gemm_paths_report_unsupported_shapes():
    import torch
    plan = pkg.Plan(64, 16, path=pkg.PFB_DFT_GEMM_BF16X3)     # P < 128
    x = torch.zeros(64 * 40, dtype=torch.complex64, device="cuda")
    with pytest.raises(pkg.PFBError) as ei:
        plan.execute(x)
    assert ei.value.status == pkg.PFB_ERR_UNSUPPORTED
    plan = pkg.Plan(256, 20, path=pkg.PFB_DFT_GEMM_BF16X3)    # T > 16
    with pytest.raises(pkg.PFBError) as ei:
        plan.execute(torch.zeros(256 * 40, dtype=torch.complex64, device="cuda"))
    assert ei.value.status == pkg.PFB_ERR_UNSUPPORTED


# ---------------------------------------------------------------------------
# factored (four-step) tensor-core DFT, variant 1 (P = 32 x 32)
# ---------------------------------------------------------------------------

def test_factored_is_the_default_at_p1024():
    plan = pkg.Plan(1024, 16, pkg.PFB_IN_C64, pkg.PFB_WIN_HANN, pkg.PFB_DFT_GEMM_BF16X3)
    assert plan.num_variants == 3 and plan.variant == 1
    plan2 = pkg.Plan(1024, 12, pkg.PFB_IN_C64, pkg.PFB_WIN_HANN, pkg.PFB_DFT_GEMM_BF16X3)
    assert plan2.variant == 2                 # T = 12 is not a compiled tap count: the two-pass product
    with pytest.raises(pkg.PFBError):
        plan2.variant = 1
    plan3 = pkg.Plan(512, 16, pkg.PFB_IN_C64, pkg.PFB_WIN_HANN, pkg.PFB_DFT_GEMM_BF16X3)
    assert plan3.variant == 0
    for P, T in ((2048, 16), (4096, 12)):   # cluster route: any T <= 16
        assert pkg.Plan(P, T, pkg.PFB_IN_C64, pkg.PFB_WIN_HANN, pkg.PFB_DFT_GEMM_BF16X3).variant == 1


@pytest.mark.parametrize("T,dt,rows", [(16, synth.IN_C64, 4 * 37 + 3), (8, synth.IN_CI8, 4 * 20 + 1),
                                       (4, synth.IN_R32, 4 * 9 + 2), (16, synth.IN_C64, 2),
                                       (16, synth.IN_R32, 4 * 160)])
def test_gemm_bf16x3_factored_parity(T, dt, rows):
    """Several 4-spectrum tiles with ragged last tiles (and a stream shorter than
    one tile) against the FP64 oracle at the split-bf16 bound."""
    P = 1024
    n = P * (T - 1 + rows) + 7
    plan, x, got = _run_variant(1, P, T, dt, n, seed=T * 7 + rows)
    ref = reference(x, dt, P, T, synth.WIN_HANN)
    assert got.shape == ref.shape == (rows, P)
    e2, em = assert_close(got, ref, TOL_BF16X3, TOL_MAX_BF16X3, what=f"bf16x3 factored T={T} rows={rows}")
    assert e2 > 1e-8


def test_gemm_bf16x3_factored_matches_model():
    """Against the FP64 model of the four-step split arithmetic: a wrong tile,
    transpose or twiddle index shows up as an O(1) error here."""
    P, T = 1024, 16
    n = P * (T - 1 + 96)
    plan, x, got = _run_variant(1, P, T, synth.IN_C64, n, seed=19)
    h = oracle.prototype(P, T, oracle.WIN_HANN)
    y = oracle.fir(oracle.dequant(x, oracle.IN_C64), P, T, h)
    model = factored_dft_model(y.astype(np.complex64), 32, 32)
    e_model = oracle.rel_l2(got, model)
    e_exact = oracle.rel_l2(got, oracle.dft(y))
    assert e_model < 2e-6, e_model
    assert e_exact < 1e-5, e_exact


def test_gemm_bf16x3_factored_batch_and_c2_sample():
    """Uneven streams in one batched launch equal their single launches; the
    full c2 workload on the factored path, sampled rows against the oracle."""
    import torch
    P, T = 1024, 16
    plan = pkg.Plan(P, T, pkg.PFB_IN_C64, synth.WIN_HAMMING, pkg.PFB_DFT_GEMM_BF16X3)
    assert plan.variant == 1
    xs = [to_device(synth.small_stream(P, T, P * (T - 1 + r) + 5, seed=r).generate()) for r in (1, 7, 64, 130)]
    singles = [plan.execute(x).clone() for x in xs]
    outs = [torch.empty_like(o) for o in singles]
    pkg.pfb_execute_batch([(plan, x, o) for x, o in zip(xs, outs)])
    torch.cuda.synchronize()
    for a, b in zip(outs, singles):
        assert torch.equal(a, b)
    spec = synth.config_c2()
    x = spec.generate()
    X = plan.execute(to_device(x))
    torch.cuda.synchronize()
    S = X.shape[0]
    rows = [0, 1, 2, 3, S // 2, S - 2, S - 1]
    h = oracle.prototype(P, T, oracle.WIN_HAMMING)
    got = X[rows].cpu().numpy()
    xin = oracle.dequant(x, oracle.IN_C64)
    ref = np.stack([oracle.dft(oracle.fir(xin, P, T, h, s0=r, ns=1))[0] for r in rows])
    assert oracle.rel_l2(got, ref) < TOL_BF16X3


@pytest.mark.parametrize("P,T,dt,rows", [(4096, 16, synth.IN_C64, 8 * 5 + 3), (2048, 8, synth.IN_CI8, 8 * 9 + 7),
                                         (4096, 12, synth.IN_R32, 8 * 3), (2048, 16, synth.IN_C64, 5)])
def test_gemm_bf16x3_factored_cluster_parity(P, T, dt, rows):
    """P = 2048 / 4096: cross-CTA radix-CS step, then the local 1024-point DFT as
    two tensor-core products; several 8-spectrum units with ragged tails."""
    n = P * (T - 1 + rows) + 11
    plan, x, got = _run_variant(1, P, T, dt, n, seed=P + T + rows)
    ref = reference(x, dt, P, T, synth.WIN_HANN)
    assert got.shape == ref.shape == (rows, P)
    e2, em = assert_close(got, ref, TOL_BF16X3, TOL_MAX_BF16X3, what=f"bf16x3 factored P={P} T={T}")
    assert e2 > 1e-8


def test_gemm_bf16x3_factored_c3_sample():
    """c3 (64 streams x 2^20, P = 4096, T = 16, Blackman) as one batched launch on the
    factored tensor-core route: sampled spectra of two streams against the oracle."""
    import torch
    specs = synth.config_c3()
    P, T, win = specs[0].P, specs[0].T, specs[0].window
    plan = pkg.Plan(P, T, pkg.PFB_IN_C64, win, pkg.PFB_DFT_GEMM_BF16X3)
    assert plan.variant == 1
    xs_host = [sp.generate() for sp in specs]
    xs = [to_device(x) for x in xs_host]
    S = plan.out_spectra(xs_host[0].size)
    outs = [torch.empty((S, P), dtype=torch.complex64, device="cuda") for _ in xs]
    pkg.pfb_execute_batch([(plan, x, o) for x, o in zip(xs, outs)])
    torch.cuda.synchronize()
    h = oracle.prototype(P, T, win)
    for i in (0, 41):
        rows = [0, 1, S // 2, S - 1]
        xin = oracle.dequant(xs_host[i], oracle.IN_C64)
        ref = np.stack([oracle.dft(oracle.fir(xin, P, T, h, s0=r, ns=1))[0] for r in rows])
        assert oracle.rel_l2(outs[i][rows].cpu().numpy(), ref) < TOL_BF16X3


@pytest.mark.parametrize("P,T,dt,rows", [(4096, 16, synth.IN_C64, 1001), (2048, 4, synth.IN_CI8, 301),
                                         (4096, 8, synth.IN_R32, 37)])
def test_gemm_bf16x3_ws_cluster_repeatable_and_matches_split_model(P, T, dt, rows):
    """The warp-specialised cluster kernel with its local DFT on the tensor cores:
    against the oracle, and bitwise repeatable over several runs at scale."""
    import torch
    n = P * (T - 1 + rows) + 3
    x = synth.small_stream(P, T, n, in_dtype=dt, seed=P * T + rows).generate()
    plan = pkg.Plan(P, T, dt, pkg.PFB_WIN_BLACKMAN, pkg.PFB_DFT_GEMM_BF16X3)
    assert plan.variant == 1
    xd = to_device(x)
    first = plan.execute(xd).clone()
    for _ in range(3):
        assert torch.equal(plan.execute(xd), first)
    ref = reference(x, dt, P, T, synth.WIN_BLACKMAN)
    assert_close(first.cpu().numpy(), ref, TOL_BF16X3, TOL_MAX_BF16X3, what=f"ws cluster tc P={P} T={T}")


def test_gemm_bf16x3_factored_p4096_batch_equals_single():
    """P = 4096 (the four-step 64 x 64 cluster kernel with its 16-point DFT steps
    on the tensor cores): uneven streams, one with no spectrum and one with a
    single spectrum (partial batches), in one launch equal to per-stream
    launches, and bitwise repeatable."""
    import torch
    P, T = 4096, 16
    plan = pkg.Plan(P, T, pkg.PFB_IN_C64, pkg.PFB_WIN_HAMMING, pkg.PFB_DFT_GEMM_BF16X3)
    assert plan.variant == 1
    lens = [P * 20 + 3, P * 3, P * 16, P * 97 + 11, P * 300, P * 41]
    xs = [to_device(synth.small_stream(P, T, n, seed=90 + i).generate()) for i, n in enumerate(lens)]
    singles = [plan.execute(x).clone() if plan.out_spectra(x.numel()) > 0 else None for x in xs]
    outs = [torch.full((max(plan.out_spectra(x.numel()), 1), P), 5.0, dtype=torch.complex64, device="cuda") for x in xs]
    for _ in range(3):
        pkg.pfb_execute_batch([(plan, x, o) for x, o in zip(xs, outs)])
        torch.cuda.synchronize()
        for sgl, o in zip(singles, outs):
            if sgl is not None:
                assert torch.equal(o[:sgl.shape[0]], sgl)
            else:
                assert torch.all(o == 5.0)
    assert plan.status() == pkg.PFB_OK
    x4 = synth.small_stream(P, T, lens[4], seed=94).generate()
    ref = reference(x4, synth.IN_C64, P, T, synth.WIN_HAMMING, s0=100, ns=5)
    assert_close(outs[4][100:105].cpu().numpy(), ref, TOL_BF16X3, TOL_MAX_BF16X3, what="factored P=4096 batch")


# ---------------------------------------------------------------------------
# dense product in two passes, variant 2 (FIR to a pre-tiled workspace, then a
# pipelined tcgen05 GEMM with double-buffered TMEM accumulators)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("P,T,dt,rows", [(1024, 16, synth.IN_C64, 128 * 2 + 45), (2048, 8, synth.IN_CI8, 128 + 1),
                                         (4096, 16, synth.IN_C64, 127), (4096, 4, synth.IN_R32, 129),
                                         (1024, 12, synth.IN_C64, 3)])
def test_gemm_bf16x3_two_pass_parity(P, T, dt, rows):
    """Ragged last M tiles (S not a multiple of 128), every input type, T
    padded to its compiled tap count (T = 12 runs with TT = 16)."""
    n = P * (T - 1 + rows) + 7
    plan, x, got = _run_variant(2, P, T, dt, n, seed=P + 3 * T + rows)
    assert plan.variant == 2
    ref = reference(x, dt, P, T, synth.WIN_HANN)
    assert got.shape == ref.shape
    e2, em = assert_close(got, ref, TOL_BF16X3, TOL_MAX_BF16X3, what=f"bf16x3 two-pass P={P} T={T} rows={rows}")
    assert e2 > 1e-8
    assert plan.status() == pkg.PFB_OK


def test_gemm_bf16x3_two_pass_matches_split_model_and_dense():
    """Against the FP64 model of the split arithmetic (indexing errors would be
    O(1)), and against the fused dense variant 0 (same products, same chunked
    accumulation: the two agree to the accumulation error)."""
    P, T = 1024, 16
    n = P * (T - 1 + 300)
    plan, x, got = _run_variant(2, P, T, synth.IN_C64, n, seed=21)
    h = oracle.prototype(P, T, oracle.WIN_HANN)
    y = oracle.fir(oracle.dequant(x, oracle.IN_C64), P, T, h)
    model = split_bf16x3_model(y.astype(np.complex64), P)
    assert oracle.rel_l2(got, model) < 3e-6
    plan0, _, got0 = _run_variant(0, P, T, synth.IN_C64, n, seed=21)
    assert oracle.rel_l2(got, got0) < 3e-6


def test_gemm_bf16x3_two_pass_batch_repeatable():
    """Uneven streams (one with 0 spectra, one of a single spectrum) in one
    batched launch: equal to per-stream launches, bitwise repeatable, and the
    workspace grows between calls of different sizes."""
    import torch
    P, T = 4096, 16
    plan = pkg.Plan(P, T, pkg.PFB_IN_C64, pkg.PFB_WIN_BLACKMAN, pkg.PFB_DFT_GEMM_BF16X3)
    plan.variant = 2
    lens = [P * (T - 1 + 200) + 3, P * 3, P * (T - 1 + 1), P * (T - 1 + 257)]
    xs = [to_device(synth.small_stream(P, T, n, seed=40 + i).generate()) for i, n in enumerate(lens)]
    singles = [plan.execute(x).clone() if plan.out_spectra(x.numel()) > 0 else None for x in xs]
    outs = [torch.full((max(plan.out_spectra(x.numel()), 1), P), 7.0, dtype=torch.complex64, device="cuda") for x in xs]
    for _ in range(3):
        pkg.pfb_execute_batch([(plan, x, o) for x, o in zip(xs, outs)])
        torch.cuda.synchronize()
        for s, o in zip(singles, outs):
            if s is not None:
                assert torch.equal(o[:s.shape[0]], s)
            else:
                assert torch.all(o == 7.0)
    assert plan.status() == pkg.PFB_OK
    x3 = synth.small_stream(P, T, lens[3], seed=43).generate()
    ref = reference(x3, synth.IN_C64, P, T, synth.WIN_BLACKMAN, s0=250, ns=7)
    assert_close(outs[3][250:257].cpu().numpy(), ref, TOL_BF16X3, TOL_MAX_BF16X3, what="two-pass batch stream 3")


def test_gemm_bf16x3_two_pass_unsupported():
    plan = pkg.Plan(512, 16, pkg.PFB_IN_C64, pkg.PFB_WIN_HANN, pkg.PFB_DFT_GEMM_BF16X3)
    assert plan.num_variants == 3
    with pytest.raises(pkg.PFBError):
        plan.variant = 2


@pytest.mark.parametrize("path,P,variant", [(pkg.PFB_DFT_GEMM_F32, 256, None), (pkg.PFB_DFT_GEMM_F32, 1024, None),
                                            (pkg.PFB_DFT_GEMM_BF16X3, 1024, 2)])
def test_two_pass_products_in_a_graph_on_fresh_plans(path, P, variant):
    """The two-pass products keep a plan-owned workspace; pfb_batch_create
    grows it before capturing, so a graph of fresh plans (never launched)
    works, and its replays equal per-stream launches bit for bit."""
    import torch
    T = 16
    plan = pkg.Plan(P, T, pkg.PFB_IN_C64, pkg.PFB_WIN_HAMMING, path)
    if variant is not None:
        plan.variant = variant
    lens = [P * (T - 1 + 300) + 5, P * (T - 1 + 1), P * 4, P * (T - 1 + 129)]
    hs = [synth.small_stream(P, T, n, seed=70 + i).generate() for i, n in enumerate(lens)]
    xs = [to_device(h) for h in hs]
    outs = [torch.full((max(plan.out_spectra(x.numel()), 1), P), 7.0, dtype=torch.complex64, device="cuda") for x in xs]
    batch = pkg.Batch([(plan, x, o) for x, o in zip(xs, outs)])
    for _ in range(2):
        batch.launch()
    torch.cuda.synchronize()
    assert plan.status() == pkg.PFB_OK
    for x, o in zip(xs, outs):
        S = plan.out_spectra(x.numel())
        if S == 0:
            assert torch.all(o == 7.0)
            continue
        assert torch.equal(o[:S], plan.execute(x))
    tol = (TOL_BF16X3, TOL_MAX_BF16X3) if path == pkg.PFB_DFT_GEMM_BF16X3 else (2e-6, 2e-5)
    assert_close(outs[0][140:146].cpu().numpy(), reference(hs[0], synth.IN_C64, P, T, synth.WIN_HAMMING, s0=140, ns=6),
                 *tol, what=f"graph of a fresh plan, path {path}, P={P}")
    # a larger launch outgrows the workspace; the graph keeps using the buffer it captured
    big = to_device(synth.small_stream(P, T, P * (T - 1 + 1500), seed=79).generate())
    plan.execute(big)
    want = [o.clone() for o in outs]
    for o in outs:
        o.fill_(7.0)
    batch.launch()
    torch.cuda.synchronize()
    assert plan.status() == pkg.PFB_OK
    for o, w in zip(outs, want):
        assert torch.equal(o, w)
    batch.close()
    plan.close()


@pytest.mark.timeout(300)
@pytest.mark.parametrize("path,P,variant", [(pkg.PFB_DFT_GEMM_F32, 256, None), (pkg.PFB_DFT_GEMM_BF16X3, 1024, 2)])
def test_two_pass_products_through_the_host_entry_points(path, P, variant):
    """pfb_execute_host and pfb_execute_batch_host on plans whose launches grow
    the plan's workspace (the host call holds the plan's staging lock while it
    launches): results equal the device path bit for bit."""
    T = 16

    def make():
        p = pkg.Plan(P, T, pkg.PFB_IN_C64, pkg.PFB_WIN_HAMMING, path)
        if variant is not None:
            p.variant = variant
        return p

    plan = make()
    x = synth.small_stream(P, T, P * (T - 1 + 700) + 9, seed=P + 5).generate()
    want = plan.execute(to_device(x)).cpu().numpy()
    plan2 = make()   # fresh: its workspace grows inside the host call
    got = plan2.execute_host(x)
    assert np.array_equal(got, want)
    out = np.zeros_like(want)
    plan3 = make()
    pkg.pfb_execute_batch_host([(plan3, x, out)])
    assert np.array_equal(out, want)
    for p in (plan, plan2, plan3):
        assert p.status() == pkg.PFB_OK
        p.close()
