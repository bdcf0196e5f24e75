"""The stream-sharded launchers on one GPU, ranks run one after another (no
rank waits on another): dealing a batch's streams to ranks, or cutting one
long stream into spectrum ranges with their halo, gives the same spectra as
the unsharded call, bit for bit (each spectrum's arithmetic does not depend on
which launch or CTA computes it)."""

import pytest

import paper_2408_16551_gb300 as pkg
from paper_2408_16551_gb300 import replicas, synth

from gpu_common import assert_close, reference, reference_hop

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2408_16551_gb300 import build
    build.build()
    torch.cuda.set_device(0)


def _uneven_batch(n_streams, cap):
    """Streams with the uneven P / T / length mix of the batched workload, lengths capped."""
    import torch
    plans, entries = {}, []
    for spec in synth.config_c4(n_streams):
        spec.n_samples = min(spec.n_samples, cap)
        key = (spec.P, spec.T, spec.window)
        if key not in plans:
            plans[key] = pkg.Plan(spec.P, spec.T, pkg.PFB_IN_C64, spec.window, pkg.PFB_DFT_FFT_F32)
        plan = plans[key]
        x = torch.from_numpy(spec.generate()).cuda()
        S = plan.out_spectra(x.numel())
        out = torch.full((max(S, 1), spec.P), float("nan"), dtype=torch.complex64, device="cuda")
        entries.append((plan, x, out))
    return plans, entries


@pytest.mark.parametrize("world", [2, 3, 5])
def test_sharded_batch_equals_whole(world):
    import torch
    plans, entries = _uneven_batch(24, 1 << 18)
    pkg.pfb_execute_batch(entries)
    torch.cuda.synchronize()
    whole = [out.clone() for _, _, out in entries]
    for _, _, out in entries:
        out.fill_(float("nan"))
    ran = []
    for rank in range(world):
        ran += replicas.execute_sharded_batch(entries, rank, world)
    torch.cuda.synchronize()
    assert sorted(ran) == list(range(len(entries)))
    for (plan, x, out), ref in zip(entries, whole):
        S = plan.out_spectra(x.numel())
        assert torch.equal(out[:S], ref[:S])
    # one stream against the oracle, so the comparison above is not between two wrong answers
    plan, x, out = max(entries, key=lambda e: e[0].out_spectra(e[1].numel()))
    S = plan.out_spectra(x.numel())
    got = out[:S].cpu().numpy()
    assert_close(got, reference(x.cpu().numpy(), pkg.PFB_IN_C64, plan.P, plan.T, plan.window),
                 what="sharded batch stream")


@pytest.mark.parametrize("P,T,in_dtype,hop,world", [
    (1024, 16, pkg.PFB_IN_C64, 0, 3),       # the fused FIR + FFT kernel, c2 shape
    (1024, 16, pkg.PFB_IN_C64, 512, 4),     # oversampled by 2
    (4096, 16, pkg.PFB_IN_C64, 0, 2),       # cluster kernel
    (16, 4, pkg.PFB_IN_R32, 0, 3),
    (4, 3, pkg.PFB_IN_CI8, 0, 3),           # 8-byte frames: shares start on even spectra
])
def test_sharded_stream_equals_whole(P, T, in_dtype, hop, world):
    import torch
    extra = 20 if P >= 4096 else (60 if P >= 1024 else 333)   # keeps the naive-DFT oracle quick
    n = P * (T + extra) + P // 2 + 1
    spec = synth.small_stream(P, T, n, in_dtype=in_dtype, seed=P + T + world)
    xh = spec.generate()
    x = torch.from_numpy(xh).cuda()
    plan = pkg.Plan(P, T, in_dtype, synth.WIN_HAMMING, pkg.PFB_DFT_FFT_F32, hop=hop)
    whole = plan.execute(x)
    torch.cuda.synchronize()
    S = whole.shape[0]
    out = torch.full((S, P), float("nan"), dtype=torch.complex64, device="cuda")
    cover = []
    for rank in range(world):
        s0, s1 = replicas.execute_sharded_stream(plan, x, out, rank, world)
        cover.append((s0, s1))
    torch.cuda.synchronize()
    assert cover[0][0] == 0 and cover[-1][1] == S
    assert all(cover[i][1] == cover[i + 1][0] for i in range(world - 1))
    assert torch.equal(out, whole)
    # and the whole stream against the oracle
    ref = reference_hop(xh, in_dtype, P, T, synth.WIN_HAMMING, hop or P)
    assert_close(out.cpu().numpy(), ref, what=f"sharded stream P={P} hop={hop}")
