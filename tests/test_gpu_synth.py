"""Parity of the synthesis (inverse) filter bank with the FP64 oracle, through
the C ABI: every supported P and tap count, both tap orders, a ragged number
of spectra, sampled frames at scale, and the adjoint relation with the
analysis kernels."""

import numpy as np
import pytest

import oracle
import paper_2408_16551_gb300 as pkg
from paper_2408_16551_gb300 import synth

from gpu_common import TOL_F32, TOL_MAX_F32, assert_close, to_device

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2408_16551_gb300 import build
    build.build()
    torch.cuda.set_device(0)


def _spectra(S, P, seed):
    rng = np.random.default_rng(seed)
    return (rng.standard_normal((S, P)) + 1j * rng.standard_normal((S, P))).astype(np.complex64)


def _taps(P, T, window, rev):
    h = oracle.prototype(P, T, window)
    return h.reshape(T, P)[::-1].reshape(-1) if rev else h


@pytest.mark.parametrize("P,T,S,rev", [(1024, 16, 37, 0), (1024, 8, 5, 1), (1024, 4, 1, 0), (512, 16, 61, 1),
                                       (512, 4, 9, 0), (1024, 3, 7, 0), (512, 12, 23, 1), (1024, 16, 300, 0)])
def test_synthesis_matches_oracle(P, T, S, rev):
    import torch
    X = _spectra(S, P, P + T + S)
    plan = pkg.Plan(P, T, pkg.PFB_IN_C64, pkg.PFB_WIN_HAMMING,
                    tap_order=pkg.PFB_TAPS_CONVOLUTION if rev else pkg.PFB_TAPS_CORRELATION)
    assert plan.synth_out_samples(S) == (S + T - 1) * P
    xh = plan.synthesize(to_device(X))
    torch.cuda.synchronize()
    ref = oracle.synth(X.astype(np.complex128), P, T, _taps(P, T, synth.WIN_HAMMING, rev))
    assert xh.shape[0] == ref.size
    assert_close(xh.cpu().numpy(), ref, TOL_F32, TOL_MAX_F32, what=f"synthesis P={P} T={T} S={S} rev={rev}")


def test_synthesis_at_scale_sampled_frames_and_repeatable():
    """16369 spectra of P = 1024 (the c2 analysis output size): sampled frames
    against the oracle, the whole output bitwise repeatable."""
    import torch
    P, T, S = 1024, 16, 16369
    X = _spectra(S, P, 4)
    plan = pkg.Plan(P, T, pkg.PFB_IN_C64, pkg.PFB_WIN_HAMMING)
    Xd = to_device(X)
    xh = plan.synthesize(Xd)
    again = plan.synthesize(Xd)
    torch.cuda.synchronize()
    assert torch.equal(xh, again)
    h = oracle.prototype(P, T, synth.WIN_HAMMING)
    frames = [0, 1, 14, 15, 16, 5000, S - 1, S, S + T - 2]
    got = np.concatenate([xh[f * P:(f + 1) * P].cpu().numpy() for f in frames])
    ref = np.concatenate([oracle.synth(X.astype(np.complex128), P, T, h, f0=f, nf=1) for f in frames])
    assert_close(got, ref, TOL_F32, TOL_MAX_F32, what="synthesis sampled frames")


@pytest.mark.parametrize("P,T", [(1024, 16), (512, 8)])
def test_synthesis_is_the_adjoint_of_the_analysis_kernel(P, T):
    """<A x, Y> = P <x, synth(Y)> with both sides computed by the library's
    kernels (analysis pfb_execute, synthesis pfb_synthesize)."""
    import torch
    S = 50
    rng = np.random.default_rng(P + T)
    x = (rng.standard_normal((S + T - 1) * P) + 1j * rng.standard_normal((S + T - 1) * P)).astype(np.complex64)
    Y = _spectra(S, P, 8)
    plan = pkg.Plan(P, T, pkg.PFB_IN_C64, pkg.PFB_WIN_BLACKMAN)
    Ax = plan.execute(to_device(x)).cpu().numpy().astype(np.complex128)
    Sy = plan.synthesize(to_device(Y)).cpu().numpy().astype(np.complex128)
    lhs = np.vdot(Ax, Y.astype(np.complex128))
    rhs = P * np.vdot(x.astype(np.complex128), Sy)
    assert abs(lhs - rhs) <= 1e-5 * np.linalg.norm(Ax) * np.linalg.norm(Y)


def test_synthesis_rejects_unsupported_plans():
    import torch
    X = to_device(_spectra(4, 64, 1))
    with pytest.raises(pkg.PFBError) as e:
        pkg.Plan(64, 8, path=pkg.PFB_DFT_GEMM_BF16X3).synthesize(X)   # no split-bf16 kernel below P = 128
    assert e.value.status == pkg.PFB_ERR_UNSUPPORTED
    X = to_device(_spectra(4, 1024, 1))
    with pytest.raises(pkg.PFBError) as e:
        pkg.Plan(1024, 16, hop=512).synthesize(X)
    assert e.value.status == pkg.PFB_ERR_UNSUPPORTED
    plan = pkg.Plan(1024, 16)
    small = torch.empty(100, dtype=torch.complex64, device="cuda")
    with pytest.raises(pkg.PFBError) as e:
        plan.synthesize(X, out=small)
    assert e.value.status == pkg.PFB_ERR_INVALID
    assert plan.synth_out_samples(0) == 0


# the routes other than the fused kernel: the FP32 inverse FFT or the split-bf16
# product with the conjugate DFT matrix, then the adjoint per-branch FIR
GENERIC = [(4096, 16, pkg.PFB_DFT_FFT_F32, 29, 0), (2048, 8, pkg.PFB_DFT_FFT_F32, 13, 1),
           (16, 4, pkg.PFB_DFT_FFT_F32, 40, 0), (4, 1, pkg.PFB_DFT_FFT_F32, 9, 0),
           (256, 40, pkg.PFB_DFT_FFT_F32, 50, 1), (1024, 64, pkg.PFB_DFT_FFT_F32, 3, 0),
           (256, 8, pkg.PFB_DFT_FFT_F32, 33, 0), (64, 3, pkg.PFB_DFT_GEMM_F32, 17, 0),
           (1024, 16, pkg.PFB_DFT_GEMM_F32, 5, 1), (1024, 16, pkg.PFB_DFT_GEMM_BF16X3, 37, 0),
           (4096, 16, pkg.PFB_DFT_GEMM_BF16X3, 21, 1), (256, 5, pkg.PFB_DFT_GEMM_BF16X3, 130, 0),
           (128, 16, pkg.PFB_DFT_GEMM_BF16X3, 7, 0), (2048, 30, pkg.PFB_DFT_GEMM_BF16X3, 4, 0)]


@pytest.mark.parametrize("P,T,path,S,rev", GENERIC)
def test_synthesis_routes_match_oracle(P, T, path, S, rev):
    """Every P, T up to 64 and every DFT path at hop P: the FP32 routes at the
    FP32 bound, the split-bf16 route (tensor-core product with the conjugate
    DFT matrix) at the split-bf16 bound, and bitwise repeatable."""
    import torch
    from gpu_common import TOL_BF16X3, TOL_MAX_BF16X3
    X = _spectra(S, P, P + T + S)
    plan = pkg.Plan(P, T, pkg.PFB_IN_C64, pkg.PFB_WIN_HANN, path,
                    tap_order=pkg.PFB_TAPS_CONVOLUTION if rev else pkg.PFB_TAPS_CORRELATION)
    Xd = to_device(X)
    xh = plan.synthesize(Xd)
    again = plan.synthesize(Xd)
    torch.cuda.synchronize()
    assert torch.equal(xh, again)
    assert plan.status() == pkg.PFB_OK
    ref = oracle.synth(X.astype(np.complex128), P, T, _taps(P, T, synth.WIN_HANN, rev))
    tol = (TOL_BF16X3, TOL_MAX_BF16X3) if path == pkg.PFB_DFT_GEMM_BF16X3 else (TOL_F32, TOL_MAX_F32)
    e2, _ = assert_close(xh.cpu().numpy(), ref, *tol, what=f"synthesis P={P} T={T} path={path} rev={rev}")
    if path == pkg.PFB_DFT_GEMM_BF16X3:
        assert e2 > 1e-8  # the split arithmetic really ran


@pytest.mark.parametrize("P,T,path", [(4096, 16, pkg.PFB_DFT_FFT_F32), (2048, 12, pkg.PFB_DFT_FFT_F32),
                                      (1024, 16, pkg.PFB_DFT_GEMM_BF16X3)])
def test_synthesis_routes_are_the_adjoint_of_the_analysis(P, T, path):
    """<A x, Y> = P <x, synth(Y)> with the analysis kernel of the same plan."""
    S = 40
    rng = np.random.default_rng(P + T + path)
    x = (rng.standard_normal((S + T - 1) * P) + 1j * rng.standard_normal((S + T - 1) * P)).astype(np.complex64)
    Y = _spectra(S, P, 9)
    plan = pkg.Plan(P, T, pkg.PFB_IN_C64, pkg.PFB_WIN_BLACKMAN, path)
    Ax = plan.execute(to_device(x)).cpu().numpy().astype(np.complex128)
    Sy = plan.synthesize(to_device(Y)).cpu().numpy().astype(np.complex128)
    lhs = np.vdot(Ax, Y.astype(np.complex128))
    rhs = P * np.vdot(x.astype(np.complex128), Sy)
    tol = 1e-4 if path == pkg.PFB_DFT_GEMM_BF16X3 else 1e-5
    assert abs(lhs - rhs) <= tol * np.linalg.norm(Ax) * np.linalg.norm(Y)
