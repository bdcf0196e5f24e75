"""One stream past 2 GiB of input and of spectra (GPU).

A complex64 stream of 2^28 + 40 * 4096 samples is 2 GiB of input; at
P = 4096 it gives 65,561 spectra and at P = 1024 262,169, so the last rows of
the output start past byte 2^31 too.  Every byte offset of the loaders, the
ring producers, the workspaces and the output stores has to be 64-bit.  The kernels that
channelise such a stream are run on it whole and compared with the FP64
oracle on sampled rows: the first, the middle, the last, the first output
row past byte 2^31 and the rows whose input frames cross byte 2^31."""

import numpy as np
import pytest

import paper_2408_16551_gb300 as pkg
from paper_2408_16551_gb300 import synth

from gpu_common import TOL_BF16X3, TOL_F32, TOL_MAX_BF16X3, TOL_MAX_F32, assert_close, reference

pytestmark = pytest.mark.gpu

N_SAMPLES = (1 << 28) + 40 * 4096
T = 16


@pytest.fixture(scope="module")
def big():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2408_16551_gb300 import build
    build.build()
    torch.cuda.set_device(0)
    rng = np.random.default_rng(91)
    spec = synth.StreamSpec(P=4096, T=T, window=synth.WIN_BLACKMAN, in_dtype=synth.IN_C64,
                            n_samples=N_SAMPLES, seed=9100, tones=synth.random_tones(rng, 4096, 2))
    x = spec.generate()
    xd = torch.from_numpy(x).cuda()
    yield x, xd
    del xd
    torch.cuda.empty_cache()


def _rows(P, S):
    row_bytes = P * 8
    out_cross = -(-(1 << 31) // row_bytes)            # first output row starting at or past byte 2^31
    in_cross = (1 << 31) // row_bytes                 # the input frame holding byte 2^31
    rows = {0, S // 2, S - 2, S - 1, out_cross, in_cross - T + 1, in_cross - 3, in_cross}
    return sorted(r for r in rows if 0 <= r < S)


@pytest.mark.parametrize("P, path, variant, tol", [
    (4096, pkg.PFB_DFT_FFT_F32, None, (TOL_F32, TOL_MAX_F32)),         # four-step cluster kernel
    (1024, pkg.PFB_DFT_FFT_F32, None, (TOL_F32, TOL_MAX_F32)),         # warp-specialised single-CTA kernel
    (4096, pkg.PFB_DFT_GEMM_BF16X3, None, (TOL_BF16X3, TOL_MAX_BF16X3)),  # factored tensor-core DFT
    (4096, pkg.PFB_DFT_GEMM_BF16X3, 2, (TOL_BF16X3, TOL_MAX_BF16X3)),     # FIR pass + dense GEMM
    (4096, pkg.PFB_DFT_GEMM_F32, None, (TOL_F32, TOL_MAX_F32)),           # FIR pass + FP32 SIMT GEMM
])
def test_stream_past_2gib(big, P, path, variant, tol):
    import torch
    x, xd = big
    plan = pkg.Plan(P, T, pkg.PFB_IN_C64, pkg.PFB_WIN_BLACKMAN, path)
    if variant is not None:
        plan.variant = variant
    S = plan.out_spectra(N_SAMPLES)
    assert (S - 1) * P * 8 >= (1 << 31) and x.nbytes >= (1 << 31)
    out = torch.empty((S, P), dtype=torch.complex64, device="cuda")
    out.view(torch.float32).fill_(float("nan"))
    plan.execute(xd, out)
    torch.cuda.synchronize()
    assert plan.status() == pkg.PFB_OK
    rows = _rows(P, S)
    got = out[rows].cpu().numpy()
    ref = np.stack([reference(x[r * P:(r + T) * P], pkg.PFB_IN_C64, P, T, synth.WIN_BLACKMAN, s0=0, ns=1)[0]
                    for r in rows])
    # the tolerance is over all checked outputs of the case, as in the other parity tests
    assert_close(got, ref, *tol, what=f"P={P} path={path} variant={plan.variant} rows {rows}")
    # every spectrum was written (no NaN left from the fill)
    assert not bool(torch.isnan(out.view(torch.float32)).any())
    del out
    plan.close()
