"""Shared helpers of the GPU parity tests (inputs from the seeded generators,
expected values from the FP64 oracle only)."""

import numpy as np

import oracle
from paper_2408_16551_gb300 import synth

# tolerances (relative L2 error vs the FP64 oracle over all outputs of a case)
TOL_F32 = 2e-6
TOL_BF16X3 = 1e-5
# max |error| / max |X_ref| guard against a few badly wrong bins hiding in the L2 norm
TOL_MAX_F32 = 2e-5
TOL_MAX_BF16X3 = 1e-4

TORCH_DTYPE = {synth.IN_R32: "float32", synth.IN_C64: "complex64", synth.IN_CI8: "int8"}


def to_device(x: np.ndarray):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def reference(x: np.ndarray, in_dtype: int, P: int, T: int, window: int, scale: float = 1.0, s0: int = 0,
              ns=None, user_taps=None):
    h = oracle.prototype(P, T, window, user_taps=user_taps)
    return oracle.pfb_input(x, in_dtype, P, T, h, scale=scale, s0=s0, ns=ns)


def max_rel(got, ref):
    den = np.max(np.abs(ref))
    return float(np.max(np.abs(got - ref)) / den) if den > 0 else float(np.max(np.abs(got)))


def assert_close(got, ref, tol_l2=TOL_F32, tol_max=TOL_MAX_F32, what=""):
    assert got.shape == ref.shape, (what, got.shape, ref.shape)
    e2 = oracle.rel_l2(got, ref)
    em = max_rel(got, ref)
    assert e2 <= tol_l2 and em <= tol_max, f"{what}: rel_l2={e2:.3e} (tol {tol_l2}) max_rel={em:.3e} (tol {tol_max})"
    return e2, em


def reference_hop(x: np.ndarray, in_dtype: int, P: int, T: int, window: int, D: int, reverse: bool = False,
                  scale: float = 1.0, s0: int = 0, ns=None):
    """Oracle output of the channeliser with hop D and tap order (reverse = convolution order)."""
    h = oracle.prototype(P, T, window)
    return oracle.pfb_hop(oracle.dequant(x, in_dtype, scale), P, T, h, D, reverse=reverse, s0=s0, ns=ns)
