"""Pins of the FP64 split-bf16 models in ``tests/split_models.py`` (CPU).

The models are test helpers, not the oracle: the GPU tests compare the
tensor-core routes with the oracle at the 1e-5 bound, and with these models
to separate split error from indexing.  The pins below tie the models to
things that do not come from them: torch's bf16 conversion, numpy.fft, and
exact arithmetic on inputs whose splits are exact.
"""

import numpy as np
import pytest

import oracle
from split_models import bf16_round, dft_block_matrix, factored_dft_model, split_bf16x3_model


def _ints(rng, shape, bits):
    """Complex values whose real and imaginary parts are integers below
    2^bits in magnitude, scaled by a power of two (exact in FP64)."""
    lim = 1 << bits
    re = rng.integers(-lim + 1, lim, size=shape).astype(np.float64)
    im = rng.integers(-lim + 1, lim, size=shape).astype(np.float64)
    return (re + 1j * im) * 2.0 ** -7


def test_bf16_round_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(21)
    v = (rng.standard_normal(20000) * 10.0 ** rng.uniform(-6, 6, 20000)).astype(np.float32)
    v = np.concatenate([v, np.float32([1.0, -1.0, 1.00390625, 1.005859375, 0.0])])  # exact and halfway cases
    ref = torch.from_numpy(v).to(torch.bfloat16).to(torch.float64).numpy()
    got = bf16_round(v.astype(np.float64))
    assert np.array_equal(got, ref)


@pytest.mark.parametrize("P", [4, 16, 64])
def test_dft_block_matrix_reproduces_dft(P):
    rng = np.random.default_rng(P)
    y = rng.standard_normal((5, P)) + 1j * rng.standard_normal((5, P))
    A = np.empty((5, 2 * P)); A[:, 0::2] = y.real; A[:, 1::2] = y.imag
    Xr = A @ dft_block_matrix(P)
    X = Xr[:, 0::2] + 1j * Xr[:, 1::2]
    assert np.max(np.abs(X - np.fft.fft(y, axis=1))) < 1e-12


def test_split_model_exact_when_the_splits_are_exact():
    """P = 4: the DFT matrix holds only 0 and +-1 (bf16-exact up to the
    1e-16 residues of cos(pi/2) and sin(pi) in FP64), and inputs of at most 16
    significant bits split exactly into hi + lo.  The three-product model must
    then reproduce numpy.fft to FP64 rounding: a lost lo*hi term (an error of
    about 2^-9 of the result), a transposed operand or a wrong interleave fails."""
    rng = np.random.default_rng(5)
    y = _ints(rng, (12, 4), 16).astype(np.complex64)
    assert np.array_equal(y.astype(np.complex128), _ints(np.random.default_rng(5), (12, 4), 16))  # exact in fp32
    X = split_bf16x3_model(y, 4)
    ref = np.fft.fft(y.astype(np.complex128), axis=1)
    assert np.max(np.abs(X - ref)) <= 1e-13 * np.max(np.abs(ref))


def test_split_model_without_the_lo_terms_is_not_exact():
    """The same inputs with more than 8 significant bits need their lo parts:
    a model that kept only hi*hi would differ from numpy.fft (this guards the
    exactness pin above against inputs that make lo vanish)."""
    rng = np.random.default_rng(6)
    y = _ints(rng, (12, 4), 16)
    hi = bf16_round(y.real) + 1j * bf16_round(y.imag)
    assert np.max(np.abs(y - hi)) > 0
    assert not np.array_equal(np.fft.fft(hi, axis=1), np.fft.fft(y, axis=1))


def test_split_model_error_is_small_but_nonzero():
    P = 64
    rng = np.random.default_rng(3)
    y = (rng.standard_normal((8, P)) + 1j * rng.standard_normal((8, P))).astype(np.complex64)
    X = split_bf16x3_model(y, P)
    ref = np.fft.fft(y.astype(np.complex128), axis=1)
    e = oracle.rel_l2(X, ref)
    assert 1e-7 < e < 1e-5


@pytest.mark.parametrize("P1,P2", [(4, 4), (2, 8), (8, 2), (32, 32), (16, 4)])
def test_factored_dft_model_unsplit_is_the_dft(P1, P2):
    """Four-step factoring (p = P2 n1 + n2, k = k1 + P1 k2, twiddle w_P^(n2 k1))
    against numpy.fft: a wrong index role, twiddle sign or output order fails."""
    rng = np.random.default_rng(P1 * 100 + P2)
    y = rng.standard_normal((6, P1 * P2)) + 1j * rng.standard_normal((6, P1 * P2))
    ref = np.fft.fft(y, axis=1)
    got = factored_dft_model(y, P1, P2, split=False)
    assert np.max(np.abs(got - ref)) < 1e-12 * np.max(np.abs(ref))


def test_factored_split_model_exact_when_the_splits_are_exact():
    """P = 2 x 2: both 2-point DFT matrices and the twiddles w_4^(n2 k1) are
    0, +-1, +-i (bf16-exact); inputs of at most 14 bits split exactly, and so
    does the twiddled intermediate Z (at most 15 bits, exact in fp32).  The
    split model must then equal numpy.fft to FP64 rounding (the cos/sin of
    multiples of pi/2 carry 1e-16 residues), which pins its operand roles,
    the hi/lo composition of both products and the twiddle."""
    rng = np.random.default_rng(7)
    y = _ints(rng, (10, 4), 14)
    got = factored_dft_model(y.astype(np.complex64), 2, 2, split=True)
    ref = np.fft.fft(y, axis=1)
    assert np.max(np.abs(got - ref)) <= 1e-13 * np.max(np.abs(ref))


def test_factored_dft_model_split_error_is_bounded():
    """Split-bf16 four-step model at P = 32 x 32: error at the split level (two
    products of hi/lo operands), inside the 1e-5 bound, and not zero."""
    rng = np.random.default_rng(31)
    y = (rng.standard_normal((6, 1024)) + 1j * rng.standard_normal((6, 1024))).astype(np.complex64)
    e = oracle.rel_l2(factored_dft_model(y, 32, 32), np.fft.fft(y.astype(np.complex128), axis=1))
    assert 1e-7 < e < 1e-5
