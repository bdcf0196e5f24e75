"""FP64 models of the split-bf16 tensor-core DFT arithmetic -- test helpers.

These are not part of the oracle (``oracle/`` holds only the paper's
definition of the channeliser).  They model, in FP64 NumPy, what the
tensor-core routes compute with bf16 hi/lo operands (hi = RN_bf16(v),
lo = RN_bf16(v - hi), three products hi*hi + hi*lo + lo*hi), so that a GPU
test can separate the error of the split arithmetic from an indexing bug.
They are pinned by ``tests/test_split_models.py``.  Nothing here is used by
the library.
"""

from __future__ import annotations

import numpy as np


def bf16_round(v) -> np.ndarray:
    """Round to the nearest bfloat16 value (8 significant bits, ties to even), in float64."""
    v = np.asarray(v, dtype=np.float64)
    m, e = np.frexp(v)                      # v = m 2^e, |m| in [0.5, 1)
    return np.ldexp(np.round(m * 256.0), e - 8)


def dft_block_matrix(P: int) -> np.ndarray:
    """Real block form of the Fourier matrix of Sec. 4.1 on interleaved (re, im)
    rows/columns: B[2p+c, 2k+d] with th = 2 pi (pk mod P)/P:
    B[2p,2k] = B[2p+1,2k+1] = cos th, B[2p+1,2k] = sin th, B[2p,2k+1] = -sin th."""
    p = np.arange(P)[:, None]
    k = np.arange(P)[None, :]
    th = 2.0 * np.pi * ((p * k) % P) / P
    B = np.zeros((2 * P, 2 * P))
    B[0::2, 0::2] = np.cos(th)
    B[1::2, 1::2] = np.cos(th)
    B[1::2, 0::2] = np.sin(th)
    B[0::2, 1::2] = -np.sin(th)
    return B


def split_bf16x3_model(y32: np.ndarray, P: int) -> np.ndarray:
    """X = A_hi (B_hi + B_lo) + A_lo B_hi in FP64, with A = interleaved fp32
    branch sums split into bf16 hi/lo and B split from its FP64 value."""
    A = np.empty((y32.shape[0], 2 * P))
    A[:, 0::2] = np.asarray(y32.real, dtype=np.float32)
    A[:, 1::2] = np.asarray(y32.imag, dtype=np.float32)
    Ah = bf16_round(A)
    Al = bf16_round(A - Ah)
    B = dft_block_matrix(P)
    Bh = bf16_round(B)
    Bl = bf16_round(B - Bh)
    Xr = Ah @ (Bh + Bl) + Al @ Bh
    return Xr[:, 0::2] + 1j * Xr[:, 1::2]


def _dft_matrix(n: int) -> np.ndarray:
    """w_n^(a b) = exp(-2 pi i (a b mod n) / n) (Sec. 4.1 DFT matrix, integer index reduction)."""
    ab = np.outer(np.arange(n), np.arange(n)) % n
    return np.cos(2 * np.pi * ab / n) - 1j * np.sin(2 * np.pi * ab / n)


def factored_dft_model(y: np.ndarray, P1: int, P2: int, split: bool = True) -> np.ndarray:
    """The DFT of Sec. 4.1 in four-step form, P = P1 * P2, p = P2 n1 + n2,
    k = k1 + P1 k2:
        Z[n2, k1]        = sum_{n1} y[P2 n1 + n2] w_P1^(n1 k1)
        X[k1 + P1 k2]    = sum_{n2} Z[n2, k1] w_P^(n2 k1) w_P2^(n2 k2)
    With split=False this is exactly the DFT, a pin on the factoring itself.
    With split=True it models the split-bf16 tensor-core route in FP64: every
    matrix product takes hi = RN_bf16(v), lo = RN_bf16(v - hi) of both operands
    (real and imaginary parts separately) and sums hi*hi + hi*lo + lo*hi; y and
    the twiddled Z are split from their fp32 values, the DFT matrices from FP64."""
    y = np.asarray(y)
    S, P = y.shape
    assert P == P1 * P2

    def sp(v, from32):
        if not split:
            return v, np.zeros_like(v)
        if from32:
            v = v.real.astype(np.float32).astype(np.float64) + 1j * v.imag.astype(np.float32).astype(np.float64)
        hi = bf16_round(v.real) + 1j * bf16_round(v.imag)
        lo = bf16_round(v.real - hi.real) + 1j * bf16_round(v.imag - hi.imag)
        return hi, lo

    def prod(a, b, subs):
        ah, al = a
        bh, bl = b
        r = np.einsum(subs, ah, bh) + np.einsum(subs, ah, bl) + np.einsum(subs, al, bh)
        return r if split else np.einsum(subs, ah, bh)

    Y = y.reshape(S, P1, P2)                                    # [s, n1, n2]
    Z = prod(sp(Y, True), sp(_dft_matrix(P1), False), "sab,ak->sbk")   # [s, n2, k1]
    nk = np.outer(np.arange(P2), np.arange(P1)) % P            # n2 * k1
    Z = Z * (np.cos(2 * np.pi * nk / P) - 1j * np.sin(2 * np.pi * nk / P))[None]
    if split:  # the kernel holds the twiddled Z in fp32 before splitting it
        Z = Z.real.astype(np.float32) + 1j * Z.imag.astype(np.float32)
    X = prod(sp(Z, True), sp(_dft_matrix(P2), False), "sbk,bm->smk")   # [s, k2, k1]
    return X.reshape(S, P)
