"""The DFT factorisations the kernels implement, written out in FP64 NumPy and
checked against numpy.fft (CPU).  They document and pin the index algebra of
each hand-off: a mistake in a twiddle exponent, a bin mapping or a
conjugation shows up here before it reaches a kernel.  (The kernels themselves
are checked against the FP64 oracle by the GPU tests.)"""

import numpy as np
import pytest


def _w(n, e):
    """exp(-2 pi i e / n)"""
    return np.exp(-2j * np.pi * np.asarray(e) / n)


def _rand(n, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal(n) + 1j * rng.standard_normal(n)


@pytest.mark.parametrize("P", [64, 256, 1024])
def test_analysis_radix4_handoff(P):
    """Single-CTA kernel at P = 4Q: FIR thread t holds y[t + Q k], k = 0..3,
    and hands over the radix-4 butterfly with output k1 times w_P^(t k1); the
    FFT warps run four Q-point DFTs; bin 4m + k1 comes from sub-transform k1."""
    Q = P // 4
    y = _rand(P, P)
    t = np.arange(Q)
    yk = [y[t + Q * k] for k in range(4)]
    a0, a1 = yk[0] + yk[2], yk[0] - yk[2]
    a2, a3 = yk[1] + yk[3], yk[1] - yk[3]
    sub = [a0 + a2, (a1 - 1j * a3) * _w(P, t), (a0 - a2) * _w(P, 2 * t), (a1 + 1j * a3) * _w(P, 3 * t)]
    X = np.empty(P, complex)
    for k1 in range(4):
        X[k1::4] = np.fft.fft(sub[k1])
    np.testing.assert_allclose(X, np.fft.fft(y), rtol=0, atol=1e-10 * np.abs(y).sum())


@pytest.mark.parametrize("P", [512, 1024])
def test_synthesis_handoff(P):
    """Synthesis kernel: V_k1 = conj(FFT_Q(conj X[4m + k1])) by the IFFT warps;
    the FIR warps form U_k1[t] = conj(w_P^(t k1)) V_k1[t] and
    y~[t + Q kk] = (1/P) sum_k1 i^(kk k1) U_k1[t], the inverse DFT."""
    Q = P // 4
    X = _rand(P, P + 1)
    t = np.arange(Q)
    U = [np.conj(_w(P, t * k1)) * np.conj(np.fft.fft(np.conj(X[k1::4]))) for k1 in range(4)]
    y = np.empty(P, complex)
    for kk in range(4):
        y[t + Q * kk] = sum((1j ** (kk * k1)) * U[k1] for k1 in range(4)) / P
    np.testing.assert_allclose(y, np.fft.ifft(X), rtol=0, atol=1e-12 * np.abs(X).sum())


@pytest.mark.parametrize("CS", [2, 4])
def test_cluster_four_step(CS):
    """Cluster kernel at P = CS * PL: the cross step forms
    Z_k1[n] = w_P^(n k1) sum_n1 y[PL n1 + n] w_CS^(n1 k1), CTA k1 takes the
    PL-point DFT of Z_k1, and bin k1 + CS k' is its output k'."""
    PL = 256
    P = CS * PL
    y = _rand(P, CS)
    n = np.arange(PL)
    X = np.empty(P, complex)
    for k1 in range(CS):
        Z = _w(P, n * k1) * sum(y[PL * n1 + n] * _w(CS, n1 * k1) for n1 in range(CS))
        X[k1::CS] = np.fft.fft(Z)
    np.testing.assert_allclose(X, np.fft.fft(y), rtol=0, atol=1e-10 * np.abs(y).sum())


def test_tensor_core_factored_dft():
    """Split-bf16 factored DFT at P = 32 x 32 (in exact arithmetic):
    Z[n2][k1] = sum_n1 y[32 n1 + n2] w_32^(n1 k1)   (product 1),
    X[k1 + 32 k2] = sum_n2 Z[n2][k1] w_P^(n2 k1) w_32^(n2 k2)   (twiddle, product 2)."""
    P, R = 1024, 32
    y = _rand(P, 7)
    F = _w(R, np.outer(np.arange(R), np.arange(R)))          # 32-point DFT matrix
    Yt = y.reshape(R, R)                                      # [n1][n2]
    Z = Yt.T @ F                                              # [n2][k1]
    Zt = Z * _w(P, np.outer(np.arange(R), np.arange(R)))      # w_P^(n2 k1)
    Xk = Zt.T @ F                                             # [k1][k2]
    X = Xk.T.reshape(P)                                       # bin k1 + 32 k2
    np.testing.assert_allclose(X, np.fft.fft(y), rtol=0, atol=1e-10 * np.abs(y).sum())


def test_real_block_form():
    """The tensor-core operands hold complex products in real block form:
    [Re z, Im z] [[Re w, Im w], [-Im w, Re w]] = [Re zw, Im zw]."""
    z, w = _rand(8, 3), _rand(8, 4)
    B = np.stack([np.stack([w.real, w.imag], -1), np.stack([-w.imag, w.real], -1)], -2)  # [8][2][2]
    zz = np.stack([z.real, z.imag], -1)[:, None, :]                                      # [8][1][2]
    got = (zz @ B)[:, 0, :]
    np.testing.assert_allclose(got[:, 0] + 1j * got[:, 1], z * w, rtol=1e-14, atol=1e-14)
