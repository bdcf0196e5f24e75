"""FP64 CPU oracle for the PFB channeliser -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import this package.  The
library under ``paper_2408_16551_gb300`` never does, and the two share no
code: the arithmetic lives in ``pfb_oracle.c`` (plain C, FP64), this module
only marshals NumPy arrays into it.

Functions and the passages they follow (TINA, arXiv 2408.16551):

* ``prototype``  -- windowed-sinc taps h[n], n < P*T, sum(h) = 1 (the taps
  "divided between the P branches" of Sec. 5.2; window/sinc is our reading).
* ``dequant``    -- input samples to complex FP64 (real input gets im = 0,
  int8 pairs are scaled).
* ``fir``        -- y[s,p] = sum_{m<T} h[mP+p] x[(s+m)P+p]: the per-branch FIR
  of Sec. 5.2 in the cross-correlation form of Sec. 4.3 (O(w)=sum_n I(w+n)K(n)).
* ``dft``        -- X[s,k] = sum_p y[s,p] exp(-2 pi i (pk mod P)/P): the
  Fourier-matrix product of Sec. 4.1.
* ``pfb``        -- ``fir`` then ``dft``.
* ``synth``      -- the synthesis (inverse) filter bank: y~ = IDFT(X) (the
  inverse Fourier-matrix product of Sec. 4.2, 1/P), then each branch spread
  over the T frames it was analysed from, xh[fP+p] = sum_m h[mP+p] y~[f-m,p]
  (the adjoint of ``fir``).
* ``pfb_hop``    -- the channeliser evaluated every D samples (oversampled for
  D < P), X[s,k] = sum_{n<PT} h'[n] x[sD+n] exp(-2 pi i nk/P), with the taps
  in the correlation order of Sec. 4.3 or reversed within each branch (the
  convolution y_p(n') = sum_m h_p(m) x_p(n'-m) of the Sec. 5.2 equation).

Every function is pinned by ``tests/test_oracle_pins.py`` against values that
do not come from this package.
"""

from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pfb_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

IN_R32, IN_C64, IN_CI8 = 0, 1, 2
WIN_HANN, WIN_HAMMING, WIN_BLACKMAN, WIN_USER = 0, 1, 2, 3


def build(force: bool = False) -> str:
    """Compile the oracle's C source into ``oracle/_build/liboracle.so``."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-std=c11", "-fno-fast-math",
                               "-ffp-contract=off", _SRC, "-o", tmp, "-lm", "-lpthread"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            d = ctypes.POINTER(ctypes.c_double)
            i64 = ctypes.c_int64
            lib.oracle_prototype.argtypes = [i64, i64, ctypes.c_int, d, d]
            lib.oracle_prototype.restype = ctypes.c_int
            lib.oracle_num_spectra.argtypes = [i64, i64, i64]
            lib.oracle_num_spectra.restype = i64
            lib.oracle_fir.argtypes = [d, d, i64, i64, i64, d, i64, i64, d, d, ctypes.c_int]
            lib.oracle_fir.restype = ctypes.c_int
            lib.oracle_dft.argtypes = [d, d, i64, i64, d, d, ctypes.c_int]
            lib.oracle_dft.restype = ctypes.c_int
            lib.oracle_pfb.argtypes = [d, d, i64, i64, i64, d, i64, i64, d, d, ctypes.c_int]
            lib.oracle_pfb.restype = ctypes.c_int
            lib.oracle_num_spectra_hop.argtypes = [i64, i64, i64, i64]
            lib.oracle_num_spectra_hop.restype = i64
            lib.oracle_pfb_hop.argtypes = [d, d, i64, i64, i64, i64, ctypes.c_int, d, i64, i64, d, d, ctypes.c_int]
            lib.oracle_pfb_hop.restype = ctypes.c_int
            lib.oracle_synth.argtypes = [d, d, i64, i64, i64, d, i64, i64, d, d]
            lib.oracle_synth.restype = ctypes.c_int
            _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _threads(threads):
    return int(threads) if threads else (os.cpu_count() or 1)


def num_spectra(n_samples: int, P: int, T: int) -> int:
    return int(_load().oracle_num_spectra(n_samples, P, T))


def prototype(P: int, T: int, window: int = WIN_HANN, user_taps=None, length: int | None = None) -> np.ndarray:
    """FP64 prototype taps h[0..L) with L = P*T (or ``length`` for direct tests)."""
    L = int(length) if length is not None else P * T
    h = np.zeros(L, dtype=np.float64)
    user = None
    if window == WIN_USER:
        user = np.ascontiguousarray(user_taps, dtype=np.float64)
        if user.shape != (L,):
            raise ValueError("user taps must have P*T entries")
    rc = _load().oracle_prototype(P, L, window, _ptr(user) if user is not None else None, _ptr(h))
    if rc != 0:
        raise ValueError("oracle_prototype rejected its arguments")
    return h


def dequant(x: np.ndarray, in_dtype: int, scale: float = 1.0):
    """Input buffer -> (re, im) FP64 arrays (step a3: load + dequant)."""
    if in_dtype == IN_R32:
        xr = np.asarray(x, dtype=np.float32).astype(np.float64)
        return xr, np.zeros_like(xr)
    if in_dtype == IN_C64:
        xc = np.asarray(x, dtype=np.complex64)
        return xc.real.astype(np.float64), xc.imag.astype(np.float64)
    if in_dtype == IN_CI8:
        xi8 = np.asarray(x, dtype=np.int8).reshape(-1, 2).astype(np.float64)
        s = float(np.float32(scale))
        return xi8[:, 0] * s, xi8[:, 1] * s
    raise ValueError(f"unknown in_dtype {in_dtype}")


def _as_split(x):
    if isinstance(x, tuple):
        xr, xi = x
    else:
        xc = np.asarray(x)
        if np.iscomplexobj(xc):
            xr, xi = xc.real, xc.imag
        else:
            xr, xi = xc, np.zeros(xc.shape)
    return (np.ascontiguousarray(xr, dtype=np.float64), np.ascontiguousarray(xi, dtype=np.float64))


def fir(x, P: int, T: int, h: np.ndarray, s0: int = 0, ns: int | None = None, threads=None) -> np.ndarray:
    """Branch sums y[s,p] for s in [s0, s0+ns) as complex128 [ns, P]."""
    xr, xi = _as_split(x)
    N = xr.shape[0]
    S = num_spectra(N, P, T)
    ns = S - s0 if ns is None else ns
    h = np.ascontiguousarray(h, dtype=np.float64)
    yr = np.zeros((max(ns, 0), P)); yi = np.zeros((max(ns, 0), P))
    rc = _load().oracle_fir(_ptr(xr), _ptr(xi), N, P, T, _ptr(h), s0, ns, _ptr(yr), _ptr(yi), _threads(threads))
    if rc != 0:
        raise ValueError("oracle_fir rejected its arguments")
    return yr + 1j * yi


def dft(y: np.ndarray, threads=None) -> np.ndarray:
    """Row-wise forward DFT (no normalisation) by the Fourier-matrix product."""
    y = np.asarray(y, dtype=np.complex128)
    rows, P = y.shape
    yr = np.ascontiguousarray(y.real); yi = np.ascontiguousarray(y.imag)
    Xr = np.zeros((rows, P)); Xi = np.zeros((rows, P))
    rc = _load().oracle_dft(_ptr(yr), _ptr(yi), rows, P, _ptr(Xr), _ptr(Xi), _threads(threads))
    if rc != 0:
        raise ValueError("oracle_dft rejected its arguments")
    return Xr + 1j * Xi


def pfb(x, P: int, T: int, h: np.ndarray, s0: int = 0, ns: int | None = None, threads=None) -> np.ndarray:
    """Channeliser output X[s,k] for s in [s0, s0+ns) as complex128 [ns, P]."""
    xr, xi = _as_split(x)
    N = xr.shape[0]
    S = num_spectra(N, P, T)
    ns = S - s0 if ns is None else ns
    h = np.ascontiguousarray(h, dtype=np.float64)
    Xr = np.zeros((max(ns, 0), P)); Xi = np.zeros((max(ns, 0), P))
    rc = _load().oracle_pfb(_ptr(xr), _ptr(xi), N, P, T, _ptr(h), s0, ns, _ptr(Xr), _ptr(Xi), _threads(threads))
    if rc != 0:
        raise ValueError("oracle_pfb rejected its arguments")
    return Xr + 1j * Xi


def num_spectra_hop(n_samples: int, P: int, T: int, D: int) -> int:
    return int(_load().oracle_num_spectra_hop(n_samples, P, T, D))


def pfb_hop(x, P: int, T: int, h: np.ndarray, D: int, reverse: bool = False, s0: int = 0, ns: int | None = None,
            threads=None) -> np.ndarray:
    """Channeliser with hop D and tap order (reverse = convolution order), X[s,k] for s in [s0, s0+ns)."""
    xr, xi = _as_split(x)
    N = xr.shape[0]
    S = num_spectra_hop(N, P, T, D)
    ns = S - s0 if ns is None else ns
    h = np.ascontiguousarray(h, dtype=np.float64)
    Xr = np.zeros((max(ns, 0), P)); Xi = np.zeros((max(ns, 0), P))
    rc = _load().oracle_pfb_hop(_ptr(xr), _ptr(xi), N, P, T, D, 1 if reverse else 0, _ptr(h), s0, ns, _ptr(Xr),
                                _ptr(Xi), _threads(threads))
    if rc != 0:
        raise ValueError("oracle_pfb_hop rejected its arguments")
    return Xr + 1j * Xi


def synth(X: np.ndarray, P: int, T: int, h: np.ndarray, f0: int = 0, nf: int | None = None) -> np.ndarray:
    """Synthesis filter bank: frames [f0, f0+nf) of xh (complex128, nf*P samples),
    xh[fP+p] = sum_m h[mP+p] y~[f-m,p] with y~ = IDFT(X) (1/P) per spectrum."""
    X = np.asarray(X, dtype=np.complex128)
    S = X.shape[0]
    F = S + T - 1 if S > 0 else 0
    nf = F - f0 if nf is None else nf
    Xr = np.ascontiguousarray(X.real); Xi = np.ascontiguousarray(X.imag)
    h = np.ascontiguousarray(h, dtype=np.float64)
    xr = np.zeros(max(nf, 0) * P); xi = np.zeros(max(nf, 0) * P)
    rc = _load().oracle_synth(_ptr(Xr), _ptr(Xi), S, P, T, _ptr(h), f0, nf, _ptr(xr), _ptr(xi))
    if rc != 0:
        raise ValueError("oracle_synth rejected its arguments")
    return xr + 1j * xi


def pfb_input(x: np.ndarray, in_dtype: int, P: int, T: int, h: np.ndarray, scale: float = 1.0,
              s0: int = 0, ns: int | None = None, threads=None) -> np.ndarray:
    """Channeliser output of a raw input buffer (dequant, FIR, DFT)."""
    return pfb(dequant(x, in_dtype, scale), P, T, h, s0=s0, ns=ns, threads=threads)


def rel_l2(a: np.ndarray, ref: np.ndarray) -> float:
    """||a - ref||_2 / ||ref||_2 in FP64 (the parity metric)."""
    a = np.asarray(a, dtype=np.complex128); ref = np.asarray(ref, dtype=np.complex128)
    den = np.linalg.norm(ref.ravel())
    num = np.linalg.norm((a - ref).ravel())
    return float(num / den) if den > 0 else float(num)
