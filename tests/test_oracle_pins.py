"""Pins for the FP64 oracle: each check compares it with something that does not
come from the oracle itself (a library routine, a closed form, brute force, an
invariant, or the paper's worked example).  CPU only."""

import os

import numpy as np
import pytest

import oracle
from paper_2408_16551_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
WINDOWS = {oracle.WIN_HANN: "hann", oracle.WIN_HAMMING: "hamming", oracle.WIN_BLACKMAN: "blackman"}


def _rand_c(rng, n):
    return rng.standard_normal(n) + 1j * rng.standard_normal(n)


# --------------------------------------------------------------------------
# window indexing: the paper's unfolding example (Sec. 4.4)
# --------------------------------------------------------------------------

def test_window_indexing_matches_paper_unfold_example():
    with open(os.path.join(GOLDEN, "unfold_example.txt")) as f:
        rows = [list(map(float, ln.split())) for ln in f if ln.strip() and not ln.startswith("#")]
    x = np.array(rows[0])
    expected = np.array(rows[1:])
    J = expected.shape[1]
    # P = 1 (one sample per frame), T = J taps.  With a unit tap at position j the
    # FIR returns column j of the unfolded matrix: y[s] = x[s + j].
    cols = []
    for j in range(J):
        taps = np.zeros(J); taps[j] = 1.0
        h = oracle.prototype(1, J, oracle.WIN_USER, user_taps=taps)
        cols.append(oracle.fir(x, 1, J, h)[:, 0].real)
    got = np.stack(cols, axis=1)
    assert got.shape == expected.shape
    assert np.array_equal(got, expected)


# --------------------------------------------------------------------------
# prototype filter
# --------------------------------------------------------------------------

@pytest.mark.parametrize("window", list(WINDOWS))
@pytest.mark.parametrize("P,T", [(16, 4), (64, 8), (1024, 16), (4096, 16)])
def test_prototype_matches_scipy_firwin(window, P, T):
    signal = pytest.importorskip("scipy.signal")
    h = oracle.prototype(P, T, window)
    ref = signal.firwin(P * T, 1.0 / P, window=WINDOWS[window])
    assert np.max(np.abs(h - ref)) <= 1e-14 * np.max(np.abs(ref)) * 10


@pytest.mark.parametrize("window", list(WINDOWS))
def test_prototype_symmetry_sum_and_sinc_zeros(window):
    P = 8
    for L in (8 * 4, 8 * 4 + 1, 8 * 7 + 1):   # even and odd lengths
        h = oracle.prototype(P, 0, window, length=L)
        assert abs(h.sum() - 1.0) < 1e-14
        assert np.max(np.abs(h - h[::-1])) < 1e-16 * 8
        if L % 2 == 1:
            c = (L - 1) // 2
            zeros = [n for n in range(L) if n != c and (n - c) % P == 0]
            assert zeros
            assert np.max(np.abs(h[zeros])) < 1e-16 * 4
            assert abs(h[c]) > 1e-3


def test_user_taps_passed_through():
    taps = np.arange(12, dtype=np.float64) - 3.5
    h = oracle.prototype(4, 3, oracle.WIN_USER, user_taps=taps)
    assert np.array_equal(h, taps)


# --------------------------------------------------------------------------
# FIR step against a library correlation; DFT step against numpy.fft
# --------------------------------------------------------------------------

@pytest.mark.parametrize("P,T,N", [(4, 1, 40), (8, 3, 203), (16, 4, 16 * 4 * 9 + 5), (32, 16, 32 * 40)])
def test_fir_matches_numpy_correlate(P, T, N):
    rng = np.random.default_rng(P * 100 + T)
    x = _rand_c(rng, N)
    h = rng.standard_normal(P * T)
    y = oracle.fir(x, P, T, h)
    F = N // P
    S = F - T + 1
    assert y.shape == (S, P)
    for p in range(P):
        xp = x[p::P][:F]
        hp = h[p::P]
        ref = np.correlate(xp, hp, mode="valid")
        assert np.max(np.abs(y[:, p] - ref)) < 1e-12


@pytest.mark.parametrize("P", [4, 16, 128, 1024])
def test_dft_matches_numpy_fft(P):
    rng = np.random.default_rng(P)
    y = _rand_c(rng, 3 * P).reshape(3, P)
    X = oracle.dft(y)
    ref = np.fft.fft(y, axis=1)
    assert np.linalg.norm(X - ref) / np.linalg.norm(ref) < 1e-13


# --------------------------------------------------------------------------
# whole channeliser: brute force via the weighted-overlap-add identity
# --------------------------------------------------------------------------

@pytest.mark.parametrize("P", [4, 8, 16])
@pytest.mark.parametrize("T", [1, 2, 3, 4])
def test_pfb_brute_force_wola(P, T):
    rng = np.random.default_rng(10 * P + T)
    N = min(256, P * (T + 6)) + 3
    x = _rand_c(rng, N)
    h = rng.standard_normal(P * T)
    X = oracle.pfb(x, P, T, h)
    S = oracle.num_spectra(N, P, T)
    assert X.shape == (S, P)
    n = np.arange(P * T)
    for s in range(S):
        seg = h * x[s * P: s * P + P * T]
        # length-PT library FFT, every T-th bin
        ref_fft = np.fft.fft(seg)[np.arange(P) * T]
        # direct fused double sum
        ref_sum = np.array([np.sum(seg * np.exp(-2j * np.pi * k * n / P)) for k in range(P)])
        assert np.max(np.abs(X[s] - ref_fft)) < 1e-12
        assert np.max(np.abs(X[s] - ref_sum)) < 1e-12


def test_T1_is_windowed_fft():
    P = 32
    rng = np.random.default_rng(5)
    x = _rand_c(rng, P * 9)
    h = oracle.prototype(P, 1, oracle.WIN_HAMMING)
    X = oracle.pfb(x, P, 1, h)
    ref = np.fft.fft(x.reshape(9, P) * h[None, :], axis=1)
    assert np.max(np.abs(X - ref)) < 1e-12


# --------------------------------------------------------------------------
# impulse responses
# --------------------------------------------------------------------------

@pytest.mark.parametrize("P,T", [(8, 4), (16, 3), (64, 16)])
def test_frame_impulse_returns_reshaped_prototype(P, T):
    h = oracle.prototype(P, T, oracle.WIN_BLACKMAN)
    F = 3 * T + 2
    j = T + 1                      # impulse frame, j >= T-1
    x = np.zeros(F * P, dtype=complex)
    x[j * P:(j + 1) * P] = 1.0
    y = oracle.fir(x, P, T, h)
    hr = h.reshape(T, P)
    for s in range(y.shape[0]):
        m = j - s
        if 0 <= m < T:
            assert np.array_equal(y[s].real, hr[m]) and not np.any(y[s].imag)
        else:
            assert not np.any(y[s])
    X = oracle.pfb(x, P, T, h)
    for m in range(T):
        ref = np.fft.fft(hr[m])
        assert np.max(np.abs(X[j - m] - ref)) < 1e-13


def test_single_sample_impulse():
    P, T = 16, 4
    h = oracle.prototype(P, T, oracle.WIN_HANN)
    j, p0 = 5, 7
    x = np.zeros(10 * P, dtype=complex)
    x[j * P + p0] = 1.0
    X = oracle.pfb(x, P, T, h)
    for m in range(T):
        assert np.max(np.abs(np.abs(X[j - m]) - abs(h[m * P + p0]))) < 1e-14


# --------------------------------------------------------------------------
# tone at a channel centre: closed form
# --------------------------------------------------------------------------

@pytest.mark.parametrize("P,T,c", [(16, 4, 3), (64, 8, 17), (256, 16, 255)])
def test_complex_tone_closed_form(P, T, c):
    A, phi = 0.75, 0.3
    h = oracle.prototype(P, T, oracle.WIN_HAMMING)
    F = T + 5
    n = np.arange(F * P)
    x = A * np.exp(1j * (2 * np.pi * c * n / P + phi))
    X = oracle.pfb(x, P, T, h)
    H = h.reshape(T, P).sum(axis=0)
    Hhat = np.fft.fft(H)
    k = np.arange(P)
    expect_row = A * np.exp(1j * phi) * Hhat[(k - c) % P]
    for s in range(X.shape[0]):
        assert np.max(np.abs(X[s] - expect_row)) < 1e-12
        assert abs(X[s, c] - A * np.exp(1j * phi) * h.sum()) < 1e-12
        assert abs(abs(X[s, c]) - A) < 1e-12      # sum(h) = 1


def test_real_cosine_and_config1_peak():
    spec = synth.config_c1()
    P, T = spec.P, spec.T
    h = oracle.prototype(P, T, spec.window)
    # closed form for a pure cosine at channel 3
    n = np.arange(P * (T + 4))
    A, phi, c = 1.0, 0.0, 3
    x = A * np.cos(2 * np.pi * c * n / P + phi)
    X = oracle.pfb(x, P, T, h)
    Hhat = np.fft.fft(h.reshape(T, P).sum(axis=0))
    k = np.arange(P)
    expect = 0.5 * A * (np.exp(1j * phi) * Hhat[(k - c) % P] + np.exp(-1j * phi) * Hhat[(k + c) % P])
    assert np.max(np.abs(X - expect[None, :])) < 1e-12
    # configuration 1 (noise + unit cosine): the time-averaged power over k <= P/2
    # peaks in bin 3, at about (1/2)^2 above the noise floor
    xs = spec.generate()
    Xc = oracle.pfb_input(xs, spec.in_dtype, P, T, h)
    assert Xc.shape == (1021, 16)
    power = np.mean(np.abs(Xc[:, : P // 2 + 1]) ** 2, axis=0)
    assert np.argmax(power) == 3
    noise = np.sum(h ** 2)                      # per-bin noise power for unit-variance input
    assert abs(power[3] - (0.25 + noise)) < 0.1 * power[3]


# --------------------------------------------------------------------------
# invariants
# --------------------------------------------------------------------------

def test_linearity():
    P, T = 32, 5
    rng = np.random.default_rng(11)
    x1, x2 = _rand_c(rng, P * 20), _rand_c(rng, P * 20)
    a, b = 0.7 - 0.2j, -1.3 + 0.4j
    h = oracle.prototype(P, T, oracle.WIN_HANN)
    lhs = oracle.pfb(a * x1 + b * x2, P, T, h)
    rhs = a * oracle.pfb(x1, P, T, h) + b * oracle.pfb(x2, P, T, h)
    assert np.max(np.abs(lhs - rhs)) < 1e-13 * np.max(np.abs(rhs))


def test_parseval():
    P, T = 64, 8
    rng = np.random.default_rng(12)
    x = _rand_c(rng, P * 30)
    h = oracle.prototype(P, T, oracle.WIN_BLACKMAN)
    y = oracle.fir(x, P, T, h)
    X = oracle.dft(y)
    lhs = np.sum(np.abs(X) ** 2, axis=1)
    rhs = P * np.sum(np.abs(y) ** 2, axis=1)
    assert np.max(np.abs(lhs - rhs) / rhs) < 1e-12


def test_time_shift_by_one_frame():
    P, T = 16, 4
    rng = np.random.default_rng(13)
    x = _rand_c(rng, P * 30)
    h = oracle.prototype(P, T, oracle.WIN_HANN)
    X = oracle.pfb(x, P, T, h)
    Xs = oracle.pfb(x[P:], P, T, h)
    assert np.array_equal(Xs, X[1:])


def test_spectra_window_selection_matches_full_run():
    P, T = 16, 4
    rng = np.random.default_rng(14)
    x = _rand_c(rng, P * 50 + 7)
    h = oracle.prototype(P, T, oracle.WIN_HANN)
    X = oracle.pfb(x, P, T, h)
    assert np.array_equal(oracle.pfb(x, P, T, h, s0=9, ns=13), X[9:22])


# --------------------------------------------------------------------------
# input handling and output counts
# --------------------------------------------------------------------------

def test_dequant_int8_and_real():
    raw = np.array([-127, 127, 0, -1, 5, -6], dtype=np.int8)
    xr, xi = oracle.dequant(raw, oracle.IN_CI8, 0.25)
    assert np.array_equal(xr, np.array([-127, 0, 5]) * 0.25)
    assert np.array_equal(xi, np.array([127, -1, -6]) * 0.25)
    r = np.array([1.5, -2.0], dtype=np.float32)
    xr, xi = oracle.dequant(r, oracle.IN_R32)
    assert np.array_equal(xr, [1.5, -2.0]) and not np.any(xi)


@pytest.mark.parametrize("N,P,T,S", [(16384, 16, 4, 1021), (1 << 24, 1024, 16, 16369),
                                     (1 << 20, 4096, 16, 241), (1 << 14, 4096, 16, 0),
                                     (4096 * 16 - 1, 4096, 16, 0), (4096 * 16, 4096, 16, 1), (0, 8, 2, 0)])
def test_num_spectra(N, P, T, S):
    assert oracle.num_spectra(N, P, T) == S


# --------------------------------------------------------------------------
# the pins catch plausible mistakes (mistakes planted on the CPU, in the oracle's inputs)
# --------------------------------------------------------------------------

def test_pins_reject_convolution_tap_order():
    """The convolution reading (taps reversed per branch) fails the impulse pin."""
    P, T = 8, 4
    h = oracle.prototype(P, T, oracle.WIN_BLACKMAN)
    h_rev = h.reshape(T, P)[::-1].ravel()
    j = T + 1
    x = np.zeros((3 * T) * P, dtype=complex)
    x[j * P:(j + 1) * P] = 1.0
    y_bad = oracle.fir(x, P, T, h_rev)
    assert not np.array_equal(y_bad[j].real, h.reshape(T, P)[0])


def test_pins_reject_positive_exponent():
    """A DFT with the wrong sign puts a channel-c tone in bin -c."""
    P, T, c = 16, 4, 3
    h = oracle.prototype(P, T, oracle.WIN_HAMMING)
    n = np.arange(P * 10)
    x = np.exp(2j * np.pi * c * n / P)
    X = oracle.pfb(x, P, T, h)
    X_wrong_sign = np.conj(oracle.pfb(np.conj(x), P, T, h))   # = DFT with +i exponent
    assert np.argmax(np.abs(X[0])) == c
    assert np.argmax(np.abs(X_wrong_sign[0])) == (-c) % P


# --------------------------------------------------------------------------
# oversampled channeliser (hop D < P) and the convolution tap order
# --------------------------------------------------------------------------

@pytest.mark.parametrize("P,T", [(8, 3), (16, 4), (32, 2)])
def test_hop_P_is_the_critically_sampled_pfb(P, T):
    rng = np.random.default_rng(P + T)
    x = _rand_c(rng, P * (T + 9) + 3)
    h = oracle.prototype(P, T, oracle.WIN_HAMMING)
    assert np.array_equal(oracle.pfb_hop(x, P, T, h, P), oracle.pfb(x, P, T, h))


@pytest.mark.parametrize("P,T,D", [(8, 3, 4), (16, 4, 2), (16, 2, 8), (32, 3, 4), (8, 1, 2)])
def test_hop_matches_numpy_wola(P, T, D):
    """Brute force with numpy: each spectrum is the P-point FFT of the folded
    window h * x[sD : sD + PT] (weighted overlap-add)."""
    rng = np.random.default_rng(3 * P + D)
    N = P * T + D * 13 + 5
    x = _rand_c(rng, N)
    h = oracle.prototype(P, T, oracle.WIN_BLACKMAN)
    S = oracle.num_spectra_hop(N, P, T, D)
    assert S == (N - P * T) // D + 1
    ref = np.stack([np.fft.fft((h * x[s * D:s * D + P * T]).reshape(T, P).sum(axis=0)) for s in range(S)])
    got = oracle.pfb_hop(x, P, T, h, D)
    assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref))


@pytest.mark.parametrize("P,T", [(8, 4), (16, 3), (4, 5)])
def test_convolution_order_matches_numpy_convolve(P, T):
    """The literal Sec. 5.2 equation y_p(n') = sum_m h_p(m) x_p(n'-m) with
    x_p(n') = x[n'P + p]: numpy.convolve per branch, valid outputs, then the FFT."""
    rng = np.random.default_rng(P * T)
    F = T + 11
    x = _rand_c(rng, P * F)
    h = oracle.prototype(P, T, oracle.WIN_HANN)
    y = np.stack([np.convolve(x[p::P], h[p::P], mode="valid") for p in range(P)], axis=1)
    ref = np.fft.fft(y, axis=1)
    got = oracle.pfb_hop(x, P, T, h, P, reverse=True)
    assert got.shape == ref.shape
    assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref))
    # and the oversampled convolution order is the WOLA with per-branch reversed taps
    hr = h.reshape(T, P)[::-1].reshape(-1)
    assert np.array_equal(oracle.pfb_hop(x, P, T, h, P // 2, reverse=True), oracle.pfb_hop(x, P, T, hr, P // 2))


def test_hop_time_shift_and_tone_closed_form():
    P, T, D = 16, 4, 4
    rng = np.random.default_rng(11)
    x = _rand_c(rng, P * T + D * 20)
    h = oracle.prototype(P, T, oracle.WIN_HAMMING)
    a = oracle.pfb_hop(x, P, T, h, D)
    b = oracle.pfb_hop(x[D:], P, T, h, D)
    assert np.array_equal(a[1:], b[:a.shape[0] - 1])
    # a tone at channel centre c: X[s,c] = A e^{i phi} e^{2 pi i c s D / P} sum(h)
    A, c, phi = 0.7, 5, 0.3
    n = np.arange(P * T + D * 9)
    xt = A * np.exp(2j * np.pi * (c * n / P + phi))
    X = oracle.pfb_hop(xt, P, T, h, D)
    s = np.arange(X.shape[0])
    want = A * np.exp(2j * np.pi * phi) * np.exp(2j * np.pi * c * s * D / P) * h.sum()
    assert np.max(np.abs(X[:, c] - want)) <= 1e-12


# --------------------------------------------------------------------------
# synthesis (inverse) filter bank
# --------------------------------------------------------------------------

@pytest.mark.parametrize("P,T,S", [(8, 3, 7), (16, 4, 5), (4, 1, 6), (32, 2, 3)])
def test_synth_is_the_adjoint_of_the_analysis(P, T, S):
    """<A x, Y> = P <x, synth(Y)> for the analysis A of the pinned oracle, random
    x and Y: the synthesis is A's adjoint (the IDFT carries 1/P)."""
    rng = np.random.default_rng(7 * P + T + S)
    N = (S + T - 1) * P
    x = _rand_c(rng, N)
    Y = rng.standard_normal((S, P)) + 1j * rng.standard_normal((S, P))
    h = oracle.prototype(P, T, oracle.WIN_HAMMING)
    lhs = np.vdot(oracle.pfb(x, P, T, h), Y)          # <A x, Y> = sum conj(Ax) Y
    rhs = P * np.vdot(x, oracle.synth(Y, P, T, h))
    assert abs(lhs - rhs) <= 1e-11 * max(1.0, abs(lhs))


def test_synth_T1_is_windowed_ifft_and_impulse_closed_form():
    P, S = 16, 5
    rng = np.random.default_rng(5)
    Y = rng.standard_normal((S, P)) + 1j * rng.standard_normal((S, P))
    h = oracle.prototype(P, 1, oracle.WIN_HANN)
    got = oracle.synth(Y, P, 1, h).reshape(S, P)
    assert np.max(np.abs(got - h[None, :] * np.fft.ifft(Y, axis=1))) <= 1e-13
    # one unit bin (s0, k0): frames s0..s0+T-1 carry h[mP+p] e^{2 pi i p k0 / P} / P
    T, s0, k0 = 4, 2, 3
    h = oracle.prototype(P, T, oracle.WIN_BLACKMAN)
    Y = np.zeros((6, P), complex); Y[s0, k0] = 1.0
    xh = oracle.synth(Y, P, T, h).reshape(-1, P)
    p = np.arange(P)
    want = np.zeros_like(xh)
    for m in range(T):
        want[s0 + m] = h[m * P + p] * np.exp(2j * np.pi * p * k0 / P) / P
    assert np.max(np.abs(xh - want)) <= 1e-15
    # frame windows: a sub-range equals the matching part of the full output
    Yr = rng.standard_normal((6, P)) + 1j * rng.standard_normal((6, P))
    full = oracle.synth(Yr, P, T, h)
    assert full.size == (6 + T - 1) * P
    assert np.array_equal(oracle.synth(Yr, P, T, h, f0=2, nf=5), full[2 * P:7 * P])
