"""FP64 reference of the Kramers-Kronig receiver front end (test infrastructure
only: tests/, __graft_entry__.smoke() and bench.py's CPU baseline may use it).

The paper's processing chain (Section "Experimental setup", processing-chain
paragraph): ADC samples to floating point; square root and logarithm; the
optical phase from a Hilbert transform computed by a pair of 1024-point
overlap-save FFTs with 100 % overlap; the field rebuilt from amplitude and
phase and shifted to DC; a static frequency-domain filter (an FFT/IFFT pair)
that also downsamples from 4 to 2 samples per symbol.  Readings:

  * 100 % overlap-save: window length N = 1024, overlap V = N/2, hop S = N/2;
    window i reads samples [iS - V/2, iS - V/2 + N) and keeps [iS, iS + S);
    samples outside the buffer contribute amplitude 0 and log-amplitude 0.
  * Field: E = a exp(j phi), a = sqrt(max(I, eps)), phi = the Hilbert image of
    ln a with the response j sign(f) (the signal sits below the carrier, so the
    reconstructed field is minimum phase with negative-frequency side band;
    Mecozzi, Antonelli, Shtaif, Optica 2016); eps = 1e-30.
  * Shift to DC: multiply by exp(+j 2 pi f_c n / fs) with n the sample's
    index in the whole stream (buffer i starts at n0 = the samples before it),
    so that consecutive buffers share one carrier phase (the carrier moves to
    +f_c, outside the RRC band, and the next filter removes it).
  * Static filter (the paper's offline-optimised filter has no closed form):
    sqrt(sps) exp(-j beta2 L w^2 / 2) times the RRC matched filter on the fs
    grid, times the constant exp(+j beta2 L w_c^2 / 2) that takes back the
    phase the carrier tone at w_c = 2 pi f_c picked up in the fibre (the
    rebuilt field is referenced to the received tone), so that symbols come
    out with unit gain and no constant phase -- what an offline fit against
    known symbols converges to; in
    overlap-save windows of N = 1024 with V = max(N/2, the textbook CD length
    rounded up to 32) (100 % overlap like the Hilbert pair, which also covers
    most of the 1 %-roll-off RRC response); downsampling keeps the N/2 bins of
    |f| < fs/4 and transforms them back with an N/2-point IDFT; the decimated
    DFT carries a factor 1/2.
"""
from __future__ import annotations

import math

import numpy as np

TWO_PI = 2.0 * math.pi
EPS = 1e-30


def grid(n: int, fs: float) -> np.ndarray:
    k = np.arange(n)
    return np.where(k < n // 2, k, k - n) * (fs / n)


def hilbert_response(N: int) -> np.ndarray:
    """j sign(f_k): +j for 0 < k < N/2, -j for k > N/2, 0 at k = 0 and N/2."""
    k = np.arange(N)
    h = np.zeros(N, np.complex128)
    h[(k > 0) & (k < N // 2)] = 1j
    h[k > N // 2] = -1j
    return h


def overlap_save(x: np.ndarray, H: np.ndarray, V: int) -> np.ndarray:
    """y = x filtered by H (length-N response) in windows of N with overlap V."""
    N = H.shape[0]
    S = N - V
    n = x.shape[0]
    y = np.zeros(n, np.complex128)
    for i in range((n + S - 1) // S):
        lo = i * S - V // 2
        w = np.zeros(N, np.complex128)
        a, b = max(lo, 0), min(lo + N, n)
        w[a - lo:b - lo] = x[a:b]
        out = np.fft.ifft(np.fft.fft(w) * H)
        e = min(i * S + S, n)
        y[i * S:e] = out[V // 2:V // 2 + (e - i * S)]
    return y


def n_cd_taps(baud: float, sps: int, L_km: float, D: float, lam_nm: float) -> int:
    T = 1.0 / (sps * baud)
    Dsm = abs(D) * 1e-12 / (1e-9 * 1e3)
    lam = lam_nm * 1e-9
    return 2 * int(math.floor(Dsm * lam * lam * L_km * 1e3 / (2.0 * 299792458.0 * T * T))) + 1


def static_filter(baud: float, fs: float, L_km: float, D: float, lam_nm: float, rolloff: float, N: int,
                  f_c: float = 0.0) -> np.ndarray:
    f = grid(N, fs)
    Dsm = D * 1e-12 / (1e-9 * 1e3)
    lam = lam_nm * 1e-9
    beta2 = -Dsm * lam * lam / (TWO_PI * 299792458.0)
    af = np.abs(f)
    f1, f2 = (1.0 - rolloff) * baud / 2.0, (1.0 + rolloff) * baud / 2.0
    rrc = np.where(af <= f1, 1.0, np.where(af <= f2, np.cos(np.pi * (af - f1) / (2.0 * rolloff * baud)), 0.0))
    gain = math.sqrt(fs / baud) * np.exp(1j * beta2 * (L_km * 1e3) * (TWO_PI * f_c) ** 2 / 2.0)
    return gain * np.exp(-1j * beta2 * (L_km * 1e3) * (TWO_PI * f) ** 2 / 2.0) * rrc


def hilbert_field(I: np.ndarray, fs: float, f_c: float, N: int = 1024, n0: int = 0) -> np.ndarray:
    """Rebuilt field shifted to DC at the input rate (complex, same length as I);
    n0 is the stream index of I[0]."""
    n = I.shape[0]
    a = np.sqrt(np.maximum(I, EPS))
    lna = np.log(a)
    phi = overlap_save(lna.astype(np.complex128), hilbert_response(N), N // 2).real
    E = a * np.exp(1j * phi)
    turns = np.mod((f_c / fs) * (n0 + np.arange(n, dtype=np.float64)), 1.0)
    return E * np.exp(1j * TWO_PI * turns)


def decimating_filter(E: np.ndarray, H: np.ndarray, V: int) -> np.ndarray:
    """Overlap-save with H on the input grid, output at half the rate (keep |f| < fs/4)."""
    N = H.shape[0]
    S = N - V
    n = E.shape[0]
    h = N // 2
    y = np.zeros(n // 2, np.complex128)
    for i in range((n + S - 1) // S):
        lo = i * S - V // 2
        w = np.zeros(N, np.complex128)
        a, b = max(lo, 0), min(lo + N, n)
        w[a - lo:b - lo] = E[a:b]
        X = np.fft.fft(w) * H
        Y = 0.5 * np.concatenate([X[:h // 2], X[N - h // 2:]])
        out = np.fft.ifft(Y)
        o0, o1 = (i * S) // 2, min((i * S + S) // 2, n // 2)
        y[o0:o1] = out[V // 4:V // 4 + (o1 - o0)]
    return y


def kk_frontend(samples: np.ndarray, in_scale: float, in_offset: float, baud: float, sps: int, f_c: float,
                L_km: float, D: float = 17.0, lam_nm: float = 1550.0, rolloff: float = 0.01, N: int = 1024,
                n0: int = 0):
    """One buffer of receiver samples, the first at stream index n0 -> (field at 2
    samples/symbol, field at the input rate, V of the filter)."""
    fs = sps * baud
    I = (np.asarray(samples, np.float64) + in_offset) * in_scale
    E = hilbert_field(I, fs, f_c, N, n0)
    V = max(N // 2, ((n_cd_taps(baud, sps, L_km, D, lam_nm) - 1 + 31) // 32) * 32)
    H = static_filter(baud, fs, L_km, D, lam_nm, rolloff, N, f_c)
    return decimating_filter(E, H, V), E, V
