"""Pins of the Kramers-Kronig front-end reference (oracle/kk.py): exact field
reconstruction of a minimum-phase signal (the sign of the Hilbert image), the
100 % overlap-save Hilbert against the whole-stream transform, the decimating
filter against plain decimation, and the end-to-end symbols of a noise-free link."""
import math

import numpy as np

import linksim as L
import linksim.kk as LK
from oracle import kk as K


def _min_phase(n, ratio, band, seed):
    """E = A + s with s periodic, band-limited to [-band, 0) (negative side), |s| << A."""
    rng = np.random.default_rng(seed)
    S = np.zeros(n, np.complex128)
    k = np.arange(1, int(band * n))
    S[n - k] = rng.standard_normal(k.size) + 1j * rng.standard_normal(k.size)
    s = np.fft.ifft(S)
    s *= ratio / np.max(np.abs(s))
    return 1.0 + s


def test_kk_relation_exact_on_periodic_minimum_phase_signal():
    E = _min_phase(4096, 0.05, 1 / 16, 1) * np.exp(0.7j)   # a constant phase is not recoverable
    I = np.abs(E) ** 2
    lna = 0.5 * np.log(I)
    phi = np.fft.ifft(np.fft.fft(lna) * K.hilbert_response(4096)).real
    Er = np.sqrt(I) * np.exp(1j * phi)
    r = Er / E
    assert np.max(np.abs(r / r[0] - 1)) < 1e-9
    # the other sign of the Hilbert image does not rebuild the field
    Ew = np.sqrt(I) * np.exp(-1j * phi)
    assert np.max(np.abs(Ew / E / (Ew[0] / E[0]) - 1)) > 1e-2


def test_overlap_save_hilbert_close_to_whole_stream():
    n = 1 << 15
    E = _min_phase(n, 0.05, 1 / 16, 2)
    I = np.abs(E) ** 2
    lna = 0.5 * np.log(I)
    Ew = np.sqrt(I) * np.exp(1j * np.fft.ifft(np.fft.fft(lna) * K.hilbert_response(n)).real)
    inner = slice(4096, n - 4096)
    errs = []
    for N in (1024, 4096):
        Eo = K.hilbert_field(I, 4.0, 0.0, N)          # f_c = 0: no shift
        errs.append(np.linalg.norm(Eo[inner] - Ew[inner]) / np.linalg.norm(Ew[inner]))
    # the Hilbert kernel decays as 1/t, so windowing leaves a slowly falling error:
    # ~1e-3 of the field at 1024 points (7 % of the side band), less at 4096
    assert errs[0] < 2e-3 and errs[1] < errs[0]
    # identity filter through the overlap-save window bookkeeping is an exact copy
    x = np.random.default_rng(3).standard_normal(5000) + 0j
    assert np.max(np.abs(K.overlap_save(x, np.ones(1024, np.complex128), 512) - x)) < 1e-13


def test_decimating_filter_is_plain_decimation_for_band_limited_input():
    n = 1 << 14
    rng = np.random.default_rng(4)
    X = np.zeros(n, np.complex128)
    k = np.r_[0:n // 4 - 8, n - n // 4 + 8:n]
    X[k] = rng.standard_normal(k.size) + 1j * rng.standard_normal(k.size)
    x = np.fft.ifft(X)
    # a periodic band-limited signal: compare in the interior, away from the zero-padded ends
    y = K.decimating_filter(x, np.ones(1024, np.complex128), 512)
    inner = slice(1024, n // 2 - 1024)
    err = np.abs(y[inner] - x[::2][inner]).max() / np.abs(x).max()
    assert err < 2e-2
    # exact when the window covers the whole (periodic) stream
    y2 = K.decimating_filter(np.tile(x, 3), np.ones(3 * n, np.complex128), 0)
    assert np.abs(y2 - np.tile(x, 3)[::2]).max() < 1e-12


def test_end_to_end_noise_free_symbols():
    lk = LK.KKLink(n_sym=1 << 14, adc="f32", snr_db=None, L_km=1000.0, cspr_db=14.0)
    g = LK.generate(lk)
    y, _, V = K.kk_frontend(g.samples, g.in_scale, g.in_offset, lk.baud, lk.sps, lk.carrier_hz, lk.L_km)
    assert V == 512
    z = y[0::2][256:-256]
    t = g.tx_symbols[256:-256]
    c = np.vdot(t, z) / np.vdot(t, t)            # the complex gain left over
    evm = np.linalg.norm(z - c * t) / np.linalg.norm(c * t)
    assert evm < 0.03, evm
    # sqrt(sps) and the carrier's dispersion phase are in the static filter: unit gain,
    # no constant phase (without the phase term the angle would be beta2 L w_c^2/2 = 0.114)
    assert abs(c - 1.0) < 2e-3, c
    # the 16QAM decisions are error-free without any correction
    d = L.map_symbols(L.random_bits(lk.seed, lk.n_sym * 4).reshape(1, -1), "16qam")[0][256:-256]
    from oracle.chain import decide
    assert np.array_equal(decide(z, "16qam"), d)


def test_static_filter_phase_term_cancels_the_carrier_dispersion_phase():
    # through CD alone, a tone at f_c picks up exp(+j beta2 L w_c^2/2); the KK field is
    # referenced to that tone, so it carries the conjugate, and the static filter's
    # constant must be the tone's own phase, whatever L and f_c
    for L_km, k in ((1000.0, 528), (7600.0, 307)):
        fc = k * 4e9 / 4096                          # on the DFT grid: a pure tone
        tone = np.exp(2j * np.pi * fc / 4e9 * np.arange(4096))
        rx = L.apply_dispersion(tone[None, :], 4e9, L_km, 17.0, 1550.0)[0]
        ph = np.angle(np.vdot(tone, rx))
        H = K.static_filter(1e9, 4e9, L_km, 17.0, 1550.0, 0.01, 1024, fc)
        assert abs(abs(H[0]) - 2.0) < 1e-12                 # sqrt(sps) at DC
        assert abs(ph) > 0.05
        assert abs(np.angle(H[0] * np.exp(-1j * ph))) < 1e-9


def test_consecutive_buffers_share_the_carrier_phase():
    # a buffer processed on its own, with its stream index n0, equals the whole-stream
    # result away from its edges (windows aligned: n0 a multiple of both hops);
    # with n0 = 0 it would carry the constant rotation exp(-j 2 pi f_c n0 / fs)
    lk = LK.KKLink(n_sym=1 << 13, adc="f32", snr_db=30.0, L_km=2000.0)
    g = LK.generate(lk)
    n = g.samples.shape[0]
    n0 = n // 2
    whole, _, V = K.kk_frontend(g.samples, g.in_scale, g.in_offset, lk.baud, lk.sps, lk.carrier_hz, lk.L_km)
    assert n0 % 512 == 0 and n0 % (1024 - V) == 0
    second, _, _ = K.kk_frontend(g.samples[n0:], g.in_scale, g.in_offset, lk.baud, lk.sps, lk.carrier_hz,
                                 lk.L_km, n0=n0)
    inner = slice(2048, n // 4 - 2048)
    ref = whole[n0 // 2:][inner]
    assert np.abs(second[inner] - ref).max() < 1e-9 * np.abs(ref).max()
    wrong, _, _ = K.kk_frontend(g.samples[n0:], g.in_scale, g.in_offset, lk.baud, lk.sps, lk.carrier_hz, lk.L_km)
    rot = np.vdot(ref, wrong[inner]) / np.vdot(ref, ref)
    assert abs(np.angle(rot) - math.remainder(-2 * math.pi * lk.carrier_hz / lk.fs * n0, 2 * math.pi)) < 1e-9
