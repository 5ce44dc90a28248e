"""Pins of the FP64 widely-linear DD-LMS reference (oracle/wl.py) against what
the mathematics fixes: the fixed point at exact taps, the plain convolution it
reduces to at zero step size, the closed-form widely-linear and linear inverses
of a transmitter IQ imbalance, the locality of the segment schedule, and the
AWGN bit-error ratio of 16QAM.
"""
import math

import numpy as np
import pytest
from scipy.special import erfc

import linksim as L
import linksim.kk as LK
from oracle import wl as W


def _symbols(K, mod, seed):
    m = L.bits_per_symbol(mod)
    bits = L.random_bits(seed, K * m)
    return bits, L.map_symbols(bits.reshape(1, -1), mod)[0]


def _two_sps(s, rng, between=1.0):
    """x[2k] = s_k, x[2k+1] an independent complex Gaussian of power `between`."""
    K = s.shape[0]
    x = np.zeros(2 * K, np.complex128)
    x[0::2] = s
    x[1::2] = math.sqrt(between / 2) * (rng.standard_normal(K) + 1j * rng.standard_normal(K))
    return x


@pytest.mark.parametrize("mod", ["qpsk", "16qam"])
def test_exact_taps_are_a_fixed_point(mod):
    # the start taps pick x[2k]: with x[2k] = s_k the error is 0 at every symbol
    rng = np.random.default_rng(3)
    bits, s = _symbols(3000 + 17, mod, 11)
    x = _two_sps(s, rng)
    p = W.WLParams(mod=mod, mu=0.05, seg_len=256, pretrain=32, acq=512)
    z, b, st = W.wl_equalise(x, p)
    assert np.array_equal(z, s)
    assert np.array_equal(b, bits)
    assert np.array_equal(st.taps, W.initial_taps(4))


def test_zero_step_is_the_plain_widely_linear_filter():
    # mu = 0: z_k = (h * x)[2k + c] + (g * conj x)[2k + c], zero outside the buffer
    rng = np.random.default_rng(5)
    K = 1000
    x = rng.standard_normal(2 * K) + 1j * rng.standard_normal(2 * K)
    taps = rng.standard_normal((2, 4)) + 1j * rng.standard_normal((2, 4))
    p = W.WLParams(mod="qpsk", mu=0.0, seg_len=64, pretrain=16, acq=96)
    z, _, st = W.wl_equalise(x, p, W.WLState(taps.copy()))
    c = 1
    full = np.convolve(x, taps[0]) + np.convolve(np.conj(x), taps[1])
    assert np.abs(z - full[2 * np.arange(K) + c]).max() < 1e-12
    assert np.array_equal(st.taps, taps)


def _iq(gain_db, phase_deg):
    return LK.iq_imbalance(LK.KKLink(iq_gain_db=gain_db, iq_phase_deg=phase_deg))


def test_widely_linear_taps_converge_to_the_closed_form_inverse():
    # x = mu s + nu s*: z = h x + g x* = s for h = mu*/(|mu|^2-|nu|^2), g = -nu/(|mu|^2-|nu|^2)
    rng = np.random.default_rng(7)
    bits, s = _symbols(20000, "16qam", 12)
    mu, nu = _iq(1.0, 5.0)
    x0 = _two_sps(s, rng)
    x = mu * x0 + nu * np.conj(x0)
    p = W.WLParams(mod="16qam", mu=1e-2, acq=20000)
    z, b, st = W.wl_equalise(x, p)
    D = abs(mu) ** 2 - abs(nu) ** 2
    want = np.zeros((2, 4), np.complex128)
    want[0, 1], want[1, 1] = np.conj(mu) / D, -nu / D
    assert np.abs(st.taps - want).max() < 1e-6
    assert np.abs(z[-1000:] - s[-1000:]).max() < 1e-6
    assert np.array_equal(b, bits)
    # the strictly linear form cannot remove the image: g stays 0, h[c] goes to the
    # linear Wiener solution E[s x*]/E|x|^2 = mu*/(|mu|^2+|nu|^2) for a proper s
    pl = W.WLParams(mod="16qam", mu=2e-3, acq=20000, linear=True)
    zl, _, stl = W.wl_equalise(x, pl)
    assert np.array_equal(stl.taps[1], np.zeros(4))
    assert abs(stl.taps[0, 1] - np.conj(mu) / (abs(mu) ** 2 + abs(nu) ** 2)) < 1e-2
    evm_l = np.sqrt(np.mean(np.abs(zl[-5000:] - s[-5000:]) ** 2))
    assert abs(evm_l - abs(nu) / math.sqrt(abs(mu) ** 2 + abs(nu) ** 2)) < 0.1 * evm_l


def test_segment_schedule_is_local():
    # segment [s0, s1) depends only on the wave-start taps and the samples its
    # regressors touch over [s0 - W, s1); the end state only on the last segment
    rng = np.random.default_rng(9)
    K, S, Wp = 4096, 512, 64
    bits, s = _symbols(K, "16qam", 13)
    x = _two_sps(s, rng, 0.3) + 0.05 * (rng.standard_normal(2 * K) + 1j * rng.standard_normal(2 * K))
    p = W.WLParams(mod="16qam", mu=5e-3, seg_len=S, pretrain=Wp, acq=1024)
    z, _, st = W.wl_equalise(x, p)
    s0, s1 = 1024 + 2 * S, 1024 + 3 * S        # the third segment
    lo, hi = 2 * (s0 - Wp) - 2, 2 * (s1 - 1) + 1   # samples its regressors read
    y = x.copy()
    y[2 * 1024:lo] *= -1j                       # after the acquisition's last regressor
    y[hi + 1:] *= -1j
    zy, _, sty = W.wl_equalise(y, p)
    assert np.array_equal(zy[s0:s1], z[s0:s1])
    assert not np.allclose(sty.taps, st.taps)  # the last segment saw the change
    # a change inside the pretraining span moves the segment's outputs
    y = x.copy()
    y[2 * (s0 - Wp) + 10] += 0.5
    zy, _, sty = W.wl_equalise(y, p)
    assert not np.array_equal(zy[s0:s1], z[s0:s1])
    # ... but not the end state, which starts from the wave-start taps again
    assert np.array_equal(sty.taps, st.taps)
    # the next call starts from the end state: with mu = 0 it is a fixed filter
    p0 = W.WLParams(mod="16qam", mu=0.0, seg_len=S, pretrain=Wp, acq=1024)
    z2, _, _ = W.wl_equalise(x, p0, W.WLState(st.taps, True))     # no previous samples
    full = np.convolve(x, st.taps[0]) + np.convolve(np.conj(x), st.taps[1])
    assert np.abs(z2 - full[2 * np.arange(K) + 1]).max() < 1e-12


def _q(a):
    return 0.5 * erfc(a / math.sqrt(2.0))


def test_awgn_ber_16qam_matches_theory():
    # AWGN only, Es/N0 = 16 dB: the equaliser at a small step adds no measurable
    # penalty; BER within the 99 % binomial interval of Pb = (3Q(a)+2Q(3a)-Q(5a))/4
    snr = 10 ** (16 / 10)
    K = 1 << 16
    bits, s = _symbols(K, "16qam", 14)
    rng = np.random.default_rng(15)
    sig = math.sqrt(1 / snr / 2)
    x = _two_sps(s, rng, 0.5)
    x[0::2] += sig * (rng.standard_normal(K) + 1j * rng.standard_normal(K))
    p = W.WLParams(mod="16qam", mu=1e-4, acq=4096)
    _, b, _ = W.wl_equalise(x, p)
    n = b.shape[0]
    err = int(np.count_nonzero(b != bits))
    a = math.sqrt(snr / 5)
    pb = (3 * _q(a) + 2 * _q(3 * a) - _q(5 * a)) / 4
    half = 2.576 * math.sqrt(pb * (1 - pb) / n)
    assert err >= 200
    assert abs(err / n - pb) < half, (err / n, pb, half)


def test_previous_buffer_samples_continue_the_regressor():
    # two calls on the halves of x equal one call on x when the second call sees
    # the first's last samples and starts from its taps: check at mu = 0 against
    # the plain convolution of the whole x
    rng = np.random.default_rng(21)
    K = 600
    x = rng.standard_normal(2 * K) + 1j * rng.standard_normal(2 * K)
    taps = rng.standard_normal((2, 4)) + 1j * rng.standard_normal((2, 4))
    p = W.WLParams(mod="qpsk", mu=0.0, seg_len=64, pretrain=16, acq=0)
    z1, _, st = W.wl_equalise(x[:K], p, W.WLState(taps.copy()))
    z2, _, _ = W.wl_equalise(x[K:], p, st)
    full = np.convolve(x, taps[0]) + np.convolve(np.conj(x), taps[1])
    z = np.concatenate([z1, z2])
    # symbol k reads x[2k-2 .. 2k+1]: within its own buffer except the 2 samples before it
    assert np.abs(z - full[2 * np.arange(K) + 1]).max() < 1e-12
    # without the previous samples the first symbol of the second half would differ
    z2b, _, _ = W.wl_equalise(x[K:], p, W.WLState(st.taps, True))
    assert abs(z2b[0] - z2[0]) > 1e-3 and np.array_equal(z2b[1:], z2[1:])
