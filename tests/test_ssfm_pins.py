"""Pins of the split-step link simulator (test infrastructure for the learned
post-equaliser) against closed forms: linear propagation, pure self-phase
modulation, ASE power, the low-pass front end and second-order convergence of
the symmetric split."""
import math

import numpy as np
import pytest

import linksim as L
from linksim import ssfm as F

torch = pytest.importorskip("torch")


def _tx(n_sym=512, sps=4, seed=3):
    bits = L.random_bits(seed, 2 * 4 * n_sym).reshape(2, -1)
    return L.tx_shape(L.map_symbols(bits, "16qam"), 32e9, 0.1, sps)


def _run(x, link, fs, noise=None):
    A = torch.from_numpy(x).to(torch.complex128)
    return F.propagate(A, link, fs, torch, noise).numpy()


def test_linear_link_equals_whole_stream_dispersion():
    # gamma = 0, no ASE: loss and gain cancel per span, dispersion accumulates over L
    link = F.SSFMLink(spans=3, span_km=80.0, step_km=10.0, gamma=0.0, ase=False)
    x = _tx() * 1e-2
    fs = 4 * 32e9
    y = _run(x, link, fs)
    ref = L.apply_dispersion(x, fs, link.L_km, link.D, link.lam_nm)
    assert np.linalg.norm(y - ref) / np.linalg.norm(ref) < 1e-10


def test_pure_spm_closed_form():
    # beta2 = 0 and alpha = 0: |A| stays constant, the Manakov phase is (8/9) gamma |A|^2 L
    link = F.SSFMLink(spans=2, span_km=50.0, step_km=5.0, D=0.0, alpha_db_km=0.0, ase=False)
    x = _tx() * 0.03
    y = _run(x, link, 4 * 32e9)
    p = np.sum(np.abs(x) ** 2, axis=0, keepdims=True)
    ref = x * np.exp(1j * (8.0 / 9.0) * link.gamma * p * link.L_km)
    assert np.max(np.abs(y - ref)) / np.max(np.abs(ref)) < 1e-12


def test_ase_power_per_span():
    link = F.SSFMLink(spans=3, span_km=100.0, step_km=50.0, gamma=0.0)
    fs = 4 * 32e9
    n = 1 << 16
    gen = torch.Generator().manual_seed(11)
    y = _run(np.zeros((2, n), np.complex128), link, fs, lambda s: torch.randn(s, generator=gen, dtype=torch.float64))
    G = math.exp(link.alpha * link.span_km)
    var1 = 10 ** (link.nf_db / 10) / 2 * F.H_PLANCK * F.C_LIGHT / (link.lam_nm * 1e-9) * (G - 1) * fs
    # each span's noise is attenuated then restored by the next gain: 3 spans add 3 x var1
    meas = np.mean(np.abs(y) ** 2)
    assert abs(meas / (3 * var1) - 1) < 0.02
    assert abs(np.mean(y.real * y.imag)) < 0.02 * meas       # circular


def test_lowpass_keeps_in_band_tones_and_removes_the_rest():
    n, m = 1024, 512
    t = np.arange(n)
    x = np.exp(2j * np.pi * 37 * t / n) + 0.5 * np.exp(-2j * np.pi * 100 * t / n) + np.exp(2j * np.pi * 400 * t / n)
    y = F.lowpass_resample(torch.from_numpy(x[None]), m, torch).numpy()[0]
    tt = np.arange(m)
    ref = np.exp(2j * np.pi * 37 * tt / m) + 0.5 * np.exp(-2j * np.pi * 100 * tt / m)
    assert np.max(np.abs(y - ref)) < 1e-12


def test_symmetric_split_is_second_order():
    # error against a fine-step reference falls ~4x per halving of dz (in the asymptotic range)
    base = dict(spans=1, span_km=100.0, ase=False)
    x = _tx(256) * 0.05
    fs = 4 * 32e9
    ref = _run(x, F.SSFMLink(step_km=100.0 / 1024, **base), fs)
    errs = [np.linalg.norm(_run(x, F.SSFMLink(step_km=100.0 / k, **base), fs) - ref) for k in (32, 64, 128)]
    assert 3.3 < errs[0] / errs[1] < 5.0 and 3.3 < errs[1] / errs[2] < 5.0
