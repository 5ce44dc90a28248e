"""CPU pins of the oracle's segment schedule, frequency-tracker grid, per-region
noise variance and near-tie rules.  Each test fixes a property that a plausible
mistake (the wrong segment seeding the next wave, a pre-training span off by a
block, a region boundary off by one, a wrong rotation sign or phase origin, a
tie rule that takes a choice outside its band) would break.
"""
import math

import numpy as np

import linksim as L
import oracle as O
from oracle import chain as C

# a short schedule: acquisition 1024 symbols, segments of 256 pre-trained on 64,
# 8 segments per wave (block of 4096 samples)
SCHED = dict(n_cma=1024, acq_min=1024, seg_len=256, seg_pretrain=64, block_samples=4096, L_km=0.0)


def _mixed_stream(K, seed, mod="qpsk", snr_db=16.0):
    """2-sps butterfly input: symbols through a fixed 2x2 mixing at even samples,
    noise everywhere (odd samples carry only noise)."""
    m = L.bits_per_symbol(mod)
    s = L.map_symbols(L.random_bits(seed, 2 * m * K).reshape(2, -1), mod)
    J = np.array([[0.9, 0.3 - 0.2j], [-0.25 + 0.1j, 0.95]])
    rng = np.random.default_rng(seed)
    sig = math.sqrt(10 ** (-snr_db / 10) / 2)
    u = sig * (rng.standard_normal((2, 2 * K)) + 1j * rng.standard_normal((2, 2 * K)))
    u[:, ::2] += J @ s
    return u, s


def _segments(p, K):
    A = p.acq_len(K)
    G = -(-(K - A) // p.seg_len)
    return A, [(A + g * p.seg_len, min(A + (g + 1) * p.seg_len, K)) for g in range(G)]


def test_wave_starts_from_last_segment_end_taps():
    # wave w+1 starts from the taps the LAST segment of wave w ends with, having
    # started from wave w's start taps and pre-trained over the W symbols before it
    p = O.RxParams(**SCHED, fo_track=False).resolved()
    K = 1024 + 3 * 8 * 256
    u, _ = _mixed_stream(K, 41)
    tr = {}
    O.equalize(u, p, tr)
    A, segs = _segments(p, K)
    P, c, T = p.wave_segments(), (p.ntaps - 1) // 2, p.ntaps
    phis = O.bps_outer_angles(p.bps_angles)
    assert len(tr["wave_taps"]) == 3
    for w in range(2):
        ks, ke = segs[(w + 1) * P - 1]
        win = C._Window(u, ks - p.seg_pretrain, ke, c)
        hh = tr["wave_taps"][w]
        for k0 in range(ks - p.seg_pretrain, ke, p.upd_block):
            _, hh = O.lms_step(hh, win.taps_input(k0, min(k0 + p.upd_block, ke), T, c), "dd", p, phis)
        assert np.array_equal(tr["wave_taps"][w + 1], hh)
        # ... and not from the first segment's
        ks0, ke0 = segs[w * P]
        win0 = C._Window(u, ks0 - p.seg_pretrain, ke0, c)
        h0 = tr["wave_taps"][w]
        for k0 in range(ks0 - p.seg_pretrain, ke0, p.upd_block):
            _, h0 = O.lms_step(h0, win0.taps_input(k0, min(k0 + p.upd_block, ke0), T, c), "dd", p, phis)
        assert not np.allclose(tr["wave_taps"][w + 1], h0)


def test_segment_schedule_is_local():
    p = O.RxParams(**SCHED, fo_track=False).resolved()
    K = 1024 + 3 * 8 * 256
    u, _ = _mixed_stream(K, 43)
    y = O.equalize(u, p)
    A, segs = _segments(p, K)
    P = p.wave_segments()
    W = p.seg_pretrain

    def rerun(mod):
        v = u.copy()
        mod(v)
        tr = {}
        return O.equalize(v, p, tr), tr

    _, tr0 = rerun(lambda v: None)
    # (1) samples read only by the last segment of wave 0: the other segments of wave 0
    #     are unchanged, wave 1 starts from other taps and its outputs move
    ks, ke = segs[P - 1]
    lo, hi = 2 * ks + 16, 2 * (ke - W) - 16
    y1, tr1 = rerun(lambda v: v.__setitem__((slice(None), slice(lo, hi)), v[:, lo:hi] * 1.3))
    for g in range(P - 1):
        a, b = segs[g]
        assert np.array_equal(y1[:, a:b], y[:, a:b]), g
    assert not np.allclose(tr1["wave_taps"][1], tr0["wave_taps"][1])
    a, b = segs[P]
    assert not np.allclose(y1[:, a:b], y[:, a:b])
    # (2) samples read only by a middle segment of wave 0: only that segment moves;
    #     wave 1 starts from the same taps and all its outputs are unchanged
    g = 3
    ks, ke = segs[g]
    lo, hi = 2 * ks + 16, 2 * (ke - W) - 16
    y2, tr2 = rerun(lambda v: v.__setitem__((slice(None), slice(lo, hi)), v[:, lo:hi] * 1.3))
    for h in range(len(segs)):
        a, b = segs[h]
        if h == g:
            assert not np.allclose(y2[:, a:b], y[:, a:b])
        else:
            assert np.array_equal(y2[:, a:b], y[:, a:b]), h
    assert np.array_equal(tr2["wave_taps"][1], tr0["wave_taps"][1])
    # (3) the pre-training span is exactly W symbols: a sample 8 symbols before it does
    #     not move segment g + 1 (it lies in segment g's own span), one 8 symbols inside it does
    ks1, ke1 = segs[g + 1]
    n_out = 2 * (ks1 - W - 8)
    y3, _ = rerun(lambda v: v.__setitem__((slice(None), n_out), v[:, n_out] + 0.7))
    assert np.array_equal(y3[:, ks1:ke1], y[:, ks1:ke1])
    assert not np.array_equal(y3[:, ks:ke], y[:, ks:ke])
    n_in = 2 * (ks1 - W + 8)
    y4, _ = rerun(lambda v: v.__setitem__((slice(None), n_in), v[:, n_in] + 0.7))
    assert not np.array_equal(y4[:, ks1:ke1], y[:, ks1:ke1])


# --------------------------------------------------------------- tracker grid
def test_fo_units_grid_rounding():
    sps = 2
    q = sps * 2 * math.pi / (1 << C.FO_GRID_BITS)        # rad/symbol per unit
    for u in (-3000, -1, 0, 1, 17, 2600):
        got, edge = C.fo_units(u * q, sps)
        assert got == u and abs(edge - 0.5) < 1e-6
        assert abs(C.units_to_rate(u, sps) - u * q) < 1e-15
    # half-way (to within the conversion's rounding) sits on the rounding boundary:
    # edge ~ 0, either neighbour
    for u in (4, 5, -7):
        got, edge = C.fo_units((u + 0.5) * q, sps)
        assert got in (u, u + 1) and edge < 1e-9
    got, edge = C.fo_units(10.3 * q, sps)
    assert got == 10 and abs(edge - 0.2) < 1e-9
    # phases: 2^(G-1) units is -pi (the signed range [-pi, pi)), whole turns vanish
    M = 1 << C.FO_GRID_BITS
    assert C.units_to_phase(M // 2) == -math.pi
    assert C.units_to_phase(3 * M + M // 4) == math.pi / 2
    assert C.units_to_phase(-M // 4) == -math.pi / 2


def test_tracker_removes_a_grid_exact_offset_exactly():
    # noise-free QPSK at even samples turned by a frequency offset of exactly d
    # units (2 pi d / 2^G rad per sample), d a multiple of 32 so that the phase is a
    # whole turn at sample 2 N_CMA (where the DD part's rotation starts): the CMA
    # leaves the identity taps alone (unit modulus), the 4th-power estimate is exact
    # and rounds to d, every rotation removes the offset exactly, the DD error is 0,
    # every per-wave step is 0, and the phase bases follow the closed form
    p = O.RxParams(**SCHED).resolved()
    K = 1024 + 3 * 8 * 256 + 100
    d = 32 * 37
    M = 1 << C.FO_GRID_BITS
    s = L.map_symbols(L.random_bits(45, 2 * 2 * K).reshape(2, -1), "qpsk")
    n = np.arange(2 * K)
    u = np.zeros((2, 2 * K), np.complex128)
    u[:, ::2] = s
    u = u * np.exp(1j * 2 * math.pi * ((n * d) % M) / M)
    tr = {}
    y = O.equalize(u, p, tr)
    A = p.acq_len(K)
    assert tr["acq_units"] == d
    assert np.max(np.abs(y[:, 2 * p.n_cma // 2:] - s[:, p.n_cma:])) < 1e-9
    PS = p.wave_segments() * p.seg_len
    for w, (phi, dw) in enumerate(tr["wave_units"]):
        assert dw == d
        assert phi == ((2 * A - 2 * p.n_cma) * d + w * 2 * PS * d) % M


def test_tracker_applies_each_wave_estimate_two_waves_on():
    # noise-free QPSK with a grid-exact offset d (as above) up to the start of wave 1,
    # then d + J: wave 0 sees no residual (its step is 0), wave 1 sees J.  Wave 1's
    # estimate moves the rate first at wave 3: d_0 = d_1 = d_2 = d, d_3 > d, and the
    # phase bases integrate the rates wave by wave
    p = O.RxParams(**SCHED).resolved()
    P, S = p.wave_segments(), p.seg_len
    K = 1024 + 5 * P * S
    d, J = 32 * 37, 32
    M = 1 << C.FO_GRID_BITS
    A = p.acq_len(K)
    n1 = 2 * (A + P * S)                       # first sample of wave 1
    s = L.map_symbols(L.random_bits(46, 2 * 2 * K).reshape(2, -1), "qpsk")
    n = np.arange(2 * K)
    ph = np.where(n < n1, n * d, n1 * d + (n - n1) * (d + J)) % M
    u = np.zeros((2, 2 * K), np.complex128)
    u[:, ::2] = s
    u = u * np.exp(1j * 2 * math.pi * ph / M)
    tr = {}
    O.equalize(u, p, tr)
    units = tr["wave_units"]
    assert len(units) == 5 and tr["acq_units"] == d
    assert [dw for _, dw in units[:3]] == [d, d, d]
    assert tr["wave_r"][0] == 0.0 or abs(tr["wave_r"][0]) < 1e-12
    inc1, _ = C.fo_units(tr["wave_r"][1] / p.fo_smooth, p.sps)
    assert inc1 > 0 and units[3][1] == d + inc1
    for w in range(4):
        assert units[w + 1][0] == (units[w][0] + 2 * P * S * units[w][1]) % M


def test_window_rotation_is_the_exact_integer_phase():
    # _Window turns sample n by exp(-j 2 pi ((phi + (n - n0) d) mod 2^G) / 2^G)
    M = 1 << C.FO_GRID_BITS
    rng = np.random.default_rng(2)
    u = rng.standard_normal((2, 500)) + 1j * rng.standard_normal((2, 500))
    phi, n0, d = 12345, 3, -4567
    win = C._Window(u, 10, 200, 7, phi, n0, d)
    idx = np.arange(win.lo, win.lo + win.seg.shape[1])
    ok = (idx >= 0) & (idx < 500)
    ref = np.array([u[:, i] * np.exp(-2j * math.pi * (((phi + (i - n0) * d) % M) / M)) for i in idx[ok]]).T
    assert np.max(np.abs(win.seg[:, ok] - ref)) < 1e-13


# --------------------------------------------------------------- near-tie rules
def test_inner_choice_is_taken_only_at_a_near_tie():
    # QPSK turned by exactly half-way between test angles b and b+1: the two block
    # sums are equal (distances under +-delta mirror each other), the oracle takes b
    # (smallest index); another implementation's b+1 is taken and logged, b+5 is not
    p = O.RxParams().resolved()
    phis = O.bps_outer_angles(p.bps_angles)
    b = 11
    mid = 0.5 * (phis[b] + phis[b + 1])
    s = L.map_symbols(L.random_bits(3, 2 * 2 * 32).reshape(2, -1), "qpsk")
    X = np.zeros((32, 2, p.ntaps), np.complex128)
    c = (p.ntaps - 1) // 2
    X[:, 0, c] = s[0] * np.exp(1j * mid)
    X[:, 1, c] = s[1] * np.exp(1j * mid)
    h = np.zeros((2, 2, p.ntaps), np.complex128)
    h[0, 0, c] = h[1, 1, c] = 1.0
    _, h_own = O.lms_step(h, X, "dd", p, phis)
    log = []
    _, h_b1 = O.lms_step(h, X, "dd", p, phis, choice=[b + 1, b + 1], log=log, where="t")
    assert len(log) == 2 and all(e[3] == b and e[4] == b + 1 and e[5] < 1e-12 for e in log)
    assert not np.allclose(h_b1, h_own)
    # the update with b+1 is the mirror image: the same step size, the opposite turn
    assert abs(np.linalg.norm(h_b1 - h) - np.linalg.norm(h_own - h)) < 1e-12
    log = []
    _, h_far = O.lms_step(h, X, "dd", p, phis, choice=[b + 5, -1], log=log)
    assert log == [] and np.array_equal(h_far, h_own)


def test_tracker_choice_is_taken_only_at_a_near_tie():
    log = []
    assert C._track_tie(7, 1e-3, 8, "wave", 0, log) == 8 and len(log) == 1
    assert C._track_tie(7, 1e-3, 6, "wave", 1, log) == 6 and len(log) == 2
    assert C._track_tie(7, 1e-3, 9, "wave", 2, log) == 7      # not a neighbour
    assert C._track_tie(7, 0.1, 8, "wave", 3, log) == 7       # not near half-way
    assert C._track_tie(7, 0.0, None, "wave", 4, log) == 7
    assert len(log) == 2


# --------------------------------------------------------------- demap regions
def test_region_sigma2_and_llr_scale():
    # symbols displaced from their constellation point by a fixed distance eps per
    # (pol, region), well inside the decision regions: sigma^2 of each region is
    # exactly eps^2, so a region boundary off by one symbol or a wrong error term
    # shows; the QPSK LLRs are the closed form 2 sqrt2 x / sigma^2
    p = O.RxParams(**SCHED).resolved()
    K = 1024 + 2 * 8 * 256 + 333
    regs = O.region_bounds(K, p)
    assert regs[0] == (0, 1024) and regs[1] == (1024, 1024 + 2048) and regs[-1][1] == K
    s = L.map_symbols(L.random_bits(47, 2 * 2 * K).reshape(2, -1), "qpsk")
    rng = np.random.default_rng(5)
    eps = 0.02 + 0.1 * rng.random((2, len(regs)))
    psi = rng.uniform(0, 2 * math.pi, (2, K))
    z = s.copy()
    for j, (a, b) in enumerate(regs):
        z[:, a:b] += eps[:, j:j + 1] * np.exp(1j * psi[:, a:b])
    bits, llr, sig = O.demap(z, p)
    assert np.max(np.abs(sig / eps ** 2 - 1)) < 1e-12
    assert np.array_equal(bits, O.hard_bits(s, "qpsk"))
    for j, (a, b) in enumerate(regs):
        for pp in range(2):
            ref = np.stack([z[pp, a:b].real, z[pp, a:b].imag], axis=-1).reshape(-1) * 2 * math.sqrt(2) / eps[pp, j] ** 2
            assert np.max(np.abs(llr[pp, 2 * a:2 * b] - ref)) < 1e-9 * np.max(np.abs(ref))
