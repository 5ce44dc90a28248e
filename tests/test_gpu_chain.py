"""GPU parity: the CUDA chain (through the C ABI) against the FP64 oracle on the
same seeded inputs, element by element.

Tolerances (FP32 path vs FP64 oracle): complex outputs of CDC, equaliser and
BPS within 1e-4 relative RMS; equaliser taps at each wave within 1e-4 relative
RMS; hard bits identical except where the oracle's soft value lies within 1e-5
of a decision boundary; BPS angle choices identical except at oracle near-ties
(best and second-best window sums within 1e-5 relative), after which the
comparison resumes from the next agreeing symbol.
"""
import dataclasses
import math

import numpy as np
import pytest

import linksim as L
import oracle as O
from chain_helpers import (REL_RMS_TOL, boundary_mask, bps_near_tie, device_ties, ensure_built, rel_rms,
                           rx_params, run_gpu)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    ensure_built()


def _theta(z, y):
    return np.angle(y * np.conj(z))       # z = y e^{-j theta}


def gpu_tracker(rx, p, K):
    """The device's equaliser state per wave: taps at each wave start, dw, Phi."""
    A = p.acq_len(K)
    S, P = p.seg_len, p.wave_segments()
    n_waves = -(-max(K - A, 0) // S)
    n_waves = -(-n_waves // P)
    h_acq, dw_acq, _ = rx.trace(-1)
    waves = [rx.trace(w) for w in range(n_waves)]
    return dict(acq_dw=dw_acq, acq_taps=h_acq, wave_taps=[w[0] for w in waves],
                wave_dw=[w[1] for w in waves], wave_Phi=[w[2] for w in waves])


def check_chain(p, g, gpu, trace=None, check_taps=True):
    """Compare every stage of one run; returns a dict of the measured errors.

    The oracle runs on its own decisions.  Where one of them is a near-tie
    (inner BPS window sums within INNER_TIE_REL, a tracker rounding within
    TRACK_TIE_UNITS of half-way) both candidates are correct; the oracle then
    follows the one the device took, and reports how often it did.  The
    frequency tracker's integer state must then equal the device's at every
    wave exactly.
    """
    K = g.samples.shape[0] // 2
    dev = gpu_tracker(gpu["rx"], p, K)
    ties = device_ties(gpu["rx"], p, K)
    trace = {} if trace is None else trace
    orc = O.run_chain(g.samples, p, trace, ties)
    assert gpu["n"] == K
    rep = {}
    rep["ties"] = len(trace["ties"])
    rep["tie_kinds"] = sorted({t[0] for t in trace["ties"]})
    rep["tie_gap_max"] = max((t[-1] for t in trace["ties"]), default=None)
    rep["fo_edge_min"] = min(trace["fo_edge"]) if trace["fo_edge"] else None
    # the frequency tracker (integers on the 2^-G turns grid): identical at every wave
    assert ties["acq_units"] == trace["acq_units"], (ties["acq_units"], trace["acq_units"])
    assert ties["wave_units"] == trace["wave_units"], [
        (w, a, b) for w, (a, b) in enumerate(zip(ties["wave_units"], trace["wave_units"])) if a != b][:5]
    # CDC
    rep["cdc"] = rel_rms(gpu["u"][:, :2 * K], orc["u"])
    assert gpu["cdc_n"] == 2 * K
    assert rep["cdc"] < REL_RMS_TOL, rep
    # equaliser
    rep["y"] = rel_rms(gpu["y"], orc["y"])
    assert rep["y"] < REL_RMS_TOL, rep
    # BPS: angle decisions (inferred from z = y e^{-j theta}) agree up to pi/2 except at near-ties
    dth = _theta(gpu["z"], gpu["y"]) - _theta(orc["z"], orc["y"])
    q = np.round(dth / (math.pi / 2))
    off = np.abs(dth - q * math.pi / 2)
    tie = bps_near_tie(orc["y"], p)
    bad = off > 1e-3
    assert not np.any(bad & ~tie), f"BPS disagrees away from near-ties at {np.argwhere(bad & ~tie)[:5]}"
    qm = np.mod(q, 4).astype(int)
    # pi/2 offsets may only appear after a near-tie flip changed the unwrap count
    for pp in range(2):
        ch = np.nonzero(np.diff(qm[pp]) != 0)[0] + 1
        for k in ch:
            assert tie[pp, max(k - 1, 0):k + 1].any() or bad[pp, max(k - 1, 0):k + 1].any(), (pp, k)
    ok = ~bad & (qm == 0)
    rep["z"] = rel_rms(gpu["z"][ok], orc["z"][ok])
    rep["z_agree"] = float(ok.mean())
    assert rep["z"] < REL_RMS_TOL, rep
    # hard bits
    m = p.bits
    bmask = boundary_mask(orc["z"], p.mod)
    okb = np.repeat(ok, m, axis=1) & ~bmask
    mism = (gpu["bits"] != orc["bits"]) & okb
    rep["bit_mismatch"] = int(mism.sum())
    rep["exempt_bits"] = int(((gpu["bits"] != orc["bits"]) & ~okb).sum())
    assert rep["bit_mismatch"] == 0, rep
    # LLRs
    rep["llr"] = rel_rms(gpu["llr"][okb], orc["llr"][okb])
    assert rep["llr"] < REL_RMS_TOL, rep
    # equaliser taps at every wave start
    if check_taps:
        assert rel_rms(dev["acq_taps"], trace["acq_taps"]) < REL_RMS_TOL
        worst = 0.0
        for w, ht in enumerate(trace["wave_taps"]):
            worst = max(worst, rel_rms(dev["wave_taps"][w], ht))
        rep["taps"] = worst
        assert worst < REL_RMS_TOL, rep
    return rep, orc


def test_c1_full_chain_parity():
    """Single channel DP-QPSK 10 GBd, 2^16 symbols/pol, 1000 km, fixed Jones, 12 dB, FP32, N=1024."""
    lk = L.workload("c1")
    g = L.generate(lk)
    p = rx_params(lk, g.in_scale, fft_n=1024)
    gpu = run_gpu(p, g.samples)
    rep, orc = check_chain(p, g, gpu)
    print("c1 parity", rep)
    # BER through the GPU counter equals the oracle's count on the same bits
    import torch
    ref = torch.from_numpy(L.pack_bits(g.tx_bits).view(np.int32)).cuda()
    e, n, sync = gpu["rx"].ber(gpu["bits_t"], ref, lk.n_sym)
    eo, no, so = O.ber_sync_count(gpu["bits"], g.tx_bits, p.mod, p.acq_len(lk.n_sym))
    assert (e, n) == (eo, no) and sync == so


def test_c2_shape_int8_short_parity():
    """10,000 km shape (int8 ADC, PMD, 100 kHz phase noise, 200 MHz FO, 9.8 dB), 2^17 symbols."""
    lk = L.workload("c2", n_sym=1 << 17)
    g = L.generate(lk)
    p = rx_params(lk, g.in_scale)
    assert p.fft_n == 4096 and p.overlap == 544
    gpu = run_gpu(p, g.samples)
    tr = {}
    rep, _ = check_chain(p, g, gpu, tr)
    print("c2-short parity", rep)


def test_16qam_parity():
    """DP-16QAM 32 GBd, 2000 km (N_CD 1117 -> V 1120, N 8192), 18 dB, int8, phase noise."""
    lk = dataclasses.replace(L.workload("c3", n_sym=1 << 16), L_km=2000.0)
    g = L.generate(lk)
    p = rx_params(lk, g.in_scale)
    assert p.fft_n == 8192
    gpu = run_gpu(p, g.samples)
    rep, _ = check_chain(p, g, gpu, {})
    print("16qam parity", rep)


def test_c3_16qam_6000km_parity():
    """DP-16QAM 32 GBd over 6000 km (N_CD 3349 -> V 3360, N 16384: one CTA per window and pol)."""
    lk = L.workload("c3", n_sym=1 << 16)
    g = L.generate(lk)
    p = rx_params(lk, g.in_scale)
    assert p.fft_n == 16384 and p.overlap == 3360
    gpu = run_gpu(p, g.samples)
    rep, _ = check_chain(p, g, gpu, {})
    print("c3 parity", rep)


@pytest.mark.parametrize("mod", ["qpsk", "16qam"])
def test_eq_eight_warps_per_row_parity(mod):
    """The equaliser's butterfly row split over 8 warps (4 taps and 4 inner angles per
    lane) follows the oracle as the default 4-warp split does: QPSK on the 10,000 km
    shape (FO, phase noise, PMD), 16QAM on a 2000 km link."""
    if mod == "qpsk":
        lk = L.workload("c2", n_sym=1 << 16)
    else:
        lk = dataclasses.replace(L.workload("c3", n_sym=1 << 16), L_km=2000.0)
    g = L.generate(lk)
    p = rx_params(lk, g.in_scale)
    gpu = run_gpu(p, g.samples, EQ_WARPS=8)
    assert gpu["rx"].get_param("EQ_WARPS") == 8
    rep, _ = check_chain(p, g, gpu, {})
    print("8 warps", mod, rep)


@pytest.mark.parametrize("chunk", [None, 40_000 * 2 + 64])
def test_eq_two_banks_are_identical(chunk):
    """Segments on two banks of CTA pairs taking the waves by turns (RX_P_EQ_ALT = 1, the
    default: 4 P CTAs) against one bank for every wave (2 P CTAs): the same update chain in
    the same order, so the equaliser output, the taps at every wave and the bits are
    identical, in one call and streamed (each call its own launches), with a ragged
    last wave."""
    lk = L.workload("c2", n_sym=(1 << 17) + 3 * 1024 + 77)
    g = L.generate(lk)
    p = rx_params(lk, g.in_scale)
    runs = {a: run_gpu(p, g.samples, chunk=chunk, EQ_ALT=a) for a in (0, 1)}
    assert runs[1]["rx"].get_param("EQ_ALT") == 1 and runs[0]["rx"].get_param("EQ_ALT") == 0
    assert runs[0]["n"] == runs[1]["n"]
    assert np.array_equal(runs[0]["y"], runs[1]["y"])
    assert np.array_equal(runs[0]["words"], runs[1]["words"])
    assert np.array_equal(runs[0]["llr"], runs[1]["llr"])
    n_waves = -(-(runs[0]["n"] - p.acq_len(runs[0]["n"])) // (p.wave_segments() * p.seg_len))
    for w in range(-1, n_waves):
        t0, t1 = runs[0]["rx"].trace(w), runs[1]["rx"].trace(w)
        assert all(np.array_equal(np.asarray(a), np.asarray(b)) for a, b in zip(t0, t1)), w


@pytest.mark.parametrize("adc,chunk", [("int8", None), ("int8", 30_000 * 2 + 64), ("f32", None)])
def test_cdc_four_step_4096(adc, chunk):
    """N = 4096 as 64 x 64 register DFTs (RX_P_CDC_4STEP = 1, the default) and as the
    radix-16 Stockham plan (0): both against the FP64 oracle's overlap-save output,
    int8 and FP32 input, one call and streamed (windows across the carried tail)."""
    lk = L.Link(n_sym=70_000 + 321, L_km=4000.0, snr_db=14.0, adc=adc, seed=4096)
    g = L.generate(lk)
    p = rx_params(lk, g.in_scale, fft_n=4096)
    assert p.fft_n == 4096
    orc_u = O.cdc_overlap_save(L.deinterleave(g.samples) * g.in_scale, O.cdc_filter(p), p.overlap)
    us = {}
    for fs in (0, 1):
        gpu = run_gpu(p, g.samples, chunk=chunk, CDC_4STEP=fs)
        assert gpu["rx"].get_param("CDC_4STEP") == fs
        us[fs] = gpu["u"][:, :orc_u.shape[1]]
        err = rel_rms(us[fs], orc_u)
        print(f"CDC_4STEP={fs} {adc} chunk={chunk}: rel RMS vs FP64 {err:.2e}")
        assert err < 1e-6, (fs, err)
    assert rel_rms(us[1], us[0]) < 1e-6


@pytest.mark.parametrize("N", [256, 512, 2048, 4096, 8192, 16384])
def test_cdc_fft_sizes(N):
    lk = L.Link(n_sym=20000 + 123, L_km=300.0, snr_db=15.0, seed=77 + N)
    g = L.generate(lk)
    p = rx_params(lk, g.in_scale, fft_n=N, overlap=64)
    gpu = run_gpu(p, g.samples)
    orc_u = O.cdc_overlap_save(L.deinterleave(g.samples), O.cdc_filter(p), p.overlap)
    assert rel_rms(gpu["u"][:, :orc_u.shape[1]], orc_u) < REL_RMS_TOL


@pytest.mark.parametrize("K", [3000, 16384 + 1000 + 37 * 2, (1 << 16) + 4444])
def test_short_and_ragged_streams(K):
    """Acquisition-only streams (K < A), a partial first wave, a ragged last segment."""
    lk = L.Link(n_sym=K, L_km=500.0, snr_db=13.0, seed=1000 + K)
    g = L.generate(lk)
    p = rx_params(lk, g.in_scale)
    gpu = run_gpu(p, g.samples)
    rep, _ = check_chain(p, g, gpu, {})
    print("ragged", K, rep)


def test_small_waves_many_segments():
    """Shorter segments and waves (S=256, W=64, 8 segments per wave) exercise the wave loop."""
    lk = L.Link(n_sym=1 << 15, L_km=800.0, snr_db=12.0, fo_hz=50e6, seed=555)
    g = L.generate(lk)
    p = rx_params(lk, g.in_scale, seg_len=256, seg_pretrain=64, block_samples=4096, n_cma=4096, acq_min=4096)
    gpu = run_gpu(p, g.samples)
    tr = {}
    rep, _ = check_chain(p, g, gpu, tr)
    assert len(tr["wave_taps"]) > 10
    print("small waves", rep)


def test_streaming_calls_equal_one_call():
    """Any split of the stream into calls gives bit-identical results on the GPU."""
    lk = L.workload("c2", n_sym=1 << 16)
    g = L.generate(lk)
    p = rx_params(lk, g.in_scale)
    one = run_gpu(p, g.samples)
    for chunk in (1 << 16, 3 * 4096 + 2, 50000):
        many = run_gpu(p, g.samples, chunk=chunk, reserve=1 << 17)
        assert many["n"] == one["n"]
        assert np.array_equal(many["y"], one["y"]), chunk
        assert np.array_equal(many["words"], one["words"]), chunk
        assert np.array_equal(many["llr"], one["llr"]), chunk


@pytest.mark.parametrize("Nb", [0, 7, 24, 32, 64])
def test_bps_other_half_windows(Nb):
    """Half windows 0, 7 and 24 take the sliding-ring BPS pass; whole multiples of 16
    (16, 32, 64) take the register blocks (for 32 and 64 with block totals between
    the two edge blocks); with phase noise the unwrap count moves, so the scan's
    boundary step of every chunk is exercised, in one call and across calls."""
    lk = L.Link(n_sym=(1 << 15) + 321, L_km=500.0, snr_db=13.0, linewidth_hz=1e6, seed=2300 + Nb)
    g = L.generate(lk)
    p = rx_params(lk, g.in_scale, bps_halfwin=Nb)
    one = run_gpu(p, g.samples)
    rep, _ = check_chain(p, g, one, {})
    print("BPS half window", Nb, rep)
    many = run_gpu(p, g.samples, chunk=3 * 4096 + 2, reserve=1 << 16)
    assert np.array_equal(many["words"], one["words"])
    assert np.array_equal(many["llr"], one["llr"])


def test_fp16_llr_output():
    """LLR_OUT = 2 writes the FP32 path's LLRs rounded to binary16 (nearest even)."""
    import torch
    from chain_helpers import make_receiver
    lk = L.Link(n_sym=20000, L_km=300.0, snr_db=12.0, seed=4242)
    g = L.generate(lk)
    p = rx_params(lk, g.in_scale)
    x = torch.from_numpy(g.samples).cuda()
    got = []
    for mode in (1, 2):
        rx = make_receiver(p, LLR_OUT=mode)
        out = rx.alloc_out(lk.n_sym + 64, llr=True)
        _, n1, _, _ = rx.process(x, out, 0)
        _, n2, _, _ = rx.process(None, out, n1)
        torch.cuda.synchronize()
        assert n1 + n2 == lk.n_sym
        assert out["llr"].dtype == (torch.float32 if mode == 1 else torch.float16)
        got.append((out["llr"][:, :lk.n_sym * p.bits].cpu().numpy(), out["bits"].cpu().numpy()))
        rx.close()
    (l32, b32), (l16, b16) = got
    assert np.array_equal(b32, b16)
    assert np.array_equal(l16, l32.astype(np.float16))


def test_state_save_restore_resumes_bit_exactly():
    import torch
    from chain_helpers import make_receiver
    lk = L.workload("c2", n_sym=1 << 16)
    g = L.generate(lk)
    p = rx_params(lk, g.in_scale)
    ref = run_gpu(p, g.samples, chunk=1 << 15, reserve=1 << 15)
    x = torch.from_numpy(g.samples).cuda()
    K = lk.n_sym
    a = make_receiver(p)
    a.reserve(1 << 15)
    out = a.alloc_out(K + 64)
    pos = 0
    half = (2 * K) // 2
    for s in range(0, half, 1 << 15):
        _, n, _, _ = a.process(x[s:s + (1 << 15)], out, sym_offset=pos)
        pos += n
    blob = a.get_state()
    a.close()
    b = make_receiver(p)
    b.set_state(blob)
    for s in range(half, 2 * K, 1 << 15):
        _, n, _, _ = b.process(x[s:s + (1 << 15)], out, sym_offset=pos)
        pos += n
    _, n, _, _ = b.process(None, out, sym_offset=pos)
    pos += n
    torch.cuda.synchronize()
    assert pos == K
    assert np.array_equal(out["bits"].cpu().numpy().view(np.uint32), ref["words"])


def test_flush_of_empty_stream_emits_nothing():
    from chain_helpers import make_receiver
    p = rx_params(L.Link(), 1.0)
    rx = make_receiver(p)
    out = rx.alloc_out(64)
    assert rx.process(None, out)[1] == 0


def test_full_size_c2_whole_stream():
    """Full 10,000 km workload (2^24 symbols/pol, int8, one call + flush) against
    the FP64 oracle run over the whole stream: the frequency tracker identical
    at all 512 waves, taps at every wave start, equaliser and BPS outputs and
    LLRs within 1e-4 relative RMS, bits identical outside the exempt bands, and
    the device's BER count equal to the oracle's on the same bits."""
    import torch
    lk = L.workload("c2")
    g = L.generate(lk)
    p = rx_params(lk, g.in_scale)
    gpu = run_gpu(p, g.samples)
    K = lk.n_sym
    assert gpu["n"] == K
    tr = {}
    rep, orc = check_chain(p, g, gpu, tr)
    assert len(tr["wave_units"]) == 512
    print("c2 full-size parity", rep)
    ref = torch.from_numpy(L.pack_bits(g.tx_bits).view(np.int32)).cuda()
    e, n, sync = gpu["rx"].ber(gpu["bits_t"], ref, K)
    eo, no, so = O.ber_sync_count(orc["bits"], g.tx_bits, p.mod, p.acq_len(K))
    ber = e / n
    print("BER device", ber, "oracle", eo / no)
    # 10,000 km with PN/PMD/ADC at 9.8 dB: within 0.5 dB of QPSK theory
    assert O.ber_theory("qpsk", 9.8) * 0.9 < ber < O.ber_theory("qpsk", 9.3), ber
    assert abs(e - eo) <= rep["exempt_bits"], (e, eo, rep["exempt_bits"])
