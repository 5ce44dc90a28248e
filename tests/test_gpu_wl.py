"""GPU parity of the widely-linear DD-LMS equaliser (include/rx_wl.h) against the
FP64 reference (oracle/wl.py), through the C ABI: outputs z within 1e-4 relative
RMS, the taps that start each next buffer within 1e-4, Gray bits identical except
where the oracle's soft value lies within 1e-5 of a decision boundary; on the
KK front end's output for a 1 GBd 16QAM link with transmitter IQ imbalance, on
QPSK, for the strictly linear variant, over several buffers with ragged tails,
an acquisition longer than the first buffer, and the argument checks."""
import numpy as np
import pytest

import linksim.kk as LK
from oracle import kk as K
from oracle import wl as W
from chain_helpers import boundary_mask, ensure_built, rel_rms

pytestmark = pytest.mark.gpu

TOL = 1e-4


@pytest.fixture(scope="module", autouse=True)
def _built():
    ensure_built()


def _unpack(words, nbits):
    b = np.unpackbits(np.ascontiguousarray(words).view(np.uint8), bitorder="little")
    return b[:nbits]


def _kk_field(mod, n_sym, iq=(1.0, 5.0), snr=25.0, L_km=1000.0, seed=2104063118):
    lk = LK.KKLink(mod=mod, n_sym=n_sym, L_km=L_km, snr_db=snr, iq_gain_db=iq[0], iq_phase_deg=iq[1], seed=seed)
    g = LK.generate(lk)
    y, _, _ = K.kk_frontend(g.samples, g.in_scale, g.in_offset, lk.baud, lk.sps, lk.carrier_hz, lk.L_km)
    return lk, g, y


def _run_both(y, cuts, p, mb):
    """Same buffers through the GPU and the oracle; returns per-buffer results."""
    import torch
    from paper_2104_06311_gb300 import WLEqualiser
    eq = WLEqualiser(mb, max(np.diff(cuts)) // 2, mu=p.mu, seg_len=p.seg_len, pretrain=p.pretrain, acq=p.acq,
                     linear=int(p.linear))
    st = None
    out = []
    for a, b in zip(cuts[:-1], cuts[1:]):
        xb = y[a:b]
        words, z = eq.process(torch.from_numpy(xb.astype(np.complex64)).cuda(), want_z=True)
        taps = eq.get_taps()
        zo, bo, st = W.wl_equalise(xb.astype(np.complex64).astype(np.complex128), p, st)
        out.append(dict(z=z.cpu().numpy().astype(np.complex128), bits=_unpack(words.cpu().numpy(), bo.shape[0]),
                        taps=taps, zo=zo, bo=bo, taps_o=st.taps.copy()))
    eq.close()
    return out


def _check(out, mod):
    for r in out:
        ez = rel_rms(r["z"], r["zo"])
        et = rel_rms(r["taps"], r["taps_o"])
        near = boundary_mask(r["zo"][:, None], mod).reshape(-1)
        diff = r["bits"] != r["bo"]
        print(f"z rel RMS {ez:.2e}, taps {et:.2e}, bit mismatches {int(diff.sum())} ({int((diff & ~near).sum())} away "
              f"from boundaries)")
        assert ez < TOL and et < TOL
        assert not np.any(diff & ~near)


@pytest.mark.parametrize("linear", [False, True])
def test_wl_matches_oracle_on_kk_output(linear):
    lk, g, y = _kk_field("16qam", 3 * 8192 + 40)
    n = y.shape[0]
    cuts = [0, 2 * 9000, 2 * 17000, n]                   # three buffers, ragged lengths
    p = W.WLParams(mod="16qam", mu=2e-3, seg_len=512, pretrain=64, acq=2048, linear=linear)
    out = _run_both(y, cuts, p, 4)
    _check(out, "16qam")
    if not linear:
        # with the image removed the decisions are error-free away from the buffer edges
        bits = np.concatenate([r["bits"] for r in out])
        tx = g.tx_bits
        K1 = bits.shape[0] // 4
        keep = np.ones(K1, bool)
        for c in cuts:
            keep[max(0, c // 2 - 400):c // 2 + 400] = False
        assert np.array_equal(bits.reshape(K1, 4)[keep], tx.reshape(-1, 4)[:K1][keep])


def test_wl_beats_linear_under_iq_imbalance():
    import torch
    from paper_2104_06311_gb300 import WLEqualiser
    lk, g, y = _kk_field("16qam", 1 << 15, iq=(1.5, 8.0), snr=30.0)
    x = torch.from_numpy(y.astype(np.complex64)).cuda()
    evm = {}
    for lin in (0, 1):
        eq = WLEqualiser(4, y.shape[0] // 2, mu=2e-3, acq=4096, linear=lin)
        _, z = eq.process(x, want_z=True)
        zz = z.cpu().numpy()[8192:-600]
        t = g.tx_symbols[8192:8192 + zz.shape[0]]
        evm[lin] = float(np.sqrt(np.mean(np.abs(zz - t) ** 2)))
        eq.close()
    mu, nu = LK.iq_imbalance(lk)
    print("EVM widely linear", evm[0], "linear", evm[1], "image/signal", abs(nu) / abs(mu))
    assert evm[1] > 0.8 * abs(nu) / abs(mu)
    assert evm[0] < 0.5 * evm[1]


def test_wl_qpsk_defaults_and_short_first_buffer():
    # the first buffer is shorter than the acquisition span: all of it is acquisition
    lk, g, y = _kk_field("qpsk", 20000, iq=(0.5, 3.0), snr=18.0, L_km=5000.0, seed=2104063119)
    p = W.WLParams(mod="qpsk", acq=8192)
    cuts = [0, 2 * 5000, 2 * 20000]
    out = _run_both(y, cuts, p, 2)
    _check(out, "qpsk")


def test_wl_arguments_and_reset():
    import torch
    from paper_2104_06311_gb300 import WLEqualiser
    from paper_2104_06311_gb300.rx import RxError
    lk, g, y = _kk_field("16qam", 4000)
    x = torch.from_numpy(y.astype(np.complex64)).cuda()
    eq = WLEqualiser(4, 4000, acq=1024, seg_len=256)
    w0, z0 = eq.process(x, want_z=True)
    w0, z0 = w0.clone(), z0.clone()
    with pytest.raises(RxError):
        eq.set_param("MU", 1e-2)                  # fixed after the first call
    with pytest.raises(RxError):
        eq.set_param("SEG_LEN", 100)              # not a multiple of 16 (checked before state)
    with pytest.raises(RxError):
        eq.process(torch.zeros(2 * 4000 + 2, dtype=torch.complex64, device="cuda"))   # over max_symbols
    with pytest.raises(RxError):
        eq.process(x[1:-1])                       # misaligned (8-byte offset)
    eq.process(x[:0])                             # no-op
    eq.reset()
    w1, z1 = eq.process(x, want_z=True)
    assert torch.equal(w0, w1) and torch.equal(z0, z1)
    # start taps round trip and the strictly linear variant's g = 0
    t = np.zeros((2, 4), np.complex128)
    t[0, 1] = 0.9 - 0.1j
    t[1, 1] = 0.05 + 0.02j
    eq.reset()
    eq.set_taps(t)
    assert np.abs(eq.get_taps() - t).max() < 1e-7
    eq.close()
    with pytest.raises(RxError):
        WLEqualiser(4, 100, ntaps=5)
