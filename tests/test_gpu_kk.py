"""GPU parity of the Kramers-Kronig front end (include/rx_kk.h) against the FP64
reference (oracle/kk.py): the rebuilt field at 4 samples/symbol and the filtered,
decimated field at 2 samples/symbol, element by element, for int8 and float32
input and two dispersion lengths.  The front end streams: buffers are pieces of
one stream, the output lags the input by a fixed delay, and the outputs of all
calls plus the flush equal the whole stream filtered at once -- whatever the
buffer boundaries."""
import numpy as np
import pytest

import linksim.kk as LK
from oracle import kk as K
from chain_helpers import ensure_built, rel_rms

pytestmark = pytest.mark.gpu

TOL = 1e-4     # FP32 log / sqrt / sincos and 1024-point transforms vs FP64


@pytest.fixture(scope="module", autouse=True)
def _built():
    ensure_built()


def _stream(fe, samples, cuts, g, field=True):
    """Feed samples[cuts[i]:cuts[i+1]] in turn, then flush; outputs with the delay removed."""
    import torch
    ys, fs = [], []
    for a, b in zip(cuts[:-1], cuts[1:]):
        x = torch.from_numpy(np.ascontiguousarray(samples[a:b])).cuda()
        y, f = fe.process(x, g.in_scale, g.in_offset, field=field)
        ys.append(y.cpu().numpy())
        if field:
            fs.append(f.cpu().numpy())
    y, f = fe.flush(field=field)
    ys.append(y.cpu().numpy())
    if field:
        fs.append(f.cpu().numpy())
    D = fe.delay
    yy = np.concatenate(ys).astype(np.complex128)
    assert np.all(yy[:D // 2] == 0)                 # before the stream start
    ff = np.concatenate(fs).astype(np.complex128)[D:] if field else None
    return yy[D // 2:], ff


@pytest.mark.parametrize("adc,n_sym,L_km,cspr", [("int8", 1 << 16, 1000.0, 12.0), ("f32", 29_952, 3000.0, 9.0),
                                                  ("int8", 4992, 0.0, 14.0)])
def test_kk_front_end_matches_oracle(adc, n_sym, L_km, cspr):
    from paper_2104_06311_gb300 import KKFrontEnd
    lk = LK.KKLink(n_sym=n_sym, adc=adc, L_km=L_km, cspr_db=cspr, snr_db=24.0, seed=2104063117 + n_sym)
    g = LK.generate(lk)
    n = g.samples.shape[0]
    fe = KKFrontEnd(lk.baud, lk.carrier_hz, lk.L_km, n)
    yg, fg = _stream(fe, g.samples, [0, n], g)
    yo, Eo, V = K.kk_frontend(g.samples, g.in_scale, g.in_offset, lk.baud, lk.sps, lk.carrier_hz, lk.L_km)
    assert fe.overlap == V
    ef = rel_rms(fg, Eo)
    ey = rel_rms(yg, yo)
    print(f"KK {adc} n={n} L={L_km}: field rel RMS {ef:.2e}, output rel RMS {ey:.2e}")
    assert ef < TOL and ey < TOL
    # symbol decisions at the even samples agree with the oracle's away from boundaries
    from oracle.chain import decide
    zo = yo[0::2]
    zd = yg[0::2]
    far = (np.abs(np.abs(zo.real) * np.sqrt(10) - 2) > 1e-3) & (np.abs(zo.real) > 1e-3) & \
          (np.abs(np.abs(zo.imag) * np.sqrt(10) - 2) > 1e-3) & (np.abs(zo.imag) > 1e-3)
    assert np.array_equal(decide(zd, "16qam")[far], decide(zo, "16qam")[far])


def test_kk_streaming_equals_the_whole_stream():
    # unequal buffers, one shorter than the look-ahead: the concatenated output is the
    # whole stream's; after the flush a new stream starts at 0; a stream started at
    # sample P runs its carrier shift from P
    from paper_2104_06311_gb300 import KKFrontEnd
    lk = LK.KKLink(n_sym=3 * 8192 + 128, adc="int8", L_km=2000.0, snr_db=24.0, seed=2104063121)
    g = LK.generate(lk)
    n = g.samples.shape[0]
    yo, Eo, _ = K.kk_frontend(g.samples, g.in_scale, g.in_offset, lk.baud, lk.sps, lk.carrier_hz, lk.L_km)
    fe = KKFrontEnd(lk.baud, lk.carrier_hz, lk.L_km, n)
    for cuts in ([0, 512 * 70, 512 * 71, 512 * 133, n], [0, 512 * 96, n]):
        yg, fg = _stream(fe, g.samples, cuts, g)
        e = (rel_rms(yg, yo), rel_rms(fg, Eo))
        print(f"KK cuts {cuts}: output / field rel RMS {e[0]:.2e} / {e[1]:.2e}")
        assert max(e) < TOL
    P = 512 * 1000
    fe.set_position(P)
    yg, _ = _stream(fe, g.samples, [0, n], g, field=False)
    yp, _, _ = K.kk_frontend(g.samples, g.in_scale, g.in_offset, lk.baud, lk.sps, lk.carrier_hz, lk.L_km, n0=P)
    assert rel_rms(yg, yp) < TOL


def test_kk_arguments():
    import torch
    from paper_2104_06311_gb300 import KKFrontEnd
    from paper_2104_06311_gb300.rx import RxError
    fe = KKFrontEnd(1e9, 0.516e9, 1000.0, 4096)
    with pytest.raises(RxError):
        fe.process(torch.zeros(1000, dtype=torch.int8, device="cuda"))      # not a multiple of 512
    with pytest.raises(RxError):
        fe.process(torch.zeros(8192, dtype=torch.int8, device="cuda"))      # over max_samples
    assert fe.delay == 1536
