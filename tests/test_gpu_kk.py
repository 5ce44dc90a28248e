"""GPU parity of the Kramers-Kronig front end (include/rx_kk.h) against the FP64
reference (oracle/kk.py): the rebuilt field at 4 samples/symbol and the filtered,
decimated field at 2 samples/symbol, element by element, for int8 and float32
input, ragged buffer lengths and two dispersion lengths."""
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


@pytest.mark.parametrize("adc,n_sym,L_km,cspr", [("int8", 1 << 16, 1000.0, 12.0), ("f32", 30_001, 3000.0, 9.0),
                                                  ("int8", 5000, 0.0, 14.0)])
def test_kk_front_end_matches_oracle(adc, n_sym, L_km, cspr):
    import torch
    from paper_2104_06311_gb300 import KKFrontEnd
    lk = LK.KKLink(n_sym=n_sym, adc=adc, L_km=L_km, cspr_db=cspr, snr_db=24.0, seed=2104063117 + n_sym)
    g = LK.generate(lk)
    n = g.samples.shape[0]
    fe = KKFrontEnd(lk.baud, lk.carrier_hz, lk.L_km, n)
    x = torch.from_numpy(np.ascontiguousarray(g.samples)).cuda()
    y, f = fe.process(x, g.in_scale, g.in_offset, field=True)
    torch.cuda.synchronize()
    yo, Eo, V = K.kk_frontend(g.samples, g.in_scale, g.in_offset, lk.baud, lk.sps, lk.carrier_hz, lk.L_km)
    assert fe.overlap == V
    ef = rel_rms(f.cpu().numpy().astype(np.complex128), Eo)
    ey = rel_rms(y.cpu().numpy().astype(np.complex128), yo)
    print(f"KK {adc} n={n} L={L_km}: field rel RMS {ef:.2e}, output rel RMS {ey:.2e}")
    assert ef < TOL and ey < TOL
    # symbol decisions at the even samples agree with the oracle's away from boundaries
    from oracle.chain import decide
    zo = yo[0::2]
    c = np.vdot(g.tx_symbols, zo) / np.vdot(g.tx_symbols, g.tx_symbols)
    zd = y.cpu().numpy().astype(np.complex128)[0::2] / c
    zo = zo / c
    far = (np.abs(np.abs(zo.real) * np.sqrt(10) - 2) > 1e-3) & (np.abs(zo.real) > 1e-3) & \
          (np.abs(np.abs(zo.imag) * np.sqrt(10) - 2) > 1e-3) & (np.abs(zo.imag) > 1e-3)
    assert np.array_equal(decide(zd, "16qam")[far], decide(zo, "16qam")[far])


def test_kk_stream_position_carries_across_calls():
    # consecutive buffers of one stream: the shift to DC continues from the samples
    # of the earlier calls; rx_kk_set_position(0) starts again at 0
    import torch
    from paper_2104_06311_gb300 import KKFrontEnd
    lk = LK.KKLink(n_sym=3 * 8192 + 100, adc="int8", L_km=2000.0, snr_db=24.0, seed=2104063121)
    g = LK.generate(lk)
    n = g.samples.shape[0]
    cuts = [0, 4 * 9001, 4 * 17003, n]
    fe = KKFrontEnd(lk.baud, lk.carrier_hz, lk.L_km, n)
    for rep in range(2):
        for a, b in zip(cuts[:-1], cuts[1:]):
            x = torch.from_numpy(np.ascontiguousarray(g.samples[a:b])).cuda()
            y, _ = fe.process(x, g.in_scale, g.in_offset)
            yo, _, _ = K.kk_frontend(g.samples[a:b], g.in_scale, g.in_offset, lk.baud, lk.sps, lk.carrier_hz,
                                     lk.L_km, n0=a)
            e = rel_rms(y.cpu().numpy().astype(np.complex128), yo)
            print(f"KK buffer at {a}: output rel RMS {e:.2e}")
            assert e < TOL
        fe.set_position(0)
    # a buffer replayed at its recorded position
    fe.set_position(cuts[2])
    x = torch.from_numpy(np.ascontiguousarray(g.samples[cuts[2]:])).cuda()
    y, _ = fe.process(x, g.in_scale, g.in_offset)
    yo, _, _ = K.kk_frontend(g.samples[cuts[2]:], g.in_scale, g.in_offset, lk.baud, lk.sps, lk.carrier_hz,
                             lk.L_km, n0=cuts[2])
    assert rel_rms(y.cpu().numpy().astype(np.complex128), yo) < TOL
