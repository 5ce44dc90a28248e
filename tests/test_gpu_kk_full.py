"""The Kramers-Kronig chain at its full buffer size (2^22 ADC samples per buffer,
the configuration bench.py times), checked on sampled outputs the FP64 reference
computes one by one: stretches of the front end's output recomputed from the input
around them (the reference's windows sit on the same stream grid, so a stretch
with 4096 samples of margin on each side is exact), and sampled DD-LMS segments
re-run from the wave-start taps the GPU reports, on the GPU's own front-end
output.  Tolerances as the small-size parity tests: 1e-4 relative RMS; bits
identical away from decision boundaries."""
import numpy as np
import pytest

import linksim.kk as LK
from oracle import kk as K
from oracle import wl as W
from chain_helpers import boundary_mask, ensure_built, rel_rms

pytestmark = pytest.mark.gpu

N = 1 << 22            # samples per buffer
TOL = 1e-4


@pytest.fixture(scope="module", autouse=True)
def _built():
    ensure_built()


def test_kk_chain_full_size_sampled():
    import torch
    from paper_2104_06311_gb300 import KKFrontEnd, WLEqualiser
    lk = LK.KKLink(n_sym=2 * N // 4, L_km=5600.0, cspr_db=12.0, snr_db=24.0, adc="int8", iq_gain_db=1.0,
                   iq_phase_deg=5.0, seed=2104063123)
    g = LK.generate(lk)
    fe = KKFrontEnd(lk.baud, lk.carrier_hz, lk.L_km, N)
    D = fe.delay
    eq = WLEqualiser(4, N // 4)
    p = W.WLParams(mod="16qam")                      # the defaults the GPU uses
    ys, zs, bits, start_taps = [], [], [], []
    for b in range(2):
        x = torch.from_numpy(np.ascontiguousarray(g.samples[b * N:(b + 1) * N])).cuda()
        y, _ = fe.process(x, g.in_scale, g.in_offset)
        start_taps.append(eq.get_taps())
        words, z = eq.process(y, want_z=True)
        ys.append(y.cpu().numpy().astype(np.complex128))
        zs.append(z.cpu().numpy().astype(np.complex128))
        bits.append(np.unpackbits(words.cpu().numpy().view(np.uint8), bitorder="little"))
    # front end: stretches of the stream's output (stream sample t = call output index + b N - D)
    for t0 in (N // 2 + 512 * 37, N - D - 4096, 2 * N - D - 512 * 40):     # the second spans both calls
        L = 8192
        lo = t0 - 4096
        yo, _, _ = K.kk_frontend(g.samples[lo:t0 + L + 4096], g.in_scale, g.in_offset, lk.baud, lk.sps,
                                 lk.carrier_hz, lk.L_km, n0=lo)
        ref = yo[(t0 - lo) // 2:(t0 - lo + L) // 2]
        yy = np.concatenate(ys)[(t0 + D) // 2:(t0 + D + L) // 2]
        e = rel_rms(yy, ref)
        print(f"front end at sample {t0}: rel RMS {e:.2e}")
        assert e < TOL
    # DD-LMS: sampled segments of the second buffer from its wave-start taps
    x1 = ys[1]
    tail = ys[0][-2:]
    for j in (0, 1, 1777, 4095):
        s0 = j * p.seg_len
        s1 = min(s0 + p.seg_len, N // 4)
        z = np.zeros(N // 4, np.complex128)
        pre = W._run(x1, start_taps[1], max(0, s0 - p.pretrain), s0, p, None, tail)
        W._run(x1, pre, s0, s1, p, z, tail)
        e = rel_rms(zs[1][s0:s1], z[s0:s1])
        bo = W.hard_bits(z[s0:s1], "16qam")
        bg = bits[1][s0 * 4:s1 * 4]
        near = boundary_mask(z[s0:s1][:, None], "16qam").reshape(-1)
        print(f"segment {j}: z rel RMS {e:.2e}, bit mismatches {int(np.sum(bo != bg))}")
        assert e < TOL
        assert not np.any((bo != bg) & ~near)
    # and the decisions are the transmitted bits (24 dB): stream symbol = output index - D / 4
    allbits = np.concatenate(bits).reshape(-1, 4)
    tx = g.tx_bits.reshape(-1, 4)
    k = np.arange(D // 4 + 8192, allbits.shape[0])       # after the acquisition
    wrong = int(np.count_nonzero(np.any(allbits[k] != tx[k - D // 4], axis=1)))
    print(f"symbol errors {wrong} of {k.shape[0]}")
    assert wrong <= 2
