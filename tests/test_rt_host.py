"""Host logic of the real-time pipeline (include/rx_rt.h) that needs no GPU: the
Q-factor of a bit-error ratio against scipy's erfcinv and against the Gray-QPSK
closed form (Q^2 = Es/N0), and the configuration checks that run before any
device call."""
import ctypes as ct
import math

import numpy as np
import pytest
from scipy.special import erfc, erfcinv


@pytest.fixture(scope="module")
def rx():
    from chain_helpers import ensure_built
    ensure_built()
    from paper_2104_06311_gb300 import rx
    return rx


def test_q_db_matches_erfcinv(rx):
    for ber in (1e-12, 1e-6, 3.8e-3, 1e-2, 0.1, 0.3, 0.49):
        want = 20 * math.log10(math.sqrt(2) * erfcinv(2 * ber))
        assert abs(rx.q_db(ber) - want) < 1e-9, ber
    # Gray QPSK: BER = Q(sqrt(Es/N0)), so Q_dB equals Es/N0 in dB
    for snr_db in (6.0, 9.8, 13.0):
        ber = 0.5 * erfc(math.sqrt(10 ** (snr_db / 10) / 2))
        assert abs(rx.q_db(ber) - snr_db) < 1e-9
    assert rx.q_db(0.0) == math.inf
    assert math.isnan(rx.q_db(0.5)) and math.isnan(rx.q_db(-1e-3))


def _cfg(rx, ref, **over):
    c = dict(baud=1e9, sps=4, mod_bits=4, carrier_hz=0.516e9, L_km=1000.0, D_ps_nm_km=17.0, rolloff=0.01,
             in_dtype=1, in_scale=1.0, in_offset=0.0, buffer_samples=1 << 16, depth=4,
             ref_bits=ref.ctypes.data, ref_nbits=ref.shape[0], bin_symbols=1 << 16, edge_symbols=2048, max_bins=16)
    c.update(over)
    return rx.rx_rt_cfg(**c)


@pytest.mark.parametrize("bad", [dict(sps=2), dict(mod_bits=3), dict(buffer_samples=1000), dict(depth=1),
                                 dict(depth=17), dict(edge_symbols=10), dict(in_dtype=7), dict(ref_nbits=33),
                                 dict(bin_symbols=100), dict(edge_symbols=1 << 13), dict(baud=0.0)])
def test_bad_configurations_are_refused_before_any_device_call(rx, bad):
    ref = np.zeros(64, np.uint8)
    h = ct.c_void_p()
    st = rx.load().rx_rt_create(ct.byref(h), ct.byref(_cfg(rx, ref, **bad)))
    assert st == rx.RX_EINVAL and not h.value
