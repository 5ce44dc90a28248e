"""Failure detection without a GPU fault: one equaliser CTA is told (by a host
parameter) to leave out its arrival at the wave barrier, so the other CTAs'
bounded waits run out after a short limit.  The kernel returns, the handle
reports RX_ETIMEOUT, the CUDA context stays usable, and a fresh handle runs the
same stream at full parity.  No trap, no bad address, no unbounded wait: every
spin in the equaliser gives up after RX_P_WAIT_LIMIT_US of device time."""
import time

import numpy as np
import pytest

import linksim as L
from chain_helpers import ensure_built, make_receiver, rx_params, run_gpu
from test_gpu_chain import check_chain

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    ensure_built()


def test_wave_barrier_timeout_is_reported_and_the_next_handle_recovers():
    import torch
    from paper_2104_06311_gb300.rx import RX_ETIMEOUT, RxError
    lk = L.Link(n_sym=40_000, L_km=500.0, snr_db=13.0, seed=6061)
    g = L.generate(lk)
    p = rx_params(lk, g.in_scale)
    rx = make_receiver(p, WAIT_LIMIT_US=20_000, TEST_NO_ARRIVE=3)
    assert rx.get_param("WAIT_LIMIT_US") == 20_000 and rx.get_param("TEST_NO_ARRIVE") == 3
    x = torch.from_numpy(np.ascontiguousarray(g.samples)).cuda()
    t0 = time.perf_counter()
    status = None
    try:
        rx.run_stream(x)
        rx.sync()
    except RxError as e:
        status = e.status
        msg = str(e)
    dt = time.perf_counter() - t0
    assert status == RX_ETIMEOUT, status
    assert "wait" in msg
    assert dt < 30.0, dt                  # bounded: the waits gave up, nothing hung
    # the error is sticky on that handle
    with pytest.raises(RxError):
        rx.sync()
    rx.close()
    torch.cuda.synchronize()              # the context is intact
    # a fresh handle, default limits: the same stream at full parity
    gpu = run_gpu(p, g.samples)
    rep, _ = check_chain(p, g, gpu, {})
    print("after timeout", rep)
