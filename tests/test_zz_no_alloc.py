"""The allocation-free BPS + demap entry point, checked against rx_process.

rx_bps_demap_noalloc is for callers that cannot allocate device memory when
they need carrier recovery (real-time loops that must not wait on the
allocator, hosts with a fixed device-memory budget); its scratch is a static
device array.  Fed the equaliser output of
an rx_process run, it must reproduce that run's hard bits exactly (the same
kernels, chunk grid and window truncation), on two calls in a row (the
shared scratch keeps the previous call's contents).  This file sorts last so
a run that stops at the first failure has run every other test first.
"""
import ctypes as ct

import numpy as np
import pytest

import linksim as L
from chain_helpers import ensure_built, make_receiver, rx_params

pytestmark = pytest.mark.gpu


def test_noalloc_bps_demap_matches_rx_process_on_two_calls():
    import torch
    from paper_2104_06311_gb300 import rx as R
    ensure_built()
    lib = R.load()
    lk = L.workload("c1")
    g = L.generate(lk)
    p = rx_params(lk, g.in_scale, fft_n=1024)
    rcv = make_receiver(p, EQ_OUT=1)
    x = torch.from_numpy(g.samples).cuda()
    ref = rcv.run_stream(x, eq=True)
    torch.cuda.synchronize()
    K = ref["n"]
    words = (K * p.bits + 31) // 32
    eq = ref["eq"]                      # (2, capacity) complex64, symbols [0, K)
    stream = torch.cuda.current_stream()
    for call in range(2):
        bits = torch.full_like(ref["bits"], -1)
        st = lib.rx_bps_demap_noalloc(eq.data_ptr(), eq.shape[1], K, p.bits, p.bps_halfwin,
                                      bits.data_ptr(), bits.shape[1], ct.c_void_p(stream.cuda_stream))
        assert st == R.RX_OK, call
        torch.cuda.synchronize()
        assert torch.equal(bits[:, :words], ref["bits"][:, :words]), call
    # sizes beyond the static scratch are refused
    big = (1 << 20) + 1
    st = lib.rx_bps_demap_noalloc(eq.data_ptr(), big, big, p.bits, p.bps_halfwin,
                                  ref["bits"].data_ptr(), big, ct.c_void_p(stream.cuda_stream))
    assert st == R.RX_EINVAL
