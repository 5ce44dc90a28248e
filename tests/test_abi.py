"""Host-side checks of the C ABI (no GPU compute): the library builds and loads,
exports every function the headers in include/ declare, resolves parameters on
the host and reports argument errors as status codes."""
import ctypes as ct
import os
import re
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2104_06311_gb300 import build as B
    if not os.path.exists(B.OUT):
        if not (shutil.which("nvcc") or os.path.exists("/usr/local/cuda/bin/nvcc")):
            pytest.skip("nvcc not available to build librx.so")
        B.build()
    from paper_2104_06311_gb300 import rx
    return rx.load()


def declared_functions():
    names = set()
    inc = os.path.join(ROOT, "include")
    for f in sorted(os.listdir(inc)):
        if f.endswith(".h"):
            text = re.sub(r"/\*.*?\*/", "", open(os.path.join(inc, f)).read(), flags=re.S)
            names |= set(re.findall(r"\b(rx_[a-z_0-9]+)\s*\(", text))
    return sorted(names)


def test_every_declared_function_is_exported(lib):
    from paper_2104_06311_gb300 import rx
    names = declared_functions()
    assert len(names) >= 25
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(rx.EXPORTS) == names   # the binding covers exactly the declared ABI


def _chan(**kw):
    from paper_2104_06311_gb300 import rx
    d = dict(baud=10e9, L_km=1000.0, D_ps_nm_km=17.0, in_scale=1.0, max_samples=1 << 17, mod_bits=2,
             ntaps=15, fft_n=0, overlap=0)
    d.update(kw)
    return rx.rx_chan_cfg(**d)


@pytest.mark.parametrize("bad,status,text", [
    (dict(mod_bits=3), "RX_EUNSUPPORTED", b"channel 1: mod_bits"),
    (dict(ntaps=16), "RX_EUNSUPPORTED", b"channel 1: ntaps"),
    (dict(max_samples=1001), "RX_EINVAL", b"channel 1: max_samples"),
    (dict(fft_n=3000), "RX_EUNSUPPORTED", b"channel 1: FFT size"),
    (dict(baud=0.0), "RX_EINVAL", b"channel 1: baud"),
    (dict(L_km=20000.0, baud=32e9), "RX_EUNSUPPORTED", b"channel 1: dispersion too large"),
])
def test_batch_create_reports_the_bad_channel(lib, bad, status, text):
    from paper_2104_06311_gb300 import rx
    cfgs = (rx.rx_chan_cfg * 3)(_chan(), _chan(**bad), _chan())
    h = ct.c_void_p()
    st = lib.rx_batch_create(ct.byref(h), 3, cfgs)
    assert st == getattr(rx, status)
    assert text in lib.rx_batch_last_error(h)
    lib.rx_batch_destroy(h)


def test_batch_create_argument_errors(lib):
    from paper_2104_06311_gb300 import rx
    h = ct.c_void_p()
    cfgs = (rx.rx_chan_cfg * 1)(_chan())
    assert lib.rx_batch_create(ct.byref(h), 0, cfgs) == rx.RX_EINVAL and not h.value
    assert lib.rx_batch_create(ct.byref(h), 1, None) == rx.RX_EINVAL and not h.value
    assert lib.rx_batch_process(None, None, None) == rx.RX_EINVAL


def test_status_strings(lib):
    for s in range(7):
        assert lib.rx_status_str(s)
    assert lib.rx_status_str(99) == b"unknown status"


def _create(lib, *args):
    h = ct.c_void_p()
    st = lib.rx_create(ct.byref(h), *args)
    return st, h


def test_create_rejects_bad_arguments(lib):
    from paper_2104_06311_gb300 import rx
    assert _create(lib, -1.0, 2, 100.0, 17.0, 15, 32)[0] == rx.RX_EINVAL
    assert _create(lib, 10e9, 4, 100.0, 17.0, 15, 32)[0] == rx.RX_EUNSUPPORTED
    assert _create(lib, 10e9, 2, 100.0, 17.0, 16, 32)[0] == rx.RX_EUNSUPPORTED
    assert _create(lib, 10e9, 2, 100.0, 17.0, 15, 64)[0] == rx.RX_EUNSUPPORTED
    st, h = _create(lib, 10e9, 2, -5.0, 17.0, 15, 32)
    assert st == rx.RX_EINVAL and not h.value


@pytest.mark.parametrize("L_km,baud,N,V", [(1000, 10e9, 1024, 64), (10000, 10e9, 4096, 544),
                                           (2000, 32e9, 8192, 1120), (0, 10e9, 1024, 32),
                                           (6000, 32e9, 16384, 3360), (10000, 32e9, 16384, 5600)])
def test_parameter_resolution_on_host(lib, L_km, baud, N, V):
    from paper_2104_06311_gb300 import rx
    st, h = _create(lib, baud, 2, float(L_km), 17.0, 15, 32)
    assert st == rx.RX_OK
    v = ct.c_double()
    assert lib.rx_get_param(h, rx.PARAMS["FFT_N"], ct.byref(v)) == rx.RX_OK and v.value == N
    assert lib.rx_get_param(h, rx.PARAMS["OVERLAP"], ct.byref(v)) == rx.RX_OK and v.value == V
    lib.rx_destroy(h)


def test_dispersion_beyond_single_cta_fft_is_reported(lib):
    from paper_2104_06311_gb300 import rx
    st, h = _create(lib, 32e9, 2, 20000.0, 17.0, 15, 32)   # N_CD 11161 -> V 11168 > 16384 / 2
    assert st == rx.RX_OK
    v = ct.c_double()
    assert lib.rx_get_param(h, rx.PARAMS["FFT_N"], ct.byref(v)) == rx.RX_EUNSUPPORTED
    assert b"dispersion too large" in lib.rx_last_error(h)
    assert lib.rx_set_param(h, rx.PARAMS["FFT_N"], 32768.0) == rx.RX_OK
    assert lib.rx_get_param(h, rx.PARAMS["FFT_N"], ct.byref(v)) == rx.RX_EUNSUPPORTED
    assert b"FFT size" in lib.rx_last_error(h)
    lib.rx_destroy(h)


def test_set_param_validation(lib):
    from paper_2104_06311_gb300 import rx
    st, h = _create(lib, 10e9, 2, 1000.0, 17.0, 15, 32)
    P = rx.PARAMS
    assert lib.rx_set_param(h, 999, 1.0) == rx.RX_EINVAL
    assert lib.rx_set_param(h, P["MOD"], 3.0) == rx.RX_EUNSUPPORTED
    assert lib.rx_set_param(h, P["MOD"], 4.0) == rx.RX_OK
    assert lib.rx_set_param(h, P["UPDATE_BLOCK"], 33.0) == rx.RX_EINVAL
    assert lib.rx_set_param(h, P["SEG_LEN"], 1000.5) == rx.RX_EINVAL
    assert lib.rx_set_param(h, P["ROLLOFF"], 0.0) == rx.RX_EINVAL
    assert lib.rx_set_param(h, P["MU_DD"], float("nan")) == rx.RX_EINVAL
    lib.rx_destroy(h)


def test_process_argument_errors_need_no_gpu(lib):
    from paper_2104_06311_gb300 import rx
    st, h = _create(lib, 10e9, 2, 1000.0, 17.0, 15, 32)
    i = rx.rx_in()
    o = rx.rx_out()
    o.bits = 16
    assert lib.rx_process(h, None, ct.byref(o)) == rx.RX_EINVAL
    i.data, i.n, i.dtype = 16, 3, rx.RX_F32x4          # odd sample count
    assert lib.rx_process(h, ct.byref(i), ct.byref(o)) == rx.RX_EINVAL
    i.n, i.dtype = 4, 7                                 # unknown dtype
    assert lib.rx_process(h, ct.byref(i), ct.byref(o)) == rx.RX_EINVAL
    i.dtype, i.data = rx.RX_F32x4, 8                    # misaligned float input
    assert lib.rx_process(h, ct.byref(i), ct.byref(o)) == rx.RX_EINVAL
    i.data, o.bits = 16, None                           # missing bit output
    assert lib.rx_process(h, ct.byref(i), ct.byref(o)) == rx.RX_EINVAL
    assert b"null bit output" in lib.rx_last_error(h)
    lib.rx_destroy(h)
