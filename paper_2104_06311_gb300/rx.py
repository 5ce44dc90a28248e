"""Thin ctypes binding of the receiver's C ABI (include/rx.h).

Argument marshalling only: every step of the chain runs in the CUDA kernels of
librx.so.  The functions carry the C names (rx_create, rx_process, rx_ber, ...);
``Receiver`` bundles them for callers that hold torch CUDA tensors.  Loading
fails loudly when the library has not been built: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as ct
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "librx.so")

RX_OK, RX_EINVAL, RX_ENOMEM, RX_ECUDA, RX_ESTATE, RX_ETIMEOUT, RX_EUNSUPPORTED = range(7)
RX_I8x4, RX_F32x4 = 1, 2

PARAMS = {
    "MOD": 1, "FFT_N": 2, "OVERLAP": 3, "ROLLOFF": 4, "LAMBDA_NM": 5, "MU_CMA": 6, "MU_DD": 7,
    "N_CMA": 8, "UPDATE_BLOCK": 9, "SEG_LEN": 10, "SEG_PRETRAIN": 11, "BPS_HALFWIN": 12,
    "BLOCK_SAMPLES": 13, "IN_SCALE": 14, "ACQ_MIN": 15, "FO_SMOOTH": 16, "FO_TRACK": 17,
    "LLR_OUT": 18, "SYM_OUT": 19, "EQ_OUT": 20, "CDC_OUT": 21, "PROFILE": 22, "PIPELINE": 23,
    "PRECISION": 24, "INNER_TRACE": 25, "WAIT_LIMIT_US": 26, "TEST_NO_ARRIVE": 27, "DFT_TC": 28, "EQ_WARPS": 29, "EQ_ALT": 30, "CDC_4STEP": 31,
}
STAGES = ["cdc", "eq", "bps", "move", "ber"]

EXPORTS = ["rx_create", "rx_set_param", "rx_get_param", "rx_set_cuda_stream", "rx_reserve",
           "rx_process", "rx_ber", "rx_trace", "rx_trace_inner", "rx_get_state", "rx_set_state", "rx_reset",
           "rx_sync", "rx_destroy", "rx_status_str", "rx_last_error", "rx_profile",
           "rx_bps_demap_noalloc", "rx_measure_alu_peak",
           "rx_batch_create", "rx_batch_set_param", "rx_batch_get_param", "rx_batch_set_cuda_stream",
           "rx_batch_process", "rx_batch_ber", "rx_batch_trace", "rx_batch_sync", "rx_batch_destroy",
           "rx_batch_last_error", "rx_batch_profile",
           "rx_cnn_create", "rx_cnn_param_count", "rx_cnn_set_params", "rx_cnn_get_params",
           "rx_cnn_set_cuda_stream", "rx_cnn_apply", "rx_cnn_grads", "rx_cnn_train_step", "rx_cnn_destroy",
           "rx_cnn_last_error", "rx_cnn_set_profile", "rx_cnn_profile", "rx_cnn_set_option",
           "rx_kk_create", "rx_kk_set_cuda_stream", "rx_kk_get_overlap", "rx_kk_process", "rx_kk_profile",
           "rx_kk_set_position", "rx_kk_flush", "rx_kk_get_delay", "rx_kk_destroy", "rx_kk_last_error",
           "rx_wl_create", "rx_wl_set_param", "rx_wl_get_param", "rx_wl_set_cuda_stream", "rx_wl_set_taps",
           "rx_wl_get_taps", "rx_wl_process", "rx_wl_reset", "rx_wl_profile", "rx_wl_destroy", "rx_wl_last_error",
           "rx_rt_create", "rx_rt_set_wl_param", "rx_rt_next_input", "rx_rt_submit", "rx_rt_submit_from", "rx_rt_flush", "rx_rt_output", "rx_rt_drain",
           "rx_rt_bins", "rx_rt_profile", "rx_rt_destroy", "rx_rt_last_error", "rx_q_db"]
WL_PARAMS = {"MU": 1, "SEG_LEN": 2, "PRETRAIN": 3, "ACQ": 4, "LINEAR": 5}
CNN_KINDS = ["fwd_hidden", "fwd_edge", "dx", "dw", "update"]
BATCH_PARAMS = {"GRAPH": 100, "EQ_CTAS": 101, "EQ_TEAM": 102, "CDC_NS_PER_SAMPLE": 103, "PROFILE": 104,
                "CDC_ENGINE": 105}


class rx_in(ct.Structure):
    _fields_ = [("data", ct.c_void_p), ("n", ct.c_int64), ("dtype", ct.c_int32), ("reserved", ct.c_int32)]


class rx_out(ct.Structure):
    _fields_ = [("bits", ct.c_void_p), ("bits_stride", ct.c_int64),
                ("llr", ct.c_void_p), ("llr_stride", ct.c_int64),
                ("sym", ct.c_void_p), ("sym_stride", ct.c_int64),
                ("eq", ct.c_void_p), ("eq_stride", ct.c_int64),
                ("cdc", ct.c_void_p), ("cdc_stride", ct.c_int64),
                ("capacity", ct.c_int64), ("n", ct.c_int64), ("first", ct.c_int64),
                ("cdc_first", ct.c_int64), ("cdc_n", ct.c_int64)]


class rx_rt_cfg(ct.Structure):
    _fields_ = [("baud", ct.c_double), ("sps", ct.c_int), ("mod_bits", ct.c_int), ("carrier_hz", ct.c_double),
                ("L_km", ct.c_double), ("D_ps_nm_km", ct.c_double), ("rolloff", ct.c_double),
                ("in_dtype", ct.c_int), ("in_scale", ct.c_float), ("in_offset", ct.c_float),
                ("buffer_samples", ct.c_int64), ("depth", ct.c_int), ("ref_bits", ct.c_void_p), ("ref_nbits", ct.c_int64), ("bin_symbols", ct.c_int64),
                ("edge_symbols", ct.c_int), ("max_bins", ct.c_int)]


class rx_chan_cfg(ct.Structure):
    _fields_ = [("baud", ct.c_double), ("L_km", ct.c_double), ("D_ps_nm_km", ct.c_double),
                ("in_scale", ct.c_double), ("max_samples", ct.c_int64), ("mod_bits", ct.c_int32),
                ("ntaps", ct.c_int32), ("fft_n", ct.c_int32), ("overlap", ct.c_int32),
                ("flags", ct.c_int32), ("bps_halfwin", ct.c_int32)]


class RxError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{msg} (status {status})")
        self.status = status


_lib = None


def load(path: str = LIB_PATH) -> ct.CDLL:
    """Load librx.so (raises if it is missing: build it with paper_2104_06311_gb300.build)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing; run `python -m paper_2104_06311_gb300.build`")
    lib = ct.CDLL(path)
    P = ct.c_void_p
    lib.rx_create.argtypes = [ct.POINTER(P), ct.c_double, ct.c_int, ct.c_double, ct.c_double, ct.c_int, ct.c_int]
    lib.rx_set_param.argtypes = [P, ct.c_int, ct.c_double]
    lib.rx_get_param.argtypes = [P, ct.c_int, ct.POINTER(ct.c_double)]
    lib.rx_set_cuda_stream.argtypes = [P, P]
    lib.rx_reserve.argtypes = [P, ct.c_int64]
    lib.rx_process.argtypes = [P, ct.POINTER(rx_in), ct.POINTER(rx_out)]
    lib.rx_ber.argtypes = [P, P, ct.c_int64, P, ct.c_int64, ct.c_int64, ct.POINTER(ct.c_uint64),
                           ct.POINTER(ct.c_uint64), ct.POINTER(ct.c_int32)]
    lib.rx_trace.argtypes = [P, ct.c_int64, ct.POINTER(ct.c_float), ct.POINTER(ct.c_double), ct.POINTER(ct.c_double)]
    lib.rx_trace_inner.argtypes = [P, ct.c_int64, ct.c_int64, P, ct.POINTER(ct.c_int64), ct.POINTER(ct.c_int32)]
    lib.rx_get_state.argtypes = [P, P, ct.POINTER(ct.c_size_t)]
    lib.rx_set_state.argtypes = [P, P, ct.c_size_t]
    lib.rx_profile.argtypes = [P, ct.POINTER(ct.c_double), ct.POINTER(ct.c_int64), ct.c_int]
    lib.rx_bps_demap_noalloc.argtypes = [P, ct.c_int64, ct.c_int64, ct.c_int, ct.c_int, P, ct.c_int64, P]
    lib.rx_measure_alu_peak.argtypes = [ct.c_int, ct.c_int, P, ct.POINTER(ct.c_double), ct.POINTER(ct.c_double)]
    lib.rx_reset.argtypes = [P]
    lib.rx_sync.argtypes = [P]
    lib.rx_destroy.argtypes = [P]
    lib.rx_destroy.restype = None
    lib.rx_status_str.argtypes = [ct.c_int]
    lib.rx_status_str.restype = ct.c_char_p
    lib.rx_last_error.argtypes = [P]
    lib.rx_last_error.restype = ct.c_char_p
    lib.rx_batch_create.argtypes = [ct.POINTER(P), ct.c_int, ct.POINTER(rx_chan_cfg)]
    lib.rx_batch_set_param.argtypes = [P, ct.c_int, ct.c_double]
    lib.rx_batch_get_param.argtypes = [P, ct.c_int, ct.c_int, ct.POINTER(ct.c_double)]
    lib.rx_batch_set_cuda_stream.argtypes = [P, P]
    lib.rx_batch_process.argtypes = [P, ct.POINTER(rx_in), ct.POINTER(rx_out)]
    lib.rx_batch_ber.argtypes = [P, ct.c_int, P, ct.c_int64, P, ct.c_int64, ct.c_int64, ct.POINTER(ct.c_uint64),
                                 ct.POINTER(ct.c_uint64), ct.POINTER(ct.c_int32)]
    lib.rx_batch_trace.argtypes = [P, ct.c_int, ct.c_int64, ct.POINTER(ct.c_float), ct.POINTER(ct.c_double),
                                   ct.POINTER(ct.c_double)]
    lib.rx_batch_profile.argtypes = [P, ct.POINTER(ct.c_double), ct.POINTER(ct.c_int64), ct.c_int]
    lib.rx_batch_sync.argtypes = [P]
    lib.rx_batch_destroy.argtypes = [P]
    lib.rx_batch_destroy.restype = None
    lib.rx_batch_last_error.argtypes = [P]
    lib.rx_batch_last_error.restype = ct.c_char_p
    lib.rx_cnn_create.argtypes = [ct.POINTER(P), ct.c_int, ct.c_int, ct.c_int, ct.c_int64]
    lib.rx_cnn_param_count.argtypes = [P]
    lib.rx_cnn_param_count.restype = ct.c_int64
    lib.rx_cnn_set_params.argtypes = [P, P]
    lib.rx_cnn_get_params.argtypes = [P, P]
    lib.rx_cnn_set_cuda_stream.argtypes = [P, P]
    lib.rx_cnn_apply.argtypes = [P, P, ct.c_int64, P, ct.c_int64, ct.c_int64]
    lib.rx_cnn_grads.argtypes = [P, P, ct.c_int64, P, ct.c_int64, ct.c_int64, P, ct.POINTER(ct.c_double)]
    lib.rx_cnn_train_step.argtypes = [P, P, ct.c_int64, P, ct.c_int64, ct.c_int64, ct.c_float, P]
    lib.rx_cnn_set_profile.argtypes = [P, ct.c_int]
    lib.rx_cnn_set_option.argtypes = [P, ct.c_int, ct.c_int]
    lib.rx_cnn_profile.argtypes = [P, ct.POINTER(ct.c_double), ct.POINTER(ct.c_int64), ct.c_int]
    lib.rx_kk_create.argtypes = [ct.POINTER(P), ct.c_double, ct.c_int, ct.c_double, ct.c_double, ct.c_double,
                                 ct.c_double, ct.c_int64]
    lib.rx_kk_set_cuda_stream.argtypes = [P, P]
    lib.rx_kk_get_overlap.argtypes = [P, ct.POINTER(ct.c_int)]
    lib.rx_kk_process.argtypes = [P, P, ct.c_int, ct.c_int64, ct.c_float, ct.c_float, P, P]
    lib.rx_kk_profile.argtypes = [P, ct.c_int, ct.POINTER(ct.c_double), ct.c_int]
    lib.rx_kk_set_position.argtypes = [P, ct.c_int64]
    lib.rx_kk_flush.argtypes = [P, P, P]
    lib.rx_kk_get_delay.argtypes = [P, ct.POINTER(ct.c_int)]
    lib.rx_kk_destroy.argtypes = [P]
    lib.rx_kk_destroy.restype = None
    lib.rx_kk_last_error.argtypes = [P]
    lib.rx_kk_last_error.restype = ct.c_char_p
    lib.rx_wl_create.argtypes = [ct.POINTER(P), ct.c_int, ct.c_int, ct.c_int64]
    lib.rx_wl_set_param.argtypes = [P, ct.c_int, ct.c_double]
    lib.rx_wl_get_param.argtypes = [P, ct.c_int, ct.POINTER(ct.c_double)]
    lib.rx_wl_set_cuda_stream.argtypes = [P, P]
    lib.rx_wl_set_taps.argtypes = [P, ct.POINTER(ct.c_float)]
    lib.rx_wl_get_taps.argtypes = [P, ct.POINTER(ct.c_double)]
    lib.rx_wl_process.argtypes = [P, P, ct.c_int64, P, P]
    lib.rx_wl_reset.argtypes = [P]
    lib.rx_wl_profile.argtypes = [P, ct.c_int, ct.POINTER(ct.c_double), ct.c_int]
    lib.rx_wl_destroy.argtypes = [P]
    lib.rx_wl_destroy.restype = None
    lib.rx_wl_last_error.argtypes = [P]
    lib.rx_wl_last_error.restype = ct.c_char_p
    lib.rx_rt_create.argtypes = [ct.POINTER(P), ct.POINTER(rx_rt_cfg)]
    lib.rx_rt_set_wl_param.argtypes = [P, ct.c_int, ct.c_double]
    lib.rx_rt_next_input.argtypes = [P, ct.POINTER(P)]
    lib.rx_rt_submit.argtypes = [P, ct.POINTER(ct.c_int64)]
    lib.rx_rt_output.argtypes = [P, ct.c_int64, ct.POINTER(P)]
    lib.rx_rt_flush.argtypes = [P, ct.POINTER(ct.c_int64)]
    lib.rx_rt_submit_from.argtypes = [P, P, ct.POINTER(ct.c_int64)]
    lib.rx_rt_drain.argtypes = [P]
    lib.rx_rt_bins.argtypes = [P, ct.c_int, ct.c_int, P, P, P, ct.POINTER(ct.c_int)]
    lib.rx_rt_profile.argtypes = [P, ct.c_int, ct.POINTER(ct.c_double), ct.c_int]
    lib.rx_rt_destroy.argtypes = [P]
    lib.rx_rt_destroy.restype = None
    lib.rx_rt_last_error.argtypes = [P]
    lib.rx_rt_last_error.restype = ct.c_char_p
    lib.rx_q_db.argtypes = [ct.c_double]
    lib.rx_q_db.restype = ct.c_double
    lib.rx_cnn_destroy.argtypes = [P]
    lib.rx_cnn_destroy.restype = None
    lib.rx_cnn_last_error.argtypes = [P]
    lib.rx_cnn_last_error.restype = ct.c_char_p
    for name in EXPORTS:
        if name not in ("rx_destroy", "rx_status_str", "rx_last_error", "rx_batch_destroy", "rx_batch_last_error",
                        "rx_cnn_param_count", "rx_cnn_destroy", "rx_cnn_last_error", "rx_kk_destroy",
                        "rx_kk_last_error", "rx_wl_destroy", "rx_wl_last_error", "rx_rt_destroy",
                        "rx_rt_last_error", "rx_q_db"):
            getattr(lib, name).restype = ct.c_int
    _lib = lib
    return lib


def measure_alu_peak(kind="fp32", iters=None, stream=None):
    """Measured FP32 / FP64 FMA throughput (TFLOP/s, ms) of this GPU (rx_measure_alu_peak)."""
    lib = load()
    k = {"fp32": 0, "fp64": 1}[kind]
    iters = iters or (8192 if k == 0 else 256)
    tf, ms = ct.c_double(), ct.c_double()
    st = lib.rx_measure_alu_peak(k, int(iters), ct.c_void_p(stream), ct.byref(tf), ct.byref(ms))
    if st != RX_OK:
        raise RxError(st, "rx_measure_alu_peak failed")
    return tf.value, ms.value


def _check(lib, h, status):
    if status != RX_OK:
        detail = lib.rx_last_error(h).decode() if h else ""
        raise RxError(status, f"{lib.rx_status_str(status).decode()}: {detail}")


class Receiver:
    """One receiver stream on the current CUDA device (torch tensors in and out)."""

    def __init__(self, baud, L_km, D=17.0, ntaps=15, bps_angles=32, sps=2, stream=None, **params):
        import torch  # device memory and streams only
        self.torch = torch
        self.lib = load()
        h = ct.c_void_p()
        _check(self.lib, None, self.lib.rx_create(ct.byref(h), baud, sps, L_km, D, ntaps, bps_angles))
        self.h = h
        self.ntaps = ntaps
        if stream is not None:
            self.set_cuda_stream(stream)
        for k, v in params.items():
            self.set_param(k, v)

    # -- C names
    def rx_set_param(self, key, value):
        _check(self.lib, self.h, self.lib.rx_set_param(self.h, PARAMS[key.upper()] if isinstance(key, str) else key, float(value)))

    set_param = rx_set_param

    def rx_get_param(self, key):
        v = ct.c_double()
        _check(self.lib, self.h, self.lib.rx_get_param(self.h, PARAMS[key.upper()] if isinstance(key, str) else key, ct.byref(v)))
        return v.value

    get_param = rx_get_param

    def set_cuda_stream(self, stream):
        ptr = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
        _check(self.lib, self.h, self.lib.rx_set_cuda_stream(self.h, ct.c_void_p(ptr)))

    def rx_reserve(self, max_call_samples):
        _check(self.lib, self.h, self.lib.rx_reserve(self.h, int(max_call_samples)))

    reserve = rx_reserve

    def rx_reset(self):
        _check(self.lib, self.h, self.lib.rx_reset(self.h))

    reset = rx_reset

    def rx_sync(self):
        _check(self.lib, self.h, self.lib.rx_sync(self.h))

    sync = rx_sync

    @property
    def bits_per_symbol(self):
        return int(self.get_param("MOD"))

    def alloc_out(self, capacity, llr=False, sym=False, eq=False, cdc=False):
        t = self.torch
        m = self.bits_per_symbol
        words = (capacity * m + 31) // 32
        o = {"bits": t.zeros((2, words), dtype=t.int32, device="cuda"), "capacity": capacity}
        if llr:
            # LLR_OUT = 2 writes binary16 LLRs
            dt = t.float16 if int(self.get_param("LLR_OUT")) == 2 else t.float32
            o["llr"] = t.zeros((2, capacity * m), dtype=dt, device="cuda")
        if sym:
            o["sym"] = t.zeros((2, capacity), dtype=t.complex64, device="cuda")
        if eq:
            o["eq"] = t.zeros((2, capacity), dtype=t.complex64, device="cuda")
        if cdc:
            o["cdc"] = t.zeros((2, 2 * capacity + 65536), dtype=t.complex64, device="cuda")
        return o

    def rx_process(self, samples, out, sym_offset=0, cdc_offset=0):
        """Process a (n, 4) int8/float32 CUDA tensor (None = flush).

        Writes into the tensors of `out` (from alloc_out) starting at symbol
        column `sym_offset` (CDC samples at column `cdc_offset`) and returns
        (first, n, cdc_first, cdc_n).
        """
        t = self.torch
        i = rx_in()
        if samples is None:
            i.data, i.n, i.dtype = None, 0, RX_F32x4
        else:
            assert samples.is_cuda and samples.is_contiguous() and samples.shape[-1] == 4
            i.data = samples.data_ptr()
            i.n = samples.shape[0]
            i.dtype = RX_I8x4 if samples.dtype == t.int8 else RX_F32x4
        o = rx_out()
        m = self.bits_per_symbol
        assert (sym_offset * m) % 32 == 0
        bits = out["bits"]
        o.bits = bits.data_ptr() + (sym_offset * m // 32) * 4
        o.bits_stride = bits.shape[1]
        if "llr" in out:
            o.llr = out["llr"].data_ptr() + sym_offset * m * out["llr"].element_size()
            o.llr_stride = out["llr"].shape[1]
        if "sym" in out:
            o.sym = out["sym"].data_ptr() + sym_offset * 8
            o.sym_stride = out["sym"].shape[1]
        if "eq" in out:
            o.eq = out["eq"].data_ptr() + sym_offset * 8
            o.eq_stride = out["eq"].shape[1]
        if "cdc" in out:
            o.cdc = out["cdc"].data_ptr() + cdc_offset * 8
            o.cdc_stride = out["cdc"].shape[1]
        o.capacity = out["capacity"] - sym_offset
        _check(self.lib, self.h, self.lib.rx_process(self.h, ct.byref(i), ct.byref(o)))
        return o.first, o.n, o.cdc_first, o.cdc_n

    process = rx_process

    def rx_ber(self, rx_bits, ref_bits, n_symbols):
        """(errors, bits_counted, sync) with rx_bits/ref_bits (2, words) int32 CUDA tensors."""
        e, n = ct.c_uint64(), ct.c_uint64()
        sync = (ct.c_int32 * 6)()
        _check(self.lib, self.h, self.lib.rx_ber(self.h, rx_bits.data_ptr(), rx_bits.shape[1], ref_bits.data_ptr(),
                                                 ref_bits.shape[1], int(n_symbols), ct.byref(e), ct.byref(n), sync))
        return e.value, n.value, [tuple(sync[3 * p:3 * p + 3]) for p in range(2)]

    ber = rx_ber

    def rx_trace(self, wave):
        import numpy as np
        taps = (ct.c_float * (2 * 2 * self.ntaps * 2))()
        dw, Phi = ct.c_double(), ct.c_double()
        _check(self.lib, self.h, self.lib.rx_trace(self.h, int(wave), taps, ct.byref(dw), ct.byref(Phi)))
        a = np.frombuffer(taps, dtype=np.float32).astype(np.float64)
        return (a[0::2] + 1j * a[1::2]).reshape(2, 2, self.ntaps), dw.value, Phi.value

    trace = rx_trace

    def rx_trace_inner(self, first=0, count=None):
        """Inner BPS angles per DD update block: (int8 array [2][count], n_acq, per_segment)."""
        import numpy as np
        if count is None:
            count = int(self.get_param("INNER_TRACE")) - first
        buf = np.full((2, max(count, 0)), -1, np.int8)
        na, ps = ct.c_int64(), ct.c_int32()
        _check(self.lib, self.h, self.lib.rx_trace_inner(self.h, int(first), int(count),
                                                         buf.ctypes.data if count > 0 else None,
                                                         ct.byref(na), ct.byref(ps)))
        return buf, na.value, ps.value

    trace_inner = rx_trace_inner

    def rx_get_state(self) -> bytes:
        n = ct.c_size_t()
        _check(self.lib, self.h, self.lib.rx_get_state(self.h, None, ct.byref(n)))
        buf = ct.create_string_buffer(n.value)
        _check(self.lib, self.h, self.lib.rx_get_state(self.h, buf, ct.byref(n)))
        return buf.raw[:n.value]

    get_state = rx_get_state

    def rx_set_state(self, blob: bytes):
        _check(self.lib, self.h, self.lib.rx_set_state(self.h, blob, len(blob)))

    set_state = rx_set_state

    def rx_profile(self, reset=False):
        """{stage: (ms, launches)} since the last reset of the counters."""
        ms = (ct.c_double * len(STAGES))()
        n = (ct.c_int64 * len(STAGES))()
        _check(self.lib, self.h, self.lib.rx_profile(self.h, ms, n, 1 if reset else 0))
        return {k: (ms[i], n[i]) for i, k in enumerate(STAGES)}

    profile = rx_profile

    def close(self):
        if getattr(self, "h", None):
            self.lib.rx_destroy(self.h)
            self.h = None

    rx_destroy = close

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def run_stream(self, samples, chunk=None, llr=False, sym=False, eq=False, cdc=False, out=None):
        """Reset, process `samples` in calls of `chunk` sample-times, flush; returns outputs."""
        n = samples.shape[0]
        K = n // 2
        chunk = chunk or n
        if out is None:
            out = self.alloc_out(K + 64, llr=llr, sym=sym, eq=eq, cdc=cdc)
        self.reset()
        pos = cpos = 0
        for a in list(range(0, n, chunk)) + [None]:
            piece = None if a is None else samples[a:a + chunk]
            first, cnt, cfirst, cn = self.process(piece, out, sym_offset=pos, cdc_offset=cpos)
            assert first == pos and (cn == 0 or cfirst == cpos)
            pos += cnt
            cpos += cn
        out["n"] = pos
        out["cdc_n"] = cpos
        return out


def _bcheck(lib, h, status):
    if status != RX_OK:
        detail = lib.rx_batch_last_error(h).decode() if h else ""
        raise RxError(status, f"{lib.rx_status_str(status).decode()}: {detail}")


class Batch:
    """Batched form (include/rx_batch.h): many channels, whole streams, one enqueue.

    cfgs: list of dicts with keys baud, L_km, D (17), in_scale (1), max_samples,
    mod_bits (2), ntaps (15), fft_n (0 = autotuned), overlap (0 = default).
    """

    def __init__(self, cfgs, stream=None):
        import torch
        self.torch = torch
        self.lib = load()
        n = len(cfgs)
        arr = (rx_chan_cfg * n)()
        for i, c in enumerate(cfgs):
            arr[i] = rx_chan_cfg(float(c["baud"]), float(c["L_km"]), float(c.get("D", 17.0)),
                                 float(c.get("in_scale", 1.0)), int(c["max_samples"]), int(c.get("mod_bits", 2)),
                                 int(c.get("ntaps", 15)), int(c.get("fft_n", 0)), int(c.get("overlap", 0)),
                                 int(c.get("flags", 0)), int(c.get("bps_halfwin", 0)))
        h = ct.c_void_p()
        st = self.lib.rx_batch_create(ct.byref(h), n, arr)
        if st != RX_OK:
            msg = self.lib.rx_batch_last_error(h).decode() if h else ""
            if h:
                self.lib.rx_batch_destroy(h)
            raise RxError(st, f"{self.lib.rx_status_str(st).decode()}: {msg}")
        self.h = h
        self.n_ch = n
        self.cfgs = [dict(c) for c in cfgs]
        if stream is not None:
            self.set_cuda_stream(stream)

    def set_cuda_stream(self, stream):
        ptr = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
        _bcheck(self.lib, self.h, self.lib.rx_batch_set_cuda_stream(self.h, ct.c_void_p(ptr)))

    def rx_batch_set_param(self, key, value):
        k = BATCH_PARAMS[key.upper()] if isinstance(key, str) else key
        _bcheck(self.lib, self.h, self.lib.rx_batch_set_param(self.h, k, float(value)))

    set_param = rx_batch_set_param

    def rx_batch_get_param(self, ch, key):
        if isinstance(key, str):
            key = BATCH_PARAMS.get(key.upper()) or PARAMS[key.upper()]
        v = ct.c_double()
        _bcheck(self.lib, self.h, self.lib.rx_batch_get_param(self.h, int(ch), key, ct.byref(v)))
        return v.value

    get_param = rx_batch_get_param

    def bits_per_symbol(self, ch):
        return int(self.cfgs[ch].get("mod_bits", 2))

    def alloc_outs(self, samples, llr=False, sym=False, eq=False, cdc=False):
        t = self.torch
        outs = []
        for ch, x in enumerate(samples):
            K = x.shape[0] // 2
            m = self.bits_per_symbol(ch)
            cap = K + 32
            o = {"bits": t.zeros((2, (cap * m + 31) // 32), dtype=t.int32, device="cuda"), "capacity": cap}
            if llr:
                o["llr"] = t.zeros((2, cap * m), dtype=t.float32, device="cuda")
            if sym:
                o["sym"] = t.zeros((2, cap), dtype=t.complex64, device="cuda")
            if eq:
                o["eq"] = t.zeros((2, cap), dtype=t.complex64, device="cuda")
            if cdc:
                o["cdc"] = t.zeros((2, x.shape[0] + 64), dtype=t.complex64, device="cuda")
            outs.append(o)
        return outs

    def rx_batch_process(self, samples, outs):
        """samples: list of (n_c, 4) int8/float32 CUDA tensors; outs from alloc_outs."""
        t = self.torch
        n = self.n_ch
        ins = (rx_in * n)()
        os_ = (rx_out * n)()
        for c in range(n):
            x = samples[c]
            if x is None or x.shape[0] == 0:
                ins[c].data, ins[c].n, ins[c].dtype = None, 0, RX_F32x4
            else:
                assert x.is_cuda and x.is_contiguous() and x.shape[-1] == 4
                ins[c].data = x.data_ptr()
                ins[c].n = x.shape[0]
                ins[c].dtype = RX_I8x4 if x.dtype == t.int8 else RX_F32x4
            o = outs[c]
            os_[c].bits = o["bits"].data_ptr()
            os_[c].bits_stride = o["bits"].shape[1]
            for k in ("llr", "sym", "eq", "cdc"):
                if k in o:
                    setattr(os_[c], k, o[k].data_ptr())
                    setattr(os_[c], k + "_stride", o[k].shape[1])
            os_[c].capacity = o["capacity"]
        _bcheck(self.lib, self.h, self.lib.rx_batch_process(self.h, ins, os_))
        for c in range(n):
            outs[c]["n"] = os_[c].n
            outs[c]["cdc_n"] = os_[c].cdc_n
        return outs

    process = rx_batch_process

    def rx_batch_ber(self, ch, rx_bits, ref_bits, n_symbols):
        e, n = ct.c_uint64(), ct.c_uint64()
        sync = (ct.c_int32 * 6)()
        _bcheck(self.lib, self.h, self.lib.rx_batch_ber(self.h, int(ch), rx_bits.data_ptr(), rx_bits.shape[1],
                                                        ref_bits.data_ptr(), ref_bits.shape[1], int(n_symbols),
                                                        ct.byref(e), ct.byref(n), sync))
        return e.value, n.value, [tuple(sync[3 * p:3 * p + 3]) for p in range(2)]

    ber = rx_batch_ber

    def rx_batch_trace(self, ch, wave):
        import numpy as np
        T = int(self.cfgs[ch].get("ntaps", 15))
        taps = (ct.c_float * (2 * 2 * T * 2))()
        dw, Phi = ct.c_double(), ct.c_double()
        _bcheck(self.lib, self.h, self.lib.rx_batch_trace(self.h, int(ch), int(wave), taps, ct.byref(dw), ct.byref(Phi)))
        a = np.frombuffer(taps, dtype=np.float32).astype(np.float64)
        return (a[0::2] + 1j * a[1::2]).reshape(2, 2, T), dw.value, Phi.value

    trace = rx_batch_trace

    def rx_batch_profile(self, reset=False):
        """{stage: (ms, launches)} since the last reset of the counters."""
        ms = (ct.c_double * len(STAGES))()
        n = (ct.c_int64 * len(STAGES))()
        _bcheck(self.lib, self.h, self.lib.rx_batch_profile(self.h, ms, n, 1 if reset else 0))
        return {k: (ms[i], n[i]) for i, k in enumerate(STAGES)}

    profile = rx_batch_profile

    def rx_batch_sync(self):
        _bcheck(self.lib, self.h, self.lib.rx_batch_sync(self.h))

    sync = rx_batch_sync

    def close(self):
        if getattr(self, "h", None):
            self.lib.rx_batch_destroy(self.h)
            self.h = None

    rx_batch_destroy = close

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _ccheck(lib, h, status):
    if status != RX_OK:
        detail = lib.rx_cnn_last_error(h).decode() if h else ""
        raise RxError(status, f"{lib.rx_status_str(status).decode()}: {detail}")


class CNN:
    """Learned post-equaliser (include/rx_cnn.h) on the current CUDA device.

    Symbols in and out are (2, K) complex64 CUDA tensors (rows = polarisations).
    """

    def __init__(self, max_symbols, layers=4, channels=64, ksize=15, stream=None):
        import torch
        self.torch = torch
        self.lib = load()
        h = ct.c_void_p()
        _ccheck(self.lib, None, self.lib.rx_cnn_create(ct.byref(h), layers, channels, ksize, int(max_symbols)))
        self.h = h
        self.layers = layers
        self.n_params = int(self.lib.rx_cnn_param_count(h))
        if stream is not None:
            ptr = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
            _ccheck(self.lib, self.h, self.lib.rx_cnn_set_cuda_stream(self.h, ct.c_void_p(ptr)))

    @staticmethod
    def flatten(params):
        """[(W (15, ci, co), b (co,)), ...] -> flat float32 in the library's layout."""
        import numpy as np
        return np.concatenate([np.concatenate([np.asarray(W, np.float64).ravel(), np.asarray(b, np.float64).ravel()])
                               for W, b in params]).astype(np.float32)

    def unflatten(self, flat, channels=64, ksize=15):
        import numpy as np
        dims = [4] + [channels] * (self.layers - 1) + [4]
        out, o = [], 0
        for l in range(self.layers):
            ci, co = dims[l], dims[l + 1]
            W = np.asarray(flat[o:o + ksize * ci * co], np.float64).reshape(ksize, ci, co)
            o += ksize * ci * co
            b = np.asarray(flat[o:o + co], np.float64)
            o += co
            out.append((W, b))
        return out

    def rx_cnn_set_params(self, params):
        import numpy as np
        flat = np.ascontiguousarray(params if isinstance(params, np.ndarray) else self.flatten(params), np.float32)
        assert flat.size == self.n_params
        _ccheck(self.lib, self.h, self.lib.rx_cnn_set_params(self.h, flat.ctypes.data))

    set_params = rx_cnn_set_params

    def rx_cnn_get_params(self):
        import numpy as np
        flat = np.empty(self.n_params, np.float32)
        _ccheck(self.lib, self.h, self.lib.rx_cnn_get_params(self.h, flat.ctypes.data))
        return flat

    get_params = rx_cnn_get_params

    def _sym(self, z):
        assert z.is_cuda and z.dtype == self.torch.complex64 and z.shape[0] == 2 and z.stride(1) == 1
        return z.data_ptr(), z.stride(0)

    def rx_cnn_apply(self, z, out=None):
        K = z.shape[1]
        if out is None:
            out = self.torch.empty_like(z)
        zp, zs = self._sym(z)
        yp, ys = self._sym(out)
        _ccheck(self.lib, self.h, self.lib.rx_cnn_apply(self.h, zp, zs, yp, ys, K))
        return out

    apply = rx_cnn_apply

    def rx_cnn_grads(self, z, t):
        """(loss, flat float32 gradient tensor on the device)."""
        g = self.torch.empty(self.n_params, dtype=self.torch.float32, device="cuda")
        loss = ct.c_double()
        zp, zs = self._sym(z)
        tp, ts = self._sym(t)
        _ccheck(self.lib, self.h, self.lib.rx_cnn_grads(self.h, zp, zs, tp, ts, z.shape[1], g.data_ptr(), ct.byref(loss)))
        return loss.value, g

    grads = rx_cnn_grads

    def rx_cnn_train_step(self, z, t, lr=1e-3, loss_acc=None):
        zp, zs = self._sym(z)
        tp, ts = self._sym(t)
        acc = loss_acc.data_ptr() if loss_acc is not None else None
        _ccheck(self.lib, self.h, self.lib.rx_cnn_train_step(self.h, zp, zs, tp, ts, z.shape[1], float(lr), acc))

    train_step = rx_cnn_train_step

    def rx_cnn_set_option(self, key, value):
        k = {"TCGEN05": 1}[key.upper()] if isinstance(key, str) else key
        _ccheck(self.lib, self.h, self.lib.rx_cnn_set_option(self.h, k, int(value)))

    set_option = rx_cnn_set_option

    def rx_cnn_set_profile(self, on=True):
        _ccheck(self.lib, self.h, self.lib.rx_cnn_set_profile(self.h, 1 if on else 0))

    set_profile = rx_cnn_set_profile

    def rx_cnn_profile(self, reset=False):
        """{kind: (ms, launches)} since the last reset."""
        ms = (ct.c_double * len(CNN_KINDS))()
        n = (ct.c_int64 * len(CNN_KINDS))()
        _ccheck(self.lib, self.h, self.lib.rx_cnn_profile(self.h, ms, n, 1 if reset else 0))
        return {k: (ms[i], n[i]) for i, k in enumerate(CNN_KINDS)}

    profile = rx_cnn_profile

    def close(self):
        if getattr(self, "h", None):
            self.lib.rx_cnn_destroy(self.h)
            self.h = None

    rx_cnn_destroy = close

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _kcheck(lib, h, status):
    if status != RX_OK:
        detail = lib.rx_kk_last_error(h).decode() if h else ""
        raise RxError(status, f"{lib.rx_status_str(status).decode()}: {detail}")


class KKFrontEnd:
    """Kramers-Kronig receiver front end (include/rx_kk.h): real intensity samples
    at 4 samples/symbol -> rebuilt field at 2 samples/symbol (complex64 tensors)."""

    def __init__(self, baud, carrier_hz, L_km, max_samples, D=17.0, rolloff=0.01, sps=4, stream=None):
        import torch
        self.torch = torch
        self.lib = load()
        h = ct.c_void_p()
        st = self.lib.rx_kk_create(ct.byref(h), float(baud), int(sps), float(carrier_hz), float(L_km), float(D),
                                   float(rolloff), int(max_samples))
        if st != RX_OK:
            msg = self.lib.rx_kk_last_error(h).decode() if h else ""
            if h:
                self.lib.rx_kk_destroy(h)
            raise RxError(st, f"{self.lib.rx_status_str(st).decode()}: {msg}")
        self.h = h
        if stream is not None:
            ptr = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
            _kcheck(self.lib, self.h, self.lib.rx_kk_set_cuda_stream(self.h, ct.c_void_p(ptr)))

    @property
    def overlap(self):
        v = ct.c_int()
        _kcheck(self.lib, self.h, self.lib.rx_kk_get_overlap(self.h, ct.byref(v)))
        return v.value

    @property
    def delay(self):
        v = ct.c_int()
        _kcheck(self.lib, self.h, self.lib.rx_kk_get_delay(self.h, ct.byref(v)))
        return v.value

    def rx_kk_flush(self, field=False, out=None):
        """The last `delay` output samples of the stream -> (y at 2 sps, field or None)."""
        t = self.torch
        d = self.delay
        y = out if out is not None else t.empty(d // 2, dtype=t.complex64, device="cuda")
        f = t.empty(d, dtype=t.complex64, device="cuda") if field else None
        _kcheck(self.lib, self.h, self.lib.rx_kk_flush(self.h, y.data_ptr(), f.data_ptr() if f is not None else None))
        return y, f

    flush = rx_kk_flush

    def rx_kk_process(self, samples, in_scale=1.0, in_offset=0.0, field=False, out=None):
        """samples: 1-D int8 or float32 CUDA tensor (a multiple of 512 long) -> (y at 2 sps,
        field at the input rate or None), both `delay` samples behind the input."""
        t = self.torch
        assert samples.is_cuda and samples.is_contiguous() and samples.dim() == 1
        n = samples.shape[0]
        dt = 1 if samples.dtype == t.int8 else 2
        y = out if out is not None else t.empty(n // 2, dtype=t.complex64, device="cuda")
        f = t.empty(n, dtype=t.complex64, device="cuda") if field else None
        _kcheck(self.lib, self.h, self.lib.rx_kk_process(self.h, samples.data_ptr(), dt, n, float(in_scale),
                                                         float(in_offset), y.data_ptr(),
                                                         f.data_ptr() if f is not None else None))
        return y, f

    process = rx_kk_process

    def rx_kk_set_position(self, pos=0):
        _kcheck(self.lib, self.h, self.lib.rx_kk_set_position(self.h, int(pos)))

    set_position = rx_kk_set_position

    def rx_kk_profile(self, on=True, reset=False):
        ms = (ct.c_double * 2)()
        _kcheck(self.lib, self.h, self.lib.rx_kk_profile(self.h, 1 if on else 0, ms, 1 if reset else 0))
        return {"hilbert": ms[0], "filter": ms[1]}

    profile = rx_kk_profile

    def close(self):
        if getattr(self, "h", None):
            self.lib.rx_kk_destroy(self.h)
            self.h = None

    rx_kk_destroy = close

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _wcheck(lib, h, status):
    if status != RX_OK:
        detail = lib.rx_wl_last_error(h).decode() if h else ""
        raise RxError(status, f"{lib.rx_status_str(status).decode()}: {detail}")


class WLEqualiser:
    """Four-tap widely-linear DD-LMS equaliser (include/rx_wl.h): complex64 field
    at 2 samples/symbol -> packed Gray bits (int32 words) and optional outputs."""

    def __init__(self, mod_bits, max_symbols, ntaps=4, stream=None, **params):
        import torch
        self.torch = torch
        self.lib = load()
        self.mod_bits = int(mod_bits)
        h = ct.c_void_p()
        st = self.lib.rx_wl_create(ct.byref(h), self.mod_bits, int(ntaps), int(max_symbols))
        if st != RX_OK:
            raise RxError(st, self.lib.rx_status_str(st).decode())
        self.h = h
        self.ntaps = int(ntaps)
        if stream is not None:
            ptr = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
            _wcheck(self.lib, self.h, self.lib.rx_wl_set_cuda_stream(self.h, ct.c_void_p(ptr)))
        for k, v in params.items():
            self.rx_wl_set_param(k, v)

    def rx_wl_set_param(self, key, value):
        _wcheck(self.lib, self.h, self.lib.rx_wl_set_param(self.h, WL_PARAMS[key.upper()], float(value)))

    set_param = rx_wl_set_param

    def rx_wl_get_param(self, key):
        v = ct.c_double()
        _wcheck(self.lib, self.h, self.lib.rx_wl_get_param(self.h, WL_PARAMS[key.upper()], ct.byref(v)))
        return v.value

    get_param = rx_wl_get_param

    def rx_wl_set_taps(self, taps):
        """taps: (2, T) complex array-like, row 0 = h on x, row 1 = g on conj(x)."""
        import numpy as np
        t = np.asarray(taps, np.complex128).reshape(2, self.ntaps)
        flat = np.stack([t.real, t.imag], -1).reshape(-1).astype(np.float32)
        _wcheck(self.lib, self.h, self.lib.rx_wl_set_taps(self.h, flat.ctypes.data_as(ct.POINTER(ct.c_float))))

    set_taps = rx_wl_set_taps

    def rx_wl_get_taps(self):
        import numpy as np
        buf = (ct.c_double * (4 * self.ntaps))()
        _wcheck(self.lib, self.h, self.lib.rx_wl_get_taps(self.h, buf))
        a = np.frombuffer(buf, np.float64).reshape(2, self.ntaps, 2)
        return a[..., 0] + 1j * a[..., 1]

    get_taps = rx_wl_get_taps

    def rx_wl_process(self, x, want_z=False, bits=None):
        """x: 1-D complex64 CUDA tensor (2 samples/symbol) -> (bits int32 words, z complex64 or None)."""
        t = self.torch
        assert x.is_cuda and x.is_contiguous() and x.dim() == 1 and x.dtype == t.complex64
        n = x.shape[0]
        K = n // 2
        words = (K * self.mod_bits + 31) // 32
        b = bits if bits is not None else t.empty(max(words, 1), dtype=t.int32, device="cuda")
        z = t.empty(K, dtype=t.complex64, device="cuda") if want_z else None
        _wcheck(self.lib, self.h, self.lib.rx_wl_process(self.h, x.data_ptr(), n, b.data_ptr(),
                                                         z.data_ptr() if z is not None else None))
        return b[:words], z

    process = rx_wl_process

    def rx_wl_reset(self):
        _wcheck(self.lib, self.h, self.lib.rx_wl_reset(self.h))

    reset = rx_wl_reset

    def rx_wl_profile(self, on=True, reset=False):
        ms = (ct.c_double * 2)()
        _wcheck(self.lib, self.h, self.lib.rx_wl_profile(self.h, 1 if on else 0, ms, 1 if reset else 0))
        return {"acquisition": ms[0], "segments": ms[1]}

    profile = rx_wl_profile

    def close(self):
        if getattr(self, "h", None):
            self.lib.rx_wl_destroy(self.h)
            self.h = None

    rx_wl_destroy = close

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _rcheck(lib, h, status):
    if status != RX_OK:
        detail = lib.rx_rt_last_error(h).decode() if h else ""
        raise RxError(status, f"{lib.rx_status_str(status).decode()}: {detail}")


def q_db(ber):
    """Q in dB of a bit-error ratio (rx_q_db, host only)."""
    return load().rx_q_db(float(ber))


class RealTime:
    """Real-time ingest pipeline of the KK receiver (include/rx_rt.h): pinned host
    input ring -> copy / front end / equaliser / copy-out streams -> bits in a pinned
    host ring, with BER counted against the transmitted pattern in Q bins."""

    def __init__(self, baud, carrier_hz, L_km, buffer_samples, mod_bits=4, depth=4, in_dtype="int8",
                 in_scale=1.0, in_offset=0.0, ref_bits=None, bin_symbols=1 << 20, edge_symbols=0,
                 max_bins=4096, D=17.0, rolloff=0.01, sps=4, **wl_params):
        import numpy as np
        self.np = np
        self.lib = load()
        self.n = int(buffer_samples)
        self.K = self.n // sps
        self.words = self.K * int(mod_bits) // 32
        self.dtype = np.int8 if in_dtype == "int8" else np.float32
        ref = None
        if ref_bits is not None:
            ref = np.ascontiguousarray(np.asarray(ref_bits, np.uint8))
        cfg = rx_rt_cfg(baud=float(baud), sps=int(sps), mod_bits=int(mod_bits), carrier_hz=float(carrier_hz),
                        L_km=float(L_km), D_ps_nm_km=float(D), rolloff=float(rolloff),
                        in_dtype=1 if in_dtype == "int8" else 2, in_scale=float(in_scale),
                        in_offset=float(in_offset), buffer_samples=self.n, depth=int(depth),
                        ref_bits=ref.ctypes.data if ref is not None else None,
                        ref_nbits=int(ref.shape[0]) if ref is not None else 0, bin_symbols=int(bin_symbols),
                        edge_symbols=int(edge_symbols), max_bins=int(max_bins))
        h = ct.c_void_p()
        st = self.lib.rx_rt_create(ct.byref(h), ct.byref(cfg))
        if st != RX_OK:
            raise RxError(st, self.lib.rx_status_str(st).decode())
        self.h = h
        for k, v in wl_params.items():
            _rcheck(self.lib, self.h, self.lib.rx_rt_set_wl_param(self.h, WL_PARAMS[k.upper()], float(v)))

    def rx_rt_next_input(self):
        """numpy view of the pinned host slot for the next buffer (write n samples, then submit)."""
        p = ct.c_void_p()
        _rcheck(self.lib, self.h, self.lib.rx_rt_next_input(self.h, ct.byref(p)))
        ctype = ct.c_int8 if self.dtype == self.np.int8 else ct.c_float
        return self.np.ctypeslib.as_array(ct.cast(p, ct.POINTER(ctype)), shape=(self.n,))

    next_input = rx_rt_next_input

    def rx_rt_submit(self):
        b = ct.c_int64()
        _rcheck(self.lib, self.h, self.lib.rx_rt_submit(self.h, ct.byref(b)))
        return b.value

    submit = rx_rt_submit

    def rx_rt_submit_from(self, samples):
        """Enqueue a buffer from the caller's host memory (a contiguous numpy array or
        pinned CPU tensor of n samples), kept unchanged until its output is read."""
        ptr = samples.data_ptr() if hasattr(samples, "data_ptr") else samples.ctypes.data
        b = ct.c_int64()
        _rcheck(self.lib, self.h, self.lib.rx_rt_submit_from(self.h, ct.c_void_p(ptr), ct.byref(b)))
        return b.value

    submit_from = rx_rt_submit_from

    def rx_rt_flush(self):
        """End of the input: the last delayed symbols as one more block; returns its index."""
        b = ct.c_int64()
        _rcheck(self.lib, self.h, self.lib.rx_rt_flush(self.h, ct.byref(b)))
        return b.value

    flush = rx_rt_flush

    def rx_rt_output(self, b):
        """numpy view (uint32 words) of buffer b's bits in the pinned host ring; waits for it."""
        p = ct.c_void_p()
        _rcheck(self.lib, self.h, self.lib.rx_rt_output(self.h, int(b), ct.byref(p)))
        return self.np.ctypeslib.as_array(ct.cast(p, ct.POINTER(ct.c_uint32)), shape=(self.words,))

    output = rx_rt_output

    def rx_rt_drain(self):
        _rcheck(self.lib, self.h, self.lib.rx_rt_drain(self.h))

    drain = rx_rt_drain

    def rx_rt_bins(self, first=0, count=None):
        np = self.np
        nb = ct.c_int()
        _rcheck(self.lib, self.h, self.lib.rx_rt_bins(self.h, 0, 0, None, None, None, ct.byref(nb)))
        count = nb.value - first if count is None else count
        count = max(count, 0)
        e = np.zeros(count, np.uint64)
        b = np.zeros(count, np.uint64)
        q = np.zeros(count, np.float64)
        _rcheck(self.lib, self.h, self.lib.rx_rt_bins(self.h, int(first), count, e.ctypes.data, b.ctypes.data,
                                                      q.ctypes.data, ct.byref(nb)))
        return {"errors": e, "bits": b, "q_db": q}

    bins = rx_rt_bins

    def rx_rt_profile(self, on=True, reset=False):
        ms = (ct.c_double * 4)()
        _rcheck(self.lib, self.h, self.lib.rx_rt_profile(self.h, 1 if on else 0, ms, 1 if reset else 0))
        return {"copy_in": ms[0], "front_end": ms[1], "equaliser": ms[2], "copy_out": ms[3]}

    profile = rx_rt_profile

    def close(self):
        if getattr(self, "h", None):
            self.lib.rx_rt_destroy(self.h)
            self.h = None

    rx_rt_destroy = close

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
