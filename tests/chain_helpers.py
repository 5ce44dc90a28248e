"""Shared helpers for the GPU parity tests: run the CUDA chain and the FP64
oracle on the same seeded input and compare them element by element."""
from __future__ import annotations

import math
import os

import numpy as np

import linksim as L
import oracle as O

# FP32 path vs FP64 oracle: relative RMS of complex outputs (the parity tolerance)
REL_RMS_TOL = 1e-4
# decisions may differ only where the oracle's soft value is this close to a boundary
BOUNDARY_EPS = 1e-5


def ensure_built():
    from paper_2104_06311_gb300 import build as B
    if not os.path.exists(B.OUT):
        B.build()


def rel_rms(a, b) -> float:
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.sqrt(np.sum(np.abs(a - b) ** 2) / max(np.sum(np.abs(b) ** 2), 1e-300)))


def rx_params(link: L.Link, in_scale: float, **over) -> O.RxParams:
    p = O.RxParams(baud=link.baud, L_km=link.L_km, D=link.D, mod=link.mod, in_scale=in_scale)
    for k, v in over.items():
        setattr(p, k, v)
    return p.resolved()


_KEYMAP = dict(fft_n="FFT_N", overlap="OVERLAP", mu_cma="MU_CMA", mu_dd="MU_DD", n_cma="N_CMA",
               upd_block="UPDATE_BLOCK", seg_len="SEG_LEN", seg_pretrain="SEG_PRETRAIN",
               bps_halfwin="BPS_HALFWIN", block_samples="BLOCK_SAMPLES", in_scale="IN_SCALE",
               acq_min="ACQ_MIN", fo_smooth="FO_SMOOTH", rolloff="ROLLOFF", lam_nm="LAMBDA_NM")


def make_receiver(p: O.RxParams, **flags):
    """A CUDA receiver with exactly the oracle's parameters."""
    from paper_2104_06311_gb300 import Receiver
    rx = Receiver(p.baud, p.L_km, D=p.D, ntaps=p.ntaps, bps_angles=p.bps_angles)
    rx.set_param("MOD", p.bits)
    for k, key in _KEYMAP.items():
        rx.set_param(key, getattr(p, k))
    rx.set_param("FO_TRACK", 1 if p.fo_track else 0)
    for k, v in flags.items():
        rx.set_param(k, v)
    return rx


def inner_capacity(p: O.RxParams, K: int) -> int:
    """Entries per butterfly row of the device's inner-angle trace for a K-symbol stream."""
    n_acq = -(-(max(p.n_cma, p.acq_min) - p.n_cma) // p.upd_block)
    spb = -(-(p.seg_pretrain + p.seg_len) // p.upd_block)
    n_seg = -(-max(K - p.acq_len(K), 0) // p.seg_len) + 1
    return n_acq + n_seg * spb


def tracker_units(dw: float, Phi: float, p: O.RxParams) -> tuple[int, int]:
    """A reported (dw rad/symbol, Phi rad) pair as the tracker's integers (phi, d)."""
    M = 1 << O.chain.FO_GRID_BITS
    d = int(round(dw / (p.sps * 2 * math.pi) * M))
    phi = int(round(Phi / (2 * math.pi) * M)) % M
    return phi, d


def device_ties(rx, p: O.RxParams, K: int) -> dict:
    """The device's choices at the equaliser's discrete decisions: the tracker's
    integer state per wave (from rx_trace) and, when recorded, the inner BPS
    angle of every DD update block (rx_trace_inner).  The oracle takes one of
    them only where its own decision is a near-tie (both candidates correct)."""
    A = p.acq_len(K)
    S, P = p.seg_len, p.wave_segments()
    n_waves = -(-(-(-max(K - A, 0) // S)) // P)
    _, dw_acq, _ = rx.trace(-1)
    waves = [rx.trace(w) for w in range(n_waves)]
    out = dict(acq_units=tracker_units(dw_acq, 0.0, p)[1],
               wave_units=[tracker_units(w[1], w[2], p) for w in waves])
    if hasattr(rx, "trace_inner") and rx.get_param("INNER_TRACE") > 0:
        inner, n_acq, spb = rx.trace_inner()
        out.update(inner=inner, inner_acq=n_acq, inner_spb=spb)
    return out


def run_gpu(p: O.RxParams, samples: np.ndarray, chunk=None, reserve=None, **flags):
    import torch
    rx = make_receiver(p, LLR_OUT=1, SYM_OUT=1, EQ_OUT=1, CDC_OUT=1,
                       INNER_TRACE=inner_capacity(p, samples.shape[0] // 2), **flags)
    x = torch.from_numpy(np.ascontiguousarray(samples)).cuda()
    if reserve:
        rx.reserve(reserve)
    out = rx.run_stream(x, chunk=chunk, llr=True, sym=True, eq=True, cdc=True)
    torch.cuda.synchronize()
    K = out["n"]
    m = p.bits
    res = dict(
        n=K,
        cdc_n=out["cdc_n"],
        u=out["cdc"][:, :out["cdc_n"]].cpu().numpy().astype(np.complex128),
        y=out["eq"][:, :K].cpu().numpy().astype(np.complex128),
        z=out["sym"][:, :K].cpu().numpy().astype(np.complex128),
        llr=out["llr"][:, :K * m].cpu().numpy().astype(np.float64),
        words=out["bits"].cpu().numpy().view(np.uint32),
        bits_t=out["bits"],
    )
    res["bits"] = L.unpack_bits(res["words"], K * m)
    res["rx"] = rx
    return res


def boundary_mask(z: np.ndarray, mod: str, eps: float = BOUNDARY_EPS) -> np.ndarray:
    """Per-bit mask: True where the oracle's soft value is within eps of that bit's boundary."""
    if mod == "qpsk":
        m = np.stack([np.abs(z.real) < eps, np.abs(z.imag) < eps], axis=-1)
    else:
        s = math.sqrt(10.0)
        m = np.stack([np.abs(z.real) < eps, np.abs(np.abs(z.real) - 2 / s) < eps,
                      np.abs(z.imag) < eps, np.abs(np.abs(z.imag) - 2 / s) < eps], axis=-1)
    return m.reshape(z.shape[:-1] + (-1,))


def bps_near_tie(y: np.ndarray, p: O.RxParams, rel: float = BOUNDARY_EPS, chunk: int = 1 << 16) -> np.ndarray:
    """(2, K) True where the oracle's best and second-best BPS window sums differ by < rel."""
    B, Nb = p.bps_angles, p.bps_halfwin
    phis = O.bps_outer_angles(B)
    K = y.shape[-1]
    out = np.zeros((2, K), bool)
    for k0 in range(0, K, chunk):
        k1 = min(k0 + chunk, K)
        a, b = max(k0 - Nb, 0), min(k1 + Nb, K)
        w = y[:, a:b, None] * np.exp(-1j * phis)
        r = w - O.decide(w, p.mod)
        d = r.real ** 2 + r.imag ** 2
        c = np.concatenate([np.zeros((2, 1, B)), np.cumsum(d, axis=1)], axis=1)
        k = np.arange(k0, k1)
        hi = np.minimum(k + Nb + 1, K) - a
        lo = np.maximum(k - Nb, 0) - a
        D = c[:, hi] - c[:, lo]
        Ds = np.sort(D, axis=-1)
        out[:, k0:k1] = (Ds[..., 1] - Ds[..., 0]) < rel * np.maximum(Ds[..., 0], 1e-30)
    return out
