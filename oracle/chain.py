"""FP64 oracle of the receiver chain, step by step.  TEST INFRASTRUCTURE ONLY.

The paper (arXiv 2104.06311, Section "Experimental setup", the paragraph on the
real-time processing chain, and Fig. 1b) processes fixed-size sample buffers
through: conversion to floating point, FFT/IFFT pairs in overlap-save form, a
frequency-domain static equaliser, a sequential decision-directed LMS
equaliser, decisions and demapping; Q-factors come from BER counts (Section
"Results and Discussion", last paragraph).  The dual-polarisation chain here
is the coherent analogue of that chain:

  ingest -> CDC (overlap-save, dispersion + matched filter) -> 2x2 butterfly
  FIR adapted by CMA then DD-LMS, with frequency-offset removal in front of it
  -> blind phase search + unwrap -> hard bits / max-log LLR -> BER.

The paper defines only the overlap-save FFT filtering, the DD-LMS and the
demapping in words; every other step is paper-silent and follows the
textbook definitions stated in the docstrings below.  All arithmetic is FP64
(complex128).  numpy's FFT serves as the DFT primitive; everything else is
written out.  Nothing here is blocked, fused or reordered beyond evaluating
the stated per-element formulas over slices of the stream.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

C_LIGHT = 299_792_458.0
TWO_PI = 2.0 * math.pi


# ---------------------------------------------------------------------------
# Parameters
# ---------------------------------------------------------------------------
def n_cd_taps(baud: float, sps: int, L_km: float, D_ps_nm_km: float, lam_nm: float = 1550.0) -> int:
    """Dispersion memory in samples, N_CD = 2*floor(|D| lam^2 L / (2 c T^2)) + 1, T = 1/fs.

    Textbook bound (Savory, "Digital filters for coherent optical receivers",
    2008) for the length of a time-domain CD compensating filter.  The paper
    is silent on it; its introduction says only that the receiver's
    equalisation takes care of dispersion compensation digitally.
    """
    T = 1.0 / (sps * baud)
    D = abs(D_ps_nm_km) * 1e-12 / (1e-9 * 1e3)
    lam = lam_nm * 1e-9
    return 2 * int(math.floor(D * lam * lam * L_km * 1e3 / (2.0 * C_LIGHT * T * T))) + 1


def default_overlap(ncd: int) -> int:
    """Overlap V >= N_CD - 1 rounded up to a multiple of 32 (at least 32)."""
    return max(32, ((ncd - 1 + 31) // 32) * 32)


def default_fft_n(V: int) -> int:
    """Smallest power of two >= 4V, at least 1024 (the paper's FFT size) and at
    most 16384 (a configuration choice the paper does not make: beyond 4V the
    overlap-save overhead V/N only shrinks slowly, and 16384 is the largest
    transform the receiver library offers)."""
    n = 1024
    while n < 4 * V and n < 16384:
        n *= 2
    return n


@dataclasses.dataclass
class RxParams:
    baud: float = 10e9
    sps: int = 2
    L_km: float = 1000.0
    D: float = 17.0
    ntaps: int = 15
    bps_angles: int = 32
    mod: str = "qpsk"
    rolloff: float = 0.1
    lam_nm: float = 1550.0
    fft_n: int = 0          # 0: default_fft_n(overlap)
    overlap: int = 0        # 0: default_overlap(N_CD)
    mu_cma: float = 1e-3
    mu_dd: float = 1e-3
    n_cma: int = 8192
    upd_block: int = 32
    seg_len: int = 1024
    seg_pretrain: int = 128
    bps_halfwin: int = 16
    block_samples: int = 1 << 16
    in_scale: float = 1.0
    acq_min: int = 1 << 14
    fo_smooth: float = 16.0
    fo_track: bool = True   # False: no frequency-offset estimation or removal

    def resolved(self) -> "RxParams":
        p = dataclasses.replace(self)
        if p.overlap == 0:
            p.overlap = default_overlap(n_cd_taps(p.baud, p.sps, p.L_km, p.D, p.lam_nm))
        if p.fft_n == 0:
            p.fft_n = default_fft_n(p.overlap)
        return p

    @property
    def bits(self) -> int:
        return {"qpsk": 2, "16qam": 4}[self.mod]

    @property
    def cma_radius(self) -> float:
        """R2 = E|s|^4 / E|s|^2 of the unit-energy constellation."""
        return {"qpsk": 1.0, "16qam": 1.32}[self.mod]

    def acq_len(self, K: int) -> int:
        return min(max(self.n_cma, self.acq_min), K)

    def wave_segments(self) -> int:
        return max(1, (self.block_samples // self.sps) // self.seg_len)


# ---------------------------------------------------------------------------
# CDC: overlap-save dispersion compensation with the matched filter fused
# ---------------------------------------------------------------------------
def _grid(p: RxParams, N: int) -> np.ndarray:
    fs = p.sps * p.baud
    k = np.arange(N)
    return np.where(k < N // 2, k, k - N) * (fs / N)


def cd_response(p: RxParams, N: int) -> np.ndarray:
    """Dispersion compensation exp(-j beta2 L w_k^2 / 2), beta2 = -D lam^2/(2 pi c).

    The inverse of the fibre's exp(+j beta2 L w^2/2) (paper-silent: the paper's
    introduction only says its equalisation compensates dispersion digitally).
    Bin k sits at f_k = k fs/N for k < N/2, (k-N) fs/N else.
    """
    w = TWO_PI * _grid(p, N)
    D = p.D * 1e-12 / (1e-9 * 1e3)
    lam = p.lam_nm * 1e-9
    beta2 = -D * lam * lam / (TWO_PI * C_LIGHT)
    return np.exp(-1j * beta2 * (p.L_km * 1e3) * w * w / 2.0)


def rrc_response(p: RxParams, N: int) -> np.ndarray:
    """Root-raised-cosine amplitude: 1 for |f| <= (1-r)R/2,
    cos(pi(|f| - (1-r)R/2) / (2rR)) up to (1+r)R/2, 0 beyond."""
    af = np.abs(_grid(p, N))
    f1 = (1.0 - p.rolloff) * p.baud / 2.0
    f2 = (1.0 + p.rolloff) * p.baud / 2.0
    rrc = np.where(af <= f1, 1.0, 0.0)
    band = (af > f1) & (af <= f2)
    rrc[band] = np.cos(math.pi * (af[band] - f1) / (2.0 * p.rolloff * p.baud))
    return rrc


def cdc_filter(p: RxParams, N: int | None = None) -> np.ndarray:
    """H_k = H_CD(w_k) * sqrt(sps) * H_rrc(f_k) on the N-point grid (default fft_n).

    The paper equalises statically in the frequency domain by multiplying with
    an offline-optimised filter through an FFT/IFFT pair (Section
    "Experimental setup", processing-chain paragraph).  Here that filter is
    the closed-form dispersion inverse times the RRC matched filter.
    """
    p = p.resolved()
    N = p.fft_n if N is None else N
    return cd_response(p, N) * math.sqrt(p.sps) * rrc_response(p, N)


def cdc_overlap_save(x: np.ndarray, H: np.ndarray, V: int) -> np.ndarray:
    """Overlap-save filtering of each row of x (complex, zero outside [0, n)).

    Hop S = N - V.  Window i holds x[iS - V/2 .. iS - V/2 + N - 1]; output
    samples n in [iS, iS+S) are element V/2 + (n - iS) of IDFT(DFT(window)*H).
    With a filter whose impulse response lies in [-V/2, V/2] this is exactly
    linear convolution with a centred filter (zero delay).  The paper's chain
    uses FFT/IFFT pairs in this overlap-save form (processing-chain paragraph).
    """
    N = H.shape[-1]
    S = N - V
    h = V // 2
    n = x.shape[-1]
    out = np.zeros(x.shape, np.complex128)
    for i in range((n + S - 1) // S):
        lo = i * S - h
        win = np.zeros(x.shape[:-1] + (N,), np.complex128)
        a, b = max(lo, 0), min(lo + N, n)
        win[..., a - lo:b - lo] = x[..., a:b]
        yw = np.fft.ifft(np.fft.fft(win, axis=-1) * H, axis=-1)
        e = min(i * S + S, n)
        out[..., i * S:e] = yw[..., h:h + e - i * S]
    return out


# ---------------------------------------------------------------------------
# Decisions, bits and LLRs (square Gray QAM)
# ---------------------------------------------------------------------------
def _levels(x: np.ndarray, mod: str) -> np.ndarray:
    """Nearest constellation level per real dimension (x >= 0 rounds to +)."""
    if mod == "qpsk":
        return np.where(x >= 0.0, 1.0, -1.0) / math.sqrt(2.0)
    s = x * math.sqrt(10.0)
    lv = np.where(s >= 0.0, np.where(s > 2.0, 3.0, 1.0), np.where(s < -2.0, -3.0, -1.0))
    return lv / math.sqrt(10.0)


def decide(z: np.ndarray, mod: str) -> np.ndarray:
    """Nearest point of the unit-energy square QAM constellation."""
    return _levels(z.real, mod) + 1j * _levels(z.imag, mod)


def hard_bits(z: np.ndarray, mod: str) -> np.ndarray:
    """Gray bits of the nearest point, shape (..., K*m).

    QPSK: b0 = [Re z < 0], b1 = [Im z < 0].  16QAM per dimension x (scaled by
    sqrt10): first bit [x < 0], second bit [|x| > 2]; I bits then Q bits.
    The paper demaps the equaliser's decisions (processing-chain paragraph).
    """
    if mod == "qpsk":
        b = np.stack([z.real < 0, z.imag < 0], axis=-1)
    else:
        si, sq = z.real * math.sqrt(10.0), z.imag * math.sqrt(10.0)
        b = np.stack([si < 0, np.abs(si) > 2.0, sq < 0, np.abs(sq) > 2.0], axis=-1)
    return b.reshape(z.shape[:-1] + (-1,)).astype(np.uint8)


def llr_maxlog(z: np.ndarray, sigma2: np.ndarray, mod: str) -> np.ndarray:
    """Max-log LLR = log P(b=0)/P(b=1) ~ (min_{s:b=1}|z-s|^2 - min_{s:b=0}|z-s|^2) / sigma2.

    Paper-silent (the paper outputs hard decisions only).  For square Gray QAM
    the minimum separates per dimension, so each bit's LLR comes from the
    one-dimensional levels it labels.  sigma2 has the shape of z.
    """
    if mod == "qpsk":
        lv = np.array([1.0, -1.0]) / math.sqrt(2.0)          # level of bit value 0 / 1
        out = []
        for x in (z.real, z.imag):
            d0 = (x - lv[0]) ** 2
            d1 = (x - lv[1]) ** 2
            out.append((d1 - d0) / sigma2)
        return np.stack(out, axis=-1).reshape(z.shape[:-1] + (-1,))
    lv = np.array([-3.0, -1.0, 1.0, 3.0]) / math.sqrt(10.0)
    # bits of each level: first bit [level < 0], second bit [|level| > 2]
    first = np.array([1, 1, 0, 0])
    second = np.array([1, 0, 0, 1])
    out = []
    for x in (z.real, z.imag):
        d = (x[..., None] - lv) ** 2
        for lab in (first, second):
            d0 = np.min(np.where(lab == 0, d, np.inf), axis=-1)
            d1 = np.min(np.where(lab == 1, d, np.inf), axis=-1)
            out.append((d1 - d0) / sigma2)
    return np.stack(out, axis=-1).reshape(z.shape[:-1] + (-1,))


# ---------------------------------------------------------------------------
# Frequency offset: differential 4th-power estimator (paper-silent)
# ---------------------------------------------------------------------------
def ring_weight(a: np.ndarray) -> np.ndarray:
    """Weight of a 16QAM symbol with power a = |y|^2 in the frequency estimate.

    Unit-energy 16QAM has rings at |s|^2 = 0.2, 1.0 and 1.8.  The inner and
    outer rings sit at odd multiples of pi/4 (their 4th power is -|s|^4, as for
    QPSK); the middle ring's 4th power is not aligned with them and only adds
    self-noise (QPSK partitioning: Fatadin, Ives, Savory, IEEE PTL 2010).  The
    weight is 0 for |a - 1| <= 0.2, 1 for |a - 1| >= 0.4 and linear between:
    a soft edge, so that the estimate is continuous in the samples.
    """
    return np.clip((np.abs(a - 1.0) - 0.2) / 0.2, 0.0, 1.0)


def fo_estimate_sum(y: np.ndarray, mod: str = "qpsk") -> complex:
    """sum over pols and adjacent pairs of w_k w_{k-1} (y_k conj(y_{k-1}))^4.

    A quarter of its argument estimates the per-symbol frequency offset (the
    4th power removes the pi/2-symmetric data).  QPSK: w = 1.  16QAM: w =
    ring_weight(|y|^2), which keeps the pi/4-aligned inner and outer rings.
    The paper's KK receiver instead downshifts a known carrier tone to DC
    (processing-chain paragraph); the estimator is the textbook one for
    coherent detection with a free-running local oscillator.
    """
    if y.shape[-1] < 2:
        return 0j
    v = y[..., 1:] * np.conj(y[..., :-1])
    v4 = v ** 4
    if mod == "16qam":
        w = ring_weight(y.real ** 2 + y.imag ** 2)
        v4 = v4 * (w[..., 1:] * w[..., :-1])
    return complex(np.sum(v4))


# ---------------------------------------------------------------------------
# 2x2 butterfly FIR with block CMA -> DD-LMS, segment schedule
# ---------------------------------------------------------------------------
def bps_outer_angles(B: int) -> np.ndarray:
    """Test angles phi_b = (b/B - 1/2) * pi/2, b = 0..B-1."""
    return (np.arange(B) / B - 0.5) * (math.pi / 2.0)


def _bps_distance(y: np.ndarray, phis: np.ndarray, mod: str) -> np.ndarray:
    """d[..., b] = |y e^{-j phi_b} - dec(y e^{-j phi_b})|^2."""
    w = y[..., None] * np.exp(-1j * phis)
    r = w - decide(w, mod)
    return r.real ** 2 + r.imag ** 2


FO_GRID_BITS = 16


def fo_units(rate: float, sps: int) -> tuple[int, float]:
    """A rate in rad/symbol as the nearest whole number of 2^-G turns per sample.

    G = FO_GRID_BITS.  Returns (units, edge): `edge` is the distance of the
    unrounded value from the nearest rounding boundary, in units (0.5 at a grid
    point, 0 exactly half-way between two).  The paper has no frequency
    tracker; this grid is a reading of the textbook estimator: every quantity
    the tracker integrates is a whole multiple of 2^-G turns, so that the phase
    it accumulates over a stream is exact (no rounding to compound from wave
    to wave) and any implementation that rounds the same estimates to the same
    grid tracks the same phase.  2^-16 turns per sample is 1.9e-4 rad per
    symbol at 2 samples per symbol (305 kHz at 10 GBd): a residual offset of
    half of that turns a symbol by < 1e-4 rad, and moves the phase by 3e-3
    rad over a 33-symbol BPS window, well inside what the phase search
    tracks, while the per-wave estimates it rounds scatter by ~3e-3 rad per
    symbol.  Ties round to even.
    """
    x = rate / (sps * TWO_PI) * float(1 << FO_GRID_BITS)
    u = int(np.rint(x))
    return u, abs(abs(x - math.floor(x)) - 0.5)


def units_to_rate(u: int, sps: int) -> float:
    """Whole 2^-G turns per sample -> rad/symbol."""
    return u * sps * TWO_PI / float(1 << FO_GRID_BITS)


def units_to_phase(phi: int) -> float:
    """A phase of phi 2^-G turns (taken mod 2^G) -> radians in [-pi, pi)."""
    M = 1 << FO_GRID_BITS
    phi %= M
    if phi >= M // 2:
        phi -= M
    return phi * TWO_PI / float(M)


class _Window:
    """Rotated FIR input for symbols [k_lo, k_hi): samples 2k_lo-c .. 2(k_hi-1)+c.

    Rotation (frequency-offset removal in front of the FIR) by
    exp(-j 2 pi t_n / 2^G), t_n = (phi + (n - n0) d) mod 2^G: phase base phi
    and per-sample increment d are whole 2^-G turns (fo_units), so t_n is an
    exact integer.  d=None means no rotation.
    """

    def __init__(self, u: np.ndarray, k_lo: int, k_hi: int, c: int,
                 phi: int = 0, n0: int = 0, d: int | None = None):
        n = u.shape[-1]
        self.lo = 2 * k_lo - c
        hi = 2 * (k_hi - 1) + c + 1
        idx = np.arange(self.lo, hi)
        ok = (idx >= 0) & (idx < n)
        seg = np.zeros((2, hi - self.lo), np.complex128)
        seg[:, ok] = u[:, idx[ok]]
        if d is not None:
            M = 1 << FO_GRID_BITS
            t = np.mod(phi + (idx.astype(np.int64) - n0) * d, M)
            seg = seg * np.exp(-1j * (TWO_PI / M) * t.astype(np.float64))[None, :]
        self.seg = seg

    def taps_input(self, k0: int, k1: int, T: int, c: int) -> np.ndarray:
        """X[k, q, i] = u_q[2k + c - i] for k in [k0, k1)."""
        k = np.arange(k0, k1)
        i = np.arange(T)
        idx = (2 * k[:, None] + c - i[None, :]) - self.lo
        return np.transpose(self.seg[:, idx], (1, 0, 2))


# Decisions where two candidates are equally correct to within rounding: the
# inner BPS argmin when the runner-up's block sum is within INNER_TIE_REL of the
# minimum (an FP32 sum of 32 order-one terms is exact to ~1e-6 of such a sum),
# and a tracker rounding when the unrounded value lies within TRACK_TIE_UNITS of
# the half-way point between two grid values.  At such a decision another
# implementation's choice is as valid as this one's; `equalize` can take it
# (passed in `ties`) and logs every decision it took that way.
INNER_TIE_REL = 1e-4
TRACK_TIE_UNITS = 2e-3


def lms_step(h: np.ndarray, X: np.ndarray, mode: str, p: RxParams, phis: np.ndarray,
             choice=None, log: list | None = None, where=None):
    """One block update of the butterfly; returns (y (2,nk), new h).

    y_p[k] = sum_{q,i} h_pq[i] u_q[2k+c-i].
    CMA error e = y(|y|^2 - R2) (Godard's constant-modulus criterion).
    DD error e = y - d e^{j theta}, d = dec(y e^{-j theta}), theta = the test
    angle minimising the summed BPS distance over this block (the inner phase;
    smallest index on exact ties).
    Update h_pq[i] -= mu * sum_k e_p[k] conj(u_q[2k+c-i]) (a block sum).
    The paper's equaliser is a decision-directed LMS adapted in time domain
    (processing-chain paragraph); CMA and the butterfly are paper-silent.

    choice: optional per-row angle indices another implementation took for
    this block (negative = none); row p takes choice[p] instead of its own
    argmin only where choice[p]'s block sum is within INNER_TIE_REL of the
    minimum, and appends (where, p, own, taken, relative gap) to `log`.
    """
    y = np.einsum("pqi,kqi->pk", h, X)
    if mode == "cma":
        e = y * (np.abs(y) ** 2 - p.cma_radius)
        mu = p.mu_cma
    else:
        d = _bps_distance(y, phis, p.mod)                 # (2, nk, B)
        D = np.sum(d, axis=1)                             # (2, B)
        b = np.argmin(D, axis=-1)                         # first minimum per pol
        if choice is not None:
            for pp in range(2):
                c = int(choice[pp])
                if 0 <= c < len(phis) and c != b[pp]:
                    gap = (D[pp, c] - D[pp, b[pp]]) / max(D[pp, b[pp]], 1e-300)
                    if gap < INNER_TIE_REL:
                        if log is not None:
                            log.append(("inner", where, pp, int(b[pp]), c, float(gap)))
                        b[pp] = c
        th = phis[b][:, None]
        rot = np.exp(1j * th)
        e = y - decide(y * np.conj(rot), p.mod) * rot
        mu = p.mu_dd
    g = np.einsum("pk,kqi->pqi", e, np.conj(X))
    return y, h - mu * g


def _track_tie(own: int, edge: float, other, kind: str, where, log: list) -> int:
    """The tracker rounding to use: `other` (another implementation's rounding
    of the same quantity) where this one's value lies within TRACK_TIE_UNITS of
    the half-way point and `other` is the neighbouring grid value, else own."""
    if other is not None and other != own and abs(other - own) == 1 and edge < TRACK_TIE_UNITS:
        log.append((kind, where, own, int(other), float(edge)))
        return int(other)
    return own


def equalize(u: np.ndarray, p: RxParams, trace: dict | None = None, ties: dict | None = None) -> np.ndarray:
    """Butterfly equaliser over the whole stream with the segment schedule.

    u: (2, n) CDC output at 2 samples/symbol; returns y (2, K), K = n // 2.

    Schedule (paper-silent; the paper chains a sequential DD-LMS across
    buffers with CUDA events, processing-chain paragraph):
      * Acquisition: symbols [0, A), A = min(max(N_CMA, 2^14), K), one chain
        of update blocks of B_u symbols.  CMA (no rotation) on [0, N_CMA');
        the frequency offset is then estimated from the CMA outputs in
        [N_CMA'/2, N_CMA') and rounded to the tracker grid, d_0 = fo_units(dw),
        and DD-LMS runs on [N_CMA', A) with sample n rotated by
        exp(-j 2 pi (n - 2 N_CMA') d_0 / 2^G).
      * Waves: symbols [A, K) in segments of S; wave w holds P segments.
        Every segment of wave w starts from the taps at the end of the last
        segment of wave w-1 (the acquisition for w = 0), pre-trains on the W
        symbols before it (DD, outputs discarded), then equalises its own
        symbols.  Its input is rotated by exp(-j 2 pi (phi_w + (n - n_w) d_w)
        / 2^G), n_w = 2 (A + w P S).
      * Frequency tracking per wave, applied two waves on: r_w is a quarter
        of the argument of fo_estimate_sum over adjacent pairs inside each
        segment of wave w; i_w = fo_units(r_w / fo_smooth); d_1 = d_0 and
        d_{w+1} = d_w + i_{w-1}; phi_0 = (2A - 2 N_CMA') d_0,
        phi_{w+1} = phi_w + 2PS d_w, all mod 2^G.  (Wave w+1's rotation is
        then fixed before wave w ends: only its start taps wait for wave w.)

    The tracker's state (phi, d) is integer (fo_units): the phase it
    integrates over the stream is exact, so implementations that round the
    same estimates to the same grid follow the same phase for the whole
    stream.  `trace` records the state at every wave start (taps, dw in
    rad/symbol, Phi in rad, and the integers), the estimates, each rounding's
    distance from its rounding boundary (fo_edge) and the tie log.

    ties: optional choices of another implementation at the chain's discrete
    decisions -- 'acq_units' (d_0), 'wave_units' ((phi_w, d_w) per wave),
    'inner' ([2][n] inner BPS angle per DD update block: the acquisition's
    'inner_acq' blocks, then 'inner_spb' per segment counted from its first
    pre-training block).  Each is taken only at a near-tie (INNER_TIE_REL,
    TRACK_TIE_UNITS); every decision taken that way is logged in
    trace['ties'].  Without `ties` the schedule runs on its own decisions only.
    """
    p = p.resolved()
    n = u.shape[-1]
    K = n // 2
    T = p.ntaps
    c = (T - 1) // 2
    Bu = p.upd_block
    M = 1 << FO_GRID_BITS
    phis = bps_outer_angles(p.bps_angles)
    y = np.zeros((2, K), np.complex128)
    h = np.zeros((2, 2, T), np.complex128)
    h[0, 0, c] = 1.0
    h[1, 1, c] = 1.0
    A = p.acq_len(K)
    tie_log: list = []
    if trace is not None:
        trace["ties"] = tie_log
    if K == 0:
        return y
    ties = ties or {}
    inner = ties.get("inner")
    n_acq_blk = int(ties.get("inner_acq", 0))
    spb = int(ties.get("inner_spb", 0))

    def inner_choice(j):
        if inner is None or j < 0 or j >= inner.shape[1]:
            return None
        return inner[:, j]

    n_cma = min(p.n_cma, A)
    rot = None if not p.fo_track else 0    # None: no rotation
    # -- acquisition, CMA part
    win = _Window(u, 0, n_cma, c)
    for k0 in range(0, n_cma, Bu):
        k1 = min(k0 + Bu, n_cma)
        y[:, k0:k1], h = lms_step(h, win.taps_input(k0, k1, T, c), "cma", p, phis)
    dw_est = 0.25 * np.angle(fo_estimate_sum(y[:, n_cma // 2:n_cma], p.mod)) if p.fo_track else 0.0
    d, edge = fo_units(dw_est, p.sps)
    edges = [edge] if p.fo_track else []
    d = _track_tie(d, edge, ties.get("acq_units"), "acq", 0, tie_log)
    # -- acquisition, DD part
    if A > n_cma:
        win = _Window(u, n_cma, A, c, 0, 2 * n_cma, d if rot is not None else None)
        for t, k0 in enumerate(range(n_cma, A, Bu)):
            k1 = min(k0 + Bu, A)
            y[:, k0:k1], h = lms_step(h, win.taps_input(k0, k1, T, c), "dd", p, phis,
                                      inner_choice(t) if t < n_acq_blk else None, tie_log, ("acq", t))
    phi = ((2 * A - 2 * n_cma) * d) % M
    if trace is not None:
        trace.update(acq_dw=units_to_rate(d, p.sps), acq_dw_est=dw_est, acq_units=d, acq_taps=h.copy(),
                     wave_taps=[], wave_dw=[], wave_Phi=[], wave_units=[], wave_r=[], fo_edge=edges)
    dev_waves = ties.get("wave_units")
    # -- waves
    S, W, P = p.seg_len, p.seg_pretrain, p.wave_segments()
    G = (K - A + S - 1) // S
    h_start = h
    inc_prev = 0          # i_{w-1}: the previous wave's increment, applied after this wave
    for w0 in range(0, G, P):
        gs = range(w0, min(w0 + P, G))
        n_w = 2 * (A + w0 * S)
        if trace is not None:
            trace["wave_taps"].append(h_start.copy())
            trace["wave_dw"].append(units_to_rate(d, p.sps))
            trace["wave_Phi"].append(units_to_phase(phi))
            trace["wave_units"].append((phi, d))
        acc = 0j
        h_last = h_start
        for g in gs:
            ks, ke = A + g * S, min(A + (g + 1) * S, K)
            kp = max(ks - W, 0)
            win = _Window(u, kp, ke, c, phi, n_w, d if rot is not None else None)
            hh = h_start
            base = n_acq_blk + g * spb
            t = 0
            for k0 in range(kp, ks, Bu):
                _, hh = lms_step(hh, win.taps_input(k0, min(k0 + Bu, ks), T, c), "dd", p, phis,
                                 inner_choice(base + t) if t < spb else None, tie_log, ("seg", g, t))
                t += 1
            for k0 in range(ks, ke, Bu):
                k1 = min(k0 + Bu, ke)
                y[:, k0:k1], hh = lms_step(hh, win.taps_input(k0, k1, T, c), "dd", p, phis,
                                           inner_choice(base + t) if t < spb else None, tie_log, ("seg", g, t))
                t += 1
            acc += fo_estimate_sum(y[:, ks:ke], p.mod)
            h_last = hh
        r = 0.25 * np.angle(acc) if p.fo_track else 0.0
        inc, edge = fo_units(r / p.fo_smooth, p.sps)
        if p.fo_track:
            edges.append(edge)
            wi = w0 // P
            # the other implementation applies i_w from wave w+2 on
            if dev_waves is not None and wi + 2 < len(dev_waves):
                inc = _track_tie(inc, edge, dev_waves[wi + 2][1] - dev_waves[wi + 1][1], "wave", wi, tie_log)
        if trace is not None:
            trace["wave_r"].append(r)
        phi = (phi + (2 * P * S) * d) % M
        d = d + inc_prev
        inc_prev = inc
        h_start = h_last
    return y


# ---------------------------------------------------------------------------
# Blind phase search with integer unwrap (paper-silent)
# ---------------------------------------------------------------------------
def bps_outer(y: np.ndarray, p: RxParams, chunk: int = 1 << 15):
    """Blind phase search per polarisation (Pfau, Hoffmann, Noe, JLT 2009).

    d_{k,b} = |y_k e^{-j phi_b} - dec(.)|^2, D_{k,b} = sum_{m=-Nb..Nb} d_{k+m,b}
    (terms outside [0, K) omitted), bhat_k = argmin_b D (smallest b on ties).
    Unwrap: r_k = +1 if bhat_{k-1} - bhat_k > B/2, -1 if < -B/2, else 0;
    m_k = m_{k-1} + r_k (m_0 = 0); theta_k = phi_bhat + m_k pi/2;
    z_k = y_k e^{-j theta_k}.  Returns (bhat (2,K) int, m (2,K) int, z (2,K)).
    The slices of `chunk` symbols (with an Nb halo) only bound memory.
    """
    p = p.resolved()
    B, Nb = p.bps_angles, p.bps_halfwin
    phis = bps_outer_angles(B)
    K = y.shape[-1]
    bhat = np.zeros((2, K), np.int64)
    for k0 in range(0, K, chunk):
        k1 = min(k0 + chunk, K)
        a, b = max(k0 - Nb, 0), min(k1 + Nb, K)
        d = _bps_distance(y[:, a:b], phis, p.mod)       # (2, b-a, B)
        Dsum = np.zeros((2, k1 - k0, B))
        for m in range(-Nb, Nb + 1):
            lo, hi = k0 + m, k1 + m                      # indices into the stream
            s_lo, s_hi = max(lo, 0), min(hi, K)
            if s_hi <= s_lo:
                continue
            Dsum[:, s_lo - lo:s_hi - lo] += d[:, s_lo - a:s_hi - a]
        bhat[:, k0:k1] = np.argmin(Dsum, axis=-1)
    r = np.zeros((2, K), np.int64)
    diff = bhat[:, :-1] - bhat[:, 1:]
    r[:, 1:] = np.where(diff > B / 2, 1, np.where(diff < -B / 2, -1, 0))
    m = np.cumsum(r, axis=1)
    theta = phis[bhat] + m * (math.pi / 2.0)
    z = y * np.exp(-1j * theta)
    return bhat, m, z


def region_bounds(K: int, p: RxParams) -> list[tuple[int, int]]:
    """LLR noise-variance regions: the acquisition, then each wave."""
    p = p.resolved()
    A = p.acq_len(K)
    out = [(0, A)] if A > 0 else []
    span = p.wave_segments() * p.seg_len
    for s in range(A, K, span):
        out.append((s, min(s + span, K)))
    return out


def demap(z: np.ndarray, p: RxParams):
    """Hard bits and max-log LLRs; sigma2 per region per pol = mean |z - dec(z)|^2.

    The paper demaps the equaliser decisions and sends them to host RAM
    (processing-chain paragraph).  Returns (bits (2, K*m) uint8,
    llr (2, K*m), sigma2 (2, n_regions)).
    """
    p = p.resolved()
    K = z.shape[-1]
    bits = hard_bits(z, p.mod)
    regs = region_bounds(K, p)
    err = np.abs(z - decide(z, p.mod)) ** 2
    sig = np.zeros((2, len(regs)))
    s2 = np.zeros((2, K))
    for j, (a, b) in enumerate(regs):
        sig[:, j] = np.mean(err[:, a:b], axis=1)
        s2[:, a:b] = sig[:, j:j + 1]
    llr = llr_maxlog(z, s2, p.mod)
    return bits, llr, sig


def run_chain(samples: np.ndarray, p: RxParams, trace: dict | None = None, ties: dict | None = None) -> dict:
    """Whole stream: ingest -> CDC -> equaliser -> BPS -> demap.

    samples: (n, 4) real [Xi, Xq, Yi, Yq] (int8 codes or floats); the ingest
    multiplies by p.in_scale (the paper's first step converts ADC samples to
    floating point, processing-chain paragraph).
    """
    p = p.resolved()
    a = np.asarray(samples, dtype=np.float64) * p.in_scale
    n = a.shape[0] - (a.shape[0] % 2)
    x = np.stack([a[:n, 0] + 1j * a[:n, 1], a[:n, 2] + 1j * a[:n, 3]])
    u = cdc_overlap_save(x, cdc_filter(p), p.overlap)
    y = equalize(u, p, trace, ties)
    bhat, m, z = bps_outer(y, p)
    bits, llr, sig = demap(z, p)
    return dict(u=u, y=y, bhat=bhat, m=m, z=z, bits=bits, llr=llr, sigma2=sig)


# ---------------------------------------------------------------------------
# BER with rotation / polarisation / delay synchronisation, Q factor
# ---------------------------------------------------------------------------
def _rotate_bits(bits: np.ndarray, rot: int, mod: str) -> np.ndarray:
    """Bits of j^rot * s for the symbols s labelled by `bits` (..., K*m)."""
    m = 2 if mod == "qpsk" else 4
    b = bits.reshape(bits.shape[:-1] + (-1, m)).astype(np.int64)
    if mod == "qpsk":
        i, q = 1 - 2 * b[..., 0], 1 - 2 * b[..., 1]
    else:
        i = (1 - 2 * b[..., 0]) * (1 + 2 * b[..., 1])
        q = (1 - 2 * b[..., 2]) * (1 + 2 * b[..., 3])
    for _ in range(rot % 4):
        i, q = -q, i                                   # multiply by j
    z = (i + 1j * q) / (math.sqrt(2.0) if mod == "qpsk" else math.sqrt(10.0))
    return hard_bits(z, mod)


def ber_sync_count(rx_bits: np.ndarray, ref_bits: np.ndarray, mod: str, A: int,
                   sync_len: int = 1 << 12, max_delay: int = 64):
    """Bit errors after synchronisation.  rx_bits, ref_bits: (2, K*m) 0/1.

    Skip symbols [0, A + sync_len); on [A + sync_len, A + 2 sync_len) choose
    per received pol p the (reference pol q, rotation r in 0..3, delay d in
    [-Dmax, Dmax]) with the fewest bit errors against bits(j^r ref_q[k + d])
    (first in (q, r, d) order on ties); then count errors on
    k in [A + 2 sync_len, K) with 0 <= k + d < K.  The paper estimates Q from
    BER counts (Section "Results and Discussion").
    Returns (errors, bits_counted, sync list of (q, r, d)).
    """
    m = 2 if mod == "qpsk" else 4
    K = rx_bits.shape[-1] // m
    rxs = rx_bits.reshape(2, K, m)
    refr = [_rotate_bits(ref_bits, r, mod).reshape(2, K, m) for r in range(4)]
    s0, s1 = A + sync_len, A + 2 * sync_len
    if s1 > K:
        return 0, 0, []
    errors = counted = 0
    sync = []
    for pp in range(2):
        best = None
        for q in range(2):
            for r in range(4):
                for d in range(-max_delay, max_delay + 1):
                    k = np.arange(s0, s1)
                    kk = k + d
                    ok = (kk >= 0) & (kk < K)
                    e = int(np.sum(rxs[pp, k[ok]] != refr[r][q, kk[ok]]))
                    if best is None or e < best[0]:
                        best = (e, q, r, d)
        _, q, r, d = best
        sync.append((q, r, d))
        k = np.arange(s1, K)
        kk = k + d
        ok = (kk >= 0) & (kk < K)
        errors += int(np.sum(rxs[pp, k[ok]] != refr[r][q, kk[ok]]))
        counted += int(np.sum(ok)) * m
    return errors, counted, sync


def q_from_ber(ber: float) -> float:
    """Q [dB] = 20 log10(sqrt2 * erfcinv(2 BER))."""
    from scipy.special import erfcinv
    return 20.0 * math.log10(math.sqrt(2.0) * float(erfcinv(2.0 * ber)))


def ber_theory(mod: str, snr_db: float) -> float:
    """Gray-coded BER in AWGN at Es/N0 = SNR (textbook closed forms).

    QPSK: Q(sqrt(SNR)).  16QAM: (3Q(a) + 2Q(3a) - Q(5a))/4, a = sqrt(SNR/5).
    """
    from scipy.special import erfc

    def Q(x):
        return 0.5 * erfc(x / math.sqrt(2.0))

    s = 10.0 ** (snr_db / 10.0)
    if mod == "qpsk":
        return float(Q(math.sqrt(s)))
    a = math.sqrt(s / 5.0)
    return float((3 * Q(a) + 2 * Q(3 * a) - Q(5 * a)) / 4.0)
