"""Seeded synthetic dual-polarisation coherent link (input generator).

This module is test and benchmark infrastructure. It builds the sampled
field a coherent receiver sees after a long-haul fibre link, at 2 samples per
symbol, so that both the FP64 oracle and the CUDA receiver can be fed the
same seeded input.  It holds none of the receiver's arithmetic: it only
creates bits, maps them to QAM symbols, shapes them, and applies the channel
impairments (chromatic dispersion, a Jones rotation, PMD waveplates, laser
phase noise, a frequency offset, AWGN and an 8-bit ADC).

The experiment the paper reports (Section "Experimental setup") ran on a real
100-span link; that link is not available here, so these synthetic links
stand in for it with the parameters of the receiver's workloads.

Conventions (shared with the receiver only through these documented facts):
  * DFT grid: bin k of an n-point grid sits at f_k = k*fs/n for k < n/2 and
    (k-n)*fs/n otherwise.
  * Channel dispersion transfer function exp(+j*beta2*L*w^2/2) with
    beta2 = -D*lambda^2/(2*pi*c).
  * One sample-time holds Xi, Xq, Yi, Yq (interleaved, 4 scalars).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np
import scipy.fft as sfft

C_LIGHT = 299_792_458.0

# ---------------------------------------------------------------------------
# Bits: SplitMix64 (S. Vigna's public-domain generator, "splitmix64.c").
# state advances by the golden-ratio increment; each output is the state
# passed through two xor-shift-multiply rounds and a final xor-shift.
# ---------------------------------------------------------------------------
_SM64_INC = np.uint64(0x9E3779B97F4A7C15)
_SM64_M1 = np.uint64(0xBF58476D1CE4E5B9)
_SM64_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, n: int) -> np.ndarray:
    """First n outputs of SplitMix64 started from state `seed` (uint64)."""
    with np.errstate(over="ignore"):
        k = np.arange(1, n + 1, dtype=np.uint64)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + k * _SM64_INC
        z = (z ^ (z >> np.uint64(30))) * _SM64_M1
        z = (z ^ (z >> np.uint64(27))) * _SM64_M2
        z = z ^ (z >> np.uint64(31))
    return z


def random_bits(seed: int, nbits: int) -> np.ndarray:
    """nbits uniform bits (uint8 0/1), LSB-first from successive SplitMix64 words."""
    nwords = (nbits + 63) // 64
    words = splitmix64(seed, nwords).astype("<u8")
    return np.unpackbits(words.view(np.uint8), bitorder="little")[:nbits].copy()


def pack_bits(bits: np.ndarray) -> np.ndarray:
    """Pack a 0/1 array (last axis) into little-endian uint32 words, LSB-first."""
    bits = np.asarray(bits, dtype=np.uint8)
    n = bits.shape[-1]
    pad = (-n) % 32
    if pad:
        bits = np.concatenate([bits, np.zeros(bits.shape[:-1] + (pad,), np.uint8)], axis=-1)
    by = np.packbits(bits, axis=-1, bitorder="little")
    return by.view("<u4").copy()


def unpack_bits(words: np.ndarray, nbits: int) -> np.ndarray:
    w = np.ascontiguousarray(words).astype("<u4")
    return np.unpackbits(w.view(np.uint8), axis=-1, bitorder="little")[..., :nbits]


def bits_per_symbol(mod: str) -> int:
    return {"qpsk": 2, "16qam": 4}[mod]


def map_symbols(bits: np.ndarray, mod: str) -> np.ndarray:
    """Gray QPSK / 16QAM with unit mean energy.

    bits: (..., K*m) 0/1.  QPSK symbol bits (b0, b1) -> ((1-2b0) + j(1-2b1))/sqrt2.
    16QAM bits (b0, b1, b2, b3) -> I=(1-2b0)(1+2b1), Q=(1-2b2)(1+2b3), /sqrt10,
    i.e. per dimension levels -3,-1,+1,+3 carry bit pairs 11,10,00,01.
    """
    m = bits_per_symbol(mod)
    b = np.asarray(bits, dtype=np.int64).reshape(bits.shape[:-1] + (-1, m))
    if mod == "qpsk":
        return ((1 - 2 * b[..., 0]) + 1j * (1 - 2 * b[..., 1])) / math.sqrt(2.0)
    i = (1 - 2 * b[..., 0]) * (1 + 2 * b[..., 1])
    q = (1 - 2 * b[..., 2]) * (1 + 2 * b[..., 3])
    return (i + 1j * q) / math.sqrt(10.0)


# ---------------------------------------------------------------------------
# Waveform pieces (whole-stream DFT filtering in FP64).
# ---------------------------------------------------------------------------
def grid_freqs(n: int, fs: float) -> np.ndarray:
    k = np.arange(n)
    return np.where(k < n // 2, k, k - n) * (fs / n)


def rrc_amplitude(f: np.ndarray, baud: float, rolloff: float) -> np.ndarray:
    """Square-root raised-cosine amplitude response (unit passband gain)."""
    af = np.abs(f)
    f1 = (1.0 - rolloff) * baud / 2.0
    f2 = (1.0 + rolloff) * baud / 2.0
    out = np.zeros_like(af)
    out[af <= f1] = 1.0
    band = (af > f1) & (af <= f2)
    out[band] = np.cos(np.pi * (af[band] - f1) / (2.0 * rolloff * baud))
    return out


def beta2_s2_per_m(D_ps_nm_km: float, lam_nm: float) -> float:
    """Group-velocity dispersion beta2 [s^2/m] from D [ps/(nm km)]."""
    D = D_ps_nm_km * 1e-12 / (1e-9 * 1e3)  # s/m^2
    lam = lam_nm * 1e-9
    return -D * lam * lam / (2.0 * math.pi * C_LIGHT)


def _fft(x, axis=-1):
    return sfft.fft(x, axis=axis, workers=-1)


def _ifft(x, axis=-1):
    return sfft.ifft(x, axis=axis, workers=-1)


def tx_shape(symbols: np.ndarray, baud: float, rolloff: float, sps: int = 2) -> np.ndarray:
    """Zero-insertion upsampling then sqrt(sps)*RRC over the whole-stream DFT grid."""
    K = symbols.shape[-1]
    n = K * sps
    up = np.zeros(symbols.shape[:-1] + (n,), np.complex128)
    up[..., ::sps] = symbols
    H = math.sqrt(sps) * rrc_amplitude(grid_freqs(n, sps * baud), baud, rolloff)
    return _ifft(_fft(up) * H)


def apply_dispersion(x: np.ndarray, fs: float, L_km: float, D_ps_nm_km: float,
                     lam_nm: float = 1550.0) -> np.ndarray:
    """Fibre chromatic dispersion, whole-stream: X(w)*exp(+j*beta2*L*w^2/2)."""
    n = x.shape[-1]
    w = 2.0 * np.pi * grid_freqs(n, fs)
    b2 = beta2_s2_per_m(D_ps_nm_km, lam_nm)
    H = np.exp(1j * b2 * (L_km * 1e3) * w * w / 2.0)
    return _ifft(_fft(x) * H)


def jones_matrix(theta: float, psi: float) -> np.ndarray:
    c, s = math.cos(theta), math.sin(theta)
    return np.array([[c, -s * np.exp(-1j * psi)], [s * np.exp(1j * psi), c]])


def apply_jones(x: np.ndarray, J: np.ndarray) -> np.ndarray:
    return np.einsum("pq,qn->pn", J, x)


def apply_pmd(x: np.ndarray, fs: float, mean_dgd_s: float, rng: np.random.Generator,
              n_sections: int = 100, block: int = 1 << 16, drift_rad: float = 1e-3,
              margin: int = 512, n_coarse: int = 257) -> np.ndarray:
    """Random-waveplate PMD whose plate angles random-walk from block to block.

    Each section is a random SU(2) rotation followed by a differential group
    delay tau_s; tau_s is set so that the concatenation has the requested mean
    DGD (Maxwellian mean = sqrt(8/(3 pi)) * rms).  The concatenated Jones
    matrix is smooth in frequency (its scale is 1/DGD, far wider than the
    signal band), so it is built on `n_coarse` frequencies spanning the band
    and interpolated linearly onto each block's DFT grid.  Each block of
    `block` samples is filtered in the frequency domain with its own matrix,
    using `margin` samples of context on either side.
    """
    n = x.shape[-1]
    tau = mean_dgd_s / (math.sqrt(n_sections) * math.sqrt(8.0 / (3.0 * math.pi)))
    ang = rng.uniform(0, 2 * np.pi, size=(n_sections, 3))
    out = np.empty_like(x)
    nblk = (n + block - 1) // block
    Lb = block + 2 * margin
    f_fine = grid_freqs(Lb, fs)
    f_c = np.linspace(-fs / 2, fs / 2, n_coarse)
    w_c = 2.0 * np.pi * f_c
    d = np.stack([np.exp(1j * w_c * tau / 2), np.exp(-1j * w_c * tau / 2)], axis=-1)   # (n_coarse, 2)
    for b in range(nblk):
        if b:
            ang = ang + rng.normal(0.0, drift_rad, size=ang.shape)
        M = np.zeros((n_coarse, 2, 2), np.complex128)
        M[:, 0, 0] = 1.0
        M[:, 1, 1] = 1.0
        ca, sa = np.cos(ang[:, 0]), np.sin(ang[:, 0])
        eb, ec = np.exp(1j * ang[:, 1]), np.exp(1j * ang[:, 2])
        for s in range(n_sections):
            U = np.array([[ca[s] * eb[s], -sa[s] / ec[s]], [sa[s] * ec[s], ca[s] / eb[s]]])
            M = d[:, :, None] * (U[None] @ M)
        Mf = np.empty((Lb, 2, 2), np.complex128)
        for i in range(2):
            for j in range(2):
                Mf[:, i, j] = (np.interp(f_fine, f_c, M[:, i, j].real)
                               + 1j * np.interp(f_fine, f_c, M[:, i, j].imag))
        lo = b * block - margin
        seg = np.zeros((2, Lb), np.complex128)
        a0, a1 = max(lo, 0), min(lo + Lb, n)
        seg[:, a0 - lo:a1 - lo] = x[:, a0:a1]
        S = _fft(seg)
        Y = np.einsum("fpq,qf->pf", Mf, S)
        y = _ifft(Y)
        e = min((b + 1) * block, n)
        out[:, b * block:e] = y[:, margin:margin + e - b * block]
    return out


def wiener_phase(n: int, linewidth_hz: float, fs: float, rng: np.random.Generator) -> np.ndarray:
    if linewidth_hz <= 0:
        return np.zeros(n)
    steps = rng.normal(0.0, math.sqrt(2.0 * math.pi * linewidth_hz / fs), size=n)
    return np.cumsum(steps)


def adc_int8(x: np.ndarray, ref_block: int = 1 << 16, clip_sigmas: float = 4.0):
    """Interleave to [n][Xi,Xq,Yi,Yq] and quantise to int8 with clipping at 4 sigma.

    sigma_q is the per-quadrature RMS over the first `ref_block` samples.
    Returns (int8 array (n,4), scale) where scale maps codes back to field units.
    """
    il = interleave(x)
    ref = il[:ref_block]
    sigma_q = float(np.sqrt(np.mean(ref * ref)))
    scale = clip_sigmas * sigma_q / 127.0
    q = np.clip(np.rint(il / scale), -128, 127).astype(np.int8)
    return q, scale


def interleave(x: np.ndarray) -> np.ndarray:
    """(2, n) complex -> (n, 4) real [Xi, Xq, Yi, Yq]."""
    return np.stack([x[0].real, x[0].imag, x[1].real, x[1].imag], axis=-1)


def deinterleave(a: np.ndarray) -> np.ndarray:
    a = np.asarray(a, dtype=np.float64)
    return np.stack([a[:, 0] + 1j * a[:, 1], a[:, 2] + 1j * a[:, 3]])


# ---------------------------------------------------------------------------
# Link description and generation
# ---------------------------------------------------------------------------
@dataclasses.dataclass
class Link:
    mod: str = "qpsk"
    baud: float = 10e9
    sps: int = 2
    n_sym: int = 1 << 16
    rolloff: float = 0.1
    L_km: float = 1000.0
    D: float = 17.0
    lam_nm: float = 1550.0
    jones: tuple | None = (math.pi / 5, math.pi / 7)   # (theta, psi); None = identity
    pmd_ps_sqrt_km: float = 0.0
    linewidth_hz: float = 0.0
    fo_hz: float = 0.0
    snr_db: float | None = 12.0                        # None = noise-free
    adc: str = "f32"                                    # "f32" or "int8"
    seed: int = 2104063111

    @property
    def fs(self) -> float:
        return self.sps * self.baud


@dataclasses.dataclass
class Generated:
    link: Link
    tx_bits: np.ndarray      # (2, K*m) uint8
    tx_symbols: np.ndarray   # (2, K) complex128
    field: np.ndarray        # (2, n) complex128, before the ADC
    samples: np.ndarray      # (n, 4) float32 or int8, what the receiver gets
    in_scale: float          # multiply codes by this to get field units

    @property
    def ref_words(self) -> np.ndarray:
        return pack_bits(self.tx_bits)


def generate(link: Link) -> Generated:
    m = bits_per_symbol(link.mod)
    K = link.n_sym
    bits = random_bits(link.seed, 2 * K * m).reshape(2, K * m)
    sym = map_symbols(bits, link.mod)
    rng = np.random.default_rng(np.random.PCG64(link.seed))
    x = tx_shape(sym, link.baud, link.rolloff, link.sps)
    n = x.shape[-1]
    if link.L_km:
        x = apply_dispersion(x, link.fs, link.L_km, link.D, link.lam_nm)
    if link.pmd_ps_sqrt_km > 0:
        dgd = link.pmd_ps_sqrt_km * 1e-12 * math.sqrt(link.L_km)
        x = apply_pmd(x, link.fs, dgd, rng)
    if link.jones is not None:
        x = apply_jones(x, jones_matrix(*link.jones))
    ph = wiener_phase(n, link.linewidth_hz, link.fs, rng)
    if link.fo_hz:
        ph = ph + 2.0 * math.pi * link.fo_hz / link.fs * np.arange(n)
    if np.any(ph):
        x = x * np.exp(1j * ph)[None, :]
    if link.snr_db is not None:
        var = 10.0 ** (-link.snr_db / 10.0)
        noise = rng.standard_normal((2, 2, n))
        x = x + math.sqrt(var / 2.0) * (noise[:, 0] + 1j * noise[:, 1])
    if link.adc == "int8":
        samples, scale = adc_int8(x)
    else:
        samples, scale = interleave(x).astype(np.float32), 1.0
    return Generated(link, bits, sym, x, samples, scale)


# Workloads of the receiver (seeded).  Sizes in symbols per polarisation.
def workload(name: str, n_sym: int | None = None) -> Link:
    if name == "c1":   # single channel DP-QPSK, 1000 km CD, fixed Jones, AWGN 12 dB, FP32
        lk = Link(mod="qpsk", baud=10e9, n_sym=1 << 16, L_km=1000.0,
                  jones=(math.pi / 5, math.pi / 7), snr_db=12.0, adc="f32",
                  seed=2104063111)
    elif name == "c2":  # 10,000 km straight-line shape, int8 ADC
        lk = Link(mod="qpsk", baud=10e9, n_sym=1 << 24, L_km=10000.0,
                  jones=(0.7, 1.9), pmd_ps_sqrt_km=0.1, linewidth_hz=100e3,
                  fo_hz=200e6, snr_db=9.80, adc="int8", seed=2104063112)
    elif name == "c3":  # DP-16QAM 32 GBd 6000 km, int8 ADC
        lk = Link(mod="16qam", baud=32e9, n_sym=1 << 22, L_km=6000.0,
                  jones=(1.1, 0.4), linewidth_hz=100e3, snr_db=18.0, adc="int8",
                  seed=2104063113)
    else:
        raise ValueError(name)
    if n_sym is not None:
        lk = dataclasses.replace(lk, n_sym=n_sym)
    return lk


def workload_batch(n_ch: int = 64, seed: int = 2104063114, log2_len=(18.0, 22.0), L_km=(2000.0, 10000.0),
                   baud=(10e9, 32e9), snr_db=(10.0, 18.0), len_quantum: int = 1 << 15) -> list:
    """Independent WDM channels of uneven length, symbol rate, dispersion and format.

    Per channel (drawn from a PCG64 stream seeded with `seed`): length 2^u
    symbols per pol with u ~ U[log2_len] rounded to a multiple of len_quantum,
    L ~ U[L_km], baud ~ U[baud], QPSK or 16QAM with probability 1/2 each,
    SNR ~ U[snr_db], a random fixed Jones rotation, int8 ADC, and its own bit
    seed seed + ch.  No inter-channel crosstalk, phase noise or frequency offset.
    """
    rng = np.random.default_rng(np.random.PCG64(seed))
    links = []
    for ch in range(n_ch):
        u = rng.uniform(*log2_len)
        n_sym = max(len_quantum, int(round(2.0 ** u / len_quantum)) * len_quantum)
        links.append(Link(mod="16qam" if rng.uniform() < 0.5 else "qpsk", baud=float(rng.uniform(*baud)),
                          n_sym=n_sym, L_km=float(rng.uniform(*L_km)),
                          jones=(float(rng.uniform(0, math.pi)), float(rng.uniform(0, 2 * math.pi))),
                          snr_db=float(rng.uniform(*snr_db)), adc="int8", seed=seed + ch))
    return links


def cnn_init_params(seed: int, channels: int = 64, ksize: int = 15, layers: int = 4, feat: int = 4):
    """Seeded initial weights of the post-equaliser CNN: He-normal W (std
    sqrt(2 / fan_in), shape (ksize, ci, co)) and zero biases; the last layer
    is scaled by 0.1 so the untrained network starts near y = x."""
    rng = np.random.default_rng(np.random.PCG64(seed))
    dims = [feat] + [channels] * (layers - 1) + [feat]
    params = []
    for l in range(layers):
        ci, co = dims[l], dims[l + 1]
        W = rng.standard_normal((ksize, ci, co)) * np.sqrt(2.0 / (ksize * ci))
        if l == layers - 1:
            W *= 0.1
        params.append((W, np.zeros(co)))
    return params


def align_rotation(z: np.ndarray, t: np.ndarray, block: int = 4096) -> np.ndarray:
    """Reference symbols t (2, K) rotated per block by the j^r (r = 0..3) that
    best matches the received z: genie-aided labels that stay aligned across
    a pi/2 cycle slip of the receiver's phase recovery (for training and
    judging a post-equaliser, not for counting errors)."""
    out = np.empty_like(t)
    for p in range(t.shape[0]):
        for b0 in range(0, t.shape[1], block):
            zz, tt = z[p, b0:b0 + block], t[p, b0:b0 + block]
            r = int(np.argmin([np.sum(np.abs(zz - (1j ** q) * tt) ** 2) for q in range(4)]))
            out[p, b0:b0 + block] = (1j ** r) * tt
    return out
