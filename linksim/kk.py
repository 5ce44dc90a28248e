"""Single-polarisation self-coherent (Kramers-Kronig) link: the paper's own
transmission set-up (Section "Experimental setup"), synthetic and seeded.

Transmitter: Gray QAM symbols at `baud`, RRC (roll-off 0.01) at `sps` samples
per symbol (the 4 GS/s ADC at 1 GBd gives 4), plus a carrier tone at
`carrier_hz` on the edge of the signal band, scaled so that carrier power /
signal power = CSPR.  Fibre: chromatic dispersion over L km (whole stream).
Optional transmitter IQ imbalance on the signal (Q arm gain 10^(g/20) and phase
skew theta): x = mu s + nu s*, mu = (1 + rho e^{j theta})/2,
nu = (1 - rho e^{j theta})/2 -- what a widely-linear equaliser undoes.
Receiver: AWGN on the optical field at Es/N0 = `snr_db` (signal power over
noise), square-law photodetection I = |E|^2, and either float32 samples or an
8-bit ADC (codes 0..255 stored as int8 c - 128; I = (c + 128) * step).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

from . import apply_dispersion, bits_per_symbol, map_symbols, random_bits, tx_shape


@dataclasses.dataclass
class KKLink:
    mod: str = "16qam"
    baud: float = 1e9
    sps: int = 4
    n_sym: int = 1 << 20
    rolloff: float = 0.01
    carrier_hz: float = 0.516e9
    cspr_db: float = 10.0
    L_km: float = 1000.0
    D: float = 17.0
    lam_nm: float = 1550.0
    snr_db: float | None = 25.0
    adc: str = "int8"
    seed: int = 2104063117
    iq_gain_db: float = 0.0
    iq_phase_deg: float = 0.0

    @property
    def fs(self) -> float:
        return self.sps * self.baud


@dataclasses.dataclass
class KKGenerated:
    link: KKLink
    tx_bits: np.ndarray      # (K*m,) uint8
    tx_symbols: np.ndarray   # (K,) complex128
    field: np.ndarray        # (n,) complex128 optical field at the receiver (carrier included)
    intensity: np.ndarray    # (n,) float64, |field|^2
    samples: np.ndarray      # (n,) int8 or float32, what the receiver gets
    in_scale: float          # I = (samples + in_offset) * in_scale
    in_offset: float


def iq_imbalance(link: KKLink) -> tuple[complex, complex]:
    """(mu, nu) of the transmitter's widely-linear distortion x = mu s + nu s*."""
    r = 10.0 ** (link.iq_gain_db / 20.0) * complex(math.cos(math.radians(link.iq_phase_deg)),
                                                   math.sin(math.radians(link.iq_phase_deg)))
    return (1.0 + r) / 2.0, (1.0 - r) / 2.0


def generate(link: KKLink) -> KKGenerated:
    m = bits_per_symbol(link.mod)
    K = link.n_sym
    bits = random_bits(link.seed, K * m)
    sym = map_symbols(bits.reshape(1, -1), link.mod)[0]
    s = tx_shape(sym[None, :], link.baud, link.rolloff, link.sps)[0]
    mu, nu = iq_imbalance(link)
    if nu != 0.0:
        s = mu * s + nu * np.conj(s)
    n = s.shape[0]
    p_s = float(np.mean(np.abs(s) ** 2))
    amp = math.sqrt(p_s * 10.0 ** (link.cspr_db / 10.0))
    t = np.arange(n)
    E = s + amp * np.exp(2j * np.pi * link.carrier_hz / link.fs * t)
    if link.L_km:
        E = apply_dispersion(E[None, :], link.fs, link.L_km, link.D, link.lam_nm)[0]
    if link.snr_db is not None:
        rng = np.random.default_rng(np.random.PCG64(link.seed))
        var = p_s * 10.0 ** (-link.snr_db / 10.0)
        E = E + math.sqrt(var / 2.0) * (rng.standard_normal(n) + 1j * rng.standard_normal(n))
    I = np.abs(E) ** 2
    if link.adc == "int8":
        step = float(np.max(I[:1 << 16])) * 1.25 / 255.0
        c = np.clip(np.rint(I / step), 0, 255)
        samples = (c - 128).astype(np.int8)
        return KKGenerated(link, bits, sym, E, I, samples, step, 128.0)
    return KKGenerated(link, bits, sym, E, I, I.astype(np.float32), 1.0, 0.0)
