"""Split-step Fourier simulation of a dual-polarisation fibre link (Manakov).

Test infrastructure: it makes the Kerr-nonlinear inputs the learned
post-equaliser trains on.  The paper's own lab link (a 1 GBd single
polarisation Kramers-Kronig system, Section "Experimental setup") is replaced
by a synthetic multi-span coherent link:

  field A = (A_x, A_y) in sqrt(W), z in km, per step dz:
    linear     dA/dz = -(alpha/2) A + dispersion, applied per frequency as
               exp((-alpha/2 + j beta2 w^2 / 2) dz)  (the sign of the rest of
               linksim: the channel multiplies by exp(+j beta2 L w^2 / 2));
    nonlinear  A_p <- A_p exp(j (8/9) gamma (|A_x|^2 + |A_y|^2) dz)
               (Manakov equation: the polarisation-averaged Kerr term);
  symmetric split (half linear, nonlinear, half linear), consecutive half
  steps merged; after each span an EDFA with power gain G = exp(alpha L_span)
  adds circular white ASE of variance n_sp h nu (G - 1) f_sim per complex
  sample and polarisation, n_sp = 10^(NF/10) / 2.

The transmitter is linksim's (Gray symbols, sqrt(sps) RRC over the DFT
grid) at `sim_sps` samples per symbol; the receiver front end is an ideal
low-pass filter (DFT truncation) to 2 samples per symbol, an AGC to unit
mean power per polarisation, and the int8 ADC of linksim.

Runs with torch on the CPU (float64, the pins) or on a GPU (float32 or
float64) for full-size streams.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

from . import (Generated, adc_int8, beta2_s2_per_m, bits_per_symbol, interleave, map_symbols,
               random_bits, tx_shape)

H_PLANCK = 6.62607015e-34
C_LIGHT = 299792458.0


@dataclasses.dataclass
class SSFMLink:
    mod: str = "16qam"
    baud: float = 32e9
    n_sym: int = 1 << 22
    rolloff: float = 0.1
    spans: int = 100
    span_km: float = 100.0
    step_km: float = 1.0
    alpha_db_km: float = 0.2
    gamma: float = 1.3          # 1/(W km)
    D: float = 17.0             # ps/(nm km)
    lam_nm: float = 1550.0
    nf_db: float = 5.0
    launch_dbm: float = 0.0     # total over both polarisations
    sim_sps: int = 4
    ase: bool = True
    adc: str = "int8"
    seed: int = 2104063115

    @property
    def L_km(self) -> float:
        return self.spans * self.span_km

    @property
    def alpha(self) -> float:   # power attenuation per km
        return self.alpha_db_km / (10.0 * math.log10(math.e))

    @property
    def beta2(self) -> float:   # s^2 per km
        return beta2_s2_per_m(self.D, self.lam_nm) * 1e3


def omega_grid(n: int, fs: float, torch, device, dtype):
    k = torch.arange(n, device=device, dtype=dtype)
    f = torch.where(k < n / 2, k, k - n) * (fs / n)
    return 2 * math.pi * f


def linear_op(link: SSFMLink, w, dz_km: float, torch):
    """exp((-alpha/2 + j beta2 w^2 / 2) dz) on the frequency grid w (rad/s)."""
    ph = (link.beta2 / 2.0) * w * w * dz_km
    return torch.exp(torch.complex(torch.full_like(w, -link.alpha / 2.0 * dz_km), ph))


def nonlinear_step(A, link: SSFMLink, dz_km: float, torch):
    p = (A.real ** 2 + A.imag ** 2).sum(dim=0, keepdim=True)
    phi = (8.0 / 9.0) * link.gamma * dz_km * p
    return A * torch.exp(torch.complex(torch.zeros_like(phi), phi))


def propagate(A, link: SSFMLink, fs: float, torch, noise_gen=None):
    """All spans: SSFM steps, then an EDFA (gain + ASE) after each span."""
    n = A.shape[-1]
    w = omega_grid(n, fs, torch, A.device, A.real.dtype)
    nstep = int(round(link.span_km / link.step_km))
    dz = link.span_km / nstep
    half = linear_op(link, w, dz / 2.0, torch)
    full = linear_op(link, w, dz, torch)
    G = math.exp(link.alpha * link.span_km)
    nu = C_LIGHT / (link.lam_nm * 1e-9)
    n_sp = 10.0 ** (link.nf_db / 10.0) / 2.0
    ase_var = n_sp * H_PLANCK * nu * (G - 1.0) * fs      # per complex sample per pol
    for _ in range(link.spans):
        X = torch.fft.fft(A, dim=-1) * half
        for s in range(nstep):
            A = nonlinear_step(torch.fft.ifft(X, dim=-1), link, dz, torch)
            X = torch.fft.fft(A, dim=-1) * (full if s < nstep - 1 else half)
        A = torch.fft.ifft(X, dim=-1) * math.sqrt(G)
        if link.ase:
            sig = math.sqrt(ase_var / 2.0)
            nr = noise_gen(A.shape) * sig
            ni = noise_gen(A.shape) * sig
            A = A + torch.complex(nr, ni)
    return A


def lowpass_resample(A, n_out: int, torch):
    """Ideal low-pass to the band of n_out samples (DFT truncation), same duration."""
    n = A.shape[-1]
    X = torch.fft.fft(A, dim=-1)
    h = n_out // 2
    Y = torch.cat([X[..., :h], X[..., n - h:]], dim=-1) * (n_out / n)
    return torch.fft.ifft(Y, dim=-1)


def generate(link: SSFMLink, device: str = "cpu", dtype: str = "float64") -> Generated:
    """Seeded bits -> symbols -> TX at sim_sps -> fibre -> 2 sps receiver samples."""
    import torch
    m = bits_per_symbol(link.mod)
    K = link.n_sym
    bits = random_bits(link.seed, 2 * K * m).reshape(2, K * m)
    sym = map_symbols(bits, link.mod)
    x = tx_shape(sym, link.baud, link.rolloff, link.sim_sps)          # (2, K*sim_sps), ~1 per sample per pol
    p_tx = float(np.mean(np.abs(x) ** 2) * 2)
    launch_w = 1e-3 * 10.0 ** (link.launch_dbm / 10.0)
    rdt = torch.float64 if dtype == "float64" else torch.float32
    cdt = torch.complex128 if dtype == "float64" else torch.complex64
    A = torch.from_numpy(x * math.sqrt(launch_w / p_tx)).to(device=device, dtype=cdt)
    gen = torch.Generator(device=device)
    gen.manual_seed(link.seed + 1)

    def noise(shape):
        return torch.randn(shape, generator=gen, device=device, dtype=rdt)

    fs = link.sim_sps * link.baud
    A = propagate(A, link, fs, torch, noise)
    y = lowpass_resample(A, 2 * K, torch)
    y = y / torch.sqrt((y.real ** 2 + y.imag ** 2).mean(dim=-1, keepdim=True))   # AGC
    field = y.to(torch.complex128).cpu().numpy()
    if link.adc == "int8":
        samples, scale = adc_int8(field)
    else:
        samples, scale = interleave(field).astype(np.float32), 1.0
    return Generated(link, bits, sym, field, samples, scale)
