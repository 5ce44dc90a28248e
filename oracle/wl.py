"""FP64 reference of the widely-linear DD-LMS equaliser that ends the paper's
Kramers-Kronig chain (test infrastructure only: tests/, __graft_entry__.smoke()
and bench.py's CPU baseline may use it).

The paper (Section "Experimental setup", processing-chain paragraph) filters
the 2-samples-per-symbol output of the static filter with a four-tap adaptive
time-domain decision-directed LMS equaliser in widely-linear form (Silva et al.),
and demaps its decisions.  Readings (the paper names the method, not its
constants):

  * Four taps per branch at T/2 spacing on the regressor x and on its
    conjugate: z_k = sum_i h[i] x[2k+c-i] + g[i] conj(x[2k+c-i]), i = 0..T-1,
    c = (T-1)//2; before the buffer x continues with the previous buffer's last
    samples (zero for the first buffer), after it x = 0.  Start: h[c] = 1, all else 0 (the
    static filter delivers unit gain and no constant phase).
  * Decision-directed error e_k = dec(z_k) - z_k on the unit-energy square
    constellation; the LMS step after every symbol (the textbook, sequential
    form): h[i] += mu e_k conj(x[2k+c-i]), g[i] += mu e_k x[2k+c-i].  The
    strictly linear variant keeps g at 0.
  * The parallel schedule is part of the definition (as for the dual-pol
    equaliser): each call is one buffer and one wave.  The very first call
    runs its first A symbols as one sequential chain (acquisition).  The rest
    of a call is cut into segments of S symbols; every segment starts from the
    taps at the end of the previous wave (the last segment of the previous
    call, or the acquisition), first trains on the up to W symbols before it
    in the buffer (outputs discarded) and then emits its own.  The taps at
    the end of the call's last segment start the next call.
  * Hard bits: the Gray bits of the decision (oracle.chain.hard_bits).
"""
from __future__ import annotations

import dataclasses

import numpy as np

from .chain import decide, hard_bits


@dataclasses.dataclass
class WLParams:
    mod: str = "16qam"
    ntaps: int = 4
    mu: float = 1e-3
    seg_len: int = 256
    pretrain: int = 128
    acq: int = 8192
    linear: bool = False


def initial_taps(T: int) -> np.ndarray:
    """(2, T) complex: row 0 = h on x, row 1 = g on conj(x); h[c] = 1."""
    w = np.zeros((2, T), np.complex128)
    w[0, (T - 1) // 2] = 1.0
    return w


def _regressor(x: np.ndarray, k: int, T: int, tail: np.ndarray) -> np.ndarray:
    """x[2k+c-i] for i = 0..T-1: tail[len(tail) + n] for n < 0 (the previous buffer's
    last samples), zero past the buffer."""
    c = (T - 1) // 2
    u = np.zeros(T, np.complex128)
    for i in range(T):
        n = 2 * k + c - i
        if 0 <= n < x.shape[0]:
            u[i] = x[n]
        elif -tail.shape[0] <= n < 0:
            u[i] = tail[tail.shape[0] + n]
    return u


def _run(x: np.ndarray, w: np.ndarray, k0: int, k1: int, p: WLParams, z: np.ndarray | None,
         tail: np.ndarray) -> np.ndarray:
    """Symbols k0..k1-1 in order from taps w (copied); z[k] written when z is given."""
    h, g = w[0].copy(), (np.zeros_like(w[1]) if p.linear else w[1].copy())
    for k in range(k0, k1):
        u = _regressor(x, k, p.ntaps, tail)
        zk = np.dot(h, u) + np.dot(g, np.conj(u))
        e = decide(np.array([zk]), p.mod)[0] - zk
        h += p.mu * e * np.conj(u)
        if not p.linear:
            g += p.mu * e * u
        if z is not None:
            z[k] = zk
    return np.stack([h, g])


@dataclasses.dataclass
class WLState:
    taps: np.ndarray
    acquired: bool = False
    tail: np.ndarray = dataclasses.field(default_factory=lambda: np.zeros(2, np.complex128))


def wl_equalise(x: np.ndarray, p: WLParams, state: WLState | None = None):
    """One buffer x (complex, 2 samples/symbol, even length) -> (z, bits, state).

    z: (K,) equaliser outputs, K = len(x)/2; bits: (K*m,) uint8 Gray bits of the
    decisions; state carries the wave-start taps and the acquisition flag.
    """
    x = np.asarray(x, np.complex128)
    if state is None:
        state = WLState(initial_taps(p.ntaps))
    K = x.shape[0] // 2
    z = np.zeros(K, np.complex128)
    w = state.taps
    tail = state.tail
    a0 = 0
    if not state.acquired:
        a0 = min(p.acq, K)
        w = _run(x, w, 0, a0, p, z, tail)
    end = w
    for s0 in range(a0, K, p.seg_len):
        s1 = min(s0 + p.seg_len, K)
        pre = _run(x, w, max(0, s0 - p.pretrain), s0, p, None, tail)
        end = _run(x, pre, s0, s1, p, z, tail)
    bits = hard_bits(z, p.mod)
    new_tail = x[-2:].copy() if x.shape[0] >= 2 else tail.copy()
    return z, bits, WLState(end, True, new_tail)
