"""The algebraic restatements the CUDA kernels make, checked in FP64 against the plain
definitions they replace (CPU only).  The GPU parity tests compare whole outputs; these
pin each identity on its own, so that a wrong constant or index in one of them is
named directly.

* 16QAM distance on the grid scaled by sqrt10 (BPS and the equaliser's inner BPS):
  per dimension (| |x'| - 2 | - 1)^2 with x' = sqrt10 x equals 10 (x - dec x)^2,
  dec the nearest of the levels {-3, -1, 1, 3} / sqrt10.
* QPSK inner-BPS cost: |w - dec w|^2 = |w|^2 + 1 - sqrt2 (|Re w| + |Im w|), so
  -(|Re w| + |Im w|) orders the test angles as the distance does.
* BPS window sums at half window 16 from two 32-symbol blocks: the 33-term sum of
  output symbol 32 q + i is the suffix of block q from i plus the prefix of block
  q + 1 up to i; positions outside the stream count zero.
* The equaliser's window rotation advances the turn of a thread's samples by
  exact modular 64-bit steps: Phi + (n - n0) delta (mod 2^64) is the same for the
  direct product and for the start value plus r times the step.
* The BER count over 32-bit words: the reference word of a received word's
  symbols, delayed by d, is the funnel shift of two neighbouring reference words by
  d m bits; the Gray rotation by j applies to every m-bit field at once with masks
  and shifts; masking the symbols outside the counted range gives the oracle's
  per-symbol count (oracle.chain.ber_sync_count's counting rule).
"""
import numpy as np

RNG = np.random.default_rng(2104063199)
S10 = np.sqrt(10.0)


def _dec16(x):
    lv = np.array([-3.0, -1.0, 1.0, 3.0]) / S10
    return lv[np.argmin(np.abs(x[..., None] - lv), axis=-1)]


def test_scaled_16qam_distance_equals_ten_times_the_grid_distance():
    x = np.concatenate([RNG.normal(0, 0.6, 200000), np.array([0.0, 2 / S10, -2 / S10, 4 / S10, -4 / S10])])
    lhs = (np.abs(np.abs(S10 * x) - 2.0) - 1.0) ** 2
    rhs = 10.0 * (x - _dec16(x)) ** 2
    assert np.max(np.abs(lhs - rhs)) < 1e-12


def test_qpsk_cost_orders_angles_like_the_distance():
    y = RNG.normal(0, 0.8, 4000) + 1j * RNG.normal(0, 0.8, 4000)
    phi = (np.arange(32) / 32 - 0.5) * np.pi / 2
    w = y[:, None] * np.exp(-1j * phi)[None, :]
    a = 1 / np.sqrt(2)
    dist = (np.abs(w.real) - a) ** 2 + (np.abs(w.imag) - a) ** 2
    cost = -(np.abs(w.real) + np.abs(w.imag))
    # the distance is the cost scaled by sqrt2 plus a per-symbol constant
    assert np.max(np.abs(dist - (np.abs(y) ** 2 + 1)[:, None] - np.sqrt(2) * cost)) < 1e-12
    assert np.array_equal(np.argmin(dist, axis=1), np.argmin(cost, axis=1))


def _direct_window_sums(d, Nb, v_lo, v_hi):
    """D_t = sum_{m=t}^{t+2Nb} d_m over valid positions (stream ends count zero)."""
    n = d.shape[0] - 2 * Nb
    dm = np.where((np.arange(d.shape[0]) >= v_lo) & (np.arange(d.shape[0]) < v_hi), d, 0.0)
    return np.array([dm[t:t + 2 * Nb + 1].sum() for t in range(n)])


def _block_window_sums(d, v_lo, v_hi):
    """The kernel's scheme at Nb = 16: suffix of block q + prefix of block q + 1."""
    nt = d.shape[0] - 32
    pad = np.zeros(nt + 64 + 32)
    pad[:d.shape[0]] = d
    pos = np.arange(pad.shape[0])
    pad = np.where((pos >= v_lo) & (pos < v_hi), pad, 0.0)
    out = np.zeros(nt)
    for base in range(0, nt, 32):
        b0 = pad[base:base + 32]
        b1 = pad[base + 32:base + 64]
        suf = np.cumsum(b0[::-1])[::-1]
        pre = np.cumsum(b1)
        cnt = min(32, nt - base)
        out[base:base + cnt] = (suf + pre)[:cnt]
    return out


def test_block_window_sums_equal_the_33_symbol_window():
    for nt, v_lo, v_hi in ((256, 0, 256 + 32), (256, 16, 256 + 32), (100, 0, 100 + 32),
                           (77, 16, 77 + 16), (32, 5, 40), (1, 16, 17)):
        d = RNG.uniform(0, 4, nt + 32)
        ref = _direct_window_sums(d, 16, v_lo, v_hi)
        got = _block_window_sums(d, v_lo, v_hi)
        assert np.max(np.abs(got - ref)) < 1e-12, (nt, v_lo, v_hi)


def test_rotation_turns_by_modular_steps():
    M = 1 << 64
    for _ in range(200):
        phi = int(RNG.integers(0, 1 << 62)) * 4 + 3
        delta = int(RNG.integers(0, 1 << 62)) * 2 + 1
        n0 = int(RNG.integers(0, 1 << 40))
        win_lo = int(RNG.integers(-7, 1 << 40))
        tid = int(RNG.integers(0, 128))
        ph0 = (phi + ((win_lo + tid - n0) % M) * delta) % M
        step = (128 * delta) % M
        for r in (0, 1, 7, 18):
            n = win_lo + tid + 128 * r
            direct = (phi + ((n - n0) % M) * delta) % M
            assert (ph0 + r * step) % M == direct


M32 = 0xFFFFFFFF


def _rotate_word(w, r, m):
    """The field-wise Gray rotation of the BER count kernel."""
    for _ in range(r):
        if m == 2:
            w = (((~w & M32) >> 1) & 0x55555555) | ((w << 1) & 0xAAAAAAAA)
        else:
            w = (((w >> 2) & 0x33333333) ^ 0x11111111) | ((w << 2) & 0xCCCCCCCC)
        w &= M32
    return w


def _count_words(rx, ref, K, m, k0, q, r, d, p):
    """The word-wide count the BER kernel makes: one 32-bit word of received bits at a
    time, the delayed reference word by a funnel shift, the valid symbols masked."""
    W, nw = 32 // m, (K * m + 31) // 32
    lo_all, hi_all = max(k0, -d), min(K, K - d)
    e = n = 0
    for w in range(k0 // W, nw):
        s0 = w * W
        lo, hi = max(lo_all, s0), min(hi_all, s0 + W)
        if hi <= lo:
            continue
        b0, b1 = (lo - s0) * m, (hi - s0) * m
        mask = (M32 if b1 >= 32 else (1 << b1) - 1) & ~((1 << b0) - 1) & M32
        bit = 32 * w + d * m
        fw = bit // 32
        sh = bit - 32 * fw
        low = int(ref[q][fw]) if 0 <= fw < nw else 0
        high = int(ref[q][fw + 1]) if 0 <= fw + 1 < nw else 0
        refw = _rotate_word(((high << 32 | low) >> sh) & M32, r, m)
        e += bin((int(rx[p][w]) ^ refw) & mask).count("1")
        n += bin(mask).count("1")
    return e, n


def test_word_wide_ber_count_equals_the_per_symbol_count():
    import oracle.chain as OC
    mods = {2: "qpsk", 4: "16qam"}
    for m in (2, 4):
        for K in (777, 1000, 1003):
            nw = (K * m + 31) // 32
            rx = RNG.integers(0, 2 ** 32, size=(2, nw), dtype=np.uint64)
            ref = RNG.integers(0, 2 ** 32, size=(2, nw), dtype=np.uint64)
            # unpacked bits (the oracle's layout: bit t of symbol k at k m + t, LSB first)
            unpack = lambda a: ((a[:, :, None] >> np.arange(32, dtype=np.uint64)) & 1).reshape(2, -1)[:, :K * m]
            rxb, refb = unpack(rx).astype(np.uint8), unpack(ref).astype(np.uint8)
            for _ in range(12):
                k0 = int(RNG.integers(0, 300))
                q, r, p, d = int(RNG.integers(0, 2)), int(RNG.integers(0, 4)), int(RNG.integers(0, 2)), \
                    int(RNG.integers(-64, 65))
                # the per-symbol definition: the oracle's rotation of the reference, delayed
                rot = OC._rotate_bits(refb, r, mods[m]).reshape(2, K, m)
                a = rxb.reshape(2, K, m)
                k = np.arange(k0, K)
                ok = (k + d >= 0) & (k + d < K)
                e = int(np.sum(a[p, k[ok]] != rot[q, (k + d)[ok]]))
                assert _count_words(rx, ref, K, m, k0, q, r, d, p) == (e, int(ok.sum()) * m)
