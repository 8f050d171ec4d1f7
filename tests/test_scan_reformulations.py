"""CPU checks of the algebra behind the scan forms of the chain recurrences.

Several kernels replace a sequential chain recurrence by a segmented scan: each lane composes the
maps of its segment, a scan over the lanes composes the segments, and each lane walks its own
segment from the value the scan gives.  That is only valid if the maps compose as claimed and the
composition order is right.  These tests emulate the three reformulations in plain numpy, with the
kernels' segment lengths and lane counts, and compare them with the sequential recurrences they
replace:

* assembly (pivot recurrences of the bit-line chains, Sec. II-A): linear-fractional maps
  x -> g_b (G + x) / (G + x + g_b) as positive 2 x 2 matrices, 32 lanes, power-of-two rescaling;
* line-model factors: positive 2 x 2 linear maps on (a, c) with ratios c_{i-1} / c_i, 4 lanes;
* line-model chain sweeps: affine maps x -> a x + b, 4 lanes.

The GPU parity tests check the kernels themselves against the oracle; these pin the derivation.
"""
import math

import numpy as np


def _rescaled(m):
    e = math.frexp(max(abs(v) for v in m))[1]
    return tuple(math.ldexp(v, -e) for v in m)


def _mul(x, y):  # 2 x 2 product x y, (a, b, c, d) = [[a, b], [c, d]]
    return _rescaled((x[0] * y[0] + x[1] * y[2], x[0] * y[1] + x[1] * y[3],
                      x[2] * y[0] + x[3] * y[2], x[2] * y[1] + x[3] * y[3]))


ID = (1.0, 0.0, 0.0, 1.0)


def _apply(m, x):
    return (m[0] * x + m[1]) / (m[2] * x + m[3])


def _seq_pivots(G, gb, go):
    M = len(G)
    alpha, a = np.zeros(M), 0.0
    for i in range(M):
        if i > 0:
            t = G[i - 1] + a
            a = gb * t / (t + gb)
        alpha[i] = a
    beta, b = np.zeros(M), go
    for i in range(M - 1, -1, -1):
        if i < M - 1:
            t = G[i + 1] + b
            b = gb * t / (t + gb)
        beta[i] = b
    return alpha, beta


def _scan_pivots(G, gb, go, lanes=32):
    """Top-down alpha and bottom-up beta as the assembly kernel forms them."""
    M = len(G)
    K = (M + lanes - 1) // lanes
    step = lambda g: (gb, gb * g, 1.0, g + gb)
    P, Q = [], []
    for L in range(lanes):
        i0, i1 = min(L * K, M), min(L * K + K, M)
        p = ID
        for i in range(i0 + 1, min(i1, M - 1) + 1):  # maps producing alpha_i, i0 < i <= i1
            p = _mul(step(G[i - 1]), p)
        q = ID
        for i in range(i0, min(i1, M - 1)):  # maps producing beta_i, composed g_i0 o ... o g_top
            q = _mul(q, step(G[i + 1]))
        P.append(p)
        Q.append(q)
    alpha, beta = np.zeros(M), np.zeros(M)
    before = ID  # maps of the lanes before L
    for L in range(lanes):
        i0, i1 = min(L * K, M), min(L * K + K, M)
        a = _apply(before, 0.0)
        for i in range(i0, i1):
            if i > i0:
                t = G[i - 1] + a
                a = gb * t / (t + gb)
            alpha[i] = a
        before = _mul(P[L], before)
    after = ID  # maps of the lanes after L
    for L in range(lanes - 1, -1, -1):
        i0, i1 = min(L * K, M), min(L * K + K, M)
        b = _apply(after, go)
        for i in range(i1 - 1, i0 - 1, -1):
            if i < M - 1:
                t = G[i + 1] + b
                b = gb * t / (t + gb)
            else:
                b = go
            beta[i] = b
        after = _mul(Q[L], after)
    return alpha, beta


def test_assembly_pivot_scan_matches_sequential():
    rng = np.random.default_rng(0)
    for M in (1, 2, 3, 31, 32, 33, 100, 256, 257, 1000, 1024):
        for gb, go in ((1.0, 0.1), (0.4, 10.0), (1e3, 1e-3)):
            G = 10 ** rng.uniform(-6, -3, M)
            a1, b1 = _seq_pivots(G, gb, go)
            a2, b2 = _scan_pivots(G, gb, go)
            np.testing.assert_allclose(a2, a1, rtol=1e-12, atol=0)
            np.testing.assert_allclose(b2, b1, rtol=1e-12, atol=0)


def _seg_len(n, lanes=4):
    """The kernels' segment length: ceil(n / lanes) raised to 8 or 24 (mod 32)."""
    S = (n + lanes - 1) // lanes
    r = S & 31
    return S + ((8 - r) if r <= 8 else ((24 - r) if r <= 24 else (40 - r)))


def _seg_affine(n, x_init, ab, lanes=4):
    """x_t = a_t x_{t-1} + b_t by segments: compose, scan over the lanes, walk."""
    S = _seg_len(n, lanes)
    comp = []
    for l in range(lanes):
        A, B = 1.0, 0.0
        for t in range(min(l * S, n), min(l * S + S, n)):
            a, b = ab(t)
            A, B = a * A, a * B + b
        comp.append((A, B))
    out = np.zeros(n)
    A, B = 1.0, 0.0  # lanes before l composed
    for l in range(lanes):
        x = A * x_init + B
        for t in range(min(l * S, n), min(l * S + S, n)):
            a, b = ab(t)
            x = a * x + b
            out[t] = x
        A, B = comp[l][0] * A, comp[l][0] * B + comp[l][1]
    return out


def test_segment_lengths_cover_and_spread_banks():
    for n in range(1, 1025):
        S = _seg_len(n)
        assert 4 * S >= n and S % 32 in (8, 24)
    # 8 chains x 4 lanes of a warp at pitch = 1 (mod 32): 32 distinct banks
    S = _seg_len(128)
    banks = {(c + S * l) % 32 for c in range(8) for l in range(4)}
    assert len(banks) == 32


def test_line_model_sweeps_as_segmented_affine_scans():
    """Bit-line sweep of the line model: s_i = (G_i f_i + g_b s_{i-1}) / E_i forward, then
    x_i = (g_b / E_i) x_{i+1} + s_i back, against the sequential form."""
    rng = np.random.default_rng(1)
    for n in (1, 2, 5, 31, 33, 100, 128, 200, 256):
        G = 10 ** rng.uniform(-6, -4, n)
        f = rng.uniform(0, 1, n)
        gb = 0.4
        e = 1.0 / (G + 2 * gb + 1e-3)
        s, sp = np.zeros(n), 0.0
        for i in range(n):
            sp = (G[i] * f[i] + gb * sp) * e[i]
            s[i] = sp
        x_seq, x = np.zeros(n), s[n - 1]
        x_seq[n - 1] = x
        for i in range(n - 2, -1, -1):
            x = gb * e[i] * x + s[i]
            x_seq[i] = x
        s2 = _seg_affine(n, 0.0, lambda t: (gb * e[t], G[t] * f[t] * e[t]))
        np.testing.assert_allclose(s2, s, rtol=1e-12)
        back = _seg_affine(n, 0.0, lambda t: (0.0 if t == 0 else gb * e[n - 1 - t], s2[n - 1 - t]))
        np.testing.assert_allclose(back[::-1], x_seq, rtol=1e-12)


def test_line_model_factor_scan_matches_sequential():
    """Pivots of a line-model chain: (a, c) <- [[g_b, G_i], [g_b, G_i + k_i]] (a, c) from (0, 1),
    1/E_i = c_{i-1} / c_i, composed per segment and scanned over 4 lanes."""
    rng = np.random.default_rng(2)
    for n in (1, 2, 3, 31, 33, 100, 128, 200, 256):
        G = 10 ** rng.uniform(-6, -4, n)
        gb, go = 0.4, 0.1
        k = lambda i: gb if i < n - 1 else go
        e_seq, a, c = np.zeros(n), 0.0, 1.0
        for i in range(n):
            an = G[i] * c + gb * a
            num = an + k(i) * c
            e_seq[i] = c / num
            a, c = an, num
        S = _seg_len(n)
        mats = []
        for l in range(4):
            p = ID
            for i in range(min(l * S, n), min(l * S + S, n)):
                p = _mul((gb, G[i], gb, G[i] + k(i)), p)
            mats.append(p)
        e_scan, before = np.zeros(n), ID
        for l in range(4):
            a, c = before[1], before[3]  # the earlier maps applied to (0, 1)
            for i in range(min(l * S, n), min(l * S + S, n)):
                an = G[i] * c + gb * a
                num = an + k(i) * c
                e_scan[i] = c / num
                a, c = an, num
            before = _mul(mats[l], before)
        np.testing.assert_allclose(e_scan, e_seq, rtol=1e-12)
