"""Checks that pin the CPU oracle to facts outside itself.

Each function raises AssertionError when the oracle disagrees with a fact the
paper or circuit theory fixes.  They are collected into tests by
``test_oracle_pins.py`` and re-run against deliberately broken copies of the
oracle by ``test_oracle_mutants.py`` (every planted mistake must trip one).

Sources of truth used here, none of which is the oracle's own code:
  * an independent dense modified-nodal-analysis "stamp" assembly: every
    resistor of the circuit (Sec. II-A) adds +g/-g to a dense matrix in a
    different node numbering, then is permuted into the paper's ordering;
  * the printed coefficients of Eqs. 5-7 (tests/golden/paper_nodal_equations.json);
  * LAPACK's pivoted dense solve (numpy.linalg.solve) on tiny crossbars;
  * series/parallel closed forms of 1x1, 1xN=2 and M=2x1 crossbars;
  * Kirchhoff conservation, linearity, reciprocity (symmetric A), the
    maximum principle and Rayleigh monotonicity of resistor networks;
  * the zero-parasitic limit I_j -> sum_i V_i G_ij with first-order rate.
"""
from __future__ import annotations

import json
import os

import numpy as np

import oracle

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


# ---------------------------------------------------------------------------------------------
# independent assembly: element stamps in a WL-block / BL-block numbering
# ---------------------------------------------------------------------------------------------
def circuit_elements(M, N, G, Rs, Rw, Rb, Rsense):
    """List of resistors (node_a, node_b, conductance); nodes ('w',i,j), ('u',i,j), ('src',i), 'gnd'."""
    el = []
    for i in range(M):
        el.append((("src", i), ("w", i, 0), 1.0 / Rs))
        for j in range(N - 1):
            el.append((("w", i, j), ("w", i, j + 1), 1.0 / Rw))
        for j in range(N):
            el.append((("w", i, j), ("u", i, j), G[i, j]))
    for j in range(N):
        for i in range(M - 1):
            el.append((("u", i, j), ("u", i + 1, j), 1.0 / Rb))
        el.append((("u", M - 1, j), "gnd", 1.0 / Rsense))
    return el


def stamp_dense(M, N, G, Rs, Rw, Rb, Rsense, V=None):
    """Dense nodal matrix (and rhs for one input vector V) by stamping each resistor.

    Numbering: all word-line nodes first (i*N+j), then all bit-line nodes
    (MN + i*N+j).  Returned already permuted into the paper's interleaved order.
    """
    k = 2 * M * N

    def num(node):
        if node[0] == "w":
            return node[1] * N + node[2]
        return M * N + node[1] * N + node[2]

    A = np.zeros((k, k))
    b = np.zeros(k)
    for a, c, g in circuit_elements(M, N, G, Rs, Rw, Rb, Rsense):
        known = [n for n in (a, c) if n == "gnd" or n[0] == "src"]
        free = [n for n in (a, c) if not (n == "gnd" or n[0] == "src")]
        if len(free) == 2:
            p, q = num(free[0]), num(free[1])
            A[p, p] += g
            A[q, q] += g
            A[p, q] -= g
            A[q, p] -= g
        else:
            p = num(free[0])
            A[p, p] += g
            if known[0] != "gnd" and V is not None:
                b[p] += g * V[known[0][1]]
    perm = np.empty(k, dtype=int)          # interleaved position -> block numbering
    for i in range(M):
        for j in range(N):
            perm[2 * (i * N + j)] = i * N + j
            perm[2 * (i * N + j) + 1] = M * N + i * N + j
    return A[np.ix_(perm, perm)], b[perm]


def rand_case(rng, M, N):
    G = np.exp(rng.uniform(np.log(1e-6), np.log(1e-2), size=(M, N)))
    R = tuple(float(x) for x in rng.uniform(0.3, 12.0, size=4))
    return G, R


# ---------------------------------------------------------------------------------------------
# pins
# ---------------------------------------------------------------------------------------------
def pin_counts():
    """nnz = 8MN - 2M - 2N, half-bandwidth 2N (Sec. II-B), 3MN resistors and 2MN nodes (Sec. II-A)."""
    facts = json.load(open(os.path.join(GOLDEN, "paper_nodal_equations.json")))
    rng = np.random.default_rng(1)
    for M, N in [(1, 1), (1, 3), (3, 1), (4, 3), (3, 4), (5, 2), (2, 5), (6, 6)]:
        G, R = rand_case(rng, M, N)
        ab, p = oracle.assemble_band(M, N, G, *R)
        A = oracle.band_to_dense(ab, p)
        assert A.shape[0] == eval(facts["counts"]["nodes"]["formula"], {"m": M, "n": N})
        assert len(circuit_elements(M, N, G, *R)) == eval(facts["counts"]["resistors"]["formula"],
                                                          {"m": M, "n": N})
        assert np.count_nonzero(A) == 8 * M * N - 2 * M - 2 * N, (M, N)
        r, c = np.nonzero(A)
        # the widest coupling is BL(i,j)-BL(i+1,j) (2N apart) when M > 1, else WL-WL (2) or WL-BL (1)
        assert np.max(np.abs(r - c)) == (2 * N if M > 1 else (2 if N > 1 else 1)), (M, N)
        assert p == oracle.half_bandwidth(M, N) == 2 * N
        assert np.array_equal(A, A.T)


def pin_stamp_assembly():
    """Band assembly equals the independent element-stamp assembly entry by entry."""
    rng = np.random.default_rng(2)
    for M in range(1, 6):
        for N in range(1, 6):
            G, R = rand_case(rng, M, N)
            V = rng.uniform(0, 0.5, size=M)
            ab, p = oracle.assemble_band(M, N, G, *R)
            A = oracle.band_to_dense(ab, p)
            As, bs = stamp_dense(M, N, G, *R, V=V)
            np.testing.assert_allclose(A, As, rtol=1e-15, atol=0)
            np.testing.assert_allclose(oracle.rhs(M, N, V[None, :], R[0])[0], bs, rtol=1e-15, atol=0)


def pin_paper_equations():
    """Rows of interior nodes carry exactly the printed coefficients of Eqs. 5, 6, 7 (R_s = R_w = R_b)."""
    facts = json.load(open(os.path.join(GOLDEN, "paper_nodal_equations.json")))
    M, N = 5, 6
    rng = np.random.default_rng(3)
    G = np.exp(rng.uniform(np.log(1e-6), np.log(1e-4), size=(M, N)))
    r_wire = 2.5
    ab, p = oracle.assemble_band(M, N, G, r_wire, r_wire, r_wire, 10.0)
    A = oracle.band_to_dense(ab, p)
    V = rng.uniform(0, 0.5, size=M)
    b = oracle.rhs(M, N, V[None, :], r_wire)[0]

    def node(name, i, j):
        base = 2 * (i * N + j)
        return base if name == "WL" else base + 1

    def parse(key, i, j):
        nm, rest = key.split("(")
        ii, jj = rest.rstrip(")").split(",")
        return node(nm, eval(ii.replace("i", str(i))), eval(jj.replace("j", str(j))))

    checked = 0
    for row in facts["rows"]:
        for i in range(M):
            for j in range(N):
                ok = eval(row["where"].replace("i", str(i + 1)).replace("j", str(j + 1))
                          .replace("m", str(M)).replace("n", str(N)))
                if not ok:
                    continue
                env = {"G_WL": 1 / r_wire, "G_BL": 1 / r_wire, "G": G[i, j], "V_i": V[i]}
                r = node(row["node"], i, j)
                expect = np.zeros(A.shape[0])
                for key, expr in row["coeffs"].items():
                    expect[parse(key, i, j)] = eval(expr, env)
                np.testing.assert_allclose(A[r], expect, rtol=1e-14, atol=0)
                np.testing.assert_allclose(b[r], eval(row["rhs"], env), rtol=1e-14, atol=0)
                checked += 1
    assert checked == M * (N - 1) + (M - 2) * N


def pin_dense_bruteforce():
    """Banded LU + substitution equals a pivoted dense solve of the stamped system (M, N <= 4)."""
    rng = np.random.default_rng(4)
    for M in range(1, 5):
        for N in range(1, 5):
            for _ in range(5):
                G, R = rand_case(rng, M, N)
                V = rng.uniform(0, 0.5, size=(3, M))
                out = oracle.solve(M, N, G, *R, V, voltages=True)
                for b in range(3):
                    As, bs = stamp_dense(M, N, G, *R, V=V[b])
                    x = np.linalg.solve(As, bs)
                    np.testing.assert_allclose(out["x"][b], x, rtol=1e-12, atol=1e-15)
                    Iref = x[[2 * ((M - 1) * N + j) + 1 for j in range(N)]] / R[3]
                    np.testing.assert_allclose(out["I"][b], Iref, rtol=1e-12, atol=0)


def pin_closed_forms():
    """1x1, 1x2 and 2x1 crossbars reduce to series/parallel resistor formulas."""
    rng = np.random.default_rng(5)
    for _ in range(20):
        Rs, Rw, Rb, Rse = rng.uniform(0.2, 20.0, size=4)
        g = np.exp(rng.uniform(np.log(1e-6), np.log(1.0), size=2))
        V = rng.uniform(0.01, 1.0, size=2)
        # 1x1: V through Rs, 1/G, Rsense in series
        I = oracle.solve(1, 1, g[:1].reshape(1, 1), Rs, Rw, Rb, Rse, V[None, :1])["I"][0, 0]
        np.testing.assert_allclose(I, V[0] / (Rs + 1 / g[0] + Rse), rtol=1e-14)
        # 1x2: node a after Rs feeds two branches: 1/G1 + Rsense  and  Rw + 1/G2 + Rsense
        r1, r2 = 1 / g[0] + Rse, Rw + 1 / g[1] + Rse
        par = r1 * r2 / (r1 + r2)
        va = V[0] * par / (Rs + par)
        I = oracle.solve(1, 2, g.reshape(1, 2), Rs, Rw, Rb, Rse, V[None, :1])["I"][0]
        np.testing.assert_allclose(I, [va / r1, va / r2], rtol=1e-13)
        # 2x1: two sources with series Rs + 1/G_i; branch 1 reaches the sense node through Rb
        # (Millman's theorem at the bottom bit-line node)
        rho1, rho2 = Rs + 1 / g[0], Rs + 1 / g[1]
        u2 = (V[0] / (rho1 + Rb) + V[1] / rho2) / (1 / (rho1 + Rb) + 1 / rho2 + 1 / Rse)
        I = oracle.solve(2, 1, g.reshape(2, 1), Rs, Rw, Rb, Rse, V[None, :])["I"][0, 0]
        np.testing.assert_allclose(I, u2 / Rse, rtol=1e-13)


def pin_kirchhoff_linearity_reciprocity():
    """Source currents sum to sense currents; I is linear in V; A^-1 is symmetric."""
    rng = np.random.default_rng(6)
    for M, N in [(7, 5), (4, 9), (12, 12)]:
        G, R = rand_case(rng, M, N)
        V = rng.uniform(0, 0.5, size=(4, M))
        f = oracle.factor(M, N, G, *R)
        out = oracle.solve_factored(f, V, voltages=True)
        np.testing.assert_allclose(out["Isrc"].sum(1), out["I"].sum(1), rtol=1e-11)
        a, b = 0.7, -1.3
        lin = oracle.solve_factored(f, a * V[:1] + b * V[1:2])["I"]
        np.testing.assert_allclose(lin, a * out["I"][:1] + b * out["I"][1:2], rtol=1e-11,
                                   atol=1e-14 * np.abs(out["I"]).max())
        Geff = oracle.transfer_matrix(f)
        np.testing.assert_allclose(V @ Geff, out["I"], rtol=1e-12)
        # reciprocity: unit current into WL(i,1) read at BL(M,j) equals the reverse
        k = 2 * M * N
        for (i, j) in [(0, 0), (M - 1, N - 1), (M // 2, N // 3)]:
            wi, uj = 2 * (i * N), 2 * ((M - 1) * N + j) + 1
            e = np.zeros((2, k))
            e[0, wi] = 1.0
            e[1, uj] = 1.0
            x = oracle.solve_band(f.lu, f.p, e)
            np.testing.assert_allclose(x[0, uj], x[1, wi], rtol=1e-12)


def pin_max_principle_rayleigh():
    """0 <= node voltages <= max V; with equal inputs the total current falls as wires lengthen."""
    rng = np.random.default_rng(7)
    M, N = 9, 11
    G = np.exp(rng.uniform(np.log(1e-6), np.log(1e-3), size=(M, N)))
    V = rng.uniform(0, 0.5, size=(5, M))
    out = oracle.solve(M, N, G, 1.0, 2.0, 2.0, 10.0, V, voltages=True)
    for b in range(5):
        assert out["vWL"][b].min() >= 0 and out["vBL"][b].min() >= 0
        assert out["vWL"][b].max() <= V[b].max() * (1 + 1e-14)
        assert out["vBL"][b].max() <= V[b].max() * (1 + 1e-14)
    Vc = np.full((1, M), 0.3)
    prev = np.inf
    for r in [0.01, 0.1, 1.0, 10.0, 100.0]:
        tot = oracle.solve(M, N, G, 1e-3, r, r, 1e-3, Vc)["I"].sum()
        assert tot <= 0.3 * G.sum() * (1 + 1e-12)
        assert tot < prev
        prev = tot


def pin_zero_parasitic_limit():
    """With every parasitic R = eps the currents tend to the ideal MVM sum_i V_i G_ij at first order."""
    rng = np.random.default_rng(8)
    M, N = 8, 6
    G = np.exp(rng.uniform(np.log(1e-6), np.log(1e-4), size=(M, N)))
    V = rng.uniform(0.05, 0.5, size=(2, M))
    ideal = V @ G
    devs = []
    for eps in [1e-1, 1e-2, 1e-3]:
        I = oracle.solve(M, N, G, eps, eps, eps, eps, V)["I"]
        dev = np.max(np.abs(I / ideal - 1.0))
        assert dev <= eps * (M + N + 2) * max(M, N) * G.max()
        devs.append(dev)
    rates = [devs[0] / devs[1], devs[1] / devs[2]]
    for r in rates:
        assert 9.0 < r < 11.0, rates


def pin_voltage_layout():
    """vWL[b, i, j] and vBL[b, i, j] are the word-line and bit-line voltages of row i, column j.

    Read against the stamp assembly's own numbering (word-line node i*N+j, bit-line node
    MN + i*N+j, before its permutation), on crossbars with M != N so that a transposed or
    swapped layout changes the values.
    """
    rng = np.random.default_rng(9)
    for M, N in [(3, 5), (4, 2)]:
        G, R = rand_case(rng, M, N)
        V = rng.uniform(0.05, 0.5, size=(2, M))
        out = oracle.solve(M, N, G, *R, V, voltages=True)
        assert out["vWL"].shape == (2, M, N) and out["vBL"].shape == (2, M, N)
        for b in range(2):
            As, bs = stamp_dense(M, N, G, *R, V=V[b])
            x = np.linalg.solve(As, bs)
            for i in range(M):
                for j in range(N):
                    np.testing.assert_allclose(out["vWL"][b, i, j], x[2 * (i * N + j)], rtol=1e-12)
                    np.testing.assert_allclose(out["vBL"][b, i, j], x[2 * (i * N + j) + 1], rtol=1e-12)
            # physical orientation: the source end of word line i is column 0; the sense end of
            # bit line j is row M-1
            np.testing.assert_allclose((V[b] - out["vWL"][b, :, 0]) / R[0], out["Isrc"][b], rtol=1e-12)
            np.testing.assert_allclose(out["vBL"][b, M - 1, :] / R[3], out["I"][b], rtol=1e-12)


ALL_PINS = [pin_counts, pin_stamp_assembly, pin_paper_equations, pin_dense_bruteforce,
            pin_closed_forms, pin_kirchhoff_linearity_reciprocity, pin_max_principle_rayleigh,
            pin_zero_parasitic_limit, pin_voltage_layout]
