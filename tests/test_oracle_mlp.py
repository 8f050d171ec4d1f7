"""Pins of the CPU surrogate oracle (oracle/mlp.py) against facts that do not come from it.

* bfloat16 rounding: against torch's float32 -> bfloat16 conversion and hand-worked ties;
* features: a hand-written 2 x 3 example (suffix row sums included);
* line model: exact against the nodal oracle when either set of lines is ideal (word lines, or
  bit lines plus sense resistor, at 1e-7 ohm), the 1 x 1 closed form, 0 < T_line < G, and with
  more passes monotone convergence to the nodal oracle's exact transfer matrix;
* target: the 1 x 1 crossbar closed forms (source, device and sense resistor in series for the
  exact current; the two one-line solves for the line model) through the nodal oracle, and the
  zero-parasitic limit where exact, line-model and ideal currents coincide;
* forward wiring: a one-path network evaluated by hand (catches transposed or swapped weights);
* backward: central finite differences of the FP64 loss with the log target held fixed.

The mutant test plants plausible mistakes in copies of mlp.py and requires a pin to fail on each.
"""
import types

import numpy as np
import pytest

import oracle
from oracle import mlp as MLP

SRC = open(MLP.__file__).read()


# ---- pins (each takes the module under test) -----------------------------------------------------
def pin_bf16(m):
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(1)
    a = np.concatenate([rng.normal(0, 1, 2000), rng.normal(0, 1e-3, 200), rng.normal(0, 1e4, 200),
                        [0.0, -0.0, 1.0, -2.5, 3.0e38]]).astype(np.float32)
    ref = torch.from_numpy(a).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(m.bf16_round(a), ref)
    # ties: half an ulp (2^-8 at 1.0) rounds to the even neighbour
    assert m.bf16_round(np.float32(1 + 2 ** -8)) == 1.0
    assert m.bf16_round(np.float32(1 + 3 * 2 ** -8)) == 1 + 2 ** -6
    assert m.bf16_round(np.float32(-(1 + 3 * 2 ** -8))) == -(1 + 2 ** -6)
    assert m.bf16_round(np.float32(1 + 2 ** -8 + 2 ** -20)) == 1 + 2 ** -7


def pin_features(m):
    G = np.array([[1e-5, 2e-5, 4e-5],
                  [3e-5, 5e-5, 1e-4]])
    V = np.array([[0.1, 0.4], [0.2, 0.0]])
    X = m.features(G, V, g_scale=1e-4, v_scale=0.5)
    # suffix row sums S(:, j) = sum over l >= j, divided by N g_scale = 3e-4
    S = [[7e-5 / 3e-4, 1.8e-4 / 3e-4], [6e-5 / 3e-4, 1.5e-4 / 3e-4], [4e-5 / 3e-4, 1e-4 / 3e-4]]
    expect = np.array([
        [0.1, 0.3, 0.2, 0.8] + S[0],   # b = 0, j = 0
        [0.2, 0.5, 0.2, 0.8] + S[1],   # b = 0, j = 1
        [0.4, 1.0, 0.2, 0.8] + S[2],   # b = 0, j = 2
        [0.1, 0.3, 0.4, 0.0] + S[0],   # b = 1, j = 0
        [0.2, 0.5, 0.4, 0.0] + S[1],
        [0.4, 1.0, 0.4, 0.0] + S[2],
    ])
    np.testing.assert_allclose(X, expect, rtol=1e-14, atol=0)
    np.testing.assert_allclose(m.ideal_currents(G, V), V @ G, rtol=1e-15)


def _nodal_transfer(G, circuit):
    M, N = G.shape
    return oracle.transfer_matrix(oracle.factor(M, N, G, *circuit))


def pin_line_model(m):
    rng = np.random.default_rng(2)
    G = np.exp(rng.uniform(np.log(1e-6), np.log(1e-4), (6, 5)))
    tiny = 1e-7
    # word lines ideal: the line model is exact (only the independent bit-line chains remain)
    c = (tiny, tiny, 2.5, 10.0)
    np.testing.assert_allclose(m.line_model(G, *c)[1], _nodal_transfer(G, c), rtol=1e-6)
    # bit lines ideal: exact as well (only the independent word-line chains remain)
    c = (1.0, 2.5, tiny, tiny)
    np.testing.assert_allclose(m.line_model(G, *c)[1], _nodal_transfer(G, c), rtol=1e-6)
    # both lines resistive: each line only loses voltage (0 < tau < 1, 0 < g_o x < 1)
    Tl = m.line_model(G, 1.0, 2.5, 2.5, 10.0)[1]
    assert np.all(Tl < G) and np.all(Tl > 0.0)
    # 1 x 1: tau = g_s/(g_s + G), x = 1/(G + g_o)
    g, Rs, Rse = 3e-4, 2.0, 30.0
    gs, go = 1 / Rs, 1 / Rse
    tau, Tl = m.line_model(np.array([[g]]), Rs, 5.0, 7.0, Rse)
    np.testing.assert_allclose(tau, gs / (gs + g), rtol=1e-14)
    np.testing.assert_allclose(Tl, g * gs * go / ((gs + g) * (g + go)), rtol=1e-14)
    # more passes: block Gauss-Seidel converges to the nodal solution
    G = np.exp(rng.uniform(np.log(1e-6), np.log(1e-4), (12, 10)))
    c = (1.0, 2.5, 2.5, 10.0)
    T = _nodal_transfer(G, c)
    errs = [np.max(np.abs(m.line_model(G, *c, passes=p)[1] / T - 1)) for p in (1, 2, 3, 6)]
    assert errs[0] > errs[1] > errs[2] > errs[3] and errs[3] < 1e-10, errs
    # heavier load (larger devices): slower contraction, same limit
    G = np.exp(rng.uniform(np.log(1e-4), np.log(1e-3), (8, 8)))
    T = _nodal_transfer(G, c)
    errs = [np.max(np.abs(m.line_model(G, *c, passes=p)[1] / T - 1)) for p in (1, 2, 4, 12)]
    assert errs[0] > errs[1] > errs[2] > errs[3] and errs[3] < 1e-9, errs
    # suffix row sums by hand
    np.testing.assert_allclose(m.suffix_row_sums(np.array([[1.0, 2.0, 4.0], [8.0, 16.0, 32.0]])),
                               [[7.0, 6.0, 4.0], [56.0, 48.0, 32.0]])


def pin_target_closed_forms(m):
    # 1 x 1 through the nodal oracle: I = V / (R_s + 1/G + R_sense)
    g, Rs, Rse = 2e-4, 3.0, 40.0
    gs, go = 1 / Rs, 1 / Rse
    G = np.array([[g]])
    V = np.array([[0.3], [0.05]])
    c = (Rs, 7.0, 11.0, Rse)
    I = oracle.solve(1, 1, G, *c, V)["I"]
    q = m.targets(G, V, I, c)
    expect = gs * go / (gs * go + g * go + g * gs) - gs * go / ((gs + g) * (g + go))
    np.testing.assert_allclose(q, expect, rtol=1e-9)
    # zero-parasitic limit: exact, line model and ideal currents coincide
    rng = np.random.default_rng(2)
    G = np.exp(rng.uniform(np.log(1e-6), np.log(1e-4), (4, 3)))
    V = rng.uniform(0, 0.5, (2, 4))
    r = 1e-9
    I = oracle.solve(4, 3, G, r, r, r, r, V)["I"]
    assert np.max(np.abs(m.targets(G, V, I, (r, r, r, r)))) < 1e-10


def pin_forward_wiring(m):
    M = 3
    P = np.zeros(m.n_params(M))
    W1, b1, W2, b2, W3, b3 = m.unpack(P, M)
    # one path: feature 4 -> hidden1 unit 2 -> hidden2 unit 5 -> output 0 (and output 1 via b3)
    W1[2, 4] = 2.0
    b1[2] = -0.5
    W2[5, 2] = 3.0
    b2[5] = 0.25
    W3[0, 5] = -1.5
    W3[1, 5] = 0.5
    b3[:] = [0.125, -1.0]
    X = np.zeros((3, 3 * M))
    X[0, 4] = 1.0    # h1 = relu(2 - 0.5) = 1.5, h2 = relu(4.5 + 0.25) = 4.75
    X[1, 4] = 0.1    # h1 = relu(0.2 - 0.5) = 0,   h2 = 0.25
    X[2, 3] = 5.0    # other feature: h1 = 0, h2 = 0.25
    n, _ = m.forward(P, X, M)
    np.testing.assert_allclose(n[:, 0], [0.125 - 1.5 * 4.75, 0.125 - 1.5 * 0.25, 0.125 - 1.5 * 0.25])
    np.testing.assert_allclose(n[:, 1], [-1.0 + 0.5 * 4.75, -1.0 + 0.5 * 0.25, -1.0 + 0.5 * 0.25])


def pin_gradient_fd(m):
    M, R = 5, 9
    rng = np.random.default_rng(3)
    P = m.init_params(M, seed=4).astype(np.float64)
    X = rng.uniform(0, 1, (R, 3 * M))
    y = rng.normal(0.3, 0.2, R)
    mu, sigma = 0.2, 0.5
    (l0, l1), g, t = m.loss_and_grad(P, X, y, M, mu, sigma)

    def L(Q):
        (a, b), _, _ = m.loss_and_grad(Q, X, y, M, mu, sigma, t=t)
        return a + m.LAMBDA * b

    W1n = m.H * m.padded_features(M)
    F = 3 * M
    blocks = {"W1": [o * m.padded_features(M) + i for o in rng.integers(0, m.H, 8) for i in rng.integers(0, F, 2)],
              "b1": list(W1n + rng.integers(0, m.H, 10)),
              "W2": list(W1n + m.H + rng.integers(0, m.H * m.H, 20)),
              "b2": list(W1n + m.H + m.H * m.H + rng.integers(0, m.H, 10)),
              "W3": list(W1n + 2 * m.H + m.H * m.H + rng.integers(0, 2 * m.H, 20)),
              "b3": [P.size - 2, P.size - 1]}
    h = 1e-6
    scale = np.max(np.abs(g))
    for name, idx in blocks.items():
        for k in idx:
            Q1, Q2 = P.copy(), P.copy()
            Q1[k] += h
            Q2[k] -= h
            fd = (L(Q1) - L(Q2)) / (2 * h)
            assert abs(fd - g[k]) <= 1e-6 * scale + 1e-6 * abs(fd), (name, k, fd, g[k])
    # padding columns of W1 see zero features: zero gradient
    Fp = m.padded_features(M)
    gW1 = g[:W1n].reshape(m.H, Fp)
    assert np.all(gW1[:, F:] == 0.0)


def pin_predict_closed_form(m):
    M, N = 2, 3
    P = np.zeros(m.n_params(M))
    b3 = m.unpack(P, M)[5]
    b3[:] = [0.5, np.log(0.02)]            # n0 = 0.5, n1 = log 0.02 for every row
    G = np.array([[1e-5, 2e-5, 3e-5], [4e-5, 5e-5, 6e-5]])
    V = np.array([[0.1, 0.2]])
    r = 1e-9                               # line model = ideal currents up to ~1e-13
    I, est = m.predict(P, G, V, (r, r, r, r), 1e-4, 0.5, mu=-0.3, sigma=0.2, c=1.5)
    q = -0.3 + 0.2 * 0.5
    np.testing.assert_allclose(I, (V @ G) * (1 + q), rtol=1e-10)
    np.testing.assert_allclose(est, 1.5 * 0.2 * 0.02 / abs(1 + q), rtol=1e-10)


PINS = [pin_bf16, pin_features, pin_line_model, pin_target_closed_forms, pin_forward_wiring,
        pin_gradient_fd, pin_predict_closed_form]


@pytest.mark.parametrize("pin", PINS, ids=[p.__name__ for p in PINS])
def test_pin(pin):
    pin(MLP)


def test_bf16_mode_is_close_to_fp64():
    M, R = 40, 64
    rng = np.random.default_rng(5)
    P = MLP.init_params(M, seed=6)
    X = rng.uniform(0, 1, (R, 3 * M))
    y = rng.normal(0, 1, R)
    (a0, a1), ga, _ = MLP.loss_and_grad(P, X, y, M)
    (b0, b1), gb, _ = MLP.loss_and_grad(P, X, y, M, precision="bf16")
    assert abs(a0 - b0) <= 2e-2 * a0
    assert np.linalg.norm(ga - gb) <= 5e-2 * np.linalg.norm(ga)


# ---- mutants ------------------------------------------------------------------------------------
MUTANTS = {
    "bf16_truncates": ("u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000", "u = u & 0xFFFF0000"),
    "feature_suffix_not_normalised_by_N": ("X[r, 2 * M:] = S[:, j] / (N * g_scale)", "X[r, 2 * M:] = S[:, j] / g_scale"),
    "feature_column_is_row": ("X[r, :M] = G[:, j] / g_scale", "X[r, :M] = G[j % M, :M] / g_scale"),
    "suffix_sums_wrong_direction": ("S[:, j] = G[:, j:].sum(axis=1)", "S[:, j] = G[:, :j + 1].sum(axis=1)"),
    "wl_source_at_far_end": ("A[0, 0] += gs", "A[N - 1, N - 1] += gs"),
    "bl_sense_at_top": ("A[M - 1, M - 1] += go", "A[0, 0] += go"),
    "line_model_ignores_bl_voltage": ("rhs = G[i] * u[i]", "rhs = G[i] * 0.0"),
    "line_model_bl_not_driven_by_w": ("u[:, j] = bl_inv[j] @ (G[:, j] * w[:, j])",
                                      "u[:, j] = bl_inv[j] @ (G[:, j] * w[:, 0])"),
    "line_model_source_row_wrong": ("                if i == k:", "                if i == 0:"),
    "target_wrong_denominator": ("- line_currents(G, V, circuit, passes)) / Iid)",
                                 "- line_currents(G, V, circuit, passes)) / np.asarray(I))"),
    "target_from_ideal": ("return ((np.asarray(I, dtype=np.float64) - line_currents(G, V, circuit, passes)) / Iid)",
                          "return ((np.asarray(I, dtype=np.float64) - Iid) / Iid)"),
    "w1_transposed_use": ("Z1 = Xp @ W1e.T + b1", "Z1 = Xp @ W1e.T[:, ::-1] + b1"),
    "no_second_relu": ("H2 = rnd(np.maximum(Z2, 0.0))", "H2 = rnd(Z2)"),
    "backward_missing_mask": ("dZ1 = rnd((dZ2 @ c[\"W2\"]) * (c[\"H1\"] > 0))", "dZ1 = rnd(dZ2 @ c[\"W2\"])"),
    "backward_wrong_lambda": ("2.0 * LAMBDA * e1 / R", "2.0 * e1 / R"),
    "bias_grad_from_wrong_layer": ("gb1 = dZ1.sum(axis=0)", "gb1 = dZ2.sum(axis=0)"),
    "predict_sigma_dropped": ("I = line_currents(G, V, circuit, passes).reshape(-1) + Iid * (mu + sigma * n[:, 0])",
                              "I = line_currents(G, V, circuit, passes).reshape(-1) + Iid * (mu + n[:, 0])"),
    "estimate_not_relative": ("est = c * sigma * np.exp(n[:, 1]) * np.abs(Iid) / np.abs(I)",
                              "est = c * sigma * np.exp(n[:, 1]) * np.abs(Iid)"),
}


def _load_mutant(name, src):
    mod = types.ModuleType(f"mlp_mutant_{name}")
    mod.__file__ = f"<mutant {name}>"
    exec(compile(src, mod.__file__, "exec"), mod.__dict__)
    return mod


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name):
    old, new = MUTANTS[name]
    assert SRC.count(old) == 1, f"mutation site for {name} not found exactly once"
    mod = _load_mutant(name, SRC.replace(old, new))
    failed = []
    for pin in PINS:
        try:
            pin(mod)
        except (AssertionError, ValueError, IndexError):
            failed.append(pin.__name__)
    assert failed, f"mutant {name} survived every pin"
