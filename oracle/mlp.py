"""CPU oracle of the per-column crossbar surrogate (forward, loss, backward), plain numpy.

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle/``: the tests, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` are its only callers; the product library never imports
it and it imports nothing from the product.

What it computes (the definition the GPU kernels implement):

* the line model of a map (a cheap physical estimate the network corrects): every word line is
  solved alone with the bit lines held at ground (source R_s, segments R_w, device conductances to
  ground), which gives the word-line voltage ratios tau[i, j] = v_WL(i, j) / V_i; then every bit
  line is solved alone with device i driven by the voltage V_i tau[i, j] (segments R_b, top open,
  R_sense to ground at the bottom, Sec. II-A Eqs. 1-7 restricted to one line).  Further passes
  solve the word lines again with their devices tied to the bit-line voltages just found, then
  the bit lines again (block Gauss-Seidel between the two sets of lines, which converges to the
  exact solution).  The result is linear in V: I_line = V @ T_line; after one pass
  T_line[i, j] = tau[i, j] G[i, j] g_o x_j[i], where x_j solves bit line j's chain for a unit
  current injected at its bottom node;
* features of bit line j of map G (M x N) for input vector V (length M), one row per (b, j),
  r = b*N + j:  x = [G(:, j)/g_scale, V/v_scale, S(:, j)/(N g_scale)]  (3M values), where
  S[i, j] = sum_{l >= j} G[i, l] are the row sums of G taken from column j to the open end (the
  load each word line still carries at column j);
* target: with the ideal currents I_ideal = V @ G (every wire resistance at zero) and the line
  model's currents I_line, the network's regression target is the line model's error relative
  to the ideal current, q = (I - I_line) / I_ideal; the predicted deviation from the ideal MVM is
  (I_line - I_ideal)/I_ideal + q;
* network 3M -> 256 -> 256 -> 2, ReLU after the two hidden layers, flat parameter vector
  [W1 (256 x Fp), b1, W2 (256 x 256), b2, W3 (2 x 256), b3] with Fp = 3M rounded up to 128 (the
  padding columns of W1 multiply zero features); W[o, i] maps input i to output o;
* loss per row: (n0 - qh)^2 + lam (n1 - t)^2 with qh = (q - mu)/sigma and t = log(|n0 - qh| + eps)
  held constant (not differentiated); both terms averaged over the rows;
* prediction: I = I_line + I_ideal (mu + sigma n0), relative-error estimate
  c sigma exp(n1) |I_ideal| / |I|.

``precision="fp64"`` evaluates all of it in float64.  ``precision="bf16"`` rounds to bfloat16
(round to nearest, ties to even) at the points where the GPU kernels store bfloat16: the features
(through float32), the weights W1 and W2, the hidden activations H1 and H2, and the back-propagated
gradients dZ2 and dZ1 fed to the products; everything else stays float64.  The two differ by the
bfloat16 rounding alone, which bounds what the GPU comparison may tolerate in each mode.
"""
from __future__ import annotations

import numpy as np

H = 256
LAMBDA = 0.1
EPS = 1e-6


def bf16_round(a) -> np.ndarray:
    """Round float32 values to the nearest bfloat16 (ties to even), returned as float64.

    bfloat16 keeps the top 16 bits of the float32 pattern; rounding adds 0x7FFF plus the lowest
    kept bit before truncating, which is round-to-nearest-even on the dropped 16 bits.
    """
    f = np.ascontiguousarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def padded_features(M: int) -> int:
    return ((3 * M + 127) // 128) * 128


def n_params(M: int) -> int:
    Fp = padded_features(M)
    return H * Fp + H + H * H + H + 2 * H + 2


def unpack(P, M: int):
    """Split the flat parameter vector into (W1, b1, W2, b2, W3, b3) as float64 views."""
    P = np.asarray(P, dtype=np.float64)
    Fp = padded_features(M)
    sizes = [H * Fp, H, H * H, H, 2 * H, 2]
    shapes = [(H, Fp), (H,), (H, H), (H,), (2, H), (2,)]
    out, o = [], 0
    for n, sh in zip(sizes, shapes):
        out.append(P[o:o + n].reshape(sh))
        o += n
    assert o == P.size, "parameter vector has the wrong length"
    return out


def _wl_matrix(G, i, gs, gw):
    """Word line i alone: source conductance at column 0, segments gw, devices to a fixed node."""
    N = G.shape[1]
    A = np.diag(G[i].copy())
    A[0, 0] += gs
    for j in range(N - 1):
        A[j, j] += gw
        A[j + 1, j + 1] += gw
        A[j, j + 1] -= gw
        A[j + 1, j] -= gw
    return A


def _bl_matrix(G, j, gb, go):
    """Bit line j alone: top (row 0) open, segments gb, sense conductance to ground at row M-1."""
    M = G.shape[0]
    A = np.diag(G[:, j].copy())
    A[M - 1, M - 1] += go
    for i in range(M - 1):
        A[i, i] += gb
        A[i + 1, i + 1] += gb
        A[i, i + 1] -= gb
        A[i + 1, i] -= gb
    return A


def line_model(G, Rs: float, Rw: float, Rb: float, Rsense: float, passes: int = 1):
    """(tau, T_line): P passes of the line model, T_line[k, j] = I_j for the unit input V = e_k.

    Pass p solves every word line alone, its devices tied to the bit-line voltages u of pass p-1
    (u = 0 before the first pass), then every bit line alone, its devices driven by the new
    word-line voltages; the last pass keeps only the sense currents.  This is block Gauss-Seidel
    on the nodal equations (Eqs. 1-7) split into word-line and bit-line unknowns, started from
    grounded bit lines; it converges to the exact currents as passes grow.  tau[i, j] is the
    word-line voltage ratio of the first pass.  Each line's system is built and solved densely.
    """
    G = np.asarray(G, dtype=np.float64)
    M, N = G.shape
    gs, gw, gb, go = 1.0 / Rs, 1.0 / Rw, 1.0 / Rb, 1.0 / Rsense
    wl_inv = [np.linalg.inv(_wl_matrix(G, i, gs, gw)) for i in range(M)]
    bl_inv = [np.linalg.inv(_bl_matrix(G, j, gb, go)) for j in range(N)]
    tau = np.stack([wl_inv[i][:, 0] * gs for i in range(M)])
    T = np.empty((M, N))
    for k in range(M):
        u = np.zeros((M, N))
        for p in range(passes):
            w = np.empty((M, N))
            for i in range(M):
                rhs = G[i] * u[i]
                if i == k:
                    rhs[0] += gs
                w[i] = wl_inv[i] @ rhs
            u = np.empty((M, N))
            for j in range(N):
                u[:, j] = bl_inv[j] @ (G[:, j] * w[:, j])
        T[k] = go * u[M - 1]
    return tau, T


def suffix_row_sums(G) -> np.ndarray:
    """S[i, j] = sum over l >= j of G[i, l]."""
    G = np.asarray(G, dtype=np.float64)
    M, N = G.shape
    S = np.zeros((M, N))
    for j in range(N):
        S[:, j] = G[:, j:].sum(axis=1)
    return S


def features(G, V, g_scale: float, v_scale: float) -> np.ndarray:
    """X[(b*N + j), :] = [G(:, j)/g_scale, V_b/v_scale, S(:, j)/(N g_scale)], shape (B*N, 3M)."""
    G = np.asarray(G, dtype=np.float64)
    V = np.atleast_2d(np.asarray(V, dtype=np.float64))
    M, N = G.shape
    B = V.shape[0]
    S = suffix_row_sums(G)
    X = np.empty((B * N, 3 * M))
    for b in range(B):
        for j in range(N):
            r = b * N + j
            X[r, :M] = G[:, j] / g_scale
            X[r, M:2 * M] = V[b] / v_scale
            X[r, 2 * M:] = S[:, j] / (N * g_scale)
    return X


def ideal_currents(G, V) -> np.ndarray:
    """I_ideal[b, j] = sum_i V[b, i] G[i, j]: the currents with every parasitic resistance at zero."""
    return np.atleast_2d(np.asarray(V, dtype=np.float64)) @ np.asarray(G, dtype=np.float64)


def line_currents(G, V, circuit, passes: int = 1) -> np.ndarray:
    """I_line = V @ T_line for circuit = (R_s, R_w, R_b, R_sense)."""
    return np.atleast_2d(np.asarray(V, dtype=np.float64)) @ line_model(G, *circuit, passes=passes)[1]


def targets(G, V, I, circuit, passes: int = 1) -> np.ndarray:
    """q[(b*N + j)] = (I[b, j] - I_line[b, j]) / I_ideal[b, j]."""
    Iid = ideal_currents(G, V)
    return ((np.asarray(I, dtype=np.float64) - line_currents(G, V, circuit, passes)) / Iid).reshape(-1)


def _prep_x(X, M, precision):
    Fp = padded_features(M)
    Xp = np.zeros((X.shape[0], Fp))
    Xp[:, :X.shape[1]] = X
    if precision == "bf16":
        Xp = bf16_round(Xp)
    return Xp


def forward(P, X, M: int, precision: str = "fp64"):
    """Network outputs n (R x 2) for features X (R x 3M) and the intermediates of the pass."""
    W1, b1, W2, b2, W3, b3 = unpack(P, M)
    Xp = _prep_x(np.asarray(X, dtype=np.float64), M, precision)
    rnd = bf16_round if precision == "bf16" else (lambda a: a)
    W1e, W2e = rnd(W1), rnd(W2)
    Z1 = Xp @ W1e.T + b1
    H1 = rnd(np.maximum(Z1, 0.0))
    Z2 = H1 @ W2e.T + b2
    H2 = rnd(np.maximum(Z2, 0.0))
    n = H2 @ W3.T + b3
    return n, dict(X=Xp, W1=W1e, W2=W2e, H1=H1, H2=H2)


def loss_and_grad(P, X, y, M: int, mu: float = 0.0, sigma: float = 1.0, precision: str = "fp64",
                  t=None):
    """(loss0, loss1), flat gradient of loss0 + LAMBDA*loss1, and the log target t used.

    loss0 = mean (n0 - yh)^2, loss1 = mean (n1 - t)^2, yh = (y - mu)/sigma; t defaults to
    log(|n0 - yh| + EPS) at P and is a constant of the loss (pass it to evaluate the same loss
    at other parameters, as a finite-difference check must).
    """
    W1, b1, W2, b2, W3, b3 = unpack(P, M)
    n, c = forward(P, X, M, precision)
    R = n.shape[0]
    yh = (np.asarray(y, dtype=np.float64) - mu) / sigma
    e0 = n[:, 0] - yh
    if t is None:
        t = np.log(np.abs(e0) + EPS)
    e1 = n[:, 1] - t
    loss = (float(np.mean(e0 ** 2)), float(np.mean(e1 ** 2)))
    rnd = bf16_round if precision == "bf16" else (lambda a: a)
    # derivatives of the mean loss with respect to the two outputs
    d = np.stack([2.0 * e0 / R, 2.0 * LAMBDA * e1 / R], axis=1)       # R x 2
    gW3 = d.T @ c["H2"]
    gb3 = d.sum(axis=0)
    dZ2 = rnd((d @ W3) * (c["H2"] > 0))                                  # R x 256
    gW2 = dZ2.T @ c["H1"]
    gb2 = dZ2.sum(axis=0)
    dZ1 = rnd((dZ2 @ c["W2"]) * (c["H1"] > 0))
    gW1 = dZ1.T @ c["X"]
    gb1 = dZ1.sum(axis=0)
    g = np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gW3.ravel(), gb3])
    return loss, g, t


def predict(P, G, V, circuit, g_scale: float, v_scale: float, mu: float = 0.0, sigma: float = 1.0,
            c: float = 1.0, precision: str = "fp64", passes: int = 1):
    """(I_pred[B x N], relative-error estimate[B x N]) of the surrogate for map G and inputs V."""
    G = np.asarray(G, dtype=np.float64)
    V = np.atleast_2d(np.asarray(V, dtype=np.float64))
    M, N = G.shape
    X = features(G, V, g_scale, v_scale)
    if precision == "bf16":
        X = X.astype(np.float32).astype(np.float64)
    n, _ = forward(P, X, M, precision)
    Iid = ideal_currents(G, V).reshape(-1)
    I = line_currents(G, V, circuit, passes).reshape(-1) + Iid * (mu + sigma * n[:, 0])
    est = c * sigma * np.exp(n[:, 1]) * np.abs(Iid) / np.abs(I)
    return I.reshape(V.shape[0], N), est.reshape(V.shape[0], N)


def init_params(M: int, seed: int = 0, scale: float = 1.0) -> np.ndarray:
    """Random parameters for tests (He-scaled normal weights, small biases), float32."""
    rng = np.random.default_rng(seed)
    Fp = padded_features(M)
    F = 3 * M
    W1 = np.zeros((H, Fp))
    W1[:, :F] = rng.normal(0.0, np.sqrt(2.0 / F), size=(H, F))
    b1 = rng.normal(0.0, 0.05, size=H)
    W2 = rng.normal(0.0, np.sqrt(2.0 / H), size=(H, H))
    b2 = rng.normal(0.0, 0.05, size=H)
    W3 = rng.normal(0.0, np.sqrt(1.0 / H), size=(2, H))
    b3 = rng.normal(0.0, 0.1, size=2)
    P = np.concatenate([W1.ravel(), b1, W2.ravel(), b2, W3.ravel(), b3]) * scale
    return P.astype(np.float32)
