"""GPU tests of the learned surrogate (xbar_surrogate_*): kernels against the CPU oracle, then
training on solves of the exact method, calibration, and prediction with exact fallback.

The forward pass and the gradients are compared with oracle/mlp.py in its bf16 mode (which
rounds at the points the kernels store bfloat16, so the remaining difference is FP32 vs FP64
accumulation order plus rare one-ulp flips of a bfloat16 rounding), and with its fp64 mode at the
looser tolerance that bfloat16 rounding itself implies.
"""
import time

import numpy as np
import pytest

from oracle import mlp as MLP
from paper_2410_19993_gb300 import inputs, xbar
from tests.gpu_common import rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GS, VS = 1e-4, 0.5
CIRCUIT = (1.0, 2.5, 2.5, 10.0)   # R_s, R_w, R_b, R_sense of the surrogate workload


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _block_err(a, b, M):
    """Relative error of each parameter block (W1, b1, W2, b2, W3, b3)."""
    out = []
    for x, y in zip(MLP.unpack(a, M), MLP.unpack(b, M)):
        out.append(np.linalg.norm(x - y) / max(np.linalg.norm(y), 1e-30))
    return out


def test_params_roundtrip():
    s = xbar.Surrogate(40, 24, CIRCUIT, seed=3)
    P = MLP.init_params(40, seed=7)
    assert s.n_params() == P.size == MLP.n_params(40)
    s.set_params(P)
    np.testing.assert_array_equal(s.get_params(), P)
    assert s.scaling() == (0.0, 1.0, 1.0)
    assert s.scaling(mu=-0.3, sigma=0.2, c=2.0) == (-0.3, 0.2, 2.0)
    s.destroy()


@pytest.mark.parametrize("M,N,B,P", [(40, 24, 7, 1), (40, 24, 7, 2), (33, 50, 3, 3), (128, 128, 3, 2),
                                     (7, 5, 3, 4), (1, 1, 2, 2), (1, 9, 2, 2), (9, 1, 2, 3),
                                     (160, 160, 2, 2), (200, 90, 2, 3)])
def test_line_model_matches_oracle(M, N, B, P):
    """All-zero network parameters and mu = 0 leave the line model: I = I_line exactly.
    160 x 160 and 200 x 90 exceed the shared-memory form and run the global-memory kernels."""
    G, V = inputs.crossbar(M, N, B, seed=7 * M + N)
    s = xbar.Surrogate(M, N, CIRCUIT, passes=P)
    s.set_params(np.zeros(MLP.n_params(M), dtype=np.float32))
    I = np.zeros((B, N))
    s.predict(G, V, I)
    # the line model's chains run in FP32 over sums of positive terms: relative error below
    # (chain length) x (a few roundings) x 2^-24, i.e. < 3e-5 up to 128 nodes per line
    err = np.max(np.abs(I / MLP.line_currents(G, V, CIRCUIT, P) - 1))
    assert err <= 3e-5, err
    s.destroy()


@pytest.mark.parametrize("M,N,B", [(40, 24, 7), (128, 128, 3), (7, 5, 3)])
def test_forward_matches_oracle(M, N, B):
    G, V = inputs.crossbar(M, N, B, seed=M * N)
    P = MLP.init_params(M, seed=11)
    s = xbar.Surrogate(M, N, CIRCUIT)
    s.set_params(P)
    mu, sigma, c = -0.3, 0.2, 1.7
    s.scaling(mu, sigma, c)
    I = np.zeros((B, N))
    est = np.zeros((B, N))
    s.predict(G, V, I, est)
    Ib, eb = MLP.predict(P, G, V, CIRCUIT, GS, VS, mu, sigma, c, precision="bf16", passes=s.passes)
    Id, _ = MLP.predict(P, G, V, CIRCUIT, GS, VS, mu, sigma, c, precision="fp64", passes=s.passes)
    Iid = MLP.ideal_currents(G, V)
    # (I - I_line) / I_ideal = mu + sigma n0: compare n0 in absolute terms
    assert np.max(np.abs(I - Ib) / Iid) <= 1e-3 * sigma
    assert np.max(np.abs(est - eb) / eb) <= 1e-3
    assert np.max(np.abs(I - Id) / Iid) <= 5e-2 * sigma
    # device pointers give the same result
    Id_dev = torch.zeros((B, N), dtype=torch.float64, device="cuda")
    s.predict(_dev(G), _dev(V), Id_dev)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(Id_dev.cpu().numpy(), I)
    s.destroy()


@pytest.mark.parametrize("M,R", [(40, 300), (128, 1000), (7, 128)])
def test_gradient_matches_oracle(M, R):
    rng = np.random.default_rng(R)
    X = rng.uniform(0, 1, (R, 3 * M)).astype(np.float32)
    y = rng.normal(0.02, 0.01, R).astype(np.float32)
    P = MLP.init_params(M, seed=13)
    s = xbar.Surrogate(M, 16, CIRCUIT)
    s.set_params(P)
    mu, sigma = 0.02, 0.01
    s.scaling(mu, sigma)
    loss, g = s.grad(X, y)
    (b0, b1), gb, _ = MLP.loss_and_grad(P, X.astype(np.float64), y.astype(np.float64), M, mu, sigma,
                                        precision="bf16")
    (d0, d1), gd, _ = MLP.loss_and_grad(P, X.astype(np.float64), y.astype(np.float64), M, mu, sigma)
    assert abs(loss[0] - b0) <= 1e-4 * b0 and abs(loss[1] - b1) <= 1e-4 * b1
    for e in _block_err(g.astype(np.float64), gb, M):
        assert e <= 3e-3, _block_err(g.astype(np.float64), gb, M)
    for e in _block_err(g.astype(np.float64), gd, M):
        assert e <= 5e-2, _block_err(g.astype(np.float64), gd, M)
    s.destroy()


def test_errors():
    with pytest.raises(xbar.XbarError) as e:
        xbar.Surrogate(0, 4, CIRCUIT)
    assert e.value.status == xbar.XBAR_EINVAL
    with pytest.raises(xbar.XbarError) as e:
        xbar.Surrogate(4, 4, (1.0, 0.0, 2.5, 10.0))
    assert e.value.status == xbar.XBAR_EINVAL
    with pytest.raises(xbar.XbarError) as e:
        xbar.Surrogate(4, 4, CIRCUIT, passes=0)
    assert e.value.status == xbar.XBAR_EINVAL
    s = xbar.Surrogate(8, 4, CIRCUIT)
    G, V = inputs.crossbar(8, 4, 2, seed=1)
    with pytest.raises(xbar.XbarError) as e:
        s.train([G], [V], [np.zeros((2, 4))], epochs=1, batch_rows=100)
    assert e.value.status == xbar.XBAR_EINVAL
    with pytest.raises(xbar.XbarError):
        s.scaling(sigma=-1.0)
    xb = xbar.Crossbar.assemble(_dev(inputs.crossbar(9, 4, 1, seed=2)[0]), *CIRCUIT)
    Vd = torch.zeros((2, 9), dtype=torch.float64, device="cuda")
    Idev = torch.zeros((2, 4), dtype=torch.float64, device="cuda")
    st, _ = s.solve(xb, Vd, Idev, raise_on_error=False)   # 9 x 4 handle, 8 x 4 surrogate
    assert st == xbar.XBAR_EINVAL
    xb.destroy()
    xb = xbar.Crossbar.assemble(_dev(inputs.crossbar(8, 4, 1, seed=2)[0]), 1.0, 2.5, 2.5, 20.0)
    st, _ = s.solve(xb, Vd[:, :8].contiguous(), Idev, raise_on_error=False)   # other R_sense
    assert st == xbar.XBAR_EINVAL
    xb.destroy()
    s.destroy()


def _exact_currents(G, V):
    xb = xbar.Crossbar.assemble(_dev(G), *CIRCUIT)
    xb.factor("fp32_ir")
    I = torch.zeros((V.shape[0], G.shape[1]), dtype=torch.float64, device="cuda")
    xb.solve(_dev(V), I, tol=1e-10, max_iter=8)
    xb.sync()
    xb.destroy()
    return I.cpu().numpy()


@pytest.fixture(scope="module")
def trained():
    """A 128 x 128 surrogate trained on 96 maps x 25 vectors of exact solves."""
    M = N = 128
    train = inputs.maps(96, M, N, 25, seed=100)
    calib = inputs.maps(8, M, N, 50, seed=200)
    test = inputs.maps(4, M, N, 200, seed=300)
    Itrain = [_exact_currents(G, V) for G, V in train]
    Icalib = [_exact_currents(G, V) for G, V in calib]
    s = xbar.Surrogate(M, N, CIRCUIT, passes=2, g_scale=GS, v_scale=VS, seed=5)
    losses = s.train([G for G, _ in train], [V for _, V in train], Itrain, epochs=40, batch_rows=2048,
                     lr=1e-3, seed=9)
    c = s.calibrate([G for G, _ in calib], [V for _, V in calib], Icalib, quantile=0.99)
    yield s, losses, c, test
    s.destroy()


def test_training_reduces_loss(trained):
    s, losses, c, _ = trained
    print("epoch losses", losses[[0, 9, 19, 39]].tolist(), "c", c, "scaling", s.scaling())
    assert np.all(np.isfinite(losses))
    assert losses[-1, 0] < 0.2 * losses[0, 0]
    assert losses[-1, 1] < losses[0, 1]
    mu, sigma, _ = s.scaling()
    assert abs(mu) < 0.05 and 0.0 < sigma < 0.05   # the line model's error relative to the ideal current


def test_surrogate_beats_ideal_mvm_and_falls_back(trained):
    s, _, c, test = trained
    bound = 0.01
    tot_acc = tot_vec = tot_bad = 0
    errs_net, errs_ideal, errs_line = [], [], []
    t_sur = t_exact = 0.0
    for G, V in test:
        Iex = _exact_currents(G, V)
        errs_ideal.append(np.abs(MLP.ideal_currents(G, V) - Iex) / np.abs(Iex))
        errs_line.append(np.abs(MLP.line_currents(G, V, CIRCUIT, s.passes) - Iex) / np.abs(Iex))
        Ip = np.zeros_like(Iex)
        s.predict(G, V, Ip)
        errs_net.append(np.abs(Ip - Iex) / np.abs(Iex))
        # prediction with fallback, on device buffers
        xb = xbar.Crossbar.assemble(_dev(G), *CIRCUIT)
        Vd = _dev(V)
        Id = torch.zeros_like(torch.from_numpy(Iex)).cuda()
        est = torch.zeros_like(Id)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st, info = s.solve(xb, Vd, Id, bound=bound, err_est=est)
        torch.cuda.synchronize()
        t_sur += time.perf_counter() - t0
        t0 = time.perf_counter()
        xb.factor("fp32_ir")
        Ix = torch.zeros_like(Id)
        xb.solve(Vd, Ix, tol=1e-8)
        xb.sync()
        t_exact += time.perf_counter() - t0
        xb.destroy()
        I = Id.cpu().numpy()
        e = est.cpu().numpy()
        acc = np.all(e <= bound, axis=1)
        tot_vec += V.shape[0]
        tot_acc += int(acc.sum())
        assert info["n_fallback"] == int((~acc).sum())
        # fallback vectors carry the exact solution, accepted ones the network's
        if (~acc).any():
            assert rel_err(I[~acc], Iex[~acc]) <= 1e-8
        true = np.abs(I[acc] - Iex[acc]) / np.abs(Iex[acc])
        tot_bad += int((true > bound).sum())
    en, ei = np.concatenate(errs_net).ravel(), np.concatenate(errs_ideal).ravel()
    el = np.concatenate(errs_line).ravel()
    print(f"median rel error: network {np.median(en):.2e}, line model {np.median(el):.2e}, "
          f"ideal MVM {np.median(ei):.2e}; "
          f"p99 network {np.quantile(en, 0.99):.2e}; accepted {tot_acc}/{tot_vec} vectors; "
          f"accepted columns above the bound {tot_bad}; time surrogate {t_sur:.3f} s vs exact {t_exact:.3f} s")
    assert np.median(en) < 0.2 * np.median(el) and np.median(el) < np.median(ei)
    # calibrated at the 99th percentile: among accepted columns few exceed the bound
    assert tot_bad <= 0.02 * max(tot_acc, 1) * 128
