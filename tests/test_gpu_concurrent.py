"""Two crossbar handles used concurrently from two host threads on two CUDA streams.

One thread sets the conductances of the next map and factors it (Sec. II-C: one decomposition
per conductance map) while the other solves a batch with the map factored before it, so the
factor kernels run beside the other handle's sweeps, residuals and updates on shared SMs.  Every
step's currents must equal, bit for bit, those of the same map solved on an idle GPU: the kernels
and their inputs are the same, only their placement and timing differ.  At 256 x 256 with 8192
vectors this schedule exposed a missing barrier in the cluster factor (a warp could overwrite
shared-memory rows of X_{j-1} before another warp had stored them), which no single-stream test
reached.  Waits are bounded so that a failing step fails the test instead of hanging it.
"""
import threading

import pytest

from paper_2410_19993_gb300 import inputs, xbar

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

R = (1.0, 1.0, 1.0, 10.0)
TIMEOUT_S = 60.0


def _pipelined(M, N, B, precision, steps, tol=1e-8):
    G, V = inputs.crossbar(M, N, B, seed=0)
    Gd, Vd = torch.from_numpy(G).cuda(), torch.from_numpy(V).cuda()
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    h = [xbar.Crossbar.assemble(Gd, *R, stream=s) for s in streams]
    ref = torch.zeros((B, N), dtype=torch.float64, device="cuda")
    h[0].factor(precision)
    h[0].solve(Vd, ref, tol=tol)  # idle GPU: nothing else runs
    h[0].sync()
    out = [torch.zeros((B, N), dtype=torch.float64, device="cuda") for _ in range(steps)]
    factored = [threading.Semaphore(0) for _ in range(steps + 1)]
    done = [threading.Semaphore(0) for _ in range(steps + 1)]
    errors = []

    def factor_thread():
        try:
            for k in range(1, steps + 1):
                if k >= 2 and not done[k - 2].acquire(timeout=TIMEOUT_S):
                    errors.append(f"step {k}: solve {k - 2} did not finish")
                    return
                x = h[k % 2]
                x.set_conductances(Gd)
                x.factor(precision)
                x.sync()
                factored[k].release()
        except Exception as e:  # reported by the main thread
            errors.append(repr(e))

    h[0].set_conductances(Gd)
    h[0].factor(precision)
    h[0].sync()
    factored[0].release()
    th = threading.Thread(target=factor_thread, daemon=True)
    th.start()
    try:
        for k in range(steps):
            assert factored[k].acquire(timeout=TIMEOUT_S), f"factor of step {k} did not finish: {errors}"
            h[k % 2].solve(Vd, out[k], tol=tol)
            done[k].release()
    finally:
        th.join(timeout=TIMEOUT_S)
        torch.cuda.synchronize()
        for x in h:
            x.destroy()
    assert not errors, errors
    return ref, out


@pytest.mark.parametrize("precision", ["fp32_ir", "fp64"])
def test_factor_beside_solve_of_another_map(precision):
    steps = 6 if precision == "fp32_ir" else 3
    ref, out = _pipelined(256, 256, 8192, precision, steps)
    for k, I in enumerate(out):
        assert torch.equal(I, ref), f"step {k}: max |dI| = {float((I - ref).abs().max())}"


def test_factor_beside_solve_small_map():
    ref, out = _pipelined(64, 48, 2048, "fp32_ir", 6)
    for k, I in enumerate(out):
        assert torch.equal(I, ref), f"step {k}"
