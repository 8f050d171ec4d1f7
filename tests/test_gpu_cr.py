"""GPU parity of the block-cyclic-reduction factor and substitution (XBAR_OPT_ALGORITHM = 1)
against the CPU FP64 oracle, element by element.

Same bars as the block-Thomas path: relative current error <= 1e-10 in XBAR_FP64 and <= 1e-8
after refinement in XBAR_FP32_IR; node voltages within the bar times max V.  The FP32 factor's
products run on the tensor cores (three-term BF16 split) when the blocks have at least 128 rows,
and on the CUDA cores when asked to (or below 128 rows); both engines are compared.
"""
import numpy as np
import pytest

import oracle
from paper_2410_19993_gb300 import inputs, xbar
from tests.gpu_common import case, oracle_factor, oracle_transfer, rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FP64_BAR = 1e-10
MIXED_BAR = 1e-8
IR_TOL = 1e-9


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _solve_cr(G, R, V, precision, products=1, voltages=False, tol=IR_TOL, max_iter=10, algorithm="cr"):
    M, N = G.shape
    B = V.shape[0]
    I = torch.zeros((B, N), dtype=torch.float64, device="cuda")
    vW = torch.zeros((B, M, N), dtype=torch.float64, device="cuda") if voltages else None
    vB = torch.zeros((B, M, N), dtype=torch.float64, device="cuda") if voltages else None
    xb = xbar.Crossbar.assemble(_dev(G), *R)
    xb.set_option("algorithm", algorithm)
    xb.set_option("cr_products", products)
    xb.factor(precision)
    _, info = xb.solve(_dev(V), I, vW, vB, tol=tol, max_iter=max_iter)
    xb.sync()
    out = {"I": I.cpu().numpy(), "info": info}
    if voltages:
        out["vWL"] = vW.cpu().numpy()
        out["vBL"] = vB.cpu().numpy()
    xb.destroy()
    return out


# ragged shapes: odd and even N (the last block of a level eliminated or kept), N = 1, M = 1,
# padded rows (M not a multiple of 16), 2 x 2 block inversion (Mp > 128, with a 16-row second block)
SHAPES = [(1, 1, 1), (1, 7, 5), (9, 1, 3), (5, 7, 37), (17, 33, 19), (33, 17, 200), (40, 3, 100),
          (3, 40, 9), (100, 20, 65), (40, 17, 50), (16, 64, 33), (130, 40, 33), (144, 9, 20)]


@pytest.mark.parametrize("M,N,B", SHAPES)
@pytest.mark.parametrize("precision,bar", [("fp64", FP64_BAR), ("fp32_ir", MIXED_BAR)])
def test_cr_ragged_against_oracle(M, N, B, precision, bar):
    G, V = case(M, N, B, None, seed=M * 1000 + N)
    R = (1.0, 2.0, 1.5, 10.0)
    ref = oracle.solve(M, N, G, *R, V, voltages=True)
    engines = [1, 0] if (precision == "fp32_ir" and M > 112) else [1]
    for products in engines:
        out = _solve_cr(G, R, V, precision, products=products, voltages=True)
        assert rel_err(out["I"], ref["I"]) <= bar, (products, rel_err(out["I"], ref["I"]))
        assert np.max(np.abs(out["vWL"] - ref["vWL"])) <= bar
        assert np.max(np.abs(out["vBL"] - ref["vBL"])) <= bar


def test_cr_xbar16_workload():
    w = inputs.WORKLOADS["xbar16_fp64"]
    G, V = inputs.workload_inputs("xbar16_fp64")
    R = w.circuits[0].as_tuple()
    ref = oracle.solve(w.M, w.N, G, *R, V, voltages=True)
    for precision, bar in (("fp64", FP64_BAR), ("fp32_ir", MIXED_BAR)):
        out = _solve_cr(G, R, V, precision, voltages=True)
        assert rel_err(out["I"], ref["I"]) <= bar
        assert np.max(np.abs(out["vWL"] - ref["vWL"])) <= 0.5 * bar


@pytest.mark.parametrize("r_wire", [0.5, 2.5, 10.0])
@pytest.mark.parametrize("precision,bar", [("fp64", FP64_BAR), ("fp32_ir", MIXED_BAR)])
def test_cr_xbar64_rsweep(r_wire, precision, bar):
    w = inputs.WORKLOADS["xbar64_rsweep_fp64"]
    G, V = inputs.workload_inputs("xbar64_rsweep_fp64")
    R = (1.0, r_wire, r_wire, 10.0)
    _, f = oracle_factor(w.M, w.N, R)
    ref = oracle.solve_factored(f, V, nthreads=0)
    out = _solve_cr(G, R, V, precision)
    err = rel_err(out["I"], ref["I"])
    assert err <= bar, err


def test_cr_agrees_with_block_thomas_on_one_handle():
    """Switching the algorithm on one handle refactors; both factorizations give the same currents."""
    G, V = case(72, 45, 130, None, seed=21)
    R = (1.0, 2.5, 2.5, 10.0)
    xb = xbar.Crossbar.assemble(_dev(G), *R)
    outs = {}
    for algo in ("thomas", "cr", "thomas", "cr"):
        xb.set_option("algorithm", algo)
        xb.factor("fp64")
        I = torch.zeros((130, 45), dtype=torch.float64, device="cuda")
        xb.solve(_dev(V), I)
        xb.sync()
        outs.setdefault(algo, []).append(I.cpu().numpy())
    xb.destroy()
    np.testing.assert_array_equal(outs["cr"][0], outs["cr"][1])
    np.testing.assert_array_equal(outs["thomas"][0], outs["thomas"][1])
    assert rel_err(outs["cr"][0], outs["thomas"][0]) <= 1e-12


def test_cr_new_conductances_and_repeated_solves():
    """The level plan is built once per shape; new maps and new batch sizes reuse or extend it."""
    M, N = 50, 31
    R = (1.0, 1.0, 1.0, 10.0)
    xb = xbar.Crossbar.assemble(_dev(case(M, N, 1, None, seed=1)[0]), *R)
    xb.set_option("algorithm", "cr")
    for seed, B in ((2, 7), (3, 40), (3, 7), (4, 1)):
        G, V = case(M, N, B, None, seed=seed)
        xb.set_conductances(_dev(G))
        for precision, bar in (("fp64", FP64_BAR), ("fp32_ir", MIXED_BAR)):
            xb.factor(precision)
            I = torch.zeros((B, N), dtype=torch.float64, device="cuda")
            xb.solve(_dev(V), I, tol=IR_TOL)
            xb.sync()
            ref = oracle.solve(M, N, G, *R, V)
            assert rel_err(I.cpu().numpy(), ref["I"]) <= bar
    xb.destroy()


def test_cr_zero_inputs_and_isolated_memristor():
    M, N = 12, 10
    R = (1.0, 1.0, 1.0, 10.0)
    G = np.zeros((M, N))
    G[3, 4] = 1e-2
    V = np.zeros((4, M))
    V[1] = 0.5
    V[2, 3] = 1.0
    ref = oracle.solve(M, N, G, *R, V)
    for precision in ["fp64", "fp32_ir"]:
        out = _solve_cr(G, R, V, precision)
        assert np.all(out["I"][0] == 0.0) and np.all(out["I"][3] == 0.0)
        nz = np.abs(ref["I"]) > 0
        assert np.max(np.abs(out["I"][nz] - ref["I"][nz]) / np.abs(ref["I"][nz])) <= MIXED_BAR


def test_cr_noalloc_refuses_cr_factorization():
    G, V = case(16, 16, 4, None)
    xb = xbar.Crossbar.assemble(_dev(G), 1.0, 1.0, 1.0, 10.0)
    xb.set_option("algorithm", "cr")
    xb.factor("fp64")
    I = torch.zeros((4, 16), dtype=torch.float64, device="cuda")
    assert xb.solve_noalloc(_dev(V), I, raise_on_error=False) == xbar.XBAR_ESTATE
    xb.destroy()


# ---------------------------------------------------------------------------------------------
# full-size blocks (M = 256: 2 x 2 inversion, tensor-core products), resistive wires and ragged N
# ---------------------------------------------------------------------------------------------
@pytest.mark.slow
@pytest.mark.parametrize("M,N,r_wire", [(256, 256, 1.0), (256, 256, 2.5), (256, 256, 10.0), (256, 17, 2.5),
                                        (256, 33, 2.5), (256, 200, 2.5)])
@pytest.mark.parametrize("precision,bar", [("fp32_ir", MIXED_BAR), ("fp64", FP64_BAR)])
def test_cr_256(M, N, r_wire, precision, bar):
    R = (1.0, r_wire, r_wire, 10.0)
    # the same maps as the block-Thomas tests (their oracle factorizations are cached and shared)
    seed = 0 if (M, N, r_wire) == (256, 256, 1.0) else 7
    G, V = case(M, N, 300, None, seed=seed)
    Geff = oracle_transfer(M, N, R, seed=seed)
    out = _solve_cr(G, R, V, precision, products=1)
    err = rel_err(out["I"], V @ Geff)
    assert err <= bar, err
    if precision == "fp32_ir":
        assert 1 <= out["info"]["iters"] <= 4, out["info"]
