"""GPU parity of blocking over rows (XBAR_OPT_ORIENTATION): the FP64 solve of the mirrored crossbar
(M' = N, N' = M, R_s <-> R_sense, R_w <-> R_b) against the CPU oracle of the original crossbar.

Every case uses four different resistances, so an exchanged pair, a reversed index or a source on
the wrong end shows up in the currents or in one of the two node-voltage fields.
"""
import numpy as np
import pytest

import oracle
from paper_2410_19993_gb300 import xbar
from tests.gpu_common import case, oracle_transfer, rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FP64_BAR = 1e-10
MIXED_BAR = 1e-8
R = (1.0, 2.0, 1.5, 10.0)


def _solve(G, V, orientation, algorithm="thomas", precision="fp64", voltages=True, host=False, R=R):
    M, N = G.shape
    B = V.shape[0]
    if host:
        Gt, Vt = np.ascontiguousarray(G), np.ascontiguousarray(V)
        I = np.zeros((B, N))
        vW = np.zeros((B, M, N)) if voltages else None
        vB = np.zeros((B, M, N)) if voltages else None
    else:
        Gt = torch.from_numpy(np.ascontiguousarray(G)).cuda()
        Vt = torch.from_numpy(np.ascontiguousarray(V)).cuda()
        I = torch.zeros((B, N), dtype=torch.float64, device="cuda")
        vW = torch.zeros((B, M, N), dtype=torch.float64, device="cuda") if voltages else None
        vB = torch.zeros((B, M, N), dtype=torch.float64, device="cuda") if voltages else None
    xb = xbar.Crossbar.assemble(Gt, *R)
    xb.set_option("orientation", orientation)
    xb.set_option("algorithm", algorithm)
    xb.factor(precision)
    _, info = xb.solve(Vt, I, vW, vB, tol=1e-9, max_iter=10)
    xb.sync()
    out = {"I": I if host else I.cpu().numpy(), "info": info, "xb": xb}
    if voltages:
        out["vWL"] = vW if host else vW.cpu().numpy()
        out["vBL"] = vB if host else vB.cpu().numpy()
    return out


SHAPES = [(128, 20, 300), (40, 3, 1000), (33, 17, 200), (9, 1, 3), (200, 5, 40), (16, 128, 64), (1, 1, 1),
          (1, 7, 5), (7, 1, 2)]


@pytest.mark.parametrize("algorithm", ["thomas", "cr"])
@pytest.mark.parametrize("M,N,B", SHAPES)
def test_rows_against_oracle(M, N, B, algorithm):
    G, V = case(M, N, B, None, seed=100 * M + N)
    ref = oracle.solve(M, N, G, *R, V, voltages=True)
    out = _solve(G, V, "rows", algorithm)
    assert rel_err(out["I"], ref["I"]) <= FP64_BAR
    assert np.max(np.abs(out["vWL"] - ref["vWL"])) <= FP64_BAR
    assert np.max(np.abs(out["vBL"] - ref["vBL"])) <= FP64_BAR
    out["xb"].destroy()


@pytest.mark.parametrize("M,N,B", [(128, 20, 96), (64, 32, 50), (24, 24, 10)])
def test_orientations_agree_and_auto(M, N, B):
    """Columns and rows give the same currents; 'auto' takes rows exactly when 2N <= M."""
    G, V = case(M, N, B, None, seed=7)
    cols = _solve(G, V, "columns", voltages=False)
    rows = _solve(G, V, "rows", voltages=False)
    auto = _solve(G, V, "auto", voltages=False)
    assert rel_err(rows["I"], cols["I"]) <= 1e-11
    same_as = rows if 2 * N <= M else cols
    np.testing.assert_array_equal(auto["I"], same_as["I"])
    for o in (cols, rows, auto):
        o["xb"].destroy()


def test_rows_host_buffers_and_refactor_after_new_map():
    """Host buffers, then xbar_set_conductances: the next factor rebuilds the mirrored map."""
    M, N, B = 96, 12, 40
    G, V = case(M, N, B, None, seed=3)
    out = _solve(G, V, "rows", host=True)
    ref = oracle.solve(M, N, G, *R, V, voltages=True)
    assert rel_err(out["I"], ref["I"]) <= FP64_BAR
    assert np.max(np.abs(out["vWL"] - ref["vWL"])) <= FP64_BAR
    xb = out["xb"]
    G2, _ = case(M, N, 1, None, seed=4)
    xb.set_conductances(np.ascontiguousarray(G2))
    xb.factor("fp64")
    I2 = np.zeros((B, N))
    xb.solve(np.ascontiguousarray(V), I2)
    ref2 = oracle.solve(M, N, G2, *R, V)
    assert rel_err(I2, ref2["I"]) <= FP64_BAR
    xb.destroy()


def test_rows_transfer_matrix():
    """G_eff of the row-blocked factorization (M unit solves through the same path) against the
    oracle's transfer matrix."""
    M, N = 80, 10
    G, _ = case(M, N, 1, None, seed=5)
    Gt = torch.from_numpy(np.ascontiguousarray(G)).cuda()
    xb = xbar.Crossbar.assemble(Gt, *R)
    xb.set_option("orientation", "rows")
    xb.factor("fp64")
    Geff = torch.zeros((M, N), dtype=torch.float64, device="cuda")
    xb.transfer_matrix(Geff=Geff)
    ref = oracle_transfer(M, N, R, seed=5)
    assert rel_err(Geff.cpu().numpy(), ref) <= FP64_BAR
    xb.destroy()


MIXED_SHAPES = [(128, 20, 300), (40, 3, 1000), (33, 17, 200), (200, 5, 40), (16, 128, 64), (1, 1, 1), (7, 1, 2),
                (256, 32, 100)]


@pytest.mark.parametrize("algorithm", ["thomas", "cr"])
@pytest.mark.parametrize("M,N,B", MIXED_SHAPES)
def test_rows_mixed_against_oracle(M, N, B, algorithm):
    """XBAR_FP32_IR blocked over rows: FP32 factor of the mirror, float-pair refinement with the
    sources on its bit-line chains, currents from its first block."""
    G, V = case(M, N, B, None, seed=200 * M + N)
    ref = oracle.solve(M, N, G, *R, V, voltages=True)
    out = _solve(G, V, "rows", algorithm, precision="fp32_ir")
    assert rel_err(out["I"], ref["I"]) <= MIXED_BAR
    assert np.max(np.abs(out["vWL"] - ref["vWL"])) <= MIXED_BAR
    assert np.max(np.abs(out["vBL"] - ref["vBL"])) <= MIXED_BAR
    assert 1 <= out["info"]["iters"] <= 4
    out["xb"].destroy()


def test_mixed_auto_keeps_columns_and_noalloc_refuses_rows():
    """Automatic orientation keeps mixed-precision factors on columns (bit for bit the column
    result); the no-allocation entry point needs a column-blocked FP64 factorization."""
    M, N, B = 128, 20, 64
    G, V = case(M, N, B, None, seed=9)
    ref = oracle.solve(M, N, G, *R, V)
    auto = _solve(G, V, "auto", precision="fp32_ir", voltages=False)
    cols = _solve(G, V, "columns", precision="fp32_ir", voltages=False)
    np.testing.assert_array_equal(auto["I"], cols["I"])
    assert rel_err(auto["I"], ref["I"]) <= MIXED_BAR
    cols["xb"].destroy()
    xb = auto["xb"]
    xb.factor("fp64")  # automatic: rows for FP64 (2N <= M)
    Vt = torch.from_numpy(np.ascontiguousarray(V)).cuda()
    I = torch.zeros((B, N), dtype=torch.float64, device="cuda")
    with pytest.raises(xbar.XbarError) as e:
        xb.solve_noalloc(Vt, I)
    assert e.value.status == xbar.XBAR_ESTATE
    xb.set_option("orientation", "columns")
    xb.factor("fp64")
    xb.solve_noalloc(Vt, I)
    xb.sync()
    assert rel_err(I.cpu().numpy(), ref["I"]) <= FP64_BAR
    xb.destroy()
