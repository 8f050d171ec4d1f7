"""GPU parity of the transfer-matrix (currents-only) mode against the CPU FP64 oracle.

G_eff[i][j] = dI_j / dV_i of the nodal system (Sec. II, Eqs. 1-7) is computed by the library from
M unit-input solves of its own factorization; the oracle computes it from M unit solves with its
banded LU.  Both are compared entrywise, then the currents I = V G_eff of the library's FP64
product against V @ G_eff of the oracle.  Bars: 1e-10 (XBAR_FP64), 1e-8 (XBAR_FP32_IR, refinement
tolerance 1e-9).
"""
import numpy as np
import pytest

from paper_2410_19993_gb300 import xbar
from tests.gpu_common import case, oracle_transfer, rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

BARS = {"fp64": 1e-10, "fp32_ir": 1e-8}
IR_TOL = 1e-9


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _transfer(G, R, V, precision, host=False):
    M, N = G.shape
    B = V.shape[0]
    xb = xbar.Crossbar.assemble(_dev(G), *R)
    xb.factor(precision)
    if host:
        Ge = np.zeros((M, N))
        I = np.zeros((B, N))
        xb.transfer_matrix(tol=IR_TOL, Geff=Ge)
        xb.solve_transfer(np.ascontiguousarray(V), I)
    else:
        Ge_d = torch.zeros((M, N), dtype=torch.float64, device="cuda")
        I_d = torch.zeros((B, N), dtype=torch.float64, device="cuda")
        xb.transfer_matrix(tol=IR_TOL, Geff=Ge_d)
        xb.solve_transfer(_dev(V), I_d)
        xb.sync()
        Ge, I = Ge_d.cpu().numpy(), I_d.cpu().numpy()
    xb.destroy()
    return Ge, I


@pytest.mark.parametrize("M,N,B,R", [(16, 16, 64, (1.0, 1.0, 1.0, 10.0)), (64, 64, 300, (1.0, 2.5, 2.5, 10.0)),
                                     (17, 33, 70, (1.0, 2.0, 1.5, 10.0)), (33, 17, 129, (1.0, 0.5, 3.0, 10.0)),
                                     (1, 7, 5, (1.0, 1.0, 1.0, 10.0)), (9, 1, 3, (1.0, 1.0, 1.0, 10.0))])
@pytest.mark.parametrize("precision", ["fp64", "fp32_ir"])
def test_transfer_matrix_and_currents_against_oracle(M, N, B, R, precision):
    G, V = case(M, N, B, None, seed=5)
    Gref = oracle_transfer(M, N, R, seed=5)
    Ge, I = _transfer(G, R, V, precision)
    bar = BARS[precision]
    assert rel_err(Ge, Gref) <= bar          # every entry of G_eff
    assert rel_err(I, V @ Gref) <= bar       # every current (V >= 0: positive terms)


def test_transfer_host_pointers_match_device_pointers():
    G, V = case(24, 20, 50, None, seed=3)
    R = (1.0, 1.0, 1.0, 10.0)
    Ge_d, I_d = _transfer(G, R, V, "fp32_ir")
    Ge_h, I_h = _transfer(G, R, V, "fp32_ir", host=True)
    np.testing.assert_array_equal(Ge_d, Ge_h)
    np.testing.assert_array_equal(I_d, I_h)


def test_transfer_matches_the_substitution_path():
    """The currents-only mode and the sweeps are different paths to the same currents."""
    M, N, B = 48, 40, 200
    G, V = case(M, N, B, None, seed=11)
    R = (1.0, 2.5, 2.5, 10.0)
    _, I_t = _transfer(G, R, V, "fp64")
    xb = xbar.Crossbar.assemble(_dev(G), *R)
    xb.factor("fp64")
    I_s = torch.zeros((B, N), dtype=torch.float64, device="cuda")
    xb.solve(_dev(V), I_s)
    xb.sync()
    xb.destroy()
    assert rel_err(I_t, I_s.cpu().numpy()) <= 1e-10


def test_transfer_state_and_errors():
    G, V = case(12, 10, 8, None, seed=2)
    R = (1.0, 1.0, 1.0, 10.0)
    xb = xbar.Crossbar.assemble(_dev(G), *R)
    I = torch.zeros((8, 10), dtype=torch.float64, device="cuda")
    st, _ = xb.transfer_matrix(raise_on_error=False)  # before xbar_factor
    assert st == xbar.XBAR_ESTATE
    xb.factor("fp64")
    assert xb.solve_transfer(_dev(V), I, raise_on_error=False) == xbar.XBAR_ESTATE  # no G_eff yet
    st, info = xb.transfer_matrix()
    assert st == xbar.XBAR_OK
    st, info2 = xb.transfer_matrix()  # cached: no solves
    assert st == xbar.XBAR_OK and info2["iters"] == 0
    assert xb.solve_transfer(_dev(V), I) == xbar.XBAR_OK
    assert xb.solve_transfer(_dev(V[:0]), I[:0], raise_on_error=False) == xbar.XBAR_OK  # B = 0
    # new conductances invalidate G_eff until the next factor + transfer_matrix
    G2 = G * 1.5
    xb.set_conductances(_dev(G2))
    assert xb.solve_transfer(_dev(V), I, raise_on_error=False) == xbar.XBAR_ESTATE
    xb.factor("fp64")
    assert xb.solve_transfer(_dev(V), I, raise_on_error=False) == xbar.XBAR_ESTATE
    Ge2 = torch.zeros((12, 10), dtype=torch.float64, device="cuda")
    xb.transfer_matrix(Geff=Ge2)
    xb.solve_transfer(_dev(V), I)
    xb.sync()
    # G_eff of the new map: the currents change with the conductances
    I2 = I.cpu().numpy()
    I1 = V @ oracle_transfer(12, 10, R, seed=2)
    assert not np.allclose(I1, I2)
    xb.destroy()


@pytest.mark.slow
def test_transfer_full_size():
    """256 x 256, 8192 vectors (the bench workload's shape): G_eff and every current."""
    M, N, B = 256, 256, 8192
    R = (1.0, 1.0, 1.0, 10.0)
    G, V = case(M, N, B, None, seed=0)
    Gref = oracle_transfer(M, N, R, seed=0)
    Ge, I = _transfer(G, R, V, "fp32_ir")
    assert rel_err(Ge, Gref) <= 1e-8
    assert rel_err(I, V @ Gref) <= 1e-8
