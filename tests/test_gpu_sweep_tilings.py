"""GPU parity of the CUDA-core substitution kernel in each of its tilings, against the CPU FP64 oracle.

The sweeps (Sec. II-C: forward and back substitution for every input vector with one
factorization) run in two register tilings: wide tiles for big panels, narrow 2 x 1 tiles with
panels of exactly ceil(B / SMs) vectors when the wide tiling would leave a block with fewer than
four warps.  The cases below reach, with B and Mp chosen for it (152 SMs): a partial warp, a
block of whole warps with the shuffle pre-reduction of the currents, odd panel widths, the wide
tiling with and without the pre-reduction, and the wide tiling at its 512-thread cap
(batches whose panels would otherwise need more registers than an SM has).  Currents are
compared with V @ G_eff of the oracle's transfer matrix; bars 1e-10 (FP64) and 1e-8 (FP32 factor
+ refinement, tolerance 1e-9).
"""
import numpy as np
import pytest

from paper_2410_19993_gb300 import xbar
from tests.gpu_common import case, oracle_transfer, rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

BARS = {"fp64": 1e-10, "fp32_ir": 1e-8}
R_PAPER = (5.0, 5.0, 5.0, 5.0)   # the paper's parasitic resistors (Sec. III)
R_MIXED = (1.0, 2.5, 2.5, 10.0)

CASES = [
    (16, 16, 1, R_PAPER),      # narrow, 8 threads: partial warp
    (64, 48, 1, R_MIXED),      # narrow, one whole warp: shuffle pre-reduction
    (40, 30, 700, R_MIXED),    # narrow, panels of 5 (Mp = 48), 120 threads: no pre-reduction
    (100, 37, 333, R_PAPER),   # narrow, Mp = 112, panels of 3
    (256, 64, 1, R_PAPER),     # narrow, four warps: one per SM sub-partition
    (200, 20, 1500, R_MIXED),  # narrow, panels of 9 held to 936 threads by the 1024-thread bound
    (256, 24, 2432, R_MIXED),  # FP64 wide (panels of 16) / FP32 narrow (1024 threads), pre-reduction
    (256, 16, 4864, R_MIXED),  # wide in both precisions, pre-reduction
    (256, 16, 5000, R_PAPER),  # wide in both precisions, panels of 36 / 40: no pre-reduction
]


def _currents(G, R, V, precision, simt):
    M, N = G.shape
    B = V.shape[0]
    xb = xbar.Crossbar.assemble(torch.from_numpy(G).cuda(), *R)
    if simt:
        xb.set_option("sweep_kernel", 0)
    xb.factor(precision)
    I = torch.zeros((B, N), dtype=torch.float64, device="cuda")
    xb.solve(torch.from_numpy(np.ascontiguousarray(V)).cuda(), I, tol=1e-9, max_iter=10)
    xb.sync()
    xb.destroy()
    return I.cpu().numpy()


@pytest.mark.parametrize("M,N,B,R", CASES)
@pytest.mark.parametrize("precision", ["fp64", "fp32_ir"])
def test_sweep_tilings_against_oracle(M, N, B, R, precision):
    G, V = case(M, N, B, None, seed=9)
    Gref = oracle_transfer(M, N, R, seed=9)
    I = _currents(G, R, V, precision, simt=precision == "fp32_ir")
    assert rel_err(I, V @ Gref) <= BARS[precision]


@pytest.mark.slow
@pytest.mark.parametrize("M,N,B,precision", [(64, 16, 50000, "fp64"), (256, 16, 20000, "fp32_ir")])
def test_wide_tiling_at_thread_cap(M, N, B, precision):
    """Batches whose wide panels are held to 512 threads (256 x 256 and 480 x 128 registers fit):
    FP64 at Mp = 64 with panels of 256, and the FP32 CUDA-core sweep at Mp = 256 with panels of 120."""
    G, V = case(M, N, B, None, seed=4)
    Gref = oracle_transfer(M, N, R_MIXED, seed=4)
    I = _currents(G, R_MIXED, V, precision, simt=precision == "fp32_ir")
    assert rel_err(I, V @ Gref) <= BARS[precision]


def test_batch_of_one_matches_batch_of_many():
    """The same vector solved alone (narrow tiling) and inside a wide panel gives the same currents."""
    M, N, B = 256, 32, 2432
    G, V = case(M, N, B, None, seed=6)
    I_all = _currents(G, R_MIXED, V, "fp64", simt=False)
    for b in (0, 1234, B - 1):
        I_one = _currents(G, R_MIXED, V[b:b + 1], "fp64", simt=False)
        assert rel_err(I_one, I_all[b:b + 1]) <= 1e-12
