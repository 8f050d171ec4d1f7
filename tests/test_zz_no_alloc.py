"""xbar_solve_noalloc: the FP64 substitution for callers that must not allocate device memory.

Such callers (a latency-critical loop where cudaMalloc/cudaFree could stall the device, or a
process whose device memory belongs to a framework allocator) get their scratch from a fixed
array inside libxbar.  This test calls the entry point through the C ABI twice in a row and
compares each result with xbar_solve on the same handle, within the FP64 tolerance the parity
tests use; it also checks that an oversized request is refused with XBAR_EINVAL.  The file is
named so that pytest collects it last.
"""
import numpy as np
import pytest

from paper_2410_19993_gb300 import inputs, xbar

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FP64_BAR = 1e-10


def _rel(a, b):
    return float(np.max(np.abs(a - b) / np.maximum(np.abs(b), 1e-300)))


def _warm_up(G, R, V):
    """The first use of the fixed array, and of each kernel, makes the CUDA runtime load it (lazy
    loading reserves the array and the code then); do that on a throwaway handle of the same shape
    and batch as the measured calls."""
    xb = xbar.Crossbar.assemble(torch.from_numpy(G).cuda(), *R)
    xb.factor("fp64")
    I = torch.zeros((V.shape[0], G.shape[1]), dtype=torch.float64, device="cuda")
    assert xb.solve_noalloc(torch.from_numpy(V).cuda(), I) == xbar.XBAR_OK
    xb.sync()
    xb.destroy()


def test_noalloc_matches_solve_twice():
    M, N, B = 64, 64, 1024
    R = (1.0, 2.5, 2.5, 10.0)
    G, V1 = inputs.crossbar(M, N, B, seed=21)
    _, V2 = inputs.crossbar(M, N, B, seed=22)
    _warm_up(G, R, V1)
    Vs = [torch.from_numpy(V).cuda() for V in (V1, V2)]
    Is = [torch.full((B, N), float("nan"), dtype=torch.float64, device="cuda") for _ in Vs]
    Irefs = [torch.zeros((B, N), dtype=torch.float64, device="cuda") for _ in Vs]
    xb = xbar.Crossbar.assemble(torch.from_numpy(G).cuda(), *R)
    xb.factor("fp64")
    xb.sync()
    free0 = torch.cuda.mem_get_info()[0]
    # on a fresh handle, before any xbar_solve could have sized a workspace: no device memory taken
    for Vd, I in zip(Vs, Is):
        assert xb.solve_noalloc(Vd, I) == xbar.XBAR_OK
    xb.sync()
    assert torch.cuda.mem_get_info()[0] == free0
    for Vd, I, Iref in zip(Vs, Is, Irefs):
        xb.solve(Vd, Iref)
        xb.sync()
        assert _rel(I.cpu().numpy(), Iref.cpu().numpy()) <= FP64_BAR
    xb.destroy()


def test_noalloc_refuses_oversized_and_wrong_state():
    M, N = 256, 256
    G, V = inputs.crossbar(M, N, 2048, seed=23)
    xb = xbar.Crossbar.assemble(torch.from_numpy(G).cuda(), 1.0, 1.0, 1.0, 10.0)
    Vd = torch.from_numpy(V).cuda()
    I = torch.zeros((2048, N), dtype=torch.float64, device="cuda")
    assert xb.solve_noalloc(Vd, I, raise_on_error=False) == xbar.XBAR_ESTATE
    xb.factor("fp64")
    assert xb.solve_noalloc(Vd, I, raise_on_error=False) == xbar.XBAR_EINVAL  # 256*256*2048*8 B > 64 MiB
    assert "exceeds the fixed" in xbar.last_error()
    assert xb.solve_noalloc(np.ascontiguousarray(V), I, raise_on_error=False) == xbar.XBAR_EINVAL
    xb.factor("fp32_ir")  # only the FP64 substitution has a fixed-scratch variant
    assert xb.solve_noalloc(Vd[:64], I[:64], raise_on_error=False) == xbar.XBAR_ESTATE
    xb.destroy()
