"""Failure detection without a GPU fault: bounded device waits that run out, host-side allocation
failures, and invalid inputs caught on the device.  Each test checks that the failure surfaces as a
status code, that nothing hangs, and that the handle (or a new one) works afterwards.
"""
import os

import numpy as np
import pytest

import oracle
from paper_2410_19993_gb300 import xbar
from tests.gpu_common import case, rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def test_wait_limit_expiry_is_reported_and_recovered():
    """A 1 ns limit makes the cross-block barriers of the cooperative FP64 factor run out: the
    blocks record the timeout and return (no hang), xbar_sync reports XBAR_ETIMEOUT, and after the
    default limit is restored the same handle factors and solves correctly."""
    M, N, B = 64, 48, 20
    R = (1.0, 2.5, 2.5, 10.0)
    G, V = case(M, N, B, None, seed=31)
    xb = xbar.Crossbar.assemble(_dev(G), *R)
    xb.set_option("factor_kernel", 0)      # the cooperative group kernel: plain spins on global flags
    xb.set_option("wait_limit_ns", 1)
    xb.factor("fp64")
    with pytest.raises(xbar.XbarError) as ei:
        xb.sync()
    assert ei.value.status == xbar.XBAR_ETIMEOUT
    assert "bounded device wait" in xbar.last_error()
    xb.sync()                              # the status word was cleared when it was reported
    xb.set_option("wait_limit_ns", -1)
    xb.factor("fp64")
    I = torch.zeros((B, N), dtype=torch.float64, device="cuda")
    xb.solve(_dev(V), I)
    xb.sync()
    ref = oracle.solve(M, N, G, *R, V)
    assert rel_err(I.cpu().numpy(), ref["I"]) <= 1e-10
    xb.destroy()


def test_injected_allocation_failure(monkeypatch):
    """XBAR_FAIL_ALLOC_AFTER=n fails the allocations after the first n: xbar_assemble and
    xbar_factor return XBAR_ENOMEM, free what they took, and work again once it is unset."""
    M, N, B = 40, 30, 9
    R = (1.0, 1.0, 1.0, 10.0)
    G, V = case(M, N, B, None, seed=32)
    Gd, Vd = _dev(G), _dev(V)
    I = torch.zeros((B, N), dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for n in (0, 3, 10):
        monkeypatch.setenv("XBAR_FAIL_ALLOC_AFTER", str(n))
        with pytest.raises(xbar.XbarError) as ei:
            xbar.Crossbar.assemble(Gd, *R)
        assert ei.value.status == xbar.XBAR_ENOMEM
        monkeypatch.delenv("XBAR_FAIL_ALLOC_AFTER")
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0          # nothing leaked by the failed assemblies
    xb = xbar.Crossbar.assemble(Gd, *R)
    monkeypatch.setenv("XBAR_FAIL_ALLOC_AFTER", "0")
    with pytest.raises(xbar.XbarError) as ei:
        xb.factor("fp32_ir")
    assert ei.value.status == xbar.XBAR_ENOMEM
    monkeypatch.delenv("XBAR_FAIL_ALLOC_AFTER")
    xb.factor("fp32_ir")
    monkeypatch.setenv("XBAR_FAIL_ALLOC_AFTER", "0")        # the solve's workspace cannot be allocated
    st, _ = xb.solve(Vd, I, raise_on_error=False)
    assert st == xbar.XBAR_ENOMEM
    monkeypatch.delenv("XBAR_FAIL_ALLOC_AFTER")
    xb.solve(Vd, I, tol=1e-9)
    xb.sync()
    ref = oracle.solve(M, N, G, *R, V)
    assert rel_err(I.cpu().numpy(), ref["I"]) <= 1e-8
    xb.destroy()


def test_invalid_device_conductances_reported_by_status():
    """A device G with a negative or non-finite entry is refused on the device: the next status
    read returns XBAR_EINVAL; a valid map afterwards gives correct currents."""
    M, N, B = 24, 20, 7
    R = (1.0, 1.0, 1.0, 10.0)
    G, V = case(M, N, B, None, seed=33)
    xb = xbar.Crossbar.assemble(_dev(G), *R)
    for bad in (-1e-6, float("nan"), float("inf")):
        Gb = G.copy()
        Gb[5, 7] = bad
        xb.set_conductances(_dev(Gb))                        # asynchronous: no host round trip
        with pytest.raises(xbar.XbarError) as ei:
            xb.sync()
        assert ei.value.status == xbar.XBAR_EINVAL
    xb.set_conductances(_dev(G))
    xb.factor("fp64")
    I = torch.zeros((B, N), dtype=torch.float64, device="cuda")
    xb.solve(_dev(V), I)
    xb.sync()
    assert rel_err(I.cpu().numpy(), oracle.solve(M, N, G, *R, V)["I"]) <= 1e-10
    xb.destroy()


def test_binding_refuses_wrong_shapes_before_the_library():
    M, N, B = 10, 12, 5
    G, V = case(M, N, B, None, seed=34)
    xb = xbar.Crossbar.assemble(_dev(G), 1.0, 1.0, 1.0, 10.0)
    xb.factor("fp64")
    I = torch.zeros((B, N), dtype=torch.float64, device="cuda")
    with pytest.raises(ValueError):
        xb.solve(_dev(V[:, :M - 1]), I)
    with pytest.raises(ValueError):
        xb.solve(_dev(V), I[:, :N - 1])
    with pytest.raises(ValueError):
        xb.solve(_dev(V), I, vWL=torch.zeros((B, N, M), dtype=torch.float64, device="cuda"))
    with pytest.raises(ValueError):
        xb.solve_transfer(_dev(V), I[:B - 1])
    with pytest.raises(ValueError):
        xb.set_conductances(_dev(G.T.copy()))
    xb.destroy()
