"""libxbar.so builds, loads and exports every entry point declared in include/xbar.h (no GPU needed)."""
import ctypes
import subprocess

from paper_2410_19993_gb300 import build, xbar


def test_header_declares_the_boundary():
    names = xbar.exported_symbols()
    for n in ["xbar_assemble", "xbar_factor", "xbar_solve", "xbar_destroy", "xbar_last_error", "xbar_sync",
              "xbar_version"]:
        assert n in names


def test_library_exports_every_declared_symbol():
    path = build.build()
    lib = ctypes.CDLL(path)
    for n in xbar.exported_symbols():
        assert hasattr(lib, n), n
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True).stdout
    for n in xbar.exported_symbols():
        assert f" T {n}" in out, n


def test_version_and_error_string_without_gpu():
    lib = xbar.load()
    assert lib.xbar_version().startswith(b"libxbar")
    assert isinstance(lib.xbar_last_error(), bytes)


def test_host_side_argument_checks_without_gpu():
    """Argument validation happens on the host before any CUDA call."""
    import numpy as np
    lib = xbar.load()
    h = ctypes.c_void_p()
    G = np.ones((4, 4))
    assert lib.xbar_assemble(0, 4, G.ctypes.data, 1, 1, 1, 1, None, ctypes.byref(h)) == xbar.XBAR_EINVAL
    assert lib.xbar_assemble(4, 4, G.ctypes.data, 1, -1, 1, 1, None, ctypes.byref(h)) == xbar.XBAR_EINVAL
    assert lib.xbar_assemble(4, 4, G.ctypes.data, 1, 1, 0.0, 1, None, ctypes.byref(h)) == xbar.XBAR_EINVAL
    assert lib.xbar_assemble(4, 4, G.ctypes.data, 1, 1, 1, float("nan"), None, ctypes.byref(h)) == xbar.XBAR_EINVAL
    assert lib.xbar_assemble(4, 4, None, 1, 1, 1, 1, None, ctypes.byref(h)) == xbar.XBAR_EINVAL
    Gbad = G.copy()
    Gbad[1, 2] = -1e-6
    assert lib.xbar_assemble(4, 4, Gbad.ctypes.data, 1, 1, 1, 1, None, ctypes.byref(h)) == xbar.XBAR_EINVAL
    assert b"G[6]" in lib.xbar_last_error()
    assert lib.xbar_factor(None, 0) == xbar.XBAR_EINVAL
    assert lib.xbar_solve(None, 1, None, None, None, None, 1e-8, 4, None) == xbar.XBAR_EINVAL
    assert lib.xbar_destroy(None) == xbar.XBAR_OK


def test_null_handles_are_rejected_without_gpu():
    """Every entry point taking a handle rejects NULL with XBAR_EINVAL before any CUDA call."""
    import numpy as np
    lib = xbar.load()
    V = np.zeros((2, 3))
    I = np.zeros((2, 3))
    G = np.zeros(9)
    assert lib.xbar_set_conductances(None, G.ctypes.data) == xbar.XBAR_EINVAL
    assert lib.xbar_set_option(None, 0, 1) == xbar.XBAR_EINVAL
    assert lib.xbar_sync(None) == xbar.XBAR_EINVAL
    assert lib.xbar_profile_enable(None, 1) == xbar.XBAR_EINVAL
    assert lib.xbar_profile_read(None, None, 0) == xbar.XBAR_EINVAL
    assert lib.xbar_transfer_matrix(None, 1e-9, 10, None, None) == xbar.XBAR_EINVAL
    assert lib.xbar_solve_transfer(None, 2, V.ctypes.data, I.ctypes.data) == xbar.XBAR_EINVAL
    assert lib.xbar_solve_noalloc(None, 2, V.ctypes.data, I.ctypes.data) == xbar.XBAR_EINVAL
    assert b"NULL" in lib.xbar_last_error()


def test_binding_marshals_only_contiguous_float64():
    """The binding passes pointers of contiguous float64 arrays and refuses anything else."""
    import numpy as np
    import pytest
    a = np.zeros((3, 4))
    assert xbar._ptr(a) == a.ctypes.data
    assert xbar._ptr(None) is None
    with pytest.raises(TypeError):
        xbar._ptr(np.zeros((3, 4), dtype=np.float32))
    with pytest.raises(TypeError):
        xbar._ptr(a[:, ::2])  # not contiguous
    with pytest.raises(TypeError):
        xbar._ptr([1.0, 2.0])


def test_injected_allocation_failure_without_gpu(monkeypatch):
    """XBAR_FAIL_ALLOC_AFTER=0 makes the first device allocation fail before cudaMalloc is called:
    xbar_assemble returns XBAR_ENOMEM ("out of memory") and no handle."""
    import numpy as np
    lib = xbar.load()
    G = np.full((6, 5), 1e-5)
    h = ctypes.c_void_p(1234)
    monkeypatch.setenv("XBAR_FAIL_ALLOC_AFTER", "0")
    assert lib.xbar_assemble(6, 5, G.ctypes.data, 1, 1, 1, 10, None, ctypes.byref(h)) == xbar.XBAR_ENOMEM
    assert b"out of memory" in lib.xbar_last_error()
    assert not h.value


def test_binding_refuses_wrong_shapes_without_gpu():
    """The binding checks array shapes before any pointer reaches the library."""
    import numpy as np
    import pytest
    xb = xbar.Crossbar(4, 3, 0)  # never reaches the library: every call below fails its shape check
    with pytest.raises(ValueError):
        xb.solve(np.zeros((2, 5)), np.zeros((2, 3)))
    with pytest.raises(ValueError):
        xb.solve(np.zeros((2, 4)), np.zeros((3, 3)))
    with pytest.raises(ValueError):
        xb.solve(np.zeros((2, 4)), np.zeros((2, 3)), vWL=np.zeros((2, 3, 4)))
    with pytest.raises(ValueError):
        xb.solve_noalloc(np.zeros((2, 4, 1)), np.zeros((2, 3)))
    with pytest.raises(ValueError):
        xb.solve_transfer(np.zeros((2, 4)), np.zeros((2, 4)))
    with pytest.raises(ValueError):
        xb.transfer_matrix(Geff=np.zeros((3, 4)))
    with pytest.raises(ValueError):
        xb.set_conductances(np.zeros((3, 4)))
    with pytest.raises(ValueError):
        xbar.Crossbar.assemble(np.zeros(12), 1, 1, 1, 10)
