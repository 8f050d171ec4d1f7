"""GPU parity of the tile batch (one CUDA-graph launch for all tiles) on the 784-256-10 mapping.

Every tile of a batch run is compared with the single-crossbar path of the same library (itself
checked against the oracle in test_gpu_parity.py), and one tile of each distinct shape directly
with the CPU oracle's transfer matrix; at the workload's full size (4096 vectors per tile) every
tile is compared with the oracle's transfer matrix.
"""
import json
import multiprocessing

import numpy as np
import pytest

import oracle
from paper_2410_19993_gb300 import inputs, xbar
from tests.gpu_common import oracle_transfer_of, rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

B_TILE = 96
IR_TOL = 1e-9


@pytest.fixture(scope="module")
def tiles():
    return inputs.fc_tiles(B=B_TILE)


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _batch(tiles):
    return xbar.Batch([(t.G, *t.circuit.as_tuple()) for t in tiles])


def _run(b, tiles, precision, Vs=None, Is=None):
    Vs = Vs if Vs is not None else [_dev(t.V) for t in tiles]
    Is = Is if Is is not None else [torch.zeros((t.V.shape[0], t.G.shape[1]), dtype=torch.float64, device="cuda")
                                    for t in tiles]
    st, infos = b.run(precision, Vs, Is, tol=IR_TOL, max_iter=6)
    return [I.cpu().numpy() for I in Is], infos


def test_shapes_of_the_mapping(tiles):
    shapes = sorted({t.G.shape for t in tiles})
    assert len(tiles) == 30
    assert shapes == [(16, 128), (128, 20), (128, 128)]
    assert sum(t.G.shape == (128, 128) for t in tiles) == 24


@pytest.mark.parametrize("precision,bar", [("fp64", 1e-10), ("fp32_ir", 1e-8)])
def test_batch_matches_single_path_and_oracle(tiles, precision, bar):
    b = _batch(tiles)
    out, infos = _run(b, tiles, precision)
    b.destroy()
    seen = set()
    for t, I, info in zip(tiles, out, infos):
        R = t.circuit.as_tuple()
        xb = xbar.Crossbar.assemble(_dev(t.G), *R)
        xb.factor("fp64")
        Iref = torch.zeros_like(torch.from_numpy(I)).cuda()
        xb.solve(_dev(t.V), Iref)
        xb.sync()
        assert rel_err(I, Iref.cpu().numpy()) <= bar
        xb.destroy()
        if precision == "fp32_ir":
            assert 1 <= info["iters"] <= 6
        if t.G.shape not in seen:  # one tile of each shape against the oracle
            seen.add(t.G.shape)
            f = oracle.factor(t.G.shape[0], t.G.shape[1], t.G, *R)
            Istar = t.V @ oracle.transfer_matrix(f)
            assert rel_err(I, Istar) <= bar


def test_graph_replay_and_recapture(tiles):
    b = _batch(tiles)
    Vs = [_dev(t.V) for t in tiles]
    Is = [torch.zeros((t.V.shape[0], t.G.shape[1]), dtype=torch.float64, device="cuda") for t in tiles]
    first, _ = _run(b, tiles, "fp32_ir", Vs, Is)
    # same buffers, new values: the captured graph is replayed and must see them
    for V in Vs:
        V.mul_(0.5)
    second, _ = _run(b, tiles, "fp32_ir", Vs, Is)
    for a, c in zip(first, second):
        np.testing.assert_allclose(c, 0.5 * a, rtol=1e-8, atol=0)  # the nodal system is linear in V
    # new buffers: recapture
    Vs2 = [V.clone() for V in Vs]
    third, _ = _run(b, tiles, "fp32_ir", Vs2, None)
    for a, c in zip(second, third):
        assert rel_err(c, a) <= 1e-8
    b.destroy()


def test_autotune_cache(tiles, tmp_path):
    path = str(tmp_path / "tune.json")
    b = _batch(tiles)
    B = [t.V.shape[0] for t in tiles]
    b.autotune("fp32_ir", B, path)
    data = json.load(open(path))
    assert len(data) == 3  # one entry per distinct (M, N, B)
    for v in data.values():
        assert v["sweep"] in (0, 1) and v["factor"] in (0, 1)
    out, _ = _run(b, tiles, "fp32_ir")
    b.destroy()
    b2 = _batch(tiles)
    b2.autotune("fp32_ir", B, path)  # served from the cache
    out2, _ = _run(b2, tiles, "fp32_ir")
    b2.destroy()
    for a, c in zip(out, out2):
        assert rel_err(c, a) <= 1e-8


@pytest.fixture(scope="module")
def full_tiles():
    """The 30 tiles with 4096 vectors each and the oracle's transfer matrix of every tile (CPU, in
    a spawned process pool: a pool forked after CUDA initialisation can hang)."""
    ts = inputs.fc_tiles(B=4096)
    with multiprocessing.get_context("spawn").Pool(min(8, multiprocessing.cpu_count())) as pool:
        T = pool.map(oracle_transfer_of, [(t.G, t.circuit.as_tuple()) for t in ts])
    return ts, T


@pytest.mark.slow
@pytest.mark.parametrize("precision,bar", [("fp64", 1e-10), ("fp32_ir", 1e-8)])
def test_batch_full_size_every_tile_against_oracle(full_tiles, precision, bar):
    ts, T = full_tiles
    b = _batch(ts)
    out, infos = _run(b, ts, precision)
    b.destroy()
    for t, I, Geff, info in zip(ts, out, T, infos):
        assert rel_err(I, t.V @ Geff) <= bar, t.G.shape
        if precision == "fp32_ir":
            assert 1 <= info["iters"] <= 6


def test_autotune_fp64_orientation(tiles, tmp_path):
    """FP64 autotuning times blocks over columns and over rows per shape; whatever it picks, the
    currents stay those of the single path."""
    path = str(tmp_path / "tune64.json")
    b = _batch(tiles)
    B = [t.V.shape[0] for t in tiles]
    b.autotune("fp64", B, path)
    data = json.load(open(path))
    assert len(data) == 3
    for v in data.values():
        assert v["orient"] in (0, 1)
        assert v["orient_ms"][0] > 0  # columns always timed
    out, _ = _run(b, tiles, "fp64")
    b.destroy()
    for t, I in zip(tiles, out):
        xb = xbar.Crossbar.assemble(_dev(t.G), *t.circuit.as_tuple())
        xb.set_option("orientation", "columns")
        xb.factor("fp64")
        Iref = torch.zeros_like(torch.from_numpy(I)).cuda()
        xb.solve(_dev(t.V), Iref)
        xb.sync()
        assert rel_err(I, Iref.cpu().numpy()) <= 1e-11
        xb.destroy()


def test_batch_rejects_host_buffers(tiles):
    b = _batch(tiles[:2])
    Vs = [np.ascontiguousarray(t.V) for t in tiles[:2]]
    Is = [np.zeros((t.V.shape[0], t.G.shape[1])) for t in tiles[:2]]
    st, _ = b.run("fp64", Vs, Is, raise_on_error=False)
    assert st == xbar.XBAR_EINVAL
    b.destroy()
