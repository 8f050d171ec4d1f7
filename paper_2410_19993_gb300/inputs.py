"""Seeded synthetic inputs for crossbar solves (shared by the oracle tests and the GPU tests).

This module only draws random numbers and arranges them into arrays; it holds
none of the solver's arithmetic.  The paper draws memristor conductances and
input voltages at random without stating distributions (Sec. III-A); the
workloads below fix them:

* conductances G_ij log-uniform in [g_lo, g_hi] siemens (equivalently R_ij
  log-uniform in [1/g_hi, 1/g_lo] ohms), drawn first, M x N row-major;
* input voltages V uniform in [0, v_max] volts, drawn second, B x M.

``WORKLOADS`` names the five standard workloads by what they are.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass(frozen=True)
class Circuit:
    """Parasitic resistances in ohms: source, word-line segment, bit-line segment, sense."""
    Rs: float = 1.0
    Rw: float = 1.0
    Rb: float = 1.0
    Rsense: float = 10.0

    def as_tuple(self):
        return (self.Rs, self.Rw, self.Rb, self.Rsense)


@dataclass(frozen=True)
class Workload:
    name: str
    M: int
    N: int
    B: int
    circuits: tuple
    v_max: float = 0.5
    g_lo: float = 1e-6
    g_hi: float = 1e-4
    seed: int = 0
    precision: str = "fp64"
    notes: str = ""
    extra: dict = field(default_factory=dict)


WORKLOADS = {
    "xbar16_fp64": Workload("xbar16_fp64", 16, 16, 64, (Circuit(1.0, 1.0, 1.0, 10.0),),
                            notes="single 16x16 crossbar, plain FP64, 64 input vectors"),
    "xbar64_rsweep_fp64": Workload("xbar64_rsweep_fp64", 64, 64, 1024,
                                   tuple(Circuit(1.0, r, r, 10.0) for r in (0.5, 2.5, 10.0)),
                                   notes="64x64, R_w=R_b swept over 0.5/2.5/10 ohm, 1024 vectors"),
    "xbar256_mixed": Workload("xbar256_mixed", 256, 256, 8192, (Circuit(1.0, 1.0, 1.0, 10.0),),
                              precision="fp32_ir",
                              notes="256x256, FP32 factor+solve with FP64 refinement, 8192 vectors"),
    "fc784_256_10_tiles": Workload("fc784_256_10_tiles", 128, 128, 4096,
                                   (Circuit(1.0, 2.5, 2.5, 10.0),), v_max=0.3,
                                   precision="fp32_ir",
                                   notes="784-256-10 FC net mapped to 30 ragged tiles, 4096 vectors each"),
    "surrogate128": Workload("surrogate128", 128, 128, 100, (Circuit(1.0, 2.5, 2.5, 10.0),),
                             notes="per-column MLP surrogate, 128x128 maps: train on 200 maps x 100 vectors, "
                                   "calibrate on 20 x 100, test on 50 held-out maps x 1000 vectors",
                             extra={"train_maps": 200, "train_B": 100, "calib_maps": 20, "calib_B": 100,
                                    "test_maps": 50, "test_B": 1000, "train_seed": 100, "calib_seed": 200,
                                    "test_seed": 300}),
}


def conductances(rng: np.random.Generator, M: int, N: int, g_lo=1e-6, g_hi=1e-4) -> np.ndarray:
    """M x N conductances, log-uniform in [g_lo, g_hi]."""
    return np.exp(rng.uniform(np.log(g_lo), np.log(g_hi), size=(M, N)))


def voltages(rng: np.random.Generator, B: int, M: int, v_max=0.5) -> np.ndarray:
    """B x M input voltages, uniform in [0, v_max]."""
    return rng.uniform(0.0, v_max, size=(B, M))


def crossbar(M: int, N: int, B: int, seed: int = 0, g_lo=1e-6, g_hi=1e-4, v_max=0.5):
    """(G[M x N], V[B x M]) drawn in that order from default_rng(seed)."""
    rng = np.random.default_rng(seed)
    G = conductances(rng, M, N, g_lo, g_hi)
    V = voltages(rng, B, M, v_max)
    return G, V


def workload_inputs(name: str, B: int | None = None):
    """(G, V) of a named single-crossbar workload; ``B`` overrides the batch size."""
    w = WORKLOADS[name]
    return crossbar(w.M, w.N, w.B if B is None else B, w.seed, w.g_lo, w.g_hi, w.v_max)


# ---------------------------------------------------------------------------------------------
# 784 -> 256 -> 10 fully connected network mapped onto ragged crossbar tiles
# ---------------------------------------------------------------------------------------------
@dataclass
class Tile:
    layer: int
    row0: int
    col0: int
    G: np.ndarray      # M x N conductances
    V: np.ndarray      # B x M input voltages
    circuit: Circuit


def _differential(w: np.ndarray, g_lo: float, g_hi: float) -> np.ndarray:
    """Map weights to interleaved (positive, negative) conductance columns in [g_lo, g_hi]."""
    wmax = float(np.max(np.abs(w)))
    gp = g_lo + (g_hi - g_lo) * np.maximum(w, 0.0) / wmax
    gn = g_lo + (g_hi - g_lo) * np.maximum(-w, 0.0) / wmax
    out = np.empty((w.shape[0], 2 * w.shape[1]))
    out[:, 0::2] = gp
    out[:, 1::2] = gn
    return out


def fc_tiles(B: int = 4096, seed: int = 0, tile: int = 128, v_max: float = 0.3,
             circuit: Circuit = Circuit(1.0, 2.5, 2.5, 10.0), g_lo=1e-6, g_hi=1e-4,
             layers=((784, 256), (256, 10))):
    """Tiles of the 784->256->10 net: weights N(0, 0.05) -> differential conductances -> tiles.

    Layer 1 (784 x 512 after the differential split) gives 6 x 4 tiles of
    128 x 128 plus 4 tiles of 16 x 128; layer 2 (256 x 20) gives 2 tiles of
    128 x 20: 30 tiles.  Tile t gets its own B x M voltages from
    default_rng(seed + 1 + t), uniform in [0, v_max].
    """
    rng = np.random.default_rng(seed)
    weights = [rng.normal(0.0, 0.05, size=shape) for shape in layers]
    tiles = []
    for li, w in enumerate(weights):
        Gl = _differential(w, g_lo, g_hi)
        R, C = Gl.shape
        for r0 in range(0, R, tile):
            for c0 in range(0, C, tile):
                Gt = np.ascontiguousarray(Gl[r0:r0 + tile, c0:c0 + tile])
                tiles.append(Tile(li, r0, c0, Gt, None, circuit))
    for t, tl in enumerate(tiles):
        trng = np.random.default_rng(seed + 1 + t)
        tl.V = voltages(trng, B, tl.G.shape[0], v_max)
    return tiles


# ---------------------------------------------------------------------------------------------
# surrogate data: many conductance maps, each with its own input batch
# ---------------------------------------------------------------------------------------------
def maps(n_maps: int, M: int, N: int, B: int, seed: int, g_lo=1e-6, g_hi=1e-4, v_max=0.5):
    """List of (G, V) pairs; map m uses default_rng([seed, m])."""
    out = []
    for m in range(n_maps):
        rng = np.random.default_rng([seed, m])
        G = conductances(rng, M, N, g_lo, g_hi)
        V = voltages(rng, B, M, v_max)
        out.append((G, V))
    return out
