"""Shared helpers for the GPU parity tests: oracle results cached per session, error metrics."""
from __future__ import annotations

import functools

import numpy as np

import oracle
from paper_2410_19993_gb300 import inputs


def rel_err(I, Iref):
    """max over (b, j) of |I - I*| / |I*|: the relative current error (guarded denominator)."""
    I = np.asarray(I)
    Iref = np.asarray(Iref)
    return float(np.max(np.abs(I - Iref) / np.maximum(np.abs(Iref), 1e-300)))


@functools.lru_cache(maxsize=16)
def oracle_factor(M, N, R, seed=0, g_lo=1e-6, g_hi=1e-4):
    G, _ = inputs.crossbar(M, N, 0, seed, g_lo, g_hi)
    return G, oracle.factor(M, N, G, *R)


@functools.lru_cache(maxsize=16)
def oracle_transfer(M, N, R, seed=0):
    _, f = oracle_factor(M, N, R, seed)
    return oracle.transfer_matrix(f)


def oracle_transfer_of(args):
    """The oracle's transfer matrix of one (G, R) pair (a process-pool worker: numpy and the oracle
    only)."""
    G, R = args
    return oracle.transfer_matrix(oracle.factor(G.shape[0], G.shape[1], G, *R))


def case(M, N, B, R, seed=0, v_max=0.5):
    """(G, V) drawn with the workload recipe; G first, then V (same stream as inputs.crossbar)."""
    return inputs.crossbar(M, N, B, seed, v_max=v_max)
