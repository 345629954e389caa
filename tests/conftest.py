"""Shared fixtures.  GPU tests carry the `gpu` marker; everything else runs on CPU."""

import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running (still part of the default run)")


@pytest.fixture(scope="session")
def gg():
    from paper_1604_08553_gb300 import graphgen
    return graphgen


@pytest.fixture(scope="session")
def orc():
    import oracle
    return oracle


@pytest.fixture(scope="session")
def er2000(gg):
    """Erdos-Renyi G(n=2000, avg degree 8), seed 1, largest component."""
    return gg.erdos_renyi(2000, 8.0, 1)


@pytest.fixture(scope="session")
def chung_lu_1m(gg):
    """Chung-Lu n=10^6, beta=2.5, mean degree 16, max 10^4, seed 1, largest component."""
    return gg.chung_lu(1_000_000, 2.5, 16.0, 10_000.0, 1)


def random_graph(gg, n, p, seed, directed=False):
    rng = np.random.default_rng(seed)
    if directed:
        e = [(i, j) for i in range(n) for j in range(n) if i != j and rng.random() < p]
    else:
        e = [(i, j) for i in range(n) for j in range(i + 1, n) if rng.random() < p]
    return gg.from_edges(n, e, directed=directed, name=f"rand{n}_{p}_{seed}_{int(directed)}")
