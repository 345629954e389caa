"""The C ABI without a GPU: the library builds, loads, exports every symbol
declared in include/kadabra.h, and its host-side steps (omega, computeDelta)
agree bit for bit with the oracle.  Compute calls are not made here."""

import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "kadabra.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = set(re.findall(r"\b(kadabra_[a-z_0-9]+)\s*\(", text))
    return sorted(names)


@pytest.fixture(scope="module")
def kd():
    from paper_1604_08553_gb300 import kadabra
    kadabra.load_library()
    return kadabra


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("kadabra_load_csr", "kadabra_run", "kadabra_free_graph", "kadabra_sample_batch",
                 "kadabra_sample_paths", "kadabra_check", "kadabra_compute_delta"):
        assert must in names


def test_library_exports_every_declared_symbol(kd):
    lib = kd.load_library()
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def header_enum(prefix):
    """name -> value of the header's enumerators KADABRA_<prefix>..."""
    text = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    return {m.group(1): int(m.group(2)) for m in re.finditer(r"\bKADABRA_(" + prefix + r"[A-Z0-9_]*)\s*=\s*(\d+)", text)}


def test_binding_constants_match_the_header(kd):
    """Every status, flag and work-counter constant of the binding has the
    header's value, and the binding names all of them."""
    for prefix in ("ERR_", "FLAG_"):
        enum = header_enum(prefix)
        assert enum, prefix
        for name, value in enum.items():
            assert getattr(kd, name) == value, name
    stats = header_enum("STAT_")
    assert len(kd.STAT_NAMES) == kd.NSTAT == len(stats)
    for name, value in stats.items():
        assert kd.STAT_NAMES[value] == name[len("STAT_"):].lower(), name


def test_config_defaults(kd):
    cfg = kd.config_default()
    assert cfg.eps == 0.001 and cfg.check_interval == 1000 and cfg.vd == 0 and not cfg.stream


def test_omega_matches_oracle_bitwise(kd, orc):
    rng = np.random.default_rng(1)
    for _ in range(500):
        lam = float(rng.uniform(1e-4, 0.2))
        delta = float(rng.uniform(1e-4, 0.9))
        vd = int(rng.integers(0, 10**6))
        assert kd.kadabra_omega(lam, delta, vd) == orc.omega(lam, delta, vd)


def _assert_delta_equal(kd, orc, count0, alpha, omega, lam, delta, eps):
    C1, l1, u1 = kd.kadabra_compute_delta(count0, alpha, omega, lam, delta, eps)
    C2, l2, u2 = orc.compute_delta(count0, alpha, omega, lam, delta, eps)
    assert C1 == C2
    assert np.array_equal(l1, l2) and np.array_equal(u1, u2)


def test_compute_delta_matches_oracle_bitwise(kd, orc, er2000):
    lam, delta, eps = 0.01, 0.1, 0.001
    vd = orc.vd_bound(er2000)
    omega = orc.omega(lam, delta, vd)
    alpha = max(1, int(omega // 100))
    rc, count0, _ = orc.accumulate(er2000, seed=1, domain=1, first_idx=0, count=alpha)
    assert rc == 0
    _assert_delta_equal(kd, orc, count0, alpha, omega, lam, delta, eps)
    rng = np.random.default_rng(2)
    for trial in range(6):
        n = int(rng.integers(2, 5000))
        c0 = (rng.poisson(0.5, n) * rng.integers(0, 50, n)).astype(np.uint32)
        a = int(rng.integers(1, 2000))
        om = float(rng.uniform(100, 2e5))
        _assert_delta_equal(kd, orc, c0, a, om, float(rng.uniform(0.002, 0.05)), 0.1, [0.001, 0.0001][trial % 2])
    _assert_delta_equal(kd, orc, np.zeros(100, dtype=np.uint32), 10, 5000.0, 0.01, 0.1, 0.001)
    _assert_delta_equal(kd, orc, np.full(7, 3, dtype=np.uint32), 10, 5000.0, 0.01, 0.1, 0.001)


def test_without_gpu_the_library_fails_loudly(kd, er2000):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(kd.KadabraError):
        kd.kadabra_load_csr(er2000)
