"""The FP64 oracle against what the paper and the mathematics fix (CPU only)."""
import os

import numpy as np
import pytest

import oracle
import oracle_pins as pins
from paper_1409_1510_gb300 import accounting

HERE = os.path.dirname(os.path.abspath(__file__))


def make(dims, X, N):
    return oracle.Oracle(dims, X, N)


@pytest.mark.parametrize("pin", pins.ALL_PINS, ids=lambda f: f.__name__)
def test_pin(pin):
    ok, detail = pin(make)
    assert ok, detail


def test_matrix_form_distinguishes_naik_hops():
    """On L = 8 the hops +-1 and +-3 reach distinct sites, so the matrix-form check also covers
    the Naik addressing (on L = 4, x+3mu is x-mu)."""
    ok, detail = pins.pin_matrix_form(make, dims=(8, 8, 8, 8))
    assert ok, detail


def _table1():
    rows = []
    with open(os.path.join(HERE, "golden", "table1_flop_per_byte.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                n, full, r14 = line.split()
                rows.append((int(n), float(full), float(r14)))
    return rows


def test_table1_arithmetic_intensity():
    """Table 1: 1146 flop per site and RHS over 16 links (18 or 14 reals for Naik) and 17
    colour vectors per RHS, in single precision, reproduces every printed value."""
    assert accounting.DSLASH_FLOPS_PER_SITE == 1146
    for n, full, r14 in _table1():
        assert abs(accounting.paper_model_intensity(n) - full) <= 0.005 + 1e-12, n
        assert abs(accounting.paper_model_intensity(n, naik_reals=14) - r14) <= 0.005 + 1e-12, n


def test_table1_derived_statements():
    """Statements after Table 1: the n -> infinity limit 1146/408 ~ 2.8 ("~2.75"), n = 8 at ~75%
    of it, n = 1 at 25-30%, and the Naik reconstruction gain ~10% (n=1) falling to ~3% (n=8)."""
    limit = accounting.DSLASH_FLOPS_PER_SITE / (17 * 6 * 4)
    assert 2.7 < limit < 2.85
    assert 0.72 < accounting.paper_model_intensity(8) / limit < 0.76
    for reals in (18, 14):
        assert 0.25 <= accounting.paper_model_intensity(1, reals) / limit <= 0.30
    g1 = accounting.paper_model_intensity(1, 14) / accounting.paper_model_intensity(1) - 1
    g8 = accounting.paper_model_intensity(8, 14) / accounting.paper_model_intensity(8) - 1
    assert 0.08 < g1 < 0.11 and 0.02 < g8 < 0.04


def test_adam_closed_form():
    """Adam with a constant gradient moves every parameter by lr * g / (|g| + eps) per step
    (bias correction makes m_hat = g and v_hat = g^2 exactly)."""
    rng = np.random.default_rng(3)
    theta = rng.standard_normal(50)
    g = rng.standard_normal(50)
    m = np.zeros(50); v = np.zeros(50)
    start = theta.copy()
    lr, eps = 1e-2, 1e-8
    for t in range(1, 6):
        oracle.adam_step(theta, g, m, v, t, lr, 0.9, 0.999, eps)
    np.testing.assert_allclose(theta, start - 5 * lr * g / (np.abs(g) + eps), rtol=0, atol=1e-12)


def test_splitmix64_published_outputs():
    """The noise generator reproduces the published first outputs of splitmix64 from seed 0."""
    rows = []
    with open(os.path.join(HERE, "golden", "splitmix64_seed0.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                i, h = line.split()
                rows.append((int(i), int(h, 16)))
    assert rows and all(oracle.splitmix64(0, i) == v for i, v in rows)


def test_z2_noise_signs_follow_the_generator():
    """Noise vector k, component e = 3 s + c is -1 exactly when the top bit of generator output
    (3 V/2) k + e is set; both signs occur in balance."""
    dims, seed = (4, 4, 4, 6), 5
    eta = oracle.z2_noise(dims, seed, 2, 3)
    per = eta.shape[1] * 3
    flat = eta.reshape(3, -1)
    for k in range(3):
        for e in (0, 1, per // 2, per - 1):
            top = oracle.splitmix64(seed, (2 + k) * per + e) >> 63
            assert flat[k, e] == (-1.0 if top else 1.0)
    assert np.all(eta.imag == 0) and np.all(np.abs(eta.real) == 1.0)
    assert abs(eta.real.mean()) < 0.1
