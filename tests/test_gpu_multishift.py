"""Multi-shift CG on the GPU through the C ABI.  Every shift is checked by the FP64 oracle's true
residual of its own system A + sigma_j = (m^2 + sigma_j) - D_eo D_oe, and the FP64 iteration also
by the oracle's multi-shift iterates."""
import math

import numpy as np
import pytest

import hisq_inputs as hi
from gpu_util import gpu

pytestmark = pytest.mark.gpu

TOL = 1e-10
SLACK = 1.0   # the library stops at 0.95 tol, so the oracle's own FP64 residual is within tol
DIMS = (8, 10, 8, 6)
MASS = 0.05                                    # m^2 = 0.0025
SHIFTS = (0.003, 0.0, 0.05, -0.002, 1.0, 0.3)  # unsorted, one negative (> -m^2)


def _ms(g, b, shifts, mass, **params):
    p = g.hisq.hisq_default_solver_params()
    for k, v in params.items():
        setattr(p, k, v)
    g.hisq.hisq_set_solver_params(p)
    xs = [np.zeros_like(b) for _ in shifts]
    g.hisq.hisq_cg_multishift(g.fat, g.naik, b, xs, shifts, mass, TOL)
    iters = np.zeros(len(shifts), dtype=np.int32)
    res = np.zeros(len(shifts))
    stats = g.hisq.hisq_last_stats(iters, res)
    return np.stack(xs), stats, iters, res


def _true(g, b, xs, shifts, mass):
    return np.array([g.oracle.true_residual(b, xs[j], math.sqrt(mass * mass + s))[0] for j, s in enumerate(shifts)])


@pytest.mark.parametrize("driver", [2, 1])
def test_fp64_multishift_matches_oracle(driver):
    """FP64 throughout, shared iteration as the persistent kernel (2) or the captured graph (1):
    every shift meets the true residual, agrees with the oracle's multi-shift solution, and stops
    at the oracle's iteration (within two)."""
    with gpu(DIMS, 0) as g:
        b = hi.gaussian_rhs(g.lat, 21)
        xs, stats, iters, res = _ms(g, b, SHIFTS, MASS, inner_prec=0, use_graph=driver)
        assert np.all(_true(g, b, xs, SHIFTS, MASS) <= TOL * SLACK)
        assert np.all(res <= TOL) and stats.converged == len(SHIFTS)
        xo, it, its, rels = g.oracle.cg_multishift(b, SHIFTS, MASS, TOL)
        assert it > 0
        for j in range(len(SHIFTS)):
            assert np.linalg.norm(xs[j] - xo[j]) / np.linalg.norm(xo[j]) <= 1e-7, j
        assert np.all(np.abs(iters - its) <= 2 + stats.refine_iterations), (iters, its)
        assert abs(stats.shared_iterations - it) <= 2


@pytest.mark.parametrize("driver", [2, 1])
@pytest.mark.parametrize("prec", [1, 2, 3])
def test_mixed_precision_every_shift_reaches_fp64_residual(prec, driver):
    """Low-precision shared iteration plus FP64 defect correction per shift: every shift reaches
    the oracle's true residual 1e-10."""
    with gpu(DIMS, prec) as g:
        b = hi.gaussian_rhs(g.lat, 22)
        xs, stats, iters, res = _ms(g, b, SHIFTS, MASS, inner_prec=prec, use_graph=driver)
        true = _true(g, b, xs, SHIFTS, MASS)
        assert np.all(true <= TOL * SLACK), true
        assert stats.converged == len(SHIFTS) and np.all(res <= TOL)
        assert stats.shared_iterations > 0 and stats.refine_iterations > 0


def test_single_zero_shift_is_plain_cg():
    """One shift of zero: the solution of A x = b, in as many iterations as the plain CG solve."""
    with gpu(DIMS, 0) as g:
        b = hi.gaussian_rhs(g.lat, 23)
        xs, stats, iters, res = _ms(g, b, (0.0,), MASS, inner_prec=0)
        assert g.oracle.true_residual(b, xs[0], MASS)[0] <= TOL * SLACK
        _, it_cg, _ = g.oracle.cg(b, MASS, TOL)
        assert abs(int(iters[0]) - it_cg) <= 2


def test_zero_rhs_and_repeated_calls():
    """b = 0 gives x_j = 0 without iterating; two identical calls (the state reset at every call)
    give identical solutions; a call with other shifts of the same smallest shift still meets the
    residual."""
    with gpu(DIMS, 1) as g:
        zero = np.zeros((g.lat.half_volume, 3), dtype=np.complex128)
        xs, stats, _, res = _ms(g, zero, SHIFTS, MASS, inner_prec=1)
        assert np.all(xs == 0) and np.all(res == 0) and stats.shared_iterations == 0
        b = hi.gaussian_rhs(g.lat, 24)
        x1, s1, i1, _ = _ms(g, b, SHIFTS, MASS, inner_prec=1)
        x2, s2, i2, _ = _ms(g, b, SHIFTS, MASS, inner_prec=1)
        assert np.array_equal(x1, x2) and np.array_equal(i1, i2)
        other = (-0.002, 0.01, 0.7)
        x3, _, _, _ = _ms(g, b, other, MASS, inner_prec=1)
        assert np.all(_true(g, b, x3, other, MASS) <= TOL * SLACK)


def test_invalid_arguments_are_rejected():
    with gpu(DIMS, 1) as g:
        b = hi.gaussian_rhs(g.lat, 25)
        p = g.hisq.hisq_default_solver_params()
        g.hisq.hisq_set_solver_params(p)
        h = g.hisq
        bad_shift = h.hisq_cg_multishift(g.fat, g.naik, b, [np.zeros_like(b)], [-MASS * MASS], MASS, TOL,
                                         raise_on_error=False)
        assert bad_shift == -1
        many = [np.zeros_like(b) for _ in range(h.MAX_SHIFTS + 1)]
        assert h.hisq_cg_multishift(g.fat, g.naik, b, many, [0.0] * len(many), MASS, TOL, raise_on_error=False) == -1
        assert h.hisq_cg_multishift(g.fat, g.naik, b, [np.zeros_like(b)], [0.0], MASS, -1.0,
                                    raise_on_error=False) == -1


@pytest.mark.parametrize("prec", [0, 1])
def test_persistent_and_graph_shared_iterations_agree(prec):
    """The two drivers of the shared iteration run the same recurrences: the same number of
    shared iterations (within one: their block sums add in different orders) and, in FP64,
    solutions that agree as closely as the oracle's does with either (1e-7)."""
    with gpu(DIMS, prec) as g:
        b = hi.gaussian_rhs(g.lat, 24)
        out = {}
        for driver in (2, 1):
            xs, stats, iters, res = _ms(g, b, SHIFTS, MASS, inner_prec=prec, use_graph=driver)
            out[driver] = (xs, stats.shared_iterations)
        assert abs(out[2][1] - out[1][1]) <= 1, (out[2][1], out[1][1])
        if prec == 0:
            for j in range(len(SHIFTS)):
                d = np.linalg.norm(out[2][0][j] - out[1][0][j]) / np.linalg.norm(out[1][0][j])
                assert d <= 1e-7, (j, d)
