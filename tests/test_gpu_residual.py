"""The FP64-accurate residual r = b - A x of the reliable updates (Sec. 1's operator
A = m^2 - D_eo D_oe from Eq. (3)), computed through hisq_residual: double-single arithmetic on the
FP32 pipe for FP32/FP16/BF16 link handles, native FP64 for FP64 handles, against the FP64 oracle."""
import numpy as np
import pytest

import hisq_inputs as hi
from gpu_util import gpu, rel_err

pytestmark = pytest.mark.gpu

MASS = 0.05


def _residual(g, b, x, mass=MASS):
    n = len(b)
    r = np.empty_like(b)
    res2 = np.zeros(n)
    g.hisq.hisq_residual(g.fat, g.naik, mass, np.ascontiguousarray(b), np.ascontiguousarray(x), r, n, res2)
    return r, res2


@pytest.mark.parametrize("prec", [1, 2, 3, 0])
@pytest.mark.parametrize("dims,n", [((8, 8, 8, 6), 1), ((12, 10, 8, 6), 3)])
def test_residual_matches_oracle(prec, dims, n):
    """Random x: every component of b - A x within 1e-12 (norm-wise, per right-hand side) of the
    oracle's FP64 value, and |r|^2 reported alongside."""
    with gpu(dims, prec) as g:
        b = np.stack([hi.gaussian_rhs(g.lat, 100 + k) for k in range(n)])
        x = np.stack([hi.gaussian_rhs(g.lat, 200 + k) for k in range(n)])
        r, res2 = _residual(g, b, x)
        want = b - np.stack([g.oracle.aop(x[k], MASS) for k in range(n)])
        assert rel_err(r, want) <= 1e-12
        assert np.allclose(res2, np.sum(np.abs(want.reshape(n, -1)) ** 2, axis=1), rtol=1e-11)


@pytest.mark.parametrize("prec", [2, 1])
def test_residual_at_convergence(prec):
    """x = the oracle's CG solution to 1e-10: the residual is ten orders of magnitude below the
    terms it is formed from (m^2 x and D_eo D_oe x, both larger than b), and the library's agrees
    with the oracle's to 1e-12 |b| (the double-single products and sums carry 48 significant bits,
    2^-48 = 3.6e-15 of those terms), so both see the same |r| / |b| to 1%, well within the 5% the
    solvers leave below tol."""
    with gpu((8, 8, 8, 6), prec) as g:
        b = hi.gaussian_rhs(g.lat, 300)
        x, _, _ = g.oracle.cg(b, MASS, 1e-10)
        r, res2 = _residual(g, b[None], x[None])
        want = g.oracle.true_residual(b, x, MASS)[0]
        bn = np.linalg.norm(b)
        assert np.linalg.norm(r[0] - (b - g.oracle.aop(x, MASS))) <= 1e-12 * bn
        assert abs(np.sqrt(res2[0]) / bn - want) <= 0.01 * want
