"""Stochastic traces (Eq. (2) without derivative factors) on the GPU through the C ABI: the Z2
noise bit for bit against the oracle's generator, and the Tr A^{-1} estimate, noise vector by noise
vector, against the oracle's estimate on the same noise."""
import numpy as np
import pytest

import hisq_inputs as hi
import oracle
from gpu_util import gpu

pytestmark = pytest.mark.gpu

DIMS = (8, 10, 8, 6)
TOL = 1e-10


def test_z2_noise_matches_oracle_bit_for_bit():
    with gpu(DIMS, 1) as g:
        n, seed, first = 3, 0x123456789ABCDEF, 5
        out = g.torch.empty((n, g.lat.half_volume, 3, 2), dtype=g.torch.float64, device=g.dev)
        g.hisq.hisq_z2_noise(out, n, seed, first)
        got = out.cpu().numpy().view(np.complex128)[..., 0]
        want = oracle.z2_noise(DIMS, seed, first, n)
        assert np.array_equal(got, want)


@pytest.mark.parametrize("prec", [0, 1, 2])
def test_trace_inverse_matches_oracle_estimate(prec):
    """Each noise vector's eta^dag A^{-1} eta agrees with the oracle's (solutions to the FP64
    true residual 1e-10 on both sides: relative agreement far inside 1e-7), so the estimate and
    its error do too; 20 vectors in bundles."""
    mass, nnoise, seed = 0.1, 20, 77
    with gpu(DIMS, prec) as g:
        p = g.hisq.hisq_default_solver_params()
        p.inner_prec = prec
        g.hisq.hisq_set_solver_params(p)
        samples = np.zeros(nnoise)
        est, err, _ = g.hisq.hisq_trace_inverse(g.fat, g.naik, mass, nnoise, seed, TOL, samples)
        want_mean, want = g.oracle.trace_inverse(mass, nnoise, seed, TOL)
        assert np.max(np.abs(samples - want) / np.abs(want)) <= 1e-7
        assert abs(est - want_mean) <= 1e-7 * abs(want_mean)
        assert abs(err - np.std(want, ddof=1) / np.sqrt(nnoise)) <= 1e-6 * abs(err)
        res = np.zeros(nnoise)
        s = g.hisq.hisq_last_stats(None, res)
        assert s.nrhs == nnoise and s.converged == nnoise and np.all(res <= TOL)


def test_trace_inverse_single_noise_and_arguments():
    with gpu(DIMS, 1) as g:
        est, err, _ = g.hisq.hisq_trace_inverse(g.fat, g.naik, 0.1, 1, 3, TOL)
        assert np.isfinite(est) and err == 0.0
        assert g.hisq.hisq_trace_inverse(g.fat, g.naik, 0.1, 0, 3, TOL, raise_on_error=False)[2] == -1
