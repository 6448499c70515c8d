"""hisq_aop_noalloc: the A-operator for callers that cannot allocate device memory.

Its scratch (odd-parity intermediate, reduction partials, block counter) lives in a static
device array inside the library, so it can serve code whose device memory belongs to another
allocator or whose hot path must not call cudaMalloc.  Checked through the C ABI against
hisq_aop, which allocates its scratch, on two calls in a row (the second call reuses the array
the first one left behind).  The file name sorts last so a run that stops at the first failure
has already run every other test.
"""
import numpy as np
import pytest

import hisq_inputs as hi
from gpu_util import PREC_TOL, gpu, rel_err

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec,n", [(1, 1), (1, 4), (2, 3), (0, 2), (3, 4)])
def test_noalloc_matches_aop_twice(prec, n):
    mass = 0.1
    with gpu((8, 10, 8, 6), prec) as g:
        for call in range(2):
            v = np.stack([hi.gaussian_rhs(g.lat, 10 * call + k) for k in range(n)])
            vin = g.pack(v)
            ref, out = g.bundle(n), g.bundle(n)
            pap_ref, pap = np.zeros(n), np.zeros(n)
            g.hisq.hisq_aop(g.fat, g.naik, mass, vin, ref, n, pap_ref)
            out.fill_(0xFF)
            g.hisq.hisq_aop_noalloc(g.fat, g.naik, mass, vin, out, n, pap)
            want = g.unpack(ref, n)
            assert rel_err(g.unpack(out, n), want) <= PREC_TOL[prec], call
            assert np.max(np.abs(pap - pap_ref) / np.abs(pap_ref)) <= PREC_TOL[prec], call


def test_noalloc_rejects_sizes_beyond_the_static_scratch():
    from paper_1409_1510_gb300 import hisq
    with gpu((32, 32, 32, 8), 1) as g:
        n = 8   # FP32 intermediate of 25 MB > 15 MiB of scratch
        vin, out = g.bundle(n), g.bundle(n)
        with pytest.raises(hisq.HisqError, match="static scratch"):
            g.hisq.hisq_aop_noalloc(g.fat, g.naik, 0.1, vin, out, n)


@pytest.mark.parametrize("prec", [1, 2])
def test_noalloc_first_call_on_a_fresh_context_matches_oracle(prec):
    """The first operator call of a new context goes through the static scratch (hisq_aop has not
    run, so no workspace exists yet) and equals the oracle's A = m^2 - D_eo D_oe."""
    mass = 0.1
    with gpu((8, 8, 8, 6), prec) as g:
        v = np.stack([hi.gaussian_rhs(g.lat, 30 + k) for k in range(2)])
        out = g.bundle(2)
        pap = np.zeros(2)
        g.hisq.hisq_aop_noalloc(g.fat, g.naik, mass, g.pack(v), out, 2, pap)
        want = np.stack([g.oracle.aop(v[k], mass) for k in range(2)])
        assert rel_err(g.unpack(out, 2), want) <= 2 * PREC_TOL[prec]
        pap_want = np.array([np.vdot(v[k], want[k]).real for k in range(2)])
        assert np.max(np.abs(pap - pap_want) / np.abs(pap_want)) <= 4 * PREC_TOL[prec]
