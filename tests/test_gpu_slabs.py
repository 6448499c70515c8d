"""The Dslash of Eq. (3)-(4) through the domain decomposition along t (hisq_slabs_*): the lattice
cut into slabs with depth-3 ghost planes, face packing, halo copies on a second stream, interior
and boundary kernels.  Checked against the FP64 oracle at the per-Dslash bounds, and bit for bit
against the undecomposed library Dslash with the same launch shape (the slabs apply the same links
to the same neighbour values in the same order)."""
import numpy as np
import pytest

import hisq_inputs as hi
from gpu_util import PREC_TOL, gpu, rel_err

pytestmark = pytest.mark.gpu


def _slab_dslash(g, h, v, parity, ms=None):
    torch = g.torch
    n = len(v)
    vin = g._dev64(np.ascontiguousarray(v))
    vout = torch.empty_like(vin)
    g.hisq.hisq_slabs_dslash(h, vin, vout, n, parity, ms)
    return vout.cpu().numpy().view(np.complex128).reshape(n, g.lat.half_volume, 3)


@pytest.mark.parametrize("dims,nslab", [((8, 8, 8, 16), 2), ((8, 6, 4, 8), 2), ((6, 4, 8, 16), 4)])
@pytest.mark.parametrize("prec", [1, 0, 2])
@pytest.mark.parametrize("n", [1, 16])
def test_slab_dslash_matches_oracle(dims, nslab, prec, n):
    """Slabs of 8 planes (interior and boundary kernels) and of 4 (boundary only); both parities."""
    with gpu(dims, prec) as g:
        h = g.hisq.hisq_slabs_create(g._dev64(g.X), g._dev64(g.N), prec, nslab)
        try:
            for parity in (0, 1):
                v = np.stack([hi.gaussian_rhs(g.lat, 70 + k) for k in range(n)])
                got = _slab_dslash(g, h, v, parity)
                want = g.oracle.dslash_eo(v, parity)
                assert rel_err(got, want) <= PREC_TOL[prec], (parity, rel_err(got, want))
        finally:
            g.hisq.hisq_slabs_destroy(h)


@pytest.mark.parametrize("prec", [1, 2])
def test_slab_dslash_equals_undecomposed(prec):
    """Same launch shape: the decomposed Dslash reproduces hisq_dslash bit for bit, and reports
    its face-packing, interior, halo and total times."""
    dims, n = (8, 8, 8, 16), 4
    with gpu(dims, prec) as g:
        g.hisq.hisq_set_launch_shape(prec, 18, n, 2, 128, 1)
        h = g.hisq.hisq_slabs_create(g._dev64(g.X), g._dev64(g.N), prec, 2)
        try:
            v = np.stack([hi.gaussian_rhs(g.lat, 90 + k) for k in range(n)])
            ms = np.zeros(4)
            got = _slab_dslash(g, h, v, 1, ms)
            vin = g.pack(v)
            vout = g.bundle(n)
            g.hisq.hisq_dslash(g.fat, g.naik, vin, vout, n, 1)
            want = g.unpack(vout, n)
            assert np.array_equal(got, want)
            assert np.all(ms >= 0) and ms[3] > 0
        finally:
            g.hisq.hisq_slabs_destroy(h)


def test_slab_arguments_are_checked():
    with gpu((8, 8, 8, 12), 1) as g:
        with pytest.raises(Exception):
            g.hisq.hisq_slabs_create(g._dev64(g.X), g._dev64(g.N), 1, 4)   # 3 planes per slab
        with pytest.raises(Exception):
            g.hisq.hisq_slabs_create(g._dev64(g.X), g._dev64(g.N), 1, 5)   # 12 / 5
