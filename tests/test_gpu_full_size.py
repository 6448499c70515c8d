"""Parity at the workload sizes: 48^3 x 12 bundles of 16 right-hand sides with uneven
convergence, 64^3 x 16 bundles of Z2-noise right-hand sides with 16-bit storage, and the
preconditioner network on 32^3 x 8.  The links are generated once per lattice; the oracle checks
whole outputs where it takes seconds and sampled right-hand sides where a full check would take
minutes (the GPU's own FP64 true residual covers the rest)."""
import numpy as np
import pytest

import hisq_inputs as hi
from gpu_util import PREC_TOL, gpu, rel_err

pytestmark = pytest.mark.gpu

TOL = 1e-10
SLACK = 1.0   # the library stops at 0.95 tol, so the oracle's own FP64 residual is within tol
D48 = (48, 48, 48, 12)
D64 = (64, 64, 64, 16)


@pytest.fixture(scope="module")
def fields48():
    lat = hi.Lattice(D48)
    return hi.fat_links(lat), hi.naik_links(lat)


@pytest.fixture(scope="module")
def fields64():
    lat = hi.Lattice(D64)
    return hi.fat_links(lat), hi.naik_links(lat)


def shaped_rhs(o, lat, n, mass, seed=2000):
    """b_k = s_k A^{q_k} g_k / |A^{q_k} g_k|: norms s_k log-uniform in [1e-3, 1e3] and spectral
    shaping q_k = k mod 3 (with a relative tolerance the norm alone does not change the
    iteration count; the shaping does)."""
    s = 10.0 ** np.random.default_rng(seed).uniform(-3.0, 3.0, n)
    out = []
    for k in range(n):
        g = hi.gaussian_rhs(lat, seed + k)
        for _ in range(k % 3):
            g = o.aop(g, mass)
        out.append(s[k] * g / np.linalg.norm(g))
    return out


def _solve(g, rhs, mass, **params):
    p = g.hisq.hisq_default_solver_params()
    for k, v in params.items():
        setattr(p, k, v)
    g.hisq.hisq_set_solver_params(p)
    xs = [np.zeros_like(b) for b in rhs]
    g.hisq.hisq_cg_solve(g.fat, g.naik, list(rhs), xs, mass, TOL)
    iters = np.zeros(len(rhs), dtype=np.int32)
    res = np.zeros(len(rhs))
    stats = g.hisq.hisq_last_stats(iters, res)
    return xs, stats, iters, res


def test_dslash_48c12_fp32_bundle16_autotuned(fields48):
    """16 right-hand sides in one autotuned launch: whole output of D_eo against the oracle,
    and D_oe on two sampled right-hand sides."""
    n = 16
    with gpu(D48, 1, 18, fields48) as g:
        g.hisq.hisq_autotune(g.fat, g.naik, n)
        v = np.stack([hi.gaussian_rhs(g.lat, 300 + k) for k in range(n)])
        vin, vout = g.pack(v), g.bundle(n)
        g.hisq.hisq_dslash(g.fat, g.naik, vin, vout, n, 0)
        assert rel_err(g.unpack(vout, n), g.oracle.dslash_eo(v, 0)) <= PREC_TOL[1]
        g.hisq.hisq_dslash(g.fat, g.naik, vin, vout, n, 1)
        got = g.unpack(vout, n)
        for k in (3, 12):
            assert rel_err(got[k:k + 1], g.oracle.dslash_eo(v[k:k + 1], 1)) <= PREC_TOL[1], k


def test_cg_48c12_uneven_bundle_graph_and_persistent(fields48):
    """m = 0.002, FP32 storage, a bundle of 16 right-hand sides with norms across 1e-3..1e3 and
    spectral shaping: every one reaches the FP64 true residual 1e-10 (GPU check on all, oracle
    on two), the converged ones are masked while the others iterate, and the captured graph and
    the persistent kernel run the same iterations (up to rounding)."""
    mass, n = 0.002, 16
    with gpu(D48, 1, 18, fields48) as g:
        rhs = shaped_rhs(g.oracle, g.lat, n, mass)
        runs = {}
        for driver in (1, 2):
            xs, s, iters, res = _solve(g, rhs, mass, inner_prec=1, use_graph=driver, bundle=n)
            assert s.converged == n and np.all(res <= TOL), (driver, res)
            runs[driver] = (xs, iters)
        assert np.all(np.abs(runs[1][1].astype(int) - runs[2][1].astype(int)) <= 1)
        iters = runs[2][1]
        assert iters.max() > iters.min()  # uneven convergence inside the bundle
        xs = runs[2][0]
        for k in (0, 7):
            assert g.oracle.true_residual(rhs[k], xs[k], mass)[0] <= TOL * SLACK, k


def test_dslash_64c16_fp16_z2_bundle16(fields64):
    """The largest lattice, 16-bit storage, 16 Z2-noise right-hand sides in one launch; the
    oracle checks two sampled right-hand sides."""
    n = 16
    with gpu(D64, 2, 18, fields64) as g:
        g.hisq.hisq_autotune(g.fat, g.naik, n)
        v = np.stack([hi.z2_rhs(g.lat, 4000 + k) for k in range(n)])
        vin, vout = g.pack(v), g.bundle(n)
        g.hisq.hisq_dslash(g.fat, g.naik, vin, vout, n, 0)
        got = g.unpack(vout, n)
        for k in (0, 9):
            assert rel_err(got[k:k + 1], g.oracle.dslash_eo(v[k:k + 1], 0)) <= PREC_TOL[2], k


def test_cg_64c16_z2_fp16_bundle(fields64):
    """m = 0.002, FP16 storage with FP64 reliable updates, 16 Z2-noise right-hand sides in one
    bundle: all reach 1e-10 by the GPU's FP64 check; the oracle re-checks two."""
    mass, n = 0.002, 16
    with gpu(D64, 2, 18, fields64) as g:
        rhs = [hi.z2_rhs(g.lat, 4100 + k) for k in range(n)]
        xs, s, iters, res = _solve(g, rhs, mass, inner_prec=2, bundle=n)
        assert s.converged == n and np.all(res <= TOL), res
        assert s.reliable_updates >= n
        for k in (2, 13):
            assert g.oracle.true_residual(rhs[k], xs[k], mass)[0] <= TOL * SLACK, k


def test_network_forward_32c8():
    """The preconditioner network on the 32^3 x 8 lattice it is trained on: GPU forward of two
    right-hand sides with random weights against the oracle's forward."""
    dims = (32, 32, 32, 8)
    rng = np.random.default_rng(11)
    W = (rng.standard_normal(408) + 1j * rng.standard_normal(408)) * 0.3
    with gpu(dims, 1, 18) as g:
        r = np.stack([hi.gaussian_rhs(g.lat, 600 + k) for k in range(2)])
        pc = g.hisq.hisq_pc_create(np.ascontiguousarray(W).view(np.float64))
        try:
            vin, vout = g.pack(r), g.bundle(2)
            g.hisq.hisq_pc_apply(pc, g.fat, g.naik, vin, vout, 2)
            got = g.unpack(vout, 2)
        finally:
            g.hisq.hisq_pc_destroy(pc)
        want = np.stack([g.oracle.pc_forward(W, r[k]) for k in range(2)])
        assert rel_err(got, want) <= 3e-5


def test_multishift_32c8_fp16_eight_shifts():
    """The multi-shift workload: 32^3 x 8, m = 0.01, shifts 0 and 1e-4..1, FP16 shared iteration
    with FP64 refinement: every shift to 1e-10 by the GPU's FP64 check; the oracle re-checks the
    hardest and the lightest shift."""
    import math
    dims, mass = (32, 32, 32, 8), 0.01
    shifts = (0.0,) + tuple(float(v) for v in 10.0 ** np.linspace(-4.0, 0.0, 7))
    with gpu(dims, 2, 18) as g:
        b = hi.gaussian_rhs(g.lat, 7000)
        p = g.hisq.hisq_default_solver_params()
        p.inner_prec = 2
        g.hisq.hisq_set_solver_params(p)
        xs = [np.zeros_like(b) for _ in shifts]
        g.hisq.hisq_cg_multishift(g.fat, g.naik, b, xs, shifts, mass, TOL)
        res = np.zeros(len(shifts))
        s = g.hisq.hisq_last_stats(None, res)
        assert s.converged == len(shifts) and np.all(res <= TOL), res
        for j in (0, len(shifts) - 1):
            m_j = math.sqrt(mass * mass + shifts[j])
            assert g.oracle.true_residual(b, xs[j], m_j)[0] <= TOL * SLACK, j
