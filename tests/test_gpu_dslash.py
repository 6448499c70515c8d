"""Link packing, Dslash (Eq. (3), (4)) and A-operator on the GPU through the C ABI, element by element against the FP64 oracle."""
import numpy as np
import pytest

import hisq_inputs as hi
from gpu_util import PREC_TOL, gpu, rel_err

pytestmark = pytest.mark.gpu

# 8 x 10 x 8 x 6: V/2 = 1920 output sites, several site tiles plus a ragged last tile; the hops
# +-1 and +-3 reach distinct sites in x, y and z.
DIMS = (8, 10, 8, 6)
CASES = [(0, 18), (1, 18), (1, 13), (1, 9), (2, 18), (2, 13), (2, 9), (3, 18), (3, 13), (3, 9)]


def _rhs(lat, n, seed=0):
    return np.stack([hi.gaussian_rhs(lat, seed + k) for k in range(n)])


@pytest.mark.parametrize("prec,recon", CASES)
@pytest.mark.parametrize("n", [1, 3, 4, 12, 16])
def test_dslash_parity(prec, recon, n):
    with gpu(DIMS, prec, recon) as g:
        v = _rhs(g.lat, n)
        vin = g.pack(v)
        vout = g.bundle(n)
        for parity in (0, 1):
            g.hisq.hisq_dslash(g.fat, g.naik, vin, vout, n, parity)
            err = rel_err(g.unpack(vout, n), g.oracle.dslash_eo(v, parity))
            assert err <= PREC_TOL[prec], (parity, err)


@pytest.mark.parametrize("prec", [0, 1, 2, 3])
def test_every_launch_shape(prec):
    """Each compiled right-hand-sides-per-thread variant and several block sizes agree."""
    n = 8
    with gpu(DIMS, prec, 18) as g:
        v = _rhs(g.lat, n, 40)
        want = g.oracle.dslash_eo(v, 1)
        vin, vout = g.pack(v), g.bundle(n)
        for R in (1, 2, 4, 8):
            if prec == 0 and R == 8:
                continue
            for S in (1, 2, 4, 8):
                if min(S, 4) * R > 8 or (S == 8 and prec == 0):
                    continue
                for threads in ((32, 96, 256) if S < 8 else (32 * (n // R), 64 * (n // R))):
                    g.hisq.hisq_set_launch_shape(prec, 18, n, R, threads, S)
                    vout.zero_()
                    g.hisq.hisq_dslash(g.fat, g.naik, vin, vout, n, 1)
                    assert rel_err(g.unpack(vout, n), want) <= PREC_TOL[prec], (R, S, threads)


@pytest.mark.parametrize("prec", [0, 1, 2, 3])
@pytest.mark.parametrize("n", [1, 3])
def test_lane_split_with_fused_epilogues(prec, n):
    """The two-lane (fat / Naik) and four-lane (two directions of one kind) splits, and the
    four-lane split with staged link records, with the A-operator epilogue and its fused dot."""
    mass = 0.2
    with gpu(DIMS, prec, 18) as g:
        v = _rhs(g.lat, n, 80)
        for S in ((1, 2, 4) if prec == 0 else (1, 2, 4, 8)):
            g.hisq.hisq_set_launch_shape(prec, 18, n, 1, 128 if S < 8 else 32 * 4 * n, S)
            vin, vout = g.pack(v), g.bundle(n)
            pap = np.zeros(n)
            g.hisq.hisq_aop(g.fat, g.naik, mass, vin, vout, n, pap)
            assert rel_err(g.unpack(vout, n), g.oracle.aop(v, mass)) <= 2 * PREC_TOL[prec], S
            vq = g.unpack(vin, n)
            want_dot = np.array([np.vdot(vq[k], g.oracle.aop(vq[k], mass)).real for k in range(n)])
            assert np.max(np.abs(pap - want_dot) / np.abs(want_dot)) <= 4 * PREC_TOL[prec], S


def test_dslash_max_nrhs_and_single_site_row():
    """HISQ_MAX_NRHS right-hand sides in one call, and the smallest lattice (4^4)."""
    with gpu((4, 4, 4, 4), 1, 18) as g:
        v = _rhs(g.lat, 64, 100)
        vin, vout = g.pack(v), g.bundle(64)
        g.hisq.hisq_dslash(g.fat, g.naik, vin, vout, 64, 0)
        assert rel_err(g.unpack(vout, 64), g.oracle.dslash_eo(v, 0)) <= 1e-5


def test_dslash_zero_input_gives_zero():
    with gpu(DIMS, 2, 18) as g:
        v = np.zeros((2, g.lat.half_volume, 3), complex)
        vin, vout = g.pack(v), g.bundle(2)
        g.hisq.hisq_dslash(g.fat, g.naik, vin, vout, 2, 0)
        assert np.all(g.unpack(vout, 2) == 0)


@pytest.mark.parametrize("prec,recon", CASES)
def test_links_export_matches_gathered_links(prec, recon):
    """The packed links decode to X_{x,mu} and -X^dag_{x-mu,mu} (N with 3 hops) of the
    canonical input, within the storage precision."""
    dims = (8, 4, 6, 4)
    with gpu(dims, prec, recon) as g:
        lat = g.lat
        c = lat.coords()
        for handle, U, hop in ((g.fat, g.X, 1), (g.naik, g.N, 3)):
            out = np.empty((2, lat.half_volume, 8, 3, 3, 2))
            g.hisq.hisq_links_export(handle, out)
            got = out.view(np.complex128)[..., 0]
            for parity in (0, 1):
                sites = lat.eo_sites(parity)
                want = np.empty((lat.half_volume, 8, 3, 3), complex)
                for mu in range(4):
                    cc = c[sites].copy()
                    cc[:, mu] = (cc[:, mu] - hop) % dims[mu]
                    back = cc[:, 0] + dims[0] * (cc[:, 1] + dims[1] * (cc[:, 2] + dims[2] * cc[:, 3]))
                    want[:, 2 * mu] = U[mu][sites]
                    want[:, 2 * mu + 1] = -U[mu][back].conj().swapaxes(-1, -2)
                scale = np.abs(want).max()
                err = np.abs(got[parity] - want).max() / scale
                # the 9-real encoding divides by |W01|^2 + |W02|^2, which is small for links near
                # the identity (its singular point), so its rounding error is amplified
                bound = {0: 1e-15, 1: 1e-6, 2: 2e-3, 3: 1e-2}[prec] * {18: 1, 13: 10, 9: 300}[recon]
                assert err <= bound, (parity, err)


@pytest.mark.parametrize("prec", [0, 1, 2, 3])
@pytest.mark.parametrize("n", [1, 5, 16])
def test_aop_and_fused_dot(prec, n):
    """A p = m^2 p - D_eo D_oe p with the fused <p, A p> in FP64."""
    mass = 0.1
    with gpu(DIMS, prec, 18) as g:
        v = _rhs(g.lat, n, 7)
        vin, vout = g.pack(v), g.bundle(n)
        pap = np.zeros(n)
        g.hisq.hisq_aop(g.fat, g.naik, mass, vin, vout, n, pap)
        want = g.oracle.aop(v, mass)
        assert rel_err(g.unpack(vout, n), want) <= 2 * PREC_TOL[prec]
        vq = g.unpack(vin, n)  # the input as stored
        want_dot = np.array([np.vdot(vq[k], g.oracle.aop(vq[k], mass)).real for k in range(n)])
        assert np.max(np.abs(pap - want_dot) / np.abs(want_dot)) <= 4 * PREC_TOL[prec]


@pytest.mark.parametrize("prec", [1, 2])
def test_full_size_dslash_32c8(prec):
    """The 32^3 x 8 lattice the benchmark runs, whole output against the oracle, n = 1 and 4."""
    dims = (32, 32, 32, 8)
    with gpu(dims, prec, 18) as g:
        for n in (1, 4):
            v = _rhs(g.lat, n, 500)
            vin, vout = g.pack(v), g.bundle(n)
            g.hisq.hisq_dslash(g.fat, g.naik, vin, vout, n, 0)
            assert rel_err(g.unpack(vout, n), g.oracle.dslash_eo(v, 0)) <= PREC_TOL[prec]


def test_launch_shape_validation():
    """Lane splits exist only for 18-real Naik records and few right-hand sides per thread."""
    from paper_1409_1510_gb300.hisq import HisqError
    with gpu(DIMS, 1, 18) as g:
        h = g.hisq
        h.hisq_set_launch_shape(1, 18, 4, 2, 128, 4)
        for bad in ((1, 18, 4, 4, 128, 4), (1, 13, 4, 1, 128, 2), (1, 18, 4, 1, 128, 3)):
            with pytest.raises(HisqError):
                h.hisq_set_launch_shape(*bad)


@pytest.mark.parametrize("prec", [1, 2, 3])
def test_staged_tiles_cover_ragged_lattice_and_report_no_timeout(prec):
    """The staged kernel on a lattice whose half volume is not a multiple of its tile (the last
    tile's bulk copies are shorter), more tiles than blocks (both stages reused), then the
    device status: no bounded wait ran out."""
    dims = (6, 10, 6, 8)  # V/2 = 1440: 11 tiles of 128 sites plus 32, 22 of 64 plus 32, 45 of 32
    with gpu(dims, prec, 18) as g:
        # FP32 records are twice as large: half the tile for one right-hand side
        for n, R, threads in ((1, 1, 512 if prec != 1 else 256), (2, 2, 256), (3, 1, 384)):
            g.hisq.hisq_set_launch_shape(prec, 18, n, R, threads, 8)
            v = _rhs(g.lat, n, 90)
            vin, vout = g.pack(v), g.bundle(n)
            for parity in (0, 1):
                g.hisq.hisq_dslash(g.fat, g.naik, vin, vout, n, parity)
                assert rel_err(g.unpack(vout, n), g.oracle.dslash_eo(v, parity)) <= PREC_TOL[prec], (n, parity)
        g.hisq.hisq_device_status()


@pytest.mark.parametrize("prec", [0, 1, 2])
def test_full_lattice_dslash_matches_eq3(prec):
    """Eq. (3) as printed, on both parities: the two halves of the output against the oracle's
    full-lattice Dslash of the same full-lattice input."""
    n = 2
    with gpu(DIMS, prec, 18) as g:
        lat = g.lat
        rng = np.random.default_rng(31)
        v = (rng.standard_normal((n, lat.volume, 3)) + 1j * rng.standard_normal((n, lat.volume, 3))) * np.sqrt(0.5)
        ev, od = lat.eo_sites(0), lat.eo_sites(1)
        half = g.hisq.hisq_vector_bytes(prec, n)
        vin = g.torch.empty(2 * half, dtype=g.torch.uint8, device=g.dev)
        vout = g.torch.empty_like(vin)
        vin[:half].copy_(g.pack(v[:, ev]))
        vin[half:].copy_(g.pack(v[:, od]))
        g.hisq.hisq_dslash_full(g.fat, g.naik, vin, vout, n)
        want = g.oracle.dslash_full(v)
        got = np.empty_like(v)
        got[:, ev] = g.unpack(vout[:half], n)
        got[:, od] = g.unpack(vout[half:], n)
        assert rel_err(got, want) <= PREC_TOL[prec]


def test_fma_peaks_are_measured():
    """The FP32 and FP64 FMA throughput the ALU-bound rooflines divide by: positive, FP32 far
    above FP64 on this part."""
    with gpu((4, 4, 4, 4), 1, 18) as g:
        f32, f64 = g.hisq.hisq_measure_fma_peaks()
        assert 1.0 < f32 < 1000.0 and 0.01 < f64 < 1000.0 and f32 > 4 * f64
