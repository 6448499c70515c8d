"""Synthetic gauge fields and right-hand sides for the HISQ Dslash workloads.

Conventions (shared by every consumer of these arrays):

* Lattice ``L = (Lx, Ly, Lz, Lt)``, every extent even.  Lexicographic site index
  ``i = x + Lx*(y + Ly*(z + Lz*t))``; parity ``(x+y+z+t) mod 2``; the even-odd index of a
  site inside its parity is ``i // 2`` (a bijection onto ``[0, V/2)`` because Lx is even).
* Direction mu = 0, 1, 2, 3 is x, y, z, t.
* Canonical link array: complex128 ``[4 mu][V][3][3]`` (row a, column b), which as float64
  is ``double[4][V][3][3][2]`` (re, im interleaved).
* Canonical even-odd vector: complex128 ``[V/2][3]`` per right-hand side.

The fields follow the synthetic recipe used throughout this project:

* random SU(3): ``U = exp(i * eps * H)`` with ``H = sum_a h_a lambda_a / 2``, ``h_a ~ N(0,1)``
  (Gell-Mann basis), computed with the Cayley-Hamilton closed form of exp(iQ) for traceless
  Hermitian Q (Morningstar and Peardon 2004), equal to the spectral definition to rounding;
* fat link: ``X_{x,mu} = eta_mu(x) b_mu(x) (U_{x,mu} o (1 + 0.05 xi))`` with xi an i.i.d.
  complex Gaussian per matrix entry (E|xi|^2 = 1), so X is not unitary, like a smeared link;
* Naik link: ``N_{x,mu} = eta_mu(x) b3_mu(x) (-1/24) U'_{x,mu} U'_{x+mu,mu} U'_{x+2mu,mu}``
  from a separately seeded field U';
* staggered phases ``eta_mu(x) = (-1)^(sum_{nu<mu} x_nu)`` folded into both links;
* fermion boundary condition antiperiodic in t, folded into the links: ``b_t = -1`` on the
  fat link leaving t = Lt-1 and on the Naik link whose three hops cross t = Lt-1.
"""
from __future__ import annotations

import concurrent.futures
import os
from dataclasses import dataclass

import numpy as np

SEED_FAT_U = 1
SEED_FAT_NOISE = 2
SEED_NAIK_U = 3
SEED_RHS_BASE = 1000
SEED_GAUGE_TRANSFORM = 7

_GELL_MANN = np.zeros((8, 3, 3), dtype=np.complex128)
_GELL_MANN[0][0, 1] = _GELL_MANN[0][1, 0] = 1
_GELL_MANN[1][0, 1], _GELL_MANN[1][1, 0] = -1j, 1j
_GELL_MANN[2][0, 0], _GELL_MANN[2][1, 1] = 1, -1
_GELL_MANN[3][0, 2] = _GELL_MANN[3][2, 0] = 1
_GELL_MANN[4][0, 2], _GELL_MANN[4][2, 0] = -1j, 1j
_GELL_MANN[5][1, 2] = _GELL_MANN[5][2, 1] = 1
_GELL_MANN[6][1, 2], _GELL_MANN[6][2, 1] = -1j, 1j
_GELL_MANN[7] = np.diag([1, 1, -2]) / np.sqrt(3)


@dataclass(frozen=True)
class Lattice:
    """Lattice extents (Lx, Ly, Lz, Lt); all must be even and >= 2."""

    dims: tuple

    def __post_init__(self):
        if len(self.dims) != 4 or any(int(d) < 2 or int(d) % 2 for d in self.dims):
            raise ValueError(f"lattice extents must be four even numbers >= 2, got {self.dims}")
        object.__setattr__(self, "dims", tuple(int(d) for d in self.dims))

    @property
    def volume(self) -> int:
        return int(np.prod(self.dims))

    @property
    def half_volume(self) -> int:
        return self.volume // 2

    def coords(self) -> np.ndarray:
        """int64 [V][4] coordinates in lexicographic order."""
        lx, ly, lz, lt = self.dims
        i = np.arange(self.volume, dtype=np.int64)
        return np.stack([i % lx, (i // lx) % ly, (i // (lx * ly)) % lz, i // (lx * ly * lz)], axis=1)

    def parity(self) -> np.ndarray:
        return self.coords().sum(axis=1) % 2

    def eo_sites(self, parity: int) -> np.ndarray:
        """Lexicographic indices of the sites of one parity, ordered by even-odd index."""
        lex = np.nonzero(self.parity() == parity)[0]
        assert np.array_equal(lex // 2, np.arange(self.half_volume))
        return lex

    def _grid(self, a: np.ndarray) -> np.ndarray:
        """View a [..., V, ...] array as [..., Lt, Lz, Ly, Lx, ...] (site axis at position 1)."""
        lx, ly, lz, lt = self.dims
        return a.reshape(a.shape[:1] + (lt, lz, ly, lx) + a.shape[2:])


def _exp_i_traceless_hermitian(q: np.ndarray) -> np.ndarray:
    """exp(iQ) for a batch of traceless Hermitian 3x3 matrices by the Cayley-Hamilton closed form
    of Morningstar and Peardon (2004): exp(iQ) = f0 + f1 Q + f2 Q^2, with the f_j functions of
    c0 = det Q and c1 = tr(Q^2) / 2 only.  Vectorised over the batch; matches the spectral
    definition q exp(i w) q^dagger to rounding."""
    q2 = np.einsum("nij,njk->nik", q, q)
    c1 = 0.5 * np.einsum("nii->n", q2).real
    c0 = (q[:, 0, 0] * (q[:, 1, 1] * q[:, 2, 2] - q[:, 1, 2] * q[:, 2, 1])
          - q[:, 0, 1] * (q[:, 1, 0] * q[:, 2, 2] - q[:, 1, 2] * q[:, 2, 0])
          + q[:, 0, 2] * (q[:, 1, 0] * q[:, 2, 1] - q[:, 1, 1] * q[:, 2, 0])).real
    neg = c0 < 0
    c0 = np.abs(c0)                       # f_j(-c0) = (-1)^j conj(f_j(c0))
    tiny = c1 < 1e-14
    c1s = np.where(tiny, 1.0, c1)
    c0max = 2.0 * (c1s / 3.0) ** 1.5
    theta = np.arccos(np.clip(c0 / c0max, -1.0, 1.0))
    u = np.sqrt(c1s / 3.0) * np.cos(theta / 3.0)
    w = np.sqrt(c1s) * np.sin(theta / 3.0)
    w2 = w * w
    small = np.abs(w) < 0.05
    xi0 = np.where(small, 1.0 - w2 / 6.0 * (1.0 - w2 / 20.0 * (1.0 - w2 / 42.0)),
                   np.sin(w) / np.where(small, 1.0, w))
    e2iu, emiu = np.exp(2j * u), np.exp(-1j * u)
    cw = np.cos(w)
    u2 = u * u
    h0 = (u2 - w2) * e2iu + emiu * (8.0 * u2 * cw + 2j * u * (3.0 * u2 + w2) * xi0)
    h1 = 2.0 * u * e2iu - emiu * (2.0 * u * cw - 1j * (3.0 * u2 - w2) * xi0)
    h2 = e2iu - emiu * (cw + 3j * u * xi0)
    den = 9.0 * u2 - w2
    f = [h / den for h in (h0, h1, h2)]
    f = [np.where(neg, (-1) ** j * np.conj(fj), fj) for j, fj in enumerate(f)]
    eye = np.eye(3)
    out = f[0][:, None, None] * eye + f[1][:, None, None] * q + f[2][:, None, None] * q2
    if np.any(tiny):                      # Q ~ 0: the series to second order is exact to rounding
        qt, q2t = q[tiny], q2[tiny]
        out[tiny] = eye + 1j * qt - 0.5 * q2t
    return out


def _workers() -> int:
    return max(1, min(8, os.cpu_count() or 1))


def random_su3(rng: np.random.Generator, count: int, eps: float) -> np.ndarray:
    """``count`` matrices exp(i*eps*H), H = sum_a h_a lambda_a/2 with h_a ~ N(0, 1).  The draws
    come first, in order; the exponentials of fixed chunks then run on a few threads (numpy
    releases the GIL), each matrix computed exactly as in a serial loop."""
    h = rng.standard_normal((count, 8))
    out = np.empty((count, 3, 3), np.complex128)
    chunk = 1 << 20

    def one(i0):
        q = eps * np.einsum("na,aij->nij", h[i0:i0 + chunk], _GELL_MANN / 2)
        out[i0:i0 + chunk] = _exp_i_traceless_hermitian(q)

    starts = range(0, count, chunk)
    if len(starts) > 1:
        with concurrent.futures.ThreadPoolExecutor(_workers()) as ex:
            list(ex.map(one, starts))
    else:
        for i0 in starts:
            one(i0)
    return out


def staggered_phases(lat: Lattice) -> np.ndarray:
    """float64 [4][V]: eta_mu(x) = (-1)^(sum_{nu<mu} x_nu)."""
    c = lat.coords()
    eta = np.ones((4, lat.volume))
    for mu in range(1, 4):
        eta[mu] = np.where(c[:, :mu].sum(axis=1) % 2 == 0, 1.0, -1.0)
    return eta


def boundary_signs(lat: Lattice, hops: int, antiperiodic_t: bool = True) -> np.ndarray:
    """float64 [4][V]: -1 on links whose ``hops`` steps in t cross the t boundary (else +1)."""
    b = np.ones((4, lat.volume))
    if antiperiodic_t:
        t = lat.coords()[:, 3]
        b[3] = np.where(t + hops >= lat.dims[3], -1.0, 1.0)
    return b


def _fold(lat: Lattice, links: np.ndarray, hops: int, antiperiodic_t: bool) -> np.ndarray:
    sign = staggered_phases(lat) * boundary_signs(lat, hops, antiperiodic_t)
    return links * sign[:, :, None, None]


def fat_links(lat: Lattice, eps: float = 0.3, noise: float = 0.05,
              seed_u: int = SEED_FAT_U, seed_noise: int = SEED_FAT_NOISE,
              antiperiodic_t: bool = True) -> np.ndarray:
    """Synthetic fat links X, complex128 [4][V][3][3], drawn in [mu][site] order."""
    v = lat.volume
    u = random_su3(np.random.default_rng(seed_u), 4 * v, eps).reshape(4, v, 3, 3)
    rng = np.random.default_rng(seed_noise)
    xi = (rng.standard_normal((4, v, 3, 3)) + 1j * rng.standard_normal((4, v, 3, 3))) * np.sqrt(0.5)
    return _fold(lat, u * (1.0 + noise * xi), 1, antiperiodic_t)


def naik_links(lat: Lattice, eps: float = 0.3, seed_u: int = SEED_NAIK_U,
               antiperiodic_t: bool = True) -> np.ndarray:
    """Synthetic Naik links N = -(1/24) U'_{x} U'_{x+mu} U'_{x+2mu}, complex128 [4][V][3][3]."""
    v = lat.volume
    u = random_su3(np.random.default_rng(seed_u), 4 * v, eps).reshape(4, v, 3, 3)
    out = np.empty_like(u)

    def one(mu):
        axis = 3 - mu  # grid axes are (t, z, y, x) after the leading direction axis is dropped
        g = lat._grid(u[mu:mu + 1])[0]
        g1 = np.roll(g, -1, axis=axis)
        g2 = np.roll(g, -2, axis=axis)
        out[mu] = (g @ g1 @ g2).reshape(v, 3, 3)

    with concurrent.futures.ThreadPoolExecutor(min(4, _workers())) as ex:
        list(ex.map(one, range(4)))
    return _fold(lat, -out / 24.0, 3, antiperiodic_t)


def free_field_links(lat: Lattice, c1: float = 9.0 / 8.0, c3: float = -1.0 / 24.0,
                     antiperiodic_t: bool = True):
    """Unit-link (free) field: X = c1 eta b 1 and N = c3 eta b3 1."""
    eye = np.broadcast_to(np.eye(3, dtype=np.complex128), (4, lat.volume, 3, 3))
    return (_fold(lat, c1 * eye, 1, antiperiodic_t), _fold(lat, c3 * eye, 3, antiperiodic_t))


def gaussian_rhs(lat: Lattice, k: int, seed_base: int = SEED_RHS_BASE, sites: int | None = None) -> np.ndarray:
    """Complex Gaussian vector with E|z|^2 = 1 per component, complex128 [V/2][3] (seed base+k)."""
    n = lat.half_volume if sites is None else sites
    rng = np.random.default_rng(seed_base + k)
    z = rng.standard_normal((n, 3, 2)) * np.sqrt(0.5)
    return z[..., 0] + 1j * z[..., 1]


def z2_rhs(lat: Lattice, k: int, seed_base: int = SEED_RHS_BASE) -> np.ndarray:
    """Z2 noise: every colour component is +1 or -1 (real), complex128 [V/2][3]."""
    rng = np.random.default_rng(seed_base + k)
    return (2.0 * rng.integers(0, 2, size=(lat.half_volume, 3)) - 1.0).astype(np.complex128)


def gauge_transform_field(lat: Lattice, seed: int = SEED_GAUGE_TRANSFORM, eps: float = 3.0) -> np.ndarray:
    """Random SU(3) matrix per site, complex128 [V][3][3]."""
    return random_su3(np.random.default_rng(seed), lat.volume, eps)


def even_odd_embed(lat: Lattice, v_even: np.ndarray, parity: int = 0) -> np.ndarray:
    """Place an even-odd vector [V/2][3] on the sites of ``parity`` of a zero full-lattice field."""
    full = np.zeros((lat.volume, 3), dtype=np.complex128)
    full[lat.eo_sites(parity)] = v_even
    return full
