"""Plain FP64 CPU oracle of the even-odd HISQ Dslash, A = m^2 - D_eo D_oe, CG, multi-shift CG,
flexible CG and the gauge-covariant preconditioner network (C library loaded through ctypes).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the benchmark's
CPU-baseline leg may use it; the CUDA library never does.  It shares no code with the CUDA
path.  Arrays are numpy complex128 in the canonical layouts:
links ``[4][V][3][3]``, full-lattice vectors ``[nrhs][V][3]``, even-odd vectors ``[nrhs][V/2][3]``.
"""
import ctypes
import os

import numpy as np

from . import build as _build

_lib = None

_D = ctypes.POINTER(ctypes.c_double)
_I4 = ctypes.c_int * 4


def lib(path: str | None = None):
    """Load (building if needed) the oracle library.  ``path`` selects another build of it."""
    global _lib
    if path is not None:
        return _bind(ctypes.CDLL(path))
    if _lib is None:
        _lib = _bind(ctypes.CDLL(_build.build()))
    return _lib


def _bind(so):
    so.oracle_dslash_full.argtypes = [_I4, _D, _D, _D, _D, ctypes.c_int]
    so.oracle_dslash_eo.argtypes = [_I4, _D, _D, _D, _D, ctypes.c_int, ctypes.c_int]
    so.oracle_aop.argtypes = [_I4, _D, _D, ctypes.c_double, _D, _D, ctypes.c_int]
    so.oracle_cg.argtypes = [_I4, _D, _D, ctypes.c_double, _D, _D, ctypes.c_double, ctypes.c_int, _D]
    so.oracle_cg.restype = ctypes.c_int
    so.oracle_pc_layer.argtypes = [_I4, _D, _D, ctypes.c_int, ctypes.c_int, _D, _D, _D]
    so.oracle_pc_num_weights.restype = ctypes.c_long
    so.oracle_pc_forward.argtypes = [_I4, _D, _D, _D, _D, _D]
    so.oracle_pc_loss_grad.argtypes = [_I4, _D, _D, ctypes.c_double, _D, ctypes.c_int, _D, _D, _D]
    so.oracle_pc_loss_grad.restype = ctypes.c_double
    so.oracle_adam_step.argtypes = [ctypes.c_long, _D, _D, _D, _D, ctypes.c_int,
                                    ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double]
    so.oracle_pc_backward.argtypes = [_I4, _D, _D, _D, _D, _D, _D]
    so.oracle_pc_adjoint.argtypes = [_I4, _D, _D, _D, _D, _D]
    so.oracle_pc_loss_grad_normal.argtypes = [_I4, _D, _D, ctypes.c_double, _D, ctypes.c_int, _D, _D, _D]
    so.oracle_pc_loss_grad_normal.restype = ctypes.c_double
    so.oracle_fcg.argtypes = [_I4, _D, _D, ctypes.c_double, _D, _D, _D, ctypes.c_double, ctypes.c_int, _D,
                              ctypes.c_int]
    so.oracle_fcg.restype = ctypes.c_int
    so.oracle_cg_multishift.argtypes = [_I4, _D, _D, ctypes.c_double, _D, ctypes.c_int, _D, _D, ctypes.c_double,
                                        ctypes.c_int, ctypes.POINTER(ctypes.c_int), _D]
    so.oracle_cg_multishift.restype = ctypes.c_int
    so.oracle_splitmix64.argtypes = [ctypes.c_ulonglong, ctypes.c_ulonglong]
    so.oracle_splitmix64.restype = ctypes.c_ulonglong
    so.oracle_z2_noise.argtypes = [_I4, ctypes.c_ulonglong, ctypes.c_ulonglong, ctypes.c_int, _D]
    so.oracle_trace_inverse.argtypes = [_I4, _D, _D, ctypes.c_double, ctypes.c_int, ctypes.c_ulonglong, ctypes.c_double,
                                        _D]
    so.oracle_trace_inverse.restype = ctypes.c_double
    return so


def _c(a, dtype=np.complex128):
    return np.ascontiguousarray(a, dtype=dtype)


def _p(a):
    return a.ctypes.data_as(_D)


class Oracle:
    """The oracle bound to one lattice and one pair of link fields (X fat, N Naik)."""

    def __init__(self, dims, fat, naik, so_path: str | None = None):
        self.dims = tuple(int(d) for d in dims)
        self.V = int(np.prod(self.dims))
        self.X = _c(fat).reshape(4, self.V, 3, 3)
        self.N = _c(naik).reshape(4, self.V, 3, 3)
        self._so = lib(so_path)
        self._L = _I4(*self.dims)

    def dslash_full(self, v):
        """Eq. (3) on the whole lattice; v: [V][3] or [nrhs][V][3]."""
        v = _c(v)
        shape = v.shape
        v = v.reshape(-1, self.V, 3)
        out = np.empty_like(v)
        self._so.oracle_dslash_full(self._L, _p(self.X), _p(self.N), _p(v), _p(out), v.shape[0])
        return out.reshape(shape)

    def dslash_eo(self, v, out_parity: int):
        """Eq. (3)/(4) restricted to output parity: v [.., V/2, 3] on parity 1-out_parity."""
        v = _c(v)
        shape = v.shape
        v = v.reshape(-1, self.V // 2, 3)
        out = np.empty_like(v)
        self._so.oracle_dslash_eo(self._L, _p(self.X), _p(self.N), _p(v), _p(out), v.shape[0], int(out_parity))
        return out.reshape(shape)

    def aop(self, v, mass: float):
        """A v = m^2 v - D_eo D_oe v on even sites; v [.., V/2, 3]."""
        v = _c(v)
        shape = v.shape
        v = v.reshape(-1, self.V // 2, 3)
        out = np.empty_like(v)
        self._so.oracle_aop(self._L, _p(self.X), _p(self.N), float(mass), _p(v), _p(out), v.shape[0])
        return out.reshape(shape)

    def cg(self, b, mass: float, tol: float = 1e-10, max_iter: int = 10000):
        """Plain FP64 CG on A from x0 = 0: returns (x, iterations or -1, true relative residual)."""
        b = _c(b).reshape(self.V // 2, 3)
        x = np.empty_like(b)
        rel = ctypes.c_double()
        it = self._so.oracle_cg(self._L, _p(self.X), _p(self.N), float(mass), _p(b), _p(x),
                                float(tol), int(max_iter), ctypes.byref(rel))
        return x, it, rel.value

    def true_residual(self, b, x, mass: float):
        """|b - A x| / |b| in FP64 for each right-hand side; b, x [.., V/2, 3]."""
        b = _c(b).reshape(-1, self.V // 2, 3)
        x = _c(x).reshape(-1, self.V // 2, 3)
        r = b - self.aop(x, mass)
        return np.linalg.norm(r.reshape(r.shape[0], -1), axis=1) / np.linalg.norm(b.reshape(b.shape[0], -1), axis=1)

    # ---- preconditioner network -------------------------------------------------------
    @property
    def pc_num_weights(self) -> int:
        return int(self._so.oracle_pc_num_weights())

    def pc_layer(self, W, h, cin: int, cout: int):
        """One network layer; W [17][cout][cin], h [cin][V][3] -> [cout][V][3]."""
        W = _c(W).reshape(17, cout, cin)
        h = _c(h).reshape(cin, self.V, 3)
        out = np.empty((cout, self.V, 3), dtype=np.complex128)
        self._so.oracle_pc_layer(self._L, _p(self.X), _p(self.N), cin, cout, _p(W), _p(h), _p(out))
        return out

    def pc_forward(self, W, r):
        """Network output on even sites for an even-site input r [V/2][3]."""
        W = _c(W).reshape(-1)
        r = _c(r).reshape(self.V // 2, 3)
        y = np.empty_like(r)
        self._so.oracle_pc_forward(self._L, _p(self.X), _p(self.N), _p(W), _p(r), _p(y))
        return y

    def pc_loss_grad(self, W, r, e, mass: float, with_grad: bool = True):
        """(loss, grad) over K pairs r, e [K][V/2][3] with A e = r:
        loss = mean_k |A (M r_k - e_k)|^2 / |r_k|^2; grad = dL/dReW + i dL/dImW."""
        W = _c(W).reshape(-1)
        r = _c(r).reshape(-1, self.V // 2, 3)
        e = _c(e).reshape(-1, self.V // 2, 3)
        g = np.zeros_like(W)
        loss = self._so.oracle_pc_loss_grad(self._L, _p(self.X), _p(self.N), float(mass), _p(W), r.shape[0],
                                            _p(r), _p(e), _p(g) if with_grad else None)
        return loss, g

    def pc_adjoint(self, W, u):
        """The adjoint network N^dag u on even sites (u [V/2][3])."""
        W = _c(W).reshape(-1)
        u = _c(u).reshape(self.V // 2, 3)
        y = np.empty_like(u)
        self._so.oracle_pc_adjoint(self._L, _p(self.X), _p(self.N), _p(W), _p(u), _p(y))
        return y

    def pc_normal(self, W, r):
        """The normal form M r = N^dag N r."""
        return self.pc_adjoint(W, self.pc_forward(W, r))

    def pc_loss_grad_normal(self, W, r, e, mass: float, with_grad: bool = True):
        """(loss, grad) of the normal form: mean_k |A (N^dag N r_k - e_k)|^2 / |r_k|^2."""
        W = _c(W).reshape(-1)
        r = _c(r).reshape(-1, self.V // 2, 3)
        e = _c(e).reshape(-1, self.V // 2, 3)
        g = np.zeros_like(W)
        loss = self._so.oracle_pc_loss_grad_normal(self._L, _p(self.X), _p(self.N), float(mass), _p(W), r.shape[0],
                                                   _p(r), _p(e), _p(g) if with_grad else None)
        return loss, g

    def pc_backward(self, W, r, gy):
        """Weight gradient (layout of W) for one input r given dL/dRe y + i dL/dIm y on even sites."""
        W = _c(W).reshape(-1)
        r = _c(r).reshape(self.V // 2, 3)
        gy = _c(gy).reshape(self.V // 2, 3)
        g = np.zeros_like(W)
        self._so.oracle_pc_backward(self._L, _p(self.X), _p(self.N), _p(W), _p(r), _p(gy), _p(g))
        return g

    def fcg(self, W, b, mass: float, tol: float = 1e-10, max_iter: int = 10000, form: int = 0):
        """Flexible CG with the network as preconditioner (form 0: M, 1: M^dag M, 2: the Hermitian
        part of M); returns (x, iterations or -1, true rel).  x is the iterate reached, also when
        max_iter ends the run first."""
        W = _c(W).reshape(-1)
        b = _c(b).reshape(self.V // 2, 3)
        x = np.empty_like(b)
        rel = ctypes.c_double()
        it = self._so.oracle_fcg(self._L, _p(self.X), _p(self.N), float(mass), _p(W), _p(b), _p(x),
                                 float(tol), int(max_iter), ctypes.byref(rel), int(form))
        return x, it, rel.value

    def cg_multishift(self, b, shifts, mass: float, tol: float = 1e-10, max_iter: int = 10000):
        """Multi-shift CG: x_j = (A + shifts[j])^{-1} b from one Krylov space.  Returns
        (x [nshift][V/2][3], base iterations or -1, per-shift stop iterations, per-shift true
        relative residuals)."""
        b = _c(b).reshape(self.V // 2, 3)
        sh = np.ascontiguousarray(shifts, dtype=np.float64).reshape(-1)
        ns = sh.size
        x = np.empty((ns, self.V // 2, 3), dtype=np.complex128)
        its = np.zeros(ns, dtype=np.int32)
        rel = np.zeros(ns)
        it = self._so.oracle_cg_multishift(self._L, _p(self.X), _p(self.N), float(mass), _p(b), ns, _p(sh),
                                           _p(x), float(tol), int(max_iter),
                                           its.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _p(rel))
        return x, it, its, rel

    def trace_inverse(self, mass: float, nnoise: int, seed: int, tol: float = 1e-10):
        """Z2-noise estimate of Tr A^{-1} on the even sites: (mean, per-noise samples)."""
        samples = np.empty(nnoise)
        mean = self._so.oracle_trace_inverse(self._L, _p(self.X), _p(self.N), float(mass), int(nnoise),
                                             seed & (2**64 - 1), float(tol), _p(samples))
        return mean, samples


def splitmix64(seed: int, i: int) -> int:
    """The i-th output (from 0) of the splitmix64 generator started from seed."""
    return int(lib().oracle_splitmix64(seed & (2**64 - 1), i))


def z2_noise(dims, seed: int, first: int, n: int):
    """n Z2 noise vectors [n][V/2][3] (complex, real parts +-1) of stream seed, from vector first."""
    vh = int(np.prod(dims)) // 2
    out = np.empty((n, vh, 3), dtype=np.complex128)
    lib().oracle_z2_noise(_I4(*dims), seed & (2**64 - 1), first, n, _p(out))
    return out


def adam_step(theta, grad, m, v, t: int, lr: float, b1: float = 0.9, b2: float = 0.999, eps: float = 1e-8):
    """One Adam step in place on float64 arrays (real parameters)."""
    for a in (theta, grad, m, v):
        assert a.dtype == np.float64 and a.flags.c_contiguous
    lib().oracle_adam_step(theta.size, _p(theta), _p(grad), _p(m), _p(v), int(t),
                           float(lr), float(b1), float(b2), float(eps))
