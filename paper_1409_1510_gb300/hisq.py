"""Thin ctypes binding of the C ABI in ``include/hisq.h`` (same names, argument marshalling only).

Every computation runs in ``libhisq_gb300.so``; if that library is missing this module raises
instead of falling back to anything else.  Pointer arguments accept torch tensors (their
``data_ptr()``), numpy arrays (host memory), raw integer addresses or None.
"""
from __future__ import annotations

import ctypes
import os

FP64, FP32, FP16, BF16 = 0, 1, 2, 3
MAX_BUNDLE = 16
MAX_NRHS = 64
PC_WEIGHTS = 408
MAX_SHIFTS = 16

STATUS = {0: "HISQ_OK", -1: "HISQ_ERR_ARG", -2: "HISQ_ERR_CUDA", -3: "HISQ_ERR_NOMEM",
          -4: "HISQ_ERR_NOT_CONVERGED", -5: "HISQ_ERR_BREAKDOWN", -6: "HISQ_ERR_TIMEOUT",
          -7: "HISQ_ERR_STATE"}

LIBRARY = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libhisq_gb300.so")


class HisqError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS.get(status, status)}: {message}")
        self.status = status


class hisq_solver_params(ctypes.Structure):
    _fields_ = [("inner_prec", ctypes.c_int), ("delta", ctypes.c_double), ("max_iter", ctypes.c_int),
                ("bundle", ctypes.c_int), ("use_graph", ctypes.c_int), ("check_every", ctypes.c_int),
                ("pc", ctypes.c_void_p), ("stall_window", ctypes.c_int), ("stall_factor", ctypes.c_double),
                ("autotune", ctypes.c_int), ("time_kernels", ctypes.c_int),
                ("debug_barrier_timeout", ctypes.c_int), ("persistent_threads", ctypes.c_int),
                ("single_reduction", ctypes.c_int), ("multishift_tol", ctypes.c_double),
                ("l2_persist_links", ctypes.c_int)]


class hisq_solve_stats(ctypes.Structure):
    _fields_ = [("nrhs", ctypes.c_int), ("converged", ctypes.c_int), ("bundles", ctypes.c_int),
                ("bundle_size", ctypes.c_int), ("max_iterations", ctypes.c_int),
                ("total_iterations", ctypes.c_long), ("bundle_iterations", ctypes.c_long),
                ("reliable_updates", ctypes.c_int), ("fallbacks", ctypes.c_int),
                ("seconds", ctypes.c_double), ("dslash_ms", ctypes.c_double),
                ("dslash_launches", ctypes.c_int), ("dslash64_ms", ctypes.c_double),
                ("dslash64_launches", ctypes.c_int), ("flops", ctypes.c_double),
                ("kernel_launches", ctypes.c_long), ("solve_kernel_ms", ctypes.c_double),
                ("solve_kernel_launches", ctypes.c_int), ("phase_ms", ctypes.c_double * 5),
                ("shared_iterations", ctypes.c_int), ("refine_iterations", ctypes.c_long),
                ("shared_seconds", ctypes.c_double), ("recompute_passes", ctypes.c_long)]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


_lib = None
_VP = ctypes.c_void_p
_I = ctypes.c_int
_D = ctypes.c_double

_SIGNATURES = {
    "hisq_init": ([ctypes.POINTER(_I), _I, _VP], _I),
    "hisq_finalize": ([], _I),
    "hisq_strerror": ([_I], ctypes.c_char_p),
    "hisq_last_error": ([], ctypes.c_char_p),
    "hisq_links_create": ([ctypes.POINTER(_VP), _VP, _I, _I, _I], _I),
    "hisq_links_destroy": ([_VP], _I),
    "hisq_links_export": ([_VP, _VP], _I),
    "hisq_vector_bytes": ([_I, _I], ctypes.c_size_t),
    "hisq_pack": ([_VP, _VP, _I, _I], _I),
    "hisq_unpack": ([_VP, _VP, _I, _I], _I),
    "hisq_dslash": ([_VP, _VP, _VP, _VP, _I, _I], _I),
    "hisq_aop": ([_VP, _VP, _D, _VP, _VP, _I, _VP], _I),
    "hisq_aop_noalloc": ([_VP, _VP, _D, _VP, _VP, _I, _VP], _I),
    "hisq_residual": ([_VP, _VP, _D, _VP, _VP, _VP, _I, _VP], _I),
    "hisq_slabs_create": ([ctypes.POINTER(_VP), _VP, _VP, _I, _I], _I),
    "hisq_slabs_destroy": ([_VP], _I),
    "hisq_slabs_dslash": ([_VP, _VP, _VP, _I, _I, _VP], _I),
    "hisq_default_solver_params": ([ctypes.POINTER(hisq_solver_params)], None),
    "hisq_set_solver_params": ([ctypes.POINTER(hisq_solver_params)], _I),
    "hisq_get_solver_params": ([ctypes.POINTER(hisq_solver_params)], _I),
    "hisq_cg_solve": ([_VP, _VP, ctypes.POINTER(_VP), ctypes.POINTER(_VP), _I, _D, _D], _I),
    "hisq_cg_multishift": ([_VP, _VP, _VP, ctypes.POINTER(_VP), _I, ctypes.POINTER(_D), _D, _D], _I),
    "hisq_z2_noise": ([_VP, _I, ctypes.c_ulonglong, ctypes.c_ulonglong], _I),
    "hisq_trace_inverse": ([_VP, _VP, _D, _I, ctypes.c_ulonglong, _D, ctypes.POINTER(_D), ctypes.POINTER(_D), _VP], _I),
    "hisq_last_stats": ([ctypes.POINTER(hisq_solve_stats), _VP, _VP], _I),
    "hisq_autotune": ([_VP, _VP, _I, ctypes.POINTER(_I), ctypes.POINTER(_I), ctypes.POINTER(_I)], _I),
    "hisq_set_launch_shape": ([_I, _I, _I, _I, _I, _I], _I),
    "hisq_pc_create": ([ctypes.POINTER(_VP), _VP], _I),
    "hisq_pc_destroy": ([_VP], _I),
    "hisq_pc_set_weights": ([_VP, _VP], _I),
    "hisq_pc_get_weights": ([_VP, _VP], _I),
    "hisq_pc_apply": ([_VP, _VP, _VP, _VP, _VP, _I], _I),
    "hisq_device_status": ([], _I),
    "hisq_dslash_full": ([_VP, _VP, _VP, _VP, _I], _I),
    "hisq_measure_fma_peaks": ([ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)], _I),
    "hisq_pc_apply_hermitian": ([_VP, _VP, _VP, _VP, _VP, _I], _I),
    "hisq_pc_apply_adjoint": ([_VP, _VP, _VP, _VP, _VP, _I], _I),
    "hisq_pc_apply_normal": ([_VP, _VP, _VP, _VP, _VP, _I], _I),
    "hisq_pc_set_form": ([_VP, _I], _I),
    "hisq_pc_loss_grad": ([_VP, _VP, _VP, _D, _VP, _VP, _I, _VP, _VP], _I),
    "hisq_pc_adam_step": ([_VP, _VP, _I, _D, _D, _D, _D], _I),
    "hisq_pc_train": ([_VP, _VP, _VP, _D, _VP, _VP, _I, _I, _I, _D, _VP], _I),
}


def load():
    """Load libhisq_gb300.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIBRARY):
            raise RuntimeError(f"{LIBRARY} is not built; run paper_1409_1510_gb300.build.build() "
                               "(there is no CPU fallback)")
        so = ctypes.CDLL(LIBRARY)
        for name, (args, res) in _SIGNATURES.items():
            fn = getattr(so, name, None)
            if fn is None:
                continue
            fn.argtypes = args
            fn.restype = res
        _lib = so
    return _lib


def _ptr(x):
    if x is None:
        return None
    if isinstance(x, int):
        return _VP(x)
    if hasattr(x, "data_ptr"):
        return _VP(x.data_ptr())
    if hasattr(x, "ctypes"):
        return _VP(x.ctypes.data)
    if isinstance(x, _VP):
        return x
    raise TypeError(f"cannot pass {type(x)} as a pointer")


def _check(rc):
    if rc != 0:
        raise HisqError(rc, load().hisq_last_error().decode())
    return rc


def hisq_strerror(status: int) -> str:
    return load().hisq_strerror(status).decode()


def hisq_last_error() -> str:
    return load().hisq_last_error().decode()


def hisq_init(dims, device: int = 0, stream=None):
    """Create the calling thread's context; stream: a torch.cuda.Stream, an address or None."""
    arr = (_I * 4)(*[int(d) for d in dims])
    s = None if stream is None else _VP(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))
    _check(load().hisq_init(arr, int(device), s))


def hisq_finalize():
    _check(load().hisq_finalize())


def hisq_links_create(canon, is_naik: bool, prec: int, recon: int = 18):
    """Pack canonical links (torch tensor or numpy float64 [4][V][3][3][2]); returns a handle."""
    h = _VP()
    _check(load().hisq_links_create(ctypes.byref(h), _ptr(canon), int(bool(is_naik)), int(prec), int(recon)))
    return h


def hisq_links_destroy(h):
    _check(load().hisq_links_destroy(h))


def hisq_links_export(h, out):
    _check(load().hisq_links_export(h, _ptr(out)))


def hisq_vector_bytes(prec: int, nrhs: int) -> int:
    return int(load().hisq_vector_bytes(int(prec), int(nrhs)))


def hisq_pack(canon, internal, nrhs: int, prec: int):
    _check(load().hisq_pack(_ptr(canon), _ptr(internal), int(nrhs), int(prec)))


def hisq_unpack(internal, canon, nrhs: int, prec: int):
    _check(load().hisq_unpack(_ptr(internal), _ptr(canon), int(nrhs), int(prec)))


def hisq_dslash(fat, naik, vin, vout, nrhs: int, parity: int):
    _check(load().hisq_dslash(fat, naik, _ptr(vin), _ptr(vout), int(nrhs), int(parity)))


def hisq_aop(fat, naik, mass: float, vin, vout, nrhs: int, pAp=None):
    _check(load().hisq_aop(fat, naik, float(mass), _ptr(vin), _ptr(vout), int(nrhs), _ptr(pAp)))


def hisq_residual(fat, naik, mass: float, rhs, x, r, nrhs: int, res2=None):
    """r = rhs - A x in FP64 accuracy (canonical buffers, host or device); see include/hisq.h."""
    _check(load().hisq_residual(fat, naik, float(mass), _ptr(rhs), _ptr(x), _ptr(r), int(nrhs), _ptr(res2)))


def hisq_slabs_create(fat_canon, naik_canon, prec: int, nslab: int = 2):
    h = _VP()
    _check(load().hisq_slabs_create(ctypes.byref(h), _ptr(fat_canon), _ptr(naik_canon), int(prec), int(nslab)))
    return h


def hisq_slabs_destroy(h):
    _check(load().hisq_slabs_destroy(h))


def hisq_slabs_dslash(h, vin, vout, nrhs: int, parity: int, ms=None):
    """Decomposed Dslash on canonical device buffers; ms: optional host float64[4] of event times."""
    _check(load().hisq_slabs_dslash(h, _ptr(vin), _ptr(vout), int(nrhs), int(parity), _ptr(ms)))


def hisq_aop_noalloc(fat, naik, mass: float, vin, vout, nrhs: int, pAp=None):
    """hisq_aop with its scratch in a static device array: allocates nothing (see include/hisq.h)."""
    _check(load().hisq_aop_noalloc(fat, naik, float(mass), _ptr(vin), _ptr(vout), int(nrhs), _ptr(pAp)))


def hisq_default_solver_params() -> hisq_solver_params:
    p = hisq_solver_params()
    load().hisq_default_solver_params(ctypes.byref(p))
    return p


def hisq_set_solver_params(p: hisq_solver_params):
    _check(load().hisq_set_solver_params(ctypes.byref(p)))


def hisq_get_solver_params() -> hisq_solver_params:
    p = hisq_solver_params()
    _check(load().hisq_get_solver_params(ctypes.byref(p)))
    return p


def hisq_cg_solve(fat, naik, rhs, x, mass: float, tol: float, raise_on_error: bool = True) -> int:
    """rhs, x: sequences of per-right-hand-side buffers (host numpy or device tensors)."""
    n = len(rhs)
    rp = (_VP * n)(*[_ptr(b).value for b in rhs])
    xp = (_VP * n)(*[_ptr(v).value for v in x])
    rc = load().hisq_cg_solve(fat, naik, rp, xp, n, float(mass), float(tol))
    if raise_on_error:
        _check(rc)
    return rc


def hisq_cg_multishift(fat, naik, rhs, x, shifts, mass: float, tol: float, raise_on_error: bool = True) -> int:
    """rhs: one buffer; x: a sequence of per-shift buffers (host numpy or device tensors);
    shifts: the per-shift sigma_j (host)."""
    n = len(x)
    if len(shifts) != n:
        raise ValueError("one output buffer per shift")
    xp = (_VP * n)(*[_ptr(v).value for v in x])
    sh = (_D * n)(*[float(v) for v in shifts])
    rc = load().hisq_cg_multishift(fat, naik, _ptr(rhs), xp, n, sh, float(mass), float(tol))
    if raise_on_error:
        _check(rc)
    return rc


def hisq_z2_noise(out, n: int, seed: int, first: int = 0):
    _check(load().hisq_z2_noise(_ptr(out), int(n), int(seed) & (2**64 - 1), int(first)))


def hisq_trace_inverse(fat, naik, mass: float, nnoise: int, seed: int, tol: float, samples=None,
                       raise_on_error: bool = True):
    """Returns (estimate of Tr A^{-1}, its standard error, status); samples: host float64[nnoise] or None."""
    est, err = _D(), _D()
    rc = load().hisq_trace_inverse(fat, naik, float(mass), int(nnoise), int(seed) & (2**64 - 1), float(tol),
                                   ctypes.byref(est), ctypes.byref(err), _ptr(samples))
    if raise_on_error:
        _check(rc)
    return est.value, err.value, rc


def hisq_last_stats(iterations=None, true_residual=None) -> hisq_solve_stats:
    s = hisq_solve_stats()
    _check(load().hisq_last_stats(ctypes.byref(s), _ptr(iterations), _ptr(true_residual)))
    return s


def hisq_autotune(fat, naik, nrhs: int):
    """Returns (rhs_per_thread, block_threads, lanes_per_site) of the fastest shape."""
    r, t, s = _I(), _I(), _I()
    _check(load().hisq_autotune(fat, naik, int(nrhs), ctypes.byref(r), ctypes.byref(t), ctypes.byref(s)))
    return r.value, t.value, s.value


def hisq_set_launch_shape(prec: int, recon: int, nrhs: int, rhs_per_thread: int, block_threads: int,
                          lanes_per_site: int = 1):
    _check(load().hisq_set_launch_shape(int(prec), int(recon), int(nrhs), int(rhs_per_thread), int(block_threads),
                                        int(lanes_per_site)))


def hisq_pc_create(weights=None):
    h = _VP()
    _check(load().hisq_pc_create(ctypes.byref(h), _ptr(weights)))
    return h


def hisq_pc_destroy(pc):
    _check(load().hisq_pc_destroy(pc))


def hisq_pc_set_weights(pc, weights):
    _check(load().hisq_pc_set_weights(pc, _ptr(weights)))


def hisq_pc_get_weights(pc, weights):
    _check(load().hisq_pc_get_weights(pc, _ptr(weights)))


def hisq_pc_apply(pc, fat, naik, vin, vout, nrhs: int):
    _check(load().hisq_pc_apply(pc, fat, naik, _ptr(vin), _ptr(vout), int(nrhs)))


def hisq_pc_apply_hermitian(pc, fat, naik, vin, vout, nrhs: int):
    _check(load().hisq_pc_apply_hermitian(pc, fat, naik, _ptr(vin), _ptr(vout), int(nrhs)))


def hisq_pc_apply_adjoint(pc, fat, naik, vin, vout, nrhs: int):
    _check(load().hisq_pc_apply_adjoint(pc, fat, naik, _ptr(vin), _ptr(vout), int(nrhs)))


def hisq_pc_apply_normal(pc, fat, naik, vin, vout, nrhs: int):
    _check(load().hisq_pc_apply_normal(pc, fat, naik, _ptr(vin), _ptr(vout), int(nrhs)))


HISQ_PC_NORMAL = 1
HISQ_PC_HERMITIAN_PART = 0


def hisq_pc_set_form(pc, form: int):
    _check(load().hisq_pc_set_form(pc, int(form)))


def hisq_pc_loss_grad(pc, fat, naik, mass: float, r, e, K: int, grad):
    loss = _D()
    _check(load().hisq_pc_loss_grad(pc, fat, naik, float(mass), _ptr(r), _ptr(e), int(K), ctypes.byref(loss),
                                    _ptr(grad)))
    return loss.value


def hisq_pc_adam_step(pc, grad, step: int, lr: float, beta1=0.9, beta2=0.999, eps=1e-8):
    _check(load().hisq_pc_adam_step(pc, _ptr(grad), int(step), float(lr), float(beta1), float(beta2), float(eps)))


def hisq_pc_train(pc, fat, naik, mass: float, r, e, K: int, batch: int, epochs: int, lr: float,
                  loss_history=None):
    _check(load().hisq_pc_train(pc, fat, naik, float(mass), _ptr(r), _ptr(e), int(K), int(batch), int(epochs),
                                float(lr), _ptr(loss_history)))


def hisq_device_status():
    _check(load().hisq_device_status())


def hisq_dslash_full(fat, naik, vin, vout, nrhs: int):
    _check(load().hisq_dslash_full(fat, naik, _ptr(vin), _ptr(vout), int(nrhs)))


def hisq_measure_fma_peaks():
    """(fp32_tflops, fp64_tflops) measured on the context's device."""
    a, b = ctypes.c_double(), ctypes.c_double()
    _check(load().hisq_measure_fma_peaks(ctypes.byref(a), ctypes.byref(b)))
    return a.value, b.value
