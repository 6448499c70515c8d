"""Helpers for the GPU parity tests: a context on one lattice with packed links, and
canonical <-> internal vector transfers through the C ABI."""
import contextlib

import numpy as np

import hisq_inputs as hi
import oracle

PREC_TOL = {0: 1e-12, 1: 1e-5, 2: 5e-3, 3: 5e-3}   # per-Dslash norm-wise bound per precision
PREC_NAME = {0: "fp64", 1: "fp32", 2: "fp16", 3: "bf16"}


def rel_err(got, want):
    """max over right-hand sides of |got - want| / |want| (norm-wise)."""
    got = np.asarray(got).reshape(len(want), -1)
    want = np.asarray(want).reshape(len(want), -1)
    return float(max(np.linalg.norm(got[k] - want[k]) / np.linalg.norm(want[k]) for k in range(len(want))))


class Gpu:
    """A HISQ context for one lattice, with links packed in one precision/reconstruction."""

    def __init__(self, dims, prec, recon=18, fields=None, stream=None):
        import torch
        from paper_1409_1510_gb300 import hisq
        self.torch, self.hisq = torch, hisq
        self.dims = tuple(dims)
        self.lat = hi.Lattice(dims)
        self.dev = torch.device("cuda:0")
        if fields is None:
            fields = (hi.fat_links(self.lat), hi.naik_links(self.lat))
        self.X, self.N = fields
        self.prec, self.recon = prec, recon
        hisq.hisq_init(dims, 0, stream)
        self.fat = hisq.hisq_links_create(self._dev64(self.X), False, prec, 18)
        self.naik = hisq.hisq_links_create(self._dev64(self.N), True, prec, recon)
        self._oracle = None

    @property
    def oracle(self):
        if self._oracle is None:
            self._oracle = oracle.Oracle(self.dims, self.X, self.N)
        return self._oracle

    def _dev64(self, a):
        a = np.ascontiguousarray(a, dtype=np.complex128)
        return self.torch.from_numpy(a.view(np.float64).copy()).to(self.dev)

    def bundle(self, n, prec=None):
        prec = self.prec if prec is None else prec
        return self.torch.empty(self.hisq.hisq_vector_bytes(prec, n), dtype=self.torch.uint8, device=self.dev)

    def pack(self, v, prec=None):
        """v: complex [n][V/2][3] numpy -> device internal bundle."""
        prec = self.prec if prec is None else prec
        v = np.asarray(v).reshape(-1, self.lat.half_volume, 3)
        buf = self.bundle(len(v), prec)
        self.hisq.hisq_pack(self._dev64(v), buf, len(v), prec)
        return buf

    def unpack(self, buf, n, prec=None):
        prec = self.prec if prec is None else prec
        out = self.torch.empty((n, self.lat.half_volume, 3, 2), dtype=self.torch.float64, device=self.dev)
        self.hisq.hisq_unpack(buf, out, n, prec)
        return out.cpu().numpy().view(np.complex128)[..., 0]

    def close(self):
        self.torch.cuda.synchronize()
        self.hisq.hisq_finalize()


@contextlib.contextmanager
def gpu(dims, prec, recon=18, fields=None, stream=None):
    g = Gpu(dims, prec, recon, fields, stream)
    try:
        yield g
    finally:
        g.close()
