"""Thin ctypes binding of libt2sh.so (C ABI in include/t2sh.h).

Argument marshalling only: every step of the solve runs in the library's CUDA kernels.
Device arrays are torch CUDA tensors (PyTorch supplies device memory and streams);
with ``host_io=True`` the plan takes host arrays (numpy or CPU tensors) and the library
does the copies.  There is no fallback: if the library is missing, loading fails.
"""
from __future__ import annotations

import ctypes
import os
import re

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libt2sh.so")
HEADER = os.path.join(os.path.dirname(_HERE), "include", "t2sh.h")

OK, EINVAL, ENOMEM, ECUDA, EUNSUPPORTED, ETIMEOUT, EBUSY = range(7)
FP32, MIXED_BF16 = 0, 1
KSPACE_TE, KSPACE_PROJ = 0, 1
NO_SHIFT, HOST_IO, EIG_FP64, FUSED_ROWS = 0x1, 0x2, 0x4, 0x8
_STATUS = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "ECUDA", 4: "EUNSUPPORTED", 5: "ETIMEOUT", 6: "EBUSY"}


class T2shError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status


class Dims(ctypes.Structure):
    _fields_ = [("ny", ctypes.c_int32), ("nz", ctypes.c_int32), ("ncoils", ctypes.c_int32),
                ("nmaps", ctypes.c_int32), ("nechoes", ctypes.c_int32), ("nbasis", ctypes.c_int32),
                ("nslices", ctypes.c_int32), ("block", ctypes.c_int32), ("lam", ctypes.c_float),
                ("iters", ctypes.c_int32), ("seed", ctypes.c_uint64), ("step", ctypes.c_float),
                ("precision", ctypes.c_int32), ("flags", ctypes.c_uint32)]


def make_dims(ny, nz, ncoils, nechoes, nbasis, nslices=1, nmaps=1, block=8, lam=0.0, iters=0, seed=0,
              step=0.0, precision=FP32, flags=0) -> Dims:
    return Dims(ny, nz, ncoils, nmaps, nechoes, nbasis, nslices, block, lam, iters, seed, step, precision, flags)


_lib = None
_vp, _i32, _u64, _f32 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_uint64, ctypes.c_float


def lib() -> ctypes.CDLL:
    """The loaded library; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_1809_04195_gb300.build.build()")
        L = ctypes.CDLL(LIB_PATH)
        sig = {
            "t2sh_plan": [ctypes.POINTER(Dims), _vp, _vp, _vp, _vp, ctypes.POINTER(_vp)],
            "t2sh_destroy": [_vp],
            "t2sh_release_cached": [],
            "t2sh_forward": [_vp, _vp, _vp, _i32],
            "t2sh_adjoint": [_vp, _vp, _i32, _vp],
            "t2sh_normal_op": [_vp, _vp, _vp],
            "t2sh_llr_prox": [_vp, _vp, _f32, _i32, _i32],
            "t2sh_solve": [_vp, _vp, _i32, _vp, ctypes.POINTER(ctypes.c_double)],
            "t2sh_solve_admm": [_vp, _vp, _i32, _vp, _f32, _i32, ctypes.POINTER(ctypes.c_double)],
            "t2sh_objective": [_vp, _vp, _i32, _vp, ctypes.POINTER(ctypes.c_double)],
            "t2sh_postprocess": [_vp, _vp, ctypes.POINTER(_i32), _i32, _f32, _vp],
            "t2sh_wavelet_denoise": [_vp, _vp, _f32, _i32],
            "t2sh_coil_compression": [ctypes.POINTER(Sparse), _vp, _i32, _i32, _vp, _vp],
            "t2sh_preprocess": [ctypes.POINTER(Sparse), _vp, _vp, _i32, _vp, _i32, _vp, _vp, _vp],
            "t2sh_get_step": [_vp, ctypes.POINTER(_f32)],
            "t2sh_shifts": [_u64, _i32, _i32, ctypes.POINTER(_i32)],
            "t2sh_workspace_bytes": [ctypes.POINTER(Dims), ctypes.POINTER(ctypes.c_size_t)],
            "t2sh_timing_enable": [_vp, _i32],
            "t2sh_solve_begin": [_vp, _vp, _i32],
            "t2sh_solve_iterate": [_vp, _i32, ctypes.POINTER(_i32)],
            "t2sh_solve_end": [_vp, _vp, ctypes.POINTER(ctypes.c_double)],
            "t2sh_solve_batch": [ctypes.POINTER(_vp), _i32, ctypes.POINTER(_vp), ctypes.POINTER(_i32),
                                 ctypes.POINTER(_vp), _vp],
            "t2sh_autotune": [_vp, _i32, ctypes.POINTER(_i32), ctypes.POINTER(_i32)],
            "t2sh_batch_schedule": [_i32],
            "t2sh_sync": [_vp],
            "t2sh_configure": [_vp, _i32, _i32],
            "t2sh_wait_selftest": [_vp, _u64],
            "t2sh_timing_read": [_vp, _i32, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_double)],
        }
        for name, args in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = ctypes.c_int
        L.t2sh_normal_op_noalloc.argtypes = [ctypes.POINTER(Dims), _vp, _vp, _vp, _vp, _vp, _vp]
        L.t2sh_normal_op_noalloc.restype = ctypes.c_int
        L.t2sh_noalloc_scratch_bytes.argtypes = []
        L.t2sh_noalloc_scratch_bytes.restype = ctypes.c_size_t
        L.t2sh_noalloc_sync.argtypes = [_vp]
        L.t2sh_noalloc_sync.restype = ctypes.c_int
        L.t2sh_noalloc_wait_selftest.argtypes = [_u64, _vp]
        L.t2sh_noalloc_wait_selftest.restype = ctypes.c_int
        L.t2sh_last_error.argtypes = []
        L.t2sh_last_error.restype = ctypes.c_char_p
        L.t2sh_version.argtypes = []
        L.t2sh_version.restype = ctypes.c_int32
        _lib = L
    return _lib


def header_symbols() -> list[str]:
    """Function names declared in include/t2sh.h."""
    with open(HEADER) as f:
        txt = f.read()
    return sorted(set(re.findall(r"^\s*(?:t2sh_status|const char\*|int32_t|size_t)\s+(t2sh_\w+)\s*\(", txt, re.M)))


def _check(status: int):
    if status != OK:
        raise T2shError(status, lib().t2sh_last_error().decode())


def last_error() -> str:
    return lib().t2sh_last_error().decode()


def version() -> int:
    return int(lib().t2sh_version())


def shifts(seed: int, iters: int, block: int) -> np.ndarray:
    """LLR shift table [iters][2] (sy, sz), host-only."""
    out = np.zeros((max(iters, 0), 2), np.int32)
    _check(lib().t2sh_shifts(seed, iters, block, out.ctypes.data_as(ctypes.POINTER(_i32))))
    return out


def release_cached() -> None:
    """Return the unused memory of the library's plan pool to the device."""
    _check(lib().t2sh_release_cached())


def workspace_bytes(dims: Dims) -> int:
    n = ctypes.c_size_t(0)
    _check(lib().t2sh_workspace_bytes(ctypes.byref(dims), ctypes.byref(n)))
    return int(n.value)


def _ptr(t, dtype, shape, host: bool):
    """Data pointer of a contiguous array with the expected dtype and shape."""
    import torch
    if isinstance(t, np.ndarray):
        if not host:
            raise TypeError("numpy arrays are host memory: pass torch CUDA tensors or use host_io=True")
        want = {torch.complex64: np.complex64, torch.float32: np.float32, torch.uint8: np.uint8}[dtype]
        if t.dtype != want or not t.flags["C_CONTIGUOUS"] or tuple(t.shape) != tuple(shape):
            raise ValueError(f"expected C-contiguous {want} {tuple(shape)}, got {t.dtype} {t.shape}")
        return ctypes.c_void_p(t.ctypes.data)
    if t.dtype != dtype or not t.is_contiguous() or tuple(t.shape) != tuple(shape):
        raise ValueError(f"expected contiguous {dtype} {tuple(shape)}, got {t.dtype} {tuple(t.shape)}")
    if host == t.is_cuda:
        raise ValueError("host_io plans take host arrays; other plans take CUDA tensors")
    return ctypes.c_void_p(t.data_ptr())


class Sparse(ctypes.Structure):
    """t2sh_sparse: the acquisition as readout lines (index arrays in host memory)."""
    _fields_ = [("nlines", ctypes.c_int32), ("nchan", ctypes.c_int32), ("nx", ctypes.c_int32),
                ("ny", ctypes.c_int32), ("nz", ctypes.c_int32), ("nechoes", ctypes.c_int32),
                ("t", ctypes.POINTER(ctypes.c_int32)), ("ky", ctypes.POINTER(ctypes.c_int32)),
                ("kz", ctypes.POINTER(ctypes.c_int32))]


def _sparse(lines, t, ky, kz, ny, nz, nechoes):
    keep = [np.ascontiguousarray(a, dtype=np.int32) for a in (t, ky, kz)]
    n, nchan, nx = (int(v) for v in lines.shape)
    if any(len(a) != n for a in keep):
        raise ValueError("t, ky, kz need one entry per line")
    ptr = [a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)) for a in keep]
    return Sparse(n, nchan, nx, int(ny), int(nz), int(nechoes), *ptr), keep


def coil_compression(lines, t, ky, kz, ny: int, nz: int, nechoes: int, window: int = 24, ncomp: int = 7,
                     stream=None):
    """Compression matrix W [nchan][ncomp] (device) from the central window of the sparse
    readout lines (device [nlines][nchan][nx] complex64); t, ky, kz: host index arrays."""
    import torch
    sp, keep = _sparse(lines, t, ky, kz, ny, nz, nechoes)
    w = torch.empty((int(lines.shape[1]), int(ncomp)), dtype=torch.complex64, device="cuda")
    st = torch.cuda.current_stream() if stream is None else stream
    _check(lib().t2sh_coil_compression(ctypes.byref(sp), _ptr(lines, torch.complex64, tuple(lines.shape), False),
                                       int(window), int(ncomp), ctypes.c_void_p(w.data_ptr()),
                                       ctypes.c_void_p(st.cuda_stream)))
    del keep
    return w


def preprocess(lines, t, ky, kz, w, phi, ny: int, nz: int, stream=None):
    """(ytil [nx][ncomp][K][ny][nz] complex64, mask [T][ny][nz] uint8), device: coil
    compression with w, readout decoupling, re-sort and projection onto phi [T][K]."""
    import torch
    T, K = (int(v) for v in phi.shape)
    sp, keep = _sparse(lines, t, ky, kz, ny, nz, T)
    ncomp = int(w.shape[1])
    nx = int(lines.shape[2])
    ytil = torch.empty((nx, ncomp, K, int(ny), int(nz)), dtype=torch.complex64, device="cuda")
    mask = torch.empty((T, int(ny), int(nz)), dtype=torch.uint8, device="cuda")
    st = torch.cuda.current_stream() if stream is None else stream
    _check(lib().t2sh_preprocess(ctypes.byref(sp), _ptr(lines, torch.complex64, tuple(lines.shape), False),
                                 _ptr(w, torch.complex64, tuple(w.shape), False), ncomp,
                                 _ptr(phi, torch.float32, (T, K), False), K, ctypes.c_void_p(ytil.data_ptr()),
                                 ctypes.c_void_p(mask.data_ptr()), ctypes.c_void_p(st.cuda_stream)))
    del keep
    return ytil, mask


def normal_op_noalloc(dims: Dims, phi, mask, maps, x, out=None, stream=None):
    """y = A^H A x without a plan and without any device allocation by the library
    (scratch in a static device array; see include/t2sh.h).  CUDA tensors only."""
    import torch
    S, C, M, K, T, ny, nz = dims.nslices, dims.ncoils, dims.nmaps, dims.nbasis, dims.nechoes, dims.ny, dims.nz
    vshape = (S, M, K, ny, nz)
    if out is None:
        out = torch.empty(vshape, dtype=torch.complex64, device=x.device)
    if stream is None:
        stream = torch.cuda.current_stream()
    _check(lib().t2sh_normal_op_noalloc(ctypes.byref(dims), _ptr(phi, torch.float32, (T, K), False),
                                        _ptr(mask, torch.uint8, (T, ny, nz), False),
                                        _ptr(maps, torch.complex64, (S, C, M, ny, nz), False),
                                        _ptr(x, torch.complex64, vshape, False), _ptr(out, torch.complex64, vshape, False),
                                        ctypes.c_void_p(stream.cuda_stream)))
    return out


def noalloc_scratch_bytes() -> int:
    return int(lib().t2sh_noalloc_scratch_bytes())


def noalloc_sync(stream=None):
    """Synchronise the stream; raises T2shError(ETIMEOUT) if a bounded device wait of
    normal_op_noalloc ran out since the last noalloc_sync (the flag is then cleared)."""
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    _check(lib().t2sh_noalloc_sync(ctypes.c_void_p(stream.cuda_stream)))


def noalloc_wait_selftest(limit_ns: int, stream=None):
    """Launch a kernel whose bounded wait runs out after limit_ns and sets the flag of the
    static array; the next noalloc_sync raises T2shError(ETIMEOUT)."""
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    _check(lib().t2sh_noalloc_wait_selftest(int(limit_ns), ctypes.c_void_p(stream.cuda_stream)))


def batch_schedule(per_scan_llr: bool):
    """solve_batch's LLR schedule: one work-list launch per iteration (False, default) or
    one launch per plan on its own stream (True)."""
    _check(lib().t2sh_batch_schedule(1 if per_scan_llr else 0))


def solve_batch(plans, kspaces, kforms=None, outs=None, stream=None):
    """Solve several plans (scans of different shapes) at once: forked streams, every
    iteration captured into one CUDA graph (t2sh_solve_batch).  Returns the outputs."""
    import torch
    n = len(plans)
    kforms = [KSPACE_PROJ] * n if kforms is None else list(kforms)
    outs = [p._empty(p.vec_shape) for p in plans] if outs is None else list(outs)
    hp = (ctypes.c_void_p * n)(*[p._h.value for p in plans])
    kp = (ctypes.c_void_p * n)(*[p._dev(k, p._kshape(f)).value for p, k, f in zip(plans, kspaces, kforms)])
    op = (ctypes.c_void_p * n)(*[p._dev(o, p.vec_shape).value for p, o in zip(plans, outs)])
    kf = (ctypes.c_int32 * n)(*kforms)
    st = torch.cuda.current_stream() if stream is None else stream
    _check(lib().t2sh_solve_batch(hp, n, kp, kf, op, ctypes.c_void_p(st.cuda_stream)))
    return outs


class Plan:
    """One batch of slices sharing a basis, a sampling pattern and dimensions.

    phi [T][K] float32, mask [T][ny][nz] uint8, maps [S][C][M][ny][nz] complex64."""

    def __init__(self, dims: Dims, phi, mask, maps, stream=None):
        import torch
        self.dims = dims
        self.host_io = bool(dims.flags & HOST_IO)
        d = dims
        self.S, self.C, self.M, self.K, self.T = d.nslices, d.ncoils, d.nmaps, d.nbasis, d.nechoes
        self.ny, self.nz = d.ny, d.nz
        self.vec_shape = (self.S, self.M, self.K, self.ny, self.nz)
        if stream is None and torch.cuda.is_available():
            stream = torch.cuda.current_stream()
        self.stream = stream
        sp = ctypes.c_void_p(stream.cuda_stream if stream is not None else 0)
        h = ctypes.c_void_p(0)
        _check(lib().t2sh_plan(ctypes.byref(d),
                               _ptr(phi, torch.float32, (self.T, self.K), self.host_io),
                               _ptr(mask, torch.uint8, (self.T, self.ny, self.nz), self.host_io),
                               _ptr(maps, torch.complex64, (self.S, self.C, self.M, self.ny, self.nz), self.host_io),
                               sp, ctypes.byref(h)))
        self._h = h

    # -- helpers --------------------------------------------------------------------
    def _kshape(self, kform):
        return (self.S, self.C, self.T if kform == KSPACE_TE else self.K, self.ny, self.nz)

    def _dev(self, t, shape):
        import torch
        return _ptr(t, torch.complex64, shape, False)

    def _empty(self, shape):
        import torch
        return torch.empty(shape, dtype=torch.complex64, device="cuda")

    @property
    def step(self) -> float:
        v = ctypes.c_float(0)
        _check(lib().t2sh_get_step(self._h, ctypes.byref(v)))
        return float(v.value)

    # -- operators ------------------------------------------------------------------
    def forward(self, x, kform=KSPACE_PROJ, out=None):
        out = self._empty(self._kshape(kform)) if out is None else out
        _check(lib().t2sh_forward(self._h, self._dev(x, self.vec_shape), self._dev(out, self._kshape(kform)), kform))
        return out

    def adjoint(self, y, kform=KSPACE_PROJ, out=None):
        out = self._empty(self.vec_shape) if out is None else out
        _check(lib().t2sh_adjoint(self._h, self._dev(y, self._kshape(kform)), kform, self._dev(out, self.vec_shape)))
        return out

    def normal_op(self, x, out=None):
        out = self._empty(self.vec_shape) if out is None else out
        _check(lib().t2sh_normal_op(self._h, self._dev(x, self.vec_shape), self._dev(out, self.vec_shape)))
        return out

    def llr_prox(self, x, tau: float, sy: int, sz: int):
        """In place."""
        _check(lib().t2sh_llr_prox(self._h, self._dev(x, self.vec_shape), float(tau), int(sy), int(sz)))
        return x

    def solve(self, kspace, kform=KSPACE_PROJ, out=None, residual: bool = False):
        """FISTA solve; returns alpha (and the per-iteration relative change if asked)."""
        import torch
        if self.host_io:
            if out is None:
                out = np.empty(self.vec_shape, np.complex64)
            kp = _ptr(kspace, torch.complex64, self._kshape(kform), True)
            op = _ptr(out, torch.complex64, self.vec_shape, True)
        else:
            out = self._empty(self.vec_shape) if out is None else out
            kp, op = self._dev(kspace, self._kshape(kform)), self._dev(out, self.vec_shape)
        res = None
        rp = None
        if residual:
            res = np.zeros(max(self.dims.iters, 0), np.float64)
            rp = res.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        _check(lib().t2sh_solve(self._h, kp, kform, op, rp))
        return (out, res) if residual else out

    def solve_admm(self, kspace, kform=KSPACE_PROJ, rho: float = 1.0, cg_iters: int = 3, out=None,
                   residual: bool = False):
        """ADMM solve (CG alpha-updates, LLR prox on v); returns v (and the per-iteration
        relative change of v if asked)."""
        import torch
        if self.host_io:
            if out is None:
                out = np.empty(self.vec_shape, np.complex64)
            kp = _ptr(kspace, torch.complex64, self._kshape(kform), True)
            op = _ptr(out, torch.complex64, self.vec_shape, True)
        else:
            out = self._empty(self.vec_shape) if out is None else out
            kp, op = self._dev(kspace, self._kshape(kform)), self._dev(out, self.vec_shape)
        res = None
        rp = None
        if residual:
            res = np.zeros(max(self.dims.iters, 0), np.float64)
            rp = res.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        _check(lib().t2sh_solve_admm(self._h, kp, kform, op, float(rho), int(cg_iters), rp))
        return (out, res) if residual else out

    def objective(self, kspace, kform, x):
        """Data term of Eq. 5 at x per slice, as (h, c) float64 arrays [S] with f = h + c:
        h = 1/2 <x, A^H A x> - Re <x, A^H y>, c = 1/2 ||P y||^2 (NaN for projected k-space)."""
        import torch
        kp = _ptr(kspace, torch.complex64, self._kshape(kform), self.host_io)
        xp = _ptr(x, torch.complex64, self.vec_shape, self.host_io)
        out = np.zeros((self.S, 2), np.float64)
        _check(lib().t2sh_objective(self._h, kp, kform, xp, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
        return out[:, 0], out[:, 1]

    def postprocess(self, alpha, te_index, pf: float = 0.65, out=None):
        """TE images [S][nte][ny][nz] (float32, device): back-projection at the echoes
        te_index, coil images, homodyne along z (partial Fourier fraction pf), RSS."""
        import torch
        te = list(int(t) for t in te_index)
        shape = (self.S, len(te), self.ny, self.nz)
        if out is None:
            out = torch.empty(shape, dtype=torch.float32, device="cuda")
        ap = self._dev(alpha, self.vec_shape)
        op = _ptr(out, torch.float32, shape, False)
        tarr = (_i32 * len(te))(*te)
        _check(lib().t2sh_postprocess(self._h, ap, tarr, len(te), float(pf), op))
        return out

    def wavelet_denoise(self, alpha, tau: float, levels: int = 1):
        """In place on alpha [S][M][K][ny][nz] (device): orthonormal 3D Haar pyramid over
        (slice, y, z) with `levels` levels, details soft-thresholded by tau, inverse."""
        import torch
        ap = _ptr(alpha, torch.complex64, self.vec_shape, False)
        _check(lib().t2sh_wavelet_denoise(self._h, ap, float(tau), int(levels)))
        return alpha

    # -- resumable solve (schedulers interleaving scans) --------------------------------
    def solve_begin(self, kspace, kform=KSPACE_PROJ):
        import torch
        self._kin = kspace  # keep the caller's array alive until the solve ends
        kp = _ptr(kspace, torch.complex64, self._kshape(kform), self.host_io)
        _check(lib().t2sh_solve_begin(self._h, kp, kform))

    def solve_iterate(self, n: int) -> int:
        done = ctypes.c_int32(0)
        _check(lib().t2sh_solve_iterate(self._h, int(n), ctypes.byref(done)))
        return int(done.value)

    def solve_end(self, out=None, residual: bool = False):
        import torch
        if self.host_io:
            out = np.empty(self.vec_shape, np.complex64) if out is None else out
            op = _ptr(out, torch.complex64, self.vec_shape, True)
        else:
            out = self._empty(self.vec_shape) if out is None else out
            op = self._dev(out, self.vec_shape)
        res = np.zeros(max(self.dims.iters, 0), np.float64) if residual else None
        rp = res.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if residual else None
        _check(lib().t2sh_solve_end(self._h, op, rp))
        self._kin = None
        return (out, res) if residual else out

    def autotune(self, probe_iters: int = 3):
        """(column-pass variant 0 TMA x8 / 4 TMA x4 / 1 cp.async x8 / 2 cp.async x4 / 3 tensor
        cores in split BF16 for MIXED_BF16 plans, fused rows) chosen for this plan's shape."""
        w, f = ctypes.c_int32(0), ctypes.c_int32(0)
        _check(lib().t2sh_autotune(self._h, int(probe_iters), ctypes.byref(w), ctypes.byref(f)))
        return int(w.value), bool(f.value)

    def configure(self, col_variant: int, fused_rows: bool = False):
        """Pin the column-pass variant (0 TMA x8, 4 TMA x4, 1 cp.async x8, 2 cp.async x4,
        3 tensor cores in split BF16) and row fusion."""
        _check(lib().t2sh_configure(self._h, int(col_variant), 1 if fused_rows else 0))

    def wait_selftest(self, limit_ns: int):
        """Launch a kernel whose bounded wait runs out after limit_ns; the next sync()
        raises T2shError(ETIMEOUT) and the plan stays usable."""
        _check(lib().t2sh_wait_selftest(self._h, int(limit_ns)))

    def sync(self):
        """Synchronise the plan's stream; raises T2shError(ETIMEOUT) if a bounded device
        wait ran out since the last call."""
        _check(lib().t2sh_sync(self._h))

    # -- kernel timing ----------------------------------------------------------------
    KERNEL_CLASSES = {0: "row_fwd", 1: "row_adj", 2: "col", 3: "llr", 5: "project", 6: "band", 7: "cg", 8: "post"}

    def timing(self, enable: bool):
        _check(lib().t2sh_timing_enable(self._h, 1 if enable else 0))

    def timing_read(self) -> dict:
        """{class name: (launches, total ms)} since timing(True)."""
        out = {}
        for c, name in self.KERNEL_CLASSES.items():
            n = ctypes.c_int64(0)
            ms = ctypes.c_double(0)
            _check(lib().t2sh_timing_read(self._h, c, ctypes.byref(n), ctypes.byref(ms)))
            out[name] = (int(n.value), float(ms.value))
        return out

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().t2sh_destroy(self._h)
            self._h = ctypes.c_void_p(0)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
