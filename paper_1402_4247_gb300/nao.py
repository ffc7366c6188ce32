"""Python binding of the C ABI in include/nao.h (argument marshalling only).

Every function has the C entry point's name and forwards device pointers (from torch
tensors) and the current CUDA stream to ``libnao.so``; all computation happens in the
library's CUDA kernels.  There is no CPU fallback: if the library cannot be loaded the
call raises.
"""
from __future__ import annotations

import ctypes
import os

import torch

from . import build as _build

NAO_OK = 0
NAO_E_INVALID = -1
NAO_E_NOMEM = -2
NAO_E_NOCONV = -3
NAO_E_TIMEOUT = -4
NAO_E_CUDA = -5
NAO_E_ALLCUT = -6
NAO_E_BUSY = -7
NAO_E_RANGE = -8
NAO_FP64 = 0
NAO_MIXED_TF32 = 1
NAO_MIXED_BF16X3 = 2

#: every symbol include/nao.h declares
EXPORTS = ("nao_config_defaults", "nao_init", "nao_get_config", "nao_set_config", "nao_destroy",
           "nao_last_error", "nao_workspace_bytes", "nao_bloch_sum",
           "nao_gen_eig", "nao_gen_eig_sized", "nao_density_matrix", "nao_profile_enable", "nao_profile_read",
           "nao_launch_count",
           "nao_fermi_level_noalloc", "nao_set_gemm_method", "nao_set_refinement", "nao_zgemm",
           "nao_gen_eig_workspace", "nao_serve_config", "nao_serve_pause", "nao_serve_submit", "nao_serve_poll",
           "nao_serve_release", "nao_serve_stats")
NAO_GEMM_FP64 = 0
NAO_GEMM_TC = 1

_lib = None


class NaoError(RuntimeError):
    pass


class NaoConfig(ctypes.Structure):
    """``nao_config`` of include/nao.h."""
    _fields_ = [("f_min", ctypes.c_double), ("inverse_iteration_max", ctypes.c_int),
                ("tc_wait_cycles", ctypes.c_longlong), ("mixed_planes", ctypes.c_int),
                ("overlap_mrrr", ctypes.c_int), ("band_width", ctypes.c_int), ("mrrr_all", ctypes.c_int),
                ("split_hprime", ctypes.c_int)]


class NaoRequest(ctypes.Structure):
    """``nao_request`` of include/nao.h."""
    _fields_ = [("n", ctypes.c_int), ("nspin", ctypes.c_int), ("nk", ctypes.c_int), ("nR", ctypes.c_int),
                ("HR", ctypes.c_void_p), ("SR", ctypes.c_void_p), ("R", ctypes.c_void_p),
                ("kpts", ctypes.c_void_p), ("wk", ctypes.c_void_p),
                ("n_electrons", ctypes.c_double), ("kT", ctypes.c_double), ("s_cut", ctypes.c_double),
                ("precision", ctypes.c_int), ("nb", ctypes.c_int), ("want_rho", ctypes.c_int)]


class NaoResult(ctypes.Structure):
    """``nao_result`` of include/nao.h."""
    _fields_ = [("status", ctypes.c_int), ("n", ctypes.c_int), ("nprob", ctypes.c_int), ("nb", ctypes.c_int),
                ("nspin", ctypes.c_int), ("nR", ctypes.c_int),
                ("eps", ctypes.c_void_p), ("C", ctypes.c_void_p), ("m_kept", ctypes.c_void_p),
                ("prob_status", ctypes.c_void_p), ("mu", ctypes.c_void_p), ("eband", ctypes.c_void_p),
                ("f", ctypes.c_void_p), ("rho", ctypes.c_void_p), ("rho_status", ctypes.c_void_p),
                ("queue_ms", ctypes.c_double), ("latency_ms", ctypes.c_double), ("batch_requests", ctypes.c_int)]


class _DeviceView:
    """A device array the library owns, seen by torch through __cuda_array_interface__."""

    def __init__(self, ptr, shape, typestr):
        self.__cuda_array_interface__ = {"shape": tuple(shape), "typestr": typestr, "data": (ptr, False),
                                         "version": 3, "strides": None}


def load_library(path: str | None = None) -> ctypes.CDLL:
    """Load libnao.so (building it first if it is missing or older than its sources)."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or _build.LIB
    if path == _build.LIB and _build.is_stale():
        _build.build()
    lib = ctypes.CDLL(path)
    vp, i32, f64, sz = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_size_t
    lib.nao_config_defaults.argtypes = [ctypes.POINTER(NaoConfig)]
    lib.nao_config_defaults.restype = None
    lib.nao_init.argtypes = [ctypes.POINTER(vp), i32, sz, ctypes.POINTER(NaoConfig)]
    lib.nao_init.restype = i32
    lib.nao_get_config.argtypes = [vp, ctypes.POINTER(NaoConfig)]
    lib.nao_get_config.restype = i32
    lib.nao_set_config.argtypes = [vp, ctypes.POINTER(NaoConfig)]
    lib.nao_set_config.restype = i32
    lib.nao_destroy.argtypes = [vp]
    lib.nao_destroy.restype = None
    lib.nao_last_error.argtypes = [vp]
    lib.nao_last_error.restype = ctypes.c_char_p
    lib.nao_workspace_bytes.argtypes = [vp]
    lib.nao_workspace_bytes.restype = sz
    lib.nao_bloch_sum.argtypes = [vp, i32, i32, vp, i32, vp, i32, vp, vp, vp]
    lib.nao_bloch_sum.restype = i32
    lib.nao_gen_eig.argtypes = [vp, i32, i32, vp, vp, vp, i32, f64, i32, i32, vp, vp, vp, vp, vp]
    lib.nao_gen_eig.restype = i32
    lib.nao_gen_eig_sized.argtypes = [vp, i32, i32, vp, vp, vp, i32, vp, f64, i32, i32, vp, vp, vp, vp, vp]
    lib.nao_gen_eig_sized.restype = i32
    lib.nao_density_matrix.argtypes = [vp, i32, i32, i32, vp, vp, vp, vp, i32, vp, f64, f64, i32, vp, vp, vp,
                                       vp, vp, vp, vp, vp]
    lib.nao_density_matrix.restype = i32
    lib.nao_profile_enable.argtypes = [vp, i32]
    lib.nao_profile_enable.restype = i32
    lib.nao_profile_read.argtypes = [vp, i32, ctypes.POINTER(ctypes.c_char_p), ctypes.POINTER(f64),
                                     ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)]
    lib.nao_profile_read.restype = i32
    lib.nao_launch_count.argtypes = [vp]
    lib.nao_launch_count.restype = ctypes.c_int64
    lib.nao_set_gemm_method.argtypes = [vp, i32]
    lib.nao_set_gemm_method.restype = i32
    lib.nao_set_refinement.argtypes = [vp, i32]
    lib.nao_set_refinement.restype = i32
    i64 = ctypes.c_longlong
    lib.nao_zgemm.argtypes = [vp, i32, i32, i32, i32, i32, f64, vp, i32, i64, i32, vp, i32, i64, i32, f64, vp, i32,
                              i64, vp]
    lib.nao_zgemm.restype = i32
    lib.nao_fermi_level_noalloc.argtypes = [i32, i32, i32, vp, vp, vp, i32, f64, f64, vp, vp, vp, vp, vp]
    lib.nao_fermi_level_noalloc.restype = i32
    lib.nao_gen_eig_workspace.argtypes = [vp, i32, i32, i32, i32, ctypes.POINTER(sz)]
    lib.nao_gen_eig_workspace.restype = i32
    lib.nao_serve_config.argtypes = [vp, sz, i32, i32]
    lib.nao_serve_config.restype = i32
    lib.nao_serve_pause.argtypes = [vp, i32]
    lib.nao_serve_pause.restype = i32
    lib.nao_serve_submit.argtypes = [vp, ctypes.POINTER(NaoRequest), ctypes.POINTER(ctypes.c_uint64)]
    lib.nao_serve_submit.restype = i32
    lib.nao_serve_poll.argtypes = [vp, ctypes.c_uint64, i32, ctypes.POINTER(NaoResult)]
    lib.nao_serve_poll.restype = i32
    lib.nao_serve_release.argtypes = [vp, ctypes.c_uint64]
    lib.nao_serve_release.restype = i32
    lib.nao_serve_stats.argtypes = [vp, ctypes.POINTER(sz), ctypes.POINTER(sz), ctypes.POINTER(i32),
                                    ctypes.POINTER(i32)]
    lib.nao_serve_stats.restype = i32
    _lib = lib
    return lib


def _ptr(t):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return ctypes.c_void_p(t.data_ptr())


def _check_tensor(name, t, dtype, shape, device):
    """Raise ValueError unless ``t`` is a contiguous tensor of ``dtype`` whose shape matches
    ``shape`` (None: any extent) on ``device``: the kernels read every extent the call
    passes, so a smaller or differently typed buffer would be read past its end."""
    if not isinstance(t, torch.Tensor):
        raise ValueError(f"{name} must be a torch tensor")
    if t.dtype != dtype:
        raise ValueError(f"{name} must be {dtype}, not {t.dtype}")
    if t.dim() != len(shape) or any(s is not None and int(e) != int(s) for e, s in zip(t.shape, shape)):
        want = "[" + ", ".join("*" if s is None else str(s) for s in shape) + "]"
        raise ValueError(f"{name} must have shape {want}, not {list(t.shape)}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if t.device != device:
        raise ValueError(f"{name} must be on {device}, not {t.device}")


def check_bloch_sum_args(MR, R, kpts, out, device):
    """Arguments of ``nao_bloch_sum``: MR float64 [nmat][nR][n][n], R int32 [nR][3], kpts
    float64 [nk][3], out complex128 [nmat][nk][n][n] (or None)."""
    _check_tensor("MR", MR, torch.float64, (None, None, None, None), device)
    nmat, nR, n, n2 = MR.shape
    if n != n2:
        raise ValueError(f"MR must hold square matrices, not {n} x {n2}")
    _check_tensor("R", R, torch.int32, (nR, 3), device)
    _check_tensor("kpts", kpts, torch.float64, (None, 3), device)
    if out is not None:
        _check_tensor("out", out, torch.complex128, (nmat, kpts.shape[0], n, n), device)


def check_gen_eig_args(H, S, s_of_prob, nb, out, s_size, device):
    """Arguments of ``nao_gen_eig``: H complex128 [nprob][n][n], S complex128 [nS][n][n], s_of_prob
    int32 [nprob] (or None: nS == nprob), 1 <= nb <= n, out = (eps float64 [nprob][n], C
    complex128 [nprob][n][nb] or None, m_kept int32 [nprob], status int32 [nprob]) or None,
    s_size int32 [nS] or None."""
    _check_tensor("H", H, torch.complex128, (None, None, None), device)
    nprob, n, n2 = H.shape
    if n != n2:
        raise ValueError(f"H must hold square matrices, not {n} x {n2}")
    _check_tensor("S", S, torch.complex128, (None, n, n), device)
    nS = S.shape[0]
    if s_of_prob is None:
        if nS != nprob:
            raise ValueError("S must have one matrix per problem unless s_of_prob is given")
    else:
        _check_tensor("s_of_prob", s_of_prob, torch.int32, (nprob,), device)
    if not 1 <= nb <= n:
        raise ValueError(f"nb must lie in [1, {n}], not {nb}")
    if s_size is not None:
        _check_tensor("s_size", s_size, torch.int32, (nS,), device)
    if out is not None:
        eps, C, m, st = out
        _check_tensor("eps", eps, torch.float64, (nprob, n), device)
        if C is not None:
            _check_tensor("C", C, torch.complex128, (nprob, n, nb), device)
        _check_tensor("m_kept", m, torch.int32, (nprob,), device)
        _check_tensor("status", st, torch.int32, (nprob,), device)


def check_density_matrix_args(wk, kpts, eps, C, m_kept, R, nspin, out, edm, device):
    """Arguments of ``nao_density_matrix``: C complex128 [nprob][n][nb] with nprob = nspin nk,
    wk float64 [nk], kpts float64 [nk][3], eps float64 [nprob][n], m_kept int32 [nprob], R int32
    [nR][3], out = (mu [1], eband [1], f [nprob][n] or None, rho [nspin][nR][n][n], all float64,
    status int32 [1]) or None, edm float64 [nspin][nR][n][n] or None."""
    _check_tensor("C", C, torch.complex128, (None, None, None), device)
    nprob, n, nb = C.shape
    _check_tensor("wk", wk, torch.float64, (None,), device)
    nk = wk.shape[0]
    if nprob != int(nspin) * nk:
        raise ValueError(f"C has {nprob} problems, expected nspin * nk = {int(nspin) * nk}")
    _check_tensor("kpts", kpts, torch.float64, (nk, 3), device)
    _check_tensor("eps", eps, torch.float64, (nprob, n), device)
    _check_tensor("m_kept", m_kept, torch.int32, (nprob,), device)
    _check_tensor("R", R, torch.int32, (None, 3), device)
    nR = R.shape[0]
    if out is not None:
        mu, eb, f, rho, st = out
        _check_tensor("mu", mu, torch.float64, (1,), device)
        _check_tensor("eband", eb, torch.float64, (1,), device)
        if f is not None:
            _check_tensor("f", f, torch.float64, (nprob, n), device)
        _check_tensor("rho", rho, torch.float64, (int(nspin), nR, n, n), device)
        _check_tensor("status", st, torch.int32, (1,), device)
    if edm is not None:
        _check_tensor("edm", edm, torch.float64, (int(nspin), nR, n, n), device)


def check_serve_request_args(HR, SR, R, kpts, wk, device):
    """Arguments of ``nao_serve_submit``: HR float64 [nspin][nR][n][n], SR float64 [nR][n][n], R
    int32 [nR][3], kpts float64 [nk][3], wk float64 [nk], all on the host or all on ``device``."""
    where = HR.device if isinstance(HR, torch.Tensor) and HR.device.type == "cpu" else device
    _check_tensor("HR", HR, torch.float64, (None, None, None, None), where)
    nspin, nR, n, n2 = HR.shape
    if n != n2:
        raise ValueError(f"HR must hold square matrices, not {n} x {n2}")
    _check_tensor("SR", SR, torch.float64, (nR, n, n), where)
    _check_tensor("R", R, torch.int32, (nR, 3), where)
    _check_tensor("kpts", kpts, torch.float64, (None, 3), where)
    _check_tensor("wk", wk, torch.float64, (kpts.shape[0],), where)


def check_zgemm_args(A, B, C, transA, transB, device):
    """Arguments of ``nao_zgemm``: A, B, C complex128 [nprob][..][..] with op(A) M x K, op(B)
    K x N and C [nprob][M][N] (or None)."""
    _check_tensor("A", A, torch.complex128, (None, None, None), device)
    nprob = A.shape[0]
    _check_tensor("B", B, torch.complex128, (nprob, None, None), device)
    M, K = (A.shape[2], A.shape[1]) if transA else (A.shape[1], A.shape[2])
    KB, N = (B.shape[2], B.shape[1]) if transB else (B.shape[1], B.shape[2])
    if K != KB:
        raise ValueError(f"op(A) has {K} columns but op(B) has {KB} rows")
    if C is not None:
        _check_tensor("C", C, torch.complex128, (nprob, M, N), device)


def _stream(stream):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def nao_config_defaults() -> dict:
    """The default ``nao_config`` as a dict (f_min, inverse_iteration_max, tc_wait_cycles)."""
    c = NaoConfig()
    load_library().nao_config_defaults(ctypes.byref(c))
    return {k: getattr(c, k) for k, _ in NaoConfig._fields_}


class Context:
    """Owns an ``nao_ctx`` (device workspace) on one CUDA device.

    ``hbm_budget_bytes`` bounds the context's workspace (0: no bound); ``config`` is a dict
    with any of the ``nao_config`` fields (the others keep their defaults)."""

    def __init__(self, device: int = 0, hbm_budget_bytes: int = 0, config: dict | None = None):
        self.lib = load_library()
        self.handle = ctypes.c_void_p()
        cfg = None
        if config is not None:
            cfg = NaoConfig()
            self.lib.nao_config_defaults(ctypes.byref(cfg))
            for k, v in config.items():
                setattr(cfg, k, v)
        rc = self.lib.nao_init(ctypes.byref(self.handle), int(device), int(hbm_budget_bytes),
                               ctypes.byref(cfg) if cfg is not None else None)
        if rc != NAO_OK:
            raise NaoError(f"nao_init failed ({rc}): {self.lib.nao_last_error(None).decode()}")
        self.device = device
        self._dev = torch.device("cuda", int(device))

    def nao_get_config(self) -> dict:
        c = NaoConfig()
        self._check(self.lib.nao_get_config(self.handle, ctypes.byref(c)), "nao_get_config")
        return {k: getattr(c, k) for k, _ in NaoConfig._fields_}

    def nao_set_config(self, **changes):
        """Replace some ``nao_config`` fields (synchronises the device first)."""
        c = NaoConfig()
        self._check(self.lib.nao_get_config(self.handle, ctypes.byref(c)), "nao_get_config")
        for k, v in changes.items():
            if k not in dict(NaoConfig._fields_):
                raise ValueError(f"unknown nao_config field {k}")
            setattr(c, k, v)
        self._check(self.lib.nao_set_config(self.handle, ctypes.byref(c)), "nao_set_config")

    def close(self):
        if self.handle:
            self.lib.nao_destroy(self.handle)
            self.handle = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc, name):
        if rc != NAO_OK:
            raise NaoError(f"{name} failed ({rc}): {self.lib.nao_last_error(self.handle).decode()}")

    def workspace_bytes(self) -> int:
        return int(self.lib.nao_workspace_bytes(self.handle))

    def nao_set_gemm_method(self, method: int):
        self._check(self.lib.nao_set_gemm_method(self.handle, int(method)), "nao_set_gemm_method")

    def nao_set_refinement(self, sweeps: int):
        """Refinement after a mixed-precision nao_gen_eig: 0 Rayleigh quotients only (default),
        1 or 2 Ritz sweeps first, -1 none."""
        self._check(self.lib.nao_set_refinement(self.handle, int(sweeps)), "nao_set_refinement")

    def nao_zgemm(self, A, B, C=None, alpha=1.0, beta=0.0, transA=0, transB=0, method=NAO_GEMM_TC, stream=None):
        """Batched C[p] = alpha op(A[p]) op(B[p]) + beta C[p] (complex128, row-major, 3-d tensors)."""
        check_zgemm_args(A, B, C, transA, transB, self._dev)
        nprob = A.shape[0]
        M = A.shape[2] if transA else A.shape[1]
        K = A.shape[1] if transA else A.shape[2]
        N = B.shape[1] if transB else B.shape[2]
        if C is None:
            C = torch.zeros((nprob, M, N), dtype=torch.complex128, device=A.device)
        rc = self.lib.nao_zgemm(self.handle, int(method), nprob, M, N, K, float(alpha), _ptr(A), A.shape[2],
                                A.shape[1] * A.shape[2], int(transA), _ptr(B), B.shape[2], B.shape[1] * B.shape[2],
                                int(transB), float(beta), _ptr(C), C.shape[2], C.shape[1] * C.shape[2],
                                _stream(stream))
        self._check(rc, "nao_zgemm")
        return C

    def nao_profile_enable(self, on: bool = True):
        self._check(self.lib.nao_profile_enable(self.handle, 1 if on else 0), "nao_profile_enable")

    def nao_profile_read(self) -> dict:
        """{stage: (total_ms, calls, launches)} from the CUDA events recorded so far."""
        cap = 64
        names = (ctypes.c_char_p * cap)()
        ms = (ctypes.c_double * cap)()
        calls = (ctypes.c_int64 * cap)()
        launches = (ctypes.c_int64 * cap)()
        k = self.lib.nao_profile_read(self.handle, cap, names, ms, calls, launches)
        if k < 0:
            self._check(k, "nao_profile_read")
        return {names[i].decode(): (ms[i], int(calls[i]), int(launches[i])) for i in range(min(k, cap))}

    def nao_launch_count(self) -> int:
        return int(self.lib.nao_launch_count(self.handle))

    # ------------------------------------------------------------------ Part 1
    def nao_bloch_sum(self, MR, R, kpts, out=None, stream=None):
        """MR float64 [nmat][nR][n][n], R int32 [nR][3], kpts float64 [nk][3] -> complex128 [nmat][nk][n][n]."""
        check_bloch_sum_args(MR, R, kpts, out, self._dev)
        nmat, nR, n, _ = MR.shape
        nk = kpts.shape[0]
        if out is None:
            out = torch.empty((nmat, nk, n, n), dtype=torch.complex128, device=MR.device)
        rc = self.lib.nao_bloch_sum(self.handle, n, nR, _ptr(R), nmat, _ptr(MR), nk, _ptr(kpts), _ptr(out),
                                    _stream(stream))
        self._check(rc, "nao_bloch_sum")
        return out

    # ------------------------------------------------------------------ Parts 2-4
    def nao_gen_eig(self, H, S, s_of_prob=None, s_cut=1e-10, nb=None, precision=NAO_FP64, want_vectors=True,
                    out=None, stream=None, s_size=None):
        """H complex128 [nprob][n][n], S complex128 [nS][n][n] -> (eps, C, m_kept, status).
        s_of_prob (int32 [nprob] on the device, optional): the S matrix of each problem; its
        entries must lie in [0, nS) (not checked: they are device data).
        s_size (int32 [nS] on the device, optional): each S matrix's order when the matrices
        are padded to n (nao_gen_eig_sized)."""
        nb = H.shape[1] if nb is None else int(nb)
        check_gen_eig_args(H, S, s_of_prob, nb, out, s_size, self._dev)
        nprob, n, _ = H.shape
        nS = S.shape[0]
        dev = H.device
        if out is None:
            eps = torch.empty((nprob, n), dtype=torch.float64, device=dev)
            C = torch.empty((nprob, n, nb), dtype=torch.complex128, device=dev) if want_vectors else None
            m = torch.empty(nprob, dtype=torch.int32, device=dev)
            st = torch.empty(nprob, dtype=torch.int32, device=dev)
        else:
            eps, C, m, st = out
        rc = self.lib.nao_gen_eig_sized(self.handle, n, nprob, _ptr(H), _ptr(S), _ptr(s_of_prob), nS, _ptr(s_size),
                                        float(s_cut), int(precision), nb, _ptr(eps), _ptr(C), _ptr(m), _ptr(st),
                                        _stream(stream))
        self._check(rc, "nao_gen_eig")
        return eps, C, m, st

    def nao_gen_eig_workspace(self, n, nprob, nS, precision=NAO_FP64) -> int:
        b = ctypes.c_size_t()
        self._check(self.lib.nao_gen_eig_workspace(self.handle, int(n), int(nprob), int(nS), int(precision),
                                                   ctypes.byref(b)), "nao_gen_eig_workspace")
        return int(b.value)

    # ------------------------------------------------------------------ serving
    def nao_serve_config(self, hbm_budget_bytes: int, max_batch_problems: int = 256, slots: int = 2):
        self._check(self.lib.nao_serve_config(self.handle, int(hbm_budget_bytes), int(max_batch_problems),
                                              int(slots)), "nao_serve_config")

    def nao_serve_pause(self, on: bool):
        self._check(self.lib.nao_serve_pause(self.handle, 1 if on else 0), "nao_serve_pause")

    def nao_serve_submit(self, HR, SR, R, kpts, wk, n_electrons, kT, s_cut=1e-10, precision=NAO_FP64, nb=0,
                         want_rho=True) -> int:
        """Queue one band step.  HR float64 [nspin][nR][n][n], SR [nR][n][n], R int32 [nR][3],
        kpts [nk][3], wk [nk]: contiguous torch tensors on the host or the device (copied
        before the call returns).  Returns the ticket."""
        check_serve_request_args(HR, SR, R, kpts, wk, self._dev)
        nspin, nR, n, _ = HR.shape
        q = NaoRequest(n=n, nspin=nspin, nk=kpts.shape[0], nR=nR, HR=HR.data_ptr(), SR=SR.data_ptr(),
                       R=R.data_ptr(), kpts=kpts.data_ptr(), wk=wk.data_ptr(), n_electrons=float(n_electrons),
                       kT=float(kT), s_cut=float(s_cut), precision=int(precision), nb=int(nb),
                       want_rho=1 if want_rho else 0)
        t = ctypes.c_uint64()
        self._check(self.lib.nao_serve_submit(self.handle, ctypes.byref(q), ctypes.byref(t)), "nao_serve_submit")
        return int(t.value)

    def nao_serve_poll(self, ticket: int, timeout_us: int = -1) -> NaoResult:
        """Wait (timeout_us < 0: without limit) and return the ``NaoResult``; its status is
        NAO_E_BUSY while the request is still queued or running."""
        res = NaoResult()
        rc = self.lib.nao_serve_poll(self.handle, ctypes.c_uint64(ticket), int(timeout_us), ctypes.byref(res))
        if rc not in (NAO_OK, NAO_E_BUSY) and res.n == 0:
            self._check(rc, "nao_serve_poll")
        return res

    def serve_result_tensors(self, res: NaoResult) -> dict:
        """Copies (torch, on the device) of a finished request's results."""
        n, P, nb, ns, nR = res.n, res.nprob, res.nb, res.nspin, res.nR
        dev = torch.device("cuda", self.device)

        def view(ptr, shape, typestr, dtype):
            if not ptr:
                return None
            return torch.as_tensor(_DeviceView(ptr, shape, typestr), device=dev).view(dtype).clone()

        return {"eps": view(res.eps, (P, n), "<f8", torch.float64),
                "C": view(res.C, (P, n, 2 * nb), "<f8", torch.float64).view(torch.complex128) if res.C else None,
                "m": view(res.m_kept, (P,), "<i4", torch.int32),
                "status": view(res.prob_status, (P,), "<i4", torch.int32),
                "mu": view(res.mu, (1,), "<f8", torch.float64), "eband": view(res.eband, (1,), "<f8", torch.float64),
                "f": view(res.f, (P, n), "<f8", torch.float64), "rho": view(res.rho, (ns, nR, n, n), "<f8", torch.float64),
                "rstatus": view(res.rho_status, (1,), "<i4", torch.int32)}

    def nao_serve_release(self, ticket: int):
        self._check(self.lib.nao_serve_release(self.handle, ctypes.c_uint64(ticket)), "nao_serve_release")

    def nao_serve_stats(self):
        """-> (used_bytes, peak_bytes, queued, running)"""
        u, pk, q, r = ctypes.c_size_t(), ctypes.c_size_t(), ctypes.c_int(), ctypes.c_int()
        self._check(self.lib.nao_serve_stats(self.handle, ctypes.byref(u), ctypes.byref(pk), ctypes.byref(q),
                                             ctypes.byref(r)), "nao_serve_stats")
        return int(u.value), int(pk.value), int(q.value), int(r.value)

    # ------------------------------------------------------------------ Parts 5-6
    def nao_density_matrix(self, wk, kpts, eps, C, m_kept, n_electrons, kT, R, nspin, want_f=True, out=None,
                           stream=None, edm=None):
        """-> (mu [1], eband [1], f [nprob][n] or None, rho [nspin][nR][n][n], status [1]).
        ``edm``: a float64 [nspin][nR][n][n] device tensor that receives the energy density
        matrix (Part 6's second output), or None."""
        check_density_matrix_args(wk, kpts, eps, C, m_kept, R, nspin, out, edm, self._dev)
        nprob, n, nb = C.shape
        nk = wk.shape[0]
        nR = R.shape[0]
        dev = C.device
        if out is None:
            mu = torch.empty(1, dtype=torch.float64, device=dev)
            eb = torch.empty(1, dtype=torch.float64, device=dev)
            f = torch.empty((nprob, n), dtype=torch.float64, device=dev) if want_f else None
            rho = torch.empty((nspin, nR, n, n), dtype=torch.float64, device=dev)
            st = torch.empty(1, dtype=torch.int32, device=dev)
        else:
            mu, eb, f, rho, st = out
        rc = self.lib.nao_density_matrix(self.handle, n, nspin, nk, _ptr(wk), _ptr(kpts), _ptr(eps), _ptr(C), nb,
                                         _ptr(m_kept), float(n_electrons), float(kT), nR, _ptr(R), _ptr(mu),
                                         _ptr(eb), _ptr(f), _ptr(rho), _ptr(edm), _ptr(st), _stream(stream))
        self._check(rc, "nao_density_matrix")
        return mu, eb, f, rho, st


def nao_fermi_level_noalloc(wk, eps, m_kept, nb, n_electrons, kT, nspin, f_out, mu_out, eband_out, status,
                            stream=None):
    """Part 5 (mu, f, E_band) through the allocation-free entry point: the library allocates
    nothing; all outputs are caller tensors on the current device."""
    lib = load_library()
    nprob, n = eps.shape
    nk = wk.shape[0]
    # the kernel walks nspin * nk rows of n entries: every buffer must hold exactly that
    if nprob != int(nspin) * nk:
        raise ValueError(f"eps has {nprob} rows, expected nspin * nk = {int(nspin) * nk}")
    if tuple(f_out.shape) != (nprob, n):
        raise ValueError(f"f_out must have shape {(nprob, n)}, not {tuple(f_out.shape)}")
    if tuple(m_kept.shape) != (nprob,):
        raise ValueError(f"m_kept must have shape {(nprob,)}, not {tuple(m_kept.shape)}")
    for name, t, dt, numel in (("wk", wk, torch.float64, nk), ("eps", eps, torch.float64, nprob * n),
                               ("m_kept", m_kept, torch.int32, nprob), ("f_out", f_out, torch.float64, nprob * n),
                               ("mu_out", mu_out, torch.float64, 1), ("eband_out", eband_out, torch.float64, 1),
                               ("status", status, torch.int32, 1)):
        if t.dtype != dt:
            raise ValueError(f"{name} must be {dt}, not {t.dtype}")
        if t.numel() < numel:
            raise ValueError(f"{name} holds {t.numel()} elements, needs {numel}")
        if not t.is_cuda or t.device.index != torch.cuda.current_device():
            raise ValueError(f"{name} must be on the current CUDA device (cuda:{torch.cuda.current_device()})")
    rc = lib.nao_fermi_level_noalloc(n, int(nspin), nk, _ptr(wk), _ptr(eps), _ptr(m_kept), int(nb),
                                     float(n_electrons), float(kT), _ptr(f_out), _ptr(mu_out), _ptr(eband_out),
                                     _ptr(status), _stream(stream))
    if rc != NAO_OK:
        raise NaoError(f"nao_fermi_level_noalloc failed ({rc}): {lib.nao_last_error(None).decode()}")
    return mu_out, eband_out, f_out, status
