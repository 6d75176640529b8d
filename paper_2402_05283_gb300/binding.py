"""ctypes binding of the C ABI declared in include/cpra.h.

Argument marshalling only: every step of the reconstruction runs in the CUDA
kernels of libcpra.so.  The functions keep the C names (``cpra_plan``,
``cpra_iterate`` ...); :class:`Plan` wraps them for convenience.  Arrays may
be numpy arrays (host memory) or torch tensors (host or CUDA memory); the
library tells host and device pointers apart itself.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libcpra.so")

OK, ERR_INVALID_ARG, ERR_OUT_OF_MEMORY, ERR_CUDA, ERR_NOT_READY, ERR_TIMEOUT, ERR_UNSUPPORTED, ERR_NONFINITE = range(8)
WRAP_LITERAL, WRAP_MIRROR = 0, 1
BLEND_STATE, BLEND_OBJECT = 0, 1
FP32, BF16_TC, FP16_TC = 0, 1, 2
UPDATE_HIO, UPDATE_RAAR = 0, 1
ENGINE_AUTO, ENGINE_TWO_PASS, ENGINE_FUSED, ENGINE_WARP, ENGINE_TUNED = 0, 1, 2, 3, 4
RESULT_PO, RESULT_STATE, RESULT_SUPPORT, RESULT_ERRORS, RESULT_VOLUME, RESULT_MERGED_SPECTRA = range(6)
(KERNEL_COLPASS, KERNEL_ROWPASS, KERNEL_PRIME, KERNEL_SHRINKWRAP, KERNEL_ASSEMBLE, KERNEL_FUSED,
 KERNEL_PREPARE, KERNEL_REFINE, KERNEL_KINDS) = range(9)
MAX_TAPS = 15

ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)


class cpra_config(C.Structure):
    _fields_ = [
        ("N", C.c_int32), ("Np", C.c_int32), ("n_ei", C.c_int32), ("n_taps", C.c_int32),
        ("alpha", C.c_double * MAX_TAPS), ("beta", C.c_float), ("wrap_mode", C.c_int32),
        ("blend_target", C.c_int32), ("hio_iters", C.c_int32), ("er_iters", C.c_int32),
        ("shrinkwrap_every", C.c_int32), ("sw_sigma", C.c_float), ("sw_tau", C.c_float),
        ("n_pre", C.c_int32), ("precision", C.c_int32), ("com_align", C.c_int32),
        ("engine", C.c_int32), ("update", C.c_int32), ("sweep", C.c_int32), ("seed", C.c_uint64), ("alloc", ALLOC_FN), ("free", FREE_FN),
        ("alloc_ctx", C.c_void_p),
    ]


class cpra_server_config(C.Structure):
    _fields_ = [("hbm_reserve_bytes", C.c_size_t), ("max_active", C.c_int32),
                ("iters_per_round", C.c_int32), ("use_graph", C.c_int32), ("stream", C.c_void_p),
                ("early_start", C.c_int32), ("early_tail", C.c_int32)]


class cpra_server_event(C.Structure):
    _fields_ = [("id", C.c_int64), ("kind", C.c_int32), ("t_event", C.c_double),
                ("t_submit", C.c_double), ("t_last_pattern", C.c_double)]


class cpra_server_request(C.Structure):
    _fields_ = [("state", C.c_int32), ("iterations_done", C.c_int64), ("angles_arrived", C.c_int32),
                ("t_submit", C.c_double), ("t_admit", C.c_double), ("t_last_pattern", C.c_double),
                ("t_first_estimate", C.c_double), ("t_final", C.c_double)]


class cpra_server_stats(C.Structure):
    _fields_ = [("submitted", C.c_int64), ("admitted", C.c_int64), ("completed", C.c_int64),
                ("rounds", C.c_int64), ("max_batch", C.c_int64), ("angle_iterations", C.c_int64)]


EVENT_FIRST_ESTIMATE, EVENT_FINAL, EVENT_FAILED = 1, 2, 3


class CpraError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"cpra status {status}: {msg}")
        self.status = status


_lib = None


def lib() -> C.CDLL:
    """Load libcpra.so; raises if it was not built (there is no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: run __graft_entry__.build() "
                              "(the CUDA library is required; there is no CPU path)")
        L = C.CDLL(LIB_PATH)
        P = C.c_void_p
        sigs = {
            "cpra_default_config": (C.c_int, [C.c_int32, C.c_int32, C.POINTER(cpra_config)]),
            "cpra_plan_bytes": (C.c_int, [C.POINTER(cpra_config), C.POINTER(C.c_size_t), C.POINTER(C.c_size_t)]),
            "cpra_plan": (C.c_int, [C.POINTER(cpra_config), P, C.POINTER(P)]),
            "cpra_load_intensities": (C.c_int, [P, P, C.c_int32, C.c_int32, P]),
            "cpra_load_support": (C.c_int, [P, P, C.c_int32]),
            "cpra_load_mask": (C.c_int, [P, P, C.c_int32]),
            "cpra_load_state": (C.c_int, [P, P, C.c_int64]),
            "cpra_iterate": (C.c_int, [P, C.c_int32, P]),
            "cpra_assemble_3d": (C.c_int, [P, P]),
            "cpra_assemble_3d_async": (C.c_int, [P, P]),
            "cpra_download_wait": (C.c_int, [P]),
            "cpra_result": (C.c_int, [P, C.c_int32, P, C.c_size_t]),
            "cpra_iteration": (C.c_int64, [P]),
            "cpra_reset": (C.c_int, [P]),
            "cpra_set_present": (C.c_int, [P, P]),
            "cpra_set_profiling": (C.c_int, [P, C.c_int32]),
            "cpra_kernel_stats": (C.c_int, [P, C.c_int32, C.POINTER(C.c_double), C.POINTER(C.c_int64)]),
            "cpra_launch_count": (C.c_int64, []),
            "cpra_shrinkwrap_static": (C.c_int, [P, P, P, C.c_int32, C.c_int32, C.c_float,
                                                 C.c_float, P]),
            "cpra_refine_3d": (C.c_int, [P, C.c_int32, C.c_int32, C.c_float, C.c_float, P]),
            "cpra_merge": (C.c_int, [C.POINTER(P), C.c_int32, C.c_int32, C.c_int32, P,
                                     C.POINTER(C.c_int32), C.POINTER(C.c_int32), P]),
            "cpra_batch_create": (C.c_int, [C.POINTER(P), C.c_int32, C.c_int32, C.POINTER(P)]),
            "cpra_batch_iterate": (C.c_int, [P, C.c_int32]),
            "cpra_batch_launches": (C.c_int64, [P, C.c_int32]),
            "cpra_batch_set_persistent": (C.c_int, [P, C.c_int32, C.c_double, C.c_int32]),
            "cpra_batch_destroy": (C.c_int, [P]),
            "cpra_autotune": (C.c_int, [C.c_int32, C.c_int32, C.c_char_p, C.POINTER(C.c_int32),
                                        C.POINTER(C.c_double)]),
            "cpra_server_default_config": (C.c_int, [C.POINTER(cpra_server_config)]),
            "cpra_server_start": (C.c_int, [C.POINTER(cpra_server_config), C.POINTER(P)]),
            "cpra_server_submit": (C.c_int, [P, C.POINTER(cpra_config), C.POINTER(C.c_int64)]),
            "cpra_server_push": (C.c_int, [P, C.c_int64, P, C.c_int32, C.c_int32, P]),
            "cpra_server_poll": (C.c_int, [P, C.POINTER(cpra_server_event), C.c_int32,
                                           C.POINTER(C.c_int32)]),
            "cpra_server_wait": (C.c_int, [P, C.c_int64, C.c_double]),
            "cpra_server_request_info": (C.c_int, [P, C.c_int64, C.POINTER(cpra_server_request)]),
            "cpra_server_result": (C.c_int, [P, C.c_int64, C.c_int32, P, C.c_size_t]),
            "cpra_server_release": (C.c_int, [P, C.c_int64]),
            "cpra_server_get_stats": (C.c_int, [P, C.POINTER(cpra_server_stats)]),
            "cpra_server_stop": (C.c_int, [P]),
            "cpra_sync": (C.c_int, [P]),
            "cpra_destroy": (C.c_int, [P]),
            "cpra_last_error": (C.c_char_p, [P]),
        }
        for name, (res, args) in sigs.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _check(st: int, plan=None):
    if st != OK:
        msg = lib().cpra_last_error(plan)
        raise CpraError(st, msg.decode() if msg else "")


def _ptr(a):
    """(pointer, keep-alive) for a numpy array or torch tensor (or None)."""
    if a is None:
        return None, None
    if isinstance(a, np.ndarray):
        a = np.ascontiguousarray(a)
        return a.ctypes.data, a
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            a = a.contiguous()
        return a.data_ptr(), a
    raise TypeError(f"unsupported array type {type(a)}")


# ------------------------------------------------------------ C-named calls
def cpra_default_config(N: int, Np: int) -> cpra_config:
    cfg = cpra_config()
    _check(lib().cpra_default_config(N, Np, C.byref(cfg)))
    return cfg


def cpra_plan_bytes(cfg: cpra_config):
    a, b = C.c_size_t(), C.c_size_t()
    _check(lib().cpra_plan_bytes(C.byref(cfg), C.byref(a), C.byref(b)))
    return a.value, b.value


def cpra_plan(cfg: cpra_config, stream: int | None = None):
    h = C.c_void_p()
    _check(lib().cpra_plan(C.byref(cfg), stream, C.byref(h)))
    return h


def cpra_load_intensities(plan, I, first: int, count: int, thetas=None):
    p, keep = _ptr(I)
    th = None
    if thetas is not None:
        th = np.ascontiguousarray(thetas, dtype=np.float64)
    _check(lib().cpra_load_intensities(plan, p, first, count,
                                       None if th is None else th.ctypes.data), plan)
    return keep


def cpra_load_support(plan, S, per_angle: int):
    p, keep = _ptr(S)
    _check(lib().cpra_load_support(plan, p, per_angle), plan)
    return keep


def cpra_load_mask(plan, mask, per_angle: int):
    p, keep = _ptr(mask)
    _check(lib().cpra_load_mask(plan, p, per_angle), plan)
    return keep


def cpra_load_state(plan, g, t: int):
    p, keep = _ptr(g)
    _check(lib().cpra_load_state(plan, p, t), plan)
    return keep


def cpra_iterate(plan, n_iters: int, err_out=None):
    p, keep = _ptr(err_out)
    _check(lib().cpra_iterate(plan, n_iters, p), plan)
    return keep


def cpra_assemble_3d(plan, out=None):
    p, keep = _ptr(out)
    _check(lib().cpra_assemble_3d(plan, p), plan)
    return keep


def cpra_assemble_3d_async(plan, out):
    """Queue the assembly and a download of the volume into out without
    waiting.  out: page-locked host memory (a pinned torch tensor or a
    registered numpy array), contiguous, N^3 complex64 (or N^3 x 2 float32);
    it is written in place, so no copy is made, and must stay alive and
    untouched until cpra_download_wait."""
    if isinstance(out, np.ndarray):
        ok, ptr = out.flags.c_contiguous, out.ctypes.data
    elif hasattr(out, "data_ptr"):
        ok, ptr = out.is_contiguous(), out.data_ptr()
    else:
        raise TypeError(f"unsupported array type {type(out)}")
    if not ok:
        raise ValueError("out must be contiguous (the download writes it in place)")
    _check(lib().cpra_assemble_3d_async(plan, ptr), plan)


def cpra_download_wait(plan):
    _check(lib().cpra_download_wait(plan), plan)


def cpra_result(plan, what: int, dst, nbytes: int):
    p, keep = _ptr(dst)
    _check(lib().cpra_result(plan, what, p, nbytes), plan)
    return keep


def cpra_merge(guesses, n_l: int, twin_ref: int, dst, prtf=None):
    """Step C merge of plan handles `guesses` into plan handle `dst`.
    Returns (selected, inverted) as lists; prtf: None, or a float32 array /
    tensor of Np * N/2 elements that receives the PRTF."""
    hs = [g.h if isinstance(g, Plan) else g for g in guesses]
    if isinstance(dst, Plan):
        dst = dst.h
    n_r = len(hs)
    arr = (C.c_void_p * n_r)(*[h.value if isinstance(h, C.c_void_p) else h for h in hs])
    sel = (C.c_int32 * max(n_l, 1))()
    inv = (C.c_int32 * max(n_l, 1))()
    p, keep = _ptr(prtf)
    _check(lib().cpra_merge(arr, n_r, n_l, twin_ref, dst, sel, inv, p), dst)
    return list(sel)[:n_l], [bool(v) for v in inv][:n_l]


def cpra_refine_3d(plan, n_iters: int, shrink_every: int = 0, sigma: float = 2.0, tau: float = 0.1,
                   err_out=None):
    p, keep = _ptr(err_out)
    _check(lib().cpra_refine_3d(plan, n_iters, shrink_every, sigma, tau, p), plan)
    return keep


def cpra_iteration(plan) -> int:
    return int(lib().cpra_iteration(plan))


def cpra_reset(plan):
    _check(lib().cpra_reset(plan), plan)


def cpra_set_present(plan, mask):
    """mask: None or a host uint8 array of Np entries."""
    p = None if mask is None else mask.ctypes.data_as(C.c_void_p)
    _check(lib().cpra_set_present(plan, p), plan)


def cpra_set_profiling(plan, on: bool):
    _check(lib().cpra_set_profiling(plan, int(bool(on))), plan)


def cpra_kernel_stats(plan, kind: int):
    ms, n = C.c_double(), C.c_int64()
    _check(lib().cpra_kernel_stats(plan, kind, C.byref(ms), C.byref(n)), plan)
    return ms.value, n.value


def cpra_launch_count() -> int:
    return int(lib().cpra_launch_count())


def _static_arg(a, name: str, dtype_np, dtype_torch: str, need: int):
    """Check one array of cpra_shrinkwrap_static without copying it: the call
    exists for callers that cannot allocate, so nothing is made contiguous or
    converted here.  Host arrays pass through to the C call, which rejects
    them (INVALID_ARG)."""
    if isinstance(a, np.ndarray):
        ok_type = a.dtype == dtype_np
        n, contig, ptr = a.size, a.flags.c_contiguous, a.ctypes.data
    elif hasattr(a, "data_ptr"):
        ok_type = str(a.dtype) == dtype_torch
        n, contig, ptr = a.numel(), a.is_contiguous(), a.data_ptr()
    else:
        raise TypeError(f"{name}: unsupported array type {type(a)}")
    if not ok_type:
        raise TypeError(f"{name} must be {dtype_torch}, got {a.dtype}")
    if n < need:
        raise ValueError(f"{name} holds {n} elements, count*N*N = {need} needed")
    if not contig:
        raise ValueError(f"{name} must be contiguous (no copy is made)")
    return ptr


def cpra_shrinkwrap_static(g, S_in, S_out, N: int, count: int, sigma: float, tau: float,
                           stream=None):
    """Shrink-wrap support update with no device allocation.

    g: float32 [count][N][N], S_in / S_out: uint8 [count][N][N], all
    contiguous device tensors on the current device; S_out may be S_in."""
    need = int(count) * int(N) * int(N)
    pg = _static_arg(g, "g", np.float32, "torch.float32", need)
    ps = _static_arg(S_in, "S_in", np.uint8, "torch.uint8", need)
    po = _static_arg(S_out, "S_out", np.uint8, "torch.uint8", need)
    _check(lib().cpra_shrinkwrap_static(pg, ps, po, N, count, sigma, tau, stream))


def cpra_batch_create(plans, use_graph: bool = True):
    hs = [p.h if isinstance(p, Plan) else p for p in plans]
    arr = (C.c_void_p * len(hs))(*[h.value if isinstance(h, C.c_void_p) else h for h in hs])
    out = C.c_void_p()
    _check(lib().cpra_batch_create(arr, len(hs), int(bool(use_graph)), C.byref(out)))
    return out


def cpra_batch_iterate(batch, n_iters: int):
    _check(lib().cpra_batch_iterate(batch, n_iters))


def cpra_batch_launches(batch, n_iters: int) -> int:
    return int(lib().cpra_batch_launches(batch, n_iters))


def cpra_batch_destroy(batch):
    _check(lib().cpra_batch_destroy(batch))


def cpra_autotune(N: int, precision: int = FP32, cache_path: str | None = None):
    eng, ms = C.c_int32(), C.c_double()
    _check(lib().cpra_autotune(N, precision, cache_path.encode() if cache_path else None,
                               C.byref(eng), C.byref(ms)))
    return eng.value, ms.value


def cpra_sync(plan):
    _check(lib().cpra_sync(plan), plan)


def cpra_destroy(plan):
    _check(lib().cpra_destroy(plan))


def cpra_last_error(plan=None) -> str:
    m = lib().cpra_last_error(plan)
    return m.decode() if m else ""


# ------------------------------------------------------------ convenience
class TorchAllocator:
    """Device memory from torch's caching allocator, handed to the library."""

    def __init__(self, device=None):
        import torch
        self.torch = torch
        self.device = device if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.blocks = {}
        self._alloc = ALLOC_FN(self._do_alloc)
        self._free = FREE_FN(self._do_free)

    def _do_alloc(self, nbytes, ctx):
        try:
            t = self.torch.empty(int(nbytes), dtype=self.torch.uint8, device=self.device)
        except Exception:  # OOM is reported to the library as NULL
            return None
        self.blocks[t.data_ptr()] = t
        return t.data_ptr()

    def _do_free(self, ptr, ctx):
        self.blocks.pop(ptr, None)


def make_config(N: int, Np: int, **kw) -> cpra_config:
    cfg = cpra_default_config(N, Np)
    alpha = kw.pop("alpha", None)
    if alpha is not None:
        cfg.n_taps = len(alpha)
        for i, a in enumerate(alpha):
            cfg.alpha[i] = float(a)
        for i in range(len(alpha), MAX_TAPS):
            cfg.alpha[i] = 0.0
    for k, v in kw.items():
        if not hasattr(cfg, k):
            raise AttributeError(f"cpra_config has no field {k}")
        setattr(cfg, k, v)
    return cfg


class Plan:
    """One reconstruction on one CUDA stream (see include/cpra.h)."""

    def __init__(self, cfg: cpra_config, stream=None, allocator: str = "torch"):
        self.cfg = cfg
        self._alloc = None
        if allocator == "torch":
            self._alloc = TorchAllocator()
            cfg.alloc = self._alloc._alloc
            cfg.free = self._alloc._free
        if stream is None:
            try:
                import torch
                stream = torch.cuda.current_stream().cuda_stream
            except Exception:
                stream = None
        self.stream = stream
        self.h = cpra_plan(cfg, stream)
        self.N, self.Np = cfg.N, cfg.Np
        self._downloads = []  # host buffers of queued downloads (assemble_3d_async)

    def load_intensities(self, I, first: int = 0, thetas=None):
        count = I.shape[0] if I.ndim == 3 else 1
        cpra_load_intensities(self.h, I, first, count, thetas)

    def load_support(self, S=None):
        per = 1 if (S is not None and S.ndim == 3) else 0
        if isinstance(S, np.ndarray):
            S = S.astype(np.uint8)
        cpra_load_support(self.h, S, per)

    def load_mask(self, mask=None):
        """Measured-pixel mask (centred; None = every pixel measured)."""
        per = 1 if (mask is not None and mask.ndim == 3) else 0
        if isinstance(mask, np.ndarray):
            mask = np.ascontiguousarray(mask.astype(np.uint8))
        cpra_load_mask(self.h, mask, per)

    def load_state(self, g, t: int):
        if isinstance(g, np.ndarray):
            g = g.astype(np.float32)
        cpra_load_state(self.h, g, t)

    def iterate(self, n: int, errors: bool = False):
        out = np.empty((n, self.Np), dtype=np.float64) if errors and n > 0 else None
        cpra_iterate(self.h, n, out)
        return out

    def assemble_3d(self, out=None):
        cpra_assemble_3d(self.h, out)
        return out

    def assemble_3d_async(self, out):
        """Assemble and queue the volume's download into out (pinned host
        memory); the plan keeps out alive until download_wait()."""
        need = self.N ** 3 * 8
        nbytes = out.nbytes if isinstance(out, np.ndarray) else out.numel() * out.element_size()
        if nbytes < need:
            raise ValueError(f"out holds {nbytes} bytes, N^3 complex64 = {need} needed")
        cpra_assemble_3d_async(self.h, out)
        self._downloads.append(out)
        return out

    def download_wait(self):
        cpra_download_wait(self.h)
        self._downloads.clear()

    def refine_3d(self, n: int, shrink_every: int = 0, sigma: float = 2.0, tau: float = 0.1):
        """Step D refinement; returns the n per-iteration errors."""
        out = np.empty(n, np.float64) if n > 0 else None
        cpra_refine_3d(self.h, n, shrink_every, sigma, tau, out)
        return out

    def result(self, what: int):
        N, Np = self.N, self.Np
        if what in (RESULT_PO, RESULT_STATE):
            a = np.empty((Np, N, N), np.float32)
        elif what == RESULT_SUPPORT:
            a = np.empty((Np, N, N), np.uint8)
        elif what == RESULT_ERRORS:
            a = np.empty((self.iteration, Np), np.float64)
        elif what == RESULT_VOLUME:
            a = np.empty((N, N, N), np.complex64)
        elif what == RESULT_MERGED_SPECTRA:
            a = np.empty((Np, N, N), np.complex64)
        else:
            raise ValueError(what)
        if a.nbytes:
            cpra_result(self.h, what, a, a.nbytes)
        return a

    def reset(self):
        cpra_reset(self.h)

    def set_present(self, mask=None):
        """Let only the angles with mask[n] != 0 iterate (None: every angle)."""
        if mask is not None:
            mask = np.ascontiguousarray(np.asarray(mask) != 0, dtype=np.uint8)
            if mask.shape != (self.Np,):
                raise ValueError("mask must hold Np entries")
        cpra_set_present(self.h, mask)

    def set_profiling(self, on: bool = True):
        cpra_set_profiling(self.h, on)

    def kernel_stats(self, kind: int):
        return cpra_kernel_stats(self.h, kind)

    @property
    def iteration(self) -> int:
        return cpra_iteration(self.h)

    def sync(self):
        cpra_sync(self.h)

    def close(self):
        if self.h:
            cpra_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Several plans iterated together (one launch per kernel and size group)."""

    def __init__(self, plans, use_graph: bool = True):
        self.plans = list(plans)  # keep the plans alive
        self.h = cpra_batch_create(self.plans, use_graph)

    def iterate(self, n: int):
        cpra_batch_iterate(self.h, n)

    def launches(self, n: int) -> int:
        return cpra_batch_launches(self.h, n)

    def set_persistent(self, mode: int = 1, wait_budget_s: float = 0.0, chunk_tiles: int = 0):
        _check(lib().cpra_batch_set_persistent(self.h, int(mode), float(wait_budget_s),
                                               int(chunk_tiles)))

    def close(self):
        if self.h:
            cpra_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """The library's serving thread (continuous batching of reconstructions)."""

    def __init__(self, hbm_reserve_bytes=None, max_active=0, iters_per_round=10, use_graph=True,
                 early_start=False, early_tail=0):
        cfg = cpra_server_config()
        _check(lib().cpra_server_default_config(C.byref(cfg)))
        if hbm_reserve_bytes is not None:
            cfg.hbm_reserve_bytes = int(hbm_reserve_bytes)
        cfg.max_active = max_active
        cfg.iters_per_round = iters_per_round
        cfg.use_graph = int(bool(use_graph))
        cfg.early_start = int(bool(early_start))
        cfg.early_tail = int(early_tail)
        self.h = C.c_void_p()
        _check(lib().cpra_server_start(C.byref(cfg), C.byref(self.h)))
        self.cfgs = {}

    def submit(self, cfg: cpra_config) -> int:
        rid = C.c_int64()
        _check(lib().cpra_server_submit(self.h, C.byref(cfg), C.byref(rid)))
        self.cfgs[rid.value] = (cfg.N, cfg.Np)
        return rid.value

    def push(self, rid: int, I, first: int, thetas=None):
        p, keep = _ptr(I)
        count = I.shape[0]
        th = None if thetas is None else np.ascontiguousarray(thetas, dtype=np.float64)
        _check(lib().cpra_server_push(self.h, rid, p, first, count,
                                      None if th is None else th.ctypes.data))
        del keep

    def poll(self, max_events: int = 64):
        evs = (cpra_server_event * max_events)()
        got = C.c_int32()
        _check(lib().cpra_server_poll(self.h, evs, max_events, C.byref(got)))
        return [dict(id=e.id, kind=e.kind, t_event=e.t_event, t_submit=e.t_submit,
                     t_last_pattern=e.t_last_pattern) for e in evs[:got.value]]

    def wait(self, rid: int, timeout_s: float = 60.0):
        _check(lib().cpra_server_wait(self.h, rid, timeout_s))

    def info(self, rid: int) -> dict:
        r = cpra_server_request()
        _check(lib().cpra_server_request_info(self.h, rid, C.byref(r)))
        return {k: getattr(r, k) for k, _ in cpra_server_request._fields_}

    def result(self, rid: int, what: int):
        N, Np = self.cfgs[rid]
        if what in (RESULT_PO, RESULT_STATE):
            a = np.empty((Np, N, N), np.float32)
        elif what == RESULT_VOLUME:
            a = np.empty((N, N, N), np.complex64)
        elif what == RESULT_MERGED_SPECTRA:
            a = np.empty((Np, N, N), np.complex64)
        elif what == RESULT_SUPPORT:
            a = np.empty((Np, N, N), np.uint8)
        elif what == RESULT_ERRORS:
            a = np.empty((self.info(rid)["iterations_done"], Np), np.float64)
        else:
            raise ValueError(what)
        _check(lib().cpra_server_result(self.h, rid, what, a.ctypes.data, a.nbytes))
        return a

    def release(self, rid: int):
        _check(lib().cpra_server_release(self.h, rid))

    def stats(self) -> dict:
        st = cpra_server_stats()
        _check(lib().cpra_server_get_stats(self.h, C.byref(st)))
        return {k: getattr(st, k) for k, _ in cpra_server_stats._fields_}

    def stop(self):
        if self.h:
            _check(lib().cpra_server_stop(self.h))
            self.h = None

    def __del__(self):
        try:
            self.stop()
        except Exception:
            pass
