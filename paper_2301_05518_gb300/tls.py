"""Python binding of the C ABI in include/tls.h (argument marshalling only).

Every function here has the name of the C entry point it calls and does no
arithmetic of its own: the smearing runs in libtls.so's CUDA kernels.  If the
library is missing or fails to load, importing this module raises: there is no
fallback path.

Arrays: pass torch tensors (CUDA or host) or numpy arrays; their data pointers
go to the library unchanged.  Complex tensors are accepted for vectors and
links (torch.complex128 / complex64 == [..., re, im] pairs of FP64 / FP32).

Paper: Gottlieb, Jeong, Strelchenko, arXiv:2301.05518, Sec. 2 (two-link
product, Eq. tlLapl1, Eq. tlSmear) and Sec. 3 (W precomputed and reused).
"""

from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libtls.so")

TLS_OK = 0
TLS_ERR_ARG = -1
TLS_ERR_NOMEM = -2
TLS_ERR_ADMIT = -3
TLS_ERR_CUDA = -4
TLS_ERR_TIMEOUT = -5
TLS_ERR_NOT_BUILT = -6
TLS_ERR_DEVICE = -7
TLS_ERR_STATE = -8
TLS_ERR_UNSUPPORTED = -9
TLS_ERR_NOT_FOUND = -10

TLS_F64, TLS_F32, TLS_F16, TLS_BF16 = 0, 1, 2, 3
TLS_R18, TLS_R12, TLS_R8 = 18, 12, 8
TLS_KERNEL_AUTO, TLS_KERNEL_SINGLE, TLS_KERNEL_MRHS, TLS_KERNEL_PERSISTENT = 0, 1, 2, 3
TLS_KERNEL_MRHS_ROWS = 4
TLS_KERNEL_MRHS_ZM = 5
TLS_ALL_T = -1
TLS_PEAK_F64, TLS_PEAK_F32, TLS_PEAK_F32X2 = 0, 1, 2

#: every symbol include/tls.h declares
EXPORTS = (
    "tls_create", "tls_destroy", "tls_last_error", "tls_version", "tls_bytes_in_use",
    "tls_load_gauge", "tls_build_twolink", "tls_free_gauge", "tls_export_twolink",
    "tls_export_gauge", "tls_smear", "tls_set_profiling", "tls_get_profile",
    "tls_smear_noalloc", "tls_build_links", "tls_ape_smear", "tls_smear_onelink", "tls_set_barrier_budget", "tls_autotune", "tls_tune_set", "tls_serve_start", "tls_serve_stop", "tls_serve_submit",
    "tls_serve_poll", "tls_serve_wait", "tls_peak_flops",
)


class tls_profile(ctypes.Structure):
    _fields_ = [
        ("ms_total", ctypes.c_double), ("ms_h2d", ctypes.c_double), ("ms_pack", ctypes.c_double),
        ("ms_iter", ctypes.c_double), ("ms_unpack", ctypes.c_double), ("ms_d2h", ctypes.c_double),
        ("ms_build", ctypes.c_double), ("launches", ctypes.c_int64),
        ("iter_launches", ctypes.c_int64), ("iter_bytes", ctypes.c_double),
        ("iter_flops", ctypes.c_double), ("kernel", ctypes.c_int), ("vecs_per_thread", ctypes.c_int),
    ]


class tls_tune_entry(ctypes.Structure):
    _fields_ = [("kernel", ctypes.c_int), ("vecs_per_thread", ctypes.c_int), ("threads", ctypes.c_int),
                ("tile", ctypes.c_int * 3), ("ms_per_step", ctypes.c_double)]


class tls_serve_opts(ctypes.Structure):
    _fields_ = [("max_slots", ctypes.c_int), ("steps_per_launch", ctypes.c_int),
                ("use_graphs", ctypes.c_int), ("reserved", ctypes.c_int * 5)]


class tls_job(ctypes.Structure):
    _fields_ = [("gauge", ctypes.c_int64), ("vecs", ctypes.c_void_p), ("vecs_on_device", ctypes.c_int),
                ("io_prec", ctypes.c_int), ("nvec", ctypes.c_int), ("N", ctypes.c_int),
                ("width", ctypes.c_double), ("timeslice", ctypes.c_int), ("storage", ctypes.c_int),
                ("reserved", ctypes.c_int * 4)]


class tls_job_result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("submit_ms", ctypes.c_double),
                ("start_ms", ctypes.c_double), ("done_ms", ctypes.c_double)]


def _load() -> ctypes.CDLL:
    if not os.path.exists(LIB_PATH):
        raise ImportError(
            "libtls.so is not built (%s); run paper_2301_05518_gb300.build.build() "
            "or __graft_entry__.build() first" % LIB_PATH)
    lib = ctypes.CDLL(LIB_PATH)
    P, I, D, I64, U64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_int64, ctypes.c_uint64
    sig = {
        "tls_create": ([ctypes.POINTER(P), I, U64], I),
        "tls_destroy": ([P], None),
        "tls_last_error": ([], ctypes.c_char_p),
        "tls_version": ([], I),
        "tls_bytes_in_use": ([P], U64),
        "tls_load_gauge": ([P, P, I, P, I, P, ctypes.POINTER(I64)], I),
        "tls_build_twolink": ([P, I64, I, I, I, P], I),
        "tls_free_gauge": ([P, I64], I),
        "tls_export_twolink": ([P, I64, P, I, P], I),
        "tls_export_gauge": ([P, I64, P, I, P], I),
        "tls_smear": ([P, I64, P, I, I, I, I, D, I, I, I, P, P], I),
        "tls_smear_noalloc": ([P, I64, P, I, I, I, D, I, I, P], I),
        "tls_build_links": ([P, I64, I, I, P], I),
        "tls_ape_smear": ([P, I64, D, I, P], I),
        "tls_smear_onelink": ([P, I64, P, I, I, I, I, D, I, I, P, P], I),
        "tls_set_profiling": ([P, I], I),
        "tls_get_profile": ([P, ctypes.POINTER(tls_profile)], I),
        "tls_set_barrier_budget": ([P, I64], I),
        "tls_autotune": ([P, I64, I, I, I, I, ctypes.POINTER(tls_tune_entry), ctypes.POINTER(tls_tune_entry),
                          I, ctypes.POINTER(I)], I),
        "tls_tune_set": ([P, I64, I, I, I, ctypes.POINTER(tls_tune_entry)], I),
        "tls_serve_start": ([P, ctypes.POINTER(tls_serve_opts)], I),
        "tls_serve_stop": ([P], I),
        "tls_serve_submit": ([P, ctypes.POINTER(tls_job), ctypes.POINTER(U64)], I),
        "tls_serve_poll": ([P, U64, ctypes.POINTER(I)], I),
        "tls_serve_wait": ([P, U64, D, ctypes.POINTER(tls_job_result)], I),
        "tls_peak_flops": ([I, I, ctypes.POINTER(D)], I),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    return lib


lib = _load()


class TLSError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__("tls status %d: %s" % (status, msg))
        self.status = status


def _check(status: int) -> int:
    if status != TLS_OK:
        raise TLSError(status, lib.tls_last_error().decode(errors="replace"))
    return status


def _ptr(a):
    """(data pointer, on_device) of a torch tensor or numpy array."""
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("array must be contiguous")
        return ctypes.c_void_p(a.data_ptr()), 1 if a.is_cuda else 0
    a = np.asarray(a)
    if not a.flags.c_contiguous:
        raise ValueError("array must be C-contiguous")
    return ctypes.c_void_p(a.ctypes.data), 0


def _stream(stream):
    if stream is None:
        return None
    if hasattr(stream, "cuda_stream"):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(int(stream))


# ---- functions with the C names -------------------------------------------------
def tls_version() -> int:
    return lib.tls_version()


def tls_last_error() -> str:
    return lib.tls_last_error().decode(errors="replace")


def tls_create(device: int = 0, hbm_cap_bytes: int = 0):
    h = ctypes.c_void_p()
    _check(lib.tls_create(ctypes.byref(h), int(device), int(hbm_cap_bytes)))
    return h


def tls_destroy(ctx) -> None:
    lib.tls_destroy(ctx)


def tls_bytes_in_use(ctx) -> int:
    return int(lib.tls_bytes_in_use(ctx))


def tls_load_gauge(ctx, U, nd: int, dims, stream=None) -> int:
    """U: [Lt, Lz, Ly, Lx, nd, 3, 3] complex128 (or the real view); dims = (Lx, Ly, Lz, Lt)."""
    p, on_dev = _ptr(U)
    d = (ctypes.c_int * 4)(*[int(x) for x in dims])
    out = ctypes.c_int64()
    _check(lib.tls_load_gauge(ctx, p, int(nd), d, on_dev, _stream(stream), ctypes.byref(out)))
    return out.value


def tls_build_twolink(ctx, gauge: int, wprec: int = TLS_F32, recon: int = TLS_R18, keep_U: int = 1,
                      stream=None) -> None:
    _check(lib.tls_build_twolink(ctx, int(gauge), int(wprec), int(recon), int(keep_U), _stream(stream)))


def tls_free_gauge(ctx, gauge: int) -> None:
    _check(lib.tls_free_gauge(ctx, int(gauge)))


def tls_export_twolink(ctx, gauge: int, out, stream=None) -> None:
    p, on_dev = _ptr(out)
    _check(lib.tls_export_twolink(ctx, int(gauge), p, on_dev, _stream(stream)))


def tls_export_gauge(ctx, gauge: int, out, stream=None) -> None:
    p, on_dev = _ptr(out)
    _check(lib.tls_export_gauge(ctx, int(gauge), p, on_dev, _stream(stream)))


def tls_smear(ctx, gauge: int, vecs, io_prec: int, nvec: int, N: int, width: float,
              timeslice: int = TLS_ALL_T, storage: int = TLS_F32, kernel: int = TLS_KERNEL_AUTO,
              stream=None, norms: bool = False):
    """Smears vecs in place; returns the FP64 norms (numpy) if norms=True, else None."""
    p, on_dev = _ptr(vecs)
    nout = np.zeros(int(nvec), dtype=np.float64) if norms else None
    nptr = ctypes.c_void_p(nout.ctypes.data) if norms else None
    _check(lib.tls_smear(ctx, int(gauge), p, int(io_prec), on_dev, int(nvec), int(N), float(width),
                         int(timeslice), int(storage), int(kernel), _stream(stream), nptr))
    return nout


def tls_build_links(ctx, gauge: int, prec: int = TLS_F32, keep_U: int = 1, stream=None) -> None:
    _check(lib.tls_build_links(ctx, int(gauge), int(prec), int(keep_U), _stream(stream)))


def tls_ape_smear(ctx, gauge: int, alpha: float, n_steps: int, stream=None) -> None:
    """Replaces the resident links by n_steps APE steps (projection onto SU(3))."""
    _check(lib.tls_ape_smear(ctx, int(gauge), float(alpha), int(n_steps), _stream(stream)))


def tls_smear_onelink(ctx, gauge: int, vecs, io_prec: int, nvec: int, N: int, alpha: float,
                      timeslice: int = TLS_ALL_T, storage: int = TLS_F32, stream=None, norms: bool = False):
    """One-link Gaussian smearing (1 + alpha H)^N (Eq. 3, C = 1), in place."""
    p, on_dev = _ptr(vecs)
    nout = np.zeros(int(nvec), dtype=np.float64) if norms else None
    nptr = ctypes.c_void_p(nout.ctypes.data) if norms else None
    _check(lib.tls_smear_onelink(ctx, int(gauge), p, int(io_prec), on_dev, int(nvec), int(N), float(alpha),
                                 int(timeslice), int(storage), _stream(stream), nptr))
    return nout


def tls_smear_noalloc(ctx, gauge: int, vecs, io_prec: int, nvec: int, N: int, width: float,
                      timeslice: int = TLS_ALL_T, storage: int = TLS_F32, stream=None) -> None:
    """The persistent smear with the library's static scratch: allocates nothing."""
    p, on_dev = _ptr(vecs)
    _check(lib.tls_smear_noalloc(ctx, int(gauge), p, int(io_prec), int(nvec), int(N), float(width),
                                 int(timeslice), int(storage), _stream(stream)))


def tls_set_profiling(ctx, on: bool = True) -> None:
    _check(lib.tls_set_profiling(ctx, 1 if on else 0))


def tls_get_profile(ctx) -> dict:
    p = tls_profile()
    _check(lib.tls_get_profile(ctx, ctypes.byref(p)))
    return {name: getattr(p, name) for name, _ in tls_profile._fields_}


def tls_set_barrier_budget(ctx, polls: int) -> None:
    _check(lib.tls_set_barrier_budget(ctx, int(polls)))


def _entry(e):
    return {"kernel": e.kernel, "vecs_per_thread": e.vecs_per_thread, "threads": e.threads,
            "tile": list(e.tile), "ms_per_step": e.ms_per_step}


def tls_autotune(ctx, gauge: int, nvec: int, storage: int, timeslice: int = TLS_ALL_T, steps: int = 4):
    """Returns (best, all candidates) as dicts; the best goes to the context's table."""
    best = tls_tune_entry()
    arr = (tls_tune_entry * 128)()
    n = ctypes.c_int()
    _check(lib.tls_autotune(ctx, int(gauge), int(nvec), int(storage), int(timeslice), int(steps),
                            ctypes.byref(best), arr, 128, ctypes.byref(n)))
    return _entry(best), [_entry(arr[k]) for k in range(min(n.value, 128))]


def tls_tune_set(ctx, gauge: int, nvec: int, storage: int, timeslice: int, kernel: int,
                 vecs_per_thread: int = 1, threads: int = 256, tile=(0, 0, 0)) -> None:
    e = tls_tune_entry(int(kernel), int(vecs_per_thread), int(threads), (ctypes.c_int * 3)(*tile), 0.0)
    _check(lib.tls_tune_set(ctx, int(gauge), int(nvec), int(storage), int(timeslice), ctypes.byref(e)))


def tls_serve_start(ctx, max_slots: int = 64, steps_per_launch: int = 1, use_graphs: int = 1) -> None:
    o = tls_serve_opts(max_slots, steps_per_launch, use_graphs)
    _check(lib.tls_serve_start(ctx, ctypes.byref(o)))


def tls_serve_stop(ctx) -> None:
    _check(lib.tls_serve_stop(ctx))


def tls_serve_submit(ctx, gauge: int, vecs, io_prec: int, nvec: int, N: int, width: float,
                     timeslice: int = TLS_ALL_T, storage: int = TLS_F32) -> int:
    p, on_dev = _ptr(vecs)
    j = tls_job(int(gauge), p.value, on_dev, int(io_prec), int(nvec), int(N), float(width),
                int(timeslice), int(storage))
    jid = ctypes.c_uint64()
    _check(lib.tls_serve_submit(ctx, ctypes.byref(j), ctypes.byref(jid)))
    return jid.value


def tls_serve_poll(ctx, job_id: int) -> bool:
    d = ctypes.c_int()
    _check(lib.tls_serve_poll(ctx, int(job_id), ctypes.byref(d)))
    return bool(d.value)


def tls_serve_wait(ctx, job_id: int, timeout_s: float = 60.0) -> dict:
    r = tls_job_result()
    _check(lib.tls_serve_wait(ctx, int(job_id), float(timeout_s), ctypes.byref(r)))
    return {"status": r.status, "submit_ms": r.submit_ms, "start_ms": r.start_ms, "done_ms": r.done_ms}


# ---- a small owner object ------------------------------------------------------
def tls_peak_flops(device: int, kind: int) -> float:
    """Measured arithmetic rate of the GPU in TFLOP/s (TLS_PEAK_F64 / F32 / F32X2)."""
    out = ctypes.c_double(0.0)
    _check(lib.tls_peak_flops(device, kind, ctypes.byref(out)))
    return out.value


class Context:
    """Owns a tls_ctx; the methods are the C entry points minus the prefix."""

    def __init__(self, device: int = 0, hbm_cap_bytes: int = 0):
        self.h = tls_create(device, hbm_cap_bytes)

    def close(self):
        if self.h is not None:
            tls_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def load_gauge(self, U, nd, dims, stream=None):
        return tls_load_gauge(self.h, U, nd, dims, stream)

    def build_twolink(self, gauge, wprec=TLS_F32, recon=TLS_R18, keep_U=1, stream=None):
        return tls_build_twolink(self.h, gauge, wprec, recon, keep_U, stream)

    def free_gauge(self, gauge):
        return tls_free_gauge(self.h, gauge)

    def export_twolink(self, gauge, out, stream=None):
        return tls_export_twolink(self.h, gauge, out, stream)

    def export_gauge(self, gauge, out, stream=None):
        return tls_export_gauge(self.h, gauge, out, stream)

    def smear(self, gauge, vecs, io_prec, nvec, N, width, timeslice=TLS_ALL_T, storage=TLS_F32,
              kernel=TLS_KERNEL_AUTO, stream=None, norms=False):
        return tls_smear(self.h, gauge, vecs, io_prec, nvec, N, width, timeslice, storage, kernel,
                         stream, norms)

    def build_links(self, gauge, prec=TLS_F32, keep_U=1, stream=None):
        return tls_build_links(self.h, gauge, prec, keep_U, stream)

    def ape_smear(self, gauge, alpha, n_steps, stream=None):
        return tls_ape_smear(self.h, gauge, alpha, n_steps, stream)

    def smear_onelink(self, gauge, vecs, io_prec, nvec, N, alpha, timeslice=TLS_ALL_T, storage=TLS_F32,
                      stream=None, norms=False):
        return tls_smear_onelink(self.h, gauge, vecs, io_prec, nvec, N, alpha, timeslice, storage, stream, norms)

    def smear_noalloc(self, gauge, vecs, io_prec, nvec, N, width, timeslice=TLS_ALL_T, storage=TLS_F32,
                      stream=None):
        return tls_smear_noalloc(self.h, gauge, vecs, io_prec, nvec, N, width, timeslice, storage, stream)

    def set_profiling(self, on=True):
        return tls_set_profiling(self.h, on)

    def get_profile(self):
        return tls_get_profile(self.h)

    def set_barrier_budget(self, polls):
        return tls_set_barrier_budget(self.h, polls)

    def autotune(self, gauge, nvec, storage, timeslice=TLS_ALL_T, steps=4):
        return tls_autotune(self.h, gauge, nvec, storage, timeslice, steps)

    def tune_set(self, gauge, nvec, storage, timeslice, kernel, vecs_per_thread=1, threads=256, tile=(0, 0, 0)):
        return tls_tune_set(self.h, gauge, nvec, storage, timeslice, kernel, vecs_per_thread, threads, tile)

    def bytes_in_use(self):
        return tls_bytes_in_use(self.h)

    def serve_start(self, max_slots=64, steps_per_launch=1, use_graphs=1):
        return tls_serve_start(self.h, max_slots, steps_per_launch, use_graphs)

    def serve_stop(self):
        return tls_serve_stop(self.h)

    def serve_submit(self, gauge, vecs, io_prec, nvec, N, width, timeslice=TLS_ALL_T, storage=TLS_F32):
        return tls_serve_submit(self.h, gauge, vecs, io_prec, nvec, N, width, timeslice, storage)

    def serve_poll(self, job_id):
        return tls_serve_poll(self.h, job_id)

    def serve_wait(self, job_id, timeout_s=60.0):
        return tls_serve_wait(self.h, job_id, timeout_s)
