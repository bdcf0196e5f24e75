"""GB300 polyphase filter bank (PFB) channeliser -- Python binding.

Thin ctypes marshalling over the C ABI declared in ``include/pfb.h``
(``libpfb.so``, built in-tree by :func:`paper_2408_16551_gb300.build.build`).
Every step of the channeliser runs in the library's CUDA kernels; PyTorch is
used only for device memory and CUDA streams.  There is no CPU fallback: if
the compiled library is missing, importing the binding's entry points raises.

The operation (TINA, arXiv 2408.16551, Sec. 5.2 with Sec. 4.3/4.1): frames of
P samples, a T-tap FIR per branch, then a P-point DFT of each spectrum:
    y[s,p] = sum_{m<T} h[mP+p] x[(s+m)P+p],   X[s,k] = sum_p y[s,p] e^{-2 pi i pk/P}.
"""

from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libpfb.so")

# ---- enums (pfb.h) --------------------------------------------------------
PFB_OK, PFB_PENDING = 0, 1
PFB_ERR_INVALID, PFB_ERR_OOM, PFB_ERR_CUDA, PFB_ERR_BUSY = -1, -2, -3, -4
PFB_ERR_TIMEOUT, PFB_ERR_INTERNAL, PFB_ERR_UNSUPPORTED = -5, -6, -7
PFB_IN_R32, PFB_IN_C64, PFB_IN_CI8 = 0, 1, 2
PFB_WIN_HANN, PFB_WIN_HAMMING, PFB_WIN_BLACKMAN, PFB_WIN_USER = 0, 1, 2, 3
PFB_DFT_FFT_F32, PFB_DFT_GEMM_F32, PFB_DFT_GEMM_BF16X3 = 0, 1, 2
PFB_TAPS_CORRELATION, PFB_TAPS_CONVOLUTION = 0, 1
PFB_HOST_ROUTE_AUTO, PFB_HOST_ROUTE_STAGED = 0, 1
HOST_ROUTE_NAMES = {0: "none", 1: "staged", 2: "mapped"}  # pfb_last_host_route
NOALLOC_SCRATCH_BYTES = 32 << 20  # PFB_NOALLOC_SCRATCH_BYTES

EXPORTED = [
    "pfb_plan_create", "pfb_plan_destroy", "pfb_out_spectra", "pfb_plan_get_taps", "pfb_execute",
    "pfb_execute_host", "pfb_execute_batch", "pfb_batch_create", "pfb_batch_launch", "pfb_batch_destroy",
    "pfb_server_create", "pfb_server_destroy", "pfb_stream_open", "pfb_stream_close",
    "pfb_stream_next_spectra", "pfb_submit", "pfb_poll", "pfb_wait", "pfb_server_get_stats",
    "pfb_status_string", "pfb_last_error", "pfb_launch_count", "pfb_plan_kernel_name",
    "pfb_plan_num_variants", "pfb_plan_variant", "pfb_plan_set_variant", "pfb_plan_autotune",
    "pfb_execute_host_noalloc", "pfb_stream_state_size", "pfb_stream_state_export", "pfb_stream_state_import",
    "pfb_synth_out_samples", "pfb_synthesize", "pfb_plan_status", "pfb_plan_set_fault",
    "pfb_execute_batch_host", "pfb_submit_chunks", "pfb_ticket_times", "pfb_set_host_route",
    "pfb_last_host_route",
]


class pfb_plan_desc(ctypes.Structure):
    _fields_ = [("P", ctypes.c_int32), ("T", ctypes.c_int32), ("in_dtype", ctypes.c_int32),
                ("in_scale", ctypes.c_float), ("window", ctypes.c_int32), ("path", ctypes.c_int32),
                ("user_taps_host", ctypes.POINTER(ctypes.c_double)), ("device", ctypes.c_int32),
                ("hop", ctypes.c_int32), ("tap_order", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class pfb_batch_item(ctypes.Structure):
    _fields_ = [("plan", ctypes.c_void_p), ("d_in", ctypes.c_void_p), ("n_samples", ctypes.c_int64),
                ("d_out", ctypes.c_void_p), ("out_cap_spectra", ctypes.c_int64)]


class pfb_server_desc(ctypes.Structure):
    _fields_ = [("hbm_budget_bytes", ctypes.c_int64), ("max_slots", ctypes.c_int32),
                ("timeout_ms", ctypes.c_int32), ("queue_when_busy", ctypes.c_int32), ("device", ctypes.c_int32)]


class pfb_server_stats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int64) for n in ("submitted", "completed", "failed", "rejected", "queued_now",
                                              "in_flight_now", "reserved_bytes_now", "peak_reserved_bytes",
                                              "samples_completed", "batches", "batched_requests")] + \
               [(n, ctypes.c_double) for n in ("p50_latency_us", "p99_latency_us", "mean_latency_us")]


class PFBError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{_status_name(status)}: {msg}")
        self.status = status


_lib = None
_lock = threading.Lock()


def _status_name(st: int) -> str:
    names = {0: "PFB_OK", 1: "PFB_PENDING", -1: "PFB_ERR_INVALID", -2: "PFB_ERR_OOM", -3: "PFB_ERR_CUDA",
             -4: "PFB_ERR_BUSY", -5: "PFB_ERR_TIMEOUT", -6: "PFB_ERR_INTERNAL", -7: "PFB_ERR_UNSUPPORTED"}
    return names.get(st, f"status {st}")


def lib() -> ctypes.CDLL:
    """Load libpfb.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libpfb.so is not built ({LIB_PATH}); run paper_2408_16551_gb300.build.build()")
        L = ctypes.CDLL(LIB_PATH)
        vp, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32
        st = ctypes.c_int
        sig = {
            "pfb_plan_create": (st, [ctypes.POINTER(pfb_plan_desc), ctypes.POINTER(vp)]),
            "pfb_plan_destroy": (st, [vp]),
            "pfb_plan_status": (st, [vp]),
            "pfb_plan_set_fault": (st, [vp, i32, i64]),
            "pfb_out_spectra": (i64, [vp, i64]),
            "pfb_plan_get_taps": (st, [vp, ctypes.POINTER(ctypes.c_double), i64]),
            "pfb_execute": (st, [vp, vp, i64, vp, i64, vp]),
            "pfb_execute_host": (st, [vp, vp, i64, vp, i64, vp]),
            "pfb_execute_host_noalloc": (st, [vp, vp, i64, vp, i64, vp]),
            "pfb_stream_state_size": (i64, [vp, i64]),
            "pfb_synth_out_samples": (i64, [vp, i64]),
            "pfb_synthesize": (st, [vp, vp, i64, vp, i64, vp]),
            "pfb_stream_state_export": (st, [vp, i64, vp, i64]),
            "pfb_stream_state_import": (st, [vp, i64, vp, i64]),
            "pfb_execute_batch": (st, [ctypes.POINTER(pfb_batch_item), i32, vp]),
            "pfb_execute_batch_host": (st, [ctypes.POINTER(pfb_batch_item), i32, vp]),
            "pfb_set_host_route": (st, [i32]),
            "pfb_last_host_route": (i32, []),
            "pfb_batch_create": (st, [ctypes.POINTER(pfb_batch_item), i32, ctypes.POINTER(vp)]),
            "pfb_batch_launch": (st, [vp, vp]),
            "pfb_batch_destroy": (st, [vp]),
            "pfb_server_create": (st, [ctypes.POINTER(pfb_server_desc), ctypes.POINTER(vp)]),
            "pfb_server_destroy": (st, [vp]),
            "pfb_stream_open": (st, [vp, vp, ctypes.POINTER(i64)]),
            "pfb_stream_close": (st, [vp, i64]),
            "pfb_stream_next_spectra": (i64, [vp, i64, i64]),
            "pfb_submit": (st, [vp, i64, vp, i64, vp, i64, ctypes.POINTER(i64)]),
            "pfb_poll": (st, [vp, i64]),
            "pfb_submit_chunks": (st, [vp, i64, vp, i32, i64, vp, i64, ctypes.POINTER(i64)]),
            "pfb_ticket_times": (st, [vp, i64, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]),
            "pfb_wait": (st, [vp, i64, i32]),
            "pfb_server_get_stats": (st, [vp, ctypes.POINTER(pfb_server_stats)]),
            "pfb_status_string": (ctypes.c_char_p, [st]),
            "pfb_last_error": (ctypes.c_char_p, []),
            "pfb_launch_count": (i64, []),
            "pfb_plan_kernel_name": (ctypes.c_char_p, [vp]),
            "pfb_plan_num_variants": (i32, [vp]),
            "pfb_plan_variant": (i32, [vp]),
            "pfb_plan_set_variant": (st, [vp, i32]),
            "pfb_plan_autotune": (st, [vp, i64, vp, ctypes.POINTER(ctypes.c_double)]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
        return L


def _check(st: int, what: str = "") -> int:
    if st < 0:
        msg = lib().pfb_last_error().decode()
        raise PFBError(st, f"{what}: {msg}" if what else msg)
    return st


def launch_count() -> int:
    return int(lib().pfb_launch_count())


# ---- torch helpers (memory and streams only) ------------------------------

def _stream_handle(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _in_samples(x, in_dtype: int) -> int:
    if in_dtype == PFB_IN_CI8:
        return x.numel() // 2
    return x.numel()


def _check_input(x, in_dtype: int):
    import torch
    want = {PFB_IN_R32: torch.float32, PFB_IN_C64: torch.complex64, PFB_IN_CI8: torch.int8}[in_dtype]
    if x.dtype != want:
        raise TypeError(f"input dtype {x.dtype} does not match the plan ({want})")
    if not x.is_cuda or not x.is_contiguous():
        raise ValueError("input must be a contiguous CUDA tensor")


# ---- plans ----------------------------------------------------------------

class Plan:
    """A channeliser plan (pfb_plan_create): P branches, T taps, dtype, DFT path."""

    def __init__(self, P: int, T: int, in_dtype: int = PFB_IN_C64, window: int = PFB_WIN_HANN,
                 path: int = PFB_DFT_FFT_F32, in_scale: float = 1.0, user_taps=None, device: int = -1,
                 hop: int = 0, tap_order: int = PFB_TAPS_CORRELATION):
        d = pfb_plan_desc()
        d.P, d.T, d.in_dtype, d.in_scale, d.window, d.path = P, T, in_dtype, in_scale, window, path
        d.device, d.hop, d.tap_order, d.reserved = device, hop, tap_order, 0
        self._taps_keep = None
        if user_taps is not None:
            arr = np.ascontiguousarray(user_taps, dtype=np.float64)
            self._taps_keep = arr
            d.user_taps_host = arr.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        h = ctypes.c_void_p()
        _check(lib().pfb_plan_create(ctypes.byref(d), ctypes.byref(h)), "pfb_plan_create")
        self.handle = h
        self.P, self.T, self.in_dtype, self.window, self.path = P, T, in_dtype, window, path
        self.hop = hop if hop else P   # samples between consecutive spectra

    def close(self):
        if getattr(self, "handle", None):
            lib().pfb_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def kernel_name(self) -> str:
        return lib().pfb_plan_kernel_name(self.handle).decode()

    @property
    def variant(self) -> int:
        return int(lib().pfb_plan_variant(self.handle))

    @variant.setter
    def variant(self, v: int):
        _check(lib().pfb_plan_set_variant(self.handle, v), "pfb_plan_set_variant")

    @property
    def num_variants(self) -> int:
        return int(lib().pfb_plan_num_variants(self.handle))

    def autotune(self, n_samples: int, stream=None) -> float:
        """pfb_plan_autotune: time each variant, keep the fastest; returns its ms per call."""
        ms = ctypes.c_double()
        _check(lib().pfb_plan_autotune(self.handle, n_samples, _stream_handle(stream), ctypes.byref(ms)),
               "pfb_plan_autotune")
        return ms.value

    def out_spectra(self, n_samples: int) -> int:
        return int(lib().pfb_out_spectra(self.handle, n_samples))

    def status(self) -> int:
        """pfb_plan_status: read and clear the kernel error word of the plan's
        launches (PFB_OK, PFB_ERR_TIMEOUT, PFB_ERR_INTERNAL); non-blocking."""
        return int(lib().pfb_plan_status(self.handle))

    def set_fault(self, mode: int, wait_ns: int = 0):
        """pfb_plan_set_fault: error-reporting test hook (mode 1: the producer of
        the single-CTA warp-specialised FFT kernel issues no copies, so its
        consumers' bounded waits of wait_ns run out; mode 0: normal)."""
        _check(lib().pfb_plan_set_fault(self.handle, mode, wait_ns), "pfb_plan_set_fault")

    def taps(self) -> np.ndarray:
        """FP64 prototype filter h[0..P*T) as generated on the GPU."""
        h = np.zeros(self.P * self.T, dtype=np.float64)
        _check(lib().pfb_plan_get_taps(self.handle, h.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), h.size),
               "pfb_plan_get_taps")
        return h

    def execute(self, x, out=None, stream=None):
        """pfb_execute on a CUDA tensor; returns complex64 [S, P] (asynchronous)."""
        import torch
        _check_input(x, self.in_dtype)
        n = _in_samples(x, self.in_dtype)
        S = self.out_spectra(n)
        if out is None:
            out = torch.empty((S, self.P), dtype=torch.complex64, device=x.device)
        cap = out.numel() // self.P
        _check(lib().pfb_execute(self.handle, ctypes.c_void_p(x.data_ptr()), n, ctypes.c_void_p(out.data_ptr()),
                                 cap, _stream_handle(stream)), "pfb_execute")
        return out[:S] if out.shape[0] != S else out

    def synth_out_samples(self, n_spectra: int) -> int:
        return int(lib().pfb_synth_out_samples(self.handle, n_spectra))

    def synthesize(self, X, out=None, stream=None):
        """pfb_synthesize: the synthesis (inverse) filter bank of complex64 spectra
        [S, P] on the device; returns complex64 [(S + T - 1) * P] (asynchronous)."""
        import torch
        if X.dtype != torch.complex64 or not X.is_cuda or not X.is_contiguous() or X.dim() != 2 or X.shape[1] != self.P:
            raise ValueError("spectra must be a contiguous complex64 CUDA tensor [S, P]")
        S = X.shape[0]
        n = self.synth_out_samples(S)
        if out is None:
            out = torch.empty((max(n, 0),), dtype=torch.complex64, device=X.device)
        _check(lib().pfb_synthesize(self.handle, ctypes.c_void_p(X.data_ptr()), S, ctypes.c_void_p(out.data_ptr()),
                                    out.numel(), _stream_handle(stream)), "pfb_synthesize")
        return out[:n] if out.numel() != n else out

    def execute_host(self, x: np.ndarray, out: np.ndarray | None = None, stream=None) -> np.ndarray:
        """pfb_execute_host: host buffers in and out (copies inside the call)."""
        n = x.size // 2 if self.in_dtype == PFB_IN_CI8 else x.size
        S = self.out_spectra(n)
        if out is None:
            out = np.empty((S, self.P), dtype=np.complex64)
        _check(lib().pfb_execute_host(self.handle, ctypes.c_void_p(x.ctypes.data), n,
                                      ctypes.c_void_p(out.ctypes.data), out.size // self.P,
                                      _stream_handle(stream)), "pfb_execute_host")
        return out

    def execute_host_noalloc(self, x: np.ndarray, out: np.ndarray | None = None, stream=None) -> np.ndarray:
        """pfb_execute_host_noalloc: as execute_host, staged through the library's
        static device area (no device allocation; input + output at most
        NOALLOC_SCRATCH_BYTES)."""
        n = x.size // 2 if self.in_dtype == PFB_IN_CI8 else x.size
        S = self.out_spectra(n)
        if out is None:
            out = np.empty((S, self.P), dtype=np.complex64)
        _check(lib().pfb_execute_host_noalloc(self.handle, ctypes.c_void_p(x.ctypes.data), n,
                                              ctypes.c_void_p(out.ctypes.data), out.size // self.P,
                                              _stream_handle(stream)), "pfb_execute_host_noalloc")
        return out


def pfb_execute(plan: Plan, x, out=None, stream=None):
    return plan.execute(x, out=out, stream=stream)


def _items(entries):
    arr = (pfb_batch_item * max(1, len(entries)))()
    for i, (plan, x, out) in enumerate(entries):
        n = _in_samples(x, plan.in_dtype)
        arr[i].plan = plan.handle.value
        arr[i].d_in = x.data_ptr()
        arr[i].n_samples = n
        arr[i].d_out = out.data_ptr() if out is not None and out.numel() else None
        arr[i].out_cap_spectra = (out.numel() // plan.P) if out is not None else 0
    return arr


def pfb_execute_batch(entries, stream=None):
    """entries: list of (Plan, input tensor, output tensor [>=S, P])."""
    arr = _items(entries)
    _check(lib().pfb_execute_batch(arr, len(entries), _stream_handle(stream)), "pfb_execute_batch")


def pfb_execute_batch_host(entries, stream=None):
    """entries: list of (Plan, host input ndarray, host output ndarray [>=S, P]
    complex64); pfb_execute_batch_host runs them in place (page-locked
    buffers and a kernel that reads them per thread) or stages them through
    the device, and returns once every output is written."""
    arr = (pfb_batch_item * max(1, len(entries)))()
    for i, (plan, x, out) in enumerate(entries):
        n = x.size // 2 if plan.in_dtype == PFB_IN_CI8 else x.size
        arr[i].plan = plan.handle.value
        arr[i].d_in = x.ctypes.data
        arr[i].n_samples = n
        arr[i].d_out = out.ctypes.data if out is not None and out.size else None
        arr[i].out_cap_spectra = (out.size // plan.P) if out is not None else 0
    _check(lib().pfb_execute_batch_host(arr, len(entries), _stream_handle(stream)), "pfb_execute_batch_host")


def set_host_route(route: int) -> None:
    """pfb_set_host_route: PFB_HOST_ROUTE_AUTO (mapped when possible) or PFB_HOST_ROUTE_STAGED."""
    _check(lib().pfb_set_host_route(route), "pfb_set_host_route")


def last_host_route() -> str:
    """The route this thread's last pfb_execute_batch_host took: "staged", "mapped" or "none"."""
    return HOST_ROUTE_NAMES.get(int(lib().pfb_last_host_route()), "none")


class Batch:
    """pfb_batch_create: a captured CUDA graph over many streams, replayed by launch()."""

    def __init__(self, entries):
        self._entries = entries  # keep tensors alive
        arr = _items(entries)
        h = ctypes.c_void_p()
        _check(lib().pfb_batch_create(arr, len(entries), ctypes.byref(h)), "pfb_batch_create")
        self.handle = h

    def launch(self, stream=None):
        _check(lib().pfb_batch_launch(self.handle, _stream_handle(stream)), "pfb_batch_launch")

    def close(self):
        if getattr(self, "handle", None):
            lib().pfb_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---- serving --------------------------------------------------------------

class Server:
    """pfb_server_*: continuous batching with resident per-stream filter state."""

    def __init__(self, hbm_budget_bytes: int, max_slots: int = 8, timeout_ms: int = 2000,
                 queue_when_busy: bool = True, device: int = -1):
        d = pfb_server_desc(hbm_budget_bytes, max_slots, timeout_ms, 1 if queue_when_busy else 0, device)
        h = ctypes.c_void_p()
        _check(lib().pfb_server_create(ctypes.byref(d), ctypes.byref(h)), "pfb_server_create")
        self.handle = h

    def open_stream(self, plan: Plan) -> int:
        sid = ctypes.c_int64()
        _check(lib().pfb_stream_open(self.handle, plan.handle, ctypes.byref(sid)), "pfb_stream_open")
        return sid.value

    def close_stream(self, sid: int):
        _check(lib().pfb_stream_close(self.handle, sid), "pfb_stream_close")

    def next_spectra(self, sid: int, n_samples: int) -> int:
        return int(lib().pfb_stream_next_spectra(self.handle, sid, n_samples))

    def submit(self, sid: int, chunk, n_samples: int, out) -> int:
        t = ctypes.c_int64()
        out_ptr = ctypes.c_void_p(out.data_ptr()) if out is not None and out.numel() else None
        cap = out.shape[0] if out is not None else 0
        _check(lib().pfb_submit(self.handle, sid, ctypes.c_void_p(chunk.data_ptr()), n_samples, out_ptr, cap,
                                ctypes.byref(t)), "pfb_submit")
        return t.value

    def submit_chunks(self, sid: int, chunks, n_chunks: int, samples_per_chunk: int, out) -> list:
        """pfb_submit_chunks: n_chunks consecutive chunks of one device buffer in
        one call; returns their tickets."""
        t = (ctypes.c_int64 * n_chunks)()
        out_ptr = ctypes.c_void_p(out.data_ptr()) if out is not None and out.numel() else None
        cap = out.shape[0] if out is not None else 0
        _check(lib().pfb_submit_chunks(self.handle, sid, ctypes.c_void_p(chunks.data_ptr()), n_chunks,
                                       samples_per_chunk, out_ptr, cap, t), "pfb_submit_chunks")
        return list(t)

    def ticket_times(self, ticket: int):
        """pfb_ticket_times: (submitted, finished) in seconds of the steady clock
        (time.monotonic() on Linux); finished is 0.0 while pending."""
        a, b = ctypes.c_double(), ctypes.c_double()
        _check(lib().pfb_ticket_times(self.handle, ticket, ctypes.byref(a), ctypes.byref(b)), "pfb_ticket_times")
        return a.value, b.value

    def poll(self, ticket: int) -> int:
        return int(lib().pfb_poll(self.handle, ticket))

    def wait(self, ticket: int, timeout_ms: int = 10000) -> int:
        return int(lib().pfb_wait(self.handle, ticket, timeout_ms))

    def export_state(self, sid: int) -> bytes:
        """pfb_stream_state_export: the stream's filter state as a byte blob
        (waits until the stream's submitted chunks have run)."""
        n = int(lib().pfb_stream_state_size(self.handle, sid))
        if n < 0:
            raise PFBError(PFB_ERR_INVALID, "unknown stream")
        buf = ctypes.create_string_buffer(n)
        _check(lib().pfb_stream_state_export(self.handle, sid, buf, n), "pfb_stream_state_export")
        return buf.raw

    def import_state(self, sid: int, blob: bytes):
        """pfb_stream_state_import: continue the exporting stream on stream `sid`."""
        buf = ctypes.create_string_buffer(bytes(blob), len(blob))
        _check(lib().pfb_stream_state_import(self.handle, sid, buf, len(blob)), "pfb_stream_state_import")

    def stats(self) -> dict:
        s = pfb_server_stats()
        _check(lib().pfb_server_get_stats(self.handle, ctypes.byref(s)), "pfb_server_get_stats")
        return {name: getattr(s, name) for name, _ in s._fields_}

    def close(self) -> int:
        if getattr(self, "handle", None):
            st = lib().pfb_server_destroy(self.handle)
            self.handle = None
            return st
        return PFB_OK

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
