"""Python binding of the C ABI in ``include/ask.h`` (argument marshalling only).

Every step of every method runs in ``libask.so``'s CUDA kernels; this module
converts Python arguments to the C structs, passes device pointers of torch
tensors and the current CUDA stream, and turns status codes into
exceptions.  If the library has not been built, :func:`lib` raises: there is
no fallback of any kind.

The dwell map is uint32 in the C ABI; torch tensors are allocated as int32
(same bits: dwell values never exceed 2^31 in practice) and numpy results are
returned as uint32 views.
"""
import ctypes
import os

from . import build as _build

ASK_MAX_LEVELS = 32

OK, EINVAL, ENOMEM, ECUDA, EOVERFLOW, ETIMEOUT, EUNSUPPORTED, ECAPACITY = range(8)
METHOD_EXHAUSTIVE, METHOD_ASK, METHOD_CDP2 = 0, 1, 2
FLAG_COUNT = 1
FLAG_TIMING = 2
FLAG_CDP2_FIRE_AND_FORGET = 4
FLAG_EXACT_BORDERS = 8
FLAG_LEAF_TILED = 16
FLAG_SBR = 32
FLAG_MBR = 64
FLAG_STAGED_COPY = 128
FLAG_SERIAL_FILL = 256
FLAG_INJECT_OVERFLOW = 512
FLAG_FLOAT_FLOAT = 1024
FLAG_PERSISTENT = 2048
FLAG_WAIT_TEST = 4096

METHODS = {"exhaustive": METHOD_EXHAUSTIVE, "ask": METHOD_ASK, "cdp2": METHOD_CDP2}


class Window(ctypes.Structure):
    _fields_ = [("re_min", ctypes.c_float), ("re_max", ctypes.c_float),
                ("im_min", ctypes.c_float), ("im_max", ctypes.c_float)]


class Window64(ctypes.Structure):
    _fields_ = [("re_min", ctypes.c_double), ("re_max", ctypes.c_double),
                ("im_min", ctypes.c_double), ("im_max", ctypes.c_double)]


class Params(ctypes.Structure):
    _fields_ = [("g", ctypes.c_uint32), ("r", ctypes.c_uint32), ("B", ctypes.c_uint32),
                ("block_x", ctypes.c_uint32), ("block_y", ctypes.c_uint32),
                ("flags", ctypes.c_uint32)]


class Stats(ctypes.Structure):
    _fields_ = [("levels", ctypes.c_uint32), ("pad_", ctypes.c_uint32),
                ("regions_per_level", ctypes.c_uint64 * ASK_MAX_LEVELS),
                ("fills_per_level", ctypes.c_uint64 * ASK_MAX_LEVELS),
                ("subdivisions_per_level", ctypes.c_uint64 * ASK_MAX_LEVELS),
                ("leaves", ctypes.c_uint64), ("fill_pixels", ctypes.c_uint64),
                ("leaf_pixels", ctypes.c_uint64), ("border_pixels", ctypes.c_uint64),
                ("iterations", ctypes.c_uint64),
                ("iterations_per_level", ctypes.c_uint64 * ASK_MAX_LEVELS),
                ("leaf_iterations", ctypes.c_uint64), ("ms_total", ctypes.c_float),
                ("ms_per_level", ctypes.c_float * ASK_MAX_LEVELS), ("ms_leaf", ctypes.c_float),
                ("ms_fill", ctypes.c_float), ("kernel_launches", ctypes.c_uint32),
                ("pad2_", ctypes.c_uint32), ("deferred_fill_pixels", ctypes.c_uint64)]

    def as_dict(self):
        L = self.levels
        return {
            "levels": L,
            "regions_per_level": list(self.regions_per_level[:L]),
            "fills_per_level": list(self.fills_per_level[:L]),
            "subdivisions_per_level": list(self.subdivisions_per_level[:L]),
            "leaves": self.leaves, "fill_pixels": self.fill_pixels,
            "leaf_pixels": self.leaf_pixels, "border_pixels": self.border_pixels,
            "iterations": self.iterations,
            "iterations_per_level": list(self.iterations_per_level[:L]),
            "leaf_iterations": self.leaf_iterations, "ms_total": self.ms_total,
            "ms_per_level": list(self.ms_per_level[:L]), "ms_leaf": self.ms_leaf,
            "ms_fill": self.ms_fill, "kernel_launches": self.kernel_launches,
            "deferred_fill_pixels": self.deferred_fill_pixels,
        }


class Timing(ctypes.Structure):
    _fields_ = [("renders", ctypes.c_uint32), ("dropped", ctypes.c_uint32),
                ("levels", ctypes.c_uint32), ("method", ctypes.c_uint32),
                ("ms_total", ctypes.c_float), ("ms_init", ctypes.c_float),
                ("ms_per_level", ctypes.c_float * ASK_MAX_LEVELS), ("ms_leaf", ctypes.c_float),
                ("ms_fill", ctypes.c_float)]

    def as_dict(self):
        L = self.levels
        return {"renders": self.renders, "dropped": self.dropped, "levels": L,
                "method": self.method, "ms_total": self.ms_total, "ms_init": self.ms_init,
                "ms_per_level": list(self.ms_per_level[:L]), "ms_leaf": self.ms_leaf,
                "ms_fill": self.ms_fill}


class Frame(ctypes.Structure):
    _fields_ = [("window", Window), ("n", ctypes.c_uint32), ("max_dwell", ctypes.c_uint32),
                ("g", ctypes.c_uint32), ("r", ctypes.c_uint32), ("B", ctypes.c_uint32),
                ("pad_", ctypes.c_uint32), ("d_dwell", ctypes.c_void_p)]


class AskError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(message)
        self.status = status


_lib = None

# Declared entry points of include/ask.h with their ctypes signatures.
_P = ctypes.POINTER
SIGNATURES = {
    "ask_ctx_create": (ctypes.c_int, [_P(ctypes.c_void_p), ctypes.c_int]),
    "ask_ctx_destroy": (None, [ctypes.c_void_p]),
    "ask_reserve": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_uint32, _P(Params)]),
    "ask_render": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, _P(Window), ctypes.c_uint32,
                                  ctypes.c_uint32, _P(Params), ctypes.c_void_p, ctypes.c_void_p,
                                  _P(Stats)]),
    "ask_render64": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, _P(Window64), ctypes.c_uint32,
                                    ctypes.c_uint32, _P(Params), ctypes.c_void_p, ctypes.c_void_p,
                                    _P(Stats)]),
    "ask_render_host": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, _P(Window), ctypes.c_uint32,
                                       ctypes.c_uint32, _P(Params), ctypes.c_void_p,
                                       ctypes.c_void_p, _P(Stats)]),
    "ask_check": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "ask_timing_read": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, _P(Timing)]),
    "ask_plan_levels": (ctypes.c_int, [ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32,
                                       ctypes.c_uint32, _P(ctypes.c_uint32), _P(ctypes.c_uint64),
                                       ctypes.c_uint32, _P(ctypes.c_uint32)]),
    "ask_render_noalloc": (ctypes.c_int, [_P(Window), ctypes.c_uint32, ctypes.c_uint32,
                                          _P(Params), ctypes.c_void_p, ctypes.c_void_p]),
    "ask_render_batch": (ctypes.c_int, [ctypes.c_void_p, _P(Frame), ctypes.c_uint32, ctypes.c_uint32,
                                        ctypes.c_void_p, _P(Stats)]),
    "ask_graph_create_batch": (ctypes.c_int, [ctypes.c_void_p, _P(Frame), ctypes.c_uint32,
                                              ctypes.c_uint32, ctypes.c_void_p,
                                              _P(ctypes.c_void_p)]),
    "ask_graph_launch": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "ask_graph_destroy": (None, [ctypes.c_void_p]),
    "ask_status_str": (ctypes.c_char_p, [ctypes.c_int]),
    "ask_last_error": (ctypes.c_char_p, [ctypes.c_void_p]),
    "ask_version": (ctypes.c_char_p, []),
}


def lib_path():
    return _build.LIB_PATH


def lib():
    """The loaded ``libask.so``.  Raises if it has not been built."""
    global _lib
    if _lib is None:
        path = lib_path()
        if not os.path.exists(path):
            raise RuntimeError("libask.so is not built (%s); run "
                               "paper_2206_02255_gb300.build.build() first" % path)
        L = ctypes.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def status_str(code):
    return lib().ask_status_str(code).decode()


def version():
    return lib().ask_version().decode()


def plan_levels(n, g, r, B):
    """Host-side level plan: (sides, max_regions) lists, one entry per level."""
    sides = (ctypes.c_uint32 * ASK_MAX_LEVELS)()
    regs = (ctypes.c_uint64 * ASK_MAX_LEVELS)()
    levels = ctypes.c_uint32()
    st = lib().ask_plan_levels(n, g, r, B, sides, regs, ASK_MAX_LEVELS, ctypes.byref(levels))
    if st != OK:
        raise AskError(st, "ask_plan_levels(%d, %d, %d, %d): %s" % (n, g, r, B, status_str(st)))
    L = levels.value
    return list(sides[:L]), list(regs[:L])


class Graph:
    """A captured batch render (``ask_graph``); ``launch`` replays it."""

    def __init__(self, handle, device):
        self._h = handle
        self.device = device

    def launch(self, stream=None):
        import torch
        s = stream if stream is not None else torch.cuda.current_stream(self.device)
        st = lib().ask_graph_launch(self._h, ctypes.c_void_p(s.cuda_stream))
        if st != OK:
            raise AskError(st, "ask_graph_launch: %s" % status_str(st))

    def close(self):
        if self._h:
            lib().ask_graph_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def render_noalloc(window, n, max_dwell, params, out, stream=None):
    """ASK render that allocates nothing on the device (``ask_render_noalloc``):
    for callers that may not call cudaMalloc.  ``out`` is a caller-owned
    contiguous CUDA tensor of n*n 4-byte elements; the scratch is the
    library's fixed device arrays (at most 2^20 regions per level), shared
    by every call, so calls must not overlap on the GPU.  Asynchronous on
    ``stream`` (default: torch's current stream on ``out``'s device)."""
    import torch
    if not out.is_cuda or out.numel() != n * n or out.element_size() != 4 or \
            not out.is_contiguous():
        raise ValueError("out must be a contiguous CUDA tensor of n*n 4-byte elements")
    s = stream if stream is not None else torch.cuda.current_stream(out.device)
    with torch.cuda.device(out.device):
        st = lib().ask_render_noalloc(ctypes.byref(_window(window)), n, max_dwell,
                                      ctypes.byref(params), ctypes.c_void_p(out.data_ptr()),
                                      ctypes.c_void_p(s.cuda_stream))
    if st != OK:
        raise AskError(st, "ask_render_noalloc: %s" % status_str(st))
    return out


def make_params(g=16, r=2, B=32, block=(16, 16), flags=0):
    return Params(g, r, B, block[0], block[1], flags)


# Zoom (relative to the 2 x 2 window of the paper's configuration) past
# which frames are rendered in double precision: at zoom 1e4 a window is
# 2e-4 wide, and a map of a few thousand pixels has a spacing near one float
# ulp of c, so neighbouring pixels start to share c in single precision.
FP64_ZOOM = 1e4


def needs_fp64(window):
    """True for a window (a 4-sequence, Window or Window64) zoomed past
    FP64_ZOOM, i.e. narrower than 2 / FP64_ZOOM."""
    if isinstance(window, (Window, Window64)):
        window = (window.re_min, window.re_max, window.im_min, window.im_max)
    re0, re1, im0, im1 = (float(v) for v in window)
    return max(re1 - re0, im1 - im0) < 2.0 / FP64_ZOOM


def _method(m):
    return METHODS[m] if isinstance(m, str) else int(m)


def _window(w):
    return w if isinstance(w, Window) else Window(*[float(v) for v in w])


def _window64(w):
    if isinstance(w, Window64):
        return w
    if isinstance(w, Window):
        return Window64(w.re_min, w.re_max, w.im_min, w.im_max)
    return Window64(*[float(v) for v in w])


class Context:
    """An ``ask_ctx`` on one CUDA device; owns the library's scratch memory."""

    def __init__(self, device=0):
        self._h = ctypes.c_void_p()
        st = lib().ask_ctx_create(ctypes.byref(self._h), device)
        if st != OK:
            raise AskError(st, "ask_ctx_create(device=%d): %s" % (device, status_str(st)))
        self.device = device

    def close(self):
        if self._h:
            lib().ask_ctx_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @property
    def handle(self):
        return self._h

    def _raise(self, st, what):
        msg = lib().ask_last_error(self._h)
        raise AskError(st, "%s: %s (%s)" % (what, status_str(st), (msg or b"").decode()))

    def reserve(self, method, n, params=None):
        st = lib().ask_reserve(self._h, _method(method), n,
                               ctypes.byref(params) if params is not None else None)
        if st != OK:
            self._raise(st, "ask_reserve")

    def render(self, method, window, n, max_dwell, params=None, out=None, stream=None,
               stats=False):
        """Render into ``out`` (a CUDA int32 tensor of n*n elements, allocated
        here if None) on ``stream`` (default: torch's current stream).
        Returns ``out`` or ``(out, stats dict)``; with ``stats`` the call
        synchronises."""
        import torch
        if out is None:
            out = torch.empty((n, n), dtype=torch.int32, device="cuda:%d" % self.device)
        if not out.is_cuda or out.numel() != n * n or not out.is_contiguous():
            raise ValueError("out must be a contiguous CUDA tensor of n*n elements")
        if out.element_size() != 4:
            raise ValueError("out must have 4-byte elements")
        s = stream if stream is not None else torch.cuda.current_stream(out.device)
        st_obj = Stats() if stats else None
        st = lib().ask_render(self._h, _method(method), ctypes.byref(_window(window)), n,
                              max_dwell, ctypes.byref(params) if params is not None else None,
                              ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(s.cuda_stream),
                              ctypes.byref(st_obj) if st_obj is not None else None)
        if st != OK:
            self._raise(st, "ask_render")
        return (out, st_obj.as_dict()) if stats else out

    def render64(self, method, window, n, max_dwell, params=None, out=None, stream=None,
                 stats=False):
        """Double-precision render (deep zooms) of ``window`` given in double:
        "exhaustive" or "ask"; otherwise as :meth:`render`."""
        import torch
        if out is None:
            out = torch.empty((n, n), dtype=torch.int32, device="cuda:%d" % self.device)
        if not out.is_cuda or out.numel() != n * n or not out.is_contiguous():
            raise ValueError("out must be a contiguous CUDA tensor of n*n elements")
        if out.element_size() != 4:
            raise ValueError("out must have 4-byte elements")
        s = stream if stream is not None else torch.cuda.current_stream(out.device)
        st_obj = Stats() if stats else None
        st = lib().ask_render64(self._h, _method(method), ctypes.byref(_window64(window)), n,
                                max_dwell, ctypes.byref(params) if params is not None else None,
                                ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(s.cuda_stream),
                                ctypes.byref(st_obj) if st_obj is not None else None)
        if st != OK:
            self._raise(st, "ask_render64")
        return (out, st_obj.as_dict()) if stats else out

    def render_host(self, method, window, n, max_dwell, params=None, out=None, stream=None,
                    stats=False):
        """Render into host memory ``out`` (numpy uint32 (n, n) or a CPU
        tensor; allocated if None).  Synchronous."""
        import numpy as np
        if out is None:
            out = np.empty((n, n), dtype=np.uint32)
        if isinstance(out, np.ndarray):
            if out.size != n * n or out.itemsize != 4 or not out.flags["C_CONTIGUOUS"]:
                raise ValueError("out must be a contiguous 4-byte array of n*n elements")
            ptr = out.ctypes.data
        else:
            if out.is_cuda or out.numel() != n * n or out.element_size() != 4 or \
                    not out.is_contiguous():
                raise ValueError("out must be a contiguous CPU tensor of n*n 4-byte elements")
            ptr = out.data_ptr()
        sptr = 0
        if stream is not None:
            sptr = stream.cuda_stream
        st_obj = Stats() if stats else None
        st = lib().ask_render_host(self._h, _method(method), ctypes.byref(_window(window)), n,
                                   max_dwell, ctypes.byref(params) if params is not None else None,
                                   ctypes.c_void_p(ptr), ctypes.c_void_p(sptr),
                                   ctypes.byref(st_obj) if st_obj is not None else None)
        if st != OK:
            self._raise(st, "ask_render_host")
        return (out, st_obj.as_dict()) if stats else out

    def timing_read(self, stream=None):
        """Per-kernel device times summed over the ASK_FLAG_TIMING renders
        since the previous read (synchronises ``stream``)."""
        import torch
        s = stream if stream is not None else torch.cuda.current_stream(self.device)
        t = Timing()
        st = lib().ask_timing_read(self._h, ctypes.c_void_p(s.cuda_stream), ctypes.byref(t))
        if st != OK:
            self._raise(st, "ask_timing_read")
        return t.as_dict()

    def _frames(self, frames):
        """frames: sequence of dicts with window, n, max_dwell, g, r, B and
        `out` (a contiguous CUDA tensor of n*n 4-byte elements)."""
        arr = (Frame * len(frames))()
        for k, f in enumerate(frames):
            out = f["out"]
            n = int(f["n"])
            if not out.is_cuda or out.numel() != n * n or out.element_size() != 4 or \
                    not out.is_contiguous():
                raise ValueError("frame %d: out must be a contiguous CUDA tensor of n*n "
                                 "4-byte elements" % k)
            arr[k] = Frame(_window(f["window"]), n, int(f["max_dwell"]), int(f["g"]),
                           int(f["r"]), int(f["B"]), 0, out.data_ptr())
        return arr

    def render_batch(self, frames, flags=0, stream=None, stats=False):
        """Render a batch of frames (see ``_frames``) with one launch chain.
        Frames zoomed past FP64_ZOOM (``needs_fp64``), whose windows a float
        cannot hold, are rendered after it on the same stream, one
        ``ask_render64`` (binary64 ASK) each.  Returns None, or, when
        ``stats`` (synchronises), the stats dict summed over the
        single-precision frames, with ``fp64_frames`` the number routed.
        Frame numbers in the library's error messages count the
        single-precision frames only."""
        import torch
        s = stream if stream is not None else torch.cuda.current_stream(self.device)
        shallow = [f for f in frames if not needs_fp64(f["window"])]
        deep = [f for f in frames if needs_fp64(f["window"])]
        out = None
        if shallow or not deep:  # an empty batch is the library's argument error
            arr = self._frames(shallow)
            st_obj = Stats() if stats else None
            st = lib().ask_render_batch(self._h, arr, len(shallow), flags,
                                        ctypes.c_void_p(s.cuda_stream),
                                        ctypes.byref(st_obj) if st_obj is not None else None)
            if st != OK:
                self._raise(st, "ask_render_batch")
            out = st_obj.as_dict() if stats else None
        for f in deep:
            self.render64("ask", f["window"], int(f["n"]), int(f["max_dwell"]),
                          make_params(int(f["g"]), int(f["r"]), int(f["B"])), out=f["out"],
                          stream=s)
        if stats:
            if out is None:
                s.synchronize()
                out = Stats().as_dict()
            out["fp64_frames"] = len(deep)
        return out

    def graph_batch(self, frames, flags=0, stream=None):
        """Capture a batch render as a CUDA graph (see :class:`Graph`).
        Single-precision frames only: a frame zoomed past FP64_ZOOM raises
        ValueError."""
        import torch
        if any(needs_fp64(f["window"]) for f in frames):
            raise ValueError("graph_batch: frames zoomed past FP64_ZOOM need render64")
        arr = self._frames(frames)
        s = stream if stream is not None else torch.cuda.current_stream(self.device)
        h = ctypes.c_void_p()
        st = lib().ask_graph_create_batch(self._h, arr, len(frames), flags,
                                          ctypes.c_void_p(s.cuda_stream), ctypes.byref(h))
        if st != OK:
            self._raise(st, "ask_graph_create_batch")
        return Graph(h, self.device)

    def check(self, stream=None):
        sptr = stream.cuda_stream if stream is not None else 0
        st = lib().ask_check(self._h, ctypes.c_void_p(sptr))
        if st != OK:
            self._raise(st, "ask_check")
