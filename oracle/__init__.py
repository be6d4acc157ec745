"""ctypes wrapper of the CPU reference for the Mandelbrot dwell map.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, the package's ``smoke()`` check
and the benchmark's CPU-baseline leg import this module.  The GPU library and
its Python binding never import it, and it imports nothing from them.

The arithmetic lives in ``oracle.c`` (plain C, single precision with
explicit ``fmaf``, and the same sequence in double with ``fma`` for deep
zooms); this module only marshals numpy buffers.  Functions:

* :func:`dwell` -- dwell of one point (Sec. 6 of the paper);
* :func:`render_exhaustive` -- the per-pixel map (Sec. 4.1, Eq. 1-2);
* :func:`render_ms` -- serial recursive Mariani-Silver (Sec. 4.2.1, Sec. 6),
  with per-level statistics and an optional log of every region visited;
* :func:`render_ms_region` -- one initial region of the g x g grid, for
  sampled parity checks on maps too large to render on the CPU (``fp64``:
  double window, binary64 or float-float);
* :func:`dwell64`, :func:`pixel_to_c64`, :func:`render_exhaustive64`,
  :func:`render_ms64` -- the same in double precision (deep zooms), the
  window given in double; with the flag ``FLOAT_FLOAT`` the maps iterate in
  float-float arithmetic instead (:func:`dwell_ff`).

:class:`Oracle` wraps one build of the library; the module-level functions
use the default build.  Tests also load deliberately broken builds through
:class:`Oracle` to show that the pins reject them.
"""
import ctypes
import os

import numpy as np

from . import build as _build

ESCAPE_LE = 1
NO_FILL = 2
FLOAT_FLOAT = 4
REGION_FILL, REGION_SUBDIVIDE, REGION_LEAF = 0, 1, 2
MAX_LEVELS = 32


class Window(ctypes.Structure):
    _fields_ = [("re_min", ctypes.c_float), ("re_max", ctypes.c_float),
                ("im_min", ctypes.c_float), ("im_max", ctypes.c_float)]


class Window64(ctypes.Structure):
    _fields_ = [("re_min", ctypes.c_double), ("re_max", ctypes.c_double),
                ("im_min", ctypes.c_double), ("im_max", ctypes.c_double)]


class MSStats(ctypes.Structure):
    _fields_ = [("levels", ctypes.c_uint32), ("pad_", ctypes.c_uint32),
                ("regions_per_level", ctypes.c_uint64 * MAX_LEVELS),
                ("fills_per_level", ctypes.c_uint64 * MAX_LEVELS),
                ("subdivisions_per_level", ctypes.c_uint64 * MAX_LEVELS),
                ("leaves", ctypes.c_uint64), ("fill_pixels", ctypes.c_uint64),
                ("leaf_pixels", ctypes.c_uint64), ("border_pixels", ctypes.c_uint64),
                ("iterations", ctypes.c_uint64)]

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
        }


REGION_DTYPE = np.dtype([(k, np.uint32) for k in
                         ("level", "x0", "y0", "w", "h", "s", "kind", "dwell")])


def default_threads():
    if hasattr(os, "sched_getaffinity"):
        return max(1, len(os.sched_getaffinity(0)))
    return max(1, os.cpu_count() or 1)


def _win(window):
    re_min, re_max, im_min, im_max = window
    return Window(re_min, re_max, im_min, im_max)


def _win64(window):
    re_min, re_max, im_min, im_max = window
    return Window64(re_min, re_max, im_min, im_max)


class Oracle:
    """One loaded build of the reference library."""

    def __init__(self, path):
        L = ctypes.CDLL(path)
        u32, u64, f32 = ctypes.c_uint32, ctypes.c_uint64, ctypes.c_float
        P = ctypes.POINTER
        L.oracle_dwell.restype = u32
        L.oracle_dwell.argtypes = [f32, f32, u32, u32]
        L.oracle_pixel_to_c.restype = None
        L.oracle_pixel_to_c.argtypes = [P(Window), u32, u32, u32, P(f32), P(f32)]
        L.oracle_render_exhaustive.restype = ctypes.c_int
        L.oracle_render_exhaustive.argtypes = [P(Window), u32, u32, u32, ctypes.c_void_p,
                                               ctypes.c_int, P(u64)]
        L.oracle_render_ms.restype = ctypes.c_int
        L.oracle_render_ms.argtypes = [P(Window), u32, u32, u32, u32, u32, u32,
                                       ctypes.c_void_p, ctypes.c_int, P(MSStats),
                                       ctypes.c_void_p, u64, P(u64)]
        L.oracle_initial_region.restype = ctypes.c_int
        L.oracle_initial_region.argtypes = [u32, u32, u32, u32, P(u32), P(u32), P(u32), P(u32)]
        f64 = ctypes.c_double
        L.oracle_dwell64.restype = u32
        L.oracle_dwell64.argtypes = [f64, f64, u32, u32]
        L.oracle_dwell_ff.restype = u32
        L.oracle_dwell_ff.argtypes = [f64, f64, u32, u32]
        L.oracle_pixel_to_c64.restype = None
        L.oracle_pixel_to_c64.argtypes = [P(Window64), u32, u32, u32, P(f64), P(f64)]
        L.oracle_render_exhaustive64.restype = ctypes.c_int
        L.oracle_render_exhaustive64.argtypes = [P(Window64), u32, u32, u32, ctypes.c_void_p,
                                                 ctypes.c_int, P(u64)]
        L.oracle_render_ms64.restype = ctypes.c_int
        L.oracle_render_ms64.argtypes = [P(Window64), u32, u32, u32, u32, u32, u32,
                                         ctypes.c_void_p, ctypes.c_int, P(MSStats),
                                         ctypes.c_void_p, u64, P(u64)]
        L.oracle_render_ms_region.restype = ctypes.c_int
        L.oracle_render_ms_region.argtypes = [P(Window), u32, u32, u32, u32, u32, u32,
                                              u32, u32, ctypes.c_void_p, ctypes.c_size_t,
                                              P(MSStats)]
        L.oracle_render_ms_region64.argtypes = [P(Window64), u32, u32, u32, u32, u32, u32,
                                              u32, u32, ctypes.c_void_p, ctypes.c_size_t,
                                              P(MSStats)]
        L.oracle_render_ms_region64.restype = ctypes.c_int
        self.lib = L
        self.path = path

    def dwell(self, cr, ci, max_dwell, flags=0):
        """Dwell of the point c = cr + i*ci (both rounded to float32)."""
        return int(self.lib.oracle_dwell(cr, ci, max_dwell, flags))

    def pixel_to_c(self, window, n, px, py):
        """The float32 point sampled by pixel (px, py): returns (cr, ci)."""
        cr, ci = ctypes.c_float(), ctypes.c_float()
        w = _win(window)
        self.lib.oracle_pixel_to_c(ctypes.byref(w), n, px, py, ctypes.byref(cr),
                                   ctypes.byref(ci))
        return cr.value, ci.value

    def dwell64(self, cr, ci, max_dwell, flags=0):
        """Dwell of the point c = cr + i*ci in double precision."""
        return int(self.lib.oracle_dwell64(cr, ci, max_dwell, flags))

    def dwell_ff(self, cr, ci, max_dwell, flags=0):
        """Dwell of c (given in double) in float-float arithmetic."""
        return int(self.lib.oracle_dwell_ff(cr, ci, max_dwell, flags))

    def pixel_to_c64(self, window, n, px, py):
        """The double-precision point sampled by pixel (px, py)."""
        cr, ci = ctypes.c_double(), ctypes.c_double()
        w = _win64(window)
        self.lib.oracle_pixel_to_c64(ctypes.byref(w), n, px, py, ctypes.byref(cr),
                                     ctypes.byref(ci))
        return cr.value, ci.value

    def render_exhaustive(self, window, n, max_dwell, flags=0, threads=None,
                          return_iterations=False, fp64=False):
        """n x n uint32 map, out[py, px] = dwell at pixel (px, py).  With
        fp64 the window and the arithmetic are double precision."""
        out = np.empty((n, n), dtype=np.uint32)
        it = ctypes.c_uint64()
        w = _win64(window) if fp64 else _win(window)
        fn = self.lib.oracle_render_exhaustive64 if fp64 else self.lib.oracle_render_exhaustive
        rc = fn(ctypes.byref(w), n, max_dwell, flags, out.ctypes.data,
                threads or default_threads(), ctypes.byref(it))
        if rc != 0:
            raise ValueError("oracle_render_exhaustive: invalid arguments (rc=%d)" % rc)
        return (out, int(it.value)) if return_iterations else out

    def render_ms(self, window, n, max_dwell, g, r, B, flags=0, threads=None, log=False,
                  fp64=False):
        """Mariani-Silver map.  Returns (map, stats dict[, region log array]).
        With fp64 the window and the arithmetic are double precision."""
        out = np.empty((n, n), dtype=np.uint32)
        st = MSStats()
        w = _win64(window) if fp64 else _win(window)
        fn = self.lib.oracle_render_ms64 if fp64 else self.lib.oracle_render_ms
        if log:
            cap = 1 << 16
            while True:
                buf = np.zeros(cap, dtype=REGION_DTYPE)
                ln = ctypes.c_uint64()
                rc = fn(ctypes.byref(w), n, max_dwell, g, r, B, flags, out.ctypes.data, 1,
                        ctypes.byref(st), buf.ctypes.data, cap, ctypes.byref(ln))
                if rc != 0:
                    raise ValueError("oracle_render_ms: invalid arguments (rc=%d)" % rc)
                if ln.value <= cap:
                    return out, st.as_dict(), buf[:ln.value].copy()
                cap = int(ln.value)
        rc = fn(ctypes.byref(w), n, max_dwell, g, r, B, flags, out.ctypes.data,
                threads or default_threads(), ctypes.byref(st), None, 0, None)
        if rc != 0:
            raise ValueError("oracle_render_ms: invalid arguments (rc=%d)" % rc)
        return out, st.as_dict()

    def initial_region(self, n, g, gx, gy):
        """(x0, y0, w, h) of initial region (gx, gy), or None if it is empty."""
        x0, y0, w, h = (ctypes.c_uint32() for _ in range(4))
        ok = self.lib.oracle_initial_region(n, g, gx, gy, ctypes.byref(x0), ctypes.byref(y0),
                                            ctypes.byref(w), ctypes.byref(h))
        return (x0.value, y0.value, w.value, h.value) if ok else None

    def render_ms_region(self, window, n, max_dwell, g, r, B, gx, gy, flags=0, fp64=False):
        """Mariani-Silver tile of initial region (gx, gy).

        Returns ((x0, y0, w, h), tile[h, w], stats dict), or None for an
        empty region.
        """
        reg = self.initial_region(n, g, gx, gy)
        if reg is None:
            return None
        x0, y0, w_, h_ = reg
        tile = np.empty((h_, w_), dtype=np.uint32)
        st = MSStats()
        w = _win64(window) if fp64 else _win(window)
        fn = self.lib.oracle_render_ms_region64 if fp64 else self.lib.oracle_render_ms_region
        rc = fn(ctypes.byref(w), n, max_dwell, g, r, B, flags, gx, gy, tile.ctypes.data, w_,
                ctypes.byref(st))
        if rc != 0:
            raise ValueError("oracle_render_ms_region failed (rc=%d)" % rc)
        return reg, tile, st.as_dict()


_default = None


def default():
    """The oracle built from ``oracle.c`` (built on first use)."""
    global _default
    if _default is None:
        _default = Oracle(_build.build())
    return _default


def dwell(*a, **k):
    return default().dwell(*a, **k)


def pixel_to_c(*a, **k):
    return default().pixel_to_c(*a, **k)


def render_exhaustive(*a, **k):
    return default().render_exhaustive(*a, **k)


def render_ms(*a, **k):
    return default().render_ms(*a, **k)


def initial_region(*a, **k):
    return default().initial_region(*a, **k)


def render_ms_region(*a, **k):
    return default().render_ms_region(*a, **k)


def dwell64(*a, **k):
    return default().dwell64(*a, **k)


def dwell_ff(*a, **k):
    return default().dwell_ff(*a, **k)


def pixel_to_c64(*a, **k):
    return default().pixel_to_c64(*a, **k)


def render_exhaustive64(window, n, max_dwell, **k):
    return default().render_exhaustive(window, n, max_dwell, fp64=True, **k)


def render_ms64(window, n, max_dwell, g, r, B, **k):
    return default().render_ms(window, n, max_dwell, g, r, B, fp64=True, **k)
