"""Workload definitions and seeded input generators.

Shared by the GPU path's tests and benchmark and by the CPU reference's
checks.  It holds no part of the method's arithmetic: only windows of the
complex plane, sizes, dwell caps, subdivision parameters and seeded samples
of them.

The paper measures on the Mandelbrot set over a fixed window with dwell 512
for n from 1024 up to 65536 (Sec. 6.1) and sweeps g, r, B and the CUDA block
shape (Sec. 6.2, Table 2, Fig. 6).  The configurations below follow that
recipe at three sizes.
"""
import itertools
import math
import os
import random

# Window corners as (re_min, re_max, im_min, im_max).  The paper's
# "[-1.5, -1] x [0.5, 1]" is read as the corners (-1.5, -1) and (0.5, 1).
WINDOW_PAPER = (-1.5, 0.5, -1.0, 1.0)
WINDOW_WIDE = (-2.0, 1.0, -1.5, 1.5)

# n = 1024, dwell 512: the small case the CPU reference renders in seconds.
C0 = dict(name="mandelbrot_n1024_d512", window=WINDOW_PAPER, n=1024, max_dwell=512,
          g=16, r=2, B=32)
# n = 16384, dwell 2048: the measured configuration, with its g, r, B sweep.
C1 = dict(name="mandelbrot_n16384_d2048", window=WINDOW_PAPER, n=16384, max_dwell=2048)
C1_G = (2, 4, 8, 16, 32)
C1_R = (2, 4, 8)
C1_B = (16, 32, 64, 128, 256)
# n = 65536, dwell 4096 (a 17.2 GB uint32 map).
C2 = dict(name="mandelbrot_n65536_d4096", window=WINDOW_WIDE, n=65536, max_dwell=4096)

# CUDA block shapes explored by the paper (Sec. 6.2, Table 2).
BLOCK_SHAPES = ((8, 8), (16, 16), (32, 32), (64, 4), (64, 8))


def c1_sweep():
    """The 75 (g, r, B) points of the n = 16384 sweep."""
    return list(itertools.product(C1_G, C1_R, C1_B))


def sample_initial_regions(g, k, seed):
    """k distinct initial-region indices (gx, gy) of a g x g grid, seeded."""
    rng = random.Random(seed)
    cells = [(gx, gy) for gy in range(g) for gx in range(g)]
    return rng.sample(cells, min(k, len(cells)))


def sample_pixels(n, k, seed):
    """k seeded pixel coordinates (px, py) in [0, n)^2."""
    rng = random.Random(seed)
    return [(rng.randrange(n), rng.randrange(n)) for _ in range(k)]


def random_windows(k, seed, span=(1e-3, 3.0)):
    """k seeded windows inside [-2.2, 1.2] x [-1.6, 1.6] with sides in span."""
    rng = random.Random(seed)
    out = []
    for _ in range(k):
        wr = rng.uniform(*span)
        wi = rng.uniform(*span)
        re0 = rng.uniform(-2.2, 1.2 - wr) if wr < 3.4 else -2.2
        im0 = rng.uniform(-1.6, 1.6 - wi) if wi < 3.2 else -1.6
        out.append((re0, re0 + wr, im0, im0 + wi))
    return out


# ---------------------------------------------------------------------------
# Batched and served workloads: frames zoomed on points of the set's boundary.
# The candidate centres are boundary pixels of the n = 1024, dwell 512 map
# (a pixel below the cap next to one at the cap), shipped with the package as
# data/boundary_centers.tsv (written once from the CPU reference by
# tests/golden/make_boundary_centers.py).
# ---------------------------------------------------------------------------
BOUNDARY_CENTERS = os.path.join(os.path.dirname(os.path.abspath(__file__)), "data",
                                "boundary_centers.tsv")


def boundary_centers():
    """[(cr, ci)] of the stored boundary pixels."""
    out = []
    with open(BOUNDARY_CENTERS) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            cols = line.split("\t")
            out.append((float(cols[2]), float(cols[3])))
    return out


def _log_uniform(rng, lo, hi):
    return math.exp(rng.uniform(math.log(lo), math.log(hi)))


def _zoom_window(center, zoom):
    # zoom 1 is the 2 x 2 window of the n = 1024 configuration
    hw = 1.0 / zoom
    cr, ci = center
    return (cr - hw, cr + hw, ci - hw, ci + hw)


def batch_frames(count=256, seed=0, sides=(512, 8192), zooms=(1.0, 1e4), dwells=(256, 8192)):
    """Frames of the batched workload: side uniform in `sides`, centre drawn
    from the boundary centres, zoom log-uniform in `zooms`, dwell cap a
    log-uniform integer in `dwells`.  Returns dicts with window, n,
    max_dwell, zoom."""
    rng = random.Random(seed)
    centers = boundary_centers()
    out = []
    for _ in range(count):
        n = rng.randint(*sides)
        c = rng.choice(centers)
        zoom = _log_uniform(rng, *zooms)
        md = int(round(_log_uniform(rng, *dwells)))
        out.append(dict(window=_zoom_window(c, zoom), n=n, max_dwell=md, zoom=zoom))
    return out


def serving_requests(count=2000, seed=7, rate=200.0, sides=(256, 4096), zooms=(1.0, 1e4),
                     dwells=(512, 4096)):
    """Requests of the served workload: Poisson arrivals at `rate` per second
    (seconds from 0 in `t`), side uniform in `sides`, centre and zoom as in
    batch_frames, dwell cap uniform in `dwells`."""
    rng = random.Random(seed)
    centers = boundary_centers()
    t = 0.0
    out = []
    for k in range(count):
        t += rng.expovariate(rate)
        n = rng.randint(*sides)
        c = rng.choice(centers)
        zoom = _log_uniform(rng, *zooms)
        md = rng.randint(*dwells)
        out.append(dict(id=k, t=t, window=_zoom_window(c, zoom), n=n, max_dwell=md, zoom=zoom))
    return out


# ---------------------------------------------------------------------------
# Deep zooms, rendered in double precision: square windows of a power-of-two
# width around points near the set's boundary, far past the zoom of 1e4 over
# the 2 x 2 window at which single precision stops separating the pixels of
# a large map.  (centre re, centre im, width, dwell cap)
# ---------------------------------------------------------------------------
DEEP_SPOTS = (
    ("spiral_2^-28", -0.10109636384562, 0.95628651080914, 2.0 ** -28, 1024),
    ("seahorse_2^-30", -0.743643887037151, 0.13182590420533, 2.0 ** -30, 4096),
    ("antenna_2^-20", -1.25066, 0.02012, 2.0 ** -20, 2048),
)


def deep_window(name):
    """(window, max_dwell) of a DEEP_SPOTS entry; the window's lower-left
    corner is the listed point, so its sides are exact doubles."""
    for nm, re0, im0, w, md in DEEP_SPOTS:
        if nm == name:
            return (re0, re0 + w, im0, im0 + w), md
    raise KeyError(name)


def deep_frames(count=16, seed=3, sides=(256, 2048), zooms=(1e5, 1e10), dwells=(512, 4096)):
    """Seeded deep-zoom frames for the double-precision path: centre drawn
    from the boundary centres, zoom log-uniform in `zooms` (relative to the
    2 x 2 window), side uniform in `sides`, dwell cap log-uniform."""
    rng = random.Random(seed)
    centers = boundary_centers()
    out = []
    for _ in range(count):
        n = rng.randint(*sides)
        c = rng.choice(centers)
        zoom = _log_uniform(rng, *zooms)
        md = int(round(_log_uniform(rng, *dwells)))
        out.append(dict(window=_zoom_window(c, zoom), n=n, max_dwell=md, zoom=zoom))
    return out
