"""Pins of the CPU reference to facts fixed outside it.

Each ``pin_*`` function takes an ``oracle.Oracle`` and raises
``AssertionError`` when the reference disagrees with:

* values hand-computed from the definition of the dwell (Sec. 6 of the paper:
  z <- z^2 + c from z = 0, counted while |z| < 2), exact in float32;
* an exact-rational brute force of tiny maps (``f32exact``), which shares no
  code with the C reference and needs no libm or FMA hardware;
* mathematics: conjugate symmetry of the set, its known area (about 1.5066),
  the exact pixel -> c mapping where the spacing is a power of two;
* structure that the subdivision rule of Sec. 4.2.1 fixes by hand on tiny
  grids (region counts per level with fills disabled), and invariants of the
  Mariani-Silver recursion on larger ones (tiling, uniform perimeters of
  filled regions, stopping side B, leaf pixels equal the exhaustive map).

``tests/test_oracle_pins.py`` runs them against the reference;
``tests/test_oracle_mutants.py`` runs them against deliberately broken
builds and expects each build to fail at least one.
"""
import os
import random

import numpy as np

import f32exact

C0_WINDOW = (-1.5, 0.5, -1.0, 1.0)
ESCAPE_LE = 1
NO_FILL = 2
FILL, SUBDIVIDE, LEAF = 0, 1, 2


# --------------------------------------------------------------------------
# dwell of single points
# --------------------------------------------------------------------------
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def closed_forms():
    """Rows of ``golden/closed_forms.tsv``: (cr, ci, max_dwell, flags, dwell)."""
    rows = []
    with open(os.path.join(GOLDEN, "closed_forms.tsv")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            cr, ci, M, flags, d = line.split("\t")[:5]
            rows.append((float(cr), float(ci), int(M), int(flags), int(d)))
    return rows


def pin_closed_forms(orc):
    """Orbits followed by hand in exact float32 arithmetic, including the
    strict (|z| < 2) and membership (|z| <= 2) readings of the escape test."""
    rows = closed_forms()
    assert len(rows) >= 20
    for cr, ci, M, flags, d in rows:
        assert orc.dwell(cr, ci, M, flags) == d, (cr, ci, M, flags, d)


def pin_exact_points(orc):
    """Random points against the exact-rational brute force."""
    rng = random.Random(20220605)
    for _ in range(150):
        cr = f32exact.to_float(f32exact.f32(rng.uniform(-2.2, 1.0)))
        ci = f32exact.to_float(f32exact.f32(rng.uniform(-1.4, 1.4)))
        assert orc.dwell(cr, ci, 48) == f32exact.dwell(cr, ci, 48), (cr, ci)


# --------------------------------------------------------------------------
# maps
# --------------------------------------------------------------------------
def pin_exact_tiny_maps(orc):
    """Tiny exhaustive maps, pixel for pixel, against the brute force; the
    windows are asymmetric so a transposed map or swapped axis fails."""
    cases = [((-2.0, 0.5, -1.1, 1.3), 1, 40), ((-2.0, 0.5, -1.1, 1.3), 2, 40),
             ((-1.9, 0.6, -0.3, 1.2), 5, 30), ((-0.8, -0.6, 0.05, 0.30), 8, 60),
             ((-2.0, 0.47, -1.12, 1.12), 7, 25)]
    for win, n, M in cases:
        got = orc.render_exhaustive(win, n, M, threads=2)
        want = np.array(f32exact.exhaustive(win, n, M), dtype=np.uint32)
        assert np.array_equal(got, want), (win, n, M)
    # pixel -> c against the brute force
    rng = random.Random(7)
    for _ in range(60):
        a, b = sorted(rng.uniform(-2.5, 2.5) for _ in range(2))
        c, d = sorted(rng.uniform(-2.5, 2.5) for _ in range(2))
        if b - a < 1e-3 or d - c < 1e-3:
            continue
        win = tuple(f32exact.to_float(f32exact.f32(v)) for v in (a, b, c, d))
        n = rng.randint(1, 70000)
        px, py = rng.randrange(n), rng.randrange(n)
        want = tuple(f32exact.to_float(v) for v in f32exact.pixel_c(win, n, px, py))
        assert orc.pixel_to_c(win, n, px, py) == want, (win, n, px, py)


def pin_c0_pixels(orc):
    """With the window [-1.5, 0.5] x [-1, 1] at n = 1024 the spacing is 2^-9,
    so pixel (px, py) samples exactly c = -1.5 + px/512 + i(-1 + py/512)."""
    for px, py in [(0, 0), (768, 512), (256, 512), (896, 512), (1023, 1023), (5, 999)]:
        assert orc.pixel_to_c(C0_WINDOW, 1024, px, py) == (-1.5 + px / 512, -1.0 + py / 512)
    m = orc.render_exhaustive(C0_WINDOW, 1024, 512, threads=4)
    assert m[512, 768] == 512   # c = 0
    assert m[512, 256] == 512   # c = -1
    assert m[512, 896] == 512   # c = 1/4
    assert m[512, 0] == 512     # c = -3/2
    # c = -1.5 - i: |z_1|^2 = 3.25, z_2 = -0.25 + 2i with |z_2|^2 = 4.0625
    assert orc.dwell(-1.5, -1.0, 512) == 2
    assert m[0, 0] == 2
    return m


def pin_symmetry_and_area(orc):
    """Conjugate symmetry (rows py and n - py of a window symmetric in Im)
    and the area of the set, about 1.5066 (finite dwell and corner sampling
    overestimate it a little)."""
    n = 1024
    m = orc.render_exhaustive(C0_WINDOW, n, 512, threads=4)
    assert np.array_equal(m[1:], m[1:][::-1])
    area = float((m == 512).mean()) * 4.0
    assert 1.49 < area < 1.54, area
    # an asymmetric spot check: c = 0.3 escapes (right of the cusp at 1/4)
    # while c = 0.3i stays bounded
    assert orc.dwell(0.3, 0.0, 512) < 512
    assert orc.dwell(0.0, 0.3, 512) == 512


def pin_no_fill_equals_exhaustive(orc):
    """With fills disabled the recursion only rearranges per-pixel work, so
    the map must equal the exhaustive one exactly, for any (g, r, B)."""
    win = (-2.0, 0.6, -1.25, 1.25)
    for n, g, r, B in [(1, 1, 2, 1), (7, 2, 2, 1), (37, 3, 2, 4), (64, 4, 2, 8),
                       (50, 2, 3, 2), (97, 5, 4, 3)]:
        ex = orc.render_exhaustive(win, n, 96, threads=2)
        ms, _ = orc.render_ms(win, n, 96, g, r, B, flags=NO_FILL, threads=2)
        assert np.array_equal(ex, ms), (n, g, r, B)


def pin_tree_by_hand(orc):
    """Region counts per level with fills disabled, worked out by hand from
    the rules s0 = ceil(n/g), child side ceil(s/r), clip to the parent, drop
    empty children, split while ceil(s/r) >= B and s > 1."""
    win = (-2.0, 0.6, -1.25, 1.25)
    # n=5, g=2: s0=3, regions 3x3, 2x3, 3x2, 2x2.  r=2: child side 2; the 2-wide
    # regions keep one column of children (the second starts at the parent's
    # end): 4 + 2 + 2 + 1 = 9 regions of side 2; then side 1: every pixel.
    _, st = orc.render_ms(win, 5, 50, 2, 2, 1, flags=NO_FILL, threads=1)
    assert st["regions_per_level"] == [4, 9, 25], st
    assert st["subdivisions_per_level"] == [4, 9, 0]
    assert st["leaves"] == 25 and st["leaf_pixels"] == 25
    # n=8, g=2, r=4, B=2: ceil(4/4) = 1 < B, so the four initial regions are leaves.
    _, st = orc.render_ms(win, 8, 50, 2, 4, 2, flags=NO_FILL, threads=1)
    assert st["regions_per_level"] == [4] and st["leaves"] == 4
    # n=7, g=3: s0=3, origins 0, 3, 6 (widths 3, 3, 1): 9 regions, then pixels.
    _, st = orc.render_ms(win, 7, 50, 3, 3, 1, flags=NO_FILL, threads=1)
    assert st["regions_per_level"] == [9, 49], st
    # n=6, g=4: s0=2, origins 0, 2, 4 and one past the edge: 9 non-empty regions.
    _, st = orc.render_ms(win, 6, 50, 4, 2, 4, flags=NO_FILL, threads=1)
    assert st["regions_per_level"] == [9] and st["leaves"] == 9
    # n=64, g=2, r=2, B=8: sides 32, 16, 8 then ceil(8/2)=4 < 8 -> leaves of side 8.
    _, st = orc.render_ms(win, 64, 50, 2, 2, 8, flags=NO_FILL, threads=1)
    assert st["regions_per_level"] == [4, 16, 64] and st["leaves"] == 64


def _perimeter(block):
    h, w = block.shape
    if h <= 2 or w <= 2:
        return block.ravel()
    return np.concatenate([block[0], block[-1], block[1:-1, 0], block[1:-1, -1]])


def check_region_log(ex, ms, st, log, n, g, r, B):
    """Invariants of one Mariani-Silver run, from its region log."""
    s0 = -(-n // g)
    lv0 = log[log["level"] == 0]
    cover = np.zeros((n, n), dtype=np.int32)
    expected0 = {(x, y) for y in range(0, n, s0) for x in range(0, n, s0)}
    assert {(int(e["x0"]), int(e["y0"])) for e in lv0} == expected0
    for e in lv0:
        assert e["s"] == s0 and e["w"] == min(s0, n - e["x0"]) and e["h"] == min(s0, n - e["y0"])
    fill_px = leaf_px = 0
    by_level = {}
    for e in log:
        by_level.setdefault(int(e["level"]), []).append(e)
    for e in log:
        x0, y0, w, h, s = int(e["x0"]), int(e["y0"]), int(e["w"]), int(e["h"]), int(e["s"])
        assert 1 <= w <= s and 1 <= h <= s and x0 + w <= n and y0 + h <= n
        per = _perimeter(ex[y0:y0 + h, x0:x0 + w])
        sc = -(-s // r)
        if e["kind"] == FILL:
            assert np.all(per == e["dwell"])
            assert np.all(ms[y0:y0 + h, x0:x0 + w] == e["dwell"])
            cover[y0:y0 + h, x0:x0 + w] += 1
            fill_px += w * h
        elif e["kind"] == LEAF:
            assert not np.all(per == per[0])
            assert s == 1 or sc < B
            assert np.array_equal(ms[y0:y0 + h, x0:x0 + w], ex[y0:y0 + h, x0:x0 + w])
            cover[y0:y0 + h, x0:x0 + w] += 1
            leaf_px += w * h
        else:
            assert e["kind"] == SUBDIVIDE
            assert not np.all(per == per[0])
            assert s > 1 and sc >= B
            kids = [k for k in by_level.get(int(e["level"]) + 1, [])
                    if x0 <= k["x0"] < x0 + w and y0 <= k["y0"] < y0 + h]
            want = set()
            for b in range(r):
                for a in range(r):
                    cx, cy = x0 + a * sc, y0 + b * sc
                    if cx < x0 + w and cy < y0 + h:
                        want.add((cx, cy, min(sc, x0 + w - cx), min(sc, y0 + h - cy), sc))
            got = {(int(k["x0"]), int(k["y0"]), int(k["w"]), int(k["h"]), int(k["s"])) for k in kids}
            assert got == want
    assert np.all(cover == 1), "fills and leaves must tile the image exactly once"
    assert fill_px == st["fill_pixels"] and leaf_px == st["leaf_pixels"]
    assert fill_px + leaf_px == n * n
    # every pixel on the perimeter of a visited region holds its own dwell
    for e in log:
        x0, y0, w, h = int(e["x0"]), int(e["y0"]), int(e["w"]), int(e["h"])
        assert np.array_equal(_perimeter(ms[y0:y0 + h, x0:x0 + w]),
                              _perimeter(ex[y0:y0 + h, x0:x0 + w]))


def pin_ms_invariants(orc):
    win_boundary = (-1.5, 0.5, -1.0, 1.0)
    for n, M, g, r, B in [(64, 64, 2, 2, 8), (100, 128, 3, 2, 5), (128, 256, 4, 4, 4),
                          (96, 200, 2, 3, 4), (250, 128, 4, 2, 16), (33, 64, 1, 2, 2)]:
        ex = orc.render_exhaustive(win_boundary, n, M, threads=2)
        ms, st, log = orc.render_ms(win_boundary, n, M, g, r, B, log=True)
        check_region_log(ex, ms, st, log, n, g, r, B)


def pin_uniform_windows(orc):
    """Every point far outside (|c| > 2) has dwell 1 and every point of the
    disk |c| < 1/4 lies in the main cardioid, so both windows fill at once."""
    _, st, log = orc.render_ms((3.0, 4.0, 3.0, 4.0), 64, 100, 4, 2, 4, log=True)
    assert st["regions_per_level"] == [16] and st["fills_per_level"] == [16]
    assert np.all(log["dwell"] == 1)
    ms, st = orc.render_ms((-0.15, 0.15, -0.15, 0.15), 64, 300, 4, 2, 4, threads=2)
    assert st["fills_per_level"] == [16] and np.all(ms == 300)


def pin_stopping_side(orc):
    """At the n = 1024, g = 16, r = 2, B = 32 configuration the sides are 64
    then 32, so there are two levels and every leaf has side exactly B."""
    ex = orc.render_exhaustive(C0_WINDOW, 1024, 512, threads=4)
    ms, st, log = orc.render_ms(C0_WINDOW, 1024, 512, 16, 2, 32, log=True)
    assert st["levels"] == 2
    leaves = log[log["kind"] == LEAF]
    assert len(leaves) > 0 and np.all(leaves["s"] == 32) and np.all(leaves["level"] == 1)
    check_region_log(ex, ms, st, log, 1024, 16, 2, 32)


def pin_threads_and_regions(orc):
    """Thread count changes nothing; one initial region rendered alone equals
    its tile of the full map."""
    win = (-2.0, 1.0, -1.5, 1.5)
    a, sa = orc.render_ms(win, 300, 256, 5, 2, 8, threads=1)
    b, sb = orc.render_ms(win, 300, 256, 5, 2, 8, threads=7)
    assert np.array_equal(a, b) and sa == sb
    it = 0
    for gy in range(5):
        for gx in range(5):
            (x0, y0, w, h), tile, st = orc.render_ms_region(win, 300, 256, 5, 2, 8, gx, gy)
            assert np.array_equal(tile, a[y0:y0 + h, x0:x0 + w])
            it += st["iterations"]
    assert it == sa["iterations"]


# --------------------------------------------------------------------------
# double precision (deep zooms)
# --------------------------------------------------------------------------
# A window 2^-28 wide in the upper spiral arm: zoom ~ 7e9 over the paper's
# 2 x 2 window, far past what single precision resolves (the float32 window
# collapses to one column of c), with dwells of 67 to 132.
DEEP_WINDOW = (-0.10109636384562, -0.10109636384562 + 2.0 ** -28,
               0.95628651080914, 0.95628651080914 + 2.0 ** -28)
# Seahorse valley, 2^-30 wide: dwells 1021 to 2000 at a cap of 2000.
SEAHORSE_WINDOW = (-0.743643887037151, -0.743643887037151 + 2.0 ** -30,
                   0.13182590420533, 0.13182590420533 + 2.0 ** -30)


def pin_closed_forms64(orc):
    """Every hand-computed orbit of the fixture takes values with few
    significant bits (exact in float32, hence in double too), so the
    double-precision dwell must give the same counts under both readings."""
    for cr, ci, M, flags, d in closed_forms():
        assert orc.dwell64(cr, ci, M, flags) == d, (cr, ci, M, flags, d)


def pin_exact_points64(orc):
    """Random double points, and points 1e-12 apart that float32 cannot tell
    apart, against the exact-rational brute force rounded to binary64."""
    rng = random.Random(20220606)
    for _ in range(100):
        cr, ci = rng.uniform(-2.2, 1.0), rng.uniform(-1.4, 1.4)
        assert orc.dwell64(cr, ci, 48) == f32exact.dwell64(cr, ci, 48), (cr, ci)
    re0, im0 = DEEP_WINDOW[0], DEEP_WINDOW[2]
    seen = set()
    for k in range(12):
        cr, ci = re0 + k * 1e-12, im0 + (k % 5) * 3e-12
        d = orc.dwell64(cr, ci, 400)
        assert d == f32exact.dwell64(cr, ci, 400), (cr, ci)
        seen.add(d)
    assert len(seen) > 1   # the points are distinct in double


def pin_exact_tiny_maps64(orc):
    """Tiny double-precision maps, pixel for pixel, against the brute force
    (asymmetric windows; one of them a deep zoom), and the pixel -> c map."""
    cases = [((-2.0, 0.5, -1.1, 1.3), 3, 40), ((-0.8, -0.6, 0.05, 0.30), 5, 60),
             (DEEP_WINDOW, 7, 200)]
    for win, n, M in cases:
        got = orc.render_exhaustive(win, n, M, threads=2, fp64=True)
        want = np.array(f32exact.exhaustive64(win, n, M), dtype=np.uint32)
        assert np.array_equal(got, want), (win, n, M)
    rng = random.Random(8)
    for _ in range(60):
        a, b = sorted(rng.uniform(-2.5, 2.5) for _ in range(2))
        c, d = sorted(rng.uniform(-2.5, 2.5) for _ in range(2))
        if b - a < 1e-9 or d - c < 1e-9:
            continue
        n = rng.randint(1, 70000)
        px, py = rng.randrange(n), rng.randrange(n)
        want = tuple(float(v) for v in f32exact.pixel_c64((a, b, c, d), n, px, py))
        assert orc.pixel_to_c64((a, b, c, d), n, px, py) == want, ((a, b, c, d), n, px, py)


def pin_deep_zoom64(orc):
    """Where the spacing is a power of two the double mapping is exact:
    2^-30 / 64 = 2^-36 and every c = re_min + px 2^-36 is a double.  Sampled
    pixels of the seahorse-valley map (dwells near 1000 to 2000) against the
    brute force; Mariani-Silver with fills off equals the exhaustive map."""
    win, n, M = SEAHORSE_WINDOW, 64, 2000
    for px, py in [(0, 0), (63, 0), (17, 40), (63, 63)]:
        assert orc.pixel_to_c64(win, n, px, py) == (win[0] + px * 2.0 ** -36,
                                                    win[2] + py * 2.0 ** -36)
    m = orc.render_exhaustive(win, n, M, threads=4, fp64=True)
    assert m.min() > 1000 and len(np.unique(m)) > 300
    rng = random.Random(64)
    for _ in range(4):
        px, py = rng.randrange(n), rng.randrange(n)
        cr, ci = orc.pixel_to_c64(win, n, px, py)
        assert m[py, px] == f32exact.dwell64(cr, ci, M), (px, py)
    ms, _ = orc.render_ms(win, n, M, 4, 2, 4, flags=NO_FILL, threads=2, fp64=True)
    assert np.array_equal(ms, m)


def pin_ms64_invariants(orc):
    """The recursion's invariants (tiling, uniform perimeters of filled
    regions, children and stopping side) on double-precision maps."""
    for win, n, M, g, r, B in [(DEEP_WINDOW, 64, 300, 4, 2, 4), (DEEP_WINDOW, 100, 300, 3, 2, 5),
                               (SEAHORSE_WINDOW, 96, 2000, 2, 3, 4),
                               ((-1.25066, -1.25066 + 2.0 ** -20, 0.02012, 0.02012 + 2.0 ** -20),
                                128, 1200, 4, 4, 4)]:
        ex = orc.render_exhaustive(win, n, M, threads=2, fp64=True)
        ms, st, log = orc.render_ms(win, n, M, g, r, B, log=True, fp64=True)
        check_region_log(ex, ms, st, log, n, g, r, B)
        assert st["fills_per_level"] != [0] * len(st["fills_per_level"]), (n, g)


# --------------------------------------------------------------------------
# float-float (deep zooms on the single-precision pipe)
# --------------------------------------------------------------------------
FLOAT_FLOAT = 4
SPIRAL_WINDOW = DEEP_WINDOW
ANTENNA_WINDOW = (-1.25066, -1.25066 + 2.0 ** -20, 0.02012, 0.02012 + 2.0 ** -20)


def pin_closed_forms_ff(orc):
    """The hand-computed orbits are exact in float-float as well (every lo
    part stays 0)."""
    for cr, ci, M, flags, d in closed_forms():
        assert orc.dwell_ff(cr, ci, M, flags) == d, (cr, ci, M, flags, d)


def pin_exact_points_ff(orc):
    """Random points, and deep-zoom points 1e-12 apart (float32 alone cannot
    separate them), against an exact-rational evaluation of the float-float
    operations (each float operation rounded once by rn32)."""
    rng = random.Random(20220607)
    for _ in range(60):
        cr, ci = rng.uniform(-2.2, 1.0), rng.uniform(-1.4, 1.4)
        assert orc.dwell_ff(cr, ci, 48) == f32exact.dwell_ff(cr, ci, 48), (cr, ci)
    seen = set()
    for k in range(10):
        cr, ci = SPIRAL_WINDOW[0] + k * 1e-12, SPIRAL_WINDOW[2] + (k % 4) * 3e-12
        d = orc.dwell_ff(cr, ci, 300)
        assert d == f32exact.dwell_ff(cr, ci, 300), (cr, ci)
        seen.add(d)
    assert len(seen) > 1


def pin_ff_tracks_double(orc):
    """Float-float carries about 48 bits, so at zooms of 1e6 to 1e9 its maps
    agree with the binary64 maps except near escape thresholds, where the
    orbit is chaotic: at least 97% of the pixels are equal, and the map
    resolves what float32 cannot (many dwells along each row)."""
    for win, n, M in [(SPIRAL_WINDOW, 48, 1024), (ANTENNA_WINDOW, 48, 2048)]:
        ff = orc.render_exhaustive(win, n, M, flags=FLOAT_FLOAT, threads=2, fp64=True)
        d64 = orc.render_exhaustive(win, n, M, threads=2, fp64=True)
        assert (ff == d64).mean() >= 0.97, (win, (ff == d64).mean())
        assert min(len(np.unique(ff[y])) for y in range(0, n, 7)) > 4


def pin_regions_alone64(orc):
    """One initial region rendered alone equals its tile of the full map, in
    binary64 and in float-float."""
    win = ANTENNA_WINDOW
    for flags in (0, FLOAT_FLOAT):
        full, st = orc.render_ms(win, 150, 600, 4, 3, 4, flags=flags, threads=2, fp64=True)
        it = 0
        for gy in range(4):
            for gx in range(4):
                (x0, y0, w, h), tile, rst = orc.render_ms_region(win, 150, 600, 4, 3, 4, gx, gy,
                                                                 flags=flags, fp64=True)
                assert np.array_equal(tile, full[y0:y0 + h, x0:x0 + w]), (flags, gx, gy)
                it += rst["iterations"]
        assert it == st["iterations"]


def pin_ms_ff_invariants(orc):
    """The recursion's invariants on float-float maps; with fills off it
    equals the float-float exhaustive map."""
    for win, n, M, g, r, B in [(SPIRAL_WINDOW, 64, 300, 4, 2, 4), (ANTENNA_WINDOW, 90, 800, 3, 3, 4)]:
        ex = orc.render_exhaustive(win, n, M, flags=FLOAT_FLOAT, threads=2, fp64=True)
        ms, st, log = orc.render_ms(win, n, M, g, r, B, flags=FLOAT_FLOAT, log=True, fp64=True)
        check_region_log(ex, ms, st, log, n, g, r, B)
        nf, _ = orc.render_ms(win, n, M, g, r, B, flags=FLOAT_FLOAT | NO_FILL, threads=2, fp64=True)
        assert np.array_equal(nf, ex)


ALL_PINS = [pin_closed_forms, pin_exact_points, pin_exact_tiny_maps,
            pin_c0_pixels, pin_symmetry_and_area, pin_no_fill_equals_exhaustive,
            pin_tree_by_hand, pin_ms_invariants, pin_uniform_windows, pin_stopping_side,
            pin_threads_and_regions, pin_closed_forms64, pin_exact_points64,
            pin_exact_tiny_maps64, pin_deep_zoom64, pin_ms64_invariants, pin_closed_forms_ff,
            pin_exact_points_ff, pin_ff_tracks_double, pin_ms_ff_invariants,
            pin_regions_alone64]
