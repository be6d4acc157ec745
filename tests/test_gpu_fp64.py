"""Deep-zoom renders (ask_render64) through the C ABI against the CPU
reference, bit for bit, in both arithmetics: binary64 against the
reference's double-precision maps, float-float (ASK_FLAG_FLOAT_FLOAT)
against its float-float maps (GPU)."""
import functools

import numpy as np
import pytest

from paper_2206_02255_gb300 import inputs

pytestmark = pytest.mark.gpu


def params(asklib, g, r, B, block=(16, 16), flags=0):
    return asklib.make_params(g, r, B, block, flags)


# (name, library flag, reference flag)
PRECISIONS = [("f64", 0, 0), ("ff", 1024, 4)]
PREC_IDS = [p[0] for p in PRECISIONS]


def host(t):
    return t.cpu().numpy().view(np.uint32)


def first_diff(got, want):
    bad = np.argwhere(got != want)
    if len(bad) == 0:
        return None
    y, x = bad[0]
    return "%d pixels differ, first (px=%d, py=%d): got %d want %d" % (
        len(bad), x, y, got[y, x], want[y, x])


DEEP = [inputs.deep_window(nm) for nm, *_ in inputs.DEEP_SPOTS]


@functools.lru_cache(maxsize=None)
def reference_exhaustive64(win, n, M, oflags=0):
    import oracle
    return oracle.render_exhaustive(win, n, M, flags=oflags, fp64=True)


@pytest.mark.parametrize("prec", PRECISIONS, ids=PREC_IDS)
@pytest.mark.parametrize("k", range(len(DEEP)), ids=[s[0] for s in inputs.DEEP_SPOTS])
@pytest.mark.parametrize("block", [(16, 16), (8, 8), (64, 4)])
def test_exhaustive64_deep(ctx, orc, asklib, k, block, prec):
    win, M = DEEP[k]
    _, flag, oflag = prec
    for n in (257, 1000):
        got = host(ctx.render64("exhaustive", win, n, M, params(asklib, 1, 2, 1, block, flag)))
        assert first_diff(got, reference_exhaustive64(win, n, M, oflag)) is None, (n, block)


@pytest.mark.parametrize("prec", PRECISIONS, ids=PREC_IDS)
def test_exhaustive64_shallow_and_ragged(ctx, orc, asklib, prec):
    """Windows where |c| > 2 occurs (the tested dwell loop runs) and ragged
    sizes, including n = 1."""
    _, flag, oflag = prec
    for win, n, M in [(inputs.WINDOW_WIDE, 1, 100), (inputs.WINDOW_WIDE, 3, 100),
                      ((-2.5, 1.5, -2.0, 2.0), 333, 300), (inputs.WINDOW_PAPER, 1024, 512)]:
        got = host(ctx.render64("exhaustive", win, n, M, params(asklib, 1, 2, 1, flags=flag)))
        want = orc.render_exhaustive(win, n, M, flags=oflag, fp64=True)
        assert first_diff(got, want) is None, (win, n)


@pytest.mark.parametrize("prec", PRECISIONS, ids=PREC_IDS)
@pytest.mark.parametrize("k", range(len(DEEP)), ids=[s[0] for s in inputs.DEEP_SPOTS])
def test_ask64_deep_maps_and_counts(ctx, orc, asklib, k, prec):
    """ASK: the map, and per-level regions, fills and splits, leaves and
    (with counting) fill and leaf pixels, equal the reference's."""
    win, M = DEEP[k]
    _, flag, oflag = prec
    for n, g, r, B in [(1024, 16, 2, 16), (1000, 8, 4, 8), (777, 5, 3, 4), (512, 64, 2, 2)]:
        out, st = ctx.render64("ask", win, n, M,
                               params(asklib, g, r, B, flags=asklib.FLAG_COUNT | flag), stats=True)
        want, ost = orc.render_ms(win, n, M, g, r, B, flags=oflag, fp64=True)
        assert first_diff(host(out), want) is None, (n, g, r, B)
        L = ost["levels"]
        assert st["levels"] == L
        assert st["regions_per_level"][:L] == ost["regions_per_level"]
        assert st["fills_per_level"][:L] == ost["fills_per_level"]
        assert st["subdivisions_per_level"][:L] == ost["subdivisions_per_level"]
        assert st["leaves"] == ost["leaves"]
        assert st["fill_pixels"] == ost["fill_pixels"] and st["leaf_pixels"] == ost["leaf_pixels"]


@pytest.mark.parametrize("prec", PRECISIONS, ids=PREC_IDS)
def test_ask64_leaf_iterations_are_leaf_dwells(ctx, orc, asklib, prec):
    """With counting, the leaf kernel's updates equal the sum of the leaf
    pixels' dwells taken from the reference's region log."""
    win, M = DEEP[1]
    n, g, r, B = 640, 8, 2, 16
    _, flag, oflag = prec
    out, st = ctx.render64("ask", win, n, M,
                           params(asklib, g, r, B, flags=asklib.FLAG_COUNT | flag), stats=True)
    want, ost, log = orc.render_ms(win, n, M, g, r, B, flags=oflag, log=True, fp64=True)
    assert first_diff(host(out), want) is None
    leaf_sum = 0
    for e in log[log["kind"] == 2]:
        x0, y0, w, h = int(e["x0"]), int(e["y0"]), int(e["w"]), int(e["h"])
        leaf_sum += int(want[y0:y0 + h, x0:x0 + w].astype(np.uint64).sum())
    assert st["leaf_iterations"] == leaf_sum
    assert st["leaf_pixels"] == ost["leaf_pixels"] > 0


@pytest.mark.parametrize("prec", PRECISIONS, ids=PREC_IDS)
def test_ask64_tiny_grids(ctx, orc, asklib, prec):
    """Every (g, r, B) in {1, 2, 3, 4, 8}^3 that is valid, on tiny ragged n."""
    win = DEEP[2][0]
    _, flag, oflag = prec
    for n in (1, 2, 3, 5, 8, 16):
        for g in (1, 2, 3, 4, 8):
            if g > n:
                continue
            for r in (2, 3, 4, 8):
                for B in (1, 2, 3, 4, 8):
                    got = host(ctx.render64("ask", win, n, 300, params(asklib, g, r, B, flags=flag)))
                    want, _ = orc.render_ms(win, n, 300, g, r, B, flags=oflag, threads=1, fp64=True)
                    assert first_diff(got, want) is None, (n, g, r, B)


@pytest.mark.parametrize("prec", PRECISIONS, ids=PREC_IDS)
def test_ask64_seeded_deep_frames(ctx, orc, asklib, prec):
    """The seeded deep-zoom frames (zoom 1e5 to 1e10 on boundary points):
    ASK and the exhaustive kernel against the reference, and the
    subdivision-vs-exhaustive mismatch reported."""
    name, flag, oflag = prec
    mism = total = 0
    for f in inputs.deep_frames(12, 3, sides=(200, 1500)):
        win, n, M = f["window"], f["n"], f["max_dwell"]
        g = max(1, min(n, n // 64))
        ask_map = host(ctx.render64("ask", win, n, M, params(asklib, g, 2, 16, flags=flag)))
        want, _ = orc.render_ms(win, n, M, g, 2, 16, flags=oflag, fp64=True)
        assert first_diff(ask_map, want) is None, (n, M, f["zoom"])
        ex = host(ctx.render64("exhaustive", win, n, M, params(asklib, 1, 2, 1, flags=flag)))
        assert first_diff(ex, orc.render_exhaustive(win, n, M, flags=oflag, fp64=True)) is None
        mism += int((ask_map != ex).sum())
        total += n * n
    print("deep frames (%s): subdivision-vs-exhaustive mismatch %d of %d pixels"
          % (name, mism, total))


def test_ask64_async_streams_and_repeat(ctx, orc, asklib):
    import torch
    win, M = DEEP[0]
    n, g, r, B = 900, 12, 2, 8
    want, _ = orc.render_ms(win, n, M, g, r, B, fp64=True)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        outs = [ctx.render64("ask", win, n, M, params(asklib, g, r, B), stream=s) for _ in range(3)]
    s.synchronize()
    ctx.check(s)
    for o in outs:
        assert first_diff(host(o), want) is None


def test_float_float_against_binary64(ctx, asklib):
    """Float-float maps of the deep windows agree with the binary64 maps on
    most pixels (they differ where the orbit is chaotic); reported."""
    for (nm, *_), (win, M) in zip(inputs.DEEP_SPOTS, DEEP):
        p64 = params(asklib, 16, 2, 16)
        pff = params(asklib, 16, 2, 16, flags=asklib.FLAG_FLOAT_FLOAT)
        a = host(ctx.render64("ask", win, 1024, M, p64))
        b = host(ctx.render64("ask", win, 1024, M, pff))
        same = float((a == b).mean())
        print("%s n=1024: float-float equals binary64 on %.2f%% of pixels" % (nm, 100 * same))
        assert same > 0.8, nm


def test_fp64_separates_what_float_cannot(ctx, asklib):
    """At a width of 2^-30 the single-precision window is empty (its corners
    round to one float), which ask_render rejects; in double every column of
    the seahorse-valley map is its own c and the map varies along each row."""
    win, M = DEEP[1]
    with pytest.raises(asklib.AskError):
        ctx.render("exhaustive", win, 256, M)
    m = host(ctx.render64("ask", win, 256, M, params(asklib, 8, 2, 8)))
    assert all(len(np.unique(m[y])) > 16 for y in (0, 100, 255))


def test_render64_invalid_arguments(ctx, asklib):
    import torch
    win, M = DEEP[0]
    out = torch.full((64, 64), 7, dtype=torch.int32, device="cuda:0")
    bad = [("cdp2", win, 64, M, params(asklib, 4, 2, 4)),
           ("ask", win, 64, M, params(asklib, 4, 2, 4, flags=asklib.FLAG_SBR)),
           ("ask", win, 64, M, params(asklib, 4, 2, 4, flags=asklib.FLAG_TIMING)),
           ("ask", win, 64, M, params(asklib, 4, 1, 4)),
           ("ask", (0.0, float("nan"), 0.0, 1.0), 64, M, params(asklib, 4, 2, 4)),
           ("ask", (1.0, 0.5, 0.0, 1.0), 64, M, params(asklib, 4, 2, 4)),
           ("exhaustive", win, 64, 0, None),
           ("ask", win, 64, M, None)]
    for method, w, n, md, p in bad:
        with pytest.raises(asklib.AskError) as e:
            ctx.render64(method, w, n, md, p, out=out)
        assert e.value.status == asklib.EINVAL, (method, w, md)
    torch.cuda.synchronize()
    assert bool((out == 7).all())


@pytest.mark.slow
@pytest.mark.parametrize("prec", PRECISIONS, ids=PREC_IDS)
def test_deep_bench_size_sampled(ctx, orc, asklib, prec):
    """The deep bench's workload at full size (n = 8192, seahorse valley
    2^-30 wide, dwell cap 4096, g=128 r=4 B=16): 24 seeded initial regions
    of the ASK map against the reference rendering each region alone, and
    600 seeded pixels of the exhaustive map against the reference dwell of
    the pixel's c."""
    import oracle
    name, flag, oflag = prec
    win, M = inputs.deep_window("seahorse_2^-30")
    n, g, r, B = 8192, 128, 4, 16
    out = ctx.render64("ask", win, n, M, params(asklib, g, r, B, flags=flag))
    got = host(out)
    for gx, gy in inputs.sample_initial_regions(g, 24, seed=8192):
        (x0, y0, w, h), tile, _ = orc.render_ms_region(win, n, M, g, r, B, gx, gy,
                                                       flags=oflag, fp64=True)
        assert first_diff(got[y0:y0 + h, x0:x0 + w], tile) is None, (name, gx, gy)
    ex = host(ctx.render64("exhaustive", win, n, M, params(asklib, 1, 2, 1, flags=flag)))
    for px, py in inputs.sample_pixels(n, 600, seed=8193):
        cr, ci = orc.pixel_to_c64(win, n, px, py)
        want = oracle.dwell_ff(cr, ci, M) if oflag else oracle.dwell64(cr, ci, M)
        assert ex[py, px] == want, (name, px, py)
