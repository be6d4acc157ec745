"""GPU parity: every method's dwell map against the CPU reference, bit for
bit, through the C ABI (``libask.so`` via the ctypes binding).

* exhaustive kernel  == reference per-pixel map (Sec. 4.1);
* ASK and CDP2       == reference serial Mariani-Silver (Sec. 4.2.1, Sec. 5),
  including the per-level region, fill and split counts;
* tiny grids with every small (g, r, B), ragged sizes, all block shapes;
* full-size n = 16384 and n = 65536 on seeded samples of initial regions
  (each region is an independent subtree, so the reference renders it alone).
"""
import numpy as np
import pytest

from paper_2206_02255_gb300 import inputs

pytestmark = pytest.mark.gpu

NO_FILL = 2


def params(asklib, g=16, r=2, B=32, block=(16, 16), count=False):
    return asklib.make_params(g, r, B, block, asklib.FLAG_COUNT if count else 0)


def gpu_map(ctx, method, window, n, M, p=None, stats=False):
    import torch
    res = ctx.render(method, window, n, M, p, stats=stats)
    out, st = res if stats else (res, None)
    torch.cuda.synchronize()
    m = out.cpu().numpy().view(np.uint32).reshape(n, n)
    return (m, st) if stats else m


def first_diff(a, b):
    idx = np.argwhere(a != b)
    if len(idx) == 0:
        return None
    py, px = idx[0]
    return "%d mismatches; first at (px=%d, py=%d): gpu %d vs oracle %d" % (
        len(idx), px, py, a[py, px], b[py, px])


# --------------------------------------------------------------------------
# exhaustive
# --------------------------------------------------------------------------
@pytest.mark.parametrize("block", inputs.BLOCK_SHAPES)
def test_exhaustive_c0(ctx, orc, asklib, block):
    C = inputs.C0
    want = orc.render_exhaustive(C["window"], C["n"], C["max_dwell"])
    got = gpu_map(ctx, "exhaustive", C["window"], C["n"], C["max_dwell"],
                  params(asklib, block=block))
    assert first_diff(got, want) is None, first_diff(got, want)


@pytest.mark.parametrize("n", [1, 2, 3, 5, 7, 31, 33, 100, 257, 1000])
def test_exhaustive_ragged(ctx, orc, asklib, n):
    for win, M, block in [((-2.0, 0.5, -1.1, 1.3), 100, (8, 4)),
                          ((-0.8, -0.6, 0.05, 0.30), 700, (32, 1)),
                          ((-2.0, 0.47, -1.12, 1.12), 1, (16, 16)),
                          ((-1.9, 0.6, -0.3, 1.2), 17, (64, 8))]:
        want = orc.render_exhaustive(win, n, M)
        got = gpu_map(ctx, "exhaustive", win, n, M, params(asklib, block=block))
        assert first_diff(got, want) is None, (win, n, M, block, first_diff(got, want))


def test_exhaustive_iteration_count(ctx, orc, asklib):
    C = inputs.C0
    want, it = orc.render_exhaustive(C["window"], C["n"], C["max_dwell"], return_iterations=True)
    got, st = gpu_map(ctx, "exhaustive", C["window"], C["n"], C["max_dwell"],
                      params(asklib, count=True), stats=True)
    assert np.array_equal(got, want)
    assert st["iterations"] == it == int(want.astype(np.uint64).sum())


# --------------------------------------------------------------------------
# ASK
# --------------------------------------------------------------------------
def _check_ms(ctx, orc, asklib, method, win, n, M, g, r, B, block=(16, 16), counts=True, flags=0):
    want, ost = orc.render_ms(win, n, M, g, r, B)
    p = params(asklib, g, r, B, block)
    p.flags |= flags
    got, st = gpu_map(ctx, method, win, n, M, p, stats=True)
    d = first_diff(got, want)
    assert d is None, (method, win, n, M, g, r, B, block, d)
    if counts:
        assert st["levels"] >= ost["levels"]
        L = ost["levels"]
        if method == "ask":
            assert st["regions_per_level"][:L] == ost["regions_per_level"]
            assert all(v == 0 for v in st["regions_per_level"][L:])
        assert st["fills_per_level"][:L] == ost["fills_per_level"]
        assert st["subdivisions_per_level"][:L] == ost["subdivisions_per_level"]
        assert st["leaves"] == ost["leaves"]
    return got, st


@pytest.mark.parametrize("block", inputs.BLOCK_SHAPES)
def test_ask_c0(ctx, orc, asklib, block):
    C = inputs.C0
    _check_ms(ctx, orc, asklib, "ask", C["window"], C["n"], C["max_dwell"], C["g"], C["r"],
              C["B"], block)


@pytest.mark.parametrize("exact", [False, True], ids=["query", "exact_borders"])
def test_ask_c0_counters(ctx, orc, asklib, exact):
    """With counting on, pixels and iterations match what the reference's
    region log implies.  Perimeter queries stop at the first two dwells that
    differ, so a level makes at most the full perimeter count; with exact
    borders the last level evaluates whole perimeters and the leaf kernel
    skips them, otherwise the leaf kernel computes whole leaves."""
    C = inputs.C0
    win, n, M = C["window"], C["n"], C["max_dwell"]
    ex = orc.render_exhaustive(win, n, M)
    want, ost, log = orc.render_ms(win, n, M, C["g"], C["r"], C["B"], log=True)
    p = params(asklib, C["g"], C["r"], C["B"], count=True)
    if exact:
        p.flags |= asklib.FLAG_EXACT_BORDERS
    got, st = gpu_map(ctx, "ask", win, n, M, p, stats=True)
    assert np.array_equal(got, want)
    assert st["fill_pixels"] == ost["fill_pixels"]
    assert st["border_pixels"] == ost["border_pixels"]
    L = ost["levels"]
    border_it = [0] * L
    leaf_px = leaf_it = 0
    for e in log:
        x0, y0, w, h = (int(e[k]) for k in ("x0", "y0", "w", "h"))
        blk = ex[y0:y0 + h, x0:x0 + w].astype(np.uint64)
        inner = blk[1:-1, 1:-1] if w > 2 and h > 2 else blk[:0, :0]
        border_it[int(e["level"])] += int(blk.sum() - inner.sum())
        if e["kind"] == 2:
            if exact:
                leaf_px += inner.size
                leaf_it += int(inner.sum())
            else:
                leaf_px += blk.size
                leaf_it += int(blk.sum())
    assert st["leaf_pixels"] == leaf_px
    assert st["leaf_iterations"] == leaf_it
    if exact:
        assert st["iterations_per_level"][L - 1] == border_it[L - 1]
    for i in range(L):
        assert 0 < st["iterations_per_level"][i] <= border_it[i]
    assert st["iterations"] == sum(st["iterations_per_level"]) + st["leaf_iterations"]


def test_ask_fill_rows_wider_than_a_band(ctx, orc, asklib):
    """A window where every |c| > 2 is uniform (dwell 1) at level 0: with
    g = 1 and n = 17000 the single region's rows are wider than one fill band
    (16384 pixels), so the fill list holds one band per row."""
    win, n, M = (2.5, 3.5, 2.5, 3.5), 17000, 64
    want = orc.dwell(*orc.pixel_to_c(win, n, 0, 0), M)
    assert want == 1
    got, st = gpu_map(ctx, "ask", win, n, M, params(asklib, 1, 2, 16, count=True), stats=True)
    assert int((got != want).sum()) == 0
    assert st["fills_per_level"][0] == 1 and sum(st["regions_per_level"][1:]) == 0
    assert st["deferred_fill_pixels"] == n * n


@pytest.mark.parametrize("n,g", [(2049, 2), (1027, 1), (4099, 3), (520, 1), (259, 2), (255, 1)])
def test_ask_fill_band_edges(ctx, orc, asklib, n, g):
    """Uniform windows (every |c| > 2, dwell 1) whose level-0 regions go to
    the fill list: odd n puts row starts and region origins off 16-byte
    boundaries, and the widths run from just above the 128 pixels where a
    band's rows are written one at a time (n = 259, g = 2: widths 130 and
    129) to several bands per region (n = 2049, g = 2: 1025 and 1024;
    n = 4099, g = 3: 1367 and 1365).  The map must be all ones, and every
    pixel must come from a deferred fill."""
    win, M = (2.5, 3.5, 2.5, 3.5), 64
    assert orc.dwell(*orc.pixel_to_c(win, n, n - 1, n - 1), M) == 1
    got, st = gpu_map(ctx, "ask", win, n, M, params(asklib, g, 2, 16, count=True), stats=True)
    assert int((got != 1).sum()) == 0
    assert st["fill_pixels"] == n * n and st["leaf_pixels"] == 0
    assert st["deferred_fill_pixels"] == n * n


def test_ask_deferred_fill_pixels(ctx, orc, asklib):
    """Uniform regions of more than 16384 pixels are left to the fill kernel;
    the counting render reports their pixels, which must be the area of the
    reference's filled regions above that size."""
    win, n, M, g, r, B = inputs.WINDOW_PAPER, 2048, 1024, 4, 4, 16
    want, ost, log = orc.render_ms(win, n, M, g, r, B, log=True)
    got, st = gpu_map(ctx, "ask", win, n, M, params(asklib, g, r, B, count=True), stats=True)
    assert np.array_equal(got, want)
    big = sum(int(e["w"]) * int(e["h"]) for e in log
              if e["kind"] == 0 and int(e["w"]) * int(e["h"]) > 16384)
    assert big > 0
    assert st["deferred_fill_pixels"] == big
    assert st["fill_pixels"] == ost["fill_pixels"]


@pytest.mark.parametrize("flags", ["EXACT_BORDERS", "LEAF_TILED", "EXACT_BORDERS|LEAF_TILED",
                                   "SERIAL_FILL", "SERIAL_FILL|EXACT_BORDERS"])
def test_ask_flag_variants(ctx, orc, asklib, flags):
    """The last-level, leaf-kernel and fill-schedule variants give the same
    map (the last three cases have uniform regions above the in-place fill
    size, some of them ragged)."""
    f = 0
    for name in flags.split("|"):
        f |= getattr(asklib, "FLAG_" + name)
    for win, n, M, g, r, B, block in [(inputs.WINDOW_PAPER, 1024, 512, 16, 2, 32, (16, 16)),
                                      (inputs.WINDOW_WIDE, 777, 300, 5, 3, 4, (8, 8)),
                                      (inputs.WINDOW_PAPER, 2048, 2048, 32, 4, 16, (32, 8)),
                                      (inputs.WINDOW_PAPER, 2048, 1024, 2, 4, 16, (16, 16)),
                                      (inputs.WINDOW_WIDE, 3001, 700, 2, 2, 8, (16, 16)),
                                      (inputs.WINDOW_WIDE, 2500, 400, 3, 5, 16, (16, 16))]:
        want, _ = orc.render_ms(win, n, M, g, r, B)
        p = params(asklib, g, r, B, block)
        p.flags = f
        got = gpu_map(ctx, "ask", win, n, M, p)
        assert first_diff(got, want) is None, (flags, n, g, r, B, first_diff(got, want))


@pytest.mark.parametrize("g,r,B", inputs.c1_sweep())
def test_ask_sweep_n2048(ctx, orc, asklib, g, r, B):
    """The (g, r, B) sweep of the n = 16384 configuration at n = 2048."""
    _check_ms(ctx, orc, asklib, "ask", inputs.WINDOW_PAPER, 2048, 2048, g, r, B)


def test_ask_tiny_all_parameters(ctx, orc, asklib):
    """Every (g, r, B) in {1, 2, 3, 4, 8}^3 (r >= 2, g <= n) on tiny grids."""
    wins = [(-2.0, 0.6, -1.25, 1.25), (-0.8, -0.6, 0.05, 0.30)]
    for n in (1, 2, 3, 5, 8, 16):
        for win in wins:
            want_nf = orc.render_exhaustive(win, n, 60)
            for g in (1, 2, 3, 4, 8):
                if g > n:
                    continue
                for r in (2, 3, 4, 8):
                    for B in (1, 2, 3, 4, 8):
                        want, _ = orc.render_ms(win, n, 60, g, r, B, threads=1)
                        got = gpu_map(ctx, "ask", win, n, 60, params(asklib, g, r, B, (8, 4)))
                        d = first_diff(got, want)
                        assert d is None, (n, win, g, r, B, d)
            assert want_nf.shape == (n, n)


@pytest.mark.parametrize("n,g,r,B", [(100, 3, 2, 4), (257, 5, 3, 2), (1000, 7, 2, 8),
                                     (1023, 16, 2, 16), (4099, 13, 4, 16), (3001, 32, 8, 1),
                                     (777, 777, 2, 1), (500, 2, 64, 1)])
def test_ask_ragged(ctx, orc, asklib, n, g, r, B):
    for win, M in [(inputs.WINDOW_PAPER, 300), (inputs.WINDOW_WIDE, 97)]:
        _check_ms(ctx, orc, asklib, "ask", win, n, M, g, r, B, (32, 8))


def test_ask_random_windows(ctx, orc, asklib):
    for k, win in enumerate(inputs.random_windows(12, seed=3)):
        n = [64, 200, 512, 999][k % 4]
        _check_ms(ctx, orc, asklib, "ask", win, n, 400, [2, 4, 8][k % 3], [2, 4][k % 2],
                  [4, 8, 16][k % 3], (16, 16))


def test_ask_repeat_and_async(ctx, orc, asklib):
    """Two renders on a side stream without synchronisation in between, then
    one with stats: identical maps."""
    import torch
    C = inputs.C0
    p = params(asklib, C["g"], C["r"], C["B"])
    s = torch.cuda.Stream()
    outs = []
    with torch.cuda.stream(s):
        for _ in range(3):
            outs.append(ctx.render("ask", C["window"], C["n"], C["max_dwell"], p))
    s.synchronize()
    ctx.check(s)
    want, _ = orc.render_ms(C["window"], C["n"], C["max_dwell"], C["g"], C["r"], C["B"])
    for o in outs:
        assert np.array_equal(o.cpu().numpy().view(np.uint32), want)


def test_contexts_on_concurrent_streams(orc, asklib):
    """Three contexts render different maps on three streams at once (their
    kernels share the GPU; each context owns its tables and counters): every
    map equals the reference, and a render with stats on one stream reports
    that context's own counts."""
    import torch
    specs = [(inputs.WINDOW_PAPER, 2048, 1024, 16, 4, 16), (inputs.WINDOW_WIDE, 1500, 600, 8, 2, 8),
             ((-0.8, -0.6, 0.05, 0.30), 1111, 2000, 5, 3, 16)]
    ctxs = [asklib.Context(0) for _ in specs]
    streams = [torch.cuda.Stream() for _ in specs]
    try:
        outs = []
        for c, s, (win, n, M, g, r, B) in zip(ctxs, streams, specs):
            with torch.cuda.stream(s):
                outs.append([c.render("ask", win, n, M, params(asklib, g, r, B), stream=s)
                             for _ in range(2)])
        for c, s in zip(ctxs, streams):
            s.synchronize()
            c.check(s)
        for (win, n, M, g, r, B), o2 in zip(specs, outs):
            want, ost = orc.render_ms(win, n, M, g, r, B)
            for o in o2:
                assert first_diff(o.cpu().numpy().view(np.uint32), want) is None, (n, g)
        win, n, M, g, r, B = specs[1]
        _, ost = orc.render_ms(win, n, M, g, r, B)
        with torch.cuda.stream(streams[1]):
            _, st = ctxs[1].render("ask", win, n, M, params(asklib, g, r, B), stream=streams[1],
                                   stats=True)
        assert st["regions_per_level"][:ost["levels"]] == ost["regions_per_level"]
    finally:
        for c in ctxs:
            c.close()


def test_render_host(ctx, orc, asklib):
    C = inputs.C0
    win, n, M = C["window"], C["n"], C["max_dwell"]
    want, _ = orc.render_ms(win, n, M, C["g"], C["r"], C["B"])
    got = ctx.render_host("ask", win, n, M, params(asklib, C["g"], C["r"], C["B"]))
    assert np.array_equal(got, want)
    got = ctx.render_host("exhaustive", win, n, M, params(asklib))
    assert np.array_equal(got, orc.render_exhaustive(win, n, M))


@pytest.mark.parametrize("method", ["ask", "cdp2", "exhaustive"])
def test_render_host_buffers(ctx, orc, asklib, method):
    """Pinned, pageable and misaligned pinned host buffers, with and without
    ASK_FLAG_STAGED_COPY, all get the reference map, also on a ragged n
    whose rows are not a multiple of 16 bytes."""
    import torch
    for win, n, M, g, r, B in [(inputs.WINDOW_PAPER, 1024, 512, 16, 2, 32),
                               (inputs.WINDOW_WIDE, 1001, 300, 7, 2, 8)]:
        if method == "exhaustive":
            want = orc.render_exhaustive(win, n, M)
        else:
            want, _ = orc.render_ms(win, n, M, g, r, B)
        p = params(asklib, g, r, B)
        pinned = torch.zeros((n, n), dtype=torch.int32, pin_memory=True)
        got = ctx.render_host(method, win, n, M, p, out=pinned)
        assert first_diff(got.numpy().view(np.uint32), want) is None, (method, n, "pinned")
        big = torch.zeros(n * n + 4, dtype=torch.int32, pin_memory=True)
        off = big[1:1 + n * n]  # 4 bytes past a 16-byte boundary
        got = ctx.render_host(method, win, n, M, p, out=off)
        assert first_diff(got.numpy().view(np.uint32).reshape(n, n), want) is None, (method, n, "unaligned")
        pageable = np.zeros((n, n), dtype=np.uint32)
        got = ctx.render_host(method, win, n, M, p, out=pageable)
        assert first_diff(got, want) is None, (method, n, "pageable")
        q = params(asklib, g, r, B)
        q.flags |= asklib.FLAG_STAGED_COPY
        pinned.zero_()
        got = ctx.render_host(method, win, n, M, q, out=pinned)
        assert first_diff(got.numpy().view(np.uint32), want) is None, (method, n, "staged")


@pytest.mark.parametrize("n,g,r,B", [(12000, 8, 2, 32), (10500, 7, 3, 8), (16384, 64, 2, 16),
                                     (7500, 5, 2, 16), (16384, 3, 4, 16)])
def test_render_host_banded(ctx, orc, asklib, n, g, r, B):
    """Maps large enough for the banded host pipeline (several bands of
    initial-region rows, a ragged last band) equal the device-output render,
    into pinned and pageable buffers; sampled initial regions also equal the
    reference."""
    import torch
    win, M = inputs.WINDOW_WIDE, 1000
    p = params(asklib, g, r, B)
    want = gpu_map(ctx, "ask", win, n, M, p)
    pinned = torch.zeros((n, n), dtype=torch.int32, pin_memory=True)
    got = ctx.render_host("ask", win, n, M, p, out=pinned).numpy().view(np.uint32)
    assert first_diff(got, want) is None
    pageable = np.zeros((n, n), dtype=np.uint32)
    assert first_diff(ctx.render_host("ask", win, n, M, p, out=pageable), want) is None
    _sampled_regions(ctx, orc, asklib, "ask", win, n, M, g, r, B, (16, 16), k=3, seed=n, full=got)


# --------------------------------------------------------------------------
# CDP2
# --------------------------------------------------------------------------
@pytest.mark.parametrize("g,r,B,block", [(16, 2, 32, (16, 16)), (32, 4, 16, (64, 8)),
                                         (8, 2, 16, (8, 8)), (4, 8, 4, (32, 32))])
def test_cdp2_c0(ctx, orc, asklib, g, r, B, block):
    C = inputs.C0
    _check_ms(ctx, orc, asklib, "cdp2", C["window"], C["n"], C["max_dwell"], g, r, B, block)


@pytest.mark.parametrize("n,g,r,B", [(5, 2, 2, 1), (37, 3, 2, 4), (257, 5, 3, 2),
                                     (1000, 7, 2, 8), (2048, 32, 4, 16)])
def test_cdp2_ragged(ctx, orc, asklib, n, g, r, B):
    _check_ms(ctx, orc, asklib, "cdp2", inputs.WINDOW_WIDE, n, 200, g, r, B, (16, 16))


# --------------------------------------------------------------------------
# the paper's SBR / MBR mappings (Sec. 4.3) for ASK and for CDP2
# --------------------------------------------------------------------------
SCHEMES = ["SBR", "MBR"]
SCHEME_RAGGED = [(1, 1, 2, 1), (5, 2, 2, 1), (37, 3, 2, 4), (257, 5, 3, 2), (1000, 7, 2, 8),
                 (2048, 32, 4, 16), (3001, 11, 8, 3)]


@pytest.mark.parametrize("scheme", SCHEMES)
@pytest.mark.parametrize("block", inputs.BLOCK_SHAPES)
def test_ask_scheme_c0(ctx, orc, asklib, scheme, block):
    C = inputs.C0
    _check_ms(ctx, orc, asklib, "ask", C["window"], C["n"], C["max_dwell"], C["g"], C["r"],
              C["B"], block, flags=getattr(asklib, "FLAG_" + scheme))


@pytest.mark.parametrize("scheme", SCHEMES)
@pytest.mark.parametrize("n,g,r,B", SCHEME_RAGGED)
def test_ask_scheme_ragged(ctx, orc, asklib, scheme, n, g, r, B):
    _check_ms(ctx, orc, asklib, "ask", inputs.WINDOW_WIDE, n, 300, g, r, B, (32, 4),
              flags=getattr(asklib, "FLAG_" + scheme))


@pytest.mark.parametrize("scheme", SCHEMES)
def test_ask_scheme_counters(ctx, orc, asklib, scheme):
    """Both mappings evaluate whole leaves in the last pass and fill the
    same pixels as the reference."""
    C = inputs.C0
    win, n, M = C["window"], C["n"], C["max_dwell"]
    ex = orc.render_exhaustive(win, n, M)
    want, ost, log = orc.render_ms(win, n, M, C["g"], C["r"], C["B"], log=True)
    p = params(asklib, C["g"], C["r"], C["B"], (16, 16), count=True)
    p.flags |= getattr(asklib, "FLAG_" + scheme)
    got, st = gpu_map(ctx, "ask", win, n, M, p, stats=True)
    assert np.array_equal(got, want)
    assert st["fill_pixels"] == ost["fill_pixels"]
    assert st["border_pixels"] == ost["border_pixels"]
    leaf_px = leaf_it = 0
    for e in log:
        if e["kind"] == 2:
            x0, y0, w, h = (int(e[k]) for k in ("x0", "y0", "w", "h"))
            blk = ex[y0:y0 + h, x0:x0 + w].astype(np.uint64)
            leaf_px += blk.size
            leaf_it += int(blk.sum())
    assert st["leaf_pixels"] == leaf_px
    assert st["leaf_iterations"] == leaf_it
    assert st["iterations"] == sum(st["iterations_per_level"]) + st["leaf_iterations"]


@pytest.mark.parametrize("ff", [False, True], ids=["tail", "fire_and_forget"])
@pytest.mark.parametrize("g,r,B,block", [(16, 2, 32, (16, 16)), (32, 4, 16, (64, 8)),
                                         (8, 2, 16, (8, 8))])
def test_cdp2_mbr_c0(ctx, orc, asklib, ff, g, r, B, block):
    C = inputs.C0
    f = asklib.FLAG_MBR | (asklib.FLAG_CDP2_FIRE_AND_FORGET if ff else 0)
    _check_ms(ctx, orc, asklib, "cdp2", C["window"], C["n"], C["max_dwell"], g, r, B, block,
              flags=f)


@pytest.mark.parametrize("n,g,r,B", SCHEME_RAGGED[:5])
def test_cdp2_mbr_ragged(ctx, orc, asklib, n, g, r, B):
    _check_ms(ctx, orc, asklib, "cdp2", inputs.WINDOW_WIDE, n, 200, g, r, B, (16, 16),
              flags=asklib.FLAG_MBR)


# --------------------------------------------------------------------------
# argument errors
# --------------------------------------------------------------------------
def _raw_render(ctx, asklib, method, win, n, M, p, ptr):
    import ctypes
    from paper_2206_02255_gb300.ask import Window, lib
    return lib().ask_render(ctx.handle, method, ctypes.byref(Window(*win)), n, M,
                            ctypes.byref(p) if p is not None else None, ctypes.c_void_p(ptr),
                            None, None)


def test_injected_overflow_is_reported_and_cleared(ctx, orc, asklib):
    """Fault injection through the ABI: with ASK_FLAG_INJECT_OVERFLOW the
    kernels see region tables of capacity 1.  The overflow is latched on the
    device and reported by the next synchronising call (a render with stats,
    or ask_check after an asynchronous render), which clears it; the context
    then renders correctly again."""
    C = inputs.C0
    win, n, M, g, r, B = C["window"], C["n"], C["max_dwell"], C["g"], C["r"], C["B"]
    bad = params(asklib, g, r, B)
    bad.flags = asklib.FLAG_INJECT_OVERFLOW
    with pytest.raises(asklib.AskError) as ei:
        gpu_map(ctx, "ask", win, n, M, bad, stats=True)
    assert ei.value.status == asklib.EOVERFLOW
    want, _ = orc.render_ms(win, n, M, g, r, B)
    got, st = gpu_map(ctx, "ask", win, n, M, params(asklib, g, r, B), stats=True)
    assert first_diff(got, want) is None
    ctx.render("ask", win, n, M, bad)  # asynchronous: nothing to report yet
    with pytest.raises(asklib.AskError) as ei:
        ctx.check()
    assert ei.value.status == asklib.EOVERFLOW
    ctx.check()  # cleared
    got = gpu_map(ctx, "ask", win, n, M, params(asklib, g, r, B))
    assert first_diff(got, want) is None


@pytest.mark.parametrize("method", ["ask", "exhaustive", "cdp2"])
def test_no_write_outside_the_map(ctx, asklib, method):
    """Guard bands before and after the n*n output keep their sentinel: no
    kernel writes outside the map (ragged n puts row ends off 16-byte
    boundaries; the window makes fills, splits and leaves)."""
    import torch
    pre, post, sentinel = 1024, 4096, 0x5A5A5A5A
    for n, g in ((1, 1), (3, 2), (37, 3), (517, 4), (1031, 2), (2053, 3)):
        buf = torch.full((pre + n * n + post,), sentinel, dtype=torch.int32, device="cuda")
        out = buf[pre:pre + n * n].view(n, n)
        ctx.render(method, inputs.WINDOW_WIDE, n, 300, params(asklib, g, 2, 8), out=out)
        torch.cuda.synchronize()
        assert int((buf[:pre] != sentinel).sum()) == 0, (method, n)
        assert int((buf[pre + n * n:] != sentinel).sum()) == 0, (method, n)
        assert int((out == sentinel).sum()) == 0, (method, n)


def test_invalid_arguments(ctx, asklib):
    """Bad arguments return EINVAL before anything is launched: the output
    keeps its old contents."""
    import torch
    W = inputs.WINDOW_PAPER
    out = torch.full((64, 64), 7, dtype=torch.int32, device="cuda")
    ptr = out.data_ptr()
    A, E, C = asklib.METHOD_ASK, asklib.METHOD_EXHAUSTIVE, asklib.METHOD_CDP2
    bad = [
        (A, W, 64, 100, params(asklib, g=0), ptr),
        (A, W, 64, 100, params(asklib, g=65), ptr),
        (A, W, 64, 100, params(asklib, r=1), ptr),
        (A, W, 64, 100, params(asklib, r=65), ptr),
        (A, W, 64, 100, params(asklib, B=0), ptr),
        (A, W, 64, 0, params(asklib), ptr),
        (A, W, 64, 0xffffffff, params(asklib), ptr),
        (A, (0.5, -1.5, -1.0, 1.0), 64, 100, params(asklib), ptr),
        (A, (-1.0, -1.0, -1.0, 1.0), 64, 100, params(asklib), ptr),
        (A, (float("nan"), 0.5, -1.0, 1.0), 64, 100, params(asklib), ptr),
        (A, (float("-inf"), 0.5, -1.0, 1.0), 64, 100, params(asklib), ptr),
        (A, W, 64, 100, params(asklib, block=(5, 5)), ptr),
        (A, W, 64, 100, params(asklib, block=(2048, 1)), ptr),
        (E, W, 64, 100, params(asklib, block=(4, 4)), ptr),
        (A, W, 64, 100, None, ptr),
        (C, W, 64, 100, None, ptr),
        (7, W, 64, 100, params(asklib), ptr),
        (A, W, 0, 100, params(asklib), ptr),
        (A, W, 65537, 100, params(asklib, g=2), ptr),
        (A, W, 64, 100, params(asklib), 0),
        (A, W, 8, 100, params(asklib, g=2, B=2), ptr + 4),      # not 16-byte aligned
        (E, W, 8, 100, params(asklib), ptr + 8),
    ]
    for f in (0x10000, asklib.FLAG_SBR | asklib.FLAG_MBR,
              asklib.FLAG_SBR | asklib.FLAG_EXACT_BORDERS, asklib.FLAG_MBR | asklib.FLAG_LEAF_TILED):
        flags_bad = params(asklib)
        flags_bad.flags = f
        bad.append((A, W, 64, 100, flags_bad, ptr))
    for method, win, n, M, p, q in bad:
        st = _raw_render(ctx, asklib, method, win, n, M, p, q)
        assert st == asklib.EINVAL, (method, win, n, M, st)
    torch.cuda.synchronize()
    assert bool((out == 7).all())
    with pytest.raises(asklib.AskError) as e:
        ctx.render("ask", W, 64, 100, params(asklib, g=0), out=out)
    assert e.value.status == asklib.EINVAL and "g must be" in str(e.value)


# --------------------------------------------------------------------------
# full size, sampled
# --------------------------------------------------------------------------
def _sampled_regions(ctx, orc, asklib, method, win, n, M, g, r, B, block, k, seed, full=None):
    if full is None:
        full = gpu_map(ctx, method, win, n, M, params(asklib, g, r, B, block))
    for gx, gy in inputs.sample_initial_regions(g, k, seed):
        res = orc.render_ms_region(win, n, M, g, r, B, gx, gy)
        if res is None:
            continue
        (x0, y0, w, h), tile, _ = res
        d = first_diff(full[y0:y0 + h, x0:x0 + w], tile)
        assert d is None, (method, n, g, r, B, gx, gy, d)
    return full


@pytest.mark.slow
@pytest.mark.parametrize("g,r,B", [(16, 4, 16), (32, 4, 16), (16, 2, 32), (32, 2, 16), (8, 8, 64)])
def test_c1_ask_sampled(ctx, orc, asklib, g, r, B):
    """n = 16384, dwell 2048 on sampled initial regions; (16, 4, 16) is the
    configuration the benchmark times."""
    C = inputs.C1
    _sampled_regions(ctx, orc, asklib, "ask", C["window"], C["n"], C["max_dwell"], g, r, B,
                     (16, 16), k=6, seed=g * 1000 + r * 10 + B)


@pytest.mark.slow
def test_c1_cdp2_equals_ask(ctx, orc, asklib):
    C = inputs.C1
    p = (C["window"], C["n"], C["max_dwell"])
    a = gpu_map(ctx, "ask", *p, params(asklib, 32, 4, 16))
    c = gpu_map(ctx, "cdp2", *p, params(asklib, 32, 4, 16))
    assert first_diff(c, a) is None
    _sampled_regions(ctx, orc, asklib, "cdp2", *p, 32, 4, 16, (16, 16), k=3, seed=5, full=c)


@pytest.mark.slow
def test_c1_schemes_equal_ask(ctx, orc, asklib):
    """ASK-SBR, ASK-MBR and DP-MBR give the default mapping's map at
    n = 16384 (which is checked against the reference on sampled regions)."""
    C = inputs.C1
    p = (C["window"], C["n"], C["max_dwell"])
    a = gpu_map(ctx, "ask", *p, params(asklib, 32, 4, 16))
    for method, f in (("ask", asklib.FLAG_SBR), ("ask", asklib.FLAG_MBR),
                      ("cdp2", asklib.FLAG_MBR | asklib.FLAG_CDP2_FIRE_AND_FORGET)):
        q = params(asklib, 32, 4, 16, (32, 8))
        q.flags |= f
        b = gpu_map(ctx, method, *p, q)
        assert first_diff(b, a) is None, (method, f)
    _sampled_regions(ctx, orc, asklib, "ask", *p, 32, 4, 16, (16, 16), k=3, seed=11, full=a)


@pytest.mark.slow
def test_c1_exhaustive_sampled(ctx, orc, asklib):
    C = inputs.C1
    win, n, M = C["window"], C["n"], C["max_dwell"]
    full = gpu_map(ctx, "exhaustive", win, n, M, params(asklib))
    for px, py in inputs.sample_pixels(n, 3000, seed=11):
        cr, ci = orc.pixel_to_c(win, n, px, py)
        assert full[py, px] == orc.dwell(cr, ci, M), (px, py)
    # one initial-region-sized block, the reference with fills disabled
    (x0, y0, w, h), tile, _ = orc.render_ms_region(win, n, M, 32, 2, 1 << 20, 20, 14, flags=NO_FILL)
    assert np.array_equal(full[y0:y0 + h, x0:x0 + w], tile)


@pytest.mark.slow
def test_c2_ask_and_exhaustive_sampled(ctx, orc, asklib):
    """n = 65536 (17.2 GB map): ASK at g = 32, r = 2, B = 16 (the
    configuration the benchmark times) and at g = 32, r = 4, B = 16 on sampled
    initial regions, the exhaustive kernel on sampled pixels."""
    import torch
    C = inputs.C2
    win, n, M = C["window"], C["n"], C["max_dwell"]
    out = torch.empty((n, n), dtype=torch.int32, device="cuda")
    for r, seed in ((2, 65536), (4, 65537)):
        ctx.render("ask", win, n, M, params(asklib, 32, r, 16), out=out)
        torch.cuda.synchronize()
        ctx.check()
        for gx, gy in inputs.sample_initial_regions(32, 3, seed=seed):
            (x0, y0, w, h), tile, _ = orc.render_ms_region(win, n, M, 32, r, 16, gx, gy)
            got = out[y0:y0 + h, x0:x0 + w].cpu().numpy().view(np.uint32)
            assert first_diff(got, tile) is None, (r, gx, gy, first_diff(got, tile))
    ctx.render("exhaustive", win, n, M, params(asklib), out=out)
    torch.cuda.synchronize()
    pts = inputs.sample_pixels(n, 2000, seed=12)
    idx = torch.tensor([py * n + px for px, py in pts], dtype=torch.int64, device="cuda")
    vals = out.view(-1)[idx].cpu().numpy().view(np.uint32)
    for (px, py), v in zip(pts, vals):
        cr, ci = orc.pixel_to_c(win, n, px, py)
        assert v == orc.dwell(cr, ci, M), (px, py)
    del out
    torch.cuda.empty_cache()
