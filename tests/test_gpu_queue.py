"""Batches rendered by one persistent kernel over a device work queue
(ASK_FLAG_PERSISTENT), through the C ABI, against the CPU oracle frame by
frame (paper Sec. 5: the region tables of ASK kept on the device; the map is
the one the oracle's serial recursion of Sec. 4.2.1 gives), and the bounded
waits of that kernel: a render whose waits run out reports ASK_ETIMEOUT and
leaves the context usable."""
import numpy as np
import pytest

from paper_2206_02255_gb300 import inputs

pytestmark = pytest.mark.gpu

MIXED = [
    (inputs.WINDOW_PAPER, 1024, 512, 16, 2, 32),
    (inputs.WINDOW_WIDE, 97, 200, 3, 2, 4),
    ((-0.8, -0.6, 0.05, 0.30), 513, 700, 7, 4, 8),
    ((-2.0, 0.47, -1.12, 1.12), 256, 64, 4, 8, 2),
    (inputs.WINDOW_PAPER, 2048, 2048, 32, 4, 16),
    ((-1.9, 0.6, -0.3, 1.2), 1000, 1, 5, 3, 16),
    ((0.25, 0.26, -0.005, 0.005), 777, 3000, 2, 2, 8),
    # one initial region with an 11996-pixel perimeter: more chunk items than
    # a region takes, so its chunks are longer than the others'
    (inputs.WINDOW_WIDE, 3000, 300, 1, 2, 16),
    # uniform regions larger than the in-place fill size: fill bands go
    # through the queue
    ((-0.3, -0.1, -0.1, 0.1), 1200, 400, 2, 2, 64),
]


def _frames(specs):
    import torch
    return [dict(window=win, n=n, max_dwell=M, g=g, r=r, B=B,
                 out=torch.full((n, n), -1, dtype=torch.int32, device="cuda"))
            for win, n, M, g, r, B in specs]


def _map(t):
    return t.cpu().numpy().view(np.uint32)


def test_persistent_batch_matches_oracle(ctx, orc, asklib):
    import torch
    frames = _frames(MIXED)
    st = ctx.render_batch(frames, flags=asklib.FLAG_PERSISTENT | asklib.FLAG_COUNT, stats=True)
    torch.cuda.synchronize()
    assert st["kernel_launches"] == 2
    regions, fills, splits, leaves = {}, {}, {}, 0
    for f, (win, n, M, g, r, B) in zip(frames, MIXED):
        want, ost = orc.render_ms(win, n, M, g, r, B)
        got = _map(f["out"])
        assert np.array_equal(got, want), (n, g, r, B, int((got != want).sum()))
        for i, v in enumerate(ost["regions_per_level"]):
            regions[i] = regions.get(i, 0) + v
        for i, v in enumerate(ost["fills_per_level"]):
            fills[i] = fills.get(i, 0) + v
        for i, v in enumerate(ost["subdivisions_per_level"]):
            splits[i] = splits.get(i, 0) + v
        leaves += ost["leaves"]
    L = len(regions)
    assert st["regions_per_level"][:L] == [regions[i] for i in range(L)]
    assert st["fills_per_level"][:L] == [fills[i] for i in range(L)]
    assert st["subdivisions_per_level"][:L] == [splits[i] for i in range(L)]
    assert st["leaves"] == leaves


def test_persistent_batch_tiny_and_ragged_frames(ctx, orc, asklib):
    """Frames of 1 to 64 pixels a side under every (g, r, B) in a small set,
    one persistent batch: regions of side 1 and 2, clipped children, a
    single initial region, leaves at the first level."""
    import itertools
    import torch
    specs = []
    for n, (g, r, B) in itertools.product((1, 2, 3, 5, 8, 16, 64),
                                          itertools.product((1, 2, 3), (2, 3), (1, 2, 4))):
        if g <= n:
            specs.append((inputs.WINDOW_WIDE if n % 2 else inputs.WINDOW_PAPER, n, 50 + n, g, r, B))
    frames = _frames(specs)
    ctx.render_batch(frames, flags=asklib.FLAG_PERSISTENT)
    torch.cuda.synchronize()
    for f, (win, n, M, g, r, B) in zip(frames, specs):
        want, _ = orc.render_ms(win, n, M, g, r, B)
        assert np.array_equal(_map(f["out"]), want), (n, g, r, B)


def test_persistent_batch_twice_and_after_the_chain(ctx, orc, asklib):
    """Renders in a row on one context (each render's queue slots carry a new
    epoch, so the previous render's items are never taken for this one's),
    with a chain-of-launches render in between; every map equals the
    oracle's."""
    import torch
    specs = MIXED[:5]
    wants = [orc.render_ms(win, n, M, g, r, B)[0] for win, n, M, g, r, B in specs]
    for flags in (asklib.FLAG_PERSISTENT, 0, asklib.FLAG_PERSISTENT, asklib.FLAG_PERSISTENT):
        frames = _frames(specs)
        ctx.render_batch(frames, flags=flags)
        torch.cuda.synchronize()
        for f, want in zip(frames, wants):
            assert np.array_equal(_map(f["out"]), want), flags
    # a smaller batch after a larger one: leftover slots of the larger render
    # stay behind the new epoch
    frames = _frames(specs[1:2])
    ctx.render_batch(frames, flags=asklib.FLAG_PERSISTENT)
    torch.cuda.synchronize()
    assert np.array_equal(_map(frames[0]["out"]), wants[1])


def test_persistent_batch_graph(ctx, orc, asklib):
    """The persistent batch captured as a CUDA graph: replays render the same
    maps (the render epoch lives on the device, so each replay's items are
    new)."""
    import torch
    specs = MIXED[:4] + MIXED[6:]
    frames = _frames(specs)
    graph = ctx.graph_batch(frames, flags=asklib.FLAG_PERSISTENT)
    wants = [orc.render_ms(win, n, M, g, r, B)[0] for win, n, M, g, r, B in specs]
    for _ in range(3):
        for f in frames:
            f["out"].fill_(-1)
        graph.launch()
        torch.cuda.synchronize()
        for f, want in zip(frames, wants):
            assert np.array_equal(_map(f["out"]), want)
    graph.close()


def test_persistent_batched_workload_subset(ctx, orc, asklib):
    """Sixteen seeded frames of the batched workload (sides 512 to 8192,
    zooms 1 to 1e4 on boundary points, dwell caps 256 to 8192), at the
    parameters the autotuner gives each frame in the benchmark's range."""
    import torch
    picks = inputs.batch_frames(count=256, seed=0)
    rng = np.random.default_rng(2206)
    idx = sorted(rng.choice(len(picks), size=16, replace=False).tolist())
    specs = []
    for k in idx:
        f = picks[k]
        s0 = 256 if f["n"] > 4096 else 128
        g = max(1, -(-f["n"] // s0))
        specs.append((f["window"], f["n"], f["max_dwell"], g, 4, 8))
    frames = _frames(specs)
    ctx.render_batch(frames, flags=asklib.FLAG_PERSISTENT)
    torch.cuda.synchronize()
    for f, (win, n, M, g, r, B) in zip(frames, specs):
        want, _ = orc.render_ms(win, n, M, g, r, B)
        got = _map(f["out"])
        assert np.array_equal(got, want), (n, M, g, int((got != want).sum()))


def test_persistent_batch_wait_runs_out(ctx, orc, asklib):
    """ASK_FLAG_WAIT_TEST cuts the idle-wait limit to one poll: a render with
    far fewer items than warps has idle warps at once, so it latches a
    timeout, and the synchronising call reports ASK_ETIMEOUT.  The context
    then renders correctly."""
    import torch
    specs = [(inputs.WINDOW_PAPER, 256, 256, 2, 2, 16)]
    frames = _frames(specs)
    with pytest.raises(asklib.AskError) as e:
        ctx.render_batch(frames, flags=asklib.FLAG_PERSISTENT | asklib.FLAG_WAIT_TEST, stats=True)
    assert e.value.status == asklib.ETIMEOUT
    assert asklib.status_str(asklib.ETIMEOUT) == "device wait timed out"
    # reported once, then cleared; the next renders are whole
    ctx.check()
    want, _ = orc.render_ms(*specs[0])
    for flags in (asklib.FLAG_PERSISTENT, 0):
        frames = _frames(specs)
        ctx.render_batch(frames, flags=flags, stats=True)
        assert np.array_equal(_map(frames[0]["out"]), want)
    torch.cuda.synchronize()


def test_persistent_batch_argument_errors(ctx, asklib):
    frames = _frames(MIXED[:2])
    with pytest.raises(asklib.AskError) as e:
        ctx.render_batch(frames, flags=asklib.FLAG_PERSISTENT | asklib.FLAG_EXACT_BORDERS)
    assert e.value.status == asklib.EINVAL
    with pytest.raises(asklib.AskError) as e:
        ctx.render_batch(frames, flags=asklib.FLAG_WAIT_TEST)
    assert e.value.status == asklib.EINVAL
    with pytest.raises(asklib.AskError):
        ctx.graph_batch(frames, flags=asklib.FLAG_PERSISTENT | asklib.FLAG_COUNT)
