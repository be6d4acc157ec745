"""Batched renders (many frames, one launch chain) and their CUDA-graph
form, through the C ABI, against the CPU reference frame by frame."""
import numpy as np
import pytest

from paper_2206_02255_gb300 import inputs

pytestmark = pytest.mark.gpu


def _frames(asklib, specs):
    import torch
    out = []
    for win, n, M, g, r, B in specs:
        out.append(dict(window=win, n=n, max_dwell=M, g=g, r=r, B=B,
                        out=torch.full((n, n), -1, dtype=torch.int32, device="cuda")))
    return out


def _map(t):
    return t.cpu().numpy().view(np.uint32)


MIXED = [
    (inputs.WINDOW_PAPER, 1024, 512, 16, 2, 32),
    (inputs.WINDOW_WIDE, 97, 200, 3, 2, 4),
    ((-0.8, -0.6, 0.05, 0.30), 513, 700, 7, 4, 8),
    ((-2.0, 0.47, -1.12, 1.12), 256, 64, 4, 8, 2),
    (inputs.WINDOW_PAPER, 2048, 2048, 32, 4, 16),
    ((-1.9, 0.6, -0.3, 1.2), 1000, 1, 5, 3, 16),
    ((0.25, 0.26, -0.005, 0.005), 777, 3000, 2, 2, 8),
    # one initial region with an 11996-pixel perimeter: more chunks than a
    # batch level takes, so its chunks are longer than the others'
    (inputs.WINDOW_WIDE, 3000, 300, 1, 2, 16),
]


@pytest.mark.parametrize("exact", [False, True], ids=["query", "exact_borders"])
def test_batch_matches_oracle(ctx, orc, asklib, exact):
    import torch
    frames = _frames(asklib, MIXED)
    flags = asklib.FLAG_COUNT | (asklib.FLAG_EXACT_BORDERS if exact else 0)
    st = ctx.render_batch(frames, flags=flags, stats=True)
    torch.cuda.synchronize()
    regions = {}
    leaves = 0
    for f, (win, n, M, g, r, B) in zip(frames, MIXED):
        want, ost = orc.render_ms(win, n, M, g, r, B)
        got = _map(f["out"])
        assert np.array_equal(got, want), (n, g, r, B, int((got != want).sum()))
        for i, v in enumerate(ost["regions_per_level"]):
            regions[i] = regions.get(i, 0) + v
        leaves += ost["leaves"]
    assert st["regions_per_level"] == [regions[i] for i in range(len(regions))]
    assert st["leaves"] == leaves


def test_batch_single_frame_and_graph(ctx, orc, asklib):
    """Zoomed boundary frames of the batched workload (sides scaled down):
    each render alone, the batch, and two replays of its graph agree, and
    every frame equals the CPU oracle's map."""
    import torch
    specs = []
    for k, f in enumerate(inputs.batch_frames(count=10, seed=3, sides=(300, 1500),
                                              dwells=(256, 4096))):
        specs.append((f["window"], f["n"], f["max_dwell"], [8, 16, 32][k % 3], [2, 4][k % 2], 16))
    frames = _frames(asklib, specs)
    alone = []
    for win, n, M, g, r, B in specs:
        o = ctx.render("ask", win, n, M, asklib.make_params(g, r, B))
        alone.append(_map(o))
    ctx.render_batch(frames)
    torch.cuda.synchronize()
    for f, a in zip(frames, alone):
        assert np.array_equal(_map(f["out"]), a)
    graph = ctx.graph_batch(frames)
    for _ in range(2):
        for f in frames:
            f["out"].fill_(-1)
        graph.launch()
        torch.cuda.synchronize()
        for f, a in zip(frames, alone):
            assert np.array_equal(_map(f["out"]), a)
    graph.close()
    # every frame against the CPU oracle (the batch and the graph equal the
    # single renders above, so they equal the oracle too)
    for k, (win, n, M, g, r, B) in enumerate(specs):
        want, _ = orc.render_ms(win, n, M, g, r, B)
        assert np.array_equal(alone[k], want), (k, n, int((alone[k] != want).sum()))


def test_batch_argument_errors(ctx, asklib):
    import torch
    frames = _frames(asklib, MIXED[:4])
    frames[2]["r"] = 1
    with pytest.raises(asklib.AskError) as e:
        ctx.render_batch(frames)
    assert e.value.status == asklib.EINVAL and "frame 2" in str(e.value)
    frames[2]["r"] = 2
    with pytest.raises(asklib.AskError):
        ctx.render_batch(frames, flags=asklib.FLAG_TIMING)
    with pytest.raises(asklib.AskError):
        ctx.graph_batch(frames, flags=asklib.FLAG_COUNT)
    with pytest.raises(asklib.AskError):
        ctx.render_batch([])
    torch.cuda.synchronize()


def test_batch_routes_deep_frames_to_double(ctx, orc, asklib):
    """Frames zoomed past 1e4 in a batch are rendered in binary64 after the
    single-precision launch chain: every map equals the reference in its
    precision, and the stats count the routed frames.  graph_batch refuses
    them."""
    deep = [(inputs.deep_window(nm)[0], 300 + 37 * k, 700, 4, 2, 8)
            for k, (nm, *_) in enumerate(inputs.DEEP_SPOTS)]
    specs = MIXED[:3] + deep[:2] + MIXED[3:5] + deep[2:]
    frames = _frames(asklib, specs)
    st = ctx.render_batch(frames, stats=True)
    assert st["fp64_frames"] == 3
    for (win, n, M, g, r, B), f in zip(specs, frames):
        fp64 = asklib.needs_fp64(win)
        want, _ = orc.render_ms(win, n, M, g, r, B, fp64=fp64)
        assert np.array_equal(_map(f["out"]), want), (n, fp64)
    with pytest.raises(ValueError):
        ctx.graph_batch(frames)
