"""The continuous-batching server: every request's map equals the CPU
oracle's map of that request (paper Sec. 6: the map is what must match;
batching only changes the schedule), and equals the same request rendered
alone, whatever batch it landed in; the memory budget bounds what is in
flight."""
import numpy as np
import pytest

from paper_2206_02255_gb300 import inputs

pytestmark = pytest.mark.gpu


def _want(orc, asklib, q):
    """The oracle's map of request q, in the precision the server uses."""
    fp64 = asklib.needs_fp64(q.window)
    want, _ = orc.render_ms(q.window, q.n, q.max_dwell, q.g, q.r, q.B, fp64=fp64)
    return want


def test_served_results_equal_oracle_and_alone(ctx, orc, asklib):
    from paper_2206_02255_gb300 import serve
    reqs = inputs.serving_requests(count=48, seed=7, rate=4000.0, sides=(256, 900),
                                   dwells=(256, 2048))
    params = [(8, 4, 16), (16, 2, 16), (32, 2, 8)]
    budget = 6 * 2 ** 20  # a few frames at a time: batches of several sizes
    srv = serve.Server(device=0, slots=2, budget_bytes=budget)
    peak = [0]
    start = srv._start

    def watch(slot, reqs):
        start(slot, reqs)
        peak[0] = max(peak[0], srv.used)
    srv._start = watch
    rs = [serve.Request(d, *params[d["id"] % 3]) for d in reqs]
    srv.run(rs)
    srv.close()
    assert peak[0] <= budget
    assert srv.batch_dispatches >= 1  # requests queued up: the batch path ran
    base = [serve.Request(d, *params[d["id"] % 3]) for d in reqs]
    serve.serve_per_frame(ctx, base)
    for q, b in zip(rs, base):
        want = _want(orc, asklib, q)
        got = q.host.numpy().view(np.uint32)
        assert np.array_equal(got, want), (q.id, int((got != want).sum()))
        assert np.array_equal(b.host.numpy().view(np.uint32), want), q.id
        alone = ctx.render("ask", q.window, q.n, q.max_dwell, asklib.make_params(q.g, q.r, q.B))
        assert np.array_equal(got, alone.cpu().numpy().view(np.uint32)), q.id
        assert q.t_done >= q.t
    s = serve.summarize(rs)
    assert s["requests"] == 48 and s["p50_ms"] <= s["p99_ms"]


def test_served_idle_requests_take_the_single_frame_path(ctx, orc, asklib):
    """Requests that arrive far apart find the GPU idle: each is dispatched
    on its own through the single-frame call, and its map equals the
    oracle's."""
    from paper_2206_02255_gb300 import serve
    reqs = inputs.serving_requests(count=6, seed=17, rate=50.0, sides=(256, 600),
                                   dwells=(256, 1024))
    srv = serve.Server(device=0, slots=2, budget_bytes=64 * 2 ** 20)
    rs = [serve.Request(d, 8, 2, 16) for d in reqs]
    srv.run(rs)
    srv.close()
    assert srv.single_dispatches >= 1
    for q in rs:
        want = _want(orc, asklib, q)
        assert np.array_equal(q.host.numpy().view(np.uint32), want), q.id


def test_served_deep_zooms_render_in_double(ctx, orc, asklib):
    """Requests zoomed past 1e4 are served in double precision: in a mix with
    single-precision requests, each deep map equals the oracle's binary64
    map and the request rendered alone by ask_render64, each other map the
    oracle's single-precision map and the request rendered by ask_render."""
    from paper_2206_02255_gb300 import serve
    shallow = inputs.serving_requests(count=12, seed=11, rate=4000.0, sides=(256, 700),
                                      dwells=(256, 1024))
    deep = inputs.deep_frames(count=8, seed=5, sides=(200, 600), dwells=(256, 2048))
    mixed = []
    for k in range(20):
        d = dict(shallow[k // 2]) if k % 2 == 0 or k // 2 >= len(deep) else dict(deep[k // 2])
        d["id"], d["t"] = k, 0.0005 * k
        mixed.append(d)
    assert sum(asklib.needs_fp64(d["window"]) for d in mixed) >= 6
    srv = serve.Server(device=0, slots=2, budget_bytes=4 * 2 ** 20)
    rs = [serve.Request(d, 8, 2, 16) for d in mixed]
    srv.run(rs)
    srv.close()
    p = asklib.make_params(8, 2, 16)
    for q in rs:
        got = q.host.numpy().view(np.uint32)
        want = _want(orc, asklib, q)
        assert np.array_equal(got, want), (q.id, int((got != want).sum()))
        if asklib.needs_fp64(q.window):
            alone = ctx.render64("ask", q.window, q.n, q.max_dwell, p)
        else:
            alone = ctx.render("ask", q.window, q.n, q.max_dwell, p)
        assert np.array_equal(got, alone.cpu().numpy().view(np.uint32)), q.id
