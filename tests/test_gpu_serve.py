"""The continuous-batching server: every request's map equals the same
request rendered alone, whatever batch it landed in; the memory budget
bounds what is in flight."""
import numpy as np
import pytest

from paper_2206_02255_gb300 import inputs

pytestmark = pytest.mark.gpu


def test_served_results_equal_alone(ctx, asklib):
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
    base = [serve.Request(d, *params[d["id"] % 3]) for d in reqs]
    serve.serve_per_frame(ctx, base)
    for q, b in zip(rs, base):
        alone = ctx.render("ask", q.window, q.n, q.max_dwell, asklib.make_params(q.g, q.r, q.B))
        want = alone.cpu().numpy().view(np.uint32)
        assert np.array_equal(q.host.numpy().view(np.uint32), want), q.id
        assert np.array_equal(b.host.numpy().view(np.uint32), want), q.id
        assert q.t_done >= q.t
    s = serve.summarize(rs)
    assert s["requests"] == 48 and s["p50_ms"] <= s["p99_ms"]


def test_served_deep_zooms_render_in_double(ctx, asklib):
    """Requests zoomed past 1e4 are served in double precision: in a mix with
    single-precision requests, each deep map equals the request rendered
    alone by ask_render64, each other map the request rendered by ask_render."""
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
        if asklib.needs_fp64(q.window):
            alone = ctx.render64("ask", q.window, q.n, q.max_dwell, p)
        else:
            alone = ctx.render("ask", q.window, q.n, q.max_dwell, p)
        assert np.array_equal(q.host.numpy().view(np.uint32), alone.cpu().numpy().view(np.uint32)), q.id
