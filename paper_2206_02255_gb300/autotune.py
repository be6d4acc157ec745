"""Autotuner for ASK's subdivision parameters (g, r, B).

The paper searches {g, r, B} exhaustively per GPU and problem size
(Sec. 6.2, Fig. 6) and derives model optima from its cost model (Sec. 4).
Here:

* :func:`sweep` times real renders of one frame over a candidate grid
  (CUDA events on the rendering stream; every render goes through the C ABI);
* :class:`BatchTuner` tunes a batch of frames of different size, zoom and
  dwell cap: it sweeps a few probe frames spread over the batch and gives
  every frame the best configuration of its nearest probe;
* :func:`model_choice` reports the cost model's optimum for the same frame,
  with the subdivision probability P estimated from the measured per-level
  counts, to set the measured choice beside the model's.
"""
import math

from . import ask, costmodel

DEFAULT_SPACE = dict(g=(2, 4, 8, 16, 32, 64), r=(2, 4, 8), B=(8, 16, 32, 64))


def candidates(n, space=None):
    """Valid (g, r, B) for an n x n frame."""
    space = space or DEFAULT_SPACE
    out = []
    for g in space["g"]:
        if g > n:
            continue
        for r in space["r"]:
            for B in space["B"]:
                try:
                    ask.plan_levels(n, g, r, B)
                except ask.AskError:
                    continue
                out.append((g, r, B))
    return out


def time_config(ctx, window, n, max_dwell, g, r, B, out, reps=2, flags=0):
    """Mean device time (ms) of `reps` ASK renders after one warm-up."""
    import torch
    p = ask.make_params(g, r, B, (16, 16), flags)
    s = torch.cuda.current_stream(out.device)
    ctx.render("ask", window, n, max_dwell, p, out=out)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(s)
    for _ in range(reps):
        ctx.render("ask", window, n, max_dwell, p, out=out)
    e1.record(s)
    e1.synchronize()
    return e0.elapsed_time(e1) / reps


def sweep(ctx, window, n, max_dwell, space=None, reps=2, out=None):
    """Time every candidate; returns [{"ms", "g", "r", "B"}] fastest first."""
    import torch
    if out is None:
        out = torch.empty((n, n), dtype=torch.int32, device="cuda:%d" % ctx.device)
    res = []
    for g, r, B in candidates(n, space):
        res.append(dict(ms=time_config(ctx, window, n, max_dwell, g, r, B, out, reps), g=g, r=r, B=B))
    res.sort(key=lambda d: d["ms"])
    return res


def model_choice(ctx, window, n, max_dwell, g, r, B, lam=None, q=None, c=128, reps=3):
    """The cost model's SBR-time optimum for this frame.  P is estimated from
    a counting render at (g, r, B); lambda, unless given, is fitted (with the
    model's time scale kappa) to the per-level and leaf device times of
    `reps` timed renders there; q = the device's SM count."""
    import torch
    out = torch.empty((n, n), dtype=torch.int32, device="cuda:%d" % ctx.device)
    _, st = ctx.render("ask", window, n, max_dwell,
                       ask.make_params(g, r, B, (16, 16), ask.FLAG_COUNT), out=out, stats=True)
    P = costmodel.estimate_p(st)
    if q is None:
        q = torch.cuda.get_device_properties(ctx.device).multi_processor_count
    kappa = None
    if lam is None:
        ctx.timing_read()  # forget older timed renders
        p = ask.make_params(g, r, B, (16, 16), ask.FLAG_TIMING)
        for _ in range(reps):
            ctx.render("ask", window, n, max_dwell, p, out=out)
        t = ctx.timing_read()
        L = st["levels"]
        R = max(1, t["renders"])
        ms = [x / R for x in t["ms_per_level"][:L]] + [t["ms_leaf"] / R]
        terms = costmodel.level_terms(n, g, r, max_dwell, q, c, st["regions_per_level"],
                                      st["subdivisions_per_level"], st["leaves"], L)
        kappa, lam = costmodel.fit_lambda(ms, terms)
    v, mg, mr, mB = costmodel.optimum(n, max_dwell, P, lam, q=q, c=c, scheme="sbr")
    return dict(P=P, lam=lam, kappa_ms=kappa, q=q, c=c, g=mg, r=mr, B=mB,
                model_speedup=costmodel.time_exhaustive(n, max_dwell, q, c) / v)


class BatchTuner:
    """Per-frame (g, r, B) for a batch, from measured sweeps of probe frames."""

    def __init__(self, ctx, probes=6, space=None, reps=1):
        self.ctx = ctx
        self.nprobes = probes
        self.space = space
        self.reps = reps
        self.probes = []  # (frame, best config, sweep)

    @staticmethod
    def _key(f):
        return (math.log(f["n"]), math.log(f["max_dwell"]), math.log(f.get("zoom", 1.0)))

    def fit(self, frames):
        import torch
        order = sorted(range(len(frames)), key=lambda k: frames[k]["n"] * frames[k]["max_dwell"])
        m = min(self.nprobes, len(frames))
        picks = sorted({order[int((j + 0.5) * len(order) / m)] for j in range(m)})
        nmax = max(frames[k]["n"] for k in picks)
        scratch = torch.empty(nmax * nmax, dtype=torch.int32, device="cuda:%d" % self.ctx.device)
        for k in picks:
            f = frames[k]
            out = scratch[: f["n"] * f["n"]].view(f["n"], f["n"])
            res = sweep(self.ctx, f["window"], f["n"], f["max_dwell"], self.space, self.reps, out)
            self.probes.append((f, res[0], res))
        del scratch
        return self

    # Largest initial-region side given to a frame of a batch: a batch splits
    # every region of a level into as many chunks as its largest region
    # needs (up to a cap), so a few huge regions cost every frame work items.
    MAX_S0 = 512

    def choose(self, frame):
        """(g, r, B) of the nearest probe (log n, log dwell cap, log zoom).
        The probe's initial-region side s0 = ceil(n / g) carries over, not its
        g, so frames larger or smaller than the probe get regions of the same
        size; s0 is kept at most MAX_S0."""
        key = self._key(frame)
        best = None
        for f, cfg, _ in self.probes:
            pk = self._key(f)
            dist = abs(key[0] - pk[0]) + abs(key[1] - pk[1]) + 0.5 * abs(key[2] - pk[2])
            if best is None or dist < best[0]:
                best = (dist, f, cfg)
        _, f, cfg = best
        n = frame["n"]
        s0 = min(-(-f["n"] // cfg["g"]), self.MAX_S0)
        g = max(1, min(-(-n // s0), n, max(DEFAULT_SPACE["g"])))
        return g, cfg["r"], cfg["B"]

    def summary(self):
        return [dict(n=f["n"], max_dwell=f["max_dwell"], zoom=round(f.get("zoom", 1.0), 2),
                     g=c["g"], r=c["r"], B=c["B"], ms=round(c["ms"], 3))
                for f, c, _ in self.probes]
