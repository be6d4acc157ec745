"""Render server with continuous batching.

Requests (window, n, dwell cap) arrive over time.  The server keeps a queue
of arrived requests and a fixed number of batch slots, each a context (its
own region tables on the device).  Whenever a slot
is free it admits queued requests, oldest first, while their dwell buffers
fit in the memory budget, and renders them as one batch (one launch chain
for every frame of the batch, region queues on the device).  Batches render
one after another on one compute stream, since each launch chain fills the
whole GPU; the maps of a batch are copied to pinned host memory on one copy
stream while the next batch renders.  (The copies of all slots share that
stream: device-to-host copies of two slots running at once on two streams
moved 65-80 GB/s together against 190 GB/s for one stream alone.)
Requests that arrive
while batches run wait for the next free slot.  A request's latency runs
from its arrival to the moment its map is in host memory.

Batching pays only when requests queue up.  A slot admits a batch only
when at least ``batch_min`` requests wait; otherwise it takes one request
and dispatches it through the single-frame call (no frame table to build
and copy), its map copied right behind its render, so a lightly loaded
server adds nothing to the per-frame path.  While work is in flight the server polls its events without
sleeping; it sleeps only when it is idle until the next arrival.

Requests zoomed past ``ask.FP64_ZOOM`` are rendered in double precision
(``ask_render64``) on the same compute stream, after their batch's
single-precision frames.

The baseline, :func:`serve_per_frame`, renders the same requests one at a
time, in arrival order, with the single-frame ASK call.
"""
import time

from . import ask


class PinnedPool:
    """Pinned host buffers by power-of-two size class, reused across
    requests: pinning memory is slow, so a served path allocates once and
    recycles (a buffer goes back when its request's result is consumed).
    Buffers are carved from pinned slabs of at least 1 GiB: device-to-host
    copies into many separately pinned buffers ran at 48-71 GB/s in some
    passes, into slices of one pinned allocation at a steady 190 GB/s."""

    SLAB_BYTES = 1 << 30

    def __init__(self):
        self.free = {}
        self.slabs = []
        self.off = 0

    def _carve(self, cls):
        import torch
        if not self.slabs or self.off + cls > self.slabs[-1].numel():
            self.slabs.append(torch.empty(max(self.SLAB_BYTES, cls), dtype=torch.uint8,
                                          pin_memory=True))
            self.off = 0
        buf = self.slabs[-1][self.off:self.off + cls]
        self.off += cls
        return buf

    def get(self, n):
        import torch
        nbytes = 4 * n * n
        cls = 1 << max(12, (nbytes - 1).bit_length())
        lst = self.free.get(cls)
        buf = lst.pop() if lst else self._carve(cls)
        return buf, buf[:nbytes].view(torch.int32).view(n, n)

    def put(self, buf):
        self.free.setdefault(buf.numel(), []).append(buf)

    def reserve(self, sides, per_class=2):
        """Carve `per_class` buffers of every size class that maps of the
        given sides need, so that serving them allocates no slab (pinning
        1 GiB takes about 75 ms)."""
        need = {}
        for n in sides:
            cls = 1 << max(12, (4 * n * n - 1).bit_length())
            need[cls] = per_class
        for cls, k in sorted(need.items()):
            have = len(self.free.get(cls, []))
            for _ in range(max(0, k - have)):
                self.put(self._carve(cls))


class DevicePool:
    """Device dwell buffers by power-of-two size class, reused across
    requests like the pinned pool: in steady state a server allocates
    nothing, so no allocation (and the device synchronisation that
    cudaMalloc can bring) falls inside a batch's lifetime.  Class sizes are
    multiples of 4 KiB, so every view starts 16-byte aligned."""

    def __init__(self, device=0):
        self.device = device
        self.free = {}

    def get(self, n):
        import torch
        nbytes = 4 * n * n
        cls = 1 << max(12, (nbytes - 1).bit_length())
        lst = self.free.get(cls)
        buf = lst.pop() if lst else torch.empty(cls, dtype=torch.uint8,
                                                device="cuda:%d" % self.device)
        return buf, buf[:nbytes].view(torch.int32).view(n, n)

    def put(self, buf):
        self.free.setdefault(buf.numel(), []).append(buf)


class Request:
    __slots__ = ("id", "t", "window", "n", "max_dwell", "g", "r", "B", "out", "host",
                 "hbuf", "dbuf", "t_done", "event")

    def __init__(self, d, g, r, B):
        self.id = d["id"]
        self.t = d["t"]
        self.window = d["window"]
        self.n = d["n"]
        self.max_dwell = d["max_dwell"]
        self.g, self.r, self.B = g, r, B
        self.out = self.host = self.hbuf = self.dbuf = self.event = None
        self.t_done = None

    @property
    def nbytes(self):
        return 4 * self.n * self.n


def percentile(xs, q):
    xs = sorted(xs)
    if not xs:
        return float("nan")
    k = (len(xs) - 1) * q / 100.0
    lo, hi = int(k), min(int(k) + 1, len(xs) - 1)
    return xs[lo] + (xs[hi] - xs[lo]) * (k - lo)


class Server:
    """Continuous-batching server over `slots` contexts on one device."""

    def __init__(self, device=0, slots=2, budget_bytes=40 * 2 ** 30, max_frames=256, pool=None,
                 keep=True, dpool=None, batch_min=4):
        import torch
        self.device = device
        self.pool = pool if pool is not None else PinnedPool()
        self.dpool = dpool if dpool is not None else DevicePool(device)
        self.keep = keep  # keep results on the requests; else recycle at completion
        self.budget = budget_bytes
        self.max_frames = max_frames
        # a slot batches only when at least batch_min requests wait; with
        # fewer, it takes one through the single-frame call (a short burst
        # renders faster as single frames back to back than as a batch)
        self.batch_min = batch_min
        self.ctxs = [ask.Context(device) for _ in range(slots)]
        self.compute = torch.cuda.Stream(device=device)
        self.copy = torch.cuda.Stream(device=device)  # the copies of every slot
        self.busy = [None] * slots       # list of requests in flight per slot
        self.used = 0                    # bytes of dwell buffers in flight
        self.single_dispatches = 0       # slots that took one request alone
        self.batch_dispatches = 0

    def close(self):
        for c in self.ctxs:
            c.close()

    def _start(self, slot, reqs):
        import torch
        c, s = self.compute, self.copy
        with torch.cuda.stream(c):
            for q in reqs:
                q.dbuf, q.out = self.dpool.get(q.n)
                q.hbuf, q.host = self.pool.get(q.n)
            if len(reqs) == 1:
                # nothing queued behind it: the single-frame call
                render_one(self.ctxs[slot], reqs[0], c)
                self.single_dispatches += 1
            else:
                frames = [dict(window=q.window, n=q.n, max_dwell=q.max_dwell, g=q.g, r=q.r,
                               B=q.B, out=q.out) for q in reqs if not ask.needs_fp64(q.window)]
                if frames:
                    self.ctxs[slot].render_batch(frames, stream=c)
                for q in reqs:
                    if ask.needs_fp64(q.window):
                        render_one(self.ctxs[slot], q, c)
                self.batch_dispatches += 1
            if len(reqs) == 1:
                # a lone request's map is copied right behind its render on
                # the compute stream, as the per-frame path does
                reqs[0].host.copy_(reqs[0].out, non_blocking=True)
                ev = torch.cuda.Event()
                ev.record(c)
            else:
                rendered = torch.cuda.Event()
                rendered.record(c)
        if len(reqs) > 1:
            s.wait_event(rendered)
            with torch.cuda.stream(s):
                for q in reqs:
                    q.host.copy_(q.out, non_blocking=True)
                ev = torch.cuda.Event()
                ev.record(s)
        for q in reqs:
            q.event = ev
        self.busy[slot] = reqs

    def run(self, requests, idle_spin_s=0.0003):
        """Serve `requests` (sorted by arrival time t, seconds from start) in
        real time; returns them with t_done set (seconds from start).  While
        batches are in flight the loop polls without sleeping; when nothing
        is in flight and nothing waits, it sleeps until `idle_spin_s` before
        the next arrival and spins from there."""
        pending = []
        k = 0
        t0 = time.perf_counter()
        done = 0
        while done < len(requests):
            now = time.perf_counter() - t0
            while k < len(requests) and requests[k].t <= now:
                pending.append(requests[k])
                k += 1
            # retire finished batches
            for slot, reqs in enumerate(self.busy):
                if reqs is not None and reqs[0].event.query():
                    tn = time.perf_counter() - t0
                    for q in reqs:
                        q.t_done = tn
                        self.used -= q.nbytes
                        self.dpool.put(q.dbuf)
                        q.out = q.dbuf = None
                        if not self.keep:
                            self.pool.put(q.hbuf)
                            q.hbuf = q.host = None
                    done += len(reqs)
                    self.busy[slot] = None
            # admit queued requests into free slots while they fit the budget
            for slot in range(len(self.ctxs)):
                if self.busy[slot] is not None or not pending:
                    continue
                take, mem = [], 0
                limit = self.max_frames if len(pending) >= self.batch_min else 1
                while pending and len(take) < limit and \
                        self.used + mem + pending[0].nbytes <= self.budget:
                    mem += pending[0].nbytes
                    take.append(pending.pop(0))
                if take:
                    self.used += mem
                    self._start(slot, take)
            if k < len(requests) and not pending and all(b is None for b in self.busy):
                # idle until the next arrival
                wait = requests[k].t - (time.perf_counter() - t0) - idle_spin_s
                if wait > 0:
                    time.sleep(min(wait, 0.01))
        return requests


def render_one(ctx, q, stream):
    """Render request q alone into q.out on `stream`: single-frame ASK, in
    double precision past ask.FP64_ZOOM."""
    p = ask.make_params(q.g, q.r, q.B)
    if ask.needs_fp64(q.window):
        ctx.render64("ask", q.window, q.n, q.max_dwell, p, out=q.out, stream=stream)
    else:
        ctx.render("ask", q.window, q.n, q.max_dwell, p, out=q.out, stream=stream)


def serve_per_frame(ctx, requests, idle_spin_s=0.0003, pool=None, keep=True, dpool=None):
    """Baseline: one request at a time in arrival order, single-frame ASK,
    map copied to pinned host memory; returns requests with t_done set.  It
    waits for an arrival as the server does: asleep until `idle_spin_s`
    before it, spinning from there."""
    import torch
    pool = pool if pool is not None else PinnedPool()
    dpool = dpool if dpool is not None else DevicePool(ctx.device)
    s = torch.cuda.Stream(device=ctx.device)
    t0 = time.perf_counter()
    for q in requests:
        wait = q.t - (time.perf_counter() - t0) - idle_spin_s
        if wait > 0:
            time.sleep(wait)
        while time.perf_counter() - t0 < q.t:
            pass
        with torch.cuda.stream(s):
            q.dbuf, q.out = dpool.get(q.n)
            q.hbuf, q.host = pool.get(q.n)
            render_one(ctx, q, s)
            q.host.copy_(q.out, non_blocking=True)
        s.synchronize()
        q.t_done = time.perf_counter() - t0
        dpool.put(q.dbuf)
        q.out = q.dbuf = None
        if not keep:
            pool.put(q.hbuf)
            q.hbuf = q.host = None
    return requests


def summarize(requests):
    lat = [1e3 * (q.t_done - q.t) for q in requests]
    px = sum(q.n * q.n for q in requests)
    span = max(q.t_done for q in requests) - min(q.t for q in requests)
    return dict(requests=len(requests), p50_ms=percentile(lat, 50), p99_ms=percentile(lat, 99),
                max_ms=max(lat), gpix_s=px / span / 1e9, span_s=span)
