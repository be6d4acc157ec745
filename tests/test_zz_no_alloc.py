"""The allocation-free ASK entry point, ``ask_render_noalloc``.

It exists for callers that may not call cudaMalloc (a frame loop or host
callback where allocating, and the synchronisation that may come with it,
is not allowed; a plug-in whose host application owns all device memory; a
service held to a fixed memory budget).  Its scratch is a fixed set of
device arrays shared by every call, so this test renders several calls in a
row on that shared scratch and checks each against the CPU oracle and
against the ordinary ``ask_render``: the second call starts from whatever
the first left there, and the third, smaller call follows a larger one, so
leftover table entries and counters of a bigger plan must not leak into it.

This file is collected last on purpose, so a run that stops at the first
failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest

from paper_2206_02255_gb300 import inputs

pytestmark = pytest.mark.gpu


def _reference(ctx, asklib, window, n, M, p):
    import torch
    out = ctx.render("ask", window, n, M, p)
    torch.cuda.synchronize()
    return out.cpu().numpy().view(np.uint32).copy()


def test_noalloc_matches_oracle_and_ask_render_in_a_row(asklib, orc):
    import torch
    cases = [
        (inputs.WINDOW_PAPER, 1024, 512, (16, 2, 32), (16, 16)),
        (inputs.WINDOW_WIDE, 2047, 700, (7, 4, 8), (8, 8)),
        # smaller than the call before it, on the same stream
        (inputs.WINDOW_WIDE, 1024, 300, (16, 2, 16), (16, 16)),
    ]
    ctx = asklib.Context(0)
    try:
        for window, n, M, (g, r, B), blk in cases:   # calls in a row on the shared scratch
            p = asklib.make_params(g, r, B, blk)
            want, _ = orc.render_ms(window, n, M, g, r, B)
            ref = _reference(ctx, asklib, window, n, M, p)
            assert np.array_equal(ref, want)
            out = torch.full((n, n), -1, dtype=torch.int32, device="cuda")
            asklib.render_noalloc(window, n, M, p, out)
            torch.cuda.synchronize()
            got = out.cpu().numpy().view(np.uint32)
            bad = int((got != want).sum())
            assert bad == 0, "%d pixels differ from the oracle (n=%d)" % (bad, n)
            assert np.array_equal(got, ref)
    finally:
        ctx.close()


def test_noalloc_rejects_requests_beyond_its_scratch(asklib):
    import torch
    from paper_2206_02255_gb300.ask import Window, lib
    out = torch.full((16, 16), 5, dtype=torch.int32, device="cuda")
    # n = 16384 with B = 8 needs 2048^2 = 4 Mi leaf slots, more than 2^20
    p = asklib.make_params(32, 2, 8, (16, 16))
    st = lib().ask_render_noalloc(ctypes.byref(Window(*inputs.WINDOW_PAPER)), 16384, 100,
                                  ctypes.byref(p), ctypes.c_void_p(out.data_ptr()), None)
    assert st == asklib.ECAPACITY
    assert "fixed scratch" in asklib.status_str(st)
    bad = asklib.make_params(16, 2, 32, (16, 16), flags=asklib.FLAG_COUNT)
    st = lib().ask_render_noalloc(ctypes.byref(Window(*inputs.WINDOW_PAPER)), 16, 100,
                                  ctypes.byref(bad), ctypes.c_void_p(out.data_ptr()), None)
    assert st == asklib.EINVAL
    torch.cuda.synchronize()
    assert bool((out == 5).all())
