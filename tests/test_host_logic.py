"""Host-side rules of the package that need no GPU: which frames render in
double precision, and the deep-zoom inputs."""
from paper_2206_02255_gb300 import ask, inputs


def test_fp64_threshold_is_zoom_1e4():
    # zoom z over the 2 x 2 window gives a window 2 / z wide
    for zoom, want in [(1.0, False), (9.9e3, False), (1.01e4, True), (1e9, True)]:
        hw = 1.0 / zoom
        assert ask.needs_fp64((-0.5 - hw, -0.5 + hw, 0.1 - hw, 0.1 + hw)) is want, zoom
    # the wider side decides: a window narrow in one direction only stays in float
    assert not ask.needs_fp64((0.0, 1.0, 0.0, 1e-6))
    # the binding's window structures are accepted too
    assert not ask.needs_fp64(ask.Window(-1.5, 0.5, -1.0, 1.0))
    assert ask.needs_fp64(ask.Window64(0.3, 0.3 + 2.0 ** -30, 0.1, 0.1 + 2.0 ** -30))


def test_batch_and_serving_workloads_stay_in_single_precision():
    """Their zooms are drawn from [1, 1e4], so no frame takes the FP64 path
    and their measurements are of the single-precision kernels."""
    assert not any(ask.needs_fp64(f["window"]) for f in inputs.batch_frames())
    assert not any(ask.needs_fp64(r["window"]) for r in inputs.serving_requests())


def test_deep_inputs():
    for name, re0, im0, w, md in inputs.DEEP_SPOTS:
        win, m = inputs.deep_window(name)
        assert m == md and ask.needs_fp64(win)
        # power-of-two widths from the listed corner: exact in double
        assert win[1] - win[0] == w and win[3] - win[2] == w
    a = inputs.deep_frames(8, 3)
    assert a == inputs.deep_frames(8, 3)            # seeded
    assert all(ask.needs_fp64(f["window"]) for f in a)
    assert all(256 <= f["n"] <= 2048 and 512 <= f["max_dwell"] <= 4096 for f in a)


def test_window64_conversion():
    w = ask._window64(ask.Window(-1.5, 0.5, -1.0, 1.0))
    assert (w.re_min, w.re_max, w.im_min, w.im_max) == (-1.5, 0.5, -1.0, 1.0)
    w = ask._window64((0.1, 0.1 + 2.0 ** -40, 0.2, 0.2 + 2.0 ** -40))
    assert w.re_max - w.re_min == 2.0 ** -40      # kept in double
