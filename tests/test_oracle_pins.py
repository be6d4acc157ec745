"""The CPU reference against its pins (see ``oracle_pins``); no GPU."""
import pytest

import oracle_pins


@pytest.mark.parametrize("pin", oracle_pins.ALL_PINS, ids=lambda f: f.__name__)
def test_pin(orc, pin):
    pin(orc)


def test_c0_mismatch_reported(orc):
    """Mariani-Silver fills are a heuristic: report, never hide, how many
    pixels of the n = 1024 configuration differ from the exhaustive map."""
    W = oracle_pins.C0_WINDOW
    ex = orc.render_exhaustive(W, 1024, 512)
    ms, st = orc.render_ms(W, 1024, 512, 16, 2, 32)
    mism = int((ex != ms).sum())
    print("C0 subdivision-vs-exhaustive mismatch: %d pixels (%.3g%%)"
          % (mism, 100.0 * mism / ex.size))
    assert st["fill_pixels"] + st["leaf_pixels"] == ex.size
