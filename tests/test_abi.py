"""The C-ABI library builds, loads and exports every entry point that
include/ask.h declares; host-only entry points work without a GPU."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    text = open(os.path.join(ROOT, "include", "ask.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[a-z_][a-z0-9_]*\s*\**\s*(ask_[a-z0-9_]+)\s*\(", text, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("ask_ctx_create", "ask_ctx_destroy", "ask_render", "ask_render_host",
                 "ask_reserve", "ask_check", "ask_plan_levels", "ask_status_str",
                 "ask_last_error", "ask_version"):
        assert must in names


def test_binding_constants_match_the_header(asklib):
    """Every ASK_FLAG_* and ask_status value of the header has the same
    value in the Python binding."""
    text = open(os.path.join(ROOT, "include", "ask.h")).read()
    flags = dict(re.findall(r"#define\s+ASK_(FLAG_[A-Z0-9_]+)\s+(\d+)u", text))
    assert len(flags) >= 10
    for name, v in flags.items():
        assert getattr(asklib, name) == int(v), name
    statuses = re.findall(r"ASK_(E[A-Z]+|OK)\s*=\s*(\d+)", text)
    assert len(statuses) == 8
    for name, v in statuses:
        assert getattr(asklib, name) == int(v), name


def test_library_exports_every_declared_symbol(asklib):
    lib = ctypes.CDLL(asklib.lib_path())
    for name in declared_functions():
        assert hasattr(lib, name), name
    assert set(declared_functions()) <= set(asklib.SIGNATURES)


def test_host_only_entry_points(asklib):
    assert "sm_103a" in asklib.version()
    assert asklib.status_str(asklib.EINVAL) == "invalid argument"
    assert asklib.status_str(99) == "unknown status"
    # n = 1024, g = 16: s0 = 64; r = 2: 32 >= B = 32 splits once; 16 < 32 stops
    sides, regs = asklib.plan_levels(1024, 16, 2, 32)
    assert sides == [64, 32] and regs == [256, 1024]
    # n = 16384, g = 32, r = 4, B = 16: 512, 128, 32, (8 < 16 stops)
    sides, regs = asklib.plan_levels(16384, 32, 4, 16)
    assert sides == [512, 128, 32] and regs == [32 ** 2, 128 ** 2, 512 ** 2]
    # ragged: n = 5, g = 2, r = 2, B = 1 -> sides 3, 2, 1; per axis 2, 3, 5 intervals
    sides, regs = asklib.plan_levels(5, 2, 2, 1)
    assert sides == [3, 2, 1] and regs == [4, 9, 25]
    for bad in [(0, 1, 2, 1), (8, 0, 2, 1), (8, 9, 2, 1), (8, 2, 1, 1), (8, 2, 2, 0), (65537, 1, 2, 1)]:
        with pytest.raises(asklib.AskError):
            asklib.plan_levels(*bad)


def test_plan_matches_oracle_tree(asklib, orc):
    """The library's level plan bounds the oracle's region counts, and with
    fills disabled (the full tree) the bound is reached exactly."""
    win = (-2.0, 0.6, -1.25, 1.25)
    for n, g, r, B in [(5, 2, 2, 1), (37, 3, 2, 4), (64, 4, 2, 8), (97, 5, 4, 3), (50, 2, 3, 2)]:
        sides, regs = asklib.plan_levels(n, g, r, B)
        _, st = orc.render_ms(win, n, 40, g, r, B, flags=2, threads=1)
        assert st["levels"] == len(sides)
        assert st["regions_per_level"] == regs


def test_context_needs_a_gb300():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2206_02255_gb300 import ask, build
    build.build()
    with pytest.raises(ask.AskError) as e:
        ask.Context(0)
    assert e.value.status == ask.EUNSUPPORTED
