"""Plant plausible mistakes in copies of the CPU reference and check that
the pins reject every one of them (CPU only; the mutants are built from the
source text into a temporary directory and never touch the real build)."""
import os
import shutil
import subprocess

import pytest

import oracle
import oracle_pins

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(os.path.dirname(HERE), "oracle")

# (name, text in oracle.c, replacement)
MUTANTS = [
    ("dropped_factor_two", "float nzi = fmaf(zr + zr, zi, ci);", "float nzi = fmaf(zr, zi, ci);"),
    ("wrong_sign_re", "float t = fmaf(-zi, zi, cr);", "float t = fmaf(zi, zi, cr);"),
    ("escape_le", "float m = fmaf(zr, zr, zi2);\n        int bounded = (flags & ORACLE_ESCAPE_LE) ? (m <= 4.0f) : (m < 4.0f);",
     "float m = fmaf(zr, zr, zi2);\n        int bounded = (flags & ORACLE_ESCAPE_LE) ? (m <= 4.0f) : (m <= 4.0f);"),
    ("check_after_update", "while (d < max_dwell) {\n        float zi2",
     "while (d < max_dwell) {\n        d++; if (d > max_dwell) break;\n        float zi2"),
    ("transposed_operand", "*ci = fmaf((float)py, dy, win->im_min);",
     "*ci = fmaf((float)py, dx, win->im_min);"),
    ("center_sampling", "*cr = fmaf((float)px, dx, win->re_min);",
     "*cr = fmaf((float)px + 0.5f, dx, win->re_min);"),
    ("transposed_layout", "j->out[(size_t)py * j->n + px] = d;",
     "j->out[(size_t)px * j->n + py] = d;"),
    ("floor_child_side", "uint32_t sc = ceil_div(s, j->r);", "uint32_t sc = s / j->r;"),
    ("strict_stop", "if (s > 1 && sc >= j->B) {", "if (s > 1 && sc > j->B) {"),
    ("clip_to_image_not_parent", "uint32_t cw = (uint32_t)((uint64_t)x0 + w - cx);",
     "uint32_t cw = (uint32_t)((uint64_t)j->n - cx);"),
    ("fill_skips_perimeter", "put(j, x, y, first);",
     "if (x != x0 && y != y0) put(j, x, y, first);"),
    ("border_misses_right_column", "uint32_t step = edge_row ? 1u : (w > 1 ? w - 1 : 1u);",
     "uint32_t step = edge_row ? 1u : w;"),
    ("floor_initial_side", "uint32_t s0 = ceil_div(n, g);", "uint32_t s0 = n / g ? n / g : 1;"),
    # the double-precision (deep-zoom) functions
    ("dropped_factor_two_64", "double nzi = fma(zr + zr, zi, ci);", "double nzi = fma(zr, zi, ci);"),
    ("wrong_sign_re_64", "double t = fma(-zi, zi, cr);", "double t = fma(zi, zi, cr);"),
    ("escape_le_64", ": (m < 4.0);", ": (m <= 4.0);"),
    ("state_in_float_64", "double zr = 0.0, zi = 0.0;", "float zr = 0.0f, zi = 0.0f;"),
    ("transposed_operand_64", "*ci = fma((double)py, dy, win->im_min);",
     "*ci = fma((double)py, dx, win->im_min);"),
    ("c_rounded_to_float_64", "*cr = fma((double)px, dx, win->re_min);",
     "*cr = (float)fma((double)px, dx, win->re_min);"),
    ("center_sampling_64", "*ci = fma((double)py, dy, win->im_min);",
     "*ci = fma((double)py + 0.5, dy, win->im_min);"),
    ("map_in_float_64", "return oracle_dwell64(cr, ci, max_dwell, flags);",
     "return oracle_dwell((float)cr, (float)ci, max_dwell, flags);"),
    # the float-float functions
    ("ff_add_drops_lo", "float w = e + (x.lo + y.lo);", "float w = e;"),
    ("ff_two_sum_sign", "float e = (x.hi - (s - bb)) + (y.hi - bb);",
     "float e = (x.hi - (s - bb)) - (y.hi - bb);"),
    ("ff_fast_two_sum_error", "r.lo = b - (r.hi - a);", "r.lo = b - r.hi;"),
    ("ff_mul_drops_cross_term", "e = fmaf(x.lo, y.hi, e);", "e = e + 0.0f;"),
    ("ff_sqr_single_cross_term", "e = fmaf(x.hi + x.hi, x.lo, e);", "e = fmaf(x.hi, x.lo, e);"),
    ("ff_split_drops_lo", "r.lo = (float)(v - (double)r.hi);", "r.lo = 0.0f;"),
    ("ff_wrong_sign_re", "ff_t neg_zi2 = {-zi2.hi, -zi2.lo};", "ff_t neg_zi2 = {zi2.hi, zi2.lo};"),
    ("ff_test_uses_lo", "float m = zr2.hi + zi2.hi;", "float m = zr2.hi + zi2.lo;"),
    ("ff_escape_le", "float m = zr2.hi + zi2.hi;\n        int bounded = (flags & ORACLE_ESCAPE_LE) ? (m <= 4.0f) : (m < 4.0f);",
     "float m = zr2.hi + zi2.hi;\n        int bounded = (flags & ORACLE_ESCAPE_LE) ? (m <= 4.0f) : (m <= 4.0f);"),
    ("ff_not_doubled", "ff_t p2 = {p.hi + p.hi, p.lo + p.lo};", "ff_t p2 = {p.hi + p.hi, p.lo};"),
]


def _build_mutant(tmpdir, name, old, new):
    src = open(os.path.join(SRC, "oracle.c")).read()
    assert src.count(old) == 1, "mutation anchor must occur exactly once: %r" % old
    d = os.path.join(tmpdir, name)
    os.makedirs(d)
    shutil.copy(os.path.join(SRC, "oracle.h"), d)
    with open(os.path.join(d, "oracle.c"), "w") as f:
        f.write(src.replace(old, new))
    lib = os.path.join(d, "liboracle_%s.so" % name)
    subprocess.run([os.environ.get("CC", "gcc"), "-std=c11", "-O2", "-ffp-contract=off",
                    "-fPIC", "-shared", "-o", lib, os.path.join(d, "oracle.c"),
                    "-lpthread", "-lm"], check=True)
    return oracle.Oracle(lib)


@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pins_reject_mutant(tmp_path, name, old, new):
    orc = _build_mutant(str(tmp_path), name, old, new)
    failed = []
    for pin in oracle_pins.ALL_PINS:
        try:
            pin(orc)
        except AssertionError:
            failed.append(pin.__name__)
            break
    assert failed, "no pin caught the planted mistake %s" % name
