"""Write paper_2206_02255_gb300/data/boundary_centers.tsv: seeded sample of
points on the boundary of the n = 1024, dwell 512 map of the window
[-1.5, 0.5] x [-1, 1].

A boundary pixel has a dwell below the cap and a 4-neighbour at the cap (it
sits just outside the set, next to a pixel inside it).  The map comes from
the CPU reference only.  The batched and served workloads take their frame
centres from this list (see paper_2206_02255_gb300/inputs.py), which ships
with the package as data; this script stays with the tests because it runs
the CPU reference.

Usage: python tests/golden/make_boundary_centers.py
"""
import os
import random
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
OUT = os.path.join(ROOT, "paper_2206_02255_gb300", "data", "boundary_centers.tsv")
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import oracle  # noqa: E402

WINDOW = (-1.5, 0.5, -1.0, 1.0)
N, MAX_DWELL, SAMPLE, SEED = 1024, 512, 2048, 0


def main():
    m = oracle.render_exhaustive(WINDOW, N, MAX_DWELL)
    inside = m == MAX_DWELL
    nb = np.zeros_like(inside)
    nb[1:, :] |= inside[:-1, :]
    nb[:-1, :] |= inside[1:, :]
    nb[:, 1:] |= inside[:, :-1]
    nb[:, :-1] |= inside[:, 1:]
    ys, xs = np.nonzero(~inside & nb)
    cells = sorted(zip(xs.tolist(), ys.tolist()))
    pick = random.Random(SEED).sample(cells, SAMPLE)
    with open(OUT, "w") as f:
        f.write("# %d of the %d boundary pixels of the n=%d, dwell %d map of window %s\n"
                % (SAMPLE, len(cells), N, MAX_DWELL, WINDOW))
        f.write("# (seed %d); written by make_boundary_centers.py from the CPU reference\n" % SEED)
        f.write("# px\tpy\tcr\tci\tdwell\n")
        for px, py in pick:
            cr, ci = oracle.pixel_to_c(WINDOW, N, px, py)
            f.write("%d\t%d\t%.9g\t%.9g\t%d\n" % (px, py, cr, ci, m[py, px]))
    print("wrote %d of %d boundary pixels" % (SAMPLE, len(cells)))


if __name__ == "__main__":
    main()
