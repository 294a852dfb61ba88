"""Write synth/cell58.txt: the seeded 58-atom CHNO cell (run: python -m synth.make_cell)."""
import os

import numpy as np

from synth.crystal import CELL, TYPE_NAMES, search_unit_cell

if __name__ == "__main__":
    types, xyz, dmin = search_unit_cell(seed=1706)
    path = os.path.join(os.path.dirname(__file__), "cell58.txt")
    with open(path, "w") as f:
        f.write("# seeded synthetic C5H8N4O12 x2 cell, a=b=%.2f c=%.2f A; search seed 1706\n" % (CELL[0], CELL[2]))
        f.write("# smallest non-bonded contact %.4f A; columns: type(0=C,1=H,2=N,3=O) x y z (A)\n" % dmin)
        for t, p in zip(types, xyz):
            f.write("%d %.10f %.10f %.10f  # %s\n" % (t, p[0], p[1], p[2], TYPE_NAMES[t]))
    print("wrote", path, "contact", dmin)
