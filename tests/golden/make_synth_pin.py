"""Writes synth_pin.txt, the determinism pin of the seeded input generator.

The generator (synth/) holds none of the solver arithmetic; this pin fixes
its output so that a change to it cannot silently change every input and
every expected value of the tests.  Integer arrays (patterns) are pinned by
SHA-256 of their little-endian int32 bytes; floating-point arrays by their
values written with 17 significant digits, compared at 1e-13 relative, since
numpy's exp, log and cos may differ by an ulp between machines.

Run from the repository root: python tests/golden/make_synth_pin.py
"""
import hashlib
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)
import synth  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "synth_pin.txt")


def cases():
    """(name, dict of arrays) for each pinned generator call."""
    yield "pressure_7pt(Grid(8,6,4),1,kz_scale=0.1)", synth.pressure_7pt(synth.Grid(8, 6, 4), 1, kz_scale=0.1)
    yield "black_oil_bsr3(Grid(4,3,3),1)", synth.black_oil_bsr3(synth.Grid(4, 3, 3), 1)
    yield "pressure_7pt(Grid(4,3,2),1)", synth.pressure_7pt(synth.Grid(4, 3, 2), 1)
    yield "black_oil_bsr3(Grid(3,2,2),1)", synth.black_oil_bsr3(synth.Grid(3, 2, 2), 1)
    yield "x_true(24,1)", {"x": synth.x_true(24, 1)}


# float arrays are written out only for the small calls
VALUES = ("pressure_7pt(Grid(4,3,2),1)", "black_oil_bsr3(Grid(3,2,2),1)", "x_true(24,1)")


def lines():
    for name, d in cases():
        for key in sorted(d):
            a = np.asarray(d[key])
            if a.dtype.kind in "iu":
                h = hashlib.sha256(a.astype("<i4").tobytes()).hexdigest()
                yield "%s %s sha256 %s" % (name, key, h)
            elif a.dtype.kind == "f" and a.ndim == 1 and name in VALUES:
                yield "%s %s values %s" % (name, key, " ".join(repr(float(v)) for v in a))


if __name__ == "__main__":
    with open(OUT, "w") as f:
        f.write("# determinism pin of synth/ (written by make_synth_pin.py; see its docstring)\n")
        for ln in lines():
            f.write(ln + "\n")
    print(OUT)
