"""Writes the stored expected values under tests/golden/ that come from the
oracle (this script calls nothing but ``oracle/``).

    python tests/golden/make_golden.py
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import fourier  # noqa: E402
from oracle.tableau import imex_tableau  # noqa: E402


def main():
    cfl, cfl_imex = {}, {}
    for N in range(5):
        t = imex_tableau(N)
        for family in (["gl", "gll"] if N > 0 else ["gl"]):
            cfl[f"{N}_{family}"] = fourier.cfl_number(N, family)
            cfl_imex[f"{N}_{family}"] = fourier.cfl_number(N, family, tableau=(t.Ae, t.be))
    out = {
        "source": "oracle.fourier.cfl_number: von Neumann analysis of cRK-FR for "
                  "linear advection (Sec. 5, under Eq. time.step.2d); readings in oracle/__init__.py; "
                  "cfl_imex: the same for the explicit part of the IMEX tableau used with a source",
        "cfl": cfl,
        "cfl_imex": cfl_imex,
    }
    with open(os.path.join(HERE, "oracle_cfl.json"), "w") as fh:
        json.dump(out, fh, indent=2)
        fh.write("\n")


if __name__ == "__main__":
    main()
