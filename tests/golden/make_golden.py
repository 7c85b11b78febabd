"""Writes the stored expected values under tests/golden/ that are not printed
in the paper.  It calls only ``oracle/`` (and the seeded input generators),
never the CUDA path.

    python tests/golden/make_golden.py
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import closed_forms  # noqa: E402


def c1_lattice_green():
    """129^2 grid, h = 1/128, f = 1, hbar = 0.01, source at node (64, 64):
    the exact discrete solution is the mirror-image sum of the lattice
    Green's function (closed form, Sec. 3.2 Green's functions, discrete
    analogue).  Stores S at a fixed set of nodes."""
    dims, h, hbar = (129, 129), 1.0 / 128, 0.01
    phi = closed_forms.image_phi(dims, h, hbar, 1.0, (64, 64))
    S = -hbar * np.log(phi)
    nodes = [(64, 64), (65, 64), (64, 66), (70, 70), (96, 64), (128, 64),
             (128, 128), (0, 0), (0, 128), (10, 100), (127, 3), (64, 0)]
    return {
        "citation": "Sec. 3.2 Eqs. (GreensFunction2D), (SfromPhi); Sec. 6 Eq. (sparse-system) with half-cell zero-flux faces; discrete Green's function by the Laplace transform of the lattice heat kernel plus mirror images",
        "dims": list(dims), "h": h, "hbar": hbar, "f": 1.0, "source": [64, 64],
        "nodes": nodes, "S": [float(S[y, x]) for (x, y) in nodes],
    }


def main():
    out = os.path.join(HERE, "c1_closed_form.json")
    with open(out, "w") as fh:
        json.dump(c1_lattice_green(), fh, indent=1)
    print("wrote", out)


if __name__ == "__main__":
    main()
