"""Writes the stored expected values under tests/golden/ from the oracle only.

Run from the repository root:  python tests/golden/make_golden.py
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle as O  # noqa: E402
from paper_2607_20766_b300 import synth  # noqa: E402


def main():
    a, b = synth.single_pair()
    g = O.grid(a, 0, b, 0, h=0.05, pad=6.5)
    out = {
        "what": "single pair: A 12 atoms (seed 0), B 15 atoms (seed 1), centred, B shifted +1 A in x; "
                "p = 2 sqrt 2, alpha = 2.41798793 / R^2",
        "V_A": O.union_volume_ie(a, 0),                 # 2^12 inclusion-exclusion
        "V_B": O.union_volume_ie(b, 0),                 # 2^15 inclusion-exclusion
        "O_union_AB": O.union_overlap_ie(a, 0, b, 0),    # 2^27 cross series
        "O_union_AA": O.union_overlap_ie(a, 0, a, 0),
        "O_fo_AB": float(O.fo_overlap(a, [0], b, [0])[0]),
        "O_fo_AA": float(O.fo_overlap(a, [0], a, [0])[0]),
        "O_fo_BB": float(O.fo_overlap(b, [0], b, [0])[0]),
        "Z_A": float(O.mixture_mass(a)[0]),
        "Z_B": float(O.mixture_mass(b)[0]),
        "grid_0.05A": {k: float(v) for k, v in g.items()},
    }
    with open(os.path.join(HERE, "single_pair_exact.json"), "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")


if __name__ == "__main__":
    main()
