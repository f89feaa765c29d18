"""Write the stored oracle values used by the regression tests.

Calls only the CPU oracle (and the seeded input generator).  Run from the repo root:
    python tests/golden/make_golden.py
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from paper_2307_09226_gb300 import synth  # noqa: E402


def main():
    f = synth.config1()
    cube = oracle.cube_literal(f.radar, f.pixels)
    rng = np.random.default_rng(20230718)
    ent = np.stack([rng.integers(0, f.radar.V, 24), rng.integers(0, f.radar.Ns, 24),
                    rng.integers(0, f.radar.L, 24)], 1)
    with open(os.path.join(HERE, "config1_entries.txt"), "w") as fh:
        fh.write("# Oracle (literal FP64 sum, Eq. 2) entries of the 32x32-pixel frame, seed 1:\n")
        fh.write("# M=2 N=4 Ns=64 L=32, lam=3.9 mm, mu=30 MHz/us, Fs=10 MHz, T_b=60 us, T_slow=M T_b.\n")
        fh.write("# columns: v n l re im ; written by tests/golden/make_golden.py\n")
        for (v, n, l) in ent:
            z = cube[v, n, l]
            fh.write(f"{v} {n} {l} {z.real:.17e} {z.imag:.17e}\n")
        fh.write(f"# norm {np.linalg.norm(cube.ravel()):.17e}\n")


if __name__ == "__main__":
    main()
