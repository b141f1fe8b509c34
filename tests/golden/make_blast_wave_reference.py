"""Writes blast_wave_ref1600.txt: density of the interacting blast waves
(Sec. 5.4; Woodward-Colella initial data, reflecting ends, t = 0.038) on a
1600-cell grid, computed only with the oracle (FP64 TENO-D GKS, CFL 0.5).
It is the fine-grid reference against which the 400-cell float32 and
float64 runs are judged: averaged over groups of 4 cells it gives the
400-cell cell averages up to the fine grid's own (much smaller) error.

Run from the repository root:  python tests/golden/make_blast_wave_reference.py
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle as O  # noqa: E402
from paper_2309_10534_gb300 import workloads as WL  # noqa: E402

N = 1600


def main():
    s = WL.blast_wave(N)
    P = O.make_problem(1, N, **s.problem_kwargs())
    W, steps, t, nfb = O.run(P, s.W, s.t_end)
    with open(os.path.join(HERE, "blast_wave_ref1600.txt"), "w") as f:
        f.write(f"# oracle density, blast waves (Sec. 5.4), {N} cells, t = {t:.17g}, "
                f"{steps} CFL steps, {nfb} positivity fallbacks\n")
        for r in W[0, 0]:
            f.write(f"{r:.17g}\n")


if __name__ == "__main__":
    main()
