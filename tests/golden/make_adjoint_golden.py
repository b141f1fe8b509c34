"""Writes adjoint_smooth24.txt: the FP64 CPU reference gradient of the
adjoint tests, computed only with the oracle (central finite differences).

Problem: seeded smooth periodic state on [0, 1]^2, 24 x 24 cells
(workloads.random_smooth_2d, seed 5, wave numbers 1..2), collision-free flux
(tau = 0, the paper's setting for smooth flow, Sec. 5.1 and 5.5), 6 S2O4
steps of fixed dt = 0.01 (CFL 0.43).  Parameter: a density perturbation
delta rho_ij at fixed (u, v, p) in every cell.  Objective
J = sum over cells of rho^2 dx dy after the 6 steps.

TENO-D's stencil choice is piecewise constant in the data, so the discrete
map has (rare) jumps where a choice flips; the adjoint differentiates with
the forward pass's choice held fixed.  Each gradient component is therefore
taken at two step sizes, 1e-6 and 2.5e-7; where the two agree to 1e-6 of
the largest component no choice flipped within the probe, and the value is
the derivative of the map with its choices fixed.  Columns: component index
(j * 24 + i, j the y index), dJ/d(delta rho) at h = 1e-6, at h = 2.5e-7,
and 1 where the oracle's TENO-D selection trace (every stencil choice of
the run, Eqs. 4.7 and 4.12) differs between the +h and -h runs at either
step size, else 0: a component whose two step sizes disagree must have a
flipped choice inside its probe.

Run from the repository root:  python tests/golden/make_adjoint_golden.py
"""
import multiprocessing as mp
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

N, STEPS, DT, SEED, KMAX = 24, 6, 0.01, 5, 2
HS = (1e-6, 2.5e-7)
GAMMA = 1.4


def primitives():
    from paper_2309_10534_gb300 import workloads as WL
    W = WL.random_smooth_2d(N, N, seed=SEED, kmax=KMAX)
    rho = W[0]
    u, v = W[1] / rho, W[2] / rho
    p = (GAMMA - 1.0) * (W[3] - 0.5 * rho * (u * u + v * v))
    return rho, u, v, p


def objective(delta, traced=False):
    import oracle as O
    from paper_2309_10534_gb300 import workloads as WL
    rho, u, v, p = primitives()
    P = O.make_problem(2, N, N, bc=("periodic",) * 4, tau="zero")
    W0 = WL.conserved_2d(rho + delta, u, v, p, GAMMA)

    def run():
        W = W0
        for _ in range(STEPS):
            W = O.step(P, W, DT)
        return float((W[0] ** 2).sum() / (N * N))

    return O.trace_selections(run) if traced else run()


def flipped(k, h):
    """True where the selection traces of the runs at +h and -h in
    component k differ."""
    e = np.zeros((N, N))
    e.flat[k] = h
    _, tp = objective(e, traced=True)
    _, tm = objective(-e, traced=True)
    return tp.size != tm.size or not np.array_equal(tp, tm)


def component(k):
    out, flip = [], False
    for h in HS:
        e = np.zeros((N, N))
        e.flat[k] = h
        (jp, tp), (jm, tm) = objective(e, traced=True), objective(-e, traced=True)
        out.append((jp - jm) / (2 * h))
        flip = flip or tp.size != tm.size or not np.array_equal(tp, tm)
    return out + [float(flip)]


def main():
    with mp.get_context("spawn").Pool(min(8, os.cpu_count() or 1)) as pool:
        g = np.array(pool.map(component, range(N * N)))
    path = os.path.join(HERE, "adjoint_smooth24.txt")
    with open(path, "w") as f:
        f.write("# dJ/d(delta rho) by central differences of the oracle; see make_adjoint_golden.py\n")
        f.write("# n=%d steps=%d dt=%r seed=%d kmax=%d h=%r,%r J=%.17e\n"
                % (N, STEPS, DT, SEED, KMAX, HS[0], HS[1], objective(np.zeros((N, N)))))
        for k in range(N * N):
            f.write("%d %.17e %.17e %d\n" % (k, g[k, 0], g[k, 1], int(g[k, 2])))
    print(path)


if __name__ == "__main__":
    main()
