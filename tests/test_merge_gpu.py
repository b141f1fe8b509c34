"""The arithmetic-average merge (Sec. 3.2: the equilibrium state as the mean
of the two reconstructed sides, for smooth flow) through the GPU path
against the FP64 oracle: single grids in 1-D and 2-D, both precisions, and
the batched ensemble; the adjoint refuses it."""
import numpy as np
import pytest

import oracle as O
from paper_2309_10534_gb300 import workloads as WL

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gks():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2309_10534_gb300 import build, gks as G
    build.build()
    return G


def rel_l1(a, b):
    a = np.asarray(a).reshape(a.shape[0], -1)
    b = np.asarray(b).reshape(b.shape[0], -1)
    return float(np.abs(a - b).sum() / np.abs(b).sum())


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32", 1e-5)])
@pytest.mark.parametrize("tau", ["zero", "euler", "ns"])
def test_2d_smooth_steps(gks, precision, tol, tau):
    """Three CFL steps on a smooth periodic 2-D state, non-square cells and a
    ragged grid (several 31 x 16 tiles plus partial tiles)."""
    nx, ny = 70, 37
    W = WL.random_smooth_2d(nx, ny, seed=9, kmax=2)
    # NS with the Prandtl correction: its heat flux takes the side terms'
    # density moments (the kinetic merge) while W0 is the average
    kw = dict(lx=1.3, ly=1.0, bc=("periodic",) * 4, tau=tau, mu=0.002, Pr=0.73 if tau == "ns" else 1.0,
              merge="average")
    P = O.make_problem(2, nx, ny, **kw)
    S = gks.Solver(2, nx, ny, precision=precision, **kw)
    S.set_state(W)
    Wo = W
    for _ in range(3):
        Wo = O.step(P, Wo, O.dt(P, Wo))
        S.step(0.0)
    err = rel_l1(S.get_state(), Wo)
    print(f"{precision} {tau}: {err:.3e}")
    assert err <= tol


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-10), ("fp32", 1e-6)])
def test_1d_advection_run(gks, precision, tol):
    """1-D smooth advection (Sec. 5.1, tau = 0) on 80 cells, 100 steps of
    dt = 0.2 dx (to t = 0.5): the whole run agrees with the oracle's."""
    n = 80
    s = WL.advection_1d(n)
    P = O.make_problem(1, n, merge="average", **s.problem_kwargs())
    dt = 0.2 * s.dx
    Wo = s.W.copy()
    for _ in range(100):
        Wo = O.step(P, Wo, dt)
    S = gks.solver_for(s, precision, merge="average")
    for _ in range(100):
        S.step(dt)
    assert rel_l1(S.get_state(), Wo) <= tol


def test_batch_matches_oracle(gks):
    """Batched smooth 1-D problems (density waves at rest, zero-gradient ends)
    with the average merge, float64, 5 steps: each equal to the oracle's."""
    sizes = [40, 123, 250, 301]
    Ws = []
    for k, n in enumerate(sizes):
        x = (np.arange(n) + 0.5) / n
        rho = 1.0 + 0.2 * np.sin(2 * np.pi * (k + 1) * x) ** 2
        Ws.append(WL.conserved_1d(rho, 0.3 + 0 * x, 1.0 + 0 * x, 1.4))
    B = gks.Batch(np.array(sizes), np.ones(len(sizes)), precision="fp64", merge="average")
    B.set_state(np.concatenate(Ws, axis=1))
    B.advance_to(1.0, max_steps=5)
    out = B.get_state()
    _, steps, err, _ = B.progress()
    assert np.all(steps == 5) and np.all(err == 0)
    off = np.concatenate([[0], np.cumsum(sizes)])
    for k, n in enumerate(sizes):
        P = O.make_problem(1, n, tau="euler", merge="average")
        Wo = O.run(P, Ws[k][:, None, :], 1.0, max_steps=5)[0][:, 0, :]
        assert rel_l1(out[:, off[k]:off[k + 1]], Wo) < 1e-12, n


def test_adjoint_refuses_average_merge(gks):
    S = gks.Solver(2, 16, 16, bc=("periodic",) * 4, precision="fp64", tau="zero", merge="average")
    S.set_state(WL.random_smooth_2d(16, 16, seed=1, kmax=2))
    with pytest.raises(gks.GKSError):
        gks.Adjoint(S, 2).forward(2, 0.01)
