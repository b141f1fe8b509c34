"""The conventional path of the paper (WENO5-Z GKS and TENO5 GKS, Sec. 3.1,
4.1; 1-D grids) through the GPU against the FP64 oracle: stages and steps on
rough data for every collision model, a smooth run, Sod against the oracle's
round-off envelope and the exact solution; 2-D grids and batches refuse it."""
import numpy as np
import pytest

import oracle as O
from paper_2309_10534_gb300 import workloads as WL

pytestmark = pytest.mark.gpu
RECONS = ["weno_z", "teno5"]


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


TOL = {"fp64": 1e-12, "fp32": 1e-5}


@pytest.mark.parametrize("recon", RECONS)
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("tau", ["zero", "euler", "ns"])
def test_stage_and_step_random(gks, recon, precision, tau):
    """Ragged grid (several 127-cell tiles), rough data with a jump."""
    rng = np.random.default_rng(21)
    n = 300
    a = 1.0 if tau != "ns" else 0.2
    rho = np.exp(rng.uniform(-a, a, n)) * (1 + 0.5 * (np.arange(n) > 150))
    u = rng.uniform(-0.5, 0.5, n) * a
    p = np.exp(rng.uniform(-a, a, n))
    W = WL.conserved_1d(rho, u, p, 1.4)[:, None, :]
    kw = dict(bc=("zerograd", "reflect", "zerograd", "zerograd"), tau=tau, mu=0.01 if tau == "ns" else 0.0,
              Pr=0.73 if tau == "ns" else 1.0, recon=recon)
    P = O.make_problem(1, n, **kw)
    S = gks.Solver(1, n, precision=precision, **kw)
    S.set_state(W)
    dt = 0.3 * O.dt(P, W)
    S.stage(1, dt)
    assert rel_l1(S.get_buffer(1), O.stage1(P, W, dt)) < TOL[precision]
    S.set_state(W)
    S.step(dt)
    assert rel_l1(S.get_state(), O.step(P, W, dt)) < TOL[precision]


@pytest.mark.parametrize("recon", RECONS)
def test_smooth_advection_run(gks, recon):
    """Sec. 5.1 advection, N = 40, 200 steps of dt = 0.2 dx to t = 2 (tau = 0): float64
    to 1e-10 and float32 to 1e-6 of the oracle, and the float64 error against
    the exact solution equals the paper's table row (within 1 %)."""
    n = 40
    s = WL.advection_1d(n)
    P = O.make_problem(1, n, recon=recon, **s.problem_kwargs())
    dt = 0.2 * s.dx
    W = s.W.copy()
    steps = int(round(2.0 / dt))
    for _ in range(steps):
        W = O.step(P, W, dt)
    # the tables' N = 40 row (mesh length 1/20)
    table = {"weno_z": 9.0136622e-07, "teno5": 8.9738457e-07}[recon]
    for precision, tol in (("fp64", 1e-10), ("fp32", 1e-6)):
        S = gks.solver_for(s, precision, recon=recon)
        for _ in range(steps):
            S.step(dt)
        got = S.get_state()
        assert rel_l1(got, W) < tol, precision
        if precision == "fp64":
            e = np.mean(abs(got[0, 0] - WL.advection_1d_exact_rho(n, 2.0)))
            assert e == pytest.approx(table, rel=1e-2)


@pytest.mark.parametrize("recon", RECONS)
def test_sod_run(gks, recon):
    """Sod (Sec. 5.2 b), 400 cells to t = 0.2: float64 within 10x the
    oracle's own round-off envelope (and 1e-10), float32 within 1e-3; both
    as close to the exact solution as the oracle (float32: within 5 %)."""
    import exact_riemann as ER
    s = WL.sod(400)
    P = O.make_problem(1, 400, recon=recon, **s.problem_kwargs())
    Wo = O.run(P, s.W, 0.2)[0]
    Wb = O.run(P, s.W * (1 + 1e-15 * np.random.default_rng(0).standard_normal(s.W.shape)), 0.2)[0]
    spread = rel_l1(Wb, Wo)
    ex = ER.cell_averages(s.extra["left"], s.extra["right"], 400, 0.2)
    e_ora = np.mean(abs(Wo[0, 0] - ex[0]))
    for precision, tol, rel in (("fp64", max(1e-10, 10 * spread), 1e-3), ("fp32", 1e-3, 5e-2)):
        S = gks.solver_for(s, precision, recon=recon)
        steps, t = S.advance_to(0.2)
        assert t == pytest.approx(0.2, abs=1e-15)
        got = S.get_state()
        err = rel_l1(got, Wo)
        print(f"{recon} {precision}: rel L1 {err:.3e} (envelope {spread:.2e})")
        assert err < tol, (precision, err, spread)
        assert np.mean(abs(got[0, 0] - ex[0])) == pytest.approx(e_ora, rel=rel)
        assert S.diagnostics().error_word == 0


def test_refused_where_not_built(gks):
    with pytest.raises(gks.GKSError):
        gks.Solver(2, 16, 16, precision="fp64", recon="weno_z")
    with pytest.raises(gks.GKSError):
        gks.Batch(np.array([50, 60]), np.ones(2), precision="fp64", recon="teno5")
