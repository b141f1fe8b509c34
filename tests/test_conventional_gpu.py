"""The conventional path of the paper (WENO5-Z GKS and TENO5 GKS, Sec. 3.1,
4.1) through the GPU against the FP64 oracle: 1-D stages and steps on rough
data for every collision model, a smooth run, Sod against the oracle's
round-off envelope and the exact solution; 2-D stages and steps on every
boundary kind, the 2-D accuracy table row, a Riemann run; batches refuse it."""
import numpy as np
import pytest

import oracle as O
from oracle_envelope import fp32_envelope
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
    """Ragged grid (several 126-cell tiles), rough data with a jump."""
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
    oracle's own round-off envelope (and 1e-10), float32 within 10x the
    oracle's spread under 1e-7 perturbations of every step's state; both as
    close to the exact solution as the oracle (float32: within 5 %)."""
    import exact_riemann as ER
    s = WL.sod(400)
    P = O.make_problem(1, 400, recon=recon, **s.problem_kwargs())
    Wo = O.run(P, s.W, 0.2)[0]
    Wb = O.run(P, s.W * (1 + 1e-15 * np.random.default_rng(0).standard_normal(s.W.shape)), 0.2)[0]
    spread = rel_l1(Wb, Wo)
    ex = ER.cell_averages(s.extra["left"], s.extra["right"], 400, 0.2)
    e_ora = np.mean(abs(Wo[0, 0] - ex[0]))
    spread32 = fp32_envelope(P, s.W, 0.2, seeds=(0, 1))[1]
    for precision, tol, rel in (("fp64", max(1e-10, 10 * spread), 1e-3), ("fp32", 10 * spread32, 5e-2)):
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
        gks.Batch(np.array([50, 60]), np.ones(2), precision="fp64", recon="teno5")


def _per_var_rel(a, b):
    a = np.asarray(a).reshape(a.shape[0], -1)
    b = np.asarray(b).reshape(b.shape[0], -1)
    scale = max(np.abs(b[0]).sum(), 1e-300)
    return [float(np.abs(a[v] - b[v]).sum() / max(np.abs(b[v]).sum(), 1e-3 * scale)) for v in range(a.shape[0])]


CASES_2D = [
    ("smooth_periodic_euler", lambda nx, ny: WL.random_smooth_2d(nx, ny, 1), ("periodic",) * 4, "euler"),
    ("rough_walls_euler", lambda nx, ny: WL.random_rough_2d(nx, ny, 2), ("zerograd", "reflect", "symmetry", "noslip"),
     "euler"),
    ("smooth_walls_ns", lambda nx, ny: WL.random_smooth_2d(nx, ny, 3), ("noslip", "noslip", "noslip", "symmetry"),
     "ns"),
    ("smooth_periodic_zero", lambda nx, ny: WL.random_smooth_2d(nx, ny, 4), ("periodic",) * 4, "zero"),
]


@pytest.mark.parametrize("recon", RECONS)
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("case", CASES_2D, ids=[c[0] for c in CASES_2D])
def test_2d_stage_and_step(gks, recon, precision, case):
    """2-D conventional path (Steps 1-4): 40 x 19 cells (two 31-cell tiles and
    a ragged tail along x, ragged row tiles along y), every boundary kind and
    collision model; one stage and one step against the oracle."""
    name, gen, bc, tau = case
    nx, ny = 40, 19
    W = gen(nx, ny)
    kw = dict(lx=1.0, ly=0.6, bc=bc, tau=tau, mu=0.02 if tau == "ns" else 0.0, Pr=0.73 if tau == "ns" else 1.0,
              recon=recon)
    P = O.make_problem(2, nx, ny, **kw)
    S = gks.Solver(2, nx, ny, precision=precision, **kw)
    S.set_state(W)
    dt = 0.4 * O.dt(P, W)
    S.stage(1, dt)
    assert max(_per_var_rel(S.get_buffer(1), O.stage1(P, W, dt))) < TOL[precision]
    S.set_state(W)
    S.step(dt)
    got, ora = S.get_state(), O.step(P, W, dt)
    assert max(_per_var_rel(got, ora)) < TOL[precision], _per_var_rel(got, ora)


@pytest.mark.parametrize("recon", RECONS)
def test_2d_accuracy_table_on_gpu(gks, recon):
    """Sec. 5.5 2-D advection, N = 20 to t = 2 at CFL 0.5 (tau = 0): the
    float64 GPU run equals the oracle's (1e-10 relative L1) and its density
    errors reproduce the paper's WENO5-Z / TENO5 table row to 3e-5."""
    n = 20
    s = WL.advection_2d(n)
    P = O.make_problem(2, n, n, recon=recon, **s.problem_kwargs())
    Wo = O.run(P, s.W, 2.0)[0]
    S = gks.solver_for(s, "fp64", recon=recon)
    S.advance_to(2.0)
    got = S.get_state()
    assert rel_l1(got, Wo) < 1e-10
    e = got[0] - WL.advection_2d_exact_rho(n, 2.0)
    errs = np.array([np.mean(abs(e)), np.sqrt(np.mean(e * e)), abs(e).max()])
    table = {"weno_z": [4.7700565e-05, 5.3254793e-05, 8.1803433e-05],
             "teno5": [4.2406682e-05, 4.7268698e-05, 6.9003512e-05]}[recon]
    assert np.all(np.abs(errs / np.array(table) - 1) < 3e-5), errs


@pytest.mark.parametrize("recon", RECONS)
def test_2d_riemann_run(gks, recon):
    """Riemann configuration 3 on 64 x 64 to t = 0.1: float64 within 10x the
    oracle's round-off envelope (and 1e-10), float32 within 10x the oracle's
    spread under 1e-7 perturbations of every step's state."""
    s = WL.riemann2d(64, split=0.8)
    P = O.make_problem(2, 64, 64, recon=recon, **s.problem_kwargs())
    Wa = O.run(P, s.W, 0.1)[0]
    Wb = O.run(P, s.W * (1 + 1e-15 * np.random.default_rng(0).standard_normal(s.W.shape)), 0.1)[0]
    spread = rel_l1(Wb, Wa)
    spread32 = fp32_envelope(P, s.W, 0.1, seeds=(0, 1))[1]
    for precision, tol in (("fp64", max(1e-10, 10 * spread)), ("fp32", 10 * spread32)):
        S = gks.solver_for(s, precision, recon=recon)
        S.advance_to(0.1)
        err = rel_l1(S.get_state(), Wa)
        print(f"{recon} {precision}: {err:.3e} (envelope {spread:.2e})")
        assert err < tol, (precision, err, spread)
