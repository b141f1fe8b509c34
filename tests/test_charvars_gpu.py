"""TENO-D in characteristic variables (Sec. 3.1: the normal reconstruction
on C = L W, with L, R the eigenvectors of the normal Euler flux Jacobian at
the mean of the face's two cells) through the GPU path, against the FP64
oracle: stages and steps at 1e-12 (float64) / 1e-5 (float32) on ragged
grids with discontinuities, whole runs within the oracle's own spread, and
the refusals of the paths that do not take it."""
import numpy as np
import pytest

import oracle as O
from oracle_envelope import oracle_envelope, rel_l1
from paper_2309_10534_gb300 import workloads as WL

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32": 1e-5}


@pytest.fixture(scope="module")
def gks():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2309_10534_gb300 import build, gks as G
    build.build()
    return G


def per_var_rel(a, b):
    a = np.asarray(a).reshape(a.shape[0], -1)
    b = np.asarray(b).reshape(b.shape[0], -1)
    scale = max(np.abs(b[0]).sum(), 1e-300)
    return [float(np.abs(a[v] - b[v]).sum() / max(np.abs(b[v]).sum(), 1e-3 * scale)) for v in range(a.shape[0])]


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("tau", ["zero", "euler", "ns"])
def test_1d_stage_and_step(gks, precision, tau):
    """300 cells (two 126-cell tiles and a ragged tail), rough data with a
    density jump, a reflecting end, every collision-time model."""
    rng = np.random.default_rng(12)
    n = 300
    a = 1.0 if tau != "ns" else 0.2
    rho = np.exp(rng.uniform(-a, a, n)) * (1 + 0.5 * (np.arange(n) > 150))
    u = rng.uniform(-0.5, 0.5, n) * a
    p = np.exp(rng.uniform(-a, a, n))
    W = WL.conserved_1d(rho, u, p, 1.4)[:, None, :]
    kw = dict(bc=("zerograd", "reflect", "zerograd", "zerograd"), tau=tau, mu=0.01 if tau == "ns" else 0.0,
              Pr=0.73 if tau == "ns" else 1.0)
    P = O.make_problem(1, n, charvars=1, **kw)
    S = gks.Solver(1, n, precision=precision, charvars=1, **kw)
    S.set_state(W)
    dt = 0.3 * O.dt(P, W)
    S.stage(1, dt)
    assert rel_l1(S.get_buffer(1), O.stage1(P, W, dt)) < TOL[precision]
    S.set_state(W)
    S.step(dt)
    assert rel_l1(S.get_state(), O.step(P, W, dt)) < TOL[precision]


CASES_2D = [
    ("rough", lambda nx, ny: WL.random_rough_2d(nx, ny, 16), ("zerograd", "reflect", "symmetry", "noslip"), "euler"),
    ("rough_tau0", lambda nx, ny: WL.random_rough_2d(nx, ny, 17), ("periodic",) * 4, "zero"),
    ("ns", lambda nx, ny: WL.random_rough_2d(nx, ny, 18), ("noslip", "noslip", "noslip", "symmetry"), "ns"),
]


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("case", CASES_2D, ids=[c[0] for c in CASES_2D])
def test_2d_stage_and_step(gks, precision, case):
    """70 x 37 cells: two 31-cell tiles and a ragged tail along x, several
    row tiles and a ragged tail along y; rough data, every boundary kind."""
    name, gen, bc, tau = case
    nx, ny = 70, 37
    W = gen(nx, ny)
    kw = dict(lx=1.0, ly=0.55, bc=bc, tau=tau, mu=0.02 if tau == "ns" else 0.0, Pr=0.73 if tau == "ns" else 1.0)
    P = O.make_problem(2, nx, ny, charvars=1, **kw)
    S = gks.Solver(2, nx, ny, precision=precision, charvars=1, **kw)
    S.set_state(W)
    dt = 0.4 * O.dt(P, W)
    S.stage(1, dt)
    assert max(per_var_rel(S.get_buffer(1), O.stage1(P, W, dt))) < TOL[precision]
    S.set_state(W)
    S.step(dt)
    got, ora = S.get_state(), O.step(P, W, dt)
    assert max(per_var_rel(got, ora)) < TOL[precision], per_var_rel(got, ora)


def test_sod_run_within_the_oracles_spread(gks):
    """Sod (Sec. 5.2 (b)), 400 cells to t = 0.2: float64 within 10x the
    oracle's spread under 1e-15 perturbations, float32 within 10x its spread
    under 1e-7 (float32-rounding) perturbations; both as close to the exact
    solution as the oracle."""
    import exact_riemann as ER
    s = WL.sod(400)
    P = O.make_problem(1, 400, charvars=1, **s.problem_kwargs())
    ex = ER.cell_averages(s.extra["left"], s.extra["right"], 400, 0.2)
    for precision, rel in (("fp64", 1e-15), ("fp32", 1e-7)):
        Wo, spread = oracle_envelope(P, s.W, 0.2, rel=rel, seeds=(0, 1, 2))
        S = gks.solver_for(s, precision, charvars=1)
        steps, t = S.advance_to(0.2)
        assert t == pytest.approx(0.2, abs=1e-15)
        got = S.get_state()
        err = rel_l1(got, Wo)
        print(f"{precision}: {err:.3e} (oracle spread {spread:.3e})")
        assert err <= 10 * spread + 1e-12, (precision, err, spread)
        e_gpu, e_ora = np.mean(abs(got[0, 0] - ex[0])), np.mean(abs(Wo[0, 0] - ex[0]))
        assert e_gpu == pytest.approx(e_ora, rel=2e-2)


def test_riemann_2d_run_within_the_oracles_spread(gks):
    """Configuration 3 of Sec. 5.6 on 48 x 48 to t = 0.05: both paths within
    10x the oracle's spread at their own rounding level."""
    s = WL.riemann2d(48, split=0.8, t_end=0.05)
    P = O.make_problem(2, 48, 48, charvars=1, **s.problem_kwargs())
    for precision, rel in (("fp64", 1e-15), ("fp32", 1e-7)):
        Wo, spread = oracle_envelope(P, s.W, 0.05, rel=rel, seeds=(0, 1))
        S = gks.solver_for(s, precision, charvars=1)
        S.advance_to(0.05)
        err = rel_l1(S.get_state(), Wo)
        print(f"{precision}: {err:.3e} (oracle spread {spread:.3e})")
        assert err <= max(10 * spread, 1e-12), (precision, err, spread)


def test_free_stream_and_conservation(gks):
    """A uniform state stays uniform; periodic rough data conserves every
    variable to round-off (float64)."""
    nx, ny = 45, 33
    W = np.zeros((4, ny, nx))
    W[0], W[1], W[2], W[3] = 0.8, 0.8 * 0.4, -0.8 * 0.3, 1.7
    S = gks.Solver(2, nx, ny, bc=("periodic",) * 4, precision="fp64", charvars=1)
    S.set_state(W)
    S.step(0.01)
    assert np.allclose(S.get_state(), W, rtol=1e-14, atol=1e-14)
    W = WL.random_rough_2d(nx, ny, 21)
    S.set_state(W)
    for _ in range(4):
        S.step(0.0)
    assert np.allclose(S.get_state().reshape(4, -1).sum(1), W.reshape(4, -1).sum(1), rtol=1e-13, atol=1e-12)


def test_refused_where_not_built(gks):
    """Characteristic variables are taken with TENO-D on single grids only."""
    with pytest.raises(gks.GKSError) as e:
        gks.Solver(1, 64, recon="weno_ao", charvars=1)
    assert e.value.status == gks.GKS_EUNSUPPORTED
    with pytest.raises(gks.GKSError):
        gks.Batch(np.array([64, 80]), np.ones(2), precision="fp64", charvars=1)
    S = gks.Solver(2, 16, 16, bc=("periodic",) * 4, precision="fp64", tau="zero", charvars=1)
    S.set_state(WL.random_smooth_2d(16, 16, seed=1, kmax=2))
    with pytest.raises(gks.GKSError):
        gks.Adjoint(S, 2).forward(2, 0.01)
