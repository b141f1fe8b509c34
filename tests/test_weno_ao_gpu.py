"""WENO5-AO reconstruction (Sec. 3.2) on the GPU path against the FP64 oracle:
the same stage/step parity bars as TENO-D, the paper's 2-D WENO-AO accuracy
table, and a Riemann run."""
import numpy as np
import pytest

import oracle as O
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


def rel_l1(a, b):
    a = np.asarray(a).reshape(a.shape[0], -1)
    b = np.asarray(b).reshape(b.shape[0], -1)
    return float(np.abs(a - b).sum() / np.abs(b).sum())


def per_var_rel(a, b):
    a = np.asarray(a).reshape(a.shape[0], -1)
    b = np.asarray(b).reshape(b.shape[0], -1)
    scale = max(np.abs(b[0]).sum(), 1e-300)
    return [float(np.abs(a[v] - b[v]).sum() / max(np.abs(b[v]).sum(), 1e-3 * scale)) for v in range(a.shape[0])]


CASES = [
    ("smooth", lambda nx, ny: WL.random_smooth_2d(nx, ny, 5), ("periodic",) * 4, "euler"),
    ("rough", lambda nx, ny: WL.random_rough_2d(nx, ny, 6), ("zerograd", "reflect", "symmetry", "noslip"), "euler"),
    ("rough_tau0", lambda nx, ny: WL.random_rough_2d(nx, ny, 7), ("zerograd",) * 4, "zero"),
    ("ns", lambda nx, ny: WL.random_rough_2d(nx, ny, 8), ("noslip", "noslip", "noslip", "symmetry"), "ns"),
]


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_2d_stage_and_step_weno_ao(gks, precision, case):
    """40 x 19 cells (ragged tiles both ways), every boundary kind."""
    name, gen, bc, tau = case
    nx, ny = 40, 19
    W = gen(nx, ny)
    kw = dict(lx=1.0, ly=0.6, bc=bc, tau=tau, mu=0.02 if tau == "ns" else 0.0, Pr=0.73 if tau == "ns" else 1.0)
    P = O.make_problem(2, nx, ny, recon="weno_ao", **kw)
    S = gks.Solver(2, nx, ny, precision=precision, recon="weno_ao", **kw)
    S.set_state(W)
    dt = 0.4 * O.dt(P, W)
    S.stage(1, dt)
    assert max(per_var_rel(S.get_buffer(1), O.stage1(P, W, dt))) < TOL[precision]
    S.set_state(W)
    S.step(dt)
    ora = O.step(P, W, dt)
    assert max(per_var_rel(S.get_state(), ora)) < TOL[precision], per_var_rel(S.get_state(), ora)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("tau", ["zero", "euler", "ns"])
def test_1d_stage_and_step_weno_ao(gks, precision, tau):
    rng = np.random.default_rng(11)
    n = 300
    a = 1.0 if tau != "ns" else 0.2
    rho = np.exp(rng.uniform(-a, a, n)) * (1 + 0.5 * (np.arange(n) > 150))
    u = rng.uniform(-0.5, 0.5, n) * a
    p = np.exp(rng.uniform(-a, a, n))
    W = WL.conserved_1d(rho, u, p, 1.4)[:, None, :]
    kw = dict(bc=("zerograd", "reflect", "zerograd", "zerograd"), tau=tau, mu=0.01 if tau == "ns" else 0.0,
              Pr=0.73 if tau == "ns" else 1.0)
    P = O.make_problem(1, n, 1, recon="weno_ao", **kw)
    S = gks.Solver(1, n, 1, precision=precision, recon="weno_ao", **kw)
    S.set_state(W)
    dt = 0.3 * O.dt(P, W)
    S.stage(1, dt)
    assert rel_l1(S.get_buffer(1), O.stage1(P, W, dt)) < TOL[precision]
    S.set_state(W)
    S.step(dt)
    assert rel_l1(S.get_state(), O.step(P, W, dt)) < TOL[precision]


def test_accuracy_2d_weno_ao_table_on_gpu(gks):
    """Sec. 5.5 WENO-AO table, row N = 20, reproduced by the float64 GPU path."""
    n = 20
    s = WL.advection_2d(n)
    S = gks.Solver(2, n, n, lx=s.lx, ly=s.ly, bc=s.bc, precision="fp64", tau="zero", cfl=s.cfl, recon="weno_ao")
    S.set_state(s.W)
    S.advance_to(2.0)
    e = S.get_state()[0] - WL.advection_2d_exact_rho(n, 2.0)
    assert np.mean(abs(e)) == pytest.approx(4.2540389e-05, rel=1e-5)


def test_riemann_weno_ao_matches_oracle(gks):
    """Configuration 3 of Sec. 5.6 on 48 x 48 to t = 0.05 with WENO5-AO: the
    weights are continuous in the data (no switching), so float64 agrees with
    the oracle to 1e-10 over the whole run."""
    s = WL.riemann2d(48, split=0.8, t_end=0.05)
    P = O.make_problem(2, 48, 48, recon="weno_ao", **s.problem_kwargs())
    Wo = O.run(P, s.W, 0.05)[0]
    S = gks.Solver(2, 48, 48, lx=s.lx, ly=s.ly, bc=s.bc, precision="fp64", tau=s.tau, cfl=s.cfl, recon="weno_ao")
    S.set_state(s.W)
    S.advance_to(0.05)
    assert rel_l1(S.get_state(), Wo) < 1e-10


def test_recon_rejected_where_unsupported(gks):
    S = gks.Solver(2, 16, 16, bc=("periodic",) * 4, precision="fp64", tau="zero", recon="weno_ao")
    with pytest.raises(gks.GKSError):
        gks.Adjoint(S, 4)
    with pytest.raises(gks.GKSError):
        gks.Batch(np.array([10]), np.ones(1), recon="weno_ao")
