"""The double Mach reflection (Sec. 5.7: inflow, wall after x = 1/6 and the
exact moving Mach 10 shock as boundaries) and the Riemann configuration 6
(Sec. 5.6 b) through the GPU path against the FP64 oracle."""
import numpy as np
import pytest

import oracle as O
from oracle_envelope import fp32_envelope
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
def test_dmr_first_step(gks, precision, tol):
    """One CFL step from the initial Mach 10 shock on 96 x 24 (ragged tiles):
    the ghosts of W at t = 0 and of W* at dt/2 come from the state-setting
    rules on the left, bottom and top."""
    s = WL.double_mach(96, 24)
    P = O.make_problem(2, 96, 24, **s.problem_kwargs())
    dt = O.dt(P, s.W)
    Wo = O.step(P, s.W, dt)
    S = gks.solver_for(s, precision)
    S.step(dt)
    err = rel_l1(S.get_state(), Wo)
    print(f"{precision}: {err:.3e}")
    assert err < tol


def test_dmr_run_fp64(gks):
    """25 CFL steps (t ~ 0.04: the top boundary's shock moves ~9 cells) on
    96 x 24, float64, against the oracle's own round-off envelope."""
    s = WL.double_mach(96, 24)
    P = O.make_problem(2, 96, 24, **s.problem_kwargs())
    Wa, steps, t, _ = O.run(P, s.W, 1.0, max_steps=25)
    rng = np.random.default_rng(0)
    Wb = O.run(P, s.W * (1 + 1e-15 * rng.standard_normal(s.W.shape)), 1.0, max_steps=25)[0]
    spread = rel_l1(Wb, Wa)
    S = gks.solver_for(s, "fp64")
    n, t_gpu = S.advance_to(1.0, max_steps=25)
    assert n == steps and t_gpu == pytest.approx(t, rel=1e-12)
    err = rel_l1(S.get_state(), Wa)
    print(f"DMR 25 steps: {err:.3e} (envelope {spread:.2e})")
    assert err <= max(1e-10, 10 * spread)


def test_dmr_run_fp32(gks):
    """The same run with the float32 flux: within 10x the oracle's spread
    under 1e-7 perturbations of every step's state (Mach 10 shocks on a
    coarse grid: float32 rounding moves TENO-D switches in the shock cells)."""
    s = WL.double_mach(96, 24)
    P = O.make_problem(2, 96, 24, **s.problem_kwargs())
    Wa, steps, t, _ = O.run(P, s.W, 1.0, max_steps=25)
    _, spread32 = fp32_envelope(P, s.W, 1.0, seeds=(0, 1), max_steps=25)
    S = gks.solver_for(s, "fp32")
    S.advance_to(t)
    err = rel_l1(S.get_state(), Wa)
    print(f"DMR fp32: {err:.3e} (oracle spread {spread32:.3e})")
    assert err < 10 * spread32
    assert S.diagnostics().error_word == 0


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_riemann_config6_run(gks, precision):
    """Configuration 6 (four contact discontinuities, Sec. 5.6 b) on 64 x 64
    to t = 0.1 at CFL 0.8: each path within 10x the oracle's spread at its
    rounding level (1e-15 initial, 1e-7 every step)."""
    s = WL.riemann2d_config6(64, t_end=0.1)
    P = O.make_problem(2, 64, 64, **s.problem_kwargs())
    Wa = O.run(P, s.W, 0.1)[0]
    if precision == "fp64":
        rng = np.random.default_rng(1)
        Wb = O.run(P, s.W * (1 + 1e-15 * rng.standard_normal(s.W.shape)), 0.1)[0]
        tol = max(1e-10, 10 * rel_l1(Wb, Wa))
    else:
        tol = 10 * fp32_envelope(P, s.W, 0.1, seeds=(0, 1))[1]
    S = gks.solver_for(s, precision)
    S.advance_to(0.1)
    err = rel_l1(S.get_state(), Wa)
    print(f"config 6 {precision}: {err:.3e} (bound {tol:.2e})")
    assert err < tol


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32", 1e-5)])
def test_inflow_1d_step(gks, precision, tol):
    """1-D inflow rule: Sod's tube with the left ghosts set to a state other
    than the edge cell's (the tube is fed with a faster flow)."""
    s = WL.sod(200)
    bcs = dict(bc_in=tuple(WL.conserved_1d(1.2, 0.4, 1.3, 1.4)))
    kw = dict(s.problem_kwargs(), bc=("inflow", "zerograd", "zerograd", "zerograd"), **bcs)
    P = O.make_problem(1, 200, **kw)
    dt = O.dt(P, s.W)
    Wo = O.step(P, s.W, dt)
    Wo = O.step(P, Wo, dt)
    S = gks.Solver(1, 200, precision=precision, bc=kw["bc"])
    S.set_boundary_states(**bcs)
    S.set_state(s.W)
    S.step(dt)
    S.step(dt)
    assert rel_l1(S.get_state(), Wo) < tol


def test_adjoint_refuses_state_setting_boundaries(gks):
    S = gks.Solver(2, 16, 16, bc=("inflow", "zerograd", "zerograd", "zerograd"), precision="fp64", tau="zero")
    S.set_state(WL.random_smooth_2d(16, 16, seed=1, kmax=2))
    with pytest.raises(gks.GKSError):
        gks.Adjoint(S, 2).forward(2, 0.01)


def test_state_setting_rules_only_on_y_sides(gks):
    with pytest.raises(gks.GKSError):
        gks.Solver(2, 16, 16, bc=("moving_shock", "zerograd", "zerograd", "zerograd"))


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32", 1e-5)])
def test_dmr_960x240_sampled_windows(gks, precision, tol):
    """Full size of the double Mach reflection (Sec. 5.7: 960 x 240 on
    [0, 4] x [0, 1]) in the launch configuration the bench times: 20 CFL
    steps on the GPU, then one step of the oracle's time step, checked on
    8 x 8 windows against the oracle stepping a cut-out of the same state with
    the window's origin and time (cut edges zero-gradient, 6 cells away), so
    the position- and time-dependent rules are exercised: the inflow edge,
    the foot of the wall at x = 1/6, the top boundary under the moving shock,
    the right edge and the interior across the shocks."""
    nx, ny = 960, 240
    s = WL.double_mach(nx, ny)
    P = O.make_problem(2, nx, ny, **s.problem_kwargs())
    S = gks.solver_for(s, precision)
    for _ in range(20):
        S.step(0.0)
    t = S.diagnostics().t
    W1 = S.get_state()
    P.t = t
    dt = O.dt(P, W1)
    S.step(dt)
    got = S.get_state()
    assert S.diagnostics().error_word == 0
    h = 4.0 / nx
    xs_top = 1.0 / 6.0 + (1.0 + 20.0 * t) / np.sqrt(3.0)  # the moving shock on y = 1
    it = int(xs_top / h) - 4
    corners = [(0, 0), (0, 116), (36, 0), (40, 0), (it, ny - 8), (it - 40, ny - 8), (nx - 8, 116), (600, 0),
               (100, 116), (int((1.0 / 6.0 + 0.5 / np.sqrt(3.0)) / h), 116)]
    M = 6
    for (i0, j0) in corners:
        xa, xb = max(i0 - M, 0), min(i0 + 8 + M, nx)
        ya, yb = max(j0 - M, 0), min(j0 + 8 + M, ny)
        bc = [P.bc[0] if xa == 0 else 1, P.bc[1] if xb == nx else 1, P.bc[2] if ya == 0 else 1,
              P.bc[3] if yb == ny else 1]
        kw = s.problem_kwargs()
        kw.update(bc=bc, lx=h * (xb - xa), ly=h * (yb - ya), ox=h * xa, oy=h * ya, t=t)
        Pw = O.make_problem(2, xb - xa, yb - ya, **kw)
        ref = O.step(Pw, np.ascontiguousarray(W1[:, ya:yb, xa:xb]), dt)[:, j0 - ya:j0 - ya + 8, i0 - xa:i0 - xa + 8]
        g = got[:, j0:j0 + 8, i0:i0 + 8]
        err = rel_l1(g, ref)
        print(f"{precision} window ({i0}, {j0}): {err:.3e}")
        assert err < tol, (i0, j0, err)


def test_dmr_paper_size_float32_stays_physical(gks):
    """The paper-size DMR (960 x 240, Sec. 5.7) in float32 for 400 CFL steps
    from the initial state and from two copies perturbed by 1e-7: every run
    stays physical, with a positivity-fallback count within 20 % of the
    float64 run's.  (Without the float32 internal-energy test, a
    reconstructed point on the incident shock with p = 7e-6 beside a cell
    at p = 21 -- a TENO-D overshoot that float64 carries harmlessly -- gave a
    float32 flux of the wrong sign and magnitude and a negative density
    within 250 steps.)"""
    s = WL.double_mach(960, 240, t_end=0.2)
    S = gks.solver_for(s, "fp64")
    S.advance_to(s.t_end, max_steps=400)
    fb64 = S.diagnostics().fallbacks
    S.close()
    for seed in (None, 1, 2):
        S = gks.solver_for(s, "fp32")
        if seed is not None:
            rng = np.random.default_rng(seed)
            S.set_state(s.W * (1 + 1e-7 * rng.standard_normal(s.W.shape)))
        n, t = S.advance_to(s.t_end, max_steps=400)
        d = S.diagnostics()
        S.close()
        print(f"seed {seed}: {n} steps to t = {t:.4f}, fallbacks {d.fallbacks} (float64 {fb64})")
        assert n == 400
        assert abs(d.fallbacks - fb64) <= 0.2 * fb64
