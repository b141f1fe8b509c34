"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Tolerances: float64 stages and steps <= 1e-12 relative L1, smooth float64
runs <= 1e-10; float32-flux / float64-accumulation path <= 1e-5 per step.
Long runs through shocks are compared against the oracle's own round-off
envelope (TENO-D switches discontinuously, so rounding-level differences can
move a switch; see _oracle_envelope).
"""
import numpy as np
import pytest

import oracle as O
from oracle_envelope import fp32_envelope
from paper_2309_10534_gb300 import workloads as WL

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2309_10534_gb300 import build
    build.build()


def G():
    from paper_2309_10534_gb300 import gks
    return gks


def rel_l1(a, b):
    a = np.asarray(a).reshape(a.shape[0], -1)
    b = np.asarray(b).reshape(b.shape[0], -1)
    return float(np.abs(a - b).sum() / np.abs(b).sum())


def per_var_rel(a, b):
    a = np.asarray(a).reshape(a.shape[0], -1)
    b = np.asarray(b).reshape(b.shape[0], -1)
    scale = max(np.abs(b[0]).sum(), 1e-300)
    return [float(np.abs(a[v] - b[v]).sum() / max(np.abs(b[v]).sum(), 1e-3 * scale)) for v in range(a.shape[0])]


def make_pair(dim, nx, ny, W, precision="fp64", **kw):
    P = O.make_problem(dim, nx, ny, **kw)
    S = G().Solver(dim, nx, ny, precision=precision, **kw)
    S.set_state(W)
    return P, S


TOL = {"fp64": 1e-12, "fp32": 1e-5}


# ------------------------------------------------------------------ 1-D
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("tau", ["zero", "euler", "ns"])
def test_1d_stage_and_step_random(precision, tau):
    """Ragged 1-D grid (several 126-cell tiles), rough data, all collision-time models."""
    rng = np.random.default_rng(11)
    n = 300
    a = 1.0 if tau != "ns" else 0.2  # cell-to-cell noise the viscous step keeps physical
    rho = np.exp(rng.uniform(-a, a, n)) * (1 + 0.5 * (np.arange(n) > 150))
    u = rng.uniform(-0.5, 0.5, n) * a
    p = np.exp(rng.uniform(-a, a, n))
    W = WL.conserved_1d(rho, u, p, 1.4)[:, None, :]
    kw = dict(bc=("zerograd", "reflect", "zerograd", "zerograd"), tau=tau, mu=0.01 if tau == "ns" else 0.0,
              Pr=0.73 if tau == "ns" else 1.0)
    P, S = make_pair(1, n, 1, W, precision, **kw)
    dt = 0.3 * O.dt(P, W)
    S.stage(1, dt)
    ws = S.get_buffer(1)
    assert rel_l1(ws, O.stage1(P, W, dt)) < TOL[precision]
    S.set_state(W)
    S.step(dt)
    assert rel_l1(S.get_state(), O.step(P, W, dt)) < TOL[precision]


def _oracle_envelope(P, W0, t_end, seeds=(0, 1)):
    """The oracle's own round-off envelope on a run: relative L1 spread between
    the unperturbed run and runs whose initial state is perturbed by 1e-15
    relative.  TENO-D switches discontinuously, so on shock problems a
    rounding-level change can move a switch and grow to ~1e-6 (several
    results are equally correct)."""
    Wa = O.run(P, W0, t_end)[0]
    spread = 0.0
    for sd in seeds:
        rng = np.random.default_rng(sd)
        Wb = O.run(P, W0 * (1 + 1e-15 * rng.standard_normal(W0.shape)), t_end)[0]
        spread = max(spread, rel_l1(Wb, Wa))
    return Wa, spread


def test_1d_sod_full_run_fp64():
    """Sec. 5.2 (b) Sod, 400 cells to t = 0.2 with CFL steps and graph replays.
    The float64 GPU run lies within 10x the oracle's own round-off envelope,
    and its distance to the exact solution equals the oracle's."""
    import exact_riemann as ER
    s = WL.sod(400)
    P, S = make_pair(1, 400, 1, s.W, "fp64", **s.problem_kwargs())
    Wo, spread = _oracle_envelope(P, s.W, 0.2)
    steps, t = S.advance_to(0.2)
    assert t == pytest.approx(0.2, abs=1e-15)
    got = S.get_state()
    assert rel_l1(got, Wo) <= 10 * spread + 1e-12, (rel_l1(got, Wo), spread)
    ex = ER.cell_averages(s.extra["left"], s.extra["right"], 400, 0.2)
    e_gpu = np.mean(abs(got[0, 0] - ex[0]))
    e_ora = np.mean(abs(Wo[0, 0] - ex[0]))
    assert e_gpu == pytest.approx(e_ora, rel=1e-3)
    assert S.diagnostics().error_word == 0


def test_1d_sod_full_run_fp32():
    """float32 flux / float64 state on the same run: within 10x the oracle's
    spread under 1e-7 perturbations of every step's state (float32 rounding
    moves TENO-D switches; measured: the float32 run lies inside that spread,
    4.7e-4 against 4.7e-4), and its distance to the exact solution within
    5 % of the oracle's (measured 1.7 %)."""
    import exact_riemann as ER
    s = WL.sod(400)
    P, S = make_pair(1, 400, 1, s.W, "fp32", **s.problem_kwargs())
    Wo, spread32 = fp32_envelope(P, s.W, 0.2)
    S.advance_to(0.2)
    got = S.get_state()
    err = rel_l1(got, Wo)
    print(f"Sod fp32: {err:.3e} (oracle spread {spread32:.3e})")
    assert err < 10 * spread32, (err, spread32)
    ex = ER.cell_averages(s.extra["left"], s.extra["right"], 400, 0.2)
    assert np.mean(abs(got[0, 0] - ex[0])) == pytest.approx(np.mean(abs(Wo[0, 0] - ex[0])), rel=5e-2)


def test_1d_advection_full_run_matches_oracle():
    """Smooth data never switches TENO-D off the large stencil: the whole run
    (Sec. 5.1, N = 40, 400 steps of dt = 0.2 dx, tau = 0) agrees to 1e-10 in
    float64 and to 1e-6 in float32."""
    n = 40
    s = WL.advection_1d(n)
    P = O.make_problem(1, n, **s.problem_kwargs())
    dt = 0.2 * s.dx
    W = s.W.copy()
    for _ in range(int(round(2.0 / dt))):
        W = O.step(P, W, dt)
    for precision, tol in (("fp64", 1e-10), ("fp32", 1e-6)):
        S = G().solver_for(s, precision)
        for _ in range(int(round(2.0 / dt))):
            S.step(dt)
        assert rel_l1(S.get_state(), W) < tol, precision


def test_1d_dt_matches_oracle():
    s = WL.sod(400)
    P, S = make_pair(1, 400, 1, s.W, "fp64", **s.problem_kwargs())
    assert S.compute_dt() == pytest.approx(O.dt(P, s.W), rel=1e-14)


# ------------------------------------------------------------------ 2-D
CASES_2D = [
    ("smooth", lambda nx, ny: WL.random_smooth_2d(nx, ny, 5), ("periodic",) * 4, "euler"),
    ("rough", lambda nx, ny: WL.random_rough_2d(nx, ny, 6), ("zerograd", "reflect", "symmetry", "noslip"), "euler"),
    ("rough_tau0", lambda nx, ny: WL.random_rough_2d(nx, ny, 7), ("zerograd",) * 4, "zero"),
    ("ns", lambda nx, ny: WL.random_rough_2d(nx, ny, 8), ("noslip", "noslip", "noslip", "symmetry"), "ns"),
]


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("case", CASES_2D, ids=[c[0] for c in CASES_2D])
def test_2d_stage_and_step(precision, case):
    """40 x 19 cells: two 31-cell tiles + ragged tail along x, three 8-row
    tiles with a ragged tail along y; every boundary kind."""
    name, gen, bc, tau = case
    nx, ny = 40, 19
    W = gen(nx, ny)
    kw = dict(lx=1.0, ly=0.6, bc=bc, tau=tau, mu=0.02 if tau == "ns" else 0.0, Pr=0.73 if tau == "ns" else 1.0)
    P, S = make_pair(2, nx, ny, W, precision, **kw)
    dt = 0.4 * O.dt(P, W)
    S.stage(1, dt)
    ora1 = O.stage1(P, W, dt)
    assert max(per_var_rel(S.get_buffer(1), ora1)) < TOL[precision]
    S.set_state(W)
    S.step(dt)
    ora = O.step(P, W, dt)
    got = S.get_state()
    assert max(per_var_rel(got, ora)) < TOL[precision], per_var_rel(got, ora)


def test_2d_dt_and_conservation_fp64():
    nx, ny = 33, 17
    W = WL.random_rough_2d(nx, ny, 9)
    P, S = make_pair(2, nx, ny, W, "fp64", lx=1.0, ly=0.5, bc=("periodic",) * 4, tau="euler")
    dt = S.compute_dt()
    assert dt == pytest.approx(O.dt(P, W), rel=1e-14)
    tot0 = W.reshape(4, -1).sum(axis=1)
    for _ in range(5):
        S.step(0.0)
    tot = S.get_state().reshape(4, -1).sum(axis=1)
    assert np.allclose(tot, tot0, rtol=1e-13, atol=1e-12)


def test_2d_riemann_advance_fp64_and_fp32():
    """Configuration 3 of Sec. 5.6 on 64 x 64 to t = 0.1 (CFL steps, graphs):
    float64 within 10x the oracle's round-off envelope (and 1e-10), float32
    within 10x the oracle's spread under 1e-7 perturbations of every step's
    state (measured 1.9e-5 against a spread of 2.6e-4)."""
    s = WL.riemann2d(64, split=0.8, t_end=0.1)
    P = O.make_problem(2, 64, 64, **s.problem_kwargs())
    Wo, spread = _oracle_envelope(P, s.W, 0.1, seeds=(0,))
    _, spread32 = fp32_envelope(P, s.W, 0.1, seeds=(0, 1))
    for precision, tol in (("fp64", max(1e-10, 10 * spread)), ("fp32", 10 * spread32)):
        S = G().solver_for(s, precision)
        steps, t = S.advance_to(0.1)
        assert t == pytest.approx(0.1, abs=1e-15)
        err = rel_l1(S.get_state(), Wo)
        assert err < tol, (precision, err, spread)


def test_accuracy_2d_table_on_gpu():
    """Sec. 5.5 TENO-D table row N = 20 reproduced by the float64 GPU path."""
    n = 20
    s = WL.advection_2d(n)
    S = G().solver_for(s, "fp64")
    S.advance_to(2.0)
    e = S.get_state()[0] - WL.advection_2d_exact_rho(n, 2.0)
    assert np.mean(abs(e)) == pytest.approx(4.2451259e-05, rel=1e-5)


def test_viscous_shock_tube_steps_fp64():
    """Sec. 5.8 setup (walls, symmetry top, NS collision time, Pr = 0.73) on a
    64 x 32 grid, 3 CFL steps."""
    s = WL.viscous_shock_tube(64, 32)
    P = O.make_problem(2, 64, 32, **s.problem_kwargs())
    W = s.W.copy()
    S = G().solver_for(s, "fp64")
    for _ in range(3):
        dt = O.dt(P, W)
        W = O.step(P, W, dt)
        S.step(dt)
    assert rel_l1(S.get_state(), W) < 1e-11


# ------------------------------------------------------------------ full size, sampled
def _window_step(P_full, W, dt, i0, j0, w, M=6):
    """Oracle step on a cut-out window; cells farther than M from a cut edge
    are exact.  Sides on the domain boundary keep the domain's BC."""
    nv, ny, nx = W.shape
    xa, xb = max(i0 - M, 0), min(i0 + w + M, nx)
    ya, yb = max(j0 - M, 0), min(j0 + w + M, ny)
    sub = np.ascontiguousarray(W[:, ya:yb, xa:xb])
    bc = [P_full.bc[k] for k in range(4)]
    cut = [xa > 0, xb < nx, ya > 0, yb < ny]
    bc = [1 if cut[k] else bc[k] for k in range(4)]
    P = O.make_problem(2, xb - xa, yb - ya, lx=P_full.dx * (xb - xa), ly=P_full.dy * (yb - ya), bc=bc,
                       tau=P_full.tau_mode, gamma=P_full.gamma, mu=P_full.mu, Pr=P_full.Pr, cfl=P_full.cfl)
    out = O.step(P, sub, dt)
    return out[:, j0 - ya:j0 - ya + w, i0 - xa:i0 - xa + w]


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_riemann_1024_sampled_windows(precision):
    """Full size of the 2-D Riemann workload (1024^2), one CFL step in the
    launch configuration the bench times; oracle on sampled windows that
    cover the quadrant corner, the boundaries and the interior."""
    s = WL.riemann2d(1024, split=0.8)
    P = O.make_problem(2, 1024, 1024, **s.problem_kwargs())
    W = s.W
    # evolve a few steps on the GPU first so the windows see developed waves
    S = G().solver_for(s, "fp64")
    for _ in range(20):
        S.step(0.0)
    W1 = S.get_state()
    dt = O.dt(P, W1)
    S2 = G().solver_for(s, precision)
    S2.set_state(W1)
    S2.step(dt)
    got = S2.get_state()
    rng = np.random.default_rng(1)
    corners = [(812, 812), (0, 0), (1016, 1016), (0, 812), (812, 1016)]
    corners += [tuple(rng.integers(0, 1016, 2)) for _ in range(3)]
    for (i0, j0) in corners:
        ref = _window_step(P, W1, dt, int(i0), int(j0), 8)
        g = got[:, j0:j0 + 8, i0:i0 + 8]
        assert rel_l1(g, ref) < TOL[precision], (i0, j0)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_viscous_2048_sampled_windows(precision):
    """Full size of the viscous shock tube (Sec. 5.8: 2048 x 1024, Re = 200,
    Pr = 0.73, no-slip walls, symmetric top, NS collision time with the
    Prandtl fix), one step in the launch configuration the bench times after
    20 float64 steps; oracle on windows at the walls, the corners, the top and
    across the shock."""
    s = WL.viscous_shock_tube(2048, 1024)
    P = O.make_problem(2, 2048, 1024, **s.problem_kwargs())
    S = G().solver_for(s, "fp64")
    for _ in range(20):
        S.step(0.0)
    W1 = S.get_state()
    dt = O.dt(P, W1)
    S2 = G().solver_for(s, precision)
    S2.set_state(W1)
    S2.step(dt)
    got = S2.get_state()
    rng = np.random.default_rng(2)
    corners = [(0, 0), (2040, 0), (0, 1016), (2040, 1016), (1020, 0), (1020, 1016), (1020, 500)]
    corners += [tuple(int(x) for x in rng.integers(0, 1016, 2)) for _ in range(2)]
    for (i0, j0) in corners:
        ref = _window_step(P, W1, dt, i0, j0, 8)
        g = got[:, j0:j0 + 8, i0:i0 + 8]
        assert rel_l1(g, ref) < TOL[precision], (i0, j0, rel_l1(g, ref))


def test_isentropic_vortex_fifth_order_on_gpu():
    """The float64 GPU path on the isentropic vortex to t = 0.5 (tau = 0):
    equal to the oracle on N = 40 (dt = 0.1 h, 1e-10 relative L1), and its
    density error against the exact vortex converges at order >= 4.8 from
    N = 64 to 128 (measured 4.95; the oracle's own pin stops at N = 80).  At
    dt = 0.1 h the fourth-order time error reaches the spatial error at
    N = 256 (measured order 4.1 from 128 to 256), so the finest pair is not
    used."""
    t_end = 0.5
    errs = {}
    for n in (40, 64, 128):
        s = WL.isentropic_vortex(n, seed=None)
        steps = int(np.ceil(t_end / (0.1 * s.dx)))
        dt = t_end / steps
        S = G().solver_for(s, "fp64")
        for _ in range(steps):
            S.step(dt)
        W = S.get_state()
        exact = WL.isentropic_vortex(n, center=(5.0 + t_end, 5.0 + t_end), seed=None).W
        errs[n] = np.mean(np.abs(W[0] - exact[0]))
        if n == 40:
            P = O.make_problem(2, n, n, **s.problem_kwargs())
            Wo = s.W.copy()
            for _ in range(steps):
                Wo = O.step(P, Wo, dt)
            assert rel_l1(W, Wo) < 1e-10
    order = np.log2(errs[64] / errs[128])
    print("vortex L1:", errs, "order 64->128 %.3f" % order)
    assert order >= 4.8, errs


def test_nonphysical_state_reported():
    W = WL.random_smooth_2d(16, 16, 3)
    W[0, 5, 5] = -1.0  # negative density
    S = G().Solver(2, 16, 16, bc=("periodic",) * 4)
    S.set_state(W)
    with pytest.raises(G().GKSError) as e:
        S.advance_to(1.0, max_steps=2)
    assert e.value.status == G().GKS_ENONPHYSICAL
