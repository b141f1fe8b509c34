"""Degenerate and edge cases of the GPU path: free-stream preservation for
every reconstruction and boundary rule that keeps a uniform state, the
smallest grids, and the arguments the C ABI refuses."""
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


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-14), ("fp32", 2e-7)])
@pytest.mark.parametrize("recon", ["teno_d", "weno_ao"])
@pytest.mark.parametrize("tau", ["zero", "euler", "ns"])
def test_uniform_flow_is_preserved_2d(gks, precision, tol, recon, tau):
    """A uniform moving state on a ragged periodic / zero-gradient grid stays
    uniform: every reconstruction returns the state with zero slopes, the
    merge returns it, and the flux differences vanish (5 CFL steps)."""
    nx, ny = 37, 29
    W = np.repeat(WL.conserved_2d(1.3, 0.4, -0.2, 0.9, 1.4)[:, None, None], nx * ny, axis=1).reshape(4, ny, nx)
    S = gks.Solver(2, nx, ny, bc=("periodic", "periodic", "zerograd", "zerograd"), precision=precision, tau=tau,
                   mu=0.01, Pr=0.73 if tau == "ns" else 1.0, recon=recon)
    S.set_state(W)
    for _ in range(5):
        S.step(0.0)
    got = S.get_state()
    assert np.abs(got - W).max() <= tol * np.abs(W).max()


@pytest.mark.parametrize("recon", ["teno_d", "weno_ao", "weno_z", "teno5"])
@pytest.mark.parametrize("precision,tol", [("fp64", 1e-14), ("fp32", 2e-7)])
def test_uniform_flow_is_preserved_1d(gks, recon, precision, tol):
    W = np.repeat(WL.conserved_1d(0.8, -0.3, 1.1, 1.4)[:, None], 130, axis=1)[:, None, :]
    S = gks.Solver(1, 130, bc=("zerograd",) * 4, precision=precision, recon=recon)
    S.set_state(W)
    for _ in range(5):
        S.step(0.0)
    assert np.abs(S.get_state() - W).max() <= tol * np.abs(W).max()


def test_state_at_rest_against_walls_stays_at_rest(gks):
    """Gas at rest between reflecting / no-slip walls and symmetry planes:
    nothing moves (the mirrored ghosts carry zero velocity)."""
    W = np.repeat(WL.conserved_2d(1.0, 0.0, 0.0, 1.0, 1.4)[:, None, None], 40 * 24, axis=1).reshape(4, 24, 40)
    S = gks.Solver(2, 40, 24, bc=("reflect", "noslip", "symmetry", "noslip"), precision="fp64", tau="ns",
                   mu=0.01, Pr=0.73)
    S.set_state(W)
    for _ in range(5):
        S.step(0.0)
    assert np.abs(S.get_state() - W).max() <= 1e-14


@pytest.mark.parametrize("dim", [1, 2])
def test_smallest_grid_matches_oracle(gks, dim):
    """The smallest grid the ABI accepts (3 cells per direction): one step
    equals the oracle's (float64)."""
    n = 3
    rng = np.random.default_rng(4)
    if dim == 1:
        W = WL.conserved_1d(np.exp(rng.uniform(-0.3, 0.3, n)), rng.uniform(-0.3, 0.3, n),
                            np.exp(rng.uniform(-0.3, 0.3, n)), 1.4)[:, None, :]
    else:
        W = WL.conserved_2d(np.exp(rng.uniform(-0.3, 0.3, (n, n))), rng.uniform(-0.3, 0.3, (n, n)),
                            rng.uniform(-0.3, 0.3, (n, n)), np.exp(rng.uniform(-0.3, 0.3, (n, n))), 1.4)
    kw = dict(bc=("periodic",) * 4)
    P = O.make_problem(dim, n, n, **kw)
    S = gks.Solver(dim, n, n, precision="fp64", **kw)
    S.set_state(W)
    dt = O.dt(P, W)
    S.step(dt)
    assert rel_l1(S.get_state(), O.step(P, W, dt)) < 1e-12


def test_refused_arguments(gks):
    """Bad arguments return an error status and leave the context usable."""
    S = gks.Solver(2, 16, 16, precision="fp64")
    S.set_state(WL.random_smooth_2d(16, 16, seed=2))
    with pytest.raises(gks.GKSError):
        S.stage(3, 1e-3)        # no such stage
    with pytest.raises(gks.GKSError):
        S.stage(1, -1.0)        # non-positive dt
    with pytest.raises(gks.GKSError):
        S.set_scheme(cfl=-0.5)  # out of range
    with pytest.raises((gks.GKSError, ValueError)):
        S.set_state(np.zeros(5))  # wrong size
    S.step(0.0)                 # still usable
    assert np.isfinite(S.get_state()).all()


def test_async_pinned_state_copies_match_the_synchronous_ones(gks):
    """GKS_HOST_PINNED_ASYNC: the state copied in from page-locked memory and
    stepped on two contexts with their own streams, alternating, gives the
    same bits as the synchronous calls on one context; the async mode is
    refused where it is not supported (gks_get_buffer) and an unknown mode
    anywhere."""
    import ctypes
    import torch
    s = WL.riemann2d(96, split=0.8, t_end=0.8)
    S = gks.solver_for(s, "fp32")
    S.set_state(s.W)
    S.step(0.0)
    ref = S.get_state()
    host_in = torch.from_numpy(np.ascontiguousarray(s.W)).pin_memory()
    pipe = []
    for _ in range(2):
        st = torch.cuda.Stream()
        P = gks.solver_for(s, "fp32")
        P.set_stream(st.cuda_stream)
        pipe.append((P, torch.empty_like(host_in).pin_memory()))
    for k in range(4):
        P, out = pipe[k % 2]
        P.set_state_async(host_in)
        P.step(0.0)
        P.get_state_async(out)
    torch.cuda.synchronize()
    for P, out in pipe:
        assert np.array_equal(out.numpy(), ref)
        d = P.diagnostics()
        assert d.steps == 1 and d.t > 0
        buf = np.empty(S.shape)
        st = gks.lib().gks_get_buffer(P.h, 0, buf.ctypes.data_as(ctypes.c_void_p), gks.GKS_HOST_PINNED_ASYNC)
        assert st == gks.GKS_EINVAL
        st = gks.lib().gks_set_state(P.h, buf.ctypes.data_as(ctypes.c_void_p), 3)
        assert st == gks.GKS_EINVAL
        P.close()
    S.close()
