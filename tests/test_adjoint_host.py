"""Hand-written reverse-mode functions of the adjoint (host builds of the
device code) against central finite differences of the forward functions."""
import numpy as np
import pytest

from paper_2309_10534_gb300 import gks as G

GAMMA = 1.4


def _conserved(rho, u, v, p):
    return np.array([rho, rho * u, rho * v, p / (GAMMA - 1) + 0.5 * rho * (u * u + v * v)])


def _flux_vec(x):
    F, dF = G.host_point_flux(2, x[0:4], x[4:8], x[8:12], x[12:16], x[16:20], x[20:24], 1e-3, tau="zero")
    return np.concatenate([F, dF])


def _fd_jacobian(f, x, h):
    cols = []
    for k in range(x.size):
        e = np.zeros_like(x)
        e[k] = h * max(1.0, abs(x[k]))
        cols.append((f(x + e) - f(x - e)) / (2 * e[k]))
    return np.stack(cols, axis=1)


SIDES = [
    # (rho, u, v, p) left / right: subsonic, opposite-sign normal velocities,
    # supersonic (large |z| tails of erfc), strong density ratio
    ((1.0, 0.3, -0.2, 1.0), (0.9, 0.25, -0.1, 0.95)),
    ((1.2, -0.4, 0.5, 0.8), (0.7, 0.6, -0.3, 1.3)),
    ((1.0, 2.5, 0.1, 0.4), (1.1, 2.4, 0.2, 0.45)),
    ((5.0, 0.1, 0.0, 3.0), (0.5, -0.2, 0.3, 0.2)),
]


@pytest.mark.parametrize("case", range(len(SIDES)))
def test_point_flux_vjp_matches_finite_differences(case):
    """Sec. 2 flux with tau = 0: J^T (gF, gdF) from the hand-written reverse
    equals the transposed central-difference Jacobian of the forward point
    flux to 1e-7 relative."""
    rng = np.random.default_rng(100 + case)
    (l, r) = SIDES[case]
    Wl, Wr = _conserved(*l), _conserved(*r)
    x = np.concatenate([Wl, 0.1 * rng.standard_normal(4), 0.1 * rng.standard_normal(4),
                        Wr, 0.1 * rng.standard_normal(4), 0.1 * rng.standard_normal(4)])
    J = _fd_jacobian(_flux_vec, x, 1e-6)
    for _ in range(3):
        g = rng.standard_normal(8)
        gl, gr = G.host_point_flux_vjp(x[0:4], x[4:8], x[8:12], x[12:16], x[16:20], x[20:24], g[:4], g[4:])
        got = np.concatenate([gl, gr])
        want = J.T @ g
        assert np.abs(got - want).max() <= 1e-7 * np.abs(want).max(), (got - want)


def test_point_flux_vjp_float32_close_to_float64():
    rng = np.random.default_rng(7)
    Wl, Wr = _conserved(1.0, 0.3, -0.2, 1.0), _conserved(0.9, 0.25, -0.1, 0.95)
    args = [Wl, 0.1 * rng.standard_normal(4), 0.1 * rng.standard_normal(4),
            Wr, 0.1 * rng.standard_normal(4), 0.1 * rng.standard_normal(4)]
    g = rng.standard_normal(8)
    a = np.concatenate(G.host_point_flux_vjp(*args, g[:4], g[4:]))
    b = np.concatenate(G.host_point_flux_vjp(*args, g[:4], g[4:], precision="fp32"))
    assert np.abs(a - b).max() <= 1e-4 * np.abs(a).max()


def _teno_vec(q):
    f, g, large = G.host_teno(q)
    return np.concatenate([f, g])


@pytest.mark.parametrize("q,large", [
    (np.array([1.0, 1.1, 1.25, 1.45, 1.7]), True),            # smooth: large stencil
    (np.array([1.0, 1.0, 1.0, 0.125, 0.125]), False),         # jump on the right: small stencils
    (np.array([0.1, 1.0, 1.02, 1.03, 1.05]), False),          # jump on the left
    (np.array([1.0, 0.2, 1.1, 0.3, 1.2]), None),              # oscillatory
])
def test_teno_transpose_is_the_frozen_linear_map(q, large):
    """Sec. 4.2 with the selection held fixed: the transpose returned by the
    adjoint equals J^T g for J the (exact, linear) map from the five cell
    averages to the face values/slopes and Gauss-point values/slopes."""
    f0, g0, lg = G.host_teno(q)
    if large is not None:
        assert lg == large
    J = _fd_jacobian(_teno_vec, q, 1e-7)
    # the selection did not move under the probe: J is the frozen linear map
    assert np.allclose(J @ q, _teno_vec(q), rtol=0, atol=1e-8 * np.abs(q).max())
    rng = np.random.default_rng(3)
    for _ in range(4):
        g = rng.standard_normal(8)
        gq, lg2 = G.host_teno_vjp(q, g[:4], g[4:])
        assert lg2 == lg
        want = J.T @ g
        assert np.abs(gq - want).max() <= 1e-8 * np.abs(want).max()
