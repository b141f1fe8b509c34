"""The library's per-point device arithmetic, compiled for the host, against
the FP64 oracle and high-precision quadrature (CPU only; the GPU parity tests
check the kernels themselves)."""
import shutil

import numpy as np
import pytest

import oracle as O

mp = pytest.importorskip("mpmath")


@pytest.fixture(scope="module")
def G():
    import os
    if not shutil.which("nvcc") and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    from paper_2309_10534_gb300 import build, gks
    build.build()
    return gks


def _phi(k, x):
    e = mp.e ** (-x)
    return [x - 1 + e, 2 - x - (x + 2) * e, x * x / 2 - x + 1 - e, 1 - e, -2 + (x + 2) * e, -(1 - e)][k]


@pytest.mark.parametrize("precision,tol", [("fp64", 2e-15), ("fp32", 3e-7)])
def test_time_coefficients_all_branches(G, precision, tol):
    """Folded coefficients (Sec. 2.2 applied to the integrals of Eq. 2.5)
    against 50-digit evaluation, across the series / closed-form switch."""
    mp.mp.dps = 50
    p = [1, 2, 2, 1, 2, 2]
    for s in [1e-4, 3e-3, 0.05, 0.24, 0.26, 0.7, 0.99, 1.01, 1.5, 1.99, 2.01, 3.0, 10.0, 99.0, 1e3]:
        cF, cD = G.host_time_coeffs(s, precision)
        S = mp.mpf(s)
        for k in range(6):
            eF = (4 * _phi(k, S / 2) - _phi(k, S)) / S ** p[k]
            eD = (_phi(k, S) - 2 * _phi(k, S / 2)) / S ** p[k]
            scale = max(abs(eF), abs(eD), 1)
            assert abs(cF[k] - eF) / scale < tol, (s, k, "F", cF[k], float(eF))
            assert abs(cD[k] - eD) / scale < tol, (s, k, "D", cD[k], float(eD))


def test_teno_matches_oracle(G):
    rng = np.random.default_rng(3)
    xs = [0.5, -0.5, -0.5 / np.sqrt(3), 0.5 / np.sqrt(3)]
    cases = [np.sin(0.3 * np.arange(5) + ph) + 2 for ph in rng.uniform(0, 6, 10)]
    cases += [rng.normal(size=5) for _ in range(30)]
    cases += [np.where(np.arange(5) < k, 1.0, 0.2) + 0.01 * rng.normal(size=5) for k in range(1, 5)]
    cases += [np.array([3.0] * 5), np.array([1.0, 1.0, 1.0, 2.0, 3.0])]
    for q in cases:
        val, dval, large, _ = O.teno_d(q, xs)
        faces, gauss, glarge = G.host_teno(q)
        assert glarge == large, q
        assert np.allclose(faces, [val[0], dval[0], val[1], dval[1]], rtol=0, atol=1e-13), q
        assert np.allclose(gauss, [val[2], dval[2], val[3], dval[3]], rtol=0, atol=1e-13), q
        f32, g32, l32 = G.host_teno(q, "fp32")
        if l32 == large:
            assert np.allclose(f32, faces, rtol=0, atol=2e-5 * (1 + abs(q).max()))
            # packed-pair selection of the float32 2-D sweep (lanes checked
            # against each other inside): the same choice, float32 values
            f2_, gp2, lp2 = G.host_teno(q, "fp32x2")
            assert lp2 == l32, q
            assert np.allclose(f2_, faces, rtol=0, atol=2e-5 * (1 + abs(q).max())), q
            assert np.allclose(gp2, g32, rtol=0, atol=2e-5 * (1 + abs(q).max())), q
            assert np.allclose(gp2, gauss, rtol=0, atol=2e-5 * (1 + abs(q).max())), q


def _state(dim, rng, rho=None):
    r = rho if rho is not None else np.exp(rng.uniform(-0.5, 0.5))
    U, V = rng.uniform(-0.8, 0.8, 2)
    p = np.exp(rng.uniform(-0.5, 0.5))
    E = p / 0.4 + 0.5 * r * (U * U + (V * V if dim == 2 else 0))
    return np.array([r, r * U, r * V if dim == 2 else 0.0, E])


@pytest.mark.parametrize("dim", [1, 2])
@pytest.mark.parametrize("tau,Pr", [("zero", 1.0), ("euler", 1.0), ("ns", 1.0), ("ns", 0.73)])
def test_point_flux_matches_oracle(G, dim, tau, Pr):
    """F and dF/dt of one point: the device arithmetic (closed-form slopes,
    folded time coefficients) against the oracle (moment-matrix solves,
    F(dt) and F(dt/2) combined as Sec. 2.2 prints); float32 within float32
    bounds."""
    rng = np.random.default_rng(7 + dim)
    P = O.make_problem(dim, 8, 8, tau=tau, mu=0.02, Pr=Pr)
    sl = [0, 1, 2, 3] if dim == 2 else [0, 1, 3]
    for trial in range(12):
        Wl, Wr = _state(dim, rng), _state(dim, rng)
        Wln, Wlt, Wrn, Wrt = (0.3 * rng.normal(size=4) for _ in range(4))
        if dim == 1:
            for a in (Wln, Wlt, Wrn, Wrt):
                a[2] = 0.0
            Wlt[:] = 0
            Wrt[:] = 0
        dt = 10 ** rng.uniform(-4, -2)
        Fd, Fh, rc = O.flux_point(P, Wl[sl], Wln[sl], Wlt[sl] if dim == 2 else None, Wr[sl], Wrn[sl],
                                  Wrt[sl] if dim == 2 else None, dt)
        assert rc == 0
        Fo = (4 * Fh - Fd) / dt
        dFo = 4 * (Fd - 2 * Fh) / dt ** 2
        F, dF = G.host_point_flux(dim, Wl, Wln, Wlt, Wr, Wrn, Wrt, dt, tau=tau, mu=0.02, Pr=Pr)
        scale = np.abs(Fo).max()
        assert np.allclose(F[sl], Fo, rtol=0, atol=1e-12 * scale), (trial, F[sl], Fo)
        # the oracle's dF/dt is a difference of two time integrals: its own
        # rounding is ~ eps |F| / dt
        assert np.allclose(dF[sl], dFo, rtol=1e-9, atol=1e-13 * scale / dt), (trial, dF[sl], dFo)
        F32, dF32 = G.host_point_flux(dim, Wl, Wln, Wlt, Wr, Wrn, Wrt, dt, precision="fp32", tau=tau,
                                      mu=0.02, Pr=Pr)
        assert np.allclose(F32[sl], Fo, rtol=0, atol=3e-6 * scale)
        # dF/dt in float32 within 2e-5 of the largest float64 component
        # (measured up to 8e-6)
        assert np.abs(dF32 - dF).max() <= 2e-5 * np.abs(dF).max()


def test_weno_ao_matches_oracle(G):
    """WENO5-AO (Sec. 3.2), host build of the device code vs the oracle:
    faces and Gauss points, values and xi-derivatives, float64 to 1e-14."""
    rng = np.random.default_rng(42)
    stencils = [np.array([1.0, 1.1, 1.25, 1.45, 1.7]), np.array([1.0, 1.0, 1.0, 0.125, 0.125]),
                np.array([0.1, 1.0, 1.02, 1.03, 1.05]), np.ones(5)] + [rng.normal(size=5) for _ in range(20)]
    g = 0.5 / np.sqrt(3.0)
    for q in stencils:
        f, gp = G.host_weno_ao(q)
        v, d, _ = O.weno_ao(q, [0.5, -0.5])
        vg, dg, _ = O.weno_ao(q, [-g, g])
        want_f = np.array([v[0], d[0], v[1], d[1]])
        want_g = np.array([vg[0], dg[0], vg[1], dg[1]])
        scale = max(1.0, np.abs(q).max())
        assert np.abs(f - want_f).max() <= 1e-14 * scale
        assert np.abs(gp - want_g).max() <= 1e-14 * scale
        f32, _ = G.host_weno_ao(q, precision="fp32")
        assert np.abs(f32 - want_f).max() <= 2e-6 * scale
        # packed-pair form of the float32 sweep (lanes checked against each other inside)
        fp2, gp2 = G.host_weno_ao(q, precision="fp32x2")
        assert np.abs(fp2 - want_f).max() <= 2e-6 * scale
        assert np.abs(gp2 - want_g).max() <= 2e-6 * scale


@pytest.mark.parametrize("teno5", [False, True])
def test_weno3_matches_oracle(G, teno5):
    """WENO5-Z and TENO5 face values with the slopes of Eq. (3.11), host build
    of the device code vs the oracle: float64 to 1e-13, float32 to 2e-6."""
    rng = np.random.default_rng(8)
    recon = "teno5" if teno5 else "weno_z"
    P = O.make_problem(1, 8, recon=recon)
    stencils = [np.array([1.0, 1.1, 1.25, 1.45, 1.7]), np.array([1.0, 1.0, 1.0, 0.125, 0.125]),
                np.array([0.1, 1.0, 1.02, 1.03, 1.05]), np.ones(5)] + [rng.normal(size=5) for _ in range(30)]
    for q in stencils:
        want = O.recon_faces(P, q)
        scale = max(1.0, np.abs(q).max())
        got = G.host_weno3(q, teno5)
        assert np.abs(got - want).max() <= 1e-13 * scale, (q, got, want)
        g32 = G.host_weno3(q, teno5, precision="fp32")
        assert np.abs(g32 - want).max() <= 2e-6 * scale, (q, g32, want)  # measured 4.4e-7


@pytest.mark.parametrize("teno5", [False, True])
def test_weno3_gauss_matches_oracle(G, teno5):
    """The 2-D conventional path's tangential WENO5-Z / TENO5 at the Gauss
    points (values and the blend's derivative), host build of the device
    code against the oracle: float64 to 1e-13, float32 to 2e-6."""
    rng = np.random.default_rng(9)
    g = 0.5 / np.sqrt(3.0)
    stencils = [np.array([1.0, 1.1, 1.25, 1.45, 1.7]), np.array([1.0, 1.0, 1.0, 0.125, 0.125]),
                np.ones(5)] + [rng.normal(size=5) for _ in range(30)]
    for q in stencils:
        v, d = O.weno3_dv(q, [-g, g], teno5=teno5)
        want = np.array([v[0], d[0], v[1], d[1]])
        scale = max(1.0, np.abs(q).max())
        assert np.abs(G.host_weno3_gauss(q, teno5) - want).max() <= 1e-13 * scale, q
        assert np.abs(G.host_weno3_gauss(q, teno5, precision="fp32") - want).max() <= 2e-6 * scale, q


@pytest.mark.parametrize("dim", [1, 2])
def test_merge_matches_half_space_quadrature(G, dim):
    """The line-averaged equilibrium state of the conventional path (Step 2):
    the kinetic merge rho_l <psi>_{u>0} + rho_r <psi>_{u<0} against adaptive
    quadrature of the Maxwellians over the half spaces (v and the internal
    degrees of freedom integrated in closed form), float64 to 1e-10."""
    from scipy.integrate import quad
    gamma = 1.4
    K = 3.0 if dim == 2 else 4.0
    rng = np.random.default_rng(10 + dim)
    for _ in range(8):
        sides = []
        for _s in range(2):
            rho, p = np.exp(rng.uniform(-0.5, 0.5, 2))
            U, V = rng.uniform(-1.5, 1.5, 2)
            V = V if dim == 2 else 0.0
            E = p / (gamma - 1) + 0.5 * rho * (U * U + V * V)
            sides.append((rho, U, V, p, np.array([rho, rho * U, rho * V, E])))
        want = np.zeros(4)
        for (rho, U, V, p, _W), (lo, hi) in zip(sides, ((0.0, np.inf), (-np.inf, 0.0))):
            lam = rho / (2 * p)
            f = lambda u, k: u ** k * np.sqrt(lam / np.pi) * np.exp(-lam * (u - U) ** 2)
            m = [quad(f, lo, hi, args=(k,), epsabs=0, epsrel=1e-13)[0] for k in range(3)]
            vv = V * V + 1 / (2 * lam) if dim == 2 else 0.0
            want += rho * np.array([m[0], m[1], V * m[0], 0.5 * (m[2] + m[0] * vv + m[0] * K / (2 * lam))])
        got = G.host_merge(dim, sides[0][4], sides[1][4])
        assert np.allclose(got, want, rtol=1e-10, atol=1e-12), (got, want)
    # equal states: the two half spaces add up to the state
    W = sides[0][4]
    assert np.allclose(G.host_merge(dim, W, W), W, rtol=1e-13)


@pytest.mark.parametrize("dim", [1, 2])
@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32", 2e-5)])
def test_char_face_matches_oracle(G, dim, precision, tol):
    """The kernels' characteristic-variable face reconstruction (closed-form
    L and R) against the oracle's pieces: its basis (R's columns from the
    eigenvectors, L by Gaussian elimination) and its fitted TENO-D per
    field, on smooth stencils and on stencils across a jump."""
    rng = np.random.default_rng(40 + dim)
    nv = dim + 2
    for trial in range(12):
        rho = rng.uniform(0.3, 2.0, 6)
        U = rng.uniform(-1, 1, 6)
        V = rng.uniform(-1, 1, 6) if dim == 2 else np.zeros(6)
        p = rng.uniform(0.3, 2.0, 6)
        if trial % 2 == 0:  # smooth stencil
            x = np.arange(6)
            rho, U, V, p = 1 + 0.05 * x, 0.2 + 0.01 * x, (0.1 - 0.02 * x) * (dim == 2), 1 + 0.03 * x
        E = p / 0.4 + 0.5 * rho * (U * U + V * V)
        w4 = np.stack([rho, rho * U, rho * V, E], axis=1)
        got = G.host_char_face(dim, w4, precision=precision)
        act = [0, 1, 2, 3] if dim == 2 else [0, 1, 3]
        Q = w4[:, act]
        R, L = O.char_basis(dim, 1.4, 0.5 * (Q[2] + Q[3]))
        C = Q @ L.T
        cl, cdl, cr, cdr = (np.zeros(nv) for _ in range(4))
        for k in range(nv):
            v, d, _, _ = O.teno_d(C[0:5, k], [0.5])
            cl[k], cdl[k] = v[0], d[0]
            v, d, _, _ = O.teno_d(C[1:6, k], [-0.5])
            cr[k], cdr[k] = v[0], d[0]
        for row, ref in zip(got, (R @ cl, R @ cdl, R @ cr, R @ cdr)):
            scale = np.abs(Q).max()
            assert np.abs(row[act] - ref).max() <= tol * scale, (trial, row[act], ref)
            if dim == 1:
                assert row[2] == 0.0


def test_float32_state_test_needs_resolvable_internal_energy(G):
    """The kernels' state test (before a point's flux, and on the cell average
    a positivity fallback takes): both precisions reject rho <= 0 and p <= 0;
    float32 also rejects a state whose internal energy is below 1e-4 of E
    (its float32 pressure has no reliable digits, and the micro slopes scale
    that error by lambda^2), which float64 accepts."""
    def state(rho, u, v, frac):
        ke = 0.5 * rho * (u * u + v * v)
        return [rho, rho * u, rho * v, ke / (1.0 - frac)]  # internal energy = frac * E
    for dim, v in ((2, -0.27), (1, 0.0)):
        cold, warm = state(1.7, 0.65, v, 5e-5), state(1.7, 0.65, v, 2e-4)
        assert G.host_physical(dim, cold, "fp64") and not G.host_physical(dim, cold, "fp32")
        assert G.host_physical(dim, warm, "fp64") and G.host_physical(dim, warm, "fp32")
        for bad in ([1.0, 1.0, 0.0, 0.4], [-1.0, 0.0, 0.0, 2.5], [1.0, 0.0, 0.0, 0.0]):
            assert not G.host_physical(dim, bad, "fp64") and not G.host_physical(dim, bad, "fp32")
        assert G.host_physical(dim, [1.4, 0.0, 0.0, 2.5], "fp32")
