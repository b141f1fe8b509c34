"""FP64 CPU oracle of the TENO-D gas-kinetic scheme -- TEST INFRASTRUCTURE.

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It wraps ``liboracle.so`` (plain C,
built by ``oracle/build.py``) with ctypes and numpy; it shares no code with
the CUDA library.  Arrays are conserved variables in SoA layout
``[nvar][ny][nx]`` (1-D: ``[3][1][nx]`` or ``[3][nx]``), float64.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import build as _build

_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        _lib = C.CDLL(path)
        _declare(_lib)
    return _lib


class Problem(C.Structure):
    """Mirror of ``or_problem`` (oracle/gks_oracle.h)."""

    _fields_ = [
        ("dim", C.c_int), ("nx", C.c_int), ("ny", C.c_int),
        ("dx", C.c_double), ("dy", C.c_double),
        ("bc", C.c_int * 4),
        ("gamma", C.c_double), ("mu", C.c_double), ("Pr", C.c_double),
        ("tau_mode", C.c_int), ("c1", C.c_double), ("c2", C.c_double), ("cfl", C.c_double),
        ("eps", C.c_double), ("qpow", C.c_double),
        ("ct1", C.c_double), ("ct2", C.c_double), ("ct1_t", C.c_double), ("ct2_t", C.c_double),
        ("positivity_fallback", C.c_int),
        ("recon", C.c_int), ("d_hi", C.c_double), ("d_lo", C.c_double), ("eps_ao", C.c_double),
        ("merge", C.c_int), ("zpow", C.c_double),
        ("t", C.c_double), ("bc_in", C.c_double * 4), ("bc_pre", C.c_double * 4),
        ("shock_x0", C.c_double), ("shock_theta", C.c_double), ("shock_speed", C.c_double),
        ("charvars", C.c_int), ("ox", C.c_double), ("oy", C.c_double),
    ]


BC = {"periodic": 0, "zerograd": 1, "symmetry": 2, "noslip": 3, "reflect": 4,
      "inflow": 5, "wall_after_x0": 6, "moving_shock": 7}
TAU = {"zero": 0, "euler": 1, "ns": 2}
RECON = {"teno_d": 0, "weno_ao": 1, "weno_z": 2, "teno5": 3}
MERGE = {"kinetic": 0, "average": 1}


def make_problem(dim, nx, ny=1, *, lx=1.0, ly=1.0, bc=("zerograd",) * 4, gamma=1.4, mu=0.0, Pr=1.0,
                 tau="euler", c1=0.01, c2=1.0, cfl=0.5, eps=1e-40, q=None, ct1=1e-7, ct2=1e-5,
                 ct1_t=None, ct2_t=None, positivity_fallback=1, recon="teno_d", d_hi=0.85, d_lo=0.85,
                 eps_ao=1e-8, merge="kinetic", zpow=1.0, t=0.0, bc_in=None, bc_pre=None, shock_x0=0.0,
                 shock_theta=np.pi / 3, shock_speed=0.0, charvars=0, ox=0.0, oy=0.0) -> Problem:
    p = Problem()
    p.dim, p.nx, p.ny = dim, nx, (ny if dim == 2 else 1)
    p.dx = lx / nx
    p.dy = (ly / ny) if dim == 2 else 1.0
    for k in range(4):
        b = bc[k]
        p.bc[k] = BC[b] if isinstance(b, str) else int(b)
    p.gamma, p.mu, p.Pr = gamma, mu, Pr
    p.tau_mode = TAU[tau] if isinstance(tau, str) else int(tau)
    p.c1, p.c2, p.cfl = c1, c2, cfl
    if q is None:  # TENO-D: q = 7 (Eq. 4.5); TENO5: q = 6 (Eq. 4.1)
        q = 6.0 if recon in ("teno5", 3) else 7.0
    p.eps, p.qpow, p.ct1, p.ct2 = eps, q, ct1, ct2
    p.ct1_t = ct1 if ct1_t is None else ct1_t
    p.ct2_t = ct2 if ct2_t is None else ct2_t
    p.positivity_fallback = positivity_fallback
    p.recon = RECON[recon] if isinstance(recon, str) else int(recon)
    p.d_hi, p.d_lo, p.eps_ao = d_hi, d_lo, eps_ao
    p.merge = MERGE[merge] if isinstance(merge, str) else int(merge)
    p.zpow = zpow
    # state-setting boundary rules: conserved states (rho, rho u, [rho v,] E)
    # stored as 4 slots with the energy last
    for name, st in (("bc_in", bc_in), ("bc_pre", bc_pre)):
        if st is not None:
            st = list(st)
            if len(st) == 3:
                st = [st[0], st[1], 0.0, st[2]]
            getattr(p, name)[:] = [float(x) for x in st]
    p.t = t
    p.shock_x0, p.shock_theta, p.shock_speed = shock_x0, shock_theta, shock_speed
    p.charvars = int(charvars)
    p.ox, p.oy = float(ox), float(oy)
    return p


_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int)
_lp = C.POINTER(C.c_long)


def _declare(L):
    L.or_fit_matrix.argtypes = [C.c_int, _ip, _dp]
    L.or_fit_matrix.restype = C.c_int
    L.or_poly_eval.argtypes = [C.c_int, _dp, C.c_double]
    L.or_poly_eval.restype = C.c_double
    L.or_poly_deriv.argtypes = [C.c_int, _dp, C.c_double]
    L.or_poly_deriv.restype = C.c_double
    L.or_beta.argtypes = [C.c_int, _dp]
    L.or_beta.restype = C.c_double
    L.or_teno_d.argtypes = [_dp, C.c_double, C.c_double, C.c_double, C.c_double, C.c_int, _dp, _dp,
                            _dp, _ip]
    L.or_teno_d.restype = C.c_int
    L.or_weno_ao.argtypes = [_dp, C.c_double, C.c_double, C.c_double, C.c_int, _dp, _dp, _dp, _dp]
    L.or_weno_ao.restype = None
    L.or_weno3.argtypes = [_dp, C.c_int, C.c_double, C.c_double, C.c_double, C.c_double, C.c_int, _dp, _dp, _dp]
    L.or_weno3.restype = C.c_int
    L.or_weno3_dv.argtypes = [_dp, C.c_int, C.c_double, C.c_double, C.c_double, C.c_double, C.c_int, _dp, _dp, _dp]
    L.or_weno3_dv.restype = C.c_int
    L.or_recon_faces.argtypes = [C.POINTER(Problem), _dp, _dp]
    L.or_recon_faces.restype = C.c_int
    L.or_moments_u.argtypes = [C.c_double, C.c_double, C.c_int, C.c_int, _dp]
    L.or_moments_u.restype = None
    L.or_micro_slope.argtypes = [C.c_int, C.c_double, C.c_double, C.c_double, C.c_double, _dp, _dp]
    L.or_micro_slope.restype = C.c_int
    L.or_time_coeffs.argtypes = [C.c_double, C.c_double, _dp]
    L.or_time_coeffs.restype = None
    L.or_char_basis.argtypes = [C.c_int, C.c_double, _dp, _dp, _dp]
    L.or_char_basis.restype = C.c_int
    L.or_face_flux.argtypes = [C.POINTER(Problem), _dp, C.c_int, C.c_int, C.c_int, C.c_double, _dp, _dp, _lp]
    L.or_face_flux.restype = C.c_int
    L.or_flux_point.argtypes = [C.POINTER(Problem)] + [_dp] * 8 + [C.c_double, _dp, _dp]
    L.or_flux_point.restype = C.c_int
    L.or_stage1.argtypes = [C.POINTER(Problem), _dp, C.c_double, _dp, _lp]
    L.or_stage1.restype = C.c_int
    L.or_step.argtypes = [C.POINTER(Problem), _dp, C.c_double, _dp, _lp]
    L.or_step.restype = C.c_int
    L.or_dt.argtypes = [C.POINTER(Problem), _dp]
    L.or_dt.restype = C.c_double
    L.or_run.argtypes = [C.POINTER(Problem), _dp, C.c_double, C.c_long, _lp, _dp, _lp]
    L.or_run.restype = C.c_int
    L.or_fill_ghosts.argtypes = [C.POINTER(Problem), _dp]
    L.or_fill_ghosts.restype = None
    L.or_trace_selections.argtypes = [C.c_void_p, C.c_long]
    L.or_trace_selections.restype = None
    L.or_trace_length.argtypes = []
    L.or_trace_length.restype = C.c_long


def _d(a):
    return a.ctypes.data_as(_dp)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def fit_matrix(offsets) -> np.ndarray:
    offs = np.ascontiguousarray(offsets, dtype=np.int32)
    n = len(offs)
    out = np.zeros((n, n))
    rc = lib().or_fit_matrix(n, offs.ctypes.data_as(_ip), _d(out))
    if rc:
        raise RuntimeError("fit failed")
    return out


def poly_eval(coef, xi):
    c = _f64(coef)
    return lib().or_poly_eval(len(c) - 1, _d(c), float(xi))


def poly_deriv(coef, xi):
    c = _f64(coef)
    return lib().or_poly_deriv(len(c) - 1, _d(c), float(xi))


def beta(coef) -> float:
    c = _f64(coef)
    return lib().or_beta(len(c) - 1, _d(c))


def teno_d(q5, xs, eps=1e-40, q=7.0, ct1=1e-7, ct2=1e-5):
    """TENO-D of Sec. 4.2 on five cell averages; returns (val, dval, large, sel)."""
    q5 = _f64(q5)
    xs = _f64(np.atleast_1d(xs))
    val = np.zeros(len(xs))
    dval = np.zeros(len(xs))
    sel = np.zeros(3, dtype=np.int32)
    large = lib().or_teno_d(_d(q5), eps, q, ct1, ct2, len(xs), _d(xs), _d(val), _d(dval),
                            sel.ctypes.data_as(_ip))
    return val, dval, bool(large), sel


def weno_ao(q5, xs, eps=1e-8, d_hi=0.85, d_lo=0.85):
    """WENO5-AO of Sec. 3.2 on five cell averages; returns (val, dval, wbar[4])."""
    q5 = _f64(q5)
    xs = _f64(np.atleast_1d(xs))
    val = np.zeros(len(xs))
    dval = np.zeros(len(xs))
    wbar = np.zeros(4)
    lib().or_weno_ao(_d(q5), eps, d_hi, d_lo, len(xs), _d(xs), _d(val), _d(dval), _d(wbar))
    return val, dval, wbar


def weno3(q5, xs, teno5=False, eps=None, zpow=1.0, q=6.0, ct=1e-7):
    """WENO5-Z (Sec. 3.1) or TENO5 (Sec. 4.1) values of five cell averages at
    the points xs; returns (val, wbar[3] at the last point)."""
    q5 = _f64(q5)
    xs = _f64(np.atleast_1d(xs))
    if eps is None:
        eps = 1e-40 if teno5 else 1e-8
    val = np.zeros(len(xs))
    wbar = np.zeros(3)
    if lib().or_weno3(_d(q5), int(bool(teno5)), eps, zpow, q, ct, len(xs), _d(xs), _d(val), _d(wbar)):
        raise ValueError("no linear weights at these points")
    return val, wbar


def weno3_dv(q5, xs, teno5=False, eps=None, zpow=1.0, q=6.0, ct=1e-7):
    """WENO5-Z / TENO5 values and xi-derivatives (the same blend) at xs."""
    q5 = _f64(q5)
    xs = _f64(np.atleast_1d(xs))
    if eps is None:
        eps = 1e-40 if teno5 else 1e-8
    val = np.zeros(len(xs))
    dval = np.zeros(len(xs))
    if lib().or_weno3_dv(_d(q5), int(bool(teno5)), eps, zpow, q, ct, len(xs), _d(xs), _d(val), _d(dval)):
        raise ValueError("no linear weights at these points")
    return val, dval


def recon_faces(P: Problem, q5):
    """The problem's normal reconstruction of one cell: (v(+1/2), dv/dxi(+1/2),
    v(-1/2), dv/dxi(-1/2))."""
    q5 = _f64(q5)
    out = np.zeros(4)
    lib().or_recon_faces(C.byref(P), _d(q5), _d(out))
    return out


def moments_u(U, lam, half=0, nmax=6):
    m = np.zeros(nmax + 1)
    lib().or_moments_u(U, lam, half, nmax, _d(m))
    return m


def micro_slope(dim, K, U, V, lam, b):
    b = _f64(b)
    a = np.zeros(dim + 2)
    if lib().or_micro_slope(dim, K, U, V, lam, _d(b), _d(a)):
        raise RuntimeError("singular moment matrix")
    return a


def face_flux(P: Problem, Wg, direction, ic, jc, dt):
    """(F(dt), F(dt/2), fallbacks) of one face of a ghost-filled array
    [nvar][ny+6][nx+6] (ghosted indices of the left / lower cell)."""
    Wg = _f64(Wg)
    nv = P.dim + 2
    Fd, Fh = np.zeros(nv), np.zeros(nv)
    nfb = C.c_long(0)
    if lib().or_face_flux(C.byref(P), _d(Wg), int(direction), int(ic), int(jc), float(dt), _d(Fd), _d(Fh),
                          C.byref(nfb)):
        raise RuntimeError("non-physical state")
    return Fd, Fh, nfb.value


def char_basis(dim, gamma, Wm):
    """(R, L) of the normal Euler flux Jacobian at the conserved state Wm
    (local frame; Sec. 3.1, the characteristic variables): R's columns are
    the right eigenvectors, L = R^-1."""
    nv = dim + 2
    Wm = _f64(Wm)
    R = np.zeros((nv, nv))
    Lm = np.zeros((nv, nv))
    if lib().or_char_basis(dim, gamma, _d(Wm), _d(R), _d(Lm)):
        raise ValueError("non-physical state")
    return R, Lm


def time_coeffs(delta, tau):
    q = np.zeros(6)
    lib().or_time_coeffs(delta, tau, _d(q))
    return q


def flux_point(P: Problem, Wl, Wln, Wlt, Wr, Wrn, Wrt, dt, Wcl=None, Wcr=None):
    """Time-integrated flux at one point (local frame) for delta = dt, dt/2."""
    nv = P.dim + 2
    args = []
    keep = []
    for a in (Wl, Wln, Wlt, Wr, Wrn, Wrt, Wcl, Wcr):
        if a is None:
            args.append(None)
        else:
            arr = _f64(a)
            keep.append(arr)
            args.append(_d(arr))
    Fd = np.zeros(nv)
    Fh = np.zeros(nv)
    rc = lib().or_flux_point(C.byref(P), *args, dt, _d(Fd), _d(Fh))
    return Fd, Fh, rc


def _state(P, W):
    nv = P.dim + 2
    W = _f64(W)
    if W.size != nv * P.nx * P.ny:
        raise ValueError("state has %d values, expected %d" % (W.size, nv * P.nx * P.ny))
    return W


def stage1(P: Problem, W, dt):
    W = _state(P, W)
    out = np.empty_like(W)
    nfb = C.c_long(0)
    rc = lib().or_stage1(C.byref(P), _d(W), dt, _d(out), C.byref(nfb))
    if rc:
        raise RuntimeError("oracle stage1 failed (%d)" % rc)
    return out


def step(P: Problem, W, dt, return_fallbacks=False):
    W = _state(P, W)
    out = np.empty_like(W)
    nfb = C.c_long(0)
    rc = lib().or_step(C.byref(P), _d(W), dt, _d(out), C.byref(nfb))
    if rc:
        raise RuntimeError("oracle step failed (%d)" % rc)
    return (out, nfb.value) if return_fallbacks else out


def dt(P: Problem, W) -> float:
    W = _state(P, W)
    return lib().or_dt(C.byref(P), _d(W))


def run(P: Problem, W, t_end, max_steps=0):
    """Advance with CFL steps to t_end; returns (W, steps, t, fallbacks)."""
    W = _state(P, W).copy()
    s = C.c_long(0)
    t = C.c_double(0.0)
    nfb = C.c_long(0)
    rc = lib().or_run(C.byref(P), _d(W), t_end, max_steps, C.byref(s), C.byref(t), C.byref(nfb))
    if rc:
        raise RuntimeError("oracle run failed (%d)" % rc)
    return W, s.value, t.value, nfb.value


def fill_ghosts(P: Problem, Wg):
    """Fill the three ghost layers of a ghosted array in place."""
    if not (Wg.dtype == np.float64 and Wg.flags.c_contiguous):
        raise ValueError("need contiguous float64")
    lib().or_fill_ghosts(C.byref(P), _d(Wg))
    return Wg


def trace_selections(fn, cap=1 << 24):
    """Call fn() with the oracle's TENO-D selection trace on (one byte per
    or_teno_d evaluation, in call order: delta_{3,1} + 2 delta_{0,2} +
    4 delta_{1,2} + 8 delta_{2,2}, Eqs. 4.7 and 4.12); returns (fn's result,
    the trace as uint8).  Two runs whose traces differ took a different
    stencil somewhere."""
    L = lib()
    buf = np.zeros(cap, dtype=np.uint8)
    L.or_trace_selections(buf.ctypes.data, cap)
    try:
        out = fn()
        n = L.or_trace_length()
    finally:
        L.or_trace_selections(None, 0)
    if n > cap:
        raise RuntimeError("selection trace overflow: %d calls > %d" % (n, cap))
    return out, buf[:n].copy()


def internal_dof(dim, gamma):
    """K of Sec. 2.1 (2-D) and its 1-D counterpart."""
    return (5 - 3 * gamma) / (gamma - 1) + 1 if dim == 2 else (3 - gamma) / (gamma - 1)


__all__ = [n for n in dir() if not n.startswith("_")]
