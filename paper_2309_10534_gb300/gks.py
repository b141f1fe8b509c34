"""ctypes binding of libgks.so (include/gks.h): the same entry points, plus a
small ``Solver`` class that only marshals arguments.

Every computation runs in the CUDA library; there is no CPU path.  Loading
fails loudly when ``libgks.so`` has not been built.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libgks.so")

GKS_OK, GKS_EINVAL, GKS_ENOMEM, GKS_ECUDA, GKS_ENONPHYSICAL, GKS_ETIMEOUT, GKS_EUNSUPPORTED = range(7)
BC = {"periodic": 0, "zerograd": 1, "symmetry": 2, "noslip": 3, "reflect": 4,
      "inflow": 5, "wall_after_x0": 6, "moving_shock": 7}
PRECISION = {"fp64": 0, "fp32": 1, "fp32x2": 2}
TAU = {"zero": 0, "euler": 1, "ns": 2}
RECON = {"teno_d": 0, "weno_ao": 1, "weno_z": 2, "teno5": 3}
MERGE = {"kinetic": 0, "average": 1}


class GridDesc(C.Structure):
    _fields_ = [("dim", C.c_int), ("nx", C.c_int), ("ny", C.c_int),
                ("x0", C.c_double), ("x1", C.c_double), ("y0", C.c_double), ("y1", C.c_double),
                ("bc", C.c_int * 4), ("precision", C.c_int)]


class Gas(C.Structure):
    _fields_ = [("gamma", C.c_double), ("mu", C.c_double), ("Pr", C.c_double)]


class BoundaryStates(C.Structure):
    _fields_ = [("inflow", C.c_double * 4), ("pre", C.c_double * 4), ("shock_x0", C.c_double),
                ("shock_theta", C.c_double), ("shock_speed", C.c_double)]


class Scheme(C.Structure):
    _fields_ = [("cfl", C.c_double), ("c1", C.c_double), ("c2", C.c_double),
                ("ct1", C.c_double), ("ct2", C.c_double), ("ct1_t", C.c_double), ("ct2_t", C.c_double),
                ("eps", C.c_double), ("q", C.c_int), ("tau_mode", C.c_int),
                ("positivity_fallback", C.c_int), ("recon", C.c_int), ("d_hi", C.c_double),
                ("d_lo", C.c_double), ("eps_ao", C.c_double), ("merge", C.c_int), ("charvars", C.c_int)]


GKS_HOST_MEMORY, GKS_DEVICE_MEMORY, GKS_HOST_PINNED_ASYNC = 0, 1, 2


def _host_ptr(W, shape):
    """Address of a contiguous float64 host array of the state's size (a
    CPU torch tensor or a numpy array)."""
    if hasattr(W, "data_ptr"):
        if W.is_cuda or W.dtype.itemsize != 8 or not W.is_contiguous() or W.numel() != int(np.prod(shape)):
            raise ValueError("need a contiguous float64 CPU tensor of the state's size")
        return W.data_ptr()
    if not (isinstance(W, np.ndarray) and W.dtype == np.float64 and W.flags.c_contiguous and W.size == int(np.prod(shape))):
        raise ValueError("need a contiguous float64 array of the state's size")
    return W.ctypes.data


class Diag(C.Structure):
    _fields_ = [("error_word", C.c_uint), ("fallbacks", C.c_longlong), ("t", C.c_double),
                ("steps", C.c_longlong), ("dt", C.c_double)]


class FlipCount(C.Structure):
    _fields_ = [("normal_flips", C.c_longlong), ("normal_selections", C.c_longlong),
                ("tangential_flips", C.c_longlong), ("tangential_selections", C.c_longlong),
                ("unresolved_flips", C.c_longlong)]


class FlopModel(C.Structure):
    _fields_ = [("flops_per_cell_update", C.c_double), ("flops_per_cell_sweep", C.c_double),
                ("transcendentals_per_cell_update", C.c_double), ("divides_per_cell_update", C.c_double),
                ("sqrt_per_cell_update", C.c_double), ("fp64_flops_per_cell_update", C.c_double)]


class GKSError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s (status %d): %s" % (_status_string(status), status, msg))
        self.status = status


_lib = None
_vp = C.c_void_p
_dp = C.POINTER(C.c_double)


def lib():
    """Load libgks.so; raises if it is missing (no fallback exists)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError("libgks.so is not built (run paper_2309_10534_gb300/build.py)")
        L = C.CDLL(LIB_PATH)
        sig = {
            "gks_create": ([C.POINTER(GridDesc), C.POINTER(_vp)], C.c_int),
            "gks_destroy": ([_vp], None),
            "gks_set_gas": ([_vp, C.POINTER(Gas)], C.c_int),
            "gks_set_scheme": ([_vp, C.POINTER(Scheme)], C.c_int),
            "gks_set_stream": ([_vp, _vp], C.c_int),
            "gks_set_state": ([_vp, _vp, C.c_int], C.c_int),
            "gks_get_state": ([_vp, _vp, C.c_int], C.c_int),
            "gks_get_buffer": ([_vp, C.c_int, _vp, C.c_int], C.c_int),
            "gks_compute_dt": ([_vp, _dp], C.c_int),
            "gks_stage": ([_vp, C.c_int, C.c_double], C.c_int),
            "gks_step": ([_vp, C.c_double], C.c_int),
            "gks_advance_to": ([_vp, C.c_double, C.c_longlong, C.POINTER(C.c_longlong), _dp], C.c_int),
            "gks_get_diagnostics": ([_vp, C.POINTER(Diag)], C.c_int),
            "gks_selection_flips": ([_vp, C.POINTER(FlipCount)], C.c_int),
            "gks_last_error": ([_vp], C.c_char_p),
            "gks_status_string": ([C.c_int], C.c_char_p),
            "gks_kernel_launches": ([_vp], C.c_longlong),
            "gks_profile_enable": ([_vp, C.c_int], C.c_int),
            "gks_profile_read": ([_vp, C.c_int, C.POINTER(C.c_longlong), _dp], C.c_int),
            "gks_count_flops": ([C.c_int, C.c_int, C.c_int, C.c_double, C.POINTER(FlopModel)], C.c_int),
        }
        for name, (args, res) in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = res
        _lib = L
    return _lib


def _status_string(s):
    try:
        return lib().gks_status_string(s).decode()
    except Exception:  # pragma: no cover - only when the library is absent
        return "status"


def default_scheme(**kw) -> Scheme:
    s = Scheme(cfl=0.5, c1=0.01, c2=1.0, ct1=1e-7, ct2=1e-5, ct1_t=1e-7, ct2_t=1e-5, eps=1e-40, q=7,
               tau_mode=TAU["euler"], positivity_fallback=1, recon=0, d_hi=0.85, d_lo=0.85, eps_ao=1e-8,
               merge=0, charvars=0)
    if kw.get("recon") in ("teno5", 3) and "q" not in kw:
        kw = dict(kw, q=6)  # TENO5's power (Eq. 4.1); TENO-D's default is 7
    for k, v in kw.items():
        if k == "tau" or k == "tau_mode":
            v = TAU[v] if isinstance(v, str) else int(v)
            k = "tau_mode"
        if k == "recon":
            v = RECON[v] if isinstance(v, str) else int(v)
        if k == "merge":
            v = MERGE[v] if isinstance(v, str) else int(v)
        setattr(s, k, v)
    if "ct1" in kw and "ct1_t" not in kw:
        s.ct1_t = kw["ct1"]
    if "ct2" in kw and "ct2_t" not in kw:
        s.ct2_t = kw["ct2"]
    return s


class Solver:
    """One grid context.  Arrays: conserved variables, float64,
    [nvar][ny][nx] (1-D: [3][1][nx] or [3][nx]); numpy (host) or a CUDA
    torch tensor (device, passed by data_ptr)."""

    def __init__(self, dim, nx, ny=1, *, lx=1.0, ly=1.0, bc=("zerograd",) * 4, precision="fp64",
                 gamma=1.4, mu=0.0, Pr=1.0, tau="euler", cfl=0.5, **scheme):
        L = lib()
        d = GridDesc()
        d.dim, d.nx, d.ny = dim, nx, (ny if dim == 2 else 1)
        d.x0, d.x1, d.y0, d.y1 = 0.0, lx, 0.0, (ly if dim == 2 else 1.0)
        for k in range(4):
            d.bc[k] = BC[bc[k]] if isinstance(bc[k], str) else int(bc[k])
        d.precision = PRECISION[precision] if isinstance(precision, str) else int(precision)
        h = _vp()
        self._check(L.gks_create(C.byref(d), C.byref(h)), None)
        self.h = h
        self.dim, self.nx, self.ny = dim, nx, d.ny
        self.nvar = dim + 2
        self.set_gas(gamma=gamma, mu=mu, Pr=Pr)
        self.set_scheme(cfl=cfl, tau=tau, **scheme)

    # -- plumbing
    def _check(self, status, h="self"):
        if status != GKS_OK:
            handle = self.h if h == "self" else h
            msg = lib().gks_last_error(handle).decode() if handle else ""
            raise GKSError(status, msg)

    def close(self):
        if getattr(self, "h", None):
            lib().gks_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def shape(self):
        return (self.nvar, self.ny, self.nx)

    def _host(self, W):
        W = np.ascontiguousarray(W, dtype=np.float64)
        if W.size != self.nvar * self.ny * self.nx:
            raise ValueError("state has %d values, expected %d" % (W.size, self.nvar * self.ny * self.nx))
        return W

    # -- API
    def set_gas(self, gamma=1.4, mu=0.0, Pr=1.0):
        self._check(lib().gks_set_gas(self.h, C.byref(Gas(gamma, mu, Pr))))

    def set_scheme(self, **kw):
        self._check(lib().gks_set_scheme(self.h, C.byref(default_scheme(**kw))))

    def set_boundary_states(self, bc_in=None, bc_pre=None, shock_x0=0.0, shock_theta=np.pi / 3, shock_speed=0.0):
        """States of the state-setting boundary rules (inflow, wall after x0,
        moving shock): conserved (rho, rho u, rho v, E) (1-D: (rho, rho u, E))."""
        b = BoundaryStates()
        for dst, st in ((b.inflow, bc_in), (b.pre, bc_pre)):
            if st is not None:
                st = [float(x) for x in st]
                if len(st) == 3:
                    st = [st[0], st[1], 0.0, st[2]]
                dst[:] = st
        b.shock_x0, b.shock_theta, b.shock_speed = shock_x0, shock_theta, shock_speed
        L = lib()
        L.gks_set_boundary_states.argtypes = [_vp, C.POINTER(BoundaryStates)]
        L.gks_set_boundary_states.restype = C.c_int
        self._check(L.gks_set_boundary_states(self.h, C.byref(b)))

    def set_stream(self, stream_handle: int):
        self._check(lib().gks_set_stream(self.h, _vp(stream_handle)))

    def set_state(self, W):
        if hasattr(W, "data_ptr"):  # torch tensor on the device
            self._check(lib().gks_set_state(self.h, _vp(W.data_ptr()), 1))
        else:
            W = self._host(W)
            self._check(lib().gks_set_state(self.h, W.ctypes.data_as(_vp), 0))

    def set_state_async(self, W):
        """Enqueue the copy-in of W (page-locked host memory: a pinned CPU
        torch tensor, or a numpy view of one) on the solver's stream and
        return at once (GKS_HOST_PINNED_ASYNC); W must stay unchanged until
        the stream has passed the copy."""
        self._check(lib().gks_set_state(self.h, _vp(_host_ptr(W, self.shape)), GKS_HOST_PINNED_ASYNC))

    def get_state_async(self, out):
        """Enqueue the copy-out into out (page-locked host memory, state
        shape) on the solver's stream and return at once; out is valid once
        the stream has passed the copy."""
        self._check(lib().gks_get_state(self.h, _vp(_host_ptr(out, self.shape)), GKS_HOST_PINNED_ASYNC))

    def get_state(self, out=None):
        if out is not None and hasattr(out, "data_ptr"):
            self._check(lib().gks_get_state(self.h, _vp(out.data_ptr()), 1))
            return out
        W = np.empty(self.shape)
        self._check(lib().gks_get_state(self.h, W.ctypes.data_as(_vp), 0))
        return W

    def get_state_into(self, out):
        """Copy the state into a caller-owned contiguous float64 host array."""
        if not (out.dtype == np.float64 and out.flags.c_contiguous and out.size == self.nvar * self.ny * self.nx):
            raise ValueError("need a contiguous float64 array of the state's size")
        self._check(lib().gks_get_state(self.h, out.ctypes.data_as(_vp), 0))
        return out

    def get_buffer(self, which):
        W = np.empty(self.shape)
        self._check(lib().gks_get_buffer(self.h, int(which), W.ctypes.data_as(_vp), 0))
        return W

    def compute_dt(self):
        dt = C.c_double(0.0)
        self._check(lib().gks_compute_dt(self.h, C.byref(dt)))
        return dt.value

    def stage(self, stage, dt):
        self._check(lib().gks_stage(self.h, int(stage), float(dt)))

    def step(self, dt=0.0):
        self._check(lib().gks_step(self.h, float(dt)))

    def advance_to(self, t_end, max_steps=0):
        n = C.c_longlong(0)
        t = C.c_double(0.0)
        self._check(lib().gks_advance_to(self.h, float(t_end), int(max_steps), C.byref(n), C.byref(t)))
        return n.value, t.value

    def diagnostics(self, check=True):
        """Error word, fallbacks, t, steps and dt; check=False returns them
        without raising on a set error word (a run that failed)."""
        d = Diag()
        st = lib().gks_get_diagnostics(self.h, C.byref(d))
        if check:
            self._check(st)
        return d

    def selection_flips(self):
        """TENO-D selections the float32 path makes otherwise than the float64
        path on the current state: dict of counts (gks_selection_flips)."""
        f = FlipCount()
        self._check(lib().gks_selection_flips(self.h, C.byref(f)))
        return {k: int(getattr(f, k)) for k, _ in FlipCount._fields_}

    def kernel_launches(self):
        return lib().gks_kernel_launches(self.h)

    def profile(self, enable=True):
        """Record CUDA events around every directly launched kernel."""
        self._check(lib().gks_profile_enable(self.h, 1 if enable else 0))

    def profile_read(self, kind=0):
        """(launches, total ms) of kernel kind 0 stage, 1 ghost, 2 other; clears."""
        n = C.c_longlong(0)
        ms = C.c_double(0.0)
        self._check(lib().gks_profile_read(self.h, int(kind), C.byref(n), C.byref(ms)))
        return n.value, ms.value


def alu_peak(precision="fp32", target_ms=200.0):
    """Measured FMA-chain throughput (TFLOP/s, 2 flops per FMA) of the device."""
    L = lib()
    L.gks_alu_peak.argtypes = [C.c_int, C.c_double, _dp]
    L.gks_alu_peak.restype = C.c_int
    v = C.c_double(0.0)
    st = L.gks_alu_peak(PRECISION[precision], float(target_ms), C.byref(v))
    if st != GKS_OK:
        raise GKSError(st, "gks_alu_peak")
    return v.value


GKS_COUNT_TENO_CHARVARS = 4


def count_flops(dim, precision="fp32", tau="euler", Pr=1.0, recon="teno_d", charvars=0):
    """Algorithmic operation count of the library's stage arithmetic per cell
    (charvars=1: TENO-D in characteristic variables)."""
    if charvars:
        recon = GKS_COUNT_TENO_CHARVARS
    m = FlopModel()
    L = lib()
    L.gks_count_flops_recon.argtypes = [C.c_int, C.c_int, C.c_int, C.c_double, C.c_int, C.POINTER(FlopModel)]
    L.gks_count_flops_recon.restype = C.c_int
    st = L.gks_count_flops_recon(int(dim), PRECISION[precision] if isinstance(precision, str) else int(precision),
                                 TAU[tau] if isinstance(tau, str) else int(tau), float(Pr),
                                 RECON[recon] if isinstance(recon, str) else int(recon), C.byref(m))
    if st != GKS_OK:
        raise GKSError(st, "gks_count_flops")
    return {k: getattr(m, k) for k, _ in FlopModel._fields_}


def solver_for(setup, precision="fp64", **kw) -> Solver:
    """Solver configured from a ``workloads.Setup``."""
    args = dict(lx=setup.lx, ly=setup.ly, bc=setup.bc, precision=precision, gamma=setup.gamma,
                mu=setup.mu, Pr=setup.Pr, tau=setup.tau, cfl=setup.cfl)
    args.update(getattr(setup, "scheme", {}))
    args.update(kw)
    s = Solver(setup.dim, setup.nx, setup.ny, **args)
    if setup.bcstate:
        s.set_boundary_states(**setup.bcstate)
    s.set_state(setup.W)
    return s


# ---------------------------------------------------------------- host replicas
def _replica():
    L = lib()
    if not getattr(L, "_replica_declared", False):
        L.gks_host_time_coeffs.argtypes = [C.c_int, C.c_double, _dp, _dp]
        L.gks_host_teno.argtypes = [C.c_int, _dp, C.c_double, C.c_int, C.c_double, C.c_double, _dp, _dp]
        L.gks_host_point_flux.argtypes = [C.c_int, C.c_int, C.c_int] + [C.c_double] * 6 + [_dp] * 8
        L.gks_host_teno_vjp.argtypes = [C.c_int, _dp] + [C.c_double, C.c_int, C.c_double, C.c_double] + [_dp] * 3
        L.gks_host_weno_ao.argtypes = [C.c_int, _dp, C.c_double, C.c_double, C.c_double, _dp, _dp]
        L.gks_host_point_flux_vjp.argtypes = [C.c_int, C.c_double] + [_dp] * 10
        L.gks_host_weno3.argtypes = [C.c_int, C.c_int, _dp, C.c_double, C.c_int, C.c_double, _dp]
        L.gks_host_weno3_gauss.argtypes = [C.c_int, C.c_int, _dp, C.c_double, C.c_int, C.c_double, _dp]
        L.gks_host_merge.argtypes = [C.c_int, C.c_int, C.c_double, _dp, _dp, _dp]
        L.gks_host_char_face.argtypes = [C.c_int, C.c_int, C.c_double, _dp, C.c_double, C.c_int, C.c_double,
                                         C.c_double, _dp]
        L.gks_host_physical.argtypes = [C.c_int, C.c_int, C.c_double, _dp]
        for f in (L.gks_host_time_coeffs, L.gks_host_teno, L.gks_host_point_flux, L.gks_host_teno_vjp,
                  L.gks_host_point_flux_vjp, L.gks_host_weno_ao, L.gks_host_weno3, L.gks_host_weno3_gauss,
                  L.gks_host_merge, L.gks_host_char_face, L.gks_host_physical):
            f.restype = C.c_int
        L._replica_declared = True
    return L


def _arr(a, n):
    x = np.zeros(n) if a is None else np.ascontiguousarray(a, dtype=np.float64)
    return x, x.ctypes.data_as(_dp)


def host_physical(dim, W, precision="fp64", gamma=1.4):
    """The kernels' state test (rho > 0, p > 0; float32 also an internal
    energy of at least 1e-4 of E) on 4 slots."""
    w, pw = _arr(W, 4)
    r = _replica().gks_host_physical(int(dim), PRECISION[precision], float(gamma), pw)
    if r < 0:
        raise ValueError("bad argument")
    return bool(r)


def host_time_coeffs(s, precision="fp64"):
    """Folded time coefficients (cF, cD) from the host build of the device code."""
    cF, pF = _arr(None, 6)
    cD, pD = _arr(None, 6)
    if _replica().gks_host_time_coeffs(PRECISION[precision], float(s), pF, pD):
        raise ValueError("bad argument")
    return cF, cD


def host_teno(q, precision="fp64", eps=1e-40, q_pow=7, ct1=1e-7, ct2=1e-5):
    """(faces[vp, dp, vm, dm], gauss[v-, d-, v+, d+], large) for one stencil."""
    qq, pq = _arr(q, 5)
    f, pf = _arr(None, 4)
    g, pg = _arr(None, 4)
    r = _replica().gks_host_teno(PRECISION[precision], pq, eps, q_pow, ct1, ct2, pf, pg)
    if r == -2:
        raise AssertionError("packed TENO-D lanes disagree")
    if r < 0:
        raise ValueError("bad argument")
    return f, g, bool(r)


def host_point_flux(dim, Wl, Wln, Wlt, Wr, Wrn, Wrt, dt, precision="fp64", tau="euler", gamma=1.4,
                    mu=0.0, Pr=1.0, c1=0.01, c2=1.0):
    """(F, dF/dt) at one point from the host build of the device code; 4 slots."""
    keep = [_arr(a, 4) for a in (Wl, Wln, Wlt, Wr, Wrn, Wrt)]
    F, pF = _arr(None, 4)
    dF, pD = _arr(None, 4)
    r = _replica().gks_host_point_flux(dim, PRECISION[precision], TAU[tau] if isinstance(tau, str) else tau,
                                       gamma, mu, Pr, c1, c2, dt, *[k[1] for k in keep], pF, pD)
    if r:
        raise ValueError("bad argument")
    return F, dF


def host_weno3(q, teno5=False, precision="fp64", eps=None, q_pow=6, ct=1e-7):
    """(vp, dp, vm, dm) of the conventional path's WENO5-Z / TENO5 face
    reconstruction for one stencil."""
    if eps is None:
        eps = 1e-40 if teno5 else 1e-8
    qq, pq = _arr(q, 5)
    f, pf = _arr(None, 4)
    if _replica().gks_host_weno3(PRECISION[precision], int(bool(teno5)), pq, eps, int(q_pow), ct, pf):
        raise ValueError("bad argument")
    return f


def host_weno3_gauss(q, teno5=False, precision="fp64", eps=None, q_pow=6, ct=1e-7):
    """(v-, d-, v+, d+) of WENO5-Z / TENO5 at the Gauss points for one stencil."""
    if eps is None:
        eps = 1e-40 if teno5 else 1e-8
    qq, pq = _arr(q, 5)
    g, pg = _arr(None, 4)
    if _replica().gks_host_weno3_gauss(PRECISION[precision], int(bool(teno5)), pq, eps, int(q_pow), ct, pg):
        raise ValueError("bad argument")
    return g


def host_char_face(dim, w6, precision="fp64", gamma=1.4, eps=1e-40, q_pow=7, ct1=1e-7, ct2=1e-5):
    """(vl, dl, vr, dr), 4 slots each: both sides of one face reconstructed
    in characteristic variables from the six cells w6[6][4] around it."""
    ww, pw = _arr(np.asarray(w6, dtype=np.float64).reshape(24), 24)
    o, po = _arr(None, 16)
    if _replica().gks_host_char_face(dim, PRECISION[precision], gamma, pw, eps, int(q_pow), ct1, ct2, po):
        raise ValueError("bad argument")
    return o.reshape(4, 4)


def host_merge(dim, Wl, Wr, precision="fp64", gamma=1.4):
    """Kinetic merge of two states' values (4 slots)."""
    keep = [_arr(a, 4) for a in (Wl, Wr)]
    W0, p0 = _arr(None, 4)
    if _replica().gks_host_merge(dim, PRECISION[precision], gamma, keep[0][1], keep[1][1], p0):
        raise ValueError("bad argument")
    return W0


def host_weno_ao(q, precision="fp64", eps_ao=1e-8, d_hi=0.85, d_lo=0.85):
    """(faces[vp, dp, vm, dm], gauss[v-, d-, v+, d+]) of WENO5-AO for one stencil."""
    qq, pq = _arr(q, 5)
    f, pf = _arr(None, 4)
    g, pg = _arr(None, 4)
    r = _replica().gks_host_weno_ao(PRECISION[precision], pq, eps_ao, d_hi, d_lo, pf, pg)
    if r == -2:
        raise AssertionError("packed WENO5-AO lanes disagree")
    if r:
        raise ValueError("bad argument")
    return f, g


def host_teno_vjp(q, gfaces, ggauss, precision="fp64", eps=1e-40, q_pow=7, ct1=1e-7, ct2=1e-5):
    """Transpose of TENO-D at q with its selection held fixed: (gq[5], large)."""
    qq, pq = _arr(q, 5)
    gf, pgf = _arr(gfaces, 4)
    gg, pgg = _arr(ggauss, 4)
    gq, pgq = _arr(None, 5)
    r = _replica().gks_host_teno_vjp(PRECISION[precision], pq, eps, q_pow, ct1, ct2, pgf, pgg, pgq)
    if r < 0:
        raise ValueError("bad argument")
    return gq, bool(r)


def host_point_flux_vjp(Wl, Wln, Wlt, Wr, Wrn, Wrt, gF, gdF, precision="fp64", gamma=1.4):
    """Cotangents (gl[12], gr[12]) of the two sides' (W, Wn, Wt) from those of
    (F, dF/dt) of the 2-D tau = 0 point flux (host build of the device code)."""
    keep = [_arr(a, 4) for a in (Wl, Wln, Wlt, Wr, Wrn, Wrt, gF, gdF)]
    gl, pl = _arr(None, 12)
    gr, pr = _arr(None, 12)
    if _replica().gks_host_point_flux_vjp(PRECISION[precision], gamma, *[k[1] for k in keep], pl, pr):
        raise ValueError("bad argument")
    return gl, gr


def step1d_noalloc(W_in, W_out, dx, dt, bc=("zerograd", "zerograd"), precision="fp64", gamma=1.4, mu=0.0,
                   Pr=1.0, stream=0, **scheme):
    """One 1-D S2O4 step through gks_step1d_noalloc (no device allocation by
    the library).  W_in, W_out: contiguous float64 CUDA tensors [3][nx] (or
    [3][1][nx]) on the current device.  Returns the error word; raises
    GKSError on a bad status, and GKSError(GKS_EINVAL) before any library
    call when a tensor is not of that kind."""
    nx = int(W_in.shape[-1]) if hasattr(W_in, "shape") and len(W_in.shape) else 0
    for t in (W_in, W_out):
        ok = (hasattr(t, "data_ptr") and t.is_cuda and t.dtype.is_floating_point and t.dtype.itemsize == 8
              and t.is_contiguous() and t.numel() == 3 * nx and nx > 0)
        if ok:
            import torch
            ok = t.device.index == torch.cuda.current_device()
        if not ok:
            raise GKSError(GKS_EINVAL, "gks_step1d_noalloc: W_in and W_out must be contiguous float64 CUDA "
                                       "tensors of 3 * nx values on the current device")
    L = lib()
    if not getattr(L, "_noalloc_declared", False):
        L.gks_step1d_noalloc.argtypes = [_vp, _vp, C.c_int, C.c_double, C.POINTER(C.c_int), C.POINTER(Gas),
                                         C.POINTER(Scheme), C.c_int, C.c_double, _vp, C.POINTER(C.c_uint)]
        L.gks_step1d_noalloc.restype = C.c_int
        L._noalloc_declared = True
    bcs = (C.c_int * 2)(*[BC[b] if isinstance(b, str) else int(b) for b in bc])
    err = C.c_uint(0)
    st = L.gks_step1d_noalloc(_vp(W_in.data_ptr()), _vp(W_out.data_ptr()), int(nx), float(dx), bcs,
                              C.byref(Gas(gamma, mu, Pr)), C.byref(default_scheme(**scheme)),
                              PRECISION[precision] if isinstance(precision, str) else int(precision),
                              float(dt), _vp(stream), C.byref(err))
    if st != GKS_OK:
        raise GKSError(st, "gks_step1d_noalloc")
    return err.value


class Batch:
    """Independent 1-D problems advanced in one persistent launch (gks_batch_*).
    W: packed [3][sum ncells] float64."""

    def __init__(self, ncells, lengths, precision="fp32", gamma=1.4, mu=0.0, Pr=1.0, tau="euler", cfl=0.5,
                 **scheme):
        L = lib()
        if not getattr(L, "_batch_declared", False):
            sig = {
                "gks_batch_create": ([C.c_int, C.POINTER(C.c_int), _dp, C.c_int, C.POINTER(_vp)], C.c_int),
                "gks_batch_destroy": ([_vp], None),
                "gks_batch_set_gas": ([_vp, C.POINTER(Gas)], C.c_int),
                "gks_batch_set_scheme": ([_vp, C.POINTER(Scheme)], C.c_int),
                "gks_batch_set_stream": ([_vp, _vp], C.c_int),
                "gks_batch_set_state": ([_vp, _vp, C.c_int], C.c_int),
                "gks_batch_get_state": ([_vp, _vp, C.c_int], C.c_int),
                "gks_batch_advance_to": ([_vp, C.c_double, C.c_longlong], C.c_int),
                "gks_batch_get_progress": ([_vp, _dp, C.POINTER(C.c_longlong), C.POINTER(C.c_uint),
                                            C.POINTER(C.c_longlong)], C.c_int),
                "gks_batch_set_launch": ([_vp, C.c_int, C.c_int], C.c_int),
                "gks_batch_tune": ([_vp, C.c_double, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int), _dp],
                                   C.c_int),
                "gks_batch_last_error": ([_vp], C.c_char_p),
                "gks_batch_launches": ([_vp], C.c_longlong),
            }
            for name, (args, res) in sig.items():
                f = getattr(L, name)
                f.argtypes = args
                f.restype = res
            L._batch_declared = True
        n = np.ascontiguousarray(ncells, dtype=np.int32)
        lens = np.ascontiguousarray(lengths, dtype=np.float64)
        self.count = len(n)
        self.total = int(n.sum())
        h = _vp()
        st = L.gks_batch_create(self.count, n.ctypes.data_as(C.POINTER(C.c_int)), lens.ctypes.data_as(_dp),
                                PRECISION[precision] if isinstance(precision, str) else int(precision), C.byref(h))
        if st != GKS_OK:
            raise GKSError(st, "gks_batch_create")
        self.h = h
        self._check(L.gks_batch_set_gas(h, C.byref(Gas(gamma, mu, Pr))))
        self._check(L.gks_batch_set_scheme(h, C.byref(default_scheme(cfl=cfl, tau=tau, **scheme))))

    def _check(self, st):
        if st != GKS_OK:
            raise GKSError(st, lib().gks_batch_last_error(self.h).decode())

    def close(self):
        if getattr(self, "h", None):
            lib().gks_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_stream(self, stream_handle):
        self._check(lib().gks_batch_set_stream(self.h, _vp(stream_handle)))

    def set_state(self, W):
        if hasattr(W, "data_ptr"):
            self._check(lib().gks_batch_set_state(self.h, _vp(W.data_ptr()), 1))
        else:
            W = np.ascontiguousarray(W, dtype=np.float64)
            if W.size != 3 * self.total:
                raise ValueError("packed state must have 3 x %d values" % self.total)
            self._check(lib().gks_batch_set_state(self.h, W.ctypes.data_as(_vp), 0))

    def get_state(self):
        W = np.empty((3, self.total))
        self._check(lib().gks_batch_get_state(self.h, W.ctypes.data_as(_vp), 0))
        return W

    def advance_to(self, t_end, max_steps=0, allow_failed=False):
        """Advance every problem to t_end.  A problem that produced a
        non-physical cell average stops there and is flagged in progress();
        with allow_failed that is not an error and the number of flagged
        problems is returned."""
        st = lib().gks_batch_advance_to(self.h, float(t_end), int(max_steps))
        if st == GKS_ENONPHYSICAL and allow_failed:
            return int(np.count_nonzero(self.progress()[2]))
        self._check(st)
        return 0

    def progress(self):
        t = np.zeros(self.count)
        steps = np.zeros(self.count, dtype=np.int64)
        err = np.zeros(self.count, dtype=np.uint32)
        fb = C.c_longlong(0)
        self._check(lib().gks_batch_get_progress(self.h, t.ctypes.data_as(_dp),
                                                 steps.ctypes.data_as(C.POINTER(C.c_longlong)),
                                                 err.ctypes.data_as(C.POINTER(C.c_uint)), C.byref(fb)))
        return t, steps, err, fb.value

    def set_launch(self, threads, blocks_per_sm):
        self._check(lib().gks_batch_set_launch(self.h, int(threads), int(blocks_per_sm)))

    def tune(self, t_probe, use_cache=True):
        th, bp, ms = C.c_int(0), C.c_int(0), C.c_double(0.0)
        self._check(lib().gks_batch_tune(self.h, float(t_probe), 1 if use_cache else 0, C.byref(th), C.byref(bp),
                                         C.byref(ms)))
        return th.value, bp.value, ms.value

    def launches(self):
        return lib().gks_batch_launches(self.h)


# ---------------------------------------------------------------- multi-GPU helpers
def partition_lpt(costs, parts):
    """Split independent problems over `parts` ranks, longest processing time
    first (each problem, in decreasing cost, goes to the least-loaded rank;
    ties by rank).  Returns one sorted index array per rank."""
    costs = np.asarray(costs, dtype=np.float64)
    order = np.argsort(-costs, kind="stable")
    load = np.zeros(parts)
    owner = np.empty(costs.size, dtype=np.int64)
    for k in order:
        r = int(np.argmin(load))
        owner[k] = r
        load[r] += costs[k]
    return [np.flatnonzero(owner == r) for r in range(parts)]


def reduce_scalars(values, op="max", dist=None, device=None):
    """Max or sum of per-rank scalars over all ranks (identity without a
    process group).  `device`: where the collective's tensor lives (a CUDA
    device for NCCL, None for the CPU / gloo)."""
    if dist is None:
        return [float(v) for v in values]
    import torch
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.SUM)
    return t.cpu().tolist()


# ---------------------------------------------------------------- adjoint
def _adj_lib():
    L = lib()
    if not getattr(L, "_adjoint_declared", False):
        sig = {
            "gks_adjoint_create": ([_vp, C.c_int, C.POINTER(_vp)], C.c_int),
            "gks_adjoint_destroy": ([_vp], None),
            "gks_adjoint_forward": ([_vp, C.c_int, C.c_double], C.c_int),
            "gks_adjoint_backward": ([_vp, _vp, _vp, C.c_int], C.c_int),
            "gks_adjoint_launches": ([_vp], C.c_longlong),
            "gks_adjoint_reserve": ([_vp, C.c_int], C.c_int),
            "gks_vjp_step": ([_vp, _vp, _vp, _vp, C.c_double, C.c_int], C.c_int),
        }
        for name, (args, res) in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = res
        L._adjoint_declared = True
    return L


def _ptr(a, shape):
    """(pointer, on_device, keep-alive) of a float64 state-shaped array."""
    if hasattr(a, "data_ptr"):
        if not (a.is_cuda and a.dtype.itemsize == 8 and a.is_contiguous() and a.numel() == int(np.prod(shape))):
            raise ValueError("need a contiguous float64 CUDA tensor of shape %s" % (shape,))
        return _vp(a.data_ptr()), 1, a
    a = np.ascontiguousarray(a, dtype=np.float64)
    if a.size != int(np.prod(shape)):
        raise ValueError("need %d values" % int(np.prod(shape)))
    return a.ctypes.data_as(_vp), 0, a


class Adjoint:
    """Checkpointed hand-written adjoint of a 2-D Solver with tau='zero'
    (gks_adjoint_*): forward(nsteps, dt) advances the solver keeping a
    checkpoint every k steps; backward(gWN) returns dJ/dW0 for the given
    dJ/dWN (numpy in -> numpy out; CUDA tensor in -> CUDA tensor out)."""

    def __init__(self, solver: Solver, checkpoint_every: int):
        L = _adj_lib()
        self.solver = solver
        h = _vp()
        solver._check(L.gks_adjoint_create(solver.h, int(checkpoint_every), C.byref(h)))
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            _adj_lib().gks_adjoint_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def reserve(self, nsteps):
        """Allocate the checkpoints and segment states of nsteps-step passes."""
        self.solver._check(_adj_lib().gks_adjoint_reserve(self.h, int(nsteps)))

    def forward(self, nsteps, dt):
        self.solver._check(_adj_lib().gks_adjoint_forward(self.h, int(nsteps), float(dt)))

    def backward(self, gWN, out=None):
        shape = self.solver.shape
        p_in, dev, keep = _ptr(gWN, shape)
        if out is None:
            out = gWN.new_empty(gWN.shape) if dev else np.empty(shape)
        p_out, dev2, _ = _ptr(out, shape)
        if dev2 != dev:
            raise ValueError("gWN and out must both be host arrays or both CUDA tensors")
        self.solver._check(_adj_lib().gks_adjoint_backward(self.h, p_in, p_out, dev))
        return out

    def launches(self):
        return int(_adj_lib().gks_adjoint_launches(self.h))


def vjp_step(solver: Solver, W, gout, dt):
    """(dS/dW)^T gout for one S2O4 step S of fixed dt at state W (host arrays).
    The solver is left at S(W)."""
    shape = solver.shape
    pW, d1, kW = _ptr(W, shape)
    pg, d2, kg = _ptr(gout, shape)
    gin = np.empty(shape)
    if d1 or d2:
        raise ValueError("vjp_step takes host arrays")
    solver._check(_adj_lib().gks_vjp_step(solver.h, pW, pg, gin.ctypes.data_as(_vp), float(dt), 0))
    return gin


_flow_cls = None


def _flow():
    global _flow_cls
    if _flow_cls is None:
        import torch

        class GKSFlow(torch.autograd.Function):
            """W_N = S^n(W_0) on a Solver; backward = the hand-written adjoint."""

            @staticmethod
            def forward(ctx, W0, solver, nsteps, dt, checkpoint_every):
                W0c = W0.detach().contiguous()
                solver.set_state(W0c)
                adj = Adjoint(solver, checkpoint_every)
                adj.forward(nsteps, dt)
                WN = torch.empty_like(W0c)
                solver.get_state(WN)
                ctx.adj = adj
                return WN

            @staticmethod
            def backward(ctx, gWN):
                g = gWN.detach().to(torch.float64).contiguous()
                gW0 = ctx.adj.backward(g)
                return gW0, None, None, None, None

        _flow_cls = GKSFlow
    return _flow_cls


def flow(W0, solver: Solver, nsteps: int, dt: float, checkpoint_every: int = 20):
    """Differentiable map W_0 -> W_N (nsteps S2O4 steps of fixed dt) for a
    float64 CUDA tensor W_0 of the solver's state shape, as a
    torch.autograd.Function whose backward is the library's adjoint."""
    return _flow().apply(W0, solver, nsteps, dt, checkpoint_every)
