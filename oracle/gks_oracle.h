/*
 * gks_oracle.h -- plain, slow FP64 CPU oracle for the fifth-order TENO-D
 * gas-kinetic scheme (GKS) with two-stage fourth-order (S2O4) time stepping.
 *
 * TEST INFRASTRUCTURE ONLY.  This code exists to check the CUDA path.  Only
 * the test suite, the smoke entry and the bench's CPU-baseline leg may load
 * it.  It shares no code, header, table or constant with the CUDA library.
 *
 * Every routine follows the paper's statement of the method:
 *   Sec. 2.1  BGK model, Maxwellian, compatibility, Eqs. (2.1)-(2.9)
 *   Sec. 2.2  two-stage fourth-order time stepping, Eqs. (2.10)-(2.20)
 *   Sec. 3.1  sub-stencil polynomials, smoothness indicators Eq. (3.7)
 *   Sec. 3.2  derivatives on the stencils, kinetic merge Eqs. (3.25)-(3.26),
 *             2-D dimension-by-dimension steps
 *   Sec. 4.2  TENO-D selection Eqs. (4.5)-(4.14)
 *   Sec. 3.2  WENO5-AO weights and AO(5,3) polynomial (the alternative
 *             reconstruction the paper compares against)
 *   Sec. 5    collision time, CFL time step
 * Readings of garbled or silent passages are listed in the .c file header.
 */
#ifndef GKS_ORACLE_H
#define GKS_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

/* boundary kinds for ghost layers */
enum { OR_BC_PERIODIC = 0, OR_BC_ZEROGRAD = 1, OR_BC_SYMMETRY = 2, OR_BC_NOSLIP = 3, OR_BC_REFLECT = 4,
       /* state-setting rules (double Mach reflection, Sec. 5.7): INFLOW sets
        * the ghosts to bc_in; WALL_AFTER_X0 (y sides) sets bc_in for ghost
        * centres with x < shock_x0 and reflects beyond; MOVING_SHOCK (y sides)
        * sets bc_in behind and bc_pre ahead of the oblique shock
        * x_s(y, t) = shock_x0 + y cot(theta) + shock_speed t / sin(theta) */
       OR_BC_INFLOW = 5, OR_BC_WALL_AFTER_X0 = 6, OR_BC_MOVING_SHOCK = 7 };
/* collision-time models (Sec. 5) */
enum { OR_TAU_ZERO = 0, OR_TAU_EULER = 1, OR_TAU_NS = 2 };

typedef struct {
    int dim;              /* 1 or 2 */
    int nx, ny;           /* interior cells; ny = 1 in 1-D */
    double dx, dy;        /* cell sizes */
    int bc[4];            /* x-low, x-high, y-low, y-high */
    double gamma;         /* ratio of specific heats */
    double mu;            /* dynamic viscosity (NS) */
    double Pr;            /* Prandtl number; 1 = no heat-flux correction */
    int tau_mode;         /* OR_TAU_* */
    double c1, c2;        /* Euler collision-time constants */
    double cfl;
    double eps;           /* TENO-D epsilon, Eq. (4.5) */
    double qpow;          /* TENO-D power q, Eq. (4.5) */
    double ct1, ct2;      /* thresholds C_T1, C_T2, normal direction */
    double ct1_t, ct2_t;  /* thresholds used in the tangential direction */
    int positivity_fallback; /* 1: first-order state when rho<=0 or p<=0 at a point */
    int recon;            /* OR_RECON_*: TENO-D (Sec. 4.2) or WENO5-AO (Sec. 3.2) */
    double d_hi, d_lo;    /* WENO5-AO linear-weight parameters d_Hi, d_Lo */
    double eps_ao;        /* WENO5-AO epsilon of Eq. (3.5) */
    int merge;            /* OR_MERGE_*: equilibrium state at the interface */
    double zpow;          /* WENO5-Z exponent of tau/(beta+eps) in Eq. (3.5) */
    double t;             /* time of the state passed in (time-dependent ghosts) */
    double bc_in[4];      /* conserved state of the INFLOW rule / behind the shock */
    double bc_pre[4];     /* conserved state ahead of the shock */
    double shock_x0, shock_theta, shock_speed; /* shock foot on y = 0, angle to the
                                                  x-axis (rad), normal speed */
    int charvars;         /* 1: normal reconstruction in characteristic variables
                             (Sec. 3.1; see or_char_basis), 0: component-wise */
    double ox, oy;        /* domain origin: cell (i, j) is centred at
                             (ox + (i + 1/2) dx, oy + (j + 1/2) dy); default 0 */
} or_problem;

/* TENO-D (Sec. 4.2), WENO5-AO (Sec. 3.2), and the conventional path
 * (Sec. 3.1, 4.1): WENO5-Z or TENO5 face values, slopes from the quadratic of
 * Eq. (3.11), equilibrium slope from the linear Eq. (3.12); in 2-D the
 * equilibrium state and slopes at the Gauss points are the linear (quartic)
 * reconstructions of the line-averaged kinetic merges and Eq. (3.12) slopes
 * (Steps 2 and 4), the non-equilibrium ones WENO-Z / TENO5 (Step 3) */
enum { OR_RECON_TENO_D = 0, OR_RECON_WENO_AO = 1, OR_RECON_WENO_Z = 2, OR_RECON_TENO5 = 3 };
/* kinetic weighting of Eqs. (3.25)-(3.26), or the arithmetic average of the
 * two sides that Sec. 3.2 allows for smooth flow */
enum { OR_MERGE_KINETIC = 0, OR_MERGE_AVERAGE = 1 };

/* ---- reconstruction primitives (Sec. 3.1, 3.2, 4.2) ---- */
/* n x n matrix (row-major) mapping cell averages at integer offsets to the
 * monomial coefficients c_k of p(xi) = sum c_k xi^k, xi = (x - x_i)/dx. */
int    or_fit_matrix(int n, const int *offsets, double *minv);
double or_poly_eval(int deg, const double *c, double xi);
double or_poly_deriv(int deg, const double *c, double xi);
/* Eq. (3.7) in the scaled variable: sum_q int_{-1/2}^{1/2} (p^(q))^2 dxi */
double or_beta(int deg, const double *c);
/* TENO-D on the 5 cell averages q[0..4] = Qbar_{i-2..i+2}; evaluates the
 * selected reconstruction and its xi-derivative at the points xs[0..n-1].
 * Returns delta_{3,1}; sel[0..2] receives delta_{k,2} (0 when large). */
/* WENO5-AO (Sec. 3.2) on the 5 cell averages: WENO-Z-type weights of Eq.
 * (3.5) on the large stencil and the three sub-stencils with the linear
 * weights of d_Hi, d_Lo, evaluated with the AO(5,3) polynomial and its
 * xi-derivative at xs[0..n-1]; wbar[0..3] (may be NULL) receives the
 * normalised weights of S0, S1, S2, S3. */
void   or_weno_ao(const double *q5, double eps, double d_hi, double d_lo, int n, const double *xs,
                  double *val, double *dval, double *wbar);
int    or_teno_d(const double *q5, double eps, double qpow, double ct1, double ct2,
                 int n, const double *xs, double *val, double *dval, int *sel);
/* Selection trace (test instrumentation; changes no result): with a buffer
 * set, every or_teno_d call, direct or inside a flux, appends one byte
 * delta_{3,1} + 2 delta_{0,2} + 4 delta_{1,2} + 8 delta_{2,2};
 * or_trace_length is the number of calls since the buffer was set (it may
 * exceed cap; bytes past cap are not stored).  NULL stops the trace. */
void   or_trace_selections(unsigned char *buf, long cap);
long   or_trace_length(void);

/* characteristic basis of the normal Euler flux (Sec. 3.1): R holds the right
 * eigenvectors of dF/dW at the conserved state Wm as columns (row-major
 * nv x nv, nv = dim + 2; eigenvalues U - c, U, [U,] U + c), L = R^-1.
 * Returns -1 when Wm is not physical. */
int    or_char_basis(int dim, double gamma, const double *Wm, double *R, double *L);

/* ---- kinetic layer (Sec. 2.1) ---- */
/* u-moments <u^n>, n = 0..nmax, of a 1-D unit-mass Maxwellian with mean U and
 * lambda; half = 0 full space, +1 over u>0, -1 over u<0. */
void   or_moments_u(double U, double lam, int half, int nmax, double *m);
/* micro slope a with M(prim) a = b, M_ab = <psi_a psi_b>; nvar = dim + 2 */
int    or_micro_slope(int dim, double K, double U, double V, double lam,
                      const double *b, double *a);
/* exact time integrals q0..q5 of the coefficients of Eq. (2.5) over [0, delta] */
void   or_time_coeffs(double delta, double tau, double *q);
/* time-integrated interface flux (Eq. 2.12) at one point in the local frame
 * (normal velocity first) for delta = dt and dt/2. Inputs are conserved
 * variables and their normal / tangential derivatives on both sides.
 * Returns 1 when the positivity fallback replaced a side, else 0;
 * -1 on a non-physical state that the fallback could not fix. */
/* WENO5-Z (Sec. 3.1, Eqs. 3.5-3.9) or TENO5 (Sec. 4.1, Eqs. 4.1-4.4) value of
 * the five cell averages q5 = Qbar_{i-2..i+2} at the points xs[0..n-1]
 * (xi = (x - x_i)/dx): the three quadratics p_k blended with weights built
 * on the linear weights d_k(xi) that combine them into the quartic at xi.
 * teno5 = 0: WENO-Z, omega_k = d_k (1 + (tau/(beta_k+eps))^zpow) normalised,
 * tau = |beta_0 - beta_2|; teno5 = 1: gamma_k = (1 + tau/(beta_k+eps))^q,
 * chi_k = gamma_k / sum gamma, delta_k = [chi_k >= ct], omega_k = d_k delta_k
 * normalised.  wbar (optional) receives the weights at the last point.
 * Returns 0, or -1 if xs admits no linear weights. */
int    or_weno3(const double *q5, int teno5, double eps, double zpow, double q, double ct, int n,
                const double *xs, double *val, double *wbar);
/* the same with xi-derivatives: the derivative of the same weighted blend of
 * the quadratics (the tangential derivative of the 2-D conventional path) */
int    or_weno3_dv(const double *q5, int teno5, double eps, double zpow, double q, double ct, int n,
                   const double *xs, double *val, double *dval);
/* the problem's normal reconstruction of one cell's five averages q5:
 * out = (value, xi-derivative at xi = +1/2, value, xi-derivative at -1/2) */
int    or_recon_faces(const or_problem *P, const double *q5, double *out);
int    or_flux_point(const or_problem *P,
                     const double *Wl, const double *Wln, const double *Wlt,
                     const double *Wr, const double *Wrn, const double *Wrt,
                     const double *Wcl, const double *Wcr,
                     double dt, double *Fdt, double *Fhalf);
/* the same with the equilibrium normal slope W0_n given (the conventional
 * path's Eq. 3.12) instead of the kinetic merge of the side slopes; NULL:
 * or_flux_point */
int    or_flux_point_eq(const or_problem *P,
                        const double *Wl, const double *Wln, const double *Wlt,
                        const double *Wr, const double *Wrn, const double *Wrt,
                        const double *Wcl, const double *Wcr, const double *W0n_lin,
                        double dt, double *Fdt, double *Fhalf);

/* ---- solver (Sec. 2.2, 3.2, 5) ---- */
/* W and Wout: interior SoA [nvar][ny][nx]; nvar = dim + 2 */
int    or_stage1(const or_problem *P, const double *W, double dt, double *Wstar, long *nfallback);
int    or_step(const or_problem *P, const double *W, double dt, double *Wout, long *nfallback);
double or_dt(const or_problem *P, const double *W);
/* advance to t_end with CFL time steps, the last one clipped to t_end */
int    or_run(const or_problem *P, double *W, double t_end, long max_steps,
              long *steps_done, double *t_out, long *nfallback);
/* the time-integrated flux of one face (Sec. 2.2, 3.2) on a ghost-filled
 * array Wg [nvar][ny+6][nx+6]: dir 0 the x face between ghosted cells
 * (ic, jc) and (ic+1, jc), dir 1 the y face between (ic, jc) and (ic, jc+1);
 * Fdt, Fhalf = the Gauss-averaged F(dt), F(dt/2) in global variable order;
 * *nfb (may be NULL) counts the fallbacks taken.  Returns -1 on a state no
 * fallback fixes. */
int    or_face_flux(const or_problem *P, const double *Wg, int dir, int ic, int jc, double dt, double *Fdt,
                    double *Fhalf, long *nfb);
/* ghost filling exposed for tests: Wg is [nvar][ny+6][nx+6] (1-D: ny+6 -> 1) */
void   or_fill_ghosts(const or_problem *P, double *Wg);

#ifdef __cplusplus
}
#endif
#endif
