/*
 * gks_host_replica.h -- host compilations of the library's per-point device
 * arithmetic, for unit tests on machines without a GPU.
 *
 * Each call runs the same templated source as the CUDA kernels (compiled for
 * the host CPU) on ONE stencil or ONE interface point.  There is no
 * grid-level entry here: stepping a grid always runs on the GPU.
 * precision: 0 = float64 arithmetic, 1 = float32 arithmetic (inputs and
 * outputs are passed as float64 either way).  Return 0, or -1 on a bad
 * argument.
 */
#ifndef GKS_HOST_REPLICA_H
#define GKS_HOST_REPLICA_H

#ifdef __cplusplus
extern "C" {
#endif

/* Folded time coefficients of Sec. 2.2 applied to the time integrals of
 * Eq. (2.5), as functions of s = dt/tau: cF[0..5], cD[0..5] with
 * F = sum cF_k dt^{p_k-1} (.), dF/dt = sum 4 cD_k dt^{p_k-2} (.),
 * p = (1,2,2,1,2,2). */
int gks_host_time_coeffs(int precision, double s, double *cF, double *cD);

/* The kernels' test of a state before its flux (and of the cell average a
 * positivity fallback takes): 1 if rho > 0 and p > 0 (finite) -- and, in
 * float32, an internal energy of at least 1e-4 of E (below that a float32
 * pressure has no reliable digits) -- else 0; -1 on a bad argument.
 * W: 4 slots (1-D: slot 2 unused). */
int gks_host_physical(int dim, int precision, double gamma, const double *W);

/* TENO-D (Sec. 4.2) on five cell averages q[0..4] = Qbar_{i-2..i+2}:
 * faces[0..3] = value and xi-derivative at xi = +1/2, then at xi = -1/2;
 * gauss[0..3] = value and xi-derivative at xi = -1/(2 sqrt 3), then +1/(2 sqrt 3);
 * returns the large-stencil flag (1/0) or -1.  precision 2: the packed-pair
 * float32 selection, faces and Gauss points of the 2-D sweep (packed
 * products and fused multiply-adds emulated on the host with the same IEEE
 * rounding); -2 if its two lanes disagree. */
int gks_host_teno(int precision, const double *q, double eps, int qpow, double ct1, double ct2,
                  double *faces, double *gauss);

/* F and dF/dt (per unit time, Sec. 2.2) at one interface point in the local
 * frame from the two sides' conserved variables and their normal (n) and
 * tangential (t) derivatives; 4 slots each, slot 2 unused in 1-D.
 * tau_mode as gks_tau_mode; Pr applies with tau_mode = 2.  No positivity
 * fallback here: both sides must be physical. */
int gks_host_point_flux(int dim, int precision, int tau_mode, double gamma, double mu, double Pr,
                        double c1, double c2, double dt,
                        const double *Wl, const double *Wln, const double *Wlt,
                        const double *Wr, const double *Wrn, const double *Wrt,
                        double *F, double *dF);

/* WENO5-AO (Sec. 3.2) on five cell averages, outputs as gks_host_teno;
 * precision 2: the packed-pair float32 form of the 2-D sweep (-2 if its two
 * lanes disagree). */
int gks_host_weno_ao(int precision, const double *q, double eps_ao, double d_hi, double d_lo,
                     double *faces, double *gauss);

/* The conventional path's face reconstruction (Sec. 3.1, 4.1) of five cell
 * averages: WENO5-Z (teno5 = 0; eps the WENO epsilon of Eq. 3.5) or TENO5
 * (teno5 = 1; eps, power qpow and cut-off ct of Eqs. 4.1-4.3); faces[0..3]
 * = value and xi-slope (Eq. 3.11) at xi = +1/2, then at -1/2. */
int gks_host_weno3(int precision, int teno5, const double *q, double eps, int qpow, double ct, double *faces);

/* The same reconstruction at the Gauss points xi = -+1/(2 sqrt 3) (the 2-D
 * conventional path's Step 3): gauss[0..3] = value and xi-derivative (the
 * derivative of the same weighted blend) at -, then at +. */
int gks_host_weno3_gauss(int precision, int teno5, const double *q, double eps, int qpow, double ct,
                         double *gauss);

/* Kinetic merge of two states' values (Eq. 3.25; the conventional path's
 * line-averaged equilibrium state, Step 2): W0 = rho_l <psi>_{u>0} +
 * rho_r <psi>_{u<0}; 4 slots (energy in slot 3; 1-D slot 2 unused). */
int gks_host_merge(int dim, int precision, double gamma, const double *Wl, const double *Wr, double *W0);

/* Transpose of TENO-D with the selection of q held fixed (the adjoint's
 * frozen selection; with it the reconstruction is linear in q): the
 * cotangents gfaces[0..3] of faces[] and ggauss[0..3] of gauss[] as in
 * gks_host_teno -> gq[0..4].  Returns the large-stencil flag or -1. */
int gks_host_teno_vjp(int precision, const double *q, double eps, int qpow, double ct1, double ct2,
                      const double *gfaces, const double *ggauss, double *gq);

/* Vector-Jacobian product of the 2-D collision-free (tau = 0) point flux:
 * cotangents gF[4], gdF[4] of F and dF/dt -> gl[12], gr[12], the cotangents
 * of (W, Wn, Wt) of the left and right side. */
int gks_host_point_flux_vjp(int precision, double gamma,
                            const double *Wl, const double *Wln, const double *Wlt,
                            const double *Wr, const double *Wrn, const double *Wrt,
                            const double *gF, const double *gdF, double *gl, double *gr);

/* Both sides of one face in characteristic variables (Sec. 3.1; the
 * kernels' normal reconstruction with gks_scheme.charvars = 1): w[24] are
 * the six cells i-2 .. i+3 around the face between cells i and i+1, 4 slots
 * each (rho, normal momentum, tangential momentum, energy; 1-D slot 2 = 0).
 * out[16] = left value, left xi-derivative (TENO-D of cells i-2 .. i+2 at
 * xi = +1/2), right value, right xi-derivative (cells i-1 .. i+3 at
 * xi = -1/2), 4 slots each, in conserved variables.  precision 0 or 1. */
int gks_host_char_face(int dim, int precision, double gamma, const double *w, double eps, int qpow,
                       double ct1, double ct2, double *out);

#ifdef __cplusplus
}
#endif
#endif
