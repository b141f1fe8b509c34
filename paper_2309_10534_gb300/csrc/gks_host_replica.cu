// gks_host_replica.cu -- host compilations of the per-point device arithmetic
// (include/gks_host_replica.h), used by unit tests without a GPU.
#include "../../include/gks_host_replica.h"
#include "gks_adjoint.cuh"
#include "gks_device.cuh"
#include "gks_pair.cuh"

namespace {

template <typename T>
int time_coeffs_t(double s, double* cF, double* cD)
{
    T f[6], d[6];
    gks::time_coeffs<T>((T)s, f, d);
    for (int k = 0; k < 6; ++k) { cF[k] = (double)f[k]; cD[k] = (double)d[k]; }
    return 0;
}

template <typename T>
int teno_t(const double* q, double eps, int qpow, double ct1, double ct2, double* faces, double* gauss)
{
    T qq[5];
    for (int k = 0; k < 5; ++k) qq[k] = (T)q[k];
    const gks::TenoParams P{eps, qpow, ct1, ct2};
    gks::TenoSel<T> S;
    gks::teno_select(qq, gks::teno_t<T>(P), S);
    T vp, dp, vm, dm;
    gks::teno_faces(qq, S, vp, dp, vm, dm);
    faces[0] = vp; faces[1] = dp; faces[2] = vm; faces[3] = dm;
    T g[4];
    gks::teno_gauss_pm(S, T(0.28867513459481288), g[0], g[1], g[2], g[3]);
    for (int i = 0; i < 4; ++i) gauss[i] = g[i];
    return S.large ? 1 : 0;
}

// packed TENO-D of the float32 2-D sweep: lane x holds q, lane y -q (the
// selection is sign-symmetric, so lane y must give exactly the negated
// values: a check that the lanes stay independent); faces and Gauss points
// from lane x; -2 if the lanes disagree
int teno_packed(const double* q, double eps, int qpow, double ct1, double ct2, double* faces, double* gauss)
{
    const int large = teno_t<float>(q, eps, qpow, ct1, ct2, faces, gauss);
    gks::f2 qq[5];
    for (int k = 0; k < 5; ++k) qq[k] = gks::f2((float)q[k], -(float)q[k]);
    const gks::TenoParams P{eps, qpow, ct1, ct2};
    gks::TenoSel2 S;
    gks::teno_select_x2(qq, gks::teno_t<float>(P), S);
    gks::f2 fv[4];
    gks::teno_faces_x2(S, fv[0], fv[1], fv[2], fv[3]);
    for (int i = 0; i < 4; ++i) {
        if (fv[i].y() != -fv[i].x()) return -2;
        faces[i] = fv[i].x();
    }
    gks::f2 gv[4];
    gks::teno_gauss_pm_x2(S, 0.28867513459481288f, gv[0], gv[1], gv[2], gv[3]);
    for (int i = 0; i < 4; ++i) {
        if (gv[i].y() != -gv[i].x()) return -2;
        gauss[i] = gv[i].x();
    }
    return large;
}

template <typename T, int DIM, bool NONEQ, bool PRFIX>
int flux_t(int tau_mode, double gamma, double mu, double Pr, double c1, double c2, double dt,
           const double* Wl, const double* Wln, const double* Wlt, const double* Wr, const double* Wrn,
           const double* Wrt, double* F, double* dF)
{
    const double K = DIM == 2 ? (5.0 - 3.0 * gamma) / (gamma - 1.0) + 1.0 : (3.0 - gamma) / (gamma - 1.0);
    gks::FluxParams<T> p;
    p.gm1 = (T)(gamma - 1.0);
    p.K = (T)K;
    p.ntot = (T)(K + DIM);
    p.inv_ntot = (T)(1.0 / (K + DIM));
    p.dt = (T)dt;
    p.c1 = (T)c1;
    p.c2 = (T)c2;
    p.mu = (T)mu;
    p.prfac = (T)(1.0 / Pr - 1.0);
    p.tau_mode = tau_mode;
    gks::Side<T> L, R;
    for (int k = 0; k < 4; ++k) {
        L.W[k] = (T)Wl[k]; L.Wn[k] = (T)Wln[k]; L.Wt[k] = (T)(Wlt ? Wlt[k] : 0.0);
        R.W[k] = (T)Wr[k]; R.Wn[k] = (T)Wrn[k]; R.Wt[k] = (T)(Wrt ? Wrt[k] : 0.0);
    }
    if (DIM == 1) { L.W[2] = L.Wn[2] = L.Wt[2] = R.W[2] = R.Wn[2] = R.Wt[2] = T(0); }
    T f[4], d[4];
    gks::point_flux<T, DIM, NONEQ, PRFIX>(L, R, p, f, d);
    for (int k = 0; k < 4; ++k) { F[k] = (double)f[k]; dF[k] = (double)d[k]; }
    return 0;
}

template <typename T, int DIM>
int flux_dispatch(int tau_mode, double gamma, double mu, double Pr, double c1, double c2, double dt,
                  const double* Wl, const double* Wln, const double* Wlt, const double* Wr,
                  const double* Wrn, const double* Wrt, double* F, double* dF)
{
    if (tau_mode == 0)
        return flux_t<T, DIM, false, false>(tau_mode, gamma, mu, Pr, c1, c2, dt, Wl, Wln, Wlt, Wr, Wrn, Wrt, F, dF);
    if (tau_mode == 2 && Pr != 1.0)
        return flux_t<T, DIM, true, true>(tau_mode, gamma, mu, Pr, c1, c2, dt, Wl, Wln, Wlt, Wr, Wrn, Wrt, F, dF);
    return flux_t<T, DIM, true, false>(tau_mode, gamma, mu, Pr, c1, c2, dt, Wl, Wln, Wlt, Wr, Wrn, Wrt, F, dF);
}

template <typename T>
int teno_vjp_t(const double* q, double eps, int qpow, double ct1, double ct2, const double* gfaces,
               const double* ggauss, double* gq)
{
    T qq[5], g[5] = {T(0), T(0), T(0), T(0), T(0)};
    for (int k = 0; k < 5; ++k) qq[k] = (T)q[k];
    const gks::TenoParams P{eps, qpow, ct1, ct2};
    gks::TenoSel<T> S;
    gks::teno_select(qq, gks::teno_t<T>(P), S);
    gks::teno_faces_T(S, (T)gfaces[0], (T)gfaces[1], (T)gfaces[2], (T)gfaces[3], g);
    gks::teno_gauss_T(S, T(-0.28867513459481288), (T)ggauss[0], (T)ggauss[1], g);
    gks::teno_gauss_T(S, T(0.28867513459481288), (T)ggauss[2], (T)ggauss[3], g);
    for (int k = 0; k < 5; ++k) gq[k] = (double)g[k];
    return S.large ? 1 : 0;
}

template <typename T>
int flux_vjp_t(double gamma, const double* Wl, const double* Wln, const double* Wlt, const double* Wr,
               const double* Wrn, const double* Wrt, const double* gF, const double* gdF, double* gl, double* gr)
{
    const double K = (5.0 - 3.0 * gamma) / (gamma - 1.0) + 1.0;
    gks::FluxParams<T> p{};
    p.gm1 = (T)(gamma - 1.0);
    p.K = (T)K;
    p.ntot = (T)(K + 2.0);
    p.inv_ntot = (T)(1.0 / (K + 2.0));
    p.tau_mode = 0;
    gks::Side<T> L, R, gL, gR;
    T f[4], d[4];
    for (int k = 0; k < 4; ++k) {
        L.W[k] = (T)Wl[k]; L.Wn[k] = (T)Wln[k]; L.Wt[k] = (T)Wlt[k];
        R.W[k] = (T)Wr[k]; R.Wn[k] = (T)Wrn[k]; R.Wt[k] = (T)Wrt[k];
        gL.W[k] = gL.Wn[k] = gL.Wt[k] = gR.W[k] = gR.Wn[k] = gR.Wt[k] = T(0);
        f[k] = (T)gF[k];
        d[k] = (T)gdF[k];
    }
    gks::point_flux_vjp(L, R, p, f, d, gL, gR);
    for (int k = 0; k < 4; ++k) {
        gl[k] = gL.W[k]; gl[4 + k] = gL.Wn[k]; gl[8 + k] = gL.Wt[k];
        gr[k] = gR.W[k]; gr[4 + k] = gR.Wn[k]; gr[8 + k] = gR.Wt[k];
    }
    return 0;
}

template <typename T>
int weno_ao_t(const double* q, double eps_ao, double d_hi, double d_lo, double* faces, double* gauss)
{
    T qq[5];
    for (int k = 0; k < 5; ++k) qq[k] = (T)q[k];
    gks::TenoParams P{1e-40, 7, 1e-7, 1e-5};
    P.recon = 1;
    P.d_hi = d_hi;
    P.d_lo = d_lo;
    P.eps_ao = eps_ao;
    gks::TenoSel<T> S;
    gks::ao_select(qq, gks::teno_t<T>(P), S);
    T vp, dp, vm, dm;
    gks::ao_faces(qq, S, vp, dp, vm, dm);
    faces[0] = vp; faces[1] = dp; faces[2] = vm; faces[3] = dm;
    T v, d;
    gks::ao_gauss(S, T(-0.28867513459481288), v, d);
    gauss[0] = v; gauss[1] = d;
    gks::ao_gauss(S, T(0.28867513459481288), v, d);
    gauss[2] = v; gauss[3] = d;
    return 0;
}

// packed WENO5-AO of the float32 2-D sweep: lane x holds q, lane y -q (its
// weights are sign-symmetric, so lane y must give exactly the negated
// values); -2 if the lanes disagree
int weno_ao_packed(const double* q, double eps_ao, double d_hi, double d_lo, double* faces, double* gauss)
{
    gks::f2 qq[5];
    for (int k = 0; k < 5; ++k) qq[k] = gks::f2((float)q[k], -(float)q[k]);
    gks::TenoParams P{1e-40, 7, 1e-7, 1e-5};
    P.recon = 1;
    P.d_hi = d_hi;
    P.d_lo = d_lo;
    P.eps_ao = eps_ao;
    const gks::TenoT<float> Pf = gks::teno_t<float>(P);
    gks::f2 fv[4], gv[4];
    gks::packed_faces<1>(qq, Pf, fv[0], fv[1], fv[2], fv[3]);
    gks::packed_gauss<1>(qq, Pf, -0.28867513459481288f, 0.28867513459481288f, gv[0], gv[1], gv[2], gv[3]);
    for (int i = 0; i < 4; ++i) {
        if (fv[i].y() != -fv[i].x() || gv[i].y() != -gv[i].x()) return -2;
        faces[i] = fv[i].x();
        gauss[i] = gv[i].x();
    }
    return 0;
}

}  // namespace

extern "C" int gks_host_weno_ao(int precision, const double* q, double eps_ao, double d_hi, double d_lo,
                                double* faces, double* gauss)
{
    if (!q || !faces || !gauss || !(d_hi > 0.0)) return -1;
    if (precision == 2) return weno_ao_packed(q, eps_ao, d_hi, d_lo, faces, gauss);
    return precision == 1 ? weno_ao_t<float>(q, eps_ao, d_hi, d_lo, faces, gauss)
                          : weno_ao_t<double>(q, eps_ao, d_hi, d_lo, faces, gauss);
}

template <typename T, int REC>
int weno3_t(const double* q, double eps, int qpow, double ct, double* faces)
{
    T qq[5];
    for (int k = 0; k < 5; ++k) qq[k] = (T)q[k];
    gks::TenoParams P{eps, qpow, ct, 0.0};
    P.recon = REC;
    P.eps_ao = eps;
    gks::TenoSel<T> S;
    gks::rec_select<REC>(qq, gks::teno_t<T>(P), S);
    T vp, dp, vm, dm;
    gks::rec_faces<REC>(qq, S, vp, dp, vm, dm);
    faces[0] = vp; faces[1] = dp; faces[2] = vm; faces[3] = dm;
    return 0;
}

template <typename T, int REC>
int weno3_gauss_t(const double* q, double eps, int qpow, double ct, double* gauss)
{
    T qq[5];
    for (int k = 0; k < 5; ++k) qq[k] = (T)q[k];
    gks::TenoParams P{eps, qpow, ct, 0.0};
    P.recon = REC;
    P.eps_ao = eps;
    gks::TenoSel<T> S;
    gks::rec_select<REC>(qq, gks::teno_t<T>(P), S);
    T g[4];
    gks::rec_gauss_pm<REC>(S, T(0.28867513459481288), g[0], g[1], g[2], g[3]);
    for (int i = 0; i < 4; ++i) gauss[i] = g[i];
    return 0;
}

template <typename T, int DIM>
int char_face_t(double gamma, const double* w, double eps, int qpow, double ct1, double ct2, double* out)
{
    T ww[6][4];
    for (int c = 0; c < 6; ++c)
        for (int v = 0; v < 4; ++v) ww[c][v] = (T)w[4 * c + v];
    const gks::TenoParams P{eps, qpow, ct1, ct2};
    T o[4][4];
    gks::char_face<T, DIM>(ww, gks::teno_t<T>(P), (T)(gamma - 1.0), o[0], o[1], o[2], o[3]);
    for (int k = 0; k < 4; ++k)
        for (int v = 0; v < 4; ++v) out[4 * k + v] = (double)o[k][v];
    return 0;
}

template <typename T>
int merge_t(int dim, double gamma, const double* Wl, const double* Wr, double* W0)
{
    const double K = dim == 2 ? (5.0 - 3.0 * gamma) / (gamma - 1.0) + 1.0 : (3.0 - gamma) / (gamma - 1.0);
    gks::FluxParams<T> p{};
    p.gm1 = (T)(gamma - 1.0);
    p.K = (T)K;
    T l[4], r[4], w0[4];
    for (int k = 0; k < 4; ++k) { l[k] = (T)Wl[k]; r[k] = (T)Wr[k]; }
    if (dim == 2) gks::merge_values<T, 2>(l, r, p, w0);
    else gks::merge_values<T, 1>(l, r, p, w0);
    for (int k = 0; k < 4; ++k) W0[k] = (double)w0[k];
    return 0;
}

extern "C" int gks_host_weno3_gauss(int precision, int teno5, const double* q, double eps, int qpow, double ct,
                                    double* gauss)
{
    if (!q || !gauss || qpow < 1 || !(eps > 0.0)) return -1;
    if (teno5)
        return precision == 1 ? weno3_gauss_t<float, 3>(q, eps, qpow, ct, gauss)
                              : weno3_gauss_t<double, 3>(q, eps, qpow, ct, gauss);
    return precision == 1 ? weno3_gauss_t<float, 2>(q, eps, qpow, ct, gauss)
                          : weno3_gauss_t<double, 2>(q, eps, qpow, ct, gauss);
}

extern "C" int gks_host_merge(int dim, int precision, double gamma, const double* Wl, const double* Wr, double* W0)
{
    if ((dim != 1 && dim != 2) || !Wl || !Wr || !W0) return -1;
    return precision == 1 ? merge_t<float>(dim, gamma, Wl, Wr, W0) : merge_t<double>(dim, gamma, Wl, Wr, W0);
}

extern "C" int gks_host_weno3(int precision, int teno5, const double* q, double eps, int qpow, double ct,
                              double* faces)
{
    if (!q || !faces || qpow < 1 || !(eps > 0.0)) return -1;
    if (teno5)
        return precision == 1 ? weno3_t<float, 3>(q, eps, qpow, ct, faces) : weno3_t<double, 3>(q, eps, qpow, ct, faces);
    return precision == 1 ? weno3_t<float, 2>(q, eps, qpow, ct, faces) : weno3_t<double, 2>(q, eps, qpow, ct, faces);
}

extern "C" int gks_host_teno_vjp(int precision, const double* q, double eps, int qpow, double ct1, double ct2,
                                 const double* gfaces, const double* ggauss, double* gq)
{
    if (!q || !gfaces || !ggauss || !gq || qpow < 1) return -1;
    return precision == 1 ? teno_vjp_t<float>(q, eps, qpow, ct1, ct2, gfaces, ggauss, gq)
                          : teno_vjp_t<double>(q, eps, qpow, ct1, ct2, gfaces, ggauss, gq);
}

extern "C" int gks_host_point_flux_vjp(int precision, double gamma, const double* Wl, const double* Wln,
                                       const double* Wlt, const double* Wr, const double* Wrn, const double* Wrt,
                                       const double* gF, const double* gdF, double* gl, double* gr)
{
    if (!Wl || !Wln || !Wlt || !Wr || !Wrn || !Wrt || !gF || !gdF || !gl || !gr) return -1;
    return precision == 1 ? flux_vjp_t<float>(gamma, Wl, Wln, Wlt, Wr, Wrn, Wrt, gF, gdF, gl, gr)
                          : flux_vjp_t<double>(gamma, Wl, Wln, Wlt, Wr, Wrn, Wrt, gF, gdF, gl, gr);
}

extern "C" int gks_host_physical(int dim, int precision, double gamma, const double* W)
{
    if (!W || (dim != 1 && dim != 2) || (precision != 0 && precision != 1) || !(gamma > 1.0)) return -1;
    if (precision == 1) {
        float w[4];
        for (int i = 0; i < 4; ++i) w[i] = (float)W[i];
        return dim == 2 ? gks::physical<float, 2>(w, (float)(gamma - 1.0)) : gks::physical<float, 1>(w, (float)(gamma - 1.0));
    }
    return dim == 2 ? gks::physical<double, 2>(W, gamma - 1.0) : gks::physical<double, 1>(W, gamma - 1.0);
}

extern "C" int gks_host_time_coeffs(int precision, double s, double* cF, double* cD)
{
    if (!cF || !cD || !(s > 0.0)) return -1;
    return precision == 1 ? time_coeffs_t<float>(s, cF, cD) : time_coeffs_t<double>(s, cF, cD);
}

extern "C" int gks_host_teno(int precision, const double* q, double eps, int qpow, double ct1, double ct2,
                             double* faces, double* gauss)
{
    if (!q || !faces || !gauss || qpow < 1) return -1;
    if (precision == 2) return teno_packed(q, eps, qpow, ct1, ct2, faces, gauss);
    return precision == 1 ? teno_t<float>(q, eps, qpow, ct1, ct2, faces, gauss)
                          : teno_t<double>(q, eps, qpow, ct1, ct2, faces, gauss);
}

extern "C" int gks_host_point_flux(int dim, int precision, int tau_mode, double gamma, double mu, double Pr,
                                   double c1, double c2, double dt, const double* Wl, const double* Wln,
                                   const double* Wlt, const double* Wr, const double* Wrn, const double* Wrt,
                                   double* F, double* dF)
{
    if ((dim != 1 && dim != 2) || tau_mode < 0 || tau_mode > 2 || !Wl || !Wln || !Wr || !Wrn || !F || !dF)
        return -1;
    if (dim == 2)
        return precision == 1 ? flux_dispatch<float, 2>(tau_mode, gamma, mu, Pr, c1, c2, dt, Wl, Wln, Wlt, Wr, Wrn, Wrt, F, dF)
                              : flux_dispatch<double, 2>(tau_mode, gamma, mu, Pr, c1, c2, dt, Wl, Wln, Wlt, Wr, Wrn, Wrt, F, dF);
    return precision == 1 ? flux_dispatch<float, 1>(tau_mode, gamma, mu, Pr, c1, c2, dt, Wl, Wln, Wlt, Wr, Wrn, Wrt, F, dF)
                          : flux_dispatch<double, 1>(tau_mode, gamma, mu, Pr, c1, c2, dt, Wl, Wln, Wlt, Wr, Wrn, Wrt, F, dF);
}

extern "C" int gks_host_char_face(int dim, int precision, double gamma, const double* w, double eps, int qpow,
                                  double ct1, double ct2, double* out)
{
    if (!w || !out || (dim != 1 && dim != 2) || (precision != 0 && precision != 1) || qpow < 1) return -1;
    if (precision == 1)
        return dim == 2 ? char_face_t<float, 2>(gamma, w, eps, qpow, ct1, ct2, out)
                        : char_face_t<float, 1>(gamma, w, eps, qpow, ct1, ct2, out);
    return dim == 2 ? char_face_t<double, 2>(gamma, w, eps, qpow, ct1, ct2, out)
                    : char_face_t<double, 1>(gamma, w, eps, qpow, ct1, ct2, out);
}
