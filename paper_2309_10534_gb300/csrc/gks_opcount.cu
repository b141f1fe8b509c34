// gks_opcount.cu -- algorithmic operation count of the library's own stage
// arithmetic.  The device functions of gks_device.cuh are replayed on the
// host with a scalar type that counts every add/sub, multiply, divide,
// square root, exp and erfc; the per-cell totals follow from how many times
// a stage applies each function (no tile halos or padding counted).
#include <cfloat>
#include <cmath>
#include <mutex>

#include "../../include/gks.h"
#include "gks_device.cuh"

namespace gks {
namespace opc {

struct Counts {
    double add = 0, mul = 0, div = 0, sqrt = 0, exp = 0, erfc = 0;
    double flops() const { return add + mul + div + sqrt; }
    Counts& operator+=(const Counts& o)
    {
        add += o.add; mul += o.mul; div += o.div; sqrt += o.sqrt; exp += o.exp; erfc += o.erfc;
        return *this;
    }
    Counts scaled(double s) const
    {
        Counts c = *this;
        c.add *= s; c.mul *= s; c.div *= s; c.sqrt *= s; c.exp *= s; c.erfc *= s;
        return c;
    }
};
static Counts g_cnt;

template <typename B> struct Cnt {
    B v;
    constexpr Cnt() : v(0) {}
    constexpr Cnt(double x) : v((B)x) {}
    friend Cnt operator+(Cnt a, Cnt b) { g_cnt.add += 1; return Cnt(a.v + b.v); }
    friend Cnt operator-(Cnt a, Cnt b) { g_cnt.add += 1; return Cnt(a.v - b.v); }
    friend Cnt operator*(Cnt a, Cnt b) { g_cnt.mul += 1; return Cnt(a.v * b.v); }
    friend Cnt operator/(Cnt a, Cnt b) { g_cnt.div += 1; return Cnt(a.v / b.v); }
    friend Cnt operator-(Cnt a) { return Cnt(-a.v); }
    friend Cnt fma(Cnt a, Cnt b, Cnt c) { g_cnt.mul += 1; g_cnt.add += 1; return Cnt(a.v * b.v + c.v); }
    Cnt& operator+=(Cnt b) { *this = *this + b; return *this; }
    Cnt& operator-=(Cnt b) { *this = *this - b; return *this; }
    Cnt& operator*=(Cnt b) { *this = *this * b; return *this; }
    friend bool operator<(Cnt a, Cnt b) { return a.v < b.v; }
    friend bool operator<=(Cnt a, Cnt b) { return a.v <= b.v; }
    friend bool operator>(Cnt a, Cnt b) { return a.v > b.v; }
    friend bool operator>=(Cnt a, Cnt b) { return a.v >= b.v; }
    friend Cnt fabs(Cnt a) { return Cnt(std::fabs((double)a.v)); }
    friend bool isfinite(Cnt a) { return std::isfinite((double)a.v); }
};

}  // namespace opc

template <typename B> struct M<opc::Cnt<B>> {
    using C = opc::Cnt<B>;
    static C erfc_(C x) { opc::g_cnt.erfc += 1; return C(std::erfc((double)x.v)); }
    static C exp_(C x) { opc::g_cnt.exp += 1; return C(std::exp((double)x.v)); }
    static C sqrt_(C x) { opc::g_cnt.sqrt += 1; return C(std::sqrt((double)x.v)); }
    static C rcp(C x) { opc::g_cnt.div += 1; return C(1.0 / (double)x.v); }
    static constexpr double tiny = M<B>::tiny;
    static constexpr int nseries = M<B>::nseries;
    static constexpr double s_series = M<B>::s_series;
    static constexpr double s_noexp = M<B>::s_noexp;
};

namespace opc {

template <typename F>
Counts measure(F&& f)
{
    g_cnt = Counts();
    f();
    return g_cnt;
}

// representative smooth inputs (the dominant branch of the workloads: large
// stencil, closed-form time coefficients)
template <typename T, int DIM>
void sample_side(Side<T>& S, double rho, double U, double V, double p, double gamma, double eps)
{
    const double E = p / (gamma - 1.0) + 0.5 * rho * (U * U + V * V);
    const double w[4] = {rho, rho * U, rho * V, E};
    for (int i = 0; i < 4; ++i) {
        S.W[i] = T(w[i] * (1.0 + eps));
        S.Wn[i] = T(0.01 * w[i]);
        S.Wt[i] = T(DIM == 2 ? -0.02 * w[i] : 0.0);
    }
    if (DIM == 1) { S.W[2] = S.Wn[2] = S.Wt[2] = T(0); }
}

template <typename B, int DIM, bool NONEQ, bool PRFIX, int REC>
void count(int tau_mode, double Pr, gks_flop_model* out)
{
    using T = Cnt<B>;
    const double gamma = 1.4;
    const double K = DIM == 2 ? (5.0 - 3.0 * gamma) / (gamma - 1.0) + 1.0 : (3.0 - gamma) / (gamma - 1.0);
    FluxParams<T> fp;
    fp.gm1 = T(gamma - 1.0);
    fp.K = T(K);
    fp.ntot = T(K + DIM);
    fp.inv_ntot = T(1.0 / (K + DIM));
    fp.dt = T(1e-3);
    fp.c1 = T(0.01);
    fp.c2 = T(1.0);
    fp.mu = T(tau_mode == 2 ? 1e-4 : 0.0);
    fp.prfac = T(1.0 / Pr - 1.0);
    fp.tau_mode = tau_mode;
    const TenoParams tp0{1e-40, 7, 1e-7, 1e-5};
    TenoT<T> tp;
    tp.eps = T(1e-40);
    tp.ct1 = T(1e-7);
    tp.ct2 = T(1e-5);
    tp.q = (REC == 3) ? 6 : tp0.q;
    {
        const TenoT<double> td = teno_t<double>(tp0);
        for (int k = 0; k < 4; ++k) tp.g[k] = T(td.g[k]);
        for (int k = 0; k < 3; ++k) tp.gr[k] = T(td.gr[k]);
        tp.ig3 = T(td.ig3);
        tp.eps_ao = T(td.eps_ao);
    }

    const T q[5] = {T(1.00), T(1.011), T(1.023), T(1.036), T(1.050)};
    constexpr int RB = rec_base(REC);
    const Counts recon = measure([&] {
        TenoSel<T> S;
        rec_select<RB>(q, tp, S);
        T a, b, c, d;
        rec_faces<RB>(q, S, a, b, c, d);
    });
    const Counts tang = measure([&] {
        TenoSel<T> S;
        rec_select<RB>(q, tp, S);
        T a, b, c, d;
        rec_gauss_pm<RB>(S, T(0.28867513459481288), a, b, c, d);
    });
    // characteristic variables: per face the basis, six projections, two
    // sides of every field and four back-projections
    Counts charface;
    if constexpr (REC == REC_TENO_CHAR) {
        T w[6][4];
        for (int c = 0; c < 6; ++c) {
            const double rho = 1.0 + 0.01 * c, U = 0.3 + 0.002 * c, V = DIM == 2 ? 0.2 - 0.001 * c : 0.0;
            const double p = 1.0 + 0.015 * c;
            w[c][0] = T(rho);
            w[c][1] = T(rho * U);
            w[c][2] = T(rho * V);
            w[c][3] = T(p / (gamma - 1.0) + 0.5 * rho * (U * U + V * V));
        }
        charface = measure([&] {
            T vl[4], dl[4], vr[4], dr[4];
            char_face<T, DIM>(w, tp, fp.gm1, vl, dl, vr, dr);
        });
    }
    Side<T> L0_, R0_;
    sample_side<T, DIM>(L0_, 1.0, 0.3, 0.2, 1.0, gamma, 0.0);
    sample_side<T, DIM>(R0_, 1.0, 0.3, 0.2, 1.0, gamma, 1e-4);
    // the conventional path in 2-D: per face one line merge and four
    // Eq. (3.12) slopes (Step 2), per Gauss point eight quartic evaluations
    // (Step 4)
    Counts conv2d;
    if constexpr (rec_conventional(REC) && DIM == 2) {
        const Counts merge = measure([&] {
            T w0[4];
            merge_values<T, 2>(L0_.W, R0_.W, fp, w0);
        });
        const Counts quart = measure([&] {
            T v, d;
            quartic_gauss(q, T(0.28867513459481288), v, d);
        });
        Counts lin;
        lin.add = 4 * 3;
        lin.mul = 4 * 3;
        conv2d += merge;
        conv2d += lin;
        conv2d += quart.scaled(16);
    }
    Side<T> L, R;
    sample_side<T, DIM>(L, 1.0, 0.3, 0.2, 1.0, gamma, 0.0);
    sample_side<T, DIM>(R, 1.0, 0.3, 0.2, 1.0, gamma, 1e-4);
    const Counts flux = measure([&] {
        T F[4], dF[4];
        point_flux<T, DIM, NONEQ, PRFIX>(L, R, fp, F, dF);
    });

    const int nv = DIM + 2;
    Counts sweep;  // per cell, one stage kernel of one direction
    if (REC == REC_TENO_CHAR) sweep += charface;   // normal TENO-D per face in characteristic variables
    else sweep += recon.scaled(nv);                // normal TENO-D, one per cell and variable
    if (DIM == 2) {
        // per face: 2 sides x 4 variables x (value, normal slope) tangential selections
        sweep += tang.scaled(16);
        sweep += flux.scaled(2);                   // two Gauss points
        sweep += conv2d;
        Counts avg;
        avg.add = 8;                               // average of F, dF over the Gauss points
        avg.mul = 8;
        sweep += avg;
    } else {
        sweep += flux;
        if (rec_conventional(REC)) {  // the equilibrium slope of Eq. (3.12) per face
            Counts lin;
            lin.add = 3 * nv;
            lin.mul = 3 * nv;
            sweep += lin;
        }
    }
    Counts upd1, upd2;                              // stage combinations and update, per cell
    upd1.add = nv * (2 + 2 + 2);                   // G1, G2 sums, two differences, two updates
    upd1.mul = nv * (3 + 2 + 2);
    upd2.add = nv * (1 + 1);
    upd2.mul = nv * (2 + 1);
    Counts s1 = sweep, s2 = sweep;
    s1 += upd1;
    s2 += upd2;
    const int sweeps = DIM;                        // sweeps per stage
    Counts step = s1.scaled(sweeps);
    step += s2.scaled(sweeps);
    out->flops_per_cell_update = step.flops();
    out->flops_per_cell_sweep = 0.5 * (s1.flops() + s2.flops());
    out->transcendentals_per_cell_update = step.exp + step.erfc;
    out->divides_per_cell_update = step.div;
    out->sqrt_per_cell_update = step.sqrt;
    // float64 arithmetic on the mixed path: the update (per sweep) only
    out->fp64_flops_per_cell_update =
        sizeof(B) == 4 ? (double)sweeps * (upd1.add + 2 * nv + upd2.add + nv) : step.flops();
}

}  // namespace opc
}  // namespace gks

namespace {
template <int REC>
void count_rec(int dim, bool f32, int tau_mode, double Pr, gks_flop_model* out)
{
    using namespace gks::opc;
    const bool pr = tau_mode == 2 && Pr != 1.0;
#define GKS_COUNT(B, D)                                                     \
    if (tau_mode == 0) count<B, D, false, false, REC>(tau_mode, Pr, out);   \
    else if (pr) count<B, D, true, true, REC>(tau_mode, Pr, out);           \
    else count<B, D, true, false, REC>(tau_mode, Pr, out);
    if (f32 && dim == 2) { GKS_COUNT(float, 2) }
    else if (f32) { GKS_COUNT(float, 1) }
    else if (dim == 2) { GKS_COUNT(double, 2) }
    else { GKS_COUNT(double, 1) }
#undef GKS_COUNT
}
}  // namespace

extern "C" gks_status gks_count_flops_recon(int dim, int precision, int tau_mode, double Pr, int recon,
                                            gks_flop_model* out)
{
    static std::mutex mu;
    std::lock_guard<std::mutex> lock(mu);
    if (!out || (dim != 1 && dim != 2) || tau_mode < 0 || tau_mode > 2 || !(Pr > 0.0) || recon < 0 ||
        (recon > 3 && recon != GKS_COUNT_TENO_CHARVARS))
        return GKS_EINVAL;
    const bool f32 = precision == GKS_FP32_FLUX;
    if (recon == GKS_COUNT_TENO_CHARVARS) count_rec<gks::REC_TENO_CHAR>(dim, f32, tau_mode, Pr, out);
    else if (recon == 1) count_rec<1>(dim, f32, tau_mode, Pr, out);
    else if (recon == 2) count_rec<2>(dim, f32, tau_mode, Pr, out);
    else if (recon == 3) count_rec<3>(dim, f32, tau_mode, Pr, out);
    else count_rec<0>(dim, f32, tau_mode, Pr, out);
    return GKS_OK;
}

extern "C" gks_status gks_count_flops(int dim, int precision, int tau_mode, double Pr, gks_flop_model* out)
{
    return gks_count_flops_recon(dim, precision, tau_mode, Pr, GKS_RECON_TENO_D, out);
}
