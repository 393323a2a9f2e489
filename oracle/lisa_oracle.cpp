// Plain, slow, FP64 CPU oracle for the spline-perturbed Whittle/Wishart log-likelihood of
// averaged A/E/T periodograms (arXiv:2507.06300, "A flexible, GPU-accelerated approach for the
// joint characterization of LISA instrumental noise and SGWBs").
//
// TEST INFRASTRUCTURE ONLY. This file exists to check the CUDA library. Only the test suite, the
// package smoke check and the benchmark's CPU-baseline leg may load it. It shares no code,
// header, table or constant generator with the CUDA path, and it never calls it.
//
// What each function follows (paper sections / equations):
//   S_TM, S_OMS ........................ Sec. II.B (test-mass and OMS PSDs)
//   A/E/T noise transfer ............... Sec. II.B, Eq. (noise_tdi)
//   power-law SGWB, S_h ................ Sec. II.C, Eq. (pl) and Eq. (Sh)
//   multiplicative perturbations ....... Sec. III.A, Eq. (splines): S * 10^P
//   knot layout (edges + in-between) ... Sec. III.A, knot placement scheme
//   linear fallback ................... Sec. III.A (fewer than two in-between knots)
//   Akima slopes and coefficients ...... Appendix A
//   per-bin Wishart term, bin sum ...... Sec. III.C (Wishart log-density, sum over bins)
//   full 3x3 covariance ................ Sec. III.A (the complete analysis with six flexible
//                                        noise terms), Sec. III.C (the same Wishart term with a
//                                        dense C), reading R16 below
//
// Readings taken where the paper is ambiguous or garbled:
//   R1  covariance: C_c = S_c (the printed factor 1/2 is dropped; the periodogram is normalised
//       to the one-sided PSD), so the per-bin term is -nu * sum_c (P_c/S_c + ln S_c).
//   R2  TDI prefactor: default exactly as printed, sin^2(u) * sin^4(u); tdi_form=1 selects
//       sin^2(u) * sin^2(2u).  1 - cos(u) is evaluated as 2 sin^2(u/2) (same value, no
//       cancellation at low frequency).
//   R3  Akima tie rule for the general knot: (m_{i-1} + m_i)/2 (Akima's original and SciPy's
//       fill value), with an exact zero test on w_i + w_{i-2}.
//   R3b Akima s_{n-1}: the mirror image of s_2 (weights w_{n-3} on m_{n-1} and w_{n-2} on
//       m_{n-2}), which is what SciPy computes; the printed form is shifted by one index.
//   R4  spline abscissa x = log10(f).
//   R5  edge knots at x_lo, x_hi given per dataset; in-between knots need x_lo < x_k < x_hi.
//   R6  in-between knots are sorted ascending; equal positions make the state invalid; a bin
//       exactly on a knot uses the interval to its right; x >= last knot uses the last interval;
//       x < first knot uses the first interval (polynomial extrapolation).
//   R7  fewer than two in-between knots (fewer than 4 points) -> linear interpolant, for both
//       spline kinds.
//   R8  f_ref (f_knee) is an input; H0/h = 100 km/s/Mpc exactly.
//   R9  broken power law (sgwb_model 2): slope n1 below f_ref, n2 at and above it.
//   R10 natural cubic spline (kind 1) is the C^2 alternative named next to Akima; its
//       coefficients come from the textbook second-derivative tridiagonal system.
//   R16 full covariance (the paper defers the construction of a positive-definite matrix from six
//       flexible terms to another reference): in the A, E, T basis,
//         C = D^{1/2} R D^{1/2} + H,  D = diag(S_n,cc 10^{P_n,c}),  H = diag(S_h,cc 10^{P_h}),
//         R = L L^T,  L = [[1, 0, 0], [r_AE, s_AE, 0], [r_AT, r_ET s_AT, s_AT s_ET]],
//         r = z / sqrt(1 + z^2),  s = 1 / sqrt(1 + z^2)  (= sqrt(1 - r^2)),
//       with z_AE, z_AT, z_ET three more variable-knot splines whose values (not exponents) are
//       the flexible off-diagonal terms: three diagonal and three correlation terms, C positive
//       definite for any spline values, and the diagonal model exactly when z = 0.  C is real, so
//       only the real parts of the averaged periodogram's off-diagonal entries enter
//       tr(C^-1 P); the oracle forms the complex trace and checks that its imaginary part
//       vanishes only through the Hermitian symmetry of P.
//
// Layouts (all row-major, caller-owned):
//   theta [S][5]              a_oms = A_OMS/1e-12, a_tm = A_TM/1e-15, log10 A, n1, n2
//   count [S][nsp]            number of in-between knots k (0..kmax)
//   kx    [S][nsp][kmax]      in-between knot positions log10 f (any order)
//   kw    [S][nsp][kmax+2]    amplitudes: slot 0 = w_0 (left edge), slot 1+j = knot j,
//                             slot kmax+1 = w_n (right edge)
//   spline index: 0..C-1 = noise of channel A, E (, T); C = the SGWB spline (if present)
//   grad  [S][5 + nsp*(2*kmax+2)]  d logL / d(theta), then per spline d/d(kw slots), d/d(kx)
//
// Status bits per state (0 = valid):
//   1 knot count outside [0, kmax]; 2 position non-finite or not strictly inside (x_lo, x_hi);
//   4 two in-between knots at the same position; 8 non-finite amplitude;
//   16 non-finite template parameter; 32 non-finite or non-positive PSD, or non-finite logL.
// An invalid state gets logL = -inf and a zero gradient.

#include <algorithm>
#include <complex>
#include <cmath>
#include <cstdint>
#include <limits>
#include <vector>

namespace {

const double kPi = 3.14159265358979323846;
const double kArm = 2.5e9;             // L, m (Sec. II.A)
const double kC = 299792458.0;         // speed of light, m/s
const double kMpc = 3.0856775814913673e22;  // m
const double kH0overh = 1.0e5 / kMpc;  // 100 km/s/Mpc in 1/s (Sec. II.C quotes ~3.24e-18 Hz)
const double kLn10 = 2.302585092994045684;

// ---------------------------------------------------------------------------------------------
// Forward-mode dual number, used only for the analytic gradient of the spline value with
// respect to one knot parameter at a time.
struct Dual {
    double v, d;
    Dual(double v_ = 0.0, double d_ = 0.0) : v(v_), d(d_) {}
};
inline Dual operator+(Dual a, Dual b) { return Dual(a.v + b.v, a.d + b.d); }
inline Dual operator-(Dual a, Dual b) { return Dual(a.v - b.v, a.d - b.d); }
inline Dual operator-(Dual a) { return Dual(-a.v, -a.d); }
inline Dual operator*(Dual a, Dual b) { return Dual(a.v * b.v, a.d * b.v + a.v * b.d); }
inline Dual operator/(Dual a, Dual b) {
    return Dual(a.v / b.v, (a.d * b.v - a.v * b.d) / (b.v * b.v));
}
inline Dual operator*(double a, Dual b) { return Dual(a * b.v, a * b.d); }
inline Dual dabs(Dual a) { return a.v < 0 ? -a : (a.v > 0 ? a : Dual(0.0, 0.0)); }
inline double dabs(double a) { return std::fabs(a); }
inline double val(double a) { return a; }
inline double val(Dual a) { return a.v; }

// ---------------------------------------------------------------------------------------------
// Sec. II.B: one-sided PSDs of the test-mass acceleration and OMS noise.
double S_tm(double f, double A_tm) {
    double lo = 0.4e-3 / f, hi = f / 8.0e-3, conv = 1.0 / (2.0 * kPi * f * kC);
    return A_tm * A_tm * (1.0 + lo * lo) * (1.0 + hi * hi * hi * hi) * conv * conv;
}
double S_oms(double f, double A_oms) {
    double lo = 2.0e-3 / f, conv = 2.0 * kPi * f / kC;
    return A_oms * A_oms * (1.0 + lo * lo * lo * lo) * conv * conv;
}

// Eq. (noise_tdi): A/E/T noise PSDs with the TDI-2 transfer functions.  out[c], c = A, E, T.
void noise_aet(int tdi_form, double f, double A_oms, double A_tm, double out[3]) {
    double u = 2.0 * kPi * f * kArm / kC;
    double su = std::sin(u), cu = std::cos(u);
    double pref;
    if (tdi_form == 0) {
        pref = su * su * su * su * su * su;          // sin^2(u) sin^4(u), as printed
    } else {
        double s2u = std::sin(2.0 * u);
        pref = su * su * s2u * s2u;                  // sin^2(u) sin^2(2u)
    }
    double s_oms = S_oms(f, A_oms), s_tm = S_tm(f, A_tm);
    double aa = 32.0 * pref * ((2.0 + cu) * s_oms + 4.0 * (1.0 + cu + cu * cu) * s_tm);
    double sh = std::sin(0.5 * u);
    double omc = 2.0 * sh * sh;                      // 1 - cos(u)
    double tt = 64.0 * pref * (omc * s_oms + 2.0 * omc * omc * s_tm);
    out[0] = aa;
    out[1] = aa;
    out[2] = tt;
}

// Eq. (pl): h^2 Omega(f) = A (f/f_knee)^n; sgwb_model 2 takes n1 below f_ref and n2 above.
double h2omega(int sgwb_model, double f, double log10A, double n1, double n2, double f_ref) {
    double n = (sgwb_model == 2 && f >= f_ref) ? n2 : n1;
    return std::pow(10.0, log10A) * std::pow(f / f_ref, n);
}

// Eq. (Sh): S_h = R(f) h^2 Omega(f) 3 (H0/h)^2 / (4 pi^2 f^3).
double sgwb_psd(double R, double h2om, double f) {
    return R * h2om * 3.0 * kH0overh * kH0overh / (4.0 * kPi * kPi * f * f * f);
}

// ---------------------------------------------------------------------------------------------
// Splines.  Knots are kept 1-based (index 0 unused) so that the Akima code below reads like
// Appendix A: knots (x_i, y_i), i = 1..n; interval slopes m_i, i = 1..n-1; w_i = |m_{i+1} - m_i|.
template <class T>
struct Spline {
    int n = 0;                         // number of knots (edges included)
    std::vector<T> x, y;               // [n+1], 1-based
    std::vector<T> a, b, c, d;         // [n], interval i = 1..n-1
};

template <class T>
void linear_coeffs(Spline<T>& sp) {
    int n = sp.n;
    for (int i = 1; i <= n - 1; ++i) {
        sp.a[i] = sp.y[i];
        sp.b[i] = (sp.y[i + 1] - sp.y[i]) / (sp.x[i + 1] - sp.x[i]);
        sp.c[i] = T(0.0);
        sp.d[i] = T(0.0);
    }
}

// Appendix A: Akima slopes with the SciPy-style end conditions, then the cubic coefficients.
template <class T>
void akima_coeffs(Spline<T>& sp) {
    int n = sp.n;  // n >= 4
    std::vector<T> m(n + 1), w(n + 1), s(n + 1);
    for (int i = 1; i <= n - 1; ++i) m[i] = (sp.y[i + 1] - sp.y[i]) / (sp.x[i + 1] - sp.x[i]);
    for (int i = 1; i <= n - 2; ++i) w[i] = dabs(m[i + 1] - m[i]);

    s[1] = 0.5 * (3.0 * m[1] - m[2]);
    if (val(w[2] + w[1]) == 0.0)
        s[2] = 0.5 * (m[3] + m[2]);
    else
        s[2] = (w[2] * m[1] + w[1] * m[2]) / (w[2] + w[1]);
    for (int i = 3; i <= n - 2; ++i) {
        if (val(w[i] + w[i - 2]) == 0.0)
            s[i] = 0.5 * (m[i - 1] + m[i]);                        // reading R3
        else
            s[i] = (w[i] * m[i - 1] + w[i - 2] * m[i]) / (w[i] + w[i - 2]);
    }
    if (val(w[n - 3] + w[n - 2]) == 0.0)
        s[n - 1] = 0.5 * (m[n - 3] + m[n - 2]);
    else
        s[n - 1] = (w[n - 3] * m[n - 1] + w[n - 2] * m[n - 2]) / (w[n - 3] + w[n - 2]);  // R3b
    s[n] = 0.5 * (3.0 * m[n - 1] - m[n - 2]);

    for (int i = 1; i <= n - 1; ++i) {
        T h = sp.x[i + 1] - sp.x[i];
        sp.a[i] = sp.y[i];
        sp.b[i] = s[i];
        sp.c[i] = (3.0 * m[i] - 2.0 * s[i] - s[i + 1]) / h;
        sp.d[i] = (s[i] + s[i + 1] - 2.0 * m[i]) / (h * h);
    }
}

// Natural cubic spline: second derivatives M_1 = M_n = 0 and, for i = 2..n-1,
//   h_{i-1} M_{i-1} + 2 (h_{i-1} + h_i) M_i + h_i M_{i+1} = 6 (m_i - m_{i-1}),
// solved with the Thomas algorithm; then a = y_i, b = m_i - h_i (2 M_i + M_{i+1}) / 6,
// c = M_i / 2, d = (M_{i+1} - M_i) / (6 h_i).
template <class T>
void natural_coeffs(Spline<T>& sp) {
    int n = sp.n;
    std::vector<T> h(n + 1), m(n + 1), M(n + 1, T(0.0));
    for (int i = 1; i <= n - 1; ++i) {
        h[i] = sp.x[i + 1] - sp.x[i];
        m[i] = (sp.y[i + 1] - sp.y[i]) / h[i];
    }
    int nu = n - 2;  // unknowns M_2..M_{n-1}
    std::vector<T> lo(nu + 1), di(nu + 1), up(nu + 1), rh(nu + 1);
    for (int r = 1; r <= nu; ++r) {
        int i = r + 1;
        lo[r] = h[i - 1];
        di[r] = 2.0 * (h[i - 1] + h[i]);
        up[r] = h[i];
        rh[r] = 6.0 * (m[i] - m[i - 1]);
    }
    for (int r = 2; r <= nu; ++r) {
        T f = lo[r] / di[r - 1];
        di[r] = di[r] - f * up[r - 1];
        rh[r] = rh[r] - f * rh[r - 1];
    }
    std::vector<T> sol(nu + 2, T(0.0));
    for (int r = nu; r >= 1; --r) {
        T acc = rh[r];
        if (r < nu) acc = acc - up[r] * sol[r + 1];
        sol[r] = acc / di[r];
    }
    for (int r = 1; r <= nu; ++r) M[r + 1] = sol[r];
    for (int i = 1; i <= n - 1; ++i) {
        sp.a[i] = sp.y[i];
        sp.b[i] = m[i] - h[i] * (2.0 * M[i] + M[i + 1]) / 6.0;
        sp.c[i] = 0.5 * M[i];
        sp.d[i] = (M[i + 1] - M[i]) / (6.0 * h[i]);
    }
}

// Validates one spline's knots and builds it.  Returns status bits (0 = valid).
//   k      number of in-between knots; xin[0..k-1] their positions (any order);
//   win    amplitudes with the kw slot layout (w_0, knots..., w_n at slot kmax+1).
template <class T>
int build_spline(int kind, int k, int kmax, const T* xin, const T* win, double x_lo, double x_hi,
                 Spline<T>& sp) {
    if (k < 0 || k > kmax) return 1;
    int st = 0;
    for (int j = 0; j < k; ++j) {
        double xv = val(xin[j]);
        if (!std::isfinite(xv) || !(xv > x_lo) || !(xv < x_hi)) st |= 2;
        if (!std::isfinite(val(win[1 + j]))) st |= 8;
    }
    if (!std::isfinite(val(win[0])) || !std::isfinite(val(win[kmax + 1]))) st |= 8;
    if (st) return st;
    std::vector<int> order(k);
    for (int j = 0; j < k; ++j) order[j] = j;
    std::sort(order.begin(), order.end(),
              [&](int p, int q) { return val(xin[p]) < val(xin[q]); });
    for (int j = 1; j < k; ++j)
        if (val(xin[order[j]]) == val(xin[order[j - 1]])) return 4;

    int n = k + 2;
    sp.n = n;
    sp.x.assign(n + 1, T(0.0));
    sp.y.assign(n + 1, T(0.0));
    sp.a.assign(n, T(0.0));
    sp.b.assign(n, T(0.0));
    sp.c.assign(n, T(0.0));
    sp.d.assign(n, T(0.0));
    sp.x[1] = T(x_lo);
    sp.y[1] = win[0];
    for (int j = 0; j < k; ++j) {
        sp.x[2 + j] = xin[order[j]];
        sp.y[2 + j] = win[1 + order[j]];
    }
    sp.x[n] = T(x_hi);
    sp.y[n] = win[kmax + 1];

    if (n < 4)
        linear_coeffs(sp);          // Sec. III.A: fewer than two in-between knots
    else if (kind == 1)
        natural_coeffs(sp);
    else
        akima_coeffs(sp);
    return 0;
}

// Appendix A: S(x) = a_i + b_i (x - x_i) + c_i (x - x_i)^2 + d_i (x - x_i)^3 on [x_i, x_{i+1}).
template <class T>
T eval_spline(const Spline<T>& sp, double x) {
    int n = sp.n;
    int i = 1;
    while (i < n - 1 && !(x < val(sp.x[i + 1]))) ++i;   // last interval also takes x >= x_n
    T t = T(x) - sp.x[i];
    return sp.a[i] + sp.b[i] * t + sp.c[i] * t * t + sp.d[i] * t * t * t;
}

struct Problem {
    int C, sgwb_model, tdi_form;
    int64_t N;
    const double *f, *nu, *P, *R;
    double x_lo, x_hi, f_ref;
    int kind, kmax;
};

int n_splines(const Problem& pb) { return pb.C + (pb.sgwb_model != 0 ? 1 : 0); }

// Per-bin building blocks of the model PSD for one state: noise template S_n,c, SGWB template
// S_h,c (both unperturbed), and the four spline values.
struct BinModel {
    double sn[3], sh[3], pert[4];
};

int build_state(const Problem& pb, const double* th, const int* cnt, const double* kx,
                const double* kw, std::vector<Spline<double>>& sps) {
    int nsp = n_splines(pb);
    int st = 0;
    for (int q = 0; q < 5; ++q)
        if (!std::isfinite(th[q])) st |= 16;
    sps.assign(nsp, Spline<double>());
    for (int a = 0; a < nsp; ++a)
        st |= build_spline<double>(pb.kind, cnt[a], pb.kmax, kx + (size_t)a * pb.kmax,
                                   kw + (size_t)a * (pb.kmax + 2), pb.x_lo, pb.x_hi, sps[a]);
    return st;
}

void bin_model(const Problem& pb, const double* th, const std::vector<Spline<double>>& sps,
               int64_t i, BinModel& bm) {
    double f = pb.f[i];
    double x = std::log10(f);
    double tmp[3];
    noise_aet(pb.tdi_form, f, th[0] * 1e-12, th[1] * 1e-15, tmp);
    double h2 = pb.sgwb_model ? h2omega(pb.sgwb_model, f, th[2], th[3], th[4], pb.f_ref) : 0.0;
    for (int c = 0; c < pb.C; ++c) {
        bm.sn[c] = tmp[c];
        bm.sh[c] = pb.sgwb_model ? sgwb_psd(pb.R[(size_t)c * pb.N + i], h2, f) : 0.0;
    }
    int nsp = n_splines(pb);
    for (int a = 0; a < nsp; ++a) bm.pert[a] = eval_spline(sps[a], x);
}

// Eq. (splines): S_c = S_n,c 10^{P_n,c} + S_h,c 10^{P_h}.
double total_psd(const Problem& pb, const BinModel& bm, int c) {
    double s = bm.sn[c] * std::pow(10.0, bm.pert[c]);
    if (pb.sgwb_model) s += bm.sh[c] * std::pow(10.0, bm.pert[pb.C]);
    return s;
}

}  // namespace

extern "C" {

// Noise templates (Eq. noise_tdi) for A, E, T at n frequencies: out [3][n].
void lo_noise_templates(int tdi_form, int64_t n, const double* f, double a_oms, double a_tm,
                        double* out) {
    for (int64_t i = 0; i < n; ++i) {
        double t[3];
        noise_aet(tdi_form, f[i], a_oms * 1e-12, a_tm * 1e-15, t);
        for (int c = 0; c < 3; ++c) out[(size_t)c * n + i] = t[c];
    }
}

// Single-link-level PSDs (Sec. II.B): out [2][n] = S_OMS, S_TM.
void lo_link_psds(int64_t n, const double* f, double a_oms, double a_tm, double* out) {
    for (int64_t i = 0; i < n; ++i) {
        out[i] = S_oms(f[i], a_oms * 1e-12);
        out[n + i] = S_tm(f[i], a_tm * 1e-15);
    }
}

// SGWB template (Eq. pl, Eq. Sh) for one response row: out[n].
void lo_sgwb_template(int sgwb_model, int64_t n, const double* f, const double* R, double log10A,
                      double n1, double n2, double f_ref, double* out) {
    for (int64_t i = 0; i < n; ++i)
        out[i] = sgwb_psd(R[i], h2omega(sgwb_model, f[i], log10A, n1, n2, f_ref), f[i]);
}

// Builds one spline and returns its sorted knots xs[k+2], ys[k+2] and coefficients
// coef[(k+1)][4] = (a, b, c, d) per interval.  Returns the status bits.
int lo_spline_coeffs(int kind, int k, int kmax, const double* kx, const double* kw, double x_lo,
                     double x_hi, double* xs, double* ys, double* coef) {
    Spline<double> sp;
    int st = build_spline<double>(kind, k, kmax, kx, kw, x_lo, x_hi, sp);
    if (st) return st;
    for (int i = 1; i <= sp.n; ++i) {
        xs[i - 1] = sp.x[i];
        ys[i - 1] = sp.y[i];
    }
    for (int i = 1; i <= sp.n - 1; ++i) {
        coef[4 * (i - 1) + 0] = sp.a[i];
        coef[4 * (i - 1) + 1] = sp.b[i];
        coef[4 * (i - 1) + 2] = sp.c[i];
        coef[4 * (i - 1) + 3] = sp.d[i];
    }
    return 0;
}

// Evaluates one spline at m abscissae.  Returns the status bits.
int lo_spline_eval(int kind, int k, int kmax, const double* kx, const double* kw, double x_lo,
                   double x_hi, int64_t m, const double* x, double* out) {
    Spline<double> sp;
    int st = build_spline<double>(kind, k, kmax, kx, kw, x_lo, x_hi, sp);
    if (st) return st;
    for (int64_t i = 0; i < m; ++i) out[i] = eval_spline(sp, x[i]);
    return 0;
}

// Model PSD S_c(f_i) for every state: out [S][C][N].  status [S].
void lo_model_psd(int C, int sgwb_model, int tdi_form, int64_t N, const double* f,
                  const double* R, double x_lo, double x_hi, double f_ref, int kind, int kmax,
                  int S, const double* theta, const int* count, const double* kx,
                  const double* kw, double* out, int* status) {
    Problem pb{C, sgwb_model, tdi_form, N, f, nullptr, nullptr, R, x_lo, x_hi, f_ref, kind, kmax};
    int nsp = n_splines(pb);
    for (int s = 0; s < S; ++s) {
        std::vector<Spline<double>> sps;
        int st = build_state(pb, theta + 5 * (size_t)s, count + (size_t)s * nsp,
                             kx + (size_t)s * nsp * kmax, kw + (size_t)s * nsp * (kmax + 2), sps);
        status[s] = st;
        for (int64_t i = 0; i < N; ++i) {
            for (int c = 0; c < C; ++c) {
                double v = std::numeric_limits<double>::quiet_NaN();
                if (!st) {
                    BinModel bm;
                    bin_model(pb, theta + 5 * (size_t)s, sps, i, bm);
                    v = total_psd(pb, bm, c);
                }
                out[((size_t)s * C + c) * N + i] = v;
            }
        }
    }
}

// Sec. III.C: log L = sum_i log p(Y(f_i)), log p = -tr(C^-1 Y) - nu log|C| with Y = nu P and
// C = diag(S_c) (reading R1):  log L = -sum_i nu_i sum_c (P_c,i / S_c,i + ln S_c,i).
void lo_loglike(int C, int sgwb_model, int tdi_form, int64_t N, const double* f, const double* nu,
                const double* P, const double* R, double x_lo, double x_hi, double f_ref,
                int kind, int kmax, int S, const double* theta, const int* count,
                const double* kx, const double* kw, double* logL, int* status) {
    Problem pb{C, sgwb_model, tdi_form, N, f, nu, P, R, x_lo, x_hi, f_ref, kind, kmax};
    int nsp = n_splines(pb);
    for (int s = 0; s < S; ++s) {
        const double* th = theta + 5 * (size_t)s;
        std::vector<Spline<double>> sps;
        int st = build_state(pb, th, count + (size_t)s * nsp, kx + (size_t)s * nsp * kmax,
                             kw + (size_t)s * nsp * (kmax + 2), sps);
        double sum = 0.0;
        if (!st) {
            for (int64_t i = 0; i < N; ++i) {
                BinModel bm;
                bin_model(pb, th, sps, i, bm);
                double bin = 0.0;
                for (int c = 0; c < C; ++c) {
                    double Sc = total_psd(pb, bm, c);
                    if (!(Sc > 0.0) || !std::isfinite(Sc)) st |= 32;
                    bin += P[(size_t)c * N + i] / Sc + std::log(Sc);
                }
                sum -= nu[i] * bin;
            }
            if (!std::isfinite(sum)) st |= 32;
        }
        status[s] = st;
        logL[s] = st ? -std::numeric_limits<double>::infinity() : sum;
    }
}

// Log-likelihood and its analytic gradient.  The template parameters are differentiated per
// bin by the chain rule; each knot parameter is differentiated by running the spline
// construction and evaluation in forward mode (dual numbers) with that parameter seeded.
//   d logL / d S_c,i = nu_i (P_c,i - S_c,i) / S_c,i^2
void lo_loglike_grad_scaled(int C, int sgwb_model, int tdi_form, int64_t N, const double* f,
                            const double* nu, const double* P, const double* R, double x_lo,
                            double x_hi, double f_ref, int kind, int kmax, int S,
                            const double* theta, const int* count, const double* kx,
                            const double* kw, double* logL, double* grad, double* gscale,
                            int* status);

void lo_loglike_grad(int C, int sgwb_model, int tdi_form, int64_t N, const double* f,
                     const double* nu, const double* P, const double* R, double x_lo,
                     double x_hi, double f_ref, int kind, int kmax, int S, const double* theta,
                     const int* count, const double* kx, const double* kw, double* logL,
                     double* grad, int* status) {
    lo_loglike_grad_scaled(C, sgwb_model, tdi_form, N, f, nu, P, R, x_lo, x_hi, f_ref, kind, kmax, S,
                           theta, count, kx, kw, logL, grad, nullptr, status);
}

// As lo_loglike_grad; if gscale is not NULL it also receives, per gradient component, the sum
// of the absolute values of the terms that component's sum is made of (the condition scale of
// the sum: a backward-stable evaluation errs by a small multiple of eps times it).  The terms
// are one per (bin, channel) for the template parameters and one per bin for the knot
// parameters (q_i dP(x_i)/d(knot), q_i summed over channels for the SGWB spline).
void lo_loglike_grad_scaled(int C, int sgwb_model, int tdi_form, int64_t N, const double* f,
                            const double* nu, const double* P, const double* R, double x_lo,
                            double x_hi, double f_ref, int kind, int kmax, int S,
                            const double* theta, const int* count, const double* kx,
                            const double* kw, double* logL, double* grad, double* gscale,
                            int* status) {
    Problem pb{C, sgwb_model, tdi_form, N, f, nu, P, R, x_lo, x_hi, f_ref, kind, kmax};
    int nsp = n_splines(pb);
    const int per_spline = 2 * kmax + 2;
    const int G = 5 + nsp * per_spline;
    std::vector<double> q((size_t)nsp * N);   // d logL / d P_alpha(x_i)
    std::vector<double> xs(N);
    for (int64_t i = 0; i < N; ++i) xs[i] = std::log10(f[i]);

    for (int s = 0; s < S; ++s) {
        const double* th = theta + 5 * (size_t)s;
        const int* cnt = count + (size_t)s * nsp;
        const double* skx = kx + (size_t)s * nsp * kmax;
        const double* skw = kw + (size_t)s * nsp * (kmax + 2);
        double* gs = grad + (size_t)s * G;
        for (int p = 0; p < G; ++p) gs[p] = 0.0;
        double* ga_s = gscale ? gscale + (size_t)s * G : nullptr;
        if (ga_s)
            for (int p = 0; p < G; ++p) ga_s[p] = 0.0;
        double sc_aoms = 0.0, sc_atm = 0.0, sc_lA = 0.0, sc_n1 = 0.0, sc_n2 = 0.0;
        std::vector<Spline<double>> sps;
        int st = build_state(pb, th, cnt, skx, skw, sps);
        double sum = 0.0;
        double g_aoms = 0.0, g_atm = 0.0, g_lA = 0.0, g_n1 = 0.0, g_n2 = 0.0;
        if (!st) {
            for (int64_t i = 0; i < N; ++i) {
                BinModel bm;
                bin_model(pb, th, sps, i, bm);
                double bin = 0.0, qh = 0.0;
                double lnf = std::log(f[i] / f_ref);
                // S_n,c is a_oms^2 U_oms,c + a_tm^2 U_tm,c, so d/d a = 2 a U.
                double u_o[3], u_t[3];
                noise_aet(tdi_form, f[i], 1e-12, 0.0, u_o);
                noise_aet(tdi_form, f[i], 0.0, 1e-15, u_t);
                for (int c = 0; c < C; ++c) {
                    double En = std::pow(10.0, bm.pert[c]);
                    double Eh = pb.sgwb_model ? std::pow(10.0, bm.pert[C]) : 0.0;
                    double Sc = bm.sn[c] * En + bm.sh[c] * Eh;
                    if (!(Sc > 0.0) || !std::isfinite(Sc)) st |= 32;
                    double Pc = P[(size_t)c * N + i];
                    bin += Pc / Sc + std::log(Sc);
                    // d(bin term)/dS = -nu (P - S) / S^2, applied to each dS/dparameter X as
                    // w (X / S) with w = nu (P - S) / S (the same product; S^2 itself, which
                    // overflows for S beyond 1e154, is never formed)
                    double w = nu[i] * (Pc - Sc) / Sc;
                    double rn = En / Sc;
                    g_aoms += w * 2.0 * th[0] * u_o[c] * rn;
                    g_atm += w * 2.0 * th[1] * u_t[c] * rn;
                    sc_aoms += std::fabs(w * 2.0 * th[0] * u_o[c] * rn);
                    sc_atm += std::fabs(w * 2.0 * th[1] * u_t[c] * rn);
                    q[(size_t)c * N + i] = w * kLn10 * bm.sn[c] * rn;
                    if (pb.sgwb_model) {
                        double shs = bm.sh[c] * Eh / Sc;
                        g_lA += w * kLn10 * shs;
                        sc_lA += std::fabs(w * kLn10 * shs);
                        if (pb.sgwb_model == 2 && f[i] >= f_ref) {
                            g_n2 += w * lnf * shs;
                            sc_n2 += std::fabs(w * lnf * shs);
                        } else {
                            g_n1 += w * lnf * shs;
                            sc_n1 += std::fabs(w * lnf * shs);
                        }
                        qh += w * kLn10 * shs;
                    }
                }
                if (pb.sgwb_model) q[(size_t)C * N + i] = qh;
                sum -= nu[i] * bin;
            }
            if (!std::isfinite(sum)) st |= 32;
        }
        status[s] = st;
        logL[s] = st ? -std::numeric_limits<double>::infinity() : sum;
        if (st) continue;
        gs[0] = g_aoms;
        gs[1] = g_atm;
        gs[2] = g_lA;
        gs[3] = g_n1;
        gs[4] = (pb.sgwb_model == 2) ? g_n2 : 0.0;
        if (ga_s) {
            ga_s[0] = sc_aoms;
            ga_s[1] = sc_atm;
            ga_s[2] = sc_lA;
            ga_s[3] = (pb.sgwb_model == 2) ? sc_n1 : sc_n1 + sc_n2;
            ga_s[4] = (pb.sgwb_model == 2) ? sc_n2 : 0.0;
        }

        // Knot parameters: seed one at a time and differentiate the spline value per bin.
        for (int a = 0; a < nsp; ++a) {
            int k = cnt[a];
            std::vector<Dual> dx(kmax > 0 ? kmax : 1), dw(kmax + 2);
            const double* ax = skx + (size_t)a * kmax;
            const double* aw = skw + (size_t)a * (kmax + 2);
            double* ga = gs + 5 + a * per_spline;
            // Active parameter slots: w slots 0, 1..k, kmax+1; x slots 0..k-1.
            std::vector<int> wslots;
            wslots.push_back(0);
            for (int j = 0; j < k; ++j) wslots.push_back(1 + j);
            wslots.push_back(kmax + 1);
            auto run = [&](int seed_kind, int slot, double* abs_sum) {
                for (int j = 0; j < kmax; ++j) dx[j] = Dual(ax[j], 0.0);
                for (int j = 0; j < kmax + 2; ++j) dw[j] = Dual(aw[j], 0.0);
                if (seed_kind == 0) dw[slot].d = 1.0; else dx[slot].d = 1.0;
                Spline<Dual> sp;
                build_spline<Dual>(kind, k, kmax, dx.data(), dw.data(), x_lo, x_hi, sp);
                double acc = 0.0, aacc = 0.0;
                for (int64_t i = 0; i < N; ++i) {
                    const double term = q[(size_t)a * N + i] * eval_spline(sp, xs[i]).d;
                    acc += term;
                    aacc += std::fabs(term);
                }
                *abs_sum = aacc;
                return acc;
            };
            double* gsa = ga_s ? ga_s + 5 + a * per_spline : nullptr;
            double dummy = 0.0;
            for (int slot : wslots) ga[slot] = run(0, slot, gsa ? &gsa[slot] : &dummy);
            for (int j = 0; j < k; ++j) ga[kmax + 2 + j] = run(1, j, gsa ? &gsa[kmax + 2 + j] : &dummy);
        }
    }
}

}  // extern "C"

namespace {
// Full covariance (reading R16).  Splines: 0..2 noise of A, E, T (exponents), 3 the SGWB (if the
// model has one), then z_AE, z_AT, z_ET (values).  cov layout per bin: C00, C11, C22, C01, C02, C12.
int n_splines_full(const Problem& pb) { return 3 + (pb.sgwb_model != 0 ? 1 : 0) + 3; }

// The 3x3 model covariance of one state at bin i (physical units).
void full_cov(const Problem& pb, const double* th, const std::vector<Spline<double>>& sps, int64_t i,
              double cov[6]) {
    const double f = pb.f[i];
    const double x = std::log10(f);
    double sn[3];
    noise_aet(pb.tdi_form, f, th[0] * 1e-12, th[1] * 1e-15, sn);
    const int zb = 3 + (pb.sgwb_model != 0 ? 1 : 0);   // first correlation spline
    double D[3], H[3] = {0.0, 0.0, 0.0};
    for (int c = 0; c < 3; ++c) D[c] = sn[c] * std::pow(10.0, eval_spline(sps[c], x));
    if (pb.sgwb_model) {
        const double h2 = h2omega(pb.sgwb_model, f, th[2], th[3], th[4], pb.f_ref);
        const double eh = std::pow(10.0, eval_spline(sps[3], x));
        for (int c = 0; c < 3; ++c) H[c] = sgwb_psd(pb.R[(size_t)c * pb.N + i], h2, f) * eh;
    }
    double r[3], sq[3];   // AE, AT, ET
    for (int k = 0; k < 3; ++k) {
        const double z = eval_spline(sps[zb + k], x);
        sq[k] = 1.0 / std::sqrt(1.0 + z * z);
        r[k] = z * sq[k];
    }
    // L rows (unit norm): R = L L^T
    const double L[3][3] = {{1.0, 0.0, 0.0},
                            {r[0], sq[0], 0.0},
                            {r[1], r[2] * sq[1], sq[1] * sq[2]}};
    double R[3][3];
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            double acc = 0.0;
            for (int k = 0; k < 3; ++k) acc += L[a][k] * L[b][k];
            R[a][b] = acc;
        }
    double C[3][3];
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) C[a][b] = std::sqrt(D[a]) * R[a][b] * std::sqrt(D[b]) + (a == b ? H[a] : 0.0);
    cov[0] = C[0][0];
    cov[1] = C[1][1];
    cov[2] = C[2][2];
    cov[3] = C[0][1];
    cov[4] = C[0][2];
    cov[5] = C[1][2];
}

}  // namespace

extern "C" {

// Full-covariance model for every state: out [S][6][N] (C00, C11, C22, C01, C02, C12).
void lo_model_cov_full(int sgwb_model, int tdi_form, int64_t N, const double* f, const double* R,
                       double x_lo, double x_hi, double f_ref, int kind, int kmax, int S,
                       const double* theta, const int* count, const double* kx, const double* kw,
                       double* out, int* status) {
    Problem pb{3, sgwb_model, tdi_form, N, f, nullptr, nullptr, R, x_lo, x_hi, f_ref, kind, kmax};
    const int nsp = n_splines_full(pb);
    for (int s = 0; s < S; ++s) {
        const double* th = theta + 5 * (size_t)s;
        int st = 0;
        for (int q = 0; q < 5; ++q)
            if (!std::isfinite(th[q])) st |= 16;
        std::vector<Spline<double>> sps(nsp);
        for (int a = 0; a < nsp; ++a)
            st |= build_spline<double>(kind, count[(size_t)s * nsp + a], kmax, kx + ((size_t)s * nsp + a) * kmax,
                                       kw + ((size_t)s * nsp + a) * (kmax + 2), x_lo, x_hi, sps[a]);
        status[s] = st;
        for (int64_t i = 0; i < N; ++i) {
            double cov[6];
            if (!st) full_cov(pb, th, sps, i, cov);
            for (int e = 0; e < 6; ++e)
                out[((size_t)s * 6 + e) * N + i] = st ? std::numeric_limits<double>::quiet_NaN() : cov[e];
        }
    }
}

// Sec. III.C with the dense covariance: log L = sum_i [ -tr(C^-1 Y) - nu log|C| ], Y = nu P, with
// P the averaged Hermitian periodogram, given as P9 [9][N] = P_AA, P_EE, P_TT, then real and
// imaginary parts of P_AE, P_AT, P_ET (P_EA = conj(P_AE) and so on).  Evaluated through the
// diagonal scaling sigma_c = sqrt(C_cc), which changes nothing in exact arithmetic and keeps
// every intermediate of order one over the whole range of the perturbations:
//   K = C / (sigma sigma^T) (unit diagonal),  P' = P / (sigma sigma^T),
//   tr(C^-1 P) = tr(K^-1 P'),  log|C| = sum_c log C_cc + log|K|,  K^-1 = adj(K) / det(K).
// A state with a C_cc that is not finite and positive, or det(K) <= 0, is invalid (bit 32).
void lo_loglike_full(int sgwb_model, int tdi_form, int64_t N, const double* f, const double* nu,
                     const double* P9, const double* R, double x_lo, double x_hi, double f_ref,
                     int kind, int kmax, int S, const double* theta, const int* count,
                     const double* kx, const double* kw, double* logL, double* im_trace_max,
                     int* status) {
    Problem pb{3, sgwb_model, tdi_form, N, f, nu, nullptr, R, x_lo, x_hi, f_ref, kind, kmax};
    const int nsp = n_splines_full(pb);
    for (int s = 0; s < S; ++s) {
        const double* th = theta + 5 * (size_t)s;
        int st = 0;
        for (int q = 0; q < 5; ++q)
            if (!std::isfinite(th[q])) st |= 16;
        std::vector<Spline<double>> sps(nsp);
        for (int a = 0; a < nsp; ++a)
            st |= build_spline<double>(kind, count[(size_t)s * nsp + a], kmax, kx + ((size_t)s * nsp + a) * kmax,
                                       kw + ((size_t)s * nsp + a) * (kmax + 2), x_lo, x_hi, sps[a]);
        double sum = 0.0, imax = 0.0;
        if (!st) {
            for (int64_t i = 0; i < N; ++i) {
                double cv[6];
                full_cov(pb, th, sps, i, cv);
                const double C[3][3] = {{cv[0], cv[3], cv[4]}, {cv[3], cv[1], cv[5]}, {cv[4], cv[5], cv[2]}};
                double sg[3];
                bool good = true;
                for (int c = 0; c < 3; ++c) {
                    good = good && C[c][c] > 0.0 && std::isfinite(C[c][c]);
                    sg[c] = std::sqrt(C[c][c]);
                }
                if (!good) {
                    st |= 32;
                    break;
                }
                double K[3][3];
                for (int a = 0; a < 3; ++a)
                    for (int b = 0; b < 3; ++b) K[a][b] = C[a][b] / (sg[a] * sg[b]);
                // adjugate (cofactor transpose) and determinant of K
                double A[3][3];
                for (int a = 0; a < 3; ++a)
                    for (int b = 0; b < 3; ++b) {
                        const int a1 = (b + 1) % 3, a2 = (b + 2) % 3, b1 = (a + 1) % 3, b2 = (a + 2) % 3;
                        A[a][b] = K[a1][b1] * K[a2][b2] - K[a1][b2] * K[a2][b1];
                    }
                const double det = K[0][0] * A[0][0] + K[0][1] * A[1][0] + K[0][2] * A[2][0];
                if (!(det > 0.0) || !std::isfinite(det)) {
                    st |= 32;
                    break;
                }
                std::complex<double> Pm[3][3];
                for (int c = 0; c < 3; ++c) Pm[c][c] = std::complex<double>(P9[(size_t)c * N + i], 0.0);
                const int pr[3][2] = {{0, 1}, {0, 2}, {1, 2}};
                for (int k = 0; k < 3; ++k) {
                    const std::complex<double> v(P9[(size_t)(3 + 2 * k) * N + i], P9[(size_t)(4 + 2 * k) * N + i]);
                    Pm[pr[k][0]][pr[k][1]] = v;
                    Pm[pr[k][1]][pr[k][0]] = std::conj(v);
                }
                // tr(K^-1 P') = sum_ab (K^-1)_ab P'_ba
                std::complex<double> tr(0.0, 0.0);
                for (int a = 0; a < 3; ++a)
                    for (int b = 0; b < 3; ++b) tr += (A[a][b] / det) * (Pm[b][a] / (sg[b] * sg[a]));
                imax = std::max(imax, std::fabs(tr.imag()) / std::max(std::fabs(tr.real()), 1e-300));
                const double logdet = std::log(C[0][0]) + std::log(C[1][1]) + std::log(C[2][2]) + std::log(det);
                sum -= nu[i] * (tr.real() + logdet);
            }
            if (!std::isfinite(sum)) st |= 32;
        }
        status[s] = st;
        logL[s] = st ? -std::numeric_limits<double>::infinity() : sum;
        if (im_trace_max) im_trace_max[s] = imax;
    }
}

}  // extern "C"
