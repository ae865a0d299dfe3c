// Host-side plan construction: parameters, PSWF window, residual-function fits, Chebyshev
// and plane-wave tables, difference-kernel and root Fourier symbols.  Everything here runs
// once per dmk_plan; nothing runs per evaluation.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <sstream>

#include "dmk_internal.h"

namespace dmk {
namespace {

using cd = std::complex<double>;
constexpr double kPi = 3.14159265358979323846;

// ---- parameter rows (Sec. 6.1, Table 1 Laplace and Table 5 Stokes kernels) -------------
// Band limits as printed, except the rotlet 1e-3 row where only c = 2 pi reproduces the
// printed N_per = 3.
struct Row { double c; int p; };
const Row kRows[4][4] = {
    {{7.00, 12}, {14.50, 20}, {21.50, 30}, {29.00, 38}},      // Laplace
    {{10.47, 13}, {17.80, 23}, {25.13, 34}, {32.46, 44}},     // Stokeslet
    {{10.47, 12}, {17.80, 23}, {25.13, 33}, {33.51, 45}},     // stresslet
    {{2 * kPi, 8}, {13.61, 18}, {20.94, 29}, {28.27, 39}},    // rotlet
};
const double kTolRows[4] = {1e-3, 1e-6, 1e-9, 1e-12};

// ---- Legendre series ----------------------------------------------------------------------
double legendre_series(const std::vector<double>& a, double x) {
    // Clenshaw for sum a_n P_n(x): b_k = a_k + alpha_k(x) b_{k+1} + beta_{k+1} b_{k+2},
    // with P_{n+1} = ((2n+1) x P_n - n P_{n-1})/(n+1).
    double b1 = 0, b2 = 0;
    for (int k = (int)a.size() - 1; k >= 0; --k) {
        double alpha = (2.0 * k + 1.0) / (k + 1.0) * x;
        double beta = -(k + 1.0) / (k + 2.0);
        double b0 = a[k] + alpha * b1 + beta * b2;
        b2 = b1;
        b1 = b0;
    }
    return b1;
}

// derivative of a Legendre series: d/dx sum a_n P_n = sum b_n P_n, b_n = (2n+1) sum_{k>n, k-n odd} a_k
std::vector<double> legendre_deriv(const std::vector<double>& a) {
    int n = (int)a.size();
    std::vector<double> b(std::max(n - 1, 1), 0.0);
    for (int m = 0; m < n - 1; ++m) {
        double s = 0;
        for (int k = m + 1; k < n; k += 2) s += a[k];
        b[m] = (2.0 * m + 1.0) * s;
    }
    return b;
}

// antiderivative vanishing at 0: int_0^x P_n = (P_{n+1} - P_{n-1})(x)/(2n+1) - same at 0
std::vector<double> legendre_integral(const std::vector<double>& a) {
    int n = (int)a.size();
    std::vector<double> b(n + 1, 0.0);
    for (int k = 0; k < n; ++k) {
        if (k == 0) {
            b[1] += a[0];
        } else {
            b[k + 1] += a[k] / (2.0 * k + 1.0);
            b[k - 1] -= a[k] / (2.0 * k + 1.0);
        }
    }
    double at0 = legendre_series(b, 0.0);
    b[0] -= at0;
    return b;
}

// ---- PSWF psi_0^c (Sec. 2.2, Eq. PSWFeig; Remark PSWF_eval) ---------------------------------
// The prolate operator -(d/dx)(1-x^2)(d/dx) + c^2 x^2 commutes with the band-limited Fourier
// transform; psi_0^c is its eigenfunction with the smallest eigenvalue.  In the normalised
// Legendre basis on even degrees it is symmetric tridiagonal.  The smallest eigenvalue is
// bracketed by Sturm-sequence bisection and the eigenvector found by inverse iteration.
struct Pswf {
    double c;
    std::vector<double> a;      // standard Legendre coefficients of psi (all degrees)
    std::vector<double> da, d2a, ia;
    double psi0, psi_int;
};

int sturm_count(const std::vector<double>& d, const std::vector<double>& e, double x) {
    // number of eigenvalues < x of the tridiagonal (d, e)
    int cnt = 0;
    double q = d[0] - x;
    if (q < 0) ++cnt;
    for (size_t i = 1; i < d.size(); ++i) {
        double qq = (q == 0.0) ? 1e-300 : q;
        q = d[i] - x - e[i - 1] * e[i - 1] / qq;
        if (q < 0) ++cnt;
    }
    return cnt;
}

Pswf make_pswf(double c) {
    int n_even = (int)std::ceil(c) + 40;
    std::vector<double> d(n_even), e(n_even - 1);
    double c2 = c * c;
    for (int i = 0; i < n_even; ++i) {
        double n = 2.0 * i;
        d[i] = n * (n + 1) + c2 * (2 * n * n + 2 * n - 1) / ((2 * n - 1) * (2 * n + 3));
        if (i + 1 < n_even)
            e[i] = c2 * (n + 1) * (n + 2) / ((2 * n + 3) * std::sqrt((2 * n + 1) * (2 * n + 5)));
    }
    // Gershgorin bounds, then bisection for the smallest eigenvalue
    double lo = 1e300, hi = -1e300;
    for (int i = 0; i < n_even; ++i) {
        double r = (i > 0 ? std::fabs(e[i - 1]) : 0) + (i + 1 < n_even ? std::fabs(e[i]) : 0);
        lo = std::min(lo, d[i] - r);
        hi = std::max(hi, d[i] + r);
    }
    for (int it = 0; it < 200; ++it) {
        double mid = 0.5 * (lo + hi);
        if (sturm_count(d, e, mid) >= 1) hi = mid; else lo = mid;
    }
    double lam = 0.5 * (lo + hi);
    // inverse iteration with (A - (lam - delta) I)
    double shift = lam - 1e-10 * std::max(1.0, std::fabs(lam));
    std::vector<double> v(n_even, 1.0), w(n_even), cp(n_even), dp(n_even);
    for (int it = 0; it < 8; ++it) {
        // Thomas algorithm for the tridiagonal solve
        double b0 = d[0] - shift;
        cp[0] = (n_even > 1 ? e[0] : 0) / b0;
        dp[0] = v[0] / b0;
        for (int i = 1; i < n_even; ++i) {
            double bi = d[i] - shift - e[i - 1] * cp[i - 1];
            cp[i] = (i + 1 < n_even ? e[i] : 0) / bi;
            dp[i] = (v[i] - e[i - 1] * dp[i - 1]) / bi;
        }
        w[n_even - 1] = dp[n_even - 1];
        for (int i = n_even - 2; i >= 0; --i) w[i] = dp[i] - cp[i] * w[i + 1];
        double nrm = 0;
        for (double x : w) nrm += x * x;
        nrm = std::sqrt(nrm);
        for (int i = 0; i < n_even; ++i) v[i] = w[i] / nrm;
    }
    Pswf P;
    P.c = c;
    P.a.assign(2 * n_even, 0.0);
    for (int i = 0; i < n_even; ++i) P.a[2 * i] = v[i] * std::sqrt(2.0 * i + 0.5);
    if (legendre_series(P.a, 0.0) < 0)
        for (double& x : P.a) x = -x;
    P.da = legendre_deriv(P.a);
    P.d2a = legendre_deriv(P.da);
    P.ia = legendre_integral(P.a);
    P.psi0 = legendre_series(P.a, 0.0);
    P.psi_int = 2.0 * P.a[0];
    return P;
}

// window functions (Eqs. wfunc_pswf, def_erfc_like_fcn, wfunchat, gammaB_in_phi)
struct Window {
    Pswf P;
    double phi(double x) const { return legendre_series(P.a, x) / P.psi_int; }
    double dphi(double x) const { return legendre_series(P.da, x) / P.psi_int; }
    double int_phi(double x) const { return legendre_series(P.ia, x) / P.psi_int; }
    double phihat(double k) const {
        if (std::fabs(k) > P.c) return 0.0;
        return legendre_series(P.a, k / P.c) / P.psi0;
    }
    double dphihat(double k) const {
        if (std::fabs(k) > P.c) return 0.0;
        return legendre_series(P.da, k / P.c) / (P.c * P.psi0);
    }
    double gammaB(double k) const { return phihat(k) - 0.5 * k * dphihat(k); }
    double d2phihat0() const { return legendre_series(P.d2a, 0.0) / (P.c * P.c * P.psi0); }
    double psi_value(double x) const { return legendre_series(P.a, x); }
    double d2phi0() const { return legendre_series(P.d2a, 0.0) / P.psi_int; }
};

// ---- Chebyshev fits on s in [0,1] -----------------------------------------------------------
template <class F>
std::vector<double> cheb_fit(F f, double rel_tol) {
    const int n = 128;
    std::vector<double> vals(n), coef(n, 0.0);
    for (int k = 0; k < n; ++k) {
        double t = std::cos(kPi * (k + 0.5) / n);
        vals[k] = f(0.5 * (t + 1.0));
    }
    double mx = 0;
    for (int j = 0; j < n; ++j) {
        double s = 0;
        for (int k = 0; k < n; ++k) s += vals[k] * std::cos(kPi * j * (k + 0.5) / n);
        coef[j] = (j == 0 ? 1.0 : 2.0) * s / n;
        mx = std::max(mx, std::fabs(coef[j]));
    }
    int deg = n - 1;
    while (deg > 0 && std::fabs(coef[deg]) < rel_tol * mx) --deg;
    coef.resize(deg + 1);
    return coef;
}

// d/ds of a Chebyshev series in t = 2s - 1
std::vector<double> cheb_deriv_s(const std::vector<double>& a) {
    int n = (int)a.size();
    if (n <= 1) return {0.0};
    std::vector<double> b(n + 1, 0.0);
    for (int k = n - 1; k >= 1; --k) b[k - 1] = b[k + 1] + 2.0 * k * a[k];
    b[0] *= 0.5;
    b.resize(n - 1);
    for (double& x : b) x *= 2.0;   // dt/ds = 2
    return b;
}

// ---- kernel operator symbols (App. B, Eqs. diffop-rel-fourier-S/T/R) -----------------------
// out[j * drho + a], complex
void op_symbol(int kernel, const double k[3], cd* out) {
    const cd I(0, 1);
    double k2 = k[0] * k[0] + k[1] * k[1] + k[2] * k[2];
    if (kernel == DMK_LAPLACE) {
        out[0] = 1.0;
    } else if (kernel == DMK_STOKESLET) {
        for (int j = 0; j < 3; ++j)
            for (int l = 0; l < 3; ++l) out[j * 3 + l] = (j == l ? k2 : 0.0) - k[j] * k[l];
    } else if (kernel == DMK_STRESSLET) {
        for (int j = 0; j < 3; ++j)
            for (int l = 0; l < 3; ++l)
                for (int m = 0; m < 3; ++m) {
                    double t = ((j == l ? k[m] : 0.0) + (m == j ? k[l] : 0.0) + (l == m ? k[j] : 0.0)) * k2
                               - 2.0 * k[j] * k[l] * k[m];
                    out[j * 9 + l * 3 + m] = I * t;
                }
    } else {   // rotlet: -1/2 i eps_jlm k_m
        for (int j = 0; j < 3; ++j)
            for (int l = 0; l < 3; ++l) {
                int m = 3 - j - l;
                double eps = 0;
                if (j != l && m >= 0 && m < 3 && m != j && m != l)
                    eps = ((j + 1) % 3 == l) ? 1.0 : -1.0;
                out[j * 3 + l] = (eps == 0) ? cd(0) : -0.5 * I * eps * k[m];
            }
    }
}

// ---- truncated Green's-function symbols (Sec. 5.2 and App. C) -------------------------------
double H1t(double a, double k, double R) {       // Eq. GreenR1D_Fourier
    k = std::fabs(k);
    if (a > 0) {
        double e = std::exp(-a * R);
        return (1 - e * std::cos(k * R) + k * e * std::sin(k * R) / a) / (a * a + k * k);
    }
    if (k > 0) return (1 - R * k * std::sin(k * R) - std::cos(k * R)) / (k * k);
    return -R * R / 2;
}
double H2t(double a, double k, double R) {       // Eq. GreenR2D_Fourier
    if (a > 0)
        return (1 + k * R * std::cyl_bessel_j(1.0, k * R) * std::cyl_bessel_k(0.0, a * R)
                - a * R * std::cyl_bessel_j(0.0, k * R) * std::cyl_bessel_k(1.0, a * R)) / (a * a + k * k);
    if (k > 0) return (1 - std::cyl_bessel_j(0.0, R * k)) / (k * k);
    return R * R / 4;
}
double B1t(double a, double k, double R) {       // Eq. BGreenR1D_Fourier
    k = std::fabs(k);
    if (a > 0) {
        double e = std::exp(-a * R), s2 = a * a + k * k;
        return (2 * a * a * a + k * e * (a * R * s2 + 3 * a * a + k * k) * std::sin(k * R)
                - a * a * e * (R * s2 + 2 * a) * std::cos(k * R)) / (2 * a * a * a * s2 * s2);
    }
    if (k > 0) return (1 - std::cos(k * R) - k * R * std::sin(k * R) / 2) / (k * k * k * k);
    return R * R * R * R / 24;
}
double B2t(double a, double k, double R) {       // Eq. BGreenR2D_Fourier
    if (a > 0) {
        double s2 = a * a + k * k;
        double K0 = std::cyl_bessel_k(0.0, a * R), K1 = std::cyl_bessel_k(1.0, a * R);
        double J0 = std::cyl_bessel_j(0.0, k * R), J1 = std::cyl_bessel_j(1.0, k * R);
        return (1 - R * J0 * (R * s2 * K0 + 2 * a * K1) / 2 + k * R * J1 * (R * s2 * K1 / (2 * a) + K0)) / (s2 * s2);
    }
    if (k > 0)
        return (1 - std::cyl_bessel_j(0.0, k * R) - k * R * std::cyl_bessel_j(1.0, k * R) / 2) / (k * k * k * k);
    return R * R * R * R / 64;
}
cd Z1t(double k3, double R) {                     // Eq. ZGreenR1D_Fourier (odd; signed kappa)
    if (k3 == 0) return 0.0;
    return cd(0, -(1 - std::cos(k3 * R)) / (2 * k3));
}
// free space (D = 0): 1/(4 pi r) truncated at R, (1 - cos kR)/k^2 (radial transform of App. A)
double H3t(double k, double R) {
    if (k > 0) return (1 - std::cos(k * R)) / (k * k);
    return R * R / 2;
}
// free space biharmonic in the C^1 gauge -r/(8pi) + R/(16pi) + r^2/(16 pi R) on r <= R
double B3t(double k, double R) {
    if (k > 0) {
        double kR = k * R, s = std::sin(kR), c = std::cos(kR);
        double I1 = (s - kR * c) / (k * k);
        double I2 = (2 * kR * s + (2 - kR * kR) * c - 2) / (k * k * k);
        double I3 = (3 * (kR * kR - 2) * s - kR * (kR * kR - 6) * c) / (k * k * k * k);
        return 4 * kPi / k * (-I2 / (8 * kPi) + R * I1 / (16 * kPi) + I3 / (16 * kPi * R));
    }
    return 4 * R * R * R * R * (-1.0 / 32 + 1.0 / 48 + 1.0 / 80);
}

int ceil_guard(double x) { return (int)std::ceil(x * (1.0 - 1e-12)); }

// N of the free node set n = -N..N (Eqs. k1set-1p, k1k2set-2p: (N-1) h <= K <= N h): the
// smallest N with N h > K, i.e. ceil(K/h) and one more where K/h is an integer (relative 1e-12)
int free_count(double K, double h) { return (int)std::floor(K / h * (1.0 + 1e-12)) + 1; }

// Length Q of the cube-index DFT along axis a of one root part, 0 if there is none: 1 on an
// axis of one cube or a lone k = 0; M_a on an exactly tiled periodic axis (k = 2 pi n / L_a,
// Sec. 3.4); on a free axis of step h, Q = 2 pi / (h s) when that is an integer >= M_a, the
// oversampled length of Sec. 5.4 (Eq. kappaqdef with q M = Q).
int dft_length(const std::vector<double>& ax, int Ma, bool periodic_axis, double s) {
    if (Ma == 1 || (ax.size() == 1 && ax[0] == 0.0)) return 1;
    long long Q = Ma;
    if (!periodic_axis) {
        if (ax.size() < 2) return 0;
        const double h = (ax.back() - ax.front()) / (double)(ax.size() - 1);
        const double Qf = 2 * kPi / (h * s);
        Q = std::llround(Qf);
        if (std::fabs(Qf - (double)Q) > 1e-9 * Qf || Q < Ma || Q > 65536) return 0;
    }
    // every wavenumber is 2 pi n / (Q s) with consecutive integers n: the evaluation reaches the
    // modes of one residue n mod Q by stepping Q indices along the axis
    double prev = 0;
    for (size_t i = 0; i < ax.size(); ++i) {
        const double n = ax[i] * (double)Q * s / (2 * kPi), nr = std::nearbyint(n);
        if (std::fabs(n - nr) > 1e-6 || (i > 0 && nr != prev + 1)) return 0;
        prev = nr;
    }
    return (int)Q;
}

// App. E (Eqs. app_m1_error_estimate, app_m2_error_estimate): the pole estimate of the error of
// the infinite trapezoidal rule with step h for the model integral I_m(alpha, b), |b| = s;
// cosh(alpha s)/E and sinh(alpha s)/E (E = e^x - 1, x = 2 pi alpha / h) formed as exponentials of
// differences.  C_gamma = 0 (the biharmonic screening; m = 1 does not use it).
double free_error_estimate(int m, double alpha, double s, double h) {
    const double x = 2 * kPi * alpha / h;
    const double den = -std::expm1(-x);
    const double ch = 0.5 * (std::exp(alpha * s - x) + std::exp(-alpha * s - x)) / den;
    if (m == 1) return 2 * kPi / alpha * ch;
    const double sh = 0.5 * (std::exp(alpha * s - x) - std::exp(-alpha * s - x)) / den;
    const double einv = std::exp(-x) / den;
    return kPi / (alpha * alpha * alpha) * std::fabs(ch - alpha * s * sh + x * ch * (1 + einv));
}

}  // namespace

dmk_status_t build_plan_tables(int kernel, int D, const double Lin[3], double tol, PlanTables& T,
                               std::string& err) {
    if (kernel < 0 || kernel > 3) { err = "kernel must be 0..3"; return DMK_ERR_INVALID_ARG; }
    if (D < 0 || D > 3) { err = "D must be 0..3"; return DMK_ERR_INVALID_ARG; }
    for (int i = 0; i < 3; ++i)
        if (!(Lin[i] > 0) || !std::isfinite(Lin[i])) { err = "lengths must be positive and finite"; return DMK_ERR_INVALID_ARG; }
    if (!(tol >= 1e-12 * (1 - 1e-9) && tol <= 1e-3 * (1 + 1e-9))) { err = "tol must lie in [1e-12, 1e-3]"; return DMK_ERR_INVALID_ARG; }
    int row = 3;
    for (int i = 0; i < 4; ++i)
        if (tol >= kTolRows[i] * (1 - 1e-9)) { row = i; break; }
    T.kernel = kernel;
    T.D = D;
    const int drho[4] = {1, 3, 9, 3}, du[4] = {1, 3, 3, 3};
    T.d_rho = drho[kernel];
    T.d_u = du[kernel];
    for (int i = 0; i < 3; ++i) T.L[i] = Lin[i];
    // cube tiling (Sec. 4.1.1; Sec. 5 for the free directions; D = 0 a single cube)
    double s = 0;
    if (D > 0) { s = Lin[0]; for (int i = 1; i < D; ++i) s = std::min(s, Lin[i]); }
    else s = std::max(Lin[0], std::max(Lin[1], Lin[2]));
    T.s = s;
    // A periodic axis that s does not divide is tiled by ceil(L_i / s) cubes (the last one cut)
    // plus one padding cube on each side; the forest does not wrap along it, and the images of
    // the sources inside Omega_ext are added as sources (Sec. 4.1.1, 4.1.2).
    double Lext[3];
    for (int i = 0; i < 3; ++i) {
        double ratio = Lin[i] / s;
        T.wrap[i] = i < D;
        T.padded[i] = 0;
        T.origin[i] = 0.0;
        if (i < D) {
            int m = (int)std::llround(ratio);
            if (std::fabs(ratio - m) <= 1e-12 * std::max(1.0, ratio)) {
                T.M[i] = m;
                Lext[i] = Lin[i];
                T.periodic[i] = 1;
            } else {
                T.M[i] = ceil_guard(ratio) + 2;
                Lext[i] = T.M[i] * s;
                T.periodic[i] = 0;
                T.padded[i] = 1;
                T.origin[i] = -s;
            }
        } else {
            T.M[i] = std::max(1, ceil_guard(ratio));
            Lext[i] = T.M[i] * s;
            T.periodic[i] = 0;
        }
    }
    long long mtot = (long long)T.M[0] * T.M[1] * T.M[2];
    if (mtot > 1024) { err = "more than 1024 cubes in the tiling"; return DMK_ERR_UNSUPPORTED; }
    // cubes inside Omega, cut by its boundary, or outside it (padding), along the padded axes
    T.cube_class.assign((size_t)mtot, 0);
    for (int m2 = 0; m2 < T.M[2]; ++m2)
        for (int m1 = 0; m1 < T.M[1]; ++m1)
            for (int m0 = 0; m0 < T.M[0]; ++m0) {
                const int mi[3] = {m0, m1, m2};
                bool inside = true, outside = false;
                for (int i = 0; i < 3; ++i) {
                    if (!T.padded[i]) continue;
                    const double lo = T.origin[i] + mi[i] * s;
                    if (lo >= Lin[i] || lo + s <= 0.0) outside = true;
                    if (lo < 0.0 || lo + s > Lin[i]) inside = false;
                }
                T.cube_class[(size_t)(m2 * T.M[1] + m1) * T.M[0] + m0] = outside ? 2 : (inside ? 0 : 1);
            }
    T.c = kRows[kernel][row].c;
    T.p = kRows[kernel][row].p;
    T.nf = ceil_guard(3.0 * T.c / kPi) - 1;        // Sec. 6.1
    T.NF = 2 * T.nf + 1;
    T.nfh = T.nf + 1;
    const int ord[4] = {0, 2, 3, 1}, pw[4] = {2, 4, 4, 2};
    T.level_power = 3 + ord[kernel] - pw[kernel];
    const bool bih = (kernel == DMK_STOKESLET || kernel == DMK_STRESSLET);

    Window W{make_pswf(T.c)};
    T.phihat_samples.clear();
    for (int j = 0; j <= 10; ++j) T.phihat_samples.push_back(W.phihat(0.099 * j * T.c));
    T.phi0 = W.phi(0.0);
    T.d2phi0 = W.d2phi0();
    T.d2phihat0 = W.d2phihat0();

    // ---- Chebyshev tables (Sec. 3.1.2; first-kind points) --------------------------------
    const int p = T.p;
    T.nodes.resize(p);
    T.bary.resize(p);
    for (int j = 0; j < p; ++j) {
        T.nodes[j] = std::cos((2.0 * j + 1.0) * kPi / (2.0 * p));
        T.bary[j] = ((j % 2) ? -1.0 : 1.0) * std::sin((2.0 * j + 1.0) * kPi / (2.0 * p));
    }
    auto lagrange_row = [&](double x, double* out) {
        for (int a = 0; a < p; ++a)
            if (x == T.nodes[a]) { for (int b = 0; b < p; ++b) out[b] = (a == b); return; }
        double den = 0;
        for (int a = 0; a < p; ++a) den += T.bary[a] / (x - T.nodes[a]);
        for (int a = 0; a < p; ++a) out[a] = T.bary[a] / (x - T.nodes[a]) / den;
    };
    T.Ioct.assign(2 * p * p, 0.0);
    for (int o = 0; o < 2; ++o)
        for (int j = 0; j < p; ++j) lagrange_row((2.0 * o - 1.0) / 2.0 + T.nodes[j] / 2.0, &T.Ioct[(o * p + j) * p]);
    T.Cm.assign(p * p, 0.0);
    for (int n = 0; n < p; ++n)
        for (int j = 0; j < p; ++j)
            T.Cm[n * p + j] = (n == 0 ? 1.0 : 2.0) / p * std::cos(n * (2.0 * j + 1.0) * kPi / (2.0 * p));

    T.Aoct.assign(2 * p * p, 0.0);
    for (int o = 0; o < 2; ++o)
        for (int n = 0; n < p; ++n)
            for (int a = 0; a < p; ++a) {
                double v = 0;
                for (int j = 0; j < p; ++j) v += T.Cm[n * p + j] * T.Ioct[(o * p + j) * p + a];
                T.Aoct[(o * p + n) * p + a] = v;
            }

    // ---- plane waves (Sec. 2.3 Eq. Dl_int_discr): h_l y = (pi/3) m eta at every level ----
    T.E.resize(T.NF * p);
    for (int m = -T.nf; m <= T.nf; ++m)
        for (int j = 0; j < p; ++j) {
            double ph = -kPi / 3.0 * m * T.nodes[j];
            T.E[(m + T.nf) * p + j] = cd(std::cos(ph), std::sin(ph));
        }
    // difference-kernel scalar at level 0: w_0 h_0^ord G_0(|h_0 m|), G_0(k) = (gamma(k nu_1) -
    // gamma(k nu_0))/k^pw, w_0 = h_0^3/(2 pi)^3, h_0 = 2 pi/(3 nu_0); Laplace m = 0 limit
    // phi-hat''(0)(nu_1^2 - nu_0^2)/2; Stokes kernels: operator symbol vanishes at m = 0.
    {
        double nu0 = s, nu1 = s / 2, h0 = 2 * kPi / (3 * nu0);
        double w0 = h0 * h0 * h0 / (8 * kPi * kPi * kPi);
        double hord = std::pow(h0, ord[kernel]);
        T.gdiff.assign((size_t)T.NF * T.NF * T.nfh, 0.0);
        for (int m1 = -T.nf; m1 <= T.nf; ++m1)
            for (int m2 = -T.nf; m2 <= T.nf; ++m2)
                for (int m3 = 0; m3 <= T.nf; ++m3) {
                    double mm = std::sqrt((double)(m1 * m1 + m2 * m2 + m3 * m3));
                    double k = h0 * mm, g;
                    if (mm == 0) {
                        g = (kernel == DMK_LAPLACE) ? T.d2phihat0 * (nu1 * nu1 - nu0 * nu0) / 2 : 0.0;
                    } else {
                        double a1 = bih ? W.gammaB(k * nu1) : W.phihat(k * nu1);
                        double a0 = bih ? W.gammaB(k * nu0) : W.phihat(k * nu0);
                        g = (a1 - a0) / std::pow(k, pw[kernel]);
                    }
                    T.gdiff[((m1 + T.nf) * T.NF + (m2 + T.nf)) * T.nfh + m3] = w0 * hord * g;
                }
    }

    // ---- residual functions (App. B; Remark scaling_stokes_split: "precomputed polynomial
    // approximations"): Chebyshev series in t = 2 rho^2 - 1 ------------------------------------
    {
        const double rt = 1e-14;      // below this the coefficients reach the FP64 rounding plateau
        T.fit_q = cheb_fit([&](double ss) { double r = std::sqrt(ss); return r > 0 ? W.int_phi(r) / r : T.phi0; }, rt);
        T.fit_f = cheb_fit([&](double ss) { return W.phi(std::sqrt(ss)); }, rt);
        T.fit_g = cheb_fit([&](double ss) { double r = std::sqrt(ss); return r > 0 ? W.dphi(r) / r : T.d2phi0; }, rt);
        T.fit_dq = cheb_deriv_s(T.fit_q);
        T.fit_df = cheb_deriv_s(T.fit_f);
        T.fit_dg = cheb_deriv_s(T.fit_g);
    }

    // ---- self correction (Sec. 2.4; App. B Eq. S_self, Remark scaling_stokes_split) ------------
    T.self_val.assign(T.d_u * T.d_rho, 0.0);
    T.self_grad.assign(3 * T.d_u * T.d_rho, 0.0);
    if (kernel == DMK_LAPLACE) T.self_val[0] = T.phi0 / (2 * kPi);
    if (kernel == DMK_STOKESLET) for (int j = 0; j < 3; ++j) T.self_val[j * 3 + j] = T.phi0 / (2 * kPi);
    if (kernel == DMK_ROTLET) {
        // d_i Omega_M,jl(0) = -phi''(0) eps_jli/(12 pi nu^3)
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j)
                for (int l = 0; l < 3; ++l) {
                    double eps = 0;
                    if (i != j && j != l && i != l) eps = ((j + 1) % 3 == l) ? 1.0 : -1.0;
                    T.self_grad[(i * 3 + j) * 3 + l] = -T.d2phi0 * eps / (12 * kPi);
                }
    }
    if (kernel == DMK_STRESSLET) {
        // d_i T_M,jlm(0) = phi''(0)(d_jl d_mi + d_lm d_ji + d_mj d_li)/(4 pi nu^3)
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j)
                for (int l = 0; l < 3; ++l)
                    for (int m = 0; m < 3; ++m) {
                        double v = (j == l && m == i) + (l == m && j == i) + (m == j && l == i);
                        T.self_grad[(i * 3 + j) * 9 + l * 3 + m] = T.d2phi0 * v / (4 * kPi);
                    }
    }

    // ---- root far field (Sec. 4.3, 5.3; readings as in the library documentation) -------------
    {
        double nu0 = s, K = T.c / nu0, dk = 0, R = 0, C = 0;
        if (D == 2) R = Lext[2] + nu0;
        if (D == 1) R = std::sqrt((Lext[1] + nu0) * (Lext[1] + nu0) + (Lext[2] + nu0) * (Lext[2] + nu0));
        if (D == 0) R = std::sqrt((Lext[0] + nu0) * (Lext[0] + nu0) + (Lext[1] + nu0) * (Lext[1] + nu0) +
                                  (Lext[2] + nu0) * (Lext[2] + nu0));
        T.R = R;
        T.dk = 0;
        int nfree = 0;
        if (D < 3) { dk = kPi / R; nfree = free_count(K, dk); T.dk = dk; }
        for (int i = 0; i < 3; ++i) {
            T.kax[i].clear();
            if (i < D) {
                int km = ceil_guard(Lin[i] * K / (2 * kPi));
                for (int n = -km; n <= km; ++n) T.kax[i].push_back(2 * kPi * n / Lin[i]);
            } else {
                for (int n = -nfree; n <= nfree; ++n) T.kax[i].push_back(dk * n);
            }
        }
        if (D == 3) C = 1.0 / (Lin[0] * Lin[1] * Lin[2]);
        if (D == 2) C = dk / (Lin[0] * Lin[1] * 2 * kPi);
        if (D == 1) C = dk * dk / (Lin[0] * 4 * kPi * kPi);
        if (D == 0) C = dk * dk * dk / (8 * kPi * kPi * kPi);
        const int n1 = (int)T.kax[0].size(), n2 = (int)T.kax[1].size(), n3 = (int)T.kax[2].size();
        const int nm = T.d_u * T.d_rho;
        T.Wroot.assign((size_t)n1 * n2 * n3 * nm, cd(0));
        T.n_root_modes = 0;
        std::vector<cd> op(27);
        const cd I(0, 1);
        for (int i1 = 0; i1 < n1; ++i1)
            for (int i2 = 0; i2 < n2; ++i2)
                for (int i3 = 0; i3 < n3; ++i3) {
                    double k[3] = {T.kax[0][i1], T.kax[1][i2], T.kax[2][i3]};
                    double kn = std::sqrt(k[0] * k[0] + k[1] * k[1] + k[2] * k[2]);
                    if (kn * nu0 > T.c * (1 + 1e-12)) continue;
                    if (D == 3 && kn == 0) continue;
                    ++T.n_root_modes;
                    double gam = bih ? W.gammaB(kn * nu0) : W.phihat(kn * nu0);
                    cd* out = &T.Wroot[(((size_t)i1 * n2 + i2) * n3 + i3) * nm];
                    op_symbol(kernel, k, op.data());
                    if (D == 3) {
                        double base = 1.0 / std::pow(kn, bih ? 4 : 2);
                        for (int e = 0; e < nm; ++e) out[e] = op[e] * base;
                    } else if (D == 0) {
                        double base = bih ? B3t(kn, R) : H3t(kn, R);
                        for (int e = 0; e < nm; ++e) out[e] = op[e] * base;
                    } else if (D == 2) {
                        double alpha = std::sqrt(k[0] * k[0] + k[1] * k[1]);
                        if (alpha > 0) {
                            double base = bih ? B1t(alpha, k[2], R) : H1t(alpha, k[2], R);
                            for (int e = 0; e < nm; ++e) out[e] = op[e] * base;
                        } else {   // App. D zero modes, Eqs. C_stokeslet_rotlet_E_2p, C_stresslet_E_2p
                            double H = H1t(0.0, k[2], R);
                            cd Z = Z1t(k[2], R);
                            if (kernel == DMK_LAPLACE) out[0] = H;
                            if (kernel == DMK_STOKESLET) { out[0] = H; out[4] = H; }
                            if (kernel == DMK_ROTLET) { out[1] = Z; out[3] = -Z; }
                            if (kernel == DMK_STRESSLET) {
                                out[0 * 9 + 0 * 3 + 2] = -2.0 * Z; out[0 * 9 + 2 * 3 + 0] = -2.0 * Z;
                                out[1 * 9 + 1 * 3 + 2] = -2.0 * Z; out[1 * 9 + 2 * 3 + 1] = -2.0 * Z;
                                out[2 * 9 + 0] = -2.0 * Z; out[2 * 9 + 4] = -2.0 * Z; out[2 * 9 + 8] = -2.0 * Z;
                            }
                        }
                    } else {   // D == 1
                        double alpha = std::fabs(k[0]);
                        double kap = std::sqrt(k[1] * k[1] + k[2] * k[2]);
                        if (alpha > 0) {
                            double base = bih ? B2t(alpha, kap, R) : H2t(alpha, kap, R);
                            for (int e = 0; e < nm; ++e) out[e] = op[e] * base;
                        } else {   // App. D: C^H H-hat_2^{0,R} + C^B B-hat_2^{0,R}
                            double H = H2t(0.0, kap, R), B = B2t(0.0, kap, R), k2 = k[1], k3 = k[2];
                            double kq = kap * kap;
                            if (kernel == DMK_LAPLACE) out[0] = H;
                            if (kernel == DMK_STOKESLET) {
                                out[0] = H;
                                out[4] = k3 * k3 * B; out[5] = -k2 * k3 * B;
                                out[7] = -k2 * k3 * B; out[8] = k2 * k2 * B;
                            }
                            if (kernel == DMK_ROTLET) {
                                out[1] = -0.5 * I * k3 * H; out[2] = 0.5 * I * k2 * H;
                                out[3] = 0.5 * I * k3 * H; out[6] = -0.5 * I * k2 * H;
                            }
                            if (kernel == DMK_STRESSLET) {
                                auto set = [&](int j, int l, int m, cd v) { out[j * 9 + l * 3 + m] += v; };
                                set(0, 0, 1, I * k2 * H); set(0, 0, 2, I * k3 * H);
                                set(0, 1, 0, I * k2 * H); set(0, 2, 0, I * k3 * H);
                                set(1, 0, 0, I * k2 * H); set(2, 0, 0, I * k3 * H);
                                set(1, 1, 1, I * k2 * (3 * kq - 2 * k2 * k2) * B);
                                set(1, 1, 2, I * k3 * (kq - 2 * k2 * k2) * B);
                                set(1, 2, 1, I * k3 * (kq - 2 * k2 * k2) * B);
                                set(1, 2, 2, I * k2 * (kq - 2 * k3 * k3) * B);
                                set(2, 1, 1, I * k3 * (kq - 2 * k2 * k2) * B);
                                set(2, 1, 2, I * k2 * (kq - 2 * k3 * k3) * B);
                                set(2, 2, 1, I * k2 * (kq - 2 * k3 * k3) * B);
                                set(2, 2, 2, I * k3 * (3 * kq - 2 * k3 * k3) * B);
                            }
                        }
                    }
                    for (int e = 0; e < nm; ++e) out[e] *= C * gam;
                }
        // The App. E switch (Sec. 5.3): the estimate at alpha_min (Eq. alphamin), |b| = L_j and the
        // original kernel's Nyquist step pi/L_j, for each free direction (m = 1 for the harmonic
        // kernels, 2 for the biharmonic ones).  At most tol in every free direction: the original
        // symbol serves alpha != 0 on that step, the truncated rectangle is cut to its alpha = 0
        // line.
        T.original_symbol = false;
        for (int i = 0; i < 3; ++i) { T.kax2[i].clear(); }
        T.Wroot2.clear();
        if (D == 1 || D == 2) {
            const double amin = 2 * kPi / (D == 2 ? std::max(Lin[0], Lin[1]) : Lin[0]);
            double est = 0;
            for (int j = D; j < 3; ++j) est = std::max(est, free_error_estimate(bih ? 2 : 1, amin, Lext[j], kPi / Lext[j]));
            T.original_symbol = est <= tol;
        }
        if (T.original_symbol) {
            // part 1: the alpha = 0 line of the truncated rectangle (periodic axes cut to k = 0)
            const int m1 = n1 / 2, m2 = D == 2 ? n2 / 2 : 0;
            const int z1 = 1, z2 = D == 2 ? 1 : n2;
            std::vector<cd> Wz((size_t)z1 * z2 * n3 * nm);
            int nz = 0;
            for (int i2 = 0; i2 < z2; ++i2)
                for (int i3 = 0; i3 < n3; ++i3) {
                    const cd* src = &T.Wroot[(((size_t)m1 * n2 + (D == 2 ? m2 : i2)) * n3 + i3) * nm];
                    cd* dst = &Wz[((size_t)i2 * n3 + i3) * nm];
                    for (int e = 0; e < nm; ++e) dst[e] = src[e];
                    const double k[3] = {0.0, D == 2 ? 0.0 : T.kax[1][i2], T.kax[2][i3]};
                    const double kn = std::sqrt(k[1] * k[1] + k[2] * k[2]);
                    if (kn * nu0 <= T.c * (1 + 1e-12)) ++nz;
                }
            T.kax[0] = {0.0};
            if (D == 2) T.kax[1] = {0.0};
            T.Wroot.swap(Wz);
            // part 2: the original symbol D-hat(k) gamma-hat(|k| nu_0)/|k|^{2,4}, alpha != 0, on the
            // free step pi/L_j, with C^{DP} of that step
            double C2 = 0;
            std::vector<double> hs;
            for (int i = 0; i < 3; ++i) {
                if (i < D) {
                    int km = ceil_guard(Lin[i] * K / (2 * kPi));
                    for (int n = -km; n <= km; ++n) T.kax2[i].push_back(2 * kPi * n / Lin[i]);
                } else {
                    const double h = kPi / Lext[i];
                    const int nf2 = free_count(K, h);
                    for (int n = -nf2; n <= nf2; ++n) T.kax2[i].push_back(h * n);
                    hs.push_back(h);
                }
            }
            C2 = D == 2 ? hs[0] / (Lin[0] * Lin[1] * 2 * kPi) : hs[0] * hs[1] / (Lin[0] * 4 * kPi * kPi);
            const int q1 = (int)T.kax2[0].size(), q2 = (int)T.kax2[1].size(), q3 = (int)T.kax2[2].size();
            T.Wroot2.assign((size_t)q1 * q2 * q3 * nm, cd(0));
            int no = 0;
            for (int i1 = 0; i1 < q1; ++i1)
                for (int i2 = 0; i2 < q2; ++i2)
                    for (int i3 = 0; i3 < q3; ++i3) {
                        double k[3] = {T.kax2[0][i1], T.kax2[1][i2], T.kax2[2][i3]};
                        const double kn = std::sqrt(k[0] * k[0] + k[1] * k[1] + k[2] * k[2]);
                        const double alpha = D == 2 ? std::sqrt(k[0] * k[0] + k[1] * k[1]) : std::fabs(k[0]);
                        if (kn * nu0 > T.c * (1 + 1e-12) || alpha == 0) continue;
                        ++no;
                        const double gam = bih ? W.gammaB(kn * nu0) : W.phihat(kn * nu0);
                        op_symbol(kernel, k, op.data());
                        const double base = C2 * gam / std::pow(kn, bih ? 4 : 2);
                        cd* out = &T.Wroot2[(((size_t)i1 * q2 + i2) * q3 + i3) * nm];
                        for (int e = 0; e < nm; ++e) out[e] = op[e] * base;
                    }
            T.n_root_modes = nz + no;
        }
        // sums over the cubes as DFTs over the cube index (Sec. 3.4, 5.4): an exact tiling of two
        // or more cubes whose every root part admits one along every axis
        {
            bool ok = mtot >= 2 && !T.padded[0] && !T.padded[1] && !T.padded[2];
            const int nparts = T.original_symbol ? 2 : 1;
            for (int part = 0; part < nparts && ok; ++part)
                for (int a = 0; a < 3; ++a) {
                    const int Q = dft_length(part == 0 ? T.kax[a] : T.kax2[a], T.M[a], a < D, s);
                    if (Q == 0) ok = false;
                    T.root_dft_Q[part][a] = Q;
                }
            T.root_dft = ok;
            if (!ok)
                for (int part = 0; part < 2; ++part)
                    for (int a = 0; a < 3; ++a) T.root_dft_Q[part][a] = 0;
        }
        // constants added to the root grid per unit summed strength
        T.root_const.assign(nm, 0.0);
        if (kernel == DMK_STOKESLET && D == 1) {        // Remark stokeslet_const_corr
            double lr = std::log(R);
            T.root_const[0] = -(1 + lr) / (2 * kPi) / Lin[0];
            T.root_const[4] = -(lr + 0.5) / (4 * kPi) / Lin[0];
            T.root_const[8] = -(lr + 0.5) / (4 * kPi) / Lin[0];
        }
        if (kernel == DMK_STOKESLET && D == 0)          // C^1 gauge of the truncated biharmonic kernel
            for (int j = 0; j < 3; ++j) T.root_const[j * 3 + j] = 1.0 / (4 * kPi * R);
    }
    return DMK_OK;
}

}  // namespace dmk
