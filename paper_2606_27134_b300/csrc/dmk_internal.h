// Internal declarations shared by the host plan code and the CUDA kernels.
#pragma once
#include <cstdint>
#include <complex>
#include <string>
#include <vector>

#include "../../include/dmk.h"

namespace dmk {

constexpr int kBits = 18;           // integer levels below a cube; also the depth cap
constexpr int kMaxLevels = kBits + 1;

// Host-side plan tables (FP64).  Layouts are documented next to each member.
struct PlanTables {
    int kernel = 0, D = 3, d_rho = 1, d_u = 1;
    double L[3] = {1, 1, 1};
    double s = 1;                   // cube side = nu_0 (Sec. 4.1.1; nu_0 reading)
    int M[3] = {1, 1, 1};           // cubes per axis (padding included)
    int periodic[3] = {1, 1, 1};    // the forest wraps along the axis (exactly tiled periodic axes)
    int wrap[3] = {1, 1, 1};        // the sum is periodic along the axis (axes 0..D-1)
    int padded[3] = {0, 0, 0};      // periodic but not exactly tiled: cut cubes + one padding cube
                                    // each side, images of the sources added (Sec. 4.1.1-4.1.2)
    double origin[3] = {0, 0, 0};   // lower corner of Omega_ext (-s on padded axes)
    std::vector<int> cube_class;    // per cube: 0 inside Omega, 1 cut, 2 outside (padding)
    double c = 0;                   // PSWF band limit
    int p = 0, nf = 0, NF = 0, nfh = 0;   // Chebyshev order, n_f, N_F = 2 n_f + 1, n_f + 1
    int level_power = 1;            // difference-kernel symbol scales as 2^(level_power * l)

    // Chebyshev first-kind nodes eta_j (j = 0..p-1), barycentric weights
    std::vector<double> nodes, bary;
    // child grid from parent grid: Ioct[o][j_child * p + a_parent], o = 0 (lower), 1 (upper)
    std::vector<double> Ioct;
    // parent grid -> Chebyshev coefficients of a child: Aoct[o][n * p + a] = sum_j Cm[n][j] Ioct[o][j][a]
    std::vector<double> Aoct;
    // grid values -> Chebyshev coefficients: Cm[n * p + j]
    std::vector<double> Cm;
    // plane waves: E[(m + nf) * p + j] = exp(-i pi/3 m eta_j), m = -nf..nf
    std::vector<std::complex<double>> E;
    // difference-kernel scalar table at level 0 on the half grid, index
    // ((m1 + nf) * NF + (m2 + nf)) * nfh + m3, m3 = 0..nf; includes w_0 h_0^ord
    std::vector<double> gdiff;
    // residual functions of s = rho^2 in [0,1] as Chebyshev series in t = 2s - 1:
    // q(s) = (int_0^rho phi)/rho, f(s) = phi(rho), g(s) = phi'(rho)/rho and their s-derivatives
    std::vector<double> fit_q, fit_f, fit_g, fit_dq, fit_df, fit_dg;
    // root: rectangle axes and weights W[((i1 * n2 + i2) * n3 + i3) * du * drho + j * drho + a]
    std::vector<double> kax[3];
    std::vector<std::complex<double>> Wroot;
    // second root part (the App. E switch, Sec. 5.3): when the original symbol serves the
    // alpha != 0 modes, kax / Wroot hold the alpha = 0 line (truncated zero-mode symbols, step
    // pi/R) and kax2 / Wroot2 the rectangle of the original symbol (step pi/L_j); else empty
    bool original_symbol = false;
    std::vector<double> kax2[3];
    std::vector<std::complex<double>> Wroot2;
    int n_root_modes = 0;           // retained modes of both parts
    // Sums over the cubes as DFTs over the cube index (Sec. 3.4 Cases 1 and 2, Sec. 5.4): on an
    // exact tiling of two or more cubes where every axis a of every root part has wavenumbers
    // k = 2 pi n / (Q_a s) for an integer Q_a >= M_a (periodic axes: Q_a = M_a; free axes: the
    // oversampled length 2 pi / (step s), e.g. 2 (M_3 + 1) for the step pi/R of D = 2), the
    // phase of cube m is exp(-2 pi i sum_a (n_a mod Q_a) m_a / Q_a) times that of cube 0.
    // root_dft_Q[part][a] = Q_a (1 on axes of one cube or a k = 0 line), all 0 if not used.
    bool root_dft = false;
    int root_dft_Q[2][3] = {{0, 0, 0}, {0, 0, 0}};
    double R = 0;                   // truncation radius (D < 3)
    std::vector<double> root_const; // d_u x d_rho constant added per unit summed strength
    // self correction at level 0 (scale 1/nu for the value, 1/nu^3 for the gradient)
    std::vector<double> self_val;   // d_u x d_rho, times nu_0
    std::vector<double> self_grad;  // 3 x d_u x d_rho, times nu_0^3
    double phi0 = 0, d2phi0 = 0, d2phihat0 = 0;
    double dk = 0;
    std::vector<double> phihat_samples;   // phi-hat(0.1 c j), j = 0..10
};

// Builds every table; returns DMK_OK or an error with a message.
dmk_status_t build_plan_tables(int kernel, int D, const double L[3], double tol, PlanTables& T,
                               std::string& err);

}  // namespace dmk
