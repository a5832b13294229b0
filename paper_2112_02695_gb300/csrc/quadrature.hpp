// Host-side (FP64) quadrature rules of the separated collision quadrature.
//
// The fast spectral solver the paper uses (Sec. 2.1) needs a radial rule on
// [0, R] and a centrally symmetric direction rule on S^{d-1}.  This file builds
// them at grid creation:
//   * Gauss-Legendre by the Golub-Welsch method: eigenvalues of the symmetric
//     Jacobi matrix of the Legendre recurrence (cyclic Jacobi rotations),
//     nodes polished by Newton steps, weights 2 / ((1 - x^2) P_n'(x)^2);
//   * circle: theta_p = 2 pi p / M;
//   * sphere: octahedrally symmetric rules (6, 14, 26, 38, 50, 86 points) whose
//     orbit weights and parameters solve the moment equations
//     sum_i w_i x^a y^b z^c = int_{S^2} x^a y^b z^c up to the design degree,
//     found by Levenberg-Marquardt from a deterministic set of starts.
#pragma once

#include <vector>

namespace boltz {

struct DirectionRule {
    std::vector<double> sigma;   // [M][d]
    std::vector<double> w;       // [M]
    std::vector<int> antipode;   // index of -sigma_p
};

// n-point Gauss-Legendre on [-1, 1], ascending.  Returns false for n < 1.
bool gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w);

// Direction rule for d = 2 (M even, >= 2) or d = 3 (M in {6,14,26,38,50,86}).
bool direction_rule(int d, int M, DirectionRule& out);

// Exact omega-average F_d(s) = int_{S^{d-1}} exp(-i s.omega) domega.
double omega_average(int d, double s);

}  // namespace boltz
