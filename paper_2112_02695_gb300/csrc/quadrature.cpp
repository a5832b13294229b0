// Host-side quadrature rules; see quadrature.hpp.
#include "quadrature.hpp"

#include <algorithm>
#include <array>
#include <cmath>
#include <cstdint>
#include <map>
#include <mutex>

namespace boltz {

namespace {

constexpr double kPi = 3.14159265358979323846;

// Legendre P_n(x) and P_n'(x) by the three-term recurrence.
void legendre(int n, double x, double& p, double& dp) {
    double p0 = 1.0, p1 = x;
    if (n == 0) { p = 1.0; dp = 0.0; return; }
    for (int k = 2; k <= n; ++k) {
        double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
    }
    p = p1;
    dp = n * (x * p1 - p0) / (x * x - 1.0);
}

// Eigenvalues of a dense symmetric matrix by cyclic Jacobi rotations.
std::vector<double> symmetric_eigenvalues(std::vector<double> a, int n) {
    for (int sweep = 0; sweep < 100; ++sweep) {
        double off = 0.0;
        for (int i = 0; i < n; ++i)
            for (int j = i + 1; j < n; ++j) off += a[i * n + j] * a[i * n + j];
        if (off < 1e-300) break;
        for (int p = 0; p < n; ++p) {
            for (int q = p + 1; q < n; ++q) {
                double apq = a[p * n + q];
                if (std::fabs(apq) < 1e-300) continue;
                double theta = (a[q * n + q] - a[p * n + p]) / (2.0 * apq);
                double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
                double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
                for (int k = 0; k < n; ++k) {      // columns p, q
                    double akp = a[k * n + p], akq = a[k * n + q];
                    a[k * n + p] = c * akp - s * akq;
                    a[k * n + q] = s * akp + c * akq;
                }
                for (int k = 0; k < n; ++k) {      // rows p, q
                    double apk = a[p * n + k], aqk = a[q * n + k];
                    a[p * n + k] = c * apk - s * aqk;
                    a[q * n + k] = s * apk + c * aqk;
                }
            }
        }
    }
    std::vector<double> ev(n);
    for (int i = 0; i < n; ++i) ev[i] = a[i * n + i];
    std::sort(ev.begin(), ev.end());
    return ev;
}

// ---------------------------------------------------------------- sphere rules

enum Orbit { A1, A2, A3, B, C };

struct RuleSpec {
    int M;
    int degree;
    std::vector<Orbit> orbits;
};

const std::vector<RuleSpec>& rule_specs() {
    static const std::vector<RuleSpec> specs = {
        {6, 3, {A1}},
        {14, 5, {A1, A3}},
        {26, 7, {A1, A2, A3}},
        {38, 9, {A1, A3, C}},
        {50, 11, {A1, A2, A3, B}},
        {86, 15, {A1, A3, B, B, C}},
    };
    return specs;
}

void add_signed_permutations(double a, double b, double c, std::vector<std::array<double, 3>>& pts) {
    std::array<double, 3> base = {a, b, c};
    std::array<int, 3> idx = {0, 1, 2};
    std::vector<std::array<double, 3>> found;
    do {
        for (int s = 0; s < 8; ++s) {
            std::array<double, 3> v = {base[idx[0]] * ((s & 1) ? -1 : 1), base[idx[1]] * ((s & 2) ? -1 : 1),
                                       base[idx[2]] * ((s & 4) ? -1 : 1)};
            bool dup = false;
            for (auto& u : found)
                if (std::fabs(u[0] - v[0]) + std::fabs(u[1] - v[1]) + std::fabs(u[2] - v[2]) < 1e-14) {
                    dup = true;
                    break;
                }
            if (!dup) found.push_back(v);
        }
    } while (std::next_permutation(idx.begin(), idx.end()));
    pts.insert(pts.end(), found.begin(), found.end());
}

std::vector<std::array<double, 3>> orbit_points(Orbit o, double t) {
    std::vector<std::array<double, 3>> pts;
    const double r2 = 1.0 / std::sqrt(2.0), r3 = 1.0 / std::sqrt(3.0);
    switch (o) {
        case A1: add_signed_permutations(1, 0, 0, pts); break;
        case A2: add_signed_permutations(0, r2, r2, pts); break;
        case A3: add_signed_permutations(r3, r3, r3, pts); break;
        case B: add_signed_permutations(t, t, std::sqrt(std::max(0.0, 1.0 - 2.0 * t * t)), pts); break;
        case C: add_signed_permutations(t, std::sqrt(std::max(0.0, 1.0 - t * t)), 0.0, pts); break;
    }
    return pts;
}

double sphere_moment(int a, int b, int c) {
    if ((a | b | c) & 1) return 0.0;
    return 2.0 * std::tgamma((a + 1) / 2.0) * std::tgamma((b + 1) / 2.0) * std::tgamma((c + 1) / 2.0) /
           std::tgamma((a + b + c + 3) / 2.0);
}

struct MomentProblem {
    const RuleSpec* spec;
    std::vector<std::array<int, 3>> exps;   // a >= b >= c, all even, sum <= degree
    int n_orb = 0, n_par = 0;

    explicit MomentProblem(const RuleSpec& s) : spec(&s) {
        for (int a = 0; a <= s.degree; a += 2)
            for (int b = 0; b <= a; b += 2)
                for (int c = 0; c <= b; c += 2)
                    if (a + b + c <= s.degree) exps.push_back({a, b, c});
        n_orb = (int)s.orbits.size();
        for (Orbit o : s.orbits) n_par += (o == B || o == C);
    }

    // residual of unknowns u = [weights (n_orb), params (n_par)]
    void residual(const std::vector<double>& u, std::vector<double>& r) const {
        r.assign(exps.size(), 0.0);
        int ip = 0;
        for (int o = 0; o < n_orb; ++o) {
            Orbit kind = spec->orbits[o];
            double t = (kind == B || kind == C) ? u[n_orb + ip++] : 0.0;
            auto pts = orbit_points(kind, t);
            for (size_t e = 0; e < exps.size(); ++e) {
                double s = 0.0;
                for (auto& p : pts)
                    s += std::pow(p[0], exps[e][0]) * std::pow(p[1], exps[e][1]) * std::pow(p[2], exps[e][2]);
                r[e] += u[o] * s;
            }
        }
        for (size_t e = 0; e < exps.size(); ++e) r[e] -= sphere_moment(exps[e][0], exps[e][1], exps[e][2]);
    }
};

// Solve the small dense system A x = b (n <= 16) by Gaussian elimination with partial pivoting.
bool solve_dense(std::vector<double> A, std::vector<double> b, int n, std::vector<double>& x) {
    for (int c = 0; c < n; ++c) {
        int piv = c;
        for (int r = c + 1; r < n; ++r)
            if (std::fabs(A[r * n + c]) > std::fabs(A[piv * n + c])) piv = r;
        if (std::fabs(A[piv * n + c]) < 1e-300) return false;
        if (piv != c) {
            for (int k = 0; k < n; ++k) std::swap(A[c * n + k], A[piv * n + k]);
            std::swap(b[c], b[piv]);
        }
        for (int r = c + 1; r < n; ++r) {
            double f = A[r * n + c] / A[c * n + c];
            for (int k = c; k < n; ++k) A[r * n + k] -= f * A[c * n + k];
            b[r] -= f * b[c];
        }
    }
    x.assign(n, 0.0);
    for (int r = n - 1; r >= 0; --r) {
        double s = b[r];
        for (int k = r + 1; k < n; ++k) s -= A[r * n + k] * x[k];
        x[r] = s / A[r * n + r];
    }
    return true;
}

double sq_norm(const std::vector<double>& r) {
    double s = 0;
    for (double v : r) s += v * v;
    return s;
}

// Levenberg-Marquardt from one start; returns the final max |residual|.
double levenberg_marquardt(const MomentProblem& P, std::vector<double>& u) {
    const int n = P.n_orb + P.n_par;
    const int m = (int)P.exps.size();
    std::vector<double> r, rp, rm, J(m * n), JtJ(n * n), g(n), step;
    P.residual(u, r);
    double lambda = 1e-3;
    for (int it = 0; it < 300; ++it) {
        for (int k = 0; k < n; ++k) {
            const double h = (k < P.n_orb) ? 1e-6 : 1e-7;
            std::vector<double> up = u, um = u;
            up[k] += h;
            um[k] -= h;
            P.residual(up, rp);
            P.residual(um, rm);
            for (int e = 0; e < m; ++e) J[e * n + k] = (rp[e] - rm[e]) / (2 * h);
        }
        for (int a = 0; a < n; ++a) {
            g[a] = 0;
            for (int e = 0; e < m; ++e) g[a] += J[e * n + a] * r[e];
            for (int b = 0; b < n; ++b) {
                double s = 0;
                for (int e = 0; e < m; ++e) s += J[e * n + a] * J[e * n + b];
                JtJ[a * n + b] = s;
            }
        }
        bool improved = false;
        for (int tries = 0; tries < 20 && !improved; ++tries) {
            std::vector<double> A = JtJ, mg(n);
            for (int a = 0; a < n; ++a) {
                A[a * n + a] += lambda * (JtJ[a * n + a] + 1e-30);
                mg[a] = -g[a];
            }
            if (!solve_dense(A, mg, n, step)) { lambda *= 10; continue; }
            std::vector<double> trial = u;
            for (int a = 0; a < n; ++a) trial[a] += step[a];
            bool ok = true;
            for (int k = 0; k < P.n_par; ++k) {
                double t = trial[P.n_orb + k];
                if (!(t > 0.0 && t < 1.0 / std::sqrt(2.0))) ok = false;
            }
            std::vector<double> rt;
            if (ok) P.residual(trial, rt);
            if (ok && sq_norm(rt) < sq_norm(r)) {
                u = trial;
                r = rt;
                lambda = std::max(lambda * 0.1, 1e-15);
                improved = true;
            } else {
                lambda *= 10;
            }
        }
        double rmax = 0;
        for (double v : r) rmax = std::max(rmax, std::fabs(v));
        if (!improved || rmax < 1e-15) break;
    }
    double rmax = 0;
    for (double v : r) rmax = std::max(rmax, std::fabs(v));
    return rmax;
}

bool solve_sphere_rule(int M, DirectionRule& out) {
    const RuleSpec* spec = nullptr;
    for (auto& s : rule_specs())
        if (s.M == M) spec = &s;
    if (!spec) return false;
    MomentProblem P(*spec);
    const int n = P.n_orb + P.n_par;
    const double hi = 1.0 / std::sqrt(2.0);
    // deterministic starts: a lattice over the orbit parameters
    std::vector<std::vector<double>> starts;
    const int per = P.n_par == 0 ? 1 : (P.n_par == 1 ? 24 : 7);
    std::vector<int> cnt(P.n_par, 0);
    while (true) {
        std::vector<double> u(n, 4.0 * kPi / M);
        for (int k = 0; k < P.n_par; ++k) u[P.n_orb + k] = hi * (cnt[k] + 0.5) / per;
        starts.push_back(u);
        int k = 0;
        while (k < P.n_par && ++cnt[k] == per) cnt[k++] = 0;
        if (k == P.n_par) break;
    }
    for (auto u : starts) {
        double rmax = levenberg_marquardt(P, u);
        bool pos = true;
        for (int o = 0; o < P.n_orb; ++o) pos = pos && u[o] > 0;
        if (rmax < 1e-13 && pos) {
            out.sigma.clear();
            out.w.clear();
            int ip = 0;
            for (int o = 0; o < P.n_orb; ++o) {
                Orbit kind = spec->orbits[o];
                double t = (kind == B || kind == C) ? u[P.n_orb + ip++] : 0.0;
                for (auto& p : orbit_points(kind, t)) {
                    out.sigma.insert(out.sigma.end(), p.begin(), p.end());
                    out.w.push_back(u[o]);
                }
            }
            return (int)out.w.size() == M;
        }
    }
    return false;
}

bool fill_antipodes(int d, DirectionRule& rule) {
    const int M = (int)rule.w.size();
    rule.antipode.assign(M, -1);
    for (int p = 0; p < M; ++p) {
        for (int q = 0; q < M; ++q) {
            double s = 0;
            for (int a = 0; a < d; ++a) s += std::fabs(rule.sigma[p * d + a] + rule.sigma[q * d + a]);
            if (s < 1e-12) { rule.antipode[p] = q; break; }
        }
        if (rule.antipode[p] < 0) return false;
    }
    return true;
}

}  // namespace

bool gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w) {
    if (n < 1) return false;
    std::vector<double> J(n * n, 0.0);
    for (int k = 1; k < n; ++k) {
        double beta = k / std::sqrt(4.0 * k * k - 1.0);
        J[(k - 1) * n + k] = beta;
        J[k * n + (k - 1)] = beta;
    }
    x = symmetric_eigenvalues(J, n);
    w.resize(n);
    for (int i = 0; i < n; ++i) {
        double p, dp;
        for (int it = 0; it < 3; ++it) {   // Newton polish
            legendre(n, x[i], p, dp);
            x[i] -= p / dp;
        }
        legendre(n, x[i], p, dp);
        w[i] = 2.0 / ((1.0 - x[i] * x[i]) * dp * dp);
    }
    return true;
}

bool direction_rule(int d, int M, DirectionRule& out) {
    if (d == 2) {
        if (M < 2 || M % 2) return false;
        out.sigma.resize(2 * M);
        out.w.assign(M, 2.0 * kPi / M);
        for (int p = 0; p < M; ++p) {
            // exact values on the axes keep the rule exactly centrally symmetric
            double th = 2.0 * kPi * p / M;
            out.sigma[2 * p] = std::cos(th);
            out.sigma[2 * p + 1] = std::sin(th);
        }
        for (int p = 0; p < M / 2; ++p) {          // enforce sigma_{p+M/2} = -sigma_p
            out.sigma[2 * (p + M / 2)] = -out.sigma[2 * p];
            out.sigma[2 * (p + M / 2) + 1] = -out.sigma[2 * p + 1];
        }
        return fill_antipodes(d, out);
    }
    if (d == 3) {
        static std::mutex mu;
        static std::map<int, DirectionRule> cache;
        std::lock_guard<std::mutex> lock(mu);
        auto it = cache.find(M);
        if (it == cache.end()) {
            DirectionRule r;
            if (!solve_sphere_rule(M, r) || !fill_antipodes(3, r)) return false;
            it = cache.emplace(M, r).first;
        }
        out = it->second;
        return true;
    }
    return false;
}

double omega_average(int d, double s) {
    if (d == 3) return (std::fabs(s) < 1e-8) ? 4.0 * kPi * (1.0 - s * s / 6.0) : 4.0 * kPi * std::sin(s) / s;
    return 2.0 * kPi * std::cyl_bessel_j(0.0, s);
}

}  // namespace boltz
