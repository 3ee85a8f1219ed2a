// Reference-element data: symmetric quadrature rules, the orthonormal modal
// basis and its tables, and the face-point permutations of the 6 relative
// face orientations.
//
// Quadrature (Sec. II-B evaluates every integral by Gaussian quadrature):
// fully symmetric rules with positive weights and interior points, exact to
// total degree 2p.  Each rule is the solution of its moment equations
//   sum_i w_i x_i^a y_i^b (z_i^c) = exact monomial integral
// over all monomials up to its degree, found by damped Gauss-Newton from a
// rough start inside the basin of the published orbit structure
// (triangle: Strang-Fix 3 points, Dunavant 6 and 12 points; tetrahedron:
// 4 points, Walkington's 14 points, Keast's 24 points).
//
// Basis (Eq. 10 fixes only the form Q = sum_j c_j b_j): orthonormal
// Proriol-Koornwinder-Dubiner polynomials on the unit tetrahedron.  With
// A = 1-eta-zeta, B = 1-zeta, a = 2 xi/A - 1, b = 2 eta/B - 1, c = 2 zeta - 1,
//   phi_ijk = 8 * 2^(2i+j) Pn_i^(0,0)(a) A^i Pn_j^(2i+1,0)(b) B^j Pn_k^(2i+2j+2,0)(c)
// where Pn_n^(alpha,0) is the Jacobi polynomial of unit weighted norm.  The
// modes are ordered by total degree, then i, then j.
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstring>

#include "dg_internal.h"

namespace dg {

const int kPerm3[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};

namespace {

double fact(int n) {
    double r = 1.0;
    for (int i = 2; i <= n; ++i) r *= i;
    return r;
}

// ---- orbit expansion -------------------------------------------------------------------
// An orbit is a base pattern of value indices whose distinct permutations give
// its points; e.g. S21 = values (a, 1-2a) on pattern (0,0,1) -> 3 points.
enum Orbit { S21, S111, S31, S22, S211 };
int orbit_nparam(Orbit o) { return (o == S111 || o == S211) ? 2 : 1; }

std::vector<std::vector<int>> orbit_patterns(Orbit o) {
    std::vector<int> base;
    switch (o) {
        case S21: base = {0, 0, 1}; break;
        case S111: base = {0, 1, 2}; break;
        case S31: base = {0, 0, 0, 1}; break;
        case S22: base = {0, 0, 1, 1}; break;
        case S211: base = {0, 0, 1, 2}; break;
    }
    std::vector<std::vector<int>> out;
    std::sort(base.begin(), base.end());
    do out.push_back(base);
    while (std::next_permutation(base.begin(), base.end()));
    return out;
}

template <typename T>
std::vector<T> orbit_values(Orbit o, const T* prm) {
    switch (o) {
        case S21: return {prm[0], T(1.0) - T(2.0) * prm[0]};
        case S111: return {prm[0], prm[1], T(1.0) - prm[0] - prm[1]};
        case S31: return {prm[0], T(1.0) - T(3.0) * prm[0]};
        case S22: return {prm[0], T(0.5) - prm[0]};
        default: return {prm[0], prm[1], T(1.0) - T(2.0) * prm[0] - prm[1]};
    }
}

struct RuleSpec {
    int dim, degree;
    std::vector<Orbit> orbits;
    std::vector<double> start;   // per orbit: params..., weight
};

RuleSpec rule_spec(int dim, int p) {
    RuleSpec s;
    s.dim = dim;
    if (dim == 2) {
        if (p == 1) { s.degree = 2; s.orbits = {S21}; s.start = {0.16, 0.1667}; }
        else if (p == 2) { s.degree = 4; s.orbits = {S21, S21}; s.start = {0.4459, 0.1117, 0.0916, 0.0550}; }
        else { s.degree = 6; s.orbits = {S21, S21, S111};
               s.start = {0.2493, 0.0584, 0.0631, 0.0254, 0.0531, 0.3104, 0.0414}; }
    } else {
        if (p == 1) { s.degree = 2; s.orbits = {S31}; s.start = {0.138, 0.0417}; }
        else if (p == 2) { s.degree = 5; s.orbits = {S31, S31, S22};
                           s.start = {0.0927, 0.01225, 0.3109, 0.01878, 0.0455, 0.00709}; }
        else { s.degree = 6; s.orbits = {S31, S31, S31, S211};
               s.start = {0.2146, 0.006654, 0.04067, 0.00168, 0.3223, 0.009226, 0.06366, 0.26967, 0.008036}; }
    }
    return s;
}

template <typename T>
void expand(const RuleSpec& s, const std::vector<T>& x, std::vector<std::vector<T>>& bary, std::vector<T>& w) {
    bary.clear();
    w.clear();
    size_t k = 0;
    for (Orbit o : s.orbits) {
        const int np = orbit_nparam(o);
        const std::vector<T> vals = orbit_values<T>(o, &x[k]);
        for (const auto& pat : orbit_patterns(o)) {
            std::vector<T> pt;
            for (int idx : pat) pt.push_back(vals[idx]);
            bary.push_back(pt);
            w.push_back(x[k + np]);
        }
        k += np + 1;
    }
}

template <typename T>
T ipow(T x, int n) {
    T r(1.0);
    for (int i = 0; i < n; ++i) r *= x;
    return r;
}

template <typename T>
void moment_residual(const RuleSpec& s, const std::vector<T>& x, std::vector<T>& r) {
    std::vector<std::vector<T>> bary;
    std::vector<T> w;
    expand(s, x, bary, w);
    r.clear();
    const int d = s.degree;
    if (s.dim == 2) {
        for (int a = 0; a <= d; ++a)
            for (int b = 0; a + b <= d; ++b) {
                T sum(0.0);
                for (size_t i = 0; i < w.size(); ++i) sum += w[i] * ipow(bary[i][1], a) * ipow(bary[i][2], b);
                r.push_back(sum - T(fact(a)) * T(fact(b)) / T(fact(a + b + 2)));
            }
    } else {
        for (int a = 0; a <= d; ++a)
            for (int b = 0; a + b <= d; ++b)
                for (int c = 0; a + b + c <= d; ++c) {
                    T sum(0.0);
                    for (size_t i = 0; i < w.size(); ++i)
                        sum += w[i] * ipow(bary[i][1], a) * ipow(bary[i][2], b) * ipow(bary[i][3], c);
                    r.push_back(sum - T(fact(a)) * T(fact(b)) * T(fact(c)) / T(fact(a + b + c + 3)));
                }
    }
}

double maxabs(const std::vector<double>& v) {
    double m = 0.0;
    for (double x : v) m = std::max(m, std::fabs(x));
    return m;
}

// Least-squares solution of the m x n system J d = rhs (m >= n) by Householder QR.
bool lstsq(std::vector<double> J, std::vector<double> rhs, int m, int n, std::vector<double>& d) {
    for (int c = 0; c < n; ++c) {
        double nrm = 0.0;
        for (int i = c; i < m; ++i) nrm += J[(size_t)i * n + c] * J[(size_t)i * n + c];
        nrm = std::sqrt(nrm);
        if (nrm == 0.0) return false;
        const double alpha = J[(size_t)c * n + c] > 0 ? -nrm : nrm;
        std::vector<double> v(m - c);
        for (int i = c; i < m; ++i) v[i - c] = J[(size_t)i * n + c];
        v[0] -= alpha;
        double vv = 0.0;
        for (double t : v) vv += t * t;
        if (vv == 0.0) continue;
        for (int k = c; k < n; ++k) {
            double dot = 0.0;
            for (int i = c; i < m; ++i) dot += v[i - c] * J[(size_t)i * n + k];
            const double f = 2.0 * dot / vv;
            for (int i = c; i < m; ++i) J[(size_t)i * n + k] -= f * v[i - c];
        }
        double dot = 0.0;
        for (int i = c; i < m; ++i) dot += v[i - c] * rhs[i];
        const double f = 2.0 * dot / vv;
        for (int i = c; i < m; ++i) rhs[i] -= f * v[i - c];
    }
    d.assign(n, 0.0);
    for (int c = n - 1; c >= 0; --c) {
        double s = rhs[c];
        for (int k = c + 1; k < n; ++k) s -= J[(size_t)c * n + k] * d[k];
        if (J[(size_t)c * n + c] == 0.0) return false;
        d[c] = s / J[(size_t)c * n + c];
    }
    return true;
}

// Gauss-Newton on the moment equations; the Jacobian by complex-step
// differentiation (exact to rounding), each step a QR least-squares solve.
bool solve_rule(const RuleSpec& s, std::vector<std::vector<double>>& bary, std::vector<double>& w,
                std::string& err) {
    using cd = std::complex<double>;
    std::vector<double> x = s.start, r;
    const int n = (int)x.size();
    moment_residual(s, x, r);
    double best = maxabs(r);
    for (int it = 0; it < 50 && best > 1e-17; ++it) {
        const int m = (int)r.size();
        std::vector<double> J((size_t)m * n), rhs(m), d;
        for (int k = 0; k < n; ++k) {
            std::vector<cd> xc(x.begin(), x.end()), rc;
            xc[k] += cd(0.0, 1e-30);
            moment_residual(s, xc, rc);
            for (int i = 0; i < m; ++i) J[(size_t)i * n + k] = rc[i].imag() / 1e-30;
        }
        for (int i = 0; i < m; ++i) rhs[i] = -r[i];
        if (!lstsq(J, rhs, m, n, d)) break;
        std::vector<double> xn(n), rn;
        for (int k = 0; k < n; ++k) xn[k] = x[k] + d[k];
        moment_residual(s, xn, rn);
        const double e = maxabs(rn);
        if (!(e < best)) break;   // converged to rounding level
        x = xn;
        r = rn;
        best = e;
    }
    // Refinement with the residual in extended precision: the moment system
    // fixes some orbit parameters only to ~1e-13 at double-precision
    // residuals; a few Gauss-Newton corrections against the extended-precision
    // residual pin the rule to double rounding.
    {
        using ld = long double;
        std::vector<ld> xl(x.begin(), x.end()), rl;
        for (int it = 0; it < 4; ++it) {
            moment_residual(s, xl, rl);
            const int m = (int)rl.size();
            std::vector<double> J((size_t)m * n), rhs(m), d;
            std::vector<cd> xc(n);
            for (int k = 0; k < n; ++k) xc[k] = cd((double)xl[k], 0.0);
            for (int k = 0; k < n; ++k) {
                std::vector<cd> xk = xc, rc;
                xk[k] += cd(0.0, 1e-30);
                moment_residual(s, xk, rc);
                for (int i = 0; i < m; ++i) J[(size_t)i * n + k] = rc[i].imag() / 1e-30;
            }
            for (int i = 0; i < m; ++i) rhs[i] = -(double)rl[i];
            if (!lstsq(J, rhs, m, n, d)) break;
            for (int k = 0; k < n; ++k) xl[k] += (ld)d[k];
        }
        for (int k = 0; k < n; ++k) x[k] = (double)xl[k];
        moment_residual(s, x, r);
        best = maxabs(r);
    }
    expand(s, x, bary, w);
    if (best > 1e-14) {
        err = "quadrature moment equations did not converge (dim " + std::to_string(s.dim) + ", degree " +
              std::to_string(s.degree) + ", residual " + std::to_string(best) + ")";
        return false;
    }
    for (size_t i = 0; i < w.size(); ++i) {
        if (!(w[i] > 0.0)) { err = "quadrature weight not positive"; return false; }
        for (double l : bary[i])
            if (!(l > 0.0)) { err = "quadrature point not interior"; return false; }
    }
    return true;
}

// ---- Jacobi polynomials ----------------------------------------------------------------
// Classical P_n^(alpha,beta)(x) by the three-term recurrence.
double jacobi(int n, double al, double be, double x) {
    if (n == 0) return 1.0;
    double p0 = 1.0, p1 = 0.5 * ((al + be + 2.0) * x + (al - be));
    for (int k = 2; k <= n; ++k) {
        double s = 2.0 * k + al + be;
        double a1 = 2.0 * k * (k + al + be) * (s - 2.0);
        double a2 = (s - 1.0) * (al * al - be * be);
        double a3 = (s - 2.0) * (s - 1.0) * s;
        double a4 = 2.0 * (k + al - 1.0) * (k + be - 1.0) * s;
        double p2 = ((a2 + a3 * x) * p1 - a4 * p0) / a1;
        p0 = p1;
        p1 = p2;
    }
    return p1;
}

// 1 / sqrt( int_{-1}^{1} (1-x)^alpha P_n^(alpha,0)(x)^2 dx ); the integral is
// 2^(alpha+1) / (2n + alpha + 1) when beta = 0.
double jacobi_inv_norm(int n, double al) {
    return std::sqrt((2.0 * n + al + 1.0) / std::pow(2.0, al + 1.0));
}

}  // namespace

void eval_basis(int p, const double xi[3], double* phi, double* grad) {
    const double x = xi[0], y = xi[1], z = xi[2];
    const double A = 1.0 - y - z, B = 1.0 - z;
    const double a = 2.0 * x / A - 1.0, b = 2.0 * y / B - 1.0, c = 2.0 * z - 1.0;
    int m = 0;
    for (int d = 0; d <= p; ++d)
        for (int i = 0; i <= d; ++i)
            for (int j = 0; i + j <= d; ++j, ++m) {
                const int k = d - i - j;
                const double al2 = 2.0 * i + 1.0, al3 = 2.0 * i + 2.0 * j + 2.0;
                const double n1 = jacobi_inv_norm(i, 0.0), n2 = jacobi_inv_norm(j, al2), n3 = jacobi_inv_norm(k, al3);
                const double P1 = n1 * jacobi(i, 0.0, 0.0, a);
                const double P2 = n2 * jacobi(j, al2, 0.0, b);
                const double P3 = n3 * jacobi(k, al3, 0.0, c);
                // derivatives of the Jacobi factors: d/dx P_n^(al,0) = (n+al+1)/2 P_{n-1}^(al+1,1)
                const double D1 = i > 0 ? n1 * 0.5 * (i + 1.0) * jacobi(i - 1, 1.0, 1.0, a) : 0.0;
                const double D2 = j > 0 ? n2 * 0.5 * (j + al2 + 1.0) * jacobi(j - 1, al2 + 1.0, 1.0, b) : 0.0;
                const double D3 = k > 0 ? n3 * 0.5 * (k + al3 + 1.0) * jacobi(k - 1, al3 + 1.0, 1.0, c) : 0.0;
                const double Ai = std::pow(A, i), Bj = std::pow(B, j);
                const double f1 = P1 * Ai, f2 = P2 * Bj, f3 = P3;
                const double scale = 8.0 * std::pow(2.0, 2 * i + j);
                phi[m] = scale * f1 * f2 * f3;
                if (grad) {
                    // f1(xi, A): d f1/d xi = 2 D1 A^(i-1); d f1/d eta = d f1/d zeta = A^(i-1) (D1 (1+a) - i P1)
                    const double Aim1 = i > 0 ? std::pow(A, i - 1) : 0.0;
                    const double Bjm1 = j > 0 ? std::pow(B, j - 1) : 0.0;
                    const double g1x = 2.0 * D1 * Aim1;
                    const double g1yz = (D1 * (1.0 + a) - i * P1) * Aim1;
                    const double g2y = 2.0 * D2 * Bjm1;
                    const double g2z = (D2 * (1.0 + b) - j * P2) * Bjm1;
                    const double g3z = 2.0 * D3;
                    grad[3 * m + 0] = scale * g1x * f2 * f3;
                    grad[3 * m + 1] = scale * (g1yz * f2 + f1 * g2y) * f3;
                    grad[3 * m + 2] = scale * ((g1yz * f2 + f1 * g2z) * f3 + f1 * f2 * g3z);
                }
            }
}

bool build_reference(int p, RefData& out, std::string& err) {
    if (p < 1 || p > 3) { err = "order must be 1, 2 or 3"; return false; }
    out.p = p;
    const TabLayout L(p);
    std::vector<std::vector<double>> vb, fb;
    std::vector<double> vw, fw;
    if (!solve_rule(rule_spec(3, p), vb, vw, err)) return false;
    if (!solve_rule(rule_spec(2, p), fb, fw, err)) return false;
    if ((int)vw.size() != L.nq || (int)fw.size() != L.nqf) { err = "unexpected rule size"; return false; }
    out.vol_xi.resize(3 * L.nq);
    out.vol_w = vw;
    for (int q = 0; q < L.nq; ++q)
        for (int d = 0; d < 3; ++d) out.vol_xi[3 * q + d] = vb[q][d + 1];
    out.face_bary.resize(3 * L.nqf);
    out.face_w = fw;
    for (int q = 0; q < L.nqf; ++q)
        for (int d = 0; d < 3; ++d) out.face_bary[3 * q + d] = fb[q][d];

    out.tab.assign(L.total, 0.0);
    std::vector<double> phi(L.nb), grad(3 * L.nb);
    for (int q = 0; q < L.nq; ++q) {
        eval_basis(p, &out.vol_xi[3 * q], phi.data(), grad.data());
        for (int j = 0; j < L.nb; ++j) {
            out.tab[L.phiq + j * L.nq + q] = phi[j];
            for (int k = 0; k < 3; ++k) out.tab[L.dphiw + (k * L.nq + q) * L.nb + j] = vw[q] * grad[3 * j + k];
        }
        out.tab[L.wq + q] = vw[q];
    }
    static const double V[4][3] = {{0, 0, 0}, {1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
    for (int f = 0; f < 4; ++f) {
        int fv[3], n = 0;
        for (int k = 0; k < 4; ++k)
            if (k != f) fv[n++] = k;
        for (int q = 0; q < L.nqf; ++q) {
            double xi[3] = {0, 0, 0};
            for (int mm = 0; mm < 3; ++mm)
                for (int d = 0; d < 3; ++d) xi[d] += out.face_bary[3 * q + mm] * V[fv[mm]][d];
            eval_basis(p, xi, phi.data(), nullptr);
            for (int j = 0; j < L.nb; ++j) {
                out.tab[L.phif + (f * L.nb + j) * L.nqf + q] = phi[j];
                out.tab[L.phifw + (f * L.nqf + q) * L.nb + j] = fw[q] * phi[j];
            }
        }
    }
    // face point permutations: orientation code c maps own point q (barycentrics
    // lambda on the own face vertices) to the neighbour point with barycentrics
    // mu_m = lambda_{perm_c(m)}
    out.fperm.assign(6 * L.nqf, -1);
    for (int c = 0; c < 6; ++c)
        for (int q = 0; q < L.nqf; ++q) {
            double mu[3];
            for (int mm = 0; mm < 3; ++mm) mu[mm] = out.face_bary[3 * q + kPerm3[c][mm]];
            for (int r = 0; r < L.nqf; ++r) {
                double dmax = 0.0;
                for (int mm = 0; mm < 3; ++mm) dmax = std::max(dmax, std::fabs(out.face_bary[3 * r + mm] - mu[mm]));
                if (dmax < 1e-12) { out.fperm[c * L.nqf + q] = (int8_t)r; break; }
            }
            if (out.fperm[c * L.nqf + q] < 0) { err = "face rule is not symmetric"; return false; }
        }
    return true;
}

}  // namespace dg
