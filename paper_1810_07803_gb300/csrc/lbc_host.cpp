// Host-side set-up: Gauss rules of Sec. III, Hermite tables, the projection rule
// of the discrete equilibrium, and the stretched grid of Eq. stretch. FP64.
#include <algorithm>
#include <cmath>
#include <mutex>
#include <string>
#include <vector>

#include "lbc_internal.h"

namespace lbc {

namespace {

// Gauss-Legendre rule on [-1, 1] by Newton's method on P_m.
void gauss_legendre(int m, std::vector<double> &x, std::vector<double> &w)
{
    x.assign(m, 0.0);
    w.assign(m, 0.0);
    for (int i = 0; i < m; ++i) {
        double t = std::cos(M_PI * (i + 0.75) / (m + 0.5));
        double dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = t;
            for (int k = 1; k < m; ++k) {
                double p2 = ((2.0 * k + 1.0) * t * p1 - k * p0) / (k + 1.0);
                p0 = p1;
                p1 = p2;
            }
            dp = m * (t * p1 - p0) / (t * t - 1.0);
            double dt = p1 / dp;
            t -= dt;
            if (std::fabs(dt) < 1e-16) break;
        }
        x[i] = t;
        w[i] = 2.0 / ((1.0 - t * t) * dp * dp);
    }
}

// Number of eigenvalues of the symmetric tridiagonal matrix (a, b) below s
// (Sturm sequence of the LDL^T pivots).
int sturm_count(const std::vector<double> &a, const std::vector<double> &b, int n, double s)
{
    int count = 0;
    double d = 1.0;
    for (int i = 0; i < n; ++i) {
        double off = i ? b[i] * b[i] / d : 0.0;
        d = a[i] - s - off;
        if (d == 0.0) d = -1e-300;
        if (d < 0.0) ++count;
    }
    return count;
}

}  // namespace

// Orthonormal three-term recurrence of the half-range Hermite polynomials h_l
// (weight exp(-z^2/2)/sqrt(2 pi) on [0, inf)), for l < n:
//   z h_l = sbeta[l+1] h_{l+1} + alpha[l] h_l + sbeta[l] h_{l-1},  h_0 = 1/sbeta[0].
// Discretized Stieltjes procedure: the weight on [0, 26] is replaced by a
// composite 24-point Gauss-Legendre rule on panels of width 1/2, whose first
// moments are exact to rounding for the degrees used here; the discrete inner
// product then gives alpha, beta by Stieltjes' formulas, with the polynomial
// vectors re-orthogonalised (twice) against all previous ones. Accumulated in
// long double (extended or quad precision, host-dependent; rounded to double).
namespace {
std::mutex g_rec_mutex;
std::vector<double> g_rec_alpha, g_rec_sbeta;   // cached: the first n coefficients do not depend on n
}  // namespace

static bool half_range_recurrence_uncached(int n, std::vector<double> &alpha, std::vector<double> &sbeta);

bool half_range_recurrence(int n, std::vector<double> &alpha, std::vector<double> &sbeta)
{
    if (n < 1 || n > 2 * kMaxQ + 4) return false;
    std::lock_guard<std::mutex> lock(g_rec_mutex);
    if ((int)g_rec_alpha.size() < n) {
        int m = std::max(n, 40);
        if (!half_range_recurrence_uncached(m, g_rec_alpha, g_rec_sbeta)) return false;
    }
    alpha.assign(g_rec_alpha.begin(), g_rec_alpha.begin() + n);
    sbeta.assign(g_rec_sbeta.begin(), g_rec_sbeta.begin() + n + 1);
    return true;
}

static bool half_range_recurrence_uncached(int n, std::vector<double> &alpha, std::vector<double> &sbeta)
{
    typedef long double ld;   // extended where the host has it: set-up only
    std::vector<double> gx, gw;
    gauss_legendre(24, gx, gw);
    const ld h = 0.5L, zmax = 26.0L;
    const int panels = static_cast<int>(zmax / h);
    const int M = panels * 24;
    std::vector<ld> t(M), W(M);
    const ld inv_s2pi = 1.0L / std::sqrt(2.0L * 3.14159265358979323846264338327950288L);
    for (int p = 0; p < panels; ++p)
        for (int k = 0; k < 24; ++k) {
            ld z = p * h + 0.5L * h * ((ld)gx[k] + 1.0L);
            t[p * 24 + k] = z;
            W[p * 24 + k] = 0.5L * h * (ld)gw[k] * std::exp(-0.5L * z * z) * inv_s2pi;
        }
    alpha.assign(n, 0.0);
    sbeta.assign(n + 1, 0.0);
    std::vector<ld> sb(n + 1, 0.0L);
    std::vector<std::vector<ld>> q;
    ld mu0 = 0;
    for (int j = 0; j < M; ++j) mu0 += W[j];
    sb[0] = std::sqrt(mu0);
    q.emplace_back(M, 1.0L / sb[0]);
    std::vector<ld> v(M);
    for (int k = 0; k < n; ++k) {
        const std::vector<ld> &qk = q[k];
        for (int j = 0; j < M; ++j) v[j] = t[j] * qk[j];
        ld a = 0;
        for (int j = 0; j < M; ++j) a += W[j] * qk[j] * v[j];
        alpha[k] = (double)a;
        for (int j = 0; j < M; ++j) v[j] -= a * qk[j] + (k ? sb[k] * q[k - 1][j] : 0.0L);
        for (int pass = 0; pass < 2; ++pass)
            for (int i = 0; i <= k; ++i) {
                ld c = 0;
                for (int j = 0; j < M; ++j) c += W[j] * q[i][j] * v[j];
                for (int j = 0; j < M; ++j) v[j] -= c * q[i][j];
            }
        ld nrm = 0;
        for (int j = 0; j < M; ++j) nrm += W[j] * v[j] * v[j];
        nrm = std::sqrt(nrm);
        sb[k + 1] = nrm;
        std::vector<ld> next(M);
        for (int j = 0; j < M; ++j) next[j] = v[j] / nrm;
        q.push_back(std::move(next));
    }
    for (int k = 0; k <= n; ++k) sbeta[k] = (double)sb[k];
    return true;
}

// Q-point Gauss rule of an orthonormal recurrence (alpha[0..Q-1], sbeta[0..Q]):
// nodes by Sturm bisection on the Jacobi matrix, polished by Newton's method on
// h_Q; weights as Christoffel numbers 1 / sum_{l<Q} h_l(z_i)^2 (all terms
// positive, so even the smallest weights keep full relative accuracy).
bool gauss_from_recurrence(int Q, const std::vector<double> &alpha, const std::vector<double> &sbeta,
                           std::vector<double> &nodes, std::vector<double> &weights)
{
    if (Q < 1 || (int)alpha.size() < Q || (int)sbeta.size() < Q + 1) return false;
    double lo = 1e300, hi = -1e300;
    for (int i = 0; i < Q; ++i) {
        double r = (i ? std::fabs(sbeta[i]) : 0.0) + (i + 1 < Q ? std::fabs(sbeta[i + 1]) : 0.0);
        lo = std::min(lo, alpha[i] - r);
        hi = std::max(hi, alpha[i] + r);
    }
    nodes.assign(Q, 0.0);
    weights.assign(Q, 0.0);
    for (int k = 0; k < Q; ++k) {
        double a = lo, b = hi;
        for (int it = 0; it < 200 && b - a > 1e-15 * std::max(1.0, std::fabs(a)); ++it) {
            double m = 0.5 * (a + b);
            if (sturm_count(alpha, sbeta, Q, m) > k) b = m; else a = m;
        }
        double z = 0.5 * (a + b);
        for (int it = 0; it < 3; ++it) {   // Newton on h_Q(z) with its derivative
            double hp = 0, h = 1.0 / sbeta[0], dp = 0, d = 0;
            for (int l = 0; l < Q; ++l) {
                double hn = ((z - alpha[l]) * h - sbeta[l] * hp) / sbeta[l + 1];
                double dn = (h + (z - alpha[l]) * d - sbeta[l] * dp) / sbeta[l + 1];
                hp = h; h = hn; dp = d; d = dn;
            }
            if (d != 0.0) {
                double step = h / d;
                if (std::fabs(step) < 1e-10 * std::max(1.0, std::fabs(z))) z -= step;
            }
        }
        nodes[k] = z;
        double hp = 0, h = 1.0 / sbeta[0], sum = h * h;
        for (int l = 0; l + 1 < Q; ++l) {
            double hn = ((z - alpha[l]) * h - sbeta[l] * hp) / sbeta[l + 1];
            hp = h; h = hn;
            sum += h * h;
        }
        weights[k] = 1.0 / sum;
    }
    return true;
}

bool half_range_rule(int Q, std::vector<double> &nodes, std::vector<double> &weights)
{
    std::vector<double> a, sb;
    if (Q < 1 || Q > kMaxQ || !half_range_recurrence(Q + 1, a, sb)) return false;
    return gauss_from_recurrence(Q, a, sb, nodes, weights);
}

// Full range: probabilists' Hermite, orthonormal He_l / sqrt(l!): alpha = 0, sbeta_l = sqrt(l), sbeta_0 = 1.
bool full_range_rule(int Q, std::vector<double> &nodes, std::vector<double> &weights)
{
    if (Q < 1 || Q > kMaxQ) return false;
    std::vector<double> a(Q + 1, 0.0), sb(Q + 2);
    sb[0] = 1.0;
    for (int l = 1; l <= Q + 1; ++l) sb[l] = std::sqrt((double)l);
    return gauss_from_recurrence(Q, a, sb, nodes, weights);
}

bool build_tables(int Qx, int Qy, int Nxe, int Nye, double p0, HostTables &t, std::string &err)
{
    t.Qx = Qx; t.Qy = Qy; t.Nxe = Nxe; t.Nye = Nye; t.p0 = p0;
    t.V = 2 * Qx * Qy;
    // Projection rule: exact for degree < 2K; the Gaussian's modulation needs
    // a margin of nodes beyond the (N+1)/2 that polynomials of degree N need.
    t.K = projection_nodes(Nxe);
    int nrec = std::max(Qx, t.K) + 1;
    if (!half_range_recurrence(nrec, t.alpha, t.sbeta)) { err = "half-range recurrence failed"; return false; }
    if (!gauss_from_recurrence(Qx, t.alpha, t.sbeta, t.zx, t.wx)) { err = "half-range rule failed"; return false; }
    if (!gauss_from_recurrence(t.K, t.alpha, t.sbeta, t.Yk, t.Wk)) { err = "projection rule failed"; return false; }
    if (!full_range_rule(Qy, t.yy, t.wy)) { err = "full-range rule failed"; return false; }
    t.hz.assign((Nxe + 1) * Qx, 0.0);
    for (int i = 0; i < Qx; ++i) {
        double hp = 0, h = 1.0 / t.sbeta[0];
        for (int l = 0; l <= Nxe; ++l) {
            t.hz[l * Qx + i] = h;
            double hn = ((t.zx[i] - t.alpha[l]) * h - t.sbeta[l] * hp) / t.sbeta[l + 1];
            hp = h; h = hn;
        }
    }
    t.He.assign((Nye + 1) * Qy, 0.0);
    for (int j = 0; j < Qy; ++j) {
        double hp = 0, h = 1.0;
        for (int l = 0; l <= Nye; ++l) {
            t.He[l * Qy + j] = h;
            double hn = t.yy[j] * h - l * hp;
            hp = h; h = hn;
        }
    }
    return true;
}

// Discrete equilibrium factors (weight-divided), Eqs. gx and gy.
//  g_x: the half-range projection c_l = int_0^inf g(p; +-u_x, T) h_l(p/p0) dp/p0 of
//  Eq. gx, evaluated stably as a Gauss sum in y = z / sqrt(T'):
//    c_l^{+-} = sum_k W_k exp(+-a Y_k - a^2/2) h_l(sqrt(T') Y_k),  a = u'/sqrt(T'),
//  exact up to the (tiny) error of approximating exp(+-a y) by polynomials of
//  degree 2K-1-N; g_{x,i}/w_i = sum_l h_l(z_i) c_l^{sigma_i}.
//  g_y: Hermite coefficients b_l = E[He_l(u' + sqrt(T') Y)] / l! by the recurrence
//  b_{l+1} = (u' b_l + (T'-1) b_{l-1}) / (l+1); g_{y,j}/w_j = sum_l He_l(y_j) b_l.
void equilibrium_host(const HostTables &t, double ux, double uy, double T, double *gx, double *gy)
{
    const int N = t.Nxe, Qx = t.Qx;
    double Tp = T / (t.p0 * t.p0), up = ux / t.p0, sT = std::sqrt(Tp), a = up / sT;
    std::vector<double> cp(N + 1, 0.0), cm(N + 1, 0.0);
    for (int k = 0; k < t.K; ++k) {
        double zeta = sT * t.Yk[k];
        double rp = t.Wk[k] * std::exp(a * t.Yk[k] - 0.5 * a * a);
        double rm = t.Wk[k] * std::exp(-a * t.Yk[k] - 0.5 * a * a);
        double hp = 0, h = 1.0 / t.sbeta[0];
        for (int l = 0; l <= N; ++l) {
            cp[l] += rp * h;
            cm[l] += rm * h;
            double hn = ((zeta - t.alpha[l]) * h - t.sbeta[l] * hp) / t.sbeta[l + 1];
            hp = h; h = hn;
        }
    }
    for (int i = 0; i < Qx; ++i) {
        double sp = 0, sm = 0;
        for (int l = 0; l <= N; ++l) {
            sp += t.hz[l * Qx + i] * cp[l];
            sm += t.hz[l * Qx + i] * cm[l];
        }
        gx[i] = sp;
        gx[Qx + i] = sm;
    }
    double uq = uy / t.p0;
    std::vector<double> b(t.Nye + 1);
    b[0] = 1.0;
    if (t.Nye >= 1) b[1] = uq;
    for (int l = 1; l < t.Nye; ++l) b[l + 1] = (uq * b[l] + (Tp - 1.0) * b[l - 1]) / (l + 1.0);
    for (int j = 0; j < t.Qy; ++j) {
        double s = 0;
        for (int l = 0; l <= t.Nye; ++l) s += t.He[l * t.Qy + j] * b[l];
        gy[j] = s;
    }
}

// Grid of Eq. stretch: x = tanh(eta)/(2A), equidistant cell-centred eta on
// [-artanh A, artanh A]; A = 0 is the uniform grid (eta = x, J = 1). half: the
// Nx nodes of 0 < x < 1/2, which are the right half of the full grid of 2 Nx nodes.
void make_grid(int Nx, double A, bool half, std::vector<double> &x, std::vector<double> &jdeta,
               std::vector<double> &inv_jdeta, double &deta, double &min_jdeta)
{
    const int Nf = half ? 2 * Nx : Nx, s0 = half ? Nx : 0;
    x.resize(Nx);
    jdeta.resize(Nx);
    inv_jdeta.resize(Nx);
    min_jdeta = 1e300;
    const double ew = A == 0.0 ? 0.5 : std::atanh(A);
    deta = 2.0 * ew / Nf;
    for (int k = 0; k < Nx; ++k) {
        const double eta = -ew + (s0 + k + 0.5) * deta;
        double J = 1.0;
        if (A == 0.0) {
            x[k] = eta;
        } else {
            const double c = std::cosh(eta);
            J = 1.0 / (2.0 * A * c * c);
            x[k] = std::tanh(eta) / (2.0 * A);
        }
        jdeta[k] = J * deta;
        inv_jdeta[k] = 1.0 / (J * deta);
        min_jdeta = std::min(min_jdeta, J * deta);
    }
}

}  // namespace lbc
