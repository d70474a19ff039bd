/*
 * FP64 CPU oracle for the mixed-quadrature lattice Boltzmann solver of the
 * reduced Shakhov equation for planar Couette flow (Ambrus, Sharipov & Sofonea,
 * arXiv:1810.07803).
 *
 * TEST INFRASTRUCTURE ONLY: plain, slow, obviously correct. Only the tests, the
 * smoke check and the CPU-baseline leg of the benchmark may load this library.
 * It shares no code, header or table generator with the CUDA path. Its tables
 * (quadratures, Phi, He_l(y_j)) come from oracle/quadrature.py.
 *
 * Each function cites the part of the paper it follows:
 *   moments                         Sec. II, moment definitions after Eq. boltz_red
 *   Shakhov factors S_phi, S_chi    Sec. II, the equation after Eq. boltz_red
 *   discrete equilibrium g_x, g_y   Sec. III, Eqs. gx and gy
 *   diffuse walls, n_w              Sec. II, Eqs. diffuse and diffuse_nw
 *   relaxation time                 Sec. II, Eq. tau with mu ~ T^omega (Eq. mu)
 *   WENO-5 advection, stretching    Sec. III (Jiang-Shu WENO-5, Eq. stretch)
 *   TVD Runge-Kutta 3               Sec. III (Shu-Osher RK-3)
 *
 * Readings of points the paper leaves open (kept identical on the CUDA side):
 *   - state is the weight-divided population ft = phi_ij / (w_i w_j);
 *   - walls: outgoing ghosts by cubic extrapolation in eta, outgoing wall face
 *     by WENO-5, incoming face and ghosts = n_w times the wall Maxwellian;
 *   - WENO epsilon acts on ft; residual = max w_i w_j |ft^{n+1} - ft^n|.
 *
 * Units: m = k_B = 1, T_ref = 1, n_ref = 1, L = 1, v_ref = 1.
 * Velocity index v = a*Qy + j: a < Qx -> p_x = +p0 z_a, a >= Qx -> p_x = -p0 z_{a-Qx}
 * (the paper's p_{x,i+Qx} = -p_{x,i}); p_y = p0 y_j; weight w_a w_j.
 * State layout f[field][v][s], field 0 = phi, 1 = chi, s = 0..Nx-1.
 */
#define _GNU_SOURCE            /* _Float128 math (erff128, expf128, ...) */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

typedef struct {
    int Nx, Qx, Qy, Nxe, Nye;       /* grid size, quadrature orders, expansion orders */
    double p0, delta, Pr, omega;
    int law, tab_n;                 /* law 0: mu = T^omega, Pr; law 1: the table of Eqs. mun, interp */
    const double *tab_T, *tab_mu, *tab_Pr;   /* [tab_n] temperatures (increasing), viscosities, Prandtl */
    double uL, uR, TL, TR;          /* wall velocities (along y) and temperatures */
    double dt, deta, eps;           /* time step, eta spacing, WENO epsilon */
    const double *J;                /* [Nx] dx/deta at the nodes */
    const double *zx, *wx;          /* [Qx] half-range nodes / weights */
    const double *yy, *wy;          /* [Qy] full-range nodes / weights */
    const double *Phi, *Phi_lo;     /* [Nxe+1][Qx] Phi_{s,i} = Phi + Phi_lo (double-double) */
    const double *He, *He_lo;       /* [Nye+1][Qy] He_l(y_j) = He + He_lo (double-double) */
    int local_dt;                   /* 1: time step dtn[s] per node and mass renormalisation */
    int mirror;                     /* 1: half channel, symmetry plane instead of the left wall */
    const double *dtn;              /* [Nx] node time steps (local_dt only) */
    double mass_ref;                /* mass the local-step iteration keeps (local_dt only) */
} orc_problem;

enum { M_N, M_UX, M_UY, M_T, M_PXX, M_PYY, M_PZZ, M_PXY, M_QX, M_QY, M_COUNT };

static int nvel(const orc_problem *P) { return 2 * P->Qx * P->Qy; }

static double px_of(const orc_problem *P, int v)
{
    int a = v / P->Qy;
    return a < P->Qx ? P->p0 * P->zx[a] : -P->p0 * P->zx[a - P->Qx];
}
static double py_of(const orc_problem *P, int v) { return P->p0 * P->yy[v % P->Qy]; }
static double w_of(const orc_problem *P, int v)
{
    int a = v / P->Qy;
    return P->wx[a % P->Qx] * P->wy[v % P->Qy];
}

/* ---- moments of (phi, chi) at one node (two-pass, central) ------------- */
void orc_cell_moments(const orc_problem *P, const double *phi, const double *chi,
                      long stride, double *m)
{
    int V = nvel(P);
    double n = 0, jx = 0, jy = 0;
    for (int v = 0; v < V; ++v) {
        double wf = w_of(P, v) * phi[v * stride];
        n += wf;
        jx += px_of(P, v) * wf;
        jy += py_of(P, v) * wf;
    }
    double ux = jx / n, uy = jy / n;
    double pxx = 0, pyy = 0, pxy = 0, pzz = 0, qx = 0, qy = 0;
    for (int v = 0; v < V; ++v) {
        double w = w_of(P, v);
        double f = w * phi[v * stride], g = w * chi[v * stride];
        double xx = px_of(P, v) - ux, xy = py_of(P, v) - uy;
        pxx += xx * xx * f;
        pyy += xy * xy * f;
        pxy += xx * xy * f;
        pzz += g;
        qx += 0.5 * (xx * xx + xy * xy) * xx * f + 0.5 * xx * g;
        qy += 0.5 * (xx * xx + xy * xy) * xy * f + 0.5 * xy * g;
    }
    m[M_N] = n; m[M_UX] = ux; m[M_UY] = uy;
    m[M_T] = (pxx + pyy + pzz) / (3.0 * n);
    m[M_PXX] = pxx; m[M_PYY] = pyy; m[M_PZZ] = pzz; m[M_PXY] = pxy;
    m[M_QX] = qx; m[M_QY] = qy;
}

void orc_moments(const orc_problem *P, const double *f, double *mom /* [M_COUNT][Nx] */)
{
    int Nx = P->Nx, V = nvel(P);
    double m[M_COUNT];
    for (int s = 0; s < Nx; ++s) {
        orc_cell_moments(P, f + s, f + (long)V * Nx + s, Nx, m);
        for (int k = 0; k < M_COUNT; ++k) mom[k * Nx + s] = m[k];
    }
}

/* ---- discrete equilibrium, Eqs. gx and gy (weight-divided) ------------- */
typedef _Float128 qreal;

/* The bracket of Eq. gx for s = 0..N:
 *   B_s = (T/(2 p0^2))^{s/2} [(1 + erf zeta) P_s^+(zeta) + 2 exp(-zeta^2)/sqrt(pi) P_s^*(zeta)],
 * with P_s^{+-}(zeta) = exp(-+zeta^2) d^s/dzeta^s exp(+-zeta^2), i.e.
 * P_{s+1}^{+-} = +-2 zeta P_s^{+-} + 2 s P_{s-1}^{+-}, and
 * P_s^* = sum_{j=0}^{s-1} C(s, j) P_j^+ P_{s-j-1}^-.
 * Evaluated in binary128: the monomial form of Eq. gx cancels heavily for
 * large N, and FP64 loses every digit at N ~ 23 (this precision is a reading:
 * the paper fixes none). */
void orc_gx_bracket(int N, double zeta_d, double T_over_2p02, double *B_hi, double *B_lo,
                    qreal *B_out)
{
    qreal zeta = zeta_d;
    qreal Pp[64], Pm[64], Ps[64], B[64];
    Pp[0] = 1; Pm[0] = 1;
    if (N >= 1) { Pp[1] = 2 * zeta; Pm[1] = -2 * zeta; }
    for (int s = 1; s < N; ++s) {
        Pp[s + 1] = 2 * zeta * Pp[s] + 2 * s * Pp[s - 1];
        Pm[s + 1] = -2 * zeta * Pm[s] - 2 * s * Pm[s - 1];
    }
    Ps[0] = 0;
    for (int s = 1; s <= N; ++s) {
        qreal acc = 0, binom = 1;                    /* C(s, j), j = 0.. */
        for (int j = 0; j < s; ++j) {
            acc += binom * Pp[j] * Pm[s - j - 1];
            binom = binom * (s - j) / (j + 1);
        }
        Ps[s] = acc;
    }
    qreal e1 = 1 + erff128(zeta);
    qreal e2 = 2 * expf128(-zeta * zeta) / sqrtf128(M_PIf128);
    qreal sc = sqrtf128((qreal)T_over_2p02), scale = 1;
    for (int s = 0; s <= N; ++s) {
        B[s] = scale * (e1 * Pp[s] + e2 * Ps[s]);
        scale *= sc;
        if (B_hi) { B_hi[s] = (double)B[s]; B_lo[s] = (double)(B[s] - (qreal)B_hi[s]); }
        if (B_out) B_out[s] = B[s];
    }
}

/* gx[a] = g_{x,a} / w_a for a = 0..2Qx-1, gy[j] = g_{y,j} / w_j. */
void orc_equilibrium_factors(const orc_problem *P, double ux, double uy, double T,
                             double *gx, double *gy)
{
    int Nxe = P->Nxe, Nye = P->Nye, Qx = P->Qx, Qy = P->Qy;
    /* Eq. gx: g_{x,i}/w_i = 1/2 sum_s B_s(zeta_i) Phi_{s,i}, zeta_i = sigma_i u_x / sqrt(2 T). */
    for (int half = 0; half < 2; ++half) {
        double sigma = half == 0 ? 1.0 : -1.0;
        qreal B[64];
        orc_gx_bracket(Nxe, sigma * ux / sqrt(2.0 * T), T / (2.0 * P->p0 * P->p0), NULL, NULL, B);
        for (int i = 0; i < Qx; ++i) {
            qreal acc = 0;
            for (int s = 0; s <= Nxe; ++s)
                acc += B[s] * ((qreal)P->Phi[s * Qx + i] + (qreal)P->Phi_lo[s * Qx + i]);
            gx[half * Qx + i] = (double)(acc / 2);
        }
    }
    /* Eq. gy: g_{y,j}/w_j = sum_l He_l(y_j) sum_{s<=l/2}
     *   (T/p0^2 - 1)^s (u_y/p0)^{l-2s} / (2^s s! (l-2s)!), also in binary128
     * (the He_l at the outer nodes are large and the sum cancels). */
    qreal tt = (qreal)T / ((qreal)P->p0 * P->p0) - 1, uu = (qreal)uy / P->p0;
    qreal b[64];
    for (int l = 0; l <= Nye; ++l) {
        qreal c = 0;
        for (int s = 0; 2 * s <= l; ++s) {
            qreal den = 1;
            for (int k = 1; k <= s; ++k) den *= 2 * k;          /* 2^s s! */
            for (int k = 1; k <= l - 2 * s; ++k) den *= k;       /* (l-2s)! */
            qreal num = 1;
            for (int k = 0; k < s; ++k) num *= tt;
            for (int k = 0; k < l - 2 * s; ++k) num *= uu;
            c += num / den;
        }
        b[l] = c;
    }
    for (int j = 0; j < Qy; ++j) {
        qreal acc = 0;
        for (int l = 0; l <= Nye; ++l)
            acc += ((qreal)P->He[l * Qy + j] + (qreal)P->He_lo[l * Qy + j]) * b[l];
        gy[j] = (double)acc;
    }
}

/* ---- relaxation target (phi_eq (1 + S_phi), chi_eq (1 + S_chi)) -------- */
/* Sec. II: phi_eq = n g_x g_y, chi_eq = T phi_eq,
 * S_phi = (1-Pr)/(n T^2) ((xi_x^2+xi_y^2)/(5T) - 4/5)(q . xi), S_chi with 2/5. */
/* ---- viscosity and Prandtl number --------------------------------------- */
/* Number of table temperatures T_n <= T (0 .. tab_n). */
static int table_index(const orc_problem *P, double T)
{
    int k = 0;
    while (k < P->tab_n && P->tab_T[k] <= T) ++k;
    return k;
}

/* Eq. mun on the segment of Eq. interp that holds T (0-based segment c covers
 * [T_c, T_{c+1}); the first and last segments extend to T -> 0 and T -> inf). */
double orc_table_mu(const orc_problem *P, double T)
{
    int c = table_index(P, T) - 1;
    if (c < 0) c = 0;
    if (c > P->tab_n - 2) c = P->tab_n - 2;
    double w = log(P->tab_mu[c + 1] / P->tab_mu[c]) / log(P->tab_T[c + 1] / P->tab_T[c]);
    return P->tab_mu[c] * pow(T / P->tab_T[c], w);
}

/* mu(T) / mu(T_ref = 1): delta is defined with mu(T_ref). */
double orc_mu_ratio(const orc_problem *P, double T)
{
    if (P->law == 0) return pow(T, P->omega);
    return orc_table_mu(P, T) / orc_table_mu(P, 1.0);
}

/* Eq. interp for Pr: Pr_1 below T_2, Pr_n on [T_n, T_{n+1}), Pr_N from T_N on. */
double orc_prandtl(const orc_problem *P, double T)
{
    if (P->law == 0) return P->Pr;
    int k = table_index(P, T);
    return P->tab_Pr[k < 1 ? 0 : k - 1];
}

void orc_target(const orc_problem *P, const double *m, double *tphi, double *tchi)
{
    int V = nvel(P), Qy = P->Qy;
    double *gx = malloc(sizeof(double) * 2 * P->Qx), *gy = malloc(sizeof(double) * Qy);
    double n = m[M_N], ux = m[M_UX], uy = m[M_UY], T = m[M_T];
    orc_equilibrium_factors(P, ux, uy, T, gx, gy);
    double c = (1.0 - orc_prandtl(P, T)) / (n * T * T);
    for (int v = 0; v < V; ++v) {
        double feq = n * gx[v / Qy] * gy[v % Qy];
        double xx = px_of(P, v) - ux, xy = py_of(P, v) - uy;
        double qxi = m[M_QX] * xx + m[M_QY] * xy;
        double x2 = (xx * xx + xy * xy) / (5.0 * T);
        tphi[v] = feq * (1.0 + c * (x2 - 0.8) * qxi);
        tchi[v] = T * feq * (1.0 + c * (x2 - 0.4) * qxi);
    }
    free(gx); free(gy);
}

/* Eq. tau with T_ref = n_ref = 1: 1/tau = n T delta sqrt(2) / (mu(T)/mu(T_ref));
 * for mu = T^omega (Eq. mu) that is n T^{1-omega} delta sqrt(2). */
static double collision_rate(const orc_problem *P, double n, double T)
{
    return n * T / orc_mu_ratio(P, T) * P->delta * sqrt(2.0);
}

/* ---- WENO-5 (Jiang & Shu) face value, upwind cell is c ------------------ */
/* Returns the reconstruction at the face between c and d from a, b, c, d, e
 * (a = c-2, b = c-1, d = c+1, e = c+2). */
double orc_weno5(double a, double b, double c, double d, double e, double eps)
{
    double q0 = (2.0 * a - 7.0 * b + 11.0 * c) / 6.0;
    double q1 = (-b + 5.0 * c + 2.0 * d) / 6.0;
    double q2 = (2.0 * c + 5.0 * d - e) / 6.0;
    double b0 = 13.0 / 12.0 * (a - 2.0 * b + c) * (a - 2.0 * b + c)
              + 0.25 * (a - 4.0 * b + 3.0 * c) * (a - 4.0 * b + 3.0 * c);
    double b1 = 13.0 / 12.0 * (b - 2.0 * c + d) * (b - 2.0 * c + d)
              + 0.25 * (b - d) * (b - d);
    double b2 = 13.0 / 12.0 * (c - 2.0 * d + e) * (c - 2.0 * d + e)
              + 0.25 * (3.0 * c - 4.0 * d + e) * (3.0 * c - 4.0 * d + e);
    double a0 = 0.1 / ((eps + b0) * (eps + b0));
    double a1 = 0.6 / ((eps + b1) * (eps + b1));
    double a2 = 0.3 / ((eps + b2) * (eps + b2));
    return (a0 * q0 + a1 * q1 + a2 * q2) / (a0 + a1 + a2);
}

/* ---- wall Maxwellians (weight-divided), incoming halves only ------------ */
/* fw_left[v] for p_x > 0, fw_right[v] for p_x < 0 (Eq. diffuse): g_x(0, T_w) g_y(u_w, T_w). */
static void wall_maxwellians(const orc_problem *P, double *fwl, double *fwr)
{
    int Qx = P->Qx, Qy = P->Qy, V = nvel(P);
    double *gx = malloc(sizeof(double) * 2 * Qx), *gy = malloc(sizeof(double) * Qy);
    orc_equilibrium_factors(P, 0.0, P->uL, P->TL, gx, gy);
    for (int v = 0; v < V; ++v) fwl[v] = gx[v / Qy] * gy[v % Qy];
    orc_equilibrium_factors(P, 0.0, P->uR, P->TR, gx, gy);
    for (int v = 0; v < V; ++v) fwr[v] = gx[v / Qy] * gy[v % Qy];
    free(gx); free(gy);
}

/* Velocity with the opposite momentum, (p_x, p_y) -> (-p_x, -p_y): the two
 * half-range halves hold opposite nodes (a <-> a + Qx), and the full-range
 * nodes are symmetric (j <-> Qy - 1 - j). */
static int mirror_velocity(const orc_problem *P, int v)
{
    int a = v / P->Qy, j = v % P->Qy;
    return ((a + P->Qx) % (2 * P->Qx)) * P->Qy + (P->Qy - 1 - j);
}

/* ---- right-hand side L(f) = advection + relaxation ---------------------- */
/* nw_out (optional) receives n_w at the left and right walls (left: 0 on the
 * half channel). Half channel (P->mirror, Sec. II's symmetry of Couette flow
 * between walls of equal temperature moving in opposite directions,
 * phi(-x, -p) = phi(x, p)): the domain is 0 < x < 1/2 and the ghost nodes left
 * of x = 0 are the mirror images of nodes 0, 1, 2 at the opposite velocity. */
void orc_rhs(const orc_problem *P, const double *f, double *L, double *nw_out)
{
    int Nx = P->Nx, V = nvel(P), Qy = P->Qy;
    long fs = (long)V * Nx;
    double *fwl = malloc(sizeof(double) * V), *fwr = malloc(sizeof(double) * V);
    double *face = malloc(sizeof(double) * (Nx + 1) * 2 * V); /* [field][v][Nx+1] */
    wall_maxwellians(P, fwl, fwr);

    /* 1) faces of outgoing populations, with cubically extrapolated ghosts
     *    (in the uniform eta coordinate, Eq. stretch). Rows are independent: the
     *    OpenMP build of this file splits them over threads, each with its own
     *    extended row ext[s+2] = cell s; without OpenMP the block runs once. */
#pragma omp parallel
    {
    double *ext = malloc(sizeof(double) * (Nx + 4));
#pragma omp for collapse(2) schedule(static)
    for (int fld = 0; fld < 2; ++fld)
        for (int v = 0; v < V; ++v) {
            const double *row = f + fld * fs + (long)v * Nx;
            double *F = face + ((long)fld * V + v) * (Nx + 1);
            double px = px_of(P, v);
            for (int s = 0; s < Nx; ++s) ext[s + 2] = row[s];
            if (px > 0) {   /* outgoing at the right wall */
                ext[Nx + 2] = 4 * row[Nx - 1] - 6 * row[Nx - 2] + 4 * row[Nx - 3] - row[Nx - 4];
                ext[Nx + 3] = 10 * row[Nx - 1] - 20 * row[Nx - 2] + 15 * row[Nx - 3] - 4 * row[Nx - 4];
                F[Nx] = orc_weno5(ext[Nx - 1], ext[Nx], ext[Nx + 1], ext[Nx + 2], ext[Nx + 3], P->eps);
            } else if (P->mirror) {   /* face at the symmetry plane: mirror ghosts */
                const double *mrow = f + fld * fs + (long)mirror_velocity(P, v) * Nx;
                ext[1] = mrow[0];
                ext[0] = mrow[1];
                F[0] = orc_weno5(ext[4], ext[3], ext[2], ext[1], ext[0], P->eps);
            } else {        /* outgoing at the left wall */
                ext[1] = 4 * row[0] - 6 * row[1] + 4 * row[2] - row[3];
                ext[0] = 10 * row[0] - 20 * row[1] + 15 * row[2] - 4 * row[3];
                F[0] = orc_weno5(ext[4], ext[3], ext[2], ext[1], ext[0], P->eps);
            }
        }

    free(ext);
    }

    /* 2) n_w from zero mass flux through each wall (Eq. diffuse_nw), phi only. */
    double outL = 0, outR = 0, inL = 0, inR = 0;
    for (int v = 0; v < V; ++v) {
        double px = px_of(P, v), w = w_of(P, v);
        const double *F = face + (long)v * (Nx + 1);
        if (px > 0) { outR += px * w * F[Nx]; inL += px * w * fwl[v]; }
        else        { outL += px * w * F[0];  inR += px * w * fwr[v]; }
    }
    double nwL = P->mirror ? 0.0 : -outL / inL, nwR = -outR / inR;
    if (nw_out) { nw_out[0] = nwL; nw_out[1] = nwR; }

    /* 3) remaining faces; incoming ghosts and wall faces = n_w f_w (chi: T_w n_w f_w). */
#pragma omp parallel
    {
    double *ext = malloc(sizeof(double) * (Nx + 4));
#pragma omp for collapse(2) schedule(static)
    for (int fld = 0; fld < 2; ++fld)
        for (int v = 0; v < V; ++v) {
            const double *row = f + fld * fs + (long)v * Nx;
            double *F = face + ((long)fld * V + v) * (Nx + 1);
            double px = px_of(P, v);
            for (int s = 0; s < Nx; ++s) ext[s + 2] = row[s];
            const double *mrow = f + fld * fs + (long)mirror_velocity(P, v) * Nx;
            if (px > 0) {
                double in = nwL * fwl[v] * (fld ? P->TL : 1.0);
                ext[0] = ext[1] = in;
                ext[Nx + 2] = 4 * row[Nx - 1] - 6 * row[Nx - 2] + 4 * row[Nx - 3] - row[Nx - 4];
                ext[Nx + 3] = 10 * row[Nx - 1] - 20 * row[Nx - 2] + 15 * row[Nx - 3] - 4 * row[Nx - 4];
                F[0] = in;
                if (P->mirror) {   /* ghosts -1, -2, -3 = nodes 0, 1, 2 at the opposite velocity */
                    ext[1] = mrow[0];
                    ext[0] = mrow[1];
                    F[0] = orc_weno5(mrow[2], mrow[1], mrow[0], row[0], row[1], P->eps);
                }
                /* face k (left of cell k), upwind cell k-1: stencil k-3..k+1 */
                for (int k = 1; k < Nx; ++k)
                    F[k] = orc_weno5(ext[k - 1], ext[k], ext[k + 1], ext[k + 2], ext[k + 3], P->eps);
            } else {
                double in = nwR * fwr[v] * (fld ? P->TR : 1.0);
                ext[Nx + 2] = ext[Nx + 3] = in;
                ext[1] = 4 * row[0] - 6 * row[1] + 4 * row[2] - row[3];
                ext[0] = 10 * row[0] - 20 * row[1] + 15 * row[2] - 4 * row[3];
                if (P->mirror) {
                    ext[1] = mrow[0];
                    ext[0] = mrow[1];
                }
                F[Nx] = in;
                /* upwind cell k: mirrored stencil k+2..k-2 */
                for (int k = 1; k < Nx; ++k)
                    F[k] = orc_weno5(ext[k + 4], ext[k + 3], ext[k + 2], ext[k + 1], ext[k], P->eps);
            }
        }

    free(ext);
    }

    /* 4) L = -(p_x / (J deta)) (F_{s+1/2} - F_{s-1/2}) - (f - f_eq (1 + S)) / tau. */
#pragma omp parallel
    {
    double *tphi = malloc(sizeof(double) * V), *tchi = malloc(sizeof(double) * V);
    double m[M_COUNT];
#pragma omp for schedule(static)
    for (int s = 0; s < Nx; ++s) {
        orc_cell_moments(P, f + s, f + fs + s, Nx, m);
        orc_target(P, m, tphi, tchi);
        double nu = collision_rate(P, m[M_N], m[M_T]);
        for (int fld = 0; fld < 2; ++fld)
            for (int v = 0; v < V; ++v) {
                const double *F = face + ((long)fld * V + v) * (Nx + 1);
                double fv = f[fld * fs + (long)v * Nx + s];
                double tgt = fld ? tchi[v] : tphi[v];
                L[fld * fs + (long)v * Nx + s] =
                    -px_of(P, v) * (F[s + 1] - F[s]) / (P->J[s] * P->deta) - nu * (fv - tgt);
            }
    }
    free(tphi); free(tchi);
    }
    (void)Qy;
    free(fwl); free(fwr); free(face);
}

/* ---- TVD RK-3 (Shu & Osher) over a generic right-hand side --------------- */
typedef void (*orc_rhs_fn)(void *ctx, const double *y, double *dy);

void orc_ssprk3(long n, double *y, double dt, orc_rhs_fn rhs, void *ctx)
{
    double *y1 = malloc(sizeof(double) * n), *y2 = malloc(sizeof(double) * n);
    double *k = malloc(sizeof(double) * n);
    rhs(ctx, y, k);
#pragma omp parallel for schedule(static)
    for (long i = 0; i < n; ++i) y1[i] = y[i] + dt * k[i];
    rhs(ctx, y1, k);
#pragma omp parallel for schedule(static)
    for (long i = 0; i < n; ++i) y2[i] = 0.75 * y[i] + 0.25 * (y1[i] + dt * k[i]);
    rhs(ctx, y2, k);
#pragma omp parallel for schedule(static)
    for (long i = 0; i < n; ++i) y[i] = y[i] / 3.0 + 2.0 / 3.0 * (y2[i] + dt * k[i]);
    free(y1); free(y2); free(k);
}

/* The same step with a time step per node: component i of y = [..][Nx] is node
 * i % Nx and advances by dtn[i % Nx]. With every dtn[s] = dt it is the step above. */
void orc_ssprk3_nodal(long n, int Nx, double *y, const double *dtn, orc_rhs_fn rhs, void *ctx)
{
    double *y1 = malloc(sizeof(double) * n), *y2 = malloc(sizeof(double) * n);
    double *k = malloc(sizeof(double) * n);
    rhs(ctx, y, k);
    for (long i = 0; i < n; ++i) y1[i] = y[i] + dtn[i % Nx] * k[i];
    rhs(ctx, y1, k);
    for (long i = 0; i < n; ++i) y2[i] = 0.75 * y[i] + 0.25 * (y1[i] + dtn[i % Nx] * k[i]);
    rhs(ctx, y2, k);
    for (long i = 0; i < n; ++i) y[i] = y[i] / 3.0 + 2.0 / 3.0 * (y2[i] + dtn[i % Nx] * k[i]);
    free(y1); free(y2); free(k);
}

static void problem_rhs(void *ctx, const double *y, double *dy)
{
    orc_rhs((const orc_problem *)ctx, y, dy, NULL);
}

/* Mass per unit wall area, sum_s J_s deta n_s with n_s = sum_v w_v phi_v,s. */
double orc_total_mass(const orc_problem *P, const double *f)
{
    int V = nvel(P), Nx = P->Nx;
    double M = 0.0;
    for (int s = 0; s < Nx; ++s) {
        double n = 0.0;
        for (int v = 0; v < V; ++v) n += w_of(P, v) * f[(long)v * Nx + s];
        M += P->J[s] * P->deta * n;
    }
    return M;
}

/* Runs up to nsteps RK-3 steps in place on f. resid[k] (optional) receives
 * max_{fld,v,s} w_v |f^{k+1} - f^k|; stops early once it drops below stop_below
 * (if > 0). Returns the number of steps taken.
 * Local steps (P->local_dt, a pseudo-time iteration for the steady state): node s
 * advances by dtn[s]; the fluxes then no longer telescope, so each step's result
 * is multiplied by mass_ref / M(f^k), M of the step's input state, which keeps
 * the mass of the iteration at mass_ref (a reading: the paper uses one time step). */
long orc_run(const orc_problem *P, double *f, long nsteps, double *resid, double stop_below)
{
    long n = 2L * nvel(P) * P->Nx;
    double *prev = malloc(sizeof(double) * n);
    long k;
    for (k = 0; k < nsteps; ++k) {
        memcpy(prev, f, sizeof(double) * n);
        if (P->local_dt) {
            orc_ssprk3_nodal(n, P->Nx, f, P->dtn, problem_rhs, (void *)P);
            double lam = P->mass_ref / orc_total_mass(P, prev);
            for (long i = 0; i < n; ++i) f[i] *= lam;
        } else {
            orc_ssprk3(n, f, P->dt, problem_rhs, (void *)P);
        }
        double r = 0;
#pragma omp parallel for reduction(max : r) schedule(static)
        for (long i = 0; i < n; ++i) {
            int v = (int)((i / P->Nx) % nvel(P));
            double d = w_of(P, v) * fabs(f[i] - prev[i]);
            if (d > r) r = d;
        }
        if (resid) resid[k] = r;
        if (stop_below > 0 && r < stop_below) { ++k; break; }
    }
    free(prev);
    return k;
}

/* Rest Maxwellian n = 1, u = 0, T = 1 at every node (weight-divided). */
void orc_rest_state(const orc_problem *P, double *f)
{
    int V = nvel(P), Nx = P->Nx, Qy = P->Qy;
    double *gx = malloc(sizeof(double) * 2 * P->Qx), *gy = malloc(sizeof(double) * Qy);
    orc_equilibrium_factors(P, 0.0, 0.0, 1.0, gx, gy);
    for (int v = 0; v < V; ++v)
        for (int s = 0; s < Nx; ++s) {
            double g = gx[v / Qy] * gy[v % Qy];
            f[(long)v * Nx + s] = g;
            f[(long)V * Nx + (long)v * Nx + s] = g;
        }
    free(gx); free(gy);
}
