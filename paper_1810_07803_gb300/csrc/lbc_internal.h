// Internal structures shared by the host set-up, the kernels and the C ABI.
#pragma once
#include <cstddef>
#include <string>
#include <vector>

#include "lbc.h"

namespace lbc {

constexpr int kMaxQ = 64;          // largest quadrature order accepted
// nodes of the half-range rule that projects the equilibrium: exact for degree
// < 2K; (N+1)/2 nodes for the polynomial part plus a margin for exp(a y)
constexpr int projection_nodes(int N) { return (N + 2) / 2 + 14; }
constexpr int kMaxK = projection_nodes(kMaxQ - 1);
constexpr int kNumRaw = 11;        // raw moment sums accumulated per node
constexpr int kResidRing = 4096;   // per-step residual slots kept on the device

// Raw sums about a per-node shift s = (s_x, s_y), xi' = p - s (weighted by w_v):
enum RawIdx { R_S0, R_SX, R_SY, R_SXX, R_SXY, R_SYY, R_CZ, R_R3X, R_R3Y, R_GX, R_GY };

// Host-side tables of one problem (FP64), built once at create time.
struct HostTables {
    int Qx = 0, Qy = 0, Nxe = 0, Nye = 0, K = 0, V = 0;
    double p0 = 1.0;
    std::vector<double> zx, wx;          // half-range rule, Qx nodes (ascending)
    std::vector<double> alpha, sbeta;    // orthonormal recurrence of h_l: alpha[0..L], sbeta[0..L+1]
    std::vector<double> hz;              // [Nxe+1][Qx]  h_l(z_i)
    std::vector<double> Yk, Wk;          // K-point half-range rule used by the projection
    std::vector<double> yy, wy;          // full-range rule, Qy nodes
    std::vector<double> He;              // [Nye+1][Qy]  He_l(y_j)
};

// Gauss rules (Sec. III). Return false on bad Q.
bool half_range_recurrence(int n, std::vector<double> &alpha, std::vector<double> &sbeta);
bool gauss_from_recurrence(int Q, const std::vector<double> &alpha, const std::vector<double> &sbeta,
                           std::vector<double> &nodes, std::vector<double> &weights);
bool full_range_rule(int Q, std::vector<double> &nodes, std::vector<double> &weights);
bool half_range_rule(int Q, std::vector<double> &nodes, std::vector<double> &weights);

bool build_tables(int Qx, int Qy, int Nxe, int Nye, double p0, HostTables &t, std::string &err);

// Discrete equilibrium factors on the host (same algorithm as the device).
void equilibrium_host(const HostTables &t, double ux, double uy, double T, double *gx, double *gy);

// Grid (Eq. stretch over the full channel, or its right half): x_s, J_s deta,
// 1/(J_s deta), deta, min_s J_s deta.
void make_grid(int Nx, double A, bool half, std::vector<double> &x, std::vector<double> &jdeta,
               std::vector<double> &inv_jdeta, double &deta, double &min_jdeta);

void set_error(const std::string &msg);

}  // namespace lbc
