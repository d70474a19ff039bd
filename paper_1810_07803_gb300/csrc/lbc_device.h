// Device-side problem description and kernel launchers (sm_103a).
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>

#include "lbc_internal.h"

namespace lbc {

constexpr int kLanes = 32;
constexpr int kTile = 31;          // nodes per CTA tile: lane l owns node c0 + l (l < 31) and face c0 + l
constexpr int kRowLen = 40;        // TMA box width of a stage-input row (halo 3 + 31 + 3, aligned start)
constexpr int kF0Len = 36;         // TMA box width of an RK base row (31 nodes, aligned start)
constexpr int kWarps = 8;          // warps per CTA
constexpr int kThreads = kWarps * 32;
constexpr int kSubV = 16;          // velocities per pipeline stage (two per warp)
constexpr int kPipe = 4;           // pipeline depth (stages in flight)
constexpr int kEqM = 9;            // per-node stage data: n ux uy T qx qy 1/tau cS 1/(5T)
constexpr int kMaxVChunk = 256;    // velocities per CTA at most (per-velocity data is staged in smem)

// Read-only problem data, passed by value to every kernel. The state is stored
// as the deviation d = ft - ft_rest from the weight-divided rest Maxwellian.
struct DevTables {
    int Nx, Nxp, Qx, Qy, Nxe, Nye, K, V;
    int ntile, nchunk, vchunk;
    double p0, dt, delta, Pr, omega, TL, TR;
    double inL, inR;               // sum_{incoming} p_x w_v fw_v (signed) for a unit wall density
    double restOutL, restOutR;     // sum_{outgoing} p_x w_v ft_rest_v at each wall
    double restP[10];              // rest power sums sum_v w p_x^a p_y^b ft_rest: 00 10 01 20 11 02 30 21 12 03
    const double *inv_jdeta;       // [Nx] 1/(J_s deta)
    const double *zx, *wx, *yy, *wy;
    const double *alpha, *sbeta;   // orthonormal recurrence of h_l
    const double *hz;              // [Nxe+1][Qx]
    const double *Yk, *Wk;         // projection rule
    const double *He;              // [Nye+1][Qy]
    const double *fwL, *fwR;       // [V] unit-density wall Maxwellians (weight-divided)
    const double *frest;           // [V] rest Maxwellian n = 1, u = 0, T = 1 (weight-divided)
    // single-precision copies for the FP32 path
    const float *f_hz, *f_He, *f_alpha, *f_isbeta, *f_sbeta, *f_Yk, *f_Wk, *f_inv_l, *f_inv_jdeta;
    // per-velocity rows [kVelCols][V] in both precisions: p_x, p_y, w, ft_rest,
    // fw_L, T_L fw_L, fw_R, T_R fw_R; and the indices a, j of each velocity
    const double *d_vel;
    const float *f_vel;
    const int *vel_aj;     // [2][V]
};
enum { VC_PX = 0, VC_PY, VC_W, VC_FR, VC_FWL, VC_FWLT, VC_FWR, VC_FWRT, kVelCols };

// Control block in device memory.
struct Ctl {
    long long base;        // steps launched so far (stage kernels add their relative index)
    long long check_from;  // early stop considers residuals of steps >= check_from only
    int stopped;           // set once a residual fell below the stop threshold
    int nonfinite;         // set if a NaN/Inf was produced
    int timeout;           // set if a bounded wait on an mbarrier gave up
    int pad;
};

// Mutable device state; arrays marked (R) hold the state precision.
struct DevState {
    void *F[3];            // (R) [2][V][Nxp] deviation from the rest state
    void *part[3];         // (R) [nchunk][kNumRaw][Nxp] raw moment sums of the deviation per velocity chunk
    void *shift[3];        // (R) [2][Nxp] velocity shift of those sums
    void *eqm[3];          // (R) [Nxp][kEqM] moments and relaxation data of buffer b
    void *eqg[3];          // (R) [ntile][2Qx + Qy][kLanes] equilibrium factors of buffer b
    int *count[3];         // [ntile] chunk CTAs done with buffer b (the last one builds eqm/eqg)
    unsigned long long *resid;   // [kResidRing] per-step residual (bits of a double >= 0)
    Ctl *ctl;
    double *mom_out;       // [LBC_NMOM][Nxp] scratch for lbc_moments
};

// TMA descriptors of the state buffers, viewed as 2-D [2V rows][Nxp columns].
struct StateMaps {
    CUtensorMap in[3];     // box kRowLen x kSubV (stage input with halo)
    CUtensorMap f0;        // box kF0Len x kSubV (RK base state, buffer 0)
};

template <typename R>
size_t stage_smem_bytes(int Qx, int Qy, int N, int Ny, int K, int vchunk);
template <typename R>
cudaError_t stage_kernel_attributes(cudaFuncAttributes *fa);
template <typename R>
cudaError_t configure_kernels();   // per-device kernel attributes; call before capture
template <typename R>
cudaError_t launch_stage(const DevTables &T, const DevState &S, const StateMaps &M, int stage, int rel,
                         double stop_eps, cudaStream_t st);
template <typename R>
cudaError_t launch_moments_partial(const DevTables &T, const DevState &S, int buf, cudaStream_t st);
template <typename R>
cudaError_t launch_tile_equilibrium(const DevTables &T, const DevState &S, int buf, cudaStream_t st);
template <typename R>
cudaError_t launch_finalize_moments(const DevTables &T, const DevState &S, int buf, cudaStream_t st);
cudaError_t launch_ctl_set(Ctl *ctl, long long base, long long check_from, int stopped, cudaStream_t st);
cudaError_t launch_ctl_bump(Ctl *ctl, long long k, cudaStream_t st);

}  // namespace lbc
