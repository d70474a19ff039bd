// Device-side problem description and kernel launchers (sm_103a).
#pragma once
#include <cuda_runtime.h>

#include "lbc_internal.h"

namespace lbc {

constexpr int kTileCells = 32;     // cells per CTA tile: one warp lane per cell
constexpr int kWarps = 8;          // warps per CTA
constexpr int kThreads = kWarps * 32;

// Read-only problem data, passed by value to every kernel.
struct DevTables {
    int Nx, Nxp, Qx, Qy, Nxe, Nye, K, V;
    int ntile, nchunk, vchunk;
    double p0, dt, delta, Pr, omega, TL, TR;
    double inL, inR;               // sum_{incoming} p_x w_v fw_v (signed) for a unit wall density
    const double *inv_jdeta;       // [Nx] 1/(J_s deta)
    const double *zx, *wx, *yy, *wy;
    const double *alpha, *sbeta;   // orthonormal recurrence of h_l
    const double *hz;              // [Nxe+1][Qx]
    const double *Yk, *Wk;         // projection rule
    const double *He;              // [Nye+1][Qy]
    const double *fwL, *fwR;       // [V] unit-density wall Maxwellians (weight-divided)
    const double *frest;           // [V] rest Maxwellian n = 1, u = 0, T = 1
};

// Control block in device memory.
struct Ctl {
    long long base;        // steps launched so far (stage kernels add their relative index)
    long long check_from;  // early stop considers residuals of steps >= check_from only
    int stopped;           // set once a residual fell below the stop threshold
    int nonfinite;         // set if a NaN/Inf was produced
};

// Mutable device state. F[b]: [2][V][Nxp] in the state precision.
struct DevState {
    void *F[3];
    double *part[3];       // [nchunk][kNumRaw][Nxp] raw moment sums per velocity chunk
    double *shift[3];      // [2][Nxp] velocity shift of those sums
    unsigned long long *resid;   // [kResidRing] per-step residual (bits of a double >= 0)
    Ctl *ctl;
    double *mom_out;       // [LBC_NMOM][Nxp] scratch for lbc_moments
};

template <typename R>
cudaError_t configure_kernels();   // per-device kernel attributes; call before capture
template <typename R>
cudaError_t launch_stage(const DevTables &T, const DevState &S, int stage, int rel,
                         double stop_eps, cudaStream_t st);
template <typename R>
cudaError_t launch_moments_partial(const DevTables &T, const DevState &S, int buf, cudaStream_t st);
template <typename R>
cudaError_t launch_init_rest(const DevTables &T, const DevState &S, cudaStream_t st);
cudaError_t launch_finalize_moments(const DevTables &T, const DevState &S, int buf, cudaStream_t st);
cudaError_t launch_ctl_set(Ctl *ctl, long long base, long long check_from, int stopped, cudaStream_t st);
cudaError_t launch_ctl_bump(Ctl *ctl, long long k, cudaStream_t st);

}  // namespace lbc
