// Device-side problem description and kernel launchers (sm_103a).
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <string>
#include <vector>

#include "lbc_internal.h"

namespace lbc {

constexpr int kLanes = 32;
constexpr int kTile = 31;          // nodes per CTA tile: lane l owns node c0 + l (l < 31) and face c0 + l
constexpr int kRowLen = 40;        // TMA box width of a stage-input row (halo 3 + 31 + 3, aligned start)
constexpr int kF0Len = 36;         // TMA box width of an RK base row (31 nodes, aligned start)
constexpr int kWarps = 8;          // warps per CTA
constexpr int kThreads = kWarps * 32;
constexpr int kSubV = 32;          // velocity rows per pipeline slot (four per warp)
constexpr int kSubV0 = 64;         // the first RK stage in FP32, which stages no RK base: eight per warp
// Rows per pipeline slot of RK stage `stage` (and the TMA box height of state buffer `stage`).
__host__ __device__ constexpr int slot_rows(int stage, bool fp32) { return stage == 0 && fp32 ? kSubV0 : kSubV; }
constexpr int kPipe = 2;           // pipeline slots (one computed while the other lands)
constexpr int kEqM = 16;           // per-node stage data: n ux uy T qx qy 1/tau cS 1/(5T) 1/(J deta)
                                   // Pxx Pyy Pzz Pxy dt_s, 1 pad (64 B per FP32 node: 16-byte-aligned bulk copies)
constexpr int kMassHdr = 32;       // doubles before the per-node mass deviations in DevState::mass
constexpr int kMaxVChunk = 256;    // velocities per CTA at most (per-velocity data is staged in smem)
// Forms of the batched stage launch (how a tile's chunk CTAs combine their moment partials).
constexpr int kFormCluster = 0, kFormSolo = 1, kFormSplit = 2;
constexpr int kNodePart = 16;      // split form: nodes per CTA of the node-step launch (two CTAs per tile)
constexpr int kMaxCluster = 16;    // chunk CTAs of a tile form one thread-block cluster (non-portable size 16)
constexpr int kMaxV = kMaxCluster * kMaxVChunk;   // largest velocity set 2 Qx Qy
constexpr int kMaxTable = 256;     // entries of a viscosity table
constexpr int kPersistHdr = 4;     // counters before the per-item ones in the persistent form's block

// Scalars derived from the parameters, in both precisions (no FP64 arithmetic in the FP32 kernels).
enum { SC_NU = 0,      // delta sqrt(2): 1/tau = SC_NU n T^(1 - omega)   (Eq. tau)
       SC_EXPO,        // 1 - omega
       SC_1MPR,        // 1 - Pr
       SC_IP0,         // 1 / p0
       SC_H0,          // h_0 = 1 / sbeta_0 (orthonormal h_0)
       SC_DT,          // time step
       SC_IINL,        // 1 / inL
       SC_IINR,        // 1 / inR
       kNumSc };

// Read-only problem data, passed by value to every kernel. The state is stored
// as the deviation d = ft - ft_rest from the weight-divided rest Maxwellian.
struct DevTables {
    int Nx, Nxp, Qx, Qy, Nxe, Nye, K, V;
    int ntile, nchunk, vchunk;
    int law, tab_n;                // viscosity law (LBC_MU_POWER / LBC_MU_TABLE), table entries
    int lts;                       // local pseudo-time steps with mass renormalisation (local_dt)
    int half;                      // half channel: symmetry plane at x = 0 instead of the left wall
    int comp;                      // FP32 state with the rounding remainder of each value (DevState::C)
    double mrest;                  // sum_s J_s deta (the mass of the rest state n = 1)
    double p0, dt, delta, Pr, omega, TL, TR;
    double inL, inR;               // sum_{incoming} p_x w_v fw_v (signed) for a unit wall density
    double restOutL, restOutR;     // sum_{outgoing} p_x w_v ft_rest_v at each wall
    double restP[10];              // rest power sums sum_v w p_x^a p_y^b ft_rest: 00 10 01 20 11 02 30 21 12 03
    float f_restP[10];
    double dsc[kNumSc];
    float fsc[kNumSc];
    const double *inv_jdeta;       // [Nx] 1/(J_s deta)
    const double *jdeta;           // [Nx] J_s deta
    const double *dtn;             // [Nx] time step of node s (the global dt unless lts)
    const float *f_dtn;
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
    const double *d_vrow;  // [V][kVRow]
    const float *f_vrow;
    const double *d_eqtab; // EqTab layout
    const float *f_eqtab;
};
enum { VC_PX = 0, VC_PY, VC_W, VC_FR, VC_FWL, VC_FWLT, VC_FWR, VC_FWRT, kVelCols };
// Per-velocity rows [V][kVRow] (both precisions), copied per velocity chunk into
// shared memory: p_x, p_y, w, ft_rest, unit-density wall Maxwellians (phi, chi;
// left, right), and the shared-memory row offsets of g_x(a) and g_y(j) in the
// tile's equilibrium block, a kLanes and (2 Qx + j) kLanes, stored as integer
// bit patterns (int32 in the FP32 table, int64 in the FP64 table). 12 values:
// three 16-byte groups per FP32 row.
enum { VR_PX = 0, VR_PY, VR_W, VR_FR, VR_FWL, VR_FWLT, VR_FWR, VR_FWRT, VR_GA, VR_GJ, VR_PAD0, VR_PAD1, kVRow };

// Tables of the equilibrium construction, one contiguous block per precision,
// each piece padded to 4 elements (16-byte pieces in FP32): recurrence of h_l,
// 1/l, projection rule, h_l(z_i) [N+1][Qx] and He_l(y_j) [Ny+1][Qy]; and, for
// the table viscosity law (Eqs. mun, interp), ntab temperatures T_n, viscosities
// mu_n / mu(T_ref), segment exponents omega_n and Prandtl numbers Pr_n.
struct EqTab {
    int alpha, sbeta, isbeta, invl, Yk, Wk, hz, He, lawT, lawMu, lawW, lawPr, len;
    __host__ __device__ EqTab(int N, int Ny, int K, int Qx, int Qy, int ntab)
    {
        alpha = 0;
        sbeta = alpha + r4(N + 2);
        isbeta = sbeta + r4(N + 2);
        invl = isbeta + r4(N + 2);
        Yk = invl + r4(Ny + 2);
        Wk = Yk + r4(K);
        hz = Wk + r4(K);
        He = hz + r4((N + 1) * Qx);
        lawT = He + r4((Ny + 1) * Qy);
        lawMu = lawT + r4(ntab);
        lawW = lawMu + r4(ntab);
        lawPr = lawW + r4(ntab);
        len = lawPr + r4(ntab);
    }
    __host__ __device__ static int r4(int x) { return (x + 3) / 4 * 4; }
};

// Control block in device memory, one per instance. The host keeps the
// authoritative copy and uploads it to (re)start a run.
struct Ctl {
    long long base;        // steps launched so far (stage kernels add their relative index)
    long long check_from;  // early stop considers residuals of steps >= check_from only
    double stop_eps;       // early-stop threshold on the previous step's residual (0: never stop)
    long long stop_step;   // the step at which the instance stopped (valid once stopped)
    int stopped;           // set once a residual fell below stop_eps
    int nonfinite;         // set if a NaN/Inf was produced
    int timeout;           // set if a bounded wait on an mbarrier gave up
    int probe;             // test hook (LBC_FAULT=wait:N): > 0 makes every stage CTA wait at most this
                           // many polls on an mbarrier that nothing arrives at, so the bounded-wait
                           // path runs and reports; 0 in normal use
    int bounds;            // range-checked build (LBC_CHECKED): the first failed index check's site
    int pad;
};

// Range check of a computed index in the range-checked build (-DLBC_CHECKED): a failed check
// records its site in the instance's control block and the access is skipped (no trap, no
// fault); the host reports it. In the normal build the check is compiled away.
enum CheckSite : int {
    CK_NONE = 0,
    CK_TMA_X,      // a TMA box's x coordinate off its 16-byte boundary
    CK_BULK,       // a bulk copy outside its shared-memory region or its source array
    CK_STENCIL,    // a stencil, ghost-node or RK-base column outside the staged row box
    CK_GTAB,       // an equilibrium factor index outside the tile's factor table
    CK_STORE,      // a state (or compensation) store outside [0, V) x [0, Nxp)
    CK_MIRROR,     // a symmetry-plane partner row outside the state
    CK_XCH,        // a cluster exchange slot outside the receiving CTA's region
    CK_EQ,         // a node-stage write outside the stage data or the scratch capacity
    CK_WORK,       // a persistent item's neighbour outside the work list or of another instance
    CK_COUNT
};
const char *check_site_name(int site);   // host: the site's description
bool checked_build();                     // host: whether the kernels carry the range checks

#ifdef LBC_CHECKED
#define LBC_CHECK(ctl, cond, site) ((cond) ? true : (atomicCAS(&(ctl)->bounds, 0, (site)), false))
#else
#define LBC_CHECK(ctl, cond, site) true
#endif

// Mutable device state; arrays marked (R) hold the state precision.
struct DevState {
    void *F[3];            // (R) [V][Nxp][2] deviation from the rest state, (phi, chi) adjacent per node
    void *part;            // (R) [nchunk][kNumRaw][Nxp] raw moment sums of the deviation per velocity chunk:
                           //     about p = 0 at set-up and in lbc_moments; about the input stage's mean
                           //     velocity in the solo form of the stage kernel (the cluster form exchanges
                           //     its partials inside the tile's cluster)
    unsigned *tcnt;        // [ntile] solo form: chunk CTAs of the tile done with the current stage (the
                           //     last resets it to 0)
    void *eqm[3];          // (R) [Nxp][kEqM] moments and relaxation data of buffer b
    void *eqg[3];          // (R) [ntile][2Qx + Qy][kLanes] equilibrium factors of buffer b
    unsigned long long *resid;   // [kResidRing] per-step residual (bits of a double >= 0)
    Ctl *ctl;
    double *mom_out;       // [LBC_NMOM][Nxp] scratch for lbc_moments
    double *mass;          // local steps: [0] reference mass minus the rest mass; from kMassHdr on,
                           // [2][Nxp] J_s deta (n_s - 1) of buffer 0 after steps of parity 0 / 1
    void *C;               // (R) compensated state: [V][Nxp][2] rounding remainder of buffer 0 (else NULL)
    void *A;               // (R) compensated state: [V][Nxp][2] the step's increment accumulated over its
                           //     stages, dt (L0 + L1) after the second (else NULL)
};

// TMA descriptors of the state buffers, viewed as 2-D [V rows][2 Nxp columns].
struct StateMaps {
    CUtensorMap in[3];     // box 2 kRowLen x kSubV (stage input with halo, both fields)
    CUtensorMap f0;        // box 2 kF0Len x kSubV (RK base state, buffer 0)
};

// Everything the stage kernel needs about one instance (one Couette problem),
// in device memory. The tensor maps come first: they need 64-byte alignment.
struct alignas(128) Inst {
    StateMaps M;
    DevTables T;
    DevState S;
};

// Host-side image of one problem: tables, grid, time step, wall and rest data,
// and the device table block (FP64 pieces, FP32 copies, the index table).
struct ProblemSetup {
    HostTables t;
    int Nxe = 0, Nye = 0;
    std::vector<double> x, jdeta, inv_jdeta, dtn;   // dtn: time step per node
    double deta = 0, min_jdeta = 0, dt = 0, mrest = 0;
    std::vector<double> fwL, fwR, frest, vel, isb, invl, vrow, eqtab;
    std::vector<double> tabT, tabMu, tabW, tabPr;   // table viscosity law: mu_n / mu(T_ref), exponents
    std::vector<int> aj;
    double inL = 0, inR = 0, restOutL = 0, restOutR = 0, restP[10] = {0};
    std::vector<unsigned char> blob;   // device table block contents
};
// Validated parameters -> ProblemSetup (time step: see lbc_create in include/lbc.h).
bool setup_problem(const lbc_params &p, int Nxe, int Nye, ProblemSetup &ps, std::string &err);
// Fills T from ps, with the table pointers into the device copy `dev` of ps.blob.
// Leaves the launch shape (vchunk, nchunk) to choose_launch_shape.
void bind_tables(const ProblemSetup &ps, const lbc_params &p, const void *dev, DevTables &T);
// Velocity chunk of an instance split over `cluster` chunk CTAs (multiple of kSubV rows).
inline int chunk_rows(int V, int cluster) { return (V + kSubV * cluster - 1) / (kSubV * cluster) * kSubV; }
// Sets the stage kernel's attributes on the current device and picks the
// cluster size for one instance (T.nchunk) and its chunk rows (T.vchunk).
// LBC_ECUDA without a device; LBC_EINVAL if no cluster shape fits.
lbc_status choose_launch_shape(bool fp32, DevTables &T);
// Cluster size (chunk CTAs per tile), form and stage shared memory of a batch (sets every
// T.nchunk, T.vchunk); cluster_in > 0 forces the size; solo_in 1 / 0 forces the solo / cluster
// form, -1 chooses.
lbc_status choose_batch_shape(bool fp32, std::vector<DevTables> &Ts, int cluster_in, int solo_in, bool &solo,
                              int &cluster, size_t &smem);
// Solo-form shape with kMaxVChunk-row chunks (the last one of each instance shorter).
lbc_status choose_full_chunk_shape(bool fp32, std::vector<DevTables> &Ts, int &cluster, size_t &smem);
// Dynamic shared memory of the stage kernel for T's launch shape.
size_t stage_launch_smem(bool fp32, const DevTables &T);
// Errors and parameter checks shared by every entry point.
lbc_status fail(lbc_status st, const std::string &msg);
// Host-side fault injection for tests, from the LBC_FAULT environment variable (read at each
// use, so a test can set and clear it): "alloc" (device allocations of create and pool
// admission report failure without allocating), "launch" (stepping calls report a failed
// stage launch without launching), "admit" (pool admission reports no room), "wait:N" (the
// control blocks uploaded carry probe = N, see Ctl), "bounds:S" (the control blocks uploaded
// carry the failed-check site S, as if a range check of the checked build had failed). Nothing
// here touches the device.
bool fault_injected(const char *kind);
int fault_wait_polls();
int fault_bounds_site();
const char *last_error();
// Validates p (defaults already applied) and resolves the expansion orders.
lbc_status validate(const lbc_params &p, int &Nxe, int &Nye);
// TMA descriptor of a state buffer viewed as [V rows][2 Nxp columns], box 2 box_nodes x kSubV.
lbc_status encode_state_map(CUtensorMap *map, void *base, bool fp32, int V, int Nxp, int box_nodes, int box_rows);

template <typename R>
size_t stage_smem_bytes(int Qx, int Qy, int N, int Ny, int K, int vchunk, int cluster, int ntab);
template <typename R>
size_t equilibrium_smem_bytes(int Qx, int Qy, int N, int Ny, int K, int ntab);
// Clusters of `cluster` stage CTAs that can be resident at once (0: not launchable),
// for the single-instance (batch = false) or the batch stage kernel; solo: the batch
// kernel's solo form (no clusters), resident CTAs / cluster.
template <typename R>
cudaError_t stage_active_clusters(size_t smem, int cluster, bool batch, bool solo, int *nclusters);
template <typename R>
cudaError_t configure_kernels();   // per-device kernel attributes; call before capture
// One RK stage of one instance: grid (ntile, nchunk), cluster dims (1, nchunk, 1);
// the descriptor travels as a kernel parameter.
template <typename R>
cudaError_t launch_stage(const Inst &I, size_t smem, int stage, int rel, cudaStream_t st);
// One RK stage of every work item: grid (nwork, cluster), cluster dims (1, cluster, 1) in the
// cluster form (kFormCluster), no clusters in the solo form (kFormSolo: the tile's last chunk CTA
// builds the next stage's data of all its nodes; DevState::tcnt counts them in) and the split form
// (kFormSplit: a second launch, node_smem bytes of shared memory per CTA, builds it);
// work[i] = (instance, tile) with descriptors in device memory, instance < 0 for an empty slot.
// ext: some instance uses the half channel or local steps (the kernel form that has them).
template <typename R>
cudaError_t launch_stage_batch(const Inst *insts, const int2 *work, int nwork, int cluster, size_t smem, int stage,
                               int rel, bool ext, int form, size_t node_smem, cudaStream_t st);
// Persistent form: nsteps RK-3 steps of every work item in one cooperative launch of nclusters
// clusters (grid (nclusters, cluster)); cnt: kPersistHdr + nwork + n device counters (zeroed here);
// the steps' residual slots are zeroed first. Work items of an instance must be its tiles in order.
template <typename R>
cudaError_t launch_persistent(const Inst *insts, const int2 *work, int nwork, int n, int cluster, int nclusters,
                              size_t smem, int nsteps, bool ext, unsigned *cnt, cudaStream_t st);
template <typename R>
cudaError_t persistent_active_clusters(size_t smem, int cluster, int *nclusters);
template <typename R>
cudaError_t launch_moments_partial(const DevTables &T, const DevState &S, int buf, cudaStream_t st);
// Stage data of buffer `buf` from the chunk partials of launch_moments_partial; for
// buffer 0 with local steps also the mass deviations and the reference mass.
template <typename R>
cudaError_t launch_tile_equilibrium(const DevTables &T, const DevState &S, int buf, cudaStream_t st);
// Moments of buffer 0 (FP64, [LBC_NMOM][Nxp] in S.mom_out) from its stage data.
template <typename R>
cudaError_t launch_moments_from_stage_data(const DevTables &T, const DevState &S, cudaStream_t st);
// FP64 [2][V][Nx] weight-divided state in device memory -> deviation rows of buffer `dst`
// and, if `carry` is not NULL, the rounding remainder of each value (sets *bad, if not
// NULL, when a value is not finite); and back (adding the remainder when given).
template <typename R>
cudaError_t launch_state_in(const double *src, void *dst, void *carry, const DevTables &T, int *bad, cudaStream_t st);
template <typename R>
cudaError_t launch_state_out(const void *src, const void *carry, double *dst, const DevTables &T, cudaStream_t st);
cudaError_t launch_ctl_bump(Ctl *ctl, int n, long long k, cudaStream_t st);
// last[k] = residual of instance slots[k]'s (k's if slots is NULL) last step taken (its stop
// step - 1 if stopped, else base - 1), k < n
cudaError_t launch_last_residuals(const Inst *insts, const int *slots, int n, double *last, cudaStream_t st);

// NVTX range over a scope (header-only NVTX v3: a no-op unless a profiler is attached).
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

inline size_t round256(size_t x) { return (x + 255) / 256 * 256; }
// Device bytes of one instance's state (partials sized for the largest cluster, so
// a launch shape can change without reallocating).
struct StateSizes {
    size_t f, eqm, eqg, part, tcnt, resid, mom, mass, carry, acc, total;
    StateSizes(const DevTables &T, bool fp32)
    {
        const size_t esz = fp32 ? sizeof(float) : sizeof(double);
        f = round256(2 * (size_t)T.V * T.Nxp * esz);
        eqm = round256((size_t)T.Nxp * kEqM * esz);
        eqg = round256((size_t)T.ntile * (2 * T.Qx + T.Qy) * kLanes * esz);
        part = round256((size_t)kMaxCluster * kNumRaw * T.Nxp * esz);
        tcnt = round256((size_t)T.ntile * sizeof(unsigned));
        resid = kResidRing * sizeof(unsigned long long);
        mom = round256((size_t)LBC_NMOM * T.Nxp * sizeof(double));
        mass = round256((kMassHdr + 2 * (size_t)T.Nxp) * sizeof(double));
        carry = T.comp ? f : 0;
        acc = T.comp ? f : 0;
        total = 3 * (f + eqm + eqg) + part + tcnt + resid + mom + mass + carry + acc;
    }
    // Points the state arrays of S into `base` (total bytes); S.ctl is set by the caller.
    void carve(char *base, DevState &S) const
    {
        char *p = base;
        for (int k = 0; k < 3; ++k) { S.F[k] = p; p += f; }
        for (int k = 0; k < 3; ++k) { S.eqm[k] = p; p += eqm; }
        for (int k = 0; k < 3; ++k) { S.eqg[k] = p; p += eqg; }
        S.part = p; p += part;
        S.tcnt = reinterpret_cast<unsigned *>(p); p += tcnt;
        S.resid = reinterpret_cast<unsigned long long *>(p); p += resid;
        S.mom_out = reinterpret_cast<double *>(p); p += mom;
        S.mass = reinterpret_cast<double *>(p); p += mass;
        S.C = carry ? p : nullptr;
        p += carry;
        S.A = acc ? p : nullptr;
    }
};

}  // namespace lbc
