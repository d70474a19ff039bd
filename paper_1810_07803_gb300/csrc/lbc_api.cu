// C ABI of the solver (include/lbc.h): validation, set-up, device memory,
// stepping (eager launches and CUDA graphs), run-to-steady, moments, state I/O.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "lbc_device.h"

namespace lbc {

namespace {
thread_local std::string g_err;
constexpr int kGraphSteps = 64;   // RK-3 steps captured per CUDA graph
}  // namespace

void set_error(const std::string &msg) { g_err = msg; }

}  // namespace lbc

using namespace lbc;

struct lbc_solver {
    lbc_params p{};
    HostTables tab;
    DevTables T{};
    DevState S{};
    StateMaps M{};
    cudaStream_t stream = nullptr;
    bool fp32 = false;
    bool poisoned = false;
    long long steps = 0;             // completed steps
    std::vector<double> x;
    std::vector<double> frest;       // weight-divided rest Maxwellian per velocity (state origin)
    void *table_block = nullptr;     // all constant tables, one allocation
    void *state_block = nullptr;     // state, moment partials, control
    cudaGraphExec_t graph = nullptr;
    unsigned long long *h_resid = nullptr;   // pinned copy of the residual ring
    Ctl *h_ctl = nullptr;                     // pinned copy of the control block
};

namespace {

#define LBC_CUDA_TRY(call)                                                                   \
    do {                                                                                     \
        cudaError_t e_ = (call);                                                             \
        if (e_ != cudaSuccess) {                                                             \
            set_error(std::string(#call) + ": " + cudaGetErrorString(e_));                   \
            return e_ == cudaErrorMemoryAllocation ? LBC_ENOMEM : LBC_ECUDA;                 \
        }                                                                                    \
    } while (0)

lbc_status fail(lbc_status st, const std::string &msg)
{
    set_error(msg);
    return st;
}

lbc_status validate(const lbc_params &p, int &Nxe, int &Nye)
{
    if (p.Qx < 1 || p.Qx > kMaxQ || p.Qy < 1 || p.Qy > kMaxQ) return fail(LBC_EINVAL, "Qx and Qy must be in [1, 64]");
    Nxe = p.Nexp_x ? p.Nexp_x : p.Qx - 1;
    Nye = p.Nexp_y ? p.Nexp_y : p.Qy - 1;
    if (Nxe < 2 || Nxe >= p.Qx) return fail(LBC_EINVAL, "expansion order Nexp_x must satisfy 2 <= N < Qx");
    if (Nye < 2 || Nye >= p.Qy) return fail(LBC_EINVAL, "expansion order Nexp_y must satisfy 2 <= N < Qy");
    if (p.Nx < 8 || p.Nx > (1 << 24)) return fail(LBC_EINVAL, "Nx must be in [8, 2^24]");
    if (!(p.delta >= 0.0) || !std::isfinite(p.delta)) return fail(LBC_EINVAL, "delta must be finite and >= 0");
    if (!(p.T_left > 0.0) || !(p.T_right > 0.0)) return fail(LBC_EINVAL, "wall temperatures must be > 0");
    if (!std::isfinite(p.u_left) || !std::isfinite(p.u_right)) return fail(LBC_EINVAL, "wall velocities must be finite");
    if (!(p.stretch_A >= 0.0 && p.stretch_A < 1.0)) return fail(LBC_EINVAL, "stretch_A must be in [0, 1)");
    if (p.p0 < 0.0 || !std::isfinite(p.p0)) return fail(LBC_EINVAL, "p0 must be > 0 (0 selects 1)");
    if (p.cfl < 0.0 || p.dt < 0.0) return fail(LBC_EINVAL, "cfl and dt must be >= 0");
    if (!std::isfinite(p.Pr) || p.Pr <= 0.0) return fail(LBC_EINVAL, "Pr must be > 0");
    if (p.mu_law != LBC_MU_POWER) return fail(LBC_EINVAL, "only the power-law viscosity (LBC_MU_POWER) is built");
    if (!std::isfinite(p.omega)) return fail(LBC_EINVAL, "omega must be finite");
    if (p.precision != LBC_FP64 && p.precision != LBC_FP32_STATE) return fail(LBC_EINVAL, "unknown precision");
    return LBC_OK;
}

template <typename R>
cudaError_t launch_step_range(lbc_solver *s, int rel0, int nsteps, double stop_eps)
{
    for (int k = 0; k < nsteps; ++k)
        for (int st = 0; st < 3; ++st) {
            cudaError_t e = launch_stage<R>(s->T, s->S, s->M, st, rel0 + k, stop_eps, s->stream);
            if (e != cudaSuccess) return e;
        }
    return cudaSuccess;
}

cudaError_t launch_steps(lbc_solver *s, int rel0, int nsteps, double stop_eps)
{
    return s->fp32 ? launch_step_range<float>(s, rel0, nsteps, stop_eps)
                   : launch_step_range<double>(s, rel0, nsteps, stop_eps);
}

// Captures kGraphSteps plain steps (no early stop) plus the step-counter bump
// into one CUDA graph, launched by lbc_step for every full group of steps.
lbc_status ensure_graph(lbc_solver *s)
{
    if (s->graph) return LBC_OK;
    cudaStream_t cap;
    LBC_CUDA_TRY(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
    cudaGraph_t g;
    cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        cudaStream_t keep = s->stream;
        s->stream = cap;
        e = launch_steps(s, 0, kGraphSteps, 0.0);
        if (e == cudaSuccess) e = launch_ctl_bump(s->S.ctl, kGraphSteps, cap);
        s->stream = keep;
        cudaError_t e2 = cudaStreamEndCapture(cap, &g);
        if (e == cudaSuccess) e = e2;
    }
    if (e == cudaSuccess) {
        e = cudaGraphInstantiate(&s->graph, g, 0);
        cudaGraphDestroy(g);
    }
    cudaStreamDestroy(cap);
    if (e != cudaSuccess) return fail(LBC_ECUDA, std::string("graph capture: ") + cudaGetErrorString(e));
    return LBC_OK;
}

}  // namespace

namespace lbc {

namespace {
struct DPiece { const std::vector<double> *src; const double **dst; };
struct FPiece { const std::vector<double> *src; const float **dst; };

// The device table block: FP64 pieces (each padded to 32 doubles), then FP32
// copies (each padded to 64 floats), then the velocity index table.
std::vector<DPiece> dpieces(const ProblemSetup &ps, DevTables &T)
{
    const HostTables &t = ps.t;
    return {{&ps.inv_jdeta, &T.inv_jdeta}, {&t.zx, &T.zx}, {&t.wx, &T.wx}, {&t.yy, &T.yy}, {&t.wy, &T.wy},
            {&t.alpha, &T.alpha}, {&t.sbeta, &T.sbeta}, {&t.hz, &T.hz}, {&t.Yk, &T.Yk}, {&t.Wk, &T.Wk},
            {&t.He, &T.He}, {&ps.fwL, &T.fwL}, {&ps.fwR, &T.fwR}, {&ps.frest, &T.frest}, {&ps.vel, &T.d_vel},
            {&ps.vrow, &T.d_vrow}, {&ps.eqtab, &T.d_eqtab}};
}
std::vector<FPiece> fpieces(const ProblemSetup &ps, DevTables &T)
{
    const HostTables &t = ps.t;
    return {{&t.hz, &T.f_hz}, {&t.He, &T.f_He}, {&t.alpha, &T.f_alpha}, {&ps.isb, &T.f_isbeta},
            {&t.sbeta, &T.f_sbeta}, {&t.Yk, &T.f_Yk}, {&t.Wk, &T.f_Wk}, {&ps.invl, &T.f_inv_l},
            {&ps.vel, &T.f_vel}, {&ps.inv_jdeta, &T.f_inv_jdeta}, {&ps.vrow, &T.f_vrow}, {&ps.eqtab, &T.f_eqtab}};
}
size_t pad_d(size_t n) { return (n + 31) / 32 * 32; }
size_t pad_f(size_t n) { return (n + 63) / 64 * 64; }
}  // namespace

bool setup_problem(const lbc_params &p, int Nxe, int Nye, ProblemSetup &ps, std::string &err)
{
    if (!build_tables(p.Qx, p.Qy, Nxe, Nye, p.p0, ps.t, err)) return false;
    const HostTables &t = ps.t;
    ps.Nxe = Nxe;
    ps.Nye = Nye;
    const int V = t.V;
    if (V > kMaxV) {
        err = "velocity set 2 Qx Qy = " + std::to_string(V) + " exceeds " + std::to_string(kMaxV);
        return false;
    }
    make_grid(p.Nx, p.stretch_A, ps.x, ps.inv_jdeta, ps.deta, ps.min_jdeta);

    // time step: CFL on the smallest cell, and half the smallest relaxation time
    double dt = p.dt > 0 ? p.dt : p.cfl * ps.min_jdeta / (t.zx.back() * p.p0);
    if (p.dt <= 0 && p.delta > 0)
        for (double Tw : {1.0, p.T_left, p.T_right})
            dt = std::min(dt, 0.5 * std::pow(Tw, p.omega - 1.0) / (p.delta * std::sqrt(2.0)));
    ps.dt = dt;

    // wall Maxwellians (unit density), incoming unit fluxes, rest Maxwellian
    std::vector<double> gx(2 * p.Qx), gy(p.Qy);
    ps.fwL.resize(V); ps.fwR.resize(V); ps.frest.resize(V);
    equilibrium_host(t, 0.0, p.u_left, p.T_left, gx.data(), gy.data());
    for (int v = 0; v < V; ++v) ps.fwL[v] = gx[v / p.Qy] * gy[v % p.Qy];
    equilibrium_host(t, 0.0, p.u_right, p.T_right, gx.data(), gy.data());
    for (int v = 0; v < V; ++v) ps.fwR[v] = gx[v / p.Qy] * gy[v % p.Qy];
    equilibrium_host(t, 0.0, 0.0, 1.0, gx.data(), gy.data());
    for (int v = 0; v < V; ++v) ps.frest[v] = gx[v / p.Qy] * gy[v % p.Qy];
    ps.vel.assign((size_t)kVelCols * V, 0.0);
    ps.aj.assign(2 * (size_t)V, 0);
    for (int v = 0; v < V; ++v) {
        const int a = v / p.Qy, j = v % p.Qy, i = a < p.Qx ? a : a - p.Qx;
        const double px = (a < p.Qx ? 1.0 : -1.0) * p.p0 * t.zx[i], py = p.p0 * t.yy[j], w = t.wx[i] * t.wy[j];
        if (px > 0) { ps.inL += px * w * ps.fwL[v]; ps.restOutR += px * w * ps.frest[v]; }
        else        { ps.inR += px * w * ps.fwR[v]; ps.restOutL += px * w * ps.frest[v]; }
        const double pw[10] = {1, px, py, px * px, px * py, py * py, px * px * px, px * px * py, px * py * py,
                               py * py * py};
        for (int k = 0; k < 10; ++k) ps.restP[k] += pw[k] * w * ps.frest[v];
        const double cols[kVelCols] = {px, py, w, ps.frest[v], ps.fwL[v], p.T_left * ps.fwL[v], ps.fwR[v],
                                       p.T_right * ps.fwR[v]};
        for (int c = 0; c < kVelCols; ++c) ps.vel[(size_t)c * V + v] = cols[c];
        ps.aj[v] = a;
        ps.aj[V + v] = j;
    }
    ps.isb.resize(t.sbeta.size());
    for (size_t k = 0; k < ps.isb.size(); ++k) ps.isb[k] = 1.0 / t.sbeta[k];
    ps.invl.assign(kMaxQ + 2, 0.0);
    for (int l = 1; l < kMaxQ + 2; ++l) ps.invl[l] = 1.0 / l;
    ps.vrow.assign((size_t)V * kVRow, 0.0);
    for (int v = 0; v < V; ++v) {
        const int cols[8] = {VC_PX, VC_PY, VC_W, VC_FR, VC_FWL, VC_FWLT, VC_FWR, VC_FWRT};
        for (int c = 0; c < 8; ++c) ps.vrow[(size_t)v * kVRow + c] = ps.vel[(size_t)cols[c] * V + v];
        ps.vrow[(size_t)v * kVRow + VR_A] = ps.aj[v];
        ps.vrow[(size_t)v * kVRow + VR_J] = ps.aj[V + v];
    }
    if ((int)t.alpha.size() < Nxe + 2 || (int)t.sbeta.size() < Nxe + 2) {
        err = "internal: recurrence table too short";
        return false;
    }
    const EqTab E(Nxe, Nye, t.K, p.Qx, p.Qy);
    ps.eqtab.assign(E.len, 0.0);
    for (int l = 0; l < Nxe + 2; ++l) {
        ps.eqtab[E.alpha + l] = t.alpha[l];
        ps.eqtab[E.sbeta + l] = t.sbeta[l];
        ps.eqtab[E.isbeta + l] = 1.0 / t.sbeta[l];
    }
    for (int l = 1; l < Nye + 2; ++l) ps.eqtab[E.invl + l] = 1.0 / l;
    for (int k = 0; k < t.K; ++k) {
        ps.eqtab[E.Yk + k] = t.Yk[k];
        ps.eqtab[E.Wk + k] = t.Wk[k];
    }
    for (int k = 0; k < (Nxe + 1) * p.Qx; ++k) ps.eqtab[E.hz + k] = t.hz[k];
    for (int k = 0; k < (Nye + 1) * p.Qy; ++k) ps.eqtab[E.He + k] = t.He[k];

    DevTables dummy{};
    size_t nd = 0, nf = 0;
    for (auto &pc : dpieces(ps, dummy)) nd += pad_d(pc.src->size());
    for (auto &pc : fpieces(ps, dummy)) nf += pad_f(pc.src->size());
    const size_t dbytes = nd * sizeof(double), fbytes = nf * sizeof(float);
    ps.blob.assign(dbytes + fbytes + ps.aj.size() * sizeof(int), 0);
    size_t off = 0;
    for (auto &pc : dpieces(ps, dummy)) {
        std::memcpy(ps.blob.data() + off * sizeof(double), pc.src->data(), pc.src->size() * sizeof(double));
        off += pad_d(pc.src->size());
    }
    off = 0;
    for (auto &pc : fpieces(ps, dummy)) {
        float *d = reinterpret_cast<float *>(ps.blob.data() + dbytes) + off;
        for (size_t k = 0; k < pc.src->size(); ++k) d[k] = (float)(*pc.src)[k];
        off += pad_f(pc.src->size());
    }
    std::memcpy(ps.blob.data() + dbytes + fbytes, ps.aj.data(), ps.aj.size() * sizeof(int));
    return true;
}

void bind_tables(const ProblemSetup &ps, const lbc_params &p, const void *dev, DevTables &T)
{
    const HostTables &t = ps.t;
    const char *base = static_cast<const char *>(dev);
    size_t off = 0;
    for (auto &pc : dpieces(ps, T)) {
        *pc.dst = reinterpret_cast<const double *>(base) + off;
        off += pad_d(pc.src->size());
    }
    const size_t dbytes = off * sizeof(double);
    off = 0;
    for (auto &pc : fpieces(ps, T)) {
        *pc.dst = reinterpret_cast<const float *>(base + dbytes) + off;
        off += pad_f(pc.src->size());
    }
    T.vel_aj = reinterpret_cast<const int *>(base + dbytes + off * sizeof(float));

    T.Nx = p.Nx;
    T.Nxp = (p.Nx + 31) / 32 * 32;
    T.Qx = p.Qx; T.Qy = p.Qy; T.Nxe = ps.Nxe; T.Nye = ps.Nye; T.K = t.K; T.V = t.V;
    T.ntile = (p.Nx + kTile - 1) / kTile;
    T.p0 = p.p0; T.dt = ps.dt; T.delta = p.delta; T.Pr = p.Pr; T.omega = p.omega;
    T.TL = p.T_left; T.TR = p.T_right; T.inL = ps.inL; T.inR = ps.inR;
    T.restOutL = ps.restOutL; T.restOutR = ps.restOutR;
    for (int k = 0; k < 10; ++k) {
        T.restP[k] = ps.restP[k];
        T.f_restP[k] = (float)ps.restP[k];
    }
    T.dsc[SC_NU] = p.delta * std::sqrt(2.0);
    T.dsc[SC_EXPO] = 1.0 - p.omega;
    T.dsc[SC_1MPR] = 1.0 - p.Pr;
    T.dsc[SC_IP0] = 1.0 / p.p0;
    T.dsc[SC_H0] = 1.0 / t.sbeta[0];
    T.dsc[SC_DT] = ps.dt;
    T.dsc[SC_IINL] = 1.0 / ps.inL;
    T.dsc[SC_IINR] = 1.0 / ps.inR;
    for (int k = 0; k < kNumSc; ++k) T.fsc[k] = (float)T.dsc[k];
}

// cuTensorMapEncodeTiled through the runtime's driver entry point (no -lcuda).
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

lbc_status encode_state_map(CUtensorMap *map, void *base, bool fp32, int V, int Nxp, int box_cols)
{
    static EncodeTiledFn fn = nullptr;
    if (!fn) {
        cudaDriverEntryPointQueryResult q;
        void *ptr = nullptr;
        cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault, &q);
        if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !ptr)
            return fail(LBC_ECUDA, "cuTensorMapEncodeTiled is not available from the driver");
        fn = reinterpret_cast<EncodeTiledFn>(ptr);
    }
    const size_t esz = fp32 ? 4 : 8;
    cuuint64_t dims[2] = {(cuuint64_t)Nxp, (cuuint64_t)(2 * V)};
    cuuint64_t strides[1] = {(cuuint64_t)Nxp * esz};
    cuuint32_t box[2] = {(cuuint32_t)box_cols, (cuuint32_t)kSubV};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = fn(map, fp32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 2, base, dims,
                    strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(LBC_ECUDA, "cuTensorMapEncodeTiled failed (code " + std::to_string((int)r) + ")");
    return LBC_OK;
}

// Velocity chunks per tile (multiples of the pipeline's kSubV rows, at most
// kMaxCluster chunks: they form one cluster): the count that minimises a wave
// model of the launch, waves x (rows per CTA + per-CTA overhead), with the
// clusters the device can hold at once.
lbc_status choose_launch_shape(bool fp32, DevTables &T)
{
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) return fail(LBC_ECUDA, "no CUDA device");
    cudaError_t e = fp32 ? configure_kernels<float>() : configure_kernels<double>();
    if (e != cudaSuccess) return fail(LBC_ECUDA, std::string("kernel attributes: ") + cudaGetErrorString(e));
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    const size_t eqs = fp32 ? equilibrium_smem_bytes<float>(T.Qx, T.Qy, T.Nxe, T.Nye, T.K)
                            : equilibrium_smem_bytes<double>(T.Qx, T.Qy, T.Nxe, T.Nye, T.K);
    if (eqs > (size_t)optin)
        return fail(LBC_EINVAL, "quadrature orders too large for the shared memory of one CTA (" +
                                    std::to_string(eqs) + " bytes)");
    const int subs = std::min((T.V + kSubV - 1) / kSubV, kMaxVChunk / kSubV);
    double best = 1e300;
    T.vchunk = T.nchunk = 0;
    for (int nsub = 1; nsub <= subs; ++nsub) {
        const int vch = nsub * kSubV, nch = (T.V + vch - 1) / vch;
        if (nch > kMaxCluster) continue;
        const size_t smem = fp32 ? stage_smem_bytes<float>(T.Qx, T.Qy, T.Nxe, T.Nye, T.K, vch)
                                 : stage_smem_bytes<double>(T.Qx, T.Qy, T.Nxe, T.Nye, T.K, vch);
        if (smem > (size_t)optin) continue;
        int ncl = 0;
        e = fp32 ? stage_active_clusters<float>(smem, nch, &ncl) : stage_active_clusters<double>(smem, nch, &ncl);
        if (e != cudaSuccess || ncl <= 0) {
            cudaGetLastError();   // an unschedulable cluster shape is not an error of the solver
            continue;
        }
        const double waves = std::ceil((double)T.ntile / ncl);
        const double cost = waves * (vch + 24.0);
        if (cost < best - 1e-9) { best = cost; T.vchunk = vch; T.nchunk = nch; }
    }
    if (T.nchunk == 0)
        return fail(LBC_EINVAL, "no schedulable cluster shape for a velocity set of " + std::to_string(T.V));
    return LBC_OK;
}

}  // namespace lbc

extern "C" {

const char *lbc_last_error(void) { return g_err.c_str(); }

lbc_status lbc_quadrature(int Q, int half_range, double *nodes, double *weights)
{
    if (!nodes || !weights) return fail(LBC_EINVAL, "nodes and weights must not be NULL");
    std::vector<double> z, w;
    bool ok = half_range ? half_range_rule(Q, z, w) : full_range_rule(Q, z, w);
    if (!ok) return fail(LBC_EINVAL, "Q must be in [1, 64]");
    std::copy(z.begin(), z.end(), nodes);
    std::copy(w.begin(), w.end(), weights);
    return LBC_OK;
}

lbc_status lbc_equilibrium(const lbc_params *params, double ux, double uy, double T, double *gx, double *gy)
{
    if (!params || !gx || !gy) return fail(LBC_EINVAL, "NULL argument");
    if (!(T > 0.0)) return fail(LBC_EINVAL, "T must be > 0");
    lbc_params p = *params;
    if (p.p0 == 0.0) p.p0 = 1.0;
    int Nxe, Nye;
    lbc_params q = p;
    if (q.Nx < 8) q.Nx = 8;   // grid-independent call: only the velocity-space fields matter
    lbc_status st = validate(q, Nxe, Nye);
    if (st != LBC_OK) return st;
    HostTables t;
    std::string err;
    if (!build_tables(p.Qx, p.Qy, Nxe, Nye, p.p0, t, err)) return fail(LBC_EINVAL, err);
    equilibrium_host(t, ux, uy, T, gx, gy);
    return LBC_OK;
}

lbc_status lbc_create(const lbc_params *params, void *cuda_stream, lbc_solver **out)
{
    if (!params || !out) return fail(LBC_EINVAL, "params and out must not be NULL");
    lbc_params p = *params;
    if (p.p0 == 0.0) p.p0 = 1.0;
    if (p.cfl == 0.0) p.cfl = 0.5;
    int Nxe, Nye;
    lbc_status st = validate(p, Nxe, Nye);
    if (st != LBC_OK) return st;

    lbc_solver *s = new (std::nothrow) lbc_solver();
    if (!s) return fail(LBC_ENOMEM, "host allocation failed");
    s->p = p;
    s->stream = static_cast<cudaStream_t>(cuda_stream);
    s->fp32 = p.precision == LBC_FP32_STATE;
    auto cleanup = [&](lbc_status code) {
        lbc_destroy(s);
        return code;
    };
    ProblemSetup ps;
    std::string err;
    if (!setup_problem(p, Nxe, Nye, ps, err)) return cleanup(fail(LBC_EINVAL, err));
    s->x = ps.x;
    s->frest = ps.frest;

    // ---- device tables (one allocation) and the launch shape ----
    cudaError_t e = cudaMallocAsync(&s->table_block, ps.blob.size(), s->stream);
    if (e != cudaSuccess) {
        set_error(std::string("cudaMallocAsync(tables): ") + cudaGetErrorString(e));
        return cleanup(e == cudaErrorMemoryAllocation ? LBC_ENOMEM : LBC_ECUDA);
    }
    e = cudaMemcpyAsync(s->table_block, ps.blob.data(), ps.blob.size(), cudaMemcpyHostToDevice, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);   // the pageable source must outlive the copy
    if (e != cudaSuccess) { set_error(std::string("table upload: ") + cudaGetErrorString(e)); return cleanup(LBC_ECUDA); }
    DevTables &T = s->T;
    bind_tables(ps, p, s->table_block, T);
    st = choose_launch_shape(s->fp32, T);
    if (st != LBC_OK) return cleanup(st);

    // ---- device state ----
    const int V = T.V;
    const size_t esz = s->fp32 ? sizeof(float) : sizeof(double);
    auto r256 = [](size_t x) { return (x + 255) / 256 * 256; };
    const size_t fbytes = r256(2 * (size_t)V * T.Nxp * esz);
    const size_t pbytes = r256((size_t)T.nchunk * kNumRaw * T.Nxp * esz);
    const size_t embytes = r256((size_t)T.Nxp * kEqM * esz);
    const size_t egbytes = r256((size_t)T.ntile * (2 * p.Qx + p.Qy) * kLanes * esz);
    const size_t rbytes = kResidRing * sizeof(unsigned long long);
    const size_t cbytes = 256;
    const size_t mbytes = r256((size_t)LBC_NMOM * T.Nxp * sizeof(double));
    const size_t sbytes = 3 * (fbytes + embytes + egbytes) + pbytes + rbytes + cbytes + mbytes;
    e = cudaMallocAsync(&s->state_block, sbytes, s->stream);
    if (e != cudaSuccess) {
        set_error(std::string("cudaMallocAsync(state): ") + cudaGetErrorString(e));
        return cleanup(e == cudaErrorMemoryAllocation ? LBC_ENOMEM : LBC_ECUDA);
    }
    e = cudaMemsetAsync(s->state_block, 0, sbytes, s->stream);
    if (e != cudaSuccess) { set_error(std::string("cudaMemsetAsync: ") + cudaGetErrorString(e)); return cleanup(LBC_ECUDA); }
    char *b = static_cast<char *>(s->state_block);
    for (int k = 0; k < 3; ++k) { s->S.F[k] = b; b += fbytes; }
    for (int k = 0; k < 3; ++k) { s->S.eqm[k] = b; b += embytes; }
    for (int k = 0; k < 3; ++k) { s->S.eqg[k] = b; b += egbytes; }
    s->S.part = b; b += pbytes;
    s->S.resid = reinterpret_cast<unsigned long long *>(b); b += rbytes;
    s->S.ctl = reinterpret_cast<Ctl *>(b); b += cbytes;
    s->S.mom_out = reinterpret_cast<double *>(b);

    e = cudaMallocHost(&s->h_resid, rbytes);
    if (e == cudaSuccess) e = cudaMallocHost(&s->h_ctl, sizeof(Ctl));
    if (e != cudaSuccess) {
        set_error(std::string("cudaMallocHost: ") + cudaGetErrorString(e));
        return cleanup(e == cudaErrorMemoryAllocation ? LBC_ENOMEM : LBC_ECUDA);
    }
    for (int k = 0; k < 3; ++k) {
        st = encode_state_map(&s->M.in[k], s->S.F[k], s->fp32, V, T.Nxp, kRowLen);
        if (st != LBC_OK) return cleanup(st);
    }
    st = encode_state_map(&s->M.f0, s->S.F[0], s->fp32, V, T.Nxp, kF0Len);
    if (st != LBC_OK) return cleanup(st);
    // The zeroed state is the rest Maxwellian (deviation 0) with zero moment partials;
    // build its stage data (moments and equilibrium factors) for the first stage.
    e = s->fp32 ? launch_tile_equilibrium<float>(T, s->S, 0, s->stream)
                : launch_tile_equilibrium<double>(T, s->S, 0, s->stream);
    if (e == cudaSuccess) e = launch_ctl_set(s->S.ctl, 0, 0, 0, s->stream);
    if (e != cudaSuccess) { set_error(std::string("init launch: ") + cudaGetErrorString(e)); return cleanup(LBC_ECUDA); }
    *out = s;
    return LBC_OK;
}

lbc_status lbc_step(lbc_solver *s, long nsteps)
{
    if (!s || nsteps < 0) return fail(LBC_EINVAL, "bad solver or nsteps");
    if (s->poisoned) return fail(LBC_ENONFINITE, "solver state is non-finite");
    long left = nsteps;
    while (left >= kGraphSteps) {
        lbc_status st = ensure_graph(s);
        if (st != LBC_OK) return st;
        LBC_CUDA_TRY(cudaGraphLaunch(s->graph, s->stream));
        left -= kGraphSteps;
    }
    if (left > 0) {
        LBC_CUDA_TRY(launch_steps(s, 0, (int)left, 0.0));
        LBC_CUDA_TRY(launch_ctl_bump(s->S.ctl, left, s->stream));
    }
    s->steps += nsteps;
    return LBC_OK;
}

lbc_status lbc_run_to_steady(lbc_solver *s, double residual, long max_steps, long *steps_done,
                             double *final_residual)
{
    if (!s || !(residual > 0.0) || max_steps < 0) return fail(LBC_EINVAL, "bad solver, residual or max_steps");
    if (s->poisoned) return fail(LBC_ENONFINITE, "solver state is non-finite");
    const long long start = s->steps;
    LBC_CUDA_TRY(launch_ctl_set(s->S.ctl, start, start, 0, s->stream));
    long done = 0;
    double last = INFINITY;
    bool converged = false;
    // chunks of up to kGraphSteps steps, each followed by a read-back of the residuals
    while (done < max_steps && !converged) {
        int k = (int)std::min<long>(kGraphSteps, max_steps - done);
        long long base = start + done;
        LBC_CUDA_TRY(launch_steps(s, 0, k, residual));
        LBC_CUDA_TRY(launch_ctl_bump(s->S.ctl, k, s->stream));
        LBC_CUDA_TRY(cudaMemcpyAsync(s->h_resid, s->S.resid, kResidRing * sizeof(unsigned long long),
                                     cudaMemcpyDeviceToHost, s->stream));
        LBC_CUDA_TRY(cudaMemcpyAsync(s->h_ctl, s->S.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s->stream));
        LBC_CUDA_TRY(cudaStreamSynchronize(s->stream));
        if (s->h_ctl->timeout) return fail(LBC_ETIMEOUT, "a bounded device wait gave up");
        if (s->h_ctl->nonfinite) {
            s->poisoned = true;
            return fail(LBC_ENONFINITE, "non-finite value in the state");
        }
        int taken = k;
        for (int i = 0; i < k; ++i) {
            unsigned long long bits = s->h_resid[(base + i) % kResidRing];
            double r;
            std::memcpy(&r, &bits, sizeof r);
            last = r;
            if (r < residual) { taken = i + 1; converged = true; break; }
        }
        done += taken;
    }
    s->steps = start + done;
    LBC_CUDA_TRY(launch_ctl_set(s->S.ctl, s->steps, s->steps, 0, s->stream));
    if (steps_done) *steps_done = done;
    if (final_residual) *final_residual = last;
    if (!converged) return fail(LBC_ENOTCONV, "max_steps reached before the residual threshold");
    return LBC_OK;
}

lbc_status lbc_moments(lbc_solver *s, double *out, double *x)
{
    if (!s || !out) return fail(LBC_EINVAL, "NULL argument");
    LBC_CUDA_TRY(s->fp32 ? launch_moments_partial<float>(s->T, s->S, 0, s->stream)
                         : launch_moments_partial<double>(s->T, s->S, 0, s->stream));
    LBC_CUDA_TRY(s->fp32 ? launch_finalize_moments<float>(s->T, s->S, s->stream)
                         : launch_finalize_moments<double>(s->T, s->S, s->stream));
    LBC_CUDA_TRY(cudaMemcpy2DAsync(out, s->p.Nx * sizeof(double), s->S.mom_out, s->T.Nxp * sizeof(double),
                                   s->p.Nx * sizeof(double), LBC_NMOM, cudaMemcpyDeviceToHost, s->stream));
    LBC_CUDA_TRY(cudaMemcpyAsync(s->h_ctl, s->S.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s->stream));
    LBC_CUDA_TRY(cudaStreamSynchronize(s->stream));
    if (x) std::copy(s->x.begin(), s->x.end(), x);
    if (s->h_ctl->timeout) return fail(LBC_ETIMEOUT, "a bounded device wait gave up");
    if (s->h_ctl->nonfinite) {
        s->poisoned = true;
        return fail(LBC_ENONFINITE, "non-finite value in the state");
    }
    return LBC_OK;
}

lbc_status lbc_get_state(lbc_solver *s, double *state)
{
    if (!s || !state) return fail(LBC_EINVAL, "NULL argument");
    const int V = s->T.V, Nx = s->T.Nx, Nxp = s->T.Nxp;
    const size_t esz = s->fp32 ? sizeof(float) : sizeof(double);
    std::vector<unsigned char> tmp(2 * (size_t)V * Nxp * esz);
    LBC_CUDA_TRY(cudaMemcpyAsync(tmp.data(), s->S.F[0], tmp.size(), cudaMemcpyDeviceToHost, s->stream));
    LBC_CUDA_TRY(cudaStreamSynchronize(s->stream));
    for (size_t r = 0; r < 2 * (size_t)V; ++r) {
        const double fr = s->frest[r % V];
        for (int c = 0; c < Nx; ++c)
            state[r * Nx + c] = fr + (s->fp32 ? (double)reinterpret_cast<float *>(tmp.data())[r * Nxp + c]
                                              : reinterpret_cast<double *>(tmp.data())[r * Nxp + c]);
    }
    if (s->h_ctl) {
        LBC_CUDA_TRY(cudaMemcpyAsync(s->h_ctl, s->S.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s->stream));
        LBC_CUDA_TRY(cudaStreamSynchronize(s->stream));
        if (s->h_ctl->timeout) return fail(LBC_ETIMEOUT, "a bounded device wait gave up");
    }
    return LBC_OK;
}

lbc_status lbc_set_state(lbc_solver *s, const double *state)
{
    if (!s || !state) return fail(LBC_EINVAL, "NULL argument");
    const int V = s->T.V, Nx = s->T.Nx, Nxp = s->T.Nxp;
    for (size_t i = 0; i < 2 * (size_t)V * Nx; ++i)
        if (!std::isfinite(state[i])) return fail(LBC_EINVAL, "state holds a NaN or Inf");
    const size_t esz = s->fp32 ? sizeof(float) : sizeof(double);
    std::vector<unsigned char> tmp(2 * (size_t)V * Nxp * esz, 0);
    for (size_t r = 0; r < 2 * (size_t)V; ++r) {
        const double fr = s->frest[r % V];
        for (int c = 0; c < Nx; ++c) {
            if (s->fp32) reinterpret_cast<float *>(tmp.data())[r * Nxp + c] = (float)(state[r * Nx + c] - fr);
            else reinterpret_cast<double *>(tmp.data())[r * Nxp + c] = state[r * Nx + c] - fr;
        }
    }
    LBC_CUDA_TRY(cudaMemcpyAsync(s->S.F[0], tmp.data(), tmp.size(), cudaMemcpyHostToDevice, s->stream));
    LBC_CUDA_TRY(s->fp32 ? launch_moments_partial<float>(s->T, s->S, 0, s->stream)
                         : launch_moments_partial<double>(s->T, s->S, 0, s->stream));
    LBC_CUDA_TRY(s->fp32 ? launch_tile_equilibrium<float>(s->T, s->S, 0, s->stream)
                         : launch_tile_equilibrium<double>(s->T, s->S, 0, s->stream));
    LBC_CUDA_TRY(cudaStreamSynchronize(s->stream));
    s->poisoned = false;
    return LBC_OK;
}

lbc_status lbc_info(const lbc_solver *s, int *Nx, int *V, double *dt, long *steps_taken)
{
    if (!s) return fail(LBC_EINVAL, "NULL solver");
    if (Nx) *Nx = s->T.Nx;
    if (V) *V = s->T.V;
    if (dt) *dt = s->T.dt;
    if (steps_taken) *steps_taken = (long)s->steps;
    return LBC_OK;
}

void lbc_destroy(lbc_solver *s)
{
    if (!s) return;
    if (s->graph) cudaGraphExecDestroy(s->graph);
    if (s->state_block) cudaFreeAsync(s->state_block, s->stream);
    if (s->table_block) cudaFreeAsync(s->table_block, s->stream);
    if (s->h_resid || s->h_ctl) cudaStreamSynchronize(s->stream);
    if (s->h_resid) cudaFreeHost(s->h_resid);
    if (s->h_ctl) cudaFreeHost(s->h_ctl);
    delete s;
}

}  // extern "C"
