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

int num_sms()
{
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return 152;
    return n > 0 ? n : 152;
}

// CTAs of the stage kernel resident per SM, from registers and shared memory.
int resident_ctas(bool fp32, int Qx, int Qy, int N, int Ny, int K, int vchunk)
{
    cudaFuncAttributes fa;
    cudaError_t e = fp32 ? stage_kernel_attributes<float>(&fa) : stage_kernel_attributes<double>(&fa);
    int dev = 0, smem_sm = 0, regs_sm = 65536;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev);
    size_t smem = fp32 ? stage_smem_bytes<float>(Qx, Qy, N, Ny, K, vchunk)
                       : stage_smem_bytes<double>(Qx, Qy, N, Ny, K, vchunk);
    int by_regs = e == cudaSuccess && fa.numRegs > 0 ? regs_sm / (fa.numRegs * kThreads) : 2;
    int by_smem = smem_sm > 0 ? (int)(smem_sm / (smem + 1024)) : 2;
    return std::max(1, std::min(by_regs, by_smem));
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
    std::string err;
    if (!build_tables(p.Qx, p.Qy, Nxe, Nye, p.p0, s->tab, err)) {
        delete s;
        return fail(LBC_EINVAL, err);
    }
    const HostTables &t = s->tab;
    const int V = t.V, Nx = p.Nx;
    std::vector<double> inv_jdeta;
    double deta, min_jdeta;
    make_grid(Nx, p.stretch_A, s->x, inv_jdeta, deta, min_jdeta);

    // time step: CFL on the smallest cell, and half the smallest relaxation time
    double zmax = t.zx.back() * p.p0;
    double dt = p.dt > 0 ? p.dt : p.cfl * min_jdeta / zmax;
    if (p.dt <= 0 && p.delta > 0) {
        for (double Tw : {1.0, p.T_left, p.T_right}) {
            double tau = std::pow(Tw, p.omega - 1.0) / (p.delta * std::sqrt(2.0));
            dt = std::min(dt, 0.5 * tau);
        }
    }

    // wall Maxwellians (unit density) and incoming unit fluxes; rest Maxwellian
    std::vector<double> gx(2 * p.Qx), gy(p.Qy), fwL(V), fwR(V), frest(V);
    double inL = 0, inR = 0, restOutL = 0, restOutR = 0, restP[10] = {0};
    equilibrium_host(t, 0.0, p.u_left, p.T_left, gx.data(), gy.data());
    for (int v = 0; v < V; ++v) fwL[v] = gx[v / p.Qy] * gy[v % p.Qy];
    equilibrium_host(t, 0.0, p.u_right, p.T_right, gx.data(), gy.data());
    for (int v = 0; v < V; ++v) fwR[v] = gx[v / p.Qy] * gy[v % p.Qy];
    equilibrium_host(t, 0.0, 0.0, 1.0, gx.data(), gy.data());
    for (int v = 0; v < V; ++v) frest[v] = gx[v / p.Qy] * gy[v % p.Qy];
    for (int v = 0; v < V; ++v) {
        int a = v / p.Qy, j = v % p.Qy, i = a < p.Qx ? a : a - p.Qx;
        double px = (a < p.Qx ? 1.0 : -1.0) * p.p0 * t.zx[i], py = p.p0 * t.yy[j], w = t.wx[i] * t.wy[j];
        if (px > 0) { inL += px * w * fwL[v]; restOutR += px * w * frest[v]; }
        else        { inR += px * w * fwR[v]; restOutL += px * w * frest[v]; }
        const double f = w * frest[v];
        const double pw[10] = {1, px, py, px * px, px * py, py * py, px * px * px, px * px * py, px * py * py,
                               py * py * py};
        for (int k = 0; k < 10; ++k) restP[k] += pw[k] * f;
    }
    s->frest = frest;

    // ---- device tables: one allocation (FP64 block, then FP32 copies) ----
    DevTables &T = s->T;
    T.Nx = Nx;
    T.Nxp = (Nx + 31) / 32 * 32;
    T.Qx = p.Qx; T.Qy = p.Qy; T.Nxe = Nxe; T.Nye = Nye; T.K = t.K; T.V = V;
    T.ntile = (Nx + kTile - 1) / kTile;
    // velocity chunks (multiples of the pipeline's kSubV rows): pick the count
    // that minimises a wave model of the launch, waves x (rows per CTA +
    // per-CTA overhead), with the resident CTAs per SM of this kernel
    {
        const int sms = num_sms(), subs = std::min((V + kSubV - 1) / kSubV, kMaxVChunk / kSubV);
        double best = 1e300;
        for (int nsub = 1; nsub <= subs; ++nsub) {
            int vch = nsub * kSubV, nch = (V + vch - 1) / vch;
            const int slots = std::max(1, sms * resident_ctas(s->fp32, p.Qx, p.Qy, Nxe, Nye, t.K, vch));
            double waves = std::ceil((double)T.ntile * nch / slots);
            double cost = waves * (vch + 24.0);
            if (cost < best - 1e-9) { best = cost; T.vchunk = vch; T.nchunk = nch; }
        }
    }
    T.p0 = p.p0; T.dt = dt; T.delta = p.delta; T.Pr = p.Pr; T.omega = p.omega;
    T.TL = p.T_left; T.TR = p.T_right; T.inL = inL; T.inR = inR;
    T.restOutL = restOutL; T.restOutR = restOutR;
    for (int k = 0; k < 10; ++k) T.restP[k] = restP[k];

    std::vector<double> vel((size_t)kVelCols * V);
    std::vector<double> aj(2 * (size_t)V);   // stored as doubles here, converted to int below
    for (int v = 0; v < V; ++v) {
        int a = v / p.Qy, j = v % p.Qy, i = a < p.Qx ? a : a - p.Qx;
        vel[VC_PX * V + v] = (a < p.Qx ? 1.0 : -1.0) * p.p0 * t.zx[i];
        vel[VC_PY * V + v] = p.p0 * t.yy[j];
        vel[VC_W * V + v] = t.wx[i] * t.wy[j];
        vel[VC_FR * V + v] = frest[v];
        vel[VC_FWL * V + v] = fwL[v];
        vel[VC_FWLT * V + v] = p.T_left * fwL[v];
        vel[VC_FWR * V + v] = fwR[v];
        vel[VC_FWRT * V + v] = p.T_right * fwR[v];
        aj[v] = a;
        aj[V + v] = j;
    }
    struct Piece { const std::vector<double> *src; const double **dst; };
    Piece pieces[] = {
        {&inv_jdeta, &T.inv_jdeta}, {&t.zx, &T.zx}, {&t.wx, &T.wx}, {&t.yy, &T.yy}, {&t.wy, &T.wy},
        {&t.alpha, &T.alpha}, {&t.sbeta, &T.sbeta}, {&t.hz, &T.hz}, {&t.Yk, &T.Yk}, {&t.Wk, &T.Wk},
        {&t.He, &T.He}, {&fwL, &T.fwL}, {&fwR, &T.fwR}, {&frest, &T.frest}, {&vel, &T.d_vel},
    };
    std::vector<double> isb(t.sbeta.size()), invl(kMaxQ + 2);
    for (size_t k = 0; k < isb.size(); ++k) isb[k] = 1.0 / t.sbeta[k];
    for (int l = 0; l < kMaxQ + 2; ++l) invl[l] = l ? 1.0 / l : 0.0;
    struct FPiece { const std::vector<double> *src; const float **dst; };
    FPiece fpieces[] = {
        {&t.hz, &T.f_hz}, {&t.He, &T.f_He}, {&t.alpha, &T.f_alpha}, {&isb, &T.f_isbeta}, {&t.sbeta, &T.f_sbeta},
        {&t.Yk, &T.f_Yk}, {&t.Wk, &T.f_Wk}, {&invl, &T.f_inv_l}, {&vel, &T.f_vel}, {&inv_jdeta, &T.f_inv_jdeta},
        {&aj, reinterpret_cast<const float **>(&T.vel_aj)},
    };
    size_t total = 0;   // in doubles
    for (auto &pc : pieces) total += (pc.src->size() + 31) / 32 * 32;
    size_t ftotal = 0;  // in floats
    for (auto &pc : fpieces) ftotal += (pc.src->size() + 63) / 64 * 64;
    const size_t dbytes = total * sizeof(double), bytes = dbytes + ftotal * sizeof(float);
    std::vector<unsigned char> host(bytes, 0);
    std::vector<size_t> offs, foffs;
    size_t off = 0;
    for (auto &pc : pieces) {
        std::memcpy(host.data() + off * sizeof(double), pc.src->data(), pc.src->size() * sizeof(double));
        offs.push_back(off);
        off += (pc.src->size() + 31) / 32 * 32;
    }
    off = 0;
    for (auto &pc : fpieces) {
        float *dst = reinterpret_cast<float *>(host.data() + dbytes) + off;
        if (pc.src == &aj) {   // integer table shares the 4-byte block
            int *di = reinterpret_cast<int *>(dst);
            for (size_t k = 0; k < pc.src->size(); ++k) di[k] = (int)(*pc.src)[k];
        } else {
            for (size_t k = 0; k < pc.src->size(); ++k) dst[k] = (float)(*pc.src)[k];
        }
        foffs.push_back(off);
        off += (pc.src->size() + 63) / 64 * 64;
    }
    auto cleanup = [&](lbc_status code) {
        lbc_destroy(s);
        return code;
    };
    cudaError_t e = cudaMallocAsync(&s->table_block, bytes, s->stream);
    if (e != cudaSuccess) {
        set_error(std::string("cudaMallocAsync(tables): ") + cudaGetErrorString(e));
        return cleanup(e == cudaErrorMemoryAllocation ? LBC_ENOMEM : LBC_ECUDA);
    }
    e = cudaMemcpyAsync(s->table_block, host.data(), bytes, cudaMemcpyHostToDevice, s->stream);
    if (e != cudaSuccess) { set_error(std::string("cudaMemcpyAsync(tables): ") + cudaGetErrorString(e)); return cleanup(LBC_ECUDA); }
    e = cudaStreamSynchronize(s->stream);   // the pageable host copy must finish before `host` goes away
    if (e != cudaSuccess) { set_error(std::string("table upload: ") + cudaGetErrorString(e)); return cleanup(LBC_ECUDA); }
    for (size_t k = 0; k < sizeof(pieces) / sizeof(pieces[0]); ++k)
        *pieces[k].dst = static_cast<const double *>(s->table_block) + offs[k];
    for (size_t k = 0; k < sizeof(fpieces) / sizeof(fpieces[0]); ++k)
        *fpieces[k].dst = reinterpret_cast<const float *>(static_cast<const char *>(s->table_block) + dbytes) + foffs[k];

    // ---- device state ----
    const size_t esz = s->fp32 ? sizeof(float) : sizeof(double);
    auto r256 = [](size_t x) { return (x + 255) / 256 * 256; };
    const size_t fbytes = r256(2 * (size_t)V * T.Nxp * esz);
    const size_t pbytes = r256((size_t)T.nchunk * kNumRaw * T.Nxp * esz);
    const size_t shbytes = r256(2 * (size_t)T.Nxp * esz);
    const size_t embytes = r256((size_t)T.Nxp * kEqM * esz);
    const size_t egbytes = r256((size_t)T.ntile * (2 * p.Qx + p.Qy) * kLanes * esz);
    const size_t cnbytes = r256((size_t)T.ntile * sizeof(int));
    const size_t rbytes = kResidRing * sizeof(unsigned long long);
    const size_t cbytes = 256;
    const size_t mbytes = r256((size_t)LBC_NMOM * T.Nxp * sizeof(double));
    const size_t sbytes = 3 * (fbytes + pbytes + shbytes + embytes + egbytes + cnbytes) + rbytes + cbytes + mbytes;
    e = cudaMallocAsync(&s->state_block, sbytes, s->stream);
    if (e != cudaSuccess) {
        set_error(std::string("cudaMallocAsync(state): ") + cudaGetErrorString(e));
        return cleanup(e == cudaErrorMemoryAllocation ? LBC_ENOMEM : LBC_ECUDA);
    }
    e = cudaMemsetAsync(s->state_block, 0, sbytes, s->stream);
    if (e != cudaSuccess) { set_error(std::string("cudaMemsetAsync: ") + cudaGetErrorString(e)); return cleanup(LBC_ECUDA); }
    char *b = static_cast<char *>(s->state_block);
    for (int k = 0; k < 3; ++k) { s->S.F[k] = b; b += fbytes; }
    for (int k = 0; k < 3; ++k) { s->S.part[k] = b; b += pbytes; }
    for (int k = 0; k < 3; ++k) { s->S.shift[k] = b; b += shbytes; }
    for (int k = 0; k < 3; ++k) { s->S.eqm[k] = b; b += embytes; }
    for (int k = 0; k < 3; ++k) { s->S.eqg[k] = b; b += egbytes; }
    for (int k = 0; k < 3; ++k) { s->S.count[k] = reinterpret_cast<int *>(b); b += cnbytes; }
    s->S.resid = reinterpret_cast<unsigned long long *>(b); b += rbytes;
    s->S.ctl = reinterpret_cast<Ctl *>(b); b += cbytes;
    s->S.mom_out = reinterpret_cast<double *>(b);

    e = cudaMallocHost(&s->h_resid, rbytes);
    if (e == cudaSuccess) e = cudaMallocHost(&s->h_ctl, sizeof(Ctl));
    if (e != cudaSuccess) {
        set_error(std::string("cudaMallocHost: ") + cudaGetErrorString(e));
        return cleanup(e == cudaErrorMemoryAllocation ? LBC_ENOMEM : LBC_ECUDA);
    }

    e = s->fp32 ? configure_kernels<float>() : configure_kernels<double>();
    if (e != cudaSuccess) { set_error(std::string("kernel attributes: ") + cudaGetErrorString(e)); return cleanup(LBC_ECUDA); }
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
    LBC_CUDA_TRY(s->fp32 ? launch_finalize_moments<float>(s->T, s->S, 0, s->stream)
                         : launch_finalize_moments<double>(s->T, s->S, 0, s->stream));
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
