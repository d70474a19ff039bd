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
    cudaStream_t stream = nullptr;
    bool fp32 = false;
    bool poisoned = false;
    long long steps = 0;             // completed steps
    std::vector<double> x;
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
            cudaError_t e = launch_stage<R>(s->T, s->S, st, rel0 + k, stop_eps, s->stream);
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
    double inL = 0, inR = 0;
    equilibrium_host(t, 0.0, p.u_left, p.T_left, gx.data(), gy.data());
    for (int v = 0; v < V; ++v) fwL[v] = gx[v / p.Qy] * gy[v % p.Qy];
    equilibrium_host(t, 0.0, p.u_right, p.T_right, gx.data(), gy.data());
    for (int v = 0; v < V; ++v) fwR[v] = gx[v / p.Qy] * gy[v % p.Qy];
    equilibrium_host(t, 0.0, 0.0, 1.0, gx.data(), gy.data());
    for (int v = 0; v < V; ++v) frest[v] = gx[v / p.Qy] * gy[v % p.Qy];
    for (int v = 0; v < V; ++v) {
        int a = v / p.Qy, j = v % p.Qy, i = a < p.Qx ? a : a - p.Qx;
        double px = (a < p.Qx ? 1.0 : -1.0) * p.p0 * t.zx[i], w = t.wx[i] * t.wy[j];
        if (px > 0) inL += px * w * fwL[v]; else inR += px * w * fwR[v];
    }

    // ---- device tables: one allocation ----
    std::vector<std::pair<const std::vector<double> *, const double **>> tabs;
    DevTables &T = s->T;
    T.Nx = Nx;
    T.Nxp = (Nx + 31) / 32 * 32;
    T.Qx = p.Qx; T.Qy = p.Qy; T.Nxe = Nxe; T.Nye = Nye; T.K = t.K; T.V = V;
    T.ntile = (Nx + kTileCells - 1) / kTileCells;
    // velocity chunks: aim at >= 2 CTAs per SM on 152 SMs, keep >= 64 velocities per chunk
    int want = std::max(1, (2 * 152 + T.ntile - 1) / T.ntile);
    int maxchunks = std::max(1, V / 64);
    T.nchunk = std::min(want, maxchunks);
    T.vchunk = (V + T.nchunk - 1) / T.nchunk;
    T.nchunk = (V + T.vchunk - 1) / T.vchunk;
    T.p0 = p.p0; T.dt = dt; T.delta = p.delta; T.Pr = p.Pr; T.omega = p.omega;
    T.TL = p.T_left; T.TR = p.T_right; T.inL = inL; T.inR = inR;

    struct Piece { const std::vector<double> *src; const double **dst; };
    std::vector<double> wall_L = fwL, wall_R = fwR, rest = frest;
    Piece pieces[] = {
        {&inv_jdeta, &T.inv_jdeta}, {&t.zx, &T.zx}, {&t.wx, &T.wx}, {&t.yy, &T.yy}, {&t.wy, &T.wy},
        {&t.alpha, &T.alpha}, {&t.sbeta, &T.sbeta}, {&t.hz, &T.hz}, {&t.Yk, &T.Yk}, {&t.Wk, &T.Wk},
        {&t.He, &T.He}, {&wall_L, &T.fwL}, {&wall_R, &T.fwR}, {&rest, &T.frest},
    };
    size_t total = 0;
    for (auto &pc : pieces) total += (pc.src->size() + 31) / 32 * 32;
    std::vector<double> host(total, 0.0);
    size_t off = 0;
    std::vector<size_t> offs;
    for (auto &pc : pieces) {
        std::copy(pc.src->begin(), pc.src->end(), host.begin() + off);
        offs.push_back(off);
        off += (pc.src->size() + 31) / 32 * 32;
    }
    auto cleanup = [&](lbc_status code) {
        lbc_destroy(s);
        return code;
    };
    cudaError_t e = cudaMallocAsync(&s->table_block, total * sizeof(double), s->stream);
    if (e != cudaSuccess) {
        set_error(std::string("cudaMallocAsync(tables): ") + cudaGetErrorString(e));
        return cleanup(e == cudaErrorMemoryAllocation ? LBC_ENOMEM : LBC_ECUDA);
    }
    e = cudaMemcpyAsync(s->table_block, host.data(), total * sizeof(double), cudaMemcpyHostToDevice, s->stream);
    if (e != cudaSuccess) { set_error(std::string("cudaMemcpyAsync(tables): ") + cudaGetErrorString(e)); return cleanup(LBC_ECUDA); }
    for (size_t k = 0; k < sizeof(pieces) / sizeof(pieces[0]); ++k)
        *pieces[k].dst = static_cast<const double *>(s->table_block) + offs[k];

    // ---- device state ----
    const size_t esz = s->fp32 ? sizeof(float) : sizeof(double);
    const size_t fbytes = (2 * (size_t)V * T.Nxp * esz + 255) / 256 * 256;
    const size_t pbytes = ((size_t)T.nchunk * kNumRaw * T.Nxp * sizeof(double) + 255) / 256 * 256;
    const size_t shbytes = (2 * (size_t)T.Nxp * sizeof(double) + 255) / 256 * 256;
    const size_t rbytes = kResidRing * sizeof(unsigned long long);
    const size_t cbytes = 256;
    const size_t mbytes = ((size_t)LBC_NMOM * T.Nxp * sizeof(double) + 255) / 256 * 256;
    const size_t sbytes = 3 * (fbytes + pbytes + shbytes) + rbytes + cbytes + mbytes;
    e = cudaMallocAsync(&s->state_block, sbytes, s->stream);
    if (e != cudaSuccess) {
        set_error(std::string("cudaMallocAsync(state): ") + cudaGetErrorString(e));
        return cleanup(e == cudaErrorMemoryAllocation ? LBC_ENOMEM : LBC_ECUDA);
    }
    e = cudaMemsetAsync(s->state_block, 0, sbytes, s->stream);
    if (e != cudaSuccess) { set_error(std::string("cudaMemsetAsync: ") + cudaGetErrorString(e)); return cleanup(LBC_ECUDA); }
    char *b = static_cast<char *>(s->state_block);
    for (int k = 0; k < 3; ++k) { s->S.F[k] = b; b += fbytes; }
    for (int k = 0; k < 3; ++k) { s->S.part[k] = reinterpret_cast<double *>(b); b += pbytes; }
    for (int k = 0; k < 3; ++k) { s->S.shift[k] = reinterpret_cast<double *>(b); b += shbytes; }
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
    e = s->fp32 ? launch_init_rest<float>(T, s->S, s->stream) : launch_init_rest<double>(T, s->S, s->stream);
    if (e == cudaSuccess)
        e = s->fp32 ? launch_moments_partial<float>(T, s->S, 0, s->stream)
                    : launch_moments_partial<double>(T, s->S, 0, s->stream);
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
    LBC_CUDA_TRY(launch_finalize_moments(s->T, s->S, 0, s->stream));
    LBC_CUDA_TRY(cudaMemcpy2DAsync(out, s->p.Nx * sizeof(double), s->S.mom_out, s->T.Nxp * sizeof(double),
                                   s->p.Nx * sizeof(double), LBC_NMOM, cudaMemcpyDeviceToHost, s->stream));
    LBC_CUDA_TRY(cudaMemcpyAsync(s->h_ctl, s->S.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s->stream));
    LBC_CUDA_TRY(cudaStreamSynchronize(s->stream));
    if (x) std::copy(s->x.begin(), s->x.end(), x);
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
    for (size_t r = 0; r < 2 * (size_t)V; ++r)
        for (int c = 0; c < Nx; ++c)
            state[r * Nx + c] = s->fp32 ? (double)reinterpret_cast<float *>(tmp.data())[r * Nxp + c]
                                        : reinterpret_cast<double *>(tmp.data())[r * Nxp + c];
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
    for (size_t r = 0; r < 2 * (size_t)V; ++r)
        for (int c = 0; c < Nx; ++c) {
            if (s->fp32) reinterpret_cast<float *>(tmp.data())[r * Nxp + c] = (float)state[r * Nx + c];
            else reinterpret_cast<double *>(tmp.data())[r * Nxp + c] = state[r * Nx + c];
        }
    LBC_CUDA_TRY(cudaMemcpyAsync(s->S.F[0], tmp.data(), tmp.size(), cudaMemcpyHostToDevice, s->stream));
    LBC_CUDA_TRY(s->fp32 ? launch_moments_partial<float>(s->T, s->S, 0, s->stream)
                         : launch_moments_partial<double>(s->T, s->S, 0, s->stream));
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
