// Instance pool (include/lbc.h, lbc_pool_*): Couette problems that join and
// leave while others run, stepped together by the batched stage kernel.
//
// Each admitted instance owns one stream-ordered allocation (its tables and
// state); the pool owns the slot-indexed descriptors, control blocks and the
// work list of (slot, tile) items. Admission is by device footprint against a
// byte budget. A run advances every active instance up to a step count with
// the early-stop threshold in each control block, so converged instances stop
// at their own step and are reported; the caller retires them and admits new
// ones between runs (continuous batching).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <numeric>
#include <string>
#include <vector>

#include "lbc_device.h"

using namespace lbc;

namespace {

#define POOL_TRY(call)                                                                       \
    do {                                                                                     \
        cudaError_t e_ = (call);                                                             \
        if (e_ != cudaSuccess) {                                                             \
            set_error(std::string(#call) + ": " + cudaGetErrorString(e_));                   \
            return e_ == cudaErrorMemoryAllocation ? LBC_ENOMEM : LBC_ECUDA;                 \
        }                                                                                    \
    } while (0)

struct Slot {
    bool used = false;
    bool reported = false;       // convergence already reported by a run
    lbc_params p{};
    std::vector<double> x, frest;
    long long steps = 0;
    double last_resid = INFINITY;
    void *block = nullptr;       // this instance's tables and state
    size_t bytes = 0;
    size_t smem = 0;             // stage-kernel shared memory of this instance
};

}  // namespace

struct lbc_pool {
    int cap = 0;                 // slots
    int max_tiles = 0;           // work-list capacity
    int cluster = 0;
    bool fp32 = false;
    size_t budget = 0, used = 0; // device bytes of the admitted instances
    cudaStream_t stream = nullptr;
    std::vector<Slot> slot;
    std::vector<Inst> inst;      // host images of the descriptors
    void *fixed = nullptr;       // descriptors, work list, slot list, control, residuals, staging
    Inst *d_inst = nullptr;
    int2 *d_work = nullptr;
    int *d_slots = nullptr;
    Ctl *d_ctl = nullptr;
    double *d_last = nullptr;
    double *d_io = nullptr;      // one instance's FP64 host-layout state
    size_t io_cap = 0;           // doubles
    int *d_bad = nullptr;
    Ctl *h_ctl = nullptr;        // pinned [cap]
    double *h_last = nullptr;    // pinned [cap]
    int *h_bad = nullptr;
    int nwork = 0;
    bool ext = false;            // some active instance uses the half channel or local steps
    std::vector<int> active;     // slots in the work list
};

namespace {

lbc_status check_slot(const lbc_pool *P, int s)
{
    if (!P) return fail(LBC_EINVAL, "NULL pool");
    if (s < 0 || s >= P->cap || !P->slot[s].used) return fail(LBC_EINVAL, "no instance in this slot");
    return LBC_OK;
}

// Work list and slot list of the active instances (longest CTAs first).
lbc_status rebuild_work(lbc_pool *P)
{
    std::vector<int> order;
    for (int s = 0; s < P->cap; ++s)
        if (P->slot[s].used) order.push_back(s);
    std::stable_sort(order.begin(), order.end(),
                     [&](int a, int b) { return P->inst[a].T.vchunk > P->inst[b].T.vchunk; });
    std::vector<int2> work;
    for (int s : order)
        for (int t = 0; t < P->inst[s].T.ntile; ++t) work.push_back(make_int2(s, t));
    if ((int)work.size() > P->max_tiles) return fail(LBC_ENOMEM, "pool work list full");
    P->nwork = (int)work.size();
    P->active = order;
    P->ext = false;
    for (int s : order) P->ext = P->ext || P->inst[s].T.half || P->inst[s].T.lts || P->inst[s].T.comp;
    // pageable sources: the copies are complete (staged) when cudaMemcpyAsync returns
    if (!work.empty())
        POOL_TRY(cudaMemcpyAsync(P->d_work, work.data(), work.size() * sizeof(int2), cudaMemcpyHostToDevice, P->stream));
    if (!order.empty())
        POOL_TRY(cudaMemcpyAsync(P->d_slots, order.data(), order.size() * sizeof(int), cudaMemcpyHostToDevice,
                                 P->stream));
    return LBC_OK;
}

template <typename R>
cudaError_t pool_steps(lbc_pool *P, long nsteps, size_t smem)
{
    for (long k = 0; k < nsteps; ++k)
        for (int stage = 0; stage < 3; ++stage) {
            cudaError_t e = launch_stage_batch<R>(P->d_inst, P->d_work, P->nwork, P->cluster, smem, stage, (int)k,
                                                  P->ext, kFormCluster, 0, P->stream);
            if (e != cudaSuccess) return e;
        }
    return launch_ctl_bump(P->d_ctl, P->cap, nsteps, P->stream);
}

}  // namespace

extern "C" {

lbc_status lbc_pool_create(int cluster, lbc_precision precision, size_t budget_bytes, int max_instances,
                           int max_tiles, void *cuda_stream, lbc_pool **out)
{
    if (!out || cluster < 1 || cluster > kMaxCluster || max_instances < 1 || max_tiles < 1)
        return fail(LBC_EINVAL, "need out, cluster in [1, 16], max_instances >= 1 and max_tiles >= 1");
    if (precision != LBC_FP64 && precision != LBC_FP32_STATE) return fail(LBC_EINVAL, "unknown precision");
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) return fail(LBC_ECUDA, "no CUDA device");
    lbc_pool *P = new (std::nothrow) lbc_pool();
    if (!P) return fail(LBC_ENOMEM, "host allocation failed");
    P->cap = max_instances;
    P->max_tiles = max_tiles;
    P->cluster = cluster;
    P->fp32 = precision == LBC_FP32_STATE;
    P->budget = budget_bytes;
    P->stream = static_cast<cudaStream_t>(cuda_stream);
    P->slot.resize(P->cap);
    P->inst.resize(P->cap);
    auto cleanup = [&](lbc_status code) {
        std::string msg = last_error();
        lbc_pool_destroy(P);
        set_error(msg);
        return code;
    };
    cudaError_t e = P->fp32 ? configure_kernels<float>() : configure_kernels<double>();
    if (e != cudaSuccess) return cleanup(fail(LBC_ECUDA, std::string("kernel attributes: ") + cudaGetErrorString(e)));
    const size_t o_inst = 0, o_work = o_inst + round256(P->cap * sizeof(Inst));
    const size_t o_slots = o_work + round256(P->max_tiles * sizeof(int2));
    const size_t o_ctl = o_slots + round256(P->cap * sizeof(int));
    const size_t o_last = o_ctl + round256(P->cap * sizeof(Ctl));
    const size_t o_bad = o_last + round256(P->cap * sizeof(double));
    const size_t bytes = o_bad + 256;
    e = cudaMallocAsync(&P->fixed, bytes, P->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(P->fixed, 0, bytes, P->stream);
    if (e != cudaSuccess) return cleanup(fail(LBC_ENOMEM, std::string("pool allocation: ") + cudaGetErrorString(e)));
    char *b = static_cast<char *>(P->fixed);
    P->d_inst = reinterpret_cast<Inst *>(b + o_inst);
    P->d_work = reinterpret_cast<int2 *>(b + o_work);
    P->d_slots = reinterpret_cast<int *>(b + o_slots);
    P->d_ctl = reinterpret_cast<Ctl *>(b + o_ctl);
    P->d_last = reinterpret_cast<double *>(b + o_last);
    P->d_bad = reinterpret_cast<int *>(b + o_bad);
    e = cudaMallocHost(&P->h_ctl, P->cap * sizeof(Ctl));
    if (e == cudaSuccess) e = cudaMallocHost(&P->h_last, P->cap * sizeof(double));
    if (e == cudaSuccess) e = cudaMallocHost(&P->h_bad, sizeof(int));
    if (e != cudaSuccess) return cleanup(fail(LBC_ENOMEM, std::string("cudaMallocHost: ") + cudaGetErrorString(e)));
    std::memset(P->h_ctl, 0, P->cap * sizeof(Ctl));
    *out = P;
    return LBC_OK;
}

lbc_status lbc_pool_footprint(const lbc_params *params, int cluster, size_t *bytes)
{
    if (!params || !bytes || cluster < 1 || cluster > kMaxCluster) return fail(LBC_EINVAL, "bad arguments");
    lbc_params p = *params;
    if (p.p0 == 0.0) p.p0 = 1.0;
    if (p.cfl == 0.0) p.cfl = 0.5;
    int Nxe, Nye;
    lbc_status st = validate(p, Nxe, Nye);
    if (st != LBC_OK) return st;
    ProblemSetup ps;
    std::string err;
    if (!setup_problem(p, Nxe, Nye, ps, err)) return fail(LBC_EINVAL, err);
    DevTables T{};
    bind_tables(ps, p, nullptr, T);
    *bytes = round256(ps.blob.size()) + StateSizes(T, p.precision == LBC_FP32_STATE).total;
    return LBC_OK;
}

lbc_status lbc_pool_add(lbc_pool *P, const lbc_params *params, int *slot_out)
{
    if (!P || !params || !slot_out) return fail(LBC_EINVAL, "NULL argument");
    lbc_params p = *params;
    if (p.p0 == 0.0) p.p0 = 1.0;
    if (p.cfl == 0.0) p.cfl = 0.5;
    int Nxe, Nye;
    lbc_status st = validate(p, Nxe, Nye);
    if (st != LBC_OK) return st;
    if ((p.precision == LBC_FP32_STATE) != P->fp32) return fail(LBC_EINVAL, "instance precision differs from the pool's");
    int s = 0;
    while (s < P->cap && P->slot[s].used) ++s;
    if (s == P->cap) return fail(LBC_ENOMEM, "no free slot in the pool");
    ProblemSetup ps;
    std::string err;
    if (!setup_problem(p, Nxe, Nye, ps, err)) return fail(LBC_EINVAL, err);
    Inst I{};
    bind_tables(ps, p, nullptr, I.T);   // sizes first; the table pointers are bound below
    I.T.nchunk = P->cluster;
    I.T.vchunk = chunk_rows(I.T.V, P->cluster);
    if (I.T.vchunk > kMaxVChunk) return fail(LBC_EINVAL, "velocity set too large for the pool's cluster size");
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    const size_t smem = stage_launch_smem(P->fp32, I.T);
    const size_t eqs = P->fp32 ? equilibrium_smem_bytes<float>(I.T.Qx, I.T.Qy, I.T.Nxe, I.T.Nye, I.T.K, I.T.tab_n)
                               : equilibrium_smem_bytes<double>(I.T.Qx, I.T.Qy, I.T.Nxe, I.T.Nye, I.T.K, I.T.tab_n);
    if (smem > (size_t)optin || eqs > (size_t)optin) return fail(LBC_EINVAL, "quadrature orders too large for one CTA");
    const StateSizes z(I.T, P->fp32);
    const size_t tbytes = round256(ps.blob.size());
    const size_t io = 2 * (size_t)I.T.V * I.T.Nx;
    const size_t need = tbytes + z.total;
    if (P->used + need > P->budget || fault_injected("admit")) return fail(LBC_ENOMEM, "pool budget exhausted");
    if ((long)P->nwork + I.T.ntile > P->max_tiles) return fail(LBC_ENOMEM, "pool work list full");
    if (io > P->io_cap) {   // the state staging (outside the budget) grows to the largest instance seen
        if (P->d_io) POOL_TRY(cudaFreeAsync(P->d_io, P->stream));
        P->d_io = nullptr;
        POOL_TRY(cudaMallocAsync(&P->d_io, io * sizeof(double), P->stream));
        P->io_cap = io;
    }
    void *block = nullptr;
    cudaError_t e = fault_injected("alloc") ? cudaErrorMemoryAllocation
                                            : cudaMallocAsync(&block, tbytes + z.total, P->stream);
    if (e != cudaSuccess) return fail(LBC_ENOMEM, std::string("instance allocation: ") + cudaGetErrorString(e));
    bind_tables(ps, p, block, I.T);
    I.T.nchunk = P->cluster;
    I.T.vchunk = chunk_rows(I.T.V, P->cluster);
    char *sb = static_cast<char *>(block) + tbytes;
    z.carve(sb, I.S);
    I.S.ctl = P->d_ctl + s;
    for (int k = 0; k < 3 && st == LBC_OK; ++k) st = encode_state_map(&I.M.in[k], I.S.F[k], P->fp32, I.T.V, I.T.Nxp, kRowLen,
                                                                 slot_rows(k, P->fp32));
    if (st == LBC_OK) st = encode_state_map(&I.M.f0, I.S.F[0], P->fp32, I.T.V, I.T.Nxp, kF0Len, kSubV);
    if (st != LBC_OK) {
        cudaFreeAsync(block, P->stream);
        return st;
    }
    // tables (pageable: staged before cudaMemcpyAsync returns), rest state, zero control
    e = cudaMemcpyAsync(block, ps.blob.data(), ps.blob.size(), cudaMemcpyHostToDevice, P->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(sb, 0, z.total, P->stream);
    Ctl zero{};
    if (e == cudaSuccess) e = cudaMemcpyAsync(P->d_ctl + s, &zero, sizeof(Ctl), cudaMemcpyHostToDevice, P->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(P->d_inst + s, &I, sizeof(Inst), cudaMemcpyHostToDevice, P->stream);
    if (e == cudaSuccess)
        e = P->fp32 ? launch_moments_partial<float>(I.T, I.S, 0, P->stream) : launch_moments_partial<double>(I.T, I.S, 0, P->stream);
    if (e == cudaSuccess)
        e = P->fp32 ? launch_tile_equilibrium<float>(I.T, I.S, 0, P->stream)
                    : launch_tile_equilibrium<double>(I.T, I.S, 0, P->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(P->stream);   // the host images above go away
    if (e != cudaSuccess) {
        cudaFreeAsync(block, P->stream);
        return fail(LBC_ECUDA, std::string("instance set-up: ") + cudaGetErrorString(e));
    }
    Slot &S = P->slot[s];
    S = Slot();
    S.used = true;
    S.p = p;
    S.x = ps.x;
    S.frest = ps.frest;
    S.block = block;
    S.bytes = tbytes + z.total;
    S.smem = smem;
    P->inst[s] = I;
    P->h_ctl[s] = zero;
    P->used += S.bytes;
    st = rebuild_work(P);
    if (st != LBC_OK) {
        lbc_pool_remove(P, s);
        return st;
    }
    *slot_out = s;
    return LBC_OK;
}

lbc_status lbc_pool_remove(lbc_pool *P, int s)
{
    lbc_status st = check_slot(P, s);
    if (st != LBC_OK) return st;
    Slot &S = P->slot[s];
    S.used = false;
    st = rebuild_work(P);   // drop its work items before the memory can be reused
    POOL_TRY(cudaFreeAsync(S.block, P->stream));
    P->used -= S.bytes;
    S = Slot();
    return st;
}

lbc_status lbc_pool_run(lbc_pool *P, double residual, long nsteps, int *finished, int *nfinished)
{
    NvtxRange nvtx_range("lbc_pool_run");
    if (!P || !(residual > 0.0) || nsteps < 0) return fail(LBC_EINVAL, "bad pool, residual or nsteps");
    if (nfinished) *nfinished = 0;
    const int na = (int)P->active.size();
    if (na == 0 || nsteps == 0) return LBC_OK;
    if (fault_injected("launch")) return fail(LBC_ECUDA, "stage launch: injected failure (LBC_FAULT=launch)");
    const int probe = fault_wait_polls(), site = fault_bounds_site();
    size_t smem = 0;
    for (int s : P->active) {
        Ctl &c = P->h_ctl[s];
        c.base = P->slot[s].steps;
        // an instance whose convergence was reported stays where it is: its first
        // check already sees the residual of its last step
        c.check_from = P->slot[s].reported ? P->slot[s].steps - 1 : P->slot[s].steps;
        c.stop_eps = residual;
        c.stop_step = 0;
        c.stopped = 0;
        c.probe = probe;
        if (site) c.bounds = site;
        smem = std::max(smem, P->slot[s].smem);
    }
    POOL_TRY(cudaMemcpyAsync(P->d_ctl, P->h_ctl, P->cap * sizeof(Ctl), cudaMemcpyHostToDevice, P->stream));
    POOL_TRY(P->fp32 ? pool_steps<float>(P, nsteps, smem) : pool_steps<double>(P, nsteps, smem));
    POOL_TRY(launch_last_residuals(P->d_inst, P->d_slots, na, P->d_last, P->stream));
    POOL_TRY(cudaMemcpyAsync(P->h_last, P->d_last, na * sizeof(double), cudaMemcpyDeviceToHost, P->stream));
    POOL_TRY(cudaMemcpyAsync(P->h_ctl, P->d_ctl, P->cap * sizeof(Ctl), cudaMemcpyDeviceToHost, P->stream));
    POOL_TRY(cudaStreamSynchronize(P->stream));
    int nf = 0;
    lbc_status st = LBC_OK;
    for (int k = 0; k < na; ++k) {
        const int s = P->active[k];
        Slot &S = P->slot[s];
        const Ctl &c = P->h_ctl[s];
        if (c.bounds && st == LBC_OK)
            st = fail(LBC_EBOUNDS, "instance " + std::to_string(s) + ": device index check failed: " +
                                       check_site_name(c.bounds));
        if (c.timeout && st == LBC_OK) st = fail(LBC_ETIMEOUT, "a bounded device wait gave up");
        if (c.nonfinite && st == LBC_OK) st = fail(LBC_ENONFINITE, "non-finite value in instance " + std::to_string(s));
        const long long start = S.steps;
        bool conv = false;
        if (c.stopped) {
            S.steps = c.stop_step;
            conv = true;
        } else {
            S.steps = start + nsteps;
            conv = P->h_last[k] < residual;
        }
        S.last_resid = P->h_last[k];
        if (conv && !S.reported) {
            S.reported = true;
            if (finished) finished[nf] = s;
            ++nf;
        }
    }
    if (nfinished) *nfinished = nf;
    return st;
}

lbc_status lbc_pool_info(const lbc_pool *P, int s, int *Nx, int *V, double *dt, long *steps_taken,
                         double *last_residual)
{
    lbc_status st = check_slot(P, s);
    if (st != LBC_OK) return st;
    const DevTables &T = P->inst[s].T;
    if (Nx) *Nx = T.Nx;
    if (V) *V = T.V;
    if (dt) *dt = T.dt;
    if (steps_taken) *steps_taken = (long)P->slot[s].steps;
    if (last_residual) *last_residual = P->slot[s].last_resid;
    return LBC_OK;
}

lbc_status lbc_pool_usage(const lbc_pool *P, size_t *used_bytes, int *instances, int *work_items)
{
    if (!P) return fail(LBC_EINVAL, "NULL pool");
    if (used_bytes) *used_bytes = P->used;
    if (instances) *instances = (int)P->active.size();
    if (work_items) *work_items = P->nwork;
    return LBC_OK;
}

lbc_status lbc_pool_moments(lbc_pool *P, int s, double *out, double *x)
{
    lbc_status st = check_slot(P, s);
    if (st != LBC_OK) return st;
    if (!out) return fail(LBC_EINVAL, "NULL argument");
    const Inst &I = P->inst[s];
    POOL_TRY(P->fp32 ? launch_moments_from_stage_data<float>(I.T, I.S, P->stream)
                     : launch_moments_from_stage_data<double>(I.T, I.S, P->stream));
    POOL_TRY(cudaMemcpy2DAsync(out, I.T.Nx * sizeof(double), I.S.mom_out, I.T.Nxp * sizeof(double),
                               I.T.Nx * sizeof(double), LBC_NMOM, cudaMemcpyDeviceToHost, P->stream));
    POOL_TRY(cudaStreamSynchronize(P->stream));
    if (x) std::copy(P->slot[s].x.begin(), P->slot[s].x.end(), x);
    return LBC_OK;
}

lbc_status lbc_pool_get_state(lbc_pool *P, int s, double *state)
{
    lbc_status st = check_slot(P, s);
    if (st != LBC_OK) return st;
    if (!state) return fail(LBC_EINVAL, "NULL argument");
    const Inst &I = P->inst[s];
    POOL_TRY(P->fp32 ? launch_state_out<float>(I.S.F[0], I.S.C, P->d_io, I.T, P->stream)
                     : launch_state_out<double>(I.S.F[0], nullptr, P->d_io, I.T, P->stream));
    POOL_TRY(cudaMemcpyAsync(state, P->d_io, 2 * (size_t)I.T.V * I.T.Nx * sizeof(double), cudaMemcpyDeviceToHost,
                             P->stream));
    POOL_TRY(cudaStreamSynchronize(P->stream));
    return LBC_OK;
}

void lbc_pool_destroy(lbc_pool *P)
{
    if (!P) return;
    for (Slot &S : P->slot)
        if (S.block) cudaFreeAsync(S.block, P->stream);
    if (P->d_io) cudaFreeAsync(P->d_io, P->stream);
    if (P->fixed) cudaFreeAsync(P->fixed, P->stream);
    if (P->h_ctl || P->h_last || P->h_bad) cudaStreamSynchronize(P->stream);
    if (P->h_ctl) cudaFreeHost(P->h_ctl);
    if (P->h_last) cudaFreeHost(P->h_last);
    if (P->h_bad) cudaFreeHost(P->h_bad);
    delete P;
}

}  // extern "C"
