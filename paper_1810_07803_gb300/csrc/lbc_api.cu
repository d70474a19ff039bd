// C ABI of the solver (include/lbc.h): batches of Couette instances and the
// single-instance solver built on them -- device memory, stepping through
// CUDA graphs, run-to-steady, moments and state I/O.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <numeric>
#include <string>
#include <vector>

#include "lbc_device.h"
#include "lbc_stall.h"

using namespace lbc;

namespace {

constexpr int kGraphSteps = 64;   // RK-3 steps captured per CUDA graph

#define LBC_CUDA_TRY(call)                                                                   \
    do {                                                                                     \
        cudaError_t e_ = (call);                                                             \
        if (e_ != cudaSuccess) {                                                             \
            set_error(std::string(#call) + ": " + cudaGetErrorString(e_));                   \
            return e_ == cudaErrorMemoryAllocation ? LBC_ENOMEM : LBC_ECUDA;                 \
        }                                                                                    \
    } while (0)

struct InstHost {
    lbc_params p{};
    std::vector<double> x;       // node positions
    std::vector<double> frest;   // weight-divided rest Maxwellian per velocity (state origin)
    long long steps = 0;         // completed steps
};

size_t r256(size_t x) { return round256(x); }

}  // namespace

struct lbc_batch {
    int n = 0;
    bool fp32 = false;
    bool single = false;          // one instance: the stage kernel with the descriptor as a parameter
    int cluster = 0;              // chunk CTAs per tile
    size_t smem = 0;              // dynamic shared memory of a stage launch
    cudaStream_t stream = nullptr;
    std::vector<InstHost> ih;
    std::vector<Inst> inst;       // host images of the device descriptors
    Inst *d_inst = nullptr;       // [n] in table_block
    int2 *d_work = nullptr;       // [nwork] (instance, tile), longest CTAs first
    int nwork = 0;
    void *table_block = nullptr;  // tables of every instance, descriptors, work list
    void *state_block = nullptr;  // states, stage data, partials, residual rings, control
    Ctl *d_ctl = nullptr;         // [n]
    double *d_last = nullptr;     // [n] last residual of each instance
    double *d_io = nullptr;       // staging of one instance's FP64 host-layout state
    int *d_bad = nullptr;         // set by the state upload when a value is not finite
    Ctl *h_ctl = nullptr;         // pinned [n]
    double *h_last = nullptr;     // pinned [n]
    int *h_bad = nullptr;         // pinned
    bool steady_mode = false;     // the device control blocks hold run-to-steady settings
    long stall_window = 0;        // run-to-steady stall rule (lbc_batch_set_stall_window); 0: off
    bool poisoned = false;        // some instance holds a NaN/Inf
    bool solo = false;            // batch kernel form without clusters: solo (the tile's last CTA builds the
                                  // node data) or, with split, split (a node-step launch builds it)
    bool split = false;
    bool full = false;            // chunks of 256 rows (choose_full_chunk_shape)
    size_t node_smem = 0;         // split form: dynamic shared memory of the node-step launch
    bool timed_out = false;       // a bounded device wait gave up: stepping is refused until set_state
    int bounds_site = 0;          // range-checked build: a device index check failed (refused the same way)
    cudaGraphExec_t graph = nullptr;
    bool ext = false;             // some instance uses the half channel or local steps
    bool persistent = false;      // steps run as the persistent form (one launch per group of steps)
    int pclusters = 0;            // clusters of a persistent launch (all resident)
    unsigned *d_cnt = nullptr;    // persistent form's counters: kPersistHdr + nwork + n
    size_t io_elems = 0;          // doubles of the largest instance's host-layout state
    // lbc_batch_set_states: a second staging buffer and a copy stream, so that the upload of
    // one instance overlaps the conversion and stage data of the previous one (made at first use)
    double *d_io2 = nullptr;
    cudaStream_t copy_stream = nullptr;
    cudaEvent_t ev_start = nullptr, ev_copied[2] = {nullptr, nullptr}, ev_free[2] = {nullptr, nullptr};
};

struct lbc_solver {
    lbc_batch *b = nullptr;
};

namespace {

int kernel_form(const lbc_batch *b) { return b->solo ? (b->split ? kFormSplit : kFormSolo) : kFormCluster; }

template <typename R>
cudaError_t launch_steps_t(lbc_batch *b, int nsteps, cudaStream_t st)
{
    for (int k = 0; k < nsteps; ++k)
        for (int stage = 0; stage < 3; ++stage) {
            cudaError_t e = b->single ? launch_stage<R>(b->inst[0], b->smem, stage, k, st)
                                      : launch_stage_batch<R>(b->d_inst, b->d_work, b->nwork, b->cluster, b->smem,
                                                              stage, k, b->ext, kernel_form(b), b->node_smem, st);
            if (e != cudaSuccess) return e;
        }
    return cudaSuccess;
}

// nsteps RK-3 steps of every instance, then the step counters.
cudaError_t launch_steps(lbc_batch *b, int nsteps, cudaStream_t st)
{
    cudaError_t e;
    if (b->persistent)
        e = b->fp32 ? launch_persistent<float>(b->d_inst, b->d_work, b->nwork, b->n, b->cluster, b->pclusters, b->smem,
                                               nsteps, b->ext, b->d_cnt, st)
                    : launch_persistent<double>(b->d_inst, b->d_work, b->nwork, b->n, b->cluster, b->pclusters,
                                                b->smem, nsteps, b->ext, b->d_cnt, st);
    else
        e = b->fp32 ? launch_steps_t<float>(b, nsteps, st) : launch_steps_t<double>(b, nsteps, st);
    if (e == cudaSuccess) e = launch_ctl_bump(b->d_ctl, b->n, nsteps, st);
    return e;
}

// kGraphSteps steps and the counter bump captured once; replayed by step and run-to-steady.
lbc_status ensure_graph(lbc_batch *b)
{
    if (b->graph) return LBC_OK;
    cudaStream_t cap;
    LBC_CUDA_TRY(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
    cudaGraph_t g;
    cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        e = launch_steps(b, kGraphSteps, cap);
        cudaError_t e2 = cudaStreamEndCapture(cap, &g);
        if (e == cudaSuccess) e = e2;
    }
    if (e == cudaSuccess) {
        e = cudaGraphInstantiate(&b->graph, g, 0);
        cudaGraphDestroy(g);
    }
    cudaStreamDestroy(cap);
    if (e != cudaSuccess) return fail(LBC_ECUDA, std::string("graph capture: ") + cudaGetErrorString(e));
    return LBC_OK;
}

lbc_status run_steps(lbc_batch *b, long nsteps)
{
    if (b->bounds_site)
        return fail(LBC_EBOUNDS, std::string("a device index check failed earlier (") + check_site_name(b->bounds_site) +
                                     "); set a state to continue");
    if (b->timed_out) return fail(LBC_ETIMEOUT, "a bounded device wait gave up earlier; set a state to continue");
    if (fault_injected("launch")) return fail(LBC_ECUDA, "stage launch: injected failure (LBC_FAULT=launch)");
    while (nsteps >= kGraphSteps) {
        lbc_status st = ensure_graph(b);
        if (st != LBC_OK) return st;
        NvtxRange nvtx_range("graph launch (64 steps)");
        LBC_CUDA_TRY(cudaGraphLaunch(b->graph, b->stream));
        nsteps -= kGraphSteps;
    }
    if (nsteps > 0) LBC_CUDA_TRY(launch_steps(b, (int)nsteps, b->stream));
    return LBC_OK;
}

lbc_status upload_ctl(lbc_batch *b, int first, int count)
{
    const int probe = fault_wait_polls(), site = fault_bounds_site();
    for (int k = first; k < first + count; ++k) {
        b->h_ctl[k].probe = probe;
        if (site) b->h_ctl[k].bounds = site;
    }
    LBC_CUDA_TRY(cudaMemcpyAsync(b->d_ctl + first, b->h_ctl + first, count * sizeof(Ctl), cudaMemcpyHostToDevice,
                                 b->stream));
    return LBC_OK;
}

// Device control blocks -> h_ctl (synchronises); reports a timeout, records non-finite instances.
lbc_status read_ctl(lbc_batch *b)
{
    LBC_CUDA_TRY(cudaMemcpyAsync(b->h_ctl, b->d_ctl, b->n * sizeof(Ctl), cudaMemcpyDeviceToHost, b->stream));
    LBC_CUDA_TRY(cudaStreamSynchronize(b->stream));
    bool any = false;
    for (int i = 0; i < b->n; ++i) {
        if (b->h_ctl[i].bounds) {
            b->bounds_site = b->h_ctl[i].bounds;
            return fail(LBC_EBOUNDS, "instance " + std::to_string(i) + ": device index check failed: " +
                                         check_site_name(b->bounds_site));
        }
        if (b->h_ctl[i].timeout) {
            b->timed_out = true;
            return fail(LBC_ETIMEOUT, "a bounded device wait gave up");
        }
        any = any || b->h_ctl[i].nonfinite;
    }
    if (any) {
        b->poisoned = true;
        return fail(LBC_ENONFINITE, "non-finite value in the state");
    }
    return LBC_OK;
}

// Device control blocks for plain stepping: counters = completed steps, no early stop.
lbc_status plain_mode(lbc_batch *b)
{
    if (!b->steady_mode) return LBC_OK;
    for (int i = 0; i < b->n; ++i) {
        Ctl &c = b->h_ctl[i];
        c.base = b->ih[i].steps;
        c.check_from = b->ih[i].steps;
        c.stop_eps = 0.0;
        c.stop_step = 0;
        c.stopped = 0;
    }
    b->steady_mode = false;
    return upload_ctl(b, 0, b->n);
}

// Stage data of buffer 0 of instance i from its state (after create or set_state).
lbc_status rebuild_stage_data(lbc_batch *b, int i)
{
    const Inst &I = b->inst[i];
    LBC_CUDA_TRY(b->fp32 ? launch_moments_partial<float>(I.T, I.S, 0, b->stream)
                         : launch_moments_partial<double>(I.T, I.S, 0, b->stream));
    LBC_CUDA_TRY(b->fp32 ? launch_tile_equilibrium<float>(I.T, I.S, 0, b->stream)
                         : launch_tile_equilibrium<double>(I.T, I.S, 0, b->stream));
    return LBC_OK;
}

// Work list: every (instance, tile), instances with the longest CTAs first.
void build_work(lbc_batch *b, std::vector<int2> &work)
{
    std::vector<int> order(b->n);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(),
                     [&](int x, int y) { return b->inst[x].T.vchunk > b->inst[y].T.vchunk; });
    work.clear();
    for (int i : order)
        for (int t = 0; t < b->inst[i].T.ntile; ++t) work.push_back(make_int2(i, t));
}

// Uploads the descriptors and the work list (at creation and after a launch-shape change).
lbc_status upload_descriptors(lbc_batch *b)
{
    std::vector<int2> work;
    build_work(b, work);
    if ((int)work.size() != b->nwork) return fail(LBC_ECUDA, "internal: work list size changed");
    LBC_CUDA_TRY(cudaMemcpyAsync(b->d_inst, b->inst.data(), b->n * sizeof(Inst), cudaMemcpyHostToDevice, b->stream));
    LBC_CUDA_TRY(cudaMemcpyAsync(b->d_work, work.data(), work.size() * sizeof(int2), cudaMemcpyHostToDevice,
                                 b->stream));
    LBC_CUDA_TRY(cudaStreamSynchronize(b->stream));   // pageable sources
    return LBC_OK;
}

lbc_status batch_create(const lbc_params *params, int n, int cluster_in, void *cuda_stream, lbc_batch **out)
{
    if (!params || !out || n < 1) return fail(LBC_EINVAL, "params, out and n >= 1 are required");
    if (cluster_in < 0 || cluster_in > kMaxCluster) return fail(LBC_EINVAL, "cluster must be in [0, 16]");
    std::vector<lbc_params> ps(params, params + n);
    std::vector<int> Nxe(n), Nye(n);
    for (int i = 0; i < n; ++i) {
        lbc_params &p = ps[i];
        if (p.p0 == 0.0) p.p0 = 1.0;
        if (p.cfl == 0.0) p.cfl = 0.5;
        lbc_status st = validate(p, Nxe[i], Nye[i]);
        if (st != LBC_OK) return n > 1 ? fail(st, "instance " + std::to_string(i) + ": " + last_error()) : st;
        if (p.precision != ps[0].precision) return fail(LBC_EINVAL, "every instance of a batch has one precision");
    }
    lbc_batch *b = new (std::nothrow) lbc_batch();
    if (!b) return fail(LBC_ENOMEM, "host allocation failed");
    auto cleanup = [&](lbc_status code) {
        std::string msg = last_error();
        lbc_batch_destroy(b);
        set_error(msg);
        return code;
    };
    b->n = n;
    b->fp32 = ps[0].precision == LBC_FP32_STATE;
    b->single = n == 1;
    b->stream = static_cast<cudaStream_t>(cuda_stream);
    b->ih.resize(n);
    b->inst.resize(n);

    // ---- host set-up of every instance; table block offsets ----
    std::vector<ProblemSetup> setup(n);
    std::vector<size_t> toff(n);
    size_t tbytes = 0;
    for (int i = 0; i < n; ++i) {
        std::string err;
        if (!setup_problem(ps[i], Nxe[i], Nye[i], setup[i], err))
            return cleanup(fail(LBC_EINVAL, (n > 1 ? "instance " + std::to_string(i) + ": " : std::string()) + err));
        b->ih[i].p = ps[i];
        b->ih[i].x = setup[i].x;
        b->ih[i].frest = setup[i].frest;
        toff[i] = tbytes;
        tbytes += r256(setup[i].blob.size());
    }
    int ntile_total = 0;
    for (int i = 0; i < n; ++i) ntile_total += (ps[i].Nx + kTile - 1) / kTile;
    b->nwork = ntile_total;
    const size_t inst_off = tbytes, work_off = inst_off + r256(n * sizeof(Inst));
    tbytes = work_off + r256(b->nwork * sizeof(int2));
    cudaError_t e = fault_injected("alloc") ? cudaErrorMemoryAllocation
                                            : cudaMallocAsync(&b->table_block, tbytes, b->stream);
    if (e != cudaSuccess) {
        set_error(std::string("cudaMallocAsync(tables): ") + cudaGetErrorString(e));
        return cleanup(e == cudaErrorMemoryAllocation ? LBC_ENOMEM : LBC_ECUDA);
    }
    char *tb = static_cast<char *>(b->table_block);
    b->d_inst = reinterpret_cast<Inst *>(tb + inst_off);
    b->d_work = reinterpret_cast<int2 *>(tb + work_off);
    for (int i = 0; i < n; ++i) {
        bind_tables(setup[i], ps[i], tb + toff[i], b->inst[i].T);
        b->ext = b->ext || ps[i].half_channel || ps[i].local_dt || ps[i].compensated;
    }

    // ---- launch shape ----
    lbc_status st;
    if (b->single) {
        st = choose_launch_shape(b->fp32, b->inst[0].T);
        if (st == LBC_OK && cluster_in > 0 && cluster_in != b->inst[0].T.nchunk) {
            b->inst[0].T.nchunk = cluster_in;
            b->inst[0].T.vchunk = chunk_rows(b->inst[0].T.V, cluster_in);
            if (b->inst[0].T.vchunk > kMaxVChunk) st = fail(LBC_EINVAL, "cluster too small for the velocity set");
        }
        if (st == LBC_OK) {
            b->cluster = b->inst[0].T.nchunk;
            b->smem = stage_launch_smem(b->fp32, b->inst[0].T);
        }
    } else {
        std::vector<DevTables> Ts(n);
        for (int i = 0; i < n; ++i) Ts[i] = b->inst[i].T;
        st = choose_batch_shape(b->fp32, Ts, cluster_in, -1, b->solo, b->cluster, b->smem);
        for (int i = 0; i < n && st == LBC_OK; ++i) b->inst[i].T = Ts[i];
        for (int i = 0; i < n && st == LBC_OK; ++i) {   // the split form's node-step launch
            const DevTables &T = b->inst[i].T;
            const size_t eq = b->fp32 ? equilibrium_smem_bytes<float>(T.Qx, T.Qy, T.Nxe, T.Nye, T.K, T.tab_n)
                                      : equilibrium_smem_bytes<double>(T.Qx, T.Qy, T.Nxe, T.Nye, T.K, T.tab_n);
            b->node_smem = std::max(b->node_smem, eq + 128);   // + alignment of the dynamic base
        }
    }
    if (st != LBC_OK) return cleanup(st);

    // ---- device state ----
    std::vector<size_t> soff(n);
    size_t sbytes = 0;
    for (int i = 0; i < n; ++i) {
        soff[i] = sbytes;
        sbytes += StateSizes(b->inst[i].T, b->fp32).total;
    }
    size_t io_elems = 0;
    for (int i = 0; i < n; ++i) io_elems = std::max(io_elems, 2 * (size_t)b->inst[i].T.V * b->inst[i].T.Nx);
    const size_t ctl_off = sbytes, last_off = ctl_off + r256(n * sizeof(Ctl));
    const size_t io_off = last_off + r256(n * sizeof(double)), bad_off = io_off + r256(io_elems * sizeof(double));
    const size_t cnt_off = bad_off + 256;
    sbytes = cnt_off + r256((kPersistHdr + (size_t)b->nwork + n) * sizeof(unsigned));
    b->io_elems = io_elems;
    e = cudaMallocAsync(&b->state_block, sbytes, b->stream);
    if (e != cudaSuccess) {
        set_error(std::string("cudaMallocAsync(state): ") + cudaGetErrorString(e));
        return cleanup(e == cudaErrorMemoryAllocation ? LBC_ENOMEM : LBC_ECUDA);
    }
    e = cudaMemsetAsync(b->state_block, 0, sbytes, b->stream);   // deviation 0 = the rest state; control zeroed
    if (e != cudaSuccess) { set_error(std::string("cudaMemsetAsync: ") + cudaGetErrorString(e)); return cleanup(LBC_ECUDA); }
    char *sb = static_cast<char *>(b->state_block);
    b->d_ctl = reinterpret_cast<Ctl *>(sb + ctl_off);
    b->d_last = reinterpret_cast<double *>(sb + last_off);
    b->d_io = reinterpret_cast<double *>(sb + io_off);
    b->d_bad = reinterpret_cast<int *>(sb + bad_off);
    b->d_cnt = reinterpret_cast<unsigned *>(sb + cnt_off);
    for (int i = 0; i < n; ++i) {
        DevTables &T = b->inst[i].T;
        DevState &S = b->inst[i].S;
        StateSizes(T, b->fp32).carve(sb + soff[i], S);
        S.ctl = b->d_ctl + i;
        StateMaps &M = b->inst[i].M;
        for (int k = 0; k < 3 && st == LBC_OK; ++k) st = encode_state_map(&M.in[k], S.F[k], b->fp32, T.V, T.Nxp, kRowLen,
                                                          slot_rows(k, b->fp32));
        if (st == LBC_OK) st = encode_state_map(&M.f0, S.F[0], b->fp32, T.V, T.Nxp, kF0Len, kSubV);
        if (st != LBC_OK) return cleanup(st);
    }
    e = cudaMallocHost(&b->h_ctl, n * sizeof(Ctl));
    if (e == cudaSuccess) e = cudaMallocHost(&b->h_last, n * sizeof(double));
    if (e == cudaSuccess) e = cudaMallocHost(&b->h_bad, sizeof(int));
    if (e != cudaSuccess) {
        set_error(std::string("cudaMallocHost: ") + cudaGetErrorString(e));
        return cleanup(e == cudaErrorMemoryAllocation ? LBC_ENOMEM : LBC_ECUDA);
    }
    std::memset(b->h_ctl, 0, n * sizeof(Ctl));

    // ---- tables, descriptors, work list; stage data of the rest state ----
    std::vector<unsigned char> image(inst_off, 0);
    for (int i = 0; i < n; ++i) std::memcpy(image.data() + toff[i], setup[i].blob.data(), setup[i].blob.size());
    e = cudaMemcpyAsync(b->table_block, image.data(), image.size(), cudaMemcpyHostToDevice, b->stream);
    if (e != cudaSuccess) { set_error(std::string("table upload: ") + cudaGetErrorString(e)); return cleanup(LBC_ECUDA); }
    st = upload_descriptors(b);   // synchronises: `image` may go away afterwards
    for (int i = 0; i < n && st == LBC_OK; ++i) st = rebuild_stage_data(b, i);
    if (st != LBC_OK) return cleanup(st);
    *out = b;
    return LBC_OK;
}

lbc_status batch_run_to_steady(lbc_batch *b, double residual, long max_steps, long *steps_done,
                               double *final_residual)
{
    if (!b || !(residual > 0.0) || max_steps < 0) return fail(LBC_EINVAL, "bad batch, residual or max_steps");
    if (b->poisoned) return fail(LBC_ENONFINITE, "a state is non-finite");
    const int n = b->n;
    std::vector<long long> start(n);
    for (int i = 0; i < n; ++i) {
        start[i] = b->ih[i].steps;
        Ctl &c = b->h_ctl[i];
        c.base = start[i];
        c.check_from = start[i];
        c.stop_eps = residual;
        c.stop_step = 0;
        c.stopped = 0;
    }
    b->steady_mode = true;
    lbc_status st = upload_ctl(b, 0, n);
    if (st != LBC_OK) return st;
    const long window = b->stall_window;
    std::vector<StallTrack> track(window > 0 ? n : 0);
    std::vector<long> stall_at(n, 0);   // steps done when the instance was found stalled
    long done = 0;
    bool all = false;
    while (done < max_steps && !all) {
        const long k = std::min<long>(kGraphSteps, max_steps - done);
        st = run_steps(b, k);
        if (st != LBC_OK) return st;
        LBC_CUDA_TRY(launch_last_residuals(b->d_inst, nullptr, n, b->d_last, b->stream));
        LBC_CUDA_TRY(cudaMemcpyAsync(b->h_last, b->d_last, n * sizeof(double), cudaMemcpyDeviceToHost, b->stream));
        st = read_ctl(b);   // synchronises: no launch of this call is in flight below
        if (st != LBC_OK) return st;
        done += k;
        all = true;
        for (int i = 0; i < n; ++i) {
            Ctl &c = b->h_ctl[i];
            if (window > 0 && !c.stopped && !track[i].stalled && !(b->h_last[i] < residual) &&
                stall_sample(track[i], done, b->h_last[i], window)) {
                track[i].stalled = true;
                stall_at[i] = done;
                c.stop_eps = INFINITY;   // any finite residual is below it: stops at its next step
                st = upload_ctl(b, i, 1);
                if (st != LBC_OK) return st;
            }
            all = all && (c.stopped || (window > 0 && track[i].stalled));
        }
    }
    int notconv = 0, stalled = 0;
    for (int i = 0; i < n; ++i) {
        const Ctl &c = b->h_ctl[i];
        const bool stall = window > 0 && track[i].stalled;
        long taken = done;
        bool conv = false;
        if (stall) {
            taken = stall_at[i];   // it stops (or stopped) at the first step after the sample
        } else if (c.stopped) {
            taken = (long)(c.stop_step - start[i]);
            conv = true;
        } else if (done > 0 && b->h_last[i] < residual) {
            conv = true;   // the last step launched fell below the threshold
        }
        notconv += !conv && !stall;
        stalled += stall;
        b->ih[i].steps = start[i] + taken;
        if (steps_done) steps_done[i] = taken;
        if (final_residual) final_residual[i] = done > 0 ? b->h_last[i] : INFINITY;
    }
    if (notconv) return fail(LBC_ENOTCONV, "max_steps reached before the residual threshold");
    if (stalled)
        return fail(LBC_ESTALLED, std::to_string(stalled) + " instance(s) stalled above the residual threshold");
    return LBC_OK;
}

lbc_status check_index(const lbc_batch *b, int i)
{
    if (!b) return fail(LBC_EINVAL, "NULL batch");
    if (i < 0 || i >= b->n) return fail(LBC_EINVAL, "instance index out of range");
    return LBC_OK;
}

lbc_status batch_moments(lbc_batch *b, int i, double *out, double *x)
{
    lbc_status st = check_index(b, i);
    if (st != LBC_OK) return st;
    if (!out) return fail(LBC_EINVAL, "NULL argument");
    const Inst &I = b->inst[i];
    LBC_CUDA_TRY(b->fp32 ? launch_moments_from_stage_data<float>(I.T, I.S, b->stream)
                         : launch_moments_from_stage_data<double>(I.T, I.S, b->stream));
    LBC_CUDA_TRY(cudaMemcpy2DAsync(out, I.T.Nx * sizeof(double), I.S.mom_out, I.T.Nxp * sizeof(double),
                                   I.T.Nx * sizeof(double), LBC_NMOM, cudaMemcpyDeviceToHost, b->stream));
    st = read_ctl(b);
    if (st != LBC_OK) return st;
    if (x) std::copy(b->ih[i].x.begin(), b->ih[i].x.end(), x);
    return LBC_OK;
}

lbc_status batch_get_state(lbc_batch *b, int i, double *state)
{
    lbc_status st = check_index(b, i);
    if (st != LBC_OK) return st;
    if (!state) return fail(LBC_EINVAL, "NULL argument");
    const Inst &I = b->inst[i];
    const size_t bytes = 2 * (size_t)I.T.V * I.T.Nx * sizeof(double);
    LBC_CUDA_TRY(b->fp32 ? launch_state_out<float>(I.S.F[0], I.S.C, b->d_io, I.T, b->stream)
                         : launch_state_out<double>(I.S.F[0], nullptr, b->d_io, I.T, b->stream));
    LBC_CUDA_TRY(cudaMemcpyAsync(state, b->d_io, bytes, cudaMemcpyDeviceToHost, b->stream));
    LBC_CUDA_TRY(cudaMemcpyAsync(b->h_ctl, b->d_ctl, b->n * sizeof(Ctl), cudaMemcpyDeviceToHost, b->stream));
    LBC_CUDA_TRY(cudaStreamSynchronize(b->stream));
    for (int k = 0; k < b->n; ++k) {
        if (b->h_ctl[k].bounds) {
            b->bounds_site = b->h_ctl[k].bounds;
            return fail(LBC_EBOUNDS, "instance " + std::to_string(k) + ": device index check failed: " +
                                         check_site_name(b->bounds_site));
        }
        if (b->h_ctl[k].timeout) {
            b->timed_out = true;
            return fail(LBC_ETIMEOUT, "a bounded device wait gave up");
        }
    }
    return LBC_OK;
}

// The host state goes to the device as it is (one copy); a kernel converts it
// into the second RK buffer (and a compensated state's remainders into the third),
// which are free between steps, and checks it, so a rejected state leaves the
// instance unchanged.
lbc_status batch_set_state(lbc_batch *b, int i, const double *state)
{
    lbc_status st = check_index(b, i);
    if (st != LBC_OK) return st;
    if (!state) return fail(LBC_EINVAL, "NULL argument");
    const Inst &I = b->inst[i];
    const size_t bytes = 2 * (size_t)I.T.V * I.T.Nx * sizeof(double);
    LBC_CUDA_TRY(cudaMemcpyAsync(b->d_io, state, bytes, cudaMemcpyHostToDevice, b->stream));
    LBC_CUDA_TRY(cudaMemsetAsync(b->d_bad, 0, sizeof(int), b->stream));
    LBC_CUDA_TRY(b->fp32 ? launch_state_in<float>(b->d_io, I.S.F[1], I.S.C ? I.S.F[2] : nullptr, I.T, b->d_bad,
                                                  b->stream)
                         : launch_state_in<double>(b->d_io, I.S.F[1], nullptr, I.T, b->d_bad, b->stream));
    LBC_CUDA_TRY(cudaMemcpyAsync(b->h_bad, b->d_bad, sizeof(int), cudaMemcpyDeviceToHost, b->stream));
    LBC_CUDA_TRY(cudaMemcpyAsync(b->h_ctl, b->d_ctl, b->n * sizeof(Ctl), cudaMemcpyDeviceToHost, b->stream));
    LBC_CUDA_TRY(cudaStreamSynchronize(b->stream));
    if (*b->h_bad) return fail(LBC_EINVAL, "state holds a NaN or Inf");
    // control blocks: keep the others' flags, clear this instance's
    b->h_ctl[i].nonfinite = 0;
    b->h_ctl[i].timeout = 0;
    b->h_ctl[i].bounds = 0;
    bool any = false, late = false;
    int site = 0;
    for (int k = 0; k < b->n; ++k) {
        any = any || b->h_ctl[k].nonfinite;
        late = late || b->h_ctl[k].timeout;
        if (!site) site = b->h_ctl[k].bounds;
    }
    const size_t esz = b->fp32 ? sizeof(float) : sizeof(double);
    LBC_CUDA_TRY(cudaMemcpyAsync(I.S.F[0], I.S.F[1], 2 * (size_t)I.T.V * I.T.Nxp * esz, cudaMemcpyDeviceToDevice,
                                 b->stream));
    if (I.S.C)
        LBC_CUDA_TRY(cudaMemcpyAsync(I.S.C, I.S.F[2], 2 * (size_t)I.T.V * I.T.Nxp * esz, cudaMemcpyDeviceToDevice,
                                     b->stream));
    st = upload_ctl(b, i, 1);
    if (st == LBC_OK) st = rebuild_stage_data(b, i);
    if (st != LBC_OK) return st;
    LBC_CUDA_TRY(cudaStreamSynchronize(b->stream));
    b->poisoned = any;
    b->timed_out = late;
    b->bounds_site = site;
    return LBC_OK;
}

// The second staging buffer, the copy stream and its events, made at the first
// lbc_batch_set_states.
lbc_status ensure_upload_pipeline(lbc_batch *b)
{
    if (b->copy_stream) return LBC_OK;
    LBC_CUDA_TRY(cudaMallocAsync(&b->d_io2, b->io_elems * sizeof(double), b->stream));
    LBC_CUDA_TRY(cudaStreamCreateWithFlags(&b->copy_stream, cudaStreamNonBlocking));
    LBC_CUDA_TRY(cudaEventCreateWithFlags(&b->ev_start, cudaEventDisableTiming));
    for (int k = 0; k < 2; ++k) {
        LBC_CUDA_TRY(cudaEventCreateWithFlags(&b->ev_copied[k], cudaEventDisableTiming));
        LBC_CUDA_TRY(cudaEventCreateWithFlags(&b->ev_free[k], cudaEventDisableTiming));
    }
    return LBC_OK;
}

// Every given instance's state in one pass. Phase 1, per instance: the host copy on
// the copy stream into one of two staging buffers, then on the batch's stream the
// conversion into RK buffer 1 (a compensated state's remainders into buffer 2) and
// the stage data of buffer 1 (free between steps), so the next instance's copy runs
// under this instance's kernels. One check for all; only then phase 2 commits: the
// buffer-1 state and stage data are copied to buffer 0 (local-step instances rebuild
// buffer 0's stage data, which also holds their mass reference). A rejected set of
// states changes nothing.
lbc_status upload_states(lbc_batch *b, const double *const *states);

lbc_status batch_set_states(lbc_batch *b, const double *const *states)
{
    if (!b || !states) return fail(LBC_EINVAL, "NULL argument");
    lbc_status st = ensure_upload_pipeline(b);
    if (st != LBC_OK) return st;
    st = upload_states(b, states);
    // on any failure no copy from the caller's host arrays is left in flight
    if (st != LBC_OK && b->copy_stream) cudaStreamSynchronize(b->copy_stream);
    return st;
}

lbc_status upload_states(lbc_batch *b, const double *const *states)
{
    lbc_status st = LBC_OK;
    LBC_CUDA_TRY(cudaMemsetAsync(b->d_bad, 0, sizeof(int), b->stream));
    LBC_CUDA_TRY(cudaEventRecord(b->ev_start, b->stream));   // earlier work on the staging buffers is done
    LBC_CUDA_TRY(cudaStreamWaitEvent(b->copy_stream, b->ev_start, 0));
    int k = 0;
    for (int i = 0; i < b->n; ++i) {
        if (!states[i]) continue;
        const Inst &I = b->inst[i];
        const int slot = k & 1;
        double *buf = slot ? b->d_io2 : b->d_io;
        if (k >= 2) LBC_CUDA_TRY(cudaStreamWaitEvent(b->copy_stream, b->ev_free[slot], 0));
        const size_t bytes = 2 * (size_t)I.T.V * I.T.Nx * sizeof(double);
        LBC_CUDA_TRY(cudaMemcpyAsync(buf, states[i], bytes, cudaMemcpyHostToDevice, b->copy_stream));
        LBC_CUDA_TRY(cudaEventRecord(b->ev_copied[slot], b->copy_stream));
        LBC_CUDA_TRY(cudaStreamWaitEvent(b->stream, b->ev_copied[slot], 0));
        LBC_CUDA_TRY(b->fp32 ? launch_state_in<float>(buf, I.S.F[1], I.S.C ? I.S.F[2] : nullptr, I.T, b->d_bad,
                                                      b->stream)
                             : launch_state_in<double>(buf, I.S.F[1], nullptr, I.T, b->d_bad, b->stream));
        LBC_CUDA_TRY(cudaEventRecord(b->ev_free[slot], b->stream));
        if (!I.T.lts) {
            LBC_CUDA_TRY(b->fp32 ? launch_moments_partial<float>(I.T, I.S, 1, b->stream)
                                 : launch_moments_partial<double>(I.T, I.S, 1, b->stream));
            LBC_CUDA_TRY(b->fp32 ? launch_tile_equilibrium<float>(I.T, I.S, 1, b->stream)
                                 : launch_tile_equilibrium<double>(I.T, I.S, 1, b->stream));
        }
        ++k;
    }
    LBC_CUDA_TRY(cudaMemcpyAsync(b->h_bad, b->d_bad, sizeof(int), cudaMemcpyDeviceToHost, b->stream));
    LBC_CUDA_TRY(cudaMemcpyAsync(b->h_ctl, b->d_ctl, b->n * sizeof(Ctl), cudaMemcpyDeviceToHost, b->stream));
    LBC_CUDA_TRY(cudaStreamSynchronize(b->stream));
    if (*b->h_bad) return fail(LBC_EINVAL, "a state holds a NaN or Inf; no instance changed");
    bool any = false, late = false;
    int site = 0;
    const size_t esz = b->fp32 ? sizeof(float) : sizeof(double);
    for (int i = 0; i < b->n; ++i) {
        if (states[i]) {
            const Inst &I = b->inst[i];
            const size_t bytes = 2 * (size_t)I.T.V * I.T.Nxp * esz;
            b->h_ctl[i].nonfinite = 0;
            b->h_ctl[i].timeout = 0;
            b->h_ctl[i].bounds = 0;
            LBC_CUDA_TRY(cudaMemcpyAsync(I.S.F[0], I.S.F[1], bytes, cudaMemcpyDeviceToDevice, b->stream));
            if (I.S.C) LBC_CUDA_TRY(cudaMemcpyAsync(I.S.C, I.S.F[2], bytes, cudaMemcpyDeviceToDevice, b->stream));
            if (I.T.lts) {
                st = rebuild_stage_data(b, i);
                if (st != LBC_OK) return st;
            } else {
                const StateSizes z(I.T, b->fp32);
                LBC_CUDA_TRY(cudaMemcpyAsync(I.S.eqm[0], I.S.eqm[1], z.eqm, cudaMemcpyDeviceToDevice, b->stream));
                LBC_CUDA_TRY(cudaMemcpyAsync(I.S.eqg[0], I.S.eqg[1], z.eqg, cudaMemcpyDeviceToDevice, b->stream));
            }
        }
        any = any || b->h_ctl[i].nonfinite;
        late = late || b->h_ctl[i].timeout;
        if (!site) site = b->h_ctl[i].bounds;
    }
    st = upload_ctl(b, 0, b->n);
    if (st != LBC_OK) return st;
    LBC_CUDA_TRY(cudaStreamSynchronize(b->stream));
    b->poisoned = any;
    b->timed_out = late;
    b->bounds_site = site;
    return LBC_OK;
}

// The moments of every instance, back to back; one synchronisation.
lbc_status batch_moments_all(lbc_batch *b, double *out)
{
    if (!b || !out) return fail(LBC_EINVAL, "NULL argument");
    size_t off = 0;
    for (int i = 0; i < b->n; ++i) {
        const Inst &I = b->inst[i];
        LBC_CUDA_TRY(b->fp32 ? launch_moments_from_stage_data<float>(I.T, I.S, b->stream)
                             : launch_moments_from_stage_data<double>(I.T, I.S, b->stream));
        LBC_CUDA_TRY(cudaMemcpy2DAsync(out + off, I.T.Nx * sizeof(double), I.S.mom_out, I.T.Nxp * sizeof(double),
                                       I.T.Nx * sizeof(double), LBC_NMOM, cudaMemcpyDeviceToHost, b->stream));
        off += (size_t)LBC_NMOM * I.T.Nx;
    }
    return read_ctl(b);
}

// Times trial_steps steps per feasible cluster size (after one warm-up step) and
// keeps the fastest; every instance starts and ends at the rest state.
// Clusters of the persistent form at the batch's launch shape (resident at once, at most one per work item).
lbc_status persistent_shape(lbc_batch *b)
{
    int nc = 0;
    cudaError_t e = b->fp32 ? persistent_active_clusters<float>(b->smem, b->cluster, &nc)
                            : persistent_active_clusters<double>(b->smem, b->cluster, &nc);
    if (e != cudaSuccess) return fail(LBC_ECUDA, std::string("persistent occupancy: ") + cudaGetErrorString(e));
    if (nc < 1) return fail(LBC_EINVAL, "the persistent form does not fit the device at this launch shape");
    b->pclusters = std::min(nc, b->nwork);
    return LBC_OK;
}

lbc_status batch_autotune(lbc_batch *b, int trial_steps, int *cluster_out)
{
    if (!b || trial_steps < 1) return fail(LBC_EINVAL, "bad batch or trial_steps");
    for (int i = 0; i < b->n; ++i)
        if (b->ih[i].steps != 0) return fail(LBC_EINVAL, "autotune needs every instance at its initial state");
    if (b->single) {
        if (cluster_out) *cluster_out = b->cluster;
        return LBC_OK;   // the single-instance shape comes from the wave model of its own launch
    }
    cudaEvent_t t0, t1;
    LBC_CUDA_TRY(cudaEventCreate(&t0));
    LBC_CUDA_TRY(cudaEventCreate(&t1));
    const std::vector<Inst> keep = b->inst;
    float best = 1e30f;
    int best_c = b->cluster;
    size_t best_smem = b->smem;
    bool best_solo = b->solo, best_full = b->full, best_split = b->split;
    const int keep_c = b->cluster;
    const size_t keep_smem = b->smem;
    const bool keep_solo = b->solo, keep_full = b->full, keep_split = b->split;
    std::vector<DevTables> best_T;
    lbc_status st = LBC_OK;
    // every cluster size in the three forms of the per-stage launches (the persistent form has one
    // form), and the solo and split forms with full chunks (the last two trials)
    const int ntrials = b->persistent ? kMaxCluster : 3 * kMaxCluster + 2;
    for (int trial = 0; trial < ntrials && st == LBC_OK; ++trial) {
        const int C = 1 + trial % kMaxCluster, kind = trial / kMaxCluster;   // 0 cluster, 1 solo, 2 split, 3 full
        std::vector<DevTables> Ts(b->n);
        for (int i = 0; i < b->n; ++i) Ts[i] = keep[i].T;
        int c = 0;
        size_t smem = 0;
        bool solo = kind > 0;
        const bool full = kind == 3, split = kind == 2 || (full && trial == 3 * kMaxCluster + 1);
        if (full) {
            if (choose_full_chunk_shape(b->fp32, Ts, c, smem) != LBC_OK) continue;
        } else if (choose_batch_shape(b->fp32, Ts, C, kind > 0 ? 1 : 0, solo, c, smem) != LBC_OK) {
            continue;
        }
        for (int i = 0; i < b->n; ++i) b->inst[i].T = Ts[i];
        b->cluster = c;
        b->smem = smem;
        b->solo = solo;
        b->split = split;
        b->full = full;
        if (b->persistent && persistent_shape(b) != LBC_OK) continue;
        st = upload_descriptors(b);
        if (st != LBC_OK) break;
        cudaError_t e = launch_steps(b, 1, b->stream);
        if (e == cudaSuccess) e = cudaEventRecord(t0, b->stream);
        if (e == cudaSuccess) e = launch_steps(b, trial_steps, b->stream);
        if (e == cudaSuccess) e = cudaEventRecord(t1, b->stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(t1);
        float ms = 0;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, t0, t1);
        if (e != cudaSuccess) { st = fail(LBC_ECUDA, std::string("autotune: ") + cudaGetErrorString(e)); break; }
        if (ms < best) {
            best = ms;
            best_c = c;
            best_smem = smem;
            best_solo = solo;
            best_full = full;
            best_split = split;
            best_T = Ts;
        }
    }
    cudaEventDestroy(t0);
    cudaEventDestroy(t1);
    if (best_T.empty()) {   // nothing measured: keep the model's choice
        b->inst = keep;
        b->cluster = keep_c;
        b->smem = keep_smem;
        b->solo = keep_solo;
        b->full = keep_full;
        b->split = keep_split;
        st = st == LBC_OK ? fail(LBC_EINVAL, "no cluster size could be timed") : st;
    } else {
        for (int i = 0; i < b->n; ++i) b->inst[i].T = best_T[i];
        b->cluster = best_c;
        b->smem = best_smem;
        b->solo = best_solo;
        b->full = best_full;
        b->split = best_split;
    }
    if (b->persistent && st == LBC_OK) st = persistent_shape(b);
    if (b->graph) {
        cudaGraphExecDestroy(b->graph);
        b->graph = nullptr;
    }
    lbc_status st2 = upload_descriptors(b);
    // back to the rest state: zero states and control, rebuild the stage data
    for (int i = 0; i < b->n && st2 == LBC_OK; ++i) {
        const DevTables &T = b->inst[i].T;
        const size_t esz = b->fp32 ? sizeof(float) : sizeof(double);
        cudaError_t e = cudaMemsetAsync(b->inst[i].S.F[0], 0, 2 * (size_t)T.V * T.Nxp * esz, b->stream);
        if (e == cudaSuccess && b->inst[i].S.C)
            e = cudaMemsetAsync(b->inst[i].S.C, 0, 2 * (size_t)T.V * T.Nxp * esz, b->stream);
        if (e != cudaSuccess) st2 = fail(LBC_ECUDA, std::string("cudaMemsetAsync: ") + cudaGetErrorString(e));
        if (st2 == LBC_OK) st2 = rebuild_stage_data(b, i);
    }
    if (st2 == LBC_OK) {
        std::memset(b->h_ctl, 0, b->n * sizeof(Ctl));
        b->steady_mode = false;
        st2 = upload_ctl(b, 0, b->n);
    }
    if (st2 == LBC_OK) LBC_CUDA_TRY(cudaStreamSynchronize(b->stream));
    if (st == LBC_OK) st = st2;
    if (st == LBC_OK && cluster_out) *cluster_out = b->cluster;
    return st;
}

}  // namespace

extern "C" {

lbc_status lbc_batch_create(const lbc_params *params, int n, int cluster, void *cuda_stream, lbc_batch **out)
{
    NvtxRange nvtx_range("lbc_batch_create");
    return batch_create(params, n, cluster, cuda_stream, out);
}

lbc_status lbc_batch_step(lbc_batch *b, long nsteps)
{
    NvtxRange nvtx_range("lbc_batch_step");
    if (!b || nsteps < 0) return fail(LBC_EINVAL, "bad batch or nsteps");
    if (b->poisoned) return fail(LBC_ENONFINITE, "a state is non-finite");
    lbc_status st = plain_mode(b);
    if (st == LBC_OK) st = run_steps(b, nsteps);
    if (st != LBC_OK) return st;
    for (int i = 0; i < b->n; ++i) b->ih[i].steps += nsteps;
    return LBC_OK;
}

lbc_status lbc_batch_run_to_steady(lbc_batch *b, double residual, long max_steps, long *steps_done,
                                   double *final_residual)
{
    NvtxRange nvtx_range("lbc_batch_run_to_steady");
    return batch_run_to_steady(b, residual, max_steps, steps_done, final_residual);
}

lbc_status lbc_batch_moments(lbc_batch *b, int i, double *out, double *x) { return batch_moments(b, i, out, x); }
lbc_status lbc_batch_get_state(lbc_batch *b, int i, double *state) { return batch_get_state(b, i, state); }
lbc_status lbc_batch_set_state(lbc_batch *b, int i, const double *state) { return batch_set_state(b, i, state); }
lbc_status lbc_batch_set_states(lbc_batch *b, const double *const *states)
{
    NvtxRange nvtx_range("lbc_batch_set_states");
    return batch_set_states(b, states);
}
lbc_status lbc_batch_moments_all(lbc_batch *b, double *out) { return batch_moments_all(b, out); }

lbc_status lbc_batch_info(const lbc_batch *b, int i, int *Nx, int *V, double *dt, long *steps_taken)
{
    lbc_status st = check_index(b, i);
    if (st != LBC_OK) return st;
    const DevTables &T = b->inst[i].T;
    if (Nx) *Nx = T.Nx;
    if (V) *V = T.V;
    if (dt) *dt = T.dt;
    if (steps_taken) *steps_taken = (long)b->ih[i].steps;
    return LBC_OK;
}

lbc_status lbc_batch_shape(const lbc_batch *b, int *cluster, int *nwork, size_t *smem_bytes)
{
    if (!b) return fail(LBC_EINVAL, "NULL batch");
    if (cluster) *cluster = b->cluster;
    if (nwork) *nwork = b->nwork;
    if (smem_bytes) *smem_bytes = b->smem;
    return LBC_OK;
}

lbc_status lbc_batch_autotune(lbc_batch *b, int trial_steps, int *cluster) { return batch_autotune(b, trial_steps, cluster); }

lbc_status lbc_batch_form(const lbc_batch *b, int *solo)
{
    if (!b || !solo) return fail(LBC_EINVAL, "NULL argument");
    *solo = (!b->single && b->solo) ? (b->split ? 3 : 1) + (b->full ? 1 : 0) : 0;
    return LBC_OK;
}

lbc_status lbc_batch_set_form(lbc_batch *b, int solo)
{
    if (!b) return fail(LBC_EINVAL, "NULL batch");
    if (b->single) return fail(LBC_EINVAL, "a single-instance batch has the cluster form only");
    std::vector<DevTables> Ts(b->n);
    for (int i = 0; i < b->n; ++i) Ts[i] = b->inst[i].T;
    if (solo < 0 || solo > 4) return fail(LBC_EINVAL, "form must be in [0, 4]");
    const bool full = solo == 2 || solo == 4;
    bool f = full;
    int c = 0;
    size_t smem = 0;
    lbc_status st = full ? choose_full_chunk_shape(b->fp32, Ts, c, smem)
                         : choose_batch_shape(b->fp32, Ts, b->cluster, solo ? 1 : 0, f, c, smem);
    if (st != LBC_OK) return st;
    LBC_CUDA_TRY(cudaStreamSynchronize(b->stream));   // no launch of the old form in flight
    for (int i = 0; i < b->n; ++i) b->inst[i].T = Ts[i];
    b->cluster = c;
    b->smem = smem;
    b->solo = f;
    b->full = full;
    b->split = solo >= 3;
    if (b->graph) {
        cudaGraphExecDestroy(b->graph);
        b->graph = nullptr;
    }
    return upload_descriptors(b);
}

lbc_status lbc_batch_set_stall_window(lbc_batch *b, long window)
{
    if (!b || window < 0) return fail(LBC_EINVAL, "bad batch or stall window");
    b->stall_window = window;
    return LBC_OK;
}

lbc_status lbc_batch_set_persistent(lbc_batch *b, int on)
{
    if (!b) return fail(LBC_EINVAL, "NULL batch");
    if (on) {
        lbc_status st = persistent_shape(b);
        if (st != LBC_OK) return st;
    }
    if (b->persistent != (on != 0) && b->graph) {   // the captured group of steps changes form
        cudaGraphExecDestroy(b->graph);
        b->graph = nullptr;
    }
    b->persistent = on != 0;
    return LBC_OK;
}

lbc_status lbc_batch_step_timed(lbc_batch *b, long nsteps, double *stage_ms)
{
    NvtxRange nvtx_range("lbc_batch_step_timed");
    if (!b || nsteps < 0 || !stage_ms) return fail(LBC_EINVAL, "bad batch, nsteps or stage_ms");
    if (b->persistent) return fail(LBC_EINVAL, "the persistent form has no separate stage launches to time");
    if (b->poisoned) return fail(LBC_ENONFINITE, "a state is non-finite");
    lbc_status st = plain_mode(b);
    if (st != LBC_OK) return st;
    const int nl = (int)(3 * nsteps);
    std::vector<cudaEvent_t> ev(2 * (size_t)nl, nullptr);
    cudaError_t e = cudaSuccess;
    for (size_t k = 0; k < ev.size() && e == cudaSuccess; ++k) e = cudaEventCreate(&ev[k]);
    for (long k = 0; k < nsteps && e == cudaSuccess; ++k)
        for (int stage = 0; stage < 3 && e == cudaSuccess; ++stage) {
            const size_t j = 2 * (size_t)(3 * k + stage);
            e = cudaEventRecord(ev[j], b->stream);
            if (e == cudaSuccess)
                e = b->fp32 ? (b->single ? launch_stage<float>(b->inst[0], b->smem, stage, (int)k, b->stream)
                                         : launch_stage_batch<float>(b->d_inst, b->d_work, b->nwork, b->cluster,
                                                                     b->smem, stage, (int)k, b->ext, kernel_form(b),
                                                                     b->node_smem, b->stream))
                            : (b->single ? launch_stage<double>(b->inst[0], b->smem, stage, (int)k, b->stream)
                                         : launch_stage_batch<double>(b->d_inst, b->d_work, b->nwork, b->cluster,
                                                                      b->smem, stage, (int)k, b->ext, kernel_form(b),
                                                                      b->node_smem, b->stream));
            if (e == cudaSuccess) e = cudaEventRecord(ev[j + 1], b->stream);
        }
    if (e == cudaSuccess) e = launch_ctl_bump(b->d_ctl, b->n, nsteps, b->stream);
    double total = 0.0;
    for (int k = 0; k < nl && e == cudaSuccess; ++k) {
        e = cudaEventSynchronize(ev[2 * k + 1]);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, ev[2 * k], ev[2 * k + 1]);
        total += ms;
    }
    for (cudaEvent_t x : ev)
        if (x) cudaEventDestroy(x);
    if (e != cudaSuccess) return fail(LBC_ECUDA, std::string("timed step: ") + cudaGetErrorString(e));
    for (int i = 0; i < b->n; ++i) b->ih[i].steps += nsteps;
    *stage_ms = total;
    return LBC_OK;
}

void lbc_batch_destroy(lbc_batch *b)
{
    if (!b) return;
    if (b->graph) cudaGraphExecDestroy(b->graph);
    if (b->copy_stream) cudaStreamSynchronize(b->copy_stream);
    if (b->d_io2) cudaFreeAsync(b->d_io2, b->stream);
    for (cudaEvent_t e : {b->ev_start, b->ev_copied[0], b->ev_copied[1], b->ev_free[0], b->ev_free[1]})
        if (e) cudaEventDestroy(e);
    if (b->copy_stream) cudaStreamDestroy(b->copy_stream);
    if (b->state_block) cudaFreeAsync(b->state_block, b->stream);
    if (b->table_block) cudaFreeAsync(b->table_block, b->stream);
    if (b->h_ctl || b->h_last) cudaStreamSynchronize(b->stream);
    if (b->h_ctl) cudaFreeHost(b->h_ctl);
    if (b->h_last) cudaFreeHost(b->h_last);
    if (b->h_bad) cudaFreeHost(b->h_bad);
    delete b;
}

// ---- the single-instance solver: a batch of one ----

lbc_status lbc_create(const lbc_params *params, void *cuda_stream, lbc_solver **out)
{
    NvtxRange nvtx_range("lbc_create");
    if (!params || !out) return fail(LBC_EINVAL, "params and out must not be NULL");
    lbc_solver *s = new (std::nothrow) lbc_solver();
    if (!s) return fail(LBC_ENOMEM, "host allocation failed");
    lbc_status st = batch_create(params, 1, 0, cuda_stream, &s->b);
    if (st != LBC_OK) {
        delete s;
        return st;
    }
    *out = s;
    return LBC_OK;
}

lbc_status lbc_step(lbc_solver *s, long nsteps)
{
    NvtxRange nvtx_range("lbc_step");
    if (!s) return fail(LBC_EINVAL, "bad solver or nsteps");
    return lbc_batch_step(s->b, nsteps);
}

lbc_status lbc_run_to_steady(lbc_solver *s, double residual, long max_steps, long *steps_done,
                             double *final_residual)
{
    NvtxRange nvtx_range("lbc_run_to_steady");
    if (!s) return fail(LBC_EINVAL, "bad solver, residual or max_steps");
    return batch_run_to_steady(s->b, residual, max_steps, steps_done, final_residual);
}

lbc_status lbc_set_stall_window(lbc_solver *s, long window)
{
    if (!s) return fail(LBC_EINVAL, "NULL solver");
    return lbc_batch_set_stall_window(s->b, window);
}

lbc_status lbc_moments(lbc_solver *s, double *out, double *x)
{
    if (!s) return fail(LBC_EINVAL, "NULL argument");
    return batch_moments(s->b, 0, out, x);
}

lbc_status lbc_get_state(lbc_solver *s, double *state)
{
    if (!s) return fail(LBC_EINVAL, "NULL argument");
    return batch_get_state(s->b, 0, state);
}

lbc_status lbc_set_state(lbc_solver *s, const double *state)
{
    NvtxRange nvtx_range("lbc_set_state");
    if (!s) return fail(LBC_EINVAL, "NULL argument");
    return batch_set_state(s->b, 0, state);
}

lbc_status lbc_info(const lbc_solver *s, int *Nx, int *V, double *dt, long *steps_taken)
{
    if (!s) return fail(LBC_EINVAL, "NULL solver");
    return lbc_batch_info(s->b, 0, Nx, V, dt, steps_taken);
}

void lbc_destroy(lbc_solver *s)
{
    if (!s) return;
    lbc_batch_destroy(s->b);
    delete s;
}

}  // extern "C"
