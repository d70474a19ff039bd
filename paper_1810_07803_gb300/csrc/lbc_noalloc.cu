// Allocation-free stepping entry point (lbc_step_noalloc, include/lbc.h).
//
// Some callers cannot call cudaMalloc: code embedded in a host application
// whose own allocator owns the device memory, or latency-critical loops in
// which an allocation (and the synchronisation it can imply) is not
// acceptable. For them this file keeps all working memory of a solve -- the
// tables, the three RK state buffers, the moment partials and stage data, the
// control block -- in one file-scope static device array, and runs the same
// stage kernels as the regular solver on a device state the caller owns.
//
// The array is part of the library image: every GPU that loads the library
// holds it until the process exits. Its device address is resolved with
// cudaGetSymbolAddress once per device, on that device's first call.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <string>
#include <type_traits>
#include <vector>

#include "lbc_device.h"

namespace lbc {

namespace {

constexpr size_t kScratchBytes = size_t(8) << 20;   // 8 MiB, documented in include/lbc.h
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
void *g_scratch_ptr[kMaxDevices] = {nullptr};

lbc_status fail_na(lbc_status st, const std::string &msg) { return fail(st, msg); }

// Device address of the scratch array on the current device (first call per
// device resolves it and sets the kernels' shared-memory limits).
lbc_status scratch_on_current_device(void **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail_na(LBC_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return fail_na(LBC_EINVAL, "device index out of range");
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p)
            return fail_na(LBC_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
        e = configure_kernels<float>();
        if (e == cudaSuccess) e = configure_kernels<double>();
        if (e != cudaSuccess) return fail_na(LBC_ECUDA, std::string("kernel attributes: ") + cudaGetErrorString(e));
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return LBC_OK;
}

struct Carve {
    char *base;
    size_t off = 0;
    explicit Carve(void *b) : base(static_cast<char *>(b)) {}
    void *take(size_t bytes)
    {
        void *p = base + off;
        off += (bytes + 255) / 256 * 256;
        return p;
    }
};

template <typename R>
lbc_status run_noalloc(const lbc_params &p, int Nxe, int Nye, double *d_state, long nsteps, cudaStream_t stream)
{
    const bool fp32 = std::is_same<R, float>::value;
    void *scratch = nullptr;
    lbc_status st = scratch_on_current_device(&scratch);
    if (st != LBC_OK) return st;

    ProblemSetup ps;
    std::string err;
    if (!setup_problem(p, Nxe, Nye, ps, err)) return fail_na(LBC_EINVAL, err);
    Inst I{};
    DevTables &T = I.T;
    bind_tables(ps, p, scratch, T);   // the tables sit at the start of the array
    st = choose_launch_shape(fp32, T);
    if (st != LBC_OK) return st;
    const size_t smem = stage_launch_smem(fp32, T);
    const int V = T.V;

    // ---- layout of the scratch array: tables, then the state ----
    Carve cv(scratch);
    cv.take(ps.blob.size());
    const size_t table_bytes = cv.off;
    const size_t esz = sizeof(R);
    DevState &S = I.S;
    for (int k = 0; k < 3; ++k) S.F[k] = cv.take(2 * (size_t)V * T.Nxp * esz);
    for (int k = 0; k < 3; ++k) S.eqm[k] = cv.take((size_t)T.Nxp * kEqM * esz);
    for (int k = 0; k < 3; ++k) S.eqg[k] = cv.take((size_t)T.ntile * (2 * p.Qx + p.Qy) * kLanes * esz);
    S.part = cv.take((size_t)T.nchunk * kNumRaw * T.Nxp * esz);
    S.tcnt = static_cast<unsigned *>(cv.take((size_t)T.ntile * sizeof(unsigned)));   // (cluster form: unused)
    S.resid = static_cast<unsigned long long *>(cv.take(kResidRing * sizeof(unsigned long long)));
    S.ctl = static_cast<Ctl *>(cv.take(sizeof(Ctl)));
    S.mom_out = static_cast<double *>(cv.take((size_t)LBC_NMOM * T.Nxp * sizeof(double)));
    if (cv.off > kScratchBytes)
        return fail_na(LBC_EINVAL, "problem needs " + std::to_string(cv.off) +
                                       " bytes of working memory; the allocation-free path has " +
                                       std::to_string(kScratchBytes));

    StateMaps &M = I.M;
    for (int k = 0; k < 3 && st == LBC_OK; ++k) st = encode_state_map(&M.in[k], S.F[k], fp32, V, T.Nxp, kRowLen, slot_rows(k, fp32));
    if (st == LBC_OK) st = encode_state_map(&M.f0, S.F[0], fp32, V, T.Nxp, kF0Len, kSubV);
    if (st != LBC_OK) return st;

#define NA_TRY(call)                                                                                          \
    do {                                                                                                      \
        cudaError_t e_ = (call);                                                                              \
        if (e_ != cudaSuccess) return fail_na(LBC_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)
    // pageable copy of the table image: the call synchronises below, before ps goes away
    NA_TRY(cudaMemcpyAsync(scratch, ps.blob.data(), ps.blob.size(), cudaMemcpyHostToDevice, stream));
    // the array keeps the previous call's contents: clear everything that must start at zero
    NA_TRY(cudaMemsetAsync(static_cast<char *>(scratch) + table_bytes, 0, cv.off - table_bytes, stream));
    NA_TRY(launch_state_in<R>(d_state, S.F[0], nullptr, T, nullptr, stream));
    NA_TRY(launch_moments_partial<R>(T, S, 0, stream));
    NA_TRY(launch_tile_equilibrium<R>(T, S, 0, stream));
    // the control block starts zeroed (the clear above): step 0, no early stop
    for (long k = 0; k < nsteps; ++k)
        for (int stage = 0; stage < 3; ++stage) NA_TRY(launch_stage<R>(I, smem, stage, (int)k, stream));
    NA_TRY(launch_state_out<R>(S.F[0], nullptr, d_state, T, stream));
    Ctl h_ctl;
    NA_TRY(cudaMemcpyAsync(&h_ctl, S.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, stream));
    NA_TRY(cudaStreamSynchronize(stream));
#undef NA_TRY
    if (h_ctl.bounds)
        return fail_na(LBC_EBOUNDS, std::string("device index check failed: ") + check_site_name(h_ctl.bounds));
    if (h_ctl.timeout) return fail_na(LBC_ETIMEOUT, "a bounded device wait gave up");
    if (h_ctl.nonfinite) return fail_na(LBC_ENONFINITE, "non-finite value in the state");
    return LBC_OK;
}

}  // namespace

}  // namespace lbc

using namespace lbc;

extern "C" lbc_status lbc_step_noalloc(const lbc_params *params, double *d_state, long nsteps, void *cuda_stream)
{
    if (!params || !d_state || nsteps < 0) return fail_na(LBC_EINVAL, "NULL params/state or negative nsteps");
    lbc_params p = *params;
    if (p.p0 == 0.0) p.p0 = 1.0;
    if (p.cfl == 0.0) p.cfl = 0.5;
    int Nxe = 0, Nye = 0;
    lbc_status st = validate(p, Nxe, Nye);
    if (st != LBC_OK) return st;
    if (p.local_dt)   // the mass reference of local steps would not survive from one call to the next
        return fail_na(LBC_EINVAL, "local_dt is not available on the allocation-free path");
    if (p.compensated)   // no room for the remainder buffer
        return fail_na(LBC_EINVAL, "compensated is not available on the allocation-free path");
    cudaStream_t stream = static_cast<cudaStream_t>(cuda_stream);
    return p.precision == LBC_FP32_STATE ? run_noalloc<float>(p, Nxe, Nye, d_state, nsteps, stream)
                                         : run_noalloc<double>(p, Nxe, Nye, d_state, nsteps, stream);
}
