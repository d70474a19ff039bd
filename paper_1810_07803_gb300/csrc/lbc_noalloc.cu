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

lbc_status fail_na(lbc_status st, const std::string &msg)
{
    set_error(msg);
    return st;
}

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

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

lbc_status encode_map(CUtensorMap *map, void *base, bool fp32, int V, int Nxp, int box_cols)
{
    static EncodeTiledFn fn = nullptr;
    if (!fn) {
        cudaDriverEntryPointQueryResult q;
        void *ptr = nullptr;
        cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault, &q);
        if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !ptr)
            return fail_na(LBC_ECUDA, "cuTensorMapEncodeTiled is not available from the driver");
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
    if (r != CUDA_SUCCESS) return fail_na(LBC_ECUDA, "cuTensorMapEncodeTiled failed");
    return LBC_OK;
}

// Caller's weight-divided FP64 state [2][V][Nx] <-> deviation buffer [2][V][Nxp] (state precision).
template <typename R>
__global__ void state_in_kernel(const double *src, R *dst, const double *frest, int V, int Nx, int Nxp)
{
    const size_t n = 2 * (size_t)V * Nx;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const size_t row = i / Nx;
        const int s = (int)(i - row * Nx);
        dst[row * Nxp + s] = R(src[i] - frest[row % V]);
    }
}

template <typename R>
__global__ void state_out_kernel(const R *src, double *dst, const double *frest, int V, int Nx, int Nxp)
{
    const size_t n = 2 * (size_t)V * Nx;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const size_t row = i / Nx;
        const int s = (int)(i - row * Nx);
        dst[i] = frest[row % V] + (double)src[row * Nxp + s];
    }
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

    HostTables t;
    std::string err;
    if (!build_tables(p.Qx, p.Qy, Nxe, Nye, p.p0, t, err)) return fail_na(LBC_EINVAL, err);
    const int V = t.V, Nx = p.Nx;
    std::vector<double> x, inv_jdeta;
    double deta, min_jdeta;
    make_grid(Nx, p.stretch_A, x, inv_jdeta, deta, min_jdeta);
    double dt = p.dt > 0 ? p.dt : p.cfl * min_jdeta / (t.zx.back() * p.p0);
    if (p.dt <= 0 && p.delta > 0)
        for (double Tw : {1.0, p.T_left, p.T_right})
            dt = std::min(dt, 0.5 * std::pow(Tw, p.omega - 1.0) / (p.delta * std::sqrt(2.0)));

    std::vector<double> gx(2 * p.Qx), gy(p.Qy), fwL(V), fwR(V), frest(V), vel((size_t)kVelCols * V), aj(2 * (size_t)V);
    DevTables T{};
    equilibrium_host(t, 0.0, p.u_left, p.T_left, gx.data(), gy.data());
    for (int v = 0; v < V; ++v) fwL[v] = gx[v / p.Qy] * gy[v % p.Qy];
    equilibrium_host(t, 0.0, p.u_right, p.T_right, gx.data(), gy.data());
    for (int v = 0; v < V; ++v) fwR[v] = gx[v / p.Qy] * gy[v % p.Qy];
    equilibrium_host(t, 0.0, 0.0, 1.0, gx.data(), gy.data());
    for (int v = 0; v < V; ++v) frest[v] = gx[v / p.Qy] * gy[v % p.Qy];
    for (int v = 0; v < V; ++v) {
        const int a = v / p.Qy, j = v % p.Qy, i = a < p.Qx ? a : a - p.Qx;
        const double px = (a < p.Qx ? 1.0 : -1.0) * p.p0 * t.zx[i], py = p.p0 * t.yy[j], w = t.wx[i] * t.wy[j];
        if (px > 0) { T.inL += px * w * fwL[v]; T.restOutR += px * w * frest[v]; }
        else        { T.inR += px * w * fwR[v]; T.restOutL += px * w * frest[v]; }
        const double pw[10] = {1, px, py, px * px, px * py, py * py, px * px * px, px * px * py, px * py * py,
                               py * py * py};
        for (int k = 0; k < 10; ++k) T.restP[k] += pw[k] * w * frest[v];
        const double cols[kVelCols] = {px, py, w, frest[v], fwL[v], p.T_left * fwL[v], fwR[v], p.T_right * fwR[v]};
        for (int c = 0; c < kVelCols; ++c) vel[(size_t)c * V + v] = cols[c];
        aj[v] = a;
        aj[V + v] = j;
    }
    T.Nx = Nx; T.Nxp = (Nx + 31) / 32 * 32;
    T.Qx = p.Qx; T.Qy = p.Qy; T.Nxe = Nxe; T.Nye = Nye; T.K = t.K; T.V = V;
    T.ntile = (Nx + kTile - 1) / kTile;
    T.vchunk = std::min(((V + kSubV - 1) / kSubV) * kSubV, 4 * kSubV);
    T.nchunk = (V + T.vchunk - 1) / T.vchunk;
    T.p0 = p.p0; T.dt = dt; T.delta = p.delta; T.Pr = p.Pr; T.omega = p.omega; T.TL = p.T_left; T.TR = p.T_right;

    // ---- layout of the scratch array: tables, then the state ----
    std::vector<double> isb(t.sbeta.size()), invl(kMaxQ + 2);
    for (size_t k = 0; k < isb.size(); ++k) isb[k] = 1.0 / t.sbeta[k];
    for (int l = 0; l < kMaxQ + 2; ++l) invl[l] = l ? 1.0 / l : 0.0;
    struct DPiece { const std::vector<double> *src; const double **dst; };
    DPiece dp[] = {{&inv_jdeta, &T.inv_jdeta}, {&t.zx, &T.zx}, {&t.wx, &T.wx}, {&t.yy, &T.yy}, {&t.wy, &T.wy},
                   {&t.alpha, &T.alpha}, {&t.sbeta, &T.sbeta}, {&t.hz, &T.hz}, {&t.Yk, &T.Yk}, {&t.Wk, &T.Wk},
                   {&t.He, &T.He}, {&fwL, &T.fwL}, {&fwR, &T.fwR}, {&frest, &T.frest}, {&vel, &T.d_vel}};
    struct FPiece { const std::vector<double> *src; const float **dst; };
    FPiece fp[] = {{&t.hz, &T.f_hz}, {&t.He, &T.f_He}, {&t.alpha, &T.f_alpha}, {&isb, &T.f_isbeta},
                   {&t.sbeta, &T.f_sbeta}, {&t.Yk, &T.f_Yk}, {&t.Wk, &T.f_Wk}, {&invl, &T.f_inv_l},
                   {&vel, &T.f_vel}, {&inv_jdeta, &T.f_inv_jdeta}};
    Carve cv(scratch);
    std::vector<std::pair<size_t, size_t>> dblocks, fblocks;   // (offset, element count)
    for (auto &pc : dp) {
        void *d = cv.take(pc.src->size() * sizeof(double));
        dblocks.emplace_back((char *)d - (char *)scratch, pc.src->size());
        *pc.dst = static_cast<const double *>(d);
    }
    for (auto &pc : fp) {
        void *d = cv.take(pc.src->size() * sizeof(float));
        fblocks.emplace_back((char *)d - (char *)scratch, pc.src->size());
        *pc.dst = static_cast<const float *>(d);
    }
    void *ajd = cv.take(aj.size() * sizeof(int));
    T.vel_aj = static_cast<const int *>(ajd);
    const size_t table_bytes = cv.off;

    const size_t esz = sizeof(R);
    DevState S{};
    for (int k = 0; k < 3; ++k) S.F[k] = cv.take(2 * (size_t)V * T.Nxp * esz);
    for (int k = 0; k < 3; ++k) S.part[k] = cv.take((size_t)T.nchunk * kNumRaw * T.Nxp * esz);
    for (int k = 0; k < 3; ++k) S.shift[k] = cv.take(2 * (size_t)T.Nxp * esz);
    for (int k = 0; k < 3; ++k) S.eqm[k] = cv.take((size_t)T.Nxp * kEqM * esz);
    for (int k = 0; k < 3; ++k) S.eqg[k] = cv.take((size_t)T.ntile * (2 * p.Qx + p.Qy) * kLanes * esz);
    for (int k = 0; k < 3; ++k) S.count[k] = static_cast<int *>(cv.take((size_t)T.ntile * sizeof(int)));
    S.resid = static_cast<unsigned long long *>(cv.take(kResidRing * sizeof(unsigned long long)));
    S.ctl = static_cast<Ctl *>(cv.take(sizeof(Ctl)));
    S.mom_out = static_cast<double *>(cv.take((size_t)LBC_NMOM * T.Nxp * sizeof(double)));
    if (cv.off > kScratchBytes)
        return fail_na(LBC_EINVAL, "problem needs " + std::to_string(cv.off) +
                                       " bytes of working memory; the allocation-free path has " +
                                       std::to_string(kScratchBytes));

    // ---- upload the tables (pageable copy: the blob stays alive until it completes) ----
    std::vector<unsigned char> blob(table_bytes, 0);
    for (size_t k = 0; k < dblocks.size(); ++k)
        std::memcpy(blob.data() + dblocks[k].first, dp[k].src->data(), dblocks[k].second * sizeof(double));
    for (size_t k = 0; k < fblocks.size(); ++k) {
        float *d = reinterpret_cast<float *>(blob.data() + fblocks[k].first);
        for (size_t i = 0; i < fblocks[k].second; ++i) d[i] = (float)(*fp[k].src)[i];
    }
    int *ajh = reinterpret_cast<int *>(blob.data() + ((char *)ajd - (char *)scratch));
    for (size_t i = 0; i < aj.size(); ++i) ajh[i] = (int)aj[i];

    StateMaps M{};
    for (int k = 0; k < 3 && st == LBC_OK; ++k) st = encode_map(&M.in[k], S.F[k], fp32, V, T.Nxp, kRowLen);
    if (st == LBC_OK) st = encode_map(&M.f0, S.F[0], fp32, V, T.Nxp, kF0Len);
    if (st != LBC_OK) return st;

#define NA_TRY(call)                                                                                          \
    do {                                                                                                      \
        cudaError_t e_ = (call);                                                                              \
        if (e_ != cudaSuccess) return fail_na(LBC_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)
    NA_TRY(cudaMemcpyAsync(scratch, blob.data(), table_bytes, cudaMemcpyHostToDevice, stream));
    // the array keeps the previous call's contents: clear everything that must start at zero
    NA_TRY(cudaMemsetAsync(static_cast<char *>(scratch) + table_bytes, 0, cv.off - table_bytes, stream));
    const int grid = std::max(1, std::min(1024, (int)((2 * (size_t)V * Nx + 255) / 256)));
    state_in_kernel<R><<<grid, 256, 0, stream>>>(d_state, static_cast<R *>(S.F[0]), T.frest, V, Nx, T.Nxp);
    NA_TRY(cudaGetLastError());
    NA_TRY(launch_moments_partial<R>(T, S, 0, stream));
    NA_TRY(launch_tile_equilibrium<R>(T, S, 0, stream));
    NA_TRY(launch_ctl_set(S.ctl, 0, 0, 0, stream));
    for (long k = 0; k < nsteps; ++k)
        for (int stage = 0; stage < 3; ++stage) NA_TRY(launch_stage<R>(T, S, M, stage, (int)k, 0.0, stream));
    state_out_kernel<R><<<grid, 256, 0, stream>>>(static_cast<const R *>(S.F[0]), d_state, T.frest, V, Nx, T.Nxp);
    NA_TRY(cudaGetLastError());
    Ctl h_ctl;
    NA_TRY(cudaMemcpyAsync(&h_ctl, S.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, stream));
    NA_TRY(cudaStreamSynchronize(stream));
#undef NA_TRY
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
    if (p.Qx < 1 || p.Qx > kMaxQ || p.Qy < 1 || p.Qy > kMaxQ) return fail_na(LBC_EINVAL, "Qx and Qy must be in [1, 64]");
    const int Nxe = p.Nexp_x ? p.Nexp_x : p.Qx - 1, Nye = p.Nexp_y ? p.Nexp_y : p.Qy - 1;
    if (Nxe < 2 || Nxe >= p.Qx || Nye < 2 || Nye >= p.Qy) return fail_na(LBC_EINVAL, "expansion orders must satisfy 2 <= N < Q");
    if (p.Nx < 8 || p.Nx > (1 << 24)) return fail_na(LBC_EINVAL, "Nx must be in [8, 2^24]");
    if (!(p.delta >= 0.0) || !(p.T_left > 0.0) || !(p.T_right > 0.0) || !(p.stretch_A >= 0.0 && p.stretch_A < 1.0) ||
        !(p.p0 > 0.0) || p.cfl < 0.0 || p.dt < 0.0 || !(p.Pr > 0.0) || p.mu_law != LBC_MU_POWER)
        return fail_na(LBC_EINVAL, "invalid physical parameters");
    cudaStream_t stream = static_cast<cudaStream_t>(cuda_stream);
    return p.precision == LBC_FP32_STATE ? run_noalloc<float>(p, Nxe, Nye, d_state, nsteps, stream)
                                         : run_noalloc<double>(p, Nxe, Nye, d_state, nsteps, stream);
}
