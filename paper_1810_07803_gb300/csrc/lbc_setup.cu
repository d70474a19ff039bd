// Host set-up shared by every entry point: errors, parameter validation, the
// problem tables (Sec. III quadratures and Hermite tables, Eq. stretch grid,
// time step), the device table image, TMA descriptors and launch shapes.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <functional>
#include <string>
#include <vector>

#include "lbc_device.h"

namespace lbc {

namespace {
thread_local std::string g_err;
}  // namespace

void set_error(const std::string &msg) { g_err = msg; }
const char *last_error() { return g_err.c_str(); }

lbc_status fail(lbc_status st, const std::string &msg)
{
    set_error(msg);
    return st;
}

bool fault_injected(const char *kind)
{
    const char *f = std::getenv("LBC_FAULT");
    return f && std::strcmp(f, kind) == 0;
}

int fault_wait_polls()
{
    const char *f = std::getenv("LBC_FAULT");
    if (!f || std::strncmp(f, "wait:", 5) != 0) return 0;
    const long n = std::strtol(f + 5, nullptr, 10);
    return n > 0 && n < (1L << 30) ? (int)n : 0;
}

int fault_bounds_site()
{
    const char *f = std::getenv("LBC_FAULT");
    if (!f || std::strncmp(f, "bounds:", 7) != 0) return 0;
    const long n = std::strtol(f + 7, nullptr, 10);
    return n > 0 && n < CK_COUNT ? (int)n : 0;
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
    if (p.mu_law == LBC_MU_TABLE) {
        if (p.tab_n < 2 || p.tab_n > kMaxTable || !p.tab_T || !p.tab_mu || !p.tab_Pr)
            return fail(LBC_EINVAL, "a viscosity table needs 2 to 256 entries of T, mu and Pr");
        for (int k = 0; k < p.tab_n; ++k) {
            if (!(p.tab_T[k] > 0.0) || !std::isfinite(p.tab_T[k]) || (k > 0 && !(p.tab_T[k] > p.tab_T[k - 1])))
                return fail(LBC_EINVAL, "table temperatures must be finite, > 0 and strictly increasing");
            if (!(p.tab_mu[k] > 0.0) || !std::isfinite(p.tab_mu[k]))
                return fail(LBC_EINVAL, "table viscosities must be finite and > 0");
            if (!(p.tab_Pr[k] > 0.0) || !std::isfinite(p.tab_Pr[k]))
                return fail(LBC_EINVAL, "table Prandtl numbers must be finite and > 0");
        }
    } else if (p.mu_law != LBC_MU_POWER) {
        return fail(LBC_EINVAL, "unknown viscosity law");
    }
    if (!std::isfinite(p.omega)) return fail(LBC_EINVAL, "omega must be finite");
    if (p.local_dt != 0 && p.local_dt != 1) return fail(LBC_EINVAL, "local_dt must be 0 or 1");
    if (p.local_dt && p.dt > 0.0) return fail(LBC_EINVAL, "local time steps are automatic: dt must be 0");
    if (p.half_channel != 0 && p.half_channel != 1) return fail(LBC_EINVAL, "half_channel must be 0 or 1");
    if (p.compensated != 0 && p.compensated != 1) return fail(LBC_EINVAL, "compensated must be 0 or 1");
    if (p.compensated && p.precision != LBC_FP32_STATE)
        return fail(LBC_EINVAL, "compensated applies to the FP32 state only");
    if (p.half_channel && (p.T_left != p.T_right || p.u_left != -p.u_right))
        return fail(LBC_EINVAL, "the half channel needs symmetric walls: T_left = T_right, u_left = -u_right");
    if (p.precision != LBC_FP64 && p.precision != LBC_FP32_STATE) return fail(LBC_EINVAL, "unknown precision");
    return LBC_OK;
}

namespace {
struct DPiece { const std::vector<double> *src; const double **dst; };
struct FPiece { const std::vector<double> *src; const float **dst; };

// The device table block: FP64 pieces (each padded to 32 doubles), then FP32
// copies (each padded to 64 floats), then the velocity index table.
std::vector<DPiece> dpieces(const ProblemSetup &ps, DevTables &T)
{
    const HostTables &t = ps.t;
    return {{&ps.inv_jdeta, &T.inv_jdeta}, {&ps.jdeta, &T.jdeta}, {&ps.dtn, &T.dtn}, {&t.zx, &T.zx}, {&t.wx, &T.wx}, {&t.yy, &T.yy}, {&t.wy, &T.wy},
            {&t.alpha, &T.alpha}, {&t.sbeta, &T.sbeta}, {&t.hz, &T.hz}, {&t.Yk, &T.Yk}, {&t.Wk, &T.Wk},
            {&t.He, &T.He}, {&ps.fwL, &T.fwL}, {&ps.fwR, &T.fwR}, {&ps.frest, &T.frest}, {&ps.vel, &T.d_vel},
            {&ps.vrow, &T.d_vrow}, {&ps.eqtab, &T.d_eqtab}};
}
std::vector<FPiece> fpieces(const ProblemSetup &ps, DevTables &T)
{
    const HostTables &t = ps.t;
    return {{&t.hz, &T.f_hz}, {&t.He, &T.f_He}, {&t.alpha, &T.f_alpha}, {&ps.isb, &T.f_isbeta},
            {&t.sbeta, &T.f_sbeta}, {&t.Yk, &T.f_Yk}, {&t.Wk, &T.f_Wk}, {&ps.invl, &T.f_inv_l},
            {&ps.vel, &T.f_vel}, {&ps.inv_jdeta, &T.f_inv_jdeta}, {&ps.vrow, &T.f_vrow}, {&ps.eqtab, &T.f_eqtab},
            {&ps.dtn, &T.f_dtn}};
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
    make_grid(p.Nx, p.stretch_A, p.half_channel != 0, ps.x, ps.jdeta, ps.inv_jdeta, ps.deta, ps.min_jdeta);
    ps.mrest = 0.0;
    for (double j : ps.jdeta) ps.mrest += j;

    // table viscosity law (Eqs. mun, interp): segment exponents omega_n, and mu_n
    // divided by mu(T_ref = 1), the viscosity that defines delta
    auto mu_ratio = [&](double Tv) { return std::pow(Tv, p.omega); };
    std::function<double(double)> mu_of = mu_ratio;
    if (p.mu_law == LBC_MU_TABLE) {
        const int nt = p.tab_n;
        ps.tabT.assign(p.tab_T, p.tab_T + nt);
        ps.tabPr.assign(p.tab_Pr, p.tab_Pr + nt);
        ps.tabW.assign(nt, 0.0);
        for (int k = 0; k + 1 < nt; ++k)
            ps.tabW[k] = std::log(p.tab_mu[k + 1] / p.tab_mu[k]) / std::log(p.tab_T[k + 1] / p.tab_T[k]);
        ps.tabW[nt - 1] = ps.tabW[nt - 2];
        auto seg = [&ps, nt](double Tv) {   // the segment of Eq. interp that holds Tv
            int k = (int)(std::upper_bound(ps.tabT.begin(), ps.tabT.end(), Tv) - ps.tabT.begin());
            return std::min(std::max(k - 1, 0), nt - 2);
        };
        const int c1 = seg(1.0);
        const double mu_ref = p.tab_mu[c1] * std::pow(1.0 / p.tab_T[c1], ps.tabW[c1]);
        ps.tabMu.assign(nt, 0.0);
        for (int k = 0; k < nt; ++k) ps.tabMu[k] = p.tab_mu[k] / mu_ref;
        mu_of = [&ps, seg](double Tv) {
            const int c = seg(Tv);
            return ps.tabMu[c] * std::pow(Tv / ps.tabT[c], ps.tabW[c]);
        };
    }

    // time step: CFL on the smallest cell, and half the smallest relaxation time
    // tau = (mu(T)/mu(T_ref)) / (n T delta sqrt(2)) at n = 1 (Eq. tau); local
    // steps take the CFL bound of each node
    double dt = p.dt > 0 ? p.dt : p.cfl * ps.min_jdeta / (t.zx.back() * p.p0);
    double dt_coll = 1e300;
    if (p.dt <= 0 && p.delta > 0)
        for (double Tw : {1.0, p.T_left, p.T_right})
            dt_coll = std::min(dt_coll, 0.5 * mu_of(Tw) / (Tw * p.delta * std::sqrt(2.0)));
    dt = std::min(dt, dt_coll);
    ps.dt = dt;
    ps.dtn.assign(p.Nx, dt);
    if (p.local_dt)
        for (int s = 0; s < p.Nx; ++s)
            ps.dtn[s] = std::min(p.cfl * ps.jdeta[s] / (t.zx.back() * p.p0), dt_coll);

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
        ps.vrow[(size_t)v * kVRow + VR_GA] = ps.aj[v] * kLanes;                  // integer bits, below
        ps.vrow[(size_t)v * kVRow + VR_GJ] = (2 * p.Qx + ps.aj[V + v]) * kLanes;
    }
    if ((int)t.alpha.size() < Nxe + 2 || (int)t.sbeta.size() < Nxe + 2) {
        err = "internal: recurrence table too short";
        return false;
    }
    const int ntab = (int)ps.tabT.size();
    const EqTab E(Nxe, Nye, t.K, p.Qx, p.Qy, ntab);
    ps.eqtab.assign(E.len, 0.0);
    for (int k = 0; k < ntab; ++k) {
        ps.eqtab[E.lawT + k] = ps.tabT[k];
        ps.eqtab[E.lawMu + k] = ps.tabMu[k];
        ps.eqtab[E.lawW + k] = ps.tabW[k];
        ps.eqtab[E.lawPr + k] = ps.tabPr[k];
    }
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
    // the row offsets of the per-velocity rows as integer bit patterns in both copies
    off = 0;
    for (auto &pc : dpieces(ps, dummy)) {
        if (pc.src == &ps.vrow)
            for (int v = 0; v < V; ++v)
                for (int c : {VR_GA, VR_GJ}) {
                    const long long bits = (long long)ps.vrow[(size_t)v * kVRow + c];
                    std::memcpy(ps.blob.data() + (off + (size_t)v * kVRow + c) * sizeof(double), &bits, 8);
                }
        off += pad_d(pc.src->size());
    }
    off = 0;
    for (auto &pc : fpieces(ps, dummy)) {
        if (pc.src == &ps.vrow)
            for (int v = 0; v < V; ++v)
                for (int c : {VR_GA, VR_GJ}) {
                    const int bits = (int)ps.vrow[(size_t)v * kVRow + c];
                    std::memcpy(ps.blob.data() + dbytes + (off + (size_t)v * kVRow + c) * sizeof(float), &bits, 4);
                }
        off += pad_f(pc.src->size());
    }
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
    T.law = p.mu_law;
    T.tab_n = (int)ps.tabT.size();
    T.lts = p.local_dt;
    T.half = p.half_channel;
    T.comp = p.compensated;
    T.mrest = ps.mrest;
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

lbc_status encode_state_map(CUtensorMap *map, void *base, bool fp32, int V, int Nxp, int box_nodes, int box_rows)
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
    cuuint64_t dims[2] = {(cuuint64_t)(2 * Nxp), (cuuint64_t)V};
    cuuint64_t strides[1] = {(cuuint64_t)(2 * Nxp) * esz};
    cuuint32_t box[2] = {(cuuint32_t)(2 * box_nodes), (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = fn(map, fp32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 2, base, dims,
                    strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(LBC_ECUDA, "cuTensorMapEncodeTiled failed (code " + std::to_string((int)r) + ")");
    return LBC_OK;
}

namespace {
// Per-CTA cost outside the row loop (prologue, cluster exchange, equilibrium of
// the CTA's nodes) in units of one velocity row of the main loop: calibrated on
// GB300 from timings of the same batch at several cluster sizes.
constexpr double kCtaOverheadRows = 150.0;

size_t stage_smem(bool fp32, const DevTables &T, int vchunk, int cluster)
{
    return fp32 ? stage_smem_bytes<float>(T.Qx, T.Qy, T.Nxe, T.Nye, T.K, vchunk, cluster, T.tab_n)
                : stage_smem_bytes<double>(T.Qx, T.Qy, T.Nxe, T.Nye, T.K, vchunk, cluster, T.tab_n);
}

int active_clusters(bool fp32, size_t smem, int cluster, bool batch, bool solo = false)
{
    int ncl = 0;
    cudaError_t e = fp32 ? stage_active_clusters<float>(smem, cluster, batch, solo, &ncl)
                         : stage_active_clusters<double>(smem, cluster, batch, solo, &ncl);
    if (e != cudaSuccess) {
        cudaGetLastError();   // an unschedulable cluster shape is not an error of the solver
        return 0;
    }
    return ncl;
}

lbc_status device_limits(bool fp32, const DevTables &T, int &optin)
{
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) return fail(LBC_ECUDA, "no CUDA device");
    cudaError_t e = fp32 ? configure_kernels<float>() : configure_kernels<double>();
    if (e != cudaSuccess) return fail(LBC_ECUDA, std::string("kernel attributes: ") + cudaGetErrorString(e));
    int dev = 0;
    optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    const size_t eqs = fp32 ? equilibrium_smem_bytes<float>(T.Qx, T.Qy, T.Nxe, T.Nye, T.K, T.tab_n)
                            : equilibrium_smem_bytes<double>(T.Qx, T.Qy, T.Nxe, T.Nye, T.K, T.tab_n);
    if (eqs > (size_t)optin)
        return fail(LBC_EINVAL, "quadrature orders too large for the shared memory of one CTA (" +
                                    std::to_string(eqs) + " bytes)");
    return LBC_OK;
}
}  // namespace

size_t stage_launch_smem(bool fp32, const DevTables &T) { return stage_smem(fp32, T, T.vchunk, T.nchunk); }

// Velocity chunks per tile (multiples of the pipeline's kSubV rows, at most
// kMaxCluster chunks: they form one cluster): the count that minimises a wave
// model of the launch, waves x (rows per CTA + per-CTA overhead), with the
// clusters the device can hold at once.
lbc_status choose_launch_shape(bool fp32, DevTables &T)
{
    int optin = 0;
    lbc_status st = device_limits(fp32, T, optin);
    if (st != LBC_OK) return st;
    const int subs = std::min((T.V + kSubV - 1) / kSubV, kMaxVChunk / kSubV);
    double best = 1e300;
    T.vchunk = T.nchunk = 0;
    for (int nsub = 1; nsub <= subs; ++nsub) {
        const int vch = nsub * kSubV, nch = (T.V + vch - 1) / vch;
        if (nch > kMaxCluster) continue;
        const size_t smem = stage_smem(fp32, T, vch, nch);
        if (smem > (size_t)optin) continue;
        const int ncl = active_clusters(fp32, smem, nch, false);
        if (ncl <= 0) continue;
        const double waves = std::ceil((double)T.ntile / ncl);
        const double cost = waves * (vch + kCtaOverheadRows);
        if (cost < best - 1e-9) { best = cost; T.vchunk = vch; T.nchunk = nch; }
    }
    if (T.nchunk == 0)
        return fail(LBC_EINVAL, "no schedulable cluster shape for a velocity set of " + std::to_string(T.V));
    return LBC_OK;
}

// Cluster size of a batch (every instance split into `cluster` chunk CTAs per
// tile): the size that minimises a wave model of the whole work list, total
// rows (plus a per-CTA overhead) over the CTAs the device holds at once, plus
// the longest single CTA. cluster_in > 0 forces the size (if it fits).
// solo_in: 1 the solo form (independent CTAs, no cluster scheduling constraint),
// 0 the cluster form, -1 the solo form when its work list fills the device at
// least once (its tiles' last CTAs then overlap the other tiles' streaming), else
// the cluster form (whose node step is spread over the cluster).
lbc_status choose_batch_shape(bool fp32, std::vector<DevTables> &Ts, int cluster_in, int solo_in, bool &solo,
                              int &cluster, size_t &smem)
{
    int optin = 0;
    for (const DevTables &T : Ts) {
        lbc_status st = device_limits(fp32, T, optin);
        if (st != LBC_OK) return st;
    }
    struct Shape {
        int C = 0;
        size_t smem = 0;
        double ctas = 0, resident = 0;
    };
    auto model = [&](bool form_solo) {
        Shape best;
        double best_cost = 1e300;
        for (int C = 1; C <= kMaxCluster; ++C) {
            if (cluster_in > 0 && C != cluster_in) continue;
            size_t smax = 0;
            double rows = 0, longest = 0, tiles = 0;
            bool fits = true;
            for (const DevTables &T : Ts) {
                const int vch = chunk_rows(T.V, C);
                if (vch > kMaxVChunk) { fits = false; break; }
                smax = std::max(smax, stage_smem(fp32, T, vch, C));
                rows += (double)T.ntile * C * (vch + kCtaOverheadRows);
                longest = std::max(longest, vch + kCtaOverheadRows);
                tiles += T.ntile;
            }
            if (!fits || smax > (size_t)optin) continue;
            const int ncl = active_clusters(fp32, smax, C, true, form_solo);
            if (ncl <= 0) continue;
            const double cost = rows / ((double)ncl * C) + longest;
            if (cost < best_cost - 1e-9) {
                best_cost = cost;
                best.C = C;
                best.smem = smax;
                best.ctas = tiles * C;
                best.resident = (double)ncl * C;
            }
        }
        return best;
    };
    Shape pick;
    if (solo_in >= 0) {
        solo = solo_in > 0;
        pick = model(solo);
    } else {
        const Shape s1 = model(true);
        solo = s1.C > 0 && s1.ctas >= s1.resident;
        pick = solo ? s1 : model(false);
    }
    cluster = pick.C;
    smem = pick.smem;
    if (cluster == 0) return fail(LBC_EINVAL, "no schedulable cluster shape for this batch");
    for (DevTables &T : Ts) {
        T.nchunk = cluster;
        T.vchunk = chunk_rows(T.V, cluster);
    }
    return LBC_OK;
}

// Solo-form batch shape with full chunks: every instance's velocity set in chunks of
// kMaxVChunk rows (the last one shorter), C = the most chunks of any instance. A tile's last
// chunk, which the dispatch order puts in the launch's last wave, then has the fewest rows,
// so the tiles' node steps start earlier (measured 72 against 74 us per stage launch on four
// C2 solves); offered to the autotuner beside the balanced shapes.
lbc_status choose_full_chunk_shape(bool fp32, std::vector<DevTables> &Ts, int &cluster, size_t &smem)
{
    int optin = 0;
    cluster = 0;
    smem = 0;
    for (const DevTables &T : Ts) {
        lbc_status st = device_limits(fp32, T, optin);
        if (st != LBC_OK) return st;
    }
    for (DevTables &T : Ts) {
        const int vch = std::min(kMaxVChunk, (T.V + kSubV - 1) / kSubV * kSubV);
        cluster = std::max(cluster, (T.V + vch - 1) / vch);
    }
    if (cluster > kMaxCluster) return fail(LBC_EINVAL, "velocity set too large for full chunks");
    for (DevTables &T : Ts) {
        T.nchunk = cluster;
        T.vchunk = std::min(kMaxVChunk, (T.V + kSubV - 1) / kSubV * kSubV);
        smem = std::max(smem, stage_smem(fp32, T, T.vchunk, cluster));
    }
    if (smem > (size_t)optin) return fail(LBC_EINVAL, "full chunks do not fit the shared memory of one CTA");
    if (active_clusters(fp32, smem, cluster, true, true) <= 0) return fail(LBC_EINVAL, "full chunks not launchable");
    return LBC_OK;
}

}  // namespace lbc

using namespace lbc;

extern "C" {

const char *lbc_last_error(void) { return last_error(); }

int lbc_checked_build(void) { return checked_build() ? 1 : 0; }

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

}  // extern "C"
