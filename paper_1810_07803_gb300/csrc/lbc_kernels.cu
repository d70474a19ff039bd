// Fused RK-3 stage kernel of the half-range LB Couette solver (sm_103a).
//
// One CTA owns a tile of 32 nodes x one chunk of the velocity set, both fields.
// Per stage it: (1) sums the raw moment partials of its nodes written by the
// previous stage and turns them into n, u, T, P, q (Sec. II); (2) builds the
// discrete equilibrium factors g_x, g_y of every node (Eqs. gx, gy) with one
// warp per node; (3) on a wall tile, computes the wall density n_w from the
// outgoing WENO-5 wall flux (Eqs. diffuse, diffuse_nw); (4) streams its
// velocity rows: WENO-5 faces (upwind by sign p_x), Shakhov target (Sec. II),
// relaxation with 1/tau from Eq. tau, TVD RK-3 combination, store; (5) reduces
// the new stage's raw moments over its velocities for the next stage; on the
// last stage also the residual max w |f^{n+1} - f^n|.
#include <cstdint>

#include "lbc_device.h"

namespace lbc {

namespace {

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// WENO-5 (Jiang & Shu) face value between c and d, upwind cell c.
template <typename R>
__device__ __forceinline__ R weno5(R a, R b, R c, R d, R e)
{
    const R eps = R(1e-6);
    R q0 = (R(2) * a - R(7) * b + R(11) * c) * R(1.0 / 6.0);
    R q1 = (-b + R(5) * c + R(2) * d) * R(1.0 / 6.0);
    R q2 = (R(2) * c + R(5) * d - e) * R(1.0 / 6.0);
    R t0 = a - R(2) * b + c, t1 = a - R(4) * b + R(3) * c;
    R t2 = b - R(2) * c + d, t3 = b - d;
    R t4 = c - R(2) * d + e, t5 = R(3) * c - R(4) * d + e;
    R b0 = R(13.0 / 12.0) * t0 * t0 + R(0.25) * t1 * t1;
    R b1 = R(13.0 / 12.0) * t2 * t2 + R(0.25) * t3 * t3;
    R b2 = R(13.0 / 12.0) * t4 * t4 + R(0.25) * t5 * t5;
    R e0 = eps + b0, e1 = eps + b1, e2 = eps + b2;
    e0 *= e0; e1 *= e1; e2 *= e2;
    // alpha_k = d_k / e_k: multiply through by e0 e1 e2 to need one division
    R a0 = R(0.1) * e1 * e2, a1 = R(0.6) * e0 * e2, a2 = R(0.3) * e0 * e1;
    return (a0 * q0 + a1 * q1 + a2 * q2) / (a0 + a1 + a2);
}

// Moments (n, u_x, u_y, T, P_xx, P_yy, P_zz, P_xy, q_x, q_y) from raw sums about shift (sx, sy).
__device__ void raw_to_moments(const double *r, double sx, double sy, double *m)
{
    double n = r[R_S0];
    double bx = r[R_SX] / n, by = r[R_SY] / n;
    double pxx = r[R_SXX] - n * bx * bx;
    double pxy = r[R_SXY] - n * bx * by;
    double pyy = r[R_SYY] - n * by * by;
    double pzz = r[R_CZ];
    double r2 = r[R_SXX] + r[R_SYY], b2 = bx * bx + by * by;
    double hx = r[R_R3X] - bx * r2 - 2.0 * (bx * r[R_SXX] + by * r[R_SXY]) + 2.0 * n * bx * b2;
    double hy = r[R_R3Y] - by * r2 - 2.0 * (bx * r[R_SXY] + by * r[R_SYY]) + 2.0 * n * by * b2;
    m[0] = n;
    m[1] = sx + bx;
    m[2] = sy + by;
    m[3] = (pxx + pyy + pzz) / (3.0 * n);
    m[4] = pxx; m[5] = pyy; m[6] = pzz; m[7] = pxy;
    m[8] = 0.5 * hx + 0.5 * (r[R_GX] - bx * pzz);
    m[9] = 0.5 * hy + 0.5 * (r[R_GY] - by * pzz);
}

// Velocity v -> (p_x, p_y, w, a, j).
__device__ __forceinline__ void velocity(const DevTables &T, int v, double &px, double &py, double &w, int &a, int &j)
{
    a = v / T.Qy;
    j = v - a * T.Qy;
    int i = a < T.Qx ? a : a - T.Qx;
    px = (a < T.Qx ? 1.0 : -1.0) * T.p0 * T.zx[i];
    py = T.p0 * T.yy[j];
    w = T.wx[i] * T.wy[j];
}

// Warp-cooperative discrete equilibrium of one node: gx[2Qx], gy[Qy] (see the
// host version for the algorithm). cbuf: per-warp scratch [2 (Nxe+1)].
template <typename R>
__device__ void warp_equilibrium(const DevTables &T, double ux, double uy, double Tc, R *gx, R *gy,
                                 double *cbuf)
{
    const int lane = threadIdx.x & 31, N = T.Nxe;
    double Tp = Tc / (T.p0 * T.p0), up = ux / T.p0, sT = sqrt(Tp), a = up / sT;
    double zt[2], rp[2], rm[2], hprev[2], h[2];
#pragma unroll
    for (int q = 0; q < 2; ++q) {
        int k = lane + 32 * q;
        bool ok = k < T.K;
        double Y = ok ? T.Yk[k] : 0.0, W = ok ? T.Wk[k] : 0.0;
        zt[q] = sT * Y;
        rp[q] = W * exp(a * Y - 0.5 * a * a);
        rm[q] = W * exp(-a * Y - 0.5 * a * a);
        hprev[q] = 0.0;
        h[q] = 1.0 / T.sbeta[0];
    }
    for (int l = 0; l <= N; ++l) {
        double vp = rp[0] * h[0] + rp[1] * h[1];
        double vm = rm[0] * h[0] + rm[1] * h[1];
        vp = warp_sum(vp);
        vm = warp_sum(vm);
        if (lane == 0) { cbuf[l] = vp; cbuf[N + 1 + l] = vm; }
        double al = T.alpha[l], sb = T.sbeta[l], sb1 = T.sbeta[l + 1];
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            double hn = ((zt[q] - al) * h[q] - sb * hprev[q]) / sb1;
            hprev[q] = h[q];
            h[q] = hn;
        }
    }
    __syncwarp();
    for (int i = lane; i < 2 * T.Qx; i += 32) {
        int ii = i < T.Qx ? i : i - T.Qx;
        const double *c = cbuf + (i < T.Qx ? 0 : N + 1);
        double s = 0.0;
        for (int l = 0; l <= N; ++l) s += T.hz[l * T.Qx + ii] * c[l];
        gx[i] = R(s);
    }
    double uq = uy / T.p0;
    for (int jj = lane; jj < T.Qy; jj += 32) {
        double bm = 1.0, b = uq;
        double s = T.He[jj];                      // l = 0
        if (T.Nye >= 1) s += T.He[T.Qy + jj] * b;
        for (int l = 1; l < T.Nye; ++l) {
            double bn = (uq * b + (Tp - 1.0) * bm) / (l + 1.0);
            bm = b;
            b = bn;
            s += T.He[(l + 1) * T.Qy + jj] * b;
        }
        gy[jj] = R(s);
    }
    __syncwarp();
}

// Outgoing WENO-5 wall face of phi at the left (px < 0) or right (px > 0) wall,
// with two ghost nodes by cubic extrapolation in eta from the four nearest nodes.
template <typename R>
__device__ __forceinline__ R outgoing_wall_face(const R *row, int Nx, bool right)
{
    if (right) {
        R f1 = row[Nx - 1], f2 = row[Nx - 2], f3 = row[Nx - 3], f4 = row[Nx - 4];
        R g1 = R(4) * f1 - R(6) * f2 + R(4) * f3 - f4;
        R g2 = R(10) * f1 - R(20) * f2 + R(15) * f3 - R(4) * f4;
        return weno5<R>(f3, f2, f1, g1, g2);
    }
    R f1 = row[0], f2 = row[1], f3 = row[2], f4 = row[3];
    R g1 = R(4) * f1 - R(6) * f2 + R(4) * f3 - f4;
    R g2 = R(10) * f1 - R(20) * f2 + R(15) * f3 - R(4) * f4;
    return weno5<R>(f3, f2, f1, g1, g2);
}

template <typename R>
struct StageSmem {
    double raw[kTileCells][kNumRaw + 1];
    double mom[kTileCells][12];     // n ux uy T qx qy nu cS (+pad)
    double cbuf[kWarps][2 * kMaxQ + 2];
    double red[kWarps][kNumRaw][kTileCells];
    double wsum[kWarps];
    double nw[2];
    R row[kWarps][2][kTileCells + 8];
    R gx[kTileCells][2 * kMaxQ];
    R gy[kTileCells][kMaxQ];
};

__device__ __forceinline__ double collision_rate(const DevTables &T, double n, double Tc)
{
    return n * T.delta * 1.4142135623730951 * pow(Tc, 1.0 - T.omega);
}

template <typename R>
__device__ void block_wall_density(const DevTables &T, const R *phi, bool right, double *wsum, double *out)
{
    // outgoing velocities: right wall p_x > 0 -> a < Qx; left wall p_x < 0 -> a >= Qx
    const int half = T.Qx * T.Qy;
    const int vbeg = right ? 0 : half;
    double acc = 0.0;
    for (int v = vbeg + threadIdx.x; v < vbeg + half; v += blockDim.x) {
        double px, py, w;
        int a, j;
        velocity(T, v, px, py, w, a, j);
        R face = outgoing_wall_face<R>(phi + (size_t)v * T.Nxp, T.Nx, right);
        acc += px * w * (double)face;
    }
    acc = warp_sum(acc);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) wsum[warp] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < kWarps; ++w) s += wsum[w];
        *out = -s / (right ? T.inR : T.inL);
    }
    __syncthreads();
}

template <typename R>
__global__ void __launch_bounds__(kThreads)
stage_kernel(DevTables T, DevState S, int stage, int rel, double stop_eps)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    StageSmem<R> &sm = *reinterpret_cast<StageSmem<R> *>(smem_raw);

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int c0 = blockIdx.x * kTileCells;
    const int chunk = blockIdx.y;
    const int in = stage, out = (stage + 1) % 3;
    const long long step = S.ctl->base + rel;

    // ---- early stop (run-to-steady): every block takes the same decision ----
    if (stop_eps > 0.0) {
        if (S.ctl->stopped) return;
        if (step - 1 >= S.ctl->check_from) {
            double rprev = __longlong_as_double((long long)S.resid[(step - 1) % kResidRing]);
            if (rprev < stop_eps) {
                if (stage == 0 && blockIdx.x == 0 && blockIdx.y == 0 && tid == 0) S.ctl->stopped = 1;
                return;
            }
        }
    }
    if (stage == 0 && blockIdx.x == 0 && blockIdx.y == 0 && tid == 0) S.resid[step % kResidRing] = 0ull;

    const R *Fin = static_cast<const R *>(S.F[in]);
    const R *F0 = static_cast<const R *>(S.F[0]);
    R *Fout = static_cast<R *>(S.F[out]);
    const size_t fstride = (size_t)T.V * T.Nxp;

    // ---- (1) stage-input moments of the tile's nodes ----
    for (int idx = tid; idx < kTileCells * kNumRaw; idx += kThreads) {
        int c = idx % kTileCells, m = idx / kTileCells, s = c0 + c;
        double acc = 0.0;
        if (s < T.Nx)
            for (int ch = 0; ch < T.nchunk; ++ch) acc += S.part[in][((size_t)ch * kNumRaw + m) * T.Nxp + s];
        sm.raw[c][m] = acc;
    }
    __syncthreads();
    if (tid < kTileCells) {
        int s = c0 + tid;
        double m[10];
        if (s < T.Nx) {
            raw_to_moments(sm.raw[tid], S.shift[in][s], S.shift[in][T.Nxp + s], m);
        } else {
            m[0] = 1.0; m[1] = m[2] = 0.0; m[3] = 1.0; m[8] = m[9] = 0.0;
        }
        sm.mom[tid][0] = m[0]; sm.mom[tid][1] = m[1]; sm.mom[tid][2] = m[2]; sm.mom[tid][3] = m[3];
        sm.mom[tid][4] = m[8]; sm.mom[tid][5] = m[9];
        sm.mom[tid][6] = collision_rate(T, m[0], m[3]);
        sm.mom[tid][7] = (1.0 - T.Pr) / (m[0] * m[3] * m[3]);
    }
    __syncthreads();

    // ---- (2) discrete equilibrium of each node: one warp per node ----
    for (int c = warp; c < kTileCells; c += kWarps)
        warp_equilibrium<R>(T, sm.mom[c][1], sm.mom[c][2], sm.mom[c][3], sm.gx[c], sm.gy[c], sm.cbuf[warp]);

    // ---- (3) wall densities (tiles whose 3-node halo reaches a wall) ----
    const bool needL = c0 == 0;
    const bool needR = c0 + kTileCells + 3 > T.Nx;
    if (needL) block_wall_density<R>(T, Fin, false, sm.wsum, &sm.nw[0]);
    if (needR) block_wall_density<R>(T, Fin, true, sm.wsum, &sm.nw[1]);
    __syncthreads();

    // ---- (4) stream the chunk's velocity rows ----
    const double ca = stage == 0 ? 0.0 : (stage == 1 ? 0.75 : 1.0 / 3.0);
    const double cb = stage == 0 ? 1.0 : (stage == 1 ? 0.25 : 2.0 / 3.0);
    const int s = c0 + lane;
    const bool active = s < T.Nx;
    const double n_c = sm.mom[lane][0], ux_c = sm.mom[lane][1], uy_c = sm.mom[lane][2];
    const double T_c = sm.mom[lane][3], qx_c = sm.mom[lane][4], qy_c = sm.mom[lane][5];
    const double nu_c = sm.mom[lane][6], cS_c = sm.mom[lane][7];
    const double ijd = active ? T.inv_jdeta[s] : 0.0;
    const double nwL = needL ? sm.nw[0] : 0.0;
    const double nwR = needR ? sm.nw[1] : 0.0;

    double acc[kNumRaw];
#pragma unroll
    for (int m = 0; m < kNumRaw; ++m) acc[m] = 0.0;
    double res = 0.0;
    bool bad = false;

    const int vbeg = chunk * T.vchunk;
    const int vend = min(T.V, vbeg + T.vchunk);
    for (int v = vbeg + warp; v < vend; v += kWarps) {
        double px, py, w;
        int a, j;
        velocity(T, v, px, py, w, a, j);
        double fo[2];
        for (int fld = 0; fld < 2; ++fld) {
            const R *row = Fin + fld * fstride + (size_t)v * T.Nxp;
            R *buf = sm.row[warp][fld];
            // buffer index b <-> node c0 - 3 + b, b in [0, 38)
            for (int b = lane; b < kTileCells + 6; b += 32) {
                int sn = c0 - 3 + b;
                buf[b] = (sn >= 0 && sn < T.Nx) ? row[sn] : R(0);
            }
            __syncwarp();
            if (lane < 2) {
                if (c0 == 0) {            // left ghosts: nodes -1 (b = 2), -2 (b = 1)
                    int b = 2 - lane;
                    R g;
                    if (px > 0) {
                        g = R(nwL * T.fwL[v] * (fld ? T.TL : 1.0));
                    } else {
                        R f1 = buf[3], f2 = buf[4], f3 = buf[5], f4 = buf[6];
                        g = lane == 0 ? R(4) * f1 - R(6) * f2 + R(4) * f3 - f4
                                      : R(10) * f1 - R(20) * f2 + R(15) * f3 - R(4) * f4;
                    }
                    buf[b] = g;
                }
                int bR = T.Nx - c0 + 3 + lane;   // right ghosts: nodes Nx (lane 0), Nx+1 (lane 1)
                if (bR < kTileCells + 6) {
                    R g;
                    if (px < 0) {
                        g = R(nwR * T.fwR[v] * (fld ? T.TR : 1.0));
                    } else {
                        int bl = T.Nx - 1 - c0 + 3;
                        R f1 = buf[bl], f2 = buf[bl - 1], f3 = buf[bl - 2], f4 = buf[bl - 3];
                        g = lane == 0 ? R(4) * f1 - R(6) * f2 + R(4) * f3 - f4
                                      : R(10) * f1 - R(20) * f2 + R(15) * f3 - R(4) * f4;
                    }
                    buf[bR] = g;
                }
            }
            __syncwarp();
            // face k = c0 + lane (left of node s); buffer index of node k is lane + 3
            auto face = [&](int k, int bk) -> R {
                if (px > 0) {
                    if (k == 0) return R(nwL * T.fwL[v] * (fld ? T.TL : 1.0));
                    return weno5<R>(buf[bk - 3], buf[bk - 2], buf[bk - 1], buf[bk], buf[bk + 1]);
                }
                if (k == T.Nx) return R(nwR * T.fwR[v] * (fld ? T.TR : 1.0));
                return weno5<R>(buf[bk + 2], buf[bk + 1], buf[bk], buf[bk - 1], buf[bk - 2]);
            };
            R fl = face(c0 + lane, lane + 3);
            R fr = __shfl_down_sync(0xffffffffu, fl, 1);
            if (lane == 31) fr = face(c0 + 32, 35);
            __syncwarp();
            double f = (double)buf[lane + 3];
            double adv = -px * ((double)fr - (double)fl) * ijd;
            double feq = n_c * (double)sm.gx[lane][a] * (double)sm.gy[lane][j];
            double xx = px - ux_c, xy = py - uy_c;
            double qxi = qx_c * xx + qy_c * xy;
            double x2 = (xx * xx + xy * xy) / (5.0 * T_c);
            double tgt = fld ? T_c * feq * (1.0 + cS_c * (x2 - 0.4) * qxi)
                             : feq * (1.0 + cS_c * (x2 - 0.8) * qxi);
            double L = adv - nu_c * (f - tgt);
            double fn = f + T.dt * L;
            double f0v = 0.0;
            if (stage > 0 && active) {
                f0v = (double)F0[fld * fstride + (size_t)v * T.Nxp + s];
                fn = ca * f0v + cb * fn;
            }
            R fnr = R(fn);
            if (active) {
                Fout[fld * fstride + (size_t)v * T.Nxp + s] = fnr;
                if (!isfinite((double)fnr)) bad = true;
                if (stage == 2) res = fmax(res, w * fabs((double)fnr - f0v));
            }
            fo[fld] = (double)fnr;
        }
        if (active) {
            double xs = px - ux_c, ys = py - uy_c;
            double fw = w * fo[0], gw = w * fo[1];
            double e2 = xs * xs + ys * ys;
            acc[R_S0] += fw;
            acc[R_SX] += xs * fw;
            acc[R_SY] += ys * fw;
            acc[R_SXX] += xs * xs * fw;
            acc[R_SXY] += xs * ys * fw;
            acc[R_SYY] += ys * ys * fw;
            acc[R_CZ] += gw;
            acc[R_R3X] += e2 * xs * fw;
            acc[R_R3Y] += e2 * ys * fw;
            acc[R_GX] += xs * gw;
            acc[R_GY] += ys * gw;
        }
    }

    // ---- (5) reduce the new stage's raw moments and the residual ----
#pragma unroll
    for (int m = 0; m < kNumRaw; ++m) sm.red[warp][m][lane] = acc[m];
    __syncthreads();
    for (int idx = tid; idx < kTileCells * kNumRaw; idx += kThreads) {
        int c = idx % kTileCells, m = idx / kTileCells, sn = c0 + c;
        double t = 0.0;
        for (int w2 = 0; w2 < kWarps; ++w2) t += sm.red[w2][m][c];
        if (sn < T.Nx) S.part[out][((size_t)chunk * kNumRaw + m) * T.Nxp + sn] = t;
    }
    if (chunk == 0 && active) {
        S.shift[out][s] = ux_c;
        S.shift[out][T.Nxp + s] = uy_c;
    }
    if (bad) S.ctl->nonfinite = 1;
    if (stage == 2) {
        for (int o = 16; o > 0; o >>= 1) res = fmax(res, __shfl_xor_sync(0xffffffffu, res, o));
        if (lane == 0 && res > 0.0) atomicMax(&S.resid[step % kResidRing], (unsigned long long)__double_as_longlong(res));
    }
}

// Raw moment sums (shift 0) of state buffer `buf`.
template <typename R>
__global__ void __launch_bounds__(kThreads) moments_partial_kernel(DevTables T, DevState S, int buf)
{
    __shared__ double red[kWarps][kNumRaw][kTileCells];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int c0 = blockIdx.x * kTileCells, chunk = blockIdx.y, s = c0 + lane;
    const bool active = s < T.Nx;
    const R *F = static_cast<const R *>(S.F[buf]);
    const size_t fstride = (size_t)T.V * T.Nxp;
    double acc[kNumRaw];
#pragma unroll
    for (int m = 0; m < kNumRaw; ++m) acc[m] = 0.0;
    const int vbeg = chunk * T.vchunk, vend = min(T.V, vbeg + T.vchunk);
    for (int v = vbeg + warp; v < vend && active; v += kWarps) {
        double px, py, w;
        int a, j;
        velocity(T, v, px, py, w, a, j);
        double fw = w * (double)F[(size_t)v * T.Nxp + s];
        double gw = w * (double)F[fstride + (size_t)v * T.Nxp + s];
        double e2 = px * px + py * py;
        acc[R_S0] += fw; acc[R_SX] += px * fw; acc[R_SY] += py * fw;
        acc[R_SXX] += px * px * fw; acc[R_SXY] += px * py * fw; acc[R_SYY] += py * py * fw;
        acc[R_CZ] += gw; acc[R_R3X] += e2 * px * fw; acc[R_R3Y] += e2 * py * fw;
        acc[R_GX] += px * gw; acc[R_GY] += py * gw;
    }
#pragma unroll
    for (int m = 0; m < kNumRaw; ++m) red[warp][m][lane] = acc[m];
    __syncthreads();
    for (int idx = tid; idx < kTileCells * kNumRaw; idx += kThreads) {
        int c = idx % kTileCells, m = idx / kTileCells, sn = c0 + c;
        double t = 0.0;
        for (int w2 = 0; w2 < kWarps; ++w2) t += red[w2][m][c];
        if (sn < T.Nx) S.part[buf][((size_t)chunk * kNumRaw + m) * T.Nxp + sn] = t;
    }
    if (chunk == 0 && active) {
        S.shift[buf][s] = 0.0;
        S.shift[buf][T.Nxp + s] = 0.0;
    }
}

template <typename R>
__global__ void init_rest_kernel(DevTables T, DevState S)
{
    R *F = static_cast<R *>(S.F[0]);
    const size_t n = (size_t)T.V * T.Nxp;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < 2 * n; i += (size_t)gridDim.x * blockDim.x) {
        size_t k = i % n;
        int v = (int)(k / T.Nxp), s = (int)(k % T.Nxp);
        F[i] = s < T.Nx ? R(T.frest[v]) : R(0);
    }
}

__global__ void finalize_moments_kernel(DevTables T, DevState S, int buf)
{
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= T.Nx) return;
    double r[kNumRaw];
    for (int m = 0; m < kNumRaw; ++m) {
        double acc = 0.0;
        for (int ch = 0; ch < T.nchunk; ++ch) acc += S.part[buf][((size_t)ch * kNumRaw + m) * T.Nxp + s];
        r[m] = acc;
    }
    double mo[10];
    raw_to_moments(r, S.shift[buf][s], S.shift[buf][T.Nxp + s], mo);
    for (int k = 0; k < LBC_NMOM; ++k) S.mom_out[(size_t)k * T.Nxp + s] = mo[k];
}

__global__ void ctl_set_kernel(Ctl *ctl, long long base, long long check_from, int stopped)
{
    ctl->base = base;
    ctl->check_from = check_from;
    ctl->stopped = stopped;
    ctl->nonfinite = 0;
}

__global__ void ctl_bump_kernel(Ctl *ctl, long long k) { ctl->base += k; }

}  // namespace

template <typename R>
cudaError_t configure_kernels()
{
    return cudaFuncSetAttribute(stage_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)sizeof(StageSmem<R>));
}

template <typename R>
cudaError_t launch_stage(const DevTables &T, const DevState &S, int stage, int rel, double stop_eps, cudaStream_t st)
{
    size_t smem = sizeof(StageSmem<R>);
    dim3 grid(T.ntile, T.nchunk);
    stage_kernel<R><<<grid, kThreads, smem, st>>>(T, S, stage, rel, stop_eps);
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_moments_partial(const DevTables &T, const DevState &S, int buf, cudaStream_t st)
{
    dim3 grid(T.ntile, T.nchunk);
    moments_partial_kernel<R><<<grid, kThreads, 0, st>>>(T, S, buf);
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_init_rest(const DevTables &T, const DevState &S, cudaStream_t st)
{
    init_rest_kernel<R><<<304, 256, 0, st>>>(T, S);
    return cudaGetLastError();
}

cudaError_t launch_finalize_moments(const DevTables &T, const DevState &S, int buf, cudaStream_t st)
{
    finalize_moments_kernel<<<(T.Nx + 127) / 128, 128, 0, st>>>(T, S, buf);
    return cudaGetLastError();
}

cudaError_t launch_ctl_set(Ctl *ctl, long long base, long long check_from, int stopped, cudaStream_t st)
{
    ctl_set_kernel<<<1, 1, 0, st>>>(ctl, base, check_from, stopped);
    return cudaGetLastError();
}

cudaError_t launch_ctl_bump(Ctl *ctl, long long k, cudaStream_t st)
{
    ctl_bump_kernel<<<1, 1, 0, st>>>(ctl, k);
    return cudaGetLastError();
}

template cudaError_t configure_kernels<double>();
template cudaError_t configure_kernels<float>();
template cudaError_t launch_stage<double>(const DevTables &, const DevState &, int, int, double, cudaStream_t);
template cudaError_t launch_stage<float>(const DevTables &, const DevState &, int, int, double, cudaStream_t);
template cudaError_t launch_moments_partial<double>(const DevTables &, const DevState &, int, cudaStream_t);
template cudaError_t launch_moments_partial<float>(const DevTables &, const DevState &, int, cudaStream_t);
template cudaError_t launch_init_rest<double>(const DevTables &, const DevState &, cudaStream_t);
template cudaError_t launch_init_rest<float>(const DevTables &, const DevState &, cudaStream_t);

}  // namespace lbc
