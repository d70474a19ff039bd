// Fused RK-3 stage kernel of the half-range LB Couette solver (sm_103a).
//
// One CTA owns a tile of 31 nodes (lane l: node c0 + l and the face on its
// left, so each lane computes one WENO-5 face per row) x one chunk of the
// velocity set, both fields; the chunk CTAs of a tile form one thread-block
// cluster. Per stage a CTA:
//  (1) reads its nodes' stage data (moments, 1/tau, Shakhov prefactor) and
//      discrete equilibrium factors g_x, g_y (Eqs. gx, gy), built by the
//      previous stage (or at set-up);
//  (2) on a tile whose stencil reaches a wall, computes the wall density n_w
//      from the outgoing WENO-5 wall flux (Eqs. diffuse, diffuse_nw);
//  (3) streams the chunk's velocity rows through a TMA pipeline (kPipe slots
//      of kSubV rows, kSubV0 in the first FP32 stage; mbarrier completion):
//      WENO-5 faces upwind by sign p_x,
//      Shakhov target (Sec. II) with 1/tau of Eq. tau, TVD RK-3 combination,
//      store, and the new stage's raw moments over the chunk's velocities;
//  (4) publishes its per-chunk moment partials in shared memory; after a
//      cluster barrier, CTA r of the cluster sums the partials of nodes
//      r, r + nchunk, ... over all chunks (distributed shared memory) and
//      builds their next-stage data (moments, equilibrium factors by the
//      stable Gauss-sum projection). On the last stage it also folds the
//      residual max w |f^{n+1} - f^n|.
// A second form of the kernels (kExt) adds what only some instances use: the
// half channel's symmetry plane (ghosts from the opposite velocity), local
// pseudo-time steps (each node's own step, the third stage's mass
// renormalisation) and the compensated FP32 state (the third stage adds the
// step's increment to d + c by TwoSum).
// The state is the deviation d = ft - ft_rest from the weight-divided rest
// Maxwellian (n = 1, u = 0, T = 1): WENO-5, the ghost extrapolation and the RK
// combination are affine-invariant, so they act on d unchanged, and the FP32
// path keeps ~1e-8 absolute resolution for near-equilibrium flows.
#include <algorithm>
#include <cstdint>
#include <type_traits>

#include "lbc_device.h"

namespace lbc {

namespace {

constexpr long kSpinLimit = 1L << 22;   // bounded mbarrier wait (try_wait suspends per call)

template <typename R> struct Tabs;
template <> struct Tabs<double> {
    __device__ static const double *vel(const DevTables &T) { return T.d_vel; }
    __device__ static const double *hz(const DevTables &T) { return T.hz; }
    __device__ static const double *He(const DevTables &T) { return T.He; }
    __device__ static const double *alpha(const DevTables &T) { return T.alpha; }
    __device__ static const double *Yk(const DevTables &T) { return T.Yk; }
    __device__ static const double *Wk(const DevTables &T) { return T.Wk; }
    __device__ static const double *ijd(const DevTables &T) { return T.inv_jdeta; }
    __device__ static const double *dtn(const DevTables &T) { return T.dtn; }
    __device__ static double sbeta(const DevTables &T, int l) { return T.sbeta[l]; }
    __device__ static double isbeta(const DevTables &T, int l) { return 1.0 / T.sbeta[l]; }
    __device__ static double inv_l(const DevTables &, int l) { return 1.0 / l; }
    __device__ static double sc(const DevTables &T, int k) { return T.dsc[k]; }
    __device__ static const double *vrow(const DevTables &T) { return T.d_vrow; }
    __device__ static const double *eqtab(const DevTables &T) { return T.d_eqtab; }
    __device__ static double restP(const DevTables &T, int k) { return T.restP[k]; }
};
template <> struct Tabs<float> {
    __device__ static const float *vel(const DevTables &T) { return T.f_vel; }
    __device__ static const float *hz(const DevTables &T) { return T.f_hz; }
    __device__ static const float *He(const DevTables &T) { return T.f_He; }
    __device__ static const float *alpha(const DevTables &T) { return T.f_alpha; }
    __device__ static const float *Yk(const DevTables &T) { return T.f_Yk; }
    __device__ static const float *Wk(const DevTables &T) { return T.f_Wk; }
    __device__ static const float *ijd(const DevTables &T) { return T.f_inv_jdeta; }
    __device__ static const float *dtn(const DevTables &T) { return T.f_dtn; }
    __device__ static float sbeta(const DevTables &T, int l) { return T.f_sbeta[l]; }
    __device__ static float isbeta(const DevTables &T, int l) { return T.f_isbeta[l]; }
    __device__ static float inv_l(const DevTables &T, int l) { return T.f_inv_l[l]; }
    __device__ static float sc(const DevTables &T, int k) { return T.fsc[k]; }
    __device__ static const float *vrow(const DevTables &T) { return T.f_vrow; }
    __device__ static const float *eqtab(const DevTables &T) { return T.f_eqtab; }
    __device__ static float restP(const DevTables &T, int k) { return T.f_restP[k]; }
};

// ---- compensated arithmetic (error-free transformations of Knuth and Dekker) ----
template <typename R>
__device__ __forceinline__ void two_sum(R a, R b, R &s, R &e)
{
    s = a + b;
    R bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

// Sum with a compensation term in FP32 (TwoSum of Knuth); plain in FP64.
template <typename R>
struct CSum {
    R s = R(0), c = R(0);
    __device__ __forceinline__ void add(R x)
    {
        if constexpr (std::is_same<R, float>::value) {
            R t, e;
            two_sum(s, x, t, e);
            s = t;
            c += e;
        } else {
            s += x;
        }
    }
    __device__ __forceinline__ R value() const { return s + c; }
};

// Dot product with a compensated accumulator in FP32 (Ogita, Rump & Oishi's
// Dot2); plain FMA chain in FP64.
template <typename R>
struct Dot {
    R s = R(0), c = R(0);
    __device__ __forceinline__ void add(R x, R y)
    {
        if constexpr (std::is_same<R, float>::value) {
            R p = x * y, ep = fmaf(x, y, -p), t, es;
            two_sum(s, p, t, es);
            s = t;
            c += ep + es;
        } else {
            s = fma(x, y, s);
        }
    }
    __device__ __forceinline__ R value() const { return s + c; }
};

template <typename R> __device__ __forceinline__ R rcp(R x);
template <> __device__ __forceinline__ float rcp<float>(float x)
{
    float r;   // hardware reciprocal approximation (MUFU), adequate for WENO weights in FP32
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
template <> __device__ __forceinline__ double rcp<double>(double x) { return 1.0 / x; }
template <typename R> __device__ __forceinline__ R fdiv(R a, R b);
template <> __device__ __forceinline__ float fdiv<float>(float a, float b) { return __fdividef(a, b); }
template <> __device__ __forceinline__ double fdiv<double>(double a, double b) { return a / b; }

// ---- packed FP32 pairs (sm_100+ f32x2 arithmetic): the two reduced
// distributions phi and chi go through identical arithmetic, so the FP32 path
// carries them as one packed pair per velocity ----
struct f2 {
    unsigned long long v;
};
__device__ __forceinline__ f2 mk2(float lo, float hi)
{
    f2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r.v) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ f2 bc2(float x) { return mk2(x, x); }
__device__ __forceinline__ void un2(f2 a, float &lo, float &hi)
{
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(a.v));
}
__device__ __forceinline__ f2 operator+(f2 a, f2 b)
{
    f2 r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
    return r;
}
__device__ __forceinline__ f2 operator-(f2 a, f2 b)
{
    f2 r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
    return r;
}
__device__ __forceinline__ f2 operator*(f2 a, f2 b)
{
    f2 r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
    return r;
}
__device__ __forceinline__ f2 fma2(f2 a, f2 b, f2 c)   // a b + c
{
    f2 r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r.v) : "l"(a.v), "l"(b.v), "l"(c.v));
    return r;
}
__device__ __forceinline__ float rcp_approx(float x)
{
    float r;   // hardware reciprocal approximation (MUFU)
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ f2 rcp2(f2 a)
{
    float lo, hi;
    un2(a, lo, hi);
    return mk2(rcp_approx(lo), rcp_approx(hi));
}
__device__ __forceinline__ f2 max2(f2 a, f2 b)
{
    float al, ah, bl, bh;
    un2(a, al, ah);
    un2(b, bl, bh);
    return mk2(fmaxf(al, bl), fmaxf(ah, bh));
}

// Brings the line of a global address into this SM's L1 (no data returned).
__device__ __forceinline__ void prefetch_l1(const void *p) { asm volatile("prefetch.L1 [%0];" ::"l"(p)); }

// One (phi, chi) pair of an interleaved row: a single 64-bit access.
__device__ __forceinline__ f2 ld2(const float *p)
{
    f2 r;
    r.v = *reinterpret_cast<const unsigned long long *>(p);
    return r;
}
__device__ __forceinline__ void st2(float *p, f2 a) { *reinterpret_cast<unsigned long long *>(p) = a.v; }

// Integer bit pattern stored in a per-velocity row entry.
__device__ __forceinline__ int row_bits(float x) { return __float_as_int(x); }
__device__ __forceinline__ int row_bits(double x) { return (int)__double_as_longlong(x); }

__device__ __forceinline__ f2 min2(f2 a, f2 b)
{
    float al, ah, bl, bh;
    un2(a, al, ah);
    un2(b, bl, bh);
    return mk2(fminf(al, bl), fminf(ah, bh));
}

// WENO-5 (Jiang & Shu) on a packed pair, face between c and d, upwind cell c.
// The nonlinear weights d_k / (eps + beta_k)^2, normalised, written as
// d_k (min_m e_m / e_k)^2 with e_k = eps + beta_k: the same weights in exact
// arithmetic, and in FP32 range for any e_k (weight-divided tails of hot-wall
// populations reach 1e10, so e_k reaches ~1e20 and e_k^2 would overflow): every
// ratio is at most 1, the smoothest stencil's is exactly 1, so the normaliser is
// at least min d_k = 0.1, and ratios that underflow belong to weights below FP32
// resolution.
__device__ __forceinline__ f2 weno5_2(f2 a, f2 b, f2 c, f2 d, f2 e)
{
    const f2 two = bc2(2.f), three = bc2(3.f), five = bc2(5.f);
    const f2 q0 = fma2(bc2(11.f), c, fma2(bc2(-7.f), b, two * a));
    const f2 q1 = fma2(two, d, fma2(five, c, bc2(0.f) - b));
    const f2 q2 = fma2(five, d, two * c) - e;
    const f2 t0 = fma2(bc2(-2.f), b, a + c), t1 = fma2(three, c, fma2(bc2(-4.f), b, a));
    const f2 t2 = fma2(bc2(-2.f), c, b + d), t3 = b - d;
    const f2 t4 = fma2(bc2(-2.f), d, c + e), t5 = fma2(bc2(-4.f), d, fma2(three, c, e));
    const f2 k1312 = bc2(13.f / 12.f), k025 = bc2(0.25f), eps = bc2(1e-6f);
    const f2 e0 = fma2(k1312, t0 * t0, fma2(k025, t1 * t1, eps));
    const f2 e1 = fma2(k1312, t2 * t2, fma2(k025, t3 * t3, eps));
    const f2 e2 = fma2(k1312, t4 * t4, fma2(k025, t5 * t5, eps));
    const f2 mn = min2(e0, min2(e1, e2));
    const f2 r0 = mn * rcp2(e0), r1 = mn * rcp2(e1), r2 = mn * rcp2(e2);
    const f2 s0 = r0 * r0, s1 = r1 * r1, s2 = r2 * r2;
    // sum_k d_k s_k q_k / (6 sum_k d_k s_k), d = (0.1, 0.6, 0.3)
    const f2 num = fma2(bc2(0.1f) * s0, q0, fma2(bc2(0.6f) * s1, q1, bc2(0.3f) * s2 * q2));
    const f2 den = fma2(bc2(0.6f), s0, fma2(bc2(3.6f), s1, bc2(1.8f) * s2));
    return num * rcp2(den);
}

// WENO-5 (Jiang & Shu) face value between c and d with upwind cell c.
template <typename R>
__device__ __forceinline__ R weno5(R a, R b, R c, R d, R e)
{
    const R eps = R(1e-6);
    R q0 = R(2) * a - R(7) * b + R(11) * c;
    R q1 = -b + R(5) * c + R(2) * d;
    R q2 = R(2) * c + R(5) * d - e;
    R t0 = a - R(2) * b + c, t1 = a - R(4) * b + R(3) * c;
    R t2 = b - R(2) * c + d, t3 = b - d;
    R t4 = c - R(2) * d + e, t5 = R(3) * c - R(4) * d + e;
    R e0 = eps + R(13.0 / 12.0) * t0 * t0 + R(0.25) * t1 * t1;
    R e1 = eps + R(13.0 / 12.0) * t2 * t2 + R(0.25) * t3 * t3;
    R e2 = eps + R(13.0 / 12.0) * t4 * t4 + R(0.25) * t5 * t5;
    R a0, a1, a2;
    if constexpr (std::is_same<R, float>::value) {
        // nonlinear weights as d_k (min e_m / e_k)^2: no square leaves the FP32 range
        const R mn = fminf(e0, fminf(e1, e2));
        const R r0 = mn * rcp<R>(e0), r1 = mn * rcp<R>(e1), r2 = mn * rcp<R>(e2);
        a0 = R(0.1) * r0 * r0;
        a1 = R(0.6) * r1 * r1;
        a2 = R(0.3) * r2 * r2;
    } else {
        // nonlinear weights d_k / (eps + beta_k)^2 (each bounded by d_k / eps^2)
        a0 = R(0.1) * rcp<R>(e0 * e0);
        a1 = R(0.6) * rcp<R>(e1 * e1);
        a2 = R(0.3) * rcp<R>(e2 * e2);
    }
    return fdiv<R>(a0 * q0 + a1 * q1 + a2 * q2, R(6) * (a0 + a1 + a2));
}

// ---- TMA and mbarrier (inline PTX) ----
__device__ __forceinline__ uint32_t smem_addr(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Shared-memory counter increment with acquire-release ordering at CTA scope.
__device__ __forceinline__ uint32_t atom_add_acq_rel(uint32_t *p, uint32_t v)
{
    uint32_t old;
    asm volatile("atom.acq_rel.cta.shared::cta.add.u32 %0, [%1], %2;" : "=r"(old) : "r"(smem_addr(p)), "r"(v) : "memory");
    return old;
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_inval(uint64_t *bar)
{
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_addr(bar)) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, long limit = kSpinLimit)
{
    const uint32_t a = smem_addr(bar);
    for (long i = 0; i < limit; ++i) {
        uint32_t ok;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(ok)
            : "r"(a), "r"(parity)
            : "memory");
        if (ok) return true;
    }
    return false;
}

__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, int x, int y, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
        ::"r"(smem_addr(dst)), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_addr(bar))
        : "memory");
}

// ---- thread-block cluster (the chunk CTAs of one tile) ----
__device__ __forceinline__ uint32_t cluster_ctarank()
{
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ void cluster_arrive_relaxed()
{
    asm volatile("barrier.cluster.arrive.relaxed.aligned;" ::: "memory");
}
__device__ __forceinline__ void cluster_arrive() { asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory"); }
__device__ __forceinline__ void cluster_wait() { asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory"); }

// Store into the shared memory of cluster CTA `rank`, at the address that `local` has in this CTA.
template <typename R> __device__ __forceinline__ void st_cluster(R *local, uint32_t rank, R v);
template <> __device__ __forceinline__ void st_cluster<float>(float *local, uint32_t rank, float v)
{
    uint32_t ra;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(ra) : "r"(smem_addr(local)), "r"(rank));
    asm volatile("st.shared::cluster.f32 [%0], %1;" ::"r"(ra), "f"(v) : "memory");
}
template <> __device__ __forceinline__ void st_cluster<double>(double *local, uint32_t rank, double v)
{
    uint32_t ra;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(ra) : "r"(smem_addr(local)), "r"(rank));
    asm volatile("st.shared::cluster.f64 [%0], %1;" ::"r"(ra), "d"(v) : "memory");
}

// Bulk copy global -> shared (16-byte aligned addresses, size a multiple of 16),
// completing on the mbarrier `bar`.
__device__ __forceinline__ void bulk_load(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
        ::"r"(smem_addr(dst)), "l"(reinterpret_cast<uint64_t>(src)), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

// ---- stage data of a set of nodes ----
constexpr int kEqLB = 16;   // orders per block of the projection: lanes = 2 signs x 16 orders

// Shared scratch of node_equilibrium for up to `ncap` nodes. The front region
// holds first the stage kernel's warp partials (`red`: the equilibrium tables
// are copied into `tab`, behind it, while those are being reduced) and then,
// once the partials are consumed, the warps' projection slices (`wk`): each
// warp works through its nodes nb at a time (two independent chains in flight
// when the projection rule fits one lane per node), one slice per node:
// projection weights r^{+-} [2][K], coefficients c^{+-} [cstride], and a block
// of kEqLB rows h_l(sqrt(T') Y_k) [kEqLB][kpad].
template <typename R>
struct EqScratch {
    size_t red, tab, raw, shf, sc, bb, wk, wbytes, total;
    int cstride, kpad, nb;
    __host__ __device__ EqScratch(int K, int N, int Ny, int Qx, int Qy, int ntab, int ncap = kTile)
    {
        cstride = 2 * (N + 1);
        kpad = K | 1;   // odd row stride: the lanes of a dot read conflict-free rows
        nb = K <= 32 ? 2 : 1;
        wbytes = al16((size_t)(2 * K + cstride + kEqLB * kpad) * sizeof(R));
        red = (size_t)kWarps * kNumRaw * kLanes * sizeof(R);
        wk = 0;
        const size_t slices = (size_t)nb * kWarps * wbytes;
        tab = al16(red > slices ? red : slices);
        raw = al16(tab + (size_t)EqTab(N, Ny, K, Qx, Qy, ntab).len * sizeof(R));
        shf = al16(raw + (size_t)ncap * kNumRaw * sizeof(R));
        sc = al16(shf + (size_t)2 * kLanes * sizeof(R));
        bb = al16(sc + (size_t)ncap * 8 * sizeof(R));
        total = al16(bb + (size_t)ncap * (Ny + 1) * sizeof(R));
    }
    __host__ __device__ static size_t al16(size_t x) { return (x + 15) / 16 * 16; }
};

// Raw sums of the rest Maxwellian about the shift (sx, sy), from its power sums P_ab.
template <typename R>
__device__ __forceinline__ void rest_raw_r(const DevTables &T, R sx, R sy, R *r)
{
    // constant indices only: the parameter block stays in the constant bank (no local copy)
    const R P00 = Tabs<R>::restP(T, 0), P10 = Tabs<R>::restP(T, 1), P01 = Tabs<R>::restP(T, 2);
    const R P20 = Tabs<R>::restP(T, 3), P11 = Tabs<R>::restP(T, 4), P02 = Tabs<R>::restP(T, 5);
    const R P30 = Tabs<R>::restP(T, 6), P21 = Tabs<R>::restP(T, 7), P12 = Tabs<R>::restP(T, 8);
    const R P03 = Tabs<R>::restP(T, 9);
    r[R_S0] = P00;
    r[R_SX] = P10 - sx * P00;
    r[R_SY] = P01 - sy * P00;
    r[R_SXX] = P20 - R(2) * sx * P10 + sx * sx * P00;
    r[R_SXY] = P11 - sx * P01 - sy * P10 + sx * sy * P00;
    r[R_SYY] = P02 - R(2) * sy * P01 + sy * sy * P00;
    r[R_CZ] = P00;                       // chi_rest = T_rest phi_rest, T_rest = 1
    const R a3 = P30 - R(3) * sx * P20 + R(3) * sx * sx * P10 - sx * sx * sx * P00;
    const R ab2 = P12 - R(2) * sy * P11 + sy * sy * P10 - sx * P02 + R(2) * sx * sy * P01 - sx * sy * sy * P00;
    const R b3 = P03 - R(3) * sy * P02 + R(3) * sy * sy * P01 - sy * sy * sy * P00;
    const R ba2 = P21 - R(2) * sx * P11 + sx * sx * P01 - sy * P20 + R(2) * sx * sy * P10 - sy * sx * sx * P00;
    r[R_R3X] = a3 + ab2;
    r[R_R3Y] = b3 + ba2;
    r[R_GX] = P10 - sx * P00;
    r[R_GY] = P01 - sy * P00;
}

// Moments from raw sums about (sx, sy), in the state precision.
template <typename R>
__device__ __forceinline__ void raw_to_moments_r(const R *r, R sx, R sy, R *m)
{
    R n = r[R_S0], in = R(1) / n;
    R bx = r[R_SX] * in, by = r[R_SY] * in;
    R pxx = r[R_SXX] - n * bx * bx;
    R pyy = r[R_SYY] - n * by * by;
    R pzz = r[R_CZ];
    R r2 = r[R_SXX] + r[R_SYY], b2 = bx * bx + by * by;
    R hx = r[R_R3X] - bx * r2 - R(2) * (bx * r[R_SXX] + by * r[R_SXY]) + R(2) * n * bx * b2;
    R hy = r[R_R3Y] - by * r2 - R(2) * (bx * r[R_SXY] + by * r[R_SYY]) + R(2) * n * by * b2;
    m[0] = n;
    m[1] = sx + bx;
    m[2] = sy + by;
    m[3] = (pxx + pyy + pzz) * in * R(1.0 / 3.0);
    m[4] = pxx; m[5] = pyy; m[6] = pzz; m[7] = r[R_SXY] - n * bx * by;
    m[8] = R(0.5) * hx + R(0.5) * (r[R_GX] - bx * pzz);
    m[9] = R(0.5) * hy + R(0.5) * (r[R_GY] - by * pzz);
}

// Hermite coefficients of g_x of NB nodes by the Gauss-sum projection (a whole warp):
// c^{+-}_l = sum_k r_k^{+-} h_l(sqrt(T') Y_k), r_k^{+-} = W_k exp(+-a Y_k - a^2/2), over the K
// nodes of the projection rule, for l <= N, into cw[b][2][N+1]. Lanes run the recurrence of
// the orthonormal h_l at projection nodes lane + 32 u (u < NU, K <= 32 NU) in blocks of kEqLB
// orders; lane (sign, l) of a block takes one compensated dot product (Dot2 in FP32) per node.
// The NB nodes' chains are independent (latency hidden by each other) and share the table
// reads; every node runs the same operations. x[b] = (sqrt(T'), a, a^2/2) of node b; rp[b]
// [2][K] and Hw[b] [kEqLB][kpad] are this warp's scratch for node b.
template <typename R, int NU, int NB>
__device__ __forceinline__ void project_coefficients(const R *const *x, int K, int N, int kpad, const R *Yk,
                                                     const R *Wk, const R *alpha, const R *sbeta,
                                                     const R *isbeta, R h0, R *const *rp, R *const *cw,
                                                     R *const *Hw)
{
    const int lane = threadIdx.x & 31;
    const int sgn = lane / kEqLB, lo = lane - sgn * kEqLB;
    R zt[NB][NU], h[NB][NU], hp[NB][NU];
#pragma unroll
    for (int u = 0; u < NU; ++u) {
        const int k = lane + 32 * u;
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            zt[b][u] = R(0);
            h[b][u] = h0;
            hp[b][u] = R(0);
        }
        if (k < K) {
            const R Y = Yk[k], W = Wk[k];
#pragma unroll
            for (int b = 0; b < NB; ++b) {
                const R a = x[b][1], a2 = x[b][2];
                rp[b][k] = W * exp(a * Y - a2);
                rp[b][K + k] = W * exp(-a * Y - a2);
                zt[b][u] = x[b][0] * Y;
            }
        }
    }
    for (int lb = 0; lb <= N; lb += kEqLB) {
        const int le = min(N, lb + kEqLB - 1);
#pragma unroll 4
        for (int l = lb; l <= le; ++l) {
            const R al = alpha[l], sb = sbeta[l], isb1 = isbeta[l + 1];
#pragma unroll
            for (int u = 0; u < NU; ++u) {
                const int k = lane + 32 * u;
#pragma unroll
                for (int b = 0; b < NB; ++b) {
                    if (k < K) Hw[b][(l - lb) * kpad + k] = h[b][u];
                    const R hn = ((zt[b][u] - al) * h[b][u] - sb * hp[b][u]) * isb1;
                    hp[b][u] = h[b][u];
                    h[b][u] = hn;
                }
            }
        }
        __syncwarp();
        if (lb + lo <= le) {
            Dot<R> d[NB];
#pragma unroll 4
            for (int k = 0; k < K; ++k)
#pragma unroll
                for (int b = 0; b < NB; ++b) d[b].add(rp[b][sgn * K + k], Hw[b][lo * kpad + k]);
#pragma unroll
            for (int b = 0; b < NB; ++b) cw[b][sgn * (N + 1) + lb + lo] = d[b].value();
        }
        __syncwarp();
    }
}

// Projection and g_x factors of nodes i (and i2 when `pair`) of a warp: its slices of the
// scratch (L.nb per warp, the first NB of them used), then the factors
// g_x/w at (node, sign a) = sum_l h_l(z_a) c_l^{sign}.
template <typename R, int NU, int NB>
__device__ __forceinline__ void equilibrium_nodes(const DevTables &T, const DevState &S, const EqScratch<R> &L, int i,
                                                  int i2, bool pair, int K, int N, int Qx, const R *Yk,
                                                  const R *Wk, const R *alpha, const R *sbeta, const R *isbeta,
                                                  R h0, const R *hz, const R *sc, unsigned char *scratch, R *eqg,
                                                  int cfirst, int cstep)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int node[2] = {i, i2};
    const R *x[NB];
    R *rp[NB], *cw[NB], *Hw[NB];
#pragma unroll
    for (int b = 0; b < NB; ++b) {
        x[b] = sc + node[b] * 8;
        rp[b] = reinterpret_cast<R *>(scratch + L.wk + (L.nb * warp + b) * L.wbytes);   // [2][K] r^+, r^-
        cw[b] = rp[b] + 2 * K;                                                         // [2][N+1] c^+, c^-
        Hw[b] = cw[b] + L.cstride;                                                     // [kEqLB][kpad]
    }
    project_coefficients<R, NU, NB>(x, K, N, L.kpad, Yk, Wk, alpha, sbeta, isbeta, h0, rp, cw, Hw);
    for (int ig = lane; ig < 2 * Qx; ig += 32) {   // g_x factors (sign, a)
        const int ii = ig < Qx ? ig : ig - Qx, off = ig < Qx ? 0 : N + 1;
        R acc[NB];
#pragma unroll
        for (int b = 0; b < NB; ++b) acc[b] = R(0);
#pragma unroll 4
        for (int l = 0; l <= N; ++l) {
            const R hv = hz[l * Qx + ii];
#pragma unroll
            for (int b = 0; b < NB; ++b) acc[b] = fma(hv, cw[b][off + l], acc[b]);
        }
#pragma unroll
        for (int b = 0; b < NB; ++b)
            if ((b == 0 || pair) && LBC_CHECK(S.ctl, cfirst + node[b] * cstep < kLanes, CK_EQ))
                eqg[(size_t)ig * kLanes + cfirst + node[b] * cstep] = acc[b];
    }
    __syncwarp();   // the next nodes reuse this warp's slices
}

// Stage data of the nodes c = cfirst + i cstep (i < nn <= ncap) of tile `tile`
// for buffer `buf` (block-wide, all threads). Input in `scratch` (EqScratch
// for ncap nodes): the equilibrium tables (EqTab), the raw moment sums of the
// deviation per node, raw[i][m], and the shift of those sums per tile node,
// shf[0][c] = s_x, shf[1][c] = s_y. Adds the rest state's share, turns the sums
// into moments, and builds the discrete equilibrium factors of Eqs. gx, gy
// (algorithm: see equilibrium_host). Writes eqm[buf] of the nodes and their
// columns of the tile's eqg[buf] block; dm_a, dm_b (either may be NULL) receive
// each node's mass deviation J_s deta (n_s - 1) (local steps, buffer 0).
// Organised for instruction count and latency: a thread per node for the
// moments and the g_y coefficients; the g_y factors over all threads, one
// (node, j) each; then a warp per node for the projection and the g_x factors
// (lanes over projection nodes, then over (sign, order), then over factors),
// with warp-level synchronisation only and the tables in shared memory.
template <typename R>
__device__ void node_equilibrium(const DevTables &T, const DevState &S, int buf, int tile, int cfirst, int cstep,
                                 int nn, int ncap, unsigned char *scratch, double *dm_a, double *dm_b)
{
    const int tid = threadIdx.x, warp = tid >> 5, c0 = tile * kTile;
    const int N = T.Nxe, K = T.K, G = 2 * T.Qx + T.Qy, Ny = T.Nye, Qx = T.Qx, Qy = T.Qy;
    const EqScratch<R> L(K, N, Ny, Qx, Qy, T.tab_n, ncap);
    const EqTab E(N, Ny, K, Qx, Qy, T.tab_n);
    const R *tab = reinterpret_cast<const R *>(scratch + L.tab);
    const R *raw = reinterpret_cast<const R *>(scratch + L.raw);   // [nn][kNumRaw]
    const R *shf = reinterpret_cast<const R *>(scratch + L.shf);   // [2][kLanes]
    R *sc = reinterpret_cast<R *>(scratch + L.sc);      // [nn][8]: sT a a^2/2 u'_y T'-1
    R *bb = reinterpret_cast<R *>(scratch + L.bb);      // [nn][Ny+1]   Hermite coefficients of g_y
    R *eqm = static_cast<R *>(S.eqm[buf]);
    R *eqg = static_cast<R *>(S.eqg[buf]) + (size_t)tile * G * kLanes;
#ifdef LBC_CHECKED
    if (!LBC_CHECK(S.ctl, nn <= ncap && tile >= 0 && tile < T.ntile, CK_EQ)) return;   // uniform over the CTA
#endif

    // ---- moments, relaxation data, per-node scalars and the g_y coefficients (thread per node) ----
    if (tid < nn) {
        const int c = cfirst + tid * cstep, s = c0 + c;
        const bool live = s < T.Nx;
        // per-node and per-instance data from global memory, loaded first so that their latency
        // overlaps the moment arithmetic
        const R ijd_s = live ? Tabs<R>::ijd(T)[s] : R(0), dtn_s = live ? Tabs<R>::dtn(T)[s] : R(0);
        const double jd_s = live && (dm_a || dm_b) ? T.jdeta[s] : 0.0;
        const R scNU = Tabs<R>::sc(T, SC_NU), ip0 = Tabs<R>::sc(T, SC_IP0);
        const R scEXPO = Tabs<R>::sc(T, SC_EXPO), sc1MPR = Tabs<R>::sc(T, SC_1MPR);
        R m[10];
        if (live) {
            const R sx = shf[c], sy = shf[kLanes + c];
            R rr[kNumRaw];
            rest_raw_r<R>(T, sx, sy, rr);
#pragma unroll
            for (int k = 0; k < kNumRaw; ++k) rr[k] += raw[tid * kNumRaw + k];
            raw_to_moments_r<R>(rr, sx, sy, m);
            if (dm_a || dm_b) {   // the deviation's own S0 is n_s - 1 (the rest state has n = 1)
                const double dm = jd_s * (double)raw[tid * kNumRaw + R_S0];
                if (dm_a) dm_a[s] = dm;
                if (dm_b) dm_b[s] = dm;
            }
            // a NaN/Inf anywhere in the node's populations reaches its moments
            if (!isfinite(m[0]) || !isfinite(m[3]) || !isfinite(m[8]) || !isfinite(m[9]) || !(m[0] > R(0)) ||
                !(m[3] > R(0)))
                S.ctl->nonfinite = 1;
        } else {
            m[0] = R(1); m[1] = m[2] = R(0); m[3] = R(1); m[4] = m[5] = m[6] = R(1); m[7] = m[8] = m[9] = R(0);
        }
        const R n = m[0], ux = m[1], uy = m[2], Tc = m[3];
        R nu, cS;   // 1/tau (Eq. tau) and the Shakhov prefactor (1 - Pr)/(n T^2)
        if (T.law == LBC_MU_TABLE) {
            // Eqs. mun, interp: k = number of table temperatures <= T; viscosity on segment
            // clamp(k - 1, 0, ntab - 2) (end segments extrapolate), Pr_{max(k - 1, 0)}
            const R *lT = tab + E.lawT;
            int lo = 0, hi = T.tab_n;
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if (lT[mid] <= Tc) lo = mid + 1;
                else hi = mid;
            }
            const int cg = min(max(lo - 1, 0), T.tab_n - 2);
            const R mu = tab[E.lawMu + cg] * pow(Tc / lT[cg], tab[E.lawW + cg]);   // mu(T) / mu(T_ref)
            nu = n * Tc / mu * scNU;
            cS = (R(1) - tab[E.lawPr + max(lo - 1, 0)]) / (n * Tc * Tc);
        } else {
            nu = n * scNU * pow(Tc, scEXPO);   // mu = T^omega (Eq. mu)
            cS = sc1MPR / (n * Tc * Tc);
        }
        if (live && LBC_CHECK(S.ctl, s < T.Nxp, CK_EQ)) {
            R *e = eqm + (size_t)s * kEqM;
            e[0] = n; e[1] = ux; e[2] = uy; e[3] = Tc; e[4] = m[8]; e[5] = m[9];
            e[6] = nu; e[7] = cS; e[8] = R(1) / (R(5) * Tc); e[9] = ijd_s;
            e[10] = m[4]; e[11] = m[5]; e[12] = m[6]; e[13] = m[7]; e[14] = dtn_s;
        }
        const R Tp = Tc * ip0 * ip0, sT = sqrt(Tp), a = ux * ip0 / sT;
        R *x = sc + tid * 8;
        x[0] = sT; x[1] = a; x[2] = R(0.5) * a * a;
        // g_y coefficients b_l = E[He_l(u' + sqrt(T') Y)] / l!: b_{l+1} = (u' b_l + (T'-1) b_{l-1}) / (l+1)
        const R uq = uy * ip0, tm1 = Tp - R(1);
        const R *invl = tab + E.invl;
        R *b = bb + tid * (Ny + 1);
        R bm = R(1), bl = uq;
        b[0] = R(1);
        b[1] = uq;
#pragma unroll 4
        for (int l = 1; l < Ny; ++l) {
            const R bn = (uq * bl + tm1 * bm) * invl[l + 1];
            bm = bl;
            bl = bn;
            b[l + 1] = bn;
        }
    }
    __syncthreads();

    // factors: g_x/w at (node, a) = sum_l h_l(z_a) c_l^{sign a}, g_y/w at (node, j) = sum_l He_l(y_j) b_l.
    // Evaluating the truncated expansions at the nodes is a plain FMA chain: where its terms
    // cancel (the far tails of hot or cold Maxwellians) the factor's absolute error stays far
    // below what the quadrature weight of that velocity lets reach any moment.
    // ---- the g_y factors need only the b_l: every thread takes (node, j) pairs ----
    const R *hz = tab + E.hz, *He = tab + E.He;
    for (int idx = tid; idx < nn * Qy; idx += kThreads) {
        const int jj = idx / nn, i = idx - jj * nn;   // consecutive threads: consecutive nodes
        const R *b = bb + i * (Ny + 1);
        R acc = R(0);
#pragma unroll 4
        for (int l = 0; l <= Ny; ++l) acc = fma(He[l * Qy + jj], b[l], acc);
        if (LBC_CHECK(S.ctl, cfirst + i * cstep < kLanes, CK_EQ))
            eqg[(size_t)(2 * Qx + jj) * kLanes + cfirst + i * cstep] = acc;
    }

    // ---- a warp per node: g_x by the stable Gauss-sum projection, then its factors ----
    const R *Yk = tab + E.Yk, *Wk = tab + E.Wk;
    const R *alpha = tab + E.alpha, *sbeta = tab + E.sbeta, *isbeta = tab + E.isbeta;
    const R h0 = Tabs<R>::sc(T, SC_H0);
    if (L.nb == 2) {
        // two nodes per warp (i, i + kWarps) with independent chains; a lone node alone
        for (int i = warp; i < nn; i += 2 * kWarps) {
            if (i + kWarps < nn)
                equilibrium_nodes<R, 1, 2>(T, S, L, i, i + kWarps, true, K, N, Qx, Yk, Wk, alpha, sbeta, isbeta, h0,
                                           hz, sc, scratch, eqg, cfirst, cstep);
            else
                equilibrium_nodes<R, 1, 1>(T, S, L, i, i, false, K, N, Qx, Yk, Wk, alpha, sbeta, isbeta, h0, hz, sc,
                                           scratch, eqg, cfirst, cstep);
        }
    } else {
        for (int i = warp; i < nn; i += kWarps)
            equilibrium_nodes<R, 2, 1>(T, S, L, i, i, false, K, N, Qx, Yk, Wk, alpha, sbeta, isbeta, h0, hz, sc,
                                       scratch, eqg, cfirst, cstep);
    }
}

// Outgoing WENO-5 wall face of the phi deviation of a state row (interleaved
// (phi, chi) per node) at the left (px < 0) or right (px > 0) wall; two ghost
// nodes by cubic extrapolation in eta.
template <typename R>
__device__ __forceinline__ R outgoing_wall_face(const R *row, int Nx, bool right)
{
    // L2 loads (.cg): in the persistent form another SM wrote these rows in the same launch
    R f1, f2, f3, f4;
    if (right) {
        f1 = __ldcg(row + 2 * (Nx - 1)); f2 = __ldcg(row + 2 * (Nx - 2));
        f3 = __ldcg(row + 2 * (Nx - 3)); f4 = __ldcg(row + 2 * (Nx - 4));
    } else {
        f1 = __ldcg(row); f2 = __ldcg(row + 2); f3 = __ldcg(row + 4); f4 = __ldcg(row + 6);
    }
    R g1 = R(4) * f1 - R(6) * f2 + R(4) * f3 - f4;
    R g2 = R(10) * f1 - R(20) * f2 + R(15) * f3 - R(4) * f4;
    return weno5<R>(f3, f2, f1, g1, g2);
}

// n_w of one wall (Eq. diffuse_nw) from the stage-input deviation, all threads;
// the flux is accumulated in FP64 so the wall mass balance holds to round-off.
template <typename R>
__device__ void block_wall_density(const DevTables &T, const R *phi, bool right, double *wsum, double *out)
{
    const int half = T.Qx * T.Qy, vbeg = right ? 0 : half;
    const R *vel = Tabs<R>::vel(T);
    double acc = 0.0;
    for (int v = vbeg + threadIdx.x; v < vbeg + half; v += blockDim.x) {
        R f = outgoing_wall_face<R>(phi + 2 * (size_t)v * T.Nxp, T.Nx, right);
        acc += (double)(vel[VC_PX * T.V + v] * vel[VC_W * T.V + v] * f);
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) wsum[warp] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = right ? T.restOutR : T.restOutL;
        for (int k = 0; k < kWarps; ++k) s += wsum[k];
        *out = -s * (right ? T.dsc[SC_IINR] : T.dsc[SC_IINL]);
    }
    __syncthreads();
}

// sum_{s < Nx} dm[s] by the whole block (256 threads) in a fixed order, so that
// every CTA that sums the same data obtains the same bits. red: 8 doubles of
// shared scratch. Returns the sum in every thread.
__device__ double block_mass_deviation(const double *dm, int Nx, double *red)
{
    double acc = 0.0;
    for (int s = threadIdx.x; s < Nx; s += kThreads) acc += __ldcg(dm + s);   // written by other tiles
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    double t = 0.0;
    for (int k = 0; k < kWarps; ++k) t += red[k];
    __syncthreads();
    return t;
}

// Dynamic shared memory layout of the stage kernel. The pipeline region is
// reused after the main loop for the moment reduction and the node stage data
// (EqScratch); `xch` receives the moment partials that the cluster's CTAs send
// to this CTA for the nodes it owns.
template <typename R>
struct Layout {
    size_t bar, pipe, fin, f0, g, eqm, vrow, xch, misc, total;
    __host__ __device__ Layout(int Qx, int Qy, int N, int Ny, int K, int vchunk, int cluster, int ntab)
    {
        size_t o = 0;
        bar = o;  o = al(o + (kPipe + 2) * sizeof(uint64_t) + (kPipe + 1) * sizeof(uint32_t));
        pipe = o;
        fin = o;
        f0 = fin + (size_t)kPipe * 2 * kSubV * kRowLen * sizeof(R);
        size_t m = f0 + (size_t)kPipe * 2 * kSubV * kF0Len * sizeof(R) - pipe;
        // the first stage's wider slots (FP32) cover the RK-base region, which that stage leaves unused
        const size_t fin0 = (size_t)kPipe * 2 * slot_rows(0, sizeof(R) == 4) * kRowLen * sizeof(R);
        m = m > fin0 ? m : fin0;
        const size_t eq_bytes = EqScratch<R>(K, N, Ny, Qx, Qy, ntab, node_cap(cluster)).total;
        m = m > eq_bytes ? m : eq_bytes;
        o = al(o + m);
        g = o;    o = al(o + (size_t)(2 * Qx + Qy) * kLanes * sizeof(R));
        eqm = o;  o = al(o + (size_t)kLanes * kEqM * sizeof(R));
        vrow = o; o = al(o + (size_t)vchunk * kVRow * sizeof(R));
        xch = o;  o = al(o + (size_t)(kTile + kMaxCluster) * kNumRaw * sizeof(R));
        misc = o; o = al(o + 16 * sizeof(double));
        total = o + 128;   // slack for aligning the dynamic base
    }
    __host__ __device__ static size_t al(size_t x) { return (x + 127) / 128 * 128; }
    // node capacity of the equilibrium scratch: a whole tile (the solo form's last CTA takes all
    // of its nodes; the cluster form's CTAs take ceil(kTile / cluster) of them)
    __host__ __device__ static int node_cap(int) { return kTile; }
};

// TVD RK-3 (Shu & Osher): stage k's output is ca f^n + cb (y_k + dt L(y_k)).
template <typename R> __host__ __device__ constexpr R ca_of(int k) { return R(k == 0 ? 0.0 : (k == 1 ? 0.75 : 1.0 / 3.0)); }
template <typename R> __host__ __device__ constexpr R cb_of(int k) { return R(k == 0 ? 1.0 : (k == 1 ? 0.25 : 2.0 / 3.0)); }

// Kahan's compensated sum on packed pairs: s + x with the rounding error carried in c.
__device__ __forceinline__ void kahan2(f2 &s, f2 &c, f2 x)
{
    const f2 y = x - c, t = s + y;
    c = (t - s) - y;
    s = t;
}
__device__ __forceinline__ void kahan1(float &s, float &c, float x)
{
    const float y = x - c, t = s + y;
    c = (t - s) - y;
    s = t;
}

// One RK stage of tile `tile` of instance I, for the CTA's velocity chunk
// blockIdx.y (body of both stage kernels below). kExt compiles in the half
// channel's symmetry plane and the local steps with mass renormalisation
// (instances without them give the same results in either form). The chunk
// CTAs of a tile combine their moment partials in one of three ways (kForm):
//  - cluster form: the tile's chunk CTAs form a thread-block cluster and
//    exchange partials through distributed shared memory; each builds the
//    next-stage data of nodes rank, rank + nchunk, ...;
//  - solo form: plain CTAs write their partials to global memory
//    (DevState::part) and count themselves in (DevState::tcnt); the tile's
//    last CTA to finish sums the partials over the chunks, in chunk order, and
//    builds the next-stage data of all the tile's nodes while the others have
//    already left;
//  - split form: plain CTAs write their partials and leave; a second launch
//    (node_step_kernel) builds every tile's next-stage data with the whole GPU.
// Same arithmetic in the same order in every form: identical results.
template <typename R, bool kExt, int kStage, int kForm>
__device__ __forceinline__ void stage_body(const Inst &I, int tile, int rel, bool persist = false)
{
    constexpr int stage = kStage;   // RK stage 0, 1, 2: a compile-time constant in every form
    constexpr int kSub = slot_rows(kStage, sizeof(R) == 4);   // rows per pipeline slot
    extern __shared__ __align__(128) unsigned char smem_dyn[];
    const DevTables &T = I.T;
    const DevState &S = I.S;
    const StateMaps &M = I.M;
    // TMA destinations want 128-byte aligned shared memory: align the base explicitly
    unsigned char *smem = smem_dyn + ((128 - (smem_addr(smem_dyn) & 127)) & 127);
    const Layout<R> L(T.Qx, T.Qy, T.Nxe, T.Nye, T.K, T.vchunk, T.nchunk, T.tab_n);
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem + L.bar);   // [kPipe] rows, data, tables
    uint64_t *bar_data = bar + kPipe, *bar_tab = bar + kPipe + 1;
    uint32_t *s_cnt = reinterpret_cast<uint32_t *>(bar + kPipe + 2);   // [kPipe] warps done with a slot
    int *s_abort = reinterpret_cast<int *>(s_cnt + kPipe);              // a warp gave up waiting
    R *s_fin = reinterpret_cast<R *>(smem + L.fin);       // [kPipe][kSub][2 kRowLen]: (phi, chi) per node
    R *s_f0 = reinterpret_cast<R *>(smem + L.f0);         // [kPipe][kSub][2 kF0Len]
    R *s_g = reinterpret_cast<R *>(smem + L.g);           // [2Qx + Qy][kLanes]
    R *s_eqm = reinterpret_cast<R *>(smem + L.eqm);       // [kTile][kEqM]
    R *s_vrow = reinterpret_cast<R *>(smem + L.vrow);     // [vchunk][kVRow]
    R *s_xch = reinterpret_cast<R *>(smem + L.xch);       // [nchunk][nn_max][kNumRaw]
    __shared__ int s_last;                                // solo form: this CTA is the tile's last
    double *s_misc = reinterpret_cast<double *>(smem + L.misc);   // wsum[8], nwL, nwR

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int c0 = tile * kTile, chunk = blockIdx.y;
    const int in = stage, out = (stage + 1) % 3;
    Ctl *ctl = S.ctl;
    const long long step = ctl->base + rel;
    const int V = T.V, G = 2 * T.Qx + T.Qy;
    const bool lead = tile == 0 && chunk == 0 && tid == 0;   // one thread per instance

    // ---- early stop (run-to-steady): every block of the instance takes the same decision ----
    const double stop_eps = ctl->stop_eps;
    if (stop_eps > 0.0) {
        if (__ldcg(&ctl->stopped)) return;
        if (step - 1 >= ctl->check_from) {
            const double rprev = __longlong_as_double((long long)__ldcg(&S.resid[(step - 1) % kResidRing]));
            if (rprev < stop_eps) {
                if (stage == 0 && lead) {
                    ctl->stop_step = step;
                    ctl->stopped = 1;
                }
                return;
            }
        }
    }
    // the step's residual slot starts at zero (the persistent form zeroes its steps' slots before
    // the launch: its stages of one step may run in any order across tiles)
    if (stage == 0 && lead && !persist) S.resid[step % kResidRing] = 0ull;

    // this CTA's velocity rows [vbeg, vend): may be empty for a small instance in a wide cluster
    const int vbeg = min(V, chunk * T.vchunk);
    const int vend = min(V, vbeg + T.vchunk);
    const int nsub = (vend - vbeg + kSub - 1) / kSub;
    const int nloc = min(kTile, T.Nx - c0);   // nodes of this tile inside the channel
    const uint32_t tx_bytes =
        (uint32_t)((2 * kSub * kRowLen + (stage > 0 ? 2 * kSub * kF0Len : 0)) * sizeof(R));
    const CUtensorMap *in_map = &M.in[in];
    // TMA x coordinates must be 16-byte aligned: start the boxes at multiples of 4 nodes
    const int x0 = ((c0 - 3) >> 2) << 2, off = c0 - 3 - x0;     // node s <-> column s - x0
    const int xf = (c0 >> 2) << 2, offf = c0 - xf;
    const int ncap = Layout<R>::node_cap(T.nchunk);
    const EqScratch<R> E(T.K, T.Nxe, T.Nye, T.Qx, T.Qy, T.tab_n, ncap);
    const uint32_t tab_bytes = (uint32_t)(EqTab(T.Nxe, T.Nye, T.K, T.Qx, T.Qy, T.tab_n).len * sizeof(R));
#ifdef LBC_CHECKED
    // the CTA's staged geometry, checked once: TMA boxes on 16-byte boundaries, bulk copies inside
    // their shared-memory regions and source arrays, stencil and RK-base columns inside the staged
    // rows, and the cluster exchange inside every CTA's region
    const bool bad =
        !LBC_CHECK(ctl, (2 * x0 * (int)sizeof(R)) % 16 == 0 && (2 * xf * (int)sizeof(R)) % 16 == 0, CK_TMA_X) ||
        !LBC_CHECK(ctl,
                   tile >= 0 && tile < T.ntile && nloc > 0 && c0 + nloc <= T.Nxp && vend - vbeg <= T.vchunk &&
                       (size_t)G * kLanes * sizeof(R) <= L.eqm - L.g && (size_t)nloc * kEqM * sizeof(R) % 16 == 0,
                   CK_BULK) ||
        !LBC_CHECK(ctl, off >= 0 && kLanes + 4 + off < kRowLen && offf >= 0 && kLanes - 1 + offf < kF0Len,
                   CK_STENCIL) ||
        !LBC_CHECK(ctl,
                   T.nchunk >= 1 && T.nchunk <= kMaxCluster &&
                       T.nchunk * ((kTile + T.nchunk - 1) / T.nchunk) <= kTile + kMaxCluster,
                   CK_XCH);
#else
    constexpr bool bad = false;
#endif

    // rows v0 .. v0 + kSub - 1 of the stage input (nodes x0 .. x0 + kRowLen - 1) and of the
    // RK base (nodes xf ..), both fields; rows past V read as zeros
    auto issue = [&](int sub) {
        int p = sub % kPipe, v0 = vbeg + sub * kSub;
        mbar_expect_tx(&bar[p], tx_bytes);
        tma_load_2d(s_fin + (size_t)p * kSub * 2 * kRowLen, in_map, 2 * x0, v0, &bar[p]);
        if (stage > 0) tma_load_2d(s_f0 + (size_t)p * kSub * 2 * kF0Len, &M.f0, 2 * xf, v0, &bar[p]);
    };

    if (tid == 0) {
        for (int p = 0; p < kPipe + 2; ++p) mbar_init(&bar[p], 1);
        for (int p = 0; p < kPipe; ++p) s_cnt[p] = 0;
        *s_abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    __syncthreads();
    // solo form: the tile's chunk CTAs count themselves in once their stores (state, partials) are
    // done; the last of them resets the count for the next launch and goes on to the node step.
    // One thread fences for the CTA: the barrier orders every thread's stores before its fence,
    // which is cumulative (release before the count; acquire after it on the last CTA, whose
    // threads then read the other CTAs' partials from L2).
    auto solo_count_in = [&]() -> bool {
        __syncthreads();
        if (tid == 0) {
            __threadfence();
            const unsigned k = atomicAdd(&S.tcnt[tile], 1u);
            s_last = k + 1u == (unsigned)T.nchunk;
            if (s_last) {
                S.tcnt[tile] = 0u;
                __threadfence();
            }
        }
        __syncthreads();
        return s_last != 0;
    };
    constexpr bool kSolo = kForm == kFormSolo, kSplit = kForm == kFormSplit;
    if constexpr (kForm == kFormCluster) cluster_arrive_relaxed();   // this CTA runs: the others may write into its shared memory after their wait
    if (bad) {   // range-checked build: give up before any copy, taking part in the cluster barriers
        if constexpr (kSolo) {
            solo_count_in();
        } else if constexpr (!kSplit) {
            cluster_wait();
            cluster_arrive();
            cluster_wait();
        }
        if (persist && tid < kPipe + 2) mbar_inval(&bar[tid]);
        return;
    }
    if (tid == 0) {
        for (int sub = 0; sub < min(kPipe, nsub); ++sub) issue(sub);
        // ---- (1) the tile's stage data and the chunk's per-velocity rows, by bulk copies ----
        const uint32_t gb = (uint32_t)(G * kLanes * sizeof(R)), eb = (uint32_t)(nloc * kEqM * sizeof(R));
        const uint32_t vb = (uint32_t)((vend - vbeg) * kVRow * sizeof(R));
        mbar_expect_tx(bar_data, gb + eb + vb);
        bulk_load(s_g, static_cast<const R *>(S.eqg[in]) + (size_t)tile * G * kLanes, gb, bar_data);
        bulk_load(s_eqm, static_cast<const R *>(S.eqm[in]) + (size_t)c0 * kEqM, eb, bar_data);
        if (vb > 0) bulk_load(s_vrow, Tabs<R>::vrow(T) + (size_t)vbeg * kVRow, vb, bar_data);
    }

    const R *Fin = static_cast<const R *>(S.F[in]);
    R *Fout = static_cast<R *>(S.F[out]);

    // ---- (2) wall densities (tiles whose stencil reaches a wall), while the copies land ----
    const bool mirror = kExt && c0 == 0 && T.half != 0;   // half channel: symmetry plane at x = 0
    const bool needL = c0 == 0 && !mirror;
    const bool needR = c0 + 33 >= T.Nx;
    if (needL) block_wall_density<R>(T, Fin, false, s_misc, &s_misc[8]);
    if (needR) block_wall_density<R>(T, Fin, true, s_misc, &s_misc[9]);
    // local steps: this step's mass correction lambda - 1 = (M_ref - M(f^n)) / M(f^n), from the
    // mass deviations of f^n that the previous step (or the set-up) left for this step's parity
    const bool renorm = kExt && T.lts != 0 && stage == 2;
    // compensated FP32 state (DevState::C, DevState::A): every stage adds its dt L to the step's
    // increment, so the third stage adds dt (L0/6 + L1/6 + 2 L2/3) to d0 + c without rounding it
    // at the size of the state first
    const bool comp_any = kExt && T.comp != 0;
    const bool comp = comp_any && stage == 2;
    double lam1 = 0.0;
    if (renorm) {
        const double dM = block_mass_deviation(S.mass + kMassHdr + (size_t)(step & 1) * T.Nxp, T.Nx, s_misc);
        lam1 = (S.mass[0] - dM) / (T.mrest + dM);
    }
    // test hook (probe > 0): wait instead on the table barrier, which nothing has armed yet, so
    // that the bounded wait gives up; the timeout path below then waits for the data copy
    const int probe = ctl->probe;
    bool timed_out = __syncthreads_or(!mbar_wait(probe > 0 ? bar_tab : bar_data, 0, probe > 0 ? probe : kSpinLimit));

    const int s = c0 + lane;
    const bool active = lane < nloc;
    R n_c = R(1), ux_c = R(0), uy_c = R(0), T_c = R(1), qx_c = R(0), qy_c = R(0), nu_c = R(0), cS_c = R(0),
      i5T = R(0.2), ijd = R(0), dt = R(0);
    if (active && !timed_out) {
        const R *e = s_eqm + lane * kEqM;
        n_c = e[0]; ux_c = e[1]; uy_c = e[2]; T_c = e[3]; qx_c = e[4]; qy_c = e[5];
        nu_c = e[6]; cS_c = e[7]; i5T = e[8]; ijd = e[9];
        dt = kExt ? e[14] : Tabs<R>::sc(T, SC_DT);   // the node's time step (the global one unless lts)
    }
    const R nwL = R(needL ? s_misc[8] : 0.0), nwR = R(needR ? s_misc[9] : 0.0);

    // ---- (3) stream the chunk's velocity rows: every warp runs its own rows of each
    // pipeline slot; the last warp to release a slot issues its refill ----
    const R ca = ca_of<R>(stage), cb = cb_of<R>(stage);
    const bool wall = needL || needR;
    const R lam1r = R(lam1);
    const int ck = lane + 3 + off;          // node column of node c0 + lane
    const int Nxp = T.Nxp, Nx = T.Nx;
    R *Fout_s = Fout + 2 * (size_t)s;       // this lane's node in row v: Fout_s + 2 Nxp v

    R acc[kNumRaw];
#pragma unroll
    for (int m = 0; m < kNumRaw; ++m) acc[m] = R(0);
    R res = R(0);
    f2 pk[5], pkc[5];   // FP32: running raw sums as packed pairs; pkc: their Kahan compensation
#pragma unroll
    for (int m = 0; m < 5; ++m) pk[m] = pkc[m] = bc2(0.f);
    float sxyc = 0.f;
    // plain FP32 form: the stage's update out = ca d0 + k1 d + k2 (target - ft_rest) + k3 p_x (F_left - F_right)
    // with the node's constants folded (k1 = cb (1 - dt/tau), k2 = cb dt/tau, k3 = cb dt/(J deta)),
    // and the Shakhov factor's cS q folded into (shA, shB) = cS (q_x, q_y)
    constexpr bool kLean = std::is_same<R, float>::value && !kExt;
    const R k1 = cb_of<R>(stage) * (R(1) - dt * nu_c), k2 = cb_of<R>(stage) * dt * nu_c;
    const R k3 = cb_of<R>(stage) * dt * ijd, shA = cS_c * qx_c, shB = cS_c * qy_c;
    constexpr int NQ = kSub / kWarps;      // rows per warp and slot: rows warp + kWarps q
    bool my_timeout = false;

    // half channel: the ghost nodes -1, -2, -3 of velocity v are nodes 0, 1, 2 of the opposite
    // velocity (Sec. II symmetry), read from the stage input one pipeline slot ahead: lane
    // 3 q + g holds node g of the partner of row warp + kWarps q (both fields)
    R mg0 = R(0), mg1 = R(0);
    auto mirror_fetch = [&](int sub) {
        if (lane < 3 * NQ && sub < nsub) {
            const int q = lane / 3, g = lane - 3 * q, v = vbeg + sub * kSub + warp + kWarps * q;
            const int a = v / T.Qy, j = v - a * T.Qy;
            const int vm = (a < T.Qx ? a + T.Qx : a - T.Qx) * T.Qy + (T.Qy - 1 - j);
            if (v < vend && LBC_CHECK(ctl, vm >= 0 && vm < T.V && g < T.Nxp, CK_MIRROR)) {
                const R *src = Fin + 2 * ((size_t)vm * T.Nxp + g);
                mg0 = __ldcg(src);
                mg1 = __ldcg(src + 1);
            }
        }
    };
    if (mirror) mirror_fetch(0);

    for (int sub = 0; sub < nsub && !timed_out; ++sub) {
        const int p = sub % kPipe;
        if (__any_sync(0xffffffffu, !mbar_wait(&bar[p], (uint32_t)((sub / kPipe) & 1))) ||
            *reinterpret_cast<volatile int *>(s_abort)) {
            my_timeout = true;
            break;
        }
        R *fin = s_fin + (size_t)p * kSub * 2 * kRowLen;
        const R *f0 = s_f0 + (size_t)p * kSub * 2 * kF0Len;
        int kq[NQ];
        bool ok[NQ];
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            kq[q] = sub * kSub + warp + kWarps * q;
            ok[q] = vbeg + kq[q] < vend;
            if (!ok[q]) kq[q] = vend - vbeg - 1;   // the chunk's last velocity row; results are discarded
        }
        if (wall) {
            // ghost nodes, both fields at once: lanes 0-7 -> (row, side, node)
            if (lane < 4 * NQ) {
                const int q = lane >> 2, side = (lane >> 1) & 1, gi = lane & 1;
                int kqq = kq[0];
                bool okq = ok[0];
#pragma unroll
                for (int qq = 1; qq < NQ; ++qq)   // select, not a dynamic index (keeps kq, ok in registers)
                    if (q == qq) { kqq = kq[qq]; okq = ok[qq]; }
                const R *x = s_vrow + kqq * kVRow;
                const bool pos = x[VR_PX] > R(0);
                R *row = fin + (size_t)(warp + kWarps * q) * 2 * kRowLen;
                if (okq && side == 0 && needL &&
                    LBC_CHECK(ctl, -x0 - 2 >= 0 && -x0 + 3 < kRowLen, CK_STENCIL)) {   // nodes -1 (gi 0), -2 (gi 1)
                    R g0, g1;
                    if (pos) {
                        g0 = nwL * x[VR_FWL] - x[VR_FR];
                        g1 = nwL * x[VR_FWLT] - x[VR_FR];
                    } else {
                        const R *f = row + 2 * (-x0);     // node 0
                        const R c1 = gi == 0 ? R(4) : R(10), c2 = gi == 0 ? R(-6) : R(-20);
                        const R c3 = gi == 0 ? R(4) : R(15), c4 = gi == 0 ? R(-1) : R(-4);
                        g0 = c1 * f[0] + c2 * f[2] + c3 * f[4] + c4 * f[6];
                        g1 = c1 * f[1] + c2 * f[3] + c3 * f[5] + c4 * f[7];
                    }
                    R *gp = row + 2 * (-1 - gi - x0);
                    gp[0] = g0;
                    gp[1] = g1;
                } else if (okq && side == 1 && needR &&
                           LBC_CHECK(ctl, Nx - 4 - x0 >= 0 && Nx - 1 - x0 < kRowLen, CK_STENCIL)) {   // nodes Nx, Nx+1
                    R g0, g1;
                    if (!pos) {
                        g0 = nwR * x[VR_FWR] - x[VR_FR];
                        g1 = nwR * x[VR_FWRT] - x[VR_FR];
                    } else {
                        const R *f = row + 2 * (Nx - 1 - x0);   // node Nx - 1
                        const R c1 = gi == 0 ? R(4) : R(10), c2 = gi == 0 ? R(-6) : R(-20);
                        const R c3 = gi == 0 ? R(4) : R(15), c4 = gi == 0 ? R(-1) : R(-4);
                        g0 = c1 * f[0] + c2 * f[-2] + c3 * f[-4] + c4 * f[-6];
                        g1 = c1 * f[1] + c2 * f[-1] + c3 * f[-3] + c4 * f[-5];
                    }
                    const int colR = Nx + gi - x0;       // beyond the box only if never referenced
                    if (colR < kRowLen) {
                        row[2 * colR] = g0;
                        row[2 * colR + 1] = g1;
                    }
                }
            }
            __syncwarp();
        }
        if (mirror) {
            if (lane < 3 * NQ) {
                const int q = lane / 3, g = lane - 3 * q;
                bool okq = ok[0];
#pragma unroll
                for (int qq = 1; qq < NQ; ++qq)
                    if (q == qq) okq = ok[qq];
                if (okq && LBC_CHECK(ctl, -3 - x0 >= 0 && -1 - x0 < kRowLen, CK_STENCIL)) {
                    R *gp = fin + (size_t)(warp + kWarps * q) * 2 * kRowLen + 2 * (-1 - g - x0);   // node -1 - g
                    gp[0] = mg0;
                    gp[1] = mg1;
                }
            }
            __syncwarp();
            mirror_fetch(sub + 1);
        }
        if constexpr (kLean) {
            // plain FP32 form: (phi, chi) as packed pairs. Rows warp + kWarps q of the slot; a
            // row past the chunk computes on the chunk's last row and stores nothing.
            const int vs = vbeg + sub * kSub;                  // first row of the slot
            const int v0 = vs + warp;                           // this warp's row q = 0
            const float *rowq = fin + (size_t)warp * 2 * kRowLen + 2 * (ck - 3);   // row q = 0, node ck - 3
            const float *b0 = f0 + (size_t)warp * 2 * kF0Len + 2 * (lane + offf);
            const int vlast = min(vs + kSub, vend) - 1, vhalf = T.Qx * T.Qy;
            f2 ps[5];
#pragma unroll
            for (int m = 0; m < 5; ++m) ps[m] = bc2(0.f);
            float psxy = 0.f;
            // The slot's rows, compiled for where they lie. Rows v < Qx Qy have p_x > 0 and upwind
            // from the left, the others from the right: a slot whose rows all lie in one half
            // (kSide 1 or -1, all slots but one per velocity set) takes its stencils at fixed
            // offsets with no per-row choice; the slot across the halves (kSide 0) chooses per
            // row. kFull: every row of the slot is inside the chunk (all but a chunk's last slot);
            // kInner: the tile's stencils reach no wall (all but the channel's end tiles).
            auto rows = [&](auto side_c, auto full_c, auto inner_c) {
                constexpr int kSide = decltype(side_c)::value;
                constexpr bool kFull = decltype(full_c)::value, kInner = decltype(inner_c)::value;
                // rows in pairs (q = qp, qp + 1): two WENO chains in flight, fewer live registers
#pragma unroll
                for (int qp = 0; qp < NQ; qp += 2) {
                    f2 fl[2], dd[2];
#pragma unroll
                    for (int qi = 0; qi < 2; ++qi) {
                        const int q = qp + qi;
                        const bool pos = kSide > 0 || (kSide == 0 && v0 + kWarps * q < vhalf);   // uniform per warp
                        const float *pp = rowq + (size_t)q * kWarps * 2 * kRowLen + (pos ? 0 : 2);
                        const f2 a = ld2(pp), b = ld2(pp + 2), c = ld2(pp + 4), d = ld2(pp + 6), e = ld2(pp + 8);
                        if constexpr (kSide > 0) {
                            fl[qi] = weno5_2(a, b, c, d, e);
                            dd[qi] = d;
                        } else if constexpr (kSide < 0) {
                            fl[qi] = weno5_2(e, d, c, b, a);
                            dd[qi] = c;
                        } else {
                            fl[qi] = weno5_2(pos ? a : e, pos ? b : d, c, pos ? d : b, pos ? e : a);
                            dd[qi] = pos ? d : c;
                        }
                    }
#pragma unroll
                    for (int qi = 0; qi < 2; ++qi) {
                        const int q = qp + qi;
                        const int v = v0 + kWarps * q;
                        const bool okq = kFull || v < vend;
                        const float *xr = s_vrow + (size_t)((kFull ? v : min(v, vend - 1)) - vbeg) * kVRow;
                        const float4 xa = *reinterpret_cast<const float4 *>(xr);       // p_x p_y w ft_rest
                        const float2 xg = *reinterpret_cast<const float2 *>(xr + VR_GA);
                        const float px = xa.x, py = xa.y, w = xa.z, fr = xa.w;
                        if (!kInner && wall) {   // wall faces: the incoming population n_w f_w (Eq. diffuse)
                            const float4 xw = *reinterpret_cast<const float4 *>(xr + VR_FWL);
                            if (needL && px > 0.f && s == 0) fl[qi] = mk2(nwL * xw.x - fr, nwL * xw.y - fr);
                            if (needR && px < 0.f && s == Nx) fl[qi] = mk2(nwR * xw.z - fr, nwR * xw.w - fr);
                        }
                        int ga = __float_as_int(xg.x), gj = __float_as_int(xg.y);
                        if (!LBC_CHECK(ctl, ga >= 0 && gj >= 0 && ga + kLanes <= G * kLanes && gj + kLanes <= G * kLanes,
                                       CK_GTAB))
                            ga = gj = 0;
                        const float feq = n_c * s_g[ga + lane] * s_g[gj + lane];
                        const float xx = px - ux_c, xy = py - uy_c;
                        const float xx2 = xx * xx, e2 = fmaf(xy, xy, xx2);
                        const float sq = fmaf(shA, xx, shB * xy);        // cS (q . xi)
                        const float h = e2 * i5T;                         // xi^2 / (5 T)
                        // Shakhov targets minus the rest state (Sec. II, the reduced S_phi, S_chi)
                        const float fT = T_c * feq;                       // chi_eq = T phi_eq
                        const float tp = fmaf(feq * sq, h - 0.8f, feq) - fr;
                        const float tc = fmaf(fT * sq, h - 0.4f, fT) - fr;
                        float fll, flh;
                        un2(fl[qi], fll, flh);
                        const float frl = __shfl_down_sync(0xffffffffu, fll, 1);
                        const float frh = __shfl_down_sync(0xffffffffu, flh, 1);
                        float dl, dh;
                        un2(dd[qi], dl, dh);
                        const float kp = k3 * px;
                        float ol = fmaf(kp, fll - frl, fmaf(k2, tp, k1 * dl));
                        float oh = fmaf(kp, flh - frh, fmaf(k2, tc, k1 * dh));
                        if constexpr (stage > 0) {
                            float d0l, d0h;
                            un2(ld2(b0 + (size_t)q * kWarps * 2 * kF0Len), d0l, d0h);
                            ol = fmaf(ca_of<float>(stage), d0l, ol);
                            oh = fmaf(ca_of<float>(stage), d0h, oh);
                            if constexpr (stage == 2)
                                if (active && okq) res = fmaxf(res, w * fmaxf(fabsf(ol - d0l), fabsf(oh - d0h)));
                        }
                        if (active && okq && LBC_CHECK(ctl, v < T.V && s < Nxp, CK_STORE)) {
                            st2(Fout_s + 2 * (size_t)Nxp * v, mk2(ol, oh));
                            // the pairs as the packed operations produce them: (fw, gw) = w (phi, chi)
                            const f2 fg = mk2(ol, oh) * bc2(w);
                            float fw, gw;
                            un2(fg, fw, gw);
                            const f2 pxy = mk2(xx, xy);
                            ps[0] = ps[0] + fg;                                           // (S0, CZ)
                            ps[1] = fma2(bc2(xx), fg, ps[1]);                             // (SX, GX)
                            ps[2] = fma2(bc2(xy), fg, ps[2]);                             // (SY, GY)
                            ps[3] = fma2(pxy * pxy, bc2(fw), ps[3]);                      // (SXX, SYY)
                            ps[4] = fma2(bc2(e2) * pxy, bc2(fw), ps[4]);                  // (R3X, R3Y)
                            psxy = fmaf(xx * xy, fw, psxy);
                        }
                    }
                }
            };
            using Pos = std::integral_constant<int, 1>;
            using Neg = std::integral_constant<int, -1>;
            using Mix = std::integral_constant<int, 0>;
            using Yes = std::true_type;
            using No = std::false_type;
            const bool full = vs + kSub <= vend;
            if (vlast < vhalf) {
                if (full && !wall) rows(Pos(), Yes(), Yes());
                else rows(Pos(), No(), No());
            } else if (vs >= vhalf) {
                if (full && !wall) rows(Neg(), Yes(), Yes());
                else rows(Neg(), No(), No());
            } else {
                rows(Mix(), No(), No());
            }
            // the slot's partial sums into the running sums, compensated (Kahan)
#pragma unroll
            for (int m = 0; m < 5; ++m) kahan2(pk[m], pkc[m], ps[m]);
            kahan1(acc[R_SXY], sxyc, psxy);
        } else if constexpr (std::is_same<R, float>::value) {
            // FP32: (phi, chi) as packed pairs, loaded and stored as one 64-bit access each.
            f2 ps[5];   // the slot's partial moment sums
#pragma unroll
            for (int m = 0; m < 5; ++m) ps[m] = bc2(0.f);
            float psxy = 0.f;
            // Face c0 + lane of each row: rows v < Qx Qy have p_x > 0 and upwind from the
            // left (nodes ck-3 .. ck+1), the others from the right (nodes ck+2 .. ck-2). A slot
            // whose rows all share a side loads its stencils at fixed offsets.
            f2 fl[NQ], dd[NQ];
            const int vq0 = vbeg + sub * kSub, vq1 = min(vq0 + kSub, vend) - 1;
            const int vhalf = T.Qx * T.Qy;
            const float *rowq = fin + (size_t)warp * 2 * kRowLen + 2 * (ck - 3);   // row warp, node ck - 3
            if (vq1 < vhalf) {
#pragma unroll
                for (int q = 0; q < NQ; ++q) {
                    const float *pp = rowq + (size_t)q * kWarps * 2 * kRowLen;
                    f2 v[5];
#pragma unroll
                    for (int i = 0; i < 5; ++i) v[i] = ld2(pp + 2 * i);
                    fl[q] = weno5_2(v[0], v[1], v[2], v[3], v[4]);
                    dd[q] = v[3];
                }
            } else if (vq0 >= vhalf) {
#pragma unroll
                for (int q = 0; q < NQ; ++q) {
                    const float *pp = rowq + (size_t)q * kWarps * 2 * kRowLen + 2;
                    f2 v[5];
#pragma unroll
                    for (int i = 0; i < 5; ++i) v[i] = ld2(pp + 2 * i);
                    fl[q] = weno5_2(v[4], v[3], v[2], v[1], v[0]);
                    dd[q] = v[2];
                }
            } else {   // the slot holds both signs: upwind order per row
#pragma unroll
                for (int q = 0; q < NQ; ++q) {
                    const float4 xa = *reinterpret_cast<const float4 *>(s_vrow + kq[q] * kVRow);   // px py w fr
                    const bool pos = xa.x > 0.f;
                    const int base = pos ? ck - 3 : ck + 2, st = pos ? 1 : -1;
                    const float *row = fin + (size_t)(warp + kWarps * q) * 2 * kRowLen;
                    f2 v[5];
#pragma unroll
                    for (int i = 0; i < 5; ++i) v[i] = ld2(row + 2 * (base + i * st));
                    fl[q] = weno5_2(v[0], v[1], v[2], v[3], v[4]);
                    dd[q] = pos ? v[3] : v[2];   // the node itself
                }
            }
            if (wall) {   // wall faces: the incoming population n_w f_w (Eq. diffuse)
#pragma unroll
                for (int q = 0; q < NQ; ++q) {
                    const float4 xa = *reinterpret_cast<const float4 *>(s_vrow + kq[q] * kVRow);
                    const float4 xw = *reinterpret_cast<const float4 *>(s_vrow + kq[q] * kVRow + 4);
                    const bool pos = xa.x > 0.f;
                    if (needL && pos && s == 0) fl[q] = mk2(nwL * xw.x - xa.w, nwL * xw.y - xa.w);
                    if (needR && !pos && s == Nx) fl[q] = mk2(nwR * xw.z - xa.w, nwR * xw.w - xa.w);
                }
            }
#pragma unroll
            for (int q = 0; q < NQ; ++q) {
                const float4 xa = *reinterpret_cast<const float4 *>(s_vrow + kq[q] * kVRow);   // px py w fr
                const float4 xg = *reinterpret_cast<const float4 *>(s_vrow + kq[q] * kVRow + 8);
                int ga = __float_as_int(xg.x), gj = __float_as_int(xg.y);
                if (!LBC_CHECK(ctl, ga >= 0 && gj >= 0 && ga + kLanes <= G * kLanes && gj + kLanes <= G * kLanes,
                               CK_GTAB))
                    ga = gj = 0;
                const int r = warp + kWarps * q, v = vbeg + kq[q];
                const float px = xa.x, py = xa.y, w = xa.z, fr = xa.w;
                const float feq = n_c * s_g[ga + lane] * s_g[gj + lane];
                const float xx = px - ux_c, xy = py - uy_c;
                const float qxi = qx_c * xx + qy_c * xy;
                const float e2 = xx * xx + xy * xy;
                float fll, flh;
                un2(fl[q], fll, flh);
                const f2 frt = mk2(__shfl_down_sync(0xffffffffu, fll, 1), __shfl_down_sync(0xffffffffu, flh, 1));
                const f2 adv = (fl[q] - frt) * bc2(px * ijd);
                // Shakhov targets minus the rest state: (phi_eq (1 + S_phi), chi_eq (1 + S_chi)) - ft_rest
                const f2 sh = fma2(bc2(cS_c * qxi), bc2(e2 * i5T) - mk2(0.8f, 0.4f), bc2(1.f));
                const f2 tgt = fma2(mk2(feq, T_c * feq), sh, bc2(-fr));
                const f2 lr = fma2(bc2(-nu_c), dd[q] - tgt, adv);   // L of this stage
                f2 dn = fma2(bc2(dt), lr, dd[q]);
                // the node's own state (and compensation) entries: stored only inside the arrays
                const bool okw = active && ok[q] && LBC_CHECK(ctl, v >= 0 && v < T.V && s < Nxp, CK_STORE);
                const f2 dtl = comp_any ? bc2(dt) * lr : bc2(0.f);
                float *ap = comp_any ? static_cast<float *>(S.A) + 2 * ((size_t)Nxp * v + s) : nullptr;
                if (comp_any && stage < 2 && okw) st2(ap, stage == 0 ? dtl : ld2(ap) + dtl);
                if (stage > 0) {
                    const f2 d0 = ld2(f0 + (size_t)r * 2 * kF0Len + 2 * (lane + offf));
                    if (comp) {
                        // the step's increment dt (L0 + L1) / 6 + 2/3 dt L2, added to d0 + c0 with its
                        // rounding error kept (TwoSum of Knuth): increments below half an ulp of d0 count
                        f2 inc = bc2(2.f / 3.f) * dtl;
                        if (okw) inc = fma2(bc2(1.f / 6.f), ld2(ap), inc);
                        if (renorm) inc = fma2(bc2(lam1r), d0 + inc + bc2(fr), inc);
                        float *cp = static_cast<float *>(S.C) + 2 * ((size_t)Nxp * v + s);
                        f2 cs = inc;
                        if (okw) cs = ld2(cp) + inc;
                        const f2 sn = d0 + cs, bv = sn - d0;
                        const f2 er = (d0 - (sn - bv)) + (cs - bv);
                        dn = sn;
                        if (okw) {
                            st2(cp, er);
                            float e0, e1;
                            un2(inc, e0, e1);
                            res = fmaxf(res, w * fmaxf(fabsf(e0), fabsf(e1)));
                        }
                    } else {
                        dn = fma2(bc2(ca), d0, bc2(cb) * dn);
                        if (renorm) dn = fma2(bc2(lam1r), dn + bc2(fr), dn);   // lambda (d + ft_rest) - ft_rest
                        if (stage == 2 && okw) {
                            float e0, e1;
                            un2(dn - d0, e0, e1);
                            res = fmaxf(res, w * fmaxf(fabsf(e0), fabsf(e1)));
                        }
                    }
                }
                if (okw) {
                    st2(Fout_s + 2 * (size_t)Nxp * v, dn);
                    const f2 fg = bc2(w) * dn;                 // (fw, gw)
                    float fw, gw;
                    un2(fg, fw, gw);
                    const f2 pxy = mk2(xx, xy);
                    ps[0] = ps[0] + fg;                        // (S0, CZ)
                    ps[1] = fma2(pxy, bc2(fw), ps[1]);         // (SX, SY)
                    ps[2] = fma2(pxy, bc2(gw), ps[2]);         // (GX, GY)
                    ps[3] = fma2(pxy * pxy, bc2(fw), ps[3]);   // (SXX, SYY)
                    ps[4] = fma2(bc2(e2) * pxy, bc2(fw), ps[4]);   // (R3X, R3Y)
                    psxy = fmaf(xx * xy, fw, psxy);
                }
            }
            // the slot's partial sums into the running sums, compensated (Kahan)
#pragma unroll
            for (int m = 0; m < 5; ++m) kahan2(pk[m], pkc[m], ps[m]);
            kahan1(acc[R_SXY], sxyc, psxy);
        } else {
            // FP64: rows in pairs (q = qp, qp + 1), which bounds the live registers
#pragma unroll
            for (int qp = 0; qp < NQ; qp += 2) {
                R fl[2][2], dd[2][2];
#pragma unroll
                for (int qi = 0; qi < 2; ++qi) {
                    const int q = qp + qi;
                    const R *x = s_vrow + kq[q] * kVRow;
                    const bool pos = x[VR_PX] > R(0);
                    const int base = pos ? ck - 3 : ck + 2, st = pos ? 1 : -1;   // upwind stencil order
                    const R *row = fin + (size_t)(warp + kWarps * q) * 2 * kRowLen;
                    R v[5][2];
#pragma unroll
                    for (int i = 0; i < 5; ++i) {
                        const double2 t = *reinterpret_cast<const double2 *>(row + 2 * (base + i * st));
                        v[i][0] = t.x;
                        v[i][1] = t.y;
                    }
#pragma unroll
                    for (int fld = 0; fld < 2; ++fld) {
                        // face c0 + lane (left of node c0 + lane)
                        fl[qi][fld] = weno5<R>(v[0][fld], v[1][fld], v[2][fld], v[3][fld], v[4][fld]);
                        dd[qi][fld] = pos ? v[3][fld] : v[2][fld];
                        if (wall) {
                            if (needL && pos && s == 0) fl[qi][fld] = nwL * x[VR_FWL + fld] - x[VR_FR];
                            if (needR && !pos && s == Nx) fl[qi][fld] = nwR * x[VR_FWR + fld] - x[VR_FR];
                        }
                    }
                }
#pragma unroll
                for (int qi = 0; qi < 2; ++qi) {
                    const int q = qp + qi;
                    const R *x = s_vrow + kq[q] * kVRow;
                    int ga = row_bits(x[VR_GA]), gj = row_bits(x[VR_GJ]);
                    if (!LBC_CHECK(ctl, ga >= 0 && gj >= 0 && ga + kLanes <= G * kLanes && gj + kLanes <= G * kLanes,
                                   CK_GTAB))
                        ga = gj = 0;
                    const int r = warp + kWarps * q, v = vbeg + kq[q];
                    const R px = x[VR_PX], py = x[VR_PY], w = x[VR_W], fr = x[VR_FR];
                    const R feq = n_c * s_g[ga + lane] * s_g[gj + lane];
                    const R xx = px - ux_c, xy = py - uy_c;
                    const R qxi = qx_c * xx + qy_c * xy;
                    const R x2 = (xx * xx + xy * xy) * i5T;
                    R fo[2];
                    const double2 d0 = stage > 0 ? *reinterpret_cast<const double2 *>(f0 + (size_t)r * 2 * kF0Len +
                                                                                     2 * (lane + offf))
                                                 : make_double2(0.0, 0.0);
#pragma unroll
                    for (int fld = 0; fld < 2; ++fld) {
                        const R frt = __shfl_down_sync(0xffffffffu, fl[qi][fld], 1);
                        const R d = dd[qi][fld];
                        const R adv = -px * (frt - fl[qi][fld]) * ijd;
                        // Shakhov target minus the rest state
                        const R tgt = fld ? T_c * feq * (R(1) + cS_c * (x2 - R(0.4)) * qxi) - fr
                                          : feq * (R(1) + cS_c * (x2 - R(0.8)) * qxi) - fr;
                        R dn = d + dt * (adv - nu_c * (d - tgt));
                        if (stage > 0) {
                            const R b0 = fld ? d0.y : d0.x;
                            dn = ca * b0 + cb * dn;
                            if (renorm) dn = fma(lam1r, dn + fr, dn);   // lambda (d + ft_rest) - ft_rest
                            if (stage == 2 && active && ok[q]) res = fmax(res, w * fabs(dn - b0));
                        }
                        fo[fld] = dn;
                    }
                    if (active && ok[q] && LBC_CHECK(ctl, v >= 0 && v < T.V && s < Nxp, CK_STORE)) {
                        *reinterpret_cast<double2 *>(Fout_s + 2 * (size_t)Nxp * v) = make_double2(fo[0], fo[1]);
                        const R fw = w * fo[0], gw = w * fo[1];
                        const R e2 = xx * xx + xy * xy;
                        acc[R_S0] += fw;
                        acc[R_SX] += xx * fw;
                        acc[R_SY] += xy * fw;
                        acc[R_SXX] += xx * xx * fw;
                        acc[R_SXY] += xx * xy * fw;
                        acc[R_SYY] += xy * xy * fw;
                        acc[R_CZ] += gw;
                        acc[R_R3X] += e2 * xx * fw;
                        acc[R_R3Y] += e2 * xy * fw;
                        acc[R_GX] += xx * gw;
                        acc[R_GY] += xy * gw;
                    }
                }
            }
        }
        // release slot p: order this warp's accesses to it before the refill's async writes;
        // the warp that completes the round issues the refill
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncwarp();
        if (lane == 0) {
            const uint32_t ticket = atom_add_acq_rel(&s_cnt[p], 1u);
            if (ticket == (uint32_t)((sub / kPipe + 1) * kWarps - 1) && sub + kPipe < nsub) issue(sub + kPipe);
        }
    }
    if (my_timeout && lane == 0) *reinterpret_cast<volatile int *>(s_abort) = 1;
    timed_out = __syncthreads_or(timed_out || my_timeout);

    const int rank = (int)cluster_ctarank(), nch = T.nchunk;
    const int nn = (kTile - rank + nch - 1) / nch;          // nodes rank, rank + nch, ... of the tile
    const int nnmax = (kTile + nch - 1) / nch;
    unsigned char *scr = smem + L.pipe;                     // EqScratch
    if (!kSplit && !timed_out && tid < (kSolo ? kTile : nn)) {   // the node step's per-node data, towards L1
        const int sp = kSolo ? c0 + tid : c0 + rank + tid * nch;
        if (sp < T.Nx) {
            prefetch_l1(Tabs<R>::ijd(T) + sp);
            prefetch_l1(Tabs<R>::dtn(T) + sp);
            if (renorm) prefetch_l1(T.jdeta + sp);
        }
    }
    if (timed_out) {
        // give up: record it and let in-flight copies land (bounded); the CTA
        // still takes part in the cluster barriers below, without touching data
        if (tid == 0) {
            atomicExch(&ctl->timeout, 1);
            // copies issued to slot p: its first fill (if p < nsub) and one refill per completed
            // release round while rows remained. A slot has at most one copy outstanding (it is
            // refilled only after every warp waited for its previous copy): wait for the last one
            for (int p = 0; p < kPipe && p < nsub; ++p) {
                const int rounds = (int)(s_cnt[p] / kWarps);
                const int fills = 1 + min(rounds, (nsub - 1 - p) / kPipe);
                mbar_wait(&bar[p], (uint32_t)((fills - 1) & 1));
            }
            mbar_wait(bar_data, 0);
        }
        __syncthreads();
        if constexpr (kSolo) {
            solo_count_in();   // keeps the tile's count consistent for the next launch
        } else if constexpr (!kSplit) {
            cluster_wait();
            cluster_arrive();
            cluster_wait();
        }
        if (persist && tid < kPipe + 2) mbar_inval(&bar[tid]);   // the next item initialises them again
        return;
    }

    // ---- (4) the chunk's raw moment partials, sent to the CTAs that own the nodes ----
    if (!kSplit && tid == 0) {   // the equilibrium tables, into the pipeline region that the loop no longer reads
        mbar_expect_tx(bar_tab, tab_bytes);
        bulk_load(scr + E.tab, Tabs<R>::eqtab(T), tab_bytes, bar_tab);
    }
    if constexpr (std::is_same<R, float>::value) {
        // Kahan's sum is s - c
#pragma unroll
        for (int m = 0; m < 5; ++m) pk[m] = pk[m] - pkc[m];
        acc[R_SXY] -= sxyc;
        un2(pk[0], acc[R_S0], acc[R_CZ]);
        if constexpr (kLean) {   // the plain loop pairs its sums by coordinate: (SX, GX), (SY, GY)
            un2(pk[1], acc[R_SX], acc[R_GX]);
            un2(pk[2], acc[R_SY], acc[R_GY]);
        } else {
            un2(pk[1], acc[R_SX], acc[R_SY]);
            un2(pk[2], acc[R_GX], acc[R_GY]);
        }
        un2(pk[3], acc[R_SXX], acc[R_SYY]);
        un2(pk[4], acc[R_R3X], acc[R_R3Y]);
    }
    R *s_red = reinterpret_cast<R *>(scr);   // [kWarps][kNumRaw][kLanes], below E.tab
#pragma unroll
    for (int m = 0; m < kNumRaw; ++m) s_red[(warp * kNumRaw + m) * kLanes + lane] = acc[m];
    if (stage == 2) {
        R rr = res;
        for (int o = 16; o > 0; o >>= 1) rr = fmax(rr, __shfl_xor_sync(0xffffffffu, rr, o));
        if (lane == 0 && rr > R(0))
            atomicMax(&S.resid[step % kResidRing], (unsigned long long)__double_as_longlong((double)rr));
    }
    __syncthreads();
    // local steps: the mass deviations of f^{n+1} (buffer 0) for the next step's parity
    double *dm = renorm ? S.mass + kMassHdr + (size_t)((step + 1) & 1) * T.Nxp : nullptr;
    if constexpr (kSolo || kSplit) {
        // ---- (4') the chunk's partials (summed over warps) to global memory [nchunk][kNumRaw][Nxp] ----
        R *part = static_cast<R *>(S.part);
        for (int idx = tid; idx < kTile * kNumRaw; idx += kThreads) {
            const int m = idx / kTile, c = idx - m * kTile;   // consecutive threads: consecutive nodes
            if (c0 + c < T.Nx) {
                CSum<R> t;
                for (int w2 = 0; w2 < kWarps; ++w2) t.add(s_red[(w2 * kNumRaw + m) * kLanes + c]);
                if (LBC_CHECK(ctl, chunk < kMaxCluster && c0 + c < T.Nxp, CK_XCH))
                    part[((size_t)chunk * kNumRaw + m) * T.Nxp + c0 + c] = t.value();
            }
        }
        if constexpr (kSplit) return;   // the node step is a launch of its own
        const bool last = solo_count_in();
        if (!last) {   // the table copy into this CTA's shared memory must land before it leaves
            if (tid == 0) mbar_wait(bar_tab, 0);
            return;
        }
        // ---- (5') the tile's last CTA: every chunk's partials (L2), the next stage's data of all nodes ----
        R *raw = reinterpret_cast<R *>(scr + E.raw);
        R *shf = reinterpret_cast<R *>(scr + E.shf);
        for (int idx = tid; idx < kTile * kNumRaw; idx += kThreads) {
            const int i = idx / kNumRaw, m = idx - i * kNumRaw;
            CSum<R> t;
            if (c0 + i < T.Nx)
                for (int ch = 0; ch < nch; ++ch) t.add(__ldcg(&part[((size_t)ch * kNumRaw + m) * T.Nxp + c0 + i]));
            raw[idx] = t.value();
        }
        if (tid < kLanes) {   // warp 0, lane = node: the sums are about the input stage's mean velocity
            shf[tid] = ux_c;
            shf[kLanes + tid] = uy_c;
        }
        const bool late = __syncthreads_or(!mbar_wait(bar_tab, 0));
        if (late) {
            if (tid == 0) atomicExch(&ctl->timeout, 1);
            return;
        }
        node_equilibrium<R>(T, S, out, tile, 0, 1, kTile, kTile, scr, dm, nullptr);
        return;
    }
    cluster_wait();   // every CTA of the cluster has started (pairs with the arrive at the top)
    for (int idx = tid; idx < kTile * kNumRaw; idx += kThreads) {
        const int c = idx / kNumRaw, m = idx - c * kNumRaw;
        CSum<R> t;
        for (int w2 = 0; w2 < kWarps; ++w2) t.add(s_red[(w2 * kNumRaw + m) * kLanes + c]);
        const int owner = c % nch, i = c / nch;
        if (LBC_CHECK(ctl, owner < nch && rank * nnmax + i < kTile + kMaxCluster, CK_XCH))
            st_cluster(&s_xch[((size_t)rank * nnmax + i) * kNumRaw + m], (uint32_t)owner, t.value());
    }
    cluster_arrive();
    cluster_wait();   // every chunk's partials of this CTA's nodes are in s_xch

    // ---- (5) the next stage's data of this CTA's nodes ----
    {
        R *raw = reinterpret_cast<R *>(scr + E.raw);
        R *shf = reinterpret_cast<R *>(scr + E.shf);
        for (int idx = tid; idx < nn * kNumRaw; idx += kThreads) {
            const int i = idx / kNumRaw, m = idx - i * kNumRaw;
            CSum<R> t;
            for (int ch = 0; ch < nch; ++ch) t.add(s_xch[((size_t)ch * nnmax + i) * kNumRaw + m]);
            raw[idx] = t.value();
        }
        if (tid < kLanes) {   // warp 0, lane = node: the sums are about the input stage's mean velocity
            shf[tid] = ux_c;
            shf[kLanes + tid] = uy_c;
        }
    }
    const bool tab_late = __syncthreads_or(!mbar_wait(bar_tab, 0));
    if (tab_late) {
        if (tid == 0) atomicExch(&ctl->timeout, 1);
        return;
    }
    node_equilibrium<R>(T, S, out, tile, rank, nch, nn, ncap, scr, dm, nullptr);
    if (persist) {   // the item's mbarriers are done with: the next item initialises them again
        __syncthreads();
        if (tid < kPipe + 2) mbar_inval(&bar[tid]);
    }
}

// Single instance: the descriptor is a kernel parameter (constant bank), grid (ntile, nchunk).
template <typename R, bool kExt, int kStage>
__global__ void __launch_bounds__(kThreads, sizeof(R) == 4 ? 4 : 2)
stage_kernel(const __grid_constant__ Inst I, int rel)
{
    stage_body<R, kExt, kStage, kFormCluster>(I, blockIdx.x, rel);
}

// Batch: descriptors in device memory, one cluster per work item (instance, tile).
// Three CTAs per SM in FP32: the descriptor fields live in registers here (in the
// single-instance kernel they are constant-bank operands), and measured on GB300
// the unspilled 3-CTA form is faster than a spilling 4-CTA form.
template <typename R, bool kExt, int kStage, int kForm>
__global__ void __launch_bounds__(kThreads, sizeof(R) == 4 ? 3 : 2)
stage_batch_kernel(const Inst *__restrict__ insts, const int2 *__restrict__ work, int rel)
{
    const int2 wk = work[blockIdx.x];
    if (wk.x < 0) return;   // empty work slot: the whole cluster (or every chunk CTA) leaves
    stage_body<R, kExt, kStage, kForm>(insts[wk.x], wk.y, rel);
}

// Split form, the RK stage's second launch: the next-stage data of nodes
// blockIdx.y * kNodePart .. of a work item's tile, from the chunk partials the stage
// launch left in DevState::part (summed over the chunks in chunk order, as the other
// forms sum them) and the input stage's mean velocities (the shift of those sums),
// by the node step of the other forms. Every tile's node step runs at once, spread
// over the whole GPU, instead of in the stage launch's last CTAs.
template <typename R>
__global__ void __launch_bounds__(kThreads)
node_step_kernel(const Inst *__restrict__ insts, const int2 *__restrict__ work, int rel, int stage)
{
    const int2 wk = work[blockIdx.x];
    if (wk.x < 0) return;   // empty work slot
    const Inst &I = insts[wk.x];
    const DevTables &T = I.T;
    const DevState &S = I.S;
    const Ctl *ctl = S.ctl;
    const long long step = ctl->base + rel;
    // early stop: the stage launch's decision, taken again from the same data
    const double stop_eps = ctl->stop_eps;
    if (stop_eps > 0.0) {
        if (__ldcg(&ctl->stopped)) return;
        if (step - 1 >= ctl->check_from) {
            const double rprev = __longlong_as_double((long long)__ldcg(&S.resid[(step - 1) % kResidRing]));
            if (rprev < stop_eps) return;
        }
    }
    extern __shared__ __align__(128) unsigned char smem_node[];
    unsigned char *scr = smem_node + ((128 - (smem_addr(smem_node) & 127)) & 127);
    const int tid = threadIdx.x, tile = wk.y, c0 = tile * kTile, cfirst = blockIdx.y * kNodePart;
    const int nn = min(kNodePart, kTile - cfirst), nch = T.nchunk, in = stage, out = (stage + 1) % 3;
    const EqScratch<R> E(T.K, T.Nxe, T.Nye, T.Qx, T.Qy, T.tab_n, kTile);
    const int tlen = EqTab(T.Nxe, T.Nye, T.K, T.Qx, T.Qy, T.tab_n).len;
    R *tab = reinterpret_cast<R *>(scr + E.tab);
    for (int k = tid; k < tlen; k += kThreads) tab[k] = Tabs<R>::eqtab(T)[k];
    R *raw = reinterpret_cast<R *>(scr + E.raw);
    R *shf = reinterpret_cast<R *>(scr + E.shf);
    const R *part = static_cast<const R *>(S.part);
    for (int idx = tid; idx < nn * kNumRaw; idx += kThreads) {
        const int i = idx / kNumRaw, m = idx - i * kNumRaw, s = c0 + cfirst + i;
        CSum<R> t;
        if (s < T.Nx)
            for (int ch = 0; ch < nch; ++ch) t.add(part[((size_t)ch * kNumRaw + m) * T.Nxp + s]);
        raw[idx] = t.value();
    }
    if (tid < kLanes) {   // lane = node of the tile: the input stage's mean velocity
        const int s = c0 + tid;
        const bool live = tid < kTile && s < T.Nx;
        const R *e = static_cast<const R *>(S.eqm[in]) + (size_t)(live ? s : 0) * kEqM;
        shf[tid] = live ? e[1] : R(0);
        shf[kLanes + tid] = live ? e[2] : R(0);
    }
    __syncthreads();
    // local steps: the mass deviations of f^{n+1} (buffer 0) for the next step's parity
    double *dm = T.lts && stage == 2 ? S.mass + kMassHdr + (size_t)((step + 1) & 1) * T.Nxp : nullptr;
    node_equilibrium<R>(T, S, out, tile, cfirst, 1, nn, kTile, scr, dm, nullptr);
}

// ---- persistent form: one launch for a group of steps of every work item ----
//
// Items (step, stage, work item) are handed out in that order from one counter to
// clusters that are all resident (cooperative launch, grid <= active clusters). An
// item waits until the tile and its two neighbours (the stencil's halo) finished
// the previous stage (done[w] counts a tile's finished stage items); an instance
// with early stop or local steps also waits, at stage 0, for its whole previous
// step (the residual and the mass are instance-wide). Every earlier item is held
// by a resident cluster, so every wait ends; each is also bounded, and on timeout
// the item's instance records it and the whole launch aborts.
__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned *p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ void st_cluster_u32(unsigned *local, uint32_t rank, unsigned v)
{
    uint32_t ra;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(ra) : "r"(smem_addr(local)), "r"(rank));
    asm volatile("st.shared::cluster.u32 [%0], %1;" ::"r"(ra), "r"(v) : "memory");
}

constexpr unsigned long long kDepWaitNs = 2000000000ull;   // 2 s per dependency wait at most

// Waits until *p >= need (acquire); false on timeout or abort.
__device__ bool wait_at_least(const unsigned *p, unsigned need, const unsigned *abort)
{
    if (ld_acquire_gpu(p) >= need) return true;
    const unsigned long long t0 = global_ns();
    for (;;) {
        __nanosleep(128);
        if (ld_acquire_gpu(p) >= need) return true;
        if (ld_acquire_gpu(abort) != 0u || global_ns() - t0 > kDepWaitNs) return false;
    }
}

template <typename R, bool kExt>
__global__ void __launch_bounds__(kThreads, sizeof(R) == 4 ? 3 : 2)
persistent_stage_kernel(const Inst *__restrict__ insts, const int2 *__restrict__ work, int nwork, int nsteps,
                        unsigned *cnt)
{
    // counters (zeroed before the launch): cnt[0] items handed out, cnt[1] abort flag, cnt[4 + w]
    // CTAs that finished a stage item of work item w, cnt[4 + nwork + i] CTAs of instance i that
    // finished a third stage
    unsigned *next = cnt, *abort = cnt + 1, *done = cnt + kPersistHdr, *inst_done = cnt + kPersistHdr + nwork;
    __shared__ unsigned s_item[2];   // this cluster's item and whether its dependencies are met
    const int tid = threadIdx.x;
    const uint32_t rank = cluster_ctarank(), csize = gridDim.y;
    const unsigned total = (unsigned)nsteps * 3u * (unsigned)nwork;
    cluster_arrive();   // every CTA of the cluster runs before the first item is written into its shared memory
    cluster_wait();
    // The cluster's first thread claims items from the counter, the next one while the current
    // one runs. A cluster takes its claimed items in increasing order and every cluster is
    // resident, so the smallest unfinished item is always running or about to run, and every
    // wait ends. That thread also checks the item's dependencies and tells the other CTAs, so
    // that every CTA of the cluster takes the same path through the stage.
    unsigned claimed = 0u;
    if (rank == 0 && tid == 0) claimed = atomicAdd(next, 1u);
    for (;;) {
        if (rank == 0 && tid == 0) {
            unsigned item = claimed, ok = 1u;
            if (item < total && ld_acquire_gpu(abort) == 0u) {
                const int rel = (int)(item / (3u * nwork)), stage = (int)((item / nwork) % 3u), w = (int)(item % nwork);
                const int2 wk = work[w];
                if (wk.x >= 0) {
                    const Inst &I = insts[wk.x];
                    const unsigned need = csize * (3u * rel + stage);
                    for (int dt = -1; dt <= 1 && ok; ++dt) {
                        const int t = wk.y + dt;
                        // the tile's neighbours are the adjacent work items of the same instance
                        if (t >= 0 && t < I.T.ntile &&
                            LBC_CHECK(I.S.ctl,
                                      w + dt >= 0 && w + dt < nwork && work[w + dt].x == wk.x && work[w + dt].y == t,
                                      CK_WORK))
                            ok = wait_at_least(&done[w + dt], need, abort);
                    }
                    // early stop and local steps use instance-wide data of the previous step
                    if (ok && stage == 0 && rel > 0 && (I.T.lts || I.S.ctl->stop_eps > 0.0))
                        ok = wait_at_least(&inst_done[wk.x], csize * (unsigned)(rel * I.T.ntile), abort);
                    if (!ok) {
                        atomicExch(&I.S.ctl->timeout, 1);
                        atomicExch(abort, 1u);
                    }
                }
            } else {
                item = total;
            }
            for (uint32_t r = 0; r < csize; ++r) {
                st_cluster_u32(&s_item[0], r, item);
                st_cluster_u32(&s_item[1], r, ok);
            }
            if (item < total && ok) claimed = atomicAdd(next, 1u);
        }
        cluster_arrive();
        cluster_wait();
        const unsigned item = s_item[0], ok = s_item[1];
        if (item >= total || !ok) break;
        if (tid == 0) {   // the producers' writes, seen by this CTA's loads and its TMA copies
            __threadfence();
            asm volatile("fence.proxy.async.global;" ::: "memory");
        }
        __syncthreads();
        const int rel = (int)(item / (3u * nwork)), stage = (int)((item / nwork) % 3u), w = (int)(item % nwork);
        const int2 wk = work[w];
        if (wk.x >= 0) {
            const Inst &I = insts[wk.x];
            if (stage == 0) stage_body<R, kExt, 0, kFormCluster>(I, wk.y, rel, true);
            else if (stage == 1) stage_body<R, kExt, 1, kFormCluster>(I, wk.y, rel, true);
            else stage_body<R, kExt, 2, kFormCluster>(I, wk.y, rel, true);
        }
        // completion: this CTA's writes fenced, then counted (the tile's stage item is done when
        // every CTA of its cluster has counted)
        __syncthreads();
        if (tid == 0) {
            __threadfence();
            atomicAdd(&done[w], 1u);
            if (stage == 2 && wk.x >= 0) atomicAdd(&inst_done[wk.x], 1u);
        }
    }
}

// Zeroes the residual slots of the steps [base, base + nsteps) of every instance (the
// persistent form's stages of a step run in any order across tiles).
__global__ void zero_resid_kernel(const Inst *insts, int n, int nsteps)
{
    for (int k = blockIdx.x; k < n; k += gridDim.x) {
        const Inst &I = insts[k];
        if (I.S.ctl->stop_eps > 0.0 && I.S.ctl->stopped) continue;   // keeps its last step's residual
        const long long base = I.S.ctl->base;
        for (int j = threadIdx.x; j < nsteps; j += blockDim.x) I.S.resid[(base + j) % kResidRing] = 0ull;
    }
}

// Stage data of every tile of buffer `buf` from the chunk partials of
// moments_partial_kernel (after set-up or lbc_set_state).
template <typename R>
__global__ void __launch_bounds__(kThreads)
tile_equilibrium_kernel(const __grid_constant__ DevTables T, const __grid_constant__ DevState S, int buf)
{
    extern __shared__ __align__(16) unsigned char smem_eq[];
    const EqScratch<R> E(T.K, T.Nxe, T.Nye, T.Qx, T.Qy, T.tab_n);
    R *tab = reinterpret_cast<R *>(smem_eq + E.tab);
    R *raw = reinterpret_cast<R *>(smem_eq + E.raw);
    R *shf = reinterpret_cast<R *>(smem_eq + E.shf);
    const R *part = static_cast<const R *>(S.part);
    const int c0 = blockIdx.x * kTile;
    const int tlen = EqTab(T.Nxe, T.Nye, T.K, T.Qx, T.Qy, T.tab_n).len;
    for (int k = threadIdx.x; k < tlen; k += kThreads) tab[k] = Tabs<R>::eqtab(T)[k];
    for (int idx = threadIdx.x; idx < kTile * kNumRaw; idx += kThreads) {
        const int c = idx / kNumRaw, m = idx - c * kNumRaw, s = c0 + c;
        CSum<R> acc;
        if (s < T.Nx)
            for (int ch = 0; ch < T.nchunk; ++ch) acc.add(part[((size_t)ch * kNumRaw + m) * T.Nxp + s]);
        raw[idx] = acc.value();
    }
    if (threadIdx.x < 2 * kLanes) shf[threadIdx.x] = R(0);   // the partials are sums about p = 0
    __syncthreads();
    // local steps: buffer 0's mass deviations serve the next step of either parity
    double *dm = T.lts && buf == 0 ? S.mass + kMassHdr : nullptr;
    node_equilibrium<R>(T, S, buf, blockIdx.x, 0, 1, kTile, kTile, smem_eq, dm, dm ? dm + T.Nxp : nullptr);
}

// Local steps: the reference mass deviation M_ref - sum_s J_s deta of a freshly
// installed state, summed exactly as the stage kernel sums M(f^n) - sum_s J_s deta.
__global__ void __launch_bounds__(kThreads) mass_reference_kernel(const double *dm, int Nx, double *ref)
{
    __shared__ double red[kWarps];
    const double t = block_mass_deviation(dm, Nx, red);
    if (threadIdx.x == 0) *ref = t;
}

// Raw moment sums (about p = 0) of the deviation in buffer `buf`, per velocity
// chunk, in the state precision (compensated sums in FP32).
template <typename R>
__global__ void __launch_bounds__(kThreads)
moments_partial_kernel(const __grid_constant__ DevTables T, const __grid_constant__ DevState S, int buf)
{
    __shared__ R red[kWarps][kNumRaw][kLanes];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int c0 = blockIdx.x * kTile, chunk = blockIdx.y, s = c0 + lane;
    const bool active = lane < kTile && s < T.Nx;
    const R *F = static_cast<const R *>(S.F[buf]);
    const R *vel = Tabs<R>::vel(T);
    CSum<R> acc[kNumRaw];
    const int vbeg = chunk * T.vchunk, vend = min(T.V, vbeg + T.vchunk);
    for (int v = vbeg + warp; v < vend && active; v += kWarps) {
        const R px = vel[VC_PX * T.V + v], py = vel[VC_PY * T.V + v], w = vel[VC_W * T.V + v];
        const R fw = w * F[2 * ((size_t)v * T.Nxp + s)];
        const R gw = w * F[2 * ((size_t)v * T.Nxp + s) + 1];
        const R e2 = px * px + py * py;
        acc[R_S0].add(fw); acc[R_SX].add(px * fw); acc[R_SY].add(py * fw);
        acc[R_SXX].add(px * px * fw); acc[R_SXY].add(px * py * fw); acc[R_SYY].add(py * py * fw);
        acc[R_CZ].add(gw); acc[R_R3X].add(e2 * px * fw); acc[R_R3Y].add(e2 * py * fw);
        acc[R_GX].add(px * gw); acc[R_GY].add(py * gw);
    }
#pragma unroll
    for (int m = 0; m < kNumRaw; ++m) red[warp][m][lane] = acc[m].value();
    __syncthreads();
    R *part = static_cast<R *>(S.part);
    for (int idx = tid; idx < kLanes * kNumRaw; idx += kThreads) {
        const int c = idx & 31, m = idx >> 5, sn = c0 + c;
        CSum<R> t;
        for (int w2 = 0; w2 < kWarps; ++w2) t.add(red[w2][m][c]);
        if (c < kTile && sn < T.Nx) part[((size_t)chunk * kNumRaw + m) * T.Nxp + sn] = t.value();
    }
}

// Moments of buffer 0 per node, FP64 [LBC_NMOM][Nxp], from its stage data (the
// stage kernel and the set-up build them for every node of every stage).
template <typename R>
__global__ void moments_from_stage_data_kernel(const R *eqm, int Nx, int Nxp, double *out)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= Nx) return;
    const R *e = eqm + (size_t)s * kEqM;
    const int src[LBC_NMOM] = {0, 1, 2, 3, 10, 11, 12, 13, 4, 5};   // n ux uy T Pxx Pyy Pzz Pxy qx qy
#pragma unroll
    for (int k = 0; k < LBC_NMOM; ++k) out[(size_t)k * Nxp + s] = (double)e[src[k]];
}

// Caller's weight-divided FP64 state [2][V][Nx] (in device memory) <-> deviation
// rows [V][Nxp][2] in the state precision. state_in sets *bad if a value is not finite.
template <typename R>
__global__ void state_in_kernel(const double *src, R *dst, R *carry, const double *frest, int V, int Nx, int Nxp,
                                int *bad)
{
    const size_t n = 2 * (size_t)V * Nx;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const size_t row = i / Nx, v = row % V, fld = row / V;
        const int s = (int)(i - row * Nx);
        const double x = src[i];
        if (bad && !isfinite(x)) *bad = 1;
        const double d = x - frest[v];
        const R dr = R(d);
        dst[2 * (v * Nxp + s) + fld] = dr;
        if (carry) carry[2 * (v * Nxp + s) + fld] = R(d - (double)dr);
    }
}

template <typename R>
__global__ void state_out_kernel(const R *src, const R *carry, double *dst, const double *frest, int V, int Nx,
                                 int Nxp)
{
    const size_t n = 2 * (size_t)V * Nx;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const size_t row = i / Nx, v = row % V, fld = row / V;
        const int s = (int)(i - row * Nx);
        const size_t k = 2 * (v * Nxp + s) + fld;
        dst[i] = frest[v] + ((double)src[k] + (carry ? (double)carry[k] : 0.0));
    }
}

__global__ void ctl_bump_kernel(Ctl *ctl, int n, long long k)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) ctl[i].base += k;
}

__global__ void last_residuals_kernel(const Inst *insts, const int *slots, int n, double *last)
{
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        const Inst &I = insts[slots ? slots[k] : k];
        const Ctl *c = I.S.ctl;
        const long long st = (c->stopped ? c->stop_step : c->base) - 1;
        last[k] = st >= 0 ? __longlong_as_double((long long)I.S.resid[st % kResidRing]) : 0.0;
    }
}

}  // namespace

template <typename R>
size_t stage_smem_bytes(int Qx, int Qy, int N, int Ny, int K, int vchunk, int cluster, int ntab)
{
    return Layout<R>(Qx, Qy, N, Ny, K, vchunk, cluster, ntab).total;
}

template <typename R>
cudaError_t configure_kernels()
{
    int dev = 0, optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    const void *stage_fns[24] = {
        (const void *)stage_kernel<R, false, 0>,              (const void *)stage_kernel<R, false, 1>,
        (const void *)stage_kernel<R, false, 2>,              (const void *)stage_kernel<R, true, 0>,
        (const void *)stage_kernel<R, true, 1>,               (const void *)stage_kernel<R, true, 2>,
        (const void *)stage_batch_kernel<R, false, 0, kFormCluster>, (const void *)stage_batch_kernel<R, false, 1, kFormCluster>,
        (const void *)stage_batch_kernel<R, false, 2, kFormCluster>, (const void *)stage_batch_kernel<R, true, 0, kFormCluster>,
        (const void *)stage_batch_kernel<R, true, 1, kFormCluster>,  (const void *)stage_batch_kernel<R, true, 2, kFormCluster>,
        (const void *)stage_batch_kernel<R, false, 0, kFormSolo>,  (const void *)stage_batch_kernel<R, false, 1, kFormSolo>,
        (const void *)stage_batch_kernel<R, false, 2, kFormSolo>,  (const void *)stage_batch_kernel<R, true, 0, kFormSolo>,
        (const void *)stage_batch_kernel<R, true, 1, kFormSolo>,   (const void *)stage_batch_kernel<R, true, 2, kFormSolo>,
        (const void *)stage_batch_kernel<R, false, 0, kFormSplit>, (const void *)stage_batch_kernel<R, false, 1, kFormSplit>,
        (const void *)stage_batch_kernel<R, false, 2, kFormSplit>, (const void *)stage_batch_kernel<R, true, 0, kFormSplit>,
        (const void *)stage_batch_kernel<R, true, 1, kFormSplit>,  (const void *)stage_batch_kernel<R, true, 2, kFormSplit>};
    // dynamic shared memory up to the opt-in limit less the kernel's static shared memory
    auto allow = [&](const void *fn) {
        cudaFuncAttributes fa = {};
        if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, fn);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    };
    for (const void *fn : stage_fns) allow(fn);
    const void *persist_fns[2] = {(const void *)persistent_stage_kernel<R, false>,
                                  (const void *)persistent_stage_kernel<R, true>};
    for (const void *fn : persist_fns) allow(fn);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(tile_equilibrium_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(node_step_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
    return e;
}

template <typename R>
size_t equilibrium_smem_bytes(int Qx, int Qy, int N, int Ny, int K, int ntab)
{
    return EqScratch<R>(K, N, Ny, Qx, Qy, ntab).total;
}

namespace {
cudaLaunchConfig_t cluster_config(unsigned nx, int cluster, size_t smem, cudaStream_t st, cudaLaunchAttribute *at)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(nx, (unsigned)cluster, 1);
    cfg.blockDim = dim3(kThreads, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = 1;
    at[0].val.clusterDim.y = (unsigned)cluster;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cfg;
}
}  // namespace

// One cluster per tile of one instance: its nchunk chunk CTAs (cluster dimension y).
template <typename R>
cudaError_t launch_stage(const Inst &I, size_t smem, int stage, int rel, cudaStream_t st)
{
    cudaLaunchAttribute at[1];
    cudaLaunchConfig_t cfg = cluster_config((unsigned)I.T.ntile, I.T.nchunk, smem, st, at);
    const bool ext = I.T.half || I.T.lts || I.T.comp;
    switch (stage + 3 * ext) {
    case 0: return cudaLaunchKernelEx(&cfg, stage_kernel<R, false, 0>, I, rel);
    case 1: return cudaLaunchKernelEx(&cfg, stage_kernel<R, false, 1>, I, rel);
    case 2: return cudaLaunchKernelEx(&cfg, stage_kernel<R, false, 2>, I, rel);
    case 3: return cudaLaunchKernelEx(&cfg, stage_kernel<R, true, 0>, I, rel);
    case 4: return cudaLaunchKernelEx(&cfg, stage_kernel<R, true, 1>, I, rel);
    case 5: return cudaLaunchKernelEx(&cfg, stage_kernel<R, true, 2>, I, rel);
    default: return cudaErrorInvalidValue;
    }
}

// Work item (instance, tile) x its `cluster` chunk CTAs: grid (nwork, cluster), with one thread-block
// cluster per work item in the cluster form and independent CTAs in the solo and split forms; the
// split form then launches the node step, grid (nwork, ceil(kTile / kNodePart)), node_smem bytes.
template <typename R>
cudaError_t launch_stage_batch(const Inst *insts, const int2 *work, int nwork, int cluster, size_t smem, int stage,
                               int rel, bool ext, int form, size_t node_smem, cudaStream_t st)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)nwork, (unsigned)cluster, 1);
    cfg.blockDim = dim3(kThreads, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = 1;
    at[0].val.clusterDim.y = (unsigned)cluster;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = form == kFormCluster ? 1 : 0;
    cudaError_t e = cudaErrorInvalidValue;
    switch (stage + 3 * ext + 6 * form) {
    case 0: e = cudaLaunchKernelEx(&cfg, stage_batch_kernel<R, false, 0, kFormCluster>, insts, work, rel); break;
    case 1: e = cudaLaunchKernelEx(&cfg, stage_batch_kernel<R, false, 1, kFormCluster>, insts, work, rel); break;
    case 2: e = cudaLaunchKernelEx(&cfg, stage_batch_kernel<R, false, 2, kFormCluster>, insts, work, rel); break;
    case 3: e = cudaLaunchKernelEx(&cfg, stage_batch_kernel<R, true, 0, kFormCluster>, insts, work, rel); break;
    case 4: e = cudaLaunchKernelEx(&cfg, stage_batch_kernel<R, true, 1, kFormCluster>, insts, work, rel); break;
    case 5: e = cudaLaunchKernelEx(&cfg, stage_batch_kernel<R, true, 2, kFormCluster>, insts, work, rel); break;
    case 6: e = cudaLaunchKernelEx(&cfg, stage_batch_kernel<R, false, 0, kFormSolo>, insts, work, rel); break;
    case 7: e = cudaLaunchKernelEx(&cfg, stage_batch_kernel<R, false, 1, kFormSolo>, insts, work, rel); break;
    case 8: e = cudaLaunchKernelEx(&cfg, stage_batch_kernel<R, false, 2, kFormSolo>, insts, work, rel); break;
    case 9: e = cudaLaunchKernelEx(&cfg, stage_batch_kernel<R, true, 0, kFormSolo>, insts, work, rel); break;
    case 10: e = cudaLaunchKernelEx(&cfg, stage_batch_kernel<R, true, 1, kFormSolo>, insts, work, rel); break;
    case 11: e = cudaLaunchKernelEx(&cfg, stage_batch_kernel<R, true, 2, kFormSolo>, insts, work, rel); break;
    case 12: e = cudaLaunchKernelEx(&cfg, stage_batch_kernel<R, false, 0, kFormSplit>, insts, work, rel); break;
    case 13: e = cudaLaunchKernelEx(&cfg, stage_batch_kernel<R, false, 1, kFormSplit>, insts, work, rel); break;
    case 14: e = cudaLaunchKernelEx(&cfg, stage_batch_kernel<R, false, 2, kFormSplit>, insts, work, rel); break;
    case 15: e = cudaLaunchKernelEx(&cfg, stage_batch_kernel<R, true, 0, kFormSplit>, insts, work, rel); break;
    case 16: e = cudaLaunchKernelEx(&cfg, stage_batch_kernel<R, true, 1, kFormSplit>, insts, work, rel); break;
    case 17: e = cudaLaunchKernelEx(&cfg, stage_batch_kernel<R, true, 2, kFormSplit>, insts, work, rel); break;
    default: break;
    }
    if (e != cudaSuccess || form != kFormSplit) return e;
    node_step_kernel<R><<<dim3((unsigned)nwork, (unsigned)((kTile + kNodePart - 1) / kNodePart), 1), kThreads, node_smem,
                          st>>>(insts, work, rel, stage);
    return cudaGetLastError();
}

// Persistent form: nsteps RK-3 steps of every work item in one cooperative launch of
// nclusters clusters of `cluster` CTAs (all resident), after zeroing the item counters
// (cnt: kPersistHdr + nwork + n) and the steps' residual slots.
template <typename R>
cudaError_t launch_persistent(const Inst *insts, const int2 *work, int nwork, int n, int cluster, int nclusters,
                              size_t smem, int nsteps, bool ext, unsigned *cnt, cudaStream_t st)
{
    cudaError_t e = cudaMemsetAsync(cnt, 0, (size_t)(kPersistHdr + nwork + n) * sizeof(unsigned), st);
    if (e != cudaSuccess) return e;
    zero_resid_kernel<<<std::min(n, 1024), 64, 0, st>>>(insts, n, nsteps);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)nclusters, (unsigned)cluster, 1);
    cfg.blockDim = dim3(kThreads, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[2];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = 1;
    at[0].val.clusterDim.y = (unsigned)cluster;
    at[0].val.clusterDim.z = 1;
    at[1].id = cudaLaunchAttributeCooperative;
    at[1].val.cooperative = 1;
    cfg.attrs = at;
    cfg.numAttrs = 2;
    if (ext) return cudaLaunchKernelEx(&cfg, persistent_stage_kernel<R, true>, insts, work, nwork, nsteps, cnt);
    return cudaLaunchKernelEx(&cfg, persistent_stage_kernel<R, false>, insts, work, nwork, nsteps, cnt);
}

// Clusters of the persistent kernel that can be resident at once.
template <typename R>
cudaError_t persistent_active_clusters(size_t smem, int cluster, int *nclusters)
{
    *nclusters = 0;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(1, cluster, 1);
    cfg.blockDim = dim3(kThreads, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = 1;
    at[0].val.clusterDim.y = (unsigned)cluster;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaOccupancyMaxActiveClusters(nclusters, persistent_stage_kernel<R, true>, &cfg);
}

template <typename R>
cudaError_t stage_active_clusters(size_t smem, int cluster, bool batch, bool solo, int *nclusters)
{
    *nclusters = 0;
    if (solo) {   // independent CTAs: the CTAs the device holds at once, in groups of `cluster`
        int dev = 0, nsm = 0, per_sm = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        if (e == cudaSuccess)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, stage_batch_kernel<R, false, 0, kFormSolo>, kThreads,
                                                              smem);
        if (e == cudaSuccess) *nclusters = per_sm * nsm / cluster;
        return e;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(1, cluster, 1);
    cfg.blockDim = dim3(kThreads, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = 1;
    at[0].val.clusterDim.y = (unsigned)cluster;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    // both forms of a kernel have the same launch bounds and shared memory: the plain one stands for both
    return batch ? cudaOccupancyMaxActiveClusters(nclusters, stage_batch_kernel<R, false, 0, kFormCluster>, &cfg)
                 : cudaOccupancyMaxActiveClusters(nclusters, stage_kernel<R, false, 0>, &cfg);
}

template <typename R>
cudaError_t launch_tile_equilibrium(const DevTables &T, const DevState &S, int buf, cudaStream_t st)
{
    tile_equilibrium_kernel<R><<<T.ntile, kThreads, EqScratch<R>(T.K, T.Nxe, T.Nye, T.Qx, T.Qy, T.tab_n).total, st>>>(T, S, buf);
    if (T.lts && buf == 0) mass_reference_kernel<<<1, kThreads, 0, st>>>(S.mass + kMassHdr, T.Nx, S.mass);
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
cudaError_t launch_moments_from_stage_data(const DevTables &T, const DevState &S, cudaStream_t st)
{
    moments_from_stage_data_kernel<R><<<(T.Nx + 127) / 128, 128, 0, st>>>(static_cast<const R *>(S.eqm[0]), T.Nx,
                                                                           T.Nxp, S.mom_out);
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_state_in(const double *src, void *dst, void *carry, const DevTables &T, int *bad, cudaStream_t st)
{
    const int grid = (int)std::min<size_t>(4096, (2 * (size_t)T.V * T.Nx + 255) / 256);
    state_in_kernel<R><<<grid, 256, 0, st>>>(src, static_cast<R *>(dst), static_cast<R *>(carry), T.frest, T.V,
                                             T.Nx, T.Nxp, bad);
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_state_out(const void *src, const void *carry, double *dst, const DevTables &T, cudaStream_t st)
{
    const int grid = (int)std::min<size_t>(4096, (2 * (size_t)T.V * T.Nx + 255) / 256);
    state_out_kernel<R><<<grid, 256, 0, st>>>(static_cast<const R *>(src), static_cast<const R *>(carry), dst,
                                              T.frest, T.V, T.Nx, T.Nxp);
    return cudaGetLastError();
}

const char *check_site_name(int site)
{
    static const char *const names[CK_COUNT] = {
        "none",
        "TMA box x coordinate off its 16-byte boundary",
        "bulk copy outside its shared-memory region or source array",
        "stencil, ghost or RK-base column outside the staged row box",
        "equilibrium factor index outside the tile's table",
        "state store outside [0, V) x [0, Nxp)",
        "symmetry-plane partner row outside the state",
        "cluster exchange slot outside the receiving CTA's region",
        "node-stage write outside the stage data or scratch capacity",
        "persistent item neighbour outside the work list or of another instance"};
    return site > 0 && site < CK_COUNT ? names[site] : "unknown site";
}

bool checked_build()
{
#ifdef LBC_CHECKED
    return true;
#else
    return false;
#endif
}

cudaError_t launch_ctl_bump(Ctl *ctl, int n, long long k, cudaStream_t st)
{
    ctl_bump_kernel<<<(n + 255) / 256, 256, 0, st>>>(ctl, n, k);
    return cudaGetLastError();
}

cudaError_t launch_last_residuals(const Inst *insts, const int *slots, int n, double *last, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    last_residuals_kernel<<<(n + 255) / 256, 256, 0, st>>>(insts, slots, n, last);
    return cudaGetLastError();
}

#define LBC_INSTANTIATE(R)                                                                                      \
    template size_t stage_smem_bytes<R>(int, int, int, int, int, int, int, int);                                     \
    template cudaError_t configure_kernels<R>();                                                                \
    template cudaError_t launch_stage<R>(const Inst &, size_t, int, int, cudaStream_t);                          \
    template cudaError_t launch_stage_batch<R>(const Inst *, const int2 *, int, int, size_t, int, int, bool, int,  \
                                               size_t, \
                                               cudaStream_t);                                                    \
    template cudaError_t launch_tile_equilibrium<R>(const DevTables &, const DevState &, int, cudaStream_t);     \
    template cudaError_t launch_moments_partial<R>(const DevTables &, const DevState &, int, cudaStream_t);      \
    template cudaError_t stage_active_clusters<R>(size_t, int, bool, bool, int *);                                    \
    template cudaError_t launch_persistent<R>(const Inst *, const int2 *, int, int, int, int, size_t, int, bool,     \
                                              unsigned *, cudaStream_t);                                          \
    template cudaError_t persistent_active_clusters<R>(size_t, int, int *);                                           \
    template size_t equilibrium_smem_bytes<R>(int, int, int, int, int, int);                                         \
    template cudaError_t launch_moments_from_stage_data<R>(const DevTables &, const DevState &, cudaStream_t);  \
    template cudaError_t launch_state_in<R>(const double *, void *, void *, const DevTables &, int *, cudaStream_t); \
    template cudaError_t launch_state_out<R>(const void *, const void *, double *, const DevTables &, cudaStream_t);
LBC_INSTANTIATE(float)
LBC_INSTANTIATE(double)

}  // namespace lbc
