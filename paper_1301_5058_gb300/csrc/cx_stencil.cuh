// cx_stencil.cuh -- the per-thread stencil machinery shared by the
// single-grid and batched step kernels: vector loads, the face fluxes of the
// scaled scheme, per-step noise, and the row march (see cx_step.cu).
#pragma once

#include "cx_internal.h"
#include "cx_philox.cuh"

namespace cx {
namespace stencil {


constexpr int kThreads = 128;  // 4 warps side by side along x
constexpr int kCells = 4;      // cells per thread along x
constexpr unsigned kFull = 0xffffffffu;

template <typename T> struct Vec;
template <> struct Vec<float> {
    // read-only path: for arrays no thread writes during the launch
    static __device__ __forceinline__ void load(const float *p, float (&v)[4])
    {
        const float4 q = __ldg(reinterpret_cast<const float4 *>(p));
        v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
    }
    // coherent path: for the array the Heun combine overwrites in place
    static __device__ __forceinline__ void load_rw(const float *p, float (&v)[4])
    {
        const float4 q = *reinterpret_cast<const float4 *>(p);
        v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
    }
    // L2 path (bypasses L1): for a persistent launch, where the arrays a
    // block reads were written by other blocks earlier in the same launch
    static __device__ __forceinline__ void load_cg(const float *p, float (&v)[4])
    {
        const float4 q = __ldcg(reinterpret_cast<const float4 *>(p));
        v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
    }
    static __device__ __forceinline__ void store(float *p, const float (&v)[4])
    {
        *reinterpret_cast<float4 *>(p) = make_float4(v[0], v[1], v[2], v[3]);
    }
};
template <> struct Vec<double> {
    static __device__ __forceinline__ void load(const double *p, double (&v)[4])
    {
        const double2 q0 = __ldg(reinterpret_cast<const double2 *>(p));
        const double2 q1 = __ldg(reinterpret_cast<const double2 *>(p) + 1);
        v[0] = q0.x; v[1] = q0.y; v[2] = q1.x; v[3] = q1.y;
    }
    static __device__ __forceinline__ void load_rw(const double *p, double (&v)[4])
    {
        const double2 q0 = reinterpret_cast<const double2 *>(p)[0];
        const double2 q1 = reinterpret_cast<const double2 *>(p)[1];
        v[0] = q0.x; v[1] = q0.y; v[2] = q1.x; v[3] = q1.y;
    }
    static __device__ __forceinline__ void load_cg(const double *p, double (&v)[4])
    {
        const double2 q0 = __ldcg(reinterpret_cast<const double2 *>(p));
        const double2 q1 = __ldcg(reinterpret_cast<const double2 *>(p) + 1);
        v[0] = q0.x; v[1] = q0.y; v[2] = q1.x; v[3] = q1.y;
    }
    static __device__ __forceinline__ void store(double *p, const double (&v)[4])
    {
        reinterpret_cast<double2 *>(p)[0] = make_double2(v[0], v[1]);
        reinterpret_cast<double2 *>(p)[1] = make_double2(v[2], v[3]);
    }
};

// ---------------------------------------------------------------------------
// Arithmetic with every rounding explicit, on one cell (float, double) or on
// a pair of cells (float2, double2).  The FP32 pair forms are Blackwell's
// paired FP32 instructions (one issue slot for two cells); each component
// rounds exactly as the scalar form, so a pair and two scalars give the same
// bits.  No operation is contracted by the compiler, so a face value or an
// update is the same bits in every kernel that evaluates it.

template <typename T> struct PairOf;
template <> struct PairOf<float> { using type = float2; };
template <> struct PairOf<double> { using type = double2; };
template <typename T> using P2 = typename PairOf<T>::type;

__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float2 add_rn(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ double2 add_rn(double2 a, double2 b)
{
    return make_double2(__dadd_rn(a.x, b.x), __dadd_rn(a.y, b.y));
}
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float2 mul_rn(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ double2 mul_rn(double2 a, double2 b)
{
    return make_double2(__dmul_rn(a.x, b.x), __dmul_rn(a.y, b.y));
}
__device__ __forceinline__ float fma_rn(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fma_rn(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float2 fma_rn(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ double2 fma_rn(double2 a, double2 b, double2 c)
{
    return make_double2(__fma_rn(a.x, b.x, c.x), __fma_rn(a.y, b.y, c.y));
}
// a - b; the pair form is fma(b, -1, a), which rounds the exact difference
// once, as the scalar subtraction does (m1 holds -1)
__device__ __forceinline__ float sub_rn(float a, float b, float) { return __fsub_rn(a, b); }
__device__ __forceinline__ double sub_rn(double a, double b, double) { return __dsub_rn(a, b); }
__device__ __forceinline__ float2 sub_rn(float2 a, float2 b, float2 m1) { return __ffma2_rn(b, m1, a); }
__device__ __forceinline__ double2 sub_rn(double2 a, double2 b, double2)
{
    return make_double2(__dsub_rn(a.x, b.x), __dsub_rn(a.y, b.y));
}
// c / q for the receptor-law weight (q = (2 + n_L + n_R)^2 >= 4).  FP32: the
// fast division (the FP32 path is judged by tolerance).  FP64: c times a
// reciprocal refined by Newton's method for 1/q, x <- x + x (1 - q x), whose
// relative error e becomes e^2 per step, from the hardware's approximate
// FP64 reciprocal (rcp.approx.ftz.f64; q is never subnormal).  Any seed within
// 2^-14 of 1/q is below FP64 rounding after the two steps (2^-28, then
// 2^-56), so the weight is within about one ulp of c / q; the seed needs no
// FP64 <-> FP32 conversions, which run on GB300's narrow FP64 pipe.
__device__ __forceinline__ float div_w(float c, float q) { return __fdividef(c, q); }
__device__ __forceinline__ double div_w(double c, double q)
{
    double x;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(x) : "d"(q));
    x = __fma_rn(x, __fma_rn(-q, x, 1.0), x);
    x = __fma_rn(x, __fma_rn(-q, x, 1.0), x);
    return __dmul_rn(c, x);
}
__device__ __forceinline__ float2 div_w(float2 c, float2 q)
{
    return make_float2(__fdividef(c.x, q.x), __fdividef(c.y, q.y));
}
__device__ __forceinline__ double2 div_w(double2 c, double2 q)
{
    return make_double2(div_w(c.x, q.x), div_w(c.y, q.y));
}
// donor-cell b: the side with the lower n (dn = nR - nL)
__device__ __forceinline__ float donor(float dn, float bL, float bR) { return dn >= 0.f ? bL : bR; }
__device__ __forceinline__ double donor(double dn, double bL, double bR) { return dn >= 0.0 ? bL : bR; }
__device__ __forceinline__ float2 donor(float2 dn, float2 bL, float2 bR)
{
    return make_float2(donor(dn.x, bL.x, bR.x), donor(dn.y, bL.y, bR.y));
}
__device__ __forceinline__ double2 donor(double2 dn, double2 bL, double2 bR)
{
    return make_double2(donor(dn.x, bL.x, bR.x), donor(dn.y, bL.y, bR.y));
}
__host__ __device__ __forceinline__ float2 pair(float x, float y) { return make_float2(x, y); }
__host__ __device__ __forceinline__ double2 pair(double x, double y) { return make_double2(x, y); }

// The scaled flux coefficients (dt folded in) as stored per grid.
template <typename T> struct CoefT {
    T cA, cChi, cG, cR, cN;
};

// The coefficients and constants of the face and update arithmetic, for
// one cell (V = T) or a pair (V = P2<T>): signs are folded in so that every
// subtraction of a product is one multiply-add.
template <typename V> struct KV {
    V cA;     // scale of the bacterial flux divergence
    V ncChi;  // -chi0 scale
    V cG;     // scale of the nutrient flux divergence
    V cR;     // growth
    V ncN;    // -consumption
    V two, four, m1, half;
};
template <typename T> __host__ __device__ __forceinline__ KV<P2<T>> make_kv(const CoefT<T> &k)
{
    KV<P2<T>> v;
    v.cA = pair(k.cA, k.cA);
    v.ncChi = pair(-k.cChi, -k.cChi);
    v.cG = pair(k.cG, k.cG);
    v.cR = pair(k.cR, k.cR);
    v.ncN = pair(-k.cN, -k.cN);
    v.two = pair(T(2), T(2));
    v.four = pair(T(4), T(4));
    v.m1 = pair(T(-1), T(-1));
    v.half = pair(T(0.5), T(0.5));
    return v;
}
template <typename T> __device__ __forceinline__ KV<T> scalar_kv(const KV<P2<T>> &k)
{
    return KV<T>{k.cA.x, k.ncChi.x, k.cG.x, k.cR.x, k.ncN.x, k.two.x, k.four.x, k.m1.x, k.half.x};
}

// Unscaled fluxes (phi, g) through the face between L (left/lower) and R,
// for one face or a pair of faces:
//   phi = s2 n2 b2 (db - hc b2 dn)          (central b^2 mobility)
//   phi = s2 n2 (b2 db - 4 hc bd^2 dn)       (donor-cell b^2)
//   g   = dn
// with s2 = sL + sR (likewise n2, b2), db = bR - bL, dn = nR - nL and
// hc = cChi / (2 + n2)^2 (receptor law) or cChi (constant chi).  The
// constant factors cA and cG are applied once per cell, to the divergence
// (cell_update), not once per face.
template <int LAW, int MOB, typename V>
__device__ __forceinline__ void face(V sL, V sR, V nL, V nR, V bL, V bR, const KV<V> &k, V &phi,
                                     V &g)
{
    const V s2 = add_rn(sL, sR), n2 = add_rn(nL, nR), b2 = add_rn(bL, bR);
    const V db = sub_rn(bR, bL, k.m1), dn = sub_rn(nR, nL, k.m1);
    V hcn = k.ncChi;  // -hc
    if (LAW == CX_CHEMO_RECEPTOR) {
        const V q = add_rn(n2, k.two);
        hcn = div_w(k.ncChi, mul_rn(q, q));
    }
    const V a = mul_rn(s2, n2);
    if (MOB == CX_MOBILITY_CENTRAL) {
        phi = mul_rn(mul_rn(a, b2), fma_rn(mul_rn(hcn, b2), dn, db));
    } else {
        const V bd = donor(dn, bL, bR);
        phi = mul_rn(a, fma_rn(mul_rn(mul_rn(mul_rn(k.four, hcn), bd), bd), dn, mul_rn(b2, db)));
    }
    g = dn;
}

// Four adjacent cells x0..x0+3 of one field, held as the pairs
// E = (x0, x0+2) and O = (x0+1, x0+3), so that the x-faces pair up too.
template <typename T> struct Cells {
    P2<T> E, O;
};
// A vector as loaded from (or stored to) a device array in pair order
// (cx_internal.h): (x0, x0+2, x0+1, x0+3), i.e. E then O.
template <typename T> __device__ __forceinline__ Cells<T> split4(const T (&v)[4])
{
    return Cells<T>{pair(v[0], v[1]), pair(v[2], v[3])};
}
template <typename T> __device__ __forceinline__ void join4(const Cells<T> &c, T (&v)[4])
{
    v[0] = c.E.x; v[1] = c.E.y; v[2] = c.O.x; v[3] = c.O.y;
}
// Four values in natural cell order x0 .. x0+3 (values made in registers,
// such as per-step sigma, and the element-wise edge stores).
template <typename T> __device__ __forceinline__ Cells<T> split4_nat(const T (&v)[4])
{
    return Cells<T>{pair(v[0], v[2]), pair(v[1], v[3])};
}
template <typename T> __device__ __forceinline__ void join4_nat(const Cells<T> &c, T (&v)[4])
{
    v[0] = c.E.x; v[1] = c.O.x; v[2] = c.E.y; v[3] = c.O.y;
}
template <typename T> __device__ __forceinline__ Cells<T> zero_cells()
{
    return Cells<T>{pair(T(0), T(0)), pair(T(0), T(0))};
}

// y-faces of four cells (between a row and the next one), as E / O pairs.
template <typename T> struct YFaces {
    P2<T> phE, phO, gE, gO;
};
template <typename T> __device__ __forceinline__ YFaces<T> zero_yfaces()
{
    const P2<T> z = pair(T(0), T(0));
    return YFaces<T>{z, z, z, z};
}
template <typename T, int LAW, int MOB>
__device__ __forceinline__ YFaces<T> row_yfaces(const Cells<T> &sL, const Cells<T> &nL,
                                                const Cells<T> &bL, const Cells<T> &sU,
                                                const Cells<T> &nU, const Cells<T> &bU,
                                                const KV<P2<T>> &k)
{
    YFaces<T> y;
    face<LAW, MOB>(sL.E, sU.E, nL.E, nU.E, bL.E, bU.E, k, y.phE, y.gE);
    face<LAW, MOB>(sL.O, sU.O, nL.O, nU.O, bL.O, bU.O, k, y.phO, y.gO);
    return y;
}

// x-faces of four cells: f_c lies between cells x0+c-1 and x0+c.  They are
// computed as A = (f0, f2), B = (f1, f3) and f4; (l*, r*) are the cells
// x0-1 and x0+4.  Faces on the walls (and past the row's end) carry zero
// flux unless INTERIOR (no wall within reach).
template <typename T> struct XFaces {
    P2<T> phA, gA, phB, gB;
    T ph4, g4;
};
template <typename T, int LAW, int MOB, bool INTERIOR>
__device__ __forceinline__ XFaces<T> row_xfaces(const Cells<T> &s, const Cells<T> &n,
                                                const Cells<T> &b, T ls, T ln, T lb, T rs, T rn,
                                                T rb, const KV<P2<T>> &k, int x0, int nx)
{
    XFaces<T> f;
    face<LAW, MOB>(pair(ls, s.O.x), s.E, pair(ln, n.O.x), n.E, pair(lb, b.O.x), b.E, k, f.phA, f.gA);
    face<LAW, MOB>(s.E, s.O, n.E, n.O, b.E, b.O, k, f.phB, f.gB);
    face<LAW, MOB>(s.O.y, rs, n.O.y, rn, b.O.y, rb, scalar_kv<T>(k), f.ph4, f.g4);
    if (!INTERIOR) {
        if (x0 == 0) f.phA.x = f.gA.x = T(0);           // west wall
        if (x0 + 1 >= nx) f.phB.x = f.gB.x = T(0);      // east wall and padding
        if (x0 + 2 >= nx) f.phA.y = f.gA.y = T(0);
        if (x0 + 3 >= nx) f.phB.y = f.gB.y = T(0);
        if (x0 + 4 >= nx) f.ph4 = f.g4 = T(0);
    }
    return f;
}

// The same x-faces when every lane of the warp holds the row's next four
// cells (the two-stage march): f4 is the right lane's f0, so each face is
// evaluated once and no right-hand neighbour is needed.  Lane 31 takes its
// own f0 for f4; the caller discards what depends on it.
template <typename T, int LAW, int MOB, bool INTERIOR>
__device__ __forceinline__ XFaces<T> row_xfaces_shfl(const Cells<T> &s, const Cells<T> &n,
                                                     const Cells<T> &b, T ls, T ln, T lb,
                                                     const KV<P2<T>> &k, int x0, int nx)
{
    XFaces<T> f;
    face<LAW, MOB>(pair(ls, s.O.x), s.E, pair(ln, n.O.x), n.E, pair(lb, b.O.x), b.E, k, f.phA, f.gA);
    face<LAW, MOB>(s.E, s.O, n.E, n.O, b.E, b.O, k, f.phB, f.gB);
    f.ph4 = __shfl_down_sync(kFull, f.phA.x, 1);
    f.g4 = __shfl_down_sync(kFull, f.gA.x, 1);
    if (!INTERIOR) {
        if (x0 == 0) f.phA.x = f.gA.x = T(0);           // west wall
        if (x0 + 1 >= nx) f.phB.x = f.gB.x = T(0);      // east wall and padding
        if (x0 + 2 >= nx) f.phA.y = f.gA.y = T(0);
        if (x0 + 3 >= nx) f.phB.y = f.gB.y = T(0);
        if (x0 + 4 >= nx) f.ph4 = f.g4 = T(0);
    }
    return f;
}

// u + reaction + div for one pair of cells: faces west/east and, in march
// order, behind/ahead (DIR +1: ahead is north):
//   b' = b + cR n b + cA div(phi),   n' = n - cN n b + cG div(g).
template <typename T, int DIR>
__device__ __forceinline__ void cell_update(P2<T> b, P2<T> n, P2<T> phW, P2<T> gW, P2<T> phE,
                                            P2<T> gE, P2<T> phB, P2<T> gB, P2<T> phA, P2<T> gA,
                                            const KV<P2<T>> &k, P2<T> &ob, P2<T> &on)
{
    const P2<T> phN = DIR > 0 ? phA : phB, phS = DIR > 0 ? phB : phA;
    const P2<T> gN = DIR > 0 ? gA : gB, gS = DIR > 0 ? gB : gA;
    const P2<T> r = mul_rn(n, b);
    const P2<T> divb = add_rn(sub_rn(phE, phW, k.m1), sub_rn(phN, phS, k.m1));
    const P2<T> divn = add_rn(sub_rn(gE, gW, k.m1), sub_rn(gN, gS, k.m1));
    ob = fma_rn(k.cA, divb, fma_rn(k.cR, r, b));
    on = fma_rn(k.cG, divn, fma_rn(k.ncN, r, n));
}
// the four cells: even cells lie between A (west) and B (east), odd cells
// between B and (f2, f4)
template <typename T, int DIR>
__device__ __forceinline__ void row_update(const Cells<T> &b, const Cells<T> &n,
                                           const XFaces<T> &x, const YFaces<T> &yB,
                                           const YFaces<T> &yA, const KV<P2<T>> &k, Cells<T> &ob,
                                           Cells<T> &on)
{
    cell_update<T, DIR>(b.E, n.E, x.phA, x.gA, x.phB, x.gB, yB.phE, yB.gE, yA.phE, yA.gE, k, ob.E,
                        on.E);
    cell_update<T, DIR>(b.O, n.O, x.phB, x.gB, pair(x.phA.y, x.ph4), pair(x.gA.y, x.g4), yB.phO,
                        yB.gO, yA.phO, yA.gO, k, ob.O, on.O);
}
// Heun's second stage: (u0 + u) / 2
template <typename T>
__device__ __forceinline__ Cells<T> heun_mean(const Cells<T> &u0, const Cells<T> &u,
                                              const KV<P2<T>> &k)
{
    return Cells<T>{mul_rn(k.half, add_rn(u0.E, u.E)), mul_rn(k.half, add_rn(u0.O, u.O))};
}

// Per-step noise: the sigma recipe of the state's precision.
template <typename T> struct NoiseT;
template <> struct NoiseT<float> {
    uint64_t seed, step;
    int dist;
    float sigma0, amp;
    uint32_t kx[10], ky[10];  // the key schedule of seed (set_keys)
    __host__ __device__ void set_keys()
    {
        uint32_t a = (uint32_t)seed, b = (uint32_t)(seed >> 32);
        for (int r = 0; r < 10; ++r) {
            kx[r] = a;
            ky[r] = b;
            a += 0x9E3779B9u;
            b += 0xBB67AE85u;
        }
    }
    __device__ __forceinline__ uint4 block(uint64_t q) const
    {
        return philox4x32_10_ks(
            make_uint4((uint32_t)q, (uint32_t)(q >> 32), (uint32_t)step, (uint32_t)(step >> 32)), kx,
            ky);
    }
    __device__ __forceinline__ float at(long long idx) const
    {
        const uint4 w = block((uint64_t)idx >> 2);
        return sigma_from_word(block_word(w, (int)(idx & 3)), dist, sigma0, amp);
    }
    // cells idx0 .. idx0+3: one Philox block when idx0 is a multiple of 4
    // (always, in rows whose width is), two otherwise (the offset is the same
    // for all threads of a row)
    __device__ __forceinline__ void four(long long idx0, float (&s)[4]) const
    {
        const uint64_t q = (uint64_t)idx0 >> 2;
        const int h = (int)(idx0 & 3);
        const uint4 w0 = block(q);
        if (h == 0) {
            s[0] = sigma_from_word(w0.x, dist, sigma0, amp);
            s[1] = sigma_from_word(w0.y, dist, sigma0, amp);
            s[2] = sigma_from_word(w0.z, dist, sigma0, amp);
            s[3] = sigma_from_word(w0.w, dist, sigma0, amp);
        } else {
            const uint4 w1 = block(q + 1);
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const int k = h + c;
                s[c] = sigma_from_word(k < 4 ? block_word(w0, k) : block_word(w1, k - 4), dist,
                                       sigma0, amp);
            }
        }
    }
};
template <> struct NoiseT<double> {
    uint64_t seed, step;
    int dist;
    double sigma0, amp;
    __device__ __forceinline__ double at(long long idx) const
    {
        return sigma_f64(seed, (uint64_t)idx, step, dist, sigma0, amp);
    }
    __device__ __forceinline__ void four(long long idx0, double (&s)[4]) const
    {
#pragma unroll
        for (int c = 0; c < 4; ++c) s[c] = at(idx0 + c);
    }
};

// Before a launch: the FP32 recipe's Philox key schedule from the seed (the
// FP64 recipe derives its keys as it goes).
inline void set_noise_keys(NoiseT<float> &nz) { nz.set_keys(); }
inline void set_noise_keys(NoiseT<double> &) {}

template <typename T> struct Ptrs {
    const T *__restrict__ b;
    const T *__restrict__ n;
    const T *__restrict__ s;
    const T *bu;  // may alias bo (in-place Heun combine)
    const T *nu;
    T *bo;
    T *no;
};

// Both marches ask L2, once per iteration, for the state row kPrefetchRows
// ahead of the one they load.  A loaded row feeds the iteration's whole
// dependence chain, so without the hint each iteration waits a full DRAM
// latency; with it the load finds the row in L2.  On the 16384^2 FP32
// workload, 1 to 3 rows ahead all gain about 18 % for the two-stage march
// (6 rows ahead gains less) and 5 % for the one-stage march.  Only rows the
// tile itself loads are asked for (a row past the tile's end would be read
// by the neighbouring tile, usually long after), at the thread's in-row
// vector offset `off` (row * pitch + in-row column).
constexpr int kPrefetchRows = 2;
template <typename T, int NOISE>
__device__ __forceinline__ void prefetch_row(const Ptrs<T> &P, long long off)
{
    asm volatile("prefetch.global.L2 [%0];" ::"l"(P.b + off));
    asm volatile("prefetch.global.L2 [%0];" ::"l"(P.n + off));
    if (NOISE == 0) asm volatile("prefetch.global.L2 [%0];" ::"l"(P.s + off));
}

template <typename T> struct Row {
    Cells<T> b, n, s;
    T hb, hn, hs;     // lane 0: cell x0-1; lane 31: cell x0+4
    Cells<T> ub, un;  // STAGE 1: the state at the start of the step
};

// One thread's march over rows j0..jend-1 in direction DIR (+1: increasing j,
// -1: decreasing j).  The y-faces shared with the row processed before
// ("behind") are carried in registers; the y-faces with the next row in
// march order ("ahead") are computed from the row loaded in this iteration.
// Face values do not depend on DIR (a face is always evaluated with L the
// lower row), so both directions give bit-identical results.  CG: read
// through L2 only (a persistent launch whose blocks read what other blocks
// wrote earlier in the same launch).  INTERIOR: the caller guarantees that
// every thread's cells and both x-neighbours of the warp lie inside the grid
// (0 < x0 and x0 + 4 < nx for all threads), so the x-wall tests drop out.
template <typename T, int LAW, int MOB, int NOISE, int STAGE, int DIR, bool CG = false,
          bool INTERIOR = false>
__device__ __forceinline__ void march(const Ptrs<T> &P, int nx, int ny, long long pitch,
                                      const KV<P2<T>> &k, const NoiseT<T> &nz, int x0, int j0,
                                      int jend)
{
    const int lane = threadIdx.x & 31;
    // threads past the right edge keep running (they take part in the
    // shuffles) but load an in-row vector and store nothing
    const long long xv = INTERIOR ? (long long)x0 : min((long long)x0, pitch - kCells);
    const bool halo_l = (lane == 0) && (INTERIOR || ((x0 > 0) && (x0 < nx)));
    const bool halo_r = (lane == 31) && (INTERIOR || (x0 + kCells < nx));
    const bool halo = halo_l || halo_r;
    const long long xh = halo_l ? (long long)x0 - 1 : (long long)x0 + kCells;

    auto vload = [](const T *p) -> Cells<T> {
        T v[kCells];
        if (CG) Vec<T>::load_cg(p, v);
        else Vec<T>::load(p, v);
        return split4(v);
    };
    auto sload = [](const T *p) -> T { return CG ? __ldcg(p) : __ldg(p); };
    auto load_row = [&](int r, Row<T> &R, bool own) {
        const long long off = (long long)r * pitch;
        R.b = vload(P.b + off + xv);
        R.n = vload(P.n + off + xv);
        if (NOISE == 0) {
            R.s = vload(P.s + off + xv);
        } else {
            T v[kCells];
            nz.four((long long)r * nx + x0, v);
            if (!INTERIOR) {
#pragma unroll
                for (int c = 0; c < kCells; ++c)
                    if (x0 + c >= nx) v[c] = T(0);  // past the row's end
            }
            R.s = split4_nat(v);
        }
        R.hb = R.hn = R.hs = T(0);
        if (halo) {
            R.hb = sload(P.b + off + xh);
            R.hn = sload(P.n + off + xh);
            R.hs = NOISE == 0 ? sload(P.s + off + xh) : nz.at((long long)r * nx + xh);
        }
        if (STAGE == 1 && own) {
            T v[kCells];
            if (CG) Vec<T>::load_cg(P.bu + off + xv, v);
            else Vec<T>::load_rw(P.bu + off + xv, v);
            R.ub = split4(v);
            if (CG) Vec<T>::load_cg(P.nu + off + xv, v);
            else Vec<T>::load_rw(P.nu + off + xv, v);
            R.un = split4(v);
        }
    };
    // y-faces between a lower row lo and an upper row hi
    auto yfaces = [&](const Row<T> &lo, const Row<T> &hi) {
        return row_yfaces<T, LAW, MOB>(lo.s, lo.n, lo.b, hi.s, hi.n, hi.b, k);
    };

    const int jfirst = DIR > 0 ? j0 : jend - 1;
    const int jbehind = jfirst - DIR;
    Row<T> cur, nxt;
    YFaces<T> yB;
    load_row(jfirst, cur, true);
    if (jbehind >= 0 && jbehind < ny) {
        Row<T> prv;
        load_row(jbehind, prv, false);
        yB = DIR > 0 ? yfaces(prv, cur) : yfaces(cur, prv);
    } else {
        yB = zero_yfaces<T>();  // wall behind
    }

    // the last row this tile loads, in march order (the row beyond its last
    // written row, or the grid's edge)
    const int plast = DIR > 0 ? min(jend, ny - 1) : max(j0 - 1, 0);
    const int rows = jend - j0;
    for (int it = 0; it < rows; ++it) {
        const int j = jfirst + DIR * it;
        const int ja = j + DIR;
        const bool has_a = (ja >= 0 && ja < ny);  // uniform across the block
        {
            const int jp = ja + DIR * kPrefetchRows;
            if (DIR > 0 ? jp <= plast : jp >= plast)
                prefetch_row<T, NOISE>(P, (long long)jp * pitch + xv);
        }
        if (has_a) load_row(ja, nxt, it + 1 < rows);

        // x-neighbours of this thread's 4 cells
        T lb = __shfl_up_sync(kFull, cur.b.O.y, 1);
        T ln = __shfl_up_sync(kFull, cur.n.O.y, 1);
        T ls = __shfl_up_sync(kFull, cur.s.O.y, 1);
        T rb = __shfl_down_sync(kFull, cur.b.E.x, 1);
        T rn = __shfl_down_sync(kFull, cur.n.E.x, 1);
        T rs = __shfl_down_sync(kFull, cur.s.E.x, 1);
        if (lane == 0) { lb = cur.hb; ln = cur.hn; ls = cur.hs; }
        if (lane == 31) { rb = cur.hb; rn = cur.hn; rs = cur.hs; }
        const XFaces<T> xf =
            row_xfaces<T, LAW, MOB, INTERIOR>(cur.s, cur.n, cur.b, ls, ln, lb, rs, rn, rb, k, x0, nx);

        // y-faces with the row ahead (a wall past the grid's first/last row)
        YFaces<T> yA;
        if (has_a) yA = DIR > 0 ? yfaces(cur, nxt) : yfaces(nxt, cur);
        else yA = zero_yfaces<T>();

        Cells<T> ob, on;
        row_update<T, DIR>(cur.b, cur.n, xf, yB, yA, k, ob, on);
        if (STAGE == 1) {
            ob = heun_mean(cur.ub, ob, k);
            on = heun_mean(cur.un, on, k);
        }
        T vb[kCells], vn[kCells];
        const long long off = (long long)j * pitch;
        if (INTERIOR || x0 + kCells <= nx) {
            join4(ob, vb);
            join4(on, vn);
            Vec<T>::store(P.bo + off + x0, vb);
            Vec<T>::store(P.no + off + x0, vn);
        } else {
            // the row's last group: cell x0 + c lives at column x0 + pair_col(c)
            join4_nat(ob, vb);
            join4_nat(on, vn);
#pragma unroll
            for (int c = 0; c < kCells; ++c)
                if (x0 + c < nx) {
                    P.bo[off + x0 + pair_col(c)] = vb[c];
                    P.no[off + x0 + pair_col(c)] = vn[c];
                }
        }

        cur = nxt;
        yB = yA;
    }
}


}  // namespace stencil
}  // namespace cx
