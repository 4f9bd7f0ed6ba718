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

// c / q for the receptor-law weight; FP32 uses the fast reciprocal (the FP32
// path is judged by tolerance), FP64 the IEEE division.
__device__ __forceinline__ float div_w(float c, float q) { return __fdividef(c, q); }
__device__ __forceinline__ double div_w(double c, double q) { return c / q; }

// The last product of a face flux is rounded on its own (never contracted
// into the additions of the divergence), so a face value does not depend on
// the code around it and every kernel that evaluates a face gets the same bits.
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }

template <typename T> struct CoefT {
    T cA, cChi, cG, cR, cN;
};

// Per-step noise: the sigma recipe of the state's precision.
template <typename T> struct NoiseT;
template <> struct NoiseT<float> {
    uint64_t seed, step;
    int dist;
    float sigma0, amp;
    __device__ __forceinline__ float at(long long idx) const
    {
        return sigma_f32(seed, (uint64_t)idx, step, dist, sigma0, amp);
    }
    // cells idx0 .. idx0+3: two Philox blocks when idx0 is even, three when
    // it is odd (the parity is the same for all threads of a row)
    __device__ __forceinline__ void four(long long idx0, float (&s)[4]) const
    {
        const uint64_t q = (uint64_t)idx0 >> 1;
        if ((idx0 & 1) == 0) {
            sigma_pair_f32(seed, q, step, dist, sigma0, amp, s[0], s[1]);
            sigma_pair_f32(seed, q + 1, step, dist, sigma0, amp, s[2], s[3]);
        } else {
            float unused0, unused1;
            sigma_pair_f32(seed, q, step, dist, sigma0, amp, unused0, s[0]);
            sigma_pair_f32(seed, q + 1, step, dist, sigma0, amp, s[1], s[2]);
            sigma_pair_f32(seed, q + 2, step, dist, sigma0, amp, s[3], unused1);
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

// Scaled fluxes (phi, g) through the face between L (left/lower) and R.
template <typename T, int LAW, int MOB>
__device__ __forceinline__ void face(T sL, T sR, T nL, T nR, T bL, T bR, const CoefT<T> &k,
                                     T &phi, T &g)
{
    const T s2 = sL + sR, n2 = nL + nR, b2 = bL + bR;
    const T db = bR - bL, dn = nR - nL;
    T hc = k.cChi;  // chi(n_f) / 2
    if (LAW == CX_CHEMO_RECEPTOR) {
        const T q = T(2) + n2;
        hc = div_w(k.cChi, q * q);
    }
    const T a = k.cA * s2 * n2;
    if (MOB == CX_MOBILITY_CENTRAL) {
        phi = mul_rn(a * b2, db - hc * b2 * dn);
    } else {
        const T bd = (dn >= T(0)) ? bL : bR;  // donor: the lower-n side
        phi = mul_rn(a, b2 * db - T(4) * hc * bd * bd * dn);
    }
    g = mul_rn(k.cG, dn);
}

template <typename T> struct Row {
    T b[kCells], n[kCells], s[kCells];
    T hb, hn, hs;              // lane 0: cell x0-1; lane 31: cell x0+4
    T ub[kCells], un[kCells];  // STAGE 1: the state at the start of the step
};

template <typename T> struct Ptrs {
    const T *__restrict__ b;
    const T *__restrict__ n;
    const T *__restrict__ s;
    const T *bu;  // may alias bo (in-place Heun combine)
    const T *nu;
    T *bo;
    T *no;
};

// One thread's march over rows j0..jend-1 in direction DIR (+1: increasing j,
// -1: decreasing j).  The y-face shared with the row processed before
// ("behind") is carried in registers; the y-face with the next row in march
// order ("ahead") is computed from the row loaded in this iteration.  Face
// values do not depend on DIR (a face is always evaluated with L the lower
// row), so both directions give bit-identical results.  CG: read through L2
// only (a persistent launch whose blocks read what other blocks wrote
// earlier in the same launch).  INTERIOR: the caller guarantees that every
// thread's cells and both x-neighbours of the warp lie inside the grid
// (0 < x0 and x0 + 4 < nx for all threads), so the x-wall tests drop out.
template <typename T, int LAW, int MOB, int NOISE, int STAGE, int DIR, bool CG = false,
          bool INTERIOR = false>
__device__ __forceinline__ void march(const Ptrs<T> &P, int nx, int ny, long long pitch,
                                      const CoefT<T> &k, const NoiseT<T> &nz, int x0, int j0,
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

    auto vload = [](const T *p, T (&v)[kCells]) {
        if (CG) Vec<T>::load_cg(p, v);
        else Vec<T>::load(p, v);
    };
    auto sload = [](const T *p) -> T { return CG ? __ldcg(p) : __ldg(p); };
    auto load_row = [&](int r, Row<T> &R, bool own) {
        const long long off = (long long)r * pitch;
        vload(P.b + off + xv, R.b);
        vload(P.n + off + xv, R.n);
        if (NOISE == 0) {
            vload(P.s + off + xv, R.s);
        } else {
            nz.four((long long)r * nx + x0, R.s);
            if (!INTERIOR) {
#pragma unroll
                for (int c = 0; c < kCells; ++c)
                    if (x0 + c >= nx) R.s[c] = T(0);  // past the row's end
            }
        }
        R.hb = R.hn = R.hs = T(0);
        if (halo) {
            R.hb = sload(P.b + off + xh);
            R.hn = sload(P.n + off + xh);
            R.hs = NOISE == 0 ? sload(P.s + off + xh) : nz.at((long long)r * nx + xh);
        }
        if (STAGE == 1 && own) {
            if (CG) {
                Vec<T>::load_cg(P.bu + off + xv, R.ub);
                Vec<T>::load_cg(P.nu + off + xv, R.un);
            } else {
                Vec<T>::load_rw(P.bu + off + xv, R.ub);
                Vec<T>::load_rw(P.nu + off + xv, R.un);
            }
        }
    };
    // y-face between a lower row lo and an upper row hi
    auto yface = [&](const Row<T> &lo, const Row<T> &hi, T (&ph)[kCells], T (&g)[kCells]) {
#pragma unroll
        for (int c = 0; c < kCells; ++c)
            face<T, LAW, MOB>(lo.s[c], hi.s[c], lo.n[c], hi.n[c], lo.b[c], hi.b[c], k, ph[c], g[c]);
    };

    const int jfirst = DIR > 0 ? j0 : jend - 1;
    const int jbehind = jfirst - DIR;
    Row<T> cur, nxt;
    T phB[kCells], gB[kCells];
    load_row(jfirst, cur, true);
    if (jbehind >= 0 && jbehind < ny) {
        Row<T> prv;
        load_row(jbehind, prv, false);
        if (DIR > 0) yface(prv, cur, phB, gB);
        else yface(cur, prv, phB, gB);
    } else {
#pragma unroll
        for (int c = 0; c < kCells; ++c) phB[c] = gB[c] = T(0);  // wall behind
    }

    const int rows = jend - j0;
    for (int it = 0; it < rows; ++it) {
        const int j = jfirst + DIR * it;
        const int ja = j + DIR;
        const bool has_a = (ja >= 0 && ja < ny);  // uniform across the block
        if (has_a) load_row(ja, nxt, it + 1 < rows);

        // x-neighbours of this thread's 4 cells
        T lb = __shfl_up_sync(kFull, cur.b[kCells - 1], 1);
        T ln = __shfl_up_sync(kFull, cur.n[kCells - 1], 1);
        T ls = __shfl_up_sync(kFull, cur.s[kCells - 1], 1);
        T rb = __shfl_down_sync(kFull, cur.b[0], 1);
        T rn = __shfl_down_sync(kFull, cur.n[0], 1);
        T rs = __shfl_down_sync(kFull, cur.s[0], 1);
        if (lane == 0) { lb = cur.hb; ln = cur.hn; ls = cur.hs; }
        if (lane == 31) { rb = cur.hb; rn = cur.hn; rs = cur.hs; }

        // x-faces: f[c] lies between cells x0+c-1 and x0+c
        T phX[kCells + 1], gX[kCells + 1];
        face<T, LAW, MOB>(ls, cur.s[0], ln, cur.n[0], lb, cur.b[0], k, phX[0], gX[0]);
#pragma unroll
        for (int c = 1; c < kCells; ++c)
            face<T, LAW, MOB>(cur.s[c - 1], cur.s[c], cur.n[c - 1], cur.n[c], cur.b[c - 1],
                              cur.b[c], k, phX[c], gX[c]);
        face<T, LAW, MOB>(cur.s[kCells - 1], rs, cur.n[kCells - 1], rn, cur.b[kCells - 1], rb, k,
                          phX[kCells], gX[kCells]);
        if (!INTERIOR) {
            if (x0 == 0) phX[0] = gX[0] = T(0);  // west wall
#pragma unroll
            for (int c = 1; c <= kCells; ++c)
                if (x0 + c >= nx) phX[c] = gX[c] = T(0);  // east wall (and padding)
        }

        // y-face with the row ahead (a wall past the grid's first/last row)
        T phA[kCells], gA[kCells];
        if (has_a) {
            if (DIR > 0) yface(cur, nxt, phA, gA);
            else yface(nxt, cur, phA, gA);
        } else {
#pragma unroll
            for (int c = 0; c < kCells; ++c) phA[c] = gA[c] = T(0);
        }

        T ob[kCells], on[kCells];
#pragma unroll
        for (int c = 0; c < kCells; ++c) {
            const T phN = DIR > 0 ? phA[c] : phB[c], phS = DIR > 0 ? phB[c] : phA[c];
            const T gN = DIR > 0 ? gA[c] : gB[c], gS = DIR > 0 ? gB[c] : gA[c];
            const T r = cur.n[c] * cur.b[c];
            const T divb = (phX[c + 1] - phX[c]) + (phN - phS);
            const T divn = (gX[c + 1] - gX[c]) + (gN - gS);
            ob[c] = (cur.b[c] + divb) + k.cR * r;
            on[c] = (cur.n[c] + divn) - k.cN * r;
            if (STAGE == 1) {
                ob[c] = T(0.5) * (cur.ub[c] + ob[c]);
                on[c] = T(0.5) * (cur.un[c] + on[c]);
            }
        }
        const long long off = (long long)j * pitch;
        if (INTERIOR || x0 + kCells <= nx) {
            Vec<T>::store(P.bo + off + x0, ob);
            Vec<T>::store(P.no + off + x0, on);
        } else {
#pragma unroll
            for (int c = 0; c < kCells; ++c)
                if (x0 + c < nx) {
                    P.bo[off + x0 + c] = ob[c];
                    P.no[off + x0 + c] = on[c];
                }
        }

        cur = nxt;
#pragma unroll
        for (int c = 0; c < kCells; ++c) { phB[c] = phA[c]; gB[c] = gA[c]; }
    }
}


}  // namespace stencil
}  // namespace cx
