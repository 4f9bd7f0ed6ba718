// cx_step.cu -- one fused forward-Euler step of the bacteria/nutrient system
// (Eq. ka-chem-model in the general form of Eq. ka-model-dim, chemotactic
// flux of Eq. chemflux, no-flux walls of Eq. bconds).
//
// One pass per step reads b, n, sigma and writes b', n'
// (20 B per cell in FP32, 40 B in FP64).  Each thread owns 4 adjacent cells
// of a row (one 16-byte vector per FP32 field) and marches down kRows rows,
// keeping the row below in registers, so every cell is loaded from HBM once
// and every y-face flux is evaluated once and reused by the two cells that
// share it.  x-neighbours come from the adjacent lanes by warp shuffles;
// lanes 0 and 31 fetch the one cell beyond the warp.  Boundary faces carry
// zero flux.
#include "cx_internal.h"

namespace cx {
namespace {

constexpr int kThreads = 128;  // 4 warps side by side along x
constexpr int kCells = 4;      // cells per thread along x
constexpr int kRows = 32;      // rows per block along y
constexpr unsigned kFull = 0xffffffffu;

template <typename T> struct Vec;
template <> struct Vec<float> {
    static __device__ __forceinline__ void load(const float *p, float (&v)[4])
    {
        const float4 q = __ldg(reinterpret_cast<const float4 *>(p));
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

template <typename T> struct CoefT {
    T cA, cChi, cG, cR, cN;
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
        phi = a * b2 * (db - hc * b2 * dn);
    } else {
        const T bd = (dn >= T(0)) ? bL : bR;  // donor: the lower-n side
        phi = a * (b2 * db - T(4) * hc * bd * bd * dn);
    }
    g = k.cG * dn;
}

template <typename T> struct Row {
    T b[kCells], n[kCells], s[kCells];
    T hb, hn, hs;  // lane 0: cell x0-1; lane 31: cell x0+4
};

template <typename T, int LAW, int MOB>
__global__ void __launch_bounds__(kThreads)
    step_kernel(const T *__restrict__ b, const T *__restrict__ n, const T *__restrict__ s,
                T *__restrict__ bo, T *__restrict__ no, int nx, int ny, long long pitch,
                CoefT<T> k)
{
    const int lane = threadIdx.x & 31;
    const int x0 = (blockIdx.x * kThreads + threadIdx.x) * kCells;
    const int j0 = blockIdx.y * kRows;
    const int jend = min(j0 + kRows, ny);
    // threads past the right edge keep running (they take part in the
    // shuffles) but load an in-row vector and store nothing
    const long long xv = min((long long)x0, pitch - kCells);
    const bool halo_l = (lane == 0) && (x0 > 0) && (x0 < nx);
    const bool halo_r = (lane == 31) && (x0 + kCells < nx);
    const bool halo = halo_l || halo_r;
    const long long xh = halo_l ? (long long)x0 - 1 : (long long)x0 + kCells;

    auto load_row = [&](int r, Row<T> &R) {
        const long long off = (long long)r * pitch;
        Vec<T>::load(b + off + xv, R.b);
        Vec<T>::load(n + off + xv, R.n);
        Vec<T>::load(s + off + xv, R.s);
        R.hb = R.hn = R.hs = T(0);
        if (halo) {
            R.hb = __ldg(b + off + xh);
            R.hn = __ldg(n + off + xh);
            R.hs = __ldg(s + off + xh);
        }
    };

    Row<T> cur, nxt;
    T phiS[kCells], gS[kCells];
    load_row(j0, cur);
    if (j0 > 0) {
        Row<T> prv;
        load_row(j0 - 1, prv);
#pragma unroll
        for (int c = 0; c < kCells; ++c)
            face<T, LAW, MOB>(prv.s[c], cur.s[c], prv.n[c], cur.n[c], prv.b[c], cur.b[c], k,
                              phiS[c], gS[c]);
    } else {
#pragma unroll
        for (int c = 0; c < kCells; ++c) phiS[c] = gS[c] = T(0);
    }

    for (int j = j0; j < jend; ++j) {
        const bool has_up = (j + 1 < ny);  // uniform across the block
        if (has_up) load_row(j + 1, nxt);

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
        if (x0 == 0) phX[0] = gX[0] = T(0);  // west wall
#pragma unroll
        for (int c = 1; c <= kCells; ++c)
            if (x0 + c >= nx) phX[c] = gX[c] = T(0);  // east wall (and padding)

        // y-faces between this row and the next
        T phiN[kCells], gN[kCells];
#pragma unroll
        for (int c = 0; c < kCells; ++c) {
            if (has_up)
                face<T, LAW, MOB>(cur.s[c], nxt.s[c], cur.n[c], nxt.n[c], cur.b[c], nxt.b[c], k,
                                  phiN[c], gN[c]);
            else
                phiN[c] = gN[c] = T(0);  // north wall
        }

        T ob[kCells], on[kCells];
#pragma unroll
        for (int c = 0; c < kCells; ++c) {
            const T r = cur.n[c] * cur.b[c];
            const T divb = (phX[c + 1] - phX[c]) + (phiN[c] - phiS[c]);
            const T divn = (gX[c + 1] - gX[c]) + (gN[c] - gS[c]);
            ob[c] = (cur.b[c] + divb) + k.cR * r;
            on[c] = (cur.n[c] + divn) - k.cN * r;
        }
        const long long off = (long long)j * pitch;
        if (x0 + kCells <= nx) {
            Vec<T>::store(bo + off + x0, ob);
            Vec<T>::store(no + off + x0, on);
        } else {
#pragma unroll
            for (int c = 0; c < kCells; ++c)
                if (x0 + c < nx) {
                    bo[off + x0 + c] = ob[c];
                    no[off + x0 + c] = on[c];
                }
        }

        cur = nxt;
#pragma unroll
        for (int c = 0; c < kCells; ++c) { phiS[c] = phiN[c]; gS[c] = gN[c]; }
    }
}

template <typename T, int LAW, int MOB>
cudaError_t launch_t(const StepArgs &a, cudaStream_t st)
{
    const CoefT<T> k{(T)a.k.cA, (T)a.k.cChi, (T)a.k.cG, (T)a.k.cR, (T)a.k.cN};
    const dim3 grid((a.nx + kThreads * kCells - 1) / (kThreads * kCells),
                    (a.ny + kRows - 1) / kRows);
    step_kernel<T, LAW, MOB><<<grid, kThreads, 0, st>>>(
        (const T *)a.b, (const T *)a.n, (const T *)a.s, (T *)a.bo, (T *)a.no, a.nx, a.ny, a.pitch,
        k);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_prec(const StepArgs &a, cudaStream_t st)
{
    if (a.law == CX_CHEMO_RECEPTOR)
        return a.mob == CX_MOBILITY_CENTRAL ? launch_t<T, CX_CHEMO_RECEPTOR, CX_MOBILITY_CENTRAL>(a, st)
                                            : launch_t<T, CX_CHEMO_RECEPTOR, CX_MOBILITY_UPWIND>(a, st);
    return a.mob == CX_MOBILITY_CENTRAL ? launch_t<T, CX_CHEMO_CONSTANT, CX_MOBILITY_CENTRAL>(a, st)
                                        : launch_t<T, CX_CHEMO_CONSTANT, CX_MOBILITY_UPWIND>(a, st);
}

}  // namespace

cudaError_t launch_step(int prec, const StepArgs &a, cudaStream_t st)
{
    return prec == CX_PREC_F64 ? launch_prec<double>(a, st) : launch_prec<float>(a, st);
}

}  // namespace cx
