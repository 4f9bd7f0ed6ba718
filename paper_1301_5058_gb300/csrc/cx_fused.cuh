// cx_fused.cuh -- the two-stage row march: one pass over the grid takes two
// explicit stages of Eq. ka-chem-model, keeping the intermediate state in
// registers (temporal blocking of depth 2).  With forward Euler the stages
// are two time steps; with Heun's scheme they are the two stages of one
// step (second-order Runge-Kutta, Sec. 3), sigma shared by both.
//
// Geometry.  A warp's 32 lanes hold 128 consecutive columns (4 per lane) and
// write the 120 held by lanes 1..30; lanes 0 and 31 hold the columns beside
// them, so the first stage is known one cell beyond the written range and
// no lane loads a halo cell of its own.  The end lanes take their own
// values for the neighbour they lack; that spoils only their outermost
// first-stage cells, which no written cell depends on.  Along y the march
// visits the state rows j0-2 .. jend+1 of a tile: the first stage lags one
// row behind the loads and the second stage two rows, so every state row is
// loaded once per tile and every y-face of either stage is evaluated once.
//
// Each stage evaluates exactly the operations of the single-stage march
// (cx_stencil.cuh) on the same operands, so a fused pass is bit for bit the
// two passes it replaces.
#pragma once

#include "cx_stencil.cuh"

namespace cx {
namespace stencil {

constexpr int kFusedCols = (32 - 2) * kCells;                  // written columns per warp
constexpr int kFusedBlockCols = (kThreads / 32) * kFusedCols;  // written columns per block

// One thread's two-stage march over the written rows j0..jend-1 in direction
// DIR.  x0: the thread's first column (may be negative or past the grid for
// the end lanes).  nz1 / nz2: the per-step noise of the first and second
// stage (NOISE 1; nz2 = nz1 under Heun).  INTERIOR: every column the warp
// holds lies inside the grid, x0 >= 0 and x0 + 4 <= nx for all threads.
template <typename T, int LAW, int MOB, int NOISE, bool HEUN, int DIR, bool INTERIOR>
__device__ __forceinline__ void march2(const Ptrs<T> &P, int nx, int ny, long long pitch,
                                       const CoefT<T> &k, const NoiseT<T> &nz1,
                                       const NoiseT<T> &nz2, int x0, int j0, int jend)
{
    // the second stage sees the first stage's sigma: static field, or Heun
    constexpr bool kSameSigma = (NOISE == 0) || HEUN;
    const int lane = threadIdx.x & 31;
    const long long xv =
        INTERIOR ? (long long)x0 : min(max((long long)x0, 0LL), pitch - (long long)kCells);
    const bool writer = lane != 0 && lane != 31;

    auto gen_sigma = [&](const NoiseT<T> &nz, int r, T (&s)[kCells]) {
        nz.four((long long)r * nx + x0, s);
        if (!INTERIOR) {
#pragma unroll
            for (int c = 0; c < kCells; ++c)
                if (x0 + c < 0 || x0 + c >= nx) s[c] = T(0);  // outside the row
        }
    };
    auto load0 = [&](int r, T (&b)[kCells], T (&n)[kCells], T (&s)[kCells]) {
        const long long off = (long long)r * pitch + xv;
        Vec<T>::load(P.b + off, b);
        Vec<T>::load(P.n + off, n);
        if (NOISE == 0) Vec<T>::load(P.s + off, s);
        else gen_sigma(nz1, r, s);
    };
    // x-faces of one row: f[c] between cells x0+c-1 and x0+c
    auto xfaces = [&](const T (&s)[kCells], const T (&n)[kCells], const T (&b)[kCells], T ls,
                      T rs, T (&ph)[kCells + 1], T (&g)[kCells + 1]) {
        const T lb = __shfl_up_sync(kFull, b[kCells - 1], 1);
        const T ln = __shfl_up_sync(kFull, n[kCells - 1], 1);
        const T rb = __shfl_down_sync(kFull, b[0], 1);
        const T rn = __shfl_down_sync(kFull, n[0], 1);
        face<T, LAW, MOB>(ls, s[0], ln, n[0], lb, b[0], k, ph[0], g[0]);
#pragma unroll
        for (int c = 1; c < kCells; ++c)
            face<T, LAW, MOB>(s[c - 1], s[c], n[c - 1], n[c], b[c - 1], b[c], k, ph[c], g[c]);
        face<T, LAW, MOB>(s[kCells - 1], rs, n[kCells - 1], rn, b[kCells - 1], rb, k,
                          ph[kCells], g[kCells]);
        if (!INTERIOR) {
            if (x0 == 0) ph[0] = g[0] = T(0);  // west wall
#pragma unroll
            for (int c = 1; c <= kCells; ++c)
                if (x0 + c >= nx) ph[c] = g[c] = T(0);  // east wall (and padding)
        }
    };
    // y-face between the lower row (sL, nL, bL) and the upper row
    auto yface = [&](const T (&sL)[kCells], const T (&nL)[kCells], const T (&bL)[kCells],
                     const T (&sU)[kCells], const T (&nU)[kCells], const T (&bU)[kCells],
                     T (&ph)[kCells], T (&g)[kCells]) {
#pragma unroll
        for (int c = 0; c < kCells; ++c)
            face<T, LAW, MOB>(sL[c], sU[c], nL[c], nU[c], bL[c], bU[c], k, ph[c], g[c]);
    };
    // u + (divergence) + reaction; faces behind / ahead in march order
    auto update = [&](const T (&b)[kCells], const T (&n)[kCells], const T (&phX)[kCells + 1],
                      const T (&gX)[kCells + 1], const T (&phB)[kCells], const T (&gB)[kCells],
                      const T (&phA)[kCells], const T (&gA)[kCells], T (&ob)[kCells],
                      T (&on)[kCells]) {
#pragma unroll
        for (int c = 0; c < kCells; ++c) {
            const T phN = DIR > 0 ? phA[c] : phB[c], phS = DIR > 0 ? phB[c] : phA[c];
            const T gN = DIR > 0 ? gA[c] : gB[c], gS = DIR > 0 ? gB[c] : gA[c];
            const T r = n[c] * b[c];
            const T divb = (phX[c + 1] - phX[c]) + (phN - phS);
            const T divn = (gX[c + 1] - gX[c]) + (gN - gS);
            ob[c] = (b[c] + divb) + k.cR * r;
            on[c] = (n[c] + divn) - k.cN * r;
        }
    };

    // Rows in march order: r (loaded this iteration), q = r - DIR (first
    // stage computed this iteration), o = q - DIR (second stage).
    T b0[kCells], n0[kCells], s0[kCells];  // state row q
    T phB0[kCells], gB0[kCells];           // first-stage face between q - DIR and q
    T b1[kCells], n1[kCells];              // first-stage row o
    T s1[kCells], ls1 = T(0), rs1 = T(0);  // second-stage sigma of row o (+ x-neighbours)
    T ub[kCells], un[kCells];              // Heun: state row o
    T phB1[kCells], gB1[kCells];           // second-stage face between o - DIR and o
    bool in_q = false;  // row q lies inside the grid
    bool in_o = false;  // the first stage of row o was computed (row o inside the grid)
#pragma unroll
    for (int c = 0; c < kCells; ++c) {
        b0[c] = n0[c] = s0[c] = b1[c] = n1[c] = s1[c] = ub[c] = un[c] = T(0);
        phB0[c] = gB0[c] = phB1[c] = gB1[c] = T(0);
    }

    const int rfirst = DIR > 0 ? j0 - 2 : jend + 1;
    const int iters = (jend - j0) + 4;
    for (int p = 0; p < iters; ++p) {
        const int r = rfirst + DIR * p;
        const bool in_r = r >= 0 && r < ny;  // uniform across the block
        T br[kCells], nr[kCells], sr[kCells];
        if (in_r) load0(r, br, nr, sr);
        else {
#pragma unroll
            for (int c = 0; c < kCells; ++c) br[c] = nr[c] = sr[c] = T(0);
        }

        // first stage of row q
        const bool do1 = in_q && p >= 2;
        T phA0[kCells], gA0[kCells];
        T b1q[kCells], n1q[kCells], ls0 = T(0), rs0 = T(0);
        if (do1) {
            if (in_r) {
                if (DIR > 0) yface(s0, n0, b0, sr, nr, br, phA0, gA0);
                else yface(sr, nr, br, s0, n0, b0, phA0, gA0);
            } else {
#pragma unroll
                for (int c = 0; c < kCells; ++c) phA0[c] = gA0[c] = T(0);  // wall ahead
            }
            ls0 = __shfl_up_sync(kFull, s0[kCells - 1], 1);
            rs0 = __shfl_down_sync(kFull, s0[0], 1);
            T phX[kCells + 1], gX[kCells + 1];
            xfaces(s0, n0, b0, ls0, rs0, phX, gX);
            update(b0, n0, phX, gX, phB0, gB0, phA0, gA0, b1q, n1q);
        } else {
#pragma unroll
            for (int c = 0; c < kCells; ++c) {
                phA0[c] = gA0[c] = T(0);
                b1q[c] = n1q[c] = T(0);
            }
            // the face ahead of q is needed behind r on the next iteration
            if (in_q && in_r) {
                if (DIR > 0) yface(s0, n0, b0, sr, nr, br, phA0, gA0);
                else yface(sr, nr, br, s0, n0, b0, phA0, gA0);
            }
        }

        // second-stage sigma of row q
        T s2q[kCells];
        if (kSameSigma) {
#pragma unroll
            for (int c = 0; c < kCells; ++c) s2q[c] = s0[c];
        } else if (do1) {
            gen_sigma(nz2, r - DIR, s2q);
        } else {
#pragma unroll
            for (int c = 0; c < kCells; ++c) s2q[c] = T(0);
        }

        // second-stage face between o and q, then the second stage of row o
        T phA1[kCells], gA1[kCells];
        if (do1 && in_o) {
            if (DIR > 0) yface(s1, n1, b1, s2q, n1q, b1q, phA1, gA1);
            else yface(s2q, n1q, b1q, s1, n1, b1, phA1, gA1);
        } else {
#pragma unroll
            for (int c = 0; c < kCells; ++c) phA1[c] = gA1[c] = T(0);  // wall (or unused)
        }
        if (p >= 4) {
            const int o = r - 2 * DIR;
            if (!kSameSigma) {
                ls1 = __shfl_up_sync(kFull, s1[kCells - 1], 1);
                rs1 = __shfl_down_sync(kFull, s1[0], 1);
            }
            T phX[kCells + 1], gX[kCells + 1];
            xfaces(s1, n1, b1, ls1, rs1, phX, gX);
            T ob[kCells], on[kCells];
            update(b1, n1, phX, gX, phB1, gB1, phA1, gA1, ob, on);
            if (HEUN) {
#pragma unroll
                for (int c = 0; c < kCells; ++c) {
                    ob[c] = T(0.5) * (ub[c] + ob[c]);
                    on[c] = T(0.5) * (un[c] + on[c]);
                }
            }
            const long long off = (long long)o * pitch;
            if (writer) {
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
            }
        }

        // shift the pipeline by one row
#pragma unroll
        for (int c = 0; c < kCells; ++c) {
            if (HEUN) { ub[c] = b0[c]; un[c] = n0[c]; }
            b1[c] = b1q[c];
            n1[c] = n1q[c];
            s1[c] = s2q[c];
            phB1[c] = phA1[c];
            gB1[c] = gA1[c];
            b0[c] = br[c];
            n0[c] = nr[c];
            s0[c] = sr[c];
            phB0[c] = phA0[c];
            gB0[c] = gA0[c];
        }
        if (kSameSigma) { ls1 = ls0; rs1 = rs0; }
        in_o = do1;
        in_q = in_r;
    }
}

}  // namespace stencil
}  // namespace cx
