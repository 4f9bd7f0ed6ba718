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

#include <type_traits>

#include "cx_stencil.cuh"

namespace cx {
namespace stencil {

constexpr int kFusedCols = (32 - 2) * kCells;                  // written columns per warp
constexpr int kFusedBlockCols = (kThreads / 32) * kFusedCols;  // ... per four-warp block

// Threads per block of a two-stage pass.  The march's warps share nothing, so
// a block can be one warp (120 written columns): a grid whose width is not a
// multiple of 480 then leaves no block slot to idle warps (1024-wide grids
// run 1.35-1.46x faster than with four-warp blocks, 16384-wide ones 1.015x).
// With sigma drawn per step, four-warp blocks stay ahead on the single grid
// (measured 1 % at 16384^2).
template <int NOISE> constexpr int fused_threads() { return NOISE ? kThreads : 32; }

// One thread's two-stage march over the written rows j0..jend-1 in direction
// DIR.  x0: the thread's first column (may be negative or past the grid for
// the end lanes).  nz1 / nz2: the per-step noise of the first and second
// stage (NOISE 1; nz2 = nz1 under Heun).  INTERIOR: every column the warp
// holds lies inside the grid, x0 >= 0 and x0 + 4 <= nx for all threads.
// OFF32: element offsets fit in 32 bits (ny * pitch < 2^31), so each address
// is one widening multiply-add; measured faster only when sigma is drawn in
// registers (the per-step passes: Heun 1.036x, Euler 1.017x at 16384^2; the
// static-sigma passes ran 1-2 % slower).
template <typename T, int LAW, int MOB, int NOISE, bool HEUN, int DIR, bool INTERIOR,
          bool OFF32 = false>
__device__ __forceinline__ void march2(const Ptrs<T> &P, int nx, int ny, long long pitch,
                                       const KV<P2<T>> &k, const NoiseT<T> &nz1,
                                       const NoiseT<T> &nz2, int x0, int j0, int jend)
{
    // the second stage sees the first stage's sigma: static field, or Heun
    constexpr bool kSameSigma = (NOISE == 0) || HEUN;
    const int lane = threadIdx.x & 31;
    const long long xv =
        INTERIOR ? (long long)x0 : min(max((long long)x0, 0LL), pitch - (long long)kCells);
    const bool writer = lane != 0 && lane != 31;

    auto vload = [](const T *p) -> Cells<T> {
        T v[kCells];
        Vec<T>::load(p, v);
        return split4(v);
    };
    auto gen_sigma = [&](const NoiseT<T> &nz, int r) -> Cells<T> {
        T v[kCells];
        nz.four((long long)r * nx + x0, v);
        if (!INTERIOR) {
#pragma unroll
            for (int c = 0; c < kCells; ++c)
                if (x0 + c < 0 || x0 + c >= nx) v[c] = T(0);  // outside the row
        }
        return split4_nat(v);
    };
    // x-faces of a row; b and n of cell x0-1 from the left lane, sigma's
    // given (ls); the face beyond x0+3 is the right lane's first.  The end
    // lanes take their own values for the neighbour they lack
    auto xfaces = [&](const Cells<T> &s, const Cells<T> &n, const Cells<T> &b, T ls) {
        const T lb = __shfl_up_sync(kFull, b.O.y, 1), ln = __shfl_up_sync(kFull, n.O.y, 1);
        return row_xfaces_shfl<T, LAW, MOB, INTERIOR>(s, n, b, ls, ln, lb, k, x0, nx);
    };
    // y-faces between row (s, n, b)_1 and row (s, n, b)_2 in march order
    auto yfaces = [&](const Cells<T> &s1, const Cells<T> &n1, const Cells<T> &b1,
                      const Cells<T> &s2, const Cells<T> &n2, const Cells<T> &b2) {
        return DIR > 0 ? row_yfaces<T, LAW, MOB>(s1, n1, b1, s2, n2, b2, k)
                       : row_yfaces<T, LAW, MOB>(s2, n2, b2, s1, n1, b1, k);
    };

    // Rows in march order: r (loaded this iteration), q = r - DIR (first
    // stage computed this iteration), o = q - DIR (second stage).
    Cells<T> b0 = zero_cells<T>(), n0 = zero_cells<T>(), s0 = zero_cells<T>();  // state row q
    YFaces<T> yB0 = zero_yfaces<T>();  // first-stage faces between q - DIR and q
    Cells<T> b1 = zero_cells<T>(), n1 = zero_cells<T>();  // first-stage row o
    Cells<T> s1 = zero_cells<T>();     // second-stage sigma of row o
    T ls1 = T(0);                      // ... and its left neighbour
    Cells<T> ub = zero_cells<T>(), un = zero_cells<T>();  // Heun: state row o
    YFaces<T> yB1 = zero_yfaces<T>();  // second-stage faces between o - DIR and o
    bool in_q = false;  // row q lies inside the grid
    bool in_o = false;  // the first stage of row o was computed (row o inside the grid)

    const int rfirst = DIR > 0 ? j0 - 2 : jend + 1;
    // the last row this tile loads, in march order, clipped to the grid
    const int plast = DIR > 0 ? min(jend + 1, ny - 1) : max(j0 - 2, 0);
    const int iters = (jend - j0) + 4;
    // One iteration.  In the steady state (STEADY: from the fifth iteration
    // on, in a tile whose rows j0-2 .. jend+1 all lie inside the grid) every
    // row is in the grid and both stages run, so the tests drop out.
    auto body = [&](int p, auto steady) {
        constexpr bool STEADY = decltype(steady)::value;
        const int r = rfirst + DIR * p;
        const bool in_r = STEADY || (r >= 0 && r < ny);  // uniform across the block
        // element offset of this thread's vector in row r (OFF32: in 32 bits)
        const long long off = OFF32 ? (long long)(r * (int)pitch + (int)xv) : (long long)r * pitch + xv;
        if (DIR > 0 ? r + kPrefetchRows <= plast : r - kPrefetchRows >= plast)
            prefetch_row<T, NOISE>(P, OFF32 ? (long long)(r * (int)pitch + (int)xv +
                                                          DIR * kPrefetchRows * (int)pitch)
                                            : off + DIR * kPrefetchRows * pitch);
        Cells<T> br = zero_cells<T>(), nr = zero_cells<T>(), sr = zero_cells<T>();
        if (in_r) {
            br = vload(P.b + off);
            nr = vload(P.n + off);
            sr = NOISE == 0 ? vload(P.s + off) : gen_sigma(nz1, r);
        }

        // first-stage faces between q and r (a wall past the grid), then the
        // first stage of row q
        const bool both = STEADY || (in_q && in_r);
        const YFaces<T> yA0 = both ? yfaces(s0, n0, b0, sr, nr, br) : zero_yfaces<T>();
        const bool do1 = STEADY || (in_q && p >= 2);
        Cells<T> b1q = zero_cells<T>(), n1q = zero_cells<T>();
        T ls0 = T(0);
        if (do1) {
            ls0 = __shfl_up_sync(kFull, s0.O.y, 1);
            const XFaces<T> xf = xfaces(s0, n0, b0, ls0);
            row_update<T, DIR>(b0, n0, xf, yB0, yA0, k, b1q, n1q);
        }

        // second-stage sigma of row q
        Cells<T> s2q = s0;
        if (!kSameSigma) s2q = do1 ? gen_sigma(nz2, r - DIR) : zero_cells<T>();

        // second-stage faces between o and q, then the second stage of row o
        const bool have_o = STEADY || (do1 && in_o);
        const YFaces<T> yA1 = have_o ? yfaces(s1, n1, b1, s2q, n1q, b1q) : zero_yfaces<T>();
        if (STEADY || p >= 4) {
            const int o = r - 2 * DIR;
            if (!kSameSigma) ls1 = __shfl_up_sync(kFull, s1.O.y, 1);
            const XFaces<T> xf = xfaces(s1, n1, b1, ls1);
            Cells<T> ob, on;
            row_update<T, DIR>(b1, n1, xf, yB1, yA1, k, ob, on);
            if (HEUN) {
                ob = heun_mean(ub, ob, k);
                on = heun_mean(un, on, k);
            }
            T vb[kCells], vn[kCells];
            const long long off = OFF32 ? (long long)(o * (int)pitch) : (long long)o * pitch;
            if (writer) {
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
            }
        }

        // shift the pipeline by one row
        if (HEUN) {
            ub = b0;
            un = n0;
        }
        b1 = b1q;
        n1 = n1q;
        s1 = s2q;
        yB1 = yA1;
        b0 = br;
        n0 = nr;
        s0 = sr;
        yB0 = yA0;
        if (kSameSigma) ls1 = ls0;
        in_o = do1;
        in_q = in_r;
    };

    const int head = iters < 4 ? iters : 4;
    int p = 0;
    for (; p < head; ++p) body(p, std::false_type{});
    // uniform across the block: the rows the remaining iterations load
    const bool rows_inside = DIR > 0 ? jend + 1 < ny : j0 >= 2;
    if (rows_inside) {
        for (; p < iters; ++p) body(p, std::true_type{});
    } else {
        for (; p < iters; ++p) body(p, std::false_type{});
    }
}

}  // namespace stencil
}  // namespace cx
