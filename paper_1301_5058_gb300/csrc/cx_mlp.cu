// cx_mlp.cu -- the surrogate network: E independent MLPs 4 -> 256 -> 256 -> 2
// (tanh), the members of an ensemble, mapping sweep parameters to
// morphology labels and trained together on the GPU with their own forward
// and backward kernels and Adam.
//
// Per member:
//   Z1 = X W1^T + b1,  H1 = tanh(Z1)               (FP32, K = 4)
//   Z2 = bf(H1) bf(W2)^T + b2,  H2 = tanh(Z2)       (tensor cores, bf16 in, FP32 accumulate)
//   Y  = H2 W3^T + b3                               (FP32, N = 2)
//   loss = sum (Y - T)^2 / (2 B)
// Backward: dY = (Y - T)/B; dZ2 = (dY W3) (1 - H2^2); dW2 = bf(dZ2)^T bf(H1)
// and dH1 = bf(dZ2) bf(W2) on the tensor cores; dZ1 = dH1 (1 - H1^2); the
// bias and thin-layer gradients are column sums over the batch.
//
// One training step of all members is four launches, grid.y = member:
//   forward_kernel   H1 is computed while the A operand is staged, the
//                    256-wide product runs on tcgen05 with its accumulator
//                    in tensor memory, and in the epilogue each thread owns
//                    one batch row: H2, Y, dY, the row's loss and dZ2;
//   backward_kernel  the dH1 tiles (epilogue: dZ1) and the dW2 tiles, on
//                    tcgen05;
//   column_sums      the thin-layer and bias gradients and the loss, in a
//                    fixed summation order;
//   adam_kernel      Adam on the FP32 master parameters, and the bf16 copies
//                    of W2 and W2^T the next step reads.
// Members share no data, so member e of an E-member network computes what a
// one-member network computes, bit for bit.
//
// Tensor-core tiles.  A CTA of 128 threads computes D (128 x 256, FP32) =
// A (128 x K) B (256 x K)^T: A and B are staged K-major in shared memory,
// 128 columns of K at a time, in the no-swizzle canonical layout (8 x 8
// core matrices of 128 contiguous bytes); one elected thread issues
// tcgen05.mma (M = 128, N = 256, K = 16 each) into 256 columns of tensor
// memory and commits them to an mbarrier; every thread waits on it (a
// bounded wait) and reads its row (TMEM lane = tile row) with tcgen05.ld.
// The operands are small and L2-resident (at most 256 x 8192 bf16 per
// member), and the forward's A operand is computed, not copied, so the
// staging is plain 16-byte loads rather than TMA.
#include <cuda_bf16.h>
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <new>

#include "cx_internal.h"

namespace {

constexpr int H = 256;   // hidden width
constexpr int NI = 4;    // inputs
constexpr int NO = 2;    // outputs
// flat parameter layout of one member (FP32): W1, b1, W2, b2, W3, b3
constexpr int OFF_W1 = 0;
constexpr int OFF_B1 = OFF_W1 + H * NI;
constexpr int OFF_W2 = OFF_B1 + H;
constexpr int OFF_B2 = OFF_W2 + H * H;
constexpr int OFF_W3 = OFF_B2 + H;
constexpr int OFF_B3 = OFF_W3 + NO * H;
constexpr int NPARAM = OFF_B3 + NO;
static_assert(NPARAM == CX_MLP_PARAMS, "parameter packing");

constexpr int kMaxMembers = 64;
constexpr int kRows = 128;          // tile rows = TMEM lanes
// 16 warps per tile: warp w reads TMEM lanes 32 (w % 4) .. + 31 (the lanes
// its rank in a group of four may access) and the columns of quarter w / 4
constexpr int kThreads = 512;
constexpr int kQuarter = 64;        // accumulator columns per warp
constexpr int kKC = 128;            // K columns staged per round
constexpr int kSmemA = kRows * kKC * 2;     // 32 KB
constexpr int kSmemB = H * kKC * 2;         // 64 KB
// Shared memory of a tile CTA: the operand buffers A and B from 0; after the
// last product, the forward epilogue's H2 tile over them (rows padded to
// 260 floats so that 8 rows' 16-byte accesses hit distinct banks); then the
// small parameter vectors, the row partial sums, and the barrier.  Each tile
// CTA takes the largest allocation, so one tile CTA runs per SM and its 256
// tensor-memory columns never wait for another's.
constexpr int kH2Stride = H + 4;
constexpr int kSmemPrm = kRows * kH2Stride * 4;            // W1, b1, b2, W3, b3
constexpr int kNPrm = H * NI + H + H + NO * H + NO;
constexpr int kSmemPart = kSmemPrm + (kNPrm * 4 + 15) / 16 * 16;  // [4][kRows][2]
constexpr int kSmemBar = kSmemPart + 4 * kRows * 2 * 4;
constexpr int kSmemTile = 232448;
static_assert(kSmemA + kSmemB <= kSmemPrm && kSmemBar + 16 <= kSmemTile, "tile shared memory");
constexpr int kTmemCols = 256;      // FP32 accumulator columns (N)
constexpr uint32_t kDrainLimit = 1u << 22;  // second wait, after a timeout

// ---- tcgen05 / mbarrier wrappers -------------------------------------------

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

// Shared-memory matrix descriptor, no swizzle: start address, leading
// dimension byte offset (between the core matrices adjacent in K), stride
// dimension byte offset (between those adjacent in M or N), each >> 4; bit
// 46 is the descriptor version Blackwell requires; layout type 0.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo)
{
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// Instruction descriptor of kind::f16: D FP32 (bits 4-5 = 1), A and B bf16
// (bits 7-9, 10-12 = 1), both K-major (bits 15, 16 = 0), N >> 3 in bits
// 17-22, M >> 4 in bits 24-28.
constexpr uint32_t idesc_bf16_f32(int M, int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) |
           ((uint32_t)(M >> 4) << 24);
}
constexpr uint32_t kIdesc = idesc_bf16_f32(kRows, H);

__device__ __forceinline__ void tmem_alloc(uint32_t slot, uint32_t ncols)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(slot),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols)
                 : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// D (TMEM) (+)= A B^T for one K = 16 slice; accumulate = 0 overwrites D.
__device__ __forceinline__ void mma_bf16(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc,
                                         uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
        : "memory");
}

// The mbarrier's phase completes once every tcgen05 operation this thread
// issued before has completed.
__device__ __forceinline__ void mma_commit(uint32_t bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}

__device__ __forceinline__ void bar_init(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Polls the phase of the given parity at most `limit` times.
__device__ __forceinline__ bool bar_wait(uint32_t bar, uint32_t parity, uint32_t limit)
{
    for (uint32_t it = 0; it < limit; ++it) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

// 16 consecutive FP32 columns of this thread's TMEM lane (32x32b shape:
// thread t of the warp reads lane base + t).
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16])
{
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n\t"
        "tcgen05.wait::ld.sync.aligned;\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
          "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// Byte offset of element (r, 8 c8 .. 8 c8 + 7) of an R-row K-major bf16
// operand in the canonical layout: row r of a core matrix at 16 (r & 7), the
// 8-row groups 128 B apart (stride byte offset), the 8-column groups R * 16
// B apart (leading byte offset).
__device__ __forceinline__ uint32_t core_off(int R, int r, int c8)
{
    return (uint32_t)(c8 * R * 16 + (r >> 3) * 128 + (r & 7) * 16);
}

// Item i of a staging round: row r and 8-column group c8 of the kKC
// columns; eight consecutive items fill one core matrix (128 contiguous
// bytes of shared memory, 16 B from each of 8 rows).
__device__ __forceinline__ void stage_item(int i, int &r, int &c8)
{
    constexpr int c8n = kKC / 8;
    c8 = (i >> 3) % c8n;
    r = (i >> 3) / c8n * 8 + (i & 7);
}

// Rows [r0, r0 + R) x columns [k0, k0 + kKC) of a row-major bf16 matrix
// (leading dimension ld, a multiple of 8) into the canonical layout at s:
// every thread issues all its loads before its first store.
template <int R>
__device__ __forceinline__ void stage_bf16(uint8_t *s, const __nv_bfloat16 *__restrict__ g,
                                           long long ld, int r0, int k0)
{
    constexpr int per = R * (kKC / 8) / kThreads;
    uint4 v[per];
#pragma unroll
    for (int u = 0; u < per; ++u) {
        int r, c8;
        stage_item(threadIdx.x + u * kThreads, r, c8);
        v[u] = *reinterpret_cast<const uint4 *>(g + (long long)(r0 + r) * ld + k0 + c8 * 8);
    }
#pragma unroll
    for (int u = 0; u < per; ++u) {
        int r, c8;
        stage_item(threadIdx.x + u * kThreads, r, c8);
        *reinterpret_cast<uint4 *>(s + core_off(R, r, c8)) = v[u];
    }
}

__device__ __forceinline__ uint32_t pack_bf16(float a, float b)
{
    const __nv_bfloat16 x = __float2bfloat16_rn(a), y = __float2bfloat16_rn(b);
    return (uint32_t)__bfloat16_as_ushort(x) | ((uint32_t)__bfloat16_as_ushort(y) << 16);
}

// Device view of an E-member network; member e's arrays start at e times
// the per-member sizes (NPARAM, H * H, Bmax * H, Bmax * NO, Bmax).
struct NetView {
    const float *P;                        // parameters
    const __nv_bfloat16 *W2b, *W2T;        // bf16 W2 and W2^T
    float *G;                              // gradients
    float *H1f, *H2, *dZ2, *dZ1;           // Bmax x H, FP32
    __nv_bfloat16 *H1T, *dZ2b, *dZ2T;      // H1^T (H x Bp), bf(dZ2) (Bp x H), bf(dZ2)^T
    float *Y, *dY;                         // Bmax x NO
    double *lrow;                          // per-row loss terms
    long long Bmax;
    int *err;                              // set when a tensor-core wait ran out
    uint32_t limit;                        // polls before that wait gives up
};

struct Tile {
    uint8_t *sA, *sB;
    uint32_t bar, tmem;
};

// Warp 0 allocates the accumulator's tensor-memory columns; thread 0
// initialises the completion barrier.
__device__ __forceinline__ Tile tile_setup(uint8_t *smem)
{
    Tile t;
    t.sA = smem;
    t.sB = smem + kSmemA;
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem + kSmemBar);
    uint32_t *slot = reinterpret_cast<uint32_t *>(bar + 1);
    t.bar = smem_u32(bar);
    if (threadIdx.x < 32) tmem_alloc(smem_u32(slot), kTmemCols);
    if (threadIdx.x == 0) bar_init(t.bar, 1);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    t.tmem = *slot;
    return t;
}

__device__ __forceinline__ void tile_teardown(const Tile &t)
{
    tc_fence_before();
    __syncthreads();
    if (threadIdx.x < 32) tmem_dealloc(t.tmem, kTmemCols);
}

// D (TMEM, 128 x 256 FP32) = A (128 x K) B (256 x K)^T, K a multiple of
// kKC, in rounds of kKC columns: stage_a(k0) and stage_b(k0) fill the
// operand buffers, thread 0 issues kKC / 16 products and commits them, and
// all threads wait for them before the buffers are refilled.  Returns false,
// in every thread alike, when a wait ran out: the error flag is set and the
// products in flight are waited for (again with a limit) so that the tensor
// memory can be released.
template <class SA, class SB>
__device__ __forceinline__ bool tile_product(const Tile &t, int K, uint32_t limit, int *err,
                                             SA stage_a, SB stage_b)
{
    uint32_t phase = 0;
    for (int k0 = 0; k0 < K; k0 += kKC) {
        stage_a(k0);
        stage_b(k0);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // stores -> tensor cores
        __syncthreads();
        if (threadIdx.x == 0) {
            tc_fence_after();
            const uint32_t a0 = smem_u32(t.sA), b0 = smem_u32(t.sB);
#pragma unroll
            for (int kk = 0; kk < kKC; kk += 16) {
                const uint64_t da = smem_desc(a0 + (uint32_t)(kk >> 3) * kRows * 16, kRows * 16, 128);
                const uint64_t db = smem_desc(b0 + (uint32_t)(kk >> 3) * H * 16, H * 16, 128);
                mma_bf16(t.tmem, da, db, kIdesc, (k0 + kk) > 0 ? 1u : 0u);
            }
            mma_commit(t.bar);
        }
        const bool ok = __syncthreads_and(bar_wait(t.bar, phase, limit));
        if (!ok) {
            if (threadIdx.x == 0) atomicExch(err, 1);
            bar_wait(t.bar, phase, kDrainLimit);
            __syncthreads();
            return false;
        }
        phase ^= 1u;
    }
    tc_fence_after();
    return true;
}

__device__ __forceinline__ void store16(float *p, const float (&v)[16])
{
#pragma unroll
    for (int i = 0; i < 16; i += 4)
        *reinterpret_cast<float4 *>(p + i) = make_float4(v[i], v[i + 1], v[i + 2], v[i + 3]);
}

// This thread's place in the epilogue: tile row r (TMEM lane 32 (w % 4) +
// lane of warp w) and the first of its 64 columns, j0 = 64 (w / 4).
struct Seat {
    int r, q, j0;
    uint32_t ta;  // tensor-memory address of (row r, column j0)
};
__device__ __forceinline__ Seat seat(const Tile &t)
{
    Seat s;
    const int w = threadIdx.x >> 5, g = w & 3;
    s.q = w >> 2;
    s.r = 32 * g + (threadIdx.x & 31);
    s.j0 = s.q * kQuarter;
    s.ta = t.tmem + ((uint32_t)(32 * g) << 16) + (uint32_t)s.j0;
    return s;
}

// Forward pass of batch rows [m0, m0 + 128) of member blockIdx.y (rows past
// nb are padding: H1 = 0, no loss, dY = 0).  BACK: also the quantities the
// backward pass reads (H1 in FP32 and as bf16 H1^T, H2, dY, the row loss,
// dZ2 in FP32, bf16 and bf16 transposed).  X and T: row-major inputs and
// targets, member e's at X + e xs and T + e ts.  Each row's two outputs are
// summed over its four column quarters, then added to b3 in quarter order.
template <bool BACK>
__global__ void __launch_bounds__(kThreads, 1)
    forward_kernel(NetView v, const float *__restrict__ X, long long xs,
                   const float *__restrict__ T, long long ts, int nb, int Bp)
{
    extern __shared__ __align__(1024) uint8_t smem[];
    const int e = blockIdx.y, m0 = blockIdx.x * kRows;
    const float *__restrict__ P = v.P + (long long)e * NPARAM;
    X += (long long)e * xs;
    const long long act = (long long)e * v.Bmax * H;
    const __nv_bfloat16 *W2b = v.W2b + (long long)e * H * H;
    // W1, b1 (contiguous in P), then b2, W3, b3 (contiguous in P)
    float *prm = reinterpret_cast<float *>(smem + kSmemPrm);
    const float *sW1 = prm, *sB1 = prm + H * NI, *sB2 = sB1 + H, *sW3 = sB2 + H, *sB3 = sW3 + NO * H;
    for (int i = threadIdx.x; i < H * NI + H; i += kThreads) prm[i] = P[OFF_W1 + i];
    for (int i = threadIdx.x; i < H + NO * H + NO; i += kThreads) prm[H * NI + H + i] = P[OFF_B2 + i];
    const Tile t = tile_setup(smem);  // (its barrier also publishes prm)

    // A = bf(H1) for the tile's rows, computed while it is staged
    auto stage_a = [&](int k0) {
        constexpr int per = kRows * (kKC / 8) / kThreads;
#pragma unroll 1
        for (int u = 0; u < per; ++u) {
            int r, c8;
            stage_item(threadIdx.x + u * kThreads, r, c8);
            const int b = m0 + r, j0 = k0 + c8 * 8;
            float h[8];
            if (b < nb) {
                const float4 x = *reinterpret_cast<const float4 *>(X + (long long)b * NI);
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const float4 w = *reinterpret_cast<const float4 *>(sW1 + (j0 + q) * NI);
                    float z = sB1[j0 + q];
                    z += w.x * x.x;
                    z += w.y * x.y;
                    z += w.z * x.z;
                    z += w.w * x.w;
                    h[q] = tanhf(z);
                }
            } else {
#pragma unroll
                for (int q = 0; q < 8; ++q) h[q] = 0.f;
            }
            *reinterpret_cast<uint4 *>(t.sA + core_off(kRows, r, c8)) =
                make_uint4(pack_bf16(h[0], h[1]), pack_bf16(h[2], h[3]), pack_bf16(h[4], h[5]),
                           pack_bf16(h[6], h[7]));
            if (BACK) {
                float *hf = v.H1f + act + (long long)b * H + j0;
                *reinterpret_cast<float4 *>(hf) = make_float4(h[0], h[1], h[2], h[3]);
                *reinterpret_cast<float4 *>(hf + 4) = make_float4(h[4], h[5], h[6], h[7]);
#pragma unroll
                for (int q = 0; q < 8; ++q)
                    v.H1T[act + (long long)(j0 + q) * Bp + b] = __float2bfloat16_rn(h[q]);
            }
        }
    };
    auto stage_b = [&](int k0) { stage_bf16<H>(t.sB, W2b, H, 0, k0); };
    const bool ok = tile_product(t, H, v.limit, v.err, stage_a, stage_b);

    if (ok) {
        const Seat st = seat(t);
        const int b = m0 + st.r;
        // the products are complete: H2 may overwrite the operand buffers
        float *h2s = reinterpret_cast<float *>(smem) + st.r * kH2Stride + st.j0;
        float *part = reinterpret_cast<float *>(smem + kSmemPart);  // [4][kRows][2]
        float s0 = 0.f, s1 = 0.f;
#pragma unroll 1
        for (int c = 0; c < kQuarter / 16; ++c) {
            float a[16];
            tmem_ld16(st.ta + 16 * c, a);
#pragma unroll
            for (int q = 0; q < 16; ++q) {
                const int j = st.j0 + 16 * c + q;
                const float h = tanhf(a[q] + sB2[j]);
                s0 += sW3[j] * h;
                s1 += sW3[H + j] * h;
                a[q] = h;
            }
            if (BACK) {
                store16(v.H2 + act + (long long)b * H + st.j0 + 16 * c, a);
                store16(h2s + 16 * c, a);
            }
        }
        part[(st.q * kRows + st.r) * 2] = s0;
        part[(st.q * kRows + st.r) * 2 + 1] = s1;
        __syncthreads();
        float y0 = sB3[0], y1 = sB3[1];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            y0 += part[(k * kRows + st.r) * 2];
            y1 += part[(k * kRows + st.r) * 2 + 1];
        }
        const long long yo = (long long)e * v.Bmax * NO + (long long)b * NO;
        if (st.q == 0) {
            v.Y[yo] = y0;
            v.Y[yo + 1] = y1;
        }
        if (BACK) {
            float d0 = 0.f, d1 = 0.f;
            double l = 0.0;
            if (b < nb) {
                T += (long long)e * ts;
                const float r0 = y0 - T[(long long)b * NO], r1 = y1 - T[(long long)b * NO + 1];
                d0 = r0 / (float)nb;
                d1 = r1 / (float)nb;
                l += 0.5 * (double)r0 * (double)r0;
                l += 0.5 * (double)r1 * (double)r1;
            }
            if (st.q == 0) {
                v.dY[yo] = d0;
                v.dY[yo + 1] = d1;
                v.lrow[(long long)e * v.Bmax + b] = l;
            }
#pragma unroll 1
            for (int c = 0; c < kQuarter / 16; ++c) {
                float a[16];
#pragma unroll
                for (int q = 0; q < 16; q += 4) {
                    const float4 h4 = *reinterpret_cast<const float4 *>(h2s + 16 * c + q);
                    a[q] = h4.x;
                    a[q + 1] = h4.y;
                    a[q + 2] = h4.z;
                    a[q + 3] = h4.w;
                }
#pragma unroll
                for (int q = 0; q < 16; ++q) {
                    const int j = st.j0 + 16 * c + q;
                    const float h = a[q];
                    float s = 0.f;
                    s += d0 * sW3[j];
                    s += d1 * sW3[H + j];
                    a[q] = s * (1.f - h * h);
                    v.dZ2T[act + (long long)j * Bp + b] = __float2bfloat16_rn(a[q]);
                }
                const long long o = act + (long long)b * H + st.j0 + 16 * c;
                store16(v.dZ2 + o, a);
                uint4 *pb = reinterpret_cast<uint4 *>(v.dZ2b + o);
                pb[0] = make_uint4(pack_bf16(a[0], a[1]), pack_bf16(a[2], a[3]), pack_bf16(a[4], a[5]),
                                   pack_bf16(a[6], a[7]));
                pb[1] = make_uint4(pack_bf16(a[8], a[9]), pack_bf16(a[10], a[11]),
                                   pack_bf16(a[12], a[13]), pack_bf16(a[14], a[15]));
            }
        }
    }
    tile_teardown(t);
}

// Backward products of member blockIdx.y.  Tiles 0 .. Bp/128 - 1: dH1 for
// batch rows [128 t, 128 t + 128) = bf(dZ2) rows times bf(W2) (B operand:
// the rows of W2^T), epilogue dZ1 = dH1 (1 - H1^2).  The last two tiles:
// dW2 rows [128 u, 128 u + 128) = bf(dZ2)^T rows times bf(H1) (B operand:
// the rows of H1^T), over K = Bp.
__global__ void __launch_bounds__(kThreads, 1) backward_kernel(NetView v, int Bp)
{
    extern __shared__ __align__(1024) uint8_t smem[];
    const int e = blockIdx.y, nt = Bp / kRows;
    const long long act = (long long)e * v.Bmax * H;
    const Tile t = tile_setup(smem);
    if ((int)blockIdx.x < nt) {
        const int m0 = blockIdx.x * kRows;
        const __nv_bfloat16 *A = v.dZ2b + act, *B = v.W2T + (long long)e * H * H;
        const bool ok = tile_product(
            t, H, v.limit, v.err, [&](int k0) { stage_bf16<kRows>(t.sA, A, H, m0, k0); },
            [&](int k0) { stage_bf16<H>(t.sB, B, H, 0, k0); });
        if (ok) {
            const Seat st = seat(t);
            const long long row = act + (long long)(m0 + st.r) * H + st.j0;
#pragma unroll 1
            for (int c = 0; c < kQuarter / 16; ++c) {
                float a[16];
                tmem_ld16(st.ta + 16 * c, a);
#pragma unroll
                for (int q = 0; q < 16; q += 4) {
                    const float4 h1 = *reinterpret_cast<const float4 *>(v.H1f + row + 16 * c + q);
                    a[q] = a[q] * (1.f - h1.x * h1.x);
                    a[q + 1] = a[q + 1] * (1.f - h1.y * h1.y);
                    a[q + 2] = a[q + 2] * (1.f - h1.z * h1.z);
                    a[q + 3] = a[q + 3] * (1.f - h1.w * h1.w);
                }
                store16(v.dZ1 + row + 16 * c, a);
            }
        }
    } else {
        const int i0 = (blockIdx.x - nt) * kRows;
        const __nv_bfloat16 *A = v.dZ2T + act, *B = v.H1T + act;
        const bool ok = tile_product(
            t, Bp, v.limit, v.err, [&](int k0) { stage_bf16<kRows>(t.sA, A, Bp, i0, k0); },
            [&](int k0) { stage_bf16<H>(t.sB, B, Bp, 0, k0); });
        if (ok) {
            // a member's block starts at e * NPARAM floats, a multiple of 8
            // bytes only: pairs, not quads
            const Seat st = seat(t);
            float *g = v.G + (long long)e * NPARAM + OFF_W2 + (long long)(i0 + st.r) * H + st.j0;
#pragma unroll 1
            for (int c = 0; c < kQuarter / 16; ++c) {
                float a[16];
                tmem_ld16(st.ta + 16 * c, a);
#pragma unroll
                for (int q = 0; q < 16; q += 2)
                    *reinterpret_cast<float2 *>(g + 16 * c + q) = make_float2(a[q], a[q + 1]);
            }
        }
    }
    tile_teardown(t);
}

// Column sums over the nb valid rows of member blockIdx.y (padding rows
// carry zero gradients), for 16 hidden units per block: dW3, db2, dW1, db1
// (with dZ1 from the backward tiles).  Each of the 32 thread rows sums
// every 32nd batch row, then the 32 partial sums are added in order.  Block
// 0 also sums db3 and the loss into loss_dst[e * loss_stride] (if given).
constexpr int kSumCols = 16, kSumRows = 32;
__global__ void __launch_bounds__(kSumCols *kSumRows)
    column_sums(NetView v, const float *__restrict__ X, long long xs, int nb, double *loss_dst,
                long long loss_stride)
{
    __shared__ float part[kSumRows][8][kSumCols];
    __shared__ float dpart[kSumRows * kSumCols][NO];
    __shared__ double lpart[kSumRows * kSumCols];
    const int e = blockIdx.y, tx = threadIdx.x, ty = threadIdx.y;
    const int j = blockIdx.x * kSumCols + tx;
    X += (long long)e * xs;
    const long long act = (long long)e * v.Bmax * H;
    const float *__restrict__ H2 = v.H2 + act;
    const float *__restrict__ dZ2 = v.dZ2 + act;
    const float *__restrict__ dZ1 = v.dZ1 + act;
    const float *__restrict__ dY = v.dY + (long long)e * v.Bmax * NO;
    float acc[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};  // dW3 (2), db2, dW1 (4), db1
#pragma unroll 4
    for (int b = ty; b < nb; b += kSumRows) {
        const long long q = (long long)b * H + j;
        const float h2 = H2[q];
        acc[0] += dY[(long long)b * NO] * h2;
        acc[1] += dY[(long long)b * NO + 1] * h2;
        acc[2] += dZ2[q];
        const float dz1 = dZ1[q];
#pragma unroll
        for (int k = 0; k < NI; ++k) acc[3 + k] += dz1 * X[(long long)b * NI + k];
        acc[7] += dz1;
    }
#pragma unroll
    for (int a = 0; a < 8; ++a) part[ty][a][tx] = acc[a];
    __syncthreads();
    float *G = v.G + (long long)e * NPARAM;
    if (ty == 0) {
        float s[8];
#pragma unroll
        for (int a = 0; a < 8; ++a) {
            s[a] = part[0][a][tx];
            for (int y = 1; y < kSumRows; ++y) s[a] += part[y][a][tx];
        }
        G[OFF_W3 + j] = s[0];
        G[OFF_W3 + H + j] = s[1];
        G[OFF_B2 + j] = s[2];
#pragma unroll
        for (int k = 0; k < NI; ++k) G[OFF_W1 + j * NI + k] = s[3 + k];
        G[OFF_B1 + j] = s[7];
    }
    if (blockIdx.x == 0) {
        const int tid = ty * kSumCols + tx, nth = kSumRows * kSumCols;
        float d0 = 0.f, d1 = 0.f;
        double l = 0.0;
        const double *lrow = v.lrow + (long long)e * v.Bmax;
        for (int b = tid; b < nb; b += nth) {
            d0 += dY[(long long)b * NO];
            d1 += dY[(long long)b * NO + 1];
            l += lrow[b];
        }
        dpart[tid][0] = d0;
        dpart[tid][1] = d1;
        lpart[tid] = l;
        __syncthreads();
        // pairwise tree in a fixed order (a serial chain of FP64 additions
        // would cost more than the rest of the kernel)
        for (int w = nth / 2; w > 0; w >>= 1) {
            if (tid < w) {
                dpart[tid][0] += dpart[tid + w][0];
                dpart[tid][1] += dpart[tid + w][1];
                lpart[tid] += lpart[tid + w];
            }
            __syncthreads();
        }
        if (tid == 0) {
            G[OFF_B3] = dpart[0][0];
            G[OFF_B3 + 1] = dpart[0][1];
            if (loss_dst) loss_dst[(long long)e * loss_stride] = lpart[0];
        }
    }
}

// Adam (Kingma & Ba, 2015) on the FP32 master parameters of every member;
// the threads of W2 entries also write the bf16 copies of W2 and W2^T.
__global__ void adam_kernel(float *__restrict__ P, const float *__restrict__ G, float *__restrict__ M,
                            float *__restrict__ V, __nv_bfloat16 *__restrict__ W2b,
                            __nv_bfloat16 *__restrict__ W2T, long long n, float lr, float b1, float b2,
                            float eps, float c1, float c2)
{
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float g = G[i];
    const float m = b1 * M[i] + (1.f - b1) * g;
    const float vv = b2 * V[i] + (1.f - b2) * g * g;
    M[i] = m;
    V[i] = vv;
    const float p = P[i] - lr * (m / c1) / (sqrtf(vv / c2) + eps);
    P[i] = p;
    const long long e = i / NPARAM;
    const int o = (int)(i - e * NPARAM) - OFF_W2;
    if (o >= 0 && o < H * H) {
        const __nv_bfloat16 w = __float2bfloat16_rn(p);
        W2b[e * H * H + o] = w;
        W2T[e * H * H + (o % H) * H + o / H] = w;
    }
}

// bf16 copies of every member's W2 (row-major) and W2^T.
__global__ void refresh_w2(const float *__restrict__ P, __nv_bfloat16 *__restrict__ W2b,
                           __nv_bfloat16 *__restrict__ W2T, long long n)
{
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const long long e = i / (H * H);
    const int o = (int)(i - e * H * H);
    const __nv_bfloat16 w = __float2bfloat16_rn(P[e * NPARAM + OFF_W2 + o]);
    W2b[i] = w;
    W2T[e * H * H + (o % H) * H + o / H] = w;
}

int mfail(int code, const char *msg) { return cx::record_error(code, msg); }

int mcuda(cudaError_t e, const char *what)
{
    char buf[300];
    snprintf(buf, sizeof buf, "%s: %s", what, cudaGetErrorString(e));
    return cx::record_error(e == cudaErrorMemoryAllocation ? CX_ERR_OOM : CX_ERR_CUDA, buf);
}

#define MX_CUDA(call, what)                                 \
    do {                                                    \
        cudaError_t e_ = (call);                            \
        if (e_ != cudaSuccess) return mcuda(e_, (what));    \
    } while (0)

}  // namespace

struct cx_mlp {
    int E = 1;          // members
    long long Bmax = 0; // padded batch capacity (multiple of 128)
    float *P = nullptr, *G = nullptr, *M = nullptr, *V = nullptr;
    __nv_bfloat16 *W2b = nullptr, *W2T = nullptr;
    float *X = nullptr, *T = nullptr;  // inputs and targets of forward / gradient calls
    float *H1f = nullptr, *H2 = nullptr, *dZ2 = nullptr, *dZ1 = nullptr, *Y = nullptr, *dY = nullptr;
    __nv_bfloat16 *H1T = nullptr, *dZ2b = nullptr, *dZ2T = nullptr;
    double *lrow = nullptr, *loss = nullptr;
    float *dataX = nullptr, *dataT = nullptr;  // training sets on the device
    long long ndata = 0;
    double *losses = nullptr;  // per-step losses of a training call, on the device
    long long nlosses = 0;
    int *err = nullptr;
    uint32_t limit = 1u << 22;  // polls before a tensor-core wait gives up
    long long adam_t = 0;
    cudaStream_t st = nullptr;
};

namespace {

void free_mlp(cx_mlp *m)
{
    if (!m) return;
    void *ptrs[] = {m->P, m->G, m->M, m->V, m->W2b, m->W2T, m->X, m->T, m->H1f, m->H2, m->dZ2,
                    m->dZ1, m->Y, m->dY, m->H1T, m->dZ2b, m->dZ2T, m->lrow, m->loss, m->dataX,
                    m->dataT, m->losses, m->err};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    if (m->st) cudaStreamDestroy(m->st);
    delete m;
}

long long pad128(long long b) { return (b + 127) / 128 * 128; }

NetView view(const cx_mlp *m)
{
    NetView v;
    v.P = m->P;
    v.W2b = m->W2b;
    v.W2T = m->W2T;
    v.G = m->G;
    v.H1f = m->H1f;
    v.H2 = m->H2;
    v.dZ2 = m->dZ2;
    v.dZ1 = m->dZ1;
    v.H1T = m->H1T;
    v.dZ2b = m->dZ2b;
    v.dZ2T = m->dZ2T;
    v.Y = m->Y;
    v.dY = m->dY;
    v.lrow = m->lrow;
    v.Bmax = m->Bmax;
    v.err = m->err;
    v.limit = m->limit;
    return v;
}

// Forward (and, with T, backward into m->G) of every member on rows
// [0, nb) of X (member e's at X + e xs; targets T + e ts).  loss_dst: the
// members' batch losses (sum of squares / 2), member e at e * loss_stride.
cudaError_t run_pass(cx_mlp *m, const float *X, long long xs, const float *T, long long ts, int nb,
                     double *loss_dst, long long loss_stride)
{
    const int Bp = (int)pad128(nb);
    const NetView v = view(m);
    const dim3 grid(Bp / kRows, m->E);
    if (!T) {
        forward_kernel<false><<<grid, kThreads, kSmemTile, m->st>>>(v, X, xs, nullptr, 0, nb, Bp);
        return cudaGetLastError();
    }
    forward_kernel<true><<<grid, kThreads, kSmemTile, m->st>>>(v, X, xs, T, ts, nb, Bp);
    backward_kernel<<<dim3(Bp / kRows + H / kRows, m->E), kThreads, kSmemTile, m->st>>>(v, Bp);
    column_sums<<<dim3(H / kSumCols, m->E), dim3(kSumCols, kSumRows), 0, m->st>>>(v, X, xs, nb, loss_dst,
                                                                                   loss_stride);
    return cudaGetLastError();
}

// After the stream has drained: CX_ERR_TIMEOUT if a tile's wait ran out
// (the flag is cleared for the next call).
int check_waits(cx_mlp *m)
{
    int h = 0;
    MX_CUDA(cudaMemcpyAsync(&h, m->err, sizeof h, cudaMemcpyDeviceToHost, m->st), "status download");
    MX_CUDA(cudaStreamSynchronize(m->st), "network synchronize");
    if (h) {
        MX_CUDA(cudaMemsetAsync(m->err, 0, sizeof(int), m->st), "status reset");
        MX_CUDA(cudaStreamSynchronize(m->st), "network synchronize");
        return mfail(CX_ERR_TIMEOUT, "a tensor-core completion wait ran out");
    }
    return CX_OK;
}

int check_batch_arg(cx_mlp *m, int nb)
{
    if (!m) return mfail(CX_ERR_INVALID_ARG, "NULL network");
    if (nb < 1 || pad128(nb) > m->Bmax) return mfail(CX_ERR_INVALID_ARG, "batch outside 1..max_batch");
    return CX_OK;
}

}  // namespace

extern "C" {

int cx_mlp_create_members(int32_t max_batch, int32_t members, cx_mlp **out)
{
    if (!out) return mfail(CX_ERR_INVALID_ARG, "out must not be NULL");
    *out = nullptr;
    if (max_batch < 1 || max_batch > (1 << 20)) return mfail(CX_ERR_INVALID_ARG, "max_batch outside 1..2^20");
    if (members < 1 || members > kMaxMembers) return mfail(CX_ERR_INVALID_ARG, "members outside 1..64");
    cx_mlp *m = new (std::nothrow) cx_mlp;
    if (!m) return mfail(CX_ERR_OOM, "host allocation");
    m->E = members;
    m->Bmax = pad128(max_batch);
    if (const char *s = getenv("CX_MMA_WAIT_LIMIT")) m->limit = (uint32_t)strtoul(s, nullptr, 10);
    const size_t E = (size_t)members, Bp = (size_t)m->Bmax;
    cudaError_t e = cudaStreamCreateWithFlags(&m->st, cudaStreamNonBlocking);
    auto A = [&](void **p, size_t bytes) {
        if (e == cudaSuccess) e = cudaMalloc(p, bytes);
        if (e == cudaSuccess) e = cudaMemset(*p, 0, bytes);
    };
    A((void **)&m->P, E * NPARAM * 4); A((void **)&m->G, E * NPARAM * 4);
    A((void **)&m->M, E * NPARAM * 4); A((void **)&m->V, E * NPARAM * 4);
    A((void **)&m->W2b, E * H * H * 2); A((void **)&m->W2T, E * H * H * 2);
    A((void **)&m->X, Bp * NI * 4); A((void **)&m->T, Bp * NO * 4);
    A((void **)&m->H1f, E * Bp * H * 4); A((void **)&m->H2, E * Bp * H * 4);
    A((void **)&m->dZ2, E * Bp * H * 4); A((void **)&m->dZ1, E * Bp * H * 4);
    A((void **)&m->H1T, E * Bp * H * 2); A((void **)&m->dZ2b, E * Bp * H * 2);
    A((void **)&m->dZ2T, E * Bp * H * 2);
    A((void **)&m->Y, E * Bp * NO * 4); A((void **)&m->dY, E * Bp * NO * 4);
    A((void **)&m->lrow, E * Bp * 8); A((void **)&m->loss, E * 8);
    A((void **)&m->err, sizeof(int));
    const void *tiles[] = {(const void *)forward_kernel<false>, (const void *)forward_kernel<true>,
                           (const void *)backward_kernel};
    for (const void *f : tiles)
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemTile);
    if (e != cudaSuccess) {
        cudaGetLastError();
        free_mlp(m);
        return mcuda(e, "network allocation");
    }
    *out = m;
    return CX_OK;
}

int cx_mlp_create(int32_t max_batch, cx_mlp **out) { return cx_mlp_create_members(max_batch, 1, out); }

int32_t cx_mlp_members(const cx_mlp *m) { return m ? m->E : 0; }

void cx_mlp_destroy(cx_mlp *m)
{
    if (m && m->st) cudaStreamSynchronize(m->st);
    free_mlp(m);
}

int cx_mlp_set_params(cx_mlp *m, const float *host, size_t count)
{
    if (!m || !host) return mfail(CX_ERR_INVALID_ARG, "NULL argument");
    const size_t n = (size_t)m->E * NPARAM;
    if (count != n) return mfail(CX_ERR_INVALID_ARG, "count != members x CX_MLP_PARAMS");
    MX_CUDA(cudaMemcpyAsync(m->P, host, n * 4, cudaMemcpyHostToDevice, m->st), "parameter upload");
    MX_CUDA(cudaMemsetAsync(m->M, 0, n * 4, m->st), "adam reset");
    MX_CUDA(cudaMemsetAsync(m->V, 0, n * 4, m->st), "adam reset");
    m->adam_t = 0;
    const long long nw = (long long)m->E * H * H;
    refresh_w2<<<(unsigned)((nw + 255) / 256), 256, 0, m->st>>>(m->P, m->W2b, m->W2T, nw);
    MX_CUDA(cudaGetLastError(), "refresh launch");
    MX_CUDA(cudaStreamSynchronize(m->st), "parameter upload synchronize");
    return CX_OK;
}

int cx_mlp_get_params(cx_mlp *m, float *host, size_t count)
{
    if (!m || !host) return mfail(CX_ERR_INVALID_ARG, "NULL argument");
    const size_t n = (size_t)m->E * NPARAM;
    if (count != n) return mfail(CX_ERR_INVALID_ARG, "count != members x CX_MLP_PARAMS");
    MX_CUDA(cudaMemcpyAsync(host, m->P, n * 4, cudaMemcpyDeviceToHost, m->st), "parameter download");
    MX_CUDA(cudaStreamSynchronize(m->st), "parameter download synchronize");
    return CX_OK;
}

int cx_mlp_forward(cx_mlp *m, const float *x, int32_t batch, float *y)
{
    int rc = check_batch_arg(m, batch);
    if (rc) return rc;
    if (!x || !y) return mfail(CX_ERR_INVALID_ARG, "NULL argument");
    cx::NvtxRange range("cx_mlp_forward");
    MX_CUDA(cudaMemcpyAsync(m->X, x, (size_t)batch * NI * 4, cudaMemcpyHostToDevice, m->st), "input upload");
    MX_CUDA(run_pass(m, m->X, 0, nullptr, 0, batch, nullptr, 0), "forward launch");
    // member e's rows at y + e * batch * NO
    MX_CUDA(cudaMemcpy2DAsync(y, (size_t)batch * NO * 4, m->Y, (size_t)m->Bmax * NO * 4,
                              (size_t)batch * NO * 4, (size_t)m->E, cudaMemcpyDeviceToHost, m->st),
            "output download");
    return check_waits(m);
}

int cx_mlp_gradient(cx_mlp *m, const float *x, const float *t, int32_t batch, float *grad,
                    double *loss)
{
    int rc = check_batch_arg(m, batch);
    if (rc) return rc;
    if (!x || !t || !grad) return mfail(CX_ERR_INVALID_ARG, "NULL argument");
    MX_CUDA(cudaMemcpyAsync(m->X, x, (size_t)batch * NI * 4, cudaMemcpyHostToDevice, m->st), "input upload");
    MX_CUDA(cudaMemcpyAsync(m->T, t, (size_t)batch * NO * 4, cudaMemcpyHostToDevice, m->st), "target upload");
    MX_CUDA(run_pass(m, m->X, 0, m->T, 0, batch, m->loss, 1), "backward launch");
    MX_CUDA(cudaMemcpyAsync(grad, m->G, (size_t)m->E * NPARAM * 4, cudaMemcpyDeviceToHost, m->st),
            "gradient download");
    double l[kMaxMembers];
    MX_CUDA(cudaMemcpyAsync(l, m->loss, (size_t)m->E * 8, cudaMemcpyDeviceToHost, m->st), "loss download");
    rc = check_waits(m);
    if (rc) return rc;
    if (loss)
        for (int e = 0; e < m->E; ++e) loss[e] = l[e] / (double)batch;
    return CX_OK;
}

int cx_mlp_train(cx_mlp *m, const float *x, const float *t, int32_t n, int32_t batch,
                 int32_t steps, float lr, double *loss_out)
{
    cx::NvtxRange range("cx_mlp_train");
    int rc = check_batch_arg(m, batch);
    if (rc) return rc;
    if (!x || !t || n < batch || steps < 0 || !(lr > 0.f))
        return mfail(CX_ERR_INVALID_ARG, "need x, t, n >= batch, steps >= 0, lr > 0");
    const long long E = m->E;
    if (m->ndata != n) {
        if (m->dataX) cudaFree(m->dataX);
        if (m->dataT) cudaFree(m->dataT);
        m->dataX = m->dataT = nullptr;
        m->ndata = 0;
        MX_CUDA(cudaMalloc((void **)&m->dataX, (size_t)(E * n * NI * 4)), "training set allocation");
        MX_CUDA(cudaMalloc((void **)&m->dataT, (size_t)(E * n * NO * 4)), "training set allocation");
        m->ndata = n;
    }
    MX_CUDA(cudaMemcpyAsync(m->dataX, x, (size_t)(E * n * NI * 4), cudaMemcpyHostToDevice, m->st),
            "training set upload");
    MX_CUDA(cudaMemcpyAsync(m->dataT, t, (size_t)(E * n * NO * 4), cudaMemcpyHostToDevice, m->st),
            "training set upload");
    // the losses stay on the device until the end, so the host queues every
    // step without waiting for the GPU
    if (loss_out && m->nlosses < E * steps) {
        if (m->losses) cudaFree(m->losses);
        m->losses = nullptr;
        m->nlosses = 0;
        MX_CUDA(cudaMalloc((void **)&m->losses, (size_t)(E * steps * 8)), "loss buffer allocation");
        m->nlosses = E * steps;
    }
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    const int nbatches = n / batch;
    const long long np = E * NPARAM;
    for (int s = 0; s < steps; ++s) {
        const long long first = (long long)(s % nbatches) * batch;  // cyclic minibatches
        MX_CUDA(run_pass(m, m->dataX + first * NI, (long long)n * NI, m->dataT + first * NO,
                         (long long)n * NO, batch, loss_out ? m->losses + s : nullptr, steps),
                "training pass");
        m->adam_t += 1;
        const float c1 = 1.f - powf(b1, (float)m->adam_t), c2 = 1.f - powf(b2, (float)m->adam_t);
        adam_kernel<<<(unsigned)((np + 255) / 256), 256, 0, m->st>>>(m->P, m->G, m->M, m->V, m->W2b,
                                                                    m->W2T, np, lr, b1, b2, eps, c1, c2);
        MX_CUDA(cudaGetLastError(), "optimiser launch");
    }
    if (loss_out && steps > 0)
        MX_CUDA(cudaMemcpyAsync(loss_out, m->losses, (size_t)(E * steps * 8), cudaMemcpyDeviceToHost, m->st),
                "loss download");
    rc = check_waits(m);
    if (rc) return rc;
    if (loss_out)
        for (long long s = 0; s < E * steps; ++s) loss_out[s] /= (double)batch;
    return CX_OK;
}

}  // extern "C"
