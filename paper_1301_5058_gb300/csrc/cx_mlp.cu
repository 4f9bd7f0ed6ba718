// cx_mlp.cu -- the surrogate network: an MLP 4 -> 256 -> 256 -> 2 (tanh)
// mapping sweep parameters to morphology labels, trained on the GPU with
// its own forward and backward kernels and Adam.
//
//   Z1 = X W1^T + b1,  H1 = tanh(Z1)               (FP32, K = 4)
//   Z2 = bf(H1) bf(W2)^T + b2,  H2 = tanh(Z2)       (tensor cores, bf16 in, FP32 accumulate)
//   Y  = H2 W3^T + b3                               (FP32, N = 2)
//   loss = sum (Y - T)^2 / (2 B)
// Backward: dY = (Y - T)/B; dZ2 = (dY W3) (1 - H2^2); dW2 = bf(dZ2)^T bf(H1)
// and dH1 = bf(dZ2) bf(W2) on the tensor cores; dZ1 = dH1 (1 - H1^2); the
// bias and thin-layer gradients are column sums over the batch.
//
// The 256 x 256 products go through one kernel, C = A B^T with A (M x K)
// and B (N x K) row-major bf16, built on mma.sync.m16n8k16 (bf16 x bf16 ->
// fp32): 4 warps per 64 x 64 tile, fragments loaded straight from global
// memory (the operands are at most 256 x 8192 and live in L2).  The network
// is tiny (67,586 parameters, 0.5 GFLOP per 256 x 256 product at batch
// 1024), so these kernels are latency-bound by design; their cost is
// negligible next to the solver runs that produce the training data.
#include <cuda_bf16.h>
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <new>
#include <vector>

#include "cx_internal.h"

namespace {

constexpr int H = 256;   // hidden width
constexpr int NI = 4;    // inputs
constexpr int NO = 2;    // outputs
// flat parameter layout (FP32): W1, b1, W2, b2, W3, b3
constexpr int OFF_W1 = 0;
constexpr int OFF_B1 = OFF_W1 + H * NI;
constexpr int OFF_W2 = OFF_B1 + H;
constexpr int OFF_B2 = OFF_W2 + H * H;
constexpr int OFF_W3 = OFF_B2 + H;
constexpr int OFF_B3 = OFF_W3 + NO * H;
constexpr int NPARAM = OFF_B3 + NO;

__device__ __forceinline__ uint32_t ld_b32(const __nv_bfloat16 *p)
{
    return *reinterpret_cast<const uint32_t *>(p);
}

// C (M x N, FP32, row-major ldc) = A (M x K) * B (N x K)^T, bf16 row-major.
// M, N multiples of 64; K a multiple of 16.  mode 1: C = tanh(C + bias[n]).
__global__ void __launch_bounds__(128)
    gemm_bf16_nt(const __nv_bfloat16 *__restrict__ A, int lda, const __nv_bfloat16 *__restrict__ B,
                 int ldb, float *__restrict__ C, int ldc, int K, const float *__restrict__ bias,
                 int mode)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int g = lane >> 2, t = lane & 3;
    const int m0 = blockIdx.y * 64 + (warp >> 1) * 32;  // warp tile 32 x 32
    const int n0 = blockIdx.x * 64 + (warp & 1) * 32;
    float acc[2][4][4];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int r = 0; r < 4; ++r) acc[i][j][r] = 0.f;
    for (int k0 = 0; k0 < K; k0 += 16) {
        uint32_t a[2][4], b[4][2];
#pragma unroll
        for (int i = 0; i < 2; ++i) {
            const __nv_bfloat16 *pa = A + (long long)(m0 + 16 * i + g) * lda + k0 + 2 * t;
            a[i][0] = ld_b32(pa);                        // row g,   k 2t..2t+1
            a[i][1] = ld_b32(pa + 8LL * lda);            // row g+8, k 2t..2t+1
            a[i][2] = ld_b32(pa + 8);                    // row g,   k 2t+8..
            a[i][3] = ld_b32(pa + 8LL * lda + 8);        // row g+8, k 2t+8..
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const __nv_bfloat16 *pb = B + (long long)(n0 + 8 * j + g) * ldb + k0 + 2 * t;
            b[j][0] = ld_b32(pb);                        // k 2t..2t+1,   n g
            b[j][1] = ld_b32(pb + 8);                    // k 2t+8..2t+9, n g
        }
#pragma unroll
        for (int i = 0; i < 2; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j)
                asm volatile(
                    "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
                    "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
                    : "+f"(acc[i][j][0]), "+f"(acc[i][j][1]), "+f"(acc[i][j][2]), "+f"(acc[i][j][3])
                    : "r"(a[i][0]), "r"(a[i][1]), "r"(a[i][2]), "r"(a[i][3]), "r"(b[j][0]),
                      "r"(b[j][1]));
    }
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int h = 0; h < 2; ++h) {  // rows g and g+8
                const int row = m0 + 16 * i + g + 8 * h;
                const int col = n0 + 8 * j + 2 * t;
                float v0 = acc[i][j][2 * h], v1 = acc[i][j][2 * h + 1];
                if (mode == 1) {
                    v0 = tanhf(v0 + bias[col]);
                    v1 = tanhf(v1 + bias[col + 1]);
                }
                *reinterpret_cast<float2 *>(C + (long long)row * ldc + col) = make_float2(v0, v1);
            }
}

// H1 = tanh(X W1^T + b1) for rows < nb (padding rows: 0), in FP32 and bf16,
// row-major (Bp x 256) and transposed (256 x Bp).
__global__ void layer1(const float *__restrict__ X, const float *__restrict__ P, int nb, int Bp,
                       float *__restrict__ H1f, __nv_bfloat16 *__restrict__ H1b,
                       __nv_bfloat16 *__restrict__ H1T)
{
    const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (e >= (long long)Bp * H) return;
    const int b = (int)(e / H), j = (int)(e % H);
    float h = 0.f;
    if (b < nb) {
        float z = P[OFF_B1 + j];
#pragma unroll
        for (int k = 0; k < NI; ++k) z += P[OFF_W1 + j * NI + k] * X[b * NI + k];
        h = tanhf(z);
    }
    H1f[e] = h;
    const __nv_bfloat16 hb = __float2bfloat16_rn(h);
    H1b[e] = hb;
    H1T[(long long)j * Bp + b] = hb;
}

// Y = H2 W3^T + b3 and dY = (Y - T) / nb for rows < nb; per-row loss terms.
__global__ void output_layer(const float *__restrict__ H2, const float *__restrict__ P,
                             const float *__restrict__ T, int nb, int Bp, float *__restrict__ Y,
                             float *__restrict__ dY, double *__restrict__ lrow)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= Bp) return;
    float y[NO], d[NO];
    double l = 0.0;
#pragma unroll
    for (int o = 0; o < NO; ++o) {
        float s = P[OFF_B3 + o];
        for (int j = 0; j < H; ++j) s += P[OFF_W3 + o * H + j] * H2[(long long)b * H + j];
        y[o] = s;
        d[o] = 0.f;
        if (b < nb && T) {
            const float r = s - T[b * NO + o];
            d[o] = r / (float)nb;
            l += 0.5 * (double)r * (double)r;
        }
        Y[b * NO + o] = y[o];
        dY[b * NO + o] = d[o];
    }
    lrow[b] = l;
}

// dZ2 = (dY W3) (1 - H2^2), as FP32 and as bf16 row-major and transposed.
__global__ void back_hidden2(const float *__restrict__ dY, const float *__restrict__ P,
                             const float *__restrict__ H2, int Bp, float *__restrict__ dZ2,
                             __nv_bfloat16 *__restrict__ dZ2b, __nv_bfloat16 *__restrict__ dZ2T)
{
    const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (e >= (long long)Bp * H) return;
    const int b = (int)(e / H), j = (int)(e % H);
    float s = 0.f;
#pragma unroll
    for (int o = 0; o < NO; ++o) s += dY[b * NO + o] * P[OFF_W3 + o * H + j];
    const float h = H2[e];
    const float v = s * (1.f - h * h);
    dZ2[e] = v;
    const __nv_bfloat16 vb = __float2bfloat16_rn(v);
    dZ2b[e] = vb;
    dZ2T[(long long)j * Bp + b] = vb;
}

// Column sums over the nb valid rows (padding rows carry zero gradients)
// in thread j: dW3, db2, dW1, db1 with dZ1 = dH1 (1 - H1^2); threads 0..1
// also db3, thread 0 the loss.
__global__ void __launch_bounds__(256)
    column_sums(const float *__restrict__ X, const float *__restrict__ H1f,
                const float *__restrict__ H2, const float *__restrict__ dY,
                const float *__restrict__ dZ2, const float *__restrict__ dH1,
                const double *__restrict__ lrow, int nb, float *__restrict__ G,
                double *__restrict__ loss)
{
    const int j = threadIdx.x;
    float w3[NO] = {0.f, 0.f}, b2 = 0.f, w1[NI] = {0.f, 0.f, 0.f, 0.f}, b1 = 0.f;
    for (int b = 0; b < nb; ++b) {
        const long long e = (long long)b * H + j;
        const float h2 = H2[e], h1 = H1f[e];
#pragma unroll
        for (int o = 0; o < NO; ++o) w3[o] += dY[b * NO + o] * h2;
        b2 += dZ2[e];
        const float dz1 = dH1[e] * (1.f - h1 * h1);
        b1 += dz1;
#pragma unroll
        for (int k = 0; k < NI; ++k) w1[k] += dz1 * X[b * NI + k];
    }
#pragma unroll
    for (int o = 0; o < NO; ++o) G[OFF_W3 + o * H + j] = w3[o];
    G[OFF_B2 + j] = b2;
#pragma unroll
    for (int k = 0; k < NI; ++k) G[OFF_W1 + j * NI + k] = w1[k];
    G[OFF_B1 + j] = b1;
    if (j < NO) {
        float s = 0.f;
        for (int b = 0; b < nb; ++b) s += dY[b * NO + j];
        G[OFF_B3 + j] = s;
    }
    if (j == 0) {
        double l = 0.0;
        for (int b = 0; b < nb; ++b) l += lrow[b];
        *loss = l;
    }
}

// Adam (Kingma & Ba, 2015) on the FP32 master parameters.
__global__ void adam(float *__restrict__ P, const float *__restrict__ G, float *__restrict__ M,
                     float *__restrict__ V, int n, float lr, float b1, float b2, float eps,
                     float c1, float c2)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float g = G[i];
    const float m = b1 * M[i] + (1.f - b1) * g;
    const float v = b2 * V[i] + (1.f - b2) * g * g;
    M[i] = m;
    V[i] = v;
    P[i] -= lr * (m / c1) / (sqrtf(v / c2) + eps);
}

// bf16 copies of W2 (row-major) and W2^T.
__global__ void refresh_w2(const float *__restrict__ P, __nv_bfloat16 *__restrict__ W2b,
                           __nv_bfloat16 *__restrict__ W2T)
{
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= H * H) return;
    const int r = e / H, c = e % H;
    const __nv_bfloat16 w = __float2bfloat16_rn(P[OFF_W2 + e]);
    W2b[e] = w;
    W2T[c * H + r] = w;
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
    int Bmax = 0;  // padded batch capacity (multiple of 64)
    float *P = nullptr, *G = nullptr, *M = nullptr, *V = nullptr;
    __nv_bfloat16 *W2b = nullptr, *W2T = nullptr;
    float *X = nullptr, *T = nullptr, *H1f = nullptr, *H2 = nullptr, *Y = nullptr, *dY = nullptr;
    float *dZ2 = nullptr, *dH1 = nullptr;
    __nv_bfloat16 *H1b = nullptr, *H1T = nullptr, *dZ2b = nullptr, *dZ2T = nullptr;
    double *lrow = nullptr, *loss = nullptr;
    float *dataX = nullptr, *dataT = nullptr;  // training set on the device
    int ndata = 0;
    double *losses = nullptr;  // per-step losses of a training call, on the device
    int nlosses = 0;
    long long adam_t = 0;
    cudaStream_t st = nullptr;
};

namespace {

void free_mlp(cx_mlp *m)
{
    if (!m) return;
    void *ptrs[] = {m->P, m->G, m->M, m->V, m->W2b, m->W2T, m->X, m->T, m->H1f, m->H2, m->Y, m->dY,
                    m->dZ2, m->dH1, m->H1b, m->H1T, m->dZ2b, m->dZ2T, m->lrow, m->loss,
                    m->dataX, m->dataT, m->losses};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    if (m->st) cudaStreamDestroy(m->st);
    delete m;
}

int pad64(int b) { return (b + 63) / 64 * 64; }

// Forward (and, with T, backward into m->G) of rows X[0..nb) already on the device.
cudaError_t run_pass(cx_mlp *m, const float *X, const float *T, int nb, bool backward)
{
    const int Bp = pad64(nb);
    const long long elems = (long long)Bp * H;
    const int tb = 256;
    const int eg = (int)((elems + tb - 1) / tb);
    layer1<<<eg, tb, 0, m->st>>>(X, m->P, nb, Bp, m->H1f, m->H1b, m->H1T);
    gemm_bf16_nt<<<dim3(H / 64, Bp / 64), 128, 0, m->st>>>(m->H1b, H, m->W2b, H, m->H2, H, H,
                                                           m->P + OFF_B2, 1);
    output_layer<<<(Bp + 127) / 128, 128, 0, m->st>>>(m->H2, m->P, T, nb, Bp, m->Y, m->dY, m->lrow);
    if (!backward) return cudaGetLastError();
    back_hidden2<<<eg, tb, 0, m->st>>>(m->dY, m->P, m->H2, Bp, m->dZ2, m->dZ2b, m->dZ2T);
    // dH1 = dZ2 W2 (B x 256): A = dZ2 (Bp x 256), B operand = W2^T rows
    gemm_bf16_nt<<<dim3(H / 64, Bp / 64), 128, 0, m->st>>>(m->dZ2b, H, m->W2T, H, m->dH1, H, H,
                                                           nullptr, 0);
    // dW2 = dZ2^T H1 (256 x 256): A = dZ2^T (256 x Bp), B operand = H1^T (256 x Bp)
    gemm_bf16_nt<<<dim3(H / 64, H / 64), 128, 0, m->st>>>(m->dZ2T, Bp, m->H1T, Bp, m->G + OFF_W2, H,
                                                          Bp, nullptr, 0);
    column_sums<<<1, H, 0, m->st>>>(X, m->H1f, m->H2, m->dY, m->dZ2, m->dH1, m->lrow, nb, m->G,
                                    m->loss);
    return cudaGetLastError();
}

int check_batch_arg(cx_mlp *m, int nb)
{
    if (!m) return mfail(CX_ERR_INVALID_ARG, "NULL network");
    if (nb < 1 || pad64(nb) > m->Bmax) return mfail(CX_ERR_INVALID_ARG, "batch outside 1..max_batch");
    return CX_OK;
}

}  // namespace

extern "C" {

int cx_mlp_create(int32_t max_batch, cx_mlp **out)
{
    if (!out) return mfail(CX_ERR_INVALID_ARG, "out must not be NULL");
    *out = nullptr;
    if (max_batch < 1 || max_batch > (1 << 20)) return mfail(CX_ERR_INVALID_ARG, "max_batch outside 1..2^20");
    cx_mlp *m = new (std::nothrow) cx_mlp;
    if (!m) return mfail(CX_ERR_OOM, "host allocation");
    m->Bmax = pad64(max_batch);
    const size_t Bp = (size_t)m->Bmax;
    cudaError_t e = cudaStreamCreateWithFlags(&m->st, cudaStreamNonBlocking);
    auto A = [&](void **p, size_t bytes) {
        if (e == cudaSuccess) e = cudaMalloc(p, bytes);
        if (e == cudaSuccess) e = cudaMemset(*p, 0, bytes);
    };
    A((void **)&m->P, NPARAM * 4); A((void **)&m->G, NPARAM * 4);
    A((void **)&m->M, NPARAM * 4); A((void **)&m->V, NPARAM * 4);
    A((void **)&m->W2b, H * H * 2); A((void **)&m->W2T, H * H * 2);
    A((void **)&m->X, Bp * NI * 4); A((void **)&m->T, Bp * NO * 4);
    A((void **)&m->H1f, Bp * H * 4); A((void **)&m->H2, Bp * H * 4);
    A((void **)&m->Y, Bp * NO * 4); A((void **)&m->dY, Bp * NO * 4);
    A((void **)&m->dZ2, Bp * H * 4); A((void **)&m->dH1, Bp * H * 4);
    A((void **)&m->H1b, Bp * H * 2); A((void **)&m->H1T, Bp * H * 2);
    A((void **)&m->dZ2b, Bp * H * 2); A((void **)&m->dZ2T, Bp * H * 2);
    A((void **)&m->lrow, Bp * 8); A((void **)&m->loss, 8);
    if (e != cudaSuccess) {
        cudaGetLastError();
        free_mlp(m);
        return mcuda(e, "network allocation");
    }
    *out = m;
    return CX_OK;
}

void cx_mlp_destroy(cx_mlp *m)
{
    if (m && m->st) cudaStreamSynchronize(m->st);
    free_mlp(m);
}

int cx_mlp_set_params(cx_mlp *m, const float *host, size_t count)
{
    if (!m || !host) return mfail(CX_ERR_INVALID_ARG, "NULL argument");
    if (count != (size_t)NPARAM) return mfail(CX_ERR_INVALID_ARG, "count != CX_MLP_PARAMS");
    MX_CUDA(cudaMemcpyAsync(m->P, host, NPARAM * 4, cudaMemcpyHostToDevice, m->st), "parameter upload");
    MX_CUDA(cudaMemsetAsync(m->M, 0, NPARAM * 4, m->st), "adam reset");
    MX_CUDA(cudaMemsetAsync(m->V, 0, NPARAM * 4, m->st), "adam reset");
    m->adam_t = 0;
    refresh_w2<<<(H * H + 255) / 256, 256, 0, m->st>>>(m->P, m->W2b, m->W2T);
    MX_CUDA(cudaGetLastError(), "refresh launch");
    MX_CUDA(cudaStreamSynchronize(m->st), "parameter upload synchronize");
    return CX_OK;
}

int cx_mlp_get_params(cx_mlp *m, float *host, size_t count)
{
    if (!m || !host) return mfail(CX_ERR_INVALID_ARG, "NULL argument");
    if (count != (size_t)NPARAM) return mfail(CX_ERR_INVALID_ARG, "count != CX_MLP_PARAMS");
    MX_CUDA(cudaMemcpyAsync(host, m->P, NPARAM * 4, cudaMemcpyDeviceToHost, m->st), "parameter download");
    MX_CUDA(cudaStreamSynchronize(m->st), "parameter download synchronize");
    return CX_OK;
}

int cx_mlp_forward(cx_mlp *m, const float *x, int32_t batch, float *y)
{
    int rc = check_batch_arg(m, batch);
    if (rc) return rc;
    if (!x || !y) return mfail(CX_ERR_INVALID_ARG, "NULL argument");
    MX_CUDA(cudaMemcpyAsync(m->X, x, (size_t)batch * NI * 4, cudaMemcpyHostToDevice, m->st), "input upload");
    MX_CUDA(run_pass(m, m->X, nullptr, batch, false), "forward launch");
    MX_CUDA(cudaMemcpyAsync(y, m->Y, (size_t)batch * NO * 4, cudaMemcpyDeviceToHost, m->st), "output download");
    MX_CUDA(cudaStreamSynchronize(m->st), "forward synchronize");
    return CX_OK;
}

int cx_mlp_gradient(cx_mlp *m, const float *x, const float *t, int32_t batch, float *grad,
                    double *loss)
{
    int rc = check_batch_arg(m, batch);
    if (rc) return rc;
    if (!x || !t || !grad) return mfail(CX_ERR_INVALID_ARG, "NULL argument");
    MX_CUDA(cudaMemcpyAsync(m->X, x, (size_t)batch * NI * 4, cudaMemcpyHostToDevice, m->st), "input upload");
    MX_CUDA(cudaMemcpyAsync(m->T, t, (size_t)batch * NO * 4, cudaMemcpyHostToDevice, m->st), "target upload");
    MX_CUDA(run_pass(m, m->X, m->T, batch, true), "backward launch");
    MX_CUDA(cudaMemcpyAsync(grad, m->G, NPARAM * 4, cudaMemcpyDeviceToHost, m->st), "gradient download");
    double l = 0.0;
    MX_CUDA(cudaMemcpyAsync(&l, m->loss, 8, cudaMemcpyDeviceToHost, m->st), "loss download");
    MX_CUDA(cudaStreamSynchronize(m->st), "gradient synchronize");
    if (loss) *loss = l / (double)batch;
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
    if (m->ndata != n) {
        if (m->dataX) cudaFree(m->dataX);
        if (m->dataT) cudaFree(m->dataT);
        m->dataX = m->dataT = nullptr;
        m->ndata = 0;
        MX_CUDA(cudaMalloc((void **)&m->dataX, (size_t)n * NI * 4), "training set allocation");
        MX_CUDA(cudaMalloc((void **)&m->dataT, (size_t)n * NO * 4), "training set allocation");
        m->ndata = n;
    }
    MX_CUDA(cudaMemcpyAsync(m->dataX, x, (size_t)n * NI * 4, cudaMemcpyHostToDevice, m->st), "training set upload");
    MX_CUDA(cudaMemcpyAsync(m->dataT, t, (size_t)n * NO * 4, cudaMemcpyHostToDevice, m->st), "training set upload");
    // the losses stay on the device until the end, so the host queues every
    // step without waiting for the GPU
    if (loss_out && m->nlosses < steps) {
        if (m->losses) cudaFree(m->losses);
        m->losses = nullptr;
        m->nlosses = 0;
        MX_CUDA(cudaMalloc((void **)&m->losses, (size_t)steps * 8), "loss buffer allocation");
        m->nlosses = steps;
    }
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    const int nbatches = n / batch;
    for (int s = 0; s < steps; ++s) {
        const long long first = (long long)(s % nbatches) * batch;  // cyclic minibatches
        MX_CUDA(run_pass(m, m->dataX + first * NI, m->dataT + first * NO, batch, true), "training pass");
        m->adam_t += 1;
        const float c1 = 1.f - powf(b1, (float)m->adam_t), c2 = 1.f - powf(b2, (float)m->adam_t);
        adam<<<(NPARAM + 255) / 256, 256, 0, m->st>>>(m->P, m->G, m->M, m->V, NPARAM, lr, b1, b2, eps, c1, c2);
        refresh_w2<<<(H * H + 255) / 256, 256, 0, m->st>>>(m->P, m->W2b, m->W2T);
        MX_CUDA(cudaGetLastError(), "optimiser launch");
        if (loss_out)
            MX_CUDA(cudaMemcpyAsync(m->losses + s, m->loss, 8, cudaMemcpyDeviceToDevice, m->st),
                    "loss record");
    }
    if (loss_out && steps > 0)
        MX_CUDA(cudaMemcpyAsync(loss_out, m->losses, (size_t)steps * 8, cudaMemcpyDeviceToHost, m->st),
                "loss download");
    MX_CUDA(cudaStreamSynchronize(m->st), "training synchronize");
    if (loss_out)
        for (int s = 0; s < steps; ++s) loss_out[s] /= (double)batch;
    return CX_OK;
}

}  // extern "C"
