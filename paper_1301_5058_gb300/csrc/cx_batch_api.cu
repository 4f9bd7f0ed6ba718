// cx_batch_api.cu -- the cx_batch_* entry points (include/cx.h): a set of
// independent simulations (one parameter sweep) stepped together by the
// batched kernels of cx_batch.cu.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <new>
#include <vector>

#include "cx_internal.h"

namespace {

int bfail(int code, const char *msg) { return cx::record_error(code, msg); }

int bcuda(cudaError_t e, const char *what)
{
    char buf[300];
    snprintf(buf, sizeof buf, "%s: %s", what, cudaGetErrorString(e));
    return cx::record_error(e == cudaErrorMemoryAllocation ? CX_ERR_OOM : CX_ERR_CUDA, buf);
}

#define BX_CUDA(call, what)                                  \
    do {                                                     \
        cudaError_t e_ = (call);                             \
        if (e_ != cudaSuccess) return bcuda(e_, (what));     \
    } while (0)

constexpr int kTileCols = 512;       // columns per tile (128 threads x 4 cells)
constexpr int kFusedTileCols = 120;  // written columns per (one-warp) tile of the two-stage march
constexpr int kDiagBlocksPerInst = 64;

size_t round_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

}  // namespace

struct cx_batch {
    int count = 0, prec = 0, law = 0, mob = 0, scheme = 0;
    int noise = 0;                  // 1: sigma redrawn every step (CX_NOISE_PER_STEP)
    long long *d_step = nullptr;    // time step the next pass starts from (noise == 1)
    std::vector<cx_grid> g;
    std::vector<cx_params> p;
    std::vector<uint64_t> seed;
    std::vector<double> dt;
    std::vector<long long> pitch;
    std::vector<void *> fb[2], fn[2], fs;
    std::vector<long long> footprint;  // device bytes of each instance's fields
    void *arena = nullptr;
    size_t elem = 4;
    void *d_inst = nullptr;
    std::vector<unsigned char> h_inst;
    int4 *d_work = nullptr;       // 512-column tiles (one stage per pass)
    std::vector<int> work_begin;  // first work item of each instance (+ total)
    int4 *d_work2 = nullptr;      // 120-column tiles (two stages per pass)
    std::vector<int> work2_begin;
    int rows = 32;
    int graph_steps = 64;
    long long group_bytes = 0;
    int time_block = 1;             // explicit stages per pass (1 or 2)
    std::vector<int> group_first;  // instance index where each group starts (+ count)
    std::vector<cudaGraphExec_t> gexec[2];  // per group, by starting parity
    std::vector<int> gend[2];               // parity after that graph
    int resident_steps = 0;         // > 0: steps per cooperative launch of a group
    void *d_barrier = nullptr;      // grid barrier state of the resident kernel
    long long spin_limit = 1 << 22; // polls before a barrier wait gives up
    int cur = 0;
    int64_t step = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    double *d_part = nullptr, *d_res = nullptr, *h_res = nullptr;
};

namespace {

void drop_graphs(cx_batch *B)
{
    for (int p = 0; p < 2; ++p) {
        for (auto &e : B->gexec[p])
            if (e) cudaGraphExecDestroy(e);
        B->gexec[p].clear();
        B->gend[p].clear();
    }
}

void free_batch(cx_batch *B)
{
    if (!B) return;
    if (B->stream) cudaStreamSynchronize(B->stream);
    drop_graphs(B);
    if (B->arena) cudaFree(B->arena);
    if (B->d_inst) cudaFree(B->d_inst);
    if (B->d_work) cudaFree(B->d_work);
    if (B->d_work2) cudaFree(B->d_work2);
    if (B->d_part) cudaFree(B->d_part);
    if (B->d_res) cudaFree(B->d_res);
    if (B->h_res) cudaFreeHost(B->h_res);
    if (B->d_barrier) cudaFree(B->d_barrier);
    if (B->d_step) cudaFree(B->d_step);
    if (B->own_stream && B->stream) cudaStreamDestroy(B->stream);
    delete B;
}

// Tile work lists for the current tile height, instance by instance: the
// one-stage march's 512-column tiles and the two-stage march's 120-column
// tiles.
int build_work(cx_batch *B)
{
    for (int f = 0; f < 2; ++f) {
        const int cols = f ? kFusedTileCols : kTileCols;
        std::vector<int> &begin = f ? B->work2_begin : B->work_begin;
        int4 *&d = f ? B->d_work2 : B->d_work;
        std::vector<int4> w;
        begin.assign(B->count + 1, 0);
        for (int i = 0; i < B->count; ++i) {
            begin[i] = (int)w.size();
            const int tx = (B->g[i].nx + cols - 1) / cols;
            const int ty = (B->g[i].ny + B->rows - 1) / B->rows;
            for (int y = 0; y < ty; ++y)
                for (int x = 0; x < tx; ++x) w.push_back(make_int4(i, x, y, 0));
        }
        begin[B->count] = (int)w.size();
        if (d) cudaFree(d);
        d = nullptr;
        BX_CUDA(cudaMalloc((void **)&d, w.size() * sizeof(int4)), "work list allocation");
        BX_CUDA(cudaMemcpy(d, w.data(), w.size() * sizeof(int4), cudaMemcpyHostToDevice),
                "work list upload");
    }
    return CX_OK;
}

// Consecutive groups of instances whose fields fit group_bytes (one group
// with every instance when group_bytes == 0; an instance larger than the
// budget forms a group of its own).
void build_groups(cx_batch *B)
{
    B->group_first.clear();
    long long acc = 0;
    for (int i = 0; i < B->count; ++i) {
        if (i == 0 || (B->group_bytes > 0 && acc + B->footprint[i] > B->group_bytes)) {
            B->group_first.push_back(i);
            acc = 0;
        }
        acc += B->footprint[i];
    }
    B->group_first.push_back(B->count);
}

// The noise argument of a pass whose first time step is step_off after the
// step last written to d_step.
cx::BatchNoise pass_noise(const cx_batch *B, int step_off)
{
    return cx::BatchNoise{B->noise, B->d_step, step_off};
}

// Before the passes (or the graph) that start at time step `step`: where the
// per-step noise reads its step from.
cudaError_t mark_step(cx_batch *B, int64_t step)
{
    return B->noise ? cx::launch_set_step(B->d_step, (long long)step, B->stream) : cudaSuccess;
}

// One time step of instances [i0, i1) at the given parity, step_off steps
// after the marked step.
cudaError_t one_step(cx_batch *B, int i0, int i1, int parity, int step_off)
{
    const int w0 = B->work_begin[i0], w1 = B->work_begin[i1];
    const int4 *work = B->d_work + w0;
    const cx::BatchNoise nz = pass_noise(B, step_off);
    cudaError_t e = cx::launch_batch_step(B->prec, B->law, B->mob, B->d_inst, work, w1 - w0,
                                          parity, B->rows, 0, nz, B->stream);
    if (e == cudaSuccess && B->scheme == CX_SCHEME_HEUN)
        e = cx::launch_batch_step(B->prec, B->law, B->mob, B->d_inst, work, w1 - w0, parity,
                                  B->rows, 1, nz, B->stream);
    return e;
}

int next_parity(const cx_batch *B, int parity) { return B->scheme == CX_SCHEME_HEUN ? parity : parity ^ 1; }

// One pass over instances [i0, i1) starting at *parity, step_off steps
// after the marked step: two stages when the depth is 2 (two Euler steps if
// at least two are left, or one Heun step), else one step.  Sets *steps to
// the time steps taken and *parity to the parity after them.
cudaError_t one_pass(cx_batch *B, int i0, int i1, int *parity, int64_t left, int step_off,
                     int *steps)
{
    const bool heun = B->scheme == CX_SCHEME_HEUN;
    if (B->time_block == 2 && (heun || left >= 2)) {
        const int w0 = B->work2_begin[i0], w1 = B->work2_begin[i1];
        const cudaError_t e = cx::launch_batch_fused(B->prec, B->law, B->mob, B->d_inst,
                                                     B->d_work2 + w0, w1 - w0, *parity, B->rows,
                                                     heun ? 1 : 0, pass_noise(B, step_off),
                                                     B->stream);
        *parity ^= 1;
        *steps = heun ? 1 : 2;
        return e;
    }
    const cudaError_t e = one_step(B, i0, i1, *parity, step_off);
    *parity = next_parity(B, *parity);
    *steps = 1;
    return e;
}

// Capture graph_steps steps of group gi starting at `parity`; *end gets the
// parity after them (a graph is kept per starting parity).
int capture_group(cx_batch *B, int gi, int parity, cudaGraphExec_t *out, int *end)
{
    cudaGraph_t graph = nullptr;
    BX_CUDA(cudaStreamBeginCapture(B->stream, cudaStreamCaptureModeThreadLocal), "graph capture begin");
    cudaError_t e = cudaSuccess;
    int par = parity;
    for (int64_t left = B->graph_steps; left > 0 && e == cudaSuccess;) {
        int taken = 1;
        e = one_pass(B, B->group_first[gi], B->group_first[gi + 1], &par, left,
                     (int)(B->graph_steps - left), &taken);
        left -= taken;
    }
    cudaError_t e2 = cudaStreamEndCapture(B->stream, &graph);
    if (e != cudaSuccess) return bcuda(e, "launch during graph capture");
    if (e2 != cudaSuccess) return bcuda(e2, "graph capture end");
    e = cudaGraphInstantiate(out, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return bcuda(e, "graph instantiate");
    *end = par;
    return CX_OK;
}

int check_batch(const cx_batch *B)
{
    if (!B) return bfail(CX_ERR_INVALID_ARG, "NULL batch");
    return CX_OK;
}

// After the stream has drained: did a resident launch's barrier wait run
// out?  The flag is cleared once reported.
int check_barrier(cx_batch *B)
{
    int err = 0;
    BX_CUDA(cudaMemcpy(&err, (char *)B->d_barrier + 8, sizeof err, cudaMemcpyDeviceToHost),
            "barrier flag read");
    if (err) {
        BX_CUDA(cudaMemset((char *)B->d_barrier + 8, 0, sizeof err), "barrier flag reset");
        return bfail(CX_ERR_TIMEOUT, "a grid barrier wait of the resident batch kernel ran out; "
                                     "the batch state is undefined");
    }
    return CX_OK;
}

// `left` steps of instances [i0, i1), the first of them time step `step`,
// by cooperative launches of resident_steps steps each; returns the parity
// after them.
int run_resident(cx_batch *B, int i0, int i1, int par, int64_t left, int64_t step, int *par_out)
{
    const int w0 = B->work_begin[i0], w1 = B->work_begin[i1];
    while (left > 0) {
        const int chunk = (int)(left < B->resident_steps ? left : B->resident_steps);
        BX_CUDA(cudaMemsetAsync(B->d_barrier, 0, 8, B->stream), "barrier reset");
        BX_CUDA(mark_step(B, step), "step mark");
        BX_CUDA(cx::launch_batch_resident(B->prec, B->law, B->mob, B->d_inst, B->d_work + w0, w1 - w0,
                                          par, B->rows, chunk, B->scheme == CX_SCHEME_HEUN,
                                          B->d_barrier, B->spin_limit, pass_noise(B, 0), B->stream),
                "resident batch launch");
        step += chunk;
        if (B->scheme == CX_SCHEME_EULER && (chunk & 1)) par ^= 1;
        left -= chunk;
    }
    *par_out = par;
    return CX_OK;
}

}  // namespace

extern "C" {

int cx_batch_create(int32_t count, const cx_grid *grids, const cx_params *params,
                    const uint64_t *seeds, cx_batch **out)
{
    if (!out) return bfail(CX_ERR_INVALID_ARG, "out must not be NULL");
    *out = nullptr;
    if (count < 1 || count > 65535) return bfail(CX_ERR_INVALID_ARG, "count must lie in 1..65535");
    if (!grids || !params || !seeds) return bfail(CX_ERR_INVALID_ARG, "grids, params and seeds must not be NULL");
    for (int i = 0; i < count; ++i) {
        int rc = cx::validate_params(&grids[i], &params[i]);
        if (rc) return rc;
        const cx_params &a = params[i], &z = params[0];
        if (a.precision != z.precision || a.scheme != z.scheme || a.chemo_law != z.chemo_law ||
            a.mobility != z.mobility || a.noise_mode != z.noise_mode)
            return bfail(CX_ERR_INVALID_ARG, "all instances of a batch must share precision, "
                                             "scheme, chemo_law, mobility and noise_mode");
    }
    cx_batch *B = new (std::nothrow) cx_batch;
    if (!B) return bfail(CX_ERR_OOM, "host allocation of the batch failed");
    B->count = count;
    B->prec = params[0].precision;
    B->law = params[0].chemo_law;
    B->mob = params[0].mobility;
    B->scheme = params[0].scheme;
    B->noise = params[0].noise_mode == CX_NOISE_PER_STEP ? 1 : 0;
    B->time_block = B->prec == CX_PREC_F32 ? 2 : 1;  // as a single grid
    // Two stages per pass recompute 4 halo rows per tile: 128-row tiles keep
    // that to 3 % (1024 instances of 1024^2: 5.6e11 cell-updates/s against
    // 4.6e11 with 32-row tiles; 64 to 256 rows within 2 % of the best)
    B->rows = B->time_block == 2 ? 128 : 32;
    B->elem = B->prec == CX_PREC_F64 ? sizeof(double) : sizeof(float);
    B->g.assign(grids, grids + count);
    B->p.assign(params, params + count);
    B->seed.assign(seeds, seeds + count);
    B->dt.resize(count);
    for (int i = 0; i < count; ++i) {
        int rc = cx::resolve_time_step(&grids[i], &params[i], &B->dt[i]);
        if (rc) { free_batch(B); return rc; }
    }
    // arena layout
    const long long align = 128 / (long long)B->elem;
    std::vector<size_t> off(5 * (size_t)count);
    size_t total = 0;
    B->pitch.resize(count);
    B->footprint.resize(count);
    for (int i = 0; i < count; ++i) {
        B->pitch[i] = ((long long)grids[i].nx + align - 1) / align * align;
        const size_t bytes = round_up((size_t)B->pitch[i] * grids[i].ny * B->elem, 256);
        for (int a = 0; a < 5; ++a) {
            off[5 * i + a] = total;
            total += bytes;
        }
        B->footprint[i] = (long long)(5 * bytes);
    }
    cudaError_t e = cudaStreamCreateWithFlags(&B->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) { free_batch(B); return bcuda(e, "stream creation"); }
    B->own_stream = true;
    e = cudaMalloc(&B->arena, total);
    if (e == cudaSuccess) e = cudaMemset(B->arena, 0, total);
    if (e != cudaSuccess) { cudaGetLastError(); free_batch(B); return bcuda(e, "arena allocation"); }
    for (int q = 0; q < 2; ++q) {
        B->fb[q].resize(count);
        B->fn[q].resize(count);
    }
    B->fs.resize(count);
    char *base = (char *)B->arena;
    for (int i = 0; i < count; ++i) {
        B->fb[0][i] = base + off[5 * i + 0];
        B->fb[1][i] = base + off[5 * i + 1];
        B->fn[0][i] = base + off[5 * i + 2];
        B->fn[1][i] = base + off[5 * i + 3];
        B->fs[i] = base + off[5 * i + 4];
    }
    // instance table
    const size_t isz = cx::inst_dev_bytes(B->prec);
    B->h_inst.assign(isz * count, 0);
    for (int i = 0; i < count; ++i)
        cx::fill_inst(B->prec, B->h_inst.data(), i, B->fb[0][i], B->fb[1][i], B->fn[0][i],
                      B->fn[1][i], B->fs[i], grids[i].nx, grids[i].ny, B->pitch[i],
                      cx::make_coef(grids[i], params[i], B->dt[i]), cx::envelope_level(params[i]),
                      seeds[i], params[i].sigma0, params[i].noise_amp, params[i].noise_dist);
    e = cudaMalloc(&B->d_inst, B->h_inst.size());
    if (e == cudaSuccess) e = cudaMemcpy(B->d_inst, B->h_inst.data(), B->h_inst.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMalloc((void **)&B->d_part, 8 * sizeof(double) * (size_t)count * kDiagBlocksPerInst);
    if (e == cudaSuccess) e = cudaMalloc((void **)&B->d_res, 8 * sizeof(double) * (size_t)count);
    if (e == cudaSuccess) e = cudaMallocHost((void **)&B->h_res, 8 * sizeof(double) * (size_t)count);
    if (e == cudaSuccess) e = cudaMalloc(&B->d_barrier, cx::grid_barrier_bytes());
    if (e == cudaSuccess) e = cudaMemset(B->d_barrier, 0, cx::grid_barrier_bytes());
    if (e == cudaSuccess && B->noise) e = cudaMalloc((void **)&B->d_step, sizeof(long long));
    if (e == cudaSuccess && B->noise) e = cudaMemset(B->d_step, 0, sizeof(long long));
    if (e != cudaSuccess) { cudaGetLastError(); free_batch(B); return bcuda(e, "batch tables"); }
    if (const char *s = getenv("CX_BARRIER_SPIN_LIMIT")) B->spin_limit = atoll(s);
    int rc = build_work(B);
    if (rc) { free_batch(B); return rc; }
    build_groups(B);
    // initial state of every instance
    for (int i = 0; i < count && e == cudaSuccess; ++i) {
        const cx_params &a = params[i];
        e = cx::launch_sigma_init(B->prec, B->fs[i], grids[i].nx, grids[i].ny, B->pitch[i], seeds[i],
                                  0, a.sigma0, a.noise_amp, a.noise_dist, 0, B->stream);
        if (e == cudaSuccess)
            e = cx::launch_initial_state(B->prec, B->fb[0][i], B->fn[0][i], grids[i].nx, grids[i].ny,
                                         B->pitch[i], grids[i].dx, a.n0, a.bM, a.r0sq, B->stream);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(B->stream);
    if (e != cudaSuccess) { free_batch(B); return bcuda(e, "batch initialisation"); }
    *out = B;
    return CX_OK;
}

void cx_batch_destroy(cx_batch *B) { free_batch(B); }

int cx_batch_set_stream(cx_batch *B, void *stream)
{
    int rc = check_batch(B);
    if (rc) return rc;
    if (!stream) return bfail(CX_ERR_INVALID_ARG, "a batch needs a non-default stream (graph capture)");
    BX_CUDA(cudaStreamSynchronize(B->stream), "synchronize old stream");
    if (B->own_stream) cudaStreamDestroy(B->stream);
    B->own_stream = false;
    B->stream = (cudaStream_t)stream;
    return CX_OK;
}

int cx_batch_set_tuning(cx_batch *B, int32_t tile_rows, int32_t graph_steps, int64_t group_bytes,
                        int32_t resident_steps)
{
    int rc = check_batch(B);
    if (rc) return rc;
    if (tile_rows < 1 || tile_rows > 4096 || graph_steps < 0 || graph_steps > 100000 ||
        group_bytes < 0 || resident_steps < 0 || resident_steps > 1000000)
        return bfail(CX_ERR_INVALID_ARG, "tile_rows 1..4096, graph_steps 0..100000, group_bytes >= 0, "
                                         "resident_steps 0..1000000");
    BX_CUDA(cudaStreamSynchronize(B->stream), "synchronize before retuning");
    drop_graphs(B);
    const bool new_rows = tile_rows != B->rows;
    B->rows = tile_rows;
    B->graph_steps = (B->scheme == CX_SCHEME_EULER && (graph_steps & 1)) ? graph_steps + 1 : graph_steps;
    B->group_bytes = group_bytes;
    B->resident_steps = resident_steps;
    if (new_rows) {
        rc = build_work(B);
        if (rc) return rc;
    }
    build_groups(B);
    return CX_OK;
}

int cx_batch_get_tuning(cx_batch *B, int32_t *tile_rows, int32_t *graph_steps, int64_t *group_bytes,
                        int32_t *resident_steps)
{
    int rc = check_batch(B);
    if (rc) return rc;
    if (tile_rows) *tile_rows = B->rows;
    if (graph_steps) *graph_steps = B->graph_steps;
    if (group_bytes) *group_bytes = B->group_bytes;
    if (resident_steps) *resident_steps = B->resident_steps;
    return CX_OK;
}

int cx_batch_set_time_block(cx_batch *B, int32_t stages)
{
    int rc = check_batch(B);
    if (rc) return rc;
    if (stages != 1 && stages != 2)
        return bfail(CX_ERR_INVALID_ARG, "time block: must be 1 or 2 stages per pass");
    BX_CUDA(cudaStreamSynchronize(B->stream), "synchronize before retuning");
    drop_graphs(B);
    B->time_block = stages;
    return CX_OK;
}

int cx_batch_get_time_block(cx_batch *B, int32_t *stages)
{
    int rc = check_batch(B);
    if (rc) return rc;
    if (!stages) return bfail(CX_ERR_INVALID_ARG, "stages must not be NULL");
    *stages = B->time_block;
    return CX_OK;
}

int cx_batch_step(cx_batch *B, int64_t n_steps)
{
    cx::NvtxRange range("cx_batch_step");
    int rc = check_batch(B);
    if (rc) return rc;
    if (n_steps < 0) return bfail(CX_ERR_INVALID_ARG, "n_steps < 0");
    if (n_steps == 0) return CX_OK;
    const int ngroups = (int)B->group_first.size() - 1;
    if (B->graph_steps > 0 && (int)B->gexec[0].size() != ngroups) {
        drop_graphs(B);
        for (int p = 0; p < 2; ++p) {
            B->gexec[p].assign(ngroups, nullptr);
            B->gend[p].assign(ngroups, 0);
        }
    }
    int end_parity = B->cur;
    for (int gi = 0; gi < ngroups; ++gi) {
        const int i0 = B->group_first[gi], i1 = B->group_first[gi + 1];
        int par = B->cur;
        int64_t left = n_steps;
        if (B->resident_steps > 0) {
            rc = run_resident(B, i0, i1, par, left, B->step, &end_parity);
            if (rc) return rc;
            continue;
        }
        if (B->graph_steps > 0) {
            while (left >= B->graph_steps) {
                if (!B->gexec[par][gi]) {
                    rc = capture_group(B, gi, par, &B->gexec[par][gi], &B->gend[par][gi]);
                    if (rc) return rc;
                }
                BX_CUDA(mark_step(B, B->step + (n_steps - left)), "step mark");
                BX_CUDA(cudaGraphLaunch(B->gexec[par][gi], B->stream), "graph launch");
                left -= B->graph_steps;
                par = B->gend[par][gi];
            }
        }
        int64_t marked = -1;  // `left` when the step was last marked
        while (left > 0) {
            if (marked < 0 || marked - left > (1 << 30)) {
                BX_CUDA(mark_step(B, B->step + (n_steps - left)), "step mark");
                marked = left;
            }
            int taken = 1;
            BX_CUDA(one_pass(B, i0, i1, &par, left, (int)(marked - left), &taken), "batch step launch");
            left -= taken;
        }
        end_parity = par;
    }
    B->cur = end_parity;
    B->step += n_steps;
    return CX_OK;
}

int cx_batch_synchronize(cx_batch *B)
{
    int rc = check_batch(B);
    if (rc) return rc;
    BX_CUDA(cudaStreamSynchronize(B->stream), "batch synchronize");
    return check_barrier(B);
}

int cx_batch_diagnostics(cx_batch *B, cx_diag *out)
{
    cx::NvtxRange range("cx_batch_diagnostics");
    int rc = check_batch(B);
    if (rc) return rc;
    if (!out) return bfail(CX_ERR_INVALID_ARG, "out must not be NULL");
    BX_CUDA(cx::launch_batch_diag(B->prec, B->d_inst, 0, B->count, kDiagBlocksPerInst, B->cur,
                                  B->d_part, B->d_res, B->stream),
            "batch diagnostics launch");
    BX_CUDA(cudaMemcpyAsync(B->h_res, B->d_res, 8 * sizeof(double) * (size_t)B->count,
                            cudaMemcpyDeviceToHost, B->stream),
            "batch diagnostics copy");
    BX_CUDA(cudaStreamSynchronize(B->stream), "batch diagnostics synchronize");
    rc = check_barrier(B);
    if (rc) return rc;
    int worst = CX_OK;
    for (int i = 0; i < B->count; ++i) {
        const double *h = B->h_res + 8LL * i;
        const double area = B->g[i].dx * B->g[i].dx;
        cx_diag &d = out[i];
        memset(&d, 0, sizeof d);
        d.step = B->step;
        d.dt = B->dt[i];
        d.t = (double)B->step * B->dt[i];
        d.mass_b = area * h[0];
        d.mass_n = area * h[1];
        d.invariant = area * (h[0] + B->p[i].theta * h[1]);
        d.min_b = h[2];
        d.min_n = h[3];
        d.max_b = h[4];
        d.r_env = h[5] >= 0.0 ? 0.5 * B->g[i].dx * sqrt(h[5]) : 0.0;
        d.area_env = area * h[7];
        d.finite = h[6] == 0.0 ? 1 : 0;
        d.status = !d.finite ? CX_ERR_NONFINITE
                             : ((d.min_b < 0.0 || d.min_n < 0.0) ? CX_ERR_NEGATIVE : CX_OK);
        if (d.status == CX_ERR_NONFINITE || (d.status != CX_OK && worst == CX_OK)) worst = d.status;
    }
    if (worst != CX_OK) return bfail(worst, "an instance of the batch is unhealthy (see status)");
    return CX_OK;
}

static int batch_io(cx_batch *B, int32_t index, int32_t which, int32_t dtype, size_t count)
{
    int rc = check_batch(B);
    if (rc) return rc;
    if (index < 0 || index >= B->count) return bfail(CX_ERR_INVALID_ARG, "instance index out of range");
    if (which < CX_FIELD_B || which > CX_FIELD_SIGMA) return bfail(CX_ERR_INVALID_ARG, "bad field");
    if (dtype != CX_F64 && dtype != CX_F32) return bfail(CX_ERR_INVALID_ARG, "bad dtype");
    if (count != (size_t)B->g[index].nx * (size_t)B->g[index].ny)
        return bfail(CX_ERR_INVALID_ARG, "count != nx*ny of the instance");
    return CX_OK;
}

static void *batch_field(cx_batch *B, int i, int which)
{
    if (which == CX_FIELD_B) return B->fb[B->cur][i];
    if (which == CX_FIELD_N) return B->fn[B->cur][i];
    return B->fs[i];
}

int cx_batch_get_field(cx_batch *B, int32_t index, int32_t which, void *host, int32_t dtype,
                       size_t count)
{
    int rc = batch_io(B, index, which, dtype, count);
    if (rc) return rc;
    if (!host) return bfail(CX_ERR_INVALID_ARG, "host must not be NULL");
    const int sd = B->prec == CX_PREC_F64 ? CX_F64 : CX_F32;
    const size_t row = (size_t)B->g[index].nx * B->elem;
    std::vector<unsigned char> tmp;
    void *dst = host;
    if (dtype != sd) {
        try { tmp.resize(count * B->elem); } catch (...) { return bfail(CX_ERR_OOM, "host staging"); }
        dst = tmp.data();
    }
    BX_CUDA(cudaStreamSynchronize(B->stream), "synchronize before field read");
    // the array in natural in-row order for the copy, and back to pair order
    void *f = batch_field(B, index, which);
    const cx_grid &g = B->g[index];
    BX_CUDA(cx::launch_pair_order(B->prec, f, g.nx, g.ny, B->pitch[index], B->stream), "reorder");
    BX_CUDA(cudaMemcpy2DAsync(dst, row, f, (size_t)B->pitch[index] * B->elem,
                              row, B->g[index].ny, cudaMemcpyDeviceToHost, B->stream),
            "field copy to host");
    BX_CUDA(cx::launch_pair_order(B->prec, f, g.nx, g.ny, B->pitch[index], B->stream), "reorder");
    BX_CUDA(cudaStreamSynchronize(B->stream), "field copy synchronize");
    if (dtype != sd) {
        if (sd == CX_F32)
            for (size_t q = 0; q < count; ++q) ((double *)host)[q] = ((const float *)dst)[q];
        else
            for (size_t q = 0; q < count; ++q) ((float *)host)[q] = (float)((const double *)dst)[q];
    }
    return CX_OK;
}

int cx_batch_set_field(cx_batch *B, int32_t index, int32_t which, const void *host, int32_t dtype,
                       size_t count)
{
    int rc = batch_io(B, index, which, dtype, count);
    if (rc) return rc;
    if (!host) return bfail(CX_ERR_INVALID_ARG, "host must not be NULL");
    const int sd = B->prec == CX_PREC_F64 ? CX_F64 : CX_F32;
    const size_t row = (size_t)B->g[index].nx * B->elem;
    std::vector<unsigned char> tmp;
    const void *src = host;
    if (dtype != sd) {
        try { tmp.resize(count * B->elem); } catch (...) { return bfail(CX_ERR_OOM, "host staging"); }
        if (sd == CX_F32)
            for (size_t q = 0; q < count; ++q) ((float *)tmp.data())[q] = (float)((const double *)host)[q];
        else
            for (size_t q = 0; q < count; ++q) ((double *)tmp.data())[q] = ((const float *)host)[q];
        src = tmp.data();
    }
    BX_CUDA(cudaStreamSynchronize(B->stream), "synchronize before field write");
    BX_CUDA(cudaMemcpy2DAsync(batch_field(B, index, which), (size_t)B->pitch[index] * B->elem, src, row,
                              row, B->g[index].ny, cudaMemcpyHostToDevice, B->stream),
            "field copy to device");
    BX_CUDA(cx::launch_pair_order(B->prec, batch_field(B, index, which), B->g[index].nx,
                                  B->g[index].ny, B->pitch[index], B->stream),
            "reorder");
    BX_CUDA(cudaStreamSynchronize(B->stream), "field copy synchronize");
    return CX_OK;
}

int cx_batch_polar_profile(cx_batch *B, int32_t index, double radius, int32_t nsamples,
                           double *host_out)
{
    int rc = check_batch(B);
    if (rc) return rc;
    if (index < 0 || index >= B->count) return bfail(CX_ERR_INVALID_ARG, "instance index out of range");
    if (!host_out || nsamples < 1 || nsamples > (1 << 24) || !(isfinite(radius) && radius >= 0.0))
        return bfail(CX_ERR_INVALID_ARG, "need host_out, 1 <= nsamples <= 2^24, radius >= 0");
    double *d = nullptr;
    BX_CUDA(cudaMalloc((void **)&d, sizeof(double) * (size_t)nsamples), "profile buffer");
    const cx_grid &g = B->g[index];
    cudaError_t e = cx::launch_polar(B->prec, B->fb[B->cur][index], g.nx, g.ny, B->pitch[index], g.dx,
                                     radius, nsamples, d, B->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(host_out, d, sizeof(double) * (size_t)nsamples, cudaMemcpyDeviceToHost,
                            B->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(B->stream);
    cudaFree(d);
    if (e != cudaSuccess) return bcuda(e, "polar profile");
    return CX_OK;
}

int cx_batch_get_time(cx_batch *B, int32_t *count, int64_t *step)
{
    int rc = check_batch(B);
    if (rc) return rc;
    if (count) *count = B->count;
    if (step) *step = B->step;
    return CX_OK;
}

}  // extern "C"
