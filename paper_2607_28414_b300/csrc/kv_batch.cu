// kv_batch.cu -- batched time stepping of several handles in one launch per
// step (parameter sweeps over uneven grids), and force sharing between handles
// on the same grid.
//
// A batch refers to existing FP32 handles (all of one step kind: homogeneous,
// pointwise or divergence-form heterogeneous; all on one stream, all at the
// same ping-pong parity). Each
// step is one launch of k_step_batch over the concatenated tile grids of all
// cases; every case keeps its own state, coefficients, envelope, sensors,
// traces and step counter. Blocks of steps replay from a CUDA graph. The case
// table (tensor maps, pointers, parameters) lives in device memory and is
// rebuilt whenever a case's parameters change.
#include <string.h>

#include <algorithm>
#include <vector>

#include "kv_internal.cuh"

struct kv_batch {
    std::vector<kv_handle *> h;
    kv::BatchCase *table_dev;
    std::vector<kv::BatchCase> table_host;  // last uploaded table
    int tx, ty, zc, ns;
    int total_blocks;
    int nt;
    size_t smem;
    void *kernel;
    cudaStream_t stream;
    cudaGraphExec_t graph[2];
    int graph_steps;
    long long launches;
    char err[512];
};

namespace {

kv_status berr(kv_batch *b, kv_status st, const char *msg) {
    if (b) snprintf(b->err, sizeof(b->err), "%s", msg);
    return kv::set_error(nullptr, st, "%s", msg);
}

void free_bgraphs(kv_batch *b) {
    for (int q = 0; q < 2; ++q)
        if (b->graph[q]) {
            cudaGraphExecDestroy(b->graph[q]);
            b->graph[q] = nullptr;
        }
}

// Build the case table for the current configuration; upload if it changed.
kv_status refresh(kv_batch *b) {
    const int n = (int)b->h.size();
    std::vector<kv::BatchCase> t(n);
    memset(t.data(), 0, sizeof(kv::BatchCase) * n);
    int begin = 0;
    for (int c = 0; c < n; ++c) {
        int blocks = 0;
        kv_status st = kv::batch_fill_case(b->h[c], &t[c], b->tx, b->ty, b->zc, begin, &blocks);
        if (st != KV_OK) return berr(b, st, "kv_batch: tensor map encoding failed");
        begin += blocks;
    }
    void *kernel;
    size_t smem;
    int nt;
    for (int c = 1; c < n; ++c)
        if (kv::step_kind(b->h[c]) != kv::step_kind(b->h[0]))
            return berr(b, KV_ERR_ARG, "kv_batch: cases must all use the same medium kind and operator");
    if (kv::batch_kernel_for(b->tx, b->ty, b->ns, kv::step_kind(b->h[0]), &kernel, &smem, &nt) != KV_OK)
        return berr(b, KV_ERR_ARG, "kv_batch: no batched kernel for this tile / stage count");
    const bool changed = b->table_host.size() != t.size() || b->kernel != kernel ||
                         memcmp(b->table_host.data(), t.data(), sizeof(kv::BatchCase) * n) != 0;
    if (!changed) return KV_OK;
    cudaError_t e = cudaStreamSynchronize(b->stream);  // no launch may still read the old table
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->table_dev, t.data(), sizeof(kv::BatchCase) * n, cudaMemcpyHostToDevice,
                            b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return berr(b, KV_ERR_CUDA, "kv_batch: case table upload failed");
    b->table_host = t;
    b->total_blocks = begin;
    b->kernel = kernel;
    b->smem = smem;
    b->nt = nt;
    free_bgraphs(b);  // graphs keep kernel and grid size
    return KV_OK;
}

kv_status check_cases(kv_batch *b) {
    for (kv_handle *h : b->h) {
        if (h->sticky) return berr(b, KV_ERR_STATE, "kv_batch: a case handle is in an error state");
        if (h->cur != b->h[0]->cur)
            return berr(b, KV_ERR_STATE, "kv_batch: cases are at different ping-pong parities");
    }
    return KV_OK;
}

kv_status launch_steps(kv_batch *b, int from, int n) {
    for (int i = 0; i < n; ++i) {
        if (kv::batch_launch(b->kernel, b->table_dev, (int)b->h.size(), b->total_blocks, b->nt, b->smem,
                             (from + i) & 1, b->stream) != KV_OK)
            return berr(b, KV_ERR_CUDA, "kv_batch: launch failed");
    }
    return KV_OK;
}

__global__ void k_rescale(float *__restrict__ dst, const float *__restrict__ src,
                          const float *__restrict__ sd, double sd_s, const float *__restrict__ ss,
                          double ss_s, long long Np) {
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < 3 * Np;
         c += (long long)gridDim.x * blockDim.x) {
        const long long q = c % Np;
        const double a = sd ? (double)sd[q] : sd_s;
        const double b = ss ? (double)ss[q] : ss_s;
        dst[c] = (b != 0.0) ? (float)((double)src[c] * (a / b)) : 0.f;
    }
}

}  // namespace

extern "C" {

kv_status kv_batch_create(kv_batch **out, int n, kv_handle *const *cases) {
    if (!out || n < 1 || !cases) return kv::set_error(nullptr, KV_ERR_ARG, "kv_batch_create: invalid arguments");
    *out = nullptr;
    for (int c = 0; c < n; ++c) {
        kv_handle *h = cases[c];
        if (!h || h->precision != KV_FP32)
            return kv::set_error(nullptr, KV_ERR_ARG, "kv_batch_create: cases must be FP32 handles");
        if (kv::step_kind(h) != kv::step_kind(cases[0]))
            return kv::set_error(nullptr, KV_ERR_ARG,
                                 "kv_batch_create: cases must all be homogeneous, all pointwise or all "
                                 "divergence-form heterogeneous");
        if (h->stream != cases[0]->stream)
            return kv::set_error(nullptr, KV_ERR_ARG, "kv_batch_create: cases must share one stream");
    }
    kv_batch *b = new kv_batch();
    b->h.assign(cases, cases + n);
    b->tx = 64;
    b->ty = 4;
    b->zc = 64;
    b->ns = 4;
    b->graph_steps = 32;
    b->stream = cases[0]->stream;
    b->graph[0] = b->graph[1] = nullptr;
    b->kernel = nullptr;
    b->err[0] = 0;
    if (cudaMalloc(&b->table_dev, sizeof(kv::BatchCase) * n) != cudaSuccess) {
        delete b;
        return kv::set_error(nullptr, KV_ERR_OOM, "kv_batch_create: table allocation failed");
    }
    *out = b;
    return KV_OK;
}

kv_status kv_batch_set_config(kv_batch *b, int tx, int ty, int zc, int ns) {
    if (!b) return KV_ERR_ARG;
    void *kernel;
    size_t smem;
    int nt;
    if (zc < 1 || kv::batch_kernel_for(tx, ty, ns, kv::step_kind(b->h[0]), &kernel, &smem, &nt) != KV_OK)
        return berr(b, KV_ERR_ARG, "kv_batch_set_config: unsupported tile, stage count or z chunk");
    b->tx = tx;
    b->ty = ty;
    b->zc = zc;
    b->ns = ns;
    return KV_OK;
}

kv_status kv_batch_step(kv_batch *b, int n) {
    if (!b || n < 0) return kv::set_error(nullptr, KV_ERR_ARG, "kv_batch_step: invalid arguments");
    kv_status st;
    if ((st = check_cases(b)) != KV_OK) return st;
    if ((st = refresh(b)) != KV_OK) return st;
    const int from0 = b->h[0]->cur;
    int from = from0;
    int left = n;
    const int G = b->graph_steps;
    if (left >= G && G > 0 && G % 2 == 0) {
        if (!b->graph[from]) {
            cudaGraph_t g = nullptr;
            cudaError_t e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal);
            if (e != cudaSuccess) return berr(b, KV_ERR_CUDA, "kv_batch_step: capture failed");
            st = launch_steps(b, from, G);
            e = cudaStreamEndCapture(b->stream, &g);
            if (st != KV_OK || e != cudaSuccess) {
                if (g) cudaGraphDestroy(g);
                return berr(b, KV_ERR_CUDA, "kv_batch_step: capture failed");
            }
            e = cudaGraphInstantiate(&b->graph[from], g, 0);
            cudaGraphDestroy(g);
            if (e != cudaSuccess) return berr(b, KV_ERR_CUDA, "kv_batch_step: graph instantiate failed");
        }
        while (left >= G) {
            if (cudaGraphLaunch(b->graph[from], b->stream) != cudaSuccess)
                return berr(b, KV_ERR_CUDA, "kv_batch_step: graph launch failed");
            left -= G;
            b->launches += G;
        }
    }
    if ((st = launch_steps(b, from, left)) != KV_OK) return st;
    b->launches += left;
    from = (from + left) & 1;
    for (kv_handle *h : b->h) {
        h->cur = (from0 + n) & 1;
        h->steps_host += n;
        h->launches += n;
    }
    return KV_OK;
}

kv_status kv_batch_autotune(kv_batch *b, int trial_steps, double *best_ms) {
    if (!b || trial_steps < 1) return KV_ERR_ARG;
    static const int tiles[][2] = {{32, 8}, {32, 16}, {64, 4}, {64, 8}, {64, 16}, {128, 2}, {128, 4}, {128, 8}};
    static const int stages[] = {4, 6, 8};
    static const int zcs[] = {16, 32, 64};
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
        return berr(b, KV_ERR_CUDA, "kv_batch_autotune: cudaEventCreate failed");
    double best = INFINITY;
    int pick[4] = {b->tx, b->ty, b->zc, b->ns};
    kv_status st = KV_OK;
    for (auto &t : tiles)
        for (int ns : stages)
            for (int zc : zcs) {
                if (kv_batch_set_config(b, t[0], t[1], zc, ns) != KV_OK) continue;
                if ((st = kv_batch_step(b, 2)) != KV_OK) break;
                cudaEventRecord(e0, b->stream);
                if ((st = kv_batch_step(b, trial_steps)) != KV_OK) break;
                cudaEventRecord(e1, b->stream);
                cudaEventSynchronize(e1);
                float ms = 0.f;
                cudaEventElapsedTime(&ms, e0, e1);
                if (ms > 0.f && ms < best) {
                    best = ms;
                    pick[0] = t[0];
                    pick[1] = t[1];
                    pick[2] = zc;
                    pick[3] = ns;
                }
            }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != KV_OK) return st;
    kv_batch_set_config(b, pick[0], pick[1], pick[2], pick[3]);
    if (best_ms) *best_ms = best / trial_steps;
    for (kv_handle *h : b->h)
        if ((st = kv_reset(h)) != KV_OK) return st;
    return KV_OK;
}

kv_status kv_batch_get_config(kv_batch *b, int *cfg) {
    if (!b || !cfg) return KV_ERR_ARG;
    cfg[0] = b->tx;
    cfg[1] = b->ty;
    cfg[2] = b->zc;
    cfg[3] = b->ns;
    return KV_OK;
}

long long kv_batch_launch_count(kv_batch *b) { return b ? b->launches : 0; }

kv_status kv_batch_destroy(kv_batch *b) {
    if (!b) return KV_OK;
    cudaStreamSynchronize(b->stream);
    free_bgraphs(b);
    if (b->table_dev) cudaFree(b->table_dev);
    delete b;
    return KV_OK;
}

kv_status kv_share_force(kv_handle *dst, kv_handle *src) {
    if (!dst || !src || dst->nx != src->nx || dst->ny != src->ny || dst->nz != src->nz ||
        dst->precision != KV_FP32 || src->precision != KV_FP32)
        return kv::set_error(dst, KV_ERR_ARG, "kv_share_force: handles must be FP32 on the same grid");
    if (!src->have_force) return kv::set_error(dst, KV_ERR_STATE, "kv_share_force: source has no projected force");
    cudaError_t e = cudaStreamSynchronize(src->stream);
    if (e != cudaSuccess) return kv::cuda_check(dst, e, "kv_share_force");
    k_rescale<<<148 * 8, 256, 0, dst->stream>>>((float *)dst->F, (const float *)src->F,
                                                 dst->het ? (const float *)dst->S : nullptr, dst->S_s,
                                                 src->het ? (const float *)src->S : nullptr, src->S_s,
                                                 dst->Np);
    dst->launches++;
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(dst->stream);
    if (e != cudaSuccess) return kv::cuda_check(dst, e, "kv_share_force");
    dst->have_force = 1;
    for (int q = 0; q < 2; ++q)
        if (dst->graph[q]) {
            cudaGraphExecDestroy(dst->graph[q]);
            dst->graph[q] = nullptr;
        }
    return KV_OK;
}

}  // extern "C"
