// kv_api.cu -- the extern "C" boundary of libkv (declared in include/kv.h).
// Argument checking, device memory ownership, staging of caller fields into
// the pitched device layout, the step loop (CUDA graph for blocks of steps)
// and the synchronising reads.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "kv_internal.cuh"

static thread_local char g_create_err[512] = "";

namespace kv {

kv_status set_error(kv_handle *h, kv_status st, const char *fmt, ...) {
    char *buf = h ? h->err : g_create_err;
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, 512, fmt, ap);
    va_end(ap);
    return st;
}

kv_status cuda_check(kv_handle *h, cudaError_t e, const char *what) {
    if (e == cudaSuccess) return KV_OK;
    if (h) h->sticky = 1;
    return set_error(h, e == cudaErrorMemoryAllocation ? KV_ERR_OOM : KV_ERR_CUDA, "%s: %s", what,
                     cudaGetErrorString(e));
}

kv_status launch_fold(kv_handle *h, const float *G, double Gs, const float *rho, double rhos,
                      const float *eta, double etas);
kv_status launch_init_velocity(kv_handle *h, const float *v_pitched);

}  // namespace kv

using namespace kv;

namespace {

bool field_ok(const kv_field &f) {
    if (f.where == KV_SCALAR) return isfinite(f.value);
    if (f.where == KV_HOST || f.where == KV_DEVICE) return f.data != nullptr;
    return false;
}

// Copy a dense caller field into a pitched float plane of the handle.
kv_status stage(kv_handle *h, const kv_field &f, float *dst) {
    cudaError_t e = cudaMemcpy2DAsync(dst, (size_t)h->px * 4, f.data, (size_t)h->nx * 4,
                                      (size_t)h->nx * 4, (size_t)h->ny * h->nz, cudaMemcpyDefault,
                                      h->stream);
    return cuda_check(h, e, "copy of an input field");
}

// Host-side stability limit over host arrays or scalars (same formula as the
// device reduction: dt <= h^2 / (nu + sqrt(nu^2 + c^2 h^2)), h^2 = dx^2 / 3).
double dt_limit_node(double g, double r, double e, double dx) {
    const double h2 = dx * dx / 3.0;
    if (!(r > 0.0) || g < 0.0 || e < 0.0 || !isfinite(g) || !isfinite(r) || !isfinite(e))
        return -1.0;
    const double c2 = g / r, nu = e / r;
    const double den = nu + sqrt(nu * nu + c2 * h2);
    return den > 0.0 ? h2 / den : INFINITY;
}

kv_status stable_dt_impl(kv_handle *h, int nx, int ny, int nz, double dx, const kv_field &G,
                         const kv_field &rho, const kv_field &eta, int op, double *out) {
    const kv_field *fs[3] = {&G, &rho, &eta};
    int n_host = 0, n_dev = 0;
    for (auto *f : fs) {
        if (!field_ok(*f)) return set_error(h, KV_ERR_ARG, "invalid medium field");
        n_host += f->where == KV_HOST;
        n_dev += f->where == KV_DEVICE;
    }
    if (n_host && n_dev)
        return set_error(h, KV_ERR_ARG, "medium arrays must all be on the host or all on the device");
    const long long n = (long long)nx * ny * nz;
    double m;
    if (n_dev) {
        kv_status st = stable_dt_device(h ? h->stream : 0, h ? h->dtmin : nullptr, nx, ny, nz, nx, dx,
                                        G.where == KV_DEVICE ? G.data : nullptr, G.value,
                                        rho.where == KV_DEVICE ? rho.data : nullptr, rho.value,
                                        eta.where == KV_DEVICE ? eta.data : nullptr, eta.value, op, &m);
        if (st != KV_OK) return set_error(h, st, "device stability reduction failed");
    } else if (n_host) {
        m = INFINITY;
        auto val = [](const kv_field &f, long long c) { return f.where == KV_HOST ? (double)f.data[c] : f.value; };
        const long long sy = nx, sz = (long long)nx * ny;
        for (long long c = 0; c < n; ++c) {
            double g = val(G, c), e = val(eta, c);
            const double r = val(rho, c);
            double v = dt_limit_node(g, r, e, dx);
            if (v >= 0.0 && op == KV_OP_DIVERGENCE) {
                const int i = (int)(c % nx), j = (int)((c / nx) % ny), k = (int)(c / sz);
                if (i >= 1 && i <= nx - 2 && j >= 1 && j <= ny - 2 && k >= 1 && k <= nz - 2) {
                    const long long nb[6] = {c - 1, c + 1, c - sy, c + sy, c - sz, c + sz};
                    double gs = 6.0 * g, es = 6.0 * e;
                    for (long long q : nb) {
                        gs += val(G, q);
                        es += val(eta, q);
                    }
                    v = dt_limit_node(gs / 12.0, r, es / 12.0, dx);
                } else {
                    v = INFINITY;  // boundary node: values checked, never updated
                }
            }
            m = fmin(m, v);
        }
    } else {
        m = dt_limit_node(G.value, rho.value, eta.value, dx);
    }
    if (m < 0.0) return set_error(h, KV_ERR_ARG, "medium has rho <= 0, G < 0, eta < 0 or non-finite values");
    *out = m;
    return KV_OK;
}

void free_graphs(kv_handle *h) {
    for (int b = 0; b < 2; ++b)
        if (h->graph[b]) {
            cudaGraphExecDestroy(h->graph[b]);
            h->graph[b] = nullptr;
        }
}

kv_status poll_flags(kv_handle *h) {
    long long flags = 0;
    cudaError_t e = cudaMemcpyAsync(&flags, h->ctrl + kErrFlags, sizeof(flags),
                                    cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_check(h, e, "synchronise");
    if (flags & 1) {
        h->sticky = 1;
        return set_error(h, KV_ERR_TIMEOUT, "a bounded device wait timed out in the step kernel");
    }
    return KV_OK;
}

template <typename P>
kv_status dalloc(kv_handle *h, P **p, size_t bytes) {
    cudaError_t e = cudaMalloc((void **)p, bytes);
    if (e != cudaSuccess) {
        *p = nullptr;
        return cuda_check(h, e, "cudaMalloc");
    }
    return KV_OK;
}

kv_status fold(kv_handle *h, const kv_field &G, const kv_field &rho, const kv_field &eta) {
    if (h->het && step_kind(h) == kKindDiv && h->coef_fields < 3) {  // third field: 1/rho
        kv_status st = cuda_check(h, cudaStreamSynchronize(h->stream), "coefficient reallocation");
        if (st != KV_OK) return st;
        cudaFree(h->coef);
        h->coef = nullptr;
        h->coef_fields = 0;
        if ((st = dalloc(h, &h->coef, 3 * (size_t)h->Np * h->esize)) != KV_OK) {
            h->sticky = 1;  // no coefficient storage left: the handle cannot step
            return st;
        }
        h->coef_fields = 3;
    }
    if (!h->het) {
        h->A_s = h->dt * h->dt * G.value / rho.value / (h->dx * h->dx);
        h->B_s = h->dt * eta.value / rho.value / (h->dx * h->dx);
        h->S_s = h->dt * h->dt / rho.value;
        return KV_OK;
    }
    // the fields were staged (pitched) into fstage by stage_medium
    const kv_field *fs[3] = {&G, &rho, &eta};
    const float *ptr[3];
    for (int q = 0; q < 3; ++q) ptr[q] = fs[q]->where != KV_SCALAR ? h->fstage + q * h->Np : nullptr;
    kv_status st = launch_fold(h, ptr[0], G.value, ptr[1], rho.value, ptr[2], eta.value);
    if (st != KV_OK) return st;
    if ((st = cuda_check(h, cudaStreamSynchronize(h->stream), "medium fold")) != KV_OK) return st;
    return medium_classify(h);
}

// Copy the medium's dense fields (host or device) into the handle's pitched
// staging planes and evaluate the stability limit of operator op there, on
// the device (a handle never loops over a host field on the CPU).
kv_status stage_medium(kv_handle *h, const kv_field &G, const kv_field &rho, const kv_field &eta, int op,
                       double *dt_max) {
    const kv_field *fs[3] = {&G, &rho, &eta};
    const float *ptr[3];
    for (int q = 0; q < 3; ++q) {
        if (!field_ok(*fs[q])) return set_error(h, KV_ERR_ARG, "invalid medium field");
        ptr[q] = nullptr;
        if (fs[q]->where != KV_SCALAR) {
            kv_status st = stage(h, *fs[q], h->fstage + q * h->Np);
            if (st != KV_OK) return st;
            ptr[q] = h->fstage + q * h->Np;
        }
    }
    double m;
    if (!ptr[0] && !ptr[1] && !ptr[2]) {
        m = dt_limit_node(G.value, rho.value, eta.value, h->dx);
    } else {
        kv_status st = stable_dt_device(h->stream, h->dtmin, h->nx, h->ny, h->nz, h->px, h->dx, ptr[0], G.value,
                                        ptr[1], rho.value, ptr[2], eta.value, op, &m);
        if (st != KV_OK) return set_error(h, st, "device stability reduction failed");
    }
    if (m < 0.0) return set_error(h, KV_ERR_ARG, "medium has rho <= 0, G < 0, eta < 0 or non-finite values");
    *dt_max = m;
    return KV_OK;
}

}  // namespace

extern "C" {

const char *kv_status_string(int s) {
    switch (s) {
        case KV_OK: return "KV_OK";
        case KV_ERR_ARG: return "KV_ERR_ARG";
        case KV_ERR_CUDA: return "KV_ERR_CUDA";
        case KV_ERR_OOM: return "KV_ERR_OOM";
        case KV_ERR_UNSTABLE_DT: return "KV_ERR_UNSTABLE_DT";
        case KV_ERR_NONFINITE: return "KV_ERR_NONFINITE";
        case KV_CG_BREAKDOWN: return "KV_CG_BREAKDOWN";
        case KV_CG_MAXITER: return "KV_CG_MAXITER";
        case KV_ERR_TIMEOUT: return "KV_ERR_TIMEOUT";
        case KV_ERR_STATE: return "KV_ERR_STATE";
        case KV_ERR_UNSUPPORTED: return "KV_ERR_UNSUPPORTED";
        default: return "KV_UNKNOWN";
    }
}

const char *kv_last_error(kv_handle *h) { return h ? h->err : g_create_err; }

kv_status kv_stable_dt(int nx, int ny, int nz, double dx, kv_field G, kv_field rho, kv_field eta,
                       double *dt_max) {
    if (nx < 3 || ny < 3 || nz < 3 || !(dx > 0.0) || !dt_max)
        return set_error(nullptr, KV_ERR_ARG, "kv_stable_dt: invalid grid, dx or output pointer");
    return stable_dt_impl(nullptr, nx, ny, nz, dx, G, rho, eta, KV_OP_POINTWISE, dt_max);
}

kv_status kv_stable_dt_op(int nx, int ny, int nz, double dx, kv_field G, kv_field rho, kv_field eta,
                          int op, double *dt_max) {
    if (nx < 3 || ny < 3 || nz < 3 || !(dx > 0.0) || !dt_max ||
        (op != KV_OP_POINTWISE && op != KV_OP_DIVERGENCE))
        return set_error(nullptr, KV_ERR_ARG, "kv_stable_dt_op: invalid grid, dx, operator or output pointer");
    return stable_dt_impl(nullptr, nx, ny, nz, dx, G, rho, eta, op, dt_max);
}

kv_status kv_destroy(kv_handle *h) {
    if (!h) return KV_OK;
    if (h->stream) cudaStreamSynchronize(h->stream);
    free_graphs(h);
    medium_labels_free(h);
    void *dev[] = {h->state[0], h->state[1], h->F, h->coef, h->S, h->g_dev, h->sens_dev,
                   h->traces, h->ctrl, h->cgv, h->phi, h->b, h->scal,
                   h->partials, h->fstage, h->dtmin, h->mg_pool, h->fcg_pool};
    for (void *p : dev)
        if (p) cudaFree(p);
    if (h->ctrl_host) cudaFreeHost(h->ctrl_host);
    if (h->scal_host) cudaFreeHost(h->scal_host);
    if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
    free(h);
    return KV_OK;
}

kv_status kv_create(kv_handle **out, int nx, int ny, int nz, double dx, double dt, kv_field G,
                    kv_field rho, kv_field eta, int precision, void *stream) {
    if (!out) return set_error(nullptr, KV_ERR_ARG, "kv_create: out is NULL");
    *out = nullptr;
    if (nx < 3 || ny < 3 || nz < 3 || !(dx > 0.0) || !(dt > 0.0) ||
        (precision != KV_FP32 && precision != KV_FP64))
        return set_error(nullptr, KV_ERR_ARG, "kv_create: invalid grid %dx%dx%d, dx, dt or precision",
                         nx, ny, nz);
    const long long px = round_up(nx, kPitchAlign);
    if (px * ny * (long long)nz > (1ll << 31) - 1)
        return set_error(nullptr, KV_ERR_ARG, "kv_create: grid too large (more than 2^31 padded nodes)");
    double dt_max = INFINITY;
    kv_status st;
    {
        const kv_field *fs[3] = {&G, &rho, &eta};
        int n_host = 0, n_dev = 0;
        for (auto *f : fs) {
            if (!field_ok(*f)) return set_error(nullptr, KV_ERR_ARG, "invalid medium field");
            n_host += f->where == KV_HOST;
            n_dev += f->where == KV_DEVICE;
        }
        if (n_host && n_dev)
            return set_error(nullptr, KV_ERR_ARG, "medium arrays must all be on the host or all on the device");
        if (!n_host && !n_dev) {  // scalars: check before allocating anything
            if ((st = stable_dt_impl(nullptr, nx, ny, nz, dx, G, rho, eta, KV_OP_POINTWISE, &dt_max)) != KV_OK)
                return st;
            if (dt > dt_max * (1.0 + 1e-12))
                return set_error(nullptr, KV_ERR_UNSTABLE_DT,
                                 "dt = %.6e s exceeds the stability limit %.6e s", dt, dt_max);
        }
    }

    kv_handle *h = (kv_handle *)calloc(1, sizeof(kv_handle));
    if (!h) return set_error(nullptr, KV_ERR_OOM, "kv_create: host allocation failed");
    h->nx = nx;
    h->ny = ny;
    h->nz = nz;
    h->px = (int)px;
    h->Np = px * ny * nz;
    h->dx = dx;
    h->dt = dt;
    h->dt_max = dt_max;
    h->precision = precision;
    h->esize = precision == KV_FP64 ? 8 : 4;
    h->het = (G.where != KV_SCALAR) || (rho.where != KV_SCALAR) || (eta.where != KV_SCALAR);
    h->op = KV_OP_POINTWISE;
    h->medium_encoding = KV_MEDIUM_AUTO;
    h->variant = 0;
    h->cg_ns = 8;
    h->tx = 64;
    h->ty = 8;
    h->zc = 32;
    h->ns_stages = 4;
    h->graph_steps = 32;
    cudaGetDevice(&h->device);
    if (stream) {
        h->stream = (cudaStream_t)stream;
    } else {
        if ((st = cuda_check(h, cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking),
                             "cudaStreamCreate")) != KV_OK)
            goto fail;
        h->own_stream = 1;
    }
    {
        const size_t Np = (size_t)h->Np, es = h->esize;
        const dim3 g((nx + 31) / 32, (ny + 7) / 8, (nz + 7) / 8);
        h->partials_len = 2 * g.x * g.y * g.z;
        if ((st = dalloc(h, &h->state[0], 6 * Np * es)) || (st = dalloc(h, &h->state[1], 6 * Np * es)) ||
            (st = dalloc(h, &h->F, 3 * Np * es)) || (st = dalloc(h, &h->fstage, 3 * Np * 4)) ||
            (st = dalloc(h, &h->cgv, 4 * Np * es)) || (st = dalloc(h, &h->phi, Np * 8)) ||
            (st = dalloc(h, &h->b, Np * 8)) || (st = dalloc(h, &h->ctrl, kCtrlWords * 8)) ||
            (st = dalloc(h, &h->scal, kCgScalars * 8)) ||
            (st = dalloc(h, &h->partials, (size_t)h->partials_len * 8)) ||
            (st = dalloc(h, &h->dtmin, kDtBlocks * 8)))
            goto fail;
        if (h->het && ((st = dalloc(h, &h->coef, 2 * Np * es)) || (st = dalloc(h, &h->S, Np * es))))
            goto fail;
        h->coef_fields = h->het ? 2 : 0;
        h->p[0] = h->cgv;
        h->r = (char *)h->cgv + Np * es;
        h->p[1] = (char *)h->cgv + 2 * Np * es;
        h->e = (char *)h->cgv + 3 * Np * es;
        if ((st = cuda_check(h, cudaMallocHost((void **)&h->ctrl_host, kCtrlWords * 8), "cudaMallocHost")) ||
            (st = cuda_check(h, cudaMallocHost((void **)&h->scal_host, kCgScalars * 8), "cudaMallocHost")))
            goto fail;
        cudaError_t e = cudaSuccess;
        void *zero[] = {h->state[0], h->state[1], h->F, h->fstage, h->cgv, h->phi, h->b};
        size_t zbytes[] = {6 * Np * es, 6 * Np * es, 3 * Np * es, 3 * Np * 4, 4 * Np * es, Np * 8,
                           Np * 8};
        for (int q = 0; q < 7 && e == cudaSuccess; ++q) e = cudaMemsetAsync(zero[q], 0, zbytes[q], h->stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(h->ctrl, 0, kCtrlWords * 8, h->stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(h->scal, 0, kCgScalars * 8, h->stream);
        if (e == cudaSuccess && h->het) e = cudaMemsetAsync(h->coef, 0, 2 * Np * es, h->stream);
        if (e == cudaSuccess && h->het) e = cudaMemsetAsync(h->S, 0, Np * es, h->stream);
        if ((st = cuda_check(h, e, "initial memset")) != KV_OK) goto fail;
    }
    if ((st = stage_medium(h, G, rho, eta, KV_OP_POINTWISE, &h->dt_max)) != KV_OK) goto fail;
    if (dt > h->dt_max * (1.0 + 1e-12)) {
        st = set_error(h, KV_ERR_UNSTABLE_DT, "dt = %.6e s exceeds the stability limit %.6e s", dt, h->dt_max);
        goto fail;
    }
    if ((st = fold(h, G, rho, eta)) != KV_OK) goto fail;
    if ((st = cuda_check(h, cudaStreamSynchronize(h->stream), "kv_create")) != KV_OK) goto fail;
    *out = h;
    return KV_OK;
fail:
    snprintf(g_create_err, sizeof(g_create_err), "%s", h->err);
    kv_destroy(h);
    return st;
}

kv_status kv_set_medium(kv_handle *h, kv_field G, kv_field rho, kv_field eta) {
    if (!h) return KV_ERR_ARG;
    if (h->sticky) return KV_ERR_STATE;
    const int het = (G.where != KV_SCALAR) || (rho.where != KV_SCALAR) || (eta.where != KV_SCALAR);
    if (het != h->het)
        return set_error(h, KV_ERR_ARG, "kv_set_medium: homogeneous/heterogeneous kind differs from kv_create");
    double dt_max;
    kv_status st = cuda_check(h, cudaStreamSynchronize(h->stream), "kv_set_medium");
    if (st != KV_OK) return st;
    if ((st = stage_medium(h, G, rho, eta, h->op, &dt_max)) != KV_OK) return st;
    if (h->dt > dt_max * (1.0 + 1e-12))
        return set_error(h, KV_ERR_UNSTABLE_DT, "dt = %.6e s exceeds the stability limit %.6e s", h->dt,
                         dt_max);
    h->dt_max = dt_max;
    free_graphs(h);
    return fold(h, G, rho, eta);
}

kv_status kv_set_medium_encoding(kv_handle *h, int encoding) {
    if (!h) return KV_ERR_ARG;
    if (h->sticky) return KV_ERR_STATE;
    if (encoding != KV_MEDIUM_AUTO && encoding != KV_MEDIUM_FIELDS)
        return set_error(h, KV_ERR_ARG, "kv_set_medium_encoding: unknown encoding %d", encoding);
    kv_status st = cuda_check(h, cudaStreamSynchronize(h->stream), "kv_set_medium_encoding");
    if (st != KV_OK) return st;
    h->medium_encoding = encoding;
    free_graphs(h);
    h->tma_ready = 0;
    return medium_classify(h);  // the folded fields are still there
}

int kv_medium_classes(kv_handle *h) { return h ? h->n_labels : -1; }

kv_status kv_set_operator(kv_handle *h, int op, kv_field G, kv_field rho, kv_field eta) {
    if (!h) return KV_ERR_ARG;
    if (op != KV_OP_POINTWISE && op != KV_OP_DIVERGENCE)
        return set_error(h, KV_ERR_ARG, "kv_set_operator: unknown operator %d", op);
    if (h->sticky) return KV_ERR_STATE;
    const int het = (G.where != KV_SCALAR) || (rho.where != KV_SCALAR) || (eta.where != KV_SCALAR);
    if (het != h->het)
        return set_error(h, KV_ERR_ARG, "kv_set_operator: homogeneous/heterogeneous kind differs from kv_create");
    if (op == KV_OP_DIVERGENCE && h->het && h->precision == KV_FP32 && h->variant >= 2)
        return set_error(h, KV_ERR_UNSUPPORTED, "kv_set_operator: the two-step kernel supports only the pointwise operator");
    double dt_max;
    kv_status st = cuda_check(h, cudaStreamSynchronize(h->stream), "kv_set_operator");
    if (st != KV_OK) return st;
    if ((st = stage_medium(h, G, rho, eta, op, &dt_max)) != KV_OK) return st;
    if (h->dt > dt_max * (1.0 + 1e-12))
        return set_error(h, KV_ERR_UNSTABLE_DT, "dt = %.6e s exceeds the stability limit %.6e s of operator %d",
                         h->dt, dt_max, op);
    h->op = op;
    h->dt_max = dt_max;
    h->tma_ready = 0;
    free_graphs(h);
    if ((st = fold(h, G, rho, eta)) != KV_OK) h->sticky = 1;  // coefficients of neither operator
    return st;
}

kv_status kv_set_envelope(kv_handle *h, const float *g, int n, int where) {
    if (!h || n < 0 || (n > 0 && !g) || (where != KV_HOST && where != KV_DEVICE))
        return set_error(h, KV_ERR_ARG, "kv_set_envelope: invalid arguments");
    if (h->sticky) return KV_ERR_STATE;
    if (n > h->n_g || !h->g_dev) {
        if (h->g_dev) {
            cudaStreamSynchronize(h->stream);
            cudaFree(h->g_dev);
            h->g_dev = nullptr;
        }
        kv_status st = dalloc(h, &h->g_dev, (size_t)std::max(n, 1) * 4);
        if (st != KV_OK) return st;
    }
    h->n_g = n;
    free_graphs(h);
    if (n == 0) return KV_OK;
    kv_status st = cuda_check(
        h, cudaMemcpyAsync(h->g_dev, g, (size_t)n * 4, cudaMemcpyDefault, h->stream), "envelope copy");
    if (st == KV_OK && where == KV_HOST)
        st = cuda_check(h, cudaStreamSynchronize(h->stream), "envelope copy");
    return st;
}

kv_status kv_set_sensors(kv_handle *h, const int *ijk, int n, int capacity) {
    if (!h || n < 0 || capacity < 0 || (n > 0 && !ijk))
        return set_error(h, KV_ERR_ARG, "kv_set_sensors: invalid arguments");
    if (h->sticky) return KV_ERR_STATE;
    for (int s = 0; s < n; ++s) {
        const int i = ijk[3 * s], j = ijk[3 * s + 1], k = ijk[3 * s + 2];
        if (i < 0 || i >= h->nx || j < 0 || j >= h->ny || k < 0 || k >= h->nz)
            return set_error(h, KV_ERR_ARG, "sensor %d at (%d,%d,%d) is outside the grid", s, i, j, k);
    }
    cudaStreamSynchronize(h->stream);
    if (h->sens_dev) cudaFree(h->sens_dev);
    if (h->traces) cudaFree(h->traces);
    h->sens_dev = nullptr;
    h->traces = nullptr;
    h->ns = 0;
    h->cap = 0;
    free_graphs(h);
    if (n == 0 || capacity == 0) return KV_OK;
    kv_status st;
    // device layout: [3n (i, j, k)] [nz + 1 plane offsets] [n sensor indices sorted by plane]
    std::vector<int> tab((size_t)3 * n + h->nz + 1 + n);
    memcpy(tab.data(), ijk, (size_t)3 * n * 4);
    int *off = tab.data() + 3 * n, *ord = off + h->nz + 1;
    for (int s = 0; s < n; ++s) off[ijk[3 * s + 2] + 1]++;
    for (int k = 0; k < h->nz; ++k) off[k + 1] += off[k];
    std::vector<int> fill(off, off + h->nz);
    for (int s = 0; s < n; ++s) ord[fill[ijk[3 * s + 2]]++] = s;
    if ((st = dalloc(h, &h->sens_dev, tab.size() * 4)) != KV_OK) return st;
    if ((st = dalloc(h, &h->traces, (size_t)capacity * n * 3 * h->esize)) != KV_OK) return st;
    cudaError_t e = cudaMemcpyAsync(h->sens_dev, tab.data(), tab.size() * 4, cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->traces, 0, (size_t)capacity * n * 3 * h->esize, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if ((st = cuda_check(h, e, "kv_set_sensors")) != KV_OK) return st;
    h->ns = n;
    h->cap = capacity;
    return KV_OK;
}

kv_status kv_reset(kv_handle *h) {
    if (!h) return KV_ERR_ARG;
    if (h->sticky) return KV_ERR_STATE;
    const size_t bytes = 6 * (size_t)h->Np * h->esize;
    cudaError_t e = cudaMemsetAsync(h->state[0], 0, bytes, h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->state[1], 0, bytes, h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->ctrl, 0, 3 * sizeof(long long), h->stream);
    if (e == cudaSuccess && h->traces)
        e = cudaMemsetAsync(h->traces, 0, (size_t)h->cap * h->ns * 3 * h->esize, h->stream);
    h->cur = 0;
    h->steps_host = 0;
    return cuda_check(h, e, "kv_reset");
}

kv_status kv_selftest_wait(kv_handle *h) {
    if (!h) return KV_ERR_ARG;
    if (h->sticky) return KV_ERR_STATE;
    kv_status st = launch_wait_selftest(h);
    if (st != KV_OK) return st;
    return poll_flags(h);  // KV_ERR_TIMEOUT, handle in the error state
}

long long kv_state_bytes(kv_handle *h) { return h ? 6 * (long long)h->Np * (long long)h->esize : 0; }

kv_status kv_save_state(kv_handle *h, void *buf, int where, long long *step) {
    if (!h || !buf || (where != KV_HOST && where != KV_DEVICE))
        return set_error(h, KV_ERR_ARG, "kv_save_state: invalid arguments");
    if (h->sticky) return KV_ERR_STATE;
    kv_status st = poll_flags(h);
    if (st != KV_OK) return st;
    cudaError_t e = cudaMemcpyAsync(buf, h->state[h->cur], (size_t)kv_state_bytes(h), cudaMemcpyDefault, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if ((st = cuda_check(h, e, "kv_save_state")) != KV_OK) return st;
    if (step) *step = h->steps_host;
    return KV_OK;
}

kv_status kv_load_state(kv_handle *h, const void *buf, int where, long long step) {
    if (!h || !buf || step < 0 || (where != KV_HOST && where != KV_DEVICE))
        return set_error(h, KV_ERR_ARG, "kv_load_state: invalid arguments");
    if (h->sticky) return KV_ERR_STATE;
    kv_status st = cuda_check(h, cudaStreamSynchronize(h->stream), "kv_load_state");
    if (st != KV_OK) return st;
    cudaError_t e = cudaMemcpyAsync(h->state[h->cur], buf, (size_t)kv_state_bytes(h), cudaMemcpyDefault, h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h->ctrl + kStep, &step, sizeof(long long), cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if ((st = cuda_check(h, e, "kv_load_state")) != KV_OK) return st;
    h->steps_host = step;
    return KV_OK;
}

kv_status kv_set_initial_velocity(kv_handle *h, kv_field vx, kv_field vy, kv_field vz) {
    if (!h) return KV_ERR_ARG;
    const kv_field *v[3] = {&vx, &vy, &vz};
    for (auto *f : v)
        if (!field_ok(*f) || (f->where == KV_SCALAR && f->value != 0.0))
            return set_error(h, KV_ERR_ARG, "initial velocity components must be arrays or 0");
    kv_status st = kv_reset(h);
    if (st != KV_OK) return st;
    cudaError_t e = cudaMemsetAsync(h->fstage, 0, 3 * (size_t)h->Np * 4, h->stream);
    if ((st = cuda_check(h, e, "kv_set_initial_velocity")) != KV_OK) return st;
    for (int q = 0; q < 3; ++q)
        if (v[q]->where != KV_SCALAR && (st = stage(h, *v[q], h->fstage + q * h->Np)) != KV_OK) return st;
    if ((st = launch_init_velocity(h, h->fstage)) != KV_OK) return st;
    return cuda_check(h, cudaStreamSynchronize(h->stream), "kv_set_initial_velocity");
}

kv_status kv_project_force(kv_handle *h, kv_field fx, kv_field fy, kv_field fz, double tol,
                           int max_iter, int mode, float *fs_out, kv_cg_stats *stats) {
    if (!h) return KV_ERR_ARG;
    if (h->sticky) return KV_ERR_STATE;
    if (mode < 0 || mode > 5)
        return set_error(h, KV_ERR_UNSUPPORTED, "projection mode %d is not available", mode);
    if ((mode == 4 || mode == 5) && h->precision != KV_FP32)
        return set_error(h, KV_ERR_UNSUPPORTED, "projection modes 4 and 5 (multigrid-preconditioned CG) need an FP32 handle");
    if ((mode == 1 || mode == 2 || mode == 5) && (!h->net || !kv_net_fits(h->net, h->nx, h->ny, h->nz)))
        return set_error(h, KV_ERR_STATE, "modes 1, 2 and 5 need a network attached with kv_attach_net that fits the grid");
    if (!(tol > 0.0)) return set_error(h, KV_ERR_ARG, "tol must be > 0");
    const kv_field *f[3] = {&fx, &fy, &fz};
    for (auto *q : f)
        if (!field_ok(*q) || (q->where == KV_SCALAR && q->value != 0.0))
            return set_error(h, KV_ERR_ARG, "force components must be arrays or 0");
    if (max_iter <= 0) max_iter = 20 * std::max(h->nx, std::max(h->ny, h->nz));
    kv_status st = cuda_check(h, cudaMemsetAsync(h->fstage, 0, 3 * (size_t)h->Np * 4, h->stream),
                              "kv_project_force");
    if (st != KV_OK) return st;
    for (int q = 0; q < 3; ++q)
        if (f[q]->where != KV_SCALAR && (st = stage(h, *f[q], h->fstage + q * h->Np)) != KV_OK) return st;
    free_graphs(h);
    h->have_force = 0;
    h->g_const_on = 0;
    return project(h, tol, max_iter, mode, fs_out, stats);
}

kv_status kv_set_cg_config(kv_handle *h, int zc) {
    if (!h || zc < 0) return set_error(h, KV_ERR_ARG, "kv_set_cg_config: invalid arguments");
    if (h->sticky) return KV_ERR_STATE;
    const long long gx = (h->px + 63) / 64, gy = (h->ny - 2 + 7) / 8;
    const int z = zc > 0 ? zc : cg_auto_zc(h);
    if (gx * gy * ((h->nz - 2 + z - 1) / z) > h->partials_len)
        return set_error(h, KV_ERR_ARG, "kv_set_cg_config: z chunk %d gives too many blocks", zc);
    h->cg_zc = zc;
    return KV_OK;
}

kv_status kv_get_cg_config(kv_handle *h, int *zc) {
    if (!h || !zc) return KV_ERR_ARG;
    *zc = h->cg_zc > 0 ? h->cg_zc : cg_auto_zc(h);
    return KV_OK;
}

kv_status kv_autotune_cg(kv_handle *h, kv_field fx, kv_field fy, kv_field fz, int iters, double *best_ms) {
    if (!h || iters < 1) return set_error(h, KV_ERR_ARG, "kv_autotune_cg: invalid arguments");
    if (h->sticky) return KV_ERR_STATE;
    if (h->precision != KV_FP32) {  // the FP64 passes have one fixed shape
        if (best_ms) *best_ms = 0.0;
        return KV_OK;
    }
    const int cand[] = {8, 16, 24, 32, 48, 64, 96, 128};
    const int saved = h->cg_zc, saved_ns = h->cg_ns;
    int best = -1, best_ns = saved_ns;
    double best_t = INFINITY;
    for (int ns : {8, 4}) {
        h->cg_ns = ns;
        for (int zc : cand) {
            if (zc > std::max(h->nz - 2, 8) || kv_set_cg_config(h, zc) != KV_OK) continue;
            double t = INFINITY;
            for (int rep = 0; rep < 2; ++rep) {  // the first run also warms the caches
                kv_cg_stats stc;
                kv_status st = kv_project_force(h, fx, fy, fz, 1e-30, iters, 0, nullptr, &stc);
                if (st != KV_OK && st != KV_CG_MAXITER) {
                    h->cg_zc = saved;
                    h->cg_ns = saved_ns;
                    return st;
                }
                t = std::min(t, stc.ms);
            }
            if (t < best_t) {
                best_t = t;
                best = zc;
                best_ns = ns;
            }
        }
    }
    h->cg_zc = best > 0 ? best : saved;
    h->cg_ns = best > 0 ? best_ns : saved_ns;
    h->have_force = 0;  // the trial projections stopped early: project again before stepping
    h->phi_valid = 0;
    if (best_ms) *best_ms = best_t;
    return KV_OK;
}

kv_status kv_step_force(kv_handle *h, kv_field fx, kv_field fy, kv_field fz, double tol, int max_iter,
                        int mode, kv_cg_stats *stats) {
    if (!h) return KV_ERR_ARG;
    if (h->sticky) return KV_ERR_STATE;
    if (mode != 0 && mode != 3 && mode != 4)
        return set_error(h, KV_ERR_ARG, "kv_step_force: mode must be 0, 3 or 4");
    if (mode == 4 && h->precision != KV_FP32)
        return set_error(h, KV_ERR_UNSUPPORTED, "kv_step_force: mode 4 needs an FP32 handle");
    if (!(tol > 0.0)) return set_error(h, KV_ERR_ARG, "tol must be > 0");
    const kv_field *f[3] = {&fx, &fy, &fz};
    for (auto *q : f)
        if (!field_ok(*q) || (q->where == KV_SCALAR && q->value != 0.0))
            return set_error(h, KV_ERR_ARG, "force components must be arrays or 0");
    if (max_iter <= 0) max_iter = 20 * std::max(h->nx, std::max(h->ny, h->nz));
    kv_status st = cuda_check(h, cudaMemsetAsync(h->fstage, 0, 3 * (size_t)h->Np * 4, h->stream),
                              "kv_step_force");
    if (st != KV_OK) return st;
    for (int q = 0; q < 3; ++q)
        if (f[q]->where != KV_SCALAR && (st = stage(h, *f[q], h->fstage + q * h->Np)) != KV_OK) return st;
    free_graphs(h);
    h->have_force = 0;
    // this step's force, projected on its own (mode 3: from the previous potential)
    if ((st = project(h, tol, max_iter, mode, nullptr, stats)) != KV_OK) return st;
    h->g_const_on = 1;
    st = step_launch(h, h->cur);
    h->g_const_on = 0;
    if (st != KV_OK) return st;
    h->cur = 1 - h->cur;
    h->steps_host++;
    return KV_OK;
}

kv_status kv_clear_force(kv_handle *h) {
    if (!h) return KV_ERR_ARG;
    h->have_force = 0;
    h->g_const_on = 0;
    free_graphs(h);
    return KV_OK;
}

namespace {
// Direct launches of n steps in the handle's current variant (no graph).
kv_status launch_steps_direct(kv_handle *h, int n) {
    kv_status st;
    if (h->precision == KV_FP32 && h->variant >= 2) {
        for (; n >= 2; n -= 2) {
            if ((st = step2_launch(h, h->cur)) != KV_OK) return st;
            h->cur = 1 - h->cur;
            h->steps_host += 2;
        }
    }
    for (; n > 0; --n) {
        if ((st = step_launch(h, h->cur)) != KV_OK) return st;
        h->cur = 1 - h->cur;
        h->steps_host++;
    }
    return KV_OK;
}
}  // namespace

kv_status kv_step(kv_handle *h, int n) {
    if (!h || n < 0) return set_error(h, KV_ERR_ARG, "kv_step: invalid arguments");
    if (h->sticky) return KV_ERR_STATE;
    kv_status st;
    const bool two = h->precision == KV_FP32 && h->variant >= 2;
    const int G = h->graph_steps;  // steps per graph; buffer swaps per graph stay even
    if (n >= G && G > 0 && G % 4 == 0) {
        if (!h->graph[h->cur]) {
            if (h->precision == KV_FP32 && h->variant != 1 && !h->tma_ready &&
                (st = step_prepare(h)) != KV_OK)
                return st;
            cudaGraph_t graph = nullptr;
            cudaError_t e = cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal);
            if ((st = cuda_check(h, e, "graph capture")) != KV_OK) return st;
            const long long before = h->launches;
            const int cur0 = h->cur;
            const long long steps0 = h->steps_host;
            st = launch_steps_direct(h, G);
            h->cur = cur0;  // the capture only records the launches
            h->steps_host = steps0;
            h->launches = before;
            e = cudaStreamEndCapture(h->stream, &graph);
            if (st != KV_OK) {
                if (graph) cudaGraphDestroy(graph);
                return st;
            }
            if ((st = cuda_check(h, e, "graph capture")) != KV_OK) return st;
            e = cudaGraphInstantiate(&h->graph[h->cur], graph, 0);
            cudaGraphDestroy(graph);
            if ((st = cuda_check(h, e, "graph instantiate")) != KV_OK) return st;
        }
        while (n >= G) {
            if ((st = cuda_check(h, cudaGraphLaunch(h->graph[h->cur], h->stream), "graph launch")) != KV_OK)
                return st;
            h->launches += two ? G / 2 : G;
            h->steps_host += G;
            n -= G;
        }
    }
    return launch_steps_direct(h, n);
}

long long kv_steps_taken(kv_handle *h) { return h ? h->steps_host : 0; }

long long kv_launch_count(kv_handle *h) { return h ? h->launches : 0; }

kv_status kv_sync(kv_handle *h) {
    if (!h) return KV_ERR_ARG;
    if (h->sticky) return KV_ERR_STATE;
    return poll_flags(h);
}

kv_status kv_read_traces(kv_handle *h, void *out, int where, int *n_written) {
    if (!h || (where != KV_HOST && where != KV_DEVICE))
        return set_error(h, KV_ERR_ARG, "kv_read_traces: invalid arguments");
    if (h->sticky) return KV_ERR_STATE;
    kv_status st = poll_flags(h);
    if (st != KV_OK) return st;
    const long long n = std::min<long long>(h->steps_host, h->cap);
    if (n_written) *n_written = (int)n;
    if (n == 0 || h->ns == 0) return KV_OK;
    if (!out) return set_error(h, KV_ERR_ARG, "kv_read_traces: out is NULL");
    cudaError_t e = cudaMemcpyAsync(out, h->traces, (size_t)n * h->ns * 3 * h->esize, cudaMemcpyDefault,
                                    h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    return cuda_check(h, e, "kv_read_traces");
}

kv_status kv_attach_net(kv_handle *h, kv_net *net) {
    if (!h) return KV_ERR_ARG;
    h->net = net;
    return KV_OK;
}

kv_status kv_read_field(kv_handle *h, int which, int comp, void *out, int where) {
    if (!h || !out || which < 0 || which > 4 || (which < 2 || which == 3) && (comp < 0 || comp > 2) ||
        (where != KV_HOST && where != KV_DEVICE))
        return set_error(h, KV_ERR_ARG, "kv_read_field: invalid arguments");
    if (h->sticky) return KV_ERR_STATE;
    kv_status st = poll_flags(h);
    if (st != KV_OK) return st;
    const char *src;
    size_t es = h->esize;
    if (which == 0) src = (const char *)h->state[h->cur] + (size_t)comp * h->Np * es;
    else if (which == 1) src = (const char *)h->state[h->cur] + (size_t)(3 + comp) * h->Np * es;
    else if (which == 2) { src = (const char *)h->phi; es = 8; }
    else if (which == 4) { src = (const char *)h->b; es = 8; }
    else src = (const char *)h->F + (size_t)comp * h->Np * es;
    cudaError_t e = cudaMemcpy2DAsync(out, (size_t)h->nx * es, src, (size_t)h->px * es, (size_t)h->nx * es,
                                      (size_t)h->ny * h->nz, cudaMemcpyDefault, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    return cuda_check(h, e, "kv_read_field");
}

kv_status kv_set_step_config(kv_handle *h, int variant, int tx, int ty, int zc, int ns) {
    if (!h) return KV_ERR_ARG;
    if (variant > 4 || (tx > 0 && tx != 32 && tx != 64 && tx != 128) ||
        (ty > 0 && ty != 2 && ty != 4 && ty != 8 && ty != 14 && ty != 16) ||
        (ns > 0 && ns != 2 && ns != 3 && ns != 4 && ns != 6 && ns != 8))
        return set_error(h, KV_ERR_ARG, "kv_set_step_config: invalid variant, tile or stage count");
    const int ntx = tx > 0 ? tx : h->tx, nty = ty > 0 ? ty : h->ty;
    const int nvar = variant >= 0 ? variant : h->variant;
    if ((nvar == 4) != (nty == 14))
        return set_error(h, KV_ERR_ARG, "kv_set_step_config: variant 4 takes tiles of 14 rows, the others not");
    if (nvar < 2 && (ntx * nty / 4 < 64 || ntx * nty / 4 > 512))
        return set_error(h, KV_ERR_ARG, "kv_set_step_config: tile %dx%d out of range", ntx, nty);
    cudaStreamSynchronize(h->stream);
    const int old[5] = {h->variant, h->tx, h->ty, h->zc, h->ns_stages};
    if (variant >= 0) h->variant = variant;
    h->tx = ntx;
    h->ty = nty;
    if (zc > 0) h->zc = zc;
    if (ns > 0) h->ns_stages = ns;
    h->tma_ready = 0;
    free_graphs(h);
    if (h->precision == KV_FP32 && h->variant != 1) {
        kv_status st = step_prepare(h);
        if (st != KV_OK) {  // keep the previous, valid configuration
            h->variant = old[0];
            h->tx = old[1];
            h->ty = old[2];
            h->zc = old[3];
            h->ns_stages = old[4];
            h->tma_ready = 0;
            return st;
        }
    }
    return KV_OK;
}

kv_status kv_get_step_config(kv_handle *h, int *cfg) {
    if (!h || !cfg) return KV_ERR_ARG;
    cfg[0] = h->variant;
    cfg[1] = h->tx;
    cfg[2] = h->ty;
    cfg[3] = h->zc;
    cfg[4] = h->ns_stages;
    return KV_OK;
}

kv_status kv_autotune_step(kv_handle *h, int trial_steps, double *best_ms) {
    if (!h || trial_steps < 1) return set_error(h, KV_ERR_ARG, "kv_autotune_step: invalid arguments");
    if (h->sticky) return KV_ERR_STATE;
    if (h->precision != KV_FP32) {
        if (best_ms) *best_ms = 0.0;
        return kv_reset(h);
    }
    struct Cand { int variant, tx, ty, ns, zc; };
    static const int tiles[][2] = {{32, 8}, {32, 16}, {64, 4}, {64, 8}, {64, 16}, {128, 2}, {128, 4}, {128, 8}};
    static const int tiles2[][2] = {{32, 4}, {32, 8}, {64, 4}, {64, 8}, {128, 4}};
    static const int tiles3[][2] = {{32, 8}, {32, 16}, {64, 4}, {64, 8}, {64, 16}, {128, 4}, {128, 8}};
    static const int zcs[] = {16, 32, 64};
    std::vector<Cand> cands;
    for (auto &t : tiles)
        for (int ns : {4, 6, 8})
            for (int zc : zcs) cands.push_back({0, t[0], t[1], ns, zc});
    for (auto &t : tiles2)
        for (int ns : {4, 6})
            for (int zc : zcs) cands.push_back({2, t[0], t[1], ns, zc});
    for (auto &t : tiles3)
        for (int ns : {4, 6})
            for (int zc : zcs) cands.push_back({3, t[0], t[1], ns, zc});
    // variant 4 marches whole columns best: add z chunks of a third, a half
    // and all of the interior depth (fewer chunks, less z halo per block)
    std::vector<int> zcs4 = {32, 64, 128};
    for (int parts : {3, 2, 1}) {
        const int zc = (h->nz - 2 + parts - 1) / parts;
        if (std::find(zcs4.begin(), zcs4.end(), zc) == zcs4.end()) zcs4.push_back(zc);
    }
    // three stages only: with four or six the 64- and 128-wide tiles spill at
    // the 96 registers of two blocks per SM, with two the copies' latency shows
    // (both slower in whole passes; short trials can rank them first)
    for (int tx : {32, 64, 128})
        for (int zc : zcs4) cands.push_back({4, tx, 14, 3, zc});
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
        return set_error(h, KV_ERR_CUDA, "kv_autotune_step: cudaEventCreate failed");
    const int saved[5] = {h->variant, h->tx, h->ty, h->zc, h->ns_stages};
    double best = INFINITY;
    Cand pick = {saved[0], saved[1], saved[2], saved[4], saved[3]};
    kv_status st = KV_OK;
    const int trial = trial_steps + (trial_steps & 1);  // even: whole two-step launches
    // time one candidate over n steps (after two warm-up steps); < 0 if it cannot run
    auto time_cand = [&](const Cand &c, int n, float *ms) -> kv_status {
        *ms = -1.f;
        if (kv_set_step_config(h, c.variant, c.tx, c.ty, c.zc, c.ns) != KV_OK) return KV_OK;
        kv_status ts;
        if ((ts = launch_steps_direct(h, 2)) != KV_OK) return ts;
        cudaEventRecord(e0, h->stream);
        if ((ts = launch_steps_direct(h, n)) != KV_OK) return ts;
        cudaEventRecord(e1, h->stream);
        if ((ts = cuda_check(h, cudaEventSynchronize(e1), "kv_autotune_step")) != KV_OK) return ts;
        cudaEventElapsedTime(ms, e0, e1);
        return KV_OK;
    };
    // first pass: every candidate over `trial` steps; second pass: the four
    // fastest again over four times as many steps, so that near-ties are
    // decided on a longer sample
    std::vector<std::pair<float, Cand>> timed;
    for (const Cand &c : cands) {
        float ms = 0.f;
        if ((st = time_cand(c, trial, &ms)) != KV_OK) break;
        if (ms > 0.f) timed.push_back({ms, c});
    }
    if (st == KV_OK) {
        std::sort(timed.begin(), timed.end(),
                  [](const std::pair<float, Cand> &a, const std::pair<float, Cand> &b) { return a.first < b.first; });
        // the second pass also takes the fastest one-step candidate: a two-step
        // kernel (half the DRAM bytes, but bound by issue rate) is kept only
        // when it beats the best one-step kernel (bound by HBM) by 3 %
        std::vector<Cand> finals;
        for (size_t q = 0; q < timed.size() && q < 4; ++q) finals.push_back(timed[q].second);
        for (const auto &tc : timed)
            if (tc.second.variant < 2) {
                bool have = false;
                for (const Cand &f : finals) have |= (f.variant == tc.second.variant && f.tx == tc.second.tx &&
                                                      f.ty == tc.second.ty && f.ns == tc.second.ns &&
                                                      f.zc == tc.second.zc);
                if (!have) finals.push_back(tc.second);
                break;
            }
        double best_one = INFINITY, best_two = INFINITY;
        Cand pick_one = pick, pick_two = pick;
        for (const Cand &c : finals) {
            float ms = 0.f;
            if ((st = time_cand(c, 4 * trial, &ms)) != KV_OK) break;
            if (!(ms > 0.f)) continue;
            const double per = ms / 4.0;
            if (c.variant < 2 && per < best_one) {
                best_one = per;
                pick_one = c;
            }
            if (c.variant >= 2 && per < best_two) {
                best_two = per;
                pick_two = c;
            }
        }
        if (best_one <= 1.03 * best_two) {
            best = best_one;
            pick = pick_one;
        } else {
            best = best_two;
            pick = pick_two;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != KV_OK) return st;
    if ((st = kv_set_step_config(h, pick.variant, pick.tx, pick.ty, pick.zc, pick.ns)) != KV_OK) return st;
    if (best_ms) *best_ms = best / trial;
    return kv_reset(h);
}

}  // extern "C"
