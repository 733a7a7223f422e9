// kv_fcg.cu -- projection mode 2: flexible CG with the attached network as a
// (nonlinear) preconditioner.
//
// The system and the stopping test are the paper's (Sec. 3.2.3: A phi = b,
// A = -L on interior nodes, phi = 0 on the outer layer, stop on the relative
// residual); only the search directions change. The network maps a
// right-hand side to an approximate potential, so z = Net(r) approximates
// A^-1 r. Because Net is not a fixed linear operator, the iteration is the
// flexible (inexact-preconditioner) form of CG in which beta takes the
// Polak-Ribiere quotient (Golub & Ye, "Inexact preconditioned conjugate
// gradient method with inner-outer iteration", SISC 1999; Notay's flexible
// CG with one stored direction):
//   r0 = b - A phi0, z0 = Net(r0), p0 = z0
//   alpha_k = (z_k . r_k) / (p_k . A p_k)
//   phi_{k+1} = phi_k + alpha_k p_k,  r_{k+1} = r_k - alpha_k A p_k
//   z_{k+1} = Net(r_{k+1})
//   beta_k = z_{k+1} . (r_{k+1} - r_k) / (z_k . r_k)
//   p_{k+1} = z_{k+1} + beta_k p_k
// All vectors are FP64 (pitched like the handle); the dots are summed per
// block and then in a fixed order on the host, so the result is
// deterministic. When the recursive residual meets the tolerance the true
// residual b - A phi is formed; if it does not, it replaces r and the
// iteration goes on. One network inference per iteration dominates the cost.
#include <math.h>

#include <vector>

#include "kv_internal.cuh"

namespace kv {

constexpr int kFcgBlocks = 148 * 8;
constexpr int kFcgThreads = 256;

struct FcgGrid {
    int nx, ny, nz, px;
    long long Np;
    double inv_dx2;
};

__device__ __forceinline__ bool fcg_interior(long long c, const FcgGrid &g) {
    const int i = (int)(c % g.px);
    const long long r = c / g.px;
    const int j = (int)(r % g.ny), k = (int)(r / g.ny);
    return i >= 1 && i <= g.nx - 2 && j >= 1 && j <= g.ny - 2 && k >= 1 && k <= g.nz - 2;
}

__device__ __forceinline__ double fcg_block_sum(double v) {
    __shared__ double sh[kFcgThreads / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < kFcgThreads / 32; ++w) s += sh[w];
    __syncthreads();
    return s;
}

// q = A p on interior nodes (0 elsewhere); partial[block] = sum p.q
__global__ void __launch_bounds__(kFcgThreads)
k_fcg_apply(const double *__restrict__ p, double *__restrict__ q, FcgGrid g, double *__restrict__ part) {
    const long long sy = g.px, sz = (long long)g.px * g.ny;
    double acc = 0.0;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < g.Np;
         c += (long long)gridDim.x * blockDim.x) {
        double v = 0.0;
        if (fcg_interior(c, g)) {
            const double s = ((p[c - 1] + p[c + 1]) + (p[c - sy] + p[c + sy])) + (p[c - sz] + p[c + sz]);
            v = (6.0 * p[c] - s) * g.inv_dx2;
            acc += p[c] * v;
        }
        q[c] = v;
    }
    const double t = fcg_block_sum(acc);
    if (threadIdx.x == 0) part[blockIdx.x] = t;
}

// r = b - A phi (interior), partial = |r|^2
__global__ void __launch_bounds__(kFcgThreads)
k_fcg_residual(const double *__restrict__ b, const double *__restrict__ phi, double *__restrict__ r, FcgGrid g,
               double *__restrict__ part) {
    const long long sy = g.px, sz = (long long)g.px * g.ny;
    double acc = 0.0;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < g.Np;
         c += (long long)gridDim.x * blockDim.x) {
        double v = 0.0;
        if (fcg_interior(c, g)) {
            const double s = ((phi[c - 1] + phi[c + 1]) + (phi[c - sy] + phi[c + sy])) +
                             (phi[c - sz] + phi[c + sz]);
            v = b[c] - (6.0 * phi[c] - s) * g.inv_dx2;
            acc += v * v;
        }
        r[c] = v;
    }
    const double t = fcg_block_sum(acc);
    if (threadIdx.x == 0) part[blockIdx.x] = t;
}

// phi += alpha p; r_old = r; r -= alpha q; partial = |r|^2
__global__ void __launch_bounds__(kFcgThreads)
k_fcg_update(double *__restrict__ phi, double *__restrict__ r, double *__restrict__ r_old,
             const double *__restrict__ p, const double *__restrict__ q, double alpha, long long Np,
             double *__restrict__ part) {
    double acc = 0.0;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < Np;
         c += (long long)gridDim.x * blockDim.x) {
        phi[c] += alpha * p[c];
        const double rv = r[c];
        r_old[c] = rv;
        const double rn = rv - alpha * q[c];
        r[c] = rn;
        acc += rn * rn;
    }
    const double t = fcg_block_sum(acc);
    if (threadIdx.x == 0) part[blockIdx.x] = t;
}

// partials: [0] z.r, [1] z.(r - r_old) (r_old may be NULL: then 0)
__global__ void __launch_bounds__(kFcgThreads)
k_fcg_zdots(const double *__restrict__ z, const double *__restrict__ r, const double *__restrict__ r_old,
            long long Np, double *__restrict__ part) {
    double a = 0.0, c2 = 0.0;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < Np;
         c += (long long)gridDim.x * blockDim.x) {
        const double zv = z[c], rv = r[c];
        a += zv * rv;
        if (r_old) c2 += zv * (rv - r_old[c]);
    }
    const double ta = fcg_block_sum(a);
    const double tc = fcg_block_sum(c2);
    if (threadIdx.x == 0) {
        part[blockIdx.x] = ta;
        part[gridDim.x + blockIdx.x] = tc;
    }
}

// p = z + beta p
__global__ void k_fcg_direction(double *__restrict__ p, const double *__restrict__ z, double beta, long long Np) {
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < Np;
         c += (long long)gridDim.x * blockDim.x)
        p[c] = z[c] + beta * p[c];
}

// pitched double <-> dense float for the network (interior nodes of z kept)
__global__ void k_fcg_to_dense(const double *__restrict__ a, float *__restrict__ o, int nx, int ny, int nz, int px) {
    const long long n = (long long)nx * ny * nz;
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < n; v += (long long)gridDim.x * blockDim.x)
        o[v] = (float)a[(v / nx) * px + v % nx];
}
__global__ void k_fcg_from_dense(const float *__restrict__ a, double *__restrict__ o, int nx, int ny, int nz,
                                 int px) {
    const long long n = (long long)nx * ny * nz;
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < n; v += (long long)gridDim.x * blockDim.x) {
        const long long r = v / nx;
        const int i = (int)(v % nx), j = (int)(r % ny), k = (int)(r / ny);
        const bool in = i >= 1 && i <= nx - 2 && j >= 1 && j <= ny - 2 && k >= 1 && k <= nz - 2;
        o[r * px + i] = in ? (double)a[v] : 0.0;
    }
}

namespace {

// Sum the block partials of one or two quantities on the host, in block order.
kv_status fcg_sums(kv_handle *h, const double *part_dev, int nq, double *out) {
    std::vector<double> hp((size_t)nq * kFcgBlocks);
    cudaError_t e = cudaMemcpyAsync(hp.data(), part_dev, hp.size() * sizeof(double), cudaMemcpyDeviceToHost,
                                    h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_check(h, e, "flexible CG reduction");
    for (int q = 0; q < nq; ++q) {
        double s = 0.0;
        for (int b = 0; b < kFcgBlocks; ++b) s += hp[(size_t)q * kFcgBlocks + b];
        out[q] = s;
    }
    return KV_OK;
}

// z = Net(r) through the network's dense staging buffers
kv_status fcg_precondition(kv_handle *h, const double *r, double *z) {
    k_fcg_to_dense<<<kFcgBlocks, kFcgThreads, 0, h->stream>>>(r, kv_net_stage_b(h->net), h->nx, h->ny, h->nz,
                                                              h->px);
    cudaError_t e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_check(h, e, "flexible CG: network input");
    kv_status st = kv_net_predict(h->net, h->nx, h->ny, h->nz, h->dx, kv_net_stage_b(h->net),
                                  kv_net_stage_phi(h->net));
    if (st != KV_OK) return set_error(h, st, "flexible CG: network inference failed");
    k_fcg_from_dense<<<kFcgBlocks, kFcgThreads, 0, h->stream>>>(kv_net_stage_phi(h->net), z, h->nx, h->ny,
                                                                h->nz, h->px);
    h->launches += 2;
    return cuda_check(h, cudaGetLastError(), "flexible CG: network output");
}

}  // namespace

// Mode 2 of kv_project_force. h->b holds the right-hand side (k_rhs); on return
// h->phi holds the potential. status: KV_OK, KV_CG_MAXITER, KV_CG_BREAKDOWN or
// KV_ERR_NONFINITE; iters, true residual^2 and |b|^2 in the outputs.
kv_status project_fcg(kv_handle *h, double tol, int max_iter, int *status, int *iters, double *true2,
                      double bb) {
    const long long Np = h->Np;
    if (!h->fcg_pool) {
        // r, r_old, z, p, q and the partials, allocated on first use and kept
        cudaError_t e = cudaMalloc(&h->fcg_pool, (5 * Np + 2 * kFcgBlocks) * sizeof(double));
        if (e != cudaSuccess) {
            h->fcg_pool = nullptr;
            return set_error(h, KV_ERR_OOM, "flexible CG: allocation of %lld doubles failed", 5 * Np);
        }
        // zeros: the row padding of every vector stays 0 (no kernel writes it)
        e = cudaMemsetAsync(h->fcg_pool, 0, (5 * Np + 2 * kFcgBlocks) * sizeof(double), h->stream);
        if (e != cudaSuccess) return cuda_check(h, e, "flexible CG memset");
    }
    double *r = h->fcg_pool, *r_old = r + Np, *z = r_old + Np, *p = z + Np, *q = p + Np, *part = q + Np;
    cudaStream_t s = h->stream;
    const FcgGrid g{h->nx, h->ny, h->nz, h->px, Np, 1.0 / (h->dx * h->dx)};
    const double stop2 = tol * tol * bb;
    kv_status st;
    double v[2];
    *status = KV_OK;
    *iters = 0;
    // phi = 0, r = b - A phi = b (interior)
    cudaError_t e = cudaMemsetAsync(h->phi, 0, Np * sizeof(double), s);
    if (e != cudaSuccess) return cuda_check(h, e, "flexible CG memset");
    k_fcg_residual<<<kFcgBlocks, kFcgThreads, 0, s>>>(h->b, h->phi, r, g, part);
    h->launches++;
    if ((st = fcg_sums(h, part, 1, v)) != KV_OK) return st;
    double rr = v[0];
    if ((st = fcg_precondition(h, r, z)) != KV_OK) return st;
    k_fcg_zdots<<<kFcgBlocks, kFcgThreads, 0, s>>>(z, r, nullptr, Np, part);
    h->launches++;
    if ((st = fcg_sums(h, part, 2, v)) != KV_OK) return st;
    double zr = v[0];
    if ((e = cudaMemcpyAsync(p, z, Np * sizeof(double), cudaMemcpyDeviceToDevice, s)) != cudaSuccess)
        return cuda_check(h, e, "flexible CG copy");
    int it = 0;
    while (true) {
        if (!isfinite(rr) || !isfinite(zr)) {
            *status = KV_ERR_NONFINITE;
            break;
        }
        if (rr < stop2) {  // recursive residual met: check the true one
            k_fcg_residual<<<kFcgBlocks, kFcgThreads, 0, s>>>(h->b, h->phi, r, g, part);
            h->launches++;
            if ((st = fcg_sums(h, part, 1, v)) != KV_OK) return st;
            rr = v[0];
            if (rr < stop2) break;
            // the true residual replaces the recursive one; restart the directions
            if ((st = fcg_precondition(h, r, z)) != KV_OK) return st;
            k_fcg_zdots<<<kFcgBlocks, kFcgThreads, 0, s>>>(z, r, nullptr, Np, part);
            h->launches++;
            if ((st = fcg_sums(h, part, 2, v)) != KV_OK) return st;
            zr = v[0];
            if ((e = cudaMemcpyAsync(p, z, Np * sizeof(double), cudaMemcpyDeviceToDevice, s)) != cudaSuccess)
                return cuda_check(h, e, "flexible CG copy");
            continue;
        }
        if (it >= max_iter) {
            *status = KV_CG_MAXITER;
            break;
        }
        k_fcg_apply<<<kFcgBlocks, kFcgThreads, 0, s>>>(p, q, g, part);
        h->launches++;
        if ((st = fcg_sums(h, part, 1, v)) != KV_OK) return st;
        const double pq = v[0];
        if (!isfinite(pq) || pq <= 0.0) {
            *status = KV_CG_BREAKDOWN;
            break;
        }
        const double alpha = zr / pq;
        k_fcg_update<<<kFcgBlocks, kFcgThreads, 0, s>>>(h->phi, r, r_old, p, q, alpha, Np, part);
        h->launches++;
        if ((st = fcg_sums(h, part, 1, v)) != KV_OK) return st;
        rr = v[0];
        ++it;
        if (rr < stop2 || !isfinite(rr)) continue;  // checked at the top of the loop
        if ((st = fcg_precondition(h, r, z)) != KV_OK) return st;
        k_fcg_zdots<<<kFcgBlocks, kFcgThreads, 0, s>>>(z, r, r_old, Np, part);
        h->launches++;
        if ((st = fcg_sums(h, part, 2, v)) != KV_OK) return st;
        const double beta = v[1] / zr;  // Polak-Ribiere: z_{k+1}.(r_{k+1} - r_k) / (z_k . r_k)
        zr = v[0];
        k_fcg_direction<<<kFcgBlocks, kFcgThreads, 0, s>>>(p, z, beta, Np);
        h->launches++;
    }
    *iters = it;
    // the true residual of the potential returned, whatever ended the loop
    k_fcg_residual<<<kFcgBlocks, kFcgThreads, 0, s>>>(h->b, h->phi, r_old, g, part);
    h->launches++;
    if ((st = fcg_sums(h, part, 1, v)) != KV_OK) return st;
    *true2 = v[0];
    return cuda_check(h, cudaGetLastError(), "flexible CG");
}

}  // namespace kv
