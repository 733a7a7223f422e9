// kv_mg.cu -- multigrid preconditioner of the projection's CG (mode 4 of
// kv_project_force). The system is the paper's (Sec. 3.2.3: A phi = b,
// A = -L, phi = 0 on the outer layer) and the stop test the same true
// residual; only the Krylov iteration is preconditioned, so it needs a few
// tens of iterations instead of hundreds.
//
// M is one symmetric V(1,1)-cycle on a cell-centred hierarchy of the interior
// unknowns: a level of n cells per axis coarsens to ceil(n/2) cells, coarse
// cell I covering fine cells 2I-1 and 2I, spacing doubled. With D = 6/h^2
// (the diagonal of A) and S = omega D^-1:
//   pre-smoothing from zero      z1 = S r
//   residual, restriction        r_c = R (r - A z1)
//   coarse correction            e_c = M_c r_c            (recursively)
//   prolongation                 z2 = z1 + P e_c
//   post-smoothing               z  = z2 + S (r - A z2)
// P is trilinear (weights 3/4 and 1/4 per axis towards the nearer and the
// farther coarse cell, ghost cells 0) and R = P^T / 8, so M = (2S - SAS) +
// (I - SA) P M_c R (I - AS) is symmetric and, for omega < 1 (D^-1 A has
// eigenvalues below 2), positive definite: plain preconditioned CG applies.
// The coarsest level (at most a few thousand cells) is solved approximately by
// a fixed number of damped Jacobi sweeps in one block's shared memory, a
// polynomial in A and so symmetric too.
//
// Every kernel returns at once unless the CG control word says "running", so
// the host can queue several iterations between polls, as for the plain CG.
#include <math.h>

#include <algorithm>

#include "kv_internal.cuh"
#include "kv_reduce.cuh"

namespace kv {

constexpr float kMgOmega = 6.f / 7.f;   // damped Jacobi weight of the smoother
constexpr int kMgCoarseMax = 4096;       // cells of the coarsest level (one block)
constexpr int kMgCoarseSweeps = 32;      // Jacobi sweeps of the coarsest solve
constexpr int kMgBX = 32, kMgBY = 8;     // 2D blocks over (x, y), z loop

__device__ __forceinline__ long long mg_idx(const MgLevel &L, int i, int j, int k) {
    return ((long long)k * (L.ny + 2) + j) * L.px + i;
}

__device__ __forceinline__ bool mg_running(const CgParams &p) {
    return __ldcg(&p.ctrl[kCgStatus]) == kCgRunning;
}

// Cells k = k0 .. k1 of this block's contiguous z chunk (gridDim.z chunks).
__device__ __forceinline__ void mg_chunk(int nz, int &k0, int &k1) {
    const int zc = (nz + (int)gridDim.z - 1) / (int)gridDim.z;
    k0 = 1 + (int)blockIdx.z * zc;
    k1 = min(nz, k0 + zc - 1);
}

// t = r - A (S r) = (1 - omega) r + (omega / 6) (sum of the six neighbours of r)
// on interior cells (r is 0 on the ghost layer). Each thread marches its z
// chunk with the z-1, z and z+1 values of r in registers.
__global__ void __launch_bounds__(kMgBX *kMgBY)
k_mg_pre(MgLevel L, CgParams p) {
    if (!mg_running(p)) return;
    const int i = 1 + blockIdx.x * kMgBX + (threadIdx.x % kMgBX);
    const int j = 1 + blockIdx.y * kMgBY + (threadIdx.x / kMgBX);
    if (i > L.nx || j > L.ny) return;
    const long long sy = L.px, sz = (long long)L.px * (L.ny + 2);
    int k0, k1;
    mg_chunk(L.nz, k0, k1);
    if (k0 > k1) return;
    long long c = mg_idx(L, i, j, k0);
    float rm = L.r[c - sz], rc = L.r[c];
    for (int k = k0; k <= k1; ++k, c += sz) {
        const float rp = L.r[c + sz];
        const float s = ((L.r[c - 1] + L.r[c + 1]) + (L.r[c - sy] + L.r[c + sy])) + (rm + rp);
        L.t[c] = (1.f - kMgOmega) * rc + (kMgOmega / 6.f) * s;
        rm = rc;
        rc = rp;
    }
}

// Per-axis weights of R = P^T / 8 over fine cells 2I-2, 2I-1, 2I, 2I+1.
__device__ __forceinline__ float mg_rw(int a) { return (a == 1 || a == 2) ? 0.75f : 0.25f; }

// r_c(I, J, K) = (1/8) sum of w_a w_b w_c t_f over the 4 x 4 x 4 fine cells
// 2I-2 .. 2I+1 (per axis) that are interior.
__global__ void __launch_bounds__(kMgBX *kMgBY)
k_mg_restrict(MgLevel F, MgLevel C, CgParams p) {
    if (!mg_running(p)) return;
    const int I = 1 + blockIdx.x * kMgBX + (threadIdx.x % kMgBX);
    const int J = 1 + blockIdx.y * kMgBY + (threadIdx.x / kMgBX);
    if (I > C.nx || J > C.ny) return;
    int K0, K1;
    mg_chunk(C.nz, K0, K1);
    for (int K = K0; K <= K1; ++K) {
        float acc = 0.f;
        for (int c = 0; c < 4; ++c) {
            const int k = 2 * K - 2 + c;
            if (k < 1 || k > F.nz) continue;
            float accy = 0.f;
            for (int b = 0; b < 4; ++b) {
                const int j = 2 * J - 2 + b;
                if (j < 1 || j > F.ny) continue;
                float accx = 0.f;
                for (int a = 0; a < 4; ++a) {
                    const int i = 2 * I - 2 + a;
                    if (i < 1 || i > F.nx) continue;
                    accx += mg_rw(a) * F.t[mg_idx(F, i, j, k)];
                }
                accy += mg_rw(b) * accx;
            }
            acc += mg_rw(c) * accy;
        }
        C.r[mg_idx(C, I, J, K)] = 0.125f * acc;
    }
}

// Trilinear prolongation of the coarse solution at fine cell (i, j, k).
__device__ __forceinline__ float mg_prolong(const MgLevel &C, int i, int j, int k) {
    const int I = (i + 1) >> 1, J = (j + 1) >> 1, K = (k + 1) >> 1;
    const int I2 = (i & 1) ? I - 1 : I + 1, J2 = (j & 1) ? J - 1 : J + 1, K2 = (k & 1) ? K - 1 : K + 1;
    const float *e = C.e;
    auto at = [&](int a, int b, int c) { return e[mg_idx(C, a, b, c)]; };
    const float x0 = 0.75f * at(I, J, K) + 0.25f * at(I2, J, K);
    const float x1 = 0.75f * at(I, J2, K) + 0.25f * at(I2, J2, K);
    const float x2 = 0.75f * at(I, J, K2) + 0.25f * at(I2, J, K2);
    const float x3 = 0.75f * at(I, J2, K2) + 0.25f * at(I2, J2, K2);
    const float y0 = 0.75f * x0 + 0.25f * x1;
    const float y1 = 0.75f * x2 + 0.25f * x3;
    return 0.75f * y0 + 0.25f * y1;
}

// z2 = S r + P e_c on interior fine cells, stored in F.t (free once the
// restriction has read it).
__global__ void __launch_bounds__(kMgBX *kMgBY)
k_mg_prolong(MgLevel F, MgLevel C, CgParams p) {
    if (!mg_running(p)) return;
    const int i = 1 + blockIdx.x * kMgBX + (threadIdx.x % kMgBX);
    const int j = 1 + blockIdx.y * kMgBY + (threadIdx.x / kMgBX);
    if (i > F.nx || j > F.ny) return;
    const float sh = kMgOmega * (float)F.h2 / 6.f;
    int k0, k1;
    mg_chunk(F.nz, k0, k1);
    for (int k = k0; k <= k1; ++k) {
        const long long c = mg_idx(F, i, j, k);
        F.t[c] = sh * F.r[c] + mg_prolong(C, i, j, k);
    }
}

// z = z2 + S (r - A z2) with z2 in F.t (0 on the ghost layer); out: the
// level's solution (F.e), or at level 0 the CG's z (out_z, pitched like the
// handle) with r.z reduced: beta and scal[kRR].
__global__ void __launch_bounds__(kMgBX *kMgBY)
k_mg_smooth(MgLevel F, float *__restrict__ out_z, CgParams p) {
    if (!mg_running(p)) return;
    const int i = 1 + blockIdx.x * kMgBX + (threadIdx.x % kMgBX);
    const int j = 1 + blockIdx.y * kMgBY + (threadIdx.x / kMgBX);
    const long long sy = F.px, sz = (long long)F.px * (F.ny + 2);
    const float h2 = (float)F.h2;
    AccFF acc;
    int k0, k1;
    mg_chunk(F.nz, k0, k1);
    if (i <= F.nx && j <= F.ny && k0 <= k1) {
        // z march with the z-1, z and z+1 values of z2 in registers
        const float *t = F.t;
        long long c = mg_idx(F, i, j, k0);
        float tm = t[c - sz], zc = t[c];
        for (int k = k0; k <= k1; ++k, c += sz) {
            const float tp = t[c + sz];
            const float s = ((t[c - 1] + t[c + 1]) + (t[c - sy] + t[c + sy])) + (tm + tp);
            const float rv = F.r[c];
            // S (r - A z2) = (omega / 6) (h^2 r - 6 z2 + sum of neighbours)
            const float z = zc + (kMgOmega / 6.f) * (h2 * rv - 6.f * zc + s);
            if (out_z) {
                out_z[c] = z;
                acc.add_prod(rv, z);
            } else {
                F.e[c] = z;
            }
            tm = zc;
            zc = tp;
        }
    }
    if (!out_z) return;
    double v[1] = {acc.value()}, sm[1];
    if (last_block_sums<1>(p, v, sm) && threadIdx.x == 0) {
        const double rz = sm[0];
        if (!isfinite(rz)) {
            p.ctrl[kCgStatus] = kCgNonfinite;
        } else if (rz <= 0.0) {
            p.ctrl[kCgStatus] = kCgBreakdown;
        } else {
            const double rz_prev = p.scal[kRR];
            p.scal[kBeta] = (p.ctrl[kCgIters] == 0 || rz_prev <= 0.0) ? 0.0 : rz / rz_prev;
            p.scal[kRR] = rz;
        }
    }
}

// Grids too small to coarsen: M = S (diagonal scaling), z = S r, r.z reduced.
__global__ void __launch_bounds__(kMgBX *kMgBY)
k_mg_diag(MgLevel F, float *__restrict__ out_z, CgParams p) {
    if (!mg_running(p)) return;
    const int i = 1 + blockIdx.x * kMgBX + (threadIdx.x % kMgBX);
    const int j = 1 + blockIdx.y * kMgBY + (threadIdx.x / kMgBX);
    const float sh = kMgOmega * (float)F.h2 / 6.f;
    AccFF acc;
    if (i <= F.nx && j <= F.ny) {
        for (int k = 1 + blockIdx.z; k <= F.nz; k += gridDim.z) {
            const long long c = mg_idx(F, i, j, k);
            const float z = sh * F.r[c];
            out_z[c] = z;
            acc.add_prod(F.r[c], z);
        }
    }
    double v[1] = {acc.value()}, sm[1];
    if (last_block_sums<1>(p, v, sm) && threadIdx.x == 0) {
        const double rz = sm[0];
        if (!isfinite(rz)) {
            p.ctrl[kCgStatus] = kCgNonfinite;
        } else if (rz <= 0.0) {
            p.ctrl[kCgStatus] = kCgBreakdown;
        } else {
            const double rz_prev = p.scal[kRR];
            p.scal[kBeta] = (p.ctrl[kCgIters] == 0 || rz_prev <= 0.0) ? 0.0 : rz / rz_prev;
            p.scal[kRR] = rz;
        }
    }
}

// Coarsest level: kMgCoarseSweeps damped Jacobi sweeps from e = S r, in one
// block's shared memory (ping-pong), ghost cells 0.
__global__ void __launch_bounds__(1024)
k_mg_coarse(MgLevel L, CgParams p) {
    if (!mg_running(p)) return;
    extern __shared__ float sm[];
    const int n = (L.nx + 2) * (L.ny + 2) * (L.nz + 2);
    float *a = sm, *b = sm + n, *rr = sm + 2 * n;
    const int sx = L.nx + 2, sy = (L.nx + 2) * (L.ny + 2);
    const float sh = kMgOmega * (float)L.h2 / 6.f;
    for (int q = threadIdx.x; q < n; q += blockDim.x) {
        const int i = q % sx, j = (q / sx) % (L.ny + 2), k = q / sy;
        const bool in = i >= 1 && i <= L.nx && j >= 1 && j <= L.ny && k >= 1 && k <= L.nz;
        const float rv = in ? L.r[mg_idx(L, i, j, k)] : 0.f;
        rr[q] = rv;
        a[q] = sh * rv;
        b[q] = 0.f;
    }
    __syncthreads();
    for (int it = 0; it < kMgCoarseSweeps; ++it) {
        for (int q = threadIdx.x; q < n; q += blockDim.x) {
            const int i = q % sx, j = (q / sx) % (L.ny + 2), k = q / sy;
            const bool in = i >= 1 && i <= L.nx && j >= 1 && j <= L.ny && k >= 1 && k <= L.nz;
            if (!in) continue;
            const float s = ((a[q - 1] + a[q + 1]) + (a[q - sx] + a[q + sx])) + (a[q - sy] + a[q + sy]);
            b[q] = a[q] + (kMgOmega / 6.f) * ((float)L.h2 * rr[q] - 6.f * a[q] + s);
        }
        __syncthreads();
        float *t = a;
        a = b;
        b = t;
    }
    for (int q = threadIdx.x; q < n; q += blockDim.x) {
        const int i = q % sx, j = (q / sx) % (L.ny + 2), k = q / sy;
        const bool in = i >= 1 && i <= L.nx && j >= 1 && j <= L.ny && k >= 1 && k <= L.nz;
        if (in) L.e[mg_idx(L, i, j, k)] = a[q];
    }
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
kv_status mg_prepare(kv_handle *h) {
    if (h->mg_levels > 0) return KV_OK;
    MgLevel L[kMgMaxLevels];
    int nl = 0;
    {
        MgLevel &f = L[nl++];
        f.nx = h->nx - 2;
        f.ny = h->ny - 2;
        f.nz = h->nz - 2;
        f.px = h->px;
        f.n = h->Np;
        f.h2 = h->dx * h->dx;
    }
    while (nl < kMgMaxLevels) {
        const MgLevel &f = L[nl - 1];
        if ((long long)f.nx * f.ny * f.nz <= 64 || std::min(f.nx, std::min(f.ny, f.nz)) < 4) break;
        MgLevel c;
        c.nx = (f.nx + 1) / 2;
        c.ny = (f.ny + 1) / 2;
        c.nz = (f.nz + 1) / 2;
        c.px = c.nx + 2;
        c.n = (long long)c.px * (c.ny + 2) * (c.nz + 2);
        c.h2 = 4.0 * f.h2;
        L[nl++] = c;
    }
    const MgLevel &last = L[nl - 1];
    if ((long long)(last.nx + 2) * (last.ny + 2) * (last.nz + 2) > kMgCoarseMax)
        return set_error(h, KV_ERR_UNSUPPORTED,
                         "multigrid: coarsest level %dx%dx%d too large for the one-block solve (grid too anisotropic)",
                         last.nx, last.ny, last.nz);
    // fine level: r and t (pitched, Np each); coarse levels: r, e, t
    long long total = 2 * h->Np;
    for (int l = 1; l < nl; ++l) total += 3 * L[l].n;
    float *pool = nullptr;
    cudaError_t e = cudaMalloc(&pool, total * sizeof(float));
    if (e != cudaSuccess) return cuda_check(h, e, "multigrid allocation");
    e = cudaMemsetAsync(pool, 0, total * sizeof(float), h->stream);
    if (e != cudaSuccess) {
        cudaFree(pool);
        return cuda_check(h, e, "multigrid memset");
    }
    float *q = pool;
    L[0].r = q;
    q += h->Np;
    L[0].t = q;
    q += h->Np;
    L[0].e = nullptr;  // level 0 writes the CG's z
    for (int l = 1; l < nl; ++l) {
        L[l].r = q;
        q += L[l].n;
        L[l].e = q;
        q += L[l].n;
        L[l].t = q;
        q += L[l].n;
    }
    kv_status st = encode_tensor_4d(h, &h->tm_mg_r, L[0].r, 1, 64, 8, 1);
    if (st != KV_OK) {
        cudaFree(pool);
        return st;
    }
    const size_t smem = (size_t)3 * (last.nx + 2) * (last.ny + 2) * (last.nz + 2) * sizeof(float);
    e = cudaFuncSetAttribute(k_mg_coarse, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) {
        cudaFree(pool);
        return cuda_check(h, e, "multigrid coarse solve attribute");
    }
    for (int l = 0; l < nl; ++l) h->mg[l] = L[l];
    h->mg_pool = pool;
    h->mg_levels = nl;
    return KV_OK;
}

static dim3 mg_grid(const MgLevel &L, int zsplit) {
    return dim3((L.nx + kMgBX - 1) / kMgBX, (L.ny + kMgBY - 1) / kMgBY, std::max(1, std::min(L.nz, zsplit)));
}

void mg_apply(kv_handle *h, const CgParams &p) {
    const int nl = h->mg_levels;
    const int nt = kMgBX * kMgBY;
    cudaStream_t s = h->stream;
    // level 0 reduces r.z over its blocks: at most partials_len blocks
    const MgLevel &f = h->mg[0];
    const long long gxy = (long long)((f.nx + kMgBX - 1) / kMgBX) * ((f.ny + kMgBY - 1) / kMgBY);
    const int zs0 = (int)std::max(1ll, std::min(16ll, h->partials_len / gxy));
    CgParams q = p;
    const dim3 g0 = mg_grid(f, zs0);
    q.nblocks = g0.x * g0.y * g0.z;
    if (nl == 1) {
        k_mg_diag<<<g0, nt, 0, s>>>(f, (float *)h->cgv + h->Np, q);
        h->launches++;
        return;
    }
    for (int l = 0; l + 1 < nl; ++l) {
        k_mg_pre<<<mg_grid(h->mg[l], 16), nt, 0, s>>>(h->mg[l], p);
        k_mg_restrict<<<mg_grid(h->mg[l + 1], 16), nt, 0, s>>>(h->mg[l], h->mg[l + 1], p);
        h->launches += 2;
    }
    const MgLevel &last = h->mg[nl - 1];
    const size_t smem = (size_t)3 * (last.nx + 2) * (last.ny + 2) * (last.nz + 2) * sizeof(float);
    if (nl > 1) {
        k_mg_coarse<<<1, 1024, smem, s>>>(last, p);
        h->launches++;
    }
    for (int l = nl - 2; l >= 0; --l) {
        k_mg_prolong<<<mg_grid(h->mg[l], 16), nt, 0, s>>>(h->mg[l], h->mg[l + 1], p);
        if (l == 0)
            k_mg_smooth<<<g0, nt, 0, s>>>(h->mg[0], (float *)h->cgv + h->Np, q);
        else
            k_mg_smooth<<<mg_grid(h->mg[l], 16), nt, 0, s>>>(h->mg[l], nullptr, p);
        h->launches += 2;
    }
}

}  // namespace kv
