// kv_cg.cu -- pre-computed solenoidal projection (Sec. 3.2, 3.3).
//
//   b    = -(D- . f) on interior nodes (backward differences), ||b||^2 in FP64
//   A phi = b, A = -L (7-point, phi = 0 on the outer layer), masked CG
//   f_S0 = f - D+ phi on every node;  F = (dt^2/rho) f_S0 for the time step
//
// Precision (KV_FP32). The CG vectors r, p and the running correction e are
// float; the potential phi and the right-hand side b are double. Every inner
// product and residual norm is accumulated with FP64-class precision: per
// thread in float-float (error-free products and sums on the FP32 pipes, whose
// rate on B300 is many times the FP64 rate), then in double across threads
// and blocks. The solution is updated in groups and the residual is replaced
// by the true one ("reliable updates"): the FP32 iterations accumulate
// e += alpha p; whenever the recursive ||r|| has dropped by kReplace since the
// last replacement (or below tol/2 relative to ||b||, or at max_iter), a
// replacement folds phi += e in double, recomputes r = b - A phi in double and
// tests the true relative residual against tol. The search direction p is
// kept across replacements, so CG does not restart. KV_FP64 runs the same
// kernels with double vectors and plain double accumulation (no intermediate
// replacements).
//
// One CG iteration is two fused stencil passes:
//   pass 1: p' = r + beta p at each node and its six neighbours, Ap' on the
//           fly, p'.Ap' reduced; p' stored (ping-pong buffer). -> alpha
//   pass 2: Ap' recomputed from p', e += alpha p', r -= alpha Ap', r.r
//           reduced. -> beta, replacement and stop tests
// Both passes march z per thread column with the z neighbours in registers.
// Each reduction ends in the last block to finish (ticket), which sums the
// per-block partials in a fixed order and updates the device scalars, so the
// host only polls the control word every few iterations.
#include <math.h>
#include <stdio.h>

#include <algorithm>
#include <chrono>

#include "kv_internal.cuh"
#include "kv_reduce.cuh"

namespace kv {

constexpr int kCgBX = 32, kCgBY = 8;  // block of one CG pass: 32 x 8 columns, zc planes
constexpr double kReplace = 1e-2;     // residual replacement after each 100x drop of ||r||

__device__ __forceinline__ bool is_interior(int i, int j, int k, int nx, int ny, int nz) {
    return i >= 1 && i <= nx - 2 && j >= 1 && j <= ny - 2 && k >= 1 && k <= nz - 2;
}

// The CG kernels use 1D blocks of kCgBX*kCgBY threads mapped to (x, y) columns.
__device__ __forceinline__ void node_of(int &i, int &j) {
    i = blockIdx.x * kCgBX + (threadIdx.x % kCgBX);
    j = blockIdx.y * kCgBY + (threadIdx.x / kCgBX);
}

// Error-free float operations (Knuth's TwoSum; the exact difference a - b of
// two floats as hi + lo), so that sums of float differences are formed on the
// FP32 pipes (B300's FP64 rate is a small fraction of its FP32 rate).
__device__ __forceinline__ void two_sum(float a, float b, float &hi, float &lo) {
    hi = __fadd_rn(a, b);
    const float bb = __fsub_rn(hi, a);
    lo = __fadd_rn(__fsub_rn(a, __fsub_rn(hi, bb)), __fsub_rn(b, bb));
}
// (hi, lo) += (bh, bl), renormalised
__device__ __forceinline__ void ff_acc(float &hi, float &lo, float bh, float bl) {
    float s, e;
    two_sum(hi, bh, s, e);
    e = __fadd_rn(e, __fadd_rn(lo, bl));
    hi = __fadd_rn(s, e);
    lo = __fsub_rn(e, __fsub_rn(hi, s));
}

// b = -(D- . f) on interior nodes, ||b||^2. The three differences of float
// neighbours are exact as float pairs and summed in float-float; b is that sum
// (to about 1e-14) times -1/dx in double.
__global__ void __launch_bounds__(kCgBX *kCgBY)
k_rhs(const float *__restrict__ f, double *__restrict__ b, CgParams p) {
    int i, j;
    node_of(i, j);
    const long long sy = p.px, sz = (long long)p.px * p.ny;
    const int k0 = blockIdx.z * p.zc, k1 = min(k0 + p.zc, p.nz);
    double acc = 0.0;
    if (i < p.nx && j < p.ny) {
        for (int k = k0; k < k1; ++k) {
            const long long c = k * sz + j * sy + i;
            double v = 0.0;
            if (is_interior(i, j, k, p.nx, p.ny, p.nz)) {
                const float *fx = f, *fy = f + p.Np, *fz = f + 2 * p.Np;
                float hi, lo, h2, l2;
                two_sum(fx[c], -fx[c - 1], hi, lo);
                two_sum(fy[c], -fy[c - sy], h2, l2);
                ff_acc(hi, lo, h2, l2);
                two_sum(fz[c], -fz[c - sz], h2, l2);
                ff_acc(hi, lo, h2, l2);
                v = -(((double)hi + (double)lo) * p.inv_dx);
            }
            b[c] = v;
            acc = __fma_rn(v, v, acc);
        }
    }
    double v1[1] = {acc}, s[1];
    if (last_block_sums<1>(p, v1, s) && threadIdx.x == 0) p.scal[kBB] = s[0];
}

// Group update of the solution: phi += e (double), e = 0. Elementwise.
template <typename T>
__global__ void k_fold_e(double *__restrict__ phi, T *__restrict__ e, long long Np, CgParams p) {
    if (__ldcg(&p.ctrl[kCgStatus]) != kCgNeedTrue) return;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < Np;
         c += (long long)gridDim.x * blockDim.x) {
        const T ev = e[c];
        if (ev != T(0)) {
            phi[c] += (double)ev;
            e[c] = T(0);
        }
    }
}

// Residual replacement: r = b - A phi (FP64), stored as T; tests the true
// residual; on continuation keeps p and sets beta from the replaced residual.
template <typename T>
__global__ void __launch_bounds__(kCgBX *kCgBY)
k_true_res(const double *__restrict__ b, const double *__restrict__ phi, T *__restrict__ r,
           CgParams p) {
    if (__ldcg(&p.ctrl[kCgStatus]) != kCgNeedTrue) return;
    // the first evaluation of a start from zero is r = b (no FP64 stencil)
    const bool phi0 = p.zero_start && __ldcg(&p.ctrl[kCgRefine]) == 0;
    int i, j;
    node_of(i, j);
    const long long sy = p.px, sz = (long long)p.px * p.ny;
    const int k0 = blockIdx.z * p.zc, k1 = min(k0 + p.zc, p.nz);
    // FP32 handles: both norms from the stored (rounded) residual, accumulated
    // in float-float (a relative 1e-7 on the true norm; the FP64 pipe keeps
    // only the residual itself); FP64 handles: in double
    typename AccOf<T>::type acc_t, acc_r;
    if (i < p.nx && j < p.ny) {
        for (int k = k0; k < k1; ++k) {
            if (!is_interior(i, j, k, p.nx, p.ny, p.nz)) continue;
            const long long c = k * sz + j * sy + i;
            double rt = b[c];  // b - A phi, A = -L
            if (!phi0) {
                const double s = ((phi[c - 1] + phi[c + 1]) + (phi[c - sy] + phi[c + sy])) +
                                 (phi[c - sz] + phi[c + sz]);
                rt += (s - 6.0 * phi[c]) * p.inv_dx2;
            }
            const T rs = T(rt);
            r[c] = rs;
            if constexpr (sizeof(T) == 8) acc_t.add_prod(rt, rt);
            else acc_t.add_prod(rs, rs);
            acc_r.add_prod(rs, rs);
        }
    }
    double v[2] = {acc_t.value(), acc_r.value()}, s[2];
    if (last_block_sums<2>(p, v, s) && threadIdx.x == 0) {
        const double bb = p.scal[kBB];
        p.scal[kTrue2] = s[0];
        p.ctrl[kCgRefine] += 1;
        if (!isfinite(s[0]) || !isfinite(s[1])) {
            p.ctrl[kCgStatus] = kCgNonfinite;
        } else if (sqrt(s[0] / bb) < p.scal[kTol]) {
            p.ctrl[kCgStatus] = kCgConverged;
        } else if (p.ctrl[kCgIters] >= p.ctrl[kCgMaxIter]) {
            p.ctrl[kCgStatus] = kCgMaxIterHit;
        } else {
            if (!p.pcg) {  // preconditioned CG: beta and r.z come from the preconditioner pass
                const double rr_prev = p.scal[kRR];
                p.scal[kBeta] = (p.ctrl[kCgIters] == 0 || rr_prev <= 0.0) ? 0.0 : s[1] / rr_prev;
                p.scal[kRR] = s[1];
            }
            p.scal[kRR0] = s[1];
            p.scal[kRRLast] = s[1];
            p.ctrl[kCgStatus] = kCgRunning;
        }
    }
}

// Pass 1: p' = r + beta p (centre and neighbours), Ap' on the fly, p'.Ap'.
template <typename T>
__global__ void __launch_bounds__(kCgBX *kCgBY)
k_cg_dir(const T *__restrict__ r, T *__restrict__ p0, T *__restrict__ p1, CgParams p) {
    if (__ldcg(&p.ctrl[kCgStatus]) != kCgRunning) return;
    // iteration k reads p[k & 1] and writes p[(k + 1) & 1] (device counter, so
    // iterations skipped after a status change never flip the parity)
    const long long it0 = __ldcg(&p.ctrl[kCgIters]);
    const T *__restrict__ pold = (it0 & 1) ? p1 : p0;
    T *__restrict__ pnew = (it0 & 1) ? p0 : p1;
    const T beta = T(__ldcg(&p.scal[kBeta]));
    int i, j;
    node_of(i, j);
    const long long sy = p.px, sz = (long long)p.px * p.ny;
    const int k0 = blockIdx.z * p.zc, k1 = min(k0 + p.zc, p.nz - 1);
    const T inv = T(p.inv_dx2);
    typename AccOf<T>::type acc;
    if (i >= 1 && i <= p.nx - 2 && j >= 1 && j <= p.ny - 2) {
        auto pn = [&](long long q) { return kv_fma(beta, pold[q], r[q]); };
        const int ks = max(k0, 1);
        long long c = ks * sz + j * sy + i;
        T zm = pn(c - sz), zc = pn(c);
        for (int k = ks; k < k1; ++k, c += sz) {
            const T zp = pn(c + sz);
            const T s = kv_add(kv_add(kv_add(pn(c - 1), pn(c + 1)), kv_add(pn(c - sy), pn(c + sy))),
                               kv_add(zm, zp));
            const T Ap = kv_fma(T(6), zc, -s) * inv;
            pnew[c] = zc;
            acc.add_prod(zc, Ap);
            zm = zc;
            zc = zp;
        }
    }
    double v[1] = {acc.value()}, sm[1];
    if (last_block_sums<1>(p, v, sm) && threadIdx.x == 0) {
        const double pAp = sm[0];
        p.scal[kPAP] = pAp;
        if (!isfinite(pAp) || pAp <= 0.0)
            p.ctrl[kCgStatus] = kCgBreakdown;
        else
            p.scal[kAlpha] = p.scal[kRR] / pAp;
    }
}

// Pass 2: Ap' from p', e += alpha p', r -= alpha Ap', r.r; beta, replacement
// and stop tests.
template <typename T>
__global__ void __launch_bounds__(kCgBX *kCgBY)
k_cg_upd(const T *__restrict__ p0, const T *__restrict__ p1, T *__restrict__ r, T *__restrict__ e,
         CgParams p) {
    if (__ldcg(&p.ctrl[kCgStatus]) != kCgRunning) return;
    const T *__restrict__ pc_ = (__ldcg(&p.ctrl[kCgIters]) & 1) ? p0 : p1;  // written by k_cg_dir
    const T alpha = T(__ldcg(&p.scal[kAlpha]));
    int i, j;
    node_of(i, j);
    const long long sy = p.px, sz = (long long)p.px * p.ny;
    const int k0 = blockIdx.z * p.zc, k1 = min(k0 + p.zc, p.nz - 1);
    const T inv = T(p.inv_dx2);
    typename AccOf<T>::type acc;
    if (i >= 1 && i <= p.nx - 2 && j >= 1 && j <= p.ny - 2) {
        const int ks = max(k0, 1);
        long long c = ks * sz + j * sy + i;
        T zm = pc_[c - sz], zc = pc_[c];
        for (int k = ks; k < k1; ++k, c += sz) {
            const T zp = pc_[c + sz];
            const T s = kv_add(kv_add(kv_add(pc_[c - 1], pc_[c + 1]), kv_add(pc_[c - sy], pc_[c + sy])),
                               kv_add(zm, zp));
            const T Ap = kv_fma(T(6), zc, -s) * inv;
            e[c] = kv_fma(alpha, zc, e[c]);
            const T rn = kv_fma(-alpha, Ap, r[c]);
            r[c] = rn;
            acc.add_prod(rn, rn);
            zm = zc;
            zc = zp;
        }
    }
    double v[1] = {acc.value()}, sm[1];
    if (last_block_sums<1>(p, v, sm) && threadIdx.x == 0) {
        const double rr = sm[0];
        const long long it = p.ctrl[kCgIters] + 1;
        p.ctrl[kCgIters] = it;
        p.scal[kRRLast] = rr;
        const double bb = p.scal[kBB];
        const double tol = p.scal[kTol], repl = p.scal[kInner];
        if (!isfinite(rr)) {
            p.ctrl[kCgStatus] = kCgNonfinite;
        } else if (rr <= 0.25 * tol * tol * bb || rr <= repl * repl * p.scal[kRR0] ||
                   it >= p.ctrl[kCgMaxIter]) {
            // k_true_res computes beta from the replaced residual and scal[kRR]
            p.ctrl[kCgStatus] = kCgNeedTrue;
        } else {
            p.scal[kBeta] = rr / p.scal[kRR];
            p.scal[kRR] = rr;
        }
    }
}

// ---------------------------------------------------------------------------
// TMA-staged CG passes (FP32 handles).
//
// The CG vectors of a handle are one allocation [pA, r, pB, e] (4 x Np floats),
// seen by TMA as a 4D tensor (x, y, z, field). A block owns a kCgTX x kCgTY
// column and marches z; every plane it needs arrives by TMA into a ring of
// NS shared-memory stages, so several planes are in flight per block while
// one is computed. The z-1 neighbour is the previous plane's centre value,
// kept in registers, so a stage is refilled as soon as its plane is done. Each thread computes four consecutive x nodes (a float4);
// x neighbours come from warp shuffles, y and z neighbours from the staged
// tiles. Per-node arithmetic is the same sequence as the plain kernels above.
// Reductions: float-float per thread and across the block, double per block.
// ---------------------------------------------------------------------------
constexpr int kCgNT = kCgTX * kCgTY / 4;
constexpr int kCgGX = kCgTX / 4;
constexpr int kCgBXh = kCgTX + 8, kCgBYh = kCgTY + 2;
constexpr int kCgHalo = kCgBXh * kCgBYh;                  // floats per halo field tile
constexpr int kCgCtr = kCgTX * kCgTY;                     // floats per centre tile
constexpr int kCgStageDir = 2 * kCgHalo;                  // (p_old, r) or (r, p_old)
constexpr int kCgHaloPad = (kCgHalo + 31) / 32 * 32;
constexpr int kCgStageUpd = kCgHaloPad + 2 * kCgCtr;      // p' halo, r and e centre
static_assert((kCgStageDir * 4) % 128 == 0 && (kCgStageUpd * 4) % 128 == 0, "stage alignment");
// NS shared-memory stages per block (4 or 8): the CG autotuner picks, with the z chunk
constexpr size_t cg_smem_dir(int ns) { return (size_t)ns * kCgStageDir * 4 + ns * 8; }
constexpr size_t cg_smem_upd(int ns) { return (size_t)ns * kCgStageUpd * 4 + ns * 8; }

// Per-block partial (thread 0's value) -> last block sums all partials.
__device__ __forceinline__ bool finish_blocks(const CgParams &p, double tot, double &sum) {
    __shared__ double sh[33];
    __shared__ int s_last;
    const int bid = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
    if (threadIdx.x == 0) p.partials[bid] = tot;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long t =
            atomicAdd(reinterpret_cast<unsigned long long *>(&p.ctrl[kCgTicket]), 1ull);
        s_last = (t == (unsigned long long)(p.nblocks - 1));
    }
    __syncthreads();
    if (!s_last) return false;
    __threadfence();
    double acc = 0.0;
    for (int b = threadIdx.x; b < p.nblocks; b += blockDim.x) acc += __ldcg(&p.partials[b]);
    sum = block_sum_d(acc, sh);
    if (threadIdx.x == 0) p.ctrl[kCgTicket] = 0;
    return true;
}

__device__ __forceinline__ void dir_finish(const CgParams &p, double pAp) {
    p.scal[kPAP] = pAp;
    if (!isfinite(pAp) || pAp <= 0.0)
        p.ctrl[kCgStatus] = kCgBreakdown;
    else
        p.scal[kAlpha] = p.scal[kRR] / pAp;
}

__device__ __forceinline__ void upd_finish(const CgParams &p, double rr) {
    const long long it = p.ctrl[kCgIters] + 1;
    p.ctrl[kCgIters] = it;
    p.scal[kRRLast] = rr;
    const double bb = p.scal[kBB];
    const double tol = p.scal[kTol], repl = p.scal[kInner];
    if (!isfinite(rr)) {
        p.ctrl[kCgStatus] = kCgNonfinite;
    } else if (rr <= 0.25 * tol * tol * bb || rr <= repl * repl * p.scal[kRR0] ||
               it >= p.ctrl[kCgMaxIter]) {
        p.ctrl[kCgStatus] = kCgNeedTrue;
    } else if (!p.pcg) {  // preconditioned CG: the preconditioner pass sets beta and r.z
        p.scal[kBeta] = rr / p.scal[kRR];
        p.scal[kRR] = rr;
    }
}

template <int NS>
struct CgTile {
    int x0, y0, k0, k1, kb, gx, gy;
    __device__ CgTile(const CgParams &p) {
        x0 = blockIdx.x * kCgTX;
        y0 = 1 + blockIdx.y * kCgTY;
        k0 = 1 + blockIdx.z * p.zc;
        k1 = min(k0 + p.zc, p.nz - 1);
        kb = k0 - 1;
        gx = threadIdx.x % kCgGX;
        gy = threadIdx.x / kCgGX;
    }
    __device__ int slot(int q) const { return (q - kb) % NS; }
    __device__ uint32_t parity(int q) const { return ((q - kb) / NS) & 1; }
};

__device__ __forceinline__ float4 ld4(const float *a) { return *reinterpret_cast<const float4 *>(a); }

// Drain every stage (bounded) after a wait gave up, then flag the timeout.
template <int NS>
__device__ __forceinline__ void ring_drain(const CgParams &p, const CgTile<NS> &t, uint32_t bar0,
                                           bool ok) {
    if (__syncthreads_or(!ok) && threadIdx.x == 0) {
        atomicOr(reinterpret_cast<unsigned long long *>(&p.ctrl[kErrFlags]), 1ull);
        const int rel_max = t.k1 - t.kb;
        for (int s = 0; s < NS && s <= rel_max; ++s) {
            const int rel_last = s + ((rel_max - s) / NS) * NS;
            mbar_wait_bounded(bar0 + 8 * s, (rel_last / NS) & 1);
        }
    }
}

template <int NS>
__global__ void __launch_bounds__(kCgNT)
k_cg_dir_tma(const __grid_constant__ CUtensorMap tm_h2, float *__restrict__ cgv, CgParams p) {
    if (__ldcg(&p.ctrl[kCgStatus]) != kCgRunning) return;
    const int par = (int)(__ldcg(&p.ctrl[kCgIters]) & 1);
    const int ps = par, rs = 1 - par;                 // smem slots of p_old and r
    float *__restrict__ pnew = cgv + (par ? 0 : 2) * p.Np;
    const float beta = (float)__ldcg(&p.scal[kBeta]);
    const float inv = (float)p.inv_dx2;
    extern __shared__ __align__(128) float smem[];
    const uint32_t bar0 = smem_u32(smem + NS * kCgStageDir);
    const CgTile<NS> t(p);
    if (threadIdx.x == 0) {
        for (int s = 0; s < NS; ++s) mbar_init(bar0 + 8 * s, 1);
        mbar_init_fence();
    }
    __syncthreads();
    auto issue = [&](int q) {
        const uint32_t bar = bar0 + 8 * t.slot(q);
        mbar_expect_tx(bar, kCgStageDir * 4);
        tma_load_4d(smem_u32(smem + t.slot(q) * kCgStageDir), &tm_h2, t.x0 - 4, t.y0 - 1, q, par, bar);
    };
    if (threadIdx.x == 0)
        for (int q = t.kb; q <= min(t.k1, t.kb + NS - 1); ++q) issue(q);

    AccFF acc;
    bool ok = true;
    const int y = t.y0 + t.gy, x = t.x0 + 4 * t.gx;
    const bool row_ok = (y <= p.ny - 2) && (x < p.px);
    const bool m0 = x >= 1 && x <= p.nx - 2, m1 = x + 1 <= p.nx - 2, m2 = x + 2 <= p.nx - 2,
               m3 = x + 3 <= p.nx - 2;
    const int o = (t.gy + 1) * kCgBXh + 4 + 4 * t.gx;
    const long long sz = (long long)p.px * p.ny;
    auto pn4 = [&](const float *st, int off) {
        const float4 pv = ld4(st + ps * kCgHalo + off), rv = ld4(st + rs * kCgHalo + off);
        return make_float4(kv_fma(beta, pv.x, rv.x), kv_fma(beta, pv.y, rv.y),
                           kv_fma(beta, pv.z, rv.z), kv_fma(beta, pv.w, rv.w));
    };
    // register-blocked z march: p' of plane k-1 (the z-1 neighbour) stays in
    // registers, so a stage is released once its plane is computed
    ok &= mbar_wait_bounded(bar0 + 8 * t.slot(t.kb), t.parity(t.kb));
    float4 prev = pn4(smem + t.slot(t.kb) * kCgStageDir, o);
    __syncthreads();
    if (threadIdx.x == 0 && t.kb + NS <= t.k1) {
        fence_proxy_async();
        issue(t.kb + NS);
    }
    ok &= mbar_wait_bounded(bar0 + 8 * t.slot(t.k0), t.parity(t.k0));
    for (int k = t.k0; k < t.k1; ++k) {
        ok &= mbar_wait_bounded(bar0 + 8 * t.slot(k + 1), t.parity(k + 1));
        const float *sc = smem + t.slot(k) * kCgStageDir;
        const float *sp = smem + t.slot(k + 1) * kCgStageDir;
        const float4 c = pn4(sc, o), ym = pn4(sc, o - kCgBXh), yp = pn4(sc, o + kCgBXh);
        const float4 zm = prev, zp = pn4(sp, o);
        prev = c;
        float left = __shfl_up_sync(0xffffffffu, c.w, 1);
        float right = __shfl_down_sync(0xffffffffu, c.x, 1);
        if (t.gx == 0) left = kv_fma(beta, sc[ps * kCgHalo + o - 1], sc[rs * kCgHalo + o - 1]);
        if (t.gx == kCgGX - 1) right = kv_fma(beta, sc[ps * kCgHalo + o + 4], sc[rs * kCgHalo + o + 4]);
        float4 sum;
        sum.x = kv_add(kv_add(kv_add(left, c.y), kv_add(ym.x, yp.x)), kv_add(zm.x, zp.x));
        sum.y = kv_add(kv_add(kv_add(c.x, c.z), kv_add(ym.y, yp.y)), kv_add(zm.y, zp.y));
        sum.z = kv_add(kv_add(kv_add(c.y, c.w), kv_add(ym.z, yp.z)), kv_add(zm.z, zp.z));
        sum.w = kv_add(kv_add(kv_add(c.z, right), kv_add(ym.w, yp.w)), kv_add(zm.w, zp.w));
        if (row_ok) {
            float4 out = c;
            float4 Ap;
            Ap.x = kv_fma(6.f, c.x, -sum.x) * inv;
            Ap.y = kv_fma(6.f, c.y, -sum.y) * inv;
            Ap.z = kv_fma(6.f, c.z, -sum.z) * inv;
            Ap.w = kv_fma(6.f, c.w, -sum.w) * inv;
            if (m0) acc.add_prod(c.x, Ap.x); else out.x = 0.f;
            if (m1) acc.add_prod(c.y, Ap.y); else out.y = 0.f;
            if (m2) acc.add_prod(c.z, Ap.z); else out.z = 0.f;
            if (m3) acc.add_prod(c.w, Ap.w); else out.w = 0.f;
            *reinterpret_cast<float4 *>(pnew + k * sz + (long long)y * p.px + x) = out;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            const int q = k + NS;
            if (q <= t.k1) {
                fence_proxy_async();
                issue(q);
            }
        }
    }
    ring_drain(p, t, bar0, ok);
    const double tot = block_total_ff(acc);
    double sum;
    if (finish_blocks(p, tot, sum) && threadIdx.x == 0) dir_finish(p, sum);
}

template <int NS>
__global__ void __launch_bounds__(kCgNT)
k_cg_upd_tma(const __grid_constant__ CUtensorMap tm_h1, const __grid_constant__ CUtensorMap tm_c1,
             const __grid_constant__ CUtensorMap tm_r, float *__restrict__ cgv, CgParams p) {
    if (__ldcg(&p.ctrl[kCgStatus]) != kCgRunning) return;
    const int par = (int)(__ldcg(&p.ctrl[kCgIters]) & 1);
    const int pf = par ? 0 : 2;                      // field of p' (written by k_cg_dir_tma)
    const float alpha = (float)__ldcg(&p.scal[kAlpha]);
    const float inv = (float)p.inv_dx2;
    float *__restrict__ rg = p.rbuf;
    float *__restrict__ eg = cgv + 3 * p.Np;
    extern __shared__ __align__(128) float smem[];
    const uint32_t bar0 = smem_u32(smem + NS * kCgStageUpd);
    const CgTile<NS> t(p);
    if (threadIdx.x == 0) {
        for (int s = 0; s < NS; ++s) mbar_init(bar0 + 8 * s, 1);
        mbar_init_fence();
    }
    __syncthreads();
    auto issue = [&](int q) {
        const uint32_t bar = bar0 + 8 * t.slot(q);
        float *st = smem + t.slot(q) * kCgStageUpd;
        const bool centre = q >= t.k0 && q < t.k1;
        mbar_expect_tx(bar, (kCgHalo + (centre ? 2 * kCgCtr : 0)) * 4);
        tma_load_4d(smem_u32(st), &tm_h1, t.x0 - 4, t.y0 - 1, q, pf, bar);
        if (centre) {
            tma_load_4d(smem_u32(st + kCgHaloPad), &tm_r, t.x0, t.y0, q, p.rfield, bar);
            tma_load_4d(smem_u32(st + kCgHaloPad + kCgCtr), &tm_c1, t.x0, t.y0, q, 3, bar);
        }
    };
    if (threadIdx.x == 0)
        for (int q = t.kb; q <= min(t.k1, t.kb + NS - 1); ++q) issue(q);

    AccFF acc;
    bool ok = true;
    const int y = t.y0 + t.gy, x = t.x0 + 4 * t.gx;
    const bool row_ok = (y <= p.ny - 2) && (x < p.px);
    const bool m0 = x >= 1 && x <= p.nx - 2, m1 = x + 1 <= p.nx - 2, m2 = x + 2 <= p.nx - 2,
               m3 = x + 3 <= p.nx - 2;
    const int o = (t.gy + 1) * kCgBXh + 4 + 4 * t.gx;
    const int oc = t.gy * kCgTX + 4 * t.gx;
    const long long sz = (long long)p.px * p.ny;
    // register-blocked z march, as in pass 1
    ok &= mbar_wait_bounded(bar0 + 8 * t.slot(t.kb), t.parity(t.kb));
    float4 prev = ld4(smem + t.slot(t.kb) * kCgStageUpd + o);
    __syncthreads();
    if (threadIdx.x == 0 && t.kb + NS <= t.k1) {
        fence_proxy_async();
        issue(t.kb + NS);
    }
    ok &= mbar_wait_bounded(bar0 + 8 * t.slot(t.k0), t.parity(t.k0));
    for (int k = t.k0; k < t.k1; ++k) {
        ok &= mbar_wait_bounded(bar0 + 8 * t.slot(k + 1), t.parity(k + 1));
        const float *sc = smem + t.slot(k) * kCgStageUpd;
        const float *sp = smem + t.slot(k + 1) * kCgStageUpd;
        const float4 c = ld4(sc + o), ym = ld4(sc + o - kCgBXh), yp = ld4(sc + o + kCgBXh);
        const float4 zm = prev, zp = ld4(sp + o);
        prev = c;
        float left = __shfl_up_sync(0xffffffffu, c.w, 1);
        float right = __shfl_down_sync(0xffffffffu, c.x, 1);
        if (t.gx == 0) left = sc[o - 1];
        if (t.gx == kCgGX - 1) right = sc[o + 4];
        float4 sum;
        sum.x = kv_add(kv_add(kv_add(left, c.y), kv_add(ym.x, yp.x)), kv_add(zm.x, zp.x));
        sum.y = kv_add(kv_add(kv_add(c.x, c.z), kv_add(ym.y, yp.y)), kv_add(zm.y, zp.y));
        sum.z = kv_add(kv_add(kv_add(c.y, c.w), kv_add(ym.z, yp.z)), kv_add(zm.z, zp.z));
        sum.w = kv_add(kv_add(kv_add(c.z, right), kv_add(ym.w, yp.w)), kv_add(zm.w, zp.w));
        if (row_ok) {
            const float4 r = ld4(sc + kCgHaloPad + oc), e = ld4(sc + kCgHaloPad + kCgCtr + oc);
            float4 rn = r, en = e;
            auto node = [&](bool m, float cv, float sv, float rv, float ev, float &ro, float &eo) {
                if (!m) return;
                const float Ap = kv_fma(6.f, cv, -sv) * inv;
                eo = kv_fma(alpha, cv, ev);
                ro = kv_fma(-alpha, Ap, rv);
                acc.add_prod(ro, ro);
            };
            node(m0, c.x, sum.x, r.x, e.x, rn.x, en.x);
            node(m1, c.y, sum.y, r.y, e.y, rn.y, en.y);
            node(m2, c.z, sum.z, r.z, e.z, rn.z, en.z);
            node(m3, c.w, sum.w, r.w, e.w, rn.w, en.w);
            const long long g = k * sz + (long long)y * p.px + x;
            *reinterpret_cast<float4 *>(rg + g) = rn;
            *reinterpret_cast<float4 *>(eg + g) = en;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            const int q = k + NS;
            if (q <= t.k1) {
                fence_proxy_async();
                issue(q);
            }
        }
    }
    ring_drain(p, t, bar0, ok);
    const double tot = block_total_ff(acc);
    double sum;
    if (finish_blocks(p, tot, sum) && threadIdx.x == 0) upd_finish(p, sum);
}

// f_S0 = f - D+ phi on every node (phi = 0 beyond the grid); F = S f_S0.
template <typename T>
__global__ void __launch_bounds__(kCgBX *kCgBY)
k_grad(const float *__restrict__ f, const double *__restrict__ phi, const T *__restrict__ S,
       double S_s, T *__restrict__ F, float *__restrict__ fs_out, CgParams p) {
    int i, j;
    node_of(i, j);
    if (i >= p.nx || j >= p.ny) return;
    const long long sy = p.px, sz = (long long)p.px * p.ny;
    const int k0 = blockIdx.z * p.zc, k1 = min(k0 + p.zc, p.nz);
    const long long Nd = (long long)p.nx * p.ny * p.nz;
    for (int k = k0; k < k1; ++k) {
        const long long c = k * sz + j * sy + i;
        const double ph = phi[c];
        const double px_ = (i + 1 < p.nx) ? phi[c + 1] : 0.0;
        const double py_ = (j + 1 < p.ny) ? phi[c + sy] : 0.0;
        const double pz_ = (k + 1 < p.nz) ? phi[c + sz] : 0.0;
        const double g[3] = {(px_ - ph) * p.inv_dx, (py_ - ph) * p.inv_dx, (pz_ - ph) * p.inv_dx};
        const long long cd = ((long long)k * p.ny + j) * p.nx + i;
        if constexpr (sizeof(T) == 4) {
            // FP32 handles: f_S0 rounded to float once, the scaling by S in FP32
            // (the FP64 pipe keeps only the gradient and the subtraction)
            const float s = S ? (float)S[c] : (float)S_s;
            for (int comp = 0; comp < 3; ++comp) {
                const float fsv = (float)((double)f[comp * p.Np + c] - g[comp]);
                F[comp * p.Np + c] = __fmul_rn(s, fsv);
                if (fs_out) fs_out[comp * Nd + cd] = fsv;
            }
        } else {
            const double s = S ? (double)S[c] : S_s;
            for (int comp = 0; comp < 3; ++comp) {
                const double fsv = (double)f[comp * p.Np + c] - g[comp];
                F[comp * p.Np + c] = T(s * fsv);
                if (fs_out) fs_out[comp * Nd + cd] = (float)fsv;
            }
        }
    }
}

// Per-node stability limit dt <= h^2 / (nu + sqrt(nu^2 + c^2 h^2)), h^2 = dx^2/3
// (the positive root of dt^2 c^2 + 2 dt nu = h^2), block minima. Fields of
// nx*ny*nz nodes in rows of pitch px (px = nx: dense). op = KV_OP_DIVERGENCE: at interior nodes c^2 and nu use the
// mean face modulus (6 G_i + sum of the neighbours' G) / 12 (Gershgorin bound
// of the flux operator); boundary nodes are only validated.
template <typename T>
__device__ __forceinline__ T dt_node_limit(long long q, int nx, int ny, int nz, int px, T h2, const float *G,
                                           double Gs, const float *rho, double rhos, const float *eta, double etas,
                                           int op) {
    // node q of the dense enumeration, at element c of rows of pitch px
    const long long c = (q / nx) * px + q % nx;
    const long long sy = px, sz = (long long)px * ny;
    T g = G ? T(G[c]) : T(Gs);
    const T r = rho ? T(rho[c]) : T(rhos);
    T e = eta ? T(eta[c]) : T(etas);
    if (!(r > T(0)) || g < T(0) || e < T(0) || !isfinite(g) || !isfinite(r) || !isfinite(e))
        return T(-1);  // invalid medium
    if (op == KV_OP_DIVERGENCE) {
        const int i = (int)(q % nx), j = (int)((q / nx) % ny), k = (int)(q / ((long long)nx * ny));
        if (!(i >= 1 && i <= nx - 2 && j >= 1 && j <= ny - 2 && k >= 1 && k <= nz - 2)) return T(INFINITY);
        const long long nb[6] = {c - 1, c + 1, c - sy, c + sy, c - sz, c + sz};
        T gs = T(6) * g, es = T(6) * e;
        for (int f = 0; f < 6; ++f) {
            gs += G ? T(G[nb[f]]) : T(Gs);
            es += eta ? T(eta[nb[f]]) : T(etas);
        }
        g = gs / T(12);
        e = es / T(12);
    }
    const T c2 = g / r, nu = e / r;
    const T den = nu + sqrt(nu * nu + c2 * h2);
    return den > T(0) ? h2 / den : T(INFINITY);
}

// Block minima of the limit. The FP64 formula is evaluated only where a
// single-precision estimate (relative error ~1e-6) comes within 1e-3 of the
// block's smallest estimate, so the result is the exact FP64 minimum while
// almost every node costs FP32 arithmetic only (B300's FP64 rate is a small
// fraction of its FP32 rate).
__global__ void k_dtmin(int nx, int ny, int nz, int px, double dx, const float *G, double Gs,
                        const float *rho, double rhos, const float *eta, double etas, int op,
                        double *out) {
    __shared__ double sh[256];
    __shared__ float shf[256];
    const long long n = (long long)nx * ny * nz;
    const long long q0 = blockIdx.x * (long long)blockDim.x + threadIdx.x, dq = (long long)gridDim.x * blockDim.x;
    float mf = INFINITY;
    for (long long q = q0; q < n; q += dq)
        mf = fminf(mf, dt_node_limit<float>(q, nx, ny, nz, px, (float)(dx * dx / 3.0), G, Gs, rho, rhos, eta,
                                            etas, op));
    shf[threadIdx.x] = mf;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) shf[threadIdx.x] = fminf(shf[threadIdx.x], shf[threadIdx.x + s]);
        __syncthreads();
    }
    const float cut = shf[0] < 0.f ? 0.f : shf[0] * 1.001f;
    double m = INFINITY;
    for (long long q = q0; q < n; q += dq) {
        const float v32 = dt_node_limit<float>(q, nx, ny, nz, px, (float)(dx * dx / 3.0), G, Gs, rho, rhos,
                                               eta, etas, op);
        if (v32 <= cut)
            m = fmin(m, dt_node_limit<double>(q, nx, ny, nz, px, dx * dx / 3.0, G, Gs, rho, rhos, eta, etas, op));
    }
    sh[threadIdx.x] = m;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) sh[threadIdx.x] = fmin(sh[threadIdx.x], sh[threadIdx.x + s]);
        __syncthreads();
    }
    if (threadIdx.x == 0) out[blockIdx.x] = sh[0];
}

kv_status stable_dt_device(cudaStream_t stream, double *scratch, int nx, int ny, int nz, int px, double dx,
                           const float *G, double Gs, const float *rho, double rhos, const float *eta,
                           double etas, int op, double *out) {
    double *d = scratch;
    if (!d && cudaMalloc(&d, kDtBlocks * sizeof(double)) != cudaSuccess) return KV_ERR_OOM;
    k_dtmin<<<kDtBlocks, 256, 0, stream>>>(nx, ny, nz, px, dx, G, Gs, rho, rhos, eta, etas, op, d);
    double hbuf[kDtBlocks];
    cudaError_t e = cudaMemcpyAsync(hbuf, d, sizeof(hbuf), cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (!scratch) cudaFree(d);
    if (e != cudaSuccess) return KV_ERR_CUDA;
    double m = INFINITY;
    for (int i = 0; i < kDtBlocks; ++i) m = fmin(m, hbuf[i]);
    *out = m;
    return KV_OK;
}

// ---------------------------------------------------------------------------
// Host driver
// ---------------------------------------------------------------------------
static CgParams cg_params(kv_handle *h, dim3 grid, int zc) {
    CgParams p{};
    p.pcg = 0;
    p.zero_start = 0;
    p.rbuf = (float *)h->cgv + h->Np;  // r in field 1 of the CG vectors
    p.rfield = 1;
    p.nx = h->nx;
    p.ny = h->ny;
    p.nz = h->nz;
    p.px = h->px;
    p.Np = h->Np;
    p.inv_dx2 = 1.0 / (h->dx * h->dx);
    p.inv_dx = 1.0 / h->dx;
    p.ctrl = h->ctrl;
    p.scal = h->scal;
    p.partials = h->partials;
    p.zc = zc;
    p.nblocks = grid.x * grid.y * grid.z;
    return p;
}

int cg_zc(const kv_handle *h) { return kCgZc; }

// Default z chunk of the TMA CG passes: about one wave of blocks (148 SMs x 4
// resident blocks of 64 x 8 columns), at least 8 and at most 128 planes.
int cg_auto_zc(const kv_handle *h) {
    const long long cols = (long long)((h->px + kCgTX - 1) / kCgTX) * ((h->ny - 2 + kCgTY - 1) / kCgTY);
    const long long per_col = std::max(1ll, 592 / std::max(1ll, cols));
    const long long zc = (h->nz - 2 + per_col - 1) / per_col;
    return (int)std::min(128ll, std::max(8ll, zc));
}

dim3 cg_grid(const kv_handle *h) {
    const int zc = cg_zc(h);
    return dim3((h->nx + kCgBX - 1) / kCgBX, (h->ny + kCgBY - 1) / kCgBY, (h->nz + zc - 1) / zc);
}

static kv_status sync_read(kv_handle *h) {
    cudaError_t e = cudaMemcpyAsync(h->ctrl_host, h->ctrl, kCtrlWords * sizeof(long long),
                                    cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(h->scal_host, h->scal, kCgScalars * sizeof(double),
                            cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    return cuda_check(h, e, "projection poll");
}

// Minimal-residual scaling of a warm start phi0: alpha = (A phi0).b / |A phi0|^2
// minimises |b - alpha A phi0|, so the starting residual is never larger than
// the zero start's (alpha = 0).
__global__ void __launch_bounds__(kCgBX *kCgBY)
k_warm_dots(const double *__restrict__ phi, const double *__restrict__ b, CgParams p) {
    int i, j;
    node_of(i, j);
    const long long sy = p.px, sz = (long long)p.px * p.ny;
    const int k0 = blockIdx.z * p.zc, k1 = min(k0 + p.zc, p.nz);
    double a = 0.0, c = 0.0;
    if (i < p.nx && j < p.ny) {
        for (int k = k0; k < k1; ++k) {
            if (!is_interior(i, j, k, p.nx, p.ny, p.nz)) continue;
            const long long q = k * sz + j * sy + i;
            const double s = ((phi[q - 1] + phi[q + 1]) + (phi[q - sy] + phi[q + sy])) +
                             (phi[q - sz] + phi[q + sz]);
            const double Ap = (6.0 * phi[q] - s) * p.inv_dx2;
            a += Ap * b[q];
            c += Ap * Ap;
        }
    }
    double v[2] = {a, c}, sm[2];
    if (last_block_sums<2>(p, v, sm) && threadIdx.x == 0) {
        p.scal[kWarmA] = sm[0];
        p.scal[kWarmC] = sm[1];
    }
}

__global__ void k_scale(double *__restrict__ phi, long long Np, double alpha) {
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < Np; c += (long long)gridDim.x * blockDim.x)
        phi[c] *= alpha;
}

// Pitched double <-> dense float (the learned warm start works on dense grids).
__global__ void k_pitched_to_dense(const double *__restrict__ a, float *__restrict__ o, int nx, int ny,
                                   int nz, int px) {
    const long long n = (long long)nx * ny * nz;
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < n; v += (long long)gridDim.x * blockDim.x) {
        const long long r = v / nx;
        o[v] = (float)a[r * px + v % nx];
    }
}
__global__ void k_dense_to_pitched(const float *__restrict__ a, double *__restrict__ o, int nx, int ny,
                                   int nz, int px) {
    const long long n = (long long)nx * ny * nz;
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < n; v += (long long)gridDim.x * blockDim.x) {
        const long long r = v / nx;
        const int i = (int)(v % nx), j = (int)(r % ny), k = (int)(r / ny);
        const bool in = i >= 1 && i <= nx - 2 && j >= 1 && j <= ny - 2 && k >= 1 && k <= nz - 2;
        o[r * px + i] = in ? (double)a[v] : 0.0;
    }
}

// TMA views of the CG vectors and the kernels' shared-memory limits.
static kv_status cg_tma_prepare(kv_handle *h) {
    if (h->cg_tma_ready) return KV_OK;
    kv_status st;
    if ((st = encode_tensor_4d(h, &h->tm_cg_h2, h->cgv, 4, kCgBXh, kCgBYh, 2)) != KV_OK) return st;
    if ((st = encode_tensor_4d(h, &h->tm_cg_h1, h->cgv, 4, kCgBXh, kCgBYh, 1)) != KV_OK) return st;
    if ((st = encode_tensor_4d(h, &h->tm_cg_c1, h->cgv, 4, kCgTX, kCgTY, 1)) != KV_OK) return st;
    cudaError_t e = cudaFuncSetAttribute(k_cg_dir_tma<8>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)cg_smem_dir(8));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_cg_upd_tma<8>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)cg_smem_upd(8));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_cg_dir_tma<4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)cg_smem_dir(4));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_cg_upd_tma<4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)cg_smem_upd(4));
    if (e != cudaSuccess) return cuda_check(h, e, "cudaFuncSetAttribute(CG)");
    h->cg_tma_ready = 1;
    return KV_OK;
}

template <typename T>
static kv_status project_t(kv_handle *h, double tol, int max_iter, int mode, float *fs_out,
                           kv_cg_stats *st) {
    const auto t0 = std::chrono::steady_clock::now();
    const dim3 grid = cg_grid(h);
    const int zc = cg_zc(h);
    const int nt = kCgBX * kCgBY;
    CgParams p = cg_params(h, grid, zc);
    cudaStream_t s = h->stream;
    cudaError_t e;
    // FP32: the two CG passes run as TMA-staged z-march kernels
    const bool use_tma = (h->precision == KV_FP32);
    const int tzc = h->cg_zc > 0 ? h->cg_zc : cg_auto_zc(h);
    const dim3 tgrid((h->px + kCgTX - 1) / kCgTX, (h->ny - 2 + kCgTY - 1) / kCgTY,
                     (h->nz - 2 + tzc - 1) / tzc);
    CgParams pt = cg_params(h, tgrid, tzc);
    // mode 4: CG preconditioned by the multigrid V-cycle (kv_mg.cu); r lives
    // in the preconditioner's fine array, z takes r's slot of the CG vectors
    const bool pcg = (mode == 4 || mode == 5);
    if (pcg) {
        if (!use_tma) return set_error(h, KV_ERR_UNSUPPORTED, "projection mode 4 needs an FP32 handle");
        kv_status ms = mg_prepare(h);
        if (ms != KV_OK) return ms;
        p.pcg = pt.pcg = 1;
        pt.rbuf = h->mg[0].r;
        pt.rfield = 0;
    }
    T *rvec = pcg ? (T *)h->mg[0].r : (T *)h->r;
    if (use_tma) {
        kv_status ts = cg_tma_prepare(h);
        if (ts != KV_OK) return ts;
        if ((long long)tgrid.x * tgrid.y * tgrid.z > h->partials_len)
            return set_error(h, KV_ERR_ARG, "CG partials buffer too small");
    }
    // reset the CG vectors and control words
    e = cudaMemsetAsync(h->r, 0, h->Np * sizeof(T), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->p[0], 0, h->Np * sizeof(T), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->p[1], 0, h->Np * sizeof(T), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->e, 0, h->Np * sizeof(T), s);
    bool phi_zero = !(mode == 3 && h->phi_valid);  // mode 3 starts from the previous phi
    if (e == cudaSuccess && phi_zero) e = cudaMemsetAsync(h->phi, 0, h->Np * sizeof(double), s);
    if (e != cudaSuccess) return cuda_check(h, e, "projection memset");
    long long *ci = h->ctrl_host;
    double *si = h->scal_host;
    e = cudaMemcpyAsync(ci, h->ctrl, kCtrlWords * sizeof(long long), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_check(h, e, "projection init");
    ci[kCgStatus] = kCgNeedTrue;
    ci[kCgIters] = 0;
    ci[kCgTicket] = 0;
    ci[kCgRefine] = 0;
    ci[kCgMaxIter] = max_iter;
    for (int q = 0; q < kCgScalars; ++q) si[q] = 0.0;
    si[kTol] = tol;
    // preconditioned CG drops the residual by 100x in two or three iterations:
    // replace it after every 1000x drop instead
    si[kInner] = (h->precision == KV_FP64) ? 0.0 : (pcg ? kReplace * 0.1 : kReplace);
    e = cudaMemcpyAsync(h->ctrl, ci, kCtrlWords * sizeof(long long), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(h->scal, si, kCgScalars * sizeof(double), cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return cuda_check(h, e, "projection init");

    k_rhs<<<grid, nt, 0, s>>>(h->fstage, h->b, p);
    h->launches++;
    kv_status ks = sync_read(h);
    if (ks != KV_OK) return ks;
    const double bb = h->scal_host[kBB];
    int status = KV_OK;
    const int fold_blocks = 148 * 8;
    if ((mode == 1 || mode == 5) && isfinite(bb) && bb > 0.0) {  // learned initial guess
        // learned warm start: phi_0 = Net(b) on interior nodes; the CG below
        // starts from it and stops on the same true residual as from zero
        k_pitched_to_dense<<<fold_blocks, 256, 0, s>>>(h->b, kv_net_stage_b(h->net), h->nx, h->ny, h->nz, h->px);
        if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return cuda_check(h, e, "warm start");
        kv_status ns = kv_net_predict(h->net, h->nx, h->ny, h->nz, h->dx, kv_net_stage_b(h->net),
                                      kv_net_stage_phi(h->net));
        if (ns != KV_OK) return set_error(h, ns, "warm start: network inference failed");
        k_dense_to_pitched<<<fold_blocks, 256, 0, s>>>(kv_net_stage_phi(h->net), h->phi, h->nx, h->ny, h->nz,
                                                       h->px);
        k_warm_dots<<<grid, nt, 0, s>>>(h->phi, h->b, p);
        h->launches += 3;
        if ((ks = sync_read(h)) != KV_OK) return ks;
        const double wa = h->scal_host[kWarmA], wc = h->scal_host[kWarmC];
        const double alpha = (isfinite(wa) && isfinite(wc) && wc > 0.0) ? wa / wc : 0.0;
        k_scale<<<fold_blocks, 256, 0, s>>>(h->phi, h->Np, alpha);
        phi_zero = false;
        h->launches++;
        h->warm_alpha = alpha;
    }
    if (bb == 0.0) {  // zero right-hand side: phi = 0 whatever the start
        if ((e = cudaMemsetAsync(h->phi, 0, h->Np * sizeof(double), s)) != cudaSuccess)
            return cuda_check(h, e, "projection memset");
    }
    int fcg_iters = 0;
    double fcg_true2 = 0.0;
    if (!isfinite(bb)) {
        status = KV_ERR_NONFINITE;
    } else if (bb > 0.0 && mode == 2) {  // flexible CG with the network as preconditioner
        kv_status fs = project_fcg(h, tol, max_iter, &status, &fcg_iters, &fcg_true2, bb);
        if (fs != KV_OK) return fs;
    } else if (bb > 0.0) {
        p.zero_start = phi_zero ? 1 : 0;
        const int chunk = pcg ? 4 : 32;  // iterations queued between polls of the control word
        while (true) {
            const long long c = h->ctrl_host[kCgStatus];
            if (c == kCgNeedTrue) {
                k_fold_e<T><<<fold_blocks, 256, 0, s>>>(h->phi, (T *)h->e, h->Np, p);
                k_true_res<T><<<grid, nt, 0, s>>>(h->b, h->phi, rvec, p);
                h->launches += 2;
            } else if (c == kCgRunning) {
                T *p0 = (T *)h->p[0], *p1 = (T *)h->p[1];
                for (int it = 0; it < chunk; ++it) {
                    if (use_tma) {
                        if (pcg) mg_apply(h, pt);
                        if (h->cg_ns == 4) {
                            k_cg_dir_tma<4><<<tgrid, kCgNT, cg_smem_dir(4), s>>>(h->tm_cg_h2, (float *)h->cgv, pt);
                            k_cg_upd_tma<4><<<tgrid, kCgNT, cg_smem_upd(4), s>>>(
                                h->tm_cg_h1, h->tm_cg_c1, pcg ? h->tm_mg_r : h->tm_cg_c1, (float *)h->cgv, pt);
                        } else {
                            k_cg_dir_tma<8><<<tgrid, kCgNT, cg_smem_dir(8), s>>>(h->tm_cg_h2, (float *)h->cgv, pt);
                            k_cg_upd_tma<8><<<tgrid, kCgNT, cg_smem_upd(8), s>>>(
                                h->tm_cg_h1, h->tm_cg_c1, pcg ? h->tm_mg_r : h->tm_cg_c1, (float *)h->cgv, pt);
                        }
                    } else {
                        k_cg_dir<T><<<grid, nt, 0, s>>>((const T *)h->r, p0, p1, p);
                        k_cg_upd<T><<<grid, nt, 0, s>>>(p0, p1, (T *)h->r, (T *)h->e, p);
                    }
                    h->launches += 2;
                }
            } else {
                break;
            }
            if ((ks = sync_read(h)) != KV_OK) return ks;
        }
        const long long c = h->ctrl_host[kCgStatus];
        if (c == kCgBreakdown)
            status = KV_CG_BREAKDOWN;
        else if (c == kCgNonfinite)
            status = KV_ERR_NONFINITE;
        else if (c == kCgMaxIterHit)
            status = KV_CG_MAXITER;
    }
    k_grad<T><<<grid, nt, 0, s>>>(h->fstage, h->phi, h->het ? (const T *)h->S : nullptr, h->S_s,
                                  (T *)h->F, fs_out, p);
    h->launches++;
    if ((ks = sync_read(h)) != KV_OK) return ks;
    h->have_force = 1;
    h->phi_valid = (status == KV_OK);
    if (h->ctrl_host[kErrFlags] & 1) {
        h->sticky = 1;
        return set_error(h, KV_ERR_TIMEOUT, "a bounded device wait timed out in a CG kernel");
    }
    if (st) {
        st->iters = mode == 2 ? fcg_iters : (int)h->ctrl_host[kCgIters];
        st->refinements = mode == 2 ? 0 : (int)std::max(0ll, h->ctrl_host[kCgRefine] - 1);
        st->status = status;
        const double t2 = mode == 2 ? fcg_true2 : h->scal_host[kTrue2];
        st->rel_res_true = bb > 0.0 ? sqrt(t2 / bb) : 0.0;
        st->rel_res_recursive = bb > 0.0 ? sqrt((mode == 2 ? fcg_true2 : h->scal_host[kRRLast]) / bb) : 0.0;
        st->ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0)
                     .count();
    }
    if (status == KV_ERR_NONFINITE) return set_error(h, KV_ERR_NONFINITE, "non-finite projection");
    if (status == KV_CG_BREAKDOWN) return set_error(h, KV_CG_BREAKDOWN, "CG breakdown (p.Ap <= 0)");
    if (status == KV_CG_MAXITER) {
        snprintf(h->err, sizeof(h->err), "CG reached max_iter=%d, true rel. residual %.3e", max_iter,
                 bb > 0.0 ? sqrt((mode == 2 ? fcg_true2 : h->scal_host[kTrue2]) / bb) : 0.0);
        return KV_CG_MAXITER;
    }
    return KV_OK;
}

kv_status project(kv_handle *h, double tol, int max_iter, int mode, float *fs_out, kv_cg_stats *st) {
    if (h->precision == KV_FP64) return project_t<double>(h, tol, max_iter, mode, fs_out, st);
    return project_t<float>(h, tol, max_iter, mode, fs_out, st);
}

}  // namespace kv

// ---------------------------------------------------------------------------
// Projection without device allocation (kv_project_force_noalloc).
//
// For callers that cannot call cudaMalloc or cudaFree: code whose device
// memory is owned by another allocator (a framework's caching allocator that
// has already reserved the pool, or a fixed memory budget), and code on a
// latency-critical stream that cannot afford the device-wide synchronisation
// cudaFree implies. The whole working set of the projection lives in one
// file-scope device array of kNoallocBytes, which every GPU that loads libkv
// holds until the process exits. The first call on a device looks up the
// array's device address with cudaGetSymbolAddress (so make that first call
// before any stream capture); later calls reuse the cached address. All calls
// share the array and it keeps the last call's contents, so each call clears
// what must start at zero, and calls that overlap on the GPU (other streams
// or other host threads) race on it.
// ---------------------------------------------------------------------------
#include <mutex>

namespace kv {

constexpr long long kNoallocMaxNodes = 1ll << 18;  // padded nodes: up to 64^3
constexpr int kNoallocMaxBlocks = 4096;            // CG blocks (partials slots)

// Layout of the scratch array (each part 256-byte aligned).
constexpr size_t kNaCtrl = 0;                                   // 16 x int64
constexpr size_t kNaScal = 256;                                 // 16 x double
constexpr size_t kNaPart = 512;                                 // 2 x kNoallocMaxBlocks doubles
constexpr size_t kNaF = kNaPart + 2 * kNoallocMaxBlocks * 8;    // 3 x Np floats (input force)
constexpr size_t kNaR = kNaF + 3 * kNoallocMaxNodes * 4;        // Np floats
constexpr size_t kNaP = kNaR + kNoallocMaxNodes * 4;            // p0, p1, e: 3 x Np floats
constexpr size_t kNaPhi = kNaP + 3 * kNoallocMaxNodes * 4;      // Np doubles
constexpr size_t kNaB = kNaPhi + kNoallocMaxNodes * 8;          // Np doubles
constexpr size_t kNoallocBytes = kNaB + kNoallocMaxNodes * 8;   // about 11 MB

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocBytes];

static std::mutex g_noalloc_mutex;
static void *g_noalloc_ptr[64];  // device address of the array, per device

static kv_status noalloc_setup(void **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return set_error(nullptr, KV_ERR_CUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
    if (dev < 0 || dev >= 64)
        return set_error(nullptr, KV_ERR_UNSUPPORTED,
                         "device %d is beyond the 64 devices the set-up table holds", dev);
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_ptr[dev]) {
        void *ptr = nullptr;
        e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (e != cudaSuccess || !ptr)
            return set_error(nullptr, KV_ERR_CUDA, "cudaGetSymbolAddress(scratch): %s",
                             cudaGetErrorString(e));
        g_noalloc_ptr[dev] = ptr;
    }
    *out = g_noalloc_ptr[dev];
    return KV_OK;
}

}  // namespace kv

extern "C" kv_status kv_project_force_noalloc(int nx, int ny, int nz, double dx, const float *fx,
                                              const float *fy, const float *fz, double tol,
                                              int max_iter, float *fs_out, kv_cg_stats *stats,
                                              void *stream) {
    using namespace kv;
    const auto t0 = std::chrono::steady_clock::now();
    if (nx < 3 || ny < 3 || nz < 3 || !(dx > 0.0) || !(tol > 0.0) || !fx || !fy || !fz || !fs_out)
        return set_error(nullptr, KV_ERR_ARG,
                         "kv_project_force_noalloc: invalid grid, dx, tol or pointer");
    const long long px = round_up(nx, kPitchAlign);
    const long long Np = px * ny * nz;
    if (Np > kNoallocMaxNodes)
        return set_error(nullptr, KV_ERR_ARG,
                         "kv_project_force_noalloc: grid %dx%dx%d needs %lld padded nodes (rows "
                         "padded to %d); the static scratch holds at most %lld",
                         nx, ny, nz, Np, kPitchAlign, kNoallocMaxNodes);
    const dim3 grid((nx + kCgBX - 1) / kCgBX, (ny + kCgBY - 1) / kCgBY, (nz + kCgZc - 1) / kCgZc);
    const long long nblocks = (long long)grid.x * grid.y * grid.z;
    if (nblocks > kNoallocMaxBlocks)
        return set_error(nullptr, KV_ERR_ARG,
                         "kv_project_force_noalloc: grid %dx%dx%d needs %lld reduction blocks; at "
                         "most %d",
                         nx, ny, nz, nblocks, kNoallocMaxBlocks);
    if (max_iter <= 0) max_iter = 20 * std::max(nx, std::max(ny, nz));
    void *base = nullptr;
    kv_status ks = noalloc_setup(&base);
    if (ks != KV_OK) return ks;
    unsigned char *sb = (unsigned char *)base;
    long long *ctrl = (long long *)(sb + kNaCtrl);
    double *scal = (double *)(sb + kNaScal);
    float *fst = (float *)(sb + kNaF);
    float *r = (float *)(sb + kNaR);
    float *p0 = (float *)(sb + kNaP);
    float *p1 = p0 + Np;
    float *ev = p1 + Np;
    double *phi = (double *)(sb + kNaPhi);
    double *b = (double *)(sb + kNaB);
    cudaStream_t s = (cudaStream_t)stream;

    CgParams p{};  // every field defined: plain (unpreconditioned) CG, no TMA residual buffer
    p.pcg = 0;
    p.rbuf = nullptr;
    p.rfield = 0;
    p.nx = nx;
    p.ny = ny;
    p.nz = nz;
    p.px = (int)px;
    p.Np = Np;
    p.inv_dx2 = 1.0 / (dx * dx);
    p.inv_dx = 1.0 / dx;
    p.ctrl = ctrl;
    p.scal = scal;
    p.partials = (double *)(sb + kNaPart);
    p.zc = kCgZc;
    p.nblocks = (int)nblocks;
    p.zero_start = 1;  // phi is cleared below

    long long ch[kCtrlWords];
    double sh[kCgScalars];
    for (int q = 0; q < kCtrlWords; ++q) ch[q] = 0;
    for (int q = 0; q < kCgScalars; ++q) sh[q] = 0.0;
    ch[kCgStatus] = kCgNeedTrue;
    ch[kCgMaxIter] = max_iter;
    sh[kTol] = tol;
    sh[kInner] = kReplace;
    auto fail = [&](cudaError_t e, const char *what) {
        return set_error(nullptr, KV_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
    };
    // clear everything that must start at zero (the array keeps the last call's contents)
    cudaError_t e = cudaMemsetAsync(sb + kNaF, 0, kNaPhi + Np * 8 - kNaF, s);
    if (e != cudaSuccess) return fail(e, "scratch clear");
    e = cudaMemcpyAsync(ctrl, ch, sizeof(ch), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(scal, sh, sizeof(sh), cudaMemcpyHostToDevice, s);
    const float *fin[3] = {fx, fy, fz};
    for (int q = 0; q < 3 && e == cudaSuccess; ++q)
        e = cudaMemcpy2DAsync(fst + q * Np, (size_t)px * 4, fin[q], (size_t)nx * 4, (size_t)nx * 4,
                              (size_t)ny * nz, cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return fail(e, "scratch set-up copies");

    auto poll = [&]() -> cudaError_t {
        cudaError_t pe = cudaMemcpyAsync(ch, ctrl, sizeof(ch), cudaMemcpyDeviceToHost, s);
        if (pe == cudaSuccess) pe = cudaMemcpyAsync(sh, scal, sizeof(sh), cudaMemcpyDeviceToHost, s);
        if (pe == cudaSuccess) pe = cudaStreamSynchronize(s);
        return pe;
    };
    const int nt = kCgBX * kCgBY;
    k_rhs<<<grid, nt, 0, s>>>(fst, b, p);
    if ((e = poll()) != cudaSuccess) return fail(e, "projection");
    const double bb = sh[kBB];
    int status = KV_OK;
    if (!isfinite(bb)) {
        status = KV_ERR_NONFINITE;
    } else if (bb > 0.0) {
        while (true) {
            const long long c = ch[kCgStatus];
            if (c == kCgNeedTrue) {
                k_fold_e<float><<<148 * 8, 256, 0, s>>>(phi, ev, Np, p);
                k_true_res<float><<<grid, nt, 0, s>>>(b, phi, r, p);
            } else if (c == kCgRunning) {
                for (int it = 0; it < 32; ++it) {
                    k_cg_dir<float><<<grid, nt, 0, s>>>(r, p0, p1, p);
                    k_cg_upd<float><<<grid, nt, 0, s>>>(p0, p1, r, ev, p);
                }
            } else {
                break;
            }
            if ((e = poll()) != cudaSuccess) return fail(e, "projection");
        }
        const long long c = ch[kCgStatus];
        if (c == kCgBreakdown) status = KV_CG_BREAKDOWN;
        else if (c == kCgNonfinite) status = KV_ERR_NONFINITE;
        else if (c == kCgMaxIterHit) status = KV_CG_MAXITER;
    }
    // f_S0 = f - D+ phi into fs_out; the unscaled copy F (S = 1) goes to the
    // p0/p1/e region, which the solve no longer needs.
    k_grad<float><<<grid, nt, 0, s>>>(fst, phi, nullptr, 1.0, p0, fs_out, p);
    if ((e = cudaGetLastError()) != cudaSuccess) return fail(e, "projection launch");
    if ((e = poll()) != cudaSuccess) return fail(e, "projection");
    if (stats) {
        stats->iters = (int)ch[kCgIters];
        stats->refinements = (int)std::max(0ll, ch[kCgRefine] - 1);
        stats->status = status;
        stats->rel_res_true = bb > 0.0 ? sqrt(sh[kTrue2] / bb) : 0.0;
        stats->rel_res_recursive = bb > 0.0 ? sqrt(sh[kRRLast] / bb) : 0.0;
        stats->ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0)
                        .count();
    }
    if (status == KV_ERR_NONFINITE) return set_error(nullptr, KV_ERR_NONFINITE, "non-finite projection");
    if (status == KV_CG_BREAKDOWN) return set_error(nullptr, KV_CG_BREAKDOWN, "CG breakdown (p.Ap <= 0)");
    if (status == KV_CG_MAXITER)
        return set_error(nullptr, KV_CG_MAXITER, "CG reached max_iter=%d, true rel. residual %.3e",
                         max_iter, bb > 0.0 ? sqrt(sh[kTrue2] / bb) : 0.0);
    return KV_OK;
}
