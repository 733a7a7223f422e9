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

#include <cudaTypedefs.h>

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

// ---------------------------------------------------------------------------
// Fused level kernels. Each marches z over fine planes staged in shared memory
// by TMA (an mbarrier ring with bounded waits), the z neighbours of a column
// in registers, so a level's arrays are read once per V-cycle leg:
//   k_mg_down   r_c = R (r - A S r)                 reads r, writes r_c
//   k_mg_up     z = z2 + S (r - A z2), z2 = S r + P e_c
//                                                   reads r and e_c, writes z
// The residual after pre-smoothing and z2 live only in shared memory. The
// cell arithmetic runs on pairs of cells (packed FP32: each lane rounds as the
// scalar operation would).
// ---------------------------------------------------------------------------

__device__ __forceinline__ float4 mg_ld4(const float *a) { return *reinterpret_cast<const float4 *>(a); }
__device__ __forceinline__ float2 mg_ld2(const float *a) { return *reinterpret_cast<const float2 *>(a); }
__device__ __forceinline__ float2 mg_f2(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ float2 mg_add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mg_fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 mg_mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 mg_dup(float a) { return make_float2(a, a); }

// 0.75 near + 0.25 far: one axis of the trilinear prolongation.
__device__ __forceinline__ float mg_lin(float near, float far) {
    return __fmaf_rn(0.75f, near, __fmul_rn(0.25f, far));
}
__device__ __forceinline__ float2 mg_lin2(float2 near, float2 far) {
    return mg_fma2(mg_dup(0.75f), near, mg_mul2(mg_dup(0.25f), far));
}

// ((l + r) + (ym + yp)) + (zm + zp): the six neighbours of a pair of cells.
__device__ __forceinline__ float2 mg_nb2(float2 l, float2 r, float2 ym, float2 yp, float2 zm, float2 zp) {
    return mg_add2(mg_add2(mg_add2(l, r), mg_add2(ym, yp)), mg_add2(zm, zp));
}
// (1 - omega) r + (omega / 6) s: r - A S r at a pair of cells (s: neighbours of r).
__device__ __forceinline__ float2 mg_t2(float2 rc, float2 s) {
    return mg_fma2(mg_dup(kMgOmega / 6.f), s, mg_mul2(mg_dup(1.f - kMgOmega), rc));
}
__device__ __forceinline__ float mg_t1(float rc, float s) {
    return __fmaf_rn(kMgOmega / 6.f, s, __fmul_rn(1.f - kMgOmega, rc));
}
__device__ __forceinline__ float mg_nb1(float l, float r, float ym, float yp, float zm, float zp) {
    return __fadd_rn(__fadd_rn(__fadd_rn(l, r), __fadd_rn(ym, yp)), __fadd_rn(zm, zp));
}

// After a wait gave up: flag the timeout and wait (bounded) for the copies
// still in flight (the last one issued into each of the ns slots), so none
// lands after the block exits. bar(q) / parity(q) give a plane's slot.
template <typename Bar, typename Par>
__device__ __forceinline__ void mg_ring_drain(const CgParams &p, int q_first, int q_last, int ns, Bar bar,
                                              Par parity) {
    atomicOr(reinterpret_cast<unsigned long long *>(&p.ctrl[kErrFlags]), 1ull);
    for (int q = max(q_first, q_last - ns + 1); q <= q_last; ++q) mbar_wait_bounded(bar(q), parity(q));
}

// k_mg_down: a block owns kDnCX x kDnCY coarse columns and a chunk of coarse
// planes. Coarse cell I covers fine cells 2I-2 .. 2I+1 per axis (weights 1/4,
// 3/4, 3/4, 1/4), so the block needs t on kDnTX x kDnTY fine columns and r
// one cell further. Per fine plane 256 threads form t at four consecutive
// cells of a row (columns 0..63) and one warp at the last two columns; t goes
// to shared memory, and one thread per coarse column restricts its 4 x 4
// cells, adds the plane into the two coarse planes it touches and stores a
// coarse cell once its four fine planes are in.
constexpr int kDnCX = 32, kDnCY = 7;         // coarse columns per block
constexpr int kDnTX = 2 * kDnCX + 2;         // 66 fine columns of t
constexpr int kDnTY = 2 * kDnCY + 2;         // 16 fine rows of t
constexpr int kDnBX = 2 * kDnCX + 8;         // staged r: x from 2 kDnCX bx - 4 (16-byte aligned)
constexpr int kDnBY = kDnTY + 2;             //           y from 2 kDnCY by - 1
constexpr int kDnTP = 68;                    // row pitch of the t plane (floats)
constexpr int kDnMain = kDnTY * 16;          // threads of columns 0..63, four each
constexpr int kDnNT = kDnMain + 32;          // + a warp for columns 64, 65
constexpr int kDnStage = (kDnBX * kDnBY + 31) / 32 * 32;  // floats per staged plane
constexpr int kDnNS = 8;                     // stages (a power of two)
constexpr int kDnT = kDnTY * kDnTP;          // floats of one t plane
constexpr size_t kDnSmem = ((size_t)kDnNS * kDnStage + 2 * kDnT) * 4 + kDnNS * 8;
static_assert(kDnTX <= kDnTP && 2 * kDnTY == 32 && kDnCX == 32, "column 64, 65 warp and coarse rows of a warp");
static_assert((kDnStage * 4) % 128 == 0 && (kDnT * 4) % 128 == 0, "stage alignment");

constexpr int kDnPerSm = 4;                  // resident blocks per SM (registers, shared memory)

__global__ void __launch_bounds__(kDnNT, kDnPerSm)
k_mg_down(const __grid_constant__ CUtensorMap tm_r, MgLevel F, MgLevel C, int zc, CgParams p) {
    if (!mg_running(p)) return;
    extern __shared__ __align__(128) float smem[];
    float *tbuf = smem + kDnNS * kDnStage;
    const uint32_t bar0 = smem_u32(tbuf + 2 * kDnT);
    const int K0 = 1 + (int)blockIdx.z * zc, K1 = min(C.nz, K0 + zc - 1);
    const int qb = 2 * K0 - 3, qe = 2 * K1 + 2;  // fine planes staged
    auto slot = [&](int q) { return (q - qb) & (kDnNS - 1); };
    auto bar = [&](int q) { return bar0 + 8 * slot(q); };
    auto parity = [&](int q) { return (uint32_t)((q - qb) / kDnNS) & 1u; };
    const int xb = 2 * kDnCX * (int)blockIdx.x - 4, yb = 2 * kDnCY * (int)blockIdx.y - 1;
    const int tid = threadIdx.x;
    if (tid == 0) {
        for (int s = 0; s < kDnNS; ++s) mbar_init(bar0 + 8 * s, 1);
        mbar_init_fence();
    }
    __syncthreads();
    auto issue = [&](int q) {
        mbar_expect_tx(bar(q), kDnBX * kDnBY * 4);
        tma_load_4d(smem_u32(smem + slot(q) * kDnStage), &tm_r, xb, yb, q, 0, bar(q));
    };
    if (tid == 0)
        for (int q = qb; q <= min(qe, qb + kDnNS - 1); ++q) issue(q);

    // t cells: main threads (x .. x+3, y), the extra warp (x, y) at column 64 or 65
    // warp index through a shuffle: the compiler then treats the role tests
    // below as uniform over a warp (they are: the roles are whole warps)
    const int warp = __shfl_sync(0xffffffffu, tid >> 5, 0);
    const bool is_main = warp < kDnMain / 32;
    const int g = tid % 16, row = is_main ? tid / 16 : (tid - kDnMain) >> 1;
    const int col = is_main ? 4 * g : 64 + (tid & 1);  // t column
    const int x = xb + 4 + col, y = yb + 1 + row;
    const bool my = y >= 1 && y <= F.ny;
    const bool m0 = my && x >= 1 && x <= F.nx, m1 = my && x + 1 <= F.nx, m2 = my && x + 2 <= F.nx,
               m3 = my && x + 3 <= F.nx;
    const int o = (row + 1) * kDnBX + 4 + col;  // staged r at the first cell
    const int ot = row * kDnTP + col;           // t plane
    // the coarse column: rows 2cj .. 2cj+3 and columns 2ci .. 2ci+3 of the t plane
    const int ci = tid % kDnCX, cj = tid / kDnCX;
    const int I = 1 + kDnCX * (int)blockIdx.x + ci, J = 1 + kDnCY * (int)blockIdx.y + cj;
    const bool cthread = warp < kDnCX * kDnCY / 32, cstore = cthread && I <= C.nx && J <= C.ny;
    const long long csz = (long long)C.px * (C.ny + 2);
    float *cr = C.r + (long long)J * C.px + I + (long long)K0 * csz;  // coarse plane K0
    const int oc = 2 * cj * kDnTP + 2 * ci;
    float accA = 0.f, accB = 0.f;  // coarse planes (k >> 1) + 1 and (k >> 1)

    bool ok = mbar_wait_bounded(bar(qb), parity(qb));
    float4 prev = is_main ? mg_ld4(smem + slot(qb) * kDnStage + o)
                       : make_float4(smem[slot(qb) * kDnStage + o], 0.f, 0.f, 0.f);
    __syncthreads();
    if (tid == 0 && qb + kDnNS <= qe) {
        fence_proxy_async();
        issue(qb + kDnNS);
    }
    ok &= mbar_wait_bounded(bar(qb + 1), parity(qb + 1));
    for (int k = qb + 1; k < qe; ++k) {
        ok &= mbar_wait_bounded(bar(k + 1), parity(k + 1));
        const float *sc = smem + slot(k) * kDnStage;
        const float *sp = smem + slot(k + 1) * kDnStage;
        const bool mz = k >= 1 && k <= F.nz;
        float *T = tbuf + (k & 1) * kDnT;
        if (is_main) {
            const float4 c = mg_ld4(sc + o), ym = mg_ld4(sc + o - kDnBX), yp = mg_ld4(sc + o + kDnBX);
            const float4 zp = mg_ld4(sp + o), zm = prev;
            prev = c;
            float left = __shfl_up_sync(0xffffffffu, c.w, 1);
            float right = __shfl_down_sync(0xffffffffu, c.x, 1);
            if (g == 0) left = sc[o - 1];
            if (g == 15) right = sc[o + 4];
            const float2 s01 = mg_nb2(mg_f2(left, c.x), mg_f2(c.y, c.z), mg_f2(ym.x, ym.y), mg_f2(yp.x, yp.y),
                                      mg_f2(zm.x, zm.y), mg_f2(zp.x, zp.y));
            const float2 s23 = mg_nb2(mg_f2(c.y, c.z), mg_f2(c.w, right), mg_f2(ym.z, ym.w), mg_f2(yp.z, yp.w),
                                      mg_f2(zm.z, zm.w), mg_f2(zp.z, zp.w));
            const float2 t01 = mg_t2(mg_f2(c.x, c.y), s01), t23 = mg_t2(mg_f2(c.z, c.w), s23);
            *reinterpret_cast<float4 *>(T + ot) =
                make_float4((mz && m0) ? t01.x : 0.f, (mz && m1) ? t01.y : 0.f, (mz && m2) ? t23.x : 0.f,
                            (mz && m3) ? t23.y : 0.f);
        } else {
            const float c = sc[o], zm = prev.x;
            prev.x = c;
            const float s = mg_nb1(sc[o - 1], sc[o + 1], sc[o - kDnBX], sc[o + kDnBX], zm, sp[o]);
            T[ot] = (mz && m0) ? mg_t1(c, s) : 0.f;
        }
        __syncthreads();
        if (tid == 0 && k + kDnNS <= qe) {
            fence_proxy_async();
            issue(k + kDnNS);
        }
        if (cthread) {
            // along x per fine row (weights 1/4 3/4 3/4 1/4), then along y;
            // along z fine plane k is the first or second of coarse plane
            // (k >> 1) + 1 and the third or fourth of coarse plane k >> 1
            const float2 wa = mg_f2(0.25f, 0.75f), wb = mg_f2(0.75f, 0.25f);
            float X[4];
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                const float *tr = T + oc + b * kDnTP;
                const float2 h = mg_fma2(wb, mg_ld2(tr + 2), mg_mul2(wa, mg_ld2(tr)));
                X[b] = __fadd_rn(h.x, h.y);
            }
            float Y = __fmul_rn(0.25f, X[0]);
            Y = __fmaf_rn(0.75f, X[1], Y);
            Y = __fmaf_rn(0.75f, X[2], Y);
            Y = __fmaf_rn(0.25f, X[3], Y);
            if ((k & 1) == 0) {
                accA = __fmaf_rn(0.25f, Y, accA);
                accB = __fmaf_rn(0.75f, Y, accB);
            } else {
                accA = __fmaf_rn(0.75f, Y, accA);
                accB = __fmaf_rn(0.25f, Y, accB);
                if ((k >> 1) >= K0) {
                    if (cstore) *cr = __fmul_rn(0.125f, accB);
                    cr += csz;
                }
                accB = accA;
                accA = 0.f;
            }
        }
    }
    if (__syncthreads_or(!ok) && tid == 0) mg_ring_drain(p, qb, qe, kDnNS, bar, parity);
}

// k_mg_up: a block owns kUpTX x kUpTY fine columns (x from kUpTX bx, y from
// 1 + kUpTY by) and a chunk of fine planes. 256 threads own four consecutive
// cells of one of the kUpTY + 2 rows (the block's rows and a halo row on each
// side), one more warp the two halo columns of those rows. Per fine plane each
// thread forms z2 = S r + P e_c at its cells (0 off the interior) into a
// three-plane shared buffer; once the next plane's z2 is in, the
// post-smoothing of the plane before writes z. P is separable: per coarse
// plane a thread interpolates e_c along x and y to its cells (Q), and the two
// Q planes around a fine plane are combined along z; the three Q planes in use
// stay in registers. The top level writes the CG's z and reduces r.z.
constexpr int kUpTX = 64, kUpTY = 14;       // fine columns per block
constexpr int kUpRows = kUpTY + 2;          // with the halo rows
constexpr int kUpBX = kUpTX + 8;            // staged r: x from kUpTX bx - 4 (16-byte aligned)
constexpr int kUpMain = kUpRows * 16;       // threads of the block's columns, four cells each
constexpr int kUpNT = kUpMain + 32;         // + a warp for the halo columns
constexpr int kUpStage = kUpBX * kUpRows;   // floats per staged fine plane (y from kUpTY by)
constexpr int kUpCBX = kUpTX / 2 + 8;       // staged e_c: x from kUpTX/2 bx - 4
constexpr int kUpCBY = kUpTY / 2 + 2;       //             y from kUpTY/2 by
constexpr int kUpCStage = (kUpCBX * kUpCBY + 31) / 32 * 32;  // floats per staged coarse plane
constexpr int kUpNS = 6, kUpNC = 4;         // fine and coarse stages (coarse: a power of two)
constexpr size_t kUpSmem = ((size_t)kUpNS * kUpStage + kUpNC * kUpCStage + 3 * kUpStage) * 4 +
                           (kUpNS + kUpNC) * 8;
static_assert(2 * kUpRows == 32, "one warp for the two halo columns of every row");
static_assert((kUpStage * 4) % 128 == 0 && (kUpCStage * 4) % 128 == 0, "stage alignment");

constexpr int kUpPerSm = 3;

template <bool kTop>
__global__ void __launch_bounds__(kUpNT, kUpPerSm)
k_mg_up(const __grid_constant__ CUtensorMap tm_r, const __grid_constant__ CUtensorMap tm_e, MgLevel F,
        float *__restrict__ out, int zc, CgParams p) {
    if (!mg_running(p)) return;
    extern __shared__ __align__(128) float smem[];
    float *csm = smem + kUpNS * kUpStage;
    float *zbuf = csm + kUpNC * kUpCStage;
    const uint32_t bar0 = smem_u32(zbuf + 3 * kUpStage), cbar0 = bar0 + 8 * kUpNS;
    const int k0 = 1 + (int)blockIdx.z * zc, k1 = min(F.nz, k0 + zc - 1);
    const int qa = k0 - 1, qz = k1 + 1;                               // fine planes of z2
    const int jb = ((qa + 1) >> 1) - 1, je = ((qz + 1) >> 1) + 1;   // coarse planes
    auto rslot = [&](int q) { return (int)((unsigned)(q - qa) % kUpNS); };
    auto rbar = [&](int q) { return bar0 + 8 * rslot(q); };
    auto rpar = [&](int q) { return ((unsigned)(q - qa) / kUpNS) & 1u; };
    auto cslot = [&](int j) { return (j - jb) & (kUpNC - 1); };
    auto cbar = [&](int j) { return cbar0 + 8 * cslot(j); };
    auto cpar = [&](int j) { return (uint32_t)((j - jb) / kUpNC) & 1u; };
    const int xb = kUpTX * (int)blockIdx.x - 4, yb = kUpTY * (int)blockIdx.y;
    const int cxb = kUpTX / 2 * (int)blockIdx.x - 4, cyb = kUpTY / 2 * (int)blockIdx.y;
    const int tid = threadIdx.x;
    if (tid == 0) {
        for (int s = 0; s < kUpNS + kUpNC; ++s) mbar_init(bar0 + 8 * s, 1);
        mbar_init_fence();
    }
    __syncthreads();
    auto issue = [&](int q) {
        mbar_expect_tx(rbar(q), kUpStage * 4);
        tma_load_4d(smem_u32(smem + rslot(q) * kUpStage), &tm_r, xb, yb, q, 0, rbar(q));
    };
    auto issue_c = [&](int j) {
        mbar_expect_tx(cbar(j), kUpCBX * kUpCBY * 4);
        tma_load_4d(smem_u32(csm + cslot(j) * kUpCStage), &tm_e, cxb, cyb, j, 0, cbar(j));
    };
    int c_issued = min(je, jb + kUpNC - 1) + 1;  // next coarse plane to stage (thread 0)
    if (tid == 0) {
        for (int q = qa; q <= min(qz, qa + kUpNS - 1); ++q) issue(q);
        for (int j = jb; j < c_issued; ++j) issue_c(j);
    }

    // main threads: cells (x .. x+3, y); halo warp: the cell (x, y) at staged
    // column 3 (x = kUpTX bx - 1) or 68 (x = kUpTX bx + kUpTX)
    const int warp = __shfl_sync(0xffffffffu, tid >> 5, 0);  // role tests uniform over a warp
    const bool is_main = warp < kUpMain / 32;
    const int g = tid % 16, row = is_main ? tid / 16 : (tid - kUpMain) >> 1;
    const int col = is_main ? 4 + 4 * g : ((tid & 1) ? 4 + kUpTX : 3);  // staged column
    const int x = xb + col, y = yb + row;
    const bool my = y >= 1 && y <= F.ny;
    const bool m0 = my && x >= 1 && x <= F.nx, m1 = my && x + 1 <= F.nx, m2 = my && x + 2 <= F.nx,
               m3 = my && x + 3 <= F.nx;
    const int o = row * kUpBX + col;
    // coarse rows J (near) and J2 (far) of this fine row; coarse columns of the cells
    const int crn = (row + 1) >> 1, crf = (row & 1) ? crn - 1 : crn + 1;
    const int ca = is_main ? 2 * g + 4 : ((tid & 1) ? 4 + kUpTX / 2 : 4);  // near column of the first cell
    const int cb = is_main ? ca + 1 : ((tid & 1) ? ca + 1 : 3);           // its far column (halo warp)
    const float sh = F.sh, h2 = F.h2f;
    const bool smooth = is_main && row >= 1 && row <= kUpTY && y <= F.ny && x < F.px;
    float *outp = out + ((long long)k0 * (F.ny + 2) + y) * F.px + x;
    const long long sz = (long long)F.px * (F.ny + 2);
    bool ok = true;
    int jn = jb;  // next coarse plane to interpolate
    // Q of coarse plane jn at the thread's cells
    auto qplane = [&](float4 &Q) {
        ok &= mbar_wait_bounded(cbar(jn), cpar(jn));
        const float *cs = csm + cslot(jn) * kUpCStage;
        const float *rn = cs + crn * kUpCBX, *rf = cs + crf * kUpCBX;
        if (is_main) {
            // cells x, x+1, x+2, x+3 take coarse columns (a, b), (b, a), (b, c), (c, b)
            const float2 abn = mg_ld2(rn + ca), abf = mg_ld2(rf + ca);
            const float cn = rn[ca + 2], cf = rf[ca + 2];
            const float2 xn01 = mg_lin2(abn, mg_f2(abn.y, abn.x)), xf01 = mg_lin2(abf, mg_f2(abf.y, abf.x));
            const float2 xn23 = mg_lin2(mg_f2(abn.y, cn), mg_f2(cn, abn.y));
            const float2 xf23 = mg_lin2(mg_f2(abf.y, cf), mg_f2(cf, abf.y));
            const float2 q01 = mg_lin2(xn01, xf01), q23 = mg_lin2(xn23, xf23);
            Q = make_float4(q01.x, q01.y, q23.x, q23.y);
        } else {
            Q.x = mg_lin(mg_lin(rn[ca], rn[cb]), mg_lin(rf[ca], rf[cb]));
        }
        ++jn;
    };
    // window Q(m-1), Q(m), Q(m+1) with m = (q + 1) >> 1: fine plane q takes
    // Q(m) as near plane and Q(m-1) (q odd) or Q(m+1) (q even) as far plane
    float4 Qa, Qb, Qc;
    qplane(Qa);
    qplane(Qb);
    qplane(Qc);
    float4 z2m = make_float4(0.f, 0.f, 0.f, 0.f), z2c = z2m, rc = z2m;
    float *zq = zbuf, *zk = zbuf + kUpStage, *zf = zbuf + 2 * kUpStage;  // planes q, q - 1, free
    AccFF acc;
    for (int q = qa; q <= qz; ++q) {
        if ((q & 1) && q > qa) {
            Qa = Qb;
            Qb = Qc;
            qplane(Qc);
        }
        ok &= mbar_wait_bounded(rbar(q), rpar(q));
        const float *sr = smem + rslot(q) * kUpStage;
        const bool mz = q >= 1 && q <= F.nz;
        const float4 Qf = (q & 1) ? Qa : Qc;
        float4 z2, rq;
        if (is_main) {
            rq = mg_ld4(sr + o);
            const float2 a = mg_fma2(mg_dup(sh), mg_f2(rq.x, rq.y), mg_lin2(mg_f2(Qb.x, Qb.y), mg_f2(Qf.x, Qf.y)));
            const float2 b = mg_fma2(mg_dup(sh), mg_f2(rq.z, rq.w), mg_lin2(mg_f2(Qb.z, Qb.w), mg_f2(Qf.z, Qf.w)));
            z2 = make_float4((mz && m0) ? a.x : 0.f, (mz && m1) ? a.y : 0.f, (mz && m2) ? b.x : 0.f,
                             (mz && m3) ? b.y : 0.f);
            *reinterpret_cast<float4 *>(zq + o) = z2;
        } else {
            rq = make_float4(sr[o], 0.f, 0.f, 0.f);
            z2 = make_float4((mz && m0) ? __fmaf_rn(sh, rq.x, mg_lin(Qb.x, Qf.x)) : 0.f, 0.f, 0.f, 0.f);
            zq[o] = z2.x;
        }
        __syncthreads();
        if (tid == 0) {
            const int c_want = min(je + 1, jn + kUpNC);
            if (q + kUpNS <= qz || c_issued < c_want) fence_proxy_async();
            if (q + kUpNS <= qz) issue(q + kUpNS);
            for (; c_issued < c_want; ++c_issued) issue_c(c_issued);
        }
        if (q >= qa + 2) {  // post-smoothing of plane q - 1 (z2 of it in zk)
            float left = __shfl_up_sync(0xffffffffu, z2c.w, 1);
            float right = __shfl_down_sync(0xffffffffu, z2c.x, 1);
            if (smooth) {
                if (g == 0) left = zk[o - 1];
                if (g == 15) right = zk[o + 4];
                const float4 ym = mg_ld4(zk + o - kUpBX), yp = mg_ld4(zk + o + kUpBX);
                const float2 c01 = mg_f2(z2c.x, z2c.y), c23 = mg_f2(z2c.z, z2c.w);
                const float2 s01 = mg_nb2(mg_f2(left, z2c.x), mg_f2(z2c.y, z2c.z), mg_f2(ym.x, ym.y),
                                          mg_f2(yp.x, yp.y), mg_f2(z2m.x, z2m.y), mg_f2(z2.x, z2.y));
                const float2 s23 = mg_nb2(mg_f2(z2c.y, z2c.z), mg_f2(z2c.w, right), mg_f2(ym.z, ym.w),
                                          mg_f2(yp.z, yp.w), mg_f2(z2m.z, z2m.w), mg_f2(z2.z, z2.w));
                // z2 + (omega / 6) (h^2 r - 6 z2 + s)
                const float2 u01 = mg_fma2(mg_dup(h2), mg_f2(rc.x, rc.y), mg_fma2(mg_dup(-6.f), c01, s01));
                const float2 u23 = mg_fma2(mg_dup(h2), mg_f2(rc.z, rc.w), mg_fma2(mg_dup(-6.f), c23, s23));
                const float2 v01 = mg_fma2(mg_dup(kMgOmega / 6.f), u01, c01);
                const float2 v23 = mg_fma2(mg_dup(kMgOmega / 6.f), u23, c23);
                const float4 z = make_float4(m0 ? v01.x : 0.f, m1 ? v01.y : 0.f, m2 ? v23.x : 0.f,
                                             m3 ? v23.y : 0.f);
                *reinterpret_cast<float4 *>(outp) = z;
                if (kTop) {  // r.z over the interior (z is 0 elsewhere)
                    const float2 pr = mg_fma2(mg_f2(rc.z, rc.w), mg_f2(z.z, z.w),
                                              mg_mul2(mg_f2(rc.x, rc.y), mg_f2(z.x, z.y)));
                    acc.add(__fadd_rn(pr.x, pr.y));
                }
            }
            outp += sz;
        }
        z2m = z2c;
        z2c = z2;
        rc = rq;
        float *zt = zf;
        zf = zk;
        zk = zq;
        zq = zt;
    }
    if (__syncthreads_or(!ok) && tid == 0) {
        mg_ring_drain(p, qa, qz, kUpNS, rbar, rpar);
        mg_ring_drain(p, jb, je, kUpNC, cbar, cpar);
    }
    if (!kTop) return;
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
// A level array seen by TMA: (px, ny + 2, nz + 2) floats, one field.
static kv_status mg_tensor_map(kv_handle *h, CUtensorMap *tm, const MgLevel &L, float *base, int bx, int by) {
    auto fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(tensor_map_encoder(h));
    if (!fn) return KV_ERR_CUDA;
    cuuint64_t dims[4] = {(cuuint64_t)L.px, (cuuint64_t)(L.ny + 2), (cuuint64_t)(L.nz + 2), 1};
    cuuint64_t strides[3] = {(cuuint64_t)L.px * 4, (cuuint64_t)L.px * (L.ny + 2) * 4, (cuuint64_t)L.n * 4};
    cuuint32_t box[4] = {(cuuint32_t)bx, (cuuint32_t)by, 1, 1};
    cuuint32_t es[4] = {1, 1, 1, 1};
    CUresult r = fn(tm, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, base, dims, strides, box, es,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS)
        return set_error(h, KV_ERR_CUDA, "multigrid: cuTensorMapEncodeTiled failed (%d) for a %dx%dx%d level", (int)r,
                         L.nx, L.ny, L.nz);
    return KV_OK;
}

// Planes per block so that a launch fills the GPU in one wave of per_sm
// resident blocks per SM (a second, partial wave would double the time).
static int mg_zchunk(int nz, long long columns, int sms, int per_sm) {
    const long long target = (long long)per_sm * sms;
    const int split = (int)std::max(1ll, std::min((long long)nz, target / columns));
    int zc = (nz + split - 1) / split;
    while (zc < nz && columns * ((nz + zc - 1) / zc) > target) ++zc;
    return zc;
}

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
        c.px = (c.nx + 2 + 3) / 4 * 4;  // rows of 16-byte multiples for TMA
        c.n = (long long)c.px * (c.ny + 2) * (c.nz + 2);
        c.h2 = 4.0 * f.h2;
        L[nl++] = c;
    }
    const MgLevel &last = L[nl - 1];
    if ((long long)(last.nx + 2) * (last.ny + 2) * (last.nz + 2) > kMgCoarseMax)
        return set_error(h, KV_ERR_UNSUPPORTED,
                         "multigrid: coarsest level %dx%dx%d too large for the one-block solve (grid too anisotropic)",
                         last.nx, last.ny, last.nz);
    // fine level: r (pitched like the handle); coarse levels: r and e
    long long total = h->Np;
    for (int l = 1; l < nl; ++l) total += 2 * L[l].n;
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
    L[0].e = nullptr;  // level 0 writes the CG's z
    for (int l = 1; l < nl; ++l) {
        L[l].r = q;
        q += L[l].n;
        L[l].e = q;
        q += L[l].n;
    }
    int sms = 148;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device);
    kv_status st = encode_tensor_4d(h, &h->tm_mg_r, L[0].r, 1, kCgTX, kCgTY, 1);
    for (int l = 0; st == KV_OK && l + 1 < nl; ++l) {
        MgLevel &f = L[l];
        const MgLevel &c = L[l + 1];
        st = mg_tensor_map(h, &h->tm_mg[l][0], f, f.r, kDnBX, kDnBY);
        if (st == KV_OK) st = mg_tensor_map(h, &h->tm_mg[l][1], f, f.r, kUpBX, kUpRows);
        if (st == KV_OK) st = mg_tensor_map(h, &h->tm_mg[l][2], c, c.e, kUpCBX, kUpCBY);
        f.dn_zc = mg_zchunk(c.nz, (long long)((c.nx + kDnCX - 1) / kDnCX) * ((c.ny + kDnCY - 1) / kDnCY), sms,
                            kDnPerSm);
        const long long up_cols = (long long)((f.nx + 1 + kUpTX - 1) / kUpTX) * ((f.ny + kUpTY - 1) / kUpTY);
        f.up_zc = mg_zchunk(f.nz, up_cols, sms, kUpPerSm);
        if (l == 0)  // the top level reduces r.z over its blocks: at most partials_len of them
            while (up_cols * ((f.nz + f.up_zc - 1) / f.up_zc) > h->partials_len) ++f.up_zc;
    }
    if (st != KV_OK) {
        cudaFree(pool);
        return st;
    }
    const size_t smem = (size_t)3 * (last.nx + 2) * (last.ny + 2) * (last.nz + 2) * sizeof(float);
    e = cudaFuncSetAttribute(k_mg_coarse, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_mg_down, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kDnSmem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_mg_up<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kUpSmem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_mg_up<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kUpSmem);
    if (e != cudaSuccess) {
        cudaFree(pool);
        return cuda_check(h, e, "multigrid kernel attributes");
    }
    for (int l = 0; l < nl; ++l) {
        L[l].h2f = (float)L[l].h2;
        L[l].sh = kMgOmega * L[l].h2f / 6.f;
        h->mg[l] = L[l];
    }
    h->mg_pool = pool;
    h->mg_levels = nl;
    return KV_OK;
}

void mg_apply(kv_handle *h, const CgParams &p) {
    const int nl = h->mg_levels;
    cudaStream_t s = h->stream;
    const MgLevel &f = h->mg[0];
    float *z = (float *)h->cgv + h->Np;  // the CG's z (r's slot of the CG vectors)
    if (nl == 1) {
        const long long gxy = (long long)((f.nx + kMgBX - 1) / kMgBX) * ((f.ny + kMgBY - 1) / kMgBY);
        const int zs = (int)std::max(1ll, std::min(16ll, h->partials_len / gxy));
        const dim3 g((f.nx + kMgBX - 1) / kMgBX, (f.ny + kMgBY - 1) / kMgBY, std::max(1, std::min(f.nz, zs)));
        CgParams q = p;
        q.nblocks = g.x * g.y * g.z;
        k_mg_diag<<<g, kMgBX * kMgBY, 0, s>>>(f, z, q);
        h->launches++;
        return;
    }
    for (int l = 0; l + 1 < nl; ++l) {
        const MgLevel &F = h->mg[l], &C = h->mg[l + 1];
        const dim3 g((C.nx + kDnCX - 1) / kDnCX, (C.ny + kDnCY - 1) / kDnCY, (C.nz + F.dn_zc - 1) / F.dn_zc);
        k_mg_down<<<g, kDnNT, kDnSmem, s>>>(h->tm_mg[l][0], F, C, F.dn_zc, p);
        h->launches++;
    }
    const MgLevel &last = h->mg[nl - 1];
    const size_t smem = (size_t)3 * (last.nx + 2) * (last.ny + 2) * (last.nz + 2) * sizeof(float);
    k_mg_coarse<<<1, 1024, smem, s>>>(last, p);
    h->launches++;
    for (int l = nl - 2; l >= 0; --l) {
        const MgLevel &F = h->mg[l];
        const dim3 g((F.nx + 1 + kUpTX - 1) / kUpTX, (F.ny + kUpTY - 1) / kUpTY, (F.nz + F.up_zc - 1) / F.up_zc);
        if (l == 0) {
            CgParams q = p;
            q.nblocks = g.x * g.y * g.z;
            k_mg_up<true><<<g, kUpNT, kUpSmem, s>>>(h->tm_mg[0][1], h->tm_mg[0][2], F, z, F.up_zc, q);
        } else {
            k_mg_up<false><<<g, kUpNT, kUpSmem, s>>>(h->tm_mg[l][1], h->tm_mg[l][2], F, F.e, F.up_zc, p);
        }
        h->launches++;
    }
}

// Dense (x fastest) <-> pitched level-0 layout; the pitched array gets 0 off
// the interior (ghost layer and row padding).
__global__ void k_mg_dense_in(const float *__restrict__ r, float *__restrict__ rp, int nx, int ny, int nz,
                              int px) {
    const long long n = (long long)px * ny * nz;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(q % px);
        const long long jk = q / px;
        const int j = (int)(jk % ny), k = (int)(jk / ny);
        const bool in = i >= 1 && i <= nx - 2 && j >= 1 && j <= ny - 2 && k >= 1 && k <= nz - 2;
        rp[q] = in ? r[((long long)k * ny + j) * nx + i] : 0.f;
    }
}

__global__ void k_mg_dense_out(const float *__restrict__ zp, float *__restrict__ z, int nx, int ny, int nz,
                               int px) {
    const long long n = (long long)nx * ny * nz;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(q % nx);
        const long long jk = q / nx;
        const int j = (int)(jk % ny), k = (int)(jk / ny);
        const bool in = i >= 1 && i <= nx - 2 && j >= 1 && j <= ny - 2 && k >= 1 && k <= nz - 2;
        z[q] = in ? zp[((long long)k * ny + j) * px + i] : 0.f;
    }
}

}  // namespace kv

using namespace kv;

extern "C" kv_status kv_apply_preconditioner(kv_handle *h, int nx, int ny, int nz, const float *r, float *z,
                                             double *rz) {
    if (!h || !r || !z) return set_error(h, KV_ERR_ARG, "kv_apply_preconditioner: null handle or pointer");
    if (nx != h->nx || ny != h->ny || nz != h->nz)
        return set_error(h, KV_ERR_ARG, "kv_apply_preconditioner: grid %dx%dx%d is not the handle's %dx%dx%d", nx, ny,
                         nz, h->nx, h->ny, h->nz);
    if (h->sticky) return KV_ERR_STATE;
    if (h->precision != KV_FP32)
        return set_error(h, KV_ERR_UNSUPPORTED, "kv_apply_preconditioner: the multigrid cycle needs an FP32 handle");
    kv_status st = mg_prepare(h);
    if (st != KV_OK) return st;
    cudaStream_t s = h->stream;
    // control block: "running" with zero iterations and ticket, r.z slot cleared
    cudaError_t e = cudaMemcpyAsync(h->ctrl_host, h->ctrl, kCtrlWords * sizeof(long long), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_check(h, e, "kv_apply_preconditioner");
    if (h->ctrl_host[kErrFlags] & 1)
        return set_error(h, KV_ERR_STATE, "kv_apply_preconditioner: the handle has an unread device timeout");
    h->ctrl_host[kCgStatus] = kCgRunning;
    h->ctrl_host[kCgIters] = 0;
    h->ctrl_host[kCgTicket] = 0;
    for (int q = 0; q < kCgScalars; ++q) h->scal_host[q] = 0.0;
    e = cudaMemcpyAsync(h->ctrl, h->ctrl_host, kCtrlWords * sizeof(long long), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(h->scal, h->scal_host, kCgScalars * sizeof(double), cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return cuda_check(h, e, "kv_apply_preconditioner");
    const int blocks = 148 * 8;
    k_mg_dense_in<<<blocks, 256, 0, s>>>(r, h->mg[0].r, h->nx, h->ny, h->nz, h->px);
    CgParams p{};
    p.pcg = 1;
    p.rbuf = h->mg[0].r;
    p.rfield = 0;
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
    p.zc = 1;
    p.nblocks = 1;  // mg_apply sets the top level's block count
    mg_apply(h, p);
    k_mg_dense_out<<<blocks, 256, 0, s>>>((const float *)h->cgv + h->Np, z, h->nx, h->ny, h->nz, h->px);
    h->launches += 2;
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_check(h, e, "kv_apply_preconditioner launch");
    e = cudaMemcpyAsync(h->ctrl_host, h->ctrl, kCtrlWords * sizeof(long long), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(h->scal_host, h->scal, kCgScalars * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_check(h, e, "kv_apply_preconditioner");
    if (h->ctrl_host[kErrFlags] & 1)
        return set_error(h, KV_ERR_TIMEOUT, "kv_apply_preconditioner: a bounded device wait gave up");
    if (rz) *rz = h->scal_host[kRR];
    // the top level sets non-finite or breakdown (r.z <= 0, e.g. r = 0) in the
    // control word; only the non-finite case is an error here
    if (h->ctrl_host[kCgStatus] == kCgNonfinite)
        return set_error(h, KV_ERR_NONFINITE, "kv_apply_preconditioner: r.z is not finite");
    return KV_OK;
}

