// kv_internal.cuh -- handle layout, launch parameters and device helpers shared
// by the libkv translation units (step kernels, projection kernels, C ABI).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "../../include/kv.h"

namespace kv {

// Rows are padded to a multiple of this many elements so that every row
// starts on a 128-byte boundary (float) and float4/TMA accesses stay aligned.
constexpr int kPitchAlign = 32;

// Planes per thread column in the CG passes.
constexpr int kCgZc = 16;

// Device control block of a handle (one allocation, int64 words).
enum CtrlWord {
    kStep = 0,       // steps taken since reset (read by every step kernel)
    kStepTicket = 1, // last-block ticket of the step kernels
    kErrFlags = 2,   // bit 0: mbarrier timeout, bit 1: trace overflow
    kCgStatus = 3,   // CG control word (CgCtl)
    kCgIters = 4,    // CG iterations so far
    kCgTicket = 5,   // last-block ticket of the CG kernels
    kCgRefine = 6,   // true-residual evaluations
    kCgMaxIter = 7,  // iteration cap
    kCtrlWords = 16
};

enum CgCtl : long long {
    kCgRunning = 0,
    kCgConverged = 1,
    kCgBreakdown = 2,
    kCgNonfinite = 3,
    kCgNeedTrue = 4,  // inner cycle finished: evaluate the true residual
    kCgMaxIterHit = 5
};

// Device scalars of the CG (doubles).
enum CgScalar {
    kRR = 0,      // r.r of the current recursive residual
    kPAP = 1,     // p.Ap
    kAlpha = 2,
    kBeta = 3,
    kBB = 4,      // ||b||^2
    kRR0 = 5,     // r.r at the start of the current inner cycle
    kTrue2 = 6,   // ||b - A phi||^2 of the last true-residual pass
    kTol = 7,     // tolerance on sqrt(true2 / bb)
    kInner = 8,   // inner-cycle reduction factor on ||r||
    kRRLast = 9,  // last recursive r.r (statistics)
    kWarmA = 10,  // (A phi0).b of a warm start
    kWarmC = 11,  // |A phi0|^2 of a warm start
    kCgScalars = 16
};

struct StepParams {
    int nx, ny, nz, px;
    long long Np;        // px * ny * nz (elements per component)
    double A, B;         // homogeneous coefficients (dt^2 G/(rho dx^2), dt eta/(rho dx^2))
    float Af, Bf;        // the same in FP32
    const float *g;      // envelope table on the device
    int n_g;
    int g_const_on;      // 1: use g_const for every step instead of the table
    float g_const;
    long long *ctrl;     // control block
    const int *sensors;  // 3 * ns node indices
    const int *sens_off; // nz + 1 offsets into sens_ord: sensors of plane k
    const int *sens_ord; // sensor indices sorted by plane
    int ns;
    void *traces;        // [cap][ns][3]
    int cap;
    int zc;              // planes per block (z chunk)
    int nblocks;         // blocks in the launch
    const float4 *lab_tab;  // per class: (A', B', -, -) pointwise, (m, e, 1/rho, -) flux form
    int n_lab;
};

// One case of a batched step (device table entry; CUtensorMap carries its own
// 64-byte alignment).
struct BatchCase {
    CUtensorMap tm_state[2];
    CUtensorMap tm_coef;
    const float *F;
    float *state[2];
    StepParams p;         // nblocks = this case's blocks
    int gx, gy, gz;       // tile grid of this case
    int block_begin;      // first block of this case in the batched launch
};

struct CgParams {
    int nx, ny, nz, px;
    long long Np;
    double inv_dx2;      // 1/dx^2
    double inv_dx;       // 1/dx
    long long *ctrl;
    double *scal;
    double *partials;    // one double per block (or two)
    int zc;
    int nblocks;
    int pcg;             // 1: preconditioned CG (z in the CG vector slot of r, r in rbuf)
    float *rbuf;         // residual of the TMA update pass (FP32)
    int rfield;          // field of rbuf's tensor map holding r
    int zero_start;      // 1: phi is 0 at the first residual evaluation (r = b, no stencil)
};

// One level of the multigrid preconditioner: nx, ny, nz interior cells, arrays
// of (nx + 2) x (ny + 2) x (nz + 2) with a zero ghost layer and row pitch px
// (level 0 is the handle's pitched grid).
constexpr int kMgMaxLevels = 12;
// Column of one block of the TMA CG passes (x, y nodes); the multigrid's fine
// residual is staged by the update pass with the same box.
constexpr int kCgTX = 64, kCgTY = 8;
struct MgLevel {
    int nx, ny, nz, px;
    long long n;         // elements of one array (px * (ny + 2) * (nz + 2))
    double h2;           // grid spacing squared
    float h2f, sh;       // h^2 and the smoother S = omega h^2 / 6 in FP32
    float *r, *e;        // right-hand side, solution (level 0: r only, z goes to the CG)
    int dn_zc, up_zc;    // planes per block: restriction to the next level (coarse
                         // planes), prolongation and post-smoothing (this level's)
};

}  // namespace kv

struct kv_handle {
    int nx, ny, nz, px;
    long long Np;
    double dx, dt;
    int precision;        // KV_FP32 / KV_FP64
    size_t esize;         // bytes per state element
    cudaStream_t stream;
    int own_stream;
    int device;

    // medium
    int het;
    int op;                // kv_operator: KV_OP_POINTWISE or KV_OP_DIVERGENCE
    double A_s, B_s, S_s;  // homogeneous scalars (A, B already divided by dx^2)
    void *coef;            // het: [2][Np] (A', B') pointwise, [3][Np] (m, e, 1/rho) divergence form
    int coef_fields;       // fields allocated in coef
    unsigned char *labels; // [Np] class of each node's coefficients when n_labels > 0
    float4 *lab_tab;       // [kMaxLabels] coefficients of each class (see StepParams)
    unsigned long long *lab_keys;  // classification scratch: hash slots, slot ids, counters
    int n_labels;          // distinct coefficient tuples of an FP32 medium (0: fields are read)
    int medium_encoding;   // KV_MEDIUM_AUTO / KV_MEDIUM_FIELDS
    void *S;               // [Np] dt^2/rho when het
    double dt_max;

    // state: two buffers of [6][Np] (u_x, u_y, u_z, d_x, d_y, d_z)
    void *state[2];
    int cur;
    void *F;               // [3][Np] dt^2 f_S0 / rho
    int have_force;

    // envelope, sensors, traces
    float *g_dev;
    int n_g;
    int *sens_dev;
    int ns;
    int cap;
    void *traces;
    long long *ctrl;       // kv::kCtrlWords
    long long steps_host;

    // projection
    void *cgv;             // [4][Np] CG vectors in one allocation: p[0], r, p[1], e
    void *r;               // [Np] residual (float or double), inside cgv
    void *p[2];            // [Np] search direction, ping-pong by iteration parity
    void *e;               // [Np] correction accumulated since the last replacement
    CUtensorMap tm_cg_h2, tm_cg_h1, tm_cg_c1;  // TMA views of cgv (FP32)
    int cg_tma_ready;
    int cg_zc;             // planes per block of the TMA CG passes (0: default)
    int cg_ns;             // shared-memory stages of the TMA CG passes (4 or 8)

    // multigrid preconditioner (projection mode 4), allocated on first use
    int mg_levels;
    kv::MgLevel mg[kv::kMgMaxLevels];
    float *mg_pool;        // all level arrays in one allocation
    double *fcg_pool;      // flexible CG (mode 2) vectors, allocated on first use
    CUtensorMap tm_mg_r;   // TMA view of the fine residual (mg[0].r)
    CUtensorMap tm_mg[kv::kMgMaxLevels][3];  // per level: r (restriction box), r (prolongation box),
                                             // next level's e (prolongation box)
    double *phi;           // [Np]
    double *b;             // [Np] right-hand side
    double *scal;          // kv::kCgScalars
    double *partials;      // reduction partials
    double *dtmin;         // kDtBlocks block minima of the stability reduction
    int partials_len;
    float *fstage;         // [3][Np] pitched copy of the force input
    long long *ctrl_host;  // pinned mirror of the control block
    double *scal_host;     // pinned mirror of the scalars

    // FP32 step kernel configuration and TMA descriptors
    int variant, tx, ty, zc, ns_stages;
    CUtensorMap tm_state[2], tm_coef;
    int tma_ready;

    // CUDA graph of a block of steps (one per starting buffer)
    cudaGraphExec_t graph[2];
    int graph_steps;

    struct kv_net *net;    // learned warm start (kv_attach_net), not owned
    double warm_alpha;     // scaling applied to the last learned start
    int g_const_on;        // steps use g = 1 (kv_step_force)
    int phi_valid;         // phi holds the last projection's potential

    long long launches;
    int sticky;
    char err[512];
};

// Learned warm start (kv_net.cu)
extern "C" {
struct kv_net;
kv_status kv_net_predict(struct kv_net *n, int nx, int ny, int nz, double dx, const float *b, float *phi);
float *kv_net_stage_b(struct kv_net *n);
float *kv_net_stage_phi(struct kv_net *n);
int kv_net_fits(struct kv_net *n, int nx, int ny, int nz);
}

namespace kv {

kv_status set_error(kv_handle *h, kv_status st, const char *fmt, ...);
kv_status cuda_check(kv_handle *h, cudaError_t e, const char *what);

// Step kernels (kv_step.cu)
kv_status step_prepare(kv_handle *h);                  // TMA maps, smem attributes
kv_status step_launch(kv_handle *h, int from_buffer);  // one step from state[from]
kv_status step2_launch(kv_handle *h, int from_buffer); // two steps (variant 2), one buffer swap
kv_status launch_wait_selftest(kv_handle *h);          // bounded wait on an mbarrier nothing completes
void *tensor_map_encoder(kv_handle *h);                // cuTensorMapEncodeTiled (NULL if unavailable)

// Step kernel kinds: homogeneous, pointwise heterogeneous (Sec. 3.1),
// divergence-form heterogeneous.
enum { kKindHomo = 0, kKindPoint = 1, kKindDiv = 2, kKindLabel = 3, kKindDivLabel = 4 };
inline int step_kind(const kv_handle *h) {
    return !h->het ? kKindHomo : (h->op == KV_OP_DIVERGENCE ? kKindDiv : kKindPoint);
}
// Kind of the single-step TMA kernel: a medium with few distinct folded
// coefficient tuples is read as one class byte per node plus a table
// (kKindLabel for the pointwise operator, kKindDivLabel for the flux form).
inline int tma_kind(const kv_handle *h) {
    const int k = step_kind(h);
    if (h->n_labels > 0 && k == kKindPoint) return kKindLabel;
    if (h->n_labels > 0 && k == kKindDiv) return kKindDivLabel;
    return k;
}

// Batched step (kv_step.cu)
kv_status batch_kernel_for(int tx, int ty, int ns, int kind, void **kernel, size_t *smem, int *nt);
kv_status batch_fill_case(kv_handle *h, struct BatchCase *bc, int tx, int ty, int zc, int begin,
                          int *blocks);
kv_status batch_launch(void *kernel, const struct BatchCase *table, int ncases, int total_blocks,
                       int nt, size_t smem, int from, cudaStream_t s);

// 4D float32 tensor map over [fields][nz][ny][px] with box (bx, by, 1, fields_box)
kv_status encode_tensor_4d(kv_handle *h, CUtensorMap *tm, void *base, int fields, int bx, int by,
                           int fields_box);

// Class encoding of an FP32 medium (kv_label.cu): after the fold, count the
// distinct folded coefficient tuples ((A', B') pointwise, (m, e, 1/rho) flux
// form); with at most kMaxLabels of them, write one class byte per node and
// the class table, else read the fields.
// Synchronises the handle's stream. medium_labels_free releases the arrays.
constexpr int kMaxLabels = 256;
constexpr int kLabSlots = 1024;  // open-addressing slots of the pair hash
kv_status medium_classify(kv_handle *h);
void medium_labels_free(kv_handle *h);

// Projection kernels (kv_cg.cu)
kv_status project(kv_handle *h, double tol, int max_iter, int mode, float *fs_out, kv_cg_stats *st);
// Flexible CG with the attached network as preconditioner (projection mode 2, kv_fcg.cu)
kv_status project_fcg(kv_handle *h, double tol, int max_iter, int *status, int *iters, double *true2,
                      double bb);

// Multigrid preconditioner (kv_mg.cu): level setup and one application
// z = M r from mg[0].r into cgv field 1, with r.z reduced into scal[kRR].
int cg_auto_zc(const kv_handle *h);  // default z chunk of the TMA CG passes
kv_status mg_prepare(kv_handle *h);
void mg_apply(kv_handle *h, const CgParams &p);

// Device stability limit over dense fields: kDtBlocks block minima in
// `scratch` (kDtBlocks doubles; NULL = a temporary allocation), synchronising.
constexpr int kDtBlocks = 592;
kv_status stable_dt_device(cudaStream_t stream, double *scratch, int nx, int ny, int nz, int px, double dx,
                           const float *G, double Gs, const float *rho, double rhos, const float *eta,
                           double etas, int op, double *out);

inline long long round_up(long long a, long long b) { return (a + b - 1) / b * b; }

}  // namespace kv

// ---------------------------------------------------------------------------
// Device helpers
// ---------------------------------------------------------------------------

template <typename T>
__device__ __forceinline__ T kv_fma(T a, T b, T c);
template <>
__device__ __forceinline__ float kv_fma<float>(float a, float b, float c) { return __fmaf_rn(a, b, c); }
template <>
__device__ __forceinline__ double kv_fma<double>(double a, double b, double c) { return __fma_rn(a, b, c); }

template <typename T>
__device__ __forceinline__ T kv_add(T a, T b);
template <>
__device__ __forceinline__ float kv_add<float>(float a, float b) { return __fadd_rn(a, b); }
template <>
__device__ __forceinline__ double kv_add<double>(double a, double b) { return __dadd_rn(a, b); }

template <typename T>
__device__ __forceinline__ T kv_sub(T a, T b);
template <>
__device__ __forceinline__ float kv_sub<float>(float a, float b) { return __fsub_rn(a, b); }
template <>
__device__ __forceinline__ double kv_sub<double>(double a, double b) { return __dsub_rn(a, b); }

template <typename T>
__device__ __forceinline__ T kv_mul(T a, T b);
template <>
__device__ __forceinline__ float kv_mul<float>(float a, float b) { return __fmul_rn(a, b); }
template <>
__device__ __forceinline__ double kv_mul<double>(double a, double b) { return __dmul_rn(a, b); }

// One node of the increment-form update. su / sd are the sums of the six
// neighbours of u / d, formed by the caller as ((xm + xp) + (ym + yp)) + (zm + zp).
//   L^u = su - 6u,  L^d = sd - 6d
//   d'  = d + A L^u + B L^d + gF,  u' = u + d'
// Every operation is an explicit rounding step so that all step kernels give
// bit-identical results.
template <typename T>
__device__ __forceinline__ void kv_update(T u, T su, T d, T sd, T A, T B, T g, T F, T &u_out,
                                          T &d_out) {
    T lu = kv_fma(T(-6), u, su);
    T ld = kv_fma(T(-6), d, sd);
    T dn = kv_fma(g, F, d);
    dn = kv_fma(B, ld, dn);
    dn = kv_fma(A, lu, dn);
    d_out = dn;
    u_out = kv_add(u, dn);
}

// One node of the divergence-form update (heterogeneous operator
// (1/rho) div(G grad u) + (1/rho) div(eta grad udot)). Neighbour order
// xm, xp, ym, yp, zm, zp; face weights wm[f] = (m_c + m_f)/2 with m = dt^2 G/dx^2,
// we[f] = (e_c + e_f)/2 with e = dt eta/dx^2; r = 1/rho at the node.
//   s  = sum_f wm[f] (u_f - u) + sum_f we[f] (d_f - d)
//   d' = d + r s + gF,  u' = u + d'
// Explicit rounding steps in a fixed order, as in kv_update.
template <typename T>
__device__ __forceinline__ T face_weight(T c, T nb) {
    return kv_mul(T(0.5), kv_add(c, nb));
}

template <typename T>
__device__ __forceinline__ void kv_update_div(T u, const T (&nu)[6], T d, const T (&nd)[6],
                                              const T (&wm)[6], const T (&we)[6], T r, T g, T F,
                                              T &u_out, T &d_out) {
    T s = kv_mul(wm[0], kv_sub(nu[0], u));
#pragma unroll
    for (int f = 1; f < 6; ++f) s = kv_fma(wm[f], kv_sub(nu[f], u), s);
#pragma unroll
    for (int f = 0; f < 6; ++f) s = kv_fma(we[f], kv_sub(nd[f], d), s);
    T dn = kv_fma(g, F, d);
    dn = kv_fma(r, s, dn);
    d_out = dn;
    u_out = kv_add(u, dn);
}

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Deterministic block sum of a double (fixed reduction tree for a given
// blockDim). Every thread of the block must call it; the result is returned
// to all threads.
__device__ __forceinline__ double block_sum_d(double v, double *sh /* >= 33 doubles */) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nw = (blockDim.x + 31) >> 5;
    v = warp_sum_d(v);
    __syncthreads();
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    double t = (threadIdx.x < nw) ? sh[threadIdx.x] : 0.0;
    if (warp == 0) t = warp_sum_d(t);
    if (threadIdx.x == 0) sh[32] = t;
    __syncthreads();
    double r = sh[32];
    __syncthreads();
    return r;
}

namespace kv {

// ---------------------------------------------------------------------------
// PTX helpers: mbarrier and TMA (sm_90+ forms, valid on sm_103a)
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_init_fence() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait: gives up after ~2^31 SM clocks (about a second at 2 GHz).
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity) {
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    while (true) {
        if (mbar_try_wait(bar, parity)) return true;
        if (clock64() - t0 > (1ll << 31)) return false;
    }
}
__device__ __forceinline__ void tma_load_4d(uint32_t dst, const CUtensorMap *tm, int c0, int c1,
                                            int c2, int c3, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(tm)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(bar)
        : "memory");
}

}  // namespace kv
