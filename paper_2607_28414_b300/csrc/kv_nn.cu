// kv_nn.cu -- tensor-core building blocks of the learned warm start: 3x3x3
// convolution forward, input gradient and weight gradient as implicit GEMMs on
// the 5th-generation tensor cores (tcgen05.mma, BF16 operands staged by TMA in
// shared memory, FP32 accumulators in tensor memory), and the bias gradient and
// weight flip.
//
// Tensors are channel-last [z][y][x][C] BF16 with C in {16, 32, 64}. Weights
// W[t][ci][co], tap t = (dz+1)*9 + (dy+1)*3 + (dx+1), zero padding of one voxel:
//   out[v][co] = bias[co] + sum_{t,ci} in[v + d(t)][ci] W[t][ci][co].
// The input gradient is the same convolution with Wt[t][co][ci] = W[26-t][ci][co].
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include <algorithm>

#include "kv_internal.cuh"

using bf16 = __nv_bfloat16;

namespace kv {

// ---------------------------------------------------------------------------
// Forward (and input-gradient) convolution on the 5th-generation tensor cores
//
// Implicit GEMM over output tiles of 4 x (128 voxels x COUT): the voxels of an
// 8 (x) x 16 (y) tile on four consecutive z planes. A tile's input brick (10 x
// 18 x 6 voxels with the one-voxel halo) arrives by one 5D TMA box in the
// canonical no-swizzle K-major layout of the tensor cores: channels in chunks of
// 8 (16 bytes), brick[cc][z][y][x][8]. For tap (dx, dy, dz) the A operand (128
// voxels x 16 channels) is the brick seen from voxel offset (dx, dy, dz + zt):
// 8-row core matrices are 8 consecutive x voxels (16-byte rows), the 16 row
// groups step by one brick row (SBO = 160 bytes), and the two 8-channel halves
// of K step by one channel chunk (LBO = 1080 x 16 bytes). So the 27 taps need no
// gather: each is a descriptor with a different start address.
//
// The three z taps of one (dx, dy) share the A operand: the brick plane p seen
// from (dx, dy) is the input of tap dz for output plane p - dz. So the weights
// of a (dy, dx) group are stacked along N in the order dz = 2, 1, 0 and one MMA
// of N = (number of valid dz) x COUT accumulates into the adjacent accumulator
// columns of output planes p - dz_hi .. p - dz_lo: per tile six planes x nine
// (dx, dy) groups of MMAs instead of 27 taps x four planes, with half the A
// reads from shared memory. Each tap's weights W[t][ci][co] arrive by TMA
// straight from their own layout: a 4D view (8 co, ci, co chunk, tap) lands as
// [co chunk][ci][8], the MN-major core matrices of the B operand (8 ci rows x
// 8 co, 128 contiguous bytes; LBO = 128 bytes along K, SBO = CIN x 16 bytes
// along N, uniform across the stacked taps). All 27 taps stay resident when
// they fit beside the bricks; otherwise the nine (dy, dx) groups of three taps
// stream through a 3-slot ring, refilled while the tensor cores work. An MMA
// covers a varying set of output planes, so the accumulators are zeroed by the
// epilogue (tcgen05.st) and every MMA accumulates.
//
// Persistent, warp-specialised blocks walk the tiles (tile = first + i x grid):
//   warp 4  (one thread) issues the TMA copies: bricks into a ring of NB
//           buffers (two when they fit, so the next tile's brick lands while
//           this one is multiplied), weights once or per group;
//   warp 5  (one thread) issues tcgen05.mma (kind::f16, BF16 operands, FP32
//           accumulators in tensor memory) into one of two accumulator sets
//           of 4 x COUT columns, and commits to mbarriers that free the brick,
//           the weight slot and hand the accumulators to the epilogue;
//   warps 0-3 read the accumulators with tcgen05.ld (warp w owns TMEM lanes
//           32w .. 32w + 31 = tile rows m = y x 8 + x), add the bias, apply
//           ReLU, store, zero the accumulator set and free it, so the
//           epilogue of tile i overlaps the MMAs of tile i + 1.
// Every wait is bounded (~1 s of SM clocks); a wait that gives up sets a
// shared abort flag and the device timeout flag, every role stops issuing,
// the copies and MMAs in flight are awaited (bounded) and the tensor memory
// is freed before the block exits.
// ---------------------------------------------------------------------------
constexpr int kTcX = 8, kTcY = 16, kTcZ = 4;                      // 4 x 128 voxels per tile
constexpr int kTcBX = kTcX + 2, kTcBY = kTcY + 2, kTcBZ = kTcZ + 2;
constexpr int kTcBrick = kTcBX * kTcBY * kTcBZ;                   // 1080 voxels with halo
constexpr int kConvThreads = 192;                                 // 4 epilogue warps + TMA + MMA

template <int CIN, int COUT>
struct ConvTc {
    static constexpr size_t kBudget = 220 * 1024;
    static constexpr size_t kBrickBytes = (size_t)(CIN / 8) * kTcBrick * 16;
    static constexpr size_t kTapBytes = (size_t)CIN * COUT * 2;
    static constexpr size_t kAllW = 27 * kTapBytes;
    static constexpr size_t kGroupBytes = 3 * kTapBytes;          // one (dy, dx) group: dz = 2, 1, 0
    static constexpr int NB = 2 * kBrickBytes + 3 * kGroupBytes <= kBudget ? 2 : 1;
    static constexpr bool kResident = NB * kBrickBytes + kAllW <= kBudget;
    static constexpr int NWS = kResident ? 1 : 3;                 // weight slots
    static constexpr size_t kWBytes = kResident ? kAllW : 3 * kGroupBytes;
    static constexpr int kBars = 2 * NB + 2 * NWS + 4;
    static constexpr size_t kSmem = NB * kBrickBytes + kWBytes + 8 * kBars + 16;
    static constexpr uint32_t kAccCols = kTcZ * COUT;             // one accumulator set
    static constexpr uint32_t kCols = 2 * kAccCols < 32 ? 32 : 2 * kAccCols;
    static_assert(kSmem <= 227 * 1024, "shared memory of a convolution block");
    static_assert(kCols <= 512, "tensor memory of a convolution block");
    // a block that takes all tensor memory must also take more than half the shared memory
    static_assert(kCols < 512 || kSmem > 114 * 1024, "one block per SM when it takes all tensor memory");
};

// Shared-memory matrix descriptor: no swizzle, K-major core matrices of 8
// rows x 16 bytes; lbo = byte stride between core matrices along K, sbo =
// byte stride between 8-row groups along M (or N).
__device__ __forceinline__ uint64_t umma_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = (uint64_t)((addr >> 4) & 0x3FFFu);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;  // descriptor version of the 5th-generation tensor cores
    return d;                // base offset 0, layout type 0 (no swizzle)
}

// Instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, both
// K-major, N and M as given.
__host__ __device__ constexpr uint32_t umma_idesc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void umma_bf16(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc,
                                          uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void umma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}

// 16 consecutive FP32 columns of this thread's TMEM lane (warp-collective).
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, "
        "%13, %14, %15}, [%16];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// Zero 16 consecutive FP32 columns of this thread's TMEM lane (warp-collective).
__device__ __forceinline__ void tmem_zero16(uint32_t taddr) {
    const uint32_t z = 0;
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, "
        "%1, %1, %1};" ::"r"(taddr),
        "r"(z)
        : "memory");
}
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

__device__ int g_conv_timeout;  // set when a bounded wait of a convolution gave up

__device__ __forceinline__ void tma_load_5d(uint32_t dst, const CUtensorMap *tm, int c0, int c1, int c2, int c3,
                                            int c4, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.5d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4, %5, %6}], [%7];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(tm)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(c4), "r"(bar)
        : "memory");
}

template <typename OutT>
__device__ __forceinline__ void store16(OutT *dst, const float (&v)[16]);
template <>
__device__ __forceinline__ void store16<float>(float *dst, const float (&v)[16]) {
#pragma unroll
    for (int i = 0; i < 16; i += 4)
        *reinterpret_cast<float4 *>(dst + i) = make_float4(v[i], v[i + 1], v[i + 2], v[i + 3]);
}
template <>
__device__ __forceinline__ void store16<bf16>(bf16 *dst, const float (&v)[16]) {
    uint32_t w[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const __nv_bfloat162 h = __floats2bfloat162_rn(v[2 * i], v[2 * i + 1]);
        w[i] = *reinterpret_cast<const uint32_t *>(&h);
    }
    *reinterpret_cast<uint4 *>(dst) = make_uint4(w[0], w[1], w[2], w[3]);
    *reinterpret_cast<uint4 *>(dst + 8) = make_uint4(w[4], w[5], w[6], w[7]);
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

template <int CIN, int COUT, typename OutT>
__global__ void __launch_bounds__(kConvThreads, 1)
k_conv_fwd(const __grid_constant__ CUtensorMap tm_in, const __grid_constant__ CUtensorMap tm_w,
           const float *__restrict__ bias, OutT *__restrict__ out, int nx, int ny, int nz, int relu) {
    using C = ConvTc<CIN, COUT>;
    constexpr int NB = C::NB, NWS = C::NWS;
    extern __shared__ __align__(1024) unsigned char sm[];
    const uint32_t sm0 = smem_u32(sm);
    const uint32_t wts0 = sm0 + (uint32_t)(NB * C::kBrickBytes);
    uint64_t *bars = reinterpret_cast<uint64_t *>(sm + NB * C::kBrickBytes + C::kWBytes);
    const uint32_t bar0 = smem_u32(bars);
    // barrier addresses: brick full / empty, weight full / empty, accumulator full / empty
    auto b_full = [&](int b) { return bar0 + 8u * (uint32_t)b; };
    auto b_empty = [&](int b) { return bar0 + 8u * (uint32_t)(NB + b); };
    auto w_full = [&](int s) { return bar0 + 8u * (uint32_t)(2 * NB + s); };
    auto w_empty = [&](int s) { return bar0 + 8u * (uint32_t)(2 * NB + NWS + s); };
    auto a_full = [&](int a) { return bar0 + 8u * (uint32_t)(2 * NB + 2 * NWS + a); };
    auto a_empty = [&](int a) { return bar0 + 8u * (uint32_t)(2 * NB + 2 * NWS + 2 + a); };
    uint32_t *tslot = reinterpret_cast<uint32_t *>(bars + C::kBars);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tslot + 1);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int ntx = (nx + kTcX - 1) / kTcX, nty = (ny + kTcY - 1) / kTcY, ntz = (nz + kTcZ - 1) / kTcZ;
    const int ntiles = ntx * nty * ntz;
    const int my_tiles = ((int)blockIdx.x < ntiles) ? (ntiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
    auto tile_origin = [&](int i, int &x0, int &y0, int &z0) {
        const int t = (int)blockIdx.x + i * (int)gridDim.x;
        x0 = (t % ntx) * kTcX;
        y0 = ((t / ntx) % nty) * kTcY;
        z0 = (t / (ntx * nty)) * kTcZ;
    };

    if (warp == 0) {  // tensor memory for the two accumulator sets
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                     "r"(C::kCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        for (int b = 0; b < NB; ++b) {
            mbar_init(b_full(b), 1);
            mbar_init(b_empty(b), 1);
        }
        for (int q = 0; q < NWS; ++q) {
            mbar_init(w_full(q), 1);
            mbar_init(w_empty(q), 1);
        }
        for (int a = 0; a < 2; ++a) {
            mbar_init(a_full(a), 1);
            mbar_init(a_empty(a), 128);
        }
        *abort_flag = 0;
        mbar_init_fence();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;
    if (warp < 4) {  // both accumulator sets start at zero (every MMA accumulates)
        for (uint32_t c = 0; c < 2 * C::kAccCols; c += 16) tmem_zero16(tmem + ((uint32_t)(32 * warp) << 16) + c);
        tmem_wait_st();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    auto give_up = [&]() {
        *abort_flag = 1;
        atomicExch(&g_conv_timeout, 1);
    };

    if (warp == 4) {
        // ---------------- TMA producer ----------------
        if (lane == 0 && my_tiles > 0) {
            int issued_b = 0, issued_w = 0;  // bricks and weight groups whose copies were issued
            // the three taps of group g = (dy, dx) in the order dz = 2, 1, 0
            auto load_group = [&](uint32_t dst, int g, uint32_t bar) {
                const int dy = g / 3, dx = g % 3;
                for (int dz = 2; dz >= 0; --dz)
                    tma_load_4d(dst + (uint32_t)((2 - dz) * C::kTapBytes), &tm_w, 0, 0, 0, dz * 9 + dy * 3 + dx,
                                bar);
            };
            if (C::kResident) {
                mbar_expect_tx(w_full(0), (uint32_t)C::kAllW);
                for (int g = 0; g < 9; ++g) load_group(wts0 + (uint32_t)(g * C::kGroupBytes), g, w_full(0));
            }
            for (int i = 0; i < my_tiles && !*abort_flag; ++i) {
                const int b = i % NB, use = i / NB;
                if (use > 0 && !mbar_wait_bounded(b_empty(b), (uint32_t)((use - 1) & 1))) {
                    give_up();
                    break;
                }
                int x0, y0, z0;
                tile_origin(i, x0, y0, z0);
                mbar_expect_tx(b_full(b), (uint32_t)C::kBrickBytes);
                tma_load_5d(sm0 + (uint32_t)(b * C::kBrickBytes), &tm_in, 0, x0 - 1, y0 - 1, z0 - 1, 0, b_full(b));
                issued_b = i + 1;
                if (!C::kResident) {
                    for (int g = 0; g < 9; ++g) {
                        const int q = issued_w % NWS, u = issued_w / NWS;
                        if (u > 0 && !mbar_wait_bounded(w_empty(q), (uint32_t)((u - 1) & 1))) {
                            give_up();
                            break;
                        }
                        mbar_expect_tx(w_full(q), (uint32_t)C::kGroupBytes);
                        load_group(wts0 + (uint32_t)(q * C::kGroupBytes), g, w_full(q));
                        ++issued_w;
                    }
                }
            }
            if (*abort_flag) {  // the copies in flight land before the block exits
                for (int b = 0; b < NB && b < issued_b; ++b) {
                    const int last = issued_b - 1 - ((issued_b - 1 - b) % NB);
                    mbar_wait_bounded(b_full(b), (uint32_t)((last / NB) & 1));
                }
                if (C::kResident) {
                    mbar_wait_bounded(w_full(0), 0);
                } else {
                    for (int q = 0; q < NWS && q < issued_w; ++q) {
                        const int last = issued_w - 1 - ((issued_w - 1 - q) % NWS);
                        mbar_wait_bounded(w_full(q), (uint32_t)((last / NWS) & 1));
                    }
                }
            }
        }
    } else if (warp == 5) {
        // ---------------- MMA issuer ----------------
        if (lane == 0 && my_tiles > 0) {
            // N = 1, 2 or 3 stacked taps of COUT channels; B MN-major
            constexpr uint32_t idesc_n[3] = {umma_idesc_bf16(128, COUT) | (1u << 16),
                                             umma_idesc_bf16(128, 2 * COUT) | (1u << 16),
                                             umma_idesc_bf16(128, 3 * COUT) | (1u << 16)};
            int used_w = 0, committed = 0;
            bool ok = !C::kResident || mbar_wait_bounded(w_full(0), 0);
            if (!ok) give_up();
            for (int i = 0; ok && i < my_tiles && !*abort_flag; ++i) {
                const int b = i % NB, a = i & 1;
                if (!mbar_wait_bounded(b_full(b), (uint32_t)((i / NB) & 1)) ||
                    (i >= 2 && !mbar_wait_bounded(a_empty(a), (uint32_t)(((i >> 1) - 1) & 1)))) {
                    give_up();
                    break;
                }
                tc_fence_after();
                const uint32_t brick = sm0 + (uint32_t)(b * C::kBrickBytes);
                const uint32_t acc = tmem + (uint32_t)a * C::kAccCols;
                for (int g = 0; g < 9; ++g) {
                    const int dy = g / 3, dx = g % 3;
                    uint32_t wg;
                    int q = 0;
                    if (C::kResident) {
                        wg = wts0 + (uint32_t)(g * C::kGroupBytes);
                    } else {
                        q = used_w % NWS;
                        if (!mbar_wait_bounded(w_full(q), (uint32_t)((used_w / NWS) & 1))) {
                            ok = false;
                            break;
                        }
                        tc_fence_after();
                        wg = wts0 + (uint32_t)(q * C::kGroupBytes);
                    }
#pragma unroll
                    for (int kk = 0; kk < CIN / 16; ++kk) {
#pragma unroll
                        for (int pz = 0; pz < kTcBZ; ++pz) {
                            // brick plane pz feeds output planes pz - dz for the dz with
                            // 0 <= pz - dz < kTcZ; their weights sit at stack rows 2 - dz
                            const int dz_hi = pz < 2 ? pz : 2, dz_lo = pz > kTcZ - 1 ? pz - (kTcZ - 1) : 0;
                            const uint64_t bd =
                                umma_desc(wg + (uint32_t)((2 - dz_hi) * C::kTapBytes + kk * 256), 128, CIN * 16);
                            const uint32_t vox = (pz * kTcBY + dy) * kTcBX + dx;
                            const uint64_t ad = umma_desc(brick + (uint32_t)((2 * kk * kTcBrick + vox) * 16),
                                                          kTcBrick * 16, kTcBX * 16);
                            umma_bf16(acc + (uint32_t)((pz - dz_hi) * COUT), ad, bd, idesc_n[dz_hi - dz_lo], 1u);
                        }
                    }
                    if (!C::kResident) {
                        umma_commit(w_empty(q));  // the slot refills once these MMAs are done
                        ++used_w;
                    }
                }
                if (!ok) {
                    give_up();
                    break;
                }
                umma_commit(b_empty(b));
                umma_commit(a_full(a));
                committed = i + 1;
            }
            if (*abort_flag && committed > 0) {  // the MMAs in flight finish before the block exits
                const int i = committed - 1;
                mbar_wait_bounded(a_full(i & 1), (uint32_t)((i >> 1) & 1));
            }
        }
    } else {
        // ---------------- epilogue (warps 0-3) ----------------
        const int m = 32 * warp + lane;
        for (int i = 0; i < my_tiles; ++i) {
            const int a = i & 1;
            if (*abort_flag || !mbar_wait_bounded(a_full(a), (uint32_t)((i >> 1) & 1))) {
                give_up();
                break;
            }
            tc_fence_after();
            int x0, y0, z0;
            tile_origin(i, x0, y0, z0);
            const int gx = x0 + (m % kTcX), gy = y0 + (m / kTcX);
#pragma unroll
            for (int zt = 0; zt < kTcZ; ++zt) {
                const int gz = z0 + zt;
                const bool inside = gx < nx && gy < ny && gz < nz;
#pragma unroll
                for (int c0 = 0; c0 < COUT; c0 += 16) {
                    float v[16];
                    tmem_ld16(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)(a * C::kAccCols + zt * COUT + c0), v);
#pragma unroll
                    for (int e = 0; e < 16; ++e) {
                        float q = v[e] + (bias ? bias[c0 + e] : 0.f);
                        v[e] = relu ? fmaxf(q, 0.f) : q;
                    }
                    if (inside) store16<OutT>(out + (((size_t)gz * ny + gy) * nx + gx) * COUT + c0, v);
                }
            }
            // the next tile on this set accumulates from zero
            for (uint32_t c = 0; c < C::kAccCols; c += 16)
                tmem_zero16(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)a * C::kAccCols + c);
            tmem_wait_st();
            tc_fence_before();
            mbar_arrive(a_empty(a));
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(C::kCols) : "memory");
}

// ---------------------------------------------------------------------------
// Weight gradient on the 5th-generation tensor cores
//
// gW[t][ci][co] = sum_v in[v + d(t)][ci] g[v][co]: a GEMM whose contraction
// runs over voxels. Both operands are taken MN-major straight from the
// channel-last tensors: a core matrix is 8 consecutive z voxels (the K rows,
// 16 bytes apart) x 8 channels (16 contiguous bytes). A block owns one dz
// (blockIdx.y) and sweeps chunks of XT x YT x 16 voxels. Per chunk, a 2-stage
// TMA ring lands
//   the input brick [y (YT+2)][x (XT+2)][channel chunk][z 16][8] from the
//     planes z + dz (zero fill outside the grid), and
//   the output-gradient tile [y][x][channel chunk][z 16][8];
// then, for every voxel column (x, y) and every dy, one thread issues MMAs with
//   A: 128 rows (dx, ci) = the brick seen from (x + dx, y + dy): consecutive dx
//      are NCC core matrices apart, so the three dx taps stack along M at one
//      uniform 256-byte stride (rows beyond 3 CIN are never stored);
//   B: N = COUT rows co of the gradient at (x, y);
//   K: the column's 16 z voxels (two core matrices, 128 bytes apart);
// into FP32 accumulators in tensor memory, one (128 x COUT) block per (dy, row
// chunk), kept across all chunks of the block. The epilogue reads them with
// tcgen05.ld and adds them to gW with vector atomics.
// ---------------------------------------------------------------------------
constexpr int kWgZ = 16;  // z voxels per chunk: two core matrices along K

template <int CIN, int COUT, int XT, int YT>
struct WgradTile {
    static constexpr int NCC = CIN / 8, NCO = COUT / 8;
    static constexpr int XB = XT + 2, YB = YT + 2;
    static constexpr size_t kBrick = (size_t)YB * XB * NCC * kWgZ * 16;
    static constexpr size_t kGrad = (size_t)YT * XT * NCO * kWgZ * 16;
    static constexpr size_t kStage = (kBrick + kGrad + 1023) / 1024 * 1024;
    static constexpr size_t kSmem = 2 * kStage + 64;  // + 4 mbarriers, TMEM address
    static constexpr bool fits() { return kSmem <= 227 * 1024; }
};

template <int CIN, int COUT>
struct WgradTc {
    // the largest voxel-column tile (8x8, 8x4, 4x4) whose two stages fit in shared memory
    static constexpr bool k88 = WgradTile<CIN, COUT, 8, 8>::fits(), k84 = WgradTile<CIN, COUT, 8, 4>::fits();
    static constexpr int TX = (k88 || k84) ? 8 : 4, TY = k88 ? 8 : 4;
    using T = WgradTile<CIN, COUT, TX, TY>;
    static constexpr int NQ = (3 * T::NCC + 15) / 16;  // 128-row chunks of the (dx, ci) rows
    static constexpr int kUsedCols = 3 * NQ * COUT;
    static constexpr uint32_t kCols = kUsedCols <= 32 ? 32 : kUsedCols <= 64 ? 64 : kUsedCols <= 128 ? 128
                                    : kUsedCols <= 256 ? 256 : 512;
    static_assert(T::fits(), "shared memory of a weight-gradient block");
    static_assert(kUsedCols <= 512, "tensor memory of a weight-gradient block");
    static_assert(kCols <= 256 || T::kSmem > 114 * 1024, "one block per SM when it takes all tensor memory");
};

template <int CIN, int COUT>
__global__ void __launch_bounds__(128)
k_conv_wgrad_tc(const __grid_constant__ CUtensorMap tm_in, const __grid_constant__ CUtensorMap tm_g,
                float *__restrict__ gW, int nx, int ny, int nz, int chunks_per_block) {
    using C = WgradTc<CIN, COUT>;
    using T = typename C::T;
    constexpr int TX = C::TX, TY = C::TY, NCC = T::NCC, NCO = T::NCO, NQ = C::NQ;
    extern __shared__ __align__(1024) unsigned char sm[];
    uint64_t *bars = reinterpret_cast<uint64_t *>(sm + 2 * T::kStage);  // full[2], empty[2]
    uint32_t *tslot = reinterpret_cast<uint32_t *>(bars + 4);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int dz = (int)blockIdx.y - 1;
    const int ntx = (nx + TX - 1) / TX, nty = (ny + TY - 1) / TY, ntz = (nz + kWgZ - 1) / kWgZ;
    const long long total = (long long)ntx * nty * ntz;
    const long long c0 = (long long)blockIdx.x * chunks_per_block;
    const int n = (int)max(0ll, min((long long)chunks_per_block, total - c0));
    const uint32_t bar0 = smem_u32(bars), sm0 = smem_u32(sm);

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                     "r"(C::kCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        for (int b = 0; b < 4; ++b) mbar_init(bar0 + 8 * b, 1);
        mbar_init_fence();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;
    bool ok = true;

    if (tid == 0 && n > 0) {
        auto load = [&](int i, int s) {  // chunk c0 + i into stage s
            const long long c = c0 + i;
            const int xt = (int)(c % ntx), yt = (int)((c / ntx) % nty), zt = (int)(c / ((long long)ntx * nty));
            const int x0 = xt * TX, y0 = yt * TY, z0 = zt * kWgZ;
            const uint32_t full = bar0 + 8 * s, st = sm0 + (uint32_t)(s * T::kStage);
            mbar_expect_tx(full, (uint32_t)(T::kBrick + T::kGrad));
            tma_load_5d(st, &tm_in, 0, z0 + dz, 0, x0 - 1, y0 - 1, full);
            tma_load_5d(st + (uint32_t)T::kBrick, &tm_g, 0, z0, 0, x0, y0, full);
        };
        constexpr uint32_t idesc = umma_idesc_bf16(128, COUT) | (1u << 15) | (1u << 16);  // A, B MN-major
        int loaded = 0, committed = 0;  // chunks whose copies / MMAs were issued
        load(0, 0);
        loaded = 1;
        for (int i = 0; i < n; ++i) {
            const int s = i & 1;
            ok &= mbar_wait_bounded(bar0 + 8 * s, (uint32_t)((i >> 1) & 1));
            if (!ok) break;
            tc_fence_after();
            const uint32_t brick = sm0 + (uint32_t)(s * T::kStage), grad = brick + (uint32_t)T::kBrick;
#pragma unroll 1
            for (int p = 0; p < TX * TY; ++p) {
                const int y = p / TX, x = p % TX;
                const uint64_t bd = umma_desc(grad + (uint32_t)(p * NCO * kWgZ * 16), 128, 256);
#pragma unroll
                for (int dy = 0; dy < 3; ++dy) {
#pragma unroll
                    for (int q = 0; q < NQ; ++q) {
                        const uint32_t a = brick + (uint32_t)((((y + dy) * T::XB + x) * NCC + 16 * q) * kWgZ * 16);
                        umma_bf16(tmem + (uint32_t)((dy * NQ + q) * COUT), umma_desc(a, 128, 256), bd, idesc,
                                  (i | p) != 0);
                    }
                }
            }
            umma_commit(bar0 + 8 * (2 + s));  // stage s is free once these MMAs are done
            committed = i + 1;
            if (i + 1 < n) {
                if (i >= 1) ok &= mbar_wait_bounded(bar0 + 8 * (2 + (s ^ 1)), (uint32_t)(((i - 1) >> 1) & 1));
                if (!ok) break;
                load(i + 1, s ^ 1);
                loaded = i + 2;
            }
        }
        if (ok) ok = mbar_wait_bounded(bar0 + 8 * (2 + ((n - 1) & 1)), (uint32_t)(((n - 1) >> 1) & 1));
        if (!ok) {
            atomicExch(&g_conv_timeout, 1);
            // the copies and MMAs still in flight get a second chance before the memory is released:
            // the last chunk loaded into / computed from each stage
            for (int s = 0; s < 2; ++s) {
                const int l = loaded - 1 - ((loaded - 1 - s) & 1), c = committed - 1 - ((committed - 1 - s) & 1);
                if (l >= 0) mbar_wait_bounded(bar0 + 8 * s, (uint32_t)((l >> 1) & 1));
                if (c >= 0) mbar_wait_bounded(bar0 + 8 * (2 + s), (uint32_t)((c >> 1) & 1));
            }
        }
    }
    ok = __syncthreads_and(ok);
    tc_fence_after();
    if (n > 0 && ok) {
        // TMEM lane m = 32 warp + lane is row m of each accumulator block
        const int m = 32 * warp + lane;
#pragma unroll
        for (int dy = 0; dy < 3; ++dy) {
#pragma unroll
            for (int q = 0; q < NQ; ++q) {
                const int j = 16 * q + m / 8;  // core-matrix row group: (dx, channel chunk)
                const bool valid = j < 3 * NCC;
                const int dx = j / NCC, ci = (j % NCC) * 8 + m % 8;
                const int t = (dz + 1) * 9 + dy * 3 + dx;
#pragma unroll
                for (int cb = 0; cb < COUT; cb += 16) {
                    float v[16];
                    tmem_ld16(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)((dy * NQ + q) * COUT + cb), v);
                    if (valid) {
                        float4 *dst = reinterpret_cast<float4 *>(gW + ((size_t)t * CIN + ci) * COUT + cb);
#pragma unroll
                        for (int e = 0; e < 4; ++e)
                            atomicAdd(dst + e, make_float4(v[4 * e], v[4 * e + 1], v[4 * e + 2], v[4 * e + 3]));
                    }
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(C::kCols) : "memory");
}

// gb[c] += sum_v g[v][c]
__global__ void k_bias_grad(const bf16 *__restrict__ g, float *__restrict__ gb, long long V, int C) {
    __shared__ float sh[64];
    for (int c = threadIdx.x; c < C; c += blockDim.x) sh[c] = 0.f;
    __syncthreads();
    float acc[64];
    for (int c = 0; c < C; ++c) acc[c] = 0.f;
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < V;
         v += (long long)gridDim.x * blockDim.x)
        for (int c = 0; c < C; ++c) acc[c] += __bfloat162float(g[v * C + c]);
    for (int c = 0; c < C; ++c) atomicAdd(&sh[c], acc[c]);
    __syncthreads();
    for (int c = threadIdx.x; c < C; c += blockDim.x) atomicAdd(&gb[c], sh[c]);
}

// Wt[t][co][ci] = W[26 - t][ci][co]
__global__ void k_flip_weights(const bf16 *__restrict__ W, bf16 *__restrict__ Wt, int cin, int cout) {
    const int n = 27 * cin * cout;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int t = i / (cin * cout), r = i % (cin * cout), co = r / cin, ci = r % cin;
        Wt[i] = W[((size_t)(26 - t) * cin + ci) * cout + co];
    }
}

// ---------------------------------------------------------------------------
// Dispatch
// ---------------------------------------------------------------------------
template <int CIN, int COUT, typename OutT>
static kv_status launch_fwd_t(int nx, int ny, int nz, const bf16 *in, const bf16 *W, const float *bias,
                              OutT *out, int relu, cudaStream_t s) {
    using C = ConvTc<CIN, COUT>;
    const size_t smem = C::kSmem;
    static int blocks_per_sm = 0;
    if (blocks_per_sm <= 0) {
        if (cudaFuncSetAttribute(k_conv_fwd<CIN, COUT, OutT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem) != cudaSuccess)
            return KV_ERR_CUDA;
        int b = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_conv_fwd<CIN, COUT, OutT>, kConvThreads, smem) !=
                cudaSuccess ||
            b <= 0)
            return KV_ERR_CUDA;
        // tensor memory: blocks on one SM must fit its 512 columns together
        blocks_per_sm = std::min(b, (int)(512 / C::kCols));
    }
    static int sms = 0;
    if (sms <= 0) {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0)
            sms = 148;
    }
    auto enc = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(tensor_map_encoder(nullptr));
    if (!enc || (reinterpret_cast<uintptr_t>(in) & 15) || (reinterpret_cast<uintptr_t>(W) & 15)) return KV_ERR_ARG;
    // 5D view of the channel-last input: (8 channels, x, y, z, channel chunk)
    CUtensorMap tm, tw;
    {
        cuuint64_t dims[5] = {8, (cuuint64_t)nx, (cuuint64_t)ny, (cuuint64_t)nz, (cuuint64_t)(CIN / 8)};
        cuuint64_t strides[4] = {(cuuint64_t)CIN * 2, (cuuint64_t)nx * CIN * 2, (cuuint64_t)nx * ny * CIN * 2, 16};
        cuuint32_t box[5] = {8, kTcBX, kTcBY, kTcBZ, CIN / 8};
        cuuint32_t es[5] = {1, 1, 1, 1, 1};
        if (enc(&tm, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, const_cast<bf16 *>(in), dims, strides, box, es,
                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return KV_ERR_CUDA;
    }
    // 4D view of the weights W[t][ci][co]: (8 co, ci, co chunk, tap), a box lands as
    // [tap][co chunk][ci][8], the MN-major core matrices of the B operand
    {
        cuuint64_t dims[4] = {8, (cuuint64_t)CIN, (cuuint64_t)(COUT / 8), 27};
        cuuint64_t strides[3] = {(cuuint64_t)COUT * 2, 16, (cuuint64_t)CIN * COUT * 2};
        cuuint32_t box[4] = {8, CIN, COUT / 8, 1};  // one tap per box
        cuuint32_t es[4] = {1, 1, 1, 1};
        if (enc(&tw, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<bf16 *>(W), dims, strides, box, es,
                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return KV_ERR_CUDA;
    }
    const long long ntiles = (long long)((nx + kTcX - 1) / kTcX) * ((ny + kTcY - 1) / kTcY) * ((nz + kTcZ - 1) / kTcZ);
    const int grid = (int)std::min<long long>(ntiles, (long long)sms * blocks_per_sm);
    k_conv_fwd<CIN, COUT, OutT><<<grid, kConvThreads, smem, s>>>(tm, tw, bias, out, nx, ny, nz, relu);
    return cudaGetLastError() == cudaSuccess ? KV_OK : KV_ERR_CUDA;
}

template <typename OutT>
static kv_status launch_fwd(int nx, int ny, int nz, int cin, int cout, const bf16 *in, const bf16 *W,
                            const float *bias, OutT *out, int relu, cudaStream_t s) {
#define KV_CONV_CASE(CI, CO)                                                                     \
    if (cin == CI && cout == CO) return launch_fwd_t<CI, CO, OutT>(nx, ny, nz, in, W, bias, out, relu, s);
    KV_CONV_CASE(16, 16) KV_CONV_CASE(16, 32) KV_CONV_CASE(16, 64) KV_CONV_CASE(32, 16)
    KV_CONV_CASE(32, 32) KV_CONV_CASE(32, 64) KV_CONV_CASE(64, 16) KV_CONV_CASE(64, 32)
    KV_CONV_CASE(64, 64)
#undef KV_CONV_CASE
    return KV_ERR_ARG;
}

template <int CIN, int COUT>
static kv_status launch_wgrad_t(int nx, int ny, int nz, const bf16 *in, const bf16 *g, float *gW,
                                cudaStream_t s) {
    using C = WgradTc<CIN, COUT>;
    const size_t smem = C::T::kSmem;
    static bool attr = false;
    if (!attr) {
        if (cudaFuncSetAttribute(k_conv_wgrad_tc<CIN, COUT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem) != cudaSuccess)
            return KV_ERR_CUDA;
        attr = true;
    }
    auto enc = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(tensor_map_encoder(nullptr));
    if (!enc || (reinterpret_cast<uintptr_t>(in) & 15) || (reinterpret_cast<uintptr_t>(g) & 15) ||
        (reinterpret_cast<uintptr_t>(gW) & 15))
        return KV_ERR_ARG;
    // 5D view (8 channels, z, channel chunk, x, y) of a channel-last tensor: a box
    // lands in shared memory as [y][x][chunk][z][8], the MN-major core matrices
    auto encode = [&](CUtensorMap *tm, const bf16 *base, int ch, int bx, int by) {
        cuuint64_t dims[5] = {8, (cuuint64_t)nz, (cuuint64_t)(ch / 8), (cuuint64_t)nx, (cuuint64_t)ny};
        cuuint64_t strides[4] = {(cuuint64_t)nx * ny * ch * 2, 16, (cuuint64_t)ch * 2, (cuuint64_t)nx * ch * 2};
        cuuint32_t box[5] = {8, (cuuint32_t)kWgZ, (cuuint32_t)(ch / 8), (cuuint32_t)bx, (cuuint32_t)by};
        cuuint32_t es[5] = {1, 1, 1, 1, 1};
        return enc(tm, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, const_cast<bf16 *>(base), dims, strides, box, es,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
    };
    CUtensorMap tm_in, tm_g;
    if (!encode(&tm_in, in, CIN, C::TX + 2, C::TY + 2) || !encode(&tm_g, g, COUT, C::TX, C::TY))
        return KV_ERR_CUDA;
    static int sms = 0;
    if (sms <= 0) {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0)
            sms = 148;
    }
    // one wave: a block per SM (the two stages fill its shared memory), a third of them per dz
    const long long total = (long long)((nx + C::TX - 1) / C::TX) * ((ny + C::TY - 1) / C::TY) *
                            ((nz + kWgZ - 1) / kWgZ);
    const long long per_dz = std::max(1, sms / 3);
    const int cpb = (int)((total + per_dz - 1) / per_dz);
    const int nblk = (int)((total + cpb - 1) / cpb);
    k_conv_wgrad_tc<CIN, COUT><<<dim3(nblk, 3), 128, smem, s>>>(tm_in, tm_g, gW, nx, ny, nz, cpb);
    return cudaGetLastError() == cudaSuccess ? KV_OK : KV_ERR_CUDA;
}

static kv_status launch_wgrad(int nx, int ny, int nz, int cin, int cout, const bf16 *in, const bf16 *g,
                              float *gW, cudaStream_t s) {
#define KV_WG_CASE(CI, CO) \
    if (cin == CI && cout == CO) return launch_wgrad_t<CI, CO>(nx, ny, nz, in, g, gW, s);
    KV_WG_CASE(16, 16) KV_WG_CASE(16, 32) KV_WG_CASE(16, 64) KV_WG_CASE(32, 16) KV_WG_CASE(32, 32)
    KV_WG_CASE(32, 64) KV_WG_CASE(64, 16) KV_WG_CASE(64, 32) KV_WG_CASE(64, 64)
#undef KV_WG_CASE
    return KV_ERR_ARG;
}

}  // namespace kv

// ---------------------------------------------------------------------------
// Layer-level C ABI (the U-Net runtime in kv_net.cu uses the same launchers)
// ---------------------------------------------------------------------------
namespace kv {
kv_status nn_conv_fwd(int nx, int ny, int nz, int cin, int cout, const void *x, const void *W,
                      const float *bias, void *out, int out_f32, int relu, cudaStream_t s) {
    if (out_f32)
        return launch_fwd<float>(nx, ny, nz, cin, cout, (const bf16 *)x, (const bf16 *)W, bias,
                                 (float *)out, relu, s);
    return launch_fwd<bf16>(nx, ny, nz, cin, cout, (const bf16 *)x, (const bf16 *)W, bias, (bf16 *)out,
                            relu, s);
}
kv_status nn_conv_wgrad(int nx, int ny, int nz, int cin, int cout, const void *x, const void *g,
                        float *gW, float *gb, cudaStream_t s) {
    kv_status st = launch_wgrad(nx, ny, nz, cin, cout, (const bf16 *)x, (const bf16 *)g, gW, s);
    if (st != KV_OK) return st;
    if (gb) {
        k_bias_grad<<<148 * 2, 256, 0, s>>>((const bf16 *)g, gb, (long long)nx * ny * nz, cout);
        if (cudaGetLastError() != cudaSuccess) return KV_ERR_CUDA;
    }
    return KV_OK;
}
// KV_ERR_TIMEOUT if a convolution's bounded wait gave up since the last call
// (the flag is cleared). Call after the stream has been synchronised.
kv_status nn_take_timeout() {
    int flag = 0;
    if (cudaMemcpyFromSymbol(&flag, g_conv_timeout, sizeof(int)) != cudaSuccess) return KV_ERR_CUDA;
    if (!flag) return KV_OK;
    const int zero = 0;
    cudaMemcpyToSymbol(g_conv_timeout, &zero, sizeof(int));
    return KV_ERR_TIMEOUT;
}
kv_status nn_flip(int cin, int cout, const void *W, void *Wt, cudaStream_t s) {
    k_flip_weights<<<64, 256, 0, s>>>((const bf16 *)W, (bf16 *)Wt, cin, cout);
    return cudaGetLastError() == cudaSuccess ? KV_OK : KV_ERR_CUDA;
}
}  // namespace kv

static bool nn_channels_ok(int c) { return c == 16 || c == 32 || c == 64; }

extern "C" {

kv_status kv_nn_conv3d_fwd(int nx, int ny, int nz, int cin, int cout, const void *x, const void *W,
                           const float *bias, void *out, int out_f32, int relu, void *stream) {
    if (nx < 1 || ny < 1 || nz < 1 || !nn_channels_ok(cin) || !nn_channels_ok(cout) || !x || !W || !out)
        return kv::set_error(nullptr, KV_ERR_ARG, "kv_nn_conv3d_fwd: invalid arguments");
    kv_status st = kv::nn_conv_fwd(nx, ny, nz, cin, cout, x, W, bias, out, out_f32, relu, (cudaStream_t)stream);
    if (st != KV_OK) return kv::set_error(nullptr, st, "kv_nn_conv3d_fwd: launch failed");
    return KV_OK;
}

kv_status kv_nn_conv3d_flip(int cin, int cout, const void *W, void *Wt, void *stream) {
    if (!nn_channels_ok(cin) || !nn_channels_ok(cout) || !W || !Wt)
        return kv::set_error(nullptr, KV_ERR_ARG, "kv_nn_conv3d_flip: invalid arguments");
    return kv::nn_flip(cin, cout, W, Wt, (cudaStream_t)stream);
}

kv_status kv_nn_conv3d_bwd_weight(int nx, int ny, int nz, int cin, int cout, const void *x,
                                  const void *g, float *gW, float *gb, void *stream) {
    if (nx < 1 || ny < 1 || nz < 1 || !nn_channels_ok(cin) || !nn_channels_ok(cout) || !x || !g || !gW)
        return kv::set_error(nullptr, KV_ERR_ARG, "kv_nn_conv3d_bwd_weight: invalid arguments");
    kv_status st = kv::nn_conv_wgrad(nx, ny, nz, cin, cout, x, g, gW, gb, (cudaStream_t)stream);
    if (st != KV_OK) return kv::set_error(nullptr, st, "kv_nn_conv3d_bwd_weight: launch failed");
    return KV_OK;
}

}  // extern "C"
