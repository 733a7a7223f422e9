// kv_nn.cu -- tensor-core building blocks of the learned warm start: 3x3x3
// convolution forward, input gradient and weight gradient as implicit GEMMs on
// BF16 operands with FP32 accumulation (WMMA 16x16x16 tiles), plus the
// channel-last elementwise pieces of a U-Net (pooling, upsampling, skips,
// ReLU gradient) and the Adam update.
//
// Tensors are channel-last [z][y][x][C] BF16 with C in {16, 32, 64}. Weights
// W[t][ci][co], tap t = (dz+1)*9 + (dy+1)*3 + (dx+1), zero padding of one voxel:
//   out[v][co] = bias[co] + sum_{t,ci} in[v + d(t)][ci] W[t][ci][co].
// The input gradient is the same convolution with Wt[t][co][ci] = W[26-t][ci][co].
#include <cuda_bf16.h>
#include <mma.h>

#include <algorithm>

#include "kv_internal.cuh"

using bf16 = __nv_bfloat16;
namespace wm = nvcuda::wmma;

namespace kv {

// ---------------------------------------------------------------------------
// Forward (and input-gradient) convolution
// ---------------------------------------------------------------------------
constexpr int kCvTX = 16, kCvTY = 4, kCvTZ = 2;                  // 128 voxels per block
constexpr int kCvBX = kCvTX + 2, kCvBY = kCvTY + 2, kCvBZ = kCvTZ + 2;
constexpr int kCvBrick = kCvBX * kCvBY * kCvBZ;                   // 432 voxels with halo

template <int CIN, int COUT>
constexpr size_t conv_fwd_smem() {
    return (size_t)kCvBrick * CIN * 2 + (size_t)CIN * COUT * 2;
}

template <typename OutT>
__device__ __forceinline__ OutT to_out(float v);
template <>
__device__ __forceinline__ float to_out<float>(float v) { return v; }
template <>
__device__ __forceinline__ bf16 to_out<bf16>(float v) { return __float2bfloat16_rn(v); }

template <int CIN, int COUT, typename OutT>
__global__ void __launch_bounds__(256)
k_conv_fwd(const bf16 *__restrict__ in, const bf16 *__restrict__ W, const float *__restrict__ bias,
           OutT *__restrict__ out, int nx, int ny, int nz, int relu) {
    extern __shared__ __align__(128) unsigned char sm[];
    bf16 *brick = reinterpret_cast<bf16 *>(sm);
    bf16 *wt = brick + kCvBrick * CIN;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int x0 = blockIdx.x * kCvTX, y0 = blockIdx.y * kCvTY, z0 = blockIdx.z * kCvTZ;

    constexpr int VPV = CIN / 8;  // 16-byte vectors per voxel
    for (int i = tid; i < kCvBrick * VPV; i += 256) {
        const int vox = i / VPV, part = i % VPV;
        const int bx = vox % kCvBX, by = (vox / kCvBX) % kCvBY, bz = vox / (kCvBX * kCvBY);
        const int gx = x0 - 1 + bx, gy = y0 - 1 + by, gz = z0 - 1 + bz;
        uint4 v = make_uint4(0, 0, 0, 0);
        if (gx >= 0 && gx < nx && gy >= 0 && gy < ny && gz >= 0 && gz < nz)
            v = *reinterpret_cast<const uint4 *>(in + (((size_t)gz * ny + gy) * nx + gx) * CIN + part * 8);
        *reinterpret_cast<uint4 *>(brick + (size_t)vox * CIN + part * 8) = v;
    }
    const int wy = warp % kCvTY, wz = warp / kCvTY;  // this warp's row of 16 voxels
    wm::fragment<wm::accumulator, 16, 16, 16, float> acc[COUT / 16];
#pragma unroll
    for (int j = 0; j < COUT / 16; ++j) wm::fill_fragment(acc[j], 0.f);
    for (int t = 0; t < 27; ++t) {
        __syncthreads();  // previous tap's weights consumed (and the brick complete)
        for (int i = tid; i < CIN * COUT / 8; i += 256)
            *reinterpret_cast<uint4 *>(wt + i * 8) =
                *reinterpret_cast<const uint4 *>(W + (size_t)t * CIN * COUT + i * 8);
        __syncthreads();
        const int dx = t % 3, dy = (t / 3) % 3, dz = t / 9;
        const bf16 *arow = brick + ((size_t)((wz + dz) * kCvBY + (wy + dy)) * kCvBX + dx) * CIN;
#pragma unroll
        for (int kc = 0; kc < CIN / 16; ++kc) {
            wm::fragment<wm::matrix_a, 16, 16, 16, bf16, wm::row_major> a;
            wm::load_matrix_sync(a, arow + kc * 16, CIN);
#pragma unroll
            for (int j = 0; j < COUT / 16; ++j) {
                wm::fragment<wm::matrix_b, 16, 16, 16, bf16, wm::row_major> b;
                wm::load_matrix_sync(b, wt + kc * 16 * COUT + j * 16, COUT);
                wm::mma_sync(acc[j], a, b, acc[j]);
            }
        }
    }
    __syncthreads();  // the brick is no longer read: reuse it for the output tiles
    float *os = reinterpret_cast<float *>(sm) + (size_t)warp * 16 * COUT;
#pragma unroll
    for (int j = 0; j < COUT / 16; ++j) wm::store_matrix_sync(os + j * 16, acc[j], COUT, wm::mem_row_major);
    __syncwarp();
    const int gy = y0 + wy, gz = z0 + wz;
    if (gy < ny && gz < nz) {
        for (int e = lane; e < 16 * COUT; e += 32) {
            const int vx = e / COUT, co = e % COUT;
            const int gx = x0 + vx;
            if (gx >= nx) continue;
            float v = os[e] + (bias ? bias[co] : 0.f);
            if (relu) v = fmaxf(v, 0.f);
            out[(((size_t)gz * ny + gy) * nx + gx) * COUT + co] = to_out<OutT>(v);
        }
    }
}

// ---------------------------------------------------------------------------
// Weight gradient: gW[t][ci][co] += sum_v in[v + d(t)][ci] g[v][co] (FP32),
// gb[co] += sum_v g[v][co]. Block (chunk, tap) sweeps its rows of 16 voxels.
// ---------------------------------------------------------------------------
constexpr int kWgRows = 8;  // rows of 16 voxels staged per step

template <int CIN, int COUT>
constexpr size_t conv_wgrad_smem() {
    return (size_t)kWgRows * 16 * (CIN + COUT) * 2 + 8 * 16 * 16 * 4;
}

template <int CIN, int COUT>
__global__ void __launch_bounds__(256)
k_conv_wgrad(const bf16 *__restrict__ in, const bf16 *__restrict__ g, float *__restrict__ gW,
             int nx, int ny, int nz, int rows_per_block) {
    extern __shared__ __align__(128) unsigned char sm[];
    bf16 *As = reinterpret_cast<bf16 *>(sm);             // [rows][16 voxels][CIN]
    bf16 *Bs = As + kWgRows * 16 * CIN;                   // [rows][16 voxels][COUT]
    float *tmp = reinterpret_cast<float *>(Bs + kWgRows * 16 * COUT);  // 8 warps x 16x16
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int t = blockIdx.y;
    const int ddx = t % 3 - 1, ddy = (t / 3) % 3 - 1, ddz = t / 9 - 1;
    const int xtiles = (nx + 15) / 16;
    const long long nrows = (long long)xtiles * ny * nz;
    const long long r0 = (long long)blockIdx.x * rows_per_block;
    const long long r1 = min(r0 + rows_per_block, nrows);
    constexpr int NCI = CIN / 16, NCO = COUT / 16, NP = NCI * NCO;
    constexpr int PPW = (NP + 7) / 8;  // (ci-tile, co-tile) pairs per warp
    wm::fragment<wm::accumulator, 16, 16, 16, float> acc[PPW];
#pragma unroll
    for (int q = 0; q < PPW; ++q) wm::fill_fragment(acc[q], 0.f);
    for (long long rb = r0; rb < r1; rb += kWgRows) {
        __syncthreads();
        constexpr int VA = CIN / 8, VB = COUT / 8;
        for (int i = tid; i < kWgRows * 16 * (VA + VB); i += 256) {
            const int isB = i >= kWgRows * 16 * VA;
            const int ii = isB ? i - kWgRows * 16 * VA : i;
            const int V8 = isB ? VB : VA;
            const int rr = ii / (16 * V8), vx = (ii / V8) % 16, part = ii % V8;
            const long long row = rb + rr;
            uint4 val = make_uint4(0, 0, 0, 0);
            if (row < r1) {
                const int xt = (int)(row % xtiles);
                const long long yz = row / xtiles;
                const int y = (int)(yz % ny), z = (int)(yz / ny);
                const int x = xt * 16 + vx;
                if (x < nx) {
                    if (isB) {
                        val = *reinterpret_cast<const uint4 *>(g + (((size_t)z * ny + y) * nx + x) * COUT + part * 8);
                    } else {
                        const int xx = x + ddx, yy = y + ddy, zz = z + ddz;
                        if (xx >= 0 && xx < nx && yy >= 0 && yy < ny && zz >= 0 && zz < nz)
                            val = *reinterpret_cast<const uint4 *>(
                                in + (((size_t)zz * ny + yy) * nx + xx) * CIN + part * 8);
                    }
                }
            }
            bf16 *dst = isB ? Bs + ((size_t)rr * 16 + vx) * COUT + part * 8
                            : As + ((size_t)rr * 16 + vx) * CIN + part * 8;
            *reinterpret_cast<uint4 *>(dst) = val;
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < PPW; ++q) {
            const int pidx = warp + 8 * q;
            if (pidx >= NP) break;
            const int cit = pidx / NCO, cot = pidx % NCO;
            for (int rr = 0; rr < kWgRows; ++rr) {
                wm::fragment<wm::matrix_a, 16, 16, 16, bf16, wm::col_major> a;  // (ci, voxel)
                wm::fragment<wm::matrix_b, 16, 16, 16, bf16, wm::row_major> b;  // (voxel, co)
                wm::load_matrix_sync(a, As + (size_t)rr * 16 * CIN + cit * 16, CIN);
                wm::load_matrix_sync(b, Bs + (size_t)rr * 16 * COUT + cot * 16, COUT);
                wm::mma_sync(acc[q], a, b, acc[q]);
            }
        }
    }
    float *mine = tmp + warp * 256;
#pragma unroll
    for (int q = 0; q < PPW; ++q) {
        const int pidx = warp + 8 * q;
        if (pidx >= NP) break;
        const int cit = pidx / NCO, cot = pidx % NCO;
        wm::store_matrix_sync(mine, acc[q], 16, wm::mem_row_major);
        __syncwarp();
        for (int e = lane; e < 256; e += 32) {
            const int ci = cit * 16 + e / 16, co = cot * 16 + e % 16;
            atomicAdd(gW + ((size_t)t * CIN + ci) * COUT + co, mine[e]);
        }
        __syncwarp();
    }
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
    const size_t smem = std::max(conv_fwd_smem<CIN, COUT>(), (size_t)8 * 16 * COUT * 4);
    static bool attr = false;
    if (!attr) {
        if (cudaFuncSetAttribute(k_conv_fwd<CIN, COUT, OutT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem) != cudaSuccess)
            return KV_ERR_CUDA;
        attr = true;
    }
    dim3 grid((nx + kCvTX - 1) / kCvTX, (ny + kCvTY - 1) / kCvTY, (nz + kCvTZ - 1) / kCvTZ);
    k_conv_fwd<CIN, COUT, OutT><<<grid, 256, smem, s>>>(in, W, bias, out, nx, ny, nz, relu);
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
    const size_t smem = conv_wgrad_smem<CIN, COUT>();
    static bool attr = false;
    if (!attr) {
        if (cudaFuncSetAttribute(k_conv_wgrad<CIN, COUT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem) != cudaSuccess)
            return KV_ERR_CUDA;
        attr = true;
    }
    const long long nrows = (long long)((nx + 15) / 16) * ny * nz;
    const int chunks = (int)std::min<long long>(64, std::max<long long>(1, nrows / kWgRows));
    int rows_per_block = (int)((nrows + chunks - 1) / chunks);
    rows_per_block = (rows_per_block + kWgRows - 1) / kWgRows * kWgRows;
    const int nblk = (int)((nrows + rows_per_block - 1) / rows_per_block);
    k_conv_wgrad<CIN, COUT><<<dim3(nblk, 27), 256, smem, s>>>(in, g, gW, nx, ny, nz, rows_per_block);
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
