// kv_net.cu -- the learned warm start of the projection: a small 3D U-Net that
// maps the Poisson right-hand side b to an approximation of the potential phi,
// trained on (b, phi) pairs produced by the plain CG, and used as the initial
// guess of the CG (which still stops on the same true residual).
//
// Architecture (levels L, channels c[0..L-1]):
//   encoder level l: x_l -> conv+ReLU -> a_l -> conv+ReLU -> s_l; x_{l+1} = avgpool2(s_l)
//   decoder level l (l = L-2 .. 0): u_l = upsample2(d_{l+1}); q_l = conv+ReLU(u_l);
//                                   h_l = q_l + s_l; d_l = conv+ReLU(h_l); d_{L-1} = s_{L-1}
//   output: y = conv(d_0) (16 channels, channel 0 used)
// Input x_0 = b * s in channel 0 of 16 (s = 1/rms(b)); the target is phi * s / dx^2
// (A = -L scales as 1/dx^2), the loss the mean squared error over the grid.
// All convolutions are the BF16 tensor-core kernels of kv_nn.cu (FP32
// accumulation); weights are kept in FP32 (Adam) and copied to BF16.
#include <cuda_bf16.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <random>
#include <vector>

#include "kv_internal.cuh"

using bf16 = __nv_bfloat16;

namespace kv {
kv_status nn_conv_fwd(int nx, int ny, int nz, int cin, int cout, const void *x, const void *W,
                      const float *bias, void *out, int out_f32, int relu, cudaStream_t s);
kv_status nn_conv_wgrad(int nx, int ny, int nz, int cin, int cout, const void *x, const void *g,
                        float *gW, float *gb, cudaStream_t s);
kv_status nn_flip(int cin, int cout, const void *W, void *Wt, cudaStream_t s);
kv_status nn_take_timeout();
}  // namespace kv

namespace {

constexpr int kIO = 16;  // padded channels of the input and output tensors

struct Dims {
    int x, y, z;
    __host__ __device__ long long v() const { return (long long)x * y * z; }
};

struct Conv {
    int cin, cout, relu;
    long long woff, boff;  // offsets into the parameter vector (weights, then bias)
};

// ---- elementwise kernels (channel-last BF16) -------------------------------
// Channel-last tensors move in 16-byte vectors of 8 channels (C is 16, 32 or 64).
__device__ __forceinline__ void unpack8(const uint4 &q, float (&f)[8]) {
    const __nv_bfloat162 *h = reinterpret_cast<const __nv_bfloat162 *>(&q);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const float2 t = __bfloat1622float2(h[i]);
        f[2 * i] = t.x;
        f[2 * i + 1] = t.y;
    }
}
__device__ __forceinline__ uint4 pack8(const float (&f)[8]) {
    uint4 q;
    __nv_bfloat162 *h = reinterpret_cast<__nv_bfloat162 *>(&q);
#pragma unroll
    for (int i = 0; i < 4; ++i) h[i] = __floats2bfloat162_rn(f[2 * i], f[2 * i + 1]);
    return q;
}
#define KV_GRID_LOOP(e, n) \
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < (n); e += (long long)gridDim.x * blockDim.x)

__global__ void k_in_prep(const float *__restrict__ b, bf16 *__restrict__ x, long long V, float s) {
    KV_GRID_LOOP(v, V) {
        float f[8] = {b[v] * s, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        uint4 *o = reinterpret_cast<uint4 *>(x + v * kIO);
        o[0] = pack8(f);
        f[0] = 0.f;
#pragma unroll
        for (int c = 1; c < kIO / 8; ++c) o[c] = pack8(f);
    }
}

__global__ void k_sumsq(const float *__restrict__ a, long long V, double *out) {
    __shared__ double sh[33];
    double acc = 0.0;
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < V; v += (long long)gridDim.x * blockDim.x)
        acc += (double)a[v] * a[v];
    acc = block_sum_d(acc, sh);
    if (threadIdx.x == 0) atomicAdd(out, acc);
}

// loss = mean (y[v][0] - t[v] * ts)^2 ; g[v][c] = c == 0 ? 2 (y - t ts) / V : 0 (BF16)
__global__ void k_loss(const float *__restrict__ y, const float *__restrict__ t, float ts, bf16 *__restrict__ g,
                       long long V, double *loss) {
    __shared__ double sh[33];
    double acc = 0.0;
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < V; v += (long long)gridDim.x * blockDim.x) {
        const float d = y[v * kIO] - t[v] * ts;
        acc += (double)d * d;
        for (int c = 0; c < kIO; ++c) g[v * kIO + c] = __float2bfloat16_rn(c == 0 ? 2.f * d / (float)V : 0.f);
    }
    acc = block_sum_d(acc, sh);
    if (threadIdx.x == 0) atomicAdd(loss, acc / (double)V);
}

// Residual loss (option KV_LOSS_RESIDUAL): with e = y - t ts on interior nodes
// (0 on the outer layer, where the potential is fixed) and r = L^ e the
// unscaled 7-point Laplacian of e on interior nodes, loss = sum r^2 / V. Since
// A = -L^/dx^2 and the target is phi s/dx^2, r = -s (A phi_hat - b): the loss
// is the squared residual of the prediction, scaled to a unit-RMS b. Its
// gradient is dloss/dy = (2/V) L^ r on interior nodes (L^ is symmetric with the
// Dirichlet layer).
__device__ __forceinline__ bool interior_v(long long v, int nx, int ny, int nz, int &i, int &j, int &k) {
    i = (int)(v % nx);
    j = (int)((v / nx) % ny);
    k = (int)(v / ((long long)nx * ny));
    return i >= 1 && i <= nx - 2 && j >= 1 && j <= ny - 2 && k >= 1 && k <= nz - 2;
}
__global__ void k_res_err(const float *__restrict__ y, const float *__restrict__ t, float ts, float *__restrict__ e,
                          int nx, int ny, int nz) {
    const long long V = (long long)nx * ny * nz;
    KV_GRID_LOOP(v, V) {
        int i, j, k;
        e[v] = interior_v(v, nx, ny, nz, i, j, k) ? y[v * kIO] - t[v] * ts : 0.f;
    }
}
__device__ __forceinline__ float lap7(const float *__restrict__ a, long long v, long long sy, long long sz) {
    return ((a[v - 1] + a[v + 1]) + (a[v - sy] + a[v + sy])) + (a[v - sz] + a[v + sz]) - 6.f * a[v];
}
__global__ void k_res_lap(const float *__restrict__ e, float *__restrict__ r, int nx, int ny, int nz, double *loss) {
    __shared__ double sh[33];
    const long long V = (long long)nx * ny * nz, sy = nx, sz = (long long)nx * ny;
    double acc = 0.0;
    KV_GRID_LOOP(v, V) {
        int i, j, k;
        const float q = interior_v(v, nx, ny, nz, i, j, k) ? lap7(e, v, sy, sz) : 0.f;
        r[v] = q;
        acc += (double)q * q;
    }
    acc = block_sum_d(acc, sh);
    if (threadIdx.x == 0) atomicAdd(loss, acc / (double)V);
}
__global__ void k_res_grad(const float *__restrict__ r, bf16 *__restrict__ g, int nx, int ny, int nz) {
    const long long V = (long long)nx * ny * nz, sy = nx, sz = (long long)nx * ny;
    KV_GRID_LOOP(v, V) {
        int i, j, k;
        const float q = interior_v(v, nx, ny, nz, i, j, k) ? 2.f * lap7(r, v, sy, sz) / (float)V : 0.f;
        for (int c = 0; c < kIO; ++c) g[v * kIO + c] = __float2bfloat16_rn(c == 0 ? q : 0.f);
    }
}

__global__ void k_out_extract(const float *__restrict__ y, float *__restrict__ phi, long long V, float scale,
                              int nx, int ny, int nz) {
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < V; v += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(v % nx), j = (int)((v / nx) % ny), k = (int)(v / ((long long)nx * ny));
        const bool in = i >= 1 && i <= nx - 2 && j >= 1 && j <= ny - 2 && k >= 1 && k <= nz - 2;
        phi[v] = in ? y[v * kIO] * scale : 0.f;
    }
}

// avg pool 2x2x2 (ceil sizes; averages over the children that exist); one
// 8-channel vector per item
__global__ void k_pool(const bf16 *__restrict__ a, bf16 *__restrict__ o, Dims da, Dims dout, int C) {
    const int nv = C / 8;
    KV_GRID_LOOP(e, dout.v() * nv) {
        const int cv = (int)(e % nv);
        const long long v = e / nv;
        const int i = (int)(v % dout.x), j = (int)((v / dout.x) % dout.y), k = (int)(v / ((long long)dout.x * dout.y));
        float s[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        int cnt = 0;
        for (int dz = 0; dz < 2; ++dz)
            for (int dy = 0; dy < 2; ++dy)
                for (int dx = 0; dx < 2; ++dx) {
                    const int x = 2 * i + dx, y = 2 * j + dy, z = 2 * k + dz;
                    if (x < da.x && y < da.y && z < da.z) {
                        float f[8];
                        unpack8(reinterpret_cast<const uint4 *>(a + (((long long)z * da.y + y) * da.x + x) * C)[cv], f);
#pragma unroll
                        for (int q = 0; q < 8; ++q) s[q] += f[q];
                        ++cnt;
                    }
                }
#pragma unroll
        for (int q = 0; q < 8; ++q) s[q] /= (float)cnt;
        reinterpret_cast<uint4 *>(o)[e] = pack8(s);
    }
}

// gradient of the pool: ga[child] (+)= g[parent] / count(parent)
__global__ void k_pool_bwd(const bf16 *__restrict__ g, bf16 *__restrict__ ga, Dims da, Dims dg, int C, int accumulate) {
    const int nv = C / 8;
    KV_GRID_LOOP(e, da.v() * nv) {
        const int cv = (int)(e % nv);
        const long long v = e / nv;
        const int x = (int)(v % da.x), y = (int)((v / da.x) % da.y), z = (int)(v / ((long long)da.x * da.y));
        const int i = x / 2, j = y / 2, k = z / 2;
        const int cnt = (min(2 * i + 2, da.x) - 2 * i) * (min(2 * j + 2, da.y) - 2 * j) * (min(2 * k + 2, da.z) - 2 * k);
        float val[8];
        unpack8(reinterpret_cast<const uint4 *>(g + (((long long)k * dg.y + j) * dg.x + i) * C)[cv], val);
#pragma unroll
        for (int q = 0; q < 8; ++q) val[q] /= (float)cnt;
        if (accumulate) {
            float f[8];
            unpack8(reinterpret_cast<const uint4 *>(ga)[e], f);
#pragma unroll
            for (int q = 0; q < 8; ++q) val[q] += f[q];
        }
        reinterpret_cast<uint4 *>(ga)[e] = pack8(val);
    }
}

// nearest upsample: o[child] = a[parent]
__global__ void k_up(const bf16 *__restrict__ a, bf16 *__restrict__ o, Dims da, Dims dout, int C) {
    const int nv = C / 8;
    KV_GRID_LOOP(e, dout.v() * nv) {
        const int cv = (int)(e % nv);
        const long long v = e / nv;
        const int x = (int)(v % dout.x), y = (int)((v / dout.x) % dout.y), z = (int)(v / ((long long)dout.x * dout.y));
        reinterpret_cast<uint4 *>(o)[e] =
            reinterpret_cast<const uint4 *>(a + (((long long)(z / 2) * da.y + y / 2) * da.x + x / 2) * C)[cv];
    }
}

// gradient of the upsample: ga[parent] = sum over its children of g[child]
__global__ void k_up_bwd(const bf16 *__restrict__ g, bf16 *__restrict__ ga, Dims da, Dims dg, int C) {
    const int nv = C / 8;
    KV_GRID_LOOP(e, da.v() * nv) {
        const int cv = (int)(e % nv);
        const long long v = e / nv;
        const int i = (int)(v % da.x), j = (int)((v / da.x) % da.y), k = (int)(v / ((long long)da.x * da.y));
        float s[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        for (int dz = 0; dz < 2; ++dz)
            for (int dy = 0; dy < 2; ++dy)
                for (int dx = 0; dx < 2; ++dx) {
                    const int x = 2 * i + dx, y = 2 * j + dy, z = 2 * k + dz;
                    if (x < dg.x && y < dg.y && z < dg.z) {
                        float f[8];
                        unpack8(reinterpret_cast<const uint4 *>(g + (((long long)z * dg.y + y) * dg.x + x) * C)[cv], f);
#pragma unroll
                        for (int q = 0; q < 8; ++q) s[q] += f[q];
                    }
                }
        reinterpret_cast<uint4 *>(ga)[e] = pack8(s);
    }
}

// o = a + b over n elements (n a multiple of 8)
__global__ void k_add(const bf16 *__restrict__ a, const bf16 *__restrict__ b, bf16 *__restrict__ o, long long n) {
    KV_GRID_LOOP(e, n / 8) {
        float fa[8], fb[8];
        unpack8(reinterpret_cast<const uint4 *>(a)[e], fa);
        unpack8(reinterpret_cast<const uint4 *>(b)[e], fb);
#pragma unroll
        for (int q = 0; q < 8; ++q) fa[q] += fb[q];
        reinterpret_cast<uint4 *>(o)[e] = pack8(fa);
    }
}

// g *= (y > 0)  (gradient through a ReLU whose output is y)
__global__ void k_relu_bwd(bf16 *__restrict__ g, const bf16 *__restrict__ y, long long n) {
    KV_GRID_LOOP(e, n / 8) {
        float fg[8], fy[8];
        unpack8(reinterpret_cast<const uint4 *>(g)[e], fg);
        unpack8(reinterpret_cast<const uint4 *>(y)[e], fy);
#pragma unroll
        for (int q = 0; q < 8; ++q)
            if (!(fy[q] > 0.f)) fg[q] = 0.f;
        reinterpret_cast<uint4 *>(g)[e] = pack8(fg);
    }
}

__global__ void k_adam(float *__restrict__ w, const float *__restrict__ g, float *__restrict__ m,
                       float *__restrict__ v, long long n, float lr, float b1, float b2, float eps,
                       float c1, float c2) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        const float gg = g[e];
        const float mm = b1 * m[e] + (1.f - b1) * gg;
        const float vv = b2 * v[e] + (1.f - b2) * gg * gg;
        m[e] = mm;
        v[e] = vv;
        w[e] -= lr * (mm / c1) / (sqrtf(vv / c2) + eps);
    }
}

__global__ void k_to_bf16(const float *__restrict__ a, bf16 *__restrict__ o, long long n) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
        o[e] = __float2bfloat16_rn(a[e]);
}

constexpr int kEwBlocks = 148 * 8;

}  // namespace

struct kv_net {
    int L;
    int ch[8];
    std::vector<Conv> conv;  // order: encoder A0,B0,A1,B1,..., decoder U_{L-2},D_{L-2},...,U_0,D_0, final
    long long nparams;
    int loss_kind;                // KV_LOSS_MSE or KV_LOSS_RESIDUAL
    float *w32, *g32, *m, *v;     // parameters, gradients, Adam moments (FP32)
    bf16 *wbf, *wflip;            // BF16 weights and flipped-transposed copies
    long long adam_t;
    Dims maxd;
    // activations and gradients per level (allocated for maxd)
    std::vector<bf16 *> x, a, s, u, q, h, d;      // forward
    std::vector<bf16 *> gA, gB, gskip;            // gradient scratch per level (64 channels)
    bf16 *x0, *gout;
    float *yout;
    float *tmp_b, *tmp_phi;                        // dense float staging for the handle path
    double *red;                                   // reduction slots
    cudaStream_t stream;
    int own_stream;
    char err[512];
};

namespace {

Dims level_dims(const Dims &d0, int l) {
    Dims d = d0;
    for (int i = 0; i < l; ++i) {
        d.x = (d.x + 1) / 2;
        d.y = (d.y + 1) / 2;
        d.z = (d.z + 1) / 2;
    }
    return d;
}

kv_status nerr(kv_net *n, kv_status st, const char *msg) {
    if (n) snprintf(n->err, sizeof(n->err), "%s", msg);
    return kv::set_error(nullptr, st, "%s", msg);
}

template <typename P>
bool nalloc(P **p, size_t bytes) {
    return cudaMalloc((void **)p, std::max<size_t>(bytes, 16)) == cudaSuccess;
}

int conv_index_enc(int l, int which) { return 2 * l + which; }                  // which 0: A, 1: B
int conv_index_dec(const kv_net *n, int l, int which) {                          // which 0: U, 1: D
    return 2 * n->L + 2 * (n->L - 2 - l) + which;
}
int conv_index_final(const kv_net *n) { return 2 * n->L + 2 * (n->L - 1); }

const bf16 *wb(const kv_net *n, int ci) { return n->wbf + n->conv[ci].woff; }
const float *bias(const kv_net *n, int ci) { return n->w32 + n->conv[ci].boff; }

kv_status run_conv(kv_net *n, int ci, Dims d, const bf16 *in, void *out, int out_f32) {
    const Conv &c = n->conv[ci];
    return kv::nn_conv_fwd(d.x, d.y, d.z, c.cin, c.cout, in, wb(n, ci), bias(n, ci), out, out_f32, c.relu,
                           n->stream);
}

// Forward pass over grid d0; input x0 must be prepared. Output in n->yout.
kv_status forward(kv_net *n, Dims d0) {
    kv_status st;
    const int L = n->L;
    for (int l = 0; l < L; ++l) {
        const Dims d = level_dims(d0, l);
        if (l > 0) {
            k_pool<<<kEwBlocks, 256, 0, n->stream>>>(n->s[l - 1], n->x[l], level_dims(d0, l - 1), d, n->ch[l - 1]);
        }
        const bf16 *xin = (l == 0) ? n->x0 : n->x[l];
        if ((st = run_conv(n, conv_index_enc(l, 0), d, xin, n->a[l], 0)) != KV_OK) return st;
        if ((st = run_conv(n, conv_index_enc(l, 1), d, n->a[l], n->s[l], 0)) != KV_OK) return st;
    }
    for (int l = L - 2; l >= 0; --l) {
        const Dims d = level_dims(d0, l), dc = level_dims(d0, l + 1);
        const bf16 *below = (l == L - 2) ? n->s[L - 1] : n->d[l + 1];
        k_up<<<kEwBlocks, 256, 0, n->stream>>>(below, n->u[l], dc, d, n->ch[l + 1]);
        if ((st = run_conv(n, conv_index_dec(n, l, 0), d, n->u[l], n->q[l], 0)) != KV_OK) return st;
        k_add<<<kEwBlocks, 256, 0, n->stream>>>(n->q[l], n->s[l], n->h[l], d.v() * n->ch[l]);
        if ((st = run_conv(n, conv_index_dec(n, l, 1), d, n->h[l], n->d[l], 0)) != KV_OK) return st;
    }
    const bf16 *top = (L == 1) ? n->s[0] : n->d[0];
    if ((st = run_conv(n, conv_index_final(n), d0, top, n->yout, 1)) != KV_OK) return st;
    return cudaGetLastError() == cudaSuccess ? KV_OK : KV_ERR_CUDA;
}

// Backward of one conv layer: weight/bias gradients from its input and the
// gradient at its (pre-activation) output g; input gradient into gin (if any).
kv_status conv_bwd(kv_net *n, int ci, Dims d, const bf16 *in, const bf16 *g, bf16 *gin) {
    const Conv &c = n->conv[ci];
    kv_status st = kv::nn_conv_wgrad(d.x, d.y, d.z, c.cin, c.cout, in, g, n->g32 + c.woff,
                                     n->g32 + c.boff, n->stream);
    if (st != KV_OK || !gin) return st;
    return kv::nn_conv_fwd(d.x, d.y, d.z, c.cout, c.cin, g, n->wflip + c.woff, nullptr, gin, 0, 0, n->stream);
}

kv_status backward(kv_net *n, Dims d0) {
    kv_status st;
    const int L = n->L;
    // output layer: gradient n->gout (16 channels at level 0)
    const bf16 *top = (L == 1) ? n->s[0] : n->d[0];
    bf16 *g_top = n->gA[0];
    if ((st = conv_bwd(n, conv_index_final(n), d0, top, n->gout, g_top)) != KV_OK) return st;
    // decoder, level 0 upward; g of d_l arrives in gA[l]
    for (int l = 0; l <= L - 2; ++l) {
        const Dims d = level_dims(d0, l), dc = level_dims(d0, l + 1);
        const long long nl = d.v() * n->ch[l];
        k_relu_bwd<<<kEwBlocks, 256, 0, n->stream>>>(n->gA[l], n->d[l], nl);
        // conv D: input h_l, gradient to h -> gB[l]
        if ((st = conv_bwd(n, conv_index_dec(n, l, 1), d, n->h[l], n->gA[l], n->gB[l])) != KV_OK) return st;
        // h = q + s: skip gradient is gB[l]; q gradient is gB[l] too
        cudaMemcpyAsync(n->gskip[l], n->gB[l], nl * sizeof(bf16), cudaMemcpyDeviceToDevice, n->stream);
        k_relu_bwd<<<kEwBlocks, 256, 0, n->stream>>>(n->gB[l], n->q[l], nl);
        // conv U: input u_l (ch[l+1] channels) -> gradient to u into gA[l] (as ch[l+1] channels)
        if ((st = conv_bwd(n, conv_index_dec(n, l, 0), d, n->u[l], n->gB[l], n->gA[l])) != KV_OK) return st;
        // upsample gradient -> g of d_{l+1} (or s_{L-1}) in gA[l+1]
        k_up_bwd<<<kEwBlocks, 256, 0, n->stream>>>(n->gA[l], n->gA[l + 1], dc, d, n->ch[l + 1]);
    }
    // encoder, bottom upward: g of s_l in gA[l] (bottom: from the decoder; others: skip + pool grad)
    for (int l = L - 1; l >= 0; --l) {
        const Dims d = level_dims(d0, l);
        const long long nl = d.v() * n->ch[l];
        if (l < L - 1) {
            // gA[l] = gskip[l] + pool_bwd(g of x_{l+1}) ; g of x_{l+1} sits in gB[l+1]
            cudaMemcpyAsync(n->gA[l], n->gskip[l], nl * sizeof(bf16), cudaMemcpyDeviceToDevice, n->stream);
            k_pool_bwd<<<kEwBlocks, 256, 0, n->stream>>>(n->gB[l + 1], n->gA[l], d, level_dims(d0, l + 1),
                                                         n->ch[l], 1);
        } else if (L == 1) {
            // single level: gradient of s_0 is the output layer's input gradient (already in gA[0])
        }
        k_relu_bwd<<<kEwBlocks, 256, 0, n->stream>>>(n->gA[l], n->s[l], nl);
        if ((st = conv_bwd(n, conv_index_enc(l, 1), d, n->a[l], n->gA[l], n->gB[l])) != KV_OK) return st;
        k_relu_bwd<<<kEwBlocks, 256, 0, n->stream>>>(n->gB[l], n->a[l], nl);
        const bf16 *xin = (l == 0) ? n->x0 : n->x[l];
        // input gradient of conv A: needed above level 0 (into gB[l] after its use as the upstream g)
        bf16 *gin = (l == 0) ? nullptr : n->gA[l];  // reuse gA[l] (free now) for g of x_l
        if ((st = conv_bwd(n, conv_index_enc(l, 0), d, xin, n->gB[l], gin)) != KV_OK) return st;
        if (l > 0) cudaMemcpyAsync(n->gB[l], n->gA[l], d.v() * n->ch[l - 1] * sizeof(bf16),
                                   cudaMemcpyDeviceToDevice, n->stream);
    }
    return cudaGetLastError() == cudaSuccess ? KV_OK : KV_ERR_CUDA;
}

kv_status refresh_bf16(kv_net *n) {
    k_to_bf16<<<kEwBlocks, 256, 0, n->stream>>>(n->w32, n->wbf, n->nparams);
    for (size_t ci = 0; ci < n->conv.size(); ++ci) {
        const Conv &c = n->conv[ci];
        if (kv::nn_flip(c.cin, c.cout, n->wbf + c.woff, n->wflip + c.woff, n->stream) != KV_OK) return KV_ERR_CUDA;
    }
    return cudaGetLastError() == cudaSuccess ? KV_OK : KV_ERR_CUDA;
}

// s = 1 / rms(b) over the grid (b = 0 gives s = 1)
kv_status input_scale(kv_net *n, const float *b, long long V, float *s_out) {
    cudaMemsetAsync(n->red, 0, sizeof(double), n->stream);
    k_sumsq<<<kEwBlocks, 256, 0, n->stream>>>(b, V, n->red);
    double ss = 0.0;
    cudaMemcpyAsync(&ss, n->red, sizeof(double), cudaMemcpyDeviceToHost, n->stream);
    if (cudaStreamSynchronize(n->stream) != cudaSuccess) return KV_ERR_CUDA;
    *s_out = ss > 0.0 ? (float)(1.0 / sqrt(ss / (double)V)) : 1.f;
    return KV_OK;
}

bool fits(const kv_net *n, int nx, int ny, int nz) {
    return nx >= 2 && ny >= 2 && nz >= 2 && nx <= n->maxd.x && ny <= n->maxd.y && nz <= n->maxd.z;
}

}  // namespace

extern "C" kv_status kv_net_destroy(kv_net *n);

extern "C" {

kv_status kv_net_create(kv_net **out, int levels, const int *channels, int max_nx, int max_ny,
                        int max_nz, void *stream) {
    if (!out || levels < 1 || levels > 6 || !channels || max_nx < 2 || max_ny < 2 || max_nz < 2)
        return kv::set_error(nullptr, KV_ERR_ARG, "kv_net_create: invalid arguments");
    for (int l = 0; l < levels; ++l)
        if (channels[l] != 16 && channels[l] != 32 && channels[l] != 64)
            return kv::set_error(nullptr, KV_ERR_ARG, "kv_net_create: channels must be 16, 32 or 64");
    kv_net *n = new kv_net();
    memset(n->err, 0, sizeof(n->err));
    n->L = levels;
    for (int l = 0; l < levels; ++l) n->ch[l] = channels[l];
    // parameter layout
    long long off = 0;
    auto add = [&](int cin, int cout, int relu) {
        Conv c{cin, cout, relu, off, off + 27LL * cin * cout};
        off += 27LL * cin * cout + cout;
        off = (off + 7) / 8 * 8;  // keep every weight block 16-byte aligned in BF16
        n->conv.push_back(c);
    };
    for (int l = 0; l < levels; ++l) {
        add(l == 0 ? kIO : channels[l - 1], channels[l], 1);
        add(channels[l], channels[l], 1);
    }
    for (int l = levels - 2; l >= 0; --l) {
        add(channels[l + 1], channels[l], 1);
        add(channels[l], channels[l], 1);
    }
    add(channels[0], kIO, 0);
    n->nparams = off;
    n->adam_t = 0;
    n->loss_kind = KV_LOSS_MSE;
    n->maxd = {max_nx, max_ny, max_nz};
    if (stream) {
        n->stream = (cudaStream_t)stream;
        n->own_stream = 0;
    } else {
        cudaStreamCreateWithFlags(&n->stream, cudaStreamNonBlocking);
        n->own_stream = 1;
    }
    bool ok = nalloc(&n->w32, off * 4) && nalloc(&n->g32, off * 4) && nalloc(&n->m, off * 4) &&
              nalloc(&n->v, off * 4) && nalloc(&n->wbf, off * 2) && nalloc(&n->wflip, off * 2) &&
              nalloc(&n->red, 64);
    const Dims d0 = n->maxd;
    const long long V0 = d0.v();
    ok = ok && nalloc(&n->x0, V0 * kIO * 2) && nalloc(&n->gout, V0 * kIO * 2) && nalloc(&n->yout, V0 * kIO * 4) &&
         nalloc(&n->tmp_b, V0 * 4) && nalloc(&n->tmp_phi, V0 * 4);
    n->x.assign(levels, nullptr);
    n->a = n->s = n->u = n->q = n->h = n->d = n->gA = n->gB = n->gskip = n->x;
    for (int l = 0; l < levels && ok; ++l) {
        const long long V = level_dims(d0, l).v();
        const int c = channels[l];
        ok = ok && nalloc(&n->a[l], V * c * 2) && nalloc(&n->s[l], V * c * 2) && nalloc(&n->gA[l], V * 64 * 2) &&
             nalloc(&n->gB[l], V * 64 * 2) && nalloc(&n->gskip[l], V * c * 2);
        if (l > 0) ok = ok && nalloc(&n->x[l], V * channels[l - 1] * 2);
        if (l < levels - 1)
            ok = ok && nalloc(&n->u[l], V * channels[l + 1] * 2) && nalloc(&n->q[l], V * c * 2) &&
                 nalloc(&n->h[l], V * c * 2) && nalloc(&n->d[l], V * c * 2);
    }
    if (!ok) {
        kv_net_destroy(n);
        return kv::set_error(nullptr, KV_ERR_OOM, "kv_net_create: device allocation failed");
    }
    cudaMemsetAsync(n->w32, 0, off * 4, n->stream);
    cudaMemsetAsync(n->m, 0, off * 4, n->stream);
    cudaMemsetAsync(n->v, 0, off * 4, n->stream);
    *out = n;
    return KV_OK;
}

kv_status kv_net_destroy(kv_net *n) {
    if (!n) return KV_OK;
    if (n->stream) cudaStreamSynchronize(n->stream);
    void *ptrs[] = {n->w32, n->g32, n->m, n->v, n->wbf, n->wflip, n->red, n->x0, n->gout, n->yout, n->tmp_b, n->tmp_phi};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    for (auto *vec : {&n->x, &n->a, &n->s, &n->u, &n->q, &n->h, &n->d, &n->gA, &n->gB, &n->gskip})
        for (bf16 *p : *vec)
            if (p) cudaFree(p);
    if (n->own_stream && n->stream) cudaStreamDestroy(n->stream);
    delete n;
    return KV_OK;
}

long long kv_net_num_params(kv_net *n) { return n ? n->nparams : 0; }

kv_status kv_net_set_loss(kv_net *n, int kind) {
    if (!n || (kind != KV_LOSS_MSE && kind != KV_LOSS_RESIDUAL))
        return nerr(n, KV_ERR_ARG, "kv_net_set_loss: unknown loss");
    n->loss_kind = kind;
    return KV_OK;
}

kv_status kv_net_init(kv_net *n, unsigned long long seed) {
    if (!n) return KV_ERR_ARG;
    std::vector<float> w(n->nparams, 0.f);
    std::mt19937_64 rng(seed);
    for (size_t ci = 0; ci < n->conv.size(); ++ci) {
        const Conv &c = n->conv[ci];
        const bool last = ci + 1 == n->conv.size();
        const int fan_in = 27 * (ci == 0 ? 1 : c.cin);
        std::normal_distribution<float> nd(0.f, (last ? 0.1f : 1.f) * sqrtf(2.f / (float)fan_in));
        for (long long e = 0; e < 27LL * c.cin * c.cout; ++e) {
            const int ciin = (int)((e / c.cout) % c.cin);
            w[c.woff + e] = (ci == 0 && ciin != 0) ? 0.f : nd(rng);  // padded input channels stay 0
        }
        for (int co = 0; co < c.cout; ++co) w[c.boff + co] = 0.f;
    }
    cudaError_t e = cudaMemcpyAsync(n->w32, w.data(), n->nparams * 4, cudaMemcpyHostToDevice, n->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(n->m, 0, n->nparams * 4, n->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(n->v, 0, n->nparams * 4, n->stream);
    n->adam_t = 0;
    kv_status st = refresh_bf16(n);
    if (e == cudaSuccess) e = cudaStreamSynchronize(n->stream);
    return (e == cudaSuccess && st == KV_OK) ? KV_OK : nerr(n, KV_ERR_CUDA, "kv_net_init failed");
}

kv_status kv_net_get_params(kv_net *n, float *host) {
    if (!n || !host) return KV_ERR_ARG;
    cudaError_t e = cudaMemcpyAsync(host, n->w32, n->nparams * 4, cudaMemcpyDeviceToHost, n->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(n->stream);
    return e == cudaSuccess ? KV_OK : nerr(n, KV_ERR_CUDA, "kv_net_get_params failed");
}

kv_status kv_net_set_params(kv_net *n, const float *host) {
    if (!n || !host) return KV_ERR_ARG;
    cudaError_t e = cudaMemcpyAsync(n->w32, host, n->nparams * 4, cudaMemcpyHostToDevice, n->stream);
    kv_status st = refresh_bf16(n);
    if (e == cudaSuccess) e = cudaStreamSynchronize(n->stream);
    return (e == cudaSuccess && st == KV_OK) ? KV_OK : nerr(n, KV_ERR_CUDA, "kv_net_set_params failed");
}

kv_status kv_net_train_step(kv_net *n, int nx, int ny, int nz, double dx, const float *b, const float *phi,
                            double lr, double *loss) {
    if (!n || !b || !phi || !(dx > 0.0) || !fits(n, nx, ny, nz))
        return nerr(n, KV_ERR_ARG, "kv_net_train_step: invalid arguments or grid larger than the net's");
    const Dims d0 = {nx, ny, nz};
    const long long V = d0.v();
    float s;
    if (input_scale(n, b, V, &s) != KV_OK) return nerr(n, KV_ERR_CUDA, "kv_net_train_step: scale failed");
    k_in_prep<<<kEwBlocks, 256, 0, n->stream>>>(b, n->x0, V, s);
    kv_status st = forward(n, d0);
    if (st != KV_OK) return nerr(n, st, "kv_net_train_step: forward failed");
    cudaMemsetAsync(n->red, 0, sizeof(double), n->stream);
    if (n->loss_kind == KV_LOSS_RESIDUAL) {
        // tmp_phi holds e, tmp_b holds r (the handle path's staging is idle here)
        k_res_err<<<kEwBlocks, 256, 0, n->stream>>>(n->yout, phi, (float)(s / (dx * dx)), n->tmp_phi, nx, ny, nz);
        k_res_lap<<<kEwBlocks, 256, 0, n->stream>>>(n->tmp_phi, n->tmp_b, nx, ny, nz, n->red);
        k_res_grad<<<kEwBlocks, 256, 0, n->stream>>>(n->tmp_b, n->gout, nx, ny, nz);
    } else {
        k_loss<<<kEwBlocks, 256, 0, n->stream>>>(n->yout, phi, (float)(s / (dx * dx)), n->gout, V, n->red);
    }
    cudaMemsetAsync(n->g32, 0, n->nparams * 4, n->stream);
    if ((st = backward(n, d0)) != KV_OK) return nerr(n, st, "kv_net_train_step: backward failed");
    n->adam_t += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    k_adam<<<kEwBlocks, 256, 0, n->stream>>>(n->w32, n->g32, n->m, n->v, n->nparams, (float)lr, b1, b2, 1e-8f,
                                              1.f - powf(b1, (float)n->adam_t), 1.f - powf(b2, (float)n->adam_t));
    if ((st = refresh_bf16(n)) != KV_OK) return nerr(n, st, "kv_net_train_step: weight copy failed");
    double l = 0.0;
    cudaMemcpyAsync(&l, n->red, sizeof(double), cudaMemcpyDeviceToHost, n->stream);
    if (cudaStreamSynchronize(n->stream) != cudaSuccess) return nerr(n, KV_ERR_CUDA, "kv_net_train_step: CUDA error");
    if ((st = kv::nn_take_timeout()) != KV_OK) return nerr(n, st, "kv_net_train_step: a convolution's bounded wait timed out");
    if (loss) *loss = l;
    return KV_OK;
}

kv_status kv_net_predict(kv_net *n, int nx, int ny, int nz, double dx, const float *b, float *phi) {
    if (!n || !b || !phi || !(dx > 0.0) || !fits(n, nx, ny, nz))
        return nerr(n, KV_ERR_ARG, "kv_net_predict: invalid arguments or grid larger than the net's");
    const Dims d0 = {nx, ny, nz};
    const long long V = d0.v();
    float s;
    if (input_scale(n, b, V, &s) != KV_OK) return nerr(n, KV_ERR_CUDA, "kv_net_predict: scale failed");
    k_in_prep<<<kEwBlocks, 256, 0, n->stream>>>(b, n->x0, V, s);
    kv_status st = forward(n, d0);
    if (st != KV_OK) return nerr(n, st, "kv_net_predict: forward failed");
    k_out_extract<<<kEwBlocks, 256, 0, n->stream>>>(n->yout, phi, V, (float)(dx * dx / s), nx, ny, nz);
    if (cudaStreamSynchronize(n->stream) != cudaSuccess) return nerr(n, KV_ERR_CUDA, "kv_net_predict: CUDA error");
    if ((st = kv::nn_take_timeout()) != KV_OK) return nerr(n, st, "kv_net_predict: a convolution's bounded wait timed out");
    return KV_OK;
}

// For the handle path (kv_cg.cu): dense staging buffers of the net.
float *kv_net_stage_b(kv_net *n) { return n->tmp_b; }
float *kv_net_stage_phi(kv_net *n) { return n->tmp_phi; }
cudaStream_t kv_net_stream(kv_net *n) { return n->stream; }
int kv_net_fits(kv_net *n, int nx, int ny, int nz) { return fits(n, nx, ny, nz); }

}  // extern "C"
