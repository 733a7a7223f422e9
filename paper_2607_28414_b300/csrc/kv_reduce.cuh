// kv_reduce.cuh -- reductions shared by the projection kernels: float-float
// accumulators (FP64-class inner products on the FP32 pipes) and the
// deterministic last-block finisher.
#pragma once

#include "kv_internal.cuh"

namespace kv {

// ---------------------------------------------------------------------------
// Accumulators: float-float for float vectors, double for double vectors.
// ---------------------------------------------------------------------------
struct AccFF {
    float hi = 0.f, lo = 0.f;
    // acc += x * y with the product and the sum formed exactly (TwoProd by FMA,
    // TwoSum), then renormalised.
    __device__ __forceinline__ void add_prod(float x, float y) {
        const float p = __fmul_rn(x, y);
        const float pe = __fmaf_rn(x, y, -p);
        const float s = __fadd_rn(hi, p);
        const float bb = __fsub_rn(s, hi);
        const float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(p, bb));
        const float t = __fadd_rn(__fadd_rn(e, pe), lo);
        hi = __fadd_rn(s, t);
        lo = __fsub_rn(t, __fsub_rn(hi, s));
    }
    // acc += v with the sum formed exactly (TwoSum), then renormalised.
    __device__ __forceinline__ void add(float v) {
        const float s = __fadd_rn(hi, v);
        const float bb = __fsub_rn(s, hi);
        const float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(v, bb));
        const float t = __fadd_rn(e, lo);
        hi = __fadd_rn(s, t);
        lo = __fsub_rn(t, __fsub_rn(hi, s));
    }
    __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};
struct AccD {
    double v = 0.0;
    __device__ __forceinline__ void add_prod(double x, double y) { v = __fma_rn(x, y, v); }
    __device__ __forceinline__ double value() const { return v; }
};
template <typename T> struct AccOf;
template <> struct AccOf<float> { using type = AccFF; };
template <> struct AccOf<double> { using type = AccD; };

// Last-block finisher: returns true in the block that finished last; sums[q]
// then holds the deterministic grand total of partial slot q.
template <int NQ>
__device__ __forceinline__ bool last_block_sums(const CgParams &p, const double (&v)[NQ],
                                                double (&sums)[NQ]) {
    __shared__ double sh[33];
    __shared__ int s_last;
    const int bid = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
    const int tid = threadIdx.x;
    for (int q = 0; q < NQ; ++q) {
        double t = block_sum_d(v[q], sh);
        if (tid == 0) p.partials[(size_t)q * p.nblocks + bid] = t;
    }
    __threadfence();
    __syncthreads();
    if (tid == 0) {
        unsigned long long t =
            atomicAdd(reinterpret_cast<unsigned long long *>(&p.ctrl[kCgTicket]), 1ull);
        s_last = (t == (unsigned long long)(p.nblocks - 1));
    }
    __syncthreads();
    if (!s_last) return false;
    __threadfence();
    for (int q = 0; q < NQ; ++q) {
        double acc = 0.0;
        for (int b = tid; b < p.nblocks; b += blockDim.x)
            acc += __ldcg(&p.partials[(size_t)q * p.nblocks + b]);
        sums[q] = block_sum_d(acc, sh);
    }
    if (tid == 0) p.ctrl[kCgTicket] = 0;
    return true;
}

__device__ __forceinline__ void ff_add(float &hi, float &lo, float bh, float bl) {
    const float s = __fadd_rn(hi, bh);
    const float bb = __fsub_rn(s, hi);
    const float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(bh, bb));
    const float t = __fadd_rn(__fadd_rn(e, lo), bl);
    hi = __fadd_rn(s, t);
    lo = __fsub_rn(t, __fsub_rn(hi, s));
}

// Block total of a float-float accumulator, as a double in thread 0.
__device__ __forceinline__ double block_total_ff(AccFF a) {
    __shared__ float sh_hi[32], sh_lo[32];
    float hi = a.hi, lo = a.lo;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float h2 = __shfl_xor_sync(0xffffffffu, hi, o);
        const float l2 = __shfl_xor_sync(0xffffffffu, lo, o);
        ff_add(hi, lo, h2, l2);
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (lane == 0) {
        sh_hi[warp] = hi;
        sh_lo[warp] = lo;
    }
    __syncthreads();
    double tot = 0.0;
    if (threadIdx.x == 0) {
        float th = 0.f, tl = 0.f;
        for (int w = 0; w < nw; ++w) ff_add(th, tl, sh_hi[w], sh_lo[w]);
        tot = (double)th + (double)tl;
    }
    return tot;
}

}  // namespace kv
