// kv_label.cu -- class encoding of an FP32 medium.
//
// The step of Sec. 3.1 reads the folded coefficients at every node: A' =
// dt^2 G/(rho dx^2) and B' = dt eta/(rho dx^2) for the pointwise operator
// (8 of the 56 bytes a heterogeneous step moves per node), m = dt^2 G/dx^2,
// e = dt eta/dx^2 and 1/rho with their halos for the flux form (12 of 60).
// Segmented media (a background with a few inclusions, a layered phantom)
// hold only a few distinct tuples. After the fold, the tuples are counted
// with an open-addressing hash on the device keyed on the first two
// coefficients (the third, 1/rho of the flux form, is checked to be the same
// for every node of a class); if there are at most kMaxLabels classes, every
// node gets one class byte and the step kernel looks its tuple up in a table
// of FP32 values that are bit for bit the folded ones. The step then moves 49
// bytes per node and computes exactly what it computes from the fields.
// Continuous media keep the field path; the count stops early once it
// overflows.
//
// Scratch (h->lab_keys, one allocation): kLabSlots 64-bit keys, kLabSlots
// slot ids, kLabSlots third coefficients, three counters.
#include "kv_internal.cuh"

namespace kv {

constexpr unsigned long long kEmptyKey = ~0ull;  // a NaN bit pattern pair: never a folded key

__device__ __forceinline__ unsigned long long pair_key(float a, float b) {
    return ((unsigned long long)__float_as_uint(a) << 32) | __float_as_uint(b);
}

__device__ __forceinline__ unsigned slot_hash(unsigned long long k) {
    k ^= k >> 33;
    k *= 0xff51afd7ed558ccdull;
    k ^= k >> 33;
    return (unsigned)k & (kLabSlots - 1);
}

// Insert every node's pair (A, B); the node that creates a slot stores its C
// (NULL: none). counters[0] = distinct pairs, counters[1] = overflow.
__global__ void k_lab_insert(const float *__restrict__ A, const float *__restrict__ B,
                             const float *__restrict__ C, long long n, unsigned long long *keys,
                             float *third, int *counters) {
    volatile unsigned long long *vk = keys;
    volatile int *vc = counters;
    unsigned long long last = kEmptyKey;
    long long it = 0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x, ++it) {
        if ((it & 63) == 0 && vc[1]) return;  // already too many classes
        const unsigned long long key = pair_key(A[i], B[i]);
        if (key == last) continue;
        last = key;
        unsigned s = slot_hash(key);
        int probe = 0;
        for (; probe < kLabSlots; ++probe, s = (s + 1) & (kLabSlots - 1)) {
            const unsigned long long cur = vk[s];
            if (cur == key) break;
            if (cur == kEmptyKey) {
                const unsigned long long prev = atomicCAS(keys + s, kEmptyKey, key);
                if (prev == kEmptyKey) {
                    third[s] = C ? C[i] : 0.f;
                    if (atomicAdd(counters, 1) >= kMaxLabels) atomicExch(counters + 1, 1);
                    break;
                }
                if (prev == key) break;
            }
        }
        if (probe == kLabSlots) {
            atomicExch(counters + 1, 1);
            return;
        }
    }
}

// One block of kLabSlots threads: slot -> class id (slot order), class table.
__global__ void __launch_bounds__(kLabSlots) k_lab_compact(const unsigned long long *__restrict__ keys,
                                                          const float *__restrict__ third,
                                                          int *__restrict__ slot_id, float4 *__restrict__ tab) {
    __shared__ int warp_count[kLabSlots / 32];
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    const unsigned long long k = keys[t];
    const bool used = k != kEmptyKey;
    const unsigned ballot = __ballot_sync(0xffffffffu, used);
    if (lane == 0) warp_count[w] = __popc(ballot);
    __syncthreads();
    int base = 0;
    for (int q = 0; q < w; ++q) base += warp_count[q];
    const int id = base + __popc(ballot & ((1u << lane) - 1u));
    slot_id[t] = used ? id : -1;
    if (used && id < kMaxLabels)
        tab[id] = make_float4(__uint_as_float((unsigned)(k >> 32)), __uint_as_float((unsigned)k), third[t], 0.f);
}

// Class byte of every node (each pair is in the table, so each probe ends);
// counters[2] is set if a node's C differs from its class's (then the fields
// stay in use).
__global__ void k_lab_assign(const float *__restrict__ A, const float *__restrict__ B,
                             const float *__restrict__ C, long long n,
                             const unsigned long long *__restrict__ keys, const int *__restrict__ slot_id,
                             const float *__restrict__ third, unsigned char *__restrict__ labels,
                             int *counters) {
    unsigned long long last = kEmptyKey;
    unsigned char last_id = 0;
    unsigned last_c = 0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const unsigned long long key = pair_key(A[i], B[i]);
        if (key != last) {
            unsigned s = slot_hash(key);
            for (int probe = 0; probe < kLabSlots && keys[s] != key; ++probe) s = (s + 1) & (kLabSlots - 1);
            last = key;
            last_id = (unsigned char)slot_id[s];
            last_c = __float_as_uint(third[s]);
        }
        if (C && __float_as_uint(C[i]) != last_c) counters[2] = 1;
        labels[i] = last_id;
    }
}

void medium_labels_free(kv_handle *h) {
    cudaFree(h->labels);
    cudaFree(h->lab_tab);
    cudaFree(h->lab_keys);
    h->labels = nullptr;
    h->lab_tab = nullptr;
    h->lab_keys = nullptr;
    h->n_labels = 0;
}

// Flux-form media are classified as well (their class path is kKindDivLabel).
constexpr bool kClassifyDiv = true;

kv_status medium_classify(kv_handle *h) {
    const int before = h->n_labels;
    h->n_labels = 0;
    // the step kernel's kind follows n_labels: its tensor maps are re-encoded
    // before the next step whenever the classes change, also on an error below
    if (before != 0) h->tma_ready = 0;
    const int kind = step_kind(h);
    if (!h->het || h->precision != KV_FP32 || h->medium_encoding == KV_MEDIUM_FIELDS ||
        !(kind == kKindPoint || (kind == kKindDiv && kClassifyDiv))) {
        if (h->labels) {
            kv_status st = cuda_check(h, cudaStreamSynchronize(h->stream), "medium classes");
            if (st != KV_OK) return st;
            medium_labels_free(h);
        }
        if (before != 0) h->tma_ready = 0;
        return KV_OK;
    }
    cudaError_t e = cudaSuccess;
    const size_t scratch = kLabSlots * (sizeof(unsigned long long) + sizeof(int) + sizeof(float)) + 4 * sizeof(int);
    if (!h->lab_keys) e = cudaMalloc((void **)&h->lab_keys, scratch);
    if (e != cudaSuccess) return cuda_check(h, e, "cudaMalloc(medium classes)");
    unsigned long long *keys = h->lab_keys;
    int *slot_id = reinterpret_cast<int *>(keys + kLabSlots);
    float *third = reinterpret_cast<float *>(slot_id + kLabSlots);
    int *counters = reinterpret_cast<int *>(third + kLabSlots);
    const float *A = static_cast<const float *>(h->coef);
    const float *B = A + h->Np;
    const float *C = kind == kKindDiv ? B + h->Np : nullptr;
    e = cudaMemsetAsync(keys, 0xff, kLabSlots * sizeof(unsigned long long), h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(counters, 0, 4 * sizeof(int), h->stream);
    if (e != cudaSuccess) return cuda_check(h, e, "medium classes");
    const int nb = 148 * 8;
    k_lab_insert<<<nb, 256, 0, h->stream>>>(A, B, C, h->Np, keys, third, counters);
    h->launches++;
    int cnt[3] = {0, 0, 0};
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(cnt, counters, sizeof(cnt), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_check(h, e, "medium classes");
    if (cnt[1] || cnt[0] > kMaxLabels || cnt[0] < 1) {  // continuous medium: read the fields
        medium_labels_free(h);
        if (before != 0) h->tma_ready = 0;
        return KV_OK;
    }
    if (!h->labels) e = cudaMalloc((void **)&h->labels, (size_t)h->Np);
    if (e == cudaSuccess && !h->lab_tab) e = cudaMalloc((void **)&h->lab_tab, kMaxLabels * sizeof(float4));
    if (e != cudaSuccess) {
        medium_labels_free(h);
        return cuda_check(h, e, "cudaMalloc(medium classes)");
    }
    k_lab_compact<<<1, kLabSlots, 0, h->stream>>>(keys, third, slot_id, h->lab_tab);
    k_lab_assign<<<nb, 256, 0, h->stream>>>(A, B, C, h->Np, keys, slot_id, third, h->labels, counters);
    h->launches += 2;
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(cnt, counters, sizeof(cnt), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_check(h, e, "medium classes");
    if (cnt[2]) {  // (m, e) does not determine 1/rho: read the fields
        medium_labels_free(h);
        if (before != 0) h->tma_ready = 0;
        return KV_OK;
    }
    h->n_labels = cnt[0];
    h->tma_ready = 0;  // the step kernel's kind and coefficient map change
    return KV_OK;
}

}  // namespace kv
