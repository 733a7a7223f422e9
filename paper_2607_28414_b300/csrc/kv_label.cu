// kv_label.cu -- class encoding of a pointwise FP32 medium.
//
// The step of Sec. 3.1 reads the folded coefficients A' = dt^2 G/(rho dx^2)
// and B' = dt eta/(rho dx^2) at every node: 8 bytes of the 56 that a
// heterogeneous step moves per node. Segmented media (a background with a
// few inclusions, a layered phantom) hold only a few distinct (A', B')
// pairs. After the fold, the pairs are counted with an open-addressing hash
// on the device; if there are at most kMaxLabels of them, every node gets one
// class byte and the step kernel looks its pair up in a table of FP32 values
// that are bit for bit the folded ones. The step then moves 49 bytes per node
// and computes exactly what it computes from the fields. Continuous media
// (more pairs) keep the field path; the count stops early once it overflows.
//
// Scratch (h->lab_keys, one allocation): kLabSlots 64-bit keys, kLabSlots
// slot ids, two counters.
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

// Insert every node's pair; counters[0] = distinct pairs, counters[1] = overflow.
__global__ void k_lab_insert(const float *__restrict__ A, const float *__restrict__ B, long long n,
                             unsigned long long *keys, int *counters) {
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
                                                          int *__restrict__ slot_id, float2 *__restrict__ tab) {
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
        tab[id] = make_float2(__uint_as_float((unsigned)(k >> 32)), __uint_as_float((unsigned)k));
}

// Class byte of every node (each pair is in the table, so each probe ends).
__global__ void k_lab_assign(const float *__restrict__ A, const float *__restrict__ B, long long n,
                             const unsigned long long *__restrict__ keys, const int *__restrict__ slot_id,
                             unsigned char *__restrict__ labels) {
    unsigned long long last = kEmptyKey;
    unsigned char last_id = 0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const unsigned long long key = pair_key(A[i], B[i]);
        if (key != last) {
            unsigned s = slot_hash(key);
            for (int probe = 0; probe < kLabSlots && keys[s] != key; ++probe) s = (s + 1) & (kLabSlots - 1);
            last = key;
            last_id = (unsigned char)slot_id[s];
        }
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

kv_status medium_classify(kv_handle *h) {
    const int before = h->n_labels;
    h->n_labels = 0;
    if (!h->het || step_kind(h) != kKindPoint || h->precision != KV_FP32 ||
        h->medium_encoding == KV_MEDIUM_FIELDS) {
        if (h->labels) {
            kv_status st = cuda_check(h, cudaStreamSynchronize(h->stream), "medium classes");
            if (st != KV_OK) return st;
            medium_labels_free(h);
        }
        if (before != 0) h->tma_ready = 0;
        return KV_OK;
    }
    cudaError_t e = cudaSuccess;
    const size_t scratch = kLabSlots * sizeof(unsigned long long) + kLabSlots * sizeof(int) + 2 * sizeof(int);
    if (!h->lab_keys) e = cudaMalloc((void **)&h->lab_keys, scratch);
    if (e != cudaSuccess) return cuda_check(h, e, "cudaMalloc(medium classes)");
    unsigned long long *keys = h->lab_keys;
    int *slot_id = reinterpret_cast<int *>(keys + kLabSlots);
    int *counters = slot_id + kLabSlots;
    const float *A = static_cast<const float *>(h->coef);
    const float *B = A + h->Np;
    e = cudaMemsetAsync(keys, 0xff, kLabSlots * sizeof(unsigned long long), h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(counters, 0, 2 * sizeof(int), h->stream);
    if (e != cudaSuccess) return cuda_check(h, e, "medium classes");
    const int nb = 148 * 8;
    k_lab_insert<<<nb, 256, 0, h->stream>>>(A, B, h->Np, keys, counters);
    h->launches++;
    int cnt[2] = {0, 0};
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
    if (e == cudaSuccess && !h->lab_tab) e = cudaMalloc((void **)&h->lab_tab, kMaxLabels * sizeof(float2));
    if (e != cudaSuccess) {
        medium_labels_free(h);
        return cuda_check(h, e, "cudaMalloc(medium classes)");
    }
    k_lab_compact<<<1, kLabSlots, 0, h->stream>>>(keys, slot_id, h->lab_tab);
    k_lab_assign<<<nb, 256, 0, h->stream>>>(A, B, h->Np, keys, slot_id, h->labels);
    h->launches += 2;
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_check(h, e, "medium classes");
    h->n_labels = cnt[0];
    h->tma_ready = 0;  // the step kernel's kind and coefficient map change
    return KV_OK;
}

}  // namespace kv
