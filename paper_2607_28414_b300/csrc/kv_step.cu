// kv_step.cu -- the fused Kelvin-Voigt time step (Sec. 3.1 explicit update with
// the pre-computed projected force of Sec. 3.3) and its helpers.
//
// State layout: two buffers of [6][nz][ny][px] (u_x, u_y, u_z, d_x, d_y, d_z),
// d = u^n - u^{n-1}; px = nx rounded up to 32 elements. One step reads buffer
// `cur` and writes the other (ping-pong), so no stencil read ever races a write.
// The Dirichlet layer and the row padding hold zeros and are never written.
//
// Per interior node, component c (L^ = unscaled 7-point stencil):
//   d' = d + A' L^u + B' L^d + g_n F,   u' = u + d'
// with A' = dt^2 G/(rho dx^2), B' = dt eta/(rho dx^2), F = dt^2 f_S0/rho. This is
// u^{n+1} = 2u^n - u^{n-1} + dt^2 a^n of Sec. 3.1 with udot = (u^n - u^{n-1})/dt,
// rewritten so that the FP32 increment d keeps its own relative precision.
//
// The last block of every step records the sensors (u^{n+1}) and advances the
// device step counter, so a block of steps can be replayed from a CUDA graph.
#include <cudaTypedefs.h>
#include <stdio.h>

#include "kv_internal.cuh"

namespace kv {

// ---------------------------------------------------------------------------
// Epilogue shared by the step kernels: the last block to finish records
// u^{n+1} at the sensors and advances the step counter.
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ void step_epilogue(const T *out, const StepParams &p, long long step) {
    __shared__ int s_last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long t =
            atomicAdd(reinterpret_cast<unsigned long long *>(&p.ctrl[kStepTicket]), 1ull);
        s_last = (t == (unsigned long long)(p.nblocks - 1));
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    if (step < p.cap) {
        T *tr = reinterpret_cast<T *>(p.traces) + (size_t)step * p.ns * 3;
        for (int s = threadIdx.x; s < p.ns; s += blockDim.x) {
            const int i = p.sensors[3 * s], j = p.sensors[3 * s + 1], k = p.sensors[3 * s + 2];
            const size_t c = ((size_t)k * p.ny + j) * p.px + i;
            for (int comp = 0; comp < 3; ++comp) tr[3 * s + comp] = __ldcg(out + comp * p.Np + c);
        }
    } else if (threadIdx.x == 0 && p.ns > 0) {
        atomicOr(reinterpret_cast<unsigned long long *>(&p.ctrl[kErrFlags]), 2ull);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        p.ctrl[kStepTicket] = 0;
        p.ctrl[kStep] = step + 1;
    }
}

// ---------------------------------------------------------------------------
// Plain per-node kernel (FP64 check mode; FP32 reference variant).
// Grid: (ceil(nx/128), ny-2, nz-2), block 128; node (i, 1+blockIdx.y, 1+blockIdx.z).
// K: kKindHomo / kKindPoint (coef = [A', B']) / kKindDiv (coef = [m, e, 1/rho]).
// ---------------------------------------------------------------------------
template <typename T, int K>
__global__ void __launch_bounds__(128)
k_step_plain(const T *__restrict__ in, T *__restrict__ out, const T *__restrict__ coef,
             const T *__restrict__ F, StepParams p) {
    const long long step = __ldcg(&p.ctrl[kStep]);
    const T g = p.g_const_on ? T(p.g_const) : (step < p.n_g) ? T(p.g[step]) : T(0);
    const bool force = (g != T(0));
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = 1 + blockIdx.y;
    const int k = 1 + blockIdx.z;
    if (i >= 1 && i <= p.nx - 2) {
        const long long sy = p.px, sz = (long long)p.px * p.ny;
        const long long c = k * sz + j * sy + i;
        const long long nb[6] = {c - 1, c + 1, c - sy, c + sy, c - sz, c + sz};
        if constexpr (K == kKindDiv) {
            const T *m = coef, *e = coef + p.Np;
            T wm[6], we[6];
#pragma unroll
            for (int f = 0; f < 6; ++f) {
                wm[f] = face_weight(m[c], m[nb[f]]);
                we[f] = face_weight(e[c], e[nb[f]]);
            }
            const T r = coef[2 * p.Np + c];
#pragma unroll
            for (int comp = 0; comp < 3; ++comp) {
                const T *u = in + comp * p.Np;
                const T *d = in + (3 + comp) * p.Np;
                T nu[6], nd[6];
#pragma unroll
                for (int f = 0; f < 6; ++f) {
                    nu[f] = u[nb[f]];
                    nd[f] = d[nb[f]];
                }
                const T Fv = force ? F[comp * p.Np + c] : T(0);
                T uo, dn;
                kv_update_div(u[c], nu, d[c], nd, wm, we, r, g, Fv, uo, dn);
                out[comp * p.Np + c] = uo;
                out[(3 + comp) * p.Np + c] = dn;
            }
        } else {
            const T A = K == kKindPoint ? coef[c] : T(p.A);
            const T B = K == kKindPoint ? coef[p.Np + c] : T(p.B);
#pragma unroll
            for (int comp = 0; comp < 3; ++comp) {
                const T *u = in + comp * p.Np;
                const T *d = in + (3 + comp) * p.Np;
                const T su = kv_add(kv_add(kv_add(u[c - 1], u[c + 1]), kv_add(u[c - sy], u[c + sy])),
                                    kv_add(u[c - sz], u[c + sz]));
                const T sd = kv_add(kv_add(kv_add(d[c - 1], d[c + 1]), kv_add(d[c - sy], d[c + sy])),
                                    kv_add(d[c - sz], d[c + sz]));
                const T Fv = force ? F[comp * p.Np + c] : T(0);
                T uo, dn;
                kv_update(u[c], su, d[c], sd, A, B, g, Fv, uo, dn);
                out[comp * p.Np + c] = uo;
                out[(3 + comp) * p.Np + c] = dn;
            }
        }
    }
    step_epilogue<T>(out, p, step);
}

// ---------------------------------------------------------------------------
// TMA-staged z-march kernel (FP32).
//
// A block owns a TX x TY column of nodes and marches planes k0..k1-1. Each
// plane of all six state fields, with a 4-node x halo (keeps the TMA x start
// 16-byte aligned) and a 1-node y halo, arrives in one 4D TMA box
// (TX+8, TY+2, 1, 6) into a ring of NS shared-memory stages; the coefficient
// (A', B') tile of the centre plane rides in the same stage. Planes k and k+1
// are resident while plane k is computed (the z-1 neighbours are plane k-1's
// centre values, kept in registers) and NS-2 further planes are in flight.
// The projected force (needed only on the few force steps) is read directly
// from global memory as float4, one plane ahead. Each thread computes four
// consecutive x nodes (one float4) of one row; its x neighbours come from warp
// shuffles (row edges from shared memory). Outputs go straight to global
// memory as float4 stores.
//
// Divergence form (K = kKindDiv): the face weights need the moduli of the six
// neighbours, so every staged plane also carries the three coefficient fields
// (m, e, 1/rho) with the same halo, in a second box (TX+8, TY+2, 1, 3).
//
// Class-encoded media (K = kKindLabel, kKindDivLabel): the coefficient box is a
// tile of class bytes instead ((TX, TY) of the centre plane; for the flux form
// (TX+32, TY+2) from x0-16, so the byte box starts on a 16-byte boundary), and
// the folded coefficients come from tables in shared memory filled at block
// start. The table values are the folded FP32 values, so both kinds compute
// bit for bit what kKindPoint and kKindDiv compute from the fields.
// ---------------------------------------------------------------------------
template <int TX, int TY, int K>
struct TmaTile {
    static constexpr int NT = TX * TY / 4;
    static constexpr int GX = TX / 4;
    static constexpr int BX = TX + 8;
    static constexpr int BY = TY + 2;
    static constexpr int FIELD = BX * BY;
    static constexpr int STATE = 6 * FIELD;
    static constexpr int BXB = TX + 32;  // class-byte rows of the flux form: x0-16 .. x0+TX+15
    static constexpr int COEF = K == kKindPoint      ? 2 * TX * TY
                                : K == kKindDiv      ? 3 * FIELD
                                : K == kKindLabel    ? TX * TY / 4   // one class byte per node
                                : K == kKindDivLabel ? BXB * BY / 4  // class bytes with the halo
                                                     : 0;
    static constexpr int STAGE = (STATE + COEF + 31) / 32 * 32;  // floats, 128 B multiple
};

// The seven-point neighbourhood of four consecutive x nodes of one staged
// field: centre, x-, x+, y-, y+, z-, z+ (each a float4 over the four nodes).
struct Nb7 {
    float4 c, xm, xp, ym, yp, zm, zp;
};

template <int BX, int GX>
__device__ __forceinline__ Nb7 gather7(const float *sc, const float4 &zm, const float *sp, int off,
                                       int gx) {
    Nb7 n;
    const float *fc = sc + off;
    n.c = *reinterpret_cast<const float4 *>(fc);
    n.ym = *reinterpret_cast<const float4 *>(fc - BX);
    n.yp = *reinterpret_cast<const float4 *>(fc + BX);
    n.zm = zm;
    n.zp = *reinterpret_cast<const float4 *>(sp + off);
    float left = __shfl_up_sync(0xffffffffu, n.c.w, 1);
    float right = __shfl_down_sync(0xffffffffu, n.c.x, 1);
    if (gx == 0) left = fc[-1];
    if (gx == GX - 1) right = fc[4];
    n.xm = make_float4(left, n.c.x, n.c.y, n.c.z);
    n.xp = make_float4(n.c.y, n.c.z, n.c.w, right);
    return n;
}

// Lane q (0..3) of a float4.
__device__ __forceinline__ float lane4(const float4 &v, int q) {
    return q == 0 ? v.x : q == 1 ? v.y : q == 2 ? v.z : v.w;
}
__device__ __forceinline__ void set_lane4(float4 &v, int q, float x) {
    if (q == 0) v.x = x;
    else if (q == 1) v.y = x;
    else if (q == 2) v.z = x;
    else v.w = x;
}

// Neighbour values of node q of a gathered neighbourhood, order xm, xp, ym, yp, zm, zp.
__device__ __forceinline__ void nb_of(const Nb7 &n, int q, float (&v)[6]) {
    v[0] = lane4(n.xm, q);
    v[1] = lane4(n.xp, q);
    v[2] = lane4(n.ym, q);
    v[3] = lane4(n.yp, q);
    v[4] = lane4(n.zm, q);
    v[5] = lane4(n.zp, q);
}

// Class-encoded media: the first two coefficients ((A', B') or (m, e)) and
// the third (1/rho of the flux form) of four consecutive nodes from their four
// class bytes (one 32-bit word) and the class tables.
__device__ __forceinline__ void class_quad2(uint32_t q, const float2 *tab, float4 &a, float4 &b) {
    const float2 t0 = tab[q & 255u], t1 = tab[(q >> 8) & 255u], t2 = tab[(q >> 16) & 255u], t3 = tab[q >> 24];
    a = make_float4(t0.x, t1.x, t2.x, t3.x);
    b = make_float4(t0.y, t1.y, t2.y, t3.y);
}
__device__ __forceinline__ float4 class_quad1(uint32_t q, const float *tab) {
    return make_float4(tab[q & 255u], tab[(q >> 8) & 255u], tab[(q >> 16) & 255u], tab[q >> 24]);
}

// gather7 of m and e from class-byte tiles (row stride BXB, this thread's
// first node at byte offset off): the centre values cm, ce were decoded one
// plane earlier (as that plane's z+ neighbours), the z-1 neighbours are the
// previous plane's centre values, the y neighbours come from the centre
// plane's bytes and the x neighbours from the warp or the edge bytes; nzm,
// nze are this plane's decoded z+ neighbours.
template <int GX>
__device__ __forceinline__ void gather7_cls(const unsigned char *bc, int off, int BXB, int gx, const float2 *tab,
                                            const float4 &cm, const float4 &ce, const float4 &zm_m,
                                            const float4 &zm_e, const float4 &nzm, const float4 &nze, Nb7 &m,
                                            Nb7 &e) {
    m.c = cm;
    e.c = ce;
    class_quad2(*reinterpret_cast<const uint32_t *>(bc + off - BXB), tab, m.ym, e.ym);
    class_quad2(*reinterpret_cast<const uint32_t *>(bc + off + BXB), tab, m.yp, e.yp);
    m.zm = zm_m;
    e.zm = zm_e;
    m.zp = nzm;
    e.zp = nze;
    float lm = __shfl_up_sync(0xffffffffu, m.c.w, 1), rm = __shfl_down_sync(0xffffffffu, m.c.x, 1);
    float le = __shfl_up_sync(0xffffffffu, e.c.w, 1), re = __shfl_down_sync(0xffffffffu, e.c.x, 1);
    if (gx == 0) {
        const float2 t = tab[bc[off - 1]];
        lm = t.x;
        le = t.y;
    }
    if (gx == GX - 1) {
        const float2 t = tab[bc[off + 4]];
        rm = t.x;
        re = t.y;
    }
    m.xm = make_float4(lm, m.c.x, m.c.y, m.c.z);
    m.xp = make_float4(m.c.y, m.c.z, m.c.w, rm);
    e.xm = make_float4(le, e.c.x, e.c.y, e.c.z);
    e.xp = make_float4(e.c.y, e.c.z, e.c.w, re);
}

// One block's work: the TX x TY column (bx, by) over planes of z chunk bz.
// tm_in / tm_coef: addresses of tensor maps in parameter or global memory.
template <int TX, int TY, int NS, int K>
__device__ __forceinline__ void step_tile(const CUtensorMap *tm_in, const CUtensorMap *tm_coef,
                                          const float *__restrict__ F, float *__restrict__ out,
                                          const StepParams &p, int bx, int by, int bz) {
    using TT = TmaTile<TX, TY, K>;
    extern __shared__ __align__(128) float smem[];
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + NS * TT::STAGE);

    const int tid = threadIdx.x;
    const int gx = tid % TT::GX, gy = tid / TT::GX;
    const int x0 = bx * TX;
    const int y0 = 1 + by * TY;
    const int k0 = 1 + bz * p.zc;
    const int k1 = min(k0 + p.zc, p.nz - 1);  // planes k0..k1-1 are computed
    const int kb = k0 - 1;                     // first staged plane
    const long long step = __ldcg(&p.ctrl[kStep]);
    const float g = p.g_const_on ? p.g_const : (step < p.n_g) ? p.g[step] : 0.f;
    const bool force = (g != 0.f);
    const uint32_t bar0 = smem_u32(bars);

    // class table of a class-encoded medium: (A', B') of every class
    constexpr bool CLS = K == kKindLabel || K == kKindDivLabel;
    __shared__ float2 s_tab[CLS ? kMaxLabels : 1];                     // (A', B') or (m, e)
    __shared__ float s_tab3[K == kKindDivLabel ? kMaxLabels : 1];       // 1/rho of the flux form
    if (CLS)
        for (int i = threadIdx.x; i < p.n_lab; i += TT::NT) {
            const float4 t = p.lab_tab[i];
            s_tab[i] = make_float2(t.x, t.y);
            if (K == kKindDivLabel) s_tab3[i] = t.z;
        }
    if (tid == 0) {
        for (int s = 0; s < NS; ++s) mbar_init(bar0 + 8 * s, 1);
        mbar_init_fence();
    }
    __syncthreads();

    auto issue = [&](int q) {  // thread 0: stage plane q (kb <= q <= k1)
        const int s = (q - kb) % NS;
        float *st = smem + s * TT::STAGE;
        const uint32_t bar = bar0 + 8 * s;
        const bool wc =
            ((K == kKindPoint || K == kKindLabel) && q >= k0 && q < k1) || K == kKindDiv || K == kKindDivLabel;
        const uint32_t bytes = TT::STATE * 4 + (wc ? TT::COEF * 4 : 0);
        mbar_expect_tx(bar, bytes);
        tma_load_4d(smem_u32(st), tm_in, x0 - 4, y0 - 1, q, 0, bar);
        if ((K == kKindPoint || K == kKindLabel) && wc)
            tma_load_4d(smem_u32(st + TT::STATE), tm_coef, x0, y0, q, 0, bar);
        if (K == kKindDiv) tma_load_4d(smem_u32(st + TT::STATE), tm_coef, x0 - 4, y0 - 1, q, 0, bar);
        if (K == kKindDivLabel) tma_load_4d(smem_u32(st + TT::STATE), tm_coef, x0 - 16, y0 - 1, q, 0, bar);
    };

    if (tid == 0) {
        const int last = min(k1, kb + NS - 1);
        for (int q = kb; q <= last; ++q) issue(q);
    }

    bool ok = true;
    const int y = y0 + gy;
    const int x = x0 + 4 * gx;
    const bool row_ok = (y <= p.ny - 2) && (x < p.px);
    const int o = (gy + 1) * TT::BX + 4 + 4 * gx;  // this thread's first node in a field tile
    const long long sy = p.px, sz = (long long)p.px * p.ny;
    const unsigned FULL = 0xffffffffu;

    // Register-blocked z march: the z-1 neighbours are the previous plane's
    // centre values, kept in registers, so a stage is free as soon as its
    // plane has been computed and NS-2 planes are in flight.
    float4 prev[6], prevc[2];
    ok &= mbar_wait_bounded(bar0, 0);  // plane kb, slot 0, first phase
#pragma unroll
    for (int f = 0; f < 6; ++f) prev[f] = *reinterpret_cast<const float4 *>(smem + f * TT::FIELD + o);
    const int ob = (gy + 1) * TT::BXB + 16 + 4 * gx;  // this thread's first node in a class-byte tile
    if (K == kKindDiv) {
        prevc[0] = *reinterpret_cast<const float4 *>(smem + TT::STATE + o);
        prevc[1] = *reinterpret_cast<const float4 *>(smem + TT::STATE + TT::FIELD + o);
    }
    if constexpr (K == kKindDivLabel)
        class_quad2(*reinterpret_cast<const uint32_t *>(reinterpret_cast<const unsigned char *>(smem + TT::STATE) + ob),
                    s_tab, prevc[0], prevc[1]);
    __syncthreads();  // every thread has read plane kb: its slot is free
    if (tid == 0 && kb + NS <= k1) {
        fence_proxy_async();
        issue(kb + NS);
    }
    ok &= mbar_wait_bounded(bar0 + 8 * ((k0 - kb) % NS), ((k0 - kb) / NS) & 1);
    // class-encoded flux form: plane k0's centre coefficients (later planes'
    // are decoded one plane ahead, as z+ neighbours)
    float4 cur_m, cur_e, cur_r;
    if constexpr (K == kKindDivLabel) {
        const uint32_t w = *reinterpret_cast<const uint32_t *>(
            reinterpret_cast<const unsigned char *>(smem + ((k0 - kb) % NS) * TT::STAGE + TT::STATE) + ob);
        class_quad2(w, s_tab, cur_m, cur_e);
        cur_r = class_quad1(w, s_tab3);
    }

    // Force steps: the projected force of the next plane is loaded one plane
    // ahead, so its latency overlaps the current plane's work.
    float4 Fn[3];
    auto load_force = [&](int kk) {
#pragma unroll
        for (int comp = 0; comp < 3; ++comp)
            Fn[comp] = (force && row_ok)
                           ? __ldg(reinterpret_cast<const float4 *>(F + comp * p.Np + kk * sz + y * sy + x))
                           : make_float4(0.f, 0.f, 0.f, 0.f);
    };
    if (force) load_force(k0);

    for (int k = k0; k < k1; ++k) {
        float4 Fc[3];
#pragma unroll
        for (int comp = 0; comp < 3; ++comp) Fc[comp] = force ? Fn[comp] : make_float4(0.f, 0.f, 0.f, 0.f);
        if (force && k + 1 < k1) load_force(k + 1);
        ok &= mbar_wait_bounded(bar0 + 8 * ((k + 1 - kb) % NS), ((k + 1 - kb) / NS) & 1);

        const float *sc = smem + ((k - kb) % NS) * TT::STAGE;
        const float *sp = smem + ((k + 1 - kb) % NS) * TT::STAGE;

        if constexpr (K == kKindDiv || K == kKindDivLabel) {
            // face weights of the four nodes, shared by the three components
            Nb7 mn, en;
            float4 r4;
            if constexpr (K == kKindDivLabel) {
                const uint32_t wz = *reinterpret_cast<const uint32_t *>(
                    reinterpret_cast<const unsigned char *>(sp + TT::STATE) + ob);
                float4 nzm, nze;
                class_quad2(wz, s_tab, nzm, nze);
                gather7_cls<TT::GX>(reinterpret_cast<const unsigned char *>(sc + TT::STATE), ob, TT::BXB, gx, s_tab,
                                    cur_m, cur_e, prevc[0], prevc[1], nzm, nze, mn, en);
                r4 = cur_r;
                cur_m = nzm;
                cur_e = nze;
                cur_r = class_quad1(wz, s_tab3);
            } else {
                mn = gather7<TT::BX, TT::GX>(sc, prevc[0], sp, TT::STATE + o, gx);
                en = gather7<TT::BX, TT::GX>(sc, prevc[1], sp, TT::STATE + TT::FIELD + o, gx);
                r4 = *reinterpret_cast<const float4 *>(sc + TT::STATE + 2 * TT::FIELD + o);
            }
            prevc[0] = mn.c;
            prevc[1] = en.c;
            float wm[4][6], we[4][6];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                float vm[6], ve[6];
                nb_of(mn, q, vm);
                nb_of(en, q, ve);
                const float mc = lane4(mn.c, q), ec = lane4(en.c, q);
#pragma unroll
                for (int f = 0; f < 6; ++f) {
                    wm[q][f] = face_weight(mc, vm[f]);
                    we[q][f] = face_weight(ec, ve[f]);
                }
            }
            const long long gbase = k * sz + y * sy + x;
#pragma unroll
            for (int comp = 0; comp < 3; ++comp) {
                const Nb7 un = gather7<TT::BX, TT::GX>(sc, prev[comp], sp, comp * TT::FIELD + o, gx);
                const Nb7 dnb = gather7<TT::BX, TT::GX>(sc, prev[3 + comp], sp, (3 + comp) * TT::FIELD + o, gx);
                prev[comp] = un.c;
                prev[3 + comp] = dnb.c;
                if (row_ok) {
                    const float4 F4 = Fc[comp];
                    float4 uo, dn;
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        float nu[6], nd[6], uq, dq;
                        nb_of(un, q, nu);
                        nb_of(dnb, q, nd);
                        kv_update_div(lane4(un.c, q), nu, lane4(dnb.c, q), nd, wm[q], we[q],
                                      lane4(r4, q), g, lane4(F4, q), uq, dq);
                        const bool inside = (x + q >= 1) && (x + q <= p.nx - 2);
                        set_lane4(uo, q, inside ? uq : 0.f);
                        set_lane4(dn, q, inside ? dq : 0.f);
                    }
                    *reinterpret_cast<float4 *>(out + comp * p.Np + gbase) = uo;
                    *reinterpret_cast<float4 *>(out + (3 + comp) * p.Np + gbase) = dn;
                }
            }
        } else {
            float4 ctr[6], sum[6];
    #pragma unroll
            for (int f = 0; f < 6; ++f) {
                const float *fc = sc + f * TT::FIELD + o;
                const float4 c = *reinterpret_cast<const float4 *>(fc);
                const float4 ym = *reinterpret_cast<const float4 *>(fc - TT::BX);
                const float4 yp = *reinterpret_cast<const float4 *>(fc + TT::BX);
                const float4 zm = prev[f];
                const float4 zp = *reinterpret_cast<const float4 *>(sp + f * TT::FIELD + o);
                float left = __shfl_up_sync(FULL, c.w, 1);
                float right = __shfl_down_sync(FULL, c.x, 1);
                if (gx == 0) left = fc[-1];
                if (gx == TT::GX - 1) right = fc[4];
                float4 s;
                s.x = kv_add(kv_add(kv_add(left, c.y), kv_add(ym.x, yp.x)), kv_add(zm.x, zp.x));
                s.y = kv_add(kv_add(kv_add(c.x, c.z), kv_add(ym.y, yp.y)), kv_add(zm.y, zp.y));
                s.z = kv_add(kv_add(kv_add(c.y, c.w), kv_add(ym.z, yp.z)), kv_add(zm.z, zp.z));
                s.w = kv_add(kv_add(kv_add(c.z, right), kv_add(ym.w, yp.w)), kv_add(zm.w, zp.w));
                ctr[f] = c;
                sum[f] = s;
                prev[f] = c;
            }
            float4 A4, B4;
            if (K == kKindPoint) {
                A4 = *reinterpret_cast<const float4 *>(sc + TT::STATE + gy * TX + 4 * gx);
                B4 = *reinterpret_cast<const float4 *>(sc + TT::STATE + TX * TY + gy * TX + 4 * gx);
            } else if (K == kKindLabel) {
                const uint32_t l4 = *reinterpret_cast<const uint32_t *>(
                    reinterpret_cast<const unsigned char *>(sc + TT::STATE) + gy * TX + 4 * gx);
                class_quad2(l4, s_tab, A4, B4);
            } else {
                A4 = make_float4((float)p.A, (float)p.A, (float)p.A, (float)p.A);
                B4 = make_float4((float)p.B, (float)p.B, (float)p.B, (float)p.B);
            }
            if (row_ok) {
                const long long gbase = k * sz + y * sy + x;
                const bool m0 = (x >= 1) && (x <= p.nx - 2);
                const bool m1 = (x + 1 >= 1) && (x + 1 <= p.nx - 2);
                const bool m2 = (x + 2 <= p.nx - 2);
                const bool m3 = (x + 3 <= p.nx - 2);
    #pragma unroll
                for (int comp = 0; comp < 3; ++comp) {
                    const float4 F4 = Fc[comp];
                    const float4 u = ctr[comp], su = sum[comp], d = ctr[3 + comp], sd = sum[3 + comp];
                    float4 uo, dn;
                    kv_update(u.x, su.x, d.x, sd.x, A4.x, B4.x, g, F4.x, uo.x, dn.x);
                    kv_update(u.y, su.y, d.y, sd.y, A4.y, B4.y, g, F4.y, uo.y, dn.y);
                    kv_update(u.z, su.z, d.z, sd.z, A4.z, B4.z, g, F4.z, uo.z, dn.z);
                    kv_update(u.w, su.w, d.w, sd.w, A4.w, B4.w, g, F4.w, uo.w, dn.w);
                    if (!m0) uo.x = dn.x = 0.f;
                    if (!m1) uo.y = dn.y = 0.f;
                    if (!m2) uo.z = dn.z = 0.f;
                    if (!m3) uo.w = dn.w = 0.f;
                    *reinterpret_cast<float4 *>(out + comp * p.Np + gbase) = uo;
                    *reinterpret_cast<float4 *>(out + (3 + comp) * p.Np + gbase) = dn;
                }
            }
        }
        __syncthreads();  // every thread is done with plane k's stage
        if (tid == 0) {
            const int q = k + NS;
            if (q <= k1) {
                fence_proxy_async();
                issue(q);
            }
        }
    }

    if (!ok) atomicOr(reinterpret_cast<unsigned long long *>(&p.ctrl[kErrFlags]), 1ull);
    // A wait that gave up may leave a copy in flight: drain every stage (bounded)
    // before the block's shared memory is released.
    if (__syncthreads_or(!ok) && tid == 0) {
        const int rel_max = k1 - kb;
        for (int s = 0; s < NS && s <= rel_max; ++s) {
            const int rel_last = s + ((rel_max - s) / NS) * NS;
            mbar_wait_bounded(bar0 + 8 * s, (rel_last / NS) & 1);
        }
    }
    step_epilogue<float>(out, p, step);
}

template <int TX, int TY, int NS, int K>
__global__ void __launch_bounds__(TX *TY / 4)
k_step_tma(const __grid_constant__ CUtensorMap tm_in, const __grid_constant__ CUtensorMap tm_coef,
           const float *__restrict__ F, float *__restrict__ out, StepParams p) {
    step_tile<TX, TY, NS, K>(&tm_in, &tm_coef, F, out, p, blockIdx.x, blockIdx.y, blockIdx.z);
}

// Batched step: one launch advances every case of a batch by one step. Block
// b belongs to the case whose [block_begin, block_begin + blocks) holds b; the
// case's own tensor maps, coefficients, envelope, sensors and control block
// come from the case table, and its last block runs that case's epilogue.
template <int TX, int TY, int NS, int K>
__global__ void __launch_bounds__(TX *TY / 4)
k_step_batch(const BatchCase *__restrict__ cases, int ncases, int from) {
    int c = 0;
    while (c + 1 < ncases && (int)blockIdx.x >= cases[c + 1].block_begin) ++c;
    const BatchCase &cs = cases[c];
    const int local = blockIdx.x - cs.block_begin;
    const int bx = local % cs.gx, by = (local / cs.gx) % cs.gy, bz = local / (cs.gx * cs.gy);
    step_tile<TX, TY, NS, K>(&cs.tm_state[from], &cs.tm_coef, cs.F, cs.state[1 - from], cs.p, bx,
                               by, bz);
}

// ---------------------------------------------------------------------------
// Two steps per sweep (temporal blocking), FP32.
//
// Each z-march iteration k first computes the intermediate state (u, d)^{n+1}
// of plane k+1 over the block's tile plus a one-node ring (rows y0-1..y0+TY,
// columns x0-4..x0+TX+3 in float4 groups) into a 2-plane shared-memory ring,
// then the final state (u, d)^{n+2} of plane k over the tile, written to global
// memory. The z-1 neighbours of both levels (input plane j-1 of an
// intermediate node, intermediate plane k-1 of an output node) stay in
// registers, and the output nodes' coefficients are read one plane ahead, so
// an input stage is refilled as soon as its plane has been used as a centre. The state at step n arrives by TMA with a 2-row y halo and the
// aligned 4-column x halo. Every node of both levels goes through kv_update
// with the same neighbour order as the single-step kernels, so two steps here
// are bit-identical to two single steps. Intermediate nodes outside the grid or
// on the Dirichlet layer are 0. The sensors of the intermediate step are
// recorded by the block that owns their node (per-plane sensor index); the
// last block records the final step and advances the step counter by two.
// ---------------------------------------------------------------------------
template <int TX, int TY, bool HET>
struct Tile2 {
    static constexpr int BX = TX + 8;
    static constexpr int BYI = TY + 4;
    static constexpr int BYM = TY + 2;
    static constexpr int IN_F = BX * BYI;
    static constexpr int MID_F = BX * BYM;
    static constexpr int IN_STATE = 6 * IN_F;
    static constexpr int IN_COEF = HET ? 2 * MID_F : 0;
    static constexpr int IN_STAGE = (IN_STATE + IN_COEF + 31) / 32 * 32;
    static constexpr int MID_STAGE = (6 * MID_F + 31) / 32 * 32;
    static constexpr int GXI = BX / 4;
    static constexpr int MID_GROUPS = GXI * BYM;
    static constexpr int GX = TX / 4;
    static constexpr int OUT_GROUPS = GX * TY;
    static constexpr int NT = 128;
};

template <typename T>
__device__ __forceinline__ void step_epilogue_n(const T *out, const StepParams &p, long long step, int nsteps) {
    __shared__ int s_last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long t =
            atomicAdd(reinterpret_cast<unsigned long long *>(&p.ctrl[kStepTicket]), 1ull);
        s_last = (t == (unsigned long long)(p.nblocks - 1));
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    const long long row = step + nsteps - 1;
    if (row < p.cap) {
        T *tr = reinterpret_cast<T *>(p.traces) + (size_t)row * p.ns * 3;
        for (int s = threadIdx.x; s < p.ns; s += blockDim.x) {
            const int i = p.sensors[3 * s], j = p.sensors[3 * s + 1], k = p.sensors[3 * s + 2];
            const size_t c = ((size_t)k * p.ny + j) * p.px + i;
            for (int comp = 0; comp < 3; ++comp) tr[3 * s + comp] = __ldcg(out + comp * p.Np + c);
        }
    } else if (threadIdx.x == 0 && p.ns > 0) {
        atomicOr(reinterpret_cast<unsigned long long *>(&p.ctrl[kErrFlags]), 2ull);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        p.ctrl[kStepTicket] = 0;
        p.ctrl[kStep] = step + nsteps;
    }
}

template <int TX, int TY, int NS, bool HET>
__global__ void __launch_bounds__(128)
k_step2_tma(const __grid_constant__ CUtensorMap tm_in, const __grid_constant__ CUtensorMap tm_coef,
            const float *__restrict__ F, float *__restrict__ out, StepParams p) {
    using T2 = Tile2<TX, TY, HET>;
    constexpr int RM = (T2::MID_GROUPS + T2::NT - 1) / T2::NT;  // intermediate groups per thread
    constexpr int RO = (T2::OUT_GROUPS + T2::NT - 1) / T2::NT;  // output groups per thread
    extern __shared__ __align__(128) float smem[];
    float *inr = smem;                                 // NS input stages
    float *mid = smem + NS * T2::IN_STAGE;             // 2 intermediate planes
    uint64_t *bars = reinterpret_cast<uint64_t *>(mid + 2 * T2::MID_STAGE);
    const uint32_t bar0 = smem_u32(bars);
    const int tid = threadIdx.x;
    const int x0 = blockIdx.x * TX, y0 = 1 + blockIdx.y * TY;
    const int k0 = 1 + blockIdx.z * p.zc;
    const int k1 = min(k0 + p.zc, p.nz - 1);  // output planes k0..k1-1
    const int qb = k0 - 2;                     // first staged input plane (may be -1)
    const long long step = __ldcg(&p.ctrl[kStep]);
    const float g0 = p.g_const_on ? p.g_const : (step < p.n_g) ? p.g[step] : 0.f;
    const float g1 = p.g_const_on ? p.g_const : (step + 1 < p.n_g) ? p.g[step + 1] : 0.f;
    const long long sy = p.px, sz = (long long)p.px * p.ny;

    if (tid == 0) {
        for (int s = 0; s < NS; ++s) mbar_init(bar0 + 8 * s, 1);
        mbar_init_fence();
    }
    __syncthreads();
    auto slot = [&](int q) { return (q - qb) % NS; };
    auto par = [&](int q) { return (uint32_t)(((q - qb) / NS) & 1); };
    auto midp = [&](int j) { return mid + ((j - (k0 - 1)) & 1) * T2::MID_STAGE; };
    auto issue = [&](int q) {
        const uint32_t bar = bar0 + 8 * slot(q);
        float *st = inr + slot(q) * T2::IN_STAGE;
        mbar_expect_tx(bar, (T2::IN_STATE + T2::IN_COEF) * 4);
        tma_load_4d(smem_u32(st), &tm_in, x0 - 4, y0 - 2, q, 0, bar);
        if (HET) tma_load_4d(smem_u32(st + T2::IN_STATE), &tm_coef, x0 - 4, y0 - 1, q, 0, bar);
    };
    int next_issue = qb;
    auto refill = [&](int upto) {  // thread 0, after a barrier: stage planes up to `upto`
        if (tid == 0) {
            fence_proxy_async();
            for (; next_issue <= min(k1 + 1, upto); ++next_issue) issue(next_issue);
        }
    };
    if (tid == 0)
        for (; next_issue <= min(k1 + 1, qb + NS - 1); ++next_issue) issue(next_issue);
    bool ok = true;

    // Register blocking in z: the z-1 neighbours of an intermediate node
    // (input plane j-1) and of an output node (intermediate plane k-1) are the
    // centre values this thread read one plane earlier.
    float4 prev_in[RM][6], prev_mid[RO][6], coef_cur[RO][2], coef_next[RO][2] = {};

    auto load_prev_in = [&](int j) {  // input plane j at this thread's intermediate groups
        const float *sc = inr + slot(j) * T2::IN_STAGE;
#pragma unroll
        for (int rr = 0; rr < RM; ++rr) {
            const int gi = tid + rr * T2::NT;
            if (gi >= T2::MID_GROUPS) continue;
            const int r = gi / T2::GXI, cg = gi % T2::GXI;
            const int oi = (r + 1) * T2::BX + 4 * cg;
#pragma unroll
            for (int f = 0; f < 6; ++f) prev_in[rr][f] = *reinterpret_cast<const float4 *>(sc + f * T2::IN_F + oi);
        }
    };
    auto load_out_coef = [&](int k, float4 (&dst)[RO][2]) {  // plane k's coefficients at the output groups
        const float *cs = inr + slot(k) * T2::IN_STAGE + T2::IN_STATE;
#pragma unroll
        for (int ro = 0; ro < RO; ++ro) {
            const int go = tid + ro * T2::NT;
            if (go >= T2::OUT_GROUPS) continue;
            const int r = go / T2::GX, gx = go % T2::GX;
            const int om = (r + 1) * T2::BX + 4 + 4 * gx;
            if (HET) {
                dst[ro][0] = *reinterpret_cast<const float4 *>(cs + om);
                dst[ro][1] = *reinterpret_cast<const float4 *>(cs + T2::MID_F + om);
            } else {
                dst[ro][0] = make_float4((float)p.A, (float)p.A, (float)p.A, (float)p.A);
                dst[ro][1] = make_float4((float)p.B, (float)p.B, (float)p.B, (float)p.B);
            }
        }
    };
    auto load_prev_mid = [&](int j) {  // intermediate plane j at this thread's output groups
        const float *mj = midp(j);
#pragma unroll
        for (int ro = 0; ro < RO; ++ro) {
            const int go = tid + ro * T2::NT;
            if (go >= T2::OUT_GROUPS) continue;
            const int r = go / T2::GX, gx = go % T2::GX;
            const int om = (r + 1) * T2::BX + 4 + 4 * gx;
#pragma unroll
            for (int f = 0; f < 6; ++f) prev_mid[ro][f] = *reinterpret_cast<const float4 *>(mj + f * T2::MID_F + om);
        }
    };

    // intermediate plane j (input plane j centre and j+1 staged, j-1 in prev_in)
    auto compute_mid = [&](int j) {
        float *mj = midp(j);
        const bool plane_in = (j >= 1 && j <= p.nz - 2);
        const float *sc = inr + slot(j) * T2::IN_STAGE;
        const float *sp = inr + slot(j + 1) * T2::IN_STAGE;
#pragma unroll
        for (int rr = 0; rr < RM; ++rr) {
            const int gi = tid + rr * T2::NT;
            if (gi >= T2::MID_GROUPS) continue;
            const int r = gi / T2::GXI, cg = gi % T2::GXI;
            const int y = y0 - 1 + r, x = x0 - 4 + 4 * cg;
            const int oi = (r + 1) * T2::BX + 4 * cg;  // input tile offset of this group
            const int om = r * T2::BX + 4 * cg;        // intermediate / coefficient tile offset
            const bool row_in = plane_in && y >= 1 && y <= p.ny - 2;
            bool m[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) m[e] = row_in && (x + e >= 1) && (x + e <= p.nx - 2);
            float4 A4, B4;
            if (HET) {
                A4 = *reinterpret_cast<const float4 *>(sc + T2::IN_STATE + om);
                B4 = *reinterpret_cast<const float4 *>(sc + T2::IN_STATE + T2::MID_F + om);
            } else {
                A4 = make_float4((float)p.A, (float)p.A, (float)p.A, (float)p.A);
                B4 = make_float4((float)p.B, (float)p.B, (float)p.B, (float)p.B);
            }
            float4 ctr[6], sum[6];
#pragma unroll
            for (int f = 0; f < 6; ++f) {
                const float *fc = sc + f * T2::IN_F + oi;
                const float4 c = *reinterpret_cast<const float4 *>(fc);
                const float4 ym = *reinterpret_cast<const float4 *>(fc - T2::BX);
                const float4 yp = *reinterpret_cast<const float4 *>(fc + T2::BX);
                const float4 zm = prev_in[rr][f];
                const float4 zp = *reinterpret_cast<const float4 *>(sp + f * T2::IN_F + oi);
                const float left = (cg == 0) ? 0.f : fc[-1];
                const float right = (cg == T2::GXI - 1) ? 0.f : fc[4];
                float4 s4;
                s4.x = kv_add(kv_add(kv_add(left, c.y), kv_add(ym.x, yp.x)), kv_add(zm.x, zp.x));
                s4.y = kv_add(kv_add(kv_add(c.x, c.z), kv_add(ym.y, yp.y)), kv_add(zm.y, zp.y));
                s4.z = kv_add(kv_add(kv_add(c.y, c.w), kv_add(ym.z, yp.z)), kv_add(zm.z, zp.z));
                s4.w = kv_add(kv_add(kv_add(c.z, right), kv_add(ym.w, yp.w)), kv_add(zm.w, zp.w));
                ctr[f] = c;
                sum[f] = s4;
                prev_in[rr][f] = c;
            }
#pragma unroll
            for (int comp = 0; comp < 3; ++comp) {
                float Fv[4] = {0.f, 0.f, 0.f, 0.f};
                if (g0 != 0.f) {
#pragma unroll
                    for (int e = 0; e < 4; ++e)
                        if (m[e]) Fv[e] = F[comp * p.Np + (long long)j * sz + (long long)y * sy + x + e];
                }
                const float4 u = ctr[comp], su = sum[comp], d = ctr[3 + comp], sd = sum[3 + comp];
                float4 uo, dn;
                kv_update(u.x, su.x, d.x, sd.x, A4.x, B4.x, g0, Fv[0], uo.x, dn.x);
                kv_update(u.y, su.y, d.y, sd.y, A4.y, B4.y, g0, Fv[1], uo.y, dn.y);
                kv_update(u.z, su.z, d.z, sd.z, A4.z, B4.z, g0, Fv[2], uo.z, dn.z);
                kv_update(u.w, su.w, d.w, sd.w, A4.w, B4.w, g0, Fv[3], uo.w, dn.w);
                if (!m[0]) uo.x = dn.x = 0.f;
                if (!m[1]) uo.y = dn.y = 0.f;
                if (!m[2]) uo.z = dn.z = 0.f;
                if (!m[3]) uo.w = dn.w = 0.f;
                *reinterpret_cast<float4 *>(mj + comp * T2::MID_F + om) = uo;
                *reinterpret_cast<float4 *>(mj + (3 + comp) * T2::MID_F + om) = dn;
            }
        }
    };

    // Prologue. Planes k0-2 .. k0+NS-3 are in flight. Each input stage is
    // released as soon as its centre values (and, for plane k, the output
    // groups' coefficients) are in registers.
    ok &= mbar_wait_bounded(bar0 + 8 * slot(qb), par(qb));
    load_prev_in(qb);
    __syncthreads();
    refill(qb + NS);
    ok &= mbar_wait_bounded(bar0 + 8 * slot(k0 - 1), par(k0 - 1));
    ok &= mbar_wait_bounded(bar0 + 8 * slot(k0), par(k0));
    compute_mid(k0 - 1);
    __syncthreads();
    refill(k0 - 1 + NS);
    ok &= mbar_wait_bounded(bar0 + 8 * slot(k0 + 1), par(k0 + 1));
    compute_mid(k0);
    load_out_coef(k0, coef_cur);
    __syncthreads();  // intermediate planes k0-1 and k0 complete
    load_prev_mid(k0 - 1);
    refill(k0 + NS);
    __syncthreads();  // plane k0-1's slot is read: the loop's first intermediate plane overwrites it

    for (int k = k0; k < k1; ++k) {
        ok &= mbar_wait_bounded(bar0 + 8 * slot(k + 2), par(k + 2));
        compute_mid(k + 1);  // into the slot of intermediate plane k-1 (now in prev_mid)
        if (k + 1 < k1) load_out_coef(k + 1, coef_next);
        __syncthreads();     // intermediate plane k+1 complete; input plane k+1 consumed
        refill(k + 1 + NS);
        // sensors of the intermediate step owned by this block (plane k)
        if (p.ns > 0 && step < p.cap) {
            const float *mk = midp(k);
            float *tr = reinterpret_cast<float *>(p.traces) + (size_t)step * p.ns * 3;
            for (int q = p.sens_off[k] + tid; q < p.sens_off[k + 1]; q += T2::NT) {
                const int s = p.sens_ord[q];
                const int i = p.sensors[3 * s], jj = p.sensors[3 * s + 1];
                if (i >= x0 && i < x0 + TX && jj >= y0 && jj < y0 + TY && jj <= p.ny - 2)
                    for (int comp = 0; comp < 3; ++comp)
                        tr[3 * s + comp] = mk[comp * T2::MID_F + (jj - y0 + 1) * T2::BX + (i - x0 + 4)];
            }
        }
        // final step of plane k from intermediate planes k-1 (registers), k, k+1
        const float *mc = midp(k);
        const float *mp = midp(k + 1);
#pragma unroll
        for (int ro = 0; ro < RO; ++ro) {
            const int go = tid + ro * T2::NT;
            if (go >= T2::OUT_GROUPS) continue;
            const int r = go / T2::GX, gx = go % T2::GX;
            const int y = y0 + r, x = x0 + 4 * gx;
            const int om = (r + 1) * T2::BX + 4 + 4 * gx;
            const float4 A4 = coef_cur[ro][0], B4 = coef_cur[ro][1];
            const bool row_ok = (y <= p.ny - 2) && (x < p.px);
            const bool m0 = (x >= 1) && (x <= p.nx - 2), m1 = (x + 1 <= p.nx - 2);
            const bool m2 = (x + 2 <= p.nx - 2), m3 = (x + 3 <= p.nx - 2);
            float4 ctr[6], sum[6];
#pragma unroll
            for (int f = 0; f < 6; ++f) {
                const float *fc = mc + f * T2::MID_F + om;
                const float4 c = *reinterpret_cast<const float4 *>(fc);
                const float4 ym = *reinterpret_cast<const float4 *>(fc - T2::BX);
                const float4 yp = *reinterpret_cast<const float4 *>(fc + T2::BX);
                const float4 zm = prev_mid[ro][f];
                const float4 zp = *reinterpret_cast<const float4 *>(mp + f * T2::MID_F + om);
                const float left = fc[-1], right = fc[4];
                float4 s4;
                s4.x = kv_add(kv_add(kv_add(left, c.y), kv_add(ym.x, yp.x)), kv_add(zm.x, zp.x));
                s4.y = kv_add(kv_add(kv_add(c.x, c.z), kv_add(ym.y, yp.y)), kv_add(zm.y, zp.y));
                s4.z = kv_add(kv_add(kv_add(c.y, c.w), kv_add(ym.z, yp.z)), kv_add(zm.z, zp.z));
                s4.w = kv_add(kv_add(kv_add(c.z, right), kv_add(ym.w, yp.w)), kv_add(zm.w, zp.w));
                ctr[f] = c;
                sum[f] = s4;
                prev_mid[ro][f] = c;
            }
            if (!row_ok) continue;
            const long long gbase = k * sz + (long long)y * sy + x;
#pragma unroll
            for (int comp = 0; comp < 3; ++comp) {
                float4 F4 = make_float4(0.f, 0.f, 0.f, 0.f);
                if (g1 != 0.f) F4 = __ldg(reinterpret_cast<const float4 *>(F + comp * p.Np + gbase));
                const float4 u = ctr[comp], su = sum[comp], d = ctr[3 + comp], sd = sum[3 + comp];
                float4 uo, dn;
                kv_update(u.x, su.x, d.x, sd.x, A4.x, B4.x, g1, F4.x, uo.x, dn.x);
                kv_update(u.y, su.y, d.y, sd.y, A4.y, B4.y, g1, F4.y, uo.y, dn.y);
                kv_update(u.z, su.z, d.z, sd.z, A4.z, B4.z, g1, F4.z, uo.z, dn.z);
                kv_update(u.w, su.w, d.w, sd.w, A4.w, B4.w, g1, F4.w, uo.w, dn.w);
                if (!m0) uo.x = dn.x = 0.f;
                if (!m1) uo.y = dn.y = 0.f;
                if (!m2) uo.z = dn.z = 0.f;
                if (!m3) uo.w = dn.w = 0.f;
                *reinterpret_cast<float4 *>(out + comp * p.Np + gbase) = uo;
                *reinterpret_cast<float4 *>(out + (3 + comp) * p.Np + gbase) = dn;
            }
        }
#pragma unroll
        for (int ro = 0; ro < RO; ++ro) {
            coef_cur[ro][0] = coef_next[ro][0];
            coef_cur[ro][1] = coef_next[ro][1];
        }
        __syncthreads();  // intermediate plane k is no longer read: its slot takes plane k+2
    }
    if (__syncthreads_or(!ok) && tid == 0) {
        atomicOr(reinterpret_cast<unsigned long long *>(&p.ctrl[kErrFlags]), 1ull);
        for (int q = qb; q < next_issue; ++q) mbar_wait_bounded(bar0 + 8 * slot(q), par(q));
    }
    step_epilogue_n<float>(out, p, step, 2);
}

// ---------------------------------------------------------------------------
// Two steps per sweep, one displacement component per block (variant 3).
//
// The pointwise operator couples the three components of u only through the
// shared coefficients, so a block can advance a single component c: it stages
// only (u_c, d_c) (two TMA boxes per plane, fields c and 3 + c of the state
// tensor) and the coefficient tile, a third of the state bytes of the
// three-component kernel. The smaller stages let two or three blocks share an
// SM, which is what the three-component two-step kernel lacks (one block of
// four warps per SM, bound by latency). Block b of the x dimension is tile
// b / 3, component b % 3, so the three component blocks of a tile run side by
// side and two of them read the tile's coefficients from L2. Per node and two
// steps the DRAM traffic is (u, d) read + write once (48 B) plus the
// coefficients once (8 B): 28 B per node and step instead of 56 B.
// The z march, the intermediate ring and the update order are those of
// k_step2_tma, so the result is bit for bit that of two single steps.
// ---------------------------------------------------------------------------
template <int TX, int TY, bool HET>
struct Tile2C {
    static constexpr int BX = TX + 8;
    static constexpr int BYI = TY + 4;
    static constexpr int BYM = TY + 2;
    static constexpr int IN_F = BX * BYI;
    static constexpr int MID_F = BX * BYM;
    static constexpr int IN_STATE = 2 * IN_F;                 // u_c, d_c
    static constexpr int IN_COEF = HET ? 2 * MID_F : 0;       // A', B' with a one-node ring
    static constexpr int IN_STAGE = (IN_STATE + IN_COEF + 31) / 32 * 32;
    static constexpr int MID_STAGE = (2 * MID_F + 31) / 32 * 32;
    static constexpr int GXI = BX / 4;
    static constexpr int MID_GROUPS = GXI * BYM;
    static constexpr int GX = TX / 4;
    static constexpr int OUT_GROUPS = GX * TY;
    static constexpr int NT = OUT_GROUPS;                     // one output group per thread
    static constexpr int RM = (MID_GROUPS + NT - 1) / NT;     // intermediate groups per thread
    static constexpr size_t smem(int ns) { return (size_t)(ns * IN_STAGE + 2 * MID_STAGE) * 4 + ns * 8; }
};

template <int TX, int TY, int NS, bool HET>
__global__ void __launch_bounds__(TX *TY / 4)
k_step2c_tma(const __grid_constant__ CUtensorMap tm_in, const __grid_constant__ CUtensorMap tm_coef,
             const float *__restrict__ F, float *__restrict__ out, StepParams p) {
    using T2 = Tile2C<TX, TY, HET>;
    constexpr int RM = T2::RM, NT = T2::NT;
    extern __shared__ __align__(128) float smem[];
    float *inr = smem;                                 // NS input stages
    float *mid = smem + NS * T2::IN_STAGE;             // 2 intermediate planes
    uint64_t *bars = reinterpret_cast<uint64_t *>(mid + 2 * T2::MID_STAGE);
    const uint32_t bar0 = smem_u32(bars);
    const int tid = threadIdx.x;
    const int comp = (int)(blockIdx.x % 3);
    const int x0 = (int)(blockIdx.x / 3) * TX, y0 = 1 + blockIdx.y * TY;
    const int k0 = 1 + blockIdx.z * p.zc;
    const int k1 = min(k0 + p.zc, p.nz - 1);  // output planes k0..k1-1
    const int qb = k0 - 2;                     // first staged input plane (may be -1)
    const long long step = __ldcg(&p.ctrl[kStep]);
    const float g0 = p.g_const_on ? p.g_const : (step < p.n_g) ? p.g[step] : 0.f;
    const float g1 = p.g_const_on ? p.g_const : (step + 1 < p.n_g) ? p.g[step + 1] : 0.f;
    const long long sy = p.px, sz = (long long)p.px * p.ny;
    const float *Fc = F + comp * p.Np;
    float *out_u = out + comp * p.Np, *out_d = out + (3 + comp) * p.Np;

    if (tid == 0) {
        for (int s = 0; s < NS; ++s) mbar_init(bar0 + 8 * s, 1);
        mbar_init_fence();
    }
    __syncthreads();
    auto slot = [&](int q) { return (q - qb) % NS; };
    auto par = [&](int q) { return (uint32_t)(((q - qb) / NS) & 1); };
    auto midp = [&](int j) { return mid + ((j - (k0 - 1)) & 1) * T2::MID_STAGE; };
    auto issue = [&](int q) {
        const uint32_t bar = bar0 + 8 * slot(q);
        float *st = inr + slot(q) * T2::IN_STAGE;
        mbar_expect_tx(bar, (T2::IN_STATE + T2::IN_COEF) * 4);
        tma_load_4d(smem_u32(st), &tm_in, x0 - 4, y0 - 2, q, comp, bar);
        tma_load_4d(smem_u32(st + T2::IN_F), &tm_in, x0 - 4, y0 - 2, q, 3 + comp, bar);
        if (HET) tma_load_4d(smem_u32(st + T2::IN_STATE), &tm_coef, x0 - 4, y0 - 1, q, 0, bar);
    };
    int next_issue = qb;
    auto refill = [&](int upto) {  // thread 0, after a barrier: stage planes up to `upto`
        if (tid == 0) {
            fence_proxy_async();
            for (; next_issue <= min(k1 + 1, upto); ++next_issue) issue(next_issue);
        }
    };
    if (tid == 0)
        for (; next_issue <= min(k1 + 1, qb + NS - 1); ++next_issue) issue(next_issue);
    bool ok = true;

    // z-1 neighbours in registers: input plane j-1 of this thread's
    // intermediate groups, intermediate plane k-1 of its output group.
    float4 prev_in[RM][2], prev_mid[2], coef_cur[2], coef_next[2] = {};
    const int ro_r = tid / T2::GX, ro_gx = tid % T2::GX;      // this thread's output group
    const int om_out = (ro_r + 1) * T2::BX + 4 + 4 * ro_gx;   // its offset in an intermediate plane

    auto load_prev_in = [&](int j) {
        const float *sc = inr + slot(j) * T2::IN_STAGE;
#pragma unroll
        for (int rr = 0; rr < RM; ++rr) {
            const int gi = tid + rr * NT;
            if (gi >= T2::MID_GROUPS) continue;
            const int r = gi / T2::GXI, cg = gi % T2::GXI;
            const int oi = (r + 1) * T2::BX + 4 * cg;
#pragma unroll
            for (int f = 0; f < 2; ++f) prev_in[rr][f] = *reinterpret_cast<const float4 *>(sc + f * T2::IN_F + oi);
        }
    };
    auto load_out_coef = [&](int k, float4 (&dst)[2]) {
        if (HET) {
            const float *cs = inr + slot(k) * T2::IN_STAGE + T2::IN_STATE;
            dst[0] = *reinterpret_cast<const float4 *>(cs + om_out);
            dst[1] = *reinterpret_cast<const float4 *>(cs + T2::MID_F + om_out);
        } else {
            dst[0] = make_float4((float)p.A, (float)p.A, (float)p.A, (float)p.A);
            dst[1] = make_float4((float)p.B, (float)p.B, (float)p.B, (float)p.B);
        }
    };
    auto load_prev_mid = [&](int j) {
        const float *mj = midp(j);
#pragma unroll
        for (int f = 0; f < 2; ++f) prev_mid[f] = *reinterpret_cast<const float4 *>(mj + f * T2::MID_F + om_out);
    };

    // intermediate plane j of component comp (input plane j centre and j+1
    // staged, j-1 in prev_in)
    auto compute_mid = [&](int j) {
        float *mj = midp(j);
        const bool plane_in = (j >= 1 && j <= p.nz - 2);
        const float *sc = inr + slot(j) * T2::IN_STAGE;
        const float *sp = inr + slot(j + 1) * T2::IN_STAGE;
#pragma unroll
        for (int rr = 0; rr < RM; ++rr) {
            const int gi = tid + rr * NT;
            if (gi >= T2::MID_GROUPS) continue;
            const int r = gi / T2::GXI, cg = gi % T2::GXI;
            const int y = y0 - 1 + r, x = x0 - 4 + 4 * cg;
            const int oi = (r + 1) * T2::BX + 4 * cg;
            const int om = r * T2::BX + 4 * cg;
            const bool row_in = plane_in && y >= 1 && y <= p.ny - 2;
            bool m[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) m[e] = row_in && (x + e >= 1) && (x + e <= p.nx - 2);
            float4 A4, B4;
            if (HET) {
                A4 = *reinterpret_cast<const float4 *>(sc + T2::IN_STATE + om);
                B4 = *reinterpret_cast<const float4 *>(sc + T2::IN_STATE + T2::MID_F + om);
            } else {
                A4 = make_float4((float)p.A, (float)p.A, (float)p.A, (float)p.A);
                B4 = make_float4((float)p.B, (float)p.B, (float)p.B, (float)p.B);
            }
            float4 ctr[2], sum[2];
#pragma unroll
            for (int f = 0; f < 2; ++f) {
                const float *fc = sc + f * T2::IN_F + oi;
                const float4 c = *reinterpret_cast<const float4 *>(fc);
                const float4 ym = *reinterpret_cast<const float4 *>(fc - T2::BX);
                const float4 yp = *reinterpret_cast<const float4 *>(fc + T2::BX);
                const float4 zm = prev_in[rr][f];
                const float4 zp = *reinterpret_cast<const float4 *>(sp + f * T2::IN_F + oi);
                const float left = (cg == 0) ? 0.f : fc[-1];
                const float right = (cg == T2::GXI - 1) ? 0.f : fc[4];
                float4 s4;
                s4.x = kv_add(kv_add(kv_add(left, c.y), kv_add(ym.x, yp.x)), kv_add(zm.x, zp.x));
                s4.y = kv_add(kv_add(kv_add(c.x, c.z), kv_add(ym.y, yp.y)), kv_add(zm.y, zp.y));
                s4.z = kv_add(kv_add(kv_add(c.y, c.w), kv_add(ym.z, yp.z)), kv_add(zm.z, zp.z));
                s4.w = kv_add(kv_add(kv_add(c.z, right), kv_add(ym.w, yp.w)), kv_add(zm.w, zp.w));
                ctr[f] = c;
                sum[f] = s4;
                prev_in[rr][f] = c;
            }
            float Fv[4] = {0.f, 0.f, 0.f, 0.f};
            if (g0 != 0.f) {
#pragma unroll
                for (int e = 0; e < 4; ++e)
                    if (m[e]) Fv[e] = Fc[(long long)j * sz + (long long)y * sy + x + e];
            }
            const float4 u = ctr[0], su = sum[0], d = ctr[1], sd = sum[1];
            float4 uo, dn;
            kv_update(u.x, su.x, d.x, sd.x, A4.x, B4.x, g0, Fv[0], uo.x, dn.x);
            kv_update(u.y, su.y, d.y, sd.y, A4.y, B4.y, g0, Fv[1], uo.y, dn.y);
            kv_update(u.z, su.z, d.z, sd.z, A4.z, B4.z, g0, Fv[2], uo.z, dn.z);
            kv_update(u.w, su.w, d.w, sd.w, A4.w, B4.w, g0, Fv[3], uo.w, dn.w);
            if (!m[0]) uo.x = dn.x = 0.f;
            if (!m[1]) uo.y = dn.y = 0.f;
            if (!m[2]) uo.z = dn.z = 0.f;
            if (!m[3]) uo.w = dn.w = 0.f;
            *reinterpret_cast<float4 *>(mj + om) = uo;
            *reinterpret_cast<float4 *>(mj + T2::MID_F + om) = dn;
        }
    };

    // Prologue, as in k_step2_tma.
    ok &= mbar_wait_bounded(bar0 + 8 * slot(qb), par(qb));
    load_prev_in(qb);
    __syncthreads();
    refill(qb + NS);
    ok &= mbar_wait_bounded(bar0 + 8 * slot(k0 - 1), par(k0 - 1));
    ok &= mbar_wait_bounded(bar0 + 8 * slot(k0), par(k0));
    compute_mid(k0 - 1);
    __syncthreads();
    refill(k0 - 1 + NS);
    ok &= mbar_wait_bounded(bar0 + 8 * slot(k0 + 1), par(k0 + 1));
    compute_mid(k0);
    load_out_coef(k0, coef_cur);
    __syncthreads();  // intermediate planes k0-1 and k0 complete
    load_prev_mid(k0 - 1);
    refill(k0 + NS);
    __syncthreads();  // plane k0-1's slot is read: the loop's first intermediate plane overwrites it

    const int y_out = y0 + ro_r, x_out = x0 + 4 * ro_gx;
    const bool row_ok = (y_out <= p.ny - 2) && (x_out < p.px);
    const bool m0 = (x_out >= 1) && (x_out <= p.nx - 2), m1 = (x_out + 1 <= p.nx - 2);
    const bool m2 = (x_out + 2 <= p.nx - 2), m3 = (x_out + 3 <= p.nx - 2);
    for (int k = k0; k < k1; ++k) {
        ok &= mbar_wait_bounded(bar0 + 8 * slot(k + 2), par(k + 2));
        compute_mid(k + 1);  // into the slot of intermediate plane k-1 (now in prev_mid)
        if (k + 1 < k1) load_out_coef(k + 1, coef_next);
        __syncthreads();     // intermediate plane k+1 complete; input plane k+1 consumed
        refill(k + 1 + NS);
        // sensors of the intermediate step owned by this block (plane k, component comp)
        if (p.ns > 0 && step < p.cap) {
            const float *mk = midp(k);
            float *tr = reinterpret_cast<float *>(p.traces) + (size_t)step * p.ns * 3;
            for (int q = p.sens_off[k] + tid; q < p.sens_off[k + 1]; q += NT) {
                const int s = p.sens_ord[q];
                const int i = p.sensors[3 * s], jj = p.sensors[3 * s + 1];
                if (i >= x0 && i < x0 + TX && jj >= y0 && jj < y0 + TY && jj <= p.ny - 2)
                    tr[3 * s + comp] = mk[(jj - y0 + 1) * T2::BX + (i - x0 + 4)];
            }
        }
        // final step of plane k from intermediate planes k-1 (registers), k, k+1
        const float *mc = midp(k);
        const float *mp = midp(k + 1);
        float4 ctr[2], sum[2];
#pragma unroll
        for (int f = 0; f < 2; ++f) {
            const float *fc = mc + f * T2::MID_F + om_out;
            const float4 c = *reinterpret_cast<const float4 *>(fc);
            const float4 ym = *reinterpret_cast<const float4 *>(fc - T2::BX);
            const float4 yp = *reinterpret_cast<const float4 *>(fc + T2::BX);
            const float4 zm = prev_mid[f];
            const float4 zp = *reinterpret_cast<const float4 *>(mp + f * T2::MID_F + om_out);
            const float left = fc[-1], right = fc[4];
            float4 s4;
            s4.x = kv_add(kv_add(kv_add(left, c.y), kv_add(ym.x, yp.x)), kv_add(zm.x, zp.x));
            s4.y = kv_add(kv_add(kv_add(c.x, c.z), kv_add(ym.y, yp.y)), kv_add(zm.y, zp.y));
            s4.z = kv_add(kv_add(kv_add(c.y, c.w), kv_add(ym.z, yp.z)), kv_add(zm.z, zp.z));
            s4.w = kv_add(kv_add(kv_add(c.z, right), kv_add(ym.w, yp.w)), kv_add(zm.w, zp.w));
            ctr[f] = c;
            sum[f] = s4;
            prev_mid[f] = c;
        }
        if (row_ok) {
            const long long gbase = k * sz + (long long)y_out * sy + x_out;
            float4 F4 = make_float4(0.f, 0.f, 0.f, 0.f);
            if (g1 != 0.f) F4 = __ldg(reinterpret_cast<const float4 *>(Fc + gbase));
            const float4 A4 = coef_cur[0], B4 = coef_cur[1];
            const float4 u = ctr[0], su = sum[0], d = ctr[1], sd = sum[1];
            float4 uo, dn;
            kv_update(u.x, su.x, d.x, sd.x, A4.x, B4.x, g1, F4.x, uo.x, dn.x);
            kv_update(u.y, su.y, d.y, sd.y, A4.y, B4.y, g1, F4.y, uo.y, dn.y);
            kv_update(u.z, su.z, d.z, sd.z, A4.z, B4.z, g1, F4.z, uo.z, dn.z);
            kv_update(u.w, su.w, d.w, sd.w, A4.w, B4.w, g1, F4.w, uo.w, dn.w);
            if (!m0) uo.x = dn.x = 0.f;
            if (!m1) uo.y = dn.y = 0.f;
            if (!m2) uo.z = dn.z = 0.f;
            if (!m3) uo.w = dn.w = 0.f;
            *reinterpret_cast<float4 *>(out_u + gbase) = uo;
            *reinterpret_cast<float4 *>(out_d + gbase) = dn;
        }
        coef_cur[0] = coef_next[0];
        coef_cur[1] = coef_next[1];
        __syncthreads();  // intermediate plane k is no longer read: its slot takes plane k+2
    }
    if (__syncthreads_or(!ok) && tid == 0) {
        atomicOr(reinterpret_cast<unsigned long long *>(&p.ctrl[kErrFlags]), 1ull);
        for (int q = qb; q < next_issue; ++q) mbar_wait_bounded(bar0 + 8 * slot(q), par(q));
    }
    step_epilogue_n<float>(out, p, step, 2);
}

// ---------------------------------------------------------------------------
// Two steps per sweep, one component per block, balanced (variant 4).
//
// Variant 3 computes the intermediate step on (TX + 8) x (TY + 2) nodes in
// groups of four, (TX / 4 + 2) (TY + 2) groups for TX TY / 4 threads, so some
// warps take two groups and the rest wait at the barrier. Here the tile is
// TX x 14: the intermediate plane's 16 rows of TX / 4 groups take one group
// per thread (16 TX / 4 threads) and one more warp computes the two halo
// columns x0 - 1 and x0 + TX of the 16 rows (one node per lane), the only
// halo nodes the second step reads. The intermediate planes rotate through
// three buffers, so one barrier per plane suffices: the buffer written at
// plane k + 1 was last read by the second step of plane k - 1, before the
// barrier of plane k. The input ring needs two stages at least (planes k + 1
// and k + 2 are read at plane k; plane k + 3 is copied into the slot of k + 1
// after the barrier). The neighbour sums and the update run on pairs of nodes
// (packed FP32; each lane rounds as the scalar operation does) in the order
// of kv_update, so the result is bit for bit that of two single steps.
//
// The kernel is bound by the shared-memory pipe, so it reads as little of it
// as it can. The second step of a group runs on the thread that computed the
// same four intermediate nodes: their planes k - 1, k and k + 1 (the z
// neighbours and the centre) stay in its registers, and only the y
// neighbours come from the buffer. The input plane below the centre stays in
// registers too. The x neighbours beyond a group are the neighbouring lanes'
// values (warp shuffles); the first and last group of a row read the tile's
// halo column in one load that the other lanes aim at one broadcast word.
// The three planes of a register set rotate, unrolled by three.
// ---------------------------------------------------------------------------
template <int TX, bool HET>
struct Tile2B {
    static constexpr int TY = 14;                              // output rows
    static constexpr int GX = TX / 4;                          // groups of four nodes per row
    static constexpr int BX = TX + 8;                          // staged row: x from x0 - 4
    static constexpr int BYI = TY + 4;                         // input rows: y from y0 - 2
    static constexpr int BYM = TY + 2;                         // intermediate rows: y from y0 - 1
    static constexpr int IN_F = (BX * BYI + 31) / 32 * 32;     // field tile, padded: every TMA
                                                               // destination on a 128-byte boundary
    static constexpr int MID_F = BX * BYM;                     // (BYM = 16: a 128-byte multiple)
    static constexpr int IN_STATE = 2 * IN_F;                  // u_c, d_c
    static constexpr int IN_COEF = HET ? 2 * MID_F : 0;        // A', B'
    static constexpr int IN_STAGE = (IN_STATE + IN_COEF + 31) / 32 * 32;
    static constexpr int TX_BYTES = (2 * BX * BYI + IN_COEF) * 4;  // bytes the copies of a stage deliver
    static constexpr int MID_STAGE = (2 * MID_F + 31) / 32 * 32;
    static constexpr int NMID = GX * BYM;                      // intermediate groups: one per thread
    static constexpr int NOUT = GX * TY;                       // output groups
    static constexpr int NT = NMID + 32;                       // + the halo-column warp
    static constexpr size_t smem(int ns) { return (size_t)(ns * IN_STAGE + 3 * MID_STAGE) * 4 + ns * 8; }
    static_assert(2 * BYM == 32, "one lane per halo node of the 16 intermediate rows");
    static_assert((MID_F * 4) % 128 == 0 && (IN_F * 4) % 128 == 0, "TMA destinations on 128-byte boundaries");
};

__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ float2 f2lo(const float4 &v) { return make_float2(v.x, v.y); }
__device__ __forceinline__ float2 f2hi(const float4 &v) { return make_float2(v.z, v.w); }

// Neighbour sums ((xm + xp) + (ym + yp)) + (zm + zp) of four consecutive
// nodes (left / right: the x neighbours beyond the group), as two pairs. The
// x sums straddle the pairs of the group, so they are formed one node at a
// time (into fresh registers that pair up without moves).
__device__ __forceinline__ void nbsum4(const float4 &c, float left, float right, const float4 &ym,
                                       const float4 &yp, const float4 &zm, const float4 &zp, float2 &s01,
                                       float2 &s23) {
    const float2 x01 = f2(__fadd_rn(left, c.y), __fadd_rn(c.x, c.z));
    const float2 x23 = f2(__fadd_rn(c.y, c.w), __fadd_rn(c.z, right));
    s01 = __fadd2_rn(__fadd2_rn(x01, __fadd2_rn(f2lo(ym), f2lo(yp))), __fadd2_rn(f2lo(zm), f2lo(zp)));
    s23 = __fadd2_rn(__fadd2_rn(x23, __fadd2_rn(f2hi(ym), f2hi(yp))), __fadd2_rn(f2hi(zm), f2hi(zp)));
}

// kv_update on a pair of nodes.
__device__ __forceinline__ void kv_update2(float2 u, float2 su, float2 d, float2 sd, float2 A, float2 B, float2 g,
                                           float2 F, float2 &u_out, float2 &d_out) {
    const float2 m6 = f2(-6.f, -6.f);
    const float2 lu = __ffma2_rn(m6, u, su);
    const float2 ld = __ffma2_rn(m6, d, sd);
    float2 dn = __ffma2_rn(g, F, d);
    dn = __ffma2_rn(B, ld, dn);
    dn = __ffma2_rn(A, lu, dn);
    d_out = dn;
    u_out = __fadd2_rn(u, dn);
}

template <int TX, int NS, bool HET>
__global__ void __launch_bounds__(Tile2B<TX, HET>::NT, TX == 128 ? 1 : 2)
k_step2b_tma(const __grid_constant__ CUtensorMap tm_in, const __grid_constant__ CUtensorMap tm_coef,
             const float *__restrict__ F, float *__restrict__ out, StepParams p) {
    using T2 = Tile2B<TX, HET>;
    constexpr int TY = T2::TY, GX = T2::GX, BX = T2::BX;
    extern __shared__ __align__(128) float smem[];
    float *inr = smem;                                 // NS input stages
    float *mid = smem + NS * T2::IN_STAGE;             // 3 intermediate planes
    const uint32_t bar0 = smem_u32(mid + 3 * T2::MID_STAGE);
    const int tid = threadIdx.x;
    const int comp = (int)(blockIdx.x % 3);
    const int x0 = (int)(blockIdx.x / 3) * TX, y0 = 1 + blockIdx.y * TY;
    const int k0 = 1 + blockIdx.z * p.zc;
    const int k1 = min(k0 + p.zc, p.nz - 1);  // output planes k0..k1-1
    const int qb = k0 - 2;                     // first staged input plane (may be -1)
    const long long step = __ldcg(&p.ctrl[kStep]);
    const float g0 = p.g_const_on ? p.g_const : (step < p.n_g) ? p.g[step] : 0.f;
    const float g1 = p.g_const_on ? p.g_const : (step + 1 < p.n_g) ? p.g[step + 1] : 0.f;
    const long long sy = p.px, sz = (long long)p.px * p.ny;
    const float *Fc = F + comp * p.Np;
    float *out_u = out + comp * p.Np, *out_d = out + (3 + comp) * p.Np;

    if (tid == 0) {
        for (int s = 0; s < NS; ++s) mbar_init(bar0 + 8 * s, 1);
        mbar_init_fence();
    }
    __syncthreads();
    auto slot = [&](int q) { return (int)((unsigned)(q - qb) % NS); };
    auto par = [&](int q) { return ((unsigned)(q - qb) / NS) & 1u; };
    auto issue_to = [&](int q, int sl) {  // plane q into stage slot sl
        const uint32_t bar = bar0 + 8 * sl;
        float *st = inr + sl * T2::IN_STAGE;
        mbar_expect_tx(bar, T2::TX_BYTES);
        tma_load_4d(smem_u32(st), &tm_in, x0 - 4, y0 - 2, q, comp, bar);
        tma_load_4d(smem_u32(st + T2::IN_F), &tm_in, x0 - 4, y0 - 2, q, 3 + comp, bar);
        if (HET) tma_load_4d(smem_u32(st + T2::IN_STATE), &tm_coef, x0 - 4, y0 - 1, q, 0, bar);
    };
    int next_issue = qb;
    auto refill = [&](int upto) {  // thread 0, after a barrier: stage planes up to `upto`
        if (tid == 0) {
            fence_proxy_async();
            for (; next_issue <= min(k1 + 1, upto); ++next_issue) issue_to(next_issue, slot(next_issue));
        }
    };
    if (tid == 0)
        for (; next_issue <= min(k1 + 1, qb + NS - 1); ++next_issue) issue_to(next_issue, slot(next_issue));
    bool ok = true;

    // Roles. A thread of the group warps owns four intermediate nodes x ..
    // x+3 of row mr and, for 1 <= mr <= TY, the second step of the same four
    // nodes (they lie in output row mr - 1). The last warp owns the
    // intermediate halo nodes x0 - 1 and x0 + TX of the 16 rows (one a lane).
    const int warp = __shfl_sync(0xffffffffu, tid >> 5, 0);
    const bool grp = warp < T2::NMID / 32;
    const int mr = grp ? tid / GX : (tid - T2::NMID) >> 1;
    const int mc = tid % GX;
    const int mcol = grp ? 4 + 4 * mc : ((tid & 1) ? 4 + TX : 3);  // staged column
    const int yr = y0 - 1 + mr, xr = x0 - 4 + mcol;                 // global row, first column
    const int oi = (mr + 1) * BX + mcol;  // in an input field tile
    const int om = mr * BX + mcol;        // in an intermediate plane (and the coefficient tile)
    const bool mrow = yr >= 1 && yr <= p.ny - 2;
    const bool mm0 = mrow && xr >= 1 && xr <= p.nx - 2, mm1 = mrow && xr + 1 <= p.nx - 2,
               mm2 = mrow && xr + 2 <= p.nx - 2, mm3 = mrow && xr + 3 <= p.nx - 2;
    const bool mload = mrow && xr >= 0 && xr < p.px;  // force row inside the pitched array
    const float *Fm = Fc + (long long)yr * sy + xr;
    const bool row_ok = grp && mr >= 1 && mr <= TY && yr <= p.ny - 2 && xr < p.px;  // output written
    // no node of the block's intermediate tile (x0 - 1 .. x0 + TX, y0 - 1 ..
    // y0 + TY) on the boundary: the masks are all true off the end planes
    const bool inner = x0 >= 2 && x0 + TX <= p.nx - 2 && y0 >= 2 && y0 + TY <= p.ny - 2;
    const float2 Ah = f2(p.Af, p.Af), Bh = f2(p.Bf, p.Bf);
    // Edge words read without branches: the first group of a row reads its
    // left neighbour, the last group its right one (a lane is at most one of
    // them), every other lane word 0 of the tile (one broadcast word on bank
    // 0, which no edge word shares), so each such load is one shared-memory
    // wavefront. Second step: lanes without an output row take row 1 as
    // their centre, inside the plane.
    const int e1 = mc == 0 ? oi - 1 : mc == GX - 1 ? oi + 4 : 0;
    const int e2 = !row_ok ? 0 : mc == 0 ? om - 1 : mc == GX - 1 ? om + 4 : 0;
    const int oc2 = row_ok ? om : BX;

    auto stage = [&](int q) { return inr + slot(q) * T2::IN_STAGE; };
    // own centre value(s) of the input plane staged at sc
    auto load_in = [&](const float *sc, float4 (&v)[2]) {
        if (grp) {
            v[0] = *reinterpret_cast<const float4 *>(sc + oi);
            v[1] = *reinterpret_cast<const float4 *>(sc + T2::IN_F + oi);
        } else {
            v[0].x = sc[oi];
            v[1].x = sc[T2::IN_F + oi];
        }
    };

    // Intermediate plane j into mj. The own nodes of input plane j-1 (zm) are
    // in registers; plane j (the centre, kept in c for the next plane) and
    // j+1 are read from the stages sc and sp, the y neighbours from sc, the x
    // neighbours beyond the group from the neighbouring lanes (at the tile's
    // halo columns, from sc). Own results, as stored, into r; own
    // coefficients into cf.
    auto compute_mid = [&](const float *sc, const float *sp, float *mj, int j, const float4 (&zm)[2],
                           float4 (&c)[2], float4 (&r)[2], float4 (&cf)[2]) {
        const bool pin = j >= 1 && j <= p.nz - 2;
        if (grp) {
            float2 s01[2], s23[2];
#pragma unroll
            for (int f = 0; f < 2; ++f) {
                const float *sf = sc + f * T2::IN_F, *fc = sf + oi;
                c[f] = *reinterpret_cast<const float4 *>(fc);
                const float ew = sf[e1];
                float left = __shfl_up_sync(0xffffffffu, c[f].w, 1);
                float right = __shfl_down_sync(0xffffffffu, c[f].x, 1);
                left = mc == 0 ? ew : left;
                right = mc == GX - 1 ? ew : right;
                const float4 ym = *reinterpret_cast<const float4 *>(fc - BX);
                const float4 yp = *reinterpret_cast<const float4 *>(fc + BX);
                const float4 zp = *reinterpret_cast<const float4 *>(sp + f * T2::IN_F + oi);
                nbsum4(c[f], left, right, ym, yp, zm[f], zp, s01[f], s23[f]);
            }
            float2 A01 = Ah, A23 = Ah, B01 = Bh, B23 = Bh;
            if (HET) {
                cf[0] = *reinterpret_cast<const float4 *>(sc + T2::IN_STATE + om);
                cf[1] = *reinterpret_cast<const float4 *>(sc + T2::IN_STATE + T2::MID_F + om);
                A01 = f2lo(cf[0]);
                A23 = f2hi(cf[0]);
                B01 = f2lo(cf[1]);
                B23 = f2hi(cf[1]);
            }
            float4 F4 = make_float4(0.f, 0.f, 0.f, 0.f);
            if (g0 != 0.f && pin && mload) F4 = __ldg(reinterpret_cast<const float4 *>(Fm + (long long)j * sz));
            const float2 g = f2(g0, g0);
            float2 u01, d01, u23, d23;
            kv_update2(f2lo(c[0]), s01[0], f2lo(c[1]), s01[1], A01, B01, g, f2lo(F4), u01, d01);
            kv_update2(f2hi(c[0]), s23[0], f2hi(c[1]), s23[1], A23, B23, g, f2hi(F4), u23, d23);
            if (inner && pin) {  // block-uniform: no node of the plane on the boundary
                r[0] = make_float4(u01.x, u01.y, u23.x, u23.y);
                r[1] = make_float4(d01.x, d01.y, d23.x, d23.y);
            } else {
                const bool q0 = pin && mm0, q1 = pin && mm1, q2 = pin && mm2, q3 = pin && mm3;
                r[0] = make_float4(q0 ? u01.x : 0.f, q1 ? u01.y : 0.f, q2 ? u23.x : 0.f, q3 ? u23.y : 0.f);
                r[1] = make_float4(q0 ? d01.x : 0.f, q1 ? d01.y : 0.f, q2 ? d23.x : 0.f, q3 ? d23.y : 0.f);
            }
            *reinterpret_cast<float4 *>(mj + om) = r[0];
            *reinterpret_cast<float4 *>(mj + T2::MID_F + om) = r[1];
        } else {
            float sv[2];
#pragma unroll
            for (int f = 0; f < 2; ++f) {
                const float *fc = sc + f * T2::IN_F + oi;
                c[f].x = fc[0];
                sv[f] = kv_add(kv_add(kv_add(fc[-1], fc[1]), kv_add(fc[-BX], fc[BX])), kv_add(zm[f].x, sp[f * T2::IN_F + oi]));
            }
            const float A = HET ? sc[T2::IN_STATE + om] : p.Af;
            const float B = HET ? sc[T2::IN_STATE + T2::MID_F + om] : p.Bf;
            const bool q0 = pin && mm0;
            const float Fv = (g0 != 0.f && q0) ? Fm[(long long)j * sz] : 0.f;
            float uo, dn;
            kv_update(c[0].x, sv[0], c[1].x, sv[1], A, B, g0, Fv, uo, dn);
            mj[om] = q0 ? uo : 0.f;
            mj[T2::MID_F + om] = q0 ? dn : 0.f;
        }
    };

    // Second step of plane k on the own nodes of a group thread with an
    // output row: intermediate planes k-1 (mz), k (mcen) and k+1 (mn) of these
    // nodes are in registers; the y neighbours and the halo columns come from
    // plane k's buffer mk, the x neighbours beyond the group from the
    // neighbouring lanes.
    auto second = [&](int k, const float *mk, const float4 (&mz)[2], const float4 (&mcen)[2],
                      const float4 (&mn)[2], const float4 (&cf)[2]) {
        if (!grp) return;  // warp-uniform
        float2 s01[2], s23[2];
#pragma unroll
        for (int f = 0; f < 2; ++f) {
            const float *sf = mk + f * T2::MID_F;
            const float ew = sf[e2];
            float left = __shfl_up_sync(0xffffffffu, mcen[f].w, 1);
            float right = __shfl_down_sync(0xffffffffu, mcen[f].x, 1);
            left = mc == 0 ? ew : left;
            right = mc == GX - 1 ? ew : right;
            const float4 ym = *reinterpret_cast<const float4 *>(sf + oc2 - BX);
            const float4 yp = *reinterpret_cast<const float4 *>(sf + oc2 + BX);
            nbsum4(mcen[f], left, right, ym, yp, mz[f], mn[f], s01[f], s23[f]);
        }
        const long long gbase = k * sz + (long long)yr * sy + xr;
        float4 F4 = make_float4(0.f, 0.f, 0.f, 0.f);
        if (g1 != 0.f && row_ok) F4 = __ldg(reinterpret_cast<const float4 *>(Fc + gbase));
        const float2 A01 = HET ? f2lo(cf[0]) : Ah, A23 = HET ? f2hi(cf[0]) : Ah;
        const float2 B01 = HET ? f2lo(cf[1]) : Bh, B23 = HET ? f2hi(cf[1]) : Bh;
        const float2 g = f2(g1, g1);
        float2 u01, d01, u23, d23;
        kv_update2(f2lo(mcen[0]), s01[0], f2lo(mcen[1]), s01[1], A01, B01, g, f2lo(F4), u01, d01);
        kv_update2(f2hi(mcen[0]), s23[0], f2hi(mcen[1]), s23[1], A23, B23, g, f2hi(F4), u23, d23);
        if (!row_ok) return;
        if (inner) {
            *reinterpret_cast<float4 *>(out_u + gbase) = make_float4(u01.x, u01.y, u23.x, u23.y);
            *reinterpret_cast<float4 *>(out_d + gbase) = make_float4(d01.x, d01.y, d23.x, d23.y);
        } else {
            *reinterpret_cast<float4 *>(out_u + gbase) =
                make_float4(mm0 ? u01.x : 0.f, mm1 ? u01.y : 0.f, mm2 ? u23.x : 0.f, mm3 ? u23.y : 0.f);
            *reinterpret_cast<float4 *>(out_d + gbase) =
                make_float4(mm0 ? d01.x : 0.f, mm1 ? d01.y : 0.f, mm2 ? d23.x : 0.f, mm3 ? d23.y : 0.f);
        }
    };

    // Own nodes in registers: input planes (IA, IB: k and k+1), intermediate
    // planes as stored (M*: k-1, k, k+1), coefficients of planes k (Ccur) and
    // k+1 (Cnext). The sets rotate, unrolled by three below.
    float4 IA[2] = {}, IB[2] = {}, M0[2] = {}, M1[2] = {}, M2[2] = {}, Ccur[2] = {}, Cnext[2] = {};
    float *const mb0 = mid, *const mb1 = mid + T2::MID_STAGE, *const mb2 = mid + 2 * T2::MID_STAGE;

    // Prologue: input plane k0-2 into registers, intermediate planes k0-1
    // and k0 (buffers mb0, mb1); input plane k0 left in IA.
    ok &= mbar_wait_bounded(bar0 + 8 * slot(qb), par(qb));
    load_in(stage(qb), IA);
    __syncthreads();
    refill(qb + NS);
    ok &= mbar_wait_bounded(bar0 + 8 * slot(k0 - 1), par(k0 - 1));
    ok &= mbar_wait_bounded(bar0 + 8 * slot(k0), par(k0));
    compute_mid(stage(k0 - 1), stage(k0), mb0, k0 - 1, IA, IB, M0, Cnext);
    __syncthreads();
    refill(k0 - 1 + NS);
    ok &= mbar_wait_bounded(bar0 + 8 * slot(k0 + 1), par(k0 + 1));
    compute_mid(stage(k0), stage(k0 + 1), mb1, k0, IB, IA, M1, Ccur);
    __syncthreads();  // intermediate planes k0-1 and k0 complete, input plane k0 consumed
    refill(k0 + NS);
    // sensors of the intermediate step: only a block whose column holds one
    // looks them up plane by plane
    bool sens = p.ns > 0 && step < p.cap;
    if (sens) {
        int hit = 0;
        for (int s = tid; s < p.ns; s += T2::NT) {
            const int i = p.sensors[3 * s], jj = p.sensors[3 * s + 1], kk = p.sensors[3 * s + 2];
            hit |= i >= x0 && i < x0 + TX && jj >= y0 && jj < y0 + TY && jj <= p.ny - 2 && kk >= k0 && kk < k1;
        }
        sens = __syncthreads_or(hit) != 0;
    }
    int so_k = sens ? __ldg(p.sens_off + k0) : 0;  // sensors of plane k: sens_ord[so_k .. so_k1)

    // one plane k: input plane k (iz) in registers, k+1 into icn (stage
    // slots s1 of plane k+1 and s2, parity par2, of plane k+2); intermediate
    // planes k-1 (mz), k (mcn) in registers, k+1 into mnx and its buffer mnb;
    // plane k's buffer mk; coefficients of plane k (ccur), plane k+1 into cnx.
    // Thread 0 then stages plane k+1+NS into slot s1.
    auto body = [&](int k, const float4 (&iz)[2], float4 (&icn)[2], const float4 (&mz)[2],
                    const float4 (&mcn)[2], float4 (&mnx)[2], const float *mk, float *mnb, int s1, int s2,
                    uint32_t par2, const float4 (&ccur)[2], float4 (&cnx)[2]) {
        ok &= mbar_wait_bounded(bar0 + 8 * s2, par2);
        compute_mid(inr + s1 * T2::IN_STAGE, inr + s2 * T2::IN_STAGE, mnb, k + 1, iz, icn, mnx, cnx);
        __syncthreads();  // intermediate plane k+1 complete; input plane k+1 consumed
        if (tid == 0 && k + 1 + NS <= k1 + 1) {
            fence_proxy_async();
            issue_to(k + 1 + NS, s1);
        }
        if (sens) {  // sensors of the intermediate step owned by this block (plane k, component comp)
            const int so_k1 = __ldg(p.sens_off + k + 1);
            float *tr = reinterpret_cast<float *>(p.traces) + (size_t)step * p.ns * 3;
            for (int q = so_k + tid; q < so_k1; q += T2::NT) {
                const int s = p.sens_ord[q];
                const int i = p.sensors[3 * s], jj = p.sensors[3 * s + 1];
                if (i >= x0 && i < x0 + TX && jj >= y0 && jj < y0 + TY && jj <= p.ny - 2)
                    tr[3 * s + comp] = mk[(jj - y0 + 1) * BX + (i - x0 + 4)];
            }
            so_k = so_k1;
        }
        second(k, mk, mz, mcn, mnx, ccur);
    };
    // Three planes per round (plane k0-1 in mb0, k0 in mb1 as set up above);
    // the input and coefficient sets alternate and are realigned once a
    // round. With three stages the slots of a round are fixed: (0, 1), (1, 2),
    // (2, 0).
    auto realign = [&]() {
        IA[0] = IB[0];
        IA[1] = IB[1];
        Ccur[0] = Cnext[0];
        Ccur[1] = Cnext[1];
    };
    if constexpr (NS == 3) {
        uint32_t rp = 0;  // parity of round r = (k - k0) / 3
        for (int k = k0; k < k1; k += 3) {
            body(k, IA, IB, M0, M1, M2, mb1, mb2, 0, 1, rp ^ 1u, Ccur, Cnext);
            if (k + 1 < k1) body(k + 1, IB, IA, M1, M2, M0, mb2, mb0, 1, 2, rp ^ 1u, Cnext, Ccur);
            if (k + 2 < k1) body(k + 2, IA, IB, M2, M0, M1, mb0, mb1, 2, 0, rp, Ccur, Cnext);
            realign();
            rp ^= 1u;
        }
    } else {
        int s1 = slot(k0 + 1), s2 = slot(k0 + 2);  // slots of planes k+1 and k+2
        uint32_t par2 = par(k0 + 2);
        auto advance = [&]() {
            s1 = s2;
            if (++s2 == NS) {
                s2 = 0;
                par2 ^= 1u;
            }
        };
        for (int k = k0; k < k1; k += 3) {
            body(k, IA, IB, M0, M1, M2, mb1, mb2, s1, s2, par2, Ccur, Cnext);
            advance();
            if (k + 1 < k1) {
                body(k + 1, IB, IA, M1, M2, M0, mb2, mb0, s1, s2, par2, Cnext, Ccur);
                advance();
            }
            if (k + 2 < k1) {
                body(k + 2, IA, IB, M2, M0, M1, mb0, mb1, s1, s2, par2, Ccur, Cnext);
                advance();
            }
            realign();
        }
    }
    next_issue = k1 + 2;  // every plane up to k1 + 1 has been staged
    if (__syncthreads_or(!ok) && tid == 0) {
        atomicOr(reinterpret_cast<unsigned long long *>(&p.ctrl[kErrFlags]), 1ull);
        for (int q = max(qb, next_issue - NS); q < next_issue; ++q) mbar_wait_bounded(bar0 + 8 * slot(q), par(q));
    }
    step_epilogue_n<float>(out, p, step, 2);
}

// ---------------------------------------------------------------------------
// Small kernels: medium fold, initial velocity
// ---------------------------------------------------------------------------
// Grid: (ceil(px/128), ny, nz), block 128.
// div = 0: coef = [A', B'] = [dt^2 G/(rho dx^2), dt eta/(rho dx^2)] (pointwise operator);
// div = 1: coef = [m, e, 1/rho] = [dt^2 G/dx^2, dt eta/dx^2, 1/rho] (divergence form).
template <typename T>
__global__ void k_fold(const float *__restrict__ G, const float *__restrict__ rho,
                       const float *__restrict__ eta, double Gs, double rhos, double etas,
                       T *__restrict__ coef, T *__restrict__ S, long long Np, int nx, int px,
                       int ny, double dt, double dx, int div) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= px) return;
    const long long c = ((long long)blockIdx.z * ny + blockIdx.y) * px + i;
    if (i >= nx) {  // row padding
        coef[c] = T(0);
        coef[Np + c] = T(0);
        if (div) coef[2 * Np + c] = T(0);
        S[c] = T(0);
        return;
    }
    const double g = G ? (double)G[c] : Gs;
    const double r = rho ? (double)rho[c] : rhos;
    const double e = eta ? (double)eta[c] : etas;
    const double inv = 1.0 / (dx * dx);
    const double rr = 1.0 / r;  // one FP64 division per node
    if (div) {
        coef[c] = T(dt * dt * g * inv);
        coef[Np + c] = T(dt * e * inv);
        coef[2 * Np + c] = T(rr);
    } else {
        coef[c] = T(dt * dt * inv * g * rr);
        coef[Np + c] = T(dt * inv * e * rr);
    }
    S[c] = T(dt * dt * rr);
}

template <typename T>
__global__ void k_init_velocity(const float *__restrict__ v, T *__restrict__ st, int nx, int ny,
                                int nz, int px, long long Np, double dt) {
    const long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (c >= Np) return;
    const int i = (int)(c % px);
    const long long r = c / px;
    const int j = (int)(r % ny);
    const int k = (int)(r / ny);
    const bool in = i >= 1 && i <= nx - 2 && j >= 1 && j <= ny - 2 && k >= 1 && k <= nz - 2;
    for (int comp = 0; comp < 3; ++comp) {
        st[comp * Np + c] = T(0);
        st[(3 + comp) * Np + c] = in ? T(dt * (double)v[comp * Np + c]) : T(0);
    }
}

// Failure-path check of the bounded waits: an mbarrier that nothing arrives
// on, waited for with the same bounded wait as the step and CG kernels; the
// give-up sets the same device error flag (bit 0 of kErrFlags).
__global__ void k_wait_selftest(long long *ctrl) {
    __shared__ __align__(8) uint64_t bar;
    const uint32_t b = smem_u32(&bar);
    if (threadIdx.x == 0) {
        mbar_init(b, 1);
        mbar_init_fence();
    }
    __syncthreads();
    const bool ok = mbar_wait_bounded(b, 0);
    if (!ok && threadIdx.x == 0) atomicOr(reinterpret_cast<unsigned long long *>(&ctrl[kErrFlags]), 1ull);
}

kv_status launch_wait_selftest(kv_handle *h) {
    k_wait_selftest<<<1, 32, 0, h->stream>>>(h->ctrl);
    h->launches++;
    return cuda_check(h, cudaGetLastError(), "wait self-test launch");
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
static PFN_cuTensorMapEncodeTiled_v12000 encode_fn(kv_handle *h) {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        cudaDriverEntryPointQueryResult q;
        void *ptr = nullptr;
        cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000,
                                                         cudaEnableDefault, &q);
        if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !ptr) {
            set_error(h, KV_ERR_CUDA, "cuTensorMapEncodeTiled not available (%s)",
                      cudaGetErrorString(e));
            return nullptr;
        }
        fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(ptr);
    }
    return fn;
}

// The driver's tensor-map encoder (also used by the convolution kernels).
void *tensor_map_encoder(kv_handle *h) { return reinterpret_cast<void *>(encode_fn(h)); }

kv_status encode_tensor_4d(kv_handle *h, CUtensorMap *tm, void *base, int fields, int bx, int by,
                           int fields_box) {
    PFN_cuTensorMapEncodeTiled_v12000 fn = encode_fn(h);
    if (!fn) return KV_ERR_CUDA;
    cuuint64_t dims[4] = {(cuuint64_t)h->px, (cuuint64_t)h->ny, (cuuint64_t)h->nz,
                          (cuuint64_t)fields};
    cuuint64_t strides[3] = {(cuuint64_t)h->px * 4, (cuuint64_t)h->px * h->ny * 4,
                             (cuuint64_t)h->Np * 4};
    cuuint32_t box[4] = {(cuuint32_t)bx, (cuuint32_t)by, 1, (cuuint32_t)fields_box};
    cuuint32_t es[4] = {1, 1, 1, 1};
    CUresult r = fn(tm, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, base, dims, strides, box, es,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS)
        return set_error(h, KV_ERR_CUDA, "cuTensorMapEncodeTiled failed (%d) box %dx%dx1x%d", (int)r,
                         bx, by, fields_box);
    return KV_OK;
}

typedef void (*TmaKernel)(const CUtensorMap, const CUtensorMap, const float *, float *, StepParams);

template <int TX, int TY, int NS, int K>
static void pick_kind(TmaKernel *k, size_t *smem) {
    *k = k_step_tma<TX, TY, NS, K>;
    *smem = NS * TmaTile<TX, TY, K>::STAGE * 4 + NS * 8;
}

template <int TX, int TY, int NS>
static bool pick(int tx, int ty, int ns, int kind, TmaKernel *k, size_t *smem, int *nt) {
    if (tx != TX || ty != TY || ns != NS) return false;
    switch (kind) {
        case kKindHomo: pick_kind<TX, TY, NS, kKindHomo>(k, smem); break;
        case kKindPoint: pick_kind<TX, TY, NS, kKindPoint>(k, smem); break;
        case kKindDiv: pick_kind<TX, TY, NS, kKindDiv>(k, smem); break;
        case kKindLabel: pick_kind<TX, TY, NS, kKindLabel>(k, smem); break;
        case kKindDivLabel: pick_kind<TX, TY, NS, kKindDivLabel>(k, smem); break;
        default: return false;
    }
    *nt = TX * TY / 4;
    return true;
}

template <int NS>
static bool pick_tile(int tx, int ty, int kind, TmaKernel *k, size_t *smem, int *nt) {
    return pick<32, 8, NS>(tx, ty, NS, kind, k, smem, nt) ||
           pick<32, 16, NS>(tx, ty, NS, kind, k, smem, nt) ||
           pick<64, 4, NS>(tx, ty, NS, kind, k, smem, nt) ||
           pick<64, 8, NS>(tx, ty, NS, kind, k, smem, nt) ||
           pick<64, 16, NS>(tx, ty, NS, kind, k, smem, nt) ||
           pick<128, 2, NS>(tx, ty, NS, kind, k, smem, nt) ||
           pick<128, 4, NS>(tx, ty, NS, kind, k, smem, nt) ||
           pick<128, 8, NS>(tx, ty, NS, kind, k, smem, nt);
}

typedef void (*BatchKernel)(const BatchCase *, int, int);

template <int TX, int TY, int NS>
static bool bpick(int tx, int ty, int ns, int kind, BatchKernel *k) {
    if (tx != TX || ty != TY || ns != NS) return false;
    switch (kind) {
        case kKindHomo: *k = k_step_batch<TX, TY, NS, kKindHomo>; return true;
        case kKindPoint: *k = k_step_batch<TX, TY, NS, kKindPoint>; return true;
        case kKindDiv: *k = k_step_batch<TX, TY, NS, kKindDiv>; return true;
    }
    return false;
}

template <int NS>
static bool bpick_tile(int tx, int ty, int kind, BatchKernel *k) {
    return bpick<32, 8, NS>(tx, ty, NS, kind, k) || bpick<32, 16, NS>(tx, ty, NS, kind, k) ||
           bpick<64, 4, NS>(tx, ty, NS, kind, k) || bpick<64, 8, NS>(tx, ty, NS, kind, k) ||
           bpick<64, 16, NS>(tx, ty, NS, kind, k) || bpick<128, 2, NS>(tx, ty, NS, kind, k) ||
           bpick<128, 4, NS>(tx, ty, NS, kind, k) || bpick<128, 8, NS>(tx, ty, NS, kind, k);
}

template <int TX, int TY, int NS>
static bool pick2(int tx, int ty, int ns, bool het, TmaKernel *k, size_t *smem, int *nt) {
    if (tx != TX || ty != TY || ns != NS) return false;
    if (het) {
        *k = k_step2_tma<TX, TY, NS, true>;
        *smem = (NS * Tile2<TX, TY, true>::IN_STAGE + 2 * Tile2<TX, TY, true>::MID_STAGE) * 4 + NS * 8;
    } else {
        *k = k_step2_tma<TX, TY, NS, false>;
        *smem = (NS * Tile2<TX, TY, false>::IN_STAGE + 2 * Tile2<TX, TY, false>::MID_STAGE) * 4 + NS * 8;
    }
    *nt = 128;
    return true;
}

template <int NS>
static bool pick2_tile(int tx, int ty, bool het, TmaKernel *k, size_t *smem, int *nt) {
    return pick2<32, 4, NS>(tx, ty, NS, het, k, smem, nt) || pick2<32, 8, NS>(tx, ty, NS, het, k, smem, nt) ||
           pick2<64, 4, NS>(tx, ty, NS, het, k, smem, nt) || pick2<64, 8, NS>(tx, ty, NS, het, k, smem, nt) ||
           pick2<128, 4, NS>(tx, ty, NS, het, k, smem, nt);
}

template <int TX, int TY, int NS>
static bool pick2c(int tx, int ty, int ns, bool het, TmaKernel *k, size_t *smem, int *nt) {
    if (tx != TX || ty != TY || ns != NS) return false;
    if (het) {
        *k = k_step2c_tma<TX, TY, NS, true>;
        *smem = Tile2C<TX, TY, true>::smem(NS);
    } else {
        *k = k_step2c_tma<TX, TY, NS, false>;
        *smem = Tile2C<TX, TY, false>::smem(NS);
    }
    *nt = TX * TY / 4;
    return true;
}

template <int NS>
static bool pick2c_tile(int tx, int ty, bool het, TmaKernel *k, size_t *smem, int *nt) {
    return pick2c<32, 8, NS>(tx, ty, NS, het, k, smem, nt) || pick2c<32, 16, NS>(tx, ty, NS, het, k, smem, nt) ||
           pick2c<64, 4, NS>(tx, ty, NS, het, k, smem, nt) || pick2c<64, 8, NS>(tx, ty, NS, het, k, smem, nt) ||
           pick2c<64, 16, NS>(tx, ty, NS, het, k, smem, nt) || pick2c<128, 4, NS>(tx, ty, NS, het, k, smem, nt) ||
           pick2c<128, 8, NS>(tx, ty, NS, het, k, smem, nt);
}

template <int TX, int NS>
static bool pick2b(int tx, int ty, int ns, bool het, TmaKernel *k, size_t *smem, int *nt) {
    if (tx != TX || ty != Tile2B<TX, true>::TY || ns != NS) return false;
    if (het) {
        *k = k_step2b_tma<TX, NS, true>;
        *smem = Tile2B<TX, true>::smem(NS);
    } else {
        *k = k_step2b_tma<TX, NS, false>;
        *smem = Tile2B<TX, false>::smem(NS);
    }
    *nt = Tile2B<TX, true>::NT;
    return true;
}

template <int NS>
static bool pick2b_tile(int tx, int ty, bool het, TmaKernel *k, size_t *smem, int *nt) {
    return pick2b<32, NS>(tx, ty, NS, het, k, smem, nt) || pick2b<64, NS>(tx, ty, NS, het, k, smem, nt) ||
           pick2b<128, NS>(tx, ty, NS, het, k, smem, nt);
}

// variant 2: three components per block; variant 3: one component per block;
// variant 4: one component per block, balanced TX x 14 tile
static bool tma2_kernel_for(int variant, int tx, int ty, int ns, bool het, TmaKernel *k, size_t *smem, int *nt) {
    if (variant == 4) {
        switch (ns) {
            case 2: return pick2b_tile<2>(tx, ty, het, k, smem, nt);
            case 3: return pick2b_tile<3>(tx, ty, het, k, smem, nt);
            case 4: return pick2b_tile<4>(tx, ty, het, k, smem, nt);
            case 6: return pick2b_tile<6>(tx, ty, het, k, smem, nt);
            default: return false;
        }
    }
    if (variant == 3) {
        switch (ns) {
            case 4: return pick2c_tile<4>(tx, ty, het, k, smem, nt);
            case 6: return pick2c_tile<6>(tx, ty, het, k, smem, nt);
            default: return false;
        }
    }
    switch (ns) {
        case 4: return pick2_tile<4>(tx, ty, het, k, smem, nt);
        case 6: return pick2_tile<6>(tx, ty, het, k, smem, nt);
        default: return false;
    }
}

static bool tma_kernel_for(int tx, int ty, int ns, int kind, TmaKernel *k, size_t *smem, int *nt) {
    switch (ns) {
        case 4: return pick_tile<4>(tx, ty, kind, k, smem, nt);
        case 6: return pick_tile<6>(tx, ty, kind, k, smem, nt);
        case 8: return pick_tile<8>(tx, ty, kind, k, smem, nt);
        default: return false;
    }
}

// Tensor map of the class bytes [nz][ny][px] of a class-encoded medium, box
// (tx, ty, 1, 1): the centre tile of one plane (tx bytes, a multiple of 16).
static kv_status encode_labels(kv_handle *h, CUtensorMap *tm, int tx, int ty) {
    auto fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(tensor_map_encoder(h));
    if (!fn) return set_error(h, KV_ERR_CUDA, "cuTensorMapEncodeTiled unavailable");
    cuuint64_t dims[4] = {(cuuint64_t)h->px, (cuuint64_t)h->ny, (cuuint64_t)h->nz, 1};
    cuuint64_t strides[3] = {(cuuint64_t)h->px, (cuuint64_t)h->px * h->ny, (cuuint64_t)h->Np};
    cuuint32_t box[4] = {(cuuint32_t)tx, (cuuint32_t)ty, 1, 1};
    cuuint32_t es[4] = {1, 1, 1, 1};
    CUresult r = fn(tm, CU_TENSOR_MAP_DATA_TYPE_UINT8, 4, h->labels, dims, strides, box, es,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS)
        return set_error(h, KV_ERR_CUDA, "cuTensorMapEncodeTiled (classes) failed (%d) box %dx%d", (int)r, tx, ty);
    return KV_OK;
}

// Tensor map of the coefficients that a kernel of `kind` stages for a tile
// (tx, ty): the centre tile of (A', B') for the pointwise operator, the haloed
// tile of (m, e, 1/rho) for the divergence form, the class bytes (centre tile
// or haloed 16-byte aligned tile) for the class kinds; unused placeholder for
// a homogeneous medium. The map's element type must match the kernel's kind:
// a class-byte map read with a float kernel's coordinates is misaligned.
static kv_status encode_coef_map(kv_handle *h, CUtensorMap *tm, int tx, int ty, int kind) {
    switch (kind) {
        case kKindLabel: return encode_labels(h, tm, tx, ty);
        case kKindDivLabel: return encode_labels(h, tm, tx + 32, ty + 2);
        case kKindPoint: return encode_tensor_4d(h, tm, h->coef, 2, tx, ty, 2);
        case kKindDiv: return encode_tensor_4d(h, tm, h->coef, 3, tx + 8, ty + 2, 3);
        default: *tm = h->tm_state[0]; return KV_OK;
    }
}

kv_status step_prepare(kv_handle *h) {
    h->tma_ready = 0;
    if (h->precision != KV_FP32 || h->variant == 1) return KV_OK;
    TmaKernel k;
    size_t smem;
    int nt;
    if (h->variant >= 2) {
        if (step_kind(h) == kKindDiv)
            return set_error(h, KV_ERR_UNSUPPORTED, "the two-step kernels support only the pointwise operator");
        if (!tma2_kernel_for(h->variant, h->tx, h->ty, h->ns_stages, h->het != 0, &k, &smem, &nt))
            return set_error(h, KV_ERR_ARG, "no two-step kernel (variant %d) for tile %dx%d with %d stages",
                             h->variant, h->tx, h->ty, h->ns_stages);
        if (smem > 227 * 1024)
            return set_error(h, KV_ERR_ARG, "two-step tile %dx%d with %d stages needs %zu bytes of shared memory",
                             h->tx, h->ty, h->ns_stages, smem);
        kv_status st;
        // variants 3 and 4 stage one field per box (u_c and d_c are fields c and 3 + c)
        const int fbox = h->variant >= 3 ? 1 : 6;
        for (int b = 0; b < 2; ++b)
            if ((st = encode_tensor_4d(h, &h->tm_state[b], h->state[b], 6, h->tx + 8, h->ty + 4, fbox)) != KV_OK)
                return st;
        if (h->het && (st = encode_tensor_4d(h, &h->tm_coef, h->coef, 2, h->tx + 8, h->ty + 2, 2)) != KV_OK)
            return st;
        if (!h->het) h->tm_coef = h->tm_state[0];
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return cuda_check(h, e, "cudaFuncSetAttribute(step2)");
        h->tma_ready = 1;
        return KV_OK;
    }
    if (!tma_kernel_for(h->tx, h->ty, h->ns_stages, tma_kind(h), &k, &smem, &nt))
        return set_error(h, KV_ERR_ARG, "no TMA step kernel for tile %dx%d with %d stages", h->tx,
                         h->ty, h->ns_stages);
    const int tk = tma_kind(h);
    const size_t static_smem = tk == kKindLabel      ? kMaxLabels * sizeof(float2)
                               : tk == kKindDivLabel ? kMaxLabels * (sizeof(float2) + sizeof(float))
                                                     : 0;  // class tables
    if (smem + static_smem > 227 * 1024)
        return set_error(h, KV_ERR_ARG, "tile %dx%d with %d stages needs %zu bytes of shared memory",
                         h->tx, h->ty, h->ns_stages, smem + static_smem);
    kv_status st;
    for (int b = 0; b < 2; ++b)
        if ((st = encode_tensor_4d(h, &h->tm_state[b], h->state[b], 6, h->tx + 8, h->ty + 2, 6)) != KV_OK)
            return st;
    if ((st = encode_coef_map(h, &h->tm_coef, h->tx, h->ty, tma_kind(h))) != KV_OK) return st;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_check(h, e, "cudaFuncSetAttribute(step)");
    h->tma_ready = 1;
    return KV_OK;
}

static StepParams make_params(kv_handle *h, int nblocks) {
    StepParams p;
    p.nx = h->nx;
    p.ny = h->ny;
    p.nz = h->nz;
    p.px = h->px;
    p.Np = h->Np;
    p.A = h->A_s;
    p.B = h->B_s;
    p.Af = (float)h->A_s;
    p.Bf = (float)h->B_s;
    p.g = h->g_dev;
    p.n_g = h->have_force ? h->n_g : 0;
    p.g_const_on = h->have_force && h->g_const_on;
    p.g_const = 1.f;
    p.ctrl = h->ctrl;
    p.sensors = h->sens_dev;
    p.sens_off = h->sens_dev ? h->sens_dev + 3 * h->ns : nullptr;
    p.sens_ord = h->sens_dev ? h->sens_dev + 3 * h->ns + h->nz + 1 : nullptr;
    p.ns = h->ns;
    p.traces = h->traces;
    p.cap = h->cap;
    p.zc = h->zc;
    p.nblocks = nblocks;
    p.lab_tab = h->lab_tab;
    p.n_lab = h->n_labels;
    return p;
}

// Two steps from state[from] into state[1 - from] (variants 2 and 3).
kv_status step2_launch(kv_handle *h, int from) {
    if (!h->tma_ready) {
        kv_status st = step_prepare(h);
        if (st != KV_OK) return st;
    }
    TmaKernel k;
    size_t smem;
    int nt;
    tma2_kernel_for(h->variant, h->tx, h->ty, h->ns_stages, h->het != 0, &k, &smem, &nt);
    const int ncomp_blocks = h->variant >= 3 ? 3 : 1;  // variants 3, 4: the three components of a tile side by side
    dim3 grid(ncomp_blocks * ((h->px + h->tx - 1) / h->tx), (h->ny - 2 + h->ty - 1) / h->ty,
              (h->nz - 2 + h->zc - 1) / h->zc);
    StepParams p = make_params(h, grid.x * grid.y * grid.z);
    k<<<grid, nt, smem, h->stream>>>(h->tm_state[from], h->tm_coef, (const float *)h->F,
                                     (float *)h->state[1 - from], p);
    h->launches++;
    return cuda_check(h, cudaGetLastError(), "step2 launch");
}

kv_status step_launch(kv_handle *h, int from) {
    void *in = h->state[from];
    void *out = h->state[1 - from];
    if (h->precision == KV_FP32 && h->variant == 0) {
        if (!h->tma_ready) {
            kv_status st = step_prepare(h);
            if (st != KV_OK) return st;
        }
        TmaKernel k;
        size_t smem;
        int nt;
        tma_kernel_for(h->tx, h->ty, h->ns_stages, tma_kind(h), &k, &smem, &nt);
        dim3 grid((h->px + h->tx - 1) / h->tx, (h->ny - 2 + h->ty - 1) / h->ty,
                  (h->nz - 2 + h->zc - 1) / h->zc);
        StepParams p = make_params(h, grid.x * grid.y * grid.z);
        k<<<grid, nt, smem, h->stream>>>(h->tm_state[from], h->tm_coef, (const float *)h->F,
                                         (float *)out, p);
    } else {
        dim3 grid((h->nx + 127) / 128, h->ny - 2, h->nz - 2);
        StepParams p = make_params(h, grid.x * grid.y * grid.z);
        const int kind = step_kind(h);
        if (h->precision == KV_FP64) {
            const double *ci = (const double *)in, *co = (const double *)h->coef, *cf = (const double *)h->F;
            double *o = (double *)out;
            if (kind == kKindDiv) k_step_plain<double, kKindDiv><<<grid, 128, 0, h->stream>>>(ci, o, co, cf, p);
            else if (kind == kKindPoint) k_step_plain<double, kKindPoint><<<grid, 128, 0, h->stream>>>(ci, o, co, cf, p);
            else k_step_plain<double, kKindHomo><<<grid, 128, 0, h->stream>>>(ci, o, nullptr, cf, p);
        } else {
            const float *ci = (const float *)in, *co = (const float *)h->coef, *cf = (const float *)h->F;
            float *o = (float *)out;
            if (kind == kKindDiv) k_step_plain<float, kKindDiv><<<grid, 128, 0, h->stream>>>(ci, o, co, cf, p);
            else if (kind == kKindPoint) k_step_plain<float, kKindPoint><<<grid, 128, 0, h->stream>>>(ci, o, co, cf, p);
            else k_step_plain<float, kKindHomo><<<grid, 128, 0, h->stream>>>(ci, o, nullptr, cf, p);
        }
    }
    h->launches++;
    return cuda_check(h, cudaGetLastError(), "step launch");
}

// Launchers used by the C ABI (kv_api.cu).
kv_status launch_fold(kv_handle *h, const float *G, double Gs, const float *rho, double rhos,
                      const float *eta, double etas) {
    const dim3 grid((h->px + 127) / 128, h->ny, h->nz);
    if (h->precision == KV_FP64)
        k_fold<double><<<grid, 128, 0, h->stream>>>(G, rho, eta, Gs, rhos, etas, (double *)h->coef,
                                                    (double *)h->S, h->Np, h->nx, h->px, h->ny,
                                                    h->dt, h->dx, step_kind(h) == kKindDiv);
    else
        k_fold<float><<<grid, 128, 0, h->stream>>>(G, rho, eta, Gs, rhos, etas, (float *)h->coef,
                                                   (float *)h->S, h->Np, h->nx, h->px, h->ny, h->dt,
                                                   h->dx, step_kind(h) == kKindDiv);
    h->launches++;
    return cuda_check(h, cudaGetLastError(), "fold launch");
}

kv_status launch_init_velocity(kv_handle *h, const float *v_pitched) {
    const int nt = 256;
    const long long nb = (h->Np + nt - 1) / nt;
    if (h->precision == KV_FP64)
        k_init_velocity<double><<<(unsigned)nb, nt, 0, h->stream>>>(
            v_pitched, (double *)h->state[h->cur], h->nx, h->ny, h->nz, h->px, h->Np, h->dt);
    else
        k_init_velocity<float><<<(unsigned)nb, nt, 0, h->stream>>>(
            v_pitched, (float *)h->state[h->cur], h->nx, h->ny, h->nz, h->px, h->Np, h->dt);
    h->launches++;
    return cuda_check(h, cudaGetLastError(), "initial velocity launch");
}

// ---------------------------------------------------------------------------
// Batched step support (kv_batch.cu)
// ---------------------------------------------------------------------------
kv_status batch_kernel_for(int tx, int ty, int ns, int kind, void **kernel, size_t *smem, int *nt) {
    TmaKernel single;
    if (!tma_kernel_for(tx, ty, ns, kind, &single, smem, nt)) return KV_ERR_ARG;
    BatchKernel k = nullptr;
    bool ok = false;
    switch (ns) {
        case 4: ok = bpick_tile<4>(tx, ty, kind, &k); break;
        case 6: ok = bpick_tile<6>(tx, ty, kind, &k); break;
        case 8: ok = bpick_tile<8>(tx, ty, kind, &k); break;
    }
    if (!ok || *smem > 227 * 1024) return KV_ERR_ARG;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)*smem);
    if (e != cudaSuccess) return KV_ERR_CUDA;
    *kernel = (void *)k;
    return KV_OK;
}

// Fill one batch table entry for handle h with tile (tx, ty), zc planes per
// block, the first block index `begin`; returns the case's block count.
kv_status batch_fill_case(kv_handle *h, BatchCase *bc, int tx, int ty, int zc, int begin, int *blocks) {
    kv_status st;
    for (int b = 0; b < 2; ++b)
        if ((st = encode_tensor_4d(h, &bc->tm_state[b], h->state[b], 6, tx + 8, ty + 2, 6)) != KV_OK)
            return st;
    if (h->het) {
        // the batch kernels read the coefficient fields (kinds 1 and 2), never class bytes
        if ((st = encode_coef_map(h, &bc->tm_coef, tx, ty, step_kind(h))) != KV_OK) return st;
    } else {
        bc->tm_coef = bc->tm_state[0];
    }
    bc->F = (const float *)h->F;
    bc->state[0] = (float *)h->state[0];
    bc->state[1] = (float *)h->state[1];
    bc->gx = (h->px + tx - 1) / tx;
    bc->gy = (h->ny - 2 + ty - 1) / ty;
    bc->gz = (h->nz - 2 + zc - 1) / zc;
    bc->block_begin = begin;
    *blocks = bc->gx * bc->gy * bc->gz;
    StepParams p = make_params(h, *blocks);
    p.zc = zc;
    bc->p = p;
    return KV_OK;
}

kv_status batch_launch(void *kernel, const BatchCase *table, int ncases, int total_blocks, int nt,
                       size_t smem, int from, cudaStream_t s) {
    BatchKernel k = (BatchKernel)kernel;
    k<<<total_blocks, nt, smem, s>>>(table, ncases, from);
    return cudaGetLastError() == cudaSuccess ? KV_OK : KV_ERR_CUDA;
}
}  // namespace kv
