// TET04 element assembly (mixed precision) for sm_103a: persistent,
// warp-specialised kernel.
//
// Per element (affine map, constant gradients) the element residual of
// Eq. momentum takes the closed forms of the 4-point rule, which is exact
// for these degree-2 integrands:
//   sum_g W N_a N_b = V (1 + delta_ab) / 20,   sum_g W N_a = V / 4,
//   r_a = - [ (G + tr G I) V/20 (u_a + sum_b u_b) + V/4 grad p
//             + 2 (nu + nu_t) V eps grad N_a ],
// grad N_k (k = 1..3) the rows of J^-1 = cofactors / det J, grad N_0 =
// -sum_k grad N_k; nu_t = c Delta^2 sqrt(B'/G:G) (Vreman, B' the sum of the
// squared cross products of the rows of G), Delta = V^(1/3).
//
// Gather -> compute -> scatter (section 2.3.3) as three kinds of warps of one
// CTA per SM, which meet only at mbarrier phases (no CTA-wide barrier):
//  * producer warp: per chunk of C = 64 NW elements, TMA bulk copies of the
//    chunk's node records (coordinates relative to the chunk), node ids,
//    element records and slot-offset table into one of kWsStages input
//    stages, then cp.async gathers of the FP32 field (u, v, w, p) of every
//    chunk node;
//  * NW compute warps: one record per thread, i.e. two elements on packed
//    FP32 (FFMA2): a face pair (two tetrahedra that share a face: five node
//    loads, the face nodes' residuals summed in registers) or two elements
//    of their own; each residual goes to its own slot of the chunk's
//    incidence list;
//  * NR reducer warps: per chunk node the sum of its slots, then one FP64
//    store (node of this chunk only) or FP64 atomic add (shared node).
// Slots are laid out incidence-major: slot (node l, its t-th incidence) at
// toff[t] + l with the nodes numbered by decreasing slot count, so that a
// reducer warp (lane = node) runs one loop over t and reads consecutive
// slots.  Two slot buffers let the reducers sum chunk i while the compute
// warps fill chunk i + 1.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>

#include "fea_internal.h"

namespace fea {
namespace {

constexpr int kWsStages = 5;   // input stages
constexpr int kWsLag = 2;      // the gathers of a chunk trail its bulk copies by this many chunks
constexpr int kWsSlots = 2;    // slot buffers
// Default wait limit: polls of a phase, each suspending the warp for at most
// kWsSuspendNs unless the phase completes first (about 2.6 s in all).
constexpr uint32_t kWsDefaultPolls = 1u << 17;
constexpr uint32_t kWsSuspendNs = 20000;

__device__ __forceinline__ uint32_t sa(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mb_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(sa(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mb_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.release.cta.shared::cta.b64 _, [%0];" ::"r"(sa(bar)) : "memory");
}
__device__ __forceinline__ void mb_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(sa(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mb_try(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.acquire.cta.shared::cta.b64 p, [%1], %2, %3;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(sa(bar)), "r"(parity), "r"(kWsSuspendNs)
        : "memory");
    return ok != 0;
}
// non-suspending test of a phase
__device__ __forceinline__ bool mb_test(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.test_wait.parity.acquire.cta.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(sa(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Limit of a bounded wait: `polls` polls of the phase, each a try_wait
// (which suspends the warp until the phase completes, for at most
// kWsSuspendNs) or, with `quick`,
// a non-suspending test_wait (a set poll limit then bounds the wait tightly).
struct WaitLimit {
    uint32_t polls;
    bool quick;
};
// Bounded wait on a phase of an mbarrier by a whole warp (every lane polls,
// the outcome is warp-uniform): false once the limit is spent, or as soon as
// another warp of the CTA has raised the abort flag (abort may be NULL).
__device__ __forceinline__ bool mb_wait(uint64_t *bar, uint32_t parity, WaitLimit lim, const volatile int *abort) {
    for (uint32_t it = 0; it < lim.polls; ++it) {
        if (__all_sync(0xffffffffu, lim.quick ? mb_test(bar, parity) : mb_try(bar, parity))) return true;
        if (abort && (it & 63u) == 63u && __any_sync(0xffffffffu, *abort != 0)) return false;
    }
    return false;
}
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile("cp.async.bulk.shared::cta.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(sa(dst)),
                 "l"(src), "r"(bytes), "r"(sa(bar))
                 : "memory");
}
__device__ __forceinline__ void cpa16(void *dst, const void *src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sa(dst)), "l"(src) : "memory");
}
// arrive on `bar` once every cp.async this thread issued so far has landed
__device__ __forceinline__ void cpa_arrive(uint64_t *bar) {
    asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(sa(bar)) : "memory");
}

// FP32 -> FP64 by integer operations for normal numbers (off the FP64 pipe);
// zero, subnormals, inf and nan take the hardware conversion.
__device__ __forceinline__ double widen(float x) {
    const uint32_t b = __float_as_uint(x);
    const uint32_t e = (b >> 23) & 0xffu;
    if (e == 0u || e == 0xffu) return (double)x;
    const uint32_t hi = (b & 0x80000000u) | ((e + 896u) << 20) | ((b & 0x7fffffu) >> 3);
    return __hiloint2double((int)hi, (int)(b << 29));
}

// per chunk: toff[t] = first slot of the t-th incidences of the nodes (the
// nodes are numbered by decreasing slot count, so the nodes with more than t
// slots are 0 .. toff[t+1] - toff[t] - 1); 65 entries used, 68 stored
constexpr int kToff = 68;

struct WsParams {
    float nu, cv;
    bool conv, pres, sgs, want_q;
};

__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float2 bc(float v) { return make_float2(v, v); }

__device__ __forceinline__ float vq(float aa, float B) {
    // sqrt(B'/G:G) = B' rsqrt(B') rsqrt(G:G); 0 for a vanishing gradient
    return (B > 0.f && aa > 0.f) ? B * rsqrtf(B) * rsqrtf(aa) : 0.f;
}

// Residuals of two tetrahedra at once (.x: element A, .y: element B).
// X*, U*: node records (chunk-relative coordinates) and field values of the
// four nodes; out r[a][i] (node a, component i).
//
// Arranged for instruction-level parallelism: with the cofactor matrix
// CF = det J^-1 (rows c_1..c_3 = grad N_1..3 times det) the products
// G' = det G, det grad p, and H c_a (H = G' + G'^T) need no division, and
// the identities det V/det = V/6 ... reduce every coefficient to
//   -V/20 (G + tr G I) = -(G' + tr G' I)/120,   -V/4 grad p = -(det grad p)/24,
//   -2 (nu + nu_t) V eps grad N_a = -(nu + nu_t)/(6 det) H c_a,
// so the reciprocal, the power and the square roots of the Vreman branch
// overlap the long FMA blocks instead of preceding them.
template <bool FULL>
__device__ __forceinline__ void tet_pair(const float4 XA[4], const float4 UA[4], const float4 XB[4], const float4 UB[4],
                                         const WsParams &tp_in, float2 r[4][3], float2 &nut, bool &bad) {
    WsParams tp = tp_in;
    if (FULL) tp.conv = tp.pres = tp.sgs = tp.want_q = true;
    // differences in scalar FP32, landing directly in packed registers
    float2 d[3][3], du[3][3], dp[3], w[3];
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        d[q][0] = f2(XA[q + 1].x - XA[0].x, XB[q + 1].x - XB[0].x);
        d[q][1] = f2(XA[q + 1].y - XA[0].y, XB[q + 1].y - XB[0].y);
        d[q][2] = f2(XA[q + 1].z - XA[0].z, XB[q + 1].z - XB[0].z);
        du[q][0] = f2(UA[q + 1].x - UA[0].x, UB[q + 1].x - UB[0].x);
        du[q][1] = f2(UA[q + 1].y - UA[0].y, UB[q + 1].y - UB[0].y);
        du[q][2] = f2(UA[q + 1].z - UA[0].z, UB[q + 1].z - UB[0].z);
        dp[q] = f2(UA[q + 1].w - UA[0].w, UB[q + 1].w - UB[0].w);
    }
    // w = u_0 + sum_b u_b
    w[0] = f2((UA[0].x + UA[1].x) + (UA[2].x + UA[3].x) + UA[0].x, (UB[0].x + UB[1].x) + (UB[2].x + UB[3].x) + UB[0].x);
    w[1] = f2((UA[0].y + UA[1].y) + (UA[2].y + UA[3].y) + UA[0].y, (UB[0].y + UB[1].y) + (UB[2].y + UB[3].y) + UB[0].y);
    w[2] = f2((UA[0].z + UA[1].z) + (UA[2].z + UA[3].z) + UA[0].z, (UB[0].z + UB[1].z) + (UB[2].z + UB[3].z) + UB[0].z);
    // cofactors: row q = det grad N_{q+1}
    float2 cf[3][3];
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        const float2 *a = d[(q + 1) % 3], *b = d[(q + 2) % 3];
        cf[q][0] = fma2(a[1], b[2], neg2(mul2(a[2], b[1])));
        cf[q][1] = fma2(a[2], b[0], neg2(mul2(a[0], b[2])));
        cf[q][2] = fma2(a[0], b[1], neg2(mul2(a[1], b[0])));
    }
    const float2 det = fma2(d[0][0], cf[0][0], fma2(d[0][1], cf[0][1], mul2(d[0][2], cf[0][2])));
    if (!(det.x > 0.f) || !(det.y > 0.f)) bad = true;
    const float2 inv = f2(__fdividef(1.f, det.x), __fdividef(1.f, det.y));
    // G' = det G, gp' = det grad p
    float2 Gp[3][3], gpp[3];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        gpp[j] = fma2(dp[0], cf[0][j], fma2(dp[1], cf[1][j], mul2(dp[2], cf[2][j])));
#pragma unroll
        for (int i = 0; i < 3; ++i)
            Gp[i][j] = fma2(du[0][i], cf[0][j], fma2(du[1][i], cf[1][j], mul2(du[2][i], cf[2][j])));
    }
    nut = bc(0.f);
    if (tp.want_q) {
        // Vreman on G = G' / det (kept in range for small elements)
        float2 G[3][3];
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j) G[i][j] = mul2(Gp[i][j], inv);
        float2 aa = bc(0.f), B = bc(0.f);
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j) aa = fma2(G[i][j], G[i][j], aa);
#pragma unroll
        for (int pq = 0; pq < 3; ++pq) {
            const int i = pq == 2 ? 1 : 0, j = pq == 0 ? 1 : 2;
            const float2 x = fma2(G[i][1], G[j][2], neg2(mul2(G[i][2], G[j][1])));
            const float2 y = fma2(G[i][2], G[j][0], neg2(mul2(G[i][0], G[j][2])));
            const float2 z = fma2(G[i][0], G[j][1], neg2(mul2(G[i][1], G[j][0])));
            B = fma2(x, x, fma2(y, y, fma2(z, z, B)));
        }
        // Delta^2 = V^(2/3), V = det/6
        const float2 d2 = f2(__powf(fabsf(det.x) * (1.f / 6.f), 2.f / 3.f), __powf(fabsf(det.y) * (1.f / 6.f), 2.f / 3.f));
        nut = mul2(mul2(bc(tp.cv), d2), f2(vq(aa.x, B.x), vq(aa.y, B.y)));
    }
    // kap = -(nu + nu_t) / (6 det)
    const float2 kap = mul2(add2(bc(tp.nu), tp.sgs ? nut : bc(0.f)), mul2(inv, bc(-1.f / 6.f)));
    // H = G' + G'^T (symmetric), and H c_a for nodes 1..3
    float2 H[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        H[i][i] = add2(Gp[i][i], Gp[i][i]);
#pragma unroll
        for (int j = i + 1; j < 3; ++j) H[i][j] = H[j][i] = add2(Gp[i][j], Gp[j][i]);
    }
    float2 tv[3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int i = 0; i < 3; ++i) tv[a][i] = fma2(H[i][0], cf[a][0], fma2(H[i][1], cf[a][1], mul2(H[i][2], cf[a][2])));
    // convective coefficients Q = -(G' + tr G' I)/120 and node 0's
    // convective and pressure part cp = Q (u_0 + sum_b u_b) - gp'/24
    const float2 trG = add2(add2(Gp[0][0], Gp[1][1]), Gp[2][2]);
    const float2 c120 = bc(tp.conv ? -1.f / 120.f : 0.f);
    float2 Q[3][3], cp[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
#pragma unroll
        for (int j = 0; j < 3; ++j) Q[i][j] = mul2(c120, i == j ? add2(Gp[i][j], trG) : Gp[i][j]);
        cp[i] = fma2(Q[i][0], w[0], fma2(Q[i][1], w[1], fma2(Q[i][2], w[2], mul2(bc(tp.pres ? -1.f / 24.f : 0.f), gpp[i]))));
    }
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        r[0][i] = fma2(kap, neg2(add2(add2(tv[0][i], tv[1][i]), tv[2][i])), cp[i]);
#pragma unroll
        for (int a = 0; a < 3; ++a)
            // node a+1: u_{a+1} + sum_b u_b = w + du_a
            r[a + 1][i] = fma2(kap, tv[a][i], fma2(Q[i][0], du[a][0], fma2(Q[i][1], du[a][1], fma2(Q[i][2], du[a][2], cp[i]))));
    }
}

// Chunk metadata (node-list offset and end, node count, face pairs) of a
// CTA's chunks c0 + k G, fetched for 32 consecutive k at a time (lane l
// holds k = base + l) and broadcast by shuffles, so that a warp pays one
// global latency per 32 chunks instead of one per chunk.
struct ChunkMeta {
    int64_t base = -1, off = 0, off1 = 0;
    int L = 0, nfp = 0;
    __device__ __forceinline__ void get(const BucketDev &b, int64_t c0, int64_t G, int64_t k, int lane, int64_t &o,
                                        int64_t &o1, int &n, int &fp) {
        const int64_t kb = k & ~(int64_t)31;
        if (kb != base) {
            base = kb;
            const int64_t c = c0 + (kb + lane) * G;
            if (c < b.ws_nch) {
                off = __ldg(&b.ws_off[c]);
                off1 = __ldg(&b.ws_off[c + 1]);
                L = __ldg(&b.ws_nodes[c]);
                nfp = __ldg(&b.ws_nfp[c]);
            }
        }
        const int src = (int)(k - kb);
        o = __shfl_sync(0xffffffffu, off, src);
        o1 = __shfl_sync(0xffffffffu, off1, src);
        n = __shfl_sync(0xffffffffu, L, src);
        fp = __shfl_sync(0xffffffffu, nfp, src);
    }
};

// Shared memory of one CTA (offsets in bytes from the dynamic base):
//   slots  [kWsSlots][4C] float4: slot (node l, its t-th incidence) at toff[t] + l
//   stage  [kWsStages] x { rec [LMP] float4, fld [LMP] float4, ids [LMP] u32, elr [C/2] uint4,
//                          toff [kToff] u32 }
//   mbarriers tma[D], full[D], empty[D], sfull[S], sempty[S]; abort flag
struct WsLayout {
    int C, LMP;
    size_t slot_bytes, stage_bytes, rec, fld, ids, elr, toff, bars, total;
    __host__ __device__ WsLayout(int C_, int LMP_) : C(C_), LMP(LMP_) {
        slot_bytes = (size_t)16 * 4 * C;
        rec = 0;
        fld = (size_t)16 * LMP;
        ids = (size_t)32 * LMP;
        elr = (size_t)36 * LMP;
        toff = elr + (size_t)8 * C;
        stage_bytes = (toff + 4 * kToff + 15) & ~(size_t)15;
        bars = kWsSlots * slot_bytes + kWsStages * stage_bytes;
        total = bars + 8 * (3 * kWsStages + 2 * kWsSlots) + 16;
    }
};

template <int NW, int NR, bool FULL>
__global__ void __launch_bounds__(32 * (NW + NR + 1), NW <= 4 ? 2 : 1)
    k_tet_ws(BucketDev b, FieldDev f, AsmArgs args, WsParams tp, WaitLimit polls) {
    constexpr int C = 64 * NW;
    extern __shared__ __align__(128) unsigned char smem[];
    const WsLayout lay(C, b.ws_lmp);
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem + lay.bars);
    uint64_t *tma = bar, *full = bar + kWsStages, *empty = bar + 2 * kWsStages;
    uint64_t *sfull = bar + 3 * kWsStages, *sempty = sfull + kWsSlots;
    volatile int *abort_flag = reinterpret_cast<volatile int *>(sempty + kWsSlots);
    auto SLOT = [&](int s) { return reinterpret_cast<float4 *>(smem + (size_t)s * lay.slot_bytes); };
    auto STG = [&](int q) { return smem + kWsSlots * lay.slot_bytes + (size_t)q * lay.stage_bytes; };
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t G = gridDim.x, c0 = blockIdx.x, nch = b.ws_nch;
    // a kernel launched after this one as a programmatic dependent (the
    // FP64-Jacobian PEN06 category) may start as soon as CTAs of this one
    // retire: it fills the SMs of this kernel's tail
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    if (threadIdx.x == 0) {
        for (int q = 0; q < kWsStages; ++q) {
            mb_init(&tma[q], 1);
            mb_init(&full[q], 32);
            mb_init(&empty[q], NW + NR);
        }
        for (int s = 0; s < kWsSlots; ++s) {
            mb_init(&sfull[s], NW);
            mb_init(&sempty[s], NR);
        }
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    bool timed_out = false, bad = false;

    if (warp == NW + NR) {
        // ---------------- producer ----------------
        // The bulk copies of chunk k are issued kWsLag steps before its
        // gathers (which need its node ids), so that the two overlap.
        ChunkMeta mt, mg;
        int64_t issued = -1, gathered = -1;   // last k whose bulk copies / gathers were issued
        for (int64_t k = 0;; ++k) {
            const int64_t c = c0 + k * G;
            if (c < nch) {
                const int q = (int)(k % kWsStages);
                int64_t nb, nb1;
                int L, nfp;
                mt.get(b, c0, G, k, lane, nb, nb1, L, nfp);
                if (!mb_wait(&empty[q], (uint32_t)(((k / kWsStages) & 1) ^ 1), polls, abort_flag)) {
                    timed_out = true;
                    break;
                }
                if (lane == 0) {
                    const uint32_t Lp = (uint32_t)(nb1 - nb);
                    const int64_t e0 = c * C;
                    const uint32_t ne = (uint32_t)min((int64_t)C, b.count - e0);
                    const uint32_t eb = 16u * ((uint32_t)nfp + (ne - 2u * (uint32_t)nfp + 1u) / 2u);
                    unsigned char *st = STG(q);
                    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                    mb_expect_tx(&tma[q], Lp * 20u + eb + 4u * kToff);
                    bulk_g2s(st + lay.rec, b.ws_rec + nb, Lp * 16u, &tma[q]);
                    bulk_g2s(st + lay.ids, b.ws_ids + nb, Lp * 4u, &tma[q]);
                    bulk_g2s(st + lay.elr, b.ws_elem + c * (C / 2), eb, &tma[q]);
                    bulk_g2s(st + lay.toff, b.ws_toff + c * kToff, 4u * kToff, &tma[q]);
                }
                issued = k;
            }
            if (k >= kWsLag) {
                const int64_t kg = k - kWsLag;
                const int64_t cg = c0 + kg * G;
                if (cg >= nch) break;
                const int qg = (int)(kg % kWsStages);
                int64_t nb, nb1;
                int L, nfp;
                mg.get(b, c0, G, kg, lane, nb, nb1, L, nfp);
                if (!mb_wait(&tma[qg], (uint32_t)((kg / kWsStages) & 1), polls, abort_flag)) {
                    timed_out = true;
                    break;
                }
                unsigned char *st = STG(qg);
                const uint32_t *ids = reinterpret_cast<const uint32_t *>(st + lay.ids);
                float4 *fld = reinterpret_cast<float4 *>(st + lay.fld);
                for (int j0 = 0; j0 < L; j0 += 128) {
                    uint32_t idv[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const int j = j0 + 32 * u + lane;
                        idv[u] = j < L ? ids[j] : 0u;
                    }
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const int j = j0 + 32 * u + lane;
                        if (j < L) cpa16(fld + j, f.up32 + (idv[u] & 0x7fffffffu));
                    }
                }
                cpa_arrive(&full[qg]);
                gathered = kg;
            }
        }
        asm volatile("cp.async.wait_all;" ::: "memory");
        if (timed_out) {
            *abort_flag = 1;
            // let every bulk copy and gather still in flight land before the
            // CTA's shared memory is released
            for (int64_t k = gathered + 1; k <= issued; ++k)
                mb_wait(&tma[k % kWsStages], (uint32_t)((k / kWsStages) & 1), WaitLimit{kWsDefaultPolls, false},
                        nullptr);
            if (gathered >= 0)
                mb_wait(&full[gathered % kWsStages], (uint32_t)((gathered / kWsStages) & 1),
                        WaitLimit{kWsDefaultPolls, false}, nullptr);
        }
    } else if (warp < NW) {
        // ---------------- compute ----------------
        // Record t of a chunk: a face pair (t < nfp; elements A = (f0, f1,
        // f2, a) and B = (f1, f0, f2, b)) or two elements of their own.
        const int t = warp * 32 + lane;
        ChunkMeta mc;
        for (int64_t i = 0;; ++i) {
            const int64_t c = c0 + i * G;
            if (c >= nch) break;
            const int q = (int)(i % kWsStages), s = (int)(i % kWsSlots);
            const uint32_t pq = (uint32_t)((i / kWsStages) & 1);
            int64_t nb, nb1;
            int L, nfp;
            mc.get(b, c0, G, i, lane, nb, nb1, L, nfp);
            if (!mb_wait(&tma[q], pq, polls, abort_flag) || !mb_wait(&full[q], pq, polls, abort_flag) ||
                !mb_wait(&sempty[s], (uint32_t)(((i / kWsSlots) & 1) ^ 1), polls, abort_flag)) {
                timed_out = true;
                break;
            }
            const int64_t e0 = c * C;
            const int ne = (int)min((int64_t)C, b.count - e0);
            const int nrest = ne - 2 * nfp;
            const unsigned char *st = STG(q);
            const float4 *rec = reinterpret_cast<const float4 *>(st + lay.rec);
            const float4 *fld = reinterpret_cast<const float4 *>(st + lay.fld);
            const uint4 *elr = reinterpret_cast<const uint4 *>(st + lay.elr);
            const uint32_t *toff = reinterpret_cast<const uint32_t *>(st + lay.toff);
            float4 *slot = SLOT(s);
            const bool face = t < nfp;
            const int u = t - nfp;
            if (face || 2 * u < nrest) {
                const bool hasb = face || 2 * u + 1 < nrest;
                const uint4 er = elr[t];
                uint32_t va[4], vb[4];
#pragma unroll
                for (int a = 0; a < 4; ++a) {
                    va[a] = ((a < 2 ? er.x : er.y) >> (16 * (a & 1))) & 0xffffu;
                    vb[a] = ((a < 2 ? er.z : er.w) >> (16 * (a & 1))) & 0xffffu;
                }
                float4 XA[4], UA[4], XB[4], UB[4];
#pragma unroll
                for (int a = 0; a < 4; ++a) {
                    XA[a] = rec[va[a] & 0x3ffu];
                    UA[a] = fld[va[a] & 0x3ffu];
                }
                if (face) {
                    // B shares A's face (f0, f1, f2) in the order (f1, f0, f2)
                    const float4 xb = rec[vb[0] & 0x3ffu], ub = fld[vb[0] & 0x3ffu];
                    XB[0] = XA[1], XB[1] = XA[0], XB[2] = XA[2], XB[3] = xb;
                    UB[0] = UA[1], UB[1] = UA[0], UB[2] = UA[2], UB[3] = ub;
                } else {
                    const uint32_t *vv = hasb ? vb : va;
#pragma unroll
                    for (int a = 0; a < 4; ++a) {
                        XB[a] = rec[vv[a] & 0x3ffu];
                        UB[a] = fld[vv[a] & 0x3ffu];
                    }
                }
                float2 r[4][3], nut;
                tet_pair<FULL>(XA, UA, XB, UB, tp, r, nut, bad);
                auto put = [&](float4, uint32_t v, float r0, float r1, float r2) {
                    slot[toff[v >> 10] + (v & 0x3ffu)] = make_float4(r0, r1, r2, 0.f);
                };
                if (face) {
                    put(XA[0], va[0], r[0][0].x + r[1][0].y, r[0][1].x + r[1][1].y, r[0][2].x + r[1][2].y);
                    put(XA[1], va[1], r[1][0].x + r[0][0].y, r[1][1].x + r[0][1].y, r[1][2].x + r[0][2].y);
                    put(XA[2], va[2], r[2][0].x + r[2][0].y, r[2][1].x + r[2][1].y, r[2][2].x + r[2][2].y);
                    put(XA[3], va[3], r[3][0].x, r[3][1].x, r[3][2].x);
                    put(XB[3], vb[0], r[3][0].y, r[3][1].y, r[3][2].y);
                } else {
#pragma unroll
                    for (int a = 0; a < 4; ++a) put(XA[a], va[a], r[a][0].x, r[a][1].x, r[a][2].x);
                    if (hasb) {
#pragma unroll
                        for (int a = 0; a < 4; ++a) put(XB[a], vb[a], r[a][0].y, r[a][1].y, r[a][2].y);
                    }
                }
                if (args.nut) {
                    float4 *nu4 = reinterpret_cast<float4 *>(args.nut);
                    nu4[__ldg(&b.ws_eorig[e0 + 2 * t])] = make_float4(nut.x, nut.x, nut.x, nut.x);
                    if (hasb) nu4[__ldg(&b.ws_eorig[e0 + 2 * t + 1])] = make_float4(nut.y, nut.y, nut.y, nut.y);
                }
            }
            __syncwarp();
            if (lane == 0) {
                mb_arrive(&sfull[s]);
                mb_arrive(&empty[q]);
            }
        }
    } else {
        // ---------------- reducers ----------------
        const int rw = warp - NW;
        ChunkMeta mr;
        for (int64_t i = 0;; ++i) {
            const int64_t c = c0 + i * G;
            if (c >= nch) break;
            const int q = (int)(i % kWsStages), s = (int)(i % kWsSlots);
            int64_t nb, nb1;
            int L, nfp;
            mr.get(b, c0, G, i, lane, nb, nb1, L, nfp);
            if (!mb_wait(&sfull[s], (uint32_t)((i / kWsSlots) & 1), polls, abort_flag) ||
                !mb_wait(&tma[q], (uint32_t)((i / kWsStages) & 1), polls, abort_flag)) {
                timed_out = true;
                break;
            }
            const unsigned char *st = STG(q);
            const uint32_t *ids = reinterpret_cast<const uint32_t *>(st + lay.ids);
            const uint32_t *toff = reinterpret_cast<const uint32_t *>(st + lay.toff);
            const float4 *slot = SLOT(s);
            // node groups of 32 (lane = node): slot t of node l at toff[t] + l,
            // one loop over t for the whole warp, consecutive lanes reading
            // consecutive slots
            // Two node groups per pass (group b = a + 32 NR), their slot
            // loads in flight together; b's nodes have no more slots than
            // a's (nodes numbered by decreasing slot count), so a's count
            // ends the loop.  Each node's slots are added in the same order.
            auto emit = [&](int l, float2 sxy, float sz) {
                const float r0 = sxy.x, r1 = sxy.y, r2 = sz;
                if (!isfinite(r0 + r1 + r2)) atomicOr(args.err, ERR_NONFINITE);
                const uint32_t id = ids[l];
                double *o = args.rhs + (id & 0x7fffffffu);
                const double v0 = widen(r0), v1 = widen(r1), v2 = widen(r2);
                if (id & 0x80000000u) {
                    atomicAdd(o, v0);
                    atomicAdd(o + f.n, v1);
                    atomicAdd(o + 2 * f.n, v2);
                } else {
                    o[0] = v0;
                    o[f.n] = v1;
                    o[2 * f.n] = v2;
                }
            };
            for (int g = rw * 32; g < L; g += 64 * NR) {
                const int gb = g + 32 * NR;
                const int la = g + lane, lb = gb + lane;
                float2 sa = make_float2(0.f, 0.f), sb = make_float2(0.f, 0.f);
                float za = 0.f, zb = 0.f;
                // four incidences per step (toff[t + 1] - toff[t] = nodes
                // with more than t slots)
                uint32_t o0 = toff[0];
                for (int t = 0; t < 64; t += 4) {
                    uint32_t o[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) o[u] = toff[t + 1 + u];
                    if (g >= (int)(o[0] - o0)) break;
                    float4 va[4], vb[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const uint32_t lo = u ? o[u - 1] : o0;
                        const int cnt = (int)(o[u] - lo);
                        va[u] = la < cnt ? slot[lo + la] : make_float4(0.f, 0.f, 0.f, 0.f);
                        vb[u] = lb < cnt ? slot[lo + lb] : make_float4(0.f, 0.f, 0.f, 0.f);
                    }
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        sa = __fadd2_rn(sa, make_float2(va[u].x, va[u].y));
                        za += va[u].z;
                        sb = __fadd2_rn(sb, make_float2(vb[u].x, vb[u].y));
                        zb += vb[u].z;
                    }
                    o0 = o[3];
                }
                if (la < L) emit(la, sa, za);
                if (lb < L) emit(lb, sb, zb);
            }
            __syncwarp();
            if (lane == 0) {
                mb_arrive(&sempty[s]);
                mb_arrive(&empty[q]);
            }
        }
    }
    if (bad) atomicOr(args.err, ERR_DETJ);
    if (timed_out) {
        *abort_flag = 1;
        if (lane == 0) atomicOr(args.err, ERR_TIMEOUT);
    }
}

}  // namespace

size_t tet_ws_smem_bytes(int nw, int lmp) { return WsLayout(64 * nw, lmp).total; }

cudaError_t launch_tet_ws(const BucketDev &b, const FieldDev &f, const AsmArgs &a, int sms, cudaStream_t s) {
    if (b.count == 0) return cudaSuccess;
    if (!b.ws_rec || b.etype != FEA_TET04 || b.ws_lmp % 4 || b.ws_lmp > 1024) return cudaErrorInvalidValue;
    const size_t smem = tet_ws_smem_bytes(b.ws_nw, b.ws_lmp);
    if (smem > kMaxBlockSmem) return cudaErrorInvalidValue;
    WsParams tp;
    tp.nu = (a.mask & FEA_TERM_VISC) ? (float)f.nu : 0.f;
    tp.cv = (float)f.c_vreman;
    tp.conv = a.mask & FEA_TERM_CONV;
    tp.pres = a.mask & FEA_TERM_PRES;
    tp.sgs = (a.mask & FEA_TERM_SGS) && a.closure == FEA_CLOSURE_VREMAN;
    tp.want_q = a.closure == FEA_CLOSURE_VREMAN && (tp.sgs || a.nut);
    const WaitLimit polls{a.wait_polls ? a.wait_polls : kWsDefaultPolls, a.wait_polls != 0};
    if (sms <= 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 148;
    }
    auto launch = [&](auto kern, int threads) -> cudaError_t {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        int per_sm = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem);
        if (e != cudaSuccess) return e;
        if (per_sm < 1) return cudaErrorInvalidConfiguration;
        const int64_t grid = std::min<int64_t>(b.ws_nch, (int64_t)per_sm * sms);
        kern<<<(unsigned)grid, threads, smem, s>>>(b, f, a, tp, polls);
        return cudaGetLastError();
    };
    const bool full = tp.conv && tp.pres && tp.sgs && tp.want_q;
#define FEA_WS_LAUNCH(NW, NR)                                                                              \
    return full ? launch(k_tet_ws<NW, NR, true>, 32 * (NW + NR + 1))                                       \
                : launch(k_tet_ws<NW, NR, false>, 32 * (NW + NR + 1))
    switch (b.ws_nw) {
        case 12: FEA_WS_LAUNCH(12, 3);
        case 8: FEA_WS_LAUNCH(8, 4);
        case 4: FEA_WS_LAUNCH(4, 2);
    }
#undef FEA_WS_LAUNCH
    return cudaErrorInvalidValue;
}

}  // namespace fea
