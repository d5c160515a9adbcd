// TET04 chunk kernel (mixed precision) for sm_103a: persistent CTAs with a
// three-stage pipeline (TMA bulk copies + cp.async gathers + compute).
//
// Per element (affine map, constant gradients) the element residual of
// Eq. momentum takes the closed forms of the 4-point rule, which is exact
// for these degree-2 integrands:
//   sum_g W N_a N_b = V (1 + delta_ab) / 20,   sum_g W N_a = V / 4,
//   r_a = - [ (G + tr G I) V/20 (u_a + sum_b u_b) + V/4 grad p
//             + 2 (nu + nu_t) V eps grad N_a ],
// with grad N_k (k = 1..3) the rows of J^-1 = cofactors / det J and
// grad N_0 = -sum_k grad N_k; nu_t = c Delta^2 sqrt(B'/G:G) (Vreman, B' the
// sum of squared cross products of the rows of G), Delta = V^(1/3).
//
// Chunk protocol (same tables as the generic chunk kernel): A. stage the
// chunk's nodes in shared memory, B. element residuals written straight to
// their positions in the chunk's node-sorted incidence list, C. per local
// node: sum its contiguous range, then one FP64 store or atomic add.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>

#include "fea_internal.h"

namespace fea {
namespace {

// FP32 -> FP64 by bit manipulation for normal numbers (keeps the conversion
// off the FP64 pipe); zero, subnormals, inf and nan take the hardware path.
__device__ __forceinline__ double f32_to_f64(float x) {
    const uint32_t b = __float_as_uint(x);
    const uint32_t e = (b >> 23) & 0xffu;
    if (e == 0u || e == 0xffu) return (double)x;
    const uint32_t hi = (b & 0x80000000u) | ((e + 896u) << 20) | ((b & 0x7fffffu) >> 3);
    return __hiloint2double((int)hi, (int)(b << 29));
}

}  // namespace

// ---- async-copy and mbarrier primitives (PTX) -------------------------------
__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// 1-D bulk copy global -> shared (TMA), completion counted on the mbarrier
__device__ __forceinline__ void bulk_load(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_addr(dst)),
                 "l"(src), "r"(bytes), "r"(smem_addr(bar))
                 : "memory");
}
__device__ __forceinline__ void cp_async16(void *dst, const void *src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// bounded wait on an mbarrier phase: false after ~2^22 polls (the caller
// records ERR_TIMEOUT and leaves the chunk loop)
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity) {
    for (int it = 0; it < (1 << 22); ++it)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

// ---- TET04 residual, one element (FP32) --------------------------------------
struct TetParams {
    float nu, cv;
    bool conv, pres, sgs, want_q;
};

__device__ __forceinline__ float vreman_q_fast(float aa, float B) {
    // c sqrt(B'/G:G) without c; 0 for a vanishing gradient
    return (B > 0.f && aa > 0.f) ? B * rsqrtf(B) * rsqrtf(aa) : 0.f;
}

template <bool FULL>
__device__ __forceinline__ void tet_element(const float4 xs[4], const float4 us[4], const TetParams &tp_in, float4 r[4],
                                            float &nut, bool &bad) {
    TetParams tp = tp_in;
    if (FULL) tp.conv = tp.pres = tp.sgs = tp.want_q = true;
    float d[3][3];
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        d[q][0] = xs[q + 1].x - xs[0].x;
        d[q][1] = xs[q + 1].y - xs[0].y;
        d[q][2] = xs[q + 1].z - xs[0].z;
    }
    // cofactors: rows of det * J^-1
    float cf[3][3];
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        const float *a = d[(q + 1) % 3], *b = d[(q + 2) % 3];
        cf[q][0] = a[1] * b[2] - a[2] * b[1];
        cf[q][1] = a[2] * b[0] - a[0] * b[2];
        cf[q][2] = a[0] * b[1] - a[1] * b[0];
    }
    const float det = d[0][0] * cf[0][0] + d[0][1] * cf[0][1] + d[0][2] * cf[0][2];
    if (!(det > 0.f)) bad = true;
    const float inv = __fdividef(1.f, det);
    const float V = det * (1.f / 6.f);
    float gN[4][3];
#pragma unroll
    for (int q = 0; q < 3; ++q)
#pragma unroll
        for (int j = 0; j < 3; ++j) gN[q + 1][j] = cf[q][j] * inv;
#pragma unroll
    for (int j = 0; j < 3; ++j) gN[0][j] = -(gN[1][j] + gN[2][j] + gN[3][j]);
    const float du[3][3] = {{us[1].x - us[0].x, us[1].y - us[0].y, us[1].z - us[0].z},
                            {us[2].x - us[0].x, us[2].y - us[0].y, us[2].z - us[0].z},
                            {us[3].x - us[0].x, us[3].y - us[0].y, us[3].z - us[0].z}};
    const float dp[3] = {us[1].w - us[0].w, us[2].w - us[0].w, us[3].w - us[0].w};
    float G[3][3], gp[3];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        gp[j] = dp[0] * gN[1][j] + dp[1] * gN[2][j] + dp[2] * gN[3][j];
#pragma unroll
        for (int i = 0; i < 3; ++i) G[i][j] = du[0][i] * gN[1][j] + du[1][i] * gN[2][j] + du[2][i] * gN[3][j];
    }
    nut = 0.f;
    if (tp.want_q) {
        float aa = 0.f, B = 0.f;
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j) aa += G[i][j] * G[i][j];
#pragma unroll
        for (int p = 0; p < 3; ++p) {
            const int i = p == 2 ? 1 : 0, j = p == 0 ? 1 : 2;
            const float x = G[i][1] * G[j][2] - G[i][2] * G[j][1];
            const float y = G[i][2] * G[j][0] - G[i][0] * G[j][2];
            const float z = G[i][0] * G[j][1] - G[i][1] * G[j][0];
            B += x * x + y * y + z * z;
        }
        // Delta^2 = V^(2/3); c sqrt(B'/G:G) = c B' rsqrt(B' G:G)
        nut = tp.cv * __powf(fabsf(V), 2.f / 3.f) * vreman_q_fast(aa, B);
    }
    // negated coefficients
    const float s2 = -2.f * (tp.nu + (tp.sgs ? nut : 0.f)) * V;
    float ns[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        ns[i][i] = s2 * G[i][i];
#pragma unroll
        for (int j = i + 1; j < 3; ++j) ns[i][j] = ns[j][i] = 0.5f * s2 * (G[i][j] + G[j][i]);
    }
    const float trG = G[0][0] + G[1][1] + G[2][2];
    const float nv20 = tp.conv ? -0.05f * V : 0.f;
    float nA[3][3], su[3], npg[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
#pragma unroll
        for (int j = 0; j < 3; ++j) nA[i][j] = nv20 * (i == j ? G[i][j] + trG : G[i][j]);
        npg[i] = tp.pres ? -0.25f * V * gp[i] : 0.f;
    }
    su[0] = us[0].x + us[1].x + us[2].x + us[3].x;
    su[1] = us[0].y + us[1].y + us[2].y + us[3].y;
    su[2] = us[0].z + us[1].z + us[2].z + us[3].z;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        const float m0 = us[a].x + su[0], m1 = us[a].y + su[1], m2 = us[a].z + su[2];
        float v[3];
#pragma unroll
        for (int i = 0; i < 3; ++i)
            v[i] = npg[i] + nA[i][0] * m0 + nA[i][1] * m1 + nA[i][2] * m2 + ns[i][0] * gN[a][0] +
                   ns[i][1] * gN[a][1] + ns[i][2] * gN[a][2];
        r[a] = make_float4(v[0], v[1], v[2], 0.f);
    }
}

// ---- TET04 residual, two elements at once (packed FP32, sm_100+) -----------
// The same arithmetic as tet_element, on float2 lanes (.x: element A, .y:
// element B) with the paired FP32 instructions (one FFMA2 / FMUL2 / FADD2
// does the operation of both elements).  Delta^2 = V^(2/3) and
// sqrt(B'/G:G) = B' rsqrt(B' G:G) use the fast hardware functions.
__device__ __forceinline__ float2 p_add(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 p_sub(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }
__device__ __forceinline__ float2 p_mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 p_fma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 p_s(float v) { return make_float2(v, v); }

template <bool FULL>
__device__ __forceinline__ void tet_element_x2(const float4 xa[4], const float4 ua[4], const float4 xb[4],
                                               const float4 ub[4], const TetParams &tp_in, float4 ra[4], float4 rb[4],
                                               float2 &nut, bool &bad) {
    TetParams tp = tp_in;
    if (FULL) tp.conv = tp.pres = tp.sgs = tp.want_q = true;
    float2 X[4][3], U[4][3], P[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        X[a][0] = make_float2(xa[a].x, xb[a].x);
        X[a][1] = make_float2(xa[a].y, xb[a].y);
        X[a][2] = make_float2(xa[a].z, xb[a].z);
        U[a][0] = make_float2(ua[a].x, ub[a].x);
        U[a][1] = make_float2(ua[a].y, ub[a].y);
        U[a][2] = make_float2(ua[a].z, ub[a].z);
        P[a] = make_float2(ua[a].w, ub[a].w);
    }
    float2 d[3][3], nd[3][3];
#pragma unroll
    for (int q = 0; q < 3; ++q)
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            d[q][k] = p_sub(X[q + 1][k], X[0][k]);
            nd[q][k] = p_sub(X[0][k], X[q + 1][k]);
        }
    // cofactors: rows of det * J^-1
    float2 cf[3][3];
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        const float2 *a = d[(q + 1) % 3], *b = d[(q + 2) % 3], *nb = nd[(q + 2) % 3];
        cf[q][0] = p_fma(a[1], b[2], p_mul(a[2], nb[1]));
        cf[q][1] = p_fma(a[2], b[0], p_mul(a[0], nb[2]));
        cf[q][2] = p_fma(a[0], b[1], p_mul(a[1], nb[0]));
    }
    const float2 det = p_fma(d[0][0], cf[0][0], p_fma(d[0][1], cf[0][1], p_mul(d[0][2], cf[0][2])));
    if (!(det.x > 0.f) || !(det.y > 0.f)) bad = true;
    const float2 inv = make_float2(__fdividef(1.f, det.x), __fdividef(1.f, det.y));
    const float2 V = p_mul(det, p_s(1.f / 6.f));
    float2 gN[4][3];
#pragma unroll
    for (int q = 0; q < 3; ++q)
#pragma unroll
        for (int j = 0; j < 3; ++j) gN[q + 1][j] = p_mul(cf[q][j], inv);
#pragma unroll
    for (int j = 0; j < 3; ++j) gN[0][j] = p_mul(p_add(p_add(gN[1][j], gN[2][j]), gN[3][j]), p_s(-1.f));
    float2 du[3][3], dp[3];
#pragma unroll
    for (int q = 0; q < 3; ++q) {
#pragma unroll
        for (int i = 0; i < 3; ++i) du[q][i] = p_sub(U[q + 1][i], U[0][i]);
        dp[q] = p_sub(P[q + 1], P[0]);
    }
    float2 G[3][3], gp[3];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        gp[j] = p_fma(dp[0], gN[1][j], p_fma(dp[1], gN[2][j], p_mul(dp[2], gN[3][j])));
#pragma unroll
        for (int i = 0; i < 3; ++i)
            G[i][j] = p_fma(du[0][i], gN[1][j], p_fma(du[1][i], gN[2][j], p_mul(du[2][i], gN[3][j])));
    }
    nut = make_float2(0.f, 0.f);
    if (tp.want_q) {
        float2 aa = p_s(0.f), B = p_s(0.f);
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j) aa = p_fma(G[i][j], G[i][j], aa);
#pragma unroll
        for (int pq = 0; pq < 3; ++pq) {
            const int i = pq == 2 ? 1 : 0, j = pq == 0 ? 1 : 2;
            const float2 x = p_sub(p_mul(G[i][1], G[j][2]), p_mul(G[i][2], G[j][1]));
            const float2 y = p_sub(p_mul(G[i][2], G[j][0]), p_mul(G[i][0], G[j][2]));
            const float2 z = p_sub(p_mul(G[i][0], G[j][1]), p_mul(G[i][1], G[j][0]));
            B = p_fma(x, x, p_fma(y, y, p_fma(z, z, B)));
        }
        // Delta^2 = V^(2/3)
        const float2 d2 = make_float2(__powf(fabsf(V.x), 2.f / 3.f), __powf(fabsf(V.y), 2.f / 3.f));
        nut = p_mul(p_mul(p_s(tp.cv), d2), make_float2(vreman_q_fast(aa.x, B.x), vreman_q_fast(aa.y, B.y)));
    }
    // negated coefficients
    const float2 s2 = p_mul(p_s(-2.f), p_mul(p_add(p_s(tp.nu), tp.sgs ? nut : p_s(0.f)), V));
    const float2 hs2 = p_mul(s2, p_s(0.5f));
    float2 ns[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        ns[i][i] = p_mul(s2, G[i][i]);
#pragma unroll
        for (int j = i + 1; j < 3; ++j) ns[i][j] = ns[j][i] = p_mul(hs2, p_add(G[i][j], G[j][i]));
    }
    const float2 trG = p_add(p_add(G[0][0], G[1][1]), G[2][2]);
    const float2 nv20 = tp.conv ? p_mul(p_s(-0.05f), V) : p_s(0.f);
    const float2 nv4 = tp.pres ? p_mul(p_s(-0.25f), V) : p_s(0.f);
    float2 nA[3][3], c[3];
    float2 su[3];
#pragma unroll
    for (int j = 0; j < 3; ++j) su[j] = p_add(p_add(U[0][j], U[1][j]), p_add(U[2][j], U[3][j]));
#pragma unroll
    for (int i = 0; i < 3; ++i) {
#pragma unroll
        for (int j = 0; j < 3; ++j) nA[i][j] = p_mul(nv20, i == j ? p_add(G[i][j], trG) : G[i][j]);
        // the node-independent part: -V/4 grad p - V/20 A sum_b u_b
        c[i] = p_fma(nA[i][0], su[0], p_fma(nA[i][1], su[1], p_fma(nA[i][2], su[2], p_mul(nv4, gp[i]))));
    }
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        float2 v[3];
#pragma unroll
        for (int i = 0; i < 3; ++i)
            v[i] = p_fma(nA[i][0], U[a][0],
                         p_fma(nA[i][1], U[a][1],
                               p_fma(nA[i][2], U[a][2],
                                     p_fma(ns[i][0], gN[a][0],
                                           p_fma(ns[i][1], gN[a][1], p_fma(ns[i][2], gN[a][2], c[i]))))));
        ra[a] = make_float4(v[0].x, v[1].x, v[2].x, 0.f);
        rb[a] = make_float4(v[0].y, v[1].y, v[2].y, 0.f);
    }
}

// Residual slot k lives at k + k/8: node ranges of 8 m incidences (24 for the
// interior nodes of a Kuhn-split grid) would otherwise start on the same
// float4 bank group in every lane of the node phase.
__device__ __forceinline__ int swz(int k) { return k + (k >> 3); }

// ---- persistent, pipelined TET04 chunk kernel ---------------------------------
// Shared memory: residual slots [4 C + C/2] (swizzled), then three stage buffers, each with
// the chunk's node records [LM], gathered (u, v, w, p) [LM], incidence ranges
// [LM] and element records [C] (4 local node ids + 4 incidence positions),
// then three mbarriers.  Iteration i computes chunk c_i while the TMA engine
// loads chunk c_{i+2} and cp.async gathers the field values of c_{i+1}.
// PAIR: each thread computes elements el and el + T together (packed FP32).
// FULL: all terms with the Vreman closure (the flags fold at compile time).
template <int T, bool PAIR, bool FULL>
__global__ void __launch_bounds__(T) k_tet_pipe(BucketDev b, FieldDev f, AsmArgs args, TetParams tp) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int C = b.chunk_elems, LM = b.max_chunk_nodes;
    float4 *sR = reinterpret_cast<float4 *>(smem);
    unsigned char *base = smem + (size_t)72 * C;
    const size_t bufsz = (size_t)36 * LM + (size_t)16 * C;
    uint64_t *mbar = reinterpret_cast<uint64_t *>(base + 3 * bufsz);
    int *abort_flag = reinterpret_cast<int *>(mbar + 3);
    auto REC = [&](int q) { return reinterpret_cast<float4 *>(base + q * bufsz); };
    auto UP = [&](int q) { return reinterpret_cast<float4 *>(base + q * bufsz + (size_t)16 * LM); };
    auto RNG = [&](int q) { return reinterpret_cast<uint32_t *>(base + q * bufsz + (size_t)32 * LM); };
    auto ELR = [&](int q) { return reinterpret_cast<uint4 *>(base + q * bufsz + (size_t)36 * LM); };
    const uint4 *elem_g = reinterpret_cast<const uint4 *>(b.lconn);
    const int tid = threadIdx.x;
    const int64_t G = gridDim.x, c0 = blockIdx.x, nch = b.n_chunks;
    // a kernel launched after this one as a programmatic dependent (the
    // FP64-Jacobian PEN06 category) may start as soon as CTAs of this one
    // retire: it fills the SMs of this kernel's tail
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    if (tid == 0) {
        for (int q = 0; q < 3; ++q) mbar_init(&mbar[q], 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    auto issue_tma = [&](int64_t c, int q) {
        if (c >= nch) return;
        const int64_t nb = b.chunk_node_off[c];
        const uint32_t Lp = (uint32_t)(b.chunk_node_off[c + 1] - nb);
        const int64_t e0 = c * C;
        const uint32_t ne = (uint32_t)min((int64_t)C, b.count - e0);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_expect_tx(&mbar[q], Lp * 20u + ne * 16u);
        bulk_load(REC(q), b.chunk_rec + nb, Lp * 16u, &mbar[q]);
        bulk_load(RNG(q), b.inc_range + nb, Lp * 4u, &mbar[q]);
        bulk_load(ELR(q), elem_g + e0, ne * 16u, &mbar[q]);
    };
    auto issue_gather = [&](int64_t c, int q) {
        const int L = b.chunk_nodes[c];
        const float4 *rec = REC(q);
        float4 *up = UP(q);
        for (int j = tid; j < L; j += T) cp_async16(up + j, f.up32 + (__float_as_int(rec[j].w) & 0x7fffffff));
        cp_async_commit();
    };
    bool bad = false;
    if (tid == 0) {
        issue_tma(c0, 0);
        issue_tma(c0 + G, 1);
    }
    if (c0 < nch) {
        if (mbar_wait_bounded(&mbar[0], 0))
            issue_gather(c0, 0);
        else
            atomicExch(abort_flag, 1);
    }
    for (int i = 0;; ++i) {
        const int64_t c = c0 + (int64_t)i * G;
        if (c >= nch) break;
        const int q = i % 3, q1 = (i + 1) % 3, q2 = (i + 2) % 3;
        const bool more = c + G < nch;
        if (more) {
            if (mbar_wait_bounded(&mbar[q1], (uint32_t)(((i + 1) / 3) & 1)))
                issue_gather(c + G, q1);
            else
                atomicExch(abort_flag, 1);
        }
        if (more)
            cp_async_wait<1>();
        else
            cp_async_wait<0>();
        __syncthreads();
        if (*abort_flag) break;
        // stage q2 last held chunk i-1, whose node phase every thread has
        // finished before the barrier above: it can be refilled now
        if (tid == 0) issue_tma(c + 2 * G, q2);
        // B: element residuals into their node-sorted incidence positions
        const int64_t e0 = c * C;
        const int ne = (int)min((int64_t)C, b.count - e0);
        const float4 *rec = REC(q);
        const float4 *up = UP(q);
        const uint4 *elr = ELR(q);
        if constexpr (PAIR) {
            for (int el = tid; el < ne; el += 2 * T) {
                const int elb = el + T;
                const bool hasb = elb < ne;
                const uint4 era = elr[el], erb = elr[hasb ? elb : el];
                const int la[4] = {(int)(era.x & 0xffffu), (int)(era.x >> 16), (int)(era.y & 0xffffu),
                                   (int)(era.y >> 16)};
                const int lb[4] = {(int)(erb.x & 0xffffu), (int)(erb.x >> 16), (int)(erb.y & 0xffffu),
                                   (int)(erb.y >> 16)};
                float4 xa[4], ua[4], xb[4], ub[4], ra[4], rb[4];
#pragma unroll
                for (int a = 0; a < 4; ++a) {
                    xa[a] = rec[la[a]];
                    ua[a] = up[la[a]];
                    xb[a] = rec[lb[a]];
                    ub[a] = up[lb[a]];
                }
                float2 nut;
                tet_element_x2<FULL>(xa, ua, xb, ub, tp, ra, rb, nut, bad);
                sR[swz((int)(era.z & 0xffffu))] = ra[0];
                sR[swz((int)(era.z >> 16))] = ra[1];
                sR[swz((int)(era.w & 0xffffu))] = ra[2];
                sR[swz((int)(era.w >> 16))] = ra[3];
                if (hasb) {
                    sR[swz((int)(erb.z & 0xffffu))] = rb[0];
                    sR[swz((int)(erb.z >> 16))] = rb[1];
                    sR[swz((int)(erb.w & 0xffffu))] = rb[2];
                    sR[swz((int)(erb.w >> 16))] = rb[3];
                }
                if (args.nut) {
                    float4 *nu4 = reinterpret_cast<float4 *>(args.nut);
                    nu4[__ldg(&b.orig[e0 + el])] = make_float4(nut.x, nut.x, nut.x, nut.x);
                    if (hasb) nu4[__ldg(&b.orig[e0 + elb])] = make_float4(nut.y, nut.y, nut.y, nut.y);
                }
            }
        } else {
            for (int el = tid; el < ne; el += T) {
                const uint4 er = elr[el];
                const int li[4] = {(int)(er.x & 0xffffu), (int)(er.x >> 16), (int)(er.y & 0xffffu),
                                   (int)(er.y >> 16)};
                const int ps[4] = {(int)(er.z & 0xffffu), (int)(er.z >> 16), (int)(er.w & 0xffffu),
                                   (int)(er.w >> 16)};
                float4 xs[4], us[4], r[4];
#pragma unroll
                for (int a = 0; a < 4; ++a) {
                    xs[a] = rec[li[a]];
                    us[a] = up[li[a]];
                }
                float nut;
                tet_element<FULL>(xs, us, tp, r, nut, bad);
#pragma unroll
                for (int a = 0; a < 4; ++a) sR[swz(ps[a])] = r[a];
                if (args.nut) {
                    const int64_t o = (int64_t)__ldg(&b.orig[e0 + el]);
                    reinterpret_cast<float4 *>(args.nut)[o] = make_float4(nut, nut, nut, nut);
                }
            }
        }
        __syncthreads();
        // C: node sums -> FP64 global RHS (store if exclusive, else atomic add).
        // The next iteration's first barrier orders this phase before the
        // residual slots and this stage's buffers are written again.
        const int L = b.chunk_nodes[c];
        const uint32_t *rng = RNG(q);
        for (int j = tid; j < L; j += T) {
            const uint32_t rg = rng[j];
            const int st = (int)(rg & 0xffffu), cnt = (int)(rg >> 16);
            float s0 = 0.f, s1 = 0.f, s2 = 0.f;
            for (int t = 0; t < cnt; ++t) {
                const float4 v = sR[swz(st + t)];
                s0 += v.x;
                s1 += v.y;
                s2 += v.z;
            }
            if (!isfinite(s0 + s1 + s2)) atomicOr(args.err, ERR_NONFINITE);
            const int bits = __float_as_int(rec[j].w);
            double *r0 = args.rhs + (bits & 0x7fffffff);
            const double v0 = f32_to_f64(s0), v1 = f32_to_f64(s1), v2 = f32_to_f64(s2);
            if (bits < 0) {
                atomicAdd(r0, v0);
                atomicAdd(r0 + f.n, v1);
                atomicAdd(r0 + 2 * f.n, v2);
            } else {
                r0[0] = v0;
                r0[f.n] = v1;
                r0[2 * f.n] = v2;
            }
        }
    }
    if (bad) atomicOr(args.err, ERR_DETJ);
    cp_async_wait<0>();
    if (*abort_flag && tid == 0) {
        atomicOr(args.err, ERR_TIMEOUT);
        // let any bulk copy still in flight land before the CTA's shared memory is released
        for (int q = 0; q < 3; ++q) mbar_wait_bounded(&mbar[q], 0), mbar_wait_bounded(&mbar[q], 1);
    }
}

size_t tet_pipe_smem_bytes(const BucketDev &b) {
    return (size_t)72 * b.chunk_elems + 3 * ((size_t)36 * b.max_chunk_nodes + (size_t)16 * b.chunk_elems) + 3 * 8 + 16;
}

cudaError_t launch_tet_pipe(const BucketDev &b, const FieldDev &f, const AsmArgs &a, int threads, int sms,
                           cudaStream_t s) {
    if (b.count == 0) return cudaSuccess;
    if (!b.lconn || b.etype != FEA_TET04 || b.max_chunk_nodes % 4) return cudaErrorInvalidValue;
    const size_t smem = tet_pipe_smem_bytes(b);
    TetParams tp;
    tp.nu = (a.mask & FEA_TERM_VISC) ? (float)f.nu : 0.f;
    tp.cv = (float)f.c_vreman;
    tp.conv = a.mask & FEA_TERM_CONV;
    tp.pres = a.mask & FEA_TERM_PRES;
    tp.sgs = (a.mask & FEA_TERM_SGS) && a.closure == FEA_CLOSURE_VREMAN;
    tp.want_q = a.closure == FEA_CLOSURE_VREMAN && (tp.sgs || a.nut);
    static int sm_count = 0;
    if (sms <= 0) {
        if (!sm_count) {
            int dev = 0;
            cudaGetDevice(&dev);
            cudaDeviceGetAttribute(&sm_count, cudaDevAttrMultiProcessorCount, dev);
        }
        sms = sm_count > 0 ? sm_count : 148;
    }
    auto launch = [&](auto kern, int T) -> cudaError_t {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        int per_sm = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, T, smem);
        if (e != cudaSuccess) return e;
        if (per_sm < 1) return cudaErrorInvalidConfiguration;
        const int64_t grid = std::min<int64_t>(b.n_chunks, (int64_t)per_sm * sms);
        kern<<<(unsigned)grid, T, smem, s>>>(b, f, a, tp);
        return cudaGetLastError();
    };
    // two elements per thread whenever every thread has at least two
    const bool pair = b.chunk_elems >= 2 * threads;
    const bool full = tp.conv && tp.pres && tp.sgs && tp.want_q;
#define FEA_TET_LAUNCH(TT)                                                                             \
    return pair ? (full ? launch(k_tet_pipe<TT, true, true>, TT) : launch(k_tet_pipe<TT, true, false>, TT)) \
                : (full ? launch(k_tet_pipe<TT, false, true>, TT) : launch(k_tet_pipe<TT, false, false>, TT))
    if (threads >= 512) FEA_TET_LAUNCH(512);
    if (threads >= 256) FEA_TET_LAUNCH(256);
    FEA_TET_LAUNCH(128);
#undef FEA_TET_LAUNCH
}

}  // namespace fea
