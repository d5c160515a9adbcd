// Learned eddy-viscosity closure: a 6 -> 64 -> 64 -> 64 -> 1 MLP (SiLU hidden
// layers, softplus output) evaluated on BF16 tensor cores with FP32
// accumulation, warp-cooperatively on tiles of 16 rows.
//
// Inputs per row (Gauss point or element), dimensionless: the invariants of
// S = (G+G^T)/2 and O = (G-G^T)/2 of the velocity gradient G_ij = du_i/dx_j
// over powers of g = |G| (g^2 = tr S^2 - tr O^2),
//   x_1..5 = (tr S^2, tr O^2, tr S^3, tr S O^2, tr S^2 O^2) / g^(2, 2, 3, 3, 4),
// and the element Reynolds number x_6 = log(Delta^2 g / nu), normalised as
// (x - mean) / std; output the coefficient C = out_scale softplus(z), and
// nu_t = C Delta^2 g (zero where g = 0, whose features are all zero).
//
// Tensor-core tiles: mma.sync m16n8k16 (row.col, BF16 in, FP32 accumulate).
// For lane l: g = l / 4, t = l % 4; an A fragment holds rows (g, g+8) and
// columns (2t, 2t+1, 2t+8, 2t+9) of a 16 x 16 tile; a C fragment holds rows
// (g, g+8), columns (2t, 2t+1) of a 16 x 8 tile.  The C fragments of the
// n-tiles 2k and 2k+1 of one layer are exactly the A fragment of k-step k of
// the next layer, so the hidden activations never leave registers.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace fea {

constexpr int kMlpIn = 6, kMlpH = 64;
constexpr int kMlpParams = kMlpH * kMlpIn + kMlpH + 2 * (kMlpH * kMlpH + kMlpH) + kMlpH + 1;  // 8,833
constexpr int kW1Pitch = 24;  // bf16 per row of W1 [64][16 used + pad]: 12 words, conflict-free fragments
constexpr int kWPitch = 72;   // bf16 per row of W2, W3 [64][64 + pad]: 36 words

// Inference part of the device-resident MLP (copied into shared memory by
// the kernels that evaluate it).
struct __align__(16) MlpInfer {
    uint16_t w1[kMlpH][kW1Pitch];  // bf16 W1[out][in], inputs 6..15 zero
    uint16_t w2[kMlpH][kWPitch];   // bf16 W2[out][in]
    uint16_t w3[kMlpH][kWPitch];
    float b1[kMlpH], b2[kMlpH], b3[kMlpH], w4[kMlpH];
    float b4;
    float mean[kMlpIn], istd[kMlpIn];
    float out_scale;
};

// Inference part plus the transposed weights used by the backward pass.
struct __align__(16) MlpWeights {
    MlpInfer inf;
    uint16_t w2t[kMlpH][kWPitch];  // bf16 W2^T[in][out]
    uint16_t w3t[kMlpH][kWPitch];
};

__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi) {
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t *>(&v);
}

__device__ __forceinline__ void mma_bf16_16816(float c[4], const uint32_t a[4], uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ float silu_f(float z) { return z / (1.0f + __expf(-z)); }
__device__ __forceinline__ float sigmoid_f(float z) { return 1.0f / (1.0f + __expf(-z)); }
__device__ __forceinline__ float softplus_f(float z) { return z > 20.0f ? z : log1pf(__expf(z)); }

// A fragment of the first layer from a per-warp shared tile of normalised
// features: feat[row][kW1Pitch] bf16 (columns 6..15 zero); `row0` selects
// the 16-row half of a 32-row warp tile.
__device__ __forceinline__ void mlp_load_a1(const uint16_t *feat, int row0, uint32_t a[4]) {
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    const uint32_t *f32 = reinterpret_cast<const uint32_t *>(feat);
    constexpr int P = kW1Pitch / 2;  // words per row
    a[0] = f32[(row0 + g) * P + t];
    a[1] = f32[(row0 + g + 8) * P + t];
    a[2] = f32[(row0 + g) * P + 4 + t];
    a[3] = f32[(row0 + g + 8) * P + 4 + t];
}

// One hidden layer: C = A W^T + b, then SiLU, returned as the next layer's
// A fragments.  K = 16 (first layer, W pitch kW1Pitch) or 64.
template <int KSTEPS, int PITCH>
__device__ __forceinline__ void mlp_layer(const uint32_t a[KSTEPS][4], const uint16_t (*W)[PITCH], const float *bias,
                                          uint32_t out[4][4], float *zs /* optional [8][4] pre-activations */) {
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    float c[8][4];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        c[j][0] = c[j][1] = c[j][2] = c[j][3] = 0.f;
        const uint32_t *row = reinterpret_cast<const uint32_t *>(W[8 * j + g]);
#pragma unroll
        for (int kk = 0; kk < KSTEPS; ++kk) mma_bf16_16816(c[j], a[kk], row[8 * kk + t], row[8 * kk + 4 + t]);
        const float b0 = bias[8 * j + 2 * t], b1 = bias[8 * j + 2 * t + 1];
        c[j][0] += b0;
        c[j][1] += b1;
        c[j][2] += b0;
        c[j][3] += b1;
        if (zs) {
#pragma unroll
            for (int q = 0; q < 4; ++q) zs[j * 4 + q] = c[j][q];
        }
    }
#pragma unroll
    for (int kk = 0; kk < 4; ++kk) {
        out[kk][0] = pack_bf16x2(silu_f(c[2 * kk][0]), silu_f(c[2 * kk][1]));
        out[kk][1] = pack_bf16x2(silu_f(c[2 * kk][2]), silu_f(c[2 * kk][3]));
        out[kk][2] = pack_bf16x2(silu_f(c[2 * kk + 1][0]), silu_f(c[2 * kk + 1][1]));
        out[kk][3] = pack_bf16x2(silu_f(c[2 * kk + 1][2]), silu_f(c[2 * kk + 1][3]));
    }
}

// z of the output layer for rows g (zg) and g+8 (zg8), valid in every lane,
// from the last hidden layer's A fragments (BF16 activations, FP32 dot).
__device__ __forceinline__ void mlp_output(const uint32_t h[4][4], const float *w4, float b4, float &zg, float &zg8) {
    const int lane = threadIdx.x & 31, t = lane & 3;
    float pg = 0.f, pg8 = 0.f;
#pragma unroll
    for (int kk = 0; kk < 4; ++kk) {
#pragma unroll
        for (int half = 0; half < 2; ++half) {
            const int col = 16 * kk + 8 * half + 2 * t;
            const __nv_bfloat162 vg = *reinterpret_cast<const __nv_bfloat162 *>(&h[kk][2 * half]);
            const __nv_bfloat162 vg8 = *reinterpret_cast<const __nv_bfloat162 *>(&h[kk][2 * half + 1]);
            pg += __low2float(vg) * w4[col] + __high2float(vg) * w4[col + 1];
            pg8 += __low2float(vg8) * w4[col] + __high2float(vg8) * w4[col + 1];
        }
    }
    pg += __shfl_xor_sync(0xffffffffu, pg, 1);
    pg += __shfl_xor_sync(0xffffffffu, pg, 2);
    pg8 += __shfl_xor_sync(0xffffffffu, pg8, 1);
    pg8 += __shfl_xor_sync(0xffffffffu, pg8, 2);
    zg = pg + b4;
    zg8 = pg8 + b4;
}

// Full forward pass of a 16-row tile given the first layer's A fragment.
__device__ __forceinline__ void mlp_tile_forward(const MlpInfer &w, const uint32_t a1[4], float &zg, float &zg8) {
    uint32_t h1[4][4], h2[4][4], h3[4][4];
    uint32_t a1k[1][4] = {{a1[0], a1[1], a1[2], a1[3]}};
    mlp_layer<1, kW1Pitch>(a1k, w.w1, w.b1, h1, nullptr);
    mlp_layer<4, kWPitch>(h1, w.w2, w.b2, h2, nullptr);
    mlp_layer<4, kWPitch>(h2, w.w3, w.b3, h3, nullptr);
    mlp_output(h3, w.w4, w.b4, zg, zg8);
}

// Copies the inference weights into shared memory (all threads of the CTA;
// ends with a barrier).
__device__ __forceinline__ void mlp_copy_infer(const MlpInfer *g, MlpInfer *s) {
    const int4 *src = reinterpret_cast<const int4 *>(g);
    int4 *dst = reinterpret_cast<int4 *>(s);
    for (int k = threadIdx.x; k < (int)(sizeof(MlpInfer) / 16); k += blockDim.x) dst[k] = src[k];
    __syncthreads();
}

// ---------------------------------------------------------------------------
// Inference layout of the same network for the fused closure and the batched
// forward.  The weights keep their BF16 values (the precision the network is
// trained with) but are stored as FP16, which holds every such value exactly,
// and the activations travel as FP16: the packed SiLU below loses about
// |z| 2^-12 to cancellation where z << 0, eight times less than in BF16.
// The hidden layers' weights and biases are stored halved, so a layer's
// accumulator holds h = z/2 and SiLU(z) = h (1 + tanh h) costs one packed
// tanh and one packed FMA per two activations.  The output weights are split
// into two FP16 rows, hi = bf16(w4) and lo = w4 - hi, so the output layer is
// one more tensor-core tile whose columns 0 and 1 add up to the FP32 dot.
// Normalised features are clamped to +-64 (far outside any training data)
// so that no FP16 value overflows.
struct __align__(16) MlpFast {
    uint16_t w1[kMlpH][8];         // f16 W1/2 [out][in], inputs 6, 7 zero
    uint16_t w2[kMlpH][kWPitch];   // f16 W2/2 [out][in]
    uint16_t w3[kMlpH][kWPitch];   // f16 W3/2
    uint16_t w4[8][kWPitch];       // rows 0, 1: hi and lo parts of w4; rows 2..7 zero
    float b1[kMlpH], b2[kMlpH], b3[kMlpH];   // halved
    float b4;
    float mean[kMlpIn], istd[kMlpIn];
    float env_lo[kMlpIn], env_hi[kMlpIn];   // training envelope, normalised units (+-inf: none)
    float out_scale;
    int env_on;                              // any finite envelope bound
};
constexpr float kFeatClamp = 64.0f;

// Per-warp scratch of the fused closure for ng Gauss points per element, 32
// elements (one per lane): normalised feature rows [ng*32][8] f16 (row
// g*32 + lane), the per-point matrices S [ng][9][32] f32 the subgrid term
// needs once nu_t is known, and nu_t [ng*32] f32.
__host__ __device__ constexpr size_t mlp_feat_bytes(int ng) { return (size_t)ng * 32 * 16; }
__host__ __device__ constexpr size_t mlp_s_bytes(int ng) { return (size_t)ng * 9 * 32 * 4; }
// after them: the network's coefficient [ng*32] f32, Vreman's q = nu_t /
// Delta^2 [ng*32] f32 (for the fallback) and g = |G| [ng*32] f32
__host__ __device__ constexpr size_t mlp_warp_scratch_bytes(int ng) {
    return mlp_feat_bytes(ng) + mlp_s_bytes(ng) + (size_t)ng * 32 * 4 * 3;
}

__device__ __forceinline__ void mlp_copy_fast(const MlpFast *g, MlpFast *s) {
    const int4 *src = reinterpret_cast<const int4 *>(g);
    int4 *dst = reinterpret_cast<int4 *>(s);
    for (int k = threadIdx.x; k < (int)(sizeof(MlpFast) / 16); k += blockDim.x) dst[k] = src[k];
    __syncthreads();
}

__device__ __forceinline__ void ldsm_x4(uint32_t r[4], const void *p) {
    const uint32_t a = (uint32_t)__cvta_generic_to_shared(p);
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(a));
}

__device__ __forceinline__ uint32_t pack_f16x2(float lo, float hi) {
    __half2 v = __floats2half2_rn(lo, hi);
    return *reinterpret_cast<uint32_t *>(&v);
}

__device__ __forceinline__ void mma_f16_16816(float c[4], const uint32_t a[4], uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ void mma_f16_1688(float c[4], uint32_t a0, uint32_t a1, uint32_t b0) {
    asm volatile(
        "mma.sync.aligned.m16n8k8.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5}, {%6}, {%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a0), "r"(a1), "r"(b0));
}

// SiLU of two halved pre-activations, packed FP16: h (1 + tanh h), h = z/2.
__device__ __forceinline__ uint32_t silu_half_f16x2(float hlo, float hhi) {
    const uint32_t h = pack_f16x2(hlo, hhi);
    uint32_t th, out;
    asm("tanh.approx.f16x2 %0, %1;" : "=r"(th) : "r"(h));
    asm("fma.rn.f16x2 %0, %1, %2, %1;" : "=r"(out) : "r"(h), "r"(th));
    return out;
}

__device__ __forceinline__ void fast_bias(float c[8][4], const float *b) {
    const int t = threadIdx.x & 3;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const float2 v = *reinterpret_cast<const float2 *>(b + 8 * j + 2 * t);
        c[j][0] = c[j][2] = v.x;
        c[j][1] = c[j][3] = v.y;
    }
}

// C fragments of 8 n-tiles -> SiLU -> A fragments of the next layer's 4 k-steps
__device__ __forceinline__ void fast_silu(const float c[8][4], uint32_t h[4][4]) {
#pragma unroll
    for (int kk = 0; kk < 4; ++kk) {
        h[kk][0] = silu_half_f16x2(c[2 * kk][0], c[2 * kk][1]);
        h[kk][1] = silu_half_f16x2(c[2 * kk][2], c[2 * kk][3]);
        h[kk][2] = silu_half_f16x2(c[2 * kk + 1][0], c[2 * kk + 1][1]);
        h[kk][3] = silu_half_f16x2(c[2 * kk + 1][2], c[2 * kk + 1][3]);
    }
}

// One 64 -> 64 hidden layer for two 16-row tiles; B fragments by ldmatrix
// (matrix q of a load: n-tile 2jp + q/2, k half q%2).
__device__ __forceinline__ void fast_layer64(const uint32_t hin[2][4][4], const uint16_t (*W)[kWPitch],
                                             const float *bias, uint32_t hout[2][4][4]) {
    const int lane = threadIdx.x & 31, mat = lane >> 3, rr = lane & 7;
    float c[2][8][4];
    fast_bias(c[0], bias);
#pragma unroll
    for (int j = 0; j < 8; ++j)
#pragma unroll
        for (int q = 0; q < 4; ++q) c[1][j][q] = c[0][j][q];
#pragma unroll
    for (int kk = 0; kk < 4; ++kk) {
#pragma unroll
        for (int jp = 0; jp < 4; ++jp) {
            uint32_t b[4];
            ldsm_x4(b, &W[16 * jp + 8 * (mat >> 1) + rr][16 * kk + 8 * (mat & 1)]);
#pragma unroll
            for (int mt = 0; mt < 2; ++mt) {
                mma_f16_16816(c[mt][2 * jp], hin[mt][kk], b[0], b[1]);
                mma_f16_16816(c[mt][2 * jp + 1], hin[mt][kk], b[2], b[3]);
            }
        }
    }
    fast_silu(c[0], hout[0]);
    fast_silu(c[1], hout[1]);
}

// Warp-cooperative nu_t of the 32 rows [32 blk, 32 blk + 32) of a feature
// tile feat[rows][8] (f16, normalised, columns 6 and 7 zero); writes
// nut[32 blk + r].  All 32 lanes call it together.
__device__ __forceinline__ void mlp_rows32(const MlpFast &w, const uint16_t *feat, float *nut, int blk) {
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3, mat = lane >> 3, rr = lane & 7;
    const uint32_t *f32 = reinterpret_cast<const uint32_t *>(feat) + (size_t)blk * 32 * 4;
    uint32_t h1[2][4][4];
    {
        float c[2][8][4];
        fast_bias(c[0], w.b1);
#pragma unroll
        for (int j = 0; j < 8; ++j)
#pragma unroll
            for (int q = 0; q < 4; ++q) c[1][j][q] = c[0][j][q];
        uint32_t b[8];
        ldsm_x4(b, &w.w1[8 * mat + rr][0]);
        ldsm_x4(b + 4, &w.w1[32 + 8 * mat + rr][0]);
#pragma unroll
        for (int mt = 0; mt < 2; ++mt) {
            const uint32_t a0 = f32[(16 * mt + g) * 4 + t], a1 = f32[(16 * mt + g + 8) * 4 + t];
#pragma unroll
            for (int j = 0; j < 8; ++j) mma_f16_1688(c[mt][j], a0, a1, b[j]);
        }
        fast_silu(c[0], h1[0]);
        fast_silu(c[1], h1[1]);
    }
    uint32_t h2[2][4][4];
    fast_layer64(h1, w.w2, w.b2, h2);
    fast_layer64(h2, w.w3, w.b3, h1);
    float c4[2][4] = {{0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}};
#pragma unroll
    for (int q = 0; q < 2; ++q) {
        uint32_t b[4];
        ldsm_x4(b, &w.w4[rr][16 * (2 * q + (mat >> 1)) + 8 * (mat & 1)]);
#pragma unroll
        for (int mt = 0; mt < 2; ++mt) {
            mma_f16_16816(c4[mt], h1[mt][2 * q], b[0], b[1]);
            mma_f16_16816(c4[mt], h1[mt][2 * q + 1], b[2], b[3]);
        }
    }
    if (t == 0) {
#pragma unroll
        for (int mt = 0; mt < 2; ++mt) {
            const float zg = c4[mt][0] + c4[mt][1] + w.b4, zg8 = c4[mt][2] + c4[mt][3] + w.b4;
            nut[32 * blk + 16 * mt + g] = w.out_scale * softplus_f(zg);
            nut[32 * blk + 16 * mt + g + 8] = w.out_scale * softplus_f(zg8);
        }
    }
}

// The five invariant features of G over powers of g = |G| (the element
// Reynolds number is the sixth, mlp_re_bits), normalised and clamped, as f16
// words: word 0 = (x1, x2), word 1 = (x3, x4), word 2 = (x5, 0).  *gout = g.
// A vanishing gradient gives zero features (and a zero nu_t: the caller
// multiplies by g).  Non-finite values (degenerate elements, idle lanes)
// become the mean.  Returns whether the five lie inside the training
// envelope (the caller falls back to Vreman's nu_t where they do not).
__device__ __forceinline__ bool mlp_gp_words(const float G[3][3], const MlpFast &w, uint32_t words[3], float *gout) {
    float S[3][3], O[3][3];
    float g2 = 0.f;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            S[i][j] = 0.5f * (G[i][j] + G[j][i]);
            O[i][j] = 0.5f * (G[i][j] - G[j][i]);
            g2 += G[i][j] * G[i][j];
        }
    float S2[3][3], O2[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            float a = 0.f, b = 0.f;
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                a += S[i][k] * S[k][j];
                b += O[i][k] * O[k][j];
            }
            S2[i][j] = a;
            O2[i][j] = b;
        }
    float I[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        I[0] += S2[i][i];
        I[1] += O2[i][i];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            I[2] += S2[i][k] * S[k][i];
            I[3] += S[i][k] * O2[k][i];
            I[4] += S2[i][k] * O2[k][i];
        }
    }
    const bool some = g2 > 0.f;
    const float ig2 = some ? 1.f / g2 : 0.f, ig = some ? rsqrtf(g2) : 0.f;
    *gout = some ? g2 * ig : 0.f;
    const float sc[5] = {ig2, ig2, ig2 * ig, ig2 * ig, ig2 * ig2};
    float xn[5];
    bool inside = true;
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        const float v = (I[k] * sc[k] - w.mean[k]) * w.istd[k];
        inside = inside && (!some || (v >= w.env_lo[k] && v <= w.env_hi[k]));   // false for NaN
        xn[k] = isfinite(v) ? fminf(fmaxf(v, -kFeatClamp), kFeatClamp) : 0.0f;
    }
    words[0] = pack_f16x2(xn[0], xn[1]);
    words[1] = pack_f16x2(xn[2], xn[3]);
    words[2] = pack_f16x2(xn[4], 0.0f);
    return inside;
}

// f16 bits of the normalised (clamped) element Reynolds number
// log(Delta^2 g / nu) (zero raw feature where g = 0); *inside: within the
// training envelope
__device__ __forceinline__ uint16_t mlp_re_bits(float delta, float g, float nu, const MlpFast &w, bool *inside) {
    const bool some = g > 0.f;
    float v = ((some ? __logf(delta * delta * g / nu) : 0.f) - w.mean[5]) * w.istd[5];
    *inside = !some || (v >= w.env_lo[5] && v <= w.env_hi[5]);
    v = isfinite(v) ? fminf(fmaxf(v, -kFeatClamp), kFeatClamp) : 0.0f;
    return (uint16_t)(pack_f16x2(v, 0.0f) & 0xffffu);
}

}  // namespace fea
