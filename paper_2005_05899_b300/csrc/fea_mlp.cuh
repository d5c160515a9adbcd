// Learned eddy-viscosity closure: a 6 -> 64 -> 64 -> 64 -> 1 MLP (SiLU hidden
// layers, softplus output) with BF16 weights and activations and FP32
// accumulation.
//
// Inputs per row (Gauss point or element), dimensionless: the invariants of
// S = (G+G^T)/2 and O = (G-G^T)/2 of the velocity gradient G_ij = du_i/dx_j
// over powers of g = |G| (g^2 = tr S^2 - tr O^2),
//   x_1..5 = (tr S^2, tr O^2, tr S^3, tr S O^2, tr S^2 O^2) / g^(2, 2, 3, 3, 4),
// and the element Reynolds number x_6 = log(Delta^2 g / nu), normalised as
// (x - mean) / std; output the coefficient C = out_scale softplus(z), and
// nu_t = C Delta^2 g (zero where g = 0, whose features are all zero).
//
// Inference (fused closure, batched forward) runs on the tcgen05 tensor
// cores over 128-row tiles, FP16 operands and activations (fea_tc.cuh).  The training step below keeps
// warp-level mma.sync m16n8k16 tiles (row.col, BF16 in, FP32 accumulate):
// for lane l, g = l / 4, t = l % 4; an A fragment holds rows (g, g+8) and
// columns (2t, 2t+1, 2t+8, 2t+9) of a 16 x 16 tile; a C fragment holds rows
// (g, g+8), columns (2t, 2t+1) of a 16 x 8 tile.  The C fragments of the
// n-tiles 2k and 2k+1 of one layer are exactly the A fragment of k-step k of
// the next layer, so the forward pass of a training tile keeps its
// activations in registers.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "fea_tc.cuh"

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

// ---------------------------------------------------------------------------
// Inference of the same network for the fused closure and the batched
// forward runs on the tcgen05 tensor cores (fea_tc.cuh): the BF16 weight
// values the network is trained with, held exactly as FP16 operands, FP16
// activations and hidden-layer accumulators, an FP32 output layer.  A
// feature row is 8 FP16 values (16 bytes):
// x1..x6 normalised and clamped to +-kFeatClamp, then 1 (the bias input)
// and 0.  Normalised features are clamped (far outside any training data)
// so that a degenerate gradient cannot overflow the products.
constexpr float kFeatClamp = 64.0f;

// Per-warp scratch of the fused closure for ng Gauss points per element, 32
// elements (one per lane): the per-point matrices S [ng][9][32] f32 the
// subgrid term needs once nu_t is known, then the network's coefficient C,
// Vreman's q = nu_t / Delta^2 (for the fallback) and g = |G|, each [ng*32]
// f32.  The feature rows live in the warpgroup's tensor-core tiles.
__host__ __device__ constexpr size_t mlp_s_bytes(int ng) { return (size_t)ng * 9 * 32 * 4; }
__host__ __device__ constexpr size_t mlp_warp_scratch_bytes(int ng) {
    return mlp_s_bytes(ng) + (size_t)ng * 32 * 4 * 3;
}

// The five invariant features of G over powers of g = |G| (the element
// Reynolds number is the sixth, mlp_re_bits), normalised and clamped, as
// FP16 pairs: word 0 = (x1, x2), word 1 = (x3, x4), word 2 = (x5, 0).
// *gout = g.
// A vanishing gradient gives zero features (and a zero nu_t: the caller
// multiplies by g).  Non-finite values (degenerate elements, idle lanes)
// become the mean.  Returns whether the five lie inside the training
// envelope (the caller falls back to Vreman's nu_t where they do not).
__device__ __forceinline__ bool mlp_gp_words(const float G[3][3], const tc::MlpTc &w, uint32_t words[3], float *gout) {
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
    words[0] = tc::pack_f16x2(xn[0], xn[1]);
    words[1] = tc::pack_f16x2(xn[2], xn[3]);
    words[2] = tc::pack_f16x2(xn[4], 0.0f);
    return inside;
}

// FP16 bits of the normalised (clamped) element Reynolds number
// log(Delta^2 g / nu) (zero raw feature where g = 0); *inside: within the
// training envelope
__device__ __forceinline__ uint16_t mlp_re_bits(float delta, float g, float nu, const tc::MlpTc &w, bool *inside) {
    const bool some = g > 0.f;
    float v = ((some ? __logf(delta * delta * g / nu) : 0.f) - w.mean[5]) * w.istd[5];
    *inside = !some || (v >= w.env_lo[5] && v <= w.env_hi[5]);
    v = isfinite(v) ? fminf(fmaxf(v, -kFeatClamp), kFeatClamp) : 0.0f;
    return (uint16_t)(tc::pack_f16x2(v, 0.0f) & 0xffffu);
}

}  // namespace fea
