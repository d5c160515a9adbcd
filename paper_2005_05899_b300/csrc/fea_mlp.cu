// MLP closure: packing, batched forward (inference) and one training step
// (forward + backward on BF16 tensor cores, FP32 gradients, Adam).
//
// Parameter vector theta (FP32, 8,833 values):
//   w1[64][6] b1[64] w2[64][64] b2[64] w3[64][64] b3[64] w4[64] b4[1].
// Training loss: mean_b (softplus(z_b) - y_b)^2 on normalised inputs.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "fea_internal.h"
#include "fea_mlp.cuh"

namespace fea {

namespace {

constexpr int OFF_W1 = 0, OFF_B1 = OFF_W1 + kMlpH * kMlpIn, OFF_W2 = OFF_B1 + kMlpH, OFF_B2 = OFF_W2 + kMlpH * kMlpH,
              OFF_W3 = OFF_B2 + kMlpH, OFF_B3 = OFF_W3 + kMlpH * kMlpH, OFF_W4 = OFF_B3 + kMlpH,
              OFF_B4 = OFF_W4 + kMlpH;

__device__ __forceinline__ uint16_t to_bf16_bits(float v) {
    __nv_bfloat16 b = __float2bfloat16_rn(v);
    return *reinterpret_cast<uint16_t *>(&b);
}

__device__ __forceinline__ float bf16_lo(uint32_t v) { return __uint_as_float(v << 16); }
__device__ __forceinline__ float bf16_hi(uint32_t v) { return __uint_as_float(v & 0xffff0000u); }

__device__ __forceinline__ uint16_t f16_bits(float v) {
    __half h = __float2half_rn(v);
    return *reinterpret_cast<uint16_t *>(&h);
}
// the BF16 rounding of v, as FP16 bits (exact unless it underflows FP16's
// normal range, where FP16 subnormals keep it to 2^-24)
__device__ __forceinline__ uint16_t bf16_as_f16_bits(float v) {
    return f16_bits(__uint_as_float((uint32_t)to_bf16_bits(v) << 16));
}
// FP16 bits of v and of the remainder v - hi: hi + lo = v to about 2^-22
// relative; hi = the FP16 value of v
__device__ __forceinline__ void f16_split(float v, uint16_t &hi, uint16_t &lo) {
    hi = f16_bits(v);
    lo = f16_bits(v - __half2float(__ushort_as_half(hi)));
}

__global__ void k_mlp_pack(const float *theta, const float *mean, const float *stdv, float out_scale, MlpWeights *w,
                           tc::MlpTc *fw) {
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    const int nth = gridDim.x * blockDim.x;
    // inference layout (tensor-core operands, K blocks of 8, FP16 bits): the
    // BF16 values of the hidden weights, halved (exact); the hidden biases
    // halved and split into hi and lo parts beside the weights; the output
    // weights and bias as hi = their BF16 value and lo = the rest
    for (int k = tid; k < 2 * kMlpH * 8; k += nth) {
        const int blk = k / (kMlpH * 8), o = (k / 8) % kMlpH, i = k % 8;
        uint16_t v = 0;
        if (blk == 0 && i < kMlpIn) {
            v = bf16_as_f16_bits(0.5f * theta[OFF_W1 + o * kMlpIn + i]);
        } else if (blk == 0) {
            uint16_t hi, lo;
            f16_split(0.5f * theta[OFF_B1 + o], hi, lo);
            v = i == 6 ? hi : lo;
        }
        fw->w1[blk][o][i] = v;
    }
    for (int k = tid; k < 10 * kMlpH * 8; k += nth) {
        const int blk = k / (kMlpH * 8), o = (k / 8) % kMlpH, i = k % 8;
        uint16_t v2 = 0, v3 = 0;
        if (blk < 8) {
            v2 = bf16_as_f16_bits(0.5f * theta[OFF_W2 + o * kMlpH + 8 * blk + i]);
            v3 = bf16_as_f16_bits(0.5f * theta[OFF_W3 + o * kMlpH + 8 * blk + i]);
        } else if (blk == 8 && i < 2) {
            uint16_t h2, l2, h3, l3;
            f16_split(0.5f * theta[OFF_B2 + o], h2, l2);
            f16_split(0.5f * theta[OFF_B3 + o], h3, l3);
            v2 = i == 0 ? h2 : l2;
            v3 = i == 0 ? h3 : l3;
        }
        fw->w2[blk][o][i] = v2;
        fw->w3[blk][o][i] = v3;
    }
    for (int k = tid; k < 10 * 16 * 8; k += nth) {
        const int blk = k / (16 * 8), o = (k / 8) % 16, i = k % 8;
        uint16_t v = 0;
        auto hilo = [&](float x, int part) {
            const float hi = __uint_as_float((uint32_t)to_bf16_bits(x) << 16);
            return part == 0 ? f16_bits(hi) : f16_bits(x - hi);
        };
        if (blk < 8 && o < 2) v = hilo(theta[OFF_W4 + 8 * blk + i], o);
        else if (blk == 8 && o == 0 && i < 2) v = hilo(theta[OFF_B4], i);
        fw->w4[blk][o][i] = v;
    }
    if (tid == 0) {
        for (int k = 0; k < kMlpIn; ++k) {
            fw->mean[k] = mean[k];
            fw->istd[k] = 1.0f / stdv[k];
            // envelope bounds follow std in the norm block: lo[6], hi[6] (raw units)
            fw->env_lo[k] = (stdv[kMlpIn + k] - mean[k]) / stdv[k];
            fw->env_hi[k] = (stdv[2 * kMlpIn + k] - mean[k]) / stdv[k];
        }
        int on = 0;
        for (int k = 0; k < kMlpIn; ++k) on |= isfinite(fw->env_lo[k]) || isfinite(fw->env_hi[k]);
        fw->env_on = on;
        fw->out_scale = out_scale;
    }
    for (int k = tid; k < kMlpH * kW1Pitch; k += nth) {
        const int o = k / kW1Pitch, i = k % kW1Pitch;
        w->inf.w1[o][i] = to_bf16_bits(i < kMlpIn ? theta[OFF_W1 + o * kMlpIn + i] : 0.f);
    }
    for (int k = tid; k < kMlpH * kWPitch; k += nth) {
        const int o = k / kWPitch, i = k % kWPitch;
        const bool in = i < kMlpH;
        w->inf.w2[o][i] = to_bf16_bits(in ? theta[OFF_W2 + o * kMlpH + i] : 0.f);
        w->inf.w3[o][i] = to_bf16_bits(in ? theta[OFF_W3 + o * kMlpH + i] : 0.f);
        w->w2t[o][i] = to_bf16_bits(in ? theta[OFF_W2 + i * kMlpH + o] : 0.f);
        w->w3t[o][i] = to_bf16_bits(in ? theta[OFF_W3 + i * kMlpH + o] : 0.f);
    }
    for (int k = tid; k < kMlpH; k += nth) {
        w->inf.b1[k] = theta[OFF_B1 + k];
        w->inf.b2[k] = theta[OFF_B2 + k];
        w->inf.b3[k] = theta[OFF_B3 + k];
        w->inf.w4[k] = theta[OFF_W4 + k];
    }
    if (tid == 0) {
        w->inf.b4 = theta[OFF_B4];
        for (int k = 0; k < kMlpIn; ++k) {
            w->inf.mean[k] = mean[k];
            w->inf.istd[k] = 1.0f / stdv[k];
        }
        w->inf.out_scale = out_scale;
    }
}

__device__ __forceinline__ void copy_weights_to_smem(const MlpWeights *g, MlpWeights *s) {
    const int4 *src = reinterpret_cast<const int4 *>(g);
    int4 *dst = reinterpret_cast<int4 *>(s);
    for (int k = threadIdx.x; k < (int)(sizeof(MlpWeights) / 16); k += blockDim.x) dst[k] = src[k];
    __syncthreads();
}

// batched forward: raw features x [B][6] -> C y [B] on the tensor cores;
// a CTA (one warpgroup of 128 threads) takes 256 rows at a time as two
// 128-row tiles (thread t: rows t and 128 + t)
constexpr int kFwdTiles = 2;
constexpr size_t kFwdSmem = sizeof(tc::MlpTc) + tc::feat_bytes(kFwdTiles) + kFwdTiles * 128 * 4 + 64;

__global__ void __launch_bounds__(128) k_mlp_forward(const tc::MlpTc *wg, const float *x, int64_t B, float *y,
                                                     unsigned *err) {
    extern __shared__ __align__(128) unsigned char fwd_smem[];
    tc::MlpTc *w = reinterpret_cast<tc::MlpTc *>(fwd_smem);
    unsigned char *feat = fwd_smem + sizeof(tc::MlpTc);
    unsigned char *zero = feat + kFwdTiles * tc::kRows * 16;
    float *outb = reinterpret_cast<float *>(zero + tc::kRows * 16);
    uint64_t *bars = reinterpret_cast<uint64_t *>(outb + kFwdTiles * tc::kRows);
    tc::Warpgroup wgs;
    tc::setup(wg, w, zero, bars, wgs, err, 0);
    const int row = threadIdx.x;
    for (int64_t base = (int64_t)blockIdx.x * (kFwdTiles * tc::kRows); base < B;
         base += (int64_t)gridDim.x * (kFwdTiles * tc::kRows)) {
        for (int t = 0; t < kFwdTiles; ++t) {
            const int64_t r = base + t * tc::kRows + row;
            float xn[kMlpIn];
#pragma unroll
            for (int k = 0; k < kMlpIn; ++k) {
                const float v = r < B ? (x[r * kMlpIn + k] - w->mean[k]) * w->istd[k] : 0.0f;
                xn[k] = isfinite(v) ? fminf(fmaxf(v, -kFeatClamp), kFeatClamp) : 0.0f;
            }
            *reinterpret_cast<uint4 *>(feat + (t * tc::kRows + row) * 16) =
                make_uint4(tc::pack_f16x2(xn[0], xn[1]), tc::pack_f16x2(xn[2], xn[3]),
                           tc::pack_f16x2(xn[4], xn[5]), tc::kOnesWord);
        }
        tc::run(wgs, w, feat, zero, kFwdTiles, outb + row, tc::kRows);
        for (int t = 0; t < kFwdTiles; ++t) {
            const int64_t r = base + t * tc::kRows + row;
            if (r < B) y[r] = outb[t * tc::kRows + row];
        }
    }
    tc::teardown(wgs);
}

// ---- training step ------------------------------------------------------------
// CTA = 4 warps, each warp one 16-row tile.  Forward keeps the SiLU
// derivatives and the hidden activations in shared memory; backward runs the
// dH GEMMs (dZ W) and the weight-gradient GEMMs (dZ^T H) on tensor cores and
// reduces the CTA's gradient in shared memory before one global atomic add
// per parameter.

constexpr int kTrainWarps = 4;
constexpr int kTilePitch = kWPitch;  // bf16 per row of a [16][64] activation tile

struct WarpTrain {
    float sd[3][32][32];                 // SiLU'(z) of layers 1..3, [value][lane]
    uint16_t h0[16][kW1Pitch];           // inputs (row-major)
    uint16_t h1[16][kTilePitch], h2[16][kTilePitch];
    uint16_t dz[16][kTilePitch];         // current dZ (row-major)
};

struct TrainGrad {
    float w1[kMlpH][16];
    float w2[kMlpH][kMlpH];
    float w3[kMlpH][kMlpH];
    float b1[kMlpH], b2[kMlpH], b3[kMlpH], w4[kMlpH], b4;
};

__device__ __forceinline__ float silu_deriv(float z) {
    const float s = sigmoid_f(z);
    return s * (1.0f + z * (1.0f - s));
}

// store A fragments (rows g, g+8; 4 k-steps) into a row-major bf16 tile
__device__ __forceinline__ void frag_to_tile(const uint32_t h[4][4], uint16_t (*tile)[kTilePitch]) {
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
#pragma unroll
    for (int kk = 0; kk < 4; ++kk) {
        uint32_t *rg = reinterpret_cast<uint32_t *>(tile[g]);
        uint32_t *rg8 = reinterpret_cast<uint32_t *>(tile[g + 8]);
        rg[8 * kk + t] = h[kk][0];
        rg8[8 * kk + t] = h[kk][1];
        rg[8 * kk + 4 + t] = h[kk][2];
        rg8[8 * kk + 4 + t] = h[kk][3];
    }
}

// dH = dZ W (M = 16 rows, N = 64, K = 64) with W^T stored row-major
__device__ __forceinline__ void back_gemm(const uint32_t dz[4][4], const uint16_t (*WT)[kWPitch], float c[8][4]) {
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        c[j][0] = c[j][1] = c[j][2] = c[j][3] = 0.f;
        const uint32_t *row = reinterpret_cast<const uint32_t *>(WT[8 * j + g]);
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) mma_bf16_16816(c[j], dz[kk], row[8 * kk + t], row[8 * kk + 4 + t]);
    }
}

// dW[o][i] += sum_r dZ[r][o] H[r][i] for one 16-row tile: M = 64 (o), N = NI*8 (i), K = 16 (r)
template <int NI, int HPITCH>
__device__ __forceinline__ void weight_grad(const uint16_t (*dz)[kTilePitch], const uint16_t (*h)[HPITCH],
                                            float *gw /* smem [64][NI*8] */) {
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    auto pk = [](uint16_t lo, uint16_t hi) { return (uint32_t)lo | ((uint32_t)hi << 16); };
#pragma unroll
    for (int mi = 0; mi < 4; ++mi) {
        const int o = 16 * mi + g;
        uint32_t a[4];
        a[0] = pk(dz[2 * t][o], dz[2 * t + 1][o]);
        a[1] = pk(dz[2 * t][o + 8], dz[2 * t + 1][o + 8]);
        a[2] = pk(dz[2 * t + 8][o], dz[2 * t + 9][o]);
        a[3] = pk(dz[2 * t + 8][o + 8], dz[2 * t + 9][o + 8]);
#pragma unroll
        for (int ni = 0; ni < NI; ++ni) {
            const int i = 8 * ni + g;
            const uint32_t b0 = pk(h[2 * t][i], h[2 * t + 1][i]);
            const uint32_t b1 = pk(h[2 * t + 8][i], h[2 * t + 9][i]);
            float c[4] = {0.f, 0.f, 0.f, 0.f};
            mma_bf16_16816(c, a, b0, b1);
            const int ic = 8 * ni + 2 * t;
            atomicAdd(&gw[o * (NI * 8) + ic], c[0]);
            atomicAdd(&gw[o * (NI * 8) + ic + 1], c[1]);
            atomicAdd(&gw[(o + 8) * (NI * 8) + ic], c[2]);
            atomicAdd(&gw[(o + 8) * (NI * 8) + ic + 1], c[3]);
        }
    }
}

// column sums over the 16 rows of a C-layout tile set (bias gradients)
__device__ __forceinline__ void col_sums(const float c[8][4], float *gb) {
    const int lane = threadIdx.x & 31, t = lane & 3;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        float s0 = c[j][0] + c[j][2], s1 = c[j][1] + c[j][3];
#pragma unroll
        for (int m = 4; m < 32; m <<= 1) {
            s0 += __shfl_xor_sync(0xffffffffu, s0, m);
            s1 += __shfl_xor_sync(0xffffffffu, s1, m);
        }
        if (lane < 4) {
            atomicAdd(&gb[8 * j + 2 * t], s0);
            atomicAdd(&gb[8 * j + 2 * t + 1], s1);
        }
    }
}

// dZ = dH o SiLU'(z) in C layout, then as bf16 A fragments and a row-major tile
__device__ __forceinline__ void apply_deriv(float c[8][4], const float (*sd)[32], uint32_t dzf[4][4],
                                            uint16_t (*tile)[kTilePitch]) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int j = 0; j < 8; ++j)
#pragma unroll
        for (int q = 0; q < 4; ++q) c[j][q] *= sd[j * 4 + q][lane];
#pragma unroll
    for (int kk = 0; kk < 4; ++kk) {
        dzf[kk][0] = pack_bf16x2(c[2 * kk][0], c[2 * kk][1]);
        dzf[kk][1] = pack_bf16x2(c[2 * kk][2], c[2 * kk][3]);
        dzf[kk][2] = pack_bf16x2(c[2 * kk + 1][0], c[2 * kk + 1][1]);
        dzf[kk][3] = pack_bf16x2(c[2 * kk + 1][2], c[2 * kk + 1][3]);
    }
    frag_to_tile(dzf, tile);
}

__global__ void __launch_bounds__(kTrainWarps * 32) k_mlp_train(const MlpWeights *wg, const float *x, const float *y,
                                                                int64_t B, float *grad, float *loss) {
    extern __shared__ __align__(16) unsigned char smem[];
    MlpWeights *wall = reinterpret_cast<MlpWeights *>(smem);
    const MlpInfer *w = &wall->inf;
    size_t off = sizeof(MlpWeights);
    TrainGrad *gs = reinterpret_cast<TrainGrad *>(smem + off);
    off += (sizeof(TrainGrad) + 15) & ~size_t(15);
    WarpTrain *wt_all = reinterpret_cast<WarpTrain *>(smem + off);
    for (int k = threadIdx.x; k < (int)(sizeof(TrainGrad) / 4); k += blockDim.x) reinterpret_cast<float *>(gs)[k] = 0.f;
    copy_weights_to_smem(wg, wall);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    WarpTrain &wt = wt_all[warp];
    const int64_t r0 = ((int64_t)blockIdx.x * kTrainWarps + warp) * 16;
    const int64_t rg = r0 + g, rg8 = r0 + g + 8;
    const bool vg = rg < B, vg8 = rg8 < B;
    // inputs: lane (g, t) holds columns 2t, 2t+1 of rows g, g+8 (columns 6.. are zero)
    float xg0 = 0.f, xg1 = 0.f, x80 = 0.f, x81 = 0.f;
    if (t < 3) {
        if (vg) {
            xg0 = (x[rg * kMlpIn + 2 * t] - w->mean[2 * t]) * w->istd[2 * t];
            xg1 = (x[rg * kMlpIn + 2 * t + 1] - w->mean[2 * t + 1]) * w->istd[2 * t + 1];
        }
        if (vg8) {
            x80 = (x[rg8 * kMlpIn + 2 * t] - w->mean[2 * t]) * w->istd[2 * t];
            x81 = (x[rg8 * kMlpIn + 2 * t + 1] - w->mean[2 * t + 1]) * w->istd[2 * t + 1];
        }
    }
    uint32_t a1[1][4] = {{pack_bf16x2(xg0, xg1), pack_bf16x2(x80, x81), 0u, 0u}};
    {
        uint32_t *rgw = reinterpret_cast<uint32_t *>(wt.h0[g]);
        uint32_t *rg8w = reinterpret_cast<uint32_t *>(wt.h0[g + 8]);
        rgw[t] = a1[0][0];
        rg8w[t] = a1[0][1];
        rgw[4 + t] = 0u;
        rg8w[4 + t] = 0u;
    }
    // forward
    uint32_t h1[4][4], h2[4][4], h3[4][4];
    float zs[32];
    mlp_layer<1, kW1Pitch>(a1, w->w1, w->b1, h1, zs);
#pragma unroll
    for (int v = 0; v < 32; ++v) wt.sd[0][v][lane] = silu_deriv(zs[v]);
    mlp_layer<4, kWPitch>(h1, w->w2, w->b2, h2, zs);
#pragma unroll
    for (int v = 0; v < 32; ++v) wt.sd[1][v][lane] = silu_deriv(zs[v]);
    mlp_layer<4, kWPitch>(h2, w->w3, w->b3, h3, zs);
#pragma unroll
    for (int v = 0; v < 32; ++v) wt.sd[2][v][lane] = silu_deriv(zs[v]);
    frag_to_tile(h1, wt.h1);
    frag_to_tile(h2, wt.h2);
    float zg, zg8;
    mlp_output(h3, w->w4, w->b4, zg, zg8);
    // loss and d loss / d z
    const float yg = vg ? y[rg] : 0.f, yg8 = vg8 ? y[rg8] : 0.f;
    const float dg = vg ? softplus_f(zg) - yg : 0.f, dg8 = vg8 ? softplus_f(zg8) - yg8 : 0.f;
    const float inv_b = 1.0f / (float)B;
    const float dzg = 2.f * dg * inv_b * sigmoid_f(zg), dzg8 = 2.f * dg8 * inv_b * sigmoid_f(zg8);
    {
        float l = (t == 0) ? dg * dg + dg8 * dg8 : 0.f;
        float db4 = (t == 0) ? dzg + dzg8 : 0.f;
#pragma unroll
        for (int m = 1; m < 32; m <<= 1) {
            l += __shfl_xor_sync(0xffffffffu, l, m);
            db4 += __shfl_xor_sync(0xffffffffu, db4, m);
        }
        if (lane == 0) {
            atomicAdd(loss, l * inv_b);
            atomicAdd(&gs->b4, db4);
        }
    }
    // output layer: dw4 and dZ3 = (dz4 w4^T) o SiLU'(z3)
    float c[8][4];
#pragma unroll
    for (int kk = 0; kk < 4; ++kk)
#pragma unroll
        for (int half = 0; half < 2; ++half) {
            const int j = 2 * kk + half;
            const int col = 8 * j + 2 * t;
            const uint32_t hg = h3[kk][2 * half], hg8 = h3[kk][2 * half + 1];
            float s0 = bf16_lo(hg) * dzg + bf16_lo(hg8) * dzg8;
            float s1 = bf16_hi(hg) * dzg + bf16_hi(hg8) * dzg8;
#pragma unroll
            for (int m = 4; m < 32; m <<= 1) {
                s0 += __shfl_xor_sync(0xffffffffu, s0, m);
                s1 += __shfl_xor_sync(0xffffffffu, s1, m);
            }
            if (lane < 4) {
                atomicAdd(&gs->w4[col], s0);
                atomicAdd(&gs->w4[col + 1], s1);
            }
            c[j][0] = dzg * w->w4[col];
            c[j][1] = dzg * w->w4[col + 1];
            c[j][2] = dzg8 * w->w4[col];
            c[j][3] = dzg8 * w->w4[col + 1];
        }
    uint32_t dzf[4][4];
    apply_deriv(c, wt.sd[2], dzf, wt.dz);
    col_sums(c, gs->b3);
    __syncwarp();
    weight_grad<8, kTilePitch>(wt.dz, wt.h2, &gs->w3[0][0]);
    back_gemm(dzf, wall->w3t, c);
    __syncwarp();
    apply_deriv(c, wt.sd[1], dzf, wt.dz);
    col_sums(c, gs->b2);
    __syncwarp();
    weight_grad<8, kTilePitch>(wt.dz, wt.h1, &gs->w2[0][0]);
    back_gemm(dzf, wall->w2t, c);
    __syncwarp();
    apply_deriv(c, wt.sd[0], dzf, wt.dz);
    col_sums(c, gs->b1);
    __syncwarp();
    weight_grad<2, kW1Pitch>(wt.dz, wt.h0, &gs->w1[0][0]);
    __syncthreads();
    // CTA gradient -> global (oracle layout)
    for (int k = threadIdx.x; k < kMlpParams; k += blockDim.x) {
        float v;
        if (k < OFF_B1) v = gs->w1[k / kMlpIn][k % kMlpIn];
        else if (k < OFF_W2) v = gs->b1[k - OFF_B1];
        else if (k < OFF_B2) v = gs->w2[(k - OFF_W2) / kMlpH][(k - OFF_W2) % kMlpH];
        else if (k < OFF_W3) v = gs->b2[k - OFF_B2];
        else if (k < OFF_B3) v = gs->w3[(k - OFF_W3) / kMlpH][(k - OFF_W3) % kMlpH];
        else if (k < OFF_W4) v = gs->b3[k - OFF_B3];
        else if (k < OFF_B4) v = gs->w4[k - OFF_W4];
        else v = gs->b4;
        atomicAdd(&grad[k], v);
    }
}

__global__ void k_adam(float *theta, const float *grad, float *m1, float *m2, int n, float lr, float b1, float b2,
                       float eps, float c1, float c2) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        const float gk = grad[k];
        const float a = b1 * m1[k] + (1.f - b1) * gk;
        const float b = b2 * m2[k] + (1.f - b2) * gk * gk;
        m1[k] = a;
        m2[k] = b;
        theta[k] -= lr * (a / c1) / (sqrtf(b / c2) + eps);
    }
}

}  // namespace

// One device block holds the training layout (MlpWeights) followed by the
// inference layout (tc::MlpTc).
constexpr size_t kFastOffset = (sizeof(MlpWeights) + 255) & ~size_t(255);

size_t mlp_weights_bytes() { return kFastOffset + sizeof(tc::MlpTc); }
int mlp_param_count() { return kMlpParams; }
const void *mlp_fast_ptr(const void *w) { return static_cast<const unsigned char *>(w) + kFastOffset; }

cudaError_t launch_mlp_pack(const float *theta, const float *mean, const float *stdv, float out_scale, void *w,
                            cudaStream_t s) {
    k_mlp_pack<<<16, 256, 0, s>>>(theta, mean, stdv, out_scale, static_cast<MlpWeights *>(w),
                                  reinterpret_cast<tc::MlpTc *>(static_cast<unsigned char *>(w) + kFastOffset));
    return cudaGetLastError();
}

cudaError_t launch_mlp_forward(const void *w, const float *x, int64_t B, float *y, int sms, unsigned *err,
                               cudaStream_t s) {
    if (B <= 0) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(k_mlp_forward, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kFwdSmem);
    if (e != cudaSuccess) return e;
    // two CTAs per SM: each holds 256 of the SM's 512 TMEM columns
    const int64_t want = (B + kFwdTiles * tc::kRows - 1) / (kFwdTiles * tc::kRows);
    const int grid = (int)std::min<int64_t>(want, (int64_t)sms * 2);
    k_mlp_forward<<<grid, 128, kFwdSmem, s>>>(static_cast<const tc::MlpTc *>(mlp_fast_ptr(w)), x, B, y, err);
    return cudaGetLastError();
}

cudaError_t launch_mlp_train(const void *w, const float *x, const float *y, int64_t B, float *grad, float *loss,
                             cudaStream_t s) {
    if (B <= 0) return cudaSuccess;
    const size_t smem = sizeof(MlpWeights) + ((sizeof(TrainGrad) + 15) & ~size_t(15)) + kTrainWarps * sizeof(WarpTrain);
    cudaError_t e = cudaFuncSetAttribute(k_mlp_train, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int64_t grid = (B + 16 * kTrainWarps - 1) / (16 * kTrainWarps);
    k_mlp_train<<<(unsigned)grid, kTrainWarps * 32, smem, s>>>(static_cast<const MlpWeights *>(w), x, y, B, grad,
                                                               loss);
    return cudaGetLastError();
}

cudaError_t launch_adam(float *theta, const float *grad, float *m1, float *m2, int n, float lr, float b1, float b2,
                        float eps, int64_t step, cudaStream_t s) {
    const float c1 = 1.f - powf(b1, (float)step), c2 = 1.f - powf(b2, (float)step);
    k_adam<<<(n + 255) / 256, 256, 0, s>>>(theta, grad, m1, m2, n, lr, b1, b2, eps, c1, c2);
    return cudaGetLastError();
}

}  // namespace fea
