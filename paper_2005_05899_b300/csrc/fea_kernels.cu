// Element-assembly kernels of the momentum RHS for sm_103a.
//
// One thread computes one element (gather -> computation -> scatter, the
// three steps of section 2.3.3).  Elements arrive in categories (one element
// type, one Jacobian precision) sorted along a Morton curve, so neighbouring
// threads touch neighbouring nodes.  The residual of Eq. momentum per node a
// and component i is
//   r_a,i = - sum_g W_g [ N_a (c_i + d_i p) + 2 (nu + nu_t) eps_ij d_j N_a ],
//   c = G u + (tr G) u,  G_ij = du_i/dx_j,  W_g = w_g det J,
// with nu_t from Vreman's model (section 2.1) at every Gauss point and the
// filter width Delta = V_e^(1/3).
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>

#include "fea_internal.h"
#include "fea_mlp.cuh"

namespace fea {

__constant__ RefTables c_ref;

// The same tables rounded to FP32 for the FP32 element arithmetic: reading
// the FP64 table and converting at every use put a conversion per shape
// function value on the FP64 pipe (1/64 of the FP32 rate on this part).
struct RefTables32 {
    float xi[4][kMaxNg][3];
    float N[4][kMaxNg][kMaxNen];
    float dN[4][kMaxNg][kMaxNen][3];
    float w[4][kMaxNg];
};
__constant__ RefTables32 c_ref32;

cudaError_t upload_ref_tables(const RefTables &t) {
    RefTables32 t32;
    for (int e = 0; e < 4; ++e)
        for (int g = 0; g < kMaxNg; ++g) {
            t32.w[e][g] = (float)t.w[e][g];
            for (int k = 0; k < 3; ++k) t32.xi[e][g][k] = (float)t.xi[e][g][k];
            for (int a = 0; a < kMaxNen; ++a) {
                t32.N[e][g][a] = (float)t.N[e][g][a];
                for (int k = 0; k < 3; ++k) t32.dN[e][g][a][k] = (float)t.dN[e][g][a][k];
            }
        }
    cudaError_t e = cudaMemcpyToSymbol(c_ref, &t, sizeof(RefTables));
    if (e != cudaSuccess) return e;
    return cudaMemcpyToSymbol(c_ref32, &t32, sizeof(RefTables32));
}

// FP64 -> FP32, round to nearest even, by integer operations for results in
// the normal FP32 range (B300's FP64 pipe runs at 1/64 of the FP32 rate and
// the stage update is otherwise bound by it); zero, subnormal, overflowing,
// infinite and NaN inputs take the hardware conversion.
__device__ __forceinline__ float f64_to_f32_rn(double x) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const unsigned hi = (unsigned)(b >> 32);
    const unsigned e = (hi >> 20) & 0x7ffu;
    if (e < 897u || e > 1150u) return __double2float_rn(x);
    const unsigned long long m = b & 0x000FFFFFFFFFFFFFull;
    const unsigned long long rem = m & 0x1FFFFFFFull;   // the 29 bits dropped
    unsigned r = (unsigned)(m >> 29);
    r += (rem > 0x10000000ull || (rem == 0x10000000ull && (r & 1u))) ? 1u : 0u;
    // a carry out of the 23-bit fraction moves into the exponent, as it must
    return __uint_as_float(((hi & 0x80000000u) | ((e - 896u) << 23)) + r);
}

// FP32 -> FP64 (exact) by integer operations for normal numbers: the
// hardware conversion is an FP64-pipe instruction (1/64 of the FP32 rate on
// this part), one per scattered component otherwise; zero, subnormals,
// infinities and NaN take the hardware conversion.
__device__ __forceinline__ double f32_to_f64_exact(float x) {
    const uint32_t b = __float_as_uint(x);
    const uint32_t e = (b >> 23) & 0xffu;
    if (e == 0u || e == 0xffu) return (double)x;
    const uint32_t hi = (b & 0x80000000u) | ((e + 896u) << 20) | ((b & 0x7fffffu) >> 3);
    return __hiloint2double((int)hi, (int)(b << 29));
}

// an R value as FP64 for the nodal sums
template <typename R>
__device__ __forceinline__ double to_f64(R x) {
    if constexpr (sizeof(R) == 4) return f32_to_f64_exact(x);
    else return x;
}

// an FP64 value in the arithmetic type R: FP64 -> FP32 by the integer
// rounding above (a hardware conversion is an FP64-pipe instruction)
template <typename R, typename JR>
__device__ __forceinline__ R to_r(JR x) {
    if constexpr (sizeof(R) == 4 && sizeof(JR) == 8) return f64_to_f32_rn(x);
    else return R(x);
}

// reference-table entries in the arithmetic type R (the FP32 copy for float)
template <typename R>
__device__ __forceinline__ R ref_N(int et, int g, int a) {
    if constexpr (sizeof(R) == 4) return c_ref32.N[et][g][a];
    else return c_ref.N[et][g][a];
}
template <typename R>
__device__ __forceinline__ R ref_dN(int et, int g, int a, int k) {
    if constexpr (sizeof(R) == 4) return c_ref32.dN[et][g][a][k];
    else return c_ref.dN[et][g][a][k];
}
template <typename R>
__device__ __forceinline__ R ref_w(int et, int g) {
    if constexpr (sizeof(R) == 4) return c_ref32.w[et][g];
    else return c_ref.w[et][g];
}
template <typename R>
__device__ __forceinline__ R ref_xi(int et, int g, int k) {
    if constexpr (sizeof(R) == 4) return c_ref32.xi[et][g][k];
    else return c_ref.xi[et][g][k];
}

template <typename R>
struct Mat3 {
    R m[3][3];
};

template <typename R>
__device__ __forceinline__ R det3(const R J[3][3]) {
    return J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) - J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
           J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
}

// adjugate / det, returns det
template <typename R>
__device__ __forceinline__ R inv3(const R J[3][3], R Ji[3][3]) {
    R c00 = J[1][1] * J[2][2] - J[1][2] * J[2][1];
    R c01 = J[1][2] * J[2][0] - J[1][0] * J[2][2];
    R c02 = J[1][0] * J[2][1] - J[1][1] * J[2][0];
    R det = J[0][0] * c00 + J[0][1] * c01 + J[0][2] * c02;
    R d = R(1) / det;
    Ji[0][0] = c00 * d;
    Ji[1][0] = c01 * d;
    Ji[2][0] = c02 * d;
    Ji[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) * d;
    Ji[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) * d;
    Ji[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) * d;
    Ji[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) * d;
    Ji[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) * d;
    Ji[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) * d;
    return det;
}

// Vreman: beta = Delta^2 alpha^T alpha with alpha = G^T, so every principal
// 2x2 minor of beta is Delta^4 |g_i x g_j|^2 (g_i = row i of G, Lagrange
// identity) and B_beta = Delta^4 (|g1 x g2|^2 + |g1 x g3|^2 + |g2 x g3|^2):
// a sum of squares, free of the cancellation of the difference form.
// nu_t = c Delta^2 sqrt(B' / (G:G)), zero when G:G == 0 or B' == 0.
template <typename R>
__device__ __forceinline__ R vreman(const R G[3][3], R delta2, R c) {
    R aa = R(0);
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) aa += G[i][j] * G[i][j];
    R B = R(0);
#pragma unroll
    for (int p = 0; p < 3; ++p) {
        const int i = p == 2 ? 1 : 0, j = p == 0 ? 1 : 2;   // (0,1), (0,2), (1,2)
        const R x = G[i][1] * G[j][2] - G[i][2] * G[j][1];
        const R y = G[i][2] * G[j][0] - G[i][0] * G[j][2];
        const R z = G[i][0] * G[j][1] - G[i][1] * G[j][0];
        B += x * x + y * y + z * z;
    }
    if (!(aa > R(0)) || !(B > R(0))) return R(0);
    return c * delta2 * sqrt(B / aa);
}

__device__ __forceinline__ double cbrt_r(double v) { return cbrt(v); }
__device__ __forceinline__ float cbrt_r(float v) { return cbrtf(v); }

__device__ __forceinline__ void set_err(unsigned *err, unsigned bit) {
    if (err) atomicOr(err, bit);
}

// ---------------------------------------------------------------------------
// gather helpers

// Vreman with a width per direction: beta = H H^T, H = G diag(dm), so
// B_beta = sum over row pairs of |h_i x h_j|^2 and nu_t = c sqrt(B_beta / G:G).
template <typename R>
__device__ __forceinline__ R vreman_aniso(const R G[3][3], const R dm[3], R c) {
    R H[3][3], aa = R(0);
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            aa += G[i][j] * G[i][j];
            H[i][j] = G[i][j] * dm[j];
        }
    R B = R(0);
#pragma unroll
    for (int p = 0; p < 3; ++p) {
        const int i = p == 2 ? 1 : 0, j = p == 0 ? 1 : 2;
        const R x = H[i][1] * H[j][2] - H[i][2] * H[j][1];
        const R y = H[i][2] * H[j][0] - H[i][0] * H[j][2];
        const R z = H[i][0] * H[j][1] - H[i][1] * H[j][0];
        B += x * x + y * y + z * z;
    }
    return (aa > R(0) && B > R(0)) ? c * sqrt(B / aa) : R(0);
}

// element extents along the axes (the per-direction filter widths)
template <int NEN, typename R, typename XR>
__device__ __forceinline__ void element_extents(const XR X[][3], R dm[3]) {
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        XR lo = X[0][i], hi = X[0][i];
#pragma unroll
        for (int a = 1; a < NEN; ++a) {
            lo = X[a][i] < lo ? X[a][i] : lo;
            hi = X[a][i] > hi ? X[a][i] : hi;
        }
        dm[i] = R(hi - lo);
    }
}

template <typename R, bool J64>
struct Gathered {
    R U[kMaxNen][3];
    R P[kMaxNen];
    typename std::conditional<J64, double, R>::type X[kMaxNen][3];
};

template <int ET, typename R, bool J64>
__device__ __forceinline__ void gather(const FieldDev &f, const int idx[], Gathered<R, J64> &g) {
    constexpr int nen = kNen[ET];
#pragma unroll
    for (int a = 0; a < nen; ++a) {
        const int64_t n = idx[a];
        if constexpr (sizeof(R) == 8) {
            g.U[a][0] = f.u64[n];
            g.U[a][1] = f.u64[f.n + n];
            g.U[a][2] = f.u64[2 * f.n + n];
            g.P[a] = f.p64[n];
        } else {
            const float4 up = __ldg(&f.up32[n]);
            g.U[a][0] = up.x;
            g.U[a][1] = up.y;
            g.U[a][2] = up.z;
            g.P[a] = up.w;
        }
        if constexpr (sizeof(R) == 8 || J64) {
            g.X[a][0] = __ldg(&f.xyz64[n]);
            g.X[a][1] = __ldg(&f.xyz64[f.n + n]);
            g.X[a][2] = __ldg(&f.xyz64[2 * f.n + n]);
        } else {
            const float4 x = __ldg(&f.xyz32[n]);
            g.X[a][0] = x.x;
            g.X[a][1] = x.y;
            g.X[a][2] = x.z;
        }
    }
}

// ---------------------------------------------------------------------------
// residual of one element at the Gauss points of its rule (all types).
// R: arithmetic type; JR: type of the Jacobian, its determinant and inverse.

template <int ET, typename R, typename JR>
__device__ __forceinline__ JR jacobian_at(const JR X[][3], int g, JR J[3][3]) {
    constexpr int nen = kNen[ET];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) J[i][j] = JR(0);
#pragma unroll
    for (int a = 0; a < nen; ++a)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const JR d = ref_dN<JR>(ET, g, a, j);
#pragma unroll
            for (int i = 0; i < 3; ++i) J[i][j] += X[a][i] * d;
        }
    return det3(J);
}

// Jacobian of a PEN06 at (r, s, zeta) from per-element edge combinations:
// the r- and s-columns are linear in zeta, the zeta-column linear in (r, s).
// The combinations are kept at twice their value (the shape functions' 1/2
// factors left out): every column is then 2x the true one, the adjugate 4x
// and the determinant 8x, all exactly (power-of-two scalings), and the
// callers rescale J^-1 and the weight instead of paying 21 FP64 multiplies
// per element.  With e, f the bottom and top edges from node 0 / 3 and h the
// vertical edges, the r-column is (e1 + f1) + zeta (f1 - e1) and the
// zeta-column h0 + r (h1 - h0) + s (h2 - h0); the twist f1 - e1 equals
// h1 - h0 (both are X4 - X3 - X1 + X0), so one difference Dr serves both and
// is formed from the short vertical edges (the more accurate rounding for a
// thin prism), and e1 + f1 = 2 e1 + Dr (likewise Ds for the s-column).  Q is
// the zeta-column at the rule's first triangle point (1/6, 1/6); at the
// other two, (2/3, 1/6) and (1/6, 2/3), it is Q + Dr / 2 and Q + Ds / 2.
template <typename JR>
struct PrismGeom {
    JR Ar[3], As[3], Dr[3], Ds[3], Q[3];
};

template <typename JR>
__device__ __forceinline__ void prism_geom2(const JR X[][3], PrismGeom<JR> &p) {
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        const JR e1 = X[1][i] - X[0][i], e2 = X[2][i] - X[0][i];
        const JR h0 = X[3][i] - X[0][i], h1 = X[4][i] - X[1][i], h2 = X[5][i] - X[2][i];
        p.Dr[i] = h1 - h0;
        p.Ds[i] = h2 - h0;
        p.Ar[i] = JR(2) * e1 + p.Dr[i];
        p.As[i] = JR(2) * e2 + p.Ds[i];
        p.Q[i] = h0 + JR(1.0 / 6.0) * (p.Dr[i] + p.Ds[i]);
    }
}

// detJ > 0 (and finite, for FP64): an FP64 comparison is an FP64-pipe
// instruction, so the double's bits are tested on the integer pipe instead
// (a positive finite double has sign bit 0 and a biased exponent below 0x7ff)
template <typename JR>
__device__ __forceinline__ bool det_positive(JR d) {
    if constexpr (sizeof(JR) == 8) {
        const long long b = __double_as_longlong(d);
        return b > 0 && b < 0x7ff0000000000000LL;
    } else {
        return d > JR(0);
    }
}

// adjugate (transposed cofactors): J^-1 = adj / det, det = J row 0 . adj column 0
template <typename JR>
__device__ __forceinline__ JR adjugate(const JR J[3][3], JR A[3][3]) {
    A[0][0] = J[1][1] * J[2][2] - J[1][2] * J[2][1];
    A[1][0] = J[1][2] * J[2][0] - J[1][0] * J[2][2];
    A[2][0] = J[1][0] * J[2][1] - J[1][1] * J[2][0];
    A[0][1] = J[0][2] * J[2][1] - J[0][1] * J[2][2];
    A[1][1] = J[0][0] * J[2][2] - J[0][2] * J[2][0];
    A[2][1] = J[0][1] * J[2][0] - J[0][0] * J[2][1];
    A[0][2] = J[0][1] * J[1][2] - J[0][2] * J[1][1];
    A[1][2] = J[0][2] * J[1][0] - J[0][0] * J[1][2];
    A[2][2] = J[0][0] * J[1][1] - J[0][1] * J[1][0];
    return J[0][0] * A[0][0] + J[0][1] * A[1][0] + J[0][2] * A[2][0];
}

// Residual of one element at the Gauss points of its rule (PYR05, PEN06,
// HEX08), in one sweep: the filter width Delta = V_e^(1/3) is known only
// after the last point, and nu_t = Delta^2 q(G) with q(G) = c sqrt(B'/G:G),
// so the subgrid term is accumulated without the Delta^2 factor and added
// once V_e is complete.  J, its adjugate and determinant are in JR (FP64
// for flagged elements), the rest in R.
// MLP closure in an element kernel (CTA = one warpgroup of 128 threads):
// the weights in shared memory, this warp's scratch (mlp_warp_scratch_bytes
// of the element's row count), the warpgroup's feature tiles (row
// 32 (warp % 4) + lane of tile g: this thread's element at Gauss point g),
// the shared zero K block and the tensor-core state.
struct MlpUse {
    const tc::MlpTc *w;
    unsigned char *scratch;
    unsigned char *feat;
    unsigned char *zero;
    tc::Warpgroup *wg;
};
__device__ __forceinline__ int mlp_row() { return 32 * ((threadIdx.x >> 5) & 3) + (threadIdx.x & 31); }

// rows of the network per element: one per Gauss point, one for TET04
// (constant gradient, so every Gauss point has the same nu_t)
__host__ __device__ constexpr int mlp_rows_per_elem(int et) {
    return et == FEA_TET04 ? 1 : (et == FEA_PYR05 ? 8 : (et == FEA_PEN06 ? 6 : 8));
}

// Returns the number of Gauss points whose nu_t fell back from the MLP to
// Vreman (outside the training envelope); 0 without the MLP.
template <int ET, typename R, bool J64, bool MLP = false, bool VAR = true>
__device__ int element_residual(const Gathered<R, J64> &el, const FieldDev &f, const AsmArgs &args, R r[][3],
                                float *nut_out, bool &bad, const MlpUse &mu = MlpUse{}) {
    using JR = typename std::conditional<J64, double, R>::type;
    constexpr int nen = kNen[ET], ng = kNg[ET];
    const uint32_t mask = args.mask;
    const bool want_q = !MLP && args.closure == FEA_CLOSURE_VREMAN && ((mask & FEA_TERM_SGS) || nut_out);
    // model variants: EMAC needs |u_a|^2 at the nodes, anisotropic Vreman the extents
    // VAR = false: the default forms only (no variant code, fewer registers)
    const bool emac = VAR && f.conv_form == 1 && (mask & FEA_TERM_CONV);
    const bool aniso = VAR && f.delta_form == 1;
    R q2[kMaxNen];
    if (emac) {
#pragma unroll
        for (int a = 0; a < nen; ++a) q2[a] = el.U[a][0] * el.U[a][0] + el.U[a][1] * el.U[a][1] + el.U[a][2] * el.U[a][2];
    }
    R dm[3] = {R(0), R(0), R(0)};
    if (aniso) element_extents<nen, R>(el.X, dm);
    const R nu = (mask & FEA_TERM_VISC) ? to_r<R>(f.nu) : R(0);
    const R cv = to_r<R>(f.c_vreman);
    R rs[kMaxNen][3];
#pragma unroll
    for (int a = 0; a < nen; ++a)
#pragma unroll
        for (int i = 0; i < 3; ++i) r[a][i] = rs[a][i] = R(0);
    PrismGeom<JR> pg;
    if constexpr (ET == FEA_PEN06) prism_geom2<JR>(el.X, pg);
    // MLP: phase 1 (this loop) stores each Gauss point's features and its
    // matrix S in the warp's scratch and assembles everything but the
    // subgrid term; phase 2 runs the network over the warp's 32 x ng rows;
    // phase 3 adds the subgrid term with the per-point nu_t.
    const int lane = threadIdx.x & 31;
    float *Stile = reinterpret_cast<float *>(mu.scratch);
    float *ntile = Stile + ng * 9 * 32;   // the network's coefficient C per point
    float *qtile = ntile + ng * 32;
    float *gtile = qtile + ng * 32;       // |G| per point
    uint32_t inside_mask = 0;   // bit g: point g inside the training envelope
    // element volume (sum of the weights W, in R: it only sets Delta)
    R V = R(0);
    // PEN06: the rule's points are 3 triangle points at each of 2 levels zeta
    // (level-major); the r- and s-columns of J and their cross product (the
    // adjugate's last row) depend on zeta only, so they are formed once per
    // level; per point only the zeta-column, two cross products and the
    // determinant c2 . (c0 x c1) remain.  Columns at twice their value
    // (prism_geom2): A = 4 adj J, detj = 8 det J, so J^-1 = 2 A / detj and
    // W = (w / 8) detj.
    JR c0[3], c1[3], a2[3];
#pragma unroll 1
    for (int g = 0; g < ng; ++g) {
        JR J[3][3];
        JR A[3][3];
        JR detj;
        if constexpr (ET == FEA_PEN06) {
            if (g % 3 == 0) {
                const JR pz = ref_xi<JR>(ET, g, 2);
#pragma unroll
                for (int i = 0; i < 3; ++i) {
                    c0[i] = pg.Ar[i] + pz * pg.Dr[i];
                    c1[i] = pg.As[i] + pz * pg.Ds[i];
                }
                a2[0] = c0[1] * c1[2] - c0[2] * c1[1];
                a2[1] = c0[2] * c1[0] - c0[0] * c1[2];
                a2[2] = c0[0] * c1[1] - c0[1] * c1[0];
            }
            // the zeta-column at triangle point q of the level (see PrismGeom)
            const int q = g % 3;
            JR c2[3];
            if (q == 0) {
#pragma unroll
                for (int i = 0; i < 3; ++i) c2[i] = pg.Q[i];
            } else {
#pragma unroll
                for (int i = 0; i < 3; ++i) c2[i] = pg.Q[i] + JR(0.5) * (q == 1 ? pg.Dr[i] : pg.Ds[i]);
            }
            // A row 0 = c1 x c2, row 1 = c2 x c0, row 2 = c0 x c1 (J^-1 = A / det)
            A[0][0] = c1[1] * c2[2] - c1[2] * c2[1];
            A[0][1] = c1[2] * c2[0] - c1[0] * c2[2];
            A[0][2] = c1[0] * c2[1] - c1[1] * c2[0];
            A[1][0] = c2[1] * c0[2] - c2[2] * c0[1];
            A[1][1] = c2[2] * c0[0] - c2[0] * c0[2];
            A[1][2] = c2[0] * c0[1] - c2[1] * c0[0];
#pragma unroll
            for (int j = 0; j < 3; ++j) A[2][j] = a2[j];
            detj = c2[0] * a2[0] + c2[1] * a2[1] + c2[2] * a2[2];
            (void)J;
        } else {
            jacobian_at<ET, R, JR>(el.X, g, J);
            detj = adjugate(J, A);
        }
        if (!det_positive(detj)) bad = true;
        constexpr bool scaled = ET == FEA_PEN06;
        const R detr = to_r<R>(detj);
        const R rdet = (scaled ? R(2) : R(1)) / detr;
        R Ji[3][3];
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j) Ji[i][j] = to_r<R>(A[i][j]) * rdet;
        const R W = detr * (scaled ? ref_w<R>(ET, g) * R(0.125) : ref_w<R>(ET, g));
        V += W;
        // reference-coordinate gradients and the Gauss-point velocity
        R Gx[3][3] = {}, px[3] = {}, ug[3] = {};
#pragma unroll
        for (int a = 0; a < nen; ++a) {
            const R Na = ref_N<R>(ET, g, a);
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const R d = ref_dN<R>(ET, g, a, k);
                px[k] += el.P[a] * d;
#pragma unroll
                for (int i = 0; i < 3; ++i) Gx[i][k] += el.U[a][i] * d;
            }
#pragma unroll
            for (int i = 0; i < 3; ++i) ug[i] += Na * el.U[a][i];
        }
        // physical gradients: G_ij = sum_k Gx_ik Ji_kj
        R G[3][3], gp[3];
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            gp[j] = px[0] * Ji[0][j] + px[1] * Ji[1][j] + px[2] * Ji[2][j];
#pragma unroll
            for (int i = 0; i < 3; ++i) G[i][j] = Gx[i][0] * Ji[0][j] + Gx[i][1] * Ji[1][j] + Gx[i][2] * Ji[2][j];
        }
        // nu_t / Delta^2 (isotropic, scaled once V is known) or nu_t itself (per-direction widths)
        R q = want_q ? (aniso ? vreman_aniso(G, dm, cv) : vreman(G, R(1), cv)) : R(0);
        const R visc_g = nu;
        if constexpr (MLP) {
            float Gf[3][3];
#pragma unroll
            for (int i = 0; i < 3; ++i)
#pragma unroll
                for (int j = 0; j < 3; ++j) Gf[i][j] = float(G[i][j]);
            uint32_t wds[3];
            const bool inside = mlp_gp_words(Gf, *mu.w, wds, &gtile[g * 32 + lane]);
            *reinterpret_cast<uint4 *>(mu.feat + (g * tc::kRows + mlp_row()) * 16) =
                make_uint4(wds[0], wds[1], wds[2], tc::kOnesWord);
            inside_mask |= (uint32_t)inside << g;
            // with an envelope, Vreman's q = nu_t / Delta^2 (nu_t itself with
            // per-direction widths) for the fallback
            if (mu.w->env_on) qtile[g * 32 + lane] = float(aniso ? vreman_aniso(G, dm, cv) : vreman(G, R(1), cv));
        } else {
            if (nut_out) nut_out[g] = float(q);
        }
        const R qs = (mask & FEA_TERM_SGS) ? q : R(0);
        const R trG = G[0][0] + G[1][1] + G[2][2];
        // EMAC: + G^T u - 1/2 grad (|u|^2)_h, the gradient from the reference derivatives
        R kx[3] = {R(0), R(0), R(0)};
        if (emac) {
            R kr[3] = {R(0), R(0), R(0)};
#pragma unroll
            for (int a = 0; a < nen; ++a)
#pragma unroll
                for (int j = 0; j < 3; ++j) kr[j] += q2[a] * ref_dN<R>(ET, g, a, j);
#pragma unroll
            for (int j = 0; j < 3; ++j) kx[j] = kr[0] * Ji[0][j] + kr[1] * Ji[1][j] + kr[2] * Ji[2][j];
        }
        R f0[3];
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            R c = R(0);
            if (mask & FEA_TERM_CONV) c = G[i][0] * ug[0] + G[i][1] * ug[1] + G[i][2] * ug[2] + trG * ug[i];
            if (emac) c += G[0][i] * ug[0] + G[1][i] * ug[1] + G[2][i] * ug[2] - R(0.5) * kx[i];
            f0[i] = W * (c + ((mask & FEA_TERM_PRES) ? gp[i] : R(0)));
        }
        // S_ik = 2 W sum_j eps_ij Ji_kj; viscous part nu S, subgrid part q S
        R S[3][3];
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            R e0 = R(0.5) * (G[i][0] + G[0][i]), e1 = R(0.5) * (G[i][1] + G[1][i]), e2 = R(0.5) * (G[i][2] + G[2][i]);
#pragma unroll
            for (int k = 0; k < 3; ++k) S[i][k] = R(2) * W * (e0 * Ji[k][0] + e1 * Ji[k][1] + e2 * Ji[k][2]);
        }
        if constexpr (MLP) {
#pragma unroll
            for (int i = 0; i < 3; ++i)
#pragma unroll
                for (int k = 0; k < 3; ++k) Stile[(g * 9 + 3 * i + k) * 32 + lane] = float(S[i][k]);
        }
#pragma unroll
        for (int a = 0; a < nen; ++a) {
            const R Na = ref_N<R>(ET, g, a);
            const R d0 = ref_dN<R>(ET, g, a, 0), d1 = ref_dN<R>(ET, g, a, 1), d2 = ref_dN<R>(ET, g, a, 2);
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                const R t = S[i][0] * d0 + S[i][1] * d1 + S[i][2] * d2;
                r[a][i] -= Na * f0[i] + visc_g * t;
                if constexpr (!MLP) rs[a][i] -= qs * t;
            }
        }
    }
    int fallbacks = 0;
    if constexpr (MLP) {
        // Delta = V^(1/3) completes every row: column 5, log(Delta^2 |G| / nu)
        const R delta = cbrt_r(V);
        const R d2 = delta * delta;
#pragma unroll 1
        for (int g = 0; g < ng; ++g) {
            bool re_inside;
            reinterpret_cast<uint16_t *>(mu.feat + (g * tc::kRows + mlp_row()) * 16)[5] =
                mlp_re_bits(float(delta), gtile[g * 32 + lane], float(f.nu), *mu.w, &re_inside);
            if (!re_inside) inside_mask &= ~(1u << g);
        }
        // phase 2: the warpgroup's 128 elements x ng points as ng tiles of 128 rows
        tc::run(*mu.wg, mu.w, mu.feat, mu.zero, ng, ntile + lane, 32);
#pragma unroll 1
        for (int g = 0; g < ng; ++g) {
            const bool use = (inside_mask >> g) & 1u;
            fallbacks += !use;
            // nu_t = C Delta^2 |G| (network) or Vreman's
            const R nt = use ? R(ntile[g * 32 + lane]) * d2 * R(gtile[g * 32 + lane])
                             : R(qtile[g * 32 + lane]) * (aniso ? R(1) : d2);
            if (nut_out) nut_out[g] = float(nt);
            if (mask & FEA_TERM_SGS) {
                R Sg[3][3];
#pragma unroll
                for (int i = 0; i < 3; ++i)
#pragma unroll
                    for (int k = 0; k < 3; ++k) Sg[i][k] = R(Stile[(g * 9 + 3 * i + k) * 32 + lane]);
#pragma unroll
                for (int a = 0; a < nen; ++a) {
                    const R d0 = ref_dN<R>(ET, g, a, 0), d1 = ref_dN<R>(ET, g, a, 1), d2 = ref_dN<R>(ET, g, a, 2);
#pragma unroll
                    for (int i = 0; i < 3; ++i) r[a][i] -= nt * (Sg[i][0] * d0 + Sg[i][1] * d1 + Sg[i][2] * d2);
                }
            }
        }
        __syncwarp();   // the scratch is rewritten for the warp's next elements
    } else {
        const R delta = cbrt_r(V);
        const R d2 = aniso ? R(1) : delta * delta;
#pragma unroll
        for (int a = 0; a < nen; ++a)
#pragma unroll
            for (int i = 0; i < 3; ++i) r[a][i] += d2 * rs[a][i];
        if (nut_out && !aniso)
            for (int g = 0; g < ng; ++g) nut_out[g] = float(R(nut_out[g]) * d2);
    }
    return fallbacks;
}

// TET04: affine map, constant gradients; the 4-point rule is exact for the
// degree-2 integrands, so the Gauss sums take their closed forms:
//   sum_g W N_a N_b = V (1 + delta_ab) / 20,  sum_g W N_a = V / 4.
template <typename R, bool J64, bool MLP = false, bool VAR = true>
__device__ int tet_residual(const Gathered<R, J64> &el, const FieldDev &f, const AsmArgs &args, R r[][3],
                            float *nut_out, bool &bad, const MlpUse &mu = MlpUse{}) {
    using JR = typename std::conditional<J64, double, R>::type;
    const uint32_t mask = args.mask;
    JR J[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int k = 0; k < 3; ++k) J[i][k] = el.X[k + 1][i] - el.X[0][i];
    JR Jd[3][3];
    const JR detj = inv3(J, Jd);
    if (!(detj > JR(0))) bad = true;
    const R V = R(detj / JR(6));
    // grad N_k (k = 1..3) = row k-1 of J^-1; grad N_0 = -sum
    R dN[4][3];
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int j = 0; j < 3; ++j) dN[k + 1][j] = R(Jd[k][j]);
#pragma unroll
    for (int j = 0; j < 3; ++j) dN[0][j] = -(dN[1][j] + dN[2][j] + dN[3][j]);
    R G[3][3], gp[3];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        gp[j] = R(0);
#pragma unroll
        for (int i = 0; i < 3; ++i) G[i][j] = R(0);
#pragma unroll
        for (int a = 1; a < 4; ++a) {
            const R d = dN[a][j];
            gp[j] += (el.P[a] - el.P[0]) * d;
#pragma unroll
            for (int i = 0; i < 3; ++i) G[i][j] += (el.U[a][i] - el.U[0][i]) * d;
        }
    }
    R nut = R(0);
    int fallbacks = 0;
    if constexpr (MLP) {
        // one row per element: the warpgroup's 128 elements as one tile
        const int lane = threadIdx.x & 31;
        float Gf[3][3];
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j) Gf[i][j] = float(G[i][j]);
        float *ntile = reinterpret_cast<float *>(mu.scratch + mlp_s_bytes(1));
        uint32_t wds[3];
        float gabs;
        const bool inside = mlp_gp_words(Gf, *mu.w, wds, &gabs);
        bool re_inside;
        const R delta0 = cbrt_r(V);
        wds[2] = (wds[2] & 0xffffu) |
                 ((uint32_t)mlp_re_bits(float(delta0), gabs, float(f.nu), *mu.w, &re_inside) << 16);
        *reinterpret_cast<uint4 *>(mu.feat + mlp_row() * 16) = make_uint4(wds[0], wds[1], wds[2], tc::kOnesWord);
        tc::run(*mu.wg, mu.w, mu.feat, mu.zero, 1, ntile + lane, 32);
        if (inside && re_inside) {
            nut = R(ntile[lane]) * delta0 * delta0 * R(gabs);   // nu_t = C Delta^2 |G|
        } else {
            const R delta = cbrt_r(V);
            if (VAR && f.delta_form == 1) {
                R dmx[3];
                element_extents<4, R>(el.X, dmx);
                nut = vreman_aniso(G, dmx, to_r<R>(f.c_vreman));
            } else {
                nut = vreman(G, delta * delta, to_r<R>(f.c_vreman));
            }
            fallbacks = 4;   // all four Gauss points
        }
        __syncwarp();
    } else if (args.closure == FEA_CLOSURE_VREMAN && ((mask & FEA_TERM_SGS) || nut_out)) {
        if (VAR && f.delta_form == 1) {
            R dmx[3];
            element_extents<4, R>(el.X, dmx);
            nut = vreman_aniso(G, dmx, to_r<R>(f.c_vreman));
        } else {
            const R delta = cbrt_r(V);
            nut = vreman(G, delta * delta, to_r<R>(f.c_vreman));
        }
    }
    if (nut_out) {
#pragma unroll
        for (int g = 0; g < 4; ++g) nut_out[g] = float(nut);
    }
    const R trG = G[0][0] + G[1][1] + G[2][2];
    R visc = R(0);
    if (mask & FEA_TERM_VISC) visc += to_r<R>(f.nu);
    if (mask & FEA_TERM_SGS) visc += nut;
    const R s2 = R(2) * visc * V;
    R sig[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) sig[i][j] = s2 * R(0.5) * (G[i][j] + G[j][i]);
    R su[3] = {el.U[0][0] + el.U[1][0] + el.U[2][0] + el.U[3][0], el.U[0][1] + el.U[1][1] + el.U[2][1] + el.U[3][1],
               el.U[0][2] + el.U[1][2] + el.U[2][2] + el.U[3][2]};
    const R v20 = V * R(0.05), v4 = V * R(0.25);
    // EMAC: + G^T u (same closed form as G u) and -1/2 grad (|u|^2)_h, constant
    // on the element, whose integral against N_a is V/4
    const bool emac = VAR && f.conv_form == 1 && (mask & FEA_TERM_CONV);
    R kq[3] = {R(0), R(0), R(0)};
    if (emac) {
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            const R q = el.U[a][0] * el.U[a][0] + el.U[a][1] * el.U[a][1] + el.U[a][2] * el.U[a][2];
#pragma unroll
            for (int j = 0; j < 3; ++j) kq[j] += q * dN[a][j];
        }
    }
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        R m[3];
#pragma unroll
        for (int i = 0; i < 3; ++i) m[i] = v20 * (el.U[a][i] + su[i]);
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            R v = R(0);
            if (mask & FEA_TERM_CONV) v += G[i][0] * m[0] + G[i][1] * m[1] + G[i][2] * m[2] + trG * m[i];
            if (emac) v += G[0][i] * m[0] + G[1][i] * m[1] + G[2][i] * m[2] - R(0.5) * v4 * kq[i];
            if (mask & FEA_TERM_PRES) v += v4 * gp[i];
            v += sig[i][0] * dN[a][0] + sig[i][1] * dN[a][1] + sig[i][2] * dN[a][2];
            r[a][i] = -v;
        }
    }
    return fallbacks;
}

// Shared memory of a fused-closure CTA (128 threads, one warpgroup) from a
// 128-byte aligned base: the weights (tc::MlpTc), the feature tiles
// [ng][128][8] BF16 and the zero K block, the four warps' scratch, then four
// mbarriers and the TMEM address.
__host__ __device__ constexpr size_t mlp_cta_bytes(int ng) {
    return sizeof(tc::MlpTc) + tc::feat_bytes(ng) + 4 * mlp_warp_scratch_bytes(ng) + 64;
}
// A fused-closure CTA's dynamic shared memory is held at no less than this,
// so that at most two such CTAs share an SM: each allocates 256 of the SM's
// 512 TMEM columns, and a third would wait for one of them to finish.
constexpr size_t kMlpMinCtaSmem = 80 * 1024;

// SMs of the current device (persistent grids of the fused closure)
static int device_sms() {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms > 0 ? sms : 148;
}

// The network's waits keep their default limit (the wait limit a context
// sets applies to the TET04 kernel).
__device__ __forceinline__ void mlp_cta_setup(unsigned char *base, int ng, const void *gw, unsigned *err,
                                              MlpUse &mu, tc::Warpgroup &wg) {
    tc::MlpTc *w = reinterpret_cast<tc::MlpTc *>(base);
    unsigned char *feat = base + sizeof(tc::MlpTc);
    unsigned char *zero = feat + (size_t)ng * tc::kRows * 16;
    unsigned char *scr = zero + tc::kRows * 16;
    uint64_t *bars = reinterpret_cast<uint64_t *>(scr + 4 * mlp_warp_scratch_bytes(ng));
    tc::setup(static_cast<const tc::MlpTc *>(gw), w, zero, bars, wg, err, 0u);
    mu.w = w;
    mu.feat = feat;
    mu.zero = zero;
    mu.scratch = scr + (threadIdx.x >> 5) * mlp_warp_scratch_bytes(ng);
    mu.wg = &wg;
}

// warp-aggregated count of MLP fallbacks (all 32 lanes call it together)
__device__ __forceinline__ void count_fallbacks(unsigned long long *counter, int n) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) n += __shfl_xor_sync(0xffffffffu, n, o);
    if (counter && (threadIdx.x & 31) == 0 && n) atomicAdd(counter, (unsigned long long)n);
}

// ---------------------------------------------------------------------------
// ATOMIC scatter kernel: thread per element, FP64 atomic adds into rhs [3][n]

// Sum of v over the lanes of `peers` (lanes whose elements have the same node
// in this local slot), left in the lowest of them; the others are added in
// increasing lane order, one per round, so the sum order is fixed.  Every
// lane of `act` calls it with its own peers (a partition of act).
__device__ __forceinline__ void peer_sum3(unsigned act, unsigned peers, double &v0, double &v1, double &v2) {
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(peers) - 1;
    unsigned rest = peers & ~(1u << leader);
    double s0 = v0, s1 = v1, s2 = v2;
    while (__any_sync(act, rest != 0u)) {
        const int src = rest ? __ffs(rest) - 1 : lane;
        const double t0 = __shfl_sync(act, v0, src), t1 = __shfl_sync(act, v1, src), t2 = __shfl_sync(act, v2, src);
        if (rest) {
            s0 += t0;
            s1 += t1;
            s2 += t2;
            rest &= rest - 1u;
        }
    }
    v0 = s0, v1 = s1, v2 = s2;
}

// AGG (FEA_SCATTER_WARP): before the FP64 atomics, the lanes of a warp whose
// elements have the same node in the same local slot sum their contributions
// (Morton-ordered neighbours often share a corner in the same slot); the
// lowest such lane issues the atomics.
// One element of the atomic scatter (e_raw may lie past the category's end:
// with the MLP such a thread repeats the last element through the network
// and stores nothing).
template <int ET, typename R, bool J64, bool MLP, bool AGG>
__device__ __forceinline__ void atomic_element(const BucketDev &b, const FieldDev &f, const AsmArgs &args,
                                               int64_t e_raw, unsigned act, const MlpUse &mu) {
    constexpr int nen = kNen[ET], ng = kNg[ET];
    const bool active = e_raw < b.count;
    const int64_t e = active ? e_raw : b.count - 1;
    int idx[nen];
#pragma unroll
    for (int a = 0; a < nen; ++a) idx[a] = __ldg(&b.conn[(int64_t)a * b.count + e]);
    Gathered<R, J64> el;
    gather<ET, R, J64>(f, idx, el);
    R r[kMaxNen][3];
    bool bad = false;
    float nut_tmp[ng];
    float *nut = args.nut ? (active ? args.nut + (int64_t)__ldg(&b.orig[e]) * ng : nut_tmp) : nullptr;
    int fb;
    if constexpr (ET == FEA_TET04)
        fb = tet_residual<R, J64, MLP>(el, f, args, r, nut, bad, mu);
    else
        fb = element_residual<ET, R, J64, MLP>(el, f, args, r, nut, bad, mu);
    if constexpr (MLP) count_fallbacks(args.mlp_fb, active ? fb : 0);
    if (!active) return;
    R chk = R(0);
#pragma unroll
    for (int a = 0; a < nen; ++a) chk += r[a][0] + r[a][1] + r[a][2];
    if (bad) set_err(args.err, ERR_DETJ);
    if (!isfinite(chk)) set_err(args.err, ERR_NONFINITE);
    if constexpr (AGG) {
        __syncwarp(act);
        const int lane = threadIdx.x & 31;
#pragma unroll
        for (int a = 0; a < nen; ++a) {
            const unsigned peers = __match_any_sync(act, idx[a]);
            double v0 = to_f64(r[a][0]), v1 = to_f64(r[a][1]), v2 = to_f64(r[a][2]);
            peer_sum3(act, peers, v0, v1, v2);
            if (lane == __ffs(peers) - 1) {
                atomicAdd(&args.rhs[idx[a]], v0);
                atomicAdd(&args.rhs[f.n + idx[a]], v1);
                atomicAdd(&args.rhs[2 * f.n + idx[a]], v2);
            }
        }
    } else {
#pragma unroll
        for (int a = 0; a < nen; ++a)
#pragma unroll
            for (int i = 0; i < 3; ++i) atomicAdd(&args.rhs[(int64_t)i * f.n + idx[a]], to_f64(r[a][i]));
    }
}

// Thread per element.  With the MLP the kernel is persistent (two CTAs of
// one warpgroup per SM, set up once): each CTA takes blocks of 128
// consecutive elements in turn, the warpgroup running the network over them
// together.
template <int ET, typename R, bool J64, bool MLP = false, bool AGG = false>
__global__ void __launch_bounds__(MLP ? 128 : 256, MLP ? 2 : 1) k_assemble_atomic(BucketDev b, FieldDev f,
                                                                                    AsmArgs args) {
    if constexpr (MLP) {
        extern __shared__ float4 smem4[];
        MlpUse mu{};
        tc::Warpgroup wg;
        mlp_cta_setup(reinterpret_cast<unsigned char *>(smem4), mlp_rows_per_elem(ET), args.mlp, args.err, mu, wg);
        for (int64_t blk = blockIdx.x; blk * 128 < b.count; blk += gridDim.x)
            atomic_element<ET, R, J64, true, false>(b, f, args, blk * 128 + threadIdx.x, 0u, mu);
        tc::teardown(wg);
    } else {
        const int64_t e_raw = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
        // lanes with an element (blocks are whole warps); taken before any lane returns
        const unsigned act = AGG ? __ballot_sync(0xffffffffu, e_raw < b.count) : 0u;
        if (e_raw >= b.count) return;
        atomic_element<ET, R, J64, false, AGG>(b, f, args, e_raw, act, MlpUse{});
    }
}

// COLOUR scatter: thread per element of one colour (elements [e0, e1) of the
// colour-ordered connectivity); no two elements of a colour share a node, so
// the FP64 sums are plain read-modify-writes, in launch (colour) order.
template <int ET, typename R, bool J64>
__global__ void __launch_bounds__(256) k_assemble_colour(BucketDev b, FieldDev f, AsmArgs args, int64_t e0,
                                                         int64_t e1) {
    constexpr int nen = kNen[ET], ng = kNg[ET];
    const int64_t e = e0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= e1) return;
    int idx[nen];
#pragma unroll
    for (int a = 0; a < nen; ++a) idx[a] = __ldg(&b.col_conn[(int64_t)a * b.count + e]);
    Gathered<R, J64> el;
    gather<ET, R, J64>(f, idx, el);
    R r[kMaxNen][3];
    bool bad = false;
    float *nut = args.nut ? args.nut + (int64_t)__ldg(&b.col_orig[e]) * ng : nullptr;
    if constexpr (ET == FEA_TET04)
        tet_residual<R, J64, false>(el, f, args, r, nut, bad);
    else
        element_residual<ET, R, J64, false>(el, f, args, r, nut, bad);
    R chk = R(0);
#pragma unroll
    for (int a = 0; a < nen; ++a) chk += r[a][0] + r[a][1] + r[a][2];
    if (bad) set_err(args.err, ERR_DETJ);
    if (!isfinite(chk)) set_err(args.err, ERR_NONFINITE);
#pragma unroll
    for (int a = 0; a < nen; ++a)
#pragma unroll
        for (int i = 0; i < 3; ++i) args.rhs[(int64_t)i * f.n + idx[a]] += to_f64(r[a][i]);
}

template <int ET>
static cudaError_t launch_colour_t(const BucketDev &b, const FieldDev &f, const AsmArgs &a, fea_prec prec, int threads,
                                   const int64_t *col_off, int n_colours, cudaStream_t s) {
    auto kern = prec == FEA_FP64 ? k_assemble_colour<ET, double, false>
                                 : (b.fp64j ? k_assemble_colour<ET, float, true> : k_assemble_colour<ET, float, false>);
    for (int c = 0; c < n_colours; ++c) {
        const int64_t e0 = col_off[c], e1 = col_off[c + 1];
        if (e1 <= e0) continue;
        kern<<<(unsigned)((e1 - e0 + threads - 1) / threads), threads, 0, s>>>(b, f, a, e0, e1);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_assemble_colour(const BucketDev &b, const FieldDev &f, const AsmArgs &a, fea_prec prec,
                                   int threads, const int64_t *col_off, int n_colours, cudaStream_t s) {
    if (b.count == 0) return cudaSuccess;
    if (!b.col_conn || !b.col_orig || !col_off || a.closure == FEA_CLOSURE_MLP) return cudaErrorInvalidValue;
    if (threads > 256) threads = 256;
    switch (b.etype) {
        case FEA_TET04: return launch_colour_t<FEA_TET04>(b, f, a, prec, threads, col_off, n_colours, s);
        case FEA_PYR05: return launch_colour_t<FEA_PYR05>(b, f, a, prec, threads, col_off, n_colours, s);
        case FEA_PEN06: return launch_colour_t<FEA_PEN06>(b, f, a, prec, threads, col_off, n_colours, s);
        case FEA_HEX08: return launch_colour_t<FEA_HEX08>(b, f, a, prec, threads, col_off, n_colours, s);
    }
    return cudaErrorInvalidValue;
}

template <int ET>
static cudaError_t launch_atomic_t(const BucketDev &b, const FieldDev &f, const AsmArgs &a, fea_prec prec,
                                   int threads, bool agg, cudaStream_t s) {
    const unsigned blocks = (unsigned)((b.count + threads - 1) / threads);
    if (a.closure == FEA_CLOSURE_MLP) {
        // one warpgroup per CTA
        const size_t smem = mlp_smem_bytes(128, mlp_rows_per_elem(ET));
        auto kern = prec == FEA_FP64 ? k_assemble_atomic<ET, double, false, true>
                                     : (b.fp64j ? k_assemble_atomic<ET, float, true, true>
                                                : k_assemble_atomic<ET, float, false, true>);
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        const int64_t blocks128 = (b.count + 127) / 128;
        kern<<<(unsigned)std::min<int64_t>(blocks128, 2 * (int64_t)device_sms()), 128, smem, s>>>(b, f, a);
    } else if (agg) {
        if (prec == FEA_FP64)
            k_assemble_atomic<ET, double, false, false, true><<<blocks, threads, 0, s>>>(b, f, a);
        else if (b.fp64j)
            k_assemble_atomic<ET, float, true, false, true><<<blocks, threads, 0, s>>>(b, f, a);
        else
            k_assemble_atomic<ET, float, false, false, true><<<blocks, threads, 0, s>>>(b, f, a);
    } else if (prec == FEA_FP64)
        k_assemble_atomic<ET, double, false><<<blocks, threads, 0, s>>>(b, f, a);
    else if (b.fp64j)
        k_assemble_atomic<ET, float, true><<<blocks, threads, 0, s>>>(b, f, a);
    else
        k_assemble_atomic<ET, float, false><<<blocks, threads, 0, s>>>(b, f, a);
    return cudaGetLastError();
}

cudaError_t launch_assemble_bucket(const BucketDev &b, const FieldDev &f, const AsmArgs &a, fea_prec prec,
                                   fea_scatter scatter, int threads, cudaStream_t s) {
    if (b.count == 0) return cudaSuccess;
    if (threads > 256) threads = 256;
    // FEA_SCATTER_WARP: warp-aggregated atomics (not with the MLP, whose
    // kernels keep plain atomics); anything else: plain atomics
    const bool agg = scatter == FEA_SCATTER_WARP && a.closure != FEA_CLOSURE_MLP;
    switch (b.etype) {
        case FEA_TET04: return launch_atomic_t<FEA_TET04>(b, f, a, prec, threads, agg, s);
        case FEA_PYR05: return launch_atomic_t<FEA_PYR05>(b, f, a, prec, threads, agg, s);
        case FEA_PEN06: return launch_atomic_t<FEA_PEN06>(b, f, a, prec, threads, agg, s);
        case FEA_HEX08: return launch_atomic_t<FEA_HEX08>(b, f, a, prec, threads, agg, s);
    }
    return cudaErrorInvalidValue;
}

// ---------------------------------------------------------------------------
// CHUNK scatter: one CTA assembles one chunk of C Morton-consecutive elements.
//   A. the chunk's L distinct nodes are staged in shared memory: FP32
//      coordinates relative to the chunk's first node (precomputed from FP64
//      at upload, so edge vectors keep full FP32 precision) and (u, v, w, p);
//   B. thread per element: gather from shared memory, element residual,
//      written to the incidences' positions in the chunk's node-sorted
//      incidence list (no atomics);
//   C. thread per local node: sums its contiguous range (FP32, or
//      compensated two-float sums), converts to FP64 and writes once to the
//      global RHS:
//      a plain store when no other chunk touches the node, else one FP64
//      atomic add per component.

__host__ __device__ __forceinline__ size_t chunk_smem_bytes_dev(const BucketDev &b) {
    const int nen = b.etype == FEA_TET04 ? 4 : (b.etype == FEA_PYR05 ? 5 : (b.etype == FEA_PEN06 ? 6 : 8));
    return sizeof(float4) * (2 * (size_t)b.max_chunk_nodes + (size_t)nen * b.chunk_elems);
}
// offset of the fused closure's block after `bytes` of chunk buffers
__host__ __device__ __forceinline__ size_t mlp_tail_offset(size_t bytes) { return (bytes + 127) & ~(size_t)127; }

__device__ __forceinline__ void two_sum_acc(float &s, float &c, float x) {
    const float t = s + x;
    const float z = t - s;
    c += (s - (t - z)) + (x - z);
    s = t;
}

template <int ET, bool J64, bool COMP, bool MLP = false, bool VAR = true>
__device__ __forceinline__ void chunk_body(const BucketDev &b, const FieldDev &f, const AsmArgs &args, int64_t k,
                                           float4 *smem4, const MlpUse &mu = MlpUse{nullptr, nullptr}) {
    constexpr int nen = kNen[ET], ng = kNg[ET];
    const int C = b.chunk_elems;
    const int64_t e0 = k * (int64_t)C;
    const int ne = (int)min((int64_t)C, b.count - e0);
    const int64_t nb = b.chunk_node_off[k];
    const int L = b.chunk_nodes[k];
    float4 *sX = smem4;
    float4 *sU = smem4 + b.max_chunk_nodes;
    float4 *sR = sU + b.max_chunk_nodes;  // [nen C] residuals in node-sorted incidence order
    constexpr int np = lconn_pitch(ET);
    for (int j = threadIdx.x; j < L; j += blockDim.x) {
        const float4 rec = __ldg(&b.chunk_rec[nb + j]);
        const int id = __float_as_int(rec.w) & 0x7fffffff;
        sX[j] = rec;
        sU[j] = __ldg(&f.up32[id]);
    }
    __syncthreads();
    bool bad = false;
    float chk = 0.0f;
    int fallbacks = 0;
    // warp-uniform trip count: with the MLP every lane of a warp joins the
    // network evaluation; lanes past the chunk's end repeat its last element
    for (int base = 0; base < ne; base += blockDim.x) {
        const int el_raw = base + threadIdx.x;
        if (!MLP && el_raw >= ne) break;
        const bool active = el_raw < ne;
        const int el = active ? el_raw : ne - 1;
        const int64_t e = e0 + el;
        Gathered<float, J64> g;
        int loc[nen];
        uint16_t lbuf[2 * np];
        if constexpr (np == 4) {
            const uint4 v = __ldg(reinterpret_cast<const uint4 *>(b.lconn) + e);
            memcpy(lbuf, &v, 16);
        } else {
            const uint4 v0 = __ldg(reinterpret_cast<const uint4 *>(b.lconn) + 2 * e);
            const uint4 v1 = __ldg(reinterpret_cast<const uint4 *>(b.lconn) + 2 * e + 1);
            memcpy(lbuf, &v0, 16);
            memcpy(lbuf + 8, &v1, 16);
        }
#pragma unroll
        for (int a = 0; a < nen; ++a) {
            loc[a] = lbuf[a];
            const float4 x = sX[loc[a]];
            const float4 u = sU[loc[a]];
            g.U[a][0] = u.x;
            g.U[a][1] = u.y;
            g.U[a][2] = u.z;
            g.P[a] = u.w;
            if constexpr (J64) {
                const int64_t id = __float_as_int(x.w) & 0x7fffffff;
                g.X[a][0] = __ldg(&f.xyz64[id]);
                g.X[a][1] = __ldg(&f.xyz64[f.n + id]);
                g.X[a][2] = __ldg(&f.xyz64[2 * f.n + id]);
            } else {
                g.X[a][0] = x.x;
                g.X[a][1] = x.y;
                g.X[a][2] = x.z;
            }
        }
        float r[kMaxNen][3];
        float nut_tmp[ng];
        float *nut = args.nut ? (active ? args.nut + (int64_t)__ldg(&b.orig[e]) * ng : nut_tmp) : nullptr;
        int fb;
        if constexpr (ET == FEA_TET04)
            fb = tet_residual<float, J64, MLP, VAR>(g, f, args, r, nut, bad, mu);
        else
            fb = element_residual<ET, float, J64, MLP, VAR>(g, f, args, r, nut, bad, mu);
        if (active) fallbacks += fb;
        if (!active) continue;
#pragma unroll
        for (int a = 0; a < nen; ++a) {
            sR[lbuf[np + a]] = make_float4(r[a][0], r[a][1], r[a][2], 0.0f);
            chk += r[a][0] + r[a][1] + r[a][2];
        }
    }
    if constexpr (MLP) count_fallbacks(args.mlp_fb, fallbacks);
    if (bad) set_err(args.err, ERR_DETJ);
    if (!isfinite(chk)) set_err(args.err, ERR_NONFINITE);
    __syncthreads();
    for (int j = threadIdx.x; j < L; j += blockDim.x) {
        const uint32_t rg = __ldg(&b.inc_range[nb + j]);
        const int start = (int)(rg & 0xffffu), cnt = (int)(rg >> 16);
        float s0 = 0.f, s1 = 0.f, s2 = 0.f, c0 = 0.f, c1 = 0.f, c2 = 0.f;
        for (int q = 0; q < cnt; ++q) {
            const float4 v = sR[start + q];
            if constexpr (COMP) {
                two_sum_acc(s0, c0, v.x);
                two_sum_acc(s1, c1, v.y);
                two_sum_acc(s2, c2, v.z);
            } else {
                s0 += v.x;
                s1 += v.y;
                s2 += v.z;
            }
        }
        const int bits = __float_as_int(sX[j].w);
        const int64_t id = bits & 0x7fffffff;
        double v0 = f32_to_f64_exact(s0), v1 = f32_to_f64_exact(s1), v2 = f32_to_f64_exact(s2);
        if constexpr (COMP) {
            v0 += f32_to_f64_exact(c0);
            v1 += f32_to_f64_exact(c1);
            v2 += f32_to_f64_exact(c2);
        }
        double *r0 = args.rhs + id, *r1 = args.rhs + f.n + id, *r2 = args.rhs + 2 * f.n + id;
        if (bits < 0) {
            atomicAdd(r0, v0);
            atomicAdd(r1, v1);
            atomicAdd(r2, v2);
        } else {
            *r0 = v0;
            *r1 = v1;
            *r2 = v2;
        }
    }
}

// FP64-Jacobian categories are held to 128 registers a thread: a 128-thread
// CTA then takes the register share of one TET04 CTA, so that these kernels
// find room beside the persistent TET04 kernel (on a side stream, or as
// its programmatic dependent filling its tail, they overlap it); the few
// spills cost less than the overlap gains.  HEX08 and PYR05
// (216 and 150 registers unbounded) are held there too: with 256 threads
// the channel mesh assembles 5 % faster (measured).
template <int ET, bool J64, bool COMP, bool MLP = false, bool VAR = true>
__global__ void __launch_bounds__(MLP ? 128 : 256, (MLP || J64 || ET == FEA_HEX08 || ET == FEA_PYR05) ? 2 : 1)
    k_assemble_chunk(BucketDev b, FieldDev f, AsmArgs args) {
    extern __shared__ float4 smem4[];
    MlpUse mu{};
    tc::Warpgroup wg;
    if constexpr (MLP) {
        // the fused closure's block after the chunk's buffers (one warpgroup)
        unsigned char *tail = reinterpret_cast<unsigned char *>(smem4) + mlp_tail_offset(chunk_smem_bytes_dev(b));
        mlp_cta_setup(tail, mlp_rows_per_elem(ET), args.mlp, args.err, mu, wg);
    }
    if constexpr (MLP) {
        // persistent: two CTAs per SM take the chunks in turn
        for (int64_t k = blockIdx.x; k < b.n_chunks; k += gridDim.x) {
            chunk_body<ET, J64, COMP, MLP, VAR>(b, f, args, k, smem4, mu);
            __syncthreads();   // the chunk buffers are refilled by the next chunk
        }
        tc::teardown(wg);
    } else {
        chunk_body<ET, J64, COMP, MLP, VAR>(b, f, args, blockIdx.x, smem4, mu);
    }
    // as a programmatic dependent: the grid it overlapped has completed (and
    // its writes are visible) before this one does, so whatever the stream
    // runs next sees both; a no-op for an ordinary launch
    asm volatile("griddepcontrol.wait;" ::: "memory");
}

// ---------------------------------------------------------------------------
// Batched persistent launch: every CTA pulls (category, chunk) work items of
// many meshes from a device counter, heaviest categories first, and runs the
// chunk body of the item's element type; per-item descriptors (category,
// field, RHS) come from device tables built by the host per call.

struct BatchItem {
    int32_t bucket;   // index into the descriptor tables
    int32_t chunk;    // chunk index within the bucket
};

template <bool MLP, bool VAR = true>
__global__ void __launch_bounds__(MLP ? 128 : 256, 2) k_assemble_batch(const BucketDev *__restrict__ bk,
                                                        const FieldDev *__restrict__ fd,
                                                        const AsmArgs *__restrict__ ag,
                                                        const BatchItem *__restrict__ items, int64_t n_items,
                                                        unsigned long long *counter, size_t chunk_bytes) {
    extern __shared__ float4 smem4[];
    __shared__ long long item_s;
    MlpUse mu{};
    tc::Warpgroup wg;
    if constexpr (MLP) {
        // element types vary per item: tiles and scratch for the largest row count
        unsigned char *tail = reinterpret_cast<unsigned char *>(smem4) + mlp_tail_offset(chunk_bytes);
        mlp_cta_setup(tail, kMaxNg, ag[0].mlp, ag[0].err, mu, wg);
    }
    for (;;) {
        if (threadIdx.x == 0) item_s = (long long)atomicAdd(counter, 1ull);
        __syncthreads();
        const long long w = item_s;
        __syncthreads();
        if (w >= n_items) break;
        const BatchItem it = items[w];
        const BucketDev b = bk[it.bucket];
        const FieldDev f = fd[it.bucket];
        const AsmArgs a = ag[it.bucket];
        switch (b.etype * 2 + b.fp64j) {
            case 0: chunk_body<FEA_TET04, false, false, MLP, VAR>(b, f, a, it.chunk, smem4, mu); break;
            case 2: chunk_body<FEA_PYR05, false, false, MLP, VAR>(b, f, a, it.chunk, smem4, mu); break;
            case 4: chunk_body<FEA_PEN06, false, false, MLP, VAR>(b, f, a, it.chunk, smem4, mu); break;
            case 5: chunk_body<FEA_PEN06, true, false, MLP, VAR>(b, f, a, it.chunk, smem4, mu); break;
            case 6: chunk_body<FEA_HEX08, false, false, MLP, VAR>(b, f, a, it.chunk, smem4, mu); break;
            default: break;   // FP64-Jacobian TET04/PYR05/HEX08: not batched (host falls back)
        }
        __syncthreads();   // shared memory is reused by the next item
    }
    if constexpr (MLP) tc::teardown(wg);
}

cudaError_t launch_assemble_batch(const void *buckets, const void *fields, const void *args, const void *items,
                                  int64_t n_items, unsigned long long *counter, size_t smem, int sms, bool mlp,
                                  bool variants, cudaStream_t s) {
    if (n_items == 0) return cudaSuccess;
    const size_t chunk_bytes = smem;
    const int threads = mlp ? 128 : 256;   // the fused closure: one warpgroup per CTA
    if (mlp) smem = mlp_tail_offset(smem) + mlp_smem_bytes(threads, kMaxNg);
    if (smem > kMaxBlockSmem) return cudaErrorInvalidConfiguration;
    auto kern = mlp ? k_assemble_batch<true> : (variants ? k_assemble_batch<false, true> : k_assemble_batch<false, false>);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    e = cudaMemsetAsync(counter, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
    if (mlp) per_sm = std::min(per_sm, 2);   // 256 TMEM columns per CTA
    const int64_t grid = std::min<int64_t>(n_items, (int64_t)per_sm * sms);
    kern<<<(unsigned)grid, threads, smem, s>>>(static_cast<const BucketDev *>(buckets),
                                           static_cast<const FieldDev *>(fields), static_cast<const AsmArgs *>(args),
                                           static_cast<const BatchItem *>(items), n_items, counter, chunk_bytes);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Pressure projection operators (Algorithm 1), FP64, one thread per element,
// FP64 atomics into the outputs:
//   K_ab = sum_g W_g grad N_a . grad N_b  into a CSR matrix over periodic
//          classes (row/column = class of the node; entry found by binary
//          search in the row);
//   B_a(u) = sum_g W_g N_a (div u)_g,   G_a(p) = sum_g W_g N_a (grad p)_g.

template <int ET>
__device__ __forceinline__ double proj_geometry(const double X[][3], int g, double dN[][3]) {
    constexpr int nen = kNen[ET];
    double J[3][3], Ji[3][3];
    jacobian_at<ET, double, double>(X, g, J);
    const double det = inv3(J, Ji);
#pragma unroll
    for (int a = 0; a < nen; ++a)
#pragma unroll
        for (int j = 0; j < 3; ++j)
            dN[a][j] = c_ref.dN[ET][g][a][0] * Ji[0][j] + c_ref.dN[ET][g][a][1] * Ji[1][j] +
                       c_ref.dN[ET][g][a][2] * Ji[2][j];
    return det;
}

__device__ __forceinline__ int64_t csr_find(const int64_t *rowptr, const int32_t *col, int32_t r, int32_t c) {
    int64_t lo = rowptr[r], hi = rowptr[r + 1] - 1;
    while (lo <= hi) {
        const int64_t mid = (lo + hi) >> 1;
        const int32_t v = col[mid];
        if (v == c) return mid;
        if (v < c)
            lo = mid + 1;
        else
            hi = mid - 1;
    }
    return -1;
}

template <int ET>
__global__ void k_lap_assemble(BucketDev b, const double *xyz, int64_t n, const int32_t *cls, const int64_t *rowptr,
                               const int32_t *col, double *val, unsigned *err) {
    constexpr int nen = kNen[ET], ng = kNg[ET];
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= b.count) return;
    int idx[nen];
    double X[nen][3];
#pragma unroll
    for (int a = 0; a < nen; ++a) {
        idx[a] = b.conn[(int64_t)a * b.count + e];
#pragma unroll
        for (int i = 0; i < 3; ++i) X[a][i] = xyz[(int64_t)i * n + idx[a]];
    }
    double K[nen][nen];
#pragma unroll
    for (int a = 0; a < nen; ++a)
#pragma unroll
        for (int c = 0; c < nen; ++c) K[a][c] = 0.0;
    bool bad = false;
    for (int g = 0; g < ng; ++g) {
        double dN[nen][3];
        const double det = proj_geometry<ET>(X, g, dN);
        if (!(det > 0.0)) bad = true;
        const double W = c_ref.w[ET][g] * det;
#pragma unroll
        for (int a = 0; a < nen; ++a)
#pragma unroll
            for (int c = 0; c < nen; ++c) K[a][c] += W * (dN[a][0] * dN[c][0] + dN[a][1] * dN[c][1] + dN[a][2] * dN[c][2]);
    }
    if (bad) set_err(err, ERR_DETJ);
#pragma unroll
    for (int a = 0; a < nen; ++a) {
        const int32_t r = cls[idx[a]];
#pragma unroll
        for (int c = 0; c < nen; ++c) {
            const int64_t pos = csr_find(rowptr, col, r, cls[idx[c]]);
            if (pos < 0)
                set_err(err, ERR_INDEX);
            else
                atomicAdd(&val[pos], K[a][c]);
        }
    }
}

// DIV: out[a] += W N_a div u;  otherwise out[i][a] += W N_a d_i p
template <int ET, bool DIV>
__global__ void k_divgrad_assemble(BucketDev b, const double *xyz, int64_t n, const double *in, double *out,
                                   unsigned *err) {
    constexpr int nen = kNen[ET], ng = kNg[ET];
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= b.count) return;
    int idx[nen];
    double X[nen][3];
#pragma unroll
    for (int a = 0; a < nen; ++a) {
        idx[a] = b.conn[(int64_t)a * b.count + e];
#pragma unroll
        for (int i = 0; i < 3; ++i) X[a][i] = xyz[(int64_t)i * n + idx[a]];
    }
    double acc[nen][3];
#pragma unroll
    for (int a = 0; a < nen; ++a) acc[a][0] = acc[a][1] = acc[a][2] = 0.0;
    bool bad = false;
    for (int g = 0; g < ng; ++g) {
        double dN[nen][3];
        const double det = proj_geometry<ET>(X, g, dN);
        if (!(det > 0.0)) bad = true;
        const double W = c_ref.w[ET][g] * det;
        double v[3] = {0.0, 0.0, 0.0};
#pragma unroll
        for (int c = 0; c < nen; ++c) {
            if constexpr (DIV) {
#pragma unroll
                for (int i = 0; i < 3; ++i) v[0] += in[(int64_t)i * n + idx[c]] * dN[c][i];
            } else {
                const double pc = in[idx[c]];
#pragma unroll
                for (int i = 0; i < 3; ++i) v[i] += pc * dN[c][i];
            }
        }
#pragma unroll
        for (int a = 0; a < nen; ++a) {
            const double wn = W * c_ref.N[ET][g][a];
#pragma unroll
            for (int i = 0; i < (DIV ? 1 : 3); ++i) acc[a][i] += wn * v[i];
        }
    }
    if (bad) set_err(err, ERR_DETJ);
#pragma unroll
    for (int a = 0; a < nen; ++a) {
        if constexpr (DIV) {
            atomicAdd(&out[idx[a]], acc[a][0]);
        } else {
#pragma unroll
            for (int i = 0; i < 3; ++i) atomicAdd(&out[(int64_t)i * n + idx[a]], acc[a][i]);
        }
    }
}

cudaError_t launch_lap_assemble(const BucketDev &b, const double *xyz, int64_t n, const int32_t *cls,
                                const int64_t *rowptr, const int32_t *col, double *val, unsigned *err,
                                cudaStream_t s) {
    if (b.count == 0) return cudaSuccess;
    const unsigned blocks = (unsigned)((b.count + 127) / 128);
    switch (b.etype) {
        case FEA_TET04: k_lap_assemble<FEA_TET04><<<blocks, 128, 0, s>>>(b, xyz, n, cls, rowptr, col, val, err); break;
        case FEA_PYR05: k_lap_assemble<FEA_PYR05><<<blocks, 128, 0, s>>>(b, xyz, n, cls, rowptr, col, val, err); break;
        case FEA_PEN06: k_lap_assemble<FEA_PEN06><<<blocks, 128, 0, s>>>(b, xyz, n, cls, rowptr, col, val, err); break;
        case FEA_HEX08: k_lap_assemble<FEA_HEX08><<<blocks, 128, 0, s>>>(b, xyz, n, cls, rowptr, col, val, err); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_divgrad_assemble(const BucketDev &b, const double *xyz, int64_t n, bool div, const double *in,
                                    double *out, unsigned *err, cudaStream_t s) {
    if (b.count == 0) return cudaSuccess;
    const unsigned blocks = (unsigned)((b.count + 127) / 128);
#define FEA_DG(ET)                                                                             \
    (div ? (k_divgrad_assemble<ET, true><<<blocks, 128, 0, s>>>(b, xyz, n, in, out, err), 0) \
         : (k_divgrad_assemble<ET, false><<<blocks, 128, 0, s>>>(b, xyz, n, in, out, err), 0))
    switch (b.etype) {
        case FEA_TET04: FEA_DG(FEA_TET04); break;
        case FEA_PYR05: FEA_DG(FEA_PYR05); break;
        case FEA_PEN06: FEA_DG(FEA_PEN06); break;
        case FEA_HEX08: FEA_DG(FEA_HEX08); break;
        default: return cudaErrorInvalidValue;
    }
#undef FEA_DG
    return cudaGetLastError();
}

// u -= dt g / M on free nodes (un = the result), p += dp, FP32 copy refreshed
__global__ void k_project_update(int64_t n, double *uk, double *un, const double *g, const double *minv,
                                 const uint8_t *dirichlet, double *p, const double *dp, float4 *up32, double dt) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double u[3];
        const bool hold = dirichlet && dirichlet[i];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            u[c] = uk[(int64_t)c * n + i];
            if (!hold) u[c] -= dt * g[(int64_t)c * n + i] * minv[i];
            uk[(int64_t)c * n + i] = u[c];
            un[(int64_t)c * n + i] = u[c];
        }
        const double pn = p[i] + dp[i];
        p[i] = pn;
        up32[i] = make_float4((float)u[0], (float)u[1], (float)u[2], (float)pn);
    }
}

cudaError_t launch_project_update(int64_t n, double *uk, double *un, const double *g, const double *minv,
                                  const uint8_t *dirichlet, double *p, const double *dp, float4 *up32, double dt,
                                  int sms, cudaStream_t s) {
    const int64_t grid = std::min<int64_t>((n + 255) / 256, (int64_t)sms * 8);
    k_project_update<<<(unsigned)grid, 256, 0, s>>>(n, uk, un, g, minv, dirichlet, p, dp, up32, dt);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Interface exchange of a partitioned mesh: classes of node copies that must
// end with one value (a node shared by parts, with its periodic copies).
// pack: out[c][cls[k]] += v[c][loc[k]]; unpack: v[c][loc[k]] = in[c][cls[k]].
// Out-of-range indices are skipped and flagged (ERR_INDEX).

__global__ void k_iface_pack(const double *v, int64_t n, const int64_t *loc, const int64_t *cls, int64_t m,
                             double *out, int64_t nc, unsigned *err) {
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < m; k += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = loc[k], c = cls[k];
        if (i < 0 || i >= n || c < 0 || c >= nc) {
            set_err(err, ERR_INDEX);
            continue;
        }
#pragma unroll
        for (int d = 0; d < 3; ++d) atomicAdd(&out[d * nc + c], v[d * n + i]);
    }
}

__global__ void k_iface_unpack(const double *in, int64_t nc, const int64_t *loc, const int64_t *cls, int64_t m,
                               double *v, int64_t n, unsigned *err) {
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < m; k += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = loc[k], c = cls[k];
        if (i < 0 || i >= n || c < 0 || c >= nc) {
            set_err(err, ERR_INDEX);
            continue;
        }
#pragma unroll
        for (int d = 0; d < 3; ++d) v[d * n + i] = in[d * nc + c];
    }
}

cudaError_t launch_iface_pack(const double *v, int64_t n, const int64_t *loc, const int64_t *cls, int64_t m,
                              double *out, int64_t nc, unsigned *err, int sms, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(out, 0, sizeof(double) * 3 * (size_t)nc, s);
    if (e != cudaSuccess || m == 0) return e;
    const int64_t grid = std::min<int64_t>((m + 255) / 256, (int64_t)sms * 8);
    k_iface_pack<<<(unsigned)grid, 256, 0, s>>>(v, n, loc, cls, m, out, nc, err);
    return cudaGetLastError();
}

cudaError_t launch_iface_unpack(const double *in, int64_t nc, const int64_t *loc, const int64_t *cls, int64_t m,
                                double *v, int64_t n, unsigned *err, int sms, cudaStream_t s) {
    if (m == 0) return cudaSuccess;
    const int64_t grid = std::min<int64_t>((m + 255) / 256, (int64_t)sms * 8);
    k_iface_unpack<<<(unsigned)grid, 256, 0, s>>>(in, nc, loc, cls, m, v, n, err);
    return cudaGetLastError();
}

size_t batch_item_bytes() { return sizeof(BatchItem); }

// zero the RHS of every mesh of a batch in one launch: blockIdx.y = mesh
__global__ void k_zero_batch(double *const *rhs, const int64_t *len) {
    double *r = rhs[blockIdx.y];
    const int64_t n = len[blockIdx.y];
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        r[i] = 0.0;
}

cudaError_t launch_zero_batch(double *const *rhs_dev, const int64_t *len_dev, int n_meshes, cudaStream_t s) {
    if (n_meshes <= 0) return cudaSuccess;
    k_zero_batch<<<dim3(64, (unsigned)n_meshes), 256, 0, s>>>(rhs_dev, len_dev);
    return cudaGetLastError();
}


size_t chunk_kernel_smem(const BucketDev &b, int compensated) {
    (void)compensated;
    return chunk_smem_bytes(b);
}

size_t chunk_smem_bytes(const BucketDev &b) { return chunk_smem_bytes_dev(b); }

size_t mlp_smem_bytes(int threads, int rows_per_elem) {
    (void)threads;   // the fused closure always runs one warpgroup (128 threads) per CTA
    return std::max(mlp_cta_bytes(rows_per_elem), kMlpMinCtaSmem);
}

size_t chunk_launch_smem(const BucketDev &b, int threads, int compensated, bool mlp) {
    if (!mlp) return chunk_kernel_smem(b, compensated);
    return mlp_tail_offset(chunk_smem_bytes(b)) + mlp_smem_bytes(threads, mlp_rows_per_elem(b.etype));
}

template <int ET, bool J64, bool COMP>
static cudaError_t launch_chunk_v(const BucketDev &b, const FieldDev &f, const AsmArgs &a, int threads,
                                  cudaStream_t s) {
    const bool mlp = a.closure == FEA_CLOSURE_MLP;
    const size_t smem = chunk_launch_smem(b, threads, 0, mlp);
    if (smem > kMaxBlockSmem) return cudaErrorInvalidConfiguration;
    if (mlp) threads = 128;   // the fused closure: one warpgroup per CTA
    const bool var = f.conv_form != 0 || f.delta_form != 0;
    auto kern = mlp ? k_assemble_chunk<ET, J64, COMP, true>
                    : (var ? k_assemble_chunk<ET, J64, COMP, false, true> : k_assemble_chunk<ET, J64, COMP, false, false>);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    const int64_t grid = mlp ? std::min<int64_t>(b.n_chunks, 2 * (int64_t)device_sms()) : b.n_chunks;
    if (!a.pdl) {
        kern<<<(unsigned)grid, threads, smem, s>>>(b, f, a);
        return cudaGetLastError();
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3((unsigned)threads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, b, f, a);
}

template <int ET>
static cudaError_t launch_chunk_t(const BucketDev &b, const FieldDev &f, const AsmArgs &a, int threads, int comp,
                                  cudaStream_t s) {
    if (b.fp64j)
        return comp ? launch_chunk_v<ET, true, true>(b, f, a, threads, s)
                    : launch_chunk_v<ET, true, false>(b, f, a, threads, s);
    return comp ? launch_chunk_v<ET, false, true>(b, f, a, threads, s)
                : launch_chunk_v<ET, false, false>(b, f, a, threads, s);
}

cudaError_t launch_assemble_chunk(const BucketDev &b, const FieldDev &f, const AsmArgs &a, int threads,
                                  int compensated, cudaStream_t s) {
    if (b.count == 0) return cudaSuccess;
    if (!b.lconn || b.n_chunks <= 0) return cudaErrorInvalidValue;
    if (b.etype == FEA_TET04 && !b.fp64j && !compensated && a.closure != FEA_CLOSURE_MLP && f.conv_form == 0 &&
        f.delta_form == 0) {
        if (b.ws_rec) return launch_tet_ws(b, f, a, 0, s);
    }
    if (threads > 256) threads = 256;
    switch (b.etype) {
        case FEA_TET04:
            return launch_chunk_t<FEA_TET04>(b, f, a, threads, compensated, s);
        case FEA_PYR05: return launch_chunk_t<FEA_PYR05>(b, f, a, threads, compensated, s);
        case FEA_PEN06: return launch_chunk_t<FEA_PEN06>(b, f, a, threads, compensated, s);
        case FEA_HEX08: return launch_chunk_t<FEA_HEX08>(b, f, a, threads, compensated, s);
    }
    return cudaErrorInvalidValue;
}

// ---------------------------------------------------------------------------
// lumped mass (FP64): M_a += sum_g W_g N_a(g); records the first element with
// det J <= 0 as (bucket-local index) in *bad.

template <int ET>
__global__ void k_lumped_mass(BucketDev b, const double *xyz, int64_t n, double *mass, unsigned *err,
                              unsigned long long *bad) {
    constexpr int nen = kNen[ET], ng = kNg[ET];
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= b.count) return;
    int idx[nen];
    double X[nen][3];
#pragma unroll
    for (int a = 0; a < nen; ++a) {
        idx[a] = b.conn[(int64_t)a * b.count + e];
#pragma unroll
        for (int i = 0; i < 3; ++i) X[a][i] = xyz[(int64_t)i * n + idx[a]];
    }
    double m[nen] = {};
    bool ok = true;
#pragma unroll
    for (int g = 0; g < ng; ++g) {
        double J[3][3];
        const double d = jacobian_at<ET, double, double>(X, g, J);
        if (!(d > 0.0)) ok = false;
        const double W = c_ref.w[ET][g] * d;
#pragma unroll
        for (int a = 0; a < nen; ++a) m[a] += W * c_ref.N[ET][g][a];
    }
    if (!ok) {
        atomicOr(err, ERR_DETJ);
        atomicMin(bad, (unsigned long long)e);
    }
#pragma unroll
    for (int a = 0; a < nen; ++a) atomicAdd(&mass[idx[a]], m[a]);
}

cudaError_t launch_lumped_mass(const BucketDev &b, const double *xyz64, int64_t n, double *mass, unsigned *err,
                               unsigned long long *bad, cudaStream_t s) {
    if (b.count == 0) return cudaSuccess;
    const int t = 128;
    const unsigned blocks = (unsigned)((b.count + t - 1) / t);
    switch (b.etype) {
        case FEA_TET04: k_lumped_mass<FEA_TET04><<<blocks, t, 0, s>>>(b, xyz64, n, mass, err, bad); break;
        case FEA_PYR05: k_lumped_mass<FEA_PYR05><<<blocks, t, 0, s>>>(b, xyz64, n, mass, err, bad); break;
        case FEA_PEN06: k_lumped_mass<FEA_PEN06><<<blocks, t, 0, s>>>(b, xyz64, n, mass, err, bad); break;
        case FEA_HEX08: k_lumped_mass<FEA_HEX08><<<blocks, t, 0, s>>>(b, xyz64, n, mass, err, bad); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// periodic fold: add slaves into masters, then copy back

__global__ void k_fold_add(const int32_t *slaves, const int32_t *masters, int64_t ns, double *v, int ncomp, int64_t n) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= ns) return;
    const int64_t s = slaves[k], m = masters[k];
    for (int c = 0; c < ncomp; ++c) atomicAdd(&v[c * n + m], v[c * n + s]);
}

__global__ void k_fold_copy(const int32_t *slaves, const int32_t *masters, int64_t ns, double *v, int ncomp,
                            int64_t n) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= ns) return;
    const int64_t s = slaves[k], m = masters[k];
    for (int c = 0; c < ncomp; ++c) v[c * n + s] = v[c * n + m];
}

cudaError_t launch_fold(const int32_t *slaves, const int32_t *masters, int64_t ns, double *v, int ncomp, int64_t n,
                        cudaStream_t s) {
    if (ns == 0) return cudaSuccess;
    const int t = 256;
    const unsigned blocks = (unsigned)((ns + t - 1) / t);
    k_fold_add<<<blocks, t, 0, s>>>(slaves, masters, ns, v, ncomp, n);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_fold_copy<<<blocks, t, 0, s>>>(slaves, masters, ns, v, ncomp, n);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// RK stage update (streaming): u^(k+1) = a u^n + b (u^(k) + dt R / M), Dirichlet
// nodes keep u^n; also refreshes the FP32 packed copy (u, v, w, p).


// u^(k+1) = a u^n + b (u^(k) + dt M^-1 R) = a u^n + b u^(k) + c R, c = b dt / M;
// A0: a = 0 (first stage) reads no u^n except at held nodes.  One node per
// thread, every load of the node issued before any is used (the hold flag
// only selects), so that each warp has all its streams in flight at once.
// un, uk_in and uk_out may alias one another (the last stage writes u^(n+1)
// over u^n; an in-place stage writes over u^(k)): every thread reads its own
// index of each before it writes it, so they carry no __restrict__.
template <bool A0>
__global__ void __launch_bounds__(256) k_rk_update(int64_t n, const double *un, const double *uk_in, double *uk_out,
                                                   double *un_out, const double *__restrict__ rhs,
                                                   const double *__restrict__ minv,
                                                   const uint8_t *__restrict__ dirichlet,
                                                   const double *__restrict__ p64, float4 *up32, double a, double b,
                                                   double bdt) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const bool hold = dirichlet && __ldg(&dirichlet[i]);
    const double c = bdt * __ldg(&minv[i]);
    const double pi = __ldg(&p64[i]);
    double r[3], k[3], o[3];
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        r[q] = __ldg(&rhs[(int64_t)q * n + i]);
        k[q] = uk_in[(int64_t)q * n + i];
        o[q] = (A0 && !hold) ? 0.0 : un[(int64_t)q * n + i];
    }
    double v[3];
#pragma unroll
    for (int q = 0; q < 3; ++q) v[q] = hold ? o[q] : (A0 ? fma(c, r[q], k[q]) : fma(c, r[q], fma(a, o[q], b * k[q])));
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        uk_out[(int64_t)q * n + i] = v[q];
        if (un_out) un_out[(int64_t)q * n + i] = v[q];
    }
    up32[i] = make_float4(f64_to_f32_rn(v[0]), f64_to_f32_rn(v[1]), f64_to_f32_rn(v[2]), f64_to_f32_rn(pi));
}

cudaError_t launch_rk_update(int64_t n, const double *un, const double *uk_in, double *uk_out, double *un_out,
                             const double *rhs, const double *minv, const uint8_t *dirichlet, const double *p64,
                             float4 *up32, double a, double b, double dt, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    const int t = 256;
    const int64_t blocks = (n + t - 1) / t;
    if (blocks > 0x7fffffffLL) return cudaErrorInvalidValue;
    if (a == 0.0 && b == 1.0)
        k_rk_update<true><<<(unsigned)blocks, t, 0, s>>>(n, un, uk_in, uk_out, un_out, rhs, minv, dirichlet, p64,
                                                         up32, a, b, b * dt);
    else
        k_rk_update<false><<<(unsigned)blocks, t, 0, s>>>(n, un, uk_in, uk_out, un_out, rhs, minv, dirichlet, p64,
                                                          up32, a, b, b * dt);
    return cudaGetLastError();
}

__global__ void k_pack_field(int64_t n, const double *u64, const double *p64, float4 *up32) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        up32[i] = make_float4(f64_to_f32_rn(u64[i]), f64_to_f32_rn(u64[n + i]), f64_to_f32_rn(u64[2 * n + i]),
                              f64_to_f32_rn(p64[i]));
}

cudaError_t launch_pack_field(int64_t n, const double *u64, const double *p64, float4 *up32, cudaStream_t s) {
    const int t = 256;
    const int64_t want = (n + t - 1) / t;
    const unsigned blocks = (unsigned)(want < 148 * 16 ? (want > 0 ? want : 1) : 148 * 16);
    k_pack_field<<<blocks, t, 0, s>>>(n, u64, p64, up32);
    return cudaGetLastError();
}

__global__ void k_f32_to_f64(const float *src, double *dst, int64_t count) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = double(src[i]);
}

cudaError_t launch_f32_to_f64(const float *src, double *dst, int64_t count, cudaStream_t s) {
    const int t = 256;
    const int64_t want = (count + t - 1) / t;
    const unsigned blocks = (unsigned)(want < 148 * 16 ? (want > 0 ? want : 1) : 148 * 16);
    k_f32_to_f64<<<blocks, t, 0, s>>>(src, dst, count);
    return cudaGetLastError();
}

__global__ void k_recip(const double *m, double *minv, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        minv[i] = m[i] > 0.0 ? 1.0 / m[i] : 0.0;
}

cudaError_t launch_recip(const double *m, double *minv, int64_t n, cudaStream_t s) {
    const int t = 256;
    const int64_t want = (n + t - 1) / t;
    const unsigned blocks = (unsigned)(want < 148 * 16 ? (want > 0 ? want : 1) : 148 * 16);
    k_recip<<<blocks, t, 0, s>>>(m, minv, n);
    return cudaGetLastError();
}

}  // namespace fea
