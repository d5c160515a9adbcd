// Boundary assembly of Algorithm 1: an equilibrium wall model, i.e. a law of
// the wall applied as a traction on the wall faces.  The paper takes the
// formulation from a reference that is not reproduced in it; this file
// implements the reading stated there in full:
//   * law of the wall (Reichardt): u+ = f(y+),
//       f(y+) = ln(1 + kappa y+) / kappa + C (1 - e^(-y+/11) - (y+/11) e^(-y+/3));
//   * at each Gauss point of a wall face the velocity and the position are
//     interpolated, with the face's shape functions, from each face node's
//     exchange node (an interior node); y is the normal distance of that
//     point from the wall and U the norm of the tangential part of the
//     velocity there;
//   * u_tau > 0 solves U = u_tau f(y u_tau / nu) by Newton from the viscous-
//     sublayer value sqrt(nu U / y);
//   * R_a += - sum_g w_g |x_xi x x_eta| N_a(g) u_tau^2 u_t / U.
// Faces: triangles (3-point degree-2 rule) and bilinear quadrilaterals (2x2
// Gauss).  One thread per face Gauss point; geometry, traction and the sums
// in FP64; u_tau to FP64 accuracy in the FP64 mode, its FP32 root in the
// mixed mode.
#include <cuda_runtime.h>
#include <stdint.h>

#include "fea_internal.h"

namespace fea {

namespace {

__device__ __forceinline__ double reichardt(double yp, double kappa, double c, double &df) {
    // 1 - e^(-y+/11) as -expm1 (no cancellation deep in the viscous sublayer)
    const double m11 = expm1(-yp / 11.0), e11 = 1.0 + m11, e3 = exp(-yp / 3.0);
    df = 1.0 / (1.0 + kappa * yp) + c * (e11 / 11.0 - e3 / 11.0 + yp * e3 / 33.0);
    return log1p(kappa * yp) / kappa + c * (-m11 - (yp / 11.0) * e3);
}

__device__ __forceinline__ float reichardt_f32(float yp, float kappa, float c, float &df) {
    const float m11 = expm1f(-yp / 11.0f), e11 = 1.0f + m11, e3 = expf(-yp / 3.0f);
    df = 1.0f / (1.0f + kappa * yp) + c * (e11 / 11.0f - e3 / 11.0f + yp * e3 / 33.0f);
    return log1pf(kappa * yp) / kappa + c * (-m11 - (yp / 11.0f) * e3);
}

// u_tau with U = u_tau f(y u_tau / nu).  Newton in FP32 from the viscous-
// sublayer value sqrt(nu U / y) until |dv| <= 1e-6 v (30 steps at most).
// F64: then Newton in FP64 from there until |dv| <= 1e-14 v (one or two
// steps: the convergence is quadratic), the FP64 iteration alone from the
// sublayer value being the fallback when the FP32 one leaves the positive
// finite range -- the same root as a pure FP64 iteration, while FP64
// transcendentals cost tens of FP64 operations each on this part and FP32
// ones a few.  !F64 (mixed precision): the FP32 root.  False if the
// iteration does not converge.
template <bool F64>
__device__ bool wall_utau(double U, double y, double nu, double kappa, double c, double &v) {
    const float Uf = (float)U, yf = (float)y, nuf = (float)nu, kf = (float)kappa, cf = (float)c;
    float w = sqrtf(nuf * Uf / yf);
    bool ok32 = false;
    for (int it = 0; it < 30; ++it) {
        float df;
        const float yp = yf * w / nuf;
        const float f = reichardt_f32(yp, kf, cf, df);
        float wn = w - (w * f - Uf) / (f + yp * df);
        if (!(wn > 0.0f)) wn = 0.5f * w;
        const float dw = fabsf(wn - w);
        w = wn;
        if (dw <= 1e-6f * w) {
            ok32 = true;
            break;
        }
    }
    ok32 = ok32 && w > 0.0f && isfinite(w);
    if constexpr (!F64) {
        v = (double)w;
        return ok32;
    }
    v = ok32 ? (double)w : sqrt(nu * U / y);
    for (int it = 0; it < 100; ++it) {
        double df;
        const double yp = y * v / nu;
        const double f = reichardt(yp, kappa, c, df);
        double vn = v - (v * f - U) / (f + yp * df);
        if (!(vn > 0.0)) vn = 0.5 * v;
        const double dv = fabs(vn - v);
        v = vn;
        if (dv <= 1e-14 * v) return true;
    }
    return false;
}

template <int NV>
__device__ __forceinline__ void face_point(int g, double N[NV], double dN[NV][2], double &w) {
    if constexpr (NV == 3) {
        const double a = 1.0 / 6.0, b = 2.0 / 3.0;
        const double xi = g == 1 ? b : a, eta = g == 2 ? b : a;
        N[0] = 1.0 - xi - eta;
        N[1] = xi;
        N[2] = eta;
        dN[0][0] = -1.0, dN[0][1] = -1.0;
        dN[1][0] = 1.0, dN[1][1] = 0.0;
        dN[2][0] = 0.0, dN[2][1] = 1.0;
        w = 1.0 / 6.0;
    } else {
        const double q = 0.57735026918962576451;   // 1/sqrt(3)
        const double xi = (g == 1 || g == 2) ? q : -q, eta = g >= 2 ? q : -q;
        const double sx[4] = {-1, 1, 1, -1}, sy[4] = {-1, -1, 1, 1};
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            N[a] = 0.25 * (1 + sx[a] * xi) * (1 + sy[a] * eta);
            dN[a][0] = 0.25 * sx[a] * (1 + sy[a] * eta);
            dN[a][1] = 0.25 * sy[a] * (1 + sx[a] * xi);
        }
        w = 1.0;
    }
}

// One thread per (face, Gauss point): the Newton solves of a face's points
// run in parallel (a thread per face left most SMs with one warp or two).
template <int NV, bool F64>
__global__ void __launch_bounds__(128) k_wall(WallDev wd, const double *__restrict__ xyz, const double *__restrict__ u,
                                              int64_t n, double nu, double *rhs, unsigned *err) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= wd.n_faces * NV) return;
    const int64_t f = t / NV;
    const int g = (int)(t - f * NV);
    int fa[NV];
    double N[NV], dN[NV][2], w;
    face_point<NV>(g, N, dN, w);
    double xg[3] = {0, 0, 0}, xs[3] = {0, 0, 0}, us[3] = {0, 0, 0}, t1[3] = {0, 0, 0}, t2[3] = {0, 0, 0};
#pragma unroll
    for (int a = 0; a < NV; ++a) {
        fa[a] = __ldg(&wd.face[a * wd.n_faces + f]);
        const int ex = __ldg(&wd.exch[a * wd.n_faces + f]);
        if (fa[a] < 0 || fa[a] >= n || ex < 0 || ex >= n) {
            atomicOr(err, ERR_INDEX);
            return;
        }
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            const double x = __ldg(&xyz[i * n + fa[a]]);
            xg[i] += N[a] * x;
            t1[i] += dN[a][0] * x;
            t2[i] += dN[a][1] * x;
            xs[i] += N[a] * __ldg(&xyz[i * n + ex]);
            us[i] += N[a] * __ldg(&u[i * n + ex]);
        }
    }
    const double nr[3] = {t1[1] * t2[2] - t1[2] * t2[1], t1[2] * t2[0] - t1[0] * t2[2], t1[0] * t2[1] - t1[1] * t2[0]};
    const double area = sqrt(nr[0] * nr[0] + nr[1] * nr[1] + nr[2] * nr[2]);
    if (!(area > 0.0)) {
        atomicOr(err, ERR_WALL_GEOM);
        return;
    }
    const double nh[3] = {nr[0] / area, nr[1] / area, nr[2] / area};
    const double y = -((xs[0] - xg[0]) * nh[0] + (xs[1] - xg[1]) * nh[1] + (xs[2] - xg[2]) * nh[2]);
    if (!(y > 0.0)) {
        atomicOr(err, ERR_WALL_GEOM);
        return;
    }
    const double un = us[0] * nh[0] + us[1] * nh[1] + us[2] * nh[2];
    const double ut[3] = {us[0] - un * nh[0], us[1] - un * nh[1], us[2] - un * nh[2]};
    const double U = sqrt(ut[0] * ut[0] + ut[1] * ut[1] + ut[2] * ut[2]);
    if (U == 0.0) return;
    double v;
    if (!wall_utau<F64>(U, y, nu, wd.kappa, wd.c_plus, v)) atomicOr(err, ERR_WALL_NEWTON);
    const double sc = -w * area * v * v / U;
#pragma unroll
    for (int a = 0; a < NV; ++a)
#pragma unroll
        for (int i = 0; i < 3; ++i) atomicAdd(&rhs[i * n + fa[a]], sc * N[a] * ut[i]);
}

}  // namespace

cudaError_t launch_wall(const WallDev &w, const double *xyz64, const double *u64, int64_t n, double nu, double *rhs,
                        unsigned *err, bool fp64, cudaStream_t s) {
    if (w.n_faces <= 0) return cudaSuccess;
    if (w.nv != 3 && w.nv != 4) return cudaErrorInvalidValue;
    const unsigned blocks = (unsigned)((w.n_faces * w.nv + 127) / 128);
    if (w.nv == 3)
        (fp64 ? k_wall<3, true> : k_wall<3, false>)<<<blocks, 128, 0, s>>>(w, xyz64, u64, n, nu, rhs, err);
    else
        (fp64 ? k_wall<4, true> : k_wall<4, false>)<<<blocks, 128, 0, s>>>(w, xyz64, u64, n, nu, rhs, err);
    return cudaGetLastError();
}

}  // namespace fea
