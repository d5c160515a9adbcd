/*
 * FP64 CPU oracle of the explicit momentum right-hand side (test infrastructure).
 *
 * This file is the plain, slow, obviously-correct definition that the CUDA
 * path is checked against.  Only the tests, the smoke check and the CPU-
 * baseline leg of the benchmark may load it; the product path never does.
 * It shares no source with the CUDA library.
 *
 * What it computes (Borrell et al., "Heterogeneous CPU/GPU co-execution of
 * CFD simulations on the POWER9 architecture", section 2.1):
 *   momentum equation (Eq. momentum), rho = 1, mu = nu:
 *     du/dt + [2 u.eps(u) + (div u) u - 1/2 grad|u|^2] - div(2 nu eps(u)) + grad p + div tau = 0,
 *     eps(u) = 1/2 (grad u + grad u^T), tau = -2 nu_t eps(u) (Vreman closure, section 2.1).
 *   Galerkin FE in space (section 2.1), element-by-element assembly with the
 *   three steps gather / computation / scatter (section 2.3.3):
 *     R_a,i = - sum_e sum_g W_g [ N_a (c_i + d_i p) + 2 (nu + nu_t) eps_ij d_j N_a ],
 *     W_g = w_g det J,  c = G u + (tr G) u  (the bracket evaluated pointwise
 *     on the FE interpolant: 2 eps u - 1/2 grad|u|^2 = G u with G_ij = du_i/dx_j).
 *   Lumped mass: row sums of the element mass matrix of the section 2.3.3
 *     listing, M_a = sum_e sum_g W_g N_a.
 *   Time integration: a three-stage Runge-Kutta momentum update (Algorithm 1);
 *     the stage coefficients are the SSP-RK3 (Shu-Osher) ones, pressure frozen.
 *   Boundary assembly (Algorithm 1): an equilibrium wall model, a law of the
 *     wall applied as a traction on wall faces (readings at orc_reichardt).
 *
 * Readings where the paper is silent (each one is listed in the design notes):
 *   - quadrature per element type (the paper only says a category is a type
 *     plus an integration rule): TET04 4-point degree-2 rule; PEN06 3-point
 *     triangle x 2-point Gauss; HEX08 2x2x2 Gauss; PYR05 8-point collapsed
 *     (Duffy) rule with 2-point Gauss-Jacobi(2,0) in the axial direction;
 *   - Vreman filter width Delta = V_e^(1/3), V_e = sum_g W_g;
 *   - Vreman nu_t = 0 when alpha:alpha == 0 or B_beta <= 0, with B_beta
 *     summed as squared cross products of the rows of G (Lagrange identity,
 *     equal to the printed minor-difference form up to rounding);
 *   - pressure term in gradient form, viscous term in 2 eps form, natural
 *     boundary terms dropped.
 *
 * Layouts (numpy-friendly): xyz, u, rhs are [n_nodes][3] row-major; conn is
 * [n_elem][n_en] with the VTK local node order; p, mass are [n_nodes].
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_TET04 0
#define ORC_PYR05 1
#define ORC_PEN06 2
#define ORC_HEX08 3

#define ORC_TERM_CONV 1u
#define ORC_TERM_VISC 2u
#define ORC_TERM_SGS 4u
#define ORC_TERM_PRES 8u

#define ORC_CLOSURE_NONE 0
#define ORC_CLOSURE_VREMAN 1
#define ORC_CLOSURE_MLP 2

#define MAXN 8
#define MAXG 8

typedef struct {
    int64_t n_nodes;
    const double *xyz;        /* [n_nodes][3] */
    int64_t n_elem[4];
    const int32_t *conn[4];   /* [n_elem][n_en] */
} orc_mesh;

/* MLP closure: 6 -> 64 -> 64 -> 64 -> 1, SiLU hidden, softplus output. */
#define MLP_IN 6
#define MLP_H 64
typedef struct {
    const double *w1, *b1;    /* [64][6], [64] */
    const double *w2, *b2;    /* [64][64], [64] */
    const double *w3, *b3;    /* [64][64], [64] */
    const double *w4, *b4;    /* [64], [1] */
    const double *feat_mean;  /* [6] */
    const double *feat_std;   /* [6] */
    double out_scale;         /* coefficient C = out_scale * softplus(z); nu_t = C Delta^2 |G| */
} orc_mlp;

typedef struct {
    double nu;
    double c_vreman;
    int closure;
    uint32_t mask;
    const orc_mlp *mlp;
    int conv_form;    /* 0: c = G u + (tr G) u;  1: EMAC, c = 2 eps u + (tr G) u - 1/2 grad (|u|^2)_h */
    int delta_form;   /* 0: Delta = V^(1/3);  1: per-direction widths (element extents) in Vreman */
} orc_params;

int orc_nnode(int etype) {
    static const int n[4] = {4, 5, 6, 8};
    return (etype >= 0 && etype < 4) ? n[etype] : 0;
}

int orc_ngauss(int etype) {
    static const int n[4] = {4, 8, 6, 8};
    return (etype >= 0 && etype < 4) ? n[etype] : 0;
}

/* ---------------------------------------------------------------------- */
/* Quadrature rules on the reference elements.
 *   TET04: {r,s,t >= 0, r+s+t <= 1}, volume 1/6.
 *   PYR05: base [-1,1]^2 at zeta = 0, apex zeta = 1, volume 4/3.
 *   PEN06: triangle {r,s >= 0, r+s <= 1} x zeta in [-1,1], volume 1.
 *   HEX08: [-1,1]^3, volume 8.                                            */
int orc_quadrature(int etype, double *pts, double *w) {
    const double g = 1.0 / sqrt(3.0);
    int n = 0;
    if (etype == ORC_TET04) {
        /* degree-2 rule: barycentric coordinates (b, a, a, a) and permutations */
        const double a = (5.0 - sqrt(5.0)) / 20.0;
        const double b = (5.0 + 3.0 * sqrt(5.0)) / 20.0;
        const double P[4][3] = {{a, a, a}, {b, a, a}, {a, b, a}, {a, a, b}};
        for (n = 0; n < 4; ++n) {
            pts[3 * n + 0] = P[n][0];
            pts[3 * n + 1] = P[n][1];
            pts[3 * n + 2] = P[n][2];
            w[n] = 1.0 / 24.0;
        }
        return 4;
    }
    if (etype == ORC_PEN06) {
        const double T[3][2] = {{1.0 / 6.0, 1.0 / 6.0}, {2.0 / 3.0, 1.0 / 6.0}, {1.0 / 6.0, 2.0 / 3.0}};
        const double Z[2] = {-g, g};
        for (int iz = 0; iz < 2; ++iz)
            for (int it = 0; it < 3; ++it) {
                pts[3 * n + 0] = T[it][0];
                pts[3 * n + 1] = T[it][1];
                pts[3 * n + 2] = Z[iz];
                w[n] = 1.0 / 6.0;
                ++n;
            }
        return 6;
    }
    if (etype == ORC_HEX08) {
        for (int k = 0; k < 2; ++k)
            for (int j = 0; j < 2; ++j)
                for (int i = 0; i < 2; ++i) {
                    pts[3 * n + 0] = i ? g : -g;
                    pts[3 * n + 1] = j ? g : -g;
                    pts[3 * n + 2] = k ? g : -g;
                    w[n] = 1.0;
                    ++n;
                }
        return 8;
    }
    if (etype == ORC_PYR05) {
        /* collapsed map (a, b, t) -> ((1-t) a, (1-t) b, t), Jacobian (1-t)^2;
         * a, b: 2-point Gauss-Legendre on [-1,1]; t: 2-point Gauss rule for
         * the weight (1-t)^2 on [0,1] (roots of the degree-2 orthogonal
         * polynomial t^2 - 2t/3 + 1/15; weights from the first two moments). */
        const double s = sqrt(2.0 / 45.0);
        const double t1 = 1.0 / 3.0 - s, t2 = 1.0 / 3.0 + s;
        const double w2 = (1.0 / 12.0 - t1 / 3.0) / (t2 - t1);
        const double w1 = 1.0 / 3.0 - w2;
        const double T[2] = {t1, t2}, WT[2] = {w1, w2};
        for (int k = 0; k < 2; ++k)
            for (int j = 0; j < 2; ++j)
                for (int i = 0; i < 2; ++i) {
                    const double t = T[k];
                    pts[3 * n + 0] = (1.0 - t) * (i ? g : -g);
                    pts[3 * n + 1] = (1.0 - t) * (j ? g : -g);
                    pts[3 * n + 2] = t;
                    w[n] = WT[k];
                    ++n;
                }
        return 8;
    }
    return 0;
}

/* ---------------------------------------------------------------------- */
/* Shape functions N[a] and reference derivatives dN[a][j] = dN_a / dxi_j. */
int orc_shape(int etype, const double *xi, double *N, double *dN) {
    const double r = xi[0], s = xi[1], t = xi[2];
    if (etype == ORC_TET04) {
        N[0] = 1.0 - r - s - t; N[1] = r; N[2] = s; N[3] = t;
        const double d[4][3] = {{-1, -1, -1}, {1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
        for (int a = 0; a < 4; ++a)
            for (int j = 0; j < 3; ++j) dN[3 * a + j] = d[a][j];
        return 4;
    }
    if (etype == ORC_PEN06) {
        const double L[3] = {1.0 - r - s, r, s};
        const double Lr[3] = {-1.0, 1.0, 0.0};
        const double Ls[3] = {-1.0, 0.0, 1.0};
        const double zm = 0.5 * (1.0 - t), zp = 0.5 * (1.0 + t);
        for (int i = 0; i < 3; ++i) {
            N[i] = L[i] * zm;
            N[i + 3] = L[i] * zp;
            dN[3 * i + 0] = Lr[i] * zm;
            dN[3 * i + 1] = Ls[i] * zm;
            dN[3 * i + 2] = -0.5 * L[i];
            dN[3 * (i + 3) + 0] = Lr[i] * zp;
            dN[3 * (i + 3) + 1] = Ls[i] * zp;
            dN[3 * (i + 3) + 2] = 0.5 * L[i];
        }
        return 6;
    }
    if (etype == ORC_HEX08) {
        const double S[8][3] = {{-1, -1, -1}, {1, -1, -1}, {1, 1, -1}, {-1, 1, -1},
                                {-1, -1, 1},  {1, -1, 1},  {1, 1, 1},  {-1, 1, 1}};
        for (int a = 0; a < 8; ++a) {
            const double fx = 1.0 + S[a][0] * r, fy = 1.0 + S[a][1] * s, fz = 1.0 + S[a][2] * t;
            N[a] = 0.125 * fx * fy * fz;
            dN[3 * a + 0] = 0.125 * S[a][0] * fy * fz;
            dN[3 * a + 1] = 0.125 * fx * S[a][1] * fz;
            dN[3 * a + 2] = 0.125 * fx * fy * S[a][2];
        }
        return 8;
    }
    if (etype == ORC_PYR05) {
        /* rational pyramid functions, base corners (xi_i, eta_i), apex N_5 = zeta:
         * N_i = 1/4 [ (1 + xi_i xi)(1 + eta_i eta) - zeta + xi_i eta_i xi eta zeta / (1 - zeta) ] */
        const double B[4][2] = {{-1, -1}, {1, -1}, {1, 1}, {-1, 1}};
        const double q = 1.0 / (1.0 - t);
        for (int i = 0; i < 4; ++i) {
            const double xi_i = B[i][0], et_i = B[i][1];
            const double c = xi_i * et_i;
            N[i] = 0.25 * ((1.0 + xi_i * r) * (1.0 + et_i * s) - t + c * r * s * t * q);
            dN[3 * i + 0] = 0.25 * (xi_i * (1.0 + et_i * s) + c * s * t * q);
            dN[3 * i + 1] = 0.25 * (et_i * (1.0 + xi_i * r) + c * r * t * q);
            dN[3 * i + 2] = 0.25 * (-1.0 + c * r * s * q * q);
        }
        N[4] = t;
        dN[12] = 0.0; dN[13] = 0.0; dN[14] = 1.0;
        return 5;
    }
    return 0;
}

/* ---------------------------------------------------------------------- */
static double det3(const double J[3][3]) {
    return J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1])
         - J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0])
         + J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
}

static void inv3(const double J[3][3], double det, double Ji[3][3]) {
    const double d = 1.0 / det;
    Ji[0][0] = (J[1][1] * J[2][2] - J[1][2] * J[2][1]) * d;
    Ji[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) * d;
    Ji[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) * d;
    Ji[1][0] = (J[1][2] * J[2][0] - J[1][0] * J[2][2]) * d;
    Ji[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) * d;
    Ji[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) * d;
    Ji[2][0] = (J[1][0] * J[2][1] - J[1][1] * J[2][0]) * d;
    Ji[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) * d;
    Ji[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) * d;
}

/* Geometry of one element at every Gauss point:
 *   J_ij = sum_a X_a,i dN_a/dxi_j,  W_g = w_g det J,
 *   dN_a/dx_i = sum_j dN_a/dxi_j (J^-1)_ji.
 * Returns 0, or -1 if some det J <= 0 (inverted / degenerate element). */
int orc_element_geometry(int etype, const double *X /*[nen][3]*/, double *N /*[ng][nen]*/,
                         double *dNdx /*[ng][nen][3]*/, double *W /*[ng]*/, double *detJ /*[ng]*/) {
    double pts[3 * MAXG], w[MAXG], Nl[MAXN], dN[3 * MAXN];
    const int ng = orc_quadrature(etype, pts, w);
    const int nen = orc_nnode(etype);
    if (ng == 0) return -2;
    for (int g = 0; g < ng; ++g) {
        orc_shape(etype, pts + 3 * g, Nl, dN);
        double J[3][3] = {{0}};
        for (int a = 0; a < nen; ++a)
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j) J[i][j] += X[3 * a + i] * dN[3 * a + j];
        const double d = det3(J);
        if (detJ) detJ[g] = d;
        if (!(d > 0.0)) return -1;
        double Ji[3][3];
        inv3(J, d, Ji);
        if (W) W[g] = w[g] * d;
        for (int a = 0; a < nen; ++a) {
            if (N) N[g * nen + a] = Nl[a];
            if (dNdx)
                for (int i = 0; i < 3; ++i) {
                    double v = 0.0;
                    for (int j = 0; j < 3; ++j) v += dN[3 * a + j] * Ji[j][i];
                    dNdx[(g * nen + a) * 3 + i] = v;
                }
        }
    }
    return 0;
}

/* ---------------------------------------------------------------------- */
/* Vreman (2004) eddy viscosity at one point, with G_ij = du_i/dx_j:
 *   alpha_ij = du_j/dx_i = G_ji,
 *   beta_ij  = Delta^2 sum_m alpha_mi alpha_mj   (beta = Delta^2 alpha^T alpha),
 *   B_beta   = b11 b22 - b12^2 + b11 b33 - b13^2 + b22 b33 - b23^2,
 *   nu_t     = c sqrt(B_beta / (alpha_ij alpha_ij)),  0 if alpha:alpha == 0 or B_beta <= 0.
 * Each term b_ii b_jj - b_ij^2 is a principal 2x2 minor of the Gram matrix
 * alpha^T alpha, equal (Lagrange identity) to Delta^4 |a_i x a_j|^2 with a_i
 * the i-th column of alpha, i.e. the i-th row of G.  B_beta is evaluated in
 * that sum-of-squares form: the same number up to rounding, without the
 * cancellation of the difference form where B_beta -> 0 (then the square
 * root would amplify rounding to ~1e-8 relative in nu_t). */
static void cross3(const double *a, const double *b, double *c) {
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}

double orc_vreman(const double *G /*[3][3]*/, double delta, double c) {
    double aa = 0.0;
    for (int k = 0; k < 9; ++k) aa += G[k] * G[k];
    const double *a1 = G, *a2 = G + 3, *a3 = G + 6;   /* columns of alpha = rows of G */
    double x12[3], x13[3], x23[3];
    cross3(a1, a2, x12);
    cross3(a1, a3, x13);
    cross3(a2, a3, x23);
    double minors = 0.0;
    for (int i = 0; i < 3; ++i) minors += x12[i] * x12[i] + x13[i] * x13[i] + x23[i] * x23[i];
    const double d2 = delta * delta;
    const double B = d2 * d2 * minors;
    if (aa == 0.0 || B <= 0.0) return 0.0;
    return c * sqrt(B / aa);
}

/* Vreman with a filter width per direction (Vreman 2004 writes the model
 * for an anisotropic grid): beta_ij = sum_m Delta_m^2 alpha_mi alpha_mj with
 * alpha = G^T, i.e. beta = H H^T for H = G diag(Delta).  Its principal 2x2
 * minors are |h_i x h_j|^2 (h_i = row i of H, Lagrange identity), so
 * B_beta = |h_1 x h_2|^2 + |h_1 x h_3|^2 + |h_2 x h_3|^2. */
double orc_vreman_aniso(const double *G /*[3][3]*/, const double *dm /*[3]*/, double c) {
    double aa = 0.0, H[9];
    for (int k = 0; k < 9; ++k) aa += G[k] * G[k];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) H[3 * i + j] = G[3 * i + j] * dm[j];
    double x12[3], x13[3], x23[3];
    cross3(H, H + 3, x12);
    cross3(H, H + 6, x13);
    cross3(H + 3, H + 6, x23);
    double B = 0.0;
    for (int i = 0; i < 3; ++i) B += x12[i] * x12[i] + x13[i] * x13[i] + x23[i] * x23[i];
    if (aa == 0.0 || B <= 0.0) return 0.0;
    return c * sqrt(B / aa);
}

/* ---------------------------------------------------------------------- */
/* MLP closure.  Features from S = (G + G^T)/2 and O = (G - G^T)/2:
 *   I1 = tr S^2, I2 = tr O^2, I3 = tr S^3, I4 = tr S O^2, I5 = tr S^2 O^2,
 *   x_k = sign(I_k) |I_k|^(1/d_k), d = (2, 2, 3, 3, 4)   (units of a rate),
 *   x_6 = log Delta;  inputs (x - mean) / std.                          */
static void mat3mul(const double A[3][3], const double B[3][3], double C[3][3]) {
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double s = 0.0;
            for (int k = 0; k < 3; ++k) s += A[i][k] * B[k][j];
            C[i][j] = s;
        }
}

static double tr3(const double A[3][3]) { return A[0][0] + A[1][1] + A[2][2]; }

/* Dimensionless inputs of the learned closure (reading of config 5's "five
 * invariants of the velocity-gradient tensor plus the element size", made
 * scale-free): with S = (G + G^T)/2, O = (G - G^T)/2 and g = |G| (Frobenius,
 * g^2 = tr S^2 - tr O^2),
 *   x = (tr S^2 / g^2, tr O^2 / g^2, tr S^3 / g^3, tr S O^2 / g^3,
 *        tr S^2 O^2 / g^4, log(Delta^2 g / nu)),
 * the last the element's Reynolds number.  A vanishing gradient (g = 0) has
 * no direction: x = 0 (and the closure is zero there).  Returns g.        */
double orc_mlp_features(const double *G, double delta, double nu, double *x /*[6]*/) {
    double S[3][3], O[3][3], S2[3][3], O2[3][3], S3[3][3], SO2[3][3], S2O2[3][3];
    double g2 = 0.0;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            S[i][j] = 0.5 * (G[3 * i + j] + G[3 * j + i]);
            O[i][j] = 0.5 * (G[3 * i + j] - G[3 * j + i]);
            g2 += G[3 * i + j] * G[3 * i + j];
        }
    if (!(g2 > 0.0)) {
        for (int k = 0; k < MLP_IN; ++k) x[k] = 0.0;
        return 0.0;
    }
    const double g = sqrt(g2);
    mat3mul(S, S, S2);
    mat3mul(O, O, O2);
    mat3mul(S2, S, S3);
    mat3mul(S, O2, SO2);
    mat3mul(S2, O2, S2O2);
    x[0] = tr3(S2) / g2;
    x[1] = tr3(O2) / g2;
    x[2] = tr3(S3) / (g2 * g);
    x[3] = tr3(SO2) / (g2 * g);
    x[4] = tr3(S2O2) / (g2 * g2);
    x[5] = log(delta * delta * g / nu);
    return g;
}

static double silu(double z) { return z / (1.0 + exp(-z)); }
static double softplus(double z) { return z > 30.0 ? z : log1p(exp(z)); }

/* Forward pass for a batch of raw (un-normalised) features; y = the
 * coefficient C = out_scale softplus(z) (the closure's nu_t is C Delta^2 |G|). */
void orc_mlp_forward(const orc_mlp *m, const double *x /*[B][6]*/, int64_t B, double *y /*[B]*/) {
    for (int64_t b = 0; b < B; ++b) {
        double in[MLP_IN], h1[MLP_H], h2[MLP_H], h3[MLP_H];
        for (int k = 0; k < MLP_IN; ++k) in[k] = (x[b * MLP_IN + k] - m->feat_mean[k]) / m->feat_std[k];
        for (int o = 0; o < MLP_H; ++o) {
            double s = m->b1[o];
            for (int k = 0; k < MLP_IN; ++k) s += m->w1[o * MLP_IN + k] * in[k];
            h1[o] = silu(s);
        }
        for (int o = 0; o < MLP_H; ++o) {
            double s = m->b2[o];
            for (int k = 0; k < MLP_H; ++k) s += m->w2[o * MLP_H + k] * h1[k];
            h2[o] = silu(s);
        }
        for (int o = 0; o < MLP_H; ++o) {
            double s = m->b3[o];
            for (int k = 0; k < MLP_H; ++k) s += m->w3[o * MLP_H + k] * h2[k];
            h3[o] = silu(s);
        }
        double z = m->b4[0];
        for (int k = 0; k < MLP_H; ++k) z += m->w4[k] * h3[k];
        y[b] = m->out_scale * softplus(z);
    }
}

/* ---------------------------------------------------------------------- */
/* Element residual of one element (the "computation" step), FP64.
 *   X [nen][3] coordinates, U [nen][3] velocity, P [nen] pressure (gathered).
 *   r [nen][3] element residual (overwritten).  nut [ng] optional output.
 * Returns 0, or -1 for det J <= 0.                                          */
static int element_rhs(int etype, const double *X, const double *U, const double *P, const orc_params *prm,
                       double *r, double *nut, double *vol) {
    double N[MAXG * MAXN], dNdx[MAXG * MAXN * 3], W[MAXG];
    const int ng = orc_ngauss(etype), nen = orc_nnode(etype);
    if (orc_element_geometry(etype, X, N, dNdx, W, NULL) != 0) return -1;
    double V = 0.0;
    for (int g = 0; g < ng; ++g) V += W[g];
    if (vol) *vol = V;
    const double delta = cbrt(V);
    /* per-direction widths: the element's extents along the axes */
    double dm[3];
    for (int i = 0; i < 3; ++i) {
        double lo = X[i], hi = X[i];
        for (int a = 1; a < nen; ++a) {
            lo = fmin(lo, X[3 * a + i]);
            hi = fmax(hi, X[3 * a + i]);
        }
        dm[i] = hi - lo;
    }
    memset(r, 0, sizeof(double) * 3 * nen);
    for (int g = 0; g < ng; ++g) {
        const double *Ng = N + g * nen;
        const double *dg = dNdx + g * nen * 3;
        double ug[3] = {0, 0, 0}, G[9] = {0}, gp[3] = {0, 0, 0};
        for (int a = 0; a < nen; ++a) {
            for (int i = 0; i < 3; ++i) {
                ug[i] += Ng[a] * U[3 * a + i];
                gp[i] += dg[3 * a + i] * P[a];
                for (int j = 0; j < 3; ++j) G[3 * i + j] += U[3 * a + i] * dg[3 * a + j];
            }
        }
        const double trG = G[0] + G[4] + G[8];
        double eps[3][3];
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) eps[i][j] = 0.5 * (G[3 * i + j] + G[3 * j + i]);
        double nut_g = 0.0;
        if ((prm->mask & ORC_TERM_SGS) || nut) {
            if (prm->closure == ORC_CLOSURE_VREMAN) {
                nut_g = prm->delta_form ? orc_vreman_aniso(G, dm, prm->c_vreman) : orc_vreman(G, delta, prm->c_vreman);
            } else if (prm->closure == ORC_CLOSURE_MLP && prm->mlp) {
                double f[MLP_IN];
                const double g = orc_mlp_features(G, delta, prm->nu, f);
                double C = 0.0;
                if (g > 0.0) orc_mlp_forward(prm->mlp, f, 1, &C);
                nut_g = C * delta * delta * g;
            }
        }
        if (nut) nut[g] = nut_g;
        double cvec[3] = {0, 0, 0};
        if (prm->mask & ORC_TERM_CONV) {
            /* EMAC: grad of the interpolated kinetic energy (|u|^2)_h = sum_a N_a |u_a|^2 */
            double k[3] = {0, 0, 0};
            if (prm->conv_form)
                for (int a = 0; a < nen; ++a) {
                    const double q = U[3 * a] * U[3 * a] + U[3 * a + 1] * U[3 * a + 1] + U[3 * a + 2] * U[3 * a + 2];
                    for (int i = 0; i < 3; ++i) k[i] += q * dg[3 * a + i];
                }
            for (int i = 0; i < 3; ++i) {
                double s = trG * ug[i];
                for (int j = 0; j < 3; ++j) s += G[3 * i + j] * ug[j];
                if (prm->conv_form)
                    for (int j = 0; j < 3; ++j) s += G[3 * j + i] * ug[j];
                cvec[i] = prm->conv_form ? s - 0.5 * k[i] : s;
            }
        }
        double f0[3];
        for (int i = 0; i < 3; ++i) f0[i] = cvec[i] + ((prm->mask & ORC_TERM_PRES) ? gp[i] : 0.0);
        double visc = 0.0;
        if (prm->mask & ORC_TERM_VISC) visc += prm->nu;
        if (prm->mask & ORC_TERM_SGS) visc += nut_g;
        for (int a = 0; a < nen; ++a)
            for (int i = 0; i < 3; ++i) {
                double s = Ng[a] * f0[i];
                for (int j = 0; j < 3; ++j) s += 2.0 * visc * eps[i][j] * dg[3 * a + j];
                r[3 * a + i] -= W[g] * s;
            }
    }
    return 0;
}

static void gather(const orc_mesh *m, int etype, int64_t e, const double *u, const double *p, double *X, double *U,
                   double *P) {
    const int nen = orc_nnode(etype);
    const int32_t *c = m->conn[etype] + e * nen;
    for (int a = 0; a < nen; ++a) {
        const int64_t n = c[a];
        for (int i = 0; i < 3; ++i) {
            X[3 * a + i] = m->xyz[3 * n + i];
            U[3 * a + i] = u[3 * n + i];
        }
        P[a] = p[n];
    }
}

static int64_t g_bad_elem = -1;
static int g_bad_type = -1;

int64_t orc_bad_element(int *etype) {
    if (etype) *etype = g_bad_type;
    return g_bad_elem;
}

/* Validates connectivity indices; returns 0 or -3. */
static int check_conn(const orc_mesh *m) {
    for (int t = 0; t < 4; ++t) {
        const int nen = orc_nnode(t);
        for (int64_t k = 0; k < m->n_elem[t] * nen; ++k)
            if (m->conn[t][k] < 0 || m->conn[t][k] >= m->n_nodes) {
                g_bad_type = t;
                g_bad_elem = k / nen;
                return -3;
            }
    }
    return 0;
}

/* Serial assembly in natural element order (types in order TET, PYR, PEN, HEX).
 *   rhs [n_nodes][3] is overwritten.  nut[t] optional [n_elem][ng] per type;
 *   vol[t] optional [n_elem] element volumes.  Returns 0, -1 (det J <= 0),
 *   -3 (index out of range).                                              */
int orc_assemble_rhs(const orc_mesh *m, const double *u, const double *p, const orc_params *prm, double *rhs,
                     double **nut, double **vol) {
    if (check_conn(m)) return -3;
    memset(rhs, 0, sizeof(double) * 3 * m->n_nodes);
    double X[3 * MAXN], U[3 * MAXN], P[MAXN], r[3 * MAXN];
    for (int t = 0; t < 4; ++t) {
        const int nen = orc_nnode(t), ng = orc_ngauss(t);
        for (int64_t e = 0; e < m->n_elem[t]; ++e) {
            gather(m, t, e, u, p, X, U, P);
            double *nut_e = (nut && nut[t]) ? nut[t] + e * ng : NULL;
            double *vol_e = (vol && vol[t]) ? vol[t] + e : NULL;
            if (element_rhs(t, X, U, P, prm, r, nut_e, vol_e) != 0) {
                g_bad_type = t;
                g_bad_elem = e;
                return -1;
            }
            const int32_t *c = m->conn[t] + e * nen;
            for (int a = 0; a < nen; ++a)
                for (int i = 0; i < 3; ++i) rhs[3 * (int64_t)c[a] + i] += r[3 * a + i];
        }
    }
    return 0;
}

/* The same assembly with OpenMP threads over elements, per-thread private
 * RHS arrays and a final reduction (timed CPU baseline). */
int orc_assemble_rhs_omp(const orc_mesh *m, const double *u, const double *p, const orc_params *prm, double *rhs,
                         int nthreads) {
    if (check_conn(m)) return -3;
    const int64_t n3 = 3 * m->n_nodes;
    int status = 0;
#ifdef _OPENMP
    if (nthreads <= 0) nthreads = omp_get_max_threads();
#else
    nthreads = 1;
#endif
    double *priv = (double *)calloc((size_t)nthreads * (size_t)n3, sizeof(double));
    if (!priv) return -4;
#ifdef _OPENMP
#pragma omp parallel num_threads(nthreads)
#endif
    {
        int tid = 0;
#ifdef _OPENMP
        tid = omp_get_thread_num();
#endif
        double *mine = priv + (size_t)tid * (size_t)n3;
        double X[3 * MAXN], U[3 * MAXN], P[MAXN], r[3 * MAXN];
        for (int t = 0; t < 4; ++t) {
            const int nen = orc_nnode(t);
#ifdef _OPENMP
#pragma omp for schedule(static)
#endif
            for (int64_t e = 0; e < m->n_elem[t]; ++e) {
                gather(m, t, e, u, p, X, U, P);
                if (element_rhs(t, X, U, P, prm, r, NULL, NULL) != 0) {
                    status = -1;
                    continue;
                }
                const int32_t *c = m->conn[t] + e * nen;
                for (int a = 0; a < nen; ++a)
                    for (int i = 0; i < 3; ++i) mine[3 * (int64_t)c[a] + i] += r[3 * a + i];
            }
        }
    }
#ifdef _OPENMP
#pragma omp parallel for schedule(static) num_threads(nthreads)
#endif
    for (int64_t k = 0; k < n3; ++k) {
        double s = 0.0;
        for (int th = 0; th < nthreads; ++th) s += priv[(size_t)th * (size_t)n3 + k];
        rhs[k] = s;
    }
    free(priv);
    return status;
}

int orc_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Lumped mass M_a = sum_e sum_g W_g N_a(g): the row sum of the element mass
 * matrix Ae_ab = sum_g J w N_a N_b of the section 2.3.3 listing. */
int orc_lumped_mass(const orc_mesh *m, double *mass) {
    if (check_conn(m)) return -3;
    memset(mass, 0, sizeof(double) * m->n_nodes);
    double X[3 * MAXN], N[MAXG * MAXN], W[MAXG];
    for (int t = 0; t < 4; ++t) {
        const int nen = orc_nnode(t), ng = orc_ngauss(t);
        for (int64_t e = 0; e < m->n_elem[t]; ++e) {
            const int32_t *c = m->conn[t] + e * nen;
            for (int a = 0; a < nen; ++a)
                for (int i = 0; i < 3; ++i) X[3 * a + i] = m->xyz[3 * (int64_t)c[a] + i];
            if (orc_element_geometry(t, X, N, NULL, W, NULL) != 0) {
                g_bad_type = t;
                g_bad_elem = e;
                return -1;
            }
            for (int a = 0; a < nen; ++a) {
                double s = 0.0;
                for (int b = 0; b < nen; ++b)
                    for (int g = 0; g < ng; ++g) s += W[g] * N[g * nen + a] * N[g * nen + b];
                mass[c[a]] += s;
            }
        }
    }
    return 0;
}

/* Consistent element mass matrix Ae_ab (listing of section 2.3.3), one element. */
int orc_element_mass(int etype, const double *X, double *Ae /*[nen][nen]*/) {
    double N[MAXG * MAXN], W[MAXG];
    const int nen = orc_nnode(etype), ng = orc_ngauss(etype);
    if (orc_element_geometry(etype, X, N, NULL, W, NULL) != 0) return -1;
    for (int a = 0; a < nen; ++a)
        for (int b = 0; b < nen; ++b) {
            double s = 0.0;
            for (int g = 0; g < ng; ++g) s += W[g] * N[g * nen + a] * N[g * nen + b];
            Ae[a * nen + b] = s;
        }
    return 0;
}

/* ---- pressure projection operators (Algorithm 1: "element assembly of the
 * Laplacian matrix", the pressure equation and the velocity correction) ----
 * Galerkin forms over every element and Gauss point, W_g = w_g det J:
 *   K_ab  = sum W_g grad N_a . grad N_b          (Laplacian, assembled once)
 *   B_a(u) = sum W_g N_a (div u)_g               (divergence of a nodal field)
 *   G_a(p) = sum W_g N_a (grad p)_g              (gradient of a nodal scalar)  */

/* K as COO triplets: entry k = e*nen^2 + a*nen + b of each type block, in the
 * order of the types 0..3 (duplicates are summed by the caller). */
int orc_assemble_laplacian_coo(const orc_mesh *m, int64_t *rows, int64_t *cols, double *vals) {
    if (check_conn(m)) return -3;
    double X[3 * MAXN], dN[MAXG * MAXN * 3], W[MAXG];
    int64_t k = 0;
    for (int t = 0; t < 4; ++t) {
        const int nen = orc_nnode(t), ng = orc_ngauss(t);
        for (int64_t e = 0; e < m->n_elem[t]; ++e) {
            const int32_t *c = m->conn[t] + e * nen;
            for (int a = 0; a < nen; ++a)
                for (int i = 0; i < 3; ++i) X[3 * a + i] = m->xyz[3 * (int64_t)c[a] + i];
            if (orc_element_geometry(t, X, NULL, dN, W, NULL) != 0) {
                g_bad_type = t;
                g_bad_elem = e;
                return -1;
            }
            for (int a = 0; a < nen; ++a)
                for (int b = 0; b < nen; ++b) {
                    double s = 0.0;
                    for (int g = 0; g < ng; ++g)
                        for (int i = 0; i < 3; ++i)
                            s += W[g] * dN[(g * nen + a) * 3 + i] * dN[(g * nen + b) * 3 + i];
                    rows[k] = c[a];
                    cols[k] = c[b];
                    vals[k] = s;
                    ++k;
                }
        }
    }
    return 0;
}

/* B(u) [n_nodes] for a nodal velocity u [n_nodes][3]. */
int orc_assemble_divergence(const orc_mesh *m, const double *u, double *out) {
    if (check_conn(m)) return -3;
    memset(out, 0, sizeof(double) * m->n_nodes);
    double X[3 * MAXN], N[MAXG * MAXN], dN[MAXG * MAXN * 3], W[MAXG];
    for (int t = 0; t < 4; ++t) {
        const int nen = orc_nnode(t), ng = orc_ngauss(t);
        for (int64_t e = 0; e < m->n_elem[t]; ++e) {
            const int32_t *c = m->conn[t] + e * nen;
            for (int a = 0; a < nen; ++a)
                for (int i = 0; i < 3; ++i) X[3 * a + i] = m->xyz[3 * (int64_t)c[a] + i];
            if (orc_element_geometry(t, X, N, dN, W, NULL) != 0) return -1;
            for (int g = 0; g < ng; ++g) {
                double div = 0.0;
                for (int b = 0; b < nen; ++b)
                    for (int i = 0; i < 3; ++i) div += u[3 * (int64_t)c[b] + i] * dN[(g * nen + b) * 3 + i];
                for (int a = 0; a < nen; ++a) out[c[a]] += W[g] * N[g * nen + a] * div;
            }
        }
    }
    return 0;
}

/* G(p) [n_nodes][3] for a nodal scalar p [n_nodes]. */
int orc_assemble_gradient(const orc_mesh *m, const double *p, double *out) {
    if (check_conn(m)) return -3;
    memset(out, 0, sizeof(double) * 3 * m->n_nodes);
    double X[3 * MAXN], N[MAXG * MAXN], dN[MAXG * MAXN * 3], W[MAXG];
    for (int t = 0; t < 4; ++t) {
        const int nen = orc_nnode(t), ng = orc_ngauss(t);
        for (int64_t e = 0; e < m->n_elem[t]; ++e) {
            const int32_t *c = m->conn[t] + e * nen;
            for (int a = 0; a < nen; ++a)
                for (int i = 0; i < 3; ++i) X[3 * a + i] = m->xyz[3 * (int64_t)c[a] + i];
            if (orc_element_geometry(t, X, N, dN, W, NULL) != 0) return -1;
            for (int g = 0; g < ng; ++g) {
                double gp[3] = {0.0, 0.0, 0.0};
                for (int b = 0; b < nen; ++b)
                    for (int i = 0; i < 3; ++i) gp[i] += p[c[b]] * dN[(g * nen + b) * 3 + i];
                for (int a = 0; a < nen; ++a)
                    for (int i = 0; i < 3; ++i) out[3 * (int64_t)c[a] + i] += W[g] * N[g * nen + a] * gp[i];
            }
        }
    }
    return 0;
}

/* Periodic fold of a nodal array with ncomp components per node:
 * every slave's value is added to its master, then copied back. */
void orc_periodic_fold(int64_t n, const int32_t *master, double *v, int ncomp) {
    for (int64_t i = 0; i < n; ++i)
        if (master[i] != i)
            for (int c = 0; c < ncomp; ++c) v[(int64_t)master[i] * ncomp + c] += v[i * ncomp + c];
    for (int64_t i = 0; i < n; ++i)
        if (master[i] != i)
            for (int c = 0; c < ncomp; ++c) v[i * ncomp + c] = v[(int64_t)master[i] * ncomp + c];
}

/* ---------------------------------------------------------------------- */
/* Equilibrium wall model: the boundary assembly of Algorithm 1 ("assembly of
 * the wall model", a law of the wall; the paper defers the formulation to a
 * reference that is absent here, so every item below is a reading).
 *   Law of the wall (Reichardt): u+ = f(y+) with
 *     f(y+) = ln(1 + kappa y+) / kappa + C (1 - exp(-y+/11) - (y+/11) exp(-y+/3)),
 *     kappa = 0.41, C = 7.8 by default.
 *   At every Gauss point of a wall face the velocity is sampled at an
 *   exchange location: the face's shape functions applied to the velocities
 *   and positions of each face node's exchange node (an interior node, e.g.
 *   the opposite node of the wall prism).  y = normal distance of that point
 *   from the wall, U = |tangential part of the sampled velocity|.
 *   u_tau > 0 solves U = u_tau f(y u_tau / nu) (Newton from the viscous-
 *   sublayer value sqrt(nu U / y)); the wall shear stress is u_tau^2 along
 *   the tangential velocity, against it on the fluid:
 *     R_a += - sum_g w_g |x_xi x x_eta| N_a(g) u_tau^2 t,  t = u_t / U.
 *   Faces: triangles (3-point degree-2 rule) and bilinear quads (2x2 Gauss);
 *   the node order makes (x_xi x x_eta) point out of the fluid.           */

/* Reichardt's f(y+) and, if df != NULL, its derivative. */
double orc_reichardt(double yp, double kappa, double c, double *df) {
    const double e11 = exp(-yp / 11.0), e3 = exp(-yp / 3.0);
    if (df) *df = 1.0 / (1.0 + kappa * yp) + c * (e11 / 11.0 - e3 / 11.0 + yp * e3 / 33.0);
    /* 1 - e^(-y+/11) as -expm1: deep in the sublayer the bracket is O(y+^2)
     * and 1 - exp() would leave it an absolute error of one ulp of 1 */
    return log1p(kappa * yp) / kappa + c * (-expm1(-yp / 11.0) - (yp / 11.0) * e3);
}

/* u_tau from U = u_tau f(y u_tau / nu): Newton on g(v) = v f(y v / nu) - U,
 * g'(v) = f + y+ f'; a step that would leave v <= 0 halves v instead.
 * Stops when |dv| <= 1e-14 v (returns 0) or after 100 steps (returns -5).
 * U = 0 gives u_tau = 0.                                                   */
int orc_wall_utau(double U, double y, double nu, double kappa, double c, double *utau, int *iters) {
    if (!(y > 0.0) || !(nu > 0.0) || !(U >= 0.0)) return -3;
    if (iters) *iters = 0;
    if (U == 0.0) {
        *utau = 0.0;
        return 0;
    }
    double v = sqrt(nu * U / y);
    for (int it = 1; it <= 100; ++it) {
        double df;
        const double yp = y * v / nu;
        const double f = orc_reichardt(yp, kappa, c, &df);
        const double g = v * f - U, dg = f + yp * df;
        double vn = v - g / dg;
        if (!(vn > 0.0)) vn = 0.5 * v;
        const double dv = fabs(vn - v);
        v = vn;
        if (iters) *iters = it;
        if (dv <= 1e-14 * v) {
            *utau = v;
            return 0;
        }
    }
    *utau = v;
    return -5;
}

/* Face rules: triangle points (1/6,1/6), (2/3,1/6), (1/6,2/3), weights 1/6;
 * quad 2x2 Gauss on [-1,1]^2, weights 1, node order (-1,-1) (1,-1) (1,1) (-1,1). */
static int face_rule(int nv, double pts[4][2], double w[4]) {
    if (nv == 3) {
        const double a = 1.0 / 6.0, b = 2.0 / 3.0;
        pts[0][0] = a; pts[0][1] = a;
        pts[1][0] = b; pts[1][1] = a;
        pts[2][0] = a; pts[2][1] = b;
        for (int g = 0; g < 3; ++g) w[g] = 1.0 / 6.0;
        return 3;
    }
    const double q = 1.0 / sqrt(3.0);
    const double sx[4] = {-q, q, q, -q}, sy[4] = {-q, -q, q, q};
    for (int g = 0; g < 4; ++g) {
        pts[g][0] = sx[g];
        pts[g][1] = sy[g];
        w[g] = 1.0;
    }
    return 4;
}

static void face_shape(int nv, const double *xi, double *N, double (*dN)[2]) {
    if (nv == 3) {
        N[0] = 1.0 - xi[0] - xi[1]; N[1] = xi[0]; N[2] = xi[1];
        dN[0][0] = -1.0; dN[0][1] = -1.0;
        dN[1][0] = 1.0;  dN[1][1] = 0.0;
        dN[2][0] = 0.0;  dN[2][1] = 1.0;
        return;
    }
    const double sx[4] = {-1, 1, 1, -1}, sy[4] = {-1, -1, 1, 1};
    for (int a = 0; a < 4; ++a) {
        N[a] = 0.25 * (1 + sx[a] * xi[0]) * (1 + sy[a] * xi[1]);
        dN[a][0] = 0.25 * sx[a] * (1 + sy[a] * xi[1]);
        dN[a][1] = 0.25 * sy[a] * (1 + sx[a] * xi[0]);
    }
}

/* Adds the wall-model boundary term of n_faces faces with nv (3 or 4) nodes
 * to rhs [n][3].  face, exch: [n_faces][nv] node ids.  Returns -3 for a
 * Gauss point whose exchange location is not on the fluid side (y <= 0) or
 * a degenerate face, -1 for a bad node id, -5 if Newton did not converge. */
int orc_wall_rhs(int64_t n, const double *xyz, const double *u, int nv, int64_t n_faces, const int32_t *face,
                 const int32_t *exch, double nu, double kappa, double c, double *rhs) {
    if (nv != 3 && nv != 4) return -2;
    double pts[4][2], w[4];
    const int ng = face_rule(nv, pts, w);
    for (int64_t f = 0; f < n_faces; ++f) {
        const int32_t *fa = face + f * nv, *ex = exch + f * nv;
        for (int a = 0; a < nv; ++a)
            if (fa[a] < 0 || fa[a] >= n || ex[a] < 0 || ex[a] >= n) return -1;
        for (int g = 0; g < ng; ++g) {
            double N[4], dN[4][2];
            face_shape(nv, pts[g], N, dN);
            double xg[3] = {0, 0, 0}, xs[3] = {0, 0, 0}, us[3] = {0, 0, 0}, t1[3] = {0, 0, 0}, t2[3] = {0, 0, 0};
            for (int a = 0; a < nv; ++a)
                for (int i = 0; i < 3; ++i) {
                    xg[i] += N[a] * xyz[3 * (int64_t)fa[a] + i];
                    xs[i] += N[a] * xyz[3 * (int64_t)ex[a] + i];
                    us[i] += N[a] * u[3 * (int64_t)ex[a] + i];
                    t1[i] += dN[a][0] * xyz[3 * (int64_t)fa[a] + i];
                    t2[i] += dN[a][1] * xyz[3 * (int64_t)fa[a] + i];
                }
            const double nr[3] = {t1[1] * t2[2] - t1[2] * t2[1], t1[2] * t2[0] - t1[0] * t2[2],
                                  t1[0] * t2[1] - t1[1] * t2[0]};
            const double area = sqrt(nr[0] * nr[0] + nr[1] * nr[1] + nr[2] * nr[2]);
            if (!(area > 0.0)) return -3;
            const double nh[3] = {nr[0] / area, nr[1] / area, nr[2] / area};   /* out of the fluid */
            const double y = -((xs[0] - xg[0]) * nh[0] + (xs[1] - xg[1]) * nh[1] + (xs[2] - xg[2]) * nh[2]);
            if (!(y > 0.0)) return -3;
            const double un = us[0] * nh[0] + us[1] * nh[1] + us[2] * nh[2];
            const double ut[3] = {us[0] - un * nh[0], us[1] - un * nh[1], us[2] - un * nh[2]};
            const double U = sqrt(ut[0] * ut[0] + ut[1] * ut[1] + ut[2] * ut[2]);
            if (U == 0.0) continue;
            double ut_;
            const int st = orc_wall_utau(U, y, nu, kappa, c, &ut_, NULL);
            if (st) return st;
            const double s = -w[g] * area * ut_ * ut_ / U;
            for (int a = 0; a < nv; ++a)
                for (int i = 0; i < 3; ++i) rhs[3 * (int64_t)fa[a] + i] += s * N[a] * ut[i];
        }
    }
    return 0;
}

/* One stage of the three-stage SSP Runge-Kutta momentum update (Shu-Osher):
 *   u^(k+1) = a_k u^n + b_k (u^(k) + dt M^-1 R(u^(k), p^n)),
 *   (a, b) = (0, 1), (3/4, 1/4), (1/3, 2/3);
 * R is folded over periodic pairs, M is the folded lumped mass, and nodes
 * with dirichlet != 0 keep u^n.  rhs_extra (optional, [n][3]) is added to
 * the element RHS before the fold (the boundary assembly of Algorithm 1,
 * evaluated by the caller at u^(k)).  uk_out may alias uk.                  */
int orc_rk_stage(const orc_mesh *m, const int32_t *master, const uint8_t *dirichlet, const double *mass_folded,
                 const double *un, const double *uk, const double *p, const orc_params *prm, int stage, double dt,
                 const double *rhs_extra, double *uk_out) {
    static const double A[3] = {0.0, 0.75, 1.0 / 3.0};
    static const double Bc[3] = {1.0, 0.25, 2.0 / 3.0};
    if (stage < 0 || stage > 2) return -2;
    const int64_t n = m->n_nodes;
    double *R = (double *)malloc(sizeof(double) * 3 * n);
    if (!R) return -4;
    int st = orc_assemble_rhs(m, uk, p, prm, R, NULL, NULL);
    if (st) {
        free(R);
        return st;
    }
    if (rhs_extra)
        for (int64_t k = 0; k < 3 * n; ++k) R[k] += rhs_extra[k];
    if (master) orc_periodic_fold(n, master, R, 3);
    for (int64_t i = 0; i < n; ++i)
        for (int c = 0; c < 3; ++c) {
            const int64_t k = 3 * i + c;
            if (dirichlet && dirichlet[i])
                uk_out[k] = un[k];
            else
                uk_out[k] = A[stage] * un[k] + Bc[stage] * (uk[k] + dt * R[k] / mass_folded[i]);
        }
    free(R);
    return 0;
}

/* ---------------------------------------------------------------------- */
/* MLP training pieces (FP64): loss and gradient by reverse-mode chain rule,
 * and one Adam step.  Parameter vector layout (8,833 values):
 *   w1[64][6] b1[64] w2[64][64] b2[64] w3[64][64] b3[64] w4[64] b4[1].
 * Inputs x are already normalised; target y and prediction are in units of
 * out_scale (pred = softplus(z)).  loss = mean_b (pred_b - y_b)^2.         */
#define MLP_NPARAM (MLP_H * MLP_IN + MLP_H + 2 * (MLP_H * MLP_H + MLP_H) + MLP_H + 1)

int orc_mlp_nparam(void) { return MLP_NPARAM; }

static double sigm(double z) { return 1.0 / (1.0 + exp(-z)); }

double orc_mlp_loss_grad(const double *theta, const double *x /*[B][6]*/, const double *y, int64_t B,
                         double *grad /*[NPARAM] or NULL*/) {
    const double *w1 = theta, *b1 = w1 + MLP_H * MLP_IN;
    const double *w2 = b1 + MLP_H, *b2 = w2 + MLP_H * MLP_H;
    const double *w3 = b2 + MLP_H, *b3 = w3 + MLP_H * MLP_H;
    const double *w4 = b3 + MLP_H, *b4 = w4 + MLP_H;
    double *gw1 = grad, *gb1 = grad ? gw1 + MLP_H * MLP_IN : NULL;
    double *gw2 = grad ? gb1 + MLP_H : NULL, *gb2 = grad ? gw2 + MLP_H * MLP_H : NULL;
    double *gw3 = grad ? gb2 + MLP_H : NULL, *gb3 = grad ? gw3 + MLP_H * MLP_H : NULL;
    double *gw4 = grad ? gb3 + MLP_H : NULL, *gb4 = grad ? gw4 + MLP_H : NULL;
    if (grad) memset(grad, 0, sizeof(double) * MLP_NPARAM);
    double loss = 0.0;
    for (int64_t b = 0; b < B; ++b) {
        const double *in = x + b * MLP_IN;
        double z1[MLP_H], h1[MLP_H], z2[MLP_H], h2[MLP_H], z3[MLP_H], h3[MLP_H];
        for (int o = 0; o < MLP_H; ++o) {
            double s = b1[o];
            for (int k = 0; k < MLP_IN; ++k) s += w1[o * MLP_IN + k] * in[k];
            z1[o] = s; h1[o] = silu(s);
        }
        for (int o = 0; o < MLP_H; ++o) {
            double s = b2[o];
            for (int k = 0; k < MLP_H; ++k) s += w2[o * MLP_H + k] * h1[k];
            z2[o] = s; h2[o] = silu(s);
        }
        for (int o = 0; o < MLP_H; ++o) {
            double s = b3[o];
            for (int k = 0; k < MLP_H; ++k) s += w3[o * MLP_H + k] * h2[k];
            z3[o] = s; h3[o] = silu(s);
        }
        double z4 = b4[0];
        for (int k = 0; k < MLP_H; ++k) z4 += w4[k] * h3[k];
        const double pred = softplus(z4);
        const double diff = pred - y[b];
        loss += diff * diff;
        if (!grad) continue;
        /* d loss_b / d z4 = 2 diff / B * softplus'(z4) */
        const double dz4 = 2.0 * diff / (double)B * sigm(z4);
        double dh3[MLP_H], dz3[MLP_H], dh2[MLP_H], dz2[MLP_H], dh1[MLP_H], dz1[MLP_H];
        gb4[0] += dz4;
        for (int k = 0; k < MLP_H; ++k) {
            gw4[k] += dz4 * h3[k];
            dh3[k] = dz4 * w4[k];
        }
        /* silu'(z) = s(z) (1 + z (1 - s(z))) */
        for (int o = 0; o < MLP_H; ++o) {
            const double s = sigm(z3[o]);
            dz3[o] = dh3[o] * s * (1.0 + z3[o] * (1.0 - s));
        }
        for (int k = 0; k < MLP_H; ++k) dh2[k] = 0.0;
        for (int o = 0; o < MLP_H; ++o) {
            gb3[o] += dz3[o];
            for (int k = 0; k < MLP_H; ++k) {
                gw3[o * MLP_H + k] += dz3[o] * h2[k];
                dh2[k] += dz3[o] * w3[o * MLP_H + k];
            }
        }
        for (int o = 0; o < MLP_H; ++o) {
            const double s = sigm(z2[o]);
            dz2[o] = dh2[o] * s * (1.0 + z2[o] * (1.0 - s));
        }
        for (int k = 0; k < MLP_H; ++k) dh1[k] = 0.0;
        for (int o = 0; o < MLP_H; ++o) {
            gb2[o] += dz2[o];
            for (int k = 0; k < MLP_H; ++k) {
                gw2[o * MLP_H + k] += dz2[o] * h1[k];
                dh1[k] += dz2[o] * w2[o * MLP_H + k];
            }
        }
        for (int o = 0; o < MLP_H; ++o) {
            const double s = sigm(z1[o]);
            dz1[o] = dh1[o] * s * (1.0 + z1[o] * (1.0 - s));
        }
        for (int o = 0; o < MLP_H; ++o) {
            gb1[o] += dz1[o];
            for (int k = 0; k < MLP_IN; ++k) gw1[o * MLP_IN + k] += dz1[o] * in[k];
        }
    }
    return loss / (double)B;
}

/* One Adam step (Kingma & Ba 2015) with bias correction; step counter t >= 1. */
void orc_adam_step(double *theta, const double *grad, double *m1, double *m2, int64_t n, double lr, double beta1,
                   double beta2, double eps, int64_t t) {
    const double c1 = 1.0 - pow(beta1, (double)t), c2 = 1.0 - pow(beta2, (double)t);
    for (int64_t k = 0; k < n; ++k) {
        m1[k] = beta1 * m1[k] + (1.0 - beta1) * grad[k];
        m2[k] = beta2 * m2[k] + (1.0 - beta2) * grad[k] * grad[k];
        theta[k] -= lr * (m1[k] / c1) / (sqrt(m2[k] / c2) + eps);
    }
}
