/*
 * fea.h -- C ABI of the B300 (sm_103a) momentum right-hand-side assembly.
 *
 * The operation is the element assembly of the explicit momentum equation of
 * Borrell et al., "Heterogeneous CPU/GPU co-execution of CFD simulations on
 * the POWER9 architecture" (FGCS 2020):
 *   - the filtered incompressible momentum equation of section 2.1
 *     (Eq. momentum) with rho = 1, mu = nu, the EMAC-form convective bracket
 *     evaluated pointwise on the finite-element interpolant, the Vreman
 *     subgrid viscosity (section 2.1) and Galerkin linear elements;
 *   - assembled element by element with the three steps gather ->
 *     computation -> scatter of section 2.3.3 ("Element and boundary
 *     assemblies"), over categories of same element type and integration
 *     rule (section 2.3.3);
 *   - advanced by the three Runge-Kutta stages of Algorithm 1 (element
 *     assembly, momentum update), here with the SSP-RK3 coefficients and a
 *     frozen pressure.
 *
 * For node a and component i the assembled right-hand side is
 *   R_a,i = - sum_e sum_g W_g [ N_a (c_i + d_i p) + 2 (nu + nu_t) eps_ij d_j N_a ]
 * with W_g = w_g det J, G_ij = du_i/dx_j, eps = (G + G^T)/2,
 * c = G u + (tr G) u, and nu_t from the closure.
 *
 * Conventions (every entry point):
 *   - All work is asynchronous on the caller's CUDA stream (cudaStream_t
 *     passed as void*, NULL = legacy default stream).  Errors that the host
 *     can detect are returned at once; errors detected on the device
 *     (det J <= 0, a non-finite residual, a bounded wait that gave up) set a
 *     device error word that fea_sync_status() reads and clears.
 *   - Node arrays are structure-of-arrays in the caller's node order:
 *     a vector field is [3][n_nodes] (all x, then all y, then all z).
 *     The library never reorders the caller's nodes; it reorders its own
 *     copy of the elements (type buckets sorted along a Morton curve).
 *   - Pointers marked "host or device" may point to either (CUDA unified
 *     addressing decides); "device" means device memory the caller owns
 *     (e.g. a torch tensor) and that must stay valid until the stream work
 *     that uses it has finished.
 *   - No exception or abort crosses this interface; every function returns
 *     a fea_status.  fea_last_error() gives a message for the last failure
 *     on that context.
 *   - Local node order per element type is the VTK one:
 *       TET04 (r,s,t) corners 0,(1,0,0),(0,1,0),(0,0,1);
 *       PYR05 base (-1,-1),(1,-1),(1,1),(-1,1) at zeta=0, apex zeta=1;
 *       PEN06 bottom triangle (zeta=-1) then top triangle (zeta=+1);
 *       HEX08 bottom face then top face, counter-clockwise.
 *   - Integration rules (one per type; a category is type + rule):
 *       TET04 4-point degree-2 rule, PYR05 8-point collapsed rule
 *       (2x2 Gauss-Legendre x 2-point Gauss-Jacobi(2,0)), PEN06 3-point
 *       triangle x 2-point Gauss, HEX08 2x2x2 Gauss.
 */
#ifndef FEA_H
#define FEA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    FEA_OK = 0,
    FEA_EINVAL = 1,    /* bad argument (null pointer, size, enum value) */
    FEA_ENOMEM = 2,    /* a device or host allocation failed */
    FEA_ECUDA = 3,     /* a CUDA runtime call failed (message has the CUDA error) */
    FEA_EMESH = 4,     /* connectivity index out of range, or det J <= 0 */
    FEA_ENUMERIC = 5,  /* a non-finite value in a residual */
    FEA_ETIMEOUT = 6,  /* a bounded device-side wait gave up */
    FEA_ESTATE = 7,    /* call out of order (e.g. assemble before field upload) */
    FEA_ENOTFOUND = 8  /* unknown mesh id */
} fea_status;

typedef enum { FEA_TET04 = 0, FEA_PYR05 = 1, FEA_PEN06 = 2, FEA_HEX08 = 3 } fea_etype;

typedef enum {
    FEA_FP64 = 0,   /* every operation in FP64 */
    FEA_MIXED = 1   /* FP32 element arithmetic; FP64 Jacobian determinant and
                       inverse for elements flagged fp64_jac; FP64 nodal sums */
} fea_prec;

typedef enum { FEA_CLOSURE_NONE = 0, FEA_CLOSURE_VREMAN = 1, FEA_CLOSURE_MLP = 2 } fea_closure;

/* term mask: which parts of the bracket above are assembled */
enum { FEA_TERM_CONV = 1, FEA_TERM_VISC = 2, FEA_TERM_SGS = 4, FEA_TERM_PRES = 8, FEA_TERM_ALL = 15 };

/* scatter strategy of the element residuals into the nodal RHS */
typedef enum {
    FEA_SCATTER_AUTO = 0,   /* the mesh's current plan (autotuned or default) */
    FEA_SCATTER_ATOMIC = 1, /* one FP64 atomic add per element node and component */
    FEA_SCATTER_CHUNK = 2,  /* CTA-local assembly of a chunk of elements in
                               shared memory; FP64 atomics only for nodes the
                               chunk shares with other chunks */
    FEA_SCATTER_COLOUR = 3, /* greedy element colouring per category (no two
                               elements of a colour share a node), one launch
                               per colour, plain FP64 read-modify-write: the sum
                               order is fixed, results are bitwise reproducible */
    FEA_SCATTER_WARP = 4    /* FP64 atomics after a warp-level sum of the lanes
                               whose element has the same node in the same local
                               slot (match_any): fewer atomics on shared nodes */
} fea_scatter;

/* convective form (section 2.1 writes the EMAC bracket; see fea_set_model) */
typedef enum {
    FEA_CONV_GU = 0,    /* c = G u + (tr G) u: the bracket evaluated pointwise on the interpolant */
    FEA_CONV_EMAC = 1   /* c = 2 eps u + (tr G) u - 1/2 grad (|u|^2)_h, (|u|^2)_h = sum_a N_a |u_a|^2 */
} fea_conv_form;

/* filter width of the Vreman closure */
typedef enum {
    FEA_DELTA_VOLUME = 0,   /* Delta = V_e^(1/3) */
    FEA_DELTA_AXES = 1      /* a width per direction: the element's extents along the axes */
} fea_delta_form;

typedef struct fea_ctx fea_ctx;

/* Mesh description for fea_mesh_upload.  All pointers: HOST memory, read
 * during the call only (the library keeps its own device copies). */
typedef struct {
    int64_t n_nodes;
    const double *xyz;                  /* [3][n_nodes] coordinates */
    int64_t n_elem[4];                  /* elements per fea_etype */
    const int32_t *conn[4];             /* [n_elem[t]][n_en(t)], 0-based node ids; NULL if n_elem[t]==0 */
    const int32_t *periodic_master;     /* optional [n_nodes]: master node id, or the node itself */
    const uint8_t *dirichlet;           /* optional [n_nodes]: 1 = velocity held (RK stages) */
    const uint8_t *fp64_jac[4];         /* optional [n_elem[t]]: 1 = FP64 Jacobian in FEA_MIXED
                                           (stretched boundary-layer elements) */
} fea_mesh_desc;

/* Launch plan of one mesh (chosen by fea_autotune or set by hand). */
typedef struct {
    int32_t scatter;            /* fea_scatter (not AUTO); under FEA_FP64 a CHUNK plan
                                   runs ATOMIC (COLOUR and WARP apply to both) */
    int32_t threads_per_block;  /* element kernels: multiple of 32 in [32, 1024] (capped at 256);
                                   the TET04 chunk kernel (FEA_MIXED) takes from it its
                                   compute warps: 12 from 384 threads, 8 from 256, else 4;
                                   with the MLP closure the element kernels run one
                                   warpgroup (128 threads) per CTA whatever this says */
    int32_t chunk_elems;        /* elements per chunk for FEA_SCATTER_CHUNK: multiple of 32 in [32, 4096]
                                   (the TET04 chunk kernel uses 64 per compute warp) */
    int32_t chunk_acc;          /* FEA_SCATTER_CHUNK nodal sums inside a chunk: 0 = FP32,
                                   1 = compensated two-float sums (about 48 significant bits);
                                   sums across chunks are FP64 atomics in both cases */
} fea_plan;

/* ---- context ------------------------------------------------------------ */

/* Creates a context on CUDA device `device` (made current for the calls on
 * this context).  *out receives the handle.  Returns FEA_ECUDA when no device
 * is usable. */
fea_status fea_create(int device, fea_ctx **out);

/* Frees every device buffer the context owns.  NULL is allowed. */
void fea_destroy(fea_ctx *ctx);

/* Message of the last failure on this context (never NULL; owned by ctx,
 * valid until the next call on ctx). */
const char *fea_last_error(const fea_ctx *ctx);

/* Library version string (static storage). */
const char *fea_version(void);

/* ---- mesh and fields ---------------------------------------------------- */

/* Mesh upload (the "mesh arrays" and category packing of section 2.3.3):
 * validates indices, buckets elements by (type, FP64-Jacobian flag), sorts
 * each bucket along a Morton curve of element centroids, builds chunk tables
 * for the CTA-local scatter, copies coordinates (FP64 and FP32) and computes
 * the lumped mass (section 2.3.3 mass-matrix listing, row sums).
 * Synchronous with respect to the host (returns when the copies are done).
 * *mesh_id receives the id.  Errors: FEA_EINVAL, FEA_EMESH (index out of
 * range or det J <= 0 at a Gauss point; the message names the element),
 * FEA_ENOMEM, FEA_ECUDA. */
fea_status fea_mesh_upload(fea_ctx *ctx, const fea_mesh_desc *desc, void *stream, int32_t *mesh_id);

/* Mesh sizes: n_nodes, and elements per type (n_elem may be NULL). */
fea_status fea_mesh_info(fea_ctx *ctx, int32_t mesh, int64_t *n_nodes, int64_t n_elem[4]);

/* Lumped mass M_a = sum_e sum_g W_g N_a(g) into out [n_nodes] (device),
 * NOT folded over periodic pairs. */
fea_status fea_lumped_mass(fea_ctx *ctx, int32_t mesh, double *out, void *stream);

/* Field upload: nodal velocity u [3][n_nodes] and pressure p [n_nodes],
 * host or device, dtype 0 = float64, 1 = float32.  Also (re)starts the RK
 * state: u^n = u^(0) = u.  nu: kinematic viscosity; c_vreman: Vreman
 * constant.  Asynchronous; host sources are staged through the library. */
fea_status fea_field_upload(fea_ctx *ctx, int32_t mesh, const void *u, const void *p, int dtype, double nu,
                            double c_vreman, void *stream);

/* ---- the hot path -------------------------------------------------------- */

/* Element assembly of the momentum RHS (Eq. momentum, section 2.3.3) from
 * the uploaded field.  rhs_out [3][n_nodes] (device) is overwritten (not
 * accumulated) in the caller's node order, NOT folded over periodic pairs.
 * nut_out (optional, device): nu_t at every Gauss point, types concatenated
 * in fea_etype order, caller element order within a type, n_gauss(t) values
 * per element (4, 8, 6, 8).  scatter: FEA_SCATTER_AUTO uses the mesh plan. */
fea_status fea_assemble_rhs(fea_ctx *ctx, int32_t mesh, fea_prec prec, fea_closure closure, uint32_t term_mask,
                            fea_scatter scatter, double *rhs_out, float *nut_out, void *stream);

/* Batched form: one persistent launch over the (mesh, category, chunk) work
 * items of n meshes (each with its own field, nu and c_vreman); CTAs pull
 * items from a device work counter, most expensive categories first.  One
 * zeroing launch for all RHS arrays precedes it.  meshes [n] (host); rhs_out
 * [n] (host array of device pointers, each [3][n_nodes(mesh)]), overwritten.
 * The same precision/closure/mask apply to all meshes.  FEA_FP64 (or a mesh
 * without chunk tables) falls back to per-mesh launches.  The descriptor
 * tables live in the context: do not overlap batched calls of one context
 * on different streams. */
fea_status fea_assemble_rhs_batched(fea_ctx *ctx, const int32_t *meshes, int32_t n, fea_prec prec,
                                    fea_closure closure, uint32_t term_mask, double *const *rhs_out,
                                    void *stream);

/* Autotuner of the batched form for these meshes (their fields uploaded):
 * times the persistent launch over chunk tables of 128, 256 and 512 elements
 * (FEA_MIXED) against per-mesh launches with the ATOMIC, WARP and COLOUR
 * scatters, and keeps the fastest: every mesh's plan is set to it, and
 * fea_assemble_rhs_batched of this context then uses the persistent launch
 * (best_out->scatter == FEA_SCATTER_CHUNK) or per-mesh launches (otherwise).
 * Synchronises the device; overwrites the meshes' library-owned RHS
 * buffers.  best_out may be NULL. */
fea_status fea_autotune_batched(fea_ctx *ctx, const int32_t *meshes, int32_t n, fea_prec prec, fea_closure closure,
                                fea_plan *best_out);

/* In-place periodic fold of v [ncomp][n_nodes] (device): every slave's value
 * is added to its master, then copied back to the slave.  No-op without a
 * periodic map. */
fea_status fea_periodic_fold(fea_ctx *ctx, int32_t mesh, double *v, int32_t ncomp, void *stream);

/* One SSP-RK3 momentum-update stage (Algorithm 1, stage index 0..2) on the
 * library-owned state:  u^(k+1) = a_k u^n + b_k (u^(k) + dt M^-1 R(u^(k))),
 * (a, b) = (0, 1), (3/4, 1/4), (1/3, 2/3); R folded, M the folded lumped
 * mass, Dirichlet nodes hold u^n, pressure frozen at the uploaded p.  R
 * includes the wall-model term when the mesh has wall faces
 * (fea_wall_setup).  Stage 2 also makes the result the new u^n. */
fea_status fea_rk_stage(fea_ctx *ctx, int32_t mesh, int32_t stage, double dt, fea_prec prec, fea_closure closure,
                        void *stream);

/* A full three-stage step replayed from a CUDA graph (captured on first use
 * for this (mesh, dt, prec, closure) and replayed afterwards). */
fea_status fea_rk_step_graph(fea_ctx *ctx, int32_t mesh, double dt, fea_prec prec, fea_closure closure,
                             void *stream);

/* Copies the current state u^(k) [3][n_nodes] to out (host or device). */
fea_status fea_state_download(fea_ctx *ctx, int32_t mesh, double *out, void *stream);

/* ---- learned closure --------------------------------------------------
 * A small network that stands in for the Vreman closure of section 2.1 (the
 * paper has no learned model): 6 -> 64 -> 64 -> 64 -> 1, SiLU hidden layers,
 * softplus output.  Inputs per Gauss point (per element for TET04), all
 * dimensionless: with G the velocity gradient, S = (G+G^T)/2, O = (G-G^T)/2
 * and g = |G| (Frobenius),
 *   x_1..5 = (tr S^2, tr O^2, tr S^3, tr S O^2, tr S^2 O^2) / g^(2, 2, 3, 3, 4),
 *   x_6 = log(Delta^2 g / nu)  (Delta = V_e^(1/3)),
 * normalised as (x - mean) / std; the network gives the coefficient
 * C = out_scale * softplus(z) and nu_t = C Delta^2 g (zero where g = 0).
 * Parameter vector theta (FP32, 8,833):
 *   w1[64][6] b1[64] w2[64][64] b2[64] w3[64][64] b3[64] w4[64] b4[1].
 * Training evaluates BF16 weights and activations with FP32 accumulation on
 * warp-level tensor-core tiles and updates the FP32 master copy by Adam.
 * Inference (fea_mlp_forward and the fused closure) runs on the tcgen05
 * tensor cores over 128-row tiles: the same BF16 weight values held as FP16
 * operands, FP16 activations and hidden-layer accumulators, an FP32 output
 * layer with the output weights to about 2^-19; normalised features are
 * clamped to +-64.  With an envelope set (fea_mlp_set_envelope), a Gauss
 * point whose features or element size lie outside it takes Vreman's nu_t
 * instead (section 2.1), so the plain closure is the network's fallback.
 * The kernels that evaluate the network run persistent CTAs of 128 threads,
 * two per SM, each holding 256 tensor-memory columns for its lifetime; a
 * kernel that allocates tensor memory on the same SMs at the same time
 * waits for those columns. */

/* Loads theta, the feature mean and std [6] (host or device) and out_scale;
 * resets the Adam state.  Errors: FEA_EINVAL (null, std <= 0, scale <= 0). */
fea_status fea_mlp_load(fea_ctx *ctx, const float *theta, const float *feat_mean, const float *feat_std,
                        double out_scale, void *stream);

/* Training envelope of the fused closure: raw-feature bounds lo [6], hi [6]
 * (host).  A Gauss point uses the network only if each of its six raw
 * features (the five invariant ratios and log(Delta^2 g / nu)) lies in
 * [lo_k, hi_k];
 * otherwise it uses Vreman's nu_t (c_vreman of the mesh's field), and the
 * point is counted (fea_mlp_fallback_read).  lo = hi = NULL removes the
 * envelope; fea_mlp_load also removes it.  Synchronises the stream.
 * Errors: FEA_ESTATE (no network loaded), FEA_EINVAL (one bound NULL, NaN). */
fea_status fea_mlp_set_envelope(fea_ctx *ctx, const float *lo, const float *hi, void *stream);

/* Number of Gauss-point evaluations of the MLP closure that fell back to
 * Vreman since the network was loaded or the last reset (reset != 0 zeroes
 * the count after reading).  Synchronises the device. */
fea_status fea_mlp_fallback_read(fea_ctx *ctx, int64_t *points, int reset);

/* Copies the current FP32 parameters to theta_out [8833] (host or device). */
fea_status fea_mlp_get(fea_ctx *ctx, float *theta_out, void *stream);

/* The network's coefficient C = out_scale * softplus(z) (nu_t / (Delta^2 g))
 * for B rows of raw features x [B][6] (device) into nut [B] (device), on
 * the tensor-core tiles of the fused closure; B = 0 is a no-op (x and nut
 * may then be NULL). */
fea_status fea_mlp_forward(fea_ctx *ctx, const float *x, int64_t B, float *nut, void *stream);

/* One training step on B samples: raw features x [B][6] and targets y [B]
 * in units of out_scale (device); loss = mean (softplus(z) - y)^2.  The
 * forward and backward GEMMs run on the tensor cores, then Adam (lr,
 * beta = 0.9, 0.999, eps = 1e-8) updates theta.  loss_out (optional, host or
 * device, 1 float) receives the loss before the update; grad_out (optional,
 * host or device, [8833]) the gradient d loss / d theta. */
fea_status fea_mlp_train_step(fea_ctx *ctx, const float *x, const float *y, int64_t B, float lr, float *loss_out,
                              float *grad_out, void *stream);

/* Model variants of a mesh's assembly (default FEA_CONV_GU, FEA_DELTA_VOLUME).
 * FEA_CONV_EMAC: the convective term with the kinetic-energy gradient taken
 * from the interpolated nodal |u|^2, which differs from the pointwise form by
 * G^T u - 1/2 grad (|u|^2)_h.  FEA_DELTA_AXES: Vreman's beta_ij =
 * sum_m Delta_m^2 alpha_mi alpha_mj with Delta_m the element's extent along
 * axis m (the model as written for anisotropic grids).  The fused TET04
 * pipeline serves the defaults; other forms run in the generic kernels.
 * Drops a captured RK graph of the mesh.  Errors: FEA_EINVAL. */
fea_status fea_set_model(fea_ctx *ctx, int32_t mesh, int32_t conv_form, int32_t delta_form);

/* ---- boundary assembly: equilibrium wall model (Algorithm 1) -------------
 * Algorithm 1's "boundary assembly" applies a law of the wall on the wall
 * faces (section 2.1 and the test-case section: an equilibrium wall model on
 * the aircraft walls; the formulation itself is in a reference the paper
 * cites, so the one here is a reading):
 *   u+ = f(y+) = ln(1 + kappa y+)/kappa + C (1 - e^(-y+/11) - (y+/11) e^(-y+/3))
 * (Reichardt).  At each Gauss point of a wall face (triangles: 3-point
 * rule; bilinear quadrilaterals: 2x2 Gauss) the velocity and position are
 * interpolated from the face nodes' exchange nodes; y = normal distance of
 * that point from the face, U = |tangential velocity|; u_tau solves
 * U = u_tau f(y u_tau / nu) (Newton); the RHS receives the wall shear stress
 * as a traction against the tangential velocity:
 *   R_a += - sum_g w_g |x_xi x x_eta| N_a u_tau^2 u_t / U.
 * Geometry, traction and sums in FP64; u_tau to FP64 accuracy under FEA_FP64
 * (and in fea_wall_assemble), its FP32 Newton root under FEA_MIXED.  The
 * term joins R in every fea_rk_stage / fea_rk_step_graph / noalloc stage of
 * the mesh (added before the periodic fold). */
typedef struct {
    int64_t n_tri;              /* triangular wall faces */
    const int32_t *tri;         /* host [n_tri][3] node ids, ordered so that
                                   (x1 - x0) x (x2 - x0) points out of the fluid */
    const int32_t *tri_exch;    /* host [n_tri][3] exchange node of each face node */
    int64_t n_quad;             /* bilinear quadrilateral wall faces */
    const int32_t *quad;        /* host [n_quad][4], counter-clockwise seen from
                                   outside the fluid: (x1 - x0) x (x3 - x0) points out */
    const int32_t *quad_exch;   /* host [n_quad][4] */
    double kappa;               /* von Karman constant (0.41) */
    double c_plus;              /* C of the law above (7.8) */
} fea_wall_desc;

/* Sets (or, with n_tri = n_quad = 0, clears) the wall faces of a mesh.  The
 * arrays are copied.  Checks every index and, on the host in FP64, that every
 * face Gauss point has a positive face area and its exchange point strictly
 * on the fluid side (FEA_EMESH otherwise).  kappa > 0 and c_plus >= 0, else
 * FEA_EINVAL.  Drops a captured RK graph of the mesh. */
fea_status fea_wall_setup(fea_ctx *ctx, int32_t mesh, const fea_wall_desc *desc);

/* Adds the wall-model term at the uploaded field (current u^(k)) to rhs
 * [3][n_nodes] (device, not folded).  A Newton iteration that does not
 * converge in 100 steps is reported by fea_sync_status (FEA_ENUMERIC).
 * FEA_ESTATE without a field; a mesh without wall faces adds nothing. */
fea_status fea_wall_assemble(fea_ctx *ctx, int32_t mesh, double *rhs, void *stream);

/* ---- pressure projection (Algorithm 1) -----------------------------------
 * Algorithm 1 assembles the Laplacian matrix once, and each time step ends
 * with the solution of the pressure equation by CG with Jacobi diagonal
 * scaling (section 2.1).  Forms (FP64, W_g = w_g det J):
 *   K_ab = sum_e sum_g W_g grad N_a . grad N_b,
 *   B_a(u) = sum_e sum_g W_g N_a (div u)_g,   G_a(p) = sum_e sum_g W_g N_a (grad p)_g.
 * The pressure unknowns are periodic classes (a node and its periodic
 * copies); pinned classes hold 0 (their rows and columns become identity),
 * which fixes the constant of the pure-Neumann / periodic problem. */

/* Builds the CSR matrix of K over periodic classes (pattern on the host,
 * values by the element kernels) and its Jacobi diagonal.  pinned: optional
 * host [n_nodes], nonzero = the node's class is pinned; NULL pins the class
 * of node 0.  Synchronous.  Errors: FEA_EMESH (det J <= 0, a missing CSR
 * entry), FEA_ENOMEM. */
fea_status fea_poisson_setup(fea_ctx *ctx, int32_t mesh, const uint8_t *pinned, void *stream);

/* Solves K x = scale * fold(b) by Jacobi-preconditioned CG: b [n_nodes]
 * (device) is summed over the copies of each class; x [n_nodes] (device) is
 * the initial guess (its masters' values) and receives the solution at
 * every copy (0 at pinned classes).  Stops when ||r|| <= rtol ||b|| or after
 * max_iter iterations; *iters and *rel_res (optional) receive the count and
 * ||r|| / ||b||.  Synchronises the stream.  Errors: FEA_ESTATE (no setup),
 * FEA_EINVAL. */
fea_status fea_poisson_solve(fea_ctx *ctx, int32_t mesh, const double *b, double scale, double *x, double rtol,
                             int32_t max_iter, int32_t *iters, double *rel_res, void *stream);

/* out [n_nodes] = B(u) for u [3][n_nodes] (device, not folded).  Async. */
fea_status fea_divergence(fea_ctx *ctx, int32_t mesh, const double *u, double *out, void *stream);

/* out [3][n_nodes] = G(p) for p [n_nodes] (device, not folded).  Async. */
fea_status fea_gradient(fea_ctx *ctx, int32_t mesh, const double *p, double *out, void *stream);

/* Projection step on the mesh's state after the Runge-Kutta stages
 * (incremental form): K dp = -(1/dt) fold(B(u)), then u <- u - dt M^-1
 * fold(G(dp)) on nodes without velocity Dirichlet (M: folded lumped mass),
 * p <- p + dp; the FP32 copy of the field is refreshed.  rtol, max_iter,
 * iters, rel_res as in fea_poisson_solve.  Synchronises the stream.
 * Errors: FEA_ESTATE (no field or no fea_poisson_setup), FEA_EINVAL. */
fea_status fea_project(fea_ctx *ctx, int32_t mesh, double dt, double rtol, int32_t max_iter, int32_t *iters,
                       double *rel_res, void *stream);

/* ---- a mesh partitioned over several devices ----------------------------
 * Section 5: the mesh is split along a space-filling curve into parts of
 * (nearly) equal cost; each device assembles its part; after the assembly
 * the contributions at nodes shared by parts are summed (the per-stage
 * exchange of section 2.3.1).  A "class" is a set of node copies that must
 * end with one value: a node shared by parts together with its periodic
 * copies, so that the periodic fold across parts is the same sum. */

/* Space-filling-curve order of n points xyz [3][n] (host): the points are
 * binned on a regular grid of 2^level cells per axis over their bounding box
 * and ordered along a Hilbert curve through the cells; points of one cell
 * keep their input order.  order [n] (host) receives the permutation.
 * level in [1, 21].  Host only (no device call, no context).
 * Errors: FEA_EINVAL. */
fea_status fea_sfc_order(int64_t n, const double *xyz, int32_t level, int64_t *order);

/* Greedy element colouring, the one FEA_SCATTER_COLOUR uses (host only, no
 * device): elements in the given order take the lowest colour that none of
 * their nodes has seen yet, so no two elements of one colour share a node.
 * conn: host [count][n_en] node ids in [0, n_nodes); colour: host [count]
 * output; *n_colours: the number of colours used.  Errors: FEA_EINVAL,
 * FEA_EMESH (a node id out of range), FEA_ENUMERIC (more than 256 colours
 * would be needed). */
fea_status fea_colour_elements(int64_t n_nodes, int32_t n_en, int64_t count, const int32_t *conn, int32_t *colour,
                               int32_t *n_colours);

/* SFC partition of a mesh's elements into nparts parts (section 5, the
 * partitioner's steps): element location = centroid, weight = Gauss points
 * of the element's rule (TET04 4, PYR05 8, PEN06 6, HEX08 8), bins of a
 * 2^level grid ordered along the Hilbert curve, the weighted 1-D sequence
 * cut into nparts contiguous runs; each bin goes to the part whose target
 * interval holds the midpoint of its weight interval.  Targets: part p gets
 * lambda[p] / sum(lambda) of the total weight (the correction coefficients
 * of the load-balancing section; NULL: equal shares).  part[t] [n_elem[t]]
 * (host) receives part ids in [0, nparts).  Host only.
 * Errors: FEA_EINVAL (nparts < 1, level out of [1, 21], NULL arrays, a
 * negative or all-zero lambda), FEA_EMESH (node index out of range). */
fea_status fea_partition_sfc(const fea_mesh_desc *desc, int32_t nparts, int32_t level, const double *lambda,
                             int32_t *const part[4]);

/* Correction coefficients of the partition from measured times (the
 * load-balancing section): observations k = 0..n_obs-1 of the cumulative
 * coefficients Lambda [n_obs][nparts+1] (Lambda_0 = 0, Lambda_P = P) and of
 * the per-part times times [n_obs][nparts]; for every splitting point i, a
 * weighted linear regression (weight 1.5^k, plus the origin with weight 1)
 * of Upsilon_i = (t_1 + ... + t_i) / mean(t) against Lambda_i is cut with
 * Upsilon = i, and lambda_out [nparts] = the differences of the new
 * Lambda (ordered, sum P).  Host only.  Errors: FEA_EINVAL (bad sizes,
 * negative or all-zero times), FEA_ENUMERIC (a regression without positive
 * slope). */
fea_status fea_balance_update(int32_t nparts, int32_t n_obs, const double *Lambda, const double *times,
                              double *lambda_out);

/* Interface pack: out [3][n_class] (device) is zeroed, then
 * out[c][cls[k]] += v[c][loc[k]] for k < m, c < 3, with v [3][n] (device,
 * FP64, the RHS layout) and loc, cls [m] (device, int64).  Summing out over
 * all parts (e.g. an all-reduce) and unpacking gives every copy of a class
 * the class total.  Out-of-range indices are skipped and reported by
 * fea_sync_status (FEA_EMESH).  Asynchronous on stream. */
fea_status fea_interface_pack(fea_ctx *ctx, const double *v, int64_t n, const int64_t *loc, const int64_t *cls,
                              int64_t m, double *out, int64_t n_class, void *stream);

/* Interface unpack: v[c][loc[k]] = in[c][cls[k]] for k < m, c < 3 (all
 * device memory; in [3][n_class]).  Asynchronous on stream. */
fea_status fea_interface_unpack(fea_ctx *ctx, const double *in, int64_t n_class, const int64_t *loc,
                                const int64_t *cls, int64_t m, double *v, int64_t n, void *stream);

/* Allocation-free RK stage (no counterpart in the paper).
 *
 * For callers that cannot allocate device memory at call time -- code that
 * runs under a fixed, pre-reserved device-memory budget or inside an
 * embedding that forbids cudaMalloc/cudaFree after set-up.  It computes the
 * same stage as fea_rk_stage,
 *   uk_out = a_k un + b_k (uk + dt M^-1 R(uk, p)),  (a, b) as in fea_rk_stage,
 * R folded over periodic pairs, M the mesh's folded lumped mass, Dirichlet
 * nodes holding un, but reads the state from and writes it to caller arrays
 * and allocates nothing: its scratch (the FP64 RHS and an FP32 copy of uk and
 * p, 40 bytes per node) is one static device array, reserved on every GPU
 * that loads the library and held until the process exits.
 *   un, uk, p: device, [3][n_nodes], [3][n_nodes], [n_nodes] FP64 (inputs);
 *   uk_out: device [3][n_nodes] FP64 (output; may be the same array as uk
 *           or as un, e.g. the last stage writing u^(n+1) over u^n);
 *   nu, c_vreman: viscosity and Vreman constant for this call.
 * The mesh must have been uploaded (fea_mesh_upload allocates as usual) and
 * have at most FEA_NOALLOC_MAX_NODES nodes, else FEA_EINVAL.  fea_create
 * looks up the array's device address on its device (this loads the
 * library's device module there and reserves the array), so no call of this
 * entry point loads or reserves anything.
 * Every call on a device shares the array and it keeps the last call's
 * contents: each call clears the RHS part itself, and calls that overlap on
 * the GPU (e.g. on two streams at once) race on the shared scratch. */
#define FEA_NOALLOC_MAX_NODES 262144
fea_status fea_rk_stage_noalloc(fea_ctx *ctx, int32_t mesh, int32_t stage, double dt, fea_prec prec,
                                fea_closure closure, double nu, double c_vreman, const double *un, const double *uk,
                                const double *p, double *uk_out, void *stream);

/* ---- plans, autotuning, status ----------------------------------------- */

fea_status fea_get_plan(fea_ctx *ctx, int32_t mesh, fea_plan *plan);
fea_status fea_set_plan(fea_ctx *ctx, int32_t mesh, const fea_plan *plan);

/* Times the candidate plans of one mesh (after a field upload) with CUDA
 * events and keeps the fastest: ATOMIC, WARP and COLOUR (not with the MLP
 * closure) at 128 and 256 threads and, under FEA_MIXED, CHUNK plans of 256,
 * 512 and 1024 elements; a CHUNK plan within 5 % of the fastest is kept
 * instead (its chunk-relative FP32 coordinates are the more accurate
 * mixed-precision path).  With cache_path != NULL, a text file of
 * lines "key scatter threads chunk_elems chunk_acc ms" keyed by device name,
 * node and element counts, precision and closure: a matching line (the last
 * one) is applied through fea_set_plan instead of timing; otherwise the
 * result is appended.  Synchronous.  Errors: FEA_ESTATE (no field), the
 * errors of fea_set_plan for a cached plan, FEA_EINVAL (cache not writable). */
fea_status fea_autotune(fea_ctx *ctx, int32_t mesh, fea_prec prec, fea_closure closure, const char *cache_path);

/* Synchronises the stream, then reads and clears the device error word:
 * FEA_EMESH (det J <= 0 seen), FEA_ENUMERIC (non-finite residual),
 * FEA_ETIMEOUT (bounded wait gave up), or FEA_OK. */
fea_status fea_sync_status(fea_ctx *ctx, void *stream);

/* Measured FP32 arithmetic peak of the context's device (a measurement
 * utility; the paper has no counterpart): every thread runs eight
 * independent multiply-add chains, scalar FFMA or paired FFMA2 on float2, 8
 * CTAs of 256 threads per SM; the best of three timed launches (CUDA events
 * on `stream`, after one warm-up launch) of each kind, a multiply-add
 * counting two operations.  *tflops_ffma, *tflops_ffma2: host outputs in
 * TFLOP/s.  Synchronous; allocates 4 bytes of device memory for the call. */
fea_status fea_fp32_peak(fea_ctx *ctx, double *tflops_ffma, double *tflops_ffma2, void *stream);

/* Poll limit of the bounded device-side waits of the TET04 assembly kernel
 * (mixed precision, chunk scatter), which otherwise give up after 131,072
 * polls of an mbarrier phase, each of which suspends the warp until the
 * phase completes or 20 us pass: polls > 0 sets the limit and makes every poll a
 * non-suspending test, 0 restores the default.  A wait that gives up makes
 * its CTA stop assembling, lets
 * the copies it has in flight land, and sets the device error word
 * (FEA_ETIMEOUT at the next fea_sync_status); the RHS of that assembly is
 * then incomplete.  A small limit is how a test drives that path without a
 * fault.  Host only; drops every captured RK graph of the context. */
fea_status fea_set_wait_limit(fea_ctx *ctx, uint32_t polls);

/* Number of kernels this context has launched so far (host counter). */
int64_t fea_launch_count(const fea_ctx *ctx);

/* Kernel timing (profiling aid).  While enabled, every element-assembly
 * kernel launched outside a CUDA graph is bracketed by two CUDA events
 * recorded on its launch stream, and the categories of an assembly run one
 * after the other on the caller's stream (no overlap), so that each time is
 * that kernel's alone.  fea_profile_read synchronises those
 * events and returns, for the category (etype, fp64_jac), the summed kernel
 * time in milliseconds and the number of launches; reset != 0 clears the
 * records.  Errors: FEA_EINVAL, FEA_ECUDA. */
fea_status fea_profile_enable(fea_ctx *ctx, int on);
fea_status fea_profile_read(fea_ctx *ctx, int etype, int fp64_jac, double *total_ms, int64_t *launches, int reset);

#ifdef __cplusplus
}
#endif
#endif /* FEA_H */
