// Internal declarations shared by the host side (fea_api.cu) and the kernel
// translation unit (fea_kernels.cu) of libfea.  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "fea.h"

namespace fea {

constexpr int kNen[4] = {4, 5, 6, 8};
constexpr int kNg[4] = {4, 8, 6, 8};
constexpr int kMaxNen = 8;
constexpr int kMaxNg = 8;

// device error word bits (OR-ed by kernels, read by fea_sync_status)
enum : unsigned {
    ERR_DETJ = 1u,      // det J <= 0 at some Gauss point
    ERR_NONFINITE = 2u, // non-finite element residual
    ERR_TIMEOUT = 4u,   // a bounded device-side wait gave up
    ERR_INDEX = 8u,     // index out of range (checked builds and upload validation)
    ERR_WALL_GEOM = 16u,   // wall model: degenerate face or exchange point not on the fluid side
    ERR_WALL_NEWTON = 32u  // wall model: the u_tau iteration did not converge
};

// Reference-element tables at the Gauss points of each type's rule.
struct RefTables {
    double xi[4][kMaxNg][3];   // Gauss points in reference coordinates
    double N[4][kMaxNg][kMaxNen];
    double dN[4][kMaxNg][kMaxNen][3];
    double w[4][kMaxNg];
};

// One category: elements of one type and one Jacobian precision, sorted
// along a Morton curve; connectivity structure-of-arrays [nen][count].
struct BucketDev {
    int etype;
    int fp64j;              // 1: FP64 Jacobian in the mixed path
    int64_t count;
    const int32_t *conn;    // [nen][count] caller node ids
    const int32_t *orig;    // [count] caller element index within its type
    // chunk tables (CTA-local scatter): chunk k holds elements
    // [k C, min((k+1) C, count)) and the L_k distinct nodes they touch
    int32_t chunk_elems;            // C
    int64_t n_chunks;
    const uint16_t *lconn;          // [count][2][np]: np chunk-local node indices of the
                                    // element, then the np positions of its incidences in
                                    // the chunk's node-sorted incidence list (np = 4 for
                                    // TET04, 8 otherwise; padded for one vector load)
    const int64_t *chunk_node_off;  // [n_chunks + 1] offsets into chunk_rec / inc_range;
                                    // each chunk's node list is padded to a multiple of 4
                                    // entries (16-byte aligned for bulk copies)
    const int32_t *chunk_nodes;     // [n_chunks] true node count L_k (without padding)
    const float4 *chunk_rec;        // per local node: FP32 coordinates relative to the
                                    // chunk's first node, and in .w the bits of the caller
                                    // node id with bit 31 set if other chunks touch it too
    const uint32_t *inc_range;      // per local node: first incidence | count << 16; local
                                    // nodes are ordered by decreasing incidence count
    int32_t max_chunk_nodes;        // max L_k
    // colouring (FEA_SCATTER_COLOUR): the elements reordered colour by colour
    const int32_t *col_conn;        // [nen][count] node ids in colour order
    const int32_t *col_orig;        // [count] caller element index, colour order
    // tables of the warp-specialised TET04 kernel (k_tet_ws): chunks of
    // C = 64 ws_nw elements, each with its L_k distinct nodes ordered by
    // decreasing incidence count, their incidences numbered node by node
    int ws_nw = 0;                  // compute warps per CTA (0: no tables)
    int32_t ws_lmp = 0;             // max padded node-list length (multiple of 4, <= 1024)
    int64_t ws_nch = 0;
    const int64_t *ws_off = nullptr;    // [ws_nch + 1] offsets into ws_rec / ws_ids
    const int32_t *ws_nodes = nullptr;  // [ws_nch] L_k
    const float4 *ws_rec = nullptr;     // per local node: FP32 coordinates relative to the
                                        // chunk's first node (.w unused); padded to a multiple
                                        // of 4 entries
    const uint32_t *ws_ids = nullptr;   // per local node: caller node id, bit 31 set when
                                        // elements outside the chunk touch it too
    const uint4 *ws_elem = nullptr;     // [ws_nch][C/2] records of 8 x u16 (local node id
                                        // (10 bits) | the incidence's rank among the node's
                                        // slots << 10): first ws_nfp face pairs
                                        // (f0, f1, f2, a, b; see the kernel), then pairs of
                                        // elements (4 + 4 nodes)
    const int32_t *ws_nfp = nullptr;    // [ws_nch] face pairs per chunk
    const uint32_t *ws_toff = nullptr;  // [ws_nch][68] first slot of the t-th incidences
                                        // (t = 0..64; nodes by decreasing slot count)
    const int32_t *ws_eorig = nullptr;  // [ws_nch][C] caller element index of record
                                        // position 2t / 2t + 1 (-1: none)
};

// Per-mesh nodal data used by the kernels.
struct FieldDev {
    int64_t n;
    const double *xyz64;  // [3][n]
    const float4 *xyz32;  // [n] (x, y, z, 0)
    const double *u64;    // [3][n] current state u^(k)
    const double *p64;    // [n]
    const float4 *up32;   // [n] (u, v, w, p), FP32 copy of the state
    double nu;
    double c_vreman;
    int conv_form = 0;    // fea_conv_form: 0 G u + (tr G) u, 1 EMAC
    int delta_form = 0;   // fea_delta_form: 0 V^(1/3), 1 widths per direction
};

struct AsmArgs {
    uint32_t mask;
    int closure;          // fea_closure
    double *rhs;          // [3][n]
    float *nut;           // optional: type block of nu_t output (already offset)
    unsigned *err;        // device error word
    const void *mlp;      // MLP closure weights (device tc::MlpTc) when closure == FEA_CLOSURE_MLP
    unsigned long long *mlp_fb = nullptr;   // count of Gauss points that fell back to Vreman (MLP only)
    // chunk kernels: launched as a programmatic dependent of the kernel before
    // it on the stream (starts while that one drains; waits for it to
    // complete before it ends itself)
    int pdl = 0;
    // bounded device waits (warp-specialised TET04 kernel): polls before a
    // wait gives up; 0 = the default (about 4 million)
    uint32_t wait_polls = 0;
};

// launchers (fea_kernels.cu); all return cudaGetLastError() of the launch
cudaError_t upload_ref_tables(const RefTables &t);
cudaError_t launch_assemble_bucket(const BucketDev &b, const FieldDev &f, const AsmArgs &a, fea_prec prec,
                                   fea_scatter scatter, int threads, cudaStream_t s);
// colour scatter: one launch per colour over [col_off[k], col_off[k+1]) of the
// colour-ordered connectivity (col_off on the host)
cudaError_t launch_assemble_colour(const BucketDev &b, const FieldDev &f, const AsmArgs &a, fea_prec prec,
                                   int threads, const int64_t *col_off, int n_colours, cudaStream_t s);
cudaError_t launch_assemble_chunk(const BucketDev &b, const FieldDev &f, const AsmArgs &a, int threads,
                                  int compensated, cudaStream_t s);
size_t chunk_smem_bytes(const BucketDev &b);
// shared memory a CTA needs for the fused MLP: weights plus per-warp scratch
size_t mlp_smem_bytes(int threads, int rows_per_elem);
// shared memory of a chunk launch with this many threads, with or without the MLP
size_t chunk_launch_smem(const BucketDev &b, int threads, int compensated, bool mlp);
constexpr size_t kMaxBlockSmem = 227 * 1024;   // opt-in dynamic shared memory per CTA
// shared memory of the chunk kernel that launch_assemble_chunk would launch
size_t chunk_kernel_smem(const BucketDev &b, int compensated);
constexpr size_t kChunkSmemLimit = 200 * 1024;
// batched persistent launch over (category, chunk) items of many meshes
cudaError_t launch_assemble_batch(const void *buckets, const void *fields, const void *args, const void *items,
                                  int64_t n_items, unsigned long long *counter, size_t smem, int sms, bool mlp,
                                  bool variants,
                                  cudaStream_t s);
size_t batch_item_bytes();
cudaError_t launch_zero_batch(double *const *rhs_dev, const int64_t *len_dev, int n_meshes, cudaStream_t s);
cudaError_t launch_tet_ws(const BucketDev &b, const FieldDev &f, const AsmArgs &a, int sms, cudaStream_t s);
size_t tet_ws_smem_bytes(int nw, int lmp);
constexpr int lconn_pitch(int etype) { return etype == FEA_TET04 ? 4 : 8; }
cudaError_t launch_lumped_mass(const BucketDev &b, const double *xyz64, int64_t n, double *mass, unsigned *err,
                               unsigned long long *bad, cudaStream_t s);
cudaError_t launch_fold(const int32_t *slaves, const int32_t *masters, int64_t n_slaves, double *v, int ncomp,
                        int64_t n, cudaStream_t s);
// stage update: reads u^n (un) and u^(k) (uk_in), writes the result to
// uk_out (and un_out if not NULL); the three may alias
cudaError_t launch_rk_update(int64_t n, const double *un, const double *uk_in, double *uk_out, double *un_out,
                             const double *rhs, const double *minv, const uint8_t *dirichlet, const double *p64,
                             float4 *up32, double a, double b, double dt, cudaStream_t s);
cudaError_t launch_pack_field(int64_t n, const double *u64, const double *p64, float4 *up32, cudaStream_t s);
// wall-model boundary term (fea_wall.cu): faces [nv][n_faces] and their
// exchange nodes, FP64; adds into rhs [3][n]
struct WallDev {
    int64_t n_faces;
    int nv;                 // 3 or 4
    const int32_t *face;    // [nv][n_faces]
    const int32_t *exch;    // [nv][n_faces]
    double kappa, c_plus;
};
// fp64: u_tau to FP64 accuracy (else its FP32 root, for the mixed mode)
cudaError_t launch_wall(const WallDev &w, const double *xyz64, const double *u64, int64_t n, double nu, double *rhs,
                        unsigned *err, bool fp64, cudaStream_t s);
cudaError_t launch_f32_to_f64(const float *src, double *dst, int64_t count, cudaStream_t s);
cudaError_t launch_recip(const double *m, double *minv, int64_t n, cudaStream_t s);
// FP32 FMA-chain peak (fea_peak.cu): TFLOP/s of scalar FFMA and of paired
// FFMA2, best of three timed launches each on stream s (synchronous)
cudaError_t measure_fp32_peak(int sms, cudaStream_t s, double *tflops_ffma, double *tflops_ffma2);

// pressure projection element operators (fea_kernels.cu), FP64
cudaError_t launch_lap_assemble(const BucketDev &b, const double *xyz, int64_t n, const int32_t *cls,
                                const int64_t *rowptr, const int32_t *col, double *val, unsigned *err,
                                cudaStream_t s);
cudaError_t launch_divgrad_assemble(const BucketDev &b, const double *xyz, int64_t n, bool div, const double *in,
                                    double *out, unsigned *err, cudaStream_t s);
cudaError_t launch_project_update(int64_t n, double *uk, double *un, const double *g, const double *minv,
                                  const uint8_t *dirichlet, double *p, const double *dp, float4 *up32, double dt,
                                  int sms, cudaStream_t s);

// pressure equation on periodic classes (fea_poisson.cu)
struct PoissonSystem;
struct PoissonBuild {
    int64_t n = 0;                        // nodes
    std::vector<const int32_t *> conn;    // per bucket, host [nen][count]
    std::vector<int64_t> count;
    std::vector<int> nen;
    const int32_t *class_of = nullptr;    // host [n]: periodic master of each node (NULL: none)
    const uint8_t *pinned = nullptr;      // host [n]: pinned nodes (NULL: the class of node 0)
};
cudaError_t poisson_build(const PoissonBuild &in, int sms, PoissonSystem **out);
cudaError_t poisson_finish(PoissonSystem *ps, unsigned *err, int sms, cudaStream_t s);
cudaError_t poisson_solve(PoissonSystem *ps, const double *b_node, double scale, double *x_node, double rtol,
                          int max_iter, int sms, cudaStream_t s, int *iters_out, double *rel_res_out, int64_t *launches);
void poisson_free(PoissonSystem *ps);
int64_t poisson_classes(const PoissonSystem *ps);
int64_t poisson_nnz(const PoissonSystem *ps);
const int32_t *poisson_cls(const PoissonSystem *ps);
const int64_t *poisson_rowptr(const PoissonSystem *ps);
const int32_t *poisson_col(const PoissonSystem *ps);
double *poisson_val(PoissonSystem *ps);

// interface exchange of a partitioned mesh (fea_kernels.cu)
cudaError_t launch_iface_pack(const double *v, int64_t n, const int64_t *loc, const int64_t *cls, int64_t m,
                              double *out, int64_t nc, unsigned *err, int sms, cudaStream_t s);
cudaError_t launch_iface_unpack(const double *in, int64_t nc, const int64_t *loc, const int64_t *cls, int64_t m,
                                double *v, int64_t n, unsigned *err, int sms, cudaStream_t s);

// space-filling curves (fea_partition.cu)
uint64_t morton_spread3(uint64_t v);
// Greedy element colouring (fea_partition.cu): elements in the given order
// take the lowest colour none of their nodes has seen (no two elements of a
// colour share a node); node a of element e is conn[e * elem_stride + a *
// node_stride].  Returns the number of colours, -1 above kColourMax, -2 for
// a node id outside [0, n_nodes).
constexpr int kColourMax = 256;
int greedy_colour(int64_t n_nodes, int nen, int64_t count, const int32_t *conn, int64_t elem_stride,
                  int64_t node_stride, int32_t *col);                              // 21 bits -> every third bit
uint64_t hilbert_key3(uint32_t x0, uint32_t x1, uint32_t x2, int bits);   // Hilbert index in a 2^bits grid

// MLP closure (fea_mlp.cu)
size_t mlp_weights_bytes();
const void *mlp_fast_ptr(const void *w);   // inference layout inside the weights block
int mlp_param_count();
cudaError_t launch_mlp_pack(const float *theta, const float *mean, const float *stdv, float out_scale, void *w,
                            cudaStream_t s);
cudaError_t launch_mlp_forward(const void *w, const float *x, int64_t B, float *y, int sms, unsigned *err,
                               cudaStream_t s);
cudaError_t launch_mlp_train(const void *w, const float *x, const float *y, int64_t B, float *grad, float *loss,
                             cudaStream_t s);
cudaError_t launch_adam(float *theta, const float *grad, float *m1, float *m2, int n, float lr, float b1, float b2,
                        float eps, int64_t step, cudaStream_t s);

// One RK stage from caller state arrays, with caller-provided scratch
// (rhs [3][n] FP64, up [n] FP32 (u, v, w, p)); used by the allocation-free
// entry point.  Implemented in fea_api.cu.
fea_status stage_with_scratch(fea_ctx *ctx, int32_t mesh, int32_t stage, double dt, fea_prec prec,
                              fea_closure closure, double nu, double c_vreman, const double *un, const double *uk,
                              const double *p, double *uk_out, double *rhs, float4 *up, int64_t max_nodes,
                              cudaStream_t s);
int context_device(const fea_ctx *ctx);
// device address of the allocation-free stage's static scratch on `device`
// (fea_noalloc.cu); looked up once per device, first at fea_create
cudaError_t noalloc_scratch_address(int device, void **out);
fea_status context_fail(fea_ctx *ctx, fea_status st, const char *msg);

}  // namespace fea
