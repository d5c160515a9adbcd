// C ABI of libfea (see include/fea.h): contexts, mesh upload and category
// packing, field upload, the assembly entry points, RK stages, CUDA-graph
// capture, plans and the device status word.
#include <cuda_runtime.h>
#include <math.h>
#include <stdarg.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <array>
#include <memory>
#include <string>
#include <vector>

#include "fea_internal.h"

using namespace fea;

namespace {

// ---------------------------------------------------------------------------
// reference elements: Gauss rules and shape functions at the Gauss points

void gauss2(double x[2]) {
    x[0] = -1.0 / sqrt(3.0);
    x[1] = 1.0 / sqrt(3.0);
}

// Quadrature points (reference coordinates) and weights per type.
int rule(int et, double pts[][3], double w[]) {
    double g[2];
    gauss2(g);
    int n = 0;
    switch (et) {
        case FEA_TET04: {
            // degree-2 rule: one barycentric coordinate b, the others a
            const double a = (5.0 - sqrt(5.0)) / 20.0, b = (5.0 + 3.0 * sqrt(5.0)) / 20.0;
            const double bary[4][4] = {{b, a, a, a}, {a, b, a, a}, {a, a, b, a}, {a, a, a, b}};
            for (int q = 0; q < 4; ++q) {
                // (r, s, t) = barycentric weights of vertices 1, 2, 3
                pts[n][0] = bary[q][1];
                pts[n][1] = bary[q][2];
                pts[n][2] = bary[q][3];
                w[n++] = 1.0 / 24.0;
            }
            // order: point q has the large weight on vertex q (q = 0 first)
            return n;
        }
        case FEA_PEN06: {
            // level-major, and these triangle points in this order: the prism
            // Jacobian of the element kernels (PrismGeom) relies on both
            const double tri[3][2] = {{1.0 / 6.0, 1.0 / 6.0}, {2.0 / 3.0, 1.0 / 6.0}, {1.0 / 6.0, 2.0 / 3.0}};
            for (int kz = 0; kz < 2; ++kz)
                for (int q = 0; q < 3; ++q) {
                    pts[n][0] = tri[q][0];
                    pts[n][1] = tri[q][1];
                    pts[n][2] = g[kz];
                    w[n++] = 1.0 / 6.0;
                }
            return n;
        }
        case FEA_HEX08: {
            for (int k = 0; k < 2; ++k)
                for (int j = 0; j < 2; ++j)
                    for (int i = 0; i < 2; ++i) {
                        pts[n][0] = g[i];
                        pts[n][1] = g[j];
                        pts[n][2] = g[k];
                        w[n++] = 1.0;
                    }
            return n;
        }
        case FEA_PYR05: {
            // (a, b, t) -> ((1-t) a, (1-t) b, t); Gauss-Legendre in a, b and
            // the 2-point rule for the weight (1-t)^2 on [0, 1] in t, whose
            // nodes are the roots of t^2 - (2/3) t + 1/15.
            const double r = sqrt(2.0 / 45.0);
            const double tn[2] = {1.0 / 3.0 - r, 1.0 / 3.0 + r};
            // weights from the moments int (1-t)^2 = 1/3 and int t (1-t)^2 = 1/12
            const double w1 = (1.0 / 12.0 - tn[0] / 3.0) / (tn[1] - tn[0]);
            const double tw[2] = {1.0 / 3.0 - w1, w1};
            for (int k = 0; k < 2; ++k)
                for (int j = 0; j < 2; ++j)
                    for (int i = 0; i < 2; ++i) {
                        pts[n][0] = (1.0 - tn[k]) * g[i];
                        pts[n][1] = (1.0 - tn[k]) * g[j];
                        pts[n][2] = tn[k];
                        w[n++] = tw[k];
                    }
            return n;
        }
    }
    return 0;
}

void shape_at(int et, const double x[3], double N[], double dN[][3]) {
    const double r = x[0], s = x[1], t = x[2];
    switch (et) {
        case FEA_TET04: {
            N[0] = 1.0 - r - s - t;
            N[1] = r;
            N[2] = s;
            N[3] = t;
            for (int a = 0; a < 4; ++a)
                for (int j = 0; j < 3; ++j) dN[a][j] = (a == 0) ? -1.0 : (a - 1 == j ? 1.0 : 0.0);
            return;
        }
        case FEA_PEN06: {
            const double L[3] = {1.0 - r - s, r, s};
            const double dLr[3] = {-1.0, 1.0, 0.0}, dLs[3] = {-1.0, 0.0, 1.0};
            for (int h = 0; h < 2; ++h) {
                const double zf = h ? 0.5 * (1.0 + t) : 0.5 * (1.0 - t);
                const double dz = h ? 0.5 : -0.5;
                for (int i = 0; i < 3; ++i) {
                    const int a = 3 * h + i;
                    N[a] = L[i] * zf;
                    dN[a][0] = dLr[i] * zf;
                    dN[a][1] = dLs[i] * zf;
                    dN[a][2] = L[i] * dz;
                }
            }
            return;
        }
        case FEA_HEX08: {
            static const int sg[8][3] = {{-1, -1, -1}, {1, -1, -1}, {1, 1, -1}, {-1, 1, -1},
                                         {-1, -1, 1},  {1, -1, 1},  {1, 1, 1},  {-1, 1, 1}};
            for (int a = 0; a < 8; ++a) {
                const double px = 0.5 * (1.0 + sg[a][0] * r), py = 0.5 * (1.0 + sg[a][1] * s),
                             pz = 0.5 * (1.0 + sg[a][2] * t);
                N[a] = px * py * pz;
                dN[a][0] = 0.5 * sg[a][0] * py * pz;
                dN[a][1] = 0.5 * sg[a][1] * px * pz;
                dN[a][2] = 0.5 * sg[a][2] * px * py;
            }
            return;
        }
        case FEA_PYR05: {
            // base corners c = (cx, cy); the rational term carries xi eta zeta / (1 - zeta)
            static const int cb[4][2] = {{-1, -1}, {1, -1}, {1, 1}, {-1, 1}};
            const double inv = 1.0 / (1.0 - t);
            const double q = r * s * t * inv;
            for (int a = 0; a < 4; ++a) {
                const double cx = cb[a][0], cy = cb[a][1];
                N[a] = 0.25 * ((1.0 + cx * r) * (1.0 + cy * s) - t + cx * cy * q);
                dN[a][0] = 0.25 * (cx * (1.0 + cy * s) + cx * cy * s * t * inv);
                dN[a][1] = 0.25 * (cy * (1.0 + cx * r) + cx * cy * r * t * inv);
                dN[a][2] = 0.25 * (-1.0 + cx * cy * r * s * inv * inv);
            }
            N[4] = t;
            dN[4][0] = 0.0;
            dN[4][1] = 0.0;
            dN[4][2] = 1.0;
            return;
        }
    }
}

RefTables make_tables() {
    RefTables T;
    memset(&T, 0, sizeof(T));
    for (int et = 0; et < 4; ++et) {
        double pts[kMaxNg][3], w[kMaxNg];
        const int ng = rule(et, pts, w);
        for (int g = 0; g < ng; ++g) {
            double N[kMaxNen], dN[kMaxNen][3];
            shape_at(et, pts[g], N, dN);
            T.w[et][g] = w[g];
            for (int j = 0; j < 3; ++j) T.xi[et][g][j] = pts[g][j];
            for (int a = 0; a < kNen[et]; ++a) {
                T.N[et][g][a] = N[a];
                for (int j = 0; j < 3; ++j) T.dN[et][g][a][j] = dN[a][j];
            }
        }
    }
    return T;
}

// ---------------------------------------------------------------------------

template <typename T>
struct DevBuf {
    T *p = nullptr;
    size_t n = 0;
    DevBuf() = default;
    DevBuf(const DevBuf &) = delete;
    DevBuf &operator=(const DevBuf &) = delete;
    ~DevBuf() { reset(); }
    void reset() {
        if (p) cudaFree(p);
        p = nullptr;
        n = 0;
    }
    cudaError_t alloc(size_t count) {
        reset();
        if (count == 0) return cudaSuccess;
        n = count;
        return cudaMalloc((void **)&p, count * sizeof(T));
    }
};

struct Bucket {
    int etype = 0, fp64j = 0;
    int64_t count = 0;
    std::vector<int32_t> conn_h;  // host copy [nen][count] (chunk tables are rebuilt from it)
    DevBuf<int32_t> conn, orig;
    // chunk tables
    int32_t chunk_elems = 0;
    int64_t n_chunks = 0;
    int32_t max_chunk_nodes = 0;
    DevBuf<uint16_t> lconn;
    DevBuf<int64_t> chunk_off;
    DevBuf<int32_t> chunk_nodes;
    DevBuf<float4> chunk_rec;
    DevBuf<uint32_t> inc_range;
    // tables of the warp-specialised TET04 kernel (mixed precision, chunk scatter)
    int ws_nw = 0, ws_want = 0;
    int32_t ws_lmp = 0;
    int64_t ws_nch = 0;
    DevBuf<int64_t> ws_off;
    DevBuf<int32_t> ws_nodes;
    DevBuf<float4> ws_rec;
    DevBuf<uint32_t> ws_ids;
    DevBuf<int32_t> ws_nfp, ws_eorig;
    DevBuf<uint32_t> ws_toff;
    DevBuf<uint4> ws_elem;
    // colouring (FEA_SCATTER_COLOUR), built on first use
    DevBuf<int32_t> col_conn, col_orig;
    std::vector<int64_t> col_off;   // [n_colours + 1] element offsets per colour
    int n_colours = 0;
    BucketDev dev() const {
        BucketDev b;
        b.etype = etype;
        b.fp64j = fp64j;
        b.count = count;
        b.conn = conn.p;
        b.orig = orig.p;
        b.chunk_elems = chunk_elems;
        b.n_chunks = n_chunks;
        b.lconn = lconn.p;
        b.chunk_node_off = chunk_off.p;
        b.chunk_nodes = chunk_nodes.p;
        b.chunk_rec = chunk_rec.p;
        b.inc_range = inc_range.p;
        b.max_chunk_nodes = max_chunk_nodes;
        b.col_conn = col_conn.p;
        b.col_orig = col_orig.p;
        b.ws_nw = ws_nw;
        b.ws_lmp = ws_lmp;
        b.ws_nch = ws_nch;
        b.ws_off = ws_off.p;
        b.ws_nodes = ws_nodes.p;
        b.ws_rec = ws_rec.p;
        b.ws_ids = ws_ids.p;
        b.ws_elem = ws_elem.p;
        b.ws_nfp = ws_nfp.p;
        b.ws_eorig = ws_eorig.p;
        b.ws_toff = ws_toff.p;
        return b;
    }
};

struct GraphCache {
    cudaGraphExec_t exec = nullptr;
    double dt = 0.0;
    int prec = -1, closure = -1;
};

struct Mesh {
    int64_t n = 0;
    int64_t n_elem[4] = {0, 0, 0, 0};
    std::vector<std::unique_ptr<Bucket>> buckets;
    DevBuf<double> xyz64;
    DevBuf<float4> xyz32;
    DevBuf<int32_t> slaves, masters;
    DevBuf<uint8_t> dirichlet;
    DevBuf<double> mass, minv;
    // state
    DevBuf<double> un, uk, p64, rhs;
    DevBuf<float4> up32;
    DevBuf<float> stage_f32;
    bool has_field = false;
    double nu = 0.0, c_vreman = 0.0;
    std::vector<double> xyz_h;          // host FP64 coordinates [3][n] (chunk-local offsets)
    std::vector<int32_t> inc_total;     // element incidences per node over all buckets
    fea_plan plan{FEA_SCATTER_CHUNK, 256, 256, 0};
    GraphCache graph;
    std::vector<int32_t> master_h;      // host periodic masters (empty: none)
    int conv_form = 0, delta_form = 0;  // model variants (fea_set_model)
    PoissonSystem *poisson = nullptr;   // pressure equation (fea_poisson_setup)
    DevBuf<double> proj_b, proj_dp, proj_g;
    // wall-model faces (fea_wall_setup): [0] triangles, [1] quads, SoA [nv][n]
    DevBuf<int32_t> wall_face[2], wall_exch[2];
    int64_t wall_n[2] = {0, 0};
    double wall_kappa = 0.41, wall_c = 7.8;
    WallDev wall_dev(int k) const {
        WallDev w;
        w.n_faces = wall_n[k];
        w.nv = k ? 4 : 3;
        w.face = wall_face[k].p;
        w.exch = wall_exch[k].p;
        w.kappa = wall_kappa;
        w.c_plus = wall_c;
        return w;
    }
    int wall_launches() const { return (wall_n[0] > 0) + (wall_n[1] > 0); }
    ~Mesh() {
        if (graph.exec) cudaGraphExecDestroy(graph.exec);
        if (poisson) poisson_free(poisson);
    }
    FieldDev field() const {
        FieldDev f;
        f.n = n;
        f.xyz64 = xyz64.p;
        f.xyz32 = xyz32.p;
        f.u64 = uk.p;
        f.p64 = p64.p;
        f.up32 = up32.p;
        f.nu = nu;
        f.c_vreman = c_vreman;
        f.conv_form = conv_form;
        f.delta_form = delta_form;
        return f;
    }
};

}  // namespace

struct ProfRec {
    int etype, fp64j;
    cudaEvent_t e0, e1;
};

struct fea_ctx {
    int device = 0;
    int sms = 148;
    bool profiling = false;
    std::vector<ProfRec> prof;
    std::string err;
    unsigned *d_err = nullptr;
    unsigned long long *d_bad = nullptr;
    std::vector<std::unique_ptr<Mesh>> meshes;
    cudaStream_t capture = nullptr;
    cudaStream_t side = nullptr;      // FP64-Jacobian categories run here, overlapped
    // batched launch: descriptor tables, work items and the work counter
    DevBuf<unsigned char> batch_bk, batch_fd, batch_ag, batch_items;
    DevBuf<double *> batch_rhs;
    DevBuf<int64_t> batch_len;
    DevBuf<unsigned long long> batch_counter;
    bool batch_per_mesh = false;   // fea_autotune_batched chose per-mesh launches over the persistent one
    // learned closure: FP32 master parameters, Adam moments, packed BF16 weights
    DevBuf<float> mlp_theta, mlp_m1, mlp_m2, mlp_grad, mlp_loss, mlp_norm;
    DevBuf<unsigned char> mlp_w;
    DevBuf<unsigned long long> mlp_fb;   // Gauss points that fell back to Vreman
    int64_t mlp_step = 0;
    double mlp_scale = 0.0;
    bool mlp_ready = false;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    int64_t launches = 0;
    uint32_t wait_polls = 0;   // fea_set_wait_limit (0: kernels' default)
};

namespace {

fea_status fail(fea_ctx *c, fea_status st, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (c) c->err = buf;
    return st;
}

#define CK(call)                                                                                      \
    do {                                                                                              \
        cudaError_t e_ = (call);                                                                      \
        if (e_ != cudaSuccess)                                                                        \
            return fail(ctx, e_ == cudaErrorMemoryAllocation ? FEA_ENOMEM : FEA_ECUDA, "%s: %s (%s:%d)", \
                        #call, cudaGetErrorString(e_), __FILE__, __LINE__);                           \
    } while (0)

fea_status get_mesh(fea_ctx *ctx, int32_t id, Mesh **m) {
    if (!ctx) return FEA_EINVAL;
    if (id < 0 || id >= (int32_t)ctx->meshes.size() || !ctx->meshes[id])
        return fail(ctx, FEA_ENOTFOUND, "unknown mesh id %d", id);
    *m = ctx->meshes[id].get();
    return FEA_OK;
}


int64_t type_nut_offset(const Mesh &m, int et) {
    int64_t off = 0;
    for (int t = 0; t < et; ++t) off += m.n_elem[t] * kNg[t];
    return off;
}

// Chunk tables of one bucket for chunks of C elements (see BucketDev).
fea_status build_chunks(fea_ctx *ctx, Mesh &m, Bucket &b, int C) {
    const int nen = kNen[b.etype];
    const int np = lconn_pitch(b.etype);
    const int64_t cnt = b.count;
    const int64_t nch = (cnt + C - 1) / C;
    std::vector<uint16_t> lconn((size_t)2 * np * cnt, 0);
    std::vector<int64_t> off((size_t)nch + 1, 0);
    std::vector<int32_t> nodes_n((size_t)nch, 0);
    std::vector<float4> recs;
    std::vector<uint32_t> ranges;
    recs.reserve((size_t)(cnt / 2 + 64));
    ranges.reserve((size_t)(cnt / 2 + 64));
    std::vector<int32_t> ids((size_t)nen * C), uniq, lcount, order, rank, lstart, fillp;
    std::vector<int32_t> tmp((size_t)nen * C);
    int32_t maxL = 0;
    const int64_t n = m.n;
    for (int64_t k = 0; k < nch; ++k) {
        const int64_t e0 = k * C;
        const int ne = (int)std::min<int64_t>(C, cnt - e0);
        size_t q = 0;
        for (int a = 0; a < nen; ++a)
            for (int el = 0; el < ne; ++el) ids[q++] = b.conn_h[(size_t)a * cnt + e0 + el];
        uniq.assign(ids.begin(), ids.begin() + q);
        std::sort(uniq.begin(), uniq.end());
        uniq.erase(std::unique(uniq.begin(), uniq.end()), uniq.end());
        const int L = (int)uniq.size();
        if (L > 65532 || nen * ne > 65535)
            return fail(ctx, FEA_EINVAL, "chunk of %d elements is too large for 16-bit local indices", C);
        maxL = std::max(maxL, (L + 3) & ~3);
        // incidence of every (element, vertex) as an index into uniq
        lcount.assign(L, 0);
        q = 0;
        for (int a = 0; a < nen; ++a)
            for (int el = 0; el < ne; ++el) {
                const int l = (int)(std::lower_bound(uniq.begin(), uniq.end(), ids[q]) - uniq.begin());
                tmp[q++] = l;
                lcount[l]++;
            }
        // local order: decreasing incidence count, then node id (uniform loops in the node phase)
        order.resize(L);
        for (int l = 0; l < L; ++l) order[l] = l;
        std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return lcount[x] > lcount[y]; });
        rank.resize(L);
        for (int l = 0; l < L; ++l) rank[order[l]] = l;
        lstart.assign(L + 1, 0);
        for (int l = 0; l < L; ++l) lstart[l + 1] = lstart[l] + lcount[order[l]];
        fillp.assign(lstart.begin(), lstart.end() - 1);
        q = 0;
        for (int a = 0; a < nen; ++a)
            for (int el = 0; el < ne; ++el) {
                const int l = rank[tmp[q++]];
                uint16_t *rec = &lconn[(size_t)2 * np * (e0 + el)];
                rec[a] = (uint16_t)l;
                rec[np + a] = (uint16_t)(fillp[l]++);
            }
        const double ox = m.xyz_h[uniq[0]], oy = m.xyz_h[n + uniq[0]], oz = m.xyz_h[2 * n + uniq[0]];
        for (int l = 0; l < L; ++l) {
            const int32_t id = uniq[order[l]];
            const bool shared = lcount[order[l]] != m.inc_total[id];
            const uint32_t bits = (uint32_t)id | (shared ? 0x80000000u : 0u);
            float w;
            memcpy(&w, &bits, 4);
            recs.push_back(make_float4((float)(m.xyz_h[id] - ox), (float)(m.xyz_h[n + id] - oy),
                                       (float)(m.xyz_h[2 * n + id] - oz), w));
            ranges.push_back((uint32_t)lstart[l] | ((uint32_t)lcount[order[l]] << 16));
        }
        const int Lp = (L + 3) & ~3;   // pad to 16-byte multiples; pad entries are never read
        for (int l = L; l < Lp; ++l) {
            recs.push_back(recs[recs.size() - 1]);
            ranges.push_back(0u);
        }
        nodes_n[k] = L;
        off[k + 1] = off[k] + Lp;
    }
    CK(b.lconn.alloc(lconn.size()));
    CK(b.chunk_off.alloc(off.size()));
    CK(b.chunk_nodes.alloc(nodes_n.size()));
    CK(b.chunk_rec.alloc(recs.size()));
    CK(b.inc_range.alloc(ranges.size()));
    CK(cudaMemcpy(b.lconn.p, lconn.data(), lconn.size() * 2, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(b.chunk_off.p, off.data(), off.size() * 8, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(b.chunk_nodes.p, nodes_n.data(), nodes_n.size() * 4, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(b.chunk_rec.p, recs.data(), recs.size() * sizeof(float4), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(b.inc_range.p, ranges.data(), ranges.size() * 4, cudaMemcpyHostToDevice));
    b.chunk_elems = C;
    b.n_chunks = nch;
    b.max_chunk_nodes = maxL;
    return FEA_OK;
}

// Compute warps of the warp-specialised TET04 kernel for a plan's
// threads_per_block: 12 from 384 threads, 8 from 256, else 4.
int ws_warps_for(int threads) { return threads >= 384 ? 12 : threads >= 256 ? 8 : 4; }

// Tables of the warp-specialised TET04 kernel (see BucketDev::ws_*): chunks
// of C = 64 NW elements, NW = want (12, 8 or 4) or, if its chunks do not
// keep below 1024 nodes and 64 slots per node or its shared memory does not
// fit one CTA, the next smaller.  No tables (the kernel is not used) when
// none fits.
//
// Within a chunk the elements are matched greedily (Morton order) into
// pairs that share a face.  A pair is stored as A = (f0, f1, f2, a) with
// det > 0 and B's fourth node b; B = (f1, f0, f2, b) then has det > 0 as
// well (b lies across the face), so the kernel loads five nodes instead of
// eight and writes one slot per face node for both elements.  Unmatched
// elements follow as plain pairs in their own node order.
fea_status build_ws_tables(fea_ctx *ctx, Mesh &m, Bucket &b, int want) {
    if (b.etype != FEA_TET04 || b.fp64j || b.count == 0) return FEA_OK;
    if (b.ws_want == want) return FEA_OK;
    b.ws_want = want;
    const int64_t cnt = b.count, n = m.n;
    std::vector<int32_t> orig_h((size_t)cnt);
    CK(cudaMemcpy(orig_h.data(), b.orig.p, sizeof(int32_t) * cnt, cudaMemcpyDeviceToHost));
    const double *X = m.xyz_h.data();
    auto det4 = [&](const int32_t v[4]) {
        double d[3][3];
        for (int q = 0; q < 3; ++q)
            for (int k = 0; k < 3; ++k) d[q][k] = X[(size_t)k * n + v[q + 1]] - X[(size_t)k * n + v[0]];
        return d[0][0] * (d[1][1] * d[2][2] - d[1][2] * d[2][1]) - d[0][1] * (d[1][0] * d[2][2] - d[1][2] * d[2][0]) +
               d[0][2] * (d[1][0] * d[2][1] - d[1][1] * d[2][0]);
    };
    for (int nw : {12, 8, 4}) {
        if (nw > want) continue;
        const int C = 64 * nw, R = C / 2;
        const int64_t nch = (cnt + C - 1) / C;
        std::vector<int64_t> off((size_t)nch + 1, 0);
        std::vector<int32_t> nodes_n((size_t)nch, 0), nfp((size_t)nch, 0), eorig((size_t)nch * C, -1);
        std::vector<uint32_t> toff((size_t)nch * 68, 0u);
        std::vector<float4> recs;
        std::vector<uint32_t> idv;
        std::vector<uint4> elem((size_t)nch * R, make_uint4(0u, 0u, 0u, 0u));
        recs.reserve((size_t)(cnt / 2 + 64));
        idv.reserve((size_t)(cnt / 2 + 64));
        // per chunk: the incidences (node ids) of each record in slot order,
        // with the record each belongs to
        std::vector<int32_t> inc, uniq, lcount, order, lrank, lstart, fill, mate, tri;
        std::vector<std::array<int32_t, 5>> fkey;   // (n0, n1, n2, element, opposite local node)
        std::vector<int> nbn;
        std::vector<std::pair<int, int>> nbv;
        int32_t lmp = 0;
        bool fits = true;
        for (int64_t k = 0; k < nch && fits; ++k) {
            const int64_t e0 = k * C;
            const int ne = (int)std::min<int64_t>(C, cnt - e0);
            auto node = [&](int el, int a) { return b.conn_h[(size_t)a * cnt + e0 + el]; };
            // face adjacency inside the chunk
            fkey.clear();
            for (int el = 0; el < ne; ++el)
                for (int o = 0; o < 4; ++o) {
                    int32_t f[3], j = 0;
                    for (int a = 0; a < 4; ++a)
                        if (a != o) f[j++] = node(el, a);
                    std::sort(f, f + 3);
                    fkey.push_back({f[0], f[1], f[2], el, o});
                }
            std::sort(fkey.begin(), fkey.end());
            // face neighbours inside the chunk: (neighbour, my opposite node), at most 4
            nbn.assign(ne, 0);
            nbv.resize((size_t)4 * ne);
            for (size_t i = 0; i + 1 < fkey.size(); ++i)
                if (fkey[i][0] == fkey[i + 1][0] && fkey[i][1] == fkey[i + 1][1] && fkey[i][2] == fkey[i + 1][2]) {
                    const int x = fkey[i][3], y = fkey[i + 1][3];
                    if (nbn[x] < 4) nbv[(size_t)4 * x + nbn[x]++] = {y, fkey[i][4]};
                    if (nbn[y] < 4) nbv[(size_t)4 * y + nbn[y]++] = {x, fkey[i + 1][4]};
                }
            mate.assign(ne, -1);
            tri.assign(ne, -1);   // opposite local node of the shared face
            for (int el = 0; el < ne; ++el) {
                if (mate[el] >= 0) continue;
                for (int h = 0; h < nbn[el]; ++h) {
                    const auto &pr = nbv[(size_t)4 * el + h];
                    if (mate[pr.first] < 0) {
                        mate[el] = pr.first;
                        mate[pr.first] = el;
                        tri[el] = pr.second;
                        for (int h2 = 0; h2 < nbn[pr.first]; ++h2)
                            if (nbv[(size_t)4 * pr.first + h2].first == el) tri[pr.first] = nbv[(size_t)4 * pr.first + h2].second;
                        break;
                    }
                }
            }
            // records: face pairs first, then the others two by two
            inc.clear();
            std::vector<int> rest;
            int n_fp = 0;
            std::vector<std::pair<int, int>> pairs;
            for (int el = 0; el < ne; ++el) {
                if (mate[el] < 0)
                    rest.push_back(el);
                else if (mate[el] > el) {
                    // B = (f1, f0, f2, b) must be positive too (b across the face from a)
                    int32_t f[3], j = 0;
                    for (int a = 0; a < 4; ++a)
                        if (a != tri[el]) f[j++] = node(el, a);
                    int32_t v[4] = {f[0], f[1], f[2], node(el, tri[el])};
                    if (!(det4(v) > 0.0)) std::swap(v[0], v[1]);
                    const int32_t w[4] = {v[1], v[0], v[2], node(mate[el], tri[mate[el]])};
                    if (det4(w) > 0.0) {
                        pairs.push_back({el, mate[el]});
                    } else {
                        rest.push_back(el);
                        rest.push_back(mate[el]);
                    }
                }
            }
            std::sort(rest.begin(), rest.end());
            n_fp = (int)pairs.size();
            std::vector<int32_t> recnodes;   // 8 node ids per record (-1 unused)
            int pos = 0;
            for (auto &pr : pairs) {
                const int A = pr.first, Bq = pr.second;
                int32_t f[3], j = 0;
                for (int a = 0; a < 4; ++a)
                    if (a != tri[A]) f[j++] = node(A, a);
                int32_t v[4] = {f[0], f[1], f[2], node(A, tri[A])};
                if (!(det4(v) > 0.0)) std::swap(v[0], v[1]);
                const int32_t bb = node(Bq, tri[Bq]);
                for (int a = 0; a < 4; ++a) recnodes.push_back(v[a]);
                recnodes.push_back(bb);
                for (int a = 0; a < 3; ++a) recnodes.push_back(-1);
                eorig[(size_t)(e0 + pos)] = orig_h[(size_t)(e0 + A)];
                eorig[(size_t)(e0 + pos + 1)] = orig_h[(size_t)(e0 + Bq)];
                pos += 2;
            }
            for (size_t i = 0; i < rest.size(); i += 2) {
                for (int h = 0; h < 2; ++h) {
                    if (i + h < rest.size()) {
                        const int el = rest[i + h];
                        for (int a = 0; a < 4; ++a) recnodes.push_back(node(el, a));
                        eorig[(size_t)(e0 + pos + h)] = orig_h[(size_t)(e0 + el)];
                    } else
                        for (int a = 0; a < 4; ++a) recnodes.push_back(-1);
                }
                pos += 2;
            }
            const int nrec = (int)(recnodes.size() / 8);
            uniq.clear();
            for (int32_t v : recnodes)
                if (v >= 0) uniq.push_back(v);
            std::sort(uniq.begin(), uniq.end());
            uniq.erase(std::unique(uniq.begin(), uniq.end()), uniq.end());
            const int L = (int)uniq.size();
            const int Lp = (L + 3) & ~3;
            if (Lp > 1024) {
                fits = false;
                break;
            }
            lmp = std::max(lmp, Lp);
            auto lof = [&](int32_t id) { return (int)(std::lower_bound(uniq.begin(), uniq.end(), id) - uniq.begin()); };
            lcount.assign(L, 0);
            for (int32_t v : recnodes)
                if (v >= 0) lcount[lof(v)]++;
            // local order: decreasing slot count (similar loop lengths in a reducer warp)
            order.resize(L);
            for (int l = 0; l < L; ++l) order[l] = l;
            std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return lcount[x] > lcount[y]; });
            lrank.resize(L);
            for (int l = 0; l < L; ++l) lrank[order[l]] = l;
            // slot (node l, its t-th incidence) at toff[t] + l: toff[t + 1] - toff[t]
            // = number of nodes with more than t slots (a prefix of the order)
            {
                uint32_t *to = &toff[(size_t)k * 68];
                int hist[68] = {};
                for (int l = 0; l < L; ++l) hist[std::min(lcount[l], 67)]++;
                int above = L;   // nodes with more than t slots
                to[0] = 0u;
                for (int t = 0; t < 67; ++t) {
                    above -= hist[t];
                    to[t + 1] = to[t] + (uint32_t)above;
                }
            }
            fill.assign(L, 0);
            for (int r = 0; r < nrec && fits; ++r) {
                uint32_t v[8] = {0, 0, 0, 0, 0, 0, 0, 0};
                for (int a = 0; a < 8; ++a) {
                    const int32_t id = recnodes[(size_t)8 * r + a];
                    if (id < 0) continue;
                    const int l = lrank[lof(id)];
                    const int rk = fill[l]++;
                    if (rk >= 64) fits = false;
                    v[a] = (uint32_t)l | ((uint32_t)rk << 10);
                }
                elem[(size_t)(k * R + r)] = make_uint4(v[0] | (v[1] << 16), v[2] | (v[3] << 16), v[4] | (v[5] << 16),
                                                       v[6] | (v[7] << 16));
            }
            const int32_t o = uniq[0];
            const double ox = X[o], oy = X[n + o], oz = X[2 * n + o];
            for (int l = 0; l < L; ++l) {
                const int32_t id = uniq[order[l]];
                recs.push_back(make_float4((float)(X[id] - ox), (float)(X[n + id] - oy), (float)(X[2 * n + id] - oz), 0.f));
                idv.push_back((uint32_t)id);
            }
            // a node is the chunk's own when all its element incidences lie in the chunk
            {
                std::vector<int> elinc(L, 0);
                for (int el = 0; el < ne; ++el)
                    for (int a = 0; a < 4; ++a) elinc[lrank[lof(node(el, a))]]++;
                for (int l = 0; l < L; ++l) {
                    uint32_t &w = idv[idv.size() - L + l];
                    if (elinc[l] != m.inc_total[(int32_t)w]) w |= 0x80000000u;
                }
            }
            for (int l = L; l < Lp; ++l) {
                recs.push_back(make_float4(0.f, 0.f, 0.f, 0.f));
                idv.push_back(0u);
            }
            nodes_n[(size_t)k] = L;
            nfp[(size_t)k] = n_fp;
            off[(size_t)k + 1] = off[(size_t)k] + Lp;
        }
        if (!fits || tet_ws_smem_bytes(nw, lmp) > kMaxBlockSmem) continue;
        CK(b.ws_off.alloc(off.size()));
        CK(b.ws_nodes.alloc(nodes_n.size()));
        CK(b.ws_nfp.alloc(nfp.size()));
        CK(b.ws_rec.alloc(recs.size()));
        CK(b.ws_ids.alloc(idv.size()));
        CK(b.ws_elem.alloc(elem.size()));
        CK(b.ws_eorig.alloc(eorig.size()));
        CK(b.ws_toff.alloc(toff.size()));
        CK(cudaMemcpy(b.ws_toff.p, toff.data(), toff.size() * 4, cudaMemcpyHostToDevice));
        CK(cudaMemcpy(b.ws_off.p, off.data(), off.size() * 8, cudaMemcpyHostToDevice));
        CK(cudaMemcpy(b.ws_nodes.p, nodes_n.data(), nodes_n.size() * 4, cudaMemcpyHostToDevice));
        CK(cudaMemcpy(b.ws_nfp.p, nfp.data(), nfp.size() * 4, cudaMemcpyHostToDevice));
        CK(cudaMemcpy(b.ws_rec.p, recs.data(), recs.size() * sizeof(float4), cudaMemcpyHostToDevice));
        CK(cudaMemcpy(b.ws_ids.p, idv.data(), idv.size() * 4, cudaMemcpyHostToDevice));
        CK(cudaMemcpy(b.ws_elem.p, elem.data(), elem.size() * sizeof(uint4), cudaMemcpyHostToDevice));
        CK(cudaMemcpy(b.ws_eorig.p, eorig.data(), eorig.size() * 4, cudaMemcpyHostToDevice));
        b.ws_nw = nw;
        b.ws_lmp = lmp;
        b.ws_nch = nch;
        return FEA_OK;
    }
    return FEA_OK;
}

// Greedy colouring of a category's elements in their (Morton) order
// (greedy_colour: each element takes the lowest colour that none of its
// nodes has seen yet, so no two elements of a colour share a node); the
// elements are then stored colour by colour (Morton order kept within a
// colour).
fea_status build_colours(fea_ctx *ctx, const Mesh &m, Bucket &b) {
    const int nen = kNen[b.etype];
    const int64_t cnt = b.count;
    std::vector<int32_t> col((size_t)cnt);
    const int n_col = greedy_colour(m.n, nen, cnt, b.conn_h.data(), 1, cnt, col.data());
    if (n_col < 0) return fail(ctx, FEA_EMESH, "colouring needs more than %d colours", kColourMax);
    std::vector<int64_t> off((size_t)n_col + 1, 0);
    for (int64_t e = 0; e < cnt; ++e) off[(size_t)col[(size_t)e] + 1]++;
    for (int c = 0; c < n_col; ++c) off[(size_t)c + 1] += off[(size_t)c];
    std::vector<int64_t> pos(off.begin(), off.end() - 1);
    std::vector<int32_t> perm((size_t)cnt);
    for (int64_t e = 0; e < cnt; ++e) perm[(size_t)pos[(size_t)col[(size_t)e]]++] = (int32_t)e;
    std::vector<int32_t> cc((size_t)nen * cnt), corig((size_t)cnt), orig_h((size_t)cnt);
    CK(cudaMemcpy(orig_h.data(), b.orig.p, sizeof(int32_t) * cnt, cudaMemcpyDeviceToHost));
    for (int64_t k = 0; k < cnt; ++k) {
        const int32_t e = perm[(size_t)k];
        for (int a = 0; a < nen; ++a) cc[(size_t)a * cnt + k] = b.conn_h[(size_t)a * cnt + e];
        corig[(size_t)k] = orig_h[(size_t)e];
    }
    CK(b.col_conn.alloc(cc.size()));
    CK(b.col_orig.alloc(corig.size()));
    CK(cudaMemcpy(b.col_conn.p, cc.data(), cc.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(b.col_orig.p, corig.data(), corig.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
    b.col_off = off;
    b.n_colours = n_col;
    return FEA_OK;
}

fea_status ensure_colours(fea_ctx *ctx, Mesh &m) {
    for (auto &bp : m.buckets) {
        if (bp->count == 0 || bp->col_conn.p) continue;
        fea_status st = build_colours(ctx, m, *bp);
        if (st) return st;
    }
    return FEA_OK;
}

fea_status ensure_chunks(fea_ctx *ctx, Mesh &m, int C) {
    for (auto &bp : m.buckets) {
        if (bp->count == 0 || (bp->lconn.p && bp->chunk_elems == C)) continue;
        fea_status st = build_chunks(ctx, m, *bp, C);
        if (st) return st;
    }
    return FEA_OK;
}

// Whether the FP64-Jacobian PEN06 category runs as a programmatic dependent
// of the persistent TET04 kernel on the caller's stream (it starts as that
// kernel's CTAs retire and fills its tail) instead of on a side stream: a
// mesh of exactly one TET04 category on the pipeline and one FP64-Jacobian
// PEN06 category, mixed precision, chunk plan, default forms, no MLP, no
// nu_t output.  Both orders overlap the two; only this one survives graph
// capture (a graph's branches were launched one after the other).
bool tail_order(const Mesh &m, fea_prec prec, fea_closure closure, fea_scatter scatter, bool want_nut) {
    if (prec != FEA_MIXED || scatter != FEA_SCATTER_CHUNK || closure == FEA_CLOSURE_MLP || want_nut ||
        m.conv_form != 0 || m.delta_form != 0 || m.plan.chunk_acc != 0)
        return false;
    int n_tet = 0, n_pen64 = 0, other = 0;
    for (auto &bp : m.buckets) {
        if (!bp->count) continue;
        if (bp->fp64j && bp->etype == FEA_PEN06 && bp->lconn.p)
            ++n_pen64;
        else if (!bp->fp64j && bp->etype == FEA_TET04 && bp->ws_rec.p)
            ++n_tet;
        else
            ++other;
    }
    return n_tet == 1 && n_pen64 == 1 && other == 0;
}

fea_status assemble_into(fea_ctx *ctx, Mesh &m, fea_prec prec, fea_closure closure, uint32_t mask,
                         fea_scatter scatter, double *rhs, float *nut, cudaStream_t s) {
    // the learned closure's last input is log(Delta^2 |G| / nu)
    if (closure == FEA_CLOSURE_MLP && !(m.nu > 0.0))
        return fail(ctx, FEA_EINVAL, "the MLP closure needs nu > 0 (its input is the element Reynolds number)");
    CK(cudaMemsetAsync(rhs, 0, sizeof(double) * 3 * m.n, s));
    FieldDev f = m.field();
    if (scatter == FEA_SCATTER_AUTO) scatter = (fea_scatter)m.plan.scatter;
    // the colour scatter's plain read-modify-writes need the categories one
    // after the other on one stream (the MLP closure keeps atomics)
    const bool colour = scatter == FEA_SCATTER_COLOUR && closure != FEA_CLOSURE_MLP;
    if (colour) {
        fea_status cs = ensure_colours(ctx, m);
        if (cs) return cs;
    }
    // FP64-Jacobian categories (FP64 pipe) go first, on a side stream, so
    // that they overlap the FP32-bound categories on the caller's stream;
    // or, in the tail order (tail_order; not while profiling per category),
    // after the TET04 kernel on the same stream as its programmatic dependent.
    const bool tail = !ctx->profiling && tail_order(m, prec, closure, scatter, nut != nullptr);
    bool forked = false;
    for (int pass = 0; pass < 2; ++pass) {
        for (auto &bp : m.buckets) {
            const Bucket &b = *bp;
            if (!b.count) continue;
            const bool first = tail ? !b.fp64j : (prec == FEA_MIXED && b.fp64j);
            if (first != (pass == 0)) continue;
            // while profiling per category every kernel runs alone on the
            // caller's stream, so its events time that kernel, not a share
            const bool side = !tail && first && !colour && !ctx->profiling;
            cudaStream_t ls = s;
            if (side) {
                if (!forked) {
                    CK(cudaEventRecord(ctx->ev_fork, s));
                    CK(cudaStreamWaitEvent(ctx->side, ctx->ev_fork, 0));
                    forked = true;
                }
                ls = ctx->side;
            }
            AsmArgs a;
            a.mask = mask;
            a.closure = closure;
            a.rhs = rhs;
            a.nut = nut ? nut + type_nut_offset(m, b.etype) : nullptr;
            a.err = ctx->d_err;
            a.mlp = closure == FEA_CLOSURE_MLP ? mlp_fast_ptr(ctx->mlp_w.p) : nullptr;
            a.mlp_fb = closure == FEA_CLOSURE_MLP ? ctx->mlp_fb.p : nullptr;
            a.pdl = tail && b.fp64j;
            a.wait_polls = ctx->wait_polls;
            cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
            if (ctx->profiling) CK(cudaStreamIsCapturing(s, &cap));
            ProfRec pr{b.etype, b.fp64j, nullptr, nullptr};
            const bool timed = ctx->profiling && cap == cudaStreamCaptureStatusNone;
            if (timed) {
                CK(cudaEventCreate(&pr.e0));
                CK(cudaEventCreate(&pr.e1));
                CK(cudaEventRecord(pr.e0, ls));
            }
            if (colour) {
                CK(launch_assemble_colour(b.dev(), f, a, prec, m.plan.threads_per_block, b.col_off.data(),
                                          b.n_colours, ls));
                ctx->launches += b.n_colours - 1;
            } else if (prec == FEA_MIXED && scatter == FEA_SCATTER_CHUNK && b.lconn.p)
                CK(launch_assemble_chunk(b.dev(), f, a, m.plan.threads_per_block, m.plan.chunk_acc, ls));
            else
                CK(launch_assemble_bucket(b.dev(), f, a, prec,
                                          scatter == FEA_SCATTER_WARP ? FEA_SCATTER_WARP : FEA_SCATTER_ATOMIC,
                                          m.plan.threads_per_block, ls));
            ctx->launches++;
            if (timed) {
                CK(cudaEventRecord(pr.e1, ls));
                ctx->prof.push_back(pr);
            }
        }
    }
    if (forked) {
        CK(cudaEventRecord(ctx->ev_join, ctx->side));
        CK(cudaStreamWaitEvent(s, ctx->ev_join, 0));
    }
    return FEA_OK;
}

fea_status check_args(fea_ctx *ctx, fea_prec prec, fea_closure closure, uint32_t mask) {
    if (prec != FEA_FP64 && prec != FEA_MIXED) return fail(ctx, FEA_EINVAL, "bad precision %d", (int)prec);
    if (closure != FEA_CLOSURE_NONE && closure != FEA_CLOSURE_VREMAN && closure != FEA_CLOSURE_MLP)
        return fail(ctx, FEA_EINVAL, "bad closure %d", (int)closure);
    if (closure == FEA_CLOSURE_MLP && !ctx->mlp_ready)
        return fail(ctx, FEA_ESTATE, "MLP closure requested before fea_mlp_load");
    if (mask & ~15u) return fail(ctx, FEA_EINVAL, "bad term mask 0x%x", mask);
    return FEA_OK;
}

// boundary assembly (Algorithm 1): the wall-model term at velocity u64 added
// to rhs; no-op without wall faces
fea_status add_wall_term(fea_ctx *ctx, const Mesh &m, const double *u64, double nu, double *rhs, fea_prec prec,
                         cudaStream_t s) {
    if (!m.wall_launches()) return FEA_OK;
    if (!(nu > 0.0)) return fail(ctx, FEA_EINVAL, "the wall model needs nu > 0");
    for (int k = 0; k < 2; ++k) {
        if (!m.wall_n[k]) continue;
        CK(launch_wall(m.wall_dev(k), m.xyz64.p, u64, m.n, nu, rhs, ctx->d_err, prec == FEA_FP64, s));
        ctx->launches++;
    }
    return FEA_OK;
}

fea_status rk_stage_impl(fea_ctx *ctx, Mesh &m, int stage, double dt, fea_prec prec, fea_closure closure,
                         cudaStream_t s) {
    static const double A[3] = {0.0, 0.75, 1.0 / 3.0};
    static const double B[3] = {1.0, 0.25, 2.0 / 3.0};
    fea_status st = assemble_into(ctx, m, prec, closure, FEA_TERM_ALL, FEA_SCATTER_AUTO, m.rhs.p, nullptr, s);
    if (st) return st;
    if ((st = add_wall_term(ctx, m, m.uk.p, m.nu, m.rhs.p, prec, s))) return st;
    if (m.slaves.n) {
        CK(launch_fold(m.slaves.p, m.masters.p, (int64_t)m.slaves.n, m.rhs.p, 3, m.n, s));
        ctx->launches += 2;
    }
    CK(launch_rk_update(m.n, m.un.p, m.uk.p, m.uk.p, stage == 2 ? m.un.p : nullptr, m.rhs.p, m.minv.p,
                        m.dirichlet.n ? m.dirichlet.p : nullptr, m.p64.p, m.up32.p, A[stage], B[stage], dt, s));
    ctx->launches++;
    return FEA_OK;
}

}  // namespace

// ---------------------------------------------------------------------------
// support for the allocation-free stage entry point (fea_noalloc.cu)

namespace fea {

int context_device(const fea_ctx *ctx) { return ctx ? ctx->device : -1; }

fea_status context_fail(fea_ctx *ctx, fea_status st, const char *msg) { return fail(ctx, st, "%s", msg); }

fea_status stage_with_scratch(fea_ctx *ctx, int32_t mesh, int32_t stage, double dt, fea_prec prec,
                              fea_closure closure, double nu, double c_vreman, const double *un, const double *uk,
                              const double *p, double *uk_out, double *rhs, float4 *up, int64_t max_nodes,
                              cudaStream_t s) {
    static const double A[3] = {0.0, 0.75, 1.0 / 3.0};
    static const double B[3] = {1.0, 0.25, 2.0 / 3.0};
    Mesh *m;
    fea_status st = get_mesh(ctx, mesh, &m);
    if (st) return st;
    if ((st = check_args(ctx, prec, closure, FEA_TERM_ALL))) return st;
    if (stage < 0 || stage > 2) return fail(ctx, FEA_EINVAL, "stage must be 0, 1 or 2");
    if (!(dt > 0.0)) return fail(ctx, FEA_EINVAL, "dt must be > 0");
    if (!(nu >= 0.0) || !(c_vreman >= 0.0)) return fail(ctx, FEA_EINVAL, "nu and c_vreman must be >= 0");
    if (closure == FEA_CLOSURE_MLP && !(nu > 0.0))
        return fail(ctx, FEA_EINVAL, "the MLP closure needs nu > 0 (its input is the element Reynolds number)");
    if (!un || !uk || !p || !uk_out) return fail(ctx, FEA_EINVAL, "null state array");
    if (closure == FEA_CLOSURE_MLP && !(nu > 0.0))
        return fail(ctx, FEA_EINVAL, "the MLP closure needs nu > 0 (its input is the element Reynolds number)");
    if (m->n > max_nodes)
        return fail(ctx, FEA_EINVAL, "mesh has %lld nodes, above the %lld-node limit of the static scratch",
                    (long long)m->n, (long long)max_nodes);
    const int64_t n = m->n;
    // FP32 copy of (u^(k), p) for the mixed kernels, in scratch
    CK(launch_pack_field(n, uk, p, up, s));
    FieldDev f;
    f.n = n;
    f.xyz64 = m->xyz64.p;
    f.xyz32 = m->xyz32.p;
    f.u64 = uk;
    f.p64 = p;
    f.up32 = up;
    f.nu = nu;
    f.c_vreman = c_vreman;
    CK(cudaMemsetAsync(rhs, 0, sizeof(double) * 3 * n, s));
    const fea_scatter scatter = (fea_scatter)m->plan.scatter;
    // colour tables are built by fea_set_plan / fea_autotune, never here
    const bool colour = scatter == FEA_SCATTER_COLOUR && closure != FEA_CLOSURE_MLP;
    if (colour)
        for (auto &bp : m->buckets)
            if (bp->count && !bp->col_conn.p) return fail(ctx, FEA_ESTATE, "colour tables missing (set the plan)");
    const bool tail = tail_order(*m, prec, closure, scatter, false);   // as in assemble_into
    bool forked = false;
    for (int pass = 0; pass < 2; ++pass) {
        for (auto &bp : m->buckets) {
            const Bucket &b = *bp;
            if (!b.count) continue;
            const bool first = tail ? !b.fp64j : (prec == FEA_MIXED && b.fp64j);
            if (first != (pass == 0)) continue;
            const bool side = !tail && first && !colour;
            cudaStream_t ls = s;
            if (side) {
                if (!forked) {
                    CK(cudaEventRecord(ctx->ev_fork, s));
                    CK(cudaStreamWaitEvent(ctx->side, ctx->ev_fork, 0));
                    forked = true;
                }
                ls = ctx->side;
            }
            AsmArgs a;
            a.mask = FEA_TERM_ALL;
            a.closure = closure;
            a.rhs = rhs;
            a.nut = nullptr;
            a.err = ctx->d_err;
            a.mlp = closure == FEA_CLOSURE_MLP ? mlp_fast_ptr(ctx->mlp_w.p) : nullptr;
            a.mlp_fb = closure == FEA_CLOSURE_MLP ? ctx->mlp_fb.p : nullptr;
            a.pdl = tail && b.fp64j;
            a.wait_polls = ctx->wait_polls;
            if (colour) {
                CK(launch_assemble_colour(b.dev(), f, a, prec, m->plan.threads_per_block, b.col_off.data(),
                                          b.n_colours, ls));
                ctx->launches += b.n_colours - 1;
            } else if (prec == FEA_MIXED && scatter == FEA_SCATTER_CHUNK && b.lconn.p)
                CK(launch_assemble_chunk(b.dev(), f, a, m->plan.threads_per_block, m->plan.chunk_acc, ls));
            else
                CK(launch_assemble_bucket(b.dev(), f, a, prec,
                                          scatter == FEA_SCATTER_WARP ? FEA_SCATTER_WARP : FEA_SCATTER_ATOMIC,
                                          m->plan.threads_per_block, ls));
            ctx->launches++;
        }
    }
    if (forked) {
        CK(cudaEventRecord(ctx->ev_join, ctx->side));
        CK(cudaStreamWaitEvent(s, ctx->ev_join, 0));
    }
    if ((st = add_wall_term(ctx, *m, uk, nu, rhs, prec, s))) return st;
    if (m->slaves.n) {
        CK(launch_fold(m->slaves.p, m->masters.p, (int64_t)m->slaves.n, rhs, 3, n, s));
        ctx->launches += 2;
    }
    CK(launch_rk_update(n, un, uk, uk_out, nullptr, rhs, m->minv.p, m->dirichlet.n ? m->dirichlet.p : nullptr, p, up,
                        A[stage], B[stage], dt, s));
    ctx->launches += 2;
    return FEA_OK;
}

}  // namespace fea

// ===========================================================================
extern "C" {

const char *fea_version(void) { return "libfea 0.1 (sm_103a)"; }

fea_status fea_create(int device, fea_ctx **out) {
    if (!out) return FEA_EINVAL;
    *out = nullptr;
    int count = 0;
    if (cudaGetDeviceCount(&count) != cudaSuccess || count == 0) {
        cudaGetLastError();
        return FEA_ECUDA;
    }
    if (device < 0 || device >= count) return FEA_EINVAL;
    auto ctx = new fea_ctx();
    ctx->device = device;
    fea_status st = FEA_OK;
    do {
        if (cudaSetDevice(device) != cudaSuccess) { st = FEA_ECUDA; break; }
        if (cudaDeviceGetAttribute(&ctx->sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) {
            st = FEA_ECUDA;
            break;
        }
        if (cudaMalloc(&ctx->d_err, sizeof(unsigned)) != cudaSuccess) { st = FEA_ENOMEM; break; }
        if (cudaMalloc(&ctx->d_bad, sizeof(unsigned long long)) != cudaSuccess) { st = FEA_ENOMEM; break; }
        if (cudaMemset(ctx->d_err, 0, sizeof(unsigned)) != cudaSuccess) { st = FEA_ECUDA; break; }
        if (cudaStreamCreateWithFlags(&ctx->capture, cudaStreamNonBlocking) != cudaSuccess) { st = FEA_ECUDA; break; }
        if (cudaStreamCreateWithFlags(&ctx->side, cudaStreamNonBlocking) != cudaSuccess) { st = FEA_ECUDA; break; }
        if (cudaEventCreateWithFlags(&ctx->ev_fork, cudaEventDisableTiming) != cudaSuccess) { st = FEA_ECUDA; break; }
        if (cudaEventCreateWithFlags(&ctx->ev_join, cudaEventDisableTiming) != cudaSuccess) { st = FEA_ECUDA; break; }
        RefTables t = make_tables();
        if (upload_ref_tables(t) != cudaSuccess) { st = FEA_ECUDA; break; }
        // the allocation-free stage's static scratch: its module is loaded
        // (and the array reserved) here, not at that entry point's first call
        void *scratch = nullptr;
        if (noalloc_scratch_address(device, &scratch) != cudaSuccess) { st = FEA_ECUDA; break; }
    } while (0);
    if (st != FEA_OK) {
        cudaGetLastError();
        fea_destroy(ctx);
        return st;
    }
    *out = ctx;
    return FEA_OK;
}

void fea_destroy(fea_ctx *ctx) {
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    ctx->meshes.clear();
    for (auto &r : ctx->prof) {
        cudaEventDestroy(r.e0);
        cudaEventDestroy(r.e1);
    }
    if (ctx->d_err) cudaFree(ctx->d_err);
    if (ctx->d_bad) cudaFree(ctx->d_bad);
    if (ctx->capture) cudaStreamDestroy(ctx->capture);
    if (ctx->side) cudaStreamDestroy(ctx->side);
    if (ctx->ev_fork) cudaEventDestroy(ctx->ev_fork);
    if (ctx->ev_join) cudaEventDestroy(ctx->ev_join);
    delete ctx;
}

const char *fea_last_error(const fea_ctx *ctx) { return ctx ? ctx->err.c_str() : "null context"; }

int64_t fea_launch_count(const fea_ctx *ctx) { return ctx ? ctx->launches : 0; }

fea_status fea_mesh_upload(fea_ctx *ctx, const fea_mesh_desc *d, void *stream, int32_t *mesh_id) {
    if (!ctx || !d || !mesh_id) return fail(ctx, FEA_EINVAL, "null argument");
    if (d->n_nodes <= 0 || d->n_nodes >= (int64_t)1 << 31 || !d->xyz)
        return fail(ctx, FEA_EINVAL, "n_nodes must be in [1, 2^31) with coordinates");
    cudaStream_t s = (cudaStream_t)stream;
    CK(cudaSetDevice(ctx->device));
    fea_status st_up = FEA_OK;
    const int64_t n = d->n_nodes;
    auto m = std::make_unique<Mesh>();
    m->n = n;
    // validation of connectivity (host)
    for (int t = 0; t < 4; ++t) {
        if (d->n_elem[t] < 0) return fail(ctx, FEA_EINVAL, "negative element count for type %d", t);
        if (d->n_elem[t] > 0 && !d->conn[t]) return fail(ctx, FEA_EINVAL, "missing connectivity for type %d", t);
        if (d->n_elem[t] >= (int64_t)1 << 31) return fail(ctx, FEA_EINVAL, "too many elements of type %d", t);
        const int nen = kNen[t];
        for (int64_t k = 0; k < d->n_elem[t] * nen; ++k) {
            const int32_t v = d->conn[t][k];
            if (v < 0 || v >= n)
                return fail(ctx, FEA_EMESH, "element %lld of type %d: node index %d out of range [0, %lld)",
                            (long long)(k / nen), t, v, (long long)n);
        }
        m->n_elem[t] = d->n_elem[t];
    }
    if (d->periodic_master)
        for (int64_t i = 0; i < n; ++i)
            if (d->periodic_master[i] < 0 || d->periodic_master[i] >= n)
                return fail(ctx, FEA_EMESH, "periodic master of node %lld out of range", (long long)i);
    // coordinates: bounding box for the Morton keys
    const double *X = d->xyz;
    double lo[3], hi[3];
    for (int i = 0; i < 3; ++i) {
        lo[i] = X[i * n];
        hi[i] = X[i * n];
    }
    for (int i = 0; i < 3; ++i)
        for (int64_t k = 0; k < n; ++k) {
            lo[i] = std::min(lo[i], X[i * n + k]);
            hi[i] = std::max(hi[i], X[i * n + k]);
        }
    double scale[3];
    for (int i = 0; i < 3; ++i) scale[i] = (hi[i] > lo[i]) ? double((1u << 21) - 1) / (hi[i] - lo[i]) : 0.0;
    // buckets: (type, fp64 flag), each sorted by the Morton key of the centroid
    for (int t = 0; t < 4; ++t) {
        const int64_t E = d->n_elem[t];
        if (!E) continue;
        const int nen = kNen[t];
        for (int flag = 0; flag < 2; ++flag) {
            std::vector<std::pair<uint64_t, int32_t>> keys;
            keys.reserve(flag ? 0 : E);
            for (int64_t e = 0; e < E; ++e) {
                const int fl = d->fp64_jac[t] ? (d->fp64_jac[t][e] ? 1 : 0) : 0;
                if (fl != flag) continue;
                double c[3] = {0, 0, 0};
                for (int a = 0; a < nen; ++a) {
                    const int32_t v = d->conn[t][e * nen + a];
                    for (int i = 0; i < 3; ++i) c[i] += X[i * n + v];
                }
                uint64_t key = 0;
                for (int i = 0; i < 3; ++i) {
                    double q = (c[i] / nen - lo[i]) * scale[i];
                    q = std::min(std::max(q, 0.0), double((1u << 21) - 1));
                    key |= morton_spread3((uint64_t)q) << i;
                }
                keys.emplace_back(key, (int32_t)e);
            }
            if (keys.empty()) continue;
            std::sort(keys.begin(), keys.end());
            const int64_t cnt = (int64_t)keys.size();
            std::vector<int32_t> conn((size_t)cnt * nen), orig((size_t)cnt);
            for (int64_t k = 0; k < cnt; ++k) {
                const int32_t e = keys[k].second;
                orig[k] = e;
                for (int a = 0; a < nen; ++a) conn[(size_t)a * cnt + k] = d->conn[t][(int64_t)e * nen + a];
            }
            auto b = std::make_unique<Bucket>();
            b->etype = t;
            b->fp64j = flag;
            b->count = cnt;
            b->conn_h = conn;
            CK(b->conn.alloc(conn.size()));
            CK(b->orig.alloc(orig.size()));
            CK(cudaMemcpy(b->conn.p, conn.data(), conn.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
            CK(cudaMemcpy(b->orig.p, orig.data(), orig.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
            m->buckets.push_back(std::move(b));
        }
    }
    // node arrays
    m->xyz_h.assign(X, X + 3 * n);
    m->inc_total.assign((size_t)n, 0);
    for (int t = 0; t < 4; ++t)
        for (int64_t k = 0; k < d->n_elem[t] * kNen[t]; ++k) m->inc_total[d->conn[t][k]]++;
    CK(m->xyz64.alloc(3 * n));
    CK(cudaMemcpy(m->xyz64.p, X, sizeof(double) * 3 * n, cudaMemcpyHostToDevice));
    {
        std::vector<float4> x32((size_t)n);
        for (int64_t k = 0; k < n; ++k)
            x32[k] = make_float4((float)X[k], (float)X[n + k], (float)X[2 * n + k], 0.0f);
        CK(m->xyz32.alloc(n));
        CK(cudaMemcpy(m->xyz32.p, x32.data(), sizeof(float4) * n, cudaMemcpyHostToDevice));
    }
    if (d->periodic_master) {
        m->master_h.assign(d->periodic_master, d->periodic_master + n);
        std::vector<int32_t> sl, ms;
        for (int64_t i = 0; i < n; ++i)
            if (d->periodic_master[i] != i) {
                sl.push_back((int32_t)i);
                ms.push_back(d->periodic_master[i]);
            }
        if (!sl.empty()) {
            CK(m->slaves.alloc(sl.size()));
            CK(m->masters.alloc(ms.size()));
            CK(cudaMemcpy(m->slaves.p, sl.data(), sl.size() * 4, cudaMemcpyHostToDevice));
            CK(cudaMemcpy(m->masters.p, ms.data(), ms.size() * 4, cudaMemcpyHostToDevice));
        }
    }
    if (d->dirichlet) {
        CK(m->dirichlet.alloc(n));
        CK(cudaMemcpy(m->dirichlet.p, d->dirichlet, n, cudaMemcpyHostToDevice));
    }
    // lumped mass + det J validation (FP64)
    CK(m->mass.alloc(n));
    CK(m->minv.alloc(n));
    CK(cudaMemsetAsync(m->mass.p, 0, sizeof(double) * n, s));
    CK(cudaMemsetAsync(ctx->d_err, 0, sizeof(unsigned), s));
    for (auto &bp : m->buckets) {
        CK(cudaMemsetAsync(ctx->d_bad, 0xFF, sizeof(unsigned long long), s));
        CK(launch_lumped_mass(bp->dev(), m->xyz64.p, n, m->mass.p, ctx->d_err, ctx->d_bad, s));
        ctx->launches++;
        unsigned long long bad = ~0ull;
        CK(cudaMemcpyAsync(&bad, ctx->d_bad, sizeof bad, cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        if (bad != ~0ull) {
            std::vector<int32_t> o(1);
            CK(cudaMemcpy(o.data(), bp->orig.p + bad, 4, cudaMemcpyDeviceToHost));
            cudaMemset(ctx->d_err, 0, sizeof(unsigned));
            return fail(ctx, FEA_EMESH, "element %d of type %d has det J <= 0 at a Gauss point", o[0], bp->etype);
        }
    }
    // folded reciprocal mass for the RK stages
    {
        DevBuf<double> folded;
        CK(folded.alloc(n));
        CK(cudaMemcpyAsync(folded.p, m->mass.p, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
        if (m->slaves.n) CK(launch_fold(m->slaves.p, m->masters.p, (int64_t)m->slaves.n, folded.p, 1, n, s));
        CK(launch_recip(folded.p, m->minv.p, n, s));
        CK(cudaStreamSynchronize(s));
    }
    if ((st_up = ensure_chunks(ctx, *m, m->plan.chunk_elems))) return st_up;
    for (auto &bp : m->buckets)
        if ((st_up = build_ws_tables(ctx, *m, *bp, ws_warps_for(m->plan.threads_per_block)))) return st_up;
    CK(m->un.alloc(3 * n));
    CK(m->uk.alloc(3 * n));
    CK(m->p64.alloc(n));
    CK(m->rhs.alloc(3 * n));
    CK(m->up32.alloc(n));
    ctx->meshes.push_back(std::move(m));
    *mesh_id = (int32_t)ctx->meshes.size() - 1;
    return FEA_OK;
}

fea_status fea_mesh_info(fea_ctx *ctx, int32_t mesh, int64_t *n_nodes, int64_t n_elem[4]) {
    Mesh *m;
    fea_status st = get_mesh(ctx, mesh, &m);
    if (st) return st;
    if (n_nodes) *n_nodes = m->n;
    if (n_elem)
        for (int t = 0; t < 4; ++t) n_elem[t] = m->n_elem[t];
    return FEA_OK;
}

fea_status fea_lumped_mass(fea_ctx *ctx, int32_t mesh, double *out, void *stream) {
    Mesh *m;
    fea_status st = get_mesh(ctx, mesh, &m);
    if (st) return st;
    if (!out) return fail(ctx, FEA_EINVAL, "null output");
    CK(cudaMemcpyAsync(out, m->mass.p, sizeof(double) * m->n, cudaMemcpyDefault, (cudaStream_t)stream));
    return FEA_OK;
}

fea_status fea_field_upload(fea_ctx *ctx, int32_t mesh, const void *u, const void *p, int dtype, double nu,
                            double c_vreman, void *stream) {
    Mesh *m;
    fea_status st = get_mesh(ctx, mesh, &m);
    if (st) return st;
    if (!u || !p) return fail(ctx, FEA_EINVAL, "null field");
    if (dtype != 0 && dtype != 1) return fail(ctx, FEA_EINVAL, "dtype must be 0 (f64) or 1 (f32)");
    if (!(nu >= 0.0) || !(c_vreman >= 0.0)) return fail(ctx, FEA_EINVAL, "nu and c_vreman must be >= 0");
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t n = m->n;
    if (dtype == 0) {
        CK(cudaMemcpyAsync(m->uk.p, u, sizeof(double) * 3 * n, cudaMemcpyDefault, s));
        CK(cudaMemcpyAsync(m->p64.p, p, sizeof(double) * n, cudaMemcpyDefault, s));
    } else {
        if (m->stage_f32.n < (size_t)(4 * n)) CK(m->stage_f32.alloc(4 * n));
        CK(cudaMemcpyAsync(m->stage_f32.p, u, sizeof(float) * 3 * n, cudaMemcpyDefault, s));
        CK(cudaMemcpyAsync(m->stage_f32.p + 3 * n, p, sizeof(float) * n, cudaMemcpyDefault, s));
        CK(launch_f32_to_f64(m->stage_f32.p, m->uk.p, 3 * n, s));
        CK(launch_f32_to_f64(m->stage_f32.p + 3 * n, m->p64.p, n, s));
        ctx->launches += 2;
    }
    CK(cudaMemcpyAsync(m->un.p, m->uk.p, sizeof(double) * 3 * n, cudaMemcpyDeviceToDevice, s));
    CK(launch_pack_field(n, m->uk.p, m->p64.p, m->up32.p, s));
    ctx->launches++;
    m->nu = nu;
    m->c_vreman = c_vreman;
    m->has_field = true;
    return FEA_OK;
}

fea_status fea_assemble_rhs(fea_ctx *ctx, int32_t mesh, fea_prec prec, fea_closure closure, uint32_t mask,
                            fea_scatter scatter, double *rhs_out, float *nut_out, void *stream) {
    Mesh *m;
    fea_status st = get_mesh(ctx, mesh, &m);
    if (st) return st;
    if ((st = check_args(ctx, prec, closure, mask))) return st;
    if (!rhs_out) return fail(ctx, FEA_EINVAL, "null rhs_out");
    if (scatter < FEA_SCATTER_AUTO || scatter > FEA_SCATTER_WARP) return fail(ctx, FEA_EINVAL, "bad scatter");
    if (!m->has_field) return fail(ctx, FEA_ESTATE, "no field uploaded for mesh %d", mesh);
    return assemble_into(ctx, *m, prec, closure, mask, scatter, rhs_out, nut_out, (cudaStream_t)stream);
}

fea_status fea_assemble_rhs_batched(fea_ctx *ctx, const int32_t *meshes, int32_t n, fea_prec prec,
                                    fea_closure closure, uint32_t mask, double *const *rhs_out, void *stream) {
    if (!ctx || !meshes || !rhs_out || n <= 0) return fail(ctx, FEA_EINVAL, "bad batch arguments");
    fea_status st = check_args(ctx, prec, closure, mask);
    if (st) return st;
    bool tables = prec == FEA_MIXED;
    for (int32_t k = 0; k < n; ++k) {
        Mesh *m;
        if ((st = get_mesh(ctx, meshes[k], &m))) return st;
        if (!m->has_field) return fail(ctx, FEA_ESTATE, "no field uploaded for mesh %d", meshes[k]);
        if (!rhs_out[k]) return fail(ctx, FEA_EINVAL, "null rhs_out[%d]", k);
        for (auto &b : m->buckets)
            if (b->count && (!b->lconn.p || (b->fp64j && b->etype != FEA_PEN06))) tables = false;
    }
    cudaStream_t s = (cudaStream_t)stream;
    if (!tables || ctx->batch_per_mesh) {  // per-mesh launches (FP64 path, or the autotuner's choice)
        for (int32_t k = 0; k < n; ++k) {
            Mesh *m = ctx->meshes[meshes[k]].get();
            const fea_scatter sc = !tables ? FEA_SCATTER_ATOMIC : FEA_SCATTER_AUTO;
            st = assemble_into(ctx, *m, prec, closure, mask, sc, rhs_out[k], nullptr, s);
            if (st) return st;
        }
        return FEA_OK;
    }
    // descriptor tables: one entry per (mesh, category); items ordered by
    // per-element cost (FP64-Jacobian, then HEX08, PYR05, PEN06, TET04)
    std::vector<BucketDev> bk;
    std::vector<FieldDev> fd;
    std::vector<AsmArgs> ag;
    std::vector<double *> rp((size_t)n);
    std::vector<int64_t> rl((size_t)n);
    size_t smem = 0;
    for (int32_t k = 0; k < n; ++k) {
        Mesh *m = ctx->meshes[meshes[k]].get();
        rp[k] = rhs_out[k];
        rl[k] = 3 * m->n;
        for (auto &b : m->buckets) {
            if (!b->count) continue;
            bk.push_back(b->dev());
            fd.push_back(m->field());
            AsmArgs a;
            a.mask = mask;
            a.closure = closure;
            a.rhs = rhs_out[k];
            a.nut = nullptr;
            a.err = ctx->d_err;
            a.mlp = closure == FEA_CLOSURE_MLP ? mlp_fast_ptr(ctx->mlp_w.p) : nullptr;
            a.mlp_fb = closure == FEA_CLOSURE_MLP ? ctx->mlp_fb.p : nullptr;
            ag.push_back(a);
            smem = std::max(smem, chunk_smem_bytes(bk.back()));
        }
    }
    auto cost = [](const BucketDev &b) { return b.fp64j ? 100 : kNen[b.etype] * kNg[b.etype]; };
    std::vector<int32_t> order(bk.size());
    for (size_t i = 0; i < order.size(); ++i) order[i] = (int32_t)i;
    std::stable_sort(order.begin(), order.end(), [&](int32_t x, int32_t y) { return cost(bk[x]) > cost(bk[y]); });
    std::vector<int32_t> items;
    for (int32_t bi : order)
        for (int64_t c = 0; c < bk[bi].n_chunks; ++c) {
            items.push_back(bi);
            items.push_back((int32_t)c);
        }
    const int64_t n_items = (int64_t)items.size() / 2;
    if (smem > kChunkSmemLimit) return fail(ctx, FEA_EINVAL, "batched chunk needs more than 200 KB of shared memory");
    if (closure == FEA_CLOSURE_MLP && ((smem + 127) & ~(size_t)127) + mlp_smem_bytes(128, kMaxNg) > kMaxBlockSmem)
        return fail(ctx, FEA_EINVAL, "batched chunk with the MLP closure needs more than 227 KB of shared memory");
    auto grow = [&](DevBuf<unsigned char> &d, size_t bytes) -> cudaError_t {
        return d.n >= bytes ? cudaSuccess : d.alloc(bytes);
    };
    CK(grow(ctx->batch_bk, bk.size() * sizeof(BucketDev)));
    CK(grow(ctx->batch_fd, fd.size() * sizeof(FieldDev)));
    CK(grow(ctx->batch_ag, ag.size() * sizeof(AsmArgs)));
    CK(grow(ctx->batch_items, items.size() * sizeof(int32_t)));
    if (ctx->batch_rhs.n < (size_t)n) CK(ctx->batch_rhs.alloc(n));
    if (ctx->batch_len.n < (size_t)n) CK(ctx->batch_len.alloc(n));
    if (!ctx->batch_counter.n) CK(ctx->batch_counter.alloc(1));
    CK(cudaMemcpyAsync(ctx->batch_bk.p, bk.data(), bk.size() * sizeof(BucketDev), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(ctx->batch_fd.p, fd.data(), fd.size() * sizeof(FieldDev), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(ctx->batch_ag.p, ag.data(), ag.size() * sizeof(AsmArgs), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(ctx->batch_items.p, items.data(), items.size() * sizeof(int32_t), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(ctx->batch_rhs.p, rp.data(), n * sizeof(double *), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(ctx->batch_len.p, rl.data(), n * sizeof(int64_t), cudaMemcpyHostToDevice, s));
    CK(launch_zero_batch(ctx->batch_rhs.p, ctx->batch_len.p, n, s));
    ProfRec pr{4, 0, nullptr, nullptr};
    if (ctx->profiling) {
        CK(cudaEventCreate(&pr.e0));
        CK(cudaEventCreate(&pr.e1));
        CK(cudaEventRecord(pr.e0, s));
    }
    bool variants = false;
    for (int32_t k = 0; k < n; ++k) {
        const Mesh *m = ctx->meshes[meshes[k]].get();
        variants |= m->conv_form != 0 || m->delta_form != 0;
    }
    CK(launch_assemble_batch(ctx->batch_bk.p, ctx->batch_fd.p, ctx->batch_ag.p, ctx->batch_items.p, n_items,
                             ctx->batch_counter.p, smem, ctx->sms, closure == FEA_CLOSURE_MLP, variants, s));
    if (ctx->profiling) {
        CK(cudaEventRecord(pr.e1, s));
        ctx->prof.push_back(pr);
    }
    ctx->launches += 2;
    return FEA_OK;
}

fea_status fea_periodic_fold(fea_ctx *ctx, int32_t mesh, double *v, int32_t ncomp, void *stream) {
    Mesh *m;
    fea_status st = get_mesh(ctx, mesh, &m);
    if (st) return st;
    if (!v || ncomp < 1 || ncomp > 16) return fail(ctx, FEA_EINVAL, "bad fold arguments");
    if (!m->slaves.n) return FEA_OK;
    CK(launch_fold(m->slaves.p, m->masters.p, (int64_t)m->slaves.n, v, ncomp, m->n, (cudaStream_t)stream));
    ctx->launches += 2;
    return FEA_OK;
}

fea_status fea_rk_stage(fea_ctx *ctx, int32_t mesh, int32_t stage, double dt, fea_prec prec, fea_closure closure,
                        void *stream) {
    Mesh *m;
    fea_status st = get_mesh(ctx, mesh, &m);
    if (st) return st;
    if ((st = check_args(ctx, prec, closure, FEA_TERM_ALL))) return st;
    if (stage < 0 || stage > 2) return fail(ctx, FEA_EINVAL, "stage must be 0, 1 or 2");
    if (!(dt > 0.0)) return fail(ctx, FEA_EINVAL, "dt must be > 0");
    if (!m->has_field) return fail(ctx, FEA_ESTATE, "no field uploaded for mesh %d", mesh);
    return rk_stage_impl(ctx, *m, stage, dt, prec, closure, (cudaStream_t)stream);
}

fea_status fea_rk_step_graph(fea_ctx *ctx, int32_t mesh, double dt, fea_prec prec, fea_closure closure,
                             void *stream) {
    Mesh *m;
    fea_status st = get_mesh(ctx, mesh, &m);
    if (st) return st;
    if ((st = check_args(ctx, prec, closure, FEA_TERM_ALL))) return st;
    if (!(dt > 0.0)) return fail(ctx, FEA_EINVAL, "dt must be > 0");
    if (!m->has_field) return fail(ctx, FEA_ESTATE, "no field uploaded for mesh %d", mesh);
    GraphCache &g = m->graph;
    if (!g.exec || g.dt != dt || g.prec != prec || g.closure != closure) {
        if (g.exec) {
            cudaGraphExecDestroy(g.exec);
            g.exec = nullptr;
        }
        CK(cudaStreamSynchronize((cudaStream_t)stream));
        cudaGraph_t graph;
        const int64_t before = ctx->launches;
        CK(cudaStreamBeginCapture(ctx->capture, cudaStreamCaptureModeThreadLocal));
        for (int k = 0; k < 3 && st == FEA_OK; ++k) st = rk_stage_impl(ctx, *m, k, dt, prec, closure, ctx->capture);
        cudaError_t e = cudaStreamEndCapture(ctx->capture, &graph);
        ctx->launches = before;
        if (st) return st;
        CK(e);
        e = cudaGraphInstantiate(&g.exec, graph, 0);
        cudaGraphDestroy(graph);
        CK(e);
        g.dt = dt;
        g.prec = prec;
        g.closure = closure;
    }
    CK(cudaGraphLaunch(g.exec, (cudaStream_t)stream));
    // kernels per step: 3 x (buckets + wall faces + fold 2 + update 1)
    int64_t per_stage = 1 + (m->slaves.n ? 2 : 0) + m->wall_launches();
    const bool colour = m->plan.scatter == FEA_SCATTER_COLOUR && closure != FEA_CLOSURE_MLP;
    for (auto &b : m->buckets) per_stage += b->count ? (colour ? b->n_colours : 1) : 0;
    ctx->launches += 3 * per_stage;
    return FEA_OK;
}

fea_status fea_state_download(fea_ctx *ctx, int32_t mesh, double *out, void *stream) {
    Mesh *m;
    fea_status st = get_mesh(ctx, mesh, &m);
    if (st) return st;
    if (!out) return fail(ctx, FEA_EINVAL, "null output");
    if (!m->has_field) return fail(ctx, FEA_ESTATE, "no field uploaded for mesh %d", mesh);
    CK(cudaMemcpyAsync(out, m->uk.p, sizeof(double) * 3 * m->n, cudaMemcpyDefault, (cudaStream_t)stream));
    return FEA_OK;
}

fea_status fea_get_plan(fea_ctx *ctx, int32_t mesh, fea_plan *plan) {
    Mesh *m;
    fea_status st = get_mesh(ctx, mesh, &m);
    if (st) return st;
    if (!plan) return fail(ctx, FEA_EINVAL, "null plan");
    *plan = m->plan;
    return FEA_OK;
}

fea_status fea_set_plan(fea_ctx *ctx, int32_t mesh, const fea_plan *plan) {
    Mesh *m;
    fea_status st = get_mesh(ctx, mesh, &m);
    if (st) return st;
    if (!plan) return fail(ctx, FEA_EINVAL, "null plan");
    if (plan->scatter != FEA_SCATTER_ATOMIC && plan->scatter != FEA_SCATTER_CHUNK &&
        plan->scatter != FEA_SCATTER_COLOUR && plan->scatter != FEA_SCATTER_WARP)
        return fail(ctx, FEA_EINVAL, "plan scatter must be ATOMIC, CHUNK, COLOUR or WARP");
    if (plan->scatter == FEA_SCATTER_COLOUR && (st = ensure_colours(ctx, *m))) return st;
    if (plan->threads_per_block < 32 || plan->threads_per_block > 1024 || plan->threads_per_block % 32)
        return fail(ctx, FEA_EINVAL, "threads_per_block must be a multiple of 32 in [32, 1024]");
    if (plan->scatter == FEA_SCATTER_CHUNK) {
        if (plan->chunk_elems < 32 || plan->chunk_elems > 4096 || plan->chunk_elems % 32)
            return fail(ctx, FEA_EINVAL, "chunk_elems must be a multiple of 32 in [32, 4096]");
        if (plan->chunk_acc != 0 && plan->chunk_acc != 1) return fail(ctx, FEA_EINVAL, "chunk_acc must be 0 or 1");
        if ((st = ensure_chunks(ctx, *m, plan->chunk_elems))) return st;
        for (auto &b : m->buckets)
            if (b->count && chunk_kernel_smem(b->dev(), plan->chunk_acc) > kChunkSmemLimit)
                return fail(ctx, FEA_EINVAL, "chunk of %d elements needs more than 220 KB of shared memory",
                            plan->chunk_elems);
        for (auto &b : m->buckets)
            if ((st = build_ws_tables(ctx, *m, *b, ws_warps_for(plan->threads_per_block)))) return st;
    }
    m->plan = *plan;
    if (m->graph.exec) {
        cudaGraphExecDestroy(m->graph.exec);
        m->graph.exec = nullptr;
    }
    return FEA_OK;
}

fea_status fea_autotune(fea_ctx *ctx, int32_t mesh, fea_prec prec, fea_closure closure, const char *cache_path) {
    Mesh *m;
    fea_status st = get_mesh(ctx, mesh, &m);
    if (st) return st;
    if ((st = check_args(ctx, prec, closure, FEA_TERM_ALL))) return st;
    if (!m->has_field) return fail(ctx, FEA_ESTATE, "no field uploaded for mesh %d", mesh);
    // cache key: device name and mesh statistics, then precision and closure
    std::string key;
    if (cache_path) {
        cudaDeviceProp prop;
        CK(cudaGetDeviceProperties(&prop, ctx->device));
        std::string dev(prop.name);
        for (char &ch : dev)
            if (ch == ' ' || ch == '\t') ch = '_';
        char buf[640];
        snprintf(buf, sizeof buf, "%s|nodes=%lld|elems=%lld,%lld,%lld,%lld|prec=%d|closure=%d", dev.c_str(),
                 (long long)m->n, (long long)m->n_elem[0], (long long)m->n_elem[1], (long long)m->n_elem[2],
                 (long long)m->n_elem[3], (int)prec, (int)closure);
        key = buf;
        if (FILE *f = fopen(cache_path, "r")) {
            char line[1024];
            fea_plan cached{};
            bool hit = false;
            while (fgets(line, sizeof line, f)) {
                char k[700];
                fea_plan p{};
                if (sscanf(line, "%699s %d %d %d %d", k, &p.scatter, &p.threads_per_block, &p.chunk_elems,
                           &p.chunk_acc) == 5 &&
                    key == k) {
                    cached = p;   // the last entry for a key wins
                    hit = true;
                }
            }
            fclose(f);
            if (hit) return fea_set_plan(ctx, mesh, &cached);
        }
    }
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    fea_plan best = m->plan, best_chunk{};
    float best_ms = 1e30f, best_chunk_ms = 1e30f;
    std::vector<fea_plan> cands;
    for (int t : {128, 256}) cands.push_back(fea_plan{FEA_SCATTER_ATOMIC, t, m->plan.chunk_elems, 0});
    for (int t : {128, 256}) cands.push_back(fea_plan{FEA_SCATTER_WARP, t, m->plan.chunk_elems, 0});
    if (closure != FEA_CLOSURE_MLP) {
        if ((st = ensure_colours(ctx, *m))) return st;
        for (int t : {128, 256}) cands.push_back(fea_plan{FEA_SCATTER_COLOUR, t, m->plan.chunk_elems, 0});
    }
    if (prec == FEA_MIXED)
        for (int C : {256, 512, 1024})
            for (int t : {128, 256, 512})
                if (t <= C) cands.push_back(fea_plan{FEA_SCATTER_CHUNK, t, C, m->plan.chunk_acc});
    for (const fea_plan &cand : cands) {
        if (cand.scatter == FEA_SCATTER_CHUNK) {
            if ((st = ensure_chunks(ctx, *m, cand.chunk_elems))) return st;
            for (auto &b : m->buckets)
                if ((st = build_ws_tables(ctx, *m, *b, ws_warps_for(cand.threads_per_block)))) return st;
            bool fits = true;
            for (auto &b : m->buckets)
                if (b->count && (chunk_kernel_smem(b->dev(), cand.chunk_acc) > kChunkSmemLimit ||
                                 (closure == FEA_CLOSURE_MLP &&
                                  chunk_launch_smem(b->dev(), cand.threads_per_block, cand.chunk_acc, true) >
                                      kMaxBlockSmem)))
                    fits = false;
            if (!fits) continue;
        }
        m->plan = cand;
        for (int rep = 0; rep < 2; ++rep)
            if ((st = assemble_into(ctx, *m, prec, closure, FEA_TERM_ALL, FEA_SCATTER_AUTO, m->rhs.p, nullptr, 0)))
                return st;
        CK(cudaEventRecord(e0, 0));
        for (int rep = 0; rep < 5; ++rep)
            if ((st = assemble_into(ctx, *m, prec, closure, FEA_TERM_ALL, FEA_SCATTER_AUTO, m->rhs.p, nullptr, 0)))
                return st;
        CK(cudaEventRecord(e1, 0));
        CK(cudaEventSynchronize(e1));
        float ms = 0;
        CK(cudaEventElapsedTime(&ms, e0, e1));
        if (ms < best_ms) {
            best_ms = ms;
            best = cand;
        }
        if (cand.scatter == FEA_SCATTER_CHUNK && ms < best_chunk_ms) {
            best_chunk_ms = ms;
            best_chunk = cand;
        }
    }
    // near-ties go to the chunk scatter: its chunk-relative FP32 coordinates
    // keep edge vectors at full FP32 precision (about 3x smaller mixed-
    // precision error than the global FP32 coordinates of the other paths)
    if (best.scatter != FEA_SCATTER_CHUNK && best_chunk_ms <= 1.05f * best_ms) {
        best = best_chunk;
        best_ms = best_chunk_ms;
    }
    if (best.scatter == FEA_SCATTER_CHUNK) {
        if ((st = ensure_chunks(ctx, *m, best.chunk_elems))) return st;
        for (auto &b : m->buckets)
            if ((st = build_ws_tables(ctx, *m, *b, ws_warps_for(best.threads_per_block)))) return st;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (cache_path) {
        FILE *f = fopen(cache_path, "a");
        if (!f) return fail(ctx, FEA_EINVAL, "cannot append to autotune cache %s", cache_path);
        fprintf(f, "%s %d %d %d %d %.6f\n", key.c_str(), best.scatter, best.threads_per_block, best.chunk_elems,
                best.chunk_acc, (double)best_ms / 5.0);
        fclose(f);
    }
    m->plan = best;
    if (m->graph.exec) {
        cudaGraphExecDestroy(m->graph.exec);
        m->graph.exec = nullptr;
    }
    return FEA_OK;
}

fea_status fea_autotune_batched(fea_ctx *ctx, const int32_t *meshes, int32_t n, fea_prec prec, fea_closure closure,
                                fea_plan *best_out) {
    if (!ctx || !meshes || n <= 0) return fail(ctx, FEA_EINVAL, "bad batch arguments");
    fea_status st = check_args(ctx, prec, closure, FEA_TERM_ALL);
    if (st) return st;
    std::vector<Mesh *> ms((size_t)n);
    for (int32_t k = 0; k < n; ++k) {
        if ((st = get_mesh(ctx, meshes[k], &ms[(size_t)k]))) return st;
        if (!ms[(size_t)k]->has_field) return fail(ctx, FEA_ESTATE, "no field uploaded for mesh %d", meshes[k]);
    }
    // candidates: the persistent batched launch over chunk tables of C
    // elements (CHUNK), or per-mesh launches with one of the other scatters
    std::vector<fea_plan> cands;
    if (prec == FEA_MIXED)
        for (int C : {128, 256, 512}) cands.push_back(fea_plan{FEA_SCATTER_CHUNK, 256, C, 0});
    cands.push_back(fea_plan{FEA_SCATTER_ATOMIC, 256, 256, 0});
    cands.push_back(fea_plan{FEA_SCATTER_WARP, 256, 256, 0});
    if (closure != FEA_CLOSURE_MLP) cands.push_back(fea_plan{FEA_SCATTER_COLOUR, 128, 256, 0});
    std::vector<double *> rhs((size_t)n);
    for (int32_t k = 0; k < n; ++k) rhs[(size_t)k] = ms[(size_t)k]->rhs.p;
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    fea_plan best{};
    float best_ms = 1e30f;
    for (const fea_plan &cand : cands) {
        bool ok = true;
        for (int32_t k = 0; k < n; ++k) {
            fea_plan p = ms[(size_t)k]->plan;
            p.scatter = cand.scatter;
            p.threads_per_block = cand.threads_per_block;
            if (cand.scatter == FEA_SCATTER_CHUNK) p.chunk_elems = cand.chunk_elems;
            if (fea_set_plan(ctx, meshes[k], &p) != FEA_OK) ok = false;   // e.g. a chunk too large for shared memory
        }
        if (!ok) continue;
        ctx->batch_per_mesh = cand.scatter != FEA_SCATTER_CHUNK;
        for (int rep = 0; rep < 2; ++rep)
            if ((st = fea_assemble_rhs_batched(ctx, meshes, n, prec, closure, FEA_TERM_ALL, rhs.data(), 0))) return st;
        CK(cudaEventRecord(e0, 0));
        for (int rep = 0; rep < 5; ++rep)
            if ((st = fea_assemble_rhs_batched(ctx, meshes, n, prec, closure, FEA_TERM_ALL, rhs.data(), 0))) return st;
        CK(cudaEventRecord(e1, 0));
        CK(cudaEventSynchronize(e1));
        float ms_ = 0;
        CK(cudaEventElapsedTime(&ms_, e0, e1));
        if (ms_ < best_ms) {
            best_ms = ms_;
            best = cand;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (best_ms >= 1e30f) return fail(ctx, FEA_EINVAL, "no batch candidate fits");
    for (int32_t k = 0; k < n; ++k) {
        fea_plan p = ms[(size_t)k]->plan;
        p.scatter = best.scatter;
        p.threads_per_block = best.threads_per_block;
        if (best.scatter == FEA_SCATTER_CHUNK) p.chunk_elems = best.chunk_elems;
        if ((st = fea_set_plan(ctx, meshes[k], &p))) return st;
    }
    ctx->batch_per_mesh = best.scatter != FEA_SCATTER_CHUNK;
    if (best_out) *best_out = best;
    return FEA_OK;
}

fea_status fea_mlp_load(fea_ctx *ctx, const float *theta, const float *feat_mean, const float *feat_std,
                        double out_scale, void *stream) {
    if (!ctx) return FEA_EINVAL;
    if (!theta || !feat_mean || !feat_std) return fail(ctx, FEA_EINVAL, "null MLP argument");
    if (!(out_scale > 0.0)) return fail(ctx, FEA_EINVAL, "out_scale must be > 0");
    for (int k = 0; k < 6; ++k) {
        float sd = 0.f;
        CK(cudaMemcpy(&sd, feat_std + k, sizeof(float), cudaMemcpyDefault));
        if (!(sd > 0.f)) return fail(ctx, FEA_EINVAL, "feature std must be > 0");
    }
    cudaStream_t s = (cudaStream_t)stream;
    const int np = mlp_param_count();
    if (!ctx->mlp_theta.n) {
        CK(ctx->mlp_theta.alloc(np));
        CK(ctx->mlp_m1.alloc(np));
        CK(ctx->mlp_m2.alloc(np));
        CK(ctx->mlp_grad.alloc(np));
        CK(ctx->mlp_loss.alloc(1));
        CK(ctx->mlp_norm.alloc(24));   // mean[6], std[6], envelope lo[6], hi[6]
        CK(ctx->mlp_w.alloc(mlp_weights_bytes()));
        CK(ctx->mlp_fb.alloc(1));
        CK(cudaMemsetAsync(ctx->mlp_fb.p, 0, sizeof(unsigned long long), s));
    }
    CK(cudaMemcpyAsync(ctx->mlp_theta.p, theta, sizeof(float) * np, cudaMemcpyDefault, s));
    CK(cudaMemcpyAsync(ctx->mlp_norm.p, feat_mean, sizeof(float) * 6, cudaMemcpyDefault, s));
    CK(cudaMemcpyAsync(ctx->mlp_norm.p + 6, feat_std, sizeof(float) * 6, cudaMemcpyDefault, s));
    // a new network starts without an envelope
    static const float open_env[12] = {-INFINITY, -INFINITY, -INFINITY, -INFINITY, -INFINITY, -INFINITY,
                                       INFINITY,  INFINITY,  INFINITY,  INFINITY,  INFINITY,  INFINITY};
    CK(cudaMemcpyAsync(ctx->mlp_norm.p + 12, open_env, sizeof(open_env), cudaMemcpyHostToDevice, s));
    CK(cudaStreamSynchronize(s));   // open_env and the caller's arrays are read before returning
    CK(cudaMemsetAsync(ctx->mlp_m1.p, 0, sizeof(float) * np, s));
    CK(cudaMemsetAsync(ctx->mlp_m2.p, 0, sizeof(float) * np, s));
    CK(launch_mlp_pack(ctx->mlp_theta.p, ctx->mlp_norm.p, ctx->mlp_norm.p + 6, (float)out_scale, ctx->mlp_w.p, s));
    ctx->launches++;
    ctx->mlp_step = 0;
    ctx->mlp_scale = out_scale;
    ctx->mlp_ready = true;
    return FEA_OK;
}

fea_status fea_set_model(fea_ctx *ctx, int32_t mesh, int32_t conv_form, int32_t delta_form) {
    Mesh *m;
    fea_status st = get_mesh(ctx, mesh, &m);
    if (st) return st;
    if (conv_form != FEA_CONV_GU && conv_form != FEA_CONV_EMAC) return fail(ctx, FEA_EINVAL, "unknown convective form");
    if (delta_form != FEA_DELTA_VOLUME && delta_form != FEA_DELTA_AXES)
        return fail(ctx, FEA_EINVAL, "unknown filter-width form");
    m->conv_form = conv_form;
    m->delta_form = delta_form;
    if (m->graph.exec) {   // a captured step holds the old field descriptor
        cudaGraphExecDestroy(m->graph.exec);
        m->graph.exec = nullptr;
    }
    return FEA_OK;
}

// ---- boundary assembly: wall model ---------------------------------------------

fea_status fea_wall_setup(fea_ctx *ctx, int32_t mesh, const fea_wall_desc *d) {
    Mesh *m;
    fea_status st = get_mesh(ctx, mesh, &m);
    if (st) return st;
    if (!d) return fail(ctx, FEA_EINVAL, "null wall descriptor");
    if (d->n_tri < 0 || d->n_quad < 0 || (d->n_tri && (!d->tri || !d->tri_exch)) ||
        (d->n_quad && (!d->quad || !d->quad_exch)))
        return fail(ctx, FEA_EINVAL, "bad wall face arrays");
    if (!(d->kappa > 0.0) || !(d->c_plus >= 0.0)) return fail(ctx, FEA_EINVAL, "need kappa > 0 and c_plus >= 0");
    CK(cudaSetDevice(ctx->device));
    const int64_t n = m->n;
    const double *X = m->xyz_h.data();   // [3][n]
    const int64_t cnt[2] = {d->n_tri, d->n_quad};
    const int32_t *fs[2] = {d->tri, d->quad}, *xs[2] = {d->tri_exch, d->quad_exch};
    std::vector<int32_t> soa_f[2], soa_x[2];
    for (int k = 0; k < 2; ++k) {
        const int nv = k ? 4 : 3;
        soa_f[k].resize((size_t)nv * cnt[k]);
        soa_x[k].resize((size_t)nv * cnt[k]);
        // face Gauss points of the same rules as the kernel (geometry check only)
        const double a6 = 1.0 / 6.0, b6 = 2.0 / 3.0, q = 1.0 / sqrt(3.0);
        const double gp[4][2] = {{k ? -q : a6, k ? -q : a6}, {k ? q : b6, k ? -q : a6}, {k ? q : a6, k ? q : b6},
                                 {-q, q}};
        for (int64_t f = 0; f < cnt[k]; ++f) {
            int32_t fa[4], ex[4];
            for (int a = 0; a < nv; ++a) {
                fa[a] = fs[k][f * nv + a];
                ex[a] = xs[k][f * nv + a];
                if (fa[a] < 0 || fa[a] >= n || ex[a] < 0 || ex[a] >= n)
                    return fail(ctx, FEA_EMESH, "wall face %lld: node id out of range", (long long)f);
                soa_f[k][(size_t)a * cnt[k] + f] = fa[a];
                soa_x[k][(size_t)a * cnt[k] + f] = ex[a];
            }
            for (int g = 0; g < nv; ++g) {
                double N[4], dN[4][2];
                const double xi = gp[g][0], eta = gp[g][1];
                if (nv == 3) {
                    N[0] = 1 - xi - eta, N[1] = xi, N[2] = eta;
                    dN[0][0] = -1, dN[0][1] = -1, dN[1][0] = 1, dN[1][1] = 0, dN[2][0] = 0, dN[2][1] = 1;
                } else {
                    const double sx[4] = {-1, 1, 1, -1}, sy[4] = {-1, -1, 1, 1};
                    for (int a = 0; a < 4; ++a) {
                        N[a] = 0.25 * (1 + sx[a] * xi) * (1 + sy[a] * eta);
                        dN[a][0] = 0.25 * sx[a] * (1 + sy[a] * eta);
                        dN[a][1] = 0.25 * sy[a] * (1 + sx[a] * xi);
                    }
                }
                double t1[3] = {0, 0, 0}, t2[3] = {0, 0, 0}, dx[3] = {0, 0, 0};
                for (int a = 0; a < nv; ++a)
                    for (int i = 0; i < 3; ++i) {
                        t1[i] += dN[a][0] * X[i * n + fa[a]];
                        t2[i] += dN[a][1] * X[i * n + fa[a]];
                        dx[i] += N[a] * (X[i * n + ex[a]] - X[i * n + fa[a]]);
                    }
                const double nr[3] = {t1[1] * t2[2] - t1[2] * t2[1], t1[2] * t2[0] - t1[0] * t2[2],
                                      t1[0] * t2[1] - t1[1] * t2[0]};
                const double y = -(dx[0] * nr[0] + dx[1] * nr[1] + dx[2] * nr[2]);   // times |nr|
                const double area2 = nr[0] * nr[0] + nr[1] * nr[1] + nr[2] * nr[2];
                if (!(area2 > 0.0) || !(y > 0.0))
                    return fail(ctx, FEA_EMESH,
                                "wall face %lld: degenerate, or its exchange point is not on the fluid side "
                                "(face normal must point out of the fluid)",
                                (long long)f);
            }
        }
    }
    for (int k = 0; k < 2; ++k) {
        m->wall_n[k] = 0;
        CK(m->wall_face[k].alloc(soa_f[k].size()));
        CK(m->wall_exch[k].alloc(soa_x[k].size()));
        if (cnt[k]) {
            CK(cudaMemcpy(m->wall_face[k].p, soa_f[k].data(), soa_f[k].size() * 4, cudaMemcpyHostToDevice));
            CK(cudaMemcpy(m->wall_exch[k].p, soa_x[k].data(), soa_x[k].size() * 4, cudaMemcpyHostToDevice));
        }
        m->wall_n[k] = cnt[k];
    }
    m->wall_kappa = d->kappa;
    m->wall_c = d->c_plus;
    if (m->graph.exec) {   // a captured step lacks (or holds stale) wall launches
        cudaGraphExecDestroy(m->graph.exec);
        m->graph.exec = nullptr;
    }
    return FEA_OK;
}

fea_status fea_wall_assemble(fea_ctx *ctx, int32_t mesh, double *rhs, void *stream) {
    Mesh *m;
    fea_status st = get_mesh(ctx, mesh, &m);
    if (st) return st;
    if (!rhs) return fail(ctx, FEA_EINVAL, "null rhs");
    if (!m->has_field) return fail(ctx, FEA_ESTATE, "no field uploaded for mesh %d", mesh);
    return add_wall_term(ctx, *m, m->uk.p, m->nu, rhs, FEA_FP64, (cudaStream_t)stream);
}

// ---- pressure projection -----------------------------------------------------

fea_status fea_poisson_setup(fea_ctx *ctx, int32_t mesh, const uint8_t *pinned, void *stream) {
    Mesh *m;
    fea_status st = get_mesh(ctx, mesh, &m);
    if (st) return st;
    cudaStream_t s = (cudaStream_t)stream;
    CK(cudaSetDevice(ctx->device));
    PoissonBuild pb;
    pb.n = m->n;
    for (auto &b : m->buckets)
        if (b->count) {
            pb.conn.push_back(b->conn_h.data());
            pb.count.push_back(b->count);
            pb.nen.push_back(kNen[b->etype]);
        }
    pb.class_of = m->master_h.empty() ? nullptr : m->master_h.data();
    pb.pinned = pinned;
    if (m->poisson) {
        CK(cudaDeviceSynchronize());
        poisson_free(m->poisson);
        m->poisson = nullptr;
    }
    CK(poisson_build(pb, ctx->sms, &m->poisson));
    CK(cudaMemsetAsync(ctx->d_err, 0, sizeof(unsigned), s));
    for (auto &b : m->buckets) {
        CK(launch_lap_assemble(b->dev(), m->xyz64.p, m->n, poisson_cls(m->poisson), poisson_rowptr(m->poisson),
                               poisson_col(m->poisson), poisson_val(m->poisson), ctx->d_err, s));
        ctx->launches += b->count ? 1 : 0;
    }
    CK(poisson_finish(m->poisson, ctx->d_err, ctx->sms, s));
    ctx->launches += 2;
    if (!m->proj_b.n) {
        CK(m->proj_b.alloc(m->n));
        CK(m->proj_dp.alloc(m->n));
        CK(m->proj_g.alloc(3 * m->n));
    }
    unsigned w = 0;
    CK(cudaMemcpyAsync(&w, ctx->d_err, sizeof w, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (w) {
        CK(cudaMemsetAsync(ctx->d_err, 0, sizeof(unsigned), s));
        poisson_free(m->poisson);
        m->poisson = nullptr;
        return fail(ctx, FEA_EMESH, "Laplacian assembly failed (device word 0x%x)", w);
    }
    return FEA_OK;
}

fea_status fea_poisson_solve(fea_ctx *ctx, int32_t mesh, const double *b, double scale, double *x, double rtol,
                             int32_t max_iter, int32_t *iters, double *rel_res, void *stream) {
    Mesh *m;
    fea_status st = get_mesh(ctx, mesh, &m);
    if (st) return st;
    if (!m->poisson) return fail(ctx, FEA_ESTATE, "fea_poisson_setup has not run for mesh %d", mesh);
    if (!b || !x || !(rtol > 0.0) || max_iter < 0) return fail(ctx, FEA_EINVAL, "bad Poisson solve arguments");
    CK(cudaSetDevice(ctx->device));
    int it = 0;
    double rr = 0.0;
    CK(poisson_solve(m->poisson, b, scale, x, rtol, max_iter, ctx->sms, (cudaStream_t)stream, &it, &rr,
                     &ctx->launches));
    if (iters) *iters = it;
    if (rel_res) *rel_res = rr;
    return FEA_OK;
}

namespace {
fea_status divgrad(fea_ctx *ctx, int32_t mesh, bool div, const double *in, double *out, cudaStream_t s) {
    Mesh *m;
    fea_status st = get_mesh(ctx, mesh, &m);
    if (st) return st;
    if (!in || !out) return fail(ctx, FEA_EINVAL, "null array");
    CK(cudaSetDevice(ctx->device));
    CK(cudaMemsetAsync(out, 0, sizeof(double) * (div ? 1 : 3) * m->n, s));
    for (auto &b : m->buckets) {
        CK(launch_divgrad_assemble(b->dev(), m->xyz64.p, m->n, div, in, out, ctx->d_err, s));
        ctx->launches += b->count ? 1 : 0;
    }
    return FEA_OK;
}
}  // namespace

fea_status fea_divergence(fea_ctx *ctx, int32_t mesh, const double *u, double *out, void *stream) {
    return divgrad(ctx, mesh, true, u, out, (cudaStream_t)stream);
}

fea_status fea_gradient(fea_ctx *ctx, int32_t mesh, const double *p, double *out, void *stream) {
    return divgrad(ctx, mesh, false, p, out, (cudaStream_t)stream);
}

fea_status fea_project(fea_ctx *ctx, int32_t mesh, double dt, double rtol, int32_t max_iter, int32_t *iters,
                       double *rel_res, void *stream) {
    Mesh *m;
    fea_status st = get_mesh(ctx, mesh, &m);
    if (st) return st;
    if (!m->has_field) return fail(ctx, FEA_ESTATE, "no field uploaded for mesh %d", mesh);
    if (!m->poisson) return fail(ctx, FEA_ESTATE, "fea_poisson_setup has not run for mesh %d", mesh);
    if (!(dt > 0.0)) return fail(ctx, FEA_EINVAL, "dt must be > 0");
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t n = m->n;
    // b = B(u*);  K dp = -(1/dt) b;  g = G(dp), folded;  u -= dt g / M;  p += dp
    if ((st = divgrad(ctx, mesh, true, m->uk.p, m->proj_b.p, s))) return st;
    CK(cudaMemsetAsync(m->proj_dp.p, 0, sizeof(double) * n, s));
    if ((st = fea_poisson_solve(ctx, mesh, m->proj_b.p, -1.0 / dt, m->proj_dp.p, rtol, max_iter, iters, rel_res,
                                stream)))
        return st;
    if ((st = divgrad(ctx, mesh, false, m->proj_dp.p, m->proj_g.p, s))) return st;
    if (m->slaves.n) {
        CK(launch_fold(m->slaves.p, m->masters.p, (int64_t)m->slaves.n, m->proj_g.p, 3, n, s));
        ctx->launches += 2;
    }
    CK(launch_project_update(n, m->uk.p, m->un.p, m->proj_g.p, m->minv.p, m->dirichlet.n ? m->dirichlet.p : nullptr,
                             m->p64.p, m->proj_dp.p, m->up32.p, dt, ctx->sms, s));
    ctx->launches++;
    return FEA_OK;
}

fea_status fea_interface_pack(fea_ctx *ctx, const double *v, int64_t n, const int64_t *loc, const int64_t *cls,
                              int64_t m, double *out, int64_t n_class, void *stream) {
    if (!ctx) return FEA_EINVAL;
    if (n < 0 || m < 0 || n_class < 0 || (m > 0 && (!v || !loc || !cls)) || (n_class > 0 && !out))
        return fail(ctx, FEA_EINVAL, "bad interface pack arguments");
    CK(cudaSetDevice(ctx->device));
    CK(launch_iface_pack(v, n, loc, cls, m, out, n_class, ctx->d_err, ctx->sms, (cudaStream_t)stream));
    ctx->launches += m > 0 ? 1 : 0;
    return FEA_OK;
}

fea_status fea_interface_unpack(fea_ctx *ctx, const double *in, int64_t n_class, const int64_t *loc,
                                const int64_t *cls, int64_t m, double *v, int64_t n, void *stream) {
    if (!ctx) return FEA_EINVAL;
    if (n < 0 || m < 0 || n_class < 0 || (m > 0 && (!v || !loc || !cls || !in)))
        return fail(ctx, FEA_EINVAL, "bad interface unpack arguments");
    CK(cudaSetDevice(ctx->device));
    CK(launch_iface_unpack(in, n_class, loc, cls, m, v, n, ctx->d_err, ctx->sms, (cudaStream_t)stream));
    ctx->launches += m > 0 ? 1 : 0;
    return FEA_OK;
}

fea_status fea_mlp_set_envelope(fea_ctx *ctx, const float *lo, const float *hi, void *stream) {
    if (!ctx) return FEA_EINVAL;
    if (!ctx->mlp_ready) return fail(ctx, FEA_ESTATE, "no MLP loaded");
    if ((lo == nullptr) != (hi == nullptr)) return fail(ctx, FEA_EINVAL, "envelope needs both bounds or neither");
    float env[12];
    for (int k = 0; k < 6; ++k) {
        env[k] = lo ? lo[k] : -INFINITY;
        env[6 + k] = hi ? hi[k] : INFINITY;
        if (env[k] != env[k] || env[6 + k] != env[6 + k]) return fail(ctx, FEA_EINVAL, "NaN envelope bound");
    }
    cudaStream_t s = (cudaStream_t)stream;
    CK(cudaMemcpyAsync(ctx->mlp_norm.p + 12, env, sizeof(env), cudaMemcpyHostToDevice, s));
    CK(launch_mlp_pack(ctx->mlp_theta.p, ctx->mlp_norm.p, ctx->mlp_norm.p + 6, (float)ctx->mlp_scale, ctx->mlp_w.p, s));
    ctx->launches++;
    CK(cudaStreamSynchronize(s));   // env is a host stack array
    return FEA_OK;
}

fea_status fea_mlp_fallback_read(fea_ctx *ctx, int64_t *points, int reset) {
    if (!ctx || !points) return ctx ? fail(ctx, FEA_EINVAL, "null output") : FEA_EINVAL;
    if (!ctx->mlp_ready) return fail(ctx, FEA_ESTATE, "no MLP loaded");
    unsigned long long v = 0;
    CK(cudaSetDevice(ctx->device));
    CK(cudaDeviceSynchronize());
    CK(cudaMemcpy(&v, ctx->mlp_fb.p, sizeof(v), cudaMemcpyDeviceToHost));
    if (reset) CK(cudaMemset(ctx->mlp_fb.p, 0, sizeof(v)));
    *points = (int64_t)v;
    return FEA_OK;
}

fea_status fea_mlp_get(fea_ctx *ctx, float *theta_out, void *stream) {
    if (!ctx) return FEA_EINVAL;
    if (!theta_out) return fail(ctx, FEA_EINVAL, "null output");
    if (!ctx->mlp_ready) return fail(ctx, FEA_ESTATE, "no MLP loaded");
    CK(cudaMemcpyAsync(theta_out, ctx->mlp_theta.p, sizeof(float) * mlp_param_count(), cudaMemcpyDefault,
                       (cudaStream_t)stream));
    return FEA_OK;
}

fea_status fea_mlp_forward(fea_ctx *ctx, const float *x, int64_t B, float *nut, void *stream) {
    if (!ctx) return FEA_EINVAL;
    if (B < 0 || (B > 0 && (!x || !nut))) return fail(ctx, FEA_EINVAL, "bad MLP forward arguments");
    if (!ctx->mlp_ready) return fail(ctx, FEA_ESTATE, "no MLP loaded");
    CK(launch_mlp_forward(ctx->mlp_w.p, x, B, nut, ctx->sms, ctx->d_err, (cudaStream_t)stream));
    ctx->launches++;
    return FEA_OK;
}

fea_status fea_mlp_train_step(fea_ctx *ctx, const float *x, const float *y, int64_t B, float lr, float *loss_out,
                              float *grad_out, void *stream) {
    if (!ctx) return FEA_EINVAL;
    if (!x || !y || B <= 0 || !(lr >= 0.f)) return fail(ctx, FEA_EINVAL, "bad MLP training arguments");
    if (!ctx->mlp_ready) return fail(ctx, FEA_ESTATE, "no MLP loaded");
    cudaStream_t s = (cudaStream_t)stream;
    const int np = mlp_param_count();
    CK(cudaMemsetAsync(ctx->mlp_grad.p, 0, sizeof(float) * np, s));
    CK(cudaMemsetAsync(ctx->mlp_loss.p, 0, sizeof(float), s));
    CK(launch_mlp_train(ctx->mlp_w.p, x, y, B, ctx->mlp_grad.p, ctx->mlp_loss.p, s));
    if (grad_out) CK(cudaMemcpyAsync(grad_out, ctx->mlp_grad.p, sizeof(float) * np, cudaMemcpyDefault, s));
    if (loss_out) CK(cudaMemcpyAsync(loss_out, ctx->mlp_loss.p, sizeof(float), cudaMemcpyDefault, s));
    ctx->mlp_step++;
    CK(launch_adam(ctx->mlp_theta.p, ctx->mlp_grad.p, ctx->mlp_m1.p, ctx->mlp_m2.p, np, lr, 0.9f, 0.999f, 1e-8f,
                   ctx->mlp_step, s));
    CK(launch_mlp_pack(ctx->mlp_theta.p, ctx->mlp_norm.p, ctx->mlp_norm.p + 6, (float)ctx->mlp_scale,
                       ctx->mlp_w.p, s));
    ctx->launches += 3;
    return FEA_OK;
}

fea_status fea_profile_enable(fea_ctx *ctx, int on) {
    if (!ctx) return FEA_EINVAL;
    ctx->profiling = on != 0;
    return FEA_OK;
}

fea_status fea_profile_read(fea_ctx *ctx, int etype, int fp64_jac, double *total_ms, int64_t *launches, int reset) {
    if (!ctx || !total_ms || !launches) return fail(ctx, FEA_EINVAL, "null argument");
    double ms = 0.0;
    int64_t cnt = 0;
    for (auto &r : ctx->prof) {
        if (r.etype != etype || r.fp64j != fp64_jac) continue;
        CK(cudaEventSynchronize(r.e1));
        float t = 0.0f;
        CK(cudaEventElapsedTime(&t, r.e0, r.e1));
        ms += t;
        ++cnt;
    }
    *total_ms = ms;
    *launches = cnt;
    if (reset) {
        for (auto &r : ctx->prof) {
            cudaEventDestroy(r.e0);
            cudaEventDestroy(r.e1);
        }
        ctx->prof.clear();
    }
    return FEA_OK;
}

fea_status fea_fp32_peak(fea_ctx *ctx, double *tflops_ffma, double *tflops_ffma2, void *stream) {
    if (!ctx) return FEA_EINVAL;
    if (!tflops_ffma || !tflops_ffma2) return fail(ctx, FEA_EINVAL, "null output");
    CK(measure_fp32_peak(ctx->sms, (cudaStream_t)stream, tflops_ffma, tflops_ffma2));
    ctx->launches += 8;
    return FEA_OK;
}

fea_status fea_set_wait_limit(fea_ctx *ctx, uint32_t polls) {
    if (!ctx) return FEA_EINVAL;
    ctx->wait_polls = polls;
    for (auto &m : ctx->meshes)
        if (m && m->graph.exec) {
            cudaGraphExecDestroy(m->graph.exec);
            m->graph.exec = nullptr;
        }
    return FEA_OK;
}

fea_status fea_sync_status(fea_ctx *ctx, void *stream) {
    if (!ctx) return FEA_EINVAL;
    CK(cudaStreamSynchronize((cudaStream_t)stream));
    unsigned w = 0;
    CK(cudaMemcpy(&w, ctx->d_err, sizeof w, cudaMemcpyDeviceToHost));
    CK(cudaMemset(ctx->d_err, 0, sizeof(unsigned)));
    if (w & ERR_TIMEOUT) return fail(ctx, FEA_ETIMEOUT, "a bounded device wait gave up (word 0x%x)", w);
    if (w & (ERR_DETJ | ERR_INDEX)) return fail(ctx, FEA_EMESH, "device saw det J <= 0 or a bad index (word 0x%x)", w);
    if (w & ERR_WALL_GEOM)
        return fail(ctx, FEA_EMESH, "wall model: degenerate face or exchange point off the fluid side (word 0x%x)", w);
    if (w & ERR_NONFINITE) return fail(ctx, FEA_ENUMERIC, "non-finite element residual (word 0x%x)", w);
    if (w & ERR_WALL_NEWTON) return fail(ctx, FEA_ENUMERIC, "wall model: u_tau iteration did not converge (word 0x%x)", w);
    return FEA_OK;
}

}  // extern "C"
