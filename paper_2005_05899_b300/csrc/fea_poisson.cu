// Pressure equation of the fractional step (Algorithm 1: "element assembly
// of the Laplacian matrix" once, then per time step "solution of the
// pressure equation with the preconditioned CG"; section 2.1: CG with Jacobi
// diagonal scaling).  The system lives on periodic classes (a node with its
// periodic copies is one unknown); classes marked as pinned carry a zero
// solution (their rows and columns become those of the identity), which
// removes the constant null space of the pure-Neumann / periodic problem.
//
// Host: the CSR pattern over classes (from the element connectivity).
// Device (FP64): the values are assembled by the element kernels into the
// CSR matrix and copied once into a sliced-ELLPACK matrix (32-row slices,
// column-major within a slice) for the iteration; one CG
// iteration is three kernels (SpMV + dot, update of x, r, z + two dots,
// update of p), the dot products finished by the last block of each kernel
// in a fixed order (deterministic), the iteration stopped by a device flag
// when ||r|| <= rtol ||b||; the host checks the flag between short batches
// of iterations and never launches more than max_iter.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <string>
#include <vector>

#include "fea_internal.h"

namespace fea {

namespace {

template <typename T>
cudaError_t dalloc(T **p, size_t n) {
    *p = nullptr;
    return n ? cudaMalloc(reinterpret_cast<void **>(p), sizeof(T) * n) : cudaSuccess;
}

constexpr int kThreads = 256;
// device scalars
enum { S_PQ = 0, S_RZ0 = 1, S_RZ1 = 2, S_RR = 3, S_BB = 4, S_COUNT = 8 };

__device__ __forceinline__ double block_sum(double v, double *sh) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) sh[w] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x < 32) {
        t = threadIdx.x < (blockDim.x >> 5) ? sh[threadIdx.x] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    }
    __syncthreads();
    return t;   // valid in thread 0
}

// Each block stores its partial sums (NV of them); the last block to finish
// adds the partials in block order and returns true in all of its threads.
template <int NV>
__device__ bool finish_partials(const double (&v)[NV], double *partial, unsigned *ticket, double *sums) {
    __shared__ double sh[32];
    __shared__ bool last;
    for (int k = 0; k < NV; ++k) {
        const double t = block_sum(v[k], sh);
        if (threadIdx.x == 0) partial[k * gridDim.x + blockIdx.x] = t;
    }
    __threadfence();
    if (threadIdx.x == 0) last = atomicAdd(ticket, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!last) return false;
    __threadfence();
    // the whole last block adds the partials: strided per thread, then the
    // block tree (a fixed order for a fixed grid, so the sums are reproducible)
    for (int k = 0; k < NV; ++k) {
        double t = 0.0;
        for (unsigned b = threadIdx.x; b < gridDim.x; b += blockDim.x)
            t += ((volatile double *)partial)[k * gridDim.x + b];
        t = block_sum(t, sh);
        if (threadIdx.x == 0) sums[k] = t;
    }
    if (threadIdx.x == 0) *ticket = 0u;
    __syncthreads();
    return true;
}

// q = A p, scal[S_PQ] = p.q.  Sliced ELLPACK: slice s holds rows 32 s ..
// 32 s + 31, entry j of the slice's rows at sell_off[s] + 32 j + lane (padding:
// value 0, column = the row), width sell_w[s].  A warp is one slice: one row
// per lane, coalesced value / column loads, the width's gathers independent.
__global__ void __launch_bounds__(kThreads) k_cg_spmv(const int64_t *sell_off, const int32_t *sell_w,
                                                      const int32_t *col, const double *val, const double *p,
                                                      double *q, int64_t nc, double *scal, double *partial,
                                                      unsigned *ticket, const int *done) {
    if (*done) return;
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t nslices = (nc + 31) >> 5;
    double dot = 0.0;
    for (int64_t sl = warp; sl < nslices; sl += warps) {
        const int64_t row = (sl << 5) + lane;
        const int64_t off = __ldg(&sell_off[sl]) + lane;
        const int w = __ldg(&sell_w[sl]);
        double acc = 0.0;
#pragma unroll 4
        for (int j = 0; j < w; ++j) {
            const int64_t k = off + ((int64_t)j << 5);
            acc += __ldg(&val[k]) * __ldg(&p[__ldg(&col[k])]);
        }
        if (row < nc) {
            q[row] = acc;
            dot += p[row] * acc;
        }
    }
    double v[1] = {dot};
    double out[1];
    if (finish_partials<1>(v, partial, ticket, out) && threadIdx.x == 0) scal[S_PQ] = out[0];
}

// CSR values -> sliced ELLPACK positions (pattern built on the host)
__global__ void k_csr_to_sell(const int64_t *rowptr, const double *val, int64_t nc, const int64_t *sell_off,
                              double *sval) {
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < nc; r += (int64_t)gridDim.x * blockDim.x) {
        const int64_t base = sell_off[r >> 5] + (r & 31);
        for (int64_t k = rowptr[r]; k < rowptr[r + 1]; ++k) sval[base + ((k - rowptr[r]) << 5)] = val[k];
    }
}

// r = b - q (q = A x0), z = D^-1 r, p = z; rz, rr, bb
__global__ void __launch_bounds__(kThreads) k_cg_init(const double *b, const double *q, const double *dinv, double *r,
                                                      double *z, double *p, int64_t nc, double *scal,
                                                      double *partial, unsigned *ticket, int *done, double rtol2) {
    double rz = 0.0, rr = 0.0, bb = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nc; i += (int64_t)gridDim.x * blockDim.x) {
        const double ri = b[i] - q[i], zi = dinv[i] * ri;
        r[i] = ri;
        z[i] = zi;
        p[i] = zi;
        rz += ri * zi;
        rr += ri * ri;
        bb += b[i] * b[i];
    }
    double v[3] = {rz, rr, bb};
    double out[3];
    if (finish_partials<3>(v, partial, ticket, out) && threadIdx.x == 0) {
        scal[S_RZ0] = out[0];
        scal[S_RR] = out[1];
        scal[S_BB] = out[2];
        *done = (out[2] == 0.0 || out[1] <= rtol2 * out[2]) ? 1 : 0;
    }
}

// b = 0: the solution is x = 0 (pinned classes fix the constant)
__global__ void k_cg_zero_if_b0(double *x, int64_t nc, const double *scal) {
    if (scal[S_BB] != 0.0) return;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nc; i += (int64_t)gridDim.x * blockDim.x)
        x[i] = 0.0;
}

// alpha = rz / pq; x += alpha p; r -= alpha q; z = D^-1 r; new rz, rr
__global__ void __launch_bounds__(kThreads) k_cg_update(double *x, double *r, double *z, const double *p,
                                                        const double *q, const double *dinv, int64_t nc,
                                                        double *scal, int par, double *partial, unsigned *ticket,
                                                        int *done, int *iters, double rtol2) {
    if (*done) return;
    const double alpha = scal[S_RZ0 + par] / scal[S_PQ];
    double rz = 0.0, rr = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nc; i += (int64_t)gridDim.x * blockDim.x) {
        x[i] += alpha * p[i];
        const double ri = r[i] - alpha * q[i], zi = dinv[i] * ri;
        r[i] = ri;
        z[i] = zi;
        rz += ri * zi;
        rr += ri * ri;
    }
    double v[2] = {rz, rr};
    double out[2];
    if (finish_partials<2>(v, partial, ticket, out) && threadIdx.x == 0) {
        scal[S_RZ0 + (par ^ 1)] = out[0];
        scal[S_RR] = out[1];
        *iters += 1;
        if (out[1] <= rtol2 * scal[S_BB]) *done = 1;
    }
}

// p = z + beta p, beta = rz_new / rz_old
__global__ void __launch_bounds__(kThreads) k_cg_pupdate(double *p, const double *z, int64_t nc, const double *scal,
                                                         int par, const int *done) {
    if (*done) return;
    const double beta = scal[S_RZ0 + (par ^ 1)] / scal[S_RZ0 + par];
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nc; i += (int64_t)gridDim.x * blockDim.x)
        p[i] = z[i] + beta * p[i];
}

// class vector b_c = scale * sum of the node values of the class
__global__ void k_fold_to_classes(const double *bn, const int32_t *cls, int64_t n, double scale, double *bc) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(&bc[cls[i]], scale * bn[i]);
}

__global__ void k_gather_classes(const double *xn, const int32_t *rep, int64_t nc, double *xc) {
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < nc; c += (int64_t)gridDim.x * blockDim.x)
        xc[c] = xn[rep[c]];
}

__global__ void k_expand_classes(const double *xc, const int32_t *cls, int64_t n, double *xn) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        xn[i] = xc[cls[i]];
}

__global__ void k_zero_at(double *v, const int32_t *at, int64_t m) {
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < m; k += (int64_t)gridDim.x * blockDim.x)
        v[at[k]] = 0.0;
}

// pinned class c: row c -> identity row, column c zeroed in the other rows
__global__ void k_pin_rows(const int64_t *rowptr, const int32_t *col, double *val, const int32_t *pins, int64_t m) {
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < m; k += (int64_t)gridDim.x * blockDim.x) {
        const int32_t c = pins[k];
        for (int64_t j = rowptr[c]; j < rowptr[c + 1]; ++j) {
            const int32_t o = col[j];
            val[j] = o == c ? 1.0 : 0.0;
            if (o == c) continue;
            for (int64_t t = rowptr[o]; t < rowptr[o + 1]; ++t)
                if (col[t] == c) val[t] = 0.0;
        }
    }
}

__global__ void k_diag_inverse(const int64_t *rowptr, const int32_t *col, const double *val, int64_t nc,
                               double *dinv, unsigned *err) {
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < nc; c += (int64_t)gridDim.x * blockDim.x) {
        double d = 0.0;
        for (int64_t j = rowptr[c]; j < rowptr[c + 1]; ++j)
            if (col[j] == c) d = val[j];
        if (!(d > 0.0)) {
            atomicOr(err, ERR_NONFINITE);
            d = 1.0;
        }
        dinv[c] = 1.0 / d;
    }
}

}  // namespace

struct PoissonSystem {
    int64_t n = 0, nc = 0, nnz = 0, npin = 0;
    int grid = 1;        // vector kernels
    int grid_mv = 1;     // SpMV grid (one 32-row slice per warp)
    int32_t *cls = nullptr, *rep = nullptr, *col = nullptr, *pins = nullptr;
    int64_t *rowptr = nullptr;
    double *val = nullptr, *dinv = nullptr;
    // sliced ELLPACK copy of the matrix for the iteration
    int64_t *sell_off = nullptr;
    int32_t *sell_w = nullptr, *sell_col = nullptr;
    double *sell_val = nullptr;
    int64_t sell_n = 0;
    double *x = nullptr, *r = nullptr, *z = nullptr, *p = nullptr, *q = nullptr, *b = nullptr;
    double *partial = nullptr, *scal = nullptr;
    unsigned *ticket = nullptr;
    int *done = nullptr, *iters = nullptr;
    ~PoissonSystem() {
        for (void *ptr : {(void *)sell_off, (void *)sell_w, (void *)sell_col, (void *)sell_val})
            if (ptr) cudaFree(ptr);
        for (void *ptr : {(void *)cls, (void *)rep, (void *)col, (void *)pins, (void *)rowptr, (void *)val, (void *)dinv,
                          (void *)x, (void *)r, (void *)z, (void *)p, (void *)q, (void *)b, (void *)partial,
                          (void *)scal, (void *)ticket, (void *)done, (void *)iters})
            if (ptr) cudaFree(ptr);
    }
};

void poisson_free(PoissonSystem *ps) { delete ps; }
int64_t poisson_classes(const PoissonSystem *ps) { return ps->nc; }
int64_t poisson_nnz(const PoissonSystem *ps) { return ps->nnz; }
const int32_t *poisson_cls(const PoissonSystem *ps) { return ps->cls; }
const int64_t *poisson_rowptr(const PoissonSystem *ps) { return ps->rowptr; }
const int32_t *poisson_col(const PoissonSystem *ps) { return ps->col; }
double *poisson_val(PoissonSystem *ps) { return ps->val; }

cudaError_t poisson_build(const PoissonBuild &in, int sms, PoissonSystem **out) {
    *out = nullptr;
    const int64_t n = in.n;
    // classes: compact numbers in the order of first appearance
    std::vector<int32_t> cidx((size_t)n), rep;
    std::vector<int32_t> of_rep((size_t)n, -1);
    for (int64_t i = 0; i < n; ++i) {
        const int32_t r = in.class_of ? in.class_of[i] : (int32_t)i;
        if (of_rep[(size_t)r] < 0) {
            of_rep[(size_t)r] = (int32_t)rep.size();
            rep.push_back(r);
        }
        cidx[(size_t)i] = of_rep[(size_t)r];
    }
    const int64_t nc = (int64_t)rep.size();
    // incidences class -> global element
    std::vector<int64_t> boff(in.conn.size() + 1, 0);
    for (size_t bk = 0; bk < in.conn.size(); ++bk) boff[bk + 1] = boff[bk] + in.count[bk];
    std::vector<int64_t> ioff((size_t)nc + 1, 0);
    for (size_t bk = 0; bk < in.conn.size(); ++bk)
        for (int a = 0; a < in.nen[bk]; ++a)
            for (int64_t e = 0; e < in.count[bk]; ++e) ioff[(size_t)cidx[(size_t)in.conn[bk][a * in.count[bk] + e]] + 1]++;
    for (int64_t c = 0; c < nc; ++c) ioff[(size_t)c + 1] += ioff[(size_t)c];
    std::vector<int64_t> inc((size_t)ioff[(size_t)nc]), fill(ioff.begin(), ioff.end() - 1);
    for (size_t bk = 0; bk < in.conn.size(); ++bk)
        for (int a = 0; a < in.nen[bk]; ++a)
            for (int64_t e = 0; e < in.count[bk]; ++e)
                inc[(size_t)fill[(size_t)cidx[(size_t)in.conn[bk][a * in.count[bk] + e]]]++] = boff[bk] + e;
    // rows: the classes of every node of every incident element
    std::vector<int64_t> rowptr((size_t)nc + 1, 0);
    std::vector<int32_t> col;
    col.reserve((size_t)nc * 16);
    std::vector<int32_t> stamp((size_t)nc, -1), row;
    for (int64_t c = 0; c < nc; ++c) {
        row.clear();
        for (int64_t k = ioff[(size_t)c]; k < ioff[(size_t)c + 1]; ++k) {
            const int64_t g = inc[(size_t)k];
            const size_t bk = (size_t)(std::upper_bound(boff.begin(), boff.end(), g) - boff.begin()) - 1;
            const int64_t e = g - boff[bk];
            for (int a = 0; a < in.nen[bk]; ++a) {
                const int32_t o = cidx[(size_t)in.conn[bk][a * in.count[bk] + e]];
                if (stamp[(size_t)o] != (int32_t)c) {
                    stamp[(size_t)o] = (int32_t)c;
                    row.push_back(o);
                }
            }
        }
        std::sort(row.begin(), row.end());
        col.insert(col.end(), row.begin(), row.end());
        rowptr[(size_t)c + 1] = (int64_t)col.size();
    }
    // sliced ELLPACK pattern: slices of 32 rows, width = longest row of the slice
    const int64_t nslices = (nc + 31) / 32;
    std::vector<int64_t> soff((size_t)nslices + 1, 0);
    std::vector<int32_t> sw((size_t)std::max<int64_t>(nslices, 1), 0);
    for (int64_t sl = 0; sl < nslices; ++sl) {
        int64_t w = 0;
        for (int64_t r = sl * 32; r < std::min(nc, sl * 32 + 32); ++r) w = std::max(w, rowptr[(size_t)r + 1] - rowptr[(size_t)r]);
        sw[(size_t)sl] = (int32_t)w;
        soff[(size_t)sl + 1] = soff[(size_t)sl] + 32 * w;
    }
    std::vector<int32_t> scol((size_t)soff[(size_t)nslices]);
    for (int64_t sl = 0; sl < nslices; ++sl)
        for (int lane = 0; lane < 32; ++lane) {
            const int64_t r = sl * 32 + lane;
            for (int64_t j = 0; j < sw[(size_t)sl]; ++j) {
                const int64_t k = r < nc ? rowptr[(size_t)r] + j : -1;
                scol[(size_t)(soff[(size_t)sl] + j * 32 + lane)] =
                    (r < nc && k < rowptr[(size_t)r + 1]) ? col[(size_t)k] : (int32_t)std::min<int64_t>(r, nc - 1);
            }
        }
    // pinned classes (the class of node 0 when none are given)
    std::vector<int32_t> pins;
    if (in.pinned) {
        std::vector<char> seen((size_t)nc, 0);
        for (int64_t i = 0; i < n; ++i)
            if (in.pinned[i] && !seen[(size_t)cidx[(size_t)i]]) {
                seen[(size_t)cidx[(size_t)i]] = 1;
                pins.push_back(cidx[(size_t)i]);
            }
    } else if (nc > 0) {
        pins.push_back(cidx[0]);
    }
    auto *ps = new PoissonSystem;
    ps->n = n;
    ps->nc = nc;
    ps->nnz = (int64_t)col.size();
    ps->npin = (int64_t)pins.size();
    ps->grid = (int)std::max<int64_t>(1, std::min<int64_t>((nc + kThreads - 1) / kThreads, (int64_t)sms * 8));
    // SpMV: one slice of 32 rows per warp
    ps->grid_mv = (int)std::max<int64_t>(1, std::min<int64_t>((nc + 255) / 256, (int64_t)sms * 16));
    cudaError_t e = cudaSuccess;
#define PS_TRY(x)                  \
    do {                           \
        e = (x);                   \
        if (e != cudaSuccess) {    \
            delete ps;             \
            return e;              \
        }                          \
    } while (0)
    PS_TRY(dalloc(&ps->cls, (size_t)n));
    PS_TRY(dalloc(&ps->rep, (size_t)nc));
    PS_TRY(dalloc(&ps->rowptr, (size_t)nc + 1));
    PS_TRY(dalloc(&ps->col, col.size()));
    PS_TRY(dalloc(&ps->val, col.size()));
    PS_TRY(dalloc(&ps->dinv, (size_t)nc));
    PS_TRY(dalloc(&ps->pins, std::max<size_t>(pins.size(), 1)));
    for (double **v : {&ps->x, &ps->r, &ps->z, &ps->p, &ps->q, &ps->b}) PS_TRY(dalloc(v, (size_t)std::max<int64_t>(nc, 1)));
    PS_TRY(dalloc(&ps->partial, (size_t)3 * std::max(ps->grid, ps->grid_mv)));
    PS_TRY(dalloc(&ps->scal, (size_t)S_COUNT));
    PS_TRY(dalloc(&ps->ticket, 1));
    PS_TRY(dalloc(&ps->done, 1));
    PS_TRY(dalloc(&ps->iters, 1));
    PS_TRY(cudaMemcpy(ps->cls, cidx.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice));
    PS_TRY(cudaMemcpy(ps->rep, rep.data(), sizeof(int32_t) * nc, cudaMemcpyHostToDevice));
    PS_TRY(cudaMemcpy(ps->rowptr, rowptr.data(), sizeof(int64_t) * (nc + 1), cudaMemcpyHostToDevice));
    PS_TRY(cudaMemcpy(ps->col, col.data(), sizeof(int32_t) * col.size(), cudaMemcpyHostToDevice));
    if (!pins.empty()) PS_TRY(cudaMemcpy(ps->pins, pins.data(), sizeof(int32_t) * pins.size(), cudaMemcpyHostToDevice));
    PS_TRY(cudaMemset(ps->val, 0, sizeof(double) * col.size()));
    ps->sell_n = (int64_t)scol.size();
    PS_TRY(dalloc(&ps->sell_off, soff.size()));
    PS_TRY(dalloc(&ps->sell_w, sw.size()));
    PS_TRY(dalloc(&ps->sell_col, std::max<size_t>(scol.size(), 1)));
    PS_TRY(dalloc(&ps->sell_val, std::max<size_t>(scol.size(), 1)));
    PS_TRY(cudaMemcpy(ps->sell_off, soff.data(), sizeof(int64_t) * soff.size(), cudaMemcpyHostToDevice));
    PS_TRY(cudaMemcpy(ps->sell_w, sw.data(), sizeof(int32_t) * sw.size(), cudaMemcpyHostToDevice));
    if (!scol.empty())
        PS_TRY(cudaMemcpy(ps->sell_col, scol.data(), sizeof(int32_t) * scol.size(), cudaMemcpyHostToDevice));
    PS_TRY(cudaMemset(ps->sell_val, 0, sizeof(double) * std::max<size_t>(scol.size(), 1)));
    PS_TRY(cudaMemset(ps->ticket, 0, sizeof(unsigned)));
#undef PS_TRY
    *out = ps;
    return cudaSuccess;
}

cudaError_t poisson_finish(PoissonSystem *ps, unsigned *err, int sms, cudaStream_t s) {
    if (ps->npin) k_pin_rows<<<(unsigned)((ps->npin + 127) / 128), 128, 0, s>>>(ps->rowptr, ps->col, ps->val, ps->pins,
                                                                                  ps->npin);
    const int64_t g = std::max<int64_t>(1, std::min<int64_t>((ps->nc + 255) / 256, (int64_t)sms * 8));
    k_diag_inverse<<<(unsigned)g, 256, 0, s>>>(ps->rowptr, ps->col, ps->val, ps->nc, ps->dinv, err);
    k_csr_to_sell<<<(unsigned)g, 256, 0, s>>>(ps->rowptr, ps->val, ps->nc, ps->sell_off, ps->sell_val);
    return cudaGetLastError();
}

cudaError_t poisson_solve(PoissonSystem *ps, const double *b_node, double scale, double *x_node, double rtol,
                          int max_iter, int sms, cudaStream_t s, int *iters_out, double *rel_res_out,
                          int64_t *launches) {
    const int64_t n = ps->n, nc = ps->nc;
    const int G = ps->grid, GM = ps->grid_mv;
    const int64_t gn = std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, (int64_t)sms * 8));
    const double rtol2 = rtol * rtol;
    cudaError_t e;
    if ((e = cudaMemsetAsync(ps->b, 0, sizeof(double) * nc, s))) return e;
    if ((e = cudaMemsetAsync(ps->done, 0, sizeof(int), s))) return e;
    if ((e = cudaMemsetAsync(ps->iters, 0, sizeof(int), s))) return e;
    k_fold_to_classes<<<(unsigned)gn, 256, 0, s>>>(b_node, ps->cls, n, scale, ps->b);
    k_gather_classes<<<(unsigned)G, kThreads, 0, s>>>(x_node, ps->rep, nc, ps->x);
    if (ps->npin) {
        k_zero_at<<<1, 128, 0, s>>>(ps->b, ps->pins, ps->npin);
        k_zero_at<<<1, 128, 0, s>>>(ps->x, ps->pins, ps->npin);
    }
    // r = b - A x0
    k_cg_spmv<<<GM, kThreads, 0, s>>>(ps->sell_off, ps->sell_w, ps->sell_col, ps->sell_val, ps->x, ps->q, nc,
                                      ps->scal, ps->partial, ps->ticket, ps->done);
    k_cg_init<<<G, kThreads, 0, s>>>(ps->b, ps->q, ps->dinv, ps->r, ps->z, ps->p, nc, ps->scal, ps->partial, ps->ticket,
                                     ps->done, rtol2);
    k_cg_zero_if_b0<<<G, kThreads, 0, s>>>(ps->x, nc, ps->scal);
    *launches += 5 + (ps->npin ? 2 : 0);
    int it = 0, done_h = 0;
    while (it < max_iter) {
        const int batch = std::min(8, max_iter - it);
        for (int k = 0; k < batch; ++k, ++it) {
            const int par = it & 1;
            k_cg_spmv<<<GM, kThreads, 0, s>>>(ps->sell_off, ps->sell_w, ps->sell_col, ps->sell_val, ps->p, ps->q,
                                              nc, ps->scal, ps->partial, ps->ticket, ps->done);
            k_cg_update<<<G, kThreads, 0, s>>>(ps->x, ps->r, ps->z, ps->p, ps->q, ps->dinv, nc, ps->scal, par,
                                               ps->partial, ps->ticket, ps->done, ps->iters, rtol2);
            k_cg_pupdate<<<G, kThreads, 0, s>>>(ps->p, ps->z, nc, ps->scal, par, ps->done);
        }
        *launches += 3 * batch;
        if ((e = cudaGetLastError())) return e;
        if ((e = cudaMemcpyAsync(&done_h, ps->done, sizeof(int), cudaMemcpyDeviceToHost, s))) return e;
        if ((e = cudaStreamSynchronize(s))) return e;
        if (done_h) break;
    }
    k_expand_classes<<<(unsigned)gn, 256, 0, s>>>(ps->x, ps->cls, n, x_node);
    *launches += 1;
    double sc[S_COUNT];
    int iters = 0;
    if ((e = cudaMemcpyAsync(sc, ps->scal, sizeof(sc), cudaMemcpyDeviceToHost, s))) return e;
    if ((e = cudaMemcpyAsync(&iters, ps->iters, sizeof(int), cudaMemcpyDeviceToHost, s))) return e;
    if ((e = cudaStreamSynchronize(s))) return e;
    if (iters_out) *iters_out = iters;
    if (rel_res_out) *rel_res_out = sc[S_BB] > 0.0 ? sqrt(sc[S_RR] / sc[S_BB]) : 0.0;
    return cudaGetLastError();
}

}  // namespace fea
