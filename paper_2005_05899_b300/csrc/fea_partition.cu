// Space-filling-curve order of points, SFC partition of a mesh's elements
// and the correction coefficients of the partition (section 5 and the
// load-balancing section).  The partitioner: a bounding box, a regular grid of
// bins inside it, bins weighted by their elements (weight = Gauss points of
// the element's rule), the bins projected to 1-D along a space-filling curve,
// and the weighted 1-D sequence cut into contiguous parts.  The curve is a
// Hilbert curve; its index is computed by J. Skilling's transpose algorithm
// ("Programming the Hilbert curve", AIP Conf. Proc. 707, 2004).  Host code
// only: no CUDA call, so it runs without a device.
#include <stdint.h>

#include <algorithm>
#include <cmath>
#include <numeric>
#include <utility>
#include <vector>

#include "fea.h"
#include "fea_internal.h"

namespace fea {

uint64_t morton_spread3(uint64_t v) {
    v &= 0x1FFFFFull;
    v = (v | (v << 32)) & 0x1F00000000FFFFull;
    v = (v | (v << 16)) & 0x1F0000FF0000FFull;
    v = (v | (v << 8)) & 0x100F00F00F00F00Full;
    v = (v | (v << 4)) & 0x10C30C30C30C30C3ull;
    v = (v | (v << 2)) & 0x1249249249249249ull;
    return v;
}

// Hilbert index of the cell (x0, x1, x2) of a 2^bits grid.  Skilling's
// method: undo the excess work of the axes (reflections and exchanges from the
// most significant bit down), Gray-encode, then read the "transposed" index
// bit-plane by bit-plane, axis 0 first.
uint64_t hilbert_key3(uint32_t x0, uint32_t x1, uint32_t x2, int bits) {
    uint32_t X[3] = {x0, x1, x2};
    const uint32_t M = 1u << (bits - 1);
    for (uint32_t Q = M; Q > 1; Q >>= 1) {
        const uint32_t P = Q - 1;
        for (int i = 0; i < 3; ++i) {
            if (X[i] & Q) {
                X[0] ^= P;   // invert the low bits of axis 0
            } else {
                const uint32_t t = (X[0] ^ X[i]) & P;   // exchange the low bits of axes 0 and i
                X[0] ^= t;
                X[i] ^= t;
            }
        }
    }
    for (int i = 1; i < 3; ++i) X[i] ^= X[i - 1];
    uint32_t t = 0;
    for (uint32_t Q = M; Q > 1; Q >>= 1)
        if (X[2] & Q) t ^= Q - 1;
    for (int i = 0; i < 3; ++i) X[i] ^= t;
    uint64_t key = 0;
    for (int b = bits - 1; b >= 0; --b)
        for (int i = 0; i < 3; ++i) key = (key << 1) | ((X[i] >> b) & 1u);
    return key;
}

namespace {

// bin keys of n points (coordinates as [3][n] with stride n), grid of 2^level
// cells per axis over the points' bounding box
void bin_keys(int64_t n, const double *xyz, int64_t stride, int level, std::vector<uint64_t> &key) {
    double lo[3], hi[3];
    for (int i = 0; i < 3; ++i) {
        lo[i] = hi[i] = n ? xyz[i * stride] : 0.0;
        for (int64_t k = 0; k < n; ++k) {
            lo[i] = std::min(lo[i], xyz[i * stride + k]);
            hi[i] = std::max(hi[i], xyz[i * stride + k]);
        }
    }
    const double cells = double(1u << level);
    key.resize((size_t)n);
    for (int64_t k = 0; k < n; ++k) {
        uint32_t c[3];
        for (int i = 0; i < 3; ++i) {
            const double w = hi[i] - lo[i];
            double q = w > 0.0 ? (xyz[i * stride + k] - lo[i]) / w * cells : 0.0;
            q = std::min(std::max(q, 0.0), cells - 1.0);
            c[i] = (uint32_t)q;
        }
        key[(size_t)k] = hilbert_key3(c[0], c[1], c[2], level);
    }
}

}  // namespace

int greedy_colour(int64_t n_nodes, int nen, int64_t count, const int32_t *conn, int64_t elem_stride,
                  int64_t node_stride, int32_t *col) {
    constexpr int W = kColourMax / 64;
    std::vector<uint64_t> seen((size_t)n_nodes * W, 0ull);
    int n_col = 0;
    for (int64_t e = 0; e < count; ++e) {
        uint64_t mask[W] = {};
        for (int a = 0; a < nen; ++a) {
            const int64_t v = conn[e * elem_stride + a * node_stride];
            if (v < 0 || v >= n_nodes) return -2;
            for (int k = 0; k < W; ++k) mask[k] |= seen[(size_t)v * W + k];
        }
        int c = -1;
        for (int k = 0; k < W && c < 0; ++k)
            if (~mask[k]) c = 64 * k + __builtin_ctzll(~mask[k]);
        if (c < 0) return -1;
        col[e] = c;
        n_col = std::max(n_col, c + 1);
        for (int a = 0; a < nen; ++a)
            seen[(size_t)conn[e * elem_stride + a * node_stride] * W + c / 64] |= 1ull << (c % 64);
    }
    return n_col;
}

}  // namespace fea

using namespace fea;

extern "C" {

fea_status fea_colour_elements(int64_t n_nodes, int32_t n_en, int64_t count, const int32_t *conn, int32_t *colour,
                               int32_t *n_colours) {
    if (n_nodes < 0 || n_en < 1 || n_en > kMaxNen || count < 0 || (count > 0 && (!conn || !colour)) || !n_colours)
        return FEA_EINVAL;
    const int nc = greedy_colour(n_nodes, n_en, count, conn, n_en, 1, colour);
    if (nc == -2) return FEA_EMESH;
    if (nc < 0) return FEA_ENUMERIC;
    *n_colours = nc;
    return FEA_OK;
}

fea_status fea_sfc_order(int64_t n, const double *xyz, int32_t level, int64_t *order) {
    if (n < 0 || (n > 0 && (!xyz || !order)) || level < 1 || level > 21) return FEA_EINVAL;
    std::vector<uint64_t> key;
    bin_keys(n, xyz, n, level, key);
    std::vector<int64_t> idx((size_t)n);
    std::iota(idx.begin(), idx.end(), int64_t(0));
    std::stable_sort(idx.begin(), idx.end(), [&](int64_t a, int64_t b) { return key[(size_t)a] < key[(size_t)b]; });
    std::copy(idx.begin(), idx.end(), order);
    return FEA_OK;
}

fea_status fea_partition_sfc(const fea_mesh_desc *desc, int32_t nparts, int32_t level, const double *lambda,
                             int32_t *const part[4]) {
    if (!desc || !part || nparts < 1 || level < 1 || level > 21 || desc->n_nodes < 0 || !desc->xyz) return FEA_EINVAL;
    // cumulative target fractions: part p ends at (lambda_0 + ... + lambda_p) / P
    std::vector<double> cum((size_t)nparts + 1, 0.0);
    for (int32_t p = 0; p < nparts; ++p) {
        const double l = lambda ? lambda[p] : 1.0;
        if (!(l >= 0.0)) return FEA_EINVAL;
        cum[(size_t)p + 1] = cum[(size_t)p] + l;
    }
    if (!(cum[(size_t)nparts] > 0.0)) return FEA_EINVAL;
    for (auto &c : cum) c /= cum[(size_t)nparts];
    const int64_t n = desc->n_nodes;
    // element centroids (the "location of each element" of the partitioner)
    std::vector<double> cen[3];
    std::vector<std::pair<int, int64_t>> who;   // (type, element) of each centroid
    std::vector<int> weight;
    for (int t = 0; t < 4; ++t) {
        const int64_t E = desc->n_elem[t];
        if (E < 0) return FEA_EINVAL;
        if (!E) continue;
        if (!desc->conn[t] || !part[t]) return FEA_EINVAL;
        const int nen = kNen[t];
        for (int64_t e = 0; e < E; ++e) {
            double c[3] = {0.0, 0.0, 0.0};
            for (int a = 0; a < nen; ++a) {
                const int32_t v = desc->conn[t][e * nen + a];
                if (v < 0 || v >= n) return FEA_EMESH;
                for (int i = 0; i < 3; ++i) c[i] += desc->xyz[i * n + v];
            }
            for (int i = 0; i < 3; ++i) cen[i].push_back(c[i] / nen);
            who.emplace_back(t, e);
            weight.push_back(kNg[t]);   // cost model: Gauss points of the element's rule
        }
    }
    const int64_t N = (int64_t)who.size();
    if (N == 0) return FEA_OK;
    std::vector<double> xyz3((size_t)(3 * N));
    for (int i = 0; i < 3; ++i) std::copy(cen[i].begin(), cen[i].end(), xyz3.begin() + (size_t)i * N);
    std::vector<uint64_t> key;
    bin_keys(N, xyz3.data(), N, level, key);
    std::vector<int64_t> idx((size_t)N);
    std::iota(idx.begin(), idx.end(), int64_t(0));
    std::stable_sort(idx.begin(), idx.end(), [&](int64_t a, int64_t b) { return key[(size_t)a] < key[(size_t)b]; });
    // 1-D partition of the weighted bin sequence: a bin goes to the part that
    // holds the midpoint of its weight interval (whole bins per part)
    double total = 0.0;
    for (int w : weight) total += w;
    double before = 0.0;
    int64_t k = 0;
    while (k < N) {
        int64_t k1 = k;
        double w = 0.0;
        while (k1 < N && key[(size_t)idx[(size_t)k1]] == key[(size_t)idx[(size_t)k]]) w += weight[(size_t)idx[(size_t)k1++]];
        // the part whose target interval holds the midpoint of the bin's weight
        const double mid = (before + 0.5 * w) / total;
        int32_t p = (int32_t)(std::upper_bound(cum.begin() + 1, cum.end(), mid) - (cum.begin() + 1));
        p = std::min(std::max(p, 0), nparts - 1);
        for (int64_t j = k; j < k1; ++j) {
            const auto &te = who[(size_t)idx[(size_t)j]];
            part[te.first][te.second] = p;
        }
        before += w;
        k = k1;
    }
    return FEA_OK;
}

fea_status fea_balance_update(int32_t nparts, int32_t n_obs, const double *Lambda, const double *times,
                              double *lambda_out) {
    if (nparts < 1 || n_obs < 1 || !Lambda || !times || !lambda_out) return FEA_EINVAL;
    const size_t P = (size_t)nparts;
    std::vector<double> Lnew(P + 1, 0.0);
    Lnew[P] = (double)nparts;
    for (size_t i = 1; i < P; ++i) {
        // weighted least squares over (Lambda_i^k, Upsilon_i^k), k = 0..n_obs-1 (weights 1.5^k),
        // plus the origin (no weight takes no time) with weight 1
        double sw = 1.0, sx = 0.0, sy = 0.0, sxx = 0.0, sxy = 0.0;
        double wk = 1.0;
        for (int32_t k = 0; k < n_obs; ++k, wk *= 1.5) {
            const double *t = times + (size_t)k * P;
            double total = 0.0, head = 0.0;
            for (size_t j = 0; j < P; ++j) {
                if (!(t[j] >= 0.0)) return FEA_EINVAL;
                total += t[j];
                if (j < i) head += t[j];
            }
            if (!(total > 0.0)) return FEA_EINVAL;
            const double x = Lambda[(size_t)k * (P + 1) + i];
            const double y = head / (total / (double)nparts);   // Upsilon_i = T_i / mean time
            sw += wk;
            sx += wk * x;
            sy += wk * y;
            sxx += wk * x * x;
            sxy += wk * x * y;
        }
        const double den = sw * sxx - sx * sx;
        if (!(std::fabs(den) > 0.0)) return FEA_ENUMERIC;
        const double beta = (sw * sxy - sx * sy) / den, alpha = (sy - beta * sx) / sw;
        if (!(beta > 0.0)) return FEA_ENUMERIC;
        Lnew[i] = ((double)i - alpha) / beta;
    }
    // keep the splitting points ordered inside [0, P]
    for (size_t i = 1; i < P; ++i) Lnew[i] = std::min(std::max(Lnew[i], Lnew[i - 1]), (double)nparts);
    for (size_t i = 0; i < P; ++i) lambda_out[i] = Lnew[i + 1] - Lnew[i];
    return FEA_OK;
}

}  // extern "C"
