// Host mesh preprocessing (runs once per mesh, before any time step).
//
//   * affine geometry: J = [x1-x0, x2-x0, x3-x0], det J > 0 required, J^-1;
//   * face matching by sorted global vertex-id triples (periodic images share
//     ids); a triple seen once is a boundary face and needs a wall or
//     far-field tag, a triple seen more than twice is an error;
//   * relative orientation of every matched face pair (which permutation of
//     the own face's vertices gives the neighbour's);
//   * element renumbering, the paper's grid-renumbering optimisation
//     (Sec. III-B): reverse Cuthill-McKee on the element adjacency graph
//     from a George-Liu pseudo-peripheral start node, or a Morton or Hilbert
//     curve of the element centroids.  Ties are broken by the lower original
//     index.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>

#include "dg_internal.h"

namespace dg {

namespace {

struct FaceKey {
    int32_t v[3];
    int64_t slot;   // 4*element + local face
};

bool key_less(const FaceKey& a, const FaceKey& b) {
    if (a.v[0] != b.v[0]) return a.v[0] < b.v[0];
    if (a.v[1] != b.v[1]) return a.v[1] < b.v[1];
    if (a.v[2] != b.v[2]) return a.v[2] < b.v[2];
    return a.slot < b.slot;
}

bool key_same(const FaceKey& a, const FaceKey& b) {
    return a.v[0] == b.v[0] && a.v[1] == b.v[1] && a.v[2] == b.v[2];
}

void face_vertices(int f, int out[3]) {
    int n = 0;
    for (int k = 0; k < 4; ++k)
        if (k != f) out[n++] = k;
}

// Breadth-first levels from `root` over unvisited-in-`mask` nodes; returns the
// last level and the depth.
int bfs_depth(const std::vector<int32_t>& nbr, int64_t root, std::vector<int32_t>& stamp, int32_t tag,
              std::vector<int64_t>& last_level) {
    std::vector<int64_t> cur{root}, next;
    stamp[root] = tag;
    int depth = 0;
    while (true) {
        next.clear();
        for (int64_t u : cur)
            for (int f = 0; f < 4; ++f) {
                int32_t w = nbr[4 * u + f];
                if (w >= 0 && stamp[w] != tag) { stamp[w] = tag; next.push_back(w); }
            }
        if (next.empty()) break;
        cur.swap(next);
        ++depth;
    }
    last_level = cur;
    return depth;
}

void rcm_order(const std::vector<int32_t>& nbr, int64_t ne, std::vector<int32_t>& order) {
    std::vector<int32_t> deg(ne, 0);
    for (int64_t e = 0; e < ne; ++e)
        for (int f = 0; f < 4; ++f) deg[e] += nbr[4 * e + f] >= 0;
    std::vector<char> done(ne, 0);
    std::vector<int32_t> stamp(ne, -1);
    int32_t tag = 0;
    order.clear();
    order.reserve(ne);
    // nodes by (degree, index) to pick component start candidates
    std::vector<int32_t> by_deg(ne);
    std::iota(by_deg.begin(), by_deg.end(), 0);
    std::stable_sort(by_deg.begin(), by_deg.end(), [&](int32_t a, int32_t b) { return deg[a] < deg[b]; });
    size_t cursor = 0;
    std::vector<int64_t> last;
    while ((int64_t)order.size() < ne) {
        while (done[by_deg[cursor]]) ++cursor;
        int64_t r = by_deg[cursor];
        // George-Liu pseudo-peripheral node
        int depth = bfs_depth(nbr, r, stamp, tag++, last);
        for (int it = 0; it < 16; ++it) {
            int64_t best = last[0];
            for (int64_t u : last)
                if (deg[u] < deg[best] || (deg[u] == deg[best] && u < best)) best = u;
            std::vector<int64_t> last2;
            int d2 = bfs_depth(nbr, best, stamp, tag++, last2);
            if (d2 > depth) { r = best; depth = d2; last = last2; }
            else break;
        }
        // Cuthill-McKee from r: children in increasing (degree, index)
        size_t head = order.size();
        order.push_back((int32_t)r);
        done[r] = 1;
        std::vector<int32_t> kids;
        while (head < order.size()) {
            int32_t u = order[head++];
            kids.clear();
            for (int f = 0; f < 4; ++f) {
                int32_t w = nbr[4 * (int64_t)u + f];
                if (w >= 0 && !done[w]) { done[w] = 1; kids.push_back(w); }
            }
            std::sort(kids.begin(), kids.end(), [&](int32_t a, int32_t b) {
                return deg[a] != deg[b] ? deg[a] < deg[b] : a < b;
            });
            order.insert(order.end(), kids.begin(), kids.end());
        }
    }
    std::reverse(order.begin(), order.end());
}

uint64_t spread3(uint64_t x) {
    x &= 0x1fffff;
    x = (x | x << 32) & 0x1f00000000ffffULL;
    x = (x | x << 16) & 0x1f0000ff0000ffULL;
    x = (x | x << 8) & 0x100f00f00f00f00fULL;
    x = (x | x << 4) & 0x10c30c30c30c30c3ULL;
    x = (x | x << 2) & 0x1249249249249249ULL;
    return x;
}

// Position along the 3D Hilbert curve of a point on the 2^21 lattice, after J. Skilling,
// "Programming the Hilbert curve" (AIP Conf. Proc. 707, 2004): the coordinates are turned in
// place into the "transposed" index (from the top bit down, each lower-bit field is either
// inverted in x or exchanged between x and the current axis; then a Gray decode), whose bits
// are then interleaved, most significant level first, x before y before z.
uint64_t hilbert_key(uint32_t x, uint32_t y, uint32_t z) {
    uint32_t X[3] = {x, y, z};
    for (uint32_t Q = 1u << 20; Q > 1; Q >>= 1) {
        const uint32_t P = Q - 1;
        for (int i = 0; i < 3; ++i) {
            if (X[i] & Q) {
                X[0] ^= P;
            } else {
                const uint32_t t = (X[0] ^ X[i]) & P;
                X[0] ^= t;
                X[i] ^= t;
            }
        }
    }
    X[1] ^= X[0];
    X[2] ^= X[1];
    uint32_t t = 0;
    for (uint32_t Q = 1u << 20; Q > 1; Q >>= 1)
        if (X[2] & Q) t ^= Q - 1;
    for (uint32_t& v : X) v ^= t;
    return (spread3(X[0]) << 2) | (spread3(X[1]) << 1) | spread3(X[2]);
}

// Space-filling-curve order of the element centroids, quantised to 21 bits per axis over their
// bounding box: Morton (bit interleave, x lowest) or Hilbert.  Ties keep the input order.
void curve_order(const double* xyz, int64_t ne, bool hilbert, std::vector<int32_t>& order) {
    double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
    std::vector<double> c(3 * ne);
    for (int64_t e = 0; e < ne; ++e)
        for (int d = 0; d < 3; ++d) {
            double s = 0.0;
            for (int k = 0; k < 4; ++k) s += xyz[12 * e + 3 * k + d];
            c[3 * e + d] = 0.25 * s;
            lo[d] = std::min(lo[d], c[3 * e + d]);
            hi[d] = std::max(hi[d], c[3 * e + d]);
        }
    std::vector<uint64_t> code(ne);
    for (int64_t e = 0; e < ne; ++e) {
        uint32_t q[3];
        for (int d = 0; d < 3; ++d) {
            double t = (c[3 * e + d] - lo[d]) / std::max(hi[d] - lo[d], 1e-300);
            q[d] = (uint32_t)std::min(2097151.0, std::max(0.0, t * 2097151.0));
        }
        code[e] = hilbert ? hilbert_key(q[0], q[1], q[2])
                          : spread3(q[0]) | (spread3(q[1]) << 1) | (spread3(q[2]) << 2);
    }
    order.resize(ne);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) { return code[a] < code[b]; });
}

}  // namespace

bool build_mesh(const int32_t* tet_vid, const double* tet_xyz, const int8_t* bc_tag, int64_t ne,
                int renumber, MeshHost& out, int& code, std::string& err) {
    code = DG_ERR_MESH;
    out = MeshHost();
    out.ne = ne;
    // geometry in caller order
    out.x0J.resize(12 * ne);
    std::vector<double> jinv_c(9 * ne);
    for (int64_t e = 0; e < ne; ++e) {
        const double* x = tet_xyz + 12 * e;
        double J[9];
        for (int r = 0; r < 3; ++r)
            for (int c = 0; c < 3; ++c) J[3 * r + c] = x[3 * (c + 1) + r] - x[r];
        double det = J[0] * (J[4] * J[8] - J[5] * J[7]) - J[1] * (J[3] * J[8] - J[5] * J[6]) +
                     J[2] * (J[3] * J[7] - J[4] * J[6]);
        if (!(det > 0.0) || !std::isfinite(det)) {
            err = "tetrahedron " + std::to_string(e) + " has non-positive volume";
            return false;
        }
        double* I = &jinv_c[9 * e];
        I[0] = (J[4] * J[8] - J[5] * J[7]) / det;
        I[1] = (J[2] * J[7] - J[1] * J[8]) / det;
        I[2] = (J[1] * J[5] - J[2] * J[4]) / det;
        I[3] = (J[5] * J[6] - J[3] * J[8]) / det;
        I[4] = (J[0] * J[8] - J[2] * J[6]) / det;
        I[5] = (J[2] * J[3] - J[0] * J[5]) / det;
        I[6] = (J[3] * J[7] - J[4] * J[6]) / det;
        I[7] = (J[1] * J[6] - J[0] * J[7]) / det;
        I[8] = (J[0] * J[4] - J[1] * J[3]) / det;
        for (int d = 0; d < 3; ++d) out.x0J[12 * e + d] = x[d];
        for (int k = 0; k < 9; ++k) out.x0J[12 * e + 3 + k] = J[k];
    }
    // face matching
    std::vector<FaceKey> keys(4 * ne);
    for (int64_t e = 0; e < ne; ++e) {
        for (int f = 0; f < 4; ++f) {
            int fv[3];
            face_vertices(f, fv);
            FaceKey& k = keys[4 * e + f];
            for (int m = 0; m < 3; ++m) k.v[m] = tet_vid[4 * e + fv[m]];
            std::sort(k.v, k.v + 3);
            if (k.v[0] == k.v[1] || k.v[1] == k.v[2]) {
                err = "tetrahedron " + std::to_string(e) + " repeats a vertex id";
                return false;
            }
            k.slot = 4 * e + f;
        }
    }
    std::sort(keys.begin(), keys.end(), key_less);
    std::vector<int32_t> nbr_c(4 * ne, -1);
    std::vector<uint8_t> fcode_c(4 * ne, 0);
    int64_t nf = 0, nbf = 0;
    for (size_t i = 0; i < keys.size();) {
        size_t j = i + 1;
        while (j < keys.size() && key_same(keys[i], keys[j])) ++j;
        if (j - i > 2) {
            err = "a face is shared by more than two tetrahedra";
            return false;
        }
        ++nf;
        if (j - i == 1) {
            int64_t s = keys[i].slot;
            int tag = bc_tag ? bc_tag[s] : 0;
            if (tag != DG_BC_WALL && tag != DG_BC_FARFIELD) {
                err = "unmatched face of tetrahedron " + std::to_string(s / 4) + " has no wall/far-field tag";
                return false;
            }
            nbr_c[s] = -1 - tag;
            ++nbf;
        } else {
            for (int side = 0; side < 2; ++side) {
                int64_t s = keys[i + side].slot, t = keys[i + 1 - side].slot;
                int64_t e = s / 4, n = t / 4;
                int f = (int)(s % 4), fn = (int)(t % 4);
                int fv[3], gv[3];
                face_vertices(f, fv);
                face_vertices(fn, gv);
                int pi[3];
                for (int m = 0; m < 3; ++m) {
                    int32_t h = tet_vid[4 * n + gv[m]];
                    pi[m] = -1;
                    for (int k = 0; k < 3; ++k)
                        if (tet_vid[4 * e + fv[k]] == h) pi[m] = k;
                }
                int oc = -1;
                for (int c = 0; c < 6; ++c)
                    if (kPerm3[c][0] == pi[0] && kPerm3[c][1] == pi[1] && kPerm3[c][2] == pi[2]) oc = c;
                if (oc < 0) {
                    err = "inconsistent face vertex ids";
                    return false;
                }
                nbr_c[s] = (int32_t)n;
                fcode_c[s] = (uint8_t)(fn | (oc << 2));
            }
        }
        i = j;
    }
    out.n_faces = nf;
    out.n_bfaces = nbf;
    // renumbering
    std::vector<int32_t> order;
    if (renumber == DG_ORDER_RCM) rcm_order(nbr_c, ne, order);
    else if (renumber == DG_ORDER_MORTON || renumber == DG_ORDER_HILBERT)
        curve_order(tet_xyz, ne, renumber == DG_ORDER_HILBERT, order);
    else { order.resize(ne); std::iota(order.begin(), order.end(), 0); }
    out.perm = order;
    out.iperm.assign(ne, -1);
    for (int64_t i = 0; i < ne; ++i) out.iperm[order[i]] = (int32_t)i;
    out.nbr.resize(4 * ne);
    out.fcode.resize(4 * ne);
    out.jinv.resize(9 * ne);
    int64_t bw0 = 0, bw1 = 0;
    for (int64_t i = 0; i < ne; ++i) {
        int64_t e = order[i];
        for (int f = 0; f < 4; ++f) {
            int32_t n = nbr_c[4 * e + f];
            if (n >= 0) {
                bw0 = std::max<int64_t>(bw0, std::llabs(e - n));
                int32_t ni = out.iperm[n];
                bw1 = std::max<int64_t>(bw1, std::llabs(i - ni));
                out.nbr[4 * i + f] = ni;
            } else {
                out.nbr[4 * i + f] = n;
            }
            out.fcode[4 * i + f] = fcode_c[4 * e + f];
        }
        for (int k = 0; k < 9; ++k) out.jinv[9 * i + k] = jinv_c[9 * e + k];
    }
    out.bw_before = bw0;
    out.bw_after = bw1;
    code = DG_OK;
    return true;
}

// Owners and canonical normals of the faces (the one-evaluation-per-face FP64/FP32 path).  A
// boundary face belongs to its element; an interior face to the element with the smaller caller
// index, so the choice, like every other input of the face flux, does not depend on the
// internal element order.  ncan holds the owner's outward unit normal -grad lambda_f /
// |grad lambda_f| (from the owner's J^-1) in both slots of the face.
void build_face_owners(const MeshHost& h, std::vector<uint8_t>& fown, std::vector<double>& ncan) {
    const int64_t ne = h.ne;
    fown.assign((size_t)4 * ne, 0);
    ncan.assign((size_t)12 * ne, 0.0);
    for (int64_t e = 0; e < ne; ++e)
        for (int f = 0; f < 4; ++f) {
            const int32_t n = h.nbr[4 * e + f];
            if (n >= 0 && h.perm[n] < h.perm[e]) continue;
            fown[4 * e + f] = 1;
            const double* I = h.jinv.data() + 9 * e;
            double g[3];
            for (int d = 0; d < 3; ++d) g[d] = f == 0 ? -(I[d] + I[3 + d] + I[6 + d]) : I[3 * (f - 1) + d];
            const double gn = std::sqrt(g[0] * g[0] + g[1] * g[1] + g[2] * g[2]);
            for (int d = 0; d < 3; ++d) {
                const double nd = -g[d] / gn;
                ncan[12 * e + 3 * f + d] = nd;
                if (n >= 0) ncan[12 * (int64_t)n + 3 * (h.fcode[4 * e + f] & 3) + d] = nd;
            }
        }
}

}  // namespace dg
