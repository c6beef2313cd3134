// Host planning: validation, rest shape, rotation clusters, pins, reordering and
// the sliced block pattern of the condensed matrix (paper §3 Eq. 5, 6, 12; §3.1).
#include "plan.h"

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <numeric>

namespace mfem {

namespace {

constexpr double kTieEps = 1.0e-10;

inline double dot3(const double* a, const double* b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

// Squared distance from P to the segment a-b.
double seg_dist2(const double* P, const double* a, const double* b) {
    double ab[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]};
    double pa[3] = {P[0] - a[0], P[1] - a[1], P[2] - a[2]};
    double t = dot3(pa, ab) / dot3(ab, ab);
    t = t < 0.0 ? 0.0 : (t > 1.0 ? 1.0 : t);
    double d[3] = {P[0] - (a[0] + t * ab[0]), P[1] - (a[1] + t * ab[1]), P[2] - (a[2] + t * ab[2])};
    return dot3(d, d);
}

struct Rig {
    int H = 0;
    const double* joints = nullptr;
    std::vector<std::pair<int, int>> bones;  // (proximal, distal), ordered by distal
    int rule = MFEM_CLUSTER_BONE;
    double tol = 0.0;

    // §3.1: nearest bone segment (or nearest joint, or nearest bone midpoint,
    // §4); a candidate wins only if closer by more than tol, so exact ties go to
    // the lowest index.
    int nearest(const double* P) const {
        bool use_bones = (rule == MFEM_CLUSTER_BONE || rule == MFEM_CLUSTER_MIDPOINT) && !bones.empty();
        int ncand = use_bones ? (int)bones.size() : H;
        double best = 0.0;
        int hbest = -1;
        for (int c = 0; c < ncand; ++c) {
            double d;
            int h;
            if (use_bones && rule == MFEM_CLUSTER_MIDPOINT) {
                const double* A = joints + 3 * bones[c].first;
                const double* B = joints + 3 * bones[c].second;
                double v[3] = {P[0] - 0.5 * (A[0] + B[0]), P[1] - 0.5 * (A[1] + B[1]), P[2] - 0.5 * (A[2] + B[2])};
                d = dot3(v, v);
                h = bones[c].first;
            } else if (use_bones) {
                d = seg_dist2(P, joints + 3 * bones[c].first, joints + 3 * bones[c].second);
                h = bones[c].first;
            } else {
                const double* J = joints + 3 * c;
                double v[3] = {P[0] - J[0], P[1] - J[1], P[2] - J[2]};
                d = dot3(v, v);
                h = c;
            }
            if (c == 0 || d < best - tol) {
                best = d;
                hbest = h;
            }
        }
        return hbest;
    }
};

bool finite_all(const double* a, size_t k) {
    for (size_t i = 0; i < k; ++i)
        if (!std::isfinite(a[i])) return false;
    return true;
}

// Inverse of a 3x3 row-major matrix by its adjugate; returns the determinant.
double inv3(const double* A, double* Ai) {
    double c00 = A[4] * A[8] - A[5] * A[7];
    double c01 = A[5] * A[6] - A[3] * A[8];
    double c02 = A[3] * A[7] - A[4] * A[6];
    double det = A[0] * c00 + A[1] * c01 + A[2] * c02;
    double id = 1.0 / det;
    Ai[0] = c00 * id;
    Ai[1] = (A[2] * A[7] - A[1] * A[8]) * id;
    Ai[2] = (A[1] * A[5] - A[2] * A[4]) * id;
    Ai[3] = c01 * id;
    Ai[4] = (A[0] * A[8] - A[2] * A[6]) * id;
    Ai[5] = (A[2] * A[3] - A[0] * A[5]) * id;
    Ai[6] = c02 * id;
    Ai[7] = (A[1] * A[6] - A[0] * A[7]) * id;
    Ai[8] = (A[0] * A[4] - A[1] * A[3]) * id;
    return det;
}

uint32_t spread10(uint32_t v) {  // 10 bits -> every third bit
    v &= 0x3ff;
    v = (v | (v << 16)) & 0x030000FF;
    v = (v | (v << 8)) & 0x0300F00F;
    v = (v | (v << 4)) & 0x030C30C3;
    v = (v | (v << 2)) & 0x09249249;
    return v;
}

uint32_t morton(const double* P, const double* lo, double inv_ext) {
    uint32_t c[3];
    for (int i = 0; i < 3; ++i) {
        double u = (P[i] - lo[i]) * inv_ext;
        int q = (int)(u * 1023.0);
        c[i] = (uint32_t)std::min(std::max(q, 0), 1023);
    }
    return spread10(c[0]) | (spread10(c[1]) << 1) | (spread10(c[2]) << 2);
}

}  // namespace

mfem_status plan_rig(const double* rest_verts, int32_t n, const int32_t* tets, int32_t m,
                     const mfem_handles* hs, Plan& p, std::string& err) {
    char buf[256];
    if (!rest_verts || !tets || !hs) { err = "null mesh or handles pointer"; return MFEM_EINVAL; }
    if (n < 4 || m < 1) { err = "mesh needs n >= 4 vertices and m >= 1 tets"; return MFEM_EINVAL; }
    if ((int64_t)m * 16 >= (int64_t)1 << 31) { err = "too many tets (16 m must fit int32)"; return MFEM_EINVAL; }
    if (!finite_all(rest_verts, (size_t)3 * n)) { err = "non-finite rest vertex coordinate"; return MFEM_EINVAL; }
    const int H = hs->n_handles;
    if (H < 1 || !hs->joints || !hs->parent) { err = "rig needs n_handles >= 1, joints and parent"; return MFEM_EINVAL; }
    if (!finite_all(hs->joints, (size_t)3 * H)) { err = "non-finite joint coordinate"; return MFEM_EINVAL; }
    for (int j = 0; j < H; ++j) {
        int pj = hs->parent[j];
        if (pj < -1 || pj >= H || pj == j) {
            snprintf(buf, sizeof buf, "parent[%d] = %d out of range", j, pj);
            err = buf;
            return MFEM_EINVAL;
        }
    }
    if (hs->cluster_rule != MFEM_CLUSTER_BONE && hs->cluster_rule != MFEM_CLUSTER_JOINT &&
        hs->cluster_rule != MFEM_CLUSTER_MIDPOINT) {
        err = "unknown cluster_rule";
        return MFEM_EINVAL;
    }
    for (int64_t i = 0; i < (int64_t)4 * m; ++i) {
        if (tets[i] < 0 || tets[i] >= n) {
            snprintf(buf, sizeof buf, "tet %lld vertex index %d out of range [0,%d)",
                     (long long)(i / 4), tets[i], n);
            err = buf;
            return MFEM_EINVAL;
        }
    }
    p.n = n;
    p.m = m;
    p.H = H;
    // bounding-box diagonal (tie margin scale)
    double lo[3] = {rest_verts[0], rest_verts[1], rest_verts[2]}, hi[3] = {lo[0], lo[1], lo[2]};
    for (int v = 0; v < n; ++v)
        for (int i = 0; i < 3; ++i) {
            lo[i] = std::min(lo[i], rest_verts[3 * v + i]);
            hi[i] = std::max(hi[i], rest_verts[3 * v + i]);
        }
    double ext[3] = {hi[0] - lo[0], hi[1] - lo[1], hi[2] - lo[2]};
    p.bbox_diag = std::sqrt(dot3(ext, ext));

    // rest shape: D_m columns X_a - X_0, W = det(D_m)/6 > 0 (Eq. 5)
    p.Dminv.assign((size_t)9 * m, 0.0);
    p.vol.assign(m, 0.0);
    for (int k = 0; k < m; ++k) {
        const double* X0 = rest_verts + 3 * tets[4 * k];
        double Dm[9];
        for (int c = 0; c < 3; ++c) {
            const double* Xa = rest_verts + 3 * tets[4 * k + 1 + c];
            for (int r = 0; r < 3; ++r) Dm[3 * r + c] = Xa[r] - X0[r];
        }
        double det = inv3(Dm, &p.Dminv[9 * (size_t)k]);
        p.vol[k] = det / 6.0;
        if (!(det > 0.0)) {
            snprintf(buf, sizeof buf, "rest tet %d has non-positive volume %.3e", k, det / 6.0);
            err = buf;
            return MFEM_EDEGEN;
        }
    }

    Rig rig;
    rig.H = H;
    rig.joints = hs->joints;
    rig.rule = hs->cluster_rule;
    rig.tol = kTieEps * p.bbox_diag * p.bbox_diag;
    for (int j = 0; j < H; ++j)
        if (hs->parent[j] >= 0) rig.bones.emplace_back(hs->parent[j], j);

    // tet clusters (§3.1) from barycenters, or the caller's override
    p.cluster_orig.assign(m, 0);
    if (hs->tet_cluster) {
        for (int k = 0; k < m; ++k) {
            int c = hs->tet_cluster[k];
            if (c < 0 || c >= H) {
                snprintf(buf, sizeof buf, "tet_cluster[%d] = %d out of range", k, c);
                err = buf;
                return MFEM_EINVAL;
            }
            p.cluster_orig[k] = c;
        }
    } else {
        for (int k = 0; k < m; ++k) {
            double b[3];
            for (int i = 0; i < 3; ++i) {
                double s = rest_verts[3 * tets[4 * k] + i] + rest_verts[3 * tets[4 * k + 1] + i];
                s += rest_verts[3 * tets[4 * k + 2] + i];
                s += rest_verts[3 * tets[4 * k + 3] + i];
                b[i] = s * 0.25;
            }
            p.cluster_orig[k] = rig.nearest(b);
        }
    }
    p.vhandle_orig.assign(n, 0);
    for (int v = 0; v < n; ++v) p.vhandle_orig[v] = rig.nearest(rest_verts + 3 * v);

    // pins: explicit list, or every vertex near a joint or a bone midpoint
    p.pinned_orig.assign(n, 0);
    p.pin_handle_orig.assign(n, -1);
    if (hs->pin_verts) {
        if (hs->n_pins < 0 || !hs->pin_handle) { err = "pin_verts needs pin_handle and n_pins >= 0"; return MFEM_EINVAL; }
        for (int i = 0; i < hs->n_pins; ++i) {
            int v = hs->pin_verts[i], h = hs->pin_handle[i];
            if (v < 0 || v >= n || h < 0 || h >= H) {
                snprintf(buf, sizeof buf, "pin %d (vertex %d, handle %d) out of range", i, v, h);
                err = buf;
                return MFEM_EINVAL;
            }
            if (p.pinned_orig[v]) {
                snprintf(buf, sizeof buf, "vertex %d pinned twice", v);
                err = buf;
                return MFEM_EINVAL;
            }
            p.pinned_orig[v] = 1;
            p.pin_handle_orig[v] = h;
        }
    } else {
        if (!(hs->pin_radius >= 0.0) || !std::isfinite(hs->pin_radius)) { err = "bad pin_radius"; return MFEM_EINVAL; }
        std::vector<double> centres(hs->joints, hs->joints + 3 * H);
        for (auto& b : rig.bones)
            for (int i = 0; i < 3; ++i)
                centres.push_back(0.5 * (hs->joints[3 * b.first + i] + hs->joints[3 * b.second + i]));
        double r2 = hs->pin_radius * hs->pin_radius + rig.tol;
        int nc = (int)centres.size() / 3;
        for (int v = 0; v < n; ++v) {
            const double* P = rest_verts + 3 * v;
            for (int c = 0; c < nc; ++c) {
                double d[3] = {P[0] - centres[3 * c], P[1] - centres[3 * c + 1], P[2] - centres[3 * c + 2]};
                if (dot3(d, d) <= r2) {
                    p.pinned_orig[v] = 1;
                    p.pin_handle_orig[v] = p.vhandle_orig[v];
                    break;
                }
            }
        }
    }
    return MFEM_OK;
}

mfem_status plan_layout(const mfem_material* mat, const double* rest_verts, const int32_t* tets,
                        Plan& p, std::string& err, int agg_request) {
    const int n = p.n, m = p.m;
    if (!mat) { err = "null material"; return MFEM_EINVAL; }
    if (mat->model < MFEM_ARAP || mat->model > MFEM_SNH) { err = "unknown material model"; return MFEM_EINVAL; }
    // --- Morton order of vertices, then tets by barycenter code ---
    double lo[3] = {rest_verts[0], rest_verts[1], rest_verts[2]}, hi[3] = {lo[0], lo[1], lo[2]};
    for (int v = 0; v < n; ++v)
        for (int i = 0; i < 3; ++i) {
            lo[i] = std::min(lo[i], rest_verts[3 * v + i]);
            hi[i] = std::max(hi[i], rest_verts[3 * v + i]);
        }
    double ext = std::max(hi[0] - lo[0], std::max(hi[1] - lo[1], hi[2] - lo[2]));
    double inv_ext = ext > 0 ? 1.0 / ext : 1.0;
    std::vector<uint32_t> code(n);
    for (int v = 0; v < n; ++v) code[v] = morton(rest_verts + 3 * v, lo, inv_ext);
    p.vinv.resize(n);
    std::iota(p.vinv.begin(), p.vinv.end(), 0);
    std::stable_sort(p.vinv.begin(), p.vinv.end(), [&](int a, int b) { return code[a] < code[b]; });
    p.vperm.resize(n);
    for (int i = 0; i < n; ++i) p.vperm[p.vinv[i]] = i;
    std::vector<uint32_t> tcode(m);
    for (int k = 0; k < m; ++k) {
        double b[3];
        for (int i = 0; i < 3; ++i)
            b[i] = 0.25 * (rest_verts[3 * tets[4 * k] + i] + rest_verts[3 * tets[4 * k + 1] + i] +
                           rest_verts[3 * tets[4 * k + 2] + i] + rest_verts[3 * tets[4 * k + 3] + i]);
        tcode[k] = morton(b, lo, inv_ext);
    }
    p.tinv.resize(m);
    std::iota(p.tinv.begin(), p.tinv.end(), 0);
    std::stable_sort(p.tinv.begin(), p.tinv.end(), [&](int a, int b) { return tcode[a] < tcode[b]; });
    p.tperm.resize(m);
    for (int i = 0; i < m; ++i) p.tperm[p.tinv[i]] = i;

    // --- reordered per-vertex and per-tet data ---
    p.X.resize((size_t)3 * n);
    p.vhandle.resize(n);
    p.pinned.assign(n, 0);
    for (int i = 0; i < n; ++i) {
        int o = p.vinv[i];
        for (int c = 0; c < 3; ++c) p.X[3 * (size_t)i + c] = rest_verts[3 * (size_t)o + c];
        p.vhandle[i] = p.vhandle_orig[o];
        p.pinned[i] = (uint8_t)p.pinned_orig[o];
        if (p.pinned[i]) {
            p.pin_vert.push_back(i);
            p.pin_handle.push_back(p.pin_handle_orig[o]);
        }
    }
    std::vector<double> Dm_old = p.Dminv, vol_old = p.vol;
    p.tet.resize((size_t)4 * m);
    p.cluster.resize(m);
    p.mu.resize(m);
    p.lam.resize(m);
    for (int k = 0; k < m; ++k) {
        int o = p.tinv[k];
        for (int a = 0; a < 4; ++a) p.tet[4 * (size_t)k + a] = p.vperm[tets[4 * (size_t)o + a]];
        for (int e = 0; e < 9; ++e) p.Dminv[9 * (size_t)k + e] = Dm_old[9 * (size_t)o + e];
        p.vol[k] = vol_old[o];
        p.cluster[k] = p.cluster_orig[o];
        double mu = mat->mu ? mat->mu[o] : mat->mu0;
        double la = mat->lambda ? mat->lambda[o] : mat->lambda0;
        if (!std::isfinite(mu) || !std::isfinite(la) || mu < 0.0 || la < 0.0) {
            err = "material constants must be finite and >= 0";
            return MFEM_EINVAL;
        }
        p.mu[k] = mu;
        p.lam[k] = la;
    }

    // --- block pattern: row i holds columns of every vertex sharing a tet ---
    std::vector<std::vector<int32_t>> nb(n);
    for (int k = 0; k < m; ++k)
        for (int a = 0; a < 4; ++a)
            for (int b = 0; b < 4; ++b) nb[p.tet[4 * (size_t)k + a]].push_back(p.tet[4 * (size_t)k + b]);
    p.nnz_blocks = 0;
    for (int i = 0; i < n; ++i) {
        auto& r = nb[i];
        std::sort(r.begin(), r.end());
        r.erase(std::unique(r.begin(), r.end()), r.end());
        p.nnz_blocks += (int64_t)r.size();
    }
    p.n_slices = (n + kSlice - 1) / kSlice;
    p.slice_ptr.assign(p.n_slices + 1, 0);
    p.slice_w.assign(p.n_slices, 0);
    for (int s = 0; s < p.n_slices; ++s) {
        int w = 0;
        for (int l = 0; l < kSlice; ++l) {
            int i = s * kSlice + l;
            if (i < n) w = std::max(w, (int)nb[i].size());
        }
        p.slice_w[s] = w;
        p.slice_ptr[s + 1] = p.slice_ptr[s] + (int64_t)w * kSlice;
    }
    const int64_t slots = p.slice_ptr[p.n_slices];
    if (slots >= ((int64_t)1 << 31)) { err = "pattern too large for int32 slot ids"; return MFEM_EINVAL; }
    p.sell_col.assign(slots, -1);
    p.diag_slot.assign(n, -1);
    p.slot_row.assign(slots, 0);
    for (int s = 0; s < p.n_slices; ++s)
        for (int64_t g = p.slice_ptr[s]; g < p.slice_ptr[s + 1]; ++g) p.slot_row[g] = (int32_t)(s * kSlice + (g - p.slice_ptr[s]) % kSlice);
    for (int i = 0; i < n; ++i) {
        int s = i / kSlice, l = i % kSlice;
        for (size_t k = 0; k < nb[i].size(); ++k) {
            int64_t slot = p.slice_ptr[s] + (int64_t)k * kSlice + l;
            p.sell_col[slot] = nb[i][k];
            if (nb[i][k] == i) p.diag_slot[i] = (int32_t)slot;
        }
    }
    // --- gather lists: which element blocks sum into each matrix block ---
    auto slot_of = [&](int i, int j) -> int64_t {
        const auto& r = nb[i];
        auto it = std::lower_bound(r.begin(), r.end(), j);
        return p.slice_ptr[i / kSlice] + (int64_t)(it - r.begin()) * kSlice + (i % kSlice);
    };
    std::vector<int32_t> cnt(slots + 1, 0);
    std::vector<int32_t> cslot((size_t)16 * m);
    for (int k = 0; k < m; ++k)
        for (int a = 0; a < 4; ++a)
            for (int b = 0; b < 4; ++b) {
                int64_t s = slot_of(p.tet[4 * (size_t)k + a], p.tet[4 * (size_t)k + b]);
                cslot[16 * (size_t)k + 4 * a + b] = (int32_t)s;
                cnt[s + 1]++;
            }
    p.contrib_ptr.assign(slots + 1, 0);
    for (int64_t s = 0; s < slots; ++s) p.contrib_ptr[s + 1] = p.contrib_ptr[s] + cnt[s + 1];
    p.contrib.assign((size_t)16 * m, 0);
    std::vector<int32_t> fill(p.contrib_ptr.begin(), p.contrib_ptr.end() - 1);
    for (int k = 0; k < m; ++k)  // tet-major, so each list is sorted by tet
        for (int c = 0; c < 16; ++c) p.contrib[fill[cslot[16 * (size_t)k + c]]++] = 16 * k + c;
    // diagonal and upper slots with their mirror slots (the lower block (j, i)
    // sums the transposes of the same element blocks as (i, j), in the same
    // tet order)
    {
        std::vector<std::pair<int64_t, int64_t>> up;
        up.reserve((size_t)(p.nnz_blocks / 2 + n));
        for (int i = 0; i < n; ++i)
            for (int j : nb[i])
                if (j >= i) up.emplace_back(slot_of(i, j), j > i ? slot_of(j, i) : -1);
        std::sort(up.begin(), up.end());
        p.up_slot.resize(up.size());
        p.up_mirror.resize(up.size());
        for (size_t t = 0; t < up.size(); ++t) {
            p.up_slot[t] = (int32_t)up[t].first;
            p.up_mirror[t] = (int32_t)up[t].second;
        }
    }
    // vertex incidence for the gradient gather
    p.vinc_ptr.assign(n + 1, 0);
    for (int k = 0; k < m; ++k)
        for (int a = 0; a < 4; ++a) p.vinc_ptr[p.tet[4 * (size_t)k + a] + 1]++;
    for (int i = 0; i < n; ++i) p.vinc_ptr[i + 1] += p.vinc_ptr[i];
    p.vinc.assign((size_t)4 * m, 0);
    std::vector<int32_t> vf(p.vinc_ptr.begin(), p.vinc_ptr.end() - 1);
    for (int k = 0; k < m; ++k)
        for (int a = 0; a < 4; ++a) p.vinc[vf[p.tet[4 * (size_t)k + a]]++] = 4 * k + a;

    // --- aggregates for the coarse space: runs of agg_size consecutive vertices
    // of the Morton order (spatially compact), the smallest power of two >= 64
    // that keeps 6 n_agg <= kCoarseMaxDof.  Rigid modes of the rest shape about
    // the centroid of the aggregate's free vertices; pins take no part.
    int agg = kCoarseUnit;
    while (6 * (int64_t)((n + agg - 1) / agg) > kCoarseMaxDof) agg *= 2;
    if (agg_request > agg) agg = agg_request;   // a power of two (checked by mfem_create)
    p.agg_size = agg;
    p.n_agg = (n + agg - 1) / agg;
    p.crel.assign((size_t)4 * n, 0.f);
    p.agg_handle.assign(p.n_agg, 0);
    for (int a = 0; a < p.n_agg; ++a) {
        const int i0 = a * agg, i1 = std::min(n, i0 + agg);
        double c[3] = {0, 0, 0};
        int nf = 0;
        for (int i = i0; i < i1; ++i)
            if (!p.pinned[i]) {
                for (int d = 0; d < 3; ++d) c[d] += p.X[3 * (size_t)i + d];
                ++nf;
            }
        for (int d = 0; d < 3; ++d) c[d] = nf ? c[d] / nf : p.X[3 * (size_t)i0 + d];
        std::vector<int> votes(p.H, 0);
        for (int i = i0; i < i1; ++i) {
            for (int d = 0; d < 3; ++d) p.crel[4 * (size_t)i + d] = (float)(p.X[3 * (size_t)i + d] - c[d]);
            p.crel[4 * (size_t)i + 3] = p.pinned[i] ? 0.f : 1.f;
            votes[p.vhandle[i]]++;
        }
        p.agg_handle[a] = (int32_t)(std::max_element(votes.begin(), votes.end()) - votes.begin());
    }
    p.cnb_ptr.assign(p.n_agg + 1, 0);
    p.cnb.clear();
    p.cnb_max = 0;
    for (int a = 0; a < p.n_agg; ++a) {
        std::vector<int32_t> js;
        for (int i = a * agg; i < std::min(n, (a + 1) * agg); ++i)
            for (int j : nb[i]) js.push_back(j / agg);
        std::sort(js.begin(), js.end());
        js.erase(std::unique(js.begin(), js.end()), js.end());
        p.cnb.insert(p.cnb.end(), js.begin(), js.end());
        p.cnb_ptr[a + 1] = (int32_t)p.cnb.size();
        p.cnb_max = std::max(p.cnb_max, (int32_t)js.size());
    }
    return MFEM_OK;
}

}  // namespace mfem
