// Host-side planning of one mesh: everything about the mesh and rig that does
// not change with the pose.  Pure C++ (no CUDA); used by mfem_create and by the
// host-only mfem_plan entry point.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/mfem.h"

namespace mfem {

// Rows of the sliced (SELL-32) block layout: 32 consecutive block rows form a
// slice; a slice stores its k-th block of every row together, so the 32 lanes
// of a warp read consecutive addresses.
constexpr int kSlice = 32;

struct Plan {
    int32_t n = 0, m = 0, H = 0;
    // --- caller order ---
    std::vector<int32_t> cluster_orig;     // [m] handle per tet
    std::vector<int32_t> pinned_orig;      // [n] 0/1
    std::vector<int32_t> pin_handle_orig;  // [n] handle or -1
    std::vector<int32_t> vhandle_orig;     // [n] handle the rest position clusters to
    // --- internal (reordered) order ---
    std::vector<int32_t> vperm;    // vperm[old] = new
    std::vector<int32_t> vinv;     // vinv[new] = old
    std::vector<int32_t> tperm;    // tperm[old] = new
    std::vector<int32_t> tinv;     // tinv[new] = old
    std::vector<int32_t> tet;      // [m][4] new vertex ids, new tet order
    std::vector<double> X;         // [n][3] rest positions, new order
    std::vector<double> Dminv;     // [m][9] row-major inverse rest edge matrix
    std::vector<double> vol;       // [m]
    std::vector<int32_t> cluster;  // [m]
    std::vector<double> mu, lam;   // [m]
    std::vector<int32_t> vhandle;  // [n]
    std::vector<uint8_t> pinned;   // [n]
    std::vector<int32_t> pin_vert, pin_handle;  // [p] (new vertex ids)
    // sliced block pattern of the Eq. 12 matrix
    int32_t n_slices = 0;
    std::vector<int64_t> slice_ptr;  // [n_slices+1] first slot of each slice
    std::vector<int32_t> slice_w;    // [n_slices] blocks per row (max in slice)
    std::vector<int32_t> sell_col;   // [slots] column block or -1
    std::vector<int32_t> diag_slot;  // [n] slot holding the diagonal block of a row
    std::vector<int32_t> slot_row;   // [slots] block row of each slot (padding slots too)
    int64_t nnz_blocks = 0;
    // element-block -> matrix-block gather lists
    std::vector<int32_t> contrib_ptr;  // [slots+1]
    std::vector<int32_t> contrib;      // [16 m] code: tet*16 + a*4 + b
    // assembly of the symmetric pattern: the diagonal and upper slots (column
    // >= row), by slot, each with the slot of its transposed block (-1 on the
    // diagonal)
    std::vector<int32_t> up_slot, up_mirror;
    std::vector<int32_t> vinc_ptr;     // [n+1]
    std::vector<int32_t> vinc;         // [4 m] code: tet*4 + a
    double bbox_diag = 0.0;
    // two-level preconditioner: aggregates of agg_size consecutive internal
    // (Morton-ordered) vertices, each carrying the six rigid modes of its rest
    // shape; n_agg = 0 when the mesh has no coarse space
    int32_t agg_size = 0, n_agg = 0;
    std::vector<float> crel;          // [n][4] X_i - c_a, w = 1 for a free vertex, 0 for a pin
    std::vector<int32_t> agg_handle;  // [n_agg] the handle most of the aggregate's vertices cluster to
    std::vector<int32_t> cnb_ptr, cnb;  // neighbour aggregates of each aggregate (sorted, incl. itself)
    int32_t cnb_max = 0;
};

// Largest coarse space (6 rigid modes per aggregate) the planner builds.
constexpr int kCoarseMaxDof = 6144;
// Aggregates never have fewer vertices than this (one unit of the restriction).
constexpr int kCoarseUnit = 64;

// Validation, rest precompute (Eq. 5), clustering (§3.1) and pins (Eq. 6).
// Fills the caller-order fields.  Returns MFEM_OK or an error with `err` set.
mfem_status plan_rig(const double* rest_verts, int32_t n, const int32_t* tets, int32_t m,
                     const mfem_handles* hs, Plan& p, std::string& err);

// Material constants, reordering and the sliced pattern (needs plan_rig first).
// agg_request: vertices per coarse aggregate (0 = smallest allowed; see
// mfem_options.coarse_agg).
mfem_status plan_layout(const mfem_material* mat, const double* rest_verts,
                        const int32_t* tets, Plan& p, std::string& err, int agg_request = 0);

}  // namespace mfem
