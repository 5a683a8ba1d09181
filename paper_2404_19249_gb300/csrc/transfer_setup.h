// Host-side structures around the transfer matrix I_H^h (Sec. 3.2, Algorithm 1; used in A_H = I^T A_h I of Sec. 3.3):
// the bucket grid used by the GPU point location, the transpose I^T, and the
// gather lists that evaluate the Galerkin product A_H = I^T A_h I on the GPU
// in two deterministic stages (W = A_h I, then A_H = I^T W).
#pragma once

#include <cstdint>
#include <vector>

#include "space.h"

namespace nas {

struct BucketGrid {
    double org[3], inv_h[3];
    int nb[3];
    std::vector<int64_t> bptr;   // [nbuckets+1]
    std::vector<int32_t> btet;   // coarse tets, ascending within a bucket
};

// Register every coarse tetrahedron in each bucket its bounding box meets.
void build_buckets(const HostSpace& C, BucketGrid& G);

// Load-balanced split of a segmented list (CSR-like `ptr` over nseg segments):
// each segment's entries are cut into consecutive pieces of at most `len`
// entries.  Pieces of segment a are [seg_piece[a], seg_piece[a+1]); piece q
// covers list entries [piece_start[q], piece_start[q+1]).  A GPU reduction then
// takes one warp per piece and sums a segment's piece results in order, so the
// work per warp is bounded whatever the segment lengths (the transfer lists are
// very uneven on graded meshes) and the result stays deterministic.
struct PieceMap {
    std::vector<int32_t> seg_piece;
    std::vector<int64_t> piece_start;
    int64_t npieces() const { return seg_piece.empty() ? 0 : seg_piece.back(); }
};
template <typename P>
void make_pieces(const std::vector<P>& ptr, int64_t len, PieceMap& pm);

struct GalerkinMaps {
    int64_t nH = 0;                      // coarse dofs
    // I^T as CSR over coarse dofs: fine rows and weights
    std::vector<int32_t> tptr, trow;
    std::vector<double> tval;
    // W = A I: pattern over fine rows, coarse columns; wrow = fine row of a slot
    std::vector<int32_t> wptr, wcol, wrow;
    std::vector<int64_t> w1ptr;          // stage-1 lists: q = p*4 + l
    std::vector<int32_t> w1con;
    // A_H pattern (coarse CSR) and stage-2 lists: r = s*4 + k
    std::vector<int32_t> hptr, hcol;
    std::vector<int64_t> h2ptr;
    std::vector<int32_t> h2con;
    // balanced pieces of the I^T rows and of the stage-2 lists
    PieceMap tpieces, h2pieces;
    int64_t wnnz() const { return wptr.empty() ? 0 : wptr.back(); }
    int64_t hnnz() const { return hptr.empty() ? 0 : hptr.back(); }
};

// icol/ival: [n_fine_dof][4] coarse dof (-1 = boundary) and weight.
void build_galerkin(const HostSpace& F, int64_t nH, const std::vector<int32_t>& icol,
                    const std::vector<double>& ival, GalerkinMaps& G);

}  // namespace nas
