// Device-side plan records shared by the host planner and the CUDA kernels.
//
// Data layout in HBM: every tensor of rank r is a dense array [2^r][B] of
// complex numbers (B = angle sets, innermost, contiguous).  Bit i of the row
// index is the tensor's i-th variable in elimination order, so the variable a
// bucket eliminates is bit 0 of each of its inputs (no index permutation ever).
#pragma once

#include <cstdint>

namespace qt {

constexpr int kDevMaxIn = 8;
constexpr int kDevMaxRuns = 6;
constexpr int kDevMaxLeaves = 16;

// One input of a bucket.  Its row index is (pext(y, mask) << 1) | x where y
// is the output row and x the eliminated variable.  pext is evaluated from
// up to kDevMaxRuns contiguous runs of the mask: run r copies `len` bits
// from bit `src` of y to bit `dst` of the input row.  nruns < 0 means the
// mask has more runs and is walked bit by bit.
struct DevInput {
  int64_t off;                 // element offset from the data base
  uint32_t mask;
  int32_t nruns;
  uint32_t run[kDevMaxRuns];   // src | len << 8 | dst << 16
  int32_t flags;               // kInLeaf: written before the launch, read through L1
  int32_t pad;
};
constexpr int32_t kInLeaf = 1;

// Work split of a bucket into warp tiles (same for every bucket of a plan,
// fixed by B).  A warp tile covers R = P * RP consecutive output rows,
// R a power of two and tiles aligned to R, so for row y = r0 + p*RP + i
// (i < RP) the input index pext(y) = pext(r0 + p*RP) + pext(i) with no carry:
// the first term is one table entry per pass, the second one register per lane.
//   Bv = vectors of VB angle sets per row (1 for B == 1)
//   Bv <= 32: RP = largest power of two <= 32 / Bv rows per pass; lane ->
//             (row i = lane / Bv, vector lane % Bv); lanes >= RP * Bv idle
//   Bv >  32: RP = 1; VC = ceil(Bv / 32) vector chunks per row
//   P = passes per tile (power of two), P * VC <= kLaneItems
constexpr int kLaneItems = 64;
struct TileGeom {
  int32_t B, Bv, RP, VC, P, R;
  int64_t data_elems;  // size of the data region, for the QT_DEVICE_CHECKS build
};

struct DevBucket {
  int64_t out_off;             // element offset of the output
  int64_t n_rows;              // 2^out_rank
  int32_t out_rank;
  int32_t n_in;
  int32_t dep;                 // bucket that must be complete before this one (-1: none)
  int32_t ntask;               // tiles of this bucket in the persistent queue
  DevInput in[kDevMaxIn];
};

// Leaf factor: product of the leaves of one bucket over the union of their
// variables, materialised per angle set.  A leaf is packed as
// kind | conj << 2 | rank << 3 | bit0 << 5 | bit1 << 10 | layer << 16.
struct DevLeafFactor {
  int64_t off;
  int32_t rank;
  int32_t n_leaves;
  uint32_t leaf[kDevMaxLeaves];
};

// Persistent-queue task.  tile >= 0: tile `tile` of bucket `bucket`.
// tile < 0: a group of -tile consecutive buckets of one edge chain, starting
// at `bucket`, each small enough for a single tile; one warp runs them in
// order with no global synchronisation between them.
struct DevTask {
  int32_t bucket;
  int32_t tile;
};

// Control words at the start of the workspace.
struct DevCtrl {
  int32_t head;      // next task of the persistent queue
  int32_t status;    // 0 ok, else a qt_status set by the device
  int32_t spins;     // diagnostic: bucket index of the wait that timed out
  int32_t bad_kind;  // QT_DEVICE_CHECKS build: 1 load, 2 store, 3 record; 0 none
  int32_t bad_bucket;
  int32_t bad_input;
  int64_t bad_index;
};

}  // namespace qt
