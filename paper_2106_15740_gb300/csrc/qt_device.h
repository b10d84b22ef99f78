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
  int32_t flags;               // kIn* bits below
  int32_t pad;
};
constexpr int32_t kInLeaf = 1;    // written before the launch, read through L1
constexpr int32_t kInNoPair = 2;  // one row per output row (no eliminated-variable bit): an adjoint
constexpr int32_t kInF64 = 4;     // float-pair plans: an adjoint tensor (output adjoint or adjoint step
                                  // target), stored, accumulated and read as FP64

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
//   wait_limit = probes of one bounded wait on a ring barrier
struct TileGeom {
  int32_t B, Bv, RP, VC, P, R;
  int32_t wait_limit;
  int64_t data_elems;  // size of the data region, for the QT_DEVICE_CHECKS build
};

// Step kinds of a network's steps.
//   kStepFwd : bucket product-sum, out[y] = sum_x prod_i in_i[(pext(y) << 1) | x]
//   kStepAdj : adjoint of one input t of a bucket (reverse sweep): for every
//              output row y of the bucket, c_x = Gbar[y] * prod_{i != t} in_i
//              at x = 0, 1 goes to row (pext(y, mask_t) << 1) | x of t's
//              adjoint -- a plain store if t holds every output variable
//              (kAdjFull), an atomic add otherwise.  in[0..n_in-1] are the
//              factors (Gbar first, flagged kInNoPair, unless kAdjUnitG),
//              in[n_in] describes the target (mask and runs; off = out_off).
//   kStepZero: clear n_rows x B elements at out_off (an atomic target).
//   kStepAdjRed: the adjoint of a target t that lacks some of the bucket's
//              variables, as a reduction over the combined space of target
//              rows k_t (2^tgt_bits) and completions c (2^comp_bits values of
//              the missing variables, bits of the complement mask), row index
//              k_t * 2^comp_bits + c, y = pdep(k_t, mask_t) | pdep(c, ~mask_t);
//              lanes sum while k_t stays fixed and add one atomic per target
//              element at each change of k_t.  in[n_in] is the target record,
//              in[n_in + 1] the complement record.
//              With kAdjRedLow (one angle set): the lanes take the bucket's
//              five lowest variables instead, so a warp's loads of the output
//              adjoint are contiguous.  Row q = (h << 5) | lane with the pass
//              index h = k_h * 2^comp_bits + c_h, y = lane | pdep(c_h,
//              in[n_in + 1].mask) | pdep(k_h, in[n_in + 2].mask): the
//              completion and target bits above bit 4 (comp_bits and tgt_bits
//              count them).  Lanes sum over the passes of one k_h, then over
//              their completion bits (a butterfly), and the lanes whose
//              completion bits are 0 add one atomic per target element.
//   kStepFwd with chain = m > 0: bucket b fused with the chain c_1 .. c_m
//              that eliminates its result: c_1 is b's consumer, c_j the
//              consumer of c_(j-1), each with no variable beyond its input's
//              (U_(c_j) = the output variables of c_(j-1)) and no other
//              intermediate input, so c_j eliminates bit j - 1 of b's rows.
//              The step iterates b's rows y (n_rows = 2^out_rank of b) and
//              writes c_m's row y >> m at out_off.  With G_0 = G_b (the
//              product-sum above, never stored):
//              G_j[y >> j] = sum_w G_(j-1)[(y >> (j-1)) | w] * L_j[pext(y', in[n_in + j - 1].mask)]
//              for y' = y with bit j - 1 set to w: L_j is c_j's leaf factor,
//              its mask over b's rows (bit j - 1 = w at bit 0 of the index),
//              or 1 when bit j - 1 of chain_noleaf is set.
constexpr int32_t kStepFwd = 0, kStepAdj = 1, kStepZero = 2, kStepAdjRed = 3;
constexpr int32_t kAdjFull = 1, kAdjUnitG = 2, kAdjRedLow = 4;
constexpr int kMaxChain = 3;  // consumers fused into one forward step at most

struct DevBucket {
  int64_t out_off;             // element offset of the output
  int64_t n_rows;              // rows iterated: 2^out_rank of the bucket
  int32_t out_rank;
  int32_t n_in;                // factors (for kStepAdj the target follows them)
  int32_t dep;                 // first entry of the step's list in the plan's dependency array
  int32_t ntask;               // chunks of this step in the persistent queue (its done count)
  int32_t kind;                // kStep*
  int32_t aflags;              // kAdj* bits (adjoint steps)
  int32_t tgt_bits;            // kStepAdjRed: target rows 2^tgt_bits (times x = 0, 1); kAdjRedLow: target bits above bit 4
  int32_t comp_bits;           // kStepAdjRed: completions per target row 2^comp_bits (>= 5); kAdjRedLow: completion bits above bit 4
  int32_t span;                // warp tiles per queue task (chunk c covers tiles [c*span, (c+1)*span))
  int32_t n_dep;               // steps that must be complete before a task of this one starts:
                               // deps[dep .. dep + n_dep) (done count of each = its ntask)
  int32_t chain;               // kStepFwd: consumers fused into the step (0 .. kMaxChain)
  int32_t chain_noleaf;        // kStepFwd: bit j - 1 set if consumer c_j has no leaf factor
  DevInput in[kDevMaxIn];
};

// Warp tiles of a step: chunks of R of its n_rows.
inline int64_t step_tiles(const DevBucket& d, int64_t R) { return (d.n_rows + R - 1) / R; }

// Leaf factor: product of the leaves of one bucket over the union of their
// variables, materialised per angle set.  A leaf is packed as
// kind | conj << 2 | rank << 3 | bit0 << 5 | bit1 << 10 | fixed0 << 15 |
// value0 << 16 | fixed1 << 17 | value1 << 18 | layer << 19, where slot r reads
// bit `bit r` of the factor's index unless slicing fixed it to `value r`.
struct DevLeafFactor {
  int64_t off;
  int32_t rank;
  int32_t n_leaves;
  int32_t net;                 // network the factor belongs to (its leaf-count row)
  int32_t pad;
  uint32_t leaf[kDevMaxLeaves];
};

// Angle table: per angle set b and layer q, kTrigStride doubles at
// trig[(b * p + q) * kTrigStride]: cos g, sin g, cos b, sin b (the values the
// leaves take), log r_g, log r_b (see trig_kernel_f32: each stored gate is
// r times the exact gate at a nearby angle; complex128 plans have r = 1).
constexpr int kTrigStride = 6;

// Leaf counts of network k: 2p + 1 int32 at counts[k * (2p + 1)]: ZZ leaves
// of layers 1..p, mixer leaves of layers 1..p, |+> leaves (ket and bra
// copies all counted).  A network built from stored gates r x exact gate is
// prod r^count times the exact network: energy_kernel and leafgrad_kernel
// divide that product out in FP64.

// Persistent-queue task (16 bytes, one load).  chunk >= 0: chunk `chunk` of step `bucket`, its
// warp tiles [chunk * span, (chunk + 1) * span).  chunk < 0: a group of
// -chunk consecutive steps of one network, starting at `bucket`, each small
// enough for a single tile; one warp runs them in order with no global
// synchronisation between them.
struct DevTask {
  int32_t bucket;
  int32_t chunk;
  int32_t dep;                 // the step's dependency list: deps[dep .. dep + n_dep) (a group:
  int32_t n_dep;               // its first step's list; the others wait on nothing)
};

// One entry of a dependency list: the step waited for and the done count
// that completes it (its number of queue tasks).
struct DevDep {
  int32_t step;
  int32_t need;
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
