// Internal host-side structures of the lightcone tensor-network library.
// Method: arXiv:2106.15740 (§QAOA algorithm, §Tensor network contraction,
// §Diagonal gate simplification).
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "qtensor.h"

namespace qt {

// Thread-local error message helpers (capi.cpp).
qt_status fail(qt_status s, const std::string& msg);

// ---------------------------------------------------------------- graph ----
struct Graph {
  int32_t n = 0;
  std::vector<int32_t> eu, ev;              // edge endpoints, eu[i] < ev[i]
  std::vector<std::vector<int32_t>> adj;    // sorted neighbour lists
};
qt_status make_graph(const qt_graph* g, Graph* out);

// -------------------------------------------------------------- network ----
// One lightcone tensor.  Every tensor of this network has rank 1 or 2 and
// its value is a closed-form function of (kind, layer, conj) and the angles
// of its layer; the network stores structure only.
struct Tensor {
  int8_t kind;      // qt_tensor_kind
  int8_t rank;      // 1 or 2 index slots
  int8_t conj;      // 1 for the bra copy (elementwise complex conjugate)
  int8_t layer;     // 1..p for ZZ/MIX, 0 for PLUS, p for OBS
  int32_t v[2];     // variable ids; MIX: v[0] = new, v[1] = old (-1 for a fixed slot)
  int8_t fix[2] = {-1, -1};  // slot fixed to 0 or 1 by slicing (-1: free)
};

struct Network {
  int32_t p = 0;
  int32_t edge = -1;
  int32_t n_vars = 0;
  std::vector<Tensor> tensors;
  std::vector<double> gamma, beta;          // angles of a single evaluation (may be empty)
};

// Build the reverse-lightcone network of edge `edge` (structure only).
void build_lightcone(const Graph& g, int32_t p, int32_t edge, Network* net);
// Build the ket network of the single amplitude <x|psi> of the full circuit,
// x given as one byte (0 or 1) per qubit; `index` labels the network.
void build_amplitude_network(const Graph& g, int32_t p, const uint8_t* bits, int32_t index, Network* net);
// Interaction structure (pairwise cliques) of the amplitude <0...0|psi> in
// one of the qt_representation gate representations (ordering cost only).
void build_representation_network(const Graph& g, int32_t p, int32_t rep, Network* net);

// ---------------------------------------------------------------- order ----
// Greedy min-fill over the interaction graph; returns the width (and, if
// `cost` is given, sum_b 2^{|U_b|} over the buckets of the order).
int32_t min_fill_order(const Network& net, std::vector<int32_t>* order, double* cost = nullptr);
// One seeded randomised greedy order: each step draws the next variable
// with probability proportional to exp(-(f_v - f_min) / tau) (f: fill-in,
// degree as tie-break).  Returns the width and the cost as above.
int32_t random_greedy_order(const Network& net, double tau, uint64_t seed, uint64_t trial,
                            std::vector<int32_t>* order, double* cost = nullptr);
// Min-fill plus `trials` randomised orders: the cheapest whose width is at
// most max(w_cap, min-fill width).  Returns its width.
int32_t search_order(const Network& net, int32_t trials, double tau, uint64_t seed, int32_t w_cap,
                     std::vector<int32_t>* order, double* cost = nullptr);

// Slicing: the network with the variables `sliced` fixed to the bits of
// `assignment` (bit i for sliced[i]); the other variables keep their order
// and are renumbered 0.. in it.
void restrict_network(const Network& net, const std::vector<int32_t>& sliced, uint32_t assignment, Network* out);
// Choose variables to fix until the width of the rest is at most w_max (at
// most max_slices), keeping the order `base` of the whole network; returns
// the width reached and the elimination order of the restricted networks
// (restricted variable ids): `base` restricted, or a fresh order of the
// restricted network (min-fill, or searched with `trials` randomised orders)
// when that is cheaper.
int32_t choose_slices(const Network& net, int32_t w_max, int32_t max_slices, const std::vector<int32_t>& base,
                      int32_t trials, double tau, uint64_t seed, std::vector<int32_t>* sliced,
                      std::vector<int32_t>* order);

// ----------------------------------------------------------------- plan ----
constexpr int kMaxIn = 8;        // inputs per bucket (intermediates + one leaf factor)
constexpr int kMaxLeafRank = 10; // variables of one leaf factor
constexpr int kMaxLeaves = 16;   // leaves folded into one leaf factor

// A leaf folded into a bucket's leaf factor: value from (kind, layer, conj),
// bit positions of its variables inside the leaf factor's index.
struct LeafRef {
  int8_t kind, layer, conj, rank;
  int8_t bit[2];   // position of a free slot's variable in the leaf factor
  int8_t fix[2];   // fixed value of a sliced slot, -1 if free
};

// One bucket of bucket elimination (§Tensor network contraction): the
// product of its inputs summed over the eliminated variable.
struct Bucket {
  int32_t var;                       // eliminated variable
  int32_t out_rank;                  // |U| - 1
  std::vector<int32_t> out_vars;     // sorted by elimination position (bit 0 first)
  // inputs: intermediates (producer bucket id) and at most one leaf factor (-1)
  std::vector<int32_t> in_src;       // producer bucket index, or -1 for the leaf factor
  std::vector<uint32_t> in_mask;     // bit j set if out_vars[j] is an index of the input
  std::vector<int32_t> in_rank;      // rank of the input (includes the eliminated var)
  std::vector<LeafRef> leaves;       // leaves folded into the leaf factor
  int32_t leaf_rank = 0;             // rank of the leaf factor (0 if none)
  int32_t consumer = -1;             // bucket consuming the output (-1: scalar result)
};

struct EdgePlan {
  int32_t edge = -1;
  int32_t slices = 0;                // sliced variables of the edge (this network is one of 2^slices)
  int32_t width = 0;
  std::vector<Bucket> buckets;
  std::vector<int32_t> scalars;      // buckets whose result has rank 0
};

// Turn (network, order) into buckets (§Tensor network contraction).
qt_status make_edge_plan(const Network& net, const std::vector<int32_t>& order, EdgePlan* ep);

}  // namespace qt
