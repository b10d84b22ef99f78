// Bucket elimination plan of one network (§Tensor network contraction;
// R. Dechter, "Bucket elimination").
//
// Every tensor goes into the bucket of its earliest-eliminated variable.
// Processing variable v multiplies every tensor in its bucket and sums over
// v; the result, over U \ {v} (U = union of the bucket's indices), goes into
// the bucket of its own earliest variable, or is a scalar factor of the
// final value when U = {v}.
//
// Layout rule (no index permutation anywhere): the indices of every tensor
// are ordered by elimination position, earliest at bit 0.  Inside a bucket
// the eliminated variable is then bit 0 of each input, and the other input
// bits are a subsequence of the output bits, so an input element is found by
// extracting the input's bits from the output index (a fixed bit mask).
//
// The leaves of a bucket (rank-1/2 gate tensors, §Diagonal gate
// simplification) are folded into one small "leaf factor" over the union of
// their indices, materialised per angle set before the contraction.
#include <algorithm>
#include <numeric>

#include "qt_internal.h"

namespace qt {

qt_status make_edge_plan(const Network& net, const std::vector<int32_t>& order, EdgePlan* ep) {
  const int32_t n = net.n_vars;
  if ((int32_t)order.size() != n) return fail(QT_EINVAL, "order length differs from variable count");
  std::vector<int32_t> pos(n, -1);
  for (int32_t i = 0; i < n; ++i) {
    int32_t v = order[i];
    if (v < 0 || v >= n || pos[v] >= 0) return fail(QT_EINVAL, "order is not a permutation of the variables");
    pos[v] = i;
  }
  auto by_pos = [&](int32_t a, int32_t b) { return pos[a] < pos[b]; };

  // An item waiting in a bucket: a leaf tensor or an earlier bucket's result.
  struct Item {
    int32_t src;                 // tensor index (leaf) or producer bucket
    bool leaf;
    std::vector<int32_t> vars;   // sorted by elimination position
  };
  std::vector<std::vector<Item>> pending(n);
  std::vector<int32_t> constants;  // tensors with every slot fixed by slicing
  for (int32_t t = 0; t < (int32_t)net.tensors.size(); ++t) {
    const Tensor& T = net.tensors[t];
    Item it{t, true, {}};
    int32_t free_slots = 0;
    for (int32_t r = 0; r < T.rank; ++r)
      if (T.fix[r] < 0) {
        it.vars.push_back(T.v[r]);
        ++free_slots;
      }
    if (free_slots == 0) {
      constants.push_back(t);
      continue;
    }
    std::sort(it.vars.begin(), it.vars.end(), by_pos);
    it.vars.erase(std::unique(it.vars.begin(), it.vars.end()), it.vars.end());
    if ((int32_t)it.vars.size() != free_slots) return fail(QT_EINVAL, "tensor repeats a variable");
    pending[pos[it.vars[0]]].push_back(std::move(it));
  }
  if (n == 0) return fail(QT_EINVAL, "network has no free variable");
  // a constant multiplies the whole network: fold it into the first bucket's leaf factor
  for (int32_t t : constants) pending[0].push_back(Item{t, true, {}});

  ep->edge = net.edge;
  ep->width = 0;
  ep->buckets.assign(n, Bucket{});
  ep->scalars.clear();
  for (int32_t i = 0; i < n; ++i) {
    const int32_t v = order[i];
    Bucket& bk = ep->buckets[i];
    bk.var = v;
    std::vector<Item>& items = pending[i];
    if (items.empty()) return fail(QT_EINVAL, "variable " + std::to_string(v) + " appears in no tensor");
    std::vector<int32_t> U{v};
    for (auto& it : items) U.insert(U.end(), it.vars.begin(), it.vars.end());
    std::sort(U.begin(), U.end(), by_pos);
    U.erase(std::unique(U.begin(), U.end()), U.end());
    // U[0] == v: every item's first variable is v.
    bk.out_vars.assign(U.begin() + 1, U.end());
    bk.out_rank = (int32_t)bk.out_vars.size();
    if (bk.out_rank > 31) return fail(QT_EWIDTH, "bucket result rank above 31");
    ep->width = std::max(ep->width, bk.out_rank);
    auto mask_of = [&](const std::vector<int32_t>& vars) {
      uint32_t m = 0;
      size_t j = 0;
      for (size_t a = 1; a < vars.size(); ++a) {   // skip v at vars[0]
        while (bk.out_vars[j] != vars[a]) ++j;
        m |= 1u << j;
      }
      return m;
    };
    std::vector<int32_t> leaf_vars;
    for (auto& it : items) {
      if (it.leaf) {
        leaf_vars.insert(leaf_vars.end(), it.vars.begin(), it.vars.end());
        continue;
      }
      bk.in_src.push_back(it.src);
      bk.in_mask.push_back(mask_of(it.vars));
      bk.in_rank.push_back((int32_t)it.vars.size());
      ep->buckets[it.src].consumer = i;
    }
    bool any_leaf = false;
    for (auto& it : items) any_leaf |= it.leaf;
    if (any_leaf) {
      leaf_vars.push_back(v);  // the leaf factor always carries the eliminated variable (bit 0)
      std::sort(leaf_vars.begin(), leaf_vars.end(), by_pos);
      leaf_vars.erase(std::unique(leaf_vars.begin(), leaf_vars.end()), leaf_vars.end());
      bk.leaf_rank = (int32_t)leaf_vars.size();
      if (bk.leaf_rank > kMaxLeafRank) return fail(QT_EINVAL, "leaf factor rank above limit");
      for (auto& it : items) {
        if (!it.leaf) continue;
        const Tensor& T = net.tensors[it.src];
        LeafRef L;
        L.kind = T.kind;
        L.layer = T.layer;
        L.conj = T.conj;
        L.rank = T.rank;
        for (int32_t r = 0; r < 2; ++r) {
          L.bit[r] = -1;
          L.fix[r] = -1;
          if (r >= T.rank) continue;
          if (T.fix[r] >= 0)
            L.fix[r] = T.fix[r];
          else
            L.bit[r] = (int8_t)(std::find(leaf_vars.begin(), leaf_vars.end(), T.v[r]) - leaf_vars.begin());
        }
        bk.leaves.push_back(L);
      }
      if ((int32_t)bk.leaves.size() > kMaxLeaves) return fail(QT_EINVAL, "too many leaves in one bucket");
      bk.in_src.push_back(-1);
      bk.in_mask.push_back(mask_of(leaf_vars));
      bk.in_rank.push_back(bk.leaf_rank);
    }
    if ((int32_t)bk.in_src.size() > kMaxIn) return fail(QT_EINVAL, "bucket fan-in above limit");
    if (bk.out_rank == 0) {
      ep->scalars.push_back(i);
    } else {
      Item res{i, false, bk.out_vars};
      pending[pos[bk.out_vars[0]]].push_back(std::move(res));
    }
    items.clear();
    items.shrink_to_fit();
  }
  return QT_OK;
}

}  // namespace qt
