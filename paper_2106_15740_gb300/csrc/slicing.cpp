// Variable slicing: the width guard for networks above the width budget.
//
// §Tensor network contraction: the width of the contraction (the largest
// bucket result) sets memory and time.  When it is above the budget, a
// variable x is fixed: the network value is the sum over x = 0, 1 of the two
// networks in which every tensor holding x is restricted to that value.  Fixing
// s variables gives 2^s restricted networks with one shared structure and a
// smaller width; they differ only in the values of the restricted leaves.
#include <algorithm>
#include <cmath>

#include "qt_internal.h"

namespace qt {

void restrict_network(const Network& net, const std::vector<int32_t>& sliced, uint32_t assignment, Network* out) {
  std::vector<int32_t> fixv(net.n_vars, -1), remap(net.n_vars, -1);
  for (size_t i = 0; i < sliced.size(); ++i) fixv[sliced[i]] = (assignment >> i) & 1u;
  int32_t nv = 0;
  for (int32_t v = 0; v < net.n_vars; ++v)
    if (fixv[v] < 0) remap[v] = nv++;
  out->p = net.p;
  out->edge = net.edge;
  out->n_vars = nv;
  out->gamma = net.gamma;
  out->beta = net.beta;
  out->tensors.clear();
  for (const Tensor& t : net.tensors) {
    Tensor r = t;
    for (int32_t k = 0; k < t.rank; ++k) {
      if (t.fix[k] >= 0) continue;  // already fixed
      if (fixv[t.v[k]] >= 0) {
        r.fix[k] = (int8_t)fixv[t.v[k]];
        r.v[k] = -1;
      } else {
        r.v[k] = remap[t.v[k]];
      }
    }
    out->tensors.push_back(r);
  }
}

namespace {

// Bucket sets U_b (result variables plus the eliminated one) of eliminating
// the network's free variables in `order`: the fill-in graph of the order.
std::vector<std::vector<int32_t>> bucket_sets(const Network& net, const std::vector<int32_t>& order) {
  const int32_t n = net.n_vars;
  std::vector<int32_t> pos(n);
  for (int32_t i = 0; i < n; ++i) pos[order[i]] = i;
  std::vector<std::vector<int32_t>> nb(n);
  for (const Tensor& t : net.tensors)
    if (t.rank == 2 && t.v[0] >= 0 && t.v[1] >= 0 && t.v[0] != t.v[1]) {
      nb[t.v[0]].push_back(t.v[1]);
      nb[t.v[1]].push_back(t.v[0]);
    }
  std::vector<std::vector<int32_t>> sets(n);
  for (int32_t i = 0; i < n; ++i) {
    const int32_t v = order[i];
    std::vector<int32_t>& a = nb[v];
    std::sort(a.begin(), a.end());
    a.erase(std::unique(a.begin(), a.end()), a.end());
    std::vector<int32_t> later;
    for (int32_t u : a)
      if (pos[u] > i) later.push_back(u);
    // eliminating v connects its later neighbours pairwise
    for (int32_t u : later)
      for (int32_t x : later)
        if (u != x) nb[u].push_back(x);
    sets[i] = later;
    sets[i].push_back(v);
  }
  return sets;
}

// Sum over buckets of 2^|U_b \ S| (the elements a bucket step touches).
double order_cost(const std::vector<std::vector<int32_t>>& sets, const std::vector<char>& in_s) {
  double c = 0.0;
  for (const auto& U : sets) {
    int32_t k = 0;
    for (int32_t v : U) k += in_s[v] ? 0 : 1;
    if (k > 0) c += std::ldexp(1.0, k);
  }
  return c;
}

}  // namespace

// Width guard.  The order of the whole network is kept and variables are
// fixed one at a time: fixing x removes it from every bucket
// set that holds it, so the width can only go down.  Each step fixes the
// variable held by the most widest bucket results (ties: the largest drop in
// total bucket elements).  The restricted network's own order (min-fill, or
// the order search) is then tried as well; the cheaper of the two orders is
// returned.
int32_t choose_slices(const Network& net, int32_t w_max, int32_t max_slices, const std::vector<int32_t>& base,
                      int32_t trials, double tau, uint64_t seed, std::vector<int32_t>* sliced,
                      std::vector<int32_t>* order_out) {
  sliced->clear();
  const std::vector<int32_t>& order = base;
  const auto sets = bucket_sets(net, order);
  std::vector<char> in_s(net.n_vars, 0);
  auto width_now = [&]() {
    int32_t w = 0;
    for (const auto& U : sets) {
      int32_t k = 0;
      for (int32_t v : U) k += in_s[v] ? 0 : 1;
      w = std::max(w, k - 1);
    }
    return w;
  };
  int32_t w = width_now();
  while (w > w_max && (int32_t)sliced->size() < max_slices) {
    std::vector<int32_t> hits(net.n_vars, 0);
    std::vector<double> gain(net.n_vars, 0.0);
    for (const auto& U : sets) {
      int32_t k = 0;
      for (int32_t v : U) k += in_s[v] ? 0 : 1;
      if (k == 0) continue;
      // fixing a variable of U (other than one whose elimination this is: the
      // result loses it as well) halves this bucket
      for (size_t j = 0; j < U.size(); ++j) {
        const int32_t v = U[j];
        if (in_s[v]) continue;
        gain[v] += std::ldexp(1.0, k - 1);
        if (k - 1 == w && j + 1 < U.size()) ++hits[v];
      }
    }
    int32_t best = -1;
    for (int32_t v = 0; v < net.n_vars; ++v) {
      if (in_s[v]) continue;
      if (best < 0 || hits[v] > hits[best] || (hits[v] == hits[best] && gain[v] > gain[best])) best = v;
    }
    in_s[best] = 1;
    sliced->push_back(best);
    w = width_now();
  }
  std::sort(sliced->begin(), sliced->end());
  // the fixed order restricted to the free variables, in restricted ids
  std::vector<int32_t> remap(net.n_vars, -1);
  int32_t nv = 0;
  for (int32_t v = 0; v < net.n_vars; ++v)
    if (!in_s[v]) remap[v] = nv++;
  order_out->clear();
  for (int32_t v : order)
    if (!in_s[v]) order_out->push_back(remap[v]);
  if (sliced->empty()) return w;
  Network red;
  restrict_network(net, *sliced, 0u, &red);
  std::vector<int32_t> reorder;
  const int32_t w2 = trials > 0 ? search_order(red, trials, tau, seed ^ 0x5bd1e995ull, w_max, &reorder)
                                : min_fill_order(red, &reorder);
  if (w2 <= std::max(w, w_max)) {
    std::vector<char> none(red.n_vars, 0);
    const double c1 = order_cost(bucket_sets(red, *order_out), none);
    const double c2 = order_cost(bucket_sets(red, reorder), none);
    if (c2 < c1) {
      *order_out = reorder;
      return w2;
    }
  }
  return w;
}

}  // namespace qt
