// Greedy min-fill elimination order (§Tensor network contraction: the order
// in which variables are summed out sets the size of the largest intermediate
// and so the cost, §Results "contraction width").
//
// Interaction graph: one vertex per variable, a clique on the variables of
// every tensor.  Step: pick the alive variable with the smallest
// (fill-in, degree, id), where fill-in is the number of non-adjacent pairs of
// its neighbours; record its degree (the rank of the bucket result); connect
// its neighbours pairwise; remove it.  Width = largest recorded degree.
//
// Adjacency is a bitset per variable; after an elimination only the
// neighbours of the eliminated variable and their neighbours can change
// fill-in, so only those are recounted.
#include <algorithm>

#include "qt_internal.h"

namespace qt {

namespace {

struct BitGraph {
  int32_t n, w;
  std::vector<uint64_t> bits;
  explicit BitGraph(int32_t n_) : n(n_), w((n_ + 63) / 64), bits((size_t)n_ * ((n_ + 63) / 64), 0) {}
  uint64_t* row(int32_t v) { return bits.data() + (size_t)v * w; }
  const uint64_t* row(int32_t v) const { return bits.data() + (size_t)v * w; }
  void set(int32_t a, int32_t b) { row(a)[b >> 6] |= 1ull << (b & 63); }
  void clear(int32_t a, int32_t b) { row(a)[b >> 6] &= ~(1ull << (b & 63)); }
  int32_t degree(int32_t v) const {
    int32_t d = 0;
    for (int32_t i = 0; i < w; ++i) d += __builtin_popcountll(row(v)[i]);
    return d;
  }
  template <class F>
  void for_each(int32_t v, F f) const {
    const uint64_t* r = row(v);
    for (int32_t i = 0; i < w; ++i) {
      uint64_t m = r[i];
      while (m) {
        int32_t b = __builtin_ctzll(m);
        f(i * 64 + b);
        m &= m - 1;
      }
    }
  }
  // Non-adjacent pairs among the neighbours of v.
  int64_t fill(int32_t v) const {
    int64_t missing = 0;
    const uint64_t* nv = row(v);
    for_each(v, [&](int32_t a) {
      const uint64_t* na = row(a);
      int32_t c = 0;
      for (int32_t i = 0; i < w; ++i) c += __builtin_popcountll(nv[i] & ~na[i]);
      missing += c - 1;  // a itself is in N(v) but not in N(a)
    });
    return missing / 2;
  }
};

}  // namespace

int32_t min_fill_order(const Network& net, std::vector<int32_t>* order) {
  const int32_t n = net.n_vars;
  BitGraph G(n);
  for (const Tensor& t : net.tensors)
    if (t.rank == 2 && t.v[0] >= 0 && t.v[1] >= 0 && t.v[0] != t.v[1]) {  // both slots free
      G.set(t.v[0], t.v[1]);
      G.set(t.v[1], t.v[0]);
    }
  std::vector<int64_t> fill(n);
  std::vector<int32_t> deg(n);
  std::vector<char> alive(n, 1);
  for (int32_t v = 0; v < n; ++v) {
    fill[v] = G.fill(v);
    deg[v] = G.degree(v);
  }
  order->clear();
  order->reserve(n);
  int32_t width = 0;
  std::vector<int32_t> nb, touched;
  std::vector<char> mark(n, 0);
  for (int32_t step = 0; step < n; ++step) {
    int32_t best = -1;
    for (int32_t v = 0; v < n; ++v) {
      if (!alive[v]) continue;
      if (best < 0 || fill[v] < fill[best] || (fill[v] == fill[best] && deg[v] < deg[best]))
        best = v;  // ascending scan keeps the smallest id on full ties
    }
    const int32_t v = best;
    nb.clear();
    G.for_each(v, [&](int32_t a) { nb.push_back(a); });
    width = std::max(width, (int32_t)nb.size());
    for (int32_t a : nb) {
      G.clear(a, v);
      for (int32_t b : nb)
        if (a != b) G.set(a, b);
    }
    std::fill(G.row(v), G.row(v) + G.w, 0ull);
    alive[v] = 0;
    order->push_back(v);
    // Recount fill-in for N(v) and their neighbours.
    touched.clear();
    for (int32_t a : nb) {
      if (!mark[a]) { mark[a] = 1; touched.push_back(a); }
      G.for_each(a, [&](int32_t b) {
        if (!mark[b]) { mark[b] = 1; touched.push_back(b); }
      });
    }
    for (int32_t u : touched) {
      mark[u] = 0;
      fill[u] = G.fill(u);
      deg[u] = G.degree(u);
    }
  }
  return width;
}

}  // namespace qt
