// Greedy min-fill elimination order (§Tensor network contraction: the order
// in which variables are summed out sets the size of the largest intermediate
// and so the cost; §Results calls its rank the contraction width).
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
#include <cmath>

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

// Eliminate every variable of `net` in the order `pick` chooses from the
// current (fill, degree, alive) arrays; returns the width and the cost
// sum_b 2^{|U_b|} (elements the bucket steps touch, up to a factor).
template <class Pick>
static int32_t greedy_eliminate(const Network& net, Pick pick, std::vector<int32_t>* order, double* cost) {
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
  double c = 0.0;
  std::vector<int32_t> nb, touched;
  std::vector<char> mark(n, 0);
  for (int32_t step = 0; step < n; ++step) {
    const int32_t v = pick(step, fill, deg, alive);
    nb.clear();
    G.for_each(v, [&](int32_t a) { nb.push_back(a); });
    width = std::max(width, (int32_t)nb.size());
    c += std::ldexp(1.0, (int)nb.size() + 1);
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
  if (cost) *cost = c;
  return width;
}

int32_t min_fill_order(const Network& net, std::vector<int32_t>* order, double* cost) {
  auto pick = [](int32_t, const std::vector<int64_t>& fill, const std::vector<int32_t>& deg,
                 const std::vector<char>& alive) {
    int32_t best = -1;
    for (int32_t v = 0; v < (int32_t)fill.size(); ++v) {
      if (!alive[v]) continue;
      if (best < 0 || fill[v] < fill[best] || (fill[v] == fill[best] && deg[v] < deg[best]))
        best = v;  // ascending scan keeps the smallest id on full ties
    }
    return best;
  };
  return greedy_eliminate(net, pick, order, cost);
}

// SplitMix64 (Steele, Lea and Flood, "Fast splittable pseudorandom number
// generators", 2014): a counter-based generator, so a trial's draws depend
// only on (seed, trial, step).
static uint64_t splitmix64(uint64_t x) {
  x += 0x9e3779b97f4a7c15ull;
  x = (x ^ (x >> 30)) * 0xbf58476d1ce4e5b9ull;
  x = (x ^ (x >> 27)) * 0x94d049bb133111ebull;
  return x ^ (x >> 31);
}

int32_t random_greedy_order(const Network& net, double tau, uint64_t seed, uint64_t trial,
                            std::vector<int32_t>* order, double* cost) {
  std::vector<double> wgt;
  auto pick = [&](int32_t step, const std::vector<int64_t>& fill, const std::vector<int32_t>& deg,
                  const std::vector<char>& alive) {
    // weight exp(-(f_v - f_min) / tau) with f = fill-in + degree / (n + 1)
    // (the degree breaks ties between equal fill-ins)
    const int32_t n = (int32_t)fill.size();
    double fmin = INFINITY;
    for (int32_t v = 0; v < n; ++v)
      if (alive[v]) fmin = std::min(fmin, (double)fill[v] + (double)deg[v] / (n + 1));
    wgt.assign(n, 0.0);
    double total = 0.0;
    for (int32_t v = 0; v < n; ++v) {
      if (!alive[v]) continue;
      const double f = (double)fill[v] + (double)deg[v] / (n + 1);
      const double x = (f - fmin) / tau;
      wgt[v] = x > 40.0 ? 0.0 : std::exp(-x);
      total += wgt[v];
    }
    const uint64_t r = splitmix64(splitmix64(splitmix64(seed) ^ trial) ^ (uint64_t)step);
    double u = (double)(r >> 11) * 0x1.0p-53 * total;
    int32_t last = -1;
    for (int32_t v = 0; v < n; ++v) {
      if (wgt[v] <= 0.0) continue;
      last = v;
      if (u < wgt[v]) return v;
      u -= wgt[v];
    }
    return last;  // rounding left u just above the total
  };
  return greedy_eliminate(net, pick, order, cost);
}

int32_t search_order(const Network& net, int32_t trials, double tau, uint64_t seed, int32_t w_cap,
                     std::vector<int32_t>* order, double* cost) {
  double best_cost = 0.0;
  int32_t best_w = min_fill_order(net, order, &best_cost);
  std::vector<int32_t> cand;
  for (int32_t t = 0; t < trials; ++t) {
    double c = 0.0;
    const int32_t w = random_greedy_order(net, tau, seed, (uint64_t)t, &cand, &c);
    if (w <= std::max(w_cap, best_w) && (c < best_cost || (c == best_cost && w < best_w))) {
      best_cost = c;
      best_w = w;
      order->swap(cand);
    }
  }
  if (cost) *cost = best_cost;
  return best_w;
}

}  // namespace qt
