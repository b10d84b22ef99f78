// Variable slicing: the width guard for networks above the width budget.
//
// §Tensor network contraction: the width of the contraction (the largest
// bucket result) sets memory and time.  When it is above the budget, a
// variable x is fixed: the network value is the sum over x = 0, 1 of the two
// networks in which every tensor holding x is restricted to that value.  Fixing
// s variables gives 2^s restricted networks with one shared structure and a
// smaller width; they differ only in the values of the restricted leaves.
#include <algorithm>

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

int32_t choose_slices(const Network& net, int32_t w_max, int32_t max_slices, std::vector<int32_t>* sliced) {
  sliced->clear();
  for (;;) {
    Network red;
    restrict_network(net, *sliced, 0u, &red);
    std::vector<int32_t> order;
    const int32_t w = min_fill_order(red, &order);
    if (w <= w_max || (int32_t)sliced->size() >= max_slices) return w;
    EdgePlan ep;
    if (make_edge_plan(red, order, &ep) != QT_OK) return w;
    // the variable that appears in the most of the widest bucket results
    std::vector<int32_t> count(red.n_vars, 0);
    for (const Bucket& b : ep.buckets)
      if (b.out_rank >= w - 1)
        for (int32_t v : b.out_vars) ++count[v];
    int32_t best = 0;
    for (int32_t v = 1; v < red.n_vars; ++v)
      if (count[v] > count[best]) best = v;
    // map the reduced id back to the original variable
    std::vector<int32_t> orig;
    std::vector<char> is_sliced(net.n_vars, 0);
    for (int32_t v : *sliced) is_sliced[v] = 1;
    for (int32_t v = 0; v < net.n_vars; ++v)
      if (!is_sliced[v]) orig.push_back(v);
    sliced->push_back(orig[best]);
  }
}

}  // namespace qt
