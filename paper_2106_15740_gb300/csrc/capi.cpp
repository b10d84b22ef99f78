// extern "C" entry points declared in include/qtensor.h.  Argument checks,
// handle management and error reporting; the work is in network.cpp,
// order.cpp, buckets.cpp, engine.cpp and the CUDA kernels.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <functional>
#include <new>
#include <thread>

#include "engine.h"
#include "kernels_api.h"

namespace qt {

static thread_local std::string g_last_error;

qt_status fail(qt_status s, const std::string& msg) {
  g_last_error = msg;
  return s;
}

static qt_status check_angles(const double* a, int64_t n, const char* name) {
  if (!a) return fail(QT_EINVAL, std::string(name) + " is NULL");
  for (int64_t i = 0; i < n; ++i)
    if (!std::isfinite(a[i])) return fail(QT_EINVAL, std::string(name) + " has a non-finite angle");
  return QT_OK;
}

// Build, order and bucket-plan every edge network of a graph.  The order is
// greedy min-fill, or the cheapest of min-fill and `order_trials` seeded
// randomised greedy orders that are no wider.  An edge above the width budget
// is rejected, or, with slicing, fixed variables are chosen until the rest
// fits and its 2^s restricted networks are planned (one order for all of
// them: they share the structure).  Edges are planned on host threads.
static constexpr int32_t kMaxSlices = 20;

struct EdgeResult {
  std::vector<EdgePlan> nets;
  int32_t width = 0, n_sliced = 0;
  qt_status st = QT_OK;
  std::string msg;
};

// Builds the network of unit e (an edge lightcone, or a bitstring's amplitude).
using NetBuilder = std::function<void(int32_t, Network*)>;

static void plan_one_edge(const NetBuilder& build, const char* unit, int32_t e, const qt_plan_options& o,
                          EdgeResult* r) {
  Network net;
  build(e, &net);
  const uint64_t seed = ((uint64_t)(uint32_t)o.order_seed << 32) ^ (uint64_t)(uint32_t)e;
  const double tau = o.order_tau > 0 ? o.order_tau : 1.0;
  std::vector<int32_t> order;
  int32_t w = o.order_trials > 0 ? search_order(net, o.order_trials, tau, seed, 0, &order)
                                 : min_fill_order(net, &order);
  std::vector<int32_t> sliced;
  if (w > o.max_width) {
    if (!o.slice) {
      r->st = QT_EWIDTH;
      r->msg = std::string(unit) + " " + std::to_string(e) + " has contraction width " + std::to_string(w) +
               " above the budget " + std::to_string(o.max_width);
      return;
    }
    const std::vector<int32_t> base = order;
    w = choose_slices(net, o.max_width, kMaxSlices, base, o.order_trials, tau, seed, &sliced, &order);
    if (w > o.max_width) {
      r->st = QT_EWIDTH;
      r->msg = std::string(unit) + " " + std::to_string(e) + " needs more than " + std::to_string(kMaxSlices) +
               " sliced variables to reach width " + std::to_string(o.max_width);
      return;
    }
  }
  const uint32_t n_slices = 1u << sliced.size();
  r->nets.reserve(n_slices);
  for (uint32_t a = 0; a < n_slices; ++a) {
    EdgePlan ep;
    qt_status st;
    if (sliced.empty()) {
      st = make_edge_plan(net, order, &ep);
    } else {
      Network rn;
      restrict_network(net, sliced, a, &rn);
      st = make_edge_plan(rn, order, &ep);
    }
    if (st != QT_OK) {
      r->st = st;
      r->msg = g_last_error;  // this thread's message
      return;
    }
    ep.edge = e;
    ep.slices = (int32_t)sliced.size();
    r->nets.push_back(std::move(ep));
  }
  r->width = w;
  r->n_sliced = (int32_t)sliced.size();
}

static qt_status plan_units(const NetBuilder& build, const char* unit, const qt_plan_options& o, int32_t e0,
                            int32_t e1, Plan* P) {
  const int32_t m = e1 - e0;
  std::vector<EdgeResult> res(m);
  const int32_t hw = (int32_t)std::max(1u, std::thread::hardware_concurrency());
  const int32_t n_threads = std::min({hw, m, 64});
  std::atomic<int32_t> next{0};
  auto worker = [&]() {
    for (int32_t k = next.fetch_add(1); k < m; k = next.fetch_add(1)) plan_one_edge(build, unit, e0 + k, o, &res[k]);
  };
  if (n_threads <= 1) {
    worker();
  } else {
    std::vector<std::thread> pool;
    for (int32_t t = 0; t < n_threads; ++t) pool.emplace_back(worker);
    for (auto& t : pool) t.join();
  }
  P->edges.clear();
  P->widths.clear();
  P->slices.clear();
  P->net_first.assign(1, 0);
  for (int32_t k = 0; k < m; ++k) {
    EdgeResult& r = res[k];
    if (r.st != QT_OK) return fail(r.st, r.msg);
    for (EdgePlan& ep : r.nets) P->edges.push_back(std::move(ep));
    P->widths.push_back(r.width);
    P->slices.push_back(r.n_sliced);
    P->net_first.push_back((int32_t)P->edges.size());
  }
  P->n_orig = m;
  return QT_OK;
}

}  // namespace qt

using namespace qt;

extern "C" {

const char* qt_last_error(void) { return g_last_error.c_str(); }

qt_status qt_build_lightcone(const qt_graph* g, int32_t p, const double* gamma, const double* beta, int32_t edge,
                             qt_network** out) {
  if (!out) return fail(QT_EINVAL, "out is NULL");
  if (p < 1 || p > 64) return fail(QT_EINVAL, "p must be in [1, 64]");
  Graph G;
  qt_status st = make_graph(g, &G);
  if (st != QT_OK) return st;
  if (edge < 0 || edge >= (int32_t)G.eu.size()) return fail(QT_EINVAL, "edge index out of range");
  if ((st = check_angles(gamma, p, "gamma")) != QT_OK) return st;
  if ((st = check_angles(beta, p, "beta")) != QT_OK) return st;
  qt_network* h = new (std::nothrow) qt_network;
  if (!h) return fail(QT_ENOMEM, "host allocation failed");
  build_lightcone(G, p, edge, &h->net);
  h->net.gamma.assign(gamma, gamma + p);
  h->net.beta.assign(beta, beta + p);
  *out = h;
  return QT_OK;
}

qt_status qt_network_info(const qt_network* net, int32_t* n_vars, int32_t* n_tensors) {
  if (!net) return fail(QT_EINVAL, "network is NULL");
  if (n_vars) *n_vars = net->net.n_vars;
  if (n_tensors) *n_tensors = (int32_t)net->net.tensors.size();
  return QT_OK;
}

qt_status qt_network_tensor(const qt_network* net, int32_t t, int32_t* kind, int32_t* layer, int32_t* conj,
                            int32_t* rank, int32_t vars[2]) {
  if (!net) return fail(QT_EINVAL, "network is NULL");
  if (t < 0 || t >= (int32_t)net->net.tensors.size()) return fail(QT_EINVAL, "tensor index out of range");
  const Tensor& T = net->net.tensors[t];
  if (kind) *kind = T.kind;
  if (layer) *layer = T.layer;
  if (conj) *conj = T.conj;
  if (rank) *rank = T.rank;
  if (vars) {
    vars[0] = T.v[0];
    vars[1] = T.rank > 1 ? T.v[1] : -1;
  }
  return QT_OK;
}

qt_status qt_order(const qt_network* net, int32_t* order, int32_t* n_vars, int32_t* width) {
  if (!net || !order) return fail(QT_EINVAL, "network or order is NULL");
  std::vector<int32_t> o;
  const int32_t w = min_fill_order(net->net, &o);
  std::copy(o.begin(), o.end(), order);
  if (n_vars) *n_vars = net->net.n_vars;
  if (width) *width = w;
  return QT_OK;
}

static qt_status contract_plan(const qt_network* net, const int32_t* order, qt_dtype dtype, Plan* P) {
  if (!net || !order) return fail(QT_EINVAL, "network or order is NULL");
  if (dtype != QT_C128 && dtype != QT_C64 && dtype != QT_C64X2) return fail(QT_EINVAL, "unknown dtype");
  std::vector<int32_t> o(order, order + net->net.n_vars);
  EdgePlan ep;
  qt_status st = make_edge_plan(net->net, o, &ep);
  if (st != QT_OK) return st;
  qt_plan_options_default(&P->opt);
  P->opt.dtype = dtype;
  P->opt.mode = QT_MODE_PER_BUCKET;
  P->opt.lane_items = 16;
  P->p = net->net.p;
  P->elem_bytes = dtype == QT_C64 ? 8 : 16;  // complex128 and float pairs: 16 bytes
  P->widths = {ep.width};
  P->slices = {0};
  P->edges.push_back(std::move(ep));
  P->n_orig = 1;
  P->net_first = {0, 1};
  return compile_plan(P);
}

qt_status qt_contract_workspace_size(const qt_network* net, const int32_t* order, qt_dtype dtype, size_t* bytes) {
  if (!bytes) return fail(QT_EINVAL, "bytes is NULL");
  Plan P;
  qt_status st = contract_plan(net, order, dtype, &P);
  if (st != QT_OK) return st;
  *bytes = P.ws.total;
  return QT_OK;
}

qt_status qt_contract(qt_network* net, const int32_t* order, qt_dtype dtype, void* stream, void* workspace,
                      size_t ws_bytes, double out_zz[2]) {
  if (!out_zz) return fail(QT_EINVAL, "out_zz is NULL");
  if (!net || net->net.gamma.size() != (size_t)net->net.p) return fail(QT_EINVAL, "network has no angles");
  Plan P;
  qt_status st = contract_plan(net, order, dtype, &P);
  if (st != QT_OK) return st;
  double energy = 0.0, zz[2] = {0.0, 0.0};
  qt_plan h;
  h.P = std::move(P);
  st = qt_plan_energy_host(&h, net->net.gamma.data(), net->net.beta.data(), &energy, zz, nullptr, workspace,
                           ws_bytes, stream);
  if (st != QT_OK) return st;
  out_zz[0] = zz[0];
  out_zz[1] = zz[1];
  return QT_OK;
}

void qt_network_free(qt_network* net) { delete net; }

void qt_plan_options_default(qt_plan_options* opt) {
  if (!opt) return;
  opt->batch = 1;
  opt->dtype = QT_C128;
  opt->mode = QT_MODE_PER_BUCKET;
  opt->gradient = 0;
  opt->max_width = 31;
  opt->lane_items = 0;
  opt->max_workspace = 0;
  opt->group_rows = 0;
  opt->edge_begin = 0;
  opt->edge_end = 0;
  opt->slice = 0;
  opt->chunk_tiles = 0;
  opt->order_trials = 0;
  opt->order_seed = 0;
  opt->order_tau = 1.0;
  opt->checkpoint_bytes = 0;
  opt->chain_steps = 0;
  opt->queue_order = 2;
  for (int32_t r = 0; r < 32; ++r) opt->chunk_tiles_by_rank[r] = 0;
  opt->fuse_chains = kMaxChain;
}

static qt_status check_options(const qt_plan_options* opt, qt_plan_options* out) {
  qt_plan_options o;
  qt_plan_options_default(&o);
  if (opt) o = *opt;
  if (o.batch < 1) return fail(QT_EINVAL, "batch must be >= 1");
  if (o.dtype != QT_C128 && o.dtype != QT_C64 && o.dtype != QT_C64X2) return fail(QT_EINVAL, "unknown dtype");
  if (o.dtype == QT_C64X2 && o.gradient && o.batch > 16)
    return fail(QT_EINVAL, "float-pair (QT_C64X2) gradient plans take at most 16 angle sets");
  if (o.mode != QT_MODE_PER_BUCKET && o.mode != QT_MODE_PERSISTENT) return fail(QT_EINVAL, "unknown mode");
  if (o.max_width <= 0 || o.max_width > 31) o.max_width = 31;
  if (o.lane_items > 0 && o.lane_items != 8 && o.lane_items != 16 && o.lane_items != 32 && o.lane_items != 64)
    return fail(QT_EINVAL, "lane_items must be 8, 16, 32 or 64");
  // by batch: one angle set in a complex64 persistent plan takes 32 passes of 32 rows per tile
  // (measured on the 60-vertex p = 4 graph: 16 passes 1.99 / 10.3 ms, 32 passes 1.72 / 9.10 ms,
  // 64 passes 2.00 / 10.3 ms for the energy / energy + gradient); complex128 and float pairs, whose
  // tiles take longer, and the per-bucket launches keep 16 (32 made them slower: per-bucket
  // complex128 loop 19.4 -> 31.1 s per bench step, complex128 amplitudes 5.1 -> 6.3 ms);
  // 2..15 angle sets 16 items, 16 or more 32
  if (o.lane_items <= 0)
    o.lane_items = (o.batch >= 16 || (o.batch == 1 && o.dtype == QT_C64 && o.mode == QT_MODE_PERSISTENT)) ? 32 : 16;
  if (o.order_trials < 0 || o.order_trials > 100000) return fail(QT_EINVAL, "order_trials must be in [0, 100000]");
  if (!(o.order_tau >= 0.0) || !std::isfinite(o.order_tau)) return fail(QT_EINVAL, "order_tau must be finite and >= 0");
  if (o.checkpoint_bytes < 0) return fail(QT_EINVAL, "checkpoint_bytes must be >= 0");
  if (o.chain_steps != 0 && o.chain_steps != 1) return fail(QT_EINVAL, "chain_steps must be 0 or 1");
  if (o.queue_order < 0 || o.queue_order > 2) return fail(QT_EINVAL, "queue_order must be 0, 1 or 2");
  if (o.fuse_chains < 0 || o.fuse_chains > kMaxChain)
    return fail(QT_EINVAL, "fuse_chains must be 0 .. " + std::to_string(kMaxChain));
  for (int32_t r = 0; r < 32; ++r)
    if (o.chunk_tiles_by_rank[r] < 0 || o.chunk_tiles_by_rank[r] > (1 << 20))
      return fail(QT_EINVAL, "chunk_tiles_by_rank entries must be in [0, 2^20]");
  *out = o;
  return QT_OK;
}

qt_status qt_plan_create(const qt_graph* g, int32_t p, const qt_plan_options* opt, qt_plan** out) {
  if (!out) return fail(QT_EINVAL, "out is NULL");
  if (p < 1 || p > 64) return fail(QT_EINVAL, "p must be in [1, 64]");
  qt_plan_options o;
  qt_status st0 = check_options(opt, &o);
  if (st0 != QT_OK) return st0;
  qt_plan* h = new (std::nothrow) qt_plan;
  if (!h) return fail(QT_ENOMEM, "host allocation failed");
  qt_status st = make_graph(g, &h->P.G);
  if (st == QT_OK) {
    h->P.p = p;
    h->P.opt = o;
    h->P.elem_bytes = o.dtype == QT_C64 ? 8 : 16;
    const int32_t m = (int32_t)h->P.G.eu.size();
    const int32_t e1 = o.edge_end <= 0 ? m : o.edge_end;
    if (o.edge_begin < 0 || o.edge_begin >= e1 || e1 > m) {
      st = fail(QT_EINVAL, "edge range out of bounds");
    } else {
      h->P.opt.edge_begin = o.edge_begin;
      h->P.opt.edge_end = e1;
      const Graph& G = h->P.G;
      st = plan_units([&](int32_t e, Network* net) { build_lightcone(G, p, e, net); }, "edge", o, o.edge_begin, e1,
                      &h->P);
    }
  }
  if (st == QT_OK) st = compile_plan(&h->P);
  if (st != QT_OK) {
    delete h;
    return st;
  }
  *out = h;
  return QT_OK;
}

qt_status qt_amplitude_plan_create(const qt_graph* g, int32_t p, const uint8_t* bits, int32_t n_strings,
                                   const qt_plan_options* opt, qt_plan** out) {
  if (!out) return fail(QT_EINVAL, "out is NULL");
  if (p < 1 || p > 64) return fail(QT_EINVAL, "p must be in [1, 64]");
  if (!bits || n_strings < 1) return fail(QT_EINVAL, "bitstrings are NULL or empty");
  qt_plan_options o;
  qt_status st = check_options(opt, &o);
  if (st != QT_OK) return st;
  if (o.gradient) return fail(QT_EINVAL, "amplitude plans have no gradient");
  qt_plan* h = new (std::nothrow) qt_plan;
  if (!h) return fail(QT_ENOMEM, "host allocation failed");
  st = make_graph(g, &h->P.G);
  if (st == QT_OK) {
    const int32_t n = h->P.G.n;
    for (int64_t i = 0; i < (int64_t)n_strings * n && st == QT_OK; ++i)
      if (bits[i] > 1) st = fail(QT_EINVAL, "bitstring bytes must be 0 or 1");
  }
  if (st == QT_OK) {
    h->P.p = p;
    h->P.opt = o;
    h->P.opt.edge_begin = 0;
    h->P.opt.edge_end = n_strings;
    h->P.elem_bytes = o.dtype == QT_C64 ? 8 : 16;
    h->P.amplitude = true;
    const Graph& G = h->P.G;
    std::vector<uint8_t> x(bits, bits + (size_t)n_strings * G.n);
    st = plan_units([&](int32_t s, Network* net) { build_amplitude_network(G, p, x.data() + (size_t)s * G.n, s, net); },
                    "bitstring", o, 0, n_strings, &h->P);
  }
  if (st == QT_OK) st = compile_plan(&h->P);
  if (st != QT_OK) {
    delete h;
    return st;
  }
  *out = h;
  return QT_OK;
}

qt_status qt_representation_cost(const qt_graph* g, int32_t p, int32_t rep, int32_t order_trials, int32_t seed,
                                 int32_t* n_vars, int32_t* width, double* log2_cost) {
  if (p < 1 || p > 64) return fail(QT_EINVAL, "p must be in [1, 64]");
  if (rep < QT_REP_DEFAULT || rep > QT_REP_ZZ_DIAGONAL) return fail(QT_EINVAL, "unknown representation");
  if (order_trials < 0 || order_trials > 100000) return fail(QT_EINVAL, "order_trials must be in [0, 100000]");
  Graph G;
  qt_status st = make_graph(g, &G);
  if (st != QT_OK) return st;
  Network net;
  build_representation_network(G, p, rep, &net);
  std::vector<int32_t> order;
  double cost = 0.0;
  const int32_t w = order_trials > 0 ? search_order(net, order_trials, 1.0, (uint64_t)(uint32_t)seed << 32, 0, &order,
                                                    &cost)
                                     : min_fill_order(net, &order, &cost);
  if (n_vars) *n_vars = net.n_vars;
  if (width) *width = w;
  if (log2_cost) *log2_cost = std::log2(cost);
  return QT_OK;
}

qt_status qt_plan_amplitudes(qt_plan* plan, const double* gamma, const double* beta, double* amp, void* workspace,
                             size_t ws_bytes, void* stream) {
  if (!plan) return fail(QT_EINVAL, "plan is NULL");
  if (!plan->P.amplitude) return fail(QT_ESTATE, "not an amplitude plan (use qt_plan_energy)");
  if (!amp) return fail(QT_EINVAL, "amp is NULL");
  return run_plan(&plan->P, gamma, beta, nullptr, amp, nullptr, workspace, ws_bytes, stream);
}

qt_status qt_plan_workspace_size(const qt_plan* plan, size_t* bytes) {
  if (!plan || !bytes) return fail(QT_EINVAL, "plan or bytes is NULL");
  *bytes = plan->P.ws.total;
  return QT_OK;
}

qt_status qt_plan_stats(const qt_plan* plan, int32_t* n_edges, int32_t* max_width, int64_t* n_buckets,
                        double* alg_bytes, double* flops) {
  if (!plan) return fail(QT_EINVAL, "plan is NULL");
  const Plan& P = plan->P;
  if (n_edges) *n_edges = P.n_orig;
  if (max_width) {
    int32_t w = 0;
    for (int32_t x : P.widths) w = std::max(w, x);
    *max_width = w;
  }
  if (n_buckets) *n_buckets = (int64_t)P.buckets.size();
  if (alg_bytes) *alg_bytes = P.alg_bytes;
  if (flops) *flops = P.flops;
  return QT_OK;
}

qt_status qt_plan_edge_widths(const qt_plan* plan, int32_t* widths) {
  if (!plan || !widths) return fail(QT_EINVAL, "plan or widths is NULL");
  std::copy(plan->P.widths.begin(), plan->P.widths.end(), widths);
  return QT_OK;
}

qt_status qt_plan_edge_bytes(const qt_plan* plan, double* bytes) {
  if (!plan || !bytes) return fail(QT_EINVAL, "plan or bytes is NULL");
  std::copy(plan->P.edge_bytes.begin(), plan->P.edge_bytes.end(), bytes);
  return QT_OK;
}

qt_status qt_plan_edge_slices(const qt_plan* plan, int32_t* slices) {
  if (!plan || !slices) return fail(QT_EINVAL, "plan or slices is NULL");
  std::copy(plan->P.slices.begin(), plan->P.slices.end(), slices);
  return QT_OK;
}

qt_status qt_plan_edge_order(const qt_plan* plan, int32_t unit, int32_t* order, int32_t* n_vars) {
  if (!plan || !n_vars) return fail(QT_EINVAL, "plan or n_vars is NULL");
  const Plan& P = plan->P;
  if (unit < 0 || unit >= P.n_orig) return fail(QT_EINVAL, "unit " + std::to_string(unit) + " out of range");
  const EdgePlan& ep = P.edges[P.net_first[unit]];
  const int32_t n = (int32_t)ep.buckets.size();
  if (order) {
    if (*n_vars < n)
      return fail(QT_EINVAL, "order holds " + std::to_string(*n_vars) + " entries, the network has " +
                                 std::to_string(n) + " variables");
    for (int32_t i = 0; i < n; ++i) order[i] = ep.buckets[i].var;
  }
  *n_vars = n;
  return QT_OK;
}

qt_status qt_plan_energy(qt_plan* plan, const double* gamma, const double* beta, double* energy, double* edge_zz,
                         double* grad, void* workspace, size_t ws_bytes, void* stream) {
  if (!plan) return fail(QT_EINVAL, "plan is NULL");
  if (plan->P.amplitude) return fail(QT_ESTATE, "amplitude plan: use qt_plan_amplitudes");
  return run_plan(&plan->P, gamma, beta, energy, edge_zz, grad, workspace, ws_bytes, stream);
}

qt_status qt_plan_check(qt_plan* plan, void* stream) {
  if (!plan) return fail(QT_EINVAL, "plan is NULL");
  return check_plan(&plan->P, stream);
}

qt_status qt_plan_energy_host(qt_plan* plan, const double* gamma, const double* beta, double* energy,
                              double* edge_zz, double* grad, void* workspace, size_t ws_bytes, void* stream) {
  if (!plan) return fail(QT_EINVAL, "plan is NULL");
  if (plan->P.amplitude) return fail(QT_ESTATE, "amplitude plan: use qt_plan_amplitudes");
  Plan& P = plan->P;
  const int32_t B = P.opt.batch, p = P.p, ne = P.n_orig;
  qt_status st;
  if ((st = check_angles(gamma, (int64_t)B * p, "gamma")) != QT_OK) return st;
  if ((st = check_angles(beta, (int64_t)B * p, "beta")) != QT_OK) return st;
  if (!workspace) return fail(QT_EINVAL, "workspace is NULL");
  if (ws_bytes < P.ws.total) return fail(QT_ENOMEM, "workspace smaller than the plan needs");
  cudaStream_t s = (cudaStream_t)stream;
  char* base = (char*)workspace;
  double* d_gamma = (double*)(base + P.ws.angles);
  double* d_beta = d_gamma + (size_t)B * p;
  double* d_energy = (double*)(base + P.ws.results);
  double* d_zz = d_energy + B;
  double* d_grad = d_zz + (size_t)ne * B * 2;
  cudaError_t ce;
  if ((ce = cudaMemcpyAsync(d_gamma, gamma, sizeof(double) * B * p, cudaMemcpyHostToDevice, s)) != cudaSuccess ||
      (ce = cudaMemcpyAsync(d_beta, beta, sizeof(double) * B * p, cudaMemcpyHostToDevice, s)) != cudaSuccess)
    return fail(QT_ECUDA, std::string("angle upload: ") + cudaGetErrorString(ce));
  st = run_plan(&P, d_gamma, d_beta, d_energy, edge_zz ? d_zz : nullptr, grad ? d_grad : nullptr, workspace,
                ws_bytes, stream);
  if (st != QT_OK) return st;
  if (energy && (ce = cudaMemcpyAsync(energy, d_energy, sizeof(double) * B, cudaMemcpyDeviceToHost, s)) != cudaSuccess)
    return fail(QT_ECUDA, std::string("energy download: ") + cudaGetErrorString(ce));
  if (edge_zz &&
      (ce = cudaMemcpyAsync(edge_zz, d_zz, sizeof(double) * ne * B * 2, cudaMemcpyDeviceToHost, s)) != cudaSuccess)
    return fail(QT_ECUDA, std::string("edge_zz download: ") + cudaGetErrorString(ce));
  if (grad &&
      (ce = cudaMemcpyAsync(grad, d_grad, sizeof(double) * B * 2 * p, cudaMemcpyDeviceToHost, s)) != cudaSuccess)
    return fail(QT_ECUDA, std::string("grad download: ") + cudaGetErrorString(ce));
  return check_plan(&P, stream);
}

qt_status qt_plan_set_profiling(qt_plan* plan, int32_t on) {
  if (!plan) return fail(QT_EINVAL, "plan is NULL");
  plan->P.profile = on != 0;
  return QT_OK;
}

qt_status qt_plan_kernel_times(qt_plan* plan, float* ms, int32_t cap, int32_t* n) {
  if (!plan || (!ms && cap > 0)) return fail(QT_EINVAL, "plan or ms is NULL");
  return plan_kernel_times(&plan->P, ms, cap, n);
}

qt_status qt_plan_trace_size(const qt_plan* plan, size_t* bytes) {
  if (!plan || !bytes) return fail(QT_EINVAL, "NULL argument");
  *bytes = sizeof(unsigned long long) * 4 * plan->P.tasks.size();
  return QT_OK;
}

qt_status qt_plan_set_trace(qt_plan* plan, void* trace, size_t bytes) {
  if (!plan) return fail(QT_EINVAL, "plan is NULL");
  Plan& P = plan->P;
  if (!trace) {
    P.trace = nullptr;
    return QT_OK;
  }
  if (P.opt.mode != QT_MODE_PERSISTENT) return fail(QT_ESTATE, "tracing needs a persistent plan");
  if (((uintptr_t)trace & 7u) != 0) return fail(QT_EINVAL, "trace buffer is not 8-byte aligned");
  if (bytes < sizeof(unsigned long long) * 4 * P.tasks.size())
    return fail(QT_ENOMEM, "trace buffer holds " + std::to_string(bytes) + " bytes, the queue needs " +
                               std::to_string(sizeof(unsigned long long) * 4 * P.tasks.size()));
  P.trace = (unsigned long long*)trace;
  return QT_OK;
}

qt_status qt_plan_tasks(const qt_plan* plan, int32_t* n_tasks, int32_t* step, int32_t* chunk, int32_t* out_rank,
                        int32_t* edge, int32_t* n_in, int32_t* kind) {
  if (!plan || !n_tasks) return fail(QT_EINVAL, "NULL argument");
  const Plan& P = plan->P;
  *n_tasks = (int32_t)P.tasks.size();
  const int32_t n_net = (int32_t)P.edge_first.size() - 1;
  std::vector<int32_t> step_edge(P.buckets.size(), 0);
  for (int32_t k = 0; k < n_net; ++k) {
    // network k belongs to the planned edge whose network range holds it
    int32_t e = 0;
    while (e + 1 < (int32_t)P.net_first.size() - 1 && P.net_first[e + 1] <= k) ++e;
    for (int32_t b = P.edge_first[k]; b < P.edge_first[k + 1]; ++b) step_edge[b] = e;
  }
  for (size_t t = 0; t < P.tasks.size(); ++t) {
    const DevTask& T = P.tasks[t];
    if (step) step[t] = T.bucket;
    if (chunk) chunk[t] = T.chunk;
    if (out_rank) out_rank[t] = P.buckets[T.bucket].out_rank;
    if (edge) edge[t] = step_edge[T.bucket];
    if (n_in) n_in[t] = P.buckets[T.bucket].n_in;
    if (kind) kind[t] = P.buckets[T.bucket].kind;
  }
  return QT_OK;
}

qt_status qt_plan_schedule(const qt_plan* plan, int32_t* n_steps, int32_t* n_deps, int32_t* n_access,
                           int32_t* dep_first, int32_t* dep_count, int32_t* deps, int32_t* acc_first,
                           int64_t* acc_lo, int64_t* acc_hi, int32_t* acc_write, int32_t* unit) {
  if (!plan || !n_steps || !n_deps || !n_access) return fail(QT_EINVAL, "NULL argument");
  const Plan& P = plan->P;
  if (P.opt.mode != QT_MODE_PERSISTENT) return fail(QT_ESTATE, "the schedule is reported for persistent plans");
  const int32_t ns = (int32_t)P.buckets.size();
  *n_steps = ns;
  *n_deps = (int32_t)P.deps.size();
  *n_access = (int32_t)P.acc_lo.size();
  if (!dep_first || !dep_count || !deps || !acc_first || !acc_lo || !acc_hi || !acc_write || !unit) return QT_OK;
  for (int32_t s = 0; s < ns; ++s) unit[s] = s;
  for (const DevTask& t : P.tasks)
    for (int32_t k = 1; k < -t.chunk; ++k) unit[t.bucket + k] = t.bucket;
  for (int32_t s = 0; s < ns; ++s) {
    dep_first[s] = P.buckets[s].dep;
    dep_count[s] = unit[s] == s ? P.buckets[s].n_dep : 0;
  }
  std::copy(P.deps.begin(), P.deps.end(), deps);
  std::copy(P.acc_first.begin(), P.acc_first.end(), acc_first);
  std::copy(P.acc_lo.begin(), P.acc_lo.end(), acc_lo);
  std::copy(P.acc_hi.begin(), P.acc_hi.end(), acc_hi);
  for (size_t a = 0; a < P.acc_w.size(); ++a) acc_write[a] = P.acc_w[a];
  return QT_OK;
}

qt_status qt_plan_set_wait_limit(qt_plan* plan, int32_t polls) {
  if (!plan || polls < 1) return fail(QT_EINVAL, "plan is NULL or polls < 1");
  plan->P.spin_limit = polls;
  return QT_OK;
}

qt_status qt_plan_inject_stall(qt_plan* plan, int32_t enable) {
  if (!plan) return fail(QT_EINVAL, "plan is NULL");
  Plan& P = plan->P;
  P.stall_step = -1;
  if (enable) {
    for (size_t t = P.tasks.size(); t-- > 0;) {
      const DevBucket& d = P.buckets[P.tasks[t].bucket];
      if (d.n_dep > 0) {
        P.stall_step = P.deps[d.dep];
        break;
      }
    }
    if (P.stall_step < 0) return fail(QT_ESTATE, "no queued task waits on another (persistent plan needed)");
  }
  P.bound_ws = nullptr;  // upload again with (or without) the stall
  return QT_OK;
}

void qt_plan_free(qt_plan* plan) { delete plan; }

qt_status qt_energy_workspace_size(const qt_graph* g, int32_t p, int32_t B, qt_dtype dtype, int32_t gradient,
                                   size_t* bytes) {
  if (!bytes) return fail(QT_EINVAL, "bytes is NULL");
  qt_plan_options o;
  qt_plan_options_default(&o);
  o.batch = B;
  o.dtype = dtype;
  o.mode = QT_MODE_PERSISTENT;
  o.gradient = gradient;
  qt_plan* h = nullptr;
  qt_status st = qt_plan_create(g, p, &o, &h);
  if (st != QT_OK) return st;
  *bytes = h->P.ws.total;
  qt_plan_free(h);
  return QT_OK;
}

qt_status qt_energy(const qt_graph* g, int32_t p, const double* gamma, const double* beta, int32_t B,
                    qt_dtype dtype, void* stream, void* workspace, size_t ws_bytes, double* energy, double* grad) {
  qt_plan_options o;
  qt_plan_options_default(&o);
  o.batch = B;
  o.dtype = dtype;
  o.mode = QT_MODE_PERSISTENT;
  o.gradient = grad ? 1 : 0;
  qt_plan* h = nullptr;
  qt_status st = qt_plan_create(g, p, &o, &h);
  if (st != QT_OK) return st;
  st = qt_plan_energy_host(h, gamma, beta, energy, nullptr, grad, workspace, ws_bytes, stream);
  qt_plan_free(h);
  return st;
}

}  // extern "C"
