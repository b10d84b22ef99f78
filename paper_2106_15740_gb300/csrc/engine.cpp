// Plan compiler and executor of the energy path.
//
// compile_plan turns the bucket plans of every edge network into device
// records (qt_device.h) and lays out the workspace:
//   [ctrl | done counters | buckets | tasks | dependency lists | leaf factors | scalar table |
//    network leaf counts | angles | results | trig table | data]
// data = [leaf-factor pool | scalar results | intermediate arenas].
// Intermediates of one edge live in an arena planned by first-fit with
// free-on-consume: a bucket's output is allocated before its inputs are
// released, so a bucket never writes over what it reads.
//
// Execution (run_plan): angle table -> leaf factors -> buckets -> energy.
// QT_MODE_PER_BUCKET launches one kernel per bucket, edge after edge, all
// edges sharing one arena.  QT_MODE_PERSISTENT issues one persistent launch
// over a queue of bucket tiles; edges are spread over "slots" (one arena
// each).  A queued step waits for the last writer of what it reads and for
// the last writer and readers of what it writes (access_deps; forward and
// adjoint steps alike), and the queue takes first the tasks with the longest
// remaining dependency path (or the slots round-robin), so independent work
// fills the GPU while a step waits.
#include "engine.h"

#include <algorithm>
#include <cstddef>
#include <cstring>
#include <functional>
#include <map>
#include <queue>

#include "kernels_api.h"

namespace qt {

namespace {

struct Arena {
  std::map<int64_t, int64_t> free_;
  int64_t top = 0, peak = 0;
  int64_t alloc(int64_t n) {
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= n) {
        const int64_t o = it->first, rem = it->second - n;
        free_.erase(it);
        if (rem) free_[o + n] = rem;
        return o;
      }
    }
    const int64_t o = top;
    top += n;
    peak = std::max(peak, top);
    return o;
  }
  void release(int64_t o, int64_t n) {
    auto it = free_.emplace(o, n).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_.erase(nx);
    }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_.erase(it);
        it = pv;
      }
    }
    if (it->first + it->second == top) {
      top = it->first;
      free_.erase(it);
    }
  }
};

void fill_runs(uint32_t mask, DevInput* in) {
  int32_t n = 0, dst = 0, bit = 0;
  while (bit < 32) {
    if (!((mask >> bit) & 1u)) {
      ++bit;
      continue;
    }
    const int32_t start = bit;
    while (bit < 32 && ((mask >> bit) & 1u)) ++bit;
    const int32_t len = bit - start;
    if (n < kDevMaxRuns) in->run[n] = (uint32_t)start | (uint32_t)len << 8 | (uint32_t)dst << 16;
    ++n;
    dst += len;
  }
  in->mask = mask;
  in->nruns = n <= kDevMaxRuns ? n : -1;
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

constexpr int32_t kMaxGroup = 4096;  // buckets in one single-tile group task
constexpr int64_t kMaxTasks = (int64_t)1 << 27;  // queue length the automatic chunk sizes aim for
constexpr int64_t kMinChunks = 8192;             // chunks per wide step, at least (about 1.7 per resident warp)

}  // namespace

// Input record of a forward step (offset filled in by the caller).
static DevInput input_record(uint32_t mask, int64_t off, int32_t flags) {
  DevInput in;
  std::memset(&in, 0, sizeof(in));
  fill_runs(mask, &in);
  in.off = off;
  in.flags = flags;
  return in;
}

// One step of a gradient network in execution order: forward steps, then,
// per checkpoint segment from the last to the first, the forward steps of
// the segment that are re-run and the segment's adjoint steps.
struct GradOp {
  int32_t kind = kStepFwd;   // kStepFwd, kStepAdj, kStepZero
  int32_t bucket = -1;
  int32_t input = -1;        // kStepAdj: input of the bucket; -2: scalar adjoint of a multi-component network
  bool recompute = false;    // kStepFwd: a re-run in the reverse sweep
  int64_t out = 0;           // arena offset of the output / target (leaf target: its leaf-pool offset)
  bool leaf = false, full = false;
  int32_t zero_rank = 0;
  int64_t gbar = -1;         // kStepAdj: arena offset of the bucket's output adjoint (-1: none)
  std::vector<int64_t> loc;  // arena offset of each intermediate input (-1 for the leaf factor)
};

// Dependencies of the steps of one workspace slot from the data elements
// they touch.  The slot runs its networks one after another, each network's
// steps in plan order (`nets`: global step ranges); that order is correct
// run sequentially, and a step may start early as long as it keeps every
// conflicting access in that order: it waits for the last writer of what it
// reads (bucket elimination: the buckets that produced its inputs) and for
// the last writer and all readers since of what it writes (the arena reuses
// released space).  An accumulating write (atomic adds) counts as a write.
// Within a network, entries that another entry already depends on
// (transitively) are dropped; entries in earlier networks of the slot are
// kept as found.  deps[s] gets global step indices, all earlier in the slot.
static void access_deps(const Plan& P, const std::vector<std::pair<int32_t, int32_t>>& nets,
                        std::vector<std::vector<int32_t>>* deps) {
  struct Seg {
    int64_t end;
    int32_t writer;
    std::vector<int32_t> readers;
  };
  std::map<int64_t, Seg> mem;  // disjoint segments of touched elements
  // split so that a segment boundary falls at x (x inside a segment)
  auto split = [&](int64_t x) {
    auto it = mem.upper_bound(x);
    if (it == mem.begin()) return;
    --it;
    if (it->first < x && it->second.end > x) {
      Seg tail = it->second;
      it->second.end = x;
      mem.emplace(x, std::move(tail));
    }
  };
  // visit the segments covering [lo, hi), creating untouched ones
  auto cover = [&](int64_t lo, int64_t hi, const std::function<void(Seg&)>& f) {
    split(lo);
    split(hi);
    int64_t x = lo;
    auto it = mem.lower_bound(lo);
    while (x < hi) {
      if (it == mem.end() || it->first > x) {
        const int64_t e = it == mem.end() ? hi : std::min(hi, it->first);
        it = mem.emplace_hint(it, x, Seg{e, -1, {}});
      }
      f(it->second);
      x = it->second.end;
      ++it;
    }
  };
  std::vector<int32_t> raw;
  std::vector<uint64_t> anc;
  for (const auto& nr : nets) {
    const int32_t s0 = nr.first, n = nr.second - nr.first, W = (n + 63) / 64;
    anc.assign((size_t)n * W, 0);
    for (int32_t s = s0; s < s0 + n; ++s) {
      raw.clear();
      const int32_t a0 = P.acc_first[s], a1 = P.acc_first[s + 1];
      for (int32_t a = a0; a < a1; ++a)
        cover(P.acc_lo[a], P.acc_hi[a], [&](Seg& g) {
          if (g.writer >= 0) raw.push_back(g.writer);
          if (P.acc_w[a]) raw.insert(raw.end(), g.readers.begin(), g.readers.end());
        });
      for (int32_t a = a0; a < a1; ++a)  // reads first: a write by the same step supersedes them
        if (!P.acc_w[a]) cover(P.acc_lo[a], P.acc_hi[a], [&](Seg& g) { g.readers.push_back(s); });
      for (int32_t a = a0; a < a1; ++a)
        if (P.acc_w[a])
          cover(P.acc_lo[a], P.acc_hi[a], [&](Seg& g) {
            g.writer = s;
            g.readers.clear();
          });
      std::sort(raw.begin(), raw.end());
      raw.erase(std::unique(raw.begin(), raw.end()), raw.end());
      raw.erase(std::remove(raw.begin(), raw.end(), s), raw.end());
      // the slot runs its networks in its own order, so an earlier network's
      // steps may have larger indices: "inside" means within [s0, s0 + n)
      auto inside = [&](int32_t d) { return d >= s0 && d < s0 + n; };
      uint64_t* ai = &anc[(size_t)(s - s0) * W];
      for (int32_t d : raw)
        if (inside(d)) {
          const uint64_t* ad = &anc[(size_t)(d - s0) * W];
          for (int32_t w = 0; w < W; ++w) ai[w] |= ad[w];
        }
      std::vector<int32_t>& out = (*deps)[s];
      out.clear();
      for (int32_t d : raw) {
        bool implied = false;
        if (inside(d))
          for (int32_t d2 : raw)
            if (d2 != d && inside(d2) && ((anc[(size_t)(d2 - s0) * W + ((d - s0) >> 6)] >> ((d - s0) & 63)) & 1u)) {
              implied = true;
              break;
            }
        if (!implied) out.push_back(d);
        if (inside(d)) ai[(d - s0) >> 6] |= (uint64_t)1 << ((d - s0) & 63);
      }
    }
  }
}

// Reverse-mode plan of one network with checkpointing.  The bucket order is
// cut into segments whose produced intermediates hold at most `budget`
// elements (one segment if budget <= 0).  A forward intermediate is kept
// through the forward pass if its consumer lies in a later segment or it
// belongs to the last segment; the others are freed when consumed and the
// reverse sweep re-runs their forward steps just before their segment's
// adjoint steps.  Every tensor shares one first-fit arena in execution order
// (an output is allocated before its step's inputs are released); a forward
// tensor is released once its consumer's adjoint steps are done, an output
// adjoint once its bucket's adjoint steps are done.  Returns the arena peak;
// *recompute_bytes gets the extra forward traffic (elements x B).
static int64_t plan_gradient_network(const EdgePlan& ep, int64_t B, int64_t budget, int64_t al,
                                     const std::vector<int64_t>& leaf_off, std::vector<GradOp>* ops,
                                     std::vector<int64_t>* fwd_loc, double* recompute_elems) {
  auto align_el = [&](int64_t x) { return (x + al - 1) / al * al; };
  const int32_t nb = (int32_t)ep.buckets.size();
  auto size_of = [&](int32_t i) {
    const int32_t r = ep.buckets[i].out_rank;
    return r > 0 ? align_el(((int64_t)1 << r) * B) : (int64_t)0;
  };
  std::vector<int32_t> seg(nb, 0);
  int32_t nseg = 1;
  if (budget > 0) {
    int64_t acc = 0;
    int32_t cur = 0;
    for (int32_t i = 0; i < nb; ++i) {
      if (acc > 0 && acc + size_of(i) > budget) {
        ++cur;
        acc = 0;
      }
      seg[i] = cur;
      acc += size_of(i);
    }
    nseg = cur + 1;
  }
  auto kept = [&](int32_t c) {
    const int32_t con = ep.buckets[c].consumer;
    return seg[c] == nseg - 1 || (con >= 0 && seg[con] > seg[c]);
  };
  Arena A;
  std::vector<int64_t> loc(nb, -1), gbar(nb, -1);
  fwd_loc->assign(nb, -1);
  *recompute_elems = 0.0;
  auto fwd_op = [&](int32_t i, bool re) {
    const Bucket& bk = ep.buckets[i];
    GradOp op;
    op.kind = kStepFwd;
    op.bucket = i;
    op.recompute = re;
    if (bk.out_rank > 0) {
      loc[i] = A.alloc(size_of(i));
      op.out = loc[i];
    }
    for (size_t k = 0; k < bk.in_src.size(); ++k) op.loc.push_back(bk.in_src[k] >= 0 ? loc[bk.in_src[k]] : -1);
    ops->push_back(op);
    if (re) {
      double el = (double)((int64_t)1 << bk.out_rank);
      for (size_t k = 0; k < bk.in_src.size(); ++k)
        if (bk.in_src[k] >= 0) el += (double)((int64_t)1 << bk.in_rank[k]);
      *recompute_elems += el * (double)B;
    }
  };
  // forward pass
  for (int32_t i = 0; i < nb; ++i) {
    fwd_op(i, false);
    (*fwd_loc)[i] = loc[i];
    for (int32_t c : ep.buckets[i].in_src)
      if (c >= 0 && !kept(c)) {
        A.release(loc[c], size_of(c));
        loc[c] = -1;
      }
  }
  // output adjoints of the scalar results of a network that split into
  // components: the product of the other scalars (rank-0 adjoint steps)
  if (ep.scalars.size() > 1)
    for (int32_t sb : ep.scalars) {
      gbar[sb] = A.alloc(align_el(2 * B));
      GradOp op;
      op.kind = kStepAdj;
      op.bucket = sb;
      op.input = -2;
      op.out = gbar[sb];
      op.full = true;
      ops->push_back(op);
    }
  // reverse sweep, segment by segment
  for (int32_t k = nseg - 1; k >= 0; --k) {
    if (k != nseg - 1)
      for (int32_t c = 0; c < nb; ++c)
        if (seg[c] == k && ep.buckets[c].out_rank > 0 && loc[c] < 0) fwd_op(c, true);
    for (int32_t b = nb - 1; b >= 0; --b) {
      if (seg[b] != k) continue;
      const Bucket& bk = ep.buckets[b];
      const uint32_t all = bk.out_rank ? ((1u << bk.out_rank) - 1u) : 0u;
      std::vector<int64_t> in_loc;
      for (int32_t c : bk.in_src) in_loc.push_back(c >= 0 ? loc[c] : -1);
      for (size_t kk = 0; kk < bk.in_src.size(); ++kk) {
        GradOp op;
        op.kind = kStepAdj;
        op.bucket = b;
        op.input = (int32_t)kk;
        op.full = bk.in_mask[kk] == all;
        op.gbar = gbar[b];
        op.loc = in_loc;
        const int32_t t = bk.in_src[kk];
        if (t >= 0) {
          gbar[t] = A.alloc(size_of(t));
          op.out = gbar[t];
          if (!op.full) {
            GradOp z;
            z.kind = kStepZero;
            z.bucket = b;
            z.out = gbar[t];
            z.zero_rank = ep.buckets[t].out_rank;
            ops->push_back(z);
          }
        } else {
          op.leaf = true;
          op.out = leaf_off[b];
        }
        ops->push_back(op);
      }
      if (gbar[b] >= 0) A.release(gbar[b], bk.out_rank > 0 ? size_of(b) : align_el(2 * B));
      gbar[b] = -1;
      for (int32_t c : bk.in_src)
        if (c >= 0) {
          A.release(loc[c], size_of(c));
          loc[c] = -1;
        }
    }
  }
  return A.peak;
}

// Largest fan-in of a chained step's first bucket on the row-wide layout (the
// fixed-fan-in chained tiles; equal to the forward tiles' fixed fan-in).
constexpr int32_t kFixedMaxFanInChain = 3;

// Warps the queue's list-scheduling simulation assumes: twice the resident
// warps (152 SMs x 4 blocks x 8), the best of a sweep on the bench step, the
// 60-vertex p = 4 gradient and its energy (3648 / 4864 / 6400 / 9728 / 14592 /
// 19456 / 38912 warps: bench 13.75 / 13.66 / 13.54 / 13.31 / 13.25 / 13.25 /
// 13.52 ms, gradient 7.89 / 7.81 / 7.70 / 7.67 / 7.77 / 7.92 / 8.27 ms).
constexpr int64_t kSimWarps = 9728;

qt_status compile_plan(Plan* P) {
  const int32_t B = P->opt.batch;
  const int32_t es = P->elem_bytes;
  const int64_t al = 256 / es;  // elements per 256 bytes
  auto align_el = [&](int64_t x) { return (x + al - 1) / al * al; };
  const int32_t n_edges = (int32_t)P->edges.size();
  const bool grad = P->opt.gradient != 0;
  const bool persistent = P->opt.mode == QT_MODE_PERSISTENT;
  if (grad && !persistent) return fail(QT_EINVAL, "gradient plans need QT_MODE_PERSISTENT");

  // ---- per-edge memory plans (offsets relative to the edge's region) ----
  // Forward intermediates: first-fit with free-on-consume.  Gradient plans
  // lay out the forward pass, the checkpoint re-runs and the adjoint buffers
  // of a network in one first-fit arena in execution order
  // (plan_gradient_network).
  std::vector<std::vector<int64_t>> out_off(n_edges), leaf_off(n_edges);
  std::vector<std::vector<GradOp>> gops(n_edges);
  std::vector<int64_t> region(n_edges), cost(n_edges);
  int64_t leaf_pool = 0, scal_pool = 0;
  P->alg_bytes = 0.0;
  P->edge_bytes.assign(P->n_orig, 0.0);
  std::vector<int32_t> orig_of(n_edges, 0);  // planned graph edge of each network
  for (int32_t o = 0; o < P->n_orig; ++o)
    for (int32_t k = P->net_first[o]; k < P->net_first[o + 1]; ++k) orig_of[k] = o;
  P->flops = 0.0;
  // Chained steps: bucket b fused with up to fuse_chains consumers c_1 .. c_m,
  // c_1 eliminating b's result and c_j that of c_(j-1), each with no variable
  // beyond its input and no other intermediate input.  Chains are taken
  // greedily in execution order (a bucket absorbed into a chain starts none).
  // The fused step runs at b's place: c_m's output is allocated there, the
  // results of b and c_1 .. c_(m-1) never are.
  const bool fuse = !grad && persistent && P->opt.fuse_chains > 0 && chain_fusion_ok(P->opt.dtype, B);
  P->has_chains = false;
  // (one angle set: one consumer at most, which the pair tile takes in lane shuffles)
  const int32_t max_chain = B == 1 ? std::min<int32_t>(P->opt.fuse_chains, 1) : P->opt.fuse_chains;
  std::vector<std::vector<std::vector<int32_t>>> chain_of(n_edges);  // per network and bucket: c_1 .. c_m
  for (int32_t e = 0; e < n_edges; ++e) {
    const EdgePlan& ep = P->edges[e];
    const int32_t nb = (int32_t)ep.buckets.size();
    chain_of[e].assign(nb, {});
    if (!fuse) continue;
    std::vector<char> absorbed(nb, 0);
    for (int32_t i = 0; i < nb; ++i) {
      if (absorbed[i]) continue;
      const int32_t n_in = (int32_t)ep.buckets[i].in_src.size();
      if (B > 1 && (P->opt.dtype != QT_C64 || n_in < 2 || n_in > kFixedMaxFanInChain))
        continue;  // row-wide layout: the fixed-fan-in chained tiles of complex64 only
      int32_t cur = i;
      while ((int32_t)chain_of[e][i].size() < max_chain && n_in + (int32_t)chain_of[e][i].size() < kDevMaxIn) {
        const int32_t c = ep.buckets[cur].consumer;
        if (c < 0 || ep.buckets[cur].out_rank < 1) break;
        const Bucket& bc = ep.buckets[c];
        int32_t n_int = 0;
        for (int32_t src : bc.in_src) n_int += src >= 0 ? 1 : 0;
        if (bc.out_rank + 1 != ep.buckets[cur].out_rank || n_int != 1) break;
        chain_of[e][i].push_back(c);
        absorbed[c] = 1;
        cur = c;
      }
    }
  }
  for (int32_t e = 0; e < n_edges; ++e) {
    const EdgePlan& ep = P->edges[e];
    const int32_t nb = (int32_t)ep.buckets.size();
    const double bytes_before = P->alg_bytes;
    std::vector<char> absorbed(nb, 0);
    for (int32_t i = 0; i < nb; ++i)
      for (int32_t c : chain_of[e][i]) absorbed[c] = 1;

    Arena arena;
    out_off[e].assign(nb, 0);
    leaf_off[e].assign(nb, -1);
    double ebytes = 0.0;
    for (int32_t i = 0; i < nb; ++i) {
      const Bucket& bk = ep.buckets[i];
      if (bk.leaf_rank > 0) {
        leaf_off[e][i] = leaf_pool;
        leaf_pool += align_el(((int64_t)1 << bk.leaf_rank) * B);
      }
      const double nin = (double)bk.in_src.size();
      P->flops += (double)B * (double)((int64_t)1 << bk.out_rank) * (2.0 * 6.0 * (nin - 1.0) + 2.0);
      if (absorbed[i]) continue;  // evaluated (and its output placed) with the bucket it is fused with
      const int32_t o = chain_of[e][i].empty() ? i : chain_of[e][i].back();  // whose output this step writes
      const int64_t rows = (int64_t)1 << ep.buckets[o].out_rank;
      if (ep.buckets[o].out_rank == 0) {
        out_off[e][o] = scal_pool;  // relative to the scalar pool
        scal_pool += align_el(B);
      } else {
        out_off[e][o] = arena.alloc(align_el(rows * B));
      }
      double bytes = (double)rows;  // output write
      for (size_t k = 0; k < bk.in_src.size(); ++k) {
        if (bk.in_src[k] < 0) continue;
        const Bucket& src = ep.buckets[bk.in_src[k]];
        if (!grad) arena.release(out_off[e][bk.in_src[k]], align_el(((int64_t)1 << src.out_rank) * B));
        bytes += (double)((int64_t)1 << bk.in_rank[k]);
      }
      ebytes += bytes;
    }
    region[e] = arena.peak;
    if (grad) {
      // reverse sweep (and checkpoint re-runs) in one arena with the forward
      // pass; reverse traffic: per adjoint step Gbar and the other inputs
      // read, the target written
      double re_el = 0.0;
      std::vector<int64_t> floc;
      region[e] = plan_gradient_network(ep, B, P->opt.checkpoint_bytes / es, al, leaf_off[e], &gops[e], &floc,
                                        &re_el);
      for (int32_t i = 0; i < nb; ++i)
        if (ep.buckets[i].out_rank > 0) out_off[e][i] = floc[i];
      P->alg_bytes += re_el * (double)es;
      for (const GradOp& op : gops[e]) {
        if (op.kind != kStepAdj || op.input < 0) continue;
        const Bucket& bk = ep.buckets[op.bucket];
        P->alg_bytes += (double)B * es * (double)(((int64_t)1 << bk.out_rank) + ((int64_t)1 << bk.in_rank[op.input]));
        for (size_t j = 0; j < bk.in_src.size(); ++j)
          if ((int32_t)j != op.input && bk.in_src[j] >= 0)
            P->alg_bytes += (double)B * es * (double)((int64_t)1 << bk.in_rank[j]);
      }
    }
    cost[e] = (int64_t)ebytes * (grad ? 3 : 1);
    P->alg_bytes += ebytes * (double)B * (double)es;
    P->edge_bytes[orig_of[e]] += P->alg_bytes - bytes_before;
  }

  // ---- region placement: per-bucket mode shares one; persistent uses slots ----
  std::vector<int64_t> edge_base(n_edges, 0);
  int64_t arena_total = 0;
  std::vector<std::vector<int32_t>> slot_edges;
  const int64_t leaf_pools = grad ? 2 * leaf_pool : leaf_pool;  // leaf factors (+ their adjoints)
  if (!persistent) {
    for (int32_t e = 0; e < n_edges; ++e) arena_total = std::max(arena_total, region[e]);
    P->n_slots = 1;
  } else {
    std::vector<int32_t> by_cost(n_edges);
    for (int32_t e = 0; e < n_edges; ++e) by_cost[e] = e;
    std::stable_sort(by_cost.begin(), by_cost.end(), [&](int32_t a, int32_t b) { return cost[a] > cost[b]; });
    const int64_t fixed = leaf_pools + scal_pool;
    const int64_t cap_el = P->opt.max_workspace > 0 ? P->opt.max_workspace / es : INT64_MAX;
    int32_t S = n_edges;
    for (;;) {
      slot_edges.assign(S, {});
      std::vector<int64_t> speak(S, 0);
      using Item = std::pair<int64_t, int32_t>;
      std::priority_queue<Item, std::vector<Item>, std::greater<Item>> heap;
      for (int32_t s = 0; s < S; ++s) heap.push({0, s});
      for (int32_t e : by_cost) {
        auto [l, s] = heap.top();
        heap.pop();
        slot_edges[s].push_back(e);
        speak[s] = std::max(speak[s], region[e]);
        heap.push({l + cost[e] + 1, s});
      }
      int64_t total = 0;
      for (int32_t s = 0; s < S; ++s) total += speak[s];
      if (total + fixed <= cap_el || S == 1) {
        if (total + fixed > cap_el) return fail(QT_ENOMEM, "plan does not fit max_workspace even one edge at a time");
        int64_t base = 0;
        for (int32_t s = 0; s < S; ++s) {
          for (int32_t e : slot_edges[s]) edge_base[e] = base;
          base += speak[s];
        }
        arena_total = base;
        break;
      }
      S = std::max(1, S * 7 / 8 < S - 1 ? S * 7 / 8 : S - 1);
    }
    P->n_slots = S;
  }

  // Data region: [leaf pool | leaf-adjoint pool | scalars | arenas].
  const int64_t lbar_shift = grad ? leaf_pool : 0;
  const int64_t scal_base = leaf_pools;
  const int64_t arena_base = scal_base + scal_pool;
  P->data_elems = arena_base + arena_total;
  P->lbar_shift = lbar_shift;
  P->lbar_elems = grad ? leaf_pool : 0;

  // ---- device records: per edge, forward steps then adjoint steps ----
  // Each record also lists the data elements it touches (acc_*), from which
  // the persistent queue derives its dependencies.
  P->acc_first.assign(1, 0);
  P->acc_lo.clear();
  P->acc_hi.clear();
  P->acc_w.clear();
  auto touch = [&](int64_t lo, int64_t n, bool w) {
    P->acc_lo.push_back(lo);
    P->acc_hi.push_back(lo + n);
    P->acc_w.push_back(w ? 1 : 0);
  };
  auto step_done = [&]() { P->acc_first.push_back((int32_t)P->acc_lo.size()); };
  const int32_t geom_bv = tile_geom(P->opt.dtype, B, P->opt.lane_items).Bv;
  P->buckets.clear();
  P->edge_first.assign(n_edges + 1, 0);
  P->leaf.clear();
  P->leaf_first.assign(P->n_orig + 1, 0);
  P->scal_off.clear();
  P->scal_begin.assign(n_edges + 1, 0);
  for (int32_t e = 0; e < n_edges; ++e) {
    const EdgePlan& ep = P->edges[e];
    const int64_t rbase = arena_base + edge_base[e];
    P->edge_first[e] = (int32_t)P->buckets.size();
    auto leaf_record = [&](int32_t i) {
      const Bucket& bk = ep.buckets[i];
      DevLeafFactor lf;
      std::memset(&lf, 0, sizeof(lf));
      lf.off = leaf_off[e][i];
      lf.rank = bk.leaf_rank;
      lf.n_leaves = (int32_t)bk.leaves.size();
      lf.net = e;
      for (int32_t l = 0; l < lf.n_leaves; ++l) {
        const LeafRef& Lr = bk.leaves[l];
        lf.leaf[l] = (uint32_t)Lr.kind | (uint32_t)Lr.conj << 2 | (uint32_t)Lr.rank << 3 |
                     (uint32_t)(Lr.bit[0] < 0 ? 0 : Lr.bit[0]) << 5 | (uint32_t)(Lr.bit[1] < 0 ? 0 : Lr.bit[1]) << 10 |
                     (uint32_t)(Lr.fix[0] >= 0) << 15 | (uint32_t)(Lr.fix[0] > 0) << 16 |
                     (uint32_t)(Lr.fix[1] >= 0) << 17 | (uint32_t)(Lr.fix[1] > 0) << 18 | (uint32_t)Lr.layer << 19;
      }
      P->leaf.push_back(lf);
    };
    // input k of bucket i with the intermediate at arena offset `at`
    auto in_record = [&](int32_t i, int32_t k, int64_t at) {
      const Bucket& bk = ep.buckets[i];
      return bk.in_src[k] >= 0 ? input_record(bk.in_mask[k], rbase + at, 0)
                               : input_record(bk.in_mask[k], leaf_off[e][i], kInLeaf);
    };
    // forward step of bucket i (output at arena offset `out`, inputs at loc)
    auto fwd_record = [&](int32_t i, int64_t out, const std::vector<int64_t>& loc) {
      const Bucket& bk = ep.buckets[i];
      DevBucket d;
      std::memset(&d, 0, sizeof(d));
      d.kind = kStepFwd;
      d.out_rank = bk.out_rank;
      d.n_rows = (int64_t)1 << bk.out_rank;
      d.out_off = bk.out_rank == 0 ? scal_base + out_off[e][i] : rbase + out;
      d.n_in = (int32_t)bk.in_src.size();
      d.dep = -1;
      d.ntask = 1;
      for (int32_t k = 0; k < d.n_in; ++k) d.in[k] = in_record(i, k, loc[k]);
      return d;
    };
    // intermediates of the network: elements of the output of bucket c
    auto tensor_el = [&](int32_t c) { return ((int64_t)1 << ep.buckets[c].out_rank) * B; };
    auto fwd_push = [&](int32_t i, int64_t out, const std::vector<int64_t>& loc) {
      const Bucket& bk = ep.buckets[i];
      P->buckets.push_back(fwd_record(i, out, loc));
      for (size_t k = 0; k < bk.in_src.size(); ++k)
        if (bk.in_src[k] >= 0) touch(rbase + loc[k], tensor_el(bk.in_src[k]), false);
      touch(P->buckets.back().out_off, P->buckets.back().n_rows * B, true);
      step_done();
    };
    if (!grad) {
      std::vector<char> absorbed(ep.buckets.size(), 0);
      for (int32_t i = 0; i < (int32_t)ep.buckets.size(); ++i)
        for (int32_t c : chain_of[e][i]) absorbed[c] = 1;
      for (int32_t i = 0; i < (int32_t)ep.buckets.size(); ++i) {
        const Bucket& bk = ep.buckets[i];
        std::vector<int64_t> loc;
        for (int32_t c : bk.in_src) loc.push_back(c >= 0 ? out_off[e][c] : -1);
        const std::vector<int32_t>& ch = chain_of[e][i];
        if (!ch.empty()) {  // b = i fused with its chain: b's rows, c_m's output, the chain's leaf factors
          const Bucket& bm = ep.buckets[ch.back()];
          DevBucket d = fwd_record(i, 0, loc);
          d.out_off = bm.out_rank == 0 ? scal_base + out_off[e][ch.back()] : rbase + out_off[e][ch.back()];
          d.chain = (int32_t)ch.size();
          P->has_chains = true;
          for (int32_t j = 0; j < d.chain; ++j) {
            const Bucket& bc = ep.buckets[ch[j]];
            int32_t lk = -1;
            for (int32_t k = 0; k < (int32_t)bc.in_src.size(); ++k)
              if (bc.in_src[k] < 0) lk = k;
            if (lk >= 0)  // over b's rows: bit j is c_(j+1)'s eliminated variable (index bit 0), bits j + 1.. its rows
              d.in[d.n_in + j] = input_record((bc.in_mask[lk] << (j + 1)) | (1u << j), leaf_off[e][ch[j]], kInLeaf);
            else
              d.chain_noleaf |= 1 << j;
          }
          P->buckets.push_back(d);
          for (size_t k = 0; k < bk.in_src.size(); ++k)
            if (bk.in_src[k] >= 0) touch(rbase + loc[k], tensor_el(bk.in_src[k]), false);
          touch(d.out_off, ((int64_t)1 << bm.out_rank) * B, true);
          step_done();
        } else if (!absorbed[i]) {
          fwd_push(i, out_off[e][i], loc);
        }
        if (bk.leaf_rank > 0) leaf_record(i);
      }
    }
    // float-pair plans keep every adjoint tensor in FP64 (native atomic adds; see kInF64)
    const int32_t adj_f64 = P->opt.dtype == QT_C64X2 ? kInF64 : 0;
    for (const GradOp& op : gops[e]) {
      const Bucket& bk = ep.buckets[op.bucket];
      for (size_t k = 0; k < op.loc.size(); ++k)  // every intermediate operand is resident
        if (bk.in_src[k] >= 0 && op.loc[k] < 0) return fail(QT_EINVAL, "internal: gradient plan reads a released tensor");
      if (op.kind == kStepFwd) {
        fwd_push(op.bucket, op.out, op.loc);
        if (!op.recompute && bk.leaf_rank > 0) leaf_record(op.bucket);
        continue;
      }
      DevBucket d;
      std::memset(&d, 0, sizeof(d));
      d.dep = -1;
      d.ntask = 1;
      if (op.input == -2) {  // scalar adjoint: product of the network's other scalar results
        d.kind = kStepAdj;
        d.out_rank = 0;
        d.n_rows = 1;
        d.out_off = rbase + op.out;
        d.aflags = kAdjFull;
        int32_t n = 0;
        for (int32_t sb : ep.scalars)
          if (sb != op.bucket) {
            if (n + 1 >= kDevMaxIn) return fail(QT_EINVAL, "too many network components for the gradient");
            d.in[n++] = input_record(0u, scal_base + out_off[e][sb], kInNoPair);
          }
        d.in[n] = input_record(0u, d.out_off, adj_f64);
        d.n_in = n;
        P->buckets.push_back(d);
        for (int32_t sb : ep.scalars)
          if (sb != op.bucket) touch(scal_base + out_off[e][sb], B, false);
        touch(d.out_off, 2 * B, true);
        step_done();
        continue;
      }
      if (op.kind == kStepZero) {
        d.kind = kStepZero;
        d.out_rank = op.zero_rank;
        d.n_rows = (int64_t)1 << op.zero_rank;
        d.out_off = rbase + op.out;
        P->buckets.push_back(d);
        touch(d.out_off, d.n_rows * B, true);
        step_done();
        continue;
      }
      if ((int32_t)bk.in_src.size() + (bk.out_rank > 0 ? 1 : 0) + 1 > kDevMaxIn)
        return fail(QT_EINVAL, "bucket fan-in above the gradient limit");
      d.kind = kStepAdj;
      d.out_rank = bk.out_rank;
      d.n_rows = (int64_t)1 << bk.out_rank;
      d.out_off = op.leaf ? op.out + lbar_shift : rbase + op.out;
      d.aflags = op.full ? kAdjFull : 0;
      const uint32_t all = bk.out_rank ? (1u << bk.out_rank) - 1u : 0u;
      int32_t n = 0;
      if (op.gbar >= 0) {  // rank > 0, or a scalar of a multi-component network
        d.in[n++] = input_record(all, rbase + op.gbar, kInNoPair | adj_f64);
      } else {
        d.aflags |= kAdjUnitG;
      }
      for (int32_t j = 0; j < (int32_t)bk.in_src.size(); ++j)
        if (j != op.input) d.in[n++] = in_record(op.bucket, j, op.loc[j]);
      const uint32_t tmask = bk.in_mask[op.input];
      d.in[n] = input_record(tmask, d.out_off, adj_f64);  // target record
      d.n_in = n;
      if (!op.full && __builtin_popcount(all & ~tmask) >= 5 && geom_bv <= 32 && n + 2 <= kDevMaxIn) {
        // reduction form (32 or more completions per target element): one warp
        // tile per (target row, chunk of completions); smaller targets keep the
        // atomic scatter, whose contention is then at most 32 per element
        d.kind = kStepAdjRed;
        if (B == 1 && n + 3 <= kDevMaxIn) {
          // one angle set: lanes on the bucket's five lowest variables (bk.out_rank >= 5 here),
          // the pass index on the completion bits above them, then the target bits
          const uint32_t comp = all & ~tmask;
          d.aflags |= kAdjRedLow;
          d.in[n + 1] = input_record(comp & ~31u, 0, 0);
          d.in[n + 2] = input_record(tmask & ~31u, 0, 0);
          d.comp_bits = __builtin_popcount(comp & ~31u);
          d.tgt_bits = __builtin_popcount(tmask & ~31u);
        } else {
          d.in[n + 1] = input_record(all & ~tmask, 0, 0);  // complement record
          d.tgt_bits = __builtin_popcount(tmask);
          d.comp_bits = __builtin_popcount(all & ~tmask);
        }
        d.n_rows = (int64_t)1 << bk.out_rank;
      }
      P->buckets.push_back(d);
      if (op.gbar >= 0) touch(rbase + op.gbar, bk.out_rank > 0 ? tensor_el(op.bucket) : 2 * B, false);
      for (int32_t j = 0; j < (int32_t)bk.in_src.size(); ++j)
        if (j != op.input && bk.in_src[j] >= 0) touch(rbase + op.loc[j], tensor_el(bk.in_src[j]), false);
      const int32_t t = bk.in_src[op.input];
      touch(d.out_off, t >= 0 ? tensor_el(t) : ((int64_t)1 << bk.leaf_rank) * B, true);
      step_done();
    }
    for (int32_t sb : ep.scalars) P->scal_off.push_back(scal_base + out_off[e][sb]);
    P->scal_begin[e + 1] = (int32_t)P->scal_off.size();
  }
  P->edge_first[n_edges] = (int32_t)P->buckets.size();
  // leaf counts of each network: ZZ and mixer leaves per layer, |+> leaves
  // (the norm of the stored gates is divided out per network on the device)
  {
    const int32_t stride = 2 * P->p + 1;
    P->net_counts.assign((size_t)n_edges * stride, 0);
    for (int32_t e = 0; e < n_edges; ++e)
      for (const Bucket& bk : P->edges[e].buckets)
        for (const LeafRef& L : bk.leaves) {
          int32_t* c = &P->net_counts[(size_t)e * stride];
          if (L.kind == QT_T_ZZ && L.layer >= 1 && L.layer <= P->p) ++c[L.layer - 1];
          else if (L.kind == QT_T_MIX && L.layer >= 1 && L.layer <= P->p) ++c[P->p + L.layer - 1];
          else if (L.kind == QT_T_PLUS) ++c[2 * P->p];
        }
  }
  // leaf factors of each planned graph edge (its networks are consecutive)
  {
    std::vector<int32_t> net_leaf(n_edges + 1, 0);
    int32_t count = 0;
    for (int32_t e = 0; e < n_edges; ++e) {
      net_leaf[e] = count;
      for (const Bucket& bk : P->edges[e].buckets) count += bk.leaf_rank > 0 ? 1 : 0;
    }
    net_leaf[n_edges] = count;
    for (int32_t o = 0; o <= P->n_orig; ++o) P->leaf_first[o] = net_leaf[P->net_first[o]];
  }

  // ---- persistent queue: chunks and groups, dependency lists, queue order ----
  P->tasks.clear();
  const TileGeom geom = tile_geom(P->opt.dtype, B, P->opt.lane_items);
  P->tile_items = geom.R;
  // By batch: one angle set never groups (its tiny steps are independent more
  // often than not and run side by side instead); larger batches group steps
  // of up to 4 passes, which saves the per-task overhead of their many tiny
  // adjoint-sweep steps.
  int64_t group_rows = P->opt.group_rows != 0 ? (int64_t)P->opt.group_rows : (B == 1 ? -1 : 4 * (int64_t)geom.RP);
  if (group_rows > geom.R) group_rows = geom.R;
  if (persistent) {
    // A step is split into chunks of `span` warp tiles, one queue task each:
    // chunk_tiles if set; else one tile per chunk while the queue stays
    // within kMaxTasks, fewer chunks per wide step (down to kMinChunks) when
    // it would not.
    int64_t cap = (int64_t)1 << 18;
    if (P->opt.chunk_tiles <= 0)
      for (;;) {
        int64_t total = 0;
        for (const DevBucket& d : P->buckets) total += std::min(step_tiles(d, geom.R), cap);
        if (total <= kMaxTasks || cap <= kMinChunks) break;
        cap >>= 1;
      }
    for (DevBucket& d : P->buckets) {
      const int64_t nt = step_tiles(d, geom.R);
      int64_t span = P->opt.chunk_tiles > 0 ? P->opt.chunk_tiles : (nt + cap - 1) / cap;
      const int32_t by_rank = d.out_rank >= 0 && d.out_rank < 32 ? P->opt.chunk_tiles_by_rank[d.out_rank] : 0;
      if (by_rank > 0) span = std::max<int64_t>(by_rank, (nt + cap - 1) / cap);
      d.span = (int32_t)std::min<int64_t>(std::max<int64_t>(span, 1), INT32_MAX);
      if ((nt + d.span - 1) / d.span > INT32_MAX / 2) return fail(QT_EWIDTH, "step too large for the task queue");
    }
    const int32_t S = P->n_slots;
    // Dependencies: with chain_steps each step of a slot waits for the task
    // queued before it; otherwise for what access_deps finds from the
    // elements the slot's steps touch.  The done counter of a grouped step is
    // its group's last step (`rep`).
    const bool chain = P->opt.chain_steps != 0;
    std::vector<std::vector<int32_t>> sdeps(P->buckets.size());
    if (!chain)
      for (int32_t s = 0; s < S; ++s) {
        std::vector<std::pair<int32_t, int32_t>> nets;
        for (int32_t e : slot_edges[s]) nets.push_back({P->edge_first[e], P->edge_first[e + 1]});
        access_deps(*P, nets, &sdeps);
      }
    std::vector<int32_t> rep(P->buckets.size());
    for (size_t b = 0; b < rep.size(); ++b) rep[b] = (int32_t)b;
    std::vector<int32_t> prev_last(S, -1);
    P->deps.clear();
    std::vector<int32_t> dl;
    auto add_deps = [&](int32_t s, int32_t b, int32_t self) {
      if (chain) {
        if (prev_last[s] >= 0) dl.push_back(prev_last[s]);
        return;
      }
      for (int32_t x : sdeps[b])
        if (rep[x] != self) dl.push_back(rep[x]);
    };
    std::vector<size_t> ei(S, 0);
    std::vector<int32_t> bi(S, 0);
    bool any = true;
    while (any) {
      any = false;
      for (int32_t s = 0; s < S; ++s) {
        if (ei[s] >= slot_edges[s].size()) continue;
        any = true;
        const int32_t e = slot_edges[s][ei[s]];
        const int32_t ns_e = P->edge_first[e + 1] - P->edge_first[e];
        const int32_t gb = P->edge_first[e] + bi[s];
        DevBucket& d = P->buckets[gb];
        const int64_t nt = (step_tiles(d, geom.R) + d.span - 1) / d.span;  // chunks of this step
        dl.clear();
        // consecutive tiny forward steps of a network run on one warp; reverse-sweep
        // steps are not grouped (a warp running hundreds of them back to back
        // left the rest of the GPU waiting on its chain)
        int32_t last = gb;
        if (d.kind == kStepFwd && step_tiles(d, geom.R) == 1 && d.n_rows <= group_rows) {
          int32_t k = 1;
          while (bi[s] + k < ns_e && k < kMaxGroup && P->buckets[gb + k].kind == kStepFwd &&
                 P->buckets[gb + k].n_rows <= group_rows && step_tiles(P->buckets[gb + k], geom.R) == 1)
            ++k;
          last = gb + k - 1;
          for (int32_t j = 0; j < k; ++j) {
            P->buckets[gb + j].ntask = 1;
            P->buckets[gb + j].span = 1;
            P->buckets[gb + j].dep = 0;
            P->buckets[gb + j].n_dep = 0;
            rep[gb + j] = last;
          }
          for (int32_t j = 0; j < (chain ? 1 : k); ++j) add_deps(s, gb + j, last);
          P->tasks.push_back(DevTask{gb, -k, 0, 0});
          bi[s] += k - 1;
        } else {
          d.ntask = (int32_t)nt;
          add_deps(s, gb, gb);
          for (int32_t c = 0; c < d.ntask; ++c) P->tasks.push_back(DevTask{gb, c, 0, 0});
        }
        std::sort(dl.begin(), dl.end());
        dl.erase(std::unique(dl.begin(), dl.end()), dl.end());
        P->buckets[gb].dep = (int32_t)P->deps.size();
        P->buckets[gb].n_dep = (int32_t)dl.size();
        P->deps.insert(P->deps.end(), dl.begin(), dl.end());
        prev_last[s] = last;
        if ((int64_t)P->tasks.size() > INT32_MAX / 2) return fail(QT_ENOMEM, "task queue too long");
        if (++bi[s] == ns_e) {
          bi[s] = 0;
          ++ei[s];
        }
      }
    }
    if (P->opt.queue_order >= 1) {
      // Priorities: the units (a step's chunks, or a group) whose remaining
      // dependency path -- estimated time through their dependents to the end
      // of the slot -- is longest go first.  A dependency's path is longer
      // than each of its dependents', so it stays earlier in the queue.
      // Estimated time of a task: 4 + 0.6 per warp pass over its rows (RP
      // rows a pass; in microseconds, from queue traces), times the rounds
      // its chunks need on about 4096 warps.
      std::vector<int64_t> ustart;
      for (int64_t t = 0; t < (int64_t)P->tasks.size(); ++t)
        if (t == 0 || P->tasks[t].bucket != P->tasks[t - 1].bucket) ustart.push_back(t);
      const int64_t nu = (int64_t)ustart.size();
      ustart.push_back((int64_t)P->tasks.size());
      std::vector<int32_t> unit_of(P->buckets.size(), -1);
      std::vector<double> w(nu, 0.0), path(nu, 0.0), below(nu, 0.0), task_us(nu, 0.0);
      for (int64_t u = 0; u < nu; ++u) {
        const DevTask& t = P->tasks[ustart[u]];
        const int32_t k = t.chunk < 0 ? -t.chunk : 1;
        for (int32_t j = 0; j < k; ++j) {
          const DevBucket& d = P->buckets[t.bucket + j];
          unit_of[t.bucket + j] = (int32_t)u;
          const int64_t rows = std::min<int64_t>(d.n_rows, (int64_t)d.span * geom.R);
          const double passes = (double)((rows + geom.RP - 1) / geom.RP);
          const double us = 4.0 + 0.6 * passes;
          w[u] += us * (double)((d.ntask + 4095) / 4096);
          task_us[u] += us;
        }
      }
      for (int64_t u = nu - 1; u >= 0; --u) {
        path[u] = w[u] + below[u];
        const DevBucket& d = P->buckets[P->tasks[ustart[u]].bucket];
        for (int32_t q = 0; q < d.n_dep; ++q) {
          const int32_t v = unit_of[P->deps[d.dep + q]];
          if (v >= 0) below[v] = std::max(below[v], path[u]);  // every queued step has a unit
        }
      }
      std::vector<DevTask> sorted;
      sorted.reserve(P->tasks.size());
      if (P->opt.queue_order == 1) {
        std::vector<int64_t> order(nu);
        for (int64_t u = 0; u < nu; ++u) order[u] = u;
        std::stable_sort(order.begin(), order.end(), [&](int64_t a, int64_t b) { return path[a] > path[b]; });
        for (int64_t u : order) sorted.insert(sorted.end(), P->tasks.begin() + ustart[u], P->tasks.begin() + ustart[u + 1]);
      } else {
        // queue_order 2: simulated list scheduling.  kSimWarps warps take the
        // ready task of the longest path whenever one is free, each task
        // taking its estimated time; a unit's tasks become ready when every
        // unit it depends on has finished; the queue is the order in which
        // the simulation starts the tasks.  A claimed task then waits less
        // often for a dependency still running (with the path order alone, a
        // dependent often sits right behind its dependency).  Every
        // dependency still comes earlier in the queue.  (Weighing the
        // estimate by step kind from queue traces, or the warp count of the
        // 3-block kernel, measured slightly slower.)
        std::vector<std::vector<int32_t>> dependents(nu);
        std::vector<int32_t> pending(nu, 0), left(nu, 0);
        for (int64_t u = 0; u < nu; ++u) {
          const DevBucket& d = P->buckets[P->tasks[ustart[u]].bucket];
          std::vector<int32_t> vs;
          for (int32_t q = 0; q < d.n_dep; ++q) {
            const int32_t v = unit_of[P->deps[d.dep + q]];
            if (v >= 0 && v != (int32_t)u) vs.push_back(v);
          }
          std::sort(vs.begin(), vs.end());
          vs.erase(std::unique(vs.begin(), vs.end()), vs.end());
          pending[u] = (int32_t)vs.size();
          for (int32_t v : vs) dependents[v].push_back((int32_t)u);
          left[u] = (int32_t)(ustart[u + 1] - ustart[u]);
        }
        using Ready = std::pair<double, int64_t>;  // (path, unit), largest path first, then lower unit
        auto ready_cmp = [](const Ready& a, const Ready& b) {
          return a.first < b.first || (a.first == b.first && a.second > b.second);
        };
        std::priority_queue<Ready, std::vector<Ready>, decltype(ready_cmp)> ready(ready_cmp);
        std::vector<int64_t> next_task(nu);  // next of the unit's tasks to start
        for (int64_t u = 0; u < nu; ++u) {
          next_task[u] = ustart[u];
          if (pending[u] == 0) ready.push({path[u], u});
        }
        using Run = std::pair<double, int64_t>;  // (finish time, unit)
        std::priority_queue<Run, std::vector<Run>, std::greater<Run>> running;
        double now = 0.0;
        int64_t busy = 0;
        while (!ready.empty() || !running.empty()) {
          while (busy < kSimWarps && !ready.empty()) {
            const int64_t u = ready.top().second;
            sorted.push_back(P->tasks[next_task[u]]);
            running.push({now + task_us[u], u});
            ++busy;
            if (++next_task[u] == ustart[u + 1]) ready.pop();  // the unit's last task has started
          }
          if (running.empty()) break;
          const Run r = running.top();
          running.pop();
          --busy;
          now = r.first;
          if (--left[r.second] == 0)
            for (int32_t v : dependents[r.second])
              if (--pending[v] == 0) ready.push({path[v], v});
        }
        if ((int64_t)sorted.size() != (int64_t)P->tasks.size())
          return fail(QT_EINVAL, "internal: the simulated queue left tasks unscheduled");
      }
      P->tasks.swap(sorted);
    }
  }

  // Device images of the queue: each task carries its step's dependency list,
  // each list entry the done count that completes the step it names.
  for (DevTask& t : P->tasks) {
    t.dep = P->buckets[t.bucket].dep;
    t.n_dep = P->buckets[t.bucket].n_dep;
  }
  P->dev_deps.resize(P->deps.size());
  for (size_t i = 0; i < P->deps.size(); ++i) P->dev_deps[i] = DevDep{P->deps[i], P->buckets[P->deps[i]].ntask};

  // Workspace layout.
  WsLayout& L = P->ws;
  const int32_t p = P->p;
  size_t o = 0;
  L.ctrl = o;
  o = align256(o + sizeof(DevCtrl));
  L.done = o;
  o = align256(o + sizeof(int32_t) * P->buckets.size());
  L.buckets = o;
  o = align256(o + sizeof(DevBucket) * P->buckets.size());
  L.tasks = o;
  o = align256(o + sizeof(DevTask) * P->tasks.size());
  L.deps = o;
  o = align256(o + sizeof(DevDep) * P->dev_deps.size());
  L.leaf = o;
  o = align256(o + sizeof(DevLeafFactor) * P->leaf.size());
  L.leaf_first = o;
  o = align256(o + sizeof(int32_t) * P->leaf_first.size());
  L.scal_off = o;
  o = align256(o + sizeof(int64_t) * P->scal_off.size());
  L.scal_begin = o;
  o = align256(o + sizeof(int32_t) * P->scal_begin.size());
  L.net_first = o;
  o = align256(o + sizeof(int32_t) * P->net_first.size());
  L.counts = o;
  o = align256(o + sizeof(int32_t) * P->net_counts.size());
  L.angles = o;
  o = align256(o + sizeof(double) * 2 * (size_t)B * p);
  L.results = o;
  o = align256(o + sizeof(double) * ((size_t)B + (size_t)P->n_orig * B * 2 + (size_t)B * 2 * p));
  L.trig = o;
  o = align256(o + sizeof(double) * kTrigStride * (size_t)B * p);
  L.dz = o;
  if (grad) o = align256(o + sizeof(double) * 2 * (size_t)P->n_orig * B * 2 * p);
  L.gpart = o;
  if (grad) o = align256(o + sizeof(double) * 2 * (size_t)P->leaf.size() * B * kDevMaxLeaves);
  L.data = o;
  o = align256(o + (size_t)es * (size_t)P->data_elems);
  L.total = o;
  P->bound_ws = nullptr;
  return QT_OK;
}

static qt_status cuda_fail(cudaError_t e, const char* what) {
  return fail(QT_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define QT_CUDA(call)                          \
  do {                                         \
    cudaError_t err_ = (call);                 \
    if (err_ != cudaSuccess) return cuda_fail(err_, #call); \
  } while (0)

qt_status run_plan(Plan* P, const double* gamma, const double* beta, double* energy, double* edge_zz,
                   double* grad, void* ws, size_t ws_bytes, void* stream) {
  if (!ws) return fail(QT_EINVAL, "workspace is NULL");
  if (((uintptr_t)ws & 255u) != 0) return fail(QT_EINVAL, "workspace is not 256-byte aligned");
  if (ws_bytes < P->ws.total)
    return fail(QT_ENOMEM, "workspace has " + std::to_string(ws_bytes) + " bytes, plan needs " +
                               std::to_string(P->ws.total));
  if (!gamma || !beta) return fail(QT_EINVAL, "angle pointer is NULL");
  if (grad && !P->opt.gradient) return fail(QT_ESTATE, "gradient requested from a plan without the adjoint sweep");
  cudaStream_t s = (cudaStream_t)stream;
  char* base = (char*)ws;
  const WsLayout& L = P->ws;
  const int32_t B = P->opt.batch;
  const int dtype = P->opt.dtype;
  int dev = -1;
  QT_CUDA(cudaGetDevice(&dev));
  if (P->bound_ws != ws || P->device != dev) {
    if (!P->buckets.empty())
      QT_CUDA(cudaMemcpyAsync(base + L.buckets, P->buckets.data(), sizeof(DevBucket) * P->buckets.size(),
                              cudaMemcpyHostToDevice, s));
    if (!P->tasks.empty())
      QT_CUDA(cudaMemcpyAsync(base + L.tasks, P->tasks.data(), sizeof(DevTask) * P->tasks.size(),
                              cudaMemcpyHostToDevice, s));
    std::vector<DevDep> stalled;
    const DevDep* deps_src = P->dev_deps.data();
    if (P->stall_step >= 0 && P->stall_step < (int32_t)P->buckets.size()) {
      // failure-detection hook: waiters of that step look for a done count that is never reached
      stalled = P->dev_deps;
      for (DevDep& d : stalled)
        if (d.step == P->stall_step) d.need = P->buckets[P->stall_step].ntask + 1;
      deps_src = stalled.data();
    }
    if (!P->dev_deps.empty())
      QT_CUDA(cudaMemcpyAsync(base + L.deps, deps_src, sizeof(DevDep) * P->dev_deps.size(), cudaMemcpyHostToDevice,
                              s));
    if (!P->leaf.empty())
      QT_CUDA(cudaMemcpyAsync(base + L.leaf, P->leaf.data(), sizeof(DevLeafFactor) * P->leaf.size(),
                              cudaMemcpyHostToDevice, s));
    if (!P->leaf_first.empty())
      QT_CUDA(cudaMemcpyAsync(base + L.leaf_first, P->leaf_first.data(), sizeof(int32_t) * P->leaf_first.size(),
                              cudaMemcpyHostToDevice, s));
    if (!P->scal_off.empty())
      QT_CUDA(cudaMemcpyAsync(base + L.scal_off, P->scal_off.data(), sizeof(int64_t) * P->scal_off.size(),
                              cudaMemcpyHostToDevice, s));
    QT_CUDA(cudaMemcpyAsync(base + L.scal_begin, P->scal_begin.data(), sizeof(int32_t) * P->scal_begin.size(),
                            cudaMemcpyHostToDevice, s));
    QT_CUDA(cudaMemcpyAsync(base + L.net_first, P->net_first.data(), sizeof(int32_t) * P->net_first.size(),
                            cudaMemcpyHostToDevice, s));
    if (!P->net_counts.empty())
      QT_CUDA(cudaMemcpyAsync(base + L.counts, P->net_counts.data(), sizeof(int32_t) * P->net_counts.size(),
                              cudaMemcpyHostToDevice, s));
    QT_CUDA(cudaStreamSynchronize(s));  // host vectors may change after return
    P->bound_ws = ws;
    P->device = dev;
  }
  void* data = base + L.data;
  double* trig = (double*)(base + L.trig);
  QT_CUDA(cudaMemsetAsync(base + L.ctrl, 0, L.buckets - L.ctrl, s));  // ctrl + done counters
  if (P->lbar_elems > 0)  // leaf-factor adjoints are accumulated with atomics
    QT_CUDA(cudaMemsetAsync(base + L.data + (size_t)P->elem_bytes * P->lbar_shift, 0,
                            (size_t)P->elem_bytes * P->lbar_elems, s));
  QT_CUDA(launch_trig(dtype, gamma, beta, P->p, B, trig, s));
  QT_CUDA(launch_leaf_factors(dtype, (const DevLeafFactor*)(base + L.leaf), (int32_t)P->leaf.size(), trig, P->p,
                              B, data, s));
  const DevBucket* dbk = (const DevBucket*)(base + L.buckets);
  cudaEvent_t ev_stop = nullptr;
  if (P->profile) {
    if (P->events_used == P->events.size()) {
      cudaEvent_t a, b;
      QT_CUDA(cudaEventCreate(&a));
      QT_CUDA(cudaEventCreate(&b));
      P->events.push_back({a, b});
    }
    QT_CUDA(cudaEventRecord(P->events[P->events_used].first, s));
    ev_stop = P->events[P->events_used].second;
    ++P->events_used;
  }
  if (P->opt.mode == QT_MODE_PERSISTENT) {
    int per_sm = 0;
    QT_CUDA(persistent_occupancy(dtype, P->opt.gradient != 0, P->has_chains, B, &per_sm));
    int n_sm = 0;
    QT_CUDA(cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev));
    const int32_t grid = std::max(1, per_sm) * n_sm;
    QT_CUDA(launch_persistent(dtype, P->opt.gradient != 0, P->has_chains, dbk, (const DevTask*)(base + L.tasks),
                              (int32_t)P->tasks.size(),
                              (DevCtrl*)(base + L.ctrl), (int32_t*)(base + L.done), B, P->opt.lane_items, data,
                              P->data_elems, grid, P->spin_limit, (const DevDep*)(base + L.deps), P->trace, s));
  } else {
    int n_sm = 0;
    QT_CUDA(cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev));
    for (size_t i = 0; i < P->buckets.size(); ++i)
      QT_CUDA(launch_bucket(dtype, P->buckets[i], B, P->opt.lane_items, data, n_sm * 8, s));
  }
  if (ev_stop) QT_CUDA(cudaEventRecord(ev_stop, s));
  QT_CUDA(launch_energy(dtype, data, (const int64_t*)(base + L.scal_off), (const int32_t*)(base + L.scal_begin),
                        (const int32_t*)(base + L.net_first), (const int32_t*)(base + L.counts), trig, P->p,
                        P->n_orig, B, energy, edge_zz, s));
  if (grad)
    QT_CUDA(launch_gradient(dtype, (const DevLeafFactor*)(base + L.leaf), (int32_t)P->leaf.size(),
                            (const int32_t*)(base + L.leaf_first), P->n_orig, P->lbar_shift, trig,
                            (const int32_t*)(base + L.counts), P->p, B, data, (double*)(base + L.gpart),
                            (double*)(base + L.dz), grad, s));
  return QT_OK;
}

qt_status check_plan(Plan* P, void* stream) {
  QT_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
  if (!P->bound_ws) return QT_OK;
  const void* ws = P->bound_ws;
  DevCtrl c;
  QT_CUDA(cudaMemcpy(&c, (const char*)ws + P->ws.ctrl, sizeof(c), cudaMemcpyDeviceToHost));
  if (c.bad_kind != 0)
    return fail(QT_EINVAL, "device check: kind " + std::to_string(c.bad_kind) + " bucket " +
                               std::to_string(c.bad_bucket) + " input " + std::to_string(c.bad_input) + " index " +
                               std::to_string(c.bad_index));
  if (c.status == QT_ETIMEOUT)
    return fail(QT_ETIMEOUT, "persistent queue wait timed out on bucket " + std::to_string(c.spins));
  if (c.status != 0) return fail((qt_status)c.status, "device reported an error");
  return QT_OK;
}

qt_status plan_kernel_times(Plan* P, float* ms, int32_t cap, int32_t* n) {
  int32_t k = 0;
  for (size_t i = 0; i < P->events_used; ++i) {
    QT_CUDA(cudaEventSynchronize(P->events[i].second));
    float t = 0.f;
    QT_CUDA(cudaEventElapsedTime(&t, P->events[i].first, P->events[i].second));
    if (k < cap) ms[k++] = t;
  }
  P->events_used = 0;
  if (n) *n = k;
  return QT_OK;
}

Plan::~Plan() {
  for (auto& e : events) {
    cudaEventDestroy(e.first);
    cudaEventDestroy(e.second);
  }
}

}  // namespace qt
