// Graph validation and reverse-lightcone network construction.
//
// §QAOA algorithm: E = sum over edges of a two-qubit local term; gates that
// commute through the local observable cancel against their conjugates (the
// lightcone).  §Diagonal gate simplification, eq. (example): a diagonal gate
// is a tensor on the indices its qubits already carry, so the ZZ phase of
// eq. (zz_gates_circ) becomes a rank-2 tensor with no new variable, and only
// the mixer X^{2 beta} opens a new variable.
#include <algorithm>
#include <cmath>
#include <set>

#include "qt_internal.h"

namespace qt {

qt_status make_graph(const qt_graph* g, Graph* out) {
  if (!g) return fail(QT_EINVAL, "graph is NULL");
  if (g->n_vertices < 2) return fail(QT_EINVAL, "graph needs at least 2 vertices");
  if (g->n_edges < 1) return fail(QT_EINVAL, "graph needs at least 1 edge");
  if (!g->edges) return fail(QT_EINVAL, "graph edge array is NULL");
  Graph G;
  G.n = g->n_vertices;
  G.adj.assign(G.n, {});
  std::set<std::pair<int32_t, int32_t>> seen;
  for (int32_t i = 0; i < g->n_edges; ++i) {
    int32_t a = g->edges[2 * i], b = g->edges[2 * i + 1];
    if (a < 0 || b < 0 || a >= G.n || b >= G.n)
      return fail(QT_EINVAL, "edge " + std::to_string(i) + " has a vertex out of range");
    if (a == b) return fail(QT_EINVAL, "edge " + std::to_string(i) + " is a self-loop");
    int32_t u = std::min(a, b), v = std::max(a, b);
    if (!seen.insert({u, v}).second)
      return fail(QT_EINVAL, "edge " + std::to_string(i) + " repeats an earlier edge");
    G.eu.push_back(u);
    G.ev.push_back(v);
    G.adj[u].push_back(v);
    G.adj[v].push_back(u);
  }
  for (auto& a : G.adj) std::sort(a.begin(), a.end());
  *out = std::move(G);
  return QT_OK;
}

void build_lightcone(const Graph& g, int32_t p, int32_t edge, Network* net) {
  const int32_t j = g.eu[edge], k = g.ev[edge];
  // top[u] = largest q with u in R_q (R_p = {j,k}, R_{q-1} = R_q + N(R_q));
  // u belongs to R_q exactly for q <= top[u], so top[u] is its mixer count.
  std::vector<int32_t> top(g.n, -1);
  top[j] = top[k] = p;
  for (int32_t q = p; q >= 1; --q)
    for (int32_t u = 0; u < g.n; ++u)
      if (top[u] >= q)
        for (int32_t w : g.adj[u]) top[w] = std::max(top[w], q - 1);

  // Canonical ids: qubits ascending; ket v^0..v^m, then bra w^{m-1}..w^0.
  std::vector<int32_t> ket_base(g.n, -1), bra_base(g.n, -1);
  int32_t nv = 0;
  for (int32_t u = 0; u < g.n; ++u) {
    if (top[u] < 0) continue;
    ket_base[u] = nv;
    nv += top[u] + 1;
    bra_base[u] = nv;          // bra level l (< m) has id bra_base + (m-1-l)
    nv += top[u];
  }
  auto ket = [&](int32_t u, int32_t l) { return ket_base[u] + l; };
  auto bra = [&](int32_t u, int32_t l) {
    return l == top[u] ? ket_base[u] + l : bra_base[u] + (top[u] - 1 - l);
  };

  net->p = p;
  net->edge = edge;
  net->n_vars = nv;
  net->tensors.clear();
  auto add = [&](int8_t kind, int8_t layer, int8_t conj, int32_t a, int32_t b) {
    Tensor t;
    t.kind = kind;
    t.layer = layer;
    t.conj = conj;
    t.rank = b < 0 ? 1 : 2;
    t.v[0] = a;
    t.v[1] = b;
    net->tensors.push_back(t);
  };
  for (int32_t u = 0; u < g.n; ++u) {
    if (top[u] < 0) continue;
    add(QT_T_PLUS, 0, 0, ket(u, 0), -1);
    add(QT_T_PLUS, 0, 1, bra(u, 0), -1);
  }
  for (int32_t q = 1; q <= p; ++q) {
    for (size_t e = 0; e < g.eu.size(); ++e) {
      int32_t a = g.eu[e], b = g.ev[e];
      if (top[a] >= q || top[b] >= q) {
        add(QT_T_ZZ, (int8_t)q, 0, ket(a, q - 1), ket(b, q - 1));
        add(QT_T_ZZ, (int8_t)q, 1, bra(a, q - 1), bra(b, q - 1));
      }
    }
    for (int32_t u = 0; u < g.n; ++u) {
      if (top[u] >= q) {
        add(QT_T_MIX, (int8_t)q, 0, ket(u, q), ket(u, q - 1));
        add(QT_T_MIX, (int8_t)q, 1, bra(u, q), bra(u, q - 1));
      }
    }
  }
  add(QT_T_OBS, (int8_t)p, 0, ket(j, top[j]), -1);
  add(QT_T_OBS, (int8_t)p, 0, ket(k, top[k]), -1);
}

// Single amplitude <x| U(gamma, beta) |+>^n (§Results: the paper's benchmark
// is one amplitude of the full circuit; §Diagonal gate simplification applies
// as above).  Every qubit takes part.  Qubit u carries ket variables
// v_u^0 .. v_u^{p-1} (canonical ids: qubits ascending, u * p + l); its output
// variable v_u^p is projected on bit x_u, so it is no variable at all: the
// last mixer's `new` slot is fixed to x_u.  Tensors: |+> on v_u^0, the
// diagonal ZZ_q on (v_a^{q-1}, v_b^{q-1}) for every edge, MIX_q on
// (v_u^q, v_u^{q-1}).  No bra copy and no observable.
void build_amplitude_network(const Graph& g, int32_t p, const uint8_t* bits, int32_t index, Network* net) {
  auto var = [&](int32_t u, int32_t l) { return u * p + l; };
  net->p = p;
  net->edge = index;
  net->n_vars = g.n * p;
  net->tensors.clear();
  auto add = [&](int8_t kind, int8_t layer, int32_t a, int32_t b) {
    Tensor t;
    t.kind = kind;
    t.layer = layer;
    t.conj = 0;
    t.rank = b < 0 && kind != QT_T_MIX ? 1 : 2;
    t.v[0] = a;
    t.v[1] = b;
    net->tensors.push_back(t);
    return &net->tensors.back();
  };
  for (int32_t u = 0; u < g.n; ++u) add(QT_T_PLUS, 0, var(u, 0), -1);
  for (int32_t q = 1; q <= p; ++q) {
    for (size_t e = 0; e < g.eu.size(); ++e) add(QT_T_ZZ, (int8_t)q, var(g.eu[e], q - 1), var(g.ev[e], q - 1));
    for (int32_t u = 0; u < g.n; ++u) {
      Tensor* t = add(QT_T_MIX, (int8_t)q, q < p ? var(u, q) : -1, var(u, q - 1));
      if (q == p) t->fix[0] = (int8_t)(bits[u] ? 1 : 0);
    }
  }
}

// Interaction structure of the amplitude <0...0| U(gamma, beta) |+>^n in one
// of the four gate representations that §Results compares (structure only:
// every gate is a clique on its variables, written as pairwise rank-2
// tensors, which is the same interaction graph, so the result serves the
// ordering code and its cost, not a contraction).  A gate opens a new
// variable for every qubit index it does not keep; an index a diagonal gate
// keeps (§Diagonal gate simplification) is shared.
//   QT_REP_DEFAULT:     ZZ(gamma) = CNOT (I x Z^{2 gamma}) CNOT, mixer = H Z^{2 beta} H
//                       (Fig. 1), every gate with new output indices
//   QT_REP_DIAGONAL:    the same gates; Z rotations keep their index, and a
//                       CNOT keeps its control index (it is diagonal in it)
//   QT_REP_ZZ:          ZZ(gamma) as one two-qubit gate and the mixer as one
//                       X^{2 beta} gate, both with new output indices
//   QT_REP_ZZ_DIAGONAL: ZZ(gamma) keeps both indices (the hot path's network)
// Each qubit's output index is projected on 0 and so is no variable.
void build_representation_network(const Graph& g, int32_t p, int32_t rep, Network* net) {
  std::vector<std::vector<int32_t>> cliques;
  std::vector<int32_t> cur(g.n), owner;
  int32_t nv = 0;
  for (int32_t u = 0; u < g.n; ++u) {
    cur[u] = nv++;
    owner.push_back(u);
    cliques.push_back({cur[u]});  // |+>
  }
  auto fresh = [&](int32_t u) {
    owner.push_back(u);
    return cur[u] = nv++;
  };
  const bool diag = rep == QT_REP_DIAGONAL || rep == QT_REP_ZZ_DIAGONAL;
  for (int32_t q = 1; q <= p; ++q) {
    for (size_t e = 0; e < g.eu.size(); ++e) {
      const int32_t a = g.eu[e], b = g.ev[e];
      if (rep == QT_REP_ZZ_DIAGONAL) {
        cliques.push_back({cur[a], cur[b]});
      } else if (rep == QT_REP_ZZ) {
        const int32_t a0 = cur[a], b0 = cur[b];
        cliques.push_back({a0, b0, fresh(a), fresh(b)});
      } else {
        for (int32_t half = 0; half < 2; ++half) {  // CNOT, Z^{2 gamma} on the target, CNOT
          const int32_t a0 = cur[a], b0 = cur[b];
          if (diag)
            cliques.push_back({a0, b0, fresh(b)});
          else
            cliques.push_back({a0, b0, fresh(a), fresh(b)});
          if (half == 0) {
            if (diag)
              cliques.push_back({cur[b]});
            else {
              const int32_t t0 = cur[b];
              cliques.push_back({t0, fresh(b)});
            }
          }
        }
      }
    }
    for (int32_t u = 0; u < g.n; ++u) {
      if (rep == QT_REP_ZZ || rep == QT_REP_ZZ_DIAGONAL) {
        const int32_t u0 = cur[u];
        cliques.push_back({u0, fresh(u)});
      } else {  // H, Z^{2 beta}, H
        int32_t u0 = cur[u];
        cliques.push_back({u0, fresh(u)});
        if (diag)
          cliques.push_back({cur[u]});
        else {
          u0 = cur[u];
          cliques.push_back({u0, fresh(u)});
        }
        u0 = cur[u];
        cliques.push_back({u0, fresh(u)});
      }
    }
  }
  // project the outputs: drop each qubit's last variable; number the rest
  // canonically, qubits ascending and each qubit's variables in the order
  // its gates opened them (for ZZ + diagonal: the amplitude network's ids)
  std::vector<int32_t> keep, remap(nv, -1);
  std::vector<char> dropped(nv, 0);
  for (int32_t u = 0; u < g.n; ++u) dropped[cur[u]] = 1;
  for (int32_t v = 0; v < nv; ++v)
    if (!dropped[v]) keep.push_back(v);
  std::stable_sort(keep.begin(), keep.end(), [&](int32_t a, int32_t b) { return owner[a] < owner[b]; });
  const int32_t m = (int32_t)keep.size();
  for (int32_t i = 0; i < m; ++i) remap[keep[i]] = i;
  net->p = p;
  net->edge = -1;
  net->n_vars = m;
  net->tensors.clear();
  for (const auto& c : cliques) {
    std::vector<int32_t> vs;
    for (int32_t v : c)
      if (remap[v] >= 0) vs.push_back(remap[v]);
    for (size_t i = 0; i < vs.size(); ++i)
      for (size_t j = i; j < vs.size(); ++j) {
        if (i == j && vs.size() > 1) continue;
        Tensor t;
        t.kind = QT_T_ZZ;
        t.layer = 0;
        t.conj = 0;
        t.rank = i == j ? 1 : 2;
        t.v[0] = vs[i];
        t.v[1] = i == j ? -1 : vs[j];
        net->tensors.push_back(t);
      }
  }
}

}  // namespace qt
