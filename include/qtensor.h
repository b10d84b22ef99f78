/*
 * qtensor.h -- C ABI of the GB300 lightcone tensor-network QAOA library.
 *
 * Method: arXiv:2106.15740, "Importance of Diagonal Gates in Tensor Network
 * Simulations".  The MaxCut energy E = sum_{(j,k)} (1 - <Z_j Z_k>)/2
 * (§QAOA algorithm) is computed edge by edge; each <Z_j Z_k> is the full
 * contraction of a reverse-lightcone tensor network (§QAOA algorithm,
 * lightcone paragraph) in which diagonal gates -- the ZZ phase and the Z
 * observable -- are tensors on the existing indices of their qubits instead of
 * new 4-index gate tensors (§Diagonal gate simplification, eq. (example)).  The
 * network is contracted by bucket elimination (§Tensor network contraction):
 * for each variable in a greedy min-fill order, every tensor holding it is
 * multiplied and the variable is summed out.
 *
 * Conventions.  Layer q (1..p) applies exp(-i gamma_q Z_j Z_k) on every edge
 * and then exp(-i beta_q X) on every qubit, starting from |+>^n.  Angles are
 * radians, float64.  Batched angle arrays are row-major [B][p].
 *
 * Errors.  Every call returns a qt_status; no call aborts or throws across
 * the ABI.  On failure, qt_last_error() returns a thread-local message that
 * stays valid until the next failing call on the same thread.  Output
 * arguments are left untouched on failure unless stated otherwise.
 *
 * Ownership.  The caller owns every buffer it passes.  Handles returned by
 * the library (qt_network, qt_plan) are owned by the caller and released with
 * the matching *_free call.  Build calls copy the graph and the angles they
 * are given.  Device workspace is caller-allocated memory on the current CUDA
 * device; the library never allocates device memory on its own (plans hold
 * their device-side descriptors in that workspace).
 *
 * Streams.  `stream` is a cudaStream_t passed as void* (NULL = legacy default
 * stream).  Calls taking device pointers are asynchronous on that stream;
 * calls taking host pointers synchronise the stream before returning.
 */
#ifndef QTENSOR_H
#define QTENSOR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  QT_OK = 0,
  QT_EINVAL = 1,    /* invalid argument (graph, p, edge, angle, size, pointer) */
  QT_ENOMEM = 2,    /* workspace smaller than the plan needs, or host allocation failed */
  QT_EWIDTH = 3,    /* contraction width above the plan's width budget */
  QT_ECUDA = 4,     /* a CUDA runtime call failed (message names it) */
  QT_ETIMEOUT = 5,  /* a bounded device-side wait gave up; results are invalid */
  QT_ESTATE = 6     /* call not valid in the handle's current state */
} qt_status;

typedef enum {
  QT_C128 = 0,      /* complex128 storage and arithmetic */
  QT_C64 = 1,       /* complex64 storage, FP32 arithmetic; gates stored as float pairs whose
                       norm is divided out per network, leaf products in float pairs, FP64
                       network products and energy sums */
  QT_C64X2 = 2      /* each real part and imaginary part an unevaluated sum of two floats
                       (hi + lo, about 48 significant bits, 16 bytes per complex number) with
                       error-free FP32 arithmetic: complex128-class results from the FP32 pipes.
                       Gradient plans take it with at most 16 angle sets */
} qt_dtype;

typedef enum {
  QT_MODE_PER_BUCKET = 0, /* one kernel launch per bucket, edges one after another */
  QT_MODE_PERSISTENT = 1  /* one persistent launch over all (edge, bucket, tile) tasks */
} qt_mode;

/* Simple undirected graph.  edges[2*i], edges[2*i+1] are the endpoints of
 * edge i, 0 <= u < v < n_vertices, no repeated edge.  (§QAOA algorithm: the
 * MaxCut instance G=(V,E).) */
typedef struct {
  int32_t n_vertices;
  int32_t n_edges;
  const int32_t* edges;
} qt_graph;

typedef struct qt_network qt_network;
typedef struct qt_plan qt_plan;

/* Tensor kinds of a lightcone network (qt_network_tensor). */
typedef enum {
  QT_T_PLUS = 0,    /* |+> leaf [1,1]/sqrt(2) on a qubit's first variable */
  QT_T_ZZ = 1,      /* diagonal ZZ phase exp(-i gamma_q z_a z_b) on two variables */
  QT_T_MIX = 2,     /* mixer <new| exp(-i beta_q X) |old> on (new, old) */
  QT_T_OBS = 3      /* observable Z: [1,-1] on a qubit's top variable */
} qt_tensor_kind;

/* Build the reverse-lightcone network of edge `edge` (0-based index into
 * g->edges) for depth p >= 1 with angles gamma[p], beta[p] (host pointers).
 * §QAOA algorithm (eq. (1), (2), lightcone paragraph), §Diagonal gate
 * simplification.  Variables get canonical ids: qubits of the lightcone in
 * ascending order; per qubit the ket variables v^0..v^m, then the bra
 * variables w^{m-1}..w^0 (v^m is shared by ket and bra).  On success *out owns
 * a new handle.  QT_EINVAL for a bad graph, p < 1, edge out of range,
 * non-finite angle or NULL pointer. */
qt_status qt_build_lightcone(const qt_graph* g, int32_t p, const double* gamma,
                             const double* beta, int32_t edge, qt_network** out);

/* Number of variables and tensors of a network. */
qt_status qt_network_info(const qt_network* net, int32_t* n_vars, int32_t* n_tensors);

/* Describe tensor t: kind (qt_tensor_kind), layer q (1..p; 0 for |+>, p for
 * the observable), conj (1 for the bra copy), rank (1 or 2) and its variable
 * ids vars[0..rank-1] (for QT_T_MIX: vars[0] = new, vars[1] = old). */
qt_status qt_network_tensor(const qt_network* net, int32_t t, int32_t* kind, int32_t* layer,
                            int32_t* conj, int32_t* rank, int32_t vars[2]);

/* Greedy min-fill elimination order (§Tensor network contraction: the order
 * sets the largest intermediate).  Repeatedly eliminates the variable with the
 * smallest (fill-in, degree, id) in the interaction graph (a clique on each
 * tensor's variables).  `order` must hold n_vars entries; on success *n_vars
 * is set and *width is the largest degree at elimination (the rank of the
 * largest bucket result, the contraction width C of §Results). */
qt_status qt_order(const qt_network* net, int32_t* order, int32_t* n_vars, int32_t* width);

/* Device workspace, in bytes, that qt_contract needs for this network and order. */
qt_status qt_contract_workspace_size(const qt_network* net, const int32_t* order,
                                     qt_dtype dtype, size_t* bytes);

/* Contract the network on the GPU in the given order (bucket elimination,
 * one kernel launch per bucket) and write <Z_j Z_k> to out_zz[0] (real part)
 * and out_zz[1] (imaginary part, zero up to rounding).  `order` is a host
 * array (a permutation of the variables).  `workspace` is device memory of at
 * least qt_contract_workspace_size bytes, 256-byte aligned.  Synchronises
 * `stream`.  QT_EINVAL if order is not a permutation, QT_ENOMEM if the
 * workspace is too small. */
qt_status qt_contract(qt_network* net, const int32_t* order, qt_dtype dtype, void* stream,
                      void* workspace, size_t ws_bytes, double out_zz[2]);

void qt_network_free(qt_network* net);

/* Energy plans: every edge lightcone of a graph, planned once (structure,
 * order, bucket descriptors, memory layout) for `batch` angle sets.  The plan
 * depends on the graph and p only, never on the angles. */
typedef struct {
  int32_t batch;          /* B >= 1 angle sets per call */
  int32_t dtype;          /* qt_dtype */
  int32_t mode;           /* qt_mode */
  int32_t gradient;       /* 1: plan also computes dE/dgamma, dE/dbeta (adjoint sweep; persistent
                             mode; QT_C64X2 with batch <= 16) */
  int32_t max_width;      /* width budget; an edge above it fails with QT_EWIDTH unless sliced
                             (<=0: 31) */
  int32_t lane_items;     /* work items per lane in one warp tile: 8, 16, 32 or 64 (<=0: by batch) */
  int64_t max_workspace;  /* cap on the bytes of the workspace's data region -- intermediates,
                             leaf factors, scalars -- (<=0: no cap); sets edge concurrency.  The
                             step descriptors and the task queue (bytes per queued task, not
                             set by concurrency) come on top */
  int32_t group_rows;     /* persistent mode: consecutive buckets of one edge with at most this many
                             rows run back to back in one task (<0: never; 0: by batch -- never
                             for B = 1, else up to 4 warp passes of rows) */
  int32_t edge_begin;     /* plan the edges [edge_begin, edge_end) of the graph; */
  int32_t edge_end;       /* edge_end <= 0 means all edges from edge_begin on.  Energies and
                             gradients then cover only those edges (a partial sum) */
  int32_t slice;          /* 1: an edge whose width is above max_width is sliced instead of
                             rejected -- variables are fixed, one at a time, until the rest of
                             the network fits, and the 2^s restricted networks are summed */
  int32_t chunk_tiles;    /* persistent mode: warp tiles per queue task (<=0: one, or more for the
                             widest steps when the queue would pass 2^27 tasks) */
  int32_t order_trials;   /* 0: greedy min-fill order.  n > 0: also n seeded randomised greedy
                             orders per edge (§Results orders with a randomised greedy, rgreedy);
                             the one with the fewest bucket elements that is no wider than
                             min-fill is kept.  Values are unchanged (up to rounding order) */
  int32_t order_seed;     /* seed of the randomised orders (with the edge index) */
  double order_tau;       /* temperature: the next variable is drawn with probability
                             proportional to exp(-(fill - min fill) / order_tau) (<=0: 1) */
  int64_t checkpoint_bytes; /* gradient plans: 0 (default) keeps every forward intermediate of a
                             network for the reverse sweep.  > 0 cuts each network's bucket order
                             into segments whose intermediates hold at most this many bytes;
                             only intermediates consumed in a later segment (and those of the
                             last segment) are kept, and the reverse sweep re-runs a segment's
                             forward steps before its adjoint steps (less memory, more traffic;
                             results equal up to rounding order) */
  int32_t chain_steps;    /* persistent mode: 0 (default) a queued step waits only for the steps
                             that last wrote what it reads (bucket elimination forms a tree: the
                             buckets that produced its inputs) and for the last writer and the
                             readers of the workspace it writes, which the arena may reuse --
                             also across the networks that share a workspace slot.  Independent
                             buckets then run at the same time; an adjoint step of a gradient
                             plan likewise waits for its bucket's output adjoint, its other
                             operands and the users of the space its target reuses.  1: every
                             step waits for the step planned before it on its slot (one chain
                             per slot).  Energies are bit-identical either way; gradients agree
                             up to the order of the atomic additions some adjoint steps make */
  int32_t queue_order;    /* persistent mode: 2 (default) the queue is the order in which a
                             list-scheduling simulation of the launch's warps (estimated task
                             times) starts the tasks, each warp taking the ready task with the
                             longest remaining dependency path; 1 the queue takes first the tasks
                             with the longest remaining dependency path (estimated time through
                             their dependents to the end of their slot); 0 it takes the slots
                             round-robin, step by step.  Results are bit-identical either way */
  int32_t chunk_tiles_by_rank[32]; /* persistent mode, per-width schedule: a step whose output rank
                             is r runs in queue tasks of chunk_tiles_by_rank[r] warp tiles when that
                             is > 0 (at least as many as the queue-length rule asks for), else as
                             chunk_tiles says.  The autotuner picks these per width band (§Results:
                             the width of a step sets its cost).  Results are bit-identical for
                             any choice */
  int32_t fuse_chains;    /* persistent energy and amplitude plans (no gradient) of one angle set,
                             or complex64 on the row-wide tiles (34 to 64 angle sets; the first
                             bucket of fan-in 2 or 3): a bucket's result
                             that the next bucket to use it only contracts with a leaf factor --
                             that consumer has no other intermediate input and no variable beyond
                             the result (§Tensor network contraction) -- is never stored: the
                             bucket and up to fuse_chains such consumers in a row (each
                             eliminating the previous one's result) are evaluated in one step,
                             the results' rows contracted with the consumers' leaf factors as
                             they are formed, which removes their writes and reads from the
                             traffic.  0 .. 3 (default 3); 0: every bucket is a step of its own.
                             Results are bit-identical for any value */
} qt_plan_options;

/* Fill `opt` with defaults: batch 1, QT_C128, QT_MODE_PER_BUCKET, no gradient,
 * all edges, tile and grouping chosen by batch. */
void qt_plan_options_default(qt_plan_options* opt);

qt_status qt_plan_create(const qt_graph* g, int32_t p, const qt_plan_options* opt, qt_plan** out);

/* Workspace bytes the plan needs (device memory, 256-byte aligned base). */
qt_status qt_plan_workspace_size(const qt_plan* plan, size_t* bytes);

/* Plan statistics: number of edges, maximum width over edges, total steps
 * (forward, re-run and adjoint), algorithmic bytes moved by the bucket kernels
 * per call (every intermediate input read once per step that reads it, every
 * output written once, times B and the element size; leaf factors of rank
 * <= 10 are not counted) and real FLOPs per call. */
qt_status qt_plan_stats(const qt_plan* plan, int32_t* n_edges, int32_t* max_width,
                        int64_t* n_buckets, double* alg_bytes, double* flops);

/* Per-edge widths (n_edges entries, host array); for a sliced edge, the width
 * of its restricted networks. */
qt_status qt_plan_edge_widths(const qt_plan* plan, int32_t* widths);

/* Per-edge algorithmic bytes of one call (n_edges entries, host array): the
 * plan's alg_bytes split by edge, summed over a sliced edge's networks.
 * The cost model for splitting a graph's edges between GPUs. */
qt_status qt_plan_edge_bytes(const qt_plan* plan, double* bytes);

/* Per-edge number of sliced variables s (the edge is evaluated as 2^s
 * restricted networks; 0 for an edge that fits the width budget). */
qt_status qt_plan_edge_slices(const qt_plan* plan, int32_t* slices);

/* Elimination order the plan contracts unit `unit` (0-based within the
 * plan's edge range, or a bitstring of an amplitude plan) in (§Tensor network
 * contraction: one bucket per variable, in this order).  Variable ids are the
 * network's canonical ids (qt_build_lightcone); for a sliced unit they are
 * the restricted network's ids (the fixed variables removed and the rest
 * renumbered in order).  Call with order = NULL to get *n_vars; otherwise
 * *n_vars holds the capacity of `order` on entry and the variable count on
 * return.  QT_EINVAL for a unit out of range or a capacity too small. */
qt_status qt_plan_edge_order(const qt_plan* plan, int32_t unit, int32_t* order, int32_t* n_vars);

/* Evaluate the plan with DEVICE pointers, asynchronously on `stream`:
 *   gamma, beta : [B][p] float64 angles
 *   energy      : [B] float64, E = sum_e (1 - Re<Z_j Z_k>_e)/2
 *   edge_zz     : [n_edges][B][2] float64 (re, im) per edge, or NULL
 *   grad        : [B][2p] float64 (dE/dgamma_1..p, dE/dbeta_1..p), or NULL;
 *                 requires a plan created with gradient = 1
 * The workspace must stay untouched until the stream reaches the end of the
 * call.  Errors found by the device (a timed-out wait) are reported by the
 * next qt_plan_check call. */
qt_status qt_plan_energy(qt_plan* plan, const double* gamma, const double* beta, double* energy,
                         double* edge_zz, double* grad, void* workspace, size_t ws_bytes,
                         void* stream);

/* Synchronise `stream` and report a device-side failure of earlier calls on
 * this plan (QT_ETIMEOUT) or QT_OK. */
qt_status qt_plan_check(qt_plan* plan, void* stream);

/* Same as qt_plan_energy with HOST pointers: copies the angles to the device,
 * evaluates, copies the results back and synchronises `stream`. */
qt_status qt_plan_energy_host(qt_plan* plan, const double* gamma, const double* beta,
                              double* energy, double* edge_zz, double* grad, void* workspace,
                              size_t ws_bytes, void* stream);

/* Kernel timing for roofline reports.  When profiling is on, every
 * qt_plan_energy call records a pair of CUDA events on its stream around the
 * bucket-contraction launch(es) (not the leaf-factor or energy kernels).
 * qt_plan_kernel_times synchronises those events and writes up to `cap`
 * durations in milliseconds, oldest first, to ms[]; *n gets the number
 * written; the recorded list is then cleared. */
qt_status qt_plan_set_profiling(qt_plan* plan, int32_t on);
qt_status qt_plan_kernel_times(qt_plan* plan, float* ms, int32_t cap, int32_t* n);

/* Allocation-free evaluation (the paper has no counterpart; this serves
 * callers that may not allocate device memory while they run, e.g. a service
 * holding a fixed device-memory budget or a plug-in whose host application
 * owns all device allocations).  Same as qt_plan_energy without the gradient,
 * but the plan's scratch space lives in a device array of
 * qt_static_scratch_bytes() bytes built into the library (held on every device
 * that loads the library until exit) instead of a caller workspace.  gamma,
 * beta, energy ([B]) and edge_zz ([n_edges][B][2] or NULL) are device pointers.
 * Allocates no device memory.  The first call in a CUDA context of a device
 * (its primary context, or a new one after a reset) looks up the array's
 * address there (cudaGetSymbolAddress) with that device current; make that
 * first call before any stream capture.  All calls share the array: the
 * library remembers, per device and context, which plan's descriptors it
 * holds.  A call whose plan is not that plan uploads its descriptors and
 * waits for `stream` before it returns; a call with the same plan only clears
 * the counters that must start at zero and is asynchronous on `stream`.
 * Calls that overlap on the GPU race on the array.  QT_ENOMEM (with the sizes
 * in the message) if the plan's workspace size is above
 * qt_static_scratch_bytes(). */
qt_status qt_plan_energy_static(qt_plan* plan, const double* gamma, const double* beta,
                                double* energy, double* edge_zz, void* stream);
size_t qt_static_scratch_bytes(void);

/* Failure-detection hooks (host-side fault injection; no device fault).
 * qt_plan_set_wait_limit sets how many polls a persistent-queue dependency
 * wait makes before it gives up (default 4194304; each poll sleeps ~0.1 us).
 * qt_plan_inject_stall(plan, 1) makes the next uploads give the dependency of
 * the last queued task that has one a tile count that is never reached, so
 * its waiters run out: the call then ends with every warp stopped and
 * qt_plan_check returns QT_ETIMEOUT; the CUDA context stays usable.
 * qt_plan_inject_stall(plan, 0) restores the plan. */
qt_status qt_plan_set_wait_limit(qt_plan* plan, int32_t polls);
qt_status qt_plan_inject_stall(qt_plan* plan, int32_t enable);

/* Single amplitudes (§Results: the paper benchmarks the cost of one amplitude
 * <x| U(gamma, beta) |+>^n of the full QAOA circuit).  Plans one ket network
 * per bitstring over all qubits -- |+> leaves, the diagonal ZZ phases on the
 * qubits' current indices (§Diagonal gate simplification), the mixers -- with
 * each qubit's output index fixed to its bit, ordered, sliced and contracted
 * like the edge networks (same options; gradient must be 0).  bits is a host
 * array [n_strings][n_vertices] of 0/1 bytes (qubit u = byte u).  The plan is
 * evaluated with qt_plan_amplitudes, whose amp output is a DEVICE array
 * [n_strings][B][2] (re, im) written asynchronously on `stream` (qt_plan_check
 * reports device failures); the per-edge calls reject amplitude plans with
 * QT_ESTATE and qt_plan_amplitudes rejects edge plans.  qt_plan_edge_widths /
 * _slices / _bytes report per bitstring. */
qt_status qt_amplitude_plan_create(const qt_graph* g, int32_t p, const uint8_t* bits, int32_t n_strings,
                                   const qt_plan_options* opt, qt_plan** out);
qt_status qt_plan_amplitudes(qt_plan* plan, const double* gamma, const double* beta, double* amp,
                             void* workspace, size_t ws_bytes, void* stream);

/* Representation cost study (§Results, Fig. diag_costs and diag_costs_vs_n:
 * the contraction cost of one amplitude <0...0|psi> of a QAOA circuit with
 * and without the gate simplifications).  Host only, no device memory.  For
 * representation `rep` (qt_representation) the amplitude's interaction graph
 * is ordered by greedy min-fill, or by the cheapest of min-fill and
 * `order_trials` seeded randomised greedy orders (seed `seed`); *n_vars gets
 * the free variables, *width the contraction width (largest bucket result
 * rank) and *log2_cost log2 of sum_b 2^{|U_b|}, the paper's FLOP measure up
 * to a constant factor.  QT_EINVAL for a bad graph, p or rep. */
typedef enum {
  QT_REP_DEFAULT = 0,     /* CNOT-Z-CNOT ZZ gates and H-Z-H mixers, every gate with new indices */
  QT_REP_DIAGONAL = 1,    /* the same gates, diagonal gates (and CNOT controls) keep their index */
  QT_REP_ZZ = 2,          /* ZZ and X mixer gates, both with new indices */
  QT_REP_ZZ_DIAGONAL = 3  /* ZZ gates keep both indices (the energy and amplitude networks) */
} qt_representation;
qt_status qt_representation_cost(const qt_graph* g, int32_t p, int32_t rep, int32_t order_trials, int32_t seed,
                                 int32_t* n_vars, int32_t* width, double* log2_cost);

/* Queue tracing (measurement; the paper has no counterpart).  With a trace
 * buffer set, every persistent launch of the plan writes, for each queue
 * task t, four uint64 words at trace[4 t .. 4 t + 3]: the device clock
 * (%globaltimer, ns) when a warp claimed the task, when the task's dependency
 * was found complete, and when its tiles were done, then the SM index << 16 |
 * warp index in the block.  `trace` is device memory of at least
 * qt_plan_trace_size() bytes, owned by the caller and left set until it is
 * replaced or cleared with NULL; QT_ESTATE for a per-bucket plan.  Each task
 * is one entry of qt_plan_tasks(): its step and chunk (chunk < 0: a group of
 * -chunk single-tile steps starting at that step), with the step's output
 * rank, edge (index into the plan's edge range), fan-in and kind (0 forward
 * bucket step, 1 adjoint of one input, 2 clearing an accumulated adjoint,
 * 3 adjoint of one input by reduction over its missing variables).  Output
 * arrays may be NULL. */
qt_status qt_plan_trace_size(const qt_plan* plan, size_t* bytes);
qt_status qt_plan_set_trace(qt_plan* plan, void* trace, size_t bytes);
qt_status qt_plan_tasks(const qt_plan* plan, int32_t* n_tasks, int32_t* step, int32_t* chunk,
                        int32_t* out_rank, int32_t* edge, int32_t* n_in, int32_t* kind);

/* Schedule of a persistent plan, for checking on the host that steps which
 * touch the same workspace elements are ordered (§bucket elimination: a
 * bucket reads the tensors earlier buckets produced; the adjoint sweep reads
 * them again).  Step s (0 <= s < n_steps, the order the plan lists them)
 * touches the data elements [acc_lo[a], acc_hi[a]) for a in acc_first[s] ..
 * acc_first[s + 1] (complex elements of the plan's dtype from the data base),
 * writing them if acc_write[a] (an accumulation counts as a write) and
 * reading them otherwise; leaf factors, written before the launch and only
 * read, are not listed.  The queue runs steps in tasks: unit[s] is the first
 * step of the task group that runs s (s itself unless single-tile steps are
 * grouped; a group runs its steps in order on one warp; the chunks of one
 * step write disjoint rows).  A task of unit u starts once every step in
 * deps[dep_first[u] .. dep_first[u] + dep_count[u]) is complete (dep_count
 * is 0 for the other steps of a group).  Arrays may be NULL to ask only for
 * n_steps, n_deps and n_access; otherwise acc_first holds n_steps + 1
 * entries, deps n_deps, acc_lo, acc_hi and acc_write n_access, and the
 * others n_steps.  QT_ESTATE for a per-bucket plan. */
qt_status qt_plan_schedule(const qt_plan* plan, int32_t* n_steps, int32_t* n_deps, int32_t* n_access,
                           int32_t* dep_first, int32_t* dep_count, int32_t* deps, int32_t* acc_first,
                           int64_t* acc_lo, int64_t* acc_hi, int32_t* acc_write, int32_t* unit);

void qt_plan_free(qt_plan* plan);

/* One-shot energy (and gradient if grad != NULL) with HOST pointers: plans
 * the graph for B angle sets in `dtype` (persistent mode), evaluates and
 * frees the plan.  workspace/ws_bytes as for qt_plan_energy; the size comes
 * from qt_energy_workspace_size with the same arguments. */
qt_status qt_energy_workspace_size(const qt_graph* g, int32_t p, int32_t B, qt_dtype dtype,
                                   int32_t gradient, size_t* bytes);
qt_status qt_energy(const qt_graph* g, int32_t p, const double* gamma, const double* beta,
                    int32_t B, qt_dtype dtype, void* stream, void* workspace, size_t ws_bytes,
                    double* energy, double* grad);

/* Thread-local message of the last failing call ("" if none). */
const char* qt_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* QTENSOR_H */
