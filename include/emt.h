/*
 * emt.h -- C ABI of the GB300 hierarchical-inverse EMT network solver.
 *
 * The library solves the per-step EMT network equation G v(t) = i_in(t) + i_his(t - dt)
 * (Sec. II, Eq. 1) as the matrix-vector product v = G^{-1} i (Eq. 2), where G^{-1} is held
 * as the hierarchical store of Sec. III: dense inverses of the leaf sub-networks plus, per
 * internal tree node, the low-rank factors P = G_l^{-1} h_l, Q = G_r^{-1} h_r of Eq. 9 and a
 * small core matrix. It updates that store locally when a branch or a fault changes G (Sec. IV).
 *
 * Conventions for every call:
 *   - Calls return emt_status and never throw or abort; emt_last_error() gives a
 *     thread-local message for the last failing call on the calling thread.
 *   - Host arrays passed in are read during the call only and copied; the caller keeps
 *     ownership. Device pointers (suffix _dev) are caller-owned CUDA device memory.
 *   - Bus indices are 0-based in the caller's original bus order; vectors passed to and
 *     from the library are in that order (the library applies its internal ordering).
 *   - `stream` is a cudaStream_t (NULL = legacy default stream). Work is enqueued on it
 *     and is asynchronous unless the call says it synchronises. Device-side failures
 *     (a non-positive modification denominator, a bounded wait that ran out) are recorded
 *     in a device status word and returned by the next synchronising call.
 *   - Handles are not thread-safe: use one handle from one host thread and one stream.
 *   - The library allocates its own device memory (cudaMalloc) for the stored inverse,
 *     its scratch and simulation state; emt_*_destroy frees it.
 */
#ifndef EMT_H
#define EMT_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  EMT_OK = 0,
  EMT_ERR_INVALID = 1,     /* bad argument or inconsistent input                     */
  EMT_ERR_NOMEM = 2,       /* device or host allocation failed                       */
  EMT_ERR_SINGULAR = 3,    /* modification would make G singular / indefinite        */
  EMT_ERR_CUDA = 4,        /* CUDA runtime error (message has the CUDA error string) */
  EMT_ERR_TIMEOUT = 5,     /* a bounded device-side wait ran out                     */
  EMT_ERR_STATE = 6,       /* call not valid in the handle's current state           */
  EMT_ERR_UNSUPPORTED = 7  /* valid request outside what this build implements       */
} emt_status;

/* Store variants (Sec. III): EXACT uses the Woodbury core S^{-1} at each node and holds the
 * exact inverse; PAPER uses the core [[0, I], [I, 0]], i.e. M = -P Q^T of Eq. 9 (Algorithm 1),
 * the paper's approximate inverse. */
enum { EMT_MODE_EXACT = 0, EMT_MODE_PAPER = 1 };

/* Arithmetic of the hot apply. FP64: double storage and arithmetic. FF64: float-float
 * pairs (8 bytes per element, ~48-bit significand) with compensated FP32 arithmetic.
 * FP32: float storage and arithmetic; emt_apply refines against the FP64 residual. */
enum { EMT_PREC_FP64 = 0, EMT_PREC_FF64 = 1, EMT_PREC_FP32 = 2 };

typedef struct emt_tree emt_tree;
typedef struct emt_hinv emt_hinv;
typedef struct emt_sim emt_sim;

/* Conductance graph (Sec. II): G = sum over branches of g_e u_e u_e^T with u_e = e_from - e_to,
 * or u_e = e_from for a branch to ground (to = -1). g_e != 0: negative values carry mutual
 * couplings (three-phase branches); G must be positive definite (EMT_ERR_SINGULAR otherwise).
 * Bus-to-bus branches are the edges the partition sees; their index in this list is their
 * branch id. */
typedef struct {
  int32_t n_bus;
  int32_t n_branch;
  const int32_t* from;     /* [n_branch] bus index                    */
  const int32_t* to;       /* [n_branch] bus index, or -1 for ground  */
  const double* g;         /* [n_branch] conductance in siemens       */
} emt_graph;

/* Build options. levels > 0: bisect to depth `levels` (2^levels leaves when sizes allow);
 * levels == 0: bisect while a set has more than d_th buses (a leaf holds at most d_th buses,
 * the node threshold of Sec. III-B).
 * nodes_per_bus = B >= 2: the graph's vertices come in groups of B consecutive indices (the three
 * nodes of a three-phase bus, Sec. III-A after Eq. 3; n_bus a multiple of B). The partition bisects
 * groups, so a leaf of b buses holds B b vertices, and cuts are block cuts: one column per (left
 * group, right vertex) of joined groups, with the B entries G[x, y] of the left group's vertices,
 * so a coupled three-phase line is one rank-3 cut (B = 3) instead of one column per vertex
 * branch; d_th counts vertices. 0 or 1: every vertex is its own unit (0 means 3 for the
 * three-phase builders emt_build_hinv_from_network3 and emt_sim3_create). */
typedef struct {
  int32_t levels;
  int32_t d_th;
  int32_t mode;            /* EMT_MODE_*  */
  int32_t precision;       /* EMT_PREC_*  */
  int32_t nodes_per_bus;   /* 0 or 1: none; B >= 2: groups of B vertices, block cuts */
} emt_hinv_opts;

const char* emt_last_error(void);
const char* emt_version(void);

/* ---- partition tree (host only; no GPU needed) ------------------------------------------
 * Recursive bisection minimising the number of cut branches (Sec. III-B, Fig. 2-3): BFS
 * growth from a pseudo-peripheral bus, Kernighan-Lin refinement, deterministic integer
 * tie-breaking. Nodes are numbered breadth first (root 0); leaves read left to right give
 * the nested ordering perm (new position -> bus), so every node is a range [lo, hi). */
emt_status emt_tree_build(const emt_graph* graph, const emt_hinv_opts* opts, emt_tree** out);
/* Sizes of the arrays emt_tree_arrays fills. */
emt_status emt_tree_sizes(const emt_tree* t, int32_t* n_node, int32_t* n_leaf, int32_t* n_cut);
/* Copy the tree out. perm: [n_bus]; lo, hi, parent (-1 at the root), left, right (-1 at
 * leaves), depth: [n_node]; cut_ptr: [n_node + 1]; cut_a, cut_b (positions in perm, a in the
 * left child, b in the right), cut_branch (branch id): [n_cut]. Trees with nodes_per_bus B >= 2
 * have one cut per block column: cut_a is the first position of the left group (its B vertices
 * follow it), cut_b the right vertex, cut_branch -1. Any pointer may be NULL. */
emt_status emt_tree_arrays(const emt_tree* t, int32_t* perm, int32_t* lo, int32_t* hi,
                           int32_t* parent, int32_t* left, int32_t* right, int32_t* depth,
                           int32_t* cut_ptr, int32_t* cut_a, int32_t* cut_b, int32_t* cut_branch);
void emt_tree_destroy(emt_tree* t);

/* ---- hierarchical inverse ---------------------------------------------------------------
 * Algorithm 1 (Sec. III-B): partition, invert every leaf block directly (Cholesky, FP64),
 * then bottom-up form P, Q (Eq. 9) by applying the children's stores to the cut columns,
 * and the node cores. Synchronises `stream` before returning. */
emt_status emt_build_hinv(const emt_graph* graph, const emt_hinv_opts* opts, void* stream,
                          emt_hinv** out);
/* The handle's tree (owned by the handle). */
const emt_tree* emt_hinv_tree(const emt_hinv* h);
/* The handle's partition (Sec. III-B): perm [n_bus] (position -> bus, the nested ordering),
 * node_lo, node_hi, parent [n_node] (node i holds positions [node_lo[i], node_hi[i]); parent -1
 * at the root). n_node comes from emt_tree_sizes(emt_hinv_tree(h), ...). Any pointer may be
 * NULL; the arrays are caller-owned host memory. Host only. EMT_ERR_INVALID for a null handle. */
emt_status emt_hinv_get_partition(const emt_hinv* h, int32_t* perm, int32_t* node_lo, int32_t* node_hi,
                                  int32_t* parent);

/* v = G^{-1} i (Eq. 2) for nrhs column vectors. i_dev, v_dev: device, column-major
 * n_bus x nrhs with leading dimension ld >= n_bus (doubles), bus order. For EMT_PREC_FP32 the
 * result is refined exactly max_refine times (0..16): r = i - G v with the FP64 matrix, then
 * v += (stored inverse) r. The count is fixed, chosen per workload by calibration, so that the
 * call stays asynchronous (a tolerance test would read the device back every pass). tol is not
 * evaluated: tol > 0 (or NaN) returns EMT_ERR_UNSUPPORTED, so that no caller believes a
 * tolerance was enforced; pass tol <= 0. FP64 and FF64 stores ignore max_refine. Asynchronous on
 * `stream`. nrhs >= 1; nrhs == 1 takes the fused single-vector kernels. */
emt_status emt_apply(emt_hinv* h, const double* i_dev, double* v_dev, int32_t nrhs, int64_t ld,
                     int32_t max_refine, double tol, void* stream);

/* G' = G + delta_g u u^T with u = e_a - e_b (bus_b >= 0: conductance change of the lowest-id
 * branch joining a and b; delta_g = -g_e trips branch e) or u = e_a (bus_b == -1: a shunt to
 * ground, e.g. a fault resistance 1/R_f). Sec. IV. EXACT stores get an exact local update
 * (Sherman-Morrison at every node on the paths from the touched leaves to the root, FP64
 * denominators); PAPER stores get Algorithm 2 (re-invert touched leaves, recompute the
 * factors on the paths to the lowest common ancestor). If a denominator is not positive the
 * store is left unchanged and EMT_ERR_SINGULAR is returned. The packed copies the apply kernels
 * read are refreshed by the next emt_apply, once for any number of modifications in between.
 * Synchronises `stream`. */
emt_status emt_modify_branch(emt_hinv* h, int32_t bus_a, int32_t bus_b, double delta_g,
                             void* stream);

/* Scratch reserved by emt_apply_noalloc on every GPU that loads this library, for the
 * life of the process. */
#define EMT_APPLY_NOALLOC_SCRATCH_BYTES (4u << 20)

/* v = G^{-1} i for one vector, like emt_apply with nrhs = 1 and no refinement, but the call
 * allocates no memory at all (no cudaMalloc, no host allocation). It is for callers that cannot
 * allocate once they are running, such as a real-time simulator loop that reserves all its memory
 * at start-up. The paper has no counterpart; it is a deployment convenience. The handle must come
 * from emt_build_hinv (which does allocate, once). The kernels keep their scratch, the per-CTA
 * partial sums of the leaf stage, in one fixed device array of EMT_APPLY_NOALLOC_SCRATCH_BYTES
 * (4 MiB). A store that would need more than that (n_leaf * ceil(max_leaf / 32) * max_leaf * 8
 * bytes) is rejected with EMT_ERR_UNSUPPORTED and a message; use emt_apply for it. FP32 stores
 * return the unrefined FP32 result. i_dev, v_dev: device, n_bus doubles each, bus order.
 * The first call on each device looks up the array's device address and sets kernel attributes.
 * Make that first call before any stream capture on that device. All calls share the array.
 * Calls that overlap on the GPU race on it: serialise calls across streams and handles. Each
 * call rewrites every scratch entry it reads, so nothing has to be cleared between calls.
 * Asynchronous on `stream`. */
emt_status emt_apply_noalloc(const emt_hinv* h, const double* i_dev, double* v_dev, void* stream);

/* Kernels of the single-vector emt_apply on stores whose leaf blocks do not stay in the caches
 * (FP64 or FF64 stores with >= 48 MB of leaf blocks). kernels = 0 (default, automatic): the
 * streaming kernels for such stores, the fused kernels of small stores otherwise. kernels = 1:
 * three kernels (leaf stream, sweep product, expansion) chained with programmatic dependent launch,
 * which also lets consecutive applies overlap, for any FP64 or FF64 store whose leaf rows fit their
 * stages (small stores included). kernels = 2: one cooperative launch of one CTA per SM whose
 * warps each stream their own leaf rows (asynchronous 16-byte copies, one row ahead), which then
 * stages the factor rows and its part of the sweep matrix and meets the other CTAs at two grid-wide
 * barriers (bounded waits: EMT_ERR_TIMEOUT at the next synchronising call if one ran out); it falls
 * back to the three kernels when its plan does not fit (shared memory, co-residency). warps
 * (0 = automatic, else 4..16) sets the warps per CTA of the single launch (a change re-plans on the
 * next emt_apply). *used (may be NULL) receives what the next single-vector apply runs: 2 the
 * single launch, 1 the three kernels, 0 the fused kernels of small stores or a plan not built yet
 * (the first emt_apply builds it). Host only; takes effect on the next emt_apply. */
emt_status emt_apply_tune(emt_hinv* h, int32_t kernels, int32_t warps, int32_t* used);

/* Wait for the handle's work on `stream` and return its device status. */
emt_status emt_hinv_sync(emt_hinv* h, void* stream);
void emt_hinv_destroy(emt_hinv* h);

/* ---- EMT simulation ---------------------------------------------------------------------
 * Element data of one network. Series branches are RL (kind 0: R, L) or RC (kind 1: R, C);
 * every bus may carry a shunt capacitor; sources are Thevenin sines Vm sin(2 pi f t + phi)
 * behind Rs; loads are sine current sinks amp sin(2 pi f t + phi). Trapezoidal companion
 * models (Sec. II) give g = 1/(R + 2L/dt), 1/(R + dt/2C), 2C/dt and 1/Rs. */
enum { EMT_KIND_RL = 0, EMT_KIND_RC = 1 };
typedef struct {
  int32_t n_bus;
  int32_t n_branch;
  const int32_t* from;
  const int32_t* to;
  const int32_t* kind;
  const double* R;
  const double* L;
  const double* C;
  const double* shunt_C;   /* [n_bus] (F) or NULL */
  int32_t n_src;
  const int32_t* src_bus;
  const double* src_Vm;
  const double* src_phi;
  const double* src_Rs;
  int32_t n_load;
  const int32_t* load_bus;
  const double* load_amp;
  const double* load_phi;
  double freq;
} emt_network;

/* emt_build_hinv on the conductance graph of an EMT network at time step dt: the trapezoidal
 * companion conductance of every series branch and shunt capacitor and 1/Rs of every source
 * (Sec. II). Series branch ids are preserved. Synchronises `stream`. */
emt_status emt_build_hinv_from_network(const emt_network* net, double dt, const emt_hinv_opts* opts, void* stream,
                                       emt_hinv** out);
/* The same for a three-phase network (the paper counts three nodes per bus): bus i carries nodes
 * 3i, 3i + 1, 3i + 2. An RL series branch has R and self inductance L per phase and mutual
 * inductance L_mut[e] (0 <= L_mut[e] < L[e]; host array of n_branch, ignored for RC branches)
 * between any two phases; its coupled companion admittance Y = (R I + (2/dt) L3)^-1 enters G as
 * Y (x) (e_a - e_b)(e_a - e_b)^T, written as node branches (phase-to-phase branches of negative
 * conductance between the ends, positive ones within each end's three nodes). RC branches, shunt
 * capacitors and sources act on each phase alone. The store and all calls on it work on the
 * 3 n_bus nodes (node = 3 bus + phase); emt_modify_branch takes nodes. Synchronises `stream`. */
emt_status emt_build_hinv_from_network3(const emt_network* net, const double* L_mut, double dt,
                                        const emt_hinv_opts* opts, void* stream, emt_hinv** out);

/* Event kinds for emt_sim_schedule. Each event is one change of G, applied to the stored
 * inverse as a local update (Sec. IV) before the step is solved. TRIP: target = branch id (the
 * branch opens; its current and history are zeroed). FAULT_ON: target = bus, value = R_f (ohm):
 * G + (1/R_f) e_a e_a^T. FAULT_OFF: target = bus: takes back exactly the conductance of the
 * oldest fault still on at that bus (delta = -1/R_f), so changes made while it was on (trips,
 * faults at other buses, further faults at the same bus) stay. emt_step returns EMT_ERR_STATE,
 * before enqueuing any work, if a FAULT_OFF in its range finds no fault on at its bus. */
enum { EMT_EVENT_TRIP = 0, EMT_EVENT_FAULT_ON = 1, EMT_EVENT_FAULT_OFF = 2 };

/* Create a simulation of `net` at time step dt with nrhs independent columns (nrhs = 1 for
 * the single-network workload). src_scale [nrhs x n_src] and load_scale [nrhs x n_load]
 * (row per column, may be NULL) scale source and load amplitudes per column. Builds the
 * hierarchical inverse; state starts at zero (sources first evaluated at t = dt). */
emt_status emt_sim_create(const emt_network* net, const emt_hinv_opts* opts, double dt,
                          int32_t nrhs, const double* src_scale, const double* load_scale,
                          void* stream, emt_sim** out);
/* A three-phase simulation (the paper counts three nodes per bus, Sec. III-A after Eq. 3; node =
 * 3 bus + phase) on the store of emt_build_hinv_from_network3. Each step injects balanced sine
 * sources and loads (phase p lags phase 0 by 2 pi p / 3), solves v = G^-1 i (Eq. 2) and updates
 * every branch's three-phase history by the trapezoidal rule: for an RL branch with the coupled
 * companion admittance Y = (R I + (2/dt) L3)^-1, i = Y v_e + I_h and
 * I_h <- Y (v_e + ((2/dt) L3 - R I) i); RC branches, shunt capacitors and source resistances act on
 * each phase alone. FP64 or FF64 stores (EMT_ERR_UNSUPPORTED otherwise). The handle works with
 * emt_sim_schedule (EMT_EVENT_TRIP of a series branch opens its three phases: one exact local
 * update of the store per node branch of the line; EMT_EVENT_FAULT_ON / FAULT_OFF with target a
 * node (3 bus + phase) connects it to ground through value = R_f ohm / takes the oldest fault still
 * on at that node back out, each one exact local update; a three-phase fault is three node faults;
 * a FAULT_OFF with no fault on at its node makes emt_step return EMT_ERR_STATE before any work),
 * emt_sim_monitor (node indices), emt_step, emt_sim_read (3 n_bus node voltages), emt_sim_reset,
 * emt_sim_stats and emt_sim_destroy. State starts at zero; sources are first evaluated at t = dt.
 * Synchronises `stream`. */
emt_status emt_sim3_create(const emt_network* net, const double* L_mut, const emt_hinv_opts* opts, double dt,
                           void* stream, emt_sim** out);
/* Schedule an event at a 1-based step (before that step is solved). column = -1: every
 * column (the shared store is modified); column >= 0: that column only (multi-column runs
 * apply it as a per-column Sherman-Morrison correction; TRIP only). */
emt_status emt_sim_schedule(emt_sim* s, int32_t step, int32_t kind, int32_t target,
                            double value, int32_t column);
/* Buses whose voltages emt_step records each step (default: none). */
emt_status emt_sim_monitor(emt_sim* s, int32_t n_mon, const int32_t* buses);
/* Advance n_steps steps. record_dev (device, may be NULL): [n_steps][nrhs][n_mon] doubles of
 * monitored voltages. Asynchronous on `stream`. */
emt_status emt_step(emt_sim* s, int32_t n_steps, double* record_dev, void* stream);
/* Synchronise and copy out state. what: 0 = bus voltages [nrhs][n_bus] (bus order),
 * 1 = current step number (one double). Returns the device status. */
emt_status emt_sim_read(emt_sim* s, int32_t what, double* host_out);
/* Tuning knob for the fused single-column kernels: rows of the leaf blocks per CTA
 * (0 = automatic). Takes effect on the next emt_step. */
emt_status emt_sim_set_rows_per_cta(emt_sim* s, int32_t rows_per_cta);
/* Launch-shape tuning. Single-column simulations: rows of a leaf per CTA (0 = automatic) and the
 * kernel generation (1 = first generation; 2 = programmatic-dependent-launch kernels with a
 * TMA-staged sweep image, used when the network fits their shared-memory limits, else 1;
 * 3 = thread-block-cluster leaf stage reduced through distributed shared memory and an FP64
 * sweep; rows_per_cta then sets the cluster size, ceil(max leaf / rows_per_cta) <= 8;
 * 4 = the whole time loop in one persistent thread-block cluster whose shared memory holds the
 * store; rows_per_cta then is the cluster size (1, 2, 4, 8 or 16 CTAs), FP64 and FF64 stores
 * only; EMT_ERR_UNSUPPORTED, with generation 2 selected instead, when the store does not fit).
 * Multi-column simulations: `kernels` selects the products of the apply (1 = FP32 CUDA cores;
 * 2 = tcgen05 tensor cores with BF16 splits for the leaf stage, and for the expansion when it has
 * a tile for every SM; 3 = tcgen05 for both; 2 and 3 need nrhs a multiple of 4 and >= 32, 2 is
 * the default then); with kernels 2 or 3, rows_per_cta (0, 64, 128, 192 or 256) is the column width of
 * a leaf-GEMM tile (0 = chosen from nrhs). Synchronises the device; takes effect on the next
 * emt_step. */
emt_status emt_sim_tune(emt_sim* s, int32_t rows_per_cta, int32_t kernels);
/* Injection kernel of a multi-column simulation (the history update and right-hand side of Eq. 1,
 * Sec. II): mode 0 chosen from nrhs (the default), 1 one column per thread, 2, 3, 4 two columns
 * per thread with 6, 3 or 2 element ends per memory round trip and 2, 3 or 4 CTAs per SM (nrhs
 * even; EMT_ERR_UNSUPPORTED otherwise; mode 0 takes 4 when nrhs is a multiple of 512, else 1);
 * positions_per_cta 1, 2, 4 or 8 bus positions per CTA, 0 chosen from the sizes (enough CTAs for
 * about sixteen per SM in mode 4, four otherwise). The two-column modes give the same
 * results bit for bit. Single-column and three-phase simulations: EMT_ERR_UNSUPPORTED.
 * Synchronises the device; takes effect on the next emt_step. */
emt_status emt_sim_set_inject(emt_sim* s, int32_t mode, int32_t positions_per_cta);
/* Autotuner: time each candidate on probe_steps steps of this simulation (after 8 untimed
 * steps), keep the fastest and remember it for every later simulation of the same shape in this
 * process (emt_sim_create applies it). Single-column simulations: cluster sizes 1..16 of
 * generation 4, rows per CTA in {4..48} of generations 3, 2 and 1; best_rpc / best_kernels
 * receive rows_per_cta and the generation. Multi-column simulations: FP32 CUDA-core products, and
 * tcgen05 products (kernels 2 and 3) with leaf-GEMM tiles 64, 128, 192 and 256 columns wide; then,
 * with those, the injection kernel with one column per thread and its three two-column variants
 * (even nrhs); best_rpc /
 * best_kernels receive the tile width and `kernels` of emt_sim_tune, emt_sim_stats the injection
 * choice. Three-phase simulations: EMT_ERR_UNSUPPORTED. Resets the simulation. Synchronises the
 * device. best_rpc / best_kernels may be NULL. */
emt_status emt_sim_autotune(emt_sim* s, int32_t probe_steps, int32_t* best_rpc, int32_t* best_kernels,
                            void* stream);
/* Return the simulation to its state right after emt_sim_create: stored inverse restored
 * (every modification undone), voltages and history zeroed, step counter 0; scheduled events
 * and the monitor list are kept. Asynchronous on `stream`. */
emt_status emt_sim_reset(emt_sim* s, void* stream);
/* Sizes of the simulation, for byte/FLOP accounting. out[0..n): n_bus, n_leaf, leaf elements
 * (sum b_j^2), factor elements (sum n_q k_q), core elements (sum (2k_q)^2), CTAs of the fused
 * kernels, element incidences, distinct cut rows, boundary-vector length (sum 2k_q), kernels
 * launched by emt_step/emt_sim_reset since creation, series branches, elements, columns per thread
 * of the injection kernel of a several-column simulation (2 when the columns fill whole blocks of
 * pairs, else 1; 0 for single-column simulations), and its variant (1 one column per thread; 2, 3,
 * 4 two columns per thread with 6, 3 or 2 element ends per memory round trip, 2, 3 or 4 CTAs per
 * SM; 0 for single-column simulations), and columns per thread of the residual kernel (as for
 * the injection; 0 for single-column simulations). */
emt_status emt_sim_stats(const emt_sim* s, int64_t* out, int32_t n);
/* Measurement aid: enqueue `reps` back-to-back launches (as one CUDA graph) of one fused
 * step kernel with the current arguments: which = 0 the leaf-partial kernel, 1 the
 * sweep/expansion kernel. With kernel generation 4 it enqueues one launch of the persistent
 * kernel running `reps` time steps (either `which`). For a simulation of several columns it
 * enqueues `reps` launches, on the operands of the last pass (step at least once first), of:
 * which = 0 the leaf-product GEMM; 1 the kernel splitting the right-hand sides into BF16 blocks
 * for the tensor-core GEMM (EMT_ERR_UNSUPPORTED with the SIMT GEMM); 2 the boundary-sweep GEMM
 * S = K Y_cut; 3 the expansion of a correction pass (with its BF16 split on the tensor-core
 * path); 4 the history update and injection; 5 the float-float residual. Leaves the simulation
 * state undefined: call emt_sim_reset afterwards. Asynchronous on `stream`. */
emt_status emt_sim_bench_kernel(emt_sim* s, int32_t which, int32_t reps, void* stream);
void emt_sim_destroy(emt_sim* s);

/* Failure-path self-test of the bounded device waits: launches one CTA that waits on an mbarrier
 * no one arrives at, with a limit of limit_us microseconds of SM clock (at most 2 s), then sets
 * the device status word. Returns EMT_ERR_TIMEOUT when the wait ran out as designed (the
 * context stays usable), EMT_OK never. Synchronises `stream`. */
emt_status emt_selftest_bounded_wait(int32_t limit_us, void* stream);

/* ---- continuous-batching server --------------------------------------------------------
 * Base networks stay resident on the GPU, each as a multi-column simulation whose columns are
 * request slots; the slot count of a network is its share of hbm_budget_bytes divided by the
 * per-slot footprint (admission by memory). Requests arrive on a wall-clock schedule (seconds
 * after emt_server_run starts); arrived requests are admitted into free slots between ticks of
 * tick_steps steps, every busy network advances one tick on its own stream, finished requests
 * free their slots. A request may carry one change: event_kind 0 trips series branch `target`
 * event_step steps after its start; 1 switches a fault R_f = value ohm to ground at bus `target`
 * for event_len steps; -1 none. Each request's voltages at the network's monitored buses are
 * kept per step. */
typedef struct emt_server emt_server;
emt_status emt_server_create(int32_t tick_steps, uint64_t hbm_budget_bytes, emt_server** out);
/* Add a base network (built now) with up to max_slots concurrent requests; returns its id. */
emt_status emt_server_add_network(emt_server* s, const emt_network* net, const emt_hinv_opts* opts, double dt,
                                  int32_t max_slots, int32_t n_mon, const int32_t* mon_buses, int32_t* net_id);
emt_status emt_server_submit(emt_server* s, int32_t net_id, double arrival_s, int32_t n_steps, int32_t event_kind,
                             int32_t target, double value, int32_t event_step, int32_t event_len, int32_t* req_id);
/* A request on its own (private) network: the network, store options, time step and monitor
 * list are copied now and keyed by their content. When the request arrives, a resident network
 * with the same key serves it (cache hit); otherwise the server builds its store and a simulation
 * of 4 request slots in the admission path (cache miss), so the build is part of this request's
 * latency. Private networks with no active or queued request are evicted, least recently used
 * first, when a new one would exceed the HBM budget; a request whose network cannot be placed yet
 * waits. The event fields are those of emt_server_submit. Host arrays only. */
emt_status emt_server_submit_network(emt_server* s, const emt_network* net, const emt_hinv_opts* opts, double dt,
                                     int32_t n_mon, const int32_t* mon_buses, double arrival_s, int32_t n_steps,
                                     int32_t event_kind, int32_t target, double value, int32_t event_step,
                                     int32_t event_len, int32_t* req_id);
/* Serve every submitted request that has not finished yet; returns when all are done. */
emt_status emt_server_run(emt_server* s);
/* Monitored voltages of a finished request ([n_steps][n_mon], may be NULL) and its times
 * (arrival, admission, completion in seconds since the start of emt_server_run; may be NULL). */
emt_status emt_server_result(const emt_server* s, int32_t req_id, double* out, double* times3);
/* out[0..n): wall seconds, bus-steps served, bus-steps per second, p50 / p99 / max latency (s),
 * largest queue length, ticks, finished requests, private-network builds, private-network cache
 * hits, seconds spent building, evictions. */
emt_status emt_server_stats(const emt_server* s, double* out, int32_t n);
void emt_server_destroy(emt_server* s);

#ifdef __cplusplus
}
#endif
#endif
