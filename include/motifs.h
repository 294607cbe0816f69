/*
 * motifs.h -- C ABI of the GB300 (sm_103a) Motifs-k library.
 *
 * The library counts, for k = 3..6, every weakly connected induced k-vertex
 * subgraph of a directed graph G and groups the counts by isomorphism class,
 * giving the histogram H_k(G) of Problem 1 ("Motifs-k", Sec. 1).  Each subgraph
 * is classified in O(1) by looking its adjacency bits up in a precomputed
 * isomorphism table (Sec. 3.2).  A degree-preserving arc-swap randomiser makes
 * the null graphs of the significance step (Sec. 1, step (c)), and a batched
 * entry point counts the original graph and R null graphs in one pass and
 * returns per-class z-scores.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Every function returns an mt_status and never aborts; no C++ exception
 *   crosses this boundary.  Input errors are reported as MT_EINVAL before any
 *   device work starts.
 * - `stream` is a cudaStream_t passed as void* (NULL = the legacy default
 *   stream).  Work is enqueued on it; unless a function says it synchronises,
 *   results are valid after the stream is synchronised.
 * - Handles (mt_graph, mt_table, mt_batch) own device memory the library
 *   allocated; the caller frees them with the matching *_free.  Buffers passed
 *   in by the caller stay the caller's.  Pointers documented as "device or host"
 *   are inspected with cudaPointerGetAttributes: a device pointer keeps the call
 *   asynchronous, a host pointer makes the call copy and synchronise the stream.
 * - A handle may be used by one host thread at a time.  Counting calls on one
 *   graph handle share its scratch memory: order them on one stream (or
 *   synchronise between them).
 * - Graphs: n vertices numbered 0..n-1 (1 <= n <= 65535), m arcs given as an
 *   int32 CSR of out-neighbours (row_ptr[n+1], col[m]); rows may be unsorted;
 *   self-loops, duplicate arcs, ids outside [0,n) and non-monotone row_ptr are
 *   MT_EINVAL (Sec. 2 defines G by its arc set; the classes of Sec. 3.2 have
 *   no diagonal, so self-loops have no place in a key).
 * - Connectivity is weak: two vertices are adjacent when an arc joins them in
 *   either direction (delta(v) = A(v) u B(v) u C(v), Sec. 2).
 *
 * Class identifiers and canonical masks
 * -------------------------------------
 * A k-vertex digraph on positions 0..k-1 is written as the k(k-1)-bit
 * "canonical-layout mask": bit i*(k-1) + (j - [j > i]) is set iff the arc from
 * position i to position j exists (the adjacency matrix of Sec. 3.2, row-major,
 * diagonal dropped).  The canonical mask of a class is the smallest such mask
 * over all k! orderings of its vertices.  Dense class ids 0..C-1 number the
 * weakly connected classes in ascending order of canonical mask, C = 13, 199,
 * 9,364 and 1,530,843 for k = 3..6 (Sec. 1 prints 1,530,842 for k = 6; the
 * Burnside count of weakly connected 6-vertex digraphs is 1,530,843).
 * Histograms are uint64[C] indexed by dense id; mt_table_class_masks maps ids
 * back to canonical masks.
 */
#ifndef MOTIFS_H_
#define MOTIFS_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  MT_OK = 0,
  MT_EINVAL = 1,        /* bad argument or malformed graph */
  MT_EUNSUPPORTED = 2,  /* k outside 3..6, n > 65535, or a degree too large */
  MT_ENOMEM = 3,        /* device or pinned-host allocation failed */
  MT_ECUDA = 4,         /* a CUDA runtime call failed */
  MT_ETIMEOUT = 5,      /* a bounded device wait expired */
  MT_EOVERFLOW = 6,     /* a device stack or queue bound was exceeded */
  MT_EBUSY = 7          /* admission refused: memory budget or slots full */
} mt_status;

typedef struct mt_graph mt_graph;
typedef struct mt_table mt_table;
typedef struct mt_batch mt_batch;
typedef struct mt_server mt_server;

/* Text for a status code (static storage). */
const char* mt_status_str(mt_status s);

/* Last CUDA error text seen by the library on this thread ("" if none). */
const char* mt_last_error(void);

/* ----------------------------------------------------------------- graphs */

/* Load a directed graph (Sec. 2: G(V,E), n = |V|, m = |E|) from a host CSR of
 * out-neighbours.  `row_ptr` (n+1 int32) and `col` (m int32) are HOST pointers,
 * only read during the call.  The library validates the arrays on the host,
 * copies them into device memory it owns, then builds on the device the sorted
 * directed CSR and the undirected neighbour CSR in which every entry carries
 * the 2-bit relation of Sec. 2 (A: both arcs, B: v->u only, C: u->v only).
 * Synchronises `stream` (a duplicate arc is detected on the device).
 * Errors: MT_EINVAL (null pointers, n < 1, m < 0, row_ptr[0] != 0,
 * row_ptr[n] != m, decreasing row_ptr, id out of range, self-loop, duplicate
 * arc), MT_EUNSUPPORTED (n > 65535), MT_ENOMEM, MT_ECUDA.  *out is set only on
 * MT_OK. */
mt_status mt_graph_load_csr(int32_t n, int32_t m, const int32_t* row_ptr, const int32_t* col,
                            void* stream, mt_graph** out);

/* Free a graph handle (NULL is accepted).  Synchronises the device first. */
mt_status mt_graph_free(mt_graph* g);

/* Sizes of a loaded graph: vertices, arcs, undirected edges (pairs joined by at
 * least one arc) and the largest undirected degree d(v) = |delta(v)|.
 * Synchronises the graph's last stream.  Any output pointer may be NULL. */
mt_status mt_graph_info(const mt_graph* g, int32_t* n, int32_t* m, int32_t* m_undirected,
                        int32_t* max_degree);

/* Copy the sorted directed CSR back to HOST arrays row_ptr[n+1], col[m].
 * Synchronises `stream`. */
mt_status mt_graph_copy_csr(const mt_graph* g, int32_t* row_ptr, int32_t* col, void* stream);

/* ----------------------------------------------------------------- tables */

/* Build the isomorphism table ISO for subgraph size k (Sec. 3.2: every
 * adjacency matrix of k vertices maps to the id of its class), entirely on
 * the device: each of the 2^(k(k-1)) keys is canonicalised by the minimum over
 * all k! vertex orderings, the connected canonical masks are ranked, and each
 * key's slot receives its dense class id, or 0xFFFFFFFF for a disconnected
 * pattern.  Device memory: 4 * 2^(k(k-1)) bytes (4 GiB for k = 6) plus
 * 2^(k(k-1))/4 bytes of scratch freed before return.
 * Key layout ("extension-order key", used by the counting kernels): the k
 * vertices are listed in the order the enumerator adds them; position p >= 1
 * owns the 2p bits starting at k(k-1) - p(p+1) (the last position in the
 * lowest bits), and within them bits 2q and 2q+1 (q < p) are set iff the arcs
 * (position q -> position p) and (position p -> position q) exist.
 * Synchronises `stream`.
 * Errors: MT_EUNSUPPORTED (k outside 3..6), MT_ENOMEM, MT_ECUDA. */
mt_status mt_table_build(int k, void* stream, mt_table** out);

/* The k = 6 table in compact form (the paper's isomorphism table, Sec. 3.2,
 * has one slot per key; it has no compact form): 199 x 2^18 uint32 slots
 * (208 MB) instead of 2^30 (4 GiB), plus a
 * 4096-entry prefix-class array and 4096 x 256 bytes of word relabellings.
 * A 6-vertex key splits into its first four vertices X (key bits 18..29), the
 * fifth vertex's word (bits 10..17) and the sixth's (bits 0..9).  X is mapped
 * to one of the 199 weakly connected 4-vertex classes by relabelling it into
 * that class's canonical order; the two words are relabelled with it (their
 * fields for the vertices of X are permuted, the sixth vertex's field for the
 * fifth is not), which leaves the class of the whole unchanged.  Slot
 * (class of X) << 18 | relabelled fifth word << 10 | relabelled sixth word
 * holds the dense id.  Built from the full table, which is freed before return
 * (peak device memory: the full table's).  Class ids and class masks are the
 * full table's.  Counting with a compact table supports the per-subgraph
 * method only (MT_METHOD_CELLS gives MT_EUNSUPPORTED); mt_table_entries reads
 * compact slots.  Synchronises `stream`.
 * Errors: MT_EUNSUPPORTED (k != 6), MT_ENOMEM, MT_ECUDA. */
mt_status mt_table_build_compact(int k, void* stream, mt_table** out);

/* *compact = 1 for a table from mt_table_build_compact, else 0. */
mt_status mt_table_is_compact(const mt_table* t, int* compact);

mt_status mt_table_free(mt_table* t);

/* k of the table and the number of weakly connected classes C. */
mt_status mt_table_k(const mt_table* t, int* k);
mt_status mt_table_num_classes(const mt_table* t, uint32_t* out);

/* Canonical masks (canonical layout, see above) of all C classes, ascending;
 * index = dense id.  `masks` is a HOST array of C uint32.  Synchronous. */
mt_status mt_table_class_masks(const mt_table* t, uint32_t* masks);

/* Copy table slots [first, first+count) (extension-order keys) to a HOST array
 * of uint32 dense ids (0xFFFFFFFF = disconnected).  Synchronous.  For a compact
 * table the slots are its 199 x 2^18 compact slots.
 * Errors: MT_EINVAL when the range leaves the table's slots. */
mt_status mt_table_entries(const mt_table* t, uint64_t first, uint64_t count, uint32_t* ids);

/* ----------------------------------------------------------------- counting */

/* H_k(G) (Problem 1, Sec. 1) with k = the table's k: for every dense class id c,
 * hist[c] = number of vertex sets S, |S| = k, with G[S] weakly connected and of
 * class c.  `hist` is uint64[C], device or host; it is overwritten.  Every
 * connected set is produced exactly once by the extension enumerator (root =
 * smallest vertex, extension by exclusive neighbours), its adjacency bits are
 * gathered from the labelled neighbour rows (the row-scan strategy of Sec. 3.1)
 * and classified by one table read (Sec. 3.2).  n < k gives all zeros.
 * The call may grow device scratch memory held by the graph handle.  At k = 6
 * that scratch includes 7 extra copies of the histogram (12 MB each): the
 * count spreads its thread blocks over 8 copies, so that fewer blocks add into
 * the same counters, and folds them into `hist` before it completes.
 * Degree limit: each warp's candidate stack holds (k-2) * d + 32 vertex ids,
 * d the largest undirected degree, and that must not exceed 65,535: d <=
 * 65,503 / 32,751 / 21,834 / 16,375 for k = 3 / 4 / 5 / 6 (hubs of the
 * "celebrity" graphs of Sec. 3.1).  Stacks too large for shared memory move
 * to global memory (see mt_count_launch_info).
 * Errors: MT_EINVAL (null handle or hist, or hist on another device than the
 * current one), MT_EUNSUPPORTED (the degree limit above), MT_EOVERFLOW
 * (device stack overflow detected, the histogram is then invalid),
 * MT_ENOMEM, MT_ECUDA. */
mt_status mt_count(const mt_graph* g, const mt_table* t, uint64_t* hist, void* stream);

/* H_k restricted to the connected k-sets whose smallest vertex lies in
 * [root_begin, root_end) (clamped to [0, n)).  Sets are assigned to their
 * smallest vertex, so histograms of disjoint root ranges add up to mt_count's:
 * the unit by which work can be split between calls or devices, and by which
 * a CPU reference can check a large graph on a sample of roots.  Arguments,
 * memory and errors as mt_count. */
mt_status mt_count_roots(const mt_graph* g, const mt_table* t, int32_t root_begin,
                         int32_t root_end, uint64_t* hist, void* stream);

/* Counting method.
 * MT_METHOD_ENUMERATE (default): every connected k-set is produced and its class
 *   read from the table (per-subgraph classification, Sec. 3.2).
 * MT_METHOD_CELLS: the enumeration stops at (k-2)-sets X; the k-sets X + {y, z}
 *   are counted per pair of cells of Part(adj(X)) (Sec. 2) with one table read
 *   per cell pair, arcs between the two added vertices corrected one by one,
 *   as Algorithm 1 of Sec. 3 does.  Same histogram, far fewer table reads.
 *   Each k-set is still counted once (the enumerator owns every (k-2)-set once
 *   and partitions the pairs above it). */
typedef enum { MT_METHOD_ENUMERATE = 0, MT_METHOD_CELLS = 1 } mt_method;

/* Launch tuning of the enumerator (all fields 0 = automatic).
 * - split_cost: estimated work (classified subgraphs) above which a first-level
 *   extension branch of a root is split into second-level work items, and the
 *   target size of first-level items; the root-split threshold.
 * - split_scale: when split_cost is 0, a multiplier of the automatic threshold
 *   (the graph's total estimate spread over 64 items per resident warp).
 *   The threshold is never set below 1/5 of the automatic one, which bounds the
 *   number of work items.
 * - warps_per_block: block size in warps, 1..32.
 * - stack_cap: candidate-stack entries per warp (the stack depth).  Automatic is
 *   (k-1) * max degree + 32, which cannot overflow; a smaller value saves shared
 *   memory, and an overflow is detected and reported as MT_EOVERFLOW.
 * - method: an mt_method. */
typedef struct {
  double split_cost;
  double split_scale;
  int warps_per_block;
  int stack_cap;
  int method;  /* mt_method */
} mt_tuning;

/* The automatic launch mt_count would make for `g` at k (host-side
 * planning only, no device work): block size in warps, number of blocks (one
 * persistent block per SM), candidate-stack entries per warp, and the memory
 * layout as bits: 1 = the graph's CSR copied into shared memory, 2 = relation
 * words in shared memory (else per-warp global slices), 4 = candidate stacks
 * in per-warp global slices (chosen when shared-memory stacks would leave
 * fewer than 16 warps, e.g. for hubs of thousands of neighbours).  Any output
 * pointer may be NULL.  The paper has no counterpart.
 * Errors: MT_EINVAL, MT_EUNSUPPORTED (k outside 3..6, or the degree limit of
 * mt_count). */
mt_status mt_count_launch_info(const mt_graph* g, int k, int32_t* warps_per_block,
                               int32_t* blocks, int32_t* stack_cap, uint32_t* layout);

/* mt_count with explicit tuning (`tuning` may be NULL = automatic).
 * Errors as mt_count, plus MT_EINVAL for out-of-range fields. */
mt_status mt_count_tuned(const mt_graph* g, const mt_table* t, uint64_t* hist,
                         const mt_tuning* tuning, void* stream);

/* mt_count for programs that must not allocate GPU memory while they run: a
 * service that reserves its whole device-memory budget at start-up (its own
 * pool, or a framework's caching allocator, owns every byte), or a
 * latency-sensitive loop that cannot afford cudaMalloc/cudaFree, which may
 * synchronise the device.  mt_count grows scratch memory on the graph handle;
 * this call instead takes the planner's and the work queue's scratch from one
 * fixed 8 MiB array compiled into the library, reserved on every GPU that loads
 * the library until the process exits, and allocates nothing (no cudaMalloc,
 * no cudaFree, no allocating library call).  The paper has no counterpart: it
 * is a deployment variant of the same count.
 * - `hist` must be device memory (uint64[C]); it is overwritten.  Results equal
 *   mt_count's.  The call is asynchronous on `stream`.
 * - The first call on each device looks up the array's device address
 *   (cudaGetSymbolAddress) with that device current; make that first call
 *   before any stream capture.
 * - All calls share the one array: calls that overlap on the GPU (other
 *   streams or host threads) race and give wrong counts.  Serialise them.
 * - The call returns once the work is enqueued, before the kernels run, so it
 *   cannot report what they find (a stack or queue overflow, an expired idle
 *   wait).  Their status word stays in the fixed array until the next call:
 *   read it with mt_count_noalloc_error after the count, before the next
 *   mt_count_noalloc.  A non-zero word means the histogram is invalid.
 * - Errors: MT_EINVAL (null handle, hist not device memory, or hist on
 *   another device than the current one), MT_EUNSUPPORTED when the graph
 *   needs more scratch than the array holds (mt_last_error() gives both
 *   sizes; use mt_count), MT_ECUDA. */
mt_status mt_count_noalloc(const mt_graph* g, const mt_table* t, uint64_t* hist, void* stream);

/* Status of the last mt_count_noalloc on the current device (the paper has
 * no counterpart).  Waits for `stream` (the stream of that count), copies the
 * device status word out of the fixed array into *err (HOST, may be NULL;
 * 0 = the histogram is exact) and returns MT_OK for 0, MT_ETIMEOUT when a
 * bounded device wait expired (see mt_set_wait_limit), MT_EOVERFLOW for a
 * stack, queue or class-id bound exceeded; in both cases the histogram is
 * invalid.  Allocates nothing.  MT_ECUDA if the copy fails. */
mt_status mt_count_noalloc_error(uint32_t* err, void* stream);

/* Caller-provided scratch for the counts of one graph handle (the paper has no
 * counterpart; for callers whose device memory comes from their own allocator,
 * e.g. a torch tensor).  mt_workspace_query: the bytes of scratch that
 * mt_count / mt_count_roots of `g` at k need (automatic launch; a tuned launch
 * may need more; at k = 6 they include the histogram copies described at
 * mt_count).  Errors: MT_EINVAL, MT_EUNSUPPORTED (k outside 3..6).
 * mt_set_workspace: attach `bytes` of DEVICE memory at `ws` (256-byte aligned;
 * the caller keeps ownership and must keep it alive until it is detached or
 * the graph is freed) as the scratch of every later count of `g`; those counts
 * then allocate no device memory, and one that needs more than `bytes` fails
 * with MT_EINVAL (mt_last_error gives both sizes).  ws = NULL detaches it (the
 * library allocates its own scratch again).  Synchronises the device (an
 * earlier count may still use the previous scratch); frees scratch the library
 * had allocated for `g`.  Counts on one handle share its scratch: order them on
 * one stream.  Errors: MT_EINVAL (not device memory, misaligned, empty). */
mt_status mt_workspace_query(const mt_graph* g, int k, size_t* bytes);

/* Limit, in nanoseconds, of the device wait of a warp that has run out of work
 * and waits for work handed over by the other warps of its block (the wait is
 * also bounded by a poll count).  When it expires the warp stops and the count
 * reports MT_ETIMEOUT (its histogram is then incomplete).  Applies to the
 * launches enqueued after the call, process-wide (a batch replays the limit in
 * force when its step was captured); 0 restores the default of 60 s.  A fault-injection hook: a limit of a few nanoseconds makes any count
 * whose warps go idle at different times report MT_ETIMEOUT, without a GPU
 * fault or hang.  The paper has no counterpart. */
mt_status mt_set_wait_limit(uint64_t ns);
mt_status mt_set_workspace(mt_graph* g, void* ws, size_t bytes);

/* Diagnostics of the last counting call on this graph: number of work items
 * the planner made, the device error word (0 = fine; non-zero = stack or queue
 * overflow, the histogram is invalid) and the enumerator's time in ms (device
 * events around planner + enumerator).  Waits for that call to finish.  With a
 * device histogram, mt_count does not synchronise, so overflow is reported
 * only here. */
mt_status mt_count_stats(const mt_graph* g, uint64_t* items, uint32_t* err, float* ms);

/* ----------------------------------------------------------------- null model */

/* One null graph by degree-preserving directed arc swaps (Sec. 1 step (c); the
 * paper names no randomisation model, the reading is the switch of Milo et al.):
 * attempt t = 0..swaps-1 draws arc positions e1, e2 from SplitMix64 outputs 2t
 * and 2t+1 of `seed` (index = floor(r * m / 2^64)); arcs (a->b), (c->d) become
 * (a->d), (c->b) unless e1 == e2, a == c, b == d, a == d, c == b, or a new arc
 * already exists; attempts run in order, one after another.  In- and
 * out-degrees are preserved.  The result is a new graph handle (sorted CSR and
 * undirected CSR rebuilt on the device).  Synchronises `stream`.
 * Errors: MT_EINVAL, MT_ENOMEM, MT_ECUDA. */
mt_status mt_randomize(const mt_graph* src, uint64_t seed, uint64_t swaps, void* stream,
                       mt_graph** out);

/* Dyad-preserving null graph (reciprocity kept; the paper names no model, this
 * is the reading that swaps mutual pairs and one-way arcs separately): the arcs
 * are split, in CSR order, into singles (u->v without v->u) and mutual dyads
 * {u,v} listed once from the smaller end.  Attempt t = 0..attempts-1 takes
 * SplitMix64 outputs 3t, 3t+1, 3t+2 of `seed`: the first picks the list
 * (singles if floor(r * (S + D) / 2^64) < S), the other two pick two entries
 * (a,b), (c,d) of it (index = floor(r * len / 2^64)), which become (a,d), (c,b)
 * unless the entries coincide, a == c, b == d, a == d, c == b, or a new pair is
 * already adjacent in either direction.  In- and out-degrees, each vertex's
 * number of mutual partners and the dyad census are preserved.  Synchronises
 * `stream`.  Graphs whose arc set does not fit shared memory (m above about
 * 17,000) keep it in global memory.  Errors: MT_EINVAL, MT_ENOMEM, MT_ECUDA. */
mt_status mt_randomize_dyads(const mt_graph* src, uint64_t seed, uint64_t attempts, void* stream,
                             mt_graph** out);

/* Batched null model: the original graph plus R null graphs (seeds[r], `swaps`
 * attempts each) counted in one persistent launch.  The handle pre-allocates
 * every buffer; the first mt_batch_run captures the whole step (randomise,
 * rebuild, plan, count, z-scores) into a CUDA graph on `stream` and later runs
 * replay it.  R >= 1. */
mt_status mt_batch_create(const mt_graph* g, const mt_table* t, int R, uint64_t swaps,
                          mt_batch** out);
mt_status mt_batch_free(mt_batch* b);

/* mt_batch_create with explicit tuning of the counting launch (NULL = automatic). */
mt_status mt_batch_create_tuned(const mt_graph* g, const mt_table* t, int R, uint64_t swaps,
                                const mt_tuning* tuning, mt_batch** out);

/* Null models of a batch: degree-preserving arc swaps (mt_randomize) or
 * dyad-preserving swaps that also keep reciprocity (mt_randomize_dyads). */
typedef enum { MT_NULL_ARC_SWAP = 0, MT_NULL_DYAD_SWAP = 1 } mt_null_model;

/* mt_batch_create with a choice of null model (an mt_null_model) and tuning
 * (NULL = automatic).  `swaps` is the number of attempts per null graph.
 * Errors: as mt_batch_create. */
mt_status mt_batch_create_ex(const mt_graph* g, const mt_table* t, int R, uint64_t swaps,
                             int null_model, const mt_tuning* tuning, mt_batch** out);

/* Run a batch.  `seeds`: HOST array of R uint64.  `hists`: uint64[(R+1)*C]
 * (row 0 = original graph, row r = null graph r), device or host.  `z`:
 * double[C], device or host, may be NULL: the z-score of each class,
 * z = (H(G) - mu) / sigma with mu and sigma the mean and population standard
 * deviation of the R null counts in float64 (sigma = 0: z = 0 if H(G) == mu,
 * else +-inf).  Errors as mt_count. */
mt_status mt_batch_run(mt_batch* b, const uint64_t* seeds, uint64_t* hists, double* z,
                       void* stream);

/* Device-side timing of the last mt_batch_run's phases, milliseconds:
 * out[0] randomise + rebuild, out[1] plan + count, out[2] z-scores. */
mt_status mt_batch_phase_ms(const mt_batch* b, float out[3]);

/* Error word of the last mt_batch_run's counting launch (0 = fine; non-zero =
 * stack or queue overflow, the histograms are invalid).  Synchronises the
 * device. */
mt_status mt_batch_error(const mt_batch* b, uint32_t* err);

/* One-shot form of the batch: create, run, free. */
mt_status mt_count_batch(const mt_graph* g, const mt_table* t, const uint64_t* seeds, int R,
                         uint64_t swaps, uint64_t* hists, double* z, void* stream);

/* ----------------------------------------------------------------- ceilings */

/* Measured ceilings of the two memory operations the classification performs
 * per subgraph: random 4-byte reads from a table of `table_words` uint32 (one
 * table read, Sec. 3.2) and random 64-bit atomic adds into `hist_words`
 * counters (one histogram add), both with hashed in-kernel indices and the
 * whole GPU busy.  Sizes are powers of two.  Synchronous; allocates and frees
 * its buffers.  Errors: MT_EINVAL, MT_ENOMEM, MT_ECUDA. */
mt_status mt_probe_rates(uint64_t table_words, uint64_t hist_words, double* gathers_per_s,
                         double* atomics_per_s);

/* ----------------------------------------------------------------- serving */

/* A request server with continuous batching (the paper has no serving layer;
 * its parallelism is threads over graphs, Sec. 4).  The per-k tables given here
 * (NULL = that k is not served) stay resident.  Requests are admitted in
 * arrival order while fewer than `max_slots` are active and their device
 * memory (graph + histogram + a planner share, counted by the server) fits in
 * `memory_budget` bytes.  Work runs in rounds: each round gives every active
 * request a root range whose estimated cost is its share of `round_cost`
 * (estimated k-subgraphs; a k-set belongs to its smallest vertex, so the
 * ranges of one request never overlap; shares are water-filled, so a request
 * needing less than an equal share finishes and the rest goes to the others)
 * and launches one enumeration per k over all requests' ranges, each k on its
 * own stream.  A request that arrives while a round runs joins the next round.
 * The server owns six CUDA streams; one host thread drives it. */
mt_status mt_server_create(const mt_table* t3, const mt_table* t4, const mt_table* t5,
                           const mt_table* t6, size_t memory_budget, int max_slots,
                           double round_cost, mt_server** out);
mt_status mt_server_free(mt_server* s);

/* Queue a count request for H_k of the graph given as a HOST CSR (copied; the
 * caller may free it on return).  Validated like mt_graph_load_csr.  *id
 * identifies the request.  Errors: MT_EINVAL, MT_EUNSUPPORTED (no table for k
 * or n > 65535). */
mt_status mt_server_submit(mt_server* s, int k, int32_t n, int32_t m, const int32_t* row_ptr,
                           const int32_t* col, uint64_t* id);

/* Run one round: admit what fits, launch this round's work, and complete the
 * requests whose last range ran in the previous round (waits for that round
 * only).  Reports how many requests completed, and how many are active and
 * pending afterwards (any pointer may be NULL). */
mt_status mt_server_step(mt_server* s, int32_t* completed, int32_t* active, int32_t* pending);

/* State of a request: 0 pending, 1 active, 2 done, 3 failed.  When done and
 * `hist` (HOST uint64[C]) is given, copies H_k and forgets the request.  A
 * failed request returns its error (MT_EINVAL for a duplicate arc found on the
 * device, MT_EBUSY when it can never fit the budget, MT_EUNSUPPORTED when its
 * k's table and the server's method do not go together -- the cell method
 * with a compact k = 6 table --, MT_ENOMEM when a round's scratch for its k
 * cannot be allocated) and is forgotten; other requests are not affected.
 * `latency_ms` = completion time - submission time on the host clock. */
mt_status mt_server_result(mt_server* s, uint64_t id, int32_t* state, uint64_t* hist,
                           double* latency_ms);

/* Counting method of the rounds launched from now on (an mt_method; the
 * default is MT_METHOD_ENUMERATE).  Results do not depend on it. */
mt_status mt_server_set_method(mt_server* s, int method);

/* Device bytes currently charged against the budget by active requests. */
mt_status mt_server_used_bytes(const mt_server* s, size_t* used);

#ifdef __cplusplus
}
#endif

#endif /* MOTIFS_H_ */
