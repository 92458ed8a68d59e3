/*
 * csp.h - C ABI of libcsp, a CUDA (sm_103a) solver for the constrained shortest path
 * problem on lattice graphs by the "water flow" cycle of I. Matic, "A parallel
 * algorithm for the constrained shortest path problem on lattice graphs"
 * (arXiv 1511.06441).
 *
 * Problem (Section 1 of the paper): an undirected lattice subgraph G of Z^d (or a general
 * graph of bounded degree, below), every edge e with a travel time f1(e) >= 1 and a weight
 * f2(e) >= 0 (integers), disjoint vertex sets A and B and a bound M.  Find F1 = min F1(pi) over paths pi from A to B with
 * F2(pi) < M, plus the endpoint X in B, the last edge x = (Y -> X) and F2 of that path
 * (what the paper's reconstruction by repeated application needs).
 *
 * Lattice layout (every entry point that takes a lattice):
 *   - d in [1, 4]; extents n_0..n_{d-1} >= 1; V = prod n_k < 2^28.
 *   - vertex id v = sum_k c_k * stride_k, coordinate 0 fastest (stride_0 = 1).
 *   - f1[k*V + v], f2[k*V + v] are travel time and weight of the edge (v, v + e_k),
 *     stored as unsigned 8-bit or 16-bit integers (weight_bytes = 1 or 2).  Entries on
 *     the upper face c_k = n_k - 1 are ignored.  f1 == 0 means the edge is absent.
 *   - direction dir = 2k + s leads from a vertex to its neighbour v + e_k (s = 0) or
 *     v - e_k (s = 1).
 *
 * General graphs (csp_create_graph, undirected; csp_create_digraph, directed; Section 1 of
 * the paper states the method for any graph, and the bounded degree is what the GPU layout
 * needs): up to 8 edges per vertex, given as adjacency slots; the direction of an edge is
 * its slot at the vertex it leaves.
 * A graph handle works wherever a csp_lattice is taken: csp_solve, csp_solve_async,
 * csp_reserve, csp_get_labels, both reconstructions, the batch API (graphs and lattices may
 * share a batch) and the server API (explicit target lists only: a graph has no
 * hyperplanes).  csp_upload_weights accepts lattices only, and csp_solve_static takes a
 * lattice's extents.
 *
 * Every call returns a csp_status and never aborts.  Pointers named *_dev are device
 * pointers; all other pointers are host pointers.  Output buffers are owned by the
 * caller.  Calls on the same lattice must not overlap (a lattice owns one workspace).
 */
#ifndef CSP_H
#define CSP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    CSP_OK = 0,
    CSP_ERR_INVALID = 1,  /* bad argument: d, extents, ids out of range, A and B not disjoint, empty A or B, M >= 2^31 - 1 */
    CSP_ERR_OOM = 2,      /* device or host allocation failed */
    CSP_ERR_CUDA = 3,     /* a CUDA call failed; csp_last_error() has the text */
    CSP_ERR_CAPACITY = 4, /* the flow pool overflowed, or arrival times would reach 2^30 */
    CSP_ERR_TIMEOUT = 5,  /* max_cycles reached, or the solve ran past its time limit (csp_options) */
    CSP_ERR_BARRIER = 6   /* a device-side barrier wait gave up after its time limit */
} csp_status;

typedef struct csp_lattice csp_lattice;

/* Result of one solve.  F1 = -1 (and X, x_src, x_dir, F2 = -1) when no path from A to
 * B has F2 < M (termination 2 of the paper, Algorithm 2). */
typedef struct {
    int64_t F1;        /* minimal travel time F1(pi) subject to F2(pi) < M */
    int64_t X;         /* endpoint in B: largest label (smallest F2), then smallest id */
    int64_t x_src;     /* Y, the other end of the last edge x */
    int64_t x_dir;     /* direction from Y to X (0 .. 2d-1; on a graph the slot of X at Y) */
    int64_t F2;        /* F2 of that path = M - Label(X) */
    int64_t cycles;    /* cycles run = distinct times at which some label improved */
    int64_t updates;   /* active-edge updates: sum over cycles of the flows alive at cycle start */
    int64_t launched;  /* water flows started, phantoms included */
    int64_t passes;    /* sweeps over the flow pool (cycles + prune-only passes) */
    int64_t max_pool;  /* largest flow-pool size seen */
    int64_t arrivals;  /* flows that delivered water (each improved its destination) */
    int64_t improved;  /* label improvements = sum over cycles of the triggered vertices */
    int64_t phantoms;  /* flows started on a directed edge that already carried one (the paper's
                          phantom edges, Step 5); counted only with a trace and CSP_OPT_PHANTOMS,
                          else -1 */
} csp_result;

typedef struct {
    int64_t max_cycles;     /* stop with CSP_ERR_TIMEOUT after this many cycles; 0 = no limit */
    int64_t pool_capacity;  /* flow slots per pool buffer, rounded up to whole chunks of 2048; each
                               CTA of a solve may leave up to two chunks part-filled in a pass.
                               0 = automatic.  csp_solve doubles it and retries on overflow;
                               csp_solve_async reports CSP_ERR_CAPACITY */
    int32_t ctas;           /* CTAs of the persistent kernel; 0 = chosen from the lattice size */
    int32_t time_limit_s;   /* watchdog of the cycle kernel in seconds; 0 = 120.  A solve that runs
                               longer stops with CSP_ERR_TIMEOUT (the GPU is left usable) */
    void *stream;           /* cudaStream_t to run on; NULL = the legacy default stream */
    void *ev_begin;         /* nullable cudaEvent_t recorded on the stream just before the cycle kernel */
    void *ev_end;           /* nullable cudaEvent_t recorded just after it */
    int32_t flags;          /* CSP_OPT_* bits */
    int32_t barrier_us;     /* longest wait at one device barrier, in microseconds, before the solve gives
                               up with CSP_ERR_BARRIER; 0 = 4 s (a barrier round never takes seconds) */
} csp_options;

/* csp_options.flags: with a trace, also count phantoms (csp_result.phantoms); costs a store
 * per staying flow and a load per started flow in every cycle. */
#define CSP_OPT_PHANTOMS 1
/* csp_options.flags: which form of the cycle loop runs the solve (both give identical
 * results, traces, counts and labels).
 *   CSP_OPT_SWEEP  every cycle sweeps every flow in flight (Step 1 as the paper states it).
 *   CSP_OPT_EVENT  a calendar of arrival times: a cycle touches only the flows that arrive,
 *                  the flows it starts and the flows it removes (per-edge queues of flows
 *                  in flight).  Needs max f1 <= 511 (CSP_ERR_INVALID otherwise) and, per
 *                  lattice, 16 B per directed edge plus 8 B per unit of f1 summed over the
 *                  directed edges, built on first use after each weight upload (that first
 *                  solve synchronises its stream once).
 * Neither flag: the library's default form for the handle (csp_default_engine).  Both:
 * CSP_ERR_INVALID.  The first event-form solve on a handle also allocates its calendar
 * (8 B per flow-pool slot of csp_reserve, plus part-filled chunks). */
#define CSP_OPT_SWEEP 2
#define CSP_OPT_EVENT 4
/* csp_options.flags, a test hook for the bounded waits: the last CTA of the solve leaves
 * before its first grid barrier, so every other CTA's wait there runs out (after barrier_us)
 * and the solve returns CSP_ERR_BARRIER with the device left usable.  Needs two CTAs or more. */
#define CSP_OPT_TEST_ABSENT_CTA 8

/* The block shape this library was built with (build parameters chosen by the shape tuner,
 * paper_1511_06441_gb300/tune.py, and cached in paper_1511_06441_gb300/shape.json):
 * shape[0] threads per CTA, shape[1] flows per thread per tile (the flow-pool chunk is their
 * product), shape[2] tiles in flight per CTA in the sweep, shape[3] CTAs per SM of the solve and
 * server kernels, shape[4] CTAs per SM of the batch kernel.  The paper has no counterpart. */
void csp_build_shape(int32_t *shape);

/* Text for a status code (static storage). */
const char *csp_status_string(csp_status s);

/* Text of the last CUDA error seen by this thread ("" if none). */
const char *csp_last_error(void);

/* Creates a lattice: copies f1 and f2 (d*V entries each, layout above) into library-owned
 * device memory and zeroes the ignored upper-face entries.  on_device = 1 means f1 and f2
 * are device pointers.  stream: cudaStream_t or NULL.  *out receives the handle.
 * Errors: CSP_ERR_INVALID (d, extents, weight_bytes), CSP_ERR_OOM, CSP_ERR_CUDA. */
csp_status csp_create_lattice(int d, const int64_t *extents, const void *f1, const void *f2,
                              int weight_bytes, int on_device, void *stream, csp_lattice **out);

/* Creates a general graph (the handle type is shared with lattices).  V in [1, 2^28);
 * slots in [1, 8].  nbr[v * slots + j] is the neighbour of v in slot j, or -1 for an empty
 * slot; f1[v * slots + j] >= 1 and f2[v * slots + j] are that edge's travel time and weight
 * (uint8 or uint16 by weight_bytes; ignored in empty slots).  The graph is undirected:
 * every edge sits in exactly one slot at each end, with the same f1 and f2, and there are
 * no self loops or parallel edges.  All arrays are host arrays and stay the caller's; the
 * library keeps per-vertex edge records and a neighbour table on the device (16 or 32 B +
 * 32 B per vertex).  stream: cudaStream_t or NULL.
 * Errors: CSP_ERR_INVALID (arguments, or a graph that breaks the rules above; the first
 * offending vertex and slot are in csp_last_error), CSP_ERR_OOM, CSP_ERR_CUDA. */
csp_status csp_create_graph(int64_t V, int32_t slots, const int64_t *nbr, const void *f1, const void *f2,
                            int weight_bytes, void *stream, csp_lattice **out);

/* Creates a directed graph: as csp_create_graph, but every slot holds a one-way edge from v to
 * nbr[v * slots + j] (listed once, at its tail), with its own f1 and f2.  In-degrees must not
 * exceed 8 either.  The direction x_dir of a result is the edge's slot at its tail.  The
 * library keeps a second table of incoming edges (32 B more per vertex).
 * Errors: as csp_create_graph ("in-degree above 8" among the reasons). */
csp_status csp_create_digraph(int64_t V, int32_t slots, const int64_t *nbr, const void *f1, const void *f2,
                              int weight_bytes, void *stream, csp_lattice **out);

/* Overwrites the weights of an existing lattice (same layout and width as at creation),
 * without allocating.  on_device as above.  CSP_ERR_INVALID on a graph. */
csp_status csp_upload_weights(csp_lattice *lat, const void *f1, const void *f2, int on_device, void *stream);

/* Frees the lattice and its workspace.  NULL is ignored. */
void csp_destroy_lattice(csp_lattice *lat);

/* Number of vertices of the lattice. */
int64_t csp_num_vertices(const csp_lattice *lat);

/* Allocates the solver workspace now (labels, offers, arrival lists, two flow-pool
 * buffers of pool_capacity slots; 0 = automatic), so that later solves allocate nothing
 * (unless a csp_solve must grow the pool or a longer trace is requested). */
csp_status csp_reserve(csp_lattice *lat, int64_t pool_capacity);

/*
 * Solves one instance: the cycle loop of Algorithm 1 (Initialization, Steps 1-9) run by
 * one persistent GPU kernel until a vertex of B receives water (F1 found) or no flow is
 * left (infeasible).
 *   A, B       host arrays of vertex ids (duplicates allowed, treated as sets); nA, nB >= 1.
 *   M          the bound, F2 < M; M <= 0 gives F1 = -1; M >= 2^31 - 1 is CSP_ERR_INVALID (the
 *              label 2^31 - 1 marks a vertex outside the graph of a reconstruction step).
 *   opt        nullable.
 *   out        result (host).
 *   trace      nullable host buffer of 3 * trace_cap int64: rows (Time, active vertices,
 *              live flows) after the removals of each cycle, row 0 = after initialisation.
 *              Requesting a trace makes the solve count active vertices (slower).
 *   trace_len  nullable; receives the number of rows the solve produced.  If it exceeds
 *              trace_cap only trace_cap rows were written (status still CSP_OK).  A solve
 *              stopped by max_cycles or the watchdog (CSP_ERR_TIMEOUT) returns the rows of
 *              the cycles it completed (rows 0 .. cycles - 1) and their counts in *out.
 * Blocks the calling thread until the result is on the host.
 */
csp_status csp_solve(csp_lattice *lat, const int64_t *A, int64_t nA, const int64_t *B, int64_t nB,
                     int64_t M, const csp_options *opt, csp_result *out,
                     int64_t *trace, int64_t trace_cap, int64_t *trace_len);

/*
 * Asynchronous solve with device-resident sets: enqueues the whole solve on opt->stream
 * and returns without waiting.  A_dev, B_dev are device arrays of int64 ids.  The result
 * is written to result_dev (device, 16 int64: status, F1, X, x_src, x_dir, F2, cycles,
 * updates, launched, passes, max_pool, trace_len, elapsed_ns, arrivals, improved, phantoms;
 * elapsed_ns = device time of the cycle loop, from %globaltimer).  Invalid ids, A and B not
 * disjoint, pool overflow etc. are reported in result_dev[0], not by the return value
 * (which reports only host-side argument errors and launch failures).  trace_dev:
 * nullable device buffer of 3 * trace_cap int64.  The workspace must have been reserved
 * (csp_reserve) with a capacity large enough for this instance.
 */
csp_status csp_solve_async(csp_lattice *lat, const int64_t *A_dev, int64_t nA, const int64_t *B_dev, int64_t nB,
                           int64_t M, const csp_options *opt, int64_t *result_dev,
                           int64_t *trace_dev, int64_t trace_cap);

/*
 * Solve without any device allocation.  The paper has no counterpart: this entry point
 * exists for callers that cannot call cudaMalloc (for example code running inside a
 * framework or runtime that owns every device allocation, or under a memory cap that
 * forbids new allocations).  The solver's scratch memory lives in one file-scope device
 * array of CSP_STATIC_WORKSPACE_BYTES bytes that every GPU loading this library holds
 * until the library is unloaded.
 *   extents, d       as for csp_create_lattice (host array).
 *   f1_dev, f2_dev   the caller's device weights, layout as above; here the upper-face
 *                    entries of f1 MUST be zero (a nonzero one is reported as
 *                    CSP_ERR_INVALID in result_dev[0]).
 *   A_dev, B_dev     device arrays of int64 vertex ids (sets, as for csp_solve_async).
 *   M, max_cycles    as for csp_solve (max_cycles 0 = no limit).
 *   stream           cudaStream_t or NULL.
 *   result_dev       device record of 16 int64, laid out as for csp_solve_async.
 * Enqueues the solve and returns without waiting.  The layout needs 28.125 bytes per vertex
 * (labels, offers, B bitmap, a 16-byte edge record; 16 more for 16-bit weights with
 * d >= 3), 28 bytes per flow-pool slot (two pool buffers and an arrival-list entry) and
 * 8 KiB of arrival list per CTA; whatever the vertex arrays leave of the static array
 * becomes the flow pool.  A lattice whose vertex arrays do not fit is rejected with
 * CSP_ERR_INVALID (csp_last_error() says so); a solve whose flows do not fit reports
 * CSP_ERR_CAPACITY in result_dev[0].  No trace is recorded.  The cycle kernel stops after
 * 120 s of device time (fixed: this entry point takes no csp_options) and then reports
 * CSP_ERR_TIMEOUT in result_dev[0], as a solve stopped by max_cycles does; it always runs the
 * sweep form of the loop.  The first call on a
 * device looks up the array's device address (cudaGetSymbolAddress) for that device;
 * make that first call before capturing any stream.  All calls share the array and
 * each call overwrites what the previous one left, so calls that may overlap on the GPU
 * (other streams, other threads) race and must be serialised by the caller.
 */
#define CSP_STATIC_WORKSPACE_BYTES (64u << 20)

csp_status csp_solve_static(int d, const int64_t *extents, const void *f1_dev, const void *f2_dev,
                            int weight_bytes, const int64_t *A_dev, int64_t nA, const int64_t *B_dev, int64_t nB,
                            int64_t M, int64_t max_cycles, void *stream, int64_t *result_dev);

/* ------------------------------------------------------------------ batched solves
 *
 * Many independent instances (each on its own lattice, with its own sets and bound) in
 * ONE persistent cooperative launch, captured once as a CUDA graph.  A list scheduler
 * (cost model: cycles x per-cycle latency + updates / rate) gives each instance a group
 * of CTAs (a power of two) and a start slot; instances never wait for each other.  The
 * paper solves one instance at a time; this mode and its scheduler are additions.
 */
typedef struct {
    const csp_lattice *lat;   /* the instance's lattice (not owned) */
    const int64_t *A;         /* host array, nA >= 1 */
    int64_t nA;
    const int64_t *B;         /* host array, nB >= 1 */
    int64_t nB;
    int64_t M;
} csp_query;

typedef struct {
    int32_t ctas;             /* CTAs of the launch; 0 = every co-resident CTA */
    int32_t max_group;        /* largest CTA group for one instance (power of 2); 0 = 64 */
    int32_t no_graph;         /* 1 = launch directly instead of through a CUDA graph */
    int32_t reserved;
    int64_t pool_capacity;    /* flow slots per pool buffer per instance (whole chunks of 2048, up to two
                                 part-filled per CTA); 0 = max(2^16, 6V) capped by the flow bound, plus
                                 two chunks per CTA of the largest group */
    int64_t max_cycles;       /* per instance; 0 = no limit */
} csp_batch_options;

typedef struct csp_batch csp_batch;

/* Allocates every instance's workspace, uploads the sets, plans the schedule and
 * captures the launch.  All lattices must use the same weight width.  The lattices must
 * outlive the batch.  Errors: CSP_ERR_INVALID (any query invalid on the host side),
 * CSP_ERR_OOM, CSP_ERR_CUDA. */
csp_status csp_batch_create(const csp_query *q, int64_t n, const csp_batch_options *opt, csp_batch **out);

/* Enqueues one run of the whole batch on stream (cudaStream_t or NULL); asynchronous. */
csp_status csp_batch_run(csp_batch *b, void *stream);

/* Waits for the device and copies the n results (out), per-instance statuses (nullable;
 * CSP_ERR_CAPACITY means that instance's pool was too small) and the per-instance device
 * time of the cycle loop in ns (nullable). */
csp_status csp_batch_results(csp_batch *b, csp_result *out, int32_t *status, int64_t *elapsed_ns);

/* The current schedule: per instance its group size, first CTA, planned start and
 * estimated duration (us); *ctas = the launch width.  Every pointer is nullable. */
csp_status csp_batch_schedule(const csp_batch *b, int32_t *group_size, int32_t *first_cta, double *start_us,
                              double *est_us, int32_t *ctas);

/* Autotuner step: refits the cost model to one measured run (elapsed_ns and results
 * from csp_batch_results), re-plans the schedule and re-captures the graph. */
csp_status csp_batch_tune(csp_batch *b, const int64_t *elapsed_ns, const csp_result *res);

/* The cost model the schedule uses (per-cycle latency of a one-CTA group and of a larger
 * group, us; updates per us per CTA) and the planned makespan (us).  Nullable outputs. */
csp_status csp_batch_model(const csp_batch *b, double *lat_single_us, double *lat_group_us, double *rate,
                           double *makespan_us);

void csp_batch_destroy(csp_batch *b);

/* Convenience: create, run, read the results, re-solve any instance whose pool
 * overflowed with csp_solve (which grows its pool), destroy.  status: nullable, n. */
csp_status csp_solve_batch(const csp_query *q, int64_t n, const csp_batch_options *opt, csp_result *out,
                           int32_t *status);

/*
 * The minimizing path by repeated application of the method (Section 1 of the paper):
 * after a solve gives X, x = (Y -> X) and F2, solve again on G' with A' = A, B' = {Y},
 * M' = F2 - f2(x) + 1 and V' = V minus (B and the path vertices found so far); each step
 * yields the next vertex back, until Y is in A.  (The paper writes B' = {X} and
 * M' = F2 - f2(x); with the strict bound F2 < M that would exclude the sub-path itself.)
 *   res    nullable: the result of csp_solve for (A, B, M); solved here when NULL.
 *   path   host buffer of cap int64: vertex ids from the A end to X.
 *   len    receives the number of vertices (0 if no path has F2 < M).  If *len > cap the
 *          call returns CSP_ERR_CAPACITY and writes nothing.
 * One full solve per path vertex; blocks until done.
 */
csp_status csp_reconstruct_path(csp_lattice *lat, const int64_t *A, int64_t nA, const int64_t *B, int64_t nB,
                                int64_t M, const csp_result *res, int64_t *path, int64_t cap, int64_t *len);

/*
 * The same path as csp_reconstruct_path from ONE solve: the solve records, for every
 * vertex, the time and winning arrival edge of its first improvement and, in a log, every
 * improvement pass by pass; a GPU backtrack then walks from (X, F1) along the recorded
 * edges (the flow on x left Y at F1 - f1(x), when Y improved; and so on back to A).
 * Repeated application would remove the path vertices found so far; no earlier vertex of
 * the path is reached sooner with better water through a later one, so the result is the
 * same path.
 *   opt           nullable, as for csp_solve.
 *   log_capacity  improvement records the log may hold (8 bytes each): > 0 that many;
 *                 0 = a quarter of the free device memory; < 0 = no log (first improvements
 *                 only, which suffice when every path vertex is reached at its first
 *                 improvement, e.g. when the bound does not bind).  A path that needs a
 *                 record the log dropped returns CSP_ERR_CAPACITY.
 *   res           receives the solve's result (as csp_solve).
 *   path, cap, len  as for csp_reconstruct_path (A end first; 0 vertices if infeasible).
 * Allocates and frees its record buffers (8 bytes per vertex plus the log); blocks until done.
 */
csp_status csp_reconstruct_fast(csp_lattice *lat, const int64_t *A, int64_t nA, const int64_t *B, int64_t nB,
                                int64_t M, const csp_options *opt, int64_t log_capacity, csp_result *res,
                                int64_t *path, int64_t cap, int64_t *len);

/* ------------------------------------------------------------------ serving
 *
 * A resident lattice answering a stream of queries with continuous batching: one
 * persistent kernel stays on the GPU; its CTAs form fixed groups, each owning one query
 * slot (its own labels, offers and flow pools).  A group claims the next submitted query
 * as soon as it is free, so queries that arrive while others run overlap on the device.
 * Queries travel through a ring in host-mapped memory; a query is admitted into the
 * ring while an entry is free (memory-based admission: slots are allocated up front from
 * the memory budget).  The paper solves one query at a time; this mode is an addition.
 */
typedef struct csp_server csp_server;

typedef struct {
    int32_t group_ctas;       /* CTAs per query slot; 0 = 16 */
    int32_t max_groups;       /* query slots; 0 = as many as fit on the GPU */
    int64_t pool_capacity;    /* flow slots per pool buffer per slot (whole chunks of 2048, up to two
                                 part-filled per CTA); 0 = max(2^16, V) capped by the flow bound, plus
                                 two chunks per CTA of the slot; a query that overflows it reports
                                 CSP_ERR_CAPACITY */
    int64_t memory_budget;    /* bytes for all slots together; 0 = no limit beyond max_groups */
    int64_t queue_capacity;   /* ring entries (queries submitted and not yet collected); 0 = 4 x slots */
    double session_seconds;   /* the persistent kernel gives up waiting after this long; 0 = 600 */
    int32_t wide_depth;       /* two modes (0 = 3): while fewer than wide_depth queries wait, the whole grid
                                 answers one query at a time (the latency of a plain solve without its
                                 launch); from wide_depth waiting queries on, the groups serve them in
                                 parallel (continuous batching) until every group is idle again.  -1 = groups
                                 only.  The wide mode has a workspace of its own, sized for the whole grid */
    int32_t reserved;         /* 0 */
} csp_server_options;

/* One query: 1..64 sources; targets either an explicit list (B, 1..64 ids) or, with
 * B = NULL, the hyperplane {v : c_{b_axis}(v) = b_coord}. */
typedef struct {
    const int64_t *A;
    int64_t nA;
    const int64_t *B;
    int64_t nB;
    int32_t b_axis;
    int32_t reserved;
    int64_t b_coord;
    int64_t M;
    int64_t max_cycles;       /* 0 = no limit */
} csp_server_query;

/* Allocates the slots and launches the persistent server kernel on its own stream.  The
 * lattice (or graph) must outlive the server; while the server runs it occupies the GPU. */
csp_status csp_server_create(csp_lattice *lat, const csp_server_options *opt, csp_server **out);

/* The server's slots (groups), CTAs per slot and ring size. */
csp_status csp_server_info(const csp_server *s, int32_t *groups, int32_t *group_ctas, int64_t *queue_capacity);

/* Submits a query without waiting; *ticket identifies it.  CSP_ERR_CAPACITY: no ring
 * entry is free (collect results first).  CSP_ERR_INVALID: bad query. */
csp_status csp_server_submit(csp_server *s, const csp_server_query *q, int64_t *ticket);

/* Non-blocking: *done = 1 once the query's result is available (then copied to out and
 * status, both nullable).  A result must be collected before queue_capacity further
 * submissions reuse its ring entry (CSP_ERR_INVALID if it was overwritten). */
csp_status csp_server_poll(csp_server *s, int64_t ticket, csp_result *out, int32_t *status, int32_t *done);

/* Replays a stream: query i arrives arrival_s[i] seconds after the call starts (sorted),
 * is submitted once a ring entry is free and collected when done.  latency_s[i] =
 * completion - arrival; every output is nullable. */
csp_status csp_server_replay(csp_server *s, const csp_server_query *q, const double *arrival_s, int64_t n,
                             csp_result *out, int32_t *status, double *latency_s, double *makespan_s);

/* How the server's queries were answered so far: by the whole grid (wide) or by a group
 * (narrow), and how often it switched between the two modes.  Nullable outputs. */
csp_status csp_server_stats(const csp_server *s, int64_t *wide_queries, int64_t *narrow_queries, int64_t *to_wide,
                            int64_t *to_narrow);

/* Stops the server (after the queries already submitted) and frees it. */
csp_status csp_server_destroy(csp_server *s);

/* Baseline for serving benchmarks: the same stream answered one query at a time with
 * csp_solve (one launch per query, in arrival order).  Same outputs as csp_server_replay. */
csp_status csp_serve_plain_replay(csp_lattice *lat, const csp_server_query *q, const double *arrival_s, int64_t n,
                                  csp_result *out, int32_t *status, double *latency_s, double *makespan_s);

/* The form (CSP_OPT_SWEEP or CSP_OPT_EVENT) a solve on this handle runs when its options
 * name neither; -1 for a NULL handle.  May prepare the event form (synchronous, once per
 * weight upload) to find out whether the handle supports it. */
int32_t csp_default_engine(csp_lattice *lat);

/* Device time of the last event-form solve on this handle, as measured by its first CTA:
 * ns[0] = 0 (reserved), ns[1] = phase A (arrivals), ns[2] = phase B (winners: commits,
 * launches, removals), ns[3] = waiting at grid barriers and reading counters.  For profiling.
 * CSP_ERR_INVALID if no event-form solve has run on it. */
csp_status csp_event_phase_times(const csp_lattice *lat, int64_t *ns);

/* Copies the labels left by the last solve (V int32: M - F2 of the best water that has
 * reached each vertex by the final time, 0 if none) to labels_host. */
csp_status csp_get_labels(csp_lattice *lat, int32_t *labels_host);

#ifdef __cplusplus
}
#endif

#endif /* CSP_H */
