/*
 * CPU oracle for the constrained shortest path method of I. Matic,
 * "A parallel algorithm for the constrained shortest path problem on lattice
 * graphs" (arXiv 1511.06441).
 *
 * TEST INFRASTRUCTURE.  Only the tests, the smoke check and the benchmark's CPU
 * baseline use this file.  The product path (the CUDA library) never links, loads
 * or calls it, and this file includes nothing from the product.
 *
 * Plain, slow, single-threaded and written for readability: int64 everywhere, no
 * blocking, no fusion.  Two independent solvers:
 *
 *   oracle_cycle     (O1) the paper's cycle loop (Algorithm 1; Steps 1-9), state =
 *                    vertex labels + a multiset of water flows, one loop iteration
 *                    per cycle; also returns the per-cycle trace, the final labels
 *                    and, on request, the active set at a given time.
 *   oracle_pareto    (O2) a label-setting Dijkstra over (vertex, quality) states with
 *                    dominance pruning; it knows nothing about cycles or flows.
 *   oracle_calendar  (O4) O1's loop driven by events (per-edge flow queues, arrival-time
 *                    buckets): a cross-check of O1 and of that reorganisation, with event
 *                    counts.
 *   oracle_lexmin    lexicographic (F1, F2) Dijkstra without a weight bound: derives the
 *                    weight bound M of the anti-correlated workload and, where that
 *                    bound does not bind, the whole answer (F1, F2, X, x).
 *
 * Lattice: box [0,n_0) x ... x [0,n_{d-1}), vertex id v = sum c_k stride_k with c_0
 * fastest.  f1[k*V+v], f2[k*V+v] are travel time and weight of the edge (v, v+e_k);
 * they are read only where c_k + 1 < n_k, and f1 <= 0 means the edge is absent.
 * Direction dir = 2k + s leads from v to v + e_k (s = 0) or v - e_k (s = 1).
 *
 * Graph (oracle_cycle_graph, oracle_pareto_graph; Section 1 states the method for any
 * graph): V vertices with S adjacency slots each; slot j of v holds the neighbour
 * nbr[v*S+j] (-1: empty) and the edge's f1[v*S+j] >= 1, f2[v*S+j].  The direction of an
 * edge is its slot at the vertex it leaves.
 *
 * Readings of the paper adopted here (where it is silent or inconsistent):
 *   - the bound is strict, F2 < M (Section 1), matching "quality 0 cannot travel";
 *   - labels only increase: an arrival of better water raises the label of an active
 *     vertex too, and the better water travels on new flows (the paper's phantoms);
 *   - time jumps by m, the smallest remaining time (Step 1); one cycle = one jump;
 *   - after each cycle every flow whose arrival quality Q - f2 no longer exceeds the
 *     current label of its destination is removed (the worked example of Section 3,
 *     flows into vertex 5 at second 6), and a vertex is active iff it is the source of
 *     at least one flow;
 *   - initialisation applies the launch rule to the edges of A (no flow into A, no flow
 *     that would arrive with quality <= 0);
 *   - termination (Algorithm 2): the first cycle in which a vertex of B improves gives
 *     F1 = Time; that cycle still finishes its launches and removals; no flow left means
 *     infeasible (F1 = -1);
 *   - X = among the B vertices improved in the last cycle, the largest label, then the
 *     smallest id; x = the arriving edge (Y -> X) with the largest arrival quality, then
 *     the smallest (Y, direction); F2 = M - Label(X) (Termination 1 of the paper).
 *
 * Pins (tests): brute-force path enumeration on tiny lattices (F1, F2, X, x and the
 * whole trace via per-vertex Pareto frontiers), plain Dijkstra when f2 = 0 (F1 and the
 * trace), closed forms for uniform weights and for a path graph, monotonicity in M,
 * and the active set on the lattice of the paper's Lemma (Section "Large sets of
 * active vertices").
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

enum { OR_OK = 0, OR_INVALID = 1, OR_OOM = 2, OR_TIMEOUT = 5 };

typedef struct {
    int d;
    int slots;                    /* directions per vertex: 2d on a lattice, S on a graph */
    int64_t ext[4], stride[4], V;
    const int32_t *f1, *f2;
    const int64_t *nbr;           /* graph only: nbr[v * S + j] = neighbour in slot j, or -1 */
    const unsigned char *removed; /* nullable: vertices not in the graph (V' of Section 1) */
} lattice_t;

static int lattice_init(lattice_t *L, int d, const int64_t *ext, const int32_t *f1, const int32_t *f2)
{
    if (d < 1 || d > 4) return OR_INVALID;
    L->d = d;
    L->V = 1;
    for (int k = 0; k < d; k++) {
        if (ext[k] < 1) return OR_INVALID;
        L->ext[k] = ext[k];
        L->stride[k] = L->V;
        L->V *= ext[k];
    }
    L->slots = 2 * d;
    L->f1 = f1;
    L->f2 = f2;
    L->nbr = NULL;
    L->removed = NULL;
    return OR_OK;
}

/* A general graph (Section 1 allows any graph; the lattice is the bounded-degree case
 * the paper implements): vertex v has S slots, slot j holding the neighbour nbr[v*S+j]
 * (-1: empty) and the edge's f1[v*S+j] >= 1 and f2[v*S+j].  An undirected edge appears
 * in a slot of each end; the oracle itself also accepts one-way edges. */
static int graph_init(lattice_t *L, int64_t V, int S, const int64_t *nbr, const int32_t *f1, const int32_t *f2)
{
    if (V < 1 || S < 1) return OR_INVALID;
    for (int64_t i = 0; i < V * S; i++)
        if (nbr[i] < -1 || nbr[i] >= V || (nbr[i] >= 0 && f1[i] < 1)) return OR_INVALID;
    L->d = 0;
    L->slots = S;
    L->V = V;
    L->f1 = f1;
    L->f2 = f2;
    L->nbr = nbr;
    L->removed = NULL;
    return OR_OK;
}

/* The neighbour of v in direction dir, or -1 if that edge does not exist.
 * *time and *weight receive f1 and f2 of the edge. */
static int64_t neighbour(const lattice_t *L, int64_t v, int dir, int64_t *time, int64_t *weight)
{
    if (L->nbr) {
        const int64_t i = v * L->slots + dir, u = L->nbr[i];
        if (u < 0) return -1;
        if (L->removed && (L->removed[u] || L->removed[v])) return -1;
        *time = L->f1[i];
        *weight = L->f2[i];
        return u;
    }
    int k = dir / 2, s = dir % 2;
    int64_t ck = (v / L->stride[k]) % L->ext[k];
    int64_t u, slot;
    if (s == 0) {
        if (ck + 1 >= L->ext[k]) return -1;
        u = v + L->stride[k];
        slot = (int64_t)k * L->V + v;
    } else {
        if (ck == 0) return -1;
        u = v - L->stride[k];
        slot = (int64_t)k * L->V + u;
    }
    if (L->f1[slot] <= 0) return -1;
    if (L->removed && (L->removed[u] || L->removed[v])) return -1;
    *time = L->f1[slot];
    *weight = L->f2[slot];
    return u;
}

/* Marks the members of S in flag (1 byte per vertex); INVALID on out-of-range ids. */
static int mark_set(const lattice_t *L, const int64_t *S, int64_t n, unsigned char *flag)
{
    for (int64_t i = 0; i < n; i++) {
        if (S[i] < 0 || S[i] >= L->V) return OR_INVALID;
        flag[S[i]] = 1;
    }
    return OR_OK;
}

static int validate_sets(const lattice_t *L, const int64_t *A, int64_t nA, const int64_t *B, int64_t nB,
                         unsigned char *inA, unsigned char *inB)
{
    if (nA < 1 || nB < 1) return OR_INVALID;
    if (mark_set(L, A, nA, inA) || mark_set(L, B, nB, inB)) return OR_INVALID;
    for (int64_t i = 0; i < nB; i++)
        if (inA[B[i]]) return OR_INVALID; /* A and B must be disjoint (Section 1) */
    return OR_OK;
}

/* ------------------------------------------------------------------ O1 */

typedef struct {
    int64_t src;   /* Source(e): the vertex the water left */
    int dir;       /* direction from src to dst */
    int64_t dst;
    int64_t Q;     /* quality of the water = Label(src) when the flow started */
    int64_t f2;    /* weight of the edge: quality lost on the way */
    int64_t r;     /* TimeRemaining(e) */
} flow_t;

typedef struct {
    flow_t *a;
    int64_t n, cap;
} flows_t;

static int flows_push(flows_t *F, flow_t f)
{
    if (F->n == F->cap) {
        int64_t nc = F->cap ? 2 * F->cap : 1024;
        flow_t *na = (flow_t *)realloc(F->a, (size_t)nc * sizeof(flow_t));
        if (!na) return OR_OOM;
        F->a = na;
        F->cap = nc;
    }
    F->a[F->n++] = f;
    return OR_OK;
}

/* Start a flow on every edge (v, u) along which water of quality Label(v) would still
 * raise Label(u): Label(v) - f2 > Label(u) (Step 4, TriggerEdges; Step 5 creates the
 * flow, a phantom if the edge already carries water).  on_edge[v * slots + dir] counts the
 * flows on each directed edge; a flow started while it is positive is a phantom. */
static int launch_from(const lattice_t *L, const int64_t *label, int64_t v, flows_t *F, int64_t *launched,
                       int64_t *on_edge, int64_t *phantoms)
{
    for (int dir = 0; dir < L->slots; dir++) {
        int64_t t, w;
        int64_t u = neighbour(L, v, dir, &t, &w);
        if (u < 0) continue;
        if (label[v] - w > label[u]) {
            flow_t f = {v, dir, u, label[v], w, t};
            if (flows_push(F, f)) return OR_OOM;
            (*launched)++;
            int64_t *c = &on_edge[v * L->slots + dir];
            if (*c > 0) (*phantoms)++;
            (*c)++;
        }
    }
    return OR_OK;
}

/* Steps 7-9: drop every flow that can no longer improve its destination. */
static void prune(flows_t *F, const int64_t *label, int64_t *on_edge, int twod)
{
    int64_t j = 0;
    for (int64_t i = 0; i < F->n; i++) {
        if (F->a[i].Q - F->a[i].f2 > label[F->a[i].dst]) F->a[j++] = F->a[i];
        else on_edge[F->a[i].src * twod + F->a[i].dir]--;
    }
    F->n = j;
}

/* Active vertices = distinct sources of the remaining flows; optionally listed. */
static int64_t count_active(const flows_t *F, int64_t *stamp, int64_t tag, int64_t *list)
{
    int64_t n = 0;
    for (int64_t i = 0; i < F->n; i++) {
        int64_t s = F->a[i].src;
        if (stamp[s] != tag) {
            stamp[s] = tag;
            if (list) list[n] = s;
            n++;
        }
    }
    return n;
}

static int cmp_i64(const void *x, const void *y)
{
    int64_t a = *(const int64_t *)x, b = *(const int64_t *)y;
    return (a > b) - (a < b);
}

/*
 * O1.  res[0..8] = F1, X, x_src, x_dir, F2, cycles, updates, flows_launched, phantoms,
 * where updates = sum over cycles of the flows alive when the cycle starts and phantoms
 * = flows started on a directed edge that already carried a flow (after the arrivals of
 * the cycle, before its removals: the paper's phantom edges, Step 5).  trace receives
 * rows (Time, active vertices, flows) after the removals of each cycle, row 0 being the
 * state after initialisation; *trace_len is the number of rows produced (it may exceed
 * trace_cap, then only trace_cap rows are written).  If snap is not NULL it receives the
 * active vertices (ascending) at the end of the last cycle whose Time <= snap_time.
 * labels_out (nullable, V entries) receives the labels at termination.  removed
 * (nullable, V bytes) lists vertices that are not part of the graph; A and B must avoid them.
 */
static int cycle_core(lattice_t L, const int64_t *A, int64_t nA, const int64_t *B, int64_t nB, int64_t M,
                      int64_t max_cycles, int64_t *res,
                      int64_t *trace, int64_t trace_cap, int64_t *trace_len,
                      int64_t snap_time, int64_t *snap, int64_t *snap_len, int64_t *labels_out,
                      const unsigned char *removed)
{
    int rc = OR_OK;
    L.removed = removed;
    const int64_t V = L.V;
    unsigned char *inA = calloc((size_t)V, 1), *inB = calloc((size_t)V, 1);
    int64_t *label = calloc((size_t)V, sizeof(int64_t));
    int64_t *stamp = malloc((size_t)V * sizeof(int64_t));
    int64_t *bq = malloc((size_t)V * sizeof(int64_t));   /* best offered quality this cycle */
    int64_t *bsrc = malloc((size_t)V * sizeof(int64_t)), *bdir = malloc((size_t)V * sizeof(int64_t));
    int64_t *touched = malloc((size_t)V * sizeof(int64_t));
    int64_t *improved = malloc((size_t)V * sizeof(int64_t));
    int64_t *xsrc = malloc((size_t)V * sizeof(int64_t)), *xdir = malloc((size_t)V * sizeof(int64_t));
    int64_t *on_edge = calloc((size_t)V * L.slots, sizeof(int64_t));
    flows_t F = {0, 0, 0};
    int64_t rows = 0, Time = 0, cycles = 0, updates = 0, launched = 0, phantoms = 0;
    if (!inA || !inB || !label || !stamp || !bq || !bsrc || !bdir || !touched || !improved || !xsrc || !xdir ||
        !on_edge) {
        rc = OR_OOM;
        goto done;
    }
    rc = validate_sets(&L, A, nA, B, nB, inA, inB);
    if (rc) goto done;
    if (removed)
        for (int64_t v = 0; v < V; v++)
            if (removed[v] && (inA[v] || inB[v])) {
                rc = OR_INVALID;
                goto done;
            }
    for (int64_t v = 0; v < V; v++) {
        stamp[v] = -1;
        bq[v] = INT64_MIN;
    }
    for (int i = 0; i < 9; i++) res[i] = -1;
    if (snap_len) *snap_len = 0;

    /* Initialization (Algorithm 3): Label = M on A, 0 elsewhere; water leaves A. */
    for (int64_t v = 0; v < V; v++)
        if (inA[v]) label[v] = M;
    for (int64_t v = 0; v < V; v++)
        if (inA[v] && (rc = launch_from(&L, label, v, &F, &launched, on_edge, &phantoms))) goto done;
    prune(&F, label, on_edge, L.slots);
    {
        int64_t act = count_active(&F, stamp, 0, NULL);
        if (rows < trace_cap) {
            trace[3 * rows] = 0;
            trace[3 * rows + 1] = act;
            trace[3 * rows + 2] = F.n;
        }
        rows++;
        if (snap && snap_time >= 0) *snap_len = count_active(&F, stamp, -2, snap);
    }

    while (F.n > 0) {
        if (cycles >= max_cycles) {
            rc = OR_TIMEOUT; /* res[5], res[6] still report the work done so far */
            break;
        }
        cycles++;
        updates += F.n;
        /* Step 1: m = smallest remaining time; every flow advances by m. */
        int64_t m = INT64_MAX;
        for (int64_t i = 0; i < F.n; i++)
            if (F.a[i].r < m) m = F.a[i].r;
        Time += m;
        /* Steps 1-3: flows that reach 0 deliver water of quality Q - f2 to their
         * destination; the best offer per destination is kept (largest quality, then
         * smallest source, then smallest direction).  Arrived flows leave the pool. */
        int64_t nt = 0, j = 0;
        for (int64_t i = 0; i < F.n; i++) {
            flow_t *f = &F.a[i];
            f->r -= m;
            if (f->r > 0) {
                F.a[j++] = *f;
                continue;
            }
            on_edge[f->src * L.slots + f->dir]--;  /* arrived: off the edge */
            int64_t q = f->Q - f->f2, u = f->dst;
            if (bq[u] == INT64_MIN) touched[nt++] = u;
            if (q > bq[u] || (q == bq[u] && (f->src < bsrc[u] || (f->src == bsrc[u] && f->dir < bdir[u])))) {
                bq[u] = q;
                bsrc[u] = f->src;
                bdir[u] = f->dir;
            }
        }
        F.n = j;
        /* Steps 2 and 8: a destination whose best offer beats its label takes it. */
        int64_t ni = 0;
        for (int64_t i = 0; i < nt; i++) {
            int64_t u = touched[i];
            if (bq[u] > label[u]) {
                label[u] = bq[u];
                xsrc[u] = bsrc[u];
                xdir[u] = bdir[u];
                improved[ni++] = u;
            }
            bq[u] = INT64_MIN;
        }
        qsort(improved, (size_t)ni, sizeof(int64_t), cmp_i64);
        /* Steps 4-5: water leaves every improved vertex (labels of this cycle). */
        for (int64_t i = 0; i < ni; i++)
            if ((rc = launch_from(&L, label, improved[i], &F, &launched, on_edge, &phantoms))) goto done;
        /* Steps 7-9. */
        prune(&F, label, on_edge, L.slots);
        int64_t act = count_active(&F, stamp, cycles, NULL);
        if (rows < trace_cap) {
            trace[3 * rows] = Time;
            trace[3 * rows + 1] = act;
            trace[3 * rows + 2] = F.n;
        }
        rows++;
        if (snap && Time <= snap_time) *snap_len = count_active(&F, stamp, -2 - cycles, snap);
        /* Step 6 / Algorithm 2. */
        int64_t X = -1;
        for (int64_t i = 0; i < ni; i++) {
            int64_t u = improved[i];
            if (inB[u] && (X < 0 || label[u] > label[X] || (label[u] == label[X] && u < X))) X = u;
        }
        if (X >= 0) {
            res[0] = Time;
            res[1] = X;
            res[2] = xsrc[X];
            res[3] = xdir[X];
            res[4] = M - label[X];
            break;
        }
    }
    res[5] = cycles;
    res[6] = updates;
    res[7] = launched;
    res[8] = phantoms;
    if (rc) goto done;
    if (snap && snap_len && *snap_len > 0) qsort(snap, (size_t)*snap_len, sizeof(int64_t), cmp_i64);
    if (labels_out) memcpy(labels_out, label, (size_t)V * sizeof(int64_t));
done:
    *trace_len = rows;
    free(inA); free(inB); free(label); free(stamp); free(bq); free(bsrc); free(bdir);
    free(touched); free(improved); free(xsrc); free(xdir); free(F.a); free(on_edge);
    return rc;
}

int oracle_cycle(int d, const int64_t *ext, const int32_t *f1, const int32_t *f2,
                 const int64_t *A, int64_t nA, const int64_t *B, int64_t nB, int64_t M,
                 int64_t max_cycles, int64_t *res,
                 int64_t *trace, int64_t trace_cap, int64_t *trace_len,
                 int64_t snap_time, int64_t *snap, int64_t *snap_len, int64_t *labels_out,
                 const unsigned char *removed)
{
    lattice_t L;
    int rc = lattice_init(&L, d, ext, f1, f2);
    if (rc) return rc;
    return cycle_core(L, A, nA, B, nB, M, max_cycles, res, trace, trace_cap, trace_len, snap_time, snap, snap_len, labels_out, removed);
}

/* O1 on a general graph (see graph_init); the same outputs, x_dir being the slot of x in
 * the adjacency of x_src. */
int oracle_cycle_graph(int64_t V, int S, const int64_t *nbr, const int32_t *f1, const int32_t *f2,
                       const int64_t *A, int64_t nA, const int64_t *B, int64_t nB, int64_t M,
                       int64_t max_cycles, int64_t *res,
                       int64_t *trace, int64_t trace_cap, int64_t *trace_len,
                       int64_t snap_time, int64_t *snap, int64_t *snap_len, int64_t *labels_out,
                       const unsigned char *removed)
{
    lattice_t L;
    int rc = graph_init(&L, V, S, nbr, f1, f2);
    if (rc) return rc;
    return cycle_core(L, A, nA, B, nB, M, max_cycles, res, trace, trace_cap, trace_len, snap_time, snap, snap_len, labels_out, removed);
}

/* ------------------------------------------------------------------ O4: event-driven form */

/*
 * O4.  The same cycle loop as O1, reorganised around events instead of a sweep over every
 * flow, to check that the reorganisation is exact (it is the calendar-queue design for the
 * GPU): the flows in flight on one directed edge form a queue in launch order, and since a
 * vertex's label only rises their qualities rise too, so both arrivals (oldest first) and
 * removals (lowest quality first) take from the front.  Flows are also listed under their
 * arrival time (one bucket per time modulo max f1 + 1, with a count of the listed flows
 * still alive), so the next cycle time is the first bucket with a live flow, and a cycle
 * touches only its arrivals, the flows it launches and the front of the queues into the
 * vertices it improves.  Outputs as O1 (res[0..8], trace, labels); res[9..13] count the
 * events: arrivals taken from buckets, bucket entries found stale (removed earlier), flows
 * pushed, removals, and queue fronts inspected by the removal step.
 */
typedef struct {
    int32_t t0; /* launch time */
    int32_t Q;  /* quality = Label(src) at launch */
} qflow_t;

typedef struct {
    int64_t *a;
    int64_t n, cap;
} ivec_t;

static int ivec_push(ivec_t *b, int64_t x)
{
    if (b->n == b->cap) {
        int64_t nc = b->cap ? 2 * b->cap : 16;
        int64_t *na = (int64_t *)realloc(b->a, (size_t)nc * sizeof(int64_t));
        if (!na) return OR_OOM;
        b->a = na;
        b->cap = nc;
    }
    b->a[b->n++] = x;
    return OR_OK;
}

static int calendar_core(lattice_t L, const int64_t *A, int64_t nA, const int64_t *B, int64_t nB, int64_t M,
                         int64_t max_cycles, int64_t *res, int64_t *trace, int64_t trace_cap, int64_t *trace_len,
                         int64_t *labels_out)
{
    const int64_t V = L.V, S = L.slots, E = V * S;
    int rc = OR_OK;
    unsigned char *inA = calloc((size_t)V, 1), *inB = calloc((size_t)V, 1);
    int64_t *label = calloc((size_t)V, sizeof(int64_t));
    int64_t *head = calloc((size_t)E, sizeof(int64_t)), *cnt = calloc((size_t)E, sizeof(int64_t));
    int64_t *et = calloc((size_t)E, sizeof(int64_t)), *ew = calloc((size_t)E, sizeof(int64_t));
    int64_t *edst = malloc((size_t)E * sizeof(int64_t)), *qoff = malloc((size_t)(E + 1) * sizeof(int64_t));
    int64_t *in_off = calloc((size_t)(V + 1), sizeof(int64_t)), *in_e = NULL;
    int64_t *out_count = calloc((size_t)V, sizeof(int64_t));
    int64_t *bq = malloc((size_t)V * sizeof(int64_t)), *bsrc = malloc((size_t)V * sizeof(int64_t));
    int64_t *bdir = malloc((size_t)V * sizeof(int64_t)), *touched = malloc((size_t)V * sizeof(int64_t));
    int64_t *improved = malloc((size_t)V * sizeof(int64_t));
    int64_t *xsrc = malloc((size_t)V * sizeof(int64_t)), *xdir = malloc((size_t)V * sizeof(int64_t));
    qflow_t *qs = NULL;
    ivec_t *bucket = NULL;
    int64_t *blive = NULL;
    int64_t W = 2, rows = 0, Time = 0, cycles = 0, updates = 0, launched = 0, phantoms = 0, live = 0, active = 0;
    int64_t n_arr = 0, n_stale = 0, n_push = 0, n_rem = 0, n_front = 0;
    for (int i = 0; i < 14; i++) res[i] = -1;
    if (!inA || !inB || !label || !head || !cnt || !et || !ew || !edst || !qoff || !in_off || !out_count || !bq ||
        !bsrc || !bdir || !touched || !improved || !xsrc || !xdir) {
        rc = OR_OOM;
        goto done;
    }
    rc = validate_sets(&L, A, nA, B, nB, inA, inB);
    if (rc) goto done;
    /* directed edges e = v * S + dir: destination, f1, f2, queue storage (f1 slots: one
     * launch per cycle, each in flight for f1 time units), and the edges into each vertex */
    qoff[0] = 0;
    for (int64_t v = 0; v < V; v++)
        for (int dir = 0; dir < S; dir++) {
            const int64_t e = v * S + dir;
            int64_t t = 0, w = 0, u = neighbour(&L, v, dir, &t, &w);
            edst[e] = u;
            et[e] = u >= 0 ? t : 0;
            ew[e] = w;
            qoff[e + 1] = qoff[e] + et[e];
            if (u >= 0) in_off[u + 1]++;
            if (et[e] + 1 > W) W = et[e] + 1;
        }
    for (int64_t v = 0; v < V; v++) in_off[v + 1] += in_off[v];
    in_e = malloc((size_t)(in_off[V] + 1) * sizeof(int64_t));
    qs = malloc((size_t)(qoff[E] + 1) * sizeof(qflow_t));
    bucket = calloc((size_t)W, sizeof(ivec_t));
    blive = calloc((size_t)W, sizeof(int64_t));
    if (!in_e || !qs || !bucket || !blive) {
        rc = OR_OOM;
        goto done;
    }
    {
        int64_t *fillp = touched; /* scratch: next free position per vertex */
        for (int64_t v = 0; v < V; v++) fillp[v] = in_off[v];
        for (int64_t e = 0; e < E; e++)
            if (edst[e] >= 0) in_e[fillp[edst[e]]++] = e;
    }
    for (int64_t v = 0; v < V; v++) bq[v] = INT64_MIN;

/* push a flow on edge e at time T with quality Q (the queue holds at most f1(e) flows) */
#define CAL_PUSH(e, T, Q)                                                            \
    do {                                                                             \
        const int64_t e_ = (e);                                                      \
        if (cnt[e_] > 0) phantoms++;                                                 \
        qs[qoff[e_] + (head[e_] + cnt[e_]) % et[e_]] = (qflow_t){(int32_t)(T), (int32_t)(Q)}; \
        cnt[e_]++;                                                                   \
        const int64_t b_ = ((T) + et[e_]) % W;                                       \
        if ((rc = ivec_push(&bucket[b_], e_))) goto done;                            \
        blive[b_]++;                                                                 \
        if (out_count[e_ / S]++ == 0) active++;                                      \
        live++;                                                                      \
        launched++;                                                                  \
        n_push++;                                                                    \
    } while (0)
/* take the front flow of edge e off the edge (arrived or removed) */
#define CAL_POP(e)                                                                   \
    do {                                                                             \
        const int64_t e_ = (e);                                                      \
        const qflow_t f_ = qs[qoff[e_] + head[e_]];                                  \
        blive[((int64_t)f_.t0 + et[e_]) % W]--;                                      \
        head[e_] = (head[e_] + 1) % et[e_];                                          \
        cnt[e_]--;                                                                   \
        if (--out_count[e_ / S] == 0) active--;                                      \
        live--;                                                                      \
    } while (0)

    /* Initialization (Algorithm 3) */
    for (int64_t v = 0; v < V; v++)
        if (inA[v]) label[v] = M;
    for (int64_t v = 0; v < V; v++)
        if (inA[v])
            for (int dir = 0; dir < S; dir++) {
                const int64_t e = v * S + dir, u = edst[e];
                if (u >= 0 && label[v] - ew[e] > label[u]) CAL_PUSH(e, 0, label[v]);
            }
    if (rows < trace_cap) {
        trace[0] = 0;
        trace[1] = active;
        trace[2] = live;
    }
    rows++;

    while (live > 0) {
        if (cycles >= max_cycles) {
            rc = OR_TIMEOUT;
            break;
        }
        /* the next time with a live arrival */
        int64_t T = Time + 1;
        while (blive[T % W] == 0) T++;
        cycles++;
        updates += live;
        Time = T;
        /* arrivals: the front flow of each listed edge, if it is the one due now */
        ivec_t *bk = &bucket[T % W];
        int64_t nt = 0;
        for (int64_t i = 0; i < bk->n; i++) {
            const int64_t e = bk->a[i];
            if (cnt[e] == 0 || (int64_t)qs[qoff[e] + head[e]].t0 + et[e] != T) {
                n_stale++; /* removed before it arrived */
                continue;
            }
            const int64_t Q = qs[qoff[e] + head[e]].Q, u = edst[e], src = e / S, dir = e % S;
            CAL_POP(e);
            n_arr++;
            const int64_t q = Q - ew[e];
            if (bq[u] == INT64_MIN) touched[nt++] = u;
            if (q > bq[u] || (q == bq[u] && (src < bsrc[u] || (src == bsrc[u] && dir < bdir[u])))) {
                bq[u] = q;
                bsrc[u] = src;
                bdir[u] = dir;
            }
        }
        bk->n = 0;
        /* commit (Steps 2, 8) */
        int64_t ni = 0;
        for (int64_t i = 0; i < nt; i++) {
            const int64_t u = touched[i];
            if (bq[u] > label[u]) {
                label[u] = bq[u];
                xsrc[u] = bsrc[u];
                xdir[u] = bdir[u];
                improved[ni++] = u;
            }
            bq[u] = INT64_MIN;
        }
        qsort(improved, (size_t)ni, sizeof(int64_t), cmp_i64);
        /* launch (Steps 4-5) under the labels at the end of the cycle */
        for (int64_t i = 0; i < ni; i++) {
            const int64_t v = improved[i];
            for (int dir = 0; dir < S; dir++) {
                const int64_t e = v * S + dir, u = edst[e];
                if (u >= 0 && label[v] - ew[e] > label[u]) CAL_PUSH(e, T, label[v]);
            }
        }
        /* removals (Steps 7-9): only a vertex whose label rose can make flows into it
         * useless, and on each edge into it the useless flows are a prefix of the queue */
        for (int64_t i = 0; i < ni; i++) {
            const int64_t v = improved[i];
            for (int64_t k = in_off[v]; k < in_off[v + 1]; k++) {
                const int64_t e = in_e[k];
                n_front++;
                while (cnt[e] > 0 && (int64_t)qs[qoff[e] + head[e]].Q - ew[e] <= label[v]) {
                    CAL_POP(e);
                    n_rem++;
                }
            }
        }
        if (rows < trace_cap) {
            trace[3 * rows] = Time;
            trace[3 * rows + 1] = active;
            trace[3 * rows + 2] = live;
        }
        rows++;
        int64_t X = -1;
        for (int64_t i = 0; i < ni; i++) {
            const int64_t u = improved[i];
            if (inB[u] && (X < 0 || label[u] > label[X] || (label[u] == label[X] && u < X))) X = u;
        }
        if (X >= 0) {
            res[0] = Time;
            res[1] = X;
            res[2] = xsrc[X];
            res[3] = xdir[X];
            res[4] = M - label[X];
            break;
        }
    }
#undef CAL_PUSH
#undef CAL_POP
    res[5] = cycles;
    res[6] = updates;
    res[7] = launched;
    res[8] = phantoms;
    res[9] = n_arr;
    res[10] = n_stale;
    res[11] = n_push;
    res[12] = n_rem;
    res[13] = n_front;
    if (!rc && labels_out) memcpy(labels_out, label, (size_t)V * sizeof(int64_t));
done:
    *trace_len = rows;
    if (bucket)
        for (int64_t b = 0; b < W; b++) free(bucket[b].a);
    free(bucket); free(blive); free(qs); free(in_e);
    free(inA); free(inB); free(label); free(head); free(cnt); free(et); free(ew); free(edst); free(qoff);
    free(in_off); free(out_count); free(bq); free(bsrc); free(bdir); free(touched); free(improved);
    free(xsrc); free(xdir);
    return rc;
}

int oracle_calendar(int d, const int64_t *ext, const int32_t *f1, const int32_t *f2, const int64_t *A, int64_t nA,
                    const int64_t *B, int64_t nB, int64_t M, int64_t max_cycles, int64_t *res, int64_t *trace,
                    int64_t trace_cap, int64_t *trace_len, int64_t *labels_out)
{
    lattice_t L;
    int rc = lattice_init(&L, d, ext, f1, f2);
    if (rc) return rc;
    return calendar_core(L, A, nA, B, nB, M, max_cycles, res, trace, trace_cap, trace_len, labels_out);
}

int oracle_calendar_graph(int64_t V, int S, const int64_t *nbr, const int32_t *f1, const int32_t *f2,
                          const int64_t *A, int64_t nA, const int64_t *B, int64_t nB, int64_t M, int64_t max_cycles,
                          int64_t *res, int64_t *trace, int64_t trace_cap, int64_t *trace_len, int64_t *labels_out)
{
    lattice_t L;
    int rc = graph_init(&L, V, S, nbr, f1, f2);
    if (rc) return rc;
    return calendar_core(L, A, nA, B, nB, M, max_cycles, res, trace, trace_cap, trace_len, labels_out);
}

/* ------------------------------------------------------------------ O2 */

typedef struct {
    int64_t t;    /* arrival time = F1 of the walk */
    int64_t q;    /* remaining quality = M - F2 of the walk */
    int64_t v, src, dir;
} state_t;

/* heap order: earlier time, then higher quality, then smaller v, src, dir */
static int state_before(const state_t *a, const state_t *b)
{
    if (a->t != b->t) return a->t < b->t;
    if (a->q != b->q) return a->q > b->q;
    if (a->v != b->v) return a->v < b->v;
    if (a->src != b->src) return a->src < b->src;
    return a->dir < b->dir;
}

typedef struct {
    state_t *a;
    int64_t n, cap;
} heap_t;

static int heap_push(heap_t *H, state_t s)
{
    if (H->n == H->cap) {
        int64_t nc = H->cap ? 2 * H->cap : 1024;
        state_t *na = (state_t *)realloc(H->a, (size_t)nc * sizeof(state_t));
        if (!na) return OR_OOM;
        H->a = na;
        H->cap = nc;
    }
    int64_t i = H->n++;
    while (i > 0) {
        int64_t p = (i - 1) / 2;
        if (!state_before(&s, &H->a[p])) break;
        H->a[i] = H->a[p];
        i = p;
    }
    H->a[i] = s;
    return OR_OK;
}

static state_t heap_pop(heap_t *H)
{
    state_t top = H->a[0], last = H->a[--H->n];
    int64_t i = 0;
    for (;;) {
        int64_t c = 2 * i + 1;
        if (c >= H->n) break;
        if (c + 1 < H->n && state_before(&H->a[c + 1], &H->a[c])) c++;
        if (!state_before(&H->a[c], &last)) break;
        H->a[i] = H->a[c];
        i = c;
    }
    if (H->n > 0) H->a[i] = last;
    return top;
}

/*
 * O2.  Walks from A are explored in order of (arrival time, -quality).  A state
 * (v, t, q) is expanded only if q exceeds every quality already settled at v; any
 * later state with no better quality is dominated (it arrives no earlier and is no
 * lighter).  The first settled vertex of B gives F1, X, x and F2 = M - q.
 * res[0..7] = F1, X, x_src, x_dir, F2, -1, states_settled, states_pushed.
 */
static int pareto_core(lattice_t L, const int64_t *A, int64_t nA, const int64_t *B, int64_t nB, int64_t M,
                       int64_t *res)
{
    int rc = OR_OK;
    const int64_t V = L.V;
    unsigned char *inA = calloc((size_t)V, 1), *inB = calloc((size_t)V, 1);
    int64_t *best = calloc((size_t)V, sizeof(int64_t)); /* best settled quality, 0 = none */
    heap_t H = {0, 0, 0};
    int64_t settled = 0, pushed = 0;
    for (int i = 0; i < 8; i++) res[i] = -1;
    if (!inA || !inB || !best) {
        rc = OR_OOM;
        goto done;
    }
    rc = validate_sets(&L, A, nA, B, nB, inA, inB);
    if (rc) goto done;
    for (int64_t v = 0; v < V; v++)
        if (inA[v]) {
            state_t s = {0, M, v, -1, -1};
            if ((rc = heap_push(&H, s))) goto done;
            pushed++;
        }
    while (H.n > 0) {
        state_t s = heap_pop(&H);
        if (s.q <= best[s.v]) continue;
        best[s.v] = s.q;
        settled++;
        if (inB[s.v]) {
            res[0] = s.t;
            res[1] = s.v;
            res[2] = s.src;
            res[3] = s.dir;
            res[4] = M - s.q;
            break;
        }
        for (int dir = 0; dir < L.slots; dir++) {
            int64_t t, w;
            int64_t u = neighbour(&L, s.v, dir, &t, &w);
            if (u < 0 || s.q - w <= best[u]) continue;
            state_t n = {s.t + t, s.q - w, u, s.v, dir};
            if ((rc = heap_push(&H, n))) goto done;
            pushed++;
        }
    }
    res[6] = settled;
    res[7] = pushed;
done:
    free(inA); free(inB); free(best); free(H.a);
    return rc;
}

int oracle_pareto(int d, const int64_t *ext, const int32_t *f1, const int32_t *f2,
                  const int64_t *A, int64_t nA, const int64_t *B, int64_t nB, int64_t M, int64_t *res)
{
    lattice_t L;
    int rc = lattice_init(&L, d, ext, f1, f2);
    if (rc) return rc;
    return pareto_core(L, A, nA, B, nB, M, res);
}

/* O2 on a general graph (see graph_init). */
int oracle_pareto_graph(int64_t V, int S, const int64_t *nbr, const int32_t *f1, const int32_t *f2,
                        const int64_t *A, int64_t nA, const int64_t *B, int64_t nB, int64_t M, int64_t *res)
{
    lattice_t L;
    int rc = graph_init(&L, V, S, nbr, f1, f2);
    if (rc) return rc;
    return pareto_core(L, A, nA, B, nB, M, res);
}

/* ------------------------------------------------------------------ lexicographic Dijkstra */

/* Unconstrained lexicographic minimum of (F1, F2) over walks from A to B: a plain
 * Dijkstra on pairs.  res[0] = F1, res[1] = F2 (both -1 if B is unreachable). */
/*
 * Lexicographic Dijkstra: walks from A explored in order of (F1, F2), each vertex settled
 * by its first (lightest among the fastest) state.  res[0..4] = F1, F2, X, x_src, x_dir of
 * the first settled vertex of B; states of equal (F1, F2) pop by smaller vertex, then
 * smaller (predecessor, direction), so X and x follow the tie rules of the solver.  When
 * F2 < M, this is the solver's answer for the bound M: the fastest walks are allowed and
 * the lightest of them reaches X (Section 1, the problem statement).
 */
/* path (nullable, cap entries): the settled predecessors from X back to A, written A first;
 * *path_len = its length (> cap: not written). */
int oracle_lexmin(int d, const int64_t *ext, const int32_t *f1, const int32_t *f2,
                  const int64_t *A, int64_t nA, const int64_t *B, int64_t nB, int64_t *res,
                  int64_t *path, int64_t cap, int64_t *path_len)
{
    lattice_t L;
    int rc = lattice_init(&L, d, ext, f1, f2);
    if (rc) return rc;
    const int64_t V = L.V;
    unsigned char *inA = calloc((size_t)V, 1), *inB = calloc((size_t)V, 1), *done_v = calloc((size_t)V, 1);
    int64_t *pred = path_len ? malloc((size_t)V * sizeof(int64_t)) : NULL;
    heap_t H = {0, 0, 0};
    for (int i = 0; i < 5; i++) res[i] = -1;
    if (path_len) *path_len = 0;
    if (!inA || !inB || !done_v || (path_len && !pred)) {
        rc = OR_OOM;
        goto done;
    }
    rc = validate_sets(&L, A, nA, B, nB, inA, inB);
    if (rc) goto done;
    /* reuse the state heap: t = F1, q = -F2 (so "higher q first" = lighter first) */
    for (int64_t v = 0; v < V; v++)
        if (inA[v]) {
            state_t s = {0, 0, v, -1, -1};
            if ((rc = heap_push(&H, s))) goto done;
        }
    while (H.n > 0) {
        state_t s = heap_pop(&H);
        if (done_v[s.v]) continue;
        done_v[s.v] = 1;
        if (pred) pred[s.v] = s.src;
        if (inB[s.v]) {
            res[0] = s.t;
            res[1] = -s.q;
            res[2] = s.v;
            res[3] = s.src;
            res[4] = s.dir;
            if (pred) {
                int64_t n = 0;
                for (int64_t v = s.v; v >= 0; v = pred[v]) n++;
                *path_len = n;
                if (path && n <= cap) {
                    int64_t i = n;
                    for (int64_t v = s.v; v >= 0; v = pred[v]) path[--i] = v;
                }
            }
            break;
        }
        for (int dir = 0; dir < L.slots; dir++) {
            int64_t t, w;
            int64_t u = neighbour(&L, s.v, dir, &t, &w);
            if (u < 0 || done_v[u]) continue;
            state_t n = {s.t + t, s.q - w, u, s.v, dir};
            if ((rc = heap_push(&H, n))) goto done;
        }
    }
done:
    free(inA); free(inB); free(done_v); free(H.a); free(pred);
    return rc;
}
