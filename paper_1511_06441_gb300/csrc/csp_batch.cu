// libcsp batched mode: many independent solves (different lattices, sizes, sets and
// bounds) in ONE persistent cooperative launch, optionally captured in a CUDA graph.
//
// The grid is shared out by a list scheduler: each instance gets a group of CTAs (a
// power of two, chosen from a cost model) and a start slot; every CTA walks its own
// list of (instance, rank, group size) entries in start-time order.  Within a group the
// CTAs synchronise with the instance's own barrier (a plain block barrier for groups of
// one), so instances never wait for each other and one instance's memory latency is
// hidden behind the work of the others on the same SMs.  Because every group meets an
// instance at the same point of its members' lists (same start time), the waits form
// no cycle, and the cooperative launch keeps every CTA resident.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <numeric>
#include <string>
#include <vector>

#include "csp.h"
#include "csp_device.cuh"
#include "csp_internal.h"

using namespace csp;

namespace {

struct BatchInstance {
    const uint4 *rec;
    const uint32_t *nbw, *nbw_in;  // general graphs: the out- and in-edge tables (null on a lattice)
    long long V;
    int d, wbytes;
    int stride[4];
    int32_t *label;
    unsigned long long *offer;
    uint32_t *isB;
    uint32_t *cand;
    unsigned int cand_cap, pool_cap;
    uint32_t *ed[2];
    int32_t *qa[2];
    int32_t *ta[2];
    unsigned long long *pk[2];  // packed pool views (nullable)
    unsigned int max_f1;
    uint32_t *fill[2];
    Control *ctl;
    long long *result;
    const int64_t *A, *B;
    long long nA, nB;
    int M;
    long long max_cycles;
};

struct BatchWork {
    int inst, rank, size, pad;
};

template <typename W>
__device__ __forceinline__ Params<W> batch_params(const BatchInstance &I, unsigned long long budget_ns)
{
    Params<W> P{};
    P.rec = I.rec;
    P.nbw = I.nbw;
    P.nbw_in = I.nbw_in;
    P.V = I.V;
    for (int k = 0; k < 4; k++) P.stride[k] = I.stride[k];
    P.label = I.label;
    P.offer = I.offer;
    P.isB = I.isB;
    P.src_stamp = nullptr;
    P.cand = I.cand;
    P.cand_cap = I.cand_cap;
    for (int b = 0; b < 2; b++) {
        P.ed[b] = I.ed[b];
        P.qa[b] = I.qa[b];
        P.ta[b] = I.ta[b];
        P.pk[b] = I.pk[b];
        P.fill[b] = I.fill[b];
    }
    P.max_f1 = I.max_f1;
    P.pool_cap = I.pool_cap;
    P.ctl = I.ctl;
    P.trace = nullptr;
    P.trace_cap = 0;
    P.result_dev = I.result;
    P.M = I.M;
    P.max_cycles = I.max_cycles;
    P.budget_ns = budget_ns;
    P.barrier_ns = budget_ns;  // a group may wait for a member still finishing its previous instance
    return P;
}

// One instance on its group, out of line: the solves of the four dimensions and of general
// graphs get registers of their own instead of sharing (and spilling) one inlined body.
template <int D, typename W>
__device__ __noinline__ void batch_solve(const Params<W> &P, const Group &g, Smem &sm, uint32_t (&parity)[NSTAGE],
                                         unsigned long long &epoch)
{
    run_solve<D, W, false>(P, g, sm, parity, epoch);
}

// One CTA per SM: the batch kernel holds the solves of all four dimensions, and with the
// 128 registers this allows it runs without spills (2 CTAs per SM at 64 registers spilled
// ~0.6 KB per thread; measured 25.4 vs 24.2 instances/s on 512 mixed instances).
#ifndef CSP_BATCH_MIN_CTAS_PER_SM
#define CSP_BATCH_MIN_CTAS_PER_SM 1
#endif

template <typename W>
__global__ void __launch_bounds__(TPB, CSP_BATCH_MIN_CTAS_PER_SM)
    k_batch(const BatchInstance *insts, const int *list_start, const BatchWork *work, unsigned long long budget_ns)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    Smem &sm = *reinterpret_cast<Smem *>(smem_raw);
    init_stage_barriers(sm);
    uint32_t parity[NSTAGE] = {};
    const int first = list_start[blockIdx.x], last = list_start[blockIdx.x + 1];
    // the instance's parameters live in shared memory (read like kernel arguments), not in
    // registers
    __shared__ Params<W> s_P;
    for (int i = first; i < last; i++) {
        const BatchWork w = work[i];
        const BatchInstance &I = insts[w.inst];
        const Group g{(uint32_t)w.rank, (uint32_t)w.size};
        __syncthreads();  // the previous instance is done with s_P
        if (threadIdx.x == 0) s_P = batch_params<W>(I, budget_ns);
        __syncthreads();
        const Params<W> &P = s_P;
        unsigned long long epoch = 0;
        group_setup<W>(P, g, I.A, I.nA, I.B, I.nB, epoch);  // a failed barrier also fails the solve's first one
        switch (I.d) {
        case 1: batch_solve<1, W>(P, g, sm, parity, epoch); break;
        case 2: batch_solve<2, W>(P, g, sm, parity, epoch); break;
        case 3: batch_solve<3, W>(P, g, sm, parity, epoch); break;
        case GRAPH: batch_solve<GRAPH, W>(P, g, sm, parity, epoch); break;
        default: batch_solve<4, W>(P, g, sm, parity, epoch); break;
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------- cost model and schedule

// What a solve costs: its cycles and its active-edge updates (predicted from the lattice
// before the first run; measured exactly afterwards, since a solve is deterministic).
struct InstStats {
    double cycles, updates;
};

// Device time (us) of one solve on a group of g CTAs: a per-cycle latency (two phases
// and their barriers; block barriers only for g = 1) plus the updates shared by the
// group at `rate` updates per us per CTA.
struct CostModel {
    double lat_single_us = 6.0;
    double lat_group_us = 16.0;
    double rate = 180.0;

    double est(const InstStats &s, int g) const
    {
        const double lat = g == 1 ? lat_single_us : lat_group_us * (1.0 + 0.05 * std::log2((double)g));
        return s.cycles * lat + s.updates / (g * rate);
    }
};

struct Plan {
    std::vector<int> group, first_cta;
    std::vector<double> start_us, est_us;
    std::vector<int> list_start;       // per CTA, into work
    std::vector<BatchWork> work;
    double makespan_us = 0;
};

// Longest first, each instance into the aligned block of g CTAs that frees up earliest.
Plan pack(const std::vector<InstStats> &st, const std::vector<int> &group, int ctas, const CostModel &cm)
{
    const int n = (int)st.size();
    Plan p;
    p.group = group;
    p.first_cta.assign(n, 0);
    p.start_us.assign(n, 0);
    p.est_us.assign(n, 0);
    for (int i = 0; i < n; i++) p.est_us[i] = cm.est(st[i], group[i]);
    std::vector<int> order(n);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return p.est_us[a] > p.est_us[b]; });
    std::vector<double> avail(ctas, 0.0);
    std::vector<std::vector<BatchWork>> lists(ctas);
    for (int i : order) {
        const int g = group[i];
        int best = 0;
        double best_t = 1e300;
        for (int b = 0; b + g <= ctas; b += g) {
            double t = 0;
            for (int c = b; c < b + g; c++) t = std::max(t, avail[c]);
            if (t < best_t) {
                best_t = t;
                best = b;
            }
        }
        p.first_cta[i] = best;
        p.start_us[i] = best_t;
        for (int c = best; c < best + g; c++) {
            avail[c] = best_t + p.est_us[i];
            // every entry starts at or after the CTA's previous entries end: each CTA's
            // list is in start-time order, and instances sharing CTAs appear in the same
            // relative order on all of them (no circular waits)
            lists[c].push_back(BatchWork{i, c - best, g, 0});
        }
        p.makespan_us = std::max(p.makespan_us, best_t + p.est_us[i]);
    }
    p.list_start.assign(ctas + 1, 0);
    for (int c = 0; c < ctas; c++) {
        p.list_start[c + 1] = p.list_start[c] + (int)lists[c].size();
        for (auto &e : lists[c]) p.work.push_back(e);
    }
    return p;
}

// Chooses group sizes for a target makespan T (smallest power of two whose estimate
// fits T, else the fastest) and packs; a bisection on T keeps the best packing.
Plan make_plan(const std::vector<InstStats> &st, int ctas, int max_group, const CostModel &cm)
{
    const int n = (int)st.size();
    double total = 0, floor_t = 0, hi = 0;
    for (int i = 0; i < n; i++) {
        total += cm.est(st[i], 1);
        double best = 1e300;
        for (int g = 1; g <= max_group && g <= ctas; g *= 2) best = std::min(best, cm.est(st[i], g));
        floor_t = std::max(floor_t, best);
        hi += cm.est(st[i], 1);
    }
    double lo = std::max(total / ctas, floor_t);
    hi = std::max(hi, lo);
    Plan best_plan;
    best_plan.makespan_us = 1e300;
    std::vector<int> group(n, 1);
    for (int it = 0; it < 24; it++) {
        const double T = it == 0 ? lo : 0.5 * (lo + hi);
        for (int i = 0; i < n; i++) {
            int g = 1, fastest = 1;
            double tf = cm.est(st[i], 1);
            for (int h = 2; h <= max_group && h <= ctas; h *= 2)
                if (cm.est(st[i], h) < tf) {
                    tf = cm.est(st[i], h);
                    fastest = h;
                }
            while (g < fastest && cm.est(st[i], g) > T) g *= 2;
            group[i] = g;
        }
        Plan p = pack(st, group, ctas, cm);
        if (p.makespan_us < best_plan.makespan_us) best_plan = p;
        if (it == 0 && p.makespan_us <= 1.02 * T) break;
        if (p.makespan_us <= 1.05 * T) hi = T;
        else lo = T;
        if (hi - lo < 0.01 * hi) break;
    }
    return best_plan;
}

constexpr size_t kSmem = sizeof(Smem);

}  // namespace

struct csp_batch {
    int64_t n = 0;
    int wbytes = 1;
    int device = 0;
    int ctas = 0;
    int max_group = 64;
    CostModel cm;
    Plan plan;
    std::vector<BatchInstance> inst;
    std::vector<InstStats> stats;
    void *ws = nullptr;
    BatchInstance *d_inst = nullptr;
    int *d_list = nullptr;
    BatchWork *d_work = nullptr;
    Control *d_ctl = nullptr;
    long long *d_res = nullptr;
    void *d_sched = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaStream_t graph_stream = nullptr;
    bool use_graph = true;
    unsigned long long budget_ns = 120ull * 1000000000ull;
};

namespace {

csp_status upload_plan(csp_batch *b)
{
    if (b->d_sched) cudaFree(b->d_sched);
    b->d_sched = nullptr;
    const size_t list_bytes = align_up(b->plan.list_start.size() * sizeof(int), 256);
    const size_t work_bytes = std::max<size_t>(1, b->plan.work.size()) * sizeof(BatchWork);
    CSP_CUDA(cudaMalloc(&b->d_sched, list_bytes + work_bytes));
    b->d_list = (int *)b->d_sched;
    b->d_work = (BatchWork *)((char *)b->d_sched + list_bytes);
    CSP_CUDA(cudaMemcpy(b->d_list, b->plan.list_start.data(), b->plan.list_start.size() * sizeof(int),
                        cudaMemcpyHostToDevice));
    if (!b->plan.work.empty())
        CSP_CUDA(cudaMemcpy(b->d_work, b->plan.work.data(), b->plan.work.size() * sizeof(BatchWork),
                            cudaMemcpyHostToDevice));
    return CSP_OK;
}

const void *batch_kernel(int wbytes)
{
    return wbytes == 1 ? (const void *)&k_batch<uint8_t> : (const void *)&k_batch<uint16_t>;
}

csp_status enqueue_batch(csp_batch *b, cudaStream_t s)
{
    CSP_CUDA(cudaMemsetAsync(b->d_ctl, 0, b->n * sizeof(Control), s));
    void *args[4] = {&b->d_inst, &b->d_list, &b->d_work, &b->budget_ns};
    CSP_CUDA(cudaLaunchCooperativeKernel(batch_kernel(b->wbytes), dim3(b->ctas), dim3(TPB), args, kSmem, s));
    return CSP_OK;
}

void drop_graph(csp_batch *b)
{
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
}

// Captures one batch run (control reset + the persistent launch) as a CUDA graph.
void capture_graph(csp_batch *b)
{
    drop_graph(b);
    if (!b->use_graph) return;
    cudaStream_t s;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        b->use_graph = false;
        return;
    }
    bool ok = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
    if (ok) {
        const bool enq = enqueue_batch(b, s) == CSP_OK;
        cudaGraph_t g = nullptr;
        ok = cudaStreamEndCapture(s, &g) == cudaSuccess && enq && g;
        if (ok) ok = cudaGraphInstantiate(&b->exec, g, 0) == cudaSuccess;
        b->graph = g;
    }
    if (!ok) {
        cudaGetLastError();
        drop_graph(b);
        b->use_graph = false;  // run the launch directly instead
    }
    cudaStreamDestroy(s);
}

}  // namespace

extern "C" {

csp_status csp_batch_create(const csp_query *q, int64_t n, const csp_batch_options *opt, csp_batch **out)
{
    if (!q || n < 1 || !out || n > (1ll << 24)) return CSP_ERR_INVALID;
    *out = nullptr;
    const int wbytes = q[0].lat ? q[0].lat->wbytes : 0;
    for (int64_t i = 0; i < n; i++) {
        const csp_query &x = q[i];
        if (!x.lat || !x.A || !x.B || x.nA < 1 || x.nB < 1 || x.M >= (1ll << 31) - 1 || x.M < -(1ll << 31) + 1 ||
            x.lat->wbytes != wbytes)
            return CSP_ERR_INVALID;
    }
    csp_batch *b = new (std::nothrow) csp_batch();
    if (!b) return CSP_ERR_OOM;
    b->n = n;
    b->wbytes = wbytes;
    cudaGetDevice(&b->device);
    if (opt && opt->max_group > 0) b->max_group = opt->max_group;
    if (opt) b->use_graph = opt->no_graph == 0;
    const void *fn = batch_kernel(wbytes);
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmem);
    int per_sm = 0;
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, TPB, kSmem);
    if (e != cudaSuccess || per_sm < 1) {
        csp_batch_destroy(b);
        return e != cudaSuccess ? cuda_fail(e, "batch kernel attributes") : CSP_ERR_CUDA;
    }
    const int max_ctas = per_sm * num_sms(b->device);
    b->ctas = opt && opt->ctas > 0 ? std::min(opt->ctas, max_ctas) : max_ctas;
    // workspace: per instance labels, offers, B bitmap, arrival list, two pools, A, B
    std::vector<size_t> off(n);
    size_t total = 0;
    auto take = [&](size_t bytes) {
        size_t o = total;
        total = align_up(total + bytes, 256);
        return o;
    };
    b->inst.resize(n);
    b->stats.resize(n);
    struct Offs {
        size_t label, offer, isB, cand, pool[2][3], fill[2], A, B;
    };
    std::vector<Offs> offs(n);
    for (int64_t i = 0; i < n; i++) {
        const csp_lattice *L = q[i].lat;
        const int64_t V = L->V;
        // default: 6V flows (at most the lattice's flow bound) plus the chunks a pass may leave
        // part-filled; an explicit capacity is taken as given (rounded up to whole chunks)
        int64_t pool = opt && opt->pool_capacity > 0
                           ? opt->pool_capacity
                           : std::min<int64_t>(std::max<int64_t>(1 << 16, 6 * V),
                                               (int64_t)std::max(L->flow_bound, 1024ull)) +
                                 chunk_slack(std::min(b->max_group, b->ctas));
        pool = std::min<int64_t>(pool, 0xF0000000ll);
        pool = (pool + TILE - 1) / TILE * TILE;  // whole chunks
        // one candidate region per CTA of the instance's group (at most max_group CTAs)
        const int64_t cand = std::max<int64_t>(V, pool + (int64_t)std::min(b->max_group, b->ctas) * TILE);
        Offs &o = offs[i];
        o.label = take(V * 4);
        o.offer = take(V * 8);
        o.isB = take(((V + 31) / 32) * 4);
        o.cand = take(cand * 4);
        for (int bb = 0; bb < 2; bb++) {
            for (int f = 0; f < 3; f++) o.pool[bb][f] = take((pool + POOL_PAD) * 4);
            o.fill[bb] = take((pool / TILE + 1) * 4);
        }
        o.A = take(q[i].nA * 8);
        o.B = take(q[i].nB * 8);
        BatchInstance &I = b->inst[i];
        std::memset(&I, 0, sizeof(I));
        I.V = V;
        I.d = L->d;
        I.wbytes = L->wbytes;
        for (int k = 0; k < 4; k++) I.stride[k] = L->stride[k];
        I.rec = (const uint4 *)L->rec;
        I.nbw = L->nbw;
        I.nbw_in = L->nbw_in;
        I.cand_cap = (unsigned int)cand;
        I.pool_cap = (unsigned int)pool;
        I.max_f1 = L->max_f1;
        I.nA = q[i].nA;
        I.nB = q[i].nB;
        I.M = (int)q[i].M;
        I.max_cycles = opt ? opt->max_cycles : 0;
        // first guess before any run: cycles ~ the time to cross the longest side,
        // updates ~ a few hundred per vertex (refined by csp_batch_tune); a graph is guessed
        // like a square lattice of V vertices
        int64_t s = 1;
        for (int k = 0; k < num_axes(L); k++) s = std::max<int64_t>(s, L->ext[k]);
        const bool flat = L->d == 2 || L->d == GRAPH;
        if (L->d == GRAPH) s = std::max<int64_t>(1, (int64_t)std::sqrt((double)V));
        b->stats[i] = InstStats{(flat ? 11.0 : 8.0) * s, (flat ? 4000.0 : 1000.0) * V};
    }
    e = cudaMalloc(&b->ws, std::max<size_t>(total, 256));
    if (e == cudaSuccess) e = cudaMalloc((void **)&b->d_inst, n * sizeof(BatchInstance));
    if (e == cudaSuccess) e = cudaMalloc((void **)&b->d_ctl, n * sizeof(Control));
    if (e == cudaSuccess) e = cudaMalloc((void **)&b->d_res, n * R_COUNT * sizeof(long long));
    if (e != cudaSuccess) {
        cudaGetLastError();
        csp_batch_destroy(b);
        return cuda_fail(e, "cudaMalloc(batch)");
    }
    char *ws = (char *)b->ws;
    for (int64_t i = 0; i < n; i++) {
        BatchInstance &I = b->inst[i];
        const Offs &o = offs[i];
        I.label = (int32_t *)(ws + o.label);
        I.offer = (unsigned long long *)(ws + o.offer);
        I.isB = (uint32_t *)(ws + o.isB);
        I.cand = (uint32_t *)(ws + o.cand);
        for (int bb = 0; bb < 2; bb++) {
            I.ed[bb] = (uint32_t *)(ws + o.pool[bb][0]);
            I.qa[bb] = (int32_t *)(ws + o.pool[bb][1]);
            I.ta[bb] = (int32_t *)(ws + o.pool[bb][2]);
            I.pk[bb] = packed_pool(I.qa[bb], I.ta[bb], (int64_t)I.pool_cap);
            I.fill[bb] = (uint32_t *)(ws + o.fill[bb]);
        }
        I.A = (const int64_t *)(ws + o.A);
        I.B = (const int64_t *)(ws + o.B);
        I.ctl = b->d_ctl + i;
        I.result = b->d_res + i * R_COUNT;
        e = cudaMemcpy((void *)I.A, q[i].A, q[i].nA * 8, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy((void *)I.B, q[i].B, q[i].nB * 8, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) {
            csp_batch_destroy(b);
            return cuda_fail(e, "cudaMemcpy(batch sets)");
        }
    }
    e = cudaMemcpy(b->d_inst, b->inst.data(), n * sizeof(BatchInstance), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        csp_batch_destroy(b);
        return cuda_fail(e, "cudaMemcpy(batch descriptors)");
    }
    b->plan = make_plan(b->stats, b->ctas, b->max_group, b->cm);
    csp_status st = upload_plan(b);
    if (st != CSP_OK) {
        csp_batch_destroy(b);
        return st;
    }
    capture_graph(b);
    *out = b;
    return CSP_OK;
}

csp_status csp_batch_run(csp_batch *b, void *stream)
{
    if (!b) return CSP_ERR_INVALID;
    cudaStream_t s = (cudaStream_t)stream;
    if (b->use_graph && b->exec) {
        CSP_CUDA(cudaGraphLaunch(b->exec, s));
        return CSP_OK;
    }
    return enqueue_batch(b, s);
}

csp_status csp_batch_results(csp_batch *b, csp_result *out, int32_t *status, int64_t *elapsed_ns)
{
    if (!b || !out) return CSP_ERR_INVALID;
    std::vector<long long> r(b->n * R_COUNT);
    CSP_CUDA(cudaDeviceSynchronize());
    CSP_CUDA(cudaMemcpy(r.data(), b->d_res, r.size() * sizeof(long long), cudaMemcpyDeviceToHost));
    for (int64_t i = 0; i < b->n; i++) {
        const long long *o = &r[i * R_COUNT];
        csp_result &x = out[i];
        x.F1 = o[R_F1];
        x.X = o[R_X];
        x.x_src = o[R_XSRC];
        x.x_dir = o[R_XDIR];
        x.F2 = o[R_F2];
        x.cycles = o[R_CYCLES];
        x.updates = o[R_UPDATES];
        x.launched = o[R_LAUNCHED];
        x.passes = o[R_PASSES];
        x.max_pool = o[R_MAXPOOL];
        x.arrivals = o[R_ARRIVALS];
        x.improved = o[R_IMPROVED];
        x.phantoms = o[R_PHANTOMS];
        if (status) status[i] = (int32_t)o[R_STATUS];
        if (elapsed_ns) elapsed_ns[i] = o[R_ELAPSED_NS];
    }
    return CSP_OK;
}

csp_status csp_batch_schedule(const csp_batch *b, int32_t *group_size, int32_t *first_cta, double *start_us,
                              double *est_us, int32_t *ctas)
{
    if (!b) return CSP_ERR_INVALID;
    for (int64_t i = 0; i < b->n; i++) {
        if (group_size) group_size[i] = b->plan.group[i];
        if (first_cta) first_cta[i] = b->plan.first_cta[i];
        if (start_us) start_us[i] = b->plan.start_us[i];
        if (est_us) est_us[i] = b->plan.est_us[i];
    }
    if (ctas) *ctas = b->ctas;
    return CSP_OK;
}

csp_status csp_batch_tune(csp_batch *b, const int64_t *elapsed_ns, const csp_result *res)
{
    if (!b || !elapsed_ns || !res) return CSP_ERR_INVALID;
    // 1) every instance's cycles and updates are now known exactly
    for (int64_t i = 0; i < b->n; i++)
        if (res[i].cycles > 0) b->stats[i] = InstStats{(double)res[i].cycles, (double)res[i].updates};
    // 2) least squares for the three constants of  t = c * lat(g) + u / (g * rate):
    //    unknowns x = (lat_single, lat_group, 1 / rate), rows (c [g==1], c [g>1], u / g)
    double A[3][3] = {{0}}, y[3] = {0};
    int rows = 0;
    for (int64_t i = 0; i < b->n; i++) {
        if (elapsed_ns[i] <= 0 || res[i].cycles <= 0) continue;
        const int g = b->plan.group[i];
        const double f = g == 1 ? 1.0 : 1.0 + 0.05 * std::log2((double)g);
        const double r[3] = {g == 1 ? (double)res[i].cycles : 0.0, g == 1 ? 0.0 : res[i].cycles * f,
                             (double)res[i].updates / g};
        const double t = elapsed_ns[i] * 1e-3;
        for (int a = 0; a < 3; a++) {
            y[a] += r[a] * t;
            for (int c = 0; c < 3; c++) A[a][c] += r[a] * r[c];
        }
        rows++;
    }
    // solve the 3x3 normal equations (Cramer); keep the old constants if singular
    auto det3 = [](double M[3][3]) {
        return M[0][0] * (M[1][1] * M[2][2] - M[1][2] * M[2][1]) - M[0][1] * (M[1][0] * M[2][2] - M[1][2] * M[2][0]) +
               M[0][2] * (M[1][0] * M[2][1] - M[1][1] * M[2][0]);
    };
    const double D = det3(A);
    if (rows >= 3 && std::fabs(D) > 1e-12) {
        double x[3];
        for (int k = 0; k < 3; k++) {
            double Mk[3][3];
            for (int a = 0; a < 3; a++)
                for (int c = 0; c < 3; c++) Mk[a][c] = c == k ? y[a] : A[a][c];
            x[k] = det3(Mk) / D;
        }
        if (x[0] > 0.1) b->cm.lat_single_us = x[0];
        if (x[1] > 0.1) b->cm.lat_group_us = x[1];
        if (x[2] > 0) b->cm.rate = 1.0 / x[2];
    }
    b->plan = make_plan(b->stats, b->ctas, b->max_group, b->cm);
    csp_status st = upload_plan(b);
    if (st != CSP_OK) return st;
    capture_graph(b);
    return CSP_OK;
}

csp_status csp_batch_model(const csp_batch *b, double *lat_single_us, double *lat_group_us, double *rate,
                           double *makespan_us)
{
    if (!b) return CSP_ERR_INVALID;
    if (lat_single_us) *lat_single_us = b->cm.lat_single_us;
    if (lat_group_us) *lat_group_us = b->cm.lat_group_us;
    if (rate) *rate = b->cm.rate;
    if (makespan_us) *makespan_us = b->plan.makespan_us;
    return CSP_OK;
}

csp_status csp_solve_batch(const csp_query *q, int64_t n, const csp_batch_options *opt, csp_result *out,
                           int32_t *status)
{
    if (!q || n < 1 || !out) return CSP_ERR_INVALID;
    csp_batch *b = nullptr;
    csp_status st = csp_batch_create(q, n, opt, &b);
    if (st != CSP_OK) return st;
    std::vector<int32_t> stat(n);
    st = csp_batch_run(b, nullptr);
    if (st == CSP_OK) st = csp_batch_results(b, out, stat.data(), nullptr);
    csp_batch_destroy(b);
    if (st != CSP_OK) return st;
    for (int64_t i = 0; i < n; i++) {
        if (stat[i] == CSP_ERR_CAPACITY) {  // pool too small in the batch: solve alone, growing the pool
            csp_options o{};
            o.max_cycles = opt ? opt->max_cycles : 0;
            stat[i] = csp_solve(const_cast<csp_lattice *>(q[i].lat), q[i].A, q[i].nA, q[i].B, q[i].nB, q[i].M, &o,
                                &out[i], nullptr, 0, nullptr);
        }
        if (status) status[i] = stat[i];
    }
    return CSP_OK;
}

void csp_batch_destroy(csp_batch *b)
{
    if (!b) return;
    drop_graph(b);
    if (b->d_sched) cudaFree(b->d_sched);
    if (b->d_res) cudaFree(b->d_res);
    if (b->d_ctl) cudaFree(b->d_ctl);
    if (b->d_inst) cudaFree(b->d_inst);
    if (b->ws) cudaFree(b->ws);
    delete b;
}

}  // extern "C"
