// libcsp serving mode: one resident lattice, a stream of (A, B, M) queries, continuous
// batching on the device.
//
// One persistent cooperative kernel runs for the whole session.  Its CTAs form fixed
// groups; each group owns one query slot (labels, offers, arrival list, flow pools) and
// loops: its leader claims the next query from a ring in host-mapped memory (written by
// the host, which on Grace-Blackwell the GPU reads coherently), the group solves it with
// the same cycle loop as csp_solve, and the leader publishes the result and a done flag
// back to host memory.  Queries that arrive while others are running are picked up by
// whichever group frees up first, so their work overlaps on the device; the host admits
// a query into the ring only while the ring (one entry per slot plus a small backlog) has
// room.  The paper solves one query at a time; this mode is an addition.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cstring>
#include <new>
#include <thread>
#include <vector>

#include "csp.h"
#include "csp_device.cuh"
#include "csp_internal.h"

using namespace csp;

namespace {

constexpr int kMaxInline = 64;  // sources (and explicit targets) carried in a descriptor

struct QueryDesc {
    long long ticket;  // ring position + 1 once written (0 = empty)
    int nA, nB;        // nB = 0 with axis >= 0: hyperplane target
    int axis, M;
    long long coord;
    long long max_cycles;
    uint32_t A[kMaxInline];
    uint32_t B[kMaxInline];
};

struct ResultSlot {
    long long r[R_COUNT];
    long long done;  // ticket of the query whose result this is (0 = none yet)
    long long pad[15];
};

constexpr int kMaxGroups = 1024;

// Host-mapped control words (written by the host, read by the kernel and vice versa).
struct HostCtl {
    alignas(128) unsigned long long tail;  // queries written so far
    alignas(128) int shutdown;             // 1 = no more queries: groups exit when idle
    alignas(128) unsigned long long served;
    // counters written by the kernel (each by one writer at a time)
    alignas(128) long long wide_queries;   // queries solved by the whole grid
    long long to_wide, to_narrow;          // switches between the two modes
    long long narrow_queries[kMaxGroups];  // queries solved by each group
};

// The server's mode word: generation (high 32 bits), wide flag (bit 31) and the number of
// narrow groups parked idle (low 31 bits).  Every change is a compare-and-swap.
constexpr unsigned long long kWideBit = 1ull << 31;
constexpr long long kCmdExit = -1, kCmdWide = -2, kCmdNarrow = -3;

__device__ __forceinline__ unsigned long long mode_word(unsigned long long gen, bool wide, unsigned long long parked)
{
    return (gen << 32) | (wide ? kWideBit : 0ull) | parked;
}

struct GroupSlot {
    int32_t *label;
    unsigned long long *offer;
    uint32_t *isB, *cand;
    unsigned int cand_cap, pool_cap;
    uint32_t *ed[2];
    int32_t *qa[2];
    int32_t *ta[2];
    unsigned long long *pk[2];  // packed pool views (nullable)
    uint32_t *fill[2];
    Control *ctl;
    long long *result;  // device copy of the current query's result
    uint32_t *touched;  // vertices whose label left 0 during the current query
    unsigned int *touched_n;
};

struct ServerArgs {
    const uint4 *rec;
    const uint32_t *nbw, *nbw_in;  // general graphs: the out- and in-edge tables (null on a lattice)
    long long V;
    int stride[4];
    unsigned int max_f1;       // largest travel time of the lattice
    const GroupSlot *slots;    // [groups] narrow slots, then the wide slot (whole grid)
    int group_ctas, groups;
    unsigned long long *head;  // device: next ring position to claim
    long long *mailbox;        // device: per group, the claimed position or a command; [groups] = the grid's
    unsigned long long *mode;  // device: the mode word
    HostCtl *hctl;             // host-mapped
    const QueryDesc *ring;     // host-mapped
    ResultSlot *results;       // host-mapped
    long long ring_size;
    unsigned long long session_ns;
    int wide_depth;            // queued queries that end the wide mode; <= 0: no wide mode
};

template <typename W>
__device__ void slot_params(Params<W> &P, const ServerArgs &S, const GroupSlot &slot)
{
    P = Params<W>{};
    P.rec = S.rec;
    P.nbw = S.nbw;
    P.nbw_in = S.nbw_in;
    P.V = S.V;
    for (int k = 0; k < 4; k++) P.stride[k] = S.stride[k];
    P.label = slot.label;
    P.offer = slot.offer;
    P.isB = slot.isB;
    P.cand = slot.cand;
    P.cand_cap = slot.cand_cap;
    for (int b = 0; b < 2; b++) {
        P.ed[b] = slot.ed[b];
        P.qa[b] = slot.qa[b];
        P.ta[b] = slot.ta[b];
        P.pk[b] = slot.pk[b];
        P.fill[b] = slot.fill[b];
    }
    P.max_f1 = S.max_f1;
    P.pool_cap = slot.pool_cap;
    P.ctl = slot.ctl;
    P.result_dev = slot.result;
    P.touched = slot.touched;
    P.touched_n = slot.touched_n;
    P.budget_ns = 120ull * 1000000000ull;
    P.barrier_ns = S.session_ns;  // an idle group waits for work at its barrier
}

__device__ __forceinline__ unsigned long long ring_tail(const ServerArgs &S)
{
    unsigned long long tail;
    asm volatile("ld.acquire.sys.global.u64 %0, [%1];" : "=l"(tail) : "l"(&S.hctl->tail) : "memory");
    return tail;
}

// The grid's leader in the wide mode: the next query to solve with the whole grid, or
// kCmdNarrow when wide_depth queries or more are waiting (continuous batching then serves
// them in parallel), or kCmdExit (shutdown with the ring drained, or the session is over).
__device__ long long wide_claim(const ServerArgs &S, unsigned long long t_begin)
{
    for (unsigned int spin = 0;; ++spin) {
        const unsigned long long tail = ring_tail(S);
        const unsigned long long h = *(volatile unsigned long long *)S.head;
        if (h < tail) {
            if (tail - h >= (unsigned long long)S.wide_depth) {
                const unsigned long long m = *(volatile unsigned long long *)S.mode;
                atomicExch(S.mode, mode_word((m >> 32) + 1, false, 0));
                *(volatile long long *)&S.hctl->to_narrow += 1;
                return kCmdNarrow;
            }
            if (atomicCAS(S.head, h, h + 1) == h) return (long long)h;
            continue;
        }
        if (*(volatile const int *)&S.hctl->shutdown) return kCmdExit;
        if ((spin & 255u) == 255u && globaltimer_ns() - t_begin > S.session_ns) return kCmdExit;
        __nanosleep(spin < 64 ? 200 : 2000);
    }
}

// A narrow group's leader: the next query for its group, or kCmdWide when the grid has
// switched to the wide mode, or kCmdExit.  A leader that finds the ring empty parks its
// group (counted in the mode word); the group that parks last while the ring is empty
// switches the grid to the wide mode.  A parked leader unparks before it claims.
__device__ long long narrow_claim(const ServerArgs &S, unsigned long long t_begin)
{
    bool parked = false;
    for (unsigned int spin = 0;; ++spin) {
        const unsigned long long m = *(volatile unsigned long long *)S.mode;
        if (m & kWideBit) return kCmdWide;
        const unsigned long long tail = ring_tail(S);
        const unsigned long long h = *(volatile unsigned long long *)S.head;
        if (h < tail) {
            if (parked) {  // unpark first (fails if the mode word moved on: look again)
                if (atomicCAS(S.mode, m, m - 1) != m) continue;
                parked = false;
            }
            if (atomicCAS(S.head, h, h + 1) == h) return (long long)h;
            continue;
        }
        if (*(volatile const int *)&S.hctl->shutdown) return kCmdExit;
        if ((spin & 255u) == 255u && globaltimer_ns() - t_begin > S.session_ns) return kCmdExit;
        if (!parked && S.wide_depth > 0) {
            if (atomicCAS(S.mode, m, m + 1) != m) continue;
            parked = true;
            if ((m & (kWideBit - 1)) + 1 == (unsigned long long)S.groups) {
                // every group is idle and the ring is empty: the whole grid takes the next query
                if (atomicCAS(S.mode, m + 1, mode_word((m >> 32) + 1, true, 0)) == m + 1) {
                    *(volatile long long *)&S.hctl->to_wide += 1;
                    return kCmdWide;
                }
            }
            continue;
        }
        __nanosleep(spin < 64 ? 200 : 2000);
    }
}

template <int D, typename W>
__global__ void __launch_bounds__(TPB, CSP_MIN_CTAS_PER_SM) k_server(ServerArgs S)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    Smem &sm = *reinterpret_cast<Smem *>(smem_raw);
    init_stage_barriers(sm);
    uint32_t parity[NSTAGE] = {};
    const int gid = blockIdx.x / S.group_ctas;
    const Group gn{(uint32_t)(blockIdx.x % S.group_ctas), (uint32_t)S.group_ctas};  // this CTA's narrow group
    const Group gw{blockIdx.x, gridDim.x};                                            // the whole grid
    // both slots' parameters live in shared memory (read like kernel arguments), not in registers
    __shared__ Params<W> s_P[2];
    if (threadIdx.x == 0) {
        slot_params<W>(s_P[0], S, S.slots[gid]);
        slot_params<W>(s_P[1], S, S.slots[S.groups]);
    }
    __syncthreads();
    unsigned long long epoch[2] = {0, 0};  // barriers passed on the narrow slot and on the wide slot
    const unsigned long long t_begin = globaltimer_ns();
    __shared__ long long s_pos;
    __shared__ QueryDesc s_q;
    bool wide = S.wide_depth > 0;  // start wide: an idle server answers its first query with every CTA
    for (;;) {
        const Group g = wide ? gw : gn;
        Params<W> &P = s_P[wide ? 1 : 0];
        unsigned long long &ep = epoch[wide ? 1 : 0];
        long long *mail = S.mailbox + (wide ? S.groups : gid);
        if (g.leader()) *mail = wide ? wide_claim(S, t_begin) : narrow_claim(S, t_begin);
        if (!group_sync(P.ctl, ep, g, P.barrier_ns)) break;
        if (threadIdx.x == 0) s_pos = *(volatile long long *)mail;
        __syncthreads();
        const long long pos = s_pos;
        __syncthreads();
        if (pos == kCmdExit) break;
        if (pos == kCmdWide || pos == kCmdNarrow) {
            wide = pos == kCmdWide;
            continue;
        }
        {
            // the descriptor lives in host memory and ring entries are reused: read it with
            // volatile (uncached) loads into shared memory
            const volatile uint32_t *src = reinterpret_cast<const volatile uint32_t *>(&S.ring[pos % S.ring_size]);
            uint32_t *dst = reinterpret_cast<uint32_t *>(&s_q);
            for (int i = threadIdx.x; i < (int)(sizeof(QueryDesc) / 4); i += TPB) dst[i] = src[i];
        }
        __syncthreads();
        const QueryDesc &q = s_q;
        if (threadIdx.x == 0) {
            P.M = q.M;
            P.max_cycles = q.max_cycles;
        }
        __syncthreads();
        const TargetSet T{nullptr, q.nB > 0 ? q.B : nullptr, q.nB, q.nB > 0 ? -1 : q.axis, q.coord};
        // the slot's labels, offers and B bitmap are all zero here (zeroed at creation and
        // undone after every query), so the set-up touches only A and B
        group_setup_sets<W>(P, g, nullptr, q.A, q.nA, T, ep, false);
        run_solve<D, W, false>(P, g, sm, parity, ep);
        if (!group_sync(P.ctl, ep, g, P.barrier_ns)) break;
        if (g.leader()) {
            ResultSlot &out = S.results[pos % S.ring_size];
            for (int i = 0; i < R_COUNT; i++) out.r[i] = __ldcg(P.result_dev + i);
            __threadfence_system();
            asm volatile("st.release.sys.global.u64 [%0], %1;" ::"l"(&out.done), "l"(pos + 1) : "memory");
            if (wide) *(volatile long long *)&S.hctl->wide_queries += 1;
            else *(volatile long long *)&S.hctl->narrow_queries[gid] += 1;
        }
        if (!group_undo<W>(P, g, q.A, q.nA, T, ep)) break;
    }
}

template <typename W>
const void *server_kernel(int d)
{
    switch (d) {
    case 1: return (const void *)&k_server<1, W>;
    case 2: return (const void *)&k_server<2, W>;
    case 3: return (const void *)&k_server<3, W>;
    case GRAPH: return (const void *)&k_server<GRAPH, W>;
    default: return (const void *)&k_server<4, W>;
    }
}

constexpr size_t kSmem = sizeof(Smem);

}  // namespace

struct csp_server {
    csp_lattice *lat = nullptr;
    int groups = 0, group_ctas = 0;
    long long ring_size = 0;
    void *ws = nullptr;
    GroupSlot *d_slots = nullptr;
    unsigned long long *d_head = nullptr;  // (with the mode word right after it)
    long long *d_mailbox = nullptr;
    void *wide_ws = nullptr;  // the wide slot's workspace
    int wide_depth = 0;
    HostCtl *hctl = nullptr;  // pinned, mapped
    QueryDesc *ring = nullptr;
    ResultSlot *results = nullptr;
    void *host_block = nullptr;
    cudaStream_t stream = nullptr;
    unsigned long long next = 0;  // tickets written so far
    bool running = false;
    double session_s = 600.0;
};

namespace {

void fill_desc(QueryDesc &d, const csp_server_query &q, long long pos)
{
    std::memset(&d, 0, sizeof(d));
    d.nA = (int)q.nA;
    for (int i = 0; i < d.nA; i++) d.A[i] = (uint32_t)q.A[i];
    d.nB = q.B ? (int)q.nB : 0;
    for (int i = 0; i < d.nB; i++) d.B[i] = (uint32_t)q.B[i];
    d.axis = q.B ? -1 : q.b_axis;
    d.coord = q.b_coord;
    d.M = (int)q.M;
    d.max_cycles = q.max_cycles;
    d.ticket = pos + 1;
}

bool valid_query(const csp_server *s, const csp_server_query &q)
{
    if (!q.A || q.nA < 1 || q.nA > kMaxInline || q.M >= (1ll << 31) - 1 || q.M < -(1ll << 31) + 1) return false;
    if (q.B) {
        if (q.nB < 1 || q.nB > kMaxInline) return false;
    } else if (q.b_axis < 0 || q.b_axis >= num_axes(s->lat) || q.b_coord < 0 || q.b_coord >= s->lat->ext[q.b_axis]) {
        return false;
    }
    return true;
}

void copy_result(const long long *o, csp_result *x, int32_t *status)
{
    x->F1 = o[R_F1];
    x->X = o[R_X];
    x->x_src = o[R_XSRC];
    x->x_dir = o[R_XDIR];
    x->F2 = o[R_F2];
    x->cycles = o[R_CYCLES];
    x->updates = o[R_UPDATES];
    x->launched = o[R_LAUNCHED];
    x->passes = o[R_PASSES];
    x->max_pool = o[R_MAXPOOL];
    x->arrivals = o[R_ARRIVALS];
    x->improved = o[R_IMPROVED];
    x->phantoms = o[R_PHANTOMS];
    if (status) *status = (int32_t)o[R_STATUS];
}

}  // namespace

extern "C" {

csp_status csp_server_create(csp_lattice *L, const csp_server_options *opt, csp_server **out)
{
    if (!L || !out) return CSP_ERR_INVALID;
    *out = nullptr;
    csp_server *s = new (std::nothrow) csp_server();
    if (!s) return CSP_ERR_OOM;
    s->lat = L;
    const void *fn = L->wbytes == 1 ? server_kernel<uint8_t>(L->d) : server_kernel<uint16_t>(L->d);
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmem);
    int per_sm = 0;
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, TPB, kSmem);
    if (e != cudaSuccess || per_sm < 1) {
        delete s;
        return e != cudaSuccess ? cuda_fail(e, "server kernel attributes") : CSP_ERR_CUDA;
    }
    const int max_ctas = per_sm * num_sms(L->device);
    int gc = opt && opt->group_ctas > 0 ? opt->group_ctas : 16;
    gc = std::max(1, std::min(gc, max_ctas));
    int groups = max_ctas / gc;
    if (opt && opt->max_groups > 0) groups = std::min(groups, opt->max_groups);
    const int64_t V = L->V;
    // default: max(2^16, V) flows (at most the lattice's flow bound) plus the chunks a pass
    // may leave part-filled; an explicit capacity is taken as given (rounded up to whole chunks)
    const int64_t base_pool = opt && opt->pool_capacity > 0
                                  ? opt->pool_capacity
                                  : std::min<int64_t>(std::max<int64_t>(1 << 16, V), (int64_t)std::max(L->flow_bound, 1024ull));
    // one slot's layout for a group of gsize CTAs: returns its bytes and fills the offsets
    struct Layout {
        int64_t pool, cand;
        size_t label, offer, isB, cand_o, ctl, res, touched, tn, pool_o[2][3], fill[2], bytes;
    };
    auto layout = [&](int64_t gsize, bool add_slack) {
        Layout y{};
        int64_t pool = add_slack ? base_pool + chunk_slack(gsize) : base_pool;
        pool = std::min<int64_t>(pool, 0xF0000000ll);
        pool = (pool + TILE - 1) / TILE * TILE;  // whole chunks
        y.pool = pool;
        y.cand = std::max<int64_t>(V, pool + gsize * TILE);  // one region per CTA of the group
        size_t per = 0;
        auto take = [&](size_t bytes) {
            size_t o = per;
            per = align_up(per + bytes, 256);
            return o;
        };
        y.label = take(V * 4);
        y.offer = take(V * 8);
        y.isB = take(((V + 31) / 32) * 4);
        y.cand_o = take(y.cand * 4);
        y.ctl = take(sizeof(Control));
        y.res = take(R_COUNT * 8);
        y.touched = take(V * 4);
        y.tn = take(256);
        for (int b = 0; b < 2; b++) {
            for (int f = 0; f < 3; f++) y.pool_o[b][f] = take((pool + POOL_PAD) * 4);
            y.fill[b] = take((pool / TILE + 1) * 4);
        }
        y.bytes = per;
        return y;
    };
    const bool explicit_pool = opt && opt->pool_capacity > 0;
    const Layout ln = layout(gc, !explicit_pool);
    const size_t per = ln.bytes;
    if (opt && opt->memory_budget > 0) groups = (int)std::max<int64_t>(1, std::min<int64_t>(groups, opt->memory_budget / per));
    groups = std::min(groups, kMaxGroups);
    const int wide_depth = opt && opt->wide_depth != 0 ? opt->wide_depth : 3;
    const Layout lw = layout((int64_t)groups * gc, true);
    s->groups = groups;
    s->group_ctas = gc;
    s->wide_depth = wide_depth;
    s->ring_size = opt && opt->queue_capacity > 0 ? opt->queue_capacity : 4 * groups;
    e = cudaMalloc(&s->ws, per * groups);
    if (e == cudaSuccess && wide_depth > 0) e = cudaMalloc(&s->wide_ws, lw.bytes);
    if (e == cudaSuccess) e = cudaMalloc((void **)&s->d_slots, (groups + 1) * sizeof(GroupSlot));
    if (e == cudaSuccess) e = cudaMalloc((void **)&s->d_head, 256);
    if (e == cudaSuccess) e = cudaMalloc((void **)&s->d_mailbox, (groups + 1) * sizeof(long long));
    const size_t host_bytes = sizeof(HostCtl) + s->ring_size * (sizeof(QueryDesc) + sizeof(ResultSlot)) + 256;
    if (e == cudaSuccess) e = cudaHostAlloc(&s->host_block, host_bytes, cudaHostAllocMapped);
    if (e != cudaSuccess) {
        cudaGetLastError();
        csp_server_destroy(s);
        return cuda_fail(e, "server allocation");
    }
    std::memset(s->host_block, 0, host_bytes);
    s->hctl = (HostCtl *)s->host_block;
    s->ring = (QueryDesc *)((char *)s->host_block + sizeof(HostCtl));
    s->results = (ResultSlot *)((char *)s->ring + s->ring_size * sizeof(QueryDesc));
    auto carve = [&](char *b, const Layout &y) {
        GroupSlot g{};
        g.label = (int32_t *)(b + y.label);
        g.offer = (unsigned long long *)(b + y.offer);
        g.isB = (uint32_t *)(b + y.isB);
        g.cand = (uint32_t *)(b + y.cand_o);
        g.cand_cap = (unsigned int)y.cand;
        g.pool_cap = (unsigned int)y.pool;
        for (int q = 0; q < 2; q++) {
            g.ed[q] = (uint32_t *)(b + y.pool_o[q][0]);
            g.qa[q] = (int32_t *)(b + y.pool_o[q][1]);
            g.ta[q] = (int32_t *)(b + y.pool_o[q][2]);
            g.pk[q] = packed_pool(g.qa[q], g.ta[q], y.pool);
            g.fill[q] = (uint32_t *)(b + y.fill[q]);
        }
        g.ctl = (Control *)(b + y.ctl);
        g.result = (long long *)(b + y.res);
        g.touched = (uint32_t *)(b + y.touched);
        g.touched_n = (unsigned int *)(b + y.tn);
        return g;
    };
    std::vector<GroupSlot> slots(groups + 1);
    char *ws = (char *)s->ws;
    for (int i = 0; i < groups; i++) slots[i] = carve(ws + per * i, ln);
    // the wide slot (the whole grid); with no wide mode it repeats slot 0 and is never used
    slots[groups] = wide_depth > 0 ? carve((char *)s->wide_ws, lw) : slots[0];
    if (e == cudaSuccess) e = cudaMemset(ws, 0, per * groups);  // all labels, offers, bitmaps and controls
    if (e == cudaSuccess && wide_depth > 0) e = cudaMemset(s->wide_ws, 0, lw.bytes);
    if (e == cudaSuccess)
        e = cudaMemcpy(s->d_slots, slots.data(), (groups + 1) * sizeof(GroupSlot), cudaMemcpyHostToDevice);
    const unsigned long long mode0 = wide_depth > 0 ? (1ull << 31) : 0ull;  // start wide
    if (e == cudaSuccess) e = cudaMemset(s->d_head, 0, 256);
    if (e == cudaSuccess) e = cudaMemcpy(s->d_head + 1, &mode0, 8, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking);
    ServerArgs a{};
    if (e == cudaSuccess) {
        a.rec = (const uint4 *)L->rec;
        a.nbw = L->nbw;
        a.nbw_in = L->nbw_in;
        a.V = V;
        for (int k = 0; k < 4; k++) a.stride[k] = L->stride[k];
        a.max_f1 = L->max_f1;
        a.slots = s->d_slots;
        a.group_ctas = gc;
        a.groups = groups;
        a.head = s->d_head;
        a.mode = s->d_head + 1;
        a.mailbox = s->d_mailbox;
        a.wide_depth = wide_depth;
        void *p = nullptr;
        e = cudaHostGetDevicePointer(&p, s->host_block, 0);
        a.hctl = (HostCtl *)p;
        a.ring = (const QueryDesc *)((char *)p + sizeof(HostCtl));
        a.results = (ResultSlot *)((char *)a.ring + s->ring_size * sizeof(QueryDesc));
        a.ring_size = s->ring_size;
        const double secs = opt && opt->session_seconds > 0 ? opt->session_seconds : 600.0;
        a.session_ns = (unsigned long long)(secs * 1e9);
        s->session_s = secs;
    }
    if (e == cudaSuccess) {
        void *args[1] = {&a};
        e = cudaLaunchCooperativeKernel(fn, dim3(groups * gc), dim3(TPB), args, kSmem, s->stream);
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        csp_server_destroy(s);
        return cuda_fail(e, "server launch");
    }
    s->running = true;
    *out = s;
    return CSP_OK;
}

csp_status csp_server_info(const csp_server *s, int32_t *groups, int32_t *group_ctas, int64_t *queue_capacity)
{
    if (!s) return CSP_ERR_INVALID;
    if (groups) *groups = s->groups;
    if (group_ctas) *group_ctas = s->group_ctas;
    if (queue_capacity) *queue_capacity = s->ring_size;
    return CSP_OK;
}

csp_status csp_server_stats(const csp_server *s, int64_t *wide_queries, int64_t *narrow_queries, int64_t *to_wide,
                            int64_t *to_narrow)
{
    if (!s || !s->hctl) return CSP_ERR_INVALID;
    const volatile HostCtl *h = s->hctl;
    if (wide_queries) *wide_queries = h->wide_queries;
    if (narrow_queries) {
        long long n = 0;
        for (int i = 0; i < s->groups; i++) n += h->narrow_queries[i];
        *narrow_queries = n;
    }
    if (to_wide) *to_wide = h->to_wide;
    if (to_narrow) *to_narrow = h->to_narrow;
    return CSP_OK;
}

csp_status csp_server_submit(csp_server *s, const csp_server_query *q, int64_t *ticket)
{
    if (!s || !q || !ticket || !s->running) return CSP_ERR_INVALID;
    if (!valid_query(s, *q)) return CSP_ERR_INVALID;
    const unsigned long long pos = s->next;
    // the ring entry must be free: the query that last used it has been served
    if (pos >= (unsigned long long)s->ring_size) {
        const ResultSlot &old = s->results[pos % s->ring_size];
        if (*(volatile long long *)&old.done != (long long)(pos - s->ring_size + 1)) return CSP_ERR_CAPACITY;
    }
    fill_desc(s->ring[pos % s->ring_size], *q, (long long)pos);
    std::atomic_thread_fence(std::memory_order_seq_cst);
    *(volatile unsigned long long *)&s->hctl->tail = pos + 1;
    s->next = pos + 1;
    *ticket = (int64_t)pos;
    return CSP_OK;
}

csp_status csp_server_poll(csp_server *s, int64_t ticket, csp_result *out, int32_t *status, int32_t *done)
{
    if (!s || !done || ticket < 0 || (unsigned long long)ticket >= s->next) return CSP_ERR_INVALID;
    const ResultSlot &r = s->results[ticket % s->ring_size];
    const long long d = *(volatile long long *)&r.done;
    *done = d == ticket + 1;
    if (d > ticket + 1) return CSP_ERR_INVALID;  // overwritten: the result was not collected in time
    if (*done) {
        std::atomic_thread_fence(std::memory_order_acquire);
        long long o[R_COUNT];
        std::memcpy(o, (const void *)r.r, sizeof(o));
        if (out) copy_result(o, out, status);
        else if (status) *status = (int32_t)o[R_STATUS];
    }
    return CSP_OK;
}

csp_status csp_server_replay(csp_server *s, const csp_server_query *q, const double *arrival_s, int64_t n,
                             csp_result *out, int32_t *status, double *latency_s, double *makespan_s)
{
    if (!s || !q || !arrival_s || n < 0 || !s->running) return CSP_ERR_INVALID;
    for (int64_t i = 0; i < n; i++)
        if (!valid_query(s, q[i])) return CSP_ERR_INVALID;
    using clk = std::chrono::steady_clock;
    const auto t0 = clk::now();
    auto now_s = [&]() { return std::chrono::duration<double>(clk::now() - t0).count(); };
    std::vector<int64_t> ticket(n, -1);
    std::vector<char> done(n, 0);
    int64_t next = 0, finished = 0, first_open = 0;
    while (finished < n) {
        bool progress = false;
        // admit arrived queries while a ring entry is free
        while (next < n && arrival_s[next] <= now_s()) {
            if (next >= s->ring_size && !done[next - s->ring_size]) break;  // its ring entry is still in use
            int64_t t = -1;
            const csp_status st = csp_server_submit(s, &q[next], &t);
            if (st == CSP_ERR_CAPACITY) break;
            if (st != CSP_OK) return st;
            ticket[next++] = t;
            progress = true;
        }
        // collect finished queries (in any order)
        for (int64_t i = first_open; i < next; i++) {
            if (done[i]) continue;
            int32_t d = 0;
            csp_result r{};
            int32_t stt = 0;
            const csp_status st = csp_server_poll(s, ticket[i], &r, &stt, &d);
            if (st != CSP_OK) return st;
            if (d) {
                done[i] = 1;
                finished++;
                if (out) out[i] = r;
                if (status) status[i] = stt;
                if (latency_s) latency_s[i] = now_s() - arrival_s[i];
                progress = true;
            }
        }
        while (first_open < next && done[first_open]) first_open++;
        if (!progress) std::this_thread::sleep_for(std::chrono::microseconds(20));
        if (now_s() > s->session_s + 60.0) return CSP_ERR_TIMEOUT;  // the kernel has given up by now
    }
    if (makespan_s) *makespan_s = now_s();
    return CSP_OK;
}

csp_status csp_server_destroy(csp_server *s)
{
    if (!s) return CSP_ERR_INVALID;
    csp_status st = CSP_OK;
    if (s->running) {
        *(volatile int *)&s->hctl->shutdown = 1;
        std::atomic_thread_fence(std::memory_order_seq_cst);
        const cudaError_t e = cudaStreamSynchronize(s->stream);
        if (e != cudaSuccess) st = cuda_fail(e, "server shutdown");
    }
    if (s->stream) cudaStreamDestroy(s->stream);
    if (s->host_block) cudaFreeHost(s->host_block);
    if (s->d_mailbox) cudaFree(s->d_mailbox);
    if (s->d_head) cudaFree(s->d_head);
    if (s->d_slots) cudaFree(s->d_slots);
    if (s->ws) cudaFree(s->ws);
    if (s->wide_ws) cudaFree(s->wide_ws);
    delete s;
    return st;
}

// Baseline for the serving benchmark: the same stream answered one query at a time by
// csp_solve (one launch per query, the whole GPU each), in arrival order.
csp_status csp_serve_plain_replay(csp_lattice *L, const csp_server_query *q, const double *arrival_s, int64_t n,
                                  csp_result *out, int32_t *status, double *latency_s, double *makespan_s)
{
    if (!L || !q || !arrival_s || n < 0) return CSP_ERR_INVALID;
    using clk = std::chrono::steady_clock;
    const auto t0 = clk::now();
    auto now_s = [&]() { return std::chrono::duration<double>(clk::now() - t0).count(); };
    std::vector<int64_t> B;
    for (int64_t i = 0; i < n; i++) {
        while (now_s() < arrival_s[i]) std::this_thread::sleep_for(std::chrono::microseconds(20));
        const int64_t *Bp = q[i].B;
        int64_t nB = q[i].nB;
        if (!Bp) {  // expand the hyperplane into an id list
            const int k = q[i].b_axis;
            if (k < 0 || k >= num_axes(L)) return CSP_ERR_INVALID;
            const int64_t st = L->stride[k], nk = L->ext[k], count = L->V / nk;
            B.resize(count);
            for (int64_t j = 0; j < count; j++) B[j] = (j / st) * st * nk + q[i].b_coord * st + (j % st);
            Bp = B.data();
            nB = count;
        }
        csp_options o{};
        o.max_cycles = q[i].max_cycles;
        csp_result r{};
        const csp_status st = csp_solve(L, q[i].A, q[i].nA, Bp, nB, q[i].M, &o, &r, nullptr, 0, nullptr);
        if (out) out[i] = r;
        if (status) status[i] = st;
        if (latency_s) latency_s[i] = now_s() - arrival_s[i];
    }
    if (makespan_s) *makespan_s = now_s();
    return CSP_OK;
}

}  // extern "C"
