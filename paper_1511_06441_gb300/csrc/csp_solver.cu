// libcsp: the C ABI of include/csp.h and the persistent cycle kernel.
//
// One solve = a few set-up kernels (labels, B bitmap, sources) and ONE cooperative
// persistent kernel that runs the whole cycle loop of Algorithm 1 on the device:
//
//   seed:  launch phase over A at Time 0 (Algorithm 3, Initialization)
//   loop:  sweep the flow pool at the predicted time Tg        (Steps 1-3, 7-9)
//          grid barrier
//          launch phase over the vertices improved in the sweep (Steps 2, 4, 5, 8)
//          grid barrier
//          every CTA evaluates the same termination test        (Step 6, Algorithm 2)
//
// Tg is the smallest arrival time in the output pool, which may still hold flows that
// died in the cycle just finished (they are removed by the next sweep, which checks
// them against that cycle's labels).  If no live flow arrives at Tg, that sweep only
// removes flows: it is not a cycle, nothing else changes, and the next sweep uses the
// exact minimum.  Results and traces are therefore those of the cycle loop itself.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstddef>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <type_traits>
#include <vector>

#include "csp.h"
#include "csp_device.cuh"
#include "csp_event.cuh"
#include "csp_internal.h"

using namespace csp;

thread_local std::string g_last_error;

csp_status cuda_fail(cudaError_t e, const char *what)
{
    g_last_error = std::string(what) + ": " + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? CSP_ERR_OOM : CSP_ERR_CUDA;
}

void set_error(const std::string &msg) { g_last_error = msg; }

// ---------------------------------------------------------------- set-up kernels

template <typename W>
__global__ void k_zero_upper_faces(W *f1, W *f2, long long V, int d, long long s0, long long s1, long long s2,
                                   long long s3, long long n0, long long n1, long long n2, long long n3)
{
    const long long st[4] = {s0, s1, s2, s3}, n[4] = {n0, n1, n2, n3};
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < d * V;
         i += (long long)gridDim.x * blockDim.x) {
        const int k = (int)(i / V);
        const long long v = i - k * V;
        if ((v / st[k]) % n[k] == n[k] - 1) {
            f1[i] = 0;
            f2[i] = 0;
        }
    }
}

// Packs, for every vertex, the (f1, f2) of its 2d edges in direction order into one
// record (f1 = 0 where the edge is absent or leaves the box).  Built once per upload.
template <typename W>
__global__ void k_build_records(const W *f1, const W *f2, long long V, int d, long long s0, long long s1, long long s2,
                                long long s3, long long n0, long long n1, long long n2, long long n3, unsigned char *rec,
                                int rec_bytes)
{
    const long long st[4] = {s0, s1, s2, s3}, n[4] = {n0, n1, n2, n3};
    const int per = rec_bytes / (int)sizeof(W);
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < V; v += (long long)gridDim.x * blockDim.x) {
        W *out = reinterpret_cast<W *>(rec + v * rec_bytes);
        for (int i = 0; i < per; i++) out[i] = 0;
        for (int dir = 0; dir < 2 * d; dir++) {
            const int k = dir >> 1;
            const long long ck = (v / st[k]) % n[k];
            long long slot = -1;
            if (!(dir & 1) && ck + 1 < n[k]) slot = k * V + v;
            if ((dir & 1) && ck > 0) slot = k * V + v - st[k];
            if (slot < 0 || f1[slot] == 0) continue;
            out[2 * dir] = f1[slot];
            out[2 * dir + 1] = f2[slot];
        }
    }
}


// Weight statistics of the (upper-face-zeroed) travel times: out[0] = sum of f1 over the
// directed edges (both directions of each edge: the most flows that can be in flight),
// out[1] = directed edges, out[2] = the largest f1.
template <typename W>
__global__ void k_flow_bound(const W *f1, long long n, unsigned long long *out)
{
    unsigned long long s = 0, c = 0;
    unsigned int mx = 0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const unsigned int f = f1[i];
        s += f;
        c += f != 0;
        mx = max(mx, f);
    }
    for (int o = 16; o > 0; o >>= 1) {
        s += __shfl_xor_sync(0xffffffffu, s, o);
        c += __shfl_xor_sync(0xffffffffu, c, o);
        mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    }
    if ((threadIdx.x & 31) == 0) {
        if (s) atomicAdd(out, 2ull * s);
        if (c) atomicAdd(out + 1, 2ull * c);
        if (mx) atomicMax(out + 2, (unsigned long long)mx);
    }
}

// Resets the control block for a new solve.
__global__ void k_reset(Control *ctl)
{
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        ctl->bar = 0;
        ctl->err = 0;
        ctl->status_in = 0;
        for (int i = 0; i < NRELEASE; i++) ctl->release[i].epoch = 0;
        for (int b = 0; b < 2; b++) {
            Counters &c = ctl->cnt[b];
            c.out_cand = c.live = c.lau_imp = c.xkey = 0;
            c.n_active = c.overflow = c.abort = c.chunks = 0;
            c.min_ta = INT_MAX;
        }
        for (int i = 0; i < R_COUNT; i++) ctl->out[i] = 0;
    }
}

// Marks B in the bitmap; out-of-range ids make the solve invalid.
__global__ void k_mark_B(const int64_t *B, long long nB, uint32_t *isB, long long V, Control *ctl)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nB; i += (long long)gridDim.x * blockDim.x) {
        const long long b = B[i];
        if (b < 0 || b >= V) atomicExch(&ctl->status_in, ST_INVALID);
        else atomicOr(isB + (b >> 5), 1u << (b & 31));
    }
}

// Vertices outside the graph G' of a reconstruction step (Section 1): their label and
// offer are set to 2^31 - 1, which no water can beat, so no flow is ever launched into
// them and they never launch one.  A removed vertex in B is an invalid request.
__global__ void k_mark_removed(const int64_t *R, long long nR, const uint32_t *isB, long long V, int32_t *label,
                               unsigned long long *offer, Control *ctl)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nR; i += (long long)gridDim.x * blockDim.x) {
        const long long r = R[i];
        if (r < 0 || r >= V || ((isB[r >> 5] >> (r & 31)) & 1u)) {
            atomicExch(&ctl->status_in, ST_INVALID);
            continue;
        }
        label[r] = INT_MAX;
        offer[r] = 0x7fffffffffffffffull;
    }
}

// Initialization (Algorithm 3): Label(a) = M for a in A (the offer word mirrors it);
// each distinct source is listed once (in the candidate list) for the seed launch.
__global__ void k_mark_A(const int64_t *A, long long nA, const uint32_t *isB, long long V, int M, int32_t *label,
                         unsigned long long *offer, uint32_t *src_list, Control *ctl)
{
    const unsigned long long key = ((unsigned long long)(uint32_t)M << 32) | 0xffffffffull;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nA; i += (long long)gridDim.x * blockDim.x) {
        const long long a = A[i];
        if (a < 0 || a >= V) {
            atomicExch(&ctl->status_in, ST_INVALID);
            continue;
        }
        if (((isB[a >> 5] >> (a & 31)) & 1u) || label[a] == INT_MAX) {
            atomicExch(&ctl->status_in, ST_INVALID);  // A and B must be disjoint; A must be in the graph
            continue;
        }
        label[a] = M;
        if (atomicExch(offer + a, key) != key) src_list[hi32(atomicAdd(&ctl->cnt[0].out_cand, 1ull << 32))] = (uint32_t)a;
    }
}

// Path reconstruction from an improvement record (one CTA).  A walk that reaches X at
// time F1 with the solve's answer entered X along x = (Y, dir); the flow on x left Y at
// t_Y = F1 - f1(x), when Y improved, so Y's improvement at t_Y names the edge that
// entered Y, and so on back to a source of A (time 0).  The improvement at t_Y is Y's
// first one when first_t[Y] = t_Y; otherwise it is looked up in the log segment of the
// pass run at t_Y (a vertex improves at most once per pass).  This is the path repeated
// application (Section 1) finds: earlier vertices on it never reach later ones sooner
// with better water, so removing them changes nothing.
// out[0] = path length (X first), out[1] = status (0, or CSP_ERR_CAPACITY if a needed log
// record was dropped, or CSP_ERR_CUDA if the record is inconsistent).
template <typename W>
__global__ void k_backtrack(const unsigned char *rec, int rec_bytes, int nslot, long long V, long long X, long long F1,
                            uint32_t code0, const int32_t *first_t, const uint32_t *first_code, const uint2 *log,
                            unsigned long long log_cap, const int32_t *pass_time, const unsigned long long *pass_off,
                            long long n_pass, long long *path, long long cap, long long *out)
{
    __shared__ long long s_v, s_t, s_n;
    __shared__ unsigned long long s_lo, s_hi;
    __shared__ uint32_t s_code;
    __shared__ int s_mode, s_status, s_found;
    if (threadIdx.x == 0) {
        s_v = X;
        s_t = F1;
        s_code = code0;
        s_n = 1;
        if (cap > 0) path[0] = X;
        s_status = ST_CUDA;  // until the walk reaches A
    }
    __syncthreads();
    for (long long step = 0; step <= F1; step++) {
        if (threadIdx.x == 0) {
            s_mode = 0;  // 0: next step, 1: scan the log, 2: stop
            const uint32_t sd = 0xffffffffu - s_code;
            const long long src = sd >> 3;
            const int dir = (int)(sd & 7u);
            // f1 of x from the edge record of its source (0: no such edge)
            const long long f =
                (src < V && dir < nslot) ? (long long)reinterpret_cast<const W *>(rec + src * rec_bytes)[2 * dir] : 0;
            const long long ty = s_t - f;
            if (s_n < cap) path[s_n] = src;
            s_n++;
            if (f <= 0 || ty < 0) {
                s_mode = 2;  // inconsistent record
            } else if (ty == 0) {
                s_status = ST_OK;  // src is a source: water leaves A at time 0 only
                s_mode = 2;
            } else if (__ldcg(first_t + src) == (int32_t)ty) {
                s_code = __ldcg(first_code + src);
                s_v = src;
                s_t = ty;
            } else {
                long long a = 1, b = n_pass;  // pass_time[1 .. n_pass] increases
                while (a < b) {
                    const long long m = (a + b) / 2;
                    if (__ldcg(pass_time + m) < ty) a = m + 1;
                    else b = m;
                }
                if (n_pass < 1 || __ldcg(pass_time + a) != (int32_t)ty) {
                    s_mode = 2;
                } else {
                    s_lo = __ldcg(pass_off + a);
                    s_hi = __ldcg(pass_off + a + 1);
                    if (s_hi > log_cap) {
                        s_status = ST_CAPACITY;
                        s_mode = 2;
                    } else {
                        s_v = src;
                        s_t = ty;
                        s_found = 0;
                        s_mode = 1;
                    }
                }
            }
        }
        __syncthreads();
        if (s_mode == 2) break;
        if (s_mode == 1) {
            for (unsigned long long i = s_lo + threadIdx.x; i < s_hi; i += blockDim.x) {
                const uint2 r = log[i];
                if ((long long)r.x == s_v) {
                    s_code = r.y;
                    s_found = 1;
                }
            }
            __syncthreads();
            if (!s_found) break;  // (uniform: read after the barrier) inconsistent record
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        out[0] = s_n;
        out[1] = s_status;
    }
}

// ---------------------------------------------------------------- the persistent kernel

template <int D, typename W, bool TRACE>
__global__ void __launch_bounds__(TPB, CSP_MIN_CTAS_PER_SM) k_cycle(Params<W> P)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    Smem &sm = *reinterpret_cast<Smem *>(smem_raw);
    init_stage_barriers(sm);
    uint32_t parity[NSTAGE] = {};
    unsigned long long epoch = 0;
    run_solve<D, W, TRACE>(P, Group{blockIdx.x, gridDim.x}, sm, parity, epoch);
}

// ---------------------------------------------------------------- host side

int num_sms(int device)
{
    int n = 0;
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, device);
    return n > 0 ? n : 1;
}

namespace {

template <int D, typename W, bool TRACE>
const void *kernel_ptr()
{
    return (const void *)&k_cycle<D, W, TRACE>;
}

template <typename W, bool TRACE>
const void *pick_kernel_w(int d)
{
    switch (d) {
    case 1: return kernel_ptr<1, W, TRACE>();
    case 2: return kernel_ptr<2, W, TRACE>();
    case 3: return kernel_ptr<3, W, TRACE>();
    case GRAPH: return kernel_ptr<GRAPH, W, TRACE>();
    default: return kernel_ptr<4, W, TRACE>();
    }
}

const void *pick_kernel(int d, int wbytes, bool trace)
{
    if (wbytes == 1) return trace ? pick_kernel_w<uint8_t, true>(d) : pick_kernel_w<uint8_t, false>(d);
    return trace ? pick_kernel_w<uint16_t, true>(d) : pick_kernel_w<uint16_t, false>(d);
}

constexpr size_t kSmem = sizeof(Smem);


csp_status ensure_workspace(csp_lattice *L, int64_t pool_cap, int64_t sets_cap)
{
    if (L->ws && pool_cap <= L->pool_cap && sets_cap <= L->sets_cap) return CSP_OK;
    pool_cap = std::max<int64_t>(pool_cap, L->pool_cap);
    sets_cap = std::max<int64_t>(sets_cap, L->sets_cap);
    if (pool_cap > 0xF0000000ll) pool_cap = 0xF0000000ll;
    pool_cap = (pool_cap + TILE - 1) / TILE * TILE;  // whole chunks
    const int64_t V = L->V;
    const int64_t trace_cap = L->trace_cap ? L->trace_cap : 1 << 16;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o = off;
        off = align_up(off + bytes, 256);
        return o;
    };
    // candidates: one region per CTA of at least (pool / CTAs + TILE) entries, so that no CTA
    // can run out of room (a CTA lists at most the flows of its ceil(chunks / CTAs) chunks)
    const int64_t cand_cap = std::max<int64_t>(V, pool_cap + (int64_t)max_group_ctas(L->device) * TILE);
    const size_t o_label = take(V * 4), o_offer = take(V * 8), o_isB = take(((V + 31) / 32) * 4),
                 o_stamp = take(((V + 3) / 4) * 16), o_estamp = take((size_t)nslots(L->d) * V * 4), o_cand = take(cand_cap * 4), o_ctl = take(sizeof(Control)),
                 o_trace = take(trace_cap * 24), o_sets = take(sets_cap * 8);
    size_t o_pool[2][3], o_fill[2];
    for (int b = 0; b < 2; b++) {
        for (int f = 0; f < 3; f++) o_pool[b][f] = take((pool_cap + POOL_PAD) * 4);
        o_fill[b] = take((pool_cap / TILE + 1) * 4);
    }
    void *ws = nullptr;
    cudaError_t e = cudaMalloc(&ws, off);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return cuda_fail(e, "cudaMalloc(workspace)");
    }
    if (L->ws) cudaFree(L->ws);
    L->ws = ws;
    L->ws_bytes = off;
    char *b = (char *)ws;
    L->label = (int32_t *)(b + o_label);
    L->offer = (unsigned long long *)(b + o_offer);
    L->isB = (uint32_t *)(b + o_isB);
    L->src_stamp = (uint32_t *)(b + o_stamp);
    L->edge_stamp = (uint32_t *)(b + o_estamp);
    L->cand = (uint32_t *)(b + o_cand);
    L->cand_cap = cand_cap;
    L->ctl = (Control *)(b + o_ctl);
    L->trace = (long long *)(b + o_trace);
    L->trace_cap = trace_cap;
    L->sets = (int64_t *)(b + o_sets);
    L->sets_cap = sets_cap;
    for (int k = 0; k < 2; k++) {
        L->ed[k] = (uint32_t *)(b + o_pool[k][0]);
        L->qa[k] = (int32_t *)(b + o_pool[k][1]);
        L->ta[k] = (int32_t *)(b + o_pool[k][2]);
        L->fill[k] = (uint32_t *)(b + o_fill[k]);
    }
    L->pool_cap = pool_cap;
    CSP_CUDA(cudaMemset(L->ctl, 0, sizeof(Control)));
    return CSP_OK;
}

int64_t default_pool_cap(const csp_lattice *L)
{
    const int64_t want = std::max<int64_t>(1 << 20, 16 * L->V);
    return (int64_t)std::min<unsigned long long>((unsigned long long)want, std::max(L->flow_bound, 1024ull)) +
           chunk_slack(max_group_ctas(L->device));
}


// The default form of the cycle loop for a handle.  The event form visits a flow when it
// starts, arrives or is removed; the sweep visits every flow in flight in every cycle, so
// the event form pays off when flows stay in flight over many cycles: measured on one
// GB300 (1024^2 lattices, f2 ~ U{1..16}, M = 12288), 0.81x the sweep's speed at a mean
// travel time of 32.5 (f1 ~ U{1..64}), 1.04x at 64.5, 1.12x at 96, 1.18x at 128 and 1.21x
// at 256 (f1 up to 511); 0.34x on the 128^3 cube (f1 ~ U{1..16}) and 0.27-0.77x on the
// anti-correlated lattices (geometric f1, mean 10).  Its per-edge queues are larger than the
// sweep's flow pool, so where cycles are dense it spends its time on random accesses that
// miss L2.  Rule: the event form when the mean f1 over directed edges is at least
// kEventMeanF1 (just above the crossover, near 59) and it supports the handle.
constexpr unsigned long long kEventMeanF1 = 64;

bool event_preferred(const csp_lattice *L)
{
    return L->n_arcs > 0 && L->max_f1 + 1 <= (unsigned int)EV_WMAX && L->flow_bound < 0xFFFFFF00ull &&
           L->flow_bound >= kEventMeanF1 * L->n_arcs;
}

// Which form of the cycle loop runs a solve: CSP_OPT_SWEEP or CSP_OPT_EVENT choose one;
// without either, event_preferred decides.  Preparing the event form (edge records, once
// per weight upload) synchronises the stream.
csp_status pick_engine(csp_lattice *L, const csp_options *opt, cudaStream_t s, bool *event)
{
    const int f = opt ? opt->flags : 0;
    *event = false;
    if ((f & CSP_OPT_SWEEP) && (f & CSP_OPT_EVENT)) {
        set_error("CSP_OPT_SWEEP and CSP_OPT_EVENT are exclusive");
        return CSP_ERR_INVALID;
    }
    if ((f & CSP_OPT_SWEEP) || (!(f & CSP_OPT_EVENT) && !event_preferred(L))) return CSP_OK;
    csp_status st = event_prepare(L, s);
    if (st != CSP_OK) return st;
    if (!event_supported(L)) {
        if (f & CSP_OPT_EVENT) {
            set_error("the event form needs max f1 <= 511");
            return CSP_ERR_INVALID;
        }
        return CSP_OK;
    }
    *event = true;
    return CSP_OK;
}

// Enqueues one solve (set-up kernels + persistent kernel) on stream s.
csp_status enqueue_solve(csp_lattice *L, const int64_t *A_dev, int64_t nA, const int64_t *B_dev, int64_t nB, int64_t M,
                         const csp_options *opt, long long *trace_dev, int64_t trace_cap, int64_t *result_dev,
                         cudaStream_t s, const int64_t *R_dev = nullptr, int64_t nR = 0, const ReconLog *rl = nullptr)
{
    const int64_t V = L->V;
    if (rl && rl->log_n) CSP_CUDA(cudaMemsetAsync(rl->log_n, 0, sizeof(unsigned long long), s));
    CSP_CUDA(cudaMemsetAsync(L->label, 0, V * 4, s));
    CSP_CUDA(cudaMemsetAsync(L->offer, 0, V * 8, s));
    CSP_CUDA(cudaMemsetAsync(L->isB, 0, ((V + 31) / 32) * 4, s));
    const bool phantoms = trace_dev && opt && (opt->flags & CSP_OPT_PHANTOMS);
    if (trace_dev) CSP_CUDA(cudaMemsetAsync(L->src_stamp, 0, ((V + 3) / 4) * 16, s));  // stamps are pass numbers >= 1
    if (phantoms) CSP_CUDA(cudaMemsetAsync(L->edge_stamp, 0, (size_t)nslots(L->d) * V * 4, s));
    const int sms = num_sms(L->device);
    k_reset<<<1, 32, 0, s>>>(L->ctl);
    k_mark_B<<<std::max<int64_t>(1, std::min<int64_t>(sms * 4, (nB + 255) / 256)), 256, 0, s>>>(B_dev, nB, L->isB, V,
                                                                                                 L->ctl);
    if (nR > 0)
        k_mark_removed<<<std::max<int64_t>(1, std::min<int64_t>(sms * 4, (nR + 255) / 256)), 256, 0, s>>>(
            R_dev, nR, L->isB, V, L->label, L->offer, L->ctl);
    k_mark_A<<<std::max<int64_t>(1, std::min<int64_t>(sms * 4, (nA + 255) / 256)), 256, 0, s>>>(
        A_dev, nA, L->isB, V, (int)M, L->label, L->offer, L->cand, L->ctl);
    CSP_CUDA(cudaGetLastError());

    const bool trace = trace_dev != nullptr;
    bool event = false;
    csp_status est = pick_engine(L, opt, s, &event);
    if (est != CSP_OK) return est;
    const void *fn = pick_kernel(L->d, L->wbytes, trace);
    int max_ctas = 0;
    if (event) {
        est = event_reserve(L, L->pool_cap);
        if (est != CSP_OK) return est;
        est = event_max_ctas(L, trace, &max_ctas);
        if (est != CSP_OK) return est;
    } else {
        static thread_local bool attr_set[2][2][GRAPH + 1] = {};
        bool &done = attr_set[L->wbytes - 1][trace][L->d];
        if (!done) {
            CSP_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmem));
            done = true;
        }
        int per_sm = 0;
        CSP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, TPB, kSmem));
        if (per_sm < 1) {
            g_last_error = "persistent kernel does not fit on an SM";
            return CSP_ERR_CUDA;
        }
        max_ctas = std::min(per_sm * sms, max_group_ctas(L->device));
    }
    int ctas = opt && opt->ctas > 0 ? opt->ctas : (int)std::min<int64_t>(max_ctas, std::max<int64_t>(1, V / 4096));
    ctas = std::max(1, std::min(ctas, max_ctas));

    Params<uint8_t> P8{};
    Params<uint16_t> P16{};
    auto fill = [&](auto &P) {
        using W = std::remove_cv_t<std::remove_pointer_t<decltype(P.f1)>>;
        P.f1 = (const W *)L->f1;
        P.f2 = (const W *)L->f2;
        P.rec = (const uint4 *)L->rec;
        P.V = V;
        for (int k = 0; k < 4; k++) P.stride[k] = L->stride[k];
        P.nbw = L->nbw;
        P.nbw_in = L->nbw_in;
        P.label = L->label;
        P.offer = L->offer;
        P.isB = L->isB;
        P.src_stamp = L->src_stamp;
        P.edge_stamp = phantoms ? L->edge_stamp : nullptr;
        P.cand = L->cand;
        P.cand_cap = (unsigned int)L->cand_cap;
        for (int b = 0; b < 2; b++) {
            P.ed[b] = L->ed[b];
            P.qa[b] = L->qa[b];
            P.ta[b] = L->ta[b];
            P.pk[b] = packed_pool(L->qa[b], L->ta[b], L->pool_cap);
            P.fill[b] = L->fill[b];
        }
        P.max_f1 = L->max_f1;
        P.pool_cap = (unsigned int)L->pool_cap;
        P.ctl = L->ctl;
        P.trace = trace_dev;
        P.trace_cap = trace_cap;
        P.result_dev = (long long *)result_dev;
        P.M = (int)M;
        P.max_cycles = opt ? opt->max_cycles : 0;
        P.budget_ns = 1000000000ull * (unsigned long long)(opt && opt->time_limit_s > 0 ? opt->time_limit_s : 120);
        P.barrier_ns = opt && opt->barrier_us > 0 ? 1000ull * (unsigned long long)opt->barrier_us
                                                  : 4000000000ull;  // one barrier round never takes seconds
        P.test_absent = opt && (opt->flags & CSP_OPT_TEST_ABSENT_CTA) ? 1 : 0;
        if (rl) {
            P.first_t = rl->first_t;
            P.first_code = rl->first_code;
            P.log = rl->log;
            P.log_cap = rl->log_cap;
            P.log_n = rl->log_n;
            P.pass_time = rl->pass_time;
            P.pass_off = rl->pass_off;
            P.pass_cap = rl->pass_cap;
        }
    };
    void *args[1];
    if (L->wbytes == 1) {
        fill(P8);
        args[0] = &P8;
    } else {
        fill(P16);
        args[0] = &P16;
    }
    if (event) return event_launch(L, args[0], trace, ctas, opt, s);
    if (opt && opt->ev_begin) CSP_CUDA(cudaEventRecord((cudaEvent_t)opt->ev_begin, s));
    CSP_CUDA(cudaLaunchCooperativeKernel(fn, dim3(ctas), dim3(TPB), args, kSmem, s));
    if (opt && opt->ev_end) CSP_CUDA(cudaEventRecord((cudaEvent_t)opt->ev_end, s));
    return CSP_OK;
}

csp_status check_sets_host(const csp_lattice *L, const int64_t *A, int64_t nA, const int64_t *B, int64_t nB)
{
    if (!A || !B || nA < 1 || nB < 1) return CSP_ERR_INVALID;
    std::vector<int64_t> a(A, A + nA), b(B, B + nB);
    std::sort(a.begin(), a.end());
    std::sort(b.begin(), b.end());
    if (a.front() < 0 || a.back() >= L->V || b.front() < 0 || b.back() >= L->V) return CSP_ERR_INVALID;
    size_t i = 0, j = 0;
    while (i < a.size() && j < b.size()) {
        if (a[i] == b[j]) return CSP_ERR_INVALID;  // A and B must be disjoint
        if (a[i] < b[j]) i++;
        else j++;
    }
    return CSP_OK;
}

}  // namespace

// ---------------------------------------------------------------- C ABI

static csp_status solve_host(csp_lattice *L, const int64_t *A, int64_t nA, const int64_t *B, int64_t nB, int64_t M,
                             const csp_options *opt, csp_result *out, int64_t *trace, int64_t trace_cap,
                             int64_t *trace_len, const int64_t *R, int64_t nR, const ReconLog *rl = nullptr);

extern "C" {

const char *csp_status_string(csp_status s)
{
    switch (s) {
    case CSP_OK: return "ok";
    case CSP_ERR_INVALID: return "invalid argument";
    case CSP_ERR_OOM: return "out of memory";
    case CSP_ERR_CUDA: return "CUDA error";
    case CSP_ERR_CAPACITY: return "flow pool capacity exceeded";
    case CSP_ERR_TIMEOUT: return "cycle limit reached";
    case CSP_ERR_BARRIER: return "device barrier timed out";
    }
    return "unknown status";
}

const char *csp_last_error(void) { return g_last_error.c_str(); }

csp_status csp_create_lattice(int d, const int64_t *extents, const void *f1, const void *f2, int weight_bytes,
                              int on_device, void *stream, csp_lattice **out)
{
    if (!out || !extents || !f1 || !f2 || d < 1 || d > 4 || (weight_bytes != 1 && weight_bytes != 2))
        return CSP_ERR_INVALID;
    *out = nullptr;
    int64_t V = 1;
    for (int k = 0; k < d; k++) {
        if (extents[k] < 1 || extents[k] >= (1ll << 28)) return CSP_ERR_INVALID;
        V *= extents[k];
        if (V >= (1ll << 28)) return CSP_ERR_INVALID;
    }
    csp_lattice *L = new (std::nothrow) csp_lattice();
    if (!L) return CSP_ERR_OOM;
    L->d = d;
    L->wbytes = weight_bytes;
    L->V = V;
    int64_t s = 1;
    for (int k = 0; k < d; k++) {
        L->ext[k] = extents[k];
        L->stride[k] = (int)s;
        s *= extents[k];
    }
    cudaGetDevice(&L->device);
    const size_t bytes = (size_t)d * V * weight_bytes;
    L->rec_bytes = record_bytes(d, weight_bytes);
    cudaError_t e = cudaMalloc(&L->f1, bytes);
    if (e == cudaSuccess) e = cudaMalloc(&L->f2, bytes);
    if (e == cudaSuccess) e = cudaMalloc(&L->rec, (size_t)V * L->rec_bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        csp_destroy_lattice(L);
        return cuda_fail(e, "cudaMalloc(lattice)");
    }
    csp_status st = csp_upload_weights(L, f1, f2, on_device, stream);
    if (st != CSP_OK) {
        csp_destroy_lattice(L);
        return st;
    }
    *out = L;
    return CSP_OK;
}

}  // extern "C"

namespace {

// Builds the device form of a general graph: per-vertex edge records (weights by out-slot),
// the out-edge table nbw (head << 3 | in-slot at the head) and, for a directed graph, the
// in-edge table nbw_in (tail << 3 | out-slot at the tail; in-slots numbered by (tail, out-slot)).
// An undirected graph lists each edge at both ends; the slot at the other end is the
// in-slot, so one table serves both.  Every id is checked here, so the kernels index only
// valid vertices.
csp_status create_graph(int64_t V, int32_t slots, const int64_t *nbr, const void *f1, const void *f2, int weight_bytes,
                        void *stream, bool directed, csp_lattice **out)
{
    const char *fn = directed ? "csp_create_digraph" : "csp_create_graph";
    if (!out || !nbr || !f1 || !f2 || V < 1 || V >= (1ll << 28) || slots < 1 || slots > 8 ||
        (weight_bytes != 1 && weight_bytes != 2))
        return CSP_ERR_INVALID;
    *out = nullptr;
    auto w1 = [&](int64_t i) -> int64_t {
        return weight_bytes == 1 ? ((const uint8_t *)f1)[i] : ((const uint16_t *)f1)[i];
    };
    auto w2 = [&](int64_t i) -> int64_t {
        return weight_bytes == 1 ? ((const uint8_t *)f2)[i] : ((const uint16_t *)f2)[i];
    };
    const int rb = record_bytes(GRAPH, weight_bytes);
    std::vector<uint32_t> nbw((size_t)V * 8), nbw_in(directed ? (size_t)V * 8 : 0);
    std::vector<uint8_t> indeg(directed ? (size_t)V : 0, 0);
    std::vector<unsigned char> rec((size_t)V * rb, 0);
    unsigned long long bound = 0, arcs = 0, maxf1 = 0;
    for (int64_t v = 0; v < V; v++)
        for (int j = 0; j < 8; j++) {  // empty slots: v itself (f1 = 0, never followed)
            nbw[(size_t)v * 8 + j] = (uint32_t)v << 3;
            if (directed) nbw_in[(size_t)v * 8 + j] = (uint32_t)v << 3;
        }
    for (int64_t v = 0; v < V; v++) {
        for (int j = 0; j < slots; j++) {
            const int64_t i = v * slots + j, u = nbr[i];
            if (u == -1) continue;
            const char *why = nullptr;
            int back = -1;
            if (u < 0 || u >= V) why = "neighbour id out of range";
            else if (u == v) why = "self loop";
            else if (w1(i) < 1) why = "travel time below 1";
            for (int k = 0; k < j && !why; k++)
                if (nbr[v * slots + k] == u) why = "parallel edge";
            if (!why && directed) {
                back = indeg[u]++;
                if (back >= 8) why = "in-degree above 8";
            } else if (!why) {
                for (int k = 0; k < slots && !why; k++)
                    if (nbr[u * slots + k] == v) {
                        if (w1(u * slots + k) != w1(i) || w2(u * slots + k) != w2(i)) why = "weights differ at the two ends";
                        back = k;
                    }
                if (!why && back < 0) why = "edge missing at its other end";
            }
            if (why) {
                set_error(std::string(fn) + ": vertex " + std::to_string(v) + " slot " + std::to_string(j) + ": " + why);
                return CSP_ERR_INVALID;
            }
            nbw[(size_t)v * 8 + j] = ((uint32_t)u << 3) | (uint32_t)back;
            if (directed) nbw_in[(size_t)u * 8 + back] = ((uint32_t)v << 3) | (uint32_t)j;
            unsigned char *r = rec.data() + (size_t)v * rb;
            if (weight_bytes == 1) {
                r[2 * j] = (uint8_t)w1(i);
                r[2 * j + 1] = (uint8_t)w2(i);
            } else {
                ((uint16_t *)r)[2 * j] = (uint16_t)w1(i);
                ((uint16_t *)r)[2 * j + 1] = (uint16_t)w2(i);
            }
            bound += (unsigned long long)w1(i);
            arcs++;
            maxf1 = std::max<unsigned long long>(maxf1, (unsigned long long)w1(i));
        }
    }
    csp_lattice *L = new (std::nothrow) csp_lattice();
    if (!L) return CSP_ERR_OOM;
    L->d = GRAPH;
    L->wbytes = weight_bytes;
    L->V = V;
    L->ext[0] = V;
    L->rec_bytes = rb;
    L->flow_bound = bound;
    L->n_arcs = arcs;
    L->max_f1 = (unsigned int)maxf1;
    cudaGetDevice(&L->device);
    cudaError_t e = cudaMalloc(&L->rec, rec.size());
    if (e == cudaSuccess) e = cudaMalloc((void **)&L->nbw, nbw.size() * 4);
    if (e == cudaSuccess && directed) e = cudaMalloc((void **)&L->nbw_in, nbw_in.size() * 4);
    if (!directed) L->nbw_in = L->nbw;
    cudaStream_t s = (cudaStream_t)stream;
    if (e == cudaSuccess) e = cudaMemcpyAsync(L->rec, rec.data(), rec.size(), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(L->nbw, nbw.data(), nbw.size() * 4, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && directed)
        e = cudaMemcpyAsync(L->nbw_in, nbw_in.data(), nbw_in.size() * 4, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        csp_destroy_lattice(L);
        return cuda_fail(e, fn);
    }
    *out = L;
    return CSP_OK;
}

}  // namespace

extern "C" {

csp_status csp_create_graph(int64_t V, int32_t slots, const int64_t *nbr, const void *f1, const void *f2,
                            int weight_bytes, void *stream, csp_lattice **out)
{
    return create_graph(V, slots, nbr, f1, f2, weight_bytes, stream, false, out);
}

csp_status csp_create_digraph(int64_t V, int32_t slots, const int64_t *nbr, const void *f1, const void *f2,
                              int weight_bytes, void *stream, csp_lattice **out)
{
    return create_graph(V, slots, nbr, f1, f2, weight_bytes, stream, true, out);
}

csp_status csp_upload_weights(csp_lattice *L, const void *f1, const void *f2, int on_device, void *stream)
{
    if (!L || !f1 || !f2 || L->d == GRAPH) return CSP_ERR_INVALID;
    cudaStream_t s = (cudaStream_t)stream;
    const size_t bytes = (size_t)L->d * L->V * L->wbytes;
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    event_invalidate(L);
    CSP_CUDA(cudaMemcpyAsync(L->f1, f1, bytes, kind, s));
    CSP_CUDA(cudaMemcpyAsync(L->f2, f2, bytes, kind, s));
    const long long n[4] = {L->ext[0], L->ext[1], L->ext[2], L->ext[3]};
    const long long st[4] = {L->stride[0], L->stride[1], L->stride[2], L->stride[3]};
    const int blocks = std::max<int64_t>(1, std::min<int64_t>(4096, (L->d * L->V + 255) / 256));
    unsigned long long *bound = nullptr;
    CSP_CUDA(cudaMallocAsync((void **)&bound, 3 * sizeof(unsigned long long), s));
    CSP_CUDA(cudaMemsetAsync(bound, 0, 3 * sizeof(unsigned long long), s));
    if (L->wbytes == 1) {
        k_zero_upper_faces<uint8_t><<<blocks, 256, 0, s>>>((uint8_t *)L->f1, (uint8_t *)L->f2, L->V, L->d, st[0], st[1],
                                                           st[2], st[3], n[0], n[1], n[2], n[3]);
        k_flow_bound<uint8_t><<<blocks, 256, 0, s>>>((const uint8_t *)L->f1, L->d * L->V, bound);
        k_build_records<uint8_t><<<blocks, 256, 0, s>>>((const uint8_t *)L->f1, (const uint8_t *)L->f2, L->V, L->d,
                                                       st[0], st[1], st[2], st[3], n[0], n[1], n[2], n[3],
                                                       (unsigned char *)L->rec, L->rec_bytes);
    } else {
        k_zero_upper_faces<uint16_t><<<blocks, 256, 0, s>>>((uint16_t *)L->f1, (uint16_t *)L->f2, L->V, L->d, st[0],
                                                            st[1], st[2], st[3], n[0], n[1], n[2], n[3]);
        k_flow_bound<uint16_t><<<blocks, 256, 0, s>>>((const uint16_t *)L->f1, L->d * L->V, bound);
        k_build_records<uint16_t><<<blocks, 256, 0, s>>>((const uint16_t *)L->f1, (const uint16_t *)L->f2, L->V, L->d,
                                                        st[0], st[1], st[2], st[3], n[0], n[1], n[2], n[3],
                                                        (unsigned char *)L->rec, L->rec_bytes);
    }
    CSP_CUDA(cudaGetLastError());
    unsigned long long stats[3] = {0, 0, 0};
    CSP_CUDA(cudaMemcpyAsync(stats, bound, sizeof(stats), cudaMemcpyDeviceToHost, s));
    CSP_CUDA(cudaFreeAsync(bound, s));
    CSP_CUDA(cudaStreamSynchronize(s));
    L->flow_bound = stats[0];
    L->n_arcs = stats[1];
    L->max_f1 = (unsigned int)stats[2];
    return CSP_OK;
}

void csp_destroy_lattice(csp_lattice *L)
{
    if (!L) return;
    if (L->f1) cudaFree(L->f1);
    if (L->f2) cudaFree(L->f2);
    if (L->rec) cudaFree(L->rec);
    if (L->nbw_in && L->nbw_in != L->nbw) cudaFree(L->nbw_in);
    if (L->nbw) cudaFree(L->nbw);
    if (L->ws) cudaFree(L->ws);
    event_release(L);
    delete L;
}

int64_t csp_num_vertices(const csp_lattice *L) { return L ? L->V : -1; }

csp_status csp_reserve(csp_lattice *L, int64_t pool_capacity)
{
    if (!L || pool_capacity < 0) return CSP_ERR_INVALID;
    return ensure_workspace(L, pool_capacity ? pool_capacity : default_pool_cap(L), std::max<int64_t>(L->sets_cap, 1024));
}

csp_status csp_solve_async(csp_lattice *L, const int64_t *A_dev, int64_t nA, const int64_t *B_dev, int64_t nB,
                           int64_t M, const csp_options *opt, int64_t *result_dev, int64_t *trace_dev, int64_t trace_cap)
{
    if (!L || !A_dev || !B_dev || nA < 1 || nB < 1 || !result_dev || M >= (1ll << 31) - 1 || M < -(1ll << 31) + 1)
        return CSP_ERR_INVALID;
    if (trace_dev && trace_cap < 1) return CSP_ERR_INVALID;
    if (!L->ws) return CSP_ERR_INVALID;  // csp_reserve first
    cudaStream_t s = opt ? (cudaStream_t)opt->stream : nullptr;
    return enqueue_solve(L, A_dev, nA, B_dev, nB, M, opt, (long long *)trace_dev, trace_dev ? trace_cap : 0, result_dev,
                         s);
}

csp_status csp_solve(csp_lattice *L, const int64_t *A, int64_t nA, const int64_t *B, int64_t nB, int64_t M,
                     const csp_options *opt, csp_result *out, int64_t *trace, int64_t trace_cap, int64_t *trace_len)
{
    return solve_host(L, A, nA, B, nB, M, opt, out, trace, trace_cap, trace_len, nullptr, 0);
}

}  // extern "C"

// One synchronous solve with host arrays; R (nullable, nR ids) lists vertices removed
// from the graph (a reconstruction step).
static csp_status solve_host(csp_lattice *L, const int64_t *A, int64_t nA, const int64_t *B, int64_t nB, int64_t M,
                      const csp_options *opt, csp_result *out, int64_t *trace, int64_t trace_cap, int64_t *trace_len,
                      const int64_t *R, int64_t nR, const ReconLog *rl)
{
    if (!L || !out || M >= (1ll << 31) - 1 || M < -(1ll << 31) + 1) return CSP_ERR_INVALID;
    if (trace && trace_cap < 0) return CSP_ERR_INVALID;
    if (nR < 0 || (nR > 0 && !R)) return CSP_ERR_INVALID;
    csp_status st = check_sets_host(L, A, nA, B, nB);
    if (st != CSP_OK) return st;
    cudaStream_t s = opt ? (cudaStream_t)opt->stream : nullptr;
    int64_t cap = opt && opt->pool_capacity > 0 ? opt->pool_capacity : std::max<int64_t>(L->pool_cap, default_pool_cap(L));
    if (trace && trace_cap > L->trace_cap) {
        L->trace_cap = trace_cap;
        if (L->ws) {  // grow the device trace buffer with the workspace
            cudaFree(L->ws);
            L->ws = nullptr;
            L->pool_cap = 0;
            L->sets_cap = 0;
        }
    }
    for (int attempt = 0;; attempt++) {
        st = ensure_workspace(L, cap, nA + nB + nR);
        if (st != CSP_OK) return st;
        CSP_CUDA(cudaMemcpyAsync(L->sets, A, nA * 8, cudaMemcpyHostToDevice, s));
        CSP_CUDA(cudaMemcpyAsync(L->sets + nA, B, nB * 8, cudaMemcpyHostToDevice, s));
        if (nR > 0) CSP_CUDA(cudaMemcpyAsync(L->sets + nA + nB, R, nR * 8, cudaMemcpyHostToDevice, s));
        st = enqueue_solve(L, L->sets, nA, L->sets + nA, nB, M, opt, trace ? L->trace : nullptr,
                           trace ? L->trace_cap : 0, nullptr, s, nR > 0 ? L->sets + nA + nB : nullptr, nR, rl);
        if (st != CSP_OK) return st;
        long long o[R_COUNT];
        CSP_CUDA(cudaMemcpyAsync(o, (char *)L->ctl + offsetof(Control, out), sizeof(o), cudaMemcpyDeviceToHost, s));
        CSP_CUDA(cudaStreamSynchronize(s));
        const int64_t most = (int64_t)std::max(L->flow_bound, 1024ull) + chunk_slack(max_group_ctas(L->device));
        if (o[R_STATUS] == ST_CAPACITY && L->pool_cap < most && L->pool_cap < 0xF0000000ll) {
            cap = std::min<int64_t>(2 * L->pool_cap, most);
            continue;  // grow the pool and run again
        }
        out->F1 = o[R_F1];
        out->X = o[R_X];
        out->x_src = o[R_XSRC];
        out->x_dir = o[R_XDIR];
        out->F2 = o[R_F2];
        out->cycles = o[R_CYCLES];
        out->updates = o[R_UPDATES];
        out->launched = o[R_LAUNCHED];
        out->passes = o[R_PASSES];
        out->max_pool = o[R_MAXPOOL];
        out->arrivals = o[R_ARRIVALS];
        out->improved = o[R_IMPROVED];
        out->phantoms = o[R_PHANTOMS];
        if (trace) {
            const int64_t rows = std::min<int64_t>(o[R_TRACELEN], trace_cap);
            if (rows > 0) CSP_CUDA(cudaMemcpy(trace, L->trace, rows * 24, cudaMemcpyDeviceToHost));
        }
        if (trace_len) *trace_len = trace ? o[R_TRACELEN] : 0;
        return (csp_status)o[R_STATUS];
    }
}

// Edge weight f2 of the edge leaving v in direction dir, from the device edge record.
static csp_status edge_f2(csp_lattice *L, int64_t v, int dir, int64_t *w2)
{
    unsigned char rec[32];
    CSP_CUDA(cudaMemcpy(rec, (const char *)L->rec + v * L->rec_bytes, L->rec_bytes, cudaMemcpyDeviceToHost));
    if (L->wbytes == 1) *w2 = rec[2 * dir + 1];
    else *w2 = ((const uint16_t *)rec)[2 * dir + 1];
    return CSP_OK;
}

extern "C" {

csp_status csp_reconstruct_path(csp_lattice *L, const int64_t *A, int64_t nA, const int64_t *B, int64_t nB, int64_t M,
                                const csp_result *res, int64_t *path, int64_t cap, int64_t *len)
{
    if (!L || !A || !B || nA < 1 || nB < 1 || !len || (cap > 0 && !path)) return CSP_ERR_INVALID;
    csp_result r{};
    csp_status st;
    if (res) {
        r = *res;
    } else {
        st = csp_solve(L, A, nA, B, nB, M, nullptr, &r, nullptr, 0, nullptr);
        if (st != CSP_OK) return st;
    }
    *len = 0;
    if (r.F1 < 0) return CSP_OK;  // infeasible: no path
    std::vector<int64_t> a(A, A + nA);
    std::sort(a.begin(), a.end());
    auto in_A = [&](int64_t v) { return std::binary_search(a.begin(), a.end(), v); };
    // V' = V minus (B and the path found so far); B' = {Y}; M' = F2 - f2(x) + 1 (strict bound)
    std::vector<int64_t> found{r.X};
    std::vector<int64_t> removed(B, B + nB);
    int64_t Y = r.x_src, dir = r.x_dir, F2 = r.F2;
    while (!in_A(Y)) {
        if ((int64_t)found.size() > L->V) return CSP_ERR_INVALID;  // cannot happen for a simple path
        int64_t w2 = 0;
        st = edge_f2(L, Y, (int)dir, &w2);
        if (st != CSP_OK) return st;
        removed.push_back(found.back());
        csp_result q{};
        st = solve_host(L, A, nA, &Y, 1, F2 - w2 + 1, nullptr, &q, nullptr, 0, nullptr, removed.data(),
                        (int64_t)removed.size());
        if (st != CSP_OK) return st;
        if (q.F1 < 0 || q.X != Y) {
            set_error("csp_reconstruct_path: a reconstruction step found no path");
            return CSP_ERR_INVALID;
        }
        found.push_back(Y);
        Y = q.x_src;
        dir = q.x_dir;
        F2 = q.F2;
    }
    found.push_back(Y);
    *len = (int64_t)found.size();
    if (*len > cap) return CSP_ERR_CAPACITY;
    for (int64_t i = 0; i < *len; i++) path[i] = found[*len - 1 - i];
    return CSP_OK;
}

csp_status csp_reconstruct_fast(csp_lattice *L, const int64_t *A, int64_t nA, const int64_t *B, int64_t nB, int64_t M,
                                const csp_options *opt, int64_t log_capacity, csp_result *res, int64_t *path,
                                int64_t cap, int64_t *len)
{
    if (!L || !A || !B || nA < 1 || nB < 1 || !len || !res || (cap > 0 && !path)) return CSP_ERR_INVALID;
    *len = 0;
    const int64_t V = L->V;
    const long long pass_cap = 1ll << 21;
    int64_t lc = 0;
    if (log_capacity > 0) {
        lc = log_capacity;
    } else if (log_capacity == 0) {
        size_t free_b = 0, total_b = 0;
        CSP_CUDA(cudaMemGetInfo(&free_b, &total_b));
        lc = (int64_t)std::min<size_t>(free_b / 4 / sizeof(uint2), 0xffffffffull);
    }
    // one allocation: first-improvement arrays, log counter, pass table, result words, log
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o = off;
        off = align_up(off + bytes, 256);
        return o;
    };
    const size_t o_ft = take(V * 4), o_fc = take(V * 4), o_n = take(8), o_pt = take((pass_cap + 1) * 4),
                 o_po = take((pass_cap + 2) * 8), o_out = take(16), o_path = take((size_t)std::max<int64_t>(cap, 1) * 8),
                 o_log = take((size_t)lc * sizeof(uint2));
    void *buf = nullptr;
    cudaError_t e = cudaMalloc(&buf, off);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return cuda_fail(e, "cudaMalloc(reconstruction record)");
    }
    char *b = (char *)buf;
    ReconLog rl;
    rl.first_t = (int32_t *)(b + o_ft);
    rl.first_code = (uint32_t *)(b + o_fc);
    rl.log = lc > 0 ? (uint2 *)(b + o_log) : nullptr;
    rl.log_cap = (unsigned long long)lc;
    rl.log_n = (unsigned long long *)(b + o_n);
    rl.pass_time = (int32_t *)(b + o_pt);
    rl.pass_off = (unsigned long long *)(b + o_po);
    rl.pass_cap = pass_cap;
    csp_status st = solve_host(L, A, nA, B, nB, M, opt, res, nullptr, 0, nullptr, nullptr, 0, &rl);
    if (st == CSP_OK && res->F1 >= 0) {
        cudaStream_t s = opt ? (cudaStream_t)opt->stream : nullptr;
        const long long n_pass = std::min<long long>(res->passes, pass_cap - 1);
        const uint32_t code0 = 0xffffffffu - (uint32_t)(res->x_src * 8 + res->x_dir);
        long long *dpath = (long long *)(b + o_path), *dout = (long long *)(b + o_out);
        if (L->wbytes == 1)
            k_backtrack<uint8_t><<<1, 512, 0, s>>>((const unsigned char *)L->rec, L->rec_bytes, nslots(L->d), V,
                                                   res->X, res->F1, code0, rl.first_t,
                                                   rl.first_code, rl.log, rl.log_cap, rl.pass_time, rl.pass_off, n_pass,
                                                   dpath, cap, dout);
        else
            k_backtrack<uint16_t><<<1, 512, 0, s>>>((const unsigned char *)L->rec, L->rec_bytes, nslots(L->d), V,
                                                    res->X, res->F1, code0, rl.first_t,
                                                    rl.first_code, rl.log, rl.log_cap, rl.pass_time, rl.pass_off,
                                                    n_pass, dpath, cap, dout);
        long long o[2] = {0, 0};
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaMemcpyAsync(o, dout, sizeof(o), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) {
            cudaFree(buf);
            return cuda_fail(e, "csp_reconstruct_fast");
        }
        *len = o[0];
        if (o[1] == ST_CAPACITY) {
            set_error("csp_reconstruct_fast: the improvement log was too small for this path");
            st = CSP_ERR_CAPACITY;
        } else if (o[1] != ST_OK) {
            set_error("csp_reconstruct_fast: inconsistent improvement record");
            st = CSP_ERR_CUDA;
        } else if (o[0] > cap) {
            st = CSP_ERR_CAPACITY;
        } else {
            std::vector<long long> h((size_t)o[0]);
            e = cudaMemcpy(h.data(), dpath, o[0] * 8, cudaMemcpyDeviceToHost);
            if (e != cudaSuccess) {
                cudaFree(buf);
                return cuda_fail(e, "csp_reconstruct_fast");
            }
            for (long long i = 0; i < o[0]; i++) path[i] = h[(size_t)(o[0] - 1 - i)];  // A end first
        }
    }
    cudaFree(buf);
    return st;
}

int32_t csp_default_engine(csp_lattice *L)
{
    if (!L) return -1;
    bool event = false;
    if (pick_engine(L, nullptr, nullptr, &event) != CSP_OK) return CSP_OPT_SWEEP;
    return event ? CSP_OPT_EVENT : CSP_OPT_SWEEP;
}

csp_status csp_event_phase_times(const csp_lattice *L, int64_t *ns)
{
    if (!L || !ns) return CSP_ERR_INVALID;
    unsigned long long t[4];
    const csp_status st = event_phase_times(L, t);
    if (st != CSP_OK) return st;
    for (int i = 0; i < 4; i++) ns[i] = (int64_t)t[i];
    return CSP_OK;
}

csp_status csp_get_labels(csp_lattice *L, int32_t *labels_host)
{
    if (!L || !labels_host || !L->ws) return CSP_ERR_INVALID;
    CSP_CUDA(cudaMemcpy(labels_host, L->label, L->V * 4, cudaMemcpyDeviceToHost));
    return CSP_OK;
}

}  // extern "C"

// ---------------------------------------------------------------- solve without allocation
//
// For callers that cannot allocate device memory (code running where cudaMalloc is not
// allowed, such as inside a memory-capped host process or a framework that owns all
// allocations).  The solver's scratch lives in one file-scope device array instead of a
// per-lattice workspace.  The array exists on every GPU that loads this library, for as
// long as the library stays loaded.  All calls share it, so calls whose work overlaps on
// the GPU (on different streams, or from different threads) race; a call clears what must
// start at zero (labels, offers, the B bitmap and the control block) before it starts.

namespace {

constexpr size_t kStaticBytes = (size_t)CSP_STATIC_WORKSPACE_BYTES;
static __device__ __align__(256) unsigned char g_static_ws[kStaticBytes];

constexpr int kMaxDevices = 64;
void *g_static_addr[kMaxDevices] = {};
std::mutex g_static_mutex;  // guards g_static_addr (calls may come from several host threads)

// Host code cannot use g_static_ws directly: on the host that name is only a stand-in.
// The device address is looked up once per device, with that device current, and kept
// for the life of the process (it does not survive a reset of the device's primary
// context, e.g. by cudaDeviceReset).
csp_status static_workspace_address(void **out)
{
    int dev = 0;
    CSP_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) {
        g_last_error = "csp_solve_static: device index out of range";
        return CSP_ERR_INVALID;
    }
    std::lock_guard<std::mutex> lock(g_static_mutex);
    if (!g_static_addr[dev]) {
        void *p = nullptr;
        CSP_CUDA(cudaGetSymbolAddress(&p, g_static_ws));
        g_static_addr[dev] = p;
    }
    *out = g_static_addr[dev];
    return CSP_OK;
}

// Flags a lattice whose upper-face travel times are not zero (the solver reads f1 = 0 as
// "no edge", and this entry point cannot zero them in a private copy).
template <typename W>
__global__ void k_check_upper_faces(const W *f1, long long V, int d, long long s0, long long s1, long long s2,
                                    long long s3, long long n0, long long n1, long long n2, long long n3, Control *ctl)
{
    const long long st[4] = {s0, s1, s2, s3}, n[4] = {n0, n1, n2, n3};
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < d * V;
         i += (long long)gridDim.x * blockDim.x) {
        const int k = (int)(i / V);
        const long long v = i - k * V;
        if ((v / st[k]) % n[k] == n[k] - 1 && f1[i] != 0) atomicExch(&ctl->status_in, ST_INVALID);
    }
}

}  // namespace

extern "C" csp_status csp_solve_static(int d, const int64_t *extents, const void *f1_dev, const void *f2_dev,
                                       int weight_bytes, const int64_t *A_dev, int64_t nA, const int64_t *B_dev,
                                       int64_t nB, int64_t M, int64_t max_cycles, void *stream, int64_t *result_dev)
{
    if (!extents || !f1_dev || !f2_dev || !A_dev || !B_dev || !result_dev || d < 1 || d > 4 ||
        (weight_bytes != 1 && weight_bytes != 2) || nA < 1 || nB < 1 || M >= (1ll << 31) - 1 || M < -(1ll << 31) + 1)
        return CSP_ERR_INVALID;
    int64_t V = 1, ext[4] = {1, 1, 1, 1};
    int stride[4] = {0, 0, 0, 0};
    for (int k = 0; k < d; k++) {
        if (extents[k] < 1 || extents[k] >= (1ll << 28)) return CSP_ERR_INVALID;
        ext[k] = extents[k];
        stride[k] = (int)V;
        V *= extents[k];
        if (V >= (1ll << 28)) return CSP_ERR_INVALID;
    }
    int dev = 0;
    CSP_CUDA(cudaGetDevice(&dev));
    const int sms = num_sms(dev);
    const void *fn = pick_kernel(d, weight_bytes, false);
    CSP_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmem));
    int per_sm = 0;
    CSP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, TPB, kSmem));
    if (per_sm < 1) {
        g_last_error = "persistent kernel does not fit on an SM";
        return CSP_ERR_CUDA;
    }
    const int ctas = (int)std::max<int64_t>(
        1, std::min<int64_t>(std::min<int64_t>((int64_t)per_sm * sms, max_group_ctas(dev)), V / 4096));
    // carve the static array: per-vertex arrays, control block, then the candidate list,
    // the two pool buffers and their chunk fill arrays (sized from what is left)
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o = off;
        off = align_up(off + bytes, 256);
        return o;
    };
    const int rbytes = record_bytes(d, weight_bytes);
    const size_t o_label = take(V * 4), o_offer = take(V * 8), o_isB = take(((V + 31) / 32) * 4),
                 o_rec = take(V * rbytes), o_ctl = take(sizeof(Control));
    // per pool slot: 6 words of the two buffers and one candidate word; candidates get
    // TILE more entries per CTA; 64 KiB of slack covers alignment, padding and fill arrays
    const size_t extra = (size_t)ctas * TILE * 4 + (64u << 10);
    size_t pool_cap = off + extra < kStaticBytes ? (kStaticBytes - off - extra) / 28 : 0;
    pool_cap = std::min<size_t>(pool_cap, 0xF0000000ull) / TILE * TILE;
    if (pool_cap < (size_t)TILE || pool_cap + (size_t)ctas * TILE < (size_t)V) {
        g_last_error = "csp_solve_static: lattice too large for the static workspace (" +
                       std::to_string(kStaticBytes >> 20) + " MiB)";
        return CSP_ERR_INVALID;
    }
    const int64_t cand_cap = (int64_t)pool_cap + (int64_t)ctas * TILE;
    const size_t o_cand = take(cand_cap * 4);
    size_t o_pool[2][3], o_fill[2];
    for (int b = 0; b < 2; b++) {
        for (int f = 0; f < 3; f++) o_pool[b][f] = take((pool_cap + POOL_PAD) * 4);
        o_fill[b] = take((pool_cap / TILE + 1) * 4);
    }
    if (off > kStaticBytes) {
        g_last_error = "csp_solve_static: workspace layout exceeds the static array";
        return CSP_ERR_INVALID;
    }
    void *base = nullptr;
    csp_status st = static_workspace_address(&base);
    if (st != CSP_OK) return st;
    char *b = (char *)base;
    int32_t *label = (int32_t *)(b + o_label);
    unsigned long long *offer = (unsigned long long *)(b + o_offer);
    uint32_t *isB = (uint32_t *)(b + o_isB);
    uint32_t *cand = (uint32_t *)(b + o_cand);
    Control *ctl = (Control *)(b + o_ctl);

    cudaStream_t s = (cudaStream_t)stream;
    CSP_CUDA(cudaMemsetAsync(label, 0, V * 4, s));
    CSP_CUDA(cudaMemsetAsync(offer, 0, V * 8, s));
    CSP_CUDA(cudaMemsetAsync(isB, 0, ((V + 31) / 32) * 4, s));
    CSP_CUDA(cudaMemsetAsync(ctl, 0, sizeof(Control), s));
    k_reset<<<1, 32, 0, s>>>(ctl);
    const long long n[4] = {ext[0], ext[1], ext[2], ext[3]};
    const long long stl[4] = {stride[0], stride[1], stride[2], stride[3]};
    const int cblocks = (int)std::max<int64_t>(1, std::min<int64_t>(sms * 4, (d * V + 255) / 256));
    if (weight_bytes == 1)
        k_check_upper_faces<uint8_t><<<cblocks, 256, 0, s>>>((const uint8_t *)f1_dev, V, d, stl[0], stl[1], stl[2],
                                                             stl[3], n[0], n[1], n[2], n[3], ctl);
    else
        k_check_upper_faces<uint16_t><<<cblocks, 256, 0, s>>>((const uint16_t *)f1_dev, V, d, stl[0], stl[1], stl[2],
                                                              stl[3], n[0], n[1], n[2], n[3], ctl);
    const int rblocks = (int)std::max<int64_t>(1, std::min<int64_t>(sms * 8, (V + 255) / 256));
    if (weight_bytes == 1)
        k_build_records<uint8_t><<<rblocks, 256, 0, s>>>((const uint8_t *)f1_dev, (const uint8_t *)f2_dev, V, d,
                                                        stl[0], stl[1], stl[2], stl[3], n[0], n[1], n[2], n[3],
                                                        (unsigned char *)(b + o_rec), rbytes);
    else
        k_build_records<uint16_t><<<rblocks, 256, 0, s>>>((const uint16_t *)f1_dev, (const uint16_t *)f2_dev, V, d,
                                                         stl[0], stl[1], stl[2], stl[3], n[0], n[1], n[2], n[3],
                                                         (unsigned char *)(b + o_rec), rbytes);
    k_mark_B<<<(int)std::max<int64_t>(1, std::min<int64_t>(sms * 4, (nB + 255) / 256)), 256, 0, s>>>(B_dev, nB, isB,
                                                                                                     V, ctl);
    k_mark_A<<<(int)std::max<int64_t>(1, std::min<int64_t>(sms * 4, (nA + 255) / 256)), 256, 0, s>>>(
        A_dev, nA, isB, V, (int)M, label, offer, cand, ctl);
    CSP_CUDA(cudaGetLastError());

    Params<uint8_t> P8{};
    Params<uint16_t> P16{};
    auto fill = [&](auto &P) {
        using W = std::remove_cv_t<std::remove_pointer_t<decltype(P.f1)>>;
        P.f1 = (const W *)f1_dev;
        P.f2 = (const W *)f2_dev;
        P.rec = (const uint4 *)(b + o_rec);
        P.V = V;
        for (int k = 0; k < 4; k++) P.stride[k] = stride[k];
        P.label = label;
        P.offer = offer;
        P.isB = isB;
        P.src_stamp = nullptr;
        P.cand = cand;
        P.cand_cap = (unsigned int)cand_cap;
        for (int q = 0; q < 2; q++) {
            P.ed[q] = (uint32_t *)(b + o_pool[q][0]);
            P.qa[q] = (int32_t *)(b + o_pool[q][1]);
            P.ta[q] = (int32_t *)(b + o_pool[q][2]);
            P.pk[q] = packed_pool(P.qa[q], P.ta[q], (int64_t)pool_cap);
            P.fill[q] = (uint32_t *)(b + o_fill[q]);
        }
        P.max_f1 = weight_bytes == 1 ? 255u : 65535u;  // (the weights are not scanned here: their type's bound)
        P.pool_cap = (unsigned int)pool_cap;
        P.ctl = ctl;
        P.trace = nullptr;
        P.trace_cap = 0;
        P.result_dev = (long long *)result_dev;
        P.M = (int)M;
        P.max_cycles = max_cycles > 0 ? max_cycles : 0;
        P.budget_ns = 120ull * 1000000000ull;
        P.barrier_ns = 4000000000ull;
    };
    void *args[1];
    if (weight_bytes == 1) {
        fill(P8);
        args[0] = &P8;
    } else {
        fill(P16);
        args[0] = &P16;
    }
    CSP_CUDA(cudaLaunchCooperativeKernel(fn, dim3(ctas), dim3(TPB), args, kSmem, s));
    return CSP_OK;
}
