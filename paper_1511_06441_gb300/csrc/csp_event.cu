// libcsp: the event-driven form of the cycle loop (csp_event.cuh) and its workspace.
//
// Per lattice (or graph), built once per weight upload: one record per directed edge
// (tail, ring offset, head, f1 | f2 << 16) and the ring offsets, an exclusive prefix sum
// of f1 over the directed edges (each edge's queue holds at most f1 flows).  Per solve:
// empty queues, a full chunk free stack, an empty calendar, then one cooperative
// persistent kernel (k_event) that runs the whole loop.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <new>
#include <string>

#include "csp.h"
#include "csp_event.cuh"
#include "csp_internal.h"

using namespace csp;

struct csp_event_ws {
    bool ready = false;          // edge records built for the current weights
    bool supported = false;      // max f1 + 1 <= EV_WMAX and the rings fit 32-bit offsets
    int W = 0;
    unsigned long long ring_len = 0;  // sum of f1 over directed edges
    uint4 *edge = nullptr;       // [S V]
    uint2 *ring = nullptr;
    // calendar and counts (per solve), one allocation
    void *cal = nullptr;
    size_t cal_bytes = 0;
    int64_t entry_cap = 0;       // bucket entries the chunk pool holds (besides part-filled chunks)
    uint32_t nch = 0;
    uint2 *bent = nullptr;
    uint32_t *bfill = nullptr, *freestk = nullptr, *bdir = nullptr, *bcount = nullptr;
    int32_t *blive = nullptr, *out_count = nullptr;
    EvCtl *ev = nullptr;
};

namespace {

constexpr int SCAN_TPB = 512;
constexpr int SCAN_PER = 4;                       // vertices per thread
constexpr int SCAN_BLOCK = SCAN_TPB * SCAN_PER;   // vertices per block

// Sum of f1 over the directed edges leaving v (from the vertex's edge record).
template <typename W>
__device__ __forceinline__ unsigned long long out_f1_sum(const unsigned char *rec, int rec_bytes, int nslot, long long v,
                                                         unsigned int &mx)
{
    const W *w = reinterpret_cast<const W *>(rec + v * rec_bytes);
    unsigned long long s = 0;
    for (int dir = 0; dir < nslot; dir++) {
        const unsigned int f = w[2 * dir];
        s += f;
        mx = max(mx, f);
    }
    return s;
}

// Block-wide exclusive scan of one value per thread (SCAN_TPB threads); returns the prefix
// and writes the block total to *total.
__device__ unsigned long long block_exclusive_scan(unsigned long long x, unsigned long long *total)
{
    __shared__ unsigned long long s_w[SCAN_TPB / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned long long inc = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) s_w[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        unsigned long long w = lane < SCAN_TPB / 32 ? s_w[lane] : 0ull;
        unsigned long long wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long y = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += y;
        }
        if (lane < SCAN_TPB / 32) s_w[lane] = wi - w;  // exclusive prefix of each warp
        if (lane == SCAN_TPB / 32 - 1) *total = wi;
    }
    __syncthreads();
    const unsigned long long r = s_w[warp] + inc - x;
    __syncthreads();
    return r;
}

// Per block of SCAN_BLOCK vertices: the sum of f1 over their out-edges; and the largest f1.
template <typename W>
__global__ void __launch_bounds__(SCAN_TPB) k_ev_sums(const unsigned char *rec, int rec_bytes, int nslot, long long V,
                                                      unsigned long long *bsum, unsigned int *maxf1)
{
    unsigned int mx = 0;
    unsigned long long s = 0;
    const long long v0 = (long long)blockIdx.x * SCAN_BLOCK + (long long)threadIdx.x * SCAN_PER;
    for (int i = 0; i < SCAN_PER; i++)
        if (v0 + i < V) s += out_f1_sum<W>(rec, rec_bytes, nslot, v0 + i, mx);
    __shared__ unsigned long long s_tot;
    block_exclusive_scan(s, &s_tot);
    for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0 && mx) atomicMax(maxf1, mx);
    if (threadIdx.x == 0) bsum[blockIdx.x] = s_tot;
}

// One block: exclusive scan of the n block sums in place; the grand total goes to bsum[n].
__global__ void __launch_bounds__(SCAN_TPB) k_ev_scan_blocks(unsigned long long *bsum, long long n)
{
    const long long per = (n + SCAN_TPB - 1) / SCAN_TPB;
    const long long a = threadIdx.x * per, b = min(n, a + per);
    unsigned long long s = 0;
    for (long long i = a; i < b; i++) s += bsum[i];
    __shared__ unsigned long long s_tot;
    unsigned long long run = block_exclusive_scan(s, &s_tot);
    for (long long i = a; i < b; i++) {
        const unsigned long long x = bsum[i];
        bsum[i] = run;
        run += x;
    }
    if (threadIdx.x == 0) bsum[n] = s_tot;
}

// The record of every directed edge: {tail 0, ring offset, head 0, f1 | f2 << 16}.
template <typename W>
__global__ void __launch_bounds__(SCAN_TPB) k_ev_edges(const unsigned char *rec, int rec_bytes, int nslot, long long V,
                                                       const unsigned long long *bpre, uint4 *edge)
{
    unsigned int mx = 0;
    unsigned long long s = 0;
    const long long v0 = (long long)blockIdx.x * SCAN_BLOCK + (long long)threadIdx.x * SCAN_PER;
    for (int i = 0; i < SCAN_PER; i++)
        if (v0 + i < V) s += out_f1_sum<W>(rec, rec_bytes, nslot, v0 + i, mx);
    __shared__ unsigned long long s_tot;
    unsigned long long off = bpre[blockIdx.x] + block_exclusive_scan(s, &s_tot);
    for (int i = 0; i < SCAN_PER; i++) {
        const long long v = v0 + i;
        if (v >= V) break;
        const W *w = reinterpret_cast<const W *>(rec + v * rec_bytes);
        for (int dir = 0; dir < nslot; dir++) {
            const unsigned int f1 = w[2 * dir], f2 = w[2 * dir + 1];
            edge[v * nslot + dir] = make_uint4(0u, (unsigned int)off, 0u, f1 | (f2 << 16));
            off += f1;
        }
    }
}

// Per solve: every queue empty (head = tail = 0), every chunk on the free stack, totals zero.
__global__ void k_ev_reset(uint4 *edge, long long n_edges, uint32_t *freestk, uint32_t nch, EvCtl *ev)
{
    const long long step = (long long)gridDim.x * blockDim.x;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n_edges; i += step) {
        edge[i].x = 0u;
        edge[i].z = 0u;
    }
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nch; i += step) freestk[i] = (uint32_t)i;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        ev->live = 0;
        ev->active = 0;
        ev->free_top = (int)nch;
        for (int i = 0; i < 4; i++) ev->phase_ns[i] = 0;
    }
}

template <int D, typename W, bool TRACE>
__global__ void __launch_bounds__(TPB, CSP_MIN_CTAS_PER_SM) k_event(Params<W> P, EvParams E)
{
    __shared__ EvSmem sm;
    unsigned long long epoch = 0;
    run_event_solve<D, W, TRACE>(P, E, Group{blockIdx.x, gridDim.x}, sm, epoch);
}

template <int D, typename W, bool TRACE>
const void *ev_kernel_ptr()
{
    return (const void *)&k_event<D, W, TRACE>;
}

template <typename W, bool TRACE>
const void *ev_pick_w(int d)
{
    switch (d) {
    case 1: return ev_kernel_ptr<1, W, TRACE>();
    case 2: return ev_kernel_ptr<2, W, TRACE>();
    case 3: return ev_kernel_ptr<3, W, TRACE>();
    case GRAPH: return ev_kernel_ptr<GRAPH, W, TRACE>();
    default: return ev_kernel_ptr<4, W, TRACE>();
    }
}

const void *ev_pick(int d, int wbytes, bool trace)
{
    if (wbytes == 1) return trace ? ev_pick_w<uint8_t, true>(d) : ev_pick_w<uint8_t, false>(d);
    return trace ? ev_pick_w<uint16_t, true>(d) : ev_pick_w<uint16_t, false>(d);
}

void free_calendar(csp_event_ws *X)
{
    if (X->cal) cudaFree(X->cal);
    X->cal = nullptr;
    X->cal_bytes = 0;
    X->entry_cap = 0;
    X->nch = 0;
}

}  // namespace

void event_release(csp_lattice *L)
{
    if (!L || !L->evw) return;
    csp_event_ws *X = L->evw;
    if (X->edge) cudaFree(X->edge);
    if (X->ring) cudaFree(X->ring);
    free_calendar(X);
    delete X;
    L->evw = nullptr;
}

void event_invalidate(csp_lattice *L)
{
    if (L && L->evw) L->evw->ready = false;
}

// Builds the edge records and ring offsets for the current weights (once; synchronous).
csp_status event_prepare(csp_lattice *L, cudaStream_t s)
{
    if (!L->evw) {
        L->evw = new (std::nothrow) csp_event_ws();
        if (!L->evw) return CSP_ERR_OOM;
    }
    csp_event_ws *X = L->evw;
    if (X->ready) return CSP_OK;
    const int S = nslots(L->d);
    const long long V = L->V, nb = (V + SCAN_BLOCK - 1) / SCAN_BLOCK;
    unsigned long long *bsum = nullptr;
    unsigned int *mx = nullptr;
    CSP_CUDA(cudaMalloc((void **)&bsum, (nb + 1) * 8 + 256));
    mx = (unsigned int *)((char *)bsum + (nb + 1) * 8 + 128);
    cudaError_t e = cudaMemsetAsync(mx, 0, 4, s);
    if (e == cudaSuccess) {
        if (L->wbytes == 1)
            k_ev_sums<uint8_t><<<(unsigned)nb, SCAN_TPB, 0, s>>>((const unsigned char *)L->rec, L->rec_bytes, S, V, bsum, mx);
        else
            k_ev_sums<uint16_t><<<(unsigned)nb, SCAN_TPB, 0, s>>>((const unsigned char *)L->rec, L->rec_bytes, S, V, bsum, mx);
        k_ev_scan_blocks<<<1, SCAN_TPB, 0, s>>>(bsum, nb);
        e = cudaGetLastError();
    }
    unsigned long long total = 0;
    unsigned int maxf1 = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&total, bsum + nb, 8, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&maxf1, mx, 4, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        cudaFree(bsum);
        return cuda_fail(e, "event_prepare");
    }
    X->W = (int)maxf1 + 1;
    X->ring_len = total;
    X->supported = X->W <= EV_WMAX && total < 0xFFFFFF00ull;
    if (X->supported) {
        if (!X->edge) e = cudaMalloc((void **)&X->edge, (size_t)S * V * sizeof(uint4));
        if (e == cudaSuccess) {
            if (X->ring) cudaFree(X->ring);
            X->ring = nullptr;
            e = cudaMalloc((void **)&X->ring, (size_t)std::max(total, 1ull) * sizeof(uint2));
        }
        if (e == cudaSuccess) {
            if (L->wbytes == 1)
                k_ev_edges<uint8_t><<<(unsigned)nb, SCAN_TPB, 0, s>>>((const unsigned char *)L->rec, L->rec_bytes, S, V,
                                                                      bsum, X->edge);
            else
                k_ev_edges<uint16_t><<<(unsigned)nb, SCAN_TPB, 0, s>>>((const unsigned char *)L->rec, L->rec_bytes, S, V,
                                                                       bsum, X->edge);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    }
    cudaFree(bsum);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return cuda_fail(e, "event_prepare");
    }
    X->ready = true;
    return CSP_OK;
}

bool event_supported(const csp_lattice *L) { return L->evw && L->evw->ready && L->evw->supported; }

// The calendar for up to entry_cap bucket entries (plus part-filled chunks: each CTA of
// the largest group keeps one open chunk per arrival time of the window).
csp_status event_reserve(csp_lattice *L, int64_t entry_cap)
{
    csp_event_ws *X = L->evw;
    if (X->cal && entry_cap <= X->entry_cap) return CSP_OK;
    entry_cap = std::max<int64_t>(entry_cap, X->entry_cap);
    const int64_t gmax = max_group_ctas(L->device);
    const int64_t nch64 = (entry_cap + EV_CH - 1) / EV_CH + gmax * (X->W + 1);
    if (nch64 >= 0x7fffff00ll) return CSP_ERR_CAPACITY;
    const uint32_t nch = (uint32_t)nch64;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o = off;
        off = align_up(off + bytes, 256);
        return o;
    };
    const size_t o_bent = take((size_t)nch * EV_CH * sizeof(uint2)), o_bfill = take((size_t)nch * 4),
                 o_free = take((size_t)nch * 4), o_bdir = take((size_t)2 * X->W * nch * 4),
                 o_bcount = take((size_t)2 * X->W * 4), o_blive = take((size_t)X->W * 4),
                 o_out = take((size_t)L->V * 4), o_ev = take(sizeof(EvCtl));
    free_calendar(X);
    void *p = nullptr;
    cudaError_t e = cudaMalloc(&p, off);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return cuda_fail(e, "cudaMalloc(event calendar)");
    }
    char *b = (char *)p;
    X->cal = p;
    X->cal_bytes = off;
    X->entry_cap = entry_cap;
    X->nch = nch;
    X->bent = (uint2 *)(b + o_bent);
    X->bfill = (uint32_t *)(b + o_bfill);
    X->freestk = (uint32_t *)(b + o_free);
    X->bdir = (uint32_t *)(b + o_bdir);
    X->bcount = (uint32_t *)(b + o_bcount);
    X->blive = (int32_t *)(b + o_blive);
    X->out_count = (int32_t *)(b + o_out);
    X->ev = (EvCtl *)(b + o_ev);
    return CSP_OK;
}

int64_t event_entry_cap(const csp_lattice *L) { return L->evw ? L->evw->entry_cap : 0; }

// Enqueues the per-solve reset and the event kernel.  params points at the Params<W>
// enqueue_solve filled; ctas as chosen there.
csp_status event_launch(csp_lattice *L, const void *params, bool trace, int ctas, const csp_options *opt,
                        cudaStream_t s)
{
    csp_event_ws *X = L->evw;
    const int S = nslots(L->d);
    const long long n_edges = (long long)S * L->V;
    CSP_CUDA(cudaMemsetAsync(X->ring, 0, (size_t)std::max(X->ring_len, 1ull) * sizeof(uint2), s));
    CSP_CUDA(cudaMemsetAsync(X->bcount, 0, (size_t)2 * X->W * 4, s));
    CSP_CUDA(cudaMemsetAsync(X->blive, 0, (size_t)X->W * 4, s));
    if (trace) CSP_CUDA(cudaMemsetAsync(X->out_count, 0, (size_t)L->V * 4, s));
    const int sms = num_sms(L->device);
    const long long rb = std::max<long long>(1, std::min<long long>(sms * 8, (std::max<long long>(n_edges, X->nch) + 255) / 256));
    k_ev_reset<<<(unsigned)rb, 256, 0, s>>>(X->edge, n_edges, X->freestk, X->nch, X->ev);
    CSP_CUDA(cudaGetLastError());
    EvParams E{};
    E.edge = X->edge;
    E.ring = X->ring;
    E.bent = X->bent;
    E.bfill = X->bfill;
    E.freestk = X->freestk;
    E.bdir = X->bdir;
    E.bcount = X->bcount;
    E.blive = X->blive;
    E.out_count = X->out_count;
    E.ev = X->ev;
    E.nch = X->nch;
    E.W = X->W;
    const void *fn = ev_pick(L->d, L->wbytes, trace);
    void *args[2] = {const_cast<void *>(params), &E};
    if (opt && opt->ev_begin) CSP_CUDA(cudaEventRecord((cudaEvent_t)opt->ev_begin, s));
    CSP_CUDA(cudaLaunchCooperativeKernel(fn, dim3(ctas), dim3(TPB), args, 0, s));
    if (opt && opt->ev_end) CSP_CUDA(cudaEventRecord((cudaEvent_t)opt->ev_end, s));
    return CSP_OK;
}

// CTAs of the event kernel that fit on the device at once (cooperative launch).
csp_status event_max_ctas(const csp_lattice *L, bool trace, int *out)
{
    const void *fn = ev_pick(L->d, L->wbytes, trace);
    int per_sm = 0;
    CSP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, TPB, 0));
    if (per_sm < 1) {
        set_error("event kernel does not fit on an SM");
        return CSP_ERR_CUDA;
    }
    *out = std::min(per_sm * num_sms(L->device), max_group_ctas(L->device));
    return CSP_OK;
}

// Leader's phase times of the last event solve (set-up, phase A, phase B, barriers), ns.
csp_status event_phase_times(const csp_lattice *L, unsigned long long *ns4)
{
    if (!L->evw || !L->evw->ev) return CSP_ERR_INVALID;
    CSP_CUDA(cudaMemcpy(ns4, L->evw->ev->phase_ns, 4 * 8, cudaMemcpyDeviceToHost));
    return CSP_OK;
}
