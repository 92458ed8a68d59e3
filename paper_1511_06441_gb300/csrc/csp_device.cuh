// Device-side building blocks of the water-flow cycle (arXiv 1511.06441, Algorithm 1):
// the flow-pool sweep (Steps 1-3 and 7-9), the launch phase (Steps 2, 4, 5 and the
// label part of Step 8), block-level compaction and a spin-limited grid barrier.
//
// Data layout in HBM (one solve):
//   label[V]  int32   committed labels, frozen while the pool is swept
//   offer[V]  uint64  running max of (quality << 32 | ~(src*8 + dir)) over all arrivals;
//                     its high half equals label[] at every cycle boundary
//   isB[V/32] uint32  bitmap of B
//   trig[]    int32   vertices whose label improves in the current cycle
//   pool[2]   SoA     ed = dst << 3 | direction back to the source (uint32),
//                     qa = quality on arrival (int32), ta = arrival time (int32)
// A flow is the paper's water flow on an active (or phantom) edge: it left its source
// at the time the source's label last improved and carries that label.
#pragma once

#include <climits>
#include <cstdint>

namespace csp {

constexpr int TPB = 512;            // threads per CTA
constexpr int IPT = 4;              // items per thread per tile
constexpr int TILE = TPB * IPT;     // items per tile
constexpr int NWARP = TPB / 32;
constexpr int TIME_LIMIT = 1 << 30; // arrival times must stay below this

enum : int { ST_OK = 0, ST_INVALID = 1, ST_OOM = 2, ST_CUDA = 3, ST_CAPACITY = 4, ST_TIMEOUT = 5, ST_BARRIER = 6 };

// result record (int64): index of each field
enum : int {
    R_STATUS = 0, R_F1, R_X, R_XSRC, R_XDIR, R_F2, R_CYCLES, R_UPDATES, R_LAUNCHED, R_PASSES,
    R_MAXPOOL, R_TRACELEN, R_NEXTTAG, R_ARRIVALS, R_IMPROVED, R_COUNT = 16
};

struct Counters {
    unsigned long long n_live;    // live flows seen by the sweep
    unsigned long long launched;  // flows emitted by the launch phase
    unsigned long long xkey;      // max over improved B vertices of (label << 32 | ~id)
    unsigned int n_out;           // flows written to the output pool
    unsigned int n_trig;          // triggered vertices appended
    unsigned int arrivals;        // live flows that arrived at the cycle time
    unsigned int n_active;        // distinct sources of live flows (trace mode)
    unsigned int overflow;        // an output list ran out of room
    int min_ta;                   // smallest arrival time written to the output pool
    unsigned int abort;           // set by the leader when the solve exceeded its time budget
    unsigned int pad;
};

struct Control {
    unsigned long long bar;       // grid-barrier arrivals, monotonic within a solve
    int err;                      // set when a barrier wait gives up
    int status_in;                // set by the set-up kernels (invalid ids, A and B overlap)
    unsigned int tag;             // next unused stamp tag (kept across solves)
    unsigned int pad;
    Counters cnt[2];
    long long out[R_COUNT];
};

template <typename W>
struct Params {
    const W *f1, *f2;              // [d][V] travel time, weight of edge (v, v + e_k)
    long long V;
    int stride[4];
    int32_t *label;
    unsigned long long *offer;
    const uint32_t *isB;
    uint32_t *stamp;               // distinct-source stamps (trace mode)
    int32_t *trig;
    unsigned int trig_cap;
    uint32_t *ed[2];
    int32_t *qa[2];
    int32_t *ta[2];
    unsigned int pool_cap;
    Control *ctl;
    long long *trace;              // device rows (Time, active, flows), nullable
    long long trace_cap;
    long long *result_dev;         // nullable mirror of ctl->out
    int M;
    long long max_cycles;
    unsigned long long budget_ns;  // wall-clock budget of one launch (watchdog)
};

// ---------------------------------------------------------------- small helpers

template <int D>
__device__ __forceinline__ int dir_offset(const int (&stride)[4], unsigned r)
{
    const unsigned k = r >> 1;
    int s = stride[0];
    if (D > 1 && k == 1) s = stride[1];
    if (D > 2 && k == 2) s = stride[2];
    if (D > 3 && k == 3) s = stride[3];
    return (r & 1) ? -s : s;
}

__device__ __forceinline__ bool in_set(const uint32_t *bits, uint32_t v)
{
    return (__ldg(bits + (v >> 5)) >> (v & 31)) & 1u;
}

// Exclusive block-wide prefix sum of x; *total receives the block sum.
__device__ __forceinline__ uint32_t block_scan_excl(uint32_t x, uint32_t &total, uint32_t *s_warp)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t v = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += y;
    }
    if (lane == 31) s_warp[warp] = v;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = lane < NWARP ? s_warp[lane] : 0u;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        if (lane < NWARP) s_warp[lane] = w;
    }
    __syncthreads();
    total = s_warp[NWARP - 1];
    return (warp ? s_warp[warp - 1] : 0u) + v - x;
}

__device__ __forceinline__ unsigned long long globaltimer_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}

// Grid-wide barrier for a cooperative (co-resident) launch.  The wait gives up after
// ~4 s or 2^26 polls, sets ctl->err and returns false; every CTA then leaves the kernel.
__device__ __forceinline__ bool grid_sync(Control *ctl, unsigned long long &epoch)
{
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        epoch += 1;
        const unsigned long long target = epoch * gridDim.x;
        __threadfence();
        atomicAdd(&ctl->bar, 1ull);
        int ok = 1;
        const unsigned long long t0 = globaltimer_ns();
        for (unsigned int spin = 0;; ++spin) {
            unsigned long long seen;
            asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(seen) : "l"(&ctl->bar) : "memory");
            if (seen >= target) break;
            if (*(volatile int *)&ctl->err) { ok = 0; break; }
            if (spin > (1u << 26) || (spin & 1023u) == 0 && globaltimer_ns() - t0 > 4000000000ull) {
                atomicExch(&ctl->err, 1);
                ok = 0;
                break;
            }
            if (spin > 64) __nanosleep(64);
        }
        __threadfence();
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

struct LocalStats {
    uint32_t live, arrivals, active, launched;
    int min_ta;
};

// Adds this block's statistics to the pass counters (one global atomic per field per CTA).
__device__ __forceinline__ void flush_stats(const LocalStats &st, Counters *C)
{
    __shared__ unsigned long long s_live, s_launched;
    __shared__ unsigned int s_arr, s_act;
    __shared__ int s_min;
    if (threadIdx.x == 0) {
        s_live = 0;
        s_launched = 0;
        s_arr = 0;
        s_act = 0;
        s_min = INT_MAX;
    }
    __syncthreads();
    uint32_t live = st.live, arr = st.arrivals, act = st.active, lau = st.launched;
    int mn = st.min_ta;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        live += __shfl_xor_sync(0xffffffffu, live, o);
        arr += __shfl_xor_sync(0xffffffffu, arr, o);
        act += __shfl_xor_sync(0xffffffffu, act, o);
        lau += __shfl_xor_sync(0xffffffffu, lau, o);
        mn = min(mn, __shfl_xor_sync(0xffffffffu, mn, o));
    }
    if ((threadIdx.x & 31) == 0) {
        if (live) atomicAdd(&s_live, (unsigned long long)live);
        if (lau) atomicAdd(&s_launched, (unsigned long long)lau);
        if (arr) atomicAdd(&s_arr, arr);
        if (act) atomicAdd(&s_act, act);
        if (mn != INT_MAX) atomicMin(&s_min, mn);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        if (s_live) atomicAdd(&C->n_live, s_live);
        if (s_launched) atomicAdd(&C->launched, s_launched);
        if (s_arr) atomicAdd(&C->arrivals, s_arr);
        if (s_act) atomicAdd(&C->n_active, s_act);
        if (s_min != INT_MAX) atomicMin(&C->min_ta, s_min);
    }
}

// Staging area for one tile of output flows (coalesced write-out).
struct TileStage {
    uint32_t ed[TILE];
    int32_t qa[TILE];
    int32_t ta[TILE];
};

// Appends the flows marked keep[i] (per thread, IPT slots) to the output pool.
// Block-compacted: one atomicAdd per tile reserves room; flows are staged in shared
// memory and written out contiguously.
template <typename W>
__device__ __forceinline__ void append_flows(const Params<W> &P, int ob, Counters *C, const bool (&keep)[IPT],
                                             const uint32_t (&e)[IPT], const int32_t (&q)[IPT],
                                             const int32_t (&t)[IPT], uint32_t nk, TileStage &stage,
                                             uint32_t *s_warp, uint32_t *s_base)
{
    uint32_t total;
    uint32_t pos = block_scan_excl(nk, total, s_warp);
    if (threadIdx.x == 0) s_base[0] = total ? atomicAdd(&C->n_out, total) : 0u;
#pragma unroll
    for (int i = 0; i < IPT; i++)
        if (keep[i]) {
            stage.ed[pos] = e[i];
            stage.qa[pos] = q[i];
            stage.ta[pos] = t[i];
            pos++;
        }
    __syncthreads();
    const uint32_t base = s_base[0];
    if (total) {
        if ((unsigned long long)base + total > P.pool_cap) {
            if (threadIdx.x == 0) atomicExch(&C->overflow, 1u);
        } else {
            uint32_t *oe = P.ed[ob];
            int32_t *oq = P.qa[ob], *ot = P.ta[ob];
            for (uint32_t j = threadIdx.x; j < total; j += TPB) {
                oe[base + j] = stage.ed[j];
                oq[base + j] = stage.qa[j];
                ot[base + j] = stage.ta[j];
            }
        }
    }
    __syncthreads();
}

// ---------------------------------------------------------------- the sweep

// One pass over the flow pool (Steps 1-3 and 7-9 of the paper).  For every flow:
//   dead   if qa <= label[dst] (labels of the end of the previous cycle): dropped;
//   arrives if it is live and ta == Tg: offers (qa, ~(src*8+dir)) to dst with a 64-bit
//          atomicMax; the first arrival at dst this cycle (the one that sees the old
//          offer still equal to the label) appends dst to the triggered list;
//   survives otherwise: copied to the output pool.
// With TRACE, live flows also stamp their source to count distinct active vertices.
template <int D, typename W, bool TRACE>
__device__ void sweep(const Params<W> &P, int ib, uint32_t n_in, int Tg, Counters *C, uint32_t tag,
                      LocalStats &st, TileStage &stage, uint32_t *s_warp, uint32_t *s_base)
{
    const uint32_t *__restrict__ ie = P.ed[ib];
    const int32_t *__restrict__ iq = P.qa[ib];
    const int32_t *__restrict__ it = P.ta[ib];
    const int ob = ib ^ 1;
    for (uint32_t base = blockIdx.x * TILE; base < n_in; base += gridDim.x * TILE) {
        uint32_t e[IPT];
        int32_t q[IPT], t[IPT], L[IPT];
        bool keep[IPT], trig[IPT];
#pragma unroll
        for (int i = 0; i < IPT; i++) {
            const uint32_t idx = base + i * TPB + threadIdx.x;
            keep[i] = trig[i] = false;
            e[i] = 0;
            q[i] = 0;
            t[i] = 0;
            if (idx < n_in) {
                e[i] = __ldcg(ie + idx);
                q[i] = __ldcg(iq + idx);
                t[i] = __ldcg(it + idx);
            }
        }
#pragma unroll
        for (int i = 0; i < IPT; i++) {
            const uint32_t idx = base + i * TPB + threadIdx.x;
            L[i] = INT_MAX;
            if (idx < n_in) L[i] = __ldcg(P.label + (e[i] >> 3));
        }
        uint32_t nk = 0, nt = 0;
#pragma unroll
        for (int i = 0; i < IPT; i++) {
            if (q[i] <= L[i]) continue;  // dead (or padding): removed
            st.live++;
            const uint32_t dst = e[i] >> 3, r = e[i] & 7u;
            const uint32_t src = (uint32_t)((int)dst + dir_offset<D>(P.stride, r));
            if (TRACE) {
                if (atomicExch(P.stamp + src, tag) != tag) st.active++;
            }
            if (t[i] == Tg) {
                st.arrivals++;
                const unsigned long long key =
                    ((unsigned long long)(uint32_t)q[i] << 32) | (0xffffffffu - (src * 8u + (r ^ 1u)));
                const unsigned long long old = atomicMax(P.offer + dst, key);
                if ((uint32_t)(old >> 32) == (uint32_t)L[i]) {
                    trig[i] = true;
                    nt++;
                }
            } else {
                keep[i] = true;
                nk++;
                st.min_ta = min(st.min_ta, t[i]);
            }
        }
        // triggered vertices: reserve with one atomic per tile, write directly
        uint32_t ttot;
        uint32_t tpos = block_scan_excl(nt, ttot, s_warp);
        if (threadIdx.x == 0) s_base[1] = ttot ? atomicAdd(&C->n_trig, ttot) : 0u;
        __syncthreads();
        if (nt) {
            const uint32_t tb = s_base[1] + tpos;
#pragma unroll
            for (int i = 0, j = 0; i < IPT; i++)
                if (trig[i]) {
                    if (tb + j < P.trig_cap) P.trig[tb + j] = (int32_t)(e[i] >> 3);
                    else atomicExch(&C->overflow, 1u);
                    j++;
                }
        }
        append_flows(P, ob, C, keep, e, q, t, nk, stage, s_warp, s_base);
    }
}

// ---------------------------------------------------------------- the launch phase

// For every triggered vertex v (items = (v, direction) pairs): commit its new label
// (Step 8), record it if it is in B (Algorithm 2), and start a flow on every edge
// (v, w) with Label(v) - f2 > Label(w) under the labels at the end of this cycle
// (Steps 4-5; a flow on an edge that already carries water is the paper's phantom).
template <int D, typename W>
__device__ void launch(const Params<W> &P, int ob, uint32_t n_trig, int Time, Counters *C, LocalStats &st,
                       TileStage &stage, uint32_t *s_warp, uint32_t *s_base)
{
    constexpr uint32_t ND = 2 * D;
    const uint32_t n_items = n_trig * ND;
    for (uint32_t base = blockIdx.x * TILE; base < n_items; base += gridDim.x * TILE) {
        uint32_t e[IPT];
        int32_t q[IPT], t[IPT];
        bool keep[IPT];
        uint32_t nk = 0;
#pragma unroll
        for (int i = 0; i < IPT; i++) {
            const uint32_t j = base + i * TPB + threadIdx.x;
            keep[i] = false;
            e[i] = 0;
            q[i] = 0;
            t[i] = 0;
            if (j >= n_items) continue;
            const uint32_t v = (uint32_t)__ldcg(P.trig + j / ND);
            const uint32_t dir = j % ND;
            const int Lv = (int)(__ldcg(P.offer + v) >> 32);
            if (dir == 0) {
                P.label[v] = Lv;
                if (in_set(P.isB, v))
                    atomicMax(&C->xkey, ((unsigned long long)(uint32_t)Lv << 32) | (0xffffffffu - v));
            }
            const uint32_t k = dir >> 1;
            const int s = dir_offset<D>(P.stride, dir);
            uint32_t w, slot;
            if (dir & 1) {
                if (v < (uint32_t)(-s)) continue;  // lower face of the box: no edge
                w = v + s;
                slot = k * (uint32_t)P.V + w;
            } else {
                w = v + s;
                slot = k * (uint32_t)P.V + v;       // upper-face entries are zero: no edge
            }
            const int t1 = (int)__ldg(P.f1 + slot);
            if (t1 == 0) continue;
            const int qa = Lv - (int)__ldg(P.f2 + slot);
            const int Lw = (int)(__ldcg(P.offer + w) >> 32);
            if (qa > Lw) {
                keep[i] = true;
                nk++;
                e[i] = (w << 3) | (dir ^ 1u);
                q[i] = qa;
                t[i] = Time + t1;
                st.min_ta = min(st.min_ta, t[i]);
                st.launched++;
            }
        }
        append_flows(P, ob, C, keep, e, q, t, nk, stage, s_warp, s_base);
    }
}

}  // namespace csp
