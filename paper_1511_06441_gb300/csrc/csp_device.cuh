// Device-side building blocks of the water-flow cycle (arXiv 1511.06441, Algorithm 1):
// the flow-pool sweep (Steps 1-3 and 7-9), the launch phase (Steps 2, 4, 5 and the
// label part of Step 8), warp-level compaction into per-CTA pool chunks, a TMA (bulk-copy)
// tile pipeline and a spin-limited grid barrier.
//
// Data layout in HBM (one solve):
//   label[V]  int32   committed labels, frozen while the pool is swept
//   offer[V]  uint64  running max of (quality << 32 | ~(src*8 + dir)) over all arrivals;
//                     its high half equals label[] at every cycle boundary
//   isB[V/32] uint32  bitmap of B
//   src_stamp uint32  per vertex: the last pass in which it sourced a live flow (trace mode)
//   nbw[8V]   uint32  general graphs only: out-slot j of v = head << 3 | the edge's in-slot at its head
//   nbw_in[8V] uint32 general graphs only: in-slot k of u = tail << 3 | the edge's out-slot at its
//                     tail (the same table as nbw on an undirected graph)
//   edge_stamp uint32 per directed edge (v * slots + dir): the last pass in which it carried a
//                     flow that did not arrive (trace mode; phantom count)
//   cand[]    uint32  arrivals of the current cycle (flow word ed of each arriving flow),
//                     one region of cand_cap / G entries per CTA of the group
//   pool[2]   SoA     ed = dst << 3 | direction back to the source (uint32),
//                     qa = quality on arrival (int32), ta = arrival time (int32);
//                     stored in chunks of TILE slots, fill[b][chunk] = slots in use.
//                     Packed form (pk[b], where the three fit in 64 bits): one word per
//                     flow, ed << (qb + tb) | qa << tb | (ta mod 2^tb), over the qa and ta
//                     arrays (see PoolFmt)
// A flow is the paper's water flow on an active (or phantom) edge: it left its source
// at the time the source's label last improved and carries that label.
#pragma once

#include <climits>
#include <cstdint>

namespace csp {

#ifndef CSP_TPB
#define CSP_TPB 512
#endif
#ifndef CSP_IPT
#define CSP_IPT 4
#endif
#ifndef CSP_MIN_CTAS_PER_SM
#define CSP_MIN_CTAS_PER_SM 2
#endif
#ifndef CSP_NSTAGE
#define CSP_NSTAGE 3
#endif
constexpr int TPB = CSP_TPB;        // threads per CTA
constexpr int IPT = CSP_IPT;        // items per thread per tile
constexpr int TILE = TPB * IPT;     // items per tile
constexpr int NWARP = TPB / 32;
constexpr int TIME_LIMIT = 1 << 30; // arrival times must stay below this
constexpr int POOL_PAD = 64;        // extra elements after each pool array (bulk copies round up)
constexpr int NSTAGE = CSP_NSTAGE;  // input stages of the sweep (tiles in flight per CTA)
constexpr int GRAPH = 5;            // template value of D for a general graph (Section 1): up to 8 slots

// Directions (edge slots) per vertex: 2d on a lattice of dimension d, 8 on a general graph.
__host__ __device__ constexpr int nslots(int D) { return D == GRAPH ? 8 : 2 * D; }

enum : int { ST_OK = 0, ST_INVALID = 1, ST_OOM = 2, ST_CUDA = 3, ST_CAPACITY = 4, ST_TIMEOUT = 5, ST_BARRIER = 6 };

// result record (int64): index of each field
enum : int {
    R_STATUS = 0, R_F1, R_X, R_XSRC, R_XDIR, R_F2, R_CYCLES, R_UPDATES, R_LAUNCHED, R_PASSES,
    R_MAXPOOL, R_TRACELEN, R_ELAPSED_NS, R_ARRIVALS, R_IMPROVED, R_PHANTOMS, R_COUNT = 16
};

__host__ __device__ __forceinline__ unsigned int lo32(unsigned long long x) { return (unsigned int)(x & 0xffffffffull); }
__host__ __device__ __forceinline__ unsigned int hi32(unsigned long long x) { return (unsigned int)(x >> 32); }

// Pass counters.  Every field that CTAs update concurrently sits on its own 128-byte line
// (L2 atomics on one line serialise), and pairs updated together are packed into one
// 64-bit word so that one atomic serves both.
struct Counters {
    alignas(128) unsigned long long out_cand;  // low 32: flows written to the output pool; high 32: arrivals listed
    alignas(128) unsigned long long live;      // live flows seen by the sweep
    alignas(128) unsigned long long lau_imp;   // low 32: flows launched; high 32: vertices improved
    alignas(128) unsigned long long xkey;      // max over improved B vertices of (label << 32 | ~id)
    alignas(128) int min_ta;                   // smallest arrival time written to the output pool
    alignas(128) unsigned int n_active;        // distinct sources of live flows (trace mode)
    alignas(128) unsigned int overflow;        // an output list ran out of room
    unsigned int abort;                        // set by the leader when the solve exceeded its time budget
    alignas(128) unsigned int chunks;          // output-pool chunks handed out in this pass
    alignas(128) unsigned long long phantoms;  // trace mode: flows started on an edge that carries one
};

constexpr int NRELEASE = 32;  // copies of the barrier's release word, one per 128-byte line
constexpr int MAX_GROUP = 1024;  // most CTAs one group may have

struct ReleaseWord {
    alignas(128) unsigned long long epoch;
};

struct Control {
    alignas(128) unsigned long long bar;  // grid-barrier arrivals, monotonic within a solve
    alignas(128) int err;                 // set when a barrier or copy wait gives up
    int status_in;                        // set by the set-up kernels (invalid ids, A and B overlap)
    ReleaseWord release[NRELEASE];        // last barrier epoch released (one copy per line)
    Counters cnt[2];
    alignas(128) long long out[R_COUNT];
};

// Per-vertex edge record: (f1, f2) of the edges of a vertex in direction (slot) order,
// f1 = 0 for a missing edge (absent, leaving the box, or an empty slot of a graph).
// 8-bit weights: 2 bytes per direction, one 16-byte record for up to 8 directions (d <= 4,
// or a graph).  16-bit weights: 4 bytes per direction, 16 bytes for d <= 2 and 32 bytes
// for up to 8 directions.
template <typename W, int D>
struct EdgeRecord {
    static constexpr int BYTES = (int)sizeof(W) * 2 * nslots(D) <= 16 ? 16 : 32;
    static constexpr int VEC = BYTES / 16;  // uint4 loads per record
    uint4 raw[VEC];
    __device__ __forceinline__ int f1(int dir) const
    {
        const W *w = reinterpret_cast<const W *>(raw);
        return (int)w[2 * dir];
    }
    __device__ __forceinline__ int f2(int dir) const
    {
        const W *w = reinterpret_cast<const W *>(raw);
        return (int)w[2 * dir + 1];
    }
};

template <typename W>
struct Params {
    const W *f1, *f2;              // [d][V] travel time, weight of edge (v, v + e_k)
    const uint4 *rec;              // per-vertex edge records (EdgeRecord<W, d>)
    long long V;
    int stride[4];                 // lattice strides (unused on a graph)
    const uint32_t *nbw;           // graph only: [8 V] out-slot j of v = head << 3 | the edge's in-slot at its head
    const uint32_t *nbw_in;        // graph only: [8 V] in-slot k of u = tail << 3 | the edge's out-slot there
    int32_t *label;
    unsigned long long *offer;
    const uint32_t *isB;
    uint32_t *src_stamp;           // trace mode: [V rounded up to 4] last pass each vertex sourced a live flow
    uint32_t *edge_stamp;          // nullable (trace mode, phantom count): [slots V] last pass each directed edge carried a staying flow
    uint32_t *cand;                // arrivals of the current cycle (the sources of A at the seed)
    unsigned int cand_cap;
    uint32_t *ed[2];
    int32_t *qa[2];
    int32_t *ta[2];
    unsigned long long *pk[2];     // nullable: the packed pool over qa[b] and ta[b] (8 B per slot)
    unsigned int max_f1;           // largest travel time of the lattice (sizes the packed time field)
    uint32_t *fill[2];             // slots in use per pool chunk (pool_cap / TILE entries)
    unsigned int pool_cap;         // slots per pool buffer, a multiple of TILE
    Control *ctl;
    long long *trace;              // device rows (Time, active, flows), nullable
    long long trace_cap;
    long long *result_dev;         // nullable mirror of ctl->out
    int M;
    long long max_cycles;
    unsigned long long budget_ns;   // wall-clock budget of one launch (watchdog)
    unsigned long long barrier_ns;  // longest wait at one barrier before giving up
    int test_absent;                // test hook: the group's last CTA leaves before its first barrier
    uint32_t *touched;              // nullable: vertices whose label left 0 are appended here
    unsigned int *touched_n;        // its length
    // Improvement record for path reconstruction (all nullable):
    int32_t *first_t;               // [V] time of the vertex's first improvement
    uint32_t *first_code;           // [V] winning arrival code ~(src * 8 + dir) of that improvement
    uint2 *log;                     // every improvement (v, code), pass by pass
    unsigned long long log_cap;     // records that fit in log
    unsigned long long *log_n;      // records produced (may exceed log_cap: the rest were dropped)
    int32_t *pass_time;             // [pass_cap] Time of each pass
    unsigned long long *pass_off;   // [pass_cap + 1] first log record of each pass
    long long pass_cap;
};

// One input stage of the sweep: a pool tile as three arrays, or (packed pool) as TILE
// 64-bit words over qa and ta.
struct Stage {
    uint32_t ed[TILE];
    int32_t qa[TILE];
    int32_t ta[TILE];
    __device__ __forceinline__ const unsigned long long *words() const
    {
        return reinterpret_cast<const unsigned long long *>(qa);
    }
};

// Dynamic shared memory of the cycle kernel: NSTAGE input stages filled by bulk copies,
// their barriers, and the CTA's output cursor.  The cursor word packs the chunk being
// filled (high half) and the slots already claimed in it (low half); next_chunk is the
// chunk allocated ahead for the warp that fills the current one.
struct Smem {
    Stage stage[NSTAGE];
    unsigned long long mbar[NSTAGE];
    unsigned long long cursor;
    uint32_t next_chunk;
    uint32_t n_cand;               // arrivals listed in this CTA's candidate region
    uint32_t read_cnt[NSTAGE];     // warps done reading stage s
    uint32_t stage_fill[NSTAGE];   // flows in the tile held by stage s
    int fail;                      // a bounded wait gave up
};

constexpr uint32_t NO_CHUNK = 0xffffffffu;    // no chunk allocated
constexpr uint32_t OVF_CHUNK = 0xfffffffeu;   // allocation beyond the pool: writes dropped, overflow set
constexpr uint32_t LAZY_CHUNK = 0xfffffffdu;  // cursor not opened yet: the first claim allocates
constexpr uint32_t FIRST_SPECIAL = 0xfffffff0u;  // chunk ids from here on name no chunk

// The CTAs that cooperate on one solve: the whole grid for a single solve, a slice of
// it in batched mode.  rank = index of this CTA in the group.
struct Group {
    uint32_t rank, size;
    __device__ __forceinline__ bool leader() const { return rank == 0 && threadIdx.x == 0; }
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


// Neighbour of v in direction dir.  On a lattice v +- stride (outside the box where the
// edge leaves it: callers check the record's f1 first or clamp); on a graph the slot's
// neighbour (an empty slot holds v itself).
template <int D, typename W>
__device__ __forceinline__ uint32_t neighbour(const Params<W> &P, uint32_t v, unsigned dir)
{
    if constexpr (D == GRAPH) return __ldg(P.nbw + (size_t)v * 8 + dir) >> 3;
    else return v + dir_offset<D>(P.stride, dir);
}

// Flow word of water leaving v in direction dir: dst << 3 | the direction from dst back to v
// (on a graph: the edge's in-slot at dst).
template <int D, typename W>
__device__ __forceinline__ uint32_t flow_word(const Params<W> &P, uint32_t v, unsigned dir)
{
    if constexpr (D == GRAPH) return __ldg(P.nbw + (size_t)v * 8 + dir);
    else return ((v + dir_offset<D>(P.stride, dir)) << 3) | (dir ^ 1u);
}

// Source of flow word ed and the flow's direction at its source.
template <int D, typename W>
__device__ __forceinline__ uint32_t flow_source(const Params<W> &P, uint32_t ed, uint32_t &sdir)
{
    if constexpr (D == GRAPH) {
        const uint32_t x = __ldg(P.nbw_in + (size_t)(ed >> 3) * 8 + (ed & 7u));
        sdir = x & 7u;
        return x >> 3;
    } else {
        sdir = (ed & 7u) ^ 1u;
        return (uint32_t)((int)(ed >> 3) + dir_offset<D>(P.stride, ed & 7u));
    }
}

// x code of the flow with word ed arriving at its destination: ~(src * 8 + dir), dir the
// direction from the source to the destination.
template <int D, typename W>
__device__ __forceinline__ uint32_t arrival_code(const Params<W> &P, uint32_t ed)
{
    uint32_t sdir;
    const uint32_t src = flow_source<D>(P, ed, sdir);
    return 0xffffffffu - (src * 8u + sdir);
}

__device__ __forceinline__ unsigned long long globaltimer_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}

// Barrier over the CTAs of a group (all co-resident: cooperative launch).  Arrivals are counted on one
// word; the last CTA to arrive publishes the new epoch to NRELEASE release words on
// separate lines, and every CTA polls its own copy (with a short sleep between polls).
// Spreading the polls keeps the waiting CTAs from saturating one L2 slice while the
// slowest CTAs are still working.  The wait gives up after limit_ns or 2^30 polls, sets
// ctl->err and returns false; every CTA then leaves the kernel.
__device__ __forceinline__ bool group_sync(Control *ctl, unsigned long long &epoch, const Group &g,
                                           unsigned long long limit_ns)
{
    __shared__ int s_ok;
    __syncthreads();
    if (g.size == 1) return true;  // one CTA: the block barrier is enough
    if (threadIdx.x == 0) {
        epoch += 1;
        const unsigned long long target = epoch * g.size;
        __threadfence();
        const unsigned long long arrived = atomicAdd(&ctl->bar, 1ull) + 1ull;
        int ok = 1;
        if (arrived == target) {
            // the last arrival has seen every other CTA's (fenced) arrival: one release
            // fence, then plain strong stores of the epoch (the pollers load with acquire)
            __threadfence();
            for (int i = 0; i < NRELEASE; i++)
                asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(&ctl->release[i].epoch), "l"(epoch)
                             : "memory");
        } else {
            const unsigned long long *word = &ctl->release[g.rank % NRELEASE].epoch;
            const unsigned long long t0 = globaltimer_ns();
            for (unsigned int spin = 0;; ++spin) {
                unsigned long long seen;
                asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(seen) : "l"(word) : "memory");
                if (seen >= epoch) break;
                if ((spin & 63u) == 63u) {
                    if (*(volatile int *)&ctl->err) { ok = 0; break; }
                    if (spin > (1u << 30) || globaltimer_ns() - t0 > limit_ns) {
                        atomicExch(&ctl->err, 1);
                        ok = 0;
                        break;
                    }
                }
                __nanosleep(64);
            }
        }
        __threadfence();
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// ---------------------------------------------------------------- bulk copies (TMA)

__device__ __forceinline__ uint32_t smem_addr(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(unsigned long long *mbar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(mbar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_init_fence()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(unsigned long long *mbar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(mbar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(unsigned long long *mbar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.b32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(mbar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// L2 eviction policies.  The flow pool streams through L2 once per cycle (read, then the
// survivors written to the other buffer) and is marked evict-first; the labels the sweep
// gathers for every flow are marked evict-last, so that the stream does not push them out.
// (Measured on one GB300: the traced 128^3 step 116.1 -> 115.0 ms, the 2048^2
// anti-correlated solve 5.65 -> 5.50 s, identical results.)
__device__ __forceinline__ unsigned long long policy_evict_first()
{
    unsigned long long p;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}

__device__ __forceinline__ unsigned long long policy_evict_last()
{
    unsigned long long p;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    return p;
}

// 1-D bulk copy global -> shared of pool data (evict-first in L2), completion counted on
// mbar (bytes: multiple of 16, both addresses 16-byte aligned).
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, unsigned long long *mbar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(mbar)), "l"(policy_evict_first())
        : "memory");
}

// 32-bit global store with an L2 cache policy.
__device__ __forceinline__ void st_policy(uint32_t *a, uint32_t v, unsigned long long pol)
{
    asm volatile("st.global.L2::cache_hint.b32 [%0], %1, %2;" ::"l"(a), "r"(v), "l"(pol) : "memory");
}

// 32-bit global load through L2 only (like __ldcg) with an L2 cache policy.
__device__ __forceinline__ int32_t ld_policy(const int32_t *a, unsigned long long pol)
{
    int32_t v;
    asm volatile("ld.global.cg.L2::cache_hint.b32 %0, [%1], %2;" : "=r"(v) : "l"(a), "l"(pol));
    return v;
}

__device__ __forceinline__ void fence_proxy_async_global()
{
    asm volatile("fence.proxy.async.global;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Format of the flow pool for one solve.  Packed (tb > 0): one 64-bit word per flow,
// ed in the high bits, the quality on arrival (1 <= qa <= M) below it in qb bits and the
// arrival time mod 2^tb in the low tb bits, where 2^tb > max f1.  Every flow a sweep at
// cycle time Tg reads arrives in [Tg, Tg + max f1] (it was started at a cycle time <= Tg,
// and Tg is at most the earliest arrival in the pool), so ta = Tg + ((word - Tg) mod 2^tb).
// The pool then moves 8 B per flow instead of 12.  Otherwise (tb = 0) the three arrays.
// Uniform over the solve: every CTA computes it from the same Params.
struct PoolFmt {
    uint32_t tb;                // bits of the arrival time field; 0 = three arrays
    uint32_t sh_e;              // tb + qb: shift of the flow word ed
    unsigned long long qmask;   // 2^qb - 1
};

template <typename W>
__device__ __forceinline__ PoolFmt pool_fmt(const Params<W> &P)
{
    PoolFmt f{0u, 0u, 0ull};
    if (P.pk[0] == nullptr || P.pk[1] == nullptr || P.M <= 0) return f;
    const uint32_t tb = 32u - (uint32_t)__clz((int)max(P.max_f1, 1u));
    const uint32_t qb = 32u - (uint32_t)__clz(P.M);
    const uint32_t eb = 64u - (uint32_t)__clzll((long long)((unsigned long long)P.V * 8ull - 1ull));
    if (tb + qb + eb > 64u) return f;
    f.tb = tb;
    f.sh_e = tb + qb;
    f.qmask = (1ull << qb) - 1ull;
    return f;
}

__device__ __forceinline__ unsigned long long pack_flow(const PoolFmt &f, uint32_t e, int32_t q, int32_t t)
{
    return ((unsigned long long)e << f.sh_e) | ((unsigned long long)(uint32_t)q << f.tb) |
           (unsigned long long)((uint32_t)t & ((1u << f.tb) - 1u));
}

__device__ __forceinline__ uint32_t packed_ed(const PoolFmt &f, unsigned long long w)
{
    return (uint32_t)(w >> f.sh_e);
}

__device__ __forceinline__ int32_t packed_qa(const PoolFmt &f, unsigned long long w)
{
    return (int32_t)((w >> f.tb) & f.qmask);
}

// Arrival time of a packed flow read by the sweep at cycle time base.
__device__ __forceinline__ int32_t packed_ta(const PoolFmt &f, unsigned long long w, int32_t base)
{
    const uint32_t m = (1u << f.tb) - 1u;
    return base + (int32_t)(((uint32_t)w - (uint32_t)base) & m);
}

// One lane: starts the bulk copy of pool chunk `tile` (buffer ib) into input stage s.
// A chunk holds fill[ib][tile] flows; the copy is rounded up to 16 bytes and the slots
// past the fill are ignored.  An empty chunk completes the stage without a copy.
template <typename W>
__device__ __forceinline__ void issue_tile(const Params<W> &P, const PoolFmt &f, Smem &sm, int s, int ib, uint32_t tile)
{
    const uint32_t n = min((uint32_t)TILE, __ldcg(P.fill[ib] + tile));
    const uint32_t start = tile * (uint32_t)TILE;
    sm.stage_fill[s] = n;
    if (f.tb) {
        const uint32_t bytes = ((n + 1u) & ~1u) * 8u;
        mbar_expect_tx(&sm.mbar[s], bytes);
        if (bytes) bulk_g2s(sm.stage[s].qa, P.pk[ib] + start, bytes, &sm.mbar[s]);
        return;
    }
    const uint32_t bytes = ((n + 3u) & ~3u) * 4u;
    mbar_expect_tx(&sm.mbar[s], 3u * bytes);
    if (bytes) {
        bulk_g2s(sm.stage[s].ed, P.ed[ib] + start, bytes, &sm.mbar[s]);
        bulk_g2s(sm.stage[s].qa, P.qa[ib] + start, bytes, &sm.mbar[s]);
        bulk_g2s(sm.stage[s].ta, P.ta[ib] + start, bytes, &sm.mbar[s]);
    }
}

// The calling warp waits for stage s (bounded).  Returns false if the copy did not
// complete in time.
__device__ __forceinline__ bool wait_stage_warp(Smem &sm, int s, uint32_t parity)
{
    for (uint32_t i = 0; i < (1u << 22); i++)
        if (mbar_try_wait(&sm.mbar[s], parity)) return true;
    return false;
}

// After a failed wait: gives copies still in flight into any stage a last chance to land
// before the CTA leaves (thread 0; bounded).
__device__ __forceinline__ void drain_stages(Smem &sm, const uint32_t (&parity)[NSTAGE], const bool (&pending)[NSTAGE])
{
    if (threadIdx.x == 0)
        for (int s = 0; s < NSTAGE; s++)
            if (pending[s])
                for (uint32_t i = 0; i < (1u << 20) && !mbar_try_wait(&sm.mbar[s], parity[s]); i++) {
                }
}

struct LocalStats {
    uint32_t live, launched, improved, active, written, cands, phantoms;
    int min_ta;
};

// Adds this block's statistics to the pass counters (one global atomic per word per CTA).
__device__ __forceinline__ void flush_stats(const LocalStats &st, Counters *C)
{
    __shared__ unsigned long long s_live, s_li, s_oc, s_ph;
    __shared__ unsigned int s_act;
    __shared__ int s_min;
    if (threadIdx.x == 0) {
        s_live = 0;
        s_li = 0;
        s_oc = 0;
        s_ph = 0;
        s_act = 0;
        s_min = INT_MAX;
    }
    __syncthreads();
    uint32_t live = st.live, lau = st.launched, imp = st.improved, act = st.active, wr = st.written,
             cd = st.cands, ph = st.phantoms;
    int mn = st.min_ta;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        live += __shfl_xor_sync(0xffffffffu, live, o);
        lau += __shfl_xor_sync(0xffffffffu, lau, o);
        imp += __shfl_xor_sync(0xffffffffu, imp, o);
        act += __shfl_xor_sync(0xffffffffu, act, o);
        wr += __shfl_xor_sync(0xffffffffu, wr, o);
        cd += __shfl_xor_sync(0xffffffffu, cd, o);
        ph += __shfl_xor_sync(0xffffffffu, ph, o);
        mn = min(mn, __shfl_xor_sync(0xffffffffu, mn, o));
    }
    if ((threadIdx.x & 31) == 0) {
        if (live) atomicAdd(&s_live, (unsigned long long)live);
        if (lau | imp) atomicAdd(&s_li, (unsigned long long)lau | ((unsigned long long)imp << 32));
        if (wr | cd) atomicAdd(&s_oc, (unsigned long long)wr | ((unsigned long long)cd << 32));
        if (act) atomicAdd(&s_act, act);
        if (ph) atomicAdd(&s_ph, (unsigned long long)ph);
        if (mn != INT_MAX) atomicMin(&s_min, mn);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        if (s_live) atomicAdd(&C->live, s_live);
        if (s_li) atomicAdd(&C->lau_imp, s_li);
        if (s_oc) atomicAdd(&C->out_cand, s_oc);
        if (s_act) atomicAdd(&C->n_active, s_act);
        if (s_ph) atomicAdd(&C->phantoms, s_ph);
        if (s_min != INT_MAX) atomicMin(&C->min_ta, s_min);
    }
}

// ---------------------------------------------------------------- output cursor

__device__ __forceinline__ unsigned long long pack_cursor(uint32_t chunk, uint32_t fill)
{
    return ((unsigned long long)chunk << 32) | fill;
}

// Thread 0, at the start of a pass: the CTA's cursor opens on its first claim (a CTA that
// writes nothing allocates nothing).
__device__ __forceinline__ void cursor_open(Smem &sm)
{
    sm.cursor = pack_cursor(LAZY_CHUNK, 0);
    sm.next_chunk = NO_CHUNK;
}

// Slots [f0, f0 + n) of the CTA's output, the part from TILE on in chunk c1.
struct Span {
    uint32_t c0, f0, c1;
};

// Warp-collective (all lanes, n >= 1 the same in every lane): claims n consecutive output
// slots from the CTA's cursor with one shared-memory atomic.  The warp whose slots reach
// the end of the current chunk moves the cursor to the chunk allocated ahead and
// allocates the next one (a global atomic, off the other warps' path); a warp whose
// atomic landed past the end waits for that move and retries.  The filled chunk's entry
// of fill_out (the output buffer's fill array) becomes TILE.  Every wait is bounded: on
// give-up the span's chunks are OVF_CHUNK (writes dropped), sm.fail and ctl->err are set.
__device__ __forceinline__ Span claim_slots(Smem &sm, Counters *C, Control *ctl, uint32_t *fill_out, uint32_t n,
                                            uint32_t n_chunks)
{
    uint32_t c0 = OVF_CHUNK, f0 = 0, c1 = OVF_CHUNK;
    if ((threadIdx.x & 31) == 0) {
        volatile unsigned long long *vcur = &sm.cursor;
        volatile uint32_t *vnext = &sm.next_chunk;
        bool done = false;
        for (uint32_t tries = 0; tries < 4096u && !done; tries++) {
            const unsigned long long old = atomicAdd(&sm.cursor, (unsigned long long)n);
            const uint32_t id = hi32(old), f = lo32(old);
            if (id == LAZY_CHUNK) {
                if (f == 0) {  // the first claim of the pass: allocate this chunk and the next
                    const uint32_t c = atomicAdd(&C->chunks, 2u);
                    c0 = c < n_chunks ? c : OVF_CHUNK;
                    *vnext = c + 1 < n_chunks ? c + 1 : OVF_CHUNK;
                    __threadfence_block();
                    atomicExch(&sm.cursor, pack_cursor(c0, n));
                    f0 = 0;
                    done = true;
                } else {  // wait for the first claim to open the cursor
                    uint32_t spin = 0;
                    for (; spin < (1u << 22) && hi32(*vcur) == LAZY_CHUNK; spin++) __nanosleep(32);
                    if (spin >= (1u << 22)) break;
                }
            } else if (f + n < (uint32_t)TILE) {  // inside the current chunk
                c0 = id;
                f0 = f;
                done = true;
            } else if (f < (uint32_t)TILE) {  // this warp fills the chunk: move the cursor on
                uint32_t nx = NO_CHUNK;
                for (uint32_t spin = 0; spin < (1u << 22); spin++) {
                    const uint32_t v = *vnext;
                    if (v == OVF_CHUNK || (v != NO_CHUNK && v != id)) {  // (a stale value equals id)
                        nx = v;
                        break;
                    }
                    __nanosleep(32);
                }
                if (nx == NO_CHUNK) break;  // gave up
                *vnext = NO_CHUNK;
                __threadfence_block();
                atomicExch(&sm.cursor, pack_cursor(nx, f + n - (uint32_t)TILE));
                if (id < FIRST_SPECIAL) fill_out[id] = (uint32_t)TILE;
                c0 = id;
                f0 = f;
                c1 = nx;
                done = true;
                const uint32_t c = nx == OVF_CHUNK ? n_chunks : atomicAdd(&C->chunks, 1u);
                *vnext = c < n_chunks ? c : OVF_CHUNK;
            } else {
                // landed past the end: wait until the filling warp has moved the cursor
                uint32_t spin = 0;
                for (; spin < (1u << 22) && hi32(*vcur) == id; spin++) __nanosleep(32);
                if (spin >= (1u << 22)) break;
            }
        }
        if (!done) {
            c0 = c1 = OVF_CHUNK;
            f0 = 0;
            sm.fail = 1;
            atomicExch(&ctl->err, 1);
        }
    }
    Span sp;
    sp.c0 = __shfl_sync(0xffffffffu, c0, 0);
    sp.f0 = __shfl_sync(0xffffffffu, f0, 0);
    sp.c1 = __shfl_sync(0xffffffffu, c1, 0);
    return sp;
}

// Global slot of position p of a span (NO index if its chunk overflowed).
__device__ __forceinline__ bool span_slot(const Span &sp, uint32_t p, uint32_t &idx)
{
    const uint32_t c = p < (uint32_t)TILE ? sp.c0 : sp.c1;
    idx = c * (uint32_t)TILE + (p < (uint32_t)TILE ? p : p - (uint32_t)TILE);
    return c < FIRST_SPECIAL;
}

// Thread 0, after the pass's last write (a __syncthreads in between): records how full the
// CTA's last chunk is and marks the chunk allocated ahead as empty.
template <typename W>
__device__ __forceinline__ void cursor_close(const Params<W> &P, Smem &sm, int ob)
{
    if (threadIdx.x == 0) {
        const unsigned long long cur = sm.cursor;
        const uint32_t id = hi32(cur), nx = sm.next_chunk;
        if (id < FIRST_SPECIAL) P.fill[ob][id] = min(lo32(cur), (uint32_t)TILE);
        if (nx < FIRST_SPECIAL) P.fill[ob][nx] = 0u;
        // (a chunk past the pool was handed out but not written to: put_flow flags a lost flow)
        sm.cursor = pack_cursor(NO_CHUNK, 0);
        sm.next_chunk = NO_CHUNK;
    }
}

// 64-bit global store with an L2 cache policy.
__device__ __forceinline__ void st_policy64(unsigned long long *a, unsigned long long v, unsigned long long pol)
{
    asm volatile("st.global.L2::cache_hint.b64 [%0], %1, %2;" ::"l"(a), "l"(v), "l"(pol) : "memory");
}

// Writes one flow to slot p of a span (evict-first in L2), or records the overflow.
template <typename W>
__device__ __forceinline__ void put_flow(const Params<W> &P, const PoolFmt &f, int ob, Counters *C, const Span &sp,
                                         uint32_t p, uint32_t e, int32_t q, int32_t t)
{
    uint32_t idx;
    if (span_slot(sp, p, idx)) {
        const unsigned long long pol = policy_evict_first();
        if (f.tb) {
            st_policy64(P.pk[ob] + idx, pack_flow(f, e, q, t), pol);
        } else {
            st_policy(P.ed[ob] + idx, e, pol);
            st_policy(reinterpret_cast<uint32_t *>(P.qa[ob]) + idx, (uint32_t)q, pol);
            st_policy(reinterpret_cast<uint32_t *>(P.ta[ob]) + idx, (uint32_t)t, pol);
        }
    } else {
        atomicExch(&C->overflow, 1u);
    }
}

// A survivor of the sweep, copied from input stage s slot j to slot p of a span.
template <typename W>
__device__ __forceinline__ void copy_flow(const Params<W> &P, const PoolFmt &f, int ob, Counters *C, const Span &sp,
                                          uint32_t p, const Stage &in, uint32_t j, uint32_t e)
{
    uint32_t idx;
    if (span_slot(sp, p, idx)) {
        const unsigned long long pol = policy_evict_first();
        if (f.tb) {
            st_policy64(P.pk[ob] + idx, in.words()[j], pol);  // (ta mod 2^tb is unchanged)
        } else {
            st_policy(P.ed[ob] + idx, e, pol);
            st_policy(reinterpret_cast<uint32_t *>(P.qa[ob]) + idx, (uint32_t)in.qa[j], pol);
            st_policy(reinterpret_cast<uint32_t *>(P.ta[ob]) + idx, (uint32_t)in.ta[j], pol);
        }
    } else {
        atomicExch(&C->overflow, 1u);
    }
}

// ---------------------------------------------------------------- the sweep

// One pass over the flow pool (Steps 1-3 and 7-9 of the paper).  For every flow:
//   dead    if qa <= label[dst] (labels of the end of the previous cycle): dropped;
//   arrives if it is live and ta == Tg: offers (qa, ~(src*8+dir)) to dst with a 64-bit
//           atomic max (no return value needed) and is listed as a candidate in this
//           CTA's region; the launch phase finds, for each improved vertex, the one
//           candidate that won;
//   survives otherwise: copied to the output pool.
// Pool chunks (one tile each) arrive by bulk copies into NSTAGE shared-memory stages; the
// warps work through their slices of a tile independently (no block barrier in the
// loop): the last warp to finish reading a stage starts the copy of the tile after next
// into it, and each warp compacts its survivors and arrivals with ballots and claims
// output room with one shared-memory atomic.  With TRACE, live flows set their source's
// stamp (src_stamp = the pass number; counted by the launch phase).
// The CTA's output cursor must be open.  Returns false (uniformly across the CTA) if a
// bounded wait gave up (ctl->err set).
#ifndef CSP_PHASE_INLINE
#define CSP_PHASE_INLINE __forceinline__
#endif

template <int D, typename W, bool TRACE>
__device__ CSP_PHASE_INLINE bool sweep(const Params<W> &P, const Group &g, int ib, uint32_t n_tiles, int Tg,
                                       int tbase, uint32_t stamp, Counters *C, LocalStats &st, Smem &sm,
                                       uint32_t (&parity)[NSTAGE], uint32_t cand_base, uint32_t cand_cap)
{
    // tbase: a time no later than any arrival in the pool and within max f1 of all of them
    // (the cycle time; decodes the packed arrival times)
    const int ob = ib ^ 1;
    const PoolFmt fmt = pool_fmt(P);
    const uint32_t n_chunks = P.pool_cap / (uint32_t)TILE;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t lt = (1u << lane) - 1u;
    // Tiles are dealt round-robin: tile rank + k G goes to stage k mod NSTAGE.  (Claiming
    // tiles from a counter balanced the CTAs but its returning atomic on the refill path cost
    // more than the balance gained: 6.1 vs 5.2 s on a 2048^2 lattice.)
    const uint32_t G = g.size;
    const unsigned long long pol_labels = policy_evict_last();
    if (threadIdx.x == 0) {
        for (int s = 0; s < NSTAGE; s++) sm.read_cnt[s] = 0;
        sm.n_cand = 0;
        sm.fail = 0;
        if (g.rank < n_tiles) fence_proxy_async_global();  // pool written by ordinary stores in the previous pass
        for (int s = 0; s < NSTAGE; s++)
            if (g.rank + s * G < n_tiles) issue_tile(P, fmt, sm, s, ib, g.rank + s * G);
    }
    __syncthreads();
    bool ok = true;
    uint32_t k = 0;
    int s = 0;  // stage of the current tile (k mod NSTAGE)
    for (uint32_t tile = g.rank; tile < n_tiles; tile += G, k++, s = s + 1 == NSTAGE ? 0 : s + 1) {
        if (!wait_stage_warp(sm, s, parity[s])) {
            ok = false;
            break;
        }
        parity[s] ^= 1u;
        const uint32_t nfill = sm.stage_fill[s];
        uint32_t e[IPT];
        int32_t L[IPT];
#pragma unroll
        for (int i = 0; i < IPT; i++) {
            const uint32_t j = (uint32_t)(warp * (32 * IPT) + i * 32 + lane);
            e[i] = j >= nfill ? 0u : fmt.tb ? packed_ed(fmt, sm.stage[s].words()[j]) : sm.stage[s].ed[j];
        }
#pragma unroll
        for (int i = 0; i < IPT; i++) {
            const uint32_t j = (uint32_t)(warp * (32 * IPT) + i * 32 + lane);
            L[i] = j < nfill ? ld_policy(P.label + (e[i] >> 3), pol_labels) : INT_MAX;
        }
        uint32_t bk[IPT], ba[IPT];
        uint32_t nk = 0, na = 0;
#pragma unroll
        for (int i = 0; i < IPT; i++) {
            const uint32_t j = (uint32_t)(warp * (32 * IPT) + i * 32 + lane);
            const int32_t q = j >= nfill ? 0 : fmt.tb ? packed_qa(fmt, sm.stage[s].words()[j]) : sm.stage[s].qa[j];
            bool keep = false, arr = false;
            const bool live = q > L[i];  // (padding has q = 0 <= INT_MAX)
            if (TRACE && live) {  // the source is active in this pass (a plain store: every writer agrees)
                uint32_t sdir;
                P.src_stamp[flow_source<D>(P, e[i], sdir)] = stamp;
            }
            if (live) {
                st.live++;
                const uint32_t dst = e[i] >> 3;
                const int32_t t = fmt.tb ? packed_ta(fmt, sm.stage[s].words()[j], tbase) : sm.stage[s].ta[j];
                if (t == Tg) {
                    const unsigned long long key =
                        ((unsigned long long)(uint32_t)q << 32) | arrival_code<D>(P, e[i]);
                    atomicMax(P.offer + dst, key);
                    arr = true;
                } else {
                    keep = true;
                    st.min_ta = min(st.min_ta, t);
                    if (TRACE && P.edge_stamp) {  // this directed edge still carries a flow when the cycle launches
                        uint32_t sdir;
                        const uint32_t src = flow_source<D>(P, e[i], sdir);
                        P.edge_stamp[(size_t)src * nslots(D) + sdir] = stamp;
                    }
                }
            }
            bk[i] = __ballot_sync(0xffffffffu, keep);
            ba[i] = __ballot_sync(0xffffffffu, arr);
            nk += __popc(bk[i]);
            na += __popc(ba[i]);
        }
        if (na) {  // list the arrivals in this CTA's candidate region
            uint32_t cb = 0;
            if (lane == 0) cb = atomicAdd(&sm.n_cand, na);
            cb = __shfl_sync(0xffffffffu, cb, 0);
            st.cands += lane == 0 ? na : 0u;
#pragma unroll
            for (int i = 0; i < IPT; i++) {
                if ((ba[i] >> lane) & 1u) {
                    const uint32_t pos = cb + __popc(ba[i] & lt);
                    if (pos < cand_cap) P.cand[cand_base + pos] = e[i];
                    else atomicExch(&C->overflow, 1u);
                }
                cb += __popc(ba[i]);
            }
        }
        if (nk) {  // survivors to the output pool, in ballot order
            const Span sp = claim_slots(sm, C, P.ctl, P.fill[ob], nk, n_chunks);
            uint32_t p = sp.f0;
            st.written += lane == 0 ? nk : 0u;
#pragma unroll
            for (int i = 0; i < IPT; i++) {
                if ((bk[i] >> lane) & 1u) {
                    const uint32_t j = (uint32_t)(warp * (32 * IPT) + i * 32 + lane);
                    copy_flow(P, fmt, ob, C, sp, p + __popc(bk[i] & lt), sm.stage[s], j, e[i]);
                }
                p += __popc(bk[i]);
            }
        }
        // this warp is done with stage s; the last warp refills it with tile + NSTAGE G
        __threadfence_block();
        __syncwarp();
        if (lane == 0) {
            const uint32_t done = atomicAdd(&sm.read_cnt[s], 1u);
            if (done == (uint32_t)NWARP - 1u) {
                __threadfence_block();
                sm.read_cnt[s] = 0;
                if (tile + NSTAGE * G < n_tiles) {
                    fence_proxy_async_global();  // (this lane's view of the pool written last pass)
                    fence_proxy_async_smem();
                    issue_tile(P, fmt, sm, s, ib, tile + NSTAGE * G);
                }
            }
        }
    }
    bool pending[NSTAGE];
    // stages that may still receive a copy (only after a give-up): the next NSTAGE tiles
    for (int q = 0; q < NSTAGE; q++) pending[(s + q) % NSTAGE] = !ok && g.rank + (k + q) * G < n_tiles;
    if (!ok) {
        sm.fail = 1;
        atomicExch(&P.ctl->err, 1);
    }
    __syncthreads();
    if (sm.fail) {
        drain_stages(sm, parity, pending);
        return false;
    }
    return true;
}

// ---------------------------------------------------------------- the launch phase

template <typename W, int D>
__device__ __forceinline__ EdgeRecord<W, D> load_record(const uint4 *rec, uint32_t v)
{
    EdgeRecord<W, D> r;
#pragma unroll
    for (int i = 0; i < EdgeRecord<W, D>::VEC; i++) r.raw[i] = __ldg(rec + (size_t)v * EdgeRecord<W, D>::VEC + i);
    return r;
}

// Label of every neighbour of v (clamped index where the edge leaves the box; the value
// is then ignored because the record's f1 is 0).
template <int D, typename W>
__device__ __forceinline__ void neighbour_labels(const Params<W> &P, uint32_t V, uint32_t v, int (&Lw)[nslots(D)])
{
#pragma unroll
    for (int dir = 0; dir < nslots(D); dir++) {
        const uint32_t w = neighbour<D>(P, v, dir);
        Lw[dir] = __ldcg(reinterpret_cast<const int *>(P.offer + (w < V ? w : v)) + 1);  // label half of offer[w]
    }
}

// Water of quality Lv leaves v along each edge (v, w) with Lv - f2 > Label(w): returns
// the bit mask of those directions (Steps 4-5).
template <typename W, int D>
__device__ __forceinline__ uint32_t launch_mask(const EdgeRecord<W, D> &r, int Lv, const int (&Lw)[nslots(D)])
{
    uint32_t mask = 0;
#pragma unroll
    for (int dir = 0; dir < nslots(D); dir++)
        if (r.f1(dir) != 0 && Lv - r.f2(dir) > Lw[dir]) mask |= 1u << dir;
    return mask;
}

// Warp-collective: appends the flows of mask (per lane, one source vertex v with label Lv)
// to the output pool with one shared-memory claim per warp.  Each lane writes its flows to
// consecutive slots (so the flows of one source stay together for the trace count of
// later sweeps).
template <typename W, int D>
__device__ __forceinline__ void emit_flows(const Params<W> &P, const PoolFmt &f, int ob, Counters *C, Smem &sm, uint32_t v, int Lv,
                                           const EdgeRecord<W, D> &r, uint32_t mask, int Time, LocalStats &st)
{
    const int lane = threadIdx.x & 31;
    const uint32_t nk = __popc(mask);
    uint32_t incl = nk;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    const uint32_t total = __shfl_sync(0xffffffffu, incl, 31);
    if (total == 0) return;
    const Span sp = claim_slots(sm, C, P.ctl, P.fill[ob], total, P.pool_cap / (uint32_t)TILE);
    st.written += lane == 0 ? total : 0u;
    uint32_t p = sp.f0 + incl - nk;
#pragma unroll
    for (int dir = 0; dir < nslots(D); dir++)
        if (mask & (1u << dir)) {
            const int t = Time + r.f1(dir);
            put_flow(P, f, ob, C, sp, p, flow_word<D>(P, v, dir), Lv - r.f2(dir), t);
            p++;
            st.min_ta = min(st.min_ta, t);
            st.launched++;
        }
}

// One thread per arrival candidate of this CTA's region.  The candidate whose code equals
// the final offer word of its destination v is the winner: v improved this cycle (Step 2).
// The winner commits the label (Step 8), records v if it is in B (Algorithm 2), and starts
// a flow on every edge (v, w) with Label(v) - f2 > Label(w) under the labels at the end of
// this cycle (Steps 4-5; a flow on an edge that already carries water is the paper's
// phantom).  Its loads (offer[v], the edge record, the neighbour labels) are issued
// together.  Warps work independently.  With TRACE, also counts the vertices the sweep
// stamped with this pass.
template <int D, typename W, bool TRACE>
__device__ CSP_PHASE_INLINE void launch(const Params<W> &P, const Group &g, int ob, uint32_t cand_cta, bool with_cands,
                                        int Time, uint32_t stamp, Counters *C, LocalStats &st, Smem &sm)
{
    const uint32_t V = (uint32_t)P.V;
    const PoolFmt fmt = pool_fmt(P);
    if (TRACE) {  // active vertices: stamped by this pass's sweep (16-byte loads, 4 vertices each)
        const uint4 *st4 = reinterpret_cast<const uint4 *>(P.src_stamp);
        const uint32_t n4 = (V + 3) / 4;
        for (uint32_t i = g.rank * TPB + threadIdx.x; i < n4; i += g.size * TPB) {
            const uint4 x = __ldcg(st4 + i);
            st.active += (x.x == stamp) + (x.y == stamp) + (x.z == stamp) + (x.w == stamp);
        }
    }
    if (!with_cands) return;
    const uint32_t n_cand = min(sm.n_cand, cand_cta), cand_base = g.rank * cand_cta;
    const uint32_t wbase = (threadIdx.x >> 5) * 32u;
    for (uint32_t base = wbase; base < n_cand; base += TPB) {
        const uint32_t j = base + (threadIdx.x & 31);
        uint32_t v = 0, mask = 0, code = 0;
        int Lv = 0;
        bool won = false;
        EdgeRecord<W, D> r{};
        if (j < n_cand) {
            const uint32_t ec = __ldcg(P.cand + cand_base + j);
            v = ec >> 3;
            code = arrival_code<D>(P, ec);
            const unsigned long long ov = __ldcg(P.offer + v);
            r = load_record<W, D>(P.rec, v);
            int Lw[nslots(D)];
            neighbour_labels<D>(P, V, v, Lw);
            const uint32_t bw = __ldcg(P.isB + (v >> 5));  // (issued with the other loads)
            if (lo32(ov) == code) {  // the winning arrival at v
                won = true;
                Lv = (int)hi32(ov);
                if ((P.touched || P.first_t) && __ldcg(P.label + v) == 0) {  // the first improvement of v
                    if (P.touched) P.touched[atomicAdd(P.touched_n, 1u)] = v;
                    if (P.first_t) {
                        P.first_t[v] = Time;
                        P.first_code[v] = code;
                    }
                }
                P.label[v] = Lv;
                st.improved++;
                if ((bw >> (v & 31)) & 1u)
                    atomicMax(&C->xkey, ((unsigned long long)(uint32_t)Lv << 32) | (0xffffffffu - v));
                mask = launch_mask<W, D>(r, Lv, Lw);
                if (TRACE && P.edge_stamp) {  // a flow started on an edge that still carries one is a phantom (Step 5)
#pragma unroll
                    for (int dir = 0; dir < nslots(D); dir++)
                        if ((mask >> dir) & 1u)
                            st.phantoms += __ldcg(P.edge_stamp + (size_t)v * nslots(D) + dir) == stamp;
                }
            }
        }
        if (P.log) {  // every improvement, in this pass's segment of the log
            const uint32_t bw = __ballot_sync(0xffffffffu, won);
            if (bw) {
                const int lane = threadIdx.x & 31;
                unsigned long long base = 0;
                if (lane == 0) base = atomicAdd(P.log_n, (unsigned long long)__popc(bw));
                base = __shfl_sync(0xffffffffu, base, 0);
                const unsigned long long i = base + __popc(bw & ((1u << lane) - 1u));
                if (won && i < P.log_cap) P.log[i] = make_uint2(v, code);
            }
        }
        emit_flows<W, D>(P, fmt, ob, C, sm, v, Lv, r, mask, Time, st);
    }
}

// Seed launch (Algorithm 3): water of quality M leaves every source a in A (listed in
// cand as plain vertex ids, label M already set) along each edge with M - f2 > Label(w).
template <int D, typename W>
__device__ CSP_PHASE_INLINE void seed(const Params<W> &P, const Group &g, uint32_t n_src, Counters *C, LocalStats &st,
                                      Smem &sm)
{
    const uint32_t V = (uint32_t)P.V;
    const PoolFmt fmt = pool_fmt(P);
    const uint32_t wbase = g.rank * TPB + (threadIdx.x >> 5) * 32u;
    for (uint32_t base = wbase; base < n_src; base += g.size * TPB) {
        const uint32_t j = base + (threadIdx.x & 31);
        uint32_t v = 0, mask = 0;
        EdgeRecord<W, D> r{};
        if (j < n_src) {
            v = __ldcg(P.cand + j);
            r = load_record<W, D>(P.rec, v);
            int Lw[nslots(D)];
            neighbour_labels<D>(P, V, v, Lw);
            mask = launch_mask<W, D>(r, P.M, Lw);
        }
        emit_flows<W, D>(P, fmt, 0, C, sm, v, P.M, r, mask, 0, st);
    }
}

// ---------------------------------------------------------------- one solve

__device__ __forceinline__ void init_stage_barriers(Smem &sm)
{
    if (threadIdx.x == 0) {
        for (int s = 0; s < NSTAGE; s++) mbar_init(&sm.mbar[s], 1);
        mbar_init_fence();
    }
    __syncthreads();
}

template <typename W>
__device__ void write_row(const Params<W> &P, long long row, long long time, long long active, long long flows)
{
    if (P.trace && row < P.trace_cap) {
        P.trace[3 * row] = time;
        P.trace[3 * row + 1] = active;
        P.trace[3 * row + 2] = flows;
    }
}

__device__ __forceinline__ void zero_counters(Counters *c)
{
    c->out_cand = c->live = c->lau_imp = c->xkey = 0;
    c->n_active = c->overflow = c->abort = c->chunks = 0;
    c->phantoms = 0;
    c->min_ta = INT_MAX;
}

// A snapshot of one pass's counters, read by every CTA after the pass's last barrier.
struct PassCounts {
    unsigned int n_out, n_cand, launched, improved, n_active, overflow, abort, chunks;
    unsigned long long n_live, xkey, phantoms;
    int min_ta;
};

// Thread 0 reads the pass counters with independent L2 loads (one round trip in all) and
// shares them through shared memory; every CTA gets the same values after the pass's
// barrier.  (Volatile loads by every thread would cost one serialised round trip per
// field per warp.)
__device__ __forceinline__ PassCounts read_counters(const Counters *c)
{
    __shared__ PassCounts s_pc;
    if (threadIdx.x == 0) {
        const unsigned long long oc = __ldcg(&c->out_cand), li = __ldcg(&c->lau_imp);
        const unsigned long long lv = __ldcg(&c->live), xk = __ldcg(&c->xkey);
        const unsigned int act = __ldcg(&c->n_active), ovf = __ldcg(&c->overflow), ab = __ldcg(&c->abort);
        const int mt = __ldcg(&c->min_ta);
        s_pc.chunks = __ldcg(&c->chunks);
        s_pc.phantoms = __ldcg(&c->phantoms);
        s_pc.n_out = lo32(oc);
        s_pc.n_cand = hi32(oc);
        s_pc.launched = lo32(li);
        s_pc.improved = hi32(li);
        s_pc.n_live = lv;
        s_pc.xkey = xk;
        s_pc.n_active = act;
        s_pc.overflow = ovf;
        s_pc.abort = ab;
        s_pc.min_ta = mt;
    }
    __syncthreads();
    const PassCounts r = s_pc;
    __syncthreads();  // s_pc may be rewritten by the next call
    return r;
}

// One counter word read by thread 0 and shared (see read_counters).
__device__ __forceinline__ unsigned long long read_shared_u64(const unsigned long long *p)
{
    __shared__ unsigned long long s_v;
    if (threadIdx.x == 0) s_v = __ldcg(p);
    __syncthreads();
    const unsigned long long v = s_v;
    __syncthreads();
    return v;
}

// Runs one whole solve (the cycle loop of Algorithm 1) on the CTAs of group g.  The
// set-up must be complete: labels and offers (M on A, 0 elsewhere), the B bitmap, the
// distinct sources listed in cand with their count in the high half of cnt[0].out_cand,
// and fresh counters.  The group leader writes the result record.
template <int D, typename W, bool TRACE>
__device__ void run_solve(const Params<W> &P, const Group &g, Smem &sm, uint32_t (&parity)[NSTAGE],
                          unsigned long long &epoch)
{
    // epoch: barriers already passed on ctl->bar (updated)
    Control *ctl = P.ctl;
    const bool leader = g.leader();
    const int M = P.M;
    const unsigned long long t_start = globaltimer_ns();

    long long cycle = 0, updates = 0, launched = 0, passes = 0, trace_len = 0, arrivals = 0, improved = 0,
              phantoms = 0;
    unsigned int max_pool = 0;
    int Time = 0, status = ST_OK;
    bool feasible = false;
    unsigned long long xkey = 0;

    if (P.test_absent && g.size > 1 && g.rank == g.size - 1) return;  // (test hook: see Params)
    if (*(volatile int *)&ctl->status_in != 0) {
        status = *(volatile int *)&ctl->status_in;
        goto finish;
    }
    if (M <= 0) {  // no walk has F2 < M <= 0
        trace_len = 1;
        if (leader) write_row(P, 0, 0, 0, 0);
        goto finish;
    }

    {
        const uint32_t n_chunks = P.pool_cap / (uint32_t)TILE;
        const uint32_t cand_cta = P.cand_cap / g.size;  // candidate region of each CTA
        const uint32_t cand_base = g.rank * cand_cta;
        // seed: water leaves A at Time 0 along every edge that can raise a label
        LocalStats st{0, 0, 0, 0, 0, 0, 0, INT_MAX};
        const uint32_t n_src = min(hi32(read_shared_u64(&ctl->cnt[0].out_cand)), P.cand_cap);
        // (the seed adds the flows it writes to the low half of out_cand; the high half keeps n_src)
        if (threadIdx.x == 0) cursor_open(sm);
        __syncthreads();
        seed<D, W>(P, g, n_src, &ctl->cnt[0], st, sm);
        __syncthreads();
        cursor_close(P, sm, 0);
        flush_stats(st, &ctl->cnt[0]);
        if (!group_sync(ctl, epoch, g, P.barrier_ns)) { status = ST_BARRIER; goto finish; }
        const PassCounts c = read_counters(&ctl->cnt[0]);
        launched += (long long)c.launched;
        if (c.overflow) { status = ST_CAPACITY; goto finish; }
        if (c.n_out == 0) {  // nothing can leave A: infeasible
            if (leader) write_row(P, 0, 0, 0, 0);
            trace_len = 1;
            goto finish;
        }
        max_pool = c.n_out;
        int Tg = c.min_ta;
        // pool chunks the next sweep reads (chunks handed out past the pool hold no flow)
        uint32_t n_tiles = min(c.chunks, n_chunks);

        for (long long pass = 1;; pass++) {
            const int ib = (int)((pass - 1) & 1), ob = ib ^ 1;
            Counters *C = &ctl->cnt[ob];
            LocalStats sa{0, 0, 0, 0, 0, 0, 0, INT_MAX};
            if (threadIdx.x == 0) cursor_open(sm);
            if (!sweep<D, W, TRACE>(P, g, ib, n_tiles, Tg, Tg, (uint32_t)pass, C, sa, sm, parity, cand_base, cand_cta)) {
                status = ST_BARRIER;
                goto finish;
            }
            flush_stats(sa, C);
            if (!group_sync(ctl, epoch, g, P.barrier_ns)) { status = ST_BARRIER; goto finish; }
            if (leader) zero_counters(&ctl->cnt[ib]);  // everyone has read the input's counts
            if (leader && P.log && pass < P.pass_cap) {  // this pass's log segment starts here
                P.pass_time[pass] = Tg;
                P.pass_off[pass] = *(volatile unsigned long long *)P.log_n;
            }
            if (leader && globaltimer_ns() - t_start > P.budget_ns) C->abort = 1u;  // read by all after the barrier
            LocalStats sb{0, 0, 0, 0, 0, 0, 0, INT_MAX};
            launch<D, W, TRACE>(P, g, ob, cand_cta, true, Tg, (uint32_t)pass, C, sb, sm);
            __syncthreads();
            cursor_close(P, sm, ob);
            flush_stats(sb, C);
            if (!group_sync(ctl, epoch, g, P.barrier_ns)) { status = ST_BARRIER; goto finish; }
            passes = pass;

            const PassCounts c = read_counters(C);
            if (c.overflow) { status = ST_CAPACITY; goto finish; }
            if (c.abort) {  // rows 0 .. cycle - 1 are complete; the counts are those of cycles 1 .. cycle
                status = ST_TIMEOUT;
                trace_len = cycle;
                goto finish;
            }
            launched += (long long)c.launched;
            arrivals += (long long)c.n_cand;
            improved += (long long)c.improved;
            phantoms += (long long)c.phantoms;
            if (c.n_cand > 0) {  // a real cycle at time Tg
                if (TRACE && leader) write_row(P, cycle, Time, c.n_active, (long long)c.n_live);
                updates += (long long)c.n_live;
                cycle++;
                Time = Tg;
                if (c.xkey) {  // a vertex of B improved: F1 = Time (Algorithm 2)
                    feasible = true;
                    xkey = c.xkey;
                    if (TRACE) {
                        // the terminal cycle's row: count the flows still alive after it
                        LocalStats sc{0, 0, 0, 0, 0, 0, 0, INT_MAX};
                        const uint32_t nt = min(c.chunks, n_chunks);
                        if (threadIdx.x == 0) cursor_open(sm);
                        if (!sweep<D, W, TRACE>(P, g, ob, nt, -1, Time, (uint32_t)pass + 1u, &ctl->cnt[ib], sc, sm, parity, cand_base,
                                                cand_cta)) {
                            status = ST_BARRIER;
                            goto finish;
                        }
                        flush_stats(sc, &ctl->cnt[ib]);
                        if (!group_sync(ctl, epoch, g, P.barrier_ns)) { status = ST_BARRIER; goto finish; }
                        LocalStats sd{0, 0, 0, 0, 0, 0, 0, INT_MAX};
                        launch<D, W, TRACE>(P, g, ib, cand_cta, false, Time, (uint32_t)pass + 1u, &ctl->cnt[ib], sd, sm);  // count sources
                        __syncthreads();
                        cursor_close(P, sm, ib);
                        flush_stats(sd, &ctl->cnt[ib]);
                        if (!group_sync(ctl, epoch, g, P.barrier_ns)) { status = ST_BARRIER; goto finish; }
                        const PassCounts cc = read_counters(&ctl->cnt[ib]);
                        if (leader) write_row(P, cycle, Time, cc.n_active, (long long)cc.n_live);
                        trace_len = cycle + 1;
                    }
                    goto finish;
                }
            } else if (c.n_live == 0) {  // the pool held no live flow: infeasible
                if (TRACE && leader) write_row(P, cycle, Time, 0, 0);
                trace_len = cycle + 1;
                goto finish;
            }
            if (c.n_out == 0) {  // no flow left after a cycle: infeasible
                if (TRACE && leader) write_row(P, cycle, Time, 0, 0);
                trace_len = cycle + 1;
                goto finish;
            }
            max_pool = max(max_pool, c.n_out);
            n_tiles = min(c.chunks, n_chunks);
            Tg = c.min_ta;
            if (P.max_cycles > 0 && cycle >= P.max_cycles) {  // rows 0 .. cycle - 1 are complete
                status = ST_TIMEOUT;
                trace_len = cycle;
                goto finish;
            }
            if (Tg >= TIME_LIMIT) { status = ST_CAPACITY; goto finish; }
        }
    }

finish:
    if (leader && P.log && passes + 1 <= P.pass_cap) P.pass_off[passes + 1] = *(volatile unsigned long long *)P.log_n;
    if (leader) {
        long long *o = ctl->out;
        for (int i = 0; i < R_COUNT; i++) o[i] = -1;
        o[R_STATUS] = status;
        if (status == ST_OK && feasible) {
            const uint32_t X = 0xffffffffu - (uint32_t)(xkey & 0xffffffffu);
            const int LX = (int)(xkey >> 32);
            const uint32_t code = 0xffffffffu - (uint32_t)(__ldcg(P.offer + X) & 0xffffffffu);
            o[R_F1] = Time;
            o[R_X] = X;
            o[R_XSRC] = code >> 3;
            o[R_XDIR] = code & 7u;
            o[R_F2] = (long long)M - LX;
        }
        o[R_CYCLES] = cycle;
        o[R_UPDATES] = updates;
        o[R_LAUNCHED] = launched;
        o[R_PASSES] = passes;
        o[R_MAXPOOL] = max_pool;
        o[R_TRACELEN] = TRACE ? trace_len : 0;
        o[R_ARRIVALS] = arrivals;
        o[R_IMPROVED] = improved;
        o[R_PHANTOMS] = TRACE && P.edge_stamp ? phantoms : -1;
        o[R_ELAPSED_NS] = (long long)(globaltimer_ns() - t_start);
        if (P.result_dev)
            for (int i = 0; i < R_COUNT; i++) P.result_dev[i] = o[i];
    }
}

// ---------------------------------------------------------------- set-up inside a kernel

// Targets of a solve started inside a kernel: an explicit id list, or the hyperplane
// {v : c_axis(v) = coord} (axis >= 0).
struct TargetSet {
    const int64_t *list64;
    const uint32_t *list32;
    long long n;
    int axis;
    long long coord;
};

// Initialization (Algorithm 3) by the CTAs of group g, for solves started inside a
// persistent kernel: labels and offers cleared, B marked, Label(a) = M on A (the offer
// word mirrors it) and the distinct sources listed in cand for the seed launch.  Invalid
// ids or A and B overlapping set ctl->status_in.  Returns false if a barrier failed.
// General form: sources as int64 (A64) or uint32 (A32) ids, targets as a TargetSet.
// (A hyperplane needs the lattice's extents; they are recovered from the strides, so
// stride[axis + 1] must be set for axis < d - 1 and 0 beyond the last dimension.)
template <typename W>
__device__ bool group_setup_sets(const Params<W> &P, const Group &g, const int64_t *A64, const uint32_t *A32,
                                 long long nA, const TargetSet &T, unsigned long long &epoch, bool clear = true)
{
    // clear = false: labels, offers and the B bitmap are already zero (the previous
    // solve on this workspace was undone by group_undo)
    Control *ctl = P.ctl;
    const long long V = P.V;
    const long long t0 = (long long)g.rank * TPB + threadIdx.x, step = (long long)g.size * TPB;
    if (clear) {
        for (long long i = t0; i < V; i += step) {
            P.label[i] = 0;
            P.offer[i] = 0ull;
        }
        for (long long i = t0; i < (V + 31) / 32; i += step) const_cast<uint32_t *>(P.isB)[i] = 0u;
    }
    if (g.leader()) {
        ctl->status_in = 0;
        for (int b = 0; b < 2; b++) {
            Counters &c = ctl->cnt[b];
            c.out_cand = c.live = c.lau_imp = c.xkey = 0;
            c.n_active = c.overflow = c.abort = c.chunks = 0;
            c.phantoms = 0;
            c.min_ta = INT_MAX;
        }
    }
    if (!group_sync(ctl, epoch, g, P.barrier_ns)) return false;
    if (T.axis >= 0) {
        // hyperplane c_axis = coord: ids hi * (stride * n) + coord * stride + lo
        const long long st = P.stride[T.axis];
        const long long nk = T.axis + 1 < 4 && P.stride[T.axis + 1] ? P.stride[T.axis + 1] / st : V / st;
        const long long count = V / nk;
        if (T.coord < 0 || T.coord >= nk) {
            if (g.leader()) atomicExch(&ctl->status_in, ST_INVALID);
        } else {
            for (long long i = t0; i < count; i += step) {
                const long long b = (i / st) * st * nk + T.coord * st + (i % st);
                atomicOr(const_cast<uint32_t *>(P.isB) + (b >> 5), 1u << (b & 31));
            }
        }
    } else {
        for (long long i = t0; i < T.n; i += step) {
            const long long b = T.list64 ? T.list64[i] : (long long)T.list32[i];
            if (b < 0 || b >= V) atomicExch(&ctl->status_in, ST_INVALID);
            else atomicOr(const_cast<uint32_t *>(P.isB) + (b >> 5), 1u << (b & 31));
        }
    }
    if (!group_sync(ctl, epoch, g, P.barrier_ns)) return false;
    const unsigned long long key = ((unsigned long long)(uint32_t)P.M << 32) | 0xffffffffull;
    for (long long i = t0; i < nA; i += step) {
        const long long a = A64 ? A64[i] : (long long)A32[i];
        if (a < 0 || a >= V) {
            atomicExch(&ctl->status_in, ST_INVALID);
            continue;
        }
        if ((__ldcg(P.isB + (a >> 5)) >> (a & 31)) & 1u) {
            atomicExch(&ctl->status_in, ST_INVALID);  // A and B must be disjoint
            continue;
        }
        P.label[a] = P.M;
        if (atomicExch(P.offer + a, key) != key) {
            const unsigned int slot = hi32(atomicAdd(&ctl->cnt[0].out_cand, 1ull << 32));
            if (slot < P.cand_cap) P.cand[slot] = (uint32_t)a;
            else atomicExch(&ctl->status_in, ST_CAPACITY);
        }
    }
    return group_sync(ctl, epoch, g, P.barrier_ns);
}

template <typename W>
__device__ bool group_setup(const Params<W> &P, const Group &g, const int64_t *A, long long nA, const int64_t *B,
                            long long nB, unsigned long long &epoch)
{
    return group_setup_sets<W>(P, g, A, nullptr, nA, TargetSet{B, nullptr, nB, -1, 0}, epoch);
}

// Returns a workspace to all-zero labels, offers and B bitmap after a solve, touching
// only what the solve changed: the vertices in P.touched (first improvements), the
// sources and the targets.  Much cheaper than clearing V entries when a solve reaches a
// small part of a large lattice.  Ends with a group barrier.
template <typename W>
__device__ bool group_undo(const Params<W> &P, const Group &g, const uint32_t *A32, long long nA, const TargetSet &T,
                           unsigned long long &epoch)
{
    const long long t0 = (long long)g.rank * TPB + threadIdx.x, step = (long long)g.size * TPB;
    const long long nt = (long long)*(volatile unsigned int *)P.touched_n;
    for (long long i = t0; i < nt; i += step) {
        const uint32_t v = __ldcg(P.touched + i);
        P.label[v] = 0;
        P.offer[v] = 0ull;
    }
    for (long long i = t0; i < nA; i += step) {
        const uint32_t a = A32[i];
        if (a < (uint32_t)P.V) {
            P.label[a] = 0;
            P.offer[a] = 0ull;
        }
    }
    uint32_t *isB = const_cast<uint32_t *>(P.isB);
    if (T.axis >= 0) {
        const long long st = P.stride[T.axis];
        const long long nk = T.axis + 1 < 4 && P.stride[T.axis + 1] ? P.stride[T.axis + 1] / st : P.V / st;
        const long long count = P.V / nk;
        if (T.coord >= 0 && T.coord < nk)
            for (long long i = t0; i < count; i += step) {
                const long long b = (i / st) * st * nk + T.coord * st + (i % st);
                isB[b >> 5] = 0u;  // every bit set in this word belongs to the hyperplane
            }
    } else {
        for (long long i = t0; i < T.n; i += step) {
            const long long b = T.list64 ? T.list64[i] : (long long)T.list32[i];
            if (b >= 0 && b < P.V) isB[b >> 5] = 0u;  // only target bits were set
        }
    }
    if (!group_sync(P.ctl, epoch, g, P.barrier_ns)) return false;
    if (g.leader()) *P.touched_n = 0u;
    return group_sync(P.ctl, epoch, g, P.barrier_ns);
}

}  // namespace csp
