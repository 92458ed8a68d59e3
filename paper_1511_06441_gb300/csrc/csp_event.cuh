// Device side of the event-driven cycle: the loop of Algorithm 1 driven by a calendar of
// arrival times instead of a sweep over every flow in flight.
//
// The sweep form (csp_device.cuh) visits every flow in every cycle, as Step 1 decrements
// every remaining time.  Here a flow is visited only when something happens to it: when
// it arrives, and when the label of its destination rises far enough to make it useless
// (Steps 7-9).  Three structures make that possible.
//
//   Edge queues.  Per directed edge e = v * S + dir (S slots per vertex) a FIFO of the
//     flows in flight on it, in a ring of f1(e) entries (quality on arrival, arrival
//     time).  Flows on one edge start at distinct cycle times and each stays f1(e) time
//     units, so at most f1(e) are in flight; they arrive in launch order and carry rising
//     qualities (labels only increase), so arrivals and removals both take from the
//     front.  edge[e] = {tail, ring offset, head, f1 | f2 << 16}; tail and head count the
//     pushes and pops (entry number s sits at ring offset + s mod f1).
//   Calendar.  For each arrival time t, kept modulo W = max f1 + 1, a list of bucket
//     entries (flow word, quality on arrival) in chunks of EV_CH entries taken from a
//     free stack; chunk lists are indexed by t mod 2W so that a round's list is never
//     reused while it is read.  blive[t mod W] counts the listed flows still in flight;
//     the next cycle time is the first t with blive > 0.
//   Running counts.  Flows in flight and, with a trace, per vertex the flows in flight
//     leaving it, whence the number of active vertices, all exact at every cycle end.
//
// One cycle at time T is two phases between grid barriers:
//   A (Steps 1-3).  The entries of round T.  An entry whose quality still exceeds the
//     label of its destination (labels of the end of the previous cycle) is the front
//     flow of its edge arriving now: it is popped, offers its water to the destination
//     with the same 64-bit atomicMax as the sweep form and is listed as a candidate.  The
//     other entries belong to flows removed earlier and are skipped.  The round's chunks
//     (and those of rounds passed without a cycle) go back to the free stack.
//   B (Steps 2, 4, 5, 7-9).  The candidate whose code equals its destination's final
//     offer word is the unique winner: it commits the label, starts a flow on every edge
//     that can still raise a label (pushed on the edge's queue and listed in the round of
//     its arrival time) and removes from the front of every queue into its vertex the
//     flows whose quality no longer exceeds the new label.
// A push and a removal may meet on the same edge in phase B (u improves and launches
// towards v while v improves).  They touch different counters (tail, head), the new
// flow is never one to remove (its quality exceeds the new label of v), and a removal
// stops at an entry that arrives by the current time: the slot a concurrent push is
// filling held a flow that arrived at least f1 time units after its start, so its old
// contents look arrived, never in flight.  No fence is needed for that.
#pragma once

#include "csp_device.cuh"

namespace csp {

constexpr int EV_CH = 512;          // bucket entries per chunk
constexpr int EV_WMAX = 512;        // largest calendar window W = max f1 + 1
constexpr int EV_BATCH = 64;        // chunks whose ids a CTA stages in shared memory at a time
constexpr uint32_t EV_WIN = 0x80000000u;

// Running totals of one event-driven solve.  Words updated by many CTAs sit on lines of
// their own.
struct EvCtl {
    alignas(128) long long live;     // flows in flight
    alignas(128) long long active;   // vertices that source a flow in flight (trace mode)
    alignas(128) int free_top;       // chunk ids on the free stack
    alignas(128) unsigned long long phase_ns[4];  // leader's time in set-up, phase A, phase B, barriers
};

struct EvParams {
    uint4 *edge;          // [S V] per directed edge: x = tail, y = ring offset, z = head, w = f1 | f2 << 16
    uint2 *ring;          // queue entries: (quality on arrival, arrival time); zero at the start of a solve
    uint2 *bent;          // bucket entries [nch][EV_CH]: (flow word, quality on arrival)
    uint32_t *bfill;      // [nch] entries written in each chunk
    uint32_t *freestk;    // [nch] free chunk ids (stack of free_top entries)
    uint32_t *bdir;       // [2 W][nch] chunks of each round (arrival time mod 2W)
    uint32_t *bcount;     // [2 W] chunks listed per round
    int32_t *blive;       // [W] flows in flight per arrival time mod W
    int32_t *out_count;   // [V] trace mode: flows in flight leaving each vertex
    EvCtl *ev;
    uint32_t nch;         // chunks in the pool
    int W;                // calendar window: max f1 + 1 (<= EV_WMAX)
};

constexpr int EV_STASH = 64;       // free chunk ids a CTA keeps at hand
constexpr int EV_NEWMAX = 8;       // chunks a CTA opens for one arrival time before listing them

// Shared memory of the event kernel.  Per arrival time b = t mod W (one time of the window
// (T, T + W) each): cursor[b] = the CTA's open chunk (high half; NO_CHUNK = none) and the
// entries written to it (low half), persistent across cycles and closed when the round of t
// comes up; newl[b] = chunks opened for t since the last listing (listed in the round's
// directory at the end of each phase); hist[b] = this phase's change of blive[b]; bcnt and
// bspan serve one append step.  Chunk ids come from a stash refilled from the free stack
// once per phase.
struct EvSmem {
    unsigned long long cursor[EV_WMAX];
    int hist[EV_WMAX];
    uint32_t bcnt[EV_WMAX];
    uint4 bspan[EV_WMAX];                  // (open chunk, first entry, entries there, first new index)
    uint32_t newl[EV_WMAX][EV_NEWMAX];
    uint32_t nnew[EV_WMAX];
    uint32_t dirty[EV_WMAX / 32];          // arrival times appended to in this phase
    uint32_t stash[EV_STASH];
    int stash_n;
    uint32_t chunk_id[EV_BATCH];
    uint32_t chunk_n[EV_BATCH];
    uint32_t free_base;
    uint32_t n_cand;
    int fail;
};

struct EvLocal {
    long long live_delta;
    int act_delta;
    uint32_t cands, improved, launched, phantoms;
};

__device__ __forceinline__ void ev_local_zero(EvLocal &s)
{
    s.live_delta = 0;
    s.act_delta = 0;
    s.cands = s.improved = s.launched = s.phantoms = 0;
}

// The time of the window (T, T + W) whose value mod W is b (b != T mod W).
__device__ __forceinline__ uint32_t ev_round_time(uint32_t b, int T, uint32_t Wn)
{
    return (uint32_t)T + (b + Wn - (uint32_t)T % Wn) % Wn;
}

// Thread 0, at the start of a phase that appends: tops the CTA's stash up from the free
// stack (one atomic).  A free stack that cannot supply it marks the solve as overflowed.
__device__ __forceinline__ void ev_refill_stash(EvSmem &sm, const EvParams &E, Counters *C)
{
    if (threadIdx.x != 0 || sm.stash_n > EV_STASH / 2) return;
    const int need = EV_STASH - sm.stash_n;
    const int old = atomicSub(&E.ev->free_top, need);
    if (old < need) {
        atomicExch(&C->overflow, 1u);
        return;
    }
    for (int i = 0; i < need; i++) sm.stash[sm.stash_n + i] = __ldcg(E.freestk + old - need + i);
    sm.stash_n += need;
}

// A chunk id from the stash (any thread; the free stack directly when the stash is empty).
__device__ __forceinline__ uint32_t ev_take_chunk(EvSmem &sm, const EvParams &E, Counters *C)
{
    const int i = atomicSub(&sm.stash_n, 1) - 1;
    if (i >= 0) return sm.stash[i];
    atomicAdd(&sm.stash_n, 1);
    const int pos = atomicSub(&E.ev->free_top, 1) - 1;
    if (pos >= 0) return __ldcg(E.freestk + pos);
    atomicExch(&C->overflow, 1u);
    return OVF_CHUNK;
}

// Lists the chunks opened for arrival time b in the directory of its round (one atomic).
__device__ __forceinline__ void ev_list_new(EvSmem &sm, const EvParams &E, uint32_t b, int T)
{
    const uint32_t m = sm.nnew[b];
    if (!m) return;
    const uint32_t Wn = (uint32_t)E.W;
    const uint32_t ridx = ev_round_time(b, T, Wn) % (2u * Wn);
    const uint32_t k = atomicAdd(E.bcount + ridx, m);
    for (uint32_t i = 0; i < m; i++)
        if (sm.newl[b][i] < FIRST_SPECIAL) E.bdir[(size_t)ridx * E.nch + k + i] = sm.newl[b][i];
    sm.nnew[b] = 0;
}

// CTA-collective append step at cycle time T.  Before it, every thread took the ranks of
// its entries (atomicAdd on bcnt[t mod W]).  One thread per arrival time reserves room for
// all of them: the rest of the open chunk, then whole new chunks from the stash.  After
// it, every thread writes its entries with ev_append_slot.  Returns false (uniformly) if
// no thread had an entry.
__device__ __forceinline__ bool ev_append_claim(EvSmem &sm, const EvParams &E, Counters *C, int T, bool any)
{
    if (!__syncthreads_or(any)) return false;
    const uint32_t Wn = (uint32_t)E.W;
    for (uint32_t b = threadIdx.x; b < Wn; b += TPB) {
        const uint32_t n = sm.bcnt[b];
        if (!n) continue;
        const unsigned long long cur = sm.cursor[b];
        const uint32_t id = hi32(cur), f = lo32(cur);
        const uint32_t room = id < FIRST_SPECIAL ? (uint32_t)EV_CH - f : 0u;
        const uint32_t take0 = min(n, room), rest = n - take0;
        const uint32_t m = (rest + EV_CH - 1) / EV_CH;
        if (sm.nnew[b] + m > (uint32_t)EV_NEWMAX) ev_list_new(sm, E, b, T);
        const uint32_t first = sm.nnew[b];
        uint32_t last = id, fill = f + take0;
        for (uint32_t i = 0; i < m; i++) {
            last = ev_take_chunk(sm, E, C);
            sm.newl[b][first + i] = last;
            if (i + 1 < m && last < FIRST_SPECIAL) E.bfill[last] = (uint32_t)EV_CH;
        }
        if (m) fill = rest - (m - 1) * (uint32_t)EV_CH;
        if (id < FIRST_SPECIAL && f + take0 == (uint32_t)EV_CH) E.bfill[id] = (uint32_t)EV_CH;
        sm.nnew[b] = first + m;
        sm.cursor[b] = pack_cursor(last, fill);
        sm.bspan[b] = make_uint4(id, f, take0, first);
        sm.hist[b] += (int)n;
        atomicOr(&sm.dirty[b >> 5], 1u << (b & 31));
        sm.bcnt[b] = 0u;
    }
    __syncthreads();
    return true;
}

// Where entry `rank` of arrival time b goes after ev_append_claim (false: dropped).
__device__ __forceinline__ bool ev_append_slot(const EvSmem &sm, uint32_t b, uint32_t rank, size_t &idx)
{
    const uint4 q = sm.bspan[b];
    uint32_t c, o;
    if (rank < q.z) {
        c = q.x;
        o = q.y + rank;
    } else {
        const uint32_t p = rank - q.z;
        c = sm.newl[b][q.w + p / EV_CH];
        o = p % EV_CH;
    }
    idx = (size_t)c * EV_CH + o;
    return c < FIRST_SPECIAL;
}

// CTA-collective: the thread's vertex v (label Lv, edge record r) starts a flow on every
// direction of mask at time T (Steps 4-5): the flow is pushed on the edge's queue and
// listed in the calendar under its arrival time.  With phantoms (a stamp array and a
// nonzero stamp), a flow started on an edge that still carries one after the cycle's
// arrivals is counted (Step 5's phantom edge; see the head and stamp protocol of
// ev_remove_into).
template <int D, typename W, bool TRACE>
__device__ __forceinline__ void ev_push_flows(const Params<W> &P, const EvParams &E, EvSmem &sm, Counters *C, uint32_t v,
                                              int Lv, const EdgeRecord<W, D> &r, uint32_t mask, int T, uint32_t stamp,
                                              EvLocal &st)
{
    constexpr int S = nslots(D);
    const uint32_t Wn = (uint32_t)E.W;
    // every load first (a load placed after a store to another array could not be hoisted
    // above it, and each launching direction would cost a round trip of its own)
    uint2 tq[S];  // (tail, ring offset) of each launching out-edge
    uint32_t words[S], heads[S], stamps[S];
#pragma unroll
    for (int dir = 0; dir < S; dir++) {
        const bool want = (mask >> dir) & 1u;
        const size_t e = (size_t)v * S + dir;
        tq[dir] = want ? __ldcg(reinterpret_cast<const uint2 *>(E.edge + e)) : make_uint2(0u, 0u);
        words[dir] = want ? flow_word<D>(P, v, dir) : 0u;
        heads[dir] = stamps[dir] = 0u;
        if (TRACE && P.edge_stamp && want) {
            asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(heads[dir]) : "l"(&E.edge[e].z) : "memory");
            stamps[dir] = __ldcg(P.edge_stamp + e);
        }
    }
    uint32_t rank[S];
#pragma unroll
    for (int dir = 0; dir < S; dir++) {
        rank[dir] = 0u;
        if ((mask >> dir) & 1u) {
            const size_t e = (size_t)v * S + dir;
            const int f1 = r.f1(dir);
            const int32_t qa = Lv - r.f2(dir);
            const int ta = T + f1;
            if (TRACE && P.edge_stamp && (heads[dir] != tq[dir].x || (stamp != 0u && stamps[dir] == stamp)))
                st.phantoms++;
            E.ring[tq[dir].y + tq[dir].x % (uint32_t)f1] = make_uint2((uint32_t)qa, (uint32_t)ta);
            E.edge[e].x = tq[dir].x + 1u;
            rank[dir] = atomicAdd(&sm.bcnt[(uint32_t)ta % Wn], 1u);
        }
    }
    if (!ev_append_claim(sm, E, C, T, mask != 0)) return;
#pragma unroll
    for (int dir = 0; dir < S; dir++) {
        if ((mask >> dir) & 1u) {
            size_t idx;
            if (ev_append_slot(sm, (uint32_t)(T + r.f1(dir)) % Wn, rank[dir], idx))
                E.bent[idx] = make_uint2(words[dir], (uint32_t)(Lv - r.f2(dir)));
            else
                atomicExch(&C->overflow, 1u);
        }
    }
    const uint32_t n = __popc(mask);
    st.launched += n;
    st.live_delta += n;
    if (TRACE && n) {
        const int old = atomicAdd(E.out_count + v, (int)n);
        if (old == 0) st.act_delta++;
    }
}

// One lane: v improved to label Lv in cycle T; removes from the front of every queue into
// v the flows of quality <= Lv (Steps 7-9: they can no longer raise Label(v)).  Entries are
// read while they are in flight (arrival time > T); an entry that looks arrived is the slot
// a concurrent push is filling, and the scan stops there (the new flow is never removed:
// it left with quality above Lv).  With phantoms the pass is stamped on the edge before its
// head moves (release), so that a concurrent push reading the head (acquire) either sees
// the flows still queued or the stamp.
template <int D, typename W, bool TRACE>
__device__ __forceinline__ void ev_remove_into(const Params<W> &P, const EvParams &E, EvSmem &sm, uint32_t v, int Lv,
                                               const EdgeRecord<W, D> &r, int T, uint32_t stamp, EvLocal &st)
{
    constexpr int S = nslots(D);
    uint32_t ein[S], src[S], tail[S];
    uint4 es[S];
#pragma unroll
    for (int dir = 0; dir < S; dir++) {
        bool ok;
        if constexpr (D == GRAPH) {
            const uint32_t x = __ldg(P.nbw_in + (size_t)v * 8 + dir);
            src[dir] = x >> 3;
            ein[dir] = x;  // = src * 8 + the edge's out-slot at src
            ok = src[dir] != v;
        } else {
            ok = r.f1(dir) != 0;
            src[dir] = ok ? v + dir_offset<D>(P.stride, dir) : v;
            ein[dir] = src[dir] * (uint32_t)S + (dir ^ 1u);
        }
        if (!ok) ein[dir] = 0xffffffffu;
    }
#pragma unroll
    for (int dir = 0; dir < S; dir++) {
        if (ein[dir] != 0xffffffffu) {
            asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(tail[dir]) : "l"(&E.edge[ein[dir]].x) : "memory");
            es[dir] = __ldcg(E.edge + ein[dir]);
        } else {
            tail[dir] = 0u;
            es[dir] = make_uint4(0u, 0u, 0u, 0u);
        }
    }
    const uint32_t Wn = (uint32_t)E.W;
    uint2 front[S];  // the front entry of every queue into v that holds a flow
#pragma unroll
    for (int dir = 0; dir < S; dir++)
        front[dir] = ein[dir] != 0xffffffffu && tail[dir] != es[dir].z
                         ? __ldcg(E.ring + es[dir].y + es[dir].z % (es[dir].w & 0xffffu))
                         : make_uint2(0x7fffffffu, 0u);
#pragma unroll
    for (int dir = 0; dir < S; dir++) {
        if ((int)front[dir].y <= T || (int)front[dir].x > Lv) continue;  // nothing to remove (or a slot being filled)
        const uint32_t head = es[dir].z, f1 = es[dir].w & 0xffffu;
        atomicSub(&sm.hist[front[dir].y % Wn], 1);
        uint32_t k = 1;
        for (; head + k != tail[dir] && k < f1; k++) {
            const uint2 ent = __ldcg(E.ring + es[dir].y + (head + k) % f1);
            if ((int)ent.y <= T || (int)ent.x > Lv) break;
            atomicSub(&sm.hist[ent.y % Wn], 1);
        }
        if (TRACE && P.edge_stamp) {
            P.edge_stamp[ein[dir]] = stamp;
            asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(&E.edge[ein[dir]].z), "r"(head + k) : "memory");
        } else {
            E.edge[ein[dir]].z = head + k;
        }
        st.live_delta -= k;
        if (TRACE) {
            const int old = atomicSub(E.out_count + src[dir], (int)k);
            if (old == (int)k) st.act_delta--;
        }
    }
}

// Seed launch (Algorithm 3): water of quality M leaves every source (listed in cand) along
// each edge with M - f2 > Label(w), at time 0.
template <int D, typename W, bool TRACE>
__device__ __noinline__ void ev_seed(const Params<W> &P, const EvParams &E, const Group &g, uint32_t n_src, EvSmem &sm, Counters *C,
                        EvLocal &st)
{
    const uint32_t V = (uint32_t)P.V;
    ev_refill_stash(sm, E, C);
    for (uint32_t base = g.rank * TPB; base < n_src; base += g.size * TPB) {  // (uniform across the CTA)
        const uint32_t j = base + threadIdx.x;
        uint32_t v = 0, mask = 0;
        EdgeRecord<W, D> r{};
        if (j < n_src) {
            v = __ldcg(P.cand + j);
            r = load_record<W, D>(P.rec, v);
            int Lw[nslots(D)];
            neighbour_labels<D>(P, V, v, Lw);
            mask = launch_mask<W, D>(r, P.M, Lw);
        }
        ev_push_flows<D, W, TRACE>(P, E, sm, C, v, P.M, r, mask, 0, 0u, st);
    }
}

// Returns a chunk to the free stack (phase A only; allocations happen in other phases).
__device__ __forceinline__ void ev_free_chunk(const EvParams &E, uint32_t c)
{
    const int pos = atomicAdd(&E.ev->free_top, 1);
    if (pos >= 0 && pos < (int)E.nch) E.freestk[pos] = c;
}

// Phase A of the cycle at time T (the previous cycle ran at Tprev): closes the CTA's
// cursors of the rounds passed, frees the chunks of rounds passed without a cycle, and
// takes the arrivals of round T.
template <int D, typename W, bool TRACE>
__device__ __noinline__ void ev_phase_a(const Params<W> &P, const EvParams &E, const Group &g, EvSmem &sm, int T, int Tprev,
                           uint32_t cand_base, uint32_t cand_cap, Counters *C, EvLocal &st)
{
    const int lane = threadIdx.x & 31;
    const uint32_t lt = (1u << lane) - 1u;
    const uint32_t Wn = (uint32_t)E.W, span = (uint32_t)(T - Tprev);
    for (uint32_t i = threadIdx.x; i < Wn; i += TPB) {
        const uint32_t dist = (i + Wn - (uint32_t)(Tprev + 1) % Wn) % Wn;  // i = (Tprev + 1 + dist) mod W
        if (dist < span) sm.cursor[i] = pack_cursor(NO_CHUNK, 0);
    }
    if (threadIdx.x == 0) sm.n_cand = 0;
    // rounds passed without a cycle: every entry belongs to a removed flow; free their chunks
    const uint32_t gt = g.rank * TPB + threadIdx.x, gstep = g.size * TPB;
    for (int t = Tprev + 1; t < T; t++) {
        const uint32_t r = (uint32_t)t % (2u * Wn);
        const uint32_t cnt = __ldcg(E.bcount + r);
        for (uint32_t k = gt; k < cnt; k += gstep) ev_free_chunk(E, __ldcg(E.bdir + (size_t)r * E.nch + k));
    }
    __syncthreads();
    const uint32_t r = (uint32_t)T % (2u * Wn);
    const uint32_t cnt = __ldcg(E.bcount + r);
    uint32_t arrivals = 0;
    // this CTA's chunks of the round: k = rank, rank + G, ...
    for (uint32_t k0 = g.rank; k0 < cnt; k0 += EV_BATCH * g.size) {
        const uint32_t nb = min((uint32_t)EV_BATCH, (cnt - k0 + g.size - 1) / g.size);
        if (threadIdx.x < nb) {
            const uint32_t c = __ldcg(E.bdir + (size_t)r * E.nch + k0 + threadIdx.x * g.size);
            sm.chunk_id[threadIdx.x] = c;
            sm.chunk_n[threadIdx.x] = min((uint32_t)EV_CH, __ldcg(E.bfill + c));
        }
        __syncthreads();
        for (uint32_t i0 = 0; i0 < nb; i0 += 4) {
            uint2 ent[4];
            int32_t L[4];
#pragma unroll
            for (int i = 0; i < 4; i++) {
                const bool has = i0 + i < nb && threadIdx.x < sm.chunk_n[i0 + i];
                ent[i] = has ? __ldcg(E.bent + (size_t)sm.chunk_id[i0 + i] * EV_CH + threadIdx.x) : make_uint2(0u, 0u);
            }
#pragma unroll
            for (int i = 0; i < 4; i++) {
                const bool has = i0 + i < nb && threadIdx.x < sm.chunk_n[i0 + i];
                L[i] = has ? __ldcg(P.label + (ent[i].x >> 3)) : INT_MAX;
            }
#pragma unroll
            for (int i = 0; i < 4; i++) {
                const bool arr = (int32_t)ent[i].y > L[i];  // (no entry: 0 > INT_MAX is false)
                if (arr) {
                    uint32_t sdir;
                    const uint32_t src = flow_source<D>(P, ent[i].x, sdir);
                    atomicAdd(&E.edge[(size_t)src * nslots(D) + sdir].z, 1u);  // pop the front flow
                    const unsigned long long key =
                        ((unsigned long long)ent[i].y << 32) | (0xffffffffu - (src * 8u + sdir));
                    atomicMax(P.offer + (ent[i].x >> 3), key);
                    if (TRACE) {
                        const int old = atomicSub(E.out_count + src, 1);
                        if (old == 1) st.act_delta--;
                    }
                }
                const uint32_t ba = __ballot_sync(0xffffffffu, arr);
                if (ba) {
                    uint32_t cb = 0;
                    if (lane == 0) cb = atomicAdd(&sm.n_cand, __popc(ba));
                    cb = __shfl_sync(0xffffffffu, cb, 0);
                    if (arr) {
                        const uint32_t pos = cb + __popc(ba & lt);
                        if (pos < cand_cap) P.cand[cand_base + pos] = ent[i].x;
                        else atomicExch(&C->overflow, 1u);
                    }
                    arrivals += lane == 0 ? __popc(ba) : 0u;
                }
            }
        }
        if (threadIdx.x == 0) sm.free_base = (uint32_t)atomicAdd(&E.ev->free_top, (int)nb);  // the batch goes back
        __syncthreads();
        if (threadIdx.x < nb && sm.free_base + threadIdx.x < E.nch) E.freestk[sm.free_base + threadIdx.x] = sm.chunk_id[threadIdx.x];
        __syncthreads();
    }
    st.cands += arrivals;
    st.live_delta -= arrivals;
    if (arrivals) atomicSub(&sm.hist[(uint32_t)T % Wn], (int)arrivals);
}

// Phase B of the cycle at time T: winners commit, launch and remove (see the file comment).
template <int D, typename W, bool TRACE>
__device__ __noinline__ void ev_phase_b(const Params<W> &P, const EvParams &E, const Group &g, EvSmem &sm, int T, uint32_t stamp,
                           uint32_t cand_base, uint32_t cand_cta, Counters *C, EvLocal &st)
{
    const uint32_t V = (uint32_t)P.V;
    const uint32_t n_cand = min(sm.n_cand, cand_cta);
    ev_refill_stash(sm, E, C);
    for (uint32_t base = 0; base < n_cand; base += TPB) {  // (uniform across the CTA)
        const uint32_t j = base + threadIdx.x;
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
            const uint32_t bw = __ldcg(P.isB + (v >> 5));
            if (lo32(ov) == code) {  // the winning arrival at v
                won = true;
                Lv = (int)hi32(ov);
                if ((P.touched || P.first_t) && __ldcg(P.label + v) == 0) {  // the first improvement of v
                    if (P.touched) P.touched[atomicAdd(P.touched_n, 1u)] = v;
                    if (P.first_t) {
                        P.first_t[v] = T;
                        P.first_code[v] = code;
                    }
                }
                P.label[v] = Lv;
                st.improved++;
                if ((bw >> (v & 31)) & 1u)
                    atomicMax(&C->xkey, ((unsigned long long)(uint32_t)Lv << 32) | (0xffffffffu - v));
                mask = launch_mask<W, D>(r, Lv, Lw);
            }
        }
        if (P.log) {  // every improvement, in this pass's segment of the log
            const uint32_t bw = __ballot_sync(0xffffffffu, won);
            if (bw) {
                const int lane = threadIdx.x & 31;
                unsigned long long lb = 0;
                if (lane == 0) lb = atomicAdd(P.log_n, (unsigned long long)__popc(bw));
                lb = __shfl_sync(0xffffffffu, lb, 0);
                const unsigned long long i = lb + __popc(bw & ((1u << lane) - 1u));
                if (won && i < P.log_cap) P.log[i] = make_uint2(v, code);
            }
        }
        ev_push_flows<D, W, TRACE>(P, E, sm, C, v, Lv, r, mask, T, stamp, st);
        if (won) ev_remove_into<D, W, TRACE>(P, E, sm, v, Lv, r, T, stamp, st);
    }
}

// End of a phase (after a __syncthreads), cycle time T: adds this CTA's calendar changes to
// blive[], lists the chunks it opened in their rounds' directories and records how full its
// open chunks written in this phase are.
__device__ __forceinline__ void ev_flush_calendar(const EvParams &E, EvSmem &sm, int T)
{
    const uint32_t Wn = (uint32_t)E.W;
    for (uint32_t i = threadIdx.x; i < Wn; i += TPB) {
        const int h = sm.hist[i];
        if (h) atomicAdd(E.blive + i, h);
        sm.hist[i] = 0;
        if ((sm.dirty[i >> 5] >> (i & 31)) & 1u) {
            ev_list_new(sm, E, i, T);
            const unsigned long long cur = sm.cursor[i];
            const uint32_t id = hi32(cur);
            if (id < FIRST_SPECIAL) E.bfill[id] = min(lo32(cur), (uint32_t)EV_CH);
        }
    }
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < EV_WMAX / 32; i += TPB) sm.dirty[i] = 0u;
}

// Adds this CTA's statistics to the cycle counters and the running totals.
__device__ __forceinline__ void ev_flush_stats(const EvLocal &st, Counters *C, EvCtl *ev)
{
    __shared__ long long s_live;
    __shared__ int s_act;
    __shared__ unsigned long long s_li, s_ph;
    __shared__ unsigned int s_cd;
    if (threadIdx.x == 0) {
        s_live = 0;
        s_act = 0;
        s_li = 0;
        s_ph = 0;
        s_cd = 0;
    }
    __syncthreads();
    long long live = st.live_delta;
    int act = st.act_delta;
    uint32_t lau = st.launched, imp = st.improved, cd = st.cands, ph = st.phantoms;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        live += __shfl_xor_sync(0xffffffffu, live, o);
        act += __shfl_xor_sync(0xffffffffu, act, o);
        lau += __shfl_xor_sync(0xffffffffu, lau, o);
        imp += __shfl_xor_sync(0xffffffffu, imp, o);
        cd += __shfl_xor_sync(0xffffffffu, cd, o);
        ph += __shfl_xor_sync(0xffffffffu, ph, o);
    }
    if ((threadIdx.x & 31) == 0) {
        if (live) atomicAdd((unsigned long long *)&s_live, (unsigned long long)live);
        if (act) atomicAdd(&s_act, act);
        if (lau | imp) atomicAdd(&s_li, (unsigned long long)lau | ((unsigned long long)imp << 32));
        if (cd) atomicAdd(&s_cd, cd);
        if (ph) atomicAdd(&s_ph, (unsigned long long)ph);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        if (s_live) atomicAdd((unsigned long long *)&ev->live, (unsigned long long)s_live);
        if (s_act) atomicAdd((unsigned long long *)&ev->active, (unsigned long long)(long long)s_act);
        if (s_li) atomicAdd(&C->lau_imp, s_li);
        if (s_cd) atomicAdd(&C->out_cand, (unsigned long long)s_cd << 32);
        if (s_ph) atomicAdd(&C->phantoms, s_ph);
    }
}

// Reads the running totals after a barrier (thread 0, shared with the CTA).
__device__ __forceinline__ void ev_read_totals(const EvCtl *ev, long long &live, long long &active)
{
    __shared__ long long s_l, s_a;
    if (threadIdx.x == 0) {
        s_l = __ldcg(&ev->live);
        s_a = __ldcg(&ev->active);
    }
    __syncthreads();
    live = s_l;
    active = s_a;
    __syncthreads();
}

// The first time after T with a flow in flight arriving (every CTA computes the same from
// blive after a barrier); -1 if there is none.
__device__ __forceinline__ int ev_next_time(const EvParams &E, int T)
{
    __shared__ int s_next;
    if (threadIdx.x < 32) {
        const uint32_t Wn = (uint32_t)E.W;
        int found = -1;
        for (uint32_t d0 = 1; d0 < Wn && found < 0; d0 += 32) {
            const uint32_t d = d0 + threadIdx.x;
            const bool live = d < Wn && __ldcg(E.blive + ((uint32_t)T + d) % Wn) > 0;
            const uint32_t b = __ballot_sync(0xffffffffu, live);
            if (b) found = T + (int)(d0 + __ffs(b) - 1);
        }
        if (threadIdx.x == 0) s_next = found;
    }
    __syncthreads();
    const int t = s_next;
    __syncthreads();
    return t;
}

// Runs one whole solve by the calendar on the CTAs of group g.  Set-up as for run_solve
// (labels, offers, B bitmap, sources listed in cand, fresh counters), plus empty queues
// (heads = tails = 0, ring zero), a full free stack, zero blive and round counts, and
// (trace mode) zero out_count.  The group leader writes the result record.
template <int D, typename W, bool TRACE>
__device__ void run_event_solve(const Params<W> &P, const EvParams &E, const Group &g, EvSmem &sm,
                                unsigned long long &epoch)
{
    Control *ctl = P.ctl;
    EvCtl *ev = E.ev;
    const bool leader = g.leader();
    const int M = P.M;
    const unsigned long long t_start = globaltimer_ns();
    unsigned long long t_mark = t_start, t_a = 0, t_b = 0, t_bar = 0;

    long long cycle = 0, updates = 0, launched = 0, trace_len = 0, arrivals = 0, improved = 0, phantoms = 0,
              max_live = 0;
    int Time = 0, status = ST_OK;
    bool feasible = false;
    unsigned long long xkey = 0;

    if (P.test_absent && g.size > 1 && g.rank == g.size - 1) return;  // (test hook: see Params)
    for (uint32_t i = threadIdx.x; i < (uint32_t)EV_WMAX; i += TPB) {
        sm.cursor[i] = pack_cursor(NO_CHUNK, 0);
        sm.hist[i] = 0;
        sm.bcnt[i] = 0u;
        sm.nnew[i] = 0u;
    }
    for (uint32_t i = threadIdx.x; i < EV_WMAX / 32; i += TPB) sm.dirty[i] = 0u;
    if (threadIdx.x == 0) {
        sm.fail = 0;
        sm.n_cand = 0;
        sm.stash_n = 0;
    }
    __syncthreads();

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
        const uint32_t cand_cta = P.cand_cap / g.size;
        const uint32_t cand_base = g.rank * cand_cta;
        EvLocal st;
        ev_local_zero(st);
        const uint32_t n_src = min(hi32(read_shared_u64(&ctl->cnt[0].out_cand)), P.cand_cap);
        ev_seed<D, W, TRACE>(P, E, g, n_src, sm, &ctl->cnt[0], st);
        __syncthreads();
        ev_flush_calendar(E, sm, 0);
        ev_flush_stats(st, &ctl->cnt[0], ev);
        if (!group_sync(ctl, epoch, g, P.barrier_ns) || sm.fail) { status = ST_BARRIER; goto finish; }
        const PassCounts c0 = read_counters(&ctl->cnt[0]);
        long long live, active;
        ev_read_totals(ev, live, active);
        launched += (long long)c0.launched;
        if (c0.overflow) { status = ST_CAPACITY; goto finish; }
        if (leader) write_row(P, 0, 0, active, live);
        trace_len = 1;
        if (live == 0) goto finish;  // nothing can leave A: infeasible
        max_live = live;
        if (leader) t_mark = globaltimer_ns();

        for (long long pass = 1;; pass++) {
            Counters *Cc = &ctl->cnt[pass & 1];
            const int Tn = ev_next_time(E, Time);
            if (Tn < 0) { status = ST_CUDA; goto finish; }  // flows in flight but none listed: inconsistent
            if (Tn >= TIME_LIMIT) { status = ST_CAPACITY; goto finish; }
            const long long live_start = live;  // flows in flight at the start of this cycle
            EvLocal sa;
            ev_local_zero(sa);
            ev_phase_a<D, W, TRACE>(P, E, g, sm, Tn, Time, cand_base, cand_cta, Cc, sa);
            __syncthreads();
            ev_flush_calendar(E, sm, Tn);
            ev_flush_stats(sa, Cc, ev);
            if (leader) {
                const unsigned long long t = globaltimer_ns();
                t_a += t - t_mark;
                t_mark = t;
            }
            if (!group_sync(ctl, epoch, g, P.barrier_ns) || sm.fail) { status = ST_BARRIER; goto finish; }
            if (leader) {
                zero_counters(&ctl->cnt[(pass + 1) & 1]);  // read by everyone one pass ago
                for (int t = Time + 1; t <= Tn; t++) E.bcount[(uint32_t)t % (2u * (uint32_t)E.W)] = 0u;  // rounds done
                if (P.log && pass < P.pass_cap) {  // this pass's log segment starts here
                    P.pass_time[pass] = Tn;
                    P.pass_off[pass] = *(volatile unsigned long long *)P.log_n;
                }
                if (globaltimer_ns() - t_start > P.budget_ns) Cc->abort = 1u;
                const unsigned long long t = globaltimer_ns();
                t_bar += t - t_mark;
                t_mark = t;
            }
            EvLocal sb;
            ev_local_zero(sb);
            ev_phase_b<D, W, TRACE>(P, E, g, sm, Tn, (uint32_t)pass, cand_base, cand_cta, Cc, sb);
            __syncthreads();
            ev_flush_calendar(E, sm, Tn);
            ev_flush_stats(sb, Cc, ev);
            if (leader) {
                const unsigned long long t = globaltimer_ns();
                t_b += t - t_mark;
                t_mark = t;
            }
            if (!group_sync(ctl, epoch, g, P.barrier_ns) || sm.fail) { status = ST_BARRIER; goto finish; }
            const PassCounts c = read_counters(Cc);
            ev_read_totals(ev, live, active);
            if (leader) {
                const unsigned long long t = globaltimer_ns();
                t_bar += t - t_mark;
                t_mark = t;
            }
            if (c.overflow) { status = ST_CAPACITY; goto finish; }
            if (c.abort) {  // reported like the sweep form: rows 0 .. cycle - 1, counts of cycles 1 .. cycle
                status = ST_TIMEOUT;
                trace_len = cycle;
                goto finish;
            }
            launched += (long long)c.launched;
            arrivals += (long long)c.n_cand;
            improved += (long long)c.improved;
            phantoms += (long long)c.phantoms;
            updates += live_start;
            cycle++;
            Time = Tn;
            if (TRACE && leader) write_row(P, cycle, Time, active, live);
            trace_len = cycle + 1;
            if (c.xkey) {  // a vertex of B improved: F1 = Time (Algorithm 2)
                feasible = true;
                xkey = c.xkey;
                goto finish;
            }
            if (live == 0) goto finish;  // no flow left: infeasible
            max_live = max(max_live, live);
            if (P.max_cycles > 0 && cycle >= P.max_cycles) {  // rows 0 .. cycle - 1, as the sweep form
                status = ST_TIMEOUT;
                trace_len = cycle;
                goto finish;
            }
        }
    }

finish:
    if (leader && P.log && cycle + 1 <= P.pass_cap) P.pass_off[cycle + 1] = *(volatile unsigned long long *)P.log_n;
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
        o[R_PASSES] = cycle;
        o[R_MAXPOOL] = max_live;
        o[R_TRACELEN] = TRACE ? trace_len : 0;
        o[R_ARRIVALS] = arrivals;
        o[R_IMPROVED] = improved;
        o[R_PHANTOMS] = TRACE && P.edge_stamp ? phantoms : -1;
        o[R_ELAPSED_NS] = (long long)(globaltimer_ns() - t_start);
        ev->phase_ns[0] = 0;
        ev->phase_ns[1] = t_a;
        ev->phase_ns[2] = t_b;
        ev->phase_ns[3] = t_bar;
        if (P.result_dev)
            for (int i = 0; i < R_COUNT; i++) P.result_dev[i] = o[i];
    }
}

}  // namespace csp
