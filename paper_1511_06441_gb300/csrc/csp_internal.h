// Host-side definitions shared by the translation units of libcsp (not part of the ABI).
#pragma once

#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <string>

#include "csp.h"
#include "csp_device.cuh"

// Records the text of a failed CUDA call (csp_last_error) and maps it to a status.
csp_status cuda_fail(cudaError_t e, const char *what);
void set_error(const std::string &msg);
extern thread_local std::string g_last_error;

#define CSP_CUDA(call)                                      \
    do {                                                    \
        cudaError_t e_ = (call);                            \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
    } while (0)

inline int record_bytes(int d, int wbytes) { return wbytes * 2 * csp::nslots(d) <= 16 ? 16 : 32; }
inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// The packed view of a pool buffer (one 64-bit word per slot) over its qa and ta arrays, when
// ta starts right after qa's pool_cap + POOL_PAD entries (so the words of pool_cap + POOL_PAD / 2
// slots fit) and qa is 16-byte aligned for bulk copies; null otherwise (the kernel then keeps
// the three arrays).
inline unsigned long long *packed_pool(int32_t *qa, int32_t *ta, int64_t pool_cap)
{
    const bool adjacent = (char *)ta == (char *)qa + (size_t)(pool_cap + csp::POOL_PAD) * 4;
    return adjacent && ((uintptr_t)qa % 16) == 0 ? reinterpret_cast<unsigned long long *>(qa) : nullptr;
}

struct csp_event_ws;

struct csp_lattice {
    int d = 0;                          // lattice dimension 1..4, or csp::GRAPH
    int wbytes = 1;
    int64_t ext[4] = {1, 1, 1, 1};
    int stride[4] = {0, 0, 0, 0};
    int64_t V = 0;
    int device = 0;
    void *f1 = nullptr, *f2 = nullptr;  // device [d][V] (lattice only)
    void *rec = nullptr;                // device per-vertex edge records
    uint32_t *nbw = nullptr;            // graph only: device [8 V] head << 3 | in-slot at the head
    uint32_t *nbw_in = nullptr;         // graph only: device [8 V] tail << 3 | out-slot at the tail (= nbw if undirected)
    int rec_bytes = 16;
    unsigned long long flow_bound = 0;  // sum of f1 over directed edges: max flows alive
    unsigned long long n_arcs = 0;      // directed edges (f1 > 0)
    unsigned int max_f1 = 0;            // largest travel time
    // workspace of csp_solve / csp_solve_async
    void *ws = nullptr;
    size_t ws_bytes = 0;
    int64_t pool_cap = 0;
    int32_t *label = nullptr;
    unsigned long long *offer = nullptr;
    uint32_t *isB = nullptr, *src_stamp = nullptr, *edge_stamp = nullptr;
    uint32_t *cand = nullptr;
    int64_t cand_cap = 0;
    uint32_t *ed[2] = {nullptr, nullptr};
    int32_t *qa[2] = {nullptr, nullptr}, *ta[2] = {nullptr, nullptr};
    uint32_t *fill[2] = {nullptr, nullptr};  // slots in use per pool chunk
    csp::Control *ctl = nullptr;
    long long *trace = nullptr;
    int64_t trace_cap = 0;
    int64_t *sets = nullptr;  // device copies of A and B
    int64_t sets_cap = 0;
    csp_event_ws *evw = nullptr;  // the event-driven form's edge queues and calendar (csp_event.cu)
};

int num_sms(int device);

// Coordinate axes of a handle: d for a lattice, 0 for a general graph (no hyperplanes).
inline int num_axes(const csp_lattice *L) { return L->d == csp::GRAPH ? 0 : L->d; }

// Device buffers that record improvements for path reconstruction (see Params).
struct ReconLog {
    int32_t *first_t = nullptr;
    uint32_t *first_code = nullptr;
    uint2 *log = nullptr;
    unsigned long long log_cap = 0;
    unsigned long long *log_n = nullptr;
    int32_t *pass_time = nullptr;
    unsigned long long *pass_off = nullptr;
    long long pass_cap = 0;
};

// Largest group of CTAs one solve may use on a device: the candidate list of a workspace
// is sized for it (one region per CTA).
inline int max_group_ctas(int device) { return std::min(4 * num_sms(device), csp::MAX_GROUP); }

// Pool slots a pass may leave unused: each CTA of a group holds one partly filled chunk
// and one chunk allocated ahead.
inline int64_t chunk_slack(int64_t group_ctas) { return 2 * group_ctas * (int64_t)csp::TILE; }

// The event-driven form of the cycle loop (csp_event.cu).
csp_status event_prepare(csp_lattice *L, cudaStream_t s);  // edge records for the current weights (synchronous)
bool event_supported(const csp_lattice *L);                // prepared, max f1 < 512, rings fit 32-bit offsets
csp_status event_reserve(csp_lattice *L, int64_t entry_cap);
int64_t event_entry_cap(const csp_lattice *L);
csp_status event_max_ctas(const csp_lattice *L, bool trace, int *out);
csp_status event_launch(csp_lattice *L, const void *params, bool trace, int ctas, const csp_options *opt,
                        cudaStream_t s);
csp_status event_phase_times(const csp_lattice *L, unsigned long long *ns4);
void event_invalidate(csp_lattice *L);  // the weights changed
void event_release(csp_lattice *L);
