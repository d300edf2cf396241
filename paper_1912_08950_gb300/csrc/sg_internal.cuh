// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "slimgraph.h"

namespace sg {

// ---------------------------------------------------------------- constants
constexpr uint32_t kTagEdge = 0x45444745u;  // Philox counter word 3 for edges
constexpr uint32_t kTagTri = 0x54524931u;   // Philox counter word 3 for triangles
constexpr unsigned kFull = 0xFFFFFFFFu;

// device error word values (set by kernels, read after a stream sync)
enum DevErr : int { kDevOk = 0, kDevLookbackTimeout = 1, kDevBadGraph = 2, kDevTableFull = 3 };

// bounded spin: polls of a not-yet-published status word before giving up
constexpr uint32_t kSpinLimit = 1u << 22;

// compaction geometry: a chunk of kWarpSpan arcs is one warp's CI slabs of 32
constexpr int CI = 8;
constexpr int kWarpSpan = 32 * CI;  // arcs per chunk
static_assert((CI & (CI - 1)) == 0 && CI <= 32, "CI is a power of two of at most 32 slabs");

// ------------------------------------------------------------- host objects
struct ProfRec {
    const char *name;
    cudaEvent_t beg, end;
};

struct Ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int num_sms = 0;
    int *d_err = nullptr;                  // device error word
    unsigned long long *d_ctr = nullptr;   // device counters [kCtrCount]
    int64_t *h_pinned = nullptr;           // pinned host scratch (small reads)
    uint64_t launches = 0;
    uint64_t eo_rounds = 0;
    uint64_t eo_listed = 0;                // triangles written to edge-once lists
    uint64_t eo_passes = 0;                // edge-once enumeration passes
    uint64_t eo_list_passes = 0;           // ... that listed triangles
    int64_t eo_list_cap = 0;               // 0 auto, -1 off, > 0 records
    bool profiling = false;
    uint32_t scan_hold = 0;                // test hook (sg_ctx_set_scan_hold): 0 off
    // grow-only device workspaces kept across calls (edge-once list and active
    // lists), so that repeated calls do not churn the stream-ordered pool
    void *ws[3] = {nullptr, nullptr, nullptr};
    size_t ws_bytes[3] = {0, 0, 0};
    std::vector<ProfRec> prof;             // events of launches since reset
    std::vector<cudaEvent_t> event_pool;   // recycled events
};

enum CtrIdx { kCtrProbes = 0, kCtrTriangles = 1, kCtrLive = 2, kCtrHeavy = 3, kCtrMaxDeg = 4, kCtrAux = 5,
              kCtrInArcs = 7, kCtrWork = 8, kCtrWorkFwd = 9, kCtrCount = 10 };  // kCtrAux holds two words

struct Graph {
    Ctx *ctx = nullptr;
    int device = 0;
    int64_t n = 0, nnz = 0;
    int64_t *off = nullptr;
    uint32_t *col = nullptr;
    float *w = nullptr;
    bool owned = true;
};

// ------------------------------------------------------------ error plumbing
void set_error(const std::string &msg);
sg_status fail(sg_status st, const std::string &msg);
sg_status cuda_fail(cudaError_t e, const char *what);

#define SG_CUDA(call)                                                   \
    do {                                                                \
        cudaError_t _e = (call);                                        \
        if (_e != cudaSuccess) return ::sg::cuda_fail(_e, #call);       \
    } while (0)

// whether a context is still alive (objects may outlive their context)
bool ctx_alive(const Ctx *c);

// stream-ordered device allocation on the context stream
sg_status dalloc(Ctx *c, void **p, size_t bytes);
// workspace `slot` of at least `bytes` bytes (contents undefined; owned by the context)
sg_status ws_get(Ctx *c, int slot, size_t bytes, void **p);
void dfree(Ctx *c, void *p);

// launch bookkeeping: brackets a launch with events when profiling
struct LaunchScope {
    Ctx *c;
    const char *name;
    cudaEvent_t b = nullptr, e = nullptr;
    LaunchScope(Ctx *c_, const char *n_);
    ~LaunchScope();
};
#define SG_CAT2_(a, b) a##b
#define SG_CAT_(a, b) SG_CAT2_(a, b)
#define SG_LAUNCH(ctx, name) ::sg::LaunchScope SG_CAT_(sg_scope_, __LINE__)((ctx), (name))

// read the device error word and reset it; map it to a status
sg_status check_device_error(Ctx *c);

// -------------------------------------------------------------- device code
#ifdef __CUDACC__

// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of a
// multiply-xor Feistel step on four 32-bit words; the two key words advance by
// Weyl increments between rounds.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t lo0 = 0xD2511F53u * c.x;
        const uint32_t hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}

__device__ __forceinline__ uint32_t lanemask_lt() {
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

__device__ __forceinline__ unsigned long long ld_volatile_u64(const unsigned long long *p) {
    unsigned long long v;
    asm volatile("ld.volatile.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_volatile_u64(unsigned long long *p, unsigned long long v) {
    asm volatile("st.volatile.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}

// first index in sorted a[lo, hi) with a[i] >= key
__device__ __forceinline__ int64_t lower_bound_u32(const uint32_t *a, int64_t lo, int64_t hi, uint32_t key) {
    while (lo < hi) {
        const int64_t mid = lo + ((hi - lo) >> 1);
        if (__ldg(a + mid) < key) lo = mid + 1; else hi = mid;
    }
    return lo;
}

#endif  // __CUDACC__

// batched compression: per-graph parameters in the disjoint union
struct BatchParam {
    int64_t vbase;              // first vertex of the graph in the union
    unsigned long long tp;      // floor(p 2^32): uniform and triangle kernels
    unsigned long long ty;      // floor(Y 2^32): spectral kernels
    uint32_t k0, k1;            // Philox key (seed low, high word)
    float yf;                   // Y rounded to float (spectral weights)
    int kernel;                 // sg_kernel
    int reweight;               // spectral: emit 1/p_uv weights
    int64_t n;                  // vertices of the graph
};

// ---------------------------------------------------------- internal entry
// compaction / edge kernels (sg_compact.cu)
struct RowMaps {
    uint32_t *chunk_row = nullptr;  // row containing arc c * kWarpSpan
    int64_t num_chunks = 0;
};
// scratch of one arc compaction
struct CompactScratch {
    uint32_t *keep = nullptr;            // keep bit of every arc: CI words per chunk
    int64_t *cexcl = nullptr;            // kept arcs per chunk, then their exclusive prefix; [num_chunks] = total
    unsigned long long *scan = nullptr;  // the chunk scan's tile status words and ticket
};
int64_t compact_scan_words(int64_t num_chunks);  // entries of CompactScratch::scan
sg_status alloc_compact_scratch(Ctx *c, int64_t num_chunks, bool with_keep, CompactScratch *s);
void free_compact_scratch(Ctx *c, CompactScratch *s);
sg_status build_row_maps(Ctx *c, const Graph *g, RowMaps *rm);
sg_status fill_row_maps(Ctx *c, const Graph *g, const RowMaps &rm);  // into allocated maps
void free_row_maps(Ctx *c, RowMaps *rm);

sg_status compress_edges(Ctx *c, const Graph *g, sg_kernel k, double p, uint64_t seed, int want_weights,
                         Graph **out);

// the degree-ordered orientation E+ (sg_compact.cu)
struct Oriented {
    int64_t n = 0, m = 0;
    int64_t *off = nullptr;      // off+[n+1]
    uint32_t *col = nullptr;     // col+[m]
    float *w = nullptr;          // w+[m] (weighted TR only)
    uint32_t *fwd_bits = nullptr;  // bit per symmetric arc: 1 iff x precedes y
    int64_t *fwd_excl = nullptr;   // forward arcs before every chunk; [num_chunks] = m
    // the reverse arcs in symmetric order: the one at symmetric position p is
    // E+ arc u->x (u = col[p] before its row x), stored as (u, arc index) at
    // rank p - (forward arcs before p); x's in-arcs are thus contiguous at
    // off(x) - off+(x), sorted by u (reverse_list)
    uint2 *inl = nullptr;
};
sg_status orient(Ctx *c, const Graph *g, const RowMaps &rm, bool weights, Oriented *o);
void free_oriented(Ctx *c, Oriented *o);
// H = G minus the edges whose oriented arc has del[] != 0
sg_status resolve_mask(Ctx *c, const Graph *g, const RowMaps &rm, const Oriented &o, const uint8_t *del,
                       Graph **out);

// batched variants over a disjoint union (sg_compact.cu)
struct BatchDev {
    const BatchParam *params;   // [count]
    const uint32_t *vgid;       // graph of every union vertex
};
sg_status batch_orient(Ctx *c, const Graph *u, const RowMaps &rm, const BatchDev &b, bool weights, Oriented *o,
                       unsigned long long *scan, int grid_per_sm);
sg_status batch_final(Ctx *c, const Graph *u, const RowMaps &rm, const Oriented &o, const BatchDev &b,
                      const uint8_t *del, uint32_t *delbits, int64_t *off_out, uint32_t *col_out, float *w_in,
                      float *w_out, const CompactScratch &cs, int grid_per_sm);
// the reverse list of o (see Oriented::inl) into inl; in a batch only the
// graphs with a triangle kernel are listed
sg_status reverse_list(Ctx *c, const Graph *g, const RowMaps &rm, const Oriented &o, uint2 *inl,
                       BatchDev batch = BatchDev{nullptr, nullptr});

// low_degree vertex kernel (sg_compact.cu)
sg_status low_degree(Ctx *c, const Graph *g, uint32_t *new_to_old, Graph **out);

// triangles (sg_triangles.cu)
sg_status tr_mark(Ctx *c, const Graph *g, const Oriented &o, sg_kernel k, double p, uint64_t seed,
                  uint8_t *del);
sg_status tr_count(Ctx *c, const Graph *g, const Oriented &o, int64_t *count, int64_t *probes, int64_t *maxdeg,
                   int64_t *in_arcs, int64_t *fwd_probes);
// batched union TR, with no host synchronisation (capturable in a CUDA graph)
struct BatchTri {
    uint32_t *heavy = nullptr;
    unsigned long long *buckets = nullptr;  // counts, fills, total
    uint32_t *din = nullptr;                // in-arcs streamed from the head's side
    uint2 *inl = nullptr;
    int log_slots = 3;
    size_t smem = 0;
    int max_deg = 1;      // largest out-degree (sizes the heavy vertex arrays)
    int light_max = 64;
    int grid_per_sm = 0;  // 0: occupancy limit
};
sg_status batch_tr_prepare(Ctx *c, const Graph *u, const Oriented &o, BatchTri *bt);
sg_status batch_tr_mark(Ctx *c, const Graph *u, const Oriented &o, const BatchDev &b, const BatchTri &bt,
                        uint8_t *del);
void batch_tr_free(Ctx *c, BatchTri *bt);

sg_status tr_vertex_counts(Ctx *c, const Graph *g, const Oriented &o, unsigned long long *vcnt);

// analytics (sg_analytics.cu)
sg_status pagerank(Ctx *c, const Graph *g, float damping, int iters, float *x_out, double *resid);
sg_status kl_divergence(Ctx *c, int64_t n, const float *P, const float *Q, double *kl);
sg_status cc_count(Ctx *c, const Graph *g, int64_t *count, uint32_t *labels);
sg_status validate_graph(Ctx *c, const Graph *g);
sg_status bfs_levels(Ctx *c, const Graph *g, int64_t root, int *level);
sg_status critical_edges(Ctx *c, const Graph *g, int64_t root, int64_t *count);
template <typename T>
sg_status reordered_neighbours(Ctx *c, const Graph *g, const T *x, const T *y, int64_t *count);
sg_status max_degree_vertex(Ctx *c, const Graph *g, int64_t *v);

uint64_t prob_threshold(double p);

}  // namespace sg
