// Triangle enumeration over the degree-ordered orientation E+ and the
// Triangle p-x-Reduction kernels of Slim Graph (Sec. 4.3; Listing 1
// p-1-reduction and p-1-reduction-EO; x = 2; the min-count "CT" choice of
// Sec. 7).
//
// Enumeration.  Every triangle {u, v, w} with u < v < w in the degree order
// (d, id) is found exactly once, at the oriented arc u->v, as w in
// N+(u) ∩ N+(v) (the forward algorithm behind the O(m^{3/2}) bound the paper
// quotes).  The intersection streams the shorter of the two lists through a
// shared-memory hash table of the longer one: every vertex x stages N+(x) in
// a table once and streams (a) N+(v) for its out-arcs x->v with
// d+(v) <= d+(x) and (b) N+(u) for its in-arcs u->x with d+(u) < d+(x); the
// in-arcs of kind (b) are gathered per vertex by one scatter pass.  Each arc
// is handled once, at the end with the longer list, so the probes number
// sum over arcs of min(d+(u), d+(v)) -- under half of the plain forward
// algorithm's sum of d+(v) on power-law graphs.  Vertices with a short N+(x)
// and few in-arcs get one warp each; the others get a whole CTA whose warps
// split the arcs; those with an N+(x) longer than one CTA's table (when there
// are at least as many as SMs) go first, to a launch of 32-warp CTAs, one per
// SM, whose larger table holds their N+(x) whole.
//
// Decisions.  A hit (a triangle) is pushed to a per-warp queue; whenever 32
// hits are queued the warp decides all of them at once with full lanes:
// Philox4x32-10 on the sorted original ids (a, b, c) selects the triangle
// (r0 < floor(p 2^32)) and picks the edge to delete (r1, the heaviest edge, or
// the edge in the fewest triangles of G, counted by an earlier EdgeCount pass);
// the p-2 kernel deletes the two edges r1 does not pick.  Union kernels store
// del[arc] = 1 (a plain, idempotent byte store).  The
// Edge-Once kernel instead reserves each edge of every live selected triangle
// with a 64-bit atomicMin of (r2 << 32 | third vertex); an edge pass then
// accepts every triangle that holds all three of its reservations.  Accepted
// triangles are edge-disjoint, mark their edges considered, delete their
// chosen edge, and the rounds repeat until no selected triangle is live.
// This reproduces exactly the sequential scan of the selected triangles in
// increasing (r2, a, b, c) order (for two triangles sharing an edge, the
// lexicographic order of (a, b, c) equals the order of their third vertices).
#include <climits>
#include <cstring>

#include "sg_internal.cuh"

namespace sg {

constexpr uint32_t kEmpty = 0xFFFFFFFFu;
constexpr int kLightMax = 64;     // largest out-degree processed by one warp
constexpr int kLightItems = 256;  // ... with at most this many lists to stream
constexpr int kLightSlots = 256;  // hash slots per warp (>= 4 * kLightMax)
constexpr int kTW = 8;            // warps per CTA
constexpr int kHeavyCap = 1024;  // largest phase-1 table (entries; 26 KB of shared memory)
constexpr int kHubTW = 32;        // warps per CTA of the hub launch (one CTA per SM)
constexpr int kHubCap = 4096;     // largest hub table (entries; 104 KB of shared memory)
constexpr int kQ = 128;           // per-warp hit ring (<= 31 left over + 2 slabs of hits fit)
constexpr int kEoBuckets = 6;     // edge-once list buckets (rounds 0..5 of the prefix schedule)
// context workspaces of the edge-once rounds: the list and the two active lists
constexpr int kWsList = 0, kWsActive0 = 1, kWsActive1 = 2;

// Count: totals only.  EdgeCount / VertexCount: add every triangle to the
// counters of its three edges / vertices.  Union*: the union-semantics TR kernels.  EoReserve: one
// edge-once bidding pass.  EoEmit: lists the live selected triangles for the
// edge-once list rounds.  BatchUnion: union kernels over a batch of graphs.
enum class Mode { Count, EdgeCount, VertexCount, UnionRandom, UnionMaxw, UnionP2, UnionMinCount, EoReserve, EoEmit,
                  BatchUnion };
// the edge-once passes skip arcs that are already considered
template <Mode M>
constexpr bool kEdgeOnce = M == Mode::EoReserve || M == Mode::EoEmit;

// Edge-once "considered" flags: one bit per oriented arc (m/8 bytes, so the
// flags stay in L2 while the triangle lists stream past them).
__device__ __forceinline__ bool considered_bit(const uint32_t *c, int64_t e) {
    return (__ldg(c + (e >> 5)) >> (e & 31)) & 1u;
}
__device__ __forceinline__ void set_considered(uint32_t *c, int64_t e) { atomicOr(c + (e >> 5), 1u << (e & 31)); }

struct TriArgs {
    const int64_t *offp;
    const uint32_t *colp;
    const int64_t *offs;          // symmetric offsets: in-arcs of x live at inl[offs(x) - offp(x) ...]
    const uint32_t *din;          // in-arcs u->x with d+(u) < d+(x), per x
    const uint2 *inl;             // (u, arc u->x) of those in-arcs
    const float *wp;
    int64_t n;
    uint32_t k0, k1;
    unsigned long long tp;
    uint8_t *del;
    const uint32_t *considered;  // edge-once flag bits (see considered_bit)
    unsigned long long *resv;
    uint32_t *tcnt;               // triangles of G through each arc of E+ (EdgeCount adds, min-count reads)
    unsigned long long *vcnt;     // triangles through each vertex (VertexCount adds)
    unsigned long long eo_theta;  // edge-once: only triangles with r2 < eo_theta bid this round
    unsigned long long *ctr;
    const uint32_t *heavy;
    int64_t n_heavy;
    int heavy_log_slots;
    int heavy_cap;               // entries of the phase-1 table; larger N+(u) go in chunks
    int light_max;               // out-degrees up to this go to the warp-per-vertex phase
    int light_items;             // ... when they also have at most this many arcs to stream
    int *err;                    // device error word (a cuckoo stash overflow)
    unsigned long long *work;    // [0] next heavy vertex, [1] next light vertex block
    const unsigned long long *n_heavy_dev;  // if set, the heavy count is read on the device
    // batched union: per-graph parameters and the graph of every vertex
    const BatchParam *bparams;
    const uint32_t *vgid;
    // edge-once: list of the live selected triangles (EoEmit), split into
    // buckets by the round in which each first bids
    uint4 *list;
    unsigned long long *list_ctr;  // [kEoBuckets] slots handed out per bucket
    unsigned long long *list_dem;  // [kEoBuckets] triangles that belong in each bucket, listed or not
    unsigned long long list_base[kEoBuckets], list_cap[kEoBuckets];
    int eo_round;                  // this enumeration's round: earlier buckets fold into it
    int eo_hi;                     // buckets from this one on are not listed (counted only)
    int *list_overflow;            // bit b: bucket b ran out of room
};

// One live selected triangle of an active list: sorted original ids
// x0 < x1 < x2, its draws r1 (edge choice) and r2 (edge-once order), and the
// oriented arcs joining (x0,x1), (x0,x2), (x1,x2).  x0 == kSentinel marks an
// unused slot.  The enumeration writes the smaller record (a, e_ab, e_ac,
// e_bc) instead -- a < b < c in the degree order, so b and c are the heads of
// e_ab and e_ac -- and a triangle is expanded when it first bids.
struct __align__(16) TriRec {
    uint32_t x0, x1, x2, r1;
    uint32_t r2, e01, e02, e12;
};
constexpr uint32_t kSentinel = 0xFFFFFFFFu;

// Bucket b of the list holds the triangles whose r2 lies in
// [2^(26+b), 2^(27+b)) (bucket 0: r2 < 2^27), i.e. those that first bid in
// edge-once round b of the doubling prefix schedule.
__device__ __forceinline__ int eo_bucket(uint32_t r2) { return r2 < (1u << 27) ? 0 : (31 - __clz((int)r2)) - 26; }
// list slots a warp claims at a time, in proportion to the bucket's share
__host__ __device__ constexpr int eo_chunk(int b) { return b <= 1 ? 64 : (32 << b); }

// Per-warp list writer: per bucket it claims chunks of slots, fills them in
// order and seals the unused tail of a chunk with sentinels.  The cursors
// live in registers spread over the lanes: lane b holds the next free slot of
// bucket b, lane 8 + b the end of its chunk and lane 16 + b how many
// triangles belong in bucket b.  Buckets from hi on are counted but not
// written: those the caller left out, and any that ran out of room (the
// lower buckets stay complete, so the caller can still use them).
struct Emitter {
    unsigned long long cur = 0;  // this lane's cursor or count (see above)
    int hi = 0;                  // warp-uniform
};

__device__ __forceinline__ void emit_seal(const TriArgs &a, unsigned long long cur, unsigned long long end) {
    const int lane = threadIdx.x & 31;
    for (unsigned long long i = cur + lane; i < end; i += 32) a.list[i].x = kSentinel;
}

__device__ __forceinline__ void emit_push(const TriArgs &a, Emitter &em, bool want, const uint4 &rec, uint32_t r2) {
    const int lane = threadIdx.x & 31;
    const int mb = want ? max(eo_bucket(r2), min(a.eo_round, kEoBuckets - 1)) : -1;
    if (!__any_sync(kFull, want)) return;
    // lanes of my bucket, and (in lanes b and 16 + b) the count of bucket b
    unsigned mine = 0, cnt_b = 0;
#pragma unroll
    for (int b = 0; b < kEoBuckets; ++b) {
        const unsigned bm = __ballot_sync(kFull, mb == b);
        if (mb == b) mine = bm;
        if ((lane & 15) == b) cnt_b = (unsigned)__popc(bm);
    }
    if (lane >= 16) em.cur += cnt_b;  // zero outside lanes 16 .. 16 + kEoBuckets - 1
    // a bucket whose chunk is too short for this group claims a new chunk (rare)
    const unsigned long long end_b = __shfl_down_sync(kFull, em.cur, 8);  // lane b: end of bucket b
    unsigned need = __ballot_sync(kFull, lane < em.hi && end_b - em.cur < cnt_b);
    while (need) {
        const int b = __ffs(need) - 1;
        need &= need - 1;
        const unsigned long long cur = __shfl_sync(kFull, em.cur, b);
        const unsigned long long end = __shfl_sync(kFull, em.cur, 8 + b);
        emit_seal(a, cur, end);
        const unsigned long long chunk = (unsigned long long)eo_chunk(b);
        unsigned long long base = 0;
        if (lane == 0) base = atomicAdd(a.list_ctr + b, chunk);
        base = __shfl_sync(kFull, base, 0);
        if (base + chunk > a.list_cap[b]) {
            // out of room: bucket b and the ones above it are no longer written
            if (lane == 0) atomicOr(a.list_overflow, 1 << b);
            em.hi = b;
            break;
        }
        if (lane == b) em.cur = a.list_base[b] + base;
        if (lane == 8 + b) em.cur = a.list_base[b] + base + chunk;
    }
    const unsigned long long cur = __shfl_sync(kFull, em.cur, mb < 0 ? 0 : mb);
    if (want && mb < em.hi) a.list[cur + __popc(mine & lanemask_lt())] = rec;
    if (lane < em.hi) em.cur += cnt_b;
}

// Per-warp ring of found triangles, waiting to be decided 32 at a time.  The
// table vertex u is the same for every entry (the ring is flushed before the
// warp moves to another table) and w is the head of the arc iuw, so an entry
// keeps v and the three arcs.  Oriented arcs are addressed with 32-bit
// indices (E+ holds fewer than 2^32 arcs).
struct HitQueue {
    uint32_t v[kQ], iuv[kQ], iuw[kQ], ivw[kQ];
};
struct QState {
    int head = 0, n = 0;
};

__device__ __forceinline__ uint32_t slot_of(uint32_t key, int log_slots) {
    return (key * 0x9E3779B1u) >> (32 - log_slots);
}

__device__ __forceinline__ int ceil_log2(int x) { return x <= 1 ? 0 : 32 - __clz(x - 1); }
static int ceil_log2_host(int x) {
    int l = 0;
    while ((1 << l) < x) ++l;
    return l;
}

template <typename T>
__device__ __forceinline__ void swap2(T &a, T &b) {
    const T t = a;
    a = b;
    b = t;
}

// The edge in the fewest triangles of G under (count, lo, hi).  The arcs are
// passed in the order (x0,x1), (x0,x2), (x1,x2) of the sorted endpoints, which
// is also their (lo, hi) order, so a tie keeps the earlier arc.
template <typename I>
__device__ __forceinline__ I mincount_arc(const uint32_t *tcnt, I e01, I e02, I e12) {
    const uint32_t c01 = __ldg(tcnt + e01), c02 = __ldg(tcnt + e02), c12 = __ldg(tcnt + e12);
    I best = e01;
    uint32_t bc = c01;
    if (c02 < bc) { best = e02; bc = c02; }
    if (c12 < bc) best = e12;
    return best;
}

// One triangle (u, v, w) with its three oriented arcs: selection and action.
// Warp-collective (the edge-once list writer uses ballots); lanes without a
// triangle pass valid = false.
template <Mode M>
__device__ __forceinline__ void decide(const TriArgs &a, bool valid, uint32_t u, uint32_t v, uint32_t w,
                                       uint32_t iuv, uint32_t iuw, uint32_t ivw, unsigned &live, Emitter &em,
                                       uint32_t head_uv = 0) {
    if constexpr (M == Mode::Count || M == Mode::EdgeCount || M == Mode::VertexCount) {
        return;
    } else {
        bool emit = false;
        uint4 rec = make_uint4(0u, 0u, 0u, 0u);
        uint32_t rec_r2 = 0;
        if constexpr (M == Mode::BatchUnion) {
            if (valid) {
                // the triangle's graph: its own seed, p and kernel, local ids as keys
                const BatchParam &P = a.bparams[__ldg(a.vgid + u)];
                const uint32_t base = (uint32_t)P.vbase;
                uint32_t x0 = u - base, x1 = v - base, x2 = w - base;
                uint32_t e01 = iuv, e02 = iuw, e12 = ivw;
                if (x0 > x1) { swap2(x0, x1); swap2(e02, e12); }
                if (x1 > x2) { swap2(x1, x2); swap2(e01, e02); }
                if (x0 > x1) { swap2(x0, x1); swap2(e02, e12); }
                const uint4 r = philox4x32_10(make_uint4(x0, x1, x2, kTagTri), P.k0, P.k1);
                if ((unsigned long long)r.x < P.tp) {
                    uint32_t best;
                    if (P.kernel == (int)SG_TR_MAXW) {
                        const float w01 = __ldg(a.wp + e01), w02 = __ldg(a.wp + e02), w12 = __ldg(a.wp + e12);
                        best = e01;
                        float bw = w01;
                        uint32_t bl = x0, bh = x1;
                        if (w02 > bw || (w02 == bw && (x0 > bl || (x0 == bl && x2 > bh)))) { best = e02; bw = w02; bl = x0; bh = x2; }
                        if (w12 > bw || (w12 == bw && (x1 > bl || (x1 == bl && x2 > bh)))) { best = e12; }
                    } else {
                        const int k = (int)(((unsigned long long)r.y * 3ull) >> 32);
                        best = k == 0 ? e01 : (k == 1 ? e02 : e12);
                        if (P.kernel == (int)SG_TR_P2) {  // the drawn edge is the one kept
                            if (k != 0) a.del[e01] = 1;
                            if (k != 1) a.del[e02] = 1;
                            if (k != 2) a.del[e12] = 1;
                            return;
                        }
                    }
                    a.del[best] = 1;
                }
            }
            return;
        }
        if (valid) {
            // sort the vertices, keeping e_ij = the arc joining x_i and x_j
            uint32_t x0 = u, x1 = v, x2 = w;
            uint32_t e01 = iuv, e02 = iuw, e12 = ivw;
            if (x0 > x1) { swap2(x0, x1); swap2(e02, e12); }
            if (x1 > x2) { swap2(x1, x2); swap2(e01, e02); }
            if (x0 > x1) { swap2(x0, x1); swap2(e02, e12); }
            const uint4 r = philox4x32_10(make_uint4(x0, x1, x2, kTagTri), a.k0, a.k1);
            if ((unsigned long long)r.x < a.tp) {  // the triangle is selected
                if constexpr (M == Mode::UnionRandom) {
                    const int k = (int)(((unsigned long long)r.y * 3ull) >> 32);
                    a.del[k == 0 ? e01 : (k == 1 ? e02 : e12)] = 1;
                } else if constexpr (M == Mode::UnionP2) {
                    // x = 2: the drawn edge stays, the other two go
                    const int k = (int)(((unsigned long long)r.y * 3ull) >> 32);
                    if (k != 0) a.del[e01] = 1;
                    if (k != 1) a.del[e02] = 1;
                    if (k != 2) a.del[e12] = 1;
                } else if constexpr (M == Mode::UnionMinCount) {
                    a.del[mincount_arc(a.tcnt, e01, e02, e12)] = 1;
                } else if constexpr (M == Mode::UnionMaxw) {
                    // heaviest edge under (weight, lo, hi)
                    const float w01 = __ldg(a.wp + e01), w02 = __ldg(a.wp + e02), w12 = __ldg(a.wp + e12);
                    uint32_t best = e01;
                    float bw = w01;
                    uint32_t bl = x0, bh = x1;
                    if (w02 > bw || (w02 == bw && (x0 > bl || (x0 == bl && x2 > bh)))) { best = e02; bw = w02; bl = x0; bh = x2; }
                    if (w12 > bw || (w12 == bw && (x1 > bl || (x1 == bl && x2 > bh)))) { best = e12; }
                    a.del[best] = 1;
                } else if constexpr (M == Mode::EoReserve) {
                    if (a.considered == nullptr || !(considered_bit(a.considered, e01) | considered_bit(a.considered, e02) |
                                                     considered_bit(a.considered, e12))) {
                        // the round's prefix of the (r2, a, b, c) order bids for its edges
                        if ((unsigned long long)r.z < a.eo_theta) {
                            const unsigned long long hi = (unsigned long long)r.z << 32;
                            atomicMin(a.resv + e01, hi | x2);
                            atomicMin(a.resv + e02, hi | x1);
                            atomicMin(a.resv + e12, hi | x0);
                        }
                        ++live;
                    }
                } else {  // EoEmit: list the live selected triangle (and bid, in case the list overflows)
                    if (a.considered == nullptr || !(considered_bit(a.considered, e01) | considered_bit(a.considered, e02) |
                                                     considered_bit(a.considered, e12))) {
                        if ((unsigned long long)r.z < a.eo_theta) {
                            const unsigned long long hi = (unsigned long long)r.z << 32;
                            atomicMin(a.resv + e01, hi | x2);
                            atomicMin(a.resv + e02, hi | x1);
                            atomicMin(a.resv + e12, hi | x0);
                        }
                        ++live;
                        emit = true;
                        rec_r2 = r.z;
                        // w is last in the degree order; of u and v the head of iuv is the later one
                        const bool u_first = head_uv == v;
                        rec = make_uint4(u_first ? u : v, iuv, u_first ? iuw : ivw, u_first ? ivw : iuw);
                    }
                }
            }
        }
        if constexpr (M == Mode::EoEmit) emit_push(a, em, emit, rec, rec_r2);
    }
}

// Decide the 32 oldest queued triangles with all lanes.
template <Mode M>
__device__ __forceinline__ void drain32_body(const TriArgs &a, const HitQueue &q, int head, uint32_t u,
                                             unsigned &live, Emitter &em) {
    const int k = (head + (threadIdx.x & 31)) & (kQ - 1);
    const uint32_t iuw = q.iuw[k];
    const uint32_t iuv = q.iuv[k];
    // the listing pass needs the head of u-v too: load it with w, before the draw
    const uint32_t huv = M == Mode::EoEmit ? __ldg(a.colp + iuv) : 0u;
    decide<M>(a, true, u, q.v[k], __ldg(a.colp + iuw), iuv, iuw, q.ivw[k], live, em, huv);
    __syncwarp();
}
template <Mode M>
__device__ __noinline__ void drain32_call(const TriArgs &a, const HitQueue &q, int head, uint32_t u, unsigned &live,
                                          Emitter &em) {
    drain32_body<M>(a, q, head, u, live, em);
}
// Out of line, so that the probe loop's register budget stays small -- except
// for the listing pass, whose 64-register budget holds it inline without the
// spills a call costs there (R-MAT s22: 80 -> 72 ms).
template <Mode M>
__device__ __forceinline__ void drain32(const TriArgs &a, const HitQueue &q, int head, uint32_t u, unsigned &live,
                                        Emitter &em) {
    drain32_body<M>(a, q, head, u, live, em);
}

// Decide everything queued for the table vertex u (the last group with idle lanes).
template <Mode M>
__device__ __forceinline__ void flush_hits(const TriArgs &a, const HitQueue &q, QState &qs, uint32_t u,
                                           unsigned &live, Emitter &em) {
    if constexpr (M != Mode::Count && M != Mode::EdgeCount && M != Mode::VertexCount) {
        const int lane = threadIdx.x & 31;
        while (qs.n >= 32) {
            drain32<M>(a, q, qs.head, u, live, em);
            qs.head = (qs.head + 32) & (kQ - 1);
            qs.n -= 32;
        }
        const bool valid = lane < qs.n;
        const int k = (qs.head + lane) & (kQ - 1);
        const uint32_t iuw = valid ? q.iuw[k] : 0u;
        const uint32_t iuv = valid ? q.iuv[k] : 0u;
        const uint32_t huv = (M == Mode::EoEmit && valid) ? __ldg(a.colp + iuv) : 0u;
        decide<M>(a, valid, u, valid ? q.v[k] : 0u, valid ? __ldg(a.colp + iuw) : 0u, iuv, iuw,
                  valid ? q.ivw[k] : 0u, live, em, huv);
        __syncwarp();
    }
    qs.head = 0;
    qs.n = 0;
}

// Shared-memory cuckoo table of N+(u) (Pagh & Rodler's cuckoo hashing; the
// concurrent exchange-based insertion follows Alcantara et al.'s GPU tables):
// every key lives in one of two slots, so a lookup reads exactly two slots
// with no probe loop and no divergence.  Load <= 1/4.  An insertion that
// keeps displacing keys for kCuckooIters exchanges leaves its homeless entry
// in a small stash that lookups then scan; a full stash raises a device error.
//
// A table of 2^L slots puts key w in slot h_j(w) = (w * K_j) >> (32 - L),
// j = 1 or 2.  The slot's 32-bit word keeps the low 32 - L bits of w * K_j
// (the slot number holds the high L bits, and multiplying by an odd K_j is a
// bijection, so word and slot give w back), which hash placed it, and w's
// position in N+(u) (< 2^(L-2) at load 1/4):
//   bits [L, 32): low bits of w * K_j;  bit L-1: j - 1;  bit L-2: 0;  bits [0, L-2): position
// An empty slot is all ones (bit L-2 set), so it matches no key, and since
// the word and slot pin down w, kEmpty (past a list's end) matches none either.
constexpr uint32_t kSlotEmpty = 0xFFFFFFFFu;
constexpr uint32_t kH1 = 0x9E3779B1u, kH2 = 0x85EBCA77u;
// inverse of an odd k modulo 2^32 (Newton's iteration doubles the correct low bits)
constexpr uint32_t inv_mod32(uint32_t k) {
    uint32_t x = k;  // k * k == 1 mod 8
    for (int i = 0; i < 5; ++i) x *= 2u - k * x;
    return x;
}
constexpr uint32_t kH1Inv = inv_mod32(kH1), kH2Inv = inv_mod32(kH2);
static_assert(kH1 * kH1Inv == 1u && kH2 * kH2Inv == 1u, "hash multipliers must be invertible");
// a stash entry is (vertex << 32 | position); this marks "not in the stash"
constexpr unsigned long long kStashNone = 0xFFFFFFFEFFFFFFFFull;
constexpr int kCuckooIters = 32;
constexpr int kStash = 16;

struct Table {
    uint32_t *slot;
    unsigned long long *stash;
    int *stash_n;
};

__device__ __forceinline__ void table_insert(const Table &t, int log_slots, uint32_t w, int i, int *err) {
    const int L = log_slots, sh = 32 - L;
    const uint32_t pmask = (1u << (L - 2)) - 1u;
    uint32_t x = w * kH1;
    uint32_t pos = x >> sh;
    uint32_t cur = (x << L) | (uint32_t)i;
    for (int it = 0; it < kCuckooIters; ++it) {
        const uint32_t old = atomicExch(t.slot + pos, cur);
        if (old == kSlotEmpty) return;
        // the evicted key moves to its other slot
        const bool by2 = (old >> (L - 1)) & 1u;
        const uint32_t wo = ((pos << sh) | (old >> L)) * (by2 ? kH2Inv : kH1Inv);
        x = wo * (by2 ? kH1 : kH2);
        pos = x >> sh;
        cur = (x << L) | ((by2 ? 0u : 1u) << (L - 1)) | (old & pmask);
    }
    const bool by2 = (cur >> (L - 1)) & 1u;
    const uint32_t wo = ((pos << sh) | (cur >> L)) * (by2 ? kH2Inv : kH1Inv);
    const int s = atomicAdd(t.stash_n, 1);
    if (s < kStash) t.stash[s] = ((unsigned long long)wo << 32) | (cur & pmask);
    else atomicExch(err, (int)kDevTableFull);
}

// w in the table's two slots?  t receives its position in N+(u).
__device__ __forceinline__ bool table_find(const Table &tb, int sh, uint32_t w, uint32_t &t) {
    const int L = 32 - sh;
    const uint32_t lim = 1u << (L - 2);
    const uint32_t x1 = w * kH1, x2 = w * kH2;
    const uint32_t a = tb.slot[x1 >> sh];
    const uint32_t b = tb.slot[x2 >> sh];
    const bool ha = (a ^ (x1 << L)) < lim;
    const bool hb = (b ^ ((x2 << L) | (lim << 1))) < lim;
    t = (ha ? a : b) & (lim - 1u);
    return ha | hb;
}

// w in the stash (the rare table whose insertion left keys there)?  Returns
// the stash entry (vertex << 32 | position), or kStashNone.
__device__ __noinline__ unsigned long long stash_find(const unsigned long long *stash, int stash_n, uint32_t w) {
    for (int k = 0; k < stash_n; ++k) {
        const unsigned long long c = stash[k];
        if ((uint32_t)(c >> 32) == w) return c;
    }
    return kStashNone;
}

// First two 32-element slabs of the list colp[ov, ov + dv) (kEmpty past its end).
__device__ __forceinline__ void first_slabs(const TriArgs &a, uint32_t ov, int dv, uint32_t &na, uint32_t &nb) {
    const int lane = threadIdx.x & 31;
    na = lane < dv ? __ldg(a.colp + ov + lane) : kEmpty;
    nb = lane + 32 < dv ? __ldg(a.colp + ov + lane + 32) : kEmpty;
}

// Stream N+(v) = colp[ov, ov + dv) through the table of N+(u): two 32-element
// slabs per iteration, the next two loaded while these are probed.  The
// caller passes the first two slabs (na, nb) already loaded, so that it can
// issue them before finishing the previous list.  Hits go to the queue.
template <Mode M>
__device__ __forceinline__ void probe_list(const TriArgs &a, const Table &tb, int log_slots, int stash_n,
                                           uint32_t u, uint32_t iuv, uint32_t ou, uint32_t v, uint32_t ov, int dv,
                                           uint32_t na, uint32_t nb, HitQueue &q, QState &qs, unsigned &live,
                                           unsigned long long &tris, Emitter &em) {
    const int lane = threadIdx.x & 31;
    const uint32_t lt = lanemask_lt();
    const uint32_t *lst = a.colp + ov;
    const int sh = 32 - log_slots;
    unsigned huv = 0;  // EdgeCount: triangles found on the arc u->v
    for (int j0 = 0; j0 < dv; j0 += 64) {
        const int ja = j0 + lane, jb = ja + 32;
        const uint32_t wa = na, wb = nb;
        uint32_t ta = 0, tb2 = 0;
        // the next two slabs are in flight while these are probed
        na = kEmpty;
        nb = kEmpty;
        if (ja + 64 < dv) na = __ldg(lst + ja + 64);
        if (jb + 64 < dv) nb = __ldg(lst + jb + 64);
        // kEmpty is never a vertex, so out-of-range lanes miss
        bool ha = table_find(tb, sh, wa, ta);
        bool hb = table_find(tb, sh, wb, tb2);
        if (stash_n != 0) {  // warp-uniform and rare
            if (!ha) {
                const unsigned long long c = stash_find(tb.stash, stash_n, wa);
                ha = c != kStashNone;
                ta = (uint32_t)c;
            }
            if (!hb) {
                const unsigned long long c = stash_find(tb.stash, stash_n, wb);
                hb = c != kStashNone;
                tb2 = (uint32_t)c;
            }
        }
        const unsigned ma = __ballot_sync(kFull, ha), mb = __ballot_sync(kFull, hb);
        if constexpr (M == Mode::EdgeCount) {
            // each hit closes a triangle through u->w and v->w; u->v is summed once
            if (ha) { atomicAdd(a.tcnt + ou + ta, 1u); atomicAdd(a.tcnt + ov + (uint32_t)ja, 1u); }
            if (hb) { atomicAdd(a.tcnt + ou + tb2, 1u); atomicAdd(a.tcnt + ov + (uint32_t)jb, 1u); }
            huv += (unsigned)(__popc(ma) + __popc(mb));
            continue;
        }
        if constexpr (M == Mode::VertexCount) {
            // each hit is a triangle through w; u and v are summed once per list
            if (ha) atomicAdd(a.vcnt + wa, 1ull);
            if (hb) atomicAdd(a.vcnt + wb, 1ull);
            huv += (unsigned)(__popc(ma) + __popc(mb));
            continue;
        }
        if constexpr (M == Mode::Count) {
            if (lane == 0) tris += (unsigned)(__popc(ma) + __popc(mb));
            continue;
        }
        if (ma | mb) {
            const int pa = __popc(ma), pb = __popc(mb);
            const int tail = qs.head + qs.n;
            if (ha) {
                const int s0 = (tail + __popc(ma & lt)) & (kQ - 1);
                q.v[s0] = v; q.iuv[s0] = iuv; q.iuw[s0] = ou + ta; q.ivw[s0] = ov + (uint32_t)ja;
            }
            if (hb) {
                const int s0 = (tail + pa + __popc(mb & lt)) & (kQ - 1);
                q.v[s0] = v; q.iuv[s0] = iuv; q.iuw[s0] = ou + tb2; q.ivw[s0] = ov + (uint32_t)jb;
            }
            qs.n += pa + pb;
            if (lane == 0) tris += (unsigned)(pa + pb);
            __syncwarp();
            while (qs.n >= 32) {
                drain32<M>(a, q, qs.head, u, live, em);
                qs.head = (qs.head + 32) & (kQ - 1);
                qs.n -= 32;
            }
        }
    }
    if constexpr (M == Mode::EdgeCount) {
        if (lane == 0 && huv) {
            atomicAdd(a.tcnt + iuv, huv);
            tris += huv;
        }
    }
    if constexpr (M == Mode::VertexCount) {
        if (lane == 0 && huv) {
            atomicAdd(a.vcnt + u, (unsigned long long)huv);
            atomicAdd(a.vcnt + v, (unsigned long long)huv);
            tris += huv;
        }
    }
}

// Stream the in-lists [first, first + cnt) (cnt <= 32) of the table vertex u:
// the lanes load the arcs' records and list bounds in parallel, then the warp
// streams the lists one by one.
template <Mode M>
__device__ __forceinline__ void stream_in_group(const TriArgs &a, const Table &tb, int log_slots, int stash_n,
                                                uint32_t u, int du, uint32_t tbase, int64_t ib, int first, int cnt,
                                                HitQueue &q, QState &qs, unsigned &live, unsigned long long &probes,
                                                unsigned long long &tris, Emitter &em, bool count_probes) {
    const int lane = threadIdx.x & 31;
    uint32_t sv = 0, so = 0, se = 0;
    int sd = 0;
    if (lane < cnt) {
        const uint2 it = __ldg(a.inl + ib + first + lane);
        sv = it.x;
        se = it.y;
        const int64_t b0 = __ldg(a.offp + sv);
        so = (uint32_t)b0;
        // an in-arc v->u whose tail has d+(v) >= d+(u) is streamed from v's side
        const int dvv = (int)(__ldg(a.offp + sv + 1) - b0);
        sd = (dvv >= du || (kEdgeOnce<M> && a.considered != nullptr && considered_bit(a.considered, se))) ? 0 : dvv;
    }
    // the next list's first slabs load while the current one is probed
    uint32_t pa, pb;
    first_slabs(a, __shfl_sync(kFull, so, 0), __shfl_sync(kFull, sd, 0), pa, pb);
    for (int i = 0; i < cnt; ++i) {
        const uint32_t v = __shfl_sync(kFull, sv, i);
        const uint32_t ov = __shfl_sync(kFull, so, i);
        const uint32_t e = __shfl_sync(kFull, se, i);
        const int dv = __shfl_sync(kFull, sd, i);
        const uint32_t ca = pa, cb = pb;
        if (i + 1 < cnt) first_slabs(a, __shfl_sync(kFull, so, i + 1), __shfl_sync(kFull, sd, i + 1), pa, pb);
        if (lane == 0 && count_probes) probes += (unsigned)dv;
        probe_list<M>(a, tb, log_slots, stash_n, u, e, tbase, v, ov, dv, ca, cb, q, qs, live, tris, em);
    }
}

template <Mode M>
__device__ __forceinline__ void finish(const TriArgs &a, unsigned live, unsigned long long probes,
                                       unsigned long long tris, Emitter &em) {
    if constexpr (M == Mode::EoEmit) {
        for (int b = 0; b < em.hi; ++b)
            emit_seal(a, __shfl_sync(kFull, em.cur, b), __shfl_sync(kFull, em.cur, 8 + b));
        const int lane = threadIdx.x & 31;
        if (lane >= 16 && lane < 16 + kEoBuckets && em.cur != 0) atomicAdd(a.list_dem + (lane - 16), em.cur);
    }
    const unsigned long long P = warp_sum(probes), T = warp_sum(tris);
    const unsigned L = warp_sum(live);
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(a.ctr + kCtrProbes, P);
        atomicAdd(a.ctr + kCtrTriangles, T);
        if (L) atomicAdd(a.ctr + kCtrLive, (unsigned long long)L);
    }
}

// One persistent launch per enumeration pass.
// Phase 1: heavy vertices (large N+(u) or many lists to stream), largest work
// bound first; a CTA stages N+(u) in a shared-memory table (plus every
// out-neighbour's list bounds) and its warps claim out-arcs one at a time and
// in-arcs 32 at a time.  Phase 2: light vertices, a warp per vertex with its
// own small table; warps claim 32 vertex ids at a time.  Probe and triangle
// totals are counted per list and per found triangle.  The counting passes
// run 5 CTAs per SM at 48 registers; the passes that decide triangles keep 64
// (4 CTAs per SM): at 48 their queue drain and record assembly spill.
//
// The hub launch (TW = kHubTW) runs phase 1 alone, before the main launch,
// over the vertices whose N+(u) is too long for the main launch's table: one
// CTA of 32 warps per SM shares a table of up to kHubCap entries, so those
// lists are streamed once instead of once per table chunk.
template <Mode M>
constexpr int kEnumCtasPerSm = (M == Mode::Count || M == Mode::EdgeCount || M == Mode::VertexCount) ? 5 : 4;

template <Mode M, int TW>
__global__ void __launch_bounds__(TW * 32, TW == kTW ? kEnumCtasPerSm<M> : 1) tri_enum_kernel(TriArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_next;
    __shared__ long long s_h;
    __shared__ int s_stash_n[TW + 1];
    __shared__ unsigned long long s_stash[TW + 1][kStash];
    HitQueue *qs = reinterpret_cast<HitQueue *>(smem);
    unsigned char *tbl = smem + sizeof(HitQueue) * TW;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    HitQueue &q = qs[warp];
    QState qst;
    unsigned live = 0;
    unsigned long long probes = 0, tris = 0;
    Emitter em;
    em.hi = a.eo_hi;
    const int64_t n_heavy = a.n_heavy_dev ? (int64_t)*a.n_heavy_dev : a.n_heavy;

    // ---- phase 1: heavy vertices
    {
        const int cap = a.heavy_cap;  // table capacity: larger N+(u) is processed in chunks
        const int slots = 4 * cap;
        Table tb{reinterpret_cast<uint32_t *>(tbl), s_stash[TW], &s_stash_n[TW]};
        uint32_t *vv = tb.slot + slots;  // v, off+(v), d+(v) of N+(u)
        uint32_t *vo = vv + cap;
        unsigned short *vd = reinterpret_cast<unsigned short *>(vo + cap);  // d+(v) <= d+(u) <= cap, else 0
        for (;;) {
            if (threadIdx.x == 0) s_h = (long long)atomicAdd(a.work, 1ull);
            __syncthreads();
            const int64_t h = s_h;
            if (h >= n_heavy) break;
            const uint32_t u = __ldg(a.heavy + h);
            const uint32_t ou = (uint32_t)__ldg(a.offp + u);
            const int d = (int)(__ldg(a.offp + u + 1) - (int64_t)ou);
            const int nin = (int)__ldg(a.din + u);
            const int items = d + (nin + 31) / 32;                    // out-arcs, then groups of 32 in-arcs
            const int64_t ib = __ldg(a.offs + u) - (int64_t)ou;       // start of u's in-arcs in inl
            const bool staged = d <= cap;  // list bounds of N+(u) kept in shared memory
            for (int c0 = 0; c0 < d; c0 += cap) {
                const int cn = min(cap, d - c0);
                const int log_slots = ceil_log2(4 * cn) < 3 ? 3 : ceil_log2(4 * cn);
                for (int s2 = threadIdx.x; s2 < (1 << log_slots); s2 += blockDim.x) tb.slot[s2] = kSlotEmpty;
                if (threadIdx.x == 0) {
                    s_next = 0;
                    *tb.stash_n = 0;
                }
                __syncthreads();
                for (int k = threadIdx.x; k < cn; k += blockDim.x) {
                    const int i = c0 + k;
                    const uint32_t v = __ldg(a.colp + ou + i);
                    const bool dead = kEdgeOnce<M> && a.considered != nullptr &&
                                      considered_bit(a.considered, (int64_t)ou + i);
                    if (staged) {
                        const int64_t ov = __ldg(a.offp + v);
                        const int dv = (int)(__ldg(a.offp + v + 1) - ov);
                        vv[i] = v;
                        vo[i] = (uint32_t)ov;
                        // a considered arc u->v closes no live triangle; an arc
                        // with d+(v) > d+(u) is streamed from v's side
                        vd[i] = (unsigned short)((dead || dv > d) ? 0 : dv);
                    }
                    if (!dead) table_insert(tb, log_slots, v, k, a.err);
                }
                __syncthreads();
                const int stash_n = min(*tb.stash_n, kStash);
                for (;;) {
                    int i = 0;
                    if (lane == 0) i = atomicAdd(&s_next, 1);
                    i = __shfl_sync(kFull, i, 0);
                    if (i >= items) break;
                    {  // hand out the in-arc groups (the larger units) first, then the out-arcs
                        const int ng = items - d;
                        i = i < ng ? d + i : i - ng;
                    }
                    if (i >= d) {  // 32 in-arcs v->u with d+(v) < d+(u): stream each N+(v)
                        const int g0 = (i - d) * 32;
                        stream_in_group<M>(a, tb, log_slots, stash_n, u, d, ou + (uint32_t)c0, ib, g0,
                                           min(32, nin - g0), q, qst, live, probes, tris, em, c0 == 0);
                        continue;
                    }
                    // out-arc u->v: stream N+(v)
                    const uint32_t e = ou + (uint32_t)i;
                    uint32_t v, ov;
                    int dv;
                    if (staged) {
                        v = vv[i];
                        ov = vo[i];
                        dv = vd[i];
                    } else {
                        v = __ldg(a.colp + e);
                        const int64_t o64 = __ldg(a.offp + v);
                        ov = (uint32_t)o64;
                        dv = (int)(__ldg(a.offp + v + 1) - o64);
                        if (dv > d || (kEdgeOnce<M> && a.considered != nullptr && considered_bit(a.considered, e))) dv = 0;
                    }
                    // algorithmic probes: a chunked N+(u) re-reads the lists, which is not counted
                    if (lane == 0 && c0 == 0) probes += (unsigned)dv;
                    uint32_t ca, cb;
                    first_slabs(a, ov, dv, ca, cb);
                    probe_list<M>(a, tb, log_slots, stash_n, u, e, ou + (uint32_t)c0, v, ov, dv, ca, cb, q, qst,
                                  live, tris, em);
                }
                __syncthreads();  // the table is rebuilt for the next chunk or vertex
            }
            flush_hits<M>(a, q, qst, u, live, em);
        }
    }

    // ---- phase 2: light vertices
    if constexpr (TW == kTW) {
        Table tb{reinterpret_cast<uint32_t *>(tbl) + warp * kLightSlots, s_stash[warp], &s_stash_n[warp]};
        for (;;) {
            unsigned long long base = 0;
            if (lane == 0) base = atomicAdd(a.work + 1, 32ull);
            base = __shfl_sync(kFull, base, 0);
            if ((int64_t)base >= a.n) break;
            const int64_t ul = (int64_t)base + lane;
            uint32_t oul = 0;
            int dl = 0, nl = 0;
            if (ul < a.n) {
                const int64_t o0 = __ldg(a.offp + ul);
                oul = (uint32_t)o0;
                dl = (int)(__ldg(a.offp + ul + 1) - o0);
                nl = (int)__ldg(a.din + ul);
            }
            // d+(u) < 2 closes no triangle at u (and then u has no in-arcs to stream)
            unsigned lm = __ballot_sync(kFull, dl >= 2 && dl <= a.light_max && dl + nl <= a.light_items);
            while (lm) {
                const int src = __ffs(lm) - 1;
                lm &= lm - 1;
                const uint32_t u = (uint32_t)(base + src);
                const uint32_t ou = __shfl_sync(kFull, oul, src);
                const int d = __shfl_sync(kFull, dl, src);
                const int nin = __shfl_sync(kFull, nl, src);
                const int log_slots = max(3, ceil_log2(4 * d));
                for (int s2 = lane; s2 < (1 << log_slots); s2 += 32) tb.slot[s2] = kSlotEmpty;
                if (lane == 0) *tb.stash_n = 0;
                __syncwarp();
                // lane k holds N+(u)[k] and N+(u)[k + 32] with their list bounds
                uint32_t n0 = kEmpty, n1 = kEmpty, o0 = 0, o1 = 0;
                int d0 = 0, d1 = 0;
                bool live0 = false, live1 = false;  // the arc u->w may close a live triangle
                if (lane < d) {
                    n0 = __ldg(a.colp + ou + lane);
                    const int64_t b0 = __ldg(a.offp + n0);
                    o0 = (uint32_t)b0;
                    d0 = (int)(__ldg(a.offp + n0 + 1) - b0);
                    live0 = !kEdgeOnce<M> || a.considered == nullptr || !considered_bit(a.considered, (int64_t)ou + lane);
                    if (live0) table_insert(tb, log_slots, n0, lane, a.err);
                    if (!live0 || d0 > d) d0 = 0;  // streamed from n0's side when d+(n0) > d+(u)
                }
                if (lane + 32 < d) {
                    n1 = __ldg(a.colp + ou + lane + 32);
                    const int64_t b1 = __ldg(a.offp + n1);
                    o1 = (uint32_t)b1;
                    d1 = (int)(__ldg(a.offp + n1 + 1) - b1);
                    live1 = !kEdgeOnce<M> || a.considered == nullptr ||
                            !considered_bit(a.considered, (int64_t)ou + lane + 32);
                    if (live1) table_insert(tb, log_slots, n1, lane + 32, a.err);
                    if (!live1 || d1 > d) d1 = 0;
                }
                __syncwarp();
                const int stash_n = min(*tb.stash_n, kStash);
                uint32_t pa, pb;  // first slabs of the next list, loading ahead
                first_slabs(a, __shfl_sync(kFull, o0, 0), __shfl_sync(kFull, d0, 0), pa, pb);
                for (int i = 0; i < d; ++i) {
                    const bool lo = i < 32;
                    const uint32_t v = __shfl_sync(kFull, lo ? n0 : n1, i & 31);
                    const uint32_t ov = __shfl_sync(kFull, lo ? o0 : o1, i & 31);
                    const int dv = __shfl_sync(kFull, lo ? d0 : d1, i & 31);
                    const uint32_t ca = pa, cb = pb;
                    if (i + 1 < d) {
                        const bool ln = i + 1 < 32;
                        first_slabs(a, __shfl_sync(kFull, ln ? o0 : o1, (i + 1) & 31),
                                    __shfl_sync(kFull, ln ? d0 : d1, (i + 1) & 31), pa, pb);
                    }
                    if (lane == 0) probes += (unsigned)dv;
                    probe_list<M>(a, tb, log_slots, stash_n, u, ou + (uint32_t)i, ou, v, ov, dv, ca, cb, q, qst,
                                  live, tris, em);
                }
                // in-arcs v->u with d+(v) < d+(u), in groups of 32
                const int64_t ib = nin > 0 ? __ldg(a.offs + u) - (int64_t)ou : 0;
                for (int c = 0; c < nin; c += 32)
                    stream_in_group<M>(a, tb, log_slots, stash_n, u, d, ou, ib, c, min(32, nin - c), q, qst,
                                       live, probes, tris, em, true);
                flush_hits<M>(a, q, qst, u, live, em);
                __syncwarp();
            }
        }
    }
    finish<M>(a, live, probes, tris, em);
}

// Heavy vertices in decreasing out-degree order, by log2 buckets: pass 1
// counts the vertices of each bucket (and the maximum out-degree), pass 2
// scatters them so that larger buckets come first.
constexpr int kBuckets = 52;  // floor(log2) of the work bound d+ (d+ + in-arcs)
// sort keys: the bucket, plus kBuckets for a hub (d+ > hub_min), so hubs come first
constexpr int kKeys = 2 * kBuckets;

__device__ __forceinline__ int bucket_of(unsigned long long d) { return 63 - __clzll(d); }

// A vertex goes to the CTA phase when its table or its arc count is too large
// for one warp; the bucket orders those vertices by the bound d+(x) * (d+(x) +
// in-arcs(x)) on the probes made there (every streamed list is at most d+(x)).
__device__ __forceinline__ bool is_heavy(int64_t d, int64_t nin, int light_max, int light_items) {
    return d >= 2 && (d > light_max || d + nin > light_items);
}
__device__ __forceinline__ int heavy_bucket(int64_t d, int64_t nin) {
    return min(bucket_of((unsigned long long)d * (unsigned long long)(d + nin)), kBuckets - 1);
}
__device__ __forceinline__ int heavy_key(int64_t d, int64_t nin, int64_t hub_min) {
    return heavy_bucket(d, nin) + (d > hub_min ? kBuckets : 0);
}

// Also writes every vertex's in-degree d(u) - d+(u): the length of its
// in-list in the reverse list (see Oriented::inl).
__global__ void classify_count_kernel(const int64_t *__restrict__ offp, const int64_t *__restrict__ offs,
                                      uint32_t *din, int64_t n, int light_max, int light_items, int64_t hub_min,
                                      unsigned long long *bucket_cnt, unsigned long long *ctr) {
    __shared__ unsigned int s_cnt[kKeys];
    if (threadIdx.x < kKeys) s_cnt[threadIdx.x] = 0;
    __syncthreads();
    unsigned long long dmax = 0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < n; u += stride) {
        const int64_t d = offp[u + 1] - offp[u];
        dmax = d > (int64_t)dmax ? (unsigned long long)d : dmax;
        int64_t nin = (offs[u + 1] - offs[u]) - d;
        nin = nin < 0 ? 0 : nin;
        din[u] = (uint32_t)nin;
        if (is_heavy(d, nin, light_max, light_items)) atomicAdd(&s_cnt[heavy_key(d, nin, hub_min)], 1u);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long t = __shfl_xor_sync(kFull, dmax, o);
        dmax = t > dmax ? t : dmax;
    }
    if ((threadIdx.x & 31) == 0) atomicMax(ctr + kCtrMaxDeg, dmax);
    __syncthreads();
    if (threadIdx.x < kKeys && s_cnt[threadIdx.x]) atomicAdd(bucket_cnt + threadIdx.x, (unsigned long long)s_cnt[threadIdx.x]);
}

__global__ void classify_scatter_kernel(const int64_t *__restrict__ offp, const uint32_t *__restrict__ din,
                                        int64_t n, int light_max, int light_items, int64_t hub_min,
                                        const unsigned long long *__restrict__ bucket_cnt,
                                        unsigned long long *bucket_fill, uint32_t *heavy,
                                        unsigned long long *total_out) {
    __shared__ unsigned long long s_off[kKeys];
    if (threadIdx.x == 0) {
        unsigned long long run = 0;
        for (int b = kKeys - 1; b >= 0; --b) {
            s_off[b] = run;
            run += bucket_cnt[b];
        }
        if (blockIdx.x == 0 && total_out) *total_out = run;
    }
    __syncthreads();
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < n; u += stride) {
        const int64_t d = offp[u + 1] - offp[u];
        const int64_t nin = din[u];
        if (is_heavy(d, nin, light_max, light_items)) {
            const int b = heavy_key(d, nin, hub_min);
            heavy[s_off[b] + atomicAdd(bucket_fill + b, 1ull)] = (uint32_t)u;
        }
    }
}

// Edge-Once acceptance: an oriented arc e = u->y holding reservation
// (r2, z) belongs to the accepted triangle {u, y, z} iff that triangle also
// holds the reservations of its two other edges.
// returns -1 when the arc is missing (never for a symmetric CSR)
__device__ __forceinline__ int64_t arc_between(const int64_t *off, const int64_t *offp, const uint32_t *colp,
                                               uint32_t p, uint32_t q) {
    const int64_t dp = __ldg(off + p + 1) - __ldg(off + p);
    const int64_t dq = __ldg(off + q + 1) - __ldg(off + q);
    const bool pq = dp < dq || (dp == dq && p < q);
    const uint32_t row = pq ? p : q, key = pq ? q : p;
    const int64_t end = __ldg(offp + row + 1);
    const int64_t i = lower_bound_u32(colp, __ldg(offp + row), end, key);
    return (i < end && __ldg(colp + i) == key) ? i : -1;
}

// Which edge an accepted triangle deletes.
enum Choice { kChoiceRandom = 0, kChoiceMaxw = 1, kChoiceMinCount = 2 };

template <int CH>
__global__ void eo_accept_kernel(TriArgs a, const int64_t *__restrict__ off, uint32_t *considered) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t u = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp; u < a.n; u += nw) {
        const int64_t ou = __ldg(a.offp + u), d = __ldg(a.offp + u + 1) - ou;
        for (int64_t i = lane; i < d; i += 32) {
            const int64_t e = ou + i;
            const unsigned long long r = a.resv[e];
            if (r == ~0ull) continue;
            const uint32_t y = __ldg(a.colp + e);
            const uint32_t z = (uint32_t)r;
            const unsigned long long hi = r & 0xFFFFFFFF00000000ull;
            const int64_t f1 = arc_between(off, a.offp, a.colp, (uint32_t)u, z);
            const int64_t f2 = arc_between(off, a.offp, a.colp, y, z);
            if (f1 < 0 || f2 < 0) continue;
            if (a.resv[f1] != (hi | y) || a.resv[f2] != (hi | (uint32_t)u)) continue;
            set_considered(considered, e);
            // which edge of the accepted triangle goes
            uint32_t x0 = (uint32_t)u, x1 = y, x2 = z;
            int64_t e01 = e, e02 = f1, e12 = f2;
            if (x0 > x1) { swap2(x0, x1); swap2(e02, e12); }
            if (x1 > x2) { swap2(x1, x2); swap2(e01, e02); }
            if (x0 > x1) { swap2(x0, x1); swap2(e02, e12); }
            int64_t chosen;
            if constexpr (CH == kChoiceMinCount) {
                chosen = mincount_arc(a.tcnt, e01, e02, e12);
            } else if constexpr (CH == kChoiceMaxw) {
                const float w01 = __ldg(a.wp + e01), w02 = __ldg(a.wp + e02), w12 = __ldg(a.wp + e12);
                chosen = e01;
                float bw = w01;
                uint32_t bl = x0, bh = x1;
                if (w02 > bw || (w02 == bw && (x0 > bl || (x0 == bl && x2 > bh)))) { chosen = e02; bw = w02; bl = x0; bh = x2; }
                if (w12 > bw || (w12 == bw && (x1 > bl || (x1 == bl && x2 > bh)))) { chosen = e12; }
            } else {
                const uint4 rr = philox4x32_10(make_uint4(x0, x1, x2, kTagTri), a.k0, a.k1);
                const int k = (int)(((unsigned long long)rr.y * 3ull) >> 32);
                chosen = k == 0 ? e01 : (k == 1 ? e02 : e12);
            }
            if (chosen == e) a.del[e] = 1;
        }
    }
}

// Edge-once rounds over the list of live selected triangles.
// Accept: a triangle holding the reservations of all three of its edges is
// accepted; accepted triangles are edge-disjoint, so their stores never race.
template <int CH>
__global__ void eo_list_accept_kernel(const TriRec *__restrict__ L, int64_t len,
                                      const unsigned long long *__restrict__ resv, uint32_t *considered,
                                      uint8_t *del, const float *__restrict__ wp, const uint32_t *__restrict__ tcnt) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < len; i += stride) {
        const TriRec r = L[i];
        if (r.x0 == kSentinel) continue;
        const unsigned long long hi = (unsigned long long)r.r2 << 32;
        if (resv[r.e01] != (hi | r.x2) || resv[r.e02] != (hi | r.x1) || resv[r.e12] != (hi | r.x0)) continue;
        set_considered(considered, (int64_t)r.e01);
        set_considered(considered, (int64_t)r.e02);
        set_considered(considered, (int64_t)r.e12);
        uint32_t chosen;
        if constexpr (CH == kChoiceMinCount) {
            chosen = mincount_arc(tcnt, r.e01, r.e02, r.e12);
        } else if constexpr (CH == kChoiceMaxw) {
            const float w01 = __ldg(wp + r.e01), w02 = __ldg(wp + r.e02), w12 = __ldg(wp + r.e12);
            chosen = r.e01;
            float bw = w01;
            uint32_t bl = r.x0, bh = r.x1;
            if (w02 > bw || (w02 == bw && (r.x0 > bl || (r.x0 == bl && r.x2 > bh)))) { chosen = r.e02; bw = w02; bl = r.x0; bh = r.x2; }
            if (w12 > bw || (w12 == bw && (r.x1 > bl || (r.x1 == bl && r.x2 > bh)))) { chosen = r.e12; }
        } else {
            const int k = (int)(((unsigned long long)r.r1 * 3ull) >> 32);
            chosen = k == 0 ? r.e01 : (k == 1 ? r.e02 : r.e12);
        }
        del[chosen] = 1;
    }
}

// Reserve: drop every triangle that lost an edge to an accepted one, reserve
// the edges of the survivors (64-bit atomicMin of (r2, third vertex)) and
// compact the survivors into `out` (block-aggregated appends).
__global__ void __launch_bounds__(256) eo_list_reserve_kernel(const TriRec *__restrict__ L, int64_t len,
                                                              TriRec *__restrict__ out,
                                                              unsigned long long *out_len,
                                                              unsigned long long *resv,
                                                              const uint32_t *__restrict__ considered,
                                                              unsigned long long theta) {
    __shared__ int s_cnt[8];
    __shared__ unsigned long long s_base;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < len; base += stride) {
        const int64_t i = base + threadIdx.x;
        bool keep = false;
        TriRec r{kSentinel, 0, 0, 0, 0, 0, 0, 0};
        if (i < len) {
            r = L[i];
            if (r.x0 != kSentinel && !(considered_bit(considered, r.e01) | considered_bit(considered, r.e02) |
                                       considered_bit(considered, r.e12))) {
                keep = true;
                if ((unsigned long long)r.r2 < theta) {
                    const unsigned long long hi = (unsigned long long)r.r2 << 32;
                    atomicMin(resv + r.e01, hi | r.x2);
                    atomicMin(resv + r.e02, hi | r.x1);
                    atomicMin(resv + r.e12, hi | r.x0);
                }
            }
        }
        const unsigned bm = __ballot_sync(kFull, keep);
        if (lane == 0) s_cnt[warp] = __popc(bm);
        __syncthreads();
        if (threadIdx.x == 0) {
            int tot = 0;
            for (int k = 0; k < 8; ++k) {
                const int c = s_cnt[k];
                s_cnt[k] = tot;
                tot += c;
            }
            s_base = tot ? atomicAdd(out_len, (unsigned long long)tot) : 0ull;
        }
        __syncthreads();
        if (keep) out[s_base + s_cnt[warp] + __popc(bm & lanemask_lt())] = r;
        __syncthreads();
    }
}

// Reserve for a bucket written by the enumeration: drop the triangles that
// lost an edge, expand the survivors to full records (vertices from the arc
// heads, draws recomputed), bid and append them to `out`.  Each thread takes
// kFreshPer records per pass (their loads overlap) and a CTA appends its
// survivors with one atomic per pass.
constexpr int kFreshPer = 4;

__global__ void __launch_bounds__(256) eo_fresh_reserve_kernel(const uint4 *__restrict__ F, int64_t len,
                                                               TriRec *__restrict__ out, unsigned long long *out_len,
                                                               unsigned long long *resv,
                                                               const uint32_t *__restrict__ considered,
                                                               unsigned long long theta,
                                                               const uint32_t *__restrict__ colp, uint32_t k0,
                                                               uint32_t k1) {
    __shared__ int s_cnt[8];
    __shared__ unsigned long long s_base;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t span = (int64_t)blockDim.x * kFreshPer;
    for (int64_t base = (int64_t)blockIdx.x * span; base < len; base += (int64_t)gridDim.x * span) {
        uint4 f[kFreshPer];
        bool keep[kFreshPer];
#pragma unroll
        for (int r = 0; r < kFreshPer; ++r) {
            const int64_t i = base + r * blockDim.x + threadIdx.x;
            f[r] = i < len ? __ldg(F + i) : make_uint4(kSentinel, 0u, 0u, 0u);
        }
#pragma unroll
        for (int r = 0; r < kFreshPer; ++r)
            keep[r] = f[r].x != kSentinel && !(considered_bit(considered, f[r].y) | considered_bit(considered, f[r].z) |
                                               considered_bit(considered, f[r].w));
        int cnt = 0;
#pragma unroll
        for (int r = 0; r < kFreshPer; ++r) cnt += keep[r];
        int inc = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(kFull, inc, o);
            if (lane >= o) inc += t;
        }
        if (lane == 31) s_cnt[warp] = inc;
        __syncthreads();
        if (threadIdx.x == 0) {
            int tot = 0;
            for (int k = 0; k < 8; ++k) {
                const int c = s_cnt[k];
                s_cnt[k] = tot;
                tot += c;
            }
            s_base = tot ? atomicAdd(out_len, (unsigned long long)tot) : 0ull;
        }
        __syncthreads();
        unsigned long long slot = s_base + s_cnt[warp] + (inc - cnt);
#pragma unroll
        for (int r = 0; r < kFreshPer; ++r) {
            if (!keep[r]) continue;
            uint32_t x0 = f[r].x, x1 = __ldg(colp + f[r].y), x2 = __ldg(colp + f[r].z);
            uint32_t e01 = f[r].y, e02 = f[r].z, e12 = f[r].w;
            if (x0 > x1) { swap2(x0, x1); swap2(e02, e12); }
            if (x1 > x2) { swap2(x1, x2); swap2(e01, e02); }
            if (x0 > x1) { swap2(x0, x1); swap2(e02, e12); }
            const uint4 d = philox4x32_10(make_uint4(x0, x1, x2, kTagTri), k0, k1);
            if ((unsigned long long)d.z < theta) {
                const unsigned long long hi = (unsigned long long)d.z << 32;
                atomicMin(resv + e01, hi | x2);
                atomicMin(resv + e02, hi | x1);
                atomicMin(resv + e12, hi | x0);
            }
            out[slot++] = TriRec{x0, x1, x2, d.y, d.z, e01, e02, e12};
        }
        __syncthreads();
    }
}

// Clear the reservations of the listed triangles' edges (cheaper than a full
// reset once the list is short): every reserved edge belongs to a listed triangle.
__global__ void eo_list_reset_kernel(const TriRec *__restrict__ L, int64_t len, unsigned long long *resv) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < len; i += stride) {
        const TriRec r = L[i];
        if (r.x0 == kSentinel) continue;
        resv[r.e01] = ~0ull;
        resv[r.e02] = ~0ull;
        resv[r.e12] = ~0ull;
    }
}

// -------------------------------------------------------------------- host
struct Plan {
    uint32_t *heavy = nullptr;
    unsigned long long *buckets = nullptr;  // counts [kKeys], fills [kKeys]
    uint32_t *din = nullptr;                // in-arcs streamed from the head's side, per vertex
    uint2 *inl = nullptr;                   // their (tail, arc), at offs(v) - offp(v) per vertex
    const int64_t *offs = nullptr;          // symmetric offsets of the graph
    int64_t n_heavy = 0, max_deg = 0;
    int64_t work = 0;    // W = sum over arcs of min(d+(u), d+(v)): the probes of one pass
    int64_t n_hubs = 0;  // the first n_hubs heavy vertices (d+ > kHeavyCap) go to the hub launch
    int hub_cap = 0;     // hub table entries
    size_t hub_smem = 0;
    int light_max = kLightMax;
    int light_items = kLightItems;
    int log_slots = 3;
    size_t smem = 0;
    int heavy_cap = 8;  // phase-1 table entries
};

static sg_status read_ctr(Ctx *c, int first, int count, unsigned long long *out) {
    SG_CUDA(cudaMemcpyAsync(c->h_pinned, c->d_ctr + first, sizeof(unsigned long long) * count,
                            cudaMemcpyDeviceToHost, c->stream));
    SG_CUDA(cudaStreamSynchronize(c->stream));
    std::memcpy(out, c->h_pinned, sizeof(unsigned long long) * count);
    return SG_OK;
}

static void free_plan(Ctx *c, Plan *pl) {
    dfree(c, pl->heavy);
    dfree(c, pl->buckets);
    dfree(c, pl->din);
    pl->heavy = nullptr;
    pl->buckets = nullptr;
    pl->din = nullptr;
    pl->inl = nullptr;
}


// inl_cap: room for in-arc records; nnz - m when E+ holds all m arcs, nnz
// when it may hold fewer (batches orient only their triangle-kernel graphs).
static sg_status make_plan(Ctx *c, const Oriented &o, const int64_t *offs, Plan *pl) {
    if (o.m >= (int64_t)0xFFFFFFFFll)
        return fail(SG_ERR_UNSUPPORTED, "triangle kernels address oriented arcs with 32 bits: m must be < 2^32");
    if (o.n >= (int64_t)0xFFFFFFFEll)
        return fail(SG_ERR_UNSUPPORTED, "triangle kernels reserve vertex ids 2^32 - 2 and 2^32 - 1");
    pl->offs = offs;
    sg_status st = dalloc(c, (void **)&pl->heavy, sizeof(uint32_t) * (size_t)std::max<int64_t>(o.n, 1));
    if (st == SG_OK) st = dalloc(c, (void **)&pl->buckets, sizeof(unsigned long long) * 2 * kKeys);
    if (st == SG_OK) st = dalloc(c, (void **)&pl->din, sizeof(uint32_t) * (size_t)std::max<int64_t>(o.n, 1));
    if (st != SG_OK) return st;
    pl->inl = o.inl;  // the orientation's reverse list (not owned by the plan)
    SG_CUDA(cudaMemsetAsync(pl->buckets, 0, sizeof(unsigned long long) * 2 * kKeys, c->stream));
    SG_CUDA(cudaMemsetAsync(c->d_ctr + kCtrMaxDeg, 0, sizeof(unsigned long long), c->stream));
    const int64_t blocks = std::max<int64_t>(1, std::min<int64_t>((o.n + 255) / 256, (int64_t)c->num_sms * 8));
    if (o.n > 0) {
        SG_LAUNCH(c, "tri_classify");
        classify_count_kernel<<<(unsigned)blocks, 256, 0, c->stream>>>(o.off, offs, pl->din, o.n, pl->light_max,
                                                                       pl->light_items, (int64_t)kHeavyCap,
                                                                       pl->buckets, c->d_ctr);
    }
    SG_CUDA(cudaGetLastError());
    SG_CUDA(cudaMemcpyAsync(c->h_pinned, pl->buckets, sizeof(unsigned long long) * kKeys, cudaMemcpyDeviceToHost,
                            c->stream));
    SG_CUDA(cudaMemcpyAsync(c->h_pinned + kKeys, c->d_ctr + kCtrMaxDeg, sizeof(unsigned long long),
                            cudaMemcpyDeviceToHost, c->stream));
    SG_CUDA(cudaMemcpyAsync(c->h_pinned + kKeys + 1, c->d_ctr + kCtrWork, sizeof(unsigned long long),
                            cudaMemcpyDeviceToHost, c->stream));
    SG_CUDA(cudaStreamSynchronize(c->stream));
    unsigned long long cnt[kKeys + 2];
    std::memcpy(cnt, c->h_pinned, sizeof(cnt));
    pl->work = (int64_t)cnt[kKeys + 1];
    pl->n_heavy = 0;
    pl->n_hubs = 0;
    for (int b = 0; b < kKeys; ++b) pl->n_heavy += (int64_t)cnt[b];
    for (int b = kBuckets; b < kKeys; ++b) pl->n_hubs += (int64_t)cnt[b];
    pl->max_deg = (int64_t)cnt[kKeys];
    // a hub launch with fewer hubs than SMs would leave most SMs idle: the
    // main launch then takes them first (they lead the list), in chunks
    if (pl->n_hubs < c->num_sms) pl->n_hubs = 0;
    if (pl->n_heavy > 0) {
        SG_LAUNCH(c, "tri_classify");
        classify_scatter_kernel<<<(unsigned)blocks, 256, 0, c->stream>>>(o.off, pl->din, o.n, pl->light_max,
                                                                         pl->light_items, (int64_t)kHeavyCap,
                                                                         pl->buckets, pl->buckets + kKeys,
                                                                         pl->heavy, nullptr);
    }
    SG_CUDA(cudaGetLastError());
    // shared memory: hit queues + the larger of the heavy table (4 slots per
    // entry, load <= 1/4, with the list bounds of N+(u)) and the light tables
    const size_t queue_bytes = sizeof(HitQueue) * kTW;
    const size_t light_bytes = (size_t)kTW * kLightSlots * sizeof(uint32_t);
    int cap = 8;
    while (cap < pl->max_deg && cap < kHeavyCap) cap *= 2;
    pl->heavy_cap = cap;
    pl->log_slots = ceil_log2_host(4 * cap);
    const size_t entry_bytes = 4 * sizeof(uint32_t) + 2 * sizeof(uint32_t) + sizeof(unsigned short);
    pl->smem = queue_bytes + std::max(light_bytes, (size_t)cap * entry_bytes);
    if (pl->n_hubs > 0) {
        int hc = kHeavyCap;
        while (hc < pl->max_deg && hc < kHubCap) hc *= 2;
        pl->hub_cap = hc;
        pl->hub_smem = sizeof(HitQueue) * kHubTW + (size_t)hc * entry_bytes;
    }
    return SG_OK;
}

template <Mode M>
static sg_status launch_enum_raw(Ctx *c, TriArgs a, size_t smem, int grid_per_sm) {
    SG_CUDA(cudaMemsetAsync(a.work, 0, 2 * sizeof(unsigned long long), c->stream));
    SG_CUDA(cudaFuncSetAttribute(tri_enum_kernel<M, kTW>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    SG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, tri_enum_kernel<M, kTW>, kTW * 32, smem));
    per_sm = std::max(per_sm, 1);
    if (grid_per_sm > 0) per_sm = std::min(per_sm, grid_per_sm);
    const int64_t grid = (int64_t)c->num_sms * per_sm;
    {
        SG_LAUNCH(c, "tri_enum");
        tri_enum_kernel<M, kTW><<<(unsigned)grid, kTW * 32, smem, c->stream>>>(a);
    }
    SG_CUDA(cudaGetLastError());
    return SG_OK;
}

template <Mode M>
static sg_status launch_enum(Ctx *c, const TriArgs &base, const Plan &pl) {
    if (base.n == 0) return SG_OK;
    TriArgs a = base;
    a.heavy = pl.heavy;
    a.n_heavy = pl.n_heavy;
    a.heavy_log_slots = pl.log_slots;
    a.heavy_cap = pl.heavy_cap;
    a.light_max = pl.light_max;
    a.light_items = pl.light_items;
    a.offs = pl.offs;
    a.din = pl.din;
    a.inl = pl.inl;
    a.work = c->d_ctr + kCtrAux;
    if (pl.n_hubs > 0) {
        // the hubs first, one 32-warp CTA per SM sharing a large table
        TriArgs h = a;
        h.n_heavy = pl.n_hubs;
        h.heavy_cap = pl.hub_cap;
        SG_CUDA(cudaMemsetAsync(h.work, 0, 2 * sizeof(unsigned long long), c->stream));
        SG_CUDA(cudaFuncSetAttribute(tri_enum_kernel<M, kHubTW>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)pl.hub_smem));
        int hub_per_sm = 0;
        SG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&hub_per_sm, tri_enum_kernel<M, kHubTW>, kHubTW * 32,
                                                              pl.hub_smem));
        const int64_t hgrid = (int64_t)c->num_sms * std::max(hub_per_sm, 1);
        {
            SG_LAUNCH(c, "tri_hubs");
            tri_enum_kernel<M, kHubTW><<<(unsigned)hgrid, kHubTW * 32, pl.hub_smem, c->stream>>>(h);
        }
        SG_CUDA(cudaGetLastError());
        a.heavy = pl.heavy + pl.n_hubs;
        a.n_heavy = pl.n_heavy - pl.n_hubs;
    }
    SG_CUDA(cudaMemsetAsync(a.work, 0, 2 * sizeof(unsigned long long), c->stream));
    SG_CUDA(cudaFuncSetAttribute(tri_enum_kernel<M, kTW>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pl.smem));
    int per_sm = 0;
    SG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, tri_enum_kernel<M, kTW>, kTW * 32, pl.smem));
    const int64_t grid = (int64_t)c->num_sms * std::max(per_sm, 1);
    {
        SG_LAUNCH(c, "tri_enum");
        tri_enum_kernel<M, kTW><<<(unsigned)grid, kTW * 32, pl.smem, c->stream>>>(a);
    }
    SG_CUDA(cudaGetLastError());
    return SG_OK;
}

static TriArgs base_args(Ctx *c, const Oriented &o) {
    TriArgs a{};
    a.offp = o.off;
    a.colp = o.col;
    a.wp = o.w;
    a.n = o.n;
    a.ctr = c->d_ctr;
    a.err = c->d_err;
    return a;
}

// Edge-once rounds.  Round r lets the live selected triangles with
// r2 < theta_r = 2^(27+r) bid (all of them from round 5 on).  A bidder that
// holds all three reservations is the smallest live triangle on each of its
// edges (every non-bidder has a larger key), so the accepted set equals the
// unrestricted greedy scan's, while most triangles die before they ever bid.
//
// The first round enumerates the triangles once and lists every live selected
// one (16 bytes each, within a quarter of free memory), split into buckets by
// the round in which it first bids.  Each later round works on lists alone:
// the survivors of the last round plus this round's bucket are filtered
// (triangles that lost an edge are dropped), bid and are compacted into the
// next active list, so a listed triangle is read once before it bids.  The
// listing pass also bids for its round's prefix, so if the list does not fit,
// the round still completes from those bids, accepting from the edges' side;
// later rounds enumerate and bid directly and retry the list once the live
// triangles fit.
static sg_status eo_rounds(Ctx *c, const Graph *g, const Oriented &o, sg_kernel k, const Plan &pl, TriArgs a) {
    const size_t m = (size_t)std::max<int64_t>(o.m, 1);
    const int choice = k == SG_TR_EO_MAXW ? kChoiceMaxw : (k == SG_TR_EO_MINCOUNT ? kChoiceMinCount : kChoiceRandom);
    uint32_t *considered = nullptr;
    const size_t cwords = (m + 31) / 32;
    // lctr: [kEoBuckets] bucket fills, [kEoBuckets] bucket counts, an out length, then the overflow bits
    unsigned long long *resv = nullptr, *lctr = nullptr;
    const size_t lctr_bytes = (2 * kEoBuckets + 1) * sizeof(unsigned long long) + sizeof(int);
    int *lovf = nullptr;
    uint4 *L = nullptr;    // bucketed list written by the enumeration (workspace kWsList)
    TriRec *A = nullptr;   // active list: this round's bidders (workspace a_slot)
    int a_slot = kWsActive1;
    int64_t lenA = 0;
    int64_t ubase[kEoBuckets] = {}, used[kEoBuckets] = {};
    // live selected triangles per bucket at the last listing pass: a bound on them now
    unsigned long long dem[kEoBuckets] = {};
    bool have_dem = false;
    int next_bucket = kEoBuckets;  // next bucket to merge into the active list
    int top = kEoBuckets;          // the list holds every live triangle of the buckets below this one
    int sched = 0;                 // step of the prefix schedule: bids come from r2 below the top of bucket sched
    bool listed = false;
    bool try_list = o.m <= (int64_t)0xFFFFFFFFll && c->eo_list_cap >= 0;
    // warps of one enumeration launch, at most: each may leave a chunk per bucket part filled
    const int64_t emit_warps = (int64_t)c->num_sms * (8 * kTW + kHubTW);
    sg_status st = dalloc(c, (void **)&considered, cwords * sizeof(uint32_t));
    if (st == SG_OK) st = dalloc(c, (void **)&resv, m * sizeof(unsigned long long));
    if (st == SG_OK) st = dalloc(c, (void **)&lctr, lctr_bytes);
    if (st == SG_OK) {
        lovf = reinterpret_cast<int *>(lctr + 2 * kEoBuckets + 1);
        if (cudaMemsetAsync(considered, 0, cwords * sizeof(uint32_t), c->stream) != cudaSuccess)
            st = cuda_fail(cudaGetLastError(), "memset");
    }
    a.considered = considered;
    a.resv = resv;
    const int64_t acc_blocks = std::min<int64_t>((o.n + 7) / 8, (int64_t)c->num_sms * 8);
    if (st == SG_OK && cudaMemsetAsync(resv, 0xFF, m * sizeof(unsigned long long), c->stream) != cudaSuccess)
        st = cuda_fail(cudaGetLastError(), "memset");
    auto list_blocks = [&](int64_t len) { return std::min<int64_t>((len + 255) / 256, (int64_t)c->num_sms * 8); };
    cudaMemPool_t pool = nullptr;
    if (cudaDeviceGetMemPool(&pool, c->device) != cudaSuccess) {
        (void)cudaGetLastError();
        pool = nullptr;
    }
    auto list_capacity = [&]() -> int64_t {
        size_t fr = 0, tot = 0;
        if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) fr = 0;
        // memory the stream-ordered pool keeps from earlier calls but does not use is free too
        uint64_t reserved = 0, used = 0;  // the pool attributes are 64-bit counts
        if (pool && cudaMemPoolGetAttribute(pool, cudaMemPoolAttrReservedMemCurrent, &reserved) == cudaSuccess &&
            cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemCurrent, &used) == cudaSuccess && reserved > used)
            fr += (size_t)(reserved - used);
        (void)cudaGetLastError();
        for (int i = 0; i < 3; ++i) fr += c->ws_bytes[i];  // the context's workspaces are reused
        int64_t cap = (int64_t)(fr / 4 / sizeof(uint4));
        if (c->eo_list_cap > 0) cap = std::min<int64_t>(cap, c->eo_list_cap);
        return cap;
    };
    for (int round = 0; st == SG_OK; ++round, ++sched) {
        if (round > 100000) { st = fail(SG_ERR_TIMEOUT, "edge-once rounds did not converge"); break; }
        const int rb = std::min(sched, kEoBuckets - 1);
        unsigned long long theta = 1ull << (27 + rb);
        if (listed && top < kEoBuckets) theta = std::min(theta, 1ull << (26 + top));  // the list's window
        a.eo_theta = theta;
        unsigned long long live = 0;
        if (!listed) {
            bool bids_done = false;
            int hi = 0;  // buckets [rb, hi) get room in the list
            if (try_list) {
                // ---- one enumeration bids for this round and lists the live selected
                // triangles of as many buckets, from rb on, as the room allows
                const int64_t cap = list_capacity();
                hi = kEoBuckets;
                int64_t run = 0;
                for (int b = 0; b < kEoBuckets; ++b) a.list_base[b] = a.list_cap[b] = 0;
                auto give = [&](int b, int64_t cb) {
                    a.list_base[b] = (unsigned long long)run;
                    a.list_cap[b] = (unsigned long long)cb;
                    ubase[b] = run;
                    run += cb;
                };
                // the shares of the draws r2 over the buckets: 1,1,2,4,8,16 of 32
                // (earlier buckets fold into rb)
                double w[kEoBuckets], wsum = 0.0;
                for (int b = 0; b < kEoBuckets; ++b) w[b] = b <= 1 ? 1.0 : (double)(1 << (b - 1));
                for (int b = 0; b < rb; ++b) { w[rb] += w[b]; w[b] = 0.0; }
                for (int b = 0; b < kEoBuckets; ++b) wsum += w[b];
                // no counts yet: a triangle is found by one probe, so at most
                // about p W are selected (W probes per pass)
                const double sel_max = (double)a.tp / 4294967296.0 * (double)pl.work;
                if (!have_dem && sel_max <= (double)cap) {
                    // everything fits: split the room by the shares
                    for (int b = rb; b < kEoBuckets; ++b) {
                        const int64_t cb = (int64_t)((double)cap * w[b] / wsum);
                        if (cb < 4 * eo_chunk(b)) { hi = b; break; }
                        give(b, cb);
                    }
                } else {
                    // Each bucket wants its bound: the last pass's count (live
                    // triangles only die) or, before the first pass, a quarter of p W
                    // (R-MAT graphs find a triangle in 12-18% of their probes), plus
                    // room for sealed chunk tails.  The bounds are loose -- deciding a
                    // window kills most of the triangles above it -- so when they do
                    // not all fit, this round's bucket gets its bound (up to half the
                    // room) and the rest is split in proportion to the bounds above:
                    // a bucket that overflows only narrows the window.
                    unsigned long long fold = 0;
                    for (int b = 0; b <= rb; ++b) fold += dem[b];
                    int64_t want[kEoBuckets] = {};
                    double above = 0.0;
                    for (int b = rb; b < kEoBuckets; ++b) {
                        const double d = have_dem ? (double)(b == rb ? fold : dem[b]) : 0.25 * sel_max * w[b] / wsum;
                        want[b] = (int64_t)(d * (1.0 + 16.0 / eo_chunk(b))) + emit_warps * eo_chunk(b);
                        if (b > rb) above += (double)want[b];
                    }
                    const int64_t first = std::min<int64_t>(want[rb], cap / 2);
                    const double rest = (double)(cap - first);
                    const double scale = above <= rest ? 1.0 : rest / above;
                    for (int b = rb; b < kEoBuckets; ++b) {
                        const int64_t cb = b == rb ? first : (int64_t)((double)want[b] * scale);
                        if (cb < 4 * eo_chunk(b)) { hi = b; break; }
                        give(b, cb);
                    }
                }
                if (hi <= rb) hi = 0;  // nothing to list: the pass only bids and counts
                if (hi > 0) {
                    const size_t lbytes = (size_t)std::max<int64_t>(run, 1) * sizeof(uint4);
                    if (ws_get(c, kWsList, lbytes, (void **)&L) != SG_OK && pool) {
                        // the pool's idle memory may be too fragmented: hand it back and retry
                        (void)cudaStreamSynchronize(c->stream);
                        (void)cudaMemPoolTrimTo(pool, 0);
                        (void)cudaGetLastError();
                        if (ws_get(c, kWsList, lbytes, (void **)&L) != SG_OK) L = nullptr;
                    }
                    if (L == nullptr) {
                        set_error("");
                        try_list = false;
                    }
                }
            }
            if (try_list) {
                a.list = L;
                a.list_ctr = lctr;
                a.list_dem = lctr + kEoBuckets;
                a.list_overflow = lovf;
                a.eo_round = rb;
                a.eo_hi = L != nullptr ? hi : 0;
                SG_CUDA(cudaMemsetAsync(lctr, 0, lctr_bytes, c->stream));
                SG_CUDA(cudaMemsetAsync(c->d_ctr + kCtrLive, 0, sizeof(unsigned long long), c->stream));
                // nothing is considered before the first acceptance: skip the flag reads
                a.considered = round == 0 ? nullptr : considered;
                st = launch_enum<Mode::EoEmit>(c, a, pl);
                ++c->eo_passes;
                a.considered = considered;
                a.list = nullptr;
                if (st != SG_OK) break;
                unsigned long long fill[2 * kEoBuckets + 1];
                int ovf = 0;
                SG_CUDA(cudaMemcpyAsync(c->h_pinned, lctr, 2 * kEoBuckets * sizeof(unsigned long long),
                                        cudaMemcpyDeviceToHost, c->stream));
                SG_CUDA(cudaMemcpyAsync(c->h_pinned + 2 * kEoBuckets, c->d_ctr + kCtrLive, sizeof(unsigned long long),
                                        cudaMemcpyDeviceToHost, c->stream));
                SG_CUDA(cudaMemcpyAsync(c->h_pinned + 2 * kEoBuckets + 1, lovf, sizeof(int), cudaMemcpyDeviceToHost,
                                        c->stream));
                SG_CUDA(cudaStreamSynchronize(c->stream));
                std::memcpy(fill, c->h_pinned, sizeof(fill));
                std::memcpy(&ovf, c->h_pinned + 2 * kEoBuckets + 1, sizeof(int));
                live = fill[2 * kEoBuckets];
                for (int b = 0; b < kEoBuckets; ++b) dem[b] = fill[kEoBuckets + b];
                have_dem = true;
                if (live == 0) break;  // no live selected triangle is left
                // the buckets below the first one that ran out of room are complete
                const int wtop = a.eo_hi > 0 ? std::min(a.eo_hi, ovf ? __builtin_ctz((unsigned)ovf) : kEoBuckets) : 0;
                if (wtop > rb) {
                    listed = true;
                    top = wtop;
                    for (int b = 0; b < kEoBuckets; ++b) used[b] = b >= rb && b < top ? (int64_t)fill[b] : 0;
                    for (int b = rb; b < top; ++b) c->eo_listed += dem[b];
                    ++c->eo_list_passes;
                    next_bucket = rb;
                } else {
                    // this round's bids are in: finish it from the edges' side
                    L = nullptr;
                    bids_done = true;
                }
            }
            if (!listed) {
                // ---- enumeration round that bids directly; acceptance from the edges' side
                if (!bids_done) {
                    SG_CUDA(cudaMemsetAsync(c->d_ctr + kCtrLive, 0, sizeof(unsigned long long), c->stream));
                    a.considered = round == 0 ? nullptr : considered;
                    st = launch_enum<Mode::EoReserve>(c, a, pl);
                    ++c->eo_passes;
                    a.considered = considered;
                    if (st != SG_OK) break;
                    st = read_ctr(c, kCtrLive, 1, &live);
                    if (st != SG_OK || live == 0) break;
                }
                ++c->eo_rounds;
                SG_LAUNCH(c, "tri_eo_accept");
                if (choice == kChoiceMaxw)
                    eo_accept_kernel<kChoiceMaxw><<<(unsigned)acc_blocks, 256, 0, c->stream>>>(a, g->off, considered);
                else if (choice == kChoiceMinCount)
                    eo_accept_kernel<kChoiceMinCount><<<(unsigned)acc_blocks, 256, 0, c->stream>>>(a, g->off,
                                                                                                  considered);
                else
                    eo_accept_kernel<kChoiceRandom><<<(unsigned)acc_blocks, 256, 0, c->stream>>>(a, g->off, considered);
                SG_CUDA(cudaGetLastError());
                SG_CUDA(cudaMemsetAsync(resv, 0xFF, m * sizeof(unsigned long long), c->stream));
                continue;
            }
        }
        // ---- list round: last round's survivors plus this round's bucket
        const int64_t fresh = next_bucket < top ? used[next_bucket] : 0;
        TriRec *B = nullptr;
        const int bslot = a_slot == kWsActive0 ? kWsActive1 : kWsActive0;
        st = ws_get(c, bslot, (size_t)std::max<int64_t>(lenA + fresh, 1) * sizeof(TriRec), (void **)&B);
        if (st != SG_OK) break;
        unsigned long long *out_len = lctr + 2 * kEoBuckets;
        SG_CUDA(cudaMemsetAsync(out_len, 0, sizeof(unsigned long long), c->stream));
        if (lenA > 0) {
            SG_LAUNCH(c, "tri_eo_list_reserve");
            eo_list_reserve_kernel<<<(unsigned)list_blocks(lenA), 256, 0, c->stream>>>(A, lenA, B, out_len, resv,
                                                                                     considered, theta);
        }
        if (fresh > 0) {
            SG_LAUNCH(c, "tri_eo_fresh_reserve");
            eo_fresh_reserve_kernel<<<(unsigned)list_blocks((fresh + kFreshPer - 1) / kFreshPer), 256, 0,
                                      c->stream>>>(
                L + ubase[next_bucket], fresh, B, out_len, resv, considered, theta, a.colp, a.k0, a.k1);
        }
        if (next_bucket < top) ++next_bucket;
        SG_CUDA(cudaGetLastError());
        SG_CUDA(cudaMemcpyAsync(c->h_pinned, out_len, sizeof(unsigned long long), cudaMemcpyDeviceToHost, c->stream));
        SG_CUDA(cudaStreamSynchronize(c->stream));
        std::memcpy(&live, c->h_pinned, sizeof(live));
        A = B;
        a_slot = bslot;
        lenA = (int64_t)live;
        if (live == 0) {
            if (next_bucket < top) continue;  // nothing bid this round
            if (top >= kEoBuckets) break;     // no triangle left anywhere
            // every triangle of the list's window is decided: list the live ones
            // above it, starting the schedule at its first bucket
            for (int b = 0; b < top; ++b) dem[b] = 0;
            L = nullptr;
            listed = false;
            sched = top - 1;
            continue;
        }
        ++c->eo_rounds;
        // ---- accept: triangles holding all three reservations.  Judging from
        // the edge side costs a pass over m reservations plus a binary search
        // per reserved arc; once the list holds at most two triangles per
        // edge, read the list instead
        if ((double)lenA <= 2.0 * (double)m) {
            SG_LAUNCH(c, "tri_eo_list_accept");
            const unsigned blocks = (unsigned)list_blocks(lenA);
            if (choice == kChoiceMaxw)
                eo_list_accept_kernel<kChoiceMaxw><<<blocks, 256, 0, c->stream>>>(A, lenA, resv, considered, a.del,
                                                                                  a.wp, a.tcnt);
            else if (choice == kChoiceMinCount)
                eo_list_accept_kernel<kChoiceMinCount><<<blocks, 256, 0, c->stream>>>(A, lenA, resv, considered,
                                                                                      a.del, a.wp, a.tcnt);
            else
                eo_list_accept_kernel<kChoiceRandom><<<blocks, 256, 0, c->stream>>>(A, lenA, resv, considered, a.del,
                                                                                    a.wp, a.tcnt);
        } else {
            SG_LAUNCH(c, "tri_eo_accept");
            if (choice == kChoiceMaxw)
                eo_accept_kernel<kChoiceMaxw><<<(unsigned)acc_blocks, 256, 0, c->stream>>>(a, g->off, considered);
            else if (choice == kChoiceMinCount)
                eo_accept_kernel<kChoiceMinCount><<<(unsigned)acc_blocks, 256, 0, c->stream>>>(a, g->off, considered);
            else
                eo_accept_kernel<kChoiceRandom><<<(unsigned)acc_blocks, 256, 0, c->stream>>>(a, g->off, considered);
        }
        SG_CUDA(cudaGetLastError());
        // ---- reset the reservations for the next round: three scattered
        // writes per listed triangle beat clearing all m words only for short lists
        if ((double)lenA * 96.0 <= 8.0 * (double)m) {
            SG_LAUNCH(c, "tri_eo_list_reset");
            eo_list_reset_kernel<<<(unsigned)list_blocks(lenA), 256, 0, c->stream>>>(A, lenA, resv);
        } else {
            SG_CUDA(cudaMemsetAsync(resv, 0xFF, m * sizeof(unsigned long long), c->stream));
        }
        SG_CUDA(cudaGetLastError());
    }

    dfree(c, lctr);
    dfree(c, considered);
    dfree(c, resv);
    return st;
}

sg_status tr_mark(Ctx *c, const Graph *g, const Oriented &o, sg_kernel k, double p, uint64_t seed, uint8_t *del) {
    Plan pl;
    sg_status st = make_plan(c, o, g->off, &pl);
    TriArgs a = base_args(c, o);
    a.k0 = (uint32_t)(seed & 0xFFFFFFFFu);
    a.k1 = (uint32_t)(seed >> 32);
    a.tp = prob_threshold(p);
    a.del = del;
    uint32_t *tcnt = nullptr;
    if (st == SG_OK && (k == SG_TR_MINCOUNT || k == SG_TR_EO_MINCOUNT)) {
        // the min-count choice needs the triangle count of every edge of G first
        const size_t bytes = sizeof(uint32_t) * (size_t)std::max<int64_t>(o.m, 1);
        st = dalloc(c, (void **)&tcnt, bytes);
        if (st == SG_OK && cudaMemsetAsync(tcnt, 0, bytes, c->stream) != cudaSuccess)
            st = cuda_fail(cudaGetLastError(), "cudaMemsetAsync(tcnt)");
        a.tcnt = tcnt;
        if (st == SG_OK) st = launch_enum<Mode::EdgeCount>(c, a, pl);
    }
    if (st == SG_OK) {
        switch (k) {
        case SG_TR_RANDOM: st = launch_enum<Mode::UnionRandom>(c, a, pl); break;
        case SG_TR_MAXW: st = launch_enum<Mode::UnionMaxw>(c, a, pl); break;
        case SG_TR_P2: st = launch_enum<Mode::UnionP2>(c, a, pl); break;
        case SG_TR_MINCOUNT: st = launch_enum<Mode::UnionMinCount>(c, a, pl); break;
        default: st = eo_rounds(c, g, o, k, pl, a); break;
        }
    }
    dfree(c, tcnt);
    free_plan(c, &pl);
    return st;
}

sg_status tr_count(Ctx *c, const Graph *g, const Oriented &o, int64_t *count, int64_t *probes, int64_t *maxdeg,
                   int64_t *in_arcs, int64_t *fwd_probes) {
    Plan pl;
    unsigned long long v0[kCtrCount] = {}, v1[kCtrCount] = {};
    sg_status st = read_ctr(c, 0, kCtrCount, v0);
    if (st == SG_OK) st = make_plan(c, o, g->off, &pl);
    if (st == SG_OK) st = launch_enum<Mode::Count>(c, base_args(c, o), pl);
    if (st == SG_OK) st = read_ctr(c, 0, kCtrCount, v1);
    if (count) *count = (int64_t)(v1[kCtrTriangles] - v0[kCtrTriangles]);
    if (probes) *probes = (int64_t)(v1[kCtrProbes] - v0[kCtrProbes]);
    if (maxdeg) *maxdeg = pl.max_deg;
    // summed afresh by this orientation's reverse list
    if (in_arcs) *in_arcs = (int64_t)v1[kCtrInArcs];
    if (fwd_probes) *fwd_probes = (int64_t)v1[kCtrWorkFwd];
    free_plan(c, &pl);
    return st;
}

// Triangles through every vertex (device uint64[n], overwritten).
sg_status tr_vertex_counts(Ctx *c, const Graph *g, const Oriented &o, unsigned long long *vcnt) {
    Plan pl;
    sg_status st = make_plan(c, o, g->off, &pl);
    if (st == SG_OK && cudaMemsetAsync(vcnt, 0, sizeof(unsigned long long) * (size_t)std::max<int64_t>(o.n, 1),
                                       c->stream) != cudaSuccess)
        st = cuda_fail(cudaGetLastError(), "cudaMemsetAsync(vcnt)");
    TriArgs a = base_args(c, o);
    a.vcnt = vcnt;
    if (st == SG_OK) st = launch_enum<Mode::VertexCount>(c, a, pl);
    free_plan(c, &pl);
    return st;
}

// ---------------------------------------------------------- batched union
sg_status batch_tr_prepare(Ctx *c, const Graph *u, const Oriented &o, BatchTri *bt) {
    Plan pl;
    pl.light_max = bt->light_max;
    pl.light_items = 4 * bt->light_max;
    sg_status st = make_plan(c, o, u->off, &pl);
    if (st == SG_OK) {
        bt->log_slots = pl.log_slots;
        bt->smem = pl.smem;
        bt->max_deg = pl.heavy_cap;
    }
    free_plan(c, &pl);
    if (st != SG_OK) return st;
    if (!bt->heavy) st = dalloc(c, (void **)&bt->heavy, sizeof(uint32_t) * (size_t)std::max<int64_t>(o.n, 1));
    if (st == SG_OK && !bt->buckets)
        st = dalloc(c, (void **)&bt->buckets, sizeof(unsigned long long) * (2 * kKeys + 1));
    if (st == SG_OK && !bt->din) st = dalloc(c, (void **)&bt->din, sizeof(uint32_t) * (size_t)std::max<int64_t>(o.n, 1));
    // Per call only the graphs with a triangle kernel are oriented, so E+ can
    // hold fewer than nnz/2 arcs and the in-list room off(v) - off+(v) then
    // reaches up to nnz: size the records for that.
    if (st == SG_OK && !bt->inl)
        st = dalloc(c, (void **)&bt->inl, sizeof(uint2) * (size_t)std::max<int64_t>(u->nnz, 1));
    return st;
}

void batch_tr_free(Ctx *c, BatchTri *bt) {
    dfree(c, bt->heavy);
    dfree(c, bt->buckets);
    dfree(c, bt->din);
    dfree(c, bt->inl);
    bt->heavy = nullptr;
    bt->buckets = nullptr;
    bt->din = nullptr;
    bt->inl = nullptr;
}

// No host synchronisation: the heavy-vertex count stays on the device.
sg_status batch_tr_mark(Ctx *c, const Graph *u, const Oriented &o, const BatchDev &b, const BatchTri &bt,
                        uint8_t *del) {
    if (o.n == 0) return SG_OK;
    const int light_items = 4 * bt.light_max;
    SG_CUDA(cudaMemsetAsync(bt.buckets, 0, sizeof(unsigned long long) * (2 * kKeys + 1), c->stream));
    sg_status st = SG_OK;  // the reverse list bt.inl was filled after the batch orientation
    if (st != SG_OK) return st;
    const int64_t blocks = std::max<int64_t>(1, std::min<int64_t>((o.n + 255) / 256, (int64_t)c->num_sms * 8));
    {
        SG_LAUNCH(c, "tri_classify");
        // no hub launch in a batch: its graphs are small, and a long N+(u) is chunked
        classify_count_kernel<<<(unsigned)blocks, 256, 0, c->stream>>>(o.off, u->off, bt.din, o.n, bt.light_max,
                                                                       light_items, INT64_MAX, bt.buckets, c->d_ctr);
    }
    {
        SG_LAUNCH(c, "tri_classify");
        classify_scatter_kernel<<<(unsigned)blocks, 256, 0, c->stream>>>(o.off, bt.din, o.n, bt.light_max,
                                                                         light_items, INT64_MAX, bt.buckets,
                                                                         bt.buckets + kKeys, bt.heavy,
                                                                         bt.buckets + 2 * kKeys);
    }
    SG_CUDA(cudaGetLastError());
    TriArgs a = base_args(c, o);
    a.del = del;
    a.heavy = bt.heavy;
    a.n_heavy = 0;
    a.n_heavy_dev = bt.buckets + 2 * kKeys;
    a.heavy_log_slots = bt.log_slots;
    a.heavy_cap = bt.max_deg;
    a.light_max = bt.light_max;
    a.light_items = light_items;
    a.offs = u->off;
    a.din = bt.din;
    a.inl = bt.inl;
    a.work = c->d_ctr + kCtrAux;
    a.bparams = b.params;
    a.vgid = b.vgid;
    return launch_enum_raw<Mode::BatchUnion>(c, a, bt.smem, bt.grid_per_sm);
}

}  // namespace sg
