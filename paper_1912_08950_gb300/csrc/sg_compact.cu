// Arc compaction of a symmetric CSR in two passes over 256-arc chunks.
//
// For every arc (x, y) a policy decides whether it stays; the kept column ids
// (and weights) move to their final positions and the new row offsets are
// off'[v] = number of kept arcs before off[v].  Rows stay sorted because arcs
// keep their order.  The same engine serves
//   * the edge kernels of Listing 1 (random_uniform, spectral_sparsify),
//   * the degree-ordered orientation E+ that triangle listing needs (Sec. 4.3:
//     O(m^{3/2}) listing), and
//   * the final mask resolution of the Triangle p-1-Reduction kernels, which
//     replaces the paper's "atomic SG.del(e)" by per-edge flags read here.
//
// Layout: a chunk is kWarpSpan = 32 * CI consecutive arcs handled by one warp
// as CI slabs of 32, one arc per lane, so every read of col[] is a 128-byte
// coalesced access and a ballot gives a slab's keep mask.  The passes are
//   decide  -- every warp decides its chunks on its own and writes their keep
//              masks and kept counts (no barrier, no wait on other warps);
//   scan    -- the exclusive prefix of the chunk counts, a single-pass scan
//              with decoupled look-back (Merrill & Garland, "Single-pass
//              parallel prefix scan with decoupled look-back", NVIDIA TR
//              2016; written here without CUB) over tiles of chunks;
//   scatter -- every warp moves the kept arcs of its chunks to the chunk's
//              prefix plus their rank in the keep masks;
//   offsets -- one thread per row: the chunk prefix of its first arc plus
//              the kept arcs before it in that chunk's masks.
// Only the short scan has waits between CTAs, and those are bounded: a wait
// that runs out reports a device error instead of hanging.
#include <climits>
#include <mutex>
#include <string>

#include "sg_internal.cuh"

namespace sg {

constexpr unsigned long long kStAgg = 1ull << 62;
constexpr unsigned long long kStInc = 2ull << 62;
constexpr unsigned long long kStVal = (1ull << 62) - 1;

uint64_t prob_threshold(double p) {
    const double t = std::floor(p * 4294967296.0);
    if (t >= 4294967296.0) return 4294967296ull;
    if (t <= 0.0) return 0;
    return (uint64_t)t;
}

static uint64_t scaled_threshold(double y) {
    const double t = std::floor(y * 4294967296.0);
    if (t >= 18446744073709551615.0) return UINT64_MAX;
    if (t <= 0.0) return 0;
    return (uint64_t)t;
}

// --------------------------------------------------------------- row maps
// chunk_row[c] = the row holding arc c * kWarpSpan.  One thread per row, no
// searches: row v owns the chunk starts that fall in its range.
__global__ void row_maps_kernel(const int64_t *__restrict__ off, int64_t n, uint32_t *__restrict__ chunk_row,
                                int64_t num_chunks) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
        const int64_t b = off[v], e = off[v + 1];
        for (int64_t c = b <= 0 ? 0 : (b + kWarpSpan - 1) / kWarpSpan; c < num_chunks && c * kWarpSpan < e; ++c)
            chunk_row[c] = (uint32_t)v;
    }
}

// Every entry of the row map gets a row in range before row_maps_kernel
// writes the ones a well-formed CSR defines: with malformed offsets (not
// non-decreasing) some entries are never written by row_maps_kernel, and the
// pre-filled 0 still keeps every compaction access inside the row range.
__global__ void prefill_row_maps_kernel(uint32_t *chunk_row, int64_t num_chunks) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < num_chunks; i += stride) chunk_row[i] = 0;
}

static void launch_row_maps(cudaStream_t stream, int num_sms, const int64_t *off, int64_t n, uint32_t *chunk_row,
                            int64_t num_chunks) {
    const int64_t pb = std::max<int64_t>(1, std::min<int64_t>((num_chunks + 255) / 256, (int64_t)num_sms * 16));
    prefill_row_maps_kernel<<<(unsigned)pb, 256, 0, stream>>>(chunk_row, num_chunks);
    const int64_t rb = std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, (int64_t)num_sms * 16));
    row_maps_kernel<<<(unsigned)rb, 256, 0, stream>>>(off, n, chunk_row, num_chunks);
}

sg_status fill_row_maps(Ctx *c, const Graph *g, const RowMaps &rm) {
    {
        SG_LAUNCH(c, "row_maps");
        launch_row_maps(c->stream, c->num_sms, g->off, g->n, rm.chunk_row, rm.num_chunks);
    }
    SG_CUDA(cudaGetLastError());
    return SG_OK;
}

sg_status build_row_maps(Ctx *c, const Graph *g, RowMaps *rm) {
    rm->num_chunks = (g->nnz + kWarpSpan - 1) / kWarpSpan;
    sg_status st = dalloc(c, (void **)&rm->chunk_row, sizeof(uint32_t) * (size_t)(rm->num_chunks + 1));
    if (st != SG_OK) return st;
    return fill_row_maps(c, g, *rm);
}

void free_row_maps(Ctx *c, RowMaps *rm) {
    dfree(c, rm->chunk_row);
    rm->chunk_row = nullptr;
}

// ------------------------------------------------------------ device parts
struct SlabCtx {
    uint32_t or_word;  // forward-arc bits of this slab (mask resolution only)
    int64_t or_base;   // E+ index of the slab's first forward arc
};

// Rows of the arcs of K consecutive 32-arc slabs starting at wbase, one arc
// per lane (arcs at or past t1 take the row of arc t1 - 1), clamped to
// [0, n - 1].  r0 is a row with off[r0] <= wbase (the row holding wbase, from
// the row map).  Lane j holds the start of row rb + 1 + j, relative to wbase,
// for one batch of 32 rows.  A slab with no row start inside it (the common
// case: most arcs lie in long rows) takes its one row from two ballots; the
// others search the batch by shuffles.  A new batch is loaded only when a slab
// runs past the batch's last start, so the slabs do not wait on one another.
template <int K>
__device__ __forceinline__ void warp_rows(const int64_t *__restrict__ off, int64_t n, int64_t r0, int64_t wbase,
                                          int64_t t1, uint32_t (&rows)[K]) {
    const int lane = threadIdx.x & 31;
    auto rel_start = [&](int64_t rb) {  // start of row rb + 1 + lane - wbase, clamped to [-1, K * 32 + 1]
        const int64_t v = rb + 1 + lane;
        const int64_t st = (v <= n) ? __ldg(off + v) - wbase : (int64_t)(K * 32 + 1);
        return st < 0 ? -1 : (st > K * 32 + 1 ? K * 32 + 1 : (int)st);
    };
    int64_t rb = r0;
    int brel = rel_start(rb);
    uint32_t prev = (uint32_t)min(r0, n - 1);
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const int64_t sbase = wbase + k * 32;
        rows[k] = prev;
        if (sbase >= t1) continue;  // warp-uniform
        const int lo = k * 32;
        const int q = sbase + lane < t1 ? lane : (int)(t1 - 1 - sbase);
        int64_t row = -1;
        for (;;) {
            const uint32_t before = __ballot_sync(kFull, brel <= lo);
            const uint32_t inside = __ballot_sync(kFull, brel > lo && brel <= lo + 31);
            if (inside == 0 && before != kFull) {  // one row for the whole slab
                if (row < 0) row = rb + __popc(before);
                break;
            }
            const int r = brel - lo < -1 ? -1 : (brel - lo > 32 ? 32 : brel - lo);
            int cnt = 0;  // batch starts at or before sbase + q
#pragma unroll
            for (int s = 16; s >= 1; s >>= 1) {
                const int v = __shfl_sync(kFull, r, cnt + s - 1);
                if (v <= q) cnt += s;
            }
            const int r31 = __shfl_sync(kFull, r, 31);
            if (cnt == 31 && r31 <= q) cnt = 32;
            if (row < 0 && cnt < 32) row = rb + cnt;
            if (!__any_sync(kFull, row < 0)) break;
            rb += 32;
            brel = rel_start(rb);
        }
        prev = (uint32_t)min(row, n - 1);
        rows[k] = prev;
    }
}

// Decoupled look-back by one warp: publish this tile's aggregate, sum the
// predecessors' values back to the first inclusive prefix, publish our own
// inclusive prefix, return the exclusive one.  Polls are bounded by `limit`.
// hold_first (a test hook) keeps tile 0 from publishing, so that the wait of
// the tile after it runs out and the error path can be exercised.
__device__ int64_t tile_lookback(unsigned long long *status, int64_t tile, int64_t agg, int *err,
                                 uint32_t limit = kSpinLimit, bool hold_first = false) {
    const int lane = threadIdx.x & 31;
    if (tile == 0) {
        if (lane == 0 && !hold_first) st_volatile_u64(status, kStInc | (unsigned long long)agg);
        return 0;
    }
    if (lane == 0) st_volatile_u64(status + tile, kStAgg | (unsigned long long)agg);
    int64_t excl = 0;
    int64_t idx = tile - 1;
    uint32_t spins = 0;
    for (;;) {
        const int64_t j = idx - lane;
        const unsigned long long s = (j >= 0) ? ld_volatile_u64(status + j) : kStInc;
        const unsigned flag = (unsigned)(s >> 62);
        if (__any_sync(kFull, flag == 0)) {
            ++spins;
            // give up after `limit` polls, or at once if another tile already
            // gave up; publish a (meaningless) inclusive value so that no
            // successor waits on this tile either
            bool quit = spins > limit;
            if ((spins & 1023u) == 0) quit = quit || (*(volatile int *)err != 0);
            if (__any_sync(kFull, quit)) {
                if (lane == 0) {
                    atomicExch(err, (int)kDevLookbackTimeout);
                    st_volatile_u64(status + tile, kStInc | (unsigned long long)agg);
                }
                return excl;
            }
            __nanosleep(64);
            continue;
        }
        const unsigned inc = __ballot_sync(kFull, flag == 2);
        const int first = inc ? __ffs(inc) - 1 : 32;
        const int64_t v = (lane <= first) ? (int64_t)(s & kStVal) : 0;
        excl += warp_sum(v);
        if (inc) break;
        idx -= 32;
    }
    if (lane == 0) st_volatile_u64(status + tile, kStInc | (unsigned long long)(excl + agg));
    return excl;
}

// ---------------------------------------------------------------- policies
// A policy decides an arc in three steps, so that the loads of all CI slabs of
// a warp are in flight together: load() issues the loads that need only the
// arc (x, y) at position p, load2() those that depend on them, keep() decides.
//   kNeedRow / kNeedCol: the decision reads x / y;
//   kOrPrefix: it reads the orientation's forward bits and their prefix;
//   kMapCol: the scatter stores map_col(y) instead of y;
//   kReweight: the scatter may replace a kept arc's weight (weight(x, y, w)),
//              when reweights() says so;
//   kMinBlocks: CTAs of 256 threads per SM the decide pass is compiled for.
struct UniformPol {
    static constexpr bool kNeedRow = true, kNeedCol = true, kOrPrefix = false, kMapCol = false, kReweight = false;
    static constexpr int kMinBlocks = 4;
    struct Pre {};
    uint32_t k0, k1;
    unsigned long long tp;
    __device__ __forceinline__ Pre load(uint32_t, uint32_t, int64_t, const SlabCtx &) const { return Pre{}; }
    __device__ __forceinline__ void load2(Pre &) const {}
    // random_uniform(E e): the edge stays iff its draw is below floor(p 2^32)
    __device__ __forceinline__ bool keep(const Pre &, uint32_t x, uint32_t y, int64_t) const {
        const uint4 r = philox4x32_10(make_uint4(min(x, y), max(x, y), 0u, kTagEdge), k0, k1);
        return (unsigned long long)r.x < tp;
    }
};

// Degrees saturated to 16 bits: 2 bytes per vertex instead of the 16-byte
// offset pair, so the random degree reads of the orientation and of spectral
// sparsification mostly hit L2
// (R-MAT s26: 134 MB against 1.07 GB of offsets).
__global__ void deg16_kernel(const int64_t *__restrict__ off, int64_t n, uint16_t *__restrict__ deg16) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
        const int64_t d = __ldg(off + v + 1) - __ldg(off + v);
        deg16[v] = (uint16_t)(d < 65535 ? d : 65535);
    }
}

// 1/p_uv for an edge kept with probability p_uv = min(1, Y / dmin)
__device__ __forceinline__ float spectral_weight(uint64_t dmin, unsigned long long ty, float yf) {
    return (dmin * 4294967296ull <= ty) ? 1.0f : __fdiv_rn(__ull2float_rn(dmin), yf);
}

struct SpectralPol {
    static constexpr bool kNeedRow = true, kNeedCol = true, kOrPrefix = false, kMapCol = false, kReweight = true;
    static constexpr int kMinBlocks = 4;
    struct Pre {
        uint64_t dmin;
    };
    const int64_t *off;
    const uint16_t *deg16;  // min(d, 65535)
    uint32_t k0, k1;
    unsigned long long ty;  // floor(Y 2^32)
    float yf;               // Y rounded to float
    bool reweight;
    // min(d_x, d_y): the smaller saturated degree is exact unless both saturate
    __device__ __forceinline__ uint64_t dmin(uint32_t x, uint32_t y) const {
        const uint32_t sm = min((uint32_t)__ldg(deg16 + x), (uint32_t)__ldg(deg16 + y));
        if (sm < 65535u) return sm;
        const uint64_t dx = (uint64_t)(__ldg(off + x + 1) - __ldg(off + x));
        const uint64_t dy = (uint64_t)(__ldg(off + y + 1) - __ldg(off + y));
        return dx < dy ? dx : dy;
    }
    __device__ __forceinline__ Pre load(uint32_t x, uint32_t y, int64_t, const SlabCtx &) const {
        return Pre{dmin(x, y)};
    }
    __device__ __forceinline__ void load2(Pre &) const {}
    // spectral_sparsify(E e): stays with probability min(1, Y / min(d_u, d_v)),
    // i.e. iff r * min(d_u, d_v) < Y 2^32
    __device__ __forceinline__ bool keep(const Pre &pr, uint32_t x, uint32_t y, int64_t) const {
        const uint4 r = philox4x32_10(make_uint4(min(x, y), max(x, y), 0u, kTagEdge), k0, k1);
        return (unsigned long long)r.x * pr.dmin < ty;
    }
    __device__ __forceinline__ bool reweights() const { return reweight; }
    // kept edges may take the weight 1/p_uv
    __device__ __forceinline__ float weight(uint32_t x, uint32_t y, float) const {
        return spectral_weight(dmin(x, y), ty, yf);
    }
};

struct OrientPol {
    static constexpr bool kNeedRow = true, kNeedCol = true, kOrPrefix = false, kMapCol = false, kReweight = false;
    static constexpr int kMinBlocks = 4;
    struct Pre {
        uint32_t sxy;  // saturated degrees of x (high half) and y (low half)
    };
    const int64_t *off;
    const uint16_t *deg16;  // min(d, 65535)
    __device__ __forceinline__ Pre load(uint32_t x, uint32_t y, int64_t, const SlabCtx &) const {
        return Pre{((uint32_t)__ldg(deg16 + x) << 16) | (uint32_t)__ldg(deg16 + y)};
    }
    __device__ __forceinline__ void load2(Pre &) const {}
    // x precedes y in the degree order (d_x, x) < (d_y, y).  Unequal saturated
    // degrees order the vertices as their degrees do; equal ones below 65535
    // are the degrees themselves; only two saturated ones need the offsets.
    __device__ __forceinline__ bool keep(const Pre &pr, uint32_t x, uint32_t y, int64_t) const {
        const uint32_t sx = pr.sxy >> 16, sy = pr.sxy & 0xFFFFu;
        if (sx != sy) return sx < sy;
        if (sx < 65535u) return x < y;
        const int64_t dx = __ldg(off + x + 1) - __ldg(off + x);
        const int64_t dy = __ldg(off + y + 1) - __ldg(off + y);
        return dx < dy || (dx == dy && x < y);
    }
};

struct MaskPol {
    static constexpr bool kNeedRow = false, kNeedCol = false, kOrPrefix = true, kMapCol = false, kReweight = false;
    static constexpr int kMinBlocks = 4;
    struct Pre {
        uint32_t idx;  // E+ index of the arc's edge, then its deletion flag
    };
    const uint32_t *fwd_bits;
    const int64_t *fwd_excl;  // forward arcs before every chunk
    const uint2 *inl;         // the reverse list (reverse_list)
    const uint32_t *delbits;  // the deletion flags, one bit per E+ arc (pack_flags_kernel)
    int64_t ninl;             // entries of inl (>= 1)
    int64_t ndel;             // E+ arcs (>= 1)
    // A forward arc's E+ index is the running prefix of forward arcs; a reverse
    // arc's rank p - (forward arcs before p) finds it in the reverse list.  The
    // indices are clamped to the arrays: an arc whose answer is not used (past
    // the end, or of a batch graph without a triangle kernel, whose reverse
    // list entries are never written) still reads inside them.
    __device__ __forceinline__ Pre load(uint32_t, uint32_t, int64_t p, const SlabCtx &s) const {
        const int lane = (int)(p & 31);
        const int64_t fwd_before = s.or_base + __popc(s.or_word & ((1u << lane) - 1u));
        int64_t idx = fwd_before;
        if (!((s.or_word >> lane) & 1u)) {
            const int64_t r = min(max(p - fwd_before, (int64_t)0), ninl - 1);
            idx = __ldg(&inl[r].y);
        }
        return Pre{(uint32_t)min(idx, ndel - 1)};
    }
    __device__ __forceinline__ void load2(Pre &pr) const {
        pr.idx = (__ldg(delbits + (pr.idx >> 5)) >> (pr.idx & 31)) & 1u;
    }
    // the arc stays iff its edge's oriented arc carries no deletion flag
    __device__ __forceinline__ bool keep(const Pre &pr, uint32_t, uint32_t, int64_t) const { return pr.idx == 0; }
};

// The deletion flags packed to one bit per E+ arc before the CSR rebuild:
// m/8 bytes (R-MAT s26: 131 MB, about the size of L2), so that the random
// flag reads of the reverse arcs mostly hit L2 instead of each fetching a
// 32-byte sector of the byte flags from DRAM.  One thread per output word.
__global__ void pack_flags_kernel(const uint8_t *__restrict__ del, int64_t m, uint32_t *__restrict__ bits) {
    const int64_t words = (m + 31) / 32;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const bool vec = (reinterpret_cast<uintptr_t>(del) & 15u) == 0;
    for (int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w < words; w += stride) {
        const int64_t b0 = w * 32;
        uint32_t v = 0;
        if (vec && b0 + 32 <= m) {  // 32 flags from two 16-byte loads
            const uint4 *p = reinterpret_cast<const uint4 *>(del + b0);
            const uint4 a = __ldg(p), b = __ldg(p + 1);
            const uint32_t x[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                // bit 7 of every nonzero byte, moved to bits 24..27 in byte order
                const uint32_t nz = (__vcmpne4(x[i], 0u) >> 7) & 0x01010101u;
                v |= ((nz * 0x01020408u) >> 24) << (4 * i);
            }
        } else {
            for (int64_t i = b0; i < m; ++i) v |= (del[i] != 0 ? 1u : 0u) << (i - b0);
        }
        bits[w] = v;
    }
}

static void launch_pack_flags(cudaStream_t stream, int num_sms, const uint8_t *del, int64_t m, uint32_t *bits) {
    const int64_t words = (m + 31) / 32;
    const int64_t blocks = std::max<int64_t>(1, std::min<int64_t>((words + 255) / 256, (int64_t)num_sms * 16));
    pack_flags_kernel<<<(unsigned)blocks, 256, 0, stream>>>(del, m, bits);
}

// ---------------------------------------------------------------- engine
struct EngineArgs {
    const int64_t *off;
    const uint32_t *col;
    const float *w;
    int64_t n, nnz, num_chunks;
    const uint32_t *chunk_row;
    uint32_t *keep;    // CI keep words per chunk
    int64_t *cexcl;    // kept arcs per chunk, then their exclusive prefix; [num_chunks] = total
    uint32_t *col_out;
    float *w_out;
};

// decide: keep masks and kept counts of every chunk, one warp per chunk
template <class Pol>
__global__ void __launch_bounds__(256, Pol::kMinBlocks) decide_kernel(EngineArgs a, Pol pol) {
    const int lane = threadIdx.x & 31;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t c = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; c < a.num_chunks; c += nw) {
        const int64_t wbase = c * kWarpSpan;
        const int64_t t1 = min(wbase + (int64_t)kWarpSpan, a.nnz);
        // independent loads first: the slabs' columns, forward bits and prefix
        uint32_t ys[CI];
        if constexpr (Pol::kNeedCol) {
            if (t1 - wbase == kWarpSpan) {  // a full chunk: no clamping
                const uint32_t *cp = a.col + wbase + lane;
#pragma unroll
                for (int k = 0; k < CI; ++k) ys[k] = __ldg(cp + k * 32);
            } else {
#pragma unroll
                for (int k = 0; k < CI; ++k) ys[k] = __ldg(a.col + min(wbase + k * 32 + lane, t1 - 1));
            }
        } else {
#pragma unroll
            for (int k = 0; k < CI; ++k) ys[k] = 0u;
        }
        uint32_t words = 0;  // lane k < CI: forward bits of slab k
        int64_t run = 0;
        if constexpr (Pol::kOrPrefix) {
            if (lane < CI) words = __ldg(pol.fwd_bits + c * CI + lane);
            run = __ldg(pol.fwd_excl + c);
        }
        uint32_t xs[CI];
        if constexpr (Pol::kNeedRow) {
            warp_rows<CI>(a.off, a.n, (int64_t)__ldg(a.chunk_row + c), wbase, t1, xs);
        } else {
#pragma unroll
            for (int k = 0; k < CI; ++k) xs[k] = 0;
        }
        typename Pol::Pre pre[CI];
#pragma unroll
        for (int k = 0; k < CI; ++k) {
            SlabCtx sc{0u, 0};
            if constexpr (Pol::kOrPrefix) {
                sc.or_word = __shfl_sync(kFull, words, k);
                sc.or_base = run;
                run += __popc(sc.or_word);
            }
            pre[k] = pol.load(xs[k], ys[k], wbase + k * 32 + lane, sc);
        }
#pragma unroll
        for (int k = 0; k < CI; ++k) pol.load2(pre[k]);
        uint32_t mine = 0;
        int cnt = 0;
#pragma unroll
        for (int k = 0; k < CI; ++k) {
            const int64_t p = wbase + k * 32 + lane;
            const bool keep = p < t1 && pol.keep(pre[k], xs[k], ys[k], p);
            const uint32_t m = __ballot_sync(kFull, keep);
            if (lane == k) mine = m;
            cnt += __popc(m);
        }
        if (lane < CI) a.keep[c * CI + lane] = mine;
        if (lane == 0) a.cexcl[c] = cnt;
    }
}

// scan: v[0, nv) -> exclusive prefix in place, v[nv] = total.  Tiles of
// kScanTile values claimed through a ticket (status[num_tiles]), so a CTA
// only waits on tiles owned by running CTAs.
constexpr int kScanPer = 4;
constexpr int kScanTile = 256 * kScanPer;

int64_t compact_scan_words(int64_t num_chunks) { return (num_chunks + kScanTile - 1) / kScanTile + 1; }

__global__ void __launch_bounds__(256) chunk_scan_kernel(int64_t *v, int64_t nv, int64_t num_tiles,
                                                         unsigned long long *status, int *err, uint32_t spin_limit,
                                                         int hold_first) {
    __shared__ long long s_warp[8];
    __shared__ long long s_tile, s_excl;
    unsigned int *ticket = reinterpret_cast<unsigned int *>(status + num_tiles);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (;;) {
        if (threadIdx.x == 0) s_tile = (long long)atomicAdd(ticket, 1u);
        __syncthreads();
        const int64_t tile = s_tile;
        if (tile >= num_tiles) break;
        const int64_t b0 = tile * kScanTile + (int64_t)threadIdx.x * kScanPer;
        int64_t x[kScanPer];
        int64_t sum = 0;
#pragma unroll
        for (int i = 0; i < kScanPer; ++i) {
            x[i] = b0 + i < nv ? v[b0 + i] : 0;
            sum += x[i];
        }
        int64_t inc = sum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int64_t t = __shfl_up_sync(kFull, inc, o);
            if (lane >= o) inc += t;
        }
        if (lane == 31) s_warp[warp] = inc;
        __syncthreads();
        if (warp == 0) {
            const int64_t wv = lane < 8 ? s_warp[lane] : 0;
            int64_t winc = wv;
#pragma unroll
            for (int o = 1; o < 8; o <<= 1) {
                const int64_t t = __shfl_up_sync(kFull, winc, o);
                if (lane >= o) winc += t;
            }
            const int64_t agg = __shfl_sync(kFull, winc, 7);
            if (lane < 8) s_warp[lane] = winc - wv;
            const int64_t excl = tile_lookback(status, tile, agg, err, spin_limit, hold_first != 0);
            if (lane == 0) {
                s_excl = excl;
                if (tile == num_tiles - 1) v[nv] = excl + agg;
            }
        }
        __syncthreads();
        int64_t run = s_excl + s_warp[warp] + (inc - sum);
#pragma unroll
        for (int i = 0; i < kScanPer; ++i) {
            if (b0 + i < nv) v[b0 + i] = run;
            run += x[i];
        }
        __syncthreads();
    }
}

// scatter: the kept arcs of every chunk to the chunk's prefix plus their rank
template <class Pol, bool kW>
__global__ void __launch_bounds__(256, 4) scatter_kernel(EngineArgs a, Pol pol) {
    const int lane = threadIdx.x & 31;
    const uint32_t lt = lanemask_lt();
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t c = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; c < a.num_chunks; c += nw) {
        const int64_t wbase = c * kWarpSpan;
        const int64_t t1 = min(wbase + (int64_t)kWarpSpan, a.nnz);
        const uint32_t word = lane < CI ? __ldg(a.keep + c * CI + lane) : 0u;
        const int64_t base = __ldg(a.cexcl + c);
        uint32_t ys[CI];
        float ws[CI];
        if (t1 - wbase == kWarpSpan) {  // a full chunk: no clamping
            const uint32_t *cp = a.col + wbase + lane;
#pragma unroll
            for (int k = 0; k < CI; ++k) ys[k] = __ldg(cp + k * 32);
        } else {
#pragma unroll
            for (int k = 0; k < CI; ++k) ys[k] = __ldg(a.col + min(wbase + k * 32 + lane, t1 - 1));
        }
        if constexpr (kW) {
#pragma unroll
            for (int k = 0; k < CI; ++k) ws[k] = a.w ? __ldg(a.w + min(wbase + k * 32 + lane, t1 - 1)) : 0.f;
        }
        if constexpr (kW && Pol::kReweight) {
            if (pol.reweights()) {
                uint32_t xs[CI];
                warp_rows<CI>(a.off, a.n, (int64_t)__ldg(a.chunk_row + c), wbase, t1, xs);
#pragma unroll
                for (int k = 0; k < CI; ++k) ws[k] = pol.weight(xs[k], ys[k], ws[k]);
            }
        }
        // kept arcs of the chunk's slabs before slab k (lanes 0..CI-1)
        int inc = __popc(word);
#pragma unroll
        for (int o = 1; o < CI; o <<= 1) {
            const int t = __shfl_up_sync(kFull, inc, o);
            if (lane >= o) inc += t;
        }
        const int excl = inc - __popc(word);
#pragma unroll
        for (int k = 0; k < CI; ++k) {
            const uint32_t wk = __shfl_sync(kFull, word, k);
            const int ek = __shfl_sync(kFull, excl, k);
            if ((wk >> lane) & 1u) {
                const int64_t g = base + ek + __popc(wk & lt);
                if constexpr (Pol::kMapCol) a.col_out[g] = pol.map_col(ys[k]);
                else a.col_out[g] = ys[k];
                if constexpr (kW) a.w_out[g] = ws[k];
            }
        }
    }
}

// offsets: off'[v] = kept arcs before off[v], for every v in [0, n]
__global__ void offsets_kernel(const int64_t *__restrict__ off, int64_t n, int64_t nnz, int64_t num_chunks,
                               const uint32_t *__restrict__ keep, const int64_t *__restrict__ cexcl,
                               int64_t *__restrict__ off_out) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v <= n; v += stride) {
        const int64_t o = __ldg(off + v);
        int64_t r;
        if (o >= nnz) {
            r = __ldg(cexcl + num_chunks);
        } else if (o <= 0) {  // (o < 0 only with malformed offsets)
            r = 0;
        } else {
            const int64_t c = o / kWarpSpan;
            const int j = (int)((o >> 5) & (CI - 1)), l = (int)(o & 31);
            const uint32_t *kw = keep + c * CI;
            r = __ldg(cexcl + c) + __popc(__ldg(kw + j) & ((1u << l) - 1u));
            for (int i = 0; i < j; ++i) r += __popc(__ldg(kw + i));
        }
        off_out[v] = r;
    }
}

// The reverse list.  A reverse arc (x, y) of the symmetric CSR -- y before x
// in the degree order -- is the E+ arc y->x, at the position of x in the
// sorted row N+(y).  One pass finds that position for every reverse arc and
// stores (y, arc index) at the arc's reverse rank p - (forward arcs before p):
// x's in-arcs then lie contiguous at off(x) - off+(x), sorted by tail, for the
// enumeration (which streams N+(y) there when d+(y) < d+(x)), and the CSR
// rebuild reads a reverse arc's deletion flag through the same entry.  The
// pass also sums the enumeration's work model: W (shorter out-list of every
// arc), W+ (head's out-list) and the arcs streamed from the head's side.
//
// Finding x is a chain of dependent loads, so every lane carries kRevK
// searches (one per 32-arc slab of its warp's span) and advances them in
// lockstep: their loads are independent and overlap.  Each search is a lower
// bound (x lies in [base, base + len]) that narrows its window until it holds
// at most kRevWin candidates, which are then loaded together and compared.
// Vertex ids carry no order of their own, so a row's ids are spread over
// [0, n): the first kRevInterp probes interpolate x's position from its value
// and bisection takes over after them (a skewed row still costs O(log)
// probes).  On rows of uniformly spread ids of length 500 / 3000 that reads
// about 1.9 / 2.4 distinct 32-byte sectors per lookup instead of 6 / 8.5, and
// those random sectors are the pass's bound.
constexpr int kRevK = 2;
static_assert(CI % kRevK == 0, "a warp's slabs lie in one chunk");
constexpr int kRevWin = 4;
constexpr int kRevInterp = 10;

__global__ void __launch_bounds__(256, 5) reverse_list_kernel(
    const int64_t *__restrict__ off, int64_t n, int64_t nnz, const uint32_t *__restrict__ col,
    const uint32_t *__restrict__ chunk_row, const uint32_t *__restrict__ fwd_bits,
    const int64_t *__restrict__ fwd_excl, const int64_t *__restrict__ offp,
    const uint32_t *__restrict__ colp, uint2 *inl, unsigned long long *ctr, int *err, BatchDev batch) {
    const int lane = threadIdx.x & 31;
    const int64_t nslabs = (nnz + 31) >> 5;
    const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    unsigned long long work = 0, fwd = 0, head = 0;
    for (int64_t s0 = wid * kRevK; s0 < nslabs; s0 += nw * kRevK) {
        int64_t base[kRevK], rank[kRevK];
        int len[kRevK];
        uint32_t xs[kRevK], ys[kRevK], vlo[kRevK], vhi[kRevK];
        bool need[kRevK];
        // forward arcs before slab s0: the orientation's prefix up to its chunk
        // plus the forward bits of the chunk's earlier slabs
        const int64_t chunk = s0 / CI;
        int64_t fwd_run = __ldg(fwd_excl + chunk);
        {
            const int64_t wa = chunk * CI + lane;
            fwd_run += warp_sum(wa < s0 ? __popc(__ldg(fwd_bits + wa)) : 0);
        }
        // independent loads first: the slabs' forward bits and columns
        const int64_t sb0 = s0 << 5;
        const int64_t r0 = (int64_t)__ldg(chunk_row + sb0 / kWarpSpan);  // a row at or before arc sb0
        uint32_t fws[kRevK];
#pragma unroll
        for (int k = 0; k < kRevK; ++k) {
            const int64_t sbase = sb0 + k * 32;
            fws[k] = sbase < nnz ? __ldg(fwd_bits + (sbase >> 5)) : 0u;
            ys[k] = sbase < nnz ? __ldg(col + min(sbase + lane, nnz - 1)) : 0u;
        }
        warp_rows<kRevK>(off, n, r0, sb0, nnz, xs);
#pragma unroll
        for (int k = 0; k < kRevK; ++k) {
            const int64_t sbase = sb0 + k * 32;
            const uint32_t fw = fws[k];
            rank[k] = sbase + lane - (fwd_run + __popc(fw & lanemask_lt()));
            fwd_run += __popc(fw);
            // in a batch, graphs without a triangle kernel have no E+ arcs to look up
            const bool tri = batch.params == nullptr ||
                             __ldg(&batch.params[__ldg(batch.vgid + xs[k])].kernel) >= (int)SG_TR_RANDOM;
            need[k] = sbase + lane < nnz && tri && !((fw >> lane) & 1u);
        }
        int64_t dxs[kRevK];
#pragma unroll
        for (int k = 0; k < kRevK; ++k) {
            const uint32_t y = need[k] ? ys[k] : 0u, x = need[k] ? xs[k] : 0u;
            base[k] = __ldg(offp + y);
            len[k] = (int)(__ldg(offp + y + 1) - base[k]);
            dxs[k] = __ldg(offp + x + 1) - __ldg(offp + x);
        }
#pragma unroll
        for (int k = 0; k < kRevK; ++k) {
            vlo[k] = 0;
            vhi[k] = (uint32_t)n;
            if (need[k]) {
                // the work model of arc y->x: d+(y) streamed against d+(x)
                const int64_t dx = dxs[k], dy = len[k];
                work += (unsigned long long)(dx < dy ? dx : dy);
                fwd += (unsigned long long)dx;
                head += dy < dx ? 1ull : 0ull;
            } else {
                len[k] = 0;
            }
        }
        // lockstep narrowing until every window [base, base + len] holds at
        // most kRevWin candidates
        for (int it = 0;; ++it) {
            bool any = false;
            uint32_t v[kRevK];
            int h[kRevK];
#pragma unroll
            for (int k = 0; k < kRevK; ++k) {
                if (it < kRevInterp) {  // interpolate from the value bracket [vlo, vhi]
                    const float f = __fdividef((float)(xs[k] - vlo[k]), (float)(vhi[k] - vlo[k]) + 1.0f);
                    h[k] = min(max((int)(f * (float)len[k]), 0), len[k] - 1);
                } else {
                    h[k] = len[k] >> 1;
                }
                v[k] = len[k] >= kRevWin ? __ldg(colp + base[k] + h[k]) : 0u;
            }
#pragma unroll
            for (int k = 0; k < kRevK; ++k) {
                if (len[k] >= kRevWin) {
                    any = true;
                    if (v[k] < xs[k]) {
                        base[k] += h[k] + 1;
                        len[k] -= h[k] + 1;
                        vlo[k] = v[k] + 1;
                    } else {
                        len[k] = h[k];
                        vhi[k] = v[k];
                    }
                }
            }
            if (!any) break;
        }
        // the windows, loaded together (base + len may be one past the row, but
        // stays inside the E+ column array, which has room for nnz >= m + 1
        // entries; the first match is x's own position)
#pragma unroll
        for (int k = 0; k < kRevK; ++k) {
            uint32_t w[kRevWin];
#pragma unroll
            for (int j = 0; j < kRevWin; ++j) w[j] = (need[k] && j <= len[k]) ? __ldg(colp + base[k] + j) : kFull;
            int64_t idx = -1;
#pragma unroll
            for (int j = kRevWin - 1; j >= 0; --j)
                if (need[k] && j <= len[k] && w[j] == xs[k]) idx = base[k] + j;
            if (need[k]) {
                if (idx < 0) atomicExch(err, (int)kDevBadGraph);  // no reverse arc: not symmetric
                else inl[rank[k]] = make_uint2(ys[k], (uint32_t)idx);
            }
        }
    }
    work = warp_sum(work);
    fwd = warp_sum(fwd);
    head = warp_sum(head);
    if (lane == 0 && work) atomicAdd(ctr + kCtrWork, work);
    if (lane == 0 && fwd) atomicAdd(ctr + kCtrWorkFwd, fwd);
    if (lane == 0 && head) atomicAdd(ctr + kCtrInArcs, head);
}

sg_status reverse_list(Ctx *c, const Graph *g, const RowMaps &rm, const Oriented &o, uint2 *inl, BatchDev batch) {
    // the work model's sums start afresh for this orientation
    SG_CUDA(cudaMemsetAsync(c->d_ctr + kCtrInArcs, 0, 3 * sizeof(unsigned long long), c->stream));
    static_assert(kCtrWork == kCtrInArcs + 1 && kCtrWorkFwd == kCtrInArcs + 2, "work counters are adjacent");
    if (g->nnz == 0) return SG_OK;
    static int per_sm = -1;
    if (per_sm < 0) {
        int b = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, reverse_list_kernel, 256, 0) != cudaSuccess || b < 1)
            b = 1;
        per_sm = b;
    }
    const int64_t warps = ((g->nnz + 31) / 32 + kRevK - 1) / kRevK;
    const int64_t grid = std::max<int64_t>(1, std::min<int64_t>((warps + 7) / 8, (int64_t)c->num_sms * per_sm));
    {
        SG_LAUNCH(c, "tri_reverse_list");
        reverse_list_kernel<<<(unsigned)grid, 256, 0, c->stream>>>(g->off, g->n, g->nnz, g->col, rm.chunk_row,
                                                                 o.fwd_bits, o.fwd_excl, o.off, o.col, inl, c->d_ctr,
                                                                 c->d_err, batch);
    }
    SG_CUDA(cudaGetLastError());
    return SG_OK;
}


// ------------------------------------------------------------------ driver
template <class K>
static int occupancy(K kernel, int threads) {
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kernel, threads, 0) != cudaSuccess || b < 1) {
        (void)cudaGetLastError();
        b = 1;
    }
    return b;
}

template <class Pol>
static int decide_per_sm() {
    static const int v = occupancy(decide_kernel<Pol>, 256);
    return v;
}

template <class Pol, bool kW>
static int scatter_per_sm() {
    static const int v = occupancy(scatter_kernel<Pol, kW>, 256);
    return v;
}

static int scan_per_sm() {
    static const int v = occupancy(chunk_scan_kernel, 256);
    return v;
}

sg_status alloc_compact_scratch(Ctx *c, int64_t num_chunks, bool with_keep, CompactScratch *s) {
    sg_status st = SG_OK;
    if (with_keep) st = dalloc(c, (void **)&s->keep, sizeof(uint32_t) * (size_t)(num_chunks * CI + 1));
    if (st == SG_OK) st = dalloc(c, (void **)&s->cexcl, sizeof(int64_t) * (size_t)(num_chunks + 1));
    if (st == SG_OK)
        st = dalloc(c, (void **)&s->scan, sizeof(unsigned long long) * (size_t)compact_scan_words(num_chunks));
    return st;
}

void free_compact_scratch(Ctx *c, CompactScratch *s) {
    dfree(c, s->keep);
    dfree(c, s->cexcl);
    dfree(c, s->scan);
    *s = CompactScratch{};
}

// The four passes of one compaction on the context stream, all under `name`.
template <class Pol>
static sg_status run_compact(Ctx *c, const Graph *g, const RowMaps &rm, const Pol &pol, const float *w_in,
                             int64_t *off_out, uint32_t *col_out, float *w_out, const CompactScratch &s,
                             const char *name, int grid_per_sm = 0) {
    if (g->nnz == 0) {
        SG_CUDA(cudaMemsetAsync(off_out, 0, sizeof(int64_t) * (size_t)(g->n + 1), c->stream));
        return SG_OK;
    }
    const int64_t nc = rm.num_chunks;
    const int64_t words = compact_scan_words(nc);  // tile status words + the ticket
    SG_CUDA(cudaMemsetAsync(s.scan, 0, sizeof(unsigned long long) * (size_t)words, c->stream));
    EngineArgs a;
    a.off = g->off;
    a.col = g->col;
    a.w = w_in;
    a.n = g->n;
    a.nnz = g->nnz;
    a.num_chunks = nc;
    a.chunk_row = rm.chunk_row;
    a.keep = s.keep;
    a.cexcl = s.cexcl;
    a.col_out = col_out;
    a.w_out = w_out;
    const bool wt = w_out != nullptr;
    auto grid_of = [&](int cap) {
        const int per_sm = grid_per_sm > 0 ? std::min(grid_per_sm, cap) : cap;
        return std::max<int64_t>(1, std::min<int64_t>((nc + 7) / 8, (int64_t)c->num_sms * per_sm));
    };
    {
        SG_LAUNCH(c, name);
        decide_kernel<Pol><<<(unsigned)grid_of(decide_per_sm<Pol>()), 256, 0, c->stream>>>(a, pol);
    }
    {
        SG_LAUNCH(c, name);
        const int64_t tiles = words - 1;
        const int64_t grid = std::min<int64_t>(tiles, (int64_t)c->num_sms * scan_per_sm());
        chunk_scan_kernel<<<(unsigned)grid, 256, 0, c->stream>>>(s.cexcl, nc, tiles, s.scan, c->d_err,
                                                                 c->scan_hold ? c->scan_hold : kSpinLimit,
                                                                 c->scan_hold != 0);
    }
    {
        SG_LAUNCH(c, name);
        if (wt)
            scatter_kernel<Pol, true><<<(unsigned)grid_of(scatter_per_sm<Pol, true>()), 256, 0, c->stream>>>(a, pol);
        else
            scatter_kernel<Pol, false><<<(unsigned)grid_of(scatter_per_sm<Pol, false>()), 256, 0, c->stream>>>(a, pol);
    }
    {
        SG_LAUNCH(c, name);
        const int64_t blocks = std::max<int64_t>(1, std::min<int64_t>((g->n + 256) / 256, (int64_t)c->num_sms * 16));
        offsets_kernel<<<(unsigned)blocks, 256, 0, c->stream>>>(g->off, g->n, g->nnz, nc, s.keep, s.cexcl, off_out);
    }
    SG_CUDA(cudaGetLastError());
    return SG_OK;
}

static sg_status read_i64(Ctx *c, const int64_t *dptr, int64_t *out) {
    SG_CUDA(cudaMemcpyAsync(c->h_pinned, dptr, sizeof(int64_t), cudaMemcpyDeviceToHost, c->stream));
    SG_CUDA(cudaStreamSynchronize(c->stream));
    *out = c->h_pinned[0];
    return SG_OK;
}

static sg_status new_graph(Ctx *c, int64_t n, int64_t nnz_cap, bool weighted, Graph **out) {
    Graph *h = new Graph;
    h->ctx = c;
    h->device = c->device;
    h->n = n;
    h->owned = true;
    sg_status st = dalloc(c, (void **)&h->off, sizeof(int64_t) * (size_t)(n + 1));
    if (st == SG_OK) st = dalloc(c, (void **)&h->col, sizeof(uint32_t) * (size_t)std::max<int64_t>(nnz_cap, 1));
    if (st == SG_OK && weighted) st = dalloc(c, (void **)&h->w, sizeof(float) * (size_t)std::max<int64_t>(nnz_cap, 1));
    if (st != SG_OK) {
        dfree(c, h->off);
        dfree(c, h->col);
        dfree(c, h->w);
        delete h;
        return st;
    }
    *out = h;
    return SG_OK;
}

static void delete_graph(Ctx *c, Graph *h) {
    if (!h) return;
    dfree(c, h->off);
    dfree(c, h->col);
    dfree(c, h->w);
    delete h;
}

sg_status compress_edges(Ctx *c, const Graph *g, sg_kernel k, double p, uint64_t seed, int want_weights,
                         Graph **out) {
    RowMaps rm;
    CompactScratch cs;
    uint16_t *deg16 = nullptr;
    sg_status st = build_row_maps(c, g, &rm);
    Graph *h = nullptr;
    const bool spectral = (k == SG_SPECTRAL_LOGN || k == SG_SPECTRAL_AVGDEG);
    const bool out_w = (spectral && want_weights) || g->w != nullptr;
    if (st == SG_OK) st = alloc_compact_scratch(c, rm.num_chunks, true, &cs);
    if (st == SG_OK) st = new_graph(c, g->n, g->nnz, out_w, &h);
    if (st == SG_OK) {
        const uint32_t k0 = (uint32_t)(seed & 0xFFFFFFFFu), k1 = (uint32_t)(seed >> 32);
        if (k == SG_UNIFORM) {
            UniformPol pol{k0, k1, prob_threshold(p)};
            st = run_compact(c, g, rm, pol, g->w, h->off, h->col, h->w, cs, "compact_uniform");
        } else {
            const int64_t m = g->nnz / 2;
            const double y = (k == SG_SPECTRAL_LOGN) ? p * std::log((double)g->n)
                                                     : (g->n > 0 ? p * (double)m / (double)g->n : 0.0);
            st = dalloc(c, (void **)&deg16, sizeof(uint16_t) * (size_t)std::max<int64_t>(g->n, 1));
            if (st == SG_OK && g->n > 0) {
                const int64_t blocks = std::min<int64_t>((g->n + 255) / 256, (int64_t)c->num_sms * 16);
                SG_LAUNCH(c, "compact_spectral");
                deg16_kernel<<<(unsigned)blocks, 256, 0, c->stream>>>(g->off, g->n, deg16);
            }
            if (st == SG_OK) {
                SpectralPol pol{g->off, deg16, k0, k1, scaled_threshold(y), (float)y, want_weights != 0};
                st = run_compact(c, g, rm, pol, g->w, h->off, h->col, h->w, cs, "compact_spectral");
            }
        }
    }
    if (st == SG_OK) st = read_i64(c, h->off + g->n, &h->nnz);
    if (st == SG_OK) st = check_device_error(c);
    free_compact_scratch(c, &cs);
    dfree(c, deg16);
    free_row_maps(c, &rm);
    if (st != SG_OK) {
        delete_graph(c, h);
        return st;
    }
    *out = h;
    return SG_OK;
}

sg_status orient(Ctx *c, const Graph *g, const RowMaps &rm, bool weights, Oriented *o) {
    o->n = g->n;
    o->m = g->nnz / 2;
    sg_status st = dalloc(c, (void **)&o->off, sizeof(int64_t) * (size_t)(g->n + 1));
    // capacity nnz, not m: an asymmetric input could orient more than m arcs
    if (st == SG_OK) st = dalloc(c, (void **)&o->col, sizeof(uint32_t) * (size_t)std::max<int64_t>(g->nnz, 1));
    if (st == SG_OK && weights) st = dalloc(c, (void **)&o->w, sizeof(float) * (size_t)std::max<int64_t>(g->nnz, 1));
    if (st == SG_OK)
        st = dalloc(c, (void **)&o->fwd_bits, sizeof(uint32_t) * (size_t)(rm.num_chunks * CI + 1));
    if (st == SG_OK) st = dalloc(c, (void **)&o->fwd_excl, sizeof(int64_t) * (size_t)(rm.num_chunks + 1));
    if (st != SG_OK) return st;
    uint16_t *deg16 = nullptr;
    CompactScratch cs;
    cs.keep = o->fwd_bits;  // the keep masks and their prefix are the orientation's
    cs.cexcl = o->fwd_excl;
    st = dalloc(c, (void **)&deg16, sizeof(uint16_t) * (size_t)std::max<int64_t>(g->n, 1));
    if (st == SG_OK)
        st = dalloc(c, (void **)&cs.scan, sizeof(unsigned long long) * (size_t)compact_scan_words(rm.num_chunks));
    if (st == SG_OK && g->n > 0) {
        const int64_t blocks = std::min<int64_t>((g->n + 255) / 256, (int64_t)c->num_sms * 16);
        SG_LAUNCH(c, "compact_orient_deg");
        deg16_kernel<<<(unsigned)blocks, 256, 0, c->stream>>>(g->off, g->n, deg16);
    }
    if (st == SG_OK) {
        OrientPol pol{g->off, deg16};
        st = run_compact(c, g, rm, pol, weights ? g->w : nullptr, o->off, o->col, weights ? o->w : nullptr, cs,
                         "compact_orient");
    }
    dfree(c, deg16);
    dfree(c, cs.scan);
    if (st != SG_OK) return st;
    int64_t mp = 0;
    st = read_i64(c, o->off + g->n, &mp);
    if (st != SG_OK) return st;
    st = check_device_error(c);
    if (st != SG_OK) return st;
    if (mp != o->m)
        return fail(SG_ERR_INVALID_GRAPH, "graph is not symmetric: oriented arcs != nnz/2");
    st = dalloc(c, (void **)&o->inl, sizeof(uint2) * (size_t)std::max<int64_t>(g->nnz - o->m, 1));
    if (st == SG_OK) st = reverse_list(c, g, rm, *o, o->inl);
    return st;
}

void free_oriented(Ctx *c, Oriented *o) {
    dfree(c, o->off);
    dfree(c, o->col);
    dfree(c, o->w);
    dfree(c, o->fwd_bits);
    dfree(c, o->fwd_excl);
    dfree(c, o->inl);
    *o = Oriented{};
}

sg_status resolve_mask(Ctx *c, const Graph *g, const RowMaps &rm, const Oriented &o, const uint8_t *del,
                       Graph **out) {
    Graph *h = nullptr;
    CompactScratch cs;
    uint32_t *delbits = nullptr;
    const int64_t m1 = std::max<int64_t>(o.m, 1);
    sg_status st = new_graph(c, g->n, g->nnz, g->w != nullptr, &h);
    if (st == SG_OK) st = alloc_compact_scratch(c, rm.num_chunks, true, &cs);
    if (st == SG_OK) st = dalloc(c, (void **)&delbits, sizeof(uint32_t) * (size_t)((m1 + 31) / 32));
    if (st == SG_OK && o.m > 0) {
        SG_LAUNCH(c, "compact_trmask");
        launch_pack_flags(c->stream, c->num_sms, del, o.m, delbits);
    }
    if (st == SG_OK) {
        MaskPol pol{o.fwd_bits, o.fwd_excl, o.inl, delbits, std::max<int64_t>(g->nnz - o.m, 1), m1};
        st = run_compact(c, g, rm, pol, g->w, h->off, h->col, h->w, cs, "compact_trmask");
    }
    if (st == SG_OK) st = read_i64(c, h->off + g->n, &h->nnz);
    if (st == SG_OK) st = check_device_error(c);
    free_compact_scratch(c, &cs);
    dfree(c, delbits);
    if (st != SG_OK) {
        delete_graph(c, h);
        return st;
    }
    *out = h;
    return SG_OK;
}

// ------------------------------------------------------- batched variants
// A batch is a disjoint union of graphs; each union vertex knows its graph and
// every graph carries its own kernel, p, seed and vertex base.  Random keys use
// the graph's local ids, so every graph's output equals its solo compression.
struct BatchOrientPol {
    static constexpr bool kNeedRow = true, kNeedCol = true, kOrPrefix = false, kMapCol = false, kReweight = false;
    static constexpr int kMinBlocks = 4;
    struct Pre {
        uint32_t g;      // the graph of x
        uint32_t first;  // x precedes y in the degree order
    };
    const int64_t *off;
    BatchDev b;
    __device__ __forceinline__ Pre load(uint32_t x, uint32_t y, int64_t, const SlabCtx &) const {
        const int64_t dx = __ldg(off + x + 1) - __ldg(off + x), dy = __ldg(off + y + 1) - __ldg(off + y);
        return Pre{__ldg(b.vgid + x), (dx < dy || (dx == dy && x < y)) ? 1u : 0u};
    }
    __device__ __forceinline__ void load2(Pre &) const {}
    // only graphs compressed by a triangle kernel need E+
    __device__ __forceinline__ bool keep(const Pre &pr, uint32_t, uint32_t, int64_t) const {
        const int kern = __ldg(&b.params[pr.g].kernel);
        return kern >= (int)SG_TR_RANDOM && pr.first != 0;
    }
};

struct BatchFinalPol {
    static constexpr bool kNeedRow = true, kNeedCol = true, kOrPrefix = true, kMapCol = true, kReweight = true;
    static constexpr int kMinBlocks = 2;  // 128 registers: its decision holds a Philox per slab
    struct Pre {
        MaskPol::Pre mp;
        uint32_t g;     // the graph of x
        uint32_t dmin;  // min(d_x, d_y) (degrees of a simple graph with n < 2^32 fit)
    };
    const int64_t *off;
    BatchDev b;
    MaskPol mask;
    const uint32_t *fwd_bits;  // = mask.fwd_bits, mask.fwd_excl (read by the decide pass)
    const int64_t *fwd_excl;
    __device__ __forceinline__ uint64_t dmin(uint32_t x, uint32_t y) const {
        const uint64_t dx = (uint64_t)(__ldg(off + x + 1) - __ldg(off + x));
        const uint64_t dy = (uint64_t)(__ldg(off + y + 1) - __ldg(off + y));
        return dx < dy ? dx : dy;
    }
    __device__ __forceinline__ Pre load(uint32_t x, uint32_t y, int64_t p, const SlabCtx &s) const {
        return Pre{mask.load(x, y, p, s), __ldg(b.vgid + x), (uint32_t)min(dmin(x, y), (uint64_t)0xFFFFFFFFu)};
    }
    __device__ __forceinline__ void load2(Pre &pr) const { mask.load2(pr.mp); }
    // a graph's own kernel decides its arcs; a triangle kernel's through the mask
    __device__ __forceinline__ bool keep(const Pre &pr, uint32_t x, uint32_t y, int64_t p) const {
        const BatchParam &P = b.params[pr.g];
        const int kern = P.kernel;
        if (kern >= (int)SG_TR_RANDOM) return mask.keep(pr.mp, x, y, p);
        const uint32_t lx = (uint32_t)(x - P.vbase), ly = (uint32_t)(y - P.vbase);
        const uint4 r = philox4x32_10(make_uint4(min(lx, ly), max(lx, ly), 0u, kTagEdge), P.k0, P.k1);
        if (kern == (int)SG_UNIFORM) return (unsigned long long)r.x < P.tp;
        return (unsigned long long)r.x * (uint64_t)pr.dmin < P.ty;
    }
    // the output is per graph: local column ids (x and y share a graph)
    __device__ __forceinline__ uint32_t map_col(uint32_t y) const {
        return y - (uint32_t)__ldg(&b.params[__ldg(b.vgid + y)].vbase);
    }
    // per graph: spectral graphs that want 1/p_uv weights take them
    __device__ __forceinline__ bool reweights() const { return true; }
    __device__ __forceinline__ float weight(uint32_t x, uint32_t y, float w) const {
        const BatchParam &P = b.params[__ldg(b.vgid + y)];
        const int kern = P.kernel;
        if (kern == (int)SG_UNIFORM || kern >= (int)SG_TR_RANDOM || !P.reweight) return w;
        return spectral_weight(dmin(x, y), P.ty, P.yf);
    }
};

sg_status batch_orient(Ctx *c, const Graph *u, const RowMaps &rm, const BatchDev &b, bool weights, Oriented *o,
                       unsigned long long *scan, int grid_per_sm) {
    BatchOrientPol pol{u->off, b};
    CompactScratch cs;
    cs.keep = o->fwd_bits;
    cs.cexcl = o->fwd_excl;
    cs.scan = scan;
    return run_compact(c, u, rm, pol, weights ? u->w : nullptr, o->off, o->col, weights ? o->w : nullptr, cs,
                       "compact_orient", grid_per_sm);
}

sg_status batch_final(Ctx *c, const Graph *u, const RowMaps &rm, const Oriented &o, const BatchDev &b,
                      const uint8_t *del, uint32_t *delbits, int64_t *off_out, uint32_t *col_out, float *w_in,
                      float *w_out, const CompactScratch &cs, int grid_per_sm) {
    if (o.m > 0) {
        SG_LAUNCH(c, "compact_final");
        launch_pack_flags(c->stream, c->num_sms, del, o.m, delbits);
    }
    // the reverse arcs of graphs without a triangle kernel are not in the
    // reverse list (BatchFinalPol decides those arcs itself); the list has room
    // for every arc of the union, delbits for its m edges
    BatchFinalPol pol{u->off, b,
                      MaskPol{o.fwd_bits, o.fwd_excl, o.inl, delbits, std::max<int64_t>(u->nnz, 1),
                              std::max<int64_t>(o.m, 1)},
                      o.fwd_bits, o.fwd_excl};
    return run_compact(c, u, rm, pol, w_in, off_out, col_out, w_out, cs, "compact_final", grid_per_sm);
}

// ------------------------------------------- low_degree (Listing 1; Sec. 4.4)
// The single-vertex kernel deletes every vertex of input degree 0 or 1 with
// its edges.  Kept vertices get new ids 0..n'-1 in increasing old id: one
// pass over tiles of kVTile vertices with the same decoupled look-back as the
// arc compaction; the arcs are then compacted with LowDegPol and the row
// offsets of the kept rows gathered into the new offset array.
constexpr uint32_t kNoVertex = 0xFFFFFFFFu;
constexpr int kVPer = 8;                 // vertices per thread
constexpr int kVTile = 256 * kVPer;      // vertices per tile

__global__ void __launch_bounds__(256) lowdeg_ids_kernel(const int64_t *__restrict__ off, int64_t n,
                                                         int64_t num_tiles, uint32_t *__restrict__ new_id,
                                                         uint32_t *__restrict__ new_to_old,
                                                         unsigned long long *status, unsigned int *ticket,
                                                         unsigned long long *kept, int *err) {
    __shared__ int s_warp[8];
    __shared__ long long s_tile, s_excl;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (;;) {
        if (threadIdx.x == 0) s_tile = (long long)atomicAdd(ticket, 1u);
        __syncthreads();
        const int64_t tile = s_tile;
        if (tile >= num_tiles) break;
        const int64_t v0 = tile * kVTile + (int64_t)threadIdx.x * kVPer;
        unsigned flags = 0;
        int cnt = 0;
#pragma unroll
        for (int k = 0; k < kVPer; ++k) {
            const int64_t v = v0 + k;
            if (v < n) {
                const int64_t d = __ldg(off + v + 1) - __ldg(off + v);
                if (d >= 2) {
                    flags |= 1u << k;
                    ++cnt;
                }
            }
        }
        // exclusive scan of cnt over the CTA
        int inc = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(kFull, inc, o);
            if (lane >= o) inc += t;
        }
        if (lane == 31) s_warp[warp] = inc;
        __syncthreads();
        if (warp == 0) {
            int wv = lane < 8 ? s_warp[lane] : 0, winc = wv;
#pragma unroll
            for (int o = 1; o < 8; o <<= 1) {
                const int t = __shfl_up_sync(kFull, winc, o);
                if (lane >= o) winc += t;
            }
            const int agg = __shfl_sync(kFull, winc, 7);
            if (lane < 8) s_warp[lane] = winc - wv;
            const int64_t excl = tile_lookback(status, tile, agg, err);
            if (lane == 0) {
                s_excl = excl;
                if (agg) atomicAdd(kept, (unsigned long long)agg);
            }
        }
        __syncthreads();
        uint32_t id = (uint32_t)(s_excl + s_warp[warp] + (inc - cnt));
#pragma unroll
        for (int k = 0; k < kVPer; ++k) {
            const int64_t v = v0 + k;
            if (v < n) {
                if ((flags >> k) & 1u) {
                    new_id[v] = id;
                    if (new_to_old) new_to_old[id] = (uint32_t)v;
                    ++id;
                } else {
                    new_id[v] = kNoVertex;
                }
            }
        }
        __syncthreads();
    }
}

struct LowDegPol {
    static constexpr bool kNeedRow = true, kNeedCol = true, kOrPrefix = false, kMapCol = true, kReweight = false;
    static constexpr int kMinBlocks = 4;
    struct Pre {
        uint32_t nx, ny;  // new ids of x and y
    };
    const uint32_t *new_id;
    __device__ __forceinline__ Pre load(uint32_t x, uint32_t y, int64_t, const SlabCtx &) const {
        return Pre{__ldg(new_id + x), __ldg(new_id + y)};
    }
    __device__ __forceinline__ void load2(Pre &) const {}
    // an arc stays iff both of its ends stay; its head is renumbered
    __device__ __forceinline__ bool keep(const Pre &pr, uint32_t, uint32_t, int64_t) const {
        return pr.nx != kNoVertex && pr.ny != kNoVertex;
    }
    __device__ __forceinline__ uint32_t map_col(uint32_t y) const { return __ldg(new_id + y); }
};

// off'[new_id[v]] = off_c[v] for every kept row v; off'[n'] = off_c[n]
__global__ void lowdeg_offsets_kernel(const int64_t *__restrict__ off_c, const uint32_t *__restrict__ new_id,
                                      int64_t n, int64_t n_kept, int64_t *__restrict__ off_out) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
        const uint32_t id = __ldg(new_id + v);
        if (id != kNoVertex) off_out[id] = __ldg(off_c + v);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) off_out[n_kept] = __ldg(off_c + n);
}

sg_status low_degree(Ctx *c, const Graph *g, uint32_t *new_to_old, Graph **out) {
    RowMaps rm;
    const int64_t vtiles = (g->n + kVTile - 1) / kVTile;
    uint32_t *new_id = nullptr;
    int64_t *off_c = nullptr;
    unsigned long long *vstatus = nullptr;
    CompactScratch cs;
    Graph *h = nullptr;
    int64_t kept = 0;
    sg_status st = build_row_maps(c, g, &rm);
    if (st == SG_OK) st = dalloc(c, (void **)&new_id, sizeof(uint32_t) * (size_t)std::max<int64_t>(g->n, 1));
    if (st == SG_OK) st = dalloc(c, (void **)&off_c, sizeof(int64_t) * (size_t)(g->n + 1));
    if (st == SG_OK) st = alloc_compact_scratch(c, rm.num_chunks, true, &cs);
    // tile status words, the tile ticket and the kept-vertex count, zeroed together
    if (st == SG_OK) st = dalloc(c, (void **)&vstatus, sizeof(unsigned long long) * (size_t)(vtiles + 2));
    if (st == SG_OK && g->n > 0) {
        if (cudaMemsetAsync(vstatus, 0, sizeof(unsigned long long) * (size_t)(vtiles + 2), c->stream) != cudaSuccess)
            st = cuda_fail(cudaGetLastError(), "cudaMemsetAsync");
        if (st == SG_OK) {
            const int64_t grid = std::max<int64_t>(1, std::min<int64_t>(vtiles, (int64_t)c->num_sms * 4));
            SG_LAUNCH(c, "lowdeg_ids");
            lowdeg_ids_kernel<<<(unsigned)grid, 256, 0, c->stream>>>(
                g->off, g->n, vtiles, new_id, new_to_old, vstatus, reinterpret_cast<unsigned int *>(vstatus + vtiles),
                vstatus + vtiles + 1, c->d_err);
            if (cudaGetLastError() != cudaSuccess) st = fail(SG_ERR_CUDA, "lowdeg_ids launch");
        }
        if (st == SG_OK) st = read_i64(c, reinterpret_cast<const int64_t *>(vstatus + vtiles + 1), &kept);
    }
    if (st == SG_OK) st = new_graph(c, kept, g->nnz, g->w != nullptr, &h);
    if (st == SG_OK && g->n > 0) {
        LowDegPol pol{new_id};
        st = run_compact(c, g, rm, pol, g->w, off_c, h->col, h->w, cs, "compact_lowdeg");
        if (st == SG_OK) {
            const int64_t blocks = std::max<int64_t>(1, std::min<int64_t>((g->n + 255) / 256, (int64_t)c->num_sms * 8));
            SG_LAUNCH(c, "lowdeg_offsets");
            lowdeg_offsets_kernel<<<(unsigned)blocks, 256, 0, c->stream>>>(off_c, new_id, g->n, kept, h->off);
            if (cudaGetLastError() != cudaSuccess) st = fail(SG_ERR_CUDA, "lowdeg_offsets launch");
        }
    } else if (st == SG_OK) {
        if (cudaMemsetAsync(h->off, 0, sizeof(int64_t), c->stream) != cudaSuccess)
            st = cuda_fail(cudaGetLastError(), "cudaMemsetAsync");
    }
    if (st == SG_OK) st = read_i64(c, h->off + kept, &h->nnz);
    if (st == SG_OK) st = check_device_error(c);
    dfree(c, new_id);
    dfree(c, off_c);
    free_compact_scratch(c, &cs);
    dfree(c, vstatus);
    free_row_maps(c, &rm);
    if (st != SG_OK) {
        delete_graph(c, h);
        return st;
    }
    *out = h;
    return SG_OK;
}

}  // namespace sg

// ----------------------------------------------------- build information
extern "C" sg_status sg_kernel_arch(int device, int *binary_version) {
    using namespace sg;
    if (!binary_version) return fail(SG_ERR_INVALID_ARG, "binary_version is NULL");
    int ndev = 0, prev = 0;
    SG_CUDA(cudaGetDeviceCount(&ndev));
    if (device < 0 || device >= ndev) return fail(SG_ERR_INVALID_ARG, "no such device");
    SG_CUDA(cudaGetDevice(&prev));
    SG_CUDA(cudaSetDevice(device));
    cudaFuncAttributes attr;
    const cudaError_t e = cudaFuncGetAttributes(&attr, row_maps_kernel);
    (void)cudaSetDevice(prev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaFuncGetAttributes");
    *binary_version = attr.binaryVersion;
    return SG_OK;
}

// ------------------------------------------------ no-allocation entry point
// Uniform edge sampling for callers that must not allocate device memory:
// the scratch (the row map, the keep masks and chunk prefixes, the chunk
// scan's status words and ticket, an error word; about 23 MB) lives in one
// fixed file-scope device array instead of the stream-ordered pool.  Every process that loads this library reserves the array on
// each GPU it touches, for as long as the library stays loaded.
namespace sg {
namespace {

constexpr int64_t kNaMaxArcs = int64_t(1) << 27;
constexpr int64_t kNaMaxChunks = kNaMaxArcs / kWarpSpan;
constexpr int64_t kNaScanWords = (kNaMaxChunks + kScanTile - 1) / kScanTile + 1;
constexpr size_t na_align(size_t x) { return (x + 255) & ~size_t(255); }
constexpr size_t kNaChunkOff = 0;
constexpr size_t kNaKeepOff = na_align(kNaChunkOff + sizeof(uint32_t) * (kNaMaxChunks + 1));
constexpr size_t kNaExclOff = na_align(kNaKeepOff + sizeof(uint32_t) * (kNaMaxChunks * CI + 1));
constexpr size_t kNaScanOff = na_align(kNaExclOff + sizeof(int64_t) * (kNaMaxChunks + 1));
constexpr size_t kNaErrOff = na_align(kNaScanOff + sizeof(unsigned long long) * kNaScanWords);
constexpr size_t kNaBytes = na_align(kNaErrOff + sizeof(int));

__device__ __align__(256) unsigned char g_noalloc_scratch[kNaBytes];

constexpr int kNaMaxDevices = 64;
std::mutex g_na_mutex;
unsigned char *g_na_ptr[kNaMaxDevices] = {};

// Device address of the scratch array on `device` (which must be current).
// Looked up once per device and cached; a cudaDeviceReset of that device
// would leave the cached address stale.
cudaError_t na_scratch(int device, unsigned char **out) {
    std::lock_guard<std::mutex> lock(g_na_mutex);
    if (!g_na_ptr[device]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_na_ptr[device] = static_cast<unsigned char *>(p);
    }
    *out = g_na_ptr[device];
    return cudaSuccess;
}

}  // namespace
}  // namespace sg

namespace sg {
namespace {

sg_status noalloc_uniform(int device, void *cuda_stream, int64_t n, int64_t nnz, const int64_t *off,
                          const uint32_t *col, double p, uint64_t seed, int64_t *off_out, uint32_t *col_out,
                          int64_t *nnz_out) {
    if (!off || !off_out || !nnz_out || (nnz > 0 && (!col || !col_out)))
        return fail(SG_ERR_INVALID_ARG, "NULL argument");
    if (n < 0 || nnz < 0) return fail(SG_ERR_INVALID_ARG, "negative size");
    if (!(p >= 0.0 && p <= 1.0)) return fail(SG_ERR_INVALID_ARG, "p must lie in [0, 1]");
    if (n >= (int64_t)4294967295ll) return fail(SG_ERR_UNSUPPORTED, "n >= 2^32 - 1: ids are uint32");
    if (nnz > kNaMaxArcs)
        return fail(SG_ERR_UNSUPPORTED, "nnz = " + std::to_string(nnz) +
                                            " exceeds the 134217728-arc limit of the fixed scratch array; "
                                            "use sg_compress instead");
    int ndev = 0;
    SG_CUDA(cudaGetDeviceCount(&ndev));
    if (device < 0 || device >= ndev || device >= kNaMaxDevices) return fail(SG_ERR_INVALID_ARG, "no such device");
    SG_CUDA(cudaSetDevice(device));
    cudaStream_t stream = static_cast<cudaStream_t>(cuda_stream);
    *nnz_out = 0;
    // the CSR's ends must match its sizes: the row maps cover [off[0], off[n]]
    int64_t ends[2] = {0, 0};
    SG_CUDA(cudaMemcpyAsync(&ends[0], off, sizeof(int64_t), cudaMemcpyDeviceToHost, stream));
    SG_CUDA(cudaMemcpyAsync(&ends[1], off + n, sizeof(int64_t), cudaMemcpyDeviceToHost, stream));
    SG_CUDA(cudaStreamSynchronize(stream));
    if (ends[0] != 0 || ends[1] != nnz)
        return fail(SG_ERR_INVALID_GRAPH, "off[0] must be 0 and off[n] must equal nnz");
    unsigned char *base = nullptr;
    SG_CUDA(na_scratch(device, &base));
    int *err = reinterpret_cast<int *>(base + kNaErrOff);
    SG_CUDA(cudaMemsetAsync(err, 0, sizeof(int), stream));
    if (nnz == 0) {
        SG_CUDA(cudaMemsetAsync(off_out, 0, sizeof(int64_t) * (size_t)(n + 1), stream));
        SG_CUDA(cudaStreamSynchronize(stream));
        return SG_OK;
    }
    int num_sms = 0;
    SG_CUDA(cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, device));
    const int64_t nc = (nnz + kWarpSpan - 1) / kWarpSpan;
    const int64_t words = compact_scan_words(nc);
    uint32_t *chunk_row = reinterpret_cast<uint32_t *>(base + kNaChunkOff);
    EngineArgs a;
    a.off = off;
    a.col = col;
    a.w = nullptr;
    a.n = n;
    a.nnz = nnz;
    a.num_chunks = nc;
    a.chunk_row = chunk_row;
    a.keep = reinterpret_cast<uint32_t *>(base + kNaKeepOff);
    a.cexcl = reinterpret_cast<int64_t *>(base + kNaExclOff);
    a.col_out = col_out;
    a.w_out = nullptr;
    unsigned long long *scan = reinterpret_cast<unsigned long long *>(base + kNaScanOff);
    // the scan's status words and ticket must start at zero on every call
    SG_CUDA(cudaMemsetAsync(scan, 0, sizeof(unsigned long long) * (size_t)words, stream));
    launch_row_maps(stream, num_sms, off, n, chunk_row, nc);
    SG_CUDA(cudaGetLastError());
    UniformPol pol{(uint32_t)(seed & 0xFFFFFFFFu), (uint32_t)(seed >> 32), prob_threshold(p)};
    const int64_t grid = std::max<int64_t>(1, std::min<int64_t>((nc + 7) / 8, (int64_t)num_sms * decide_per_sm<UniformPol>()));
    decide_kernel<UniformPol><<<(unsigned)grid, 256, 0, stream>>>(a, pol);
    const int64_t sgrid = std::min<int64_t>(words - 1, (int64_t)num_sms * scan_per_sm());
    chunk_scan_kernel<<<(unsigned)sgrid, 256, 0, stream>>>(a.cexcl, nc, words - 1, scan, err, kSpinLimit, 0);
    const int64_t xgrid =
        std::max<int64_t>(1, std::min<int64_t>((nc + 7) / 8, (int64_t)num_sms * scatter_per_sm<UniformPol, false>()));
    scatter_kernel<UniformPol, false><<<(unsigned)xgrid, 256, 0, stream>>>(a, pol);
    const int64_t ob = std::max<int64_t>(1, std::min<int64_t>((n + 256) / 256, (int64_t)num_sms * 16));
    offsets_kernel<<<(unsigned)ob, 256, 0, stream>>>(off, n, nnz, nc, a.keep, a.cexcl, off_out);
    SG_CUDA(cudaGetLastError());
    int64_t count = 0;
    int code = 0;
    SG_CUDA(cudaMemcpyAsync(&count, off_out + n, sizeof(int64_t), cudaMemcpyDeviceToHost, stream));
    SG_CUDA(cudaMemcpyAsync(&code, err, sizeof(int), cudaMemcpyDeviceToHost, stream));
    SG_CUDA(cudaStreamSynchronize(stream));
    if (code != kDevOk) return fail(SG_ERR_TIMEOUT, "a device-side wait of the prefix scan gave up; outputs are invalid");
    *nnz_out = count;
    return SG_OK;
}

}  // namespace
}  // namespace sg

extern "C" sg_status sg_compress_uniform_noalloc(int device, void *cuda_stream, int64_t n, int64_t nnz,
                                                 const int64_t *off, const uint32_t *col, double p, uint64_t seed,
                                                 int64_t *off_out, uint32_t *col_out, int64_t *nnz_out) {
    // the caller's current device is put back whatever happens
    int prev = -1;
    if (cudaGetDevice(&prev) != cudaSuccess) {
        (void)cudaGetLastError();
        prev = -1;
    }
    const sg_status st = sg::noalloc_uniform(device, cuda_stream, n, nnz, off, col, p, seed, off_out, col_out,
                                             nnz_out);
    if (prev >= 0) (void)cudaSetDevice(prev);
    return st;
}

