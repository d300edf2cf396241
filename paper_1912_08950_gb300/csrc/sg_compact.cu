// Arc-tiled stream compaction of a symmetric CSR with a single-pass
// decoupled-lookback prefix scan (Merrill & Garland, "Single-pass parallel
// prefix scan with decoupled look-back", NVIDIA TR 2016), written without CUB.
//
// One pass over the arc array decides, for every arc (x, y), whether it stays,
// scatters the kept column ids (and weights) to their final positions and
// writes the new row offsets: off'[v] = number of kept arcs before off[v].
// Rows stay sorted because arcs keep their order.  The same engine serves
//   * the edge kernels of Listing 1 (random_uniform, spectral_sparsify),
//   * the degree-ordered orientation E+ that triangle listing needs (Sec. 4.3:
//     O(m^{3/2}) listing), and
//   * the final mask resolution of the Triangle p-1-Reduction kernels, which
//     replaces the paper's "atomic SG.del(e)" by per-edge flags read here.
//
// Layout: a tile is kTile consecutive arcs handled by one CTA; warp w owns
// arcs [t0 + w*kWarpSpan, +kWarpSpan) as CI slabs of 32 consecutive arcs, one
// per lane, so every global read of col[] is a 128-byte coalesced access and
// ballots give the slab's keep mask directly.  Tiles are claimed through an
// atomic ticket, so a CTA only ever waits on tiles already owned by running
// CTAs; every wait is bounded and reports a device error instead of hanging.
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
// chunk_row[c] = the row holding arc c*kWarpSpan; tile_vlo[t] = first row v
// with off[v] >= t*kTile (tile_vlo[num_tiles] = n + 1).  One thread per row,
// no searches: row v owns the chunk and tile starts that fall in its range.
__global__ void row_maps_kernel(const int64_t *__restrict__ off, int64_t n, uint32_t *__restrict__ chunk_row,
                                int64_t num_chunks, int64_t *__restrict__ tile_vlo, int64_t num_tiles) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v <= n; v += stride) {
        const int64_t b = off[v];
        const int64_t a = (v == 0) ? -1 : off[v - 1];
        for (int64_t t = (a < 0) ? 0 : a / kTile + 1; t < num_tiles && t * kTile <= b; ++t) tile_vlo[t] = v;
        if (v < n) {
            const int64_t e = off[v + 1];
            for (int64_t c = (b + kWarpSpan - 1) / kWarpSpan; c < num_chunks && c * kWarpSpan < e; ++c)
                chunk_row[c] = (uint32_t)v;
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) tile_vlo[num_tiles] = n + 1;
}

// Every entry of the row maps gets a value in range before row_maps_kernel
// writes the ones a well-formed CSR defines: chunk rows 0, tile rows n + 1.
// With malformed offsets (not non-decreasing) some entries are never written
// by row_maps_kernel; pre-filled, they still keep every compaction access
// inside the row range and the offset array.
__global__ void prefill_row_maps_kernel(uint32_t *chunk_row, int64_t num_chunks, int64_t *tile_vlo,
                                        int64_t num_tiles, int64_t n) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i <= num_tiles || i < num_chunks; i += stride) {
        if (i < num_chunks) chunk_row[i] = 0;
        if (i <= num_tiles) tile_vlo[i] = n + 1;
    }
}

static void prefill_row_maps(cudaStream_t stream, int num_sms, uint32_t *chunk_row, int64_t num_chunks,
                             int64_t *tile_vlo, int64_t num_tiles, int64_t n) {
    const int64_t items = std::max(num_chunks, num_tiles + 1);
    const int64_t blocks = std::max<int64_t>(1, std::min<int64_t>((items + 255) / 256, (int64_t)num_sms * 16));
    prefill_row_maps_kernel<<<(unsigned)blocks, 256, 0, stream>>>(chunk_row, num_chunks, tile_vlo, num_tiles, n);
}

sg_status fill_row_maps(Ctx *c, const Graph *g, const RowMaps &rm) {
    const int threads = 256;
    const int64_t blocks = std::min<int64_t>((g->n + 1 + threads - 1) / threads, (int64_t)c->num_sms * 16);
    {
        SG_LAUNCH(c, "row_maps");
        prefill_row_maps(c->stream, c->num_sms, rm.chunk_row, rm.num_chunks, rm.tile_vlo, rm.num_tiles, g->n);
    }
    {
        SG_LAUNCH(c, "row_maps");
        row_maps_kernel<<<(unsigned)std::max<int64_t>(blocks, 1), threads, 0, c->stream>>>(
            g->off, g->n, rm.chunk_row, rm.num_chunks, rm.tile_vlo, rm.num_tiles);
    }
    SG_CUDA(cudaGetLastError());
    return SG_OK;
}

sg_status build_row_maps(Ctx *c, const Graph *g, RowMaps *rm) {
    rm->num_tiles = (g->nnz + kTile - 1) / kTile;
    rm->num_chunks = (g->nnz + kWarpSpan - 1) / kWarpSpan;
    sg_status st = dalloc(c, (void **)&rm->chunk_row, sizeof(uint32_t) * (size_t)(rm->num_chunks + 1));
    if (st != SG_OK) return st;
    st = dalloc(c, (void **)&rm->tile_vlo, sizeof(int64_t) * (size_t)(rm->num_tiles + 1));
    if (st != SG_OK) return st;
    return fill_row_maps(c, g, *rm);
}

void free_row_maps(Ctx *c, RowMaps *rm) {
    dfree(c, rm->chunk_row);
    dfree(c, rm->tile_vlo);
    rm->chunk_row = nullptr;
    rm->tile_vlo = nullptr;
}

// ------------------------------------------------------------ device parts
struct CompactArgs {
    const int64_t *off;
    const uint32_t *col;
    const float *w;
    int64_t n, nnz, num_tiles;
    const uint32_t *chunk_row;
    const int64_t *tile_vlo;
    int64_t *off_out;
    uint32_t *col_out;
    float *w_out;
    unsigned long long *status;
    unsigned int *ticket;
    int *err;
    uint32_t *keep_bits;  // optional: the keep mask of every 32-arc slab
    uint32_t spin_limit;  // polls of a look-back wait before it gives up
    int hold_first;       // test hook: tile 0 never publishes its prefix
};

struct SlabCtx {
    uint32_t or_word;  // forward-arc bits of this slab (mask resolution only)
    int64_t or_base;   // E+ index of the slab's first forward arc
};

// Rows of the arcs of K consecutive 32-arc slabs starting at wbase, one arc
// per lane (arcs at or past t1 take the row of arc t1 - 1), clamped to
// [0, n - 1].  r0 is a row with off[r0] <= wbase (the row holding wbase, from
// the row maps).  Lane j holds the start off[rb + 1 + j] of one batch of 32
// rows; a slab's rows follow from a search of that batch by shuffles, and a
// new batch is loaded only when a slab runs past the batch's last start, so
// the searches of the K slabs do not wait on one another's loads.
template <int K>
__device__ __forceinline__ void warp_rows(const int64_t *__restrict__ off, int64_t n, int64_t r0, int64_t wbase,
                                          int64_t t1, uint32_t (&rows)[K]) {
    const int lane = threadIdx.x & 31;
    int64_t rb = r0;
    int64_t bst = (rb + 1 + lane <= n) ? __ldg(off + rb + 1 + lane) : LLONG_MAX;
    uint32_t prev = (uint32_t)min(r0, n - 1);
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const int64_t sbase = wbase + k * 32;
        rows[k] = prev;
        if (sbase >= t1) continue;  // warp-uniform
        const int q = sbase + lane < t1 ? lane : (int)(t1 - 1 - sbase);
        int64_t row = -1;
        for (;;) {
            const int64_t rel = bst - sbase;
            const int r = rel < 0 ? -1 : (rel > 32 ? 32 : (int)rel);
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
            bst = (rb + 1 + lane <= n) ? __ldg(off + rb + 1 + lane) : LLONG_MAX;
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

// A policy decides the arcs of a slab in three steps, so that the loads of all
// CI slabs of a warp are in flight together: load() issues the loads that need
// only the arc (x, y) at p, load2() those that depend on them, keep() decides.
// kW: the launch carries weights (read from a.w when present, written to
// a.w_out; a policy may set the weight of a kept arc).
template <class Pol, bool kW>
__global__ void __launch_bounds__(CW * 32, 4) compact_kernel(CompactArgs a, Pol pol) {
    __shared__ uint32_t s_mask[CW][CI];
    __shared__ int s_slab_excl[CW][CI];
    __shared__ int s_warp_cnt[CW];
    __shared__ int s_warp_excl[CW + 1];
    __shared__ long long s_tile_excl;
    __shared__ long long s_tile;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t lt = lanemask_lt();

    for (;;) {
        if (threadIdx.x == 0) s_tile = (long long)atomicAdd(a.ticket, 1u);
        __syncthreads();
        const int64_t tile = s_tile;
        if (tile >= a.num_tiles) break;
        const int64_t t0 = tile * kTile;
        const int64_t t1 = min(t0 + (int64_t)kTile, a.nnz);
        const int64_t wbase = t0 + (int64_t)warp * kWarpSpan;

        // independent loads first: the warp's first row, its slabs' columns
        // (and weights), their forward bits
        const int64_t r0 = (wbase < t1) ? (int64_t)__ldg(a.chunk_row + wbase / kWarpSpan) : 0;
        uint32_t ys[CI];
        float ws[CI];
#pragma unroll
        for (int k = 0; k < CI; ++k) {
            const int64_t sbase = wbase + k * 32;
            const int64_t pe = min(sbase + lane, t1 - 1);
            ys[k] = sbase < t1 ? __ldg(a.col + pe) : 0u;
            if constexpr (kW) ws[k] = (sbase < t1 && a.w) ? __ldg(a.w + pe) : 0.f;
        }
        uint32_t or_words = 0;  // lane k < CI: forward bits of slab k
        int64_t or_run = 0;     // forward arcs before the warp's span
        if constexpr (Pol::kOrPrefix) {
            const int64_t w0 = t0 >> 5, ww = wbase >> 5;
            if (lane < CI && ww + lane < ((t1 + 31) >> 5)) or_words = __ldg(pol.fwd_bits + ww + lane);
            // the tile's earlier warps hold at most (CW - 1) * CI words
            static_assert((CW - 1) * CI <= 64, "two words per lane");
            const int64_t wa = w0 + lane, wb = w0 + 32 + lane;
            const int cnt = (wa < ww ? __popc(__ldg(pol.fwd_bits + wa)) : 0) +
                            (wb < ww ? __popc(__ldg(pol.fwd_bits + wb)) : 0);
            or_run = pol.tile_or_excl(tile) + warp_sum(cnt);
        }

        uint32_t xs[CI];
        warp_rows<CI>(a.off, a.n, r0, wbase, t1, xs);

        typename Pol::Pre pre[CI];
#pragma unroll
        for (int k = 0; k < CI; ++k) {
            SlabCtx sc{0u, 0};
            if constexpr (Pol::kOrPrefix) {
                sc.or_word = __shfl_sync(kFull, or_words, k);
                sc.or_base = or_run;
                or_run += __popc(sc.or_word);
            }
            pre[k] = pol.load(xs[k], ys[k], wbase + k * 32 + lane, sc);
        }
#pragma unroll
        for (int k = 0; k < CI; ++k) pol.load2(pre[k]);

        uint32_t masks[CI];
#pragma unroll
        for (int k = 0; k < CI; ++k) {
            const int64_t sbase = wbase + k * 32;
            masks[k] = 0;
            if (sbase < t1) {  // warp-uniform
                const int64_t p = sbase + lane;
                float wv = 0.f;
                if constexpr (kW) wv = ws[k];
                const bool keep = p < t1 && pol.keep(pre[k], xs[k], ys[k], p, wv);
                if constexpr (kW) ws[k] = wv;
                masks[k] = __ballot_sync(kFull, keep);
                if constexpr (Pol::kMapCol) ys[k] = pol.map_col(pre[k], xs[k], ys[k]);
                if (a.keep_bits != nullptr && lane == 0) a.keep_bits[sbase >> 5] = masks[k];
            }
        }
        if (lane == 0) {
            int run = 0;
#pragma unroll
            for (int k = 0; k < CI; ++k) {
                s_mask[warp][k] = masks[k];
                s_slab_excl[warp][k] = run;
                run += __popc(masks[k]);
            }
            s_warp_cnt[warp] = run;
        }
        __syncthreads();
        if (warp == 0) {
            int agg = 0;
            if (lane == 0) {
                for (int i = 0; i < CW; ++i) {
                    s_warp_excl[i] = agg;
                    agg += s_warp_cnt[i];
                }
                s_warp_excl[CW] = agg;
            }
            agg = __shfl_sync(kFull, agg, 0);
            const int64_t excl = tile_lookback(a.status, tile, agg, a.err, a.spin_limit, a.hold_first != 0);
            if (lane == 0) s_tile_excl = excl;
        }
        __syncthreads();
        const int64_t texcl = s_tile_excl;
        const int64_t wexcl = texcl + s_warp_excl[warp];
#pragma unroll
        for (int k = 0; k < CI; ++k) {
            if ((masks[k] >> lane) & 1u) {
                const int64_t g = wexcl + s_slab_excl[warp][k] + __popc(masks[k] & lt);
                a.col_out[g] = ys[k];
                if constexpr (kW) a.w_out[g] = ws[k];
            }
        }
        // new row offsets for the rows whose start lies in this tile
        // (both in [0, n + 1] whatever the offsets: see prefill_row_maps)
        const int64_t v0 = __ldg(a.tile_vlo + tile), v1 = __ldg(a.tile_vlo + tile + 1);
        const int64_t tlen = t1 - t0;
        for (int64_t v = v0 + threadIdx.x; v < v1; v += blockDim.x) {
            const int64_t q = __ldg(a.off + v) - t0;
            int local;
            if (q >= tlen) {
                local = s_warp_excl[CW];
            } else if (q < 0) {  // only with offsets that are not non-decreasing
                local = 0;
            } else {
                const int wq = (int)(q / kWarpSpan), kq = (int)((q >> 5) % CI), lq = (int)(q & 31);
                local = s_warp_excl[wq] + s_slab_excl[wq][kq] + __popc(s_mask[wq][kq] & ((1u << lq) - 1u));
            }
            a.off_out[v] = texcl + local;
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------- policies
struct UniformPol {
    static constexpr bool kOrPrefix = false;
    static constexpr bool kMapCol = false;
    struct Pre {};
    uint32_t k0, k1;
    unsigned long long tp;
    __device__ __forceinline__ Pre load(uint32_t, uint32_t, int64_t, const SlabCtx &) const { return Pre{}; }
    __device__ __forceinline__ void load2(Pre &) const {}
    // random_uniform(E e): the edge stays iff its draw is below floor(p 2^32)
    __device__ __forceinline__ bool keep(const Pre &, uint32_t x, uint32_t y, int64_t, float &) const {
        const uint4 r = philox4x32_10(make_uint4(min(x, y), max(x, y), 0u, kTagEdge), k0, k1);
        return (unsigned long long)r.x < tp;
    }
};

struct SpectralPol {
    static constexpr bool kOrPrefix = false;
    static constexpr bool kMapCol = false;
    struct Pre {
        uint64_t dmin;
    };
    const int64_t *off;
    uint32_t k0, k1;
    unsigned long long ty;  // floor(Y 2^32)
    float yf;               // Y rounded to float
    bool reweight;
    __device__ __forceinline__ Pre load(uint32_t x, uint32_t y, int64_t, const SlabCtx &) const {
        const uint64_t dx = (uint64_t)(__ldg(off + x + 1) - __ldg(off + x));
        const uint64_t dy = (uint64_t)(__ldg(off + y + 1) - __ldg(off + y));
        return Pre{dx < dy ? dx : dy};
    }
    __device__ __forceinline__ void load2(Pre &) const {}
    // spectral_sparsify(E e): stays with probability min(1, Y / min(d_u, d_v)),
    // i.e. iff r * min(d_u, d_v) < Y 2^32; kept edges may take weight 1/p_uv.
    __device__ __forceinline__ bool keep(const Pre &pr, uint32_t x, uint32_t y, int64_t, float &w) const {
        const uint64_t dmin = pr.dmin;
        const uint4 r = philox4x32_10(make_uint4(min(x, y), max(x, y), 0u, kTagEdge), k0, k1);
        if (reweight) w = (dmin * 4294967296ull <= ty) ? 1.0f : __fdiv_rn(__ull2float_rn(dmin), yf);
        return (unsigned long long)r.x * dmin < ty;
    }
};

// Degrees saturated to 16 bits: 2 bytes per vertex instead of the 16-byte
// offset pair, so the random degree reads of the orientation mostly hit L2
// (R-MAT s26: 134 MB against 1.07 GB of offsets).
__global__ void deg16_kernel(const int64_t *__restrict__ off, int64_t n, uint16_t *__restrict__ deg16) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
        const int64_t d = __ldg(off + v + 1) - __ldg(off + v);
        deg16[v] = (uint16_t)(d < 65535 ? d : 65535);
    }
}

struct OrientPol {
    static constexpr bool kOrPrefix = false;
    static constexpr bool kMapCol = false;
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
    __device__ __forceinline__ bool keep(const Pre &pr, uint32_t x, uint32_t y, int64_t, float &) const {
        const uint32_t sx = pr.sxy >> 16, sy = pr.sxy & 0xFFFFu;
        if (sx != sy) return sx < sy;
        if (sx < 65535u) return x < y;
        const int64_t dx = __ldg(off + x + 1) - __ldg(off + x);
        const int64_t dy = __ldg(off + y + 1) - __ldg(off + y);
        return dx < dy || (dx == dy && x < y);
    }
};

struct MaskPol {
    static constexpr bool kOrPrefix = true;
    static constexpr bool kMapCol = false;
    struct Pre {
        uint32_t idx;  // E+ index of the arc's edge, then its deletion flag
    };
    const uint32_t *fwd_bits;
    const unsigned long long *or_status;
    const uint2 *inl;  // the reverse list (reverse_list)
    const uint8_t *del;
    int64_t ninl;      // entries of inl (>= 1)
    int64_t ndel;      // entries of del (>= 1)
    __device__ __forceinline__ int64_t tile_or_excl(int64_t tile) const {
        return tile == 0 ? 0 : (int64_t)(ld_volatile_u64(or_status + tile - 1) & kStVal);
    }
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
    __device__ __forceinline__ void load2(Pre &pr) const { pr.idx = __ldg(del + pr.idx); }
    // the arc stays iff its edge's oriented arc carries no deletion flag
    __device__ __forceinline__ bool keep(const Pre &pr, uint32_t, uint32_t, int64_t, float &) const {
        return pr.idx == 0;
    }
};

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
constexpr int kRevK = 4;
constexpr int kRevWin = 4;
constexpr int kRevInterp = 6;

__global__ void __launch_bounds__(256, 4) reverse_list_kernel(
    const int64_t *__restrict__ off, int64_t n, int64_t nnz, const uint32_t *__restrict__ col,
    const uint32_t *__restrict__ chunk_row, const uint32_t *__restrict__ fwd_bits,
    const unsigned long long *__restrict__ or_status, const int64_t *__restrict__ offp,
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
        // forward arcs before slab s0: the orientation's prefix up to its tile
        // plus the forward bits of the tile's earlier slabs
        const int64_t tile = (s0 << 5) / kTile;
        const int64_t w0 = (tile * kTile) >> 5;  // the tile's first slab
        int64_t fwd_run = tile == 0 ? 0 : (int64_t)(__ldg(or_status + tile - 1) & kStVal);
        {
            const int64_t wa = w0 + lane, wb = w0 + 32 + lane;
            int cnt = (wa < s0 ? __popc(__ldg(fwd_bits + wa)) : 0) + (wb < s0 ? __popc(__ldg(fwd_bits + wb)) : 0);
            fwd_run += warp_sum(cnt);
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
                                                                 o.fwd_bits, o.status, o.off, o.col, inl, c->d_ctr,
                                                                 c->d_err, batch);
    }
    SG_CUDA(cudaGetLastError());
    return SG_OK;
}


// ------------------------------------------------------------------ driver
template <class Pol, bool kW>
static int blocks_per_sm() {
    static int cached = -1;
    if (cached < 0) {
        int b = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, compact_kernel<Pol, kW>, CW * 32, 0) != cudaSuccess ||
            b < 1)
            b = 1;
        cached = b;
    }
    return cached;
}

template <class Pol>
static sg_status run_compact(Ctx *c, const Graph *g, const RowMaps &rm, const Pol &pol, const float *w_in,
                             int64_t *off_out, uint32_t *col_out, float *w_out, uint32_t *keep_bits,
                             unsigned long long *status, const char *name, int grid_per_sm = 0) {
    if (g->nnz == 0) {
        SG_CUDA(cudaMemsetAsync(off_out, 0, sizeof(int64_t) * (size_t)(g->n + 1), c->stream));
        return SG_OK;
    }
    // status words for every tile + the tile ticket, zeroed together
    SG_CUDA(cudaMemsetAsync(status, 0, sizeof(unsigned long long) * (size_t)(rm.num_tiles + 1), c->stream));
    CompactArgs a;
    a.off = g->off;
    a.col = g->col;
    a.w = w_in;
    a.n = g->n;
    a.nnz = g->nnz;
    a.num_tiles = rm.num_tiles;
    a.chunk_row = rm.chunk_row;
    a.tile_vlo = rm.tile_vlo;
    a.off_out = off_out;
    a.col_out = col_out;
    a.w_out = w_out;
    a.status = status;
    a.ticket = reinterpret_cast<unsigned int *>(status + rm.num_tiles);
    a.err = c->d_err;
    a.keep_bits = keep_bits;
    a.spin_limit = c->scan_hold ? c->scan_hold : kSpinLimit;
    a.hold_first = c->scan_hold != 0;
    const bool wt = w_out != nullptr;
    const int cap = wt ? blocks_per_sm<Pol, true>() : blocks_per_sm<Pol, false>();
    const int per_sm = grid_per_sm > 0 ? std::min(grid_per_sm, cap) : cap;
    const int64_t grid = std::min<int64_t>(rm.num_tiles, (int64_t)c->num_sms * per_sm);
    {
        SG_LAUNCH(c, name);
        if (wt)
            compact_kernel<Pol, true><<<(unsigned)grid, CW * 32, 0, c->stream>>>(a, pol);
        else
            compact_kernel<Pol, false><<<(unsigned)grid, CW * 32, 0, c->stream>>>(a, pol);
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
    sg_status st = build_row_maps(c, g, &rm);
    unsigned long long *status = nullptr;
    Graph *h = nullptr;
    const bool spectral = (k == SG_SPECTRAL_LOGN || k == SG_SPECTRAL_AVGDEG);
    const bool out_w = (spectral && want_weights) || g->w != nullptr;
    if (st == SG_OK) st = dalloc(c, (void **)&status, sizeof(unsigned long long) * (size_t)(rm.num_tiles + 1));
    if (st == SG_OK) st = new_graph(c, g->n, g->nnz, out_w, &h);
    if (st == SG_OK) {
        const uint32_t k0 = (uint32_t)(seed & 0xFFFFFFFFu), k1 = (uint32_t)(seed >> 32);
        if (k == SG_UNIFORM) {
            UniformPol pol{k0, k1, prob_threshold(p)};
            st = run_compact(c, g, rm, pol, g->w, h->off, h->col, h->w, nullptr, status, "compact_uniform");
        } else {
            const int64_t m = g->nnz / 2;
            const double y = (k == SG_SPECTRAL_LOGN) ? p * std::log((double)g->n)
                                                     : (g->n > 0 ? p * (double)m / (double)g->n : 0.0);
            SpectralPol pol{g->off, k0, k1, scaled_threshold(y), (float)y, want_weights != 0};
            st = run_compact(c, g, rm, pol, g->w, h->off, h->col, h->w, nullptr, status, "compact_spectral");
        }
    }
    if (st == SG_OK) st = read_i64(c, h->off + g->n, &h->nnz);
    if (st == SG_OK) st = check_device_error(c);
    dfree(c, status);
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
    if (st == SG_OK)
        st = dalloc(c, (void **)&o->status, sizeof(unsigned long long) * (size_t)(rm.num_tiles + 1));
    if (st != SG_OK) return st;
    uint16_t *deg16 = nullptr;
    st = dalloc(c, (void **)&deg16, sizeof(uint16_t) * (size_t)std::max<int64_t>(g->n, 1));
    if (st != SG_OK) return st;
    if (g->n > 0) {
        const int64_t blocks = std::min<int64_t>((g->n + 255) / 256, (int64_t)c->num_sms * 16);
        SG_LAUNCH(c, "compact_orient_deg");
        deg16_kernel<<<(unsigned)blocks, 256, 0, c->stream>>>(g->off, g->n, deg16);
    }
    OrientPol pol{g->off, deg16};
    st = run_compact(c, g, rm, pol, weights ? g->w : nullptr, o->off, o->col, weights ? o->w : nullptr,
                     o->fwd_bits, o->status, "compact_orient");
    dfree(c, deg16);
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
    dfree(c, o->status);
    dfree(c, o->inl);
    *o = Oriented{};
}

sg_status resolve_mask(Ctx *c, const Graph *g, const RowMaps &rm, const Oriented &o, const uint8_t *del,
                       Graph **out) {
    Graph *h = nullptr;
    unsigned long long *status = nullptr;
    sg_status st = new_graph(c, g->n, g->nnz, g->w != nullptr, &h);
    if (st == SG_OK) st = dalloc(c, (void **)&status, sizeof(unsigned long long) * (size_t)(rm.num_tiles + 1));
    if (st == SG_OK) {
        MaskPol pol{o.fwd_bits, o.status, o.inl, del, std::max<int64_t>(g->nnz - o.m, 1),
                    std::max<int64_t>(o.m, 1)};
        st = run_compact(c, g, rm, pol, g->w, h->off, h->col, h->w, nullptr, status, "compact_trmask");
    }
    if (st == SG_OK) st = read_i64(c, h->off + g->n, &h->nnz);
    if (st == SG_OK) st = check_device_error(c);
    dfree(c, status);
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
    static constexpr bool kOrPrefix = false;
    static constexpr bool kMapCol = false;
    struct Pre {
        uint32_t g;  // the graph of x
        int64_t dx, dy;
    };
    const int64_t *off;
    BatchDev b;
    __device__ __forceinline__ Pre load(uint32_t x, uint32_t y, int64_t, const SlabCtx &) const {
        return Pre{__ldg(b.vgid + x), __ldg(off + x + 1) - __ldg(off + x), __ldg(off + y + 1) - __ldg(off + y)};
    }
    __device__ __forceinline__ void load2(Pre &) const {}
    // only graphs compressed by a triangle kernel need E+
    __device__ __forceinline__ bool keep(const Pre &pr, uint32_t x, uint32_t y, int64_t, float &) const {
        const int kern = __ldg(&b.params[pr.g].kernel);
        if (kern < (int)SG_TR_RANDOM) return false;
        return pr.dx < pr.dy || (pr.dx == pr.dy && x < y);
    }
};

struct BatchFinalPol {
    static constexpr bool kOrPrefix = true;
    static constexpr bool kMapCol = true;
    struct Pre {
        MaskPol::Pre mp;
        uint32_t g;  // the graph of x
        uint64_t dmin;
    };
    const int64_t *off;
    BatchDev b;
    MaskPol mask;
    const uint32_t *fwd_bits;  // = mask.fwd_bits (read directly by the tile prologue)
    __device__ __forceinline__ int64_t tile_or_excl(int64_t tile) const { return mask.tile_or_excl(tile); }
    __device__ __forceinline__ Pre load(uint32_t x, uint32_t y, int64_t p, const SlabCtx &s) const {
        const uint64_t dx = (uint64_t)(__ldg(off + x + 1) - __ldg(off + x));
        const uint64_t dy = (uint64_t)(__ldg(off + y + 1) - __ldg(off + y));
        return Pre{mask.load(x, y, p, s), __ldg(b.vgid + x), dx < dy ? dx : dy};
    }
    __device__ __forceinline__ void load2(Pre &pr) const { mask.load2(pr.mp); }
    __device__ __forceinline__ uint32_t map_col(const Pre &pr, uint32_t, uint32_t y) const {
        return y - (uint32_t)__ldg(&b.params[pr.g].vbase);
    }
    // a graph's own kernel decides its arcs; a triangle kernel's through the mask
    __device__ __forceinline__ bool keep(const Pre &pr, uint32_t x, uint32_t y, int64_t p, float &w) const {
        const BatchParam &P = b.params[pr.g];
        const int kern = P.kernel;
        if (kern >= (int)SG_TR_RANDOM) return mask.keep(pr.mp, x, y, p, w);
        const uint32_t lx = (uint32_t)(x - P.vbase), ly = (uint32_t)(y - P.vbase);
        const uint4 r = philox4x32_10(make_uint4(min(lx, ly), max(lx, ly), 0u, kTagEdge), P.k0, P.k1);
        if (kern == (int)SG_UNIFORM) return (unsigned long long)r.x < P.tp;
        const uint64_t dmin = pr.dmin;
        if (P.reweight) w = (dmin * 4294967296ull <= P.ty) ? 1.0f : __fdiv_rn(__ull2float_rn(dmin), P.yf);
        return (unsigned long long)r.x * dmin < P.ty;
    }
};

sg_status batch_orient(Ctx *c, const Graph *u, const RowMaps &rm, const BatchDev &b, bool weights, Oriented *o,
                       unsigned long long *status, int grid_per_sm) {
    BatchOrientPol pol{u->off, b};
    return run_compact(c, u, rm, pol, weights ? u->w : nullptr, o->off, o->col, weights ? o->w : nullptr,
                       o->fwd_bits, status, "compact_orient", grid_per_sm);
}

sg_status batch_final(Ctx *c, const Graph *u, const RowMaps &rm, const Oriented &o, const BatchDev &b,
                      const uint8_t *del, int64_t *off_out, uint32_t *col_out, float *w_in, float *w_out,
                      unsigned long long *status, int grid_per_sm) {
    // the reverse arcs of graphs without a triangle kernel are not in the
    // reverse list (BatchFinalPol decides those arcs itself)
    // (its reverse list has room for every arc of the union, del for its m edges)
    BatchFinalPol pol{u->off, b,
                      MaskPol{o.fwd_bits, o.status, o.inl, del, std::max<int64_t>(u->nnz, 1), std::max<int64_t>(o.m, 1)},
                      o.fwd_bits};
    return run_compact(c, u, rm, pol, w_in, off_out, col_out, w_out, nullptr, status, "compact_final",
                       grid_per_sm);
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
    static constexpr bool kOrPrefix = false;
    static constexpr bool kMapCol = true;
    struct Pre {
        uint32_t nx, ny;  // new ids of x and y
    };
    const uint32_t *new_id;
    __device__ __forceinline__ Pre load(uint32_t x, uint32_t y, int64_t, const SlabCtx &) const {
        return Pre{__ldg(new_id + x), __ldg(new_id + y)};
    }
    __device__ __forceinline__ void load2(Pre &) const {}
    // an arc stays iff both of its ends stay; its head is renumbered
    __device__ __forceinline__ bool keep(const Pre &pr, uint32_t, uint32_t, int64_t, float &) const {
        return pr.nx != kNoVertex && pr.ny != kNoVertex;
    }
    __device__ __forceinline__ uint32_t map_col(const Pre &pr, uint32_t, uint32_t) const { return pr.ny; }
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
    unsigned long long *status = nullptr, *vstatus = nullptr;
    Graph *h = nullptr;
    int64_t kept = 0;
    sg_status st = build_row_maps(c, g, &rm);
    if (st == SG_OK) st = dalloc(c, (void **)&new_id, sizeof(uint32_t) * (size_t)std::max<int64_t>(g->n, 1));
    if (st == SG_OK) st = dalloc(c, (void **)&off_c, sizeof(int64_t) * (size_t)(g->n + 1));
    if (st == SG_OK) st = dalloc(c, (void **)&status, sizeof(unsigned long long) * (size_t)(rm.num_tiles + 1));
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
        st = run_compact(c, g, rm, pol, g->w, off_c, h->col, h->w, nullptr, status, "compact_lowdeg");
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
    dfree(c, status);
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
// the scratch (row maps, tile status words, the tile ticket and an error
// word) lives in one fixed file-scope device array instead of the stream-
// ordered pool.  Every process that loads this library reserves the array on
// each GPU it touches, for as long as the library stays loaded.
namespace sg {
namespace {

constexpr int64_t kNaMaxArcs = int64_t(1) << 27;
constexpr int64_t kNaMaxChunks = kNaMaxArcs / kWarpSpan;
constexpr int64_t kNaMaxTiles = kNaMaxArcs / kTile;
constexpr size_t na_align(size_t x) { return (x + 255) & ~size_t(255); }
constexpr size_t kNaChunkOff = 0;
constexpr size_t kNaTileOff = na_align(kNaChunkOff + sizeof(uint32_t) * (kNaMaxChunks + 1));
constexpr size_t kNaStatusOff = na_align(kNaTileOff + sizeof(int64_t) * (kNaMaxTiles + 1));
constexpr size_t kNaErrOff = na_align(kNaStatusOff + sizeof(unsigned long long) * (kNaMaxTiles + 1));
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
    const int64_t num_tiles = (nnz + kTile - 1) / kTile;
    const int64_t num_chunks = (nnz + kWarpSpan - 1) / kWarpSpan;
    uint32_t *chunk_row = reinterpret_cast<uint32_t *>(base + kNaChunkOff);
    int64_t *tile_vlo = reinterpret_cast<int64_t *>(base + kNaTileOff);
    unsigned long long *status = reinterpret_cast<unsigned long long *>(base + kNaStatusOff);
    // the status words and the ticket must start at zero on every call
    SG_CUDA(cudaMemsetAsync(status, 0, sizeof(unsigned long long) * (size_t)(num_tiles + 1), stream));
    const int64_t rb = std::min<int64_t>((n + 1 + 255) / 256, (int64_t)num_sms * 16);
    prefill_row_maps(stream, num_sms, chunk_row, num_chunks, tile_vlo, num_tiles, n);
    row_maps_kernel<<<(unsigned)std::max<int64_t>(rb, 1), 256, 0, stream>>>(off, n, chunk_row, num_chunks, tile_vlo,
                                                                           num_tiles);
    SG_CUDA(cudaGetLastError());
    CompactArgs a;
    a.off = off;
    a.col = col;
    a.w = nullptr;
    a.n = n;
    a.nnz = nnz;
    a.num_tiles = num_tiles;
    a.chunk_row = chunk_row;
    a.tile_vlo = tile_vlo;
    a.off_out = off_out;
    a.col_out = col_out;
    a.w_out = nullptr;
    a.status = status;
    a.ticket = reinterpret_cast<unsigned int *>(status + num_tiles);
    a.err = err;
    a.keep_bits = nullptr;
    a.spin_limit = kSpinLimit;
    a.hold_first = 0;
    UniformPol pol{(uint32_t)(seed & 0xFFFFFFFFu), (uint32_t)(seed >> 32), prob_threshold(p)};
    int per_sm = 0;
    SG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, compact_kernel<UniformPol, false>, CW * 32, 0));
    const int64_t grid = std::min<int64_t>(num_tiles, (int64_t)num_sms * std::max(per_sm, 1));
    compact_kernel<UniformPol, false><<<(unsigned)grid, CW * 32, 0, stream>>>(a, pol);
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

