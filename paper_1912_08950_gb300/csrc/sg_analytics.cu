// Accuracy analytics of Slim Graph (Sec. 5): PageRank (Table 1), the
// Kullback-Leibler divergence of two PageRank distributions (Sec. 5.2.3) and
// the number of connected components (Table 1), plus CSR validation.
//
// PageRank is FP32 with a fixed reduction order (no floating-point atomics),
// so a graph always yields the same vector; the dangling mass and the final
// L1 residual are reduced in fixed block order.  KL is evaluated in FP64 from
// the FP32 vectors.  Connected components use concurrent union-find: roots
// hook to the smaller root with atomicCAS, then pointer jumping flattens the
// forest; the count of self-parented vertices is exact whatever the schedule.
// The edges are taken in the order of Sutton et al.'s Afforest (IPDPS'18):
// every vertex first links its first kCcSample neighbours, the most frequent
// root among sampled vertices is taken as the giant component, and then only
// the rows of vertices outside it link their remaining neighbours (an edge
// leaving the giant component is seen from its other end).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "sg_internal.cuh"

namespace sg {

constexpr int kPrThreads = 256;
constexpr int kPrWarps = kPrThreads / 32;

// x'_v = (1-d)/n + d (sum_{u in N(v)} y_u + D/n), y_u = x_u / d_u; emits
// y' = x'/d and, per block, the FP32 dangling mass of x' (and, on the last
// iteration, the FP64 partial L1 residual |x' - x|).
//
// Row sums: a warp owns 32 consecutive rows.  Rows longer than 32 arcs are
// summed by the whole warp, one row at a time (lanes stride the row, then a
// fixed shuffle tree).  The short rows are summed together: their arcs are
// numbered consecutively across the 32 rows and streamed in slabs of 32, a
// lane finds its arc's row among the rows' starts (binary search over the
// lanes), a segmented shuffle scan sums each row's run inside the slab and the
// run's last lane adds it to the row's slot in shared memory.  Every order is
// fixed, so a graph always gives the same vector.
constexpr int kShortRow = 32;
constexpr int kHubRow = 1024;    // longer rows are summed in chunks by whole CTAs
constexpr int kHubChunk = 8192;  // arcs per chunk

__global__ void __launch_bounds__(kPrThreads) pr_iter_kernel(
    const int64_t *__restrict__ off, const uint32_t *__restrict__ col, int64_t n, const float *__restrict__ x,
    const float *__restrict__ y, const float *__restrict__ dangling_in, float base, float damping, float inv_n,
    float *__restrict__ x_new, float *__restrict__ y_new, float *__restrict__ dangling_part,
    double *__restrict__ resid_part, const int *__restrict__ hub_slot, const float *__restrict__ hub_part) {
    __shared__ float s_dang[kPrWarps];
    __shared__ double s_res[kPrWarps];
    __shared__ float s_acc[kPrWarps][32];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const float dterm = dangling_in[0] * inv_n;
    float dang = 0.f;
    double res = 0.0;
    const int64_t nwarps = (int64_t)gridDim.x * kPrWarps;
    for (int64_t r0 = ((int64_t)blockIdx.x * kPrWarps + warp) * 32; r0 < n; r0 += nwarps * 32) {
        const int64_t v = r0 + lane;
        int64_t b = 0, e = 0;
        if (v < n) {
            b = __ldg(off + v);
            e = __ldg(off + v + 1);
        }
        const int64_t deg = e - b;
        const bool longr = deg > kShortRow;
        // short rows: consecutive numbering of their arcs
        const int sdeg = longr ? 0 : (int)deg;
        int vs = sdeg;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(kFull, vs, o);
            if (lane >= o) vs += t;
        }
        const int total = __shfl_sync(kFull, vs, 31);
        vs -= sdeg;  // exclusive start of this row's arcs
        s_acc[warp][lane] = 0.f;
        __syncwarp();
        for (int s0 = 0; s0 < total; s0 += 32) {
            const int i = s0 + lane;
            const bool valid = i < total;
            int k = 0;  // the last row whose start is <= i
#pragma unroll
            for (int step = 16; step >= 1; step >>= 1) {
                const int sk = __shfl_sync(kFull, vs, k + step);
                if (sk <= i) k += step;
            }
            const int64_t bk = __shfl_sync(kFull, b, k);
            const int vk = __shfl_sync(kFull, vs, k);
            float val = valid ? __ldg(y + __ldg(col + bk + (i - vk))) : 0.f;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const float t = __shfl_up_sync(kFull, val, o);
                const int kt = __shfl_up_sync(kFull, k, o);
                if (lane >= o && kt == k) val += t;
            }
            const int kn = __shfl_down_sync(kFull, k, 1);
            if (valid && (lane == 31 || kn != k || i + 1 >= total)) s_acc[warp][k] += val;
            __syncwarp();
        }
        float s = s_acc[warp][lane];
        __syncwarp();
        // hub rows: their chunk sums, in chunk order
        if (deg > kHubRow) {
            const int first = __ldg(hub_slot + v);
            const int nch = (int)((deg + kHubChunk - 1) / kHubChunk);
            float t = 0.f;
            for (int c2 = 0; c2 < nch; ++c2) t += __ldg(hub_part + first + c2);
            s = t;
        }
        // long rows: the whole warp, one row at a time, fixed tree order
        unsigned longm = __ballot_sync(kFull, longr && deg <= kHubRow);
        while (longm) {
            const int src = __ffs(longm) - 1;
            longm &= longm - 1;
            const int64_t lb = __shfl_sync(kFull, b, src), le = __shfl_sync(kFull, e, src);
            float t = 0.f;
            for (int64_t i = lb + lane; i < le; i += 32) t += __ldg(y + __ldg(col + i));
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(kFull, t, o);
            if (lane == src) s = t;
        }
        if (v < n) {
            const float xv = base + damping * (s + dterm);
            x_new[v] = xv;
            y_new[v] = deg > 0 ? xv / (float)deg : 0.f;
            if (deg == 0) dang += xv;
            if (resid_part) res += fabs((double)xv - (double)__ldg(x + v));
        }
    }
    // fixed-order reductions: lanes, then warps, per block
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        dang += __shfl_xor_sync(kFull, dang, o);
        res += __shfl_xor_sync(kFull, res, o);
    }
    if (lane == 0) {
        s_dang[warp] = dang;
        s_res[warp] = res;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        float bd = 0.f;
        double br = 0.0;
        for (int i = 0; i < kPrWarps; ++i) {
            bd += s_dang[i];
            br += s_res[i];
        }
        dangling_part[blockIdx.x] = bd;
        if (resid_part) resid_part[blockIdx.x] = br;
    }
}

// Hub rows (more than kHubRow arcs) are cut into chunks of kHubChunk arcs;
// a CTA sums one chunk (threads stride it, then a fixed tree) into its slot.
__global__ void __launch_bounds__(kPrThreads) pr_hub_kernel(const uint32_t *__restrict__ col,
                                                            const float *__restrict__ y,
                                                            const int64_t *__restrict__ chunk_begin,
                                                            const int64_t *__restrict__ chunk_end,
                                                            float *__restrict__ hub_part) {
    __shared__ float s[kPrWarps];
    const int64_t b = chunk_begin[blockIdx.x], e = chunk_end[blockIdx.x];
    float t = 0.f;
    for (int64_t i = b + threadIdx.x; i < e; i += kPrThreads) t += __ldg(y + __ldg(col + i));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(kFull, t, o);
    if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = t;
    __syncthreads();
    if (threadIdx.x == 0) {
        float acc = 0.f;
        for (int w = 0; w < kPrWarps; ++w) acc += s[w];
        hub_part[blockIdx.x] = acc;
    }
}

// Hub rows and their chunk count (the list order is whatever the atomics give).
__global__ void pr_find_hubs_kernel(const int64_t *__restrict__ off, int64_t n, uint32_t *hubs,
                                    unsigned long long *counts) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
        const int64_t deg = off[v + 1] - off[v];
        if (deg > kHubRow) {
            hubs[atomicAdd(counts, 1ull)] = (uint32_t)v;
            atomicAdd(counts + 1, (unsigned long long)((deg + kHubChunk - 1) / kHubChunk));
        }
    }
}

// One CTA: each hub's first chunk slot (a running block scan over the hub
// list, 1024 hubs at a time) and the chunk bounds.
__global__ void __launch_bounds__(1024) pr_hub_chunks_kernel(const int64_t *__restrict__ off,
                                                             const uint32_t *__restrict__ hubs, int num_hubs,
                                                             int *hub_slot, int64_t *chunk_begin,
                                                             int64_t *chunk_end) {
    __shared__ int s_warp[32];
    __shared__ int s_run;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) s_run = 0;
    __syncthreads();
    for (int h0 = 0; h0 < num_hubs; h0 += 1024) {
        const int h = h0 + threadIdx.x;
        int64_t b = 0, e = 0;
        uint32_t v = 0;
        int nch = 0;
        if (h < num_hubs) {
            v = hubs[h];
            b = off[v];
            e = off[v + 1];
            nch = (int)((e - b + kHubChunk - 1) / kHubChunk);
        }
        int inc = nch;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(kFull, inc, o);
            if (lane >= o) inc += t;
        }
        if (lane == 31) s_warp[warp] = inc;
        __syncthreads();
        if (warp == 0) {
            const int wv = s_warp[lane];
            int wi = wv;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int t = __shfl_up_sync(kFull, wi, o);
                if (lane >= o) wi += t;
            }
            s_warp[lane] = wi - wv;
        }
        __syncthreads();
        int slot = s_run + s_warp[warp] + inc - nch;
        if (h < num_hubs) {
            hub_slot[v] = slot;
            for (int64_t c = b; c < e; c += kHubChunk, ++slot) {
                chunk_begin[slot] = c;
                chunk_end[slot] = c + kHubChunk < e ? c + kHubChunk : e;
            }
        }
        __syncthreads();
        if (threadIdx.x == 1023) s_run = slot;  // the last thread's next slot is the running total
        __syncthreads();
    }
}

// x0 = 1/n, y0 = x0/d, per-block dangling mass of x0
__global__ void __launch_bounds__(kPrThreads) pr_init_kernel(const int64_t *__restrict__ off, int64_t n, float x0,
                                                             float *__restrict__ x, float *__restrict__ y,
                                                             float *__restrict__ dangling_part) {
    __shared__ float s_dang[kPrWarps];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float dang = 0.f;
    const int64_t nwarps = (int64_t)gridDim.x * kPrWarps;
    for (int64_t r0 = ((int64_t)blockIdx.x * kPrWarps + warp) * 32; r0 < n; r0 += nwarps * 32) {
        const int64_t v = r0 + lane;
        if (v < n) {
            const int64_t deg = __ldg(off + v + 1) - __ldg(off + v);
            x[v] = x0;
            y[v] = deg > 0 ? x0 / (float)deg : 0.f;
            if (deg == 0) dang += x0;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) dang += __shfl_xor_sync(kFull, dang, o);
    if (lane == 0) s_dang[warp] = dang;
    __syncthreads();
    if (threadIdx.x == 0) {
        float bd = 0.f;
        for (int i = 0; i < kPrWarps; ++i) bd += s_dang[i];
        dangling_part[blockIdx.x] = bd;
    }
}

// one block: sum the per-block partials in a fixed order
template <typename T>
__global__ void __launch_bounds__(kPrThreads) reduce_parts_kernel(const T *__restrict__ parts, int count,
                                                                  T *__restrict__ out) {
    __shared__ T s[kPrThreads];
    T acc = 0;
    for (int i = threadIdx.x; i < count; i += kPrThreads) acc += parts[i];
    s[threadIdx.x] = acc;
    __syncthreads();
    for (int h = kPrThreads / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h) s[threadIdx.x] += s[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[0] = s[0];
}

sg_status pagerank(Ctx *c, const Graph *g, float damping, int iters, float *x_out, double *resid) {
    const int64_t n = g->n;
    *resid = 0.0;
    if (n == 0) return SG_OK;
    const int blocks = (int)std::min<int64_t>((n + kPrThreads - 1) / kPrThreads, (int64_t)c->num_sms * 8);
    float *buf = nullptr;
    // x_a, y_a, x_b, y_b, dangling partials, dangling total
    const size_t nn = (size_t)n;
    sg_status st = dalloc(c, (void **)&buf, sizeof(float) * (4 * nn + (size_t)blocks + 4));
    double *dres = nullptr;
    if (st == SG_OK) st = dalloc(c, (void **)&dres, sizeof(double) * ((size_t)blocks + 1));
    if (st != SG_OK) {
        dfree(c, buf);
        return st;
    }
    float *xa = buf, *ya = buf + nn, *xb = buf + 2 * nn, *yb = buf + 3 * nn;
    float *dpart = buf + 4 * nn, *dtot = dpart + blocks;
    const float inv_n = (float)(1.0 / (double)n);
    const float base = (float)((1.0 - (double)damping) / (double)n);
    // hub rows: list them once, then their chunks are summed before every iteration
    uint32_t *hubs = nullptr;
    unsigned long long *hcnt = nullptr;
    int *hub_slot = nullptr;
    int64_t *chunk_b = nullptr, *chunk_e = nullptr;
    float *hub_part = nullptr;
    int64_t num_hubs = 0, num_chunks = 0;
    st = dalloc(c, (void **)&hcnt, 2 * sizeof(unsigned long long));
    if (st == SG_OK) st = dalloc(c, (void **)&hubs, sizeof(uint32_t) * nn);
    if (st == SG_OK && cudaMemsetAsync(hcnt, 0, 2 * sizeof(unsigned long long), c->stream) != cudaSuccess)
        st = cuda_fail(cudaGetLastError(), "cudaMemsetAsync");
    if (st == SG_OK) {
        SG_LAUNCH(c, "pr_hubs");
        pr_find_hubs_kernel<<<blocks, kPrThreads, 0, c->stream>>>(g->off, n, hubs, hcnt);
        if (cudaMemcpyAsync(c->h_pinned, hcnt, 2 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, c->stream) !=
                cudaSuccess ||
            cudaStreamSynchronize(c->stream) != cudaSuccess)
            st = cuda_fail(cudaGetLastError(), "PageRank hub count");
        num_hubs = c->h_pinned[0];
        num_chunks = c->h_pinned[1];
    }
    if (st == SG_OK && num_hubs > 0) {
        st = dalloc(c, (void **)&hub_slot, sizeof(int) * nn);
        if (st == SG_OK) st = dalloc(c, (void **)&chunk_b, sizeof(int64_t) * (size_t)num_chunks);
        if (st == SG_OK) st = dalloc(c, (void **)&chunk_e, sizeof(int64_t) * (size_t)num_chunks);
        if (st == SG_OK) st = dalloc(c, (void **)&hub_part, sizeof(float) * (size_t)num_chunks);
        if (st == SG_OK) {
            SG_LAUNCH(c, "pr_hubs");
            pr_hub_chunks_kernel<<<1, 1024, 0, c->stream>>>(g->off, hubs, (int)num_hubs, hub_slot, chunk_b, chunk_e);
        }
    }
    if (st != SG_OK) {
        dfree(c, hubs); dfree(c, hcnt); dfree(c, hub_slot); dfree(c, chunk_b); dfree(c, chunk_e); dfree(c, hub_part);
        dfree(c, buf); dfree(c, dres);
        return st;
    }
    {
        SG_LAUNCH(c, "pr_init");
        pr_init_kernel<<<blocks, kPrThreads, 0, c->stream>>>(g->off, n, inv_n, xa, ya, dpart);
    }
    {
        SG_LAUNCH(c, "pr_reduce");
        reduce_parts_kernel<float><<<1, kPrThreads, 0, c->stream>>>(dpart, blocks, dtot);
    }
    for (int it = 0; it < iters; ++it) {
        const bool last = (it == iters - 1);
        float *xo = last ? x_out : xb;
        if (num_chunks > 0) {
            SG_LAUNCH(c, "pr_hub");
            pr_hub_kernel<<<(unsigned)num_chunks, kPrThreads, 0, c->stream>>>(g->col, ya, chunk_b, chunk_e, hub_part);
        }
        {
            SG_LAUNCH(c, "pr_iter");
            pr_iter_kernel<<<blocks, kPrThreads, 0, c->stream>>>(g->off, g->col, n, xa, ya, dtot, base, damping, inv_n,
                                                                 xo, yb, dpart, last ? dres : nullptr, hub_slot,
                                                                 hub_part);
        }
        if (!last) {
            SG_LAUNCH(c, "pr_reduce");
            reduce_parts_kernel<float><<<1, kPrThreads, 0, c->stream>>>(dpart, blocks, dtot);
        }
        std::swap(xa, xb);
        std::swap(ya, yb);
    }
    {
        SG_LAUNCH(c, "pr_reduce");
        reduce_parts_kernel<double><<<1, kPrThreads, 0, c->stream>>>(dres, blocks, dres + blocks);
    }
    SG_CUDA(cudaGetLastError());
    SG_CUDA(cudaMemcpyAsync(c->h_pinned, dres + blocks, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    SG_CUDA(cudaStreamSynchronize(c->stream));
    std::memcpy(resid, c->h_pinned, sizeof(double));
    dfree(c, hubs);
    dfree(c, hcnt);
    dfree(c, hub_slot);
    dfree(c, chunk_b);
    dfree(c, chunk_e);
    dfree(c, hub_part);
    dfree(c, buf);
    dfree(c, dres);
    return SG_OK;
}

// ---------------------------------------------------------------------- KL
__global__ void __launch_bounds__(kPrThreads) sum2_kernel(const float *__restrict__ P, const float *__restrict__ Q,
                                                          int64_t n, double *__restrict__ parts) {
    __shared__ double s[2][kPrThreads];
    double a = 0.0, b = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * kPrThreads + threadIdx.x; i < n; i += (int64_t)gridDim.x * kPrThreads) {
        a += (double)P[i];
        b += (double)Q[i];
    }
    s[0][threadIdx.x] = a;
    s[1][threadIdx.x] = b;
    __syncthreads();
    for (int h = kPrThreads / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h) {
            s[0][threadIdx.x] += s[0][threadIdx.x + h];
            s[1][threadIdx.x] += s[1][threadIdx.x + h];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        parts[2 * blockIdx.x] = s[0][0];
        parts[2 * blockIdx.x + 1] = s[1][0];
    }
}

// Per-vertex terms in FP32, summed in FP64.  With p_i = P_i / S_P and
// q_i = Q_i / S_Q (S the FP64 sums), sum_i p_i log2(p_i / q_i)
//   = (sum_i P_i log2(P_i / Q_i)) / S_P + log2(S_Q / S_P),
// so a term is the FP32 product P_i * log2f(P_i / Q_i) of the raw values and
// the normalisation enters once, in FP64, after the sum.
__global__ void __launch_bounds__(kPrThreads) kl_terms_kernel(const float *__restrict__ P, const float *__restrict__ Q,
                                                              int64_t n, double *__restrict__ parts) {
    __shared__ double s[kPrThreads];
    double acc = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * kPrThreads + threadIdx.x; i < n; i += (int64_t)gridDim.x * kPrThreads) {
        const float p = P[i];
        if (p > 0.f) acc += (double)(p * log2f(p / Q[i]));
    }
    s[threadIdx.x] = acc;
    __syncthreads();
    for (int h = kPrThreads / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h) s[threadIdx.x] += s[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) parts[blockIdx.x] = s[0];
}

__global__ void reduce_pairs_kernel(const double *__restrict__ parts, int count, double *__restrict__ out) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double a = 0.0, b = 0.0;
        for (int i = 0; i < count; ++i) {
            a += parts[2 * i];
            b += parts[2 * i + 1];
        }
        out[0] = a;
        out[1] = b;
    }
}

sg_status kl_divergence(Ctx *c, int64_t n, const float *P, const float *Q, double *kl) {
    *kl = 0.0;
    if (n == 0) return SG_OK;
    const int blocks = (int)std::min<int64_t>((n + kPrThreads - 1) / kPrThreads, (int64_t)c->num_sms * 4);
    double *buf = nullptr;
    sg_status st = dalloc(c, (void **)&buf, sizeof(double) * (3 * (size_t)blocks + 4));
    if (st != SG_OK) return st;
    double *pairs = buf, *sums = buf + 2 * blocks, *terms = sums + 2, *tot = terms + blocks;
    {
        SG_LAUNCH(c, "kl_sums");
        sum2_kernel<<<blocks, kPrThreads, 0, c->stream>>>(P, Q, n, pairs);
    }
    {
        SG_LAUNCH(c, "kl_reduce");
        reduce_pairs_kernel<<<1, 32, 0, c->stream>>>(pairs, blocks, sums);
    }
    {
        SG_LAUNCH(c, "kl_terms");
        kl_terms_kernel<<<blocks, kPrThreads, 0, c->stream>>>(P, Q, n, terms);
    }
    {
        SG_LAUNCH(c, "kl_reduce");
        reduce_parts_kernel<double><<<1, kPrThreads, 0, c->stream>>>(terms, blocks, tot);
    }
    SG_CUDA(cudaGetLastError());
    // sums (S_P, S_Q) and the term total are adjacent: one copy
    static_assert(sizeof(double) == sizeof(int64_t), "pinned scratch holds doubles");
    SG_CUDA(cudaMemcpyAsync(c->h_pinned, sums, sizeof(double) * 2, cudaMemcpyDeviceToHost, c->stream));
    SG_CUDA(cudaMemcpyAsync(c->h_pinned + 2, tot, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    SG_CUDA(cudaStreamSynchronize(c->stream));
    double h[3];
    std::memcpy(h, c->h_pinned, sizeof(h));
    // FP64: the sum of the FP32 terms, normalised (see kl_terms_kernel)
    *kl = (h[0] > 0.0 && h[1] > 0.0) ? h[2] / h[0] + std::log2(h[1] / h[0]) : 0.0;
    dfree(c, buf);
    return SG_OK;
}

// ---------------------------------------------------------------------- CC
__global__ void cc_init_kernel(uint32_t *parent, int64_t n) {
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
        parent[v] = (uint32_t)v;
}

__device__ __forceinline__ uint32_t cc_find(uint32_t *parent, uint32_t v) {
    uint32_t p = parent[v];
    while (p != v) {
        const uint32_t gp = parent[p];
        if (gp != p) parent[v] = gp;  // path halving; gp is still an ancestor of v
        v = p;
        p = gp;
    }
    return v;
}

constexpr int kCcSample = 2;     // neighbours every vertex links first
constexpr int kCcProbes = 1024;  // sampled vertices that name the giant component

// join the trees of x and y: the larger root hooks under the smaller
__device__ __forceinline__ void cc_link(uint32_t *parent, uint32_t x, uint32_t y) {
    uint32_t rx = cc_find(parent, x), ry = cc_find(parent, y);
    while (rx != ry) {
        const uint32_t hi = rx > ry ? rx : ry, lo = rx > ry ? ry : rx;
        const uint32_t old = atomicCAS(parent + hi, hi, lo);
        if (old == hi) break;
        rx = cc_find(parent, hi);
        ry = cc_find(parent, lo);
    }
}

// thread per vertex: link its first kCcSample neighbours
__global__ void cc_sample_kernel(const int64_t *__restrict__ off, const uint32_t *__restrict__ col, int64_t n,
                                 uint32_t *parent) {
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n; x += (int64_t)gridDim.x * blockDim.x) {
        const int64_t b = __ldg(off + x), e = __ldg(off + x + 1);
        for (int64_t i = b; i < e && i < b + kCcSample; ++i) cc_link(parent, (uint32_t)x, __ldg(col + i));
    }
}

__global__ void cc_compress_kernel(uint32_t *parent, int64_t n) {
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
        parent[v] = cc_find(parent, (uint32_t)v);
}

// roots of kCcProbes vertices spread over [0, n) by a fixed multiplicative hash
__global__ void cc_probe_kernel(const uint32_t *parent, int64_t n, uint32_t *out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < kCcProbes) {
        const uint64_t v = ((uint64_t)((uint32_t)i * 0x9E3779B1u) * (uint64_t)n) >> 32;
        out[i] = parent[v];
    }
}

// warp per row outside the giant component: link the neighbours after the sampled ones
__global__ void cc_rest_kernel(const int64_t *__restrict__ off, const uint32_t *__restrict__ col, int64_t n,
                               uint32_t *parent, uint32_t giant) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t x = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp; x < n; x += nw) {
        const int64_t b = __ldg(off + x), e = __ldg(off + x + 1);
        if (e - b <= kCcSample) continue;
        uint32_t r = 0;
        if (lane == 0) r = cc_find(parent, (uint32_t)x);
        if (__shfl_sync(0xFFFFFFFFu, r, 0) == giant) continue;
        for (int64_t i = b + kCcSample + lane; i < e; i += 32) cc_link(parent, (uint32_t)x, __ldg(col + i));
    }
}

__global__ void __launch_bounds__(256) cc_finish_kernel(uint32_t *parent, int64_t n, unsigned long long *roots) {
    unsigned long long cnt = 0;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t r = cc_find(parent, (uint32_t)v);
        if (r == (uint32_t)v) ++cnt;
    }
    cnt = warp_sum(cnt);
    if ((threadIdx.x & 31) == 0 && cnt) atomicAdd(roots, cnt);
}

__global__ void cc_label_kernel(const uint32_t *parent, int64_t n, uint32_t *labels) {
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        uint32_t r = parent[v];
        while (parent[r] != r) r = parent[r];
        labels[v] = r;
    }
}

sg_status cc_count(Ctx *c, const Graph *g, int64_t *count, uint32_t *labels) {
    *count = 0;
    const int64_t n = g->n;
    if (n == 0) return SG_OK;
    uint32_t *parent = nullptr;
    unsigned long long *roots = nullptr;
    sg_status st = dalloc(c, (void **)&parent, sizeof(uint32_t) * (size_t)n);
    // roots: the root count, then kCcProbes sampled roots
    if (st == SG_OK) st = dalloc(c, (void **)&roots, sizeof(unsigned long long) + sizeof(uint32_t) * kCcProbes);
    if (st != SG_OK) {
        dfree(c, parent);
        return st;
    }
    const int blocks = (int)std::min<int64_t>((n + 255) / 256, (int64_t)c->num_sms * 8);
    SG_CUDA(cudaMemsetAsync(roots, 0, sizeof(unsigned long long), c->stream));
    {
        SG_LAUNCH(c, "cc_init");
        cc_init_kernel<<<blocks, 256, 0, c->stream>>>(parent, n);
    }
    {
        SG_LAUNCH(c, "cc_sample");
        cc_sample_kernel<<<blocks, 256, 0, c->stream>>>(g->off, g->col, n, parent);
    }
    {
        SG_LAUNCH(c, "cc_compress");
        cc_compress_kernel<<<blocks, 256, 0, c->stream>>>(parent, n);
    }
    {
        SG_LAUNCH(c, "cc_probe");
        cc_probe_kernel<<<(kCcProbes + 255) / 256, 256, 0, c->stream>>>(parent, n, reinterpret_cast<uint32_t *>(roots + 1));
    }
    SG_CUDA(cudaGetLastError());
    SG_CUDA(cudaMemcpyAsync(c->h_pinned, roots + 1, sizeof(uint32_t) * kCcProbes, cudaMemcpyDeviceToHost, c->stream));
    SG_CUDA(cudaStreamSynchronize(c->stream));
    uint32_t giant = 0;
    {
        // the most frequent root among the probes (ties: the smaller root)
        std::vector<uint32_t> pr(kCcProbes);
        std::memcpy(pr.data(), c->h_pinned, sizeof(uint32_t) * kCcProbes);
        std::sort(pr.begin(), pr.end());
        int best = 0;
        for (int i = 0; i < kCcProbes;) {
            int j = i;
            while (j < kCcProbes && pr[j] == pr[i]) ++j;
            if (j - i > best) { best = j - i; giant = pr[i]; }
            i = j;
        }
    }
    {
        SG_LAUNCH(c, "cc_rest");
        const int hb = (int)std::min<int64_t>((n + 7) / 8, (int64_t)c->num_sms * 8);
        cc_rest_kernel<<<hb, 256, 0, c->stream>>>(g->off, g->col, n, parent, giant);
    }
    {
        SG_LAUNCH(c, "cc_finish");
        cc_finish_kernel<<<blocks, 256, 0, c->stream>>>(parent, n, roots);
    }
    if (labels) {
        SG_LAUNCH(c, "cc_label");
        cc_label_kernel<<<blocks, 256, 0, c->stream>>>(parent, n, labels);
    }
    SG_CUDA(cudaGetLastError());
    SG_CUDA(cudaMemcpyAsync(c->h_pinned, roots, sizeof(unsigned long long), cudaMemcpyDeviceToHost, c->stream));
    SG_CUDA(cudaStreamSynchronize(c->stream));
    unsigned long long r = 0;
    std::memcpy(&r, c->h_pinned, sizeof(r));
    *count = (int64_t)r;
    dfree(c, parent);
    dfree(c, roots);
    return SG_OK;
}

// ------------------------------------------------------ BFS levels (Sec. 5.3)
// Level-synchronous BFS over an int32 level array (-1 = unreached).  Each step
// is top-down (the frontier pushes L + 1 into unreached neighbours) or, once
// the frontier holds more than n/32 vertices, bottom-up (every unreached
// vertex looks for a neighbour on level L) -- the direction switch of Beamer,
// Asanovic and Patterson (SC'12).  Concurrent writes of L + 1 to one entry
// store the same value, so no atomics are needed; levels are unique, whatever
// the order of the writes.
__global__ void __launch_bounds__(256) bfs_top_down_kernel(const int64_t *__restrict__ off,
                                                           const uint32_t *__restrict__ col, int64_t n,
                                                           int *level, int L) {
    const int lane = threadIdx.x & 31;
    const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t base = ((int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * 32; base < n;
         base += nw * 32) {
        const int64_t v = base + lane;
        unsigned fm = __ballot_sync(kFull, v < n && level[v] == L);
        while (fm) {
            const int src = __ffs(fm) - 1;
            fm &= fm - 1;
            const int64_t x = base + src;
            const int64_t o = __ldg(off + x), d = __ldg(off + x + 1) - o;
            for (int64_t i = lane; i < d; i += 32) {
                const uint32_t y = __ldg(col + o + i);
                if (level[y] < 0) level[y] = L + 1;
            }
        }
    }
}

__global__ void __launch_bounds__(256) bfs_bottom_up_kernel(const int64_t *__restrict__ off,
                                                            const uint32_t *__restrict__ col, int64_t n,
                                                            int *level, int L) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
        if (level[v] >= 0) continue;
        const int64_t e = __ldg(off + v + 1);
        for (int64_t i = __ldg(off + v); i < e; ++i)
            if (level[__ldg(col + i)] == L) {
                level[v] = L + 1;
                break;
            }
    }
}

__global__ void __launch_bounds__(256) count_level_kernel(const int *__restrict__ level, int64_t n, int L,
                                                          unsigned long long *cnt) {
    unsigned long long k = 0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) k += level[v] == L;
    k = warp_sum(k);
    if ((threadIdx.x & 31) == 0 && k) atomicAdd(cnt, k);
}

__global__ void set_root_kernel(int *level, int64_t root) { level[root] = 0; }

sg_status bfs_levels(Ctx *c, const Graph *g, int64_t root, int *level) {
    if (g->n == 0) return SG_OK;
    SG_CUDA(cudaMemsetAsync(level, 0xFF, sizeof(int) * (size_t)g->n, c->stream));
    if (root < 0 || root >= g->n) return SG_OK;  // nothing is reached
    {
        SG_LAUNCH(c, "bfs_root");
        set_root_kernel<<<1, 1, 0, c->stream>>>(level, root);
    }
    unsigned long long *cnt = nullptr;
    sg_status st = dalloc(c, (void **)&cnt, sizeof(unsigned long long));
    if (st != SG_OK) return st;
    const int64_t blocks = std::max<int64_t>(1, std::min<int64_t>((g->n + 255) / 256, (int64_t)c->num_sms * 8));
    unsigned long long frontier = 1;
    for (int L = 0; frontier > 0 && st == SG_OK; ++L) {
        if (L > (int)std::min<int64_t>(g->n, INT32_MAX - 1)) { st = fail(SG_ERR_CUDA, "BFS did not terminate"); break; }
        if (frontier * 32 > (unsigned long long)g->n) {
            SG_LAUNCH(c, "bfs_step");
            bfs_bottom_up_kernel<<<(unsigned)blocks, 256, 0, c->stream>>>(g->off, g->col, g->n, level, L);
        } else {
            SG_LAUNCH(c, "bfs_step");
            bfs_top_down_kernel<<<(unsigned)blocks, 256, 0, c->stream>>>(g->off, g->col, g->n, level, L);
        }
        if (cudaMemsetAsync(cnt, 0, sizeof(unsigned long long), c->stream) != cudaSuccess) {
            st = cuda_fail(cudaGetLastError(), "cudaMemsetAsync");
            break;
        }
        {
            SG_LAUNCH(c, "bfs_count");
            count_level_kernel<<<(unsigned)blocks, 256, 0, c->stream>>>(level, g->n, L + 1, cnt);
        }
        if (cudaGetLastError() != cudaSuccess) { st = fail(SG_ERR_CUDA, "BFS launch"); break; }
        if (cudaMemcpyAsync(c->h_pinned, cnt, sizeof(unsigned long long), cudaMemcpyDeviceToHost, c->stream) !=
                cudaSuccess ||
            cudaStreamSynchronize(c->stream) != cudaSuccess) {
            st = cuda_fail(cudaGetLastError(), "BFS frontier count");
            break;
        }
        frontier = c->h_pinned[0];
    }
    dfree(c, cnt);
    return st;
}

// |E_cr| (Sec. 5.3): undirected edges joining BFS levels L and L + 1, each
// counted once from its lower end.
__global__ void __launch_bounds__(256) critical_kernel(const int64_t *__restrict__ off,
                                                       const uint32_t *__restrict__ col, int64_t n,
                                                       const int *__restrict__ level, unsigned long long *cnt) {
    const int lane = threadIdx.x & 31;
    const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
    unsigned long long k = 0;
    for (int64_t base = ((int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * 32; base < n;
         base += nw * 32) {
        const int64_t v = base + lane;
        const int lv = v < n ? __ldg(level + v) : -1;
        unsigned fm = __ballot_sync(kFull, lv >= 0);
        while (fm) {
            const int src = __ffs(fm) - 1;
            fm &= fm - 1;
            const int64_t x = base + src;
            const int lx = __shfl_sync(kFull, lv, src);
            const int64_t o = __ldg(off + x), d = __ldg(off + x + 1) - o;
            for (int64_t i = lane; i < d; i += 32) k += __ldg(level + __ldg(col + o + i)) == lx + 1;
        }
    }
    k = warp_sum(k);
    if (lane == 0 && k) atomicAdd(cnt, k);
}

sg_status critical_edges(Ctx *c, const Graph *g, int64_t root, int64_t *count) {
    *count = 0;
    if (g->n == 0) return SG_OK;
    int *level = nullptr;
    unsigned long long *cnt = nullptr;
    sg_status st = dalloc(c, (void **)&level, sizeof(int) * (size_t)g->n);
    if (st == SG_OK) st = dalloc(c, (void **)&cnt, sizeof(unsigned long long));
    if (st == SG_OK) st = bfs_levels(c, g, root, level);
    if (st == SG_OK && cudaMemsetAsync(cnt, 0, sizeof(unsigned long long), c->stream) != cudaSuccess)
        st = cuda_fail(cudaGetLastError(), "cudaMemsetAsync");
    if (st == SG_OK) {
        const int64_t blocks = std::max<int64_t>(1, std::min<int64_t>((g->n + 255) / 256, (int64_t)c->num_sms * 8));
        SG_LAUNCH(c, "critical_edges");
        critical_kernel<<<(unsigned)blocks, 256, 0, c->stream>>>(g->off, g->col, g->n, level, cnt);
        if (cudaGetLastError() != cudaSuccess) st = fail(SG_ERR_CUDA, "critical_edges launch");
    }
    if (st == SG_OK) {
        if (cudaMemcpyAsync(c->h_pinned, cnt, sizeof(unsigned long long), cudaMemcpyDeviceToHost, c->stream) !=
                cudaSuccess ||
            cudaStreamSynchronize(c->stream) != cudaSuccess)
            st = cuda_fail(cudaGetLastError(), "critical_edges read");
        else
            *count = (int64_t)c->h_pinned[0];
    }
    dfree(c, level);
    dfree(c, cnt);
    return st;
}

// ----------------------------------------------- A_REN (Sec. 5.2.2)
// Edges {u,v} of G (each once, from its smaller end) whose endpoint scores
// change relative order: sign(x_u - x_v) != sign(y_u - y_v), compared in the
// scores' own type.
template <typename T>
__device__ __forceinline__ int order_sign(T a, T b) {
    return (int)(a > b) - (int)(a < b);
}

template <typename T>
__global__ void __launch_bounds__(256) reordered_kernel(const int64_t *__restrict__ off,
                                                        const uint32_t *__restrict__ col, int64_t n,
                                                        const T *__restrict__ x, const T *__restrict__ y,
                                                        unsigned long long *cnt) {
    const int lane = threadIdx.x & 31;
    const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
    unsigned long long k = 0;
    for (int64_t u = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); u < n; u += nw) {
        const int64_t o = __ldg(off + u), d = __ldg(off + u + 1) - o;
        const T xu = x[u], yu = y[u];
        for (int64_t i = lane; i < d; i += 32) {
            const uint32_t v = __ldg(col + o + i);
            if ((int64_t)v > u) k += order_sign(xu, x[v]) != order_sign(yu, y[v]);
        }
    }
    k = warp_sum(k);
    if (lane == 0 && k) atomicAdd(cnt, k);
}

template <typename T>
sg_status reordered_neighbours(Ctx *c, const Graph *g, const T *x, const T *y, int64_t *count) {
    *count = 0;
    if (g->n == 0) return SG_OK;
    unsigned long long *cnt = nullptr;
    sg_status st = dalloc(c, (void **)&cnt, sizeof(unsigned long long));
    if (st == SG_OK && cudaMemsetAsync(cnt, 0, sizeof(unsigned long long), c->stream) != cudaSuccess)
        st = cuda_fail(cudaGetLastError(), "cudaMemsetAsync");
    if (st == SG_OK) {
        const int64_t blocks = std::max<int64_t>(1, std::min<int64_t>((g->n + 7) / 8, (int64_t)c->num_sms * 8));
        SG_LAUNCH(c, "reordered");
        reordered_kernel<T><<<(unsigned)blocks, 256, 0, c->stream>>>(g->off, g->col, g->n, x, y, cnt);
        if (cudaGetLastError() != cudaSuccess) st = fail(SG_ERR_CUDA, "reordered launch");
    }
    if (st == SG_OK) {
        if (cudaMemcpyAsync(c->h_pinned, cnt, sizeof(unsigned long long), cudaMemcpyDeviceToHost, c->stream) !=
                cudaSuccess ||
            cudaStreamSynchronize(c->stream) != cudaSuccess)
            st = cuda_fail(cudaGetLastError(), "reordered read");
        else
            *count = (int64_t)c->h_pinned[0];
    }
    dfree(c, cnt);
    return st;
}
template sg_status reordered_neighbours<float>(Ctx *, const Graph *, const float *, const float *, int64_t *);
template sg_status reordered_neighbours<unsigned long long>(Ctx *, const Graph *, const unsigned long long *,
                                                            const unsigned long long *, int64_t *);

// The vertex of largest degree (smallest id on ties): the default BFS root.
__global__ void max_degree_kernel(const int64_t *__restrict__ off, int64_t n, unsigned long long *best) {
    unsigned long long b = 0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
        const unsigned long long d = (unsigned long long)(off[v + 1] - off[v]);
        const unsigned long long key = (d << 32) | (0xFFFFFFFFull - (unsigned long long)v);
        b = key > b ? key : b;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long t = __shfl_xor_sync(kFull, b, o);
        b = t > b ? t : b;
    }
    if ((threadIdx.x & 31) == 0) atomicMax(best, b);
}

sg_status max_degree_vertex(Ctx *c, const Graph *g, int64_t *v) {
    *v = -1;
    if (g->n == 0) return SG_OK;
    unsigned long long *best = nullptr;
    sg_status st = dalloc(c, (void **)&best, sizeof(unsigned long long));
    if (st == SG_OK && cudaMemsetAsync(best, 0, sizeof(unsigned long long), c->stream) != cudaSuccess)
        st = cuda_fail(cudaGetLastError(), "cudaMemsetAsync");
    if (st == SG_OK) {
        const int64_t blocks = std::max<int64_t>(1, std::min<int64_t>((g->n + 255) / 256, (int64_t)c->num_sms * 8));
        SG_LAUNCH(c, "max_degree");
        max_degree_kernel<<<(unsigned)blocks, 256, 0, c->stream>>>(g->off, g->n, best);
        if (cudaGetLastError() != cudaSuccess) st = fail(SG_ERR_CUDA, "max_degree launch");
    }
    if (st == SG_OK) {
        if (cudaMemcpyAsync(c->h_pinned, best, sizeof(unsigned long long), cudaMemcpyDeviceToHost, c->stream) !=
                cudaSuccess ||
            cudaStreamSynchronize(c->stream) != cudaSuccess)
            st = cuda_fail(cudaGetLastError(), "max_degree read");
        else
            *v = (int64_t)(0xFFFFFFFFull - (c->h_pinned[0] & 0xFFFFFFFFull));
    }
    dfree(c, best);
    return st;
}


// ---------------------------------------------------------------- validate
__global__ void validate_kernel(const int64_t *__restrict__ off, const uint32_t *__restrict__ col, int64_t n,
                                int64_t nnz, int *err) {
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n; x += (int64_t)gridDim.x * blockDim.x) {
        const int64_t b = off[x], e = off[x + 1];
        bool bad = b < 0 || (x == 0 && b != 0) || e < b || (x == n - 1 && e != nnz) || e > nnz;
        for (int64_t i = b; !bad && i < e; ++i) {
            const uint32_t y = col[i];
            if (y >= (uint64_t)n || y == (uint32_t)x || (i > b && col[i - 1] >= y)) {
                bad = true;
                break;
            }
            // the reverse arc must exist
            const int64_t yb = off[y], ye = off[y + 1];
            if (yb < 0 || ye > nnz || ye < yb) { bad = true; break; }
            const int64_t k = lower_bound_u32(col, yb, ye, (uint32_t)x);
            if (k >= ye || col[k] != (uint32_t)x) bad = true;
        }
        if (bad) atomicExch(err, (int)kDevBadGraph);
    }
}

sg_status validate_graph(Ctx *c, const Graph *g) {
    if (g->n == 0) {
        if (g->nnz != 0) return fail(SG_ERR_INVALID_GRAPH, "an empty vertex set cannot hold arcs");
        return SG_OK;
    }
    const int blocks = (int)std::min<int64_t>((g->n + 255) / 256, (int64_t)c->num_sms * 8);
    {
        SG_LAUNCH(c, "validate");
        validate_kernel<<<blocks, 256, 0, c->stream>>>(g->off, g->col, g->n, g->nnz, c->d_err);
    }
    SG_CUDA(cudaGetLastError());
    return check_device_error(c);
}

}  // namespace sg
