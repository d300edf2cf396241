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
#include <cmath>
#include <cstring>

#include "sg_internal.cuh"

namespace sg {

constexpr int kPrThreads = 256;
constexpr int kPrWarps = kPrThreads / 32;
constexpr int kShortRow = 16;  // rows up to this degree are summed by one lane

// x'_v = (1-d)/n + d (sum_{u in N(v)} y_u + D/n), y_u = x_u / d_u; emits
// y' = x'/d and, per block, the FP32 dangling mass of x' (and, on the last
// iteration, the FP64 partial L1 residual |x' - x|).
__global__ void __launch_bounds__(kPrThreads) pr_iter_kernel(
    const int64_t *__restrict__ off, const uint32_t *__restrict__ col, int64_t n, const float *__restrict__ x,
    const float *__restrict__ y, const float *__restrict__ dangling_in, float base, float damping, float inv_n,
    float *__restrict__ x_new, float *__restrict__ y_new, float *__restrict__ dangling_part,
    double *__restrict__ resid_part) {
    __shared__ float s_dang[kPrWarps];
    __shared__ double s_res[kPrWarps];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const float dterm = dangling_in[0] * inv_n;
    float dang = 0.f;
    double res = 0.0;
    const int64_t nwarps = (int64_t)gridDim.x * kPrWarps;
    // each warp owns blocks of 32 consecutive rows
    for (int64_t r0 = ((int64_t)blockIdx.x * kPrWarps + warp) * 32; r0 < n; r0 += nwarps * 32) {
        const int64_t v = r0 + lane;
        int64_t b = 0, e = 0;
        if (v < n) {
            b = __ldg(off + v);
            e = __ldg(off + v + 1);
        }
        const int64_t deg = e - b;
        float s = 0.f;
        if (deg <= kShortRow) {
            for (int64_t i = b; i < e; ++i) s += __ldg(y + __ldg(col + i));
        }
        // long rows: the whole warp, one row at a time, fixed tree order
        unsigned longm = __ballot_sync(kFull, deg > kShortRow);
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
        {
            SG_LAUNCH(c, "pr_iter");
            pr_iter_kernel<<<blocks, kPrThreads, 0, c->stream>>>(g->off, g->col, n, xa, ya, dtot, base, damping, inv_n,
                                                                 xo, yb, dpart, last ? dres : nullptr);
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

__global__ void __launch_bounds__(kPrThreads) kl_terms_kernel(const float *__restrict__ P, const float *__restrict__ Q,
                                                              int64_t n, const double *__restrict__ sums,
                                                              double *__restrict__ parts) {
    __shared__ double s[kPrThreads];
    const double sp = sums[0], sq = sums[1];
    double acc = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * kPrThreads + threadIdx.x; i < n; i += (int64_t)gridDim.x * kPrThreads) {
        const double p = (double)P[i] / sp;
        const double q = (double)Q[i] / sq;
        if (p > 0.0) acc += p * log2(p / q);
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
        kl_terms_kernel<<<blocks, kPrThreads, 0, c->stream>>>(P, Q, n, sums, terms);
    }
    {
        SG_LAUNCH(c, "kl_reduce");
        reduce_parts_kernel<double><<<1, kPrThreads, 0, c->stream>>>(terms, blocks, tot);
    }
    SG_CUDA(cudaGetLastError());
    SG_CUDA(cudaMemcpyAsync(c->h_pinned, tot, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    SG_CUDA(cudaStreamSynchronize(c->stream));
    std::memcpy(kl, c->h_pinned, sizeof(double));
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

// warp per row; every edge {x < y} hooks the larger root under the smaller
__global__ void cc_hook_kernel(const int64_t *__restrict__ off, const uint32_t *__restrict__ col, int64_t n,
                               uint32_t *parent) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t x = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp; x < n; x += nw) {
        const int64_t b = __ldg(off + x), e = __ldg(off + x + 1);
        for (int64_t i = b + lane; i < e; i += 32) {
            const uint32_t y = __ldg(col + i);
            if (y <= (uint32_t)x) continue;
            uint32_t rx = cc_find(parent, (uint32_t)x), ry = cc_find(parent, y);
            while (rx != ry) {
                const uint32_t hi = rx > ry ? rx : ry, lo = rx > ry ? ry : rx;
                const uint32_t old = atomicCAS(parent + hi, hi, lo);
                if (old == hi) break;
                rx = cc_find(parent, hi);
                ry = cc_find(parent, lo);
            }
        }
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
    if (st == SG_OK) st = dalloc(c, (void **)&roots, sizeof(unsigned long long));
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
        SG_LAUNCH(c, "cc_hook");
        const int hb = (int)std::min<int64_t>((n + 7) / 8, (int64_t)c->num_sms * 8);
        cc_hook_kernel<<<hb, 256, 0, c->stream>>>(g->off, g->col, n, parent);
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
