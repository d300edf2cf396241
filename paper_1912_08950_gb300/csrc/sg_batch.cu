// Batched compression: many independent graphs, each with its own kernel, p and
// seed, compressed by one CUDA-graph launch.
//
// The graphs are packed once into a device-resident disjoint union (vertex and
// arc bases per graph, the graph of every vertex).  Every step of compress()
// then runs once over the whole union -- row maps, degree orientation (only for
// graphs that use a triangle kernel), triangle enumeration with per-graph
// decisions, the final keep/mask compaction with per-graph kernels, and a fix-up
// that turns the union's offsets into per-graph CSRs with local ids.  Random
// keys use each graph's local ids and seed, so every graph's output equals its
// own sg_compress() result bit for bit.  None of these steps synchronises with
// the host, so the sequence is captured once into a CUDA graph and replayed.
// The work-partition knobs (light/heavy out-degree split, CTAs per SM of the
// compaction and enumeration kernels) are chosen by timing each candidate's
// captured graph on the batch itself; the winner is kept with the batch.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "sg_internal.cuh"

namespace sg {

struct PackDesc {
    const int64_t *off;
    const uint32_t *col;
    const float *w;
    int64_t n, nnz, vbase, abase;
};

// blockIdx.y = graph; threads stride over the graph's vertices and arcs
__global__ void batch_pack_kernel(const PackDesc *__restrict__ d, int64_t *off_u, uint32_t *col_u, float *w_u,
                                  uint32_t *vgid) {
    const PackDesc g = d[blockIdx.y];
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (int64_t v = t0; v < g.n; v += stride) {
        off_u[g.vbase + v] = g.abase + g.off[v];
        vgid[g.vbase + v] = blockIdx.y;
    }
    for (int64_t i = t0; i < g.nnz; i += stride) {
        col_u[g.abase + i] = g.col[i] + (uint32_t)g.vbase;
        if (w_u) w_u[g.abase + i] = g.w[i];  // every graph with arcs is weighted here
    }
}

// per-graph local offsets from the union's compacted offsets
__global__ void batch_fix_offsets_kernel(const int64_t *__restrict__ off_c, const uint32_t *__restrict__ vgid,
                                         const BatchParam *__restrict__ P, int64_t n_total, int64_t *out_off) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n_total; v += stride) {
        const uint32_t g = vgid[v];
        out_off[v + g] = off_c[v] - off_c[P[g].vbase];
    }
}

// the closing offset of every graph, and where its arcs start and how many
__global__ void batch_fix_tails_kernel(const int64_t *__restrict__ off_c, const BatchParam *__restrict__ P, int count,
                                       int64_t *out_off, int64_t *info) {
    for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < count; g += gridDim.x * blockDim.x) {
        const int64_t vb = P[g].vbase, n = P[g].n;
        const int64_t base = off_c[vb], end = off_c[vb + n];
        out_off[vb + g + n] = end - base;
        info[2 * g] = base;
        info[2 * g + 1] = end - base;
    }
}

struct Tune {
    int light_max = 64;
    int compact_per_sm = 0;
    int enum_per_sm = 0;
};

struct Batch {
    Ctx *c = nullptr;
    int count = 0;
    Graph u;                       // the union (library-owned)
    uint32_t *vgid = nullptr;
    std::vector<int64_t> n, nnz, vbase, abase;
    BatchParam *d_params = nullptr;
    BatchParam *h_params = nullptr;  // pinned
    // per-call scratch, sized once
    RowMaps rm;
    Oriented o;
    uint8_t *del = nullptr;
    unsigned long long *scan = nullptr;  // chunk-scan status words (orientation, then output)
    CompactScratch final_cs;              // the output compaction's keep masks and chunk prefixes
    uint32_t *delbits = nullptr;          // the deletion flags packed to bits
    BatchTri bt;
    int64_t *off_c = nullptr;      // union offsets after compaction
    int64_t *out_off = nullptr;    // per-graph offsets, n_g + 1 each
    uint32_t *out_col = nullptr;
    float *out_w = nullptr;
    int64_t *d_info = nullptr, *h_info = nullptr;  // (arc start, arc count) per graph
    // captured pipeline
    cudaGraphExec_t exec = nullptr;
    Tune tune;
    bool tuned = false;
    uint64_t launches_per_exec = 0;
    double tuned_ms = 0.0;
};

static sg_status enqueue_pipeline(Batch *b, const Tune &t) {
    Ctx *c = b->c;
    BatchDev dev{b->d_params, b->vgid};
    SG_CUDA(cudaMemcpyAsync(b->d_params, b->h_params, sizeof(BatchParam) * (size_t)b->count,
                            cudaMemcpyHostToDevice, c->stream));
    sg_status st = SG_OK;
    if (b->u.nnz == 0) {
        SG_CUDA(cudaMemsetAsync(b->off_c, 0, sizeof(int64_t) * (size_t)(b->u.n + 1), c->stream));
    } else {
        st = fill_row_maps(c, &b->u, b->rm);
        if (st != SG_OK) return st;
        st = batch_orient(c, &b->u, b->rm, dev, b->o.w != nullptr, &b->o, b->scan, t.compact_per_sm);
        if (st != SG_OK) return st;
        st = reverse_list(c, &b->u, b->rm, b->o, b->bt.inl, dev);
        if (st != SG_OK) return st;
        SG_CUDA(cudaMemsetAsync(b->del, 0, (size_t)std::max<int64_t>(b->u.nnz / 2, 1), c->stream));
        BatchTri bt = b->bt;
        bt.light_max = t.light_max;
        bt.grid_per_sm = t.enum_per_sm;
        st = batch_tr_mark(c, &b->u, b->o, dev, bt, b->del);
        if (st != SG_OK) return st;
        st = batch_final(c, &b->u, b->rm, b->o, dev, b->del, b->delbits, b->off_c, b->out_col, b->u.w, b->out_w,
                         b->final_cs, t.compact_per_sm);
        if (st != SG_OK) return st;
    }
    const int threads = 256;
    const int64_t vb = std::max<int64_t>(1, std::min<int64_t>((b->u.n + threads - 1) / threads, (int64_t)c->num_sms * 8));
    {
        SG_LAUNCH(c, "batch_fix");
        batch_fix_offsets_kernel<<<(unsigned)vb, threads, 0, c->stream>>>(b->off_c, b->vgid, b->d_params, b->u.n,
                                                                         b->out_off);
    }
    {
        SG_LAUNCH(c, "batch_fix");
        batch_fix_tails_kernel<<<(b->count + threads - 1) / threads, threads, 0, c->stream>>>(
            b->off_c, b->d_params, b->count, b->out_off, b->d_info);
    }
    SG_CUDA(cudaGetLastError());
    SG_CUDA(cudaMemcpyAsync(b->h_info, b->d_info, sizeof(int64_t) * 2 * (size_t)b->count, cudaMemcpyDeviceToHost,
                            c->stream));
    return SG_OK;
}

// Capture the pipeline for one tuning into an executable CUDA graph.
static sg_status capture(Batch *b, const Tune &t, cudaGraphExec_t *exec, uint64_t *launches) {
    Ctx *c = b->c;
    // row maps are allocated outside the capture once and rebuilt inside it
    const bool prof = c->profiling;
    c->profiling = false;
    const uint64_t l0 = c->launches;
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeRelaxed);
    sg_status st = (e == cudaSuccess) ? enqueue_pipeline(b, t) : cuda_fail(e, "cudaStreamBeginCapture");
    cudaError_t e2 = cudaStreamEndCapture(c->stream, &graph);
    c->profiling = prof;
    *launches = c->launches - l0;
    c->launches = l0;
    if (st != SG_OK) {
        if (graph) cudaGraphDestroy(graph);
        return st;
    }
    if (e2 != cudaSuccess) return cuda_fail(e2, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
    return SG_OK;
}

static sg_status run_exec(Batch *b, cudaGraphExec_t exec, uint64_t launches) {
    Ctx *c = b->c;
    b->c->launches += launches;
    if (c->profiling) {
        // the whole replay is one timed unit for the profiler
        LaunchScope scope(c, "batch_graph");
        c->launches -= 1;
        SG_CUDA(cudaGraphLaunch(exec, c->stream));
    } else {
        SG_CUDA(cudaGraphLaunch(exec, c->stream));
    }
    return SG_OK;
}

static sg_status autotune(Batch *b) {
    Ctx *c = b->c;
    std::vector<Tune> cands;
    for (int lm : {32, 64})
        for (int cp : {0, 2})
            for (int ep : {0, 2}) cands.push_back(Tune{lm, cp, ep});
    cudaEvent_t e0, e1;
    SG_CUDA(cudaEventCreate(&e0));
    SG_CUDA(cudaEventCreate(&e1));
    double best = 1e30;
    cudaGraphExec_t best_exec = nullptr;
    uint64_t best_launches = 0;
    Tune best_t;
    sg_status st = SG_OK;
    for (const Tune &t : cands) {
        cudaGraphExec_t ex = nullptr;
        uint64_t nl = 0;
        st = capture(b, t, &ex, &nl);
        if (st != SG_OK) break;
        // one warm replay, then the timed median-of-three
        float ms[3] = {0, 0, 0};
        cudaError_t e = cudaGraphLaunch(ex, c->stream);
        for (int r = 0; r < 3 && e == cudaSuccess; ++r) {
            cudaEventRecord(e0, c->stream);
            e = cudaGraphLaunch(ex, c->stream);
            cudaEventRecord(e1, c->stream);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms[r], e0, e1);
        }
        if (e != cudaSuccess) {
            cudaGraphExecDestroy(ex);
            st = cuda_fail(e, "autotune replay");
            break;
        }
        std::sort(ms, ms + 3);
        if (ms[1] < best) {
            if (best_exec) cudaGraphExecDestroy(best_exec);
            best = ms[1];
            best_exec = ex;
            best_launches = nl;
            best_t = t;
        } else {
            cudaGraphExecDestroy(ex);
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != SG_OK) {
        if (best_exec) cudaGraphExecDestroy(best_exec);
        return st;
    }
    if (b->exec) cudaGraphExecDestroy(b->exec);
    b->exec = best_exec;
    b->launches_per_exec = best_launches;
    b->tune = best_t;
    b->tuned = true;
    b->tuned_ms = best;
    return check_device_error(c);
}

}  // namespace sg

using namespace sg;

struct sg_batch : Batch {};
struct sg_graph : Graph {};

extern "C" {

sg_status sg_batch_create(sg_ctx *ctx, int count, const sg_graph *const *graphs, sg_batch **out) {
    if (!ctx || !graphs || !out || count < 1 || count > 65535)
        return fail(SG_ERR_INVALID_ARG, "bad argument (count must be in [1, 65535])");
    *out = nullptr;
    Ctx *c = reinterpret_cast<Ctx *>(ctx);
    SG_CUDA(cudaSetDevice(c->device));
    // graphs without arcs carry no weights either way
    bool weighted = false;
    for (int i = 0; i < count; ++i) {
        if (!graphs[i]) return fail(SG_ERR_INVALID_ARG, "NULL graph");
        if (graphs[i]->nnz > 0 && graphs[i]->w) weighted = true;
    }
    for (int i = 0; i < count; ++i)
        if (graphs[i]->nnz > 0 && (graphs[i]->w != nullptr) != weighted)
            return fail(SG_ERR_INVALID_ARG, "a batch is either all weighted or all unweighted");
    sg_batch *b = new (std::nothrow) sg_batch;
    if (!b) return fail(SG_ERR_OOM, "host allocation failed");
    b->c = c;
    b->count = count;
    int64_t nt = 0, at = 0;
    for (int i = 0; i < count; ++i) {
        b->n.push_back(graphs[i]->n);
        b->nnz.push_back(graphs[i]->nnz);
        b->vbase.push_back(nt);
        b->abase.push_back(at);
        nt += graphs[i]->n;
        at += graphs[i]->nnz;
    }
    sg_status st = SG_OK;
    if (nt >= (int64_t)4294967295ll) st = fail(SG_ERR_UNSUPPORTED, "the union of the batch exceeds 2^32 - 1 vertices");
    Graph &u = b->u;
    u.ctx = c;
    u.device = c->device;
    u.n = nt;
    u.nnz = at;
    u.owned = true;
    PackDesc *d_desc = nullptr;
    if (st == SG_OK) st = dalloc(c, (void **)&u.off, sizeof(int64_t) * (size_t)(nt + 1));
    if (st == SG_OK) st = dalloc(c, (void **)&u.col, sizeof(uint32_t) * (size_t)std::max<int64_t>(at, 1));
    if (st == SG_OK && weighted) st = dalloc(c, (void **)&u.w, sizeof(float) * (size_t)std::max<int64_t>(at, 1));
    if (st == SG_OK) st = dalloc(c, (void **)&b->vgid, sizeof(uint32_t) * (size_t)std::max<int64_t>(nt, 1));
    if (st == SG_OK) st = dalloc(c, (void **)&d_desc, sizeof(PackDesc) * (size_t)count);
    if (st == SG_OK) st = dalloc(c, (void **)&b->d_params, sizeof(BatchParam) * (size_t)count);
    if (st == SG_OK && cudaMallocHost((void **)&b->h_params, sizeof(BatchParam) * (size_t)count) != cudaSuccess)
        st = fail(SG_ERR_OOM, "pinned host allocation failed");
    if (st == SG_OK && cudaMallocHost((void **)&b->h_info, sizeof(int64_t) * 2 * (size_t)count) != cudaSuccess)
        st = fail(SG_ERR_OOM, "pinned host allocation failed");
    std::vector<PackDesc> desc(count);
    if (st == SG_OK) {
        int64_t maxlen = 1;
        for (int i = 0; i < count; ++i) {
            desc[i] = PackDesc{graphs[i]->off, graphs[i]->col, graphs[i]->w, b->n[i], b->nnz[i], b->vbase[i], b->abase[i]};
            maxlen = std::max(maxlen, std::max(b->n[i], b->nnz[i]));
        }
        cudaError_t e = cudaMemcpyAsync(d_desc, desc.data(), sizeof(PackDesc) * (size_t)count, cudaMemcpyHostToDevice,
                                        c->stream);
        if (e == cudaSuccess) {
            dim3 grid((unsigned)std::min<int64_t>((maxlen + 255) / 256, 64), (unsigned)count);
            SG_LAUNCH(c, "batch_pack");
            batch_pack_kernel<<<grid, 256, 0, c->stream>>>(d_desc, u.off, u.col, u.w, b->vgid);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaMemcpyAsync(u.off + nt, &at, sizeof(int64_t), cudaMemcpyHostToDevice, c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) st = cuda_fail(e, "batch packing");
    }
    dfree(c, d_desc);
    // per-call scratch
    const int64_t m = at / 2;
    if (st == SG_OK) {
        b->rm.num_chunks = (at + kWarpSpan - 1) / kWarpSpan;
        Oriented &o = b->o;
        o.n = nt;
        o.m = m;
        st = dalloc(c, (void **)&o.off, sizeof(int64_t) * (size_t)(nt + 1));
        if (st == SG_OK) st = dalloc(c, (void **)&o.col, sizeof(uint32_t) * (size_t)std::max<int64_t>(at, 1));
        if (st == SG_OK && weighted) st = dalloc(c, (void **)&o.w, sizeof(float) * (size_t)std::max<int64_t>(at, 1));
        if (st == SG_OK) st = dalloc(c, (void **)&o.fwd_bits, sizeof(uint32_t) * (size_t)(b->rm.num_chunks * CI + 1));
        if (st == SG_OK) st = dalloc(c, (void **)&o.fwd_excl, sizeof(int64_t) * (size_t)(b->rm.num_chunks + 1));
        if (st == SG_OK)
            st = dalloc(c, (void **)&b->scan,
                        sizeof(unsigned long long) * (size_t)compact_scan_words(b->rm.num_chunks));
        if (st == SG_OK) st = alloc_compact_scratch(c, b->rm.num_chunks, true, &b->final_cs);
        if (st == SG_OK) st = dalloc(c, (void **)&b->del, (size_t)std::max<int64_t>(m, 1));
        if (st == SG_OK)
            st = dalloc(c, (void **)&b->delbits, sizeof(uint32_t) * (size_t)((std::max<int64_t>(m, 1) + 31) / 32));
        if (st == SG_OK) st = dalloc(c, (void **)&b->off_c, sizeof(int64_t) * (size_t)(nt + 1));
        if (st == SG_OK) st = dalloc(c, (void **)&b->out_off, sizeof(int64_t) * (size_t)(nt + count));
        if (st == SG_OK) st = dalloc(c, (void **)&b->out_col, sizeof(uint32_t) * (size_t)std::max<int64_t>(at, 1));
        if (st == SG_OK) st = dalloc(c, (void **)&b->out_w, sizeof(float) * (size_t)std::max<int64_t>(at, 1));
        if (st == SG_OK) st = dalloc(c, (void **)&b->d_info, sizeof(int64_t) * 2 * (size_t)count);
    }
    // the shared-memory plan: orient as if every graph used a triangle kernel
    if (st == SG_OK && at > 0) {
        for (int i = 0; i < count; ++i) {
            BatchParam &P = b->h_params[i];
            std::memset(&P, 0, sizeof(P));
            P.vbase = b->vbase[i];
            P.n = b->n[i];
            P.kernel = (int)SG_TR_RANDOM;
        }
        SG_CUDA(cudaMemcpyAsync(b->d_params, b->h_params, sizeof(BatchParam) * (size_t)count, cudaMemcpyHostToDevice,
                                c->stream));
        RowMaps rm;
        st = build_row_maps(c, &u, &rm);
        if (st == SG_OK) {
            b->rm.chunk_row = rm.chunk_row;
        }
        if (st == SG_OK)
            st = batch_orient(c, &u, b->rm, BatchDev{b->d_params, b->vgid}, false, &b->o, b->scan, 0);
        if (st == SG_OK) st = batch_tr_prepare(c, &u, b->o, &b->bt);
        if (st == SG_OK) b->o.inl = b->bt.inl;  // the mask resolution reads the batch's reverse list
        if (st == SG_OK) st = check_device_error(c);
    }
    if (st != SG_OK) {
        sg_batch_free(b);
        return st;
    }
    *out = b;
    return SG_OK;
}

void sg_batch_free(sg_batch *b) {
    if (!b) return;
    Ctx *c = b->c;
    if (!ctx_alive(c)) {
        // the context is gone: release synchronously, without its stream
        (void)cudaSetDevice(b->u.device);
        if (b->exec) cudaGraphExecDestroy(b->exec);
        for (void *p : {(void *)b->u.off, (void *)b->u.col, (void *)b->u.w, (void *)b->vgid, (void *)b->d_params,
                        (void *)b->rm.chunk_row, (void *)b->o.off, (void *)b->o.col, (void *)b->o.w,
                        (void *)b->o.fwd_bits, (void *)b->o.fwd_excl, (void *)b->scan, (void *)b->final_cs.keep,
                        (void *)b->final_cs.cexcl, (void *)b->final_cs.scan, (void *)b->delbits,
                        (void *)b->del, (void *)b->bt.heavy, (void *)b->bt.buckets, (void *)b->bt.din,
                        (void *)b->bt.inl, (void *)b->off_c,
                        (void *)b->out_off, (void *)b->out_col, (void *)b->out_w, (void *)b->d_info})
            if (p) (void)cudaFree(p);
        if (b->h_params) cudaFreeHost(b->h_params);
        if (b->h_info) cudaFreeHost(b->h_info);
        delete b;
        return;
    }
    (void)cudaSetDevice(c->device);
    (void)cudaStreamSynchronize(c->stream);
    if (b->exec) cudaGraphExecDestroy(b->exec);
    dfree(c, b->u.off);
    dfree(c, b->u.col);
    dfree(c, b->u.w);
    dfree(c, b->vgid);
    dfree(c, b->d_params);
    free_row_maps(c, &b->rm);
    b->o.inl = nullptr;  // owned by b->bt, freed below
    free_oriented(c, &b->o);
    dfree(c, b->scan);
    free_compact_scratch(c, &b->final_cs);
    dfree(c, b->delbits);
    dfree(c, b->del);
    batch_tr_free(c, &b->bt);
    dfree(c, b->off_c);
    dfree(c, b->out_off);
    dfree(c, b->out_col);
    dfree(c, b->out_w);
    dfree(c, b->d_info);
    if (b->h_params) cudaFreeHost(b->h_params);
    if (b->h_info) cudaFreeHost(b->h_info);
    (void)cudaStreamSynchronize(c->stream);
    delete b;
}

sg_status sg_compress_batch(sg_ctx *ctx, sg_batch *b, const sg_kernel *kernels, const double *ps,
                            const uint64_t *seeds, int want_weights, sg_graph **outs) {
    if (!ctx || !b || !kernels || !ps || !seeds || !outs) return fail(SG_ERR_INVALID_ARG, "NULL argument");
    Ctx *c = reinterpret_cast<Ctx *>(ctx);
    if (c != b->c) return fail(SG_ERR_INVALID_ARG, "the batch belongs to another context");
    SG_CUDA(cudaSetDevice(c->device));
    for (int i = 0; i < b->count; ++i) {
        const int k = (int)kernels[i];
        if (!(ps[i] >= 0.0 && ps[i] <= 1.0)) return fail(SG_ERR_INVALID_ARG, "p must lie in [0, 1]");
        if (k < (int)SG_UNIFORM || k > (int)SG_TR_EO_MINCOUNT) return fail(SG_ERR_INVALID_ARG, "unknown kernel");
        if (k == (int)SG_TR_EO || k == (int)SG_TR_EO_MAXW || k == (int)SG_TR_EO_MINCOUNT)
            return fail(SG_ERR_UNSUPPORTED, "edge-once kernels need host-driven rounds; use sg_compress");
        if (k == (int)SG_TR_MINCOUNT)
            return fail(SG_ERR_UNSUPPORTED, "the min-count kernel needs a counting pass; use sg_compress");
        if (k == (int)SG_TR_MAXW && !b->u.w && b->nnz[i] > 0)
            return fail(SG_ERR_NEEDS_WEIGHTS, "the max-weight kernel needs weights");
    }
    SG_CUDA(cudaStreamSynchronize(c->stream));  // the pinned parameters may still be read by a replay
    for (int i = 0; i < b->count; ++i) {
        BatchParam &P = b->h_params[i];
        std::memset(&P, 0, sizeof(P));
        P.vbase = b->vbase[i];
        P.n = b->n[i];
        P.kernel = (int)kernels[i];
        P.k0 = (uint32_t)(seeds[i] & 0xFFFFFFFFu);
        P.k1 = (uint32_t)(seeds[i] >> 32);
        P.tp = prob_threshold(ps[i]);
        if (kernels[i] == SG_SPECTRAL_LOGN || kernels[i] == SG_SPECTRAL_AVGDEG) {
            const double m = (double)(b->nnz[i] / 2), n = (double)b->n[i];
            const double y = (kernels[i] == SG_SPECTRAL_LOGN) ? ps[i] * std::log(n) : (n > 0 ? ps[i] * m / n : 0.0);
            const double t = std::floor(y * 4294967296.0);
            P.ty = t >= 18446744073709551615.0 ? UINT64_MAX : (t <= 0.0 ? 0ull : (unsigned long long)t);
            P.yf = (float)y;
            P.reweight = want_weights ? 1 : 0;
        }
    }
    sg_status st = SG_OK;
    if (!b->tuned) st = autotune(b);
    if (st == SG_OK) st = run_exec(b, b->exec, b->launches_per_exec);
    if (st == SG_OK) {
        cudaError_t e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) st = cuda_fail(e, "batch replay");
    }
    if (st == SG_OK) st = check_device_error(c);
    if (st != SG_OK) return st;
    const bool out_w = b->u.w != nullptr || want_weights;
    for (int i = 0; i < b->count; ++i) {
        sg_graph *g = new (std::nothrow) sg_graph;
        if (!g) {
            for (int j = 0; j < i; ++j) {
                delete outs[j];
                outs[j] = nullptr;
            }
            return fail(SG_ERR_OOM, "host allocation failed");
        }
        const int64_t a0 = b->h_info[2 * i], na = b->h_info[2 * i + 1];
        g->ctx = c;
        g->device = c->device;
        g->n = b->n[i];
        g->nnz = na;
        g->off = b->out_off + b->vbase[i] + i;
        g->col = b->out_col + a0;
        const bool spectral = kernels[i] == SG_SPECTRAL_LOGN || kernels[i] == SG_SPECTRAL_AVGDEG;
        g->w = (b->u.w != nullptr || (want_weights && spectral)) && out_w ? b->out_w + a0 : nullptr;
        g->owned = false;
        outs[i] = g;
    }
    return SG_OK;
}

sg_status sg_batch_info(const sg_batch *b, int64_t *vertices, int64_t *arcs, int *light_max, int *compact_per_sm,
                        int *enum_per_sm, double *tuned_ms) {
    if (!b) return fail(SG_ERR_INVALID_ARG, "NULL batch");
    if (vertices) *vertices = b->u.n;
    if (arcs) *arcs = b->u.nnz;
    if (light_max) *light_max = b->tune.light_max;
    if (compact_per_sm) *compact_per_sm = b->tune.compact_per_sm;
    if (enum_per_sm) *enum_per_sm = b->tune.enum_per_sm;
    if (tuned_ms) *tuned_ms = b->tuned_ms;
    return SG_OK;
}

}  // extern "C"
