// The extern "C" boundary of the library: contexts, graphs, error reporting,
// launch accounting and the dispatch of compress / divergence to the kernels.
#include <cmath>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <unordered_set>

#include "sg_internal.cuh"

namespace sg {

static thread_local std::string g_last_error;

// Contexts that are alive: a graph freed after its context was destroyed
// must not touch the context's (freed) stream.
static std::mutex g_ctx_mutex;
static std::unordered_set<const Ctx *> g_live_ctx;

bool ctx_alive(const Ctx *c) {
    std::lock_guard<std::mutex> lock(g_ctx_mutex);
    return g_live_ctx.count(c) != 0;
}

void set_error(const std::string &msg) { g_last_error = msg; }

sg_status fail(sg_status st, const std::string &msg) {
    g_last_error = msg;
    return st;
}

sg_status cuda_fail(cudaError_t e, const char *what) {
    g_last_error = std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
    if (e == cudaErrorMemoryAllocation) return SG_ERR_OOM;
    return SG_ERR_CUDA;
}

sg_status dalloc(Ctx *c, void **p, size_t bytes) {
    *p = nullptr;
    if (bytes == 0) bytes = 16;
    cudaError_t e = cudaMallocAsync(p, bytes, c->stream);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        *p = nullptr;
        return fail(e == cudaErrorMemoryAllocation ? SG_ERR_OOM : SG_ERR_CUDA,
                    std::string("device allocation of ") + std::to_string(bytes) + " bytes failed: " +
                        cudaGetErrorString(e));
    }
    return SG_OK;
}

void dfree(Ctx *c, void *p) {
    if (p) (void)cudaFreeAsync(p, c->stream);
}

sg_status ws_get(Ctx *c, int slot, size_t bytes, void **p) {
    if (c->ws[slot] && c->ws_bytes[slot] >= bytes) {
        *p = c->ws[slot];
        return SG_OK;
    }
    dfree(c, c->ws[slot]);
    c->ws[slot] = nullptr;
    c->ws_bytes[slot] = 0;
    // a quarter more than asked: list fills vary a little from call to call
    // (the order in which warps claim chunks), and each regrowth maps new memory
    size_t want = bytes + bytes / 4;
    if (dalloc(c, p, want) != SG_OK) {
        want = bytes;
        set_error("");
        sg_status st = dalloc(c, p, want);
        if (st != SG_OK) return st;
    }
    c->ws[slot] = *p;
    c->ws_bytes[slot] = want;
    return SG_OK;
}

static cudaEvent_t take_event(Ctx *c) {
    if (!c->event_pool.empty()) {
        cudaEvent_t e = c->event_pool.back();
        c->event_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
}

LaunchScope::LaunchScope(Ctx *c_, const char *n_) : c(c_), name(n_) {
    ++c->launches;
    if (c->profiling) {
        b = take_event(c);
        e = take_event(c);
        if (b && e) cudaEventRecord(b, c->stream);
    }
}

LaunchScope::~LaunchScope() {
    if (c->profiling && b && e) {
        cudaEventRecord(e, c->stream);
        c->prof.push_back(ProfRec{name, b, e});
    }
}

sg_status check_device_error(Ctx *c) {
    SG_CUDA(cudaMemcpyAsync(c->h_pinned, c->d_err, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    SG_CUDA(cudaStreamSynchronize(c->stream));
    int code = 0;
    std::memcpy(&code, c->h_pinned, sizeof(int));
    if (code == kDevOk) return SG_OK;
    SG_CUDA(cudaMemsetAsync(c->d_err, 0, sizeof(int), c->stream));
    switch (code) {
    case kDevLookbackTimeout:
        return fail(SG_ERR_TIMEOUT, "a device-side wait of the prefix scan gave up; outputs are invalid");
    case kDevBadGraph:
        return fail(SG_ERR_INVALID_GRAPH, "the CSR failed validation");
    case kDevTableFull:
        return fail(SG_ERR_CUDA, "a shared-memory cuckoo table overflowed its stash; outputs are invalid");
    default:
        return fail(SG_ERR_CUDA, "device error code " + std::to_string(code));
    }
}

static sg_status compress_tr(Ctx *c, const Graph *g, sg_kernel k, double p, uint64_t seed, Graph **out) {
    const bool maxw = (k == SG_TR_MAXW || k == SG_TR_EO_MAXW);
    RowMaps rm;
    Oriented o;
    uint8_t *del = nullptr;
    sg_status st = build_row_maps(c, g, &rm);
    if (st == SG_OK) st = orient(c, g, rm, maxw, &o);
    if (st == SG_OK) st = dalloc(c, (void **)&del, (size_t)std::max<int64_t>(o.m, 1));
    if (st == SG_OK) {
        cudaError_t e = cudaMemsetAsync(del, 0, (size_t)std::max<int64_t>(o.m, 1), c->stream);
        if (e != cudaSuccess) st = cuda_fail(e, "cudaMemsetAsync(del)");
    }
    if (st == SG_OK) st = tr_mark(c, g, o, k, p, seed, del);
    if (st == SG_OK) st = resolve_mask(c, g, rm, o, del, out);
    dfree(c, del);
    free_oriented(c, &o);
    free_row_maps(c, &rm);
    return st;
}

}  // namespace sg

using namespace sg;

struct sg_ctx : Ctx {};
struct sg_graph : Graph {};

static Ctx *C_(sg_ctx *c) { return static_cast<Ctx *>(c); }
static const Graph *G_(const sg_graph *g) { return static_cast<const Graph *>(g); }

static sg_status set_device(Ctx *c) {
    SG_CUDA(cudaSetDevice(c->device));
    return SG_OK;
}

extern "C" {

const char *sg_last_error(void) { return g_last_error.c_str(); }

sg_status sg_ctx_create(int device, void *cuda_stream, sg_ctx **out) {
    if (!out) return fail(SG_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    int ndev = 0;
    SG_CUDA(cudaGetDeviceCount(&ndev));
    if (device < 0 || device >= ndev) return fail(SG_ERR_INVALID_ARG, "no such CUDA device");
    SG_CUDA(cudaSetDevice(device));
    sg_ctx *c = new (std::nothrow) sg_ctx;
    if (!c) return fail(SG_ERR_OOM, "host allocation failed");
    c->device = device;
    cudaError_t e = cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device);
    if (e == cudaSuccess) {
        if (cuda_stream) {
            c->stream = static_cast<cudaStream_t>(cuda_stream);
        } else {
            e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
            c->own_stream = (e == cudaSuccess);
        }
    }
    if (e == cudaSuccess) e = cudaMalloc((void **)&c->d_err, sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc((void **)&c->d_ctr, sizeof(unsigned long long) * kCtrCount);
    if (e == cudaSuccess) e = cudaMallocHost((void **)&c->h_pinned, 4096);
    if (e == cudaSuccess) e = cudaMemset(c->d_err, 0, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(c->d_ctr, 0, sizeof(unsigned long long) * kCtrCount);
    if (e == cudaSuccess) {
        // keep freed stream-ordered memory in the pool between calls
        cudaMemPool_t pool;
        if (cudaDeviceGetDefaultMemPool(&pool, device) == cudaSuccess) {
            uint64_t thr = UINT64_MAX;
            (void)cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
        }
    }
    if (e != cudaSuccess) {
        sg_status st = cuda_fail(e, "context setup");
        sg_ctx_destroy(c);
        return st;
    }
    {
        std::lock_guard<std::mutex> lock(g_ctx_mutex);
        g_live_ctx.insert(c);
    }
    *out = c;
    return SG_OK;
}

void sg_ctx_destroy(sg_ctx *ctx) {
    if (!ctx) return;
    Ctx *c = C_(ctx);
    {
        std::lock_guard<std::mutex> lock(g_ctx_mutex);
        g_live_ctx.erase(c);
    }
    (void)cudaSetDevice(c->device);
    for (int i = 0; i < 3; ++i) dfree(c, c->ws[i]);
    if (c->stream) (void)cudaStreamSynchronize(c->stream);
    for (auto &r : c->prof) {
        (void)cudaEventDestroy(r.beg);
        (void)cudaEventDestroy(r.end);
    }
    for (auto e : c->event_pool) (void)cudaEventDestroy(e);
    if (c->d_err) (void)cudaFree(c->d_err);
    if (c->d_ctr) (void)cudaFree(c->d_ctr);
    if (c->h_pinned) (void)cudaFreeHost(c->h_pinned);
    if (c->own_stream) (void)cudaStreamDestroy(c->stream);
    delete ctx;
}

sg_status sg_ctx_synchronize(sg_ctx *ctx) {
    if (!ctx) return fail(SG_ERR_INVALID_ARG, "ctx is NULL");
    SG_CUDA(cudaStreamSynchronize(C_(ctx)->stream));
    return SG_OK;
}

sg_status sg_ctx_stats(sg_ctx *ctx, sg_stats *out, int reset) {
    if (!ctx || !out) return fail(SG_ERR_INVALID_ARG, "NULL argument");
    Ctx *c = C_(ctx);
    sg_status st = set_device(c);
    if (st != SG_OK) return st;
    SG_CUDA(cudaMemcpyAsync(c->h_pinned, c->d_ctr, sizeof(unsigned long long) * 2, cudaMemcpyDeviceToHost,
                            c->stream));
    SG_CUDA(cudaStreamSynchronize(c->stream));
    unsigned long long v[2];
    std::memcpy(v, c->h_pinned, sizeof(v));
    out->kernel_launches = c->launches;
    out->probes = v[kCtrProbes];
    out->triangles = v[kCtrTriangles];
    out->eo_rounds = c->eo_rounds;
    out->eo_listed = c->eo_listed;
    out->eo_passes = c->eo_passes;
    out->eo_list_passes = c->eo_list_passes;
    if (reset) {
        c->launches = 0;
        c->eo_rounds = 0;
        c->eo_listed = 0;
        c->eo_passes = 0;
        c->eo_list_passes = 0;
        SG_CUDA(cudaMemsetAsync(c->d_ctr, 0, sizeof(unsigned long long) * 2, c->stream));
        SG_CUDA(cudaStreamSynchronize(c->stream));
    }
    return SG_OK;
}

sg_status sg_ctx_set_profiling(sg_ctx *ctx, int on) {
    if (!ctx) return fail(SG_ERR_INVALID_ARG, "ctx is NULL");
    C_(ctx)->profiling = on != 0;
    return SG_OK;
}

sg_status sg_ctx_set_eo_list_capacity(sg_ctx *ctx, int64_t records) {
    if (!ctx || records < -1) return fail(SG_ERR_INVALID_ARG, "bad argument");
    C_(ctx)->eo_list_cap = records;
    return SG_OK;
}

sg_status sg_ctx_release_workspace(sg_ctx *ctx) {
    if (!ctx) return fail(SG_ERR_INVALID_ARG, "ctx is NULL");
    Ctx *c = C_(ctx);
    sg_status st = set_device(c);
    if (st != SG_OK) return st;
    for (int i = 0; i < 3; ++i) {
        dfree(c, c->ws[i]);
        c->ws[i] = nullptr;
        c->ws_bytes[i] = 0;
    }
    return SG_OK;
}

sg_status sg_ctx_set_scan_hold(sg_ctx *ctx, uint32_t spin_limit) {
    if (!ctx) return fail(SG_ERR_INVALID_ARG, "ctx is NULL");
    C_(ctx)->scan_hold = spin_limit;
    return SG_OK;
}

sg_status sg_device_free_memory(int device, uint64_t *free_out) {
    if (!free_out) return fail(SG_ERR_INVALID_ARG, "free_out is NULL");
    int ndev = 0, prev = 0;
    SG_CUDA(cudaGetDeviceCount(&ndev));
    if (device < 0 || device >= ndev) return fail(SG_ERR_INVALID_ARG, "no such device");
    SG_CUDA(cudaGetDevice(&prev));
    SG_CUDA(cudaSetDevice(device));
    size_t fr = 0, tot = 0;
    cudaError_t e = cudaMemGetInfo(&fr, &tot);
    uint64_t total = fr;
    cudaMemPool_t pool;
    if (e == cudaSuccess && cudaDeviceGetDefaultMemPool(&pool, device) == cudaSuccess) {
        // memory the stream-ordered pool keeps from freed allocations is free too
        uint64_t reserved = 0, used = 0;
        if (cudaMemPoolGetAttribute(pool, cudaMemPoolAttrReservedMemCurrent, &reserved) == cudaSuccess &&
            cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemCurrent, &used) == cudaSuccess && reserved > used)
            total += reserved - used;
    }
    (void)cudaSetDevice(prev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemGetInfo");
    *free_out = total;
    return SG_OK;
}

sg_status sg_ctx_kernel_time(sg_ctx *ctx, const char *prefix, double *ms, int64_t *launches) {
    if (!ctx || !prefix || !ms || !launches) return fail(SG_ERR_INVALID_ARG, "NULL argument");
    Ctx *c = C_(ctx);
    SG_CUDA(cudaStreamSynchronize(c->stream));
    double total = 0.0;
    int64_t count = 0;
    const size_t plen = std::strlen(prefix);
    for (auto &r : c->prof) {
        if (std::strncmp(r.name, prefix, plen) != 0) continue;
        float t = 0.f;
        SG_CUDA(cudaEventElapsedTime(&t, r.beg, r.end));
        total += t;
        ++count;
    }
    *ms = total;
    *launches = count;
    return SG_OK;
}

sg_status sg_ctx_reset_profile(sg_ctx *ctx) {
    if (!ctx) return fail(SG_ERR_INVALID_ARG, "ctx is NULL");
    Ctx *c = C_(ctx);
    SG_CUDA(cudaStreamSynchronize(c->stream));
    for (auto &r : c->prof) {
        c->event_pool.push_back(r.beg);
        c->event_pool.push_back(r.end);
    }
    c->prof.clear();
    return SG_OK;
}

sg_status sg_graph_from_device(sg_ctx *ctx, const sg_csr_view *in, int copy, int validate, sg_graph **out) {
    if (!ctx || !in || !out) return fail(SG_ERR_INVALID_ARG, "NULL argument");
    *out = nullptr;
    if (in->n < 0 || in->nnz < 0) return fail(SG_ERR_INVALID_ARG, "negative size");
    if (in->n >= (int64_t)4294967295ll) return fail(SG_ERR_UNSUPPORTED, "n >= 2^32 - 1: ids are uint32");
    if (!in->off || (in->nnz > 0 && !in->col)) return fail(SG_ERR_INVALID_ARG, "NULL CSR array");
    if (in->nnz % 2) return fail(SG_ERR_INVALID_GRAPH, "a symmetric CSR has an even arc count");
    if (in->n == 0 && in->nnz > 0) return fail(SG_ERR_INVALID_GRAPH, "arcs without vertices");
    Ctx *c = C_(ctx);
    sg_status st = set_device(c);
    if (st != SG_OK) return st;
    sg_graph *g = new (std::nothrow) sg_graph;
    if (!g) return fail(SG_ERR_OOM, "host allocation failed");
    g->ctx = c;
    g->device = c->device;
    g->n = in->n;
    g->nnz = in->nnz;
    if (!copy) {
        g->owned = false;
        g->off = const_cast<int64_t *>(in->off);
        g->col = const_cast<uint32_t *>(in->col);
        g->w = const_cast<float *>(in->w);
    } else {
        g->owned = true;
        st = dalloc(c, (void **)&g->off, sizeof(int64_t) * (size_t)(in->n + 1));
        if (st == SG_OK) st = dalloc(c, (void **)&g->col, sizeof(uint32_t) * (size_t)std::max<int64_t>(in->nnz, 1));
        if (st == SG_OK && in->w) st = dalloc(c, (void **)&g->w, sizeof(float) * (size_t)std::max<int64_t>(in->nnz, 1));
        if (st == SG_OK) {
            cudaError_t e = cudaMemcpyAsync(g->off, in->off, sizeof(int64_t) * (size_t)(in->n + 1),
                                            cudaMemcpyDeviceToDevice, c->stream);
            if (e == cudaSuccess && in->nnz)
                e = cudaMemcpyAsync(g->col, in->col, sizeof(uint32_t) * (size_t)in->nnz, cudaMemcpyDeviceToDevice,
                                    c->stream);
            if (e == cudaSuccess && in->w && in->nnz)
                e = cudaMemcpyAsync(g->w, in->w, sizeof(float) * (size_t)in->nnz, cudaMemcpyDeviceToDevice, c->stream);
            if (e != cudaSuccess) st = cuda_fail(e, "graph copy");
        }
    }
    if (st == SG_OK && validate) st = validate_graph(c, g);
    if (st != SG_OK) {
        sg_graph_free(g);
        return st;
    }
    *out = g;
    return SG_OK;
}

sg_status sg_graph_from_host(sg_ctx *ctx, int64_t n, int64_t nnz, const int64_t *off, const uint32_t *col,
                             const float *w, sg_graph **out) {
    if (!ctx || !out || !off || (nnz > 0 && !col)) return fail(SG_ERR_INVALID_ARG, "NULL argument");
    *out = nullptr;
    if (n < 0 || nnz < 0) return fail(SG_ERR_INVALID_ARG, "negative size");
    if (n >= (int64_t)4294967295ll) return fail(SG_ERR_UNSUPPORTED, "n >= 2^32 - 1: ids are uint32");
    if (nnz % 2) return fail(SG_ERR_INVALID_GRAPH, "a symmetric CSR has an even arc count");
    if (n == 0 && nnz > 0) return fail(SG_ERR_INVALID_GRAPH, "arcs without vertices");
    Ctx *c = C_(ctx);
    sg_status st = set_device(c);
    if (st != SG_OK) return st;
    sg_graph *g = new (std::nothrow) sg_graph;
    if (!g) return fail(SG_ERR_OOM, "host allocation failed");
    g->ctx = c;
    g->device = c->device;
    g->n = n;
    g->nnz = nnz;
    g->owned = true;
    st = dalloc(c, (void **)&g->off, sizeof(int64_t) * (size_t)(n + 1));
    if (st == SG_OK) st = dalloc(c, (void **)&g->col, sizeof(uint32_t) * (size_t)std::max<int64_t>(nnz, 1));
    if (st == SG_OK && w) st = dalloc(c, (void **)&g->w, sizeof(float) * (size_t)std::max<int64_t>(nnz, 1));
    if (st == SG_OK) {
        cudaError_t e = cudaMemcpyAsync(g->off, off, sizeof(int64_t) * (size_t)(n + 1), cudaMemcpyHostToDevice,
                                        c->stream);
        if (e == cudaSuccess && nnz)
            e = cudaMemcpyAsync(g->col, col, sizeof(uint32_t) * (size_t)nnz, cudaMemcpyHostToDevice, c->stream);
        if (e == cudaSuccess && w && nnz)
            e = cudaMemcpyAsync(g->w, w, sizeof(float) * (size_t)nnz, cudaMemcpyHostToDevice, c->stream);
        if (e != cudaSuccess) st = cuda_fail(e, "graph upload");
    }
    if (st != SG_OK) {
        sg_graph_free(g);
        return st;
    }
    *out = g;
    return SG_OK;
}

sg_status sg_graph_view(const sg_graph *g, sg_csr_view *out) {
    if (!g || !out) return fail(SG_ERR_INVALID_ARG, "NULL argument");
    out->n = g->n;
    out->nnz = g->nnz;
    out->off = g->off;
    out->col = g->col;
    out->w = g->w;
    return SG_OK;
}

sg_status sg_graph_download(sg_ctx *ctx, const sg_graph *g, int64_t *off, uint32_t *col, float *w) {
    if (!ctx || !g || !off || (g->nnz > 0 && !col)) return fail(SG_ERR_INVALID_ARG, "NULL argument");
    Ctx *c = C_(ctx);
    sg_status st = set_device(c);
    if (st != SG_OK) return st;
    SG_CUDA(cudaMemcpyAsync(off, g->off, sizeof(int64_t) * (size_t)(g->n + 1), cudaMemcpyDeviceToHost, c->stream));
    if (g->nnz)
        SG_CUDA(cudaMemcpyAsync(col, g->col, sizeof(uint32_t) * (size_t)g->nnz, cudaMemcpyDeviceToHost, c->stream));
    if (w && g->w && g->nnz)
        SG_CUDA(cudaMemcpyAsync(w, g->w, sizeof(float) * (size_t)g->nnz, cudaMemcpyDeviceToHost, c->stream));
    SG_CUDA(cudaStreamSynchronize(c->stream));
    return SG_OK;
}

void sg_graph_free(sg_graph *g) {
    if (!g) return;
    if (g->owned && g->ctx) {
        Ctx *c = g->ctx;
        if (ctx_alive(c)) {
            (void)cudaSetDevice(c->device);
            dfree(c, g->off);
            dfree(c, g->col);
            dfree(c, g->w);
        } else {
            // the context is gone: free synchronously, without its stream
            (void)cudaSetDevice(g->device);
            for (void *p : {(void *)g->off, (void *)g->col, (void *)g->w})
                if (p) (void)cudaFree(p);
        }
    }
    delete g;
}

sg_status sg_compress(sg_ctx *ctx, const sg_graph *g, sg_kernel kernel, double p, uint64_t seed, int want_weights,
                      sg_graph **out) {
    if (!ctx || !g || !out) return fail(SG_ERR_INVALID_ARG, "NULL argument");
    *out = nullptr;
    if (!(p >= 0.0 && p <= 1.0)) return fail(SG_ERR_INVALID_ARG, "p must lie in [0, 1]");
    if ((int)kernel < (int)SG_UNIFORM || (int)kernel > (int)SG_TR_EO_MINCOUNT)
        return fail(SG_ERR_INVALID_ARG, "unknown kernel");
    if ((kernel == SG_TR_MAXW || kernel == SG_TR_EO_MAXW) && !g->w && g->nnz > 0)
        return fail(SG_ERR_NEEDS_WEIGHTS, "the max-weight kernels need edge weights");
    Ctx *c = C_(ctx);
    sg_status st = set_device(c);
    if (st != SG_OK) return st;
    Graph *h = nullptr;
    if (kernel == SG_UNIFORM || kernel == SG_SPECTRAL_LOGN || kernel == SG_SPECTRAL_AVGDEG)
        st = compress_edges(c, G_(g), kernel, p, seed, want_weights, &h);
    else
        st = compress_tr(c, G_(g), kernel, p, seed, &h);
    if (st != SG_OK) return st;
    sg_graph *r = new (std::nothrow) sg_graph;
    if (!r) {
        dfree(c, h->off);
        dfree(c, h->col);
        dfree(c, h->w);
        delete h;
        return fail(SG_ERR_OOM, "host allocation failed");
    }
    static_cast<Graph &>(*r) = *h;
    delete h;
    *out = r;
    return SG_OK;
}

sg_status sg_pagerank(sg_ctx *ctx, const sg_graph *g, float damping, int iters, float *x_out, double *residual_out) {
    if (!ctx || !g || (!x_out && g->n > 0)) return fail(SG_ERR_INVALID_ARG, "NULL argument");
    if (iters < 1 || !(damping >= 0.f && damping <= 1.f)) return fail(SG_ERR_INVALID_ARG, "bad PageRank parameters");
    Ctx *c = C_(ctx);
    sg_status st = set_device(c);
    if (st != SG_OK) return st;
    double r = 0.0;
    st = pagerank(c, G_(g), damping, iters, x_out, &r);
    if (st == SG_OK) st = check_device_error(c);
    if (residual_out) *residual_out = r;
    return st;
}

sg_status sg_kl_divergence(sg_ctx *ctx, int64_t n, const float *P, const float *Q, double *kl_out) {
    if (!ctx || !kl_out || (n > 0 && (!P || !Q)) || n < 0) return fail(SG_ERR_INVALID_ARG, "bad argument");
    Ctx *c = C_(ctx);
    sg_status st = set_device(c);
    if (st != SG_OK) return st;
    return kl_divergence(c, n, P, Q, kl_out);
}

sg_status sg_cc_count(sg_ctx *ctx, const sg_graph *g, int64_t *count_out, uint32_t *labels_out) {
    if (!ctx || !g || !count_out) return fail(SG_ERR_INVALID_ARG, "NULL argument");
    Ctx *c = C_(ctx);
    sg_status st = set_device(c);
    if (st != SG_OK) return st;
    return cc_count(c, G_(g), count_out, labels_out);
}

sg_status sg_divergence(sg_ctx *ctx, const sg_graph *g, const sg_graph *h, float damping, int iters,
                        sg_div_result *out) {
    if (!ctx || !g || !h || !out) return fail(SG_ERR_INVALID_ARG, "NULL argument");
    if (g->n != h->n) return fail(SG_ERR_INVALID_ARG, "G and H must have the same vertex count");
    if (iters < 1 || !(damping >= 0.f && damping <= 1.f)) return fail(SG_ERR_INVALID_ARG, "bad PageRank parameters");
    Ctx *c = C_(ctx);
    sg_status st = set_device(c);
    if (st != SG_OK) return st;
    float *P = nullptr, *Q = nullptr;
    st = dalloc(c, (void **)&P, sizeof(float) * (size_t)std::max<int64_t>(g->n, 1));
    if (st == SG_OK) st = dalloc(c, (void **)&Q, sizeof(float) * (size_t)std::max<int64_t>(g->n, 1));
    if (st == SG_OK) st = pagerank(c, G_(g), damping, iters, P, &out->pr_residual_g);
    if (st == SG_OK) st = pagerank(c, G_(h), damping, iters, Q, &out->pr_residual_h);
    if (st == SG_OK) st = kl_divergence(c, g->n, P, Q, &out->kl_bits);
    if (st == SG_OK) st = cc_count(c, G_(g), &out->cc_g, nullptr);
    if (st == SG_OK) st = cc_count(c, G_(h), &out->cc_h, nullptr);
    if (st == SG_OK) st = check_device_error(c);
    out->m_g = g->nnz / 2;
    out->m_h = h->nnz / 2;
    dfree(c, P);
    dfree(c, Q);
    return st;
}

sg_status sg_bfs_levels(sg_ctx *ctx, const sg_graph *g, int64_t root, int32_t *levels) {
    if (!ctx || !g || (!levels && g->n > 0)) return fail(SG_ERR_INVALID_ARG, "NULL argument");
    if (root < 0 || root >= g->n) return fail(SG_ERR_INVALID_ARG, "root out of range");
    Ctx *c = C_(ctx);
    sg_status st = set_device(c);
    if (st == SG_OK) st = bfs_levels(c, G_(g), root, reinterpret_cast<int *>(levels));
    if (st == SG_OK) st = check_device_error(c);
    return st;
}

sg_status sg_critical_edges(sg_ctx *ctx, const sg_graph *g, int64_t root, int64_t *count_out) {
    if (!ctx || !g || !count_out) return fail(SG_ERR_INVALID_ARG, "NULL argument");
    if (root < 0 || root >= g->n) return fail(SG_ERR_INVALID_ARG, "root out of range");
    Ctx *c = C_(ctx);
    sg_status st = set_device(c);
    if (st == SG_OK) st = critical_edges(c, G_(g), root, count_out);
    if (st == SG_OK) st = check_device_error(c);
    return st;
}

sg_status sg_reordered_neighbours(sg_ctx *ctx, const sg_graph *g, const float *x, const float *y,
                                  int64_t *count_out) {
    if (!ctx || !g || !count_out || ((!x || !y) && g->n > 0)) return fail(SG_ERR_INVALID_ARG, "NULL argument");
    Ctx *c = C_(ctx);
    sg_status st = set_device(c);
    if (st == SG_OK) st = reordered_neighbours<float>(c, G_(g), x, y, count_out);
    if (st == SG_OK) st = check_device_error(c);
    return st;
}

sg_status sg_vertex_triangle_counts(sg_ctx *ctx, const sg_graph *g, uint64_t *counts) {
    if (!ctx || !g || (!counts && g->n > 0)) return fail(SG_ERR_INVALID_ARG, "NULL argument");
    Ctx *c = C_(ctx);
    sg_status st = set_device(c);
    if (st != SG_OK) return st;
    RowMaps rm;
    Oriented o;
    st = build_row_maps(c, G_(g), &rm);
    if (st == SG_OK) st = orient(c, G_(g), rm, false, &o);
    if (st == SG_OK) st = tr_vertex_counts(c, G_(g), o, reinterpret_cast<unsigned long long *>(counts));
    if (st == SG_OK) st = check_device_error(c);
    free_oriented(c, &o);
    free_row_maps(c, &rm);
    return st;
}

sg_status sg_accuracy(sg_ctx *ctx, const sg_graph *g, const sg_graph *h, float damping, int iters, int64_t root,
                      sg_accuracy_result *out) {
    if (!ctx || !g || !h || !out) return fail(SG_ERR_INVALID_ARG, "NULL argument");
    if (g->n != h->n) return fail(SG_ERR_INVALID_ARG, "G and H must have the same vertex count");
    if (iters < 1 || !(damping >= 0.f && damping <= 1.f)) return fail(SG_ERR_INVALID_ARG, "bad PageRank parameters");
    if (root >= g->n) return fail(SG_ERR_INVALID_ARG, "root out of range");
    Ctx *c = C_(ctx);
    sg_status st = set_device(c);
    if (st != SG_OK) return st;
    *out = sg_accuracy_result{};
    out->m_g = g->nnz / 2;
    const size_t n1 = (size_t)std::max<int64_t>(g->n, 1);
    float *P = nullptr, *Q = nullptr;
    unsigned long long *tg = nullptr, *th = nullptr;
    double rg = 0.0, rh = 0.0;
    st = dalloc(c, (void **)&P, sizeof(float) * n1);
    if (st == SG_OK) st = dalloc(c, (void **)&Q, sizeof(float) * n1);
    if (st == SG_OK) st = dalloc(c, (void **)&tg, sizeof(unsigned long long) * n1);
    if (st == SG_OK) st = dalloc(c, (void **)&th, sizeof(unsigned long long) * n1);
    // A_REN of the PageRank vectors
    if (st == SG_OK) st = pagerank(c, G_(g), damping, iters, P, &rg);
    if (st == SG_OK) st = pagerank(c, G_(h), damping, iters, Q, &rh);
    if (st == SG_OK) st = reordered_neighbours<float>(c, G_(g), P, Q, &out->pr_reordered);
    // A_REN of the per-vertex triangle counts
    if (st == SG_OK) st = sg_vertex_triangle_counts(ctx, g, reinterpret_cast<uint64_t *>(tg));
    if (st == SG_OK) st = sg_vertex_triangle_counts(ctx, h, reinterpret_cast<uint64_t *>(th));
    if (st == SG_OK) st = reordered_neighbours<unsigned long long>(c, G_(g), tg, th, &out->tc_reordered);
    // BFS critical edges from the same root
    if (st == SG_OK && root < 0) st = max_degree_vertex(c, G_(g), &root);
    out->root = root;
    if (st == SG_OK && g->n > 0) st = critical_edges(c, G_(g), root, &out->critical_g);
    if (st == SG_OK && g->n > 0) st = critical_edges(c, G_(h), root, &out->critical_h);
    if (st == SG_OK) st = check_device_error(c);
    const double m = (double)out->m_g;
    out->pr_aren = m > 0 ? (double)out->pr_reordered / m : 0.0;
    out->tc_aren = m > 0 ? (double)out->tc_reordered / m : 0.0;
    out->critical_fraction = out->critical_g > 0 ? (double)out->critical_h / (double)out->critical_g : 1.0;
    dfree(c, P);
    dfree(c, Q);
    dfree(c, tg);
    dfree(c, th);
    return st;
}

sg_status sg_low_degree(sg_ctx *ctx, const sg_graph *g, uint32_t *new_to_old, sg_graph **out) {
    if (!ctx || !g || !out) return fail(SG_ERR_INVALID_ARG, "NULL argument");
    *out = nullptr;
    Ctx *c = C_(ctx);
    sg_status st = set_device(c);
    if (st != SG_OK) return st;
    Graph *h = nullptr;
    st = low_degree(c, G_(g), new_to_old, &h);
    if (st != SG_OK) return st;
    sg_graph *r = new (std::nothrow) sg_graph;
    if (!r) {
        dfree(c, h->off);
        dfree(c, h->col);
        dfree(c, h->w);
        delete h;
        return fail(SG_ERR_OOM, "host allocation failed");
    }
    static_cast<Graph &>(*r) = *h;
    delete h;
    *out = r;
    return SG_OK;
}

sg_status sg_tr_work(sg_ctx *ctx, const sg_graph *g, int64_t *m_out, int64_t *probes_out, int64_t *max_out_degree,
                     int64_t *triangles_out, int64_t *head_arcs_out, int64_t *forward_probes_out) {
    if (!ctx || !g) return fail(SG_ERR_INVALID_ARG, "NULL argument");
    Ctx *c = C_(ctx);
    sg_status st = set_device(c);
    if (st != SG_OK) return st;
    RowMaps rm;
    Oriented o;
    int64_t t = 0, w = 0, md = 0, ha = 0, wf = 0;
    st = build_row_maps(c, G_(g), &rm);
    if (st == SG_OK) st = orient(c, G_(g), rm, false, &o);
    if (st == SG_OK) st = tr_count(c, G_(g), o, &t, &w, &md, &ha, &wf);
    if (st == SG_OK) st = check_device_error(c);
    if (m_out) *m_out = g->nnz / 2;
    if (probes_out) *probes_out = w;
    if (max_out_degree) *max_out_degree = md;
    if (triangles_out) *triangles_out = t;
    if (head_arcs_out) *head_arcs_out = ha;
    if (forward_probes_out) *forward_probes_out = wf;
    free_oriented(c, &o);
    free_row_maps(c, &rm);
    return st;
}

sg_status sg_triangle_count(sg_ctx *ctx, const sg_graph *g, int64_t *count_out) {
    if (!count_out) return fail(SG_ERR_INVALID_ARG, "NULL argument");
    return sg_tr_work(ctx, g, nullptr, nullptr, nullptr, count_out, nullptr, nullptr);
}

}  // extern "C"
