/*
 * slimgraph.h -- C ABI of the GB300 (sm_103a) Slim Graph compression library.
 *
 * Slim Graph (Besta et al., arXiv 1912.08950) compresses a graph lossily by
 * running small "compression kernels" over its edges or triangles (Sec. 3.1,
 * Sec. 4.1, Listing 1) in one concurrent pass (Listing 2: run_kernels once for
 * every scheme except summarisation), and judges the result with accuracy
 * metrics such as the KL divergence of PageRank distributions (Sec. 5.2.3).
 * This library implements that data-parallel hot path with hand-written CUDA
 * kernels: compress(graph, kernel, p, seed) -> graph, and divergence(G, H).
 *
 * Conventions shared by every entry point
 *  - Graphs are undirected, simple and stored as a symmetric CSR: row offsets
 *    off[n+1] (int64, off[0] = 0, non-decreasing), column ids col[nnz]
 *    (uint32, each row strictly increasing, no self-loops, every arc (x,y)
 *    matched by (y,x)), optional weights w[nnz] (float32, equal on both arcs
 *    of an edge).  nnz = 2m arcs for m undirected edges.  n < 2^32.
 *  - "device" pointers are CUDA global-memory addresses on the context's
 *    device; "host" pointers are ordinary CPU memory (pinned memory makes the
 *    copies faster but is not required).
 *  - Every call returns an sg_status.  Nothing throws, traps or aborts; on a
 *    non-OK status sg_last_error() returns a message for the calling thread.
 *  - All device work is ordered on the context's stream.  Calls that return
 *    results to the host (counts, sizes, scalars) synchronise that stream.
 *  - Randomness: every decision draws Philox4x32-10 (Salmon et al., SC'11)
 *    keyed by the 64-bit seed (key = low word, high word).  An edge {lo<hi}
 *    uses counter (lo, hi, 0, 0x45444745); a triangle {a<b<c} uses counter
 *    (a, b, c, 0x54524931).  A probability p becomes the threshold
 *    floor(p * 2^32) and an event fires iff a 32-bit draw is below it.  Keys
 *    are original vertex ids, so results do not depend on launch shape.
 */
#ifndef SLIMGRAPH_H
#define SLIMGRAPH_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum sg_status {
    SG_OK = 0,
    SG_ERR_INVALID_ARG = 1,   /* bad pointer, size or parameter (p outside [0,1], NaN, ...) */
    SG_ERR_INVALID_GRAPH = 2, /* CSR fails validation (only checked when asked) */
    SG_ERR_NEEDS_WEIGHTS = 3, /* a max-weight kernel on an unweighted graph */
    SG_ERR_OOM = 4,           /* device allocation failed */
    SG_ERR_CUDA = 5,          /* a CUDA runtime call failed */
    SG_ERR_TIMEOUT = 6,       /* a bounded device-side wait expired; outputs are invalid */
    SG_ERR_UNSUPPORTED = 7    /* outside the supported envelope (n >= 2^32, ...) */
} sg_status;

/*
 * Compression kernels (Listing 1; Table 4).
 *  SG_UNIFORM          random_uniform(E e): each edge stays with probability p
 *                      (Sec. 4.2.2).
 *  SG_SPECTRAL_LOGN    spectral_sparsify(E e) with Y = p ln n (Sec. 4.2.1):
 *                      edge (u,v) stays with probability min(1, Y/min(d_u,d_v));
 *                      kept edges get weight 1/p_uv when weights are wanted.
 *  SG_SPECTRAL_AVGDEG  the same with Y = p m / n.
 *  SG_TR_RANDOM        Triangle p-1-Reduction (Sec. 4.3): every triangle of the
 *                      input is selected with probability p and deletes one
 *                      uniformly chosen edge; deletions accumulate (union).
 *  SG_TR_MAXW          as SG_TR_RANDOM, deleting the heaviest edge of each
 *                      selected triangle (ties by endpoint pair); keeps the
 *                      MST weight and the connected components (Sec. 4.3, 6).
 *  SG_TR_EO            Edge-Once p-1-TR (Sec. 4.3; Sec. 6): only edge-disjoint
 *                      triangles are considered -- selected triangles in order
 *                      of (r2, a, b, c), each accepted iff none of its edges was
 *                      already considered; keeps the connected components.
 *  SG_TR_EO_MAXW       Edge-Once with the max-weight choice.
 *  SG_TR_P2            Triangle p-2-Reduction (Sec. 4.3, x = 2): every selected
 *                      triangle deletes two of its edges and keeps only the
 *                      one its draw r1 names; deletions accumulate (union).
 *  SG_TR_MINCOUNT      as SG_TR_RANDOM, deleting the edge of each selected
 *                      triangle that lies in the fewest triangles of G (ties by
 *                      endpoint pair); one extra enumeration pass counts them.
 *  SG_TR_EO_MINCOUNT   Edge-Once with the min-count choice (the "CT" variant
 *                      of Sec. 7); keeps the connected components.
 */
typedef enum sg_kernel {
    SG_UNIFORM = 0,
    SG_SPECTRAL_LOGN = 1,
    SG_SPECTRAL_AVGDEG = 2,
    SG_TR_RANDOM = 3,
    SG_TR_MAXW = 4,
    SG_TR_EO = 5,
    SG_TR_EO_MAXW = 6,
    SG_TR_P2 = 7,
    SG_TR_MINCOUNT = 8,
    SG_TR_EO_MINCOUNT = 9
} sg_kernel;

/* Opaque context: device, stream, device error word, launch statistics. */
typedef struct sg_ctx sg_ctx;
/* Opaque device-resident CSR graph, owned by the library unless borrowed. */
typedef struct sg_graph sg_graph;

/* Borrowed view of a device CSR (all pointers are device pointers). */
typedef struct sg_csr_view {
    int64_t n;
    int64_t nnz;
    const int64_t *off;
    const uint32_t *col;
    const float *w; /* may be NULL */
} sg_csr_view;

/* Result of the accuracy analytics of one compression (Sec. 5). */
typedef struct sg_div_result {
    double kl_bits;       /* D_KL(PR_G || PR_H) in bits (Sec. 5.2.3) */
    int64_t cc_g, cc_h;   /* connected components of G and H (Table 1) */
    int64_t m_g, m_h;     /* undirected edge counts of G and H */
    double pr_residual_g; /* FP64 L1 norm of the last PageRank update of G */
    double pr_residual_h; /* ... of H */
} sg_div_result;

/* Launch accounting of a context (for benchmarks and profiles). */
typedef struct sg_stats {
    uint64_t kernel_launches; /* kernels this library launched on the context */
    uint64_t probes;          /* wedge-closing probes done by triangle kernels */
    uint64_t triangles;       /* triangles found by triangle kernels */
    uint64_t eo_rounds;       /* Edge-Once reservation rounds run */
    uint64_t eo_listed;       /* triangles written to Edge-Once lists (16 bytes each) */
    uint64_t eo_passes;       /* Edge-Once enumeration passes (each bids for its round) */
    uint64_t eo_list_passes;  /* ... of them that listed triangles for later rounds */
} sg_stats;

/* ---------------------------------------------------------------- context */

/* Create a context on CUDA device `device`.  `cuda_stream` is a cudaStream_t
 * owned by the caller (NULL: the library creates and owns a stream).  The
 * context must outlive every graph created through it.
 * Errors: SG_ERR_INVALID_ARG (out == NULL), SG_ERR_CUDA. */
sg_status sg_ctx_create(int device, void *cuda_stream, sg_ctx **out);
/* Destroy a context (synchronises its stream first).  NULL is ignored. */
void sg_ctx_destroy(sg_ctx *ctx);
/* Block until all work queued on the context's stream has finished. */
sg_status sg_ctx_synchronize(sg_ctx *ctx);
/* Read (and optionally reset) the launch accounting of the context. */
sg_status sg_ctx_stats(sg_ctx *ctx, sg_stats *out, int reset);
/* Per-kernel timing: when on, every launch is bracketed by CUDA events on the
 * context stream.  sg_ctx_kernel_time returns the summed device time (ms) and
 * launch count of kernels whose name starts with `prefix` since the last reset. */
sg_status sg_ctx_set_profiling(sg_ctx *ctx, int on);
sg_status sg_ctx_kernel_time(sg_ctx *ctx, const char *prefix, double *ms, int64_t *launches);
sg_status sg_ctx_reset_profile(sg_ctx *ctx);
/* Memory bound of the Edge-Once kernels.  An enumeration lists the live
 * selected triangles (16 bytes each, 32 once they bid), grouped by the round
 * of the prefix schedule in which they first bid, so that later reservation
 * rounds need no new enumeration.  When they do not all fit, the list keeps
 * the earliest groups that do (a window of the schedule); once every triangle
 * in the window is decided, one more enumeration lists the live ones above
 * it.  records > 0 caps the list at that many triangles, 0 (default) sizes it
 * at a quarter of free device memory, -1 disables it (every round then
 * enumerates the triangles again).  The result is the same in every setting;
 * only time and memory change. */
sg_status sg_ctx_set_eo_list_capacity(sg_ctx *ctx, int64_t records);
/* The Edge-Once lists live in device workspaces that the context keeps and
 * reuses across calls (grown when a call needs more).  This frees them, in
 * stream order; the next Edge-Once call allocates them again.
 * Errors: SG_ERR_INVALID_ARG (ctx == NULL). */
sg_status sg_ctx_release_workspace(sg_ctx *ctx);

/* Test hook for the SG_ERR_TIMEOUT contract (the paper has no counterpart).
 * With spin_limit > 0, the first tile of every chunk-count prefix scan the
 * context runs (in the CSR rebuild, the orientation, the edge kernels) never
 * publishes its prefix, and a tile waiting on a predecessor gives up after
 * spin_limit polls; a graph whose scan has a single tile (under about 262,000
 * arcs) has no wait to give up.  The call returns SG_ERR_TIMEOUT, its outputs
 * are invalid, and the context stays usable.  0 (the default) restores normal operation, where
 * a wait gives up only after 2^22 polls.
 * Errors: SG_ERR_INVALID_ARG (ctx == NULL). */
sg_status sg_ctx_set_scan_hold(sg_ctx *ctx, uint32_t spin_limit);

/* Device memory free for new work on CUDA device `device`, in bytes: what
 * the driver reports free (cudaMemGetInfo) plus what the device's default
 * stream-ordered pool holds from freed allocations but does not use (this
 * library keeps freed memory in that pool between calls).  The paper has no
 * counterpart: serving admits jobs by it.  The caller's current device is
 * left unchanged.
 * Errors: SG_ERR_INVALID_ARG (free_out == NULL, no such device), SG_ERR_CUDA. */
sg_status sg_device_free_memory(int device, uint64_t *free_out);

/* ----------------------------------------------------------------- graphs */

/* Wrap or copy a device CSR.  copy = 0 borrows the caller's buffers (they must
 * stay alive and unchanged until sg_graph_free); copy = 1 makes library-owned
 * copies.  validate = 1 checks the CSR conventions above on the device and
 * returns SG_ERR_INVALID_GRAPH on a violation.
 * Errors: SG_ERR_INVALID_ARG, SG_ERR_UNSUPPORTED (n >= 2^32), SG_ERR_OOM, SG_ERR_CUDA. */
sg_status sg_graph_from_device(sg_ctx *ctx, const sg_csr_view *in, int copy, int validate, sg_graph **out);
/* Copy a host CSR to the device (library-owned).  w may be NULL. */
sg_status sg_graph_from_host(sg_ctx *ctx, int64_t n, int64_t nnz, const int64_t *off, const uint32_t *col,
                             const float *w, sg_graph **out);
/* Borrow the device pointers of a graph (valid until sg_graph_free). */
sg_status sg_graph_view(const sg_graph *g, sg_csr_view *out);
/* Copy a graph to caller-owned host buffers off[n+1], col[nnz] and, if the
 * graph is weighted and w != NULL, w[nnz].  Synchronises the stream. */
sg_status sg_graph_download(sg_ctx *ctx, const sg_graph *g, int64_t *off, uint32_t *col, float *w);
/* Free a graph (stream-ordered on the context stream).  NULL is ignored. */
void sg_graph_free(sg_graph *g);

/* ------------------------------------------------------------ compression */

/* compress(G, kernel, p, seed) -> H  (Listing 1 kernels, one run_kernels pass,
 * Listing 2).  H is a new library-owned graph with the same n whose edge set is
 * a subset of G's; G is never modified (the paper's SG.del mutates in place).
 * Weights of H: the spectral kernels with want_weights = 1 produce 1/p_uv
 * (Sec. 4.2.1); otherwise the input weights of the kept edges are carried.
 * Errors: SG_ERR_INVALID_ARG (p not in [0,1] or NaN, bad kernel),
 * SG_ERR_NEEDS_WEIGHTS, SG_ERR_OOM, SG_ERR_CUDA, SG_ERR_TIMEOUT. */
sg_status sg_compress(sg_ctx *ctx, const sg_graph *g, sg_kernel kernel, double p, uint64_t seed,
                      int want_weights, sg_graph **out);

/* ---------------------------------------------------------------- batches */

/* Many independent graphs compressed together (the paper runs one graph per
 * pass; batching is this library's addition).  A batch packs `count` graphs
 * (copied, so the inputs may be freed afterwards) into one device-resident
 * disjoint union; all graphs must be weighted or all unweighted; count is at
 * most 65535 and the union must have fewer than 2^32 vertices.
 * Errors: SG_ERR_INVALID_ARG, SG_ERR_UNSUPPORTED, SG_ERR_OOM, SG_ERR_CUDA. */
typedef struct sg_batch sg_batch;
sg_status sg_batch_create(sg_ctx *ctx, int count, const sg_graph *const *graphs, sg_batch **out);
void sg_batch_free(sg_batch *b);
/* Compress graph i of the batch with kernels[i], ps[i], seeds[i] -- the same
 * result, bit for bit, as sg_compress on that graph alone.  Every step runs
 * once over the whole union and the sequence is replayed as one CUDA graph;
 * the first call times a few work-partition settings on this batch (CTAs per
 * SM of the compaction and enumeration kernels, the warp-per-vertex out-degree
 * limit) and keeps the fastest.  outs[i] receives a handle whose arrays live
 * inside the batch: they stay valid until the next sg_compress_batch on this
 * batch or sg_batch_free; release each handle with sg_graph_free.  Edge-once
 * kernels need host-driven rounds and SG_TR_MINCOUNT a counting pass: they
 * return SG_ERR_UNSUPPORTED here. */
sg_status sg_compress_batch(sg_ctx *ctx, sg_batch *b, const sg_kernel *kernels, const double *ps,
                            const uint64_t *seeds, int want_weights, sg_graph **outs);
/* Size of the union and the work-partition setting the autotuner chose
 * (light_max: largest out-degree given one warp; *_per_sm: CTAs per SM, 0 =
 * occupancy limit; tuned_ms: the winner's replay time).  Any pointer may be NULL. */
sg_status sg_batch_info(const sg_batch *b, int64_t *vertices, int64_t *arcs, int *light_max, int *compact_per_sm,
                        int *enum_per_sm, double *tuned_ms);

/* ------------------------------------------------------------- analytics */

/* divergence(G, H): PageRank of both graphs (damping, iters; FP32 values,
 * deterministic order), KL divergence of the two distributions summed in FP64
 * (Sec. 5.2.3), and the connected-component counts (Table 1).  Graphs are
 * treated as unweighted.  G and H must have the same n. */
sg_status sg_divergence(sg_ctx *ctx, const sg_graph *g, const sg_graph *h, float damping, int iters,
                        sg_div_result *out);
/* PageRank (Table 1): x0 = 1/n, x' = (1-d)/n + d (sum_{u in N(v)} x_u/d_u + D/n),
 * D = rank held by degree-0 vertices.  x_out: device float[n].  residual_out
 * (may be NULL): FP64 L1 norm of the last update. */
sg_status sg_pagerank(sg_ctx *ctx, const sg_graph *g, float damping, int iters, float *x_out,
                      double *residual_out);
/* D_KL(P || Q) = sum_i P_i log2(P_i / Q_i) of two device float[n] vectors,
 * each normalised by its FP64 sum (Sec. 5.2.3). */
sg_status sg_kl_divergence(sg_ctx *ctx, int64_t n, const float *P, const float *Q, double *kl_out);
/* Number of connected components (isolated vertices count).  labels_out: a
 * device uint32[n] receiving the smallest vertex id of each component, or NULL. */
sg_status sg_cc_count(sg_ctx *ctx, const sg_graph *g, int64_t *count_out, uint32_t *labels_out);
/* Number of triangles of G (each counted once), with the degree-ordered
 * enumeration used by the TR kernels. */
sg_status sg_triangle_count(sg_ctx *ctx, const sg_graph *g, int64_t *count_out);
/* Work model of the degree-ordered enumeration of G (runs one counting pass):
 * m; the probe count W = sum over oriented arcs u->v of the shorter of
 * d+(u), d+(v) (each arc streams its shorter list through a table of the
 * longer one, ties to d+(v)); the maximum out-degree; the triangle count; and
 * the number of arcs streamed from the head's side (those with
 * d+(u) < d+(v), gathered into per-vertex in-lists of 8 bytes each); and
 * W+ = sum over oriented arcs u->v of d+(v), the probes of the plain forward
 * algorithm that streams N+(v) for every arc (Sec. 4.3's listing cost).  Used
 * to turn kernel times into algorithmic bytes.  Any out pointer may be NULL. */
sg_status sg_tr_work(sg_ctx *ctx, const sg_graph *g, int64_t *m_out, int64_t *probes_out,
                     int64_t *max_out_degree, int64_t *triangles_out, int64_t *head_arcs_out,
                     int64_t *forward_probes_out);

/* ------------------------------------------ accuracy metrics (Sec. 5) */

/* BFS levels from `root` (Sec. 5.3): levels is a device int32[n] receiving
 * the hop distance of every vertex, -1 where root does not reach.  Levels are
 * unique, so the result does not depend on traversal order.
 * Errors: SG_ERR_INVALID_ARG (root outside [0, n)), SG_ERR_OOM, SG_ERR_CUDA. */
sg_status sg_bfs_levels(sg_ctx *ctx, const sg_graph *g, int64_t root, int32_t *levels);
/* |E_cr| of a BFS from `root` (Sec. 5.3): the tree edges plus every edge that
 * could replace one, i.e. the undirected edges joining levels L and L + 1. */
sg_status sg_critical_edges(sg_ctx *ctx, const sg_graph *g, int64_t root, int64_t *count_out);
/* The numerator of A_REN (Sec. 5.2.2): the number of undirected edges {u,v}
 * of g whose endpoint order under the device score vector x (float[n])
 * differs from their order under y: sign(x_u - x_v) != sign(y_u - y_v),
 * compared in float. */
sg_status sg_reordered_neighbours(sg_ctx *ctx, const sg_graph *g, const float *x, const float *y,
                                  int64_t *count_out);
/* Triangles through every vertex (the per-vertex output "TC" of Table 1):
 * counts is a device uint64[n], overwritten. */
sg_status sg_vertex_triangle_counts(sg_ctx *ctx, const sg_graph *g, uint64_t *counts);

/* The vertex-level accuracy metrics of one compression G -> H (same n). */
typedef struct sg_accuracy_result {
    int64_t m_g;               /* undirected edges of G: the A_REN denominator */
    int64_t pr_reordered;      /* edges of G whose PageRank order differs in H (FP32 PageRank) */
    double pr_aren;            /* pr_reordered / m_g */
    int64_t tc_reordered;      /* the same for the per-vertex triangle counts */
    double tc_aren;            /* tc_reordered / m_g */
    int64_t root;              /* the BFS root used */
    int64_t critical_g;        /* |E_cr| of G */
    int64_t critical_h;        /* |E~_cr|: critical edges of H for the same root */
    double critical_fraction;  /* critical_h / critical_g (1 when critical_g = 0) */
} sg_accuracy_result;
/* PageRank (damping, iters as in sg_divergence) and per-vertex triangle
 * counts of G and H with their A_REN, and the BFS critical-edge fraction
 * |E~_cr| / |E_cr| from `root` (root < 0: the vertex of largest degree in
 * G, the smallest id on ties).
 * Errors: SG_ERR_INVALID_ARG (n differs, bad PageRank parameters, root >= n),
 * SG_ERR_OOM, SG_ERR_CUDA. */
sg_status sg_accuracy(sg_ctx *ctx, const sg_graph *g, const sg_graph *h, float damping, int iters, int64_t root,
                      sg_accuracy_result *out);

/* ------------------------------------------------ single-vertex kernel */

/* low_degree(V v) (Listing 1; Sec. 4.4): H is G without its vertices of
 * degree 0 or 1 -- decided in one pass over the input degrees -- and without
 * their edges; the kept vertices are renumbered 0..n'-1 in increasing order
 * of their ids in G, so H has n' <= n vertices.  Weights of kept edges are
 * carried.  new_to_old: a device uint32 array with room for n entries (or
 * NULL); entry i < n' receives the id in G of H's vertex i.  *out receives a
 * new graph owned by the library (release it with sg_graph_free).
 * Errors: SG_ERR_INVALID_ARG, SG_ERR_OOM, SG_ERR_CUDA. */
sg_status sg_low_degree(sg_ctx *ctx, const sg_graph *g, uint32_t *new_to_old, sg_graph **out);

/* ------------------------------------------------- no-allocation variant */

/* Uniform edge sampling (SG_UNIFORM) that allocates no device memory.  The
 * paper has no counterpart: this exists for callers that cannot call
 * cudaMalloc -- for example a host framework whose own allocator owns the
 * whole GPU memory budget and must account for every byte, or a caller that
 * reserved device memory up front and cannot let a library grow it.  Such a
 * caller passes device buffers for the input CSR (off[n+1], col[nnz]) and for
 * the output (off_out[n+1], col_out with room for nnz arcs, since the output
 * is a subset of the input); the result equals sg_compress(G, SG_UNIFORM, p,
 * seed) bit for bit and *nnz_out (host) receives its arc count.
 * The input must be a valid symmetric CSR as defined at the top of this
 * header; the call checks only that off[0] = 0 and off[n] = nnz
 * (SG_ERR_INVALID_GRAPH otherwise).
 * Scratch lives in one fixed device array inside the library (about 23 MB per
 * GPU that loads it, held until the process exits), which caps the input at
 * nnz <= 134217728 arcs; larger inputs return SG_ERR_UNSUPPORTED.
 * The first call on a device looks up that array's device address and keeps
 * it for the life of the process (a cudaDeviceReset of that device makes the
 * kept address stale).  The call synchronises cuda_stream and reads its
 * result into host memory, so it cannot be recorded in a stream capture; it
 * leaves the caller's current device as it found it.  All calls of a process
 * share the one array on a device: calls that overlap on the GPU (different
 * streams or threads of that process) race and must be serialised by the
 * caller.  No context is needed; errors are
 * reported as by every other entry point (sg_last_error). */
sg_status sg_compress_uniform_noalloc(int device, void *cuda_stream, int64_t n, int64_t nnz, const int64_t *off,
                                      const uint32_t *col, double p, uint64_t seed, int64_t *off_out,
                                      uint32_t *col_out, int64_t *nnz_out);

/* Architecture of the library's device code as loaded on `device`
 * (cudaFuncAttributes.binaryVersion of one of its kernels: 103 for sm_103a).
 * The paper has no counterpart: it lets a caller check at run time that the
 * build matches the GPU.  The caller's current device is left unchanged.
 * Errors: SG_ERR_INVALID_ARG (NULL, no such device), SG_ERR_CUDA (no image
 * for this device). */
sg_status sg_kernel_arch(int device, int *binary_version);

/* Message describing the last non-OK status returned on this thread. */
const char *sg_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* SLIMGRAPH_H */
