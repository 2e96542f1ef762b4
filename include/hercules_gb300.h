/*
 * hercules_gb300.h -- C ABI of the GB300 Hercules exact k-NN library.
 *
 * The library builds a Hercules index (Echihabi et al., PVLDB 15(10), 2022)
 * over N float32 data series of length n, resident in the memory of one GPU,
 * and answers exact k-NN queries under the Euclidean distance against it.
 *
 * Conventions for every entry point:
 *   - Return value: HK_OK (0) or a negative HK_E* code.  hk_last_error()
 *     then returns a message for the calling thread.  A failed call leaves
 *     its outputs unspecified and releases what it allocated.
 *   - Pointers to series, queries and outputs may be host or device
 *     memory of the current CUDA device; the library finds out which with
 *     cudaPointerGetAttributes and copies as needed.  The caller keeps
 *     ownership of every buffer it passes, except as HK_BUILD_ADOPT says.
 *   - Layouts are row-major: X[i*n + j] is point j of series i.
 *   - stream: a cudaStream_t (NULL = the legacy default stream).  Calls are
 *     synchronous with respect to the host: outputs are complete on return.
 *   - The library never normalises the series (the paper's collections are
 *     z-normalised beforehand, Sec. 4.1); NaN or Inf in X or Q is rejected.
 */
#ifndef HERCULES_GB300_H
#define HERCULES_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define HK_OK 0
#define HK_EINVAL (-1)    /* bad argument: sizes, null pointers, NaN/Inf     */
#define HK_ENOMEM (-2)    /* device or host allocation failed                */
#define HK_ECUDA (-3)     /* a CUDA runtime call failed                      */
#define HK_ETIMEOUT (-4)  /* a bounded device or host wait ran out           */
#define HK_EBUSY (-5)     /* the object is in use (server slots full)        */
#define HK_EINTERNAL (-6) /* an internal consistency check failed            */
#define HK_EIO (-7)       /* a file could not be opened, read or written     */

#define HK_ISAX_SEGMENTS 16   /* iSAX word length (Sec. 2)                     */
#define HK_ISAX_ALPHABET 256  /* iSAX alphabet (Sec. 2)                        */
#define HK_MIN_LEN 16
#define HK_MAX_LEN 4096
#define HK_MAX_K 1024

typedef struct hk_index hk_index;

/* Build flags. */
#define HK_BUILD_ADOPT 1u  /* X is a device buffer from cudaMalloc that the
                              index takes over and frees once it no longer
                              needs it (saves one copy of the collection).  */
#define HK_BUILD_BF16 2u   /* also keep a bfloat16 copy of the collection
                              and its norms (precision form).               */
#define HK_BUILD_FP16 4u   /* the same with float16 instead (three more bits
                              of precision; values must fit float16:
                              |x| <= 65504, else HK_EINVAL)                 */

typedef struct {
    int32_t leaf_capacity;  /* tau, the leaf threshold (Sec. 3.2); >= 1      */
    int32_t eval_cap;       /* series a split policy is chosen from: the
                               node's first min(tau+1, eval_cap); 0 = 4096    */
    uint32_t flags;         /* HK_BUILD_*                                     */
    int32_t reserved;
} hk_build_opts;

/*
 * hk_build -- build an index (Sec. 3.2-3.3, Algorithm InsertSeriesToNode;
 * Algorithms WriteIndexWorker / WriteLeafData for the leaf-ordered layout).
 *
 * X: N*n float32 (host or device).  N >= 1, 16 <= n <= 4096, n % 16 == 0.
 * The tree is the one sequential insertion in id order produces with the
 * library's split policy (4 root segments; H- and V-splits chosen by the
 * smallest size-weighted synopsis spread).  The raw series are stored in
 * leaf (inorder) order with their iSAX words (LRDFile/LSDFile, Sec. 3.3).
 * On success *out owns all device memory of the index; free it with hk_free.
 */
int hk_build(const float *X, int64_t N, int32_t n, const hk_build_opts *opts,
             void *stream, hk_index **out);

int hk_free(hk_index *idx);

typedef struct {
    int64_t N;
    int32_t n;
    int32_t leaf_capacity;
    int64_t leaves;
    int32_t max_segments;    /* most segments of any leaf                     */
    int32_t depth;           /* levels of splits                              */
    int64_t distinct_segments;
    int64_t device_bytes;    /* device memory the index holds                 */
    int32_t has_bf16;
    int32_t reserved;
} hk_index_info;

int hk_index_info_get(const hk_index *idx, hk_index_info *out);

/*
 * hk_save -- write the index to the file at path (created or truncated): the
 * tree (links, position ranges, segmentations and synopses of its leaves and
 * internal nodes), the leaf-ordered raw series, their positions' original
 * ids and iSAX words, and the 16-bit copy when the index has one -- the
 * paper's HTree, LRDFile and LSDFile (Sec. 3.3) in one file.
 * Layout: the tag "HKIDX002", a header of sizes, then each array as a 64-bit
 * byte count followed by its bytes, then an FNV-1a 64-bit checksum of all
 * array bytes; integers and floats in this machine's byte order.  Returns
 * HK_EIO if the file cannot be written.  The index is not modified.
 *
 * hk_load -- read a file written by hk_save into a new index (device memory
 * allocated on the current device, copies on `stream`); *out as for
 * hk_build.  A file that does not start with the tag, whose header is
 * inconsistent, whose arrays have the wrong lengths or whose checksum does
 * not match returns HK_EINVAL with nothing allocated; an unreadable file
 * returns HK_EIO.  Answers from the loaded index equal the saved index's.
 */
int hk_save(const hk_index *idx, const char *path);
int hk_load(const char *path, void *stream, hk_index **out);

/* Query flags. */
#define HK_Q_NOSAX 1u      /* skip LB_SAX filtering (ablation, Sec. 4.2)      */
#define HK_Q_NOTHRESH 2u   /* ignore EAPCA_TH / SAX_TH (ablation)             */
#define HK_Q_NOPRUNE 4u    /* scan every series (parallel-scan baseline)      */
#define HK_Q_TIMING 8u     /* time the scan kernels with CUDA events on the
                              call's stream (hk_query_stats.scan_ns)          */
#define HK_Q_BF16 16u      /* precision form: distances of the candidate
                              leaves on the tensor cores from the index's
                              16-bit copy (HK_BUILD_BF16 or HK_BUILD_FP16,
                              n <= 256), certified error bound, exact rescore */
#define HK_Q_GRAPH 32u     /* replay the query pass from a CUDA graph: the
                              first call with a given (nq, k, options) runs
                              normally and records the pass; later calls with
                              the same key copy Q into the index's graph work
                              space and replay it (same answers).  The index
                              holds one graph; calls on one index must not run
                              concurrently.  HK_Q_TIMING is ignored.          */
#define HK_Q_TREE 64u      /* prune with the tree's internal-node synopses
                              (Sec. 3.3): the approximate search walks the
                              tree best-first by LB_EAPCA (Approx-kNN), and
                              candidate leaves come from a top-down pass that
                              evaluates a node only where its parent stayed,
                              pruning whole subtrees (same answers; fewer
                              LB_EAPCA evaluations when leaves are many).
                              Not with HK_Q_NOPRUNE.                          */

typedef struct {
    int32_t l_max;        /* leaves visited by the approximate search per query
                             (Sec. 3.4, Approx-kNN); 0 = 1                     */
    float eapca_th;       /* EAPCA_TH; < 0 = 0.25 (Sec. 4.2)                   */
    float sax_th;         /* SAX_TH; < 0 = 0.50 (Sec. 4.2)                     */
    uint32_t flags;       /* HK_Q_*                                            */
    int32_t query_group;  /* queries sharing one scan work item; 0 = auto      */
    int32_t series_tile;  /* series per scan work item; 0 = auto              */
} hk_query_opts;

typedef struct {
    int64_t queries;
    int64_t leaves_total;         /* leaves x queries                          */
    int64_t leaves_approx;        /* (leaf, query) pairs of the approximate step */
    int64_t leaves_candidate;     /* (leaf, query) pairs in LCList               */
    int64_t series_candidate;     /* (series, query) pairs in candidate leaves   */
    int64_t series_sax_pruned;    /* pruned by LB_SAX                            */
    int64_t series_abandoned;     /* distance computation abandoned early        */
    int64_t series_full;          /* distance computed over all n points         */
    int64_t points_computed;      /* (q - x)^2 terms evaluated                   */
    int64_t rescored;             /* binary64 boundary rescores                  */
    int64_t fallback_queries;     /* queries finished by the exhaustive collect  */
    int64_t retried_queries;      /* queries run again from their final bound
                                     after a candidate list or pool overflowed  */
    int64_t work_items;           /* scan work items launched                    */
    int64_t skip_sequential;      /* queries scanned without LB_SAX (EAPCA_TH)   */
    int64_t scan_ns;              /* float32 scan kernel time (HK_Q_TIMING), ns  */
    int64_t kernel_launches;      /* kernels this call launched                  */
    int64_t scan_bytes;           /* series bytes the scan read: 64 B per 16-point
                                     chunk loaded + 16 B per iSAX word, per item */
    int64_t tc_pairs;             /* (query, series) distances on tensor cores   */
    int64_t tc_candidates;        /* of those, kept for the exact rescore        */
    int64_t tc_ns;                /* tensor-core kernel time (HK_Q_TIMING), ns   */
    int64_t tc_bytes;             /* 16-bit rows and norms the tensor-core kernel
                                     copied in (per query block)                 */
    int64_t tc_approx_pairs;      /* the approximate step's distances on tensor
                                     cores (k <= 16; tc_* count the exact step)  */
    int64_t tc_approx_ns;         /* its kernel time (HK_Q_TIMING), ns           */
    int64_t tc_approx_bytes;      /* its 16-bit rows and norms copied in         */
    int64_t tc_leaf_bytes;        /* 16-bit rows and norms of the leaves the exact
                                     step scans, each leaf once: the least DRAM
                                     traffic that step can have                  */
    int64_t lb_evaluations;       /* (query, node) LB_EAPCA evaluations: queries x
                                     leaves without HK_Q_TREE, the nodes visited
                                     with it                                     */
} hk_query_stats;

/*
 * hk_query_opts_default -- write the options that opts = NULL stands for,
 * with every "0 / < 0 = default" field resolved: l_max = 1 (Sec. 3.4,
 * Approx-kNN step 1: one leaf by default), eapca_th = 0.25 and sax_th = 0.50
 * (the thresholds of Sec. 4.2, Parameterization), flags 0, query_group and
 * series_tile 0 (chosen per call).  Host-only; needs no GPU.  HK_EINVAL if
 * out is NULL.
 */
int hk_query_opts_default(hk_query_opts *out);

/*
 * hk_query -- exact k-NN (Sec. 3.4, Algorithm Exact-kNN and its steps
 * Approx-kNN, FindCandidateLeaves, CSWorker, CRWorker), for nq queries
 * answered together.
 *
 * Q: nq*n float32 (host or device).  1 <= k <= min(N, 1024).
 * out_ids: nq*k int64 original row ids; out_dist: nq*k float32 Euclidean
 * distances (sqrt of the binary64 squared distance, rounded to float32).
 * Row i lists query i's neighbours ascending by (binary64 squared distance
 * summed in index order, id): the brute-force answer, ties to the lower id.
 * stats may be NULL; opts may be NULL (defaults).
 * Calls on one index share its work space (and its staging buffer for host
 * queries): they must not run concurrently; the server (hk_server_*) answers
 * concurrent requests.
 */
int hk_query(hk_index *idx, const float *Q, int32_t nq, int32_t k,
             const hk_query_opts *opts, void *stream, int64_t *out_ids,
             float *out_dist, hk_query_stats *stats);

/*
 * hk_query_dtw -- exact k-NN under Dynamic Time Warping (Sec. 2: Hercules
 * supports any distance with a lower-bounding distance, e.g. DTW with the
 * bound of Keogh and Ratanamahatana, KAIS 2005), on the same index.
 * Distance: squared point costs summed along the cheapest warping path that
 * stays within the Sakoe-Chiba band |i - j| <= band (0 <= band <=
 * min(16, n-1); band 0 is the squared Euclidean distance):
 *   D(i,j) = (q_i - x_j)^2 + min(D(i-1,j-1), D(i-1,j), D(i,j-1)).
 * Pruning: the query's envelope against each leaf synopsis (segment means),
 * against each series' iSAX word, and LB_Keogh against its raw points, then
 * the DTW with early abandoning; all in float32 with certified rounding,
 * candidates rescored in binary64.  Outputs as hk_query: ids ascending by
 * (binary64 DTW, id), out_dist = sqrt(DTW).  opts: l_max and HK_Q_NOSAX are
 * used, other fields ignored; NULL = defaults.  Calls on one index must not
 * run concurrently (they share its DTW work space).
 */
int hk_query_dtw(hk_index *idx, const float *Q, int32_t nq, int32_t k, int32_t band,
                 const hk_query_opts *opts, void *stream, int64_t *out_ids, float *out_dist,
                 hk_query_stats *stats);

/*
 * hk_scan_knn -- exact k-NN by scanning every series of a collection (no
 * index): the parallel scan the paper compares against (PSCAN, Sec. 2 and
 * Sec. 4.1), with the same answer definition and outputs as hk_query.
 * X: N*n float32, Q: nq*n float32 (host or device).
 */
int hk_scan_knn(const float *X, int64_t N, int32_t n, const float *Q,
                int32_t nq, int32_t k, void *stream, int64_t *out_ids,
                float *out_dist);

/*
 * hk_scan_knn_noalloc -- hk_scan_knn for callers that cannot allocate device
 * memory.  The paper has no counterpart: it is an interface for callers
 * that must not call cudaMalloc or cudaFree, e.g. a process whose device
 * memory is held by another allocator (a framework's caching allocator can
 * leave too little free for a raw cudaMalloc), or a latency-bound caller
 * sharing the GPU (cudaFree waits for the whole device).
 *
 * Same answer definition as hk_scan_knn.  X (N*n), Q (nq*n), out_ids and
 * out_dist (nq*k) must all be device memory; nothing is copied and nothing
 * is allocated: the work space is a fixed 6 MiB array compiled into the
 * library, held on every GPU that loads it until the process exits.
 * Limits: 1 <= nq <= 64, 1 <= k <= min(N, 64), and at most 65,536
 * near-tied candidates per query; larger sizes return HK_EINVAL (HK_ENOMEM
 * for the tie limit) with a message.  Each query pools at most 4,096
 * candidates (hk_scan_knn pools max(4,096, 64 * (k + 32 rounded up to 32)),
 * more once k > 32): a query with more near-ties than its pool holds is
 * finished by an exhaustive collect, so for k > 32 near-tied queries take
 * that slower path more often here than in hk_scan_knn (same answers).
 * The first call on a device looks up the array's device address and
 * should come before any stream capture; the address is kept for the life
 * of the process, so resetting a device (cudaDeviceReset) after that first
 * call is not supported.
 * All calls share the array and it keeps the last call's contents (each
 * call clears what must start at zero): calls whose GPU work overlaps, on
 * different streams or host threads, race on it.
 */
int hk_scan_knn_noalloc(const float *X, int64_t N, int32_t n, const float *Q,
                        int32_t nq, int32_t k, void *stream, int64_t *out_ids,
                        float *out_dist);

/* ---- serving: continuous batching --------------------------------------------- */

typedef struct hk_server hk_server;

typedef struct {
    int32_t max_batch;     /* most requests answered by one batch; 0 = 1024     */
    int32_t max_wait_us;   /* how long a worker lingers to fill a batch once a
                              request is pending; 0 = take what is pending      */
    int64_t hbm_budget;    /* device bytes the workers' query work spaces may
                              use in total; the batch size is capped to fit;
                              0 = no cap                                        */
    uint32_t query_flags;  /* HK_Q_* applied to every batch (HK_Q_BF16 uses the
                              tensor-core form where the index has a copy)     */
    int32_t workers;       /* concurrent batches (threads, CUDA streams); 0 = 2,
                              or 3 with persistent                            */
    int32_t persistent;    /* 1: the tensor-core scans of all batches in flight
                              run in one resident launch that takes each
                              batch's scan from a device-resident ring while
                              it runs (batches of different collections and
                              series lengths interleave in it); 0: each batch
                              launches its own kernels                        */
} hk_server_opts;

typedef struct {
    int64_t batches;       /* batches answered                                  */
    int64_t served;        /* requests answered                                 */
    int64_t max_batch;     /* largest batch so far                              */
    int64_t errors;        /* batches that failed                               */
    int64_t pending;       /* requests waiting for a batch                      */
    int64_t busy_ns;       /* summed wall time of the batches                   */
    int64_t budget_peak;   /* most device bytes the batches in flight held      */
    int64_t scan_launches; /* persistent: resident scan launches started        */
    int64_t scan_jobs;     /* persistent: batch scans published to the ring     */
    int64_t scan_jobs_inflight;  /* of those, published while a launch ran      */
    int64_t scan_max_collections; /* most collections one launch served          */
} hk_server_stats;

/*
 * A server answers exact k-NN requests against registered indexes by
 * continuous batching (Sec. 4.1: queries arrive asynchronously): each worker
 * takes the pending requests of one collection and answers them as one batch
 * with k = the batch's largest k; each request receives the first k_i entries,
 * which equal what hk_query returns for it alone.  A batch holds device
 * memory from hbm_budget until it completes; a worker admits as many pending
 * requests as the budget has room for beside the batches in flight (at least
 * one when none is), else waits for memory to free up.  With persistent = 1
 * the batches' tensor-core scans run in one resident launch, each admitted
 * batch's scan joining it while it runs.  The server does not own the
 * indexes; they must outlive it.  hk_server_destroy must not race with other
 * calls on the same server.
 */
int hk_server_create(const hk_server_opts *opts, hk_server **out);
int hk_server_add(hk_server *sv, hk_index *idx, int32_t *coll_id);
/*
 * hk_server_add_opts -- hk_server_add with the query configuration this
 * collection's batches use, e.g. the opts hk_tune chose for it (the paper
 * tunes its parameters per workload, Sec. 4.2): l_max, EAPCA_TH, SAX_TH,
 * query_group, series_tile and flags, checked as hk_query checks them
 * (HK_EINVAL otherwise).  HK_Q_TIMING and HK_Q_GRAPH are dropped.  The
 * server's query_flags do not apply to this collection.  opts NULL: as
 * hk_server_add.  Answers equal hk_query's with the same opts.
 */
int hk_server_add_opts(hk_server *sv, hk_index *idx, const hk_query_opts *opts, int32_t *coll_id);
/* q: host pointer to n floats (copied before return); k <= min(N, 1024). */
int hk_submit(hk_server *sv, int32_t coll_id, const float *q, int32_t k,
              uint64_t *ticket);
/*
 * Wait up to timeout_us for the request; on HK_OK the k ids / float32
 * distances are written (host pointers) and the ticket is released; on
 * HK_ETIMEOUT the ticket stays valid.  latency_ns (may be NULL): time from
 * hk_submit to the batch's completion.
 */
int hk_poll(hk_server *sv, uint64_t ticket, int64_t *ids, float *dist,
            int32_t timeout_us, int64_t *latency_ns);
int hk_server_stats_get(hk_server *sv, hk_server_stats *out);
int hk_server_destroy(hk_server *sv);

/* ---- tuning ------------------------------------------------------------------ */

typedef struct {
    hk_query_opts opts;     /* the fastest configuration found               */
    double ms_per_query;    /* its wall time per query on the sample          */
    int32_t tried;          /* configurations timed                           */
    int32_t tensor_cores;   /* 1: the fastest uses the precision form          */
} hk_tune_result;

/*
 * hk_tune -- choose the query path's configuration for a workload by timing
 * the candidates on a sample batch Q[nq][n] (host or device) with k
 * neighbours.  The paper tunes its parameters by hand (Sec. 4.2,
 * Parameterization); every candidate gives the same exact answer, so only
 * time decides.  Candidates: the float32 form with query_group in {2, 4, 8},
 * series_tile in {4096, 8192, 16384} and EAPCA_TH in {0.25, 1.01 (every
 * query skip-sequential)}; and, when the index has a 16-bit copy and
 * n <= 256, the precision form (HK_Q_BF16) with series_tile in {16384,
 * 32768, 65536, 131072}.  Each candidate runs once untimed, then twice
 * timed (the faster counts); a candidate whose untimed run already takes
 * over twice the best time so far is dropped.  keep_flags (HK_Q_NOSAX,
 * HK_Q_NOTHRESH) are kept in every candidate; l_max and sax_th take their
 * defaults.  The result's opts can be passed to hk_query as they are.
 */
int hk_tune(hk_index *idx, const float *Q, int32_t nq, int32_t k, uint32_t keep_flags, void *stream,
            hk_tune_result *out);

/*
 * hk_isax_breakpoints -- the 255 iSAX breakpoints the library uses
 * (Sec. 2: alphabet 256; beta_j the standard normal quantile of j/256),
 * as float32.  Host-only; needs no GPU.
 */
int hk_isax_breakpoints(float out[255]);

/* ---- inspection: copies of index internals and single steps, for tests ---- */

/*
 * hk_index_export -- copy the leaf layout to host buffers (any may be NULL):
 *   perm[N]            original id of the series at each leaf-order position
 *   leaf_off[L+1]      first position of each leaf (inorder)
 *   leaf_nseg[L]       segments of each leaf
 *   seg_end[L*64]      right endpoints of each leaf's segments (row of 64)
 *   env[L*64*4]        synopsis (mu_min, mu_max, sd_min, sd_max) per segment,
 *                      binary64 (Sec. 3.2)
 *   sax[N*16]          iSAX words in leaf order
 * L = hk_index_info.leaves; max_segments <= 64.
 */
int hk_index_export(const hk_index *idx, int64_t *perm, int64_t *leaf_off,
                    int32_t *leaf_nseg, int32_t *seg_end, double *env,
                    uint8_t *sax);

/*
 * hk_index_export_tree -- copy the whole tree (HTree, Sec. 3.3) to host
 * buffers (any may be NULL), for T = 2L - 1 nodes: leaves 0..L-1 in leaf
 * order, internal nodes L..T-1 with parents before children:
 *   parent[T], left[T], right[T]   node ids (-1: none)
 *   beg[T], end[T]                 the leaf-order positions of the node's
 *                                  series: [beg, end)
 *   nseg[T], seg_end[T*64]         segmentation (row of 64 per node)
 *   env[T*64*4]                    synopsis per segment (mu_min, mu_max,
 *                                  sd_min, sd_max) over every series that
 *                                  traversed the node (Sec. 3.3), binary64
 */
int hk_index_export_tree(const hk_index *idx, int32_t *parent, int32_t *left, int32_t *right,
                         int64_t *beg, int64_t *end, int32_t *nseg, int32_t *seg_end,
                         double *env);

/*
 * hk_debug_lb_eapca -- LB_EAPCA (squared, binary64) of each query to each
 * leaf synopsis: out[q*L + leaf].  Q host or device; out host.
 */
int hk_debug_lb_eapca(hk_index *idx, const float *Q, int32_t nq, double *out);

/*
 * hk_debug_lb_sax -- the certified lower value of LB_SAX (squared, float32)
 * that the scan compares, for each query and each series in leaf order:
 * out[q*N + pos].  Q host or device; out host.
 */
int hk_debug_lb_sax(hk_index *idx, const float *Q, int32_t nq, float *out);

/*
 * hk_debug_tc_dist -- the certified interval [lo, up] that the tensor-core
 * form puts around the squared distance of every query and every series in
 * leaf order, lo[q*N + pos], up[q*N + pos] (index built with HK_BUILD_BF16):
 * D~ = |q|^2 + |x|^2 - 2 q^.x^ (bfloat16 operands, float32 accumulation)
 * minus / plus its error bound.  Host outputs.
 */
int hk_debug_tc_dist(hk_index *idx, const float *Q, int32_t nq, float *lo, float *up);

/* ---- test hooks: no counterpart in the paper; they exist so the tests can
 *      check the library's resource and failure behaviour ---------------- */

/*
 * hk_debug_device_allocs -- *count = device allocations (cudaMalloc calls)
 * the library has made in this process so far, over all indexes, work
 * spaces and calls.  Host-only; HK_EINVAL if count is NULL.
 */
int hk_debug_device_allocs(int64_t *count);

/*
 * hk_debug_fail_device_alloc -- arm a one-shot failure: the library's
 * (after+1)-th device allocation from now fails as a failed cudaMalloc
 * would (the call returns HK_ENOMEM and releases what it allocated);
 * after < 0 disarms.  Process-wide; for tests of HK_ENOMEM handling.
 */
int hk_debug_fail_device_alloc(int64_t after);

/*
 * hk_debug_tc_wait -- the tensor-core scan's bounded waits (each mbarrier
 * wait of its producer, MMA and epilogue roles gives up after a limit and
 * the call returns HK_ETIMEOUT): limit_ns sets that limit for later calls
 * (0 = the default, 2 s); stall != 0 makes one epilogue warp of each CTA
 * wait, at its first work item, for a barrier nothing arrives at, so that
 * its wait runs out.  An aborting CTA waits (up to 200 ms) for its copies
 * and tensor-core operations in flight and frees its tensor memory before
 * it exits.  Process-wide; for tests.
 */
int hk_debug_tc_wait(uint64_t limit_ns, int32_t stall);

const char *hk_last_error(void);
const char *hk_version(void);

#ifdef __cplusplus
}
#endif
#endif /* HERCULES_GB300_H */
