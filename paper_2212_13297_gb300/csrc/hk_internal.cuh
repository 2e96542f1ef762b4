// Internal declarations of the GB300 Hercules library (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/hercules_gb300.h"

namespace hk {

constexpr int kMaxSeg = 64;          // segments a leaf may have (V-splits stop here)
constexpr int kRootSegments = 4;     // root segmentation: 4 equal segments
constexpr int kWord = HK_ISAX_SEGMENTS;
constexpr int kAlpha = HK_ISAX_ALPHABET;
constexpr int kDefaultEvalCap = 4096;
// Query parameters a zero / negative option stands for: L_max is 1 by
// default (Sec. 3.4, Approx-kNN step 1); EAPCA_TH 0.25 and SAX_TH 0.50 are
// the values of the paper's experiments (Sec. 4.2, Parameterization).
constexpr int kDefaultLMax = 1;
constexpr float kDefaultEapcaTh = 0.25f;
constexpr float kDefaultSaxTh = 0.50f;

// ---------------------------------------------------------------- errors
struct Error {
    int code;
    std::string msg;
};
[[noreturn]] void fail(int code, const char *fmt, ...);
void set_last_error(int code, const std::string &msg);
void clear_last_error();

#define HK_CHECK_CUDA(call)                                                    \
    do {                                                                       \
        cudaError_t e_ = (call);                                               \
        if (e_ != cudaSuccess)                                                 \
            ::hk::fail(e_ == cudaErrorMemoryAllocation ? HK_ENOMEM : HK_ECUDA, \
                       "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), \
                       __FILE__, __LINE__);                                    \
    } while (0)

extern thread_local long long g_launches;   // kernels launched by this thread
#define HK_CHECK_LAUNCH()                       \
    do {                                        \
        HK_CHECK_CUDA(cudaGetLastError());      \
        ++::hk::g_launches;                     \
    } while (0)

// ---------------------------------------------------------------- device memory
// Every device allocation of the library goes through DevBuf::alloc, which
// counts it (hk_debug_device_allocs) and fails it with HK_ENOMEM when a test
// armed a failure (hk_debug_fail_device_alloc).
void note_device_alloc(size_t bytes);

// Owning device buffer.  cudaMalloc/cudaFree: cudaFree waits for the device,
// so a buffer can be released whichever stream last used it.
template <class T>
struct DevBuf {
    T *p = nullptr;
    size_t n = 0;
    DevBuf() = default;
    DevBuf(const DevBuf &) = delete;
    DevBuf &operator=(const DevBuf &) = delete;
    DevBuf(DevBuf &&o) noexcept { *this = std::move(o); }
    DevBuf &operator=(DevBuf &&o) noexcept {
        if (this != &o) {
            release();
            p = o.p; n = o.n;
            o.p = nullptr; o.n = 0;
        }
        return *this;
    }
    ~DevBuf() { release(); }
    void alloc(size_t count, cudaStream_t = nullptr) {
        release();
        if (count == 0) return;
        note_device_alloc(count * sizeof(T));
        HK_CHECK_CUDA(cudaMalloc((void **)&p, count * sizeof(T)));
        n = count;
    }
    // Grow to at least count elements (contents are not kept).
    void reserve(size_t count, cudaStream_t s = nullptr) {
        if (count > n || p == nullptr) alloc(count < 1 ? 1 : count, s);
    }
    void release() {
        if (p) cudaFree(p);
        p = nullptr;
        n = 0;
    }
    size_t bytes() const { return n * sizeof(T); }
};

// ---------------------------------------------------------------- host helpers
bool is_device_ptr(const void *p);
void isax_breakpoints(float out[255]);   // library's own computation

// Exclusive scan of int32 counts on the device: out[i] = sum_{j<i} in[j],
// out[n] = total.  Stream-ordered, no host synchronisation.
void exclusive_scan_i32(const int32_t *in, int32_t *out, int64_t n, cudaStream_t s,
                        DevBuf<int32_t> &scratch);
void exclusive_scan_i64(const int32_t *in, int64_t *out, int64_t n, cudaStream_t s,
                        DevBuf<int64_t> &scratch);

// ---------------------------------------------------------------- query workspace
struct Workspace {
    DevBuf<float> Q;            // nq * n
    DevBuf<double> qseg;        // nq * S * 2  (mu, sd) per distinct segment
    DevBuf<float> sax_paa;      // nq * 32: PAA rounded down (16), then up (16)
    DevBuf<double> lb;          // nq * L
    DevBuf<uint32_t> U;         // nq   bound on the k-th distance (float bits)
    DevBuf<uint8_t> qmode;      // nq   bit0: LB_SAX filter on
    DevBuf<int32_t> qcand;      // nq   candidate leaves per query
    DevBuf<uint8_t> mask;       // L * nq  (leaf-major): 1 approx, 2 candidate
    DevBuf<int32_t> leaf_qcnt;  // L
    DevBuf<int32_t> leaf_qoff;  // L + 1
    DevBuf<int32_t> leaf_q;     // <= L * nq
    DevBuf<int32_t> leaf_items; // L
    DevBuf<int64_t> item_off;   // L + 1
    DevBuf<int32_t> counters;   // scan work counter and flags
    DevBuf<float> pool_d;       // nq * C
    DevBuf<int32_t> pool_p;     // nq * C
    DevBuf<int32_t> pool_cnt;   // nq
    DevBuf<int32_t> qflag;      // nq   bit0 overflow
    DevBuf<double> rs_d;        // nq * C  binary64 rescored distances
    DevBuf<int64_t> stats;      // counters (hk_query_stats layout)
    DevBuf<int32_t> scan_tmp32;
    DevBuf<int64_t> scan_tmp64;
    DevBuf<int64_t> out_ids;    // nq * k
    DevBuf<float> out_dist;     // nq * k
    DevBuf<int32_t> approx;     // nq * A
    DevBuf<uint16_t> Qb;        // bfloat16 queries (tensor-core form)
    DevBuf<float> q2, qa, qoff; // query |q|^2 (1-eb) - abs term, error coefficient, 2 x abs term
    DevBuf<int> bad;            // a query outside the 16-bit format's range
    DevBuf<int32_t> cand_cnt;   // nq    tensor-core candidates per query
    DevBuf<int32_t> rs_items;   // nq    rescore work items per query
    DevBuf<int32_t> rs_off;     // nq + 1  their exclusive scan
    DevBuf<int32_t> cand_p;     // nq * cand_C
    DevBuf<float> cand_lb;      // nq * cand_C  lower bound D~ - E
    DevBuf<uint32_t> Uinit;     // retry pass: starting bounds
    DevBuf<int32_t> sel;        // retry pass: rows of the batch it answers
    DevBuf<unsigned long long> tree_front;  // HK_Q_TREE: two frontiers of (node << 32 | query)
    DevBuf<int32_t> tree_cnt;   // HK_Q_TREE: frontier sizes, one per level
    struct TcEngine *engine = nullptr;   // served: tensor-core scans go to this resident launch
    // graph mode: the captured pass (reading Q, writing out_*) and its key
    cudaGraphExec_t gexec = nullptr;
    uint64_t gkey[4] = {0, 0, 0, 0};
    long long glaunches = 0;    // kernels in the graph
    cudaStream_t gstream = nullptr;   // the stream graph-mode work runs on (capturable)
    cudaEvent_t gev[2] = {nullptr, nullptr};
    Workspace() = default;
    Workspace(const Workspace &) = delete;
    Workspace &operator=(const Workspace &) = delete;
    ~Workspace() {
        drop_graph();
        if (gstream) cudaStreamDestroy(gstream);
        for (cudaEvent_t e : gev)
            if (e) cudaEventDestroy(e);
    }
    void drop_graph() {
        if (gexec) cudaGraphExecDestroy(gexec);
        gexec = nullptr;
    }
};

// Work space of DTW queries (hk_dtw.cu).
constexpr int kDtwMaxBand = 16;      // largest Sakoe-Chiba half-width
struct DtwWork {
    DevBuf<float> envL, envU, paa, pool_d, out_dist;
    DevBuf<double> qseg, lb, rs;
    DevBuf<uint8_t> mask, sel;
    DevBuf<int64_t> list, out_ids;
    DevBuf<uint32_t> U;
    DevBuf<int32_t> pool_p, pool_cnt, qflag, ctr;
    DevBuf<long long> stats;
};

// Device view of a collection laid out by leaves (an index, or a plain
// collection seen as one leaf for the exhaustive scan).
struct LeafView {
    const float *X = nullptr;       // N * n, leaf order
    const int64_t *perm = nullptr;  // position -> original id (nullptr: identity)
    const uint8_t *sax = nullptr;   // N * 16 (nullptr: no LB_SAX)
    const int64_t *leaf_off = nullptr;  // L + 1
    int64_t N = 0;
    int n = 0;
    int64_t L = 0;
};

}  // namespace hk

// ---------------------------------------------------------------- the index
struct hk_index {
    cudaStream_t stream = nullptr;
    int64_t N = 0;
    int n = 0;
    int tau = 0;
    int eval_cap = 0;
    int64_t L = 0;
    int max_m = 0;
    int depth = 0;
    int64_t S = 0;   // distinct segments over all leaves

    hk::DevBuf<float> X;           // N*n  leaf order
    hk::DevBuf<int64_t> perm;      // N
    hk::DevBuf<uint8_t> sax;       // N*16
    hk::DevBuf<int64_t> leaf_off;  // L+1
    hk::DevBuf<int32_t> leaf_nseg; // L
    hk::DevBuf<int32_t> leaf_seg;  // L*kMaxSeg distinct-segment ids
    hk::DevBuf<double> env;        // L*kMaxSeg*4
    hk::DevBuf<int32_t> seg_ab;    // S*2  (a, b)
    hk::DevBuf<float> bp;          // 255 breakpoints
    hk::DevBuf<uint16_t> Xb;       // bfloat16 copy in core-matrix order (HK_BUILD_BF16)
    hk::DevBuf<float2> xq;         // {|x|^2 (1-eb) rounded down, |x| rounded up} per series
    int64_t Npad = 0;
    bool has_bf16 = false;         // a 16-bit copy exists (format fmt16)
    int fmt16 = 1;                 // kFmtBF16 or kFmtF16
    double xn_max = 0.0;           // largest |x| (rounded up)
    hk::DevBuf<float> qstage;      // device copy of host queries (grows, kept between calls)

    std::vector<int64_t> h_leaf_off;
    std::vector<int32_t> h_leaf_nseg;
    std::vector<int32_t> h_seg_end;   // L*kMaxSeg

    // The whole tree (HTree, Sec. 3.3).  Node ids: leaves 0..L-1 in leaf
    // (inorder) order, internal nodes L..T-1, parents before children; every
    // split makes two children, so T = 2L - 1.  A node's series occupy the
    // leaf-order positions [tree_beg, tree_end).
    int64_t T = 0;
    std::vector<int32_t> h_tree_parent, h_tree_left, h_tree_right, h_tree_level;   // T
    std::vector<int64_t> h_tree_beg, h_tree_end;                                   // T
    std::vector<int32_t> h_inode_nseg;       // T - L
    std::vector<int32_t> h_inode_seg_end;    // (T - L) * kMaxSeg
    std::vector<int32_t> h_inode_seg;        // (T - L) * kMaxSeg distinct-segment ids
    hk::DevBuf<int32_t> tree_parent, tree_left, tree_right;   // T
    hk::DevBuf<int64_t> tree_beg, tree_end;                   // T
    hk::DevBuf<int32_t> inode_nseg;          // T - L
    hk::DevBuf<int32_t> inode_seg;           // (T - L) * kMaxSeg distinct-segment ids
    hk::DevBuf<double> ienv;                 // (T - L) * kMaxSeg * 4 internal synopses
    std::vector<int32_t> h_level_off;        // depth + 2: nodes of level d are
    hk::DevBuf<int32_t> level_nodes;         //   level_nodes[h_level_off[d] .. h_level_off[d+1])

    hk::Workspace ws;
    hk::Workspace ws_retry;
    hk::Workspace ws_graph;    // HK_Q_GRAPH calls only: its buffers stay where the graph points
    hk::DtwWork dtw;           // hk_query_dtw
};

namespace hk {
// Build (hk_build.cu)
void build_index(hk_index *idx, const float *X, int64_t N, int n, const hk_build_opts &o,
                 cudaStream_t s);
// Device copies of the tree arrays (from the h_tree_* / h_inode_* vectors);
// sizes ienv (filled by the caller).  Also forms the level lists.
void upload_tree(hk_index *idx, cudaStream_t s);
// The checks hk_query applies to its options on this index (HK_EINVAL).
void check_query_opts(const hk_index *idx, const hk_query_opts &o);
// Query (hk_query.cu)
void run_query(hk_index *idx, const float *Qdev, int nq, int k, const hk_query_opts &o,
               cudaStream_t s, int64_t *out_ids_host_or_dev, float *out_dist_host_or_dev,
               hk_query_stats *stats);
// The same with caller-owned work spaces (one pair per concurrent caller).
void run_query_ws(hk_index *idx, Workspace &ws, Workspace &ws_retry, const float *Qdev, int nq, int k,
                  const hk_query_opts &o, cudaStream_t s, int64_t *out_ids, float *out_dist,
                  hk_query_stats *stats);
void run_scan(const float *Xdev, int64_t N, int n, const float *Qdev, int nq, int k,
              cudaStream_t s, int64_t *out_ids, float *out_dist);
// DTW (hk_dtw.cu)
void run_query_dtw(hk_index *idx, const float *Qd, int nq, int k, int band, const hk_query_opts &o,
                   cudaStream_t s, int64_t *out_ids, float *out_dist, hk_query_stats *stats);
void debug_lb_eapca(hk_index *idx, const float *Qdev, int nq, double *out_host);
void debug_lb_sax(hk_index *idx, const float *Qdev, int nq, float *out_host);
void debug_tc_dist(hk_index *idx, const float *Qdev, int nq, float *lo_host, float *up_host);
void check_finite(const float *p, int64_t count, cudaStream_t s, const char *what);
void check_finite_with(const float *p, int64_t count, cudaStream_t s, const char *what,
                       unsigned long long *dev_counter);

// Device buffers, carved by the caller from memory it already owns, for an
// exhaustive scan that allocates nothing (see hk_noalloc.cu).
struct ScanScratch {
    uint32_t *U;             // nq
    float *pool_d;           // nq * pool_C
    int32_t *pool_p;         // nq * pool_C
    double *rs_d;            // nq * pool_C
    int32_t *pool_cnt;       // nq
    int32_t *qflag;          // nq
    int32_t *leaf_qoff;      // 2
    int32_t *leaf_q;         // nq
    int64_t *item_off;       // 2
    int64_t *leaf_off;       // 2
    int32_t *counters;       // 4
    long long *stats;        // 24
    float *col_d;            // col_cap
    int32_t *col_p;          // col_cap
    double *col_r;           // col_cap
    int32_t *col_cnt;        // 2
    int32_t *qsel;           // 1
    int pool_C;
    int col_cap;
    int max_nq;
};
// Arguments of the tensor-core distance scan (hk_tc.cu).
struct TcArgs {
    const uint16_t *Xb;          // bfloat16 collection, core-matrix order, padded rows
    const float2 *xq;            // per position: {|x|^2 (1-eb) rounded down, |x| rounded up}
    int n;
    const uint16_t *Qb;          // bfloat16 queries, row-major
    const float *q2e, *qa;       // per query: |q|^2 (1-eb) - abs term rounded down, c |q| rounded up
    const float *qoff2;          // per query: twice the absolute error term
    float eb2;                   // 2 eb / (1 - eb) with margin: the upper bound's norm term
    const int64_t *leaf_off;
    int64_t L;
    const int32_t *leaf_qoff, *leaf_q;
    const int64_t *item_off;
    int32_t *work_ctr;
    int S_T;
    uint32_t *U;
    int k;
    int32_t *cand_cnt, *cand_p;
    float *cand_lb;
    int cand_C;
    int32_t *qflag;
    int32_t *err;
    long long *stats;
    int stat_pairs, stat_cands, stat_bytes;
    uint32_t idesc;
    float *dbg_lo, *dbg_up;      // if set: certified interval of every pair, [q * N + pos]
    int64_t N;
    uint64_t wait_ns;            // limit of each bounded wait (0: the default, 2 s)
    int dbg_stall;               // test hook: one epilogue warp per CTA waits for a barrier
                                 // nothing arrives at, so its wait runs out (HK_ETIMEOUT)
};
// Test hooks of the tensor-core scan's bounded waits (hk_debug_tc_wait).
void tc_wait_hooks(uint64_t &wait_ns, int &stall);

// Served form of the tensor-core scan: one resident launch takes the scans
// of many batches (jobs) from a ring as they are published.
constexpr int kTcRing = 64;          // jobs in flight at most, per lane
constexpr int kTcLanes = 2;          // lane 0 (approximate steps) is served before lane 1
struct TcJob {                       // device memory, written before publication
    TcArgs args;
    int64_t total;                   // work items of the job (> 0)
    uint32_t seq;                    // publication number
    uint32_t pad;
};
struct TcServe {                     // the served launch's view of the ring's lanes
    TcJob *jobs;                     // kTcLanes * kTcRing (lane-major)
    unsigned long long *word;        // per lane: (sequence of its current job << 32) | next item
    int32_t *done;                   // kTcLanes * kTcRing items finished per slot
    const volatile uint32_t *published;   // host-mapped, per lane: jobs published so far
    volatile uint32_t *done_seq;     // host-mapped, kTcLanes * kTcRing: last completed sequence
    uint64_t idle_ns;                // a CTA leaves after this long without work
};
struct TcEngine;                     // host side (hk_tc.cu)
TcEngine *tc_engine_create(int spare_sms);
void tc_engine_destroy(TcEngine *e);
// Publish one scan (arguments as for launch_tc_scan, `items` work items) to
// the served launch (starting it if none runs) and wait, bounded by
// timeout_ns, until its items are done.  The caller's stream must have
// produced the scan's inputs already (synchronised).
void tc_engine_run(TcEngine *e, const TcArgs &a, int64_t items, uint64_t timeout_ns, int lane);
struct TcEngineStats {
    long long launches;              // served launches started
    long long jobs;                  // jobs published
    long long jobs_inflight;         // of those, published while a launch was running
    long long max_colls_per_launch;  // most distinct collections one launch served
};
void tc_engine_stats(TcEngine *e, TcEngineStats *out);
void launch_tc_scan(const TcArgs &a, cudaStream_t s);
constexpr int kFmtF16 = 0;    // tcgen05 kind::f16 operand encodings
constexpr int kFmtBF16 = 1;
void launch_make_16(const float *X, int64_t N, int n, int64_t Npad, int fmt, void *Xb, void *xq,
                    int *bad, cudaStream_t s);
void launch_tc_qprep(const float *Q, int nq, int n, int fmt, double xn_max, void *Qb, float *q2e,
                     float *qa, float *qoff2, int *bad, cudaStream_t s);
void launch_tc_rescore(const float *Q, const float *X, int n, int nq, const int32_t *cand_cnt,
                       const int32_t *cand_p, const float *cand_lb, int cand_C, const uint32_t *U,
                       float *pool_d, int32_t *pool_p, int32_t *pool_cnt, int pool_C, int32_t *qflag,
                       long long *stats, int stat_slot, int32_t *items, int32_t *item_off,
                       DevBuf<int32_t> &scan_tmp, cudaStream_t s);
size_t tc_smem_bytes(int n);
void launch_max_norm(const void *xq, int64_t N, unsigned *out, cudaStream_t s);
uint32_t tc_idesc(int fmt);
double tc_error_coefficient(int n, int fmt);
float tc_eb2();
constexpr int kTcMaxLen = 256;     // longest series the tensor-core form takes
constexpr int kTcLocalK = 16;     // largest k whose best upper bounds the tensor-core scan tracks
// Candidate-list and pool length per query in the precision form: its
// certified band admits the near neighbours around the k-th distance, more
// of them as k grows (an overflow reruns the query on the float32 path).
// At least 262,144: with a bfloat16 copy (band 8x float16's) hard queries
// average about 9K candidates at 100M x 256, with a tail past 65K.
inline int tc_list_cap(int k) {
    const int c = k * 4096 < (1 << 20) ? k * 4096 : (1 << 20);
    return c > 262144 ? c : 262144;
}

// Exhaustive exact k-NN into caller device buffers using only `sc`.
void scan_knn_scratch(const float *Xd, int64_t N, int n, const float *Qd, int nq, int k,
                      cudaStream_t s, int64_t *ids_dev, float *dist_dev, const ScanScratch &sc);
}  // namespace hk
