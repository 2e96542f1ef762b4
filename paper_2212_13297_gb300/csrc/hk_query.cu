// Exact k-NN query answering on the GPU (Sec. 3.4, Algorithm Exact-kNN).
//
// A batch of queries is answered together.  Per query the steps are the
// paper's: the approximate search scans the leaves with the smallest
// LB_EAPCA (Approx-kNN; with lower bounds that grow from parent to child,
// best-first order over the tree is ascending leaf LB order) and sets BSF_k;
// leaves whose LB_EAPCA cannot beat BSF_k are pruned (FindCandidateLeaves);
// within the remaining leaves LB_SAX prunes series (CSWorker) unless pruning
// was too weak (EAPCA_TH, then the leaves are scanned whole as in the
// skip-sequential scan); the rest get their squared Euclidean distance with
// early abandoning and update the k best (CRWorker).
//
// GPU organisation: work is leaf-major.  A work item is one tile of a leaf's
// series and a group of up to G queries for which that leaf is a candidate;
// its CTA reads each series once for all of them.  Each item keeps, per
// query, a sorted list of its best candidates in shared memory and publishes
// them to a per-query pool at the end; the k-th entry of a list bounds the
// query's k-th distance, so it tightens a global per-query bound U (atomicMin)
// that every later item prunes and abandons against.
//
// Exactness.  Distances here are float32; the answer is ranked by the
// binary64 squared distance summed in index order (ties to the lower id).
// With rho >= gamma_{n+2} = (n+2)u/(1-(n+2)u), u = 2^-24, every float32
// distance or partial sum s of a true (real) value D satisfies
// s <= D(1+rho) and D <= s(1+rho).  U is always an upper bound on the true
// k-th distance (the (1+rho)-inflated k-th float32 distance of some k
// series), and a series is dropped only when a certified lower bound on its
// distance (LB_EAPCA, LB_SAX, or a partial sum) exceeds U, or when its
// float32 distance exceeds T(U) = U(1+rho) rounded up.  The final step
// recomputes in binary64 every pooled candidate at or below T(U_final) and
// ranks them by (binary64 distance, id).  If a list or pool overflows (more
// near-ties than it holds), that query is answered again on the float32 path
// starting from its final bound (tight, so few candidates qualify); if that
// overflows too, every series at or below T(U_final) is collected
// exhaustively.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <vector>

#include <cuda_fp16.h>

#include "hk_device.cuh"
#include "hk_internal.cuh"

namespace hk {
namespace {

constexpr int kBT = 128;       // scan CTA threads = series per chunk
constexpr int kSlack = 32;     // room for near-ties beyond k in an item list
constexpr int kRing = 2;       // scan: chunks (2 KB per warp) in flight per warp
constexpr int kRound1Leaves = 8;   // precision form, k > 16: leaves per query in the first round
constexpr int kMaxG = 8;
constexpr int kStatSlots = 32;
constexpr int kAmax = 256;     // most leaves the approximate step visits

enum StatIdx {
    ST_QUERIES = 0, ST_LEAVES_TOTAL, ST_LEAVES_APPROX, ST_LEAVES_CAND, ST_SERIES_CAND,
    ST_SAX_PRUNED, ST_ABANDONED, ST_FULL, ST_POINTS, ST_RESCORED, ST_FALLBACK,
    ST_ITEMS, ST_SKIPSEQ, ST_SCAN_NS, ST_LAUNCHES, ST_SCAN_BYTES, ST_RETRIED, ST_TC_PAIRS,
    ST_TC_CANDS, ST_TC_BYTES, ST_TCA_PAIRS, ST_TCA_CANDS, ST_TCA_BYTES, ST_TC_LEAF_BYTES, ST_LB_EVALS,
    ST_COUNT
};
static_assert(ST_COUNT <= kStatSlots, "stat slots");

struct ScanArgs {
    LeafView v;
    const float *Q;
    int nq;
    const float *sax_paa;      // nq*32: PAA rounded down (16), then up (16); nullptr: no LB_SAX
    const float *bp;           // the 255 iSAX breakpoints
    const uint8_t *qmode;      // nq (bit0: LB_SAX on) or nullptr
    const double *lb;          // nq*L or nullptr
    uint32_t *U;               // nq float bits
    const int32_t *leaf_qoff;  // L+1
    const int32_t *leaf_q;
    const int64_t *item_off;   // L+1
    int32_t *work_ctr;
    int S_T;
    int k;
    int cap;                   // list capacity
    int p2;                    // sort length (power of two >= cap + kBT)
    float rho;
    float *pool_d;
    int32_t *pool_p;
    int32_t *pool_cnt;
    int pool_C;
    int32_t *qflag;
    long long *stats;
    int use_sax;
};

__device__ __forceinline__ float upper_f(float d, float rho) { return __fmul_ru(d, 1.0f + rho); }

// --------------------------------------------------------------------------
// a1: query preparation.  Per query: mean and std of every distinct leaf
// segment (binary64, the build's exact definition) and the PAA over 16
// segments (binary64) bracketed by the float32 values just below and just
// above it, from which the scan forms LB_SAX rounded down.
__global__ void k_qprep(const float *__restrict__ Q, int n, const int32_t *__restrict__ seg_ab,
                        int64_t S, double *__restrict__ qseg, float *__restrict__ paa_out) {
    extern __shared__ float qs[];
    const int q = blockIdx.x;
    for (int j = threadIdx.x; j < n; j += blockDim.x) qs[j] = Q[(int64_t)q * n + j];
    __syncthreads();
    if (qseg) {
        for (int64_t s = threadIdx.x; s < S; s += blockDim.x) {
            double mu, sd;
            seg_stats64(qs, seg_ab[2 * s], seg_ab[2 * s + 1], mu, sd);
            qseg[((int64_t)q * S + s) * 2] = mu;
            qseg[((int64_t)q * S + s) * 2 + 1] = sd;
        }
    }
    if (paa_out && threadIdx.x < kWord) {
        // PAA (binary64) bracketed by float32 values below and above it
        const int l = n / kWord;
        const double m = seg_mean64(qs, threadIdx.x * l, (threadIdx.x + 1) * l);
        paa_out[(int64_t)q * 2 * kWord + threadIdx.x] = __double2float_rd(m);
        paa_out[(int64_t)q * 2 * kWord + kWord + threadIdx.x] = __double2float_ru(m);
    }
}

// a5: LB_SAX of one iSAX word against one query, rounded down at every
// step, so it never exceeds the exact value (binary64 PAA against the
// float32 cells).  B[257]: -inf, the 255 breakpoints, +inf (cell of symbol s
// is [B[s], B[s+1])); lo, hi: the word's cells; paa_lo / paa_hi: the query's
// PAA rounded down / up; w = n/16.
__device__ __forceinline__ float lb_sax_lower(const float (&lo)[kWord], const float (&hi)[kWord],
                                             const float *paa_lo, const float *paa_hi, float w) {
    float acc = 0.0f;
#pragma unroll
    for (int i = 0; i < kWord; ++i) {
        const float a = __fsub_rd(lo[i], paa_hi[i]);   // <= cell's low end - PAA
        const float b = __fsub_rd(paa_lo[i], hi[i]);   // <= PAA - cell's high end
        const float d = fmaxf(fmaxf(a, b), 0.0f);
        acc = __fmaf_rd(d, d, acc);
    }
    return __fmul_rd(acc, w);
}

__device__ __forceinline__ void sax_cells(uint4 w4, const float *B, float (&lo)[kWord], float (&hi)[kWord]) {
    const uint32_t wv[4] = {w4.x, w4.y, w4.z, w4.w};
#pragma unroll
    for (int i = 0; i < kWord; ++i) {
        const int sym = (wv[i >> 2] >> ((i & 3) * 8)) & 0xff;
        lo[i] = B[sym];
        hi[i] = B[sym + 1];
    }
}

// The synopses of every node of the tree: leaves 0..L-1 (leaf tables),
// internal nodes L..T-1 (internal tables), links and levels.
struct TreeView {
    int64_t L, T;
    const int32_t *leaf_nseg, *leaf_seg;    // L, L * kMaxSeg distinct-segment ids
    const double *env;                      // L * kMaxSeg * 4
    const int32_t *inode_nseg, *inode_seg;  // T - L, (T - L) * kMaxSeg
    const double *ienv;                     // (T - L) * kMaxSeg * 4
    const int32_t *seg_ab;                  // S * 2
    const int32_t *parent, *left, *right;   // T
    const int64_t *beg, *end;               // T: leaf-order position ranges
};

// LB_EAPCA (squared, binary64) of query q to node u's synopsis: the segment
// sum in segment order, exactly the definition (Sec. 2, Sec. 3.4).
__device__ __forceinline__ double node_lb(const TreeView &t, const double *__restrict__ qseg, int64_t S,
                                          int q, int64_t u) {
    const bool leaf = u < t.L;
    const int64_t j0 = leaf ? u : u - t.L;
    const int m = leaf ? t.leaf_nseg[j0] : t.inode_nseg[j0];
    const int32_t *segs = (leaf ? t.leaf_seg : t.inode_seg) + j0 * kMaxSeg;
    const double *env = (leaf ? t.env : t.ienv) + j0 * kMaxSeg * 4;
    double acc = 0.0;
    for (int j = 0; j < m; ++j) {
        const int sid = segs[j];
        const double l = (double)(t.seg_ab[2 * sid + 1] - t.seg_ab[2 * sid]);
        const double mu = qseg[((int64_t)q * S + sid) * 2];
        const double sd = qseg[((int64_t)q * S + sid) * 2 + 1];
        const double *z = env + j * 4;
        const double dm = dist_to_range64(mu, z[0], z[1]);
        const double ds = dist_to_range64(sd, z[2], z[3]);
        const double tt = __dadd_rn(__dmul_rn(dm, dm), __dmul_rn(ds, ds));
        acc = __dadd_rn(acc, __dmul_rn(l, tt));
    }
    return acc;
}

// a2: LB_EAPCA of every query to every leaf synopsis.
__global__ void k_lb_eapca(const double *__restrict__ qseg, int64_t S, TreeView tv, int nq,
                           double *__restrict__ lb) {
    const int64_t leaf = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (leaf >= tv.L) return;
    for (int q = blockIdx.y; q < nq; q += gridDim.y) lb[(int64_t)q * tv.L + leaf] = node_lb(tv, qseg, S, q, leaf);
}

// Certified lower value of a binary64 LB (absorbs its rounding).
__device__ __forceinline__ double lb_lower(double lb) { return __dmul_rd(lb, 1.0 - 0x1p-40); }

constexpr int kHeapCap = 512;   // tree mode: queue entries per query

// a3 with HK_Q_TREE: the approximate search as the paper's best-first
// traversal (Approx-kNN, Sec. 3.4): a priority queue of nodes keyed by
// LB_EAPCA, starting at the root; an internal node taken from it puts its two
// children in, a leaf taken from it is visited, until at least l_max leaves
// and k series.  One thread per query walks its queue in shared memory (four
// queries per block).  A full queue drops the node being added; if the queue
// then runs dry before k series, the remaining leaves are taken in ascending
// leaf-LB order.  Any visited leaves give a valid bound U.
__global__ void __launch_bounds__(128) k_tree_approx(const double *__restrict__ qseg, int64_t S, TreeView tv,
                                                     int root, int l_max, int k, int nq, int amax,
                                                     int32_t *__restrict__ approx, int32_t *__restrict__ napprox,
                                                     uint8_t *__restrict__ mask, double *__restrict__ lb,
                                                     long long *__restrict__ stats) {
    __shared__ double keys_s[4][kHeapCap];
    __shared__ int32_t node_s[4][kHeapCap];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int q = blockIdx.x * 4 + warp;
    if (q >= nq || lane != 0) return;
    double *hk = keys_s[warp];
    int32_t *hn = node_s[warp];
    int hs = 0;
    auto less = [&](int i, int j) { return hk[i] < hk[j] || (hk[i] == hk[j] && hn[i] < hn[j]); };
    auto swap = [&](int i, int j) {
        const double a = hk[i]; hk[i] = hk[j]; hk[j] = a;
        const int32_t b = hn[i]; hn[i] = hn[j]; hn[j] = b;
    };
    auto push = [&](double key, int32_t node) {
        int i = hs++;
        hk[i] = key;
        hn[i] = node;
        while (i > 0 && less(i, (i - 1) / 2)) {
            swap(i, (i - 1) / 2);
            i = (i - 1) / 2;
        }
    };
    auto pop = [&](double &key, int32_t &node) {
        key = hk[0];
        node = hn[0];
        --hs;
        hk[0] = hk[hs];
        hn[0] = hn[hs];
        int i = 0;
        for (;;) {
            const int l = 2 * i + 1, r = l + 1;
            int m = i;
            if (l < hs && less(l, m)) m = l;
            if (r < hs && less(r, m)) m = r;
            if (m == i) break;
            swap(i, m);
            i = m;
        }
    };
    long long evals = 1;
    push(node_lb(tv, qseg, S, q, root), root);
    int nch = 0;
    long long covered = 0;
    while (hs > 0 && nch < amax && (nch < l_max || covered < k)) {
        double key;
        int32_t u;
        pop(key, u);
        if (u < tv.L) {
            approx[(int64_t)q * amax + nch++] = u;
            mask[(int64_t)u * nq + q] = 1;
            covered += tv.end[u] - tv.beg[u];
            lb[(int64_t)q * tv.L + u] = key;
        } else {
            for (int c = 0; c < 2; ++c) {
                const int32_t v = c ? tv.right[u] : tv.left[u];
                const double key_v = node_lb(tv, qseg, S, q, v);
                ++evals;
                if (hs < kHeapCap) push(key_v, v);
            }
        }
    }
    while (nch < amax && covered < k) {
        // the queue ran dry after dropping nodes: ascending (leaf LB, leaf)
        double best = INFINITY;
        int64_t bl = -1;
        for (int64_t f = 0; f < tv.L; ++f) {
            if (mask[f * nq + q] != 0) continue;
            const double v = node_lb(tv, qseg, S, q, f);
            ++evals;
            if (bl < 0 || v < best) { best = v; bl = f; }
        }
        if (bl < 0) break;
        approx[(int64_t)q * amax + nch++] = (int32_t)bl;
        mask[bl * nq + q] = 1;
        covered += tv.end[bl] - tv.beg[bl];
        lb[(int64_t)q * tv.L + bl] = best;
    }
    napprox[q] = nch;
    stat_add(&stats[ST_LB_EVALS], evals);
}

// a4 with HK_Q_TREE: candidate leaves by a top-down pass over the tree
// (FindCandidateLeaves over the hierarchy of node synopses, Sec. 3.3-3.4).
// A frontier holds the (internal node, query) pairs that stayed at one
// level; each pass evaluates LB_EAPCA for the two children of every pair in
// it and keeps a child unless its certified LB exceeds U: every series below
// a node is at least the node's LB away, so a pruned node prunes its whole
// subtree, and the work follows the pairs that stay.  A leaf that stays
// becomes a candidate unless the approximate search visited it; an internal
// node goes to the next frontier.  A pair is packed as (node << 32) | query.
__global__ void k_tree_expand(const double *__restrict__ qseg, int64_t S, TreeView tv,
                              const unsigned long long *__restrict__ in, const int32_t *__restrict__ n_in,
                              unsigned long long *__restrict__ out, int32_t *__restrict__ n_out, int nq,
                              const uint32_t *__restrict__ U, uint8_t *__restrict__ mask,
                              int32_t *__restrict__ qcand, double *__restrict__ lb, long long *__restrict__ stats) {
    const int cnt = *n_in;
    const int lane = threadIdx.x & 31;
    long long ev = 0;
    for (int64_t i0 = (int64_t)blockIdx.x * blockDim.x; i0 < 2 * (int64_t)cnt;
         i0 += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = i0 + threadIdx.x;
        bool push = false;
        unsigned long long pair = 0;
        if (i < 2 * (int64_t)cnt) {
            const unsigned long long p = in[i >> 1];
            const int64_t u = (int64_t)(p >> 32);
            const int q = (int)(p & 0xffffffffu);
            const int64_t c = (i & 1) ? tv.right[u] : tv.left[u];
            const double v = node_lb(tv, qseg, S, q, c);
            ++ev;
            const bool stays = !(lb_lower(v) > (double)__uint_as_float(U[q]));
            if (c < tv.L) {
                lb[(int64_t)q * tv.L + c] = v;
                if (stays && mask[c * nq + q] == 0) {
                    mask[c * nq + q] = 2;
                    atomicAdd(&qcand[q], 1);
                }
            } else if (stays) {
                push = true;
                pair = ((unsigned long long)c << 32) | (unsigned)q;
            }
        }
        // warp-aggregated append to the next frontier
        const unsigned bal = __ballot_sync(0xffffffffu, push);
        int base = 0;
        if (lane == 0 && bal) base = atomicAdd(n_out, __popc(bal));
        base = __shfl_sync(0xffffffffu, base, 0);
        if (push) out[base + __popc(bal & ((1u << lane) - 1))] = pair;
    }
    ev = warp_sum_ll(ev);
    if (lane == 0 && ev) stat_add(&stats[ST_LB_EVALS], ev);
}

// The first frontier: the root for every query whose root LB stays (one
// evaluation per query); a single-leaf tree makes its leaf a candidate.
__global__ void k_tree_root(const double *__restrict__ qseg, int64_t S, TreeView tv, int64_t root, int nq,
                            const uint32_t *__restrict__ U, unsigned long long *__restrict__ out,
                            int32_t *__restrict__ n_out, uint8_t *__restrict__ mask, int32_t *__restrict__ qcand,
                            double *__restrict__ lb, long long *__restrict__ stats) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nq) return;
    const double v = node_lb(tv, qseg, S, q, root);
    stat_add(&stats[ST_LB_EVALS], 1);
    const bool stays = !(lb_lower(v) > (double)__uint_as_float(U[q]));
    if (root < tv.L) {
        lb[(int64_t)q * tv.L + root] = v;
        if (stays && mask[root * nq + q] == 0) {
            mask[root * nq + q] = 2;
            atomicAdd(&qcand[q], 1);
        }
    } else if (stays) {
        out[atomicAdd(n_out, 1)] = ((unsigned long long)root << 32) | (unsigned)q;
    }
}

// a3 (selection): the leaves the approximate search visits: ascending
// (LB_EAPCA, leaf) until at least l_max leaves and at least k series.
__global__ void k_approx_select(const double *__restrict__ lb, int64_t L,
                                const int64_t *__restrict__ leaf_off, int l_max, int k, int nq,
                                int amax, int32_t *__restrict__ approx, int32_t *__restrict__ napprox,
                                uint8_t *__restrict__ mask) {
    __shared__ double bd[32];
    __shared__ long long bl[32];
    __shared__ int chosen[kAmax];
    __shared__ int nch;
    __shared__ long long covered;
    const int q = blockIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) { nch = 0; covered = 0; }
    __syncthreads();
    for (;;) {
        if (!(nch < amax && (nch < l_max || covered < k))) break;
        double best = INFINITY;
        long long bleaf = -1;
        for (int64_t f = threadIdx.x; f < L; f += blockDim.x) {
            bool taken = false;
            for (int c = 0; c < nch; ++c) taken |= (chosen[c] == (int)f);
            if (taken) continue;
            const double v = lb[(int64_t)q * L + f];
            if (bleaf < 0 || v < best || (v == best && f < bleaf)) { best = v; bleaf = f; }
        }
        for (int o = 16; o > 0; o >>= 1) {
            const double ov = __shfl_xor_sync(0xffffffffu, best, o);
            const long long ol = __shfl_xor_sync(0xffffffffu, bleaf, o);
            if (ol >= 0 && (bleaf < 0 || ov < best || (ov == best && ol < bleaf))) { best = ov; bleaf = ol; }
        }
        if (lane == 0) { bd[warp] = best; bl[warp] = bleaf; }
        __syncthreads();
        if (threadIdx.x == 0) {
            double b = INFINITY;
            long long f = -1;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w)
                if (bl[w] >= 0 && (f < 0 || bd[w] < b || (bd[w] == b && bl[w] < f))) { b = bd[w]; f = bl[w]; }
            if (f < 0) {
                covered = (long long)1 << 62;   // nothing left: stop
                chosen[nch] = -1;
            } else {
                chosen[nch] = (int)f;
                approx[(int64_t)q * amax + nch] = (int)f;
                mask[f * nq + q] = 1;
                covered += leaf_off[f + 1] - leaf_off[f];
                nch = nch + 1;
            }
        }
        __syncthreads();
        if (covered >= ((long long)1 << 62)) break;
    }
    if (threadIdx.x == 0) napprox[q] = nch;
}

// a4: leaf prune (FindCandidateLeaves): a leaf stays a candidate for a query
// unless its certified LB_EAPCA exceeds U.
__global__ void k_mask_candidates(const double *__restrict__ lb, int64_t L, int nq,
                                  const uint32_t *__restrict__ U, int noprune,
                                  uint8_t *__restrict__ mask, int32_t *__restrict__ qcand) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= L * (int64_t)nq) return;
    const int64_t leaf = t / nq;
    const int q = (int)(t % nq);
    if (mask[t] != 0) return;
    bool cand = noprune != 0;
    if (!cand) {
        const double u = (double)__uint_as_float(U[q]);
        cand = !(lb_lower(lb[(int64_t)q * L + leaf]) > u);
    }
    if (cand) {
        mask[t] = 2;
        atomicAdd(&qcand[q], 1);
    }
}

// Precision form, k beyond what the tensor-core scan tightens in flight:
// each query's `r` candidate leaves (mask 2) with the smallest LB_EAPCA go
// first (mask 3), as in the paper's best-first order of the leaves
// (Sec. 3.4, Exact-kNN), so that U is exact over many series before the rest.
__global__ void k_round1_select(const double *__restrict__ lb, int64_t L, int nq, int r,
                                uint8_t *__restrict__ mask) {
    __shared__ double bd[32];
    __shared__ long long bl[32];
    const int q = blockIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int it = 0; it < r; ++it) {
        double best = INFINITY;
        long long bleaf = -1;
        for (int64_t f = threadIdx.x; f < L; f += blockDim.x) {
            if (mask[f * nq + q] != 2) continue;
            const double v = lb[(int64_t)q * L + f];
            if (bleaf < 0 || v < best || (v == best && f < bleaf)) { best = v; bleaf = f; }
        }
        for (int o = 16; o > 0; o >>= 1) {
            const double ov = __shfl_xor_sync(0xffffffffu, best, o);
            const long long ol = __shfl_xor_sync(0xffffffffu, bleaf, o);
            if (ol >= 0 && (bleaf < 0 || ov < best || (ov == best && ol < bleaf))) { best = ov; bleaf = ol; }
        }
        if (lane == 0) { bd[warp] = best; bl[warp] = bleaf; }
        __syncthreads();
        if (threadIdx.x == 0) {
            double b = INFINITY;
            long long f = -1;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w)
                if (bl[w] >= 0 && (f < 0 || bd[w] < b || (bd[w] == b && bl[w] < f))) { b = bd[w]; f = bl[w]; }
            if (f >= 0) mask[f * nq + q] = 3;
            bl[0] = f;
        }
        __syncthreads();
        const bool done = bl[0] < 0;
        __syncthreads();
        if (done) break;
    }
}

// After the first round: candidate leaves (mask 2) whose certified LB now
// exceeds U drop out.
__global__ void k_reprune(const double *__restrict__ lb, int64_t L, int nq, const uint32_t *__restrict__ U,
                          uint8_t *__restrict__ mask, long long *__restrict__ stats) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= L * (int64_t)nq) return;
    if (mask[t] != 2) return;
    const int64_t leaf = t / nq;
    const int q = (int)(t % nq);
    if (lb_lower(lb[(int64_t)q * L + leaf]) > (double)__uint_as_float(U[q])) {
        mask[t] = 0;
        stat_add(&stats[ST_LEAVES_CAND], -1);
    }
}

// Per-query mode: LB_SAX filter on unless disabled or EAPCA pruning fell
// below EAPCA_TH (then the candidate leaves are scanned whole).
__global__ void k_qmode(const int32_t *__restrict__ qcand, int64_t L, int nq, float eapca_th,
                        int nosax, int nothresh, uint8_t *__restrict__ qmode,
                        long long *__restrict__ stats) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nq) return;
    const double pr = 1.0 - (double)qcand[q] / (double)L;
    int on = nosax ? 0 : 1;
    if (on && !nothresh && pr < (double)eapca_th) {
        on = 0;
        stat_add(&stats[ST_SKIPSEQ], 1);
    }
    qmode[q] = (uint8_t)on;
    stat_add(&stats[ST_LEAVES_CAND], qcand[q]);
}

// Leaf-major lists: per leaf, the queries whose mask equals v, and the number
// of work items (query groups x series tiles).
__global__ void k_leaf_count(const uint8_t *__restrict__ mask, int nq, uint8_t v,
                             const int64_t *__restrict__ leaf_off, int G, int S_T,
                             int32_t *__restrict__ qcnt, int32_t *__restrict__ items) {
    __shared__ int red[32];
    const int64_t leaf = blockIdx.x;
    int c = 0;
    for (int q = threadIdx.x; q < nq; q += blockDim.x) c += mask[leaf * nq + q] == v;
    c = warp_sum_i(c);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        int tot = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot += red[w];
        qcnt[leaf] = tot;
        const int64_t size = leaf_off[leaf + 1] - leaf_off[leaf];
        const int64_t tiles = (size + S_T - 1) / S_T;
        items[leaf] = tot == 0 ? 0 : (int32_t)(((tot + G - 1) / G) * tiles);
    }
}

__global__ void k_leaf_fill(const uint8_t *__restrict__ mask, int nq, uint8_t v,
                            const int32_t *__restrict__ qoff, int32_t *__restrict__ leaf_q) {
    __shared__ int wsum[32];
    __shared__ int base;
    const int64_t leaf = blockIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (threadIdx.x == 0) base = qoff[leaf];
    __syncthreads();
    for (int q0 = 0; q0 < nq; q0 += blockDim.x) {
        const int q = q0 + threadIdx.x;
        const bool hit = q < nq && mask[leaf * nq + q] == v;
        const unsigned bal = __ballot_sync(0xffffffffu, hit);
        if (lane == 0) wsum[warp] = __popc(bal);
        __syncthreads();
        int off = 0;
        for (int w = 0; w < warp; ++w) off += wsum[w];
        if (hit) leaf_q[base + off + __popc(bal & ((1u << lane) - 1))] = q;
        __syncthreads();
        if (threadIdx.x == 0) {
            int tot = 0;
            for (int w = 0; w < nw; ++w) tot += wsum[w];
            base += tot;
        }
        __syncthreads();
    }
}

// 16-byte asynchronous copy global -> shared (L2 only), and its groups.
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(smem)),
                 "l"(gmem)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// max(a, b, c) in one instruction (three-input max.f32, sm_100 and later).
__device__ __forceinline__ float max3f(float a, float b, float c) {
    float r;
    asm("max.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}

// Packed float32 pairs (the f32x2 pipes): a += (q - x)^2 lane-wise.
__device__ __forceinline__ uint64_t pack2(float lo, float hi) {
    uint64_t r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ void unpack2(uint64_t v, float &lo, float &hi) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ uint64_t sub_rd2(uint64_t a, uint64_t b) {
    uint64_t d;
    asm("sub.rm.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ uint64_t sqacc_rd2(uint64_t d, uint64_t acc) {
    uint64_t r;
    asm("fma.rm.f32x2 %0, %1, %1, %2;" : "=l"(r) : "l"(d), "l"(acc));
    return r;
}
__device__ __forceinline__ void sq_acc2(uint64_t &a, uint64_t q, uint64_t x) {
    uint64_t d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(q), "l"(x));
    asm("fma.rn.f32x2 %0, %1, %1, %2;" : "=l"(a) : "l"(d), "l"(a));
}

// --------------------------------------------------------------------------
// a5-a7: the scan.  One CTA per work item at a time (persistent grid).
template <int G>
__global__ void __launch_bounds__(kBT, 4) k_scan(ScanArgs A) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int n = A.v.n;
    float4 *ring_all = reinterpret_cast<float4 *>(smem_raw);          // kBT/32 warps * kRing * 2 KB
    float *q_s = reinterpret_cast<float *>(ring_all + (kBT / 32) * kRing * 128);   // G*n
    float *stage_d = q_s + G * n;
    int32_t *stage_p = reinterpret_cast<int32_t *>(stage_d + G * kBT);
    float *list_d = reinterpret_cast<float *>(stage_p + G * kBT);     // G*p2
    int32_t *list_p = reinterpret_cast<int32_t *>(list_d + G * A.p2);

    __shared__ int64_t s_item;
    __shared__ int s_qid[G];
    __shared__ float s_U[G], s_T[G], s_Tsax[G];
    __shared__ int s_alive[G], s_sax[G];
    __shared__ int s_stage[G], s_list[G];
    __shared__ int64_t s_s0, s_s1;
    __shared__ int s_gq, s_leaf;
    __shared__ float s_B[kAlpha + 1];          // cell ends: -inf, breakpoints, +inf
    __shared__ float s_paa[G][2 * kWord];      // per query: PAA rounded down, then up
    __shared__ float4 s_pp[(G + 1) / 2][kWord]; // per query pair: (down g, down g+1, up g, up g+1)

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t total = A.item_off[A.v.L];
    const float rho = A.rho;
    long long my_sax = 0, my_ab = 0, my_full = 0, my_pts = 0, my_bytes = 0;
    if (A.sax_paa) {
        for (int j = tid; j <= kAlpha; j += kBT)
            s_B[j] = j == 0 ? -INFINITY : (j == kAlpha ? INFINITY : A.bp[j - 1]);
    }
    const float w_sax = (float)(n / kWord);

    for (;;) {
        if (tid == 0) s_item = atomicAdd(A.work_ctr, 1);
        __syncthreads();
        const int64_t it = s_item;
        if (it >= total) break;
        if (tid == 0) {
            const int leaf = find_segment<int64_t>(A.item_off, (int)A.v.L + 1, it);
            // skip leaves with no items (equal offsets): find the last leaf
            // whose offset <= it, which find_segment already returns
            const int64_t local = it - A.item_off[leaf];
            const int nql = A.leaf_qoff[leaf + 1] - A.leaf_qoff[leaf];
            const int ngroups = (nql + G - 1) / G;
            const int64_t tile = local / ngroups;
            const int grp = (int)(local % ngroups);
            const int64_t lo = A.v.leaf_off[leaf], hi = A.v.leaf_off[leaf + 1];
            s_s0 = lo + tile * A.S_T;
            s_s1 = min(s_s0 + (int64_t)A.S_T, hi);
            s_gq = min(G, nql - grp * G);
            s_leaf = leaf;
            for (int g = 0; g < G; ++g) {
                s_alive[g] = 0;
                if (g < s_gq) {
                    const int q = A.leaf_q[A.leaf_qoff[leaf] + grp * G + g];
                    s_qid[g] = q;
                    const float u = __uint_as_float(A.U[q]);
                    s_U[g] = u;
                    bool alive = true;
                    if (A.lb) alive = !(lb_lower(A.lb[(int64_t)q * A.v.L + leaf]) > (double)u);
                    s_alive[g] = alive;
                    s_sax[g] = (A.use_sax && A.qmode && (A.qmode[q] & 1)) ? 1 : 0;
                    s_T[g] = __fmul_ru(u, 1.0f + rho);
                    s_Tsax[g] = __fmul_ru(u, 1.0f + 0x1p-18f);
                }
                s_stage[g] = 0;
                s_list[g] = 0;
            }
        }
        __syncthreads();
        const int gq = s_gq;
        unsigned alive_mask = 0, sax_mask = 0;
        for (int g = 0; g < gq; ++g) {
            if (s_alive[g]) alive_mask |= 1u << g;
            if (s_alive[g] && s_sax[g]) sax_mask |= 1u << g;
        }
        if (!alive_mask) {
            __syncthreads();
            continue;
        }
        // stage the queries (and LB_SAX tables) in shared memory
        for (int g = 0; g < gq; ++g) {
            if (!(alive_mask >> g & 1)) continue;
            const float4 *src = reinterpret_cast<const float4 *>(A.Q + (int64_t)s_qid[g] * n);
            float4 *dst = reinterpret_cast<float4 *>(q_s + g * n);
            for (int j = tid; j < (n >> 2); j += kBT) dst[j] = src[j];
            if ((sax_mask >> g & 1) && tid < 2 * kWord)
                s_paa[g][tid] = A.sax_paa[(int64_t)s_qid[g] * 2 * kWord + tid];
        }
        __syncthreads();
        if (G > 1 && tid < kWord) {
            for (int pr = 0; pr < G / 2; ++pr) {
                const int g0 = 2 * pr, g1 = 2 * pr + 1;
                const bool u0 = sax_mask >> g0 & 1, u1 = sax_mask >> g1 & 1;
                s_pp[pr][tid] = make_float4(u0 ? s_paa[g0][tid] : 0.f, u1 ? s_paa[g1][tid] : 0.f,
                                            u0 ? s_paa[g0][kWord + tid] : 0.f, u1 ? s_paa[g1][kWord + tid] : 0.f);
            }
        }
        __syncthreads();

        const int64_t s0 = s_s0, s1 = s_s1;
        // this warp's ring of chunk buffers: chunk c of the warp's 32 series
        // (16 points each), float4 slot 4*series + (part ^ ((series >> 1) & 3))
        float4 *ring = ring_all + warp * (kRing * 128);
        const int nch = n >> 4;
        for (int64_t c0 = s0; c0 < s1; c0 += kBT) {
            const int64_t s = c0 + tid;
            const bool valid = s < s1;
            unsigned act = valid ? alive_mask : 0u;
            float T[G];
#pragma unroll
            for (int g = 0; g < G; ++g) T[g] = s_T[g];
            if (sax_mask && valid) {
                const uint4 w4 = __ldg(reinterpret_cast<const uint4 *>(A.v.sax) + s);
                float clo[kWord], chi[kWord];
                sax_cells(w4, s_B, clo, chi);
                if (G == 1) {
                    const float lbs = lb_sax_lower(clo, chi, s_paa[0], s_paa[0] + kWord, w_sax);
                    if (lbs > s_Tsax[0]) {
                        act &= ~1u;
                        ++my_sax;
                    }
                } else {
                    // two queries per packed instruction, the same rounded-down
                    // steps as lb_sax_lower
#pragma unroll
                    for (int pr = 0; pr < G / 2; ++pr) {
                        const unsigned pm = (sax_mask >> (2 * pr)) & 3u;
                        if (!pm) continue;
                        uint64_t acc2 = 0ull;
#pragma unroll
                        for (int i = 0; i < kWord; ++i) {
                            const float4 v = s_pp[pr][i];
                            const uint64_t a2 = sub_rd2(pack2(clo[i], clo[i]), pack2(v.z, v.w));
                            const uint64_t b2 = sub_rd2(pack2(v.x, v.y), pack2(chi[i], chi[i]));
                            float a0, a1, b0, b1;
                            unpack2(a2, a0, a1);
                            unpack2(b2, b0, b1);
                            acc2 = sqacc_rd2(pack2(max3f(a0, b0, 0.0f), max3f(a1, b1, 0.0f)), acc2);
                        }
                        float l0, l1;
                        unpack2(acc2, l0, l1);
                        if ((pm & 1u) && __fmul_rd(l0, w_sax) > s_Tsax[2 * pr]) {
                            act &= ~(1u << (2 * pr));
                            ++my_sax;
                        }
                        if ((pm & 2u) && __fmul_rd(l1, w_sax) > s_Tsax[2 * pr + 1]) {
                            act &= ~(1u << (2 * pr + 1));
                            ++my_sax;
                        }
                    }
                }
                my_bytes += kWord;
            }
            // per query four partial sums, as two packed pairs: the sum runs
            // as four interleaved chains (any order of the n terms stays
            // within rho), on the packed float32 pipes
            uint64_t accA[G], accB[G];
#pragma unroll
            for (int g = 0; g < G; ++g) accA[g] = accB[g] = 0ull;
            float acc[G];
#pragma unroll
            for (int g = 0; g < G; ++g) acc[g] = 0.0f;
            // a6: the warp copies the next chunks of its live series into its
            // ring (coalesced 64-byte pieces, kRing - 1 ahead) while each lane
            // works through its own series; a chunk is fetched only for series
            // that were still live when it was requested
            const int64_t wbase = c0 + (warp << 5);
            unsigned need = __ballot_sync(0xffffffffu, act != 0);
            auto issue = [&](int c) {
                float4 *slot = ring + (c % kRing) * 128;
#pragma unroll
                for (int m = 0; m < 4; ++m) {
                    const int f = lane + 32 * m, sl = f >> 2, part = f & 3;
                    if (need >> sl & 1)
                        cp_async16(slot + 4 * sl + (part ^ ((sl >> 1) & 3)),
                                   A.v.X + (wbase + sl) * n + 16 * c + 4 * part);
                }
            };
#pragma unroll
            for (int c = 0; c < kRing - 1; ++c) {
                if (c < nch && need) issue(c);
                cp_async_commit();
            }
            for (int c = 0; c < nch && need; ++c) {
                if (c + kRing - 1 < nch) issue(c + kRing - 1);
                cp_async_commit();
                cp_async_wait<kRing - 1>();
                __syncwarp();
                const float4 *slot = ring + (c % kRing) * 128 + 4 * lane;
                const int sw = (lane >> 1) & 3;
                const float4 x0 = slot[0 ^ sw], x1 = slot[1 ^ sw], x2 = slot[2 ^ sw], x3 = slot[3 ^ sw];
                if (act) {
                    my_bytes += 64;
                    const int j = c << 4;
                    const uint64_t X0 = pack2(x0.x, x0.y), X1 = pack2(x0.z, x0.w), X2 = pack2(x1.x, x1.y),
                                   X3 = pack2(x1.z, x1.w), X4 = pack2(x2.x, x2.y), X5 = pack2(x2.z, x2.w),
                                   X6 = pack2(x3.x, x3.y), X7 = pack2(x3.z, x3.w);
#pragma unroll
                    for (int g = 0; g < G; ++g) {
                        if (!(act >> g & 1)) continue;
                        const float4 *qv = reinterpret_cast<const float4 *>(q_s + g * n + j);
                        const float4 q0 = qv[0], q1 = qv[1], q2 = qv[2], q3 = qv[3];
                        uint64_t a = accA[g], b = accB[g];
                        sq_acc2(a, pack2(q0.x, q0.y), X0);
                        sq_acc2(b, pack2(q0.z, q0.w), X1);
                        sq_acc2(a, pack2(q1.x, q1.y), X2);
                        sq_acc2(b, pack2(q1.z, q1.w), X3);
                        sq_acc2(a, pack2(q2.x, q2.y), X4);
                        sq_acc2(b, pack2(q2.z, q2.w), X5);
                        sq_acc2(a, pack2(q3.x, q3.y), X6);
                        sq_acc2(b, pack2(q3.z, q3.w), X7);
                        accA[g] = a;
                        accB[g] = b;
                        float a0, a1, b0, b1;
                        unpack2(a, a0, a1);
                        unpack2(b, b0, b1);
                        acc[g] = (a0 + a1) + (b0 + b1);
                        if (acc[g] > T[g]) {
                            act &= ~(1u << g);
                            ++my_ab;
                            my_pts += 16 * (c + 1);
                        }
                    }
                }
                __syncwarp();   // the slot is read by every lane before it is refilled
                need = __ballot_sync(0xffffffffu, act != 0);
            }
            cp_async_wait<0>();   // copies still in flight for series that died
            __syncwarp();
            if (valid) {
#pragma unroll
                for (int g = 0; g < G; ++g) {
                    if (!(act >> g & 1)) continue;
                    ++my_full;
                    my_pts += n;
                    const int slot = atomicAdd(&s_stage[g], 1);
                    stage_d[g * kBT + slot] = acc[g];
                    stage_p[g * kBT + slot] = (int32_t)s;
                }
            }
            __syncthreads();
            // merge: warp w owns the lists of queries w, w + kBT/32, ...
            for (int g = warp; g < gq; g += kBT / 32) {
                if (!(alive_mask >> g & 1)) continue;
                float *ld = list_d + g * A.p2;
                int32_t *lp = list_p + g * A.p2;
                const int sc = s_stage[g];
                const int cnt = s_list[g];
                float U = s_U[g];
                const float ug = __uint_as_float(A.U[s_qid[g]]);
                U = fminf(U, ug);
                if (sc > 0) {
                    for (int i = lane; i < sc; i += 32) {
                        ld[cnt + i] = stage_d[g * kBT + i];
                        lp[cnt + i] = stage_p[g * kBT + i];
                    }
                    const int tot = cnt + sc;
                    int P = 32;
                    while (P < tot) P <<= 1;
                    for (int i = tot + lane; i < P; i += 32) {
                        ld[i] = INFINITY;
                        lp[i] = 0x7fffffff;
                    }
                    __syncwarp();
                    for (int size = 2; size <= P; size <<= 1) {
                        for (int stride = size >> 1; stride > 0; stride >>= 1) {
                            for (int i = lane; i < (P >> 1); i += 32) {
                                const int lo = 2 * stride * (i / stride) + (i % stride);
                                const int hi = lo + stride;
                                const bool asc = (lo & size) == 0;
                                const float a = ld[lo], b = ld[hi];
                                const int32_t pa = lp[lo], pb = lp[hi];
                                const bool gt = (a > b) || (a == b && pa > pb);
                                if (gt == asc) {
                                    ld[lo] = b; ld[hi] = a;
                                    lp[lo] = pb; lp[hi] = pa;
                                }
                            }
                            __syncwarp();
                        }
                    }
                    if (tot >= A.k) U = fminf(U, upper_f(ld[A.k - 1], rho));
                    const float T = __fmul_ru(U, 1.0f + rho);
                    // keep the prefix with d <= T
                    int keep = 0;
                    for (int i = lane; i < tot; i += 32) keep += (ld[i] <= T) ? 1 : 0;
                    keep = warp_sum_i(keep);
                    if (keep > A.cap) {
                        if (lane == 0) atomicOr(&A.qflag[s_qid[g]], 1);
                        keep = A.cap;
                    }
                    if (lane == 0) s_list[g] = keep;
                }
                if (lane == 0) {
                    s_U[g] = U;
                    s_T[g] = __fmul_ru(U, 1.0f + rho);
                    s_Tsax[g] = __fmul_ru(U, 1.0f + 0x1p-18f);
                    s_stage[g] = 0;
                }
            }
            __syncthreads();
        }
        // publish: entries at or below T(min(U_item, U_global)), then tighten U
        for (int g = warp; g < gq; g += kBT / 32) {
            if (!(alive_mask >> g & 1)) continue;
            const int q = s_qid[g];
            const float Uf = fminf(s_U[g], __uint_as_float(A.U[q]));
            const float T = __fmul_ru(Uf, 1.0f + rho);
            const float *ld = list_d + g * A.p2;
            const int32_t *lp = list_p + g * A.p2;
            const int cnt = s_list[g];
            int e = 0;
            for (int i = lane; i < cnt; i += 32) e += (ld[i] <= T) ? 1 : 0;
            e = warp_sum_i(e);
            int base = 0;
            if (lane == 0 && e > 0) base = atomicAdd(&A.pool_cnt[q], e);
            base = __shfl_sync(0xffffffffu, base, 0);
            int ew = e;
            if (base + e > A.pool_C) {
                ew = max(0, A.pool_C - base);
                if (lane == 0) atomicOr(&A.qflag[q], 1);
            }
            for (int i = lane; i < ew; i += 32) {
                A.pool_d[(int64_t)q * A.pool_C + base + i] = ld[i];
                A.pool_p[(int64_t)q * A.pool_C + base + i] = lp[i];
            }
            if (lane == 0) atomicMin(&A.U[q], __float_as_uint(s_U[g]));
        }
        __syncthreads();
    }
    // statistics
    my_sax = warp_sum_ll(my_sax);
    my_ab = warp_sum_ll(my_ab);
    my_full = warp_sum_ll(my_full);
    my_pts = warp_sum_ll(my_pts);
    my_bytes = warp_sum_ll(my_bytes);
    if (lane == 0) {
        stat_add(&A.stats[ST_SCAN_BYTES], my_bytes);
        stat_add(&A.stats[ST_SAX_PRUNED], my_sax);
        stat_add(&A.stats[ST_ABANDONED], my_ab);
        stat_add(&A.stats[ST_FULL], my_full);
        stat_add(&A.stats[ST_POINTS], my_pts);
    }
}

// U = min(U, (1+rho) x k-th smallest pooled float32 distance).
__global__ void k_stats_init(long long *__restrict__ stats, int nq, long long L, long long lb_evals) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        stats[ST_QUERIES] = nq;
        stats[ST_LEAVES_TOTAL] = (long long)nq * L;
        stats[ST_LB_EVALS] = lb_evals;
    }
}

// U[q] from the k-th smallest pooled distance (rounded up by T's factor):
// a radix select over the distances' bit patterns (non-negative floats order
// as their bits), four passes of 8 bits with a shared-memory histogram.
__global__ void k_pool_kth(const float *__restrict__ pool_d, const int32_t *__restrict__ pool_cnt,
                           int C, int k, float rho, uint32_t *__restrict__ U) {
    __shared__ int hist[256];
    __shared__ uint32_t s_prefix;
    __shared__ int s_rank;
    const int q = blockIdx.x;
    const int cnt = min(pool_cnt[q], C);
    if (cnt < k) return;
    const uint32_t *d = reinterpret_cast<const uint32_t *>(pool_d + (int64_t)q * C);
    const int lane = threadIdx.x & 31;
    uint32_t prefix = 0, mask = 0;
    int rank = k;   // rank of the wanted key among those matching the prefix
    // keys are read kKthUnroll per thread at a time, so that a large pool's
    // pass is not a chain of single dependent loads
    constexpr int kKthUnroll = 8;
    const int span = blockDim.x * kKthUnroll;
    const int rounds = (cnt + span - 1) / span;
    for (int shift = 24; shift >= 0; shift -= 8) {
        for (int b = threadIdx.x; b < 256; b += blockDim.x) hist[b] = 0;
        __syncthreads();
        for (int r = 0; r < rounds; ++r) {
            uint32_t key[kKthUnroll];
#pragma unroll
            for (int u = 0; u < kKthUnroll; ++u) {
                const int i = r * span + u * blockDim.x + threadIdx.x;
                key[u] = i < cnt ? d[i] : 0xffffffffu;
            }
#pragma unroll
            for (int u = 0; u < kKthUnroll; ++u) {
                const int i = r * span + u * blockDim.x + threadIdx.x;
                int digit = 256;   // no count
                if (i < cnt && (key[u] & mask) == prefix) digit = (int)((key[u] >> shift) & 255u);
                const unsigned peers = __match_any_sync(0xffffffffu, digit);
                if (digit < 256 && lane == __ffs(peers) - 1) atomicAdd(&hist[digit], __popc(peers));
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            int cum = 0, b = 0;
            for (; b < 255 && cum + hist[b] < rank; ++b) cum += hist[b];
            s_prefix = prefix | ((uint32_t)b << shift);
            s_rank = rank - cum;
        }
        __syncthreads();
        prefix = s_prefix;
        rank = s_rank;
        mask |= 255u << shift;
        __syncthreads();
    }
    if (threadIdx.x == 0) atomicMin(&U[q], __float_as_uint(upper_f(__uint_as_float(prefix), rho)));
}

// a8: binary64 rescore of every pooled candidate at or below T(U) and the
// final top-k by (binary64 distance, original id).  The candidates at or
// below T are normally few (about k): their positions are gathered first so
// that every lane of a warp rescores one (the binary64 pipe is narrow and
// issues whole warps), then they are sorted in shared memory (bitonic, by
// (distance, id)).  A larger set takes k block-wide argmin passes over the
// pool in global memory.
constexpr int kFinalCap = 1024;
constexpr int kFinalQLen = 1024;   // longest query held as binary64 in shared memory
__global__ void k_final(const float *__restrict__ Q, const float *__restrict__ X, int n,
                        const int64_t *__restrict__ perm, const float *__restrict__ pool_d,
                        const int32_t *__restrict__ pool_p, const int32_t *__restrict__ pool_cnt,
                        int C, const uint32_t *__restrict__ U, const int32_t *__restrict__ qflag,
                        int k, float rho, double *__restrict__ rs, int64_t *__restrict__ out_ids,
                        float *__restrict__ out_dist, long long *__restrict__ stats,
                        int32_t *__restrict__ err, const int32_t *__restrict__ qsel) {
    __shared__ double bd[32];
    __shared__ long long bi[32];
    __shared__ int be[32];
    __shared__ double sv[kFinalCap];
    __shared__ long long sid[kFinalCap];
    __shared__ double qd[kFinalQLen];
    __shared__ int ns;
    const int q = qsel ? qsel[blockIdx.x] : blockIdx.x;
    const int64_t slot = qsel ? blockIdx.x : q;   // row of the pool for this block
    if (qflag && (qflag[q] & 1)) return;
    if (threadIdx.x == 0) ns = 0;
    const float *qr = Q + (int64_t)q * n;
    if (n <= kFinalQLen)
        for (int j = threadIdx.x; j < n; j += blockDim.x) qd[j] = (double)qr[j];
    __syncthreads();
    const int cnt = min(pool_cnt[slot], C);
    const float T = __fmul_ru(__uint_as_float(U[q]), 1.0f + rho);
    const float *pd = pool_d + slot * C;
    const int32_t *pp = pool_p + slot * C;
    double *r = rs + slot * C;
    // the candidates at or below T, positions into sid (as pool indices);
    // eight loads in flight per thread
    for (int i0 = 0; i0 < cnt; i0 += 8 * blockDim.x) {
        float dv[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int i = i0 + u * blockDim.x + threadIdx.x;
            dv[u] = i < cnt ? pd[i] : INFINITY;
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int i = i0 + u * blockDim.x + threadIdx.x;
            if (i < cnt && dv[u] <= T) {
                const int e = atomicAdd(&ns, 1);
                if (e < kFinalCap) sid[e] = i;
            }
        }
    }
    __syncthreads();
    const int m = ns;
    if (threadIdx.x == 0 && m) stat_add(&stats[ST_RESCORED], m);
    if (m <= kFinalCap) {
        for (int e = threadIdx.x; e < m; e += blockDim.x) {
            const int64_t pos = pp[sid[e]];
            const float *x = X + pos * n;
            double v = 0.0;   // dist2_64, with the query's binary64 values from shared memory
            if (n <= kFinalQLen) {
                for (int j = 0; j < n; ++j) {
                    const double d = __dsub_rn(qd[j], (double)x[j]);
                    v = __dadd_rn(v, __dmul_rn(d, d));
                }
            } else {
                v = dist2_64(qr, x, n);
            }
            sv[e] = v;
            sid[e] = perm ? perm[pos] : pos;
        }
        int P = 1;
        while (P < m) P <<= 1;
        for (int i = m + threadIdx.x; i < P; i += blockDim.x) {
            sv[i] = INFINITY;
            sid[i] = 0x7fffffffffffffffLL;
        }
        __syncthreads();
        for (int size = 2; size <= P; size <<= 1)
            for (int stride = size >> 1; stride > 0; stride >>= 1) {
                for (int t = threadIdx.x; t < P / 2; t += blockDim.x) {
                    const int i = 2 * t - (t & (stride - 1)), j = i + stride;
                    const bool gt = sv[i] > sv[j] || (sv[i] == sv[j] && sid[i] > sid[j]);
                    if (gt == ((i & size) == 0)) {
                        const double tv = sv[i];
                        sv[i] = sv[j];
                        sv[j] = tv;
                        const long long ti = sid[i];
                        sid[i] = sid[j];
                        sid[j] = ti;
                    }
                }
                __syncthreads();
            }
        for (int t = threadIdx.x; t < k; t += blockDim.x) {
            if (t < m) {
                out_ids[(int64_t)q * k + t] = sid[t];
                out_dist[(int64_t)q * k + t] = __double2float_rn(__dsqrt_rn(sv[t]));
            } else {
                atomicOr(err, 1);
                out_ids[(int64_t)q * k + t] = -1;
                out_dist[(int64_t)q * k + t] = INFINITY;
            }
        }
        return;
    }
    for (int i = threadIdx.x; i < cnt; i += blockDim.x)
        r[i] = pd[i] <= T ? dist2_64(qr, X + (int64_t)pp[i] * n, n) : INFINITY;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int t = 0; t < k; ++t) {
        double b = INFINITY;
        long long id = -1;
        int e = -1;
        for (int i = threadIdx.x; i < cnt; i += blockDim.x) {
            const double v = r[i];
            if (v == INFINITY) continue;
            const long long pid = perm ? perm[pp[i]] : (long long)pp[i];
            if (e < 0 || v < b || (v == b && pid < id)) { b = v; id = pid; e = i; }
        }
        for (int o = 16; o > 0; o >>= 1) {
            const double ov = __shfl_xor_sync(0xffffffffu, b, o);
            const long long oid = __shfl_xor_sync(0xffffffffu, id, o);
            const int oe = __shfl_xor_sync(0xffffffffu, e, o);
            if (oe >= 0 && (e < 0 || ov < b || (ov == b && oid < id))) { b = ov; id = oid; e = oe; }
        }
        if (lane == 0) { bd[warp] = b; bi[warp] = id; be[warp] = e; }
        __syncthreads();
        if (threadIdx.x == 0) {
            double bb = INFINITY;
            long long ii = -1;
            int ee = -1;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w)
                if (be[w] >= 0 && (ee < 0 || bd[w] < bb || (bd[w] == bb && bi[w] < ii))) {
                    bb = bd[w]; ii = bi[w]; ee = be[w];
                }
            if (ee < 0) {
                atomicOr(err, 1);
                out_ids[(int64_t)q * k + t] = -1;
                out_dist[(int64_t)q * k + t] = INFINITY;
            } else {
                out_ids[(int64_t)q * k + t] = ii;
                out_dist[(int64_t)q * k + t] = __double2float_rn(__dsqrt_rn(bb));
                r[ee] = INFINITY;
            }
        }
        __syncthreads();
    }
}

// Last-resort fallback: every series of the collection whose float32
// distance to query q is at or below T (pass 0 counts, pass 1 writes).  One
// warp per series, coalesced reads; any summation order obeys the same
// rounding bound.
__global__ void k_collect(const float *__restrict__ Q, int q, const float *__restrict__ X, int n,
                          int64_t N, float T, int pass, int32_t *__restrict__ cnt,
                          float *__restrict__ out_d, int32_t *__restrict__ out_p, int cap) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const float *qq = Q + (int64_t)q * n;
    for (int64_t s = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; s < N; s += warps) {
        const float *x = X + s * n;
        float a = 0.0f;
        for (int j = lane; j < n; j += 32) {
            const float d = qq[j] - x[j];
            a = fmaf(d, d, a);
        }
        for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
        if (lane == 0 && a <= T) {
            const int slot = atomicAdd(cnt, 1);
            if (pass == 1 && slot < cap) {
                out_d[slot] = a;
                out_p[slot] = (int32_t)s;
            }
        }
    }
}

// Rows sel[i] of Q and U into compact arrays (the queries of a retry pass).
__global__ void k_gather_queries(const float *__restrict__ Q, int n, const int32_t *__restrict__ sel,
                                 int nsel, const uint32_t *__restrict__ U, float *__restrict__ Qo,
                                 uint32_t *__restrict__ Uo) {
    const int i = blockIdx.x;
    if (i >= nsel) return;
    const int q = sel[i];
    for (int j = threadIdx.x; j < n; j += blockDim.x) Qo[(int64_t)i * n + j] = Q[(int64_t)q * n + j];
    if (threadIdx.x == 0) Uo[i] = U[q];
}

// Results of a retry pass back into the batch's rows.
__global__ void k_scatter_results(const int64_t *__restrict__ ids, const float *__restrict__ dist,
                                  const int32_t *__restrict__ sel, int nsel, int k,
                                  int64_t *__restrict__ ids_o, float *__restrict__ dist_o) {
    const int i = blockIdx.x;
    if (i >= nsel) return;
    const int q = sel[i];
    for (int t = threadIdx.x; t < k; t += blockDim.x) {
        ids_o[(int64_t)q * k + t] = ids[(int64_t)i * k + t];
        dist_o[(int64_t)q * k + t] = dist[(int64_t)i * k + t];
    }
}

__global__ void k_fill_u32(uint32_t *p, int64_t n, uint32_t v) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        p[i] = v;
}

__global__ void k_debug_lbsax(const float *__restrict__ paa, const float *__restrict__ bp,
                              const uint8_t *__restrict__ sax, int64_t N, int n, int nq,
                              float *__restrict__ out) {
    __shared__ float B[kAlpha + 1];
    for (int j = threadIdx.x; j <= kAlpha; j += blockDim.x)
        B[j] = j == 0 ? -INFINITY : (j == kAlpha ? INFINITY : bp[j - 1]);
    __syncthreads();
    const float w = (float)(n / kWord);
    for (int q = blockIdx.y; q < nq; q += gridDim.y)
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < N;
         s += (int64_t)gridDim.x * blockDim.x) {
        float lo[kWord], hi[kWord];
        sax_cells(*reinterpret_cast<const uint4 *>(sax + s * kWord), B, lo, hi);
        const float *pq = paa + (int64_t)q * 2 * kWord;
        const float lbs = lb_sax_lower(lo, hi, pq, pq + kWord, w);
        // the scan prunes when lbs > U(1 + 2^-18): the certified value is
        // lbs / (1 + 2^-18) rounded down
        out[(int64_t)q * N + s] = __fdiv_rd(lbs, 1.0f + 0x1p-18f);
    }
}

// ---------------------------------------------------------------- host side
float rho_for(int n) {
    const double u = std::ldexp(1.0, -24);
    const double m = (double)(n + 2) * u;
    const double g = m / (1.0 - m);
    return (float)(g * 1.0001 + std::ldexp(1.0, -40));
}

int sm_count() {
    int dev = 0, sms = 0;
    HK_CHECK_CUDA(cudaGetDevice(&dev));
    HK_CHECK_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    return sms;
}

TreeView tree_view(const hk_index *idx) {
    TreeView t{};
    t.L = idx->L;
    t.T = idx->T;
    t.leaf_nseg = idx->leaf_nseg.p;
    t.leaf_seg = idx->leaf_seg.p;
    t.env = idx->env.p;
    t.inode_nseg = idx->inode_nseg.p;
    t.inode_seg = idx->inode_seg.p;
    t.ienv = idx->ienv.p;
    t.seg_ab = idx->seg_ab.p;
    t.parent = idx->tree_parent.p;
    t.left = idx->tree_left.p;
    t.right = idx->tree_right.p;
    t.beg = idx->tree_beg.p;
    t.end = idx->tree_end.p;
    return t;
}

struct ScanConfig {
    int G;
    int p2;
    int cap;
    size_t smem;
};

size_t scan_smem(int G, int n, int p2, bool sax) {
    (void)sax;
    return (size_t)(kBT / 32) * kRing * 2048 + (size_t)G * n * 4 + (size_t)G * kBT * 8 +
           (size_t)G * p2 * 8;
}

ScanConfig choose_scan(int n, int k, bool sax, int want_G) {
    ScanConfig c;
    c.cap = ((k + kSlack + 31) / 32) * 32;
    c.p2 = 32;
    while (c.p2 < c.cap + kBT) c.p2 <<= 1;
    const size_t limit = 200 * 1024;   // bytes of dynamic shared memory
    int G = want_G > 0 ? std::min(want_G, kMaxG) : kMaxG;
    while (G > 1 && scan_smem(G, n, c.p2, sax) > limit) G >>= 1;
    if (G != 1 && G != 2 && G != 4 && G != 8) G = G >= 8 ? 8 : G >= 4 ? 4 : G >= 2 ? 2 : 1;
    c.G = G;
    c.smem = scan_smem(G, n, c.p2, sax);
    if (c.smem > limit) fail(HK_EINVAL, "k=%d with n=%d needs %zu bytes of shared memory", k, n, c.smem);
    return c;
}

template <int G>
void launch_scan_g(const ScanArgs &a, size_t smem, cudaStream_t s) {
    static std::once_flag once;
    std::call_once(once, [] {
        HK_CHECK_CUDA(cudaFuncSetAttribute(k_scan<G>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           200 * 1024));
    });
    int per_sm = 0;
    HK_CHECK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_scan<G>, kBT, smem));
    if (per_sm < 1) per_sm = 1;
    k_scan<G><<<(unsigned)(sm_count() * per_sm), kBT, smem, s>>>(a);
    HK_CHECK_LAUNCH();
}

void launch_scan(const ScanArgs &a, const ScanConfig &c, cudaStream_t s) {
    switch (c.G) {
        case 8: launch_scan_g<8>(a, c.smem, s); break;
        case 4: launch_scan_g<4>(a, c.smem, s); break;
        case 2: launch_scan_g<2>(a, c.smem, s); break;
        default: launch_scan_g<1>(a, c.smem, s); break;
    }
}

// CUDA events bracketing each scan launch on its stream (HK_Q_TIMING).
struct ScanTimer {
    bool on = false;
    std::vector<cudaEvent_t> ev;
    ~ScanTimer() {
        for (cudaEvent_t e : ev) cudaEventDestroy(e);
    }
    void mark(cudaStream_t s) {
        if (!on) return;
        cudaEvent_t e;
        HK_CHECK_CUDA(cudaEventCreate(&e));
        ev.push_back(e);
        HK_CHECK_CUDA(cudaEventRecord(e, s));
    }
    // total of (end - start) over the recorded pairs, after the stream finished
    long long total_ns() {
        double ms = 0.0;
        for (size_t i = 0; i + 1 < ev.size(); i += 2) {
            float t = 0.f;
            HK_CHECK_CUDA(cudaEventElapsedTime(&t, ev[i], ev[i + 1]));
            ms += t;
        }
        return (long long)(ms * 1e6);
    }
};

// Build leaf-major lists for mask value v and run the scan over them.
// Leaf-major work lists for mask value `val`: per leaf the queries for which
// it is a candidate, and work items of G queries x S_T series.
void build_lists(Workspace &ws, const LeafView &v, int G, int S_T, uint8_t val, int nq, cudaStream_t s) {
    const int64_t L = v.L;
    k_leaf_count<<<(unsigned)L, 256, 0, s>>>(ws.mask.p, nq, val, v.leaf_off, G, S_T, ws.leaf_qcnt.p,
                                            ws.leaf_items.p);
    HK_CHECK_LAUNCH();
    exclusive_scan_i32(ws.leaf_qcnt.p, ws.leaf_qoff.p, L, s, ws.scan_tmp32);
    exclusive_scan_i64(ws.leaf_items.p, ws.item_off.p, L, s, ws.scan_tmp64);
    k_leaf_fill<<<(unsigned)L, 256, 0, s>>>(ws.mask.p, nq, val, ws.leaf_qoff.p, ws.leaf_q.p);
    HK_CHECK_LAUNCH();
    HK_CHECK_CUDA(cudaMemsetAsync(ws.counters.p, 0, sizeof(int32_t), s));
}

void scan_phase(Workspace &ws, const LeafView &v, ScanArgs a, const ScanConfig &c, uint8_t val,
                int nq, cudaStream_t s, ScanTimer *timer = nullptr) {
    build_lists(ws, v, c.G, a.S_T, val, nq, s);
    a.leaf_qoff = ws.leaf_qoff.p;
    a.leaf_q = ws.leaf_q.p;
    a.item_off = ws.item_off.p;
    a.work_ctr = ws.counters.p;
    if (timer) timer->mark(s);
    launch_scan(a, c, s);
    if (timer) timer->mark(s);
}

// a5-a7 on the tensor cores over the leaves whose mask value is `val`:
// distances with a certified bound (k_tc_scan), then the exact float32
// rescore of the survivors at or below U into the pool.  U only falls: the
// scan lowers it from the k best upper bounds each thread has seen.
void tc_phase(hk_index *idx, Workspace &ws, const LeafView &v, const float *Qd, int nq, int k, int S_tc,
              uint8_t val, int pool_C, float rho, int stat_pairs, int stat_cands, int stat_bytes,
              cudaStream_t s, ScanTimer *tctimer, bool capture) {
    const int n = idx->n;
    const int cand_C = tc_list_cap(k);
    ws.cand_cnt.reserve(nq, s);
    ws.rs_items.reserve(nq, s);
    ws.rs_off.reserve((size_t)nq + 1, s);
    ws.cand_p.reserve((size_t)nq * cand_C, s);
    ws.cand_lb.reserve((size_t)nq * cand_C, s);
    HK_CHECK_CUDA(cudaMemsetAsync(ws.cand_cnt.p, 0, nq * sizeof(int32_t), s));
    build_lists(ws, v, 128, S_tc, val, nq, s);
    TcArgs t{};
    t.Xb = idx->Xb.p;
    t.xq = idx->xq.p;
    t.n = n;
    t.Qb = ws.Qb.p;
    t.q2e = ws.q2.p;
    t.qa = ws.qa.p;
    t.qoff2 = ws.qoff.p;
    t.eb2 = tc_eb2();
    t.leaf_off = v.leaf_off;
    t.L = v.L;
    t.leaf_qoff = ws.leaf_qoff.p;
    t.leaf_q = ws.leaf_q.p;
    t.item_off = ws.item_off.p;
    t.work_ctr = ws.counters.p;
    t.S_T = S_tc;
    t.U = ws.U.p;
    t.k = k;
    t.cand_cnt = ws.cand_cnt.p;
    t.cand_p = ws.cand_p.p;
    t.cand_lb = ws.cand_lb.p;
    t.cand_C = cand_C;
    t.qflag = ws.qflag.p;
    t.err = ws.counters.p + 2;
    t.stats = (long long *)ws.stats.p;
    t.stat_pairs = stat_pairs;
    t.stat_cands = stat_cands;
    t.stat_bytes = stat_bytes;
    t.idesc = tc_idesc(idx->fmt16);
    t.dbg_lo = nullptr;
    t.dbg_up = nullptr;
    t.N = idx->N;
    tc_wait_hooks(t.wait_ns, t.dbg_stall);
    if (ws.engine && !capture) {
        // served: the scan is a job of the resident launch, which also runs
        // other batches' scans (its inputs must be ready first)
        int64_t items = 0;
        HK_CHECK_CUDA(cudaMemcpyAsync(&items, ws.item_off.p + v.L, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        HK_CHECK_CUDA(cudaStreamSynchronize(s));
        // approximate steps (val 1) take the ring's first lane: they are
        // short and every batch waits on one before its exact step
        if (items > 0) tc_engine_run(ws.engine, t, items, 120ull * 1000000000ull, val == 1 ? 0 : 1);
    } else {
        if (tctimer) tctimer->mark(s);
        launch_tc_scan(t, s);
        if (tctimer) tctimer->mark(s);
    }
    k_pool_kth<<<nq, 512, 0, s>>>(ws.pool_d.p, ws.pool_cnt.p, pool_C, k, rho, ws.U.p);
    HK_CHECK_LAUNCH();
    launch_tc_rescore(Qd, v.X, n, nq, ws.cand_cnt.p, ws.cand_p.p, ws.cand_lb.p, cand_C, ws.U.p,
                      ws.pool_d.p, ws.pool_p.p, ws.pool_cnt.p, pool_C, ws.qflag.p,
                      (long long *)ws.stats.p, ST_FULL, ws.rs_items.p, ws.rs_off.p, ws.scan_tmp32, s);
    if (capture) return;
    int32_t terr = 0;
    HK_CHECK_CUDA(cudaMemcpyAsync(&terr, ws.counters.p + 2, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    HK_CHECK_CUDA(cudaStreamSynchronize(s));
    if (terr) fail(HK_ETIMEOUT, "tensor-core scan: a bounded wait ran out (flag %d)", terr);
}

struct Prepared {
    int pool_C;
    ScanConfig cfg;
};

void reserve_common(Workspace &ws, int nq, int64_t L, int k, int pool_C, cudaStream_t s) {
    ws.U.reserve(nq, s);
    ws.qmode.reserve(nq, s);
    ws.qcand.reserve(nq, s);
    ws.mask.reserve((size_t)L * nq, s);
    ws.leaf_qcnt.reserve(L, s);
    ws.leaf_qoff.reserve(L + 1, s);
    ws.leaf_q.reserve((size_t)L * nq, s);
    ws.leaf_items.reserve(L, s);
    ws.item_off.reserve(L + 1, s);
    ws.counters.reserve(4, s);
    ws.pool_d.reserve((size_t)nq * pool_C, s);
    ws.pool_p.reserve((size_t)nq * pool_C, s);
    ws.pool_cnt.reserve(nq, s);
    ws.qflag.reserve(nq, s);
    ws.rs_d.reserve((size_t)nq * pool_C, s);
    ws.stats.reserve(kStatSlots, s);
    ws.out_ids.reserve((size_t)nq * k, s);
    ws.out_dist.reserve((size_t)nq * k, s);
}

void copy_out(const Workspace &ws, int nq, int k, int64_t *ids, float *dist, cudaStream_t s) {
    const cudaMemcpyKind ki = is_device_ptr(ids) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    const cudaMemcpyKind kd = is_device_ptr(dist) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    HK_CHECK_CUDA(cudaMemcpyAsync(ids, ws.out_ids.p, (size_t)nq * k * sizeof(int64_t), ki, s));
    HK_CHECK_CUDA(cudaMemcpyAsync(dist, ws.out_dist.p, (size_t)nq * k * sizeof(float), kd, s));
}

// a8: tighten U from the pool, rescore in binary64 and select.  Returns the
// per-query flags (bit0: a list or the pool overflowed) and bounds on the host.
void final_select(Workspace &ws, const LeafView &v, const float *Qd, int nq, int k, int pool_C,
                  float rho, cudaStream_t s, std::vector<int32_t> &flags, std::vector<uint32_t> &U,
                  bool capture = false) {
    k_pool_kth<<<nq, 512, 0, s>>>(ws.pool_d.p, ws.pool_cnt.p, pool_C, k, rho, ws.U.p);
    HK_CHECK_LAUNCH();
    HK_CHECK_CUDA(cudaMemsetAsync(ws.counters.p + 1, 0, sizeof(int32_t), s));
    k_final<<<nq, 256, 0, s>>>(Qd, v.X, v.n, v.perm, ws.pool_d.p, ws.pool_p.p, ws.pool_cnt.p, pool_C,
                               ws.U.p, ws.qflag.p, k, rho, ws.rs_d.p, ws.out_ids.p, ws.out_dist.p,
                               (long long *)ws.stats.p, ws.counters.p + 1, nullptr);
    HK_CHECK_LAUNCH();
    if (capture) return;
    flags.assign(nq, 0);
    U.assign(nq, 0);
    int32_t err = 0;
    HK_CHECK_CUDA(cudaMemcpyAsync(flags.data(), ws.qflag.p, nq * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    HK_CHECK_CUDA(cudaMemcpyAsync(U.data(), ws.U.p, nq * sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    HK_CHECK_CUDA(cudaMemcpyAsync(&err, ws.counters.p + 1, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    HK_CHECK_CUDA(cudaStreamSynchronize(s));
    if (err) fail(HK_EINTERNAL, "a query had fewer than k candidates after the scan");
}

// Exhaustive answer for row q of Qd: collect every series at or below
// T(U[q]), rescore and select into row q of ws.out_*.
void exhaustive_one(Workspace &ws, const LeafView &v, const float *Qd, int q, uint32_t Ubits, int k,
                    float rho, cudaStream_t s) {
    const int sms = sm_count();
    float u;
    std::memcpy(&u, &Ubits, 4);
    const float T = std::nextafter(u * (1.0f + rho), INFINITY);   // >= the device's T(U)
    DevBuf<int32_t> cnt;
    cnt.alloc(2, s);
    HK_CHECK_CUDA(cudaMemsetAsync(cnt.p, 0, 2 * sizeof(int32_t), s));
    k_collect<<<sms * 16, 256, 0, s>>>(Qd, q, v.X, v.n, v.N, T, 0, cnt.p, nullptr, nullptr, 0);
    HK_CHECK_LAUNCH();
    int32_t c = 0;
    HK_CHECK_CUDA(cudaMemcpyAsync(&c, cnt.p, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    HK_CHECK_CUDA(cudaStreamSynchronize(s));
    if (c < k) fail(HK_EINTERNAL, "exhaustive collection for query %d found %d < k candidates", q, c);
    DevBuf<float> fd;
    DevBuf<int32_t> fp;
    DevBuf<double> fr;
    DevBuf<int32_t> qsel;
    fd.alloc(c, s);
    fp.alloc(c, s);
    fr.alloc(c, s);
    qsel.alloc(1, s);
    HK_CHECK_CUDA(cudaMemsetAsync(cnt.p, 0, sizeof(int32_t), s));
    k_collect<<<sms * 16, 256, 0, s>>>(Qd, q, v.X, v.n, v.N, T, 1, cnt.p, fd.p, fp.p, c);
    HK_CHECK_LAUNCH();
    HK_CHECK_CUDA(cudaMemcpyAsync(qsel.p, &q, sizeof(int32_t), cudaMemcpyHostToDevice, s));
    k_final<<<1, 256, 0, s>>>(Qd, v.X, v.n, v.perm, fd.p, fp.p, cnt.p, c, ws.U.p, nullptr, k, rho,
                              fr.p, ws.out_ids.p, ws.out_dist.p, (long long *)ws.stats.p,
                              ws.counters.p + 1, qsel.p);
    HK_CHECK_LAUNCH();
    int32_t err = 0;
    HK_CHECK_CUDA(cudaMemcpyAsync(&err, ws.counters.p + 1, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    HK_CHECK_CUDA(cudaStreamSynchronize(s));
    if (err) fail(HK_EINTERNAL, "exhaustive collection for query %d: selection failed", q);
}

void copy_stats(const Workspace &ws, hk_query_stats *stats, cudaStream_t s, ScanTimer *timer,
                long long launches) {
    if (!stats) return;
    long long st[kStatSlots];
    HK_CHECK_CUDA(cudaMemcpyAsync(st, ws.stats.p, sizeof(st), cudaMemcpyDeviceToHost, s));
    HK_CHECK_CUDA(cudaStreamSynchronize(s));
    std::memset(stats, 0, sizeof(*stats));
    stats->queries = st[ST_QUERIES];
    stats->leaves_total = st[ST_LEAVES_TOTAL];
    stats->leaves_approx = st[ST_LEAVES_APPROX];
    stats->leaves_candidate = st[ST_LEAVES_CAND];
    stats->series_candidate = st[ST_SERIES_CAND];
    stats->series_sax_pruned = st[ST_SAX_PRUNED];
    stats->series_abandoned = st[ST_ABANDONED];
    stats->series_full = st[ST_FULL];
    stats->points_computed = st[ST_POINTS];
    stats->rescored = st[ST_RESCORED];
    stats->fallback_queries = st[ST_FALLBACK];
    stats->work_items = st[ST_ITEMS];
    stats->skip_sequential = st[ST_SKIPSEQ];
    stats->scan_bytes = st[ST_SCAN_BYTES];
    stats->retried_queries = st[ST_RETRIED];
    stats->tc_pairs = st[ST_TC_PAIRS];
    stats->tc_candidates = st[ST_TC_CANDS];
    stats->tc_bytes = st[ST_TC_BYTES];
    stats->tc_approx_pairs = st[ST_TCA_PAIRS];
    stats->tc_approx_bytes = st[ST_TCA_BYTES];
    stats->tc_leaf_bytes = st[ST_TC_LEAF_BYTES];
    stats->lb_evaluations = st[ST_LB_EVALS];
    stats->scan_ns = timer ? timer->total_ns() : 0;
    stats->kernel_launches = launches;
}

__global__ void k_count_items_and_series(const int64_t *__restrict__ item_off, int64_t L,
                                         const int32_t *__restrict__ qcnt,
                                         const int64_t *__restrict__ leaf_off,
                                         long long *__restrict__ stats, int series_slot,
                                         int leaves_slot) {
    long long ser = 0, lv = 0;
    for (int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; f < L;
         f += (int64_t)gridDim.x * blockDim.x) {
        ser += (long long)qcnt[f] * (leaf_off[f + 1] - leaf_off[f]);
        lv += qcnt[f];
    }
    ser = warp_sum_ll(ser);
    lv = warp_sum_ll(lv);
    if ((threadIdx.x & 31) == 0) {
        if (series_slot >= 0 && ser)
            stat_add(&stats[series_slot], ser);
        if (leaves_slot >= 0 && lv)
            stat_add(&stats[leaves_slot], lv);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0)
        stat_add(&stats[ST_ITEMS], item_off[L]);
}

// The exact tensor-core step's algorithmic DRAM bytes: the 16-bit rows and
// norms of every leaf some query of the batch scans, each counted once.
__global__ void k_tc_leaf_bytes(const int32_t *__restrict__ qcnt, const int64_t *__restrict__ leaf_off,
                                int64_t L, int n, long long *__restrict__ stats, int slot) {
    long long b = 0;
    for (int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; f < L;
         f += (int64_t)gridDim.x * blockDim.x)
        if (qcnt[f] > 0) b += (leaf_off[f + 1] - leaf_off[f]) * (long long)(2 * n + 8);
    b = warp_sum_ll(b);
    if ((threadIdx.x & 31) == 0 && b) stat_add(&stats[slot], b);
}

}  // namespace

namespace {

// One pass of the query path over a batch (a1-a8 without the retries).
// U_init: initial bounds (device, float bits) or nullptr for +inf; with
// bounds given, the approximate search is skipped.
// capture: only enqueue work (the pass is being recorded into a graph); the
// flags, bounds and error words stay on the device for the caller to read.
void query_pass(hk_index *idx, Workspace &ws, const float *Qd, int nq, int k, const hk_query_opts &o,
                cudaStream_t s, const uint32_t *U_init, ScanTimer *timer, ScanTimer *tctimer, ScanTimer *tcatimer,
                std::vector<int32_t> &flags, std::vector<uint32_t> &Uh, bool capture = false) {
    const int n = idx->n;
    const int64_t L = idx->L;
    const float rho = rho_for(n);
    const bool noprune = (o.flags & HK_Q_NOPRUNE) != 0;
    const bool tc = (o.flags & HK_Q_BF16) != 0;
    const bool tree = (o.flags & HK_Q_TREE) != 0;
    const TreeView tv = tree_view(idx);
    const bool nosax = noprune || tc || (o.flags & HK_Q_NOSAX) != 0;
    const int l_max = o.l_max > 0 ? o.l_max : kDefaultLMax;
    const float eapca_th = o.eapca_th >= 0 ? o.eapca_th : kDefaultEapcaTh;
    ScanConfig cfg = choose_scan(n, k, !nosax, o.query_group);
    const int S_T = o.series_tile > 0 ? o.series_tile : 8192;
    // the precision form's bound admits a band of near candidates around the
    // k-th distance (a few thousand on hard queries): give its pool room
    const int pool_C = tc ? tc_list_cap(k) : std::min(65536, std::max(4096, 64 * cfg.cap));

    reserve_common(ws, nq, L, k, pool_C, s);
    ws.qseg.reserve((size_t)nq * idx->S * 2, s);
    if (!nosax) ws.sax_paa.reserve((size_t)nq * 2 * kWord, s);
    ws.lb.reserve((size_t)nq * L, s);
    ws.approx.reserve((size_t)nq * kAmax, s);

    HK_CHECK_CUDA(cudaMemsetAsync(ws.stats.p, 0, kStatSlots * sizeof(long long), s));
    HK_CHECK_CUDA(cudaMemsetAsync(ws.pool_cnt.p, 0, nq * sizeof(int32_t), s));
    HK_CHECK_CUDA(cudaMemsetAsync(ws.qflag.p, 0, nq * sizeof(int32_t), s));
    HK_CHECK_CUDA(cudaMemsetAsync(ws.qcand.p, 0, nq * sizeof(int32_t), s));
    HK_CHECK_CUDA(cudaMemsetAsync(ws.mask.p, 0, (size_t)L * nq, s));
    if (U_init) {
        HK_CHECK_CUDA(cudaMemcpyAsync(ws.U.p, U_init, nq * sizeof(uint32_t), cudaMemcpyDeviceToDevice, s));
    } else {
        k_fill_u32<<<64, 256, 0, s>>>(ws.U.p, nq, 0x7f800000u);
        HK_CHECK_LAUNCH();
    }
    k_stats_init<<<1, 32, 0, s>>>((long long *)ws.stats.p, nq, L, tree ? 0 : (long long)nq * L);
    HK_CHECK_LAUNCH();
    HK_CHECK_CUDA(cudaMemsetAsync(ws.counters.p, 0, 4 * sizeof(int32_t), s));

    if (tc) {
        ws.Qb.reserve((size_t)nq * n, s);
        ws.q2.reserve(nq, s);
        ws.qa.reserve(nq, s);
        ws.qoff.reserve(nq, s);
        ws.bad.reserve(1, s);
        HK_CHECK_CUDA(cudaMemsetAsync(ws.bad.p, 0, sizeof(int), s));
        launch_tc_qprep(Qd, nq, n, idx->fmt16, idx->xn_max, ws.Qb.p, ws.q2.p, ws.qa.p, ws.qoff.p,
                        ws.bad.p, s);
        if (!capture) {
            int bad = 0;
            HK_CHECK_CUDA(cudaMemcpyAsync(&bad, ws.bad.p, sizeof(int), cudaMemcpyDeviceToHost, s));
            HK_CHECK_CUDA(cudaStreamSynchronize(s));
            if (bad) fail(HK_EINVAL, "queries have values beyond the 16-bit copy's range");
        }
    }
    const int S_tc = o.series_tile > 0 ? o.series_tile : 65536;
    // a1 + a2
    k_qprep<<<nq, 256, n * sizeof(float), s>>>(Qd, n, idx->seg_ab.p, idx->S, ws.qseg.p,
                                               nosax ? nullptr : ws.sax_paa.p);
    HK_CHECK_LAUNCH();
    if (!tree) {
        k_lb_eapca<<<dim3((unsigned)((L + 127) / 128), std::min(nq, 65535)), 128, 0, s>>>(
            ws.qseg.p, idx->S, tv, nq, ws.lb.p);
        HK_CHECK_LAUNCH();
    }

    LeafView v;
    v.X = idx->X.p;
    v.perm = idx->perm.p;
    v.sax = idx->sax.p;
    v.leaf_off = idx->leaf_off.p;
    v.N = idx->N;
    v.n = n;
    v.L = L;

    ScanArgs a{};
    a.v = v;
    a.Q = Qd;
    a.nq = nq;
    a.sax_paa = nosax ? nullptr : ws.sax_paa.p;
    a.bp = idx->bp.p;
    a.qmode = ws.qmode.p;
    a.lb = noprune ? nullptr : ws.lb.p;
    a.U = ws.U.p;
    a.S_T = S_T;
    a.k = k;
    a.cap = cfg.cap;
    a.p2 = cfg.p2;
    a.rho = rho;
    a.pool_d = ws.pool_d.p;
    a.pool_p = ws.pool_p.p;
    a.pool_cnt = ws.pool_cnt.p;
    a.pool_C = pool_C;
    a.qflag = ws.qflag.p;
    a.stats = (long long *)ws.stats.p;
    a.use_sax = nosax ? 0 : 1;

    // a3: approximate search (no LB_SAX: these leaves are scanned whole)
    if (!noprune && !U_init) {
        if (tree) {
            const int root = L > 1 ? (int)L : 0;   // the first internal node, or the only leaf
            k_tree_approx<<<(nq + 3) / 4, 128, 0, s>>>(ws.qseg.p, idx->S, tv, root, l_max, k, nq, kAmax,
                                                      ws.approx.p, ws.qcand.p, ws.mask.p, ws.lb.p,
                                                      (long long *)ws.stats.p);
        } else {
            k_approx_select<<<nq, 256, 0, s>>>(ws.lb.p, L, idx->leaf_off.p, l_max, k, nq, kAmax, ws.approx.p,
                                               ws.qcand.p, ws.mask.p);
        }
        HK_CHECK_LAUNCH();
        if (tc && k <= kTcLocalK) {
            // on the tensor cores from U = +inf: each thread's k best upper
            // bounds lower U after its first tile, so only the first tile of
            // a row keeps every column for the exact rescore
            tc_phase(idx, ws, v, Qd, nq, k, S_tc, 1, pool_C, rho, ST_TCA_PAIRS, ST_TCA_CANDS, ST_TCA_BYTES,
                     s, tcatimer, capture);
        } else {
            ScanArgs aa = a;
            aa.use_sax = 0;
            aa.lb = nullptr;
            scan_phase(ws, v, aa, cfg, 1, nq, s, timer);
        }
        k_count_items_and_series<<<8, 256, 0, s>>>(ws.item_off.p, L, ws.leaf_qcnt.p, idx->leaf_off.p,
                                                   (long long *)ws.stats.p, -1, ST_LEAVES_APPROX);
        HK_CHECK_LAUNCH();
        k_pool_kth<<<nq, 512, 0, s>>>(ws.pool_d.p, ws.pool_cnt.p, pool_C, k, rho, ws.U.p);
        HK_CHECK_LAUNCH();
        HK_CHECK_CUDA(cudaMemsetAsync(ws.qcand.p, 0, nq * sizeof(int32_t), s));
    }
    // a4: candidate leaves, per-query mode
    {
        const int64_t pairs = L * (int64_t)nq;
        if (tree) {
            // frontiers of (internal node, query) pairs, one pass per level;
            // a level holds fewer internal nodes than the tree has leaves
            const size_t cap = (size_t)nq * (size_t)std::max<int64_t>(1, L);
            const int levels = (int)idx->h_level_off.size() - 1;
            ws.tree_front.reserve(2 * cap, s);
            ws.tree_cnt.reserve((size_t)levels + 1, s);
            HK_CHECK_CUDA(cudaMemsetAsync(ws.tree_cnt.p, 0, ((size_t)levels + 1) * sizeof(int32_t), s));
            const int64_t root = L > 1 ? L : 0;
            k_tree_root<<<(nq + 255) / 256, 256, 0, s>>>(ws.qseg.p, idx->S, tv, root, nq, ws.U.p,
                                                         ws.tree_front.p, ws.tree_cnt.p, ws.mask.p, ws.qcand.p,
                                                         ws.lb.p, (long long *)ws.stats.p);
            HK_CHECK_LAUNCH();
            const int grid = sm_count() * 8;
            for (int d = 0; d + 1 < levels; ++d) {
                unsigned long long *fin = ws.tree_front.p + (d & 1) * cap;
                unsigned long long *fout = ws.tree_front.p + ((d + 1) & 1) * cap;
                k_tree_expand<<<grid, 256, 0, s>>>(ws.qseg.p, idx->S, tv, fin, ws.tree_cnt.p + d, fout,
                                                   ws.tree_cnt.p + d + 1, nq, ws.U.p, ws.mask.p, ws.qcand.p,
                                                   ws.lb.p, (long long *)ws.stats.p);
                HK_CHECK_LAUNCH();
            }
        } else {
            k_mask_candidates<<<(unsigned)((pairs + 255) / 256), 256, 0, s>>>(ws.lb.p, L, nq, ws.U.p,
                                                                            noprune ? 1 : 0, ws.mask.p,
                                                                            ws.qcand.p);
            HK_CHECK_LAUNCH();
        }
        k_qmode<<<(nq + 255) / 256, 256, 0, s>>>(ws.qcand.p, L, nq, eapca_th, nosax ? 1 : 0,
                                                 (o.flags & HK_Q_NOTHRESH) ? 1 : 0, ws.qmode.p,
                                                 (long long *)ws.stats.p);
        HK_CHECK_LAUNCH();
    }
    // a5-a7: scan of the candidate leaves
    if (tc) {
        // a9: tensor-core distances with a certified bound, then the exact
        // float32 rescore of the survivors into the pool
        if (k > kTcLocalK && !noprune) {
            // the scan cannot lower U in flight for this k: first each
            // query's best leaves, then U from their exact distances, then
            // the rest of the candidates against it
            k_round1_select<<<nq, 256, 0, s>>>(ws.lb.p, L, nq, kRound1Leaves, ws.mask.p);
            HK_CHECK_LAUNCH();
            tc_phase(idx, ws, v, Qd, nq, k, S_tc, 3, pool_C, rho, ST_TC_PAIRS, ST_TC_CANDS, ST_TC_BYTES, s,
                     tctimer, capture);
            k_count_items_and_series<<<8, 256, 0, s>>>(ws.item_off.p, L, ws.leaf_qcnt.p, idx->leaf_off.p,
                                                       (long long *)ws.stats.p, ST_SERIES_CAND, -1);
            HK_CHECK_LAUNCH();
            k_pool_kth<<<nq, 512, 0, s>>>(ws.pool_d.p, ws.pool_cnt.p, pool_C, k, rho, ws.U.p);
            HK_CHECK_LAUNCH();
            const int64_t pairs = L * (int64_t)nq;
            k_reprune<<<(unsigned)((pairs + 255) / 256), 256, 0, s>>>(ws.lb.p, L, nq, ws.U.p, ws.mask.p,
                                                                     (long long *)ws.stats.p);
            HK_CHECK_LAUNCH();
        }
        tc_phase(idx, ws, v, Qd, nq, k, S_tc, 2, pool_C, rho, ST_TC_PAIRS, ST_TC_CANDS, ST_TC_BYTES, s,
                 tctimer, capture);
        k_tc_leaf_bytes<<<8, 256, 0, s>>>(ws.leaf_qcnt.p, idx->leaf_off.p, L, n, (long long *)ws.stats.p,
                                          ST_TC_LEAF_BYTES);
        HK_CHECK_LAUNCH();
    } else {
        scan_phase(ws, v, a, cfg, 2, nq, s, timer);
    }
    k_count_items_and_series<<<8, 256, 0, s>>>(ws.item_off.p, L, ws.leaf_qcnt.p, idx->leaf_off.p,
                                               (long long *)ws.stats.p, ST_SERIES_CAND, -1);
    HK_CHECK_LAUNCH();
    // a8: boundary rescore and answer
    final_select(ws, v, Qd, nq, k, pool_C, rho, s, flags, Uh, capture);
}

}  // namespace

void run_query(hk_index *idx, const float *Qd, int nq, int k, const hk_query_opts &o, cudaStream_t s,
               int64_t *out_ids, float *out_dist, hk_query_stats *stats) {
    run_query_ws(idx, idx->ws, idx->ws_retry, Qd, nq, k, o, s, out_ids, out_dist, stats);
}

namespace {

// The rest of a query after its pass: retries of the queries whose lists or
// pool overflowed, the answers out, the counters.
void finish_query(hk_index *idx, Workspace &ws, Workspace &ws_retry, const float *Qd, int nq, int k,
                  const hk_query_opts &o, cudaStream_t s, int64_t *out_ids, float *out_dist,
                  hk_query_stats *stats, const std::vector<int32_t> &flags, long long launches0,
                  ScanTimer &timer, ScanTimer &tctimer, ScanTimer &tcatimer);

// Graph mode: the pass for this (batch size, k, options) is captured once
// into a CUDA graph over the graph work space and replayed; the queries are
// copied into the work space's input buffer first.  The first call with a
// new key answers with an ordinary pass (which sizes every buffer), then
// records the same pass for the calls after it.
void run_query_graph_on(hk_index *idx, const float *Qd, int nq, int k, const hk_query_opts &o, cudaStream_t s,
                        int64_t *out_ids, float *out_dist, hk_query_stats *stats);

void run_query_graph(hk_index *idx, const float *Qd, int nq, int k, const hk_query_opts &o, cudaStream_t s,
                     int64_t *out_ids, float *out_dist, hk_query_stats *stats) {
    // the work runs on the work space's own stream (the caller's may be the
    // legacy default stream, which cannot be captured), ordered after the
    // caller's stream and before what the caller enqueues next
    Workspace &ws = idx->ws_graph;
    if (!ws.gstream) {
        HK_CHECK_CUDA(cudaStreamCreateWithFlags(&ws.gstream, cudaStreamNonBlocking));
        HK_CHECK_CUDA(cudaEventCreateWithFlags(&ws.gev[0], cudaEventDisableTiming));
        HK_CHECK_CUDA(cudaEventCreateWithFlags(&ws.gev[1], cudaEventDisableTiming));
    }
    HK_CHECK_CUDA(cudaEventRecord(ws.gev[0], s));
    HK_CHECK_CUDA(cudaStreamWaitEvent(ws.gstream, ws.gev[0], 0));
    try {
        run_query_graph_on(idx, Qd, nq, k, o, ws.gstream, out_ids, out_dist, stats);
    } catch (...) {
        cudaEventRecord(ws.gev[1], ws.gstream);
        cudaStreamWaitEvent(s, ws.gev[1], 0);
        throw;
    }
    HK_CHECK_CUDA(cudaEventRecord(ws.gev[1], ws.gstream));
    HK_CHECK_CUDA(cudaStreamWaitEvent(s, ws.gev[1], 0));
}

void run_query_graph_on(hk_index *idx, const float *Qd, int nq, int k, const hk_query_opts &o, cudaStream_t s,
                        int64_t *out_ids, float *out_dist, hk_query_stats *stats) {
    Workspace &ws = idx->ws_graph;
    const long long launches0 = g_launches;
    ScanTimer timer, tctimer, tcatimer;   // off: a replay is not timed per kernel
    const int n = idx->n;
    hk_query_opts oq = o;
    oq.flags &= ~(uint32_t)(HK_Q_GRAPH | HK_Q_TIMING);
    uint64_t key[4];
    key[0] = ((uint64_t)(uint32_t)nq << 32) | (uint32_t)k;
    key[1] = ((uint64_t)oq.flags << 32) | (uint32_t)oq.l_max;
    key[2] = ((uint64_t)(uint32_t)oq.query_group << 32) | (uint32_t)oq.series_tile;
    uint32_t th[2];
    std::memcpy(&th[0], &oq.eapca_th, 4);
    std::memcpy(&th[1], &oq.sax_th, 4);
    key[3] = ((uint64_t)th[0] << 32) | th[1];
    const float *in_before = ws.Q.p;
    ws.Q.reserve((size_t)nq * n, s);
    const bool fresh = ws.gexec == nullptr || ws.Q.p != in_before ||
                       std::memcmp(key, ws.gkey, sizeof(key)) != 0;
    HK_CHECK_CUDA(cudaMemcpyAsync(ws.Q.p, Qd, (size_t)nq * n * sizeof(float), cudaMemcpyDeviceToDevice, s));
    std::vector<int32_t> flags;
    std::vector<uint32_t> Uh;
    if (fresh) {
        ws.drop_graph();
        query_pass(idx, ws, ws.Q.p, nq, k, oq, s, nullptr, nullptr, nullptr, nullptr, flags, Uh);
        const long long l0 = g_launches;
        cudaGraph_t g = nullptr;
        HK_CHECK_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
        try {
            std::vector<int32_t> f2;
            std::vector<uint32_t> u2;
            query_pass(idx, ws, ws.Q.p, nq, k, oq, s, nullptr, nullptr, nullptr, nullptr, f2, u2, true);
        } catch (...) {
            cudaStreamEndCapture(s, &g);
            if (g) cudaGraphDestroy(g);
            throw;
        }
        HK_CHECK_CUDA(cudaStreamEndCapture(s, &g));
        const cudaError_t e = cudaGraphInstantiate(&ws.gexec, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            ws.gexec = nullptr;
            fail(HK_ECUDA, "graph instantiation: %s", cudaGetErrorString(e));
        }
        ws.glaunches = g_launches - l0;
        g_launches = l0;   // recorded, not run
        std::memcpy(ws.gkey, key, sizeof(key));
    } else {
        HK_CHECK_CUDA(cudaGraphLaunch(ws.gexec, s));
        g_launches += ws.glaunches;
        flags.assign(nq, 0);
        int32_t ctr[4] = {0, 0, 0, 0};
        int bad = 0;
        HK_CHECK_CUDA(cudaMemcpyAsync(flags.data(), ws.qflag.p, nq * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        HK_CHECK_CUDA(cudaMemcpyAsync(ctr, ws.counters.p, sizeof(ctr), cudaMemcpyDeviceToHost, s));
        if (oq.flags & HK_Q_BF16)
            HK_CHECK_CUDA(cudaMemcpyAsync(&bad, ws.bad.p, sizeof(int), cudaMemcpyDeviceToHost, s));
        HK_CHECK_CUDA(cudaStreamSynchronize(s));
        if (bad) fail(HK_EINVAL, "queries have values beyond the 16-bit copy's range");
        if (ctr[2]) fail(HK_ETIMEOUT, "tensor-core scan: a bounded wait ran out (flag %d)", ctr[2]);
        if (ctr[1]) fail(HK_EINTERNAL, "a query had fewer than k candidates after the scan");
    }
    finish_query(idx, ws, idx->ws_retry, ws.Q.p, nq, k, oq, s, out_ids, out_dist, stats, flags, launches0,
                 timer, tctimer, tcatimer);
}

}  // namespace

void run_query_ws(hk_index *idx, Workspace &ws, Workspace &ws_retry, const float *Qd, int nq, int k,
                  const hk_query_opts &o, cudaStream_t s, int64_t *out_ids, float *out_dist,
                  hk_query_stats *stats) {
    if (o.flags & HK_Q_GRAPH) {
        run_query_graph(idx, Qd, nq, k, o, s, out_ids, out_dist, stats);
        return;
    }
    const long long launches0 = g_launches;
    ScanTimer timer, tctimer, tcatimer;
    timer.on = tctimer.on = tcatimer.on = (o.flags & HK_Q_TIMING) != 0;
    std::vector<int32_t> flags;
    std::vector<uint32_t> Uh;
    query_pass(idx, ws, Qd, nq, k, o, s, nullptr, &timer, &tctimer, &tcatimer, flags, Uh);
    finish_query(idx, ws, ws_retry, Qd, nq, k, o, s, out_ids, out_dist, stats, flags, launches0, timer, tctimer,
                 tcatimer);
}

namespace {

void finish_query(hk_index *idx, Workspace &ws, Workspace &ws_retry, const float *Qd, int nq, int k,
                  const hk_query_opts &o, cudaStream_t s, int64_t *out_ids, float *out_dist,
                  hk_query_stats *stats, const std::vector<int32_t> &flags, long long launches0,
                  ScanTimer &timer, ScanTimer &tctimer, ScanTimer &tcatimer) {
    // Queries whose lists or pool overflowed: run them again starting from
    // their final bound, which is tight, so far fewer candidates qualify.
    std::vector<int32_t> sel;
    for (int q = 0; q < nq; ++q)
        if (flags[q] & 1) sel.push_back(q);
    if (!sel.empty()) {
        const int nsub = (int)sel.size();
        Workspace &w2 = ws_retry;
        w2.Q.reserve((size_t)nsub * idx->n, s);
        w2.Uinit.reserve(nsub, s);
        w2.sel.reserve(nsub, s);
        HK_CHECK_CUDA(cudaMemcpyAsync(w2.sel.p, sel.data(), nsub * sizeof(int32_t), cudaMemcpyHostToDevice, s));
        k_gather_queries<<<nsub, 256, 0, s>>>(Qd, idx->n, w2.sel.p, nsub, ws.U.p, w2.Q.p, w2.Uinit.p);
        HK_CHECK_LAUNCH();
        std::vector<int32_t> flags2;
        std::vector<uint32_t> U2;
        // the retry takes the float32 path: its bound is ~1e-5 relative, so
        // near-ties that crowd the precision form's wider band fit its lists
        hk_query_opts o2 = o;
        o2.flags &= ~HK_Q_BF16;
        query_pass(idx, w2, w2.Q.p, nsub, k, o2, s, w2.Uinit.p, &timer, &tctimer, &tcatimer, flags2, U2);
        LeafView v;
        v.X = idx->X.p;
        v.perm = idx->perm.p;
        v.sax = idx->sax.p;
        v.leaf_off = idx->leaf_off.p;
        v.N = idx->N;
        v.n = idx->n;
        v.L = idx->L;
        long long exhaustive = 0;
        for (int i = 0; i < nsub; ++i) {
            if (!(flags2[i] & 1)) continue;
            exhaustive_one(w2, v, w2.Q.p, i, U2[i], k, rho_for(idx->n), s);
            ++exhaustive;
        }
        k_scatter_results<<<nsub, 128, 0, s>>>(w2.out_ids.p, w2.out_dist.p, w2.sel.p, nsub, k,
                                               ws.out_ids.p, ws.out_dist.p);
        HK_CHECK_LAUNCH();
        // fold the retry's counters into the batch's
        std::vector<long long> a(kStatSlots), b(kStatSlots);
        HK_CHECK_CUDA(cudaMemcpyAsync(a.data(), ws.stats.p, kStatSlots * sizeof(long long), cudaMemcpyDeviceToHost, s));
        HK_CHECK_CUDA(cudaMemcpyAsync(b.data(), w2.stats.p, kStatSlots * sizeof(long long), cudaMemcpyDeviceToHost, s));
        HK_CHECK_CUDA(cudaStreamSynchronize(s));
        for (int i = ST_LEAVES_APPROX; i < kStatSlots; ++i)
            if (i != ST_QUERIES && i != ST_LEAVES_TOTAL) a[i] += b[i];
        a[ST_RETRIED] += nsub;
        a[ST_FALLBACK] += exhaustive;
        HK_CHECK_CUDA(cudaMemcpyAsync(ws.stats.p, a.data(), kStatSlots * sizeof(long long), cudaMemcpyHostToDevice, s));
    }
    copy_out(ws, nq, k, out_ids, out_dist, s);
    HK_CHECK_CUDA(cudaStreamSynchronize(s));
    copy_stats(ws, stats, s, &timer, g_launches - launches0);
    if (stats) {
        stats->tc_ns = tctimer.total_ns();
        stats->tc_approx_ns = tcatimer.total_ns();
    }
}

}  // namespace

void run_scan(const float *Xd, int64_t N, int n, const float *Qd, int nq, int k, cudaStream_t s,
              int64_t *out_ids, float *out_dist) {
    Workspace ws;
    const float rho = rho_for(n);
    ScanConfig cfg = choose_scan(n, k, false, 0);
    const int S_T = 2048;
    const int pool_C = std::min(65536, std::max(4096, 64 * cfg.cap));
    reserve_common(ws, nq, 1, k, pool_C, s);
    DevBuf<int64_t> leaf_off;
    leaf_off.alloc(2, s);
    const int64_t lo[2] = {0, N};
    HK_CHECK_CUDA(cudaMemcpyAsync(leaf_off.p, lo, sizeof(lo), cudaMemcpyHostToDevice, s));
    HK_CHECK_CUDA(cudaMemsetAsync(ws.stats.p, 0, kStatSlots * sizeof(long long), s));
    HK_CHECK_CUDA(cudaMemsetAsync(ws.pool_cnt.p, 0, nq * sizeof(int32_t), s));
    HK_CHECK_CUDA(cudaMemsetAsync(ws.qflag.p, 0, nq * sizeof(int32_t), s));
    HK_CHECK_CUDA(cudaMemsetAsync(ws.mask.p, 2, (size_t)nq, s));
    k_fill_u32<<<64, 256, 0, s>>>(ws.U.p, nq, 0x7f800000u);
    HK_CHECK_LAUNCH();
    LeafView v;
    v.X = Xd;
    v.perm = nullptr;
    v.sax = nullptr;
    v.leaf_off = leaf_off.p;
    v.N = N;
    v.n = n;
    v.L = 1;
    ScanArgs a{};
    a.v = v;
    a.Q = Qd;
    a.nq = nq;
    a.U = ws.U.p;
    a.S_T = S_T;
    a.k = k;
    a.cap = cfg.cap;
    a.p2 = cfg.p2;
    a.rho = rho;
    a.pool_d = ws.pool_d.p;
    a.pool_p = ws.pool_p.p;
    a.pool_cnt = ws.pool_cnt.p;
    a.pool_C = pool_C;
    a.qflag = ws.qflag.p;
    a.stats = (long long *)ws.stats.p;
    a.use_sax = 0;
    scan_phase(ws, v, a, cfg, 2, nq, s);
    std::vector<int32_t> flags;
    std::vector<uint32_t> Uh;
    final_select(ws, v, Qd, nq, k, pool_C, rho, s, flags, Uh);
    for (int q = 0; q < nq; ++q)
        if (flags[q] & 1) exhaustive_one(ws, v, Qd, q, Uh[q], k, rho, s);
    copy_out(ws, nq, k, out_ids, out_dist, s);
    HK_CHECK_CUDA(cudaStreamSynchronize(s));
}

void scan_knn_scratch(const float *Xd, int64_t N, int n, const float *Qd, int nq, int k,
                      cudaStream_t s, int64_t *ids_dev, float *dist_dev, const ScanScratch &sc) {
    const float rho = rho_for(n);
    ScanConfig cfg = choose_scan(n, k, false, 0);
    const int S_T = 2048;
    // the single-leaf work list, built on the host (stack arrays only)
    int32_t h_qoff[2] = {0, nq};
    int32_t h_q[64];
    for (int q = 0; q < nq; ++q) h_q[q] = q;
    const int64_t items = (int64_t)((nq + cfg.G - 1) / cfg.G) * ((N + S_T - 1) / S_T);
    int64_t h_item_off[2] = {0, items};
    int64_t h_leaf_off[2] = {0, N};
    HK_CHECK_CUDA(cudaMemcpyAsync(sc.leaf_qoff, h_qoff, sizeof(h_qoff), cudaMemcpyHostToDevice, s));
    HK_CHECK_CUDA(cudaMemcpyAsync(sc.leaf_q, h_q, nq * sizeof(int32_t), cudaMemcpyHostToDevice, s));
    HK_CHECK_CUDA(cudaMemcpyAsync(sc.item_off, h_item_off, sizeof(h_item_off), cudaMemcpyHostToDevice, s));
    HK_CHECK_CUDA(cudaMemcpyAsync(sc.leaf_off, h_leaf_off, sizeof(h_leaf_off), cudaMemcpyHostToDevice, s));
    // the scratch keeps the previous call's contents: clear what must start at zero
    HK_CHECK_CUDA(cudaMemsetAsync(sc.pool_cnt, 0, nq * sizeof(int32_t), s));
    HK_CHECK_CUDA(cudaMemsetAsync(sc.qflag, 0, nq * sizeof(int32_t), s));
    HK_CHECK_CUDA(cudaMemsetAsync(sc.counters, 0, 4 * sizeof(int32_t), s));
    HK_CHECK_CUDA(cudaMemsetAsync(sc.stats, 0, kStatSlots * sizeof(long long), s));
    k_fill_u32<<<1, 64, 0, s>>>(sc.U, nq, 0x7f800000u);
    HK_CHECK_LAUNCH();
    LeafView v;
    v.X = Xd;
    v.perm = nullptr;
    v.sax = nullptr;
    v.leaf_off = sc.leaf_off;
    v.N = N;
    v.n = n;
    v.L = 1;
    ScanArgs a{};
    a.v = v;
    a.Q = Qd;
    a.nq = nq;
    a.U = sc.U;
    a.leaf_qoff = sc.leaf_qoff;
    a.leaf_q = sc.leaf_q;
    a.item_off = sc.item_off;
    a.work_ctr = sc.counters;
    a.S_T = S_T;
    a.k = k;
    a.cap = cfg.cap;
    a.p2 = cfg.p2;
    a.rho = rho;
    a.pool_d = sc.pool_d;
    a.pool_p = sc.pool_p;
    a.pool_cnt = sc.pool_cnt;
    a.pool_C = sc.pool_C;
    a.qflag = sc.qflag;
    a.stats = sc.stats;
    a.use_sax = 0;
    launch_scan(a, cfg, s);
    k_pool_kth<<<nq, 512, 0, s>>>(sc.pool_d, sc.pool_cnt, sc.pool_C, k, rho, sc.U);
    HK_CHECK_LAUNCH();
    k_final<<<nq, 256, 0, s>>>(Qd, Xd, n, nullptr, sc.pool_d, sc.pool_p, sc.pool_cnt, sc.pool_C, sc.U,
                               sc.qflag, k, rho, sc.rs_d, ids_dev, dist_dev, sc.stats, sc.counters + 1,
                               nullptr);
    HK_CHECK_LAUNCH();
    int32_t flags[64];
    uint32_t U[64];
    int32_t err = 0;
    HK_CHECK_CUDA(cudaMemcpyAsync(flags, sc.qflag, nq * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    HK_CHECK_CUDA(cudaMemcpyAsync(U, sc.U, nq * sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    HK_CHECK_CUDA(cudaMemcpyAsync(&err, sc.counters + 1, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    HK_CHECK_CUDA(cudaStreamSynchronize(s));
    if (err) fail(HK_EINTERNAL, "a query had fewer than k candidates after the scan");
    const int sms = sm_count();
    for (int q = 0; q < nq; ++q) {
        if (!(flags[q] & 1)) continue;
        // more near-ties than the lists hold: collect every series at or
        // below the final bound into the scratch's collection area
        float u;
        std::memcpy(&u, &U[q], 4);
        const float T = std::nextafter(u * (1.0f + rho), INFINITY);
        HK_CHECK_CUDA(cudaMemsetAsync(sc.col_cnt, 0, 2 * sizeof(int32_t), s));
        k_collect<<<sms * 16, 256, 0, s>>>(Qd, q, Xd, n, N, T, 1, sc.col_cnt, sc.col_d, sc.col_p,
                                           sc.col_cap);
        HK_CHECK_LAUNCH();
        int32_t c = 0;
        HK_CHECK_CUDA(cudaMemcpyAsync(&c, sc.col_cnt, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        HK_CHECK_CUDA(cudaStreamSynchronize(s));
        if (c > sc.col_cap)
            fail(HK_ENOMEM, "query %d has %d near-tied candidates; the fixed scratch holds %d", q, c,
                 sc.col_cap);
        HK_CHECK_CUDA(cudaMemcpyAsync(sc.qsel, &q, sizeof(int32_t), cudaMemcpyHostToDevice, s));
        k_final<<<1, 256, 0, s>>>(Qd, Xd, n, nullptr, sc.col_d, sc.col_p, sc.col_cnt, c, sc.U, nullptr,
                                  k, rho, sc.col_r, ids_dev, dist_dev, sc.stats, sc.counters + 1,
                                  sc.qsel);
        HK_CHECK_LAUNCH();
        HK_CHECK_CUDA(cudaMemcpyAsync(&err, sc.counters + 1, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        HK_CHECK_CUDA(cudaStreamSynchronize(s));
        if (err) fail(HK_EINTERNAL, "selection failed for query %d", q);
    }
    HK_CHECK_CUDA(cudaStreamSynchronize(s));
}

// The certified interval [lo, up] of every (query, series) pair as the
// tensor-core kernel forms it, for tests of the bound.
void debug_tc_dist(hk_index *idx, const float *Qd, int nq, float *lo_host, float *up_host) {
    cudaStream_t s = idx->stream;
    Workspace ws;
    const int n = idx->n;
    const int64_t L = idx->L, N = idx->N;
    ws.Qb.reserve((size_t)nq * n, s);
    ws.q2.reserve(nq, s);
    ws.qa.reserve(nq, s);
    ws.qoff.reserve(nq, s);
    ws.bad.reserve(1, s);
    HK_CHECK_CUDA(cudaMemsetAsync(ws.bad.p, 0, sizeof(int), s));
    launch_tc_qprep(Qd, nq, n, idx->fmt16, idx->xn_max, ws.Qb.p, ws.q2.p, ws.qa.p, ws.qoff.p, ws.bad.p, s);
    reserve_common(ws, nq, L, 1, 1, s);
    HK_CHECK_CUDA(cudaMemsetAsync(ws.mask.p, 2, (size_t)L * nq, s));
    k_fill_u32<<<64, 256, 0, s>>>(ws.U.p, nq, 0x7f800000u);
    HK_CHECK_LAUNCH();
    HK_CHECK_CUDA(cudaMemsetAsync(ws.qflag.p, 0, nq * sizeof(int32_t), s));
    HK_CHECK_CUDA(cudaMemsetAsync(ws.counters.p, 0, 4 * sizeof(int32_t), s));
    LeafView v;
    v.leaf_off = idx->leaf_off.p;
    v.L = L;
    const int S_tc = 4096;
    build_lists(ws, v, 128, S_tc, 2, nq, s);
    const int cand_C = 1;
    ws.cand_cnt.reserve(nq, s);
    ws.cand_p.reserve((size_t)nq * cand_C, s);
    ws.cand_lb.reserve((size_t)nq * cand_C, s);
    HK_CHECK_CUDA(cudaMemsetAsync(ws.cand_cnt.p, 0, nq * sizeof(int32_t), s));
    DevBuf<float> dlo, dup;
    dlo.alloc((size_t)nq * N, s);
    dup.alloc((size_t)nq * N, s);
    HK_CHECK_CUDA(cudaMemsetAsync(dlo.p, 0xff, (size_t)nq * N * sizeof(float), s));   // NaN
    HK_CHECK_CUDA(cudaMemsetAsync(dup.p, 0xff, (size_t)nq * N * sizeof(float), s));
    TcArgs t{};
    t.Xb = idx->Xb.p;
    t.xq = idx->xq.p;
    t.n = n;
    t.Qb = ws.Qb.p;
    t.q2e = ws.q2.p;
    t.qa = ws.qa.p;
    t.qoff2 = ws.qoff.p;
    t.eb2 = tc_eb2();
    t.leaf_off = v.leaf_off;
    t.L = L;
    t.leaf_qoff = ws.leaf_qoff.p;
    t.leaf_q = ws.leaf_q.p;
    t.item_off = ws.item_off.p;
    t.work_ctr = ws.counters.p;
    t.S_T = S_tc;
    t.U = ws.U.p;
    t.k = 1;
    t.cand_cnt = ws.cand_cnt.p;
    t.cand_p = ws.cand_p.p;
    t.cand_lb = ws.cand_lb.p;
    t.cand_C = cand_C;
    t.qflag = ws.qflag.p;
    t.err = ws.counters.p + 2;
    t.stats = nullptr;
    t.idesc = tc_idesc(idx->fmt16);
    t.dbg_lo = dlo.p;
    t.dbg_up = dup.p;
    t.N = N;
    launch_tc_scan(t, s);
    int32_t terr = 0;
    HK_CHECK_CUDA(cudaMemcpyAsync(&terr, ws.counters.p + 2, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    HK_CHECK_CUDA(cudaMemcpyAsync(lo_host, dlo.p, (size_t)nq * N * sizeof(float), cudaMemcpyDeviceToHost, s));
    HK_CHECK_CUDA(cudaMemcpyAsync(up_host, dup.p, (size_t)nq * N * sizeof(float), cudaMemcpyDeviceToHost, s));
    HK_CHECK_CUDA(cudaStreamSynchronize(s));
    if (terr) fail(HK_ETIMEOUT, "tensor-core scan: a bounded wait ran out (flag %d)", terr);
}

void debug_lb_eapca(hk_index *idx, const float *Qd, int nq, double *out_host) {
    cudaStream_t s = idx->stream;
    Workspace &ws = idx->ws;
    ws.qseg.reserve((size_t)nq * idx->S * 2, s);
    ws.lb.reserve((size_t)nq * idx->L, s);
    k_qprep<<<nq, 256, idx->n * sizeof(float), s>>>(Qd, idx->n, idx->seg_ab.p, idx->S, ws.qseg.p, nullptr);
    HK_CHECK_LAUNCH();
    k_lb_eapca<<<dim3((unsigned)((idx->L + 127) / 128), std::min(nq, 65535)), 128, 0, s>>>(
        ws.qseg.p, idx->S, tree_view(idx), nq, ws.lb.p);
    HK_CHECK_LAUNCH();
    HK_CHECK_CUDA(cudaMemcpyAsync(out_host, ws.lb.p, (size_t)nq * idx->L * sizeof(double),
                                  cudaMemcpyDeviceToHost, s));
    HK_CHECK_CUDA(cudaStreamSynchronize(s));
}

void debug_lb_sax(hk_index *idx, const float *Qd, int nq, float *out_host) {
    cudaStream_t s = idx->stream;
    Workspace &ws = idx->ws;
    ws.sax_paa.reserve((size_t)nq * 2 * kWord, s);
    k_qprep<<<nq, 256, idx->n * sizeof(float), s>>>(Qd, idx->n, idx->seg_ab.p, idx->S, nullptr, ws.sax_paa.p);
    HK_CHECK_LAUNCH();
    DevBuf<float> out;
    out.alloc((size_t)nq * idx->N, s);
    k_debug_lbsax<<<dim3(256, std::min(nq, 65535)), 256, 0, s>>>(ws.sax_paa.p, idx->bp.p, idx->sax.p, idx->N,
                                                                  idx->n, nq, out.p);
    HK_CHECK_LAUNCH();
    HK_CHECK_CUDA(cudaMemcpyAsync(out_host, out.p, (size_t)nq * idx->N * sizeof(float),
                                  cudaMemcpyDeviceToHost, s));
    HK_CHECK_CUDA(cudaStreamSynchronize(s));
}

}  // namespace hk
