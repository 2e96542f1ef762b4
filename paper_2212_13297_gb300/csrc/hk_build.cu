// Index construction on the GPU (Sec. 3.2-3.3).
//
// The paper inserts series one at a time (Algorithm InsertSeriesToNode) and
// splits a leaf when it exceeds tau, choosing the split from the series the
// leaf holds at that moment.  With insertion in id order, the series a node
// holds when it overflows are its first tau+1 series by id, and every later
// series is routed by the split chosen then.  This file builds the same tree
// level by level: all series of a level's over-full nodes are routed at once,
// each node's policy is chosen from its first min(tau+1, eval_cap) members,
// and a stable partition keeps every node's members in ascending id order, so
// "first by id" is simply "first in the node's range".  Stable partitions
// also leave the leaves in inorder order, which is the LRDFile layout
// (Algorithms WriteIndexWorker / WriteLeafData, Sec. 3.3).
//
// Split policy (the paper defers it to DSTree): candidates per segment i, for
// the mean then the std: H-split on SG_i, V-split testing the left half, the
// right half (halves cut at floor((a+b)/2), only when b-a >= 2 and the node
// has fewer than 64 segments); threshold (v_min+v_max)*0.5, left when the
// value is below it; score n_l*E(N_l) + n_r*E(N_r), E = sum_j l_j((mu range)^2
// + (sd range)^2) over the child's segments; the first strict minimum wins;
// a candidate with an empty side is invalid; a node without a valid
// candidate stays a leaf.  All of it in binary64 with the operation order
// written here.
#include <algorithm>
#include <cstring>
#include <map>
#include <utility>

#include "hk_device.cuh"
#include "hk_internal.cuh"

namespace hk {
namespace {

constexpr int kSlotsPerSeg = 3;   // whole segment, left half, right half

struct EvalNode {          // one node whose policy is being chosen (device)
    int64_t member_off;    // first member position in ids
    int32_t E;             // members the policy is chosen from
    int32_t m;             // segments
    int32_t slot_base;     // first unit (slot) of this node
    int32_t pad;
    int32_t seg_a[kMaxSeg];
    int32_t seg_b[kMaxSeg];
    int32_t slot_whole[kMaxSeg];
    int32_t slot_h0[kMaxSeg];   // -1 when the segment cannot be halved
    int32_t slot_h1[kMaxSeg];
};

struct EvalUnit {          // (node, slot): E members' statistics over [a, b)
    int64_t member_off;
    int64_t st_off;        // offset of mu[E], sd[E] in the stats buffer
    int32_t E;
    int32_t a, b;
    int32_t pad;
};

struct PolicyOut {
    double threshold;
    int32_t valid;
    int32_t kind;          // 0 = H, 1 = V
    int32_t seg;
    int32_t half;          // -1, 0, 1
    int32_t stat;          // 0 = mean, 1 = std
    int32_t a, b;
    int32_t pad;
};

struct RouteNode {         // every node of the level, in position order
    double threshold;
    int32_t split;         // 1: route members by (a, b, stat, threshold)
    int32_t a, b, stat;
};

__global__ void k_iota(int32_t *__restrict__ ids, int64_t N) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N;
         i += (int64_t)gridDim.x * blockDim.x)
        ids[i] = (int32_t)i;
}

// Statistics of one slot for the first E members of a node.
__global__ void k_eval_stats(const float *__restrict__ X, int n, const int32_t *__restrict__ ids,
                             const EvalUnit *__restrict__ units, double *__restrict__ st) {
    const EvalUnit u = units[blockIdx.x];
    for (int j = threadIdx.x; j < u.E; j += blockDim.x) {
        const int64_t row = ids[u.member_off + j];
        double mu, sd;
        seg_stats64(X + row * (int64_t)n, u.a, u.b, mu, sd);
        st[u.st_off + j] = mu;
        st[u.st_off + u.E + j] = sd;
    }
}

// Choose the split policy of one node (block per node, 8 warps).
__global__ void __launch_bounds__(256) k_eval_choose(const EvalNode *__restrict__ nodes,
                                                     const EvalUnit *__restrict__ units,
                                                     const double *__restrict__ st,
                                                     PolicyOut *__restrict__ out) {
    __shared__ double rmin[kMaxSeg * kSlotsPerSeg][2];
    __shared__ double rmax[kMaxSeg * kSlotsPerSeg][2];
    __shared__ double score[kMaxSeg * 6];
    __shared__ int valid[kMaxSeg * 6];
    __shared__ int cslot[kMaxSeg * 6];
    __shared__ int cstat[kMaxSeg * 6];
    __shared__ int ckind[kMaxSeg * 6];
    __shared__ int cseg[kMaxSeg * 6];
    __shared__ int chalf[kMaxSeg * 6];
    __shared__ int nc_s;

    const EvalNode &nd = nodes[blockIdx.x];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    const int E = nd.E, m = nd.m;
    int nslot = 0;
    // slots are numbered slot_base .. slot_base + nslot - 1
    for (int i = 0; i < m; ++i) nslot += (nd.slot_h0[i] >= 0) ? 3 : 1;

    // ranges of every slot's statistics
    for (int s = warp; s < nslot; s += nwarp) {
        const EvalUnit &u = units[nd.slot_base + s];
        double mn0 = INFINITY, mx0 = -INFINITY, mn1 = INFINITY, mx1 = -INFINITY;
        for (int e = lane; e < E; e += 32) {
            const double mu = st[u.st_off + e], sd = st[u.st_off + E + e];
            mn0 = fmin(mn0, mu); mx0 = fmax(mx0, mu);
            mn1 = fmin(mn1, sd); mx1 = fmax(mx1, sd);
        }
        mn0 = warp_min_d(mn0); mx0 = warp_max_d(mx0);
        mn1 = warp_min_d(mn1); mx1 = warp_max_d(mx1);
        if (lane == 0) {
            rmin[s][0] = mn0; rmax[s][0] = mx0;
            rmin[s][1] = mn1; rmax[s][1] = mx1;
        }
    }
    // candidate list in tie-break order
    if (threadIdx.x == 0) {
        int c = 0;
        for (int i = 0; i < m; ++i) {
            for (int stat = 0; stat < 2; ++stat) {
                cslot[c] = nd.slot_whole[i] - nd.slot_base; cstat[c] = stat;
                ckind[c] = 0; cseg[c] = i; chalf[c] = -1; ++c;
                if (nd.slot_h0[i] >= 0 && m < kMaxSeg) {
                    cslot[c] = nd.slot_h0[i] - nd.slot_base; cstat[c] = stat;
                    ckind[c] = 1; cseg[c] = i; chalf[c] = 0; ++c;
                    cslot[c] = nd.slot_h1[i] - nd.slot_base; cstat[c] = stat;
                    ckind[c] = 1; cseg[c] = i; chalf[c] = 1; ++c;
                }
            }
        }
        nc_s = c;
    }
    __syncthreads();
    const int nc = nc_s;

    for (int c = warp; c < nc; c += nwarp) {
        const int ts = cslot[c], tstat = cstat[c];
        const double thr = __dmul_rn(__dadd_rn(rmin[ts][tstat], rmax[ts][tstat]), 0.5);
        const double *tv = st + units[nd.slot_base + ts].st_off + (tstat ? E : 0);
        int nl = 0;
        for (int e = lane; e < E; e += 32) nl += (tv[e] < thr) ? 1 : 0;
        nl = warp_sum_i(nl);
        const int nr = E - nl;
        if (nl == 0 || nr == 0) {
            if (lane == 0) { valid[c] = 0; score[c] = INFINITY; }
            continue;
        }
        // child segments in position order
        const int vseg = ckind[c] ? cseg[c] : -1;
        const int nchild = ckind[c] ? m + 1 : m;
        double el = 0.0, er = 0.0;
        for (int j = 0; j < nchild; ++j) {
            // child segment j: parent segments keep their slot; a V-split
            // segment becomes its left half (j == vseg) and right half
            int slot, len;
            if (vseg < 0 || j < vseg) {
                slot = nd.slot_whole[j] - nd.slot_base;
                len = nd.seg_b[j] - nd.seg_a[j];
            } else if (j == vseg) {
                slot = nd.slot_h0[vseg] - nd.slot_base;
                len = (nd.seg_a[vseg] + nd.seg_b[vseg]) / 2 - nd.seg_a[vseg];
            } else if (j == vseg + 1) {
                slot = nd.slot_h1[vseg] - nd.slot_base;
                len = nd.seg_b[vseg] - (nd.seg_a[vseg] + nd.seg_b[vseg]) / 2;
            } else {
                slot = nd.slot_whole[j - 1] - nd.slot_base;
                len = nd.seg_b[j - 1] - nd.seg_a[j - 1];
            }
            const double *mu_v = st + units[nd.slot_base + slot].st_off;
            const double *sd_v = mu_v + E;
            double lmn0 = INFINITY, lmx0 = -INFINITY, lmn1 = INFINITY, lmx1 = -INFINITY;
            double rmn0 = INFINITY, rmx0 = -INFINITY, rmn1 = INFINITY, rmx1 = -INFINITY;
            for (int e = lane; e < E; e += 32) {
                const double mu = mu_v[e], sd = sd_v[e];
                if (tv[e] < thr) {
                    lmn0 = fmin(lmn0, mu); lmx0 = fmax(lmx0, mu);
                    lmn1 = fmin(lmn1, sd); lmx1 = fmax(lmx1, sd);
                } else {
                    rmn0 = fmin(rmn0, mu); rmx0 = fmax(rmx0, mu);
                    rmn1 = fmin(rmn1, sd); rmx1 = fmax(rmx1, sd);
                }
            }
            lmn0 = warp_min_d(lmn0); lmx0 = warp_max_d(lmx0);
            lmn1 = warp_min_d(lmn1); lmx1 = warp_max_d(lmx1);
            rmn0 = warp_min_d(rmn0); rmx0 = warp_max_d(rmx0);
            rmn1 = warp_min_d(rmn1); rmx1 = warp_max_d(rmx1);
            const double l = (double)len;
            {
                const double dm = __dsub_rn(lmx0, lmn0), ds = __dsub_rn(lmx1, lmn1);
                const double t = __dadd_rn(__dmul_rn(dm, dm), __dmul_rn(ds, ds));
                el = __dadd_rn(el, __dmul_rn(l, t));
            }
            {
                const double dm = __dsub_rn(rmx0, rmn0), ds = __dsub_rn(rmx1, rmn1);
                const double t = __dadd_rn(__dmul_rn(dm, dm), __dmul_rn(ds, ds));
                er = __dadd_rn(er, __dmul_rn(l, t));
            }
        }
        if (lane == 0) {
            valid[c] = 1;
            score[c] = __dadd_rn(__dmul_rn((double)nl, el), __dmul_rn((double)nr, er));
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int best = -1;
        for (int c = 0; c < nc; ++c)
            if (valid[c] && (best < 0 || score[c] < score[best])) best = c;
        PolicyOut p;
        p.pad = 0;
        if (best < 0) {
            p.valid = 0; p.kind = 0; p.seg = 0; p.half = -1; p.stat = 0; p.a = 0; p.b = 0;
            p.threshold = 0.0;
        } else {
            const int ts = cslot[best];
            p.valid = 1;
            p.kind = ckind[best];
            p.seg = cseg[best];
            p.half = chalf[best];
            p.stat = cstat[best];
            p.a = units[nd.slot_base + ts].a;
            p.b = units[nd.slot_base + ts].b;
            p.threshold = __dmul_rn(__dadd_rn(rmin[ts][p.stat], rmax[ts][p.stat]), 0.5);
        }
        out[blockIdx.x] = p;
    }
}

// Route every member of a splitting node: flag 1 = goes left.
__global__ void k_route(const float *__restrict__ X, int n, const int32_t *__restrict__ ids,
                        int64_t N, const int64_t *__restrict__ node_off, int P,
                        const RouteNode *__restrict__ rn, int32_t *__restrict__ left) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int p = find_segment<int64_t>(node_off, P + 1, i);
        const RouteNode r = rn[p];
        int32_t f = 0;
        if (r.split) {
            double mu, sd;
            seg_stats64(X + (int64_t)ids[i] * n, r.a, r.b, mu, sd);
            const double v = r.stat ? sd : mu;
            f = (v < r.threshold) ? 1 : 0;
        }
        left[i] = f;
    }
}

// Stable partition within each node: left members first, both sides in order.
__global__ void k_scatter(const int32_t *__restrict__ ids, int64_t N,
                          const int64_t *__restrict__ node_off, int P,
                          const RouteNode *__restrict__ rn, const int32_t *__restrict__ left,
                          const int32_t *__restrict__ pre, int32_t *__restrict__ out) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int p = find_segment<int64_t>(node_off, P + 1, i);
        int64_t dst = i;
        if (rn[p].split) {
            const int64_t o = node_off[p], e = node_off[p + 1];
            const int64_t po = pre[o];
            const int64_t nl = (int64_t)pre[e] - po;
            const int64_t lr = (int64_t)pre[i] - po;
            dst = left[i] ? o + lr : o + nl + (i - o - lr);
        }
        out[dst] = ids[i];
    }
}

__global__ void k_gather_left_counts(const int64_t *__restrict__ node_off, int P,
                                     const int32_t *__restrict__ pre, int32_t *__restrict__ nl) {
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p < P) nl[p] = pre[node_off[p + 1]] - pre[node_off[p]];
}

// X_leaf[i] = X[ids[i]] and perm[i] = ids[i]; one warp per row.
__global__ void k_gather_rows(const float *__restrict__ X, int n, const int32_t *__restrict__ ids,
                              int64_t N, float *__restrict__ Y, int64_t *__restrict__ perm) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int nv = n >> 2;
    for (int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < N; i += warps) {
        const int64_t src = ids[i];
        const float4 *s = reinterpret_cast<const float4 *>(X + src * n);
        float4 *d = reinterpret_cast<float4 *>(Y + i * n);
        for (int v = lane; v < nv; v += 32) d[v] = __ldg(s + v);
        if (lane == 0) perm[i] = src;
    }
}

// Node synopsis (Sec. 3.2-3.3): per segment of the node's segmentation,
// min/max of mean and std over the series at positions [beg, end) -- a leaf's
// own series, or for an internal node every series that traversed it (a
// node's series occupy a contiguous run of leaf-order positions).  This is
// what the paper's ProcessLeaf / VSplitSynopsis / HSplitSynopsis fold
// arrives at.  Block per node.
__global__ void __launch_bounds__(256) k_envelope(const float *__restrict__ Y, int n,
                                                  const int64_t *__restrict__ beg,
                                                  const int64_t *__restrict__ end,
                                                  const int32_t *__restrict__ leaf_nseg,
                                                  const int32_t *__restrict__ seg_end,
                                                  double *__restrict__ env) {
    __shared__ double red[4][8];
    const int64_t leaf = blockIdx.x;
    const int64_t o = beg[leaf], e = end[leaf];
    const int m = leaf_nseg[leaf];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int a = 0;
    for (int j = 0; j < m; ++j) {
        const int b = seg_end[leaf * kMaxSeg + j];
        double mn0 = INFINITY, mx0 = -INFINITY, mn1 = INFINITY, mx1 = -INFINITY;
        for (int64_t r = o + threadIdx.x; r < e; r += blockDim.x) {
            double mu, sd;
            seg_stats64(Y + r * n, a, b, mu, sd);
            mn0 = fmin(mn0, mu); mx0 = fmax(mx0, mu);
            mn1 = fmin(mn1, sd); mx1 = fmax(mx1, sd);
        }
        mn0 = warp_min_d(mn0); mx0 = warp_max_d(mx0);
        mn1 = warp_min_d(mn1); mx1 = warp_max_d(mx1);
        if (lane == 0) {
            red[0][warp] = mn0; red[1][warp] = mx0; red[2][warp] = mn1; red[3][warp] = mx1;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            double v0 = INFINITY, v1 = -INFINITY, v2 = INFINITY, v3 = -INFINITY;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
                v0 = fmin(v0, red[0][w]); v1 = fmax(v1, red[1][w]);
                v2 = fmin(v2, red[2][w]); v3 = fmax(v3, red[3][w]);
            }
            double *z = env + (leaf * kMaxSeg + j) * 4;
            z[0] = v0; z[1] = v1; z[2] = v2; z[3] = v3;
        }
        __syncthreads();
        a = b;
    }
}

// iSAX word of every series (Sec. 2): PAA over 16 equal segments in binary64,
// symbol = number of breakpoints (float32) not above the mean.
__global__ void k_isax(const float *__restrict__ Y, int n, int64_t N,
                       const float *__restrict__ bp, uint8_t *__restrict__ sax) {
    __shared__ float bps[255];
    for (int j = threadIdx.x; j < 255; j += blockDim.x) bps[j] = bp[j];
    __syncthreads();
    const int l = n / kWord;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N;
         i += (int64_t)gridDim.x * blockDim.x) {
        const float *x = Y + i * n;
        uint32_t w[4] = {0, 0, 0, 0};
        for (int s = 0; s < kWord; ++s) {
            const double v = seg_mean64(x, s * l, (s + 1) * l);
            int lo = 0, hi = 255;   // count of bps[j] <= v: first index with bps > v
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if ((double)bps[mid] <= v) lo = mid + 1; else hi = mid;
            }
            w[s >> 2] |= (uint32_t)lo << ((s & 3) * 8);
        }
        reinterpret_cast<uint4 *>(sax)[i] = make_uint4(w[0], w[1], w[2], w[3]);
    }
}

struct HostNode {
    int64_t off, cnt;
    std::vector<int32_t> seg_end;
    bool unsplittable = false;
    int32_t tid = 0;          // its record in the tree
};

// Every node the build creates (the tree the paper writes as HTree).
struct TreeRec {
    int64_t off, cnt;         // its series: leaf-order positions [off, off + cnt)
    std::vector<int32_t> seg_end;
    int32_t parent = -1, left = -1, right = -1;
    int32_t level = 0;
};

unsigned grid_for(int64_t work, int per_block, int sms) {
    int64_t b = (work + per_block - 1) / per_block;
    const int64_t cap = (int64_t)sms * 32;
    if (b > cap) b = cap;
    if (b < 1) b = 1;
    return (unsigned)b;
}

}  // namespace

void upload_tree(hk_index *idx, cudaStream_t s) {
    const int64_t T = idx->T, L = idx->L, I = T - L;
    // nodes by level
    int maxl = 0;
    for (int64_t u = 0; u < T; ++u) maxl = std::max(maxl, idx->h_tree_level[u]);
    idx->h_level_off.assign(maxl + 2, 0);
    for (int64_t u = 0; u < T; ++u) ++idx->h_level_off[idx->h_tree_level[u] + 1];
    for (int d = 0; d <= maxl; ++d) idx->h_level_off[d + 1] += idx->h_level_off[d];
    std::vector<int32_t> lv(T), fill(idx->h_level_off.begin(), idx->h_level_off.end() - 1);
    for (int64_t u = 0; u < T; ++u) lv[fill[idx->h_tree_level[u]]++] = (int32_t)u;
    auto up32 = [&](DevBuf<int32_t> &d, const std::vector<int32_t> &h) {
        d.alloc(h.size(), s);
        if (!h.empty())
            HK_CHECK_CUDA(cudaMemcpyAsync(d.p, h.data(), h.size() * sizeof(int32_t), cudaMemcpyHostToDevice, s));
    };
    auto up64 = [&](DevBuf<int64_t> &d, const std::vector<int64_t> &h) {
        d.alloc(h.size(), s);
        if (!h.empty())
            HK_CHECK_CUDA(cudaMemcpyAsync(d.p, h.data(), h.size() * sizeof(int64_t), cudaMemcpyHostToDevice, s));
    };
    up32(idx->tree_parent, idx->h_tree_parent);
    up32(idx->tree_left, idx->h_tree_left);
    up32(idx->tree_right, idx->h_tree_right);
    up64(idx->tree_beg, idx->h_tree_beg);
    up64(idx->tree_end, idx->h_tree_end);
    up32(idx->inode_nseg, idx->h_inode_nseg);
    up32(idx->inode_seg, idx->h_inode_seg);
    up32(idx->level_nodes, lv);
    if (idx->ienv.n != (size_t)I * kMaxSeg * 4) idx->ienv.alloc((size_t)I * kMaxSeg * 4, s);
    HK_CHECK_CUDA(cudaStreamSynchronize(s));   // the host vectors above go out of scope
}

void build_index(hk_index *idx, const float *Xsrc, int64_t N, int n, const hk_build_opts &o,
                 cudaStream_t s) {
    int dev = 0, sms = 0;
    HK_CHECK_CUDA(cudaGetDevice(&dev));
    HK_CHECK_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int tau = o.leaf_capacity;
    const int eval_cap = o.eval_cap > 0 ? o.eval_cap : kDefaultEvalCap;
    idx->N = N;
    idx->n = n;
    idx->tau = tau;
    idx->eval_cap = eval_cap;

    DevBuf<int32_t> ids, ids_tmp, left, pre;
    ids.alloc(N, s);
    ids_tmp.alloc(N, s);
    left.alloc(N, s);
    pre.alloc(N + 1, s);
    DevBuf<int32_t> scan_scratch;
    k_iota<<<grid_for(N, 256, sms), 256, 0, s>>>(ids.p, N);
    HK_CHECK_LAUNCH();

    std::vector<HostNode> nodes;
    std::vector<TreeRec> tree;
    {
        HostNode root;
        root.off = 0;
        root.cnt = N;
        for (int i = 0; i < kRootSegments; ++i) root.seg_end.push_back(n / kRootSegments * (i + 1));
        root.tid = 0;
        nodes.push_back(root);
        TreeRec r;
        r.off = 0;
        r.cnt = N;
        r.seg_end = root.seg_end;
        tree.push_back(r);
    }

    DevBuf<EvalNode> d_enodes;
    DevBuf<EvalUnit> d_units;
    DevBuf<double> d_st;
    DevBuf<PolicyOut> d_pol;
    DevBuf<int64_t> d_node_off;
    DevBuf<RouteNode> d_rn;
    DevBuf<int32_t> d_nl;
    const size_t st_budget = (size_t)256 << 20;   // bytes of statistics per eval batch
    int depth = 0;

    for (;;) {
        std::vector<int> split;
        for (int p = 0; p < (int)nodes.size(); ++p)
            if (nodes[p].cnt > tau && !nodes[p].unsplittable) split.push_back(p);
        if (split.empty()) break;
        ++depth;

        // ---- choose policies, in batches bounded by the statistics budget
        std::vector<PolicyOut> pol(split.size());
        size_t bi = 0;
        while (bi < split.size()) {
            std::vector<EvalNode> en;
            std::vector<EvalUnit> un;
            int64_t st_used = 0;
            size_t bj = bi;
            for (; bj < split.size(); ++bj) {
                const HostNode &h = nodes[split[bj]];
                const int E = (int)std::min<int64_t>({h.cnt, (int64_t)tau + 1, (int64_t)eval_cap});
                const int m = (int)h.seg_end.size();
                int nslot = 0;
                for (int i = 0; i < m; ++i) {
                    const int a = i ? h.seg_end[i - 1] : 0;
                    nslot += (h.seg_end[i] - a >= 2) ? 3 : 1;
                }
                const int64_t need = (int64_t)nslot * 2 * E * (int64_t)sizeof(double);
                if (bj > bi && (st_used + need) > (int64_t)st_budget) break;
                EvalNode e{};
                e.member_off = h.off;
                e.E = E;
                e.m = m;
                e.slot_base = (int32_t)un.size();
                for (int i = 0; i < m; ++i) {
                    const int a = i ? h.seg_end[i - 1] : 0, b = h.seg_end[i];
                    e.seg_a[i] = a;
                    e.seg_b[i] = b;
                    EvalUnit u{};
                    u.member_off = h.off;
                    u.E = E;
                    u.a = a;
                    u.b = b;
                    u.st_off = st_used;
                    st_used += 2 * (int64_t)E;
                    e.slot_whole[i] = (int32_t)un.size();
                    un.push_back(u);
                    if (b - a >= 2) {
                        const int mid = (a + b) / 2;
                        u.a = a; u.b = mid; u.st_off = st_used; st_used += 2 * (int64_t)E;
                        e.slot_h0[i] = (int32_t)un.size();
                        un.push_back(u);
                        u.a = mid; u.b = b; u.st_off = st_used; st_used += 2 * (int64_t)E;
                        e.slot_h1[i] = (int32_t)un.size();
                        un.push_back(u);
                    } else {
                        e.slot_h0[i] = -1;
                        e.slot_h1[i] = -1;
                    }
                }
                en.push_back(e);
            }
            d_enodes.reserve(en.size(), s);
            d_units.reserve(un.size(), s);
            d_st.reserve((size_t)st_used, s);
            d_pol.reserve(en.size(), s);
            HK_CHECK_CUDA(cudaMemcpyAsync(d_enodes.p, en.data(), en.size() * sizeof(EvalNode),
                                          cudaMemcpyHostToDevice, s));
            HK_CHECK_CUDA(cudaMemcpyAsync(d_units.p, un.data(), un.size() * sizeof(EvalUnit),
                                          cudaMemcpyHostToDevice, s));
            k_eval_stats<<<(unsigned)un.size(), 256, 0, s>>>(Xsrc, n, ids.p, d_units.p, d_st.p);
            HK_CHECK_LAUNCH();
            k_eval_choose<<<(unsigned)en.size(), 256, 0, s>>>(d_enodes.p, d_units.p, d_st.p,
                                                               d_pol.p);
            HK_CHECK_LAUNCH();
            HK_CHECK_CUDA(cudaMemcpyAsync(pol.data() + bi, d_pol.p, en.size() * sizeof(PolicyOut),
                                          cudaMemcpyDeviceToHost, s));
            HK_CHECK_CUDA(cudaStreamSynchronize(s));
            bi = bj;
        }

        // ---- route and partition
        const int P = (int)nodes.size();
        std::vector<int64_t> off(P + 1);
        std::vector<RouteNode> rn(P);
        for (int p = 0; p < P; ++p) {
            off[p] = nodes[p].off;
            rn[p] = RouteNode{0.0, 0, 0, 0, 0};
        }
        off[P] = N;
        int nsplit = 0;
        for (size_t t = 0; t < split.size(); ++t) {
            const PolicyOut &q = pol[t];
            if (!q.valid) {
                nodes[split[t]].unsplittable = true;
                continue;
            }
            rn[split[t]] = RouteNode{q.threshold, 1, q.a, q.b, q.stat};
            ++nsplit;
        }
        if (nsplit == 0) continue;
        d_node_off.reserve(P + 1, s);
        d_rn.reserve(P, s);
        d_nl.reserve(P, s);
        HK_CHECK_CUDA(cudaMemcpyAsync(d_node_off.p, off.data(), (P + 1) * sizeof(int64_t),
                                      cudaMemcpyHostToDevice, s));
        HK_CHECK_CUDA(cudaMemcpyAsync(d_rn.p, rn.data(), P * sizeof(RouteNode),
                                      cudaMemcpyHostToDevice, s));
        k_route<<<grid_for(N, 256, sms), 256, 0, s>>>(Xsrc, n, ids.p, N, d_node_off.p, P, d_rn.p,
                                                      left.p);
        HK_CHECK_LAUNCH();
        exclusive_scan_i32(left.p, pre.p, N, s, scan_scratch);
        k_scatter<<<grid_for(N, 256, sms), 256, 0, s>>>(ids.p, N, d_node_off.p, P, d_rn.p, left.p,
                                                        pre.p, ids_tmp.p);
        HK_CHECK_LAUNCH();
        k_gather_left_counts<<<(P + 255) / 256, 256, 0, s>>>(d_node_off.p, P, pre.p, d_nl.p);
        HK_CHECK_LAUNCH();
        std::vector<int32_t> nl(P);
        HK_CHECK_CUDA(cudaMemcpyAsync(nl.data(), d_nl.p, P * sizeof(int32_t),
                                      cudaMemcpyDeviceToHost, s));
        HK_CHECK_CUDA(cudaStreamSynchronize(s));
        std::swap(ids, ids_tmp);

        std::vector<HostNode> next;
        next.reserve(nodes.size() + nsplit);
        std::vector<int> pol_of(P, -1);
        for (size_t t = 0; t < split.size(); ++t) pol_of[split[t]] = (int)t;
        for (int p = 0; p < P; ++p) {
            if (!rn[p].split) {
                next.push_back(nodes[p]);
                continue;
            }
            const PolicyOut &q = pol[pol_of[p]];
            std::vector<int32_t> cs = nodes[p].seg_end;
            if (q.kind == 1) {
                const int a = q.seg ? cs[q.seg - 1] : 0, b = cs[q.seg];
                cs.insert(cs.begin() + q.seg, (a + b) / 2);
            }
            if (nl[p] <= 0 || nl[p] >= nodes[p].cnt)
                fail(HK_EINTERNAL, "split produced an empty child (node %d, %d of %lld left)", p,
                     nl[p], (long long)nodes[p].cnt);
            HostNode L, R;
            L.off = nodes[p].off;
            L.cnt = nl[p];
            L.seg_end = cs;
            R.off = nodes[p].off + nl[p];
            R.cnt = nodes[p].cnt - nl[p];
            R.seg_end = cs;
            const int32_t pt = nodes[p].tid;
            for (HostNode *c : {&L, &R}) {
                c->tid = (int32_t)tree.size();
                TreeRec r;
                r.off = c->off;
                r.cnt = c->cnt;
                r.seg_end = cs;
                r.parent = pt;
                r.level = tree[pt].level + 1;
                tree.push_back(r);
            }
            tree[pt].left = L.tid;
            tree[pt].right = R.tid;
            next.push_back(L);
            next.push_back(R);
        }
        nodes.swap(next);
    }
    left.release();
    pre.release();
    ids_tmp.release();
    d_st.release();

    // ---- leaves in position (= inorder) order
    const int64_t L = (int64_t)nodes.size();
    idx->L = L;
    idx->depth = depth;
    idx->h_leaf_off.resize(L + 1);
    idx->h_leaf_nseg.resize(L);
    idx->h_seg_end.assign(L * kMaxSeg, 0);
    std::map<std::pair<int, int>, int> segid;
    std::vector<int32_t> leaf_seg(L * kMaxSeg, 0);
    int max_m = 0;
    for (int64_t p = 0; p < L; ++p) {
        idx->h_leaf_off[p] = nodes[p].off;
        const int m = (int)nodes[p].seg_end.size();
        idx->h_leaf_nseg[p] = m;
        max_m = std::max(max_m, m);
        int a = 0;
        for (int j = 0; j < m; ++j) {
            const int b = nodes[p].seg_end[j];
            idx->h_seg_end[p * kMaxSeg + j] = b;
            auto key = std::make_pair(a, b);
            auto it = segid.find(key);
            int id;
            if (it == segid.end()) {
                id = (int)segid.size();
                segid.emplace(key, id);
            } else {
                id = it->second;
            }
            leaf_seg[p * kMaxSeg + j] = id;
            a = b;
        }
    }
    idx->h_leaf_off[L] = N;
    idx->max_m = max_m;
    // internal nodes: unified node ids are leaves 0..L-1 (position order),
    // then internal nodes L..T-1 in creation order (parents before children)
    std::vector<int32_t> uid(tree.size(), -1);
    for (int64_t p = 0; p < L; ++p) uid[nodes[p].tid] = (int32_t)p;
    int32_t next_id = (int32_t)L;
    for (size_t t = 0; t < tree.size(); ++t)
        if (tree[t].left >= 0) uid[t] = next_id++;
    const int64_t T = next_id, I = T - L;
    idx->T = T;
    idx->h_tree_parent.assign(T, -1);
    idx->h_tree_left.assign(T, -1);
    idx->h_tree_right.assign(T, -1);
    idx->h_tree_level.assign(T, 0);
    idx->h_tree_beg.assign(T, 0);
    idx->h_tree_end.assign(T, 0);
    idx->h_inode_nseg.assign(I, 0);
    idx->h_inode_seg_end.assign(I * kMaxSeg, 0);
    idx->h_inode_seg.assign(I * kMaxSeg, 0);
    std::vector<int32_t> &inode_seg = idx->h_inode_seg;
    for (size_t t = 0; t < tree.size(); ++t) {
        const TreeRec &r = tree[t];
        const int32_t u = uid[t];
        idx->h_tree_parent[u] = r.parent >= 0 ? uid[r.parent] : -1;
        idx->h_tree_left[u] = r.left >= 0 ? uid[r.left] : -1;
        idx->h_tree_right[u] = r.right >= 0 ? uid[r.right] : -1;
        idx->h_tree_level[u] = r.level;
        idx->h_tree_beg[u] = r.off;
        idx->h_tree_end[u] = r.off + r.cnt;
        if (u < L) continue;
        const int64_t j0 = u - L;
        const int m = (int)r.seg_end.size();
        idx->h_inode_nseg[j0] = m;
        int a = 0;
        for (int j = 0; j < m; ++j) {
            const int b = r.seg_end[j];
            idx->h_inode_seg_end[j0 * kMaxSeg + j] = b;
            auto key = std::make_pair(a, b);
            auto it = segid.find(key);
            int id;
            if (it == segid.end()) {
                id = (int)segid.size();
                segid.emplace(key, id);
            } else {
                id = it->second;
            }
            inode_seg[j0 * kMaxSeg + j] = id;
            a = b;
        }
    }
    idx->S = (int64_t)segid.size();
    std::vector<int32_t> seg_ab(2 * segid.size());
    for (auto &kv : segid) {
        seg_ab[2 * kv.second] = kv.first.first;
        seg_ab[2 * kv.second + 1] = kv.first.second;
    }

    idx->leaf_off.alloc(L + 1, s);
    idx->leaf_nseg.alloc(L, s);
    idx->leaf_seg.alloc(L * kMaxSeg, s);
    idx->env.alloc(L * kMaxSeg * 4, s);
    idx->seg_ab.alloc(seg_ab.size(), s);
    DevBuf<int32_t> d_seg_end;
    d_seg_end.alloc(L * kMaxSeg, s);
    HK_CHECK_CUDA(cudaMemcpyAsync(idx->leaf_off.p, idx->h_leaf_off.data(), (L + 1) * sizeof(int64_t),
                                  cudaMemcpyHostToDevice, s));
    HK_CHECK_CUDA(cudaMemcpyAsync(idx->leaf_nseg.p, idx->h_leaf_nseg.data(), L * sizeof(int32_t),
                                  cudaMemcpyHostToDevice, s));
    HK_CHECK_CUDA(cudaMemcpyAsync(idx->leaf_seg.p, leaf_seg.data(), leaf_seg.size() * sizeof(int32_t),
                                  cudaMemcpyHostToDevice, s));
    HK_CHECK_CUDA(cudaMemcpyAsync(d_seg_end.p, idx->h_seg_end.data(), L * kMaxSeg * sizeof(int32_t),
                                  cudaMemcpyHostToDevice, s));
    HK_CHECK_CUDA(cudaMemcpyAsync(idx->seg_ab.p, seg_ab.data(), seg_ab.size() * sizeof(int32_t),
                                  cudaMemcpyHostToDevice, s));

    // ---- leaf-ordered raw series (LRDFile) and ids
    idx->X.alloc((size_t)N * n, s);
    idx->perm.alloc(N, s);
    k_gather_rows<<<grid_for(N * 32, 256, sms), 256, 0, s>>>(Xsrc, n, ids.p, N, idx->X.p,
                                                             idx->perm.p);
    HK_CHECK_LAUNCH();
    ids.release();

    // ---- synopses and iSAX words (LSDFile)
    k_envelope<<<(unsigned)L, 256, 0, s>>>(idx->X.p, n, idx->leaf_off.p, idx->leaf_off.p + 1,
                                           idx->leaf_nseg.p, d_seg_end.p, idx->env.p);
    HK_CHECK_LAUNCH();
    upload_tree(idx, s);
    if (I > 0) {
        DevBuf<int32_t> d_iseg_end;
        d_iseg_end.alloc(I * kMaxSeg, s);
        HK_CHECK_CUDA(cudaMemcpyAsync(d_iseg_end.p, idx->h_inode_seg_end.data(), I * kMaxSeg * sizeof(int32_t),
                                      cudaMemcpyHostToDevice, s));
        k_envelope<<<(unsigned)I, 256, 0, s>>>(idx->X.p, n, idx->tree_beg.p + L, idx->tree_end.p + L,
                                               idx->inode_nseg.p, d_iseg_end.p, idx->ienv.p);
        HK_CHECK_LAUNCH();
        HK_CHECK_CUDA(cudaStreamSynchronize(s));
    }
    float hbp[255];
    isax_breakpoints(hbp);
    idx->bp.alloc(255, s);
    HK_CHECK_CUDA(cudaMemcpyAsync(idx->bp.p, hbp, sizeof(hbp), cudaMemcpyHostToDevice, s));
    idx->sax.alloc((size_t)N * kWord, s);
    k_isax<<<grid_for(N, 256, sms), 256, 0, s>>>(idx->X.p, n, N, idx->bp.p, idx->sax.p);
    HK_CHECK_LAUNCH();
    if (o.flags & (HK_BUILD_BF16 | HK_BUILD_FP16)) {
        // 16-bit copy for the tensor-core form: rows padded so a 128-series
        // tile starting at any 8-aligned position stays inside the buffer
        const int fmt = (o.flags & HK_BUILD_FP16) ? kFmtF16 : kFmtBF16;
        idx->Npad = ((N + 7) / 8) * 8 + 136;
        idx->Xb.alloc((size_t)idx->Npad * n, s);
        idx->xq.alloc(idx->Npad, s);
        DevBuf<unsigned> flags;
        flags.alloc(2, s);
        HK_CHECK_CUDA(cudaMemsetAsync(flags.p, 0, 2 * sizeof(unsigned), s));
        launch_make_16(idx->X.p, N, n, idx->Npad, fmt, idx->Xb.p, idx->xq.p,
                       reinterpret_cast<int *>(flags.p), s);
        launch_max_norm(idx->xq.p, N, flags.p + 1, s);
        unsigned h[2];
        HK_CHECK_CUDA(cudaMemcpyAsync(h, flags.p, sizeof(h), cudaMemcpyDeviceToHost, s));
        HK_CHECK_CUDA(cudaStreamSynchronize(s));
        if (h[0]) fail(HK_EINVAL, "HK_BUILD_FP16: the collection has values beyond float16's range");
        float xm;
        std::memcpy(&xm, &h[1], 4);
        idx->xn_max = (double)xm;
        idx->fmt16 = fmt;
        idx->has_bf16 = true;
    }
    HK_CHECK_CUDA(cudaStreamSynchronize(s));
}

}  // namespace hk
