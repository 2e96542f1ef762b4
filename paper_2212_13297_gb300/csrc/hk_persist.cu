// Index persistence: hk_save / hk_load (one file holding what the paper
// keeps in HTree, LRDFile and LSDFile, Sec. 3.3).
#include <cstdio>
#include <cstring>
#include <memory>
#include <vector>

#include "hk_internal.cuh"

namespace {

constexpr char kTag[8] = {'H', 'K', 'I', 'D', 'X', '0', '0', '2'};
constexpr size_t kStage = (size_t)64 << 20;   // bytes per host staging copy

struct Header {
    int64_t N, n, tau, eval_cap, L, max_m, depth, S, Npad, has_bf16, fmt16;
    double xn_max;
    int64_t T;   // tree nodes (leaves and internal)
};

struct Fnv {
    uint64_t h = 1469598103934665603ull;
    void add(const void *p, size_t bytes) {
        const unsigned char *c = static_cast<const unsigned char *>(p);
        for (size_t i = 0; i < bytes; ++i) {
            h ^= c[i];
            h *= 1099511628211ull;
        }
    }
};

struct File {
    FILE *f = nullptr;
    ~File() {
        if (f) std::fclose(f);
    }
};

void put(File &F, const void *p, size_t bytes) {
    if (bytes && std::fwrite(p, 1, bytes, F.f) != bytes) hk::fail(HK_EIO, "write failed");
}
void get(File &F, void *p, size_t bytes) {
    if (bytes && std::fread(p, 1, bytes, F.f) != bytes) hk::fail(HK_EINVAL, "file is shorter than its header says");
}

// One array: its byte count, then its bytes (device arrays staged through
// pinned host memory).
void put_array(File &F, Fnv &sum, const void *src, size_t bytes, bool device, unsigned char *stage) {
    const uint64_t b = bytes;
    put(F, &b, sizeof(b));
    for (size_t off = 0; off < bytes; off += kStage) {
        const size_t c = std::min(kStage, bytes - off);
        const unsigned char *p = static_cast<const unsigned char *>(src) + off;
        if (device) {
            HK_CHECK_CUDA(cudaMemcpy(stage, p, c, cudaMemcpyDeviceToHost));
            p = stage;
        }
        sum.add(p, c);
        put(F, p, c);
    }
}

void get_array(File &F, Fnv &sum, void *dst, size_t bytes, bool device, unsigned char *stage, cudaStream_t s) {
    uint64_t b = 0;
    get(F, &b, sizeof(b));
    if (b != bytes) hk::fail(HK_EINVAL, "array of %llu bytes where %zu were expected", (unsigned long long)b, bytes);
    for (size_t off = 0; off < bytes; off += kStage) {
        const size_t c = std::min(kStage, bytes - off);
        unsigned char *p = static_cast<unsigned char *>(dst) + off;
        if (device) {
            get(F, stage, c);
            sum.add(stage, c);
            HK_CHECK_CUDA(cudaMemcpyAsync(p, stage, c, cudaMemcpyHostToDevice, s));
            HK_CHECK_CUDA(cudaStreamSynchronize(s));
        } else {
            get(F, p, c);
            sum.add(p, c);
        }
    }
}

struct Pinned {
    unsigned char *p = nullptr;
    ~Pinned() {
        if (p) cudaFreeHost(p);
    }
};

// The arrays of an index, in file order: (pointer, bytes, on the device)
struct Part {
    void *p;
    size_t bytes;
    bool device;
};

std::vector<Part> parts(hk_index *x) {
    const size_t N = (size_t)x->N, n = (size_t)x->n, L = (size_t)x->L, S = (size_t)x->S;
    const size_t T = (size_t)x->T, I = T - L;
    std::vector<Part> v = {
        {x->X.p, N * n * sizeof(float), true},
        {x->perm.p, N * sizeof(int64_t), true},
        {x->sax.p, N * hk::kWord, true},
        {x->leaf_off.p, (L + 1) * sizeof(int64_t), true},
        {x->leaf_nseg.p, L * sizeof(int32_t), true},
        {x->leaf_seg.p, L * hk::kMaxSeg * sizeof(int32_t), true},
        {x->env.p, L * hk::kMaxSeg * 4 * sizeof(double), true},
        {x->seg_ab.p, S * 2 * sizeof(int32_t), true},
        {x->bp.p, 255 * sizeof(float), true},
        {x->h_leaf_off.data(), (L + 1) * sizeof(int64_t), false},
        {x->h_leaf_nseg.data(), L * sizeof(int32_t), false},
        {x->h_seg_end.data(), L * hk::kMaxSeg * sizeof(int32_t), false},
        // the tree (HTree): links, levels, position ranges, internal segmentations and synopses
        {x->h_tree_parent.data(), T * sizeof(int32_t), false},
        {x->h_tree_left.data(), T * sizeof(int32_t), false},
        {x->h_tree_right.data(), T * sizeof(int32_t), false},
        {x->h_tree_level.data(), T * sizeof(int32_t), false},
        {x->h_tree_beg.data(), T * sizeof(int64_t), false},
        {x->h_tree_end.data(), T * sizeof(int64_t), false},
        {x->h_inode_nseg.data(), I * sizeof(int32_t), false},
        {x->h_inode_seg_end.data(), I * hk::kMaxSeg * sizeof(int32_t), false},
        {x->h_inode_seg.data(), I * hk::kMaxSeg * sizeof(int32_t), false},
        {x->ienv.p, I * hk::kMaxSeg * 4 * sizeof(double), true},
    };
    if (x->has_bf16) {
        v.push_back({x->Xb.p, (size_t)x->Npad * n * sizeof(uint16_t), true});
        v.push_back({x->xq.p, (size_t)x->Npad * sizeof(float2), true});
    }
    return v;
}

}  // namespace

extern "C" {

int hk_save(const hk_index *idx, const char *path) {
    try {
        hk::clear_last_error();
        if (!idx || !path) hk::fail(HK_EINVAL, "NULL argument");
        File F;
        F.f = std::fopen(path, "wb");
        if (!F.f) hk::fail(HK_EIO, "cannot open %s for writing", path);
        Header h{idx->N, idx->n, idx->tau, idx->eval_cap, idx->L, idx->max_m, idx->depth, idx->S,
                 idx->Npad, idx->has_bf16 ? 1 : 0, idx->fmt16, idx->xn_max, idx->T};
        put(F, kTag, sizeof(kTag));
        put(F, &h, sizeof(h));
        HK_CHECK_CUDA(cudaDeviceSynchronize());
        Pinned stage;
        HK_CHECK_CUDA(cudaMallocHost((void **)&stage.p, kStage));
        Fnv sum;
        for (const Part &pt : parts(const_cast<hk_index *>(idx)))
            put_array(F, sum, pt.p, pt.bytes, pt.device, stage.p);
        put(F, &sum.h, sizeof(sum.h));
        if (std::fflush(F.f) != 0) hk::fail(HK_EIO, "write failed");
        return HK_OK;
    } catch (const hk::Error &e) {
        hk::set_last_error(e.code, e.msg);
        return e.code;
    } catch (const std::bad_alloc &) {
        hk::set_last_error(HK_ENOMEM, "host allocation failed");
        return HK_ENOMEM;
    }
}

int hk_load(const char *path, void *stream, hk_index **out) {
    try {
        hk::clear_last_error();
        if (!path || !out) hk::fail(HK_EINVAL, "NULL argument");
        *out = nullptr;
        File F;
        F.f = std::fopen(path, "rb");
        if (!F.f) hk::fail(HK_EIO, "cannot open %s", path);
        char tag[8];
        if (std::fread(tag, 1, sizeof(tag), F.f) != sizeof(tag) || std::memcmp(tag, kTag, sizeof(tag)) != 0)
            hk::fail(HK_EINVAL, "%s is not an index file written by hk_save", path);
        Header h;
        get(F, &h, sizeof(h));
        const bool ok = h.N >= 1 && h.N <= 0x7fffffffLL && h.n >= HK_MIN_LEN && h.n <= HK_MAX_LEN &&
                        h.n % HK_ISAX_SEGMENTS == 0 && h.L >= 1 && h.L <= h.N && h.S >= 1 &&
                        h.S <= (2 * h.L - 1) * hk::kMaxSeg && h.max_m >= 1 && h.max_m <= hk::kMaxSeg && h.tau >= 1 &&
                        (h.has_bf16 == 0 || h.has_bf16 == 1) && (h.fmt16 == hk::kFmtF16 || h.fmt16 == hk::kFmtBF16) &&
                        (h.has_bf16 == 0 || h.Npad >= h.N) && h.T == 2 * h.L - 1 && h.depth >= 0 &&
                        h.depth < h.T;
        if (!ok) hk::fail(HK_EINVAL, "%s: inconsistent header", path);
        cudaStream_t s = (cudaStream_t)stream;
        std::unique_ptr<hk_index> idx(new hk_index());
        idx->stream = s;
        idx->N = h.N;
        idx->n = (int)h.n;
        idx->tau = (int)h.tau;
        idx->eval_cap = (int)h.eval_cap;
        idx->L = h.L;
        idx->max_m = (int)h.max_m;
        idx->depth = (int)h.depth;
        idx->S = h.S;
        idx->Npad = h.Npad;
        idx->has_bf16 = h.has_bf16 != 0;
        idx->fmt16 = (int)h.fmt16;
        idx->xn_max = h.xn_max;
        const size_t N = (size_t)h.N, n = (size_t)h.n, L = (size_t)h.L;
        idx->X.alloc(N * n, s);
        idx->perm.alloc(N, s);
        idx->sax.alloc(N * hk::kWord, s);
        idx->leaf_off.alloc(L + 1, s);
        idx->leaf_nseg.alloc(L, s);
        idx->leaf_seg.alloc(L * hk::kMaxSeg, s);
        idx->env.alloc(L * hk::kMaxSeg * 4, s);
        idx->seg_ab.alloc((size_t)h.S * 2, s);
        idx->bp.alloc(255, s);
        idx->h_leaf_off.resize(L + 1);
        idx->h_leaf_nseg.resize(L);
        idx->h_seg_end.resize(L * hk::kMaxSeg);
        const size_t T = (size_t)h.T, I = T - L;
        idx->T = h.T;
        idx->h_tree_parent.resize(T);
        idx->h_tree_left.resize(T);
        idx->h_tree_right.resize(T);
        idx->h_tree_level.resize(T);
        idx->h_tree_beg.resize(T);
        idx->h_tree_end.resize(T);
        idx->h_inode_nseg.resize(I);
        idx->h_inode_seg_end.resize(I * hk::kMaxSeg);
        idx->h_inode_seg.resize(I * hk::kMaxSeg);
        idx->ienv.alloc(I * hk::kMaxSeg * 4, s);
        if (idx->has_bf16) {
            idx->Xb.alloc((size_t)h.Npad * n, s);
            idx->xq.alloc((size_t)h.Npad, s);
        }
        Pinned stage;
        HK_CHECK_CUDA(cudaMallocHost((void **)&stage.p, kStage));
        Fnv sum;
        for (const Part &pt : parts(idx.get())) get_array(F, sum, pt.p, pt.bytes, pt.device, stage.p, s);
        uint64_t want = 0;
        get(F, &want, sizeof(want));
        if (want != sum.h) hk::fail(HK_EINVAL, "%s: checksum mismatch", path);
        // the host tables must describe a partition of [0, N)
        if (idx->h_leaf_off[0] != 0 || idx->h_leaf_off[L] != h.N)
            hk::fail(HK_EINVAL, "%s: leaf offsets do not cover the collection", path);
        for (size_t i = 0; i < L; ++i)
            if (idx->h_leaf_off[i + 1] < idx->h_leaf_off[i] || idx->h_leaf_nseg[i] < 1 ||
                idx->h_leaf_nseg[i] > hk::kMaxSeg)
                hk::fail(HK_EINVAL, "%s: inconsistent leaf table", path);
        // the tree: children of internal nodes are valid later ids, leaves
        // have none, ranges lie inside [0, N), levels fit the depth
        for (size_t u = 0; u < T; ++u) {
            const int32_t lf = idx->h_tree_left[u], rt = idx->h_tree_right[u];
            const bool internal = u >= L;
            const bool links = internal ? (lf >= 0 && rt >= 0 && (size_t)lf < T && (size_t)rt < T &&
                                           idx->h_tree_parent[lf] == (int32_t)u &&
                                           idx->h_tree_parent[rt] == (int32_t)u)
                                        : (lf == -1 && rt == -1);
            const bool range = idx->h_tree_beg[u] >= 0 && idx->h_tree_beg[u] < idx->h_tree_end[u] &&
                               idx->h_tree_end[u] <= h.N;
            const bool level = idx->h_tree_level[u] >= 0 && idx->h_tree_level[u] <= h.depth;
            const bool segs = !internal || (idx->h_inode_nseg[u - L] >= 1 && idx->h_inode_nseg[u - L] <= hk::kMaxSeg);
            if (!links || !range || !level || !segs) hk::fail(HK_EINVAL, "%s: inconsistent tree table", path);
        }
        for (size_t j = 0; j < I * hk::kMaxSeg; ++j)
            if (idx->h_inode_seg[j] < 0 || idx->h_inode_seg[j] >= h.S)
                hk::fail(HK_EINVAL, "%s: inconsistent tree table", path);
        hk::upload_tree(idx.get(), s);
        *out = idx.release();
        return HK_OK;
    } catch (const hk::Error &e) {
        hk::set_last_error(e.code, e.msg);
        return e.code;
    } catch (const std::bad_alloc &) {
        hk::set_last_error(HK_ENOMEM, "host allocation failed");
        return HK_ENOMEM;
    }
}

}  // extern "C"
