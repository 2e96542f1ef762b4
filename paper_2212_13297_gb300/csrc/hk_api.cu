// C ABI entry points: argument checks, host/device pointer handling, errors.
#include <cstring>
#include <memory>

#include "hk_internal.cuh"

#include <atomic>

namespace hk {
const char *last_error_cstr();

namespace {
std::atomic<long long> g_device_allocs{0};   // DevBuf allocations in this process
std::atomic<long long> g_fail_after{-1};     // armed: allocations left before one fails
std::atomic<unsigned long long> g_tc_wait_ns{0};
std::atomic<int> g_tc_stall{0};
}  // namespace

void note_device_alloc(size_t bytes) {
    g_device_allocs.fetch_add(1);
    long long f = g_fail_after.load();
    while (f >= 0) {
        if (g_fail_after.compare_exchange_weak(f, f - 1)) {
            if (f == 0)
                fail(HK_ENOMEM, "device allocation of %zu bytes failed (injected by "
                                "hk_debug_fail_device_alloc)", bytes);
            break;
        }
    }
}

void tc_wait_hooks(uint64_t &wait_ns, int &stall) {
    wait_ns = g_tc_wait_ns.load();
    stall = g_tc_stall.load();
}

void check_query_opts(const hk_index *idx, const hk_query_opts &o) {
    if (o.l_max < 0) fail(HK_EINVAL, "l_max=%d must be >= 0", o.l_max);
    if (o.query_group < 0 || o.series_tile < 0) fail(HK_EINVAL, "tile sizes must be >= 0");
    if (o.flags & HK_Q_BF16) {
        if (!idx->has_bf16) fail(HK_EINVAL, "HK_Q_BF16 needs an index built with HK_BUILD_BF16 or HK_BUILD_FP16");
        if (idx->n > kTcMaxLen) fail(HK_EINVAL, "HK_Q_BF16 takes series of length <= %d (n=%d)", kTcMaxLen, idx->n);
        if (o.flags & HK_Q_NOPRUNE) fail(HK_EINVAL, "HK_Q_BF16 and HK_Q_NOPRUNE exclude each other");
    }
    if ((o.flags & HK_Q_TREE) && (o.flags & HK_Q_NOPRUNE))
        fail(HK_EINVAL, "HK_Q_TREE and HK_Q_NOPRUNE exclude each other");
}
}  // namespace hk

namespace {

template <class F>
int guard(F &&f) {
    try {
        hk::clear_last_error();
        f();
        return HK_OK;
    } catch (const hk::Error &e) {
        hk::set_last_error(e.code, e.msg);
        return e.code;
    } catch (const std::bad_alloc &) {
        hk::set_last_error(HK_ENOMEM, "host allocation failed");
        return HK_ENOMEM;
    } catch (...) {
        hk::set_last_error(HK_EINTERNAL, "unexpected exception");
        return HK_EINTERNAL;
    }
}

void check_len(int32_t n) {
    if (n < HK_MIN_LEN || n > HK_MAX_LEN || n % HK_ISAX_SEGMENTS != 0)
        hk::fail(HK_EINVAL, "series length n=%d must be in [%d, %d] and divisible by %d", n,
                 HK_MIN_LEN, HK_MAX_LEN, HK_ISAX_SEGMENTS);
}

// A device copy of a host array, or the device pointer itself.
const float *device_view(const float *p, size_t count, cudaStream_t s, hk::DevBuf<float> &tmp) {
    if (hk::is_device_ptr(p)) return p;
    tmp.alloc(count, s);
    HK_CHECK_CUDA(cudaMemcpyAsync(tmp.p, p, count * sizeof(float), cudaMemcpyHostToDevice, s));
    return tmp.p;
}

}  // namespace

extern "C" {

const char *hk_version(void) { return "hercules-gb300 0.1 (sm_103a)"; }

const char *hk_last_error(void) { return hk::last_error_cstr(); }

int hk_query_opts_default(hk_query_opts *out) {
    return guard([&] {
        if (!out) hk::fail(HK_EINVAL, "out is NULL");
        std::memset(out, 0, sizeof(*out));
        out->l_max = hk::kDefaultLMax;
        out->eapca_th = hk::kDefaultEapcaTh;
        out->sax_th = hk::kDefaultSaxTh;
    });
}

int hk_debug_device_allocs(int64_t *count) {
    return guard([&] {
        if (!count) hk::fail(HK_EINVAL, "count is NULL");
        *count = hk::g_device_allocs.load();
    });
}

int hk_debug_fail_device_alloc(int64_t after) {
    return guard([&] { hk::g_fail_after.store(after < 0 ? -1 : after); });
}

int hk_debug_tc_wait(uint64_t limit_ns, int32_t stall) {
    return guard([&] {
        hk::g_tc_wait_ns.store(limit_ns);
        hk::g_tc_stall.store(stall ? 1 : 0);
    });
}

int hk_isax_breakpoints(float out[255]) {
    return guard([&] {
        if (!out) hk::fail(HK_EINVAL, "out is NULL");
        hk::isax_breakpoints(out);
    });
}

int hk_build(const float *X, int64_t N, int32_t n, const hk_build_opts *opts, void *stream,
             hk_index **out) {
    return guard([&] {
        if (!out) hk::fail(HK_EINVAL, "out is NULL");
        *out = nullptr;
        if (!X) hk::fail(HK_EINVAL, "X is NULL");
        if (N < 1 || N > 0x7fffffffLL) hk::fail(HK_EINVAL, "N=%lld must be in [1, 2^31-1]", (long long)N);
        check_len(n);
        hk_build_opts o;
        if (opts) {
            o = *opts;
        } else {
            std::memset(&o, 0, sizeof(o));
            o.leaf_capacity = 1000;
        }
        if (o.leaf_capacity < 1) hk::fail(HK_EINVAL, "leaf_capacity=%d must be >= 1", o.leaf_capacity);
        if (o.eval_cap < 0) hk::fail(HK_EINVAL, "eval_cap=%d must be >= 0", o.eval_cap);
        if ((o.flags & HK_BUILD_BF16) && (o.flags & HK_BUILD_FP16))
            hk::fail(HK_EINVAL, "HK_BUILD_BF16 and HK_BUILD_FP16 exclude each other");
        cudaStream_t s = (cudaStream_t)stream;
        const bool dev = hk::is_device_ptr(X);
        if ((o.flags & HK_BUILD_ADOPT) && !dev) hk::fail(HK_EINVAL, "HK_BUILD_ADOPT needs a device X");
        std::unique_ptr<hk_index> idx(new hk_index());
        idx->stream = s;
        hk::DevBuf<float> tmp;
        const float *Xd = device_view(X, (size_t)N * n, s, tmp);
        hk::check_finite(Xd, (int64_t)N * n, s, "X");
        hk::build_index(idx.get(), Xd, N, n, o, s);
        tmp.release();
        if (o.flags & HK_BUILD_ADOPT) HK_CHECK_CUDA(cudaFree(const_cast<float *>(X)));
        *out = idx.release();
    });
}

int hk_free(hk_index *idx) {
    return guard([&] {
        if (!idx) return;
        cudaDeviceSynchronize();
        delete idx;
    });
}

int hk_index_info_get(const hk_index *idx, hk_index_info *out) {
    return guard([&] {
        if (!idx || !out) hk::fail(HK_EINVAL, "NULL argument");
        std::memset(out, 0, sizeof(*out));
        out->N = idx->N;
        out->n = idx->n;
        out->leaf_capacity = idx->tau;
        out->leaves = idx->L;
        out->max_segments = idx->max_m;
        out->depth = idx->depth;
        out->distinct_segments = idx->S;
        out->device_bytes = (int64_t)(idx->X.bytes() + idx->perm.bytes() + idx->sax.bytes() +
                                      idx->leaf_off.bytes() + idx->leaf_nseg.bytes() +
                                      idx->leaf_seg.bytes() + idx->env.bytes() +
                                      idx->seg_ab.bytes() + idx->bp.bytes());
        out->has_bf16 = idx->has_bf16 ? 1 : 0;
        out->device_bytes += (int64_t)(idx->Xb.bytes() + idx->xq.bytes());
    });
}

int hk_query(hk_index *idx, const float *Q, int32_t nq, int32_t k, const hk_query_opts *opts,
             void *stream, int64_t *out_ids, float *out_dist, hk_query_stats *stats) {
    return guard([&] {
        if (!idx || !Q || !out_ids || !out_dist) hk::fail(HK_EINVAL, "NULL argument");
        if (nq < 1) hk::fail(HK_EINVAL, "nq=%d must be >= 1", nq);
        if (k < 1 || k > HK_MAX_K || (int64_t)k > idx->N)
            hk::fail(HK_EINVAL, "k=%d must be in [1, min(N=%lld, %d)]", k, (long long)idx->N, HK_MAX_K);
        hk_query_opts o;
        if (opts) {
            o = *opts;
        } else {
            std::memset(&o, 0, sizeof(o));
            o.eapca_th = -1.0f;
            o.sax_th = -1.0f;
        }
        hk::check_query_opts(idx, o);
        cudaStream_t s = (cudaStream_t)stream;
        idx->stream = s;
        // host queries go through the index's staging buffer: no device
        // allocation (and no cudaFree, which waits for the device) per call
        const float *Qd = Q;
        if (!hk::is_device_ptr(Q)) {
            const size_t count = (size_t)nq * idx->n;
            idx->qstage.reserve(count, s);
            HK_CHECK_CUDA(cudaMemcpyAsync(idx->qstage.p, Q, count * sizeof(float), cudaMemcpyHostToDevice, s));
            Qd = idx->qstage.p;
        }
        hk::check_finite(Qd, (int64_t)nq * idx->n, s, "Q");
        hk::run_query(idx, Qd, nq, k, o, s, out_ids, out_dist, stats);
    });
}

int hk_query_dtw(hk_index *idx, const float *Q, int32_t nq, int32_t k, int32_t band,
                 const hk_query_opts *opts, void *stream, int64_t *out_ids, float *out_dist,
                 hk_query_stats *stats) {
    return guard([&] {
        if (!idx || !Q || !out_ids || !out_dist) hk::fail(HK_EINVAL, "NULL argument");
        if (nq < 1) hk::fail(HK_EINVAL, "nq=%d must be >= 1", nq);
        if (k < 1 || k > HK_MAX_K || (int64_t)k > idx->N)
            hk::fail(HK_EINVAL, "k=%d must be in [1, min(N=%lld, %d)]", k, (long long)idx->N, HK_MAX_K);
        if (band < 0 || band > hk::kDtwMaxBand || band >= idx->n)
            hk::fail(HK_EINVAL, "band=%d must be in [0, min(%d, n-1)]", band, hk::kDtwMaxBand);
        hk_query_opts o;
        if (opts) {
            o = *opts;
        } else {
            std::memset(&o, 0, sizeof(o));
        }
        if (o.l_max < 0) hk::fail(HK_EINVAL, "l_max=%d must be >= 0", o.l_max);
        cudaStream_t s = (cudaStream_t)stream;
        idx->stream = s;
        const float *Qd = Q;
        if (!hk::is_device_ptr(Q)) {
            const size_t count = (size_t)nq * idx->n;
            idx->qstage.reserve(count, s);
            HK_CHECK_CUDA(cudaMemcpyAsync(idx->qstage.p, Q, count * sizeof(float), cudaMemcpyHostToDevice, s));
            Qd = idx->qstage.p;
        }
        hk::check_finite(Qd, (int64_t)nq * idx->n, s, "Q");
        hk::run_query_dtw(idx, Qd, nq, k, band, o, s, out_ids, out_dist, stats);
    });
}

int hk_scan_knn(const float *X, int64_t N, int32_t n, const float *Q, int32_t nq, int32_t k,
                void *stream, int64_t *out_ids, float *out_dist) {
    return guard([&] {
        if (!X || !Q || !out_ids || !out_dist) hk::fail(HK_EINVAL, "NULL argument");
        if (N < 1 || N > 0x7fffffffLL) hk::fail(HK_EINVAL, "N=%lld must be in [1, 2^31-1]", (long long)N);
        check_len(n);
        if (nq < 1) hk::fail(HK_EINVAL, "nq=%d must be >= 1", nq);
        if (k < 1 || k > HK_MAX_K || (int64_t)k > N)
            hk::fail(HK_EINVAL, "k=%d must be in [1, min(N, %d)]", k, HK_MAX_K);
        cudaStream_t s = (cudaStream_t)stream;
        hk::DevBuf<float> tx, tq;
        const float *Xd = device_view(X, (size_t)N * n, s, tx);
        const float *Qd = device_view(Q, (size_t)nq * n, s, tq);
        hk::check_finite(Xd, N * (int64_t)n, s, "X");
        hk::check_finite(Qd, nq * (int64_t)n, s, "Q");
        hk::run_scan(Xd, N, n, Qd, nq, k, s, out_ids, out_dist);
    });
}

int hk_index_export(const hk_index *idx, int64_t *perm, int64_t *leaf_off, int32_t *leaf_nseg,
                    int32_t *seg_end, double *env, uint8_t *sax) {
    return guard([&] {
        if (!idx) hk::fail(HK_EINVAL, "idx is NULL");
        const int64_t L = idx->L, N = idx->N;
        if (perm) HK_CHECK_CUDA(cudaMemcpy(perm, idx->perm.p, N * sizeof(int64_t), cudaMemcpyDeviceToHost));
        if (leaf_off) std::memcpy(leaf_off, idx->h_leaf_off.data(), (L + 1) * sizeof(int64_t));
        if (leaf_nseg) std::memcpy(leaf_nseg, idx->h_leaf_nseg.data(), L * sizeof(int32_t));
        if (seg_end) std::memcpy(seg_end, idx->h_seg_end.data(), L * hk::kMaxSeg * sizeof(int32_t));
        if (env)
            HK_CHECK_CUDA(cudaMemcpy(env, idx->env.p, L * hk::kMaxSeg * 4 * sizeof(double),
                                     cudaMemcpyDeviceToHost));
        if (sax)
            HK_CHECK_CUDA(cudaMemcpy(sax, idx->sax.p, N * hk::kWord, cudaMemcpyDeviceToHost));
    });
}

int hk_index_export_tree(const hk_index *idx, int32_t *parent, int32_t *left, int32_t *right,
                         int64_t *beg, int64_t *end, int32_t *nseg, int32_t *seg_end, double *env) {
    return guard([&] {
        if (!idx) hk::fail(HK_EINVAL, "idx is NULL");
        const int64_t L = idx->L, T = idx->T, I = T - L;
        if (parent) std::memcpy(parent, idx->h_tree_parent.data(), T * sizeof(int32_t));
        if (left) std::memcpy(left, idx->h_tree_left.data(), T * sizeof(int32_t));
        if (right) std::memcpy(right, idx->h_tree_right.data(), T * sizeof(int32_t));
        if (beg) std::memcpy(beg, idx->h_tree_beg.data(), T * sizeof(int64_t));
        if (end) std::memcpy(end, idx->h_tree_end.data(), T * sizeof(int64_t));
        if (nseg) {
            std::memcpy(nseg, idx->h_leaf_nseg.data(), L * sizeof(int32_t));
            std::memcpy(nseg + L, idx->h_inode_nseg.data(), I * sizeof(int32_t));
        }
        if (seg_end) {
            std::memcpy(seg_end, idx->h_seg_end.data(), L * hk::kMaxSeg * sizeof(int32_t));
            std::memcpy(seg_end + L * hk::kMaxSeg, idx->h_inode_seg_end.data(), I * hk::kMaxSeg * sizeof(int32_t));
        }
        if (env) {
            HK_CHECK_CUDA(cudaMemcpy(env, idx->env.p, L * hk::kMaxSeg * 4 * sizeof(double), cudaMemcpyDeviceToHost));
            if (I > 0)
                HK_CHECK_CUDA(cudaMemcpy(env + L * hk::kMaxSeg * 4, idx->ienv.p, I * hk::kMaxSeg * 4 * sizeof(double),
                                         cudaMemcpyDeviceToHost));
        }
    });
}

int hk_debug_lb_eapca(hk_index *idx, const float *Q, int32_t nq, double *out) {
    return guard([&] {
        if (!idx || !Q || !out || nq < 1) hk::fail(HK_EINVAL, "bad argument");
        hk::DevBuf<float> tmp;
        const float *Qd = device_view(Q, (size_t)nq * idx->n, idx->stream, tmp);
        hk::debug_lb_eapca(idx, Qd, nq, out);
    });
}

int hk_debug_lb_sax(hk_index *idx, const float *Q, int32_t nq, float *out) {
    return guard([&] {
        if (!idx || !Q || !out || nq < 1) hk::fail(HK_EINVAL, "bad argument");
        hk::DevBuf<float> tmp;
        const float *Qd = device_view(Q, (size_t)nq * idx->n, idx->stream, tmp);
        hk::debug_lb_sax(idx, Qd, nq, out);
    });
}

int hk_debug_tc_dist(hk_index *idx, const float *Q, int32_t nq, float *lo, float *up) {
    return guard([&] {
        if (!idx || !Q || !lo || !up || nq < 1) hk::fail(HK_EINVAL, "bad argument");
        if (!idx->has_bf16) hk::fail(HK_EINVAL, "index built without a 16-bit copy");
        if (idx->n > hk::kTcMaxLen) hk::fail(HK_EINVAL, "n=%d > %d", idx->n, hk::kTcMaxLen);
        hk::DevBuf<float> tmp;
        const float *Qd = device_view(Q, (size_t)nq * idx->n, idx->stream, tmp);
        hk::debug_tc_dist(idx, Qd, nq, lo, up);
    });
}

}  // extern "C"
