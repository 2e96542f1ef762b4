// hk_scan_knn_noalloc: the exhaustive exact k-NN scan for callers that must
// not allocate device memory.
//
// Some callers cannot call cudaMalloc or cudaFree: a process whose device
// memory is all owned by another allocator (a framework's caching allocator
// can leave too little free memory for a raw cudaMalloc to succeed), or a
// latency-bound caller sharing the GPU with other streams (cudaFree waits for
// the whole device).  This entry point works only in buffers the caller
// passes and in a fixed scratch area compiled into the library.
//
// The scratch is a file-scope __device__ array of kScratchBytes.  Every GPU
// that loads the library holds it until the process exits.  Host code cannot
// use the array's name as a device address (on the host it names a stand-in),
// so the first call on each device, with that device current, looks the
// address up with cudaGetSymbolAddress and keeps it; that first call should
// come before any stream capture.  All calls share the array and it keeps the
// previous call's contents: each call clears what must start at zero, and
// calls whose work overlaps on the GPU (different streams, or different host
// threads on the same device) race on it.
#include <mutex>

#include "hk_internal.cuh"

namespace {

constexpr int kMaxNq = 64;               // queries per call
constexpr int kMaxK = 64;                // neighbours per query
constexpr int kPoolC = 4096;             // pooled candidates per query
constexpr int kColCap = 65536;           // near-tied candidates one query may have
constexpr size_t kScratchBytes = 6u << 20;

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_addr[kMaxDevices] = {};

// Device address of g_scratch on the current device (looked up once).
unsigned char *scratch_base() {
    int dev = 0;
    HK_CHECK_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) hk::fail(HK_EINVAL, "device %d out of range", dev);
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess || !p)
            hk::fail(HK_ECUDA, "cudaGetSymbolAddress of the scratch failed: %s", cudaGetErrorString(e));
        g_addr[dev] = p;
    }
    return static_cast<unsigned char *>(g_addr[dev]);
}

// Carve 256-byte-aligned pieces out of the scratch.
struct Carver {
    unsigned char *base;
    size_t off = 0;
    template <class T>
    T *take(size_t count) {
        off = (off + 255) & ~size_t(255);
        T *p = reinterpret_cast<T *>(base + off);
        off += count * sizeof(T);
        // the last 256 bytes hold the NaN/Inf counter
        if (off > kScratchBytes - 256)
            hk::fail(HK_EINTERNAL, "scratch layout exceeds %zu bytes", kScratchBytes - 256);
        return p;
    }
};

hk::ScanScratch carve(unsigned char *base) {
    Carver c{base};
    hk::ScanScratch s{};
    s.pool_C = kPoolC;
    s.col_cap = kColCap;
    s.max_nq = kMaxNq;
    s.U = c.take<uint32_t>(kMaxNq);
    s.pool_d = c.take<float>((size_t)kMaxNq * kPoolC);
    s.pool_p = c.take<int32_t>((size_t)kMaxNq * kPoolC);
    s.rs_d = c.take<double>((size_t)kMaxNq * kPoolC);
    s.pool_cnt = c.take<int32_t>(kMaxNq);
    s.qflag = c.take<int32_t>(kMaxNq);
    s.leaf_qoff = c.take<int32_t>(2);
    s.leaf_q = c.take<int32_t>(kMaxNq);
    s.item_off = c.take<int64_t>(2);
    s.leaf_off = c.take<int64_t>(2);
    s.counters = c.take<int32_t>(4);
    s.stats = c.take<long long>(24);
    s.col_d = c.take<float>(kColCap);
    s.col_p = c.take<int32_t>(kColCap);
    s.col_r = c.take<double>(kColCap);
    s.col_cnt = c.take<int32_t>(2);
    s.qsel = c.take<int32_t>(1);
    return s;
}

unsigned long long *nonfinite_counter(unsigned char *base) {
    return reinterpret_cast<unsigned long long *>(base + kScratchBytes - 256);
}

}  // namespace

extern "C" int hk_scan_knn_noalloc(const float *X, int64_t N, int32_t n, const float *Q, int32_t nq,
                                   int32_t k, void *stream, int64_t *out_ids, float *out_dist) {
    try {
        hk::clear_last_error();
        if (!X || !Q || !out_ids || !out_dist) hk::fail(HK_EINVAL, "NULL argument");
        if (N < 1 || N > 0x7fffffffLL) hk::fail(HK_EINVAL, "N=%lld must be in [1, 2^31-1]", (long long)N);
        if (n < HK_MIN_LEN || n > HK_MAX_LEN || n % HK_ISAX_SEGMENTS != 0)
            hk::fail(HK_EINVAL, "series length n=%d must be in [%d, %d] and divisible by %d", n,
                     HK_MIN_LEN, HK_MAX_LEN, HK_ISAX_SEGMENTS);
        if (nq < 1 || nq > kMaxNq)
            hk::fail(HK_EINVAL, "nq=%d: this entry point answers 1..%d queries per call", nq, kMaxNq);
        if (k < 1 || k > kMaxK || (int64_t)k > N)
            hk::fail(HK_EINVAL, "k=%d: this entry point answers 1..min(N, %d) neighbours", k, kMaxK);
        if (!hk::is_device_ptr(X) || !hk::is_device_ptr(Q) || !hk::is_device_ptr(out_ids) ||
            !hk::is_device_ptr(out_dist))
            hk::fail(HK_EINVAL, "X, Q and both outputs must be device memory (nothing is copied)");
        cudaStream_t s = (cudaStream_t)stream;
        unsigned char *base = scratch_base();
        const hk::ScanScratch sc = carve(base);
        hk::check_finite_with(X, N * (int64_t)n, s, "X", nonfinite_counter(base));
        hk::check_finite_with(Q, nq * (int64_t)n, s, "Q", nonfinite_counter(base));
        hk::scan_knn_scratch(X, N, n, Q, nq, k, s, out_ids, out_dist, sc);
        return HK_OK;
    } catch (const hk::Error &e) {
        hk::set_last_error(e.code, e.msg);
        return e.code;
    } catch (...) {
        hk::set_last_error(HK_EINTERNAL, "unexpected exception");
        return HK_EINTERNAL;
    }
}
