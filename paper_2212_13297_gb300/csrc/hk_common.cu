// Errors, pointer classification, iSAX breakpoints, device scans.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>

#include "hk_internal.cuh"

namespace hk {

thread_local long long g_launches = 0;

namespace {
thread_local std::string g_last_error;
}

void set_last_error(int code, const std::string &msg) {
    (void)code;
    g_last_error = msg;
}
void clear_last_error() { g_last_error.clear(); }
const char *last_error_cstr() { return g_last_error.c_str(); }

[[noreturn]] void fail(int code, const char *fmt, ...) {
    char buf[1024];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    throw Error{code, std::string(buf)};
}

bool is_device_ptr(const void *p) {
    cudaPointerAttributes a;
    cudaError_t e = cudaPointerGetAttributes(&a, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// iSAX breakpoints (Sec. 2: alphabet 256): beta_j solves Phi(beta) = j/256,
// Phi(x) = erfc(-x/sqrt 2)/2.  Newton's method from x = 0: Phi is convex left
// of 0 and concave right of it, so the iterates approach each root
// monotonically from the side of 0; stop when the step stops changing x.
void isax_breakpoints(float out[255]) {
    const double inv_sqrt2 = 0.70710678118654752440;
    const double inv_sqrt2pi = 0.39894228040143267794;
    for (int j = 1; j <= 255; ++j) {
        const double p = (double)j / 256.0;
        double x = 0.0;
        for (int it = 0; it < 200; ++it) {
            const double f = 0.5 * erfc(-x * inv_sqrt2) - p;
            const double d = inv_sqrt2pi * exp(-0.5 * x * x);
            const double nx = x - f / d;
            if (nx == x || fabs(nx - x) <= 1e-17 * fabs(x)) {
                x = nx;
                break;
            }
            x = nx;
        }
        out[j - 1] = (float)x;
    }
}

// ---------------------------------------------------------------- scans
namespace {
constexpr int kScanBlock = 1024;
constexpr int kScanItems = 4;   // elements per thread
constexpr int kScanTile = kScanBlock * kScanItems;

template <class OutT>
__device__ OutT block_exclusive_scan(OutT v, OutT *smem_warp, OutT &total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    OutT x = v;
    for (int o = 1; o < 32; o <<= 1) {
        OutT y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) smem_warp[warp] = x;
    __syncthreads();
    if (warp == 0) {
        OutT w = (lane < (int)(blockDim.x >> 5)) ? smem_warp[lane] : OutT(0);
        for (int o = 1; o < 32; o <<= 1) {
            OutT y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        smem_warp[lane] = w;
    }
    __syncthreads();
    OutT base = warp > 0 ? smem_warp[warp - 1] : OutT(0);
    total = smem_warp[(blockDim.x >> 5) - 1];
    __syncthreads();
    return base + x - v;
}

template <class OutT>
__global__ void k_tile_sums(const int32_t *__restrict__ in, int64_t n, OutT *__restrict__ sums) {
    __shared__ OutT sw[32];
    const int64_t base = (int64_t)blockIdx.x * kScanTile;
    OutT acc = 0;
    for (int i = 0; i < kScanItems; ++i) {
        int64_t p = base + (int64_t)threadIdx.x * kScanItems + i;
        if (p < n) acc += (OutT)in[p];
    }
    OutT total;
    block_exclusive_scan<OutT>(acc, sw, total);
    if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

// Single block: exclusive scan of the tile sums in place (any length).
template <class OutT>
__global__ void k_scan_sums(OutT *__restrict__ sums, int64_t m) {
    __shared__ OutT sw[32];
    __shared__ OutT carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int64_t base = 0; base < m; base += blockDim.x) {
        int64_t p = base + threadIdx.x;
        OutT v = p < m ? sums[p] : OutT(0);
        OutT total;
        OutT ex = block_exclusive_scan<OutT>(v, sw, total);
        if (p < m) sums[p] = carry + ex;
        __syncthreads();
        if (threadIdx.x == 0) carry += total;
        __syncthreads();
    }
    if (threadIdx.x == 0) sums[m] = carry;
}

template <class OutT>
__global__ void k_scan_tiles(const int32_t *__restrict__ in, int64_t n,
                             const OutT *__restrict__ sums, OutT *__restrict__ out) {
    __shared__ OutT sw[32];
    const int64_t base = (int64_t)blockIdx.x * kScanTile;
    OutT v[kScanItems];
    OutT acc = 0;
    for (int i = 0; i < kScanItems; ++i) {
        int64_t p = base + (int64_t)threadIdx.x * kScanItems + i;
        v[i] = p < n ? (OutT)in[p] : OutT(0);
        acc += v[i];
    }
    OutT total;
    OutT ex = block_exclusive_scan<OutT>(acc, sw, total) + sums[blockIdx.x];
    for (int i = 0; i < kScanItems; ++i) {
        int64_t p = base + (int64_t)threadIdx.x * kScanItems + i;
        if (p < n) out[p] = ex;
        ex += v[i];
    }
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) {
        // out[n] = grand total
        out[n] = sums[gridDim.x];
    }
}

template <class OutT>
void exclusive_scan_impl(const int32_t *in, OutT *out, int64_t n, cudaStream_t s,
                         DevBuf<OutT> &scratch) {
    int64_t tiles = (n + kScanTile - 1) / kScanTile;
    if (tiles == 0) {
        HK_CHECK_CUDA(cudaMemsetAsync(out, 0, sizeof(OutT), s));
        return;
    }
    scratch.reserve((size_t)tiles + 1, s);
    k_tile_sums<OutT><<<(unsigned)tiles, kScanBlock, 0, s>>>(in, n, scratch.p);
    HK_CHECK_LAUNCH();
    k_scan_sums<OutT><<<1, kScanBlock, 0, s>>>(scratch.p, tiles);
    HK_CHECK_LAUNCH();
    k_scan_tiles<OutT><<<(unsigned)tiles, kScanBlock, 0, s>>>(in, n, scratch.p, out);
    HK_CHECK_LAUNCH();
}
}  // namespace

void exclusive_scan_i32(const int32_t *in, int32_t *out, int64_t n, cudaStream_t s,
                        DevBuf<int32_t> &scratch) {
    exclusive_scan_impl<int32_t>(in, out, n, s, scratch);
}
void exclusive_scan_i64(const int32_t *in, int64_t *out, int64_t n, cudaStream_t s,
                        DevBuf<int64_t> &scratch) {
    exclusive_scan_impl<int64_t>(in, out, n, s, scratch);
}

// ---------------------------------------------------------------- finiteness check
namespace {
__global__ void k_count_nonfinite(const float *__restrict__ p, int64_t count,
                                  unsigned long long *__restrict__ bad) {
    unsigned long long local = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count;
         i += (int64_t)gridDim.x * blockDim.x)
        local += isfinite(p[i]) ? 0ull : 1ull;
    for (int o = 16; o > 0; o >>= 1) local += __shfl_xor_sync(0xffffffffu, local, o);
    if ((threadIdx.x & 31) == 0 && local) atomicAdd(bad, local);
}
}  // namespace

// Count NaN/Inf values into a caller-provided device counter (zeroed here)
// and fail if there are any.  Synchronises the stream.
void check_finite_with(const float *p, int64_t count, cudaStream_t s, const char *what,
                       unsigned long long *dev_counter) {
    if (count <= 0) return;
    HK_CHECK_CUDA(cudaMemsetAsync(dev_counter, 0, sizeof(unsigned long long), s));
    int dev = 0, sms = 0;
    HK_CHECK_CUDA(cudaGetDevice(&dev));
    HK_CHECK_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    int64_t blocks = (count + 255) / 256;
    if (blocks > (int64_t)sms * 16) blocks = (int64_t)sms * 16;
    k_count_nonfinite<<<(unsigned)blocks, 256, 0, s>>>(p, count, dev_counter);
    HK_CHECK_LAUNCH();
    unsigned long long h = 0;
    HK_CHECK_CUDA(cudaMemcpyAsync(&h, dev_counter, sizeof(h), cudaMemcpyDeviceToHost, s));
    HK_CHECK_CUDA(cudaStreamSynchronize(s));
    if (h) fail(HK_EINVAL, "%s holds %llu NaN or Inf values", what, h);
}

void check_finite(const float *p, int64_t count, cudaStream_t s, const char *what) {
    if (count <= 0) return;
    DevBuf<unsigned long long> bad;
    bad.alloc(1, s);
    HK_CHECK_CUDA(cudaMemsetAsync(bad.p, 0, sizeof(unsigned long long), s));
    int dev = 0, sms = 0;
    HK_CHECK_CUDA(cudaGetDevice(&dev));
    HK_CHECK_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    int64_t blocks = (count + 255) / 256;
    if (blocks > (int64_t)sms * 16) blocks = (int64_t)sms * 16;
    k_count_nonfinite<<<(unsigned)blocks, 256, 0, s>>>(p, count, bad.p);
    HK_CHECK_LAUNCH();
    unsigned long long h = 0;
    HK_CHECK_CUDA(cudaMemcpyAsync(&h, bad.p, sizeof(h), cudaMemcpyDeviceToHost, s));
    HK_CHECK_CUDA(cudaStreamSynchronize(s));
    if (h) fail(HK_EINVAL, "%s holds %llu NaN or Inf values", what, h);
}

}  // namespace hk
