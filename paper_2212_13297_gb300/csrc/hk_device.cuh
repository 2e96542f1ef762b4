// Device helpers shared by the build and query kernels.
//
// Binary64 arithmetic that must reproduce a definition exactly (segment
// statistics, LB_EAPCA, the final squared distance) is written with the
// explicit round-to-nearest intrinsics so the compiler cannot fuse a multiply
// and an add, and every sum runs sequentially in index order.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace hk {

// Mean and population standard deviation of x[a..b) (EAPCA segment
// statistics, Sec. 3.2): two passes, binary64, sequential sums.
__device__ __forceinline__ void seg_stats64(const float *__restrict__ x, int a, int b,
                                            double &mu, double &sd) {
    const double l = (double)(b - a);
    double s = 0.0;
    for (int j = a; j < b; ++j) s = __dadd_rn(s, (double)x[j]);
    const double m = __ddiv_rn(s, l);
    double v = 0.0;
    for (int j = a; j < b; ++j) {
        const double d = __dsub_rn((double)x[j], m);
        v = __dadd_rn(v, __dmul_rn(d, d));
    }
    mu = m;
    sd = __dsqrt_rn(__ddiv_rn(v, l));
}

__device__ __forceinline__ double seg_mean64(const float *__restrict__ x, int a, int b) {
    double s = 0.0;
    for (int j = a; j < b; ++j) s = __dadd_rn(s, (double)x[j]);
    return __ddiv_rn(s, (double)(b - a));
}

// Distance from v to the closed range [lo, hi].
__device__ __forceinline__ double dist_to_range64(double v, double lo, double hi) {
    if (v < lo) return __dsub_rn(lo, v);
    if (v > hi) return __dsub_rn(v, hi);
    return 0.0;
}

// Squared Euclidean distance in binary64, summed in index order: the
// definition the answer is ranked by.
__device__ __forceinline__ double dist2_64(const float *__restrict__ q,
                                           const float *__restrict__ x, int n) {
    double s = 0.0;
    for (int j = 0; j < n; ++j) {
        const double d = __dsub_rn((double)q[j], (double)x[j]);
        s = __dadd_rn(s, __dmul_rn(d, d));
    }
    return s;
}

// Order-preserving maps between doubles and unsigned 64-bit keys (for
// atomic min/max on binary64 values).
__device__ __forceinline__ unsigned long long dkey(double v) {
    unsigned long long u = (unsigned long long)__double_as_longlong(v);
    return (u & 0x8000000000000000ULL) ? ~u : (u | 0x8000000000000000ULL);
}
__device__ __forceinline__ double dkey_inv(unsigned long long u) {
    u = (u & 0x8000000000000000ULL) ? (u & 0x7fffffffffffffffULL) : ~u;
    return __longlong_as_double((long long)u);
}

__device__ __forceinline__ double warp_min_d(double v) {
    for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}
__device__ __forceinline__ double warp_max_d(double v) {
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}
__device__ __forceinline__ int warp_sum_i(int v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ long long warp_sum_ll(long long v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ void stat_add(long long *p, long long v) {
    atomicAdd(reinterpret_cast<unsigned long long *>(p), (unsigned long long)v);
}

// Binary search: index p with off[p] <= pos < off[p+1] (off ascending, count+1 entries).
template <class T>
__device__ __forceinline__ int find_segment(const T *__restrict__ off, int count, T pos) {
    int lo = 0, hi = count - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (off[mid] <= pos) lo = mid; else hi = mid - 1;
    }
    return lo;
}

}  // namespace hk
