// Exact k-NN under DTW (Sec. 2: Hercules answers queries under any distance
// that has a lower-bounding distance, e.g. DTW with the bound of Keogh and
// Ratanamahatana, KAIS 2005).
//
// Distance: squared point costs and a Sakoe-Chiba band of half-width r,
//   D(i, j) = (q_i - x_j)^2 + min(D(i-1, j-1), D(i-1, j), D(i, j-1)),
// |i - j| <= r, D(-1, -1) = 0, the distance D(n-1, n-1); r = 0 is the squared
// Euclidean distance.  The answer is ranked by D in binary64 computed in that
// order (rows, then columns; one rounding for the difference, the square and
// the addition), ties to the lower id.
//
// Lower bounds, from the query's envelope L_j = min q[j-r..j+r], U_j = max:
//   * per node (leaf): sum over segments of l * gap([mu_min, mu_max],
//     [mean L, mean U])^2 -- dist(x_j, [L_j, U_j])^2 is jointly convex, so a
//     segment's sum is at least l times its value at the means (binary64);
//   * per series, from its iSAX word: (n/16) sum gap(cell, [PAA(L), PAA(U)])^2
//     (float32, rounded down);
//   * per series, from its raw points: LB_Keogh = sum dist(x_j, [L_j, U_j])^2
//     (float32, rounded down).
// Every warping path matches x_j to some q_i inside [L_j, U_j], so each bound
// is at most D.
//
// Search (the steps of Sec. 3.4 with these bounds): the leaves with the
// smallest node bound are scanned first (>= l_max leaves, >= k series); U,
// the k-th float32 distance inflated by rho, bounds the k-th distance; the
// candidate leaves (node bound <= U) are scanned next, each series pruned by
// its word's bound and then by LB_Keogh, the rest get the float32 DTW with
// early abandoning (every path crosses every row, so a row whose smallest cell
// exceeds T(U) ends the series).  A float32 DTW is within rho = gamma_{2n+4}
// of D: a cell rounds its difference, then adds its square to the best
// neighbour in one fused multiply-add (one rounding), so a path of at most
// 2n - 1 cells is a recursive sum of its costs, each carrying (1 + delta)^2,
// within gamma_{2n+1} of its exact value, and the minimum over paths is
// exact; series with float32 distance <= T(U) = U(1 + rho) go to the query's
// pool, and the final step rescores the pool's entries <= T(U_final) in
// binary64.  A pool that overflows makes its query run again from its pool's
// (tighter) bound.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "hk_device.cuh"
#include "hk_internal.cuh"

namespace hk {
namespace {

constexpr int kW = 2 * kDtwMaxBand + 1;   // cells of a band row
constexpr int kDtwAmax = 256;             // most leaves the approximate step visits
constexpr int kDtwThreads = 128;
constexpr int kDtwFinalCap = 1024;

enum DtwStat {
    DS_LEAVES_APPROX = 0, DS_LEAVES_CAND, DS_SERIES_CAND, DS_SAX_PRUNED, DS_KEOGH_PRUNED, DS_ABANDONED,
    DS_FULL, DS_CELLS, DS_RESCORED, DS_COUNT
};

__device__ __forceinline__ double gap64(double a1, double b1, double a2, double b2) {
    if (a1 > b2) return __dsub_rn(a1, b2);
    if (a2 > b1) return __dsub_rn(a2, b1);
    return 0.0;
}

// a1: envelope (exact float32 min / max), its mean over every distinct leaf
// segment (binary64, sequential), its PAA over 16 segments bracketed outward.
__global__ void k_dtw_prep(const float *__restrict__ Q, int n, int r, const int32_t *__restrict__ seg_ab,
                           int64_t S, float *__restrict__ envL, float *__restrict__ envU,
                           double *__restrict__ qseg, float *__restrict__ paa) {
    extern __shared__ float sh[];
    float *qs = sh, *Ls = sh + n, *Us = sh + 2 * n;
    const int q = blockIdx.x;
    for (int j = threadIdx.x; j < n; j += blockDim.x) qs[j] = Q[(int64_t)q * n + j];
    __syncthreads();
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
        const int a = max(0, j - r), b = min(n - 1, j + r);
        float lo = qs[a], hi = qs[a];
        for (int t = a + 1; t <= b; ++t) {
            lo = fminf(lo, qs[t]);
            hi = fmaxf(hi, qs[t]);
        }
        Ls[j] = lo;
        Us[j] = hi;
        envL[(int64_t)q * n + j] = lo;
        envU[(int64_t)q * n + j] = hi;
    }
    __syncthreads();
    for (int64_t sg = threadIdx.x; sg < S; sg += blockDim.x) {
        const int a = seg_ab[2 * sg], b = seg_ab[2 * sg + 1];
        qseg[((int64_t)q * S + sg) * 2] = seg_mean64(Ls, a, b);
        qseg[((int64_t)q * S + sg) * 2 + 1] = seg_mean64(Us, a, b);
    }
    if (threadIdx.x < kWord) {
        const int l = n / kWord, i = threadIdx.x;
        paa[(int64_t)q * 2 * kWord + i] = __double2float_rd(seg_mean64(Ls, i * l, (i + 1) * l));
        paa[(int64_t)q * 2 * kWord + kWord + i] = __double2float_ru(seg_mean64(Us, i * l, (i + 1) * l));
    }
}

// a2: the node bound of every query to every leaf (binary64, segment order).
__global__ void k_dtw_lb_leaf(const double *__restrict__ qseg, int64_t S, const int32_t *__restrict__ leaf_nseg,
                              const int32_t *__restrict__ leaf_seg, const int32_t *__restrict__ seg_ab,
                              const double *__restrict__ env, int64_t L, int nq, double *__restrict__ lb) {
    const int64_t leaf = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (leaf >= L) return;
    const int m = leaf_nseg[leaf];
    for (int q = blockIdx.y; q < nq; q += gridDim.y) {
        double acc = 0.0;
        for (int j = 0; j < m; ++j) {
            const int sid = leaf_seg[leaf * kMaxSeg + j];
            const double l = (double)(seg_ab[2 * sid + 1] - seg_ab[2 * sid]);
            const double *z = env + (leaf * kMaxSeg + j) * 4;
            const double g = gap64(z[0], z[1], qseg[((int64_t)q * S + sid) * 2], qseg[((int64_t)q * S + sid) * 2 + 1]);
            acc = __dadd_rn(acc, __dmul_rn(l, __dmul_rn(g, g)));
        }
        lb[(int64_t)q * L + leaf] = acc;
    }
}

// a3 (selection): ascending (bound, leaf) until >= l_max leaves and >= k
// series; mask 1 marks them.  Block per query.
__global__ void k_dtw_approx(const double *__restrict__ lb, int64_t L, const int64_t *__restrict__ leaf_off,
                             int l_max, int k, int nq, uint8_t *__restrict__ mask, long long *__restrict__ st) {
    __shared__ double bd[32];
    __shared__ long long bl[32];
    __shared__ long long covered;
    __shared__ int nch;
    const int q = blockIdx.x, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) { covered = 0; nch = 0; }
    __syncthreads();
    while (nch < kDtwAmax && (nch < l_max || covered < k)) {
        double best = INFINITY;
        long long bleaf = -1;
        for (int64_t f = threadIdx.x; f < L; f += blockDim.x) {
            if (mask[f * nq + q]) continue;
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
                nch = kDtwAmax;
            } else {
                mask[f * nq + q] = 1;
                covered += leaf_off[f + 1] - leaf_off[f];
                ++nch;
                stat_add(&st[DS_LEAVES_APPROX], 1);
            }
        }
        __syncthreads();
    }
}

// a4: candidate leaves: certified node bound <= U, not scanned already.
__global__ void k_dtw_mask(const double *__restrict__ lb, int64_t L, int nq, const uint32_t *__restrict__ U,
                           uint8_t *__restrict__ mask, long long *__restrict__ st) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= L * (int64_t)nq) return;
    const int64_t leaf = t / nq;
    const int q = (int)(t % nq);
    if (mask[t] != 0) return;
    const double u = (double)__uint_as_float(U[q]);
    if (!(__dmul_rd(lb[(int64_t)q * L + leaf], 1.0 - 0x1p-40) > u)) {
        mask[t] = 2;
        stat_add(&st[DS_LEAVES_CAND], 1);
    }
}

// The (leaf, query) pairs whose mask is in [vlo, vhi], for queries with
// sel[q] set (all when sel is null), appended to a list.
__global__ void k_dtw_list(const uint8_t *__restrict__ mask, int64_t L, int nq, uint8_t vlo, uint8_t vhi,
                           const uint8_t *__restrict__ sel, int64_t *__restrict__ list, int32_t *__restrict__ cnt) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= L * (int64_t)nq) return;
    const uint8_t m = mask[t];
    if (m < vlo || m > vhi) return;
    if (sel && !sel[t % nq]) return;
    list[atomicAdd(cnt, 1)] = t;
}

struct DtwScanArgs {
    const float *X;
    const uint8_t *sax;
    const float *bp;
    const int64_t *leaf_off;
    int n, r, nq;
    const float *Q, *envL, *envU, *paa;
    const uint32_t *U;
    float rho;
    int use_sax;
    const int64_t *list;
    const int32_t *list_cnt;
    int32_t *work;
    float *pool_d;
    int32_t *pool_p;
    int32_t *pool_cnt;
    int pool_C;
    int32_t *qflag;
    long long *st;
};

// One row i of the banded DTW: cell w is column j = i + w - r, from the
// row above (prev, +inf past the band) and the cell to its left; returns
// the row's smallest cell (with kMin; +inf otherwise).  Rows whose band
// lies inside [0, n) skip the column checks; the arithmetic per cell is the
// same.
template <int KW, bool kExact, bool kMin>
__device__ __forceinline__ float dtw_row(int i, float qi, const float (&prev)[KW + 1], float (&cur)[KW + 1],
                                         const float (&xw)[KW + 1], int n, int r) {
    const int wmax = kExact ? KW - 1 : 2 * r;
    float rowmin = INFINITY;
    if (i >= r && i + r < n && i > 0) {
#pragma unroll
        for (int w = 0; w < KW; ++w) {
            if (w <= wmax) {
                const float c = w >= 1 ? cur[w - 1] : INFINITY;
                const float best = fminf(fminf(prev[w], prev[w + 1]), c);
                const float d = __fsub_rn(qi, xw[w]);
                const float v = __fmaf_rn(d, d, best);
                cur[w] = v;
                if (kMin) rowmin = fminf(rowmin, v);
            }
        }
    } else {
#pragma unroll
        for (int w = 0; w < KW; ++w) {
            if (w <= wmax) {
                const int j = i + w - r;
                float v = INFINITY;
                if (j >= 0 && j < n) {
                    float best;
                    if (i == 0 && j == 0) {
                        best = 0.0f;
                    } else {
                        const float c = w >= 1 ? cur[w - 1] : INFINITY;
                        best = fminf(fminf(prev[w], prev[w + 1]), c);
                    }
                    const float d = __fsub_rn(qi, xw[w]);
                    v = __fmaf_rn(d, d, best);
                }
                cur[w] = v;
                if (kMin) rowmin = fminf(rowmin, v);
            }
        }
    }
    return rowmin;
}

// Slide the band's window of x one column right (the column entering at
// row i + 1 is i + 1 + r).
template <int KW, bool kExact>
__device__ __forceinline__ void dtw_slide(float (&xw)[KW + 1], const float *__restrict__ x, int i, int n, int r) {
    const int wmax = kExact ? KW - 1 : 2 * r;
    const int jn = i + 1 + r;
    const float xn = jn < n ? x[jn] : 0.0f;
#pragma unroll
    for (int w = 0; w < KW; ++w) xw[w] = (w == wmax) ? xn : xw[w + 1];
}

// Float32 DTW of series x against the query in shared memory, two rows in
// registers used in turn (n is a multiple of 16, so rows come in groups of
// four; cells past the band stay +inf), abandoned once the smallest cell of
// the last row of a group exceeds T (every path crosses that row, so D > T):
// returns the distance, and sets `abandoned` if it stopped early.
// kExact: the band fills all KW cells (r = (KW - 1) / 2), so the cell loop
// needs no test of the band's width.
template <int KW, bool kExact>
__device__ __forceinline__ float dtw_band(const float *__restrict__ x, const float *__restrict__ qs, int n,
                                          int r_arg, float T, long long &cells, bool &abandoned) {
    const int r = kExact ? (KW - 1) / 2 : r_arg;
    const int wmax = kExact ? KW - 1 : 2 * r;
    float pa[KW + 1], pb[KW + 1], xw[KW + 1];
#pragma unroll
    for (int w = 0; w <= KW; ++w) {
        pa[w] = INFINITY;
        pb[w] = INFINITY;
        const int j = w - r;                     // the window of row 0
        xw[w] = (w <= wmax && j >= 0 && j < n) ? x[j] : 0.0f;
    }
    for (int i = 0; i < n; i += 4) {
        dtw_row<KW, kExact, false>(i, qs[i], pa, pb, xw, n, r);
        dtw_slide<KW, kExact>(xw, x, i, n, r);
        dtw_row<KW, kExact, false>(i + 1, qs[i + 1], pb, pa, xw, n, r);
        dtw_slide<KW, kExact>(xw, x, i + 1, n, r);
        dtw_row<KW, kExact, false>(i + 2, qs[i + 2], pa, pb, xw, n, r);
        dtw_slide<KW, kExact>(xw, x, i + 2, n, r);
        const float m = dtw_row<KW, kExact, true>(i + 3, qs[i + 3], pb, pa, xw, n, r);
        cells += 4 * (wmax + 1);
        if (m > T) {
            abandoned = true;
            return INFINITY;
        }
        dtw_slide<KW, kExact>(xw, x, i + 3, n, r);
    }
    float d = INFINITY;                        // column n - 1 of row n - 1 (n % 4 == 3): cell r of pa
#pragma unroll
    for (int w = 0; w < KW; ++w)
        if (w == r) d = pa[w];
    return d;
}

constexpr int kDtwWindow = 1024;   // series a block screens before their DTWs

// a5-a6: one (leaf, query) pair per block at a time (persistent grid).  The
// block screens a window of the leaf's series (the word bound, one series
// per thread, then LB_Keogh, one series per warp), queues the survivors in
// shared memory, then its threads take queued series one at a time for the
// DTW with early abandoning, so a thread whose series ended early takes the
// next.
template <int KW>
__global__ void __launch_bounds__(kDtwThreads, 4) k_dtw_scan(DtwScanArgs A) {
    extern __shared__ float sh[];
    const int n = A.n, r = A.r;
    float *qs = sh, *Ls = sh + n, *Us = sh + 2 * n;
    __shared__ float B[kAlpha + 1];
    __shared__ float pl[kWord], pu[kWord];
    __shared__ int64_t s_e;
    __shared__ int s_pn, s_qn, s_take;
    __shared__ int16_t s_pre[kDtwWindow];     // the window's series left by the word bound
    __shared__ int16_t s_queue[kDtwWindow];   // ... and by LB_Keogh: their DTWs to do
    for (int j = threadIdx.x; j <= kAlpha; j += blockDim.x)
        B[j] = j == 0 ? -INFINITY : (j == kAlpha ? INFINITY : A.bp[j - 1]);
    const float w_sax = (float)(n / kWord);
    long long c_cand = 0, c_sax = 0, c_keogh = 0, c_ab = 0, c_full = 0, c_cells = 0;
    const int total = *A.list_cnt;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) s_e = atomicAdd(A.work, 1);
        __syncthreads();
        const int e = (int)s_e;
        if (e >= total) break;
        const int64_t t = A.list[e];
        const int64_t leaf = t / A.nq;
        const int q = (int)(t % A.nq);
        for (int j = threadIdx.x; j < n; j += blockDim.x) {
            qs[j] = A.Q[(int64_t)q * n + j];
            Ls[j] = A.envL[(int64_t)q * n + j];
            Us[j] = A.envU[(int64_t)q * n + j];
        }
        if (threadIdx.x < kWord) {
            pl[threadIdx.x] = A.paa[(int64_t)q * 2 * kWord + threadIdx.x];
            pu[threadIdx.x] = A.paa[(int64_t)q * 2 * kWord + kWord + threadIdx.x];
        }
        __syncthreads();
        const float u = __uint_as_float(A.U[q]);
        const float T = __fmul_ru(u, 1.0f + A.rho);
        const int64_t s0 = A.leaf_off[leaf], s1 = A.leaf_off[leaf + 1];
        for (int64_t w0 = s0; w0 < s1; w0 += kDtwWindow) {
            const int64_t w1 = min(w0 + (int64_t)kDtwWindow, s1);
            if (threadIdx.x == 0) {
                s_pn = 0;
                s_qn = 0;
                s_take = 0;
            }
            __syncthreads();
            // the word bound, one series per thread
            for (int64_t s = w0 + threadIdx.x; s < w1; s += blockDim.x) {
                ++c_cand;
                if (A.use_sax) {
                    const uint4 w4 = *reinterpret_cast<const uint4 *>(A.sax + s * kWord);
                    const uint32_t wv[4] = {w4.x, w4.y, w4.z, w4.w};
                    float acc = 0.0f;
#pragma unroll
                    for (int i = 0; i < kWord; ++i) {
                        const int sym = (wv[i >> 2] >> ((i & 3) * 8)) & 0xff;
                        const float a = __fsub_rd(B[sym], pu[i]);        // cell low end - PAA(U)
                        const float b = __fsub_rd(pl[i], B[sym + 1]);    // PAA(L) - cell high end
                        const float g = fmaxf(fmaxf(a, b), 0.0f);
                        acc = __fmaf_rd(g, g, acc);
                    }
                    if (__fmul_rd(acc, w_sax) > u) {
                        ++c_sax;
                        continue;
                    }
                }
                s_pre[atomicAdd(&s_pn, 1)] = (int16_t)(s - w0);
            }
            __syncthreads();
            // LB_Keogh from the raw points, one series per warp (lane l takes
            // points 4l.., 4l+128.., so a row is read in coalesced 512-byte
            // pieces); every partial sum rounded down, so the total stays
            // below the exact bound
            {
                const int pn = s_pn, lane = threadIdx.x & 31;
                const float4 *L4 = reinterpret_cast<const float4 *>(Ls);
                const float4 *U4 = reinterpret_cast<const float4 *>(Us);
                for (int i = threadIdx.x >> 5; i < pn; i += kDtwThreads / 32) {
                    const int off = s_pre[i];
                    const float4 *x4 = reinterpret_cast<const float4 *>(A.X + (w0 + off) * n);
                    float part = 0.0f;
                    for (int f = lane; f < (n >> 2); f += 32) {
                        const float4 xv = x4[f], lv = L4[f], uv = U4[f];
                        float g;
                        g = fmaxf(fmaxf(__fsub_rd(lv.x, xv.x), __fsub_rd(xv.x, uv.x)), 0.0f);
                        part = __fmaf_rd(g, g, part);
                        g = fmaxf(fmaxf(__fsub_rd(lv.y, xv.y), __fsub_rd(xv.y, uv.y)), 0.0f);
                        part = __fmaf_rd(g, g, part);
                        g = fmaxf(fmaxf(__fsub_rd(lv.z, xv.z), __fsub_rd(xv.z, uv.z)), 0.0f);
                        part = __fmaf_rd(g, g, part);
                        g = fmaxf(fmaxf(__fsub_rd(lv.w, xv.w), __fsub_rd(xv.w, uv.w)), 0.0f);
                        part = __fmaf_rd(g, g, part);
                    }
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) part = __fadd_rd(part, __shfl_xor_sync(0xffffffffu, part, o));
                    if (lane == 0) {
                        if (part > u) ++c_keogh;
                        else s_queue[atomicAdd(&s_qn, 1)] = (int16_t)off;
                    }
                }
            }
            __syncthreads();
            const int qn = s_qn;
            for (;;) {
                const int idx = atomicAdd(&s_take, 1);
                if (idx >= qn) break;
                const int64_t s = w0 + s_queue[idx];
                bool abandoned = false;
                const float d = 2 * r + 1 == KW ? dtw_band<KW, true>(A.X + s * n, qs, n, r, T, c_cells, abandoned)
                                                : dtw_band<KW, false>(A.X + s * n, qs, n, r, T, c_cells, abandoned);
                if (abandoned) {
                    ++c_ab;
                    continue;
                }
                ++c_full;
                if (!(d <= T)) continue;
                const int slot = atomicAdd(&A.pool_cnt[q], 1);
                if (slot < A.pool_C) {
                    A.pool_d[(int64_t)q * A.pool_C + slot] = d;
                    A.pool_p[(int64_t)q * A.pool_C + slot] = (int32_t)s;
                } else {
                    atomicOr(&A.qflag[q], 1);
                }
            }
            __syncthreads();
        }
    }
    c_cand = warp_sum_ll(c_cand);
    c_sax = warp_sum_ll(c_sax);
    c_keogh = warp_sum_ll(c_keogh);
    c_ab = warp_sum_ll(c_ab);
    c_full = warp_sum_ll(c_full);
    c_cells = warp_sum_ll(c_cells);
    if ((threadIdx.x & 31) == 0) {
        stat_add(&A.st[DS_SERIES_CAND], c_cand);
        stat_add(&A.st[DS_SAX_PRUNED], c_sax);
        stat_add(&A.st[DS_KEOGH_PRUNED], c_keogh);
        stat_add(&A.st[DS_ABANDONED], c_ab);
        stat_add(&A.st[DS_FULL], c_full);
        stat_add(&A.st[DS_CELLS], c_cells);
    }
}

// U[q] = (1 + rho) x the k-th smallest pooled float32 distance (block per
// query, k passes of a block-wide minimum over the distinct values).
__global__ void k_dtw_kth(const float *__restrict__ pool_d, const int32_t *__restrict__ pool_cnt, int C, int k,
                          float rho, uint32_t *__restrict__ U) {
    __shared__ int rc[32];
    __shared__ float s_v;
    const int q = blockIdx.x, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int cnt = min(pool_cnt[q], C);
    if (cnt < k) return;
    const float *d = pool_d + (int64_t)q * C;
    // the k-th smallest: the smallest v with #{d <= v} >= k, found by
    // bisection over the float bit patterns (non-negative floats order as
    // their bits)
    uint32_t lo = 0, hi = 0x7f800000u;
    while (lo < hi) {
        const uint32_t mid = lo + (hi - lo) / 2;
        const float mv = __uint_as_float(mid);
        int c = 0;
        for (int i = threadIdx.x; i < cnt; i += blockDim.x) c += d[i] <= mv;
        c = warp_sum_i(c);
        if (lane == 0) rc[warp] = c;
        __syncthreads();
        if (threadIdx.x == 0) {
            int tot = 0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot += rc[w];
            s_v = tot >= k ? 1.0f : 0.0f;
        }
        __syncthreads();
        if (s_v != 0.0f) hi = mid; else lo = mid + 1;
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const float kth = __uint_as_float(lo);
        atomicMin(&U[q], __float_as_uint(__fmul_ru(kth, 1.0f + rho)));
    }
}

// Binary64 DTW in the oracle's operation order.
__device__ double dtw64(const float *__restrict__ q, const float *__restrict__ x, int n, int r) {
    double prev[kW], cur[kW];
#pragma unroll
    for (int w = 0; w < kW; ++w) {
        prev[w] = INFINITY;
        cur[w] = INFINITY;
    }
    for (int i = 0; i < n; ++i) {
        const double qi = (double)q[i];
#pragma unroll
        for (int w = 0; w < kW; ++w) {
            if (w > 2 * r) break;
            const int j = i + w - r;
            double v = INFINITY;
            if (j >= 0 && j < n) {
                double best;
                if (i == 0 && j == 0) {
                    best = 0.0;
                } else {
                    const double a = prev[w];
                    const double b = (w + 1 <= 2 * r) ? prev[w + 1] : INFINITY;
                    const double c = (w >= 1) ? cur[w - 1] : INFINITY;
                    best = a < b ? a : b;
                    best = c < best ? c : best;
                }
                const double d = __dsub_rn(qi, (double)x[j]);
                v = __dadd_rn(__dmul_rn(d, d), best);
            }
            cur[w] = v;
        }
#pragma unroll
        for (int w = 0; w < kW; ++w) prev[w] = cur[w];
    }
    double out = INFINITY;
#pragma unroll
    for (int w = 0; w < kW; ++w)
        if (w == r) out = prev[w];
    return out;
}

// a8: binary64 rescore of the pooled series at or below T(U), top-k by
// (D, id).  Block per query.
__global__ void k_dtw_final(const float *__restrict__ Q, const float *__restrict__ X, int n, int r,
                            const int64_t *__restrict__ perm, const float *__restrict__ pool_d,
                            const int32_t *__restrict__ pool_p, const int32_t *__restrict__ pool_cnt, int C,
                            const uint32_t *__restrict__ U, const int32_t *__restrict__ qflag, int k, float rho,
                            double *__restrict__ rs, int64_t *__restrict__ out_ids, float *__restrict__ out_dist,
                            long long *__restrict__ st, int32_t *__restrict__ err) {
    __shared__ double sv[kDtwFinalCap];
    __shared__ long long sid[kDtwFinalCap];
    __shared__ int ns;
    __shared__ double bd[32];
    __shared__ long long bi[32];
    __shared__ int be[32];
    const int q = blockIdx.x;
    if (qflag[q] & 1) return;
    if (threadIdx.x == 0) ns = 0;
    __syncthreads();
    const int cnt = min(pool_cnt[q], C);
    const float T = __fmul_ru(__uint_as_float(U[q]), 1.0f + rho);
    const float *pd = pool_d + (int64_t)q * C;
    const int32_t *pp = pool_p + (int64_t)q * C;
    const float *qr = Q + (int64_t)q * n;
    for (int i = threadIdx.x; i < cnt; i += blockDim.x)
        if (pd[i] <= T) {
            const int e = atomicAdd(&ns, 1);
            if (e < kDtwFinalCap) sid[e] = i;
        }
    __syncthreads();
    const int m = ns;
    if (threadIdx.x == 0 && m) stat_add(&st[DS_RESCORED], m);
    if (m <= kDtwFinalCap) {
        for (int e = threadIdx.x; e < m; e += blockDim.x) {
            const int64_t pos = pp[sid[e]];
            sv[e] = dtw64(qr, X + pos * n, n, r);
            sid[e] = perm[pos];
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
    // more candidates than the shared arrays hold: k block-wide minima
    double *rr = rs + (int64_t)q * C;
    for (int i = threadIdx.x; i < cnt; i += blockDim.x)
        rr[i] = pd[i] <= T ? dtw64(qr, X + (int64_t)pp[i] * n, n, r) : INFINITY;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int t = 0; t < k; ++t) {
        double b = INFINITY;
        long long id = -1;
        int e = -1;
        for (int i = threadIdx.x; i < cnt; i += blockDim.x) {
            const double v = rr[i];
            if (v == INFINITY) continue;
            const long long pid = perm[pp[i]];
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
                rr[ee] = INFINITY;
            }
        }
        __syncthreads();
    }
}

__global__ void k_dtw_fill(uint32_t *p, int n, uint32_t v) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) p[i] = v;
}

// Flagged (overflowed) queries: empty their pools for the rerun, mark them.
__global__ void k_dtw_rearm(int32_t *__restrict__ qflag, int32_t *__restrict__ pool_cnt, uint8_t *__restrict__ sel,
                            int nq) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nq) return;
    const bool f = qflag[q] & 1;
    sel[q] = f ? 1 : 0;
    if (f) {
        pool_cnt[q] = 0;
        qflag[q] = 0;
    }
}

float rho_dtw(int n) {
    const double u = std::ldexp(1.0, -24);
    const double m = (double)(2 * n + 4) * u;
    return (float)(m / (1.0 - m) * 1.0001 + std::ldexp(1.0, -40));
}

}  // namespace

void run_query_dtw(hk_index *idx, const float *Qd, int nq, int k, int band, const hk_query_opts &o,
                   cudaStream_t s, int64_t *out_ids, float *out_dist, hk_query_stats *stats) {
    const long long launches0 = g_launches;
    const int n = idx->n;
    const int64_t L = idx->L;
    const int r = band;
    const float rho = rho_dtw(n);
    const int l_max = o.l_max > 0 ? o.l_max : kDefaultLMax;
    const bool use_sax = (o.flags & HK_Q_NOSAX) == 0;
    // a pool holds every series of the approximate leaves (scanned with no
    // bound), so at least twice the leaf capacity
    const int C = std::min(1 << 21, std::max({65536, 4096 * k, 2 * idx->tau}));
    DtwWork &w = idx->dtw;
    w.envL.reserve((size_t)nq * n, s);
    w.envU.reserve((size_t)nq * n, s);
    w.qseg.reserve((size_t)nq * idx->S * 2, s);
    w.paa.reserve((size_t)nq * 2 * kWord, s);
    w.lb.reserve((size_t)nq * L, s);
    w.mask.reserve((size_t)nq * L, s);
    w.list.reserve((size_t)nq * L, s);
    w.U.reserve(nq, s);
    w.pool_d.reserve((size_t)nq * C, s);
    w.pool_p.reserve((size_t)nq * C, s);
    w.pool_cnt.reserve(nq, s);
    w.qflag.reserve(nq, s);
    w.sel.reserve(nq, s);
    w.ctr.reserve(4, s);
    w.stats.reserve(DS_COUNT, s);
    w.out_ids.reserve((size_t)nq * k, s);
    w.out_dist.reserve((size_t)nq * k, s);
    HK_CHECK_CUDA(cudaMemsetAsync(w.mask.p, 0, (size_t)nq * L, s));
    HK_CHECK_CUDA(cudaMemsetAsync(w.pool_cnt.p, 0, nq * sizeof(int32_t), s));
    HK_CHECK_CUDA(cudaMemsetAsync(w.qflag.p, 0, nq * sizeof(int32_t), s));
    HK_CHECK_CUDA(cudaMemsetAsync(w.stats.p, 0, DS_COUNT * sizeof(long long), s));
    k_dtw_fill<<<(nq + 255) / 256, 256, 0, s>>>(w.U.p, nq, 0x7f800000u);
    HK_CHECK_LAUNCH();
    k_dtw_prep<<<nq, 128, 3 * n * sizeof(float), s>>>(Qd, n, r, idx->seg_ab.p, idx->S, w.envL.p, w.envU.p,
                                                     w.qseg.p, w.paa.p);
    HK_CHECK_LAUNCH();
    k_dtw_lb_leaf<<<dim3((unsigned)((L + 127) / 128), std::min(nq, 65535)), 128, 0, s>>>(
        w.qseg.p, idx->S, idx->leaf_nseg.p, idx->leaf_seg.p, idx->seg_ab.p, idx->env.p, L, nq, w.lb.p);
    HK_CHECK_LAUNCH();
    k_dtw_approx<<<nq, 256, 0, s>>>(w.lb.p, L, idx->leaf_off.p, l_max, k, nq, w.mask.p, w.stats.p);
    HK_CHECK_LAUNCH();

    int sms = 0, dev = 0;
    HK_CHECK_CUDA(cudaGetDevice(&dev));
    HK_CHECK_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int64_t pairs = L * (int64_t)nq;
    const size_t smem = 3 * (size_t)n * sizeof(float);
    auto scan = [&](uint8_t vlo, uint8_t vhi, const uint8_t *sel, int sax) {
        HK_CHECK_CUDA(cudaMemsetAsync(w.ctr.p, 0, 4 * sizeof(int32_t), s));
        k_dtw_list<<<(unsigned)((pairs + 255) / 256), 256, 0, s>>>(w.mask.p, L, nq, vlo, vhi, sel, w.list.p,
                                                                   w.ctr.p);
        HK_CHECK_LAUNCH();
        DtwScanArgs a{};
        a.X = idx->X.p;
        a.sax = idx->sax.p;
        a.bp = idx->bp.p;
        a.leaf_off = idx->leaf_off.p;
        a.n = n;
        a.r = r;
        a.nq = nq;
        a.Q = Qd;
        a.envL = w.envL.p;
        a.envU = w.envU.p;
        a.paa = w.paa.p;
        a.U = w.U.p;
        a.rho = rho;
        a.use_sax = sax;
        a.list = w.list.p;
        a.list_cnt = w.ctr.p;
        a.work = w.ctr.p + 1;
        a.pool_d = w.pool_d.p;
        a.pool_p = w.pool_p.p;
        a.pool_cnt = w.pool_cnt.p;
        a.pool_C = C;
        a.qflag = w.qflag.p;
        a.st = w.stats.p;
        // band cells rounded up to a compiled width
        if (r <= 4)
            k_dtw_scan<9><<<sms * 8, kDtwThreads, smem, s>>>(a);
        else if (r <= 8)
            k_dtw_scan<17><<<sms * 8, kDtwThreads, smem, s>>>(a);
        else if (r <= 12)
            k_dtw_scan<25><<<sms * 8, kDtwThreads, smem, s>>>(a);
        else
            k_dtw_scan<kW><<<sms * 8, kDtwThreads, smem, s>>>(a);
        HK_CHECK_LAUNCH();
        k_dtw_kth<<<nq, 256, 0, s>>>(w.pool_d.p, w.pool_cnt.p, C, k, rho, w.U.p);
        HK_CHECK_LAUNCH();
    };
    // a3: the approximate leaves whole (U = +inf: no pruning), then U
    scan(1, 1, nullptr, 0);
    // a4-a7: candidate leaves against U
    k_dtw_mask<<<(unsigned)((pairs + 255) / 256), 256, 0, s>>>(w.lb.p, L, nq, w.U.p, w.mask.p, w.stats.p);
    HK_CHECK_LAUNCH();
    scan(2, 2, nullptr, use_sax ? 1 : 0);
    // pools that overflowed: those queries again, every leaf they scanned,
    // from the bound their pools now give (tighter after each round)
    long long retried = 0;
    std::vector<int32_t> flags(nq);
    std::vector<uint32_t> Ub(nq), Ub_prev(nq, 0xffffffffu);
    for (int round = 0;; ++round) {
        HK_CHECK_CUDA(cudaMemcpyAsync(flags.data(), w.qflag.p, nq * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        HK_CHECK_CUDA(cudaMemcpyAsync(Ub.data(), w.U.p, nq * sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
        HK_CHECK_CUDA(cudaStreamSynchronize(s));
        int nf = 0;
        for (int q = 0; q < nq; ++q) {
            if (!(flags[q] & 1)) continue;
            ++nf;
            if (round > 0 && Ub[q] >= Ub_prev[q])
                fail(HK_ENOMEM, "DTW query %d: more than %d series within the bound of its k-th distance", q, C);
        }
        if (!nf) break;
        retried += nf;
        Ub_prev = Ub;
        k_dtw_rearm<<<(nq + 255) / 256, 256, 0, s>>>(w.qflag.p, w.pool_cnt.p, w.sel.p, nq);
        HK_CHECK_LAUNCH();
        scan(1, 2, w.sel.p, use_sax ? 1 : 0);
    }
    // a8
    w.rs.reserve((size_t)nq * C, s);
    HK_CHECK_CUDA(cudaMemsetAsync(w.ctr.p + 2, 0, sizeof(int32_t), s));
    k_dtw_final<<<nq, 256, 0, s>>>(Qd, idx->X.p, n, r, idx->perm.p, w.pool_d.p, w.pool_p.p, w.pool_cnt.p, C, w.U.p,
                                   w.qflag.p, k, rho, w.rs.p, w.out_ids.p, w.out_dist.p, w.stats.p, w.ctr.p + 2);
    HK_CHECK_LAUNCH();
    int32_t err = 0;
    HK_CHECK_CUDA(cudaMemcpyAsync(&err, w.ctr.p + 2, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    const bool ids_dev = is_device_ptr(out_ids), dist_dev = is_device_ptr(out_dist);
    HK_CHECK_CUDA(cudaMemcpyAsync(out_ids, w.out_ids.p, (size_t)nq * k * sizeof(int64_t),
                                  ids_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
    HK_CHECK_CUDA(cudaMemcpyAsync(out_dist, w.out_dist.p, (size_t)nq * k * sizeof(float),
                                  dist_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
    long long st[DS_COUNT];
    HK_CHECK_CUDA(cudaMemcpyAsync(st, w.stats.p, sizeof(st), cudaMemcpyDeviceToHost, s));
    HK_CHECK_CUDA(cudaStreamSynchronize(s));
    if (err) fail(HK_EINTERNAL, "DTW: a query had fewer than k candidates");
    if (stats) {
        std::memset(stats, 0, sizeof(*stats));
        stats->queries = nq;
        stats->leaves_total = (long long)nq * L;
        stats->leaves_approx = st[DS_LEAVES_APPROX];
        stats->leaves_candidate = st[DS_LEAVES_CAND];
        stats->series_candidate = st[DS_SERIES_CAND];
        stats->series_sax_pruned = st[DS_SAX_PRUNED];
        stats->series_abandoned = st[DS_KEOGH_PRUNED] + st[DS_ABANDONED];
        stats->series_full = st[DS_FULL];
        stats->points_computed = st[DS_CELLS];
        stats->rescored = st[DS_RESCORED];
        stats->retried_queries = retried;
        stats->lb_evaluations = (long long)nq * L;
        stats->kernel_launches = g_launches - launches0;
    }
}

}  // namespace hk
