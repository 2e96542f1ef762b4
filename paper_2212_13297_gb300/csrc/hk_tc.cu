// Precision form: squared distances on the tcgen05 tensor cores.
//
// The 16-bit copy is bfloat16 (the default) or float16 (HK_BUILD_FP16: three
// more bits of precision for collections inside float16's range).
//
// For a block of up to 128 queries and a run of series, D~(q,x) =
// |q|^2 + |x|^2 - 2 q^.x^ with the dot products of the 16-bit roundings q^,
// x^ accumulated in float32 in tensor memory.  Each D~ carries a
// certified error bound E(q,x) = A_q |x| + B (|q|^2 + |x|^2):
//   |q^.x^ - q.x| <= (2u + u^2 + g(1+u)^2) |q||x| + (subnormal term),
//   u = 2^-8 (bfloat16) or 2^-11 (float16),
//   g = n w / (1 - n w), w = 2^-20,
// doubled for the -2 factor, plus a relative term covering the float32
// rounding of the norms and of the epilogue arithmetic.
//
// Where g comes from.  Fasi, Higham, Mikaitis and Pranesh ("Numerical
// behavior of NVIDIA tensor cores", PeerJ Computer Science 7:e330, 2021)
// measured that tensor cores of earlier generations (V100, T4, A100) form
// d = c + sum_{i<m} a_i b_i for a block of m products as follows: products
// exact; the m + 1 addends aligned to the largest, with the bits below that
// addend's 24-bit significand truncated; the aligned addends summed exactly;
// the sum normalised to float32 by truncation.  The block size m and the
// number of bits kept varied by generation; no published study covers
// tcgen05.  The bound assumes the same family for any m >= 1 and at least
// 24 kept bits.  Then one block step errs by less than (m+1) 2^-23 M for the
// alignment plus 2^-23 |d| for the normalisation, where M is the largest
// addend; both are at most P = sum |a_i b_i| over the whole dot product
// (the accumulator holds a partial sum, itself bounded by P up to these
// errors).  Over n/m steps the error is below (n/m)(m+2) 2^-23 P <=
// 3 n 2^-23 P (worst at m = 1), and P <= |q^||x^| <= (1+u)^2 |q||x| by
// Cauchy-Schwarz.  g >= n 2^-20 covers 3 n 2^-23 with a factor 8/3; it
// still covers the case of only 22 kept bits when m >= 2.  The per-pair
// bound is checked against binary64 distances on benign and adversarial
// inputs (cancellation, alternating signs, values near the format's largest,
// wide exponent ranges, the float16 subnormal range, n = 16 ... 256).  A series stays a
// candidate of a query while D~ - E <= U (U bounds the query's true k-th
// distance); D~ + E of k series bounds it from above, so each query's row
// keeps its k smallest D~ + E and tightens U with them.  Candidates are
// rescored exactly afterwards, so the answer stays exact.
//
// Data layout.  The 16-bit copy of the collection is stored in the
// tensor core's no-swizzle K-major "core matrix" order: series are grouped
// by 8 (leaf order); a group is n/8 blocks of 8 series x 8 points (128 bytes),
// block k holding points 8k..8k+7.  A tile of 128 consecutive series (16
// groups, 8-aligned) is then one contiguous run of 128*n*2 bytes that a
// single bulk copy (cp.async.bulk) places in shared memory in exactly the
// layout the MMA descriptor describes: leading-dimension offset 128 bytes
// (next 8 points), stride-dimension offset (n/8)*128 bytes (next 8 series).
// The query block lives in tensor memory (row i in lane i, two 16-bit
// points per 32-bit column), so each MMA reads only the series tile from
// shared memory.
//
// CTA roles (10 warps): warp 0 claims work items (a 32-way search over the
// item offsets) and, from one thread, issues the bulk copies (a whole series
// tile and its norm pairs per stage); warp 1 (one thread) issues tcgen05.mma
// and tcgen05.commit; warps 2-9 write the query block into tensor memory at
// the start of each item, then read the accumulators with tcgen05.ld and
// filter: warp w reads TMEM lane quarter w%4 (query rows 32(w%4)..+31) and
// half of the tile's columns.  Per element the filter is two FMAs and a
// minimum; the per-column test and the exact bounds are formed only when a
// minimum reaches the row's threshold.
// Three shared-memory stages for series tiles, three TMEM accumulators.  Every
// mbarrier wait is bounded; on a timeout the CTA raises an error flag,
// drains, frees its tensor memory and stops.
//
// Served form (k_tc_serve): the same roles and pipeline in a resident launch
// that takes its items from the scans (jobs) of many batches published to a
// device-resident ring while it runs, each item with its own job's arguments;
// the host side (TcEngine, at the end of this file) publishes jobs and waits
// for their completion flags in host-mapped memory.
#include <cuda_bf16.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "hk_device.cuh"
#include "hk_internal.cuh"

namespace hk {
namespace {

constexpr int kTcM = 128;        // queries per block (MMA M)
constexpr int kTcN = 128;        // series per tile (MMA N)
// Series tiles (128 series, 16 groups of 8: one contiguous run in the
// core-matrix layout) stream through kTcStages shared-memory stages, one
// bulk copy each.
constexpr int kTcStages = 3;
constexpr int kTcStageBytes = kTcN * 256 * 2;   // longest series (256 points)
// Norm slots: tile g uses slot g % 8.  The producer writes tile g's norms
// after the MMA finished tile g - kTcStages, which it issued after the
// epilogue released the accumulator of tile g - kTcStages - kAcc.  The
// epilogue releases a tile's accumulator once it is in registers, before
// reading that tile's norms, but only after it finished every earlier tile:
// tile g - kTcStages - kAcc - 1 = g-7 and so g-8 (the slot's previous user)
// were read before.
constexpr int kNormSlots = 8;
constexpr int kTcEpiWarps = 8;   // two per TMEM lane quarter, each half the columns
constexpr int kTcEpiThreads = 32 * kTcEpiWarps;
constexpr int kEpiChunks = kTcN / 32 / (kTcEpiWarps / 4);   // 32-column chunks per epilogue warp
constexpr int kTcThreads = 32 * (2 + kTcEpiWarps);
constexpr int kAcc = 3;          // accumulators in tensor memory
constexpr int kTmemCols = 512;   // kAcc accumulators of kTcN columns, then the query block
constexpr int kTmemA = kAcc * kTcN; // first column of the query block (n/2 <= 128 columns)
static_assert(kTmemA + 128 <= kTmemCols, "tensor memory overflow");
static_assert(kNormSlots >= kTcStages + kAcc + 1, "norm slot reuse distance");
constexpr uint64_t kWaitNs = 2000000000ull;   // 2 s: far above any legitimate wait
constexpr uint64_t kDrainNs = 200000000ull;   // 200 ms for copies / MMAs in flight to land
constexpr int kLocalK = kTcLocalK;   // k-best upper bounds kept per epilogue thread
constexpr double kTcEb = 0x1p-19;   // relative term for norm and epilogue rounding
constexpr float kF16Max = 65504.0f;      // largest finite float16: the float16 copy's range

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}
// Bounded wait for the phase with the given parity to complete: gives up
// after limit_ns of wall time or when the CTA is aborting (then returns
// false; on its own timeout it sets the abort flag).
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, volatile int *abort_flag,
                                          uint64_t limit_ns) {
    if (mbar_try(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    for (uint32_t it = 1;; ++it) {
        if (mbar_try(bar, parity)) return true;
        if (*abort_flag) return false;
        if ((it & 255) == 0 && global_ns() - t0 > limit_ns) {
            *abort_flag = 1;
            return false;
        }
    }
}
// Wait for a phase without regard to the abort flag, until a deadline of
// %globaltimer (the drain of an aborting CTA); false if the deadline passed.
__device__ __forceinline__ bool mbar_wait_until(uint64_t *bar, uint32_t parity, uint64_t deadline) {
    for (uint32_t it = 0;; ++it) {
        if (mbar_try(bar, parity)) return true;
        if ((it & 255) == 255 && global_ns() > deadline) return false;
    }
}
// The same, decided once for a whole warp (every lane polls, all agree).
__device__ __forceinline__ bool mbar_wait_warp(uint64_t *bar, uint32_t parity, volatile int *abort_flag,
                                               uint64_t limit_ns) {
    const uint64_t t0 = global_ns();
    for (uint32_t it = 0;; ++it) {
        const bool ok = mbar_try(bar, parity);
        if (__all_sync(0xffffffffu, ok)) return true;
        const bool stop = *abort_flag != 0;
        if (__any_sync(0xffffffffu, stop)) return false;
        if ((it & 255) == 255) {
            const bool late = global_ns() - t0 > limit_ns;
            if (__any_sync(0xffffffffu, late)) {
                *abort_flag = 1;
                return false;
            }
        }
    }
}
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
// Shared memory matrix descriptor: no swizzle, K-major.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;   // descriptor version for tcgen05
    return d;                 // base offset 0, swizzle none
}
// D (tensor memory) += A (tensor memory) * B (shared memory descriptor)^T
__device__ __forceinline__ void mma_ts(uint32_t d_tmem, uint32_t a_tmem, uint64_t b, uint32_t idesc,
                                       uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n\t}" ::"r"(d_tmem),
        "r"(a_tmem), "l"(b), "r"(idesc), "r"(accumulate)
        : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_u32(bar))
                 : "memory");
}
// Issue one 64-column TMEM load (lanes of this warp's quarter; columns in
// register order, 32 per row of r); the values are valid only after
// tmem_wait_ld().
__device__ __forceinline__ void tmem_ld64_issue(uint32_t taddr, uint32_t (&r)[2][32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x64.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,"
        "%32,%33,%34,%35,%36,%37,%38,%39,%40,%41,%42,%43,%44,%45,%46,%47,"
        "%48,%49,%50,%51,%52,%53,%54,%55,%56,%57,%58,%59,%60,%61,%62,%63}, [%64];"
        : "=r"(r[0][0]), "=r"(r[0][1]), "=r"(r[0][2]), "=r"(r[0][3]), "=r"(r[0][4]), "=r"(r[0][5]), "=r"(r[0][6]),
          "=r"(r[0][7]), "=r"(r[0][8]), "=r"(r[0][9]), "=r"(r[0][10]), "=r"(r[0][11]), "=r"(r[0][12]), "=r"(r[0][13]),
          "=r"(r[0][14]), "=r"(r[0][15]), "=r"(r[0][16]), "=r"(r[0][17]), "=r"(r[0][18]), "=r"(r[0][19]),
          "=r"(r[0][20]), "=r"(r[0][21]), "=r"(r[0][22]), "=r"(r[0][23]), "=r"(r[0][24]), "=r"(r[0][25]),
          "=r"(r[0][26]), "=r"(r[0][27]), "=r"(r[0][28]), "=r"(r[0][29]), "=r"(r[0][30]), "=r"(r[0][31]),
          "=r"(r[1][0]), "=r"(r[1][1]), "=r"(r[1][2]), "=r"(r[1][3]), "=r"(r[1][4]), "=r"(r[1][5]), "=r"(r[1][6]),
          "=r"(r[1][7]), "=r"(r[1][8]), "=r"(r[1][9]), "=r"(r[1][10]), "=r"(r[1][11]), "=r"(r[1][12]), "=r"(r[1][13]),
          "=r"(r[1][14]), "=r"(r[1][15]), "=r"(r[1][16]), "=r"(r[1][17]), "=r"(r[1][18]), "=r"(r[1][19]),
          "=r"(r[1][20]), "=r"(r[1][21]), "=r"(r[1][22]), "=r"(r[1][23]), "=r"(r[1][24]), "=r"(r[1][25]),
          "=r"(r[1][26]), "=r"(r[1][27]), "=r"(r[1][28]), "=r"(r[1][29]), "=r"(r[1][30]), "=r"(r[1][31])
        : "r"(taddr));
}
__device__ __forceinline__ void tmem_st32(uint32_t taddr, const uint32_t (&r)[32]) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], "
        "{%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,"
        "%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32};" ::"r"(taddr),
        "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]),
        "r"(r[8]), "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15]),
        "r"(r[16]), "r"(r[17]), "r"(r[18]), "r"(r[19]), "r"(r[20]), "r"(r[21]), "r"(r[22]),
        "r"(r[23]), "r"(r[24]), "r"(r[25]), "r"(r[26]), "r"(r[27]), "r"(r[28]), "r"(r[29]),
        "r"(r[30]), "r"(r[31])
        : "memory");
}
__device__ __forceinline__ void tmem_wait_st() {
    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_wait_ld() {
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// One work item: series [s0, s1) of a leaf against a block of up to 128 of
// the leaf's queries; tiles of 128 series start at base (8-aligned).
struct TcItem {
    int64_t it;            // item number; >= the item count: no more work
    int64_t s0, s1, base;
    int tiles, gq;
    int qid[kTcM];         // query ids of the block's rows, -1 past gq
};

struct TcShared {
    uint64_t full[kTcStages];
    uint64_t empty[kTcStages];
    uint64_t acc_full[kAcc];
    uint64_t acc_empty[kAcc];
    uint64_t never;        // test hook (dbg_stall): a barrier nothing arrives at
    uint32_t tmem_base;
    int abort_flag;
    TcItem item;
};

// Claim the next work item and describe it in D (one warp).  The leaf is
// the last l with item_off[l] <= it, found by a 32-way search (three rounds
// of one coalesced probe each for ~2,000 leaves).
__device__ void fetch_item(const TcArgs &A, int64_t total, TcItem &D, int lane) {
    int64_t it = 0;
    if (lane == 0) it = atomicAdd(A.work_ctr, 1);
    it = __shfl_sync(0xffffffffu, it, 0);
    if (lane == 0) D.it = it;
    if (it >= total) {
        __syncwarp();
        return;
    }
    int lo = 0, hi = (int)A.L;   // item_off[lo] <= it < item_off[hi + 1]
    while (hi - lo > 31) {
        const int64_t span = hi - lo;
        const int pos = lo + (int)(span * (lane + 1) / 32);
        const unsigned m = __ballot_sync(0xffffffffu, A.item_off[pos] <= it);
        const int last = m ? 31 - __clz((int)m) : -1;
        const int nlo = last >= 0 ? lo + (int)(span * (last + 1) / 32) : lo;
        const int nhi = last < 31 ? lo + (int)(span * (last + 2) / 32) - 1 : hi;
        lo = nlo;
        hi = nhi;
    }
    {
        const int pos = lo + lane;
        const unsigned m = __ballot_sync(0xffffffffu, pos <= hi && A.item_off[pos] <= it);
        lo += 31 - __clz((int)m);
    }
    const int leaf = lo;
    const int64_t local = it - A.item_off[leaf];
    const int qoff = A.leaf_qoff[leaf];
    const int nql = A.leaf_qoff[leaf + 1] - qoff;
    const int ngroups = (nql + kTcM - 1) / kTcM;
    const int64_t tile = local / ngroups;
    const int grp = (int)(local % ngroups);
    const int gq = min(kTcM, nql - grp * kTcM);
    if (lane == 0) {
        const int64_t lo_s = A.leaf_off[leaf], hi_s = A.leaf_off[leaf + 1];
        D.s0 = lo_s + tile * A.S_T;
        D.s1 = min(D.s0 + (int64_t)A.S_T, hi_s);
        D.base = D.s0 & ~(int64_t)7;
        D.tiles = (int)((D.s1 - D.base + kTcN - 1) / kTcN);
        D.gq = gq;
    }
    const int32_t *lq = A.leaf_q + qoff + grp * kTcM;
    for (int g = lane; g < kTcM; g += 32) D.qid[g] = g < gq ? lq[g] : -1;
    __syncwarp();
}


// Shared state of the served kernel: the batch kernel's, plus its current job.
struct TcServeShared : TcShared {
    TcArgs job_args;
    int64_t job_total;
    int job_slot;
    uint32_t job_seq;
    int quit;
};

// Describe work item `it` in D (one warp).  The leaf is the last l with
// item_off[l] <= it, found by a 32-way search (three rounds of one coalesced
// probe each for ~2,000 leaves).
__device__ void describe_item(const TcArgs &A, int64_t it, TcItem &D, int lane) {
    if (lane == 0) D.it = it;
    int lo = 0, hi = (int)A.L;   // item_off[lo] <= it < item_off[hi + 1]
    while (hi - lo > 31) {
        const int64_t span = hi - lo;
        const int pos = lo + (int)(span * (lane + 1) / 32);
        const unsigned m = __ballot_sync(0xffffffffu, A.item_off[pos] <= it);
        const int last = m ? 31 - __clz((int)m) : -1;
        const int nlo = last >= 0 ? lo + (int)(span * (last + 1) / 32) : lo;
        const int nhi = last < 31 ? lo + (int)(span * (last + 2) / 32) - 1 : hi;
        lo = nlo;
        hi = nhi;
    }
    {
        const int pos = lo + lane;
        const unsigned m = __ballot_sync(0xffffffffu, pos <= hi && A.item_off[pos] <= it);
        lo += 31 - __clz((int)m);
    }
    const int leaf = lo;
    const int64_t local = it - A.item_off[leaf];
    const int qoff = A.leaf_qoff[leaf];
    const int nql = A.leaf_qoff[leaf + 1] - qoff;
    const int ngroups = (nql + kTcM - 1) / kTcM;
    const int64_t tile = local / ngroups;
    const int grp = (int)(local % ngroups);
    const int gq = min(kTcM, nql - grp * kTcM);
    if (lane == 0) {
        const int64_t lo_s = A.leaf_off[leaf], hi_s = A.leaf_off[leaf + 1];
        D.s0 = lo_s + tile * A.S_T;
        D.s1 = min(D.s0 + (int64_t)A.S_T, hi_s);
        D.base = D.s0 & ~(int64_t)7;
        D.tiles = (int)((D.s1 - D.base + kTcN - 1) / kTcN);
        D.gq = gq;
    }
    const int32_t *lq = A.leaf_q + qoff + grp * kTcM;
    for (int g = lane; g < kTcM; g += 32) D.qid[g] = g < gq ? lq[g] : -1;
    __syncwarp();
}

// Served form (one warp): claim the next item of the oldest published job
// that has items left -- in lane 0 (approximate steps, short and on every
// batch's critical path) before lane 1 -- copy that job's arguments into
// shared memory and describe the item.  A claim is one compare-and-swap on
// the lane's word (job sequence, next item), so an item is claimed once, and
// only while its job is the lane's current one (a ring slot is rewritten only
// after its job completed).  Sets S.quit when no job came for V.idle_ns.
__device__ void serve_fetch(const TcServe &V, TcServeShared &S, int lane) {
    int slot = -1;
    long long item = 0;
    uint32_t seq = 0;
    if (lane == 0) {
        uint64_t idle0 = 0;
        int ln = 0;
        for (;;) {
            const unsigned long long w = atomicAdd(V.word + ln, 0ull);
            const uint32_t cur = (uint32_t)(w >> 32), i = (uint32_t)w;
            if (cur == V.published[ln]) {   // nothing in this lane beyond its current job
                if (ln + 1 < kTcLanes) {
                    ++ln;
                    continue;
                }
                const uint64_t now = global_ns();
                if (idle0 == 0) {
                    idle0 = now;
                } else if (now - idle0 > V.idle_ns) {
                    break;
                }
                __nanosleep(2000);
                ln = 0;
                continue;
            }
            idle0 = 0;
            const int sl = ln * kTcRing + (int)(cur % kTcRing);
            const long long total = __ldcg(&V.jobs[sl].total);
            const unsigned long long nw =
                (long long)i < total ? w + 1 : ((unsigned long long)(cur + 1) << 32);
            if (atomicCAS(V.word + ln, w, nw) == w && (long long)i < total) {
                slot = sl;
                item = i;
                seq = cur;
                break;
            }
            ln = 0;   // lost a race or finished a job: look at the first lane again
        }
    }
    slot = __shfl_sync(0xffffffffu, slot, 0);
    item = __shfl_sync(0xffffffffu, item, 0);
    seq = __shfl_sync(0xffffffffu, seq, 0);
    if (slot < 0) {
        if (lane == 0) S.quit = 1;
        __syncwarp();
        return;
    }
    // the job's arguments, read past L1 (the slot's earlier contents may sit there)
    const int words = (int)(sizeof(TcArgs) / 4);
    const uint32_t *src = reinterpret_cast<const uint32_t *>(&V.jobs[slot].args);
    uint32_t *dst = reinterpret_cast<uint32_t *>(&S.job_args);
    for (int j = lane; j < words; j += 32) dst[j] = __ldcg(src + j);
    if (lane == 0) {
        S.job_total = __ldcg(&V.jobs[slot].total);
        S.job_slot = slot;
        S.job_seq = seq;
    }
    __syncwarp();
    describe_item(S.job_args, item, S.item, lane);
}

// Served form: one item of the current job done (thread 0, after the CTA
// finished it); the job's last item publishes its completion to the host.
__device__ void serve_done(const TcServe &V, const TcServeShared &S) {
    __threadfence();
    const int32_t d = atomicAdd(&V.done[S.job_slot], 1) + 1;
    if ((int64_t)d == S.job_total) {
        __threadfence_system();
        V.done_seq[S.job_slot] = S.job_seq;
    }
}

}  // namespace

// One CTA per SM; loops over (leaf, query block, series range) items.
// kHooks: the test hooks of the bounded waits (a wait limit from the
// arguments, an epilogue warp stalled on a barrier nothing arrives at); the
// ordinary launch is compiled without them.
template <bool kHooks>
__global__ void __launch_bounds__(kTcThreads, 1) k_tc_scan(TcArgs A) {
    extern __shared__ __align__(1024) unsigned char tc_smem[];
    const int n = A.n;
    const uint32_t b_bytes = (uint32_t)kTcN * n * 2;             // a whole tile
    const int nst = kTcStages;
    unsigned char *sB = tc_smem;                             // 1024-aligned stages
    float2 *sX = reinterpret_cast<float2 *>(sB + kTcStages * kTcStageBytes);  // kNormSlots * kTcN
    float *kbest = reinterpret_cast<float *>(sX + kNormSlots * kTcN);      // kTcEpiThreads * kLocalK
    TcShared &S = *reinterpret_cast<TcShared *>(kbest + kTcEpiThreads * kLocalK);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (tid == 0) {
        for (int s = 0; s < kTcStages; ++s) {
            mbar_init(&S.full[s], 1);
            mbar_init(&S.empty[s], 1);
        }
        for (int b = 0; b < kAcc; ++b) {
            mbar_init(&S.acc_full[b], 1);
            mbar_init(&S.acc_empty[b], 32 * kTcEpiWarps);
        }
        mbar_init(&S.never, 1);
        S.abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {   // the MMA warp owns the tensor memory
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&S.tmem_base)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = S.tmem_base;
    const int64_t total = A.item_off[A.L];
    const uint32_t lbo = 128, sbo = (uint32_t)(n / 8) * 128;   // series tile, K-major core matrices

    // running counts of barrier completions (phases), kept per role
    uint32_t g_tile = 0;   // tiles processed by this CTA so far (all roles agree)
    uint32_t issued = 0;   // producer: tiles whose copies it issued; MMA warp: tiles it committed
    const uint64_t wait_ns = (kHooks && A.wait_ns) ? A.wait_ns : kWaitNs;
    long long my_cand = 0, my_pairs = 0, my_bytes = 0;

    // Items are claimed when a CTA is ready for one, so the query blocks of
    // a leaf range start together and share its tiles in L2.
    for (;;) {
        if (warp == 0) fetch_item(A, total, S.item, lane);
        __syncthreads();
        const TcItem &D = S.item;
        if (D.it >= total || S.abort_flag) break;
        // the query block into tensor memory: epilogue warp w writes lane
        // quarter w%4, 32-column chunks c (points 64c..64c+63) of its column
        // group (w-2)/4; zeros past gq and past n
        if (warp >= 2) {
            const int r = (warp & 3) * 32 + lane;
            const int q = D.qid[r];
#pragma unroll 1
            for (int h = 0; h < kEpiChunks; ++h) {
                const int c = ((warp - 2) >> 2) * kEpiChunks + h;
                if (64 * c >= n) break;
                uint32_t w[32];
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    uint4 v = make_uint4(0, 0, 0, 0);
                    const int k0 = 64 * c + 8 * i;
                    if (q >= 0 && k0 < n) v = *reinterpret_cast<const uint4 *>(A.Qb + (int64_t)q * n + k0);
                    w[4 * i + 0] = v.x;
                    w[4 * i + 1] = v.y;
                    w[4 * i + 2] = v.z;
                    w[4 * i + 3] = v.w;
                }
                tmem_st32(tmem + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)(kTmemA + 32 * c), w);
            }
            tmem_wait_st();
        }
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        const int T = D.tiles;
        const int64_t base = D.base, s0 = D.s0, s1 = D.s1;
        if (tid == 0) my_bytes += (long long)T * (b_bytes + kTcN * (long long)sizeof(float2));

        if (warp == 0) {
            // ---------------- producer: one bulk copy per tile, plus its norms
            if (lane == 0) {
                for (int t = 0; t < T; ++t) {
                    const uint32_t gt = g_tile + t;
                    const int s = gt % nst;
                    const uint32_t use = gt / nst;
                    if (use > 0 && !mbar_wait(&S.empty[s], (use - 1) & 1, &S.abort_flag, wait_ns)) break;
                    const int64_t row0 = base + (int64_t)t * kTcN;
                    const uint32_t norm_bytes = kTcN * (uint32_t)sizeof(float2);
                    mbar_arrive_expect_tx(&S.full[s], b_bytes + norm_bytes);
                    bulk_g2s(sB + s * kTcStageBytes, A.Xb + row0 * n, b_bytes, &S.full[s]);
                    bulk_g2s(sX + (gt % kNormSlots) * kTcN, A.xq + row0, norm_bytes, &S.full[s]);
                    issued = gt + 1;
                }
            }
        } else if (warp == 1) {
            // ---------------- MMA issuer
            if (lane == 0) {
                const uint32_t a_tmem = tmem + (uint32_t)kTmemA;
                const int ksteps = n / 16;
                for (int t = 0; t < T; ++t) {
                    const uint32_t gt = g_tile + t;
                    const int s = gt % nst;
                    const uint32_t use = gt / nst;
                    const int b = gt % kAcc;
                    const uint32_t ause = gt / kAcc;
                    if (ause > 0 && !mbar_wait(&S.acc_empty[b], (ause - 1) & 1, &S.abort_flag, wait_ns)) break;
                    if (!mbar_wait(&S.full[s], use & 1, &S.abort_flag, wait_ns)) break;
                    tc_fence_after();
                    const uint32_t b_base = smem_u32(sB + s * kTcStageBytes);
                    const uint32_t d = tmem + (uint32_t)(b * kTcN);
                    for (int ks = 0; ks < ksteps; ++ks) {
                        // K step: 16 points = 8 columns of A, 2 core matrices of B
                        const uint64_t bd = smem_desc(b_base + ks * 2 * 128, lbo, sbo);
                        mma_ts(d, a_tmem + (uint32_t)(ks * 8), bd, A.idesc, ks > 0 ? 1u : 0u);
                    }
                    mma_commit(&S.empty[s]);
                    mma_commit(&S.acc_full[b]);
                    issued = gt + 1;
                }
            }
        } else {
            // ---------------- epilogue: thread owns query row r, a quarter of the columns
            const int r = (warp & 3) * 32 + lane;   // TMEM lane quarter of this warp
            const int cq = (warp - 2) >> 2;         // column group
            const int q = D.qid[r];
            float q2e = 0.f, qa = 0.f, qoff2 = 0.f, U = 0.f;
            if (q >= 0) {
                q2e = A.q2e[q];
                qa = A.qa[q];
                qoff2 = A.qoff2[q];
                U = __uint_as_float(A.U[q]);
            }
            // the k best upper bounds of this thread: slot i of epilogue thread
            // e at kbest[i * kTcEpiThreads + e] (conflict-free); the column
            // quarters of a row keep separate lists
            float *kb = kbest + (tid - 64);
            const int kl = (A.k <= kLocalK) ? A.k : 0;
            for (int i = 0; i < kl; ++i) kb[i * kTcEpiThreads] = INFINITY;
            float kth = INFINITY;      // k-th smallest upper bound seen by this thread
            long long pairs = 0;
            // test hook: one epilogue warp waits for a barrier nothing
            // arrives at, so its bounded wait runs out and the CTA aborts
            const bool stalled = kHooks && A.dbg_stall && warp == 2 && g_tile == 0 &&
                                 !mbar_wait_warp(&S.never, 0, &S.abort_flag, wait_ns);
            for (int t = 0; t < T && !stalled; ++t) {
                const uint32_t gt = g_tile + t;
                const int b = gt % kAcc;
                const uint32_t ause = gt / kAcc;
                if (!mbar_wait_warp(&S.acc_full[b], ause & 1, &S.abort_flag, wait_ns)) break;
                tc_fence_after();
                if (q >= 0 && (t & 7) == 0) U = fminf(U, __uint_as_float(A.U[q]));
                const int64_t row0 = base + (int64_t)t * kTcN;
                // columns of this tile inside [s0, s1)
                const int jlo = (int)max((int64_t)0, s0 - row0);
                const int jhi = (int)min((int64_t)kTcN, s1 - row0);
                const float thr = U - q2e;   // lo <= U  <=>  x2e - qa|x| - 2v <= U - q2e
                const float2 *xs = sX + (gt % kNormSlots) * kTcN;
                uint32_t raw[kEpiChunks][32];
                static_assert(kEpiChunks == 2, "one 64-column load per thread and tile");
                tmem_ld64_issue(tmem + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)(b * kTcN + cq * 64), raw);
                tmem_wait_ld();
                // the accumulator is in registers: release it to the MMAs
                // before filtering
                tc_fence_before();
                mbar_arrive(&S.acc_empty[b]);
#pragma unroll
                for (int h = 0; h < kEpiChunks; ++h) {
                const int cb = (cq * kEpiChunks + h) * 32;
                // columns of this thread inside [s0, s1)
                const int a = max(jlo - cb, 0), z = min(jhi - cb, 32);
                if (q >= 0 && a < z) {
                    pairs += z - a;
                    // the filter value of every column, reduced to its minimum:
                    // a column survives iff its value is <= thr, so a minimum
                    // above thr (the common case) clears all 32 at once
                    float m0 = INFINITY, m1 = INFINITY, m2 = INFINITY, m3 = INFINITY;
#pragma unroll
                    for (int j = 0; j < 32; j += 4) {
                        const float4 x01 = *reinterpret_cast<const float4 *>(xs + cb + j);
                        const float4 x23 = *reinterpret_cast<const float4 *>(xs + cb + j + 2);
                        m0 = fminf(m0, fmaf(-2.0f, __uint_as_float(raw[h][j + 0]), fmaf(-qa, x01.y, x01.x)));
                        m1 = fminf(m1, fmaf(-2.0f, __uint_as_float(raw[h][j + 1]), fmaf(-qa, x01.w, x01.z)));
                        m2 = fminf(m2, fmaf(-2.0f, __uint_as_float(raw[h][j + 2]), fmaf(-qa, x23.y, x23.x)));
                        m3 = fminf(m3, fmaf(-2.0f, __uint_as_float(raw[h][j + 3]), fmaf(-qa, x23.w, x23.z)));
                    }
                    const bool any = fminf(fminf(m0, m1), fminf(m2, m3)) <= thr;
                    if (any || A.dbg_lo) {
                        const uint32_t valid =
                            (z >= 32 ? 0xffffffffu : ((1u << z) - 1u)) & ~((1u << a) - 1u);
                        float v[32];
#pragma unroll
                        for (int j = 0; j < 32; ++j) v[j] = __uint_as_float(raw[h][j]);
                        uint32_t hit = 0;
#pragma unroll
                        for (int j = 0; j < 32; ++j) {
                            const float2 xv = xs[cb + j];
                            const float lhs = fmaf(-2.0f, v[j], fmaf(-qa, xv.y, xv.x));
                            hit |= (lhs <= thr ? 1u : 0u) << j;
                        }
                        hit &= valid;
                        if (A.dbg_lo) {
                            for (int j = a; j < z; ++j) {
                                const float2 xv = xs[cb + j];
                                const float lo = fmaf(-2.0f, v[j], fmaf(-qa, xv.y, xv.x)) + q2e;
                                const float bs = lo + 2.0f * qa * xv.y;
                                A.dbg_lo[(int64_t)q * A.N + row0 + cb + j] = lo;
                                A.dbg_up[(int64_t)q * A.N + row0 + cb + j] =
                                    bs + fabsf(bs) * 0x1p-18f + A.eb2 * (q2e + xv.x) + qoff2;
                            }
                        }
                        while (hit) {
                            // survivor: exact lower / upper bounds in the
                            // certified form (rounded outward)
                            const int j = __ffs(hit) - 1;
                            hit &= hit - 1;
                            const float2 xv = xs[cb + j];
                            const float lo = fmaf(-2.0f, v[j], fmaf(-qa, xv.y, xv.x)) + q2e;
                            const float bs = lo + 2.0f * qa * xv.y;
                            const float up = bs + fabsf(bs) * 0x1p-18f + A.eb2 * (q2e + xv.x) + qoff2;
                            if (kl && up < kth) {
                                int mi = 0;
                                for (int i = 1; i < kl; ++i)
                                    if (kb[i * kTcEpiThreads] > kb[mi * kTcEpiThreads]) mi = i;
                                kb[mi * kTcEpiThreads] = up;
                                float mx = kb[0];
                                for (int i = 1; i < kl; ++i) mx = fmaxf(mx, kb[i * kTcEpiThreads]);
                                kth = mx;
                            }
                            if (lo <= U) {
                                const int slot = atomicAdd(&A.cand_cnt[q], 1);
                                if (slot < A.cand_C) {
                                    A.cand_p[(int64_t)q * A.cand_C + slot] = (int32_t)(row0 + cb + j);
                                    A.cand_lb[(int64_t)q * A.cand_C + slot] = lo;
                                    ++my_cand;
                                } else {
                                    atomicOr(&A.qflag[q], 1);
                                }
                            }
                        }
                    }
                }
                }
                if (q >= 0 && kth < U) {
                    U = kth;
                    atomicMin(&A.U[q], __float_as_uint(kth));
                }
            }
            my_pairs += pairs;
        }
        g_tile += T;
        __syncthreads();
    }
    // drain: a CTA that aborted may have copies or MMAs in flight.  The
    // producer waits for the copies of the last kTcStages tiles it issued
    // (earlier ones were consumed by the MMA warp, so they landed); the MMA
    // warp waits for the commits of the last tile it issued (a commit
    // arrives once every earlier MMA of the thread completed).  Each wait
    // ends by a deadline; then the tensor memory is freed.
    if (S.abort_flag) {
        if (tid == 0) atomicOr(A.err, 2);
        const uint64_t deadline = global_ns() + kDrainNs;
        bool landed = true;
        if (warp == 0 && lane == 0) {
            for (uint32_t gt = issued > (uint32_t)nst ? issued - nst : 0; gt < issued; ++gt)
                landed &= mbar_wait_until(&S.full[gt % nst], (gt / nst) & 1, deadline);
        } else if (warp == 1 && lane == 0 && issued > 0) {
            const uint32_t last = issued - 1;
            landed &= mbar_wait_until(&S.empty[last % nst], (last / nst) & 1, deadline);
            landed &= mbar_wait_until(&S.acc_full[last % kAcc], (last / kAcc) & 1, deadline);
        }
        if (!landed) atomicOr(A.err, 4);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols)
                     : "memory");
    }
    my_pairs = warp_sum_ll(my_pairs);
    my_cand = warp_sum_ll(my_cand);
    if (lane == 0 && A.stats) {
        stat_add(&A.stats[A.stat_pairs], my_pairs);
        stat_add(&A.stats[A.stat_cands], my_cand);
        if (tid == 0) stat_add(&A.stats[A.stat_bytes], my_bytes);
    }
}

// The served form of k_tc_scan: the same roles and pipeline, with items taken
// from the jobs of a ring (V) until none comes for V.idle_ns; each item's
// arguments are its job's (copied into shared memory).  The batch kernel is
// kept as its own function so its code stays exactly as measured.
__global__ void __launch_bounds__(kTcThreads, 1) k_tc_serve(TcServe V) {
    constexpr bool kHooks = false, kServe = true;
    const TcArgs P{};
    extern __shared__ __align__(1024) unsigned char tc_smem[];
    const int nst = kTcStages;
    unsigned char *sB = tc_smem;                             // 1024-aligned stages
    float2 *sX = reinterpret_cast<float2 *>(sB + kTcStages * kTcStageBytes);  // kNormSlots * kTcN
    float *kbest = reinterpret_cast<float *>(sX + kNormSlots * kTcN);      // kTcEpiThreads * kLocalK
    TcServeShared &S = *reinterpret_cast<TcServeShared *>(kbest + kTcEpiThreads * kLocalK);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (tid == 0) {
        for (int s = 0; s < kTcStages; ++s) {
            mbar_init(&S.full[s], 1);
            mbar_init(&S.empty[s], 1);
        }
        for (int b = 0; b < kAcc; ++b) {
            mbar_init(&S.acc_full[b], 1);
            mbar_init(&S.acc_empty[b], 32 * kTcEpiWarps);
        }
        mbar_init(&S.never, 1);
        S.abort_flag = 0;
        S.quit = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {   // the MMA warp owns the tensor memory
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&S.tmem_base)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = S.tmem_base;
    const TcArgs &A = kServe ? S.job_args : P;   // the current item's arguments
    int64_t total = 0;
    if constexpr (!kServe) total = P.item_off[P.L];

    // running counts of barrier completions (phases), kept per role
    uint32_t g_tile = 0;   // tiles processed by this CTA so far (all roles agree)
    uint32_t issued = 0;   // producer: tiles whose copies it issued; MMA warp: tiles it committed
    const uint64_t wait_ns = (kHooks && P.wait_ns) ? P.wait_ns : kWaitNs;
    long long my_cand = 0, my_pairs = 0, my_bytes = 0;

    // Items are claimed when a CTA is ready for one, so the query blocks of
    // a leaf range start together and share its tiles in L2.
    for (;;) {
        if (warp == 0) {
            if constexpr (kServe)
                serve_fetch(V, S, lane);
            else
                fetch_item(P, total, S.item, lane);
        }
        __syncthreads();
        const TcItem &D = S.item;
        if constexpr (kServe) {
            if (S.quit || S.abort_flag) break;
        } else {
            if (D.it >= total || S.abort_flag) break;
        }
        const int n = A.n;
        const uint32_t b_bytes = (uint32_t)kTcN * n * 2;             // a whole tile
        const uint32_t lbo = 128, sbo = (uint32_t)(n / 8) * 128;   // series tile, K-major core matrices
        // the query block into tensor memory: epilogue warp w writes lane
        // quarter w%4, 32-column chunks c (points 64c..64c+63) of its column
        // group (w-2)/4; zeros past gq and past n
        if (warp >= 2) {
            const int r = (warp & 3) * 32 + lane;
            const int q = D.qid[r];
#pragma unroll 1
            for (int h = 0; h < kEpiChunks; ++h) {
                const int c = ((warp - 2) >> 2) * kEpiChunks + h;
                if (64 * c >= n) break;
                uint32_t w[32];
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    uint4 v = make_uint4(0, 0, 0, 0);
                    const int k0 = 64 * c + 8 * i;
                    if (q >= 0 && k0 < n) v = *reinterpret_cast<const uint4 *>(A.Qb + (int64_t)q * n + k0);
                    w[4 * i + 0] = v.x;
                    w[4 * i + 1] = v.y;
                    w[4 * i + 2] = v.z;
                    w[4 * i + 3] = v.w;
                }
                tmem_st32(tmem + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)(kTmemA + 32 * c), w);
            }
            tmem_wait_st();
        }
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        const int T = D.tiles;
        const int64_t base = D.base, s0 = D.s0, s1 = D.s1;
        if (tid == 0) my_bytes += (long long)T * (b_bytes + kTcN * (long long)sizeof(float2));

        if (warp == 0) {
            // ---------------- producer: one bulk copy per tile, plus its norms
            if (lane == 0) {
                for (int t = 0; t < T; ++t) {
                    const uint32_t gt = g_tile + t;
                    const int s = gt % nst;
                    const uint32_t use = gt / nst;
                    if (use > 0 && !mbar_wait(&S.empty[s], (use - 1) & 1, &S.abort_flag, wait_ns)) break;
                    const int64_t row0 = base + (int64_t)t * kTcN;
                    const uint32_t norm_bytes = kTcN * (uint32_t)sizeof(float2);
                    mbar_arrive_expect_tx(&S.full[s], b_bytes + norm_bytes);
                    bulk_g2s(sB + s * kTcStageBytes, A.Xb + row0 * n, b_bytes, &S.full[s]);
                    bulk_g2s(sX + (gt % kNormSlots) * kTcN, A.xq + row0, norm_bytes, &S.full[s]);
                    issued = gt + 1;
                }
            }
        } else if (warp == 1) {
            // ---------------- MMA issuer
            if (lane == 0) {
                const uint32_t a_tmem = tmem + (uint32_t)kTmemA;
                const int ksteps = n / 16;
                for (int t = 0; t < T; ++t) {
                    const uint32_t gt = g_tile + t;
                    const int s = gt % nst;
                    const uint32_t use = gt / nst;
                    const int b = gt % kAcc;
                    const uint32_t ause = gt / kAcc;
                    if (ause > 0 && !mbar_wait(&S.acc_empty[b], (ause - 1) & 1, &S.abort_flag, wait_ns)) break;
                    if (!mbar_wait(&S.full[s], use & 1, &S.abort_flag, wait_ns)) break;
                    tc_fence_after();
                    const uint32_t b_base = smem_u32(sB + s * kTcStageBytes);
                    const uint32_t d = tmem + (uint32_t)(b * kTcN);
                    for (int ks = 0; ks < ksteps; ++ks) {
                        // K step: 16 points = 8 columns of A, 2 core matrices of B
                        const uint64_t bd = smem_desc(b_base + ks * 2 * 128, lbo, sbo);
                        mma_ts(d, a_tmem + (uint32_t)(ks * 8), bd, A.idesc, ks > 0 ? 1u : 0u);
                    }
                    mma_commit(&S.empty[s]);
                    mma_commit(&S.acc_full[b]);
                    issued = gt + 1;
                }
            }
        } else {
            // ---------------- epilogue: thread owns query row r, a quarter of the columns
            const int r = (warp & 3) * 32 + lane;   // TMEM lane quarter of this warp
            const int cq = (warp - 2) >> 2;         // column group
            const int q = D.qid[r];
            float q2e = 0.f, qa = 0.f, qoff2 = 0.f, U = 0.f;
            if (q >= 0) {
                q2e = A.q2e[q];
                qa = A.qa[q];
                qoff2 = A.qoff2[q];
                U = __uint_as_float(A.U[q]);
            }
            // the k best upper bounds of this thread: slot i of epilogue thread
            // e at kbest[i * kTcEpiThreads + e] (conflict-free); the column
            // quarters of a row keep separate lists
            float *kb = kbest + (tid - 64);
            const int kl = (A.k <= kLocalK) ? A.k : 0;
            for (int i = 0; i < kl; ++i) kb[i * kTcEpiThreads] = INFINITY;
            float kth = INFINITY;      // k-th smallest upper bound seen by this thread
            long long pairs = 0;
            // test hook: one epilogue warp waits for a barrier nothing
            // arrives at, so its bounded wait runs out and the CTA aborts
            const bool stalled = kHooks && P.dbg_stall && warp == 2 && g_tile == 0 &&
                                 !mbar_wait_warp(&S.never, 0, &S.abort_flag, wait_ns);
            for (int t = 0; t < T && !stalled; ++t) {
                const uint32_t gt = g_tile + t;
                const int b = gt % kAcc;
                const uint32_t ause = gt / kAcc;
                if (!mbar_wait_warp(&S.acc_full[b], ause & 1, &S.abort_flag, wait_ns)) break;
                tc_fence_after();
                if (q >= 0 && (t & 7) == 0) U = fminf(U, __uint_as_float(A.U[q]));
                const int64_t row0 = base + (int64_t)t * kTcN;
                // columns of this tile inside [s0, s1)
                const int jlo = (int)max((int64_t)0, s0 - row0);
                const int jhi = (int)min((int64_t)kTcN, s1 - row0);
                const float thr = U - q2e;   // lo <= U  <=>  x2e - qa|x| - 2v <= U - q2e
                const float2 *xs = sX + (gt % kNormSlots) * kTcN;
                uint32_t raw[kEpiChunks][32];
                static_assert(kEpiChunks == 2, "one 64-column load per thread and tile");
                tmem_ld64_issue(tmem + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)(b * kTcN + cq * 64), raw);
                tmem_wait_ld();
                // the accumulator is in registers: release it to the MMAs
                // before filtering
                tc_fence_before();
                mbar_arrive(&S.acc_empty[b]);
#pragma unroll
                for (int h = 0; h < kEpiChunks; ++h) {
                const int cb = (cq * kEpiChunks + h) * 32;
                // columns of this thread inside [s0, s1)
                const int a = max(jlo - cb, 0), z = min(jhi - cb, 32);
                if (q >= 0 && a < z) {
                    pairs += z - a;
                    // the filter value of every column, reduced to its minimum:
                    // a column survives iff its value is <= thr, so a minimum
                    // above thr (the common case) clears all 32 at once
                    float m0 = INFINITY, m1 = INFINITY, m2 = INFINITY, m3 = INFINITY;
#pragma unroll
                    for (int j = 0; j < 32; j += 4) {
                        const float4 x01 = *reinterpret_cast<const float4 *>(xs + cb + j);
                        const float4 x23 = *reinterpret_cast<const float4 *>(xs + cb + j + 2);
                        m0 = fminf(m0, fmaf(-2.0f, __uint_as_float(raw[h][j + 0]), fmaf(-qa, x01.y, x01.x)));
                        m1 = fminf(m1, fmaf(-2.0f, __uint_as_float(raw[h][j + 1]), fmaf(-qa, x01.w, x01.z)));
                        m2 = fminf(m2, fmaf(-2.0f, __uint_as_float(raw[h][j + 2]), fmaf(-qa, x23.y, x23.x)));
                        m3 = fminf(m3, fmaf(-2.0f, __uint_as_float(raw[h][j + 3]), fmaf(-qa, x23.w, x23.z)));
                    }
                    const bool any = fminf(fminf(m0, m1), fminf(m2, m3)) <= thr;
                    if (any || A.dbg_lo) {
                        const uint32_t valid =
                            (z >= 32 ? 0xffffffffu : ((1u << z) - 1u)) & ~((1u << a) - 1u);
                        float v[32];
#pragma unroll
                        for (int j = 0; j < 32; ++j) v[j] = __uint_as_float(raw[h][j]);
                        uint32_t hit = 0;
#pragma unroll
                        for (int j = 0; j < 32; ++j) {
                            const float2 xv = xs[cb + j];
                            const float lhs = fmaf(-2.0f, v[j], fmaf(-qa, xv.y, xv.x));
                            hit |= (lhs <= thr ? 1u : 0u) << j;
                        }
                        hit &= valid;
                        if (A.dbg_lo) {
                            for (int j = a; j < z; ++j) {
                                const float2 xv = xs[cb + j];
                                const float lo = fmaf(-2.0f, v[j], fmaf(-qa, xv.y, xv.x)) + q2e;
                                const float bs = lo + 2.0f * qa * xv.y;
                                A.dbg_lo[(int64_t)q * A.N + row0 + cb + j] = lo;
                                A.dbg_up[(int64_t)q * A.N + row0 + cb + j] =
                                    bs + fabsf(bs) * 0x1p-18f + A.eb2 * (q2e + xv.x) + qoff2;
                            }
                        }
                        while (hit) {
                            // survivor: exact lower / upper bounds in the
                            // certified form (rounded outward)
                            const int j = __ffs(hit) - 1;
                            hit &= hit - 1;
                            const float2 xv = xs[cb + j];
                            const float lo = fmaf(-2.0f, v[j], fmaf(-qa, xv.y, xv.x)) + q2e;
                            const float bs = lo + 2.0f * qa * xv.y;
                            const float up = bs + fabsf(bs) * 0x1p-18f + A.eb2 * (q2e + xv.x) + qoff2;
                            if (kl && up < kth) {
                                int mi = 0;
                                for (int i = 1; i < kl; ++i)
                                    if (kb[i * kTcEpiThreads] > kb[mi * kTcEpiThreads]) mi = i;
                                kb[mi * kTcEpiThreads] = up;
                                float mx = kb[0];
                                for (int i = 1; i < kl; ++i) mx = fmaxf(mx, kb[i * kTcEpiThreads]);
                                kth = mx;
                            }
                            if (lo <= U) {
                                const int slot = atomicAdd(&A.cand_cnt[q], 1);
                                if (slot < A.cand_C) {
                                    A.cand_p[(int64_t)q * A.cand_C + slot] = (int32_t)(row0 + cb + j);
                                    A.cand_lb[(int64_t)q * A.cand_C + slot] = lo;
                                    ++my_cand;
                                } else {
                                    atomicOr(&A.qflag[q], 1);
                                }
                            }
                        }
                    }
                }
                }
                if (q >= 0 && kth < U) {
                    U = kth;
                    atomicMin(&A.U[q], __float_as_uint(kth));
                }
            }
            my_pairs += pairs;
        }
        g_tile += T;
        __syncthreads();
        if constexpr (kServe) {
            if (tid == 0 && !S.abort_flag) serve_done(V, S);
        }
    }
    // drain: a CTA that aborted may have copies or MMAs in flight.  The
    // producer waits for the copies of the last kTcStages tiles it issued
    // (earlier ones were consumed by the MMA warp, so they landed); the MMA
    // warp waits for the commits of the last tile it issued (a commit
    // arrives once every earlier MMA of the thread completed).  Each wait
    // ends by a deadline; then the tensor memory is freed.
    if (S.abort_flag) {
        if (tid == 0) atomicOr(A.err, 2);
        const uint64_t deadline = global_ns() + kDrainNs;
        bool landed = true;
        if (warp == 0 && lane == 0) {
            for (uint32_t gt = issued > (uint32_t)nst ? issued - nst : 0; gt < issued; ++gt)
                landed &= mbar_wait_until(&S.full[gt % nst], (gt / nst) & 1, deadline);
        } else if (warp == 1 && lane == 0 && issued > 0) {
            const uint32_t last = issued - 1;
            landed &= mbar_wait_until(&S.empty[last % nst], (last / nst) & 1, deadline);
            landed &= mbar_wait_until(&S.acc_full[last % kAcc], (last / kAcc) & 1, deadline);
        }
        if (!landed) atomicOr(A.err, 4);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols)
                     : "memory");
    }
    my_pairs = warp_sum_ll(my_pairs);
    my_cand = warp_sum_ll(my_cand);
    if (lane == 0 && P.stats) {
        stat_add(&P.stats[P.stat_pairs], my_pairs);
        stat_add(&P.stats[P.stat_cands], my_cand);
        if (tid == 0) stat_add(&P.stats[P.stat_bytes], my_bytes);
    }
}

// 16-bit copy (bfloat16 or float16) of the leaf-ordered collection in
// core-matrix order, and per series {|x|^2 (1 - eb) rounded down, |x|
// rounded up} from binary64 sums.  Values a float16 cannot hold set *bad.
__device__ __forceinline__ uint16_t to16(float v, int fmt) {
    if (fmt == kFmtBF16) return __bfloat16_as_ushort(__float2bfloat16_rn(v));
    return __half_as_ushort(__float2half_rn(v));
}

__global__ void k_make_16(const float *__restrict__ X, int64_t N, int n, int64_t Npad, int fmt,
                          uint16_t *__restrict__ Xb, float2 *__restrict__ xq, int *__restrict__ bad) {
    const int nk = n / 8;
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < Npad * nk;
         c += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = c / nk;
        const int k8 = (int)(c % nk);
        uint16_t h[8];
        if (i < N) {
            const float4 a = *reinterpret_cast<const float4 *>(X + i * n + k8 * 8);
            const float4 b = *reinterpret_cast<const float4 *>(X + i * n + k8 * 8 + 4);
            const float f[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                if (fmt == kFmtF16 && fabsf(f[e]) > kF16Max) *bad = 1;
                h[e] = to16(f[e], fmt);
            }
        } else {
            for (int e = 0; e < 8; ++e) h[e] = 0;
        }
        const int64_t off = (((i >> 3) * nk + k8) * 8 + (i & 7)) * 8;
        *reinterpret_cast<uint4 *>(Xb + off) = *reinterpret_cast<const uint4 *>(h);
    }
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < Npad;
         i += (int64_t)gridDim.x * blockDim.x) {
        double s = 0.0;
        if (i < N)
            for (int j = 0; j < n; ++j) s += (double)X[i * n + j] * (double)X[i * n + j];
        xq[i] = make_float2(__double2float_rd(s * (1.0 - kTcEb)), __double2float_ru(sqrt(s)));
    }
}

// Queries: 16-bit rows, |q|^2 (1 - eb) lowered by the query's absolute
// error term (rounded down), the coefficient c |q| (rounded up) and twice
// the absolute term (for the interval's upper end).
__global__ void k_tc_qprep(const float *__restrict__ Q, int nq, int n, int fmt, double c_rel,
                           double abs_unit, double xn_max, uint16_t *__restrict__ Qb,
                           float *__restrict__ q2e, float *__restrict__ qa, float *__restrict__ qoff2,
                           int *__restrict__ bad) {
    const int q = blockIdx.x;
    if (q >= nq) return;
    __shared__ double red[32];
    double s = 0.0;
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
        const float v = Q[(int64_t)q * n + j];
        if (fmt == kFmtF16 && fabsf(v) > kF16Max) *bad = 1;
        Qb[(int64_t)q * n + j] = to16(v, fmt);
        s += (double)v * (double)v;
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
        const double qn = sqrt(t);
        // sum_j |q^_j x^_j - q_j x_j| beyond the relative term: at most
        // a (|q_j| (2+u) + |x_j| (1+u)) + a^2 per point, a the half spacing
        // of the format's subnormals; summed and doubled for the -2 factor
        const double off = 2.0 * (abs_unit * sqrt((double)n) * (2.01 * qn + 1.01 * xn_max) +
                                  (double)n * abs_unit * abs_unit);
        q2e[q] = __double2float_rd(t * (1.0 - kTcEb) - off);
        qa[q] = __double2float_ru(c_rel * qn);
        qoff2[q] = __double2float_ru(2.0 * off);
    }
}

// Exact float32 distances of the candidates at or below the final bound into
// the query's pool.  Work items are runs of kRescoreChunk candidates of one
// query (item_off: exclusive scan of the items per query), spread over a
// persistent grid so that a query with many candidates does not hold up the
// launch.  A warp reads 32 candidates' bounds and positions at once, then
// rescores the live ones four rows at a time with 16-byte loads.  Any
// summation order stays within the rounding bound that T(U) allows for.
constexpr int kRescoreChunk = 256;
__global__ void k_rescore_items(const int32_t *__restrict__ cand_cnt, int nq, int cand_C,
                                int32_t *__restrict__ items) {
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < nq; q += gridDim.x * blockDim.x)
        items[q] = (min(cand_cnt[q], cand_C) + kRescoreChunk - 1) / kRescoreChunk;
}

__global__ void k_tc_rescore(const float *__restrict__ Q, const float *__restrict__ X, int n, int nq,
                             const int32_t *__restrict__ item_off,
                             const int32_t *__restrict__ cand_cnt, const int32_t *__restrict__ cand_p,
                             const float *__restrict__ cand_lb, int cand_C,
                             const uint32_t *__restrict__ U, float *__restrict__ pool_d,
                             int32_t *__restrict__ pool_p, int32_t *__restrict__ pool_cnt, int pool_C,
                             int32_t *__restrict__ qflag, long long *__restrict__ stats, int stat_slot) {
    const int lane = threadIdx.x & 31;
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int total = item_off[nq];
    const int n4 = n / 4;
    long long done = 0;
    for (int64_t it = gw; it < total; it += nw) {
        // the item's query: the last q with item_off[q] <= it
        int lo = 0, hi = nq - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (item_off[mid] <= it) lo = mid; else hi = mid - 1;
        }
        const int q = lo;
        const int cnt = min(cand_cnt[q], cand_C);
        const int cb = (int)(it - item_off[q]) * kRescoreChunk;
        const int ce = min(cb + kRescoreChunk, cnt);
        const float u = __uint_as_float(U[q]);
        const float4 *q4 = reinterpret_cast<const float4 *>(Q + (int64_t)q * n);
        for (int c0 = cb; c0 < ce; c0 += 32) {
            const int c = c0 + lane;
            float lb = INFINITY;
            int32_t pos = 0;
            if (c < ce) {
                lb = cand_lb[(int64_t)q * cand_C + c];
                pos = cand_p[(int64_t)q * cand_C + c];
            }
            unsigned live = __ballot_sync(0xffffffffu, lb <= u);
            while (live) {
                // up to four live candidates at once (repeats of the last
                // one fill the slots and are not stored)
                int ii[4];
                int m = 0;
#pragma unroll
                for (int r = 0; r < 4; ++r) {
                    if (live) {
                        ii[r] = __ffs(live) - 1;
                        live &= live - 1;
                        m = r + 1;
                    } else {
                        ii[r] = ii[r > 0 ? r - 1 : 0];
                    }
                }
                int32_t pr[4];
                const float4 *xr[4];
                float a[4];
#pragma unroll
                for (int r = 0; r < 4; ++r) {
                    pr[r] = __shfl_sync(0xffffffffu, pos, ii[r]);
                    xr[r] = reinterpret_cast<const float4 *>(X + (int64_t)pr[r] * n);
                    a[r] = 0.0f;
                }
                for (int j = lane; j < n4; j += 32) {
                    const float4 qv = q4[j];
#pragma unroll
                    for (int r = 0; r < 4; ++r) {
                        const float4 xv = xr[r][j];
                        float d;
                        d = qv.x - xv.x; a[r] = fmaf(d, d, a[r]);
                        d = qv.y - xv.y; a[r] = fmaf(d, d, a[r]);
                        d = qv.z - xv.z; a[r] = fmaf(d, d, a[r]);
                        d = qv.w - xv.w; a[r] = fmaf(d, d, a[r]);
                    }
                }
#pragma unroll
                for (int r = 0; r < 4; ++r)
                    for (int o = 16; o > 0; o >>= 1) a[r] += __shfl_xor_sync(0xffffffffu, a[r], o);
                if (lane == 0) {
                    done += m;
                    const int slot = atomicAdd(&pool_cnt[q], m);
#pragma unroll
                    for (int r = 0; r < 4; ++r)
                        if (r < m && slot + r < pool_C) {
                            pool_d[(int64_t)q * pool_C + slot + r] = a[r];
                            pool_p[(int64_t)q * pool_C + slot + r] = pr[r];
                        }
                    if (slot + m > pool_C) atomicOr(&qflag[q], 1);
                }
            }
        }
    }
    if (lane == 0 && done) stat_add(&stats[stat_slot], done);
}

size_t tc_serve_smem_bytes() {
    return (size_t)kTcStages * kTcStageBytes + (size_t)kNormSlots * kTcN * 8 +
           (size_t)kTcEpiThreads * kLocalK * 4 + sizeof(TcServeShared) + 1024;
}

size_t tc_smem_bytes(int n) {
    (void)n;   // stages are sized for the longest series
    return (size_t)kTcStages * kTcStageBytes + (size_t)kNormSlots * kTcN * 8 +
           (size_t)kTcEpiThreads * kLocalK * 4 + sizeof(TcShared) + 1024;
}

uint32_t tc_idesc(int fmt) {
    uint32_t d = 0;
    d |= 1u << 4;                          // D format: float32
    d |= (uint32_t)fmt << 7;               // A format: 0 float16, 1 bfloat16
    d |= (uint32_t)fmt << 10;              // B format: the same as A
    d |= (uint32_t)(kTcN >> 3) << 17;      // N
    d |= (uint32_t)(kTcM >> 4) << 24;      // M
    return d;                              // both operands K-major, dense
}

float tc_eb2() { return (float)(2.0 * kTcEb / (1.0 - kTcEb) * (1.0 + 0x1p-10)); }

double tc_error_coefficient(int n, int fmt) {
    const double u = std::ldexp(1.0, fmt == kFmtBF16 ? -8 : -11);   // unit roundoff of the format
    const double w = std::ldexp(1.0, -20);
    const double g = n * w / (1.0 - n * w);
    const double c1 = 2 * u + u * u + g * (1 + u) * (1 + u);
    return (2.0 * c1 + std::ldexp(1.0, -18)) * (1.0 + std::ldexp(1.0, -10));
}

void launch_tc_scan(const TcArgs &a, cudaStream_t s) {
    const size_t smem = tc_smem_bytes(a.n);
    static std::once_flag once;
    std::call_once(once, [] {
        HK_CHECK_CUDA(cudaFuncSetAttribute(k_tc_scan<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)tc_smem_bytes(256)));
        HK_CHECK_CUDA(cudaFuncSetAttribute(k_tc_scan<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)tc_smem_bytes(256)));
    });
    int dev = 0, sms = 0;
    HK_CHECK_CUDA(cudaGetDevice(&dev));
    HK_CHECK_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    if (a.wait_ns || a.dbg_stall)
        k_tc_scan<true><<<sms, kTcThreads, smem, s>>>(a);
    else
        k_tc_scan<false><<<sms, kTcThreads, smem, s>>>(a);
    HK_CHECK_LAUNCH();
}

// ---------------------------------------------------------------- served form (host)
// One resident launch of the served scan takes the scans (jobs) of all
// batches in flight, from any collection with a 16-bit copy: a job's
// arguments go to a ring slot in device memory, then the count of
// published jobs (host-mapped memory, read by the launch) moves on; the
// launch writes each finished job's sequence number back to host-mapped
// memory.  A launch leaves after idle_ns without work; a job published
// after it left starts another.  Every wait is bounded.
struct TcEngine {
    int ctas = 0;
    cudaStream_t stream = nullptr;   // the resident launch
    cudaStream_t pub = nullptr;      // the ring's copies
    DevBuf<TcJob> jobs;
    DevBuf<unsigned long long> word;
    DevBuf<int32_t> done;
    uint32_t *ctl_h = nullptr;       // mapped: [lane] published, [kTcLanes + slot] last completed sequence
    uint32_t *ctl_d = nullptr;
    uint32_t published[kTcLanes] = {};
    bool launched = false;
    cudaEvent_t ev = nullptr;        // recorded after the last launch
    std::mutex mu;
    TcEngineStats st{};
    std::vector<const void *> colls;   // collections the current launch took jobs of
    uint64_t idle_ns = 2000000;
};

namespace {

bool engine_running(TcEngine *e) {
    if (!e->launched) return false;
    const cudaError_t r = cudaEventQuery(e->ev);
    if (r == cudaErrorNotReady) return true;
    HK_CHECK_CUDA(r);
    return false;
}

void engine_launch(TcEngine *e) {
    TcServe V{};
    V.jobs = e->jobs.p;
    V.word = e->word.p;
    V.done = e->done.p;
    V.published = e->ctl_d;
    V.done_seq = e->ctl_d + kTcLanes;
    V.idle_ns = e->idle_ns;
    k_tc_serve<<<e->ctas, kTcThreads, tc_serve_smem_bytes(), e->stream>>>(V);
    HK_CHECK_LAUNCH();
    HK_CHECK_CUDA(cudaEventRecord(e->ev, e->stream));
    e->launched = true;
    e->st.launches += 1;
    e->colls.clear();
}

void engine_note_coll(TcEngine *e, const void *x) {
    if (std::find(e->colls.begin(), e->colls.end(), x) == e->colls.end()) e->colls.push_back(x);
    e->st.max_colls_per_launch = std::max<long long>(e->st.max_colls_per_launch, (long long)e->colls.size());
}

}  // namespace

TcEngine *tc_engine_create(int spare_sms) {
    std::unique_ptr<TcEngine> e(new TcEngine());
    int dev = 0, sms = 0;
    HK_CHECK_CUDA(cudaGetDevice(&dev));
    HK_CHECK_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    // a few SMs stay free for the batches' other kernels, which cannot share
    // an SM with the resident launch's shared memory
    e->ctas = std::max(1, sms - spare_sms);
    HK_CHECK_CUDA(cudaFuncSetAttribute(k_tc_serve, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)tc_serve_smem_bytes()));
    HK_CHECK_CUDA(cudaStreamCreateWithFlags(&e->stream, cudaStreamNonBlocking));
    HK_CHECK_CUDA(cudaStreamCreateWithFlags(&e->pub, cudaStreamNonBlocking));
    HK_CHECK_CUDA(cudaEventCreateWithFlags(&e->ev, cudaEventDisableTiming));
    e->jobs.alloc(kTcLanes * kTcRing, e->pub);
    e->word.alloc(kTcLanes, e->pub);
    e->done.alloc(kTcLanes * kTcRing, e->pub);
    HK_CHECK_CUDA(cudaMemsetAsync(e->word.p, 0, kTcLanes * sizeof(unsigned long long), e->pub));
    HK_CHECK_CUDA(cudaMemsetAsync(e->done.p, 0, kTcLanes * kTcRing * sizeof(int32_t), e->pub));
    HK_CHECK_CUDA(cudaHostAlloc((void **)&e->ctl_h, (kTcLanes + kTcLanes * kTcRing) * sizeof(uint32_t),
                                cudaHostAllocMapped));
    for (int i = 0; i < kTcLanes; ++i) e->ctl_h[i] = 0;
    for (int i = 0; i < kTcLanes * kTcRing; ++i) e->ctl_h[kTcLanes + i] = 0xffffffffu;
    HK_CHECK_CUDA(cudaHostGetDevicePointer((void **)&e->ctl_d, e->ctl_h, 0));
    HK_CHECK_CUDA(cudaStreamSynchronize(e->pub));
    return e.release();
}

void tc_engine_destroy(TcEngine *e) {
    if (!e) return;
    // the launch leaves by itself once idle (bounded)
    if (e->stream) cudaStreamSynchronize(e->stream);
    if (e->pub) cudaStreamSynchronize(e->pub);
    if (e->ev) cudaEventDestroy(e->ev);
    if (e->stream) cudaStreamDestroy(e->stream);
    if (e->pub) cudaStreamDestroy(e->pub);
    if (e->ctl_h) cudaFreeHost(e->ctl_h);
    delete e;
}

void tc_engine_stats(TcEngine *e, TcEngineStats *out) {
    std::lock_guard<std::mutex> lk(e->mu);
    *out = e->st;
}

void tc_engine_run(TcEngine *e, const TcArgs &a, int64_t items, uint64_t timeout_ns, int lane) {
    using clock = std::chrono::steady_clock;
    const auto t0 = clock::now();
    auto late = [&] {
        return (uint64_t)std::chrono::duration_cast<std::chrono::nanoseconds>(clock::now() - t0).count() >
               timeout_ns;
    };
    volatile uint32_t *done_seq = e->ctl_h + kTcLanes;
    uint32_t seq;
    int slot;
    {
        std::unique_lock<std::mutex> lk(e->mu);
        seq = e->published[lane];
        slot = lane * kTcRing + (int)(seq % kTcRing);
        // the slot's previous job must have completed before it is rewritten
        while (seq >= (uint32_t)kTcRing && done_seq[slot] != seq - kTcRing) {
            if (late()) fail(HK_ETIMEOUT, "served scan: ring slot %d still busy", slot);
            if (!engine_running(e)) engine_launch(e);
            lk.unlock();
            std::this_thread::sleep_for(std::chrono::microseconds(20));
            lk.lock();
        }
        TcJob j{};
        j.args = a;
        j.args.stats = nullptr;      // per-launch counters do not apply to a shared launch
        j.args.work_ctr = nullptr;
        j.total = items;
        j.seq = seq;
        HK_CHECK_CUDA(cudaMemcpyAsync(e->jobs.p + slot, &j, sizeof(j), cudaMemcpyHostToDevice, e->pub));
        HK_CHECK_CUDA(cudaMemsetAsync(e->done.p + slot, 0, sizeof(int32_t), e->pub));
        HK_CHECK_CUDA(cudaStreamSynchronize(e->pub));
        std::atomic_thread_fence(std::memory_order_seq_cst);
        e->published[lane] = seq + 1;
        *(volatile uint32_t *)(e->ctl_h + lane) = seq + 1;
        e->st.jobs += 1;
        if (engine_running(e)) {
            e->st.jobs_inflight += 1;
        } else {
            engine_launch(e);
        }
        engine_note_coll(e, a.Xb);
    }
    for (int spin = 0;; ++spin) {
        if (done_seq[slot] == seq) break;
        if (late()) fail(HK_ETIMEOUT, "served scan: job %u not finished in time", seq);
        if (!engine_running(e)) {
            std::lock_guard<std::mutex> lk(e->mu);
            if (done_seq[slot] != seq && !engine_running(e)) {
                // the launch left without finishing this job: an aborted CTA
                // (a bounded wait ran out) leaves its error word set
                int32_t err = 0;
                HK_CHECK_CUDA(cudaMemcpyAsync(&err, a.err, sizeof(int32_t), cudaMemcpyDeviceToHost, e->pub));
                HK_CHECK_CUDA(cudaStreamSynchronize(e->pub));
                if (err) fail(HK_ETIMEOUT, "served scan: a bounded wait ran out (flag %d)", err);
                engine_launch(e);   // it went idle before this job was published
            }
        }
        // spin (yielding) through short jobs, then sleep between looks
        if (spin < 4096)
            std::this_thread::yield();
        else
            std::this_thread::sleep_for(std::chrono::microseconds(20));
    }
    std::atomic_thread_fence(std::memory_order_seq_cst);
}

double tc_abs_unit(int fmt) {
    // half the spacing of the format's subnormals
    return std::ldexp(1.0, fmt == kFmtBF16 ? -134 : -25);
}

void launch_make_16(const float *X, int64_t N, int n, int64_t Npad, int fmt, void *Xb, void *xq,
                    int *bad, cudaStream_t s) {
    int dev = 0, sms = 0;
    HK_CHECK_CUDA(cudaGetDevice(&dev));
    HK_CHECK_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    k_make_16<<<sms * 16, 256, 0, s>>>(X, N, n, Npad, fmt, reinterpret_cast<uint16_t *>(Xb),
                                       reinterpret_cast<float2 *>(xq), bad);
    HK_CHECK_LAUNCH();
}

void launch_tc_qprep(const float *Q, int nq, int n, int fmt, double xn_max, void *Qb, float *q2e,
                     float *qa, float *qoff2, int *bad, cudaStream_t s) {
    k_tc_qprep<<<nq, 128, 0, s>>>(Q, nq, n, fmt, tc_error_coefficient(n, fmt), tc_abs_unit(fmt), xn_max,
                                  reinterpret_cast<uint16_t *>(Qb), q2e, qa, qoff2, bad);
    HK_CHECK_LAUNCH();
}

__global__ void k_max_norm(const float2 *__restrict__ xq, int64_t N, unsigned *__restrict__ out) {
    float m = 0.f;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N;
         i += (int64_t)gridDim.x * blockDim.x)
        m = fmaxf(m, xq[i].y);
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out, __float_as_uint(m));
}

void launch_max_norm(const void *xq, int64_t N, unsigned *out, cudaStream_t s) {
    k_max_norm<<<256, 256, 0, s>>>(reinterpret_cast<const float2 *>(xq), N, out);
    HK_CHECK_LAUNCH();
}

void launch_tc_rescore(const float *Q, const float *X, int n, int nq, const int32_t *cand_cnt,
                       const int32_t *cand_p, const float *cand_lb, int cand_C, const uint32_t *U,
                       float *pool_d, int32_t *pool_p, int32_t *pool_cnt, int pool_C, int32_t *qflag,
                       long long *stats, int stat_slot, int32_t *items, int32_t *item_off,
                       DevBuf<int32_t> &scan_tmp, cudaStream_t s) {
    k_rescore_items<<<(nq + 255) / 256, 256, 0, s>>>(cand_cnt, nq, cand_C, items);
    HK_CHECK_LAUNCH();
    exclusive_scan_i32(items, item_off, nq, s, scan_tmp);
    int dev = 0, sms = 0;
    HK_CHECK_CUDA(cudaGetDevice(&dev));
    HK_CHECK_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    k_tc_rescore<<<sms * 8, 256, 0, s>>>(Q, X, n, nq, item_off, cand_cnt, cand_p, cand_lb, cand_C, U,
                                         pool_d, pool_p, pool_cnt, pool_C, qflag, stats, stat_slot);
    HK_CHECK_LAUNCH();
}

}  // namespace hk
