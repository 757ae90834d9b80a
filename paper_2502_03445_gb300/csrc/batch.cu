// Batched persistent launch: many independent reconstructions (plans of
// uneven sizes) drained by one persistent kernel from a device work list.
//
// Work items, in dependency levels: ingest chunks of every plan's leaf
// operands, then the tiles of each pairwise step (CUDA-core tiles, 64 x 64
// or the small-K form, or tensor-core 128 x BN tiles).  Every item names at most two counters it
// waits for (its operands' producers) and one it increments.  CTAs claim
// items in list order with an atomic counter, so an item only ever waits for
// items already claimed by running CTAs: no co-residency is needed, and the
// launch is stream-ordered and capturable in a CUDA graph.  Every wait is
// bounded (about one second); a wait that gives up raises an error word that
// tqc_batch_status reports, and the remaining CTAs stop at their next item.
//
// One CTA per SM: tensor-core items (ranges of 16 tiles of one step) run
// through a producer / MMA / direct-epilogue pipeline like the standalone
// step kernel's; CUDA-core items are taken by four 4-warp groups.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "device_common.cuh"
#include "launch.h"
#include "smallk.cuh"

struct tqc_plan {
    tqc::Plan p;
};

namespace tqc {
namespace {

constexpr int BT = 576;                    // 18 warps: producer, MMA issuer, 16 epilogue / worker warps
constexpr int EPIW = 16;
constexpr int EPI = 32 * EPIW;
constexpr long long BWAIT = 2000000000ll;  // ~1 s at the boost clock
constexpr int64_t CHUNK = 1 << 16;          // ingest elements per item
constexpr int RING = 196608;               // operand ring (tensor-core items) / worker buffers (CUDA-core items)
constexpr int MAXST = 16;
constexpr int BM = 128;

enum ItemKind { IT_INGEST = 0, IT_STEP = 1, IT_STALL = 2 };

struct alignas(128) BStep {
    CUtensorMap maps[4];  // A, B, A lo, B lo (tensor-core steps)
    StepArgs a;
    int32_t klass, prec, bn, k_blocks, bres;
    int32_t gmode;        // CUDA-core tiles: gather mode of the staged write-out
    int32_t smallk;       // CUDA-core tiles of the small-K form (smallk.cuh), with
    SmallkLayout sk;      // its write-out layout
    int64_t col_tiles;
    int32_t dep[2];
    int64_t need[2];
    int32_t done;
};

struct BIngest {
    IngestArgs g;
    int64_t lo, hi;
    int32_t done;
};

struct BItem {
    int32_t kind, idx;
    int64_t tile, count;  // a range of tiles of one step
};

// CUDA-core worker group: 4 warps, one 64 x 64 tile at a time
constexpr int G_BK = 16, G_PA = 68, G_PB = 68, G_PS = 68;
constexpr int G_STAGE = G_BK * (G_PA + G_PB) * 4;
constexpr int G_TABLES = 2 * G_STAGE + 64 * G_PS * 4;  // the step's write-out tables, copied per item
constexpr int G_BYTES = G_TABLES + (int)sizeof(EpiTables);
static_assert(4 * G_BYTES <= RING, "worker buffers alias the ring");
static_assert(SMALLK_BYTES <= G_TABLES, "a small-K tile fits a worker buffer");

constexpr int SM_MISC = 2048;
constexpr int SMEM = 1024 + RING + SM_MISC;

__device__ __forceinline__ uint32_t s_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void bmbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(s_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ bool bmbar_try(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(s_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait for a phase; gives up (raising the CTA's abort flag) after
// about a second or when another role already gave up.
__device__ __forceinline__ bool bmbar_wait(uint64_t *bar, uint32_t parity, volatile int *abort_flag) {
    const long long t0 = clock64();
    while (!bmbar_try(bar, parity)) {
        if (*abort_flag) return false;
        if (clock64() - t0 > BWAIT) {
            *abort_flag = 1;
            return false;
        }
    }
    return true;
}
__device__ __forceinline__ void bmbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(s_u32(bar)) : "memory");
}
__device__ __forceinline__ void bmbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(s_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void btma_load(void *dst, const CUtensorMap *map, int c0, int c1, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            s_u32(dst)),
        "l"((uint64_t)map), "r"(c0), "r"(c1), "r"(s_u32(bar))
        : "memory");
}
__device__ __forceinline__ void btma_load3(void *dst, const CUtensorMap *map, int c0, int c1, int c2, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::
            "r"(s_u32(dst)),
        "l"((uint64_t)map), "r"(c0), "r"(c1), "r"(c2), "r"(s_u32(bar))
        : "memory");
}
// One k-block of an operand from element kel of K and row `row`; K-blocked
// operands ([K / 64][rows][64]) are addressed as (kel mod 64, row, kel / 64).
__device__ __forceinline__ void btma_op(void *dst, const CUtensorMap *map, int kel, int row, uint64_t *bar,
                                        bool kblk) {
    if (kblk) btma_load3(dst, map, kel & 63, row, kel >> 6, bar);
    else btma_load(dst, map, kel, row, bar);
}
__device__ __forceinline__ void bcommit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(s_u32(bar))
                 : "memory");
}

__device__ __forceinline__ unsigned long long ld_acquire(const unsigned long long *p) {
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

// Bounded wait for counter >= need (thread 0 only).
__device__ bool wait_counter(const unsigned long long *c, unsigned long long need, const int *err) {
    const long long t0 = clock64();
    while (ld_acquire(c) < need) {
        if (*(volatile const int *)err) return false;
        if (clock64() - t0 > BWAIT) return false;
        __nanosleep(200);
    }
    return true;
}

__device__ __forceinline__ void tc_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void bar_sync(int id, int n) { asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory"); }

__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
    uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)1 << 16;
    d |= (uint64_t)(1024 >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;
    return d;
}

__device__ __forceinline__ void mma_issue(int prec, uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    if (prec == TQC_PREC_TF32)
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
            "l"(a), "l"(b), "r"(idesc), "r"(acc));
    else
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
            "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

// 16 accumulator columns of the warp's 32 TMEM lanes (16 values in
// registers keep the epilogue warps under their 96-register share)
__device__ __forceinline__ void tmem_load16(uint32_t taddr, uint32_t (&r)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// The elements it.lo + tid + k nt of an ingest chunk.  nt (512) is a power
// of two and it.lo a multiple of it, so a thread's elements share their low
// log2(nt) bits: that part of the source offset is summed once.
__device__ void ingest_range(const BIngest &it, int tid, int nt) {
    const IngestArgs &g = it.g;
    const int lg = __ffs(nt) - 1;
    const int64_t d0 = it.lo + tid;
    int64_t s_lo = g.src_base;
    for (int b = 0; b < g.nbits && b < lg; ++b)
        if (d0 >> b & 1) s_lo += 1ll << g.srcpos[b];
    for (int64_t d = d0; d < it.hi; d += nt) {
        int64_t s = s_lo;
        for (int b = lg; b < g.nbits; ++b)
            if (d >> b & 1) s += 1ll << g.srcpos[b];
        const double v64 = g.src_dtype == TQC_F64 ? ((const double *)g.src)[s] : (double)((const float *)g.src)[s];
        if (g.scaled) {
            ((float *)g.dst)[d] = (float)(v64 * g.zinfo[1]);
            continue;
        }
        const float v = (float)v64;
        switch (g.storage) {
            case ST_F32: ((float *)g.dst)[d] = v; break;
            case ST_TF32: ((float *)g.dst)[d] = to_tf32(v); break;
            case ST_BF16: ((__nv_bfloat16 *)g.dst)[d] = __float2bfloat16_rn(v); break;
            case ST_BF16X2: {  // the standalone ingest's split, from the FP32 value
                const __nv_bfloat16 h = __float2bfloat16_rn(v);
                ((__nv_bfloat16 *)g.dst)[d] = h;
                ((__nv_bfloat16 *)g.dst_lo)[d] = __float2bfloat16_rn(v - __bfloat162float(h));
            } break;
            default: break;
        }
    }
}

__device__ __forceinline__ void cp_async4(float *dst, const float *src, bool valid) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(s_u32(dst)), "l"(src), "r"(valid ? 4 : 0)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// Issue the copies of one K chunk of a 64 x 64 tile's operands into a stage
// (A transposed to [k][row], B to [k][col]; rows / columns past the step's
// extent read as zeros).
__device__ __forceinline__ void simt_load(const BStep &st, int64_t tile, int64_t k0, float *stage, int gt) {
    const StepArgs &a = st.a;
    const EpiParams &e = a.epi;
    const int Me = 1 << e.a_bits, Ne = 1 << e.b_bits;
    const int64_t K = 1ll << a.kb;
    const int lkc = a.kb < 4 ? a.kb : 4, kc = 1 << lkc;
    const float *A = (const float *)a.A, *B = (const float *)a.B;
    const int64_t rt = tile / st.col_tiles, ct = tile - rt * st.col_tiles;
    const int64_t r0 = rt << e.a_bits, c0 = ct << e.b_bits;
    float *As = stage, *Bs = stage + G_BK * G_PA;
    for (int idx = gt; idx < (64 << lkc); idx += 128) {
        const int i = idx >> lkc, kk = idx & (kc - 1);
        cp_async4(&As[kk * G_PA + i], A + (i < Me ? (r0 + i) * K + k0 + kk : 0), i < Me);
    }
    for (int idx = gt; idx < (64 << lkc); idx += 128) {
        const int j = idx >> lkc, kk = idx & (kc - 1);
        cp_async4(&Bs[kk * G_PB + j], B + (j < Ne ? (c0 + j) * K + k0 + kk : 0), j < Ne);
    }
}

// The tiles t0, t0 + 4, ... < t_end of one CUDA-core step, computed by one
// 4-warp group (named barrier `bid`, 128 threads, gt = thread index in the
// group): 64 x 64 tiles, 4 x 8 results per thread, staged row-major and
// written in destination order.  The first K chunk of the next tile is
// copied (cp.async) into the other stage while the current tile computes and
// writes out.
__device__ void simt_range(const BStep &st, const EpiTables *tb, int64_t t0, int64_t t_end, uint8_t *buf, int bid,
                           int gt) {
    constexpr int TM = 4, TN = 8;
    const StepArgs &a = st.a;
    const EpiParams &e = a.epi;
    float *stage[2] = {(float *)buf, (float *)(buf + G_STAGE)};
    float *stg = (float *)(buf + 2 * G_STAGE);
    const int Me = 1 << e.a_bits, Ne = 1 << e.b_bits;
    const int64_t K = 1ll << a.kb;
    const int lkc = a.kb < 4 ? a.kb : 4, kc = 1 << lkc;
    const int tx = gt % 8, ty = gt / 8;
    if (t0 < t_end) simt_load(st, t0, 0, stage[0], gt);
    cp_async_commit();
    int cur = 0;
    for (int64_t tile = t0; tile < t_end; tile += 4, cur ^= 1) {
        const bool pre = tile + 4 < t_end;
        if (pre) simt_load(st, tile + 4, 0, stage[cur ^ 1], gt);
        cp_async_commit();
        cp_async_wait<1>();  // everything but the prefetch just issued
        bar_sync(bid, 128);
        float acc[TM][TN];
#pragma unroll
        for (int u = 0; u < TM; ++u)
#pragma unroll
            for (int v = 0; v < TN; ++v) acc[u][v] = 0.f;
        for (int64_t k0 = 0; k0 < K; k0 += kc) {
            float *As = stage[cur], *Bs = As + G_BK * G_PA;
            if (k0 > 0) {  // further K chunks: loaded in place, synchronously
                bar_sync(bid, 128);
                simt_load(st, tile, k0, stage[cur], gt);
                cp_async_commit();
                cp_async_wait<0>();
                bar_sync(bid, 128);
            }
            for (int kk = 0; kk < kc; ++kk) {
                float af[TM], bf[TN];
#pragma unroll
                for (int u = 0; u < TM; ++u) af[u] = As[kk * G_PA + ty * TM + u];
#pragma unroll
                for (int v = 0; v < TN; v += 4) *(float4 *)&bf[v] = *(const float4 *)&Bs[kk * G_PB + tx * TN + v];
#pragma unroll
                for (int u = 0; u < TM; ++u)
#pragma unroll
                    for (int v = 0; v < TN; ++v) acc[u][v] = fmaf(af[u], bf[v], acc[u][v]);
            }
        }
#pragma unroll
        for (int u = 0; u < TM; ++u)
#pragma unroll
            for (int v = 0; v < TN; v += 4)
                *(float4 *)&stg[(ty * TM + u) * G_PS + tx * TN + v] =
                    make_float4(acc[u][v], acc[u][v + 1], acc[u][v + 2], acc[u][v + 3]);
        bar_sync(bid, 128);
        const int64_t rt = tile / st.col_tiles, ct = tile - rt * st.col_tiles;
        epi_readout(tb, stg, e, tile_base(e, (uint64_t)rt, (uint64_t)ct), Me * Ne, gt, 128, st.gmode);
        bar_sync(bid, 128);
    }
    cp_async_wait<0>();
}

// Shared control block of the CTA (after the ring).
struct Ctl {
    uint64_t full[MAXST], empty[MAXST];
    uint64_t tfull[2], tempty[2], bfull, drain;
    uint32_t tmem;
    int abort_flag;
    int64_t item;
    int ok;
};

// One CTA per SM drains the work list.  A tensor-core item is a range of
// tiles of one step, run through the same pipeline as the standalone kernel:
// warp 0 loads k-blocks with TMA into a ring of stages, warp 1 issues
// tcgen05.mma into one of two TMEM accumulators, and the 16 other warps load
// each accumulator and store it straight to the result layout.  Every stage
// keeps its own phase bits, so items of different stage sizes restart the
// ring at stage 0.  A CUDA-core item is a range of tiles (64 x 64, or the
// small-K form of smallk.cuh) taken by four 4-warp groups; an ingest item a
// range of leaf elements.  Between items the whole CTA synchronises: the
// ring and the group buffers share memory.
__global__ void __launch_bounds__(BT, 1)
    batch_kernel(const BItem *items, int64_t n_items, const BStep *steps, const EpiTables *tables, const BIngest *ing,
                 unsigned long long *counters, unsigned long long *next, int *err) {
    extern __shared__ uint8_t raw[];
    uint8_t *sm = (uint8_t *)(((uintptr_t)raw + 1023) & ~(uintptr_t)1023);
    uint8_t *ring = sm;
    Ctl *ctl = (Ctl *)(sm + RING);
    volatile int *abort_flag = &ctl->abort_flag;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (tid == 0) {
        for (int s = 0; s < MAXST; ++s) {
            bmbar_init(&ctl->full[s], 1);
            bmbar_init(&ctl->empty[s], 1);
        }
        for (int a = 0; a < 2; ++a) {
            bmbar_init(&ctl->tfull[a], 1);
            bmbar_init(&ctl->tempty[a], EPIW);
        }
        bmbar_init(&ctl->bfull, 1);
        bmbar_init(&ctl->drain, 1);
        ctl->abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(s_u32(&ctl->tmem))
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_before();
    __syncthreads();
    tc_after();
    const uint32_t tmem = ctl->tmem;
    // role state that persists across items
    uint32_t used = 0, eph = 0, fph = 0;  // producer: stage used / empty phase bits; MMA: full phase bits
    uint32_t bph = 0;                     // resident-B phase (producer and MMA)
    int64_t lt = 0;                       // accumulator sequence (MMA and epilogue)
    bool issued = false;                  // MMA: anything to drain at exit
    for (;;) {
        if (tid == 0) {
            const int64_t it = (*(volatile int *)err || *abort_flag) ? n_items : (int64_t)atomicAdd(next, 1ull);
            int ok = 1;
            if (it < n_items) {
                const BItem item = items[it];
                if (item.kind == IT_STALL) {
                    ok = wait_counter(&counters[item.idx], 1ull, err) ? 1 : 0;  // nothing increments it
                } else if (item.kind == IT_STEP) {
                    const BStep &st = steps[item.idx];
                    for (int d = 0; d < 2 && ok; ++d)
                        if (st.dep[d] >= 0 && !wait_counter(&counters[st.dep[d]], (unsigned long long)st.need[d], err))
                            ok = 0;
                    if (ok && st.klass == KC_UMMA) asm volatile("fence.proxy.async.global;" ::: "memory");
                }
                if (!ok) atomicExch(err, 1);
            }
            ctl->item = it;
            ctl->ok = ok;
        }
        __syncthreads();
        const int64_t it = ctl->item;
        if (it >= n_items) break;
        const BItem item = items[it];
        const bool run = ctl->ok && item.kind != IT_STALL;
        if (run && item.kind == IT_INGEST) {
            if (warp >= 2) ingest_range(ing[item.idx], tid - 64, EPI);
        } else if (run && steps[item.idx].klass != KC_UMMA) {
            if (warp >= 2) {
                const int g = (warp - 2) >> 2, gt = (tid - 64) & 127;
                uint8_t *buf = ring + g * G_BYTES;
                // the tables sit in shared memory while the group uses them
                EpiTables *tb = (EpiTables *)(buf + G_TABLES);
                const uint4 *src = (const uint4 *)&tables[item.idx];
                for (int i = gt; i < (int)(sizeof(EpiTables) / 16); i += 128) ((uint4 *)tb)[i] = src[i];
                bar_sync(2 + g, 128);
                const BStep &st = steps[item.idx];
                if (st.smallk)
                    smallk_dispatch<true>(st.a, tb, st.sk, st.col_tiles, item.tile + g, item.tile + item.count, 4,
                                          (float *)buf, gt, 2 + g);
                else
                    simt_range(st, tb, item.tile + g, item.tile + item.count, buf, 2 + g, gt);
            }
        } else if (run) {
            const BStep &st = steps[item.idx];
            const bool x3 = st.prec == TQC_PREC_BF16X3;
            const int planes = x3 ? 2 : 1;
            const int a_bytes = BM * 128, b_bytes = st.bn * 128;
            const int sbytes = st.bres ? planes * a_bytes : planes * (a_bytes + b_bytes);
            const int nfit = (RING - (st.bres ? planes * b_bytes : 0)) / sbytes;
            const int nst = nfit < MAXST ? nfit : MAXST;
            uint8_t *bsm = ring + RING - planes * b_bytes;
            const int bk = st.prec == TQC_PREC_TF32 ? 32 : 64;
            const bool kblk = st.a.kblk != 0;
            const int64_t t_end = item.tile + item.count;
            if (warp == 0) {
                // ---------------------------------------- TMA producer
                if (lane == 0) {
                    if (st.bres) {
                        bmbar_expect_tx(&ctl->bfull, (uint32_t)(planes * b_bytes));
                        btma_op(bsm, &st.maps[1], 0, 0, &ctl->bfull, kblk);
                        if (x3) btma_op(bsm + b_bytes, &st.maps[3], 0, 0, &ctl->bfull, kblk);
                    }
                    int s = 0;
                    for (int64_t tile = item.tile; tile < t_end && !*abort_flag; ++tile) {
                        const int rt = (int)(tile / st.col_tiles), ct = (int)(tile - (int64_t)rt * st.col_tiles);
                        for (int kb = 0; kb < st.k_blocks; ++kb) {
                            if (used >> s & 1) {
                                if (!bmbar_wait(&ctl->empty[s], eph >> s & 1, abort_flag)) break;
                                eph ^= 1u << s;
                            }
                            used |= 1u << s;
                            uint8_t *sa = ring + s * sbytes;
                            bmbar_expect_tx(&ctl->full[s], (uint32_t)sbytes);
                            btma_op(sa, &st.maps[0], kb * bk, rt * BM, &ctl->full[s], kblk);
                            if (st.bres) {
                                if (x3) btma_op(sa + a_bytes, &st.maps[2], kb * bk, rt * BM, &ctl->full[s], kblk);
                            } else {
                                btma_op(sa + a_bytes, &st.maps[1], kb * bk, ct * st.bn, &ctl->full[s], kblk);
                                if (x3) {
                                    btma_op(sa + a_bytes + b_bytes, &st.maps[2], kb * bk, rt * BM, &ctl->full[s], kblk);
                                    btma_op(sa + 2 * a_bytes + b_bytes, &st.maps[3], kb * bk, ct * st.bn, &ctl->full[s],
                                            kblk);
                                }
                            }
                            s = s + 1 == nst ? 0 : s + 1;
                        }
                    }
                }
            } else if (warp == 1) {
                // ---------------------------------------- MMA issuer
                if (lane == 0) {
                    const uint32_t idesc = (1u << 4) | ((st.prec == TQC_PREC_TF32 ? 2u : 1u) << 7) |
                                           ((st.prec == TQC_PREC_TF32 ? 2u : 1u) << 10) |
                                           ((uint32_t)(st.bn >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
                    bool ok = true;
                    if (st.bres) {
                        ok = bmbar_wait(&ctl->bfull, bph, abort_flag);
                        tc_after();
                    }
                    int s = 0;
                    for (int64_t tile = item.tile; ok && tile < t_end; ++tile, ++lt) {
                        const int acc = (int)(lt & 1);
                        if (!bmbar_wait(&ctl->tempty[acc], (uint32_t)(((lt >> 1) & 1) ^ 1), abort_flag)) break;
                        tc_after();
                        const uint32_t d = tmem + (uint32_t)(acc * 256);
                        for (int kb = 0; kb < st.k_blocks; ++kb) {
                            if (!bmbar_wait(&ctl->full[s], fph >> s & 1, abort_flag)) {
                                ok = false;
                                break;
                            }
                            fph ^= 1u << s;
                            tc_after();
                            const uint32_t a0 = s_u32(ring + s * sbytes);
                            const uint32_t b0 = st.bres ? s_u32(bsm) : a0 + (uint32_t)a_bytes;
                            const uint32_t al = st.bres ? a0 + (uint32_t)a_bytes : b0 + (uint32_t)b_bytes;
                            const uint32_t bl = st.bres ? b0 + (uint32_t)b_bytes : al + (uint32_t)a_bytes;
#pragma unroll
                            for (int k = 0; k < 4; ++k) {
                                const uint64_t da = sw128_desc(a0 + 32 * k), db = sw128_desc(b0 + 32 * k);
                                mma_issue(st.prec, d, da, db, idesc, (kb | k) != 0);
                                if (x3) {
                                    mma_issue(st.prec, d, da, sw128_desc(bl + 32 * k), idesc, 1u);
                                    mma_issue(st.prec, d, sw128_desc(al + 32 * k), db, idesc, 1u);
                                }
                            }
                            bcommit(&ctl->empty[s]);
                            issued = true;
                            s = s + 1 == nst ? 0 : s + 1;
                        }
                        if (!ok) break;
                        bcommit(&ctl->tfull[acc]);
                    }
                    if (st.bres) bph ^= 1u;
                }
            } else {
                // ---------------------------------------- direct epilogue
                const EpiParams &e = st.a.epi;
                const int q = (warp - 2) >> 2, lane_grp = warp & 3;
                const int row = lane_grp * 32 + lane;
                const int Me = 1 << e.a_bits, Ne = 1 << e.b_bits;
                const int subs = st.bn / 64;
                const uint64_t grow = pdep64((uint64_t)pdep32((uint32_t)row, e.lowRc), e.tileMask);
                const uint64_t colmask = pdep64((uint64_t)e.lowCc, e.tileMask);
                const bool full = Me == BM && Ne == 64;
                const int vw = !full ? 1 : (((e.lowCc & 3u) == 3u && e.L >= 2) ? 4 : ((e.lowCc & 1u) && e.L >= 1 ? 2 : 1));
                const uint64_t mstep = vw == 4 ? colmask & (colmask - 1) & ((colmask & (colmask - 1)) - 1)
                                               : (vw == 2 ? colmask & (colmask - 1) : colmask);
                const double sd = (e.mode == EPI_OUT_F32 || e.mode == EPI_OUT_F64) ? e.zinfo[1] : 1.0;
                const float sf = (float)sd;
                int64_t my_lt = lt;
                for (int64_t tile = item.tile; tile < t_end; ++tile, ++my_lt) {
                    const int acc = (int)(my_lt & 1);
                    if (lane == 0) bmbar_wait(&ctl->tfull[acc], (uint32_t)((my_lt >> 1) & 1), abort_flag);
                    __syncwarp();
                    if (*abort_flag) break;
                    tc_after();
                    const uint64_t rt = (uint64_t)(tile / st.col_tiles);
                    const uint64_t ct = (uint64_t)(tile - (int64_t)rt * st.col_tiles);
                    const uint64_t base = warp_pdep64(rt, e.highR) | warp_pdep64(ct * (uint64_t)subs, e.highC);
                    // this warp's 32-column chunks: q, q + 4, ... below BN (none for
                    // q >= 2 when BN = 64); every warp frees the accumulator once
                    const int nch = q * 32 < st.bn ? (st.bn - q * 32 + 127) / 128 : 0;
                    if (nch == 0) {
                        tc_before();
                        __syncwarp();
                        if (lane == 0) bmbar_arrive(&ctl->tempty[acc]);
                    }
                    // in halves of 16 columns: j0 is a multiple of 16, so the
                    // deposits of j0 and of j < 16 add (disjoint bits)
                    for (int c = 0; c < 2 * nch; ++c) {
                        const int col0 = q * 32 + 128 * (c >> 1) + 16 * (c & 1);
                        uint32_t r[16];
                        tmem_load16(tmem + ((uint32_t)(lane_grp * 32) << 16) + (uint32_t)(acc * 256 + col0), r);
                        if (c == 2 * nch - 1) {
                            tc_before();
                            __syncwarp();
                            if (lane == 0) bmbar_arrive(&ctl->tempty[acc]);
                        }
                        const int j0 = col0 % 64;
                        const uint64_t o = base + grow + pdep64((uint64_t)j0, colmask) +
                                           pdep64((uint64_t)(col0 / 64), e.highC);
                        if (full) {
                            direct_run32_any<16>(e, vw, o, mstep, r, sf, sd);
                        } else if (row < Me && j0 < Ne) {
                            uint64_t x = 0;
                            const int nc = Ne - j0 < 16 ? Ne - j0 : 16;
                            for (int j = 0; j < nc; ++j) {
                                const float v = __uint_as_float(r[j]);
                                store_run_f32(e, o + x, &v, 1, sd);
                                x = ((x | ~colmask) + 1) & colmask;
                            }
                        }
                    }
                }
            }
            // the accumulator sequence advances by the item's tiles in every role
            if (warp != 1) lt += item.count;
        }
        // the ring and the group buffers share memory: order generic writes
        // before the next item's TMA writes, and finish every role first
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __threadfence();
        __syncthreads();
        if (tid == 0) {
            if (*abort_flag) atomicExch(err, 1);
            else if (run) atomicAdd(&counters[item.kind == IT_INGEST ? ing[item.idx].done : steps[item.idx].done], 1ull);
        }
    }
    if (warp == 1 && lane == 0 && issued) {
        // every MMA issued so far has completed once this commit arrives
        bcommit(&ctl->drain);
        const long long t0 = clock64();
        while (!bmbar_try(&ctl->drain, 0) && clock64() - t0 < BWAIT) {
        }
    }
    tc_before();
    __syncthreads();
    if (warp == 1) {
        tc_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem) : "memory");
    }
}

// ------------------------------------------------------------------ host side
uint64_t h_pdep(uint64_t src, uint64_t mask) {
    uint64_t r = 0;
    while (mask) {
        uint64_t low = mask & (~mask + 1);
        if (src & 1) r |= low;
        src >>= 1;
        mask ^= low;
    }
    return r;
}
uint32_t h_pext(uint32_t x, uint32_t mask) {
    uint32_t r = 0, k = 0;
    while (mask) {
        uint32_t low = mask & (~mask + 1);
        if (x & low) r |= 1u << k;
        ++k;
        mask ^= low;
    }
    return r;
}

void host_tables(EpiTables *tb, const EpiParams &e, bool rowmajor, int pitch) {
    for (int u = 0; u < 384; ++u) {
        const bool lo = u < 128;
        const uint32_t t = lo ? (uint32_t)u : (uint32_t)(u - 128) << 7;
        const uint32_t i = h_pext(t, e.lowRc), j = h_pext(t, e.lowCc);
        const uint32_t s = rowmajor ? i * pitch + j : j * pitch + i;
        const uint64_t g = h_pdep(t, e.tileMask);
        if (lo) {
            tb->s_lo[u] = s;
            tb->g_lo[u] = g;
        } else {
            tb->s_hi[u - 128] = s;
            tb->g_hi[u - 128] = g;
        }
    }
}

// A plan's steps from its first large one on (predicted by the cost model
// to take at least g_tail_s) run after the persistent kernel as ordinary
// step launches: a large step fills the GPU by itself and runs faster in its
// own kernels (all warps of every SM, its own register budget) than as
// items of the persistent kernel, while the small ones gain from sharing it.
struct BatchTail {
    Plan *p;
    size_t first;
    void *out;
};

// The large steps of different plans are independent: they run on a few
// streams forked from the caller's (and joined back before the call
// returns), so one plan's last wave and the gaps between launches overlap
// another plan's steps.  Plans are spread by their predicted time, longest
// first onto the least loaded stream.
constexpr int TAIL_STREAMS = 4;

struct Batch {
    std::vector<const void *> key;
    std::vector<BatchTail> tails;
    std::vector<int> tail_stream;  // stream of each tail
    BItem *d_items = nullptr;
    BStep *d_steps = nullptr;
    EpiTables *d_tables = nullptr;
    BIngest *d_ing = nullptr;
    unsigned long long *d_counters = nullptr;  // [counters..., next]
    int *d_err = nullptr;
    int64_t n_items = 0, n_counters = 0;
    void release() {
        cudaFree(d_items);
        cudaFree(d_steps);
        cudaFree(d_tables);
        cudaFree(d_ing);
        cudaFree(d_counters);
        cudaFree(d_err);
        *this = Batch();
    }
};

std::mutex g_batch_mu;
Batch g_batch;
int g_inject_stall = 0;
double g_tail_s = 16e-6;
// process-wide, created on first use (the tail streams of every device's
// batches; streams and events are per device, so they are created for the
// device current at first use)
cudaStream_t g_tail_ts[TAIL_STREAMS] = {};
cudaEvent_t g_tail_fork = nullptr, g_tail_join[TAIL_STREAMS] = {};
int g_tail_device = -1;

template <typename T>
cudaError_t upload(T **dst, const std::vector<T> &v) {
    if (v.empty()) {
        *dst = nullptr;
        return cudaSuccess;
    }
    cudaError_t e = cudaMalloc((void **)dst, sizeof(T) * v.size());
    if (e != cudaSuccess) return e;
    return cudaMemcpy(*dst, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice);
}

tqc_status build_batch(Plan *const *plans, void *const *outs, int n, Batch *b) {
    std::vector<double> tail_time;  // predicted seconds of each plan's large steps
    std::vector<BItem> items;
    std::vector<BStep> steps;
    std::vector<EpiTables> tables;
    std::vector<BIngest> ing;
    std::vector<int> step_level;
    std::vector<std::pair<int, BItem>> leveled;  // (level, item)
    int n_counters = 0;
    for (int pi = 0; pi < n; ++pi) {
        Plan &p = *plans[pi];
        if (!p.ready) return fail(TQC_ERR_INVALID, "batch: plan " + std::to_string(pi) + " was never contracted");
        if (p.n_slices() > 1) return fail(TQC_ERR_UNSUPPORTED, "batch: plan " + std::to_string(pi) + " is sliced");
        if (p.z_version != p.net->version)
            return fail(TQC_ERR_INVALID, "batch: plan " + std::to_string(pi) + " has changed tensors; contract it once");
        // ingest chunks (all leaves of the plan count on one counter)
        const int ing_counter = n_counters++;
        int64_t n_chunks = 0;
        for (int j = 0; j < p.m; ++j) {
            const TensorPlan &t = p.tensors[j];
            BIngest bi;
            bi.g = exec_leaf_args(p, t, j, p.fixed_bits.data());
            if (p.m == 1) {
                bi.g.dst = outs[pi];
                bi.g.scaled = 1;
                bi.g.zinfo = p.d_zinfo;
            } else {
                bi.g.dst = (char *)p.d_ws + t.offset;
                if (t.storage == ST_BF16X2) bi.g.dst_lo = (char *)p.d_ws + t.offset + t.plane_bytes;
                bi.g.storage = t.storage;
            }
            bi.done = ing_counter;
            const int64_t total = p.m == 1 ? p.out_elems() : ((int64_t)1 << t.nbits());
            for (int64_t lo = 0; lo < total; lo += CHUNK) {
                bi.lo = lo;
                bi.hi = std::min(total, lo + CHUNK);
                leveled.push_back({0, BItem{IT_INGEST, (int)ing.size(), 0, 1}});
                ing.push_back(bi);
                ++n_chunks;
            }
        }
        // steps
        std::vector<int> counter_of(p.tensors.size(), -1), level_of(p.tensors.size(), 0);
        std::vector<int64_t> tiles_of(p.tensors.size(), 0);
        for (int j = 0; j < p.m; ++j) {
            counter_of[j] = ing_counter;
            tiles_of[j] = n_chunks;
        }
        size_t first_tail = p.steps.size();
        const CostConsts cc;
        for (size_t i = 0; i < p.steps.size(); ++i) {
            const StepPlan &sp = p.steps[i];
            if (step_cost(sp.mb, sp.nb, sp.kb, sp.klass, sp.prec, cc).time_s - cc.launch_s >= g_tail_s) {
                first_tail = i;
                break;
            }
        }
        if (first_tail < p.steps.size() && first_tail > 0 && p.steps[first_tail].fuse == 2) --first_tail;
        if (first_tail < p.steps.size()) {
            b->tails.push_back(BatchTail{&p, first_tail, outs[pi]});
            double t = 0;
            for (size_t i = first_tail; i < p.steps.size(); ++i) {
                const StepPlan &sp = p.steps[i];
                t += step_cost(sp.mb, sp.nb, sp.kb, sp.klass, sp.prec, cc).time_s;
            }
            tail_time.push_back(t);
        }
        for (size_t si0 = 0; si0 < first_tail; ++si0) {
            const StepPlan &sp = p.steps[si0];
            BStep bs;
            std::memset((void *)&bs, 0, sizeof bs);
            bs.klass = sp.klass;
            bs.prec = sp.prec;
            const bool smallk = sp.klass != KC_UMMA && sp.tile == SIMT_SMALLK;
            TileShape ts = sp.klass == KC_UMMA ? TileShape{7, 6}
                                               : (smallk ? smallk_tile(sp.mb, sp.nb, sp.kb) : TileShape{6, 6});
            bs.a = exec_step_args(p, sp, ts);
            const TensorPlan &tc = p.tensors[sp.c];
            bs.a.epi.zinfo = p.d_zinfo;
            if (sp.final) {
                bs.a.epi.out = outs[pi];
                bs.a.epi.mode = EPI_OUT_F32;
            } else {
                bs.a.epi.out = (char *)p.d_ws + tc.offset;
                if (tc.storage == ST_BF16X2) bs.a.epi.out_lo = (char *)p.d_ws + tc.offset + tc.plane_bytes;
                bs.a.epi.mode = exec_epi_mode(tc.storage);
            }
            int64_t row_tiles = (int64_t)1 << (sp.mb - bs.a.epi.a_bits);
            int64_t per_item;
            if (sp.klass == KC_UMMA) {
                // the tile width of the plan's own configuration (the autotuner's
                // choice when the plan was tuned), run with the direct epilogue
                const int want = sp.tile == UMMA_128x256_DEEP ? 256 : (sp.tile == UMMA_128x64 ? 64 : 128);
                bs.bn = std::min(want, sp.nb >= 8 ? 256 : (sp.nb >= 7 ? 128 : 64));
                const int lbn = bs.bn == 256 ? 8 : (bs.bn == 128 ? 7 : 6);
                bs.col_tiles = sp.nb >= lbn ? (int64_t)1 << (sp.nb - lbn) : 1;
                bs.k_blocks = (int)(((int64_t)1 << sp.kb) / (sp.prec == TQC_PREC_TF32 ? 32 : 64));
                if (bs.k_blocks < 1) return fail(TQC_ERR_UNSUPPORTED, "batch: tensor-core step with K below one k-block");
                bs.bres = bs.k_blocks == 1 && bs.col_tiles == 1;
                if (umma_make_maps(sp.prec, bs.a, bs.bn, bs.maps) != cudaSuccess)
                    return fail(TQC_ERR_CUDA, "batch: tensor map of plan " + std::to_string(pi));
            } else {
                bs.bn = 64;
                bs.col_tiles = (int64_t)1 << (sp.nb - bs.a.epi.b_bits);
                bs.gmode = gather_mode(bs.a.epi.lowCc);
                if (smallk) {
                    bs.smallk = 1;
                    bs.sk = smallk_layout(bs.a.epi);
                }
            }
            const int64_t n_tiles = row_tiles * bs.col_tiles;
            // items of 16 tiles, larger for large steps (fewer pipeline drains),
            // still about two per SM
            per_item = std::min<int64_t>(128, std::max<int64_t>(16, n_tiles / (2 * (int64_t)sm_count()) / 4 * 4));
            const int64_t n_step_items = (n_tiles + per_item - 1) / per_item;
            bs.dep[0] = counter_of[sp.a];
            bs.need[0] = tiles_of[sp.a];
            bs.dep[1] = counter_of[sp.b];
            bs.need[1] = tiles_of[sp.b];
            if (bs.dep[1] == bs.dep[0]) bs.dep[1] = -1;
            bs.done = n_counters++;
            counter_of[sp.c] = bs.done;
            tiles_of[sp.c] = n_step_items;  // the counter counts finished items
            const int lvl = 1 + std::max(level_of[sp.a], level_of[sp.b]);
            level_of[sp.c] = lvl;
            EpiTables tb;
            // staged write-out of the CUDA-core tiles (64 x 64 row-major, or the small-K form's)
            if (bs.smallk) host_tables(&tb, bs.a.epi, true, 0);  // the gather's element offsets
            else host_tables(&tb, bs.a.epi, true, 68);
            const int si = (int)steps.size();
            steps.push_back(bs);
            tables.push_back(tb);
            for (int64_t t = 0; t < n_tiles; t += per_item)
                leveled.push_back({lvl, BItem{IT_STEP, si, t, std::min(per_item, n_tiles - t)}});
        }
    }
    {
        std::vector<size_t> order(tail_time.size());
        for (size_t i = 0; i < order.size(); ++i) order[i] = i;
        std::stable_sort(order.begin(), order.end(), [&](size_t x, size_t y) { return tail_time[x] > tail_time[y]; });
        double load[TAIL_STREAMS] = {0};
        b->tail_stream.assign(tail_time.size(), 0);
        for (size_t i : order) {
            const int k = (int)(std::min_element(load, load + TAIL_STREAMS) - load);
            b->tail_stream[i] = k;
            load[k] += tail_time[i];
        }
    }
    if (g_inject_stall) leveled.insert(leveled.begin(), {0, BItem{IT_STALL, n_counters++, 0, 0}});
    std::stable_sort(leveled.begin(), leveled.end(), [](auto &x, auto &y) { return x.first < y.first; });
    for (auto &li : leveled) items.push_back(li.second);
    b->n_items = (int64_t)items.size();
    b->n_counters = n_counters;
    cudaError_t e = upload(&b->d_items, items);
    if (e == cudaSuccess) e = upload(&b->d_steps, steps);
    if (e == cudaSuccess) e = upload(&b->d_tables, tables);
    if (e == cudaSuccess) e = upload(&b->d_ing, ing);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_counters, sizeof(unsigned long long) * (n_counters + 1));
    if (e == cudaSuccess) e = cudaMalloc(&b->d_err, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(b->d_err, 0, sizeof(int));
    if (e != cudaSuccess) {
        cudaGetLastError();
        b->release();
        return fail(TQC_ERR_OOM, std::string("batch set-up: ") + cudaGetErrorString(e));
    }
    return TQC_OK;
}

}  // namespace
}  // namespace tqc

using namespace tqc;

extern "C" {

tqc_status tqc_contract_batch(const tqc_plan_t *plans, void *const *d_outs, int32_t n, void *cuda_stream) {
    if (!plans || !d_outs || n < 1) return fail(TQC_ERR_INVALID, "bad batch arguments");
    for (int i = 0; i < n; ++i)
        if (!plans[i] || !d_outs[i]) return fail(TQC_ERR_INVALID, "NULL plan or output in batch");
    std::lock_guard<std::mutex> lk(g_batch_mu);
    // the batch (and every replay of a graph that captured it) rewrites these
    // plans' workspaces: they keep no intermediates across tqc_contract calls
    for (int i = 0; i < n; ++i) plans[i]->p.batched = true;
    std::vector<const void *> key;
    for (int i = 0; i < n; ++i) {
        key.push_back(plans[i]);
        key.push_back(d_outs[i]);
    }
    key.push_back((const void *)(intptr_t)g_inject_stall);
    key.push_back((const void *)(intptr_t)(int64_t)(std::min(g_tail_s, 1e6) * 1e9));
    if (key != g_batch.key) {
        g_batch.release();
        std::vector<Plan *> ps;
        for (int i = 0; i < n; ++i) ps.push_back(&plans[i]->p);
        tqc_status st = build_batch(ps.data(), d_outs, n, &g_batch);
        if (st != TQC_OK) return st;
        g_batch.key = key;
        static bool attr = false;
        if (!attr) {
            if (cudaFuncSetAttribute(batch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM) != cudaSuccess)
                return fail(TQC_ERR_CUDA, "batch kernel attributes");
            attr = true;
        }
    }
    cudaStream_t s = (cudaStream_t)cuda_stream;
    cudaError_t e = cudaMemsetAsync(g_batch.d_counters, 0, sizeof(unsigned long long) * (g_batch.n_counters + 1), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(g_batch.d_err, 0, sizeof(int), s);
    if (e != cudaSuccess) return fail(TQC_ERR_CUDA, std::string("batch reset: ") + cudaGetErrorString(e));
    const int grid = sm_count();
    batch_kernel<<<grid, BT, SMEM, s>>>(g_batch.d_items, g_batch.n_items, g_batch.d_steps, g_batch.d_tables,
                                        g_batch.d_ing, g_batch.d_counters, g_batch.d_counters + g_batch.n_counters,
                                        g_batch.d_err);
    e = cudaGetLastError();
    if (e != cudaSuccess) return fail(TQC_ERR_CUDA, std::string("batch launch: ") + cudaGetErrorString(e));
    if (g_batch.tails.empty()) return TQC_OK;
    int dev = 0;
    cudaGetDevice(&dev);
    if (g_tail_device != dev) {
        if (g_tail_device >= 0) return fail(TQC_ERR_UNSUPPORTED, "batched launches on a second device");
        for (int k = 0; k < TAIL_STREAMS && e == cudaSuccess; ++k) {
            e = cudaStreamCreateWithFlags(&g_tail_ts[k], cudaStreamNonBlocking);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&g_tail_join[k], cudaEventDisableTiming);
        }
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&g_tail_fork, cudaEventDisableTiming);
        if (e != cudaSuccess) return fail(TQC_ERR_CUDA, std::string("batch tail streams: ") + cudaGetErrorString(e));
        g_tail_device = dev;
    }
    // fork: every tail stream waits for the persistent kernel
    e = cudaEventRecord(g_tail_fork, s);
    for (int k = 0; k < TAIL_STREAMS && e == cudaSuccess; ++k) e = cudaStreamWaitEvent(g_tail_ts[k], g_tail_fork, 0);
    if (e != cudaSuccess) return fail(TQC_ERR_CUDA, std::string("batch fork: ") + cudaGetErrorString(e));
    tqc_status st = TQC_OK;
    for (size_t i = 0; i < g_batch.tails.size() && st == TQC_OK; ++i) {
        const BatchTail &t = g_batch.tails[i];
        st = exec_run_tail(*t.p, t.first, t.out, g_tail_ts[g_batch.tail_stream[i]]);
    }
    // join (also after a failed launch, so the caller's stream stays ordered)
    for (int k = 0; k < TAIL_STREAMS; ++k) {
        cudaError_t ej = cudaEventRecord(g_tail_join[k], g_tail_ts[k]);
        if (ej == cudaSuccess) ej = cudaStreamWaitEvent(s, g_tail_join[k], 0);
        if (ej != cudaSuccess && st == TQC_OK) st = fail(TQC_ERR_CUDA, std::string("batch join: ") + cudaGetErrorString(ej));
    }
    return st;
}

tqc_status tqc_batch_status(void *cuda_stream) {
    std::lock_guard<std::mutex> lk(g_batch_mu);
    if (!g_batch.d_err) return fail(TQC_ERR_INVALID, "no batch launched");
    int h = 0;
    cudaError_t e = cudaMemcpyAsync(&h, g_batch.d_err, sizeof(int), cudaMemcpyDeviceToHost, (cudaStream_t)cuda_stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize((cudaStream_t)cuda_stream);
    if (e != cudaSuccess) return fail(TQC_ERR_CUDA, std::string("batch status: ") + cudaGetErrorString(e));
    if (h) return fail(TQC_ERR_TIMEOUT, "a bounded wait in the batched launch gave up");
    // the large steps' error words (their plans' own): every one that is set
    // is cleared, so the next call reports only its own
    bool timed_out = false;
    for (const BatchTail &t : g_batch.tails) {
        int w = 0;
        e = cudaMemcpyAsync(&w, t.p->d_zinfo + 2, sizeof(int), cudaMemcpyDeviceToHost, (cudaStream_t)cuda_stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize((cudaStream_t)cuda_stream);
        if (e == cudaSuccess && w) e = cudaMemsetAsync(t.p->d_zinfo + 2, 0, sizeof(int), (cudaStream_t)cuda_stream);
        if (e != cudaSuccess) return fail(TQC_ERR_CUDA, std::string("batch status: ") + cudaGetErrorString(e));
        timed_out = timed_out || w != 0;
    }
    if (timed_out) return fail(TQC_ERR_TIMEOUT, "a tensor-core step of the batch gave up waiting on its pipeline");
    return TQC_OK;
}

tqc_status tqc_batch_launches(int64_t *launches, int64_t *tail_steps) {
    if (!launches) return fail(TQC_ERR_INVALID, "NULL launches");
    std::lock_guard<std::mutex> lk(g_batch_mu);
    if (!g_batch.d_err) return fail(TQC_ERR_INVALID, "no batch launched");
    int64_t n = 1, steps = 0;  // the persistent kernel, then each large step's launches
    for (const BatchTail &t : g_batch.tails)
        for (size_t i = t.first; i < t.p->steps.size(); ++i) {
            const StepPlan &sp = t.p->steps[i];
            ++steps;
            if (sp.fuse == 2) continue;
            n += sp.ksplit > 1 ? 2 : 1;
        }
    *launches = n;
    if (tail_steps) *tail_steps = steps;
    return TQC_OK;
}

tqc_status tqc_batch_tail_threshold(double seconds) {
    if (!(seconds >= 0.0)) return fail(TQC_ERR_INVALID, "threshold must be >= 0");
    std::lock_guard<std::mutex> lk(g_batch_mu);
    g_tail_s = seconds;
    return TQC_OK;
}

tqc_status tqc_batch_inject_stall(int32_t enable) {
    std::lock_guard<std::mutex> lk(g_batch_mu);
    g_inject_stall = enable ? 1 : 0;
    return TQC_OK;
}

}  // extern "C"
