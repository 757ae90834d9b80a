// One tile of a small-K CUDA-core step (K = 1, 4 or 16: one subcircuit pair
// sharing at most two cut edges), computed by a group of 128 threads.
//
// Such a step moves far more bytes than it multiplies: a result element
// costs K multiply-adds and 4 bytes of HBM writes, so the tile is shaped for
// the write-out, not for arithmetic reuse.  It spans a + b = 12 result bits
// (4096 elements; fewer when the step is smaller or the operands would not
// fit the buffer): the lowest a row bits and lowest b column bits of the
// result layout, so that the rows (and columns) it reads are contiguous
// operand memory, loaded with 16-byte loads and stored transposed ([k][row],
// [k][col]) in shared memory.  Every thread then forms 4 x 8 (or 8 x 4)
// results as outer products of float4 quads and writes them to HBM straight
// from registers when the layout allows, else through a staged copy of the
// tile in destination order, gathered 16 bytes at a time (SmallkLayout).
// The staging buffer aliases the operand buffer.
#pragma once

#include "device_common.cuh"
#include "launch.h"

namespace tqc {

// Shared memory of a small-K tile: its operands, or its staged results
// (which alias them).
constexpr int SMALLK_BYTES = 34816;

__host__ __device__ inline int smallk_op_bytes(int a, int b, int kb) {
    return (1 << kb) * ((1 << a) + 4 + (1 << b) + 4) * 4;
}
// The staged tile: 2^(a+b) floats in the tile's destination order.
__host__ __device__ inline int smallk_stage_bytes(int a, int b) { return 4 << (a + b); }

// How a small-K step writes its tiles.  direct: the result's lowest bits
// (at least four) are bits of one dimension of the tile, so each thread's
// float4 quads along that dimension are 16 contiguous bytes and the lanes
// of a warp run along it: results go from registers straight to their
// destination, with no staging.  Otherwise the tile is staged in its own
// destination order: element t of the tile (t = the tile's result bits,
// compacted, lowest first) at word 4 swz(t >> 2) + (t & 3), swz an XOR of
// the 16-byte chunk index that spreads the chunks of a warp's writes over
// the banks.  The two lowest bits of t are two of the four lowest bits of
// the tile's rows and columns, so every aligned four results of the
// destination lie in one thread's 4 x 4 block: the thread writes them as
// one float4 and the gather reads 16 bytes per four results, for any
// layout.  pat says which: 0 rows 0, 1; 1 columns 0, 1; 2 row 0 then column
// 0; 3 column 0 then row 0.  pr0 / pr1 / pc0 / pc1: the bit of t holding
// row bit 0 / 1 and column bit 0 / 1.  rowmajor says which dimension the
// lanes run along (columns when set); qm: row quads per thread (1: 4 x 8
// results, 2: 8 x 4), 2 when the lanes run along rows.
struct SmallkLayout {
    int direct, rowmajor, qm, pat;
    uint32_t pr0, pr1, pc0, pc1;
};

__device__ __forceinline__ uint32_t sk_swz(uint32_t q) { return q ^ (((q >> 3) ^ (q >> 6) ^ (q >> 9)) & 7u); }

// The layout of a step with these epilogue parameters (host; simt.cu).
SmallkLayout smallk_layout(const EpiParams &e);

// Direct stores of a thread's QM x QN quads (output mode MODE): along
// columns (RM) the quad of row i of column quad v goes to base + gr + gc[v],
// gr stepping through the quad's rows by masked increments of mR; along rows
// the quad of column j of row quad u goes to base + gr[u] + gc.
template <int MODE, int QM, int QN, bool RM>
__device__ __forceinline__ void sk_direct_store(const EpiParams &e, const float (&acc)[4 * QM][4 * QN], uint64_t base,
                                                const uint64_t (&gr)[QM], const uint64_t (&gc)[QN], uint64_t mR,
                                                uint64_t mC, float sf, double sd) {
    if constexpr (RM) {
#pragma unroll
        for (int u = 0; u < QM; ++u) {
            uint64_t g = base + gr[u];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
#pragma unroll
                for (int v = 0; v < QN; ++v) {
                    const float w[4] = {acc[4 * u + i][4 * v], acc[4 * u + i][4 * v + 1], acc[4 * u + i][4 * v + 2],
                                        acc[4 * u + i][4 * v + 3]};
                    store_vals<MODE, 4>(e, g + gc[v], w, sf, sd);
                }
                g = (((g - base) | ~mR) + 1 & mR) + base;
            }
        }
    } else {
#pragma unroll
        for (int v = 0; v < QN; ++v) {
            uint64_t g = gc[v];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
#pragma unroll
                for (int u = 0; u < QM; ++u) {
                    const float w[4] = {acc[4 * u][4 * v + j], acc[4 * u + 1][4 * v + j], acc[4 * u + 2][4 * v + j],
                                        acc[4 * u + 3][4 * v + j]};
                    store_vals<MODE, 4>(e, base + gr[u] + g, w, sf, sd);
                }
                g = ((g | ~mC) + 1) & mC;
            }
        }
    }
}

// Stage a thread's 4 QM x 4 QN results in the tile's destination order (the
// layout above).  trq[u] / tcq[v]: the bits of t of the thread's row quad u /
// column quad v (their rows 0..3 / columns 0..3 add the bits pr0, pr1 /
// pc0, pc1).
template <int QM, int QN>
__device__ __forceinline__ void sk_stage(float *stg, const float (&acc)[4 * QM][4 * QN], const SmallkLayout &L,
                                         const uint64_t (&trq)[QM], const uint64_t (&tcq)[QN]) {
    auto put = [&](uint32_t t, float x0, float x1, float x2, float x3) {
        *(float4 *)(stg + (sk_swz(t >> 2) << 2)) = make_float4(x0, x1, x2, x3);
    };
    const uint32_t R0 = 1u << L.pr0, R1 = 1u << L.pr1, C0 = 1u << L.pc0, C1 = 1u << L.pc1;
#pragma unroll
    for (int u = 0; u < QM; ++u)
#pragma unroll
        for (int v = 0; v < QN; ++v) {
            const uint32_t t0 = (uint32_t)(trq[u] | tcq[v]);
            const int r = 4 * u, c = 4 * v;
            if (L.pat == 0) {  // rows 0..3 of one column
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    put(t0 | ((j & 1) ? C0 : 0u) | ((j & 2) ? C1 : 0u), acc[r][c + j], acc[r + 1][c + j],
                        acc[r + 2][c + j], acc[r + 3][c + j]);
            } else if (L.pat == 1) {  // columns 0..3 of one row
#pragma unroll
                for (int i = 0; i < 4; ++i)
                    put(t0 | ((i & 1) ? R0 : 0u) | ((i & 2) ? R1 : 0u), acc[r + i][c], acc[r + i][c + 1],
                        acc[r + i][c + 2], acc[r + i][c + 3]);
            } else {  // 2 x 2 blocks: (row 0, column 0) or (column 0, row 0) lowest
#pragma unroll
                for (int i = 0; i < 4; i += 2)
#pragma unroll
                    for (int j = 0; j < 4; j += 2) {
                        const uint32_t t = t0 | (i ? R1 : 0u) | (j ? C1 : 0u);
                        if (L.pat == 2)
                            put(t, acc[r + i][c + j], acc[r + i + 1][c + j], acc[r + i][c + j + 1],
                                acc[r + i + 1][c + j + 1]);
                        else
                            put(t, acc[r + i][c + j], acc[r + i][c + j + 1], acc[r + i + 1][c + j],
                                acc[r + i + 1][c + j + 1]);
                    }
            }
        }
}

// Write the staged tile (E results) to the destination: thread gt takes
// the aligned fours t = 4 gt + 512 n; element offset of t = g_hi[t >> 7] +
// g_lo[t & 127] (t & 127 fixed per thread).  MODE: the output mode, or -1
// to dispatch it per store (fewer live registers).
template <int MODE>
__device__ __forceinline__ void sk_gather(const EpiTables *tb, const float *stg, const EpiParams &e, uint64_t base,
                                          int E, int gt) {
    const int mode = MODE >= 0 ? MODE : e.mode;
    const double sd = (mode == EPI_OUT_F32 || mode == EPI_OUT_F64) ? e.zinfo[1] : 1.0;
    const float sf = (float)sd;
    const uint64_t gb = base + tb->g_lo[(gt * 4) & 127];
#pragma unroll 4
    for (int t = gt * 4; t < E; t += 512) {
        const float4 q = *(const float4 *)(stg + (sk_swz((uint32_t)t >> 2) << 2));
        const float v[4] = {q.x, q.y, q.z, q.w};
        if constexpr (MODE >= 0) store_vals<MODE, 4>(e, gb + tb->g_hi[t >> 7], v, sf, sd);
        else store_run_f32(e, gb + tb->g_hi[t >> 7], v, 4, sd);
    }
}

__device__ __forceinline__ void sk_bar(int id) { asm volatile("bar.sync %0, 128;" ::"r"(id) : "memory"); }

// Tiles t0, t0 + stride, ... < t_end of a small-K step (col_tiles: a power
// of two).  KB = log2 K; QM x QN float4 quads per thread (1 x 2 or 2 x 1);
// RM: the lanes run along columns.  gt: the thread's index in the group,
// bid: the group's named barrier; tb: the step's element-offset tables (the
// staged form's gather).  Every thread's place in the tile is fixed across
// tiles.
// The tile's row / column block and its base element advance by masked
// additions instead of a division and two bit deposits per tile: with every
// bit outside mask M set, pdep(x, M) + pdep(d, M) carries across the gaps,
// so ((P | ~M) + pdep(d, M)) & M = pdep(x + d, M) (modulo the mask's width:
// the column block wraps and carries into the row block).  LEAN (for a
// caller with a tight register budget, which runs this loop as a call and
// saves its live registers once per call): the tile base is deposited per
// tile and the output mode dispatched per store, which keep fewer values
// live.
template <int KB, int QM, bool RM, bool LEAN>
__device__ __forceinline__ void smallk_tiles_body(const StepArgs &sa, const EpiTables *tb, const SmallkLayout L,
                                                  int64_t col_tiles, int64_t t0, int64_t t_end, int64_t stride,
                                                  float *buf, int gt, int bid) {
    const int direct = L.direct;
    constexpr int K = 1 << KB;
    constexpr int QN = 3 - QM;
    if (t0 >= t_end) return;
    __builtin_assume(__isShared(buf));
    __builtin_assume(__isShared(tb));
    const EpiParams &e = sa.epi;
    const int a = e.a_bits, b = e.b_bits;
    const int Me = 1 << a, Ne = 1 << b;
    const int PA = Me + 4, PB = Ne + 4;
    float *As = buf, *Bs = buf + K * PA;
    float *const stg = buf;  // aliases the operands, read before it is written
    // thread (tx, ty) owns row quads ty + Y u and column quads tx + X v; the
    // lanes of a warp run along the staging buffer's contiguous dimension
    // (columns when it is row-major), so that its float4 writes are
    // conflict-free
    const int lX = b - 2 - (QN - 1), lY = a - 2 - (QM - 1);  // X = 2^lX, Y = 2^lY
    const int tx = RM ? gt & ((1 << lX) - 1) : gt >> lY;
    const int ty = RM ? gt >> lX : gt & ((1 << lY) - 1);
    const bool active = gt < (1 << (lX + lY));
    int oa[QM], ob[QN];
#pragma unroll
    for (int u = 0; u < QM; ++u) oa[u] = 4 * (ty + (u << lY));
#pragma unroll
    for (int v = 0; v < QN; ++v) ob[v] = 4 * (tx + (v << lX));
    // direct stores: element offsets (in the tile) of the thread's first row
    // of each row quad and first column of each column quad; the rows and
    // columns within a quad follow by masked increments
    const uint64_t mR = pdep64(e.lowRc, e.tileMask), mC = pdep64(e.lowCc, e.tileMask);
    // (staged form: the same arrays hold the bits of t of the thread's quads)
    uint64_t gr[QM], gc[QN];
#pragma unroll
    for (int u = 0; u < QM; ++u) gr[u] = direct ? pdep64((uint64_t)oa[u], mR) : pdep32((uint32_t)oa[u], e.lowRc);
#pragma unroll
    for (int v = 0; v < QN; ++v) gc[v] = direct ? pdep64((uint64_t)ob[v], mC) : pdep32((uint32_t)ob[v], e.lowCc);
    // tile counts fit 32 bits (2^31 tiles of 2^12 results would be 2^43 results)
    const int lct = __ffsll((long long)col_tiles) - 1;
    const int cmask = (int)col_tiles - 1;
    const int sc = (int)stride & cmask, sr = (int)(stride >> lct);
    int rt = (int)(t0 >> lct), ct = (int)t0 & cmask;
    uint64_t pr = 0, pc = 0, dc = 0, dr0 = 0, dr1 = 0;
    if constexpr (!LEAN) {
        pr = pdep64((uint64_t)rt, e.highR);
        pc = pdep64((uint64_t)ct, e.highC);
        dc = pdep64((uint64_t)sc, e.highC);
        dr0 = pdep64((uint64_t)sr, e.highR);
        dr1 = pdep64((uint64_t)sr + 1, e.highR);
    }
    for (int t = (int)t0; t < (int)t_end; t += (int)stride) {
        if constexpr (LEAN) {
            rt = t >> lct;
            ct = t & cmask;
        }
        const float *A = (const float *)sa.A + ((int64_t)rt << a) * K;
        const float *B = (const float *)sa.B + ((int64_t)ct << b) * K;
        // operands: rows [rt 2^a, (rt + 1) 2^a) of A and the tile's columns of
        // B, contiguous in memory; transposed to [k][row] / [k][col]
        if constexpr (K == 1) {
            for (int f = gt; f < Me / 4; f += 128) *(float4 *)&As[4 * f] = *(const float4 *)(A + 4 * f);
            for (int f = gt; f < Ne / 4; f += 128) *(float4 *)&Bs[4 * f] = *(const float4 *)(B + 4 * f);
        } else {
            constexpr int KQ = K / 4, LKQ = KB - 2;
            for (int f = gt; f < Me * KQ; f += 128) {
                const float4 v = *(const float4 *)(A + 4 * (int64_t)f);
                float *d = As + (f & (KQ - 1)) * 4 * PA + (f >> LKQ);
                d[0] = v.x;
                d[PA] = v.y;
                d[2 * PA] = v.z;
                d[3 * PA] = v.w;
            }
            for (int f = gt; f < Ne * KQ; f += 128) {
                const float4 v = *(const float4 *)(B + 4 * (int64_t)f);
                float *d = Bs + (f & (KQ - 1)) * 4 * PB + (f >> LKQ);
                d[0] = v.x;
                d[PB] = v.y;
                d[2 * PB] = v.z;
                d[3 * PB] = v.w;
            }
        }
        sk_bar(bid);
        float acc[4 * QM][4 * QN];
#pragma unroll
        for (int u = 0; u < 4 * QM; ++u)
#pragma unroll
            for (int v = 0; v < 4 * QN; ++v) acc[u][v] = 0.f;
        if (active) {
#pragma unroll
            for (int k = 0; k < K; ++k) {
                float4 av[QM], bv[QN];
#pragma unroll
                for (int u = 0; u < QM; ++u) av[u] = *(const float4 *)&As[k * PA + oa[u]];
#pragma unroll
                for (int v = 0; v < QN; ++v) bv[v] = *(const float4 *)&Bs[k * PB + ob[v]];
#pragma unroll
                for (int u = 0; u < QM; ++u) {
                    const float ar[4] = {av[u].x, av[u].y, av[u].z, av[u].w};
#pragma unroll
                    for (int v = 0; v < QN; ++v) {
                        const float br[4] = {bv[v].x, bv[v].y, bv[v].z, bv[v].w};
#pragma unroll
                        for (int i = 0; i < 4; ++i)
#pragma unroll
                            for (int j = 0; j < 4; ++j)
                                acc[4 * u + i][4 * v + j] = fmaf(ar[i], br[j], acc[4 * u + i][4 * v + j]);
                    }
                }
            }
        }
        sk_bar(bid);  // operands read: the staging buffer aliases them
        const uint64_t base = LEAN ? tile_base(e, (uint64_t)rt, (uint64_t)ct) : (pr | pc);
        if (direct) {
            if (active) {
                const double sd = (e.mode == EPI_OUT_F32 || e.mode == EPI_OUT_F64) ? e.zinfo[1] : 1.0;
                const float sf = (float)sd;
#define TQC_SK_DIRECT(M) \
    case M: sk_direct_store<M, QM, QN, RM>(e, acc, base, gr, gc, mR, mC, sf, sd); break;
                switch (e.mode) {
                    TQC_SK_DIRECT(EPI_F32)
                    TQC_SK_DIRECT(EPI_TF32)
                    TQC_SK_DIRECT(EPI_BF16)
                    TQC_SK_DIRECT(EPI_BF16X2)
                    TQC_SK_DIRECT(EPI_F64_SET)
                    TQC_SK_DIRECT(EPI_F64_ADD)
                    TQC_SK_DIRECT(EPI_OUT_F32)
                    TQC_SK_DIRECT(EPI_OUT_F64)
                    default: break;
                }
#undef TQC_SK_DIRECT
            }
        } else {
            if (active) sk_stage<QM, QN>(stg, acc, L, gr, gc);
            sk_bar(bid);
            if constexpr (LEAN) {
                sk_gather<-1>(tb, stg, e, base, Me * Ne, gt);
            } else {
#define TQC_SK_GATHER(M) \
    case M: sk_gather<M>(tb, stg, e, base, Me * Ne, gt); break;
                switch (e.mode) {
                    TQC_SK_GATHER(EPI_F32)
                    TQC_SK_GATHER(EPI_TF32)
                    TQC_SK_GATHER(EPI_BF16)
                    TQC_SK_GATHER(EPI_BF16X2)
                    TQC_SK_GATHER(EPI_F64_SET)
                    TQC_SK_GATHER(EPI_F64_ADD)
                    TQC_SK_GATHER(EPI_OUT_F32)
                    TQC_SK_GATHER(EPI_OUT_F64)
                    default: break;
                }
#undef TQC_SK_GATHER
            }
            sk_bar(bid);  // the next tile's operands overwrite the staging buffer
        }
        if constexpr (!LEAN) {
            const int c2 = ct + sc;
            const int carry = c2 >> lct;
            ct = c2 & cmask;
            rt += sr + carry;
            pc = ((pc | ~e.highC) + dc) & e.highC;
            pr = ((pr | ~e.highR) + (carry ? dr1 : dr0)) & e.highR;
        }
    }
}

template <int KB, int QM, bool RM>
__device__ __noinline__ void smallk_tiles_lean(const StepArgs &sa, const EpiTables *tb, const SmallkLayout L,
                                               int64_t col_tiles, int64_t t0, int64_t t_end, int64_t stride,
                                               float *buf, int gt, int bid) {
    smallk_tiles_body<KB, QM, RM, true>(sa, tb, L, col_tiles, t0, t_end, stride, buf, gt, bid);
}

template <int KB, int QM, bool RM, bool LEAN>
__device__ __forceinline__ void smallk_tiles(const StepArgs &sa, const EpiTables *tb, const SmallkLayout &L,
                                             int64_t col_tiles, int64_t t0, int64_t t_end, int64_t stride, float *buf,
                                             int gt, int bid) {
    if constexpr (LEAN) smallk_tiles_lean<KB, QM, RM>(sa, tb, L, col_tiles, t0, t_end, stride, buf, gt, bid);
    else smallk_tiles_body<KB, QM, RM, false>(sa, tb, L, col_tiles, t0, t_end, stride, buf, gt, bid);
}

// The instance for the step's K, tile width and staging orientation.
template <bool LEAN>
__device__ __forceinline__ void smallk_dispatch(const StepArgs &sa, const EpiTables *tb, const SmallkLayout &L,
                                                int64_t col_tiles, int64_t t0, int64_t t_end, int64_t stride,
                                                float *buf, int gt, int bid) {
#define TQC_SMALLK_CASE(KBV, QMV, RMV)                                                                         \
    if (sa.kb == KBV && L.qm == QMV && (L.rowmajor != 0) == RMV) {                                             \
        smallk_tiles<KBV, QMV, RMV, LEAN>(sa, tb, L, col_tiles, t0, t_end, stride, buf, gt, bid);            \
        return;                                                                                                \
    }
    TQC_SMALLK_CASE(0, 1, true)
    TQC_SMALLK_CASE(0, 1, false)
    TQC_SMALLK_CASE(0, 2, true)
    TQC_SMALLK_CASE(0, 2, false)
    TQC_SMALLK_CASE(2, 1, true)
    TQC_SMALLK_CASE(2, 1, false)
    TQC_SMALLK_CASE(2, 2, true)
    TQC_SMALLK_CASE(2, 2, false)
    TQC_SMALLK_CASE(4, 1, true)
    TQC_SMALLK_CASE(4, 1, false)
    TQC_SMALLK_CASE(4, 2, true)
    TQC_SMALLK_CASE(4, 2, false)
#undef TQC_SMALLK_CASE
}

}  // namespace tqc
