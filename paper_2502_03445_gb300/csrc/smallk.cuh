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
// results as outer products of float4 quads, the tile is staged in the
// orientation that makes the destination-order gather conflict-free, and
// the staged tile is written with runs of consecutive addresses
// (epi_readout).  The staging buffer aliases the operand buffer.
#pragma once

#include "device_common.cuh"
#include "launch.h"

namespace tqc {

// Shared memory a small-K tile uses (operands and staging alias).
constexpr int SMALLK_BYTES = 34816;

__host__ __device__ inline int smallk_op_bytes(int a, int b, int kb) {
    return (1 << kb) * ((1 << a) + 4 + (1 << b) + 4) * 4;
}
__host__ __device__ inline int smallk_stage_bytes(int a, int b, bool rowmajor) {
    return rowmajor ? (1 << a) * ((1 << b) + 4) * 4 : (1 << b) * ((1 << a) + 4) * 4;
}

// How a small-K step writes its tiles.  direct: the result's lowest bits
// (at least four) are bits of one dimension of the tile, so each thread's
// float4 quads along that dimension are 16 contiguous bytes and the lanes
// of a warp run along it: results go from registers straight to their
// destination, with no staging.  Otherwise the tile is staged (rowmajor,
// pitch) and gathered in destination order (gmode).  rowmajor also says
// which dimension the lanes run along: columns when set.  qm: row quads per
// thread (1: 4 x 8 results, 2: 8 x 4), 2 when the lanes run along rows.
struct SmallkLayout {
    int direct, rowmajor, pitch, gmode, qm;
};

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

__device__ __forceinline__ void sk_bar(int id) { asm volatile("bar.sync %0, 128;" ::"r"(id) : "memory"); }

// Tiles t0, t0 + stride, ... < t_end of a small-K step (col_tiles: a power
// of two).  KB = log2 K; QM x QN float4 quads per thread (1 x 2 or 2 x 1);
// RM: the lanes run along columns (a staging buffer is row-major).  gt: the thread's index in the group, bid: the group's named
// barrier; pitch / gmode: the staging pitch and gather mode the tables `tb`
// were built for.  Every thread's place in the tile is fixed across tiles.
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
__device__ __forceinline__ void smallk_tiles_body(const StepArgs &sa, const EpiTables *tb, int direct, int pitch,
                                                  int gmode, int64_t col_tiles, int64_t t0, int64_t t_end,
                                                  int64_t stride, float *buf, int gt, int bid) {
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
    uint64_t gr[QM], gc[QN];
    if (direct) {
#pragma unroll
        for (int u = 0; u < QM; ++u) gr[u] = pdep64((uint64_t)oa[u], mR);
#pragma unroll
        for (int v = 0; v < QN; ++v) gc[v] = pdep64((uint64_t)ob[v], mC);
    }
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
            if constexpr (!LEAN) {
                const int c2 = ct + sc;
                const int carry = c2 >> lct;
                ct = c2 & cmask;
                rt += sr + carry;
                pc = ((pc | ~e.highC) + dc) & e.highC;
                pr = ((pr | ~e.highR) + (carry ? dr1 : dr0)) & e.highR;
            }
            continue;
        }
        float *stg = buf;
        if (active) {
#pragma unroll
            for (int u = 0; u < QM; ++u)
#pragma unroll
                for (int v = 0; v < QN; ++v) {
                    float *d = RM ? stg + oa[u] * pitch + ob[v] : stg + ob[v] * pitch + oa[u];
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        if constexpr (RM)
                            *(float4 *)(d + i * pitch) = make_float4(acc[4 * u + i][4 * v], acc[4 * u + i][4 * v + 1],
                                                                     acc[4 * u + i][4 * v + 2], acc[4 * u + i][4 * v + 3]);
                        else
                            *(float4 *)(d + i * pitch) = make_float4(acc[4 * u][4 * v + i], acc[4 * u + 1][4 * v + i],
                                                                     acc[4 * u + 2][4 * v + i], acc[4 * u + 3][4 * v + i]);
                    }
                }
        }
        sk_bar(bid);
        if constexpr (LEAN) {
            epi_readout_rt(tb, stg, e, base, Me * Ne, gt, 128, gmode);
        } else {
            epi_readout(tb, stg, e, base, Me * Ne, gt, 128, gmode);
            const int c2 = ct + sc;
            const int carry = c2 >> lct;
            ct = c2 & cmask;
            rt += sr + carry;
            pc = ((pc | ~e.highC) + dc) & e.highC;
            pr = ((pr | ~e.highR) + (carry ? dr1 : dr0)) & e.highR;
        }
        sk_bar(bid);  // the next tile's operands overwrite the staging buffer
    }
}

template <int KB, int QM, bool RM>
__device__ __noinline__ void smallk_tiles_lean(const StepArgs &sa, const EpiTables *tb, int direct, int pitch,
                                               int gmode, int64_t col_tiles, int64_t t0, int64_t t_end,
                                               int64_t stride, float *buf, int gt, int bid) {
    smallk_tiles_body<KB, QM, RM, true>(sa, tb, direct, pitch, gmode, col_tiles, t0, t_end, stride, buf, gt, bid);
}

template <int KB, int QM, bool RM, bool LEAN>
__device__ __forceinline__ void smallk_tiles(const StepArgs &sa, const EpiTables *tb, const SmallkLayout &L,
                                             int64_t col_tiles, int64_t t0, int64_t t_end, int64_t stride, float *buf,
                                             int gt, int bid) {
    if constexpr (LEAN)
        smallk_tiles_lean<KB, QM, RM>(sa, tb, L.direct, L.pitch, L.gmode, col_tiles, t0, t_end, stride, buf, gt, bid);
    else
        smallk_tiles_body<KB, QM, RM, false>(sa, tb, L.direct, L.pitch, L.gmode, col_tiles, t0, t_end, stride, buf, gt,
                                             bid);
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
