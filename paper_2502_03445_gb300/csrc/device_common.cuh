// Device helpers shared by the step kernels: bit deposit, precision
// conversions, and the scatter epilogue that writes a staged GEMM tile into a
// bit-permuted tensor layout.
//
// A tile of Me x Ne results sits in shared memory, row-major (pitch Ne + 4)
// or column-major (pitch Me + 4).  Its elements are written in the order of
// the destination layout: the tile-local output index t enumerates the
// tile's result bits (tileMask) from the lowest, so runs of consecutive t are
// runs of consecutive addresses (2^L long).  Two small tables split every
// index computation into a low part (t & 127) and a high part (t >> 7):
//   staging index   s(t) = s_lo[t & 127] + s_hi[t >> 7]
//   element offset  g(t) = g_lo[t & 127] + g_hi[t >> 7]
// (both are sums because the row and column bits occupy disjoint positions).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "tqc_internal.h"

namespace tqc {

// Deposit the low bits of `src` into the set bits of `mask`, lowest first.
__device__ __forceinline__ uint64_t pdep64(uint64_t src, uint64_t mask) {
    uint64_t r = 0;
    while (mask) {
        uint64_t low = mask & (~mask + 1);
        if (src & 1) r |= low;
        src >>= 1;
        mask ^= low;
    }
    return r;
}

__device__ __forceinline__ uint32_t pdep32(uint32_t src, uint32_t mask) {
    uint32_t r = 0;
    while (mask) {
        uint32_t low = mask & (~mask + 1);
        if (src & 1) r |= low;
        src >>= 1;
        mask ^= low;
    }
    return r;
}

// Gather the bits of `x` at the set bits of `mask` into the low bits.
__device__ __forceinline__ uint32_t pext32(uint32_t x, uint32_t mask) {
    uint32_t r = 0, k = 0;
    while (mask) {
        uint32_t low = mask & (~mask + 1);
        if (x & low) r |= 1u << k;
        ++k;
        mask ^= low;
    }
    return r;
}

// FP32 -> TF32 (round to nearest, ties away), returned as FP32 bits.
__device__ __forceinline__ float to_tf32(float v) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(v));
    return __uint_as_float(r);
}

// Base element offset of the tile (rt, ct) in the result layout.
__device__ __forceinline__ uint64_t tile_base(const EpiParams &e, uint64_t rt, uint64_t ct) {
    return pdep64(rt, e.highR) | pdep64(ct, e.highC);
}

__device__ __forceinline__ uint32_t pack_bf16x2(float a, float b) {
    __nv_bfloat162 p = __floats2bfloat162_rn(a, b);
    return *(uint32_t *)&p;
}

// Store `vw` (1, 2 or 4) values to consecutive elements starting at `off`;
// `s` is the output scale zinfo[1] for the EPI_OUT_* modes (read once per
// tile by the caller).
__device__ __forceinline__ void store_run_f32(const EpiParams &e, uint64_t off, const float *v, int vw,
                                              double s = 1.0) {
    switch (e.mode) {
        case EPI_F32: {
            float *o = (float *)e.out + off;
            if (vw == 4) *(float4 *)o = make_float4(v[0], v[1], v[2], v[3]);
            else if (vw == 2) *(float2 *)o = make_float2(v[0], v[1]);
            else o[0] = v[0];
        } break;
        case EPI_TF32: {
            float *o = (float *)e.out + off;
            if (vw == 4) *(float4 *)o = make_float4(to_tf32(v[0]), to_tf32(v[1]), to_tf32(v[2]), to_tf32(v[3]));
            else if (vw == 2) *(float2 *)o = make_float2(to_tf32(v[0]), to_tf32(v[1]));
            else o[0] = to_tf32(v[0]);
        } break;
        case EPI_BF16: {
            __nv_bfloat16 *o = (__nv_bfloat16 *)e.out + off;
            if (vw == 4) *(uint2 *)o = make_uint2(pack_bf16x2(v[0], v[1]), pack_bf16x2(v[2], v[3]));
            else if (vw == 2) *(uint32_t *)o = pack_bf16x2(v[0], v[1]);
            else o[0] = __float2bfloat16_rn(v[0]);
        } break;
        case EPI_BF16X2: {
            __nv_bfloat16 *oh = (__nv_bfloat16 *)e.out + off;
            __nv_bfloat16 *ol = (__nv_bfloat16 *)e.out_lo + off;
            float h[4], l[4];
            for (int i = 0; i < vw; ++i) {
                __nv_bfloat16 b = __float2bfloat16_rn(v[i]);
                h[i] = __bfloat162float(b);
                l[i] = v[i] - h[i];
            }
            if (vw == 4) {
                *(uint2 *)oh = make_uint2(pack_bf16x2(h[0], h[1]), pack_bf16x2(h[2], h[3]));
                *(uint2 *)ol = make_uint2(pack_bf16x2(l[0], l[1]), pack_bf16x2(l[2], l[3]));
            } else if (vw == 2) {
                *(uint32_t *)oh = pack_bf16x2(h[0], h[1]);
                *(uint32_t *)ol = pack_bf16x2(l[0], l[1]);
            } else {
                oh[0] = __float2bfloat16_rn(h[0]);
                ol[0] = __float2bfloat16_rn(l[0]);
            }
        } break;
        case EPI_F64_SET: {
            double *o = (double *)e.out + off;
            if (vw == 4) {
                ((double2 *)o)[0] = make_double2(v[0], v[1]);
                ((double2 *)o)[1] = make_double2(v[2], v[3]);
            } else if (vw == 2) {
                ((double2 *)o)[0] = make_double2(v[0], v[1]);
            } else {
                o[0] = v[0];
            }
        } break;
        case EPI_F64_ADD: {
            double *o = (double *)e.out + off;
            if (vw == 4) {
                double2 a = ((double2 *)o)[0], b = ((double2 *)o)[1];
                ((double2 *)o)[0] = make_double2(a.x + v[0], a.y + v[1]);
                ((double2 *)o)[1] = make_double2(b.x + v[2], b.y + v[3]);
            } else if (vw == 2) {
                double2 a = ((double2 *)o)[0];
                ((double2 *)o)[0] = make_double2(a.x + v[0], a.y + v[1]);
            } else {
                o[0] += v[0];
            }
        } break;
        case EPI_OUT_F32: {
            const float sf = (float)s;
            float *o = (float *)e.out + off;
            if (vw == 4) *(float4 *)o = make_float4(v[0] * sf, v[1] * sf, v[2] * sf, v[3] * sf);
            else if (vw == 2) *(float2 *)o = make_float2(v[0] * sf, v[1] * sf);
            else o[0] = v[0] * sf;
        } break;
        case EPI_OUT_F64: {
            double *o = (double *)e.out + off;
            if (vw == 4) {
                ((double2 *)o)[0] = make_double2(v[0] * s, v[1] * s);
                ((double2 *)o)[1] = make_double2(v[2] * s, v[3] * s);
            } else if (vw == 2) {
                ((double2 *)o)[0] = make_double2(v[0] * s, v[1] * s);
            } else {
                o[0] = v[0] * s;
            }
        } break;
        default: break;
    }
}

struct EpiTables {
    uint32_t s_lo[128];
    uint32_t s_hi[256];
    uint64_t g_lo[128];
    uint64_t g_hi[256];
};

// Fill the tables (tile independent) for a staging buffer of the given
// orientation and pitch.  Threads [0, nthreads) of the caller cooperate.
__device__ __forceinline__ void epi_tables_init(EpiTables *tb, const EpiParams &e, bool rowmajor, int pitch,
                                                int tid, int nthreads) {
    for (int u = tid; u < 384; u += nthreads) {
        const bool lo = u < 128;
        const uint32_t t = lo ? (uint32_t)u : (uint32_t)(u - 128) << 7;
        const uint32_t i = pext32(t, e.lowRc), j = pext32(t, e.lowCc);
        const uint32_t s = rowmajor ? i * pitch + j : j * pitch + i;
        const uint64_t g = pdep64(t, e.tileMask);
        if (lo) {
            tb->s_lo[u] = s;
            tb->g_lo[u] = g;
        } else {
            tb->s_hi[u - 128] = s;
            tb->g_hi[u - 128] = g;
        }
    }
}

// How a thread's four consecutive output elements t..t+3 sit in the staging
// buffer: which of t's two lowest bits run along its contiguous dimension.
enum GatherMode { G_VEC4 = 0, G_PAIR01 = 1, G_PAIR02 = 2, G_SCALAR = 3 };

struct StagePick {
    int rowmajor;  // 1: staging [row][col] (columns contiguous), 0: [col][row]
    int gmode;
};

// Choose the staging orientation so that the bits that vary across the
// lanes of a warp (t bits 2..6) and the thread's own low bits fall on the
// contiguous dimension as far as possible: conflict-free, vectorised
// gathers.  `lowRc` / `lowCc` mark the row / column bits of t.
__host__ __device__ inline int gather_mode(uint32_t contig) {
    const bool b0 = contig & 1u, b1 = contig & 2u;
    return (b0 && b1) ? G_VEC4 : b0 ? G_PAIR01 : b1 ? G_PAIR02 : G_SCALAR;
}

__host__ __device__ inline StagePick pick_staging(uint32_t lowRc, uint32_t lowCc) {
    StagePick p;
    int rows = 0, cols = 0;
    for (int k = 0; k < 7; ++k) {
        rows += (lowRc >> k) & 1u;
        cols += (lowCc >> k) & 1u;
    }
    p.rowmajor = cols >= rows ? 1 : 0;
    p.gmode = gather_mode(p.rowmajor ? lowCc : lowRc);
    return p;
}

// Store VW (1, 2 or 4) consecutive values of an epilogue in output mode MODE
// (the compile-time twin of store_run_f32, for loops that dispatch the mode
// once instead of per store); sf / sd: the EPI_OUT_* scale in FP32 / FP64.
template <int MODE, int VW>
__device__ __forceinline__ void store_vals(const EpiParams &e, uint64_t off, const float *v, float sf, double sd) {
    if constexpr (MODE == EPI_F32 || MODE == EPI_TF32 || MODE == EPI_OUT_F32) {
        float w[VW];
#pragma unroll
        for (int i = 0; i < VW; ++i)
            w[i] = MODE == EPI_TF32 ? to_tf32(v[i]) : (MODE == EPI_OUT_F32 ? v[i] * sf : v[i]);
        float *o = (float *)e.out + off;
        if constexpr (VW == 4) *(float4 *)o = make_float4(w[0], w[1], w[2], w[3]);
        else if constexpr (VW == 2) *(float2 *)o = make_float2(w[0], w[1]);
        else o[0] = w[0];
    } else if constexpr (MODE == EPI_BF16) {
        __nv_bfloat16 *o = (__nv_bfloat16 *)e.out + off;
        if constexpr (VW == 4) *(uint2 *)o = make_uint2(pack_bf16x2(v[0], v[1]), pack_bf16x2(v[2], v[3]));
        else if constexpr (VW == 2) *(uint32_t *)o = pack_bf16x2(v[0], v[1]);
        else o[0] = __float2bfloat16_rn(v[0]);
    } else if constexpr (MODE == EPI_BF16X2) {
        float h[VW], l[VW];
#pragma unroll
        for (int i = 0; i < VW; ++i) {
            h[i] = __bfloat162float(__float2bfloat16_rn(v[i]));
            l[i] = v[i] - h[i];
        }
        __nv_bfloat16 *oh = (__nv_bfloat16 *)e.out + off;
        __nv_bfloat16 *ol = (__nv_bfloat16 *)e.out_lo + off;
        if constexpr (VW == 4) {
            *(uint2 *)oh = make_uint2(pack_bf16x2(h[0], h[1]), pack_bf16x2(h[2], h[3]));
            *(uint2 *)ol = make_uint2(pack_bf16x2(l[0], l[1]), pack_bf16x2(l[2], l[3]));
        } else if constexpr (VW == 2) {
            *(uint32_t *)oh = pack_bf16x2(h[0], h[1]);
            *(uint32_t *)ol = pack_bf16x2(l[0], l[1]);
        } else {
            oh[0] = __float2bfloat16_rn(h[0]);
            ol[0] = __float2bfloat16_rn(l[0]);
        }
    } else {  // FP64 modes
        double w[VW];
        double *o = (double *)e.out + off;
#pragma unroll
        for (int i = 0; i < VW; ++i) w[i] = MODE == EPI_OUT_F64 ? (double)v[i] * sd : (double)v[i];
        if constexpr (MODE == EPI_F64_ADD) {
#pragma unroll
            for (int i = 0; i < VW; i += 2) {
                if constexpr (VW == 1) {
                    o[0] += w[0];
                } else {
                    const double2 a = ((const double2 *)o)[i / 2];
                    ((double2 *)o)[i / 2] = make_double2(a.x + w[i], a.y + w[i + 1]);
                }
            }
        } else {
            if constexpr (VW == 1) {
                o[0] = w[0];
            } else {
#pragma unroll
                for (int i = 0; i < VW; i += 2) ((double2 *)o)[i / 2] = make_double2(w[i], w[i + 1]);
            }
        }
    }
}

// Write the staged tile (E = 2^(a+b) elements) to its destination.
// nthreads is a multiple of 32: a thread's t advances by a multiple of 128,
// so its low table entries (t & 127) are read once, not once per run (the
// lanes of a warp read them at a stride of four entries: bank conflicts).
// The output mode is dispatched once per tile (MODE >= 0), or per store
// (MODE = -1: fewer registers, for kernels with a tight budget).  The tables
// and the staged tile are in shared memory.
template <int MODE>
__device__ __forceinline__ void epi_readout_m(const EpiTables *tb, const float *stg, const EpiParams &e,
                                              uint64_t base, int E, int tid, int nthreads, int gmode) {
    __builtin_assume(__isShared(tb));
    __builtin_assume(__isShared(stg));
    const int mode = MODE >= 0 ? MODE : e.mode;
    const double sd = (mode == EPI_OUT_F32 || mode == EPI_OUT_F64) ? e.zinfo[1] : 1.0;
    const float sf = (float)sd;
    if (e.L >= 2) {
        const int tl = (tid * 4) & 127;
        const uint32_t l0 = tb->s_lo[tl], l1 = tb->s_lo[tl + 1], l2 = tb->s_lo[tl + 2], l3 = tb->s_lo[tl + 3];
        const uint64_t gbase = base + tb->g_lo[tl];
#pragma unroll 4
        for (int t = tid * 4; t < E; t += nthreads * 4) {
            const float *sp = stg + tb->s_hi[t >> 7];
            float v[4];
            if (gmode == G_VEC4) {
                const float4 q = *(const float4 *)(sp + l0);
                v[0] = q.x;
                v[1] = q.y;
                v[2] = q.z;
                v[3] = q.w;
            } else if (gmode == G_PAIR01) {
                const float2 a = *(const float2 *)(sp + l0);
                const float2 b = *(const float2 *)(sp + l2);
                v[0] = a.x;
                v[1] = a.y;
                v[2] = b.x;
                v[3] = b.y;
            } else if (gmode == G_PAIR02) {
                const float2 a = *(const float2 *)(sp + l0);
                const float2 b = *(const float2 *)(sp + l1);
                v[0] = a.x;
                v[1] = b.x;
                v[2] = a.y;
                v[3] = b.y;
            } else {
                v[0] = sp[l0];
                v[1] = sp[l1];
                v[2] = sp[l2];
                v[3] = sp[l3];
            }
            if constexpr (MODE >= 0) store_vals<MODE, 4>(e, gbase + tb->g_hi[t >> 7], v, sf, sd);
            else store_run_f32(e, gbase + tb->g_hi[t >> 7], v, 4, sd);
        }
    } else {
        for (int t = tid; t < E; t += nthreads) {
            float v = stg[tb->s_hi[t >> 7] + tb->s_lo[t & 127]];
            if constexpr (MODE >= 0) store_vals<MODE, 1>(e, base + tb->g_hi[t >> 7] + tb->g_lo[t & 127], &v, sf, sd);
            else store_run_f32(e, base + tb->g_hi[t >> 7] + tb->g_lo[t & 127], &v, 1, sd);
        }
    }
}

__device__ __forceinline__ void epi_readout_rt(const EpiTables *tb, const float *stg, const EpiParams &e,
                                               uint64_t base, int E, int tid, int nthreads, int gmode) {
    epi_readout_m<-1>(tb, stg, e, base, E, tid, nthreads, gmode);
}

__device__ __forceinline__ void epi_readout(const EpiTables *tb, const float *stg, const EpiParams &e,
                                            uint64_t base, int E, int tid, int nthreads, int gmode) {
    switch (e.mode) {
        case EPI_F32: epi_readout_m<EPI_F32>(tb, stg, e, base, E, tid, nthreads, gmode); break;
        case EPI_TF32: epi_readout_m<EPI_TF32>(tb, stg, e, base, E, tid, nthreads, gmode); break;
        case EPI_BF16: epi_readout_m<EPI_BF16>(tb, stg, e, base, E, tid, nthreads, gmode); break;
        case EPI_BF16X2: epi_readout_m<EPI_BF16X2>(tb, stg, e, base, E, tid, nthreads, gmode); break;
        case EPI_F64_SET: epi_readout_m<EPI_F64_SET>(tb, stg, e, base, E, tid, nthreads, gmode); break;
        case EPI_F64_ADD: epi_readout_m<EPI_F64_ADD>(tb, stg, e, base, E, tid, nthreads, gmode); break;
        case EPI_OUT_F32: epi_readout_m<EPI_OUT_F32>(tb, stg, e, base, E, tid, nthreads, gmode); break;
        case EPI_OUT_F64: epi_readout_m<EPI_OUT_F64>(tb, stg, e, base, E, tid, nthreads, gmode); break;
        default: break;
    }
}

// Direct stores of NV (32 or 16) consecutive accumulator columns of one
// row, VW at a time: run j (j = 0, VW, 2 VW, ...) goes to o + x_j, where x_j is the
// deposit of j into the result bits of the column index; the next deposit
// is ((x | ~m) + 1) & m with m = those bits minus the VW-run bits.
template <int MODE, int VW, int NV = 32>
__device__ __forceinline__ void direct_run32(const EpiParams &e, uint64_t o, uint64_t m, const uint32_t *r, float sf,
                                             double sd) {
    uint64_t x = 0;
#pragma unroll
    for (int j = 0; j < NV; j += VW) {
        float v[VW];
#pragma unroll
        for (int i = 0; i < VW; ++i) v[i] = __uint_as_float(r[j + i]);
        store_vals<MODE, VW>(e, o + x, v, sf, sd);
        x = ((x | ~m) + 1) & m;
    }
}

template <int MODE, int NV = 32>
__device__ __forceinline__ void direct_run32_vw(const EpiParams &e, int vw, uint64_t o, uint64_t m, const uint32_t *r,
                                                float sf, double sd) {
    if (vw == 4) direct_run32<MODE, 4, NV>(e, o, m, r, sf, sd);
    else if (vw == 2) direct_run32<MODE, 2, NV>(e, o, m, r, sf, sd);
    else direct_run32<MODE, 1, NV>(e, o, m, r, sf, sd);
}

// Mode dispatch, once per NV values.
template <int NV = 32>
__device__ __forceinline__ void direct_run32_any(const EpiParams &e, int vw, uint64_t o, uint64_t m, const uint32_t *r,
                                                 float sf, double sd) {
    switch (e.mode) {
        case EPI_F32: direct_run32_vw<EPI_F32, NV>(e, vw, o, m, r, sf, sd); break;
        case EPI_TF32: direct_run32_vw<EPI_TF32, NV>(e, vw, o, m, r, sf, sd); break;
        case EPI_BF16: direct_run32_vw<EPI_BF16, NV>(e, vw, o, m, r, sf, sd); break;
        case EPI_BF16X2: direct_run32_vw<EPI_BF16X2, NV>(e, vw, o, m, r, sf, sd); break;
        case EPI_F64_SET: direct_run32_vw<EPI_F64_SET, NV>(e, vw, o, m, r, sf, sd); break;
        case EPI_F64_ADD: direct_run32_vw<EPI_F64_ADD, NV>(e, vw, o, m, r, sf, sd); break;
        case EPI_OUT_F32: direct_run32_vw<EPI_OUT_F32, NV>(e, vw, o, m, r, sf, sd); break;
        case EPI_OUT_F64: direct_run32_vw<EPI_OUT_F64, NV>(e, vw, o, m, r, sf, sd); break;
        default: break;
    }
}

// pdep64 computed by a whole warp: lane l deposits bits l and l + 32 of x,
// then an OR reduction (every lane of the warp must call it).
__device__ __forceinline__ uint64_t warp_pdep64(uint64_t x, uint64_t mask) {
    const int ln = threadIdx.x & 31;
    const uint32_t mlo = (uint32_t)mask, mhi = (uint32_t)(mask >> 32);
    const int plo = __popc(mlo), ptot = plo + __popc(mhi);
    uint64_t v = 0;
#pragma unroll
    for (int hw = 0; hw < 2; ++hw) {
        const int idx = ln + 32 * hw;
        if (idx < ptot && ((x >> idx) & 1)) {
            const int pos = idx < plo ? (int)__fns(mlo, 0, idx + 1) : 32 + (int)__fns(mhi, 0, idx - plo + 1);
            v |= 1ull << pos;
        }
    }
    const uint32_t lo = __reduce_or_sync(0xffffffffu, (uint32_t)v);
    const uint32_t hi = __reduce_or_sync(0xffffffffu, (uint32_t)(v >> 32));
    return ((uint64_t)hi << 32) | lo;
}

}  // namespace tqc
