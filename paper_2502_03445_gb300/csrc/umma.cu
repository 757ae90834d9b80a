// tcgen05 tensor-core pairwise step for sm_103a.
//
// C[r, c] = sum_k A[r, k] B[c, k] over the shared cut edges of two subcircuit
// tensors (§III-B, Fig. tensor_contraction) when K = 4^{#shared cuts} is large
// enough for the step to be a real contraction.  Operands are K-major BF16
// (or TF32, or a BF16 hi/lo pair for the split form) written by the producing
// step's epilogue; the result goes through the same bit-scatter epilogue as
// the CUDA-core step (Kronecker expansion of output indices for the last
// step, Eq. reconstruction).
//
// One persistent CTA per SM, warp-specialised:
//   warp 0      TMA producer: 128B-swizzled A and B k-blocks into a ring of
//               shared-memory stages (mbarrier complete_tx)
//   warp 1      allocates TMEM (two FP32 accumulators of 128 x BN) and issues
//               tcgen05.mma from one thread; tcgen05.commit frees stages and
//               hands accumulators to the epilogue
//   warps 2..17 epilogue (staged form): tcgen05.ld 32 columns at a time,
//               stage the tile in shared memory in the orientation that
//               makes the result's lowest bits contiguous, then write
//               16-byte runs to HBM
// The direct form (deep-K steps, and layouts whose warp stores fill whole
// sectors) drops the staging buffers: every epilogue warp loads its 32-row
// block from TMEM 16 columns at a time, frees the accumulator and stores
// straight to HBM, which the next tile's K loop hides; the freed shared
// memory deepens the operand ring (192 KB in flight) and allows 128 x 256
// MMA tiles.  A step with one k-block and one column tile keeps B resident.
// In the direct form a tile's K loop may be split into ranges run as
// separate units (split s of every tile after split s - 1), each storing an
// FP32 partial that a reduce pass sums: this evens the waves of a step with
// few tiles.
// Every wait is bounded (clock64); a wait that gives up sets an error word,
// drains the copies and MMAs it issued, frees TMEM and returns.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <atomic>
#include <mutex>

#include "device_common.cuh"
#include "launch.h"
#include "tc_ptx.cuh"

namespace tqc {

namespace {

using namespace tc;

constexpr int BM = 128;
constexpr int EPI_WARPS = 16;
constexpr int EPI_THREADS = 32 * EPI_WARPS;
constexpr int NTHREADS = 64 + EPI_THREADS;
constexpr int STAGE_WARPS = 8;  // epilogue warpgroups 0 and 1 move accumulators out of TMEM
std::atomic<int> g_umma_stall{0};  // tqc_step_inject_stall


struct UmmaParams {
    int64_t n_tiles;
    int64_t n_units;       // n_tiles * ksplit: unit u is split u / n_tiles of tile u % n_tiles
    int64_t col_tiles;
    int64_t split_stride;  // elements between the FP32 partials of the splits
    int32_t ksplit;        // K ranges per tile (deep form only)
    int32_t sw64;          // deep form: 64-byte swizzled k-blocks (half the K per stage, twice the stages)
    int32_t kblk;          // operands K-blocked ([K / 64][rows][64]): 3-D copies
    int32_t k_blocks;
    int32_t rowmajor;  // staging orientation (pick_staging)
    int32_t gmode;     // gather mode of the write-out (pick_staging)
    int32_t bres;      // B stays resident in shared memory (one k-block, one column tile; deep form)
    int32_t stall;     // test hook: CTA 0 never issues its first k-block's copies
    EpiParams epi;
    int *err;
};

template <int BN, int KIND, bool DEEP>
struct Cfg {
    static constexpr int ELEM = KIND == K_TF32 ? 4 : 2;
    static constexpr int BK = 128 / ELEM;          // one 128-byte swizzle atom of K
    static constexpr int PLANES = KIND == K_BF16X3 ? 2 : 1;
    static constexpr int A_BYTES = BM * 128;
    static constexpr int B_BYTES = BN * 128;
    static constexpr int STAGE_BYTES = PLANES * (A_BYTES + B_BYTES);
    static constexpr int STAGES = DEEP ? 196608 / STAGE_BYTES : (KIND == K_BF16X3 ? 2 : (BN == 64 ? 6 : 4));
    static constexpr int SUB_N = 64;               // epilogue sub-tile: 128 x 64
    static constexpr int PITCH_R = SUB_N + 4;      // row-major staging pitch (floats)
    static constexpr int PITCH_C = BM + 4;         // column-major staging pitch
    static constexpr int STG_FLOATS = BM * PITCH_R > SUB_N * PITCH_C ? BM * PITCH_R : SUB_N * PITCH_C;
    static constexpr int STG_BYTES = DEEP ? 0 : 2 * STG_FLOATS * 4;  // two buffers (ping-pong)
    static constexpr int BAR_BYTES = 1024;
    static constexpr int RING = STAGES * STAGE_BYTES;      // bytes of the operand ring
    static constexpr int MAXST = DEEP ? 16 : STAGES;        // barrier slots of the ring
    static constexpr int SMEM = 1024 + STAGES * STAGE_BYTES + STG_BYTES + (int)sizeof(EpiTables) + BAR_BYTES;
    static constexpr int TMEM_COLS = 2 * BN;
    static_assert(SMEM <= 232448, "shared memory per CTA");
    static_assert(STAGES >= 2, "operand ring");
    // instruction descriptor: D = F32, A/B = BF16 (1) or TF32 (2), K-major, N >> 3, M >> 4
    static constexpr uint32_t IDESC = (1u << 4) | ((KIND == K_TF32 ? 2u : 1u) << 7) |
                                      ((KIND == K_TF32 ? 2u : 1u) << 10) | ((uint32_t)(BN >> 3) << 17) |
                                      ((uint32_t)(BM >> 4) << 24);
};



template <int BN, int KIND, bool DEEP>
__global__ void __launch_bounds__(NTHREADS, 1)
    umma_step_kernel(const __grid_constant__ CUtensorMap tA, const __grid_constant__ CUtensorMap tB,
                     const __grid_constant__ CUtensorMap tAl, const __grid_constant__ CUtensorMap tBl,
                     const UmmaParams P) {
    using C = Cfg<BN, KIND, DEEP>;
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint8_t *stages = smem;
    float *stg = (float *)(smem + C::RING);
    EpiTables *tb = (EpiTables *)(smem + C::RING + C::STG_BYTES);
    uint64_t *full = (uint64_t *)(smem + C::RING + C::STG_BYTES + sizeof(EpiTables));
    uint64_t *empty = full + C::MAXST;
    uint64_t *tfull = empty + C::MAXST;
    uint64_t *tempty = tfull + 2;
    uint64_t *drain = tempty + 2;
    uint64_t *bfull = drain + 1;
    uint32_t *tmem_slot = (uint32_t *)(bfull + 1);
    // With B resident (deep form, a single k-block and column tile: B is the
    // same for every tile) the ring holds A only and B sits at its end.
    const bool bres = DEEP && P.bres;
    // bytes of K per operand row in one k-block (the swizzle span), and the
    // plane sizes of a stage
    const int rowb = (DEEP && P.sw64) ? 64 : 128;
    const bool kblk = P.kblk != 0;
    const int bk = rowb / C::ELEM, ksl = rowb / 32;  // elements of K per k-block; 32-byte MMA slices
    const int ab = BM * rowb, bb = BN * rowb;
    const int sbytes = bres ? C::PLANES * ab : C::PLANES * (ab + bb);
    const int nfit = (C::RING - (bres ? C::PLANES * bb : 0)) / sbytes;
    const int nst = nfit < C::MAXST ? nfit : (int)C::MAXST;
    uint8_t *bsm = stages + C::RING - C::PLANES * bb;
    volatile int *abort_flag = (volatile int *)(tmem_slot + 1);
    uint64_t *tile_base_slot = (uint64_t *)(tmem_slot + 2);  // epilogue: base offsets of two sub-tiles
    uint8_t *tb_pos = (uint8_t *)(tile_base_slot + 2);       // epilogue: tile-index bit positions

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < nst; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(bfull, 1);
        for (int a = 0; a < 2; ++a) {
            mbar_init(&tfull[a], 1);
            mbar_init(&tempty[a], DEEP ? EPI_WARPS : STAGE_WARPS);
        }
        mbar_init(drain, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"((uint32_t)C::TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;
    const EpiParams &e = P.epi;

    if (warp == 0) {
        // ------------------------------------------------ TMA producer
        if (lane == 0) {
            asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&tA) : "memory");
            asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&tB) : "memory");
            int64_t it = 0;
            bool ok = true, skipped0 = false;
            if (bres) {  // the one B tile, loaded once
                mbar_expect_tx(bfull, C::PLANES * bb);
                tma_load_op(bsm, &tB, 0, 0, bfull, kblk);
                if (KIND == K_BF16X3) tma_load_op(bsm + bb, &tBl, 0, 0, bfull, kblk);
            }
            for (int64_t u = blockIdx.x; ok && u < P.n_units; u += gridDim.x) {
                const int64_t sp = u / P.n_tiles, tile = u - sp * P.n_tiles;
                const int rt = (int)(tile / P.col_tiles), ct = (int)(tile - (int64_t)rt * P.col_tiles);
                const int kb0 = (int)(sp * P.k_blocks / P.ksplit), kb1 = (int)((sp + 1) * P.k_blocks / P.ksplit);
                for (int kb = kb0; kb < kb1; ++kb, ++it) {
                    const int s = (int)(it % nst);
                    const uint32_t ph = (uint32_t)((it / nst) & 1);
                    if (!mbar_wait(&empty[s], ph ^ 1u, abort_flag)) {
                        ok = false;
                        break;
                    }
                    if (P.stall && blockIdx.x == 0 && it == 0) {
                        // test hook: stage 0 never fills, so the MMA issuer's bounded wait gives up
                        skipped0 = true;
                        continue;
                    }
                    uint8_t *sa = stages + s * sbytes;
                    mbar_expect_tx(&full[s], (uint32_t)sbytes);
                    tma_load_op(sa, &tA, kb * bk, rt * BM, &full[s], kblk);
                    if (bres) {
                        if (KIND == K_BF16X3) tma_load_op(sa + ab, &tAl, kb * bk, rt * BM, &full[s], kblk);
                    } else {
                        tma_load_op(sa + ab, &tB, kb * bk, ct * BN, &full[s], kblk);
                        if (KIND == K_BF16X3) {
                            tma_load_op(sa + ab + bb, &tAl, kb * bk, rt * BM, &full[s], kblk);
                            tma_load_op(sa + 2 * ab + bb, &tBl, kb * bk, ct * BN, &full[s], kblk);
                        }
                    }
                }
            }
            if (!ok || skipped0) {
                // drain: wait (bounded) for the copies still in flight in every stage
                for (int64_t j = it > nst ? it - nst : 0; j < it; ++j) {
                    if (skipped0 && j == 0) continue;  // never issued
                    long long t0 = clock64();
                    while (!mbar_try_wait(&full[j % nst], (uint32_t)((j / nst) & 1)) && clock64() - t0 < WAIT_CYCLES) {
                    }
                }
                if (bres) {
                    long long t0 = clock64();
                    while (!mbar_try_wait(bfull, 0) && clock64() - t0 < WAIT_CYCLES) {
                    }
                }
            }
        }
    } else if (warp == 1) {
        // ------------------------------------------------ MMA issuer
        if (lane == 0) {
            int64_t it = 0, lt = 0;
            bool ok = true;
            if (bres) {
                ok = mbar_wait(bfull, 0, abort_flag);
                tc_fence_after();
            }
            for (int64_t u = blockIdx.x; ok && u < P.n_units; u += gridDim.x, ++lt) {
                const int64_t sp = u / P.n_tiles;
                const int kb0 = (int)(sp * P.k_blocks / P.ksplit), kb1 = (int)((sp + 1) * P.k_blocks / P.ksplit);
                const int acc = (int)(lt & 1);
                const uint32_t aph = (uint32_t)((lt >> 1) & 1);
                if (!mbar_wait(&tempty[acc], aph ^ 1u, abort_flag)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t d = tmem_base + (uint32_t)(acc * BN);
                for (int kb = kb0; kb < kb1; ++kb, ++it) {
                    const int s = (int)(it % nst);
                    const uint32_t ph = (uint32_t)((it / nst) & 1);
                    if (!mbar_wait(&full[s], ph, abort_flag)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t a0 = smem_u32(stages + s * sbytes);
                    const uint32_t b0 = bres ? smem_u32(bsm) : a0 + ab;
                    const uint32_t al = bres ? a0 + ab : b0 + bb;
                    const uint32_t bl = bres ? b0 + bb : al + ab;
#pragma unroll
                    for (int k = 0; k < 4; ++k) {  // 32-byte K slices of the swizzled row: 4 (128 B) or 2 (64 B)
                        if (k < ksl) {
                            const uint64_t da = umma_desc(a0 + 32 * k, rowb), db = umma_desc(b0 + 32 * k, rowb);
                            umma<KIND>(d, da, db, C::IDESC, ((kb - kb0) | k) != 0);
                            if (KIND == K_BF16X3) {
                                umma<KIND>(d, da, umma_desc(bl + 32 * k, rowb), C::IDESC, 1u);
                                umma<KIND>(d, umma_desc(al + 32 * k, rowb), db, C::IDESC, 1u);
                            }
                        }
                    }
                    umma_commit(&empty[s]);
                }
                if (ok) umma_commit(&tfull[acc]);
            }
            // every MMA issued so far has completed once this commit arrives
            umma_commit(drain);
            long long t0 = clock64();
            while (!mbar_try_wait(drain, 0) && clock64() - t0 < WAIT_CYCLES) {
            }
        }
    } else if constexpr (DEEP) {
        // ------------------------------------------------ direct epilogue
        // Warp (lane group g, quarter q) owns accumulator rows 32g..32g+31
        // and the 32-column chunks q, q + 4, ...; it frees the accumulator as
        // soon as its loads land and then stores every value straight to its
        // place in the result layout: tile base + row part + column part,
        // each a deposit of the tile-local index bits into result bits.
        constexpr int CH = BN / 128;     // chunks per warp
        constexpr int SUBS = BN / C::SUB_N;
        const int q = (warp - 2) >> 2;
        const int lane_grp = warp & 3;
        const int row = lane_grp * 32 + lane;
        const uint64_t grow = pdep64((uint64_t)pdep32((uint32_t)row, e.lowRc), e.tileMask);
        const uint64_t colmask = pdep64((uint64_t)e.lowCc, e.tileMask);  // result bits of the column index
        // runs of 2^w columns are contiguous when the w lowest tile bits are
        // column bits at result bits 0..w-1
        const int vw = ((e.lowCc & 3u) == 3u && e.L >= 2) ? 4 : ((e.lowCc & 1u) && e.L >= 1 ? 2 : 1);
        const uint64_t mstep = vw == 4 ? colmask & (colmask - 1) & ((colmask & (colmask - 1)) - 1)
                                       : (vw == 2 ? colmask & (colmask - 1) : colmask);
        uint64_t coff[CH];  // column part of each chunk's first column, sub-tile index included
#pragma unroll
        for (int c = 0; c < CH; ++c) {
            const int col0 = (q + 4 * c) * 32;
            coff[c] = pdep64((uint64_t)(col0 % C::SUB_N), colmask) | pdep64((uint64_t)(col0 / C::SUB_N), e.highC);
        }
        const double sd = (e.mode == EPI_OUT_F32 || e.mode == EPI_OUT_F64) ? e.zinfo[1] : 1.0;
        const float sf = (float)sd;
        // column 16 of a chunk (chunks start at multiples of 32, so its
        // deposit adds to the chunk's: the bits are disjoint)
        const uint64_t off16 = pdep64(16, colmask);
        int64_t lt = 0;
        for (int64_t u = blockIdx.x; u < P.n_units; u += gridDim.x, ++lt) {
            const int acc = (int)(lt & 1);
            if (lane == 0) mbar_wait(&tfull[acc], (uint32_t)((lt >> 1) & 1), abort_flag);
            __syncwarp();
            if (*abort_flag) break;
            tc_fence_after();
            const int64_t sp = u / P.n_tiles, tile = u - sp * P.n_tiles;
            const uint64_t rt = (uint64_t)(tile / P.col_tiles);
            const uint64_t ct = (uint64_t)(tile - (int64_t)rt * P.col_tiles);
            // sub-tile column index ct * SUBS + h: the h bits are the lowest bits of highC (in coff);
            // split sp stores its partial sp * split_stride elements further on
            const uint64_t base = (warp_pdep64(rt, e.highR) | warp_pdep64(ct * SUBS, e.highC)) +
                                  (uint64_t)sp * (uint64_t)P.split_stride;
            // one half chunk (16 columns) at a time: 16 values in registers
            // keep the warp under its 96-register share without spills; the
            // accumulator is freed once the last half has been loaded
#pragma unroll
            for (int c = 0; c < 2 * CH; ++c) {
                uint32_t r[16];
                tmem_ld16(tmem_base + ((uint32_t)(lane_grp * 32) << 16) +
                              (uint32_t)(acc * BN + (q + 4 * (c >> 1)) * 32 + (c & 1) * 16), r);
                if (c == 2 * CH - 1) {
                    tc_fence_before();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&tempty[acc]);
                }
                direct_run32_any<16>(e, vw, base + grow + coff[c >> 1] + ((c & 1) ? off16 : 0), mstep, r, sf, sd);
            }
        }
    } else {
        // ------------------------------------------------ epilogue
        // Software pipeline over 128 x 64 sub-tiles (BN / 64 per MMA tile):
        // iteration k writes sub-tile k out of one staging buffer while the
        // staging warps (warpgroups 0 and 1, one 32-column chunk each) move
        // sub-tile k+1 from TMEM into the other buffer.
        constexpr int SUBS = BN / C::SUB_N;
        const int wg = (warp - 2) >> 2;         // warpgroup 0..3
        const int lane_grp = warp & 3;          // TMEM lanes this warp may read
        const int row = lane_grp * 32 + lane;   // accumulator row
        const int etid = threadIdx.x - 64;      // 0..EPI_THREADS-1
        const int Me = 1 << e.a_bits, Ne = 1 << e.b_bits;
        const int E = Me * Ne;
        const int pitch = P.rowmajor ? C::PITCH_R : C::PITCH_C;
        float *stgbuf[2] = {stg, stg + C::STG_FLOATS};
        epi_tables_init(tb, e, P.rowmajor != 0, pitch, etid, EPI_THREADS);
        // bit positions of the result bits that carry the tile indices
        int8_t(*pos)[64] = (int8_t(*)[64])tb_pos;
        int *npos = (int *)(tb_pos + 128);
        if (etid < 2) {
            uint64_t m = etid == 0 ? e.highR : e.highC;
            int n = 0;
            while (m) {
                pos[etid][n++] = (int8_t)__ffsll((long long)m) - 1;
                m &= m - 1;
            }
            npos[etid] = n;
        }
        asm volatile("bar.sync 1, %0;" ::"n"(EPI_THREADS) : "memory");
        // Full sub-tiles: the staging and destination offsets of this thread's
        // runs are the same for every sub-tile, so they live in registers.
        constexpr int ITERS = BM * C::SUB_N / (4 * EPI_THREADS);
        const bool reg_path = E == BM * C::SUB_N && e.L >= 2 && P.gmode != G_SCALAR && (e.tileMask >> 32) == 0;
        uint32_t r_s0[ITERS], r_s1[ITERS], r_g[ITERS];
        if (reg_path) {
#pragma unroll
            for (int it = 0; it < ITERS; ++it) {
                const int t = (etid + it * EPI_THREADS) * 4;
                const uint32_t sh = tb->s_hi[t >> 7];
                const int tl = t & 127;
                r_s0[it] = sh + tb->s_lo[tl];
                r_s1[it] = sh + tb->s_lo[tl + (P.gmode == G_PAIR01 ? 2 : 1)];
                r_g[it] = (uint32_t)(tb->g_hi[t >> 7] + tb->g_lo[tl]);
            }
        }
        const double sc = (e.mode == EPI_OUT_F32 || e.mode == EPI_OUT_F64) ? e.zinfo[1] : 1.0;
        const int64_t my_tiles =
            (int64_t)blockIdx.x < P.n_tiles ? (P.n_tiles - 1 - (int64_t)blockIdx.x) / gridDim.x + 1 : 0;
        const int64_t n_sub = my_tiles * SUBS;
        // stage sub-tile k into buffer k & 1 (staging warps only); returns false on abort
        auto stage_sub = [&](int64_t k) {
            const int64_t lt = k / SUBS;
            const int h = (int)(k % SUBS);
            const int acc = (int)(lt & 1);
            if (h == 0) {
                if (lane == 0) mbar_wait(&tfull[acc], (uint32_t)((lt >> 1) & 1), abort_flag);
                __syncwarp();
                tc_fence_after();
            }
            if (*abort_flag) return;
            float *sb = stgbuf[k & 1];
            const int col0 = wg * 32;  // column chunk of this warpgroup inside the sub-tile
            uint32_t r[32];
            tmem_ld32(tmem_base + ((uint32_t)(lane_grp * 32) << 16) + (uint32_t)(acc * BN + h * C::SUB_N + col0), r);
            if (row < Me) {
                if (P.rowmajor) {
                    float *dst = sb + row * C::PITCH_R + col0;
#pragma unroll
                    for (int j = 0; j < 32; j += 4)
                        if (col0 + j < Ne)
                            *(float4 *)(dst + j) = make_float4(__uint_as_float(r[j]), __uint_as_float(r[j + 1]),
                                                               __uint_as_float(r[j + 2]), __uint_as_float(r[j + 3]));
                } else {
#pragma unroll
                    for (int j = 0; j < 32; ++j)
                        if (col0 + j < Ne) sb[(col0 + j) * C::PITCH_C + row] = __uint_as_float(r[j]);
                }
            }
            if (h == SUBS - 1) {  // last read of this accumulator by this warp
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&tempty[acc]);
            }
        };
        // Base offset of a sub-tile, computed by one warp: lane l deposits bit
        // l (and l + 32) of the row / column tile index, then an OR reduction.
        auto sub_base_warp = [&](int64_t k) {
            const int64_t tile = (int64_t)blockIdx.x + (k / SUBS) * gridDim.x;
            const uint64_t rt = (uint64_t)(tile / P.col_tiles);
            const uint64_t ct = (uint64_t)((tile - (int64_t)rt * P.col_tiles) * SUBS + k % SUBS);
            uint64_t v = 0;
#pragma unroll
            for (int hw = 0; hw < 2; ++hw) {
                const int b = lane + 32 * hw;
                if (b < npos[0] && ((rt >> b) & 1)) v |= 1ull << pos[0][b];
                if (b < npos[1] && ((ct >> b) & 1)) v |= 1ull << pos[1][b];
            }
            const uint32_t lo = __reduce_or_sync(0xffffffffu, (uint32_t)v);
            const uint32_t hi = __reduce_or_sync(0xffffffffu, (uint32_t)(v >> 32));
            return ((uint64_t)hi << 32) | lo;
        };
        if (n_sub > 0) {
            if (wg < 2) stage_sub(0);
            if (etid < 32) {
                const uint64_t b = sub_base_warp(0);
                if (etid == 0) tile_base_slot[0] = b;
            }
        }
        bool stop = epi_barrier_or(EPI_THREADS, *abort_flag != 0);
        for (int64_t k = 0; k < n_sub && !stop; ++k) {
            if (k + 1 < n_sub) {
                if (wg < 2) stage_sub(k + 1);
                if (etid < 32) {
                    const uint64_t b = sub_base_warp(k + 1);
                    if (etid == 0) tile_base_slot[(k + 1) & 1] = b;
                }
            }
            const float *cur = stgbuf[k & 1];
            const uint64_t base = tile_base_slot[k & 1];
            if (reg_path) {
#pragma unroll
                for (int it = 0; it < ITERS; ++it) {
                    float v[4];
                    if (P.gmode == G_VEC4) {
                        const float4 q = *(const float4 *)(cur + r_s0[it]);
                        v[0] = q.x;
                        v[1] = q.y;
                        v[2] = q.z;
                        v[3] = q.w;
                    } else {
                        const float2 a = *(const float2 *)(cur + r_s0[it]);
                        const float2 b = *(const float2 *)(cur + r_s1[it]);
                        if (P.gmode == G_PAIR01) {
                            v[0] = a.x;
                            v[1] = a.y;
                            v[2] = b.x;
                            v[3] = b.y;
                        } else {
                            v[0] = a.x;
                            v[1] = b.x;
                            v[2] = a.y;
                            v[3] = b.y;
                        }
                    }
                    store_run_f32(e, base + r_g[it], v, 4, sc);
                }
            } else {
                epi_readout_rt(tb, cur, e, base, E, etid, EPI_THREADS, P.gmode);
            }
            stop = epi_barrier_or(EPI_THREADS, *abort_flag != 0);
        }
    }
    __syncthreads();
    if (threadIdx.x == 0 && *abort_flag && P.err) atomicExch(P.err, 1);
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base),
                     "r"((uint32_t)C::TMEM_COLS)
                     : "memory");
    }
}

PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
std::once_flag g_encode_once;

cudaError_t get_encode() {
    std::call_once(g_encode_once, [] {
        void *fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            g_encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
    });
    return g_encode ? cudaSuccess : cudaErrorNotSupported;
}

// K-major operand of `rows` rows of `k` elements, box = (bk elements,
// box_rows), bk * elem bytes (128 or 64) swizzled over that span.  Row-major
// operands are 2-D (k, rows); K-blocked ones ([k / 64][rows][64]) are 3-D
// (64, rows, k / 64) with a box one block deep.
cudaError_t encode(CUtensorMap *m, const void *ptr, int elem, uint64_t k, uint64_t rows, uint32_t bk,
                   uint32_t box_rows, bool kblk = false) {
    const uint32_t span = bk * (uint32_t)elem;
    if (span != 128 && span != 64) return cudaErrorInvalidValue;
    if (!ptr || ((uintptr_t)ptr & 15) || rows > (1ull << 32)) return cudaErrorInvalidValue;
    if (kblk && (k % 64 != 0 || bk > 64)) return cudaErrorInvalidValue;
    cuuint64_t dims[3] = {k, rows, 1};
    cuuint64_t strides[2] = {k * (uint64_t)elem, 0};
    cuuint32_t box[3] = {bk, box_rows, 1};
    cuuint32_t estr[3] = {1, 1, 1};
    if (kblk) {
        dims[0] = 64;
        dims[2] = k / 64;
        strides[0] = 64 * (uint64_t)elem;
        strides[1] = rows * 64 * (uint64_t)elem;
    }
    CUresult r = g_encode(m, elem == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16,
                          kblk ? 3 : 2, const_cast<void *>(ptr), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                          span == 128 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

template <int BN, int KIND, bool DEEP>
cudaError_t launch_kind(const StepArgs &a, int *d_err, cudaStream_t s) {
    using C = Cfg<BN, KIND, DEEP>;
    constexpr int lbn = BN == 256 ? 8 : (BN == 128 ? 7 : 6);
    // the direct epilogue writes whole 128 x BN tiles
    if (DEEP && (a.epi.a_bits != 7 || a.epi.b_bits != 6 || a.nb < lbn)) return cudaErrorInvalidValue;
    cudaError_t e = get_encode();
    if (e != cudaSuccess) return e;
    static bool attr = false;
    if (!attr) {
        e = cudaFuncSetAttribute(umma_step_kernel<BN, KIND, DEEP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 C::SMEM);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    const uint64_t M = 1ull << a.mb, N = 1ull << a.nb, K = 1ull << a.kb;
    // Long K loops take 64-byte k-blocks: stages of half the bytes, so twice
    // as many copies are in flight ahead of the tensor pipe.  Not for rows
    // longer than 64 KB: a box then spans many pages, and twice the boxes
    // per byte cost more in address translation than the deeper ring gains.
    const bool sw64 = DEEP && KIND != K_TF32 && !a.kblk && K >= ((uint64_t)1 << SW64_MIN_LOG2_K) &&
                      K * C::ELEM <= ((uint64_t)1 << 16);
    const uint32_t bk = (sw64 ? 64 : 128) / C::ELEM;
    if (K < (uint64_t)bk) return cudaErrorInvalidValue;
    CUtensorMap tA, tB, tAl, tBl;
    const bool kb3 = a.kblk != 0;
    if ((e = encode(&tA, a.A, C::ELEM, K, M, bk, BM, kb3)) != cudaSuccess) return e;
    if ((e = encode(&tB, a.B, C::ELEM, K, N, bk, BN, kb3)) != cudaSuccess) return e;
    if (KIND == K_BF16X3) {
        if ((e = encode(&tAl, a.A_lo, C::ELEM, K, M, bk, BM, kb3)) != cudaSuccess) return e;
        if ((e = encode(&tBl, a.B_lo, C::ELEM, K, N, bk, BN, kb3)) != cudaSuccess) return e;
    } else {
        tAl = tA;
        tBl = tB;
    }
    UmmaParams p;
    p.epi = a.epi;
    // MMA tiles are 128 x BN; the epilogue parameters describe 128 x 64 sub-tiles
    if (BN >= 128 && a.nb < lbn) return cudaErrorInvalidValue;
    const int64_t row_tiles = (int64_t)1 << (a.mb - a.epi.a_bits);
    p.col_tiles = a.nb >= lbn ? (int64_t)1 << (a.nb - lbn) : 1;
    p.n_tiles = row_tiles * p.col_tiles;
    p.k_blocks = (int)(K / bk);
    p.sw64 = sw64;
    p.kblk = kb3;
    // K split (deep form): every split needs at least one k-block, and its
    // partial is stored as FP32
    if (a.ksplit < 1 || a.ksplit > p.k_blocks || (a.ksplit > 1 && (!DEEP || a.epi.mode != EPI_F32)))
        return cudaErrorInvalidValue;
    p.ksplit = a.ksplit;
    p.n_units = p.n_tiles * a.ksplit;
    p.split_stride = a.ksplit > 1 ? a.split_stride : 0;
    p.bres = DEEP && p.k_blocks == 1 && p.col_tiles == 1;
    const StagePick pk = pick_staging(a.epi.lowRc, a.epi.lowCc);
    p.rowmajor = pk.rowmajor;
    p.gmode = pk.gmode;
    p.err = d_err;
    p.stall = g_umma_stall.load(std::memory_order_relaxed);
    const int64_t grid = std::min<int64_t>(p.n_units, sm_count());
    umma_step_kernel<BN, KIND, DEEP><<<(unsigned)grid, NTHREADS, C::SMEM, s>>>(tA, tB, tAl, tBl, p);
    return cudaGetLastError();
}

template <int BN, bool DEEP>
cudaError_t launch_bn(int prec, const StepArgs &a, int *d_err, cudaStream_t s) {
    switch (prec) {
        case TQC_PREC_BF16: return launch_kind<BN, K_BF16, DEEP>(a, d_err, s);
        case TQC_PREC_BF16X3: return launch_kind<BN, K_BF16X3, DEEP>(a, d_err, s);
        case TQC_PREC_TF32: return launch_kind<BN, K_TF32, DEEP>(a, d_err, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace

// Tensor maps of a step's operands for a 128 x bn MMA tile (the batched
// launch builds them once at set-up): maps[0..3] = A, B, A lo, B lo.
cudaError_t umma_make_maps(int prec, const StepArgs &a, int bn, void *maps_out) {
    cudaError_t e = get_encode();
    if (e != cudaSuccess) return e;
    CUtensorMap *m = (CUtensorMap *)maps_out;
    const int elem = prec == TQC_PREC_TF32 ? 4 : 2;
    const uint32_t bk = 128 / elem;
    const uint64_t M = 1ull << a.mb, N = 1ull << a.nb, K = 1ull << a.kb;
    if (K < bk) return cudaErrorInvalidValue;
    const bool kb3 = a.kblk != 0;
    if ((e = encode(&m[0], a.A, elem, K, M, bk, BM, kb3)) != cudaSuccess) return e;
    if ((e = encode(&m[1], a.B, elem, K, N, bk, (uint32_t)bn, kb3)) != cudaSuccess) return e;
    if (prec == TQC_PREC_BF16X3) {
        if ((e = encode(&m[2], a.A_lo, elem, K, M, bk, BM, kb3)) != cudaSuccess) return e;
        if ((e = encode(&m[3], a.B_lo, elem, K, N, bk, (uint32_t)bn, kb3)) != cudaSuccess) return e;
    } else {
        m[2] = m[0];
        m[3] = m[1];
    }
    return cudaSuccess;
}

// Epilogue tile of every configuration (the MMA tile is 128 x 64, 128 x 128 or 128 x 256).
TileShape umma_tile(int cfg) {
    (void)cfg;
    return TileShape{7, 6};
}

cudaError_t launch_umma_step(int cfg, int prec, const StepArgs &a, int *d_err, cudaStream_t s) {
    switch (cfg) {
        case UMMA_128x64: return launch_bn<64, false>(prec, a, d_err, s);
        case UMMA_128x128: return launch_bn<128, false>(prec, a, d_err, s);
        case UMMA_128x128_DEEP: return launch_bn<128, true>(prec, a, d_err, s);
        case UMMA_128x256_DEEP: return launch_bn<256, true>(prec, a, d_err, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace tqc

extern "C" tqc_status tqc_step_inject_stall(int32_t enable) {
    tqc::g_umma_stall.store(enable ? 1 : 0, std::memory_order_relaxed);
    tqc::fused_set_stall(enable);
    return TQC_OK;
}
