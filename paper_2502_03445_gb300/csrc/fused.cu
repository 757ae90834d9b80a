// Fused pair of consecutive tensor-core steps for sm_103a.
//
// Step s computes C0 = A0 B0^T (K0 = 64) and step s + 1 computes
// C1 = C0' B1^T (K1 = 256, N1 = 128), where C0' is C0 in step s + 1's
// operand layout: K1 lowest, then the rows of step s + 1 (§III-B: the
// result of one pairwise contraction is an operand of the next).  When the
// planner's layouts line up -- the 7 lowest row bits of A0 and the 8 lowest
// column bits of B0 land on the 15 lowest bits of C0', with B0's column bits
// 0..3 on C0' bits 0, 1, 6, 7 -- every 128 x 256 tile of C0 is exactly one
// 128-row tile of C0' with all of K1.  The pair then runs as one kernel and
// the intermediate C0 never reaches HBM:
//
//   per unit (one 128-row tile of step s + 1)
//     TMA      A0 tile (128 x 64) and B0 tile (256 x 64), split-BF16 planes
//     MMA      D0 = A0 B0^T into tensor memory (128 x 256, FP32)
//     convert  D0 -> BF16 hi / lo planes of the 4 k-blocks of the C0' tile
//              (64 K each) in 128-byte-swizzled shared memory, one k-block
//              at a time, following the bit permutation above
//     MMA      D1 += C0'_j B1_j^T, j = 0..3 (B1 k-blocks by TMA)
//     store    D1 (128 x 128) -> step s + 1's result through the direct
//              epilogue (its own output mode and layout)
//
// Roles (608 threads, one CTA per SM, persistent over units): warp 0 copies
// A0/B0, warp 1 issues MMAs, warp 2 copies B1 k-blocks, warps 3-10 convert
// (two per tensor-memory lane group, each taking half of the column runs),
// warps 11-18 store.  Tensor memory: D0 (256 columns) and a double-buffered
// D1 (2 x 128).  Shared memory: A0/B0 96 KB, B1 and C0' k-block rings of two
// 32 KB slots each.  Every wait is bounded; a wait that gives up raises the
// CTA's abort flag and the error word, drains the copies and MMAs in flight,
// frees tensor memory and returns.
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

constexpr int F_THREADS = 608;
constexpr int F_CONVERT0 = 3;   // first convert warp
constexpr int F_CONVERT_WARPS = 8;
constexpr int F_EPI0 = F_CONVERT0 + F_CONVERT_WARPS;  // first store warp
constexpr int F_EPI_WARPS = 8;
constexpr int A0_BYTES = 128 * 128;         // one plane: 128 rows x 64 bf16
constexpr int B0_BYTES = 256 * 128;
constexpr int KB_BYTES = 128 * 128;         // one plane of a 128-row k-block
constexpr int OFF_A0 = 0;                   // hi, lo
constexpr int OFF_B0 = 2 * A0_BYTES;        // hi, lo
constexpr int OFF_B1 = OFF_B0 + 2 * B0_BYTES;       // 2 slots x (hi, lo)
constexpr int OFF_A1 = OFF_B1 + 2 * 2 * KB_BYTES;   // 2 slots x (hi, lo)
constexpr int OFF_BAR = OFF_A1 + 2 * 2 * KB_BYTES;
constexpr int F_SMEM = 1024 + OFF_BAR + 512;
static_assert(F_SMEM <= 232448, "shared memory per CTA");
// instruction descriptors: D = F32, A/B = BF16, K-major, N >> 3, M >> 4
constexpr uint32_t IDESC0 = (1u << 4) | (1u << 7) | (1u << 10) | ((256u >> 3) << 17) | ((128u >> 4) << 24);
constexpr uint32_t IDESC1 = (1u << 4) | (1u << 7) | (1u << 10) | ((128u >> 3) << 17) | ((128u >> 4) << 24);

struct FusedParams {
    int64_t n_units;          // 128-row tiles of step s + 1
    uint64_t maskR0, maskC0;  // C0' bits of A0's row bits and of B0's column bits
    uint32_t dC[16];          // C0' bits of B0 column bits 4..7 (run m): pdep(m << 4, maskC0)
    EpiParams epi1;           // step s + 1's epilogue (128 x 64 sub-tiles)
    int stall;                // test hook: CTA 0 never issues its first A0/B0 copy
    int *err;
};

__device__ __forceinline__ uint64_t pext64(uint64_t x, uint64_t m) {
    uint64_t r = 0;
    int k = 0;
    while (m) {
        const uint64_t low = m & (~m + 1);
        if (x & low) r |= 1ull << k;
        ++k;
        m ^= low;
    }
    return r;
}

__device__ __forceinline__ void fence_async_shared() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__global__ void __launch_bounds__(F_THREADS, 1)
    fused_pair_kernel(const __grid_constant__ CUtensorMap tA0, const __grid_constant__ CUtensorMap tA0l,
                      const __grid_constant__ CUtensorMap tB0, const __grid_constant__ CUtensorMap tB0l,
                      const __grid_constant__ CUtensorMap tB1, const __grid_constant__ CUtensorMap tB1l,
                      const FusedParams P) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint64_t *bar = (uint64_t *)(smem + OFF_BAR);
    uint64_t *ab_full = bar + 0, *ab_empty = bar + 1;
    uint64_t *b1_full = bar + 2, *b1_empty = bar + 4;   // [2] each
    uint64_t *a1_full = bar + 6, *a1_empty = bar + 8;   // [2] each
    uint64_t *d0_full = bar + 10, *d0_empty = bar + 11;
    uint64_t *d1_full = bar + 12, *d1_empty = bar + 14;  // [2] each
    uint64_t *drain = bar + 16;
    uint32_t *tmem_slot = (uint32_t *)(bar + 17);
    volatile int *abort_flag = (volatile int *)(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        mbar_init(ab_full, 1);
        mbar_init(ab_empty, 1);
        for (int i = 0; i < 2; ++i) {
            mbar_init(&b1_full[i], 1);
            mbar_init(&b1_empty[i], 1);
            mbar_init(&a1_full[i], F_CONVERT_WARPS);
            mbar_init(&a1_empty[i], 1);
            mbar_init(&d1_full[i], 1);
            mbar_init(&d1_empty[i], F_EPI_WARPS);
        }
        mbar_init(d0_full, 1);
        mbar_init(d0_empty, F_CONVERT_WARPS);
        mbar_init(drain, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(512u)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;

    if (warp == 0) {
        // ------------------------------------------------ A0 / B0 copies
        if (lane == 0) {
            int64_t lt = 0;
            bool ok = true, issued = false, skipped = false;
            for (int64_t u = blockIdx.x; u < P.n_units; u += gridDim.x, ++lt) {
                if (!mbar_wait(ab_empty, (uint32_t)((lt & 1) ^ 1), abort_flag)) {
                    ok = false;
                    break;
                }
                if (P.stall && blockIdx.x == 0 && lt == 0) {  // test hook: this unit's operands never arrive
                    skipped = true;
                    continue;
                }
                const uint64_t t = (uint64_t)u << 15;  // C0' index of the unit's first element
                const int rt0 = (int)(pext64(t, P.maskR0) >> 7), ct0 = (int)(pext64(t, P.maskC0) >> 8);
                mbar_expect_tx(ab_full, 2 * (A0_BYTES + B0_BYTES));
                tma_load_2d(smem + OFF_A0, &tA0, 0, rt0 * 128, ab_full);
                tma_load_2d(smem + OFF_A0 + A0_BYTES, &tA0l, 0, rt0 * 128, ab_full);
                tma_load_2d(smem + OFF_B0, &tB0, 0, ct0 * 256, ab_full);
                tma_load_2d(smem + OFF_B0 + B0_BYTES, &tB0l, 0, ct0 * 256, ab_full);
                issued = true;
            }
            if ((!ok || skipped) && issued) {  // drain the last copy if it was issued
                long long t0 = clock64();
                while (!mbar_try_wait(ab_full, (uint32_t)((lt - 1) & 1)) && clock64() - t0 < WAIT_CYCLES) {
                }
            }
        }
    } else if (warp == 2) {
        // ------------------------------------------------ B1 k-block copies
        if (lane == 0) {
            int64_t it = 0;
            bool ok = true;
            for (int64_t u = blockIdx.x; ok && u < P.n_units; u += gridDim.x) {
                for (int j = 0; j < 4; ++j, ++it) {
                    const int sl = (int)(it & 1);
                    if (!mbar_wait(&b1_empty[sl], (uint32_t)(((it >> 1) & 1) ^ 1), abort_flag)) {
                        ok = false;
                        break;
                    }
                    uint8_t *dst = smem + OFF_B1 + sl * 2 * KB_BYTES;
                    mbar_expect_tx(&b1_full[sl], 2 * KB_BYTES);
                    tma_load_2d(dst, &tB1, 64 * j, 0, &b1_full[sl]);
                    tma_load_2d(dst + KB_BYTES, &tB1l, 64 * j, 0, &b1_full[sl]);
                }
            }
            if (!ok) {
                for (int64_t j = it > 2 ? it - 2 : 0; j < it; ++j) {
                    long long t0 = clock64();
                    while (!mbar_try_wait(&b1_full[j & 1], (uint32_t)((j >> 1) & 1)) && clock64() - t0 < WAIT_CYCLES) {
                    }
                }
            }
        }
    } else if (warp == 1) {
        // ------------------------------------------------ MMA issuer
        // The next unit's step-s MMAs are issued ahead of this unit's last
        // k-block of step s + 1 (as soon as the convert warps have read all
        // of D0), so the tensor pipe has that k-block's MMAs to run while the
        // convert warps start on the next D0; issued in unit order, the pipe
        // would idle for the first k-block's conversion of every unit.
        if (lane == 0) {
            int64_t lt = 0, itb = 0;
            bool ok = true;
            const uint32_t d0 = tmem_base;
            // step s: D0 = A0 B0^T for the unit with sequence number n
            auto issue_step0 = [&](int64_t n) -> bool {
                if (!mbar_wait(ab_full, (uint32_t)(n & 1), abort_flag) ||
                    !mbar_wait(d0_empty, (uint32_t)((n & 1) ^ 1), abort_flag))
                    return false;
                tc_fence_after();
                const uint32_t a = smem_u32(smem + OFF_A0), al = a + A0_BYTES;
                const uint32_t b = smem_u32(smem + OFF_B0), bl = b + B0_BYTES;
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const uint64_t da = umma_desc(a + 32 * k, 128), db = umma_desc(b + 32 * k, 128);
                    umma<K_BF16X3>(d0, da, db, IDESC0, k != 0);
                    umma<K_BF16X3>(d0, da, umma_desc(bl + 32 * k, 128), IDESC0, 1u);
                    umma<K_BF16X3>(d0, umma_desc(al + 32 * k, 128), db, IDESC0, 1u);
                }
                umma_commit(ab_empty);
                umma_commit(d0_full);
                return true;
            };
            if ((int64_t)blockIdx.x < P.n_units) ok = issue_step0(0);
            for (int64_t u = blockIdx.x; ok && u < P.n_units; u += gridDim.x, ++lt) {
                // step s + 1: D1 = sum_j C0'_j B1_j^T
                const int acc = (int)(lt & 1);
                const uint32_t d1 = tmem_base + 256u + (uint32_t)(acc * 128);
                if (!mbar_wait(&d1_empty[acc], (uint32_t)(((lt >> 1) & 1) ^ 1), abort_flag)) {
                    ok = false;
                    break;
                }
                for (int j = 0; j < 4; ++j, ++itb) {
                    if (j == 3 && u + gridDim.x < P.n_units && !issue_step0(lt + 1)) {
                        ok = false;
                        break;
                    }
                    const int sl = (int)(itb & 1);
                    const uint32_t ph = (uint32_t)((itb >> 1) & 1);
                    if (!mbar_wait(&b1_full[sl], ph, abort_flag) || !mbar_wait(&a1_full[sl], ph, abort_flag)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t a = smem_u32(smem + OFF_A1 + sl * 2 * KB_BYTES), al = a + KB_BYTES;
                    const uint32_t b = smem_u32(smem + OFF_B1 + sl * 2 * KB_BYTES), bl = b + KB_BYTES;
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        const uint64_t da = umma_desc(a + 32 * k, 128), db = umma_desc(b + 32 * k, 128);
                        umma<K_BF16X3>(d1, da, db, IDESC1, (j | k) != 0);
                        umma<K_BF16X3>(d1, da, umma_desc(bl + 32 * k, 128), IDESC1, 1u);
                        umma<K_BF16X3>(d1, umma_desc(al + 32 * k, 128), db, IDESC1, 1u);
                    }
                    umma_commit(&b1_empty[sl]);
                    umma_commit(&a1_empty[sl]);
                }
                if (ok) umma_commit(&d1_full[acc]);
            }
            umma_commit(drain);  // every MMA issued so far has completed once this arrives
            long long t0 = clock64();
            while (!mbar_try_wait(drain, 0) && clock64() - t0 < WAIT_CYCLES) {
            }
        }
    } else if (warp < F_EPI0) {
        // ------------------------------------------------ convert D0 -> C0' k-blocks
        // lane: D0 row r0 (tensor-memory lane); its C0' bits from A0's row bits;
        // the warp takes column runs 8 half .. 8 half + 7 of every k-block
        const int lane_grp = warp & 3, half = (warp - F_CONVERT0) >> 2;
        const int r0 = lane_grp * 32 + lane;
        const uint32_t dR = (uint32_t)pdep64((uint64_t)r0, P.maskR0);
        const uint32_t lane_addr = (uint32_t)(lane_grp * 32) << 16;
        int64_t lt = 0, ita = 0;
        for (int64_t u = blockIdx.x; u < P.n_units; u += gridDim.x, ++lt) {
            if (lane == 0) mbar_wait(d0_full, (uint32_t)(lt & 1), abort_flag);
            __syncwarp();
            if (*abort_flag) break;
            tc_fence_after();
            bool stop = false;
            for (int j = 0; j < 4; ++j, ++ita) {
                const int sl = (int)(ita & 1);
                if (lane == 0) mbar_wait(&a1_empty[sl], (uint32_t)(((ita >> 1) & 1) ^ 1), abort_flag);
                __syncwarp();
                if (*abort_flag) {
                    stop = true;
                    break;
                }
                uint8_t *hi = smem + OFF_A1 + sl * 2 * KB_BYTES, *lo = hi + KB_BYTES;
                // runs of 4 D0 columns (c0 = 16 m + 4 j + i): C0' row r1 = t >> 8, k = t & 63
                {
                    uint32_t v[8][4];
#pragma unroll
                    for (int mm = 0; mm < 8; ++mm)
                        tmem_ld4_nowait(tmem_base + lane_addr + (uint32_t)(((half * 8 + mm) << 4) + (j << 2)), v[mm]);
                    tmem_wait_ld16(v[0], v[1], v[2], v[3]);  // the wait carries the loaded registers, so
                    tmem_wait_ld16(v[4], v[5], v[6], v[7]);  // no use of them is scheduled before it
#pragma unroll
                    for (int mm = 0; mm < 8; ++mm) {
                        const uint32_t t = dR | P.dC[half * 8 + mm] | ((uint32_t)j << 6);
                        const uint32_t r1 = t >> 8, k = t & 63u;
                        const uint32_t off = r1 * 128u + ((((k >> 3) ^ (r1 & 7u)) << 4) | ((k & 7u) * 2u));
                        float h[4], l[4];
#pragma unroll
                        for (int i = 0; i < 4; ++i) {
                            const float x = __uint_as_float(v[mm][i]);
                            const __nv_bfloat16 b = __float2bfloat16_rn(x);
                            h[i] = __bfloat162float(b);
                            l[i] = x - h[i];
                        }
                        *(uint2 *)(hi + off) = make_uint2(pack_bf16x2(h[0], h[1]), pack_bf16x2(h[2], h[3]));
                        *(uint2 *)(lo + off) = make_uint2(pack_bf16x2(l[0], l[1]), pack_bf16x2(l[2], l[3]));
                    }
                }
                if (j == 3) {  // every D0 column of this unit is in registers or shared memory
                    tc_fence_before();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(d0_empty);
                }
                fence_async_shared();  // generic-proxy stores -> visible to the tensor cores
                __syncwarp();
                if (lane == 0) mbar_arrive(&a1_full[sl]);
            }
            if (stop) break;
        }
    } else {
        // ------------------------------------------------ store D1 (direct epilogue)
        const EpiParams &e = P.epi1;
        const int lane_grp = warp & 3, h = (warp - F_EPI0) >> 2;  // columns 64 h .. 64 h + 63
        const int row = lane_grp * 32 + lane;
        const uint64_t grow = pdep64((uint64_t)pdep32((uint32_t)row, e.lowRc), e.tileMask);
        const uint64_t colmask = pdep64((uint64_t)e.lowCc, e.tileMask);
        const int vw = ((e.lowCc & 3u) == 3u && e.L >= 2) ? 4 : ((e.lowCc & 1u) && e.L >= 1 ? 2 : 1);
        const uint64_t mstep = vw == 4 ? colmask & (colmask - 1) & ((colmask & (colmask - 1)) - 1)
                                       : (vw == 2 ? colmask & (colmask - 1) : colmask);
        uint64_t coff[2];  // the warp's two 32-column chunks: sub-tile h, columns 0 and 32
#pragma unroll
        for (int c = 0; c < 2; ++c) coff[c] = pdep64((uint64_t)(32 * c), colmask) | pdep64((uint64_t)h, e.highC);
        const uint64_t off16 = pdep64(16, colmask);
        int64_t lt = 0;
        for (int64_t u = blockIdx.x; u < P.n_units; u += gridDim.x, ++lt) {
            const int acc = (int)(lt & 1);
            if (lane == 0) mbar_wait(&d1_full[acc], (uint32_t)((lt >> 1) & 1), abort_flag);
            __syncwarp();
            if (*abort_flag) break;
            tc_fence_after();
            const uint64_t base = warp_pdep64((uint64_t)u, e.highR);  // one column tile (N = 128)
#pragma unroll
            for (int c = 0; c < 4; ++c) {  // 16 columns at a time
                uint32_t r[16];
                tmem_ld16(tmem_base + ((uint32_t)(lane_grp * 32) << 16) +
                              (uint32_t)(256 + acc * 128 + h * 64 + (c >> 1) * 32 + (c & 1) * 16),
                          r);
                if (c == 3) {
                    tc_fence_before();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&d1_empty[acc]);
                }
                direct_run32_any<16>(e, vw, base + grow + coff[c >> 1] + ((c & 1) ? off16 : 0), mstep, r, 1.0f, 1.0);
            }
        }
    }
    __syncthreads();
    if (threadIdx.x == 0 && *abort_flag && P.err) atomicExch(P.err, 1);
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(512u) : "memory");
    }
}

}  // namespace

// Whether steps s and s + 1 of a plan can run as one fused kernel: both
// split-BF16 tensor-core steps on row-major operands, the first with
// K = 64 and at least 128 x 256 results, writing the row operand of the
// second (K = 256, N = 128, not the last step); the bit alignment described
// at the top of this file; the same slice dependence.
bool fused_pair_ok(const Plan &p, size_t s) {
    if (s + 1 >= p.steps.size()) return false;
    const StepPlan &a = p.steps[s], &b = p.steps[s + 1];
    if (a.klass != KC_UMMA || b.klass != KC_UMMA || a.prec != TQC_PREC_BF16X3 || b.prec != TQC_PREC_BF16X3)
        return false;
    if (a.kblk || b.kblk || a.final || b.final || b.a != a.c) return false;
    if (a.kb != 6 || a.mb < 7 || a.nb < 8 || b.kb != 8 || b.nb != 7 || b.mb < 7) return false;
    if (p.tensors[(size_t)a.c].slice_dep != p.tensors[(size_t)b.c].slice_dep) return false;
    auto pdep = [](uint64_t src, uint64_t mask) {
        uint64_t r = 0;
        while (mask) {
            const uint64_t low = mask & (~mask + 1);
            if (src & 1) r |= low;
            src >>= 1;
            mask ^= low;
        }
        return r;
    };
    if ((pdep(0x7f, a.maskR) | pdep(0xff, a.maskC)) != 0x7fffu) return false;  // the 15 lowest bits of C0'
    return pdep(0xf, a.maskC) == 0xC3u;  // column bits 0..3 -> C0' bits 0, 1, 6, 7
}

namespace {

std::atomic<int> g_fused_stall{0};
PFN_cuTensorMapEncodeTiled_v12000 g_enc = nullptr;
std::once_flag g_enc_once;

cudaError_t map2d(CUtensorMap *m, const void *ptr, uint64_t k, uint64_t rows, uint32_t box_rows) {
    std::call_once(g_enc_once, [] {
        void *fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            g_enc = (PFN_cuTensorMapEncodeTiled_v12000)fn;
    });
    if (!g_enc) return cudaErrorNotSupported;
    if (!ptr || ((uintptr_t)ptr & 15)) return cudaErrorInvalidValue;
    cuuint64_t dims[2] = {k, rows};
    cuuint64_t strides[1] = {k * 2};
    cuuint32_t box[2] = {64, box_rows};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = g_enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(ptr), dims, strides, box, estr,
                       CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                       CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

uint64_t host_pdep(uint64_t src, uint64_t mask) {
    uint64_t r = 0;
    while (mask) {
        const uint64_t low = mask & (~mask + 1);
        if (src & 1) r |= low;
        src >>= 1;
        mask ^= low;
    }
    return r;
}

}  // namespace

void fused_set_stall(int enable) { g_fused_stall.store(enable ? 1 : 0, std::memory_order_relaxed); }

// a0: step s's operands (its epilogue unused); a1: step s + 1's operands and
// epilogue (128 x 64 sub-tiles, output mode set); maskR0 / maskC0: step s's
// result masks.
cudaError_t launch_fused_pair(const StepArgs &a0, const StepArgs &a1, uint64_t maskR0, uint64_t maskC0, int *d_err,
                              cudaStream_t s) {
    if (a0.kb != 6 || a1.kb != 8 || a1.nb != 7 || a0.mb < 7 || a0.nb < 8 || a1.mb < 7) return cudaErrorInvalidValue;
    if (a1.epi.a_bits != 7 || a1.epi.b_bits != 6) return cudaErrorInvalidValue;
    if (!a0.A_lo || !a0.B_lo || !a1.B_lo) return cudaErrorInvalidValue;
    static bool attr = false;
    cudaError_t e;
    if (!attr) {
        e = cudaFuncSetAttribute(fused_pair_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, F_SMEM);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    CUtensorMap tA0, tA0l, tB0, tB0l, tB1, tB1l;
    const uint64_t M0 = 1ull << a0.mb, N0 = 1ull << a0.nb;
    if ((e = map2d(&tA0, a0.A, 64, M0, 128)) != cudaSuccess) return e;
    if ((e = map2d(&tA0l, a0.A_lo, 64, M0, 128)) != cudaSuccess) return e;
    if ((e = map2d(&tB0, a0.B, 64, N0, 256)) != cudaSuccess) return e;
    if ((e = map2d(&tB0l, a0.B_lo, 64, N0, 256)) != cudaSuccess) return e;
    if ((e = map2d(&tB1, a1.B, 256, 128, 128)) != cudaSuccess) return e;
    if ((e = map2d(&tB1l, a1.B_lo, 256, 128, 128)) != cudaSuccess) return e;
    FusedParams p;
    p.n_units = (int64_t)1 << (a1.mb - 7);
    p.maskR0 = maskR0;
    p.maskC0 = maskC0;
    for (int m = 0; m < 16; ++m) p.dC[m] = (uint32_t)host_pdep((uint64_t)m << 4, maskC0);
    p.epi1 = a1.epi;
    p.stall = g_fused_stall.load(std::memory_order_relaxed);
    p.err = d_err;
    const int64_t grid = std::min<int64_t>(p.n_units, sm_count());
    fused_pair_kernel<<<(unsigned)grid, F_THREADS, F_SMEM, s>>>(tA0, tA0l, tB0, tB0l, tB1, tB1l, p);
    return cudaGetLastError();
}

}  // namespace tqc
