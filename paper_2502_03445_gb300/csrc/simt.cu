// CUDA-core kernels: the plain FP32 pairwise step (also used for the small-K
// steps of the tensor-core form), its FP64 twin for the total-mass network,
// tensor ingest (bin restriction, slicing, layout permutation, cast), the
// total-mass reduction and the FP64 slice-sum finalisation.
//
// A pairwise step is the contraction of two subcircuit tensors over their
// shared cut edges (§III-B, Fig. tensor_contraction): C[r, c] = sum_k A[r, k]
// B[c, k] with A, B row-major and k (the shared cuts) contiguous.  Row and
// column indices are bit fields of the result tensor, so the epilogue stages
// each tile in shared memory in the result's bit order and writes runs of
// consecutive addresses (the Kronecker expansion of output indices, Eq.
// reconstruction, when the result is the final probability vector).
#include <algorithm>

#include "device_common.cuh"
#include "launch.h"
#include "smallk.cuh"

namespace tqc {

namespace {

template <typename T>
__device__ __forceinline__ T ld_src(const void *p, int dtype, int64_t i) {
    return dtype == TQC_F64 ? (T)((const double *)p)[i] : (T)((const float *)p)[i];
}

// One tile per iteration of a grid-stride loop over tiles.
template <int BM, int BN, int TM, int TN, int BK>
__global__ void __launch_bounds__((BM / TM) * (BN / TN))
    simt_step_f32(StepArgs args, int64_t n_tiles, int64_t col_tiles) {
    constexpr int NT = (BM / TM) * (BN / TN);
    constexpr int PA = BM + 4, PB = BN + 4, PS = BN + 4;  // padded pitches (bank spread)
    extern __shared__ __align__(16) unsigned char smem_raw[];
    EpiTables *tb = (EpiTables *)smem_raw;
    float *As = (float *)(smem_raw + sizeof(EpiTables));  // [BK][PA]
    float *Bs = As + BK * PA;                              // [BK][PB]
    float *stg = As;                                       // [BM][PS], reused after the main loop
    const EpiParams &e = args.epi;
    const int a = e.a_bits, b = e.b_bits;
    const int Me = 1 << a, Ne = 1 << b;
    const int64_t K = 1ll << args.kb;
    const int lkc = args.kb < 4 ? args.kb : 4;  // log2 of the K chunk (BK = 16)
    const int kc = 1 << lkc;
    const float *A = (const float *)args.A;
    const float *B = (const float *)args.B;
    const int tid = threadIdx.x;
    const int tx = tid % (BN / TN), ty = tid / (BN / TN);
    epi_tables_init(tb, e, true, PS, tid, NT);
    const int E = Me * Ne;
    for (int64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
        const int64_t rt = tile / col_tiles, ct = tile - rt * col_tiles;
        const int64_t r0 = rt << a, c0 = ct << b;
        float acc[TM][TN];
#pragma unroll
        for (int u = 0; u < TM; ++u)
#pragma unroll
            for (int v = 0; v < TN; ++v) acc[u][v] = 0.f;
        for (int64_t k0 = 0; k0 < K; k0 += kc) {
            for (int idx = tid; idx < (BM << lkc); idx += NT) {
                int i = idx >> lkc, kk = idx & (kc - 1);
                As[kk * PA + i] = i < Me ? A[(r0 + i) * K + k0 + kk] : 0.f;
            }
            for (int idx = tid; idx < (BN << lkc); idx += NT) {
                int j = idx >> lkc, kk = idx & (kc - 1);
                Bs[kk * PB + j] = j < Ne ? B[(c0 + j) * K + k0 + kk] : 0.f;
            }
            __syncthreads();
            for (int kk = 0; kk < kc; ++kk) {
                float af[TM], bf[TN];
#pragma unroll
                for (int u = 0; u < TM; u += 4) *(float4 *)&af[u] = *(const float4 *)&As[kk * PA + ty * TM + u];
#pragma unroll
                for (int v = 0; v < TN; v += 4) *(float4 *)&bf[v] = *(const float4 *)&Bs[kk * PB + tx * TN + v];
#pragma unroll
                for (int u = 0; u < TM; ++u)
#pragma unroll
                    for (int v = 0; v < TN; ++v) acc[u][v] = fmaf(af[u], bf[v], acc[u][v]);
            }
            __syncthreads();
        }
        // stage row-major; rows >= Me and columns >= Ne are never read back
#pragma unroll
        for (int u = 0; u < TM; ++u)
#pragma unroll
            for (int v = 0; v < TN; v += 4)
                *(float4 *)&stg[(ty * TM + u) * PS + tx * TN + v] =
                    make_float4(acc[u][v], acc[u][v + 1], acc[u][v + 2], acc[u][v + 3]);
        __syncthreads();
        epi_readout(tb, stg, e, tile_base(e, rt, ct), E, tid, NT, gather_mode(e.lowCc));
        __syncthreads();
    }
}


// Small-K step (smallk.cuh): one 128-thread CTA per tile slot, one kernel
// per K, tile width and orientation (each with its own register budget);
// when the tiles are staged, the staging tables are built once per CTA.
template <int KB, int QM, bool RM>
__global__ void __launch_bounds__(128, (QM == 1) == RM ? 8 : 6)
    simt_smallk_f32(StepArgs args, int64_t n_tiles, int64_t col_tiles, SmallkLayout L) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    EpiTables *tb = (EpiTables *)smem_raw;
    float *buf = (float *)(smem_raw + sizeof(EpiTables));
    if (!L.direct) {  // the gather's element offsets (its staging offsets are unused)
        epi_tables_init(tb, args.epi, true, 0, threadIdx.x, 128);
        __syncthreads();
    }
    smallk_tiles_body<KB, QM, RM, false>(args, tb, L, col_tiles, blockIdx.x, n_tiles, gridDim.x, buf, threadIdx.x, 1);
}

// FP64 twin for the scalar total-mass network (small; one config).
template <int BM, int BN, int TM, int TN>
__global__ void __launch_bounds__((BM / TM) * (BN / TN))
    simt_step_f64(StepArgs args, int64_t n_tiles, int64_t col_tiles) {
    constexpr int NT = (BM / TM) * (BN / TN);
    constexpr int BK = 16;
    __shared__ double As[BK * BM], Bs[BK * BN];
    __shared__ double stage[BM * BN];
    const EpiParams &e = args.epi;
    const int a = e.a_bits, b = e.b_bits;
    const int Me = 1 << a, Ne = 1 << b;
    const int64_t K = 1ll << args.kb;
    const int lkc = args.kb < 4 ? args.kb : 4;
    const int kc = 1 << lkc;
    const double *A = (const double *)args.A;
    const double *B = (const double *)args.B;
    const int tid = threadIdx.x;
    const int tx = tid % (BN / TN), ty = tid / (BN / TN);
    for (int64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
        const int64_t rt = tile / col_tiles, ct = tile - rt * col_tiles;
        const int64_t r0 = rt << a, c0 = ct << b;
        double acc[TM][TN];
        for (int u = 0; u < TM; ++u)
            for (int v = 0; v < TN; ++v) acc[u][v] = 0.0;
        for (int64_t k0 = 0; k0 < K; k0 += kc) {
            for (int idx = tid; idx < (BM << lkc); idx += NT) {
                int i = idx >> lkc, kk = idx & (kc - 1);
                As[kk * BM + i] = i < Me ? A[(r0 + i) * K + k0 + kk] : 0.0;
            }
            for (int idx = tid; idx < (BN << lkc); idx += NT) {
                int j = idx >> lkc, kk = idx & (kc - 1);
                Bs[kk * BN + j] = j < Ne ? B[(c0 + j) * K + k0 + kk] : 0.0;
            }
            __syncthreads();
            for (int kk = 0; kk < kc; ++kk)
                for (int u = 0; u < TM; ++u)
                    for (int v = 0; v < TN; ++v)
                        acc[u][v] = fma(As[kk * BM + ty * TM + u], Bs[kk * BN + tx * TN + v], acc[u][v]);
            __syncthreads();
        }
        for (int u = 0; u < TM; ++u)
            for (int v = 0; v < TN; ++v) {
                int i = ty * TM + u, j = tx * TN + v;
                if (i < Me && j < Ne) stage[pdep32(i, e.lowRc) | pdep32(j, e.lowCc)] = acc[u][v];
            }
        __syncthreads();
        const uint64_t base = tile_base(e, rt, ct);
        double *o = (double *)e.out;
        for (int t = tid; t < Me * Ne; t += NT) o[base + pdep64((uint64_t)t, e.tileMask)] = stage[t];
        __syncthreads();
    }
}

// Gather a node tensor into an operand layout: destination bit b reads
// source bit srcpos[b]; src_base carries the fixed output bits of the bin and
// the values of sliced cuts.  With reduce_bits > 0 (total mass) one warp sums
// the 2^reduce_bits consecutive source elements in FP64.
__global__ void ingest_kernel(IngestArgs g, int64_t n_dst) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    if (g.reduce_bits > 0) {
        const int lane = threadIdx.x & 31;
        const int64_t wstride = stride >> 5;
        const int64_t nx = 1ll << g.reduce_bits;
        for (int64_t d = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; d < n_dst; d += wstride) {
            int64_t s = g.src_base;
            for (int b = 0; b < g.nbits; ++b)
                if (d >> b & 1) s += 1ll << g.srcpos[b];
            double acc = 0.0;
            for (int64_t x = lane; x < nx; x += 32) acc += ld_src<double>(g.src, g.src_dtype, s + x);
            for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
            if (lane == 0) ((double *)g.dst)[d] = acc;
        }
        return;
    }
    // The grid is a power of two threads (2^lg): a thread's destination
    // indices share their lg low bits, so their part of the source offset is
    // summed once and each element adds only its bits from lg up.
    const int lg = __ffsll((long long)stride) - 1;
    const int64_t d0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t s_lo = g.src_base;
    for (int b = 0; b < g.nbits && b < lg; ++b)
        if (d0 >> b & 1) s_lo += 1ll << g.srcpos[b];
    for (int64_t d = d0; d < n_dst; d += stride) {
        int64_t s = s_lo;
        for (int b = lg; b < g.nbits; ++b)
            if (d >> b & 1) s += 1ll << g.srcpos[b];
        if (g.scaled) {
            double v = ld_src<double>(g.src, g.src_dtype, s) * g.zinfo[1];
            if (g.out_f64) ((double *)g.dst)[d] = v;
            else ((float *)g.dst)[d] = (float)v;
            continue;
        }
        const float v = ld_src<float>(g.src, g.src_dtype, s);
        switch (g.storage) {
            case ST_F32: ((float *)g.dst)[d] = v; break;
            case ST_TF32: ((float *)g.dst)[d] = to_tf32(v); break;
            case ST_BF16: ((__nv_bfloat16 *)g.dst)[d] = __float2bfloat16_rn(v); break;
            case ST_BF16X2: {
                // hi = bf16(v), lo = bf16(v - hi) from the FP32 value (v - hi is
                // exact in FP32); one FP64 conversion per element, which matters
                // on a part whose FP64 rate is a small fraction of its FP32 rate
                const __nv_bfloat16 h = __float2bfloat16_rn(v);
                ((__nv_bfloat16 *)g.dst)[d] = h;
                ((__nv_bfloat16 *)g.dst_lo)[d] = __float2bfloat16_rn(v - __bfloat162float(h));
            } break;
            case ST_F64: ((double *)g.dst)[d] = ld_src<double>(g.src, g.src_dtype, s); break;
            default: break;
        }
    }
}

// Z = sum over slices of the scalar network; scale = 2^{-|E|} / Z (or
// 2^{-|E|} without renormalisation).
__global__ void zfinal_kernel(const double *zslice, int n, int n_cuts, int renorm, double *zinfo) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double z = 0.0;
        for (int i = 0; i < n; ++i) z += zslice[i];
        double z_scaled = ldexp(z, -n_cuts);  // Z includes the 1/2 per cut
        zinfo[0] = z_scaled;
        zinfo[1] = renorm ? ldexp(1.0, -n_cuts) / z_scaled : ldexp(1.0, -n_cuts);
    }
}

__global__ void finalize_kernel(const double *acc, void *out, int out_f64, const double *zinfo, int64_t n) {
    const double s = zinfo[1];
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        double v = acc[i] * s;
        if (out_f64) ((double *)out)[i] = v;
        else ((float *)out)[i] = (float)v;
    }
}

// Sum of the FP32 partials of a K-split step (split s at part + s * n), in
// FP64, stored in the step's own output mode: the scaled final output
// (FP32 / FP64) or the FP64 slice sum (set / add).
__global__ void ksplit_reduce_kernel(const float *part, int ksplit, int64_t n, int mode, void *out,
                                     const double *zinfo) {
    const double sc = (mode == EPI_OUT_F32 || mode == EPI_OUT_F64) ? zinfo[1] : 1.0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        double v = 0.0;
        for (int s = 0; s < ksplit; ++s) v += (double)part[s * n + i];
        switch (mode) {
            case EPI_OUT_F32: ((float *)out)[i] = (float)(v * sc); break;
            case EPI_OUT_F64: ((double *)out)[i] = v * sc; break;
            case EPI_F64_SET: ((double *)out)[i] = v; break;
            case EPI_F64_ADD: ((double *)out)[i] += v; break;
            default: break;
        }
    }
}

int g_sms = 0;

template <int BM, int BN, int TM, int TN>
cudaError_t launch_cfg(const StepArgs &a, cudaStream_t s) {
    constexpr int NT = (BM / TM) * (BN / TN);
    constexpr int BK = 16;
    size_t smem = sizeof(EpiTables) + std::max((size_t)BK * (BM + 4 + BN + 4) * sizeof(float),
                                               (size_t)BM * (BN + 4) * sizeof(float));
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(simt_step_f32<BM, BN, TM, TN, BK>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    int64_t row_tiles = 1ll << (a.mb - a.epi.a_bits);
    int64_t col_tiles = 1ll << (a.nb - a.epi.b_bits);
    int64_t n_tiles = row_tiles * col_tiles;
    int64_t grid = std::min<int64_t>(n_tiles, (int64_t)sm_count() * 16);
    simt_step_f32<BM, BN, TM, TN, BK><<<(unsigned)grid, NT, smem, s>>>(a, n_tiles, col_tiles);
    return cudaGetLastError();
}

}  // namespace

int sm_count() {
    if (!g_sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&g_sms, cudaDevAttrMultiProcessorCount, dev);
        if (g_sms <= 0) g_sms = 1;
    }
    return g_sms;
}

TileShape simt_tile(int cfg) {
    switch (cfg) {
        case SIMT_128x128: return {7, 7};
        case SIMT_128x64: return {7, 6};
        default: return {6, 6};
    }
}

TileShape simt_f64_tile() { return {5, 5}; }

bool smallk_ok(int mb, int nb, int kb, bool kblk) {
    return (kb == 0 || kb == 2 || kb == 4) && !kblk && mb >= 2 && nb >= 2 && mb + nb >= 7;
}

// Start from 64 x 64, grow the side the step still has until the tile holds
// 2^12 results, then shrink the larger side until operands and staging fit
// SMALLK_BYTES.
TileShape smallk_tile(int mb, int nb, int kb) {
    int a = std::min(mb, 6), b = std::min(nb, 6);
    while (a + b < 12 && (a < mb || b < nb)) {
        if (a < mb && (a <= b || b >= nb)) ++a;
        else ++b;
    }
    auto fits = [&](int x, int y) {
        return smallk_op_bytes(x, y, kb) <= SMALLK_BYTES && smallk_stage_bytes(x, y) <= SMALLK_BYTES;
    };
    while (!fits(a, b) && (a > 2 || b > 2)) {
        if (a >= b && a > 2) --a;
        else --b;
    }
    return TileShape{a, b};
}

static uint64_t host_pdep64(uint64_t src, uint64_t mask) {
    uint64_t r = 0;
    while (mask) {
        const uint64_t low = mask & (~mask + 1);
        if (src & 1) r |= low;
        src >>= 1;
        mask ^= low;
    }
    return r;
}

// Direct stores when the result's lowest four or more bits are bits of one
// tile dimension and at least two lanes run along it (whole 32-byte sectors
// per warp store), else the tile staged in destination order with the lanes
// along the dimension that has more of the tile's seven lowest result bits.
SmallkLayout smallk_layout(const EpiParams &e) {
    SmallkLayout L;
    const uint64_t mR = host_pdep64(e.lowRc, e.tileMask), mC = host_pdep64(e.lowCc, e.tileMask);
    auto run = [](uint64_t m) {
        int r = 0;
        while (r < 64 && (m >> r & 1)) ++r;
        return r;
    };
    // two quads along the lanes' dimension when the tile allows (8 of them)
    const int a = e.a_bits, b = e.b_bits;
    auto qm_for = [&](int rm) { return ((!rm && a >= 3) || b < 3) ? 2 : 1; };
    auto lanes = [&](int rm) {  // log2 of the lanes along that dimension
        const int qm = qm_for(rm);
        return rm ? b - 2 - (2 - qm) : a - 2 - (qm - 1);
    };
    // bit of t holding the n-th lowest bit of a compact mask
    auto nth = [](uint32_t m, int n) {
        for (int i = 0; i < n; ++i) m &= m - 1;
        return (uint32_t)__builtin_ctz(m);
    };
    L.rowmajor = pick_staging(e.lowRc, e.lowCc).rowmajor;
    L.direct = 0;
    if (run(mC) >= 4 && lanes(1) >= 1) {
        L.direct = 1;
        L.rowmajor = 1;
    } else if (run(mR) >= 4 && lanes(0) >= 1) {
        L.direct = 1;
        L.rowmajor = 0;
    }
    L.qm = qm_for(L.rowmajor);
    L.pr0 = nth(e.lowRc, 0);
    L.pr1 = nth(e.lowRc, 1);
    L.pc0 = nth(e.lowCc, 0);
    L.pc1 = nth(e.lowCc, 1);
    const bool r0 = e.lowRc & 1u, r1 = e.lowRc & 2u;
    L.pat = (r0 && r1) ? 0 : (!r0 && !r1) ? 1 : (r0 ? 2 : 3);
    return L;
}

cudaError_t launch_smallk(const StepArgs &a, cudaStream_t s) {
    const EpiParams &e = a.epi;
    if (!smallk_ok(a.mb, a.nb, a.kb, a.kblk != 0) || e.a_bits < 2 || e.b_bits < 2 || a.ksplit != 1)
        return cudaErrorInvalidValue;
    if (e.L < 2) return cudaErrorInvalidValue;  // the result's two lowest bits lie in every tile
    const SmallkLayout L = smallk_layout(e);
    const int bytes = std::max(smallk_op_bytes(e.a_bits, e.b_bits, a.kb),
                               L.direct ? 0 : smallk_stage_bytes(e.a_bits, e.b_bits));
    if (bytes > SMALLK_BYTES) return cudaErrorInvalidValue;
    const size_t smem = sizeof(EpiTables) + (size_t)bytes;
    const int64_t col_tiles = 1ll << (a.nb - e.b_bits);
    const int64_t n_tiles = (1ll << (a.mb - e.a_bits)) * col_tiles;
    const unsigned grid = (unsigned)std::min<int64_t>(n_tiles, (int64_t)sm_count() * 16);
    const bool rm = L.rowmajor != 0;
    static bool attr[3][2][2] = {};
#define TQC_SMALLK_LAUNCH(KBV, QMV, RMV)                                                                      \
    if (a.kb == KBV && L.qm == QMV && rm == RMV) {                                                           \
        bool &done = attr[KBV / 2][QMV - 1][RMV ? 1 : 0];                                                    \
        if (!done) {                                                                                         \
            cudaError_t err = cudaFuncSetAttribute(simt_smallk_f32<KBV, QMV, RMV>,                           \
                                                   cudaFuncAttributeMaxDynamicSharedMemorySize,             \
                                                   (int)(sizeof(EpiTables) + SMALLK_BYTES));                 \
            if (err != cudaSuccess) return err;                                                              \
            done = true;                                                                                     \
        }                                                                                                    \
        simt_smallk_f32<KBV, QMV, RMV><<<grid, 128, smem, s>>>(a, n_tiles, col_tiles, L);                    \
        return cudaGetLastError();                                                                           \
    }
    TQC_SMALLK_LAUNCH(0, 1, true)
    TQC_SMALLK_LAUNCH(0, 1, false)
    TQC_SMALLK_LAUNCH(0, 2, true)
    TQC_SMALLK_LAUNCH(0, 2, false)
    TQC_SMALLK_LAUNCH(2, 1, true)
    TQC_SMALLK_LAUNCH(2, 1, false)
    TQC_SMALLK_LAUNCH(2, 2, true)
    TQC_SMALLK_LAUNCH(2, 2, false)
    TQC_SMALLK_LAUNCH(4, 1, true)
    TQC_SMALLK_LAUNCH(4, 1, false)
    TQC_SMALLK_LAUNCH(4, 2, true)
    TQC_SMALLK_LAUNCH(4, 2, false)
#undef TQC_SMALLK_LAUNCH
    return cudaErrorInvalidValue;
}

cudaError_t launch_simt_step(int cfg, const StepArgs &a, cudaStream_t s) {
    switch (cfg) {
        case SIMT_SMALLK: return launch_smallk(a, s);
        case SIMT_128x128: return launch_cfg<128, 128, 8, 8>(a, s);
        case SIMT_128x64: return launch_cfg<128, 64, 8, 4>(a, s);
        default: return launch_cfg<64, 64, 4, 4>(a, s);
    }
}

cudaError_t launch_simt_step_f64(const StepArgs &a, cudaStream_t s) {
    int64_t row_tiles = 1ll << (a.mb - a.epi.a_bits);
    int64_t col_tiles = 1ll << (a.nb - a.epi.b_bits);
    int64_t n_tiles = row_tiles * col_tiles;
    int64_t grid = std::min<int64_t>(n_tiles, (int64_t)sm_count() * 8);
    simt_step_f64<32, 32, 2, 2><<<(unsigned)grid, 256, 0, s>>>(a, n_tiles, col_tiles);
    return cudaGetLastError();
}

cudaError_t launch_ingest(const IngestArgs &g, int64_t n_dst, cudaStream_t s) {
    int64_t threads = g.reduce_bits > 0 ? n_dst * 32 : n_dst;
    int64_t blocks = std::min<int64_t>((threads + 255) / 256, (int64_t)sm_count() * 32);
    if (blocks < 1) blocks = 1;
    // a power of two (the gather's stride; see ingest_kernel)
    while (blocks & (blocks - 1)) blocks &= blocks - 1;
    ingest_kernel<<<(unsigned)blocks, 256, 0, s>>>(g, n_dst);
    return cudaGetLastError();
}

cudaError_t launch_zfinal(const double *zslice, int n, int n_cuts, int renorm, double *zinfo, cudaStream_t s) {
    zfinal_kernel<<<1, 32, 0, s>>>(zslice, n, n_cuts, renorm, zinfo);
    return cudaGetLastError();
}

cudaError_t launch_finalize(const double *acc, void *out, int out_f64, const double *zinfo, int64_t n,
                            cudaStream_t s) {
    int64_t blocks = std::min<int64_t>((n + 255) / 256, (int64_t)sm_count() * 32);
    if (blocks < 1) blocks = 1;
    finalize_kernel<<<(unsigned)blocks, 256, 0, s>>>(acc, out, out_f64, zinfo, n);
    return cudaGetLastError();
}

cudaError_t launch_ksplit_reduce(const float *part, int ksplit, int64_t n, int mode, void *out, const double *zinfo,
                                 cudaStream_t s) {
    if (ksplit < 1 || n < 1) return cudaErrorInvalidValue;
    if (mode != EPI_OUT_F32 && mode != EPI_OUT_F64 && mode != EPI_F64_SET && mode != EPI_F64_ADD)
        return cudaErrorInvalidValue;
    const int64_t blocks = std::min<int64_t>((n + 255) / 256, (int64_t)sm_count() * 32);
    ksplit_reduce_kernel<<<(unsigned)blocks, 256, 0, s>>>(part, ksplit, n, mode, out, zinfo);
    return cudaGetLastError();
}

EpiParams make_epi(uint64_t maskR, uint64_t maskC, int mb, int nb, TileShape t) {
    EpiParams e;
    int a = std::min(t.log_bm, mb), b = std::min(t.log_bn, nb);
    uint64_t lowR = 0, lowC = 0;
    {
        uint64_t m = maskR;
        for (int i = 0; i < a; ++i) {
            uint64_t low = m & (~m + 1);
            lowR |= low;
            m ^= low;
        }
        m = maskC;
        for (int i = 0; i < b; ++i) {
            uint64_t low = m & (~m + 1);
            lowC |= low;
            m ^= low;
        }
    }
    e.highR = maskR & ~lowR;
    e.highC = maskC & ~lowC;
    e.tileMask = lowR | lowC;
    // compact positions of the tile's row / column bits inside tileMask
    uint32_t rc = 0, cc = 0;
    int k = 0;
    for (int bit = 0; bit < 64; ++bit) {
        if (!(e.tileMask >> bit & 1)) continue;
        if (lowR >> bit & 1) rc |= 1u << k;
        else cc |= 1u << k;
        ++k;
    }
    e.lowRc = rc;
    e.lowCc = cc;
    e.a_bits = a;
    e.b_bits = b;
    int L = 0;
    while (L < 64 && (e.tileMask >> L & 1)) ++L;
    e.L = L;
    return e;
}

}  // namespace tqc
