// Host-side launchers of the device kernels (one per kernel family).
#pragma once

#include <cuda_runtime.h>

#include "tqc_internal.h"

namespace tqc {

// CUDA-core step tiles (FP32), chosen by the autotuner; SIMT_SMALLK: the
// write-out-shaped tile of steps with K = 1, 4 or 16 (smallk.cuh)
enum SimtCfg { SIMT_64x64 = 0, SIMT_128x128 = 1, SIMT_128x64 = 2, SIMT_SMALLK = 3, SIMT_N_CFG = 4 };

struct TileShape {
    int log_bm, log_bn;
};

TileShape simt_tile(int cfg);
// Whether a CUDA-core step can take SIMT_SMALLK (K of 1, 4 or 16 over plain
// row-major FP32 operands, at least 4 rows, 4 columns and 128 results), and
// its tile shape.
bool smallk_ok(int mb, int nb, int kb, bool kblk);
TileShape smallk_tile(int mb, int nb, int kb);
TileShape simt_f64_tile();
int sm_count();

cudaError_t launch_simt_step(int cfg, const StepArgs &a, cudaStream_t s);
cudaError_t launch_simt_step_f64(const StepArgs &a, cudaStream_t s);
cudaError_t launch_ingest(const IngestArgs &g, int64_t n_dst, cudaStream_t s);
cudaError_t launch_zfinal(const double *zslice, int n, int n_cuts, int renorm, double *zinfo, cudaStream_t s);
cudaError_t launch_finalize(const double *acc, void *out, int out_f64, const double *zinfo, int64_t n,
                            cudaStream_t s);
// Sum of a K-split step's FP32 partials (split s at part + s * n) into its
// output mode (EPI_OUT_F32 / EPI_OUT_F64 / EPI_F64_SET / EPI_F64_ADD).
cudaError_t launch_ksplit_reduce(const float *part, int ksplit, int64_t n, int mode, void *out, const double *zinfo,
                                 cudaStream_t s);

// tcgen05 step (umma.cu)
// *_DEEP: direct epilogue and a deeper operand ring, for steps with a long K loop
enum UmmaCfg { UMMA_128x128 = 0, UMMA_128x64 = 1, UMMA_128x128_DEEP = 2, UMMA_128x256_DEEP = 3, UMMA_N_CFG = 4 };
TileShape umma_tile(int cfg);
// prec: TQC_PREC_BF16 / TQC_PREC_BF16X3 / TQC_PREC_TF32
cudaError_t launch_umma_step(int cfg, int prec, const StepArgs &a, int *d_err, cudaStream_t s);
cudaError_t umma_make_maps(int prec, const StepArgs &a, int bn, void *maps_out);  // 4 CUtensorMap

// Fused pair of tensor-core steps (fused.cu): whether steps s and s + 1 of a
// plan qualify, the launch (a0: step s's operands; a1: step s + 1's operands
// and epilogue), and the test hook shared with tqc_step_inject_stall.
bool fused_pair_ok(const Plan &p, size_t s);
cudaError_t launch_fused_pair(const StepArgs &a0, const StepArgs &a1, uint64_t maskR0, uint64_t maskC0, int *d_err,
                              cudaStream_t s);
void fused_set_stall(int enable);

// Argument blocks the executor builds (executor.cu), reused by the batched launch.
IngestArgs exec_leaf_args(const Plan &p, const TensorPlan &t, int j, const uint8_t *fixed);
StepArgs exec_step_args(const Plan &p, const StepPlan &st, TileShape tile);
int exec_epi_mode(int storage);

// Tile configuration of a step when it is not autotuned (out_esize: bytes
// per result element its epilogue writes).
constexpr int DEEP_MIN_LOG2_K = 12;
// Direct-form steps from this K on (rows up to 64 KB) use 64-byte k-blocks:
// measured 6% faster at K = 2^14, slower at K = 2^10 (short loops) and at
// K = 2^18 (rows of 512 KB: twice the boxes per byte, each across pages).
constexpr int SW64_MIN_LOG2_K = 12;
int default_step_tile(const StepPlan &st, int out_esize, bool smallk = true);
// K splits of a final tensor-core step with too few tiles to fill the GPU
// evenly (1 = no split); max_part_bytes caps the FP32 partials it stores.
int step_ksplit(const StepPlan &st, int64_t out_elems, int64_t max_part_bytes);
int step_out_esize(const Plan &p, const StepPlan &st);
double direct_store_efficiency(const EpiParams &e, int esize);

// Epilogue parameters for a step given its result masks and tile shape.
EpiParams make_epi(uint64_t maskR, uint64_t maskC, int mb, int nb, TileShape t);

}  // namespace tqc
