// Allocation-free reconstruction entry point (tqc_contract_noalloc).
//
// Some callers cannot allocate device memory at the moment they need a
// reconstruction: a serving process whose device memory is entirely owned by
// its framework's caching allocator or an MPS client with a hard memory cap,
// a latency-critical loop where the implicit device synchronisation of
// cudaMalloc/cudaFree would stall other streams, or code that must not touch
// the allocator at all for policy reasons.  For them this entry point runs
// the same launch sequence as tqc_contract, reading the caller's device
// tensors and writing the caller's output buffer, with every intermediate
// (bin-restricted operands, pairwise-step results, the total-mass network,
// the FP64 slice sum) carved from one file-scope device array instead of a
// workspace allocated per plan.
//
// Cost and limits:
//   * the array is TQC_NOALLOC_SCRATCH_BYTES (16 MiB); every GPU on which the
//     library's device code is loaded holds it until the process exits;
//   * a plan whose scratch needs exceed it is rejected with
//     TQC_ERR_UNSUPPORTED before any device work;
//   * all calls share the one array and it keeps the last call's contents:
//     calls that overlap on the GPU (different streams, or different host
//     threads) race on it and give wrong results;
//   * the first call on a device looks up the array's device address with
//     cudaGetSymbolAddress (which may load the module); make that first call
//     before any stream capture;
//   * each call ends by reading its error word back to the host (a 4-byte
//     copy into a stack variable), so it synchronises the caller's stream and
//     reports a bounded device wait that gave up as TQC_ERR_TIMEOUT.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "launch.h"
#include "tqc_internal.h"

#ifndef TQC_NOALLOC_SCRATCH_BYTES
#define TQC_NOALLOC_SCRATCH_BYTES (16u << 20)
#endif

namespace {

// The scratch array.  Host code must not use its name as a device address;
// it passes the address obtained from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_noalloc_scratch[TQC_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_scratch_addr[kMaxDevices] = {nullptr};

int64_t align256(int64_t x) { return (x + 255) & ~int64_t(255); }

}  // namespace

struct tqc_plan {
    tqc::Plan p;
};

using namespace tqc;

extern "C" int64_t tqc_noalloc_scratch_bytes(void) { return (int64_t)TQC_NOALLOC_SCRATCH_BYTES; }

extern "C" tqc_status tqc_contract_noalloc(tqc_plan_t plan, const void *const *d_tensors, int32_t in_dtype,
                                           const uint8_t *fixed_bits, void *d_out, int32_t out_dtype,
                                           void *cuda_stream) {
    if (!plan || !d_tensors || !d_out) return fail(TQC_ERR_INVALID, "NULL argument");
    if (out_dtype != TQC_F32 && out_dtype != TQC_F64) return fail(TQC_ERR_INVALID, "out_dtype must be TQC_F32 or TQC_F64");
    if (in_dtype != TQC_F32 && in_dtype != TQC_F64) return fail(TQC_ERR_INVALID, "in_dtype must be TQC_F32 or TQC_F64");
    Plan &p = plan->p;
    for (int j = 0; j < p.m; ++j)
        if (!d_tensors[j]) return fail(TQC_ERR_INVALID, "d_tensors[" + std::to_string(j) + "] is NULL");

    // scratch layout: [zinfo + error word | Z network, then its per-slice sums | main workspace]
    const int64_t zinfo_bytes = 256;
    const int64_t zws_off = zinfo_bytes;
    const int64_t ws_off = zws_off + align256(p.zws_bytes + 8 * p.n_slices());
    const int64_t need = ws_off + align256(p.ws_bytes);
    if (need > (int64_t)TQC_NOALLOC_SCRATCH_BYTES)
        return fail(TQC_ERR_UNSUPPORTED, "plan needs " + std::to_string(need) + " bytes of scratch; the allocation-free "
                                         "entry point has " + std::to_string((int64_t)TQC_NOALLOC_SCRATCH_BYTES));

    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(TQC_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return fail(TQC_ERR_UNSUPPORTED, "device ordinal beyond 63");
    void *base = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        if (!g_scratch_addr[dev]) {
            void *ptr = nullptr;
            e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
            if (e != cudaSuccess)
                return fail(TQC_ERR_CUDA, std::string("cudaGetSymbolAddress(scratch): ") + cudaGetErrorString(e));
            g_scratch_addr[dev] = ptr;
        }
        base = g_scratch_addr[dev];
    }
    cudaStream_t s = (cudaStream_t)cuda_stream;
    // The zinfo block (Z, scale, error word) must start at zero on every
    // call; everything else is written before it is read (operands by
    // ingest, intermediates by their step, the FP64 slice sum by the first
    // slice, the per-slice masses by the total-mass network).
    e = cudaMemsetAsync(base, 0, (size_t)zinfo_bytes, s);
    if (e != cudaSuccess) return fail(TQC_ERR_CUDA, std::string("scratch clear: ") + cudaGetErrorString(e));

    // Every buffer of this call is in the scratch array or the caller's: the
    // plan's and the network's own device state is neither read nor changed,
    // so other calls on the same plan or network are unaffected.  Tiles are
    // the default ones, unsplit (the autotuner and the K-split partials would
    // allocate).
    ExecCtx c;
    c.zinfo = (double *)base;
    c.zws = (char *)base + zws_off;  // the per-slice masses follow the Z network buffers
    c.ws = (char *)base + ws_off;
    c.node_data = d_tensors;
    c.node_dtype = in_dtype;
    c.default_tiles = true;
    c.compute_z = true;              // the caller's tensors: always compute the total mass
    tqc_status st = exec_run(p, c, fixed_bits, d_out, out_dtype, cuda_stream, nullptr);
    if (st != TQC_OK) return st;
    // The error word of this call's tensor-core steps: read back into a host
    // stack variable (no allocation) after the stream has drained.
    int werr = 0;
    e = cudaMemcpyAsync(&werr, c.zinfo + 2, sizeof werr, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fail(TQC_ERR_CUDA, std::string("noalloc status: ") + cudaGetErrorString(e));
    if (werr != 0) return fail(TQC_ERR_TIMEOUT, "a tensor-core step gave up waiting on its pipeline");
    return TQC_OK;
}
