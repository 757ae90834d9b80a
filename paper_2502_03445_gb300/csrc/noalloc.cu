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
//     before any stream capture.
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
    // The error word in the zinfo block must start at zero on every call;
    // everything else is written before it is read (operands by ingest,
    // intermediates by their step, the FP64 slice sum by the first slice, the
    // per-slice masses by the total-mass network).
    e = cudaMemsetAsync(base, 0, (size_t)zinfo_bytes, s);
    if (e != cudaSuccess) return fail(TQC_ERR_CUDA, std::string("scratch clear: ") + cudaGetErrorString(e));

    // Point the plan's device state and the network's tensors at the scratch
    // and the caller's tensors for the duration of this call (no heap use:
    // at most 63 subcircuits and 62 steps).
    Net &net = *p.net;
    void *saved_data[64];
    int saved_dtype[64];
    int sv_tiles[64], sv_ksplit[64];
    for (int j = 0; j < p.m; ++j) {
        saved_data[j] = net.nodes[j].d_data;
        saved_dtype[j] = net.nodes[j].dtype;
        net.nodes[j].d_data = const_cast<void *>(d_tensors[j]);
        net.nodes[j].dtype = in_dtype;
    }
    void *sv_ws = p.d_ws, *sv_zws = p.d_zws;
    double *sv_zinfo = p.d_zinfo;
    const bool sv_ready = p.ready;
    const uint64_t sv_zver = p.z_version;
    p.z_version = 0;  // the caller's tensors: always compute the total mass
    const int sv_profile = p.profile;
    const int sv_autotune = p.autotune;  // no tile timing here: it would allocate (events, K-split partials)
    const int sv_device = net.device;
    for (size_t i = 0; i < p.steps.size(); ++i) {
        sv_tiles[i] = p.steps[i].tile;
        sv_ksplit[i] = p.steps[i].ksplit;
    }
    p.d_zinfo = (double *)base;
    p.d_zws = (char *)base + zws_off;  // the per-slice masses follow the Z network buffers
    p.d_ws = (char *)base + ws_off;
    p.ready = true;
    p.profile = 0;
    p.autotune = 0;
    net.device = dev;
    for (auto &st : p.steps) {  // the tile rule of the allocating path, unsplit (no partials buffer)
        st.tile = default_step_tile(st, step_out_esize(p, st));
        st.ksplit = 1;
    }
    tqc_status st = exec_contract(&p, fixed_bits, d_out, out_dtype, nullptr, cuda_stream);
    // restore
    for (int j = 0; j < p.m; ++j) {
        net.nodes[j].d_data = saved_data[j];
        net.nodes[j].dtype = saved_dtype[j];
    }
    p.d_ws = sv_ws;
    p.d_zws = sv_zws;
    p.d_zinfo = sv_zinfo;
    p.ready = sv_ready;
    p.z_version = sv_zver;
    p.profile = sv_profile;
    p.autotune = sv_autotune;
    net.device = sv_device;
    for (size_t i = 0; i < p.steps.size(); ++i) {
        p.steps[i].tile = sv_tiles[i];
        p.steps[i].ksplit = sv_ksplit[i];
    }
    return st;
}
