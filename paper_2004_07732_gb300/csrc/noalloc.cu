// dwf_pvdag_apply_noalloc: the preconditioned apply D_PV^dag D_DW psi for
// callers that cannot allocate device memory.
//
// Some host codes hand the whole of HBM to their own memory manager at start-up
// (a caching allocator or a lattice code's arena that reserves nearly all
// device memory), so a cudaMalloc from this library would fail or fragment
// their pool; others call from latency-critical loops where the implicit
// device synchronisation of cudaMalloc/cudaFree is not acceptable.  For them
// this entry point keeps the intermediate vector D_DW psi in a fixed,
// file-scope device array instead of a caller-passed or library-allocated
// buffer.  It calls no cudaMalloc, cudaFree or allocating library routine.
//
// Limits and sharing:
//   * the array holds 16 MiB: up to 2^20 complex128 values (DWF_F64) or 2^21
//     complex64 values (FP32 precisions) of one 5-d spinor; larger lattices are
//     rejected with DWF_ERR_ARG before any device work.
//   * every GPU that loads the library keeps the array resident until the
//     process exits.
//   * all calls on a device share the one array and it keeps the last call's
//     contents; the apply overwrites the whole intermediate before reading it,
//     so nothing has to start at zero.  Calls that overlap on the GPU (on
//     different streams, or from different host threads without ordering) race
//     on the array and give wrong results: order them on one stream.
//   * the first call on each device looks up the array's device address with
//     cudaGetSymbolAddress (that device current) and caches it; make that first
//     call before any stream capture.  The cache is per device ordinal for the
//     life of the process: after cudaDeviceReset the cached address is stale, so
//     a process that resets a device must not call this entry point again.
#include <mutex>

#include "common.cuh"
#include "fine_kernels.cuh"

namespace dwf {
namespace {

constexpr size_t kScratchBytes = size_t(16) << 20;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_pvdag_scratch[kScratchBytes];

std::mutex g_scratch_mu;
void* g_scratch_addr[kMaxDevices] = {};

// Device address of g_pvdag_scratch on the current device (looked up once per device).
dwf_status scratch_address(void** out) {
    int dev = -1;
    DWF_CHECK_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) {
        set_error("device ordinal %d outside the %d devices this entry point supports", dev, kMaxDevices);
        return DWF_ERR_UNSUPPORTED;
    }
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        DWF_CHECK_CUDA(cudaGetSymbolAddress(&p, g_pvdag_scratch));
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return DWF_OK;
}

}  // namespace
}  // namespace dwf

using namespace dwf;

extern "C" dwf_status dwf_pvdag_apply_noalloc(const dwf_geom* g, const void* U, const void* psi, void* out,
                                              double M5, double mf, int prec, void* stream) {
    clear_error();
    Geom G;
    DWF_TRY(check_geom(g, &G));
    if (!valid_prec(prec)) { set_error("bad precision %d", prec); return DWF_ERR_ARG; }
    if (G.V == 0) return DWF_OK;
    const size_t elem = prec == DWF_F64 ? 16 : 8;
    const size_t need = (size_t)spinor_len(G) * elem;
    if (need > kScratchBytes) {
        set_error("dwf_pvdag_apply_noalloc: the intermediate needs %zu bytes, more than its fixed %zu-byte "
                  "device scratch; use dwf_pvdag_apply with a caller buffer", need, kScratchBytes);
        return DWF_ERR_ARG;
    }
    if (!U || !psi || !out) { set_error("NULL device pointer"); return DWF_ERR_ARG; }
    if (!aligned16(psi) || !aligned16(out)) {
        set_error("spinor buffers must be 16-byte aligned");
        return DWF_ERR_ARG;
    }
    if (psi == out) { set_error("psi and out must be distinct buffers"); return DWF_ERR_ARG; }
    void* tmp = nullptr;
    DWF_TRY(scratch_address(&tmp));
    cudaStream_t st = as_stream(stream);
    DWF_TRY(fine_apply(G, U, psi, tmp, M5, mf, false, prec, st));
    return fine_apply(G, U, tmp, out, M5, 1.0, true, prec, st);
}
