// D_DW (Eq. DWoperator) on host-resident spinors: the host-to-device copy, the
// apply and the device-to-host copy are pipelined over chunks of s-slices on
// three streams, so that slices still in flight to the device overlap the
// apply of earlier ones and the copy back of finished ones.  The apply of a
// chunk needs the slices on both sides of it (the P_+- s-hops) and, at the
// walls, slices 0 and Ls - 1, so the last chunk is copied first.
#include <mutex>
#include <vector>

#include "common.cuh"
#include "fine_kernels.cuh"

namespace dwf {
namespace {

constexpr int HP_MAX_CHUNKS = 64;

struct HostPipe {
    bool ready = false;
    cudaStream_t s_in = nullptr, s_comp = nullptr, s_out = nullptr;
    cudaEvent_t start = nullptr, end = nullptr;
    cudaEvent_t in_done[HP_MAX_CHUNKS] = {};
    cudaEvent_t app_done[HP_MAX_CHUNKS] = {};
};

std::mutex g_hp_mutex;
HostPipe g_hp[64];

dwf_status host_pipe(HostPipe** out) {
    int dev = 0;
    DWF_CHECK_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) { set_error("device ordinal out of range"); return DWF_ERR_UNSUPPORTED; }
    HostPipe& hp = g_hp[dev];
    if (!hp.ready) {
        DWF_CHECK_CUDA(cudaStreamCreateWithFlags(&hp.s_in, cudaStreamNonBlocking));
        DWF_CHECK_CUDA(cudaStreamCreateWithFlags(&hp.s_comp, cudaStreamNonBlocking));
        DWF_CHECK_CUDA(cudaStreamCreateWithFlags(&hp.s_out, cudaStreamNonBlocking));
        DWF_CHECK_CUDA(cudaEventCreateWithFlags(&hp.start, cudaEventDisableTiming));
        DWF_CHECK_CUDA(cudaEventCreateWithFlags(&hp.end, cudaEventDisableTiming));
        for (int c = 0; c < HP_MAX_CHUNKS; ++c) {
            DWF_CHECK_CUDA(cudaEventCreateWithFlags(&hp.in_done[c], cudaEventDisableTiming));
            DWF_CHECK_CUDA(cudaEventCreateWithFlags(&hp.app_done[c], cudaEventDisableTiming));
        }
        hp.ready = true;
    }
    *out = &hp;
    return DWF_OK;
}

size_t link_bytes(int prec) {
    return prec == DWF_F64 ? 16 : (prec == DWF_F32 ? 8 : 4);
}

}  // namespace
}  // namespace dwf

using namespace dwf;

extern "C" dwf_status dwf_apply_host(const dwf_geom* g, const void* U_host, const void* psi_host, void* out_host,
                                     void* U_dev, void* psi_dev, void* out_dev, double M5, double mf, int dagger,
                                     int prec, int nchunks, void* stream) {
    clear_error();
    Geom G;
    DWF_TRY(check_geom(g, &G));
    if (G.nd != 2) { set_error("dwf_apply_host: 2-d lattices only"); return DWF_ERR_UNSUPPORTED; }
    if (!valid_prec(prec)) { set_error("bad precision %d", prec); return DWF_ERR_ARG; }
    if (G.V == 0) return DWF_OK;
    if (!U_host || !psi_host || !out_host || !U_dev || !psi_dev || !out_dev) {
        set_error("NULL pointer");
        return DWF_ERR_ARG;
    }
    if (!aligned16(psi_dev) || !aligned16(out_dev)) { set_error("spinor buffers must be 16-byte aligned"); return DWF_ERR_ARG; }
    if (psi_dev == out_dev) { set_error("psi_dev and out_dev must be distinct buffers"); return DWF_ERR_ARG; }
    const int Ls = G.Ls;
    int n = nchunks > 0 ? nchunks : 4;
    if (n > Ls) n = Ls;
    if (n > HP_MAX_CHUNKS) n = HP_MAX_CHUNKS;
    std::lock_guard<std::mutex> lock(g_hp_mutex);
    HostPipe* hp = nullptr;
    DWF_TRY(host_pipe(&hp));
    cudaStream_t user = as_stream(stream);
    const size_t plane = (size_t)G.V * site_dof(G) * (prec == DWF_F64 ? sizeof(double2) : sizeof(float2));
    const size_t ubytes = (size_t)link_len(G) * link_bytes(prec);
    auto lo = [&](int c) { return (int)((long long)c * Ls / n); };
    auto hi = [&](int c) { return (int)((long long)(c + 1) * Ls / n); };
    const char* ph = static_cast<const char*>(psi_host);
    char* oh = static_cast<char*>(out_host);
    char* pd = static_cast<char*>(psi_dev);
    char* od = static_cast<char*>(out_dev);
    // start after the caller's earlier work on `stream`
    DWF_CHECK_CUDA(cudaEventRecord(hp->start, user));
    DWF_CHECK_CUDA(cudaStreamWaitEvent(hp->s_in, hp->start, 0));
    DWF_CHECK_CUDA(cudaStreamWaitEvent(hp->s_comp, hp->start, 0));
    DWF_CHECK_CUDA(cudaStreamWaitEvent(hp->s_out, hp->start, 0));
    DWF_CHECK_CUDA(cudaMemcpyAsync(U_dev, U_host, ubytes, cudaMemcpyHostToDevice, hp->s_in));
    for (int k = 0; k < n; ++k) {                          // chunk order n - 1, 0, 1, ..., n - 2
        const int c = (k + n - 1) % n;
        DWF_CHECK_CUDA(cudaMemcpyAsync(pd + (size_t)lo(c) * plane, ph + (size_t)lo(c) * plane,
                                       (size_t)(hi(c) - lo(c)) * plane, cudaMemcpyHostToDevice, hp->s_in));
        DWF_CHECK_CUDA(cudaEventRecord(hp->in_done[c], hp->s_in));
    }
    for (int c = 0; c < n; ++c) {
        // slices lo(c) - 1 .. hi(c), with the walls: chunks c - 1, c, c + 1 (cyclically)
        DWF_CHECK_CUDA(cudaStreamWaitEvent(hp->s_comp, hp->in_done[(c + n - 1) % n], 0));
        DWF_CHECK_CUDA(cudaStreamWaitEvent(hp->s_comp, hp->in_done[c], 0));
        DWF_CHECK_CUDA(cudaStreamWaitEvent(hp->s_comp, hp->in_done[(c + 1) % n], 0));
        DWF_TRY(fine_apply_2d_range(G, U_dev, psi_dev, out_dev, M5, mf, dagger != 0, prec, lo(c), hi(c), hp->s_comp));
        DWF_CHECK_CUDA(cudaEventRecord(hp->app_done[c], hp->s_comp));
        DWF_CHECK_CUDA(cudaStreamWaitEvent(hp->s_out, hp->app_done[c], 0));
        DWF_CHECK_CUDA(cudaMemcpyAsync(oh + (size_t)lo(c) * plane, od + (size_t)lo(c) * plane,
                                       (size_t)(hi(c) - lo(c)) * plane, cudaMemcpyDeviceToHost, hp->s_out));
    }
    // the caller's stream continues once the last copy back has landed (and the input streams are done)
    DWF_CHECK_CUDA(cudaEventRecord(hp->end, hp->s_out));
    DWF_CHECK_CUDA(cudaStreamWaitEvent(user, hp->end, 0));
    DWF_CHECK_CUDA(cudaEventRecord(hp->end, hp->s_comp));
    DWF_CHECK_CUDA(cudaStreamWaitEvent(user, hp->end, 0));
    return DWF_OK;
}
