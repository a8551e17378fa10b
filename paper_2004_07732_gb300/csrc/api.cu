// C ABI entry points of libdwfmg: argument checks, layout conversions and
// dispatch to the operator kernels.
#include <string.h>

#include "common.cuh"
#include "fine_kernels.cuh"
#include "blas.cuh"

namespace dwf {

static thread_local char g_err[1024] = "";

void set_error(const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}
void clear_error() { g_err[0] = 0; }

bool valid_prec(int prec) { return prec >= DWF_F64 && prec <= DWF_F32_LBF16; }

dwf_status check_geom(const dwf_geom* g, Geom* out) {
    if (!g) { set_error("geometry pointer is NULL"); return DWF_ERR_ARG; }
    if (g->nd != 2 && g->nd != 4) { set_error("nd must be 2 or 4 (got %d)", g->nd); return DWF_ERR_ARG; }
    if (g->nd == 2 && g->group != DWF_U1) { set_error("2-d lattices take group U(1)"); return DWF_ERR_ARG; }
    if (g->nd == 4 && g->group != DWF_SU3) { set_error("4-d lattices take group SU(3)"); return DWF_ERR_ARG; }
    if (g->Ls < 1) { set_error("Ls must be >= 1 (got %d)", g->Ls); return DWF_ERR_ARG; }
    long long V = 1;
    for (int mu = 0; mu < g->nd; ++mu) {
        if (g->L[mu] < 1) { set_error("L[%d] must be >= 1 (got %d)", mu, g->L[mu]); return DWF_ERR_ARG; }
        V *= g->L[mu];
    }
    if (V * (long long)g->Ls > (1LL << 40)) { set_error("lattice too large"); return DWF_ERR_ARG; }
    out->nd = g->nd;
    for (int mu = 0; mu < 4; ++mu) {
        out->L[mu] = mu < g->nd ? g->L[mu] : 1;
        out->anti[mu] = mu < g->nd ? (g->antiperiodic[mu] != 0) : 0;
    }
    out->Ls = g->Ls;
    out->group = g->group;
    out->V = V;
    out->nspin = g->nd == 2 ? 2 : 4;
    out->ncol = g->group == DWF_U1 ? 1 : 3;
    return DWF_OK;
}

// ----------------------------------------------------------------------------
// link conversion FP64 -> storage format
// ----------------------------------------------------------------------------
template <class T> __device__ __forceinline__ T cvt_link(double2 v);
template <> __device__ __forceinline__ double2 cvt_link<double2>(double2 v) { return v; }
template <> __device__ __forceinline__ float2 cvt_link<float2>(double2 v) {
    return make_float2(__double2float_rn(v.x), __double2float_rn(v.y));
}
template <> __device__ __forceinline__ __half2 cvt_link<__half2>(double2 v) {
    return __halves2half2(__double2half(v.x), __double2half(v.y));
}
template <> __device__ __forceinline__ __nv_bfloat162 cvt_link<__nv_bfloat162>(double2 v) {
    return __halves2bfloat162(__double2bfloat16(v.x), __double2bfloat16(v.y));
}

template <class T>
__global__ void k_convert_links(const double2* __restrict__ in, T* __restrict__ out, long long n) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        out[i] = cvt_link<T>(in[i]);
}

}  // namespace dwf

using namespace dwf;

extern "C" {

const char* dwf_last_error(void) { return g_err; }

size_t dwf_spinor_size(const dwf_geom* g) {
    Geom G;
    if (check_geom(g, &G) != DWF_OK) return 0;
    return (size_t)spinor_len(G);
}

size_t dwf_link_size(const dwf_geom* g) {
    Geom G;
    if (check_geom(g, &G) != DWF_OK) return 0;
    return (size_t)link_len(G);
}

dwf_status dwf_convert_links(const dwf_geom* g, const void* U64, void* U_out, int prec, void* stream) {
    clear_error();
    Geom G;
    DWF_TRY(check_geom(g, &G));
    if (!valid_prec(prec)) { set_error("bad precision %d", prec); return DWF_ERR_ARG; }
    long long n = link_len(G);
    if (n == 0) return DWF_OK;
    if (!U64 || !U_out) { set_error("NULL link pointer"); return DWF_ERR_ARG; }
    cudaStream_t st = as_stream(stream);
    int blocks = (int)std::min<long long>((n + 255) / 256, 152LL * 16);
    auto in = reinterpret_cast<const double2*>(U64);
    switch (prec) {
        case DWF_F64: k_convert_links<double2><<<blocks, 256, 0, st>>>(in, (double2*)U_out, n); break;
        case DWF_F32: k_convert_links<float2><<<blocks, 256, 0, st>>>(in, (float2*)U_out, n); break;
        case DWF_F32_L16: k_convert_links<__half2><<<blocks, 256, 0, st>>>(in, (__half2*)U_out, n); break;
        default: k_convert_links<__nv_bfloat162><<<blocks, 256, 0, st>>>(in, (__nv_bfloat162*)U_out, n); break;
    }
    DWF_CHECK_LAUNCH();
    return DWF_OK;
}

static dwf_status apply_checked(const dwf_geom* g, const void* U, const void* psi, void* out, double M5,
                                double mf, int dagger, int prec, void* stream) {
    clear_error();
    Geom G;
    DWF_TRY(check_geom(g, &G));
    if (!valid_prec(prec)) { set_error("bad precision %d", prec); return DWF_ERR_ARG; }
    if (G.V == 0) return DWF_OK;
    if (!U || !psi || !out) { set_error("NULL device pointer"); return DWF_ERR_ARG; }
    if (!aligned16(psi) || !aligned16(out)) { set_error("spinor buffers must be 16-byte aligned"); return DWF_ERR_ARG; }
    if (psi == out) { set_error("psi and out must be distinct buffers"); return DWF_ERR_ARG; }
    return fine_apply(G, U, psi, out, M5, mf, dagger != 0, prec, as_stream(stream));
}

dwf_status dwf_apply(const dwf_geom* g, const void* U, const void* psi, void* out, double M5, double mf,
                     int dagger, int prec, void* stream) {
    return apply_checked(g, U, psi, out, M5, mf, dagger, prec, stream);
}

dwf_status pv_apply(const dwf_geom* g, const void* U, const void* psi, void* out, double M5, int dagger,
                    int prec, void* stream) {
    return apply_checked(g, U, psi, out, M5, 1.0, dagger, prec, stream);
}

dwf_status dwf_pvdag_apply(const dwf_geom* g, const void* U, const void* psi, void* tmp, void* out, double M5,
                           double mf, int prec, void* stream) {
    if (tmp == psi || tmp == out) { set_error("tmp must differ from psi and out"); return DWF_ERR_ARG; }
    DWF_TRY(apply_checked(g, U, psi, tmp, M5, mf, 0, prec, stream));
    return apply_checked(g, U, tmp, out, M5, 1.0, 1, prec, stream);
}

dwf_status dwf_apply_batched(int nrhs, const dwf_geom* geoms, const void* const* U, const void* const* psi,
                             void* const* out, double M5, double mf, int dagger, int prec, void* stream) {
    clear_error();
    if (nrhs < 0 || nrhs > BATCH_MAX) { set_error("nrhs must be in [0, %d]", BATCH_MAX); return DWF_ERR_ARG; }
    if (nrhs == 0) return DWF_OK;
    if (!geoms || !U || !psi || !out) { set_error("NULL argument array"); return DWF_ERR_ARG; }
    if (!valid_prec(prec)) { set_error("bad precision %d", prec); return DWF_ERR_ARG; }
    for (int r = 0; r < nrhs; ++r) {
        Geom G;
        DWF_TRY(check_geom(&geoms[r], &G));
        if (G.nd != 2) { set_error("batched apply: right-hand side %d is not a 2-d lattice", r); return DWF_ERR_UNSUPPORTED; }
        if (!U[r] || !psi[r] || !out[r]) { set_error("batched apply: NULL pointer for right-hand side %d", r); return DWF_ERR_ARG; }
        if (!aligned16(psi[r]) || !aligned16(out[r])) { set_error("spinor buffers must be 16-byte aligned"); return DWF_ERR_ARG; }
        if (psi[r] == out[r]) { set_error("psi and out must be distinct buffers"); return DWF_ERR_ARG; }
    }
    cudaStream_t st = as_stream(stream);
    // launches of at most BATCH_LAUNCH_MAX right-hand sides (one for nrhs <= 128)
    static thread_local BatchArgs2d args;
    for (int r0 = 0; r0 < nrhs; r0 += BATCH_LAUNCH_MAX) {
        const int cnt = nrhs - r0 < BATCH_LAUNCH_MAX ? nrhs - r0 : BATCH_LAUNCH_MAX;
        long long blocks = 0;
        for (int k = 0; k < cnt; ++k) {
            Geom G;
            check_geom(&geoms[r0 + k], &G);
            Fine2dParams& p = args.d[k].p;
            p.V = G.V; p.L0 = G.L[0]; p.L1 = G.L[1]; p.Ls = G.Ls;
            p.anti0 = G.anti[0]; p.anti1 = G.anti[1];
            p.diag = (double)G.nd - M5 + 1.0;
            p.mf = mf;
            p.s_chunk = G.Ls;
            p.s_base = 0;
            p.s_end = G.Ls;
            args.d[k].U = U[r0 + k];
            args.d[k].psi = psi[r0 + k];
            args.d[k].out = out[r0 + k];
            args.d[k].block0 = blocks;
            blocks += (G.V + 255) / 256;
        }
        args.nrhs = cnt;
        args.total_blocks = blocks;
        if (blocks > 0) DWF_TRY(fine_apply_2d_batched(args, dagger != 0, prec, st));
    }
    return DWF_OK;
}

dwf_status dwf_dot(const void* x, const void* y, size_t n, int prec, double* result_host, void* stream) {
    clear_error();
    if (!result_host) { set_error("NULL result pointer"); return DWF_ERR_ARG; }
    if (!valid_prec(prec)) { set_error("bad precision %d", prec); return DWF_ERR_ARG; }
    result_host[0] = result_host[1] = 0.0;
    if (n == 0) return DWF_OK;
    if (!x || !y) { set_error("NULL device pointer"); return DWF_ERR_ARG; }
    cudaStream_t st = as_stream(stream);
    Workspace ws;
    DWF_TRY(ws.reserve(st));
    DWF_TRY(dot_device(x, y, (long long)n, prec == DWF_F64, ws.red(), ws.scal, st, true));
    double h[2];
    DWF_CHECK_CUDA(cudaMemcpyAsync(h, ws.scal, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
    DWF_CHECK_CUDA(cudaStreamSynchronize(st));
    result_host[0] = h[0];
    result_host[1] = h[1];
    return DWF_OK;
}

}  // extern "C"
