// Transfer-operator diagnostics (the paper's discussion section, Sec. 4.1): for a
// fine vector v (typically a low eigenvector of A = D_PV^dag D_DW)
//   local colinearity   (1 - P R) v,
//   oblique projector   (1 - P Ahat^-1 R A) v,   Ahat = Dhat_PV^dag Dhat_DW,
// with the handle's transfer (the walls of Eq. TruncProjectInterpolate, or every
// slice with transfer = 1).  Ahat^-1 is a restarted GCR solve on the coarse level
// to a caller tolerance (mg_coarse_solve), FP32 vectors with FP64 scalars; the
// host drives it one step at a time (a diagnostic, not the solver's hot loop).
#include <string.h>
#include <vector>

#include "mg.cuh"

namespace dwf {
namespace {

constexpr int DG_K = 16;    // GCR restart length of the diagnostic coarse solve

#define DG_LOOP(i, n) for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < (n); i += (long long)gridDim.x * blockDim.x)

struct DgPtrs { const float2* p[DG_K]; };

// out[j] = <X_j, y> (FP64), one block per j
__global__ void __launch_bounds__(RED_THREADS) k_dg_dots(DgPtrs X, const float2* __restrict__ y, long long n,
                                                         double2* __restrict__ out) {
    const float2* x = X.p[blockIdx.x];
    double re = 0.0, im = 0.0;
    for (long long i = threadIdx.x; i < n; i += blockDim.x) {
        const float2 a = x[i], b = y[i];
        re += (double)a.x * b.x + (double)a.y * b.y;
        im += (double)a.x * b.y - (double)a.y * b.x;
    }
    double v[2] = {re, im};
    block_sum<2>(v);
    if (threadIdx.x == 0) out[blockIdx.x] = make_double2(v[0], v[1]);
}

// y -= sum_{j<k} c_j X_j
__global__ void k_dg_sub(DgPtrs X, const double2* __restrict__ c, int k, long long n, float2* __restrict__ y) {
    DG_LOOP(i, n) {
        float2 a = y[i];
        for (int j = 0; j < k; ++j) {
            const float2 x = X.p[j][i];
            const float cr = (float)c[j].x, ci = (float)c[j].y;
            a.x -= cr * x.x - ci * x.y;
            a.y -= cr * x.y + ci * x.x;
        }
        y[i] = a;
    }
}

// y = a x + y (a complex, host value)
__global__ void k_dg_axpy(float2* __restrict__ y, const float2* __restrict__ x, float ar, float ai, long long n) {
    DG_LOOP(i, n) {
        const float2 u = x[i];
        float2 v = y[i];
        v.x += ar * u.x - ai * u.y;
        v.y += ar * u.y + ai * u.x;
        y[i] = v;
    }
}

__global__ void k_dg_scale(float2* __restrict__ y, float s, long long n) {
    DG_LOOP(i, n) { float2 v = y[i]; v.x *= s; v.y *= s; y[i] = v; }
}

__global__ void k_dg_sub2(float2* __restrict__ out, const float2* __restrict__ a, const float2* __restrict__ b,
                          long long n) {
    DG_LOOP(i, n) { const float2 u = a[i], v = b[i]; out[i] = make_float2(u.x - v.x, u.y - v.y); }
}

inline int dg_grid(long long n) {
    long long b = (n + 255) / 256;
    return (int)(b < 1216 ? (b < 1 ? 1 : b) : 1216);
}

struct DgBuf {
    std::vector<void*> p;
    cudaStream_t st;
    ~DgBuf() { for (void* q : p) cudaFreeAsync(q, st); }
    dwf_status take(void** out, size_t bytes) {
        cudaError_t e = cudaMallocAsync(out, bytes, st);
        if (e != cudaSuccess) { set_error("diagnostic work vectors: %s", cudaGetErrorString(e)); return DWF_ERR_OOM; }
        p.push_back(*out);
        return DWF_OK;
    }
};

// <x, y> of two device vectors, read back (one block)
dwf_status dg_dot(const float2* x, const float2* y, long long n, double2* dscr, double2* out, cudaStream_t st) {
    DgPtrs X;
    X.p[0] = x;
    k_dg_dots<<<1, RED_THREADS, 0, st>>>(X, y, n, dscr);
    DWF_CHECK_LAUNCH();
    DWF_CHECK_CUDA(cudaMemcpyAsync(out, dscr, sizeof(double2), cudaMemcpyDeviceToHost, st));
    DWF_CHECK_CUDA(cudaStreamSynchronize(st));
    return DWF_OK;
}

// restarted GCR(DG_K) on Ahat e = r (coarse, FP32), e = 0 start, to |r - Ahat e| <= tol |r|
dwf_status coarse_gcr_solve(dwf_mg* h, const float2* rc, float2* ec, double tol, int maxiter, int* iters,
                            cudaStream_t st) {
    const long long n = coarse_len(h);
    const size_t vb = (size_t)n * sizeof(float2);
    DgBuf B{{}, st};
    float2 *r, *t;
    float2* Z[DG_K];
    float2* W[DG_K];
    double2* d;
    DWF_TRY(B.take((void**)&r, vb));
    DWF_TRY(B.take((void**)&t, vb));
    for (int k = 0; k < DG_K; ++k) { DWF_TRY(B.take((void**)&Z[k], vb)); DWF_TRY(B.take((void**)&W[k], vb)); }
    DWF_TRY(B.take((void**)&d, sizeof(double2) * (DG_K + 1)));
    const int g = dg_grid(n);
    DWF_CHECK_CUDA(cudaMemcpyAsync(r, rc, vb, cudaMemcpyDeviceToDevice, st));
    DWF_CHECK_CUDA(cudaMemsetAsync(ec, 0, vb, st));
    double2 hb;
    DWF_TRY(dg_dot(r, r, n, d, &hb, st));
    const double ref2 = tol * tol * hb.x;
    double rr2 = hb.x;
    int it = 0;
    std::vector<double2> hc(DG_K);
    while (rr2 > ref2 && it < maxiter) {
        for (int k = 0; k < DG_K && rr2 > ref2 && it < maxiter; ++k, ++it) {
            // z = r, w = Ahat z, orthogonalised (classical Gram-Schmidt, twice) against W_0..W_{k-1}
            DWF_CHECK_CUDA(cudaMemcpyAsync(Z[k], r, vb, cudaMemcpyDeviceToDevice, st));
            DWF_TRY(coarse_dwf_apply(h, Z[k], t, h->mf, false, nullptr, st));
            DWF_TRY(coarse_dwf_apply(h, t, W[k], 1.0, true, nullptr, st));
            DgPtrs Wp, Zp;
            for (int j = 0; j < DG_K; ++j) { Wp.p[j] = W[j]; Zp.p[j] = Z[j]; }
            for (int pass = 0; pass < 2 && k > 0; ++pass) {
                k_dg_dots<<<k, RED_THREADS, 0, st>>>(Wp, W[k], n, d);
                k_dg_sub<<<g, 256, 0, st>>>(Wp, d, k, n, W[k]);
                k_dg_sub<<<g, 256, 0, st>>>(Zp, d, k, n, Z[k]);
                DWF_CHECK_LAUNCH();
            }
            double2 ww, wr;
            DWF_TRY(dg_dot(W[k], W[k], n, d, &ww, st));
            if (!(ww.x > 0.0)) { rr2 = 0.0; break; }
            const float inv = (float)(1.0 / sqrt(ww.x));
            k_dg_scale<<<g, 256, 0, st>>>(W[k], inv, n);
            k_dg_scale<<<g, 256, 0, st>>>(Z[k], inv, n);
            DWF_CHECK_LAUNCH();
            DWF_TRY(dg_dot(W[k], r, n, d, &wr, st));
            k_dg_axpy<<<g, 256, 0, st>>>(ec, Z[k], (float)wr.x, (float)wr.y, n);
            k_dg_axpy<<<g, 256, 0, st>>>(r, W[k], (float)-wr.x, (float)-wr.y, n);
            DWF_CHECK_LAUNCH();
            DWF_TRY(dg_dot(r, r, n, d, &hb, st));
            rr2 = hb.x;
        }
    }
    if (iters) *iters = it;
    return DWF_OK;
}

}  // namespace
}  // namespace dwf

using namespace dwf;

extern "C" {

dwf_status mg_coarse_solve(dwf_mg* h, const void* rc, void* ec, double tol, int maxiter, int* iters, void* stream) {
    clear_error();
    if (!h || !rc || !ec) { set_error("NULL argument"); return DWF_ERR_ARG; }
    if (rc == ec) { set_error("rc and ec must be distinct buffers"); return DWF_ERR_ARG; }
    if (!(tol > 0.0) || maxiter < 0) { set_error("bad tolerance or iteration cap"); return DWF_ERR_ARG; }
    return coarse_gcr_solve(h, (const float2*)rc, (float2*)ec, tol, maxiter, iters, as_stream(stream));
}

dwf_status mg_transfer_colinearity(dwf_mg* h, const void* v, void* out, void* stream) {
    clear_error();
    if (!h || !v || !out) { set_error("NULL argument"); return DWF_ERR_ARG; }
    if (v == out) { set_error("v and out must be distinct buffers"); return DWF_ERR_ARG; }
    cudaStream_t st = as_stream(stream);
    const long long nf = fine_len(h), nc = coarse_len(h);
    DgBuf B{{}, st};
    float2* c;
    DWF_TRY(B.take((void**)&c, (size_t)nc * sizeof(float2)));
    DWF_TRY(restrict_wall(h, (const float2*)v, c, nullptr, st));
    DWF_TRY(prolong_wall(h, c, (float2*)out, nullptr, st));
    k_dg_sub2<<<dg_grid(nf), 256, 0, st>>>((float2*)out, (const float2*)v, (const float2*)out, nf);
    DWF_CHECK_LAUNCH();
    return DWF_OK;
}

dwf_status mg_transfer_oblique(dwf_mg* h, const void* v, void* out, double tol, int* iters, void* stream) {
    clear_error();
    if (!h || !v || !out) { set_error("NULL argument"); return DWF_ERR_ARG; }
    if (v == out) { set_error("v and out must be distinct buffers"); return DWF_ERR_ARG; }
    if (!(tol > 0.0)) { set_error("tol must be > 0"); return DWF_ERR_ARG; }
    cudaStream_t st = as_stream(stream);
    const long long nf = fine_len(h), nc = coarse_len(h);
    DgBuf B{{}, st};
    float2 *t, *a, *rc, *ec;
    DWF_TRY(B.take((void**)&t, (size_t)nf * sizeof(float2)));
    DWF_TRY(B.take((void**)&a, (size_t)nf * sizeof(float2)));
    DWF_TRY(B.take((void**)&rc, (size_t)nc * sizeof(float2)));
    DWF_TRY(B.take((void**)&ec, (size_t)nc * sizeof(float2)));
    // a = A v = D_PV^dag D_DW v (FP32 spinors, the handle's fine link storage)
    DWF_TRY(fine_apply(h->G, h->Ulo, v, t, h->M5, h->mf, false, h->prm.fine_prec, st));
    DWF_TRY(fine_apply(h->G, h->Ulo, t, a, h->M5, 1.0, true, h->prm.fine_prec, st));
    DWF_TRY(restrict_wall(h, a, rc, nullptr, st));
    DWF_TRY(coarse_gcr_solve(h, rc, ec, tol, 1 << 20, iters, st));
    DWF_TRY(prolong_wall(h, ec, (float2*)out, nullptr, st));
    k_dg_sub2<<<dg_grid(nf), 256, 0, st>>>((float2*)out, (const float2*)v, (const float2*)out, nf);
    DWF_CHECK_LAUNCH();
    return DWF_OK;
}

}  // extern "C"
