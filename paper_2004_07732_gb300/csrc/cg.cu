// FP64 conjugate gradient on the normal equations (CGNR), Sec. 2.1 and the
// baseline of Fig. iterationscompare: D^dag D x = D^dag b, stopped on the true
// residual ||b - D x|| / ||b|| of the original system.
//
// Per iteration: q = D p; alpha = |r|^2 / |q|^2 (device scalar); w = D^dag q;
// x += alpha p, rr -= alpha q, r -= alpha w with |rr|^2, |r|^2 reduced in the
// same pass; p = r + beta p.  The scalars never leave the device; the host
// reads |rr|^2 every `check` iterations to test convergence.
#include <chrono>

#include "common.cuh"
#include "fine_kernels.cuh"
#include "blas.cuh"

namespace dwf {

struct CgScalars {
    double rn2;     // |r|^2, r = D^dag rr
    double alpha;
    double beta;
    double rr2;     // |rr|^2, rr = b - D x (recursive)
    double bn2;
    double breakdown;
};

__global__ void __launch_bounds__(RED_THREADS) k_cg_norm_init(const double2* __restrict__ r, const double2* __restrict__ b,
                                                              long long n, RedScratch rs, CgScalars* sc) {
    double v[2] = {0.0, 0.0};
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        double2 a = r[i], c = b[i];
        v[0] += a.x * a.x + a.y * a.y;
        v[1] += c.x * c.x + c.y * c.y;
    }
    grid_reduce<2>(v, rs, [=] __device__(double* t) {
        sc->rn2 = t[0]; sc->bn2 = t[1]; sc->rr2 = t[1]; sc->breakdown = 0.0;
    });
}

__global__ void __launch_bounds__(RED_THREADS) k_cg_alpha(const double2* __restrict__ q, long long n, RedScratch rs,
                                                          CgScalars* sc) {
    double v[1] = {0.0};
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        double2 a = q[i];
        v[0] += a.x * a.x + a.y * a.y;
    }
    grid_reduce<1>(v, rs, [=] __device__(double* t) {
        if (t[0] > 0.0) sc->alpha = sc->rn2 / t[0];
        else { sc->alpha = 0.0; sc->breakdown = 1.0; }
    });
}

__global__ void __launch_bounds__(RED_THREADS) k_cg_update(double2* __restrict__ x, double2* __restrict__ rr,
                                                           double2* __restrict__ r, const double2* __restrict__ p,
                                                           const double2* __restrict__ q, const double2* __restrict__ w,
                                                           long long n, RedScratch rs, CgScalars* sc) {
    const double a = sc->alpha;
    double v[2] = {0.0, 0.0};
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        double2 pi = p[i], qi = q[i], wi = w[i];
        double2 xi = x[i], rri = rr[i], ri = r[i];
        xi.x += a * pi.x; xi.y += a * pi.y;
        rri.x -= a * qi.x; rri.y -= a * qi.y;
        ri.x -= a * wi.x; ri.y -= a * wi.y;
        x[i] = xi; rr[i] = rri; r[i] = ri;
        v[0] += rri.x * rri.x + rri.y * rri.y;
        v[1] += ri.x * ri.x + ri.y * ri.y;
    }
    grid_reduce<2>(v, rs, [=] __device__(double* t) {
        sc->rr2 = t[0];
        sc->beta = sc->rn2 > 0.0 ? t[1] / sc->rn2 : 0.0;
        sc->rn2 = t[1];
    });
}

__global__ void k_cg_p(double2* __restrict__ p, const double2* __restrict__ r, long long n, const CgScalars* sc) {
    const double b = sc->beta;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        double2 pi = p[i], ri = r[i];
        p[i] = make_double2(ri.x + b * pi.x, ri.y + b * pi.y);
    }
}

// rr = b - t (the true residual from t = D x)
__global__ void k_sub(double2* __restrict__ rr, const double2* __restrict__ b, const double2* __restrict__ t, long long n) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        double2 bi = b[i], ti = t[i];
        rr[i] = make_double2(bi.x - ti.x, bi.y - ti.y);
    }
}

static int ew_grid(long long n) {
    long long b = (n + 255) / 256;
    return (int)(b < 152LL * 8 ? b : 152LL * 8);
}

}  // namespace dwf

using namespace dwf;

extern "C" dwf_status cgne_solve(const dwf_geom* g, const void* U, const void* b, void* x, double M5, double mf,
                                 double tol, int maxiter, dwf_solve_stats* stats, void* stream) {
    clear_error();
    auto t0 = std::chrono::steady_clock::now();
    Geom G;
    DWF_TRY(check_geom(g, &G));
    if (stats) memset(stats, 0, sizeof(*stats));
    const long long n = spinor_len(G);
    if (n == 0) return DWF_OK;
    if (!U || !b || !x) { set_error("NULL device pointer"); return DWF_ERR_ARG; }
    if (!(tol > 0.0)) { set_error("tol must be > 0"); return DWF_ERR_ARG; }
    if (maxiter < 0) { set_error("maxiter must be >= 0"); return DWF_ERR_ARG; }
    cudaStream_t st = as_stream(stream);
    const size_t vb = (size_t)n * sizeof(double2);

    Workspace ws;
    DWF_TRY(ws.reserve(st));
    void* buf = nullptr;
    {
        cudaError_t e = cudaMallocAsync(&buf, 5 * vb, st);
        if (e != cudaSuccess) { set_error("CGNR work vectors (%zu bytes): %s", 5 * vb, cudaGetErrorString(e)); return DWF_ERR_OOM; }
    }
    struct Free { void* p; cudaStream_t s; ~Free() { cudaFreeAsync(p, s); } } fr{buf, st};
    double2* rr = (double2*)buf;
    double2* r = rr + n;
    double2* p = r + n;
    double2* q = p + n;
    double2* w = q + n;
    double2* X = (double2*)x;
    const double2* B = (const double2*)b;
    CgScalars* sc = (CgScalars*)ws.scal;
    CgScalars* hsc = nullptr;
    DWF_CHECK_CUDA(cudaMallocHost(&hsc, sizeof(CgScalars)));
    struct FreeH { void* p; ~FreeH() { cudaFreeHost(p); } } frh{hsc};

    const int eg = ew_grid(n), rg = red_grid(n);
    long long applies = 0;
    int restarts = 0;

    // x = 0, rr = b, r = D^dag b, p = r
    DWF_CHECK_CUDA(cudaMemsetAsync(X, 0, vb, st));
    DWF_CHECK_CUDA(cudaMemcpyAsync(rr, B, vb, cudaMemcpyDeviceToDevice, st));
    auto restart_from_rr = [&]() -> dwf_status {
        DWF_TRY(fine_apply(G, U, rr, r, M5, mf, true, DWF_F64, st));
        ++applies;
        DWF_CHECK_CUDA(cudaMemcpyAsync(p, r, vb, cudaMemcpyDeviceToDevice, st));
        k_cg_norm_init<<<rg, RED_THREADS, 0, st>>>(r, B, n, ws.red(), sc);
        DWF_CHECK_LAUNCH();
        return DWF_OK;
    };
    DWF_TRY(restart_from_rr());
    DWF_CHECK_CUDA(cudaMemcpyAsync(hsc, sc, sizeof(CgScalars), cudaMemcpyDeviceToHost, st));
    DWF_CHECK_CUDA(cudaStreamSynchronize(st));
    const double bn2 = hsc->bn2;
    dwf_status status = DWF_ERR_NOCONV;
    double true_res = 1.0;
    if (bn2 == 0.0) {
        status = DWF_OK;
        true_res = 0.0;
    }
    const int check = 16;
    int it = 0;
    while (status != DWF_OK && it < maxiter) {
        int todo = check < maxiter - it ? check : maxiter - it;
        for (int k = 0; k < todo; ++k) {
            DWF_TRY(fine_apply(G, U, p, q, M5, mf, false, DWF_F64, st));
            k_cg_alpha<<<rg, RED_THREADS, 0, st>>>(q, n, ws.red(), sc);
            DWF_TRY(fine_apply(G, U, q, w, M5, mf, true, DWF_F64, st));
            k_cg_update<<<rg, RED_THREADS, 0, st>>>(X, rr, r, p, q, w, n, ws.red(), sc);
            k_cg_p<<<eg, 256, 0, st>>>(p, r, n, sc);
            DWF_CHECK_LAUNCH();
            applies += 2;
        }
        it += todo;
        DWF_CHECK_CUDA(cudaMemcpyAsync(hsc, sc, sizeof(CgScalars), cudaMemcpyDeviceToHost, st));
        DWF_CHECK_CUDA(cudaStreamSynchronize(st));
        if (hsc->breakdown != 0.0) { set_error("CGNR breakdown (|D p| = 0)"); break; }
        if (hsc->rr2 <= tol * tol * bn2) {
            // confirm on the true residual b - D x; restart from it if the
            // recursion has drifted
            DWF_TRY(fine_apply(G, U, X, q, M5, mf, false, DWF_F64, st));
            ++applies;
            k_sub<<<eg, 256, 0, st>>>(rr, B, q, n);
            DWF_CHECK_LAUNCH();
            DWF_TRY(dot_device(rr, rr, n, true, ws.red(), ws.scal + 32, st));
            double tr[2];
            DWF_CHECK_CUDA(cudaMemcpyAsync(tr, ws.scal + 32, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
            DWF_CHECK_CUDA(cudaStreamSynchronize(st));
            true_res = sqrt(tr[0] / bn2);
            if (true_res <= tol) { status = DWF_OK; break; }
            ++restarts;
            DWF_TRY(restart_from_rr());
        }
    }
    if (status != DWF_OK) {
        // final true residual for the report
        DWF_TRY(fine_apply(G, U, X, q, M5, mf, false, DWF_F64, st));
        ++applies;
        k_sub<<<eg, 256, 0, st>>>(rr, B, q, n);
        DWF_TRY(dot_device(rr, rr, n, true, ws.red(), ws.scal + 32, st));
        double tr[2];
        DWF_CHECK_CUDA(cudaMemcpyAsync(tr, ws.scal + 32, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
        DWF_CHECK_CUDA(cudaStreamSynchronize(st));
        true_res = bn2 > 0 ? sqrt(tr[0] / bn2) : 0.0;
        if (status == DWF_ERR_NOCONV && dwf_last_error()[0] == 0)
            set_error("CGNR reached maxiter=%d with true residual %.3e > tol %.3e", maxiter, true_res, tol);
    }
    if (stats) {
        stats->iterations = it;
        stats->restarts = restarts;
        stats->fine_applies = applies;
        stats->true_residual = true_res;
        stats->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
    return status;
}
