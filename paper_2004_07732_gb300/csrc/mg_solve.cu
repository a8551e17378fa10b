// The K-cycle solve of Sec. 2.3 ("Summary") with the Table kcycle parameters.
//
// Outer loop, FP64 (reliable updates): r = b - D_DW x with the FP64 operator;
// stop when ||r|| / ||b|| <= tol; otherwise solve the left-preconditioned
// correction system  D_PV^dag D_DW e = D_PV^dag r  approximately in FP32
// (spinors FP32, links in the handle's fine storage) and add e to x in FP64.
//
// Inner solver: flexible GCR, restart gcr_restart, on A = D_PV^dag D_DW with
// the preconditioner M(r):
//   1. restrict the wall of r onto the coarse walls (Eq. TruncProjectInterpolate);
//   2. solve Dhat_PV^dag Dhat_DW e_c = r_c with CGNR on the coarse normal
//      operator to coarse_tol (at most coarse_maxiter iterations);
//   3. prolong e_c onto the fine walls;
//   4. post-smooth: post_smooth GCR iterations on A z = r starting from the
//      prolonged correction (0 pre-smoothing).
// The smoother's final residual gives A z = r - r_s without another apply.
// All Krylov scalars stay on the device (FP64 reductions); the host reads them
// once per outer iteration and once per batch of coarse iterations.
#include <chrono>
#include <string.h>

#include "mg.cuh"

namespace dwf {

constexpr int GCR_MAXK = 32;

struct GcrScal {
    double coef[GCR_MAXK][2];
    double nrm[GCR_MAXK];
    double alpha[2];
    double rr2;
    double pad;
};

struct CoarseCg {
    double rn2, bn2, alpha, beta, rr2;
    int done, iters;
};

struct SolveScal {
    GcrScal outer;
    GcrScal smooth;
    GcrScal cgcr;        // coarse GCR
    int cdone, citers;   // coarse GCR stop flag and iteration count (per solve)
    double cref2;        // |r_c|^2 of the coarse right-hand side
    CoarseCg ccg;
    double misc[8];
    double pcg_rr2;
    int pcg_iters;
    int pad;
    unsigned bar[4];
};

// --------------------------------------------------------------------------
// FP32 vector kernels with FP64 reductions
// --------------------------------------------------------------------------
#define GRID_LOOP(i, n) for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < (n); i += (long long)gridDim.x * blockDim.x)

// coef = <Wj, w> / nrm_j
__global__ void __launch_bounds__(RED_THREADS) k_ortho_first(const float2* __restrict__ Wj, const float2* __restrict__ w,
                                                             long long n, RedScratch rs, double* coef, const double* nrm_j,
                                                             const int* skip) {
    if (skip && *skip) return;
    double v[2] = {0.0, 0.0};
    GRID_LOOP(i, n) {
        float2 a = Wj[i], b = w[i];
        v[0] += (double)a.x * b.x + (double)a.y * b.y;
        v[1] += (double)a.x * b.y - (double)a.y * b.x;
    }
    grid_reduce<2>(v, rs, [=] __device__(double* t) {
        const double nn = *nrm_j;
        coef[0] = nn > 0 ? t[0] / nn : 0.0;
        coef[1] = nn > 0 ? t[1] / nn : 0.0;
    });
}

// w -= c Wj, z -= c Zj (if Wj != null); then either
//   next coef = <Wn, w> / nrm_next           (Wn != null), or
//   nrm_out = |w|^2, alpha = <w, r> / |w|^2 (Wn == null)
template <bool LAST>
__global__ void __launch_bounds__(RED_THREADS) k_ortho_step(float2* __restrict__ w, float2* __restrict__ z,
                                                            const float2* __restrict__ Wj, const float2* __restrict__ Zj,
                                                            const double* coef, const float2* __restrict__ Wn,
                                                            const float2* __restrict__ r, long long n, RedScratch rs,
                                                            double* out, const double* nrm_next, double* alpha_out,
                                                            const int* skip) {
    if (skip && *skip) return;
    float cr = 0.f, ci = 0.f;
    if (Wj) { cr = (float)coef[0]; ci = (float)coef[1]; }
    double v[3] = {0.0, 0.0, 0.0};
    GRID_LOOP(i, n) {
        float2 wi = w[i];
        if (Wj) {
            float2 a = Wj[i], b = Zj[i], zi = z[i];
            wi.x -= cr * a.x - ci * a.y; wi.y -= cr * a.y + ci * a.x;
            zi.x -= cr * b.x - ci * b.y; zi.y -= cr * b.y + ci * b.x;
            w[i] = wi; z[i] = zi;
        }
        if (!LAST) {
            float2 a = Wn[i];
            v[0] += (double)a.x * wi.x + (double)a.y * wi.y;
            v[1] += (double)a.x * wi.y - (double)a.y * wi.x;
        } else {
            float2 ri = r[i];
            v[0] += (double)wi.x * wi.x + (double)wi.y * wi.y;
            v[1] += (double)wi.x * ri.x + (double)wi.y * ri.y;
            v[2] += (double)wi.x * ri.y - (double)wi.y * ri.x;
        }
    }
    grid_reduce<3>(v, rs, [=] __device__(double* t) {
        if (!LAST) {
            const double nn = *nrm_next;
            out[0] = nn > 0 ? t[0] / nn : 0.0;
            out[1] = nn > 0 ? t[1] / nn : 0.0;
        } else {
            out[0] = t[0];
            alpha_out[0] = t[0] > 0 ? t[1] / t[0] : 0.0;
            alpha_out[1] = t[0] > 0 ? t[2] / t[0] : 0.0;
        }
    });
}

// x += alpha z, r -= alpha w, rr2 = |r|^2.  With a stop flag: skipped once
// *done is set, and *done is set when rr2 <= tol2 * (*ref2) or the iteration
// counter reaches maxit.
__global__ void __launch_bounds__(RED_THREADS) k_gcr_update(float2* __restrict__ x, float2* __restrict__ r,
                                                            const float2* __restrict__ z, const float2* __restrict__ w,
                                                            const double* alpha, long long n, RedScratch rs, double* rr2,
                                                            int* done, const double* ref2, double tol2, int* iters,
                                                            int maxit) {
    if (done && *done) return;
    const float ar = (float)alpha[0], ai = (float)alpha[1];
    double v[1] = {0.0};
    GRID_LOOP(i, n) {
        float2 zi = z[i], wi = w[i], xi = x[i], ri = r[i];
        xi.x += ar * zi.x - ai * zi.y; xi.y += ar * zi.y + ai * zi.x;
        ri.x -= ar * wi.x - ai * wi.y; ri.y -= ar * wi.y + ai * wi.x;
        x[i] = xi; r[i] = ri;
        v[0] += (double)ri.x * ri.x + (double)ri.y * ri.y;
    }
    grid_reduce<1>(v, rs, [=] __device__(double* t) {
        *rr2 = t[0];
        if (done) {
            *iters += 1;
            if (t[0] <= tol2 * (*ref2) || *iters >= maxit) *done = 1;
        }
    });
}

__global__ void k_sub32(float2* __restrict__ out, const float2* __restrict__ a, const float2* __restrict__ b, long long n) {
    GRID_LOOP(i, n) { float2 x = a[i], y = b[i]; out[i] = make_float2(x.x - y.x, x.y - y.y); }
}

__global__ void k_sub64(double2* __restrict__ out, const double2* __restrict__ a, const double2* __restrict__ b, long long n) {
    GRID_LOOP(i, n) { double2 x = a[i], y = b[i]; out[i] = make_double2(x.x - y.x, x.y - y.y); }
}

__global__ void k_d2f_scale(float2* __restrict__ out, const double2* __restrict__ a, double s, long long n) {
    GRID_LOOP(i, n) { double2 x = a[i]; out[i] = make_float2((float)(x.x * s), (float)(x.y * s)); }
}

__global__ void k_axpy_64_32(double2* __restrict__ x, const float2* __restrict__ e, double s, long long n) {
    GRID_LOOP(i, n) { double2 v = x[i]; float2 d = e[i]; v.x += s * d.x; v.y += s * d.y; x[i] = v; }
}

// ---- coarse CGNR -----------------------------------------------------------
__global__ void __launch_bounds__(RED_THREADS) k_ccg_init(const float2* __restrict__ r, const float2* __restrict__ rhat,
                                                          long long n, RedScratch rs, CoarseCg* S) {
    double v[2] = {0.0, 0.0};
    GRID_LOOP(i, n) {
        float2 a = r[i], b = rhat[i];
        v[0] += (double)a.x * a.x + (double)a.y * a.y;
        v[1] += (double)b.x * b.x + (double)b.y * b.y;
    }
    grid_reduce<2>(v, rs, [=] __device__(double* t) {
        S->rn2 = t[0]; S->bn2 = t[1]; S->rr2 = t[1]; S->iters = 0;
        S->done = (t[1] == 0.0 || t[0] == 0.0) ? 1 : 0;
    });
}

__global__ void __launch_bounds__(RED_THREADS) k_ccg_alpha(const float2* __restrict__ q, long long n, RedScratch rs, CoarseCg* S) {
    if (S->done) return;
    double v[1] = {0.0};
    GRID_LOOP(i, n) { float2 a = q[i]; v[0] += (double)a.x * a.x + (double)a.y * a.y; }
    grid_reduce<1>(v, rs, [=] __device__(double* t) {
        if (t[0] > 0.0) S->alpha = S->rn2 / t[0];
        else { S->alpha = 0.0; S->done = 1; }
    });
}

__global__ void __launch_bounds__(RED_THREADS) k_ccg_upd1(float2* __restrict__ e, float2* __restrict__ rr,
                                                          const float2* __restrict__ p, const float2* __restrict__ q,
                                                          long long n, RedScratch rs, CoarseCg* S, double tol2, int maxiter) {
    if (S->done) return;
    const float a = (float)S->alpha;
    double v[1] = {0.0};
    GRID_LOOP(i, n) {
        float2 pi = p[i], qi = q[i], ei = e[i], ri = rr[i];
        ei.x += a * pi.x; ei.y += a * pi.y;
        ri.x -= a * qi.x; ri.y -= a * qi.y;
        e[i] = ei; rr[i] = ri;
        v[0] += (double)ri.x * ri.x + (double)ri.y * ri.y;
    }
    grid_reduce<1>(v, rs, [=] __device__(double* t) {
        S->rr2 = t[0];
        S->iters += 1;
        if (t[0] <= tol2 * S->bn2 || S->iters >= maxiter) S->done = 1;
    });
}

__global__ void __launch_bounds__(RED_THREADS) k_ccg_upd2(float2* __restrict__ r, const float2* __restrict__ w, long long n,
                                                          RedScratch rs, CoarseCg* S) {
    if (S->done) return;
    const float a = (float)S->alpha;
    double v[1] = {0.0};
    GRID_LOOP(i, n) {
        float2 ri = r[i], wi = w[i];
        ri.x -= a * wi.x; ri.y -= a * wi.y;
        r[i] = ri;
        v[0] += (double)ri.x * ri.x + (double)ri.y * ri.y;
    }
    grid_reduce<1>(v, rs, [=] __device__(double* t) {
        S->beta = S->rn2 > 0 ? t[0] / S->rn2 : 0.0;
        S->rn2 = t[0];
    });
}

__global__ void k_ccg_p(float2* __restrict__ p, const float2* __restrict__ r, long long n, const CoarseCg* S) {
    if (S->done) return;
    const float b = (float)S->beta;
    GRID_LOOP(i, n) { float2 pi = p[i], ri = r[i]; p[i] = make_float2(ri.x + b * pi.x, ri.y + b * pi.y); }
}

static int ew_grid(long long n) {
    long long b = (n + 255) / 256;
    return (int)(b < 152LL * 8 ? b : 152LL * 8);
}

// --------------------------------------------------------------------------
// solver state
// --------------------------------------------------------------------------
struct Solver {
    dwf_mg* h;
    cudaStream_t st;
    long long nf, nc;
    int rg, eg, rgc, egc;
    SolveScal* d;        // device scalars
    SolveScal* hs;       // pinned host mirror
    // fine FP32
    float2 *rA, *r, *e, *tmp, *zs, *rs_, *ps;
    float2 *Z[GCR_MAXK], *W[GCR_MAXK];
    float2 *Ps[GCR_MAXK], *Qs[GCR_MAXK];
    // coarse FP32
    float2 *rc, *ec, *crr, *cr, *cp, *cq, *cw, *ct;
    // FP64
    double2 *r64, *t64;
    double* partials;    // persistent coarse solver partial sums
    float2 *Zc[GCR_MAXK], *Wc[GCR_MAXK];   // coarse GCR basis
    long long fine_applies, coarse_applies, coarse_iters, coarse_solves;
};

static dwf_status ensure_workspace(dwf_mg* h) {
    if (h->ws_ready) return DWF_OK;
    const long long nf = fine_len(h), nc = coarse_len(h);
    const int K = h->prm.gcr_restart, S = h->prm.post_smooth;
    const int nfine = 7 + 2 * K + 2 * S;
    for (int k = 0; k < nfine; ++k) {
        void* p = nullptr;
        cudaError_t e = cudaMalloc(&p, nf * sizeof(float2));
        if (e != cudaSuccess) { set_error("solver vectors: %s", cudaGetErrorString(e)); return DWF_ERR_OOM; }
        h->fine_vecs.push_back(p);
    }
    const int KC = h->prm.coarse_restart;
    for (int k = 0; k < 9 + 2 * KC; ++k) {   // 8 coarse vectors, persistent-solver partials, coarse GCR basis
        void* p = nullptr;
        cudaError_t e = cudaMalloc(&p, k == 8 ? 3 * 4096 * sizeof(double) : nc * sizeof(float2) + 256);
        if (e != cudaSuccess) { set_error("coarse vectors: %s", cudaGetErrorString(e)); return DWF_ERR_OOM; }
        h->coarse_vecs.push_back(p);
    }
    DWF_TRY(mg_alloc(h, &h->r64, nf * sizeof(double2)));
    DWF_TRY(mg_alloc(h, &h->x64, nf * sizeof(double2)));    // used as the FP64 apply temporary
    void* d = nullptr;
    DWF_CHECK_CUDA(cudaMalloc(&d, sizeof(SolveScal)));
    h->coarse_vecs.push_back(d);       // last coarse slot: device scalars
    DWF_CHECK_CUDA(cudaMallocHost((void**)&h->hsc, sizeof(SolveScal)));
    h->ws_ready = true;
    return DWF_OK;
}

static void bind(Solver& s, dwf_mg* h) {
    s.h = h;
    s.st = h->st;
    s.nf = fine_len(h);
    s.nc = coarse_len(h);
    s.rg = red_grid(s.nf);
    s.eg = ew_grid(s.nf);
    s.rgc = red_grid(s.nc);
    s.egc = ew_grid(s.nc);
    int i = 0;
    auto F = [&]() { return (float2*)h->fine_vecs[i++]; };
    s.rA = F(); s.r = F(); s.e = F(); s.tmp = F(); s.zs = F(); s.rs_ = F(); s.ps = F();
    for (int k = 0; k < h->prm.gcr_restart; ++k) { s.Z[k] = F(); s.W[k] = F(); }
    for (int k = 0; k < h->prm.post_smooth; ++k) { s.Ps[k] = F(); s.Qs[k] = F(); }
    auto C = [&](int j) { return (float2*)h->coarse_vecs[j]; };
    s.rc = C(0); s.ec = C(1); s.crr = C(2); s.cr = C(3); s.cp = C(4); s.cq = C(5); s.cw = C(6); s.ct = C(7);
    s.partials = (double*)h->coarse_vecs[8];
    for (int k = 0; k < h->prm.coarse_restart; ++k) {
        s.Zc[k] = (float2*)h->coarse_vecs[9 + 2 * k];
        s.Wc[k] = (float2*)h->coarse_vecs[10 + 2 * k];
    }
    s.d = (SolveScal*)h->coarse_vecs[9 + 2 * h->prm.coarse_restart];
    s.hs = (SolveScal*)h->hsc;
    s.r64 = (double2*)h->r64;
    s.t64 = (double2*)h->x64;
    s.fine_applies = s.coarse_applies = s.coarse_iters = s.coarse_solves = 0;
}

// out = A in = D_PV^dag D_DW in (FP32, fine link storage)
static dwf_status apply_A(Solver& s, const float2* in, float2* out) {
    dwf_mg* h = s.h;
    DWF_TRY(fine_apply(h->G, h->Ulo, in, s.tmp, h->M5, h->mf, false, h->prm.fine_prec, s.st));
    DWF_TRY(fine_apply(h->G, h->Ulo, s.tmp, out, h->M5, 1.0, true, h->prm.fine_prec, s.st));
    s.fine_applies += 2;
    return DWF_OK;
}

// Orthogonalise (z, w) = (Z[k], W[k]) against the first k pairs of the basis
// and compute nrm[k], alpha = <w, r> / nrm[k].
static dwf_status gcr_orthogonalise(Solver& s, GcrScal* g, float2** Zb, float2** Wb, int k, const float2* r, long long n,
                                    const int* skip = nullptr) {
    RedScratch rs = s.h->ws.red();
    const int rg = red_grid(n);
    if (k == 0) {
        k_ortho_step<true><<<rg, RED_THREADS, 0, s.st>>>(Wb[0], Zb[0], nullptr, nullptr, nullptr, nullptr, r, n, rs,
                                                         &g->nrm[0], nullptr, g->alpha, skip);
        DWF_CHECK_LAUNCH();
        return DWF_OK;
    }
    k_ortho_first<<<rg, RED_THREADS, 0, s.st>>>(Wb[0], Wb[k], n, rs, g->coef[0], &g->nrm[0], skip);
    for (int j = 0; j < k; ++j) {
        if (j + 1 < k)
            k_ortho_step<false><<<rg, RED_THREADS, 0, s.st>>>(Wb[k], Zb[k], Wb[j], Zb[j], g->coef[j], Wb[j + 1], nullptr,
                                                              n, rs, g->coef[j + 1], &g->nrm[j + 1], nullptr, skip);
        else
            k_ortho_step<true><<<rg, RED_THREADS, 0, s.st>>>(Wb[k], Zb[k], Wb[j], Zb[j], g->coef[j], nullptr, r, n, rs,
                                                             &g->nrm[k], nullptr, g->alpha, skip);
    }
    DWF_CHECK_LAUNCH();
    return DWF_OK;
}

// Coarse solve with restarted GCR on B e = r_c, B = Dhat_PV^dag Dhat_DW (the
// paper's level-2 operator and solver type; B's spectrum lies in the right
// half plane, App. B).  Iterations run in batches of one restart cycle with a
// device-side stop flag; the host reads the flag once per cycle.
static dwf_status coarse_solve_gcr(Solver& s) {
    dwf_mg* h = s.h;
    const long long n = s.nc;
    RedScratch rs = h->ws.red();
    GcrScal* g = &s.d->cgcr;
    int* done = &s.d->cdone;
    const int K = h->prm.coarse_restart;
    const int maxit = h->prm.coarse_maxiter;
    const double tol2 = h->prm.coarse_tol * h->prm.coarse_tol;
    DWF_CHECK_CUDA(cudaMemsetAsync(s.ec, 0, n * sizeof(float2), s.st));
    DWF_CHECK_CUDA(cudaMemcpyAsync(s.crr, s.rc, n * sizeof(float2), cudaMemcpyDeviceToDevice, s.st));
    DWF_CHECK_CUDA(cudaMemsetAsync(&s.d->cdone, 0, 2 * sizeof(int), s.st));
    DWF_TRY(dot_device(s.rc, s.rc, n, false, rs, s.d->misc + 4, s.st));
    DWF_CHECK_CUDA(cudaMemcpyAsync(&s.d->cref2, s.d->misc + 4, sizeof(double), cudaMemcpyDeviceToDevice, s.st));
    int launched = 0;
    while (launched < maxit) {
        for (int k = 0; k < K && launched < maxit; ++k, ++launched) {
            DWF_CHECK_CUDA(cudaMemcpyAsync(s.Zc[k], s.crr, n * sizeof(float2), cudaMemcpyDeviceToDevice, s.st));
            DWF_TRY(coarse_dwf_apply(h, s.Zc[k], s.ct, h->mf, false, done, s.st));
            DWF_TRY(coarse_dwf_apply(h, s.ct, s.Wc[k], 1.0, true, done, s.st));
            DWF_TRY(gcr_orthogonalise(s, g, s.Zc, s.Wc, k, s.crr, n, done));
            k_gcr_update<<<s.rgc, RED_THREADS, 0, s.st>>>(s.ec, s.crr, s.Zc[k], s.Wc[k], g->alpha, n, rs, &g->rr2, done,
                                                          &s.d->cref2, tol2, &s.d->citers, maxit);
            DWF_CHECK_LAUNCH();
        }
        DWF_CHECK_CUDA(cudaMemcpyAsync(&s.hs->cdone, &s.d->cdone, 2 * sizeof(int), cudaMemcpyDeviceToHost, s.st));
        DWF_CHECK_CUDA(cudaStreamSynchronize(s.st));
        if (s.hs->cdone) break;
    }
    s.coarse_iters += s.hs->citers;
    s.coarse_applies += 2LL * s.hs->citers;
    s.coarse_solves += 1;
    return DWF_OK;
}

// Coarse solve: CGNR on B^dag B e = B^dag r, B = Dhat_PV^dag Dhat_DW.
static dwf_status coarse_solve(Solver& s) {
    dwf_mg* h = s.h;
    if (h->prm.coarse_solver == 1) return coarse_solve_gcr(s);
    if (h->prm.coarse_persistent && h->mg.ncd == 16 && h->mg.Ls_c <= 4 && h->mg.nd == 2) {
        float2* v6[6] = {s.crr, s.cr, s.cp, s.cq, s.ct, s.cw};
        DWF_TRY(coarse_cgnr_persistent(h, s.rc, s.ec, v6, s.partials, s.d->bar, &s.d->pcg_iters, &s.d->pcg_rr2, s.st));
        s.coarse_solves += 1;
        return DWF_OK;
    }
    RedScratch rs = h->ws.red();
    CoarseCg* S = &s.d->ccg;
    const int* done = &S->done;
    const long long n = s.nc;
    const double mf = h->mf;
    // B^dag x = Dhat_DW^dag Dhat_PV x
    DWF_CHECK_CUDA(cudaMemsetAsync(s.ec, 0, n * sizeof(float2), s.st));
    DWF_CHECK_CUDA(cudaMemcpyAsync(s.crr, s.rc, n * sizeof(float2), cudaMemcpyDeviceToDevice, s.st));
    DWF_TRY(coarse_dwf_apply(h, s.crr, s.ct, 1.0, false, nullptr, s.st));
    DWF_TRY(coarse_dwf_apply(h, s.ct, s.cr, mf, true, nullptr, s.st));
    s.coarse_applies += 2;
    k_ccg_init<<<s.rgc, RED_THREADS, 0, s.st>>>(s.cr, s.rc, n, rs, S);
    DWF_CHECK_CUDA(cudaMemcpyAsync(s.cp, s.cr, n * sizeof(float2), cudaMemcpyDeviceToDevice, s.st));
    const double tol2 = h->prm.coarse_tol * h->prm.coarse_tol;
    const int maxit = h->prm.coarse_maxiter;
    int launched = 0;
    const int batch = 32;
    while (launched < maxit) {
        for (int k = 0; k < batch && launched < maxit; ++k, ++launched) {
            DWF_TRY(coarse_dwf_apply(h, s.cp, s.ct, mf, false, done, s.st));      // t = Dhat_DW p
            DWF_TRY(coarse_dwf_apply(h, s.ct, s.cq, 1.0, true, done, s.st));      // q = Dhat_PV^dag t
            k_ccg_alpha<<<s.rgc, RED_THREADS, 0, s.st>>>(s.cq, n, rs, S);
            k_ccg_upd1<<<s.rgc, RED_THREADS, 0, s.st>>>(s.ec, s.crr, s.cp, s.cq, n, rs, S, tol2, maxit);
            DWF_TRY(coarse_dwf_apply(h, s.cq, s.ct, 1.0, false, done, s.st));     // t = Dhat_PV q
            DWF_TRY(coarse_dwf_apply(h, s.ct, s.cw, mf, true, done, s.st));       // w = Dhat_DW^dag t
            k_ccg_upd2<<<s.rgc, RED_THREADS, 0, s.st>>>(s.cr, s.cw, n, rs, S);
            k_ccg_p<<<s.egc, 256, 0, s.st>>>(s.cp, s.cr, n, S);
            DWF_CHECK_LAUNCH();
        }
        DWF_CHECK_CUDA(cudaMemcpyAsync(&s.hs->ccg, S, sizeof(CoarseCg), cudaMemcpyDeviceToHost, s.st));
        DWF_CHECK_CUDA(cudaStreamSynchronize(s.st));
        if (s.hs->ccg.done) break;
    }
    s.coarse_iters += s.hs->ccg.iters;
    s.coarse_applies += 4LL * s.hs->ccg.iters;
    s.coarse_solves += 1;
    return DWF_OK;
}

// z = M(r): restrict, coarse solve, prolong, post-smooth.  Writes z into zout
// and w = A z into wout.
static dwf_status precondition(Solver& s, const float2* r, float2* zout, float2* wout) {
    dwf_mg* h = s.h;
    const long long n = s.nf;
    RedScratch rs = h->ws.red();
    DWF_TRY(restrict_wall(h, r, s.rc, nullptr, s.st));
    DWF_TRY(coarse_solve(s));
    DWF_TRY(prolong_wall(h, s.ec, zout, nullptr, s.st));
    const int S = h->prm.post_smooth;
    if (S == 0) return apply_A(s, zout, wout);
    // smoother residual r_s = r - A z0
    DWF_TRY(apply_A(s, zout, s.ps));
    k_sub32<<<s.eg, 256, 0, s.st>>>(s.rs_, r, s.ps, n);
    DWF_CHECK_LAUNCH();
    GcrScal* g = &s.d->smooth;
    for (int j = 0; j < S; ++j) {
        DWF_CHECK_CUDA(cudaMemcpyAsync(s.Ps[j], s.rs_, n * sizeof(float2), cudaMemcpyDeviceToDevice, s.st));
        DWF_TRY(apply_A(s, s.Ps[j], s.Qs[j]));
        DWF_TRY(gcr_orthogonalise(s, g, s.Ps, s.Qs, j, s.rs_, n));
        k_gcr_update<<<s.rg, RED_THREADS, 0, s.st>>>(zout, s.rs_, s.Ps[j], s.Qs[j], g->alpha, n, rs, &g->rr2,
                                                     nullptr, nullptr, 0.0, nullptr, 0);
        DWF_CHECK_LAUNCH();
    }
    // A z = r - r_s
    k_sub32<<<s.eg, 256, 0, s.st>>>(wout, r, s.rs_, n);
    DWF_CHECK_LAUNCH();
    return DWF_OK;
}

static dwf_status true_residual(Solver& s, const double2* b, const double2* x, double* rn2) {
    dwf_mg* h = s.h;
    DWF_TRY(fine_apply(h->G, h->U64, x, s.t64, h->M5, h->mf, false, DWF_F64, s.st));
    s.fine_applies += 1;
    k_sub64<<<s.eg, 256, 0, s.st>>>(s.r64, b, s.t64, s.nf);
    DWF_CHECK_LAUNCH();
    DWF_TRY(dot_device(s.r64, s.r64, s.nf, true, h->ws.red(), s.d->misc, s.st));
    DWF_CHECK_CUDA(cudaMemcpyAsync(s.hs->misc, s.d->misc, 2 * sizeof(double), cudaMemcpyDeviceToHost, s.st));
    DWF_CHECK_CUDA(cudaStreamSynchronize(s.st));
    *rn2 = s.hs->misc[0];
    return DWF_OK;
}

}  // namespace dwf

using namespace dwf;

extern "C" dwf_status mg_solve(dwf_mg* h, const void* b, void* x, double tol, int maxiter, dwf_solve_stats* stats,
                               void* stream) {
    clear_error();
    auto t0 = std::chrono::steady_clock::now();
    if (stats) memset(stats, 0, sizeof(*stats));
    if (!h || !b || !x) { set_error("NULL argument"); return DWF_ERR_ARG; }
    if (!(tol > 0.0)) { set_error("tol must be > 0"); return DWF_ERR_ARG; }
    if (h->prm.gcr_restart > GCR_MAXK || h->prm.post_smooth > GCR_MAXK || h->prm.coarse_restart > GCR_MAXK ||
        h->prm.coarse_restart < 1) {
        set_error("gcr_restart, post_smooth and coarse_restart must be in [1, %d]", GCR_MAXK); return DWF_ERR_ARG;
    }
    if (stream) h->st = as_stream(stream);
    DWF_TRY(ensure_workspace(h));
    Solver s;
    bind(s, h);
    const long long n = s.nf;
    const double2* B = (const double2*)b;
    double2* X = (double2*)x;
    RedScratch rs = h->ws.red();
    DWF_CHECK_CUDA(cudaMemsetAsync(X, 0, n * sizeof(double2), s.st));
    DWF_CHECK_CUDA(cudaMemsetAsync(&s.d->pcg_iters, 0, sizeof(int), s.st));
    DWF_CHECK_CUDA(cudaMemsetAsync(s.d->bar, 0, sizeof(s.d->bar), s.st));
    DWF_TRY(dot_device(B, B, n, true, rs, s.d->misc, s.st));
    DWF_CHECK_CUDA(cudaMemcpyAsync(s.hs->misc, s.d->misc, 2 * sizeof(double), cudaMemcpyDeviceToHost, s.st));
    DWF_CHECK_CUDA(cudaStreamSynchronize(s.st));
    const double bn2 = s.hs->misc[0];
    dwf_status status = DWF_ERR_NOCONV;
    double res = bn2 > 0 ? 1.0 : 0.0;
    int outer = 0, restarts = 0;
    if (bn2 == 0.0) status = DWF_OK;
    GcrScal* g = &s.d->outer;
    const int K = h->prm.gcr_restart;
    while (status != DWF_OK) {
        double rn2;
        if (restarts == 0) {
            DWF_CHECK_CUDA(cudaMemcpyAsync(s.r64, B, n * sizeof(double2), cudaMemcpyDeviceToDevice, s.st));
            rn2 = bn2;
        } else {
            DWF_TRY(true_residual(s, B, X, &rn2));
        }
        res = sqrt(rn2 / bn2);
        if (res <= tol) { status = DWF_OK; break; }
        if (outer >= maxiter || restarts > h->prm.max_restarts) break;
        ++restarts;
        // correction system in FP32: A e = D_PV^dag r / |r|
        const double rn = sqrt(rn2);
        k_d2f_scale<<<s.eg, 256, 0, s.st>>>(s.ps, s.r64, 1.0 / rn, n);
        DWF_TRY(fine_apply(h->G, h->Ulo, s.ps, s.rA, h->M5, 1.0, true, h->prm.fine_prec, s.st));
        s.fine_applies += 1;
        DWF_CHECK_CUDA(cudaMemcpyAsync(s.r, s.rA, n * sizeof(float2), cudaMemcpyDeviceToDevice, s.st));
        DWF_CHECK_CUDA(cudaMemsetAsync(s.e, 0, n * sizeof(float2), s.st));
        DWF_TRY(dot_device(s.rA, s.rA, n, false, rs, s.d->misc + 2, s.st));
        DWF_CHECK_CUDA(cudaMemcpyAsync(s.hs->misc + 2, s.d->misc + 2, sizeof(double), cudaMemcpyDeviceToHost, s.st));
        DWF_CHECK_CUDA(cudaStreamSynchronize(s.st));
        const double rA2 = s.hs->misc[2];
        double delta = h->prm.inner_tol;
        const double need = 0.5 * tol * sqrt(bn2) / rn;
        if (need > delta) delta = need;
        for (int k = 0; k < K && outer < maxiter; ++k) {
            DWF_TRY(precondition(s, s.r, s.Z[k], s.W[k]));
            DWF_TRY(gcr_orthogonalise(s, g, s.Z, s.W, k, s.r, n));
            k_gcr_update<<<s.rg, RED_THREADS, 0, s.st>>>(s.e, s.r, s.Z[k], s.W[k], g->alpha, n, rs, &g->rr2,
                                                         nullptr, nullptr, 0.0, nullptr, 0);
            DWF_CHECK_LAUNCH();
            ++outer;
            DWF_CHECK_CUDA(cudaMemcpyAsync(&s.hs->outer.rr2, &g->rr2, sizeof(double), cudaMemcpyDeviceToHost, s.st));
            DWF_CHECK_CUDA(cudaMemcpyAsync(s.hs->bar, s.d->bar, sizeof(s.d->bar), cudaMemcpyDeviceToHost, s.st));
            DWF_CHECK_CUDA(cudaStreamSynchronize(s.st));
            if (s.hs->bar[2] != 0u) {
                set_error("persistent coarse solver: a grid barrier timed out");
                return DWF_ERR_TIMEOUT;
            }
            if (s.hs->outer.rr2 <= delta * delta * rA2) break;
        }
        k_axpy_64_32<<<s.eg, 256, 0, s.st>>>(X, s.e, rn, n);
        DWF_CHECK_LAUNCH();
    }
    if (h->prm.coarse_solver == 0 && h->prm.coarse_persistent && h->mg.ncd == 16 && h->mg.Ls_c <= 4 && h->mg.nd == 2) {
        DWF_CHECK_CUDA(cudaMemcpyAsync(&s.hs->pcg_iters, &s.d->pcg_iters, sizeof(int), cudaMemcpyDeviceToHost, s.st));
        DWF_CHECK_CUDA(cudaMemcpyAsync(s.hs->bar, s.d->bar, sizeof(s.d->bar), cudaMemcpyDeviceToHost, s.st));
        DWF_CHECK_CUDA(cudaStreamSynchronize(s.st));
        s.coarse_iters = s.hs->pcg_iters;
        s.coarse_applies = 2 * s.coarse_solves + 4LL * s.coarse_iters;
        if (s.hs->bar[2] != 0u) {
            set_error("persistent coarse solver: a grid barrier or bulk copy timed out");
            status = DWF_ERR_TIMEOUT;
        }
    }
    {
        int st1 = 0;
        DWF_CHECK_CUDA(cudaMemcpyAsync(&st1, h->status + 1, sizeof(int), cudaMemcpyDeviceToHost, s.st));
        DWF_CHECK_CUDA(cudaStreamSynchronize(s.st));
        if (st1 != 0) {
            set_error("coarse stencil: a bulk copy wait timed out");
            status = DWF_ERR_TIMEOUT;
        }
    }
    if (status != DWF_OK && dwf_last_error()[0] == 0)
        set_error("mg_solve stopped after %d outer iterations with true residual %.3e > tol %.3e", outer, res, tol);
    if (stats) {
        stats->iterations = outer;
        stats->restarts = restarts;
        stats->fine_applies = s.fine_applies;
        stats->coarse_applies = s.coarse_applies;
        stats->coarse_avg_iters = s.coarse_solves ? (double)s.coarse_iters / s.coarse_solves : 0.0;
        stats->true_residual = res;
        stats->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
    return status;
}
