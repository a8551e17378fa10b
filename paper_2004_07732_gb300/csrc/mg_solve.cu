// The K-cycle solve of Sec. 2.3 ("Summary") with the Table kcycle parameters.
//
// mg_solve hands the default configuration (restarted GCR as the coarse
// solver, coarse_persistent != 2) to the batched K-cycle of mg_batched.cu with
// one right-hand side.  This file runs the same iteration for the CGNR coarse
// solver and for the persistent coarse GCR:
//
// Outer loop, FP64 (reliable updates): r = b - D_DW x with the FP64 operator;
// stop when ||r|| / ||b|| <= tol; otherwise solve the left-preconditioned
// correction system  D_PV^dag D_DW e = D_PV^dag r  approximately in FP32
// (spinors FP32, links in the handle's fine storage) and add e to x in FP64.
//
// Inner solver: flexible GCR, restart gcr_restart, on A = D_PV^dag D_DW with
// the preconditioner M(r):
//   1. restrict the wall of r onto the coarse walls (Eq. TruncProjectInterpolate);
//   2. solve Dhat_PV^dag Dhat_DW e_c = r_c to coarse_tol (at most
//      coarse_maxiter iterations): CGNR on the coarse normal operator, or the
//      persistent restarted GCR;
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
    float acc = 0.f;     // per-thread FP32 partial; FP64 from the warp sum on
    double v[1] = {0.0};
    float4* x4 = reinterpret_cast<float4*>(x);
    float4* r4 = reinterpret_cast<float4*>(r);
    const float4* z4 = reinterpret_cast<const float4*>(z);
    const float4* w4 = reinterpret_cast<const float4*>(w);
    const long long n2 = n >> 1;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n2; i += (long long)gridDim.x * blockDim.x) {
        const float4 zi = z4[i], wi = w4[i];
        float4 xi = x4[i], ri = r4[i];
        xi.x += ar * zi.x - ai * zi.y; xi.y += ar * zi.y + ai * zi.x;
        xi.z += ar * zi.z - ai * zi.w; xi.w += ar * zi.w + ai * zi.z;
        ri.x -= ar * wi.x - ai * wi.y; ri.y -= ar * wi.y + ai * wi.x;
        ri.z -= ar * wi.z - ai * wi.w; ri.w -= ar * wi.w + ai * wi.z;
        x4[i] = xi; r4[i] = ri;
        acc += ri.x * ri.x + ri.y * ri.y + ri.z * ri.z + ri.w * ri.w;
    }
    v[0] = acc;
    if ((n & 1) && blockIdx.x == 0 && threadIdx.x == 0) {
        const float2 zi = z[n - 1], wi = w[n - 1];
        float2 xi = x[n - 1], ri = r[n - 1];
        xi.x += ar * zi.x - ai * zi.y; xi.y += ar * zi.y + ai * zi.x;
        ri.x -= ar * wi.x - ai * wi.y; ri.y -= ar * wi.y + ai * wi.x;
        x[n - 1] = xi; r[n - 1] = ri;
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

// ---- classical Gram-Schmidt ------------------------------------------------
// Vectors are read as float4 (two complex values) so that every load moves 16
// bytes; loops are unrolled so several loads are in flight per thread.
// coef[j] (+)= <W_j, w> / nrm[j] for j < k.  Grid (B, k): block (b, j) reduces
// a slice of row j; the last block of row j (per-row completion counter)
// finalises coef[j] in a fixed order.
constexpr int MDOT_BLOCKS = 152;

// per-thread partials of FP32 products are kept in FP32 (a few terms per
// thread); the cross-thread sums are FP64
__device__ __forceinline__ void cdot_acc(const float4 a, const float4 b, float& re, float& im) {
    re += a.x * b.x + a.y * b.y + a.z * b.z + a.w * b.w;
    im += a.x * b.y - a.y * b.x + a.z * b.w - a.w * b.z;
}

__global__ void __launch_bounds__(RED_THREADS) k_mdot(float2* const* __restrict__ W, const float2* __restrict__ w,
                                                      long long n, double* __restrict__ part, unsigned* counters,
                                                      double (*coef)[2], const double* nrm, int accumulate,
                                                      const int* skip) {
    if (skip && *skip) return;
    const int j = blockIdx.y;
    const float4* Wj = reinterpret_cast<const float4*>(W[j]);
    const float4* w4 = reinterpret_cast<const float4*>(w);
    const long long n2 = n >> 1;
    float re = 0.f, im = 0.f;
    const long long stride = (long long)gridDim.x * blockDim.x;
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    for (; i + 3 * stride < n2; i += 4 * stride) {
        const float4 a0 = Wj[i], a1 = Wj[i + stride], a2 = Wj[i + 2 * stride], a3 = Wj[i + 3 * stride];
        const float4 b0 = w4[i], b1 = w4[i + stride], b2 = w4[i + 2 * stride], b3 = w4[i + 3 * stride];
        cdot_acc(a0, b0, re, im);
        cdot_acc(a1, b1, re, im);
        cdot_acc(a2, b2, re, im);
        cdot_acc(a3, b3, re, im);
    }
    for (; i < n2; i += stride) cdot_acc(Wj[i], w4[i], re, im);
    if ((n & 1) && blockIdx.x == 0 && threadIdx.x == 0) {
        const float2 a = W[j][n - 1], b = w[n - 1];
        re += a.x * b.x + a.y * b.y;
        im += a.x * b.y - a.y * b.x;
    }
    double v[2] = {re, im};
    block_sum<2>(v);
    if (threadIdx.x == 0) {
        part[(2 * j) * MDOT_BLOCKS + blockIdx.x] = v[0];
        part[(2 * j + 1) * MDOT_BLOCKS + blockIdx.x] = v[1];
    }
    if (!grid_last_block(counters + (size_t)j * (RED_GROUPS + 1) * RED_CSTRIDE)) return;
    __threadfence();
    // the partials of row j are summed by the whole block (strided, then a
    // fixed-order block reduction)
    double w2[2] = {0.0, 0.0};
    for (unsigned bb = threadIdx.x; bb < gridDim.x; bb += blockDim.x) {
        w2[0] += __ldcg(part + (2 * j) * MDOT_BLOCKS + bb);
        w2[1] += __ldcg(part + (2 * j + 1) * MDOT_BLOCKS + bb);
    }
    block_sum<2>(w2);
    if (threadIdx.x == 0) {
        const double nn = nrm[j];
        const double re = nn > 0 ? w2[0] / nn : 0.0;
        const double im = nn > 0 ? w2[1] / nn : 0.0;
        if (accumulate) { coef[j][0] += re; coef[j][1] += im; }
        else { coef[j][0] = re; coef[j][1] = im; }
    }
}

// w -= sum_j c_j W_j and z -= sum_j c_j Z_j.  FINAL: also nrm_out = |w|^2 and
// alpha = <w, r> / |w|^2 (grid reduction).
__device__ __forceinline__ void csub2(float4& x, const float4 a, const float2 c) {
    x.x -= c.x * a.x - c.y * a.y; x.y -= c.x * a.y + c.y * a.x;
    x.z -= c.x * a.z - c.y * a.w; x.w -= c.x * a.w + c.y * a.z;
}

template <bool FINAL>
__global__ void __launch_bounds__(RED_THREADS) k_maxpy(float2* __restrict__ w, float2* __restrict__ z,
                                                       float2* const* __restrict__ W, float2* const* __restrict__ Z,
                                                       const double (*coef)[2], int k, const float2* __restrict__ r,
                                                       long long n, RedScratch rs, double* nrm_out, double* alpha_out,
                                                       const int* skip) {
    if (skip && *skip) return;
    __shared__ float2 c[GCR_MAXK];
    __shared__ const float4* Wp[GCR_MAXK];
    __shared__ const float4* Zp[GCR_MAXK];
    for (int j = threadIdx.x; j < k; j += blockDim.x) {
        c[j] = make_float2((float)coef[j][0], (float)coef[j][1]);
        Wp[j] = reinterpret_cast<const float4*>(W[j]);
        Zp[j] = reinterpret_cast<const float4*>(Z[j]);
    }
    __syncthreads();
    float4* w4 = reinterpret_cast<float4*>(w);
    float4* z4 = reinterpret_cast<float4*>(z);
    const float4* r4 = reinterpret_cast<const float4*>(r);
    const long long n2 = n >> 1;
    float f0 = 0.f, f1 = 0.f, f2 = 0.f;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n2; i += (long long)gridDim.x * blockDim.x) {
        float4 wi = w4[i], zi = k > 0 ? z4[i] : make_float4(0.f, 0.f, 0.f, 0.f);
        int j = 0;
        for (; j + 3 < k; j += 4) {
            const float4 a0 = Wp[j][i], a1 = Wp[j + 1][i], a2 = Wp[j + 2][i], a3 = Wp[j + 3][i];
            const float4 b0 = Zp[j][i], b1 = Zp[j + 1][i], b2 = Zp[j + 2][i], b3 = Zp[j + 3][i];
            csub2(wi, a0, c[j]); csub2(wi, a1, c[j + 1]); csub2(wi, a2, c[j + 2]); csub2(wi, a3, c[j + 3]);
            csub2(zi, b0, c[j]); csub2(zi, b1, c[j + 1]); csub2(zi, b2, c[j + 2]); csub2(zi, b3, c[j + 3]);
        }
        for (; j < k; ++j) { csub2(wi, Wp[j][i], c[j]); csub2(zi, Zp[j][i], c[j]); }
        if (k > 0) { w4[i] = wi; z4[i] = zi; }
        if (FINAL) {
            const float4 ri = r4[i];
            f0 += wi.x * wi.x + wi.y * wi.y + wi.z * wi.z + wi.w * wi.w;
            cdot_acc(wi, ri, f1, f2);
        }
    }
    double v[3] = {f0, f1, f2};
    if ((n & 1) && blockIdx.x == 0 && threadIdx.x == 0) {     // odd tail element
        float2 wi = w[n - 1], zi = z[n - 1];
        for (int j = 0; j < k; ++j) {
            const float2 a = W[j][n - 1], b = Z[j][n - 1];
            wi.x -= c[j].x * a.x - c[j].y * a.y; wi.y -= c[j].x * a.y + c[j].y * a.x;
            zi.x -= c[j].x * b.x - c[j].y * b.y; zi.y -= c[j].x * b.y + c[j].y * b.x;
        }
        if (k > 0) { w[n - 1] = wi; z[n - 1] = zi; }
        if (FINAL) {
            const float2 ri = r[n - 1];
            v[0] += (double)wi.x * wi.x + (double)wi.y * wi.y;
            v[1] += (double)wi.x * ri.x + (double)wi.y * ri.y;
            v[2] += (double)wi.x * ri.y - (double)wi.y * ri.x;
        }
    }
    if (FINAL)
        grid_reduce<3>(v, rs, [=] __device__(double* t) {
            *nrm_out = t[0];
            alpha_out[0] = t[0] > 0 ? t[1] / t[0] : 0.0;
            alpha_out[1] = t[0] > 0 ? t[2] / t[0] : 0.0;
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
    float2** dptr;       // device copies of the basis pointer arrays: Z, W, Ps, Qs, Zc, Wc
    double* mpart;       // CGS partial sums [2 GCR_MAXK][MDOT_BLOCKS]
    unsigned* mcount;    // CGS per-row completion counters [GCR_MAXK]
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
    {
        void* p = nullptr;   // 6 pointer arrays + CGS partials + counters
        const size_t bytes = 6 * GCR_MAXK * sizeof(float2*) + 2 * GCR_MAXK * MDOT_BLOCKS * sizeof(double) +
                             (size_t)GCR_MAXK * (RED_GROUPS + 1) * RED_CSTRIDE * sizeof(unsigned);
        cudaError_t e = cudaMalloc(&p, bytes);
        if (e != cudaSuccess) { set_error("solver pointer arrays: %s", cudaGetErrorString(e)); return DWF_ERR_OOM; }
        DWF_CHECK_CUDA(cudaMemset(p, 0, bytes));
        h->solver_meta = p;
    }
    const int KC = h->prm.coarse_restart;
    for (int k = 0; k < 9 + 2 * KC; ++k) {   // 8 coarse vectors, persistent-solver partials, coarse GCR basis
        void* p = nullptr;
        cudaError_t e = cudaMalloc(&p, k == 8 ? 64 * 1024 * sizeof(double) : nc * sizeof(float2) + 256);
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
    s.rg = red_grid4(s.nf);
    s.eg = ew_grid(s.nf);
    s.rgc = red_grid4(s.nc);
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
    s.dptr = (float2**)h->solver_meta;
    s.mpart = (double*)(s.dptr + 6 * GCR_MAXK);
    s.mcount = (unsigned*)(s.mpart + 2 * GCR_MAXK * MDOT_BLOCKS);
    if (!h->solver_meta_ready) {
        float2* hp[6 * GCR_MAXK] = {};
        for (int k = 0; k < GCR_MAXK; ++k) {
            hp[0 * GCR_MAXK + k] = k < h->prm.gcr_restart ? s.Z[k] : nullptr;
            hp[1 * GCR_MAXK + k] = k < h->prm.gcr_restart ? s.W[k] : nullptr;
            hp[2 * GCR_MAXK + k] = k < h->prm.post_smooth ? s.Ps[k] : nullptr;
            hp[3 * GCR_MAXK + k] = k < h->prm.post_smooth ? s.Qs[k] : nullptr;
            hp[4 * GCR_MAXK + k] = k < h->prm.coarse_restart ? s.Zc[k] : nullptr;
            hp[5 * GCR_MAXK + k] = k < h->prm.coarse_restart ? s.Wc[k] : nullptr;
        }
        cudaMemcpy(s.dptr, hp, sizeof(hp), cudaMemcpyHostToDevice);
        h->solver_meta_ready = true;
    }
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
// Orthogonalise (z, w) = (Zb[k], Wb[k]) against the first k pairs of the basis
// by classical Gram-Schmidt applied twice, then nrm[k] = |w|^2 and
// alpha = <w, r> / |w|^2.  dZ / dW: device copies of the pointer arrays.
static dwf_status gcr_orthogonalise(Solver& s, GcrScal* g, float2** Zb, float2** Wb, int k, const float2* r, long long n,
                                    float2* const* dZ, float2* const* dW, const int* skip = nullptr) {
    RedScratch rs = s.h->ws.red();
    const int rg = red_grid4(n);
    if (k > 0) {
        dim3 mgrid((unsigned)(rg < MDOT_BLOCKS ? rg : MDOT_BLOCKS), (unsigned)k);
        const long long n2 = (n + 1) / 2;
        const int eg = (int)((n2 + RED_THREADS - 1) / RED_THREADS < 152LL * 16 ? (n2 + RED_THREADS - 1) / RED_THREADS
                                                                               : 152LL * 16);
        const int passes = s.h->prm.cgs_passes;
        for (int pass = 0; pass < passes; ++pass) {
            k_mdot<<<mgrid, RED_THREADS, 0, s.st>>>(dW, Wb[k], n, s.mpart, s.mcount, g->coef, g->nrm, 0, skip);
            if (pass + 1 < passes)
                k_maxpy<false><<<eg, RED_THREADS, 0, s.st>>>(Wb[k], Zb[k], dW, dZ, g->coef, k, r, n, rs, nullptr,
                                                             nullptr, skip);
            else
                k_maxpy<true><<<rg, RED_THREADS, 0, s.st>>>(Wb[k], Zb[k], dW, dZ, g->coef, k, r, n, rs, &g->nrm[k],
                                                            g->alpha, skip);
        }
    } else {
        k_maxpy<true><<<rg, RED_THREADS, 0, s.st>>>(Wb[0], Zb[0], dW, dZ, g->coef, 0, r, n, rs, &g->nrm[0], g->alpha,
                                                    skip);
    }
    DWF_CHECK_LAUNCH();
    return DWF_OK;
}

// Coarse solve with restarted GCR on B e = r_c, B = Dhat_PV^dag Dhat_DW (the
// paper's level-2 operator and solver type; B's spectrum lies in the right
// half plane, App. B).  One restart cycle is a fixed launch sequence whose
// kernels skip their work once the device-side stop flag is set; it is
// captured once per handle as a CUDA graph (plus a variant that starts with
// the prologue), and the host reads the flag once per cycle.
static dwf_status coarse_gcr_prologue(Solver& s) {
    const long long n = s.nc;
    DWF_CHECK_CUDA(cudaMemsetAsync(s.ec, 0, n * sizeof(float2), s.st));
    DWF_CHECK_CUDA(cudaMemcpyAsync(s.crr, s.rc, n * sizeof(float2), cudaMemcpyDeviceToDevice, s.st));
    DWF_CHECK_CUDA(cudaMemsetAsync(&s.d->cdone, 0, 2 * sizeof(int), s.st));
    DWF_TRY(dot_device(s.rc, s.rc, n, false, s.h->ws.red(), s.d->misc + 4, s.st));
    DWF_CHECK_CUDA(cudaMemcpyAsync(&s.d->cref2, s.d->misc + 4, sizeof(double), cudaMemcpyDeviceToDevice, s.st));
    return DWF_OK;
}

static dwf_status coarse_gcr_cycle(Solver& s) {
    dwf_mg* h = s.h;
    const long long n = s.nc;
    RedScratch rs = h->ws.red();
    GcrScal* g = &s.d->cgcr;
    int* done = &s.d->cdone;
    const int K = h->prm.coarse_restart;
    const double tol2 = h->prm.coarse_tol * h->prm.coarse_tol;
    for (int k = 0; k < K; ++k) {
        DWF_CHECK_CUDA(cudaMemcpyAsync(s.Zc[k], s.crr, n * sizeof(float2), cudaMemcpyDeviceToDevice, s.st));
        DWF_TRY(coarse_dwf_apply(h, s.Zc[k], s.ct, h->mf, false, done, s.st));
        DWF_TRY(coarse_dwf_apply(h, s.ct, s.Wc[k], 1.0, true, done, s.st));
        DWF_TRY(gcr_orthogonalise(s, g, s.Zc, s.Wc, k, s.crr, n, s.dptr + 4 * GCR_MAXK, s.dptr + 5 * GCR_MAXK, done));
        k_gcr_update<<<s.rgc, RED_THREADS, 0, s.st>>>(s.ec, s.crr, s.Zc[k], s.Wc[k], g->alpha, n, rs, &g->rr2, done,
                                                      &s.d->cref2, tol2, &s.d->citers, h->prm.coarse_maxiter);
        DWF_CHECK_LAUNCH();
    }
    return DWF_OK;
}

// Records the launch sequence on the handle's private capture stream (the
// caller's stream may be the legacy default stream, which cannot capture);
// the instantiated graph is launched on the caller's stream.
static dwf_status capture(Solver& s, bool with_prologue, cudaGraphExec_t* out) {
    cudaGraph_t graph = nullptr;
    if (!s.h->cap_stream) DWF_CHECK_CUDA(cudaStreamCreateWithFlags(&s.h->cap_stream, cudaStreamNonBlocking));
    const cudaStream_t user = s.st;
    s.st = s.h->cap_stream;
    DWF_CHECK_CUDA(cudaStreamBeginCapture(s.st, cudaStreamCaptureModeThreadLocal));
    dwf_status st = DWF_OK;
    if (with_prologue) st = coarse_gcr_prologue(s);
    if (st == DWF_OK) st = coarse_gcr_cycle(s);
    cudaError_t e = cudaStreamEndCapture(s.st, &graph);
    s.st = user;
    if (st != DWF_OK) { if (graph) cudaGraphDestroy(graph); return st; }
    if (e != cudaSuccess) { set_error("graph capture: %s", cudaGetErrorString(e)); return DWF_ERR_CUDA; }
    e = cudaGraphInstantiate(out, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) { set_error("graph instantiation: %s", cudaGetErrorString(e)); return DWF_ERR_CUDA; }
    return DWF_OK;
}

static dwf_status coarse_solve_gcr(Solver& s) {
    dwf_mg* h = s.h;
    const int K = h->prm.coarse_restart;
    const int maxit = h->prm.coarse_maxiter;
    if (!h->coarse_graph_first) {
        DWF_TRY(capture(s, true, &h->coarse_graph_first));
        DWF_TRY(capture(s, false, &h->coarse_graph_cycle));
    }
    int launched = 0;
    for (;;) {
        DWF_CHECK_CUDA(cudaGraphLaunch(launched == 0 ? h->coarse_graph_first : h->coarse_graph_cycle, s.st));
        launched += K;
        DWF_CHECK_CUDA(cudaMemcpyAsync(&s.hs->cdone, &s.d->cdone, 2 * sizeof(int), cudaMemcpyDeviceToHost, s.st));
        DWF_CHECK_CUDA(cudaStreamSynchronize(s.st));
        if (s.hs->cdone || launched >= maxit) break;
    }
    s.coarse_iters += s.hs->citers;
    s.coarse_applies += 2LL * s.hs->citers;
    s.coarse_solves += 1;
    return DWF_OK;
}

// Coarse solve: CGNR on B^dag B e = B^dag r, B = Dhat_PV^dag Dhat_DW.
static bool persistent_coarse(const dwf_mg* h) {
    if (!h->prm.coarse_persistent) return false;
    if (h->prm.coarse_solver == 1) return h->prm.coarse_persistent == 2 && coarse_gcr_persistent_ok(h);
    return h->mg.ncd == 16 && h->mg.Ls_c <= 4 && h->mg.nd == 2;
}

static dwf_status coarse_solve(Solver& s) {
    dwf_mg* h = s.h;
    if (h->prm.coarse_solver == 1 && persistent_coarse(h)) {
        // one cooperative launch per coarse solve; residual slots Zc[0..KC-1] and crr
        float2* S[GCR_MAXK + 1];
        const int KC = h->prm.coarse_restart;
        for (int k = 0; k < KC; ++k) S[k] = s.Zc[k];
        S[KC] = s.crr;
        DWF_TRY(coarse_gcr_persistent(h, s.rc, s.ec, S, s.Wc, s.ct, s.partials, s.d->bar, &s.d->pcg_iters,
                                      &s.d->pcg_rr2, s.st));
        s.coarse_solves += 1;
        return DWF_OK;
    }
    if (h->prm.coarse_solver == 1) return coarse_solve_gcr(s);
    if (persistent_coarse(h)) {
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
        DWF_TRY(gcr_orthogonalise(s, g, s.Ps, s.Qs, j, s.rs_, n, s.dptr + 2 * GCR_MAXK, s.dptr + 3 * GCR_MAXK));
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
    if ((h->prm.coarse_solver == 1 && h->prm.coarse_persistent != 2) || h->lvl3) {
        // the same K-cycle through the right-hand-side-batched implementation with one
        // column: its GCR updates only w and r per step and assembles the solution
        // once per cycle (fewer passes over the fine vectors)
        return mg_solve_batched_impl(h, 1, (const double2*)b, (double2*)x, tol, maxiter, stats);
    }
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
            DWF_TRY(gcr_orthogonalise(s, g, s.Z, s.W, k, s.r, n, s.dptr + 0 * GCR_MAXK, s.dptr + 1 * GCR_MAXK));
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
    if (persistent_coarse(h)) {
        DWF_CHECK_CUDA(cudaMemcpyAsync(&s.hs->pcg_iters, &s.d->pcg_iters, sizeof(int), cudaMemcpyDeviceToHost, s.st));
        DWF_CHECK_CUDA(cudaMemcpyAsync(s.hs->bar, s.d->bar, sizeof(s.d->bar), cudaMemcpyDeviceToHost, s.st));
        DWF_CHECK_CUDA(cudaStreamSynchronize(s.st));
        s.coarse_iters = s.hs->pcg_iters;
        s.coarse_applies = h->prm.coarse_solver == 1 ? 2LL * s.coarse_iters + s.coarse_solves
                                                     : 2 * s.coarse_solves + 4LL * s.coarse_iters;
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
