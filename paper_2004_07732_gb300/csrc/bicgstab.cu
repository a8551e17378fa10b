// BiCGStab(l) (Sleijpen & Fokkema 1993) on the Pauli-Villars preconditioned
// system D_PV^dag D_DW x = D_PV^dag b: the direct Krylov solver the paper sets
// beside CGNR and multigrid (Sec. 2.3, Sec. 3, Fig. iterationscompare; valid
// because spec(D_PV^dag D_DW) lies in the right half plane, App. B).
//
// Precision: FP64 reliable updates of the true residual r = b - D_DW x around
// inner BiCGStab(l) solves of A e = D_PV^dag r / |r| in the inner precision
// (FP32 spinors with FP32 / FP16 / BF16 links, or all FP64).  Each inner solve
// runs until its recursive residual has fallen by `delta`, then x += |r| e and
// r is recomputed in FP64.
//
// One cycle = l BiCG steps (each: rho = <rt, r_j>, u_i = r_i - beta u_i,
// u_{j+1} = A u_j, alpha = rho / <rt, u_{j+1}>, r_i -= alpha u_{i+1},
// r_{j+1} = A r_j, x += alpha u_0) and the minimal-residual step (Gram-Schmidt
// of r_1..r_l, then r_0 -= sum gamma'_j r_j, u_0 -= sum gamma_j u_j,
// x += gamma_1 r_0 + sum gamma''_j r_j).  Every Krylov scalar is computed and
// kept on the device (complex FP64); the host reads |r_0|^2 once per cycle.
// The Gram-Schmidt step is classical (all projections of r_j from one pass)
// where the oracle uses the modified form: the two agree in exact arithmetic.
#include <chrono>
#include <string.h>

#include "common.cuh"
#include "fine_kernels.cuh"
#include "blas.cuh"

namespace dwf {
namespace {

constexpr int BS_MAX_L = 8;
constexpr int BS_RED_ROWS = 2 * BS_MAX_L + 2;   // quantities of one reduction kernel

struct BsScal {
    double2 rho0, alpha, omega, beta;
    double2 tau[BS_MAX_L + 1][BS_MAX_L + 1];
    double2 gp[BS_MAX_L + 1], g[BS_MAX_L + 1], g2[BS_MAX_L + 1];
    double sigma[BS_MAX_L + 1];
    double rr2;          // |r_0|^2 after the last cycle
    double f2;           // |f|^2 of the inner right-hand side
    int breakdown;
};

__device__ __forceinline__ double2 zmul(double2 a, double2 b) { return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
__device__ __forceinline__ double2 zdiv(double2 a, double2 b) {
    const double d = b.x * b.x + b.y * b.y;
    return make_double2((a.x * b.x + a.y * b.y) / d, (a.y * b.x - a.x * b.y) / d);
}
__device__ __forceinline__ double2 zsub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 zadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }

// Vector element and real types of a precision.
template <class C> struct Real;
template <> struct Real<float2> { using T = float; };
template <> struct Real<double2> { using T = double; };

template <class C> __device__ __forceinline__ C cpx(double2 z) { C c; c.x = (decltype(c.x))z.x; c.y = (decltype(c.y))z.y; return c; }

// a - z b, a + z b
template <class C> __device__ __forceinline__ C caxmy(C a, C z, C b) {
    a.x -= z.x * b.x - z.y * b.y; a.y -= z.x * b.y + z.y * b.x; return a;
}
template <class C> __device__ __forceinline__ C caxpy(C a, C z, C b) {
    a.x += z.x * b.x - z.y * b.y; a.y += z.x * b.y + z.y * b.x; return a;
}

// Per-thread partial sums: FP32 data accumulates a few products per thread in
// FP32 (FP64 across threads), FP64 data accumulates in FP64.
template <class C> struct Acc { using T = typename Real<C>::T; };

struct VecSet {                 // device pointers of up to BS_MAX_L + 1 vectors
    void* p[BS_MAX_L + 1];
};

#define BS_LOOP(i) for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)

// rho1 = <rt, r_j>; beta = alpha rho1 / rho0; rho0 = rho1
template <class C>
__global__ void __launch_bounds__(RED_THREADS) k_bs_rho(const C* __restrict__ rt, const C* __restrict__ rj, long long n,
                                                        RedScratch rs, BsScal* S) {
    using A = typename Acc<C>::T;
    A re = 0, im = 0;
    BS_LOOP(i) {
        const C a = rt[i], b = rj[i];
        re += a.x * b.x + a.y * b.y;
        im += a.x * b.y - a.y * b.x;
    }
    const A v[2] = {re, im};
    grid_reduce_any<2>(v, rs, [=] __device__(double* t) {
        const double2 rho1 = make_double2(t[0], t[1]);
        if (S->rho0.x == 0.0 && S->rho0.y == 0.0) { S->breakdown = 1; S->beta = make_double2(0.0, 0.0); }
        else S->beta = zdiv(zmul(S->alpha, rho1), S->rho0);
        S->rho0 = rho1;
    });
}

// u_i = r_i - beta u_i, i = 0..j
template <class C>
__global__ void k_bs_upd_u(VecSet R, VecSet U, int j, long long n, const BsScal* S) {
    const C beta = cpx<C>(S->beta);
    BS_LOOP(e) {
        for (int i = 0; i <= j; ++i) {
            C* u = (C*)U.p[i];
            const C r = ((const C*)R.p[i])[e];
            u[e] = caxmy(r, beta, u[e]);
        }
    }
}

// alpha = rho0 / <rt, u_{j+1}>
template <class C>
__global__ void __launch_bounds__(RED_THREADS) k_bs_alpha(const C* __restrict__ rt, const C* __restrict__ u, long long n,
                                                          RedScratch rs, BsScal* S) {
    using A = typename Acc<C>::T;
    A re = 0, im = 0;
    BS_LOOP(i) {
        const C a = rt[i], b = u[i];
        re += a.x * b.x + a.y * b.y;
        im += a.x * b.y - a.y * b.x;
    }
    const A v[2] = {re, im};
    grid_reduce_any<2>(v, rs, [=] __device__(double* t) {
        const double2 gam = make_double2(t[0], t[1]);
        if (gam.x == 0.0 && gam.y == 0.0) { S->breakdown = 1; S->alpha = make_double2(0.0, 0.0); }
        else S->alpha = zdiv(S->rho0, gam);
    });
}

// r_i -= alpha u_{i+1}, i = 0..j; x += alpha u_0
template <class C>
__global__ void k_bs_upd_r(VecSet R, VecSet U, C* __restrict__ x, int j, long long n, const BsScal* S) {
    const C alpha = cpx<C>(S->alpha);
    BS_LOOP(e) {
        for (int i = 0; i <= j; ++i) {
            C* r = (C*)R.p[i];
            r[e] = caxmy(r[e], alpha, ((const C*)U.p[i + 1])[e]);
        }
        x[e] = caxpy(x[e], alpha, ((const C*)U.p[0])[e]);
    }
}

// tau_ij = <r_i, r_j> / sigma_i for i = 1..j-1 (one pass over r_j)
template <class C, int JM>
__global__ void __launch_bounds__(RED_THREADS) k_bs_proj(VecSet R, int j, long long n, RedScratch rs, BsScal* S) {
    using A = typename Acc<C>::T;
    A re[JM], im[JM];
#pragma unroll
    for (int i = 0; i < JM; ++i) { re[i] = 0; im[i] = 0; }
    const C* rj = (const C*)R.p[j];
    BS_LOOP(e) {
        const C b = rj[e];
#pragma unroll
        for (int i = 0; i < JM; ++i)
            if (i + 1 < j) {
                const C a = ((const C*)R.p[i + 1])[e];
                re[i] += a.x * b.x + a.y * b.y;
                im[i] += a.x * b.y - a.y * b.x;
            }
    }
    A v[2 * JM];
#pragma unroll
    for (int i = 0; i < JM; ++i) { v[2 * i] = re[i]; v[2 * i + 1] = im[i]; }
    grid_reduce_any<2 * JM>(v, rs, [=] __device__(double* t) {
        for (int i = 1; i < j; ++i) {
            const double s = S->sigma[i];
            S->tau[i][j] = s > 0.0 ? make_double2(t[2 * (i - 1)] / s, t[2 * (i - 1) + 1] / s) : make_double2(0.0, 0.0);
        }
    });
}

// r_j -= sum_{i<j} tau_ij r_i; sigma_j = |r_j|^2; gamma'_j = <r_j, r_0> / sigma_j
template <class C>
__global__ void __launch_bounds__(RED_THREADS) k_bs_gs(VecSet R, int j, long long n, RedScratch rs, BsScal* S) {
    using A = typename Acc<C>::T;
    __shared__ C tau[BS_MAX_L + 1];
    if (threadIdx.x <= BS_MAX_L) tau[threadIdx.x] = threadIdx.x >= 1 && (int)threadIdx.x < j ? cpx<C>(S->tau[threadIdx.x][j]) : C{};
    __syncthreads();
    C* rj = (C*)R.p[j];
    const C* r0 = (const C*)R.p[0];
    A s2 = 0, gr = 0, gi = 0;
    BS_LOOP(e) {
        C b = rj[e];
        for (int i = 1; i < j; ++i) b = caxmy(b, tau[i], ((const C*)R.p[i])[e]);
        rj[e] = b;
        const C a = r0[e];
        s2 += b.x * b.x + b.y * b.y;
        gr += b.x * a.x + b.y * a.y;
        gi += b.x * a.y - b.y * a.x;
    }
    const A v[3] = {s2, gr, gi};
    grid_reduce_any<3>(v, rs, [=] __device__(double* t) {
        S->sigma[j] = t[0];
        if (t[0] > 0.0) S->gp[j] = make_double2(t[1] / t[0], t[2] / t[0]);
        else { S->gp[j] = make_double2(0.0, 0.0); S->breakdown = 1; }
    });
}

// gamma by back substitution, gamma'' and omega (one thread)
__global__ void k_bs_coef(int l, BsScal* S) {
    S->g[l] = S->gp[l];
    S->omega = S->g[l];
    for (int j = l - 1; j >= 1; --j) {
        double2 a = S->gp[j];
        for (int i = j + 1; i <= l; ++i) a = zsub(a, zmul(S->tau[j][i], S->g[i]));
        S->g[j] = a;
    }
    for (int j = 1; j < l; ++j) {
        double2 a = S->g[j + 1];
        for (int i = j + 1; i < l; ++i) a = zadd(a, zmul(S->tau[j][i], S->g[i + 1]));
        S->g2[j] = a;
    }
    // the next cycle's rho0 = -omega rho0
    S->rho0 = make_double2(-(S->omega.x * S->rho0.x - S->omega.y * S->rho0.y),
                           -(S->omega.x * S->rho0.y + S->omega.y * S->rho0.x));
}

// x += gamma_1 r_0 + sum_{j<l} gamma''_j r_j; r_0 -= sum_{j<=l} gamma'_j r_j; u_0 -= sum_{j<=l} gamma_j u_j;
// rr2 = |r_0|^2
template <class C>
__global__ void __launch_bounds__(RED_THREADS) k_bs_mr(VecSet R, VecSet U, C* __restrict__ x, int l, long long n,
                                                       RedScratch rs, BsScal* S) {
    using A = typename Acc<C>::T;
    __shared__ C gp[BS_MAX_L + 1], g[BS_MAX_L + 1], g2[BS_MAX_L + 1];
    if (threadIdx.x <= BS_MAX_L) {
        const int j = threadIdx.x;
        gp[j] = j <= l ? cpx<C>(S->gp[j]) : C{};
        g[j] = j <= l ? cpx<C>(S->g[j]) : C{};
        g2[j] = j < l ? cpx<C>(S->g2[j]) : C{};
    }
    __syncthreads();
    C* r0 = (C*)R.p[0];
    C* u0 = (C*)U.p[0];
    A acc = 0;
    BS_LOOP(e) {
        C r = r0[e], u = u0[e], xx = x[e];
        xx = caxpy(xx, g[1], r);
        for (int j = 1; j <= l; ++j) {
            const C rj = ((const C*)R.p[j])[e];
            r = caxmy(r, gp[j], rj);
            u = caxmy(u, g[j], ((const C*)U.p[j])[e]);
            if (j < l) xx = caxpy(xx, g2[j], rj);
        }
        r0[e] = r; u0[e] = u; x[e] = xx;
        acc += r.x * r.x + r.y * r.y;
    }
    const A v[1] = {acc};
    grid_reduce_any<1>(v, rs, [=] __device__(double* t) { S->rr2 = t[0]; });
}

// inner start: r_0 = rt = f (copied by the host), u_0 = 0, x = 0; scalars rho0 = alpha = omega = 1
__global__ void k_bs_init(BsScal* S, double f2) {
    S->rho0 = make_double2(1.0, 0.0);
    S->alpha = make_double2(0.0, 0.0);
    S->omega = make_double2(1.0, 0.0);
    S->beta = make_double2(0.0, 0.0);
    S->rr2 = f2;
    S->f2 = f2;
    S->breakdown = 0;
}

// FP64 helpers of the reliable updates
__global__ void __launch_bounds__(RED_THREADS) k_bs_norm64(const double2* __restrict__ a, long long n, RedScratch rs,
                                                           double* out) {
    double v[1] = {0.0};
    BS_LOOP(i) { const double2 z = a[i]; v[0] += z.x * z.x + z.y * z.y; }
    grid_reduce<1>(v, rs, [=] __device__(double* t) { *out = t[0]; });
}

template <class C>
__global__ void __launch_bounds__(RED_THREADS) k_bs_norm(const C* __restrict__ a, long long n, RedScratch rs, double* out) {
    using A = typename Acc<C>::T;
    A acc = 0;
    BS_LOOP(i) { const C z = a[i]; acc += z.x * z.x + z.y * z.y; }
    const A v[1] = {acc};
    grid_reduce_any<1>(v, rs, [=] __device__(double* t) { *out = t[0]; });
}

template <class C>
__global__ void k_bs_scale_in(C* __restrict__ out, const double2* __restrict__ a, double s, long long n) {
    BS_LOOP(i) { const double2 z = a[i]; out[i] = cpx<C>(make_double2(z.x * s, z.y * s)); }
}

// X += s e
template <class C>
__global__ void k_bs_accum(double2* __restrict__ X, const C* __restrict__ e, double s, long long n) {
    BS_LOOP(i) { const C z = e[i]; double2 x = X[i]; x.x += s * (double)z.x; x.y += s * (double)z.y; X[i] = x; }
}

__global__ void k_bs_sub64(double2* __restrict__ r, const double2* __restrict__ b, const double2* __restrict__ t, long long n) {
    BS_LOOP(i) { const double2 u = b[i], v = t[i]; r[i] = make_double2(u.x - v.x, u.y - v.y); }
}

static int bs_grid(long long n) {
    long long b = (n + 255) / 256;
    return (int)(b < 152LL * 8 ? b : 152LL * 8);
}

struct BsCtx {
    Geom G;
    const void* Ulo;
    int prec;
    double M5, mf;
    cudaStream_t st;
    long long n;
    RedScratch rs;
    BsScal* S;
    void* tmp;          // D_DW v of the preconditioned apply
    long long applies = 0;
};

// out = D_PV^dag D_DW in
static dwf_status bs_apply_A(BsCtx& c, const void* in, void* out) {
    DWF_TRY(fine_apply(c.G, c.Ulo, in, c.tmp, c.M5, c.mf, false, c.prec, c.st));
    DWF_TRY(fine_apply(c.G, c.Ulo, c.tmp, out, c.M5, 1.0, true, c.prec, c.st));
    c.applies += 2;
    return DWF_OK;
}

template <class C>
static void launch_proj(VecSet R, int j, long long n, RedScratch rs, BsScal* S, cudaStream_t st) {
    const int g = red_grid4(n);
    if (j <= 3) k_bs_proj<C, 2><<<g, RED_THREADS, 0, st>>>(R, j, n, rs, S);
    else if (j <= 5) k_bs_proj<C, 4><<<g, RED_THREADS, 0, st>>>(R, j, n, rs, S);
    else k_bs_proj<C, 7><<<g, RED_THREADS, 0, st>>>(R, j, n, rs, S);
}

// One cycle (l BiCG steps and the minimal-residual step) on the inner vectors.
template <class C>
static dwf_status bs_cycle(BsCtx& c, int l, VecSet R, VecSet U, const C* rt, C* x) {
    const long long n = c.n;
    const int rg = red_grid4(n), eg = bs_grid(n);
    for (int j = 0; j < l; ++j) {
        k_bs_rho<C><<<rg, RED_THREADS, 0, c.st>>>(rt, (const C*)R.p[j], n, c.rs, c.S);
        k_bs_upd_u<C><<<eg, 256, 0, c.st>>>(R, U, j, n, c.S);
        DWF_CHECK_LAUNCH();
        DWF_TRY(bs_apply_A(c, U.p[j], U.p[j + 1]));
        k_bs_alpha<C><<<rg, RED_THREADS, 0, c.st>>>(rt, (const C*)U.p[j + 1], n, c.rs, c.S);
        k_bs_upd_r<C><<<eg, 256, 0, c.st>>>(R, U, x, j, n, c.S);
        DWF_CHECK_LAUNCH();
        DWF_TRY(bs_apply_A(c, R.p[j], R.p[j + 1]));
    }
    for (int j = 1; j <= l; ++j) {
        if (j > 1) launch_proj<C>(R, j, n, c.rs, c.S, c.st);
        k_bs_gs<C><<<rg, RED_THREADS, 0, c.st>>>(R, j, n, c.rs, c.S);
    }
    k_bs_coef<<<1, 1, 0, c.st>>>(l, c.S);
    k_bs_mr<C><<<rg, RED_THREADS, 0, c.st>>>(R, U, x, l, n, c.rs, c.S);
    DWF_CHECK_LAUNCH();
    return DWF_OK;
}

template <class C>
static dwf_status bs_solve(BsCtx& c, const void* U64, const double2* B, double2* X, int l, double tol, int maxiter,
                           double inner_tol, dwf_solve_stats* stats, std::chrono::steady_clock::time_point t0) {
    const long long n = c.n;
    const size_t vb = (size_t)n * sizeof(C), vb64 = (size_t)n * sizeof(double2);
    // inner vectors: R[0..l], U[0..l], rt, x, tmp; FP64: r64, t64; reduction rows and scalars
    const size_t nvec = 2 * (size_t)(l + 1) + 3;
    const size_t red_bytes = sizeof(double) * BS_RED_ROWS * RED_BLOCKS;
    const size_t cnt_bytes = sizeof(unsigned) * (RED_GROUPS + 1) * RED_CSTRIDE;
    const size_t total = nvec * vb + 2 * vb64 + red_bytes + cnt_bytes + sizeof(BsScal) + 4096;
    void* buf = nullptr;
    {
        cudaError_t e = cudaMallocAsync(&buf, total, c.st);
        if (e != cudaSuccess) { set_error("BiCGStab work vectors (%zu bytes): %s", total, cudaGetErrorString(e)); return DWF_ERR_OOM; }
    }
    struct Free { void* p; cudaStream_t s; ~Free() { cudaFreeAsync(p, s); } } fr{buf, c.st};
    char* q = (char*)buf;
    auto take = [&](size_t bytes) { char* p = q; q += (bytes + 255) & ~(size_t)255; return p; };
    VecSet R, U;
    for (int i = 0; i <= BS_MAX_L; ++i) { R.p[i] = nullptr; U.p[i] = nullptr; }
    for (int i = 0; i <= l; ++i) { R.p[i] = take(vb); U.p[i] = take(vb); }
    C* rt = (C*)take(vb);
    C* xe = (C*)take(vb);
    c.tmp = take(vb);
    double2* r64 = (double2*)take(vb64);
    double2* t64 = (double2*)take(vb64);
    c.rs.partials = (double*)take(red_bytes);
    c.rs.counter = (unsigned*)take(cnt_bytes);
    c.S = (BsScal*)take(sizeof(BsScal));
    double* dnorm = (double*)take(64);
    DWF_CHECK_CUDA(cudaMemsetAsync(c.rs.counter, 0, cnt_bytes, c.st));
    BsScal* hS = nullptr;
    DWF_CHECK_CUDA(cudaMallocHost(&hS, sizeof(BsScal)));
    struct FreeH { void* p; ~FreeH() { cudaFreeHost(p); } } frh{hS};
    double* hnorm = &hS->f2;     // host staging of one double (reuses a field of the pinned copy)

    const int rg64 = red_grid(n), eg = bs_grid(n);
    auto norm64 = [&](const double2* v, double* out) -> dwf_status {
        k_bs_norm64<<<rg64, RED_THREADS, 0, c.st>>>(v, n, c.rs, dnorm);
        DWF_CHECK_LAUNCH();
        DWF_CHECK_CUDA(cudaMemcpyAsync(hnorm, dnorm, sizeof(double), cudaMemcpyDeviceToHost, c.st));
        DWF_CHECK_CUDA(cudaStreamSynchronize(c.st));
        *out = *hnorm;
        return DWF_OK;
    };

    DWF_CHECK_CUDA(cudaMemsetAsync(X, 0, vb64, c.st));
    DWF_CHECK_CUDA(cudaMemcpyAsync(r64, B, vb64, cudaMemcpyDeviceToDevice, c.st));
    double bn2 = 0.0;
    DWF_TRY(norm64(B, &bn2));
    dwf_status status = DWF_ERR_NOCONV;
    double res = 1.0, rn2 = bn2;
    int steps = 0, restarts = 0, stalls = 0;
    double best = 1e300;
    if (bn2 == 0.0) { status = DWF_OK; res = 0.0; }
    while (status != DWF_OK) {
        res = sqrt(rn2 / bn2);
        if (res <= tol) { status = DWF_OK; break; }
        if (steps >= maxiter) break;
        // a reliable-update cycle that did not reduce the true residual twice in a row: give up
        if (res >= best) { if (++stalls >= 2) { set_error("BiCGStab(%d) stagnates at residual %.3e", l, res); break; } }
        else { stalls = 0; best = res; }
        ++restarts;
        const double rn = sqrt(rn2);
        // f = D_PV^dag r / |r| in the inner precision; r_0 = rt = f, u_0 = 0, x = 0
        k_bs_scale_in<C><<<eg, 256, 0, c.st>>>(xe, r64, 1.0 / rn, n);
        DWF_CHECK_LAUNCH();
        DWF_TRY(fine_apply(c.G, c.Ulo, xe, R.p[0], c.M5, 1.0, true, c.prec, c.st));
        c.applies += 1;
        DWF_CHECK_CUDA(cudaMemcpyAsync(rt, R.p[0], vb, cudaMemcpyDeviceToDevice, c.st));
        DWF_CHECK_CUDA(cudaMemsetAsync(U.p[0], 0, vb, c.st));
        DWF_CHECK_CUDA(cudaMemsetAsync(xe, 0, vb, c.st));
        k_bs_norm<C><<<red_grid4(n), RED_THREADS, 0, c.st>>>((const C*)R.p[0], n, c.rs, dnorm);
        DWF_CHECK_LAUNCH();
        DWF_CHECK_CUDA(cudaMemcpyAsync(hnorm, dnorm, sizeof(double), cudaMemcpyDeviceToHost, c.st));
        DWF_CHECK_CUDA(cudaStreamSynchronize(c.st));
        const double f2 = *hnorm;
        k_bs_init<<<1, 1, 0, c.st>>>(c.S, f2);
        DWF_CHECK_LAUNCH();
        double delta = inner_tol;
        const double need = 0.5 * tol * sqrt(bn2) / rn;
        if (need > delta) delta = need;
        for (;;) {
            DWF_TRY(bs_cycle<C>(c, l, R, U, rt, xe));
            steps += l;
            DWF_CHECK_CUDA(cudaMemcpyAsync(hS, c.S, sizeof(BsScal), cudaMemcpyDeviceToHost, c.st));
            DWF_CHECK_CUDA(cudaStreamSynchronize(c.st));
            if (hS->breakdown || !(hS->rr2 == hS->rr2)) break;   // restart from the true residual
            if (hS->rr2 <= delta * delta * f2 || steps >= maxiter) break;
        }
        // x += |r| e; r = b - D_DW x in FP64
        k_bs_accum<C><<<eg, 256, 0, c.st>>>(X, xe, rn, n);
        DWF_CHECK_LAUNCH();
        DWF_TRY(fine_apply(c.G, U64, X, t64, c.M5, c.mf, false, DWF_F64, c.st));
        c.applies += 1;
        k_bs_sub64<<<eg, 256, 0, c.st>>>(r64, B, t64, n);
        DWF_CHECK_LAUNCH();
        DWF_TRY(norm64(r64, &rn2));
    }
    res = bn2 > 0 ? sqrt(rn2 / bn2) : 0.0;
    if (status == DWF_ERR_NOCONV && dwf_last_error()[0] == 0)
        set_error("BiCGStab(%d) stopped after %d BiCG steps at true residual %.3e > tol %.3e", l, steps, res, tol);
    if (stats) {
        stats->iterations = steps;
        stats->restarts = restarts;
        stats->fine_applies = c.applies;
        stats->true_residual = res;
        stats->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
    return status;
}

}  // namespace
}  // namespace dwf

using namespace dwf;

extern "C" dwf_status bicgstab_solve(const dwf_geom* g, const void* U, const void* b, void* x, double M5, double mf,
                                     int ell, double tol, int maxiter, int inner_prec, dwf_solve_stats* stats,
                                     void* stream) {
    clear_error();
    auto t0 = std::chrono::steady_clock::now();
    if (stats) memset(stats, 0, sizeof(*stats));
    Geom G;
    DWF_TRY(check_geom(g, &G));
    const long long n = spinor_len(G);
    if (n == 0) return DWF_OK;
    if (!U || !b || !x) { set_error("NULL device pointer"); return DWF_ERR_ARG; }
    if (!aligned16(b) || !aligned16(x)) { set_error("b and x must be 16-byte aligned"); return DWF_ERR_ARG; }
    if (b == x) { set_error("b and x must be distinct buffers"); return DWF_ERR_ARG; }
    if (ell < 1 || ell > BS_MAX_L) { set_error("ell must be in [1, %d]", BS_MAX_L); return DWF_ERR_ARG; }
    if (!(tol > 0.0)) { set_error("tol must be > 0"); return DWF_ERR_ARG; }
    if (maxiter < 0) { set_error("maxiter must be >= 0"); return DWF_ERR_ARG; }
    if (!valid_prec(inner_prec)) { set_error("bad inner precision %d", inner_prec); return DWF_ERR_ARG; }
    cudaStream_t st = as_stream(stream);
    BsCtx c;
    c.G = G;
    c.prec = inner_prec;
    c.M5 = M5;
    c.mf = mf;
    c.st = st;
    c.n = n;
    void* Ulo = nullptr;
    struct Free { void* p; cudaStream_t s; ~Free() { if (p) cudaFreeAsync(p, s); } } fr{nullptr, st};
    if (inner_prec == DWF_F64) {
        c.Ulo = U;
    } else {
        const size_t lb = inner_prec == DWF_F32 ? 8 : 4;
        cudaError_t e = cudaMallocAsync(&Ulo, (size_t)link_len(G) * lb, st);
        if (e != cudaSuccess) { set_error("inner links: %s", cudaGetErrorString(e)); return DWF_ERR_OOM; }
        fr.p = Ulo;
        DWF_TRY(dwf_convert_links(g, U, Ulo, inner_prec, st));
        c.Ulo = Ulo;
    }
    const double inner_tol = inner_prec == DWF_F64 ? 1e-12 : 1e-4;
    if (inner_prec == DWF_F64)
        return bs_solve<double2>(c, U, (const double2*)b, (double2*)x, ell, tol, maxiter, inner_tol, stats, t0);
    return bs_solve<float2>(c, U, (const double2*)b, (double2*)x, ell, tol, maxiter, inner_tol, stats, t0);
}
