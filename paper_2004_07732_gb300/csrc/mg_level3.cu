// The third multigrid level and the deflation of the coarsest level.
//
// Table kcycle of the paper runs three levels: on every level l > 1 the setup
// is repeated on the Galerkin kernel of the level above (12 near-null vectors,
// 2^2 aggregates), the intermediate level is solved by GCR on
// Dhat_PV^dag Dhat_DW to a relative residual of 0.25 (at most 16 steps, 8
// post-smoothing steps), and the coarsest level by CGNR on the normal operator
// of Dhat2_PV^dag Dhat2_DW to 0.05 (at most 1024 iterations).  Table
// zerospacing adds a deflation of 128 low modes on the coarsest level.
//
// Setup (FP64 unless noted), given the two-level handle:
//   1. near-null vectors of the coarse kernel: CG on S S^dag v = 0 with
//      S = Dhat_W(m_s) = Dhat_W(-M5) + (m_s + M5) 1 (P^dag P = 1 lets the
//      Wilson mass pass through the Galerkin product), from caller starts;
//   2. chiral doubling by sigma_3 and Gram-Schmidt per aggregate of coarse
//      sites: the prolongator P2 with sigma_3 P2 = P2 sigma_3;
//   3. the level-3 Galerkin kernel Dhat2_W = P2^dag Dhat_W P2, one block per
//      level-3 site and hop direction (FP32 column-major copy for the stencil);
//   4. deflation: Lanczos with full reorthogonalisation on the level-3 normal
//      operator N3 = A3^dag A3 (A3 = Dhat2_PV^dag Dhat2_DW) from a caller start;
//      the lowest n_deflate eigenvalues of the Lanczos matrix T by bisection and
//      their vectors by inverse iteration, orthonormalised; the deflation basis
//      V = Q S and the Cholesky factor of H = V^dag N3 V = S^dag T S.
//
// Solve, one right-hand side, FP32 vectors with FP64 Krylov scalars:
//   level 2: flexible GCR on Ahat e = r, preconditioned by z = M2(r):
//     restrict the wall to level 3 (Eq. TruncProjectInterpolate), level-3 solve,
//     prolong, post_smooth GCR steps on Ahat from the prolonged correction;
//   level 3: CGNR on A3^dag A3 e = A3^dag r from the deflated start
//     x0 = V H^-1 V^dag A3^dag r (the exact Galerkin solution of the normal
//     equations on span V), under a CUDA graph of 8 iterations with a device
//     stop flag.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <new>
#include <string.h>
#include <string>
#include <vector>

#include "mg.cuh"

namespace dwf {
namespace {

constexpr int L2_MAXK = 32;          // bound on the level-2 GCR and smoother lengths
constexpr int L3_GRAPH_ITERS = 8;    // CGNR iterations per graph launch
constexpr int DEFL_MAX = 256;        // bound on the deflation space
constexpr int LANCZOS_MAX = 2048;

struct GScal {                       // Krylov scalars of one GCR (level 2, its smoother, level 3)
    double c[L2_MAXK][2];
    double alpha[2];
    double inv;
    double rr2, ref2;
    int done, steps, maxit, pad;
};

struct Cg3 {                         // coarsest CGNR
    double rn2, rr2, bn2, alpha, beta, tol2;
    int done, iters, maxit, pad;
};

struct Level3 {
    // geometry: level 2 = the handle's coarse lattice, level 3 its aggregation
    int L2[4], b2[4], L3[4];
    long long V2, V3;
    int nb2, nvec1, ncd2, nvec2, ncd3, Ls2, Ls3;
    long long n2, n3;                // complex values of a level-2 / level-3 vector
    dwf_mg_level_params prm;
    CoarseParams p3;                 // level-3 stencil (mf set per call)
    std::vector<void*> allocs;
    double2 *nullv2, *P2_64, *Y3_64;
    float2 *P2_32, *Y3_32;           // Y3_32: the stencil's FP32 blocks (block_prec DWF_F32)
    __half2* Y3_16;                  // the stencil's FP16 blocks (block_prec DWF_F32_L16), else nullptr
    // deflation
    int ndefl;                       // columns of V in use
    float2* Vd;                      // [ndefl][n3]
    double2* Hl;                     // Cholesky factor of H, lower, [ndefl][ndefl]
    std::vector<double> ritz;        // Rayleigh quotients of the deflation vectors (ascending)
    double filter_cut = 0.0, filter_top = 0.0;   // the Chebyshev filter's interval [a, b]
    int filter_passes = 0;
    // level-2 solver vectors
    float2 *r2, *e2, *rs, *es, *t2, *a2;
    float2 *Z[L2_MAXK], *W[L2_MAXK], *Zs[L2_MAXK], *Ws[L2_MAXK];
    // level-3 vectors
    float2 *b3, *x3, *rr3, *r3, *p3v, *q3, *w3, *t3;
    float2 *Z3[L2_MAXK], *W3[L2_MAXK];   // coarsest GCR basis
    double2* dc;                     // deflation coefficients [DEFL_MAX]
    GScal *g2, *gs, *g3;
    cudaGraphExec_t gcr3_graph = nullptr;
    Cg3* cg;
    double* red_part;                // reduction rows [L2_MAXK + 1][RED_MAX * RED_BLOCKS]
    unsigned* red_cnt;               // completion counters [L2_MAXK + 1][(RED_GROUPS + 1) * RED_CSTRIDE]
    int* status;                     // bulk-copy wait status of the per-site stencil
    void* hpin;                      // pinned host staging
    cudaGraphExec_t cg_graph;
    cudaStream_t cap_stream;
    int last_l2, last_l3;
};

constexpr int CROW3 = (RED_GROUPS + 1) * RED_CSTRIDE;
constexpr int PROW3 = RED_MAX * RED_BLOCKS;

__host__ __device__ inline RedScratch row_rs(double* part, unsigned* cnt, int r) {
    return RedScratch{part + (size_t)r * PROW3, cnt + (size_t)r * CROW3};
}

dwf_status l3_alloc(Level3* L, void** p, size_t bytes) {
    cudaError_t e = cudaMalloc(p, bytes < 256 ? 256 : bytes);
    if (e != cudaSuccess) {
        set_error("third-level allocation of %zu bytes failed: %s", bytes, cudaGetErrorString(e));
        *p = nullptr;
        return DWF_ERR_OOM;
    }
    L->allocs.push_back(*p);
    return DWF_OK;
}

// ---------------------------------------------------------------------------
// level-2 kernel Dhat_W(-M5) + shift (FP64, one slice) and its adjoint
// ---------------------------------------------------------------------------
__device__ __forceinline__ long long nbr_site(const int* L, int nd, long long x, int dir) {
    if (dir == 0) return x;
    const int mu = (dir - 1) >> 1;
    long long stride = 1;
    for (int nu = 0; nu < mu; ++nu) stride *= L[nu];
    const int c = (int)((x / stride) % L[mu]);
    const int cn = ((dir - 1) & 1) ? (c == 0 ? L[mu] - 1 : c - 1) : (c == L[mu] - 1 ? 0 : c + 1);
    return x + (long long)(cn - c) * stride;
}

struct Lat { int L[4]; int nd; };

// out[x][i] = sum_dir sum_j B_dir(x)[i][j] in[nb][j] + shift in[x][i], B = Y (row-major, dagger = 0)
// or the adjoint blocks Y(nb, opp)^dag (dagger = 1)
__global__ void k_kernel64(const double2* __restrict__ Y, const double2* __restrict__ in, double2* __restrict__ out,
                           Lat lat, long long V, int ncd, double shift, int dagger) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= V * ncd) return;
    const long long x = t / ncd;
    const int i = (int)(t % ncd);
    const int ndir = 2 * lat.nd + 1;
    const long long bsz = (long long)ncd * ncd;
    double2 acc = in[t];
    acc.x *= shift; acc.y *= shift;
    for (int dir = 0; dir < ndir; ++dir) {
        const long long nb = nbr_site(lat.L, lat.nd, x, dir);
        const double2* v = in + nb * ncd;
        if (!dagger) {
            const double2* y = Y + (x * ndir + dir) * bsz + (long long)i * ncd;
            for (int j = 0; j < ncd; ++j) {
                const double2 a = y[j], b = v[j];
                acc.x += a.x * b.x - a.y * b.y;
                acc.y += a.x * b.y + a.y * b.x;
            }
        } else {
            const int opp = dir == 0 ? 0 : (((dir - 1) & 1) ? dir - 1 : dir + 1);
            const double2* y = Y + (nb * ndir + opp) * bsz + i;          // column i of block (nb, opp)
            for (int j = 0; j < ncd; ++j) {
                const double2 a = y[(long long)j * ncd], b = v[j];          // conj(Y[j][i]) b_j
                acc.x += a.x * b.x + a.y * b.y;
                acc.y += a.x * b.y - a.y * b.x;
            }
        }
    }
    out[t] = acc;
}

// ---------------------------------------------------------------------------
// level-3 Galerkin kernel Dhat2_W = P2^dag Dhat_W P2 (FP64)
// ---------------------------------------------------------------------------
// One block per (level-3 site, direction).  Level-2 hop (x, d2) feeds direction
// dir3 = +-mu when it leaves x's aggregate in that direction, else the self
// block, as for the fine Galerkin product.  P2[(x * 2 + c) * nv1 + l][k].
__global__ void k_galerkin_l3(const double2* __restrict__ Y2, const double2* __restrict__ P2,
                              double2* __restrict__ Y3, AggIndex ai, int nv1, int nv2) {
    const long long xc = blockIdx.x;
    const int dir3 = blockIdx.y;
    const int nd = ai.nd, ndir = 2 * nd + 1;
    const int ncd2 = 2 * nv1, ncd3 = 2 * nv2;
    const long long bsz2 = (long long)ncd2 * ncd2;
    int nb = 1;
    for (int mu = 0; mu < nd; ++mu) nb *= ai.b[mu];
    for (int e = threadIdx.x; e < ncd3 * ncd3; e += blockDim.x) {
        const int i = e / ncd3, j = e % ncd3;
        const int ci = i / nv2, ki = i % nv2, cj = j / nv2, kj = j % nv2;
        double sre = 0.0, sim = 0.0;
        for (int l = 0; l < nb; ++l) {
            const long long x = ai.fine_site(xc, l);
            // local coordinates of x in its aggregate
            int lc[4];
            {
                long long rem = x;
                for (int mu = 0; mu < nd; ++mu) { lc[mu] = (int)(rem % ai.L[mu]) % ai.b[mu]; rem /= ai.L[mu]; }
            }
            for (int d2 = 0; d2 < ndir; ++d2) {
                int want = 0;
                if (d2 > 0) {
                    const int mu = (d2 - 1) >> 1;
                    const bool fwd = ((d2 - 1) & 1) == 0;
                    const bool crosses = fwd ? (lc[mu] == ai.b[mu] - 1) : (lc[mu] == 0);
                    want = crosses ? d2 : 0;
                }
                if (want != dir3) continue;
                const long long y = nbr_site(ai.L, nd, x, d2);
                const double2* yb = Y2 + (x * ndir + d2) * bsz2;
                // sum_{a in ci, b in cj} conj(P2(x)[a][ki]) Y[a][b] P2(y)[b][kj]
                for (int la = 0; la < nv1; ++la) {
                    const double2 px = P2[((x * 2 + ci) * nv1 + la) * nv2 + ki];
                    double qre = 0.0, qim = 0.0;
                    for (int lb = 0; lb < nv1; ++lb) {
                        const double2 a = yb[(long long)(ci * nv1 + la) * ncd2 + cj * nv1 + lb];
                        const double2 py = P2[((y * 2 + cj) * nv1 + lb) * nv2 + kj];
                        qre += a.x * py.x - a.y * py.y;
                        qim += a.x * py.y + a.y * py.x;
                    }
                    sre += px.x * qre + px.y * qim;
                    sim += px.x * qim - px.y * qre;
                }
            }
        }
        Y3[(xc * ndir + dir3) * (long long)(ncd3 * ncd3) + e] = make_double2(sre, sim);
    }
}

// ---------------------------------------------------------------------------
// wall transfers between levels 2 and 3 (Eq. TruncProjectInterpolate)
// ---------------------------------------------------------------------------
struct Xfer23 {
    AggIndex ai;
    long long V2, V3;
    int nv1, nv2, Ls2, Ls3, nb;
};

__device__ __forceinline__ long long agg_of_site(const AggIndex& ai, long long x) {
    long long xc = 0, stride = 1, rem = x;
    for (int mu = 0; mu < ai.nd; ++mu) {
        const int c = (int)(rem % ai.L[mu]);
        rem /= ai.L[mu];
        xc += (long long)(c / ai.b[mu]) * stride;
        stride *= ai.Lc[mu];
    }
    return xc;
}

// r3 on slice 1: Phat_- P2^dag Phat_- r2_1; on slice Ls3: Phat_+ P2^dag Phat_+ r2_Ls2; zero elsewhere
__global__ void k_restrict23(const float2* __restrict__ P2, const float2* __restrict__ r2, float2* __restrict__ r3,
                             Xfer23 p) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int ncd2 = 2 * p.nv1, ncd3 = 2 * p.nv2;
    if (t >= p.V3 * p.Ls3 * ncd3) return;
    const int i = (int)(t % ncd3);
    const long long rest = t / ncd3;
    const long long xc = rest % p.V3;
    const int s = (int)(rest / p.V3);
    const int c = i / p.nv2, k = i % p.nv2;
    int sf = -1;
    if (c == 1 && s == 0) sf = 0;
    if (c == 0 && s == p.Ls3 - 1) sf = p.Ls2 - 1;
    float2 acc = make_float2(0.f, 0.f);
    if (sf >= 0) {
        const float2* rs = r2 + (long long)sf * p.V2 * ncd2;
        for (int l = 0; l < p.nb; ++l) {
            const long long x = p.ai.fine_site(xc, l);
            for (int a = 0; a < p.nv1; ++a) {
                const float2 w = P2[((x * 2 + c) * p.nv1 + a) * p.nv2 + k], v = rs[x * ncd2 + c * p.nv1 + a];
                acc.x += w.x * v.x + w.y * v.y;
                acc.y += w.x * v.y - w.y * v.x;
            }
        }
    }
    r3[t] = acc;
}

// e2 on slice 1: Phat_- P2 e3_1; on slice Ls2: Phat_+ P2 e3_Ls3; zero elsewhere
__global__ void k_prolong23(const float2* __restrict__ P2, const float2* __restrict__ e3, float2* __restrict__ e2,
                            Xfer23 p) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int ncd2 = 2 * p.nv1, ncd3 = 2 * p.nv2;
    if (t >= p.V2 * p.Ls2 * ncd2) return;
    const int d = (int)(t % ncd2);
    const long long rest = t / ncd2;
    const long long x = rest % p.V2;
    const int s = (int)(rest / p.V2);
    const int c = d / p.nv1, a = d % p.nv1;
    int sc = -1;
    if (c == 1 && s == 0) sc = 0;
    if (c == 0 && s == p.Ls2 - 1) sc = p.Ls3 - 1;
    float2 acc = make_float2(0.f, 0.f);
    if (sc >= 0) {
        const long long xc = agg_of_site(p.ai, x);
        const float2* ev = e3 + ((long long)sc * p.V3 + xc) * ncd3 + c * p.nv2;
        const float2* pr = P2 + ((x * 2 + c) * p.nv1 + a) * p.nv2;
        for (int k = 0; k < p.nv2; ++k) {
            const float2 w = pr[k], v = ev[k];
            acc.x += w.x * v.x - w.y * v.y;
            acc.y += w.x * v.y + w.y * v.x;
        }
    }
    e2[t] = acc;
}

// ---------------------------------------------------------------------------
// small-vector BLAS (FP32 data, FP64 scalars)
// ---------------------------------------------------------------------------
#define L3_LOOP(i, n) for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < (n); i += (long long)gridDim.x * blockDim.x)

struct Ptrs { const float2* p[L2_MAXK]; };

inline int sgrid(long long n) {
    long long b = (n + 255) / 256;
    if (b < 1) b = 1;
    return (int)(b < 304 ? b : 304);
}

// c[j] = <W_j, w>, j < k: grid (B, k), one reduction row per j
__global__ void __launch_bounds__(RED_THREADS) k_l3_mdot(Ptrs W, const float2* __restrict__ w, long long n,
                                                         double* part, unsigned* cnt, GScal* g, const int* skip) {
    if (skip && *skip) return;
    const int j = blockIdx.y;
    const float2* a = W.p[j];
    float re = 0.f, im = 0.f;
    L3_LOOP(i, n) {
        const float2 u = a[i], v = w[i];
        re += u.x * v.x + u.y * v.y;
        im += u.x * v.y - u.y * v.x;
    }
    const float v2[2] = {re, im};
    grid_reduce_f<2>(v2, row_rs(part, cnt, j), [=] __device__(double* t) { g->c[j][0] = t[0]; g->c[j][1] = t[1]; });
}

// w -= sum_{j<k} c_j W_j, z -= sum_{j<k} c_j Z_j; then inv = 1 / |w|, alpha = <w, r> / |w|^2
__global__ void __launch_bounds__(RED_THREADS) k_l3_orth(Ptrs W, Ptrs Z, int k, float2* __restrict__ w,
                                                         float2* __restrict__ z, const float2* __restrict__ r,
                                                         long long n, RedScratch rs, GScal* g, const int* skip) {
    if (skip && *skip) return;
    __shared__ float2 c[L2_MAXK];
    if (threadIdx.x < L2_MAXK) c[threadIdx.x] = (int)threadIdx.x < k
        ? make_float2((float)g->c[threadIdx.x][0], (float)g->c[threadIdx.x][1]) : make_float2(0.f, 0.f);
    __syncthreads();
    float nn = 0.f, ar = 0.f, ai = 0.f;
    L3_LOOP(i, n) {
        float2 a = w[i], b = z[i];
        for (int j = 0; j < k; ++j) {
            const float2 wj = W.p[j][i], zj = Z.p[j][i], cj = c[j];
            a.x -= cj.x * wj.x - cj.y * wj.y; a.y -= cj.x * wj.y + cj.y * wj.x;
            b.x -= cj.x * zj.x - cj.y * zj.y; b.y -= cj.x * zj.y + cj.y * zj.x;
        }
        if (k > 0) { w[i] = a; z[i] = b; }
        const float2 ri = r[i];
        nn += a.x * a.x + a.y * a.y;
        ar += a.x * ri.x + a.y * ri.y;
        ai += a.x * ri.y - a.y * ri.x;
    }
    const float v[3] = {nn, ar, ai};
    grid_reduce_f<3>(v, rs, [=] __device__(double* t) {
        if (t[0] > 0.0) {
            g->inv = 1.0 / sqrt(t[0]);
            g->alpha[0] = t[1] / t[0];
            g->alpha[1] = t[2] / t[0];
        } else {
            g->inv = 0.0; g->alpha[0] = 0.0; g->alpha[1] = 0.0;
        }
    });
}

// e += alpha z, r -= alpha w, then w *= inv, z *= inv (the stored normalised pair); |r|^2,
// steps += 1, done once |r|^2 <= ref2
__global__ void __launch_bounds__(RED_THREADS) k_l3_upd(float2* __restrict__ w, float2* __restrict__ z,
                                                        float2* __restrict__ e, float2* __restrict__ r, long long n,
                                                        RedScratch rs, GScal* g, const int* skip) {
    if (skip && *skip) return;
    const float ar = (float)g->alpha[0], ai = (float)g->alpha[1], inv = (float)g->inv;
    float acc = 0.f;
    L3_LOOP(i, n) {
        float2 a = w[i], b = z[i], ei = e[i], ri = r[i];
        ei.x += ar * b.x - ai * b.y; ei.y += ar * b.y + ai * b.x;
        ri.x -= ar * a.x - ai * a.y; ri.y -= ar * a.y + ai * a.x;
        e[i] = ei; r[i] = ri;
        w[i] = make_float2(a.x * inv, a.y * inv);
        z[i] = make_float2(b.x * inv, b.y * inv);
        acc += ri.x * ri.x + ri.y * ri.y;
    }
    const float v[1] = {acc};
    grid_reduce_f<1>(v, rs, [=] __device__(double* t) {
        g->rr2 = t[0];
        g->steps += 1;
        if (t[0] <= g->ref2 || g->steps >= g->maxit) g->done = 1;
    });
}

__global__ void __launch_bounds__(RED_THREADS) k_l3_norm(const float2* __restrict__ a, long long n, RedScratch rs,
                                                         double* out) {
    float acc = 0.f;
    L3_LOOP(i, n) { const float2 u = a[i]; acc += u.x * u.x + u.y * u.y; }
    const float v[1] = {acc};
    grid_reduce_f<1>(v, rs, [=] __device__(double* t) { *out = t[0]; });
}

__global__ void k_l3_sub(float2* __restrict__ out, const float2* __restrict__ a, const float2* __restrict__ b,
                         long long n) {
    L3_LOOP(i, n) { const float2 u = a[i], v = b[i]; out[i] = make_float2(u.x - v.x, u.y - v.y); }
}

// rr2 = |r0|^2, ref2 = tol^2 |ref|^2 (ref = r0 when ref2 is null), no steps yet
__global__ void k_l3_gscal_init(GScal* g, const double* r2, const double* refn2, double tol, int maxit) {
    g->rr2 = *r2;
    g->ref2 = tol * tol * (refn2 ? *refn2 : *r2);
    g->steps = 0;
    g->maxit = maxit;
    g->done = (*r2 <= g->ref2 || maxit <= 0) ? 1 : 0;
}

__global__ void k_l3_copy(float2* __restrict__ out, const float2* __restrict__ in, long long n, const int* skip) {
    if (skip && *skip) return;
    L3_LOOP(i, n) out[i] = in[i];
}

// ---------------------------------------------------------------------------
// coarsest CGNR (device stop flag; every kernel returns at once when done)
// ---------------------------------------------------------------------------
// alpha = |r|^2 / |q|^2
__global__ void __launch_bounds__(RED_THREADS) k_cg3_alpha(const float2* __restrict__ q, long long n, RedScratch rs,
                                                           Cg3* S) {
    if (S->done) return;
    float acc = 0.f;
    L3_LOOP(i, n) { const float2 u = q[i]; acc += u.x * u.x + u.y * u.y; }
    const float v[1] = {acc};
    grid_reduce_f<1>(v, rs, [=] __device__(double* t) {
        if (t[0] > 0.0) S->alpha = S->rn2 / t[0];
        else { S->alpha = 0.0; S->done = 1; }
    });
}

// x += alpha p, rr -= alpha q; |rr|^2; iters += 1; done on tolerance or cap
__global__ void __launch_bounds__(RED_THREADS) k_cg3_upd1(float2* __restrict__ x, float2* __restrict__ rr,
                                                          const float2* __restrict__ p, const float2* __restrict__ q,
                                                          long long n, RedScratch rs, Cg3* S) {
    if (S->done) return;
    const float a = (float)S->alpha;
    float acc = 0.f;
    L3_LOOP(i, n) {
        float2 xi = x[i], ri = rr[i];
        const float2 pi = p[i], qi = q[i];
        xi.x += a * pi.x; xi.y += a * pi.y;
        ri.x -= a * qi.x; ri.y -= a * qi.y;
        x[i] = xi; rr[i] = ri;
        acc += ri.x * ri.x + ri.y * ri.y;
    }
    const float v[1] = {acc};
    grid_reduce_f<1>(v, rs, [=] __device__(double* t) {
        S->rr2 = t[0];
        S->iters += 1;
        if (t[0] <= S->tol2 * S->bn2 || S->iters >= S->maxit) S->done = 1;
    });
}

// r -= alpha w; beta = |r|^2 / |r_old|^2
__global__ void __launch_bounds__(RED_THREADS) k_cg3_upd2(float2* __restrict__ r, const float2* __restrict__ w,
                                                          long long n, RedScratch rs, Cg3* S) {
    if (S->done) return;
    const float a = (float)S->alpha;
    float acc = 0.f;
    L3_LOOP(i, n) {
        float2 ri = r[i];
        const float2 wi = w[i];
        ri.x -= a * wi.x; ri.y -= a * wi.y;
        r[i] = ri;
        acc += ri.x * ri.x + ri.y * ri.y;
    }
    const float v[1] = {acc};
    grid_reduce_f<1>(v, rs, [=] __device__(double* t) {
        S->beta = S->rn2 > 0.0 ? t[0] / S->rn2 : 0.0;
        S->rn2 = t[0];
    });
}

__global__ void k_cg3_p(float2* __restrict__ p, const float2* __restrict__ r, long long n, const Cg3* S) {
    if (S->done) return;
    const float b = (float)S->beta;
    L3_LOOP(i, n) { const float2 ri = r[i], pi = p[i]; p[i] = make_float2(ri.x + b * pi.x, ri.y + b * pi.y); }
}

// start: rn2 = |r|^2, rr2 = |rr|^2, bn2 = |b|^2 (three reductions), done if b = 0 or rr small
__global__ void __launch_bounds__(RED_THREADS) k_cg3_init(const float2* __restrict__ r, const float2* __restrict__ rr,
                                                          const float2* __restrict__ b, long long n, RedScratch rs,
                                                          Cg3* S, double tol, int maxit) {
    float a0 = 0.f, a1 = 0.f, a2 = 0.f;
    L3_LOOP(i, n) {
        const float2 u = r[i], v = rr[i], w = b[i];
        a0 += u.x * u.x + u.y * u.y;
        a1 += v.x * v.x + v.y * v.y;
        a2 += w.x * w.x + w.y * w.y;
    }
    const float v[3] = {a0, a1, a2};
    grid_reduce_f<3>(v, rs, [=] __device__(double* t) {
        S->rn2 = t[0]; S->rr2 = t[1]; S->bn2 = t[2]; S->tol2 = tol * tol;
        S->iters = 0; S->maxit = maxit;
        S->done = (t[2] == 0.0 || t[1] <= tol * tol * t[2] || maxit <= 0) ? 1 : 0;
    });
}

// ---------------------------------------------------------------------------
// deflation: dense pieces
// ---------------------------------------------------------------------------
// c_i = <V_i, f> (FP64), one block per basis vector
__global__ void __launch_bounds__(RED_THREADS) k_defl_dots(const float2* __restrict__ V, const float2* __restrict__ f,
                                                           long long n, double2* __restrict__ c) {
    const float2* v = V + (long long)blockIdx.x * n;
    double re = 0.0, im = 0.0;
    for (long long i = threadIdx.x; i < n; i += blockDim.x) {
        const float2 a = v[i], b = f[i];
        re += (double)a.x * b.x + (double)a.y * b.y;
        im += (double)a.x * b.y - (double)a.y * b.x;
    }
    double w[2] = {re, im};
    block_sum<2>(w);
    if (threadIdx.x == 0) c[blockIdx.x] = make_double2(w[0], w[1]);
}

// y = H^-1 c with H = L L^dag (L lower, row-major k x k): forward then back substitution, one block
__global__ void k_defl_solve(const double2* __restrict__ Lf, double2* __restrict__ c, int k) {
    __shared__ double2 y[DEFL_MAX];
    for (int i = threadIdx.x; i < k; i += blockDim.x) y[i] = c[i];
    __syncthreads();
    for (int i = 0; i < k; ++i) {              // L u = c
        if (threadIdx.x == 0) {
            const double2 d = Lf[(long long)i * k + i];
            y[i] = make_double2(y[i].x / d.x, y[i].y / d.x);   // diagonal is real
        }
        __syncthreads();
        for (int r = i + 1 + threadIdx.x; r < k; r += blockDim.x) {
            const double2 l = Lf[(long long)r * k + i];
            y[r].x -= l.x * y[i].x - l.y * y[i].y;
            y[r].y -= l.x * y[i].y + l.y * y[i].x;
        }
        __syncthreads();
    }
    for (int i = k - 1; i >= 0; --i) {         // L^dag y = u
        if (threadIdx.x == 0) {
            const double2 d = Lf[(long long)i * k + i];
            y[i] = make_double2(y[i].x / d.x, y[i].y / d.x);
        }
        __syncthreads();
        for (int r = threadIdx.x; r < i; r += blockDim.x) {
            const double2 l = Lf[(long long)i * k + r];      // (L^dag)[r][i] = conj(L[i][r])
            y[r].x -= l.x * y[i].x + l.y * y[i].y;
            y[r].y -= l.x * y[i].y - l.y * y[i].x;
        }
        __syncthreads();
    }
    for (int i = threadIdx.x; i < k; i += blockDim.x) c[i] = y[i];
}

// x = sum_i V_i y_i
__global__ void k_defl_combine(const float2* __restrict__ V, const double2* __restrict__ y, int k, long long n,
                               float2* __restrict__ x) {
    __shared__ float2 ys[DEFL_MAX];
    for (int i = threadIdx.x; i < k; i += blockDim.x) ys[i] = make_float2((float)y[i].x, (float)y[i].y);
    __syncthreads();
    L3_LOOP(e, n) {
        float2 acc = make_float2(0.f, 0.f);
        for (int i = 0; i < k; ++i) {
            const float2 a = V[(long long)i * n + e], b = ys[i];
            acc.x += a.x * b.x - a.y * b.y;
            acc.y += a.x * b.y + a.y * b.x;
        }
        x[e] = acc;
    }
}

// ---- Lanczos with full reorthogonalisation (FP32 basis, FP64 scalars) ----
// c_i = <Q_i, w> for i < j, one block per i (into c), FP64
__global__ void __launch_bounds__(RED_THREADS) k_lz_dots(const float2* __restrict__ Q, const float2* __restrict__ w,
                                                         long long n, double2* __restrict__ c) {
    const float2* q = Q + (long long)blockIdx.x * n;
    double re = 0.0, im = 0.0;
    for (long long i = threadIdx.x; i < n; i += blockDim.x) {
        const float2 a = q[i], b = w[i];
        re += (double)a.x * b.x + (double)a.y * b.y;
        im += (double)a.x * b.y - (double)a.y * b.x;
    }
    double v[2] = {re, im};
    block_sum<2>(v);
    if (threadIdx.x == 0) c[blockIdx.x] = make_double2(v[0], v[1]);
}

// w -= sum_{i<j} Q_i c_i; acc[i] += c_i (the accumulated projections)
__global__ void k_lz_sub(const float2* __restrict__ Q, const double2* __restrict__ c, int j, long long n,
                         float2* __restrict__ w) {
    L3_LOOP(e, n) {
        float2 a = w[e];
        for (int i = 0; i < j; ++i) {
            const float2 q = Q[(long long)i * n + e];
            const float cr = (float)c[i].x, ci = (float)c[i].y;
            a.x -= q.x * cr - q.y * ci;
            a.y -= q.x * ci + q.y * cr;
        }
        w[e] = a;
    }
}

__global__ void k_lz_scale(const float2* __restrict__ w, float2* __restrict__ q, long long n, const double* nrm2) {
    const float s = (float)(1.0 / sqrt(*nrm2));
    L3_LOOP(e, n) { const float2 a = w[e]; q[e] = make_float2(a.x * s, a.y * s); }
}

__global__ void __launch_bounds__(RED_THREADS) k_lz_norm64in(const double2* __restrict__ a, long long n,
                                                             float2* __restrict__ q) {
    // one block: q = a / |a| (the Lanczos start)
    double s = 0.0;
    for (long long i = threadIdx.x; i < n; i += blockDim.x) s += a[i].x * a[i].x + a[i].y * a[i].y;
    double v[1] = {s};
    block_sum<1>(v);
    __shared__ double inv;
    if (threadIdx.x == 0) inv = v[0] > 0.0 ? 1.0 / sqrt(v[0]) : 0.0;
    __syncthreads();
    for (long long i = threadIdx.x; i < n; i += blockDim.x) q[i] = make_float2((float)(a[i].x * inv), (float)(a[i].y * inv));
}

// ---- the Lanczos matrix T (alpha diagonal, beta off-diagonal, size m), FP64 ----
// number of eigenvalues of T below x (Sturm sequence of the LDL^T pivots)
__device__ int sturm_count(const double* a, const double* b, int m, double x) {
    int cnt = 0;
    double d = 1.0;
    for (int i = 0; i < m; ++i) {
        const double bb = i > 0 ? b[i - 1] * b[i - 1] : 0.0;
        d = (a[i] - x) - (i > 0 ? bb / d : 0.0);
        if (d == 0.0) d = -1e-300;
        if (d < 0.0) ++cnt;
    }
    return cnt;
}

// eigenvalue idx (ascending) of T by bisection on the Sturm count; its vector by inverse
// iteration: Gaussian elimination with partial pivoting of T - lam 1 (rows i, i+1 swapped when
// the sub-diagonal entry is the larger), three solves from a fixed start, normalised.
// scratch: 6 m doubles per thread (U diagonal, two superdiagonals, multipliers, swap flags, z).
__global__ void k_tridiag_eig(const double* __restrict__ a, const double* __restrict__ b, int m, int k,
                              double* __restrict__ lam, double* __restrict__ S, double* __restrict__ scratch) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= k) return;
    double lo = 1e300, hi = -1e300;
    for (int i = 0; i < m; ++i) {            // Gershgorin interval
        const double r = (i > 0 ? fabs(b[i - 1]) : 0.0) + (i + 1 < m ? fabs(b[i]) : 0.0);
        lo = fmin(lo, a[i] - r);
        hi = fmax(hi, a[i] + r);
    }
    const double span = fmax(hi - lo, 1e-300);
    lo -= 1e-12 * span;
    hi += 1e-12 * span;
    for (int it = 0; it < 300 && hi - lo > 4e-16 * fmax(fabs(lo), fabs(hi)) + 1e-300; ++it) {
        const double mid = 0.5 * (lo + hi);
        if (sturm_count(a, b, m, mid) > idx) hi = mid; else lo = mid;
    }
    const double x = 0.5 * (lo + hi);
    lam[idx] = x;
    double* D = scratch + (size_t)idx * 6 * m;
    double* U1 = D + m;
    double* U2 = U1 + m;
    double* Lm = U2 + m;
    double* sw = Lm + m;
    double* z = sw + m;
    for (int i = 0; i < m; ++i) { D[i] = a[i] - x; U1[i] = i + 1 < m ? b[i] : 0.0; U2[i] = 0.0; }
    for (int i = 0; i + 1 < m; ++i) {
        const double c = b[i];                  // entry (i + 1, i)
        if (fabs(D[i]) >= fabs(c)) {
            const double l = D[i] != 0.0 ? c / D[i] : 0.0;
            D[i + 1] -= l * U1[i];
            Lm[i] = l;
            sw[i] = 0.0;
        } else {
            // new row i = old row i + 1 = (c, D[i+1], U1[i+1]); new row i + 1 = old row i - l new row i
            const double l = D[i] / c;
            const double t1 = D[i + 1], t2 = U1[i + 1];
            D[i] = c;
            D[i + 1] = U1[i] - l * t1;
            U1[i] = t1;
            U2[i] = t2;
            U1[i + 1] = -l * t2;
            Lm[i] = l;
            sw[i] = 1.0;
        }
        if (D[i] == 0.0) D[i] = 1e-300 * span;
    }
    if (D[m - 1] == 0.0) D[m - 1] = 1e-300 * span;
    for (int i = 0; i < m; ++i) z[i] = 1.0 + 0.5 * (double)((i * 7919 + idx * 104729) % 211) / 211.0;
    for (int pass = 0; pass < 3; ++pass) {
        for (int i = 0; i + 1 < m; ++i) {     // the row operations
            if (sw[i] != 0.0) { const double t = z[i]; z[i] = z[i + 1]; z[i + 1] = t; }
            z[i + 1] -= Lm[i] * z[i];
        }
        for (int i = m - 1; i >= 0; --i) {    // back substitution with U
            double v = z[i];
            if (i + 1 < m) v -= U1[i] * z[i + 1];
            if (i + 2 < m) v -= U2[i] * z[i + 2];
            z[i] = v / D[i];
        }
        double mx = 0.0;
        for (int i = 0; i < m; ++i) mx = fmax(mx, fabs(z[i]));
        const double sc = mx > 0.0 ? 1.0 / mx : 0.0;
        for (int i = 0; i < m; ++i) z[i] *= sc;
    }
    double nn = 0.0;
    for (int i = 0; i < m; ++i) nn += z[i] * z[i];
    const double inv = nn > 0.0 ? 1.0 / sqrt(nn) : 0.0;
    for (int i = 0; i < m; ++i) S[(size_t)idx * m + i] = z[i] * inv;
}

// classical Gram-Schmidt (twice) of the k columns S[c][0..m) in the Lanczos space, one block;
// a column left with norm below 1e-8 of its own is dropped (set to zero)
__global__ void k_small_orth(double* __restrict__ S, int m, int k) {
    __shared__ double red[32];
    for (int c = 0; c < k; ++c) {
        double* sc = S + (size_t)c * m;
        double n0 = 0.0;
        for (int i = threadIdx.x; i < m; i += blockDim.x) n0 += sc[i] * sc[i];
        // block reduce
        for (int o = 16; o > 0; o >>= 1) n0 += __shfl_down_sync(0xffffffffu, n0, o);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = n0;
        __syncthreads();
        if (threadIdx.x < 32) {
            double v = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
            for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
            if (threadIdx.x == 0) red[0] = v;
        }
        __syncthreads();
        n0 = red[0];
        __syncthreads();
        for (int pass = 0; pass < 2; ++pass) {
            for (int p = 0; p < c; ++p) {
                const double* sp = S + (size_t)p * m;
                double d = 0.0;
                for (int i = threadIdx.x; i < m; i += blockDim.x) d += sp[i] * sc[i];
                for (int o = 16; o > 0; o >>= 1) d += __shfl_down_sync(0xffffffffu, d, o);
                if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = d;
                __syncthreads();
                if (threadIdx.x < 32) {
                    double v = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
                    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
                    if (threadIdx.x == 0) red[0] = v;
                }
                __syncthreads();
                d = red[0];
                __syncthreads();
                for (int i = threadIdx.x; i < m; i += blockDim.x) sc[i] -= d * sp[i];
                __syncthreads();
            }
        }
        double nn = 0.0;
        for (int i = threadIdx.x; i < m; i += blockDim.x) nn += sc[i] * sc[i];
        for (int o = 16; o > 0; o >>= 1) nn += __shfl_down_sync(0xffffffffu, nn, o);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = nn;
        __syncthreads();
        if (threadIdx.x < 32) {
            double v = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
            for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
            if (threadIdx.x == 0) red[0] = v;
        }
        __syncthreads();
        nn = red[0];
        __syncthreads();
        const double inv = (nn > 1e-16 * n0 && nn > 0.0) ? 1.0 / sqrt(nn) : 0.0;
        for (int i = threadIdx.x; i < m; i += blockDim.x) sc[i] *= inv;
        __syncthreads();
    }
}

// in-place Cholesky H = L L^dag (lower, row-major), one block; a non-positive pivot (a dropped
// column) becomes 1 with its row and column of L zero, so that direction contributes nothing
__global__ void k_cholesky(double2* __restrict__ H, int k) {
    __shared__ double piv;
    double hmax = 0.0;
    for (int i = 0; i < k; ++i) hmax = fmax(hmax, H[(long long)i * k + i].x);
    for (int j = 0; j < k; ++j) {
        if (threadIdx.x == 0) {
            double d = H[(long long)j * k + j].x;
            for (int p = 0; p < j; ++p) {
                const double2 l = H[(long long)j * k + p];
                d -= l.x * l.x + l.y * l.y;
            }
            piv = d > 1e-13 * hmax ? sqrt(d) : 0.0;
            H[(long long)j * k + j] = make_double2(piv > 0.0 ? piv : 1.0, 0.0);
        }
        __syncthreads();
        for (int r = j + 1 + threadIdx.x; r < k; r += blockDim.x) {
            if (piv == 0.0) { H[(long long)r * k + j] = make_double2(0.0, 0.0); continue; }
            double2 s = H[(long long)r * k + j];
            for (int p = 0; p < j; ++p) {
                const double2 a = H[(long long)r * k + p], c = H[(long long)j * k + p];   // a conj(c)
                s.x -= a.x * c.x + a.y * c.y;
                s.y -= a.y * c.x - a.x * c.y;
            }
            H[(long long)r * k + j] = make_double2(s.x / piv, s.y / piv);
        }
        __syncthreads();
    }
    for (int t = threadIdx.x; t < k * k; t += blockDim.x)          // zero the strict upper triangle
        if (t % k > t / k) H[t] = make_double2(0.0, 0.0);
}

// V[c] = sum_r Q[r] S[c][r] for the columns c of one chunk of 16
__global__ void k_ritz_vectors(const float2* __restrict__ Q, const double* __restrict__ S, int m, int k, long long n,
                               float2* __restrict__ V) {
    const int c0 = blockIdx.y * 16;
    L3_LOOP(e, n) {
        float2 acc[16];
#pragma unroll
        for (int u = 0; u < 16; ++u) acc[u] = make_float2(0.f, 0.f);
        for (int r = 0; r < m; ++r) {
            const float2 q = Q[(long long)r * n + e];
#pragma unroll
            for (int u = 0; u < 16; ++u)
                if (c0 + u < k) {
                    const float s = (float)S[(size_t)(c0 + u) * m + r];
                    acc[u].x += s * q.x;
                    acc[u].y += s * q.y;
                }
        }
#pragma unroll
        for (int u = 0; u < 16; ++u)
            if (c0 + u < k) V[(long long)(c0 + u) * n + e] = acc[u];
    }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
inline Level3* L3(const dwf_mg* h) { return reinterpret_cast<Level3*>(h->lvl3); }

Xfer23 xfer_params(const Level3& L) {
    Xfer23 p;
    p.ai.nd = 2;
    for (int mu = 0; mu < 4; ++mu) { p.ai.L[mu] = L.L2[mu]; p.ai.b[mu] = L.b2[mu]; p.ai.Lc[mu] = L.L3[mu]; }
    p.V2 = L.V2; p.V3 = L.V3; p.nv1 = L.nvec1; p.nv2 = L.nvec2; p.Ls2 = L.Ls2; p.Ls3 = L.Ls3; p.nb = L.nb2;
    return p;
}

dwf_status l3_apply(const Level3& L, const float2* in, float2* out, double mf, bool dagger, const int* skip,
                    cudaStream_t st) {
    CoarseParams p = L.p3;
    p.mf = (float)mf;
    if (L.Y3_16) return coarse_site_apply(p, L.Y3_16, in, out, dagger, skip, L.status, st);
    return coarse_site_apply(p, L.Y3_32, in, out, dagger, skip, L.status, st);
}

// out = A3 in = Dhat2_PV^dag Dhat2_DW in (tmp: scratch); dag: A3^dag = Dhat2_DW^dag Dhat2_PV
dwf_status l3_apply_A(const dwf_mg* h, const Level3& L, const float2* in, float2* out, float2* tmp, bool dag,
                      const int* skip, cudaStream_t st) {
    if (!dag) {
        DWF_TRY(l3_apply(L, in, tmp, h->mf, false, skip, st));
        return l3_apply(L, tmp, out, 1.0, true, skip, st);
    }
    DWF_TRY(l3_apply(L, in, tmp, 1.0, false, skip, st));
    return l3_apply(L, tmp, out, h->mf, true, skip, st);
}

// out = Ahat in on level 2 (the handle's coarse operator)
dwf_status l2_apply_A(dwf_mg* h, const float2* in, float2* out, float2* tmp, cudaStream_t st) {
    DWF_TRY(coarse_dwf_apply(h, in, tmp, h->mf, false, nullptr, st));
    return coarse_dwf_apply(h, tmp, out, 1.0, true, nullptr, st);
}

// one CGNR iteration on level 3 (device stop flag)
dwf_status cg3_iteration(const dwf_mg* h, Level3& L, cudaStream_t st) {
    const long long n = L.n3;
    const int g = sgrid(n);
    RedScratch rs = row_rs(L.red_part, L.red_cnt, 0);
    const int* skip = &L.cg->done;
    DWF_TRY(l3_apply_A(h, L, L.p3v, L.q3, L.t3, false, skip, st));
    k_cg3_alpha<<<g, RED_THREADS, 0, st>>>(L.q3, n, rs, L.cg);
    k_cg3_upd1<<<g, RED_THREADS, 0, st>>>(L.x3, L.rr3, L.p3v, L.q3, n, rs, L.cg);
    DWF_CHECK_LAUNCH();
    DWF_TRY(l3_apply_A(h, L, L.q3, L.w3, L.t3, true, skip, st));
    k_cg3_upd2<<<g, RED_THREADS, 0, st>>>(L.r3, L.w3, n, rs, L.cg);
    k_cg3_p<<<g, 256, 0, st>>>(L.p3v, L.r3, n, L.cg);
    DWF_CHECK_LAUNCH();
    return DWF_OK;
}

dwf_status cg3_capture(const dwf_mg* h, Level3& L) {
    if (!L.cap_stream) DWF_CHECK_CUDA(cudaStreamCreateWithFlags(&L.cap_stream, cudaStreamNonBlocking));
    cudaGraph_t graph = nullptr;
    DWF_CHECK_CUDA(cudaStreamBeginCapture(L.cap_stream, cudaStreamCaptureModeThreadLocal));
    dwf_status s = DWF_OK;
    for (int k = 0; k < L3_GRAPH_ITERS && s == DWF_OK; ++k) s = cg3_iteration(h, L, L.cap_stream);
    cudaError_t e = cudaStreamEndCapture(L.cap_stream, &graph);
    if (s != DWF_OK) { if (graph) cudaGraphDestroy(graph); return s; }
    if (e != cudaSuccess) { set_error("graph capture: %s", cudaGetErrorString(e)); return DWF_ERR_CUDA; }
    e = cudaGraphInstantiate(&L.cg_graph, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) { set_error("graph instantiation: %s", cudaGetErrorString(e)); return DWF_ERR_CUDA; }
    return DWF_OK;
}

dwf_status level3_gcr(const dwf_mg* h, Level3& L, double tol, int maxit, int* iters, cudaStream_t st);

// x3 = (deflated) CGNR solution of A3 x = b3 to tol (or restarted GCR on A3 x = b3 with
// coarsest_solver = 1); iteration count out
dwf_status level3_solve_impl(const dwf_mg* h, Level3& L, const float2* b3, float2* x3, double tol, int maxit,
                             bool deflate, int* iters, cudaStream_t st) {
    const long long n = L.n3;
    const size_t vb = (size_t)n * sizeof(float2);
    const int g = sgrid(n);
    RedScratch rs = row_rs(L.red_part, L.red_cnt, 0);
    if (b3 != L.b3) DWF_CHECK_CUDA(cudaMemcpyAsync(L.b3, b3, vb, cudaMemcpyDeviceToDevice, st));
    if (deflate && L.ndefl > 0) {
        // x0 = V H^-1 V^dag A3^dag b
        DWF_TRY(l3_apply_A(h, L, L.b3, L.w3, L.t3, true, nullptr, st));
        k_defl_dots<<<L.ndefl, RED_THREADS, 0, st>>>(L.Vd, L.w3, n, L.dc);
        k_defl_solve<<<1, 256, 0, st>>>(L.Hl, L.dc, L.ndefl);
        k_defl_combine<<<g, 256, 0, st>>>(L.Vd, L.dc, L.ndefl, n, L.x3);
        DWF_CHECK_LAUNCH();
        DWF_TRY(l3_apply_A(h, L, L.x3, L.q3, L.t3, false, nullptr, st));
        k_l3_sub<<<g, 256, 0, st>>>(L.rr3, L.b3, L.q3, n);
        DWF_CHECK_LAUNCH();
    } else {
        DWF_CHECK_CUDA(cudaMemsetAsync(L.x3, 0, vb, st));
        DWF_CHECK_CUDA(cudaMemcpyAsync(L.rr3, L.b3, vb, cudaMemcpyDeviceToDevice, st));
    }
    if (L.prm.coarsest_solver == 1) {
        DWF_TRY(level3_gcr(h, L, tol, maxit, iters, st));
        if (x3 != L.x3) DWF_CHECK_CUDA(cudaMemcpyAsync(x3, L.x3, vb, cudaMemcpyDeviceToDevice, st));
        return DWF_OK;
    }
    DWF_TRY(l3_apply_A(h, L, L.rr3, L.r3, L.t3, true, nullptr, st));
    DWF_CHECK_CUDA(cudaMemcpyAsync(L.p3v, L.r3, vb, cudaMemcpyDeviceToDevice, st));
    k_cg3_init<<<g, RED_THREADS, 0, st>>>(L.r3, L.rr3, L.b3, n, rs, L.cg, tol, maxit);
    DWF_CHECK_LAUNCH();
    if (!L.cg_graph) DWF_TRY(cg3_capture(h, L));
    Cg3* hc = reinterpret_cast<Cg3*>(L.hpin);
    for (;;) {
        DWF_CHECK_CUDA(cudaMemcpyAsync(hc, L.cg, sizeof(Cg3), cudaMemcpyDeviceToHost, st));
        DWF_CHECK_CUDA(cudaStreamSynchronize(st));
        if (hc->done) break;
        DWF_CHECK_CUDA(cudaGraphLaunch(L.cg_graph, st));
    }
    if (x3 != L.x3) DWF_CHECK_CUDA(cudaMemcpyAsync(x3, L.x3, vb, cudaMemcpyDeviceToDevice, st));
    *iters = hc->iters;
    return DWF_OK;
}

// one GCR step on n-value vectors: w (= A z, unnormalised) and z are orthogonalised against the k
// stored pairs (W, Z), then e += alpha z, r -= alpha w and the normalised pair is stored in place;
// skip: device stop flag (may be null)
dwf_status gcr_step(Level3& L, long long n, float2* const* W, float2* const* Z, int k, float2* w, float2* z,
                    float2* e, float2* r, GScal* gs, const int* skip, cudaStream_t st) {
    const int g = sgrid(n);
    Ptrs Wp, Zp;
    for (int j = 0; j < L2_MAXK; ++j) { Wp.p[j] = j < k ? W[j] : nullptr; Zp.p[j] = j < k ? Z[j] : nullptr; }
    if (k > 0)
        k_l3_mdot<<<dim3(g, k), RED_THREADS, 0, st>>>(Wp, w, n, L.red_part + PROW3, L.red_cnt + CROW3, gs, skip);
    k_l3_orth<<<g, RED_THREADS, 0, st>>>(Wp, Zp, k, w, z, r, n, row_rs(L.red_part, L.red_cnt, 0), gs, skip);
    k_l3_upd<<<g, RED_THREADS, 0, st>>>(w, z, e, r, n, row_rs(L.red_part, L.red_cnt, 0), gs, skip);
    DWF_CHECK_LAUNCH();
    return DWF_OK;
}

dwf_status gcr2_step(Level3& L, float2* const* W, float2* const* Z, int k, float2* w, float2* z, float2* e,
                     float2* r, GScal* gs, cudaStream_t st) {
    return gcr_step(L, L.n2, W, Z, k, w, z, e, r, gs, nullptr, st);
}

// one restart cycle of the coarsest GCR (coarsest_restart steps, every launch skipped once done)
dwf_status gcr3_cycle(const dwf_mg* h, Level3& L, cudaStream_t st) {
    const long long n = L.n3;
    const int* skip = &L.g3->done;
    for (int k = 0; k < L.prm.coarsest_restart; ++k) {
        k_l3_copy<<<sgrid(n), 256, 0, st>>>(L.Z3[k], L.rr3, n, skip);
        DWF_CHECK_LAUNCH();
        DWF_TRY(l3_apply_A(h, L, L.Z3[k], L.W3[k], L.t3, false, skip, st));
        DWF_TRY(gcr_step(L, n, L.W3, L.Z3, k, L.W3[k], L.Z3[k], L.x3, L.rr3, L.g3, skip, st));
    }
    return DWF_OK;
}

// restarted GCR on A3 x = b3 from x3 with residual rr3 (both set by the caller), to
// |r| <= tol |b3| or maxit steps, the restart cycle under one CUDA graph
dwf_status level3_gcr(const dwf_mg* h, Level3& L, double tol, int maxit, int* iters, cudaStream_t st) {
    const long long n = L.n3;
    const int g = sgrid(n);
    double* d = reinterpret_cast<double*>(L.cg) + 48;           // |r0|^2, |b|^2 (spare slots)
    k_l3_norm<<<g, RED_THREADS, 0, st>>>(L.rr3, n, row_rs(L.red_part, L.red_cnt, 0), d);
    k_l3_norm<<<g, RED_THREADS, 0, st>>>(L.b3, n, row_rs(L.red_part, L.red_cnt, 0), d + 1);
    k_l3_gscal_init<<<1, 1, 0, st>>>(L.g3, d, d + 1, tol, maxit);
    DWF_CHECK_LAUNCH();
    if (!L.gcr3_graph) {
        if (!L.cap_stream) DWF_CHECK_CUDA(cudaStreamCreateWithFlags(&L.cap_stream, cudaStreamNonBlocking));
        cudaGraph_t graph = nullptr;
        DWF_CHECK_CUDA(cudaStreamBeginCapture(L.cap_stream, cudaStreamCaptureModeThreadLocal));
        dwf_status s = gcr3_cycle(h, L, L.cap_stream);
        cudaError_t e = cudaStreamEndCapture(L.cap_stream, &graph);
        if (s != DWF_OK) { if (graph) cudaGraphDestroy(graph); return s; }
        if (e != cudaSuccess) { set_error("graph capture: %s", cudaGetErrorString(e)); return DWF_ERR_CUDA; }
        e = cudaGraphInstantiate(&L.gcr3_graph, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) { set_error("graph instantiation: %s", cudaGetErrorString(e)); return DWF_ERR_CUDA; }
    }
    GScal* hg = reinterpret_cast<GScal*>(reinterpret_cast<char*>(L.hpin) + 1024);
    for (;;) {
        DWF_CHECK_CUDA(cudaMemcpyAsync(hg, L.g3, sizeof(GScal), cudaMemcpyDeviceToHost, st));
        DWF_CHECK_CUDA(cudaStreamSynchronize(st));
        if (hg->done) break;
        DWF_CHECK_CUDA(cudaGraphLaunch(L.gcr3_graph, st));
    }
    *iters = hg->steps;
    return DWF_OK;
}

// z = M2(r): restrict, level-3 solve, prolong, post-smooth on Ahat; returns with rs = r - Ahat z
dwf_status level2_precondition(dwf_mg* h, Level3& L, const float2* r, float2* z, int* l3it, cudaStream_t st) {
    const long long n = L.n2;
    const size_t vb = (size_t)n * sizeof(float2);
    const int g = sgrid(n);
    const Xfer23 xp = xfer_params(L);
    k_restrict23<<<(unsigned)((L.n3 + 255) / 256), 256, 0, st>>>(L.P2_32, r, L.b3, xp);
    DWF_CHECK_LAUNCH();
    int it = 0;
    DWF_TRY(level3_solve_impl(h, L, L.b3, L.x3, L.prm.coarsest_tol, L.prm.coarsest_maxiter, true, &it, st));
    *l3it += it;
    k_prolong23<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(L.P2_32, L.x3, z, xp);
    DWF_CHECK_LAUNCH();
    // rs = r - Ahat z
    DWF_TRY(l2_apply_A(h, z, L.a2, L.t2, st));
    k_l3_sub<<<g, 256, 0, st>>>(L.rs, r, L.a2, n);
    DWF_CHECK_LAUNCH();
    const int S = L.prm.post_smooth;
    if (S > 0) {
        DWF_CHECK_CUDA(cudaMemcpyAsync(L.es, z, vb, cudaMemcpyDeviceToDevice, st));
        for (int j = 0; j < S; ++j) {
            DWF_CHECK_CUDA(cudaMemcpyAsync(L.Zs[j], L.rs, vb, cudaMemcpyDeviceToDevice, st));
            DWF_TRY(l2_apply_A(h, L.Zs[j], L.Ws[j], L.t2, st));
            DWF_TRY(gcr2_step(L, L.Ws, L.Zs, j, L.Ws[j], L.Zs[j], L.es, L.rs, L.gs, st));
        }
        DWF_CHECK_CUDA(cudaMemcpyAsync(z, L.es, vb, cudaMemcpyDeviceToDevice, st));
    }
    return DWF_OK;
}

}  // namespace

void level3_free(dwf_mg* h) {
    if (!h || !h->lvl3) return;
    Level3* L = L3(h);
    cudaStreamSynchronize(h->st);
    for (void* p : L->allocs) cudaFree(p);
    if (L->hpin) cudaFreeHost(L->hpin);
    if (L->cg_graph) cudaGraphExecDestroy(L->cg_graph);
    if (L->gcr3_graph) cudaGraphExecDestroy(L->gcr3_graph);
    if (L->cap_stream) cudaStreamDestroy(L->cap_stream);
    delete L;
    h->lvl3 = nullptr;
}

dwf_status level2_solve(dwf_mg* h, const float2* rc, float2* ec, int* l2_iters, int* l3_iters, cudaStream_t st) {
    Level3& L = *L3(h);
    const long long n = L.n2;
    const size_t vb = (size_t)n * sizeof(float2);
    const int g = sgrid(n);
    DWF_CHECK_CUDA(cudaMemcpyAsync(L.r2, rc, vb, cudaMemcpyDeviceToDevice, st));
    DWF_CHECK_CUDA(cudaMemsetAsync(L.e2, 0, vb, st));
    double* r0n = reinterpret_cast<double*>(L.cg) + 32;     // a spare slot after the CGNR scalars
    k_l3_norm<<<g, RED_THREADS, 0, st>>>(L.r2, n, row_rs(L.red_part, L.red_cnt, 0), r0n);
    k_l3_gscal_init<<<1, 1, 0, st>>>(L.g2, r0n, nullptr, L.prm.tol, 1 << 30);
    DWF_CHECK_LAUNCH();
    GScal* hg = reinterpret_cast<GScal*>(reinterpret_cast<char*>(L.hpin) + 256);
    int k = 0, l3 = 0;
    const int K = L.prm.gcr_maxiter;
    for (; k < K; ++k) {
        DWF_CHECK_CUDA(cudaMemcpyAsync(hg, L.g2, sizeof(GScal), cudaMemcpyDeviceToHost, st));
        DWF_CHECK_CUDA(cudaStreamSynchronize(st));
        if (hg->done) break;
        // z_k = M2(r); w_k = Ahat z_k = r - rs (the smoother's residual)
        DWF_TRY(level2_precondition(h, L, L.r2, L.Z[k], &l3, st));
        k_l3_sub<<<g, 256, 0, st>>>(L.W[k], L.r2, L.rs, n);
        DWF_CHECK_LAUNCH();
        DWF_TRY(gcr2_step(L, L.W, L.Z, k, L.W[k], L.Z[k], L.e2, L.r2, L.g2, st));
    }
    DWF_CHECK_CUDA(cudaMemcpyAsync(ec, L.e2, vb, cudaMemcpyDeviceToDevice, st));
    int stat = 0;
    DWF_CHECK_CUDA(cudaMemcpyAsync(&stat, L.status, sizeof(int), cudaMemcpyDeviceToHost, st));
    DWF_CHECK_CUDA(cudaStreamSynchronize(st));
    if (stat) { set_error("level-3 stencil: a bulk copy wait timed out"); return DWF_ERR_TIMEOUT; }
    *l2_iters = k;
    *l3_iters = l3;
    L.last_l2 = k;
    L.last_l3 = l3;
    return DWF_OK;
}

namespace {

// Chebyshev filter p(N) = T_deg(l(N)), l(x) = (2 x - (b + a)) / (b - a): |p| <= 1 on [a, b] and
// |p| grows fast below a, so the low end of spec N becomes the top of spec p(N).  deg = 0: N itself.
struct Filter {
    int deg;
    double a, b;
};

// y = c1 (N x) + c0 x + cm z  (the three-term recurrence of the filter), element-wise
__global__ void k_cheb_step(float2* __restrict__ y, const float2* __restrict__ Nx, const float2* __restrict__ x,
                            const float2* __restrict__ z, float c1, float c0, float cm, long long n) {
    L3_LOOP(e, n) {
        const float2 a = Nx[e], b = x[e];
        float2 r = make_float2(c1 * a.x + c0 * b.x, c1 * a.y + c0 * b.y);
        if (z) { const float2 c = z[e]; r.x += cm * c.x; r.y += cm * c.y; }
        y[e] = r;
    }
}

// out = N in (deg = 0) or p(N) in, with N = A3^dag A3; work vectors x3, rr3, r3, w3, q3, t3
dwf_status apply_filtered(const dwf_mg* h, Level3& L, const Filter& f, const float2* in, float2* out,
                          cudaStream_t st) {
    const long long n = L.n3;
    const int g = sgrid(n);
    auto applyN = [&](const float2* x, float2* y) -> dwf_status {
        DWF_TRY(l3_apply_A(h, L, x, L.q3, L.t3, false, nullptr, st));
        return l3_apply_A(h, L, L.q3, y, L.t3, true, nullptr, st);
    };
    if (f.deg == 0) return applyN(in, out);
    const float c1 = (float)(2.0 / (f.b - f.a)), c0 = (float)(-(f.b + f.a) / (f.b - f.a));
    // y_0 = x, y_1 = l(N) x, y_{j+1} = 2 l(N) y_j - y_{j-1}
    float2* buf[3] = {L.x3, L.rr3, L.r3};
    const float2* prev = in;
    const float2* cur = f.deg == 1 ? out : buf[0];
    DWF_TRY(applyN(in, L.w3));
    k_cheb_step<<<g, 256, 0, st>>>(const_cast<float2*>(cur), L.w3, in, nullptr, c1, c0, 0.f, n);
    DWF_CHECK_LAUNCH();
    for (int j = 1; j < f.deg; ++j) {
        float2* nxt = out;
        if (j + 1 < f.deg)
            for (float2* b : buf)
                if (b != cur && b != prev) { nxt = b; break; }
        DWF_TRY(applyN(cur, L.w3));
        k_cheb_step<<<g, 256, 0, st>>>(nxt, L.w3, cur, prev, 2.f * c1, 2.f * c0, -1.f, n);
        DWF_CHECK_LAUNCH();
        prev = cur;
        cur = nxt;
    }
    return DWF_OK;
}

// p(N) from the fixed buffer b3 to p3v, captured once per filter as one CUDA graph
struct FilterGraph {
    cudaGraphExec_t exec = nullptr;
    ~FilterGraph() { if (exec) cudaGraphExecDestroy(exec); }
};

dwf_status filter_graph(const dwf_mg* h, Level3& L, const Filter& f, FilterGraph& fg) {
    if (fg.exec) { cudaGraphExecDestroy(fg.exec); fg.exec = nullptr; }
    if (!L.cap_stream) DWF_CHECK_CUDA(cudaStreamCreateWithFlags(&L.cap_stream, cudaStreamNonBlocking));
    cudaGraph_t graph = nullptr;
    DWF_CHECK_CUDA(cudaStreamBeginCapture(L.cap_stream, cudaStreamCaptureModeThreadLocal));
    dwf_status s = apply_filtered(h, L, f, L.b3, L.p3v, L.cap_stream);
    cudaError_t e = cudaStreamEndCapture(L.cap_stream, &graph);
    if (s != DWF_OK) { if (graph) cudaGraphDestroy(graph); return s; }
    if (e != cudaSuccess) { set_error("graph capture: %s", cudaGetErrorString(e)); return DWF_ERR_CUDA; }
    e = cudaGraphInstantiate(&fg.exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) { set_error("graph instantiation: %s", cudaGetErrorString(e)); return DWF_ERR_CUDA; }
    return DWF_OK;
}

// Lanczos on the operator of f from `start` (complex128, n3), full reorthogonalisation (two
// classical passes); T = (alpha, beta) of size *m_eff; Q: (m + 1) x n3 FP32
dwf_status lanczos(dwf_mg* h, Level3& L, const Filter& f, const double2* start, int m, float2* Q, double* d_alpha,
                   double* d_beta, int* m_eff, std::vector<double>& ha, std::vector<double>& hb, cudaStream_t st) {
    const long long n = L.n3;
    const size_t vb = (size_t)n * sizeof(float2);
    const int g = sgrid(n);
    FilterGraph fg;
    if (f.deg > 0) DWF_TRY(filter_graph(h, L, f, fg));
    double2* cc = nullptr;
    DWF_CHECK_CUDA(cudaMallocAsync(&cc, sizeof(double2) * 2 * (size_t)(m + 1), st));
    struct Free { void* p; cudaStream_t s; ~Free() { cudaFreeAsync(p, s); } } fr{cc, st};
    double2* c1 = cc;
    double2* c2 = cc + (m + 1);
    k_lz_norm64in<<<1, RED_THREADS, 0, st>>>(start, n, Q);
    DWF_CHECK_LAUNCH();
    ha.clear();
    hb.clear();
    double2 h1, h2;
    double* nrm = reinterpret_cast<double*>(L.cg) + 40;
    double* hn = reinterpret_cast<double*>(reinterpret_cast<char*>(L.hpin) + 2048);
    double anorm = 0.0;
    for (int j = 0; j < m; ++j) {
        const float2* qj = Q + (long long)j * n;
        float2* w = Q + (long long)(j + 1) * n;        // w is built in the next slot
        if (f.deg > 0) {
            DWF_CHECK_CUDA(cudaMemcpyAsync(L.b3, qj, vb, cudaMemcpyDeviceToDevice, st));
            DWF_CHECK_CUDA(cudaGraphLaunch(fg.exec, st));
            DWF_CHECK_CUDA(cudaMemcpyAsync(w, L.p3v, vb, cudaMemcpyDeviceToDevice, st));
        } else {
            DWF_TRY(apply_filtered(h, L, f, qj, w, st));
        }
        k_lz_dots<<<j + 1, RED_THREADS, 0, st>>>(Q, w, n, c1);
        k_lz_sub<<<g, 256, 0, st>>>(Q, c1, j + 1, n, w);
        k_lz_dots<<<j + 1, RED_THREADS, 0, st>>>(Q, w, n, c2);
        k_lz_sub<<<g, 256, 0, st>>>(Q, c2, j + 1, n, w);
        k_l3_norm<<<g, RED_THREADS, 0, st>>>(w, n, row_rs(L.red_part, L.red_cnt, 0), nrm);
        DWF_CHECK_LAUNCH();
        DWF_CHECK_CUDA(cudaMemcpyAsync(&h1, c1 + j, sizeof(double2), cudaMemcpyDeviceToHost, st));
        DWF_CHECK_CUDA(cudaMemcpyAsync(&h2, c2 + j, sizeof(double2), cudaMemcpyDeviceToHost, st));
        DWF_CHECK_CUDA(cudaMemcpyAsync(hn, nrm, sizeof(double), cudaMemcpyDeviceToHost, st));
        DWF_CHECK_CUDA(cudaStreamSynchronize(st));
        const double aj = h1.x + h2.x;
        const double bj = sqrt(*hn);
        ha.push_back(aj);
        anorm = fmax(anorm, fabs(aj) + bj + (hb.empty() ? 0.0 : hb.back()));
        if (!(bj > 1e-10 * anorm) || j + 1 == m) break;      // invariant subspace, or the last step
        hb.push_back(bj);
        k_lz_scale<<<g, 256, 0, st>>>(w, w, n, nrm);
        DWF_CHECK_LAUNCH();
    }
    *m_eff = (int)ha.size();
    hb.resize(ha.size(), 0.0);
    DWF_CHECK_CUDA(cudaMemcpyAsync(d_alpha, ha.data(), sizeof(double) * ha.size(), cudaMemcpyHostToDevice, st));
    DWF_CHECK_CUDA(cudaMemcpyAsync(d_beta, hb.data(), sizeof(double) * hb.size(), cudaMemcpyHostToDevice, st));
    DWF_CHECK_CUDA(cudaStreamSynchronize(st));
    return DWF_OK;
}

// H[i][j] = <V_i, W_j> (k x k, FP64 accumulation), 16 x 16 tiles; chunks of 32 elements staged
// in shared memory
__global__ void __launch_bounds__(256) k_gram(const float2* __restrict__ V, const float2* __restrict__ W, long long n,
                                              int k, double2* __restrict__ H) {
    __shared__ float2 vs[16][33], ws[16][33];
    const int ti = threadIdx.x >> 4, tj = threadIdx.x & 15;
    const int i0 = blockIdx.y * 16, j0 = blockIdx.x * 16;
    double re = 0.0, im = 0.0;
    for (long long e0 = 0; e0 < n; e0 += 32) {
        for (int t = threadIdx.x; t < 16 * 32; t += 256) {
            const int r = t >> 5, c = t & 31;
            const long long e = e0 + c;
            vs[r][c] = (i0 + r < k && e < n) ? V[(long long)(i0 + r) * n + e] : make_float2(0.f, 0.f);
            ws[r][c] = (j0 + r < k && e < n) ? W[(long long)(j0 + r) * n + e] : make_float2(0.f, 0.f);
        }
        __syncthreads();
        float pr = 0.f, pi = 0.f;
#pragma unroll 8
        for (int c = 0; c < 32; ++c) {
            const float2 a = vs[ti][c], b = ws[tj][c];
            pr += a.x * b.x + a.y * b.y;
            pi += a.x * b.y - a.y * b.x;
        }
        re += pr;
        im += pi;
        __syncthreads();
    }
    if (i0 + ti < k && j0 + tj < k) H[(long long)(i0 + ti) * k + j0 + tj] = make_double2(re, im);
}

// H = (H + H^dag) / 2 (the Rayleigh-Ritz matrix of a Hermitian operator, symmetrised)
__global__ void k_herm(double2* __restrict__ H, int k) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= k * k) return;
    const int i = t / k, j = t % k;
    if (j < i) return;
    const double2 a = H[(long long)i * k + j], b = H[(long long)j * k + i];
    const double2 m = make_double2(0.5 * (a.x + b.x), 0.5 * (a.y - b.y));
    H[(long long)i * k + j] = m;
    H[(long long)j * k + i] = make_double2(m.x, -m.y);
}

dwf_status build_deflation(dwf_mg* h, Level3& L, const double2* start, cudaStream_t st) {
    const int want = L.prm.n_deflate;
    if (want <= 0) { L.ndefl = 0; return DWF_OK; }
    const long long n = L.n3;
    int m = L.prm.lanczos_steps;
    if (m < 2 * want) m = 2 * want;
    if (m > n) m = (int)n;
    void* buf = nullptr;
    const size_t qbytes = (size_t)(m + 1) * n * sizeof(float2);
    {
        cudaError_t e = cudaMallocAsync(&buf, qbytes + sizeof(double) * 4 * (size_t)(m + 1) + 256, st);
        if (e != cudaSuccess) { set_error("Lanczos basis (%zu bytes): %s", qbytes, cudaGetErrorString(e)); return DWF_ERR_OOM; }
    }
    struct Free { void* p; cudaStream_t s; ~Free() { cudaFreeAsync(p, s); } } fr{buf, st};
    float2* Q = (float2*)buf;
    double* d_alpha = (double*)((char*)buf + ((qbytes + 255) & ~(size_t)255));
    double* d_beta = d_alpha + (m + 1);
    std::vector<double> ha, hb;
    int meff = 0;
    // the top of spec N from a short plain Lanczos run (extreme Ritz values converge first): the
    // largest Ritz value plus the last residual coefficient bounds lambda_max
    const int m0 = m < 40 ? m : 40;
    DWF_TRY(lanczos(h, L, Filter{0, 0.0, 0.0}, start, m0, Q, d_alpha, d_beta, &meff, ha, hb, st));
    double* lam0 = nullptr;
    double* S0 = nullptr;
    double* scr0 = nullptr;
    DWF_CHECK_CUDA(cudaMallocAsync(&lam0, sizeof(double) * 8, st));
    DWF_CHECK_CUDA(cudaMallocAsync(&S0, sizeof(double) * (size_t)meff, st));
    DWF_CHECK_CUDA(cudaMallocAsync(&scr0, sizeof(double) * 6 * (size_t)meff, st));
    // the largest eigenvalue of T = the smallest of -T
    for (auto& v : ha) v = -v;
    DWF_CHECK_CUDA(cudaMemcpyAsync(d_alpha, ha.data(), sizeof(double) * meff, cudaMemcpyHostToDevice, st));
    k_tridiag_eig<<<1, 32, 0, st>>>(d_alpha, d_beta, meff, 1, lam0, S0, scr0);
    DWF_CHECK_LAUNCH();
    double tmax = 0.0;
    DWF_CHECK_CUDA(cudaMemcpyAsync(&tmax, lam0, sizeof(double), cudaMemcpyDeviceToHost, st));
    DWF_CHECK_CUDA(cudaStreamSynchronize(st));
    cudaFreeAsync(lam0, st);
    cudaFreeAsync(S0, st);
    cudaFreeAsync(scr0, st);
    const bool full = m0 >= n || meff < m0;                    // the short run exhausted the space
    const double bmax = -tmax * 1.05 + (hb.empty() ? 0.0 : hb[meff > 1 ? meff - 2 : 0]);
    // filtered Lanczos: the k largest eigenvalues of p(N) are the k smallest of N; the cut a is
    // raised until the k modes found lie below it
    Filter f{0, 0.0, 0.0};
    double acut = 2e-3 * bmax;
    const int k = want < m ? want : m;
    double *lam = nullptr, *S = nullptr, *scr = nullptr;
    DWF_CHECK_CUDA(cudaMallocAsync(&lam, sizeof(double) * k, st));
    DWF_CHECK_CUDA(cudaMallocAsync(&S, sizeof(double) * (size_t)k * m, st));
    DWF_CHECK_CUDA(cudaMallocAsync(&scr, sizeof(double) * 6 * (size_t)k * m, st));
    struct Free3 { void* a; void* b; void* c; cudaStream_t s;
                   ~Free3() { cudaFreeAsync(a, s); cudaFreeAsync(b, s); cudaFreeAsync(c, s); } } fr3{lam, S, scr, st};
    DWF_TRY(l3_alloc(&L, (void**)&L.Hl, sizeof(double2) * (size_t)k * k));
    DWF_TRY(l3_alloc(&L, (void**)&L.Vd, sizeof(float2) * (size_t)k * n));
    float2* Wd = nullptr;
    DWF_CHECK_CUDA(cudaMallocAsync(&Wd, sizeof(float2) * (size_t)k * n, st));
    struct FreeW { void* p; cudaStream_t s; ~FreeW() { cudaFreeAsync(p, s); } } frw{Wd, st};
    std::vector<double2> Hh((size_t)k * k);
    int kk = k;
    int passes = 0;
    for (int pass = 0; pass < 4; ++pass) {
        ++passes;
        f = full ? Filter{0, 0.0, 0.0} : Filter{L.prm.filter_degree, acut, bmax};
        DWF_TRY(lanczos(h, L, f, start, m, Q, d_alpha, d_beta, &meff, ha, hb, st));
        kk = k < meff ? k : meff;
        // wanted: the largest of T for the filtered operator (the smallest of -T: both the diagonal
        // and the off-diagonal negated, so that the eigenvectors are T's), the smallest for N itself
        if (f.deg > 0) {
            for (auto& v : ha) v = -v;
            for (auto& v : hb) v = -v;
            DWF_CHECK_CUDA(cudaMemcpyAsync(d_alpha, ha.data(), sizeof(double) * meff, cudaMemcpyHostToDevice, st));
            DWF_CHECK_CUDA(cudaMemcpyAsync(d_beta, hb.data(), sizeof(double) * meff, cudaMemcpyHostToDevice, st));
        }
        k_tridiag_eig<<<(kk + 63) / 64, 64, 0, st>>>(d_alpha, d_beta, meff, kk, lam, S, scr);
        k_small_orth<<<1, 256, 0, st>>>(S, meff, kk);
        k_ritz_vectors<<<dim3(sgrid(n), (kk + 15) / 16), 256, 0, st>>>(Q, S, meff, kk, n, L.Vd);
        DWF_CHECK_LAUNCH();
        // Rayleigh-Ritz with N itself: H = V^dag N V
        for (int c = 0; c < kk; ++c)
            DWF_TRY(apply_filtered(h, L, Filter{0, 0.0, 0.0}, L.Vd + (long long)c * n, Wd + (long long)c * n, st));
        k_gram<<<dim3((kk + 15) / 16, (kk + 15) / 16), 256, 0, st>>>(L.Vd, Wd, n, kk, L.Hl);
        k_herm<<<(kk * kk + 255) / 256, 256, 0, st>>>(L.Hl, kk);
        DWF_CHECK_LAUNCH();
        DWF_CHECK_CUDA(cudaMemcpyAsync(Hh.data(), L.Hl, sizeof(double2) * (size_t)kk * kk, cudaMemcpyDeviceToHost, st));
        DWF_CHECK_CUDA(cudaStreamSynchronize(st));
        // the pass is done once every kept mode lies below the cut (each was amplified by the
        // filter); otherwise the cut grows fourfold, at most to a quarter of the top of the spectrum
        int below = 0;
        bool finite = true;
        for (int c = 0; c < kk; ++c) {
            const double rq = Hh[(size_t)c * kk + c].x;
            finite = finite && std::isfinite(rq);
            below += rq <= acut ? 1 : 0;
        }
        if (!finite) { set_error("the deflation setup produced non-finite Rayleigh quotients"); return DWF_ERR_NOCONV; }
        if (f.deg == 0 || below >= kk || pass == 3 || acut >= 0.25 * bmax) break;
        acut = fmin(4.0 * acut, 0.25 * bmax);
    }
    L.filter_passes = passes;
    k_cholesky<<<1, 256, 0, st>>>(L.Hl, kk);
    DWF_CHECK_LAUNCH();
    L.ritz.resize(kk);
    for (int c = 0; c < kk; ++c) L.ritz[c] = Hh[(size_t)c * kk + c].x;
    std::sort(L.ritz.begin(), L.ritz.end());
    L.filter_cut = f.deg > 0 ? acut : 0.0;
    L.filter_top = bmax;
    DWF_CHECK_CUDA(cudaStreamSynchronize(st));
    L.ndefl = kk;
    return DWF_OK;
}

// CG on S S^dag v = 0, S = Dhat_W + shift (level 2, FP64) from v, as relax_null does on the fine level
dwf_status relax_level2(dwf_mg* h, Level3& L, double2* v, double2* r, double2* p, double2* t, double2* Ap, NvState* S,
                        double shift, cudaStream_t st) {
    const long long n = L.V2 * L.ncd2;
    Lat lat;
    lat.nd = 2;
    for (int mu = 0; mu < 4; ++mu) lat.L[mu] = L.L2[mu];
    const int rg = red_grid(n), eg = level_ew_grid(n);
    const unsigned kg = (unsigned)((n + 255) / 256);
    const double tol2 = L.prm.setup_tol * L.prm.setup_tol;
    const int maxit = L.prm.setup_maxiter;
    RedScratch rs = h->ws.red();
    k_kernel64<<<kg, 256, 0, st>>>(h->Y64, v, t, lat, L.V2, L.ncd2, shift, 1);
    k_kernel64<<<kg, 256, 0, st>>>(h->Y64, t, Ap, lat, L.V2, L.ncd2, shift, 0);
    k_nv_init<<<rg, RED_THREADS, 0, st>>>(r, Ap, n, rs, S, maxit);
    DWF_CHECK_CUDA(cudaMemcpyAsync(p, r, n * sizeof(double2), cudaMemcpyDeviceToDevice, st));
    int launched = 0;
    NvState hs;
    for (;;) {
        DWF_CHECK_CUDA(cudaMemcpyAsync(&hs, S, sizeof(NvState), cudaMemcpyDeviceToHost, st));
        DWF_CHECK_CUDA(cudaStreamSynchronize(st));
        if (hs.done || launched >= maxit) break;
        for (int k = 0; k < 16 && launched < maxit; ++k, ++launched) {
            k_kernel64<<<kg, 256, 0, st>>>(h->Y64, p, t, lat, L.V2, L.ncd2, shift, 1);
            k_nv_alpha<<<rg, RED_THREADS, 0, st>>>(t, n, rs, S);
            k_kernel64<<<kg, 256, 0, st>>>(h->Y64, t, Ap, lat, L.V2, L.ncd2, shift, 0);
            k_nv_update<<<rg, RED_THREADS, 0, st>>>(v, r, p, Ap, n, rs, S, tol2, maxit);
            k_nv_p<<<eg, 256, 0, st>>>(p, r, n, S);
            DWF_CHECK_LAUNCH();
        }
    }
    return DWF_OK;
}

dwf_status add_level_impl(dwf_mg* h, Level3& L, const double2* starts, const double2* lstart, cudaStream_t st) {
    const long long n1 = L.V2 * L.ncd2;
    // 1. near-null vectors of the coarse kernel
    DWF_TRY(l3_alloc(&L, (void**)&L.nullv2, sizeof(double2) * L.nvec2 * n1));
    DWF_CHECK_CUDA(cudaMemcpyAsync(L.nullv2, starts, sizeof(double2) * L.nvec2 * n1, cudaMemcpyDeviceToDevice, st));
    if (L.prm.setup_maxiter > 0) {
        void* tmp = nullptr;
        DWF_CHECK_CUDA(cudaMallocAsync(&tmp, 4 * n1 * sizeof(double2) + 256, st));
        struct Free { void* p; cudaStream_t s; ~Free() { cudaFreeAsync(p, s); } } fr{tmp, st};
        double2* r = (double2*)tmp;
        NvState* S = (NvState*)(h->ws.scal + 16);
        const double shift = L.prm.setup_mass + h->M5;
        for (int k = 0; k < L.nvec2; ++k)
            DWF_TRY(relax_level2(h, L, L.nullv2 + k * n1, r, r + n1, r + 2 * n1, r + 3 * n1, S, shift, st));
    }
    // 2. prolongator
    const long long Psz = L.V2 * 2 * L.nvec1 * L.nvec2;
    DWF_TRY(l3_alloc(&L, (void**)&L.P2_64, Psz * sizeof(double2)));
    DWF_TRY(l3_alloc(&L, (void**)&L.P2_32, Psz * sizeof(float2)));
    AggIndex ai;
    ai.nd = 2;
    for (int mu = 0; mu < 4; ++mu) { ai.L[mu] = L.L2[mu]; ai.b[mu] = L.b2[mu]; ai.Lc[mu] = L.L3[mu]; }
    DWF_CHECK_CUDA(cudaMemsetAsync(h->status, 0, sizeof(int), st));
    {
        const size_t sh = (size_t)L.nvec2 * L.nb2 * L.nvec1 * sizeof(double2);
        if (sh > 48 * 1024) DWF_CHECK_CUDA(cudaFuncSetAttribute(k_block_ortho, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh));
        k_block_ortho<<<dim3((unsigned)L.V3, 2), 32, sh, st>>>(L.nullv2, L.P2_64, ai, L.nvec1, 1, L.ncd2, L.nvec2, L.V2,
                                                               L.nb2, h->status, L.nvec1);
        DWF_CHECK_LAUNCH();
    }
    k_d2f<<<level_ew_grid(Psz), 256, 0, st>>>(L.P2_64, L.P2_32, Psz);
    // 3. Galerkin kernel of level 3
    const long long nblk = L.V3 * 5;
    DWF_TRY(l3_alloc(&L, (void**)&L.Y3_64, nblk * L.ncd3 * L.ncd3 * sizeof(double2)));
    k_galerkin_l3<<<dim3((unsigned)L.V3, 5), 256, 0, st>>>(h->Y64, L.P2_64, L.Y3_64, ai, L.nvec1, L.nvec2);
    if (L.prm.block_prec == DWF_F32_L16) {
        DWF_TRY(l3_alloc(&L, (void**)&L.Y3_16, nblk * L.ncd3 * L.ncd3 * sizeof(__half2)));
        k_blocks_to_f16<<<level_ew_grid(nblk * L.ncd3 * L.ncd3), 256, 0, st>>>(L.Y3_64, L.Y3_16, nblk, L.ncd3);
    } else {
        DWF_TRY(l3_alloc(&L, (void**)&L.Y3_32, nblk * L.ncd3 * L.ncd3 * sizeof(float2)));
        k_blocks_to_f32<<<level_ew_grid(nblk * L.ncd3 * L.ncd3), 256, 0, st>>>(L.Y3_64, L.Y3_32, nblk, L.ncd3);
    }
    DWF_CHECK_LAUNCH();
    int hstat = 0;
    DWF_CHECK_CUDA(cudaMemcpyAsync(&hstat, h->status, sizeof(int), cudaMemcpyDeviceToHost, st));
    DWF_CHECK_CUDA(cudaStreamSynchronize(st));
    if (hstat) { set_error("a level-2 near-null vector vanishes on an aggregate: the prolongator is rank deficient");
                 return DWF_ERR_ARG; }
    // solver vectors
    const size_t v2 = (size_t)L.n2 * sizeof(float2), v3 = (size_t)L.n3 * sizeof(float2);
    float2** p2[] = {&L.r2, &L.e2, &L.rs, &L.es, &L.t2, &L.a2};
    for (float2** q : p2) DWF_TRY(l3_alloc(&L, (void**)q, v2));
    for (int k = 0; k < L.prm.gcr_maxiter; ++k) {
        DWF_TRY(l3_alloc(&L, (void**)&L.Z[k], v2));
        DWF_TRY(l3_alloc(&L, (void**)&L.W[k], v2));
    }
    for (int k = 0; k < L.prm.post_smooth; ++k) {
        DWF_TRY(l3_alloc(&L, (void**)&L.Zs[k], v2));
        DWF_TRY(l3_alloc(&L, (void**)&L.Ws[k], v2));
    }
    float2** p3[] = {&L.b3, &L.x3, &L.rr3, &L.r3, &L.p3v, &L.q3, &L.w3, &L.t3};
    for (float2** q : p3) DWF_TRY(l3_alloc(&L, (void**)q, v3));
    DWF_TRY(l3_alloc(&L, (void**)&L.dc, sizeof(double2) * DEFL_MAX));
    if (L.prm.coarsest_solver == 1)
        for (int k = 0; k < L.prm.coarsest_restart; ++k) {
            DWF_TRY(l3_alloc(&L, (void**)&L.Z3[k], v3));
            DWF_TRY(l3_alloc(&L, (void**)&L.W3[k], v3));
        }
    DWF_TRY(l3_alloc(&L, (void**)&L.g3, sizeof(GScal)));
    DWF_TRY(l3_alloc(&L, (void**)&L.g2, sizeof(GScal)));
    DWF_TRY(l3_alloc(&L, (void**)&L.gs, sizeof(GScal)));
    DWF_TRY(l3_alloc(&L, (void**)&L.cg, 1024));
    DWF_TRY(l3_alloc(&L, (void**)&L.red_part, sizeof(double) * PROW3 * (L2_MAXK + 1)));
    DWF_TRY(l3_alloc(&L, (void**)&L.red_cnt, sizeof(unsigned) * CROW3 * (L2_MAXK + 1)));
    DWF_TRY(l3_alloc(&L, (void**)&L.status, 256));
    DWF_CHECK_CUDA(cudaMemsetAsync(L.red_cnt, 0, sizeof(unsigned) * CROW3 * (L2_MAXK + 1), st));
    DWF_CHECK_CUDA(cudaMemsetAsync(L.status, 0, 256, st));
    DWF_CHECK_CUDA(cudaMemsetAsync(L.cg, 0, 1024, st));
    DWF_CHECK_CUDA(cudaMemsetAsync(L.gs, 0, sizeof(GScal), st));
    DWF_CHECK_CUDA(cudaMallocHost(&L.hpin, 4096));
    // 4. deflation
    return build_deflation(h, L, lstart, st);
}

}  // namespace
}  // namespace dwf

using namespace dwf;

extern "C" {

void dwf_mg_default_level_params(dwf_mg_level_params* p) {
    if (!p) return;
    memset(p, 0, sizeof(*p));
    p->nvec = 12;
    p->block[0] = p->block[1] = p->block[2] = p->block[3] = 2;
    p->Ls_c = 4;
    p->setup_maxiter = 250;
    p->setup_tol = 1e-4;
    p->setup_mass = 0.0;
    p->gcr_maxiter = 16;
    p->tol = 0.25;
    p->post_smooth = 8;
    p->coarsest_tol = 0.05;
    p->coarsest_maxiter = 1024;
    p->n_deflate = 128;
    p->lanczos_steps = 256;
    p->filter_degree = 64;
    p->coarsest_solver = 0;
    p->coarsest_restart = 8;
    p->block_prec = DWF_F32;
}

dwf_status mg_add_level(dwf_mg* h, const dwf_mg_level_params* p, const void* null_starts, const void* lanczos_start,
                        void* stream) {
    clear_error();
    if (!h || !null_starts) { set_error("NULL argument"); return DWF_ERR_ARG; }
    if (h->lvl3) { set_error("the hierarchy already has a third level"); return DWF_ERR_ARG; }
    if (h->mg.nd != 2) { set_error("the third level is built for 2-d hierarchies"); return DWF_ERR_UNSUPPORTED; }
    dwf_mg_level_params prm;
    if (p) prm = *p; else dwf_mg_default_level_params(&prm);
    if (prm.n_deflate > 0 && !lanczos_start) { set_error("deflation needs a Lanczos start vector"); return DWF_ERR_ARG; }
    if (prm.nvec < 1 || 2 * prm.nvec * prm.Ls_c > 512 || 2 * prm.nvec < 24 || prm.Ls_c < 1) {
        set_error("the level-3 stencil takes 12 <= nvec with 2 nvec Ls_c <= 512 (nvec %d, Ls_c %d)", prm.nvec,
                  prm.Ls_c);
        return DWF_ERR_ARG;
    }
    if (prm.gcr_maxiter < 1 || prm.gcr_maxiter > L2_MAXK || prm.post_smooth < 0 || prm.post_smooth > L2_MAXK ||
        prm.coarsest_maxiter < 0 || prm.setup_maxiter < 0 || prm.n_deflate < 0 || prm.n_deflate > DEFL_MAX ||
        prm.lanczos_steps < 0 || prm.lanczos_steps > LANCZOS_MAX || prm.filter_degree < 0 ||
        prm.filter_degree > 4096 || !(prm.tol > 0.0) || !(prm.coarsest_tol > 0.0) ||
        (prm.coarsest_solver != 0 && prm.coarsest_solver != 1) || prm.coarsest_restart < 1 ||
        prm.coarsest_restart > L2_MAXK || (prm.block_prec != DWF_F32 && prm.block_prec != DWF_F32_L16)) {
        set_error("bad level parameters");
        return DWF_ERR_ARG;
    }
    Level3* L = new (std::nothrow) Level3();
    if (!L) { set_error("host allocation failed"); return DWF_ERR_OOM; }
    L->prm = prm;
    L->V2 = h->mg.Vc;
    L->V3 = 1;
    L->nb2 = 1;
    for (int mu = 0; mu < 4; ++mu) {
        L->L2[mu] = mu < 2 ? h->mg.Lc[mu] : 1;
        L->b2[mu] = mu < 2 ? prm.block[mu] : 1;
        if (L->b2[mu] < 1 || L->L2[mu] % L->b2[mu]) {
            set_error("block[%d] = %d must divide the coarse extent %d", mu, L->b2[mu], L->L2[mu]);
            delete L;
            return DWF_ERR_ARG;
        }
        L->L3[mu] = L->L2[mu] / L->b2[mu];
        L->V3 *= L->L3[mu];
        L->nb2 *= L->b2[mu];
    }
    L->nvec1 = h->mg.nvec;
    L->ncd2 = h->mg.ncd;
    L->nvec2 = prm.nvec;
    L->ncd3 = 2 * prm.nvec;
    L->Ls2 = h->mg.Ls_c;
    L->Ls3 = prm.Ls_c;
    L->n2 = L->V2 * L->Ls2 * L->ncd2;
    L->n3 = L->V3 * L->Ls3 * L->ncd3;
    if ((long long)L->nb2 * L->nvec1 < L->nvec2) {
        set_error("aggregates of %lld dof per chirality cannot hold %d orthonormal vectors",
                  (long long)L->nb2 * L->nvec1, L->nvec2);
        delete L;
        return DWF_ERR_ARG;
    }
    L->p3.Vc = L->V3;
    L->p3.nd = 2;
    for (int mu = 0; mu < 4; ++mu) L->p3.Lc[mu] = L->L3[mu];
    L->p3.Ls_c = L->Ls3;
    L->p3.ncd = L->ncd3;
    L->p3.nvec = L->nvec2;
    L->p3.ndir = 5;
    L->p3.mf = (float)h->mf;
    h->lvl3 = L;
    cudaStream_t st = stream ? as_stream(stream) : h->st;
    dwf_status s = add_level_impl(h, *L, (const double2*)null_starts, (const double2*)lanczos_start, st);
    if (s != DWF_OK) {
        std::string msg = dwf_last_error();
        level3_free(h);
        set_error("%s", msg.c_str());
    }
    return s;
}

dwf_status mg_level_geom(const dwf_mg* h, dwf_geom* c, int* ncdof) {
    clear_error();
    if (!h || !c) { set_error("NULL argument"); return DWF_ERR_ARG; }
    if (!h->lvl3) { set_error("the hierarchy has no third level"); return DWF_ERR_ARG; }
    const Level3& L = *L3(h);
    memset(c, 0, sizeof(*c));
    c->nd = 2;
    c->L[0] = L.L3[0];
    c->L[1] = L.L3[1];
    c->Ls = L.Ls3;
    c->group = h->G.group;
    if (ncdof) *ncdof = L.ncd3;
    return DWF_OK;
}

dwf_status mg_level_get(const dwf_mg* h, int what, void* out, void* stream) {
    clear_error();
    if (!h || !out) { set_error("NULL argument"); return DWF_ERR_ARG; }
    if (!h->lvl3) { set_error("the hierarchy has no third level"); return DWF_ERR_ARG; }
    const Level3& L = *L3(h);
    cudaStream_t st = as_stream(stream);
    const void* src = nullptr;
    size_t bytes = 0;
    if (what == 0) { src = L.nullv2; bytes = sizeof(double2) * L.nvec2 * L.V2 * L.ncd2; }
    else if (what == 1) { src = L.P2_64; bytes = sizeof(double2) * L.V2 * 2 * L.nvec1 * L.nvec2; }
    else if (what == 2) { src = L.Y3_64; bytes = sizeof(double2) * L.V3 * 5 * L.ncd3 * L.ncd3; }
    else { set_error("what must be 0, 1 or 2"); return DWF_ERR_ARG; }
    DWF_CHECK_CUDA(cudaMemcpyAsync(out, src, bytes, cudaMemcpyDeviceToDevice, st));
    return DWF_OK;
}

dwf_status mg_level_apply(const dwf_mg* h, const void* in, void* out, double mf, int dagger, void* stream) {
    clear_error();
    if (!h || !in || !out) { set_error("NULL argument"); return DWF_ERR_ARG; }
    if (!h->lvl3) { set_error("the hierarchy has no third level"); return DWF_ERR_ARG; }
    if (in == out) { set_error("in and out must be distinct buffers"); return DWF_ERR_ARG; }
    return l3_apply(*L3(h), (const float2*)in, (float2*)out, mf, dagger != 0, nullptr, as_stream(stream));
}

dwf_status mg_level_restrict(const dwf_mg* h, const void* r2, void* r3, void* stream) {
    clear_error();
    if (!h || !r2 || !r3) { set_error("NULL argument"); return DWF_ERR_ARG; }
    if (!h->lvl3) { set_error("the hierarchy has no third level"); return DWF_ERR_ARG; }
    const Level3& L = *L3(h);
    k_restrict23<<<(unsigned)((L.n3 + 255) / 256), 256, 0, as_stream(stream)>>>(L.P2_32, (const float2*)r2,
                                                                                  (float2*)r3, xfer_params(L));
    DWF_CHECK_LAUNCH();
    return DWF_OK;
}

dwf_status mg_level_prolong(const dwf_mg* h, const void* e3, void* e2, void* stream) {
    clear_error();
    if (!h || !e3 || !e2) { set_error("NULL argument"); return DWF_ERR_ARG; }
    if (!h->lvl3) { set_error("the hierarchy has no third level"); return DWF_ERR_ARG; }
    const Level3& L = *L3(h);
    k_prolong23<<<(unsigned)((L.n2 + 255) / 256), 256, 0, as_stream(stream)>>>(L.P2_32, (const float2*)e3,
                                                                                 (float2*)e2, xfer_params(L));
    DWF_CHECK_LAUNCH();
    return DWF_OK;
}

dwf_status mg_level_coarsest_solve(dwf_mg* h, const void* b3, void* x3, double tol, int maxiter, int deflate,
                                   int* iters, void* stream) {
    clear_error();
    if (!h || !b3 || !x3) { set_error("NULL argument"); return DWF_ERR_ARG; }
    if (!h->lvl3) { set_error("the hierarchy has no third level"); return DWF_ERR_ARG; }
    if (!(tol > 0.0) || maxiter < 0) { set_error("bad tolerance or iteration cap"); return DWF_ERR_ARG; }
    int it = 0;
    DWF_TRY(level3_solve_impl(h, *L3(h), (const float2*)b3, (float2*)x3, tol, maxiter, deflate != 0, &it,
                              as_stream(stream)));
    if (iters) *iters = it;
    return DWF_OK;
}

int mg_level_ritz_values(const dwf_mg* h, double* out, int cap) {
    if (!h || !h->lvl3) return 0;
    const Level3& L = *L3(h);
    const int k = (int)L.ritz.size();
    for (int i = 0; i < k && i < cap && out; ++i) out[i] = L.ritz[i];
    return k;
}

dwf_status mg_level_deflation_info(const dwf_mg* h, double* info) {
    clear_error();
    if (!h || !h->lvl3 || !info) { set_error("NULL argument or no third level"); return DWF_ERR_ARG; }
    const Level3& L = *L3(h);
    info[0] = L.ndefl;
    info[1] = L.filter_cut;
    info[2] = L.filter_top;
    info[3] = L.filter_passes;
    return DWF_OK;
}

dwf_status mg_level_last_iterations(const dwf_mg* h, int* l2_iters, int* l3_iters) {
    clear_error();
    if (!h || !h->lvl3) { set_error("the hierarchy has no third level"); return DWF_ERR_ARG; }
    if (l2_iters) *l2_iters = L3(h)->last_l2;
    if (l3_iters) *l3_iters = L3(h)->last_l3;
    return DWF_OK;
}

}  // extern "C"
