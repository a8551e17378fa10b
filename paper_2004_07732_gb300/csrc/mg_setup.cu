// Multigrid setup (Sec. 2.3 and Sec. 3, Table kcycle), all on the GPU in FP64:
//   1. near-null vectors: CG on the homogeneous system D_W(m) D_W(m)^dag v = 0
//      from caller-supplied Gaussian starts (at most setup_maxiter steps or a
//      residual reduction setup_tol);
//   2. chiral doubling and block orthonormalisation: per aggregate and
//      chirality, Gram-Schmidt of the vectors' P_+ / P_- halves (applied twice
//      for stability), giving a prolongator with gamma_5 P = P sigma_3 and
//      P^dag P = 1 (Eq. gamma5);
//   3. the Galerkin kernel Dhat_W = P^dag D_W(-M5) P, one (2 nvec)^2 block per
//      coarse site for the self term and each of the 2d hop directions.
#include <chrono>
#include <new>
#include <string>
#include <string.h>

#include "mg.cuh"

namespace dwf {

// ---------------------------------------------------------------------------
// 1. near-null relaxation: FP64 CG kernels with a device-side stop flag
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(RED_THREADS) k_nv_init(double2* __restrict__ r, const double2* __restrict__ Av, long long n,
                                                         RedScratch rs, NvState* S, int maxiter) {
    double v[1] = {0.0};
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        double2 a = Av[i];
        r[i] = make_double2(-a.x, -a.y);
        v[0] += a.x * a.x + a.y * a.y;
    }
    grid_reduce<1>(v, rs, [=] __device__(double* t) {
        S->rr = t[0]; S->rr0 = t[0]; S->iters = 0;
        S->done = (t[0] == 0.0 || maxiter <= 0) ? 1 : 0;
    });
}

__global__ void __launch_bounds__(RED_THREADS) k_nv_alpha(const double2* __restrict__ t, long long n, RedScratch rs, NvState* S) {
    if (S->done) return;
    double v[1] = {0.0};
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        double2 a = t[i];
        v[0] += a.x * a.x + a.y * a.y;
    }
    grid_reduce<1>(v, rs, [=] __device__(double* tt) {
        if (tt[0] > 0.0) S->alpha = S->rr / tt[0];
        else { S->alpha = 0.0; S->done = 1; }
    });
}

__global__ void __launch_bounds__(RED_THREADS) k_nv_update(double2* __restrict__ x, double2* __restrict__ r, const double2* __restrict__ p,
                                                           const double2* __restrict__ Ap, long long n, RedScratch rs, NvState* S,
                                                           double tol2, int maxiter) {
    if (S->done) return;
    const double a = S->alpha;
    double v[1] = {0.0};
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        double2 pi = p[i], qi = Ap[i], xi = x[i], ri = r[i];
        xi.x += a * pi.x; xi.y += a * pi.y;
        ri.x -= a * qi.x; ri.y -= a * qi.y;
        x[i] = xi; r[i] = ri;
        v[0] += ri.x * ri.x + ri.y * ri.y;
    }
    grid_reduce<1>(v, rs, [=] __device__(double* t) {
        S->beta = S->rr > 0.0 ? t[0] / S->rr : 0.0;
        S->rr = t[0];
        S->iters += 1;
        if (t[0] <= tol2 * S->rr0 || S->iters >= maxiter) S->done = 1;
    });
}

__global__ void k_nv_p(double2* __restrict__ p, const double2* __restrict__ r, long long n, const NvState* S) {
    if (S->done) return;
    const double b = S->beta;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        double2 pi = p[i], ri = r[i];
        p[i] = make_double2(ri.x + b * pi.x, ri.y + b * pi.y);
    }
}

static int ew_grid(long long n) {
    long long b = (n + 255) / 256;
    return (int)(b < 152LL * 8 ? b : 152LL * 8);
}

// CG on D_W(m) D_W(m)^dag v = 0 in place on v (d-dim, FP64).  D_W(m) is the
// Ls = 1 domain-wall apply with wall mass 1 and height -m (diagonal d + m).
static dwf_status relax_null(dwf_mg* h, double2* v, double2* r, double2* p, double2* t, double2* Ap, NvState* S,
                             int* iters_out) {
    Geom W = h->G;
    W.Ls = 1;
    const long long n = W.V * site_dof(W);
    const double M5w = -h->prm.setup_mass;
    cudaStream_t st = h->st;
    const int rg = red_grid(n), eg = ew_grid(n);
    const double tol2 = h->prm.setup_tol * h->prm.setup_tol;
    const int maxit = h->prm.setup_maxiter;
    DWF_TRY(fine_apply(W, h->U64, v, t, M5w, 1.0, true, DWF_F64, st));
    DWF_TRY(fine_apply(W, h->U64, t, Ap, M5w, 1.0, false, DWF_F64, st));
    k_nv_init<<<rg, RED_THREADS, 0, st>>>(r, Ap, n, h->ws.red(), S, maxit);
    DWF_CHECK_CUDA(cudaMemcpyAsync(p, r, n * sizeof(double2), cudaMemcpyDeviceToDevice, st));
    int launched = 0;
    NvState hs;
    for (;;) {
        DWF_CHECK_CUDA(cudaMemcpyAsync(&hs, S, sizeof(NvState), cudaMemcpyDeviceToHost, st));
        DWF_CHECK_CUDA(cudaStreamSynchronize(st));
        if (hs.done || launched >= maxit) break;
        const int batch = 16;
        for (int k = 0; k < batch && launched < maxit; ++k, ++launched) {
            DWF_TRY(fine_apply(W, h->U64, p, t, M5w, 1.0, true, DWF_F64, st));
            k_nv_alpha<<<rg, RED_THREADS, 0, st>>>(t, n, h->ws.red(), S);
            DWF_TRY(fine_apply(W, h->U64, t, Ap, M5w, 1.0, false, DWF_F64, st));
            k_nv_update<<<rg, RED_THREADS, 0, st>>>(v, r, p, Ap, n, h->ws.red(), S, tol2, maxit);
            k_nv_p<<<eg, 256, 0, st>>>(p, r, n, S);
            DWF_CHECK_LAUNCH();
        }
    }
    *iters_out = hs.iters;
    return DWF_OK;
}

// ---------------------------------------------------------------------------
// 2. chiral doubling + block Gram-Schmidt
// ---------------------------------------------------------------------------
// fine dof index within a site of chirality c, chirality-local index l
__host__ __device__ __forceinline__ int chiral_dof(int nd, int ncol, int c, int l) {
    if (nd == 2) return c;                        // spin c, one colour
    return (2 * c + l / ncol) * ncol + l % ncol;  // spins 2c, 2c+1; colours
}

// One warp per (aggregate, chirality): Gram-Schmidt (twice) of the nvec
// vectors' chirality-c halves restricted to the aggregate.  cblock = 0: fine
// sites (spin / colour dof, chirality from gamma_5); cblock > 0: coarse sites
// whose dof are [chirality][cblock] (chirality from sigma_3).
__global__ void k_block_ortho(const double2* __restrict__ vecs, double2* __restrict__ P, AggIndex ai, int nchd,
                              int ncol, int dof, int nvec, long long V, int nb, int* status, int cblock) {
    extern __shared__ double2 smem[];   // [nvec][nb*nchd]
    const long long xc = blockIdx.x;
    const int c = blockIdx.y;
    const int lane = threadIdx.x;
    const int na = nb * nchd;
    for (int k = 0; k < nvec; ++k)
        for (int e = lane; e < na; e += 32) {
            int l = e / nchd, cd = e % nchd;
            long long site = ai.fine_site(xc, l);
            smem[k * na + e] = vecs[(long long)k * V * dof + site * dof +
                                    (cblock ? c * cblock + cd : chiral_dof(ai.nd, ncol, c, cd))];
        }
    __syncwarp();
    for (int k = 0; k < nvec; ++k) {
        double2* vk = smem + k * na;
        for (int pass = 0; pass < 2; ++pass) {
            for (int j = 0; j < k; ++j) {
                const double2* vj = smem + j * na;
                double re = 0.0, im = 0.0;
                for (int e = lane; e < na; e += 32) {
                    double2 a = vj[e], b = vk[e];
                    re += a.x * b.x + a.y * b.y;
                    im += a.x * b.y - a.y * b.x;
                }
                for (int off = 16; off > 0; off >>= 1) {
                    re += __shfl_xor_sync(0xffffffffu, re, off);
                    im += __shfl_xor_sync(0xffffffffu, im, off);
                }
                for (int e = lane; e < na; e += 32) {
                    double2 a = vj[e], b = vk[e];
                    b.x -= re * a.x - im * a.y;
                    b.y -= re * a.y + im * a.x;
                    vk[e] = b;
                }
                __syncwarp();
            }
        }
        double nn = 0.0;
        for (int e = lane; e < na; e += 32) nn += vk[e].x * vk[e].x + vk[e].y * vk[e].y;
        for (int off = 16; off > 0; off >>= 1) nn += __shfl_xor_sync(0xffffffffu, nn, off);
        if (!(nn > 0.0)) {
            if (lane == 0) atomicExch(status, 1);
            nn = 1.0;
        }
        const double inv = 1.0 / sqrt(nn);
        for (int e = lane; e < na; e += 32) { vk[e].x *= inv; vk[e].y *= inv; }
        __syncwarp();
    }
    for (int k = 0; k < nvec; ++k)
        for (int e = lane; e < na; e += 32) {
            int l = e / nchd, cd = e % nchd;
            long long site = ai.fine_site(xc, l);
            P[((site * 2 + c) * nchd + cd) * nvec + k] = smem[k * na + e];
        }
}

// ---------------------------------------------------------------------------
// 3. Galerkin kernel Dhat_W = P^dag D_W P, 2-d U(1)
// ---------------------------------------------------------------------------
// (1 + sgn gamma_mu)[a][b] in the 2-d basis gamma_1 = sigma_1, gamma_2 = sigma_2
__device__ __forceinline__ double2 spin2(int mu, int sgn, int a, int b) {
    if (a == b) return make_double2(1.0, 0.0);
    if (mu == 0) return make_double2((double)sgn, 0.0);
    // gamma_2 = [[0, -i], [i, 0]]
    return (a == 0) ? make_double2(0.0, -(double)sgn) : make_double2(0.0, (double)sgn);
}

__global__ void k_galerkin_2d(const double2* __restrict__ U, const double2* __restrict__ P, double2* __restrict__ Y,
                              AggIndex ai, int nvec, long long V, double diag, int anti0, int anti1) {
    const long long xc = blockIdx.x;
    const int dir = blockIdx.y;         // 0 self, 1 +0, 2 -0, 3 +1, 4 -1
    const int ncd = 2 * nvec;
    const int nb = ai.b[0] * ai.b[1];
    const int L0 = ai.L[0], L1 = ai.L[1];
    for (int e = threadIdx.x; e < ncd * ncd; e += blockDim.x) {
        const int i = e / ncd, j = e % ncd;
        const int ci = i / nvec, ki = i % nvec, cj = j / nvec, kj = j % nvec;
        double sre = 0.0, sim = 0.0;
        for (int l = 0; l < nb; ++l) {
            const long long x = ai.fine_site(xc, l);
            const int x0 = (int)(x % L0), x1 = (int)(x / L0);
            const int l0 = x0 % ai.b[0], l1 = x1 % ai.b[1];
            const double2 pxi = P[(x * 2 + ci) * nvec + ki];
            // sum over terms feeding (x -> y) for this block
            for (int term = 0; term < 5; ++term) {
                double2 coef;      // spin entry [ci][cj] times link, including -1/2 and phases
                long long y;
                if (term == 0) {
                    if (dir != 0 || ci != cj) continue;
                    coef = make_double2(diag, 0.0);
                    y = x;
                } else {
                    const int mu = (term - 1) / 2;
                    const int fwd = ((term - 1) % 2) == 0;
                    const int lc = mu == 0 ? l0 : l1;
                    const int bm = ai.b[mu];
                    const bool crosses = fwd ? (lc == bm - 1) : (lc == 0);
                    const int want_dir = crosses ? (1 + 2 * mu + (fwd ? 0 : 1)) : 0;
                    if (want_dir != dir) continue;
                    int y0 = x0, y1 = x1;
                    bool wrap;
                    if (mu == 0) { y0 = fwd ? x0 + 1 : x0 - 1; wrap = (y0 < 0 || y0 >= L0); y0 = (y0 + L0) % L0; }
                    else         { y1 = fwd ? x1 + 1 : x1 - 1; wrap = (y1 < 0 || y1 >= L1); y1 = (y1 + L1) % L1; }
                    y = (long long)y1 * L0 + y0;
                    const double ph = (wrap && (mu == 0 ? anti0 : anti1)) ? -1.0 : 1.0;
                    double2 u = fwd ? U[mu * V + x] : U[mu * V + y];
                    if (!fwd) u.y = -u.y;                          // U_mu(x - mu)^*
                    const double2 sm = spin2(mu, fwd ? -1 : 1, ci, cj);
                    coef = make_double2(-0.5 * ph * (sm.x * u.x - sm.y * u.y), -0.5 * ph * (sm.x * u.y + sm.y * u.x));
                }
                const double2 pyj = P[(y * 2 + cj) * nvec + kj];
                // conj(pxi) * coef * pyj
                const double ar = pxi.x * coef.x + pxi.y * coef.y, ai_ = pxi.x * coef.y - pxi.y * coef.x;
                sre += ar * pyj.x - ai_ * pyj.y;
                sim += ar * pyj.y + ai_ * pyj.x;
            }
        }
        Y[(xc * 5 + dir) * (long long)(ncd * ncd) + (long long)i * ncd + j] = make_double2(sre, sim);
    }
}

// ---------------------------------------------------------------------------
// 3'. Galerkin kernel Dhat_W = P^dag D_W P, 4-d SU(3), FP32 arithmetic
// ---------------------------------------------------------------------------
// gamma_mu in the chiral basis: [[0, A_mu], [A_mu^dag, 0]] with A = -i sigma_1,
// -i sigma_2, -i sigma_3, 1 (the basis of the fine 4-d operator)
__device__ __forceinline__ float2 amat(int mu, int r, int c) {   // A_mu[r][c], r, c in {0, 1}
    if (mu == 0) return r != c ? make_float2(0.f, -1.f) : make_float2(0.f, 0.f);          // -i sigma_1
    if (mu == 1) return (r == 0 && c == 1) ? make_float2(-1.f, 0.f)
                        : (r == 1 && c == 0) ? make_float2(1.f, 0.f) : make_float2(0.f, 0.f);  // -i sigma_2
    if (mu == 2) return r != c ? make_float2(0.f, 0.f) : make_float2(0.f, r == 0 ? -1.f : 1.f); // -i sigma_3
    return r == c ? make_float2(1.f, 0.f) : make_float2(0.f, 0.f);
}
__device__ __forceinline__ float2 gamma4(int mu, int a, int b) {
    if (a < 2 && b >= 2) return amat(mu, a, b - 2);
    if (a >= 2 && b < 2) { const float2 A = amat(mu, b, a - 2); return make_float2(A.x, -A.y); }
    return make_float2(0.f, 0.f);
}

constexpr int GAL4_THREADS = 256;
constexpr int GAL4_MAXE = 16;           // Y entries per thread: ncd^2 <= 16 * 256 (ncd <= 64)

// One block per (coarse site, direction): Y_dir = sum_x P(x)^dag Q(x) with
// Q(x) = sum over the hops from x that land in the aggregate of xc + dir (and
// the diagonal for dir 0) of D_W(x, y) P(y).  P(x) is 12 x ncd, block diagonal
// in chirality (rows of spins 2c, 2c+1 feed columns c*nvec ...).
__global__ void __launch_bounds__(GAL4_THREADS) k_galerkin_4d(const double2* __restrict__ U,
                                                              const float2* __restrict__ P, double2* __restrict__ Y,
                                                              AggIndex ai, int nvec, long long V, float diag,
                                                              int4 anti) {
    extern __shared__ float2 g4sm[];
    const int ncd = 2 * nvec;
    float2* Py = g4sm;                  // [12][nvec]: rows of the fine dof, columns of that row's chirality
    float2* Px = Py + 12 * nvec;        // [12][nvec]
    float2* Q = Px + 12 * nvec;         // [12][ncd]
    __shared__ float Ul[9][2];
    const long long xc = blockIdx.x;
    const int dir = blockIdx.y;
    const int nb = ai.b[0] * ai.b[1] * ai.b[2] * ai.b[3];
    const int nent = ncd * ncd;
    float2 acc[GAL4_MAXE];
#pragma unroll
    for (int u = 0; u < GAL4_MAXE; ++u) acc[u] = make_float2(0.f, 0.f);
    const int anti_[4] = {anti.x, anti.y, anti.z, anti.w};
    for (int l = 0; l < nb; ++l) {
        const long long x = ai.fine_site(xc, l);
        int xcrd[4];
        {
            long long rem = x;
            for (int mu = 0; mu < 4; ++mu) { xcrd[mu] = (int)(rem % ai.L[mu]); rem /= ai.L[mu]; }
        }
        for (int e = threadIdx.x; e < 12 * ncd; e += blockDim.x) Q[e] = make_float2(0.f, 0.f);
        bool any = false;
        for (int term = 0; term < 9; ++term) {
            long long y = x;
            int mu = 0, fwd = 1;
            float ph = 1.f;
            if (term == 0) {
                if (dir != 0) continue;
            } else {
                mu = (term - 1) / 2;
                fwd = ((term - 1) % 2) == 0;
                const int lc = xcrd[mu] % ai.b[mu];
                const bool crosses = fwd ? (lc == ai.b[mu] - 1) : (lc == 0);
                const int want = crosses ? (1 + 2 * mu + (fwd ? 0 : 1)) : 0;
                if (want != dir) continue;
                int ycrd[4] = {xcrd[0], xcrd[1], xcrd[2], xcrd[3]};
                ycrd[mu] += fwd ? 1 : -1;
                const bool wrap = ycrd[mu] < 0 || ycrd[mu] >= ai.L[mu];
                ycrd[mu] = (ycrd[mu] + ai.L[mu]) % ai.L[mu];
                y = 0;
                long long st = 1;
                for (int nu = 0; nu < 4; ++nu) { y += ycrd[nu] * st; st *= ai.L[nu]; }
                if (wrap && anti_[mu]) ph = -1.f;
            }
            any = true;
            __syncthreads();                       // previous term's Py / Ul fully used
            for (int e = threadIdx.x; e < 12 * nvec; e += blockDim.x) {
                const int d = e / nvec, k = e % nvec;
                const int sp = d / 3, c = sp / 2, lch = (sp % 2) * 3 + d % 3;
                Py[e] = P[((y * 2 + c) * 6 + lch) * nvec + k];
            }
            if (term > 0 && threadIdx.x < 9) {
                const int a = threadIdx.x / 3, b = threadIdx.x % 3;
                // forward: U_mu(x)[a][b]; backward: U_mu(y)^dag[a][b] = conj(U_mu(y)[b][a])
                const double2 u = fwd ? U[((long long)mu * V + x) * 9 + a * 3 + b] : U[((long long)mu * V + y) * 9 + b * 3 + a];
                Ul[threadIdx.x][0] = (float)u.x;
                Ul[threadIdx.x][1] = fwd ? (float)u.y : -(float)u.y;
            }
            __syncthreads();
            // Q[a][j] += sum_{b: chirality of column j} D[a][b] Py[b][kj]
            for (int e = threadIdx.x; e < 12 * ncd; e += blockDim.x) {
                const int a = e / ncd, j = e % ncd;
                const int cj = j / nvec, kj = j % nvec;
                const int sa = a / 3, ca = a % 3;
                float2 q = Q[e];
                for (int bl = 0; bl < 6; ++bl) {
                    const int sb = 2 * cj + bl / 3, cb = bl % 3, b = sb * 3 + cb;
                    float2 dab;
                    if (term == 0) {
                        if (b != a) continue;
                        dab = make_float2(diag, 0.f);
                    } else {
                        // -1/2 ph (1 -+ gamma_mu)[sa][sb] U[ca][cb]   (- for forward)
                        float2 sg = gamma4(mu, sa, sb);
                        const float sgn = fwd ? -1.f : 1.f;
                        float2 spin = make_float2((sa == sb ? 1.f : 0.f) + sgn * sg.x, sgn * sg.y);
                        if (spin.x == 0.f && spin.y == 0.f) continue;
                        const float ur = Ul[ca * 3 + cb][0], ui = Ul[ca * 3 + cb][1];
                        dab = make_float2(-0.5f * ph * (spin.x * ur - spin.y * ui), -0.5f * ph * (spin.x * ui + spin.y * ur));
                    }
                    const float2 pv = Py[b * nvec + kj];
                    q.x += dab.x * pv.x - dab.y * pv.y;
                    q.y += dab.x * pv.y + dab.y * pv.x;
                }
                Q[e] = q;
            }
        }
        if (!any) continue;                        // uniform over the block
        __syncthreads();
        for (int e = threadIdx.x; e < 12 * nvec; e += blockDim.x) {
            const int d = e / nvec, k = e % nvec;
            const int sp = d / 3, c = sp / 2, lch = (sp % 2) * 3 + d % 3;
            Px[e] = P[((x * 2 + c) * 6 + lch) * nvec + k];
        }
        __syncthreads();
        // Y[i][j] += sum_{a in chirality ci} conj(Px[a][ki]) Q[a][j]
#pragma unroll
        for (int u = 0; u < GAL4_MAXE; ++u) {
            const int e = threadIdx.x + u * GAL4_THREADS;
            if (e < nent) {
                const int i = e / ncd, j = e % ncd;
                const int ci = i / nvec, ki = i % nvec;
                float2 s = acc[u];
                for (int al = 0; al < 6; ++al) {
                    const int a = (2 * ci + al / 3) * 3 + al % 3;
                    const float2 pv = Px[a * nvec + ki], qv = Q[a * ncd + j];
                    s.x += pv.x * qv.x + pv.y * qv.y;
                    s.y += pv.x * qv.y - pv.y * qv.x;
                }
                acc[u] = s;
            }
        }
        __syncthreads();                           // Q and Px are rewritten by the next site
    }
#pragma unroll
    for (int u = 0; u < GAL4_MAXE; ++u) {
        const int e = threadIdx.x + u * GAL4_THREADS;
        if (e < nent) Y[((long long)xc * 9 + dir) * nent + e] = make_double2(acc[u].x, acc[u].y);
    }
}

__global__ void k_blocks_to_f32(const double2* __restrict__ Y, float2* __restrict__ Y32, long long nblocks, int ncd) {
    const long long n = nblocks * ncd * ncd;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
        const long long blk = t / (ncd * ncd);
        const int e = (int)(t % (ncd * ncd));
        const int i = e / ncd, j = e % ncd;            // row-major source
        double2 v = Y[t];
        Y32[blk * ncd * ncd + (long long)j * ncd + i] = make_float2((float)v.x, (float)v.y);
    }
}

__global__ void k_blocks_to_f16(const double2* __restrict__ Y, __half2* __restrict__ Y16, long long nblocks, int ncd) {
    const long long n = nblocks * ncd * ncd;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
        const long long blk = t / (ncd * ncd);
        const int e = (int)(t % (ncd * ncd));
        const int i = e / ncd, j = e % ncd;            // row-major source
        const double2 v = Y[t];
        Y16[blk * ncd * ncd + (long long)j * ncd + i] = __halves2half2(__double2half(v.x), __double2half(v.y));
    }
}

// Blocks of the 48-dof coarse operator in the fragment order of k_coarse_mma:
// the real form A = [Re Y; Im Y] (96 x 48) of each direction's block, cut in
// 6 row tiles of 16 and 6 column tiles of 8.  Per coarse site, direction d,
// column-tile pair kp and row tile mt, lane l = 4 g + t holds eight halves: the
// m16n8k8 A fragment {A(g, t), A(g + 8, t), A(g, t + 4), A(g + 8, t + 4)} of
// column tile 2 kp, then that of column tile 2 kp + 1.  FP16 rounding as in
// k_blocks_to_f16.
__global__ void k_blocks_to_mma(const double2* __restrict__ Y, __half* __restrict__ Ym, long long nsites) {
    constexpr int per_site = 9 * 3 * 6 * 32 * 8;
    const long long n = nsites * per_site;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
        const long long site = t / per_site;
        const int r = (int)(t % per_site);
        const int e = r & 7, lane = (r >> 3) & 31, f = r >> 8;     // f = (dir 3 + kp) 6 + mt
        const int mt = f % 6, kp = (f / 6) % 3, dir = f / 18;
        const int g = lane >> 2, tq = lane & 3, kt = 2 * kp + (e >> 2), q = e & 3;
        const int row = mt * 16 + g + ((q & 1) ? 8 : 0);
        const int col = kt * 8 + tq + ((q & 2) ? 4 : 0);
        const double2 v = Y[((site * 9 + dir) * 48 + row % 48) * 48 + col];
        Ym[t] = __double2half(row < 48 ? v.x : v.y);
    }
}

// *differ = 1 if any complex value of a and b differs bitwise
__global__ void k_links_differ(const double2* __restrict__ a, const double2* __restrict__ b, long long n, int* differ) {
    bool d = false;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
        const double2 u = a[t], v = b[t];
        d = d || __double_as_longlong(u.x) != __double_as_longlong(v.x) ||
            __double_as_longlong(u.y) != __double_as_longlong(v.y);
    }
    if (__any_sync(0xffffffffu, d) && (threadIdx.x & 31) == 0) atomicExch(differ, 1);
}

__global__ void k_d2f(const double2* __restrict__ a, float2* __restrict__ b, long long n) {
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x)
        b[t] = make_float2((float)a[t].x, (float)a[t].y);
}

dwf_status mg_alloc(dwf_mg* h, void** p, size_t bytes) {
    cudaError_t e = cudaMalloc(p, bytes < 256 ? 256 : bytes);
    if (e != cudaSuccess) {
        set_error("multigrid allocation of %zu bytes failed: %s", bytes, cudaGetErrorString(e));
        *p = nullptr;
        return DWF_ERR_OOM;
    }
    h->allocs.push_back(*p);
    return DWF_OK;
}

static dwf_status setup_impl(dwf_mg* h, const void* U, const void* starts) {
    const MgGeom& m = h->mg;
    const Geom& G = h->G;
    cudaStream_t st = h->st;
    const long long dof = site_dof(G);
    const long long n1 = G.V * dof;     // one d-dim vector
    DWF_TRY(h->ws.reserve(st));
    DWF_TRY(mg_alloc(h, &h->U64, link_len(G) * sizeof(double2)));
    DWF_CHECK_CUDA(cudaMemcpyAsync(h->U64, U, link_len(G) * sizeof(double2), cudaMemcpyDeviceToDevice, st));
    size_t lo_b = h->prm.fine_prec == DWF_F64 ? 16 : (h->prm.fine_prec == DWF_F32 ? 8 : 4);
    DWF_TRY(mg_alloc(h, &h->Ulo, link_len(G) * lo_b));
    {
        dwf_geom g;
        g.nd = G.nd; g.Ls = G.Ls; g.group = G.group;
        for (int mu = 0; mu < 4; ++mu) { g.L[mu] = G.L[mu]; g.antiperiodic[mu] = G.anti[mu]; }
        DWF_TRY(dwf_convert_links(&g, h->U64, h->Ulo, h->prm.fine_prec, st));
        // the K-cycle's FP32 fine vectors in the slice-paired layout: links packed once
        h->pk = h->prm.fine_layout == 0 && G.nd == 4 && G.Ls % 2 == 0 && G.V % 32 == 0;
        if (h->pk) {
            DWF_TRY(mg_alloc(h, &h->Upk, dwf_packed_link_size(&g) * lo_b));
            DWF_TRY(dwf_pack_links(&g, h->U64, h->Upk, h->prm.fine_prec, st));
        }
    }
    DWF_TRY(mg_alloc(h, (void**)&h->nullv, m.nvec * n1 * sizeof(double2)));
    DWF_CHECK_CUDA(cudaMemcpyAsync(h->nullv, starts, m.nvec * n1 * sizeof(double2), cudaMemcpyDeviceToDevice, st));
    DWF_TRY(mg_alloc(h, (void**)&h->status, 256));
    DWF_CHECK_CUDA(cudaMemsetAsync(h->status, 0, 256, st));

    // 1. relaxation
    if (h->prm.setup_maxiter > 0) {
        void* tmp = nullptr;
        DWF_CHECK_CUDA(cudaMallocAsync(&tmp, 4 * n1 * sizeof(double2) + 256, st));
        double2* r = (double2*)tmp;
        double2* p = r + n1;
        double2* t = p + n1;
        double2* Ap = t + n1;
        NvState* S = (NvState*)(h->ws.scal + 16);
        dwf_status s = DWF_OK;
        for (int k = 0; k < m.nvec && s == DWF_OK; ++k) {
            int it = 0;
            s = relax_null(h, h->nullv + k * n1, r, p, t, Ap, S, &it);
        }
        cudaFreeAsync(tmp, st);
        DWF_TRY(s);
    }
    // 2. prolongator
    const long long Psz = G.V * 2 * m.nchd * m.nvec;
    DWF_TRY(mg_alloc(h, (void**)&h->P64, Psz * sizeof(double2)));
    DWF_TRY(mg_alloc(h, (void**)&h->P32, Psz * sizeof(float2)));
    AggIndex ai;
    ai.nd = m.nd;
    for (int mu = 0; mu < 4; ++mu) { ai.L[mu] = m.L[mu]; ai.b[mu] = m.b[mu]; ai.Lc[mu] = m.Lc[mu]; }
    {
        dim3 grid((unsigned)m.Vc, 2);
        size_t sh = (size_t)m.nvec * m.nb * m.nchd * sizeof(double2);
        if (sh > 48 * 1024) DWF_CHECK_CUDA(cudaFuncSetAttribute(k_block_ortho, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh));
        k_block_ortho<<<grid, 32, sh, st>>>(h->nullv, h->P64, ai, m.nchd, G.ncol, (int)dof, m.nvec, G.V, m.nb, h->status,
                                            0);
        DWF_CHECK_LAUNCH();
    }
    k_d2f<<<ew_grid(Psz), 256, 0, st>>>(h->P64, h->P32, Psz);
    DWF_CHECK_LAUNCH();
    // 3. Galerkin blocks
    const long long nblk = m.Vc * m.ndir;
    DWF_TRY(mg_alloc(h, (void**)&h->Y64, nblk * m.ncd * m.ncd * sizeof(double2)));
    DWF_TRY(mg_alloc(h, (void**)&h->Y32, nblk * m.ncd * m.ncd * sizeof(float2)));
    DWF_TRY(mg_alloc(h, (void**)&h->Yd32, nblk * m.ncd * m.ncd * sizeof(float2)));
    if (m.nd == 2) {
        dim3 grid((unsigned)m.Vc, 5);
        int thr = m.ncd * m.ncd < 256 ? m.ncd * m.ncd : 256;
        k_galerkin_2d<<<grid, thr, 0, st>>>((const double2*)h->U64, h->P64, h->Y64, ai, m.nvec, G.V,
                                             (double)G.nd - h->M5, G.anti[0], G.anti[1]);
        DWF_CHECK_LAUNCH();
    } else {
        if (G.group != DWF_SU3 || m.ncd > 64 || m.nchd != 6) {
            set_error("4-d multigrid setup supports SU(3) with nvec <= 32");
            return DWF_ERR_UNSUPPORTED;
        }
        const size_t sh = (size_t)(12 * m.nvec * 2 + 12 * m.ncd) * sizeof(float2);
        dim3 grid((unsigned)m.Vc, 9);
        k_galerkin_4d<<<grid, GAL4_THREADS, sh, st>>>((const double2*)h->U64, h->P32, h->Y64, ai, m.nvec, G.V,
                                                      (float)((double)G.nd - h->M5),
                                                      make_int4(G.anti[0], G.anti[1], G.anti[2], G.anti[3]));
        DWF_CHECK_LAUNCH();
    }
    k_blocks_to_f32<<<ew_grid(nblk * m.ncd * m.ncd), 256, 0, st>>>(h->Y64, h->Y32, nblk, m.ncd);
    DWF_CHECK_LAUNCH();
    DWF_TRY(build_adjoint_blocks(h, st));
    if (h->prm.coarse_block_prec == DWF_F32_L16) {
        DWF_TRY(mg_alloc(h, &h->Ytile, nblk * m.ncd * m.ncd * sizeof(__half2)));
        k_blocks_to_f16<<<ew_grid(nblk * m.ncd * m.ncd), 256, 0, st>>>(h->Y64, (__half2*)h->Ytile, nblk, m.ncd);
        DWF_CHECK_LAUNCH();
        h->ytile_half = 1;
        if (m.ncd == 48 && m.ndir == 9 && m.Ls_c <= 4) {
            DWF_TRY(mg_alloc(h, &h->Ymma, nblk * m.ncd * m.ncd * sizeof(__half2)));
            k_blocks_to_mma<<<ew_grid(nblk * m.ncd * m.ncd * 2), 256, 0, st>>>(h->Y64, (__half*)h->Ymma, m.Vc);
            DWF_CHECK_LAUNCH();
        }
    } else {
        h->Ytile = h->Y32;
        h->ytile_half = 0;
    }
    int hstat = 0;
    DWF_CHECK_CUDA(cudaMemcpyAsync(&hstat, h->status, sizeof(int), cudaMemcpyDeviceToHost, st));
    DWF_CHECK_CUDA(cudaStreamSynchronize(st));
    if (hstat) {
        set_error("a near-null vector vanishes on an aggregate: the prolongator is rank deficient");
        return DWF_ERR_ARG;
    }
    return DWF_OK;
}

}  // namespace dwf

using namespace dwf;

extern "C" {

void dwf_mg_default_params(dwf_mg_params* p) {
    if (!p) return;
    memset(p, 0, sizeof(*p));
    p->nvec = 8;
    p->block[0] = p->block[1] = p->block[2] = p->block[3] = 4;
    p->Ls_c = 4;
    p->setup_maxiter = 250;
    p->setup_tol = 1e-4;
    p->setup_mass = 0.0;
    p->gcr_restart = 16;
    p->pre_smooth = 0;
    p->post_smooth = 8;
    p->coarse_tol = 0.25;
    p->coarse_maxiter = 1024;
    p->fine_prec = DWF_F32_L16;
    p->inner_tol = 1e-5;
    p->max_restarts = 1000;
    p->coarse_persistent = 1;
    p->coarse_solver = 1;
    p->coarse_restart = 8;
    p->coarse_block_prec = DWF_F32_L16;
    p->cgs_passes = 1;
    p->coarse_tc = 0;
    p->transfer = 0;
    p->fine_layout = 0;
}

dwf_status mg_setup(const dwf_geom* g, const void* U, double M5, double mf, const dwf_mg_params* p,
                    const void* null_starts, dwf_mg** out, void* stream) {
    clear_error();
    if (!out) { set_error("NULL handle pointer"); return DWF_ERR_ARG; }
    *out = nullptr;
    Geom G;
    DWF_TRY(check_geom(g, &G));
    dwf_mg_params prm;
    if (p) prm = *p; else dwf_mg_default_params(&prm);
    if (!U || !null_starts) { set_error("NULL device pointer"); return DWF_ERR_ARG; }
    if (prm.nvec < 1 || prm.nvec > MG_MAX_NVEC) { set_error("nvec must be in [1, %d]", MG_MAX_NVEC); return DWF_ERR_ARG; }
    if (prm.Ls_c < 1) { set_error("Ls_c must be >= 1"); return DWF_ERR_ARG; }
    if (!valid_prec(prm.fine_prec) || prm.fine_prec == DWF_F64) {
        set_error("fine_prec must be one of the FP32 precisions"); return DWF_ERR_ARG;
    }
    if (prm.cgs_passes != 1 && prm.cgs_passes != 2) { set_error("cgs_passes must be 1 or 2"); return DWF_ERR_ARG; }
    if (prm.coarse_tc < 0 || prm.coarse_tc > 6) { set_error("coarse_tc must be in [0, 6]"); return DWF_ERR_ARG; }
    if (prm.coarse_block_prec != DWF_F32 && prm.coarse_block_prec != DWF_F32_L16) {
        set_error("coarse_block_prec must be DWF_F32 or DWF_F32_L16"); return DWF_ERR_ARG;
    }
    if (prm.transfer != 0 && prm.transfer != 1) { set_error("transfer must be 0 (walls) or 1 (bulk)"); return DWF_ERR_ARG; }
    if (prm.fine_layout != 0 && prm.fine_layout != 1) { set_error("fine_layout must be 0 or 1"); return DWF_ERR_ARG; }
    if (prm.transfer == 1 && prm.Ls_c != G.Ls) {
        set_error("the bulk transfer keeps every slice: Ls_c must equal Ls (%d)", G.Ls); return DWF_ERR_ARG;
    }
    if (prm.gcr_restart < 1 || prm.post_smooth < 0 || prm.coarse_maxiter < 1 || prm.setup_maxiter < 0) {
        set_error("bad solver parameters"); return DWF_ERR_ARG;
    }
    MgGeom m;
    memset(&m, 0, sizeof(m));
    m.nd = G.nd;
    m.V = G.V;
    m.Vc = 1;
    m.nb = 1;
    for (int mu = 0; mu < 4; ++mu) {
        m.L[mu] = G.L[mu];
        m.b[mu] = mu < G.nd ? prm.block[mu] : 1;
        if (m.b[mu] < 1 || m.L[mu] % m.b[mu]) {
            set_error("block[%d] = %d must divide L[%d] = %d", mu, m.b[mu], mu, m.L[mu]);
            return DWF_ERR_ARG;
        }
        m.Lc[mu] = m.L[mu] / m.b[mu];
        m.Vc *= m.Lc[mu];
        m.nb *= m.b[mu];
    }
    m.nchd = G.nspin / 2 * G.ncol;
    m.nvec = prm.nvec;
    m.ncd = 2 * prm.nvec;
    m.ndir = 2 * G.nd + 1;
    m.Ls = G.Ls;
    m.Ls_c = prm.Ls_c;
    if ((long long)m.nb * m.nchd < m.nvec) {
        set_error("aggregates of %d dof per chirality cannot hold %d orthonormal vectors", m.nb * m.nchd, m.nvec);
        return DWF_ERR_ARG;
    }
    dwf_mg* h = new (std::nothrow) dwf_mg();
    if (!h) { set_error("host allocation failed"); return DWF_ERR_OOM; }
    h->G = G;
    h->mg = m;
    h->M5 = M5;
    h->mf = mf;
    h->prm = prm;
    h->st = as_stream(stream);
    h->ws_ready = false;
    h->hsc = nullptr;
    h->x64 = h->r64 = nullptr;
    h->solver_meta = nullptr;
    h->solver_meta_ready = false;
    h->coarse_graph_first = nullptr;
    h->coarse_graph_cycle = nullptr;
    h->cap_stream = nullptr;
    h->batched = nullptr;
    h->lvl3 = nullptr;
    dwf_status s = coarse_init_attributes();
    if (s == DWF_OK) s = setup_impl(h, U, null_starts);
    if (s != DWF_OK) {
        std::string msg = dwf_last_error();
        mg_destroy(h);
        set_error("%s", msg.c_str());
        return s;
    }
    *out = h;
    return DWF_OK;
}

void mg_destroy(dwf_mg* h) {
    if (!h) return;
    cudaStreamSynchronize(h->st);
    batched_state_free(h);
    level3_free(h);
    for (void* p : h->allocs) cudaFree(p);
    for (void* p : h->fine_vecs) cudaFree(p);
    for (void* p : h->coarse_vecs) cudaFree(p);
    if (h->solver_meta) cudaFree(h->solver_meta);
    if (h->coarse_graph_first) cudaGraphExecDestroy(h->coarse_graph_first);
    if (h->coarse_graph_cycle) cudaGraphExecDestroy(h->coarse_graph_cycle);
    if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
    if (h->hsc) cudaFreeHost(h->hsc);
    delete h;
}

dwf_status mg_check_operator(const dwf_mg* h, const void* U, double M5, double mf, void* stream) {
    clear_error();
    if (!h || !U) { set_error("NULL argument"); return DWF_ERR_ARG; }
    if (M5 != h->M5 || mf != h->mf) {
        set_error("the hierarchy was set up for M5 = %.17g, mf = %.17g, not M5 = %.17g, mf = %.17g", h->M5, h->mf,
                  M5, mf);
        return DWF_ERR_ARG;
    }
    cudaStream_t st = as_stream(stream);
    const long long n = link_len(h->G);
    int* flag = h->status + 8;                 // spare word of the setup status block
    DWF_CHECK_CUDA(cudaMemsetAsync(flag, 0, sizeof(int), st));
    k_links_differ<<<ew_grid(n), 256, 0, st>>>((const double2*)h->U64, (const double2*)U, n, flag);
    DWF_CHECK_LAUNCH();
    int differ = 0;
    DWF_CHECK_CUDA(cudaMemcpyAsync(&differ, flag, sizeof(int), cudaMemcpyDeviceToHost, st));
    DWF_CHECK_CUDA(cudaStreamSynchronize(st));
    if (differ) {
        set_error("the links differ from those the hierarchy was set up with: run mg_setup on the new links");
        return DWF_ERR_ARG;
    }
    return DWF_OK;
}

dwf_status mg_coarse_geom(const dwf_mg* h, dwf_geom* c, int* ncdof) {
    clear_error();
    if (!h || !c) { set_error("NULL argument"); return DWF_ERR_ARG; }
    memset(c, 0, sizeof(*c));
    c->nd = h->mg.nd;
    for (int mu = 0; mu < 4; ++mu) c->L[mu] = mu < h->mg.nd ? h->mg.Lc[mu] : 0;
    c->Ls = h->mg.Ls_c;
    c->group = h->G.group;
    if (ncdof) *ncdof = h->mg.ncd;
    return DWF_OK;
}

dwf_status mg_get_prolongator(const dwf_mg* h, void* P_out, void* stream) {
    clear_error();
    if (!h || !P_out) { set_error("NULL argument"); return DWF_ERR_ARG; }
    const long long n = h->G.V * 2 * h->mg.nchd * h->mg.nvec;
    DWF_CHECK_CUDA(cudaMemcpyAsync(P_out, h->P64, n * sizeof(double2), cudaMemcpyDeviceToDevice, as_stream(stream)));
    return DWF_OK;
}

dwf_status mg_get_null_vectors(const dwf_mg* h, void* v_out, void* stream) {
    clear_error();
    if (!h || !v_out) { set_error("NULL argument"); return DWF_ERR_ARG; }
    const long long n = h->mg.nvec * h->G.V * site_dof(h->G);
    DWF_CHECK_CUDA(cudaMemcpyAsync(v_out, h->nullv, n * sizeof(double2), cudaMemcpyDeviceToDevice, as_stream(stream)));
    return DWF_OK;
}

dwf_status mg_get_coarse_links(const dwf_mg* h, void* Y_out, void* stream) {
    clear_error();
    if (!h || !Y_out) { set_error("NULL argument"); return DWF_ERR_ARG; }
    const long long n = h->mg.Vc * h->mg.ndir * h->mg.ncd * h->mg.ncd;
    DWF_CHECK_CUDA(cudaMemcpyAsync(Y_out, h->Y64, n * sizeof(double2), cudaMemcpyDeviceToDevice, as_stream(stream)));
    return DWF_OK;
}

}  // extern "C"
