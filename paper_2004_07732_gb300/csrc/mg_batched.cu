// Batched K-cycle (Sec. 2.3, "Summary"; Table kcycle): nrhs right-hand sides
// that share one hierarchy (one gauge field) are solved together.
//
// Every vector of the one-vector solver becomes a block of nrhs vectors stored
// back to back, and every Krylov scalar an array over the right-hand sides.
// Each launch covers all right-hand sides (grid.y, or grid.z where grid.y is
// the basis index); a right-hand side whose flag is set is skipped by every
// block of its row, so one fixed launch sequence serves any set of
// still-active systems and the coarse cycle stays a single CUDA graph.  The
// coarse operator on the nrhs * Ls_c columns is the tensor-core contraction
// (mg_coarse_tc.cu).  With one right-hand side it is the one-vector stencil:
// that is the path mg_solve takes with the GCR coarse solver on 2-d and 4-d
// lattices (4-d hierarchies take one right-hand side per call).  Per
// right-hand side the iteration is exactly the
// one-vector solver's: FP64 reliable updates of the true residual around
// FGCR(gcr_restart) in FP32, the wall restriction, coarse GCR to coarse_tol,
// prolongation and post_smooth GCR steps.
//
// Reductions: one row of partial sums and completion counters per right-hand
// side (and per basis vector for the Gram-Schmidt dots of vectors that fit in
// L2; larger vectors take all basis vectors in one pass over w), so the rows
// finish independently and each result is summed in a fixed order.
#include <chrono>
#include <mutex>
#include <string.h>
#include <string>
#include <thread>
#include <vector>

#include "mg.cuh"

namespace dwf {
namespace {

constexpr int BK_MAX = 32;            // bound on the restart lengths
constexpr int BMDOT_BLOCKS = 608;     // partial slots per (right-hand side, basis vector) of a Gram-Schmidt dot
constexpr int BMDOT_ROW_BLOCKS = 152; // blocks per row of the per-row form
constexpr long long BMDOT_FUSE_N = 8LL << 20;   // complex values from which the fused form is used
constexpr int CROW = (RED_GROUPS + 1) * RED_CSTRIDE;   // unsigneds of completion counters per row
constexpr int PROW = RED_MAX * RED_BLOCKS;             // doubles of partial sums per row

// Krylov scalars of one right-hand side.  The GCR iterations keep only the
// orthogonalised images w_k = A p'_k and the residual up to date; the search
// directions are p'_k = p_k - sum_{j<k} C[k][j] p'_j of the stored raw
// directions p_k, so the solution update sum_k A[k] p'_k is assembled once per
// cycle as sum_j y_j p_j with (I + C)^T y = A (back substitution): every step
// then reads and writes the raw basis only once.
struct BGcr {
    double coef[BK_MAX][2];          // projection coefficients of the current pass
    double nrm[BK_MAX];              // |w_k|^2
    double alpha[2];                 // alpha of the current step
    double rr2;                      // |r|^2 after the current step
    double pad;
    double C[BK_MAX][BK_MAX][2];     // C[k][j], j < k: summed over the Gram-Schmidt passes of step k
    double A[BK_MAX][2];             // alpha of step k
};

__device__ __forceinline__ RedScratch row_scratch(RedScratch base, int r) {
    return RedScratch{base.partials + (size_t)r * PROW, base.counter + (size_t)r * CROW};
}

__device__ __forceinline__ void cdot4(const float4 a, const float4 b, float& re, float& im) {
    re += a.x * b.x + a.y * b.y + a.z * b.z + a.w * b.w;
    im += a.x * b.y - a.y * b.x + a.z * b.w - a.w * b.z;
}

__device__ __forceinline__ void csub4(float4& x, const float4 a, const float2 c) {
    x.x -= c.x * a.x - c.y * a.y; x.y -= c.x * a.y + c.y * a.x;
    x.z -= c.x * a.z - c.y * a.w; x.w -= c.x * a.w + c.y * a.z;
}

__device__ __forceinline__ void cadd4(float4& x, const float4 a, const float2 c) {
    x.x += c.x * a.x - c.y * a.y; x.y += c.x * a.y + c.y * a.x;
    x.z += c.x * a.z - c.y * a.w; x.w += c.x * a.w + c.y * a.z;
}

#define ROW_LOOP(i, n2) for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < (n2); i += (long long)gridDim.x * blockDim.x)

// ---- element-wise kernels; n = complex values per right-hand side (even) ----
__global__ void k_bcopy(float2* __restrict__ out, const float2* __restrict__ in, long long n, const int* skip) {
    const int r = blockIdx.y;
    if (skip && skip[r]) return;
    const float4* a = reinterpret_cast<const float4*>(in + r * n);
    float4* o = reinterpret_cast<float4*>(out + r * n);
    ROW_LOOP(i, n >> 1) o[i] = a[i];
}

__global__ void k_bsub32(float2* __restrict__ out, const float2* __restrict__ a, const float2* __restrict__ b,
                         long long n, const int* skip) {
    const int r = blockIdx.y;
    if (skip && skip[r]) return;
    const float4* x = reinterpret_cast<const float4*>(a + r * n);
    const float4* y = reinterpret_cast<const float4*>(b + r * n);
    float4* o = reinterpret_cast<float4*>(out + r * n);
    ROW_LOOP(i, n >> 1) {
        const float4 u = x[i], v = y[i];
        o[i] = make_float4(u.x - v.x, u.y - v.y, u.z - v.z, u.w - v.w);
    }
}

__global__ void k_bsub64(double2* __restrict__ out, const double2* __restrict__ a, const double2* __restrict__ b,
                         long long n, const int* skip) {
    const int r = blockIdx.y;
    if (skip && skip[r]) return;
    a += r * n; b += r * n; out += r * n;
    ROW_LOOP(i, n) { const double2 u = a[i], v = b[i]; out[i] = make_double2(u.x - v.x, u.y - v.y); }
}

// out (FP32) = a (FP64) * scale[r]
__global__ void k_bd2f_scale(float2* __restrict__ out, const double2* __restrict__ a, const double* scale, long long n,
                             const int* skip) {
    const int r = blockIdx.y;
    if (skip && skip[r]) return;
    const double s = scale[r];
    a += r * n; out += r * n;
    ROW_LOOP(i, n) { const double2 u = a[i]; out[i] = make_float2((float)(u.x * s), (float)(u.y * s)); }
}

// Slice-paired packed FP32 fine vectors (4-d, one right-hand side): packed float4 i holds
// element d of site x on slices 2j and 2j+1; pk_canon gives the canonical complex index of the
// slice-2j value (the slice-2j+1 value is V dof further).
struct PackIdx {
    long long V, NB;
    int dof;
};
__device__ __forceinline__ long long pk_canon(const PackIdx& q, long long i) {
    const int lane = (int)(i & 31);
    const long long t = i >> 5;
    const int d = (int)(t % q.dof);
    const long long t2 = t / q.dof;
    const long long x = (t2 % q.NB) * 32 + lane;
    const long long j = t2 / q.NB;
    return ((2 * j) * q.V + x) * q.dof + d;
}

// out (packed FP32) = scale * a (canonical FP64)
__global__ void k_bd2f_scale_pk(float2* __restrict__ out, const double2* __restrict__ a, const double* scale,
                                long long n, const int* skip, PackIdx q) {
    if (skip && skip[0]) return;
    const double s = scale[0];
    float4* o = reinterpret_cast<float4*>(out);
    const long long sv = q.V * q.dof;
    ROW_LOOP(i, n >> 1) {
        const long long c = pk_canon(q, i);
        const double2 u = a[c], w = a[c + sv];
        o[i] = make_float4((float)(u.x * s), (float)(u.y * s), (float)(w.x * s), (float)(w.y * s));
    }
}

// out[r] = |x_r|^2.  FP64 data: every product in FP64; FP32 data: per-thread
// FP32 partials over a few elements, FP64 across threads.
__global__ void __launch_bounds__(RED_THREADS) k_bnorm2_64(const double2* __restrict__ x, long long n, RedScratch rs,
                                                           double* out, const int* skip) {
    const int r = blockIdx.y;
    if (skip && skip[r]) return;
    x += r * n;
    double v[1] = {0.0};
    ROW_LOOP(i, n) { const double2 a = x[i]; v[0] += a.x * a.x + a.y * a.y; }
    grid_reduce<1>(v, row_scratch(rs, r), [=] __device__(double* t) { out[r] = t[0]; });
}

__global__ void __launch_bounds__(RED_THREADS) k_bnorm2_32(const float2* __restrict__ x, long long n, RedScratch rs,
                                                           double* out, const int* skip) {
    const int r = blockIdx.y;
    if (skip && skip[r]) return;
    const float4* a = reinterpret_cast<const float4*>(x + r * n);
    float acc = 0.f;
    ROW_LOOP(i, n >> 1) { const float4 u = a[i]; acc += u.x * u.x + u.y * u.y + u.z * u.z + u.w * u.w; }
    const float v[1] = {acc};
    grid_reduce_f<1>(v, row_scratch(rs, r), [=] __device__(double* t) { out[r] = t[0]; });
}

// rout = rin - alpha w, rr2 = |rout|^2 per right-hand side (rout may be rin).
// With `done`: iters[r] += 1 and done[r] = 1 once rr2 <= tol2 * ref2[r] or
// iters[r] >= maxit.  `skip` and `done` may be the same array: every block of a
// row reads the flag before the row's last block (the only writer) runs its
// finaliser.
__global__ void __launch_bounds__(RED_THREADS) k_bres_update(const float2* rin, float2* rout,
                                                             const float2* __restrict__ w, BGcr* g, long long n,
                                                             RedScratch rs, const int* skip, int* done,
                                                             const double* ref2, double tol2, int* iters, int maxit) {
    const int r = blockIdx.y;
    if (skip && skip[r]) return;
    const float ar = (float)g[r].alpha[0], ai = (float)g[r].alpha[1];
    const float4* a4 = reinterpret_cast<const float4*>(rin + r * n);
    float4* o4 = reinterpret_cast<float4*>(rout + r * n);
    const float4* w4 = reinterpret_cast<const float4*>(w + r * n);
    float acc = 0.f;
    ROW_LOOP(i, n >> 1) {
        const float4 wi = w4[i];
        float4 ri = a4[i];
        ri.x -= ar * wi.x - ai * wi.y; ri.y -= ar * wi.y + ai * wi.x;
        ri.z -= ar * wi.z - ai * wi.w; ri.w -= ar * wi.w + ai * wi.z;
        o4[i] = ri;
        acc += ri.x * ri.x + ri.y * ri.y + ri.z * ri.z + ri.w * ri.w;
    }
    const float v[1] = {acc};
    grid_reduce_f<1>(v, row_scratch(rs, r), [=] __device__(double* t) {
        g[r].rr2 = t[0];
        if (done) {
            iters[r] += 1;
            if (t[0] <= tol2 * ref2[r] || iters[r] >= maxit) done[r] = 1;
        }
    });
}

// Classical Gram-Schmidt dots: coef[j] = <W_j, w> / nrm[j] for j < k (k =
// gridDim.y), per right-hand side, also summed into C[k][j] (set on the first
// pass).  Grid (B, k, nrhs); W: device array of basis block pointers.
__global__ void __launch_bounds__(RED_THREADS) k_bmdot_rows(float2* const* __restrict__ W, const float2* __restrict__ w,
                                                       long long n, double* __restrict__ part, unsigned* counters,
                                                       BGcr* g, int first, const int* skip) {
    const int r = blockIdx.z, j = blockIdx.y;
    if (skip && skip[r]) return;
    const float4* Wj = reinterpret_cast<const float4*>(W[j] + r * n);
    const float4* w4 = reinterpret_cast<const float4*>(w + r * n);
    const long long n2 = n >> 1;
    float re = 0.f, im = 0.f;
    const long long stride = (long long)gridDim.x * blockDim.x;
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    for (; i + 3 * stride < n2; i += 4 * stride) {
        const float4 a0 = Wj[i], a1 = Wj[i + stride], a2 = Wj[i + 2 * stride], a3 = Wj[i + 3 * stride];
        const float4 b0 = w4[i], b1 = w4[i + stride], b2 = w4[i + 2 * stride], b3 = w4[i + 3 * stride];
        cdot4(a0, b0, re, im); cdot4(a1, b1, re, im); cdot4(a2, b2, re, im); cdot4(a3, b3, re, im);
    }
    for (; i < n2; i += stride) cdot4(Wj[i], w4[i], re, im);
    const float vf[2] = {re, im};
    double v[2];
    block_sum_f<2>(vf, v);
    const size_t rowi = (size_t)r * BK_MAX + j;
    double* pr = part + rowi * 2 * BMDOT_BLOCKS;
    if (threadIdx.x == 0) {
        pr[blockIdx.x] = v[0];
        pr[BMDOT_BLOCKS + blockIdx.x] = v[1];
    }
    if (!grid_last_block(counters + rowi * CROW)) return;
    __threadfence();
    double w2[2];
    grid_final_sum<2>(pr, BMDOT_BLOCKS, w2);
    if (threadIdx.x == 0) {
        const double nn = g[r].nrm[j];
        const double cr = nn > 0 ? w2[0] / nn : 0.0, ci = nn > 0 ? w2[1] / nn : 0.0;
        const int k = gridDim.y;
        g[r].coef[j][0] = cr;
        g[r].coef[j][1] = ci;
        g[r].C[k][j][0] = first ? cr : g[r].C[k][j][0] + cr;
        g[r].C[k][j][1] = first ? ci : g[r].C[k][j][1] + ci;
    }
}

// The same dots for vectors larger than L2: coef[j] = <W_j, w> / nrm[j] for j < k, per
// right-hand side, also summed into C[k][j] (set on the first pass).  Grid
// (B, nrhs): each thread reads its elements of w once and of every W_j once
// (k + 1 vectors per pass instead of 2 k), keeping the k partial dots in
// registers (KM >= k, unrolled with guards).  The last block of a row sums the
// per-block partials of every j in a fixed order.  W: device array of basis
// block pointers.
template <int KM>
__global__ void __launch_bounds__(RED_THREADS) k_bmdot(float2* const* __restrict__ W, const float2* __restrict__ w,
                                                       long long n, int k, double* __restrict__ part,
                                                       unsigned* counters, BGcr* g, int first, const int* skip) {
    const int r = blockIdx.y;
    if (skip && skip[r]) return;
    __shared__ const float4* Wp[KM];
    for (int j = threadIdx.x; j < k; j += blockDim.x) Wp[j] = reinterpret_cast<const float4*>(W[j] + r * n);
    __syncthreads();
    const float4* w4 = reinterpret_cast<const float4*>(w + r * n);
    float re[KM], im[KM];
#pragma unroll
    for (int j = 0; j < KM; ++j) { re[j] = 0.f; im[j] = 0.f; }
    ROW_LOOP(i, n >> 1) {
        const float4 wi = w4[i];
#pragma unroll
        for (int j = 0; j < KM; ++j)
            if (j < k) cdot4(Wp[j][i], wi, re[j], im[j]);
    }
    double* pr = part + (size_t)r * BK_MAX * 2 * BMDOT_BLOCKS;     // [j][re / im][block]
#pragma unroll
    for (int j0 = 0; j0 < KM; j0 += 4) {
        if (j0 >= k) break;                                       // block-uniform
        float vf[8];
#pragma unroll
        for (int q = 0; q < 4; ++q) { vf[2 * q] = re[j0 + q]; vf[2 * q + 1] = im[j0 + q]; }
        double v[8];
        block_sum_f<8>(vf, v);
        if (threadIdx.x == 0)
#pragma unroll
            for (int q = 0; q < 4; ++q)
                if (j0 + q < k) {
                    pr[(size_t)(j0 + q) * 2 * BMDOT_BLOCKS + blockIdx.x] = v[2 * q];
                    pr[(size_t)(j0 + q) * 2 * BMDOT_BLOCKS + BMDOT_BLOCKS + blockIdx.x] = v[2 * q + 1];
                }
    }
    if (!grid_last_block(counters + (size_t)r * BK_MAX * CROW)) return;
    __threadfence();
    // quantity q = 2 j + (0: Re, 1: Im) of block b at pr[q * BMDOT_BLOCKS + b]; warp w sums q = w, w + 8, ...
    __shared__ double tot[2 * KM];
    {
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        for (int q = warp; q < 2 * k; q += RED_THREADS / 32) {
            double sq = 0.0;
            for (unsigned bb = lane; bb < gridDim.x; bb += 32) sq += __ldcg(pr + (size_t)q * BMDOT_BLOCKS + bb);
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) sq += __shfl_down_sync(0xffffffffu, sq, off);
            if (lane == 0) tot[q] = sq;
        }
    }
    __syncthreads();
    for (int j = 0; j < k; ++j) {
        if (threadIdx.x == 0) {
            const double nn = g[r].nrm[j];
            const double cr = nn > 0 ? tot[2 * j] / nn : 0.0, ci = nn > 0 ? tot[2 * j + 1] / nn : 0.0;
            g[r].coef[j][0] = cr;
            g[r].coef[j][1] = ci;
            g[r].C[k][j][0] = first ? cr : g[r].C[k][j][0] + cr;
            g[r].C[k][j][1] = first ? ci : g[r].C[k][j][1] + ci;
        }
    }
}

static void launch_bmdot(dim3 grid, float2* const* W, const float2* w, long long n, int k, double* part,
                         unsigned* counters, BGcr* g, int first, const int* skip, cudaStream_t st) {
    if (k <= 4)       k_bmdot<4><<<grid, RED_THREADS, 0, st>>>(W, w, n, k, part, counters, g, first, skip);
    else if (k <= 8)  k_bmdot<8><<<grid, RED_THREADS, 0, st>>>(W, w, n, k, part, counters, g, first, skip);
    else if (k <= 16) k_bmdot<16><<<grid, RED_THREADS, 0, st>>>(W, w, n, k, part, counters, g, first, skip);
    else              k_bmdot<32><<<grid, RED_THREADS, 0, st>>>(W, w, n, k, part, counters, g, first, skip);
}

// w -= sum_{j<k} coef_j W_j per right-hand side.  FINAL: also nrm[k] = |w|^2,
// alpha = A[k] = <w, res> / |w|^2, and steps[r] = k + 1 (steps may be null).
template <bool FINAL>
__global__ void __launch_bounds__(RED_THREADS) k_bmaxpy(float2* __restrict__ w, float2* const* __restrict__ W, BGcr* g,
                                                        int k, const float2* __restrict__ res, long long n,
                                                        RedScratch rs, int* steps, const int* skip) {
    const int r = blockIdx.y;
    if (skip && skip[r]) return;
    __shared__ float2 c[BK_MAX];
    __shared__ const float4* Wp[BK_MAX];
    for (int j = threadIdx.x; j < k; j += blockDim.x) {
        c[j] = make_float2((float)g[r].coef[j][0], (float)g[r].coef[j][1]);
        Wp[j] = reinterpret_cast<const float4*>(W[j] + r * n);
    }
    __syncthreads();
    float4* w4 = reinterpret_cast<float4*>(w + r * n);
    const float4* r4 = reinterpret_cast<const float4*>(res + r * n);
    float f0 = 0.f, f1 = 0.f, f2 = 0.f;
    ROW_LOOP(i, n >> 1) {
        float4 wi = w4[i];
        int j = 0;
        for (; j + 3 < k; j += 4) {
            const float4 a0 = Wp[j][i], a1 = Wp[j + 1][i], a2 = Wp[j + 2][i], a3 = Wp[j + 3][i];
            csub4(wi, a0, c[j]); csub4(wi, a1, c[j + 1]); csub4(wi, a2, c[j + 2]); csub4(wi, a3, c[j + 3]);
        }
        for (; j < k; ++j) csub4(wi, Wp[j][i], c[j]);
        if (k > 0) w4[i] = wi;
        if (FINAL) {
            f0 += wi.x * wi.x + wi.y * wi.y + wi.z * wi.z + wi.w * wi.w;
            cdot4(wi, r4[i], f1, f2);
        }
    }
    if (FINAL) {
        const float v[3] = {f0, f1, f2};
        grid_reduce_f<3>(v, row_scratch(rs, r), [=] __device__(double* t) {
            const double ar = t[0] > 0 ? t[1] / t[0] : 0.0, ai = t[0] > 0 ? t[2] / t[0] : 0.0;
            g[r].nrm[k] = t[0];
            g[r].alpha[0] = ar; g[r].alpha[1] = ai;
            g[r].A[k][0] = ar; g[r].A[k][1] = ai;
            if (steps) steps[r] = k + 1;
        });
    }
}

// One GCR step of the coarse solve with a single classical Gram-Schmidt pass,
// in one reduction pass and one element-wise pass.  The reduction reads the
// image w = A p_k, the residual r and the orthogonalised images W_j (j < k)
// once and sums d_j = <W_j, w>, |w|^2, <w, r> and |r|^2.  The W_j are mutually
// orthogonal and r is orthogonal to every W_j, so with w' = w - sum_j c_j W_j:
//   c_j = d_j / |W_j|^2,   |w'|^2 = |w|^2 - sum_j |d_j|^2 / |W_j|^2,
//   alpha = <w', r> / |w'|^2 = <w, r> / |w'|^2,
//   |r - alpha w'|^2 = |r|^2 - |<w, r>|^2 / |w'|^2,
// and the element-wise pass forms w' and r - alpha w' without a reduction.
// The residual norm is exact at every step (|r|^2 is summed afresh); only the
// one-step prediction decides convergence.  A direction with |w'|^2 below
// BSTEP_BREAK |w|^2 is not resolved by FP32 sums: its row stops (alpha = 0).
constexpr int BSTEP_BLOCKS = 512;     // bound on the blocks per row of the reduction pass
constexpr double BSTEP_BREAK = 1e-5;

template <int KM>
__global__ void __launch_bounds__(RED_THREADS) k_bstep_dots(float2* const* __restrict__ W, const float2* __restrict__ w,
                                                            const float2* __restrict__ res, long long n, int k,
                                                            double* __restrict__ part, unsigned* counters, BGcr* g,
                                                            int* steps, int* done, const double* ref2, double tol2,
                                                            int* iters, int maxit) {
    constexpr int NQ = 2 * KM + 4;     // |w|^2, Re / Im <w, r>, |r|^2, then Re / Im d_j
    const int r = blockIdx.y;
    if (done[r]) return;
    __shared__ const float4* Wp[KM];
    __shared__ double sh[NQ][RED_THREADS / 32];
    __shared__ double tot[NQ];
    for (int j = threadIdx.x; j < k; j += blockDim.x) Wp[j] = reinterpret_cast<const float4*>(W[j] + r * n);
    __syncthreads();
    const float4* w4 = reinterpret_cast<const float4*>(w + r * n);
    const float4* r4 = reinterpret_cast<const float4*>(res + r * n);
    float re[KM], im[KM];
#pragma unroll
    for (int j = 0; j < KM; ++j) { re[j] = 0.f; im[j] = 0.f; }
    float ww = 0.f, wr = 0.f, wi = 0.f, rr = 0.f;
    ROW_LOOP(i, n >> 1) {
        const float4 a = w4[i], b = r4[i];
#pragma unroll
        for (int j = 0; j < KM; ++j)
            if (j < k) cdot4(Wp[j][i], a, re[j], im[j]);
        ww += a.x * a.x + a.y * a.y + a.z * a.z + a.w * a.w;
        cdot4(a, b, wr, wi);
        rr += b.x * b.x + b.y * b.y + b.z * b.z + b.w * b.w;
    }
    const int nq = 2 * k + 4;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // the tree over each warp in FP32, every sum across warps and blocks in FP64
    float v[NQ];
    v[0] = ww; v[1] = wr; v[2] = wi; v[3] = rr;
#pragma unroll
    for (int j = 0; j < KM; ++j) { v[4 + 2 * j] = re[j]; v[5 + 2 * j] = im[j]; }
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
        if (q < nq) {                                             // block-uniform
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) v[q] += __shfl_down_sync(0xffffffffu, v[q], off);
            if (lane == 0) sh[q][warp] = (double)v[q];
        }
    }
    __syncthreads();
    const int B = gridDim.x;
    double* pr = part + (size_t)r * BK_MAX * 2 * BMDOT_BLOCKS;       // [quantity][block]
    for (int q = threadIdx.x; q < nq; q += blockDim.x) {
        double s = 0.0;
        for (int u = 0; u < RED_THREADS / 32; ++u) s += sh[q][u];
        pr[(size_t)q * B + blockIdx.x] = s;
        __threadfence();
    }
    __syncthreads();
    if (!grid_last_block(counters + (size_t)r * BK_MAX * CROW)) return;
    __threadfence();
    for (int q = warp; q < nq; q += RED_THREADS / 32) {
        double s = 0.0;
        for (int b = lane; b < B; b += 32) s += __ldcg(pr + (size_t)q * B + b);
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
        if (lane == 0) tot[q] = s;
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    BGcr& G = g[r];
    double proj = 0.0;
    for (int j = 0; j < k; ++j) {
        const double nn = G.nrm[j], dr = tot[4 + 2 * j], di = tot[5 + 2 * j];
        const double cr = nn > 0 ? dr / nn : 0.0, ci = nn > 0 ? di / nn : 0.0;
        G.coef[j][0] = cr; G.coef[j][1] = ci;
        G.C[k][j][0] = cr; G.C[k][j][1] = ci;
        if (nn > 0) proj += (dr * dr + di * di) / nn;
    }
    const double wp = tot[0] - proj;
    const bool ok = wp > BSTEP_BREAK * tot[0];
    const double ar = ok ? tot[1] / wp : 0.0, ai = ok ? tot[2] / wp : 0.0;
    const double rn = ok ? tot[3] - (tot[1] * tot[1] + tot[2] * tot[2]) / wp : tot[3];
    G.nrm[k] = ok ? wp : 0.0;
    G.alpha[0] = ar; G.alpha[1] = ai;
    G.A[k][0] = ar; G.A[k][1] = ai;
    G.rr2 = rn;
    steps[r] = k + 1;
    iters[r] += 1;
    if (!ok || rn <= tol2 * ref2[r] || iters[r] >= maxit) done[r] = 1;
}

static void launch_bstep_dots(dim3 grid, float2* const* W, const float2* w, const float2* res, long long n, int k,
                              double* part, unsigned* counters, BGcr* g, int* steps, int* done, const double* ref2,
                              double tol2, int* iters, int maxit, cudaStream_t st) {
#define DWF_BSTEP(KM) k_bstep_dots<KM><<<grid, RED_THREADS, 0, st>>>(W, w, res, n, k, part, counters, g, steps, done, \
                                                                     ref2, tol2, iters, maxit)
    if (k <= 4)       DWF_BSTEP(4);
    else if (k <= 8)  DWF_BSTEP(8);
    else if (k <= 16) DWF_BSTEP(16);
    else              DWF_BSTEP(32);
#undef DWF_BSTEP
}

// The element-wise pass of the step: w' = w - sum_{j<k} coef_j W_j (stored in
// place) and rout = rin - alpha w'.  Rows whose solve ended at this step skip.
__global__ void __launch_bounds__(RED_THREADS) k_bstep_update(float2* __restrict__ w, float2* const* __restrict__ W,
                                                              const BGcr* g, int k, const float2* __restrict__ rin,
                                                              float2* __restrict__ rout, long long n,
                                                              const int* skip) {
    const int r = blockIdx.y;
    if (skip[r]) return;
    __shared__ float2 c[BK_MAX];
    __shared__ const float4* Wp[BK_MAX];
    for (int j = threadIdx.x; j < k; j += blockDim.x) {
        c[j] = make_float2((float)g[r].coef[j][0], (float)g[r].coef[j][1]);
        Wp[j] = reinterpret_cast<const float4*>(W[j] + r * n);
    }
    __syncthreads();
    const float2 al = make_float2((float)g[r].alpha[0], (float)g[r].alpha[1]);
    float4* w4 = reinterpret_cast<float4*>(w + r * n);
    const float4* a4 = reinterpret_cast<const float4*>(rin + r * n);
    float4* o4 = reinterpret_cast<float4*>(rout + r * n);
    ROW_LOOP(i, n >> 1) {
        float4 wi = w4[i];
        const float4 ri0 = a4[i];
        int j = 0;
        for (; j + 3 < k; j += 4) {
            const float4 b0 = Wp[j][i], b1 = Wp[j + 1][i], b2 = Wp[j + 2][i], b3 = Wp[j + 3][i];
            csub4(wi, b0, c[j]); csub4(wi, b1, c[j + 1]); csub4(wi, b2, c[j + 2]); csub4(wi, b3, c[j + 3]);
        }
        for (; j < k; ++j) csub4(wi, Wp[j][i], c[j]);
        if (k > 0) w4[i] = wi;
        float4 ri = ri0;
        csub4(ri, wi, al);
        o4[i] = ri;
    }
}

// y of the deferred solution update for the first m steps: (I + C)^T y = A,
// y_j = A_j - sum_{k>j} C[k][j] y_k (one thread, FP64)
__device__ __forceinline__ void back_substitute(const BGcr& g, int m, float2* y) {
    double yr[BK_MAX], yi[BK_MAX];
    for (int j = m - 1; j >= 0; --j) {
        double a = g.A[j][0], b = g.A[j][1];
        for (int k = j + 1; k < m; ++k) {
            const double cr = g.C[k][j][0], ci = g.C[k][j][1];
            a -= cr * yr[k] - ci * yi[k];
            b -= cr * yi[k] + ci * yr[k];
        }
        yr[j] = a; yi[j] = b;
        y[j] = make_float2((float)a, (float)b);
    }
}

// out += sum_{j<m} y_j P_j (FP32), m = nsteps[r] or m_fixed when nsteps is
// null; rows with m == 0 are left alone.  With wout: also wout = ra - rb.
__global__ void __launch_bounds__(RED_THREADS) k_bcombine32(float2* __restrict__ out, float2* const* __restrict__ P,
                                                            const BGcr* g, const int* nsteps, int m_fixed, long long n,
                                                            const float2* __restrict__ ra, const float2* __restrict__ rb,
                                                            float2* __restrict__ wout, const int* skip) {
    const int r = blockIdx.y;
    if (skip && skip[r]) return;
    const int m = nsteps ? nsteps[r] : m_fixed;
    __shared__ float2 y[BK_MAX];
    __shared__ const float4* Pp[BK_MAX];
    if (threadIdx.x == 0 && m > 0) back_substitute(g[r], m, y);
    for (int j = threadIdx.x; j < m; j += blockDim.x) Pp[j] = reinterpret_cast<const float4*>(P[j] + r * n);
    __syncthreads();
    float4* o4 = reinterpret_cast<float4*>(out + r * n);
    const float4* a4 = wout ? reinterpret_cast<const float4*>(ra + r * n) : nullptr;
    const float4* b4 = wout ? reinterpret_cast<const float4*>(rb + r * n) : nullptr;
    float4* w4 = wout ? reinterpret_cast<float4*>(wout + r * n) : nullptr;
    ROW_LOOP(i, n >> 1) {
        if (m > 0) {
            float4 x = o4[i];
            for (int j = 0; j < m; ++j) cadd4(x, Pp[j][i], y[j]);
            o4[i] = x;
        }
        if (wout) {
            const float4 u = a4[i], v = b4[i];
            w4[i] = make_float4(u.x - v.x, u.y - v.y, u.z - v.z, u.w - v.w);
        }
    }
}

// X (FP64) += s[r] * sum_{j<m} y_j Z_j, m = nsteps[r]; rows with m == 0 are left alone
__global__ void __launch_bounds__(RED_THREADS) k_bcombine64(double2* __restrict__ X, float2* const* __restrict__ Z,
                                                            const BGcr* g, const int* nsteps, const double* s,
                                                            long long n) {
    const int r = blockIdx.y;
    const int m = nsteps[r];
    if (m <= 0) return;
    __shared__ float2 y[BK_MAX];
    __shared__ const float4* Zp[BK_MAX];
    if (threadIdx.x == 0) back_substitute(g[r], m, y);
    for (int j = threadIdx.x; j < m; j += blockDim.x) Zp[j] = reinterpret_cast<const float4*>(Z[j] + r * n);
    __syncthreads();
    const double sc = s[r];
    double2* x2 = X + r * n;
    ROW_LOOP(i, n >> 1) {
        float4 e = make_float4(0.f, 0.f, 0.f, 0.f);
        for (int j = 0; j < m; ++j) cadd4(e, Zp[j][i], y[j]);
        double2 a = x2[2 * i], b = x2[2 * i + 1];
        a.x += sc * e.x; a.y += sc * e.y; b.x += sc * e.z; b.y += sc * e.w;
        x2[2 * i] = a; x2[2 * i + 1] = b;
    }
}

// k_bcombine64 with the basis in the packed layout and X canonical (one right-hand side)
__global__ void __launch_bounds__(RED_THREADS) k_bcombine64_pk(double2* __restrict__ X, float2* const* __restrict__ Z,
                                                               const BGcr* g, const int* nsteps, const double* s,
                                                               long long n, PackIdx q) {
    const int m = nsteps[0];
    if (m <= 0) return;
    __shared__ float2 y[BK_MAX];
    __shared__ const float4* Zp[BK_MAX];
    if (threadIdx.x == 0) back_substitute(g[0], m, y);
    for (int j = threadIdx.x; j < m; j += blockDim.x) Zp[j] = reinterpret_cast<const float4*>(Z[j]);
    __syncthreads();
    const double sc = s[0];
    const long long sv = q.V * q.dof;
    ROW_LOOP(i, n >> 1) {
        float4 e = make_float4(0.f, 0.f, 0.f, 0.f);
        for (int j = 0; j < m; ++j) cadd4(e, Zp[j][i], y[j]);
        const long long c = pk_canon(q, i);
        double2 a = X[c], b = X[c + sv];
        a.x += sc * e.x; a.y += sc * e.y; b.x += sc * e.z; b.y += sc * e.w;
        X[c] = a; X[c + sv] = b;
    }
}

// --------------------------------------------------------------------------
// workspace: one arena per handle, sized for `cap` right-hand sides
// --------------------------------------------------------------------------
struct BView {
    int nrhs;
    long long nf, nc;
    float2 *rA, *r, *tmp, *rs_, *ps;
    float2 *Z[BK_MAX], *W[BK_MAX], *Ps[BK_MAX], *Qs[BK_MAX];
    float2 *rc, *ec, *crr, *ct;
    float2 *Zc[BK_MAX], *Wc[BK_MAX];
    double2 *r64, *t64;
    float2** dptr;            // device pointer arrays: Z, W, Ps, Qs, Zc, Wc (BK_MAX each)
    double* mpart;            // Gram-Schmidt partials [nrhs][BK_MAX][2][BMDOT_BLOCKS]
    unsigned* mcount;         // Gram-Schmidt counters [nrhs][BK_MAX][CROW]
    RedScratch red;           // reductions: [nrhs][PROW] partials, [nrhs][CROW] counters
    BGcr *outer, *smooth, *cgcr;
    double *bn2, *rn2, *rA2, *ref2, *cref2, *scale, *rn;
    int *odone, *idone, *cdone, *iters, *citers, *csteps;
    double* pg_part;          // persistent coarse GCR (one right-hand side): partial sums
    unsigned* pg_bar;         // its grid barrier state (count, gen, error, pad)
    int* pg_iters;            // its step counter
    double* pg_rr2;
};

struct Carver {
    char* base;
    size_t off = 0;
    template <class T> T* take(size_t count) {
        off = (off + 255) & ~(size_t)255;
        T* p = reinterpret_cast<T*>(base ? base + off : nullptr);
        off += count * sizeof(T);
        return p;
    }
};

static void carve(const dwf_mg* h, int nrhs, char* base, BView& v, size_t* total, size_t* zero_begin,
                  size_t* zero_end) {
    Carver c{base};
    const int K = h->prm.gcr_restart, S = h->prm.post_smooth, KC = h->prm.coarse_restart;
    v.nrhs = nrhs;
    v.nf = fine_len(h);
    v.nc = coarse_len(h);
    const size_t F = (size_t)nrhs * v.nf, C = (size_t)nrhs * v.nc;
    v.rA = c.take<float2>(F); v.r = c.take<float2>(F);
    v.tmp = c.take<float2>(F); v.rs_ = c.take<float2>(F); v.ps = c.take<float2>(F);
    for (int k = 0; k < BK_MAX; ++k) {
        v.Z[k] = k < K ? c.take<float2>(F) : nullptr;
        v.W[k] = k < K ? c.take<float2>(F) : nullptr;
        v.Ps[k] = k < S ? c.take<float2>(F) : nullptr;
        v.Qs[k] = k < S ? c.take<float2>(F) : nullptr;
    }
    v.r64 = c.take<double2>(F); v.t64 = c.take<double2>(F);
    v.rc = c.take<float2>(C); v.ec = c.take<float2>(C); v.crr = c.take<float2>(C); v.ct = c.take<float2>(C);
    for (int k = 0; k < BK_MAX; ++k) {
        v.Zc[k] = k < KC ? c.take<float2>(C) : nullptr;
        v.Wc[k] = k < KC ? c.take<float2>(C) : nullptr;
    }
    v.dptr = c.take<float2*>(6 * BK_MAX);
    v.mpart = c.take<double>((size_t)nrhs * BK_MAX * 2 * BMDOT_BLOCKS);
    v.red.partials = c.take<double>((size_t)nrhs * PROW);
    v.outer = c.take<BGcr>(nrhs); v.smooth = c.take<BGcr>(nrhs); v.cgcr = c.take<BGcr>(nrhs);
    v.bn2 = c.take<double>(nrhs); v.rn2 = c.take<double>(nrhs); v.rA2 = c.take<double>(nrhs);
    v.ref2 = c.take<double>(nrhs); v.cref2 = c.take<double>(nrhs); v.scale = c.take<double>(nrhs);
    v.rn = c.take<double>(nrhs);
    v.pg_part = c.take<double>(64 * 1024);
    v.pg_rr2 = c.take<double>(1);
    // from here on the arena is zeroed once at allocation (counters must start at 0)
    c.off = (c.off + 255) & ~(size_t)255;
    *zero_begin = c.off;
    v.mcount = c.take<unsigned>((size_t)nrhs * BK_MAX * CROW);
    v.red.counter = c.take<unsigned>((size_t)nrhs * CROW);
    v.odone = c.take<int>(nrhs); v.idone = c.take<int>(nrhs); v.cdone = c.take<int>(nrhs);
    v.iters = c.take<int>(nrhs); v.citers = c.take<int>(nrhs); v.csteps = c.take<int>(nrhs);
    v.pg_bar = c.take<unsigned>(4);
    v.pg_iters = c.take<int>(1);
    *zero_end = c.off;
    *total = c.off;
}

struct BatchedState {
    void* arena = nullptr;
    int cap = 0;
    BView v{};
    int* hflags = nullptr;            // pinned: odone, idone, cdone, iters, citers [5][cap], + 2 spare
    double* hvals = nullptr;          // pinned: bn2, rn2, rA2, ref2, scale, rn [6][cap]
    cudaGraphExec_t gfirst = nullptr, gcycle = nullptr;
    int gnrhs = 0;                    // right-hand sides the graphs were captured for
    ~BatchedState() {
        if (gfirst) cudaGraphExecDestroy(gfirst);
        if (gcycle) cudaGraphExecDestroy(gcycle);
        if (arena) cudaFree(arena);
        if (hflags) cudaFreeHost(hflags);
        if (hvals) cudaFreeHost(hvals);
    }
};

static dwf_status ensure_batched(dwf_mg* h, int nrhs) {
    BatchedState*& bs = reinterpret_cast<BatchedState*&>(h->batched);
    if (bs && bs->cap >= nrhs) {
        if (bs->v.nrhs != nrhs) {
            size_t total, z0, z1;
            carve(h, nrhs, (char*)bs->arena, bs->v, &total, &z0, &z1);
            // a different row count moves the carved regions: zero the counters and flags again
            DWF_CHECK_CUDA(cudaStreamSynchronize(h->st));
            DWF_CHECK_CUDA(cudaMemset((char*)bs->arena + z0, 0, z1 - z0));
        }
    } else {
        if (bs) {
            cudaStreamSynchronize(h->st);
            delete bs;
            bs = nullptr;
        }
        BatchedState* n = new (std::nothrow) BatchedState();
        if (!n) { set_error("host allocation failed"); return DWF_ERR_OOM; }
        size_t total, z0, z1;
        carve(h, nrhs, nullptr, n->v, &total, &z0, &z1);
        cudaError_t e = cudaMalloc(&n->arena, total);
        if (e != cudaSuccess) {
            delete n;
            set_error("batched solver workspace of %zu bytes: %s", total, cudaGetErrorString(e));
            return DWF_ERR_OOM;
        }
        carve(h, nrhs, (char*)n->arena, n->v, &total, &z0, &z1);
        if (cudaMemset((char*)n->arena + z0, 0, z1 - z0) != cudaSuccess ||
            cudaMallocHost((void**)&n->hflags, (5 * nrhs + 2) * sizeof(int)) != cudaSuccess ||
            cudaMallocHost((void**)&n->hvals, 6 * sizeof(double) * nrhs) != cudaSuccess) {
            delete n;
            set_error("batched solver workspace setup failed");
            return DWF_ERR_OOM;
        }
        n->cap = nrhs;
        bs = n;
    }
    BView& v = bs->v;
    float2* hp[6 * BK_MAX];
    for (int k = 0; k < BK_MAX; ++k) {
        hp[0 * BK_MAX + k] = v.Z[k]; hp[1 * BK_MAX + k] = v.W[k];
        hp[2 * BK_MAX + k] = v.Ps[k]; hp[3 * BK_MAX + k] = v.Qs[k];
        hp[4 * BK_MAX + k] = v.Zc[k]; hp[5 * BK_MAX + k] = v.Wc[k];
    }
    DWF_CHECK_CUDA(cudaMemcpy(v.dptr, hp, sizeof(hp), cudaMemcpyHostToDevice));
    if (bs->gnrhs != nrhs) {
        if (bs->gfirst) cudaGraphExecDestroy(bs->gfirst);
        if (bs->gcycle) cudaGraphExecDestroy(bs->gcycle);
        bs->gfirst = bs->gcycle = nullptr;
        bs->gnrhs = 0;
    }
    return DWF_OK;
}

// --------------------------------------------------------------------------
// solver
// --------------------------------------------------------------------------
struct BSolver {
    dwf_mg* h;
    BatchedState* bs;
    BView* v;
    cudaStream_t st;
    int nrhs;
    bool pk = false;             // FP32 fine vectors in the slice-paired layout (4-d, one right-hand side)
    long long l3_iters = 0;      // coarsest iterations of a three-level hierarchy
    long long l3_solves = 0;     // and coarsest solves
};

static dim3 row_grid(long long n2, int nrhs, int cap = 1216) {
    long long b = (n2 + 255) / 256;
    if (b < 1) b = 1;
    if (b > cap) b = cap;
    return dim3((unsigned)b, (unsigned)nrhs);
}

static dwf_status bapply_A(BSolver& s, const float2* in, float2* out, const int* skip) {
    dwf_mg* h = s.h;
    if (s.pk) {
        DWF_TRY(fine_apply_4d_paired(h->G, h->Upk, in, s.v->tmp, h->M5, h->mf, false, h->prm.fine_prec, s.st, skip));
        return fine_apply_4d_paired(h->G, h->Upk, s.v->tmp, out, h->M5, 1.0, true, h->prm.fine_prec, s.st, skip);
    }
    DWF_TRY(fine_apply_rhs(h->G, h->Ulo, in, s.v->tmp, h->M5, h->mf, false, h->prm.fine_prec, s.nrhs, skip, s.st));
    DWF_TRY(fine_apply_rhs(h->G, h->Ulo, s.v->tmp, out, h->M5, 1.0, true, h->prm.fine_prec, s.nrhs, skip, s.st));
    return DWF_OK;
}

// Orthogonalise Wb[k] against Wb[0..k-1] (classical Gram-Schmidt, cgs_passes
// passes), then nrm[k], alpha = A[k] = <w, res> / |w|^2; steps[r] = k + 1.
static dwf_status borthogonalise(BSolver& s, BGcr* g, float2* const* Wb, int k, const float2* res, long long n,
                                 float2* const* dW, int* steps, const int* skip) {
    BView& v = *s.v;
    const int rg = red_grid4(n);
    const dim3 rgrid((unsigned)rg, (unsigned)s.nrhs);
    if (k > 0) {
        const bool fused = n >= BMDOT_FUSE_N;
        const int nb = fused ? BMDOT_BLOCKS : BMDOT_ROW_BLOCKS;
        const dim3 mgrid((unsigned)(rg < nb ? rg : nb), fused ? (unsigned)s.nrhs : (unsigned)k,
                         fused ? 1u : (unsigned)s.nrhs);
        const dim3 egrid = row_grid(n >> 1, s.nrhs, 152 * 16);
        const int passes = s.h->prm.cgs_passes;
        for (int pass = 0; pass < passes; ++pass) {
            if (fused) launch_bmdot(mgrid, dW, Wb[k], n, k, v.mpart, v.mcount, g, pass == 0, skip, s.st);
            else k_bmdot_rows<<<mgrid, RED_THREADS, 0, s.st>>>(dW, Wb[k], n, v.mpart, v.mcount, g, pass == 0, skip);
            if (pass + 1 < passes)
                k_bmaxpy<false><<<egrid, RED_THREADS, 0, s.st>>>(Wb[k], dW, g, k, res, n, v.red, steps, skip);
            else
                k_bmaxpy<true><<<rgrid, RED_THREADS, 0, s.st>>>(Wb[k], dW, g, k, res, n, v.red, steps, skip);
        }
    } else {
        k_bmaxpy<true><<<rgrid, RED_THREADS, 0, s.st>>>(Wb[0], dW, g, 0, res, n, v.red, steps, skip);
    }
    DWF_CHECK_LAUNCH();
    return DWF_OK;
}

// Coarse GCR on every right-hand side with idone == 0 (cdone starts as a copy
// of idone).  The residual at the start of a restart cycle is crr; step k
// keeps its residual in Zc[k] (the raw direction of step k) and writes the
// next one to Zc[k + 1], or to crr after the last step; the cycle ends with
// ec += sum_j y_j Zc[j] over the csteps[r] steps that right-hand side took.
static dwf_status bcoarse_prologue(BSolver& s) {
    BView& v = *s.v;
    const long long n = v.nc;
    DWF_CHECK_CUDA(cudaMemsetAsync(v.ec, 0, (size_t)s.nrhs * n * sizeof(float2), s.st));
    DWF_CHECK_CUDA(cudaMemcpyAsync(v.crr, v.rc, (size_t)s.nrhs * n * sizeof(float2), cudaMemcpyDeviceToDevice, s.st));
    DWF_CHECK_CUDA(cudaMemcpyAsync(v.cdone, v.idone, s.nrhs * sizeof(int), cudaMemcpyDeviceToDevice, s.st));
    DWF_CHECK_CUDA(cudaMemsetAsync(v.citers, 0, s.nrhs * sizeof(int), s.st));
    k_bnorm2_32<<<dim3((unsigned)red_grid4(n), (unsigned)s.nrhs), RED_THREADS, 0, s.st>>>(v.rc, n, v.red, v.cref2,
                                                                                           v.idone);
    DWF_CHECK_LAUNCH();
    return DWF_OK;
}

static dwf_status bcoarse_cycle(BSolver& s) {
    dwf_mg* h = s.h;
    BView& v = *s.v;
    const long long n = v.nc;
    const int KC = h->prm.coarse_restart;
    const double tol2 = h->prm.coarse_tol * h->prm.coarse_tol;
    const dim3 eg = row_grid(n >> 1, s.nrhs);
    const dim3 rg((unsigned)red_grid4(n), (unsigned)s.nrhs);
    DWF_CHECK_CUDA(cudaMemsetAsync(v.csteps, 0, s.nrhs * sizeof(int), s.st));
    k_bcopy<<<eg, 256, 0, s.st>>>(v.Zc[0], v.crr, n, v.cdone);
    DWF_CHECK_LAUNCH();
    for (int k = 0; k < KC; ++k) {
        if (s.nrhs == 1) {
            // one column: the shared-memory tile stencil has the shorter latency
            DWF_TRY(coarse_dwf_apply(h, v.Zc[k], v.ct, h->mf, false, v.cdone, s.st));
            DWF_TRY(coarse_dwf_apply(h, v.ct, v.Wc[k], 1.0, true, v.cdone, s.st));
        } else {
            DWF_TRY(coarse_apply_multi_tc(h, s.nrhs, v.Zc[k], v.ct, h->mf, false, v.cdone, s.st));
            DWF_TRY(coarse_apply_multi_tc(h, s.nrhs, v.ct, v.Wc[k], 1.0, true, v.cdone, s.st));
        }
        float2* rnext = k + 1 < KC ? v.Zc[k + 1] : v.crr;
        if (h->prm.cgs_passes == 1) {
            // one reduction pass and one element-wise pass per step
            const dim3 dg((unsigned)(rg.x < BSTEP_BLOCKS ? rg.x : BSTEP_BLOCKS), (unsigned)s.nrhs);
            launch_bstep_dots(dg, v.dptr + 5 * BK_MAX, v.Wc[k], v.Zc[k], n, k, v.mpart, v.mcount, v.cgcr, v.csteps,
                              v.cdone, v.cref2, tol2, v.citers, h->prm.coarse_maxiter, s.st);
            k_bstep_update<<<eg, RED_THREADS, 0, s.st>>>(v.Wc[k], v.dptr + 5 * BK_MAX, v.cgcr, k, v.Zc[k], rnext, n,
                                                         v.cdone);
        } else {
            DWF_TRY(borthogonalise(s, v.cgcr, v.Wc, k, v.Zc[k], n, v.dptr + 5 * BK_MAX, v.csteps, v.cdone));
            k_bres_update<<<rg, RED_THREADS, 0, s.st>>>(v.Zc[k], rnext, v.Wc[k], v.cgcr, n, v.red, v.cdone, v.cdone,
                                                        v.cref2, tol2, v.citers, h->prm.coarse_maxiter);
        }
        DWF_CHECK_LAUNCH();
    }
    k_bcombine32<<<eg, RED_THREADS, 0, s.st>>>(v.ec, v.dptr + 4 * BK_MAX, v.cgcr, v.csteps, 0, n, nullptr, nullptr,
                                               nullptr, nullptr);
    DWF_CHECK_LAUNCH();
    return DWF_OK;
}

static dwf_status bcapture(BSolver& s, bool with_prologue, cudaGraphExec_t* out) {
    cudaGraph_t graph = nullptr;
    if (!s.h->cap_stream) DWF_CHECK_CUDA(cudaStreamCreateWithFlags(&s.h->cap_stream, cudaStreamNonBlocking));
    const cudaStream_t user = s.st;
    s.st = s.h->cap_stream;
    DWF_CHECK_CUDA(cudaStreamBeginCapture(s.st, cudaStreamCaptureModeThreadLocal));
    dwf_status st = DWF_OK;
    if (with_prologue) st = bcoarse_prologue(s);
    if (st == DWF_OK) st = bcoarse_cycle(s);
    cudaError_t e = cudaStreamEndCapture(s.st, &graph);
    s.st = user;
    if (st != DWF_OK) { if (graph) cudaGraphDestroy(graph); return st; }
    if (e != cudaSuccess) { set_error("graph capture: %s", cudaGetErrorString(e)); return DWF_ERR_CUDA; }
    e = cudaGraphInstantiate(out, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) { set_error("graph instantiation: %s", cudaGetErrorString(e)); return DWF_ERR_CUDA; }
    return DWF_OK;
}

// runs the coarse GCR until every active right-hand side is done; citers_out[r]
// receives the iterations of right-hand side r
static dwf_status bcoarse_solve(BSolver& s, int* citers_out) {
    dwf_mg* h = s.h;
    BatchedState* bs = s.bs;
    BView& v = *s.v;
    if (s.nrhs == 1 && h->prm.coarse_persistent == 2 && coarse_gcr_persistent_ok(h)) {
        // one right-hand side: the whole coarse GCR in one cooperative launch
        const int KC = h->prm.coarse_restart;
        float2* S[BK_MAX + 1];
        for (int k = 0; k < KC; ++k) S[k] = v.Zc[k];
        S[KC] = v.crr;
        DWF_CHECK_CUDA(cudaMemsetAsync(v.pg_iters, 0, sizeof(int), s.st));
        DWF_TRY(coarse_gcr_persistent(h, v.rc, v.ec, S, v.Wc, v.ct, v.pg_part, v.pg_bar, v.pg_iters, v.pg_rr2,
                                      s.st));
        unsigned* hb = reinterpret_cast<unsigned*>(bs->hflags + 5 * bs->cap);   // spare slot
        DWF_CHECK_CUDA(cudaMemcpyAsync(citers_out, v.pg_iters, sizeof(int), cudaMemcpyDeviceToHost, s.st));
        DWF_CHECK_CUDA(cudaMemcpyAsync(hb, v.pg_bar + 2, sizeof(unsigned), cudaMemcpyDeviceToHost, s.st));
        DWF_CHECK_CUDA(cudaStreamSynchronize(s.st));
        if (*hb != 0u) { set_error("persistent coarse GCR: a grid barrier or bulk copy timed out"); return DWF_ERR_TIMEOUT; }
        return DWF_OK;
    }
    if (!bs->gfirst) {
        // the contraction's form is chosen by timing, before it is frozen into the graphs
        if (s.nrhs > 1 && h->prm.coarse_tc == 0) DWF_TRY(coarse_tc_tune(h, s.nrhs, v.Zc[0], v.ct, s.st));
        DWF_TRY(bcapture(s, true, &bs->gfirst));
        DWF_TRY(bcapture(s, false, &bs->gcycle));
        bs->gnrhs = s.nrhs;
    }
    int* hcd = bs->hflags + 2 * bs->cap;
    int launched = 0;
    for (;;) {
        DWF_CHECK_CUDA(cudaGraphLaunch(launched == 0 ? bs->gfirst : bs->gcycle, s.st));
        launched += h->prm.coarse_restart;
        DWF_CHECK_CUDA(cudaMemcpyAsync(hcd, v.cdone, s.nrhs * sizeof(int), cudaMemcpyDeviceToHost, s.st));
        DWF_CHECK_CUDA(cudaStreamSynchronize(s.st));
        bool all = true;
        for (int r = 0; r < s.nrhs; ++r) all = all && hcd[r];
        if (all || launched >= h->prm.coarse_maxiter) break;
    }
    DWF_CHECK_CUDA(cudaMemcpyAsync(citers_out, v.citers, s.nrhs * sizeof(int), cudaMemcpyDeviceToHost, s.st));
    DWF_CHECK_CUDA(cudaStreamSynchronize(s.st));
    return DWF_OK;
}

// z = M(r) and w = A z for every right-hand side with idone == 0.  The
// smoother's step j keeps its residual in Ps[j] and writes the next one to
// Ps[j + 1] (rs_ after the last step); z += sum_j y_j Ps[j] and w = r - rs_
// come out of one final pass.
static dwf_status bprecondition(BSolver& s, const float2* res, float2* zout, float2* wout, int* citers_out) {
    dwf_mg* h = s.h;
    BView& v = *s.v;
    const long long n = v.nf;
    const dim3 eg = row_grid(n >> 1, s.nrhs);
    DWF_TRY(restrict_wall(h, res, v.rc, v.idone, s.st, s.nrhs, s.pk));
    if (h->lvl3) {
        // three levels: flexible GCR on the intermediate level, preconditioned by the coarsest solve
        int l2 = 0, l3 = 0;
        DWF_TRY(level2_solve(h, v.rc, v.ec, &l2, &l3, s.st));
        citers_out[0] = l2;
        s.l3_iters += l3;
        s.l3_solves += l2;
    } else {
        DWF_TRY(bcoarse_solve(s, citers_out));
    }
    DWF_TRY(prolong_wall(h, v.ec, zout, v.idone, s.st, s.nrhs, s.pk));
    const int S = h->prm.post_smooth;
    if (S == 0) return bapply_A(s, zout, wout, v.idone);
    DWF_TRY(bapply_A(s, zout, v.ps, v.idone));
    k_bsub32<<<eg, 256, 0, s.st>>>(v.Ps[0], res, v.ps, n, v.idone);
    DWF_CHECK_LAUNCH();
    const dim3 rg((unsigned)red_grid4(n), (unsigned)s.nrhs);
    for (int j = 0; j < S; ++j) {
        DWF_TRY(bapply_A(s, v.Ps[j], v.Qs[j], v.idone));
        DWF_TRY(borthogonalise(s, v.smooth, v.Qs, j, v.Ps[j], n, v.dptr + 3 * BK_MAX, nullptr, v.idone));
        k_bres_update<<<rg, RED_THREADS, 0, s.st>>>(v.Ps[j], j + 1 < S ? v.Ps[j + 1] : v.rs_, v.Qs[j], v.smooth, n,
                                                    v.red, v.idone, nullptr, nullptr, 0.0, nullptr, 0);
        DWF_CHECK_LAUNCH();
    }
    k_bcombine32<<<eg, RED_THREADS, 0, s.st>>>(zout, v.dptr + 2 * BK_MAX, v.smooth, nullptr, S, n, res, v.rs_, wout,
                                               v.idone);
    DWF_CHECK_LAUNCH();
    return DWF_OK;
}

}  // namespace

void batched_state_free(dwf_mg* h) {
    if (h && h->batched) {
        delete reinterpret_cast<BatchedState*>(h->batched);
        h->batched = nullptr;
    }
}

dwf_status mg_solve_batched_impl(dwf_mg* h, int nrhs, const double2* B, double2* X, double tol, int maxiter,
                                 dwf_solve_stats* stats) {
    auto t0 = std::chrono::steady_clock::now();
    if (stats) memset(stats, 0, sizeof(*stats) * (size_t)(nrhs > 0 ? nrhs : 0));
    if (!h || !B || !X) { set_error("NULL argument"); return DWF_ERR_ARG; }
    if (nrhs < 1 || nrhs > 65535) { set_error("nrhs must be in [1, 65535]"); return DWF_ERR_ARG; }
    if (!(tol > 0.0)) { set_error("tol must be > 0"); return DWF_ERR_ARG; }
    if (nrhs > 1 && h->lvl3) {
        set_error("a three-level hierarchy solves one right-hand side per call");
        return DWF_ERR_UNSUPPORTED;
    }
    if (nrhs > 1 && (h->mg.nd != 2 || h->mg.ncd != 16)) {
        set_error("more than one right-hand side per hierarchy needs a 2-d lattice with nvec = 8");
        return DWF_ERR_UNSUPPORTED;
    }
    if (h->prm.gcr_restart < 1 || h->prm.gcr_restart > BK_MAX || h->prm.post_smooth > BK_MAX ||
        h->prm.coarse_restart < 1 || h->prm.coarse_restart > BK_MAX) {
        set_error("gcr_restart, post_smooth and coarse_restart must be in [1, %d]", BK_MAX); return DWF_ERR_ARG;
    }
    DWF_TRY(ensure_batched(h, nrhs));
    BSolver s;
    s.h = h;
    s.bs = reinterpret_cast<BatchedState*>(h->batched);
    s.v = &s.bs->v;
    s.st = h->st;
    s.nrhs = nrhs;
    s.pk = h->pk != 0 && nrhs == 1;
    const PackIdx pq{h->G.V, (h->G.V + 31) / 32, (int)site_dof(h->G)};
    BView& v = *s.v;
    BatchedState& bs = *s.bs;
    const long long n = v.nf;
    const int cap = bs.cap;
    int* hod = bs.hflags;             // odone
    int* hid = bs.hflags + cap;       // idone
    int* hit = bs.hflags + 3 * cap;   // iters
    int* hci = bs.hflags + 4 * cap;   // coarse iterations of the last coarse solve
    double* hbn2 = bs.hvals;
    double* hrn2 = bs.hvals + cap;
    double* hrA2 = bs.hvals + 2 * cap;
    double* href2 = bs.hvals + 3 * cap;
    double* hscale = bs.hvals + 4 * cap;
    double* hrn = bs.hvals + 5 * cap;
    const dim3 eg64 = row_grid(n, nrhs);
    const dim3 eg32 = row_grid(n >> 1, nrhs);
    const dim3 rg64((unsigned)red_grid(n), (unsigned)nrhs);
    const dim3 rg32((unsigned)red_grid4(n), (unsigned)nrhs);

    DWF_CHECK_CUDA(cudaMemsetAsync(X, 0, (size_t)nrhs * n * sizeof(double2), s.st));
    k_bnorm2_64<<<rg64, RED_THREADS, 0, s.st>>>(B, n, v.red, v.bn2, nullptr);
    DWF_CHECK_LAUNCH();
    DWF_CHECK_CUDA(cudaMemcpyAsync(hbn2, v.bn2, nrhs * sizeof(double), cudaMemcpyDeviceToHost, s.st));
    DWF_CHECK_CUDA(cudaStreamSynchronize(s.st));

    std::vector<int> outer(nrhs, 0), restarts(nrhs, 0), conv(nrhs, 0);
    std::vector<long long> fine(nrhs, 0), coarse_it(nrhs, 0), coarse_solves(nrhs, 0);
    std::vector<double> res(nrhs, 1.0);
    for (int r = 0; r < nrhs; ++r) {
        hod[r] = 0;
        if (hbn2[r] == 0.0) { hod[r] = 1; conv[r] = 1; res[r] = 0.0; }
    }
    const int K = h->prm.gcr_restart, S = h->prm.post_smooth;
    bool first = true;
    for (;;) {
        if (first) {
            DWF_CHECK_CUDA(cudaMemcpyAsync(v.r64, B, (size_t)nrhs * n * sizeof(double2), cudaMemcpyDeviceToDevice,
                                           s.st));
            for (int r = 0; r < nrhs; ++r) hrn2[r] = hbn2[r];
            first = false;
        } else {
            DWF_CHECK_CUDA(cudaMemcpyAsync(v.odone, hod, nrhs * sizeof(int), cudaMemcpyHostToDevice, s.st));
            DWF_TRY(fine_apply_rhs(h->G, h->U64, X, v.t64, h->M5, h->mf, false, DWF_F64, nrhs, v.odone, s.st));
            k_bsub64<<<eg64, 256, 0, s.st>>>(v.r64, B, v.t64, n, v.odone);
            k_bnorm2_64<<<rg64, RED_THREADS, 0, s.st>>>(v.r64, n, v.red, v.rn2, v.odone);
            DWF_CHECK_LAUNCH();
            DWF_CHECK_CUDA(cudaMemcpyAsync(hrn2, v.rn2, nrhs * sizeof(double), cudaMemcpyDeviceToHost, s.st));
            DWF_CHECK_CUDA(cudaStreamSynchronize(s.st));
            for (int r = 0; r < nrhs; ++r) if (!hod[r]) fine[r] += 1;
        }
        bool any = false;
        for (int r = 0; r < nrhs; ++r) {
            if (hod[r]) continue;
            res[r] = sqrt(hrn2[r] / hbn2[r]);
            if (res[r] <= tol) { hod[r] = 1; conv[r] = 1; continue; }
            if (outer[r] >= maxiter || restarts[r] > h->prm.max_restarts) { hod[r] = 1; continue; }
            any = true;
        }
        if (!any) break;
        for (int r = 0; r < nrhs; ++r) {
            hid[r] = hod[r];
            hrn[r] = hod[r] ? 0.0 : sqrt(hrn2[r]);
            hscale[r] = hod[r] ? 0.0 : 1.0 / hrn[r];
            if (!hod[r]) { restarts[r] += 1; fine[r] += 1; }
        }
        DWF_CHECK_CUDA(cudaMemcpyAsync(v.odone, hod, nrhs * sizeof(int), cudaMemcpyHostToDevice, s.st));
        DWF_CHECK_CUDA(cudaMemcpyAsync(v.idone, hid, nrhs * sizeof(int), cudaMemcpyHostToDevice, s.st));
        DWF_CHECK_CUDA(cudaMemcpyAsync(v.scale, hscale, nrhs * sizeof(double), cudaMemcpyHostToDevice, s.st));
        DWF_CHECK_CUDA(cudaMemcpyAsync(v.rn, hrn, nrhs * sizeof(double), cudaMemcpyHostToDevice, s.st));
        // correction system in FP32: A e = D_PV^dag r / |r|
        if (s.pk) {
            k_bd2f_scale_pk<<<eg32, 256, 0, s.st>>>(v.ps, v.r64, v.scale, n, v.idone, pq);
            DWF_CHECK_LAUNCH();
            DWF_TRY(fine_apply_4d_paired(h->G, h->Upk, v.ps, v.rA, h->M5, 1.0, true, h->prm.fine_prec, s.st, v.idone));
        } else {
            k_bd2f_scale<<<eg64, 256, 0, s.st>>>(v.ps, v.r64, v.scale, n, v.idone);
            DWF_CHECK_LAUNCH();
            DWF_TRY(fine_apply_rhs(h->G, h->Ulo, v.ps, v.rA, h->M5, 1.0, true, h->prm.fine_prec, nrhs, v.idone, s.st));
        }
        k_bcopy<<<eg32, 256, 0, s.st>>>(v.r, v.rA, n, v.idone);
        k_bnorm2_32<<<rg32, RED_THREADS, 0, s.st>>>(v.rA, n, v.red, v.rA2, v.idone);
        DWF_CHECK_LAUNCH();
        DWF_CHECK_CUDA(cudaMemcpyAsync(hrA2, v.rA2, nrhs * sizeof(double), cudaMemcpyDeviceToHost, s.st));
        DWF_CHECK_CUDA(cudaStreamSynchronize(s.st));
        for (int r = 0; r < nrhs; ++r) {
            if (hid[r]) { href2[r] = 0.0; continue; }
            double delta = h->prm.inner_tol;
            const double need = 0.5 * tol * sqrt(hbn2[r]) / hrn[r];
            if (need > delta) delta = need;
            href2[r] = delta * delta * hrA2[r];
        }
        DWF_CHECK_CUDA(cudaMemcpyAsync(v.ref2, href2, nrhs * sizeof(double), cudaMemcpyHostToDevice, s.st));
        DWF_CHECK_CUDA(cudaMemsetAsync(v.iters, 0, nrhs * sizeof(int), s.st));
        const dim3 rg((unsigned)red_grid4(n), (unsigned)nrhs);
        for (int k = 0; k < K; ++k) {
            bool active = false;
            for (int r = 0; r < nrhs; ++r) active = active || !hid[r];
            if (!active) break;
            DWF_TRY(bprecondition(s, v.r, v.Z[k], v.W[k], hci));
            for (int r = 0; r < nrhs; ++r)
                if (!hid[r]) { coarse_it[r] += hci[r]; coarse_solves[r] += 1; fine[r] += 2 + 2 * S; outer[r] += 1; }
            DWF_TRY(borthogonalise(s, v.outer, v.W, k, v.r, n, v.dptr + 1 * BK_MAX, nullptr, v.idone));
            k_bres_update<<<rg, RED_THREADS, 0, s.st>>>(v.r, v.r, v.W[k], v.outer, n, v.red, v.idone, v.idone,
                                                        v.ref2, 1.0, v.iters, K);
            DWF_CHECK_LAUNCH();
            DWF_CHECK_CUDA(cudaMemcpyAsync(hid, v.idone, nrhs * sizeof(int), cudaMemcpyDeviceToHost, s.st));
            DWF_CHECK_CUDA(cudaStreamSynchronize(s.st));
            for (int r = 0; r < nrhs; ++r)
                if (!hod[r] && outer[r] >= maxiter) hid[r] = 1;    // iteration cap: leave the cycle
            DWF_CHECK_CUDA(cudaMemcpyAsync(v.idone, hid, nrhs * sizeof(int), cudaMemcpyHostToDevice, s.st));
        }
        // x += |r| sum_k y_k Z_k over the iters[r] steps of this cycle
        if (s.pk)
            k_bcombine64_pk<<<row_grid(n >> 1, 1), RED_THREADS, 0, s.st>>>(X, v.dptr + 0 * BK_MAX, v.outer, v.iters,
                                                                            v.rn, n, pq);
        else
            k_bcombine64<<<row_grid(n >> 1, nrhs), RED_THREADS, 0, s.st>>>(X, v.dptr + 0 * BK_MAX, v.outer, v.iters,
                                                                            v.rn, n);
        DWF_CHECK_LAUNCH();
    }
    (void)hit;
    {
        int st1 = 0;    // bounded bulk-copy waits of the tile stencil (one-column coarse solves)
        DWF_CHECK_CUDA(cudaMemcpyAsync(&st1, h->status + 1, sizeof(int), cudaMemcpyDeviceToHost, s.st));
        DWF_CHECK_CUDA(cudaStreamSynchronize(s.st));
        if (st1 != 0) {
            set_error("coarse stencil: a bulk copy wait timed out");
            return DWF_ERR_TIMEOUT;
        }
    }
    int nconv = 0;
    for (int r = 0; r < nrhs; ++r) nconv += conv[r];
    const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (stats)
        for (int r = 0; r < nrhs; ++r) {
            stats[r].iterations = outer[r];
            stats[r].restarts = restarts[r];
            stats[r].fine_applies = fine[r];
            stats[r].coarse_applies = 2 * coarse_it[r];
            stats[r].coarse_avg_iters = coarse_solves[r] ? (double)coarse_it[r] / coarse_solves[r] : 0.0;
            stats[r].coarsest_avg_iters = s.l3_solves ? (double)s.l3_iters / s.l3_solves : 0.0;
            stats[r].true_residual = res[r];
            stats[r].seconds = secs;
        }
    if (nconv < nrhs) {
        double worst = 0.0;
        for (int r = 0; r < nrhs; ++r) if (!conv[r] && res[r] > worst) worst = res[r];
        set_error("mg_solve_batched: %d of %d right-hand sides stopped above tol %.3e (worst %.3e)", nrhs - nconv,
                  nrhs, tol, worst);
        return DWF_ERR_NOCONV;
    }
    return DWF_OK;
}

}  // namespace dwf

using namespace dwf;

extern "C" dwf_status mg_solve_batched(dwf_mg* h, int nrhs, const void* b, void* x, double tol, int maxiter,
                                       dwf_solve_stats* stats, void* stream) {
    clear_error();
    if (h && stream) h->st = as_stream(stream);
    return mg_solve_batched_impl(h, nrhs, (const double2*)b, (double2*)x, tol, maxiter, stats);
}

extern "C" dwf_status mg_solve_groups(int ngroups, dwf_mg* const* handles, const int* nrhs, const void* const* b,
                                      void* const* x, double tol, int maxiter, dwf_solve_stats* const* stats) {
    clear_error();
    if (ngroups < 1 || !handles || !nrhs || !b || !x) { set_error("NULL argument or ngroups < 1"); return DWF_ERR_ARG; }
    for (int i = 0; i < ngroups; ++i) {
        if (!handles[i]) { set_error("handle %d is NULL", i); return DWF_ERR_ARG; }
        for (int j = 0; j < i; ++j)
            if (handles[j] == handles[i]) { set_error("handles %d and %d are the same hierarchy", j, i); return DWF_ERR_ARG; }
    }
    // each hierarchy gets its own non-blocking stream and host thread, so the
    // groups' launches overlap on the device
    std::vector<cudaStream_t> streams(ngroups, nullptr);
    std::vector<cudaStream_t> saved(ngroups, nullptr);
    for (int i = 0; i < ngroups; ++i) {
        if (cudaStreamCreateWithFlags(&streams[i], cudaStreamNonBlocking) != cudaSuccess) {
            for (int j = 0; j < i; ++j) cudaStreamDestroy(streams[j]);
            set_error("stream creation failed");
            return DWF_ERR_CUDA;
        }
        saved[i] = handles[i]->st;
    }
    // the caller's prior work on the handles' streams must be complete
    for (int i = 0; i < ngroups; ++i) cudaStreamSynchronize(saved[i]);
    std::vector<dwf_status> st(ngroups, DWF_OK);
    std::vector<std::string> msg(ngroups);
    int dev = 0;
    cudaGetDevice(&dev);
    std::vector<std::thread> th;
    for (int i = 0; i < ngroups; ++i) {
        th.emplace_back([&, i]() {
            cudaSetDevice(dev);
            handles[i]->st = streams[i];
            st[i] = mg_solve_batched_impl(handles[i], nrhs[i], (const double2*)b[i], (double2*)x[i], tol, maxiter,
                                          stats ? stats[i] : nullptr);
            if (st[i] != DWF_OK) msg[i] = dwf_last_error();
            cudaStreamSynchronize(streams[i]);
        });
    }
    for (auto& t : th) t.join();
    dwf_status out = DWF_OK;
    for (int i = 0; i < ngroups; ++i) {
        handles[i]->st = saved[i];
        cudaStreamDestroy(streams[i]);
        if (st[i] != DWF_OK && out == DWF_OK) {
            out = st[i];
            set_error("group %d: %s", i, msg[i].c_str());
        }
    }
    return out;
}
