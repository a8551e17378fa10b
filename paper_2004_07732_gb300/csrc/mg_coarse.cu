// Coarse-level operators of the multigrid (Sec. 2.3):
//   * the coarse Shamir operator Dhat_DW(m) of Eq. coarsenDW: on every coarse
//     slice the Galerkin kernel Dhat_W (self block + one block per hop
//     direction) plus 1, the Phat_pm = (1 pm sigma_3)/2 s-hops and the -m wall
//     terms; the adjoint uses the transposed neighbour blocks, so it is the
//     exact adjoint of the stored operator;
//   * truncated wall restriction / prolongation (Eq. TruncProjectInterpolate).
// Coarse vectors are [s][coarse site][chirality][vec], complex64.
#include <mutex>

#include "mg.cuh"
#include "async_copy.cuh"
#include "mma_tf32.cuh"

namespace dwf {

__device__ __forceinline__ long long coarse_neighbour(const CoarseParams& p, long long xc, int dir) {
    if (dir == 0) return xc;
    const int mu = (dir - 1) >> 1;
    const int step = ((dir - 1) & 1) ? -1 : 1;
    // extent and stride of direction mu without indexing the parameter arrays dynamically
    const long long L0 = p.Lc[0], L1 = p.Lc[1], L2 = p.Lc[2], L3 = p.Lc[3];
    const long long Lm = mu == 0 ? L0 : mu == 1 ? L1 : mu == 2 ? L2 : L3;
    const long long stride = mu == 0 ? 1 : mu == 1 ? L0 : mu == 2 ? L0 * L1 : L0 * L1 * L2;
    const long long c = (xc / stride) % Lm;
    long long cn = c + step;
    if (cn < 0) cn += Lm;
    if (cn >= Lm) cn -= Lm;
    return xc + (cn - c) * stride;
}

__device__ __forceinline__ float2 cfma(float2 a, float2 b, float2 acc) {
    acc.x = fmaf(a.x, b.x, fmaf(-a.y, b.y, acc.x));
    acc.y = fmaf(a.x, b.y, fmaf(a.y, b.x, acc.y));
    return acc;
}
__device__ __forceinline__ float2 cfma_conj(float2 a, float2 b, float2 acc) {   // conj(a) * b
    acc.x = fmaf(a.x, b.x, fmaf(a.y, b.y, acc.x));
    acc.y = fmaf(a.x, b.y, fmaf(-a.y, b.x, acc.y));
    return acc;
}

// One warp per coarse site.  B holds (2 nvec)^2 blocks column-major per
// [coarse site][dir]: the Galerkin blocks of Dhat_W for the operator, or the
// pre-transposed blocks of Dhat_W^dag (block (x, dir) = Y(x + dir, -dir)^dag)
// for the adjoint, so both read B coalesced.  Lane l owns rows
// i = (l & 15) + 16 k and slices s = 8 g + (l >> 4) + 2 k' (g = 0, 1, .. for Ls_c > 8); the j loop is unrolled so
// every block and input load of a direction is in flight together.  CG = true
// reads the input through L2 (other blocks of a persistent launch wrote it).
// Returns the lane's share of |out|^2.
template <int NCD, bool CG>
__device__ __forceinline__ double warp_site_apply(const float2* __restrict__ B, const float2* __restrict__ in,
                                                  float2* __restrict__ out, const CoarseParams& p, long long xc,
                                                  float mf, bool dag, int lane) {
    const int ncd = NCD > 0 ? NCD : p.ncd;
    const long long slice = p.Vc * ncd;
    const long long bsz = (long long)ncd * ncd;
    const int sg = lane >> 4;
    double nrm = 0.0;
    // slices in groups of 8 (the blocks of a later group come from L1/L2)
    for (int s0 = 0; s0 < p.Ls_c; s0 += 8)
    for (int i = lane & 15; i < ncd; i += 16) {
        float2 acc[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int s = s0 + sg + 2 * k;
            acc[k] = make_float2(0.f, 0.f);
            if (s < p.Ls_c) acc[k] = CG ? __ldcg(in + s * slice + xc * ncd + i) : __ldg(in + s * slice + xc * ncd + i);
        }
        for (int dir = 0; dir < p.ndir; ++dir) {
            const long long nb = coarse_neighbour(p, xc, dir);
            const float2* Bb = B + (xc * p.ndir + dir) * bsz + i;
            const float2* v = in + nb * ncd;
#pragma unroll
            for (int j = 0; j < ncd; ++j) {
                const float2 y = __ldg(Bb + (long long)j * ncd);
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const int s = s0 + sg + 2 * k;
                    if (s < p.Ls_c) acc[k] = cfma(y, CG ? __ldcg(v + s * slice + j) : __ldg(v + s * slice + j), acc[k]);
                }
            }
        }
        const int c = i / p.nvec;
        const bool from_below = dag ? (c == 1) : (c == 0);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int s = s0 + sg + 2 * k;
            if (s >= p.Ls_c) break;
            long long hi;
            float sc = 1.f;
            if (from_below) { if (s > 0) hi = (s - 1) * slice; else { hi = (p.Ls_c - 1) * slice; sc = -mf; } }
            else            { if (s < p.Ls_c - 1) hi = (s + 1) * slice; else { hi = 0; sc = -mf; } }
            const float2 h = CG ? __ldcg(in + hi + xc * ncd + i) : __ldg(in + hi + xc * ncd + i);
            acc[k].x += sc * h.x;
            acc[k].y += sc * h.y;
            out[s * slice + xc * ncd + i] = acc[k];
            nrm += (double)acc[k].x * acc[k].x + (double)acc[k].y * acc[k].y;
        }
    }
    return nrm;
}

// Specialisation for 2 nvec = 16 coarse dof and Ls_c <= 4: lane i = l & 15,
// slices sg = l >> 4 and sg + 2.  For each direction all 16 block columns and
// both 16-value input rows are loaded into registers before any arithmetic
// (the inputs as 128-bit broadcast loads), so a warp keeps 32 loads in flight.
template <bool CG>
__device__ __forceinline__ float4 ld4(const float2* p) {
    return CG ? __ldcg(reinterpret_cast<const float4*>(p)) : __ldg(reinterpret_cast<const float4*>(p));
}

template <bool CG>
__device__ __forceinline__ double warp_site16(const float2* __restrict__ B, const float2* __restrict__ in,
                                              float2* __restrict__ out, const CoarseParams& p, long long xc, float mf,
                                              bool dag, int lane) {
    const long long slice = p.Vc * 16;
    const int i = lane & 15, sg = lane >> 4;
    const bool h0 = sg < p.Ls_c, h1 = sg + 2 < p.Ls_c;
    const int s0 = h0 ? sg : 0, s1 = h1 ? sg + 2 : 0;
    float2 acc0 = CG ? __ldcg(in + s0 * slice + xc * 16 + i) : __ldg(in + s0 * slice + xc * 16 + i);
    float2 acc1 = CG ? __ldcg(in + s1 * slice + xc * 16 + i) : __ldg(in + s1 * slice + xc * 16 + i);
    for (int dir = 0; dir < p.ndir; ++dir) {
        const long long nb = coarse_neighbour(p, xc, dir);
        const float2* Bb = B + (xc * p.ndir + dir) * 256 + i;
        const float2* va = in + s0 * slice + nb * 16;
        const float2* vb = in + s1 * slice + nb * 16;
        float2 y[16];
        float4 a[8], b[8];
#pragma unroll
        for (int j = 0; j < 16; ++j) y[j] = __ldg(Bb + j * 16);
#pragma unroll
        for (int m = 0; m < 8; ++m) a[m] = ld4<CG>(va + 2 * m);
#pragma unroll
        for (int m = 0; m < 8; ++m) b[m] = ld4<CG>(vb + 2 * m);
#pragma unroll
        for (int m = 0; m < 8; ++m) {
            acc0 = cfma(y[2 * m], make_float2(a[m].x, a[m].y), acc0);
            acc0 = cfma(y[2 * m + 1], make_float2(a[m].z, a[m].w), acc0);
            acc1 = cfma(y[2 * m], make_float2(b[m].x, b[m].y), acc1);
            acc1 = cfma(y[2 * m + 1], make_float2(b[m].z, b[m].w), acc1);
        }
    }
    const int c = i / p.nvec;
    const bool from_below = dag ? (c == 1) : (c == 0);
    double nrm = 0.0;
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const bool has = k == 0 ? h0 : h1;
        if (!has) continue;
        const int s = k == 0 ? s0 : s1;
        float2 acc = k == 0 ? acc0 : acc1;
        long long hi;
        float sc = 1.f;
        if (from_below) { if (s > 0) hi = (s - 1) * slice; else { hi = (p.Ls_c - 1) * slice; sc = -mf; } }
        else            { if (s < p.Ls_c - 1) hi = (s + 1) * slice; else { hi = 0; sc = -mf; } }
        const float2 hv = CG ? __ldcg(in + hi + xc * 16 + i) : __ldg(in + hi + xc * 16 + i);
        acc.x += sc * hv.x;
        acc.y += sc * hv.y;
        out[s * slice + xc * 16 + i] = acc;
        nrm += (double)acc.x * acc.x + (double)acc.y * acc.y;
    }
    return nrm;
}

// ---------------------------------------------------------------------------
// 2-d tile kernel (16 coarse dof, Ls_c <= 4).  A block of 8 warps applies the
// operator on a 4 x 2 tile of coarse sites, one warp per site:
//   * the five 16 x 16 blocks of every site of the tile (10 KB contiguous per
//     site) are copied into shared memory by one cp.async.bulk per site,
//     completing on an mbarrier (asynchronous: no registers, all in flight);
//   * meanwhile the threads stage the tile's inputs and their one-site halo
//     (6 x 4 sites x Ls_c slices x 16 values) into shared memory;
//   * the warp then multiplies from shared memory only.
// The mbarrier wait is bounded (%globaltimer); on expiry the block records
// an error in *status, waits once more (bounded) for its copies and returns.
// ---------------------------------------------------------------------------
constexpr int TILE_X = 4, TILE_Y = 2, TILE_HX = TILE_X + 2, TILE_HY = TILE_Y + 2;
constexpr int TILE_SITES = TILE_X * TILE_Y;
constexpr int TILE_THREADS = 32 * TILE_SITES;
// BT: storage of the Galerkin blocks, float2 (FP32) or __half2 (FP16)
template <class BT>
struct TileSmemT {
    BT Y[TILE_SITES][5][256];              // column-major blocks per direction
    float2 v[4][TILE_HY][TILE_HX][16];     // staged inputs with halo
    unsigned long long mbar;
};
template <class BT> __host__ __device__ constexpr unsigned site_block_bytes() { return 5u * 256u * (unsigned)sizeof(BT); }

__device__ __forceinline__ float2 to_f2(float2 a) { return a; }
__device__ __forceinline__ float2 to_f2(__half2 a) { return __half22float2(a); }

template <bool CG, class BT>
__device__ __forceinline__ void tile_stage(TileSmemT<BT>& sm, const float2* __restrict__ in, const CoarseParams& p,
                                           int x0, int y0) {
    const int L0 = p.Lc[0], L1 = p.Lc[1];
    const long long slice = p.Vc * 16;
    const int total = p.Ls_c * TILE_HY * TILE_HX * 16;
    for (int e = threadIdx.x; e < total; e += blockDim.x) {
        const int j = e & 15;
        const int h = (e >> 4) % (TILE_HY * TILE_HX);
        const int s = (e >> 4) / (TILE_HY * TILE_HX);
        const int hx = h % TILE_HX, hy = h / TILE_HX;
        int gx = x0 + hx - 1, gy = y0 + hy - 1;
        gx = (gx % L0 + L0) % L0;
        gy = (gy % L1 + L1) % L1;
        const long long site = (long long)gy * L0 + gx;
        sm.v[s][hy][hx][j] = CG ? __ldcg(in + s * slice + site * 16 + j) : __ldg(in + s * slice + site * 16 + j);
    }
}

// Thread 0 starts the bulk copies of the tile's blocks (phase completes when
// all bytes have landed).  Returns the number of bytes expected.
template <class BT>
__device__ __forceinline__ void tile_issue_blocks(TileSmemT<BT>& sm, const BT* __restrict__ B, const CoarseParams& p,
                                                  int x0, int y0) {
    if (threadIdx.x != 0) return;
    constexpr unsigned SITE_BLOCK_BYTES = site_block_bytes<BT>();
    unsigned bytes = 0;
    for (int w = 0; w < TILE_SITES; ++w) {
        const int gx = x0 + w % TILE_X, gy = y0 + w / TILE_X;
        if (gx < p.Lc[0] && gy < p.Lc[1]) bytes += SITE_BLOCK_BYTES;
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    mbar_expect_tx(&sm.mbar, bytes);
    for (int w = 0; w < TILE_SITES; ++w) {
        const int gx = x0 + w % TILE_X, gy = y0 + w / TILE_X;
        if (gx < p.Lc[0] && gy < p.Lc[1]) {
            const long long xc = (long long)gy * p.Lc[0] + gx;
            bulk_g2s(&sm.Y[w][0][0], B + xc * 5 * 256, SITE_BLOCK_BYTES, &sm.mbar);
        }
    }
}

// Multiply for this warp's site from shared memory; returns the lane's |out|^2.
// The adjoint uses gamma_5-hermiticity of the Galerkin kernel: the chirality-
// preserving prolongator gives Dhat_W^dag = sigma_3 Dhat_W sigma_3 (P^dag gamma_5
// D_W gamma_5 P), so the same blocks serve with sign flips on the chirality -
// components of input and output (2 nvec = 16: components 8..15).
// optional epilogue of tile_site: called with (index, value) of every output written
struct NoEpilogue {
    __device__ __forceinline__ void operator()(long long, float2) const {}
};

template <class BT, class Epi = NoEpilogue>
__device__ __forceinline__ double tile_site(const TileSmemT<BT>& sm, float2* __restrict__ out, const CoarseParams& p,
                                            int x0, int y0, float mf, bool dag, Epi epi = Epi()) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int tx = warp % TILE_X, ty = warp / TILE_X;
    const int gx = x0 + tx, gy = y0 + ty;
    if (gx >= p.Lc[0] || gy >= p.Lc[1]) return 0.0;
    const long long xc = (long long)gy * p.Lc[0] + gx;
    const long long slice = p.Vc * 16;
    const int i = lane & 15, sg = lane >> 4;
    const bool h0 = sg < p.Ls_c, h1 = sg + 2 < p.Ls_c;
    const int s0 = h0 ? sg : 0, s1 = h1 ? sg + 2 : 0;
    const int hx = tx + 1, hy = ty + 1;
    float2 acc0 = make_float2(0.f, 0.f), acc1 = make_float2(0.f, 0.f);   // hopping sums for the up / down halves
    float2 acm0 = make_float2(0.f, 0.f), acm1 = make_float2(0.f, 0.f);   // contributions of chirality - inputs
#pragma unroll
    for (int dir = 0; dir < 5; ++dir) {
        const int nx = hx + (dir == 1 ? 1 : dir == 2 ? -1 : 0);
        const int ny = hy + (dir == 3 ? 1 : dir == 4 ? -1 : 0);
        const BT* Yd = &sm.Y[warp][dir][i];
        const float4* va = reinterpret_cast<const float4*>(&sm.v[s0][ny][nx][0]);
        const float4* vb = reinterpret_cast<const float4*>(&sm.v[s1][ny][nx][0]);
#pragma unroll
        for (int m = 0; m < 8; ++m) {
            const float4 a = va[m], b = vb[m];
            const float2 y0v = to_f2(Yd[(2 * m) * 16]), y1v = to_f2(Yd[(2 * m + 1) * 16]);
            if (m < 4) {
                acc0 = cfma(y0v, make_float2(a.x, a.y), acc0);
                acc0 = cfma(y1v, make_float2(a.z, a.w), acc0);
                acc1 = cfma(y0v, make_float2(b.x, b.y), acc1);
                acc1 = cfma(y1v, make_float2(b.z, b.w), acc1);
            } else {
                acm0 = cfma(y0v, make_float2(a.x, a.y), acm0);
                acm0 = cfma(y1v, make_float2(a.z, a.w), acm0);
                acm1 = cfma(y0v, make_float2(b.x, b.y), acm1);
                acm1 = cfma(y1v, make_float2(b.z, b.w), acm1);
            }
        }
    }
    // hop sum: Dhat_W v (operator) or sigma_3 Dhat_W sigma_3 v (adjoint)
    const float si = (dag && i >= 8) ? -1.f : 1.f;
    const float sm_ = dag ? -1.f : 1.f;
    const float2 hop0 = make_float2(si * (acc0.x + sm_ * acm0.x), si * (acc0.y + sm_ * acm0.y));
    const float2 hop1 = make_float2(si * (acc1.x + sm_ * acm1.x), si * (acc1.y + sm_ * acm1.y));
    const int c = i / p.nvec;
    const bool from_below = dag ? (c == 1) : (c == 0);
    double nrm = 0.0;
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const bool has = k == 0 ? h0 : h1;
        if (!has) continue;
        const int s = k == 0 ? s0 : s1;
        const float2 hop = k == 0 ? hop0 : hop1;
        const float2 self = sm.v[s][hy][hx][i];                 // the "+1" of Dhat_W + 1
        int sh;
        float sc = 1.f;
        if (from_below) { if (s > 0) sh = s - 1; else { sh = p.Ls_c - 1; sc = -mf; } }
        else            { if (s < p.Ls_c - 1) sh = s + 1; else { sh = 0; sc = -mf; } }
        const float2 hv = sm.v[sh][hy][hx][i];
        float2 acc;
        acc.x = hop.x + self.x + sc * hv.x;
        acc.y = hop.y + self.y + sc * hv.y;
        out[s * slice + xc * 16 + i] = acc;
        epi(s * slice + xc * 16 + i, acc);
        nrm += (double)acc.x * acc.x + (double)acc.y * acc.y;
    }
    return nrm;
}

constexpr unsigned long long TILE_WAIT_NS = 2000000000ULL;   // 2 s

template <class BT>
__global__ void __launch_bounds__(TILE_THREADS) k_coarse_tile(const BT* __restrict__ B, const float2* __restrict__ in,
                                                              float2* __restrict__ out, CoarseParams p, bool dag,
                                                              const int* skip, int* status) {
    if (skip && *skip) return;
    extern __shared__ __align__(128) unsigned char tile_raw[];
    TileSmemT<BT>& sm = *reinterpret_cast<TileSmemT<BT>*>(tile_raw);
    const int ntx = (p.Lc[0] + TILE_X - 1) / TILE_X;
    const int x0 = (blockIdx.x % ntx) * TILE_X, y0 = (blockIdx.x / ntx) * TILE_Y;
    if (threadIdx.x == 0) mbar_init(&sm.mbar, 1);
    __syncthreads();
    tile_issue_blocks(sm, B, p, x0, y0);
    tile_stage<false, BT>(sm, in, p, x0, y0);
    __syncthreads();
    if (!mbar_wait_bounded(&sm.mbar, 0, TILE_WAIT_NS)) {
        if (threadIdx.x == 0) atomicExch(status, 2);
        mbar_wait_bounded(&sm.mbar, 0, TILE_WAIT_NS);     // let the copies land before the block exits
        return;
    }
    tile_site(sm, out, p, x0, y0, p.mf, dag);
}

static bool tile_ok(const CoarseParams& p) { return p.nd == 2 && p.ncd == 16 && p.Ls_c <= 4; }

static dwf_status site_init_attributes();

dwf_status coarse_init_attributes() {
    DWF_CHECK_CUDA(cudaFuncSetAttribute(k_coarse_tile<float2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)sizeof(TileSmemT<float2>)));
    DWF_CHECK_CUDA(cudaFuncSetAttribute(k_coarse_tile<__half2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)sizeof(TileSmemT<__half2>)));
    return site_init_attributes();
}

template <int NCD>
__global__ void __launch_bounds__(256) k_coarse_dwf(const float2* __restrict__ B, const float2* __restrict__ in,
                                                    float2* __restrict__ out, CoarseParams p, bool dag, const int* skip) {
    if (skip && *skip) return;
    const long long xc = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (xc >= p.Vc) return;
    if (NCD == 16 && p.Ls_c <= 4) warp_site16<false>(B, in, out, p, xc, p.mf, dag, threadIdx.x & 31);
    else warp_site_apply<NCD, false>(B, in, out, p, xc, p.mf, dag, threadIdx.x & 31);
}

// ---------------------------------------------------------------------------
// Per-site kernel for wide coarse blocks (4-d: 9 directions, 2 nvec = 48 dof).
// One block per coarse site: the site's ndir blocks (contiguous, 83 KB in FP16
// at 48 dof) arrive in shared memory by one cp.async.bulk on an mbarrier while
// the threads stage the neighbours' inputs; thread (i, s) then forms output row
// i of slice s from shared memory only.  At one right-hand side the blocks are
// read once per apply, so the kernel is bound by their HBM traffic.  The
// adjoint uses sigma_3 (Dhat_W^dag = sigma_3 Dhat_W sigma_3), so the same blocks
// serve both.
// ---------------------------------------------------------------------------
// neighbour of coarse site xc in direction dir (0 self, 1 + 2 mu forward, 2 + 2 mu
// backward) with 32-bit index arithmetic (coarse lattices have < 2^31 sites)
__device__ __forceinline__ int coarse_nb32(const CoarseParams& p, int xc, int dir) {
    if (dir == 0) return xc;
    const int mu = (dir - 1) >> 1;
    const int L0 = p.Lc[0], L1 = p.Lc[1], L2 = p.Lc[2], L3 = p.Lc[3];
    const int Lm = mu == 0 ? L0 : mu == 1 ? L1 : mu == 2 ? L2 : L3;
    const int stride = mu == 0 ? 1 : mu == 1 ? L0 : mu == 2 ? L0 * L1 : L0 * L1 * L2;
    const int c = (xc / stride) % Lm;
    const int cn = ((dir - 1) & 1) ? (c == 0 ? Lm - 1 : c - 1) : (c == Lm - 1 ? 0 : c + 1);
    return xc + (cn - c) * stride;
}

template <class BT>
__host__ __device__ constexpr size_t site_smem_bytes(int ndir, int ncd, int Ls_c) {
    return ((size_t)ndir * ncd * ncd * sizeof(BT) + 15) / 16 * 16 + (size_t)ndir * Ls_c * ncd * sizeof(float2) + 16;
}

template <class BT>
__global__ void __launch_bounds__(512) k_coarse_site(const BT* __restrict__ B, const float2* __restrict__ in,
                                                     float2* __restrict__ out, CoarseParams p, bool dag,
                                                     const int* skip, int* status) {
    if (skip && *skip) return;
    extern __shared__ __align__(128) unsigned char site_raw[];
    const int ncd = p.ncd, ndir = p.ndir, Ls_c = p.Ls_c;
    const size_t yb_bytes = ((size_t)ndir * ncd * ncd * sizeof(BT) + 15) / 16 * 16;
    BT* yb = reinterpret_cast<BT*>(site_raw);
    float2* vs = reinterpret_cast<float2*>(site_raw + yb_bytes);                 // [dir][s][j]
    unsigned long long* mbar = reinterpret_cast<unsigned long long*>(site_raw + yb_bytes +
                                                                     (size_t)ndir * Ls_c * ncd * sizeof(float2));
    const long long xc = blockIdx.x;
    const long long slice = p.Vc * ncd;
    const unsigned bytes = (unsigned)((size_t)ndir * ncd * ncd * sizeof(BT));
    if (threadIdx.x == 0) {
        mbar_init(mbar, 1);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_expect_tx(mbar, bytes);
        bulk_g2s(yb, B + xc * (long long)ndir * ncd * ncd, bytes, mbar);
    }
    __shared__ int nbs[MG_MAX_DIRS];
    if (threadIdx.x < ndir) nbs[threadIdx.x] = coarse_nb32(p, (int)xc, threadIdx.x);
    __syncthreads();
    const int nv = ndir * Ls_c * ncd;
    for (int e = threadIdx.x; e < nv; e += blockDim.x) {
        const int j = e % ncd, s = (e / ncd) % Ls_c, dir = e / (ncd * Ls_c);
        vs[e] = __ldg(in + s * slice + (long long)nbs[dir] * ncd + j);
    }
    __syncthreads();
    if (!mbar_wait_bounded(mbar, 0, TILE_WAIT_NS)) {
        if (threadIdx.x == 0) atomicExch(status, 2);
        mbar_wait_bounded(mbar, 0, TILE_WAIT_NS);          // let the copy land before the block exits
        return;
    }
    const int i = threadIdx.x % ncd, s = threadIdx.x / ncd;
    if (s >= Ls_c) return;
    const int nvec = p.nvec;
    // inputs j < nvec / j >= nvec, each summed in four independent chains (j mod 4)
    float2 a_lo[4], a_hi[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) { a_lo[u] = make_float2(0.f, 0.f); a_hi[u] = a_lo[u]; }
    for (int dir = 0; dir < ndir; ++dir) {
        const BT* yd = yb + (size_t)dir * ncd * ncd + i;
        const float2* v = vs + (dir * Ls_c + s) * ncd;
        int j = 0;
        for (; j + 4 <= nvec; j += 4) {
#pragma unroll
            for (int u = 0; u < 4; ++u) a_lo[u] = cfma(to_f2(yd[(j + u) * ncd]), v[j + u], a_lo[u]);
        }
        for (; j < nvec; ++j) a_lo[0] = cfma(to_f2(yd[j * ncd]), v[j], a_lo[0]);
        for (; j + 4 <= ncd; j += 4) {
#pragma unroll
            for (int u = 0; u < 4; ++u) a_hi[u] = cfma(to_f2(yd[(j + u) * ncd]), v[j + u], a_hi[u]);
        }
        for (; j < ncd; ++j) a_hi[0] = cfma(to_f2(yd[j * ncd]), v[j], a_hi[0]);
    }
    const float2 lo = make_float2((a_lo[0].x + a_lo[1].x) + (a_lo[2].x + a_lo[3].x),
                                  (a_lo[0].y + a_lo[1].y) + (a_lo[2].y + a_lo[3].y));
    const float2 hi = make_float2((a_hi[0].x + a_hi[1].x) + (a_hi[2].x + a_hi[3].x),
                                  (a_hi[0].y + a_hi[1].y) + (a_hi[2].y + a_hi[3].y));
    const float sj = dag ? -1.f : 1.f;                   // sigma_3 on the inputs
    const float si = (dag && i >= nvec) ? -1.f : 1.f;    // sigma_3 on the output
    float2 acc = make_float2(si * (lo.x + sj * hi.x), si * (lo.y + sj * hi.y));
    const float2* v0 = vs;                               // dir 0 = the site itself
    const float2 self = v0[s * ncd + i];
    const int c = i / nvec;
    const bool from_below = dag ? (c == 1) : (c == 0);
    int sh;
    float sc = 1.f;
    if (from_below) { if (s > 0) sh = s - 1; else { sh = Ls_c - 1; sc = -p.mf; } }
    else            { if (s < Ls_c - 1) sh = s + 1; else { sh = 0; sc = -p.mf; } }
    const float2 hv = v0[sh * ncd + i];
    acc.x += self.x + sc * hv.x;
    acc.y += self.y + sc * hv.y;
    out[s * slice + xc * ncd + i] = acc;
}

// ---------------------------------------------------------------------------
// Tensor-core form of the 48-dof stencil (4-d, FP16 blocks, Ls_c <= 4).  One
// warp per coarse site.  Per direction the complex product Y v over the Ls_c
// slices is the real product of A = [Re Y; Im Y] (96 x 48, FP16, exact in
// TF32) with B = [Re v | Im v] (48 x 2 Ls_c): C = A B holds Re Y Re v, Re Y Im v
// (rows < 48) and Im Y Re v, Im Y Im v (rows >= 48), so
// Re(Y v) = C[i][Re] - C[48 + i][Im] and Im(Y v) = C[48 + i][Re] + C[i][Im].
// B column n = 4 part + s; the FP32 inputs are split into TF32 high and low
// parts multiplied separately (FP32-level accuracy).  A streams from HBM in
// fragment order (one coalesced 16-byte load per lane per row tile and column
// tile pair, no shared-memory staging), so many warps per SM keep enough bytes
// in flight; the products accumulate over the 9 directions in registers.
// ---------------------------------------------------------------------------
constexpr int CM_WARPS = 4;
__device__ __forceinline__ uint32_t f16_bits_to_f32(uint32_t w, int hi) {
    return __float_as_uint(__half2float(__ushort_as_half((unsigned short)(hi ? (w >> 16) : (w & 0xffffu)))));
}

__global__ void __launch_bounds__(CM_WARPS * 32, 3) k_coarse_mma(const uint4* __restrict__ Ym,
                                                                 const float2* __restrict__ in,
                                                                 float2* __restrict__ out, CoarseParams p, bool dag,
                                                                 const int* skip) {
    if (skip && *skip) return;
    __shared__ float Ps[CM_WARPS][96][9];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    const int xc = blockIdx.x * CM_WARPS + warp;
    if (xc >= p.Vc) return;                              // whole warps; no block-wide barrier below
    const int Ls_c = p.Ls_c;
    const long long slice = p.Vc * 48;
    const int part = g >> 2, sB = g & 3;                 // B column n = g
    const bool colv = sB < Ls_c;
    float acc[6][2][4];
#pragma unroll
    for (int mt = 0; mt < 6; ++mt)
#pragma unroll
        for (int h = 0; h < 2; ++h)
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[mt][h][q] = 0.f;
    const uint4* A = Ym + (long long)xc * (9 * 3 * 6 * 32) + lane;
#pragma unroll 1
    for (int dir = 0; dir < 9; ++dir) {
        // L2 prefetch of the next direction's 18 fragment rows (one lane per 128-byte line)
        if (dir + 1 < 9 && (lane & 7) == 0) {
#pragma unroll
            for (int q = 0; q < 18; ++q) asm volatile("prefetch.global.L2 [%0];" ::"l"(A + ((dir + 1) * 18 + q) * 32));
        }
        const int nb = coarse_nb32(p, xc, dir);
        const float* vin = reinterpret_cast<const float*>(in + (colv ? sB : 0) * slice + (long long)nb * 48) + part;
#pragma unroll
        for (int kp = 0; kp < 3; ++kp) {
            uint4 a[6];
#pragma unroll
            for (int mt = 0; mt < 6; ++mt) a[mt] = __ldg(A + ((dir * 3 + kp) * 6 + mt) * 32);
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int kt = 2 * kp + h;                 // input dof 8 kt .. 8 kt + 7
                float b0 = colv ? __ldg(vin + 2 * (8 * kt + t)) : 0.f;
                float b1 = colv ? __ldg(vin + 2 * (8 * kt + t + 4)) : 0.f;
                if (dag && kt >= 3) { b0 = -b0; b1 = -b1; }   // sigma_3 on the chirality - inputs
                uint32_t bh[2], bl[2];
                split_tf32(b0, bh[0], bl[0]);
                split_tf32(b1, bh[1], bl[1]);
#pragma unroll
                for (int mt = 0; mt < 6; ++mt) {
                    const uint32_t w0 = h ? a[mt].z : a[mt].x, w1 = h ? a[mt].w : a[mt].y;
                    const uint32_t af[4] = {f16_bits_to_f32(w0, 0), f16_bits_to_f32(w0, 1), f16_bits_to_f32(w1, 0),
                                            f16_bits_to_f32(w1, 1)};
                    mma_tf32(acc[mt][0], af, bh);
                    mma_tf32(acc[mt][1], af, bl);
                }
            }
        }
    }
    // C fragment: c0 (g, 2t), c1 (g, 2t + 1), c2 (g + 8, 2t), c3 (g + 8, 2t + 1)
#pragma unroll
    for (int mt = 0; mt < 6; ++mt)
#pragma unroll
        for (int q = 0; q < 4; ++q)
            Ps[warp][mt * 16 + g + ((q & 2) ? 8 : 0)][2 * t + (q & 1)] = acc[mt][0][q] + acc[mt][1][q];
    __syncwarp();
    const int nvec = p.nvec;
    for (int idx = lane; idx < 48 * Ls_c; idx += 32) {
        const int s = idx / 48, r = idx % 48;
        const float re = Ps[warp][r][s] - Ps[warp][48 + r][4 + s];
        const float im = Ps[warp][48 + r][s] + Ps[warp][r][4 + s];
        const float si = (dag && r >= nvec) ? -1.f : 1.f;  // sigma_3 on the output
        const float2 self = __ldg(in + s * slice + (long long)xc * 48 + r);
        const int c = r / nvec;
        const bool from_below = dag ? (c == 1) : (c == 0);
        int sh;
        float sc = 1.f;
        if (from_below) { if (s > 0) sh = s - 1; else { sh = Ls_c - 1; sc = -p.mf; } }
        else            { if (s < Ls_c - 1) sh = s + 1; else { sh = 0; sc = -p.mf; } }
        const float2 hv = __ldg(in + sh * slice + (long long)xc * 48 + r);
        out[s * slice + (long long)xc * 48 + r] = make_float2(si * re + self.x + sc * hv.x, si * im + self.y + sc * hv.y);
    }
}

constexpr size_t SITE_SMEM_MAX = 200 * 1024;
static dwf_status site_init_attributes() {
    DWF_CHECK_CUDA(cudaFuncSetAttribute(k_coarse_site<float2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)SITE_SMEM_MAX));
    DWF_CHECK_CUDA(cudaFuncSetAttribute(k_coarse_site<__half2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)SITE_SMEM_MAX));
    return DWF_OK;
}

// the per-site kernel: 4-d blocks (or wide 2-d ones) whose shared-memory copy fits in a block
static bool site_ok(const CoarseParams& p, int half) {
    if (p.ncd < 24 || p.ncd * p.Ls_c > 512) return false;
    const size_t b = half ? site_smem_bytes<__half2>(p.ndir, p.ncd, p.Ls_c) : site_smem_bytes<float2>(p.ndir, p.ncd, p.Ls_c);
    return b <= SITE_SMEM_MAX;
}

static CoarseParams coarse_params(const dwf_mg* h, double mf) {
    CoarseParams p;
    p.Vc = h->mg.Vc;
    p.nd = h->mg.nd;
    for (int mu = 0; mu < 4; ++mu) p.Lc[mu] = h->mg.Lc[mu];
    p.Ls_c = h->mg.Ls_c;
    p.ncd = h->mg.ncd;
    p.nvec = h->mg.nvec;
    p.ndir = h->mg.ndir;
    p.mf = (float)mf;
    return p;
}

dwf_status coarse_dwf_apply(const dwf_mg* h, const float2* in, float2* out, double mf, bool dagger, const int* skip,
                            cudaStream_t st) {
    CoarseParams p = coarse_params(h, mf);
    const int thr = 256;
    const unsigned grid = (unsigned)((p.Vc * 32 + thr - 1) / thr);
    const float2* B = dagger ? h->Yd32 : h->Y32;
    if (tile_ok(p)) {
        const int ntiles = ((p.Lc[0] + TILE_X - 1) / TILE_X) * ((p.Lc[1] + TILE_Y - 1) / TILE_Y);
        if (h->ytile_half)
            k_coarse_tile<__half2><<<ntiles, TILE_THREADS, sizeof(TileSmemT<__half2>), st>>>(
                (const __half2*)h->Ytile, in, out, p, dagger, skip, h->status + 1);
        else
            k_coarse_tile<float2><<<ntiles, TILE_THREADS, sizeof(TileSmemT<float2>), st>>>(
                (const float2*)h->Ytile, in, out, p, dagger, skip, h->status + 1);
    } else if (h->Ymma && p.ncd == 48 && p.ndir == 9 && p.Ls_c <= 4) {
        const unsigned grid1 = (unsigned)((p.Vc + CM_WARPS - 1) / CM_WARPS);
        k_coarse_mma<<<grid1, CM_WARPS * 32, 0, st>>>((const uint4*)h->Ymma, in, out, p, dagger, skip);
    } else if (site_ok(p, h->ytile_half)) {
        const int threads = p.ncd * p.Ls_c;
        if (h->ytile_half)
            k_coarse_site<__half2><<<(unsigned)p.Vc, threads, site_smem_bytes<__half2>(p.ndir, p.ncd, p.Ls_c), st>>>(
                (const __half2*)h->Ytile, in, out, p, dagger, skip, h->status + 1);
        else
            k_coarse_site<float2><<<(unsigned)p.Vc, threads, site_smem_bytes<float2>(p.ndir, p.ncd, p.Ls_c), st>>>(
                (const float2*)h->Ytile, in, out, p, dagger, skip, h->status + 1);
    } else if (p.ncd == 16) k_coarse_dwf<16><<<grid, thr, 0, st>>>(B, in, out, p, dagger, skip);
    else             k_coarse_dwf<0><<<grid, thr, 0, st>>>(B, in, out, p, dagger, skip);
    DWF_CHECK_LAUNCH();
    return DWF_OK;
}

dwf_status coarse_site_apply(const CoarseParams& p, const __half2* B, const float2* in, float2* out, bool dagger,
                             const int* skip, int* status, cudaStream_t st) {
    if (!site_ok(p, 1)) { set_error("the per-site coarse stencil does not take %d dof on %d slices", p.ncd, p.Ls_c);
                          return DWF_ERR_UNSUPPORTED; }
    k_coarse_site<__half2><<<(unsigned)p.Vc, p.ncd * p.Ls_c, site_smem_bytes<__half2>(p.ndir, p.ncd, p.Ls_c), st>>>(
        B, in, out, p, dagger, skip, status);
    DWF_CHECK_LAUNCH();
    return DWF_OK;
}

dwf_status coarse_site_apply(const CoarseParams& p, const float2* B, const float2* in, float2* out, bool dagger,
                             const int* skip, int* status, cudaStream_t st) {
    if (!site_ok(p, 0)) { set_error("the per-site coarse stencil does not take %d dof on %d slices", p.ncd, p.Ls_c);
                          return DWF_ERR_UNSUPPORTED; }
    k_coarse_site<float2><<<(unsigned)p.Vc, p.ncd * p.Ls_c, site_smem_bytes<float2>(p.ndir, p.ncd, p.Ls_c), st>>>(
        B, in, out, p, dagger, skip, status);
    DWF_CHECK_LAUNCH();
    return DWF_OK;
}

// Yd[x][dir] (column-major) = Y[x + dir][-dir]^dag from the row-major FP64 blocks.
__global__ void k_adjoint_blocks(const double2* __restrict__ Y, float2* __restrict__ Yd, CoarseParams p) {
    const int ncd = p.ncd;
    const long long bsz = (long long)ncd * ncd;
    const long long n = p.Vc * p.ndir * bsz;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
        const long long blk = t / bsz;
        const int e = (int)(t % bsz);           // column-major index j * ncd + i
        const long long xc = blk / p.ndir;
        const int dir = (int)(blk % p.ndir);
        const int opp = dir == 0 ? 0 : (((dir - 1) % 2 == 0) ? dir + 1 : dir - 1);
        const long long nb = coarse_neighbour(p, xc, dir);
        // element (i, j) of the adjoint block = conj(Y_nb,opp(j, i)); row-major (j, i) sits at j * ncd + i
        const double2 v = Y[(nb * p.ndir + opp) * bsz + e];
        Yd[t] = make_float2((float)v.x, (float)-v.y);
    }
}

dwf_status build_adjoint_blocks(dwf_mg* h, cudaStream_t st) {
    CoarseParams p = coarse_params(h, h->mf);
    const long long n = p.Vc * p.ndir * (long long)p.ncd * p.ncd;
    const int grid = (int)((n + 255) / 256 < 152 * 16 ? (n + 255) / 256 : 152 * 16);
    k_adjoint_blocks<<<grid, 256, 0, st>>>(h->Y64, h->Yd32, p);
    DWF_CHECK_LAUNCH();
    return DWF_OK;
}

// ---------------------------------------------------------------------------
// truncated restriction / prolongation
// ---------------------------------------------------------------------------
struct TransferParams {
    int nd, L[4], b[4], Lc[4];
    long long V, Vc;
    int Ls, Ls_c, nvec, ncd, nchd, dof, ncol, nb;
    int bulk;            // 1: P^dag / P on every slice (Lhat_s = Ls) instead of the walls
    int packed;          // 1: fine vectors in the slice-paired 4-d layout
    long long NB;        // blocks of 32 sites of the packed layout
};

// complex index of fine element (s, site, d) in the canonical or the slice-paired layout
// (float4 ((s/2 NB + site/32) dof + d) 32 + site%32 holds slices 2j and 2j+1 as two complex values)
__device__ __forceinline__ long long fine_idx(const TransferParams& p, int s, long long x, int d) {
    if (!p.packed) return ((long long)s * p.V + x) * p.dof + d;
    return 2 * (((((long long)(s >> 1)) * p.NB + (x >> 5)) * p.dof + d) * 32 + (x & 31)) + (s & 1);
}

__device__ __forceinline__ long long agg_of(const TransferParams& p, long long site) {
    long long xc = 0, stride = 1;
    long long rem = site;
    for (int mu = 0; mu < p.nd; ++mu) {
        const int c = (int)(rem % p.L[mu]);
        rem /= p.L[mu];
        xc += (long long)(c / p.b[mu]) * stride;
        stride *= p.Lc[mu];
    }
    return xc;
}

__device__ __forceinline__ long long agg_site(const TransferParams& p, long long xc, int l) {
    long long site = 0, stride = 1;
    long long rem = xc;
    int lr = l;
    for (int mu = 0; mu < p.nd; ++mu) {
        const int c = (int)(rem % p.Lc[mu]);
        rem /= p.Lc[mu];
        const int lc = lr % p.b[mu];
        lr /= p.b[mu];
        site += (long long)(c * p.b[mu] + lc) * stride;
        stride *= p.L[mu];
    }
    return site;
}

__device__ __forceinline__ int chir_dof(const TransferParams& p, int c, int cd) {
    if (p.nd == 2) return c;
    return (2 * c + cd / p.ncol) * p.ncol + cd % p.ncol;
}

// grid.y = right-hand side (vectors back to back); skip[r]: per right-hand side
__global__ void k_restrict(const float2* __restrict__ P, const float2* __restrict__ r, float2* __restrict__ out,
                           TransferParams p, const int* skip) {
    if (skip && skip[blockIdx.y]) return;
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long total = p.Vc * p.Ls_c * p.ncd;
    if (t >= total) return;
    r += (long long)blockIdx.y * p.V * p.Ls * p.dof;
    out += (long long)blockIdx.y * total;
    const int i = (int)(t % p.ncd);
    const long long rest = t / p.ncd;
    const long long xc = rest % p.Vc;
    const int s = (int)(rest / p.Vc);
    const int c = i / p.nvec, k = i % p.nvec;
    float2 acc = make_float2(0.f, 0.f);
    int sf = -1;
    if (c == 1 && s == 0) sf = 0;                 // Phat_- P^dag P_- r_1 on coarse slice 1
    if (c == 0 && s == p.Ls_c - 1) sf = p.Ls - 1; // Phat_+ P^dag P_+ r_Ls on coarse slice Lhat_s
    if (p.bulk) sf = s;                           // bulk: every slice
    if (sf >= 0) {
        for (int l = 0; l < p.nb; ++l) {
            const long long x = agg_site(p, xc, l);
            for (int cd = 0; cd < p.nchd; ++cd)
                acc = cfma_conj(P[((x * 2 + c) * p.nchd + cd) * p.nvec + k], r[fine_idx(p, sf, x, chir_dof(p, c, cd))],
                                acc);
        }
    }
    out[t] = acc;
}

__global__ void k_prolong(const float2* __restrict__ P, const float2* __restrict__ e, float2* __restrict__ out,
                          TransferParams p, const int* skip) {
    if (skip && skip[blockIdx.y]) return;
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long total = p.V * p.Ls * p.dof;
    if (t >= total) return;
    e += (long long)blockIdx.y * p.Vc * p.Ls_c * p.ncd;
    out += (long long)blockIdx.y * total;
    // thread t writes element t of the output layout: (s, site, d) from the canonical or packed order
    int d, s;
    long long x;
    if (!p.packed) {
        d = (int)(t % p.dof);
        const long long rest = t / p.dof;
        x = rest % p.V;
        s = (int)(rest / p.V);
    } else {
        const int s1 = (int)(t & 1);
        const long long q = t >> 1;
        const int i = (int)(q & 31);
        const long long q2 = q >> 5;
        d = (int)(q2 % p.dof);
        const long long q3 = q2 / p.dof;
        x = (q3 % p.NB) * 32 + i;
        s = (int)(q3 / p.NB) * 2 + s1;
    }
    int c, cd;
    if (p.nd == 2) { c = d; cd = 0; }
    else { const int spin = d / p.ncol; c = spin / 2; cd = (spin % 2) * p.ncol + d % p.ncol; }
    float2 acc = make_float2(0.f, 0.f);
    int sc = -1;
    if (c == 1 && s == 0) sc = 0;                 // P_- P e_1 on fine slice 1
    if (c == 0 && s == p.Ls - 1) sc = p.Ls_c - 1; // P_+ P e_{Lhat_s} on fine slice Ls
    if (p.bulk) sc = s;                           // bulk: every slice
    if (sc >= 0) {
        const long long xc = agg_of(p, x);
        const float2* ev = e + ((long long)sc * p.Vc + xc) * p.ncd + c * p.nvec;
        const float2* Pr = P + ((x * 2 + c) * p.nchd + cd) * p.nvec;
        for (int k = 0; k < p.nvec; ++k) acc = cfma(Pr[k], ev[k], acc);
    }
    out[t] = acc;
}

static TransferParams transfer_params(const dwf_mg* h) {
    TransferParams p;
    p.nd = h->mg.nd;
    for (int mu = 0; mu < 4; ++mu) { p.L[mu] = h->mg.L[mu]; p.b[mu] = h->mg.b[mu]; p.Lc[mu] = h->mg.Lc[mu]; }
    p.V = h->mg.V;
    p.Vc = h->mg.Vc;
    p.Ls = h->mg.Ls;
    p.Ls_c = h->mg.Ls_c;
    p.nvec = h->mg.nvec;
    p.ncd = h->mg.ncd;
    p.nchd = h->mg.nchd;
    p.dof = (int)site_dof(h->G);
    p.ncol = h->G.ncol;
    p.nb = h->mg.nb;
    p.bulk = h->prm.transfer == 1 ? 1 : 0;
    p.packed = 0;
    p.NB = (p.V + 31) / 32;
    return p;
}

static dwf_status check_packed_transfer(const TransferParams& p) {
    if (p.nd != 4 || p.Ls % 2 || p.V % 32) {
        set_error("packed transfers need a 4-d lattice, even Ls and a multiple of 32 sites");
        return DWF_ERR_UNSUPPORTED;
    }
    return DWF_OK;
}

dwf_status restrict_wall(const dwf_mg* h, const float2* r_fine, float2* r_coarse, const int* skip, cudaStream_t st,
                         int nrhs, bool packed) {
    TransferParams p = transfer_params(h);
    if (packed) { DWF_TRY(check_packed_transfer(p)); p.packed = 1; }
    const long long total = p.Vc * p.Ls_c * p.ncd;
    if (nrhs < 1 || nrhs > 65535) { set_error("nrhs must be in [1, 65535]"); return DWF_ERR_ARG; }
    k_restrict<<<dim3((unsigned)((total + 255) / 256), (unsigned)nrhs), 256, 0, st>>>(h->P32, r_fine, r_coarse, p,
                                                                                       skip);
    DWF_CHECK_LAUNCH();
    return DWF_OK;
}

dwf_status prolong_wall(const dwf_mg* h, const float2* e_coarse, float2* e_fine, const int* skip, cudaStream_t st,
                        int nrhs, bool packed) {
    TransferParams p = transfer_params(h);
    if (packed) { DWF_TRY(check_packed_transfer(p)); p.packed = 1; }
    const long long total = p.V * p.Ls * p.dof;
    if (nrhs < 1 || nrhs > 65535) { set_error("nrhs must be in [1, 65535]"); return DWF_ERR_ARG; }
    k_prolong<<<dim3((unsigned)((total + 255) / 256), (unsigned)nrhs), 256, 0, st>>>(h->P32, e_coarse, e_fine, p,
                                                                                      skip);
    DWF_CHECK_LAUNCH();
    return DWF_OK;
}

}  // namespace dwf

using namespace dwf;

extern "C" {

dwf_status mg_restrict(const dwf_mg* h, const void* r_fine, void* r_coarse, void* stream) {
    clear_error();
    if (!h || !r_fine || !r_coarse) { set_error("NULL argument"); return DWF_ERR_ARG; }
    return restrict_wall(h, (const float2*)r_fine, (float2*)r_coarse, nullptr, as_stream(stream));
}

dwf_status mg_prolong(const dwf_mg* h, const void* e_coarse, void* e_fine, void* stream) {
    clear_error();
    if (!h || !e_coarse || !e_fine) { set_error("NULL argument"); return DWF_ERR_ARG; }
    return prolong_wall(h, (const float2*)e_coarse, (float2*)e_fine, nullptr, as_stream(stream));
}

dwf_status mg_coarse_apply(const dwf_mg* h, const void* in, void* out, double mf, int dagger, void* stream) {
    clear_error();
    if (!h || !in || !out) { set_error("NULL argument"); return DWF_ERR_ARG; }
    if (in == out) { set_error("in and out must be distinct buffers"); return DWF_ERR_ARG; }
    return coarse_dwf_apply(h, (const float2*)in, (float2*)out, mf, dagger != 0, nullptr, as_stream(stream));
}

}  // extern "C"

// ===========================================================================
// Persistent coarse CGNR: one cooperative launch per coarse solve.
//
// Solves (Dhat_PV^dag Dhat_DW)^dag (Dhat_PV^dag Dhat_DW) e = (..)^dag r_c by CG
// (the coarsest-level CGNR of Table kcycle), with every block resident for
// the whole solve and phases separated by a software grid barrier.  The
// barrier's spin is bounded by a %globaltimer deadline: on expiry the block
// raises an error flag that every other block sees at its next barrier, and
// all blocks return (the host reports DWF_ERR_TIMEOUT).  Reductions: each
// block writes one FP64 partial per quantity; after the barrier every block
// sums all partials in the same order, so all blocks hold identical scalars.
// Mutable vectors are read through L2 (ld.global.cg) because other blocks wrote
// them earlier in the same launch.
// ===========================================================================
namespace dwf {

constexpr int PCG_THREADS = 256;

struct PcgBarrier {
    unsigned count;
    unsigned gen;
    int error;
    int pad;
};

struct PcgArgs {
    CoarseParams cp;
    const float2* Y;    // Galerkin blocks (column-major)
    const float2* Yd;   // adjoint blocks (column-major)
    const float2* rc;   // right-hand side
    float2* e;          // solution
    float2 *rr, *r, *p, *q, *t, *w;
    double* partials;   // [3][gridDim.x]
    PcgBarrier* bar;
    int* out_iters;
    double* out_rr2;    // final |rr|^2 / |rc|^2
    double tol2;
    int maxiter;
    double mf;
    unsigned long long timeout_ns;
};

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Returns false if the barrier timed out here or anywhere else, or if this
// block reports a failure of its own (local_ok == false).
__device__ bool pcg_sync(PcgBarrier* b, unsigned long long deadline, bool local_ok = true) {
    __shared__ int ok;
    __shared__ int any_fail;
    if (threadIdx.x == 0) any_fail = 0;
    __syncthreads();
    if (!local_ok) any_fail = 1;
    __syncthreads();
    if (threadIdx.x == 0) {
        if (any_fail) atomicExch(&b->error, 1);
        volatile unsigned* vgen = &b->gen;
        volatile int* verr = &b->error;
        const unsigned g = *vgen;
        __threadfence();
        const unsigned arrived = atomicAdd(&b->count, 1u);
        if (arrived == gridDim.x - 1) {
            b->count = 0u;
            __threadfence();
            atomicAdd(&b->gen, 1u);
        } else {
            while (*vgen == g) {
                if (*verr) break;
                if (global_ns() > deadline) { atomicExch(&b->error, 1); break; }
                __nanosleep(64);
            }
        }
        __threadfence();
        ok = (*verr == 0);
    }
    __syncthreads();
    return ok != 0;
}

// block-sum of up to 3 doubles into partials[k * grid + block]
__device__ void pcg_partial(double (&v)[3], int nv, double* partials) {
    __shared__ double sh[3][PCG_THREADS / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int k = 0; k < nv; ++k)
        for (int off = 16; off > 0; off >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], off);
    if (lane == 0)
        for (int k = 0; k < nv; ++k) sh[k][warp] = v[k];
    __syncthreads();
    if (threadIdx.x == 0)
        for (int k = 0; k < nv; ++k) {
            double s = 0.0;
            for (int w = 0; w < PCG_THREADS / 32; ++w) s += sh[k][w];
            partials[k * gridDim.x + blockIdx.x] = s;
        }
    __syncthreads();
}

// every block: fixed-order total of partial k (strided loads by all threads,
// then a fixed-order block reduction)
__device__ double pcg_total(const double* partials, int k) {
    __shared__ double sh[PCG_THREADS / 32];
    __shared__ double tot;
    double v = 0.0;
    for (unsigned b = threadIdx.x; b < gridDim.x; b += blockDim.x) v += __ldcg(partials + k * gridDim.x + b);
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < PCG_THREADS / 32; ++w) s += sh[w];
        tot = s;
    }
    __syncthreads();
    const double r = tot;
    __syncthreads();
    return r;
}

// out = Dhat_DW(m) in (or adjoint) over all tiles (grid-stride), shared-memory
// tiles as in k_coarse_tile.  `phase` is this block's mbarrier parity, flipped
// per tile.  Returns this thread's share of |out|^2; false in *ok on a timeout.
__device__ double pcg_apply(const PcgArgs& a, TileSmemT<float2>& sm, unsigned& phase, const float2* __restrict__ in,
                            float2* __restrict__ out, double mf, bool dag, bool* ok) {
    const CoarseParams& p = a.cp;
    const float2* B = a.Y;
    const int ntx = (p.Lc[0] + TILE_X - 1) / TILE_X;
    const int ntiles = ntx * ((p.Lc[1] + TILE_Y - 1) / TILE_Y);
    double nrm = 0.0;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int x0 = (tile % ntx) * TILE_X, y0 = (tile / ntx) * TILE_Y;
        __syncthreads();                        // previous tile's shared data fully consumed
        tile_issue_blocks(sm, B, p, x0, y0);
        tile_stage<true, float2>(sm, in, p, x0, y0);
        __syncthreads();
        const bool okw = mbar_wait_bounded(&sm.mbar, phase, TILE_WAIT_NS);
        if (__syncthreads_or(!okw)) {                      // the whole block leaves together
            mbar_wait_bounded(&sm.mbar, phase, TILE_WAIT_NS);
            *ok = false;
            return nrm;
        }
        phase ^= 1u;
        nrm += tile_site(sm, out, p, x0, y0, (float)mf, dag);
    }
    return nrm;
}

#define PCG_LOOP(k, n) for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < (n); k += (long long)gridDim.x * blockDim.x)

__global__ void __launch_bounds__(PCG_THREADS) k_coarse_cgnr_persistent(PcgArgs a) {
    extern __shared__ __align__(128) unsigned char pcg_raw[];
    TileSmemT<float2>& sm = *reinterpret_cast<TileSmemT<float2>*>(pcg_raw);
    const long long n = a.cp.Vc * a.cp.Ls_c * a.cp.ncd;
    const unsigned long long deadline = global_ns() + a.timeout_ns;
    const double mf = a.mf;
    unsigned phase = 0;
    bool ok = true;
    if (threadIdx.x == 0) mbar_init(&sm.mbar, 1);
    __syncthreads();
    // prologue: e = 0, rr = rc, t = Dhat_PV rr, r = Dhat_DW^dag t (= B^dag rr), p = r
    PCG_LOOP(k, n) { a.e[k] = make_float2(0.f, 0.f); a.rr[k] = __ldcg(a.rc + k); }
    if (!pcg_sync(a.bar, deadline, ok)) return;
    pcg_apply(a, sm, phase, a.rr, a.t, 1.0, false, &ok);
    if (!pcg_sync(a.bar, deadline, ok)) return;
    double v[3] = {pcg_apply(a, sm, phase, a.t, a.r, mf, true, &ok), 0.0, 0.0};
    PCG_LOOP(k, n) {
        float2 y = __ldcg(a.rc + k);
        v[1] += (double)y.x * y.x + (double)y.y * y.y;
    }
    pcg_partial(v, 2, a.partials);
    if (!pcg_sync(a.bar, deadline, ok)) return;
    PCG_LOOP(k, n) a.p[k] = __ldcg(a.r + k);
    double rn2 = pcg_total(a.partials, 0);
    const double bn2 = pcg_total(a.partials, 1);
    double rr2 = bn2;
    int it = 0;
    if (bn2 > 0.0 && rn2 > 0.0) {
        while (it < a.maxiter) {
            // q = Dhat_PV^dag Dhat_DW p  (p = r on the first pass: r is complete,
            // the copy into p is not visible to other blocks yet)
            pcg_apply(a, sm, phase, it == 0 ? a.r : a.p, a.t, mf, false, &ok);
            if (!pcg_sync(a.bar, deadline, ok)) return;
            double u[3] = {pcg_apply(a, sm, phase, a.t, a.q, 1.0, true, &ok), 0.0, 0.0};
            pcg_partial(u, 1, a.partials);
            if (!pcg_sync(a.bar, deadline, ok)) return;
            const double qq = pcg_total(a.partials, 0);
            if (!(qq > 0.0)) break;
            const double alpha = rn2 / qq;
            const float af = (float)alpha;
            // e += alpha p; rr -= alpha q; t = Dhat_PV q (q is complete)
            double u2[3] = {0.0, 0.0, 0.0};
            PCG_LOOP(k, n) {
                float2 pk = __ldcg(a.p + k), qk = __ldcg(a.q + k), ek = __ldcg(a.e + k), rk = __ldcg(a.rr + k);
                ek.x += af * pk.x; ek.y += af * pk.y;
                rk.x -= af * qk.x; rk.y -= af * qk.y;
                a.e[k] = ek; a.rr[k] = rk;
                u2[0] += (double)rk.x * rk.x + (double)rk.y * rk.y;
            }
            pcg_partial(u2, 1, a.partials + 2 * gridDim.x);
            pcg_apply(a, sm, phase, a.q, a.t, 1.0, false, &ok);
            if (!pcg_sync(a.bar, deadline, ok)) return;
            rr2 = pcg_total(a.partials, 2);
            ++it;
            if (rr2 <= a.tol2 * bn2) break;
            // w = Dhat_DW^dag t; r -= alpha w
            pcg_apply(a, sm, phase, a.t, a.w, mf, true, &ok);
            if (!pcg_sync(a.bar, deadline, ok)) return;
            double u3[3] = {0.0, 0.0, 0.0};
            PCG_LOOP(k, n) {
                float2 rk = __ldcg(a.r + k), wk = __ldcg(a.w + k);
                rk.x -= af * wk.x; rk.y -= af * wk.y;
                a.r[k] = rk;
                u3[0] += (double)rk.x * rk.x + (double)rk.y * rk.y;
            }
            pcg_partial(u3, 1, a.partials + gridDim.x);
            if (!pcg_sync(a.bar, deadline, ok)) return;
            const double rn2n = pcg_total(a.partials, 1);
            const float beta = (float)(rn2n / rn2);
            rn2 = rn2n;
            PCG_LOOP(k, n) {
                float2 pk = __ldcg(a.p + k), rk = __ldcg(a.r + k);
                a.p[k] = make_float2(rk.x + beta * pk.x, rk.y + beta * pk.y);
            }
            if (!pcg_sync(a.bar, deadline, ok)) return;
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        *a.out_iters += it;                       // running total over solves
        *a.out_rr2 = bn2 > 0 ? rr2 / bn2 : 0.0;
    }
}

struct PcgPlan {
    int grid = 0;
};

static PcgPlan g_pcg_plan[64];

dwf_status coarse_cgnr_persistent(const dwf_mg* h, const float2* rc, float2* ec, float2* const* vec6, double* partials,
                                  void* bar, int* out_iters, double* out_rr2, cudaStream_t st) {
    int dev = 0;
    DWF_CHECK_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) { set_error("device ordinal out of range"); return DWF_ERR_UNSUPPORTED; }
    if (h->mg.Ls_c > 4 || h->mg.ncd != 16 || h->mg.nd != 2) {
        set_error("persistent coarse solver supports 2-d, 16 coarse dof and Ls_c <= 4");
        return DWF_ERR_UNSUPPORTED;
    }
    PcgPlan& plan = g_pcg_plan[dev];
    if (plan.grid == 0) {
        int nsm = 0, per = 0;
        DWF_CHECK_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
        DWF_CHECK_CUDA(cudaFuncSetAttribute(k_coarse_cgnr_persistent, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            (int)sizeof(TileSmemT<float2>)));
        DWF_CHECK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_coarse_cgnr_persistent, PCG_THREADS,
                                                                     sizeof(TileSmemT<float2>)));
        if (per < 1) { set_error("persistent coarse solver cannot be resident"); return DWF_ERR_UNSUPPORTED; }
        plan.grid = nsm * per;
    }
    PcgArgs a;
    a.cp = coarse_params(h, h->mf);
    a.Y = h->Y32;
    a.Yd = h->Yd32;
    a.rc = rc;
    a.e = ec;
    a.rr = vec6[0]; a.r = vec6[1]; a.p = vec6[2]; a.q = vec6[3]; a.t = vec6[4]; a.w = vec6[5];
    a.partials = partials;
    a.bar = (PcgBarrier*)bar;
    a.out_iters = out_iters;
    a.out_rr2 = out_rr2;
    a.tol2 = h->prm.coarse_tol * h->prm.coarse_tol;
    a.maxiter = h->prm.coarse_maxiter;
    a.mf = h->mf;
    a.timeout_ns = 5000000000ULL;   // 5 s per solve
    const int ntiles = ((a.cp.Lc[0] + TILE_X - 1) / TILE_X) * ((a.cp.Lc[1] + TILE_Y - 1) / TILE_Y);
    int grid = plan.grid < ntiles ? plan.grid : ntiles;
    if (grid < 1) grid = 1;
    DWF_CHECK_CUDA(cudaMemsetAsync(bar, 0, 2 * sizeof(unsigned), st));   // count, gen; the error flag persists
    void* args[] = {&a};
    DWF_CHECK_CUDA(cudaLaunchCooperativeKernel((const void*)k_coarse_cgnr_persistent, dim3(grid), dim3(PCG_THREADS), args,
                                               sizeof(TileSmemT<float2>), st));
    return DWF_OK;
}


// ===========================================================================
// Persistent coarse GCR: one cooperative launch per coarse solve.
//
// Restarted GCR(KC) on B e = r_c, B = Dhat_PV^dag Dhat_DW (the level-2 solver
// type), to |r| <= coarse_tol |r_c| or maxiter steps.  Per step three bounded
// grid barriers separate the phases:
//   A. r_k = r_{k-1} - alpha_{k-1} w_{k-1} is formed while the tiles and their
//      halos are staged (each tile stores its own sites of r_k), and
//      t = Dhat_DW r_k is applied; partial |r_k|^2.          -> barrier
//      Stop if |r_k|^2 <= tol^2 |r_c|^2.
//   B. w = Dhat_PV^dag t, with the classical Gram-Schmidt dots <w_j, w>,
//      j < k, accumulated in the stencil's epilogue.         -> barrier
//   C. w_k = w - sum_j c_j w_j; partial |w_k|^2, <w_k, r_k>. -> barrier
//      alpha_k = <w_k, r_k> / |w_k|^2.
// The solution is not updated per step: the residuals r_j of a cycle are the
// raw search directions, and e += sum_j y_j r_j with (I + C)^T y = alpha is
// added once per cycle (during phase A of the next cycle's first step, or at
// the end).  The residual slots rotate over KC + 1 vectors so that the new
// cycle's first residual never overwrites a direction still being combined.
// Every block computes the same scalars from the same partials in the same
// order; barrier waits and bulk-copy waits are bounded (%globaltimer) and end
// in an error flag that the host reports as DWF_ERR_TIMEOUT.
// ===========================================================================
constexpr int PG_MAXK = 16;
constexpr int PGCR_BLOCKS_PER_SM = 2;     // resident blocks per SM used by the persistent GCR
constexpr int PG_NQ = 1 + 2 * PG_MAXK + 3;     // partial quantities: |r|^2 | dots | |w|^2, <w, r>

struct PgcrArgs {
    CoarseParams cp;
    const void* Y;          // Galerkin blocks (column-major, FP32 or FP16)
    const float2* rc;
    float2* e;
    float2* S[PG_MAXK + 1]; // residual slots
    float2* W[PG_MAXK];     // orthogonalised images
    float2* t;
    double* partials;       // [PG_NQ][gridDim.x]
    PcgBarrier* bar;
    int* out_iters;         // running total of steps over solves
    double* out_rr2;        // final |r|^2 / |r_c|^2
    double tol2;
    int maxiter;
    int KC;
    unsigned long long timeout_ns;
};

struct PgcrShared {
    double C[PG_MAXK][PG_MAXK][2];
    double A[PG_MAXK][2];
    double nrm[PG_MAXK];
    float2 coef[PG_MAXK];
    float2 y[PG_MAXK];
    double tot[PG_NQ];
};

// totals of nq partial quantities (layout [q][gridDim.x], gridDim.x <= 2 *
// blockDim.x) into out[q0 + q]: thread t adds partials t and t + blockDim.x of
// every quantity (all loads issued together), then a fixed-order block tree, so
// every block obtains bitwise identical totals after one round trip to L2
constexpr int PG_TOT_MAX = 36;
constexpr int PG_TOT_CHUNK = 8;      // quantities whose loads are in flight together
__device__ void pg_totals(const double* part, int q0, int nq, double* out) {
    __shared__ double sh[PG_TOT_CHUNK][TILE_THREADS / 32];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const unsigned b0 = threadIdx.x, b1 = threadIdx.x + blockDim.x;
    for (int c0 = 0; c0 < nq; c0 += PG_TOT_CHUNK) {
        double v[PG_TOT_CHUNK];
#pragma unroll
        for (int q = 0; q < PG_TOT_CHUNK; ++q) {
            v[q] = 0.0;
            if (c0 + q < nq) {
                const double* pq = part + (size_t)(q0 + c0 + q) * gridDim.x;
                const double x0 = b0 < gridDim.x ? __ldcg(pq + b0) : 0.0;
                const double x1 = b1 < gridDim.x ? __ldcg(pq + b1) : 0.0;
                v[q] = x0 + x1;
            }
        }
#pragma unroll
        for (int q = 0; q < PG_TOT_CHUNK; ++q) {
            if (c0 + q < nq) {
                double d = v[q];
                for (int off = 16; off > 0; off >>= 1) d += __shfl_down_sync(0xffffffffu, d, off);
                if (lane == 0) sh[q][warp] = d;
            }
        }
        __syncthreads();
        if (threadIdx.x < PG_TOT_CHUNK && c0 + (int)threadIdx.x < nq) {
            double sum = 0.0;
            for (int w = 0; w < TILE_THREADS / 32; ++w) sum += sh[threadIdx.x][w];
            out[q0 + c0 + threadIdx.x] = sum;
        }
        __syncthreads();
    }
}

// block partials of NQ per-thread FP32 values (first nq used) into part[(q0 + q) * grid + block]
template <int NQ>
__device__ void pg_partials(const float (&v)[NQ], int nq, double* part, int q0) {
    __shared__ double sh[NQ][TILE_THREADS / 32];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
        if (q < nq) {
            double d = v[q];
            for (int off = 16; off > 0; off >>= 1) d += __shfl_down_sync(0xffffffffu, d, off);
            if (lane == 0) sh[q][warp] = d;
        }
    }
    __syncthreads();
    for (int q = threadIdx.x; q < nq; q += blockDim.x) {
        double sum = 0.0;
        for (int w = 0; w < TILE_THREADS / 32; ++w) sum += sh[q][w];
        part[(size_t)(q0 + q) * gridDim.x + blockIdx.x] = sum;
    }
    __syncthreads();
}

// stage r = a - alpha b (b may be null) for the tile and its halo; the tile's
// own sites of r are stored to rout and their |r|^2 added to *nrm.  At most
// PG_STAGE elements per thread: all loads are issued before any use.
constexpr int PG_STAGE = (4 * TILE_HY * TILE_HX * 16 + TILE_THREADS - 1) / TILE_THREADS;
template <class BT>
__device__ __forceinline__ void pg_stage_axpy(TileSmemT<BT>& sm, const float2* a, const float2* b, float2 alpha,
                                              float2* rout, const CoarseParams& p, int x0, int y0, float& nrm) {
    const int L0 = p.Lc[0], L1 = p.Lc[1];
    const long long slice = p.Vc * 16;
    const int total = p.Ls_c * TILE_HY * TILE_HX * 16;
    long long idx[PG_STAGE];
    float2 va[PG_STAGE], vb[PG_STAGE];
#pragma unroll
    for (int u = 0; u < PG_STAGE; ++u) {
        const int e = threadIdx.x + u * TILE_THREADS;
        idx[u] = -1;
        if (e < total) {
            const int j = e & 15;
            const int h = (e >> 4) % (TILE_HY * TILE_HX);
            const int s = (e >> 4) / (TILE_HY * TILE_HX);
            const int hx = h % TILE_HX, hy = h / TILE_HX;
            const int gx = ((x0 + hx - 1) % L0 + L0) % L0, gy = ((y0 + hy - 1) % L1 + L1) % L1;
            idx[u] = s * slice + ((long long)gy * L0 + gx) * 16 + j;
            va[u] = __ldcg(a + idx[u]);
            vb[u] = b ? __ldcg(b + idx[u]) : make_float2(0.f, 0.f);
        }
    }
#pragma unroll
    for (int u = 0; u < PG_STAGE; ++u) {
        const int e = threadIdx.x + u * TILE_THREADS;
        if (e < total) {
            const int j = e & 15;
            const int h = (e >> 4) % (TILE_HY * TILE_HX);
            const int s = (e >> 4) / (TILE_HY * TILE_HX);
            const int hx = h % TILE_HX, hy = h / TILE_HX;
            float2 v = va[u];
            v.x -= alpha.x * vb[u].x - alpha.y * vb[u].y;
            v.y -= alpha.x * vb[u].y + alpha.y * vb[u].x;
            sm.v[s][hy][hx][j] = v;
            const bool own = hx >= 1 && hx <= TILE_X && hy >= 1 && hy <= TILE_Y && x0 + hx - 1 < L0 && y0 + hy - 1 < L1;
            if (own) {
                rout[idx[u]] = v;
                nrm += v.x * v.x + v.y * v.y;
            }
        }
    }
}

// stage the tile and its halo of `in` (all loads issued before any use)
template <class BT>
__device__ __forceinline__ void pg_stage(TileSmemT<BT>& sm, const float2* in, const CoarseParams& p, int x0, int y0) {
    const int L0 = p.Lc[0], L1 = p.Lc[1];
    const long long slice = p.Vc * 16;
    const int total = p.Ls_c * TILE_HY * TILE_HX * 16;
    float2 va[PG_STAGE];
#pragma unroll
    for (int u = 0; u < PG_STAGE; ++u) {
        const int e = threadIdx.x + u * TILE_THREADS;
        if (e < total) {
            const int j = e & 15;
            const int h = (e >> 4) % (TILE_HY * TILE_HX);
            const int s = (e >> 4) / (TILE_HY * TILE_HX);
            const int hx = h % TILE_HX, hy = h / TILE_HX;
            const int gx = ((x0 + hx - 1) % L0 + L0) % L0, gy = ((y0 + hy - 1) % L1 + L1) % L1;
            va[u] = __ldcg(in + s * slice + ((long long)gy * L0 + gx) * 16 + j);
        }
    }
#pragma unroll
    for (int u = 0; u < PG_STAGE; ++u) {
        const int e = threadIdx.x + u * TILE_THREADS;
        if (e < total) {
            const int j = e & 15;
            const int h = (e >> 4) % (TILE_HY * TILE_HX);
            const int s = (e >> 4) / (TILE_HY * TILE_HX);
            sm.v[s][h / TILE_HX][h % TILE_HX][j] = va[u];
        }
    }
}

// e += sum_{j<m} y_j S[(base + j) mod (KC + 1)] (grid-stride; y in shared memory)
__device__ __forceinline__ void pg_combine(const PgcrArgs& a, const PgcrShared& sh, int base, int m, long long n) {
    if (m <= 0) return;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i0 = (long long)blockIdx.x * blockDim.x + threadIdx.x; i0 < n; i0 += 4 * stride) {
        float2 x[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) if (i0 + u * stride < n) x[u] = a.e[i0 + u * stride];
        for (int j = 0; j < m; ++j) {
            const float2* Sj = a.S[(base + j) % (a.KC + 1)];
            const float2 y = sh.y[j];
            float2 r[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) if (i0 + u * stride < n) r[u] = __ldcg(Sj + i0 + u * stride);
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                x[u].x += y.x * r[u].x - y.y * r[u].y;
                x[u].y += y.x * r[u].y + y.y * r[u].x;
            }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) if (i0 + u * stride < n) a.e[i0 + u * stride] = x[u];
    }
}

// y of the deferred update over m steps: (I + C)^T y = A (thread 0, FP64)
__device__ __forceinline__ void pg_back_substitute(PgcrShared& sh, int m) {
    if (threadIdx.x == 0) {
        double yr[PG_MAXK], yi[PG_MAXK];
        for (int j = m - 1; j >= 0; --j) {
            double ar = sh.A[j][0], ai = sh.A[j][1];
            for (int k = j + 1; k < m; ++k) {
                ar -= sh.C[k][j][0] * yr[k] - sh.C[k][j][1] * yi[k];
                ai -= sh.C[k][j][0] * yi[k] + sh.C[k][j][1] * yr[k];
            }
            yr[j] = ar; yi[j] = ai;
            sh.y[j] = make_float2((float)ar, (float)ai);
        }
    }
    __syncthreads();
}

template <class BT>
__global__ void __launch_bounds__(TILE_THREADS, 2) k_coarse_gcr_persistent(PgcrArgs a) {
    extern __shared__ __align__(128) unsigned char pg_raw[];
    TileSmemT<BT>& sm = *reinterpret_cast<TileSmemT<BT>*>(pg_raw);
    __shared__ PgcrShared sh;
    const CoarseParams& p = a.cp;
    const BT* Y = reinterpret_cast<const BT*>(a.Y);
    const long long n = p.Vc * p.Ls_c * 16;
    const int KC = a.KC;
    const unsigned long long deadline = global_ns() + a.timeout_ns;
    const int ntx = (p.Lc[0] + TILE_X - 1) / TILE_X;
    const int ntiles = ntx * ((p.Lc[1] + TILE_Y - 1) / TILE_Y);
    double* partA = a.partials;                                   // quantity 0
    unsigned phase = 0;
    bool ok = true;
    if (threadIdx.x == 0) mbar_init(&sm.mbar, 1);
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        a.e[i] = make_float2(0.f, 0.f);
    __syncthreads();
    int base = 0, m = 0, it = 0;
    const float2* prevR = a.rc;          // r_{k-1} (or r_c before the first step)
    const float2* prevW = nullptr;       // w_{k-1}
    float2 prevA = make_float2(0.f, 0.f);
    double bn2 = 0.0, rr2 = 0.0;
    for (;;) {
        // ---- phase A: r_k and t = Dhat_DW r_k ----
        const bool roll = m == KC;
        if (roll) pg_back_substitute(sh, KC);                     // y of the cycle that just ended
        const int slot = (base + m) % (KC + 1);
        float2* Rk = a.S[slot];
        float nrA = 0.f;
        for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
            const int x0 = (tile % ntx) * TILE_X, y0 = (tile / ntx) * TILE_Y;
            __syncthreads();
            tile_issue_blocks(sm, Y, p, x0, y0);
            pg_stage_axpy(sm, prevR, prevW, prevA, Rk, p, x0, y0, nrA);
            __syncthreads();
            const bool okw = mbar_wait_bounded(&sm.mbar, phase, TILE_WAIT_NS);
            if (__syncthreads_or(!okw)) {                  // the whole block leaves together
                mbar_wait_bounded(&sm.mbar, phase, TILE_WAIT_NS);
                ok = false;
                break;
            }
            phase ^= 1u;
            tile_site(sm, a.t, p, x0, y0, p.mf, false);
        }
        if (roll) {                                               // e += sum_j y_j r_j of the ended cycle
            pg_combine(a, sh, base, KC, n);
            base = slot;
            m = 0;
        }
        {
            float v[1] = {nrA};
            pg_partials<1>(v, 1, partA, 0);
        }
        if (!pcg_sync(a.bar, deadline, ok)) return;
        pg_totals(a.partials, 0, 1, sh.tot);
        rr2 = sh.tot[0];
        if (it == 0) bn2 = rr2;
        if (bn2 == 0.0 || rr2 <= a.tol2 * bn2 || it >= a.maxiter) break;
        // ---- phase B: w = Dhat_PV^dag t with the dots <w_j, w>, j < m ----
        float dots[2 * (PG_MAXK - 1)];
#pragma unroll
        for (int q = 0; q < 2 * (PG_MAXK - 1); ++q) dots[q] = 0.f;
        float2* Wm = a.W[m];
        const int mm = m;
        for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
            const int x0 = (tile % ntx) * TILE_X, y0 = (tile / ntx) * TILE_Y;
            __syncthreads();
            tile_issue_blocks(sm, Y, p, x0, y0);
            pg_stage(sm, a.t, p, x0, y0);
            __syncthreads();
            const bool okw = mbar_wait_bounded(&sm.mbar, phase, TILE_WAIT_NS);
            if (__syncthreads_or(!okw)) {                  // the whole block leaves together
                mbar_wait_bounded(&sm.mbar, phase, TILE_WAIT_NS);
                ok = false;
                break;
            }
            phase ^= 1u;
            tile_site(sm, Wm, p, x0, y0, 1.0f, true, [&](long long idx, float2 w) {
#pragma unroll
                for (int j = 0; j < PG_MAXK - 1; ++j) {
                    if (j < mm) {
                        const float2 u = __ldcg(a.W[j] + idx);
                        dots[2 * j] += u.x * w.x + u.y * w.y;
                        dots[2 * j + 1] += u.x * w.y - u.y * w.x;
                    }
                }
            });
        }
        pg_partials<2 * (PG_MAXK - 1)>(dots, 2 * m, a.partials, 1);
        if (!pcg_sync(a.bar, deadline, ok)) return;
        if (m > 0) pg_totals(a.partials, 1, 2 * m, sh.tot);
        if (threadIdx.x < m) {
            const int j = threadIdx.x;
            const double nn = sh.nrm[j];
            const double cr = nn > 0 ? sh.tot[1 + 2 * j] / nn : 0.0, ci = nn > 0 ? sh.tot[2 + 2 * j] / nn : 0.0;
            sh.C[m][j][0] = cr;
            sh.C[m][j][1] = ci;
            sh.coef[j] = make_float2((float)cr, (float)ci);
        }
        __syncthreads();
        // ---- phase C: w_m = w - sum_j c_j w_j; |w_m|^2, <w_m, r_m> ----
        float vc[3] = {0.f, 0.f, 0.f};
        {
            const long long stride = (long long)gridDim.x * blockDim.x;
            for (long long i0 = (long long)blockIdx.x * blockDim.x + threadIdx.x; i0 < n; i0 += 4 * stride) {
                float2 w[4], r[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const long long i = i0 + u * stride;
                    if (i < n) { w[u] = __ldcg(Wm + i); r[u] = __ldcg(Rk + i); }
                }
                for (int j = 0; j < m; ++j) {
                    const float2 c = sh.coef[j];
                    float2 q[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const long long i = i0 + u * stride;
                        if (i < n) q[u] = __ldcg(a.W[j] + i);
                    }
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        w[u].x -= c.x * q[u].x - c.y * q[u].y;
                        w[u].y -= c.x * q[u].y + c.y * q[u].x;
                    }
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const long long i = i0 + u * stride;
                    if (i < n) {
                        if (m > 0) Wm[i] = w[u];
                        vc[0] += w[u].x * w[u].x + w[u].y * w[u].y;
                        vc[1] += w[u].x * r[u].x + w[u].y * r[u].y;
                        vc[2] += w[u].x * r[u].y - w[u].y * r[u].x;
                    }
                }
            }
        }
        pg_partials<3>(vc, 3, a.partials, 1 + 2 * PG_MAXK);
        if (!pcg_sync(a.bar, deadline, ok)) return;
        pg_totals(a.partials, 1 + 2 * PG_MAXK, 3, sh.tot);
        {
            const double ww = sh.tot[1 + 2 * PG_MAXK];
            const double ar = ww > 0 ? sh.tot[2 + 2 * PG_MAXK] / ww : 0.0;
            const double ai = ww > 0 ? sh.tot[3 + 2 * PG_MAXK] / ww : 0.0;
            if (threadIdx.x == 0) {
                sh.nrm[m] = ww;
                sh.A[m][0] = ar;
                sh.A[m][1] = ai;
            }
            prevA = make_float2((float)ar, (float)ai);
        }
        __syncthreads();
        prevR = Rk;
        prevW = Wm;
        ++m;
        ++it;
    }
    // final update with the steps of the current cycle
    pg_back_substitute(sh, m);
    pg_combine(a, sh, base, m, n);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        *a.out_iters += it;
        *a.out_rr2 = bn2 > 0 ? rr2 / bn2 : 0.0;
    }
}

// resident blocks per SM of the persistent coarse GCR, set up once per (device, block storage)
// under a mutex (the kernel's shared-memory limit is a per-device attribute)
template <class BT>
static dwf_status pgcr_blocks_per_sm(int* out) {
    static std::mutex mu;
    static int per_sm[64] = {0};
    int dev = 0;
    DWF_CHECK_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) { set_error("device ordinal %d out of range", dev); return DWF_ERR_UNSUPPORTED; }
    std::lock_guard<std::mutex> lock(mu);
    if (per_sm[dev] == 0) {
        const size_t smem = sizeof(TileSmemT<BT>);
        int per = 0;
        DWF_CHECK_CUDA(cudaFuncSetAttribute(k_coarse_gcr_persistent<BT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            (int)smem));
        DWF_CHECK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_coarse_gcr_persistent<BT>, TILE_THREADS,
                                                                     smem));
        if (per < 1) { set_error("persistent coarse GCR cannot be resident"); return DWF_ERR_UNSUPPORTED; }
        per_sm[dev] = per < PGCR_BLOCKS_PER_SM ? per : PGCR_BLOCKS_PER_SM;
    }
    *out = per_sm[dev];
    return DWF_OK;
}

template <class BT>
static dwf_status launch_pgcr(PgcrArgs& a, int nsm, cudaStream_t st) {
    const size_t smem = sizeof(TileSmemT<BT>);
    int per = 0;
    DWF_TRY(pgcr_blocks_per_sm<BT>(&per));
    const int ntiles = ((a.cp.Lc[0] + TILE_X - 1) / TILE_X) * ((a.cp.Lc[1] + TILE_Y - 1) / TILE_Y);
    int grid = nsm * per;
    if (grid > ntiles) grid = ntiles;
    if (grid < 1) grid = 1;
    void* args[] = {&a};
    DWF_CHECK_CUDA(cudaLaunchCooperativeKernel((const void*)k_coarse_gcr_persistent<BT>, dim3(grid), dim3(TILE_THREADS),
                                               args, smem, st));
    return DWF_OK;
}

bool coarse_gcr_persistent_ok(const dwf_mg* h) {
    return h->mg.nd == 2 && h->mg.ncd == 16 && h->mg.Ls_c <= 4 && h->prm.coarse_restart <= PG_MAXK &&
           h->prm.coarse_restart >= 1;
}

dwf_status coarse_gcr_persistent(const dwf_mg* h, const float2* rc, float2* ec, float2* const* S, float2* const* W,
                                 float2* t, double* partials, void* bar, int* out_iters, double* out_rr2,
                                 cudaStream_t st) {
    if (!coarse_gcr_persistent_ok(h)) {
        set_error("persistent coarse GCR supports 2-d, 16 coarse dof, Ls_c <= 4 and coarse_restart <= %d", PG_MAXK);
        return DWF_ERR_UNSUPPORTED;
    }
    int dev = 0, nsm = 0;
    DWF_CHECK_CUDA(cudaGetDevice(&dev));
    DWF_CHECK_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    PgcrArgs a;
    a.cp = coarse_params(h, h->mf);
    a.rc = rc;
    a.e = ec;
    const int KC = h->prm.coarse_restart;
    for (int k = 0; k <= PG_MAXK; ++k) a.S[k] = k <= KC ? S[k] : nullptr;
    for (int k = 0; k < PG_MAXK; ++k) a.W[k] = k < KC ? W[k] : nullptr;
    a.t = t;
    a.partials = partials;
    a.bar = (PcgBarrier*)bar;
    a.out_iters = out_iters;
    a.out_rr2 = out_rr2;
    a.tol2 = h->prm.coarse_tol * h->prm.coarse_tol;
    a.maxiter = h->prm.coarse_maxiter;
    a.KC = KC;
    a.timeout_ns = 5000000000ULL;   // 5 s per solve
    DWF_CHECK_CUDA(cudaMemsetAsync(bar, 0, 2 * sizeof(unsigned), st));   // count, gen; the error flag persists
    if (h->ytile_half) {
        a.Y = h->Ytile;
        return launch_pgcr<__half2>(a, nsm, st);
    }
    a.Y = h->Y32;
    return launch_pgcr<float2>(a, nsm, st);
}

}  // namespace dwf
