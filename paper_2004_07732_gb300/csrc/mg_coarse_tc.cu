// Coarse operator on many right-hand sides with tensor cores (Eq. coarsenDW).
//
// With nrhs coarse vectors on Ls_c slices the stencil at a coarse site is a
// dense contraction: out[:, c] = sum_dir Y_dir in_nbr(dir)[:, c] over the
// N = nrhs * Ls_c columns c = (rhs, slice).  In real arithmetic each complex
// 16 x 16 block is the 32 x 32 matrix [[Yr, -Yi], [Yi, Yr]] acting on
// [Re in; Im in].  One warp owns (site, 8 columns) and accumulates
// 2 (m-tiles) x 4 (k-tiles) x 5 (directions) mma.sync.m16n8k8 products in
// FP32.  Operands are FP32 data split into TF32 high and low parts (three
// products per term: hi*hi + hi*lo + lo*hi), which keeps FP32-level accuracy.
// The adjoint uses gamma_5-hermiticity, Dhat_W^dag = sigma_3 Dhat_W sigma_3.
// Vectors: the 16 complex64 values of one (column, coarse site) pair are
// contiguous; pair (c, x) starts at c * cs + x * ss complex values.  Two
// layouts: slice-major [rhs][s][coarse site][16] (cs = Vc * 16, ss = 16; the
// batched solver's) and site-major [coarse site][rhs][s][16] (cs = 16,
// ss = ncols * 16), where the 128 columns of one site are one contiguous
// 16 KB run.  Blocks: the FP32 column-major Galerkin blocks, or the FP16 copy.
// With FP16 blocks the contraction also has tcgen05 forms (accumulators in
// tensor memory): k_coarse_umma and k_coarse_umma_p keep both operands in
// shared memory (from 128 columns), k_coarse_umma_t keeps the data operand in
// tensor memory (from 64 columns).  The autotuner (coarse_tc = 0) times the
// eligible forms on first use and keeps the fastest; coarse_tc 1-6 fix one.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <mutex>

#include "mg.cuh"
#include "async_copy.cuh"
#include "mma_tf32.cuh"

namespace dwf {
namespace {

struct TcParams {
    long long Vc;
    int Lc0, Lc1;
    int Ls_c, nrhs, ncols;
    float mf;
    int dag;
    long long cs, ss;     // complex values between columns and between coarse sites
};

__device__ __forceinline__ long long nbr2d(const TcParams& p, long long xc, int dir) {
    if (dir == 0) return xc;
    const int x = (int)(xc % p.Lc0), y = (int)(xc / p.Lc0);
    int nx = x, ny = y;
    if (dir == 1) nx = x + 1 == p.Lc0 ? 0 : x + 1;
    else if (dir == 2) nx = x == 0 ? p.Lc0 - 1 : x - 1;
    else if (dir == 3) ny = y + 1 == p.Lc1 ? 0 : y + 1;
    else ny = y == 0 ? p.Lc1 - 1 : y - 1;
    return (long long)ny * p.Lc0 + nx;
}

// blockDim = 256 (8 warps); warp -> (site, group of NT column tiles of 8).
// The k dimension is walked in two halves (input components j = t + {0, 4} and
// j = 8 + t + {0, 4}); each half covers the real and the imaginary k-tile of the
// same input values, so every input value is loaded and split once.
__device__ __forceinline__ float2 block_val(const float2* p) { return __ldg(p); }
__device__ __forceinline__ float2 block_val(const __half2* p) { return __half22float2(__ldg(p)); }

// BT = float2: FP32 blocks, split into TF32 high and low parts (three products
// per term).  BT = __half2: FP16 blocks, exact in TF32 (same 11-bit
// significand), so only the vectors are split (two products per term).
template <int NT, class BT>
__global__ void __launch_bounds__(256, 2) k_coarse_tc(const BT* __restrict__ Y, const float2* __restrict__ in,
                                                      float2* __restrict__ out, TcParams p,
                                                      const int* __restrict__ skip_rhs) {
    constexpr bool SPLIT_A = sizeof(BT) == sizeof(float2);
    const int lane = threadIdx.x & 31;
    const long long wid = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int ngroup = (p.ncols + 8 * NT - 1) / (8 * NT);
    const long long xc = wid / ngroup;
    const int cg = (int)(wid % ngroup);
    if (xc >= p.Vc) return;
    const int g = lane >> 2, t = lane & 3;
    long long baseB[NT];
    bool okB[NT];
#pragma unroll
    for (int k = 0; k < NT; ++k) {
        const int col = (cg * NT + k) * 8 + g;           // B column owned by this lane in tile k
        okB[k] = col < p.ncols && !(skip_rhs && skip_rhs[col / p.Ls_c]);
        baseB[k] = okB[k] ? (long long)col * p.cs : 0;
    }
    bool any = false;
#pragma unroll
    for (int k = 0; k < NT; ++k) any |= okB[k];
    if (!__any_sync(0xffffffffu, any)) return;        // every column of this warp is skipped
    float acc[NT][2][4];
#pragma unroll
    for (int k = 0; k < NT; ++k)
#pragma unroll
        for (int m = 0; m < 2; ++m)
#pragma unroll
            for (int u = 0; u < 4; ++u) acc[k][m][u] = 0.f;
    const float sgn_hi = p.dag ? -1.f : 1.f;             // sigma_3 on input components 8..15
#pragma unroll 1
    for (int dir = 0; dir < 5; ++dir) {
        const long long nb = nbr2d(p, xc, dir);
        const BT* Yb = Y + (xc * 5 + dir) * 256;
#pragma unroll
        for (int half = 0; half < 2; ++half) {
            // block entries Y[i][j], i = g + 8h, j = 8 half + t + 4 w (column-major: j * 16 + i)
            float2 y[2][2];
#pragma unroll
            for (int h = 0; h < 2; ++h)
#pragma unroll
                for (int w = 0; w < 2; ++w) y[h][w] = block_val(Yb + (8 * half + t + 4 * w) * 16 + g + 8 * h);
            // A fragments of [[Yr, -Yi], [Yi, Yr]] for m-tile mt (real / imaginary output rows) and the
            // real (ri = 0) or imaginary (ri = 1) input k-tile: a0 (g, t), a1 (g+8, t), a2 (g, t+4), a3 (g+8, t+4)
            uint32_t ah[2][2][4], al[2][2][4];
#pragma unroll
            for (int mt = 0; mt < 2; ++mt)
#pragma unroll
                for (int ri = 0; ri < 2; ++ri)
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const float2 yy = y[u & 1][u >> 1];
                        const float e = mt == 0 ? (ri == 0 ? yy.x : -yy.y) : (ri == 0 ? yy.y : yy.x);
                        if (SPLIT_A) split_tf32(e, ah[mt][ri][u], al[mt][ri][u]);
                        else { ah[mt][ri][u] = __float_as_uint(e); al[mt][ri][u] = 0u; }
                    }
#pragma unroll
            for (int k = 0; k < NT; ++k) {
                // B fragments: b0 = k-row t, b1 = k-row t + 4 of column g
                float2 v0 = make_float2(0.f, 0.f), v1 = make_float2(0.f, 0.f);
                if (okB[k]) {
                    const float2* src = in + baseB[k] + nb * p.ss + 8 * half + t;
                    v0 = __ldg(src);
                    v1 = __ldg(src + 4);
                }
                if (half == 1) { v0.x *= sgn_hi; v0.y *= sgn_hi; v1.x *= sgn_hi; v1.y *= sgn_hi; }
                uint32_t bh[2][2], bl[2][2];
                split_tf32(v0.x, bh[0][0], bl[0][0]);
                split_tf32(v1.x, bh[0][1], bl[0][1]);
                split_tf32(v0.y, bh[1][0], bl[1][0]);
                split_tf32(v1.y, bh[1][1], bl[1][1]);
#pragma unroll
                for (int mt = 0; mt < 2; ++mt)
#pragma unroll
                    for (int ri = 0; ri < 2; ++ri) {
                        mma_tf32(acc[k][mt], ah[mt][ri], bh[ri]);
                        mma_tf32(acc[k][mt], ah[mt][ri], bl[ri]);
                        if (SPLIT_A) mma_tf32(acc[k][mt], al[mt][ri], bh[ri]);
                    }
            }
        }
    }
    // epilogue: lane owns rows i = g + 8h and columns 2t + w of each tile; adds the identity and the
    // chiral hopping along the coarse fifth dimension
#pragma unroll
    for (int k = 0; k < NT; ++k)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int i = g + 8 * h;
            const float so = (p.dag && h == 1) ? -1.f : 1.f;
            const bool from_below = p.dag ? (h == 1) : (h == 0);
#pragma unroll
            for (int w = 0; w < 2; ++w) {
                const int col = (cg * NT + k) * 8 + 2 * t + w;
                if (col >= p.ncols) continue;
                const int r = col / p.Ls_c, s = col % p.Ls_c;
                if (skip_rhs && skip_rhs[r]) continue;
                const long long rb = (long long)r * p.Ls_c * p.cs + xc * p.ss + i;
                const float hr = so * acc[k][0][2 * h + w], hi = so * acc[k][1][2 * h + w];
                const float2 self = __ldg(in + rb + (long long)s * p.cs);
                int sh;
                float sc = 1.f;
                if (from_below) { if (s > 0) sh = s - 1; else { sh = p.Ls_c - 1; sc = -p.mf; } }
                else            { if (s < p.Ls_c - 1) sh = s + 1; else { sh = 0; sc = -p.mf; } }
                const float2 hv = __ldg(in + rb + (long long)sh * p.cs);
                out[rb + (long long)s * p.cs] = make_float2(hr + self.x + sc * hv.x, hi + self.y + sc * hv.y);
            }
        }
}

// ---------------------------------------------------------------------------
// tcgen05 form (5th-generation tensor cores, accumulator in tensor memory).
//
// Transposed contraction per coarse site: D[c][n] = sum_dir sum_k A_dir[c][k]
// B_dir[n][k], where the rows c are a tile of 128 columns (rhs, slice), A_dir
// holds the real form [Re v_j | Im v_j] (k < 32) of the neighbour's input
// vectors and B_dir[n][k] the real form [[Yr, -Yi], [Yi, Yr]] of the block
// (rows n: Re out_i, then Im out_i).  One CTA per (site, column tile): the
// five weight matrices are staged once, the inputs of one direction at a time
// into one of two buffers (TF32 high and low parts, so that A = A_hi + A_lo
// keeps FP32 accuracy; FP16 blocks are exact in TF32), and one thread issues
// the K = 8 MMAs of each direction; a tcgen05.commit on the buffer's mbarrier
// frees the buffer for the direction after next.  Operands sit in shared
// memory in the K-major layout without swizzle (8 rows x 16 bytes per core
// matrix, 128 bytes between K-adjacent core matrices, 1024 bytes between row
// groups).  The 128 x 32 FP32 accumulator lives in 32 TMEM columns; warps 0-3
// read it back (lane = row) and add the identity and the s-hops.  Measured at
// 64^2 x 4 coarse sites and 64 right-hand sides: 400 us against 224 us for the
// mma.sync kernel -- one site per CTA leaves the staging and the five
// commit/wait steps unhidden at two CTAs per SM -- so it is opt-in.
// ---------------------------------------------------------------------------
constexpr int UM_M = 128, UM_K = 32, UM_N = 32, UM_THREADS = 256, UM_DIRS = 5;
constexpr uint32_t UM_LBO = 128, UM_SBO = 1024;
constexpr unsigned long long UM_WAIT_NS = 2000000000ULL;
struct UmSmem {
    float a[2][2][UM_M * UM_K];          // [buffer][hi, lo]
    float b[UM_DIRS][UM_N * UM_K];       // weights per direction
    unsigned long long mbar[3];          // buffers 0, 1; all MMAs done
    uint32_t tmem;
};

// float offset of element (row, k) in the K-major no-swizzle layout
__device__ __forceinline__ int um_off(int row, int k) {
    return (row >> 3) * (UM_SBO / 4) + (k >> 2) * (UM_LBO / 4) + (row & 7) * 4 + (k & 3);
}

__device__ __forceinline__ uint64_t um_desc(const void* base) {
    uint64_t d = 0;
    d |= (uint64_t)((smem_u32(base) >> 4) & 0x3FFF);
    d |= (uint64_t)((UM_LBO >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)((UM_SBO >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;                                  // descriptor version; no swizzle, base offset 0
    return d;
}

__device__ __forceinline__ void um_mma(uint32_t dt, uint64_t da, uint64_t db, uint32_t idesc, uint32_t acc) {
    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                 "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}"
                 ::"r"(dt), "l"(da), "l"(db), "r"(idesc), "r"(acc) : "memory");
}

__device__ __forceinline__ void um_commit(unsigned long long* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

// inputs of direction d for the tile's 128 columns: thread t holds half jh = t & 1 (8 complex values)
// of column t >> 1; zeros for columns past the end or of skipped right-hand sides
__device__ __forceinline__ void um_load_a(float4 (&v)[4], const float2* __restrict__ in, const TcParams& p, long long nb,
                                          int col0, const int* skip_rhs) {
    const int t = threadIdx.x, m = t >> 1, jh = t & 1;
    const int col = col0 + m;
    bool ok = col < p.ncols;
    if (ok && skip_rhs) ok = skip_rhs[col / p.Ls_c] == 0;
    if (ok) {
        const float4* src = reinterpret_cast<const float4*>(in + (long long)col * p.cs + nb * p.ss + 8 * jh);
#pragma unroll
        for (int q = 0; q < 4; ++q) v[q] = __ldg(src + q);
    } else {
#pragma unroll
        for (int q = 0; q < 4; ++q) v[q] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
}

// the held values as TF32 high and low parts in the operand layout (hi, lo: one operand buffer each)
__device__ __forceinline__ void um_store_ab(float* __restrict__ ahi, float* __restrict__ alo, const float4 (&v)[4],
                                            const TcParams& p) {
    const int t = threadIdx.x, m = t >> 1, jh = t & 1;
    const float sg = (p.dag && jh == 1) ? -1.f : 1.f;       // sigma_3 on input components 8..15
    float re[8], im[8];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        re[2 * q] = sg * v[q].x; im[2 * q] = sg * v[q].y;
        re[2 * q + 1] = sg * v[q].z; im[2 * q + 1] = sg * v[q].w;
    }
#pragma unroll
    for (int half = 0; half < 2; ++half) {                  // real parts at k = 8 jh .., imaginary at 16 + 8 jh ..
        const float* x = half == 0 ? re : im;
        const int k0 = 16 * half + 8 * jh;
#pragma unroll
        for (int g = 0; g < 2; ++g) {
            float hi[4], lo[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                hi[u] = __uint_as_float(to_tf32(x[4 * g + u]));
                lo[u] = x[4 * g + u] - hi[u];
            }
            const int o = um_off(m, k0 + 4 * g);
            *reinterpret_cast<float4*>(&ahi[o]) = make_float4(hi[0], hi[1], hi[2], hi[3]);
            *reinterpret_cast<float4*>(&alo[o]) = make_float4(lo[0], lo[1], lo[2], lo[3]);
        }
    }
}

// weights of the five directions: B_d[n][k] (real form of the FP16 block Y[xc][d], column-major
// j * 16 + i), written by threads t0 of nt
__device__ __forceinline__ void um_build_b(float (*b)[UM_N * UM_K], const __half2* __restrict__ Y, long long xc, int t0,
                                           int nt) {
    for (int e = t0; e < UM_DIRS * 256; e += nt) {
        const int d = e >> 8, j = (e >> 4) & 15, i = e & 15;
        const float2 y = __half22float2(__ldg(Y + (xc * UM_DIRS + d) * 256 + e % 256));
        float* bd = b[d];
        bd[um_off(i, j)] = y.x;
        bd[um_off(i, 16 + j)] = -y.y;
        bd[um_off(16 + i, j)] = y.y;
        bd[um_off(16 + i, 16 + j)] = y.x;
    }
}

__global__ void __launch_bounds__(UM_THREADS) k_coarse_umma(const __half2* __restrict__ Y, const float2* __restrict__ in,
                                                           float2* __restrict__ out, TcParams p,
                                                           const int* __restrict__ skip_rhs, int* status) {
    extern __shared__ __align__(1024) unsigned char um_raw[];
    UmSmem& sm = *reinterpret_cast<UmSmem*>(um_raw);
    const int t = threadIdx.x, warp = t >> 5;
    const int ntile = (p.ncols + UM_M - 1) / UM_M;
    const long long xc = blockIdx.x / ntile;
    const int col0 = (int)(blockIdx.x % ntile) * UM_M;
    if (t == 0) {
        for (int b = 0; b < 3; ++b) mbar_init(&sm.mbar[b], 1);
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&sm.tmem)),
                     "r"(UM_N) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    // every direction's inputs are requested before anything waits on them
    const TcParams& pp = p;
    float4 va[UM_DIRS][4];
#pragma unroll
    for (int d = 0; d < UM_DIRS; ++d) um_load_a(va[d], in, pp, nbr2d(pp, xc, d), col0, skip_rhs);
    um_build_b(sm.b, Y, xc, t, UM_THREADS);
    um_store_ab(sm.a[0][0], sm.a[0][1], va[0], pp);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t dt = sm.tmem;
    // D F32, A and B TF32, both K-major, N = 32, M = 128
    const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(UM_N >> 3) << 17) | ((uint32_t)(UM_M >> 4) << 24);
    bool ok = true;
#pragma unroll
    for (int d = 0; d < UM_DIRS; ++d) {
        const int buf = d & 1;
        if (t == 0) {
#pragma unroll
            for (int ks = 0; ks < UM_K / 8; ++ks) {
                const uint64_t db = um_desc(reinterpret_cast<const char*>(sm.b[d]) + ks * 2 * UM_LBO);
                const uint64_t dah = um_desc(reinterpret_cast<const char*>(sm.a[buf][0]) + ks * 2 * UM_LBO);
                const uint64_t dal = um_desc(reinterpret_cast<const char*>(sm.a[buf][1]) + ks * 2 * UM_LBO);
                um_mma(dt, dah, db, idesc, (d > 0 || ks > 0) ? 1u : 0u);
                um_mma(dt, dal, db, idesc, 1u);
            }
            um_commit(&sm.mbar[buf]);
            if (d == UM_DIRS - 1) um_commit(&sm.mbar[2]);
        }
        if (d + 1 < UM_DIRS) {
            const int nb_buf = (d + 1) & 1;
            if (d + 1 >= 2)                                   // the MMAs of direction d - 1 have read the buffer
                ok = ok && mbar_wait_bounded(&sm.mbar[nb_buf], (unsigned)(((d - 1) >> 1) & 1), UM_WAIT_NS);
            um_store_ab(sm.a[nb_buf][0], sm.a[nb_buf][1], va[d + 1 < UM_DIRS ? d + 1 : 0], pp);
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncthreads();
        }
    }
    ok = ok && mbar_wait_bounded(&sm.mbar[2], 0u, UM_WAIT_NS);
    if (!ok) {                                       // record, then give the MMAs a second bounded wait
        if (t == 0) atomicExch(status, 3);
        mbar_wait_bounded(&sm.mbar[2], 0u, UM_WAIT_NS);
    }
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    // After a timed-out wait the accumulator is not read (its warp skips the tensor-memory load
    // together), no output is written, status 3 reports the failure, and the TMEM is freed at the
    // end without further waiting.
    const bool warp_ok = __all_sync(0xffffffffu, ok);
    if (warp < 4 && warp_ok) {
        // row m = t of D: column col0 + t
        uint32_t r[32];
        const uint32_t taddr = dt + ((uint32_t)(32 * warp) << 16);
        asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
                     "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                     : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                       "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
                       "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
                       "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
                       "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
                     : "r"(taddr));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        const int col = col0 + t;
        bool live = ok && col < p.ncols;
        if (live && skip_rhs) live = skip_rhs[col / p.Ls_c] == 0;
        if (live) {
            const int rr = col / p.Ls_c, s = col % p.Ls_c;
            const long long rb = (long long)rr * p.Ls_c * p.cs + xc * p.ss;
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                const float so = (p.dag && i >= 8) ? -1.f : 1.f;
                const bool from_below = p.dag ? (i >= 8) : (i < 8);
                int sh;
                float sc = 1.f;
                if (from_below) { if (s > 0) sh = s - 1; else { sh = p.Ls_c - 1; sc = -p.mf; } }
                else            { if (s < p.Ls_c - 1) sh = s + 1; else { sh = 0; sc = -p.mf; } }
                const float2 self = __ldg(in + rb + (long long)s * p.cs + i);
                const float2 hv = __ldg(in + rb + (long long)sh * p.cs + i);
                out[rb + (long long)s * p.cs + i] =
                    make_float2(so * __uint_as_float(r[i]) + self.x + sc * hv.x,
                                so * __uint_as_float(r[16 + i]) + self.y + sc * hv.y);
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(dt), "r"(UM_N) : "memory");
}

// ---------------------------------------------------------------------------
// Persistent, warp-specialised tcgen05 form.  One CTA per SM walks the work
// items (coarse site, tile of 128 columns) item = blockIdx.x + k gridDim.x, so
// the CTAs together sweep the lattice in site order and a site's inputs, read
// by the items of its four neighbours, are found in L2.
//
// Here the K index of the real form runs over (Re v_j, Im v_j) pairs, k = 2 j
// and 2 j + 1: the order of the complex inputs in memory.  One tensor copy (TMA)
// per (item, direction) stage then brings the tile's 128 column rows straight
// into the K-major operand layout with the 128-byte swizzle, where the tensor core
// reads them as TF32 (the high part, mantissa truncated); the producer threads
// add the low part x - trunc(x) as a second operand in the same layout.  The weight matrices take the same K order,
// and the sigma_3 signs of the adjoint (on input components 8..15 and output
// components 8..15) are folded into them.
//
// Roles:
//   warps 0-7   producers: thread 0 issues the tensor copy of each stage UP_DIST
//               stages ahead into a ring of UP_OPS operand stages; every thread
//               writes the low parts of its share once a stage has landed; per
//               item the five weight matrices (double-buffered by item) from FP16
//               blocks loaded one item ahead;
//   warp 12     lane 0 issues the 8 MMAs of each direction into that direction's
//               TMEM accumulator (32 columns; 2 items x 5 directions) and commits
//               each stage back to the producers and each finished item to the
//               epilogue;
//   warps 8-11  epilogue: the sum of the previous item's five accumulators from
//               TMEM, plus the identity and the s-hops (the item's own inputs, by
//               tensor copy), staged through shared memory so that each warp
//               stores whole 128-byte column rows, while the next item's MMAs run.
// Every mbarrier wait is bounded by %globaltimer; a wait that runs out sets the
// status word and an abort flag that ends every role's loop; thread 0 then waits
// (bounded) for its tensor copies in flight, the issuing thread for its MMAs,
// and the TMEM is freed.
// ---------------------------------------------------------------------------
constexpr int UP_HI = 6;                       // stages of raw inputs (the TF32 high parts), filled by TMA
constexpr int UP_LO = 2;                       // stages of low parts
constexpr int UP_DIST = UP_HI - 2;             // tensor copies in flight ahead of the current stage
constexpr int UP_PROD = 256, UP_EPI = 128, UP_THREADS = UP_PROD + UP_EPI + 32;
constexpr uint32_t UP_STAGE_BYTES = UM_M * UM_K * 4;
constexpr int UP_OROW = UM_K + 4;              // floats per row of the padded output staging tile
// one 32-column TMEM accumulator per (item parity, direction): the 8 MMAs of a direction form
// the only dependent chain, so the directions' MMAs overlap in the tensor pipe
constexpr int UP_TMEM_COLS = 512;
struct UpSmem {
    float hi[UP_HI][UM_M * UM_K];                // raw FP32 inputs of a stage (core-matrix order)
    float lo[UP_LO][UM_M * UM_K];                // x - trunc_tf32(x) of a stage
    float b[2][UM_DIRS][UM_N * UM_K];            // weights, double-buffered by item
    float e[2][UM_M * UM_K];                     // the item's own inputs for the epilogue (core-matrix order)
    float o[UM_M * UP_OROW];                     // output staging, [column][32 floats + pad]
    unsigned long long tma[UP_HI], ehi[UP_HI], full[UP_LO], elo[UP_LO];
    unsigned long long wfull[2], wempty[2], tfull[2], tempty[2], efull[2], done;
    uint32_t tmem;
    int abort;
};

// Bounded wait that also gives up once another role has aborted.  SLEEP > 0 backs off
// between polls (roles whose wait is not on the critical path).
template <int SLEEP>
__device__ __forceinline__ bool up_wait(UpSmem& sm, unsigned long long* bar, unsigned parity, int* status) {
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = now_ns();
    for (unsigned it = 1;; ++it) {
        if (SLEEP > 0) __nanosleep(SLEEP);
        if (mbar_try_wait(bar, parity)) return true;
        if ((it & 15) == 0) {
            if (*(volatile int*)&sm.abort) return false;
            if (now_ns() - t0 > UM_WAIT_NS) {
                *(volatile int*)&sm.abort = 1;
                atomicExch(status, 3);
                return false;
            }
        }
    }
}
__device__ __forceinline__ void up_arrive(unsigned long long* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
// named barrier 1 over the 128 epilogue threads; epi_any also returns the OR of v over them
__device__ __forceinline__ void epi_sync() { asm volatile("bar.sync 1, 128;" ::: "memory"); }
__device__ __forceinline__ bool epi_any(bool v) {
    uint32_t r;
    asm volatile("{\n\t.reg .pred p, q;\n\tsetp.ne.u32 p, %1, 0;\n\tbar.red.or.pred q, 1, 128, p;\n\t"
                 "selp.u32 %0, 1, 0, q;\n\t}"
                 : "=r"(r) : "r"((uint32_t)v) : "memory");
    return r != 0;
}
// bounded wait for a tensor copy that nobody else waits for (before the CTA ends)
__device__ __forceinline__ void up_drain(unsigned long long* bar, unsigned parity) {
    const unsigned long long t0 = now_ns();
    while (!mbar_try_wait(bar, parity) && now_ns() - t0 < UM_WAIT_NS) {}
}

// Operand A of the persistent form in the K-major layout with the 128-byte swizzle: row r
// (a column of the tile) holds its 32 K values in 128 bytes, 16-byte chunk c of the row at
// chunk position c ^ (r & 7); 8-row groups are 1024 bytes apart.  Float offset of (r, k):
__device__ __forceinline__ int sw_off(int r, int k) { return r * 32 + ((((k >> 2) ^ r) & 7) << 2) + (k & 3); }
// its shared-memory descriptor (the K position within the row advances the start address)
__device__ __forceinline__ uint64_t sw_desc(const void* base) {
    uint64_t d = 0;
    d |= (uint64_t)((smem_u32(base) >> 4) & 0x3FFF);
    d |= (uint64_t)1 << 16;                                  // leading byte offset: unused with the swizzle
    d |= (uint64_t)(1024 >> 4) << 32;                        // stride byte offset: 8 rows x 128 bytes
    d |= (uint64_t)1 << 46;                                  // descriptor version
    d |= (uint64_t)2 << 61;                                  // 128-byte swizzle
    return d;
}

// Inputs of one tile at one site as one tensor copy.  The tensor map views the input vectors
// as 3-d FP32 data (k, column, site) with strides (4 B, cs, ss), k = 2 j + (0: Re, 1: Im) of
// input component j, column = rhs Ls_c + s; the box (32, 128, 1) of columns
// 128 t .. 128 t + 127 at site nb lands in shared memory as 128 rows of 128 bytes with the
// 128-byte swizzle, the layout of operand A.  Columns past the last one are filled with zeros.
__device__ __forceinline__ void up_tma(float* dst, unsigned long long* bar, const CUtensorMap* tmap, int tile,
                                       long long nb) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(UP_STAGE_BYTES)
                 : "memory");
    asm volatile("cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
                 " [%0], [%1, {%2, %3, %4}], [%5];"
                 ::"r"(smem_u32(dst)), "l"(reinterpret_cast<uint64_t>(tmap)), "r"(0), "r"(UM_M * tile), "r"((int)nb),
                   "r"(smem_u32(bar))
                 : "memory");
}

__global__ void __launch_bounds__(UP_THREADS, 1) k_coarse_umma_p(const __half2* __restrict__ Y,
                                                                const float2* __restrict__ in,
                                                                float2* __restrict__ out, TcParams p,
                                                                const int* __restrict__ skip_rhs, int* status,
                                                                const __grid_constant__ CUtensorMap tmap) {
    extern __shared__ __align__(1024) unsigned char up_raw[];
    UpSmem& sm = *reinterpret_cast<UpSmem*>(up_raw);
    const int t = threadIdx.x, warp = t >> 5;
    const int ntile = (p.ncols + UM_M - 1) / UM_M;
    const long long nitems = p.Vc * ntile;
    if (t == 0) {
        for (int i = 0; i < UP_HI; ++i) { mbar_init(&sm.tma[i], 1); mbar_init(&sm.ehi[i], 1); }
        for (int i = 0; i < UP_LO; ++i) { mbar_init(&sm.full[i], UP_PROD); mbar_init(&sm.elo[i], 1); }
        for (int i = 0; i < 2; ++i) {
            mbar_init(&sm.wfull[i], UP_PROD);
            mbar_init(&sm.wempty[i], 1);
            mbar_init(&sm.tfull[i], 1);
            mbar_init(&sm.tempty[i], UP_EPI);
            mbar_init(&sm.efull[i], 1);
        }
        mbar_init(&sm.done, 1);
        // the swizzled tensor copies and operands need 1024-byte aligned buffers
        sm.abort = ((smem_u32(sm.hi) | smem_u32(sm.lo) | smem_u32(sm.e)) & 1023u) != 0;
        if (sm.abort) atomicExch(status, 3);
    }
    if (warp == 12) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&sm.tmem)),
                     "r"(UP_TMEM_COLS) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = sm.tmem;
    // items of this CTA: il = 0 .. nmine - 1, item = blockIdx.x + il gridDim.x
    const long long nmine = (blockIdx.x < nitems && !sm.abort) ? (nitems - 1 - blockIdx.x) / gridDim.x + 1 : 0;
    const long long nstages = nmine * UM_DIRS;
    auto item_of = [&](long long il) { return blockIdx.x + il * gridDim.x; };

    if (warp < 8) {
        // ---------------- producers ----------------
        // thread t writes the low parts of chunk c = t & 7 of rows (t >> 3) + 32 i (a quarter-warp
        // covers one whole 128-byte row)
        const int cq = t & 7, rb = t >> 3;
        auto stage_tma = [&](long long g) {
            const long long item = item_of(g / UM_DIRS);
            const int s = (int)(g % UP_HI);
            up_tma(sm.hi[s], &sm.tma[s], &tmap, (int)(item % ntile), nbr2d(p, item / ntile, (int)(g % UM_DIRS)));
        };
        long long issued = 0, landed = 0;             // tensor copies issued (thread 0) and waited for
        if (t == 0) {
            asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmap)) : "memory");
            for (; issued < UP_DIST && issued < nstages; ++issued) stage_tma(issued);
        }
        __half2 yv[UM_DIRS];
        if (nmine > 0) {
            const long long xc0 = blockIdx.x / ntile;
#pragma unroll
            for (int k = 0; k < UM_DIRS; ++k) yv[k] = __ldg(Y + xc0 * (UM_DIRS * 256) + t + 256 * k);
        }
        for (long long g = 0; g < nstages; ++g) {
            const long long il = g / UM_DIRS;
            const int d = (int)(g % UM_DIRS);
            if (d == 0) {
                // the weights of item il (Y loaded one item ahead): B[n][k] with k = 2 j (Re v_j),
                // 2 j + 1 (Im v_j); rows n < 16: Re out_n, n = 16 + i: Im out_i
                const int bb = (int)(il & 1);
                const long long ub = il >> 1;
                if (ub >= 1 && !up_wait<0>(sm, &sm.wempty[bb], (unsigned)((ub - 1) & 1), status)) break;
#pragma unroll
                for (int k = 0; k < UM_DIRS; ++k) {
                    const int e = t + 256 * k;
                    const int j = (e >> 4) & 15, i = e & 15;
                    float2 y = __half22float2(yv[k]);
                    if (p.dag && ((i >= 8) != (j >= 8))) { y.x = -y.x; y.y = -y.y; }   // sigma_3 Y sigma_3
                    float* bd = sm.b[bb][k];
                    bd[um_off(i, 2 * j)] = y.x;
                    bd[um_off(i, 2 * j + 1)] = -y.y;
                    bd[um_off(16 + i, 2 * j)] = y.y;
                    bd[um_off(16 + i, 2 * j + 1)] = y.x;
                }
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                up_arrive(&sm.wfull[bb]);
                if (il + 1 < nmine) {
                    const long long xn = item_of(il + 1) / ntile;
#pragma unroll
                    for (int k = 0; k < UM_DIRS; ++k) yv[k] = __ldg(Y + xn * (UM_DIRS * 256) + t + 256 * k);
                }
            }
            // the tensor copy of stage g has landed and the low-part slot is free: x - trunc_tf32(x)
            const int s = (int)(g % UP_HI), l = (int)(g % UP_LO);
            if (!up_wait<0>(sm, &sm.tma[s], (unsigned)((g / UP_HI) & 1), status)) break;
            landed = g + 1;
            if (g >= UP_LO && !up_wait<0>(sm, &sm.elo[l], (unsigned)(((g - UP_LO) / UP_LO) & 1), status)) break;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int o = sw_off(rb + 32 * q, 4 * cq);
                const float4 v = *reinterpret_cast<const float4*>(&sm.hi[s][o]);
                float4 lo;
                lo.x = v.x - __uint_as_float(__float_as_uint(v.x) & 0xffffe000u);
                lo.y = v.y - __uint_as_float(__float_as_uint(v.y) & 0xffffe000u);
                lo.z = v.z - __uint_as_float(__float_as_uint(v.z) & 0xffffe000u);
                lo.w = v.w - __uint_as_float(__float_as_uint(v.w) & 0xffffe000u);
                *reinterpret_cast<float4*>(&sm.lo[l][o]) = lo;
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            up_arrive(&sm.full[l]);
            // stage g + UP_DIST goes into the raw slot of stage g - 2 once its MMAs are done
            if (t == 0 && g + UP_DIST < nstages) {
                const long long gn = g + UP_DIST;
                if (gn >= UP_HI && !up_wait<0>(sm, &sm.ehi[gn % UP_HI], (unsigned)(((gn - UP_HI) / UP_HI) & 1), status))
                    break;
                stage_tma(gn);
                issued = gn + 1;
            }
        }
        // after an early exit: the tensor copies still in flight land before the CTA ends
        if (t == 0)
            for (long long g = landed; g < issued; ++g) up_drain(&sm.tma[g % UP_HI], (unsigned)((g / UP_HI) & 1));
    } else if (warp < 12) {
        // ---------------- epilogue ----------------
        const int te = t - UP_PROD;                  // row of the accumulator = column of the tile
        const int wq = warp & 3;                     // TMEM lanes 32 wq .. 32 wq + 31
        long long eissued = 0, elanded = 0;          // own-input copies issued (te == 0) and waited for
        auto item_tma = [&](long long il) {
            const long long item = item_of(il);
            up_tma(sm.e[il & 1], &sm.efull[il & 1], &tmap, (int)(item % ntile), item / ntile);
        };
        if (te == 0)
            for (; eissued < 2 && eissued < nmine; ++eissued) item_tma(eissued);
        for (long long il = 0; il < nmine; ++il) {
            const int acc = (int)(il & 1), eb = (int)(il & 1);
            const unsigned par = (unsigned)((il >> 1) & 1);
            bool ok = up_wait<64>(sm, &sm.tfull[acc], par, status);
            ok = ok && up_wait<64>(sm, &sm.efull[eb], par, status);
            if (epi_any(!ok)) break;                  // all epilogue threads leave together
            if (te == 0) elanded = il + 1;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            // the sum of the item's five direction accumulators
            float racc[32];
#pragma unroll
            for (int d = 0; d < UM_DIRS; ++d) {
                uint32_t r[32];
                const uint32_t taddr = tmem + (uint32_t)((acc * UM_DIRS + d) * UM_N) + ((uint32_t)(32 * wq) << 16);
                asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,"
                             "%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                             : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                               "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
                               "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
                               "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
                               "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
                             : "r"(taddr));
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
                for (int i = 0; i < 32; ++i) racc[i] = d == 0 ? __uint_as_float(r[i]) : racc[i] + __uint_as_float(r[i]);
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            up_arrive(&sm.tempty[acc]);               // the accumulators may be overwritten
            const long long item = item_of(il);
            const long long xc = item / ntile;
            const int tile = (int)(item % ntile);
            const int col = tile * UM_M + te;
            // identity and s-hop terms from the item's own inputs (the s-hop partner column of the
            // same right-hand side lies in the same tile: Ls_c divides 128)
            float4 res[8];
            if (col < p.ncols) {
                const int sl = col % p.Ls_c;
                int mh[2];
                float sc[2];
#pragma unroll
                for (int h = 0; h < 2; ++h) {           // components 8 h .. 8 h + 7 share one s-hop
                    const bool from_below = p.dag ? (h == 1) : (h == 0);
                    int sh;
                    sc[h] = 1.f;
                    if (from_below) { if (sl > 0) sh = sl - 1; else { sh = p.Ls_c - 1; sc[h] = -p.mf; } }
                    else            { if (sl < p.Ls_c - 1) sh = sl + 1; else { sh = 0; sc[h] = -p.mf; } }
                    mh[h] = te - sl + sh;
                }
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const int h = q >> 2;
                    const float4 a = *reinterpret_cast<const float4*>(&sm.e[eb][sw_off(te, 4 * q)]);
                    const float4 v = *reinterpret_cast<const float4*>(&sm.e[eb][sw_off(mh[h], 4 * q)]);
                    res[q] = make_float4(racc[2 * q] + a.x + sc[h] * v.x, racc[16 + 2 * q] + a.y + sc[h] * v.y,
                                         racc[2 * q + 1] + a.z + sc[h] * v.z, racc[17 + 2 * q] + a.w + sc[h] * v.w);
                }
            }
            epi_sync();                               // every thread has read e[eb]
            if (te == 0 && il + 2 < nmine) {          // e[eb] takes the inputs of item il + 2
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                item_tma(il + 2);
                eissued = il + 3;
            }
            // results into the padded staging tile (own row), then whole column rows to memory
            if (col < p.ncols) {
#pragma unroll
                for (int q = 0; q < 8; ++q) *reinterpret_cast<float4*>(&sm.o[te * UP_OROW + 4 * q]) = res[q];
            }
            epi_sync();
            {
                const int q = te & 7;
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    const int mm = (te >> 3) + 16 * i;
                    const int c = tile * UM_M + mm;
                    if (c < p.ncols && !(skip_rhs && skip_rhs[c / p.Ls_c])) {
                        float4* o4 = reinterpret_cast<float4*>(out + (long long)c * p.cs + xc * p.ss);
                        o4[q] = *reinterpret_cast<const float4*>(&sm.o[mm * UP_OROW + 4 * q]);
                    }
                }
            }
            epi_sync();                               // the staging tile is read before the next item
        }
        if (te == 0)
            for (long long g = elanded; g < eissued; ++g) up_drain(&sm.efull[g & 1], (unsigned)((g >> 1) & 1));
    } else if (t == 32 * 12) {
        // ---------------- MMA issue ----------------
        // D F32, A and B TF32, both K-major, N = 32, M = 128
        const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(UM_N >> 3) << 17) |
                               ((uint32_t)(UM_M >> 4) << 24);
        bool ok = true;
        for (long long il = 0; ok && il < nmine; ++il) {
            const int acc = (int)(il & 1), bb = (int)(il & 1);
            const long long ua = il >> 1;
            if (ua >= 1 && !up_wait<0>(sm, &sm.tempty[acc], (unsigned)((ua - 1) & 1), status)) break;
            if (!up_wait<0>(sm, &sm.wfull[bb], (unsigned)(ua & 1), status)) break;
            for (int d = 0; d < UM_DIRS; ++d) {
                const uint32_t dt = tmem + (uint32_t)((acc * UM_DIRS + d) * UM_N);
                const long long g = il * UM_DIRS + d;
                const int s = (int)(g % UP_HI), l = (int)(g % UP_LO);
                if (!up_wait<0>(sm, &sm.full[l], (unsigned)((g / UP_LO) & 1), status) ||
                    !up_wait<0>(sm, &sm.tma[s], (unsigned)((g / UP_HI) & 1), status)) { ok = false; break; }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
                for (int ks = 0; ks < UM_K / 8; ++ks) {
                    const uint64_t db = um_desc(reinterpret_cast<const char*>(sm.b[bb][d]) + ks * 2 * UM_LBO);
                    const uint64_t dah = sw_desc(reinterpret_cast<const char*>(sm.hi[s]) + ks * 32);
                    const uint64_t dal = sw_desc(reinterpret_cast<const char*>(sm.lo[l]) + ks * 32);
                    um_mma(dt, dah, db, idesc, ks > 0 ? 1u : 0u);
                    um_mma(dt, dal, db, idesc, 1u);
                }
                um_commit(&sm.ehi[s]);
                um_commit(&sm.elo[l]);
            }
            if (!ok) break;
            um_commit(&sm.tfull[acc]);
            um_commit(&sm.wempty[bb]);
        }
        // every MMA issued by this thread has finished before the TMEM is released
        um_commit(&sm.done);
        up_drain(&sm.done, 0u);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 12)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(UP_TMEM_COLS) : "memory");
}


// ---------------------------------------------------------------------------
// tcgen05 form with the data operand in tensor memory.
//
// Same transposed contraction as above (rows c: 128 columns of a tile; per
// direction K = 32 real values in the (Re v_j, Im v_j) order of memory; the
// weights B[n][k] the real form of the FP16 block with the sigma_3 signs of the
// adjoint folded in).  The shared-memory-fed forms above keep both parts of A
// in shared memory, where the tensor core reads them for each K step and a
// producer pass reads the high part again to write the low part; with N = 32
// the A operand dominates their shared-memory traffic.  Here the tensor core
// reads A from tensor memory: per (item, direction) stage one tensor copy
// (TMA, 128-byte swizzle) lands the tile's 128 column rows in a ring slot of
// the group; each thread of the 4-warp group reads its row (conflict-free
// thanks to the swizzle), splits it into TF32 high and low parts and writes
// both into tensor memory (tcgen05.st); one thread of the group issues the 8
// MMAs (tcgen05.mma kind::tf32, A from tensor memory, B from shared memory).
// The row's own inputs (the last of the five stages) stay in registers for the
// epilogue: identity and s-hops (the s-hop partner column lies in the same
// warp, Ls_c | 32) plus the accumulator read back with tcgen05.ld, stored as
// whole 128-byte rows.
//
// Three groups per CTA, one CTA per SM (persistent; CTA items
// item = blockIdx.x + il gridDim.x, group q takes il = q, q + 3, ...).  Per
// group: a ring of UT_RING input slots (the copy of stage g + 2 is issued when
// stage g starts: its slot was read by every thread of the group before the
// barrier that ended stage g - 1), two tensor-memory A slots (hi 32 + lo 32
// columns; stage g waits for the MMAs of stage g - 2 through the slot's
// `empty` mbarrier) and a 32-column accumulator (`full`: the item's MMAs are
// done; then the epilogue, then the next item's weights).  All waits are
// bounded; a timeout sets the status word and an abort flag, each group leaves
// its loop together (bar.red votes), its copy issuer waits (bounded) for the
// copies in flight and its MMA issuer for its MMAs before the tensor memory is
// freed.
// ---------------------------------------------------------------------------
constexpr int UT_GCOLS = 160;                 // 2 x (hi 32 + lo 32) + accumulator 32
constexpr int UT_TMEM_COLS = 512;
constexpr int UT_YPT = UM_DIRS * 256 / 128;   // FP16 block entries per thread per item

// NG groups of 128 threads; RING input slots per group (copies RING - 1 stages ahead).  Measured
// at 64^2 x 4 coarse sites and 64 right-hand sides: 3 groups x 3 slots 194 us, 2 groups x 5 slots
// 244 us (the number of groups working at once counts, not how far the copies run ahead)
constexpr int UT_NG = 3, UT_NR = 3;
template <int NG, int RING>
struct UtSmem {
    float in[NG][RING][UM_M * UM_K];            // swizzled input rows (1024-byte aligned slots)
    float w[NG][UM_DIRS][UM_N * UM_K];          // weights of the group's current item
    unsigned long long tma[NG][RING], empty[NG][2], full[NG], done[NG];
    uint32_t tmem;
    int abort;
};

__device__ __forceinline__ bool ut_wait(int* abort_flag, unsigned long long* bar, unsigned parity, int* status) {
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = now_ns();
    for (unsigned it = 1;; ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((it & 15) == 0) {
            if (*(volatile int*)abort_flag) return false;
            if (now_ns() - t0 > UM_WAIT_NS) {
                *(volatile int*)abort_flag = 1;
                atomicExch(status, 3);
                return false;
            }
        }
    }
}
// named barrier 1 + q over the 128 threads of group q; ut_all: the AND of v over them
__device__ __forceinline__ void ut_sync(int q) { asm volatile("bar.sync %0, 128;" ::"r"(1 + q) : "memory"); }
__device__ __forceinline__ bool ut_all(int q, bool v) {
    uint32_t r;
    asm volatile("{\n\t.reg .pred p, r;\n\tsetp.ne.u32 p, %1, 0;\n\tbar.red.and.pred r, %2, 128, p;\n\t"
                 "selp.u32 %0, 1, 0, r;\n\t}"
                 : "=r"(r) : "r"((uint32_t)v), "r"(1 + q) : "memory");
    return r != 0;
}
__device__ __forceinline__ void um_mma_ta(uint32_t dt, uint32_t at, uint64_t db, uint32_t idesc, uint32_t acc) {
    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                 "tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n\t}"
                 ::"r"(dt), "r"(at), "l"(db), "r"(idesc), "r"(acc) : "memory");
}
__device__ __forceinline__ void tm_st8(uint32_t taddr, const uint32_t (&r)[8]) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};"
                 ::"r"(taddr), "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7])
                 : "memory");
}
__device__ __forceinline__ void tm_ld8(uint32_t taddr, uint32_t (&r)[8]) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr));
}

// direction of stage d: the four hops first, the site itself last (its inputs stay in registers
// for the epilogue)
__device__ __forceinline__ int ut_dir(int d) { return d < 4 ? d + 1 : 0; }

template <int UT_GROUPS, int UT_RING>
__global__ void __maxnreg__(128) k_coarse_umma_t(const __half2* __restrict__ Y,
                                                                     float2* __restrict__ out, TcParams p,
                                                                     const int* __restrict__ skip_rhs, int* status,
                                                                     const __grid_constant__ CUtensorMap tmap) {
    extern __shared__ __align__(1024) unsigned char ut_raw[];
    UtSmem<UT_GROUPS, UT_RING>& sm = *reinterpret_cast<UtSmem<UT_GROUPS, UT_RING>*>(ut_raw);
    const int t = threadIdx.x, warp = t >> 5, q = warp >> 2, tr = t & 127;
    if (t == 0) {
        for (int g = 0; g < UT_GROUPS; ++g) {
            for (int r = 0; r < UT_RING; ++r) mbar_init(&sm.tma[g][r], 1);
            mbar_init(&sm.empty[g][0], 1);
            mbar_init(&sm.empty[g][1], 1);
            mbar_init(&sm.full[g], 1);
            mbar_init(&sm.done[g], 1);
        }
        // the swizzled copies need 1024-byte aligned slots
        sm.abort = (smem_u32(sm.in) & 1023u) != 0;
        if (sm.abort) atomicExch(status, 3);
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&sm.tmem)),
                     "r"(UT_TMEM_COLS) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tq = sm.tmem + (uint32_t)(q * UT_GCOLS);              // group's columns, lane 0
    const uint32_t tl = tq + ((uint32_t)(32 * (warp & 3)) << 16);        // this warp's lanes
    const int ntile = (p.ncols + UM_M - 1) / UM_M;
    const int nitems = (int)(p.Vc * ntile);
    const int ncta = (blockIdx.x < nitems && !sm.abort) ? (nitems - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
    const int nli = ncta > q ? (ncta - 1 - q) / UT_GROUPS + 1 : 0;      // this group's items
    const long long G = (long long)nli * UM_DIRS;                        // and stages
    auto item_of = [&](int li) { return (int)blockIdx.x + (q + UT_GROUPS * li) * (int)gridDim.x; };
    // D F32, A and B TF32, K-major, N = 32, M = 128
    const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(UM_N >> 3) << 17) |
                           ((uint32_t)(UM_M >> 4) << 24);
    long long issued = 0, landed = 0;          // copies issued by thread tr == 0 and waited for

    auto copy_stage = [&](long long g) {       // thread tr == 0
        const int item = item_of((int)(g / UM_DIRS));
        const int d = (int)(g % UM_DIRS), r = (int)(g % UT_RING);
        up_tma(sm.in[q][r], &sm.tma[q][r], &tmap, item % ntile, nbr2d(p, item / ntile, ut_dir(d)));
        issued = g + 1;
    };
    __half2 yv[UT_YPT];
    auto load_y = [&](int li) {
        const long long xc = item_of(li) / ntile;
#pragma unroll
        for (int k = 0; k < UT_YPT; ++k) {
            const int e = tr + 128 * k, d = e >> 8;
            yv[k] = __ldg(Y + (xc * UM_DIRS + ut_dir(d)) * 256 + (e & 255));
        }
    };

    auto stage = [&](long long g) -> bool {
        if (tr == 0 && g + UT_RING - 1 < G) copy_stage(g + UT_RING - 1);
        const int li = (int)(g / UM_DIRS), d = (int)(g % UM_DIRS), s = (int)(g & 1), r = (int)(g % UT_RING);
        bool ok = ut_wait(&sm.abort, &sm.tma[q][r], (unsigned)((g / UT_RING) & 1), status);
        if (g >= 2)                                          // the MMAs of stage g - 2 have read A slot s
            ok = ok && ut_wait(&sm.abort, &sm.empty[q][s], (unsigned)(((g - 2) >> 1) & 1), status);
        if (!ut_all(q, ok)) return false;
        if (tr == 0) landed = g + 1;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        float4 cur[8];                                       // this row's 32 K values
        {
            const float* row = sm.in[q][r];
#pragma unroll
            for (int c = 0; c < 8; ++c) cur[c] = *reinterpret_cast<const float4*>(&row[sw_off(tr, 4 * c)]);
        }
        if (d == 0) {
            // weights of item li (the MMAs of item li - 1, which read them, are done: its epilogue
            // waited for them): B[n][k], k = 2 j (Re v_j), 2 j + 1 (Im v_j); n < 16: Re out_n,
            // n = 16 + i: Im out_i; sigma_3 Y sigma_3 for the adjoint
#pragma unroll
            for (int k = 0; k < UT_YPT; ++k) {
                const int e = tr + 128 * k, dd = e >> 8, j = (e >> 4) & 15, i = e & 15;
                float2 y = __half22float2(yv[k]);
                if (p.dag && ((i >= 8) != (j >= 8))) { y.x = -y.x; y.y = -y.y; }
                float* bd = sm.w[q][dd];
                bd[um_off(i, 2 * j)] = y.x;
                bd[um_off(i, 2 * j + 1)] = -y.y;
                bd[um_off(16 + i, 2 * j)] = y.y;
                bd[um_off(16 + i, 2 * j + 1)] = y.x;
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            if (li + 1 < nli) load_y(li + 1);
        }
#pragma unroll
        for (int c = 0; c < 4; ++c) {                       // K values 8 c .. 8 c + 7
            uint32_t hi[8], lo[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const float4 v4 = cur[2 * c + (u >> 2)];
                const float x = (u & 3) == 0 ? v4.x : (u & 3) == 1 ? v4.y : (u & 3) == 2 ? v4.z : v4.w;
                hi[u] = __float_as_uint(x) & 0xffffe000u;
                lo[u] = __float_as_uint(x - __uint_as_float(hi[u]));
            }
            tm_st8(tl + (uint32_t)(64 * s + 8 * c), hi);
            tm_st8(tl + (uint32_t)(64 * s + 32 + 8 * c), lo);
        }
        asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        ut_sync(q);                                          // also: every thread has read input slot r
        if (tr == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
            for (int ks = 0; ks < UM_K / 8; ++ks) {
                const uint64_t db = um_desc(reinterpret_cast<const char*>(sm.w[q][d]) + ks * 2 * UM_LBO);
                const uint32_t ah = tq + (uint32_t)(64 * s + 8 * ks), al = ah + 32u;
                um_mma_ta(tq + 128u, ah, db, idesc, (d > 0 || ks > 0) ? 1u : 0u);
                um_mma_ta(tq + 128u, al, db, idesc, 1u);
            }
            um_commit(&sm.empty[q][s]);
            if (d == UM_DIRS - 1) um_commit(&sm.full[q]);
        }
        if (d == UM_DIRS - 1) {
            // epilogue of item li: cur holds the site's own inputs
            ok = ut_wait(&sm.abort, &sm.full[q], (unsigned)(li & 1), status);
            if (!ut_all(q, ok)) return false;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const int item = item_of(li);
            const long long xc = item / ntile;
            const int col = (item % ntile) * UM_M + tr;
            const int sl = col % p.Ls_c, lane = tr & 31;
            int pl[2];
            float sc[2];
#pragma unroll
            for (int h = 0; h < 2; ++h) {                // components 8 h .. 8 h + 7 share one s-hop
                const bool from_below = p.dag ? (h == 1) : (h == 0);
                int sh;
                sc[h] = 1.f;
                if (from_below) { if (sl > 0) sh = sl - 1; else { sh = p.Ls_c - 1; sc[h] = -p.mf; } }
                else            { if (sl < p.Ls_c - 1) sh = sl + 1; else { sh = 0; sc[h] = -p.mf; } }
                pl[h] = lane - sl + sh;
            }
            bool live = col < p.ncols;
            if (live && skip_rhs) live = skip_rhs[col / p.Ls_c] == 0;
            float4* o4 = reinterpret_cast<float4*>(out + (long long)(live ? col : 0) * p.cs + xc * p.ss);
#pragma unroll
            for (int h = 0; h < 2; ++h) {                // output components 8 h .. 8 h + 7
                uint32_t re[8], im[8];
                tm_ld8(tl + 128u + (uint32_t)(8 * h), re);
                tm_ld8(tl + 128u + (uint32_t)(16 + 8 * h), im);
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
                for (int kk = 0; kk < 4; ++kk) {
                    const int k = 4 * h + kk;
                    const float4 a = cur[k];
                    float4 v;
                    v.x = __shfl_sync(0xffffffffu, a.x, pl[h]);
                    v.y = __shfl_sync(0xffffffffu, a.y, pl[h]);
                    v.z = __shfl_sync(0xffffffffu, a.z, pl[h]);
                    v.w = __shfl_sync(0xffffffffu, a.w, pl[h]);
                    const float4 res = make_float4(__uint_as_float(re[2 * kk]) + a.x + sc[h] * v.x,
                                                   __uint_as_float(im[2 * kk]) + a.y + sc[h] * v.y,
                                                   __uint_as_float(re[2 * kk + 1]) + a.z + sc[h] * v.z,
                                                   __uint_as_float(im[2 * kk + 1]) + a.w + sc[h] * v.w);
                    if (live) o4[k] = res;
                }
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        }
        return true;
    };

    if (tr == 0)
        for (long long g = 0; g < UT_RING - 1 && g < G; ++g) copy_stage(g);
    if (G > 0) load_y(0);
    for (long long g = 0; g < G; ++g)
        if (!stage(g)) break;
    if (tr == 0) {
        // copies still in flight after an early exit land before the CTA ends
        for (long long g = landed; g < issued; ++g) up_drain(&sm.tma[q][g % UT_RING], (unsigned)((g / UT_RING) & 1));
        // every MMA this group issued has finished before the tensor memory is released
        if (G > 0) {
            um_commit(&sm.done[q]);
            up_drain(&sm.done[q], 0u);
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(sm.tmem), "r"(UT_TMEM_COLS) : "memory");
}

}  // namespace

// forms of the contraction: 1, 2, 4 = mma.sync with that many column tiles per warp; TC_UMMA = tcgen05,
// one item per CTA; TC_UMMA_P = tcgen05, persistent and warp-specialised
constexpr int TC_UMMA = 0x100;
constexpr int TC_UMMA_P = 0x101;
constexpr int TC_UMMA_T = 0x102;

static bool umma_eligible(const dwf_mg* h, int ncols) { return h->ytile_half && ncols >= UM_M; }
// the persistent form's epilogue finds each column's s-hop partner in the same 128-column tile
// (Ls_c divides 128)
static bool umma_p_eligible(const dwf_mg* h, int ncols) { return umma_eligible(h, ncols) && UM_M % h->mg.Ls_c == 0; }
// the tensor-memory-operand form's epilogue takes the s-hop partner column from a lane of the same
// warp (Ls_c divides 32); partial tiles are fine (their rows are independent), so it starts at 64
// columns
static bool umma_t_eligible(const dwf_mg* h, int ncols) {
    return h->ytile_half && ncols >= UM_M / 2 && 32 % h->mg.Ls_c == 0;
}

// cuTensorMapEncodeTiled from the driver, looked up once
static PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = []() -> PFN_cuTensorMapEncodeTiled_v12000 {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            return nullptr;
        return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
    }();
    return fn;
}

// the 5-d view of the input vectors read by the persistent form (see up_tma)
static dwf_status input_tensor_map(CUtensorMap* tm, const float2* in, const TcParams& p) {
    auto enc = tensor_map_encoder();
    if (!enc) { set_error("cuTensorMapEncodeTiled is not available from the driver"); return DWF_ERR_CUDA; }
    if ((reinterpret_cast<uintptr_t>(in) & 15u) != 0) { set_error("coarse vectors must be 16-byte aligned"); return DWF_ERR_ARG; }
    const cuuint64_t dims[3] = {32, (cuuint64_t)p.ncols, (cuuint64_t)p.Vc};
    const cuuint64_t strides[2] = {(cuuint64_t)p.cs * sizeof(float2), (cuuint64_t)p.ss * sizeof(float2)};
    const cuuint32_t box[3] = {32, (cuuint32_t)UM_M, 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    const CUresult r = enc(tm, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float2*>(in), dims, strides, box, estr,
                           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) { set_error("cuTensorMapEncodeTiled failed (%d)", (int)r); return DWF_ERR_CUDA; }
    return DWF_OK;
}

// Once per device (the current one): the dynamic shared-memory limit of the three tcgen05 forms,
// and the device's SM count (the persistent forms launch one CTA per SM).  Guarded by a mutex:
// mg_solve_groups runs hierarchies from several host threads.
static dwf_status tc_device_init(int* sms_out) {
    static std::mutex mu;
    static int sms_of[64] = {0};                 // 0: this device is not set up yet
    int dev = 0;
    DWF_CHECK_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) { set_error("device ordinal %d out of range", dev); return DWF_ERR_UNSUPPORTED; }
    std::lock_guard<std::mutex> lock(mu);
    if (sms_of[dev] == 0) {
        DWF_CHECK_CUDA(cudaFuncSetAttribute(k_coarse_umma, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            (int)sizeof(UmSmem)));
        DWF_CHECK_CUDA(cudaFuncSetAttribute(k_coarse_umma_p, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            (int)sizeof(UpSmem)));
        DWF_CHECK_CUDA(cudaFuncSetAttribute(k_coarse_umma_t<UT_NG, UT_NR>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            (int)sizeof(UtSmem<UT_NG, UT_NR>)));
        int sms = 0;
        DWF_CHECK_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        if (sms <= 0) { set_error("no multiprocessors reported"); return DWF_ERR_CUDA; }
        sms_of[dev] = sms;
    }
    *sms_out = sms_of[dev];
    return DWF_OK;
}

static dwf_status launch_form(const dwf_mg* h, int form, const TcParams& p, const float2* in, float2* out,
                              const int* skip_rhs, cudaStream_t st) {
    if (form == TC_UMMA_T) {
        int sms = 0;
        DWF_TRY(tc_device_init(&sms));
        const long long nitems = p.Vc * ((p.ncols + UM_M - 1) / UM_M);
        if (nitems > 0x7fffffffLL) { set_error("coarse batch too large for one launch"); return DWF_ERR_ARG; }
        const long long grid = nitems < sms ? nitems : sms;
        if (grid < 1) return DWF_OK;
        alignas(64) CUtensorMap tm;
        DWF_TRY(input_tensor_map(&tm, in, p));
        k_coarse_umma_t<UT_NG, UT_NR><<<(unsigned)grid, 128 * UT_NG, sizeof(UtSmem<UT_NG, UT_NR>), st>>>(
            (const __half2*)h->Ytile, out, p, skip_rhs, h->status + 1, tm);
        DWF_CHECK_LAUNCH();
        return DWF_OK;
    }
    if (form == TC_UMMA_P) {
        int sms = 0;
        DWF_TRY(tc_device_init(&sms));
        const long long nitems = p.Vc * ((p.ncols + UM_M - 1) / UM_M);
        const long long grid = nitems < sms ? nitems : sms;
        if (grid < 1) return DWF_OK;
        alignas(64) CUtensorMap tm;
        DWF_TRY(input_tensor_map(&tm, in, p));
        k_coarse_umma_p<<<(unsigned)grid, UP_THREADS, sizeof(UpSmem), st>>>((const __half2*)h->Ytile, in, out, p,
                                                                           skip_rhs, h->status + 1, tm);
        DWF_CHECK_LAUNCH();
        return DWF_OK;
    }
    if (form == TC_UMMA) {
        int sms = 0;
        DWF_TRY(tc_device_init(&sms));
        const long long ctas = p.Vc * ((p.ncols + UM_M - 1) / UM_M);
        if (ctas > 0x7fffffffLL) { set_error("coarse batch too large for one launch"); return DWF_ERR_ARG; }
        k_coarse_umma<<<(unsigned)ctas, UM_THREADS, sizeof(UmSmem), st>>>((const __half2*)h->Ytile, in, out, p,
                                                                          skip_rhs, h->status + 1);
        DWF_CHECK_LAUNCH();
        return DWF_OK;
    }
    const int NT = form;
    const long long warps = p.Vc * ((p.ncols + 8 * NT - 1) / (8 * NT));
    const long long blocks = (warps * 32 + 255) / 256;
    if (blocks > 0x7fffffffLL) { set_error("coarse batch too large for one launch"); return DWF_ERR_ARG; }
#define DWF_TC_LAUNCH(N)                                                                                              \
    if (h->ytile_half)                                                                                                 \
        k_coarse_tc<N, __half2><<<(unsigned)blocks, 256, 0, st>>>((const __half2*)h->Ytile, in, out, p, skip_rhs);   \
    else                                                                                                               \
        k_coarse_tc<N, float2><<<(unsigned)blocks, 256, 0, st>>>(h->Y32, in, out, p, skip_rhs);
    if (NT == 1) { DWF_TC_LAUNCH(1) }
    else if (NT == 2) { DWF_TC_LAUNCH(2) }
    else { DWF_TC_LAUNCH(4) }
#undef DWF_TC_LAUNCH
    DWF_CHECK_LAUNCH();
    return DWF_OK;
}

static TcParams tc_params(const dwf_mg* h, int nrhs, double mf, bool dagger, int layout) {
    TcParams p;
    p.Vc = h->mg.Vc;
    p.Lc0 = h->mg.Lc[0];
    p.Lc1 = h->mg.Lc[1];
    p.Ls_c = h->mg.Ls_c;
    p.nrhs = nrhs;
    p.ncols = nrhs * h->mg.Ls_c;
    p.mf = (float)mf;
    p.dag = dagger ? 1 : 0;
    if (layout == DWF_COARSE_SITE_MAJOR) { p.cs = 16; p.ss = (long long)p.ncols * 16; }
    else { p.cs = p.Vc * 16; p.ss = 16; }
    return p;
}

// autotuner key: nrhs for the slice-major layout, -nrhs for the site-major one
static int tc_key(int nrhs, int layout) { return layout == DWF_COARSE_SITE_MAJOR ? -nrhs : nrhs; }

dwf_status coarse_tc_tune(const dwf_mg* h, int nrhs, const float2* in, float2* out, cudaStream_t st, int layout) {
    if (h->mg.nd != 2 || h->mg.ncd != 16 || nrhs < 1) return DWF_OK;
    if (h->tc_choice.count(tc_key(nrhs, layout))) return DWF_OK;
    const TcParams p = tc_params(h, nrhs, h->mf, false, layout);
    int forms[6] = {1, 2, 4, 0, 0, 0};
    int nforms = 3;
    if (umma_eligible(h, p.ncols)) forms[nforms++] = TC_UMMA;
    if (umma_p_eligible(h, p.ncols)) forms[nforms++] = TC_UMMA_P;
    if (umma_t_eligible(h, p.ncols)) forms[nforms++] = TC_UMMA_T;
    cudaEvent_t a, b;
    DWF_CHECK_CUDA(cudaEventCreate(&a));
    DWF_CHECK_CUDA(cudaEventCreate(&b));
    int best = 4;
    float best_ms = 1e30f;
    dwf_status status = DWF_OK;
    for (int f = 0; f < nforms && status == DWF_OK; ++f) {
        for (int w = 0; w < 2 && status == DWF_OK; ++w) status = launch_form(h, forms[f], p, in, out, nullptr, st);
        if (status != DWF_OK) break;
        cudaEventRecord(a, st);
        for (int r = 0; r < 5 && status == DWF_OK; ++r) status = launch_form(h, forms[f], p, in, out, nullptr, st);
        cudaEventRecord(b, st);
        if (cudaEventSynchronize(b) != cudaSuccess) { set_error("autotuner timing failed"); status = DWF_ERR_CUDA; break; }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, a, b);
        if (ms < best_ms) { best_ms = ms; best = forms[f]; }
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (status == DWF_OK) h->tc_choice[tc_key(nrhs, layout)] = best;
    return status;
}

dwf_status coarse_apply_multi_tc(const dwf_mg* h, int nrhs, const float2* in, float2* out, double mf, bool dagger,
                                 const int* skip_rhs, cudaStream_t st, int layout) {
    if (h->mg.nd != 2 || h->mg.ncd != 16) {
        set_error("the tensor-core coarse stencil supports 2-d lattices with 16 coarse dof");
        return DWF_ERR_UNSUPPORTED;
    }
    const TcParams p = tc_params(h, nrhs, mf, dagger, layout);
    int form = 4;
    if (h->prm.coarse_tc == 6 && umma_t_eligible(h, p.ncols)) form = TC_UMMA_T;
    else if (h->prm.coarse_tc == 1 && umma_p_eligible(h, p.ncols)) form = TC_UMMA_P;
    else if (h->prm.coarse_tc == 1 && umma_eligible(h, p.ncols)) form = TC_UMMA;
    else if (h->prm.coarse_tc == 5 && umma_eligible(h, p.ncols)) form = TC_UMMA;
    else if (h->prm.coarse_tc >= 2 && h->prm.coarse_tc <= 4) form = h->prm.coarse_tc == 2 ? 1 : h->prm.coarse_tc == 3 ? 2 : 4;
    else if (h->prm.coarse_tc == 0) {
        auto it = h->tc_choice.find(tc_key(nrhs, layout));
        if (it != h->tc_choice.end()) form = it->second;
    }
    return launch_form(h, form, p, in, out, skip_rhs, st);
}

}  // namespace dwf

using namespace dwf;

extern "C" dwf_status mg_coarse_apply_multi_layout(const dwf_mg* h, int nrhs, const void* in, void* out, double mf,
                                                   int dagger, int layout, void* stream) {
    clear_error();
    if (!h || !in || !out) { set_error("NULL argument"); return DWF_ERR_ARG; }
    if (nrhs < 1) { set_error("nrhs must be >= 1"); return DWF_ERR_ARG; }
    if (in == out) { set_error("in and out must be distinct buffers"); return DWF_ERR_ARG; }
    if (layout != DWF_COARSE_SLICE_MAJOR && layout != DWF_COARSE_SITE_MAJOR) {
        set_error("unknown coarse vector layout %d", layout);
        return DWF_ERR_ARG;
    }
    if (!aligned16(in) || !aligned16(out)) { set_error("coarse vectors must be 16-byte aligned"); return DWF_ERR_ARG; }
    cudaStream_t st = as_stream(stream);
    // the first call for a new (nrhs, layout) picks the fastest form of the contraction (using in / out
    // as scratch)
    if (h->prm.coarse_tc == 0) DWF_TRY(coarse_tc_tune(h, nrhs, (const float2*)in, (float2*)out, st, layout));
    return coarse_apply_multi_tc(h, nrhs, (const float2*)in, (float2*)out, mf, dagger != 0, nullptr, st, layout);
}

extern "C" dwf_status mg_coarse_apply_multi(const dwf_mg* h, int nrhs, const void* in, void* out, double mf, int dagger,
                                            void* stream) {
    return mg_coarse_apply_multi_layout(h, nrhs, in, out, mf, dagger, DWF_COARSE_SLICE_MAJOR, stream);
}

extern "C" int mg_coarse_tc_form_layout(const dwf_mg* h, int nrhs, int layout) {
    if (!h) return 0;
    auto it = h->tc_choice.find(tc_key(nrhs, layout));
    return it == h->tc_choice.end() ? 0 : it->second;
}

extern "C" int mg_coarse_tc_form(const dwf_mg* h, int nrhs) {
    return mg_coarse_tc_form_layout(h, nrhs, DWF_COARSE_SLICE_MAJOR);
}
