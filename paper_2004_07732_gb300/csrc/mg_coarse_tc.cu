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
// Vectors: [rhs][s][coarse site][16] complex64; blocks: the FP32 column-major
// Galerkin blocks.
#include "mg.cuh"

namespace dwf {
namespace {

struct TcParams {
    long long Vc;
    int Lc0, Lc1;
    int Ls_c, nrhs, ncols;
    float mf;
    int dag;
};

__device__ __forceinline__ uint32_t to_tf32(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ void split_tf32(float x, uint32_t& hi, uint32_t& lo) {
    hi = to_tf32(x);
    lo = to_tf32(x - __uint_as_float(hi));
}

__device__ __forceinline__ void mma_tf32(float (&c)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
    asm volatile("mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
                 "{%0,%1,%2,%3};"
                 : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
                 : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

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
    const long long slice = p.Vc * 16;                   // one slice of one right-hand side
    const long long rhs_stride = slice * p.Ls_c;
    long long baseB[NT];
    bool okB[NT];
#pragma unroll
    for (int k = 0; k < NT; ++k) {
        const int col = (cg * NT + k) * 8 + g;           // B column owned by this lane in tile k
        okB[k] = col < p.ncols && !(skip_rhs && skip_rhs[col / p.Ls_c]);
        baseB[k] = okB[k] ? (long long)(col / p.Ls_c) * rhs_stride + (long long)(col % p.Ls_c) * slice : 0;
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
                    const float2* src = in + baseB[k] + nb * 16 + 8 * half + t;
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
                const long long rb = (long long)r * rhs_stride;
                const float hr = so * acc[k][0][2 * h + w], hi = so * acc[k][1][2 * h + w];
                const float2 self = __ldg(in + rb + (long long)s * slice + xc * 16 + i);
                int sh;
                float sc = 1.f;
                if (from_below) { if (s > 0) sh = s - 1; else { sh = p.Ls_c - 1; sc = -p.mf; } }
                else            { if (s < p.Ls_c - 1) sh = s + 1; else { sh = 0; sc = -p.mf; } }
                const float2 hv = __ldg(in + rb + (long long)sh * slice + xc * 16 + i);
                out[rb + (long long)s * slice + xc * 16 + i] =
                    make_float2(hr + self.x + sc * hv.x, hi + self.y + sc * hv.y);
            }
        }
}

}  // namespace

dwf_status coarse_apply_multi_tc(const dwf_mg* h, int nrhs, const float2* in, float2* out, double mf, bool dagger,
                                 const int* skip_rhs, cudaStream_t st) {
    if (h->mg.nd != 2 || h->mg.ncd != 16) {
        set_error("the tensor-core coarse stencil supports 2-d lattices with 16 coarse dof");
        return DWF_ERR_UNSUPPORTED;
    }
    TcParams p;
    p.Vc = h->mg.Vc;
    p.Lc0 = h->mg.Lc[0];
    p.Lc1 = h->mg.Lc[1];
    p.Ls_c = h->mg.Ls_c;
    p.nrhs = nrhs;
    p.ncols = nrhs * h->mg.Ls_c;
    p.mf = (float)mf;
    p.dag = dagger ? 1 : 0;
    constexpr int NT = 4;
    const long long warps = p.Vc * ((p.ncols + 8 * NT - 1) / (8 * NT));
    const long long blocks = (warps * 32 + 255) / 256;
    if (blocks > 0x7fffffffLL) { set_error("coarse batch too large for one launch"); return DWF_ERR_ARG; }
    if (h->ytile_half)
        k_coarse_tc<NT, __half2><<<(unsigned)blocks, 256, 0, st>>>((const __half2*)h->Ytile, in, out, p, skip_rhs);
    else
        k_coarse_tc<NT, float2><<<(unsigned)blocks, 256, 0, st>>>(h->Y32, in, out, p, skip_rhs);
    DWF_CHECK_LAUNCH();
    return DWF_OK;
}

}  // namespace dwf

using namespace dwf;

extern "C" dwf_status mg_coarse_apply_multi(const dwf_mg* h, int nrhs, const void* in, void* out, double mf, int dagger,
                                            void* stream) {
    clear_error();
    if (!h || !in || !out) { set_error("NULL argument"); return DWF_ERR_ARG; }
    if (nrhs < 1) { set_error("nrhs must be >= 1"); return DWF_ERR_ARG; }
    if (in == out) { set_error("in and out must be distinct buffers"); return DWF_ERR_ARG; }
    return coarse_apply_multi_tc(h, nrhs, (const float2*)in, (float2*)out, mf, dagger != 0, nullptr, as_stream(stream));
}
