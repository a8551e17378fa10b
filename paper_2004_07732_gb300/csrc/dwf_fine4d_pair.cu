// 4-d SU(3) Shamir operator (Eq. DWoperator) on the slice-paired packed layout.
//
// The operator is applied on every s slice with the same links, so two slices
// can share one instruction stream: the layout interleaves slices 2j and 2j+1
// at the level of single real numbers, and every real operation of the Wilson
// hop becomes one packed FP32 operation (fadd2 / ffma2) over the pair.  The
// colour multiply of a hop (18 complex multiply-adds) thus costs 36 packed FMAs
// for two slices instead of 144 scalar ones; the link is loaded and converted
// once per pair.
//
// Layout (FP32 spinors; Ls even): sites in blocks of 32 (NB = ceil(V / 32)), slice
// pairs j = 0 .. Ls/2 - 1.  For pair j, block b, complex element k (spin-major,
// colour fastest, 12 per site) a plane of 32 float4 holds, for site 32 b + i,
//   (Re psi_{2j}[k], Im psi_{2j}[k], Re psi_{2j+1}[k], Im psi_{2j+1}[k])
// at float4 index ((j NB + b) 12 + k) 32 + i.  A warp reads each element of 32
// sites' spinors as one contiguous 512-byte run.  Each complex value stays a
// (re, im) pair in memory, so complex BLAS runs on packed vectors unchanged (the
// layout only permutes complex elements); the kernel regroups a loaded float4 into
// the (slice 2j, slice 2j+1) pairs of its real and imaginary parts.  Links: nine planes of 32
// entries per (mu, block), entry 3 a + b of U_mu(32 b + i) at ((mu NB + b) 9 + e) 32 + i.
// Padding sites (V not a multiple of 32) are zero and are not written by the apply.
#include <algorithm>

#include "common.cuh"
#include "fine_kernels.cuh"

namespace dwf {
namespace {


// a complex value on two slices: re = (Re_s0, Re_s1), im = (Im_s0, Im_s1)
struct CP {
    float2 re, im;
};

__device__ __forceinline__ float2 f2s(float s) { return make_float2(s, s); }
// acc + s a for a real scalar s on both slices (two packed FMAs)
__device__ __forceinline__ CP cp_fma_s(float s, CP a, CP acc) {
    const float2 ss = f2s(s);
    return CP{__ffma2_rn(ss, a.re, acc.re), __ffma2_rn(ss, a.im, acc.im)};
}

struct LayP2 {
    long long NB;
    int NP;
    __device__ __forceinline__ long long idx(int j, int site, int k) const {
        return (((long long)j * NB + (site >> 5)) * 12 + k) * 32 + (site & 31);
    }
    __device__ __forceinline__ long long lk(int mu, int site) const {
        return ((long long)mu * NB + (site >> 5)) * 288 + (site & 31);
    }
};

__device__ __forceinline__ CP ld_cp(const float4* p, long long i) {
    const float4 a = __ldg(p + i);
    return CP{make_float2(a.x, a.z), make_float2(a.y, a.w)};
}

// one link entry, as FP32 (re, im)
__device__ __forceinline__ float2 lk_val(const float2* U, long long i) { return __ldg(U + i); }
__device__ __forceinline__ float2 lk_val(const __half2* U, long long i) { return __half22float2(__ldg(U + i)); }
__device__ __forceinline__ float2 lk_val(const __nv_bfloat162* U, long long i) {
    return __bfloat1622float2(__ldg(U + i));
}

// h = v + sg (A l) on the upper spin pair, A = -i sigma_1, -i sigma_2, -i sigma_3, 1 for mu = 0..3
// (l: the lower spin pair); every real operation is one packed FMA with a constant +-sg pair.
// With -i z = (Im z, -Re z) and i z = (-Im z, Re z):
//   mu 0: (A l)_0 = -i l_1, (A l)_1 = -i l_0;  mu 1: -l_1, l_0;  mu 2: -i l_0, i l_1;  mu 3: l_0, l_1
__device__ __forceinline__ void pair_project(int mu, float sg, const CP (&v)[4][3], CP (&h)[2][3]) {
    const float2 P = f2s(sg), M = f2s(-sg);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const CP l0 = v[2][c], l1 = v[3][c], v0 = v[0][c], v1 = v[1][c];
        if (mu == 0) {
            h[0][c] = CP{__ffma2_rn(P, l1.im, v0.re), __ffma2_rn(M, l1.re, v0.im)};
            h[1][c] = CP{__ffma2_rn(P, l0.im, v1.re), __ffma2_rn(M, l0.re, v1.im)};
        } else if (mu == 1) {
            h[0][c] = CP{__ffma2_rn(M, l1.re, v0.re), __ffma2_rn(M, l1.im, v0.im)};
            h[1][c] = CP{__ffma2_rn(P, l0.re, v1.re), __ffma2_rn(P, l0.im, v1.im)};
        } else if (mu == 2) {
            h[0][c] = CP{__ffma2_rn(P, l0.im, v0.re), __ffma2_rn(M, l0.re, v0.im)};
            h[1][c] = CP{__ffma2_rn(M, l1.im, v1.re), __ffma2_rn(P, l1.re, v1.im)};
        } else {
            h[0][c] = CP{__ffma2_rn(P, l0.re, v0.re), __ffma2_rn(P, l0.im, v0.im)};
            h[1][c] = CP{__ffma2_rn(P, l1.re, v1.re), __ffma2_rn(P, l1.im, v1.im)};
        }
    }
}

// lo += t (A^dag u) for the lower spin pair:
//   mu 0: (A^dag u)_0 = i u_1, (A^dag u)_1 = i u_0;  mu 1: u_1, -u_0;  mu 2: i u_0, -i u_1;  mu 3: u_0, u_1
__device__ __forceinline__ void pair_lower(int mu, float t, const CP (&u)[2][3], CP (&lo)[2][3]) {
    const float2 P = f2s(t), M = f2s(-t);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const CP u0 = u[0][c], u1 = u[1][c];
        CP& a0 = lo[0][c];
        CP& a1 = lo[1][c];
        if (mu == 0) {
            a0 = CP{__ffma2_rn(M, u1.im, a0.re), __ffma2_rn(P, u1.re, a0.im)};
            a1 = CP{__ffma2_rn(M, u0.im, a1.re), __ffma2_rn(P, u0.re, a1.im)};
        } else if (mu == 1) {
            a0 = CP{__ffma2_rn(P, u1.re, a0.re), __ffma2_rn(P, u1.im, a0.im)};
            a1 = CP{__ffma2_rn(M, u0.re, a1.re), __ffma2_rn(M, u0.im, a1.im)};
        } else if (mu == 2) {
            a0 = CP{__ffma2_rn(M, u0.im, a0.re), __ffma2_rn(P, u0.re, a0.im)};
            a1 = CP{__ffma2_rn(P, u1.im, a1.re), __ffma2_rn(M, u1.re, a1.im)};
        } else {
            a0 = CP{__ffma2_rn(P, u0.re, a0.re), __ffma2_rn(P, u0.im, a0.im)};
            a1 = CP{__ffma2_rn(P, u1.re, a1.re), __ffma2_rn(P, u1.im, a1.im)};
        }
    }
}

// One hop direction: accumulate the Wilson hop from the neighbour spinor v (both slices of the
// pair) into the upper / lower spin-pair accumulators.  Forward hops multiply by U_mu(x), backward
// ones by U_mu(x - mu)^dag; l0 indexes the link's first plane, ph is the boundary phase.
template <class LT, bool DAG>
__device__ __forceinline__ void pair_hop(int mu, bool fwd, float ph, const CP (&v)[4][3],
                                         const typename LT::store* __restrict__ U, long long l0, CP (&up)[2][3],
                                         CP (&lo)[2][3]) {
    const bool minus = (fwd != DAG);
    CP h[2][3];
    pair_project(mu, minus ? -1.f : 1.f, v, h);
    CP uh[2][3];
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int c = 0; c < 3; ++c) uh[a][c] = CP{make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            const float2 u = lk_val(U, l0 + (long long)(fwd ? (c * 3 + b) : (b * 3 + c)) * 32);
            const float ur = u.x, ui = fwd ? u.y : -u.y;
            const float2 UR = make_float2(ur, ur), UI = make_float2(ui, ui), NUI = make_float2(-ui, -ui);
#pragma unroll
            for (int a = 0; a < 2; ++a) {
                CP& acc = uh[a][c];
                acc.re = __ffma2_rn(UR, h[a][b].re, acc.re);
                acc.re = __ffma2_rn(NUI, h[a][b].im, acc.re);
                acc.im = __ffma2_rn(UR, h[a][b].im, acc.im);
                acc.im = __ffma2_rn(UI, h[a][b].re, acc.im);
            }
        }
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int c = 0; c < 3; ++c) up[a][c] = cp_fma_s(ph, uh[a][c], up[a][c]);
    pair_lower(mu, minus ? -ph : ph, uh, lo);
}

// Output element e of the pair: diag psi + s-hop - 1/2 (Wilson hops).  sv: the site's own value on
// both slices; q: the element of the neighbouring pair that holds this half's s-hop source
// (jb = the pair below for a hop from s - 1, ja = the pair above for one from s + 1).
template <bool DAG>
__device__ __forceinline__ CP pair_out(int e, CP sv, CP q, CP acc, float fb, float fa, float diag) {
    const bool below = (e < 6) != DAG;                // this half's hop comes from s - 1
    CP hop;
    if (below) hop = CP{make_float2(fb * q.re.y, sv.re.x), make_float2(fb * q.im.y, sv.im.x)};
    else       hop = CP{make_float2(sv.re.y, fa * q.re.x), make_float2(sv.im.y, fa * q.im.x)};
    CP r = cp_fma_s(-0.5f, acc, hop);
    return cp_fma_s(diag, sv, r);
}

// neighbour of `site` in direction d = 2 mu + (0 forward, 1 backward); cross: the hop wraps
// around the lattice boundary
__device__ __forceinline__ int pair_nb(const Fine4dParams& p, int site, int d, bool& cross) {
    const int mu = d >> 1;
    int st = 1;
#pragma unroll
    for (int m = 0; m < 4; ++m)
        if (m < mu) st *= p.L[m];
    const int L = p.L[mu];
    const int c = (site / st) % L;
    if ((d & 1) == 0) { cross = c == L - 1; return cross ? site - (L - 1) * st : site + st; }
    cross = c == 0;
    return cross ? site + (L - 1) * st : site - st;
}

constexpr int PAIR_PY = 2;                    // slice pairs per block
constexpr int PAIR_THREADS = 32 * PAIR_PY;

// Block: 32 sites x 2 slice pairs; blocks numbered pair group fastest, so the blocks running at
// one time cover a compact stretch of the lattice and the neighbour loads of one block find the
// other blocks' spinors in L2.  128 registers give eight blocks (16 warps) per SM; the neighbour
// spinors of one direction are loaded together, and their latency is hidden across warps.
// Measured at 16^3 x 32 x 16: 119 us with 2 pairs per block, 119 us with 1, 122.5 us with 4,
// 137 us with 8.
template <class LT, bool DAG>
__global__ void __launch_bounds__(PAIR_THREADS, 8) k_dwf4d_pair(const typename LT::store* __restrict__ U,
                                                       const float4* __restrict__ psi, float4* __restrict__ out,
                                                       Fine4dParams p, LayP2 lay, int ngroups, const int* skip) {
    if (skip && *skip) return;
    const int site = (int)(blockIdx.x / ngroups) * 32 + threadIdx.x;
    const int j = (int)(blockIdx.x % ngroups) * PAIR_PY + threadIdx.y;
    if (site >= p.V || j >= lay.NP) return;
    const int jb = j > 0 ? j - 1 : lay.NP - 1;        // pair holding slice 2j - 1 (or the wall Ls - 1)
    const int ja = j + 1 < lay.NP ? j + 1 : 0;        // pair holding slice 2j + 2 (or the wall 0)
    CP up[2][3], lo[2][3];
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            up[a][c] = CP{make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
            lo[a][c] = up[a][c];
        }
#pragma unroll
    for (int d = 0; d < 8; ++d) {
        const int mu = d >> 1;
        const bool fwd = (d & 1) == 0;
        bool cross;
        const int nb = pair_nb(p, site, d, cross);
        CP v[4][3];
#pragma unroll
        for (int e = 0; e < 12; ++e) v[e / 3][e % 3] = ld_cp(psi, lay.idx(j, nb, e));
        const float ph = (cross && p.anti[mu]) ? -1.f : 1.f;
        pair_hop<LT, DAG>(mu, fwd, ph, v, U, lay.lk(mu, fwd ? site : nb), up, lo);
    }
    const float mf = p.mf_f;
    const float fb = j > 0 ? 1.f : -mf, fa = j + 1 < lay.NP ? 1.f : -mf;
    CP self[12];
#pragma unroll
    for (int e = 0; e < 12; ++e) self[e] = ld_cp(psi, lay.idx(j, site, e));
#pragma unroll
    for (int e = 0; e < 12; ++e) {
        const CP sv = self[e];
        const CP q = ld_cp(psi, lay.idx(((e < 6) != DAG) ? jb : ja, site, e));
        const int e6 = e % 6;
        const CP acc = e < 6 ? up[e6 / 3][e6 % 3] : lo[e6 / 3][e6 % 3];
        const CP r = pair_out<DAG>(e, sv, q, acc, fb, fa, p.diag_f);
        __stcs(out + lay.idx(j, site, e), make_float4(r.re.x, r.im.x, r.re.y, r.im.y));
    }
}

template <class LT>
dwf_status launch_pair(const void* U, const void* psi, void* out, const Fine4dParams& p, const LayP2& lay, bool dagger,
                       cudaStream_t st, const int* skip) {
    const long long ng = (lay.NP + PAIR_PY - 1) / PAIR_PY;
    const long long blocks = lay.NB * ng;
    if (blocks > 0x7fffffffLL) { set_error("4-d lattice too large for one launch"); return DWF_ERR_ARG; }
    dim3 block(32, PAIR_PY);
    auto Ut = reinterpret_cast<const typename LT::store*>(U);
    if (dagger) k_dwf4d_pair<LT, true><<<(unsigned)blocks, block, 0, st>>>(Ut, (const float4*)psi, (float4*)out, p, lay, (int)ng, skip);
    else        k_dwf4d_pair<LT, false><<<(unsigned)blocks, block, 0, st>>>(Ut, (const float4*)psi, (float4*)out, p, lay, (int)ng, skip);
    DWF_CHECK_LAUNCH();
    return DWF_OK;
}

// ---- conversions canonical <-> slice-paired packed ----
// one thread per (pair, site, element): sites past V are written as zero
__global__ void k_pack_pair(const float2* __restrict__ in, float4* __restrict__ out, long long V, long long NB, int NP) {
    const long long n = (long long)NP * NB * 32 * 12;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(t & 31);
        const long long r = t >> 5;
        const int k = (int)(r % 12);
        const long long jb = r / 12;
        const long long b = jb % NB, j = jb / NB;
        const long long site = b * 32 + i;
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (site < V) {
            const float2 a = in[((2 * j) * V + site) * 12 + k], c = in[((2 * j + 1) * V + site) * 12 + k];
            v = make_float4(a.x, a.y, c.x, c.y);
        }
        out[t] = v;
    }
}

__global__ void k_unpack_pair(const float4* __restrict__ in, float2* __restrict__ out, long long V, long long NB,
                              int NP) {
    const long long n = (long long)NP * V * 12;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
        const int k = (int)(t % 12);
        const long long r = t / 12;
        const long long site = r % V, j = r / V;
        const float4 v = in[((j * NB + (site >> 5)) * 12 + k) * 32 + (site & 31)];
        out[((2 * j) * V + site) * 12 + k] = make_float2(v.x, v.y);
        out[((2 * j + 1) * V + site) * 12 + k] = make_float2(v.z, v.w);
    }
}

int pair_grid(long long n) { return (int)std::min<long long>((n + 255) / 256, 152LL * 16); }

}  // namespace

dwf_status fine_apply_4d_paired(const Geom& g, const void* U, const void* psi, void* out, double M5, double mf,
                                bool dagger, int prec, cudaStream_t st, const int* skip) {
    if (g.Ls % 2) { set_error("the slice-paired layout needs an even Ls (got %d)", g.Ls); return DWF_ERR_UNSUPPORTED; }
    if (g.V > (1LL << 28)) { set_error("4-d lattices are limited to 2^28 sites"); return DWF_ERR_UNSUPPORTED; }
    Fine4dParams p;
    p.V = g.V;
    for (int mu = 0; mu < 4; ++mu) { p.L[mu] = g.L[mu]; p.anti[mu] = g.anti[mu]; }
    p.Ls = g.Ls;
    p.diag = (double)g.nd - M5 + 1.0;
    p.mf = mf;
    p.diag_f = (float)p.diag;
    p.mf_f = (float)mf;
    p.s_chunk = 0;
    LayP2 lay{(g.V + 31) / 32, g.Ls / 2};
    switch (prec) {
        case DWF_F32:       return launch_pair<LinkF32>(U, psi, out, p, lay, dagger, st, skip);
        case DWF_F32_L16:   return launch_pair<LinkH16>(U, psi, out, p, lay, dagger, st, skip);
        case DWF_F32_LBF16: return launch_pair<LinkBF16>(U, psi, out, p, lay, dagger, st, skip);
        default: set_error("the packed layout takes FP32 spinors (precision %d)", prec); return DWF_ERR_ARG;
    }
}

dwf_status pack_spinor_paired(const Geom& g, const void* psi, void* packed, cudaStream_t st) {
    if (g.Ls % 2) { set_error("the slice-paired layout needs an even Ls (got %d)", g.Ls); return DWF_ERR_UNSUPPORTED; }
    const long long NB = (g.V + 31) / 32, n = (long long)(g.Ls / 2) * NB * 32 * 12;
    k_pack_pair<<<pair_grid(n), 256, 0, st>>>((const float2*)psi, (float4*)packed, g.V, NB, g.Ls / 2);
    DWF_CHECK_LAUNCH();
    return DWF_OK;
}

dwf_status unpack_spinor_paired(const Geom& g, const void* packed, void* psi, cudaStream_t st) {
    if (g.Ls % 2) { set_error("the slice-paired layout needs an even Ls (got %d)", g.Ls); return DWF_ERR_UNSUPPORTED; }
    const long long NB = (g.V + 31) / 32, n = (long long)(g.Ls / 2) * g.V * 12;
    k_unpack_pair<<<pair_grid(n), 256, 0, st>>>((const float4*)packed, (float2*)psi, g.V, NB, g.Ls / 2);
    DWF_CHECK_LAUNCH();
    return DWF_OK;
}

}  // namespace dwf
