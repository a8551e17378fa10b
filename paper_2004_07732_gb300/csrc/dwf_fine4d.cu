// 4-d SU(3) Shamir operator: Eq. DWoperator with the 4-d Wilson kernel on
// 4 spins x 3 colours, chiral basis gamma_5 = diag(1, 1, -1, -1).
//
// One thread per 5-d site; a block is 32 consecutive sites x 8 slices, so the
// eight threads of a site that differ in s read its links through L1.  In the
// chiral basis gamma_mu = [[0, A_mu], [A_mu^dag, 0]] (A = -i sigma_k, or 1 for
// mu = 3); (1 -+ gamma_mu) psi = (h, -+ A^dag h) with the half spinor
// h = psi_up -+ A psi_low, so each hop multiplies two colour vectors by the
// link (the spin projection of the Wilson operator).  P_+ / P_- are the upper /
// lower spin pairs, so the s-hops add half spinors of psi_{s-1} and psi_{s+1}.
//
// Layout: canonical, psi[s][site][spin][colour] and U[mu][site][3][3], as the
// C ABI defines them.  The packed layout (dwf_pack_spinor / dwf_apply_packed) has
// its own kernel in dwf_fine4d_pair.cu; this file keeps the packed links'
// conversion and the packed entry points.
#include "common.cuh"
#include "fine_kernels.cuh"

namespace dwf {

template <class C> struct HalfSp { C v[2][3]; };   // 2 spins x 3 colours

template <class R> struct Spin4 { typename cplx<R>::T v[4][3]; };

// Canonical layout.  f4(s, site): float4 index of piece 0 of an FP32 spinor,
// pieces KS apart; rec(s, site): site record of an FP64 spinor (12 double2);
// lk(mu, site): index of entry 0 of a link, entries JS apart.  Sites are
// 32-bit (a 4-d lattice has at most 2^28 of them); slice and direction
// offsets are 64-bit.
struct LayCanon {
    static constexpr int KS = 1, JS = 1;
    long long V;
    __device__ __forceinline__ long long f4(int s, int site) const { return (long long)s * (V * 6) + (long long)site * 6; }
    __device__ __forceinline__ long long rec(int s, int site) const { return (long long)s * V + site; }
    __device__ __forceinline__ long long lk(int mu, int site) const { return (long long)mu * (V * 9) + (long long)site * 9; }
};
template <class LAY>
__device__ __forceinline__ void ld_spin4(const float2* p, const LAY& L, int s, int site, Spin4<float>& v) {
    const float4* q = reinterpret_cast<const float4*>(p) + L.f4(s, site);
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        float4 a = __ldg(q + k * LAY::KS);
        const int e0 = 2 * k, e1 = 2 * k + 1;
        v.v[e0 / 3][e0 % 3] = make_float2(a.x, a.y);
        v.v[e1 / 3][e1 % 3] = make_float2(a.z, a.w);
    }
}
__device__ __forceinline__ void ld_spin4(const double2* p, const LayCanon& L, int s, int site, Spin4<double>& v) {
    const double2* q = p + L.rec(s, site) * 12;
#pragma unroll
    for (int e = 0; e < 12; ++e) v.v[e / 3][e % 3] = __ldg(q + e);
}
// spins 2 hi, 2 hi + 1 (hi = 0: upper pair, 1: lower pair) into h[0..1]
template <class LAY>
__device__ __forceinline__ void ld_half(const float2* p, const LAY& L, int s, int site, int hi, float2 (&h)[2][3]) {
    const float4* q = reinterpret_cast<const float4*>(p) + L.f4(s, site) + 3 * hi * LAY::KS;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        float4 a = __ldg(q + k * LAY::KS);
        const int e0 = 2 * k, e1 = 2 * k + 1;
        h[e0 / 3][e0 % 3] = make_float2(a.x, a.y);
        h[e1 / 3][e1 % 3] = make_float2(a.z, a.w);
    }
}
__device__ __forceinline__ void ld_half(const double2* p, const LayCanon& L, int s, int site, int hi, double2 (&h)[2][3]) {
    const double2* q = p + L.rec(s, site) * 12 + 6 * hi;
#pragma unroll
    for (int e = 0; e < 6; ++e) h[e / 3][e % 3] = __ldg(q + e);
}
template <class LAY>
__device__ __forceinline__ void st_spin4(float2* p, const LAY& L, int s, int site, const Spin4<float>& v) {
    float4* q = reinterpret_cast<float4*>(p) + L.f4(s, site);
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        const int e0 = 2 * k, e1 = 2 * k + 1;
        __stcs(q + k * LAY::KS, make_float4(v.v[e0 / 3][e0 % 3].x, v.v[e0 / 3][e0 % 3].y, v.v[e1 / 3][e1 % 3].x,
                                            v.v[e1 / 3][e1 % 3].y));
    }
}
__device__ __forceinline__ void st_spin4(double2* p, const LayCanon& L, int s, int site, const Spin4<double>& v) {
    double2* q = p + L.rec(s, site) * 12;
#pragma unroll
    for (int e = 0; e < 12; ++e) __stcs(q + e, v.v[e / 3][e % 3]);
}

// 3x3 link, row-major complex, in the storage of the link precision
template <class LT, class LAY, class C>
__device__ __forceinline__ void ld_link3(const typename LT::store* U, const LAY& L, int mu, int site, C (&u)[3][3]) {
    const long long b0 = L.lk(mu, site);
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            auto v = load_link(U, b0 + (a * 3 + b) * LAY::JS);
            u[a][b].x = v.x;
            u[a][b].y = v.y;
        }
}

// A psi_low for direction mu (A = -i sigma_1, -i sigma_2, -i sigma_3, 1)
template <class C>
__device__ __forceinline__ void apply_A(int mu, const C (&l)[2][3], C (&o)[2][3]) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        if (mu == 0) { o[0][c] = mk<C>(l[1][c].y, -l[1][c].x); o[1][c] = mk<C>(l[0][c].y, -l[0][c].x); }      // -i l1, -i l0
        else if (mu == 1) { o[0][c] = mk<C>(-l[1][c].x, -l[1][c].y); o[1][c] = l[0][c]; }                      // -l1, l0
        else if (mu == 2) { o[0][c] = mk<C>(l[0][c].y, -l[0][c].x); o[1][c] = mk<C>(-l[1][c].y, l[1][c].x); }  // -i l0, i l1
        else { o[0][c] = l[0][c]; o[1][c] = l[1][c]; }
    }
}
// A^dag h
template <class C>
__device__ __forceinline__ void apply_Adag(int mu, const C (&h)[2][3], C (&o)[2][3]) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        if (mu == 0) { o[0][c] = mk<C>(-h[1][c].y, h[1][c].x); o[1][c] = mk<C>(-h[0][c].y, h[0][c].x); }      // i h1, i h0
        else if (mu == 1) { o[0][c] = h[1][c]; o[1][c] = mk<C>(-h[0][c].x, -h[0][c].y); }                      // h1, -h0
        else if (mu == 2) { o[0][c] = mk<C>(-h[0][c].y, h[0][c].x); o[1][c] = mk<C>(h[1][c].y, -h[1][c].x); }  // i h0, -i h1
        else { o[0][c] = h[0][c]; o[1][c] = h[1][c]; }
    }
}

// Block: 32 consecutive sites x 8 slices.  Blocks are numbered slice group
// fastest, so the slice groups of one set of sites run together and share its
// links and boundary slices in L2.
template <class R> __device__ __forceinline__ R param_cast(double d, float f);
template <> __device__ __forceinline__ double param_cast<double>(double d, float) { return d; }
template <> __device__ __forceinline__ float param_cast<float>(double, float f) { return f; }

template <class LT, class R, bool DAG, class LAY>
__global__ void __launch_bounds__(256, 3) k_dwf4d(const typename LT::store* __restrict__ U,
                                               const typename cplx<R>::T* __restrict__ psi,
                                               typename cplx<R>::T* __restrict__ out, Fine4dParams p, LAY lay,
                                               int ngroups, const int* skip) {
    if (skip && *skip) return;
    using C = typename cplx<R>::T;
    const int site = (int)(blockIdx.x / ngroups) * 32 + threadIdx.x;
    const int s = (int)(blockIdx.x % ngroups) * 8 + threadIdx.y;
    if (site >= p.V || s >= p.Ls) return;
    int stride[4];
    int coord[4];
    {
        int st = 1, rem = site;
#pragma unroll
        for (int mu = 0; mu < 4; ++mu) {
            stride[mu] = st;
            coord[mu] = rem % p.L[mu];
            rem /= p.L[mu];
            st *= p.L[mu];
        }
    }
    C up[2][3], lo[2][3];     // accumulated -1/2 sum of hops, upper / lower spin pairs
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int c = 0; c < 3; ++c) { up[a][c] = mk<C>(R(0), R(0)); lo[a][c] = mk<C>(R(0), R(0)); }

#pragma unroll
    for (int mu = 0; mu < 4; ++mu) {
        const int L = p.L[mu];
        // forward: y = x + mu, link U_mu(x); backward: y = x - mu, link U_mu(y)^dag
#pragma unroll
        for (int dirn = 0; dirn < 2; ++dirn) {
            const bool fwd = dirn == 0;
            const bool cross = fwd ? (coord[mu] == L - 1) : (coord[mu] == 0);
            const int nb = fwd ? (cross ? site - (L - 1) * stride[mu] : site + stride[mu])
                               : (cross ? site + (L - 1) * stride[mu] : site - stride[mu]);
            const R ph = (cross && p.anti[mu]) ? R(-1) : R(1);
            // projector sign: D uses (1 - gamma) forward, (1 + gamma) backward; D^dag the opposite
            const bool minus = (fwd != DAG);
            Spin4<R> v;
            ld_spin4(psi + 0, lay, s, nb, v);
            C lw[2][3] = {{v.v[2][0], v.v[2][1], v.v[2][2]}, {v.v[3][0], v.v[3][1], v.v[3][2]}};
            C Al[2][3];
            apply_A(mu, lw, Al);
            C h[2][3];
#pragma unroll
            for (int a = 0; a < 2; ++a)
#pragma unroll
                for (int c = 0; c < 3; ++c) h[a][c] = minus ? (v.v[a][c] - Al[a][c]) : (v.v[a][c] + Al[a][c]);
            C u[3][3];
            ld_link3<LT>(U, lay, mu, fwd ? site : nb, u);
            C uh[2][3];
#pragma unroll
            for (int a = 0; a < 2; ++a)
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    C acc = mk<C>(R(0), R(0));
#pragma unroll
                    for (int b = 0; b < 3; ++b) {
                        // forward: U h; backward: U^dag h
                        const C uu = fwd ? u[c][b] : mk<C>(u[b][c].x, -u[b][c].y);
                        acc = acc + cmul(uu, h[a][b]);
                    }
                    uh[a][c] = acc;
                }
            C Ad[2][3];
            apply_Adag(mu, uh, Ad);
#pragma unroll
            for (int a = 0; a < 2; ++a)
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    // the boundary phase rides on the accumulating multiply-adds
                    up[a][c] = up[a][c] + scale(uh[a][c], ph);
                    lo[a][c] = lo[a][c] + scale(Ad[a][c], minus ? -ph : ph);
                }
        }
    }
    const R diag = param_cast<R>(p.diag, p.diag_f);
    const R mf = param_cast<R>(p.mf, p.mf_f);
    Spin4<R> self;
    ld_spin4(psi + 0, lay, s, site, self);
    // s-hops: D: up += psi_{s-1}.up (or -m psi_{Ls-1}.up), lo += psi_{s+1}.lo (or -m psi_0.lo)
    //         D^dag: up from s+1 / wall psi_0, lo from s-1 / wall psi_{Ls-1}
    const int s_up = DAG ? (s + 1 < p.Ls ? s + 1 : 0) : (s > 0 ? s - 1 : p.Ls - 1);
    const int s_lo = DAG ? (s > 0 ? s - 1 : p.Ls - 1) : (s + 1 < p.Ls ? s + 1 : 0);
    const R f_up = DAG ? (s + 1 < p.Ls ? R(1) : -mf) : (s > 0 ? R(1) : -mf);
    const R f_lo = DAG ? (s > 0 ? R(1) : -mf) : (s + 1 < p.Ls ? R(1) : -mf);
    C hu[2][3], hl[2][3];
    ld_half(psi + 0, lay, s_up, site, 0, hu);
    ld_half(psi + 0, lay, s_lo, site, 1, hl);
    Spin4<R> o;
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            o.v[a][c] = scale(up[a][c], R(-0.5)) + scale(self.v[a][c], diag) + scale(hu[a][c], f_up);
            o.v[a + 2][c] = scale(lo[a][c], R(-0.5)) + scale(self.v[a + 2][c], diag) + scale(hl[a][c], f_lo);
        }
    st_spin4(out + 0, lay, s, site, o);
}

static dwf_status grid4d(const Fine4dParams& p, unsigned* blocks, int* ngroups) {
    if (p.V > (1LL << 28)) { set_error("4-d lattices are limited to 2^28 sites"); return DWF_ERR_UNSUPPORTED; }
    const long long nb = (p.V + 31) / 32, ng = (p.Ls + 7) / 8;
    if (nb * ng > 0x7fffffffLL) { set_error("4-d lattice too large for one launch"); return DWF_ERR_ARG; }
    *blocks = (unsigned)(nb * ng);
    *ngroups = (int)ng;
    return DWF_OK;
}

template <class LT, class R, class LAY>
static dwf_status launch4d(const void* U, const void* psi, void* out, const Fine4dParams& p, const LAY& lay,
                           bool dagger, cudaStream_t st, const int* skip = nullptr) {
    unsigned blocks;
    int ng;
    DWF_TRY(grid4d(p, &blocks, &ng));
    dim3 block(32, 8);
    using C = typename cplx<R>::T;
    auto Ut = reinterpret_cast<const typename LT::store*>(U);
    auto pi = reinterpret_cast<const C*>(psi);
    auto po = reinterpret_cast<C*>(out);
    if (dagger) k_dwf4d<LT, R, true, LAY><<<blocks, block, 0, st>>>(Ut, pi, po, p, lay, ng, skip);
    else        k_dwf4d<LT, R, false, LAY><<<blocks, block, 0, st>>>(Ut, pi, po, p, lay, ng, skip);
    return DWF_OK;
}

static Fine4dParams params4d(const Geom& g, double M5, double mf) {
    Fine4dParams p;
    p.V = g.V;
    for (int mu = 0; mu < 4; ++mu) { p.L[mu] = g.L[mu]; p.anti[mu] = g.anti[mu]; }
    p.Ls = g.Ls;
    p.diag = (double)g.nd - M5 + 1.0;
    p.mf = mf;
    p.diag_f = (float)p.diag;
    p.mf_f = (float)mf;
    p.s_chunk = 0;
    return p;
}

dwf_status fine_apply_4d(const Geom& g, const void* U, const void* psi, void* out, double M5, double mf,
                         bool dagger, int prec, int s_chunk, cudaStream_t st, const int* skip) {
    (void)s_chunk;
    const Fine4dParams p = params4d(g, M5, mf);
    LayCanon lay{g.V};
    switch (prec) {
        case DWF_F64:       DWF_TRY((launch4d<LinkF64, double>(U, psi, out, p, lay, dagger, st, skip))); break;
        case DWF_F32:       DWF_TRY((launch4d<LinkF32, float>(U, psi, out, p, lay, dagger, st, skip))); break;
        case DWF_F32_L16:   DWF_TRY((launch4d<LinkH16, float>(U, psi, out, p, lay, dagger, st, skip))); break;
        case DWF_F32_LBF16: DWF_TRY((launch4d<LinkBF16, float>(U, psi, out, p, lay, dagger, st, skip))); break;
        default: set_error("bad precision %d", prec); return DWF_ERR_ARG;
    }
    DWF_CHECK_LAUNCH();
    return DWF_OK;
}

template <class T> __device__ __forceinline__ T cvt_link_p(double2 v);
template <> __device__ __forceinline__ float2 cvt_link_p<float2>(double2 v) {
    return make_float2(__double2float_rn(v.x), __double2float_rn(v.y));
}
template <> __device__ __forceinline__ __half2 cvt_link_p<__half2>(double2 v) {
    return __halves2half2(__double2half(v.x), __double2half(v.y));
}
template <> __device__ __forceinline__ __nv_bfloat162 cvt_link_p<__nv_bfloat162>(double2 v) {
    return __halves2bfloat162(__double2bfloat16(v.x), __double2bfloat16(v.y));
}
// one thread per packed link entry (mu, block, j, slot); entries of sites past V are zero
template <class T>
__global__ void k_pack_links(const double2* __restrict__ in, T* __restrict__ out, long long V, long long NB, long long n) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const long long slot = i & 31, j = (i >> 5) % 9, blk = (i >> 5) / 9;
        const long long mu = blk / NB, site = (blk % NB) * 32 + slot;
        out[i] = site < V ? cvt_link_p<T>(in[(mu * V + site) * 9 + j]) : cvt_link_p<T>(make_double2(0.0, 0.0));
    }
}

static dwf_status check_packed(const dwf_geom* g, Geom* G) {
    DWF_TRY(check_geom(g, G));
    if (G->nd != 4) { set_error("the packed layout is defined for 4-d SU(3) lattices"); return DWF_ERR_UNSUPPORTED; }
    return DWF_OK;
}
static int grid_for(long long n) { return (int)std::min<long long>((n + 255) / 256, 152LL * 16); }

}  // namespace dwf

using namespace dwf;

extern "C" {

size_t dwf_packed_spinor_size(const dwf_geom* g) {
    Geom G;
    if (check_geom(g, &G) != DWF_OK || G.nd != 4 || G.Ls % 2) return 0;
    return (size_t)(G.Ls * ((G.V + 31) / 32) * 32 * 12);
}

size_t dwf_packed_link_size(const dwf_geom* g) {
    Geom G;
    if (check_geom(g, &G) != DWF_OK || G.nd != 4) return 0;
    return (size_t)(4 * ((G.V + 31) / 32) * 32 * 9);
}

dwf_status dwf_pack_links(const dwf_geom* g, const void* U64, void* U_packed, int prec, void* stream) {
    clear_error();
    Geom G;
    DWF_TRY(check_packed(g, &G));
    if (prec != DWF_F32 && prec != DWF_F32_L16 && prec != DWF_F32_LBF16) {
        set_error("packed links take precision F32, F32_L16 or F32_LBF16 (got %d)", prec);
        return DWF_ERR_ARG;
    }
    const long long NB = (G.V + 31) / 32, n = 4 * NB * 32 * 9;
    if (!U64 || !U_packed) { set_error("NULL link pointer"); return DWF_ERR_ARG; }
    cudaStream_t st = as_stream(stream);
    auto in = reinterpret_cast<const double2*>(U64);
    const int blocks = grid_for(n);
    if (prec == DWF_F32) k_pack_links<float2><<<blocks, 256, 0, st>>>(in, (float2*)U_packed, G.V, NB, n);
    else if (prec == DWF_F32_L16) k_pack_links<__half2><<<blocks, 256, 0, st>>>(in, (__half2*)U_packed, G.V, NB, n);
    else k_pack_links<__nv_bfloat162><<<blocks, 256, 0, st>>>(in, (__nv_bfloat162*)U_packed, G.V, NB, n);
    DWF_CHECK_LAUNCH();
    return DWF_OK;
}

dwf_status dwf_pack_spinor(const dwf_geom* g, const void* psi, void* packed, void* stream) {
    clear_error();
    Geom G;
    DWF_TRY(check_packed(g, &G));
    if (!psi || !packed) { set_error("NULL device pointer"); return DWF_ERR_ARG; }
    if (!aligned16(psi) || !aligned16(packed)) { set_error("spinor buffers must be 16-byte aligned"); return DWF_ERR_ARG; }
    if (psi == packed) { set_error("psi and packed must be distinct buffers"); return DWF_ERR_ARG; }
    return pack_spinor_paired(G, psi, packed, as_stream(stream));
}

dwf_status dwf_unpack_spinor(const dwf_geom* g, const void* packed, void* psi, void* stream) {
    clear_error();
    Geom G;
    DWF_TRY(check_packed(g, &G));
    if (!psi || !packed) { set_error("NULL device pointer"); return DWF_ERR_ARG; }
    if (!aligned16(psi) || !aligned16(packed)) { set_error("spinor buffers must be 16-byte aligned"); return DWF_ERR_ARG; }
    if (psi == packed) { set_error("psi and packed must be distinct buffers"); return DWF_ERR_ARG; }
    return unpack_spinor_paired(G, packed, psi, as_stream(stream));
}

dwf_status dwf_apply_packed(const dwf_geom* g, const void* U_packed, const void* psi, void* out, double M5,
                            double mf, int dagger, int prec, void* stream) {
    clear_error();
    Geom G;
    DWF_TRY(check_packed(g, &G));
    if (!U_packed || !psi || !out) { set_error("NULL device pointer"); return DWF_ERR_ARG; }
    if (!aligned16(psi) || !aligned16(out)) { set_error("spinor buffers must be 16-byte aligned"); return DWF_ERR_ARG; }
    if (psi == out) { set_error("psi and out must be distinct buffers"); return DWF_ERR_ARG; }
    return fine_apply_4d_paired(G, U_packed, psi, out, M5, mf, dagger != 0, prec, as_stream(stream));
}

}  // extern "C"
