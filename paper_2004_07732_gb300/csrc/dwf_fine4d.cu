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
#include "common.cuh"
#include "fine_kernels.cuh"

namespace dwf {

template <class C> struct HalfSp { C v[2][3]; };   // 2 spins x 3 colours

template <class R> struct Spin4 { typename cplx<R>::T v[4][3]; };

__device__ __forceinline__ void ld_spin4(const float2* p, long long site, Spin4<float>& s) {
    const float4* q = reinterpret_cast<const float4*>(p + site * 12);
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        float4 a = __ldg(q + k);
        const int e0 = 2 * k, e1 = 2 * k + 1;
        s.v[e0 / 3][e0 % 3] = make_float2(a.x, a.y);
        s.v[e1 / 3][e1 % 3] = make_float2(a.z, a.w);
    }
}
__device__ __forceinline__ void ld_spin4(const double2* p, long long site, Spin4<double>& s) {
    const double2* q = p + site * 12;
#pragma unroll
    for (int e = 0; e < 12; ++e) s.v[e / 3][e % 3] = __ldg(q + e);
}
__device__ __forceinline__ void st_spin4(float2* p, long long site, const Spin4<float>& s) {
    float4* q = reinterpret_cast<float4*>(p + site * 12);
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        const int e0 = 2 * k, e1 = 2 * k + 1;
        __stcs(q + k, make_float4(s.v[e0 / 3][e0 % 3].x, s.v[e0 / 3][e0 % 3].y, s.v[e1 / 3][e1 % 3].x,
                                  s.v[e1 / 3][e1 % 3].y));
    }
}
__device__ __forceinline__ void st_spin4(double2* p, long long site, const Spin4<double>& s) {
    double2* q = p + site * 12;
#pragma unroll
    for (int e = 0; e < 12; ++e) __stcs(q + e, s.v[e / 3][e % 3]);
}

// 3x3 link, row-major complex, in the storage of the link precision
template <class LT, class C>
__device__ __forceinline__ void ld_link3(const typename LT::store* U, long long idx, C (&u)[3][3]) {
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            auto v = load_link(U, idx * 9 + a * 3 + b);
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

template <class LT, class R, bool DAG>
__global__ void __launch_bounds__(256) k_dwf4d(const typename LT::store* __restrict__ U,
                                               const typename cplx<R>::T* __restrict__ psi,
                                               typename cplx<R>::T* __restrict__ out, Fine4dParams p) {
    using C = typename cplx<R>::T;
    const long long site = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int s = blockIdx.y * blockDim.y + threadIdx.y;
    if (site >= p.V || s >= p.Ls) return;
    const long long V = p.V;
    long long stride[4];
    int coord[4];
    {
        long long st = 1, rem = site;
#pragma unroll
        for (int mu = 0; mu < 4; ++mu) {
            stride[mu] = st;
            coord[mu] = (int)(rem % p.L[mu]);
            rem /= p.L[mu];
            st *= p.L[mu];
        }
    }
    const long long base = (long long)s * V;
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
            const long long nb = fwd ? (cross ? site - (long long)(L - 1) * stride[mu] : site + stride[mu])
                                     : (cross ? site + (long long)(L - 1) * stride[mu] : site - stride[mu]);
            const R ph = (cross && p.anti[mu]) ? R(-1) : R(1);
            // projector sign: D uses (1 - gamma) forward, (1 + gamma) backward; D^dag the opposite
            const bool minus = (fwd != DAG);
            Spin4<R> v;
            ld_spin4(psi + 0, base + nb, v);
            C lw[2][3] = {{v.v[2][0], v.v[2][1], v.v[2][2]}, {v.v[3][0], v.v[3][1], v.v[3][2]}};
            C Al[2][3];
            apply_A(mu, lw, Al);
            C h[2][3];
#pragma unroll
            for (int a = 0; a < 2; ++a)
#pragma unroll
                for (int c = 0; c < 3; ++c) h[a][c] = minus ? (v.v[a][c] - Al[a][c]) : (v.v[a][c] + Al[a][c]);
            C u[3][3];
            ld_link3<LT, C>(U, (long long)mu * V + (fwd ? site : nb), u);
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
                    uh[a][c] = scale(acc, ph);
                }
            C Ad[2][3];
            apply_Adag(mu, uh, Ad);
#pragma unroll
            for (int a = 0; a < 2; ++a)
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    up[a][c] = up[a][c] + uh[a][c];
                    lo[a][c] = minus ? (lo[a][c] - Ad[a][c]) : (lo[a][c] + Ad[a][c]);
                }
        }
    }
    const R diag = R(p.diag);
    const R mf = R(p.mf);
    Spin4<R> self;
    ld_spin4(psi + 0, base + site, self);
    // s-hops: D: up += psi_{s-1}.up (or -m psi_{Ls-1}.up), lo += psi_{s+1}.lo (or -m psi_0.lo)
    //         D^dag: up from s+1 / wall psi_0, lo from s-1 / wall psi_{Ls-1}
    const int s_up = DAG ? (s + 1 < p.Ls ? s + 1 : 0) : (s > 0 ? s - 1 : p.Ls - 1);
    const int s_lo = DAG ? (s > 0 ? s - 1 : p.Ls - 1) : (s + 1 < p.Ls ? s + 1 : 0);
    const R f_up = DAG ? (s + 1 < p.Ls ? R(1) : -mf) : (s > 0 ? R(1) : -mf);
    const R f_lo = DAG ? (s > 0 ? R(1) : -mf) : (s + 1 < p.Ls ? R(1) : -mf);
    Spin4<R> o;
    const C* pu = psi + ((long long)s_up * V + site) * 12;
    const C* pl = psi + ((long long)s_lo * V + site) * 12;
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            o.v[a][c] = scale(up[a][c], R(-0.5)) + scale(self.v[a][c], diag) + scale(__ldg(pu + a * 3 + c), f_up);
            o.v[a + 2][c] = scale(lo[a][c], R(-0.5)) + scale(self.v[a + 2][c], diag) + scale(__ldg(pl + (a + 2) * 3 + c), f_lo);
        }
    st_spin4(out + 0, base + site, o);
}

template <class LT, class R>
static void launch4d(const void* U, const void* psi, void* out, const Fine4dParams& p, bool dagger, cudaStream_t st) {
    dim3 block(32, 8);
    dim3 grid((unsigned)((p.V + 31) / 32), (unsigned)((p.Ls + 7) / 8));
    using C = typename cplx<R>::T;
    auto Ut = reinterpret_cast<const typename LT::store*>(U);
    auto pi = reinterpret_cast<const C*>(psi);
    auto po = reinterpret_cast<C*>(out);
    if (dagger) k_dwf4d<LT, R, true><<<grid, block, 0, st>>>(Ut, pi, po, p);
    else        k_dwf4d<LT, R, false><<<grid, block, 0, st>>>(Ut, pi, po, p);
}

dwf_status fine_apply_4d(const Geom& g, const void* U, const void* psi, void* out, double M5, double mf,
                         bool dagger, int prec, int s_chunk, cudaStream_t st) {
    (void)s_chunk;
    Fine4dParams p;
    p.V = g.V;
    for (int mu = 0; mu < 4; ++mu) { p.L[mu] = g.L[mu]; p.anti[mu] = g.anti[mu]; }
    p.Ls = g.Ls;
    p.diag = (double)g.nd - M5 + 1.0;
    p.mf = mf;
    p.s_chunk = 0;
    switch (prec) {
        case DWF_F64:       launch4d<LinkF64, double>(U, psi, out, p, dagger, st); break;
        case DWF_F32:       launch4d<LinkF32, float>(U, psi, out, p, dagger, st); break;
        case DWF_F32_L16:   launch4d<LinkH16, float>(U, psi, out, p, dagger, st); break;
        case DWF_F32_LBF16: launch4d<LinkBF16, float>(U, psi, out, p, dagger, st); break;
        default: set_error("bad precision %d", prec); return DWF_ERR_ARG;
    }
    DWF_CHECK_LAUNCH();
    return DWF_OK;
}

}  // namespace dwf
