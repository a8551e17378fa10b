// Fine-level Shamir domain-wall operator D_DW(m) (Eq. DWoperator, Sec. 2) and
// its Pauli-Villars / dagger variants, 2-d U(1) and 4-d SU(3).
//
// One thread owns one d-dim site and walks a chunk of s slices with a sliding
// window: psi_{s+1}(x) is loaded once and reused for slice s+1, so every
// spinor is read from HBM once per apply; the Wilson neighbours psi_s(x +- mu)
// of the same slice are shared between threads through L1/L2.  The links of
// the site are loaded once per s-chunk and reused on every slice (they do not
// depend on s).  The s-hops P_+ psi_{s-1} and P_- psi_{s+1} are a component
// select in the chiral basis (gamma_5 diagonal), fused into the same pass.
#include "common.cuh"
#include "fine_kernels.cuh"

namespace dwf {

// ----------------------------------------------------------------------------
// 2-d U(1): spinor = 2 complex components (chirality +, -)
// ----------------------------------------------------------------------------
template <class R> struct Sp2 { typename cplx<R>::T c0, c1; };

__device__ __forceinline__ Sp2<float> ld_sp(const Sp2<float>* p, long long i) {
    float4 v = __ldg(reinterpret_cast<const float4*>(p) + i);
    Sp2<float> s; s.c0 = make_float2(v.x, v.y); s.c1 = make_float2(v.z, v.w); return s;
}
__device__ __forceinline__ Sp2<double> ld_sp(const Sp2<double>* p, long long i) {
    const double2* q = reinterpret_cast<const double2*>(p) + 2 * i;
    Sp2<double> s; s.c0 = __ldg(q); s.c1 = __ldg(q + 1); return s;
}
__device__ __forceinline__ void st_sp(Sp2<float>* p, long long i, const Sp2<float>& s) {
    reinterpret_cast<float4*>(p)[i] = make_float4(s.c0.x, s.c0.y, s.c1.x, s.c1.y);
}
__device__ __forceinline__ void st_sp(Sp2<double>* p, long long i, const Sp2<double>& s) {
    double2* q = reinterpret_cast<double2*>(p) + 2 * i;
    q[0] = s.c0; q[1] = s.c1;
}
// one chirality component of a spinor: comp 0 = P_+, comp 1 = P_-
template <class R>
__device__ __forceinline__ typename cplx<R>::T ld_comp(const Sp2<R>* p, long long i, int comp) {
    const typename cplx<R>::T* q = reinterpret_cast<const typename cplx<R>::T*>(p) + 2 * i + comp;
    return __ldg(q);
}

// Wilson hopping term -1/2 sum_mu [ (1 -+ gamma_mu) U psi(x+mu) + (1 +- gamma_mu) U^dag psi(x-mu) ]
// (upper signs: D_W; lower: D_W^dag = gamma_5 D_W gamma_5).
template <class R, bool DAG>
__device__ __forceinline__ Sp2<R> hop2d(const Sp2<R>& xf, const Sp2<R>& xb, const Sp2<R>& yf, const Sp2<R>& yb,
                                        typename cplx<R>::T u0f, typename cplx<R>::T u0b,
                                        typename cplx<R>::T u1f, typename cplx<R>::T u1b) {
    using C = typename cplx<R>::T;
    C s0, s1;
    if (!DAG) {
        C t0f = cmul(u0f, xf.c0 - xf.c1);               // (1 - g1): (h, -h)
        C t0b = cmulc(u0b, xb.c0 + xb.c1);              // (1 + g1): (h,  h)
        C t1f = cmul(u1f, yf.c0 + times_i(yf.c1));     // (1 - g2): (h, -i h)
        C t1b = cmulc(u1b, yb.c0 - times_i(yb.c1));     // (1 + g2): (h,  i h)
        s0 = t0f + t0b + t1f + t1b;
        s1 = (t0b - t0f) + times_i(t1b - t1f);
    } else {
        C t0f = cmul(u0f, xf.c0 + xf.c1);               // (1 + g1): (h,  h)
        C t0b = cmulc(u0b, xb.c0 - xb.c1);              // (1 - g1): (h, -h)
        C t1f = cmul(u1f, yf.c0 - times_i(yf.c1));      // (1 + g2): (h,  i h)
        C t1b = cmulc(u1b, yb.c0 + times_i(yb.c1));     // (1 - g2): (h, -i h)
        s0 = t0f + t0b + t1f + t1b;
        s1 = (t0f - t0b) + times_i(t1f - t1b);
    }
    Sp2<R> o;
    o.c0 = scale(s0, R(-0.5));
    o.c1 = scale(s1, R(-0.5));
    return o;
}

// streaming (evict-first) store of an output spinor: the output is not read
// again by this kernel, so it should not displace input planes from L2
__device__ __forceinline__ void st_sp_cs(Sp2<float>* p, long long i, const Sp2<float>& s) {
    __stcs(reinterpret_cast<float4*>(p) + i, make_float4(s.c0.x, s.c0.y, s.c1.x, s.c1.y));
}
__device__ __forceinline__ void st_sp_cs(Sp2<double>* p, long long i, const Sp2<double>& s) {
    double2* q = reinterpret_cast<double2*>(p) + 2 * i;
    __stcs(q, s.c0);
    __stcs(q + 1, s.c1);
}

// PF = prefetch depth of the s-window: while slice s is computed, the loads of
// psi_{s+1} .. psi_{s+PF} at this site are already in flight.
// One site, slices [s0, s1): the body shared by the single-lattice kernel and
// the batched (many right-hand sides, mixed lattices) kernel.
template <class LT, class R, bool DAG, int PF>
__device__ __forceinline__ void dwf2d_site(const typename LT::store* __restrict__ U, const Sp2<R>* __restrict__ psi,
                                           Sp2<R>* __restrict__ out, const Fine2dParams& p, long long site, int s0,
                                           int s1) {
    using C = typename cplx<R>::T;
    const long long V = p.V;
    const int Lx = p.L0;
    const int x = (int)(site % Lx);
    const long long yrow = site - x;  // y * Lx
    const int Ls = p.Ls;

    // neighbour sites with periodic wrap
    const long long xf_site = (x == Lx - 1) ? yrow : site + 1;
    const long long xb_site = (x == 0) ? yrow + Lx - 1 : site - 1;
    const long long yf_site = (site + Lx >= V) ? site + Lx - V : site + Lx;
    const long long yb_site = (site - Lx < 0) ? site - Lx + V : site - Lx;

    // links, loaded once for all s (antiperiodic boundaries flip the hop sign)
    C u0f = load_link(U, site);
    C u1f = load_link(U, V + site);
    C u0b = load_link(U, xb_site);
    C u1b = load_link(U, V + yb_site);
    if (p.anti0) {
        if (x == Lx - 1) u0f = scale(u0f, R(-1));
        if (x == 0) u0b = scale(u0b, R(-1));
    }
    if (p.anti1) {
        if (site + Lx >= V) u1f = scale(u1f, R(-1));
        if (site - Lx < 0) u1b = scale(u1b, R(-1));
    }
    const R diag = R(p.diag);
    const R mf = R(p.mf);
    // component fed from below (s-1) and from above (s+1):
    //   D:     out.c0 += psi_{s-1}.c0, out.c1 += psi_{s+1}.c1
    //   D^dag: out.c0 += psi_{s+1}.c0, out.c1 += psi_{s-1}.c1
    const int cb = DAG ? 1 : 0;   // component taken from s-1
    const int ca = DAG ? 0 : 1;   // component taken from s+1
    const int slast = s1 < Ls ? s1 : Ls - 1;   // last plane the window needs

    // win[0] = psi_s, win[k] = psi_{s+k} (loads in flight)
    Sp2<R> win[PF + 1];
#pragma unroll
    for (int k = 0; k <= PF; ++k)
        if (s0 + k <= slast) win[k] = ld_sp(psi, (long long)(s0 + k) * V + site);
    C below = (s0 > 0) ? ld_comp(psi, (long long)(s0 - 1) * V + site, cb)
                       : scale(ld_comp(psi, (long long)(Ls - 1) * V + site, cb), -mf);
    C wall0 = (s0 == 0) ? (ca == 0 ? win[0].c0 : win[0].c1) : C();

    for (int s = s0; s < s1; ++s) {
        const long long base = (long long)s * V;
        C above;
        if (s + 1 < Ls) {
            above = (ca == 0) ? win[1].c0 : win[1].c1;
        } else {
            C w = (s0 == 0) ? wall0 : ld_comp(psi, site, ca);
            above = scale(w, -mf);
        }
        Sp2<R> nb_xf = ld_sp(psi, base + xf_site);
        Sp2<R> nb_xb = ld_sp(psi, base + xb_site);
        Sp2<R> nb_yf = ld_sp(psi, base + yf_site);
        Sp2<R> nb_yb = ld_sp(psi, base + yb_site);
        const Sp2<R> cur = win[0];
        // advance the window and start the load of psi_{s+PF+1}
#pragma unroll
        for (int k = 0; k < PF; ++k) win[k] = win[k + 1];
        if (s + PF + 1 <= slast) win[PF] = ld_sp(psi, (long long)(s + PF + 1) * V + site);
        // L2 prefetch two planes beyond the window, one lane per 128-byte line:
        // more bytes in flight without the registers of a deeper window
        if (s + PF + 3 <= slast && (threadIdx.x & (128 / sizeof(Sp2<R>) - 1)) == 0)
            asm volatile("prefetch.global.L2 [%0];" ::"l"(psi + (long long)(s + PF + 3) * V + site));
        Sp2<R> o = hop2d<R, DAG>(nb_xf, nb_xb, nb_yf, nb_yb, u0f, u0b, u1f, u1b);
        o.c0 = o.c0 + scale(cur.c0, diag);
        o.c1 = o.c1 + scale(cur.c1, diag);
        if (cb == 0) { o.c0 = o.c0 + below; o.c1 = o.c1 + above; }
        else         { o.c1 = o.c1 + below; o.c0 = o.c0 + above; }
        st_sp_cs(out, base + site, o);
        below = (cb == 0) ? cur.c0 : cur.c1;
    }
}

template <class LT, class R, bool DAG, int PF>
__global__ void __launch_bounds__(256)
k_dwf2d(const typename LT::store* __restrict__ U, const Sp2<R>* __restrict__ psi, Sp2<R>* __restrict__ out,
        Fine2dParams p) {
    const long long site = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (site >= p.V) return;
    const int s0 = p.s_base + blockIdx.y * p.s_chunk;
    if (s0 >= p.s_end) return;
    dwf2d_site<LT, R, DAG, PF>(U, psi, out, p, site, s0, min(s0 + p.s_chunk, p.s_end));
}

// nrhs right-hand sides on the same lattice and links, stored back to back
// (stride V * Ls spinors): grid.z walks the right-hand sides; skip[r] != 0
// (device flags, may be null) leaves right-hand side r untouched.
template <class LT, class R, bool DAG>
__global__ void __launch_bounds__(256)
k_dwf2d_multi(const typename LT::store* __restrict__ U, const Sp2<R>* __restrict__ psi, Sp2<R>* __restrict__ out,
              Fine2dParams p, const int* __restrict__ skip) {
    const int r = blockIdx.z;
    if (skip && skip[r]) return;
    const long long site = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (site >= p.V) return;
    const int s0 = blockIdx.y * p.s_chunk;
    if (s0 >= p.Ls) return;
    const long long off = (long long)r * p.V * p.Ls;
    dwf2d_site<LT, R, DAG, 1>(U, psi + off, out + off, p, site, s0, min(s0 + p.s_chunk, p.Ls));
}

template <class LT, class R>
static void launch2d_multi(const void* U, const void* psi, void* out, const Fine2dParams& p, int nrhs,
                           const int* skip, bool dagger, cudaStream_t st) {
    dim3 grid((unsigned)((p.V + 255) / 256), (unsigned)((p.Ls + p.s_chunk - 1) / p.s_chunk), (unsigned)nrhs);
    auto Ut = reinterpret_cast<const typename LT::store*>(U);
    auto pi = reinterpret_cast<const Sp2<R>*>(psi);
    auto po = reinterpret_cast<Sp2<R>*>(out);
    if (dagger) k_dwf2d_multi<LT, R, true><<<grid, 256, 0, st>>>(Ut, pi, po, p, skip);
    else        k_dwf2d_multi<LT, R, false><<<grid, 256, 0, st>>>(Ut, pi, po, p, skip);
}

// Many right-hand sides on possibly different lattices in one launch: virtual
// block vb of the concatenated block ranges maps to (right-hand side r, block
// within r) through the descriptors' block offsets (binary search).
template <class LT, class R, bool DAG>
__global__ void __launch_bounds__(256, 4)
k_dwf2d_batched(const __grid_constant__ BatchArgs2d a) {
    for (long long vb = blockIdx.x; vb < a.total_blocks; vb += gridDim.x) {
        int lo = 0, hi = a.nrhs - 1;                              // last r with block0 <= vb
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (a.d[mid].block0 <= vb) lo = mid; else hi = mid - 1;
        }
        const BatchDesc2d& q = a.d[lo];
        const long long site = (vb - q.block0) * blockDim.x + threadIdx.x;
        if (site < q.p.V)
            dwf2d_site<LT, R, DAG, 1>(reinterpret_cast<const typename LT::store*>(q.U),
                                      reinterpret_cast<const Sp2<R>*>(q.psi), reinterpret_cast<Sp2<R>*>(q.out), q.p,
                                      site, 0, q.p.Ls);
    }
}

template <class LT, class R>
static void launch2d_batched(const BatchArgs2d& a, int grid, bool dagger, cudaStream_t st) {
    if (dagger) k_dwf2d_batched<LT, R, true><<<grid, 256, 0, st>>>(a);
    else        k_dwf2d_batched<LT, R, false><<<grid, 256, 0, st>>>(a);
}

dwf_status fine_apply_2d_batched(const BatchArgs2d& a, bool dagger, int prec, cudaStream_t st) {
    // one block per 256-site range of every right-hand side, all in one launch:
    // like the single-lattice apply, many short blocks hide the s-walk latency
    // better than a few persistent ones (measured: 608 persistent blocks reached
    // 24% of HBM on the 64-source batch)
    long long g = a.total_blocks < (1LL << 31) - 1 ? a.total_blocks : (1LL << 31) - 1;
    const int grid = (int)(g < 1 ? 1 : g);
    switch (prec) {
        case DWF_F64:       launch2d_batched<LinkF64, double>(a, grid, dagger, st); break;
        case DWF_F32:       launch2d_batched<LinkF32, float>(a, grid, dagger, st); break;
        case DWF_F32_L16:   launch2d_batched<LinkH16, float>(a, grid, dagger, st); break;
        case DWF_F32_LBF16: launch2d_batched<LinkBF16, float>(a, grid, dagger, st); break;
        default: set_error("bad precision %d", prec); return DWF_ERR_ARG;
    }
    DWF_CHECK_LAUNCH();
    return DWF_OK;
}

dwf_status fine_apply_2d_range(const Geom& g, const void* U, const void* psi, void* out, double M5, double mf,
                               bool dagger, int prec, int s_lo, int s_hi, cudaStream_t st, int s_chunk);

template <class LT, class R>
static void launch2d(const void* U, const void* psi, void* out, const Fine2dParams& p, bool dagger,
                     cudaStream_t st) {
    const int threads = 256;
    dim3 grid((unsigned)((p.V + threads - 1) / threads),
              (unsigned)((p.s_end - p.s_base + p.s_chunk - 1) / p.s_chunk));
    auto Ut = reinterpret_cast<const typename LT::store*>(U);
    auto pi = reinterpret_cast<const Sp2<R>*>(psi);
    auto po = reinterpret_cast<Sp2<R>*>(out);
    // one plane of look-ahead: measured best on GB300 (deeper windows lower the
    // achieved bandwidth); full-Ls chunks unless the lattice is small
    constexpr int PF = 1;
    if (dagger) k_dwf2d<LT, R, true, PF><<<grid, threads, 0, st>>>(Ut, pi, po, p);
    else        k_dwf2d<LT, R, false, PF><<<grid, threads, 0, st>>>(Ut, pi, po, p);
}

int choose_s_chunk(long long V, int Ls) {
    // enough threads to fill 152 SMs x 2048 threads several times over; a
    // longer chunk keeps more of the s-window reuse (fewer boundary re-reads)
    const long long target = 152LL * 2048LL * 2LL;
    long long nchunks = (target + V - 1) / V;
    if (nchunks < 1) nchunks = 1;
    if (nchunks > Ls) nchunks = Ls;
    int chunk = (int)((Ls + nchunks - 1) / nchunks);
    return chunk < 1 ? 1 : chunk;
}

dwf_status fine_apply_2d(const Geom& g, const void* U, const void* psi, void* out, double M5, double mf,
                         bool dagger, int prec, int s_chunk, cudaStream_t st) {
    return fine_apply_2d_range(g, U, psi, out, M5, mf, dagger, prec, 0, g.Ls, st, s_chunk);
}

dwf_status fine_apply_2d_range(const Geom& g, const void* U, const void* psi, void* out, double M5, double mf,
                               bool dagger, int prec, int s_lo, int s_hi, cudaStream_t st) {
    return fine_apply_2d_range(g, U, psi, out, M5, mf, dagger, prec, s_lo, s_hi, st, 0);
}

dwf_status fine_apply_2d_range(const Geom& g, const void* U, const void* psi, void* out, double M5, double mf,
                               bool dagger, int prec, int s_lo, int s_hi, cudaStream_t st, int s_chunk) {
    if (s_lo < 0 || s_hi > g.Ls || s_lo >= s_hi) { set_error("bad slice range [%d, %d)", s_lo, s_hi); return DWF_ERR_ARG; }
    Fine2dParams p;
    p.s_base = s_lo;
    p.s_end = s_hi;
    p.V = g.V;
    p.L0 = g.L[0];
    p.L1 = g.L[1];
    p.Ls = g.Ls;
    p.anti0 = g.anti[0];
    p.anti1 = g.anti[1];
    p.diag = (double)g.nd - M5 + 1.0;
    p.mf = mf;
    p.s_chunk = s_chunk > 0 ? s_chunk : choose_s_chunk(g.V, s_hi - s_lo);
    switch (prec) {
        case DWF_F64:      launch2d<LinkF64, double>(U, psi, out, p, dagger, st); break;
        case DWF_F32:      launch2d<LinkF32, float>(U, psi, out, p, dagger, st); break;
        case DWF_F32_L16:  launch2d<LinkH16, float>(U, psi, out, p, dagger, st); break;
        case DWF_F32_LBF16: launch2d<LinkBF16, float>(U, psi, out, p, dagger, st); break;
        default: set_error("bad precision %d", prec); return DWF_ERR_ARG;
    }
    DWF_CHECK_LAUNCH();
    return DWF_OK;
}

dwf_status fine_apply_2d_multi(const Geom& g, const void* U, const void* psi, void* out, double M5, double mf,
                               bool dagger, int prec, int nrhs, const int* skip, cudaStream_t st) {
    if (g.nd != 2) { set_error("multi-right-hand-side fine apply: 2-d lattices only"); return DWF_ERR_UNSUPPORTED; }
    if (nrhs < 1 || nrhs > 65535) { set_error("nrhs must be in [1, 65535]"); return DWF_ERR_ARG; }
    Fine2dParams p;
    p.V = g.V;
    p.L0 = g.L[0];
    p.L1 = g.L[1];
    p.Ls = g.Ls;
    p.anti0 = g.anti[0];
    p.anti1 = g.anti[1];
    p.diag = (double)g.nd - M5 + 1.0;
    p.mf = mf;
    p.s_chunk = choose_s_chunk(g.V * nrhs, g.Ls);
    p.s_base = 0;
    p.s_end = g.Ls;
    switch (prec) {
        case DWF_F64:       launch2d_multi<LinkF64, double>(U, psi, out, p, nrhs, skip, dagger, st); break;
        case DWF_F32:       launch2d_multi<LinkF32, float>(U, psi, out, p, nrhs, skip, dagger, st); break;
        case DWF_F32_L16:   launch2d_multi<LinkH16, float>(U, psi, out, p, nrhs, skip, dagger, st); break;
        case DWF_F32_LBF16: launch2d_multi<LinkBF16, float>(U, psi, out, p, nrhs, skip, dagger, st); break;
        default: set_error("bad precision %d", prec); return DWF_ERR_ARG;
    }
    DWF_CHECK_LAUNCH();
    return DWF_OK;
}

}  // namespace dwf
