// Coarse-level operators of the multigrid (Sec. 2.3):
//   * the coarse Shamir operator Dhat_DW(m) of Eq. coarsenDW: on every coarse
//     slice the Galerkin kernel Dhat_W (self block + one block per hop
//     direction) plus 1, the Phat_pm = (1 pm sigma_3)/2 s-hops and the -m wall
//     terms; the adjoint uses the transposed neighbour blocks, so it is the
//     exact adjoint of the stored operator;
//   * truncated wall restriction / prolongation (Eq. TruncProjectInterpolate).
// Coarse vectors are [s][coarse site][chirality][vec], complex64.
#include "mg.cuh"

namespace dwf {

struct CoarseParams {
    long long Vc;
    int nd;
    int Lc[4];
    int Ls_c;
    int ncd, nvec, ndir;
    float mf;
};

__device__ __forceinline__ long long coarse_neighbour(const CoarseParams& p, long long xc, int dir) {
    if (dir == 0) return xc;
    const int mu = (dir - 1) / 2;
    const int step = ((dir - 1) % 2 == 0) ? 1 : -1;
    long long stride = 1;
    for (int k = 0; k < mu; ++k) stride *= p.Lc[k];
    const int c = (int)((xc / stride) % p.Lc[mu]);
    int cn = c + step;
    if (cn < 0) cn += p.Lc[mu];
    if (cn >= p.Lc[mu]) cn -= p.Lc[mu];
    return xc + (long long)(cn - c) * stride;
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

template <bool DAG>
__global__ void __launch_bounds__(256) k_coarse_dwf(const float2* __restrict__ Y, const float2* __restrict__ in,
                                                    float2* __restrict__ out, CoarseParams p, const int* skip) {
    if (skip && *skip) return;
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int ncd = p.ncd;
    const long long total = p.Vc * p.Ls_c * ncd;
    if (t >= total) return;
    const int i = (int)(t % ncd);
    const long long rest = t / ncd;
    const long long xc = rest % p.Vc;
    const int s = (int)(rest / p.Vc);
    const long long slice = p.Vc * ncd;
    const float2* ins = in + (long long)s * slice;
    float2 acc = ins[xc * ncd + i];                     // the "+1" of Dhat_W + 1
    const long long bsz = (long long)ncd * ncd;
    for (int dir = 0; dir < p.ndir; ++dir) {
        const long long nb = coarse_neighbour(p, xc, dir);
        const float2* v = ins + nb * ncd;
        if (!DAG) {
            const float2* Yb = Y + (xc * p.ndir + dir) * bsz + i;     // column-major: (i, j) at j*ncd + i
#pragma unroll 4
            for (int j = 0; j < ncd; ++j) acc = cfma(__ldg(Yb + (long long)j * ncd), v[j], acc);
        } else {
            const int opp = dir == 0 ? 0 : (((dir - 1) % 2 == 0) ? dir + 1 : dir - 1);
            const float2* Yb = Y + (nb * p.ndir + opp) * bsz + (long long)i * ncd;   // (j, i) at i*ncd + j
#pragma unroll 4
            for (int j = 0; j < ncd; ++j) acc = cfma_conj(__ldg(Yb + j), v[j], acc);
        }
    }
    const int c = i / p.nvec;
    const bool from_below = DAG ? (c == 1) : (c == 0);
    float2 h;
    if (from_below) {
        if (s > 0) h = in[(long long)(s - 1) * slice + xc * ncd + i];
        else { h = in[(long long)(p.Ls_c - 1) * slice + xc * ncd + i]; h.x *= -p.mf; h.y *= -p.mf; }
    } else {
        if (s < p.Ls_c - 1) h = in[(long long)(s + 1) * slice + xc * ncd + i];
        else { h = in[xc * ncd + i]; h.x *= -p.mf; h.y *= -p.mf; }
    }
    acc.x += h.x;
    acc.y += h.y;
    out[t] = acc;
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
    const long long total = p.Vc * p.Ls_c * p.ncd;
    const int thr = 256;
    const unsigned grid = (unsigned)((total + thr - 1) / thr);
    if (dagger) k_coarse_dwf<true><<<grid, thr, 0, st>>>(h->Y32, in, out, p, skip);
    else        k_coarse_dwf<false><<<grid, thr, 0, st>>>(h->Y32, in, out, p, skip);
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
};

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

__global__ void k_restrict(const float2* __restrict__ P, const float2* __restrict__ r, float2* __restrict__ out,
                           TransferParams p, const int* skip) {
    if (skip && *skip) return;
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long total = p.Vc * p.Ls_c * p.ncd;
    if (t >= total) return;
    const int i = (int)(t % p.ncd);
    const long long rest = t / p.ncd;
    const long long xc = rest % p.Vc;
    const int s = (int)(rest / p.Vc);
    const int c = i / p.nvec, k = i % p.nvec;
    float2 acc = make_float2(0.f, 0.f);
    int sf = -1;
    if (c == 1 && s == 0) sf = 0;                 // Phat_- P^dag P_- r_1 on coarse slice 1
    if (c == 0 && s == p.Ls_c - 1) sf = p.Ls - 1; // Phat_+ P^dag P_+ r_Ls on coarse slice Lhat_s
    if (sf >= 0) {
        const float2* rs = r + (long long)sf * p.V * p.dof;
        for (int l = 0; l < p.nb; ++l) {
            const long long x = agg_site(p, xc, l);
            for (int cd = 0; cd < p.nchd; ++cd)
                acc = cfma_conj(P[((x * 2 + c) * p.nchd + cd) * p.nvec + k], rs[x * p.dof + chir_dof(p, c, cd)], acc);
        }
    }
    out[t] = acc;
}

__global__ void k_prolong(const float2* __restrict__ P, const float2* __restrict__ e, float2* __restrict__ out,
                          TransferParams p, const int* skip) {
    if (skip && *skip) return;
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long total = p.V * p.Ls * p.dof;
    if (t >= total) return;
    const int d = (int)(t % p.dof);
    const long long rest = t / p.dof;
    const long long x = rest % p.V;
    const int s = (int)(rest / p.V);
    int c, cd;
    if (p.nd == 2) { c = d; cd = 0; }
    else { const int spin = d / p.ncol; c = spin / 2; cd = (spin % 2) * p.ncol + d % p.ncol; }
    float2 acc = make_float2(0.f, 0.f);
    int sc = -1;
    if (c == 1 && s == 0) sc = 0;                 // P_- P e_1 on fine slice 1
    if (c == 0 && s == p.Ls - 1) sc = p.Ls_c - 1; // P_+ P e_{Lhat_s} on fine slice Ls
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
    return p;
}

dwf_status restrict_wall(const dwf_mg* h, const float2* r_fine, float2* r_coarse, const int* skip, cudaStream_t st) {
    TransferParams p = transfer_params(h);
    const long long total = p.Vc * p.Ls_c * p.ncd;
    k_restrict<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(h->P32, r_fine, r_coarse, p, skip);
    DWF_CHECK_LAUNCH();
    return DWF_OK;
}

dwf_status prolong_wall(const dwf_mg* h, const float2* e_coarse, float2* e_fine, const int* skip, cudaStream_t st) {
    TransferParams p = transfer_params(h);
    const long long total = p.V * p.Ls * p.dof;
    k_prolong<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(h->P32, e_coarse, e_fine, p, skip);
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
