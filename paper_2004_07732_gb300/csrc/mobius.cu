// The Mobius domain wall operator and the polynomial Pauli-Villars correction:
// the two generalisations of the Shamir method the paper names (its conclusions:
// the DW / PV factorisation carries over to Mobius and related forms because each
// factor is a linear functional of the Wilson kernel; Sec. 2.3 and App. A: the
// PV inverse [D_PV D_PV^dag]^-1 approximated by a polynomial in D_PV D_PV^dag).
//
// Mobius, in the sign convention of Eq. DWoperator (b5 = 1, c5 = 0 is Shamir):
//   D_M = (1_s x D_W) K + S,   K = b5 - c5 H_s,   S = 1 + H_s,
// H_s the fifth-dimension hops (P_- from s + 1, P_+ from s - 1, -m on the walls).
// With the Shamir kernel D_DW = (1_s x D_W) + S the apply reuses it:
//   D_M psi     = D_DW (K psi) + (1 + H_s)(psi - K psi)
//   D_M^dag psi = K^dag w + S^dag psi,   w = D_W^dag psi = D_DW^dag psi - S^dag psi,
// each a Shamir apply plus element-wise passes that read a site's dof on
// neighbouring slices (H_s and H_s^dag act on s and chirality only).
#include "common.cuh"
#include "fine_kernels.cuh"

namespace dwf {
namespace {

struct SHop {
    long long V;      // d-dim sites
    int Ls, dof, half;   // dof per site; dof < half are chirality + (P_+)
    double mf;
};

// (H_s v)(s, x, d) (dag = false) or (H_s^dag v)(s, x, d) (dag = true); v indexed [s][x][dof]
template <class C>
__device__ __forceinline__ C hop_s(const C* __restrict__ v, const SHop& p, int s, long long xd, int d, bool dag) {
    const bool plus = d < p.half;
    // H_s: + from s - 1 (wall: -m v_{Ls-1}), - from s + 1 (wall: -m v_0); H_s^dag the mirror
    const bool from_below = plus != dag;
    int t;
    double f = 1.0;
    if (from_below) { if (s > 0) t = s - 1; else { t = p.Ls - 1; f = -p.mf; } }
    else            { if (s < p.Ls - 1) t = s + 1; else { t = 0; f = -p.mf; } }
    C a = v[(long long)t * p.V * p.dof + xd];
    a.x *= f;
    a.y *= f;
    return a;
}

#define MB_LOOP(t, n) for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < (n); t += (long long)gridDim.x * blockDim.x)

// chi = b5 psi - c5 H_s psi
template <class C>
__global__ void k_mob_chi(const C* __restrict__ psi, C* __restrict__ chi, SHop p, double b5, double c5) {
    const long long slice = p.V * p.dof, n = slice * p.Ls;
    MB_LOOP(t, n) {
        const int s = (int)(t / slice);
        const long long xd = t % slice;
        const int d = (int)(xd % p.dof);
        const C a = psi[t], h = hop_s(psi, p, s, xd, d, false);
        C o;
        o.x = b5 * a.x - c5 * h.x;
        o.y = b5 * a.y - c5 * h.y;
        chi[t] = o;
    }
}

// out += delta + H_s delta with delta = psi - chi = (1 - b5) psi + c5 H_s psi
template <class C>
__device__ __forceinline__ C mob_delta(const C* __restrict__ psi, const SHop& p, int s, long long xd, int d, double b5,
                                       double c5) {
    const C a = psi[(long long)s * p.V * p.dof + xd], h = hop_s(psi, p, s, xd, d, false);
    C o;
    o.x = (1.0 - b5) * a.x + c5 * h.x;
    o.y = (1.0 - b5) * a.y + c5 * h.y;
    return o;
}

template <class C>
__global__ void k_mob_fix(const C* __restrict__ psi, C* __restrict__ out, SHop p, double b5, double c5) {
    const long long slice = p.V * p.dof, n = slice * p.Ls;
    MB_LOOP(t, n) {
        const int s = (int)(t / slice);
        const long long xd = t % slice;
        const int d = (int)(xd % p.dof);
        const C dl = mob_delta(psi, p, s, xd, d, b5, c5);
        // H_s delta at s: delta on the neighbouring slice (or the wall), times the wall factor
        const bool plus = d < p.half;
        int t2;
        double f = 1.0;
        if (plus) { if (s > 0) t2 = s - 1; else { t2 = p.Ls - 1; f = -p.mf; } }
        else      { if (s < p.Ls - 1) t2 = s + 1; else { t2 = 0; f = -p.mf; } }
        const C dn = mob_delta(psi, p, t2, xd, d, b5, c5);
        C o = out[t];
        o.x += dl.x + f * dn.x;
        o.y += dl.y + f * dn.y;
        out[t] = o;
    }
}

// out = b5 w - c5 H_s^dag w + psi + H_s^dag psi, w = u - psi - H_s^dag psi (u = D_DW^dag psi)
template <class C>
__device__ __forceinline__ C mob_w(const C* __restrict__ u, const C* __restrict__ psi, const SHop& p, int s,
                                   long long xd, int d) {
    const long long i = (long long)s * p.V * p.dof + xd;
    const C a = u[i], b = psi[i], h = hop_s(psi, p, s, xd, d, true);
    C o;
    o.x = a.x - b.x - h.x;
    o.y = a.y - b.y - h.y;
    return o;
}

template <class C>
__global__ void k_mob_dag(const C* __restrict__ u, const C* __restrict__ psi, C* __restrict__ out, SHop p, double b5,
                          double c5) {
    const long long slice = p.V * p.dof, n = slice * p.Ls;
    MB_LOOP(t, n) {
        const int s = (int)(t / slice);
        const long long xd = t % slice;
        const int d = (int)(xd % p.dof);
        const C w = mob_w(u, psi, p, s, xd, d);
        const bool plus = d < p.half;
        int t2;
        double f = 1.0;
        if (!plus) { if (s > 0) t2 = s - 1; else { t2 = p.Ls - 1; f = -p.mf; } }    // H_s^dag: - from below
        else       { if (s < p.Ls - 1) t2 = s + 1; else { t2 = 0; f = -p.mf; } }    //          + from above
        const C wn = mob_w(u, psi, p, t2, xd, d);
        const C a = psi[t], h = hop_s(psi, p, s, xd, d, true);
        C o;
        o.x = b5 * w.x - c5 * f * wn.x + a.x + h.x;
        o.y = b5 * w.y - c5 * f * wn.y + a.y + h.y;
        out[t] = o;
    }
}

// z = c y
template <class C>
__global__ void k_poly_scale(C* __restrict__ z, const C* __restrict__ y, double c, long long n) {
    MB_LOOP(t, n) {
        const C a = y[t];
        C o;
        o.x = c * a.x;
        o.y = c * a.y;
        z[t] = o;
    }
}

// z = c y + w
template <class C>
__global__ void k_poly_axpy(C* __restrict__ z, const C* __restrict__ y, const C* __restrict__ w, double c, long long n) {
    MB_LOOP(t, n) {
        const C a = y[t], b = w[t];
        C o;
        o.x = c * a.x + b.x;
        o.y = c * a.y + b.y;
        z[t] = o;
    }
}

inline int mb_grid(long long n) {
    long long b = (n + 255) / 256;
    return (int)(b < 152LL * 16 ? b : 152LL * 16);
}

template <class C>
dwf_status mobius_impl(const Geom& G, const void* U, const void* psi, void* out, void* tmp, double M5, double mf,
                       double b5, double c5, bool dagger, int prec, cudaStream_t st) {
    SHop p;
    p.V = G.V;
    p.Ls = G.Ls;
    p.dof = (int)site_dof(G);
    p.half = p.dof / 2;
    p.mf = mf;
    const long long n = spinor_len(G);
    const int g = mb_grid(n);
    if (!dagger) {
        k_mob_chi<C><<<g, 256, 0, st>>>((const C*)psi, (C*)tmp, p, b5, c5);
        DWF_CHECK_LAUNCH();
        DWF_TRY(fine_apply(G, U, tmp, out, M5, mf, false, prec, st));
        k_mob_fix<C><<<g, 256, 0, st>>>((const C*)psi, (C*)out, p, b5, c5);
    } else {
        DWF_TRY(fine_apply(G, U, psi, tmp, M5, mf, true, prec, st));
        k_mob_dag<C><<<g, 256, 0, st>>>((const C*)tmp, (const C*)psi, (C*)out, p, b5, c5);
    }
    DWF_CHECK_LAUNCH();
    return DWF_OK;
}

dwf_status mobius_apply(const Geom& G, const void* U, const void* psi, void* out, void* tmp, double M5, double mf,
                        double b5, double c5, bool dagger, int prec, cudaStream_t st) {
    if (b5 == 1.0 && c5 == 0.0) return fine_apply(G, U, psi, out, M5, mf, dagger, prec, st);
    if (prec == DWF_F64) return mobius_impl<double2>(G, U, psi, out, tmp, M5, mf, b5, c5, dagger, prec, st);
    return mobius_impl<float2>(G, U, psi, out, tmp, M5, mf, b5, c5, dagger, prec, st);
}

dwf_status check_spinor_args(const dwf_geom* g, Geom* G, const void* U, const void* psi, const void* out, int prec) {
    DWF_TRY(check_geom(g, G));
    if (!valid_prec(prec)) { set_error("bad precision %d", prec); return DWF_ERR_ARG; }
    if (G->V == 0) return DWF_OK;
    if (!U || !psi || !out) { set_error("NULL device pointer"); return DWF_ERR_ARG; }
    if (!aligned16(psi) || !aligned16(out)) { set_error("spinor buffers must be 16-byte aligned"); return DWF_ERR_ARG; }
    if (psi == out) { set_error("psi and out must be distinct buffers"); return DWF_ERR_ARG; }
    return DWF_OK;
}

}  // namespace
}  // namespace dwf

using namespace dwf;

extern "C" dwf_status dwf_mobius_apply(const dwf_geom* g, const void* U, const void* psi, void* out, void* tmp,
                                       double M5, double mf, double b5, double c5, int dagger, int prec,
                                       void* stream) {
    clear_error();
    Geom G;
    DWF_TRY(check_spinor_args(g, &G, U, psi, out, prec));
    if (G.V == 0) return DWF_OK;
    if (!tmp || tmp == psi || tmp == out) { set_error("tmp must be a third, distinct buffer"); return DWF_ERR_ARG; }
    if (!aligned16(tmp)) { set_error("tmp must be 16-byte aligned"); return DWF_ERR_ARG; }
    return mobius_apply(G, U, psi, out, tmp, M5, mf, b5, c5, dagger != 0, prec, as_stream(stream));
}

extern "C" dwf_status dwf_pv_poly_apply(const dwf_geom* g, const void* U, const void* psi, void* out, void* tmp,
                                        double M5, double mf, double b5, double c5, const double* coeffs, int ncoef,
                                        int prec, void* stream) {
    clear_error();
    Geom G;
    DWF_TRY(check_spinor_args(g, &G, U, psi, out, prec));
    if (G.V == 0) return DWF_OK;
    if (!coeffs || ncoef < 1 || ncoef > 64) { set_error("coeffs must hold 1 to 64 values"); return DWF_ERR_ARG; }
    if (!tmp || !aligned16(tmp)) { set_error("tmp must be a 16-byte aligned buffer of four spinors"); return DWF_ERR_ARG; }
    cudaStream_t st = as_stream(stream);
    const long long n = spinor_len(G);
    const size_t eb = prec == DWF_F64 ? sizeof(double2) : sizeof(float2);
    char* base = static_cast<char*>(tmp);
    void* y = base;
    void* z = base + n * eb;
    void* t = base + 2 * n * eb;
    void* m = base + 3 * n * eb;          // the Mobius apply's own scratch
    if ((psi >= (const void*)base && psi < (const void*)(base + 4 * n * eb)) ||
        (out >= (void*)base && out < (void*)(base + 4 * n * eb))) {
        set_error("psi and out must not overlap tmp");
        return DWF_ERR_ARG;
    }
    const int grid = mb_grid(n);
    // y = D psi; z = c_{n-1} y; z = c_k y + D_PV D_PV^dag z for k = n - 2 .. 0; out = D_PV^dag z
    DWF_TRY(mobius_apply(G, U, psi, y, m, M5, mf, b5, c5, false, prec, st));
    if (prec == DWF_F64) k_poly_scale<double2><<<grid, 256, 0, st>>>((double2*)z, (const double2*)y, coeffs[ncoef - 1], n);
    else k_poly_scale<float2><<<grid, 256, 0, st>>>((float2*)z, (const float2*)y, coeffs[ncoef - 1], n);
    DWF_CHECK_LAUNCH();
    for (int k = ncoef - 2; k >= 0; --k) {
        DWF_TRY(mobius_apply(G, U, z, t, m, M5, 1.0, b5, c5, true, prec, st));
        DWF_TRY(mobius_apply(G, U, t, z, m, M5, 1.0, b5, c5, false, prec, st));
        if (prec == DWF_F64) k_poly_axpy<double2><<<grid, 256, 0, st>>>((double2*)z, (const double2*)y,
                                                                         (const double2*)z, coeffs[k], n);
        else k_poly_axpy<float2><<<grid, 256, 0, st>>>((float2*)z, (const float2*)y, (const float2*)z, coeffs[k], n);
        DWF_CHECK_LAUNCH();
    }
    return mobius_apply(G, U, z, out, m, M5, 1.0, b5, c5, true, prec, st);
}
