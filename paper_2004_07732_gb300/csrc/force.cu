// Differentiation of x = D_DW^-1 b with respect to the links: U(1) link
// angles (2-d), and for any group the complex link gradient and (SU(3)) the
// force projected onto the algebra.
//
// For a real loss L(x) with upstream gradient g = dL/dRe x + i dL/dIm x, the
// adjoint solution lambda = D_DW^-dag g gives dL/db = lambda and
//   dL/dtheta_mu(y) = -Re( lambda^dag (dD_DW / dtheta_mu(y)) x ).
// Only the Wilson hops of D_W (Sec. 2) depend on U_mu(y) = exp(i theta_mu(y)),
// on every s slice: the forward hop -1/2 (1 - gamma_mu) U_mu(y) (row y, column
// y + mu) differentiates to -1/2 (1 - gamma_mu) i U_mu(y), the backward hop
// -1/2 (1 + gamma_mu) U_mu(y)^* (row y + mu, column y) to
// -1/2 (1 + gamma_mu) (-i) U_mu(y)^*.
//
// The adjoint solve uses Gamma_5 = gamma_5 R (Sec. 2.1): D^dag = Gamma_5 D Gamma_5,
// so D^-dag g = Gamma_5 D^-1 Gamma_5 g and any forward solver serves.
#include "common.cuh"
#include "fine_kernels.cuh"

namespace dwf {

__global__ void k_links_from_angles(const double* __restrict__ th, double2* __restrict__ U, long long n) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        double sn, cs;
        sincos(th[i], &sn, &cs);
        U[i] = make_double2(cs, sn);
    }
}

// out_s = gamma_5 in_{Ls-1-s}; chirality - components change sign.
template <class C>
__global__ void k_gamma5_reflect(const C* __restrict__ in, C* __restrict__ out, long long V, int Ls, int dof,
                                 int half) {
    const long long n = V * Ls * dof;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
        const int d = (int)(t % dof);
        const long long rest = t / dof;
        const long long x = rest % V;
        const int s = (int)(rest / V);
        C v = in[((long long)(Ls - 1 - s) * V + x) * dof + d];
        if (d >= half) { v.x = -v.x; v.y = -v.y; }
        out[t] = v;
    }
}

// conj(a) . M . b for a 2x2 spin matrix M = (1 + sgn gamma_mu) (2-d basis)
__device__ __forceinline__ double2 bilinear(double2 a0, double2 a1, double2 b0, double2 b1, int mu, int sgn) {
    // M b
    double2 m0, m1;
    if (mu == 0) {           // gamma_1 = sigma_1
        m0 = make_double2(b0.x + sgn * b1.x, b0.y + sgn * b1.y);
        m1 = make_double2(b1.x + sgn * b0.x, b1.y + sgn * b0.y);
    } else {                 // gamma_2 = sigma_2 = [[0,-i],[i,0]]
        m0 = make_double2(b0.x + sgn * b1.y, b0.y - sgn * b1.x);   // b0 - i sgn b1
        m1 = make_double2(b1.x - sgn * b0.y, b1.y + sgn * b0.x);   // b1 + i sgn b0
    }
    return make_double2(a0.x * m0.x + a0.y * m0.y + a1.x * m1.x + a1.y * m1.y,
                        a0.x * m0.y - a0.y * m0.x + a1.x * m1.y - a1.y * m1.x);
}

__global__ void k_force_u1_2d(const double2* __restrict__ U, const double2* __restrict__ lam,
                              const double2* __restrict__ x, double* __restrict__ F, int L0, long long V, int Ls,
                              int anti0, int anti1) {
    const long long site = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (site >= V) return;
    const int x0 = (int)(site % L0);
    for (int mu = 0; mu < 2; ++mu) {
        long long nb;
        bool cross;
        if (mu == 0) { cross = (x0 == L0 - 1); nb = cross ? site - (L0 - 1) : site + 1; }
        else         { cross = (site + L0 >= V); nb = cross ? site + L0 - V : site + L0; }
        const double ph = (cross && (mu == 0 ? anti0 : anti1)) ? -1.0 : 1.0;
        const double2 u = U[mu * V + site];
        double2 acc1 = make_double2(0.0, 0.0), acc2 = make_double2(0.0, 0.0);
        for (int s = 0; s < Ls; ++s) {
            const long long b = (long long)s * V;
            const double2* l0 = lam + 2 * (b + site);
            const double2* xn = x + 2 * (b + nb);
            const double2* ln = lam + 2 * (b + nb);
            const double2* x0p = x + 2 * (b + site);
            // lambda(site)^dag (1 - gamma_mu) x(site + mu)
            double2 t1 = bilinear(l0[0], l0[1], xn[0], xn[1], mu, -1);
            // lambda(site + mu)^dag (1 + gamma_mu) x(site)
            double2 t2 = bilinear(ln[0], ln[1], x0p[0], x0p[1], mu, +1);
            acc1.x += t1.x; acc1.y += t1.y;
            acc2.x += t2.x; acc2.y += t2.y;
        }
        // -1/2 * i U * acc1  +  -1/2 * (-i) conj(U) * acc2, real part
        const double2 iu = make_double2(-u.y, u.x);                 // i U
        const double2 miuc = make_double2(-u.y, -u.x);              // -i conj(U)
        const double r1 = iu.x * acc1.x - iu.y * acc1.y;
        const double r2 = miuc.x * acc2.x - miuc.y * acc2.y;
        F[mu * V + site] = -0.5 * ph * (r1 + r2);
    }
}

// Complex link gradient of the 2-d U(1) hops: G_mu(y) with
// Re(lam^dag dD x) = Re(conj(G) dU) for any change dU of U_mu(y) (the backward
// hop reads conj(U)): G = -1/2 ph [ conj(lam(y)^dag (1 - gamma_mu) x(y + mu))
//                                 + lam(y + mu)^dag (1 + gamma_mu) x(y) ], summed over s.
__global__ void k_linkgrad_u1_2d(const double2* __restrict__ lam, const double2* __restrict__ x,
                                 double2* __restrict__ G, int L0, long long V, int Ls, int anti0, int anti1) {
    const long long site = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (site >= V) return;
    const int x0 = (int)(site % L0);
    for (int mu = 0; mu < 2; ++mu) {
        long long nb;
        bool cross;
        if (mu == 0) { cross = (x0 == L0 - 1); nb = cross ? site - (L0 - 1) : site + 1; }
        else         { cross = (site + L0 >= V); nb = cross ? site + L0 - V : site + L0; }
        const double ph = (cross && (mu == 0 ? anti0 : anti1)) ? -1.0 : 1.0;
        double2 acc = make_double2(0.0, 0.0);
        for (int s = 0; s < Ls; ++s) {
            const long long b = (long long)s * V;
            const double2* l0 = lam + 2 * (b + site);
            const double2* xn = x + 2 * (b + nb);
            const double2* ln = lam + 2 * (b + nb);
            const double2* x0p = x + 2 * (b + site);
            const double2 t1 = bilinear(l0[0], l0[1], xn[0], xn[1], mu, -1);
            const double2 t2 = bilinear(ln[0], ln[1], x0p[0], x0p[1], mu, +1);
            acc.x += t1.x + t2.x;
            acc.y += -t1.y + t2.y;
        }
        G[mu * V + site] = make_double2(-0.5 * ph * acc.x, -0.5 * ph * acc.y);
    }
}

// gamma_mu[a][b] of the 4-d chiral basis: [[0, A_mu], [A_mu^dag, 0]] with
// A_mu = -i sigma_1, -i sigma_2, -i sigma_3, 1 (the basis of the fine operator)
__device__ __forceinline__ double2 amat64(int mu, int r, int c) {
    if (mu == 0) return r != c ? make_double2(0.0, -1.0) : make_double2(0.0, 0.0);
    if (mu == 1) return (r == 0 && c == 1) ? make_double2(-1.0, 0.0)
                        : (r == 1 && c == 0) ? make_double2(1.0, 0.0) : make_double2(0.0, 0.0);
    if (mu == 2) return r != c ? make_double2(0.0, 0.0) : make_double2(0.0, r == 0 ? -1.0 : 1.0);
    return r == c ? make_double2(1.0, 0.0) : make_double2(0.0, 0.0);
}
__device__ __forceinline__ double2 gamma64(int mu, int a, int b) {
    if (a < 2 && b >= 2) return amat64(mu, a, b - 2);
    if (a >= 2 && b < 2) { const double2 A = amat64(mu, b, a - 2); return make_double2(A.x, -A.y); }
    return make_double2(0.0, 0.0);
}

// y = (1 + sgn gamma_mu) v on one site's 4 x 3 spinor
__device__ __forceinline__ void spin_proj4(const double2* __restrict__ v, int mu, double sgn, double2 (&y)[12]) {
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            double2 acc = v[a * 3 + c];
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                const double2 gm = gamma64(mu, a, b);
                if (gm.x == 0.0 && gm.y == 0.0) continue;
                const double2 w = v[b * 3 + c];
                acc.x += sgn * (gm.x * w.x - gm.y * w.y);
                acc.y += sgn * (gm.x * w.y + gm.y * w.x);
            }
            y[a * 3 + c] = acc;
        }
}

// 4-d SU(3) link gradient G_mu(y) (3 x 3): Re(lam^dag dD x) = Re sum_ij conj(G_ij) dU_ij for any change
// dU of U_mu(y): G = -1/2 ph [ sum_a lam_a(y) y_a^dag + sum_a z_a lam_a(y + mu)^dag ], summed over s,
// with y = (1 - gamma_mu) x(y + mu), z = (1 + gamma_mu) x(y) (colour outer products over the spins a).
// FORCE: the su(3) projection F = Pi(i U G^dag) (traceless Hermitian part), for which
// Re(lam^dag dD x) = tr(H F) under U -> exp(i eps H) U.
template <bool FORCE>
__global__ void k_linkgrad_su3(const double2* __restrict__ U, const double2* __restrict__ lam,
                               const double2* __restrict__ x, double2* __restrict__ out, int4 L, long long V, int Ls,
                               int4 anti) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 4 * V) return;
    const int mu = (int)(t / V);
    const long long site = t % V;
    const int Lm = mu == 0 ? L.x : mu == 1 ? L.y : mu == 2 ? L.z : L.w;
    const long long stride = mu == 0 ? 1 : mu == 1 ? (long long)L.x : mu == 2 ? (long long)L.x * L.y
                                                                              : (long long)L.x * L.y * L.z;
    const int c = (int)((site / stride) % Lm);
    const bool cross = c == Lm - 1;
    const long long nb = cross ? site - (long long)(Lm - 1) * stride : site + stride;
    const int am = mu == 0 ? anti.x : mu == 1 ? anti.y : mu == 2 ? anti.z : anti.w;
    const double ph = (cross && am) ? -1.0 : 1.0;
    double2 G[9];
#pragma unroll
    for (int e = 0; e < 9; ++e) G[e] = make_double2(0.0, 0.0);
    for (int s = 0; s < Ls; ++s) {
        const long long b = (long long)s * V;
        double2 y[12], z[12];
        spin_proj4(x + 12 * (b + nb), mu, -1.0, y);
        spin_proj4(x + 12 * (b + site), mu, +1.0, z);
        const double2* l0 = lam + 12 * (b + site);
        const double2* ln = lam + 12 * (b + nb);
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int i = 0; i < 3; ++i)
#pragma unroll
                for (int j = 0; j < 3; ++j) {
                    const double2 li = l0[a * 3 + i], yj = y[a * 3 + j];      // lam_i conj(y_j)
                    const double2 zi = z[a * 3 + i], mj = ln[a * 3 + j];      // z_i conj(lam'_j)
                    G[i * 3 + j].x += li.x * yj.x + li.y * yj.y + zi.x * mj.x + zi.y * mj.y;
                    G[i * 3 + j].y += li.y * yj.x - li.x * yj.y + zi.y * mj.x - zi.x * mj.y;
                }
    }
#pragma unroll
    for (int e = 0; e < 9; ++e) G[e] = make_double2(-0.5 * ph * G[e].x, -0.5 * ph * G[e].y);
    double2* o = out + 9 * t;
    if (!FORCE) {
#pragma unroll
        for (int e = 0; e < 9; ++e) o[e] = G[e];
        return;
    }
    // A = i U G^dag; F = (A + A^dag) / 2 - tr / 3
    const double2* u = U + 9 * t;
    double2 A[9];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            double re = 0.0, im = 0.0;       // sum_k U_ik conj(G_jk)
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const double2 a = u[i * 3 + k], g = G[j * 3 + k];
                re += a.x * g.x + a.y * g.y;
                im += a.y * g.x - a.x * g.y;
            }
            A[i * 3 + j] = make_double2(-im, re);    // times i
        }
    const double tr = (A[0].x + A[4].x + A[8].x) / 3.0;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const double2 a = A[i * 3 + j], b = A[j * 3 + i];
            double2 f = make_double2(0.5 * (a.x + b.x), 0.5 * (a.y - b.y));
            if (i == j) f.x -= tr;
            o[i * 3 + j] = f;
        }
}

}  // namespace dwf

using namespace dwf;

extern "C" {

dwf_status dwf_links_from_angles(const dwf_geom* g, const double* theta, void* U_out, void* stream) {
    clear_error();
    Geom G;
    DWF_TRY(check_geom(g, &G));
    if (G.group != DWF_U1) { set_error("link angles apply to U(1) only"); return DWF_ERR_ARG; }
    const long long n = link_len(G);
    if (n == 0) return DWF_OK;
    if (!theta || !U_out) { set_error("NULL device pointer"); return DWF_ERR_ARG; }
    const int grid = (int)((n + 255) / 256 < 152 * 16 ? (n + 255) / 256 : 152 * 16);
    k_links_from_angles<<<grid, 256, 0, as_stream(stream)>>>(theta, (double2*)U_out, n);
    DWF_CHECK_LAUNCH();
    return DWF_OK;
}

dwf_status dwf_gamma5_reflect(const dwf_geom* g, const void* in, void* out, int prec, void* stream) {
    clear_error();
    Geom G;
    DWF_TRY(check_geom(g, &G));
    if (!valid_prec(prec)) { set_error("bad precision %d", prec); return DWF_ERR_ARG; }
    const long long n = spinor_len(G);
    if (n == 0) return DWF_OK;
    if (!in || !out) { set_error("NULL device pointer"); return DWF_ERR_ARG; }
    if (in == out) { set_error("in and out must be distinct buffers"); return DWF_ERR_ARG; }
    const int dof = (int)site_dof(G);
    const int half = dof / 2;
    const int grid = (int)((n + 255) / 256 < 152 * 16 ? (n + 255) / 256 : 152 * 16);
    cudaStream_t st = as_stream(stream);
    if (prec == DWF_F64) k_gamma5_reflect<double2><<<grid, 256, 0, st>>>((const double2*)in, (double2*)out, G.V, G.Ls, dof, half);
    else                 k_gamma5_reflect<float2><<<grid, 256, 0, st>>>((const float2*)in, (float2*)out, G.V, G.Ls, dof, half);
    DWF_CHECK_LAUNCH();
    return DWF_OK;
}

dwf_status dwf_link_force(const dwf_geom* g, const void* U, const void* lam, const void* x, double* force,
                          void* stream) {
    clear_error();
    Geom G;
    DWF_TRY(check_geom(g, &G));
    if (G.V == 0) return DWF_OK;
    if (!U || !lam || !x || !force) { set_error("NULL device pointer"); return DWF_ERR_ARG; }
    const int thr = 256;
    cudaStream_t st = as_stream(stream);
    if (G.nd == 2 && G.group == DWF_U1) {
        k_force_u1_2d<<<(unsigned)((G.V + thr - 1) / thr), thr, 0, st>>>(
            (const double2*)U, (const double2*)lam, (const double2*)x, force, G.L[0], G.V, G.Ls, G.anti[0], G.anti[1]);
    } else if (G.nd == 4 && G.group == DWF_SU3) {
        k_linkgrad_su3<true><<<(unsigned)((4 * G.V + thr - 1) / thr), thr, 0, st>>>(
            (const double2*)U, (const double2*)lam, (const double2*)x, (double2*)force,
            make_int4(G.L[0], G.L[1], G.L[2], G.L[3]), G.V, G.Ls, make_int4(G.anti[0], G.anti[1], G.anti[2], G.anti[3]));
    } else {
        set_error("the link force is built for 2-d U(1) and 4-d SU(3)");
        return DWF_ERR_UNSUPPORTED;
    }
    DWF_CHECK_LAUNCH();
    return DWF_OK;
}

dwf_status dwf_link_grad(const dwf_geom* g, const void* lam, const void* x, void* grad, void* stream) {
    clear_error();
    Geom G;
    DWF_TRY(check_geom(g, &G));
    if (G.V == 0) return DWF_OK;
    if (!lam || !x || !grad) { set_error("NULL device pointer"); return DWF_ERR_ARG; }
    const int thr = 256;
    cudaStream_t st = as_stream(stream);
    if (G.nd == 2 && G.group == DWF_U1) {
        k_linkgrad_u1_2d<<<(unsigned)((G.V + thr - 1) / thr), thr, 0, st>>>(
            (const double2*)lam, (const double2*)x, (double2*)grad, G.L[0], G.V, G.Ls, G.anti[0], G.anti[1]);
    } else if (G.nd == 4 && G.group == DWF_SU3) {
        k_linkgrad_su3<false><<<(unsigned)((4 * G.V + thr - 1) / thr), thr, 0, st>>>(
            nullptr, (const double2*)lam, (const double2*)x, (double2*)grad,
            make_int4(G.L[0], G.L[1], G.L[2], G.L[3]), G.V, G.Ls, make_int4(G.anti[0], G.anti[1], G.anti[2], G.anti[3]));
    } else {
        set_error("the link gradient is built for 2-d U(1) and 4-d SU(3)");
        return DWF_ERR_UNSUPPORTED;
    }
    DWF_CHECK_LAUNCH();
    return DWF_OK;
}

}  // extern "C"
