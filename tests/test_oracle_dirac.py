"""Pins of the oracle's fine operators against closed forms and the paper's identities.

Every check here is independent of the oracle's own assembly code: plane-wave
symbols written out from the definition, printed spectra, algebraic identities
of Sec. 2.2 and App. A/B, gauge covariance and dense brute force.
"""
import math
import os

import numpy as np
import pytest

import synth
from oracle import dirac

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rand_u1(dims, sigma, seed):
    rng = np.random.default_rng(seed)
    return synth.u1_links(synth.u1_angles(rng, dims, sigma))


def _plane_wave(dims, p, chi, Ls, ns):
    """psi_{s,x,spin} = exp(i p.x) chi_{s,spin}."""
    c = dirac.site_coords(dims)
    ph = np.exp(1j * (c @ np.asarray(p)))
    return (chi.reshape(Ls, 1, ns) * ph[None, :, None]).reshape(-1), ph


@pytest.mark.parametrize("dims,anti", [((4, 6), (0, 0)), ((6, 4), (0, 1)), ((3, 5), (1, 0))])
@pytest.mark.parametrize("M5,mf", [(1.0, 0.03), (1.3, 0.2)])
def test_free_field_plane_wave_2d(dims, anti, M5, mf):
    """U = 1: D_DW acts on exp(ipx) chi as the momentum block of Sec. 2.2 (with the i)."""
    Ls, ns = 4, 2
    U = np.ones((2, int(np.prod(dims))), dtype=complex)
    D = dirac.dwf_matrix(U, dims, Ls, M5, mf, antiperiodic=list(anti))
    rng = np.random.default_rng(7)
    for k0 in range(dims[0]):
        for k1 in (0, 1, dims[1] - 1):
            p = [2 * math.pi * (k0 + 0.5 * anti[0]) / dims[0], 2 * math.pi * (k1 + 0.5 * anti[1]) / dims[1]]
            chi = synth.gaussian_complex(rng, (Ls * ns,))
            psi, ph = _plane_wave(dims, p, chi, Ls, ns)
            got = D @ psi
            # symbol written out directly: m + sum_mu [i gamma_mu sin p + 2 sin^2(p/2)]
            s1 = np.array([[0, 1], [1, 0]]); s2 = np.array([[0, -1j], [1j, 0]])
            Dw = (-M5 + 2 * math.sin(p[0] / 2) ** 2 + 2 * math.sin(p[1] / 2) ** 2) * np.eye(2) \
                + 1j * s1 * math.sin(p[0]) + 1j * s2 * math.sin(p[1])
            B = np.zeros((Ls * 2, Ls * 2), dtype=complex)
            Pp, Pm = np.diag([1.0, 0.0]), np.diag([0.0, 1.0])
            for s in range(Ls):
                B[2 * s:2 * s + 2, 2 * s:2 * s + 2] = Dw + np.eye(2)
                if s + 1 < Ls:
                    B[2 * s:2 * s + 2, 2 * s + 2:2 * s + 4] = Pm
                    B[2 * s + 2:2 * s + 4, 2 * s:2 * s + 2] = Pp
            B[0:2, 2 * Ls - 2:] += -mf * Pp
            B[2 * Ls - 2:, 0:2] += -mf * Pm
            want, _ = _plane_wave(dims, p, B @ chi, Ls, ns)
            assert np.abs(got - want).max() < 1e-12
            # the oracle's own symbol helper agrees with the written-out block
            if not any(anti):
                assert np.abs(dirac.free_dwf_symbol(p, Ls, M5, mf, 2) - B).max() < 1e-13


def test_free_wilson_plane_wave_4d():
    """4-d Wilson kernel at U = 1 acts as m + sum [i gamma sin p + 2 sin^2(p/2)]."""
    dims = (2, 3, 2, 4)
    V = int(np.prod(dims))
    U = np.broadcast_to(np.eye(3), (4, V, 3, 3)).astype(complex)
    mass = -1.8
    D = dirac.wilson_matrix(U, dims, mass, group="su3")
    g, g5 = dirac.gammas(4)
    rng = np.random.default_rng(3)
    c = dirac.site_coords(dims)
    for trial in range(6):
        k = [rng.integers(0, L) for L in dims]
        p = [2 * math.pi * k[i] / dims[i] for i in range(4)]
        chi = synth.gaussian_complex(rng, (4, 3))
        ph = np.exp(1j * (c @ np.asarray(p)))
        psi = (ph[:, None, None] * chi[None]).reshape(-1)
        S = mass * np.eye(4, dtype=complex)
        for mu in range(4):
            S = S + 1j * g[mu] * math.sin(p[mu]) + 2 * math.sin(p[mu] / 2) ** 2 * np.eye(4)
        want = (ph[:, None, None] * (S @ chi)[None]).reshape(-1)
        assert np.abs(D @ psi - want).max() < 1e-12
    assert np.allclose(g5, np.diag([1, 1, -1, -1]))


def test_free_zero_momentum_spectrum_golden():
    """Printed free spectrum at p = 0: lambda_n = m^(1/Ls) exp(i(2n+1)pi/Ls) (Sec. 2.1)."""
    rows = [l.split() for l in open(os.path.join(GOLDEN, "free_spectrum_p0.txt")) if not l.startswith("#")]
    for Ls_s, m_s, n_s, mod_s, arg_s in rows:
        Ls, m, n = int(Ls_s), float(m_s), int(n_s)
        ev = np.linalg.eigvals(dirac.free_dwf_symbol([0.0, 0.0], Ls, 1.0, m, 2))
        target = float(mod_s) * np.exp(1j * float(arg_s))
        d = np.sort(np.abs(ev - target))
        assert d[0] < 1e-10 and d[1] < 1e-10        # once per chirality
        assert abs(abs(ev).min() - m ** (1.0 / Ls)) < 1e-12


def test_free_full_lattice_smallest_modulus():
    """Whole 4x4 free lattice: the smallest |eigenvalue| is the p = 0 value m^(1/Ls)."""
    dims, Ls, m = (4, 4), 4, 0.01
    U = np.ones((2, 16), dtype=complex)
    ev = np.linalg.eigvals(dirac.dwf_matrix(U, dims, Ls, 1.0, m).toarray())
    assert abs(np.abs(ev).min() - 0.01 ** 0.25) < 1e-10


def test_gamma5_hermiticity():
    """Gamma_5 D_DW is Hermitian, Gamma_5 = gamma_5 R (Sec. 2.1)."""
    dims, Ls = (4, 4), 4
    U = _rand_u1(dims, 0.5, 11)
    D = dirac.dwf_matrix(U, dims, Ls, 1.0, 0.05).toarray()
    G = dirac.reflection_gamma5(16, Ls, 2, 1).toarray()
    H = G @ D
    assert np.abs(H - H.conj().T).max() < 1e-13
    # and the normal operator is its square: D^dag D = (Gamma_5 D)^2
    assert np.abs(D.conj().T @ D - H @ H).max() < 1e-12


def test_gauge_covariance_u1():
    """D(U^g) (g psi) = g D(U) psi with U^g_mu(x) = g(x) U_mu(x) g(x+mu)^* (same g on all s)."""
    dims, Ls = (4, 6), 3
    V = 24
    U = _rand_u1(dims, 0.7, 5)
    rng = np.random.default_rng(9)
    gx = synth.gauge_transform_u1(rng, V)
    Ug = np.empty_like(U)
    for mu in range(2):
        fwd, _ = dirac.neighbour(dims, mu, +1)
        Ug[mu] = gx * U[mu] * np.conj(gx[fwd])
    psi = synth.gaussian_spinor(rng, dims, Ls)
    G = gx[None, :, None, None]
    lhs = dirac.dwf_apply(Ug, G * psi, dims, Ls, 1.0, 0.02)
    rhs = G * dirac.dwf_apply(U, psi, dims, Ls, 1.0, 0.02)
    assert np.abs(lhs - rhs).max() < 1e-12


def test_gauge_covariance_su3():
    dims = (2, 2, 2, 4)
    V = 32
    rng = np.random.default_rng(21)
    U = synth.su3_links(rng, dims, 0.3)
    g = synth.su3_links(rng, (V,), 1.0)[0]
    Ug = np.empty_like(U)
    for mu in range(4):
        fwd, _ = dirac.neighbour(dims, mu, +1)
        Ug[mu] = g @ U[mu] @ np.conj(np.swapaxes(g[fwd], -1, -2))
    psi = synth.gaussian_complex(rng, (V, 4, 3))
    gpsi = np.einsum("vab,vsb->vsa", g, psi)
    lhs = dirac.wilson_matrix(Ug, dims, -1.8, group="su3") @ gpsi.reshape(-1)
    rhs = np.einsum("vab,vsb->vsa", g, (dirac.wilson_matrix(U, dims, -1.8, group="su3") @ psi.reshape(-1)).reshape(V, 4, 3))
    assert np.abs(lhs - rhs.reshape(-1)).max() < 1e-12
    # unitarity of the synthetic links
    assert np.abs(U[0, 3] @ np.conj(U[0, 3]).T - np.eye(3)).max() < 1e-13


def test_pv_minus_dw_corner_structure():
    """D_PV - D_DW(m) is the dyadic U V^dag of Sec. 2.2 on the corner blocks only.

    With the literal signs of Eq. DWoperator (-m P_+ on block (1, Ls)) the
    difference is -(1-m) U V^dag; the printed Sherman-Morrison form carries
    +(1-m), a sign the operator itself does not support (a reading: the
    dyadic structure is what the identity pins).
    """
    dims, Ls, m = (4, 4), 5, 0.07
    U = _rand_u1(dims, 0.5, 2)
    Dd = dirac.dwf_matrix(U, dims, Ls, 1.0, m).toarray()
    Dp = dirac.pv_matrix(U, dims, Ls, 1.0).toarray()
    n = 32
    Pp = np.kron(np.eye(16), np.diag([1.0, 0.0]))
    Pm = np.kron(np.eye(16), np.diag([0.0, 1.0]))
    Uc = np.zeros((Ls * n, n)); Uc[:n] = Pp; Uc[-n:] = Pm
    Vr = np.zeros((n, Ls * n)); Vr[:, :n] = Pm; Vr[:, -n:] = Pp
    # the dyadic form of the paper gives the (1,Ls) and (Ls,1) corner blocks;
    # its diagonal blocks P_+P_- and P_-P_+ vanish
    assert np.abs((Dp - Dd) + (1 - m) * Uc @ Vr).max() < 1e-14


def test_kdw_block_structure_and_overlap():
    """K_DW = (D_PV P)^-1 D_DW(m) P: columns s > 1 are the identity; K_11 = D_ov (Eq. DWFmatrix)."""
    dims, Ls, m = (4, 4), 4, 0.01
    V = 16
    U = _rand_u1(dims, 0.5, 4)
    Dd = dirac.dwf_matrix(U, dims, Ls, 1.0, m).toarray()
    Dp = dirac.pv_matrix(U, dims, Ls, 1.0).toarray()
    P = dirac.chiral_permutation(V, Ls, 2, 1).toarray()
    assert np.abs(P.conj().T @ P - np.eye(P.shape[0])).max() < 1e-14
    K = np.linalg.solve(Dp @ P, Dd @ P)
    n = 2 * V
    for s in range(1, Ls):
        blk = K[:, s * n:(s + 1) * n]
        want = np.zeros_like(blk); want[s * n:(s + 1) * n] = np.eye(n)
        assert np.abs(blk - want).max() < 1e-10
    Dw = dirac.wilson_matrix(U, dims, -1.0).toarray()
    Dov = dirac.overlap_kernel_first_block(Dw, Ls, m, 2, 1, V)
    assert np.abs(K[:n, :n] - Dov).max() < 1e-10
    # the mass shift identity D_ov(m) = m + (1-m) D_ov(0) (Eq. Overlap)
    Dov0 = dirac.overlap_kernel_first_block(Dw, Ls, 0.0, 2, 1, V)
    assert np.abs(Dov - (m * np.eye(n) + (1 - m) * Dov0)).max() < 1e-12


def test_ginsparg_wilson_violation_decreases_with_Ls():
    """gamma_5 D + D gamma_5 - 2 D gamma_5 D -> 0 as Ls grows for D = D_ov(0) (Sec. 2)."""
    dims = (4, 4)
    V = 16
    U = _rand_u1(dims, 0.5, 4)
    Dw = dirac.wilson_matrix(U, dims, -1.0).toarray()
    G5 = np.kron(np.eye(V), np.diag([1.0, -1.0]))
    viol = []
    for Ls in (2, 4, 8, 16):
        D = dirac.overlap_kernel_first_block(Dw, Ls, 0.0, 2, 1, V)
        viol.append(np.linalg.norm(G5 @ D + D @ G5 - 2 * D @ G5 @ D))
    assert all(a > b for a, b in zip(viol, viol[1:]))
    assert viol[-1] < 0.1 * viol[0]


def test_right_half_plane():
    """Re spec(D_PV^dag D_DW) > 0 for m > 0 (App. B)."""
    dims, Ls = (4, 4), 4
    U = _rand_u1(dims, 0.5, 8)
    A = dirac.pvdag_dwf_matrix(U, dims, Ls, 1.0, 0.01).toarray()
    assert np.linalg.eigvals(A).real.min() > 0


def test_free_pv_normal_bounded_by_one():
    """Free field at the optimum bulk mass: D_PV^dag D_PV >= 1, with equality reached (App. A)."""
    dims, Ls = (4, 4), 4
    U = np.ones((2, 16), dtype=complex)
    Dp = dirac.pv_matrix(U, dims, Ls, 1.0).toarray()
    sv = np.linalg.svd(Dp, compute_uv=False)
    assert abs(sv.min() - 1.0) < 1e-12


def test_dense_solve_unique():
    """x = D_DW^-1 b from a dense solve satisfies the system to rounding."""
    dims, Ls = (4, 4), 4
    U = _rand_u1(dims, 0.5, 12)
    D = dirac.dwf_matrix(U, dims, Ls, 1.0, 0.01).toarray()
    b = synth.gaussian_complex(np.random.default_rng(1), (D.shape[0],))
    x = np.linalg.solve(D, b)
    assert np.linalg.norm(b - D @ x) / np.linalg.norm(b) < 1e-13


@pytest.mark.parametrize("anti", [None, [1, 1]])
@pytest.mark.parametrize("dag", [False, True])
def test_point_evaluator_matches_assembled_operator(anti, dag):
    """The per-point evaluator used for large-lattice spot checks equals the sparse operator."""
    dims, Ls = (6, 5), 4
    rng = synth.rng_for(3)
    U = synth.u1_links(synth.u1_angles(rng, dims, 0.6))
    psi = synth.gaussian_spinor(rng, dims, Ls)
    full = dirac.dwf_apply(U, psi, dims, Ls, 1.0, 0.07, dagger_=dag, antiperiodic=anti).reshape(Ls, 30, 2)
    pts = [(s, x) for s in range(Ls) for x in range(30)]
    pv = dirac.dwf_apply_points_2d(U, psi, dims, Ls, 1.0, 0.07, pts, dagger_=dag, antiperiodic=anti)
    assert np.abs(pv - np.array([full[s, x] for s, x in pts])).max() < 1e-13


@pytest.mark.parametrize("group,dims", [("u1", (5, 4)), ("su3", (2, 3, 2, 4))])
@pytest.mark.parametrize("dag", [False, True])
def test_generic_point_evaluator_matches_assembled_operator(group, dims, dag):
    Ls = 3
    rng = synth.rng_for(8)
    if group == "u1":
        U = synth.u1_links(synth.u1_angles(rng, dims, 0.6))
    else:
        U = synth.su3_links(rng, dims, 0.3)
    psi = synth.gaussian_spinor(rng, dims, Ls, group)
    V = int(np.prod(dims))
    anti = [1] + [0] * (len(dims) - 1)
    full = dirac.dwf_apply(U, psi, dims, Ls, 1.3, 0.05, dagger_=dag, group=group, antiperiodic=anti)
    full = full.reshape(Ls, V, -1)
    pts = [(s, x) for s in range(Ls) for x in range(V)]
    pv = dirac.dwf_apply_points(U, psi, dims, Ls, 1.3, 0.05, pts, group=group, dagger_=dag, antiperiodic=anti)
    assert np.abs(pv.reshape(len(pts), -1) - np.array([full[s, x] for s, x in pts])).max() < 1e-13


@pytest.mark.parametrize("b5,c5", [(1.5, 0.5), (2.0, 1.0), (1.3, 0.1)])
def test_mobius_overlap_identity_and_shamir_limit(b5, c5):
    """The Mobius form reduces to Shamir at b5 = 1, c5 = 0, and its K_DW = (D_PV P)^-1 D_M P has identity
    columns s > 1 and K_11 = (1+m)/2 - (1-m)/2 eps_Ls[X] gamma_5 with the Mobius kernel
    X = gamma_5 (b5 + c5) D_W (2 + (b5 - c5) D_W)^-1 (the Shamir identity of Eq. DWFmatrix, R6,
    with the kernel scaled as the Mobius family prescribes)."""
    dims, Ls, m = (4, 4), 4, 0.05
    V, n = 16, 32
    U = _rand_u1(dims, 0.5, 4)
    assert abs(dirac.mobius_matrix(U, dims, Ls, 1.0, m, 1.0, 0.0) - dirac.dwf_matrix(U, dims, Ls, 1.0, m)).max() == 0
    Dd = dirac.mobius_matrix(U, dims, Ls, 1.0, m, b5, c5).toarray()
    Dp = dirac.mobius_matrix(U, dims, Ls, 1.0, 1.0, b5, c5).toarray()
    P = dirac.chiral_permutation(V, Ls, 2, 1).toarray()
    K = np.linalg.solve(Dp @ P, Dd @ P)
    for s in range(1, Ls):
        want = np.zeros((Ls * n, n)); want[s * n:(s + 1) * n] = np.eye(n)
        assert np.abs(K[:, s * n:(s + 1) * n] - want).max() < 1e-10
    Dw = dirac.wilson_matrix(U, dims, -1.0).toarray()
    G5 = np.kron(np.eye(V), np.diag([1.0, -1.0]))
    I = np.eye(n)
    X = G5 @ ((b5 + c5) * Dw) @ np.linalg.inv(2 * I + (b5 - c5) * Dw)
    A = np.linalg.matrix_power(I - X, Ls)
    B = np.linalg.matrix_power(I + X, Ls)
    Dov = 0.5 * (1 + m) * I - 0.5 * (1 - m) * ((A - B) @ np.linalg.inv(A + B)) @ G5
    assert np.abs(K[:n, :n] - Dov).max() < 1e-10
    # a wrong sign of c5 breaks the identity
    Dd2 = dirac.mobius_matrix(U, dims, Ls, 1.0, m, b5, -c5).toarray()
    Dp2 = dirac.mobius_matrix(U, dims, Ls, 1.0, 1.0, b5, -c5).toarray()
    K2 = np.linalg.solve(Dp2 @ P, Dd2 @ P)
    assert np.abs(K2[:n, :n] - Dov).max() > 1e-3


def test_pv_polynomial_orders_in_the_free_field():
    """Free field at the optimal height (momentum blocks of D_PV, Ls 8): the truncations c = (1),
    (2, -1), (3, -3, 1) of D_PV^-1 = D_PV^dag [D_PV D_PV^dag]^-1 each gain two powers of p (App. A):
    the error halving p shrinks by ~4, ~16, ~64."""
    Ls = 8
    orders = [(1.0,), (2.0, -1.0), (3.0, -3.0, 1.0)]

    def err(p0, c):
        B = dirac.free_dwf_symbol((p0, 0.7 * p0), Ls, 1.0, 1.0, 2)
        N = B @ B.conj().T
        poly = sum(ck * np.linalg.matrix_power(N, k) for k, ck in enumerate(c))
        return np.linalg.norm(np.linalg.inv(B) - B.conj().T @ poly, 2)

    for k, c in enumerate(orders):
        r = err(0.1, c) / err(0.05, c)
        assert abs(r / 4 ** (k + 1) - 1) < 0.1, (c, r)


def test_pv_poly_operator_limits():
    """c = (1) is D_PV^dag D_DW; with the exact polynomial of a tiny lattice's D_PV D_PV^dag (its
    characteristic polynomial gives [D_PV D_PV^dag]^-1 exactly) the operator is D_PV^-1 D_DW."""
    dims, Ls, m = (2, 2), 2, 0.05
    U = _rand_u1(dims, 0.5, 9)
    Dd = dirac.dwf_matrix(U, dims, Ls, 1.0, m)
    Dp = dirac.pv_matrix(U, dims, Ls, 1.0)
    assert abs(dirac.pv_poly_operator(Dd, Dp, (1.0,)) - dirac.pvdag_dwf_matrix(U, dims, Ls, 1.0, m)).max() < 1e-14
    N = (Dp @ dirac.dagger(Dp)).toarray()
    ch = np.poly(N)                       # N^n + a_1 N^(n-1) + ... + a_n = 0 (Cayley-Hamilton)
    n = N.shape[0]
    # N^-1 = -(N^(n-1) + a_1 N^(n-2) + ... + a_(n-1)) / a_n
    coeffs = [-ch[n - 1 - k] / ch[n] for k in range(n - 1)] + [-1.0 / ch[n]]
    got = dirac.pv_poly_operator(Dd, Dp, coeffs).toarray()
    want = np.linalg.solve(Dp.toarray(), Dd.toarray())
    assert np.abs(got - want).max() < 1e-6 * np.abs(want).max()


@pytest.mark.parametrize("coeffs", [(1.0,), (2.0, -1.0), (3.0, -3.0, 1.0), (0.5, 0.25, -0.125, 2.0)])
def test_pv_poly_apply_is_the_operator_on_a_vector(coeffs):
    """The matrix-vector (Horner) form gives the assembled polynomial operator times the vector;
    with the Cayley-Hamilton coefficients of a tiny lattice it gives D_PV^-1 D_DW psi."""
    dims, Ls, m = (4, 4), 4, 0.05
    U = _rand_u1(dims, 0.5, 11)
    Dd = dirac.dwf_matrix(U, dims, Ls, 1.0, m)
    Dp = dirac.pv_matrix(U, dims, Ls, 1.0)
    psi = np.random.default_rng(3).standard_normal(Dd.shape[0]) * (1 + 0.5j)
    want = dirac.pv_poly_operator(Dd, Dp, coeffs) @ psi
    got = dirac.pv_poly_apply(Dd, Dp, coeffs, psi)
    assert np.linalg.norm(got - want) < 1e-13 * np.linalg.norm(want)
    dims, Ls = (2, 2), 2
    U = _rand_u1(dims, 0.5, 9)
    Dd = dirac.dwf_matrix(U, dims, Ls, 1.0, m)
    Dp = dirac.pv_matrix(U, dims, Ls, 1.0)
    N = (Dp @ dirac.dagger(Dp)).toarray()
    ch = np.poly(N)
    n = N.shape[0]
    ck = [-ch[n - 1 - k] / ch[n] for k in range(n - 1)] + [-1.0 / ch[n]]
    x = np.random.default_rng(4).standard_normal(n) + 0j
    exact = np.linalg.solve(Dp.toarray(), Dd.toarray() @ x)
    # the Cayley-Hamilton coefficients are large and alternate, so rounding in either order of the
    # products leaves ~1e-6 of the result
    assert np.linalg.norm(dirac.pv_poly_apply(Dd, Dp, ck, x) - exact) < 1e-5 * np.linalg.norm(exact)
