/*
 * dwf.h -- C ABI of the GB300 domain-wall multigrid library (libdwfmg.so).
 *
 * The operations follow Brower, Clark, Howarth, Weinberg, "Multigrid for
 * chiral lattice fermions: domain wall" (arXiv:2004.07732).  Every pointer
 * argument named U, psi, out, b, x is a DEVICE pointer owned by the caller;
 * the library never frees caller memory.  All calls are ordered on the CUDA
 * stream passed as `stream` (a cudaStream_t; NULL = the legacy default
 * stream).  Applies are asynchronous; solvers synchronise the stream only to
 * read convergence scalars.  Nothing is thrown across the ABI: every call
 * returns a dwf_status and leaves a thread-local message for dwf_last_error().
 *
 * Canonical layouts (complex numbers interleaved re, im; x0 fastest):
 *   5-d spinor  psi[s][x_{nd-1}]...[x_0][spin][color], s = 0..Ls-1
 *               (2 spins x 1 color for 2-d U(1); 4 spins x 3 colors for 4-d SU(3))
 *   gauge links U[mu][x_{nd-1}]...[x_0]          (U(1): one complex number)
 *               U[mu][x_{nd-1}]...[x_0][a][b]    (SU(3): 3x3 complex, row-major)
 * gamma basis: d = 2: gamma_1 = sigma_1, gamma_2 = sigma_2, gamma_5 = sigma_3;
 *              d = 4: chiral basis, gamma_5 = diag(1, 1, -1, -1).
 * P_+ = (1 + gamma_5)/2 therefore selects spin 0 (d = 2) or spins 0, 1 (d = 4).
 *
 * Mass convention: M5 is the domain-wall height (> 0).  The Wilson kernel is
 * the paper's D_W(M5_paper) with M5_paper = -M5, i.e. diagonal d - M5.
 */
#ifndef DWF_H
#define DWF_H

#include <stddef.h>

#if defined(__GNUC__)
#define DWF_API __attribute__((visibility("default")))
#else
#define DWF_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    DWF_OK = 0,
    DWF_ERR_ARG = 1,        /* invalid geometry, pointer, size or parameter     */
    DWF_ERR_CUDA = 2,       /* a CUDA call failed (message has the CUDA error)  */
    DWF_ERR_NOCONV = 3,     /* solver hit its iteration cap; x = last iterate   */
    DWF_ERR_TIMEOUT = 4,    /* a bounded device-side wait gave up               */
    DWF_ERR_OOM = 5,        /* a library-owned allocation failed                */
    DWF_ERR_UNSUPPORTED = 6 /* valid request outside what this build implements */
} dwf_status;

/* Arithmetic / storage precision of an operator application.
 * F64:      complex128 spinors and links, FP64 arithmetic.
 * F32:      complex64 spinors and links, FP32 arithmetic.
 * F32_L16:  complex64 spinors, links stored as IEEE half pairs (re, im), FP32 arithmetic.
 * F32_LBF16: complex64 spinors, links stored as bfloat16 pairs, FP32 arithmetic. */
typedef enum { DWF_F64 = 0, DWF_F32 = 1, DWF_F32_L16 = 2, DWF_F32_LBF16 = 3 } dwf_prec;

typedef enum { DWF_U1 = 1, DWF_SU3 = 3 } dwf_group;

/* Lattice geometry.  nd = 2 (group U(1)) or nd = 4 (group SU(3)); L[mu] >= 1
 * for mu < nd; Ls >= 1.  antiperiodic[mu] != 0 puts a factor -1 on hops that
 * cross the mu boundary (periodic otherwise). */
typedef struct {
    int nd;
    int L[4];
    int Ls;
    int group;
    int antiperiodic[4];
} dwf_geom;

/* Message of the last failed call on this thread ("" if none). */
DWF_API const char* dwf_last_error(void);

/* Number of complex values of a 5-d spinor / of the link field of geometry g. */
DWF_API size_t dwf_spinor_size(const dwf_geom* g);
DWF_API size_t dwf_link_size(const dwf_geom* g);

/* Convert FP64 links (complex128, canonical layout) to the link storage of
 * `prec` (complex128 copy, complex64, half pairs or bfloat16 pairs, rounded to
 * nearest even).  U_out must hold dwf_link_size(g) values of that format. */
DWF_API dwf_status dwf_convert_links(const dwf_geom* g, const void* U64, void* U_out, int prec, void* stream);

/* out = D_DW(mf) psi, or D_DW(mf)^dag psi if dagger != 0.
 * Shamir operator of Eq. DWoperator (Sec. 2): diagonal blocks D_W(-M5) + 1,
 * block (s, s+1) = P_-, block (s+1, s) = P_+, block (1, Ls) = -mf P_+,
 * block (Ls, 1) = -mf P_-, with the Wilson kernel
 * D_W(U, m)_{x,y} = -1/2 (1-gamma_mu) U_mu(x) delta_{x+mu,y}
 *                  -1/2 (1+gamma_mu) U_mu(x-mu)^dag delta_{x-mu,y} + (d+m) delta_{x,y}.
 * psi and out hold dwf_spinor_size(g) complex values (complex128 for F64,
 * complex64 otherwise); U is in the link storage of `prec`.  psi and out must
 * not overlap.  Returns DWF_ERR_ARG on a bad geometry or NULL pointer with a
 * non-empty lattice; an empty lattice is a no-op. */
DWF_API dwf_status dwf_apply(const dwf_geom* g, const void* U, const void* psi, void* out,
                     double M5, double mf, int dagger, int prec, void* stream);

/* D_DW(mf) psi (or its adjoint) for spinors that live in host memory (2-d).
 * psi_host / out_host: host spinors in the canonical layout (pinned memory
 * lets the copies overlap); U_host: links already in the storage of `prec`
 * (as dwf_convert_links writes them).  U_dev, psi_dev, out_dev: caller-owned
 * device buffers of the link and spinor sizes, used as staging.  The copy in,
 * the apply and the copy back are pipelined over `nchunks` ranges of s-slices
 * (<= 0: 4) on library streams; the call is ordered on `stream`: out_host is
 * complete once `stream` reaches this point.  Same errors as dwf_apply;
 * DWF_ERR_UNSUPPORTED for 4-d lattices.  Calls from several host threads on
 * one device are serialised. */
DWF_API dwf_status dwf_apply_host(const dwf_geom* g, const void* U_host, const void* psi_host, void* out_host,
                                  void* U_dev, void* psi_dev, void* out_dev, double M5, double mf, int dagger,
                                  int prec, int nchunks, void* stream);

/* Batched apply: out_r = D_DW(mf) psi_r (or the adjoint) for nrhs right-hand
 * sides, each on its own 2-d U(1) lattice geoms[r] with links U[r] (pointers may
 * repeat), all in ONE kernel launch over the concatenated site ranges (one
 * thread block per range of sites of one right-hand side).  geoms, U, psi, out are HOST arrays of nrhs entries (the latter three
 * holding device pointers).  Operator, layouts and precisions as dwf_apply.
 * nrhs <= 256.  (The paper treats one system at a time; this is the
 * many-right-hand-side form of the same operator.) */
DWF_API dwf_status dwf_apply_batched(int nrhs, const dwf_geom* geoms, const void* const* U, const void* const* psi,
                                     void* const* out, double M5, double mf, int dagger, int prec, void* stream);

/* out = D_PV psi (or D_PV^dag psi): the Pauli-Villars operator D_PV = D_DW(1)
 * (Sec. 2.2).  Same arguments and layouts as dwf_apply. */
DWF_API dwf_status pv_apply(const dwf_geom* g, const void* U, const void* psi, void* out,
                    double M5, int dagger, int prec, void* stream);

/* out = D_PV^dag D_DW(mf) psi, the approximately PV-preconditioned operator of
 * Eq. NormalExp (Sec. 2.3).  `tmp` is caller-owned device scratch of
 * dwf_spinor_size(g) complex values in the precision of `prec`; it receives
 * D_DW(mf) psi.  psi, tmp and out must be three distinct buffers. */
DWF_API dwf_status dwf_pvdag_apply(const dwf_geom* g, const void* U, const void* psi, void* tmp, void* out,
                           double M5, double mf, int prec, void* stream);

/* out = D_PV^dag D_DW(mf) psi, like dwf_pvdag_apply but without any allocation
 * and without a caller scratch buffer.  The paper has no counterpart: this is
 * for callers that cannot allocate device memory (a host code whose own
 * allocator has reserved nearly all of HBM, or a latency-critical loop that
 * cannot take cudaMalloc's implicit synchronisation).  The intermediate
 * D_DW psi lives in a fixed 16 MiB device array inside the library, resident on
 * every GPU that loads it until the process exits; lattices whose spinor needs
 * more than 16 MiB (2^20 complex128 or 2^21 complex64 values) return
 * DWF_ERR_ARG.  All calls on a device share that array: calls that overlap on
 * the GPU race and must be ordered on one stream.  The first call on each device
 * looks up the array's address (cudaGetSymbolAddress); make it before any
 * stream capture.  The address is cached per device ordinal for the life of
 * the process, so do not call this entry point on a device after
 * cudaDeviceReset.  Arguments as dwf_pvdag_apply without `tmp`. */
DWF_API dwf_status dwf_pvdag_apply_noalloc(const dwf_geom* g, const void* U, const void* psi, void* out,
                                   double M5, double mf, int prec, void* stream);

/* out = D_M(mf) psi (dagger != 0: D_M(mf)^dag psi), the Mobius domain wall
 * operator, the generalisation of the Shamir form the paper's method carries
 * over to (its conclusions: each factor of the DW / PV factorisation is linear
 * in the Wilson kernel).  In the sign convention of Eq. DWoperator:
 *   D_M = (1_s x D_W(-M5)) (b5 - c5 H_s) + 1 + H_s,
 * H_s = the fifth-dimension hops of Eq. DWoperator (P_- on (s, s+1), P_+ on
 * (s+1, s), -mf P_+ on (1, Ls), -mf P_- on (Ls, 1)); b5 = 1, c5 = 0 is dwf_apply
 * exactly.  Its effective operator is the overlap operator of the Mobius kernel
 * gamma_5 (b5 + c5) D_W (2 + (b5 - c5) D_W)^-1.  tmp: caller-owned scratch of one
 * spinor (unused when b5 = 1, c5 = 0); psi, out, tmp distinct.  Layouts,
 * precisions and errors as dwf_apply; 2-d and 4-d. */
DWF_API dwf_status dwf_mobius_apply(const dwf_geom* g, const void* U, const void* psi, void* out, void* tmp,
                                    double M5, double mf, double b5, double c5, int dagger, int prec, void* stream);

/* out = D_PV^dag p(D_PV D_PV^dag) D(mf) psi with p(y) = sum_k coeffs[k] y^k
 * (ncoef in [1, 64], host array): the Pauli-Villars preconditioned operator
 * with [D_PV D_PV^dag]^-1 approximated by a polynomial (Sec. 2.3 and App. A);
 * coeffs = {1} is dwf_pvdag_apply's D_PV^dag D_DW, {2, -1} the next order.  D is
 * the Mobius operator of (b5, c5) (Shamir for 1, 0) and D_PV = D(1).  tmp:
 * caller-owned scratch of four spinors, not overlapping psi or out.  Horner's
 * scheme: 2 (ncoef - 1) + 2 operator applications. */
DWF_API dwf_status dwf_pv_poly_apply(const dwf_geom* g, const void* U, const void* psi, void* out, void* tmp,
                                     double M5, double mf, double b5, double c5, const double* coeffs, int ncoef,
                                     int prec, void* stream);

/* Packed (slice-paired) layout of 4-d SU(3) fields (FP32 spinors, even Ls), a
 * private alternative to the canonical layout with the same operator (Eq.
 * DWoperator, Sec. 2).  Sites are taken in blocks of 32 consecutive canonical
 * site indices (NB = ceil(V / 32) blocks; sites past V pad the last block) and
 * slices in pairs (2j, 2j+1).  For pair j, block b and complex element k of a
 * site (spin-major, colour fastest, k < 12) a plane of 32 float4 holds, for
 * site 32 b + i, (Re psi_2j[k], Im psi_2j[k], Re psi_2j+1[k], Im psi_2j+1[k]) at
 * float4 index ((j NB + b) 12 + k) 32 + i: every real operation of the hop
 * then runs as one packed FP32 instruction over the two slices, and a warp
 * reads each element of 32 neighbour spinors as one contiguous run.  Complex
 * values stay (re, im) pairs, so a packed spinor is a permutation of the complex
 * values of the canonical one (plus zero padding) and complex BLAS (dwf_dot)
 * applies to it unchanged.  A link
 * block holds nine planes of 32 entries: entry e = 3 row + column of
 * U_mu(site) at ((mu NB + site / 32) 9 + e) 32 + site % 32, in the storage of
 * `prec` (complex64, half pairs or bfloat16 pairs).  4-d lattices with even Ls
 * only (DWF_ERR_UNSUPPORTED otherwise).  Sizes are in complex values (0 for a
 * bad, 2-d or odd-Ls geometry). */
DWF_API size_t dwf_packed_spinor_size(const dwf_geom* g);
DWF_API size_t dwf_packed_link_size(const dwf_geom* g);

/* FP64 canonical links -> packed links in the storage of prec (F32, F32_L16
 * or F32_LBF16), rounded to nearest even; entries of padding sites are 0. */
DWF_API dwf_status dwf_pack_links(const dwf_geom* g, const void* U64, void* U_packed, int prec, void* stream);

/* FP32 canonical spinor (dwf_spinor_size complex64) -> packed spinor
 * (dwf_packed_spinor_size complex64; padding sites written as 0), and back.
 * Buffers are 16-byte aligned and distinct. */
DWF_API dwf_status dwf_pack_spinor(const dwf_geom* g, const void* psi, void* packed, void* stream);
DWF_API dwf_status dwf_unpack_spinor(const dwf_geom* g, const void* packed, void* psi, void* stream);

/* out = D_DW(mf) psi (dagger != 0: D_DW(mf)^dag psi) with psi, out and U in
 * the packed layout; the same operator as dwf_apply.  prec is F32, F32_L16 or
 * F32_LBF16 and must match the links' storage.  Padding sites of out are not
 * written.  psi and out are distinct, 16-byte aligned buffers. */
DWF_API dwf_status dwf_apply_packed(const dwf_geom* g, const void* U_packed, const void* psi, void* out,
                                    double M5, double mf, int dagger, int prec, void* stream);

/* Inner product <x, y> = sum conj(x_i) y_i over n complex values (complex128
 * if prec == DWF_F64, complex64 otherwise), accumulated in FP64 by a
 * warp-shuffle / block / grid reduction with a fixed summation order (the
 * result is bitwise reproducible run to run).  result_host receives
 * {re, im}; the call synchronises `stream`. */
DWF_API dwf_status dwf_dot(const void* x, const void* y, size_t n, int prec, double* result_host, void* stream);

/* Solver statistics (Sec. 3 counts D_DW, D_DW^dag and D_PV^dag as one fine
 * application each). */
typedef struct {
    int iterations;            /* CGNR iterations, or outer GCR iterations of mg_solve */
    int restarts;              /* reliable updates / restart cycles                    */
    long long fine_applies;    /* fine-operator applications                           */
    long long coarse_applies;  /* coarse-operator applications                         */
    double coarse_avg_iters;   /* average coarsest-solver iterations per cycle          */
    double true_residual;      /* final ||b - D_DW x|| / ||b||, recomputed in FP64     */
    double seconds;            /* wall time of the call                                 */
    double coarsest_avg_iters; /* three-level hierarchies: average coarsest-level CGNR
                                  iterations per coarsest solve (coarse_avg_iters is then
                                  the intermediate GCR steps per intermediate solve)   */
} dwf_solve_stats;

/* Conjugate gradient on the normal equations D_DW^dag D_DW x = D_DW^dag b
 * (CGNR, Sec. 2.1 and Fig. iterationscompare), entirely in FP64 on the GPU,
 * from x = 0.  Stops when ||b - D_DW x|| / ||b|| <= tol, confirmed on the
 * recomputed true residual.  U, b, x are complex128.  Returns DWF_ERR_NOCONV
 * after maxiter iterations (x then holds the last iterate).  stats may be NULL. */
DWF_API dwf_status cgne_solve(const dwf_geom* g, const void* U, const void* b, void* x,
                      double M5, double mf, double tol, int maxiter,
                      dwf_solve_stats* stats, void* stream);

/* BiCGStab(l) (Sleijpen & Fokkema) on the Pauli-Villars preconditioned system
 * D_PV^dag D_DW(mf) x = D_PV^dag b: the solver the paper compares with CGNR and
 * multigrid as "BiCGStab-6 on D_PV^dag D_DW" (Sec. 2.3, Sec. 3, Fig.
 * iterationscompare; convergent because spec(D_PV^dag D_DW) lies in the right
 * half plane, App. B).  U, b, x: complex128 (canonical layouts), x = 0 on
 * entry is not required (it is overwritten).  ell in [1, 8] (the paper's 6).
 * FP64 reliable updates of the true residual r = b - D_DW x surround inner
 * BiCGStab(ell) solves of D_PV^dag D_DW e = D_PV^dag r / |r| in inner_prec:
 * DWF_F64 (complex128 vectors and links), or DWF_F32 / DWF_F32_L16 /
 * DWF_F32_LBF16 (complex64 vectors, links converted to that storage by the
 * library); each inner solve reduces its residual by 1e-4 (FP32) or 1e-12
 * (FP64), or to what tol still needs.  Stops when ||b - D_DW x|| / ||b|| <= tol
 * (recomputed in FP64).  maxiter caps the BiCG steps (ell per cycle; each step
 * applies D_PV^dag D_DW twice).  Returns DWF_ERR_NOCONV (x = last iterate) at
 * the cap or when two reliable updates in a row fail to lower the residual.
 * stats (may be NULL): iterations = BiCG steps, restarts = reliable updates,
 * fine_applies = D_DW, D_PV^dag applications (Sec. 3 counting).  The work
 * vectors (2 ell + 5) are allocated stream-ordered for the call. */
DWF_API dwf_status bicgstab_solve(const dwf_geom* g, const void* U, const void* b, void* x, double M5, double mf,
                                  int ell, double tol, int maxiter, int inner_prec, dwf_solve_stats* stats,
                                  void* stream);

/* Diagnostic for failure detection (no paper counterpart): runs a kernel
 * whose bounded device wait cannot complete -- which = 0: an mbarrier that
 * expects one arrival more than it gets; which = 1: a cooperative software grid
 * barrier that expects one block more than the grid -- and returns
 * DWF_ERR_TIMEOUT once the wait has given up after `seconds` (at most 10).  This
 * is the path every device-side wait of the library takes; no fault, trap or
 * hang is involved and the context stays usable.  Synchronises `stream`. */
DWF_API dwf_status dwf_check_wait_timeout(int which, double seconds, void* stream);

/* ------------------------------------------------------------------------
 * Differentiation of x = D_DW^-1 b with respect to the links (derived from
 * the Wilson hops of Sec. 2: only they depend on U, on every s slice)
 * ------------------------------------------------------------------------ */

/* U_mu(x) = exp(i theta_mu(x)) on the GPU; theta is FP64 [mu][site], U_out
 * complex128 in the canonical link layout.  U(1) only. */
DWF_API dwf_status dwf_links_from_angles(const dwf_geom* g, const double* theta, void* U_out, void* stream);

/* out = Gamma_5 in with Gamma_5 = gamma_5 R, R_{ss'} = delta_{(s+s'-1) % Ls, 0}
 * (Sec. 2.1): out_s = gamma_5 in_{Ls+1-s} (1-based s).  D_DW^dag = Gamma_5 D_DW
 * Gamma_5, so an adjoint solve is Gamma_5 D_DW^-1 Gamma_5.  in != out. */
DWF_API dwf_status dwf_gamma5_reflect(const dwf_geom* g, const void* in, void* out, int prec, void* stream);

/* The link force of lam^dag D_DW x, FP64 (U, lam, x complex128), summed over
 * all s slices.
 * 2-d U(1), U = exp(i theta): force[mu][site] = Re( lam^dag (dD_DW /
 *   dtheta_mu(site)) x ), nd * V doubles.
 * 4-d SU(3): force[mu][site] is the traceless Hermitian 3 x 3 matrix F (complex128
 *   row-major, the link layout: 18 doubles per link) with
 *   Re( lam^dag (dD_DW / d eps) x ) = tr(H F) for the variation
 *   U_mu(site) -> exp(i eps H) U_mu(site), H traceless Hermitian: the
 *   derivative projected onto su(3).
 * With lam = D_DW^-dag g for the upstream gradient g of a real loss L,
 * dL/dtheta = -force (U(1)) and dL/d eps = -tr(H F) (SU(3)). */
DWF_API dwf_status dwf_link_force(const dwf_geom* g, const void* U, const void* lam, const void* x, double* force,
                                  void* stream);

/* The complex link gradient G of Re(lam^dag D_DW x), for 2-d U(1) and 4-d
 * SU(3): Re( lam^dag dD_DW x ) = Re sum conj(G_ij) dU_ij for any change dU of
 * the links (the backward hops read U^dag).  Per link G is the colour outer
 * product of lam and the spin-projected x along the link, summed over s:
 * G_mu(y) = -1/2 ph sum_s [ lam(y) ((1 - gamma_mu) x(y + mu))^dag
 *                         + ((1 + gamma_mu) x(y)) lam(y + mu)^dag ]
 * (ph = -1 on antiperiodic boundary-crossing links).  grad: complex128 in the
 * link layout.  With lam = D_DW^-dag g, PyTorch's gradient of L with respect
 * to U (dL/dRe U + i dL/dIm U) is -G. */
DWF_API dwf_status dwf_link_grad(const dwf_geom* g, const void* lam, const void* x, void* grad, void* stream);

/* ------------------------------------------------------------------------
 * Multigrid (Sec. 2.3, Sec. 3, Table kcycle)
 * ------------------------------------------------------------------------ */

/* Parameters of the two-level PV-preconditioned K-cycle.  Defaults
 * (dwf_mg_default_params) follow Table kcycle of the paper. */
typedef struct {
    int nvec;             /* near-null vectors before chiral doubling (8); coarse dof = 2*nvec */
    int block[4];         /* aggregate extent per direction (4, 4)                             */
    int Ls_c;             /* coarse fifth-dimension extent Lhat_s (4)                          */
    int setup_maxiter;    /* CG iterations per near-null vector (250); 0 = use the starts as is */
    double setup_tol;     /* CG residual reduction per near-null vector (1e-4)                 */
    double setup_mass;    /* Wilson mass m of the setup operator D_W(m) D_W(m)^dag             */
    int gcr_restart;      /* outer flexible GCR restart length (16)                            */
    int pre_smooth;       /* GCR pre-smoothing iterations (0)                                  */
    int post_smooth;      /* GCR post-smoothing iterations on the accumulated error (8)        */
    double coarse_tol;    /* coarse-solve relative residual tolerance: 0.25 with GCR (the
                             paper's level-2 value), 0.05 for CGNR (its coarsest level)  */
    int coarse_maxiter;   /* coarse-solve iteration cap (1024)                                 */
    int fine_prec;        /* storage of the fine links in the inner solve (DWF_F32_L16)        */
    double inner_tol;     /* floor of the residual reduction of one reliable-update cycle      */
    int max_restarts;     /* reliable-update cycles before giving up                          */
    int coarse_persistent;/* 1: the coarsest CGNR runs as one cooperative persistent launch;
                             2: the coarse GCR too (one launch per coarse solve; measured
                             slower than the graph-launched GCR at 64^2 x 4, so not the
                             default); 0: launched kernels throughout (default 1)         */
    int coarse_solver;    /* 0: CGNR on the coarse normal operator (Table kcycle, coarsest
                             level); 1: restarted GCR on Dhat_PV^dag Dhat_DW (the paper's
                             level-2 solver; valid by the right-half-plane property, App. B) */
    int coarse_restart;   /* restart length of the coarse GCR (8)                         */
    int coarse_block_prec;/* storage of the Galerkin blocks read by the coarse stencil:
                             DWF_F32 or DWF_F32_L16 (FP16 blocks, FP32 arithmetic; default) */
    int cgs_passes;       /* classical Gram-Schmidt passes per GCR step: 1 (default), or 2
                             (re-orthogonalised).  With 1, a coarse GCR step takes its
                             projections, |w'|^2, alpha and the next |r|^2 from one reduction
                             pass (the orthogonality of the basis and of r to it gives |w'|^2
                             and the next |r|^2 by Pythagoras) followed by one element-wise
                             pass; a step whose |w'|^2 falls below 1e-5 |w|^2 ends that
                             right-hand side's coarse solve                                  */
    int coarse_tc;        /* form of the many-right-hand-side coarse contraction: 0 (default) =
                             autotuned -- the first use for a given nrhs times mma.sync with 1, 2
                             and 4 column tiles per warp and, with FP16 blocks, the tcgen05 forms
                             (accumulator in tensor memory; the one with the data operand in
                             tensor memory from 64 columns, the two with both operands in shared
                             memory from 128), and keeps the fastest; 1 = the persistent
                             warp-specialised tcgen05 form wherever
                             eligible (mma.sync with 4 tiles elsewhere); 2, 3, 4 = mma.sync with
                             1, 2, 4 column tiles per warp; 5 = tcgen05 with one (site, column
                             tile) per thread block; 6 = the tcgen05 form with the data
                             operand in tensor memory wherever eligible (fixed forms, for
                             testing each one)                                                 */
    int transfer;         /* 0 (default): the truncated wall transfer of Eq. TruncProjectInterpolate;
                             1: the bulk transfer the paper compares it with (Sec. 4.1), P^dag /
                             P on every slice, which needs Ls_c = Ls                           */
    int fine_layout;      /* layout of the FP32 fine vectors inside the K-cycle: 0 (default) = the
                             slice-paired packed layout (dwf_pack_spinor) wherever it applies
                             (4-d, even Ls, V a multiple of 32), canonical elsewhere; 1 =
                             canonical always.  The caller's b and x are canonical either way. */
} dwf_mg_params;

typedef struct dwf_mg dwf_mg;

/* Fill p with the Table kcycle defaults of the paper's level 2 on the coarse
 * level: restarted GCR on Dhat_PV^dag Dhat_DW to a relative residual of 0.25
 * (coarse_solver = 1, coarse_restart 8, coarse_maxiter 1024), FP16 coarse blocks,
 * 8 post-smoothing steps, outer FGCR(16). */
DWF_API void dwf_mg_default_params(dwf_mg_params* p);

/* Set up the two-level hierarchy of Sec. 2.3 for D_DW(mf) with links U
 * (complex128, canonical layout; copied, the caller may free U afterwards).
 * null_starts: nvec Gaussian d-dim vectors (complex128, [vec][site][spin][color])
 * -- the random starts of the near-null relaxation are an input.  Steps, all on
 * the GPU in FP64: CG on D_W(m) D_W(m)^dag v = 0 from each start (Table kcycle),
 * chiral doubling P_+ v, P_- v, Gram-Schmidt per aggregate and chirality (the
 * gamma_5-preserving prolongator, Eq. gamma5), and the Galerkin kernel
 * Dhat_W = P^dag D_W(-M5) P (Sec. 2.3), stored per coarse site as the self block
 * and one block per hop direction.  Returns an owning handle in *out. */
DWF_API dwf_status mg_setup(const dwf_geom* g, const void* U, double M5, double mf, const dwf_mg_params* p,
                            const void* null_starts, dwf_mg** out, void* stream);

/* Solve D_DW(mf) x = b (complex128 b, x) with the K-cycle of Sec. 2.3:
 * FP64 reliable updates of the true residual around restarted flexible GCR on
 * D_PV^dag D_DW (FP32 spinors, fine_prec links), preconditioned by truncated
 * wall restriction (Eq. TruncProjectInterpolate), a coarse solve to coarse_tol
 * (coarse_solver = 1, the default: restarted GCR on Dhat_PV^dag Dhat_DW;
 * coarse_solver = 0: CGNR on (Dhat_PV^dag Dhat_DW)^dag (Dhat_PV^dag Dhat_DW)),
 * prolongation and post_smooth GCR iterations.  Stops when ||b - D_DW x|| / ||b|| <= tol
 * (recomputed in FP64); DWF_ERR_NOCONV after maxiter outer iterations. */
DWF_API dwf_status mg_solve(dwf_mg* h, const void* b, void* x, double tol, int maxiter, dwf_solve_stats* stats,
                            void* stream);

/* Free the handle and everything it owns. */
DWF_API void mg_destroy(dwf_mg* h);

/* DWF_OK if the hierarchy h was set up for exactly these links (complex128,
 * canonical layout, compared bitwise on the GPU), M5 and mf; DWF_ERR_ARG with
 * a message otherwise.  mg_solve always solves with the operator of mg_setup,
 * so a caller whose links may have moved since (a training step, a
 * finite-difference probe) checks here first.  The paper has no counterpart.
 * Synchronises `stream`. */
DWF_API dwf_status mg_check_operator(const dwf_mg* h, const void* U, double M5, double mf, void* stream);

/* Coarse geometry (nd, coarse L, Ls = Ls_c) and coarse dof per site (2*nvec). */
DWF_API dwf_status mg_coarse_geom(const dwf_mg* h, dwf_geom* coarse, int* ncdof);

/* Copy the FP64 prolongator, complex128 [site][chirality +,-][chirality dof][vec],
 * V * 2 * (nspin/2 * ncolor) * nvec values; or the relaxed near-null vectors
 * (complex128 [vec][site][spin][color]).  Device pointers; async on stream. */
DWF_API dwf_status mg_get_prolongator(const dwf_mg* h, void* P_out, void* stream);
DWF_API dwf_status mg_get_null_vectors(const dwf_mg* h, void* v_out, void* stream);

/* Copy the FP64 Galerkin blocks of Dhat_W = P^dag D_W(-M5) P:
 * complex128 [coarse site][dir][row][col], dir 0 = self, then +mu, -mu for
 * mu = 0..nd-1; each block is (2 nvec) x (2 nvec) over the coarse dof
 * [chirality][vec].  Block (x, +mu) couples coarse site x to x + mu. */
DWF_API dwf_status mg_get_coarse_links(const dwf_mg* h, void* Y_out, void* stream);

/* Truncated restriction / prolongation of Eq. TruncProjectInterpolate on the
 * handle's prolongator, complex64 vectors: r_fine has the fine 5-d layout,
 * r_coarse the coarse layout [s][coarse site][chirality][vec] over Ls_c slices.
 * Restriction writes Phat_- P^dag P_- r_1 on coarse slice 1 and
 * Phat_+ P^dag P_+ r_Ls on slice Ls_c (zero elsewhere); prolongation writes
 * P_- P e_1 on fine slice 1 and P_+ P e_{Ls_c} on slice Ls (zero elsewhere). */
DWF_API dwf_status mg_restrict(const dwf_mg* h, const void* r_fine, void* r_coarse, void* stream);
DWF_API dwf_status mg_prolong(const dwf_mg* h, const void* e_coarse, void* e_fine, void* stream);
/* (With transfer = 1 both act on every slice instead: P^dag r_s and P e_s.) */

/* Transfer-operator diagnostics of the paper's discussion (Sec. 4.1), for a
 * complex64 fine vector v (typically a low eigenvector of D_PV^dag D_DW) and the
 * handle's transfer (walls, or every slice with transfer = 1):
 *   mg_transfer_colinearity: out = (1 - P R) v, the local colinearity;
 *   mg_transfer_oblique:     out = (1 - P Ahat^-1 R A) v, the oblique projector,
 *     A = D_PV^dag D_DW (FP32, fine_prec links), Ahat = Dhat_PV^dag Dhat_DW, with
 *     Ahat^-1 a coarse GCR solve to relative residual tol (*iters: its steps).
 * mg_coarse_solve: that coarse solve on its own (restarted GCR(16) on Ahat e = r
 * from e = 0, complex64 coarse vectors).  All three allocate their work vectors
 * stream-ordered and synchronise; they are diagnostics, not the solver's path. */
DWF_API dwf_status mg_transfer_colinearity(dwf_mg* h, const void* v, void* out, void* stream);
DWF_API dwf_status mg_transfer_oblique(dwf_mg* h, const void* v, void* out, double tol, int* iters, void* stream);
DWF_API dwf_status mg_coarse_solve(dwf_mg* h, const void* rc, void* ec, double tol, int maxiter, int* iters,
                                   void* stream);

/* Coarse Dhat_DW(mf) (or its adjoint) of Eq. coarsenDW on complex64 coarse
 * vectors; mf = 1 gives Dhat_PV.  FP32 arithmetic on the handle's coarse block
 * storage (coarse_block_prec: FP16 blocks by default, or the FP32 copy); the
 * adjoint reads the same blocks through Dhat_W^dag = sigma_3 Dhat_W sigma_3
 * (the generic narrow-block stencil reads pre-transposed FP32 adjoint blocks). */
DWF_API dwf_status mg_coarse_apply(const dwf_mg* h, const void* in, void* out, double mf, int dagger,
                                   void* stream);

/* The same coarse operator on nrhs right-hand sides at once, on the tensor
 * cores: in / out hold nrhs coarse vectors back to back ([rhs][s][site][dof],
 * complex64).  Per coarse site the stencil is a dense contraction over the
 * nrhs * Ls_c columns, evaluated on the tensor cores with TF32 products of
 * FP32 data split into high and low parts (FP32-level accuracy) and FP32
 * accumulation: tcgen05 (accumulator in tensor memory; the data operand in
 * tensor memory or in shared memory) or mma.sync.  The blocks are the handle's
 * coarse block storage (coarse_block_prec), as for mg_coarse_apply; the
 * tcgen05 forms need FP16 blocks.  With coarse_tc = 0 the first call for a new
 * nrhs times the candidate forms (using in and out as scratch, synchronising
 * `stream`) and keeps the fastest.  2-d, 16 coarse dof. */
DWF_API dwf_status mg_coarse_apply_multi(const dwf_mg* h, int nrhs, const void* in, void* out, double mf,
                                         int dagger, void* stream);

/* Layouts of a block of nrhs coarse vectors (complex64; column c = rhs * Ls_c + s;
 * the 16 dof of one (column, coarse site) pair are contiguous):
 *   DWF_COARSE_SLICE_MAJOR  [rhs][s][site][dof]: the vectors back to back (the
 *                           layout of mg_coarse_apply_multi and of the batched
 *                           solver);
 *   DWF_COARSE_SITE_MAJOR   [site][rhs][s][dof]: all columns of one coarse site
 *                           in one contiguous run (nrhs * Ls_c * 128 bytes), so
 *                           the contraction reads each neighbour's columns as
 *                           one stream instead of one 128-byte row per column. */
enum { DWF_COARSE_SLICE_MAJOR = 0, DWF_COARSE_SITE_MAJOR = 1 };

/* mg_coarse_apply_multi on vectors in the given layout (Eq. coarsenDW, the same
 * operator and arithmetic).  The autotuner keeps one choice per (nrhs, layout).
 * in and out: distinct, 16-byte aligned device buffers of nrhs coarse vectors.
 * Errors: DWF_ERR_ARG for an unknown layout, NULL, misaligned or aliased
 * buffers or nrhs < 1; DWF_ERR_UNSUPPORTED off 2-d / 16 dof. */
DWF_API dwf_status mg_coarse_apply_multi_layout(const dwf_mg* h, int nrhs, const void* in, void* out, double mf,
                                                int dagger, int layout, void* stream);

/* The form the autotuner chose for nrhs right-hand sides: 1, 2 or 4 (mma.sync
 * with that many 8-column tiles per warp), 256 (tcgen05, one (site, column
 * tile) per thread block), 257 (persistent warp-specialised tcgen05) or 258
 * (tcgen05 with the data operand in tensor memory); 0
 * before the first tuned call for that nrhs.  _layout: the choice for vectors
 * in that layout. */
DWF_API int mg_coarse_tc_form(const dwf_mg* h, int nrhs);
DWF_API int mg_coarse_tc_form_layout(const dwf_mg* h, int nrhs, int layout);

/* Batched K-cycle: nrhs right-hand sides that share the hierarchy h (one
 * gauge field) solved together (the multi-right-hand-side form of the solve
 * of Sec. 2.3).  b and x hold nrhs complex128 fine vectors back to back; x is
 * overwritten.  Per right-hand side the iteration is mg_solve's (FP64
 * reliable updates around FP32 FGCR with the K-cycle preconditioner, stopping
 * on the FP64 true residual <= tol); every launch covers all right-hand sides,
 * the coarse operator runs as the tensor-core contraction over the
 * nrhs * Ls_c columns, and converged systems drop out of the work.  stats:
 * NULL or an array of nrhs records.  nrhs > 1 takes 2-d lattices with
 * nvec = 8; nrhs = 1 any hierarchy (mg_solve uses this path).  Returns
 * DWF_ERR_NOCONV if any right-hand side stopped above tol (x holds its last
 * iterate).  The handle keeps a workspace sized for the largest nrhs seen
 * (about (6 + 2 gcr_restart + 2 post_smooth) FP32 + 2 FP64 fine vectors per
 * right-hand side) until mg_destroy. */
DWF_API dwf_status mg_solve_batched(dwf_mg* h, int nrhs, const void* b, void* x, double tol, int maxiter,
                                    dwf_solve_stats* stats, void* stream);

/* Several hierarchies (e.g. lattices of different sizes) solved concurrently:
 * group i runs mg_solve_batched(handles[i], nrhs[i], b[i], x[i], ...) on its
 * own non-blocking stream and host thread; the call returns when every group
 * has finished.  The handles must be distinct; stats[i]: NULL or nrhs[i]
 * records (stats itself may be NULL).  Returns the first failing group's
 * status, with its index in the message. */
DWF_API dwf_status mg_solve_groups(int ngroups, dwf_mg* const* handles, const int* nrhs, const void* const* b,
                                   void* const* x, double tol, int maxiter, dwf_solve_stats* const* stats);

/* ------------------------------------------------------------------------
 * Third level and coarsest-level deflation (Sec. 3: Table kcycle, levels
 * l > 1; Table zerospacing, deflation of the coarsest level)
 * ------------------------------------------------------------------------ */

/* Parameters of the level built on the handle's coarse Wilson kernel.  The
 * defaults (dwf_mg_default_level_params) are Table kcycle's: */
typedef struct {
    int nvec;             /* near-null vectors of the coarse kernel before chiral doubling (12) */
    int block[4];         /* aggregate of coarse sites per direction (2, 2)                      */
    int Ls_c;             /* fifth-dimension extent of the new (coarsest) level (4)              */
    int setup_maxiter;    /* CG iterations per near-null vector (250)                            */
    double setup_tol;     /* CG residual reduction per near-null vector (1e-4)                   */
    double setup_mass;    /* Wilson mass m of the setup operator (0: set it to the level-1 value) */
    int gcr_maxiter;      /* flexible GCR steps of the intermediate solve (16, no restart)       */
    double tol;           /* intermediate relative residual tolerance (0.25)                     */
    int post_smooth;      /* GCR post-smoothing steps on the intermediate level (8)              */
    double coarsest_tol;  /* CGNR tolerance of the coarsest solve (0.05)                         */
    int coarsest_maxiter; /* and its iteration cap (1024)                                        */
    int n_deflate;        /* low modes of the coarsest normal operator deflated (128; 0 = none)  */
    int lanczos_steps;    /* Lanczos steps that build the deflation space (256; at least
                             2 n_deflate are taken)                                           */
    int filter_degree;    /* degree of the Chebyshev filter the Lanczos runs on (64; 0: none) */
    int coarsest_solver;  /* 0: CGNR on the normal operator (Table kcycle, default); 1: restarted
                             GCR on Dhat2_PV^dag Dhat2_DW itself (valid by the right-half-plane
                             property, App. B), same tolerance and start                      */
    int coarsest_restart; /* restart length of that GCR (8)                                    */
    int block_prec;       /* storage of the new level's Galerkin blocks for its stencil:
                             DWF_F32 (default) or DWF_F32_L16 (FP16); the arithmetic is FP32
                             either way                                                        */
} dwf_mg_level_params;

DWF_API void dwf_mg_default_level_params(dwf_mg_level_params* p);

/* Add a third level to a 2-d two-level hierarchy (mg_setup), making it the
 * paper's three-level K-cycle: mg_solve then solves the intermediate system
 * Dhat_PV^dag Dhat_DW e = r by flexible GCR (tol, gcr_maxiter), preconditioned
 * by the truncated wall restriction to the new level (Eq.
 * TruncProjectInterpolate), the coarsest solve, the prolongation and
 * post_smooth GCR steps; the coarsest solve is CGNR on the normal operator of
 * Dhat2_PV^dag Dhat2_DW to coarsest_tol, started from the deflated guess.
 * Setup, on the GPU: CG on S S^dag v = 0 with S = Dhat_W(setup_mass) =
 * Dhat_W(-M5) + (setup_mass + M5) 1 (the Galerkin image of the shifted Wilson
 * kernel) from null_starts (nvec complex128 coarse vectors [vec][site][dof], FP64);
 * chiral doubling by sigma_3 and Gram-Schmidt per aggregate (the prolongator
 * P2); Dhat2_W = P2^dag Dhat_W P2 (FP64, FP32 copy for the stencil).  Deflation
 * (n_deflate > 0): Lanczos with full reorthogonalisation from lanczos_start
 * (one complex128 coarsest vector, [s][site][dof]) on p(N), the Chebyshev
 * polynomial of degree filter_degree of the coarsest normal operator N that is
 * bounded by 1 on [a, b] and grows below a (b: an upper bound of spec N from 40
 * plain Lanczos steps; a: raised until the wanted modes lie below it, at most
 * three runs), so that the lowest modes of N are the top of spec p(N); the
 * largest n_deflate eigenvalues of the Lanczos matrix (bisection) and their
 * vectors (inverse iteration), orthonormalised, give the basis V = Q S, and the
 * Rayleigh-Ritz matrix H = V^dag N V is factorised (Cholesky): every coarsest
 * solve starts from x0 = V H^-1 V^dag A^dag r, the exact solution of the normal
 * equations on span V.  2-d, one right-hand side per solve
 * (mg_solve; mg_solve_batched with nrhs = 1).  The handle owns the level until
 * mg_destroy; DWF_ERR_ARG if it already has one. */
DWF_API dwf_status mg_add_level(dwf_mg* h, const dwf_mg_level_params* p, const void* null_starts,
                                const void* lanczos_start, void* stream);

/* The new level's lattice (nd, L, Ls = its Ls_c) and dof per site (2 nvec). */
DWF_API dwf_status mg_level_geom(const dwf_mg* h, dwf_geom* coarse, int* ncdof);

/* Copy one of the new level's FP64 setup outputs (device pointer out, async):
 * what = 0: the relaxed near-null vectors, complex128 [vec][coarse site][dof];
 * 1: the prolongator P2, complex128 [coarse site][chirality +,-][coarse dof of
 *    that chirality][vec];
 * 2: the Galerkin blocks of Dhat2_W, complex128 [site][dir][row][col] (dir as
 *    for mg_get_coarse_links). */
DWF_API dwf_status mg_level_get(const dwf_mg* h, int what, void* out, void* stream);

/* Dhat2_DW(mf) (dagger != 0: its adjoint) of Eq. coarsenDW on the new level,
 * complex64 [s][site][dof] vectors, FP32 blocks and arithmetic. */
DWF_API dwf_status mg_level_apply(const dwf_mg* h, const void* in, void* out, double mf, int dagger, void* stream);

/* Truncated restriction (coarse -> new level) and prolongation (new level ->
 * coarse) of Eq. TruncProjectInterpolate with P2 and the sigma_3 projectors,
 * complex64 vectors. */
DWF_API dwf_status mg_level_restrict(const dwf_mg* h, const void* r2, void* r3, void* stream);
DWF_API dwf_status mg_level_prolong(const dwf_mg* h, const void* e3, void* e2, void* stream);

/* The coarsest solve on its own: CGNR on A^dag A x = A^dag b, A = Dhat2_PV^dag
 * Dhat2_DW (complex64 b, x), to ||b - A x|| <= tol ||b|| or maxiter
 * iterations, from the deflated guess (deflate != 0) or from 0.  maxiter = 0
 * returns the starting guess.  *iters (may be NULL) = iterations.  Synchronises. */
DWF_API dwf_status mg_level_coarsest_solve(dwf_mg* h, const void* b, void* x, double tol, int maxiter, int deflate,
                                           int* iters, void* stream);

/* The Lanczos estimates of the lowest eigenvalues of the coarsest normal
 * operator (ascending) that set up the deflation: copies up to cap of them to
 * the host array out and returns how many there are (0 without deflation). */
DWF_API int mg_level_ritz_values(const dwf_mg* h, double* out, int cap);

/* How the deflation space was built: info[0] = vectors kept, info[1] = the
 * filter's final cut a, info[2] = its top b (the bound of spec N), info[3] =
 * filtered Lanczos runs made (the cut starts at 2e-3 b and grows fourfold, at
 * most to b / 4, until every kept mode's Rayleigh quotient lies below it). */
DWF_API dwf_status mg_level_deflation_info(const dwf_mg* h, double* info);

/* Intermediate (GCR) and coarsest (CGNR) iterations of the last intermediate
 * solve. */
DWF_API dwf_status mg_level_last_iterations(const dwf_mg* h, int* l2_iters, int* l3_iters);

#ifdef __cplusplus
}
#endif

#endif /* DWF_H */
