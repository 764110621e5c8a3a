/*
 * mgw.h -- C ABI of libmgw: the density-fitted construction of moment-
 * conserving GW self-energy moments on one GB300 (sm_103a), after
 * Backhouse, Allen, Scott & Booth, arXiv:2504.17439.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Array arguments are DEVICE pointers to row-major float64 data owned by
 *    the caller, unless a parameter says "host".  They must stay valid until
 *    the work queued on the handle's stream has completed.
 *  - Calls are stream ordered on the stream given to mgw_create (or
 *    mgw_set_stream).  Arguments are checked before anything is queued.
 *    Calls whose outputs include host scalars synchronise the stream.
 *  - The library owns its workspace (device memory inside the handle).  It
 *    grows to the largest size a call has needed and is released by
 *    mgw_destroy.  A handle is used by one host thread at a time.
 *  - Index conventions: orbitals are ordered occupied first (ascending
 *    energy) then virtual; particle-hole pairs ia are ordered i-major,
 *    a fastest (ia = i*nvir + a); moments are indexed n = 0..nmom-1.
 *  - Nothing throws across the ABI.  A failing call returns a negative
 *    mgw_status and mgw_last_error() describes it.  Numerical failures
 *    (a non positive definite matrix, a broken-down recurrence) are reported
 *    as statuses, never as a device fault.
 *
 * Notation of the paper: V_{P,ia} is the particle-hole block of the DF
 * tensor (here Lov), eta~(n) the aux-basis response moment, D_ia the
 * orbital-energy differences, Sigma(n,<)/(n,>) the hole/particle moments.
 */
#ifndef MGW_H
#define MGW_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  MGW_OK = 0,
  MGW_ERR_ARG = -1,         /* bad size, null pointer, NaN in an input scalar */
  MGW_ERR_CUDA = -2,        /* a CUDA runtime or library call failed */
  MGW_ERR_NOMEM = -3,       /* workspace allocation failed */
  MGW_ERR_NOT_PD = -4,      /* a matrix required positive definite was not */
  MGW_ERR_BREAKDOWN = -5,   /* block Lanczos lost rank it could not handle */
  MGW_ERR_NO_CONV = -6,     /* an iteration hit its cap before converging */
  MGW_ERR_TIMEOUT = -7,     /* a bounded device wait gave up */
  MGW_ERR_UNSUPPORTED = -8  /* option or size outside what is built */
} mgw_status;

typedef enum { MGW_TDA = 0, MGW_RPA = 1 } mgw_screening;

/* Arithmetic of the bulk contractions.  FP64: float64 FMA units throughout.
 * FP64_TC: the response and Sigma-build contractions on the BF16 tensor
 * cores as FP64-accurate digit-sliced products (see mgw_gemm_fp64_emu), 28
 * BF16 products per product.
 * MIXED: the DF tensor enters as a BF16 hi/lo split on one fixed-point grid:
 * L (and V for the TDA response) rounded to a multiple of 2^(e-16) where
 * max |L| < 2^(e-1), i.e. to 16 bits of the largest element, and carried as
 * two BF16 digits; the moment-carrying operands (eta~, W, Z) keep seven
 * digits, 13 BF16 products per product, each exact, their sums exact down to
 * 2^-40 of the top and in FP32 below.  Its contractions need naux <= 65536
 * (K per launch of the tensor-core kernel; longer K elsewhere is split).
 * The results are the FP64-accurate moments of the system with the rounded
 * tensor, a consistent moment sequence (no amplification by the block
 * Lanczos step): QP energies move by a few 1e-5 to 1e-4 meV at the frontier
 * and by at most about 0.06 meV elsewhere on the synthetic workloads (N = 5
 * and 7).  The RPA response takes V unrounded (as FP64_TC).
 * BF16X3 is only the standalone mgw_gemm_bf16x3 product (FP32 accumulation
 * is too coarse for the moment-to-Lanczos step, so no path uses it). */
typedef enum { MGW_FP64 = 0, MGW_BF16X3 = 1, MGW_FP64_TC = 2, MGW_MIXED = 3 } mgw_precision;

typedef struct mgw_handle mgw_handle;

typedef struct {
  int screening;     /* mgw_screening; default MGW_TDA */
  int precision;     /* mgw_precision; default MGW_FP64 */
  int nquad;         /* quadrature nodes for the RPA eta~(0) (Eqs. 24-25); default 48, even, >= 2 */
  int xchunk;        /* Green's-function indices x per pass of the Sigma build; 0 = automatic */
  double rank_tol;   /* relative eigenvalue cut for inverse square roots; default 1e-12 */
  int max_iter;      /* iteration cap of self-consistent loops; default 50 */
  double conv_e;     /* energy threshold, Ha; default 5 meV = 1.8375e-4 Ha (Sec. IV B) */
  double conv_mom;   /* max |delta Sigma(n)| threshold; default 1e-4 (Sec. IV B) */
  int diis_space;    /* DIIS vectors kept in the Fock loop; default 12 (Sec. IV B) */
  int batch_graph;   /* mgw_sigma_moments_batched: capture the whole build in a CUDA graph and
                        replay it while the problem table is unchanged; default 1 */
  int batch_autotune;/* mgw_sigma_moments_batched: time the candidate tile shapes of each grouped
                        stage on the first call for a problem table and keep the fastest; default 1 */
  int rpa_offset;    /* G_offset of the RPA eta~(0) (Eq. 25): 0 by the quadrature nodes of Eq. 24;
                        1 in closed form, V D + 4 (V D)[(V^T V) o C] with C_jb,ia = 1/(D_jb + D_ia),
                        in column blocks of V^T V (4 ov^2 naux flops against the quadrature's
                        4 nquad naux^2 ov: cheaper where ov < nquad naux); default 0 */
} mgw_options;

/* Fill *o with the defaults listed above. */
void mgw_options_default(mgw_options* o);

/* Create a handle on CUDA device `device`, queueing on `cuda_stream`
 * (a cudaStream_t, or NULL for the default stream). */
mgw_status mgw_create(mgw_handle** h, int device, void* cuda_stream);
mgw_status mgw_destroy(mgw_handle* h);
mgw_status mgw_set_stream(mgw_handle* h, void* cuda_stream);
/* Text of the last error on this handle ("" if none).  Owned by the handle. */
const char* mgw_last_error(const mgw_handle* h);
/* Bytes of device workspace the handle currently holds. */
size_t mgw_workspace_bytes(const mgw_handle* h);

/*
 * Tracing.  mgw_profile(h, 1) clears the record and starts timing every
 * GEMM-class kernel the handle launches with a pair of CUDA events on its
 * stream; mgw_profile(h, 0) stops (both synchronise).  mgw_profile_query
 * sums the recorded launches whose kernel name equals `name` ("*" for all):
 * names are "w_gemm", "t_update", "sigma_y_binomial", "sigma_gemm2",
 * "gemm_nn", "gemm_nt", "gemm_tn".  mgw_launch_count returns the number of
 * kernels of this library the handle has launched since creation (solver
 * library kernels are not counted).
 */
mgw_status mgw_profile(mgw_handle* h, int enable);
mgw_status mgw_profile_query(mgw_handle* h, const char* name, long* count, double* total_ms);
long mgw_launch_count(const mgw_handle* h);

/*
 * mgw_extract_ov -- V_{Q,ia} = L[Q][i][nocc + a]: copy the particle-hole
 * block of the DF tensor into its own array (the first of the two
 * transformed copies of Algorithm 1).
 *   L   [naux][nmo][nmo]   in
 *   Lov [naux][nocc*nvir]  out
 */
mgw_status mgw_extract_ov(mgw_handle* h, int nocc, int nvir, int naux,
                          const double* L, double* Lov);

/*
 * mgw_response_moments -- W(n) = eta~(n) V^T for n = 0..nmom-1.
 * TDA (Sec. II C, Eqs. 32-33): eta~(0) = V, eta~(n) = eta~(n-1)(D + 2 V^T V).
 * RPA (Sec. II B, Eqs. 23-30): eta~(0) by the quadrature of Eqs. 24-28 with
 *   o->nquad nodes, eta~(1) = V D, eta~(n) = eta~(n-2)(D^2 + 4 V^T V D).
 * D_ia = eps_W[nocc+a] - eps_W[i] (Eq. 20); W(n) is the naux x naux inner
 * factor of Eq. 15 (no spin factor).
 *   eps_W [nmo]                 in   orbital energies defining D
 *   Lov   [naux][nocc*nvir]     in   V
 *   Wmom  [nmom][naux][naux]    out  symmetric
 * Requires nocc, nvir, naux >= 1, 1 <= nmom <= 64, D_ia > 0 for RPA.
 * o->precision MGW_FP64_TC runs every contraction (the recursion's two
 * products per order and, for the RPA, the products of each quadrature node)
 * as FP64-accurate digit-sliced tensor-core GEMMs; the RPA's per-node
 * Cholesky solves stay on the FP64 units.
 */
mgw_status mgw_response_moments(mgw_handle* h, const mgw_options* o,
                                int nocc, int nvir, int naux, int nmom,
                                const double* eps_W, const double* Lov,
                                double* Wmom);

/*
 * mgw_sigma_moments -- hole and particle self-energy moments, Eqs. 6-7 with
 * Eq. 15, with the t-th screened moment inside the sum over t and the
 * restricted spin factor 2:
 *   Sigma(n,<)_pq = 2 sum_t C(n,t) (-1)^t sum_k eps_k^(n-t) [L_k^T W(t) L_k]_pq
 *   Sigma(n,>)_pq = 2 sum_t C(n,t)        sum_c eps_c^(n-t) [L_c^T W(t) L_c]_pq
 * where (L_x)_{P,p} = L[P][p][x].
 *   eps_G    [nmo]               in   Green's-function energies
 *   L        [naux][nmo][nmo]    in   symmetric in its last two indices
 *   Wmom     [nmom][naux][naux]  in   from mgw_response_moments
 *   sig_hole [nmom][nmo][nmo]    out
 *   sig_part [nmom][nmo][nmo]    out
 * Requires 1 <= nmom <= 24.
 */
mgw_status mgw_sigma_moments(mgw_handle* h, const mgw_options* o,
                             int nocc, int nvir, int naux, int nmom,
                             const double* eps_G, const double* L,
                             const double* Wmom,
                             double* sig_hole, double* sig_part);

/*
 * mgw_sigma_moments_x -- mgw_sigma_moments over a Green's-function space of
 * its own: x = 0..nx-1 with energies eps_x, the first nhole of them holes,
 * and Lx [naux][nx][nmo] holding L_{P,x q} in row x of slab P (for the
 * orbitals themselves nx = nmo and Lx = L).  The space of the quasi-molecular
 * orbitals of scGW / G0W (Algorithm 5), where x runs over every pole of H~.
 *   eps_x [nx], Lx [naux][nx][nmo], Wmom [nmom][naux][naux] in;
 *   sig_hole, sig_part [nmom][nmo][nmo] out.  Precisions as mgw_sigma_moments.
 */
mgw_status mgw_sigma_moments_x(mgw_handle* h, const mgw_options* o, int nmo, int nx, int nhole, int naux, int nmom,
                               const double* eps_x, const double* Lx, const double* Wmom,
                               double* sig_hole, double* sig_part);

/*
 * mgw_qmo_tensors -- the DF tensor carried to the quasi-molecular orbitals of
 * H~ (Algorithm 5, reading S1: the map is the physical rows chi_px of H~'s
 * eigenvectors), with the first m poles occupied (Eq. 40, reading S2):
 *   Lt [naux][nx][nmo], Lt[Q][x][p] = sum_q L[Q][p][q] chi[q][x]  (for mgw_sigma_moments_x)
 *   Via [naux][m][nx-m], Via[Q][i][a] = sum_p chi[p][i] Lt[Q][m+a][p]  (for mgw_response_moments)
 * L [naux][nmo][nmo] symmetric slabs, chi [nmo][nx] as written by
 * mgw_qp_solve.  FP64 GEMMs.  Via is not written when m is 0 or nx.
 */
mgw_status mgw_qmo_tensors(mgw_handle* h, int nmo, int naux, int nx, int m, const double* L, const double* chi,
                           double* Lt, double* Via);

/*
 * mgw_block_lanczos -- moment-conserving upfolding of one sector (Eqs. 9-10):
 * coupling S0^(1/2), diagonal blocks alpha_0..alpha_{nblk-1} and
 * off-diagonal blocks beta_1..beta_{nblk-1} of a block tridiagonal T with
 *   Sigma(n) = S0^(1/2) (T^n)_{00} S0^(1/2),  n = 0..2 nblk - 1,
 * nblk = nmom / 2.  Symmetric positive square roots are used for S0 and for
 * every beta, so the blocks are unique.  Moments are centred on
 * c = tr Sigma(1)/tr Sigma(0) and scaled by s = (tr M(2nblk-2)/tr M(0))^(1/(2nblk-2))
 * inside (exact in exact arithmetic).  Eigenvalues below
 * o->rank_tol * lambda_max of Sigma(0) are dropped; the retained rank r is
 * returned and, when r < nmo, the blocks are r x r in the leading corner of
 * each nmo x nmo slot (basis: retained eigenvectors of Sigma(0)).
 *   sig   [nmom][nmo][nmo]        in   one sector, symmetric
 *   coup  [nmo][nmo]              out
 *   alpha [nblk][nmo][nmo]        out
 *   beta  [nblk-1][nmo][nmo]      out  (may be NULL when nblk == 1)
 *   rank  host int                out  (synchronises)
 * Requires nmom even, 2 <= nmom <= 24.
 */
mgw_status mgw_block_lanczos(mgw_handle* h, const mgw_options* o,
                             int nmo, int nmom, const double* sig,
                             double* coup, double* alpha, double* beta,
                             int* rank);

/*
 * mgw_qp_solve -- diagonalise the upfolded Hamiltonian of Eq. 9
 *   H~ = [[fock, W~], [W~^T, d~ + zeta]],  W~ = [coup_h 0 .. | coup_p 0 ..],
 *   d~ = blockdiag(T_h, T_p),
 * block order physical | hole chain | particle chain, dim = nmo + nblk (r_h + r_p).
 * Then the QP energies of Eq. 34 (argmax of |chi_{p alpha}|^2, ties to the
 * lowest alpha), the Aufbau filling of Eq. 40 (m minimising |N(m) - nelec|,
 * ties to the smaller m, mu = (E_{m-1} + E_m)/2) and the correlated density
 * rho = 2 sum_{alpha < m} chi chi^T.
 *   fock [nmo][nmo]; coup_*, alpha_*, beta_* as written by mgw_block_lanczos
 *   (leading r x r of each nmo x nmo slot is used)              in
 *   E [dim] ascending, weight [dim] = sum_p chi_{p alpha}^2      out
 *   chi_phys [nmo][dim] (or NULL), eps_qp [nmo], rho [nmo][nmo] (or NULL)  out
 *   mu_host, nelec_host, m_host: host scalars (may be NULL)      out (synchronises)
 */
mgw_status mgw_qp_solve(mgw_handle* h, const mgw_options* o,
                        int nmo, int nblk, int rank_h, int rank_p,
                        const double* fock,
                        const double* coup_h, const double* alpha_h, const double* beta_h,
                        const double* coup_p, const double* alpha_p, const double* beta_p,
                        double zeta, double nelec,
                        double* E, double* weight, double* chi_phys,
                        double* eps_qp, double* rho,
                        double* mu_host, double* nelec_host, int* m_host);

/*
 * mgw_sigma_moments_batched -- TDA response moments and Sigma(n,<),
 * Sigma(n,>) of many independent systems of uneven size at once (the same
 * quantities as mgw_response_moments + mgw_sigma_moments per system).  Each
 * stage is one grouped launch over all systems: per moment order one launch
 * for every W_s(t) and one for every update of eta~_s; per round of
 * Green's-function index chunks one launch for every Y stage and one for
 * every GEMM2 (a CTA finds its system and tile from a prefix sum of tile
 * counts).  Not in the paper (which treats one molecule at a time).
 * With o->batch_autotune, the first call for a problem table times the
 * candidate tile shapes of each stage kind (response GEMM, update, Y stage,
 * GEMM2) on that table and keeps the fastest; with o->batch_graph the whole
 * sequence is captured once into a CUDA graph (on a stream the handle owns)
 * and later calls with the same table (sizes and pointers) and workspace
 * replay it on the handle's stream.  The graph reads the inputs' current
 * contents; it is rebuilt when the table, nmom or the workspace changes.
 * With o->precision == MGW_MIXED the stages are the same on the tensor cores:
 * one grouped launch of the mixed digit-sliced kernel per stage over all
 * systems (tensor maps and epilogue parameters per system in a device table),
 * the digit slicing between stages per system, the whole sequence captured as
 * one CUDA graph (o->batch_graph) and replayed; the rounds of Green's-function
 * indices are the fewest that fit half of the free device memory.  Results
 * as mgw_response_moments + mgw_sigma_moments under MGW_MIXED per system.
 * Needs nmom <= 16 and nocc nvir, naux <= 65536.  The call returns after the
 * work has finished (it reads the wait status).
 * With o->precision == MGW_FP64_TC each system instead runs the
 * single-system FP64-accurate tensor-core pipeline (mgw_response_moments and
 * mgw_sigma_moments), the systems spread, largest first, over four internal
 * sub-handles with streams and workspaces of their own so that small systems
 * run concurrently; the call forks from and joins back to the handle's
 * stream, and returns after the work has finished (it reads the pipelines'
 * wait status once at the end).
 *   sys: HOST array of nsys descriptors whose pointers are device pointers
 *   1 <= nmom <= 24; o->screening must be MGW_TDA.
 */
typedef struct {
  int nocc, nvir, naux;
  const double* eps;      /* [nmo]              in */
  const double* L;        /* [naux][nmo][nmo]   in */
  double* sig_hole;       /* [nmom][nmo][nmo]   out */
  double* sig_part;       /* [nmom][nmo][nmo]   out */
} mgw_system;

mgw_status mgw_sigma_moments_batched(mgw_handle* h, const mgw_options* o, int nsys, int nmom,
                                     const mgw_system* sys);

/*
 * mgw_g0w0_batched -- the whole G0W0 chain for many independent systems:
 * for each, the response moments (o->screening), the Sigma moments, block
 * Lanczos of both sectors (Eqs. 9-10) and the QP solve of mgw_qp_solve with
 * F = diag(eps) (a canonical Hartree-Fock reference, Sigma_inf = 0), zeta = 0
 * and N = 2 nocc, in o->precision.  Systems are spread, largest first, over
 * four internal sub-handles, each driven by a host thread of its own (the
 * Lanczos ranks and the QP's host scalars synchronise), so small systems
 * and the host-side decisions of one system overlap the others' GPU work;
 * each system gets exactly the result of the single-system calls.  The
 * call returns when every system is done.  Not in the paper.
 *   sys: HOST array; eps [nmo], L [naux][nmo][nmo] device in; eps_qp [nmo]
 *   device out; mu, nelec, rank_h, rank_p host out.  0 <= nmom_max <= 11.
 */
typedef struct {
  int nocc, nvir, naux;
  const double* eps;      /* [nmo]              in */
  const double* L;        /* [naux][nmo][nmo]   in */
  double* eps_qp;         /* [nmo]              out */
  double mu, nelec;       /* host out: Aufbau chemical potential and count */
  int rank_h, rank_p;     /* host out: retained ranks of the two Sigma(0) */
} mgw_g0w0_system;

mgw_status mgw_g0w0_batched(mgw_handle* h, const mgw_options* o, int nsys, int nmom_max,
                            mgw_g0w0_system* sys);

/*
 * mgw_response_moments_batched -- mgw_response_moments for many independent
 * systems, spread over the same sub-handles and host threads as
 * mgw_g0w0_batched.  Not in the paper.
 *   sys: HOST array of device pointers eps_W [nmo], Lov [naux][nocc*nvir] in,
 *   Wmom [nmom][naux][naux] out.
 */
typedef struct {
  int nocc, nvir, naux;
  const double* eps_W;
  const double* Lov;
  double* Wmom;
} mgw_response_system;

mgw_status mgw_response_moments_batched(mgw_handle* h, const mgw_options* o, int nsys, int nmom,
                                        const mgw_response_system* sys);

/*
 * mgw_sync_status -- wait for everything queued on the handle's stream and
 * report a CUDA error that any of it raised (MGW_ERR_CUDA), else MGW_OK.
 */
mgw_status mgw_sync_status(mgw_handle* h);

/*
 * mgw_fsgw_step -- one outer iteration of Fock self-consistent GW
 * (Algorithm 2, Sec. III F).  In the reference orbital basis of h and L:
 *   1. L' = C^T L C; response moments, Sigma moments and both block-Lanczos
 *      chains in the orbitals C with energies eps (o->screening, o->nquad);
 *   2. the chains' coupling is carried to the reference basis (W~ = C W~');
 *   3. zeta (the shift of d~ in Eq. 9) is chosen so that the Aufbau count of
 *      Eq. 40 meets N = 2 nocc (the root of N(zeta) - N nearest to the current
 *      zeta: outward scan in 0.01 Ha steps, Illinois regula falsi; golden
 *      section on |N(zeta) - N| over [-1, 1] Ha if no root), then F is made
 *      consistent with the correlated density, F = h + J[rho] - K[rho]/2,
 *      by a Pulay-DIIS Fock loop (space o->diis_space) at fixed zeta; the two
 *      alternate until both hold (at most 20 rounds);
 *   4. eps, C <- eigh(F), and the QP energies of Eq. 34 in that basis.
 * Start from F = diag(eps_ref), C = I, eps = eps_ref, zeta = 0 for a
 * canonical Hartree-Fock reference (h chosen so that F[rho_HF] = diag(eps)),
 * or set init = 1 to have the step first take eps, C from eigh(F).
 * Repeat until the moments and QP energies stop changing (o->conv_mom,
 * o->conv_e); the convergence test is the caller's.
 */
typedef struct {
  int nocc, nvir, naux, nmom_max; /* sizes; nmom_max <= 11 */
  const double* h;        /* [nmo][nmo]        in   core Hamiltonian, reference basis */
  const double* L;        /* [naux][nmo][nmo]  in   DF tensor, reference basis */
  double* F;              /* [nmo][nmo]        in/out Fock matrix, reference basis */
  double* C;              /* [nmo][nmo]        in/out orbitals (columns) of the last F */
  double* eps;            /* [nmo]             in/out their energies */
  double* eps_qp;         /* [nmo]             out  QP energies (Eq. 34) in the new orbitals */
  double* sigma_ref;      /* [nmom][nmo][nmo]  out  Sigma(n,<) + Sigma(n,>) in the reference basis, or NULL */
  double zeta;            /* host in/out */
  double mu, nelec;       /* host out: chemical potential and Aufbau count at the end */
  int inner_iters;        /* host out: Fock-loop iterations in this step */
  int zeta_evals;         /* host out: H~ diagonalisations spent on zeta */
  int init;               /* host in: 1 = derive eps, C from F first (cleared by the step) */
  /* learned warm start of the first zeta search of the step (not in the paper):
   * a network of the mgw_mlp_* family with d_in = MGW_WS_FEATURES, d_out = 1
   * predicts zeta - zeta_prev from ws_feat; NULL params = the plain search */
  const float* ws_params;
  const unsigned short* ws_wbf16;
  int ws_width;
  float ws_feat[8];       /* host out: the features of the first search */
  double ws_target;       /* host out: zeta found by it minus zeta_prev (a training target) */
  int ws_hit;             /* host out: 1 if the predicted bracket held the root */
  /* learned Fock-matrix proposal (not in the paper): with F_prev != NULL and
   * fock_hist = 1, the step first moves F to F + beta (F - F_prev), beta from
   * a network of the same family (d_in = MGW_WS_FEATURES, d_out = 1, input
   * wf_feat, clamped to [-0.5, 2]); the plain DIIS Fock loop then starts from
   * it (NULL wf_params: beta = 0).  At the end the step sets F_prev to its
   * own starting F and fock_hist = 1. */
  double* F_prev;         /* [nmo][nmo] in/out, or NULL: no proposal, nothing recorded */
  int fock_hist;          /* host in/out: 1 when F_prev holds the previous step's start */
  const float* wf_params;
  const unsigned short* wf_wbf16;
  int wf_width;
  float wf_feat[8];       /* host out: the proposal's features (zero without history) */
  double wf_target;       /* host in/out: least-squares beta that reaches the step's converged F
                             along F - F_prev (a training target); read as a feature next step */
  double wf_beta;         /* host out: the beta applied */
} mgw_fsgw_state;

#define MGW_WS_FEATURES 8

mgw_status mgw_fsgw_step(mgw_handle* h, const mgw_options* o, mgw_fsgw_state* st);

/*
 * mgw_hf_core -- the core Hamiltonian h = diag(eps) - J[rho] + K[rho]/2 of a
 * canonical restricted Hartree-Fock reference (rho = 2 on the first nocc
 * orbitals), i.e. the h for which the Fock build F[rho] = h + J - K/2 of the
 * fsGW loop (Algorithm 2, Sec. III F) returns diag(eps) at the reference
 * density; it prepares the inputs of mgw_fsgw_step for a system given by its
 * orbital energies and DF tensor.
 *   eps [nmo], L [naux][nmo][nmo] in; hcore [nmo][nmo] out
 */
mgw_status mgw_hf_core(mgw_handle* h, int nocc, int nmo, int naux, const double* eps, const double* L,
                       double* hcore);

/*
 * mgw_naf_compress -- natural auxiliary functions (Sec. II D, Eq. 14):
 * M_PQ = sum_vw L[P][v][w] L[Q][v][w] over every orbital pair (all_pairs != 0)
 * or over all but the virtual-virtual block (all_pairs == 0, the paper's
 * default outside self-consistency); the eigenvectors of M with eigenvalue
 * above eps_naf (an absolute threshold) define
 *   L_naf[A][p][q] = sum_P U[P][A] L[P][p][q],  A = 0..n_naf-1 in descending
 * eigenvalue order; later calls take n_naf in place of naux.  Each row is
 * fixed up to its sign (that of the eigenvector).
 *   L       [naux][nmo][nmo]   in   device, nmo = nocc + nvir
 *   L_naf   [naux][nmo][nmo]   out  device, rows 0..n_naf-1 written, the rest untouched
 *   lam     [naux]             out  device, every eigenvalue of M, descending
 *   n_naf                      out  host (the call synchronises the stream)
 * M is formed with FP64 GEMMs and diagonalised with cuSOLVER syevd.
 * Returns MGW_ERR_ARG for bad sizes or null pointers, MGW_ERR_NO_CONV if the
 * eigensolver does not converge.
 */
mgw_status mgw_naf_compress(mgw_handle* h, int nocc, int nvir, int naux, const double* L, double eps_naf,
                            int all_pairs, double* L_naf, double* lam, int* n_naf);

/*
 * mgw_spectral_function -- A(w) of Eq. 12 from the poles of H~ (Eq. 11)
 * with a Lorentzian broadening delta > 0:
 *   A[j] = (1/pi) sum_a weight[a] delta / ((omega[j] - E[a])^2 + delta^2),
 * E and weight as returned by mgw_qp_solve (weight_a = sum_p chi_pa^2).
 *   E, weight [dim], omega [nomega] in; A [nomega] out; all device, FP64.
 * Stream-ordered, no synchronisation.  Returns MGW_ERR_ARG for dim or nomega
 * below 1, delta not positive or a null pointer.
 */
mgw_status mgw_spectral_function(mgw_handle* h, int dim, const double* E, const double* weight, double delta,
                                 int nomega, const double* omega, double* A);

/*
 * mgw_qsgw_potential -- the static potential of qsGW (Sec. III D) from the
 * hole and particle chains of mgw_block_lanczos (same padded layout: coup
 * [nmo][nmo] with rank columns used, alpha [nblk][nmo][nmo], beta
 * [nblk-1][nmo][nmo] with rank x rank blocks used).  Each chain's external
 * block is diagonalised, T = U diag(e) U^T, giving couplings v = [coup, 0..] U
 * and pole energies e (pole decoupling); with D_pl = eps_p - e_l:
 *   reg 0 (Eqs. 36-37): V = (A + A^T)/2, A_pq = sum_l v_pl v_ql D_pl / (D_pl^2 + delta^2)
 *   reg 1 (Eqs. 38-39): V_pq = sum_l (D_pl + D_ql) / (D_pl^2 + D_ql^2) v_pl v_ql (1 - exp(-(D_pl^2 + D_ql^2) s))
 * The pair with D_pl = D_ql = 0 contributes 0.
 *   eps [nmo] in (the energies the chains were built with); V [nmo][nmo] out;
 *   all device, FP64.  The eigensolves (cuSOLVER syevd) synchronise the stream.
 * Returns MGW_ERR_ARG for bad sizes, reg not 0 or 1, delta <= 0 (reg 0),
 * s < 0 (reg 1) or missing blocks; MGW_ERR_NO_CONV if an eigensolve fails.
 */
mgw_status mgw_qsgw_potential(mgw_handle* h, int nmo, int nblk, int rank_h, int rank_p, const double* eps,
                              const double* coup_h, const double* alpha_h, const double* beta_h,
                              const double* coup_p, const double* alpha_p, const double* beta_p, int reg,
                              double delta, double srg_s, double* V);

/*
 * mgw_qsgw_step -- one outer iteration of quasiparticle self-consistent GW
 * (Sec. III D).  In the reference orbital basis of h and L:
 *   1. L' = C^T L C; response moments, Sigma moments and both block-Lanczos
 *      chains in the orbitals C with energies eps (o->screening, o->precision);
 *   2. the static potential of mgw_qsgw_potential in those orbitals (reg 0:
 *      Eqs. 36-37 with delta; reg 1: Eqs. 38-39 with srg_s), carried to the
 *      reference basis: V = C V' C^T (written to st->V);
 *   3. Eq. 35 with V held fixed: F = h + J[rho] - K[rho]/2 + V, rho = 2 C_occ
 *      C_occ^T over the nocc lowest orbitals of F, Pulay DIIS (space
 *      diis_space, extrapolating once three vectors are held) on the
 *      commutator F rho - rho F, until max |delta rho| < scf_tol and
 *      max |F rho - rho F| < 1e3 scf_tol (at most scf_max_iter iterations);
 *   4. eps, C <- eigh(F of the final density); de = max |eps_new - eps_old|.
 * Start from C = I, eps = the reference energies for a canonical
 * Hartree-Fock reference (h from mgw_hf_core); repeat until de is below the
 * caller's tolerance.  The eigensolves are cuSOLVER syevd (they synchronise).
 */
typedef struct {
  int nocc, nvir, naux, nmom_max; /* sizes; nmom_max <= 11 */
  const double* h;        /* [nmo][nmo]        in   core Hamiltonian, reference basis */
  const double* L;        /* [naux][nmo][nmo]  in   DF tensor, reference basis */
  double* C;              /* [nmo][nmo]        in/out orbitals (columns) */
  double* eps;            /* [nmo]             in/out orbital energies (ascending on output) */
  double* F;              /* [nmo][nmo]        out  the field of Eq. 35 at the end of the step */
  double* V;              /* [nmo][nmo]        out  the static potential in the reference basis */
  int reg;                /* host in: 0 = delta-broadened (Eqs. 36-37), 1 = SRG (Eqs. 38-39) */
  double delta, srg_s;    /* host in: broadening (reg 0, > 0) and flow parameter (reg 1, >= 0) */
  int diis_space;         /* host in: DIIS vectors kept (1..32) */
  int scf_max_iter;       /* host in: cap of the Eq. 35 iterations */
  double scf_tol;         /* host in: density tolerance of the Eq. 35 loop */
  double de;              /* host out */
  int scf_iters;          /* host out */
  int scf_converged;      /* host out: 1 if the Eq. 35 loop met its tolerance */
} mgw_qsgw_state;

mgw_status mgw_qsgw_step(mgw_handle* h, const mgw_options* o, mgw_qsgw_state* st);

/*
 * Warm-start network (not in the paper): three dense layers with SiLU,
 *   z1 = W1 x + b1, a1 = silu(z1); z2 = W2 a1 + b2, a2 = silu(z2); y = W3 a2 + b3.
 * params: FP32 master vector [W1 | b1 | W2 | b2 | W3 | b3] (W row-major
 * [out][in]); wbf16: the same layout in BF16, the copy every product reads.
 * All device pointers; float32 data.
 *  mgw_mlp_nparams   length of the packed vector
 *  mgw_mlp_round     wbf16 = bf16(params)
 *  mgw_mlp_forward   Y [batch][d_out] from X [batch][d_in]; acts (or NULL)
 *                    receives z1, a1, z2, a2 ([4][batch][width]) for backward
 *  mgw_mlp_backward  grad [nparams] of sum_b <dY_b, y_b> (BF16 rounding of the
 *                    weights passed through as identity)
 *  mgw_mlp_mse       dY = (Y - T)/batch, loss (device float) = |Y - T|^2 / (2 batch)
 *  mgw_mlp_adam      one Adam step (beta 0.9, 0.999, eps 1e-8) on params,
 *                    refreshing wbf16; step counts from 1
 */
long mgw_mlp_nparams(int d_in, int width, int d_out);
mgw_status mgw_mlp_round(mgw_handle* h, long n, const float* params, unsigned short* wbf16);
mgw_status mgw_mlp_forward(mgw_handle* h, int d_in, int width, int d_out, const float* params,
                           const unsigned short* wbf16, int batch, const float* X, float* Y, float* acts);
mgw_status mgw_mlp_backward(mgw_handle* h, int d_in, int width, int d_out, const unsigned short* wbf16,
                            int batch, const float* X, const float* acts, const float* dY, float* grad);
mgw_status mgw_mlp_mse(mgw_handle* h, int batch, int d_out, const float* Y, const float* T, float* dY,
                       float* loss);
mgw_status mgw_mlp_adam(mgw_handle* h, long n, float* params, unsigned short* wbf16, const float* grad,
                        float* m, float* v, int step, float lr);

/*
 * mgw_gemm_fp64_emu -- C = A B^T to FP64 accuracy on the BF16 tensor cores
 * (tcgen05, TMA, TMEM).  Each row of A and B is scaled by a power of two and
 * cut into 7 signed base-256 digits held exactly in BF16; the 28 digit
 * products above 2^-64 of the leading term are integer GEMMs, accumulated
 * exactly in FP32 over K chunks (1024 / (s + u - 1) wide) for the 21
 * products of levels s + u <= 7 and flushed into 64-bit integers, the 7 of
 * level 8 in FP32 over all of K.  Error:
 * a few units of 2^-53 times sum_k |A_ik| |B_jk|, as an FP64 GEMM.  Not in
 * the paper; it is how the FP64 contractions of the path reach the tensor
 * cores of a GPU whose FP64 units are few.
 *   A [M][K], B [N][K] in (FP64, row-major);  C [M][N] out (FP64)
 */
mgw_status mgw_gemm_fp64_emu(mgw_handle* h, int M, int N, int K,
                             const double* A, const double* B, double* C);

/*
 * The DF tensor on the mixed precision's grid, held as 16-bit integers: for
 * systems whose FP64 tensor does not fit the GPU (or the host) -- 2147
 * orbitals and 8588 auxiliary functions make 317 GB in FP64, 79 GB here.
 *   mgw_grid_exponent -- e with absmax < 2^(e-1), i.e. floor(log2 absmax) + 2
 *     (0 for absmax 0); the grid of MGW_MIXED is the multiples of 2^(e-16).
 *   mgw_df_absmax -- max |L| over `count` consecutive FP64 values (device),
 *     written to *absmax_host (synchronises): the maxima of the pieces of a
 *     tensor give its grid.
 *   mgw_df_quantize -- Lq = round(L 2^(16-e)) (ties away from zero) for
 *     `count` consecutive values: any slab range, so a tensor is quantized
 *     piece by piece as it is produced.  A value with |L| >= 2^(e-1) is stored
 *     as 0 and, when overflow_host is given, reported there (the call then
 *     synchronises and returns MGW_ERR_ARG).
 *   mgw_response_moments_q, mgw_sigma_moments_q -- mgw_response_moments (TDA)
 *     and mgw_sigma_moments in the MGW_MIXED precision (whatever o->precision
 *     says) from Lq [naux][nmo][nmo] with exponent e; the response takes V'
 *     from Lq's particle-hole block directly.  The results equal those of the
 *     FP64 calls on the tensor L' = Lq 2^(e-16).
 */
int mgw_grid_exponent(double absmax);
mgw_status mgw_df_absmax(mgw_handle* h, long count, const double* L, double* absmax_host);
mgw_status mgw_df_quantize(mgw_handle* h, long count, const double* L, int e, short* Lq, int* overflow_host);
mgw_status mgw_response_moments_q(mgw_handle* h, const mgw_options* o, int nocc, int nvir, int naux, int nmom,
                                  const double* eps_W, const short* Lq, int e, double* Wmom);
mgw_status mgw_sigma_moments_q(mgw_handle* h, const mgw_options* o, int nocc, int nvir, int naux, int nmom,
                               const double* eps_G, const short* Lq, int e, const double* Wmom,
                               double* sig_hole, double* sig_part);

/*
 * mgw_gemm_mixed -- C = A B'^T on the BF16 tensor cores, B' = B rounded to one
 * fixed-point grid (multiples of 2^(e-16), max |B| < 2^(e-1)), the product
 * of the MGW_MIXED precision: B' as two BF16 digits, A as seven per-row
 * digits, the 13 digit products above 2^-64 of the top, each exact; the K
 * loop runs in chunks of 128 so that each digit tile loaded serves every
 * product it takes part in, every level accumulating in its own TMEM
 * accumulator (exact levels over windows of 4-8 chunks, then added into
 * 64-bit integers; the two lowest levels in FP32).  K above 65536 runs in
 * splits summed in FP64.  Error against the exact A B'^T: a few units of
 * 2^-53 times sum_k |A_ik||B'_jk|.  Not in the paper.
 *   A [M][K], B [N][K] in (FP64, row-major);  C [M][N] out (FP64)
 */
mgw_status mgw_gemm_mixed(mgw_handle* h, int M, int N, int K,
                          const double* A, const double* B, double* C);

/*
 * mgw_gemm_bf16x3 -- C = A B^T on the tensor cores (tcgen05, TMA, TMEM):
 * each FP64 operand is split as x = hi + lo with hi = bf16(x),
 * lo = bf16(x - hi), and C accumulates hi*hi + hi*lo + lo*hi in FP32, then is
 * written as FP64.  Relative error about 1e-5 of |A||B| per element, too
 * coarse for the moment-to-block step (inconsistent moment errors are
 * amplified about 1e2 per block), so no path uses it; MGW_MIXED rounds the
 * input tensor instead and keeps every product exact.  Not in the paper.
 *   A [M][K], B [N][K] in (FP64, row-major);  C [M][N] out (FP64)
 */
mgw_status mgw_gemm_bf16x3(mgw_handle* h, int M, int N, int K,
                           const double* A, const double* B, double* C);

/*
 * mgw_selftest_bounded_wait -- exercise the error path of the tensor-core
 * kernels' bounded waits: one CTA waits, with the same time-bounded mbarrier
 * wait, on a barrier that nothing arrives at.  The wait gives up after
 * limit_s seconds (0 < limit_s <= 10), raises the status word, and the call
 * returns MGW_ERR_TIMEOUT with the text in mgw_last_error; the context and
 * the handle stay usable.  (In the GEMM kernels the same status word also
 * stops every CTA that starts after it is raised.)  Not in the paper.
 */
mgw_status mgw_selftest_bounded_wait(mgw_handle* h, double limit_s);

/*
 * mgw_response_moments_tda_noalloc -- the TDA branch of mgw_response_moments
 * (same W(n) = eta~(n) V^T, same arguments except the handle) for callers
 * that cannot allocate device memory: code running where cudaMalloc is
 * unavailable or forbidden (a host callback, a region that must not
 * synchronise, a process whose device memory belongs to another allocator,
 * or embedded callers that size memory up front).  The paper has no
 * counterpart; this is an interface of this library only.
 *
 * It allocates nothing: no cudaMalloc/cudaFree, no library routine that
 * allocates.  Its scratch (D and the running eta~) is one statically
 * allocated device array of 4 Mi doubles (32 MiB) that every GPU loading the
 * library holds until process exit; hence nocc*nvir*(naux + 1) must not
 * exceed about 4.19e6, else it returns MGW_ERR_UNSUPPORTED without queueing
 * anything.  The first call on a device does the set-up: it looks up the
 * array's device address (cudaGetSymbolAddress with that device current), so
 * that first call should come before any stream capture.  Every call shares
 * the array, which keeps the previous call's contents; nothing in it needs
 * clearing, since D and eta~ are written in full before they are read.
 * Calls whose GPU work overlaps (other streams, other host threads) race on
 * the array and must be serialised by the caller.
 *   cuda_stream: cudaStream_t (or NULL) on which the work is queued
 *   eps_W [nmo], Lov [naux][nocc*nvir] in; Wmom [nmom][naux][naux] out
 * Returns MGW_ERR_ARG on bad sizes or null pointers, MGW_ERR_CUDA if a launch
 * or the symbol lookup fails.  There is no handle, so no mgw_last_error text:
 * the status code is all a failing call reports.
 */
mgw_status mgw_response_moments_tda_noalloc(void* cuda_stream, int nocc, int nvir, int naux, int nmom,
                                            const double* eps_W, const double* Lov, double* Wmom);

#ifdef __cplusplus
}
#endif

#endif /* MGW_H */
