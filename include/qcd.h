/*
 * libqcd -- GB300 (sm_103a) hot path of the GD-lambda-AMG eigensolver for the
 * Hermitian Wilson-clover operator Q = Gamma5 D (Frommer, Kahl, Knechtli,
 * Rottmann, Strebel, Zwaan, arXiv 2004.08146).
 *
 * Conventions shared by every call
 * --------------------------------
 *  - Lattice dims = {L0, L1, L2, L3}; mu = 0 is time; the site index is
 *    lexicographic, site = ((x0*L1 + x1)*L2 + x2)*L3 + x3 (Sec. 2: N_t x N_s^3).
 *  - Gauge links U: [site][mu][row][col], complex128 stored as interleaved
 *    (re, im) doubles, HOST memory, copied in by qcd_set_gauge.
 *  - Fine spinor fields: [site][spin 4][colour 3] complex; complex128 for the
 *    FP64 entry points, complex64 where an entry point says so.  They are
 *    DEVICE pointers owned by the caller and used on the context's stream.
 *  - gamma matrices: chiral basis with gamma5 = diag(1, 1, -1, -1) (Sec. 2);
 *    gamma0 = -[[0, I],[I, 0]], gamma_k = [[0, -i sigma_k],[i sigma_k, 0]].
 *  - D = (m0 + 4) + clover - 1/2 sum_mu [(1 - gamma_mu) U_mu(x) psi(x+mu)
 *        + (1 + gamma_mu) U_mu(x-mu)^H psi(x-mu)]  (Eq. 2.5, a = 1), clover
 *    c_sw (i/4) sum_{mu,nu} sigma_{mu nu} F_{mu nu}, F = (Q_{mu nu} - h.c.)/8.
 *  - Every call returns 0 (QCD_OK) or one of the QCD_E* codes below; no
 *    exception crosses the ABI; qcd_last_error() gives a message.
 *  - Calls on one context are not thread safe; use one context per stream.
 */
#ifndef QCD_H
#define QCD_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define QCD_OK        0
#define QCD_EINVAL    1   /* bad argument, size or aliasing */
#define QCD_ENOMEM    2   /* device allocation failed */
#define QCD_ENOTSETUP 3   /* gauge field or multigrid hierarchy missing */
#define QCD_ENOCONV   4   /* iteration cap reached; outputs hold the best iterate */
#define QCD_ETIMEOUT  5   /* a bounded device-side wait gave up (reported by
                             qcd_mg_setup, the shifted solves and qcd_eigs,
                             which synchronise anyway; outputs unreliable) */
#define QCD_ECUDA     6   /* a CUDA runtime call failed */

/* Operators for qcd_apply */
#define QCD_OP_D   0      /* out = (D - tau Gamma5) in   (Eq. 3.7; tau = 0 gives D) */
#define QCD_OP_Q   1      /* out = (Q - tau) in          (Eq. 3.6) */

/* Precisions */
#define QCD_FP64   0      /* complex128 fields, FP64 arithmetic */
#define QCD_FP32   1      /* complex64 fields, FP32 arithmetic */
#define QCD_MIXED  1      /* solver mode: FP32 inner solves, FP64 outer */

/* Smoothers */
#define QCD_SMOOTHER_SAP   0
#define QCD_SMOOTHER_GMRES 1

#define QCD_EXTRACT_HARMONIC 0
#define QCD_EXTRACT_RITZ     1

typedef struct qcd_ctx qcd_ctx;

/* Parameters; defaults (qcd_default_params) are Table 2 of the paper. */
typedef struct qcd_params {
    int    antiperiodic_t;   /* 1: hops across the time boundary get -1 (default 1) */
    int    precision;        /* QCD_FP64 or QCD_MIXED for solves and eigs (default MIXED) */
    int    correction_form;  /* QCD_OP_D: (D - theta G5) t = G5 r (Eq. 3.7, default);
                                QCD_OP_Q: (Q - theta) t = r (Eq. 3.6) */
    int    use_mg;           /* 0: plain GMRES inner solve; 1: FGMRES + two-level MG */
    int    setup_iters;      /* adaptive setup iterations (Table 2: 6) */
    int    smoother;         /* QCD_SMOOTHER_SAP (default) or QCD_SMOOTHER_GMRES */
    int    nu;               /* post-smoothing steps (Table 2: 4) */
    int    sap_block[4];     /* SAP block extents (default 2,2,2,2) */
    int    sap_block_iters;  /* GMRES steps per SAP block solve (Sec. 4: 10; 1..32) */
    double sap_block_tol;    /* block residual reduction (Sec. 4: 1e-1) */
    int    gmres_smooth_iters; /* GMRES smoother steps per smoothing step (4) */
    double inner_tol;        /* FGMRES relative residual (Table 2: 1e-1) */
    int    inner_maxiter;    /* FGMRES iterations (Table 2: 5) */
    double coarse_tol;       /* coarse GMRES reduction (Table 2: 5e-1) */
    int    coarse_maxiter;   /* coarse GMRES iteration cap (default 64, <= 200) */
    int    plain_maxiter;    /* plain GMRES inner iterations without MG (default 20) */
    int    m_min;            /* Table 2: 30 */
    int    m_max;            /* Table 2: 50 */
    int    block;            /* targets per outer iteration (>= 1; default 2).  Keep
                                m_max - m_min >= 2 * block: with one outer step
                                between restarts a dense cluster can lose an
                                eigenvalue (16 targets at m_min 30, m_max 48
                                did on a 32x16^3 field) */
    int    n_init;           /* random start vectors when use_mg = 0 (default 8) */
    int    shift_rho;        /* 1: correction-equation shift = Rayleigh quotient rho of the
                                target vector (default); 0: its harmonic Ritz value theta */
    int    update_every;     /* interpolation rebuild every k locks (default 1; 0: never,
                                the no-update variant of Sec. 4) */
    int    extraction;       /* QCD_EXTRACT_HARMONIC: harmonic Ritz pairs (Theorem 1,
                                default); QCD_EXTRACT_RITZ: Rayleigh-Ritz pairs of
                                V^H Q V (the Ritz-Galerkin condition of Sec. 3) */
    int    max_outer;        /* outer iteration cap (default 100000) */
    unsigned long long seed; /* counter-based RNG seed for setup / start vectors */
    int    verbose;          /* 1: per-lock progress on stderr */
    int    levels;           /* 2 (default) or 3: the coarse solve becomes the K-cycle --
                                FGMRES on D_c to coarse_tol, preconditioned by a
                                two-level cycle on the coarse lattice */
    int    nv2;              /* level-2 test vectors: the first nv2 fine test vectors
                                restricted by P^H (default 8, <= Nv) */
    int    agg2[4];          /* level-2 aggregate extents on the coarse lattice (2,2,2,2) */
    int    nu2;              /* GMRES smoothing steps on the coarse lattice per level-1
                                cycle (gmres_smooth_iters iterations each; default 2) */
    int    coarse_layout;    /* data placement of the one-launch coarse GMRES: 0 automatic
                                (default); 1 stencil blocks and Krylov basis in shared
                                memory; 2 Krylov basis in shared memory; 3 Krylov basis
                                in global memory (any coarse lattice).  A forced layout
                                that does not fit returns EINVAL. */
    int    coarse_tensor;    /* FP32 coarse-stencil applies of the level-1 operator:
                                0 (default) on the FMA units, stencil blocks and vectors
                                staged into shared memory by bulk asynchronous copies
                                (16-byte aligned vectors; plain loads otherwise); 1 on the
                                tensor cores (mma.sync, 2 Nv a multiple of 8), TF32 inputs
                                split in big + small parts (three products, FP32
                                accumulation) -- 3x slower than 0 on 16 right-hand sides */
    int    sap_half;         /* 1: FP32 SAP block solves on 16-site blocks store their
                                Krylov basis in FP16 (half the shared memory, more block
                                solves resident; default 0) */
    int    confirm;          /* completion check of qcd_eigs: once k pairs are locked
                                and no harmonic Ritz value lies below the k-th
                                smallest locked |lambda|, the search continues until
                                this many correction equations (for the smallest values
                                above that bound) have left none below it; a value
                                below it resets the count.  0 returns at the first such
                                check (default 32: two outer iterations at 16 targets,
                                eight at 4; <= 1024) */
    int    coarse_ctas;      /* CTAs of the one-launch coarse GMRES: 0 (default) one per
                                SM; n > 0 at most n (fewer CTAs make its grid-wide
                                barriers cheaper on small coarse lattices) */
    int    guard;            /* qcd_eigs locks k + guard pairs before its completion check
                                and returns the k smallest |lambda| (an interior eigensolver
                                can skip an eigenvalue near the end of its run; the extra
                                pairs keep the search there longer).  Default 0, <= 256 */
} qcd_params;

typedef struct qcd_solve_info {
    int    iterations;       /* FGMRES / GMRES iterations (summed over refinements) */
    int    refinements;      /* FP64 refinement steps (mixed precision) */
    double residual;         /* final ||b - (Q - tau) x|| / ||b|| in FP64 */
    double seconds;          /* wall time of the call */
} qcd_solve_info;

typedef struct qcd_eig_info {
    int    outer;            /* outer (Davidson) iterations */
    int    inner;            /* inner FGMRES/GMRES iterations, all targets */
    int    locked;           /* pairs locked (>= k when converged) */
    int    updates;          /* interpolation rebuilds */
    int    converged;        /* 1 when all k pairs met tol */
    double max_residual;     /* max ||Q v - lambda v|| over the returned pairs */
    double seconds;          /* wall time of the call */
    long long coarse_solves;     /* coarse-grid GMRES solves (per right-hand side) */
    long long coarse_iterations; /* coarse-grid GMRES iterations, summed */
} qcd_eig_info;

/* Fill *p with the defaults above. */
void qcd_default_params(qcd_params* p);

/* Create a context bound to a CUDA stream (cudaStream_t; NULL = legacy
 * default stream) on the current device.  *ctx is owned by the caller and
 * released by qcd_destroy.  EINVAL on a NULL ctx or p. */
int qcd_create(qcd_ctx** ctx, const qcd_params* p, void* cuda_stream);
int qcd_destroy(qcd_ctx* ctx);
const char* qcd_last_error(qcd_ctx* ctx);

/* Change parameters after creation (solver knobs only; the multigrid
 * hierarchy is rebuilt by the next qcd_mg_setup). */
int qcd_set_params(qcd_ctx* ctx, const qcd_params* p);

/* Load the gauge field (Sec. 2, Eq. 2.5): U is a HOST array of
 * dims[0]*dims[1]*dims[2]*dims[3]*4*9 complex128 in [site][mu][row][col]
 * order; the library copies it, builds the clover term on the device and
 * keeps FP64 and FP32 copies.  m0 and csw as in Eq. 2.5 / Table 1.  Every
 * extent must be >= 2; a previous hierarchy is dropped.  EINVAL on bad dims. */
int qcd_set_gauge(qcd_ctx* ctx, const double* U, const int dims[4], double m0, double csw);

/* out = (Q - tau) in  (Eq. 1.1 with A = Q; Eq. 3.6).  in/out: device
 * complex128 fields of 12 * V elements; in == out returns EINVAL. */
int qcd_apply_Q(qcd_ctx* ctx, const void* in, void* out, double tau);

/* Multi-right-hand-side operator apply (Eq. 2.5 / 3.6 / 3.7): for
 * j < nrhs, out_j = op(tau[j]) in_j where op is QCD_OP_D (D - tau Gamma5) or
 * QCD_OP_Q (Q - tau).  in/out are device arrays of nrhs consecutive fields
 * (complex128 for QCD_FP64, complex64 for QCD_FP32); tau is a HOST array
 * of nrhs doubles; 1 <= nrhs <= 64; in and out must not overlap. */
int qcd_apply(qcd_ctx* ctx, int op, int prec, int nrhs, const void* in, void* out,
              const double* tau);

/* Multigrid setup (Sec. 2 "Algebraic multigrid methods", Table 2): draw Nv
 * seeded random test vectors, run params.setup_iters adaptive setup
 * iterations and build the chirality-split aggregation P over blocks of
 * extent block[4] (each must divide the lattice) and the Galerkin coarse
 * operator D_c = P^H D P (Eq. 2.8, 2.9).  Requires qcd_set_gauge. */
int qcd_mg_setup(qcd_ctx* ctx, int Nv, const int block[4]);

/* Rebuild P and D_c from nvec given fine vectors (Sec. 3, "Local coherence";
 * Algorithm 2 interpolation update).  V: DEVICE array of nvec consecutive
 * complex128 fields.  Without a prior qcd_mg_setup, block = params.sap_block
 * is used for the aggregates.  1 <= nvec <= 32. */
int qcd_mg_update_from_eigvecs(qcd_ctx* ctx, const void* V, int nvec);

/* Solve (Q - tau) x = b to ||b - (Q - tau) x|| <= tol ||b|| (Eq. 1.1):
 * FGMRES preconditioned by the two-level cycle on the Gamma5 form (Eq. 3.7),
 * FP32 inner solves wrapped by FP64 iterative refinement in QCD_MIXED mode.
 * b, x: device complex128 fields; x is the output (its input is ignored).
 * ENOCONV leaves the best iterate in x and its residual in info. */
int qcd_shifted_solve(qcd_ctx* ctx, const void* b, void* x, double tau, double tol,
                      qcd_solve_info* info);

/* Batched form: nrhs systems with distinct shifts tau[j] (HOST array) solved
 * together, b[j], x[j] device complex128 fields; 1 <= nrhs <= 64. */
int qcd_shifted_solve_batched(qcd_ctx* ctx, int nrhs, const void* const* b, void* const* x,
                              const double* tau, double tol, qcd_solve_info* info);

/* GD-lambda-AMG (Algorithm 2): the k eigenpairs of Q of smallest |lambda| to
 * ||Q v - lambda v|| <= tol (||v|| = 1).  lambda: HOST array of k doubles,
 * ascending |lambda| (ties ascending lambda); V: DEVICE array of k
 * consecutive complex128 fields (may be NULL).  Uses the hierarchy from
 * qcd_mg_setup when params.use_mg = 1 (ENOTSETUP otherwise). */
int qcd_eigs(qcd_ctx* ctx, int k, double tol, double* lambda, void* V, qcd_eig_info* info);

/* ---------------------------------------------------------------------
 * Component entry points (the pieces of the hot path, for tests and for
 * callers that build their own solvers).  Coarse vectors are
 * [coarse site][chirality][i < Nv] complex; prec selects complex128 or
 * complex64 buffers; all pointers are DEVICE pointers unless stated.
 * ------------------------------------------------------------------- */

/* Sizes of the current hierarchy: out[0] = coarse sites, out[1] = Nv,
 * out[2..5] = coarse dims, out[6] = block sites. */
int qcd_mg_info(qcd_ctx* ctx, int out[8]);

/* x_c = P^H r (Eq. 2.8, R = P^H) for nrhs fields. */
int qcd_mg_restrict(qcd_ctx* ctx, int prec, int nrhs, const void* r, void* xc);

/* x = P x_c for nrhs coarse vectors (overwrites x). */
int qcd_mg_prolong(qcd_ctx* ctx, int prec, int nrhs, const void* xc, void* x);

/* Third level (params.levels = 3; QCD_ENOTSETUP otherwise).  out[0] = level-2
 * sites, out[1] = nv2, out[2..5] = level-2 dims, out[6] = coarse sites per
 * level-2 aggregate, out[7] = Nv of level 1. */
int qcd_mg_info2(qcd_ctx* ctx, int out[8]);

/* Copy P2 (HOST complex128 [level-2 site][chi][j < nv2][aggregate site][i < Nv]):
 * the restricted test vectors of each (aggregate, chirality) orthonormalised by
 * modified Gram-Schmidt applied twice. */
int qcd_mg_get_P2(qcd_ctx* ctx, double* P_host);

/* Copy the level-2 stencil P2^H D_c P2 (HOST complex128 [site][d][row][col],
 * d as for qcd_mg_get_coarse). */
int qcd_mg_get_coarse2(qcd_ctx* ctx, double* A_host);

/* y_j = (D_c - tau_j Gamma5^c) x_j (op QCD_OP_D) or (Gamma5^c D_c - tau_j) x_j
 * (op QCD_OP_Q), coarse stencil of Eq. 2.8 / 2.9; tau HOST array. */
int qcd_coarse_apply(qcd_ctx* ctx, int op, int prec, int nrhs, const void* x, void* y,
                     const double* tau);

/* Eigenvalue derivatives along a link direction (no counterpart in the paper;
 * the differentiation form of the eigensolver's operator, Eq. 2.5 plus the
 * clover term): for links moved as U_mu(x) -> exp(i eps X_mu(x)) U_mu(x),
 * out[k] = d lambda_k / d eps = v_k^H Gamma5 (dD/d eps) v_k / v_k^H v_k
 * (Hellmann-Feynman; valid for simple eigenvalues and eigenvectors v_k of Q).
 * X: HOST complex128 [site][mu][3][3] traceless Hermitian; V: DEVICE
 * complex128 [nvec][V*12] eigenvectors (16-byte aligned); out: HOST nvec
 * doubles.  FP64 throughout; dD/d eps is the stencil with dU = i X U and the
 * product-rule derivative of every clover leaf.  Errors: ENOTSETUP before
 * qcd_set_gauge; EINVAL for nvec < 0, NULL or misaligned pointers; nvec = 0
 * does nothing; a zero vector gives 0. */
int qcd_eig_derivative(qcd_ctx* ctx, const double* X, int nvec, const void* V, double* out);

/* The same derivative resolved per link (the force of each eigenvalue):
 * F[k] = the traceless Hermitian 3x3 fields F_mu(x) with
 * d lambda_k / d eps = sum_{x,mu} tr(X_mu(x) F_mu(x)) for every traceless
 * Hermitian X, normalised by v_k^H v_k.  Hop terms contribute the colour
 * outer product of v_k(x + mu) and Gamma5 v_k(x) through the spin projector;
 * the clover term the plaquettes above and below each link with the clover
 * insertion at each corner.  V: DEVICE complex128 [nvec][V*12]; F: DEVICE
 * complex128 [nvec][site][mu][3][3] (gauge-field layout), caller-owned and
 * overwritten; both 16-byte aligned.  FP64 throughout.  Errors: ENOTSETUP
 * before qcd_set_gauge; EINVAL for nvec < 0, NULL or misaligned pointers;
 * nvec = 0 does nothing.  A zero vector gives a zero force. */
int qcd_eig_force(qcd_ctx* ctx, int nvec, const void* V, void* F);

/* Link gradient of a real bilinear form (no counterpart in the paper; the
 * backward pass of psi -> (Q - tau) psi with respect to the links, for
 * autograd): for each k < nvec, F[k] = the traceless Hermitian 3x3 fields
 * F_mu(x) with d/d eps Re <g_k, Q(U(eps)) psi_k> = sum_{x,mu} tr(X_mu(x)
 * F_mu(x)) for links moving as U -> exp(i eps X) U (X traceless Hermitian);
 * grad = 1 returns instead the tangent vectors i F_mu(x) U_mu(x), whose real
 * inner product Re tr(G^H dU) with any such dU = i X U is that derivative.
 * Hop terms: the two forward outer products of psi and Gamma5 g (Q' is
 * Hermitian); clover term: plaquettes above and below each link with the
 * insertion of sigma psi (Gamma5 g)^H at each corner.  G, Psi: DEVICE
 * complex128 [nvec][V*12]; F: DEVICE complex128 [nvec][site][mu][3][3],
 * caller-owned and overwritten; all 16-byte aligned.  FP64.  Errors:
 * ENOTSETUP before qcd_set_gauge; EINVAL for nvec < 0, NULL or misaligned
 * pointers, grad not 0 or 1; nvec = 0 does nothing. */
int qcd_bilinear_force(qcd_ctx* ctx, int nvec, const void* G, const void* Psi, int grad, void* F);

/* Local coherence lc(v) = ||Pi v|| / ||v|| (Sec. 3, the local coherence
 * measure) of nvec FP64 fine vectors V (DEVICE, complex128 [nvec][V*12],
 * 16-byte aligned) with respect to the current interpolation P; Pi = P P^H is
 * the orthogonal projection on range(P) (P has orthonormal columns, so
 * lc(v) = ||P^H v|| / ||v||).  out: HOST array of nvec doubles (0 for v = 0).
 * Needs qcd_mg_setup or qcd_mg_update_from_eigvecs first (QCD_ENOTSETUP). */
int qcd_local_coherence(qcd_ctx* ctx, int nvec, const void* V, double* out);

/* Copy P (HOST complex128 [coarse site][chi][i][block site][spin 2][colour 3])
 * and the coarse stencil (HOST complex128 [coarse site][9][row][col];
 * direction 0 = self, 1+mu = +mu, 5+mu = -mu) out of the library. */
int qcd_mg_get_P(qcd_ctx* ctx, double* P_host);
int qcd_mg_get_coarse(qcd_ctx* ctx, double* A_host);

/* The small projected eigenproblem of one Davidson step (Sec. 3): with
 * extraction QCD_EXTRACT_HARMONIC, the harmonic Ritz pencil of Theorem 1 /
 * Eq. 3.5, (W^H V) s = (1/theta) (W^H W) s, given G = W^H W (Hermitian
 * positive definite) and H = W^H V (Hermitian) for W = Q V; with
 * QCD_EXTRACT_RITZ the Ritz-Galerkin problem H s = theta s for orthonormal V
 * (G is ignored and may be NULL).  G, H: HOST complex128 m x m column-major,
 * 1 <= m <= 112 (the library's Davidson basis cap).  Outputs (HOST): theta[m]
 * sorted by ascending |theta| (ties ascending theta) and S (complex128
 * m x m column-major, column i the coefficient vector of pair i, normalised
 * so that S^H G S = I; S^H S = I for Rayleigh-Ritz).  Computed by the kernels
 * of qcd_eigs: Cholesky, FP32 Jacobi and FP64 refinement of every pair.
 * EINVAL on bad arguments or a G that is not positive definite. */
int qcd_projected_eig(qcd_ctx* ctx, int m, const double* G, const double* H, int extraction, double* theta,
                      double* S);

/* `sweeps` SAP sweeps (Eq. 2.10; colour 0 blocks, then colour 1) on
 * op(tau) x = b with GMRES block solves of params.sap_block_iters steps to
 * params.sap_block_tol (block_tol < 0 forces exactly sap_block_iters
 * steps); x is updated in place.  nrhs fields, tau HOST array. */
int qcd_sap(qcd_ctx* ctx, int op, int prec, int nrhs, const void* b, void* x,
            const double* tau, int sweeps, double block_tol);

/* One two-level cycle x = M b (Eq. 2.8 with post-smoothing only) on op(tau). */
int qcd_mg_cycle(qcd_ctx* ctx, int op, int prec, int nrhs, const void* b, void* x,
                 const double* tau);

/* qcd_sap with no memory allocation (the paper has no counterpart: this
 * serves callers that cannot allocate device memory while they run, e.g. an
 * application that gives the library a fixed memory budget up front, or a
 * plugin whose host owns every allocation).  Same arguments, layout and
 * result as qcd_sap; all scratch (colour block lists, nrhs residual fields,
 * block-GMRES vectors for every block size other than 16 and 32 sites, whose
 * kernels keep them in shared memory) comes from one 64 MiB
 * file-scope device array that every GPU loading libqcd keeps until the
 * process exits.  Needs lists + 12 * V * nrhs complex fields (+ Krylov
 * vectors) <= 64 MiB, else EINVAL with a message.  The first call on a device
 * looks up that array's device address (cudaGetSymbolAddress) and must be
 * made with that device current; make it before any stream capture.  The
 * call allocates nothing (no cudaMalloc/cudaFree, no library allocator) and
 * records no launch statistics; it clears nothing because every scratch word
 * is written before it is read.  All calls share the array: calls that
 * overlap on the GPU (other streams, other threads) race.  Returns after the
 * context's stream has synchronised. */
int qcd_sap_static(qcd_ctx* ctx, int op, int prec, int nrhs, const void* b, void* x,
                   const double* tau, int sweeps, double block_tol);

/* ---------------------------------------------------------------------
 * Launch accounting (process-wide, not part of the method): every libqcd
 * kernel launch is counted with its algorithmic bytes and flops; with
 * mode 1 every launch, with mode 2 only launches of the kernel named
 * `filter`, is bracketed by CUDA events on its stream.  qcd_stats_read waits
 * for the recorded events and returns up to `max` per-kernel records (*n =
 * number of kernels seen).  EINVAL on a bad mode or NULL n.
 * ------------------------------------------------------------------- */
typedef struct qcd_kernel_stat {
    char      name[40];
    long long launches;      /* launches since the last reset */
    long long timed;         /* launches timed with events */
    double    total_ms;      /* summed event time of the timed launches */
    double    bytes;         /* algorithmic bytes, all launches */
    double    flops;         /* algorithmic flops, all launches */
    double    timed_bytes;   /* algorithmic bytes of the timed launches */
    double    timed_flops;   /* algorithmic flops of the timed launches */
} qcd_kernel_stat;

int qcd_stats_reset(int mode, const char* filter);
int qcd_stats_read(qcd_kernel_stat* out, int max, int* n);

/* Work of the SAP block solves (Eq. 2.10, block GMRES) since the last
 * qcd_stats_reset, summed over every block solve of every launch:
 * *site_steps = sum (block sites x GMRES steps k), *site_steps_tri =
 * sum (block sites x k (k + 1) / 2); a flop model of one block solve
 * (operator applies plus Gram-Schmidt) turns them into the flops actually
 * executed.  Waits for nothing: read after synchronising.  EINVAL on NULL. */
int qcd_stats_sap_work(double* site_steps, double* site_steps_tri);

/* Number of bounded device-side waits that gave up since the library was
 * loaded (a kernel waiting on its own asynchronous shared-memory copies gives
 * up after about half a second, skips its output and counts itself here; 0
 * in every correct run).  ECUDA if the read fails, EINVAL on NULL. */
int qcd_stats_wait_timeouts(unsigned long long* n);

/* Self-test of the bounded device-side waits: launches on the context's
 * stream a one-warp kernel that waits on an mbarrier nothing arrives at; the
 * wait gives up after 2^21 clocks (about 1 ms), counts itself, and the call
 * returns QCD_ETIMEOUT with the context still usable (a later call that
 * reports timeouts sees only newer ones).  Faults nothing, hangs nothing. */
int qcd_selftest_wait_limit(qcd_ctx* ctx);

/* Measured fused multiply-add throughput of the current device in TFLOP/s
 * (2 flops per FMA) for prec QCD_FP32 or QCD_FP64 (FMA units), or prec 2 for
 * FP64 on the tensor cores (mma m8n8k4 f64): a kernel of independent chains
 * on every SM, best of five timed launches on the default stream (the
 * roofline denominator of FP32- and FP64-bound kernels; the SM clock at the
 * time of the call sets the value).  EINVAL on a bad prec or NULL; ECUDA when
 * the launch fails. */
int qcd_fma_peak(int prec, double* tflops);

#ifdef __cplusplus
}
#endif
#endif /* QCD_H */
