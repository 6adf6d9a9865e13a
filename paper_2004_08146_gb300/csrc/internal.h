// Internal declarations shared by the libqcd translation units.
#pragma once

#include <cuda_runtime.h>
#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>
#include <map>
#include <type_traits>

#include "common.cuh"

namespace qcd {

// ------------------------------------------------------------------ launch accounting
// Counts a launch with its algorithmic bytes/flops; optionally times it with
// events on `st` (see qcd_stats_reset).  Construct right before the launch.
class KTimer {
public:
    KTimer(const char* name, double bytes, double flops, cudaStream_t st);
    ~KTimer();
    KTimer(const KTimer&) = delete;
    KTimer& operator=(const KTimer&) = delete;
private:
    const char* name_;
    cudaStream_t st_;
    double bytes_, flops_;
    cudaEvent_t ea_ = nullptr, eb_ = nullptr;
};

// While one of these lives on a thread, KTimer records nothing (no host
// allocation for the accounting map).
class QuietAccounting {
public:
    QuietAccounting();
    ~QuietAccounting();
private:
    bool prev_;
};

// ------------------------------------------------------------------ fine operator
struct FineOp {
    Geom g{};
    double2* U64 = nullptr;   // [V][4][3][3]
    float2* U32 = nullptr;
    float2* U32s = nullptr;   // FP32 links site-fastest: [(mu * 9 + k) * V + site]
    double* A64 = nullptr;    // [V][2][36]: (m0 + 4) + clover, packed Hermitian 6x6
    float* A32 = nullptr;
    float4* A32s = nullptr;   // FP32 clover site-fastest: [q * V + site], q < 18 (16-byte pieces)
    double m0 = 0, csw = 0;
};

// ------------------------------------------------------------------ blocking
// A partition of the lattice into blocks of extent b[4]; blocks and local
// sites are lexicographic (mu = 3 fastest), like the fine sites.
struct Blocking {
    int b[4] = {0, 0, 0, 0};   // block extents
    int cd[4] = {0, 0, 0, 0};  // coarse (block-grid) extents
    int bs = 0;                // sites per block
    int nb = 0;                // number of blocks
};

__host__ __device__ __forceinline__ int block_fine_site(const Geom& g, const Blocking& B, int blk, int l) {
    int c[4], o[4], x[4];
    int t = blk;
    c[3] = t % B.cd[3]; t /= B.cd[3];
    c[2] = t % B.cd[2]; t /= B.cd[2];
    c[1] = t % B.cd[1]; c[0] = t / B.cd[1];
    t = l;
    o[3] = t % B.b[3]; t /= B.b[3];
    o[2] = t % B.b[2]; t /= B.b[2];
    o[1] = t % B.b[1]; o[0] = t / B.b[1];
    for (int mu = 0; mu < 4; ++mu) x[mu] = c[mu] * B.b[mu] + o[mu];
    return site_index(g, x);
}

// ------------------------------------------------------------------ coarse level
struct Coarse {
    Blocking B;
    Geom gc{};                // coarse lattice (antiperiodic unused)
    int nv = 0, nc = 0;       // nc = 2 nv
    double2* P64 = nullptr;   // [Vc][2][nv][bs][2][3]
    float2* P32 = nullptr;
    double2* A64 = nullptr;   // [Vc][9][col][row]  (column-major blocks)
    float2* A32 = nullptr;
    bool a64_stale = false;   // A32 was built in FP32 and A64 is out of date
    bool ready = false;
    int ctas = 0;             // CTAs of the one-launch coarse GMRES (0: one per SM)
};

// ------------------------------------------------------------------ kernels (dirac.cu)
void launch_clover_build(const FineOp& f, cudaStream_t st);
// max |U U^H - I| over nlinks device FP64 links (+inf if any entry is not
// finite); `scratch` is one device word.  Synchronises the stream.
double gauge_unitarity_deviation(const double2* U, size_t nlinks, unsigned long long* scratch, cudaStream_t st);
// `act` (device, per right-hand side, may be null): skip right-hand sides
// whose flag is 0 (converged systems of a batched Krylov solve).
// dU = i X U (V*36 double2) and the packed clover derivative dA (V*72 double)
// for U -> exp(i eps X) U (X: device FP64 traceless Hermitian [V][4][3][3]);
// then out_j = (dD/deps) in_j, FP64.
void tangent_fields(const FineOp& f, const double2* X, double2* dU, double* dA, cudaStream_t st);
void apply_tangent(const FineOp& f, const double2* dU, const double* dA, int nrhs, const double2* in, double2* out,
                   cudaStream_t st);
// Per-link force of the eigenvalue v^H Q v / v^H v: insertion fields Bt
// ([V][6][9]) then F ([V][4][9], traceless Hermitian); nrm: device v^H v.
void eig_force(const FineOp& f, const double2* v, const double2* nrm, double2* Bt, double2* F, cudaStream_t st);
// Force of Re <gv, Q' psi> per link (F [V][4][9], traceless Hermitian), or
// with grad = 1 the link gradient i F U; nrm (device, may be null) divides.
void bilinear_force(const FineOp& f, const double2* gv, const double2* psi, const double2* nrm, int grad, double2* Bt,
                    double2* F, cudaStream_t st);
void apply_op(const FineOp& f, int prec, int op, int nrhs, const void* in, void* out,
              const double* tau, cudaStream_t st, const int* act = nullptr);
void residual_op(const FineOp& f, int prec, int op, int nrhs, const void* b, const void* x, void* r,
                 const double* tau, cudaStream_t st, const int* act = nullptr);

// ------------------------------------------------------------------ kernels (blas.cu)
// All vectors are complex (double2 / float2) of length n; "sets" are arrays of
// nvec vectors for each of nrhs right-hand sides laid out [vec][rhs][n].
void blas_zero(int prec, void* x, size_t n, cudaStream_t st);
void blas_copy(int prec, const void* x, void* y, size_t n, cudaStream_t st);
void blas_convert(int prec_in, const void* x, int prec_out, void* y, size_t n, cudaStream_t st);
// dots[i*nrhs + j] = <X[i][j], w[j]> for i < nvec (FP64 results, device).
// partial: >= 64 * nvec * nrhs double2 of scratch; counters: >= nvec * nrhs
// unsigned that are zero on entry and are left zero (one launch: the last
// CTA of each dot adds the partial sums).
void blas_multidot(int prec, const void* X, int nvec, size_t xstride_vec, const void* w, int nrhs,
                   size_t n, double2* dots, double2* partial, unsigned* counters, cudaStream_t st,
                   const int* act = nullptr);
// w[j] += sign * sum_i c[i*nrhs + j] X[i][j]
void blas_multiaxpy(int prec, const void* X, int nvec, size_t xstride_vec, const double2* c, double sign,
                    void* w, int nrhs, size_t n, cudaStream_t st, const int* act = nullptr);
// y[j] = alpha_j x[j] (+ y[j] when accumulate), alpha from device array of nrhs complex
void blas_scale_dev(int prec, const void* x, void* y, const double2* alpha, int nrhs, size_t n,
                    bool invert_real, bool accumulate, cudaStream_t st, const int* act = nullptr);
void blas_gamma5(int prec, const void* x, void* y, size_t nsites_times_rhs, cudaStream_t st);
void blas_gaussian(double2* x, size_t n, unsigned long long seed, unsigned long long offset, cudaStream_t st);
// y = a*x + b*y (host scalars), complex
void blas_axpby(int prec, double2 a, const void* x, double2 b, void* y, size_t n, cudaStream_t st);

// ------------------------------------------------------------------ double-float (ff.cu)
// Internal storage precision of the Davidson basis: complex numbers as two
// FP32 pairs (hi + lo, 16 bytes, ~2^-48 relative), arithmetic by error-free
// transformations on the FP32 units.  Not an ABI precision.
constexpr int QCD_FF = 2;
// FP64 <-> FF, FF -> FP32 (hi + lo rounded), FP32 -> FF
void ff_convert(int prec_in, const void* x, int prec_out, void* y, size_t n, cudaStream_t st);
void ff_multidot(const void* X, int nvec, size_t xstride_vec, const void* w, int nrhs, size_t n, double2* dots,
                 double2* partial, unsigned* counters, cudaStream_t st, const int* act);
void ff_multiaxpy(const void* X, int nvec, size_t xstride_vec, const double2* c, double sign, void* w, int nrhs,
                  size_t n, cudaStream_t st, const int* act);
void ff_scale_dev(const void* x, void* y, const double2* alpha, int nrhs, size_t n, bool accumulate, cudaStream_t st,
                  const int* act);
void ff_axpby(double2 a, const void* x, double2 b, void* y, size_t n, cudaStream_t st);
void ff_gamma5(const void* x, void* y, size_t nsites, cudaStream_t st);
// A[j] <- sum_i C[i + j m] A[i] (j < p <= m) in place; cf_scratch: m * p * 16 bytes
void ff_transform_inplace(void* A, int m, const double2* C, int p, size_t n, void* cf_scratch, cudaStream_t st);
// Householder deflation of the pair (A0, A1) by the reflector hw (m + 1 entries); wf_scratch (m + 1) * 16 bytes
void ff_deflate(void* A0, void* A1, int m, size_t n, const double2* hw, void* wf_scratch, cudaStream_t st);

// ------------------------------------------------------------------ kernels (mg.cu)
void mg_build_P(const FineOp& f, Coarse& c, const double2* vecs, int nvec, cudaStream_t st);
void mg_build_coarse(const FineOp& f, Coarse& c, cudaStream_t st, bool fp32_only = false);
void mg_restrict(const FineOp& f, const Coarse& c, int prec, int nrhs, const void* r, void* xc, cudaStream_t st,
                 const int* act = nullptr);
void mg_prolong(const FineOp& f, const Coarse& c, int prec, int nrhs, const void* xc, void* x, bool accumulate,
                cudaStream_t st, const int* act = nullptr);
// tensor: FP32 applies with 2 Nv a multiple of 8 run on the tensor cores
// (3xTF32); otherwise, and for FP64, on the CUDA cores
void coarse_apply(const Coarse& c, int prec, int op, int nrhs, const void* x, void* y, const double* tau,
                  cudaStream_t st, bool tensor = true);

// ------------------------------------------------------------------ kernels (mg2.cu)
// Third level: c2.B blocks the level-1 lattice c1.gc; P2 [b2][chi][j][l][i < Nv1]
// (FP64 + FP32); the level-2 stencil in c2.A64/A32 like the level-1 one.
// W: FP64 level-2 test vectors [nv2][V1 * 2 Nv1].  mg2_build_coarse needs
// c1.A64 current.
void mg2_build_P(const Coarse& c1, Coarse& c2, const double2* W, cudaStream_t st);
void mg2_build_coarse(const Coarse& c1, Coarse& c2, cudaStream_t st);
void mg2_restrict(const Coarse& c1, const Coarse& c2, int prec, int nrhs, const void* r, void* xc, cudaStream_t st,
                  const int* act = nullptr);
void mg2_prolong(const Coarse& c1, const Coarse& c2, int prec, int nrhs, const void* xc, void* x, cudaStream_t st,
                 const int* act = nullptr);

struct SapPlan {
    Blocking B;
    int* blocks_of_colour[2] = {nullptr, nullptr};  // device lists of block ids
    int ncol[2] = {0, 0};
};
// x += block solves of op(tau) on the blocks of `colour`, rhs r (full fields)
// half: FP32 solves on 16-site blocks keep the block Krylov basis in FP16
void sap_blocks(const FineOp& f, const SapPlan& sp, int colour, int prec, int op, int nrhs,
                const void* r, void* x, const double* tau, int iters, double tol,
                void* scratch, cudaStream_t st, const int* act = nullptr, bool half = false);
// Global scratch of sap_blocks: blocks of 16 and 32 sites keep their Krylov
// basis in shared memory (0 bytes); every other block size needs
// (iters + 1) block vectors per block of the larger colour and per rhs.
bool sap_needs_scratch(const Blocking& B);
// SAP work counters (device-wide; see qcd_stats_sap_work): reset / read
// [sum bs k, sum bs k (k + 1) / 2] over the block solves since the reset.
void sap_work_reset();
void sap_work_read(double out[2]);
// bounded shared-memory waits that gave up (since the library was loaded)
unsigned long long wait_timeouts_read();
// one-warp kernel whose bounded wait on an mbarrier nobody arrives at gives up
void wait_probe(cudaStream_t st);
// FP32 / FP64 fused multiply-add throughput of the current device (TFLOP/s)
double fma_peak_tflops(int prec, cudaStream_t st);
size_t sap_scratch_bytes(const SapPlan& sp, int prec, int nrhs, int iters);

// ------------------------------------------------------------------ kernels (krylov.cu)
constexpr int kMaxKry = 64;        // fine (F)GMRES steps per solve
// Davidson basis size cap (m_max + targets per iteration): the harmonic
// pencil kernel keeps two FP32 m x m matrices in shared memory (200 KB at 112)
constexpr int kMaxBasis = 112;
constexpr int kMaxCoarse = 200;    // coarse GMRES steps per solve
constexpr int kMaxCoarseRhs = 16;  // right-hand sides per coarse launch

// Device-resident state of a batched (F)GMRES solve (see krylov.cu).
struct KryDev {
    int nrhs = 0, maxit = 0;
    double tol = 0;
    double* beta = nullptr;    // [nrhs] ||b_j||
    double* resid = nullptr;   // [nrhs] relative residual estimates
    int* active = nullptr;     // [nrhs] 1 while right-hand side j iterates
    int* k = nullptr;          // [nrhs] steps taken
    double* cs = nullptr;      // [nrhs][maxit]
    double2* sn = nullptr;     // [nrhs][maxit]
    double2* g = nullptr;      // [nrhs][maxit + 1]
    double2* R = nullptr;      // [nrhs][maxit][maxit] rotated Hessenberg
    double2* coef = nullptr;   // [maxit][nrhs] solution coefficients
    double2* scale = nullptr;  // [nrhs] normalisation of the next basis vector
};
size_t kry_bytes(int nrhs, int maxit);
KryDev kry_layout(void* buf, int nrhs, int maxit, double tol);
void kry_init(const KryDev& K, const double2* nrm, const int* outer_act, cudaStream_t st);
void kry_step(const KryDev& K, int it, const double2* h1, const double2* h2, const double2* nrm, cudaStream_t st);
void kry_finish(const KryDev& K, cudaStream_t st);
// Whole batched GMRES on the coarse stencil in one cooperative launch;
// returns 0 on success, < 0 when the cooperative launch is not possible.
// want_layout: 0 automatic; 1 stencil blocks and Krylov basis in shared
// memory; 2 basis in shared memory; 3 basis in global memory (any size).
size_t coarse_gmres_scratch(const Coarse& c, int prec, int nrhs, int maxit, int want_layout);
int coarse_gmres_grid();
int coarse_gmres_group(const Coarse& c, int prec, int maxit, int want_layout);   // right-hand sides per launch
int coarse_gmres_layout(const Coarse& c, int prec, int nrhs, int maxit, int want_layout);
int coarse_gmres(const Coarse& c, int prec, int op, int nrhs, const void* b, void* x, const double* tau_dev,
                 const int* act, double tol, int maxit, void* scratch, int* iters, double* resid,
                 unsigned long long* counter, int want_layout, cudaStream_t st);

// ------------------------------------------------------------------ kernels (eig.cu)
// Harmonic Ritz pairs of the pencil G s = theta H s (G = W^H W, H = W^H V):
// returns mu = 1/theta and S (column-major m x m) in device buffers.
// L^-1 and L^-1 H L^-H (G = L L^H) are kept in `state` (3 * ld * ld double2:
// those two and the FP32 eigenvectors of the latter) between calls: rows
// m0..m-1 are appended, m0 = 0 recomputes.
void small_harmonic_eig_inc(const double2* G, const double2* H, int m, int ld, int m0, double* mu, double2* S,
                            double2* state, int* status, cudaStream_t st);
// FP64 refinement of the targeted pairs (columns idx[0..nb) of S; their
// eigenvalues go to mu_out[0..nb)) from the state left by
// small_harmonic_eig_inc.
void small_refine_targets(const double2* state, int m, int ld, double2* S, const double* mu, double* mu_out,
                          const int* idx, int nb, cudaStream_t st);
// Orthonormal Q (m x k <= kMaxBasis, column-major, leading dim m) of the columns of S
// (m x k, leading dimension lds) by modified Gram-Schmidt applied twice.
void small_qr(const double2* S, int m, int k, int lds, double2* Q, double2* work, cudaStream_t st);
// C (m x p) = A^H B for small column-major matrices: used for Gram updates
void small_gram_transform(const double2* M, int m, int ldm, const double2* C, int p, double2* out,
                          int ldo, double2* work, cudaStream_t st);

}  // namespace qcd
