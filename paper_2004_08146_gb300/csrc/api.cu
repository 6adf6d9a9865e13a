// libqcd C ABI and host-side control: context, gauge upload, operator
// applies, the multigrid hierarchy (setup and interpolation updates),
// batched (F)GMRES, the two-level cycle, shifted solves with FP64 iterative
// refinement and the GD-lambda-AMG outer iteration (Algorithm 2).  The host
// only reads back scalars (dot products, norms, harmonic Ritz values) to take
// control decisions; every vector operation runs in the kernels of the other
// translation units.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <complex>
#include <cstdio>
#include <cstring>
#include <functional>
#include <memory>
#include <numeric>
#include <stdexcept>

#include "internal.h"

using namespace qcd;

namespace {

struct QcdError : std::runtime_error {
    int code;
    QcdError(int c, const std::string& m) : std::runtime_error(m), code(c) {}
};

#define CK(call)                                                                              \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess)                                                                \
            throw QcdError(QCD_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_));    \
    } while (0)

void check_launch(const char* what) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) throw QcdError(QCD_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

using cd = std::complex<double>;

struct DevBuf {
    void* p = nullptr;
    size_t bytes = 0;
};

double now_s() {
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

}  // namespace

struct qcd_ctx {
    qcd_params p{};
    cudaStream_t st = nullptr;
    std::string err;
    bool have_gauge = false;
    FineOp f;
    Coarse c;
    Coarse c2;                        // third level (params.levels = 3)
    SapPlan sap;
    bool have_sap = false;
    std::map<std::string, DevBuf> ws;
    double2* pinned = nullptr;   // host staging for small read-backs
    size_t pinned_n = 0;
    double2* test_vectors = nullptr;  // FP64 setup vectors [nv][V*12]
    int n_test = 0;
    int c2_nv1 = 0;                   // Nv of level 1 when c2 was allocated
    bool no_coop = false;             // cooperative coarse launch unavailable: host-driven GMRES
    unsigned* md_cnt = nullptr;       // zeroed dot-product completion counters (blas_multidot)
    size_t md_cnt_n = 0;

    ~qcd_ctx() { release(); }

    void release() {
        for (auto& kv : ws) if (kv.second.p) cudaFree(kv.second.p);
        ws.clear();
        auto fr = [](void* q) { if (q) cudaFree(q); };
        fr(f.U64); fr(f.U32); fr(f.U32s); fr(f.A64); fr(f.A32); fr(f.A32s);
        f.U64 = nullptr; f.U32 = nullptr; f.U32s = nullptr; f.A64 = nullptr; f.A32 = nullptr; f.A32s = nullptr;
        drop_mg();
        fr(sap.blocks_of_colour[0]); fr(sap.blocks_of_colour[1]);
        sap.blocks_of_colour[0] = sap.blocks_of_colour[1] = nullptr;
        have_sap = false;
        if (pinned) cudaFreeHost(pinned);
        pinned = nullptr;
        pinned_n = 0;
        fr(md_cnt);
        md_cnt = nullptr;
        md_cnt_n = 0;
    }
    void drop_mg() {
        auto fr = [](void* q) { if (q) cudaFree(q); };
        fr(c.P64); fr(c.P32); fr(c.A64); fr(c.A32); fr(test_vectors);
        c.P64 = nullptr; c.P32 = nullptr; c.A64 = nullptr; c.A32 = nullptr;
        test_vectors = nullptr;
        n_test = 0;
        c.ready = false;
        drop_level2();
    }
    void drop_level2() {
        auto fr = [](void* q) { if (q) cudaFree(q); };
        fr(c2.P64); fr(c2.P32); fr(c2.A64); fr(c2.A32);
        c2.P64 = nullptr; c2.P32 = nullptr; c2.A64 = nullptr; c2.A32 = nullptr;
        c2.nv = c2.nc = 0;
        c2.ready = false;
    }

    void drop_buf(const std::string& name) {
        auto it = ws.find(name);
        if (it == ws.end()) return;
        if (it->second.p) cudaFree(it->second.p);
        ws.erase(it);
    }
    void* buf(const std::string& name, size_t bytes) {
        DevBuf& b = ws[name];
        if (b.bytes < bytes) {
            if (b.p) CK(cudaFree(b.p));
            b.p = nullptr;
            b.bytes = 0;
            if (cudaMalloc(&b.p, bytes) != cudaSuccess) {
                cudaGetLastError();
                throw QcdError(QCD_ENOMEM, "device allocation of " + std::to_string(bytes) + " bytes for " + name);
            }
            b.bytes = bytes;
        }
        return b.p;
    }
    // completion counters for dot products, zero between launches
    unsigned* dot_counters(size_t n) {
        if (md_cnt_n < n) {
            n = std::max<size_t>(n, 4096);
            if (md_cnt) {
                CK(cudaStreamSynchronize(st));
                CK(cudaFree(md_cnt));
            }
            md_cnt = nullptr;
            md_cnt_n = 0;
            if (cudaMalloc(&md_cnt, n * sizeof(unsigned)) != cudaSuccess) {
                cudaGetLastError();
                throw QcdError(QCD_ENOMEM, "device allocation of dot-product counters");
            }
            CK(cudaMemsetAsync(md_cnt, 0, n * sizeof(unsigned), st));
            md_cnt_n = n;
        }
        return md_cnt;
    }
    double2* host(size_t n) {
        if (pinned_n < n) {
            if (pinned) CK(cudaFreeHost(pinned));
            pinned = nullptr;
            CK(cudaMallocHost((void**)&pinned, n * sizeof(double2)));
            pinned_n = n;
        }
        return pinned;
    }
    // copy n complex values from the device and wait
    const double2* fetch(const double2* d, size_t n) {
        double2* h = host(n);
        CK(cudaMemcpyAsync(h, d, n * sizeof(double2), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        return h;
    }
    size_t nfine() const { return (size_t)f.g.V * 12; }
    // device counters: [0] coarse solves, [1] coarse iterations
    unsigned long long* counters() { return (unsigned long long*)buf("counters", 2 * sizeof(unsigned long long)); }
};

namespace {

size_t esz(int prec) { return prec == QCD_FP64 ? sizeof(double2) : sizeof(float2); }

void validate_params(const qcd_params& p) {
    if (p.m_min < 1 || p.m_max < p.m_min + 1 || p.m_max > kMaxBasis - 1)
        throw QcdError(QCD_EINVAL, "need 1 <= m_min < m_max < " + std::to_string(kMaxBasis));
    if (p.block < 1 || p.block > 32) throw QcdError(QCD_EINVAL, "block must be in [1, 32]");
    if (p.update_every < 0) throw QcdError(QCD_EINVAL, "update_every must be >= 0");
    if (p.extraction != QCD_EXTRACT_HARMONIC && p.extraction != QCD_EXTRACT_RITZ)
        throw QcdError(QCD_EINVAL, "bad extraction");
    if (p.m_max + p.block > kMaxBasis)
        throw QcdError(QCD_EINVAL, "need m_max + block <= " + std::to_string(kMaxBasis));
    if (p.nu < 0 || p.sap_block_iters < 1 || p.sap_block_iters > 32) throw QcdError(QCD_EINVAL, "bad smoother params");
    if (p.inner_maxiter < 1 || p.inner_maxiter > 64 || p.coarse_maxiter < 1 || p.coarse_maxiter > 200 ||
        p.plain_maxiter < 1 || p.plain_maxiter > 200)
        throw QcdError(QCD_EINVAL, "bad iteration caps");
    if (p.precision != QCD_FP64 && p.precision != QCD_MIXED) throw QcdError(QCD_EINVAL, "bad precision");
    if (p.correction_form != QCD_OP_D && p.correction_form != QCD_OP_Q) throw QcdError(QCD_EINVAL, "bad correction_form");
    if (p.levels != 2 && p.levels != 3) throw QcdError(QCD_EINVAL, "levels must be 2 or 3");
    if (p.nv2 < 1 || p.nv2 > 32 || p.nu2 < 0) throw QcdError(QCD_EINVAL, "need 1 <= nv2 <= 32 and nu2 >= 0");
    for (int mu = 0; mu < 4; ++mu)
        if (p.agg2[mu] < 1) throw QcdError(QCD_EINVAL, "agg2 extents must be >= 1");
    if (p.coarse_layout < 0 || p.coarse_layout > 3) throw QcdError(QCD_EINVAL, "coarse_layout must be in [0, 3]");
    if (p.coarse_tensor != 0 && p.coarse_tensor != 1) throw QcdError(QCD_EINVAL, "coarse_tensor must be 0 or 1");
    if (p.sap_half != 0 && p.sap_half != 1) throw QcdError(QCD_EINVAL, "sap_half must be 0 or 1");
    if (p.confirm < 0 || p.confirm > 1024) throw QcdError(QCD_EINVAL, "confirm must be in [0, 1024]");
    if (p.coarse_ctas < 0) throw QcdError(QCD_EINVAL, "coarse_ctas must be >= 0");
    if (p.guard < 0 || p.guard > 256) throw QcdError(QCD_EINVAL, "guard must be in [0, 256]");
}

// ------------------------------------------------------------------ linear operators
// operator / preconditioner: out = op(in) for the right-hand sides whose
// device flag in `act` is set (act may be null: all)
using OpFn = std::function<void(const void* in, void* out, const int* act)>;

struct GmresResult {
    std::vector<int> iters;
    std::vector<double> resest;   // relative residual estimates
};

// Batched (F)GMRES from a zero initial guess: nrhs independent systems of
// length n in precision prec; Arnoldi by classical Gram-Schmidt applied
// twice; complex Givens rotations; system j stops at |g_{k+1}| <= tol ||b_j||.
// With a preconditioner M this is flexible GMRES (right preconditioning).
GmresResult gmres_batched(qcd_ctx* ctx, int prec, size_t n, int nrhs, const OpFn& A, const OpFn* M,
                          const void* b, void* x, double tol, int maxit, const std::string& tag) {
    cudaStream_t st = ctx->st;
    const size_t vs = n * nrhs;                 // one "vector set" (all rhs)
    const size_t eb = esz(prec);
    char* Vk = (char*)ctx->buf(tag + ".V", (size_t)(maxit + 1) * vs * eb);
    char* Zk = M ? (char*)ctx->buf(tag + ".Z", (size_t)maxit * vs * eb) : nullptr;
    void* w = ctx->buf(tag + ".w", vs * eb);
    double2* dd = (double2*)ctx->buf(tag + ".dots", (size_t)(2 * (maxit + 2) + 2) * nrhs * sizeof(double2));
    double2* part = (double2*)ctx->buf(tag + ".part", (size_t)(maxit + 2) * nrhs * 64 * sizeof(double2));
    double2* coef = (double2*)ctx->buf(tag + ".coef", (size_t)(maxit + 1) * nrhs * sizeof(double2));
    double2* h1 = dd;
    double2* h2 = dd + (size_t)(maxit + 1) * nrhs;
    double2* nr = dd + (size_t)2 * (maxit + 1) * nrhs;

    GmresResult out;
    out.iters.assign(nrhs, 0);
    out.resest.assign(nrhs, 1.0);
    // beta_j = ||b_j||
    blas_multidot(prec, b, 1, vs, b, nrhs, n, nr, part, ctx->dot_counters(nrhs), st);
    const double2* hb = ctx->fetch(nr, nrhs);
    std::vector<double> beta(nrhs);
    std::vector<double2> scl(nrhs);
    for (int j = 0; j < nrhs; ++j) {
        beta[j] = std::sqrt(std::max(hb[j].x, 0.0));
        scl[j] = make_double2(beta[j] > 0 ? 1.0 / beta[j] : 0.0, 0.0);
    }
    blas_zero(prec, x, vs, st);
    CK(cudaMemcpyAsync(coef, scl.data(), nrhs * sizeof(double2), cudaMemcpyHostToDevice, st));
    blas_scale_dev(prec, b, Vk, coef, nrhs, n, false, false, st);
    std::vector<std::vector<cd>> H(nrhs, std::vector<cd>((size_t)(maxit + 1) * maxit, 0.0));
    std::vector<std::vector<double>> cs(nrhs, std::vector<double>(maxit, 0.0));
    std::vector<std::vector<cd>> sn(nrhs, std::vector<cd>(maxit, 0.0));
    std::vector<std::vector<cd>> g(nrhs, std::vector<cd>(maxit + 1, 0.0));
    std::vector<char> active(nrhs, 0);
    int nactive = 0;
    for (int j = 0; j < nrhs; ++j) {
        g[j][0] = beta[j];
        active[j] = beta[j] > 0;
        nactive += active[j];
    }
    int steps = 0;
    for (int it = 0; it < maxit && nactive > 0; ++it) {
        void* vj = Vk + (size_t)it * vs * eb;
        if (M) {
            void* zj = Zk + (size_t)it * vs * eb;
            (*M)(vj, zj, nullptr);
            A(zj, w, nullptr);
        } else {
            A(vj, w, nullptr);
        }
        blas_multidot(prec, Vk, it + 1, vs, w, nrhs, n, h1, part, ctx->dot_counters((size_t)(it + 1) * nrhs), st);
        blas_multiaxpy(prec, Vk, it + 1, vs, h1, -1.0, w, nrhs, n, st);
        blas_multidot(prec, Vk, it + 1, vs, w, nrhs, n, h2, part, ctx->dot_counters((size_t)(it + 1) * nrhs), st);
        blas_multiaxpy(prec, Vk, it + 1, vs, h2, -1.0, w, nrhs, n, st);
        blas_multidot(prec, w, 1, vs, w, nrhs, n, nr, part, ctx->dot_counters(nrhs), st);
        check_launch("gmres iteration");
        const double2* hh = ctx->fetch(dd, (size_t)(2 * (maxit + 1) + 1) * nrhs);
        const double2* hh1 = hh;
        const double2* hh2 = hh + (size_t)(maxit + 1) * nrhs;
        const double2* hnr = hh + (size_t)2 * (maxit + 1) * nrhs;
        for (int j = 0; j < nrhs; ++j) {
            double hn = std::sqrt(std::max(hnr[j].x, 0.0));
            scl[j] = make_double2(hn > 0 ? 1.0 / hn : 0.0, 0.0);
            if (!active[j]) continue;
            auto& Hj = H[j];
            for (int i = 0; i <= it; ++i)
                Hj[(size_t)i * maxit + it] = cd(hh1[i * nrhs + j].x + hh2[i * nrhs + j].x,
                                                hh1[i * nrhs + j].y + hh2[i * nrhs + j].y);
            Hj[(size_t)(it + 1) * maxit + it] = hn;
            for (int i = 0; i < it; ++i) {
                cd a = Hj[(size_t)i * maxit + it], c = Hj[(size_t)(i + 1) * maxit + it];
                Hj[(size_t)i * maxit + it] = cs[j][i] * a + sn[j][i] * c;
                Hj[(size_t)(i + 1) * maxit + it] = -std::conj(sn[j][i]) * a + cs[j][i] * c;
            }
            cd a = Hj[(size_t)it * maxit + it], c = Hj[(size_t)(it + 1) * maxit + it];
            double aa = std::abs(a), rr = std::sqrt(aa * aa + std::norm(c));
            if (aa > 0) {
                cs[j][it] = aa / rr;
                sn[j][it] = (a / aa) * std::conj(c) / rr;
            } else {
                cs[j][it] = 0.0;
                sn[j][it] = 1.0;
            }
            Hj[(size_t)it * maxit + it] = cs[j][it] * a + sn[j][it] * c;
            Hj[(size_t)(it + 1) * maxit + it] = 0.0;
            g[j][it + 1] = -std::conj(sn[j][it]) * g[j][it];
            g[j][it] = cs[j][it] * g[j][it];
            out.iters[j] = it + 1;
            out.resest[j] = beta[j] > 0 ? std::abs(g[j][it + 1]) / beta[j] : 0.0;
            if (std::abs(g[j][it + 1]) <= tol * beta[j]) {
                active[j] = 0;
                --nactive;
            }
        }
        steps = it + 1;
        if (nactive == 0 || it + 1 == maxit) break;
        CK(cudaMemcpyAsync(coef, scl.data(), nrhs * sizeof(double2), cudaMemcpyHostToDevice, st));
        blas_scale_dev(prec, w, Vk + (size_t)(it + 1) * vs * eb, coef, nrhs, n, false, false, st);
    }
    // x_j = sum_i y_ji (Z or V)_i
    if (steps > 0) {
        std::vector<double2> cf((size_t)steps * nrhs, make_double2(0, 0));
        for (int j = 0; j < nrhs; ++j) {
            int k = out.iters[j];
            std::vector<cd> y(k, 0.0);
            for (int i = k - 1; i >= 0; --i) {
                cd s = g[j][i];
                for (int l = i + 1; l < k; ++l) s -= H[j][(size_t)i * maxit + l] * y[l];
                cd d = H[j][(size_t)i * maxit + i];
                y[i] = std::abs(d) > 0 ? s / d : 0.0;
            }
            for (int i = 0; i < k; ++i) cf[(size_t)i * nrhs + j] = make_double2(y[i].real(), y[i].imag());
        }
        CK(cudaMemcpyAsync(coef, cf.data(), cf.size() * sizeof(double2), cudaMemcpyHostToDevice, st));
        blas_multiaxpy(prec, M ? (const void*)Zk : (const void*)Vk, steps, vs, coef, 1.0, x, nrhs, n, st);
        check_launch("gmres update");
        CK(cudaStreamSynchronize(st));   // coef and scl live on the host stack
    }
    return out;
}

// Batched (F)GMRES with device-side control: the same algorithm as
// gmres_batched (CGS twice, Givens), but the Hessenberg bookkeeping runs in
// kry_* kernels and converged right-hand sides are skipped through the
// device `active` flags, so the solve is one launch sequence with no host
// round trip.  `outer_act` (may be null) masks right-hand sides from the start.
// poll > 0: every `poll` steps the host reads the active flags (one small
// copy) and stops once every right-hand side has converged, so a solve that
// usually ends far below maxit launches only the steps it needs.
struct DevGmresOut {
    KryDev K;
    int steps = 0;   // steps launched
};
DevGmresOut gmres_dev(qcd_ctx* ctx, int prec, size_t n, int nrhs, const OpFn& A, const OpFn* M, const void* b,
                      void* x, double tol, int maxit, const std::string& tag, const int* outer_act, int poll = 0) {
    cudaStream_t st = ctx->st;
    if (maxit > kMaxKry) throw QcdError(QCD_EINVAL, "too many Krylov steps");
    const size_t vs = n * nrhs;
    const size_t eb = esz(prec);
    char* Vk = (char*)ctx->buf(tag + ".V", (size_t)(maxit + 1) * vs * eb);
    char* Zk = M ? (char*)ctx->buf(tag + ".Z", (size_t)maxit * vs * eb) : nullptr;
    void* w = ctx->buf(tag + ".w", vs * eb);
    double2* h1 = (double2*)ctx->buf(tag + ".h1", (size_t)(maxit + 1) * nrhs * sizeof(double2));
    double2* h2 = (double2*)ctx->buf(tag + ".h2", (size_t)(maxit + 1) * nrhs * sizeof(double2));
    double2* nr = (double2*)ctx->buf(tag + ".nr", (size_t)nrhs * sizeof(double2));
    double2* part = (double2*)ctx->buf(tag + ".part", (size_t)(maxit + 2) * nrhs * 64 * sizeof(double2));
    KryDev K = kry_layout(ctx->buf(tag + ".K", kry_bytes(nrhs, maxit)), nrhs, maxit, tol);
    blas_multidot(prec, b, 1, vs, b, nrhs, n, nr, part, ctx->dot_counters(nrhs), st);
    kry_init(K, nr, outer_act, st);
    blas_zero(prec, x, vs, st);
    blas_scale_dev(prec, b, Vk, K.scale, nrhs, n, false, false, st, K.active);
    int steps = 0;
    for (int it = 0; it < maxit; ++it) {
        void* vj = Vk + (size_t)it * vs * eb;
        if (M) {
            void* zj = Zk + (size_t)it * vs * eb;
            (*M)(vj, zj, K.active);
            A(zj, w, K.active);
        } else {
            A(vj, w, K.active);
        }
        blas_multidot(prec, Vk, it + 1, vs, w, nrhs, n, h1, part, ctx->dot_counters((size_t)(it + 1) * nrhs), st, K.active);
        blas_multiaxpy(prec, Vk, it + 1, vs, h1, -1.0, w, nrhs, n, st, K.active);
        blas_multidot(prec, Vk, it + 1, vs, w, nrhs, n, h2, part, ctx->dot_counters((size_t)(it + 1) * nrhs), st, K.active);
        blas_multiaxpy(prec, Vk, it + 1, vs, h2, -1.0, w, nrhs, n, st, K.active);
        blas_multidot(prec, w, 1, vs, w, nrhs, n, nr, part, ctx->dot_counters(nrhs), st, K.active);
        kry_step(K, it, h1, h2, nr, st);
        if (it + 1 < maxit) blas_scale_dev(prec, w, Vk + (size_t)(it + 1) * vs * eb, K.scale, nrhs, n, false, false, st,
                                           K.active);
        steps = it + 1;
        if (poll > 0 && steps % poll == 0 && steps < maxit) {
            // (the staging buffer is taken here: preconditioner calls may regrow it)
            int* hact = (int*)ctx->host(((size_t)nrhs * sizeof(int) + sizeof(double2) - 1) / sizeof(double2));
            CK(cudaMemcpyAsync(hact, K.active, nrhs * sizeof(int), cudaMemcpyDeviceToHost, st));
            CK(cudaStreamSynchronize(st));
            bool any = false;
            for (int j = 0; j < nrhs; ++j) any = any || hact[j] != 0;
            if (!any) break;
        }
    }
    kry_finish(K, st);
    if (steps > 0)
        blas_multiaxpy(prec, M ? (const void*)Zk : (const void*)Vk, steps, vs, K.coef, 1.0, x, nrhs, n, st, outer_act);
    check_launch("gmres_dev");
    DevGmresOut out;
    out.K = K;
    out.steps = steps;
    return out;
}

// per-right-hand-side steps of a finished gmres_dev (one device-to-host copy)
std::vector<int> kry_iters(qcd_ctx* ctx, const KryDev& K) {
    std::vector<int> it(K.nrhs);
    CK(cudaMemcpyAsync(it.data(), K.k, K.nrhs * sizeof(int), cudaMemcpyDeviceToHost, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    return it;
}

// ------------------------------------------------------------------ hierarchy pieces
void require_gauge(qcd_ctx* ctx) {
    if (!ctx->have_gauge) throw QcdError(QCD_ENOTSETUP, "no gauge field: call qcd_set_gauge first");
}
void require_mg(qcd_ctx* ctx) {
    require_gauge(ctx);
    if (!ctx->c.ready) throw QcdError(QCD_ENOTSETUP, "no multigrid hierarchy: call qcd_mg_setup first");
}

Blocking make_blocking(const Geom& g, const int b[4]) {
    Blocking B;
    B.bs = 1;
    B.nb = 1;
    for (int mu = 0; mu < 4; ++mu) {
        if (b[mu] < 1 || g.L[mu] % b[mu]) throw QcdError(QCD_EINVAL, "block extents must divide the lattice");
        B.b[mu] = b[mu];
        B.cd[mu] = g.L[mu] / b[mu];
        B.bs *= b[mu];
        B.nb *= B.cd[mu];
    }
    return B;
}

void ensure_sap(qcd_ctx* ctx) {
    if (ctx->have_sap) return;
    Blocking B = make_blocking(ctx->f.g, ctx->p.sap_block);
    for (int mu = 0; mu < 4; ++mu)
        if (B.cd[mu] % 2) throw QcdError(QCD_EINVAL, "SAP needs an even number of blocks in every direction");
    if (B.bs & (B.bs - 1) || B.bs > 1024) throw QcdError(QCD_EINVAL, "SAP block sites must be a power of two <= 1024");
    std::vector<int> lists[2];
    for (int b = 0; b < B.nb; ++b) {
        int t = b, c3 = t % B.cd[3]; t /= B.cd[3];
        int c2 = t % B.cd[2]; t /= B.cd[2];
        int c1 = t % B.cd[1], c0 = t / B.cd[1];
        lists[(c0 + c1 + c2 + c3) % 2].push_back(b);
    }
    for (int c = 0; c < 2; ++c) {
        CK(cudaMalloc(&ctx->sap.blocks_of_colour[c], lists[c].size() * sizeof(int)));
        CK(cudaMemcpy(ctx->sap.blocks_of_colour[c], lists[c].data(), lists[c].size() * sizeof(int), cudaMemcpyHostToDevice));
        ctx->sap.ncol[c] = (int)lists[c].size();
    }
    ctx->sap.B = B;
    ctx->have_sap = true;
}

// nu SAP sweeps (Eq. 2.10) on op(tau) x = b, x updated in place
void sap_smooth(qcd_ctx* ctx, int prec, int op, int nrhs, const void* b, void* x, const double* tau, int sweeps,
                double tol, const int* act = nullptr) {
    ensure_sap(ctx);
    const size_t n = ctx->nfine();
    void* r = ctx->buf("sap.r", n * nrhs * esz(prec));
    void* scr = ctx->buf("sap.scratch", sap_scratch_bytes(ctx->sap, prec, nrhs, ctx->p.sap_block_iters));
    for (int s = 0; s < sweeps; ++s) {
        for (int colour = 0; colour < 2; ++colour) {
            residual_op(ctx->f, prec, op, nrhs, b, x, r, tau, ctx->st, act);
            sap_blocks(ctx->f, ctx->sap, colour, prec, op, nrhs, r, x, tau, ctx->p.sap_block_iters, tol, scr, ctx->st,
                       act, ctx->p.sap_half != 0);
        }
    }
    check_launch("sap");
}

void smooth(qcd_ctx* ctx, int prec, int op, int nrhs, const void* b, void* x, const double* tau,
            const int* act = nullptr) {
    if (ctx->p.nu <= 0) return;
    if (ctx->p.smoother == QCD_SMOOTHER_SAP) {
        sap_smooth(ctx, prec, op, nrhs, b, x, tau, ctx->p.nu, ctx->p.sap_block_tol, act);
        return;
    }
    const size_t n = ctx->nfine();
    void* r = ctx->buf("gsm.r", n * nrhs * esz(prec));
    void* e = ctx->buf("gsm.e", n * nrhs * esz(prec));
    std::vector<double> tv(tau, tau + nrhs);
    OpFn A = [ctx, prec, op, nrhs, tv](const void* in, void* out, const int* a) {
        apply_op(ctx->f, prec, op, nrhs, in, out, tv.data(), ctx->st, a);
    };
    double2* one = (double2*)ctx->buf("gsm.one", (size_t)nrhs * sizeof(double2));
    {
        std::vector<double2> ones(nrhs, make_double2(1, 0));
        CK(cudaMemcpyAsync(one, ones.data(), nrhs * sizeof(double2), cudaMemcpyHostToDevice, ctx->st));
    }
    for (int s = 0; s < ctx->p.nu; ++s) {
        residual_op(ctx->f, prec, op, nrhs, b, x, r, tau, ctx->st, act);
        gmres_dev(ctx, prec, n, nrhs, A, nullptr, r, e, 0.0, ctx->p.gmres_smooth_iters, "gsm", act);
        blas_scale_dev(prec, e, x, one, nrhs, n, false, true, ctx->st, act);
    }
}

// two-level cycle x = M b (Eq. 2.8, post-smoothing only)
void ensure_coarse64(qcd_ctx* ctx);

// Level-2 solve of the K-cycle: GMRES on the level-2 operator to coarse_tol,
// one cooperative launch per group (host-driven GMRES when cooperative
// launches are unavailable).
void level2_solve(qcd_ctx* ctx, int prec, int op, int nrhs, const void* rc, void* xc, const double* tau,
                  const double* taud, const int* act) {
    const Coarse& c2 = ctx->c2;
    const size_t nco2 = (size_t)c2.gc.V * c2.nc;
    const int maxit = std::min(ctx->p.coarse_maxiter, kMaxCoarse);
    bool done = !ctx->no_coop;
    if (done) {
        const int lay = ctx->p.coarse_layout;
        const int grp = std::min(nrhs, coarse_gmres_group(c2, prec, maxit, lay));
        if (grp < 1) throw QcdError(QCD_EINVAL, "level-2 GMRES: the coarse_layout asked for does not fit in shared memory");
        void* scr = ctx->buf("l2.scr", coarse_gmres_scratch(c2, prec, grp, maxit, lay));
        int* its = (int*)ctx->buf("l2.its", (size_t)nrhs * sizeof(int));
        double* res = (double*)ctx->buf("l2.res", (size_t)nrhs * sizeof(double));
        for (int j0 = 0; j0 < nrhs && done; j0 += grp) {
            const int nj = std::min(grp, nrhs - j0);
            const int rcode = coarse_gmres(c2, prec, op, nj, (const char*)rc + (size_t)j0 * nco2 * esz(prec),
                                           (char*)xc + (size_t)j0 * nco2 * esz(prec), taud + j0,
                                           act ? act + j0 : nullptr, ctx->p.coarse_tol, maxit, scr, its + j0,
                                           res + j0, ctx->counters(), lay, ctx->st);
            if (rcode != 0) {
                cudaGetLastError();
                if (j0 > 0) throw QcdError(QCD_ECUDA, "cooperative level-2 solve failed mid-batch");
                ctx->no_coop = true;
                done = false;
            }
        }
    }
    if (!done) {
        std::vector<double> tv(tau, tau + nrhs);
        OpFn A2 = [ctx, prec, op, nrhs, tv](const void* in, void* out, const int*) {
            coarse_apply(ctx->c2, prec, op, nrhs, in, out, tv.data(), ctx->st, ctx->p.coarse_tensor != 0);
        };
        gmres_batched(ctx, prec, nco2, nrhs, A2, nullptr, rc, xc, ctx->p.coarse_tol, ctx->p.coarse_maxiter, "l2g");
    }
}

// The level-1 two-level cycle of the K-cycle: x1 = P2 (level-2 solve of
// P2^H r1), then nu2 GMRES smoothing steps (gmres_smooth_iters each) on the
// level-1 system (D_c - tau Gamma5^c or Q_c - tau, as `op`).
void level1_cycle(qcd_ctx* ctx, int prec, int op, int nrhs, const void* r1, void* x1, const double* tau,
                  const double* taud, const int* act) {
    const Coarse& c = ctx->c;
    const Coarse& c2 = ctx->c2;
    const size_t nco = (size_t)c.gc.V * c.nc, nco2 = (size_t)c2.gc.V * c2.nc;
    void* rc2 = ctx->buf("l2.rc", nco2 * nrhs * esz(prec));
    void* xc2 = ctx->buf("l2.xc", nco2 * nrhs * esz(prec));
    blas_zero(prec, rc2, nco2 * nrhs, ctx->st);
    blas_zero(prec, x1, nco * nrhs, ctx->st);   // masked right-hand sides stay zero
    mg2_restrict(c, c2, prec, nrhs, r1, rc2, ctx->st, act);
    level2_solve(ctx, prec, op, nrhs, rc2, xc2, tau, taud, act);
    mg2_prolong(c, c2, prec, nrhs, xc2, x1, ctx->st, act);
    if (ctx->p.nu2 <= 0) return;
    std::vector<double> tv(tau, tau + nrhs);
    OpFn A1 = [ctx, prec, op, nrhs, tv](const void* in, void* out, const int*) {
        coarse_apply(ctx->c, prec, op, nrhs, in, out, tv.data(), ctx->st, ctx->p.coarse_tensor != 0);
    };
    void* w = ctx->buf("l1c.w", nco * nrhs * esz(prec));
    void* e = ctx->buf("l1c.e", nco * nrhs * esz(prec));
    double2* one = (double2*)ctx->buf("l1c.one", (size_t)nrhs * sizeof(double2));
    {
        std::vector<double2> ones(nrhs, make_double2(1, 0));
        CK(cudaMemcpyAsync(one, ones.data(), nrhs * sizeof(double2), cudaMemcpyHostToDevice, ctx->st));
    }
    for (int s = 0; s < ctx->p.nu2; ++s) {
        // w = r1 - A1 x1
        coarse_apply(c, prec, op, nrhs, x1, w, tv.data(), ctx->st, ctx->p.coarse_tensor != 0);
        blas_axpby(prec, make_double2(1, 0), r1, make_double2(-1, 0), w, nco * nrhs, ctx->st);
        gmres_dev(ctx, prec, nco, nrhs, A1, nullptr, w, e, 0.0, ctx->p.gmres_smooth_iters, "l1s", act);
        blas_scale_dev(prec, e, x1, one, nrhs, nco, false, true, ctx->st, act);
    }
}

void mg_cycle_impl(qcd_ctx* ctx, int prec, int op, int nrhs, const void* b, void* x, const double* tau,
                   const int* act = nullptr) {
    if (prec == QCD_FP64) ensure_coarse64(ctx);
    const Coarse& c = ctx->c;
    const size_t nco = (size_t)c.gc.V * c.nc;
    void* rc = ctx->buf("cyc.rc", nco * nrhs * esz(prec));
    void* xc = ctx->buf("cyc.xc", nco * nrhs * esz(prec));
    mg_restrict(ctx->f, c, prec, nrhs, b, rc, ctx->st, act);
    // coarse solve: one cooperative launch per group of <= kMaxCoarseRhs right-hand sides
    double* taud = (double*)ctx->buf("cyc.tau", (size_t)nrhs * sizeof(double));
    CK(cudaMemcpyAsync(taud, tau, nrhs * sizeof(double), cudaMemcpyHostToDevice, ctx->st));
    if (ctx->p.levels == 3 && ctx->c2.ready) {
        // K-cycle: FGMRES on the level-1 operator to coarse_tol, preconditioned
        // by the level-1 two-level cycle.  Device-controlled (Givens and
        // stopping in kry_* kernels, converged right-hand sides skipped); the
        // host looks at the active flags every 4 steps to stop early.
        std::vector<double> tv(tau, tau + nrhs);
        OpFn A1 = [ctx, prec, op, nrhs, tv](const void* in, void* out, const int*) {
            coarse_apply(ctx->c, prec, op, nrhs, in, out, tv.data(), ctx->st, ctx->p.coarse_tensor != 0);
        };
        OpFn M1 = [ctx, prec, op, nrhs, tv, taud, act](const void* in, void* out, const int* a) {
            level1_cycle(ctx, prec, op, nrhs, in, out, tv.data(), taud, a ? a : act);
        };
        const int kmax = std::min(ctx->p.coarse_maxiter, kMaxKry);
        gmres_dev(ctx, prec, nco, nrhs, A1, &M1, rc, xc, ctx->p.coarse_tol, kmax, "kc1", act, 4);
        mg_prolong(ctx->f, c, prec, nrhs, xc, x, false, ctx->st, act);
        smooth(ctx, prec, op, nrhs, b, x, tau, act);
        check_launch("mg k-cycle");
        return;
    }
    const int maxit = std::min(ctx->p.coarse_maxiter, kMaxCoarse);
    bool done = !ctx->no_coop;
    if (done) {
        const int lay = ctx->p.coarse_layout;
        const int grp = std::min(nrhs, coarse_gmres_group(c, prec, maxit, lay));
        if (grp < 1) throw QcdError(QCD_EINVAL, "coarse GMRES: the coarse_layout asked for does not fit in shared memory");
        void* scr = ctx->buf("cyc.scr", coarse_gmres_scratch(c, prec, grp, maxit, lay));
        int* its = (int*)ctx->buf("cyc.its", (size_t)nrhs * sizeof(int));
        double* res = (double*)ctx->buf("cyc.res", (size_t)nrhs * sizeof(double));
        for (int j0 = 0; j0 < nrhs && done; j0 += grp) {
            const int nj = std::min(grp, nrhs - j0);
            int rcode = coarse_gmres(c, prec, op, nj, (const char*)rc + (size_t)j0 * nco * esz(prec),
                                     (char*)xc + (size_t)j0 * nco * esz(prec), taud + j0, act ? act + j0 : nullptr,
                                     ctx->p.coarse_tol, maxit, scr, its + j0, res + j0, ctx->counters(), lay,
                                     ctx->st);
            if (rcode != 0) {
                cudaGetLastError();
                if (j0 > 0) throw QcdError(QCD_ECUDA, "cooperative coarse solve failed mid-batch");
                ctx->no_coop = true;
                done = false;
            }
        }
    }
    if (!done) {
        std::vector<double> tv(tau, tau + nrhs);
        OpFn Ac = [ctx, prec, op, nrhs, tv](const void* in, void* out, const int*) {
            coarse_apply(ctx->c, prec, op, nrhs, in, out, tv.data(), ctx->st, ctx->p.coarse_tensor != 0);
        };
        gmres_batched(ctx, prec, nco, nrhs, Ac, nullptr, rc, xc, ctx->p.coarse_tol, ctx->p.coarse_maxiter, "coarse");
    }
    mg_prolong(ctx->f, c, prec, nrhs, xc, x, false, ctx->st, act);
    smooth(ctx, prec, op, nrhs, b, x, tau, act);
    check_launch("mg cycle");
}

void normalize_set(qcd_ctx* ctx, double2* X, int nvec, size_t n) {
    double2* nr = (double2*)ctx->buf("nrm.d", nvec * sizeof(double2));
    double2* part = (double2*)ctx->buf("nrm.part", (size_t)nvec * 64 * sizeof(double2));
    blas_multidot(QCD_FP64, X, 1, (size_t)nvec * n, X, nvec, n, nr, part, ctx->dot_counters(nvec), ctx->st);
    const double2* h = ctx->fetch(nr, nvec);
    std::vector<double2> s(nvec);
    for (int i = 0; i < nvec; ++i) s[i] = make_double2(h[i].x > 0 ? 1.0 / std::sqrt(h[i].x) : 0.0, 0.0);
    double2* sd = (double2*)ctx->buf("nrm.s", nvec * sizeof(double2));
    CK(cudaMemcpyAsync(sd, s.data(), nvec * sizeof(double2), cudaMemcpyHostToDevice, ctx->st));
    blas_scale_dev(QCD_FP64, X, X, sd, nvec, n, false, false, ctx->st);
    CK(cudaStreamSynchronize(ctx->st));
}

// the FP64 coarse operator, rebuilt if only the FP32 one is current
void ensure_coarse64(qcd_ctx* ctx) {
    if (ctx->c.a64_stale) {
        mg_build_coarse(ctx->f, ctx->c, ctx->st, false);
        check_launch("coarse rebuild");
    }
}

// Third level (reading of Sec. 2 applied recursively): its test vectors are
// the first nv2 fine test vectors restricted by P^H; P2 aggregates blocks of
// params.agg2 level-1 sites; the level-2 operator is P2^H D_c P2 in FP64 (and
// an FP32 copy).
void build_level2(qcd_ctx* ctx, const double2* V, int nvec) {
    const Coarse& c = ctx->c;
    Coarse& c2 = ctx->c2;
    const int nv2 = ctx->p.nv2;
    if (nv2 > nvec) throw QcdError(QCD_EINVAL, "nv2 exceeds the number of fine test vectors");
    Blocking B2 = make_blocking(c.gc, ctx->p.agg2);
    if (B2.bs * c.nv < nv2) throw QcdError(QCD_EINVAL, "level-2 aggregate smaller than nv2");
    const bool realloc = !c2.P64 || c2.nv != nv2 || memcmp(c2.B.b, B2.b, sizeof(B2.b)) != 0 ||
                         memcmp(c2.B.cd, B2.cd, sizeof(B2.cd)) != 0 || ctx->c2_nv1 != c.nv;
    if (realloc) {
        ctx->drop_level2();
        c2.B = B2;
        c2.nv = nv2;
        c2.nc = 2 * nv2;
        c2.ctas = ctx->p.coarse_ctas;
        for (int mu = 0; mu < 4; ++mu) c2.gc.L[mu] = B2.cd[mu];
        c2.gc.V = B2.nb;
        c2.gc.antiperiodic = 0;
        const size_t np = (size_t)B2.nb * 2 * nv2 * B2.bs * c.nv;
        const size_t na = (size_t)B2.nb * 9 * c2.nc * c2.nc;
        CK(cudaMalloc(&c2.P64, np * sizeof(double2)));
        CK(cudaMalloc(&c2.P32, np * sizeof(float2)));
        CK(cudaMalloc(&c2.A64, na * sizeof(double2)));
        CK(cudaMalloc(&c2.A32, na * sizeof(float2)));
        ctx->c2_nv1 = c.nv;
    }
    // an FP64 context builds level 2 from the FP64 level-1 operator; a
    // mixed-precision one from the FP32 operator its cycles use (no FP64
    // Galerkin rebuild per interpolation update)
    if (ctx->p.precision == QCD_FP64) ensure_coarse64(ctx);
    const size_t nco = (size_t)c.gc.V * c.nc;
    double2* W2 = (double2*)ctx->buf("l2.W", (size_t)nv2 * nco * sizeof(double2));
    mg_restrict(ctx->f, c, QCD_FP64, nv2, V, W2, ctx->st);
    mg2_build_P(c, c2, W2, ctx->st);
    mg2_build_coarse(c, c2, ctx->st);
    check_launch("level-2 build");
    c2.ready = true;
}

void build_from_vectors(qcd_ctx* ctx, const double2* V, int nvec, const int block[4]) {
    Coarse& c = ctx->c;
    Blocking B = make_blocking(ctx->f.g, block);
    if (nvec < 1 || nvec > 32) throw QcdError(QCD_EINVAL, "need 1 <= Nv <= 32");
    if (B.bs * 6 < nvec) throw QcdError(QCD_EINVAL, "aggregate smaller than Nv");
    bool realloc = !c.P64 || c.nv != nvec || memcmp(c.B.b, B.b, sizeof(B.b)) != 0;
    if (realloc) {
        auto fr = [](void* q) { if (q) cudaFree(q); };
        fr(c.P64); fr(c.P32); fr(c.A64); fr(c.A32);
        c.P64 = nullptr; c.P32 = nullptr; c.A64 = nullptr; c.A32 = nullptr;
        c.B = B;
        c.nv = nvec;
        c.nc = 2 * nvec;
        c.ctas = ctx->p.coarse_ctas;
        for (int mu = 0; mu < 4; ++mu) c.gc.L[mu] = B.cd[mu];
        c.gc.V = B.nb;
        c.gc.antiperiodic = 0;
        size_t np = (size_t)B.nb * 2 * nvec * B.bs * 6;
        size_t na = (size_t)B.nb * 9 * c.nc * c.nc;
        CK(cudaMalloc(&c.P64, np * sizeof(double2)));
        CK(cudaMalloc(&c.P32, np * sizeof(float2)));
        CK(cudaMalloc(&c.A64, na * sizeof(double2)));
        CK(cudaMalloc(&c.A32, na * sizeof(float2)));
    }
    mg_build_P(ctx->f, c, V, nvec, ctx->st);
    // a mixed-precision context runs its cycles in FP32: build only that
    // operator; FP64 users rebuild the FP64 one on demand (ensure_coarse64)
    mg_build_coarse(ctx->f, c, ctx->st, ctx->p.precision != QCD_FP64);
    check_launch("mg build");
    c.ready = true;
    if (ctx->p.levels == 3) build_level2(ctx, V, nvec);
    else ctx->c2.ready = false;
}

void mg_setup_impl(qcd_ctx* ctx, int Nv, const int block[4]) {
    require_gauge(ctx);
    const size_t n = ctx->nfine();
    const int prec = ctx->p.precision == QCD_FP64 ? QCD_FP64 : QCD_FP32;
    if (ctx->test_vectors) CK(cudaFree(ctx->test_vectors));
    ctx->test_vectors = nullptr;
    CK(cudaMalloc(&ctx->test_vectors, (size_t)Nv * n * sizeof(double2)));
    ctx->n_test = Nv;
    double2* W = ctx->test_vectors;
    blas_gaussian(W, (size_t)Nv * n, ctx->p.seed, 0x5e7000000000ull, ctx->st);
    std::vector<double> zero_tau(Nv, 0.0);
    void* wp = ctx->buf("setup.w", (size_t)Nv * n * esz(prec));
    void* bp = ctx->buf("setup.b", (size_t)Nv * n * esz(prec));
    void* xp = ctx->buf("setup.x", (size_t)Nv * n * esz(prec));
    // iteration 1: smooth D x = 0 starting from the random vectors
    blas_convert(QCD_FP64, W, prec, wp, (size_t)Nv * n, ctx->st);
    blas_zero(prec, bp, (size_t)Nv * n, ctx->st);
    smooth(ctx, prec, QCD_OP_D, Nv, bp, wp, zero_tau.data());
    blas_convert(prec, wp, QCD_FP64, W, (size_t)Nv * n, ctx->st);
    normalize_set(ctx, W, Nv, n);
    build_from_vectors(ctx, W, Nv, block);
    // later iterations: w <- M w (inverse iteration with the current cycle)
    for (int it = 1; it < ctx->p.setup_iters; ++it) {
        blas_convert(QCD_FP64, W, prec, bp, (size_t)Nv * n, ctx->st);
        mg_cycle_impl(ctx, prec, QCD_OP_D, Nv, bp, xp, zero_tau.data());
        blas_convert(prec, xp, QCD_FP64, W, (size_t)Nv * n, ctx->st);
        normalize_set(ctx, W, Nv, n);
        build_from_vectors(ctx, W, Nv, block);
    }
    CK(cudaStreamSynchronize(ctx->st));
    // the setup work fields (3 Nv fine fields) are not needed afterwards
    ctx->drop_buf("setup.w");
    ctx->drop_buf("setup.b");
    ctx->drop_buf("setup.x");
}

// ------------------------------------------------------------------ shifted solves
// Correction solves: nrhs systems op(tau_j) t_j = rhs_j to inner_tol (or tol),
// in precision prec, FGMRES + MG or plain GMRES.  Returns iterations.
GmresResult inner_solve(qcd_ctx* ctx, int prec, int op, int nrhs, const void* rhs, void* t, const double* tau,
                        double tol, int maxit) {
    const size_t n = ctx->nfine();
    std::vector<double> tv(tau, tau + nrhs);
    OpFn A = [ctx, prec, op, nrhs, tv](const void* in, void* out, const int* a) {
        apply_op(ctx->f, prec, op, nrhs, in, out, tv.data(), ctx->st, a);
    };
    DevGmresOut d;
    if (ctx->p.use_mg) {
        require_mg(ctx);
        OpFn M = [ctx, prec, op, nrhs, tv](const void* in, void* out, const int* a) {
            mg_cycle_impl(ctx, prec, op, nrhs, in, out, tv.data(), a);
        };
        d = gmres_dev(ctx, prec, n, nrhs, A, &M, rhs, t, tol, maxit, "fine", nullptr);
    } else {
        d = gmres_dev(ctx, prec, n, nrhs, A, nullptr, rhs, t, tol, maxit, "fine", nullptr);
    }
    GmresResult out;
    out.iters = kry_iters(ctx, d.K);
    out.resest.assign(nrhs, 0.0);
    return out;
}

// (Q - tau_j) x_j = b_j to relative tol, FP64 residuals; b, x arrays of
// nrhs FP64 fields (contiguous).  Returns the max relative residual.
double shifted_solve_impl(qcd_ctx* ctx, int nrhs, const double2* b, double2* x, const double* tau, double tol,
                          qcd_solve_info* info) {
    require_gauge(ctx);
    const size_t n = ctx->nfine();
    const int form = ctx->p.correction_form;
    const int prec = ctx->p.precision == QCD_FP64 ? QCD_FP64 : QCD_FP32;
    double2* r = (double2*)ctx->buf("ss.r", n * nrhs * sizeof(double2));
    double2* rr = (double2*)ctx->buf("ss.rr", n * nrhs * sizeof(double2));
    void* rl = ctx->buf("ss.rl", n * nrhs * esz(prec));
    void* tl = ctx->buf("ss.tl", n * nrhs * esz(prec));
    double2* nr = (double2*)ctx->buf("ss.nr", 2 * nrhs * sizeof(double2));
    double2* part = (double2*)ctx->buf("ss.part", (size_t)2 * nrhs * 64 * sizeof(double2));
    blas_multidot(QCD_FP64, b, 1, n * nrhs, b, nrhs, n, nr, part, ctx->dot_counters(nrhs), ctx->st);
    std::vector<double> bn(nrhs);
    {
        const double2* h = ctx->fetch(nr, nrhs);
        for (int j = 0; j < nrhs; ++j) bn[j] = std::sqrt(h[j].x);
    }
    blas_zero(QCD_FP64, x, n * nrhs, ctx->st);
    blas_copy(QCD_FP64, b, r, n * nrhs, ctx->st);
    const double floor_tol = prec == QCD_FP64 ? 1e-13 : 2e-5;
    int iters = 0, refine = 0;
    double worst = 1.0;
    const int max_refine = 200;
    const int restart = std::max(ctx->p.inner_maxiter, 20);
    std::vector<double> relres(nrhs, 1.0);
    // best iterate of each right-hand side so far (returned on ENOCONV)
    double2* xbest = (double2*)ctx->buf("ss.xbest", n * nrhs * sizeof(double2));
    std::vector<double> best(nrhs, INFINITY);
    for (;; ++refine) {
        // current residuals
        blas_multidot(QCD_FP64, r, 1, n * nrhs, r, nrhs, n, nr, part, ctx->dot_counters(nrhs), ctx->st);
        const double2* h = ctx->fetch(nr, nrhs);
        worst = 0.0;
        for (int j = 0; j < nrhs; ++j) {
            relres[j] = bn[j] > 0 ? std::sqrt(h[j].x) / bn[j] : 0.0;
            worst = std::max(worst, relres[j]);
        }
        for (int j = 0; j < nrhs; ++j)
            if (relres[j] < best[j]) {
                best[j] = relres[j];
                blas_copy(QCD_FP64, x + (size_t)j * n, xbest + (size_t)j * n, n, ctx->st);
            }
        if (worst <= tol) break;
        if (refine == max_refine) {
            // cap reached: return the best iterate of every right-hand side
            blas_copy(QCD_FP64, xbest, x, n * nrhs, ctx->st);
            worst = *std::max_element(best.begin(), best.end());
            break;
        }
        // correction equation on the chosen form: (D - tau G5) c = G5 r or (Q - tau) c = r
        if (form == QCD_OP_D) blas_gamma5(QCD_FP64, r, rr, (size_t)ctx->f.g.V * nrhs, ctx->st);
        else blas_copy(QCD_FP64, r, rr, n * nrhs, ctx->st);
        blas_convert(QCD_FP64, rr, prec, rl, n * nrhs, ctx->st);
        double itol = std::max(floor_tol, std::min(0.5, 0.5 * tol / std::max(worst, 1e-300)));
        GmresResult g = inner_solve(ctx, prec, form, nrhs, rl, tl, tau, itol, restart);
        iters += *std::max_element(g.iters.begin(), g.iters.end());
        blas_convert(prec, tl, QCD_FP64, rr, n * nrhs, ctx->st);
        blas_axpby(QCD_FP64, make_double2(1, 0), rr, make_double2(1, 0), x, n * nrhs, ctx->st);
        residual_op(ctx->f, QCD_FP64, QCD_OP_Q, nrhs, b, x, r, tau, ctx->st);
        check_launch("refinement");
    }
    if (info) {
        info->iterations = iters;
        info->refinements = refine;
        info->residual = worst;
    }
    return worst;
}

// ------------------------------------------------------------------ GD-lambda-AMG
// G[i][m] = d1[i], G[m][i] = conj d1[i]; Hm[i][m] = d2[i]; Hm[m][i] = conj d2[i]  (ld = column stride).
// H = W^H V = V^H Q V is Hermitian because Q is (Sec. 2), so its new row
// is the conjugate of its new column.
__global__ void gram_update_kernel(double2* G, double2* Hm, int ld, int m, const double2* d1, const double2* d2) {
    int i = threadIdx.x;
    if (i > m) return;
    G[(size_t)m * ld + i] = d1[i];
    G[(size_t)i * ld + m] = conj(d1[i]);
    Hm[(size_t)m * ld + i] = d2[i];
    Hm[(size_t)i * ld + m] = conj(d2[i]);
}
__global__ void gather_columns_kernel(const double2* S, int m, const int* idx, int p, double2* out) {
    for (int e = threadIdx.x; e < m * p; e += blockDim.x) out[e] = S[(size_t)idx[e / m] * m + e % m];
}
// Deflation of a converged direction s (a column of S, m entries) by the
// Householder reflector Hh = I - f w w^H that maps s/||s|| to a multiple of
// e_0: w = s/||s|| + e^{i arg s_0} e_0, f = 2 / (w^H w).  Columns 1..m-1 of
// Hh are orthonormal and orthogonal to s.  Writes w to hw[0..m) and f to
// hw[m].x.
__global__ void householder_vector_kernel(const double2* __restrict__ s, int m, double2* __restrict__ hw) {
    __shared__ double nn, ww;
    if (threadIdx.x == 0) {
        double a = 0;
        for (int i = 0; i < m; ++i) a += s[i].x * s[i].x + s[i].y * s[i].y;
        nn = a > 0 ? 1.0 / sqrt(a) : 0.0;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const double2 s0 = nn * s[0];
        const double a0 = sqrt(s0.x * s0.x + s0.y * s0.y);
        const double2 ph = a0 > 0 ? (1.0 / a0) * s0 : make_double2(1, 0);
        // w^H w = 2 (1 + |s_0|) for unit s
        ww = 2.0 * (1.0 + a0);
        hw[0] = s0 + ph;
    }
    for (int i = 1 + threadIdx.x; i < m; i += blockDim.x) hw[i] = nn * s[i];
    __syncthreads();
    if (threadIdx.x == 0) hw[m] = make_double2(2.0 / ww, 0.0);
}
// out = Hh M Hh restricted to rows and columns 1..m-1 (M: G or H, ld = ld):
//   out[i-1][j-1] = M_ij - f w_i conj(b_j) - f a_i conj(w_j) + f^2 g w_i conj(w_j)
// with a = M w, b = M^H w, g = w^H M w.  blockIdx.x selects (G, Gt) or (H, Ht).
__global__ void householder_gram_kernel(const double2* __restrict__ G, double2* __restrict__ Gt,
                                        const double2* __restrict__ Hm, double2* __restrict__ Hmt, int m, int ld,
                                        const double2* __restrict__ hw) {
    __shared__ double2 w[kMaxBasis + 1], a[kMaxBasis], b[kMaxBasis];
    __shared__ double2 g;
    const double2* M = blockIdx.x ? Hm : G;
    double2* out = blockIdx.x ? Hmt : Gt;
    for (int i = threadIdx.x; i <= m; i += blockDim.x) w[i] = hw[i];
    __syncthreads();
    const double f = w[m].x;
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
        double2 ai = make_double2(0, 0), bi = make_double2(0, 0);
        for (int k = 0; k < m; ++k) {
            ai += M[(size_t)k * ld + i] * w[k];
            bi += conj(M[(size_t)i * ld + k]) * w[k];
        }
        a[i] = ai;
        b[i] = bi;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double2 acc = make_double2(0, 0);
        for (int i = 0; i < m; ++i) acc += conj(w[i]) * a[i];
        g = acc;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < (m - 1) * (m - 1); e += blockDim.x) {
        const int i = 1 + e % (m - 1), j = 1 + e / (m - 1);
        out[(size_t)(j - 1) * ld + (i - 1)] = M[(size_t)j * ld + i] - f * (w[i] * conj(b[j])) -
                                               f * (a[i] * conj(w[j])) + (f * f) * (g * (w[i] * conj(w[j])));
    }
}

struct GD {
    qcd_ctx* ctx;
    size_t n;
    int mcap, kcap;
    // V, W = Q V, X and u, Qu, r are stored double-float (QCD_FF, 16 bytes per
    // complex number); R, T and tmp, tmp2 are FP64
    double2 *V, *W, *X, *G, *Hm, *Gt, *Hmt, *S, *work, *C, *dots, *part, *u, *Qu, *rff, *R, *T, *tmp, *tmp2;
    double2 *ffc, *ffw;   // double-float copies of transform / reflector coefficients
    double* mu;
    double* mu_ref;   // refined eigenvalues of the targets
    int* status;
    int* idx;
    int m = 0;        // current basis size
    int m_fact = 0;   // leading rows of the factored pencil state still valid
    double2* hstate = nullptr;   // L^-1, L^-1 H L^-H of the pencil (ld = mcap) and its FP32 eigenvectors
    bool ritz = false;           // Rayleigh-Ritz extraction: the pencil with the identity for W^H W
    double2* Iden = nullptr;     // mcap x mcap identity (Rayleigh-Ritz only)
    int nlock = 0;
    std::vector<double> lam, lres;

    void alloc(int mcap_, int kcap_, int block) {
        mcap = mcap_;
        kcap = kcap_;
        auto B = [&](const char* nm, size_t cnt) { return (double2*)ctx->buf(std::string("gd.") + nm, cnt * sizeof(double2)); };
        V = B("V", (size_t)mcap * n); W = B("W", (size_t)mcap * n);
        X = B("X", (size_t)kcap * n);
        G = B("G", (size_t)mcap * mcap); Hm = B("Hm", (size_t)mcap * mcap);
        Gt = B("Gt", (size_t)mcap * mcap); Hmt = B("Hmt", (size_t)mcap * mcap);
        S = B("S", (size_t)mcap * mcap); work = B("work", (size_t)(6 + block) * mcap * mcap); C = B("C", (size_t)mcap * mcap);
        dots = B("dots", (size_t)4 * (mcap + kcap + 8));
        part = B("part", (size_t)(mcap + kcap + 8) * 64);
        u = B("u", n); Qu = B("Qu", n); rff = B("rff", n); R = B("R", (size_t)block * n); T = B("T", (size_t)block * n);
        tmp = B("tmp", n); tmp2 = B("tmp2", n);
        ffc = B("ffc", (size_t)mcap * mcap); ffw = B("ffw", (size_t)mcap + 1);
        mu = (double*)ctx->buf("gd.mu", mcap * sizeof(double));
        mu_ref = (double*)ctx->buf("gd.mu_ref", mcap * sizeof(double));
        status = (int*)ctx->buf("gd.status", 4 * sizeof(int));
        idx = (int*)ctx->buf("gd.idx", mcap * sizeof(int));
        hstate = B("hstate", (size_t)3 * mcap * mcap);
        if (ritz) {
            // V is orthonormal, so V^H Q V s = theta s is the pencil with W^H W -> I
            Iden = B("Iden", (size_t)mcap * mcap);
            std::vector<double2> id((size_t)mcap * mcap, make_double2(0, 0));
            for (int i = 0; i < mcap; ++i) id[(size_t)i * mcap + i] = make_double2(1, 0);
            CK(cudaMemcpyAsync(Iden, id.data(), id.size() * sizeof(double2), cudaMemcpyHostToDevice, ctx->st));
            CK(cudaStreamSynchronize(ctx->st));
        }
        m_fact = 0;
        CK(cudaMemsetAsync(status, 0, 4 * sizeof(int), ctx->st));
    }
    void applyQ(const double2* in, double2* out) {
        double z = 0.0;
        apply_op(ctx->f, QCD_FP64, QCD_OP_Q, 1, in, out, &z, ctx->st);
    }
    // t orthogonalised against [V X] by classical Gram-Schmidt, normalised
    // into V[m]; W[m] = Q V[m].  The second pass runs only when the first one
    // removed more than half of |t|^2 (|t1| < |t| / sqrt 2, the Kahan-Parlett
    // criterion); |t1|^2 = |t|^2 - |[V X]^H t|^2 otherwise gives the norm
    // without another pass.
    bool add_vector(const double2* t) {
        cudaStream_t st = ctx->st;
        double2* v = V + (size_t)m * n;
        double2* dx = dots + m + 1;
        blas_convert(QCD_FP64, t, QCD_FF, v, n, st);
        blas_multidot(QCD_FF, V, m + 1, n, v, 1, n, dots, part, ctx->dot_counters(m + 1), st);
        if (nlock > 0) blas_multidot(QCD_FF, X, nlock, n, v, 1, n, dx, part, ctx->dot_counters(nlock), st);
        if (m > 0) blas_multiaxpy(QCD_FF, V, m, n, dots, -1.0, v, 1, n, st);
        if (nlock > 0) blas_multiaxpy(QCD_FF, X, nlock, n, dx, -1.0, v, 1, n, st);
        const double2* h = ctx->fetch(dots, m + 1 + nlock);
        const double t0 = h[m].x;
        double c2 = 0.0;
        for (int i = 0; i < m + 1 + nlock; ++i)
            if (i != m) c2 += h[i].x * h[i].x + h[i].y * h[i].y;
        double nt2 = t0 - c2;
        if (!(nt2 >= 0.5 * t0)) {
            if (m > 0) {
                blas_multidot(QCD_FF, V, m, n, v, 1, n, dots, part, ctx->dot_counters(m), st);
                blas_multiaxpy(QCD_FF, V, m, n, dots, -1.0, v, 1, n, st);
            }
            if (nlock > 0) {
                blas_multidot(QCD_FF, X, nlock, n, v, 1, n, dots, part, ctx->dot_counters(nlock), st);
                blas_multiaxpy(QCD_FF, X, nlock, n, dots, -1.0, v, 1, n, st);
            }
            blas_multidot(QCD_FF, v, 1, n, v, 1, n, dots, part, ctx->dot_counters(1), st);
            nt2 = ctx->fetch(dots, 1)[0].x;
        }
        const double nt = std::sqrt(std::max(nt2, 0.0));
        if (!(nt > 1e-12) || !std::isfinite(nt)) return false;
        blas_axpby(QCD_FF, make_double2(0, 0), v, make_double2(1.0 / nt, 0), v, n, st);
        // W[m] = Q v in FP64 (v and W are stored double-float)
        blas_convert(QCD_FF, v, QCD_FP64, tmp, n, st);
        applyQ(tmp, tmp2);
        blas_convert(QCD_FP64, tmp2, QCD_FF, W + (size_t)m * n, n, st);
        // new Gram column / row
        blas_multidot(QCD_FF, W, m + 1, n, W + (size_t)m * n, 1, n, dots, part, ctx->dot_counters(m + 1), st);
        blas_multidot(QCD_FF, W, m + 1, n, v, 1, n, dots + mcap, part, ctx->dot_counters(m + 1), st);
        KTimer kt("gram_update", 0.0, 0.0, st);
        gram_update_kernel<<<1, kMaxBasis + 1, 0, st>>>(G, Hm, mcap, m, dots, dots + mcap);
        check_launch("add_vector");
        ++m;
        return true;
    }
    // appends the converged unit vector u to X
    void lock_vector(const double2* uv) {
        blas_copy(QCD_FF, uv, X + (size_t)nlock * n, n, ctx->st);
        ++nlock;
    }
    // harmonic Ritz pairs of the current basis; returns theta sorted by |theta| with the column index
    void harmonic(std::vector<double>& theta, std::vector<int>& col) {
        if (m_fact > m) m_fact = 0;
        small_harmonic_eig_inc(ritz ? Iden : G, Hm, m, mcap, m_fact, mu, S, hstate, status, ctx->st);
        m_fact = m;
        check_launch("harmonic eig");
        double* hm = (double*)ctx->host(m);
        CK(cudaMemcpyAsync(hm, mu, m * sizeof(double), cudaMemcpyDeviceToHost, ctx->st));
        CK(cudaStreamSynchronize(ctx->st));
        theta.resize(m);
        col.resize(m);
        for (int i = 0; i < m; ++i) {
            theta[i] = ritz ? hm[i] : (hm[i] != 0.0 ? 1.0 / hm[i] : INFINITY);
            col[i] = i;
        }
        std::sort(col.begin(), col.end(), [&](int a, int b) {
            double fa = std::fabs(theta[a]), fb = std::fabs(theta[b]);
            if (fa != fb) return fa < fb;
            return theta[a] < theta[b];
        });
        std::vector<double> th(m);
        for (int i = 0; i < m; ++i) th[i] = theta[col[i]];
        theta = th;
    }
    // replace the basis by V C (m x p), W C and the Gram matrices by C^H G C
    void transform(const double2* Cm, int p) {
        cudaStream_t st = ctx->st;
        ff_transform_inplace(V, m, Cm, p, n, ffc, st);
        ff_transform_inplace(W, m, Cm, p, n, ffc, st);
        small_gram_transform(G, m, mcap, Cm, p, Gt, mcap, work, st);
        small_gram_transform(Hm, m, mcap, Cm, p, Hmt, mcap, work, st);
        std::swap(G, Gt);
        std::swap(Hm, Hmt);
        check_launch("basis transform");
        m = p;
        m_fact = 0;   // the pencil changed as a whole
    }
    // lock-time deflation V <- V Hh[:, 1:], W <- W Hh[:, 1:] and the Gram
    // matrices accordingly, for the Householder reflector Hh of the column
    // s (device, m entries): a rank-one update instead of an m x (m-1) product
    void deflate(const double2* s) {
        cudaStream_t st = ctx->st;
        double2* hw = work;   // m + 1 entries
        {
            KTimer kt("householder", 0.0, 0.0, st);
            householder_vector_kernel<<<1, 64, 0, st>>>(s, m, hw);
            householder_gram_kernel<<<2, 256, 0, st>>>(G, Gt, Hm, Hmt, m, mcap, hw);
        }
        ff_deflate(V, W, m, n, hw, ffw, st);
        std::swap(G, Gt);
        std::swap(Hm, Hmt);
        check_launch("deflate");
        --m;
        m_fact = 0;
    }
};

std::vector<int> select_targets(const std::vector<double>& theta, int b, const std::vector<char>& allowed) {
    std::vector<int> same, other, out;
    int first = -1;
    for (int i = 0; i < (int)theta.size(); ++i) {
        if (!allowed[i]) continue;
        if (first < 0) first = i;
        ((theta[i] >= 0) == (theta[first] >= 0) ? same : other).push_back(i);
    }
    size_t a = 0, c = 0;
    while ((int)out.size() < b && (a < same.size() || c < other.size())) {
        if (a < same.size()) out.push_back(same[a++]);
        if ((int)out.size() < b && c < other.size()) out.push_back(other[c++]);
        if (b == 1) break;
    }
    return out;
}

int eigs_impl(qcd_ctx* ctx, int k, double tol, double* lambda, double2* Vout, qcd_eig_info* info) {
    require_gauge(ctx);
    const qcd_params& P = ctx->p;
    if (P.use_mg) require_mg(ctx);
    const size_t n = ctx->nfine();
    const int block = P.block;
    const int prec = P.precision == QCD_FP64 ? QCD_FP64 : QCD_FP32;
    cudaStream_t st = ctx->st;
    GD gd{};
    gd.ctx = ctx;
    gd.n = n;
    gd.ritz = P.extraction == QCD_EXTRACT_RITZ;
    const int n0 = P.use_mg ? ctx->n_test : P.n_init;
    if (n0 + block > P.m_max) throw QcdError(QCD_EINVAL, "m_max too small for the start basis");
    // locked-pair slots: k plus room for the pairs locked while the last
    // targets finish; when they are full, a new lock replaces the locked
    // pair of largest |lambda| (or is dropped if it is larger still)
    gd.alloc(P.m_max + block, k + P.guard + 2 * block + 8, block);
    CK(cudaMemsetAsync(ctx->counters(), 0, 2 * sizeof(unsigned long long), st));
    double2* t0 = gd.tmp;
    // start basis: setup test vectors (or random vectors without MG)
    for (int i = 0; i < n0; ++i) {
        if (P.use_mg) blas_copy(QCD_FP64, ctx->test_vectors + (size_t)i * n, t0, n, st);
        else blas_gaussian(t0, n, P.seed, 0x1a0000000000ull + (unsigned long long)i * n, st);
        gd.add_vector(t0);
    }
    for (int j = 0; j < block; ++j) blas_gaussian(gd.T + (size_t)j * n, n, P.seed, 0x2b0000000000ull + j * n, st);
    int nT = block;
    int outer = 0, inner = 0, updates = 0, locks_since_update = 0;
    bool finished = false;
    // completion: once k pairs are locked and no harmonic Ritz value lies
    // below the k-th smallest locked |lambda|, the search goes on until
    // P.confirm correction equations (aimed at the smallest values above that
    // bound) have expanded the space; a value that falls below it restarts
    // the count
    int confirm_done = 0;
    bool confirming = false;
    // interpolation updates stage their vectors in the test-vector buffer
    // (the setup vectors are in the start basis already)
    double2* vbuf = ctx->test_vectors;
    std::vector<double> theta;
    std::vector<int> col;
    std::vector<double> tsel;
    int rnd = 0;
    while (!finished && outer < P.max_outer) {
        ++outer;
        int added = 0;
        for (int j = 0; j < nT; ++j) added += gd.add_vector(gd.T + (size_t)j * n) ? 1 : 0;
        if (added == 0) {
            blas_gaussian(gd.T, n, P.seed, 0x3c0000000000ull + (unsigned long long)(rnd++) * n, st);
            nT = 1;
            continue;
        }
        std::vector<int> tg;
        while (true) {
            gd.harmonic(theta, col);
            std::vector<char> allowed(theta.size(), 1);
            // the completion check runs on k + guard pairs (the k smallest are returned)
            const int kk = k + P.guard;
            if (gd.nlock >= kk) {
                std::vector<double> al(gd.lam.size());
                for (size_t i = 0; i < al.size(); ++i) al[i] = std::fabs(gd.lam[i]);
                std::nth_element(al.begin(), al.begin() + (kk - 1), al.end());
                double lim = al[kk - 1];
                int cnt = 0;
                for (size_t i = 0; i < theta.size(); ++i) { allowed[i] = std::fabs(theta[i]) < lim; cnt += allowed[i]; }
                confirming = cnt == 0;
                if (confirming) {
                    if (confirm_done >= P.confirm) { finished = true; break; }
                    std::fill(allowed.begin(), allowed.end(), 1);
                } else {
                    confirm_done = 0;
                }
            }
            tg = select_targets(theta, block, allowed);
            // FP64 refinement of the targeted pairs (the full decomposition is FP32)
            {
                std::vector<int> cols(tg.size());
                for (size_t q = 0; q < tg.size(); ++q) cols[q] = col[tg[q]];
                CK(cudaMemcpyAsync(gd.idx, cols.data(), cols.size() * sizeof(int), cudaMemcpyHostToDevice, st));
                small_refine_targets(gd.hstate, gd.m, gd.mcap, gd.S, gd.mu, gd.mu_ref, gd.idx, (int)cols.size(), st);
                double* hm = (double*)ctx->host(cols.size());
                CK(cudaMemcpyAsync(hm, gd.mu_ref, cols.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
                CK(cudaStreamSynchronize(st));
                for (size_t q = 0; q < tg.size(); ++q)
                    theta[tg[q]] = gd.ritz ? hm[q] : (hm[q] != 0.0 ? 1.0 / hm[q] : INFINITY);
            }
            bool locked = false;
            tsel.clear();
            int nr = 0;
            for (int ti : tg) {
                const double2* s = gd.S + (size_t)col[ti] * gd.m;   // column of S (ld = m)
                blas_zero(QCD_FF, gd.u, n, st);
                blas_zero(QCD_FF, gd.Qu, n, st);
                blas_multiaxpy(QCD_FF, gd.V, gd.m, n, s, 1.0, gd.u, 1, n, st);
                blas_multiaxpy(QCD_FF, gd.W, gd.m, n, s, 1.0, gd.Qu, 1, n, st);
                blas_multidot(QCD_FF, gd.u, 1, n, gd.u, 1, n, gd.dots, gd.part, gd.ctx->dot_counters(1), st);
                blas_multidot(QCD_FF, gd.u, 1, n, gd.Qu, 1, n, gd.dots + 1, gd.part, gd.ctx->dot_counters(1), st);
                const double2* h = ctx->fetch(gd.dots, 2);
                const double uu = h[0].x;
                const double rho = h[1].x / uu;
                const double iu = 1.0 / std::sqrt(uu);
                double2* rj = gd.R + (size_t)nr * n;
                // r = (Qu - rho u)/||u|| ; u <- u/||u||
                blas_copy(QCD_FF, gd.Qu, gd.rff, n, st);
                blas_axpby(QCD_FF, make_double2(-rho * iu, 0), gd.u, make_double2(iu, 0), gd.rff, n, st);
                blas_axpby(QCD_FF, make_double2(0, 0), gd.u, make_double2(iu, 0), gd.u, n, st);
                blas_multidot(QCD_FF, gd.rff, 1, n, gd.rff, 1, n, gd.dots, gd.part, gd.ctx->dot_counters(1), st);
                blas_convert(QCD_FF, gd.rff, QCD_FP64, rj, n, st);
                const double2* hr = ctx->fetch(gd.dots, 1);
                const double rn = std::sqrt(std::max(hr[0].x, 0.0));
                if (rn <= tol) {
                    if (gd.nlock < gd.kcap) {
                        gd.lock_vector(gd.u);
                        gd.lam.push_back(rho);
                        gd.lres.push_back(rn);
                    } else {
                        int big = 0;
                        for (int q = 1; q < gd.nlock; ++q)
                            if (std::fabs(gd.lam[q]) > std::fabs(gd.lam[big])) big = q;
                        if (std::fabs(rho) < std::fabs(gd.lam[big])) {
                            blas_copy(QCD_FF, gd.u, gd.X + (size_t)big * n, n, st);
                            gd.lam[big] = rho;
                            gd.lres[big] = rn;
                        }
                    }
                    // deflate: V <- V C with C the complement of s/||s||
                    gd.deflate(s);
                    ++locks_since_update;
                    locked = true;
                    if (P.verbose)
                        fprintf(stderr, "[qcd_eigs] lock %d lambda=% .12e res=%.2e outer=%d m=%d\n", gd.nlock, rho, rn,
                                outer, gd.m);
                    break;
                }
                if (P.verbose > 1)
                    fprintf(stderr, "[qcd_eigs] outer=%d m=%d theta=% .6e rho=% .10e res=%.3e\n", outer, gd.m,
                            theta[ti], rho, rn);
                tsel.push_back(P.shift_rho ? rho : theta[ti]);
                ++nr;
            }
            if (!locked) break;
            if (gd.m == 0) break;
            if (P.use_mg && P.update_every > 0 && gd.nlock >= ctx->n_test && locks_since_update >= P.update_every) {
                std::vector<double> th2;
                std::vector<int> c2;
                gd.harmonic(th2, c2);
                double target = th2[0];
                std::vector<int> ord(gd.nlock);
                std::iota(ord.begin(), ord.end(), 0);
                std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) {
                    return std::fabs(gd.lam[a] - target) < std::fabs(gd.lam[b] - target);
                });
                std::vector<int> pick(ord.begin(), ord.begin() + ctx->n_test);
                std::sort(pick.begin(), pick.end());
                for (int i = 0; i < ctx->n_test; ++i)
                    blas_convert(QCD_FF, gd.X + (size_t)pick[i] * n, QCD_FP64, vbuf + (size_t)i * n, n, st);
                build_from_vectors(ctx, vbuf, ctx->n_test, ctx->c.B.b);
                locks_since_update = 0;
                ++updates;
            }
        }
        if (finished) break;
        if (gd.m == 0 || tsel.empty()) {
            blas_gaussian(gd.T, n, P.seed, 0x3c0000000000ull + (unsigned long long)(rnd++) * n, st);
            nT = 1;
            continue;
        }
        // correction equations, batched over the targets
        const int nb = (int)tsel.size();
        void* rl = ctx->buf("gd.rl", (size_t)nb * n * esz(prec));
        void* tl = ctx->buf("gd.tl", (size_t)nb * n * esz(prec));
        if (P.correction_form == QCD_OP_D) blas_gamma5(QCD_FP64, gd.R, gd.R, (size_t)ctx->f.g.V * nb, st);
        blas_convert(QCD_FP64, gd.R, prec, rl, (size_t)nb * n, st);
        GmresResult g = inner_solve(ctx, prec, P.correction_form, nb, rl, tl, tsel.data(), P.inner_tol,
                                    P.use_mg ? P.inner_maxiter : P.plain_maxiter);
        for (int v : g.iters) inner += v;
        blas_convert(prec, tl, QCD_FP64, gd.T, (size_t)nb * n, st);
        nT = nb;
        if (confirming) confirm_done += nb;
        // thick restart
        if (gd.m + nT > P.m_max) {
            std::vector<double> th;
            std::vector<int> cl;
            gd.harmonic(th, cl);
            int keep = std::min(P.m_min, gd.m);
            CK(cudaMemcpyAsync(gd.idx, cl.data(), keep * sizeof(int), cudaMemcpyHostToDevice, st));
            {
                KTimer kt("gather_columns", 0.0, 0.0, st);
                gather_columns_kernel<<<1, 256, 0, st>>>(gd.S, gd.m, gd.idx, keep, gd.work);
            }
            small_qr(gd.work, gd.m, keep, gd.m, gd.C, nullptr, st);
            gd.transform(gd.C, keep);
            CK(cudaStreamSynchronize(st));
        }
    }
    // output: k smallest |lambda| of the locked pairs
    std::vector<int> ord(gd.nlock);
    std::iota(ord.begin(), ord.end(), 0);
    std::sort(ord.begin(), ord.end(), [&](int a, int b) {
        double fa = std::fabs(gd.lam[a]), fb = std::fabs(gd.lam[b]);
        if (fa != fb) return fa < fb;
        return gd.lam[a] < gd.lam[b];
    });
    const int nout = std::min(k, gd.nlock);
    double maxres = 0.0;
    for (int i = 0; i < nout; ++i) {
        lambda[i] = gd.lam[ord[i]];
        maxres = std::max(maxres, gd.lres[ord[i]]);
        if (Vout) blas_convert(QCD_FF, gd.X + (size_t)ord[i] * n, QCD_FP64, Vout + (size_t)i * n, n, st);
    }
    for (int i = nout; i < k; ++i) lambda[i] = NAN;
    CK(cudaStreamSynchronize(st));
    const bool ok = finished && nout == k;
    if (info) {
        unsigned long long cnt[2] = {0, 0};
        CK(cudaMemcpy(cnt, ctx->counters(), sizeof(cnt), cudaMemcpyDeviceToHost));
        info->coarse_solves = (long long)cnt[0];
        info->coarse_iterations = (long long)cnt[1];
        info->outer = outer;
        info->inner = inner;
        info->locked = gd.nlock;
        info->updates = updates;
        info->converged = ok ? 1 : 0;
        info->max_residual = maxres;
    }
    return ok ? QCD_OK : QCD_ENOCONV;
}

void check_align(const void* p, const char* what) {
    if (((uintptr_t)p) & 15) throw QcdError(QCD_EINVAL, std::string(what) + " must be 16-byte aligned");
}

// Bounded device-side waits that gave up since the last check: the calls
// that end with their results on the host (setup, solves, eigs) read the
// library-wide counter after synchronising and report QCD_ETIMEOUT when it
// grew (their outputs are then unreliable).
std::atomic<unsigned long long> g_timeouts_seen{0};
void check_wait_timeouts(qcd_ctx* ctx) {
    CK(cudaStreamSynchronize(ctx->st));
    const unsigned long long n = wait_timeouts_read();
    unsigned long long seen = g_timeouts_seen.load();
    if (n > seen) {
        g_timeouts_seen.store(n);
        throw QcdError(QCD_ETIMEOUT, "a device-side wait gave up (" + std::to_string(n - seen) + ")");
    }
}

template <typename F>
int guarded(qcd_ctx* ctx, F&& fn) {
    if (!ctx) return QCD_EINVAL;
    try {
        ctx->err.clear();
        return fn();
    } catch (const QcdError& e) {
        ctx->err = e.what();
        return e.code;
    } catch (const std::exception& e) {
        ctx->err = e.what();
        return QCD_ECUDA;
    }
}

}  // namespace

// ====================================================================== C ABI
extern "C" {

void qcd_default_params(qcd_params* p) {
    if (!p) return;
    memset(p, 0, sizeof(*p));
    p->antiperiodic_t = 1;
    p->precision = QCD_MIXED;
    p->correction_form = QCD_OP_D;
    p->use_mg = 1;
    p->setup_iters = 6;
    p->smoother = QCD_SMOOTHER_SAP;
    p->nu = 4;
    for (int mu = 0; mu < 4; ++mu) p->sap_block[mu] = 2;
    p->sap_block_iters = 10;
    p->sap_block_tol = 1e-1;
    p->gmres_smooth_iters = 4;
    p->inner_tol = 1e-1;
    p->inner_maxiter = 5;
    p->coarse_tol = 0.5;
    p->coarse_maxiter = 64;
    p->plain_maxiter = 20;
    p->m_min = 30;
    p->m_max = 50;
    p->block = 2;
    p->n_init = 8;
    p->shift_rho = 1;
    p->update_every = 1;
    p->extraction = QCD_EXTRACT_HARMONIC;
    p->max_outer = 100000;
    p->seed = 20200417ull;
    p->verbose = 0;
    p->levels = 2;
    p->nv2 = 8;
    for (int mu = 0; mu < 4; ++mu) p->agg2[mu] = 2;
    p->nu2 = 2;
    p->coarse_layout = 0;
    p->coarse_tensor = 0;
    p->sap_half = 0;
    p->confirm = 32;
    p->coarse_ctas = 0;
    p->guard = 0;
}

int qcd_create(qcd_ctx** out, const qcd_params* p, void* stream) {
    if (!out || !p) return QCD_EINVAL;
    *out = nullptr;
    qcd_ctx* ctx = new (std::nothrow) qcd_ctx();
    if (!ctx) return QCD_ENOMEM;
    try {
        validate_params(*p);
    } catch (const QcdError& e) {
        delete ctx;
        return e.code;
    }
    ctx->p = *p;
    ctx->c.ctas = ctx->c2.ctas = p->coarse_ctas;
    ctx->st = (cudaStream_t)stream;
    *out = ctx;
    return QCD_OK;
}

int qcd_destroy(qcd_ctx* ctx) {
    if (!ctx) return QCD_EINVAL;
    cudaStreamSynchronize(ctx->st);
    delete ctx;
    return QCD_OK;
}

const char* qcd_last_error(qcd_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

int qcd_set_params(qcd_ctx* ctx, const qcd_params* p) {
    return guarded(ctx, [&]() {
        if (!p) throw QcdError(QCD_EINVAL, "null params");
        validate_params(*p);
        bool sap_changed = memcmp(p->sap_block, ctx->p.sap_block, sizeof(p->sap_block)) != 0;
        bool bc_changed = p->antiperiodic_t != ctx->p.antiperiodic_t;
        const bool l2_changed = p->levels != ctx->p.levels || p->nv2 != ctx->p.nv2 ||
                                memcmp(p->agg2, ctx->p.agg2, sizeof(p->agg2)) != 0;
        ctx->p = *p;
        ctx->c.ctas = ctx->c2.ctas = p->coarse_ctas;
        if (l2_changed) {
            ctx->c2.ready = false;
            if (p->levels == 3 && ctx->c.ready && ctx->test_vectors) build_level2(ctx, ctx->test_vectors, ctx->n_test);
        }
        if (sap_changed && ctx->have_sap) {
            cudaFree(ctx->sap.blocks_of_colour[0]);
            cudaFree(ctx->sap.blocks_of_colour[1]);
            ctx->sap.blocks_of_colour[0] = ctx->sap.blocks_of_colour[1] = nullptr;
            ctx->have_sap = false;
        }
        if (bc_changed) ctx->f.g.antiperiodic = p->antiperiodic_t;
        return QCD_OK;
    });
}

int qcd_set_gauge(qcd_ctx* ctx, const double* U, const int dims[4], double m0, double csw) {
    return guarded(ctx, [&]() {
        if (!U || !dims) throw QcdError(QCD_EINVAL, "null gauge field or dims");
        long long V = 1;
        for (int mu = 0; mu < 4; ++mu) {
            if (dims[mu] < 2 || dims[mu] > 4096) throw QcdError(QCD_EINVAL, "lattice extents must be in [2, 4096]");
            V *= dims[mu];
        }
        if (V > (1ll << 28)) throw QcdError(QCD_EINVAL, "lattice too large");
        if (!std::isfinite(m0) || !std::isfinite(csw)) throw QcdError(QCD_EINVAL, "m0 and csw must be finite");
        CK(cudaStreamSynchronize(ctx->st));
        ctx->release();
        ctx->have_gauge = false;
        FineOp& f = ctx->f;
        for (int mu = 0; mu < 4; ++mu) f.g.L[mu] = dims[mu];
        f.g.V = (int)V;
        f.g.antiperiodic = ctx->p.antiperiodic_t;
        f.m0 = m0;
        f.csw = csw;
        const size_t nl = (size_t)V * 36;
        CK(cudaMalloc(&f.U64, nl * sizeof(double2)));
        CK(cudaMalloc(&f.U32, nl * sizeof(float2)));
        CK(cudaMalloc(&f.A64, (size_t)V * 72 * sizeof(double)));
        CK(cudaMalloc(&f.A32, (size_t)V * 72 * sizeof(float)));
        CK(cudaMalloc(&f.U32s, nl * sizeof(float2)));
        CK(cudaMalloc(&f.A32s, (size_t)V * 18 * sizeof(float4)));
        CK(cudaMemcpyAsync(f.U64, U, nl * sizeof(double2), cudaMemcpyHostToDevice, ctx->st));
        // the links must be SU(3) matrices (Sec. 2): finite and unitary
        const double dev = gauge_unitarity_deviation(f.U64, (size_t)V * 4, ctx->counters(), ctx->st);
        check_launch("gauge check");
        if (!(dev <= 1e-6)) {
            ctx->release();
            throw QcdError(QCD_EINVAL, std::isfinite(dev) ? "gauge links are not unitary (max |U U^H - I| = " +
                                                                std::to_string(dev) + ")"
                                                          : "gauge links contain non-finite entries");
        }
        blas_convert(QCD_FP64, f.U64, QCD_FP32, f.U32, nl, ctx->st);
        launch_clover_build(f, ctx->st);
        check_launch("set_gauge");
        CK(cudaStreamSynchronize(ctx->st));
        ctx->have_gauge = true;
        return QCD_OK;
    });
}

int qcd_apply(qcd_ctx* ctx, int op, int prec, int nrhs, const void* in, void* out, const double* tau) {
    return guarded(ctx, [&]() {
        require_gauge(ctx);
        if (op != QCD_OP_D && op != QCD_OP_Q) throw QcdError(QCD_EINVAL, "bad op");
        if (prec != QCD_FP64 && prec != QCD_FP32) throw QcdError(QCD_EINVAL, "bad precision");
        if (nrhs < 1 || nrhs > kMaxRhs || !in || !out || !tau) throw QcdError(QCD_EINVAL, "bad nrhs or pointers");
        check_align(in, "in");
        check_align(out, "out");
        const size_t bytes = ctx->nfine() * nrhs * esz(prec);
        const char* a = (const char*)in;
        const char* b = (const char*)out;
        if (a < b + bytes && b < a + bytes) throw QcdError(QCD_EINVAL, "in and out overlap");
        apply_op(ctx->f, prec, op, nrhs, in, out, tau, ctx->st);
        check_launch("apply");
        return QCD_OK;
    });
}

int qcd_apply_Q(qcd_ctx* ctx, const void* in, void* out, double tau) {
    return qcd_apply(ctx, QCD_OP_Q, QCD_FP64, 1, in, out, &tau);
}

int qcd_mg_setup(qcd_ctx* ctx, int Nv, const int block[4]) {
    return guarded(ctx, [&]() {
        if (!block) throw QcdError(QCD_EINVAL, "null block");
        if (Nv < 1 || Nv > 32) throw QcdError(QCD_EINVAL, "need 1 <= Nv <= 32");
        mg_setup_impl(ctx, Nv, block);
        check_wait_timeouts(ctx);
        return QCD_OK;
    });
}

int qcd_mg_update_from_eigvecs(qcd_ctx* ctx, const void* V, int nvec) {
    return guarded(ctx, [&]() {
        require_gauge(ctx);
        if (!V || nvec < 1 || nvec > 32) throw QcdError(QCD_EINVAL, "need 1 <= nvec <= 32");
        const int* blk = ctx->c.ready ? ctx->c.B.b : ctx->p.sap_block;
        int b[4] = {blk[0], blk[1], blk[2], blk[3]};
        build_from_vectors(ctx, (const double2*)V, nvec, b);
        if (ctx->n_test != nvec || !ctx->test_vectors) {
            if (ctx->test_vectors) CK(cudaFree(ctx->test_vectors));
            CK(cudaMalloc(&ctx->test_vectors, (size_t)nvec * ctx->nfine() * sizeof(double2)));
            ctx->n_test = nvec;
        }
        CK(cudaMemcpyAsync(ctx->test_vectors, V, (size_t)nvec * ctx->nfine() * sizeof(double2),
                           cudaMemcpyDeviceToDevice, ctx->st));
        CK(cudaStreamSynchronize(ctx->st));
        return QCD_OK;
    });
}

int qcd_mg_info(qcd_ctx* ctx, int out[8]) {
    return guarded(ctx, [&]() {
        require_mg(ctx);
        out[0] = ctx->c.gc.V;
        out[1] = ctx->c.nv;
        for (int mu = 0; mu < 4; ++mu) out[2 + mu] = ctx->c.gc.L[mu];
        out[6] = ctx->c.B.bs;
        out[7] = 0;
        return QCD_OK;
    });
}

int qcd_mg_restrict(qcd_ctx* ctx, int prec, int nrhs, const void* r, void* xc) {
    return guarded(ctx, [&]() {
        require_mg(ctx);
        if (nrhs < 1 || nrhs > kMaxRhs || !r || !xc) throw QcdError(QCD_EINVAL, "bad arguments");
        mg_restrict(ctx->f, ctx->c, prec, nrhs, r, xc, ctx->st);
        check_launch("restrict");
        return QCD_OK;
    });
}

int qcd_local_coherence(qcd_ctx* ctx, int nvec, const void* V, double* out) {
    return guarded(ctx, [&]() {
        require_mg(ctx);
        if (nvec < 0 || (nvec > 0 && (!V || !out))) throw QcdError(QCD_EINVAL, "bad arguments");
        check_align(V, "V");
        const size_t n = ctx->nfine();
        const Coarse& c = ctx->c;
        const size_t nco = (size_t)c.gc.V * c.nc;
        const int chunk = kMaxRhs;
        double2* xc = (double2*)ctx->buf("lc.xc", (size_t)chunk * nco * sizeof(double2));
        double2* dots = (double2*)ctx->buf("lc.dots", (size_t)2 * chunk * sizeof(double2));
        double2* part = (double2*)ctx->buf("lc.part", (size_t)chunk * 64 * sizeof(double2));
        for (int j0 = 0; j0 < nvec; j0 += chunk) {
            const int nb = std::min(chunk, nvec - j0);
            const double2* v = (const double2*)V + (size_t)j0 * n;
            mg_restrict(ctx->f, c, QCD_FP64, nb, v, xc, ctx->st);
            blas_multidot(QCD_FP64, xc, 1, nco, xc, nb, nco, dots, part, ctx->dot_counters(nb), ctx->st);
            blas_multidot(QCD_FP64, v, 1, n, v, nb, n, dots + chunk, part, ctx->dot_counters(nb), ctx->st);
            const double2* h = ctx->fetch(dots, 2 * chunk);
            for (int j = 0; j < nb; ++j) {
                const double pv = h[j].x, vv = h[chunk + j].x;
                out[j0 + j] = vv > 0 ? std::sqrt(std::max(pv, 0.0) / vv) : 0.0;
            }
        }
        check_launch("local coherence");
        return QCD_OK;
    });
}

int qcd_eig_derivative(qcd_ctx* ctx, const double* X, int nvec, const void* V, double* out) {
    return guarded(ctx, [&]() {
        require_gauge(ctx);
        if (nvec < 0 || (nvec > 0 && (!X || !V || !out))) throw QcdError(QCD_EINVAL, "bad arguments");
        if (nvec == 0) return QCD_OK;
        check_align(V, "V");
        const FineOp& f = ctx->f;
        const size_t n = ctx->nfine(), nl = (size_t)f.g.V * 36;
        double2* Xd = (double2*)ctx->buf("der.X", nl * sizeof(double2));
        double2* dU = (double2*)ctx->buf("der.dU", nl * sizeof(double2));
        double* dA = (double*)ctx->buf("der.dA", (size_t)f.g.V * 72 * sizeof(double));
        CK(cudaMemcpyAsync(Xd, X, nl * sizeof(double2), cudaMemcpyHostToDevice, ctx->st));
        tangent_fields(f, Xd, dU, dA, ctx->st);
        const int chunk = kMaxRhs;
        double2* w = (double2*)ctx->buf("der.w", (size_t)chunk * n * sizeof(double2));
        double2* g5v = (double2*)ctx->buf("der.g5v", (size_t)chunk * n * sizeof(double2));
        double2* dots = (double2*)ctx->buf("der.dots", (size_t)2 * chunk * sizeof(double2));
        double2* part = (double2*)ctx->buf("der.part", (size_t)chunk * 64 * sizeof(double2));
        for (int j0 = 0; j0 < nvec; j0 += chunk) {
            const int nb = std::min(chunk, nvec - j0);
            const double2* v = (const double2*)V + (size_t)j0 * n;
            apply_tangent(f, dU, dA, nb, v, w, ctx->st);
            blas_gamma5(QCD_FP64, v, g5v, (size_t)f.g.V * nb, ctx->st);
            blas_multidot(QCD_FP64, g5v, 1, n, w, nb, n, dots, part, ctx->dot_counters(nb), ctx->st);
            blas_multidot(QCD_FP64, v, 1, n, v, nb, n, dots + chunk, part, ctx->dot_counters(nb), ctx->st);
            const double2* h = ctx->fetch(dots, 2 * chunk);
            for (int j = 0; j < nb; ++j) out[j0 + j] = h[chunk + j].x > 0 ? h[j].x / h[chunk + j].x : 0.0;
        }
        check_launch("eig derivative");
        return QCD_OK;
    });
}

int qcd_eig_force(qcd_ctx* ctx, int nvec, const void* V, void* F) {
    return guarded(ctx, [&]() {
        require_gauge(ctx);
        if (nvec < 0 || (nvec > 0 && (!V || !F))) throw QcdError(QCD_EINVAL, "bad arguments");
        if (nvec == 0) return QCD_OK;
        check_align(V, "V");
        check_align(F, "F");
        const FineOp& f = ctx->f;
        const size_t n = ctx->nfine(), nl = (size_t)f.g.V * 36;
        double2* Bt = (double2*)ctx->buf("force.Bt", (size_t)f.g.V * 54 * sizeof(double2));
        double2* nrm = (double2*)ctx->buf("force.nrm", sizeof(double2));
        double2* part = (double2*)ctx->buf("force.part", (size_t)64 * sizeof(double2));
        for (int j = 0; j < nvec; ++j) {
            const double2* v = (const double2*)V + (size_t)j * n;
            blas_multidot(QCD_FP64, v, 1, n, v, 1, n, nrm, part, ctx->dot_counters(1), ctx->st);
            eig_force(f, v, nrm, Bt, (double2*)F + (size_t)j * nl, ctx->st);
        }
        check_launch("eig force");
        return QCD_OK;
    });
}

int qcd_bilinear_force(qcd_ctx* ctx, int nvec, const void* G, const void* Psi, int grad, void* F) {
    return guarded(ctx, [&]() {
        require_gauge(ctx);
        if (nvec < 0 || (nvec > 0 && (!G || !Psi || !F)) || (grad != 0 && grad != 1))
            throw QcdError(QCD_EINVAL, "bad arguments");
        if (nvec == 0) return QCD_OK;
        check_align(G, "G");
        check_align(Psi, "Psi");
        check_align(F, "F");
        const FineOp& f = ctx->f;
        const size_t n = ctx->nfine(), nl = (size_t)f.g.V * 36;
        double2* Bt = (double2*)ctx->buf("force.Bt", (size_t)f.g.V * 54 * sizeof(double2));
        for (int j = 0; j < nvec; ++j)
            bilinear_force(f, (const double2*)G + (size_t)j * n, (const double2*)Psi + (size_t)j * n, nullptr, grad, Bt,
                           (double2*)F + (size_t)j * nl, ctx->st);
        check_launch("bilinear force");
        return QCD_OK;
    });
}

int qcd_mg_prolong(qcd_ctx* ctx, int prec, int nrhs, const void* xc, void* x) {
    return guarded(ctx, [&]() {
        require_mg(ctx);
        if (nrhs < 1 || nrhs > kMaxRhs || !x || !xc) throw QcdError(QCD_EINVAL, "bad arguments");
        mg_prolong(ctx->f, ctx->c, prec, nrhs, xc, x, false, ctx->st);
        check_launch("prolong");
        return QCD_OK;
    });
}

int qcd_coarse_apply(qcd_ctx* ctx, int op, int prec, int nrhs, const void* x, void* y, const double* tau) {
    return guarded(ctx, [&]() {
        require_mg(ctx);
        if (nrhs < 1 || nrhs > kMaxRhs || !x || !y || !tau) throw QcdError(QCD_EINVAL, "bad arguments");
        if (prec == QCD_FP64) ensure_coarse64(ctx);
        coarse_apply(ctx->c, prec, op, nrhs, x, y, tau, ctx->st, ctx->p.coarse_tensor != 0);
        check_launch("coarse apply");
        return QCD_OK;
    });
}

int qcd_mg_get_P(qcd_ctx* ctx, double* P_host) {
    return guarded(ctx, [&]() {
        require_mg(ctx);
        size_t np = (size_t)ctx->c.B.nb * 2 * ctx->c.nv * ctx->c.B.bs * 6;
        CK(cudaMemcpyAsync(P_host, ctx->c.P64, np * sizeof(double2), cudaMemcpyDeviceToHost, ctx->st));
        CK(cudaStreamSynchronize(ctx->st));
        return QCD_OK;
    });
}

int qcd_mg_get_coarse(qcd_ctx* ctx, double* A_host) {
    return guarded(ctx, [&]() {
        require_mg(ctx);
        ensure_coarse64(ctx);
        const int nc = ctx->c.nc;
        size_t na = (size_t)ctx->c.B.nb * 9 * nc * nc;
        std::vector<double2> tmp(na);
        CK(cudaMemcpyAsync(tmp.data(), ctx->c.A64, na * sizeof(double2), cudaMemcpyDeviceToHost, ctx->st));
        CK(cudaStreamSynchronize(ctx->st));
        // device storage is [site][d][col][row]; the ABI returns [site][d][row][col]
        double2* out = (double2*)A_host;
        for (size_t blk = 0; blk < (size_t)ctx->c.B.nb * 9; ++blk)
            for (int r = 0; r < nc; ++r)
                for (int c = 0; c < nc; ++c) out[(blk * nc + r) * nc + c] = tmp[(blk * nc + c) * nc + r];
        return QCD_OK;
    });
}

void require_level2(qcd_ctx* ctx) {
    require_mg(ctx);
    if (ctx->p.levels != 3 || !ctx->c2.ready) throw QcdError(QCD_ENOTSETUP, "no third level: set params.levels = 3");
}

int qcd_mg_info2(qcd_ctx* ctx, int out[8]) {
    return guarded(ctx, [&]() {
        require_level2(ctx);
        if (!out) throw QcdError(QCD_EINVAL, "null out");
        out[0] = ctx->c2.gc.V;
        out[1] = ctx->c2.nv;
        for (int mu = 0; mu < 4; ++mu) out[2 + mu] = ctx->c2.gc.L[mu];
        out[6] = ctx->c2.B.bs;
        out[7] = ctx->c.nv;
        return QCD_OK;
    });
}

int qcd_mg_get_P2(qcd_ctx* ctx, double* P_host) {
    return guarded(ctx, [&]() {
        require_level2(ctx);
        if (!P_host) throw QcdError(QCD_EINVAL, "null output");
        const size_t np = (size_t)ctx->c2.B.nb * 2 * ctx->c2.nv * ctx->c2.B.bs * ctx->c.nv;
        CK(cudaMemcpyAsync(P_host, ctx->c2.P64, np * sizeof(double2), cudaMemcpyDeviceToHost, ctx->st));
        CK(cudaStreamSynchronize(ctx->st));
        return QCD_OK;
    });
}

int qcd_mg_get_coarse2(qcd_ctx* ctx, double* A_host) {
    return guarded(ctx, [&]() {
        require_level2(ctx);
        if (!A_host) throw QcdError(QCD_EINVAL, "null output");
        const int nc = ctx->c2.nc;
        const size_t na = (size_t)ctx->c2.B.nb * 9 * nc * nc;
        std::vector<double2> tmp(na);
        CK(cudaMemcpyAsync(tmp.data(), ctx->c2.A64, na * sizeof(double2), cudaMemcpyDeviceToHost, ctx->st));
        CK(cudaStreamSynchronize(ctx->st));
        double2* out = (double2*)A_host;
        for (size_t blk = 0; blk < (size_t)ctx->c2.B.nb * 9; ++blk)
            for (int r = 0; r < nc; ++r)
                for (int c = 0; c < nc; ++c) out[(blk * nc + r) * nc + c] = tmp[(blk * nc + c) * nc + r];
        return QCD_OK;
    });
}

int qcd_projected_eig(qcd_ctx* ctx, int m, const double* G, const double* H, int extraction, double* theta,
                      double* S) {
    return guarded(ctx, [&]() {
        if (m < 1 || m > kMaxBasis || !H || !theta || !S || (extraction == QCD_EXTRACT_HARMONIC && !G))
            throw QcdError(QCD_EINVAL, "bad arguments");
        if (extraction != QCD_EXTRACT_HARMONIC && extraction != QCD_EXTRACT_RITZ)
            throw QcdError(QCD_EINVAL, "bad extraction");
        const size_t mm = (size_t)m * m;
        double2* Gd = (double2*)ctx->buf("pe.G", mm * sizeof(double2));
        double2* Hd = (double2*)ctx->buf("pe.H", mm * sizeof(double2));
        double2* Sd = (double2*)ctx->buf("pe.S", mm * sizeof(double2));
        double2* state = (double2*)ctx->buf("pe.state", 3 * mm * sizeof(double2));
        double* mu = (double*)ctx->buf("pe.mu", (size_t)m * sizeof(double));
        double* mu_ref = (double*)ctx->buf("pe.mu_ref", (size_t)m * sizeof(double));
        int* idx = (int*)ctx->buf("pe.idx", (size_t)m * sizeof(int));
        int* status = (int*)ctx->buf("pe.status", 4 * sizeof(int));
        std::vector<double2> hG(mm, make_double2(0, 0));
        if (extraction == QCD_EXTRACT_HARMONIC) memcpy(hG.data(), G, mm * sizeof(double2));
        else for (int i = 0; i < m; ++i) hG[(size_t)i * m + i] = make_double2(1, 0);
        std::vector<int> all(m);
        std::iota(all.begin(), all.end(), 0);
        CK(cudaMemcpyAsync(Gd, hG.data(), mm * sizeof(double2), cudaMemcpyHostToDevice, ctx->st));
        CK(cudaMemcpyAsync(Hd, H, mm * sizeof(double2), cudaMemcpyHostToDevice, ctx->st));
        CK(cudaMemcpyAsync(idx, all.data(), m * sizeof(int), cudaMemcpyHostToDevice, ctx->st));
        CK(cudaMemsetAsync(status, 0, 4 * sizeof(int), ctx->st));
        small_harmonic_eig_inc(Gd, Hd, m, m, 0, mu, Sd, state, status, ctx->st);
        small_refine_targets(state, m, m, Sd, mu, mu_ref, idx, m, ctx->st);
        check_launch("projected eig");
        std::vector<double> hmu(m);
        std::vector<double2> hS(mm);
        int hst = 0;
        CK(cudaMemcpyAsync(hmu.data(), mu_ref, m * sizeof(double), cudaMemcpyDeviceToHost, ctx->st));
        CK(cudaMemcpyAsync(hS.data(), Sd, mm * sizeof(double2), cudaMemcpyDeviceToHost, ctx->st));
        CK(cudaMemcpyAsync(&hst, status, sizeof(int), cudaMemcpyDeviceToHost, ctx->st));
        CK(cudaStreamSynchronize(ctx->st));
        if (hst != 0) throw QcdError(QCD_EINVAL, "G is not positive definite");
        std::vector<double> th(m);
        for (int i = 0; i < m; ++i)
            th[i] = extraction == QCD_EXTRACT_RITZ ? hmu[i] : (hmu[i] != 0.0 ? 1.0 / hmu[i] : INFINITY);
        std::vector<int> ord(all);
        std::sort(ord.begin(), ord.end(), [&](int a, int b) {
            const double fa = std::fabs(th[a]), fb = std::fabs(th[b]);
            if (fa != fb) return fa < fb;
            return th[a] < th[b];
        });
        for (int i = 0; i < m; ++i) {
            theta[i] = th[ord[i]];
            memcpy(S + (size_t)2 * i * m, hS.data() + (size_t)ord[i] * m, m * sizeof(double2));
        }
        return QCD_OK;
    });
}

int qcd_sap(qcd_ctx* ctx, int op, int prec, int nrhs, const void* b, void* x, const double* tau, int sweeps,
            double block_tol) {
    return guarded(ctx, [&]() {
        require_gauge(ctx);
        if (nrhs < 1 || nrhs > kMaxRhs || !b || !x || !tau || sweeps < 0) throw QcdError(QCD_EINVAL, "bad arguments");
        check_align(b, "b");
        check_align(x, "x");
        sap_smooth(ctx, prec, op, nrhs, b, x, tau, sweeps, block_tol);
        CK(cudaStreamSynchronize(ctx->st));
        return QCD_OK;
    });
}

int qcd_mg_cycle(qcd_ctx* ctx, int op, int prec, int nrhs, const void* b, void* x, const double* tau) {
    return guarded(ctx, [&]() {
        require_mg(ctx);
        if (nrhs < 1 || nrhs > kMaxRhs || !b || !x || !tau) throw QcdError(QCD_EINVAL, "bad arguments");
        check_align(b, "b");
        check_align(x, "x");
        mg_cycle_impl(ctx, prec, op, nrhs, b, x, tau);
        CK(cudaStreamSynchronize(ctx->st));
        return QCD_OK;
    });
}

int qcd_shifted_solve_batched(qcd_ctx* ctx, int nrhs, const void* const* b, void* const* x, const double* tau,
                              double tol, qcd_solve_info* info) {
    return guarded(ctx, [&]() {
        require_gauge(ctx);
        if (nrhs < 1 || nrhs > kMaxRhs || !b || !x || !tau || !(tol > 0)) throw QcdError(QCD_EINVAL, "bad arguments");
        double t0 = now_s();
        const size_t n = ctx->nfine();
        double2* bb = (double2*)ctx->buf("ssb.b", n * nrhs * sizeof(double2));
        double2* xx = (double2*)ctx->buf("ssb.x", n * nrhs * sizeof(double2));
        for (int j = 0; j < nrhs; ++j) {
            if (!b[j] || !x[j]) throw QcdError(QCD_EINVAL, "null field");
            CK(cudaMemcpyAsync(bb + (size_t)j * n, b[j], n * sizeof(double2), cudaMemcpyDeviceToDevice, ctx->st));
        }
        double res = shifted_solve_impl(ctx, nrhs, bb, xx, tau, tol, info);
        for (int j = 0; j < nrhs; ++j)
            CK(cudaMemcpyAsync(x[j], xx + (size_t)j * n, n * sizeof(double2), cudaMemcpyDeviceToDevice, ctx->st));
        check_wait_timeouts(ctx);
        if (info) info->seconds = now_s() - t0;
        return res <= tol ? QCD_OK : QCD_ENOCONV;
    });
}

int qcd_shifted_solve(qcd_ctx* ctx, const void* b, void* x, double tau, double tol, qcd_solve_info* info) {
    const void* bs[1] = {b};
    void* xs[1] = {x};
    return qcd_shifted_solve_batched(ctx, 1, bs, xs, &tau, tol, info);
}

int qcd_selftest_wait_limit(qcd_ctx* ctx) {
    return guarded(ctx, [&]() {
        wait_probe(ctx->st);
        check_launch("wait probe");
        check_wait_timeouts(ctx);
        return QCD_OK;
    });
}

int qcd_eigs(qcd_ctx* ctx, int k, double tol, double* lambda, void* V, qcd_eig_info* info) {
    return guarded(ctx, [&]() {
        if (k < 1 || !lambda || !(tol > 0)) throw QcdError(QCD_EINVAL, "bad arguments");
        double t0 = now_s();
        int rc = eigs_impl(ctx, k, tol, lambda, (double2*)V, info);
        check_wait_timeouts(ctx);
        if (info) info->seconds = now_s() - t0;
        if (rc == QCD_ENOCONV) ctx->err = "qcd_eigs: outer iteration cap reached";
        return rc;
    });
}

}  // extern "C"

// ====================================================================== allocation-free SAP
// qcd_sap_static: the SAP sweeps of qcd_sap for callers that cannot allocate
// device memory (a host application that hands the library a fixed memory
// budget up front, or a plugin whose host owns every allocation).  All
// scratch -- the colour block lists, the residual fields and, for block
// sizes other than 16 and 32 sites (whose kernels keep the Krylov basis in
// shared memory), the block-GMRES Krylov vectors -- lives in one
// file-scope device array of kSapStaticBytes that every GPU loading the
// library keeps until the process exits.
namespace {

constexpr size_t kSapStaticBytes = 64ull << 20;   // 64 MiB
__device__ __align__(256) unsigned char g_sap_static[kSapStaticBytes];

constexpr int kStaticMaxDevices = 64;
// device address of g_sap_static, per device; first calls on several host
// threads may race to fill a slot, which they do with the same value
std::atomic<void*> g_sap_static_ptr[kStaticMaxDevices] = {};

// block lists of the two colours: with an even block-grid extent in mu = 3
// the blocks of each colour are exactly every second block, so block b goes
// to position b / 2 of its colour's list (ascending, like the host-built lists)
__global__ void sap_colour_lists_kernel(Blocking B, int* list0, int* list1) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B.nb) return;
    int t = b;
    const int c3 = t % B.cd[3]; t /= B.cd[3];
    const int c2 = t % B.cd[2]; t /= B.cd[2];
    const int c1 = t % B.cd[1], c0 = t / B.cd[1];
    ((c0 + c1 + c2 + c3) % 2 ? list1 : list0)[b / 2] = b;
}

int static_fail(qcd_ctx* ctx, int code, const char* msg) {
    ctx->err.assign(msg);
    return code;
}

}  // namespace

extern "C" int qcd_sap_static(qcd_ctx* ctx, int op, int prec, int nrhs, const void* b, void* x, const double* tau,
                              int sweeps, double block_tol) {
    if (!ctx) return QCD_EINVAL;
    if (!ctx->have_gauge) return static_fail(ctx, QCD_ENOTSETUP, "no gauge field: call qcd_set_gauge first");
    if ((op != QCD_OP_D && op != QCD_OP_Q) || (prec != QCD_FP64 && prec != QCD_FP32) || nrhs < 1 ||
        nrhs > kMaxRhs || !b || !x || !tau || sweeps < 0)
        return static_fail(ctx, QCD_EINVAL, "qcd_sap_static: bad arguments");
    if ((((uintptr_t)b) & 15) || (((uintptr_t)x) & 15))
        return static_fail(ctx, QCD_EINVAL, "qcd_sap_static: b and x must be 16-byte aligned");
    // the SAP blocking, as qcd_sap builds it
    Blocking B;
    B.bs = 1;
    B.nb = 1;
    for (int mu = 0; mu < 4; ++mu) {
        const int e = ctx->p.sap_block[mu];
        if (e < 1 || ctx->f.g.L[mu] % e) return static_fail(ctx, QCD_EINVAL, "qcd_sap_static: block must divide the lattice");
        B.b[mu] = e;
        B.cd[mu] = ctx->f.g.L[mu] / e;
        if (B.cd[mu] % 2) return static_fail(ctx, QCD_EINVAL, "qcd_sap_static: SAP needs an even block count per direction");
        B.bs *= e;
        B.nb *= B.cd[mu];
    }
    if ((B.bs & (B.bs - 1)) || B.bs > 1024)
        return static_fail(ctx, QCD_EINVAL, "qcd_sap_static: SAP block sites must be a power of two <= 1024");
    // scratch layout in the static array: [lists][residual fields][Krylov vectors]
    SapPlan plan;
    plan.B = B;
    plan.ncol[0] = plan.ncol[1] = B.nb / 2;
    const size_t n = ctx->nfine();
    const size_t lists = ((size_t)B.nb * sizeof(int) + 255) & ~size_t(255);
    const size_t rbytes = ((n * nrhs * esz(prec)) + 255) & ~size_t(255);
    // Krylov vectors of the block solves, for exactly the block sizes whose
    // kernel keeps them in global memory (the same predicate sap_blocks uses)
    const size_t kbytes = sap_scratch_bytes(plan, prec, nrhs, ctx->p.sap_block_iters);
    if (lists + rbytes + kbytes > kSapStaticBytes)
        return static_fail(ctx, QCD_EINVAL, "qcd_sap_static: problem needs more scratch than the 64 MiB static array");
    // set-up, once per device, with that device current
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kStaticMaxDevices)
        return static_fail(ctx, QCD_ECUDA, "qcd_sap_static: no usable current device");
    void* sym = g_sap_static_ptr[dev].load(std::memory_order_acquire);
    if (sym == nullptr) {
        if (cudaGetSymbolAddress(&sym, g_sap_static) != cudaSuccess || sym == nullptr) {
            cudaGetLastError();
            return static_fail(ctx, QCD_ECUDA, "qcd_sap_static: cudaGetSymbolAddress failed");
        }
        g_sap_static_ptr[dev].store(sym, std::memory_order_release);
    }
    unsigned char* base = (unsigned char*)sym;
    plan.blocks_of_colour[0] = (int*)base;
    plan.blocks_of_colour[1] = (int*)base + B.nb / 2;
    void* r = base + lists;
    void* scr = base + lists + rbytes;
    QuietAccounting quiet;
    sap_colour_lists_kernel<<<(B.nb + 255) / 256, 256, 0, ctx->st>>>(B, plan.blocks_of_colour[0],
                                                                      plan.blocks_of_colour[1]);
    for (int s = 0; s < sweeps; ++s) {
        for (int colour = 0; colour < 2; ++colour) {
            residual_op(ctx->f, prec, op, nrhs, b, x, r, tau, ctx->st);
            sap_blocks(ctx->f, plan, colour, prec, op, nrhs, r, x, tau, ctx->p.sap_block_iters, block_tol, scr,
                       ctx->st);
        }
    }
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->st);
    if (e != cudaSuccess) return static_fail(ctx, QCD_ECUDA, "qcd_sap_static: kernel launch failed");
    return QCD_OK;
}
