// Device-resident Krylov control.
//
// (1) The Hessenberg bookkeeping of batched (F)GMRES -- Givens rotations,
//     residual estimates, per-right-hand-side stopping and the final
//     triangular solve -- as tiny kernels, so that a whole (F)GMRES solve is a
//     fixed launch sequence without host round trips (converged right-hand
//     sides are skipped by every kernel through the `active` flags).
// (2) A persistent cooperative kernel that runs a complete batched GMRES on
//     the coarse stencil (the coarse-grid solve to a fixed reduction, Table 2
//     "coarse grid tolerance") in one launch: operator apply, classical
//     Gram-Schmidt applied twice, Givens and the solution update, separated by
//     grid-wide barriers of the cooperative launch.
#include <cooperative_groups.h>

#include <algorithm>
#include "internal.h"

namespace cg = cooperative_groups;

namespace qcd {

namespace {

__device__ __forceinline__ double cabs2(double2 a) { return a.x * a.x + a.y * a.y; }

// Givens update of column `it` of one right-hand side; h[0..it] is the new
// Hessenberg column, hn its sub-diagonal entry.  Returns |g_{it+1}|.
// (FP64: the host-side FGMRES bookkeeping and FP64 coarse solves.)
__device__ double givens_column(double2* h, double hn, double* cs, double2* sn, double2* g, int it) {
    for (int i = 0; i < it; ++i) {
        double2 a = h[i], c = h[i + 1];
        h[i] = cs[i] * a + sn[i] * c;
        h[i + 1] = cs[i] * c - conj(sn[i]) * a;
    }
    double2 a = h[it];
    double2 c = make_double2(hn, 0.0);
    double aa = sqrt(cabs2(a)), rr = sqrt(aa * aa + hn * hn);
    if (aa > 0) {
        cs[it] = aa / rr;
        sn[it] = (1.0 / rr) * ((1.0 / aa) * a * conj(c));
    } else {
        cs[it] = 0.0;
        sn[it] = make_double2(1, 0);
    }
    h[it] = cs[it] * a + sn[it] * c;
    g[it + 1] = -1.0 * (conj(sn[it]) * g[it]);
    g[it] = cs[it] * g[it];
    return sqrt(cabs2(g[it + 1]));
}

// Same update in the working precision R of a coarse solve (FP32 for the
// mixed-precision path: the coarse system only needs a 0.5 reduction).
template <typename R>
__device__ double givens_column_t(cplx<R>* h, R hn, R* cs, cplx<R>* sn, cplx<R>* g, int it) {
    for (int i = 0; i < it; ++i) {
        cplx<R> a = h[i], c = h[i + 1];
        h[i] = cs[i] * a + sn[i] * c;
        h[i + 1] = cs[i] * c - conj(sn[i]) * a;
    }
    cplx<R> a = h[it];
    cplx<R> c = mk<R>(hn, R(0));
    R aa = sqrt(a.x * a.x + a.y * a.y), rr = sqrt(aa * aa + hn * hn);
    if (aa > R(0)) {
        cs[it] = aa / rr;
        sn[it] = (R(1) / rr) * ((R(1) / aa) * a * conj(c));
    } else {
        cs[it] = R(0);
        sn[it] = mk<R>(R(1), R(0));
    }
    h[it] = cs[it] * a + sn[it] * c;
    g[it + 1] = R(-1) * (conj(sn[it]) * g[it]);
    g[it] = cs[it] * g[it];
    return (double)sqrt(g[it + 1].x * g[it + 1].x + g[it + 1].y * g[it + 1].y);
}

__global__ void kry_init_kernel(KryDev K, const double2* __restrict__ nrm, const int* __restrict__ outer_act) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= K.nrhs) return;
    const double b = sqrt(fmax(nrm[j].x, 0.0));
    const bool on = b > 0.0 && (outer_act == nullptr || outer_act[j] != 0);
    K.beta[j] = b;
    K.g[(size_t)j * (K.maxit + 1)] = make_double2(b, 0.0);
    K.active[j] = on ? 1 : 0;
    K.k[j] = 0;
    K.scale[j] = make_double2(on ? 1.0 / b : 0.0, 0.0);
}

__global__ void kry_step_kernel(KryDev K, int it, const double2* __restrict__ h1, const double2* __restrict__ h2,
                                const double2* __restrict__ nrm) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= K.nrhs || !K.active[j]) return;
    double2 h[kMaxKry + 1];
    for (int i = 0; i <= it; ++i) h[i] = h1[i * K.nrhs + j] + h2[i * K.nrhs + j];
    const double hn = sqrt(fmax(nrm[j].x, 0.0));
    double* cs = K.cs + (size_t)j * K.maxit;
    double2* sn = K.sn + (size_t)j * K.maxit;
    double2* g = K.g + (size_t)j * (K.maxit + 1);
    const double res = givens_column(h, hn, cs, sn, g, it);
    double2* R = K.R + (size_t)j * K.maxit * K.maxit;
    for (int i = 0; i <= it; ++i) R[(size_t)i * K.maxit + it] = h[i];
    K.k[j] = it + 1;
    K.scale[j] = make_double2(hn > 0 ? 1.0 / hn : 0.0, 0.0);
    if (res <= K.tol * K.beta[j]) K.active[j] = 0;
    K.resid[j] = K.beta[j] > 0 ? res / K.beta[j] : 0.0;
}

__global__ void kry_finish_kernel(KryDev K) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= K.nrhs) return;
    const int kd = K.k[j];
    const double2* R = K.R + (size_t)j * K.maxit * K.maxit;
    const double2* g = K.g + (size_t)j * (K.maxit + 1);
    double2 y[kMaxKry];
    for (int i = kd - 1; i >= 0; --i) {
        double2 s = g[i];
        for (int l = i + 1; l < kd; ++l) s -= R[(size_t)i * K.maxit + l] * y[l];
        double2 d = R[(size_t)i * K.maxit + i];
        double den = cabs2(d);
        y[i] = den > 0 ? (1.0 / den) * cmulc(d, s) : make_double2(0, 0);
    }
    for (int i = 0; i < K.maxit; ++i) K.coef[(size_t)i * K.nrhs + j] = i < kd ? y[i] : make_double2(0, 0);
}

// ------------------------------------------------------------------ coarse GMRES
// Each CTA owns the chunk [lo, hi) of every coarse vector.  It keeps its
// chunk of the whole Krylov basis in shared memory; only the newest basis
// vector is published to global memory (double-buffered) for the neighbour
// reads of the stencil.  Inner products are accumulated into FP64 totals
// with atomics, one grid barrier per reduction; the totals are double-
// buffered by iteration parity, so zeroing the next iteration's buffer never
// races with readers of the current one.  Every CTA performs the (tiny)
// Givens updates itself on identical totals.
template <typename Z, typename R>
struct CoarseArgs {
    Geom gc;
    int nc;
    const Z* A;          // [Vc][9][col][row]
    const Z* b;          // nrhs coarse vectors
    Z* x;                // nrhs coarse vectors (output)
    Z* Vg;               // [2][nrhs][nco] newest basis vector, double-buffered
    double2* tot;        // [2 parities][2 passes][npair] FP64 totals
    double2* Rg;         // [nrhs][maxit][maxit] triangular factor (written by CTA 0)
    double2* yv;         // [nrhs][maxit]
    int* iters;          // [nrhs] iterations used (written by CTA 0)
    unsigned long long* counter;   // [2] solves, iterations (accumulated, may be null)
    double* resid;       // [nrhs] relative residual estimates
    int op;
    const double* tau;   // device [nrhs]
    const int* act;      // device [nrhs] or null
    double tol;
    int maxit;
    int nrhs;
    int E;               // chunk length per CTA (= sites per CTA * nc)
    int sps;             // coarse sites per CTA
    int a_smem;          // 1: this CTA's stencil blocks are staged in shared memory
    Z* Vglob;            // non-null: the Krylov basis and w chunks live in global
    Z* wglob;            //   memory ([CTA][(maxit+1)][nrhs][E] and [CTA][nrhs][E])
};

template <typename Z, typename R>
__device__ __forceinline__ void coarse_row(const CoarseArgs<Z, R>& a, const Z* xj, int s, int r, const int c[4], R tj,
                                           Z& out) {
    Z acc; acc.x = 0; acc.y = 0;
    for (int d = 0; d < 9; ++d) {
        int sn = s;
        if (d > 0) {
            int mu = (d - 1) & 3, step = d <= 4 ? 1 : -1;
            int cn[4] = {c[0], c[1], c[2], c[3]};
            cn[mu] = (cn[mu] + step + a.gc.L[mu]) % a.gc.L[mu];
            sn = site_index(a.gc, cn);
        }
        const Z* am = a.A + (((size_t)s * 9 + d) * a.nc) * a.nc + r;
        const Z* xs = xj + (size_t)sn * a.nc;
        for (int col = 0; col < a.nc; ++col) acc += am[(size_t)col * a.nc] * xs[col];
    }
    const R sg = r < a.nc / 2 ? R(1) : R(-1);
    Z xv = xj[(size_t)s * a.nc + r];
    if (a.op == QCD_OP_D) { acc -= (tj * sg) * xv; }
    else { acc = sg * acc; acc -= tj * xv; }
    out = acc;
}

struct CoarseSmem { size_t As, xn, nbr, Vs, ws, hc, h1, hr, hcol, cs, sn, g, beta, after, live, kd, again, total; };
// Shared-memory layout of one CTA.  sps = 0: no staged stencil blocks;
// basis_in_smem = false: the Krylov basis and w chunks are in global memory.
template <typename Z>
__host__ __device__ inline CoarseSmem coarse_smem(int nrhs, int maxit, int E, int sps = 0, int nc = 0,
                                                  bool basis_in_smem = true) {
    auto up = [](size_t v) { return (v + 15) & ~size_t(15); };
    const size_t Eb = basis_in_smem ? (size_t)E : 0;
    CoarseSmem L;
    size_t o = 0;
    L.As = o;   o = up(o + sizeof(Z) * (size_t)sps * 9 * nc * nc);
    L.xn = o;   o = up(o + sizeof(Z) * (size_t)nrhs * sps * 9 * nc);
    L.nbr = o;  o = up(o + sizeof(int) * (size_t)sps * 9);
    L.Vs = o;   o = up(o + sizeof(Z) * (size_t)(maxit + 1) * nrhs * Eb);
    L.ws = o;   o = up(o + sizeof(Z) * (size_t)nrhs * Eb);
    L.hc = o;   o = up(o + sizeof(Z) * (size_t)(maxit + 2) * nrhs);
    L.h1 = o;   o = up(o + sizeof(Z) * (size_t)(maxit + 2) * nrhs);
    L.hr = o;   o = up(o + sizeof(Z) * (size_t)(maxit + 1) * nrhs);
    L.hcol = o; o = up(o + sizeof(Z) * (size_t)(maxit + 1) * nrhs);
    L.cs = o;   o = up(o + sizeof(Z) * (size_t)nrhs * maxit);
    L.sn = o;   o = up(o + sizeof(Z) * (size_t)nrhs * maxit);
    L.g = o;    o = up(o + sizeof(Z) * (size_t)nrhs * (maxit + 1));
    L.beta = o; o = up(o + sizeof(double) * nrhs);
    L.after = o; o = up(o + sizeof(Z) * nrhs);
    L.live = o; o = up(o + sizeof(int) * nrhs);
    L.kd = o;   o = up(o + sizeof(int) * nrhs);
    L.again = o; o = up(o + sizeof(int) * 4);
    L.total = o;
    return L;
}

template <typename Z, typename R>
__global__ void __launch_bounds__(256) coarse_gmres_kernel(CoarseArgs<Z, R> a) {
    cg::grid_group grid = cg::this_grid();
    extern __shared__ __align__(16) unsigned char sraw[];
    const int nrhs = a.nrhs, maxit = a.maxit, E = a.E, nc = a.nc;
    const bool gbasis = a.Vglob != nullptr;
    const CoarseSmem LY = coarse_smem<Z>(nrhs, maxit, E, a.a_smem ? a.sps : 0, a.a_smem ? nc : 0, !gbasis);
    Z* As = reinterpret_cast<Z*>(sraw + LY.As);          // [sps][9][col][row] stencil blocks of my sites
    Z* xn = reinterpret_cast<Z*>(sraw + LY.xn);          // [nrhs][sps][9][nc] neighbour vectors
    int* nbr = reinterpret_cast<int*>(sraw + LY.nbr);    // [sps][9] neighbour sites
    // [(maxit+1)][nrhs][E] basis chunk and [nrhs][E] w chunk of this CTA
    Z* Vs = gbasis ? a.Vglob + (size_t)blockIdx.x * (maxit + 1) * nrhs * E : reinterpret_cast<Z*>(sraw + LY.Vs);
    Z* ws = gbasis ? a.wglob + (size_t)blockIdx.x * nrhs * E : reinterpret_cast<Z*>(sraw + LY.ws);
    // the serial per-iteration bookkeeping runs in the working precision R:
    // a dependent chain of FP64 operations is very slow on this part
    Z* hc = reinterpret_cast<Z*>(sraw + LY.hc);          // coefficients of the current pass (+ norms)
    Z* h1s = reinterpret_cast<Z*>(sraw + LY.h1);         // pass-1 coefficients, kept for the Hessenberg column
    Z* hr = reinterpret_cast<Z*>(sraw + LY.hr);               // current-pass coefficients in the working precision
    Z* hcol = reinterpret_cast<Z*>(sraw + LY.hcol);      // [nrhs][maxit+1] column under rotation
    R* cs = reinterpret_cast<R*>(sraw + LY.cs);
    Z* sn = reinterpret_cast<Z*>(sraw + LY.sn);
    Z* g = reinterpret_cast<Z*>(sraw + LY.g);
    double* beta = reinterpret_cast<double*>(sraw + LY.beta);
    int* live = reinterpret_cast<int*>(sraw + LY.live);
    int* kd = reinterpret_cast<int*>(sraw + LY.kd);
    R* after = reinterpret_cast<R*>(sraw + LY.after);   // [nrhs] ||w||^2 after pass 1
    int* againf = reinterpret_cast<int*>(sraw + LY.again);

    const size_t nco = (size_t)a.gc.V * a.nc;
    const size_t lo = (size_t)blockIdx.x * E;
    const int len = lo >= nco ? 0 : (int)min((size_t)E, nco - lo);
    const int s0 = blockIdx.x * a.sps;
    const int nsl = len / nc;                               // sites owned by this CTA
    if (a.a_smem) {
        const Z* src = a.A + (size_t)s0 * 9 * nc * nc;
        for (size_t t = threadIdx.x; t < (size_t)nsl * 9 * nc * nc; t += blockDim.x) As[t] = src[t];
        for (int t = threadIdx.x; t < nsl * 9; t += blockDim.x) {
            const int sl = t / 9, d = t % 9;
            int c[4];
            site_coords(a.gc, s0 + sl, c);
            int sn = s0 + sl;
            if (d > 0) {
                int mu = (d - 1) & 3, step = d <= 4 ? 1 : -1;
                c[mu] = (c[mu] + step + a.gc.L[mu]) % a.gc.L[mu];
                sn = site_index(a.gc, c);
            }
            nbr[t] = sn;
        }
    }
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
    const int npair = (maxit + 2) * nrhs;
    auto TOT = [&](int parity, int pass) { return a.tot + ((size_t)parity * 2 + pass) * npair; };
    auto VS = [&](int i, int j) { return Vs + ((size_t)i * nrhs + j) * E; };

    // partial inner products of this chunk: <Vs_i[j], ws[j]> for i < ni (+ ||ws_j||^2), added to `tot`
    auto dots = [&](double2* tot, int ni, bool with_norm, const Z* Y) {
        const int np = ni * nrhs + (with_norm ? nrhs : 0);
        // two pairs per warp and round (independent shuffle chains overlap);
        // this CTA's share in the working precision R, only the cross-CTA
        // totals are FP64 (FP64 throughput per SM is tiny on this part)
        for (int p0 = 2 * warp; p0 < np; p0 += 2 * nw) {
            R re[2] = {0, 0}, im[2] = {0, 0};
            int slot[2] = {-1, -1};
            for (int q = 0; q < 2; ++q) {
                const int p = p0 + q;
                if (p >= np) break;
                int j;
                const Z* xa;
                if (p < ni * nrhs) { j = p % nrhs; xa = VS(p / nrhs, j); }
                else { j = p - ni * nrhs; xa = Y + (size_t)j * E; }
                if (!live[j]) continue;
                const Z* ya = Y + (size_t)j * E;
                for (int e = lane; e < len; e += 32) {
                    Z u = xa[e], v = ya[e];
                    re[q] += u.x * v.x + u.y * v.y;
                    im[q] += u.x * v.y - u.y * v.x;
                }
                slot[q] = p < ni * nrhs ? p : (maxit + 1) * nrhs + j;
            }
            for (int o = 16; o > 0; o >>= 1) {
                re[0] += __shfl_xor_sync(0xffffffffu, re[0], o);
                im[0] += __shfl_xor_sync(0xffffffffu, im[0], o);
                re[1] += __shfl_xor_sync(0xffffffffu, re[1], o);
                im[1] += __shfl_xor_sync(0xffffffffu, im[1], o);
            }
            if (lane == 0 && len > 0)
                for (int q = 0; q < 2; ++q)
                    if (slot[q] >= 0) {
                        atomicAdd(&tot[slot[q]].x, (double)re[q]);
                        atomicAdd(&tot[slot[q]].y, (double)im[q]);
                    }
        }
    };
    // ws[j] -= sum_i hc[i][j] Vs_i[j]
    auto project = [&](int ni) {
        for (int t = tid; t < nrhs * len; t += blockDim.x) {
            const int j = t / len, e = t % len;
            if (!live[j]) continue;
            Z acc = ws[(size_t)j * E + e];
            for (int i = 0; i < ni; ++i) acc -= hr[i * nrhs + j] * VS(i, j)[e];
            ws[(size_t)j * E + e] = acc;
        }
    };

    // ---- load b, beta = ||b||
    for (int j = tid; j < nrhs; j += blockDim.x) live[j] = (a.act == nullptr || a.act[j]) ? 1 : 0;
    for (int t = tid; t < nrhs * len; t += blockDim.x) {
        const int j = t / len, e = t % len;
        ws[(size_t)j * E + e] = a.b[(size_t)j * nco + lo + e];
    }
    __syncthreads();
    dots(TOT(1, 1), 0, true, ws);           // parity 1 pass 1 region: unused by iteration 0
    grid.sync();
    for (int j = tid; j < nrhs; j += blockDim.x) {
        const double bb = live[j] ? sqrt(fmax(TOT(1, 1)[(maxit + 1) * nrhs + j].x, 0.0)) : 0.0;
        beta[j] = bb;
        if (!(bb > 0)) live[j] = 0;
        kd[j] = 0;
        g[(size_t)j * (maxit + 1)] = mk<R>((R)bb, R(0));
    }
    __syncthreads();
    for (int t = tid; t < nrhs * len; t += blockDim.x) {
        const int j = t / len, e = t % len;
        const R ib = live[j] ? (R)(1.0 / beta[j]) : R(0);
        Z v = ws[(size_t)j * E + e];
        v.x *= ib; v.y *= ib;
        VS(0, j)[e] = v;
        a.Vg[(size_t)j * nco + lo + e] = v;
    }
    int it = 0;
    for (; it < maxit; ++it) {
        int any = 0;
        for (int j = 0; j < nrhs; ++j) any |= live[j];
        if (!any) break;
        const int par = it & 1;
        grid.sync();
        // zero the other parity's totals: every CTA has passed the barrier, so
        // nobody still reads them (they held the previous iteration's sums, or
        // beta in iteration 0), and the next atomics into them follow the
        // next barrier
        if (blockIdx.x == 0)
            for (int t = tid; t < 2 * npair; t += blockDim.x) a.tot[(size_t)(par ^ 1) * 2 * npair + t] = make_double2(0, 0);
        // w = A v_it on this chunk
        const Z* Vit = a.Vg + (size_t)par * nrhs * nco;
        if (a.a_smem) {
            // gather the 9 neighbour blocks of every owned site, then multiply from shared memory
            for (int t = tid; t < nrhs * nsl * 9 * nc; t += blockDim.x) {
                const int col = t % nc, d = (t / nc) % 9, sl = (t / (9 * nc)) % nsl, j = t / (9 * nc * nsl);
                if (!live[j]) continue;
                xn[(((size_t)j * nsl + sl) * 9 + d) * nc + col] = Vit[(size_t)j * nco + (size_t)nbr[sl * 9 + d] * nc + col];
            }
            __syncthreads();
            // tpr consecutive threads share one row (idle threads otherwise)
            const int items = nrhs * len;
            int tpr = 1;
            while (tpr < 4 && items * tpr * 2 <= (int)blockDim.x) tpr *= 2;
            const int span = (9 * nc + tpr - 1) / tpr;
            for (int t0 = tid; t0 < ((items * tpr + 31) / 32) * 32; t0 += blockDim.x) {
                const int item = t0 / tpr, sub = t0 % tpr;
                const bool ok = item < items && live[item / len];
                Z acc; acc.x = 0; acc.y = 0;
                int j = 0, e = 0, sl = 0, r = 0;
                if (ok) {
                    j = item / len; e = item % len;
                    sl = e / nc; r = e % nc;
                    const Z* am = As + (size_t)sl * 9 * nc * nc + r;
                    const Z* xs = xn + ((size_t)j * nsl + sl) * 9 * nc;
                    const int d0 = sub * span, d1 = min(9 * nc, d0 + span);
                    for (int dc = d0; dc < d1; ++dc) acc += am[(size_t)dc * nc] * xs[dc];
                }
                for (int o = tpr / 2; o > 0; o >>= 1) {
                    acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
                    acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
                }
                if (ok && sub == 0) {
                    const Z* xs = xn + ((size_t)j * nsl + sl) * 9 * nc;
                    const R sg = r < nc / 2 ? R(1) : R(-1);
                    const R tj = (R)a.tau[j];
                    const Z xv = xs[r];      // direction 0 is the site itself
                    if (a.op == QCD_OP_D) { acc -= (tj * sg) * xv; }
                    else { acc = sg * acc; acc -= tj * xv; }
                    ws[(size_t)j * E + e] = acc;
                }
            }
        } else {
            for (int t = tid; t < nrhs * len; t += blockDim.x) {
                const int j = t / len, e = t % len;
                if (!live[j]) continue;
                const size_t ge = lo + e;
                const int s = (int)(ge / a.nc), r = (int)(ge % a.nc);
                int c[4];
                site_coords(a.gc, s, c);
                Z out;
                coarse_row<Z, R>(a, Vit + (size_t)j * nco, s, r, c, (R)a.tau[j], out);
                ws[(size_t)j * E + e] = out;
            }
        }
        __syncthreads();
        // classical Gram-Schmidt, pass 1, with ||w||^2 before the projection
        dots(TOT(par, 0), it + 1, true, ws);
        grid.sync();
        for (int t = tid; t < (it + 1) * nrhs; t += blockDim.x) {
            const double2 v = TOT(par, 0)[t];
            hc[t] = h1s[t] = hr[t] = mk<R>((R)v.x, (R)v.y);
        }
        if (tid == 0) againf[0] = 0;
        __syncthreads();
        // second pass only if some right-hand side lost more than 90% of its
        // squared norm in the first (a Kahan-Parlett test, loosened for a
        // solve that only needs a 0.5 reduction); every CTA takes the same
        // decision from the same totals
        if (tid < nrhs) {
            const int j = tid;
            const R before = (R)TOT(par, 0)[(maxit + 1) * nrhs + j].x;
            R proj = 0;
            for (int i = 0; i <= it; ++i) proj += h1s[i * nrhs + j].x * h1s[i * nrhs + j].x + h1s[i * nrhs + j].y * h1s[i * nrhs + j].y;
            after[j] = before - proj;
            if (live[j] && before - proj < R(0.1) * before) atomicOr(againf, 1);
        }
        __syncthreads();
        const int again = againf[0];
        project(it + 1);
        __syncthreads();
        if (again) {
            dots(TOT(par, 1), it + 1, true, ws);
            grid.sync();
            for (int t = tid; t < (it + 1) * nrhs; t += blockDim.x) {
                const double2 v = TOT(par, 1)[t];
                hc[t] = hr[t] = mk<R>((R)v.x, (R)v.y);
            }
            for (int t = tid; t < nrhs; t += blockDim.x) {
                const double2 v = TOT(par, 1)[(maxit + 1) * nrhs + t];
                hc[(maxit + 1) * nrhs + t] = mk<R>((R)v.x, (R)v.y);
            }
            __syncthreads();
            project(it + 1);
        } else {
            // no second pass: its coefficients are zero, ||w||^2 by Pythagoras
            for (int t = tid; t < (it + 1) * nrhs; t += blockDim.x) hc[t] = mk<R>(R(0), R(0));
            for (int j = tid; j < nrhs; j += blockDim.x) hc[(maxit + 1) * nrhs + j] = mk<R>(after[j], R(0));
            __syncthreads();
        }
        if (tid < nrhs) {
            const int j = tid;
            if (live[j]) {
                Z* h = hcol + (size_t)j * (maxit + 1);
                R h2n = 0;
                for (int i = 0; i <= it; ++i) {
                    const Z p2 = hc[i * nrhs + j];
                    h[i] = h1s[i * nrhs + j] + p2;
                    h2n += p2.x * p2.x + p2.y * p2.y;
                }
                const R hn2 = hc[(maxit + 1) * nrhs + j].x - h2n;
                const R hn = hn2 > R(0) ? sqrt(hn2) : R(0);
                hc[(maxit + 1) * nrhs + j] = mk<R>(hn, R(0));
                const double res = givens_column_t<R>(h, hn, cs + (size_t)j * maxit, sn + (size_t)j * maxit,
                                                      g + (size_t)j * (maxit + 1), it);
                if (blockIdx.x == 0) {
                    Z* Rj = reinterpret_cast<Z*>(a.Rg) + (size_t)j * maxit * maxit;
                    for (int i = 0; i <= it; ++i) Rj[(size_t)i * maxit + it] = h[i];
                    a.resid[j] = beta[j] > 0 ? res / beta[j] : 0.0;
                }
                kd[j] = it + 1;
                if (res <= a.tol * beta[j]) live[j] = -1;   // converged: finish this step, then stop
            }
        }
        __syncthreads();
        // v_{it+1} = w / hn
        for (int t = tid; t < nrhs * len; t += blockDim.x) {
            const int j = t / len, e = t % len;
            if (kd[j] != it + 1) continue;
            const R hn = hc[(maxit + 1) * nrhs + j].x;
            const R ih = hn > R(0) ? R(1) / hn : R(0);
            Z v = ws[(size_t)j * E + e];
            v.x *= ih; v.y *= ih;
            VS(it + 1, j)[e] = v;
            a.Vg[((size_t)(par ^ 1) * nrhs + j) * nco + lo + e] = v;
        }
        __syncthreads();
        for (int j = tid; j < nrhs; j += blockDim.x) if (live[j] < 0) live[j] = 0;
        __syncthreads();
    }
    // triangular solve (CTA 0) and x = V y
    if (blockIdx.x == 0 && tid < nrhs) {
        const int j = tid, k = kd[j];
        const Z* Rj = reinterpret_cast<const Z*>(a.Rg) + (size_t)j * maxit * maxit;
        const Z* gj = g + (size_t)j * (maxit + 1);
        Z* y = reinterpret_cast<Z*>(a.yv) + (size_t)j * maxit;
        for (int i = k - 1; i >= 0; --i) {
            Z sacc = gj[i];
            for (int l = i + 1; l < k; ++l) sacc -= Rj[(size_t)i * maxit + l] * y[l];
            const Z d = Rj[(size_t)i * maxit + i];
            const R den = d.x * d.x + d.y * d.y;
            y[i] = den > R(0) ? (R(1) / den) * cmulc(d, sacc) : mk<R>(R(0), R(0));
        }
        a.iters[j] = k;
        if (a.counter != nullptr && (a.act == nullptr || a.act[j])) {
            atomicAdd(a.counter, 1ull);
            atomicAdd(a.counter + 1, (unsigned long long)k);
        }
    }
    grid.sync();
    for (int t = tid; t < nrhs * len; t += blockDim.x) {
        const int j = t / len, e = t % len;
        if (a.act != nullptr && !a.act[j]) continue;
        const int k = kd[j];
        const Z* y = reinterpret_cast<const Z*>(a.yv) + (size_t)j * maxit;
        Z o; o.x = 0; o.y = 0;
        for (int i = 0; i < k; ++i) o += y[i] * VS(i, j)[e];
        a.x[(size_t)j * nco + lo + e] = o;
    }
}

}  // namespace

size_t kry_bytes(int nrhs, int maxit) {
    return sizeof(double) * nrhs * 2 + sizeof(int) * nrhs * 2 + sizeof(double) * (size_t)nrhs * maxit +
           sizeof(double2) * ((size_t)nrhs * maxit + (size_t)nrhs * (maxit + 1) + (size_t)nrhs * maxit * maxit +
                              (size_t)maxit * nrhs + nrhs) + 256;
}

KryDev kry_layout(void* buf, int nrhs, int maxit, double tol) {
    KryDev K;
    K.nrhs = nrhs;
    K.maxit = maxit;
    K.tol = tol;
    char* p = (char*)buf;
    auto take = [&](size_t bytes) { char* q = p; p += (bytes + 15) & ~size_t(15); return (void*)q; };
    K.g = (double2*)take(sizeof(double2) * (size_t)nrhs * (maxit + 1));
    K.sn = (double2*)take(sizeof(double2) * (size_t)nrhs * maxit);
    K.R = (double2*)take(sizeof(double2) * (size_t)nrhs * maxit * maxit);
    K.coef = (double2*)take(sizeof(double2) * (size_t)maxit * nrhs);
    K.scale = (double2*)take(sizeof(double2) * nrhs);
    K.cs = (double*)take(sizeof(double) * (size_t)nrhs * maxit);
    K.beta = (double*)take(sizeof(double) * nrhs);
    K.resid = (double*)take(sizeof(double) * nrhs);
    K.active = (int*)take(sizeof(int) * nrhs);
    K.k = (int*)take(sizeof(int) * nrhs);
    return K;
}

void kry_init(const KryDev& K, const double2* nrm, const int* outer_act, cudaStream_t st) {
    KTimer kt("kry_init", 0.0, 0.0, st);
    kry_init_kernel<<<1, 64, 0, st>>>(K, nrm, outer_act);
}
void kry_step(const KryDev& K, int it, const double2* h1, const double2* h2, const double2* nrm, cudaStream_t st) {
    KTimer kt("kry_step", 0.0, 0.0, st);
    kry_step_kernel<<<1, 64, 0, st>>>(K, it, h1, h2, nrm);
}
void kry_finish(const KryDev& K, cudaStream_t st) {
    KTimer kt("kry_finish", 0.0, 0.0, st);
    kry_finish_kernel<<<1, 64, 0, st>>>(K);
}

int coarse_gmres_grid() {
    static int nct = 0;
    if (nct == 0) {
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        nct = sms > 0 ? sms : 1;
    }
    return nct;
}

// Site-based partition: each CTA owns `sps` consecutive coarse sites.
static void coarse_partition(const Coarse& c, int& sps, int& nblk) {
    const int nct = c.ctas > 0 ? std::min(c.ctas, coarse_gmres_grid()) : coarse_gmres_grid();
    sps = (c.gc.V + nct - 1) / nct;
    nblk = (c.gc.V + sps - 1) / sps;
}
constexpr size_t kCoarseSmemCap = 200 * 1024;

// Where the cooperative kernel keeps its data, in order of preference:
// stencil blocks and Krylov basis in shared memory (layout 1), basis only
// (layout 2), basis in global memory (layout 3).  `want` = 0 picks the first
// that fits; 1..3 forces one (it must fit).
struct CoarseMode {
    int layout = 0;       // 1, 2, 3; 0: nothing fits
    size_t smem = 0;
};
static CoarseMode coarse_mode(const Coarse& c, int prec, int nrhs, int maxit, int want) {
    int sps, nblk;
    coarse_partition(c, sps, nblk);
    const int E = sps * c.nc;
    CoarseMode m;
    for (int layout = 1; layout <= 3; ++layout) {
        if (want != 0 && layout != want) continue;
        const int s = layout == 1 ? sps : 0, nc = layout == 1 ? c.nc : 0;
        const bool smem_basis = layout != 3;
        const size_t t = prec == QCD_FP64 ? coarse_smem<double2>(nrhs, maxit, E, s, nc, smem_basis).total
                                          : coarse_smem<float2>(nrhs, maxit, E, s, nc, smem_basis).total;
        if (t <= kCoarseSmemCap) {
            m.layout = layout;
            m.smem = t;
            return m;
        }
    }
    return m;
}

size_t coarse_gmres_scratch(const Coarse& c, int prec, int nrhs, int maxit, int want_layout) {
    const size_t nco = (size_t)c.gc.V * c.nc;
    const size_t es = prec == QCD_FP64 ? sizeof(double2) : sizeof(float2);
    const size_t npair = (size_t)(maxit + 2) * nrhs;
    size_t bytes = es * nco * nrhs * 2 + sizeof(double2) * (4 * npair + (size_t)nrhs * maxit * maxit + (size_t)nrhs * maxit) +
                   4096;
    if (coarse_mode(c, prec, nrhs, maxit, want_layout).layout == 3) {
        int sps, nblk;
        coarse_partition(c, sps, nblk);
        const size_t E = (size_t)sps * c.nc;
        bytes += es * nblk * E * nrhs * (size_t)(maxit + 2) + 1024;
    }
    return bytes;
}

// Right-hand sides per launch: the library's cap whenever some layout fits
// (the global-memory basis always does unless the bookkeeping alone is too big).
int coarse_gmres_group(const Coarse& c, int prec, int maxit, int want_layout) {
    for (int g = kMaxCoarseRhs; g >= 1; --g)
        if (coarse_mode(c, prec, g, maxit, want_layout).layout != 0) return g;
    return 0;
}

int coarse_gmres_layout(const Coarse& c, int prec, int nrhs, int maxit, int want_layout) {
    return coarse_mode(c, prec, nrhs, maxit, want_layout).layout;
}

template <typename Z, typename R>
static int launch_coarse(const Coarse& c, int op, int nrhs, const void* b, void* x, const double* tau_dev,
                         const int* act, double tol, int maxit, void* scratch, int* iters, double* resid,
                         unsigned long long* counter, int want_layout, cudaStream_t st) {
    const size_t nco = (size_t)c.gc.V * c.nc;
    int sps, nblk;
    coarse_partition(c, sps, nblk);
    const int E = sps * c.nc;
    const CoarseMode md = coarse_mode(c, std::is_same<R, double>::value ? QCD_FP64 : QCD_FP32, nrhs, maxit,
                                      want_layout);
    if (md.layout == 0) return -4;
    const size_t npair = (size_t)(maxit + 2) * nrhs;
    char* p = (char*)scratch;
    auto take = [&](size_t bytes) { char* q = p; p += (bytes + 255) & ~size_t(255); return (void*)q; };
    CoarseArgs<Z, R> a;
    a.gc = c.gc;
    a.nc = c.nc;
    a.A = std::is_same<R, double>::value ? (const Z*)c.A64 : (const Z*)c.A32;
    a.b = (const Z*)b;
    a.x = (Z*)x;
    a.Vg = (Z*)take(sizeof(Z) * nco * nrhs * 2);
    a.tot = (double2*)take(sizeof(double2) * 4 * npair);
    a.Rg = (double2*)take(sizeof(double2) * (size_t)nrhs * maxit * maxit);
    a.yv = (double2*)take(sizeof(double2) * (size_t)nrhs * maxit);
    a.Vglob = nullptr;
    a.wglob = nullptr;
    if (md.layout == 3) {
        a.Vglob = (Z*)take(sizeof(Z) * (size_t)nblk * (maxit + 1) * nrhs * E);
        a.wglob = (Z*)take(sizeof(Z) * (size_t)nblk * nrhs * E);
    }
    a.iters = iters;
    a.counter = counter;
    a.resid = resid;
    a.op = op;
    a.tau = tau_dev;
    a.act = act;
    a.tol = tol;
    a.maxit = maxit;
    a.nrhs = nrhs;
    a.E = E;
    a.sps = sps;
    a.a_smem = md.layout == 1 ? 1 : 0;
    cudaMemsetAsync(a.tot, 0, sizeof(double2) * 4 * npair, st);
    auto kern = coarse_gmres_kernel<Z, R>;
    const size_t sm = md.smem;
    if (sm + 1024 > 48 * 1024) cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 256, sm);
    if (per_sm < 1) return -1;
    void* args[] = {&a};
    const double es = sizeof(Z);
    KTimer kt(std::is_same<R, double>::value ? "coarse_gmres_f64" : "coarse_gmres_f32",
              es * ((double)c.gc.V * 9 * c.nc * c.nc + 4.0 * nrhs * nco), 0.0, st);
    cudaError_t e = cudaLaunchCooperativeKernel((void*)kern, dim3(nblk), dim3(256), args, sm, st);
    return e == cudaSuccess ? 0 : -2;
}

int coarse_gmres(const Coarse& c, int prec, int op, int nrhs, const void* b, void* x, const double* tau_dev,
                 const int* act, double tol, int maxit, void* scratch, int* iters, double* resid,
                 unsigned long long* counter, int want_layout, cudaStream_t st) {
    if (nrhs < 1 || nrhs > kMaxCoarseRhs || maxit < 1 || maxit > kMaxCoarse) return -3;
    if (prec == QCD_FP64)
        return launch_coarse<double2, double>(c, op, nrhs, b, x, tau_dev, act, tol, maxit, scratch, iters, resid,
                                              counter, want_layout, st);
    return launch_coarse<float2, float>(c, op, nrhs, b, x, tau_dev, act, tol, maxit, scratch, iters, resid, counter,
                                        want_layout, st);
}

}  // namespace qcd
