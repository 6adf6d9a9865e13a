// Multigrid kernels: chirality-split aggregation P (Sec. 2, above Eq. 2.9),
// restriction P^H and prolongation P (Eq. 2.8), the Galerkin coarse stencil
// D_c = P^H D P (Eq. 2.8, 2.9) and the SAP block solves of Eq. 2.10.
#include <algorithm>

#include <cuda_fp16.h>

#include "internal.h"
#include "dirac.cuh"

namespace qcd {

namespace {

// Work counters of the SAP block solves (for the FP32-ALU roofline): [0] sums
// block sites x GMRES steps, [1] block sites x k (k + 1) / 2 over all block
// solves; 64 slots per counter spread the atomics of one launch.
__device__ unsigned long long g_sap_work[2][64];

__device__ __forceinline__ void count_sap_work(int bs, int kdim) {
    const int slot = (blockIdx.x + 7 * blockIdx.y) & 63;
    atomicAdd(&g_sap_work[0][slot], (unsigned long long)bs * kdim);
    atomicAdd(&g_sap_work[1][slot], (unsigned long long)bs * kdim * (kdim + 1) / 2);
}

// sum of a double2 over the first blockDim.x (power of two) threads
__device__ __forceinline__ double2 block_sum2(double2 v, double2* red) {
    const int t = threadIdx.x;
    red[t] = v;
    __syncthreads();
    for (int s = blockDim.x >> 1; s > 0; s >>= 1) {
        if (t < s) red[t] += red[t + s];
        __syncthreads();
    }
    double2 r = red[0];
    __syncthreads();
    return r;
}

__device__ __forceinline__ void block_coords(const Blocking& B, int blk, int c[4]) {
    int t = blk;
    c[3] = t % B.cd[3]; t /= B.cd[3];
    c[2] = t % B.cd[2]; t /= B.cd[2];
    c[1] = t % B.cd[1]; c[0] = t / B.cd[1];
}
__device__ __forceinline__ void local_coords(const Blocking& B, int l, int o[4]) {
    int t = l;
    o[3] = t % B.b[3]; t /= B.b[3];
    o[2] = t % B.b[2]; t /= B.b[2];
    o[1] = t % B.b[1]; o[0] = t / B.b[1];
}
__device__ __forceinline__ int coarse_index(const Blocking& B, const int c[4]) {
    return ((c[0] * B.cd[1] + c[1]) * B.cd[2] + c[2]) * B.cd[3] + c[3];
}
__device__ __forceinline__ int local_index(const Blocking& B, const int o[4]) {
    return ((o[0] * B.b[1] + o[1]) * B.b[2] + o[2]) * B.b[3] + o[3];
}

// ------------------------------------------------------------------ P build
// One CTA per (coarse site, chirality): gather the nvec restricted test
// vectors, then modified Gram-Schmidt applied twice (FP64).
__global__ void build_P_kernel(Geom g, Blocking B, int nv, const double2* __restrict__ vecs, double2* __restrict__ P64,
                               float2* __restrict__ P32) {
    extern __shared__ double2 red[];
    const int blk = blockIdx.x, chi = blockIdx.y;
    const int nloc = B.bs * 6;
    double2* Pb = P64 + ((size_t)blk * 2 + chi) * nv * nloc;
    for (int i = 0; i < nv; ++i)
        for (int d = threadIdx.x; d < nloc; d += blockDim.x) {
            int l = d / 6, sc = d % 6;
            int site = block_fine_site(g, B, blk, l);
            Pb[(size_t)i * nloc + d] = vecs[(size_t)i * g.V * 12 + (size_t)site * 12 + 6 * chi + sc];
        }
    __syncthreads();
    for (int pass = 0; pass < 2; ++pass) {
        for (int i = 0; i < nv; ++i) {
            double2* pi = Pb + (size_t)i * nloc;
            for (int j = 0; j < i; ++j) {
                const double2* pj = Pb + (size_t)j * nloc;
                double2 h = make_double2(0, 0);
                for (int d = threadIdx.x; d < nloc; d += blockDim.x) h += cmulc(pj[d], pi[d]);
                h = block_sum2(h, red);
                for (int d = threadIdx.x; d < nloc; d += blockDim.x) pi[d] -= h * pj[d];
                __syncthreads();
            }
            double2 nn = make_double2(0, 0);
            for (int d = threadIdx.x; d < nloc; d += blockDim.x) nn.x += pi[d].x * pi[d].x + pi[d].y * pi[d].y;
            nn = block_sum2(nn, red);
            double inv = nn.x > 0 ? 1.0 / sqrt(nn.x) : 0.0;
            for (int d = threadIdx.x; d < nloc; d += blockDim.x) pi[d] = inv * pi[d];
            __syncthreads();
        }
    }
    float2* Pb32 = P32 + ((size_t)blk * 2 + chi) * nv * nloc;
    for (int d = threadIdx.x; d < nv * nloc; d += blockDim.x) Pb32[d] = cvt<float2>(Pb[d]);
}

// ------------------------------------------------------------------ restrict / prolong
// One warp per (coarse site, chirality, vector i): <P_i, r_j> over the
// aggregate for a chunk of up to kRestrictRC right-hand sides at a time, so
// each entry of P is read once per chunk instead of once per right-hand side.
constexpr int kRestrictRC = 8;
template <typename Z, typename R>
__global__ void restrict_kernel(Geom g, Blocking B, int nv, const Z* __restrict__ P, const Z* __restrict__ r,
                                Z* __restrict__ xc, int nrhs, const int* __restrict__ act) {
    const int nc = 2 * nv;
    const int nloc = B.bs * 6;
    const long total = (long)B.nb * nc;
    const int lane = threadIdx.x & 31;
    const size_t fstride = (size_t)g.V * 12;
    for (long w = (blockIdx.x * (long)blockDim.x + threadIdx.x) >> 5; w < total; w += ((long)gridDim.x * blockDim.x) >> 5) {
        const int blk = (int)(w / nc), ci = (int)(w % nc);
        const int chi = ci / nv, i = ci % nv;
        const Z* p = P + (((size_t)blk * 2 + chi) * nv + i) * nloc;
        for (int j0 = 0; j0 < nrhs; j0 += kRestrictRC) {
            R re[kRestrictRC], im[kRestrictRC];
#pragma unroll
            for (int q = 0; q < kRestrictRC; ++q) { re[q] = 0; im[q] = 0; }
            for (int d = lane; d < nloc; d += 32) {
                const int l = d / 6, sc = d % 6;
                const size_t off = (size_t)block_fine_site(g, B, blk, l) * 12 + 6 * chi + sc;
                const Z a = p[d];
#pragma unroll
                for (int q = 0; q < kRestrictRC; ++q) {
                    const int j = j0 + q;
                    if (j >= nrhs || (act != nullptr && !act[j])) continue;
                    const Z b = r[(size_t)j * fstride + off];
                    re[q] += a.x * b.x + a.y * b.y;
                    im[q] += a.x * b.y - a.y * b.x;
                }
            }
#pragma unroll
            for (int q = 0; q < kRestrictRC; ++q) {
                re[q] = warp_sum(re[q]);
                im[q] = warp_sum(im[q]);
            }
            if (lane == 0)
#pragma unroll
                for (int q = 0; q < kRestrictRC; ++q) {
                    const int j = j0 + q;
                    if (j >= nrhs || (act != nullptr && !act[j])) continue;
                    Z o; o.x = re[q]; o.y = im[q];
                    xc[(size_t)j * B.nb * nc + (size_t)blk * nc + ci] = o;
                }
        }
    }
}

// One CTA per (aggregate, chirality, chunk of RC right-hand sides): the
// aggregate's half of each fine vector (nloc = 6 x block sites entries) is
// gathered into shared memory once ([rhs][d], conflict-free for consecutive
// d), then the warps take the nv vectors P_i in turn, so every fine entry is
// read from memory once and every entry of P once per chunk.
template <typename Z, typename R, int RC>
__global__ void __launch_bounds__(256) restrict_agg_kernel(Geom g, Blocking B, int nv, const Z* __restrict__ P,
                                                           const Z* __restrict__ r, Z* __restrict__ xc, int nrhs,
                                                           const int* __restrict__ act) {
    extern __shared__ __align__(16) unsigned char rsm[];
    Z* rs = reinterpret_cast<Z*>(rsm);   // [RC][nloc]
    const int nc = 2 * nv;
    const int nloc = B.bs * 6;
    const int blk = blockIdx.x >> 1, chi = blockIdx.x & 1;
    const int j0 = blockIdx.y * RC;
    const size_t fstride = (size_t)g.V * 12;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarp = blockDim.x >> 5;
    for (int e = tid; e < nloc * RC; e += blockDim.x) {
        const int q = e / nloc, d = e % nloc, j = j0 + q;
        Z v;
        v.x = 0;
        v.y = 0;
        if (j < nrhs && (act == nullptr || act[j])) {
            const int l = d / 6, sc = d % 6;
            v = r[(size_t)j * fstride + (size_t)block_fine_site(g, B, blk, l) * 12 + 6 * chi + sc];
        }
        rs[(size_t)q * nloc + d] = v;
    }
    __syncthreads();
    for (int i = warp; i < nv; i += nwarp) {
        const Z* p = P + (((size_t)blk * 2 + chi) * nv + i) * nloc;
        R re[RC], im[RC];
#pragma unroll
        for (int q = 0; q < RC; ++q) { re[q] = 0; im[q] = 0; }
        for (int d = lane; d < nloc; d += 32) {
            const Z a = p[d];
#pragma unroll
            for (int q = 0; q < RC; ++q) {
                const Z b = rs[(size_t)q * nloc + d];
                re[q] += a.x * b.x + a.y * b.y;
                im[q] += a.x * b.y - a.y * b.x;
            }
        }
#pragma unroll
        for (int q = 0; q < RC; ++q) {
            re[q] = warp_sum(re[q]);
            im[q] = warp_sum(im[q]);
        }
        if (lane == 0) {
#pragma unroll
            for (int q = 0; q < RC; ++q) {
                const int j = j0 + q;
                if (j >= nrhs || (act != nullptr && !act[j])) continue;
                Z o;
                o.x = re[q];
                o.y = im[q];
                xc[(size_t)j * B.nb * nc + (size_t)blk * nc + chi * nv + i] = o;
            }
        }
    }
}

// One thread per fine degree of freedom of an aggregate (coarse site,
// chirality, local index d); the nv entries P_i[d] are read once per chunk of
// kProlongRC right-hand sides.
constexpr int kProlongRC = 4;
template <typename Z>
__global__ void prolong_kernel(Geom g, Blocking B, int nv, const Z* __restrict__ P, const Z* __restrict__ xc,
                               Z* __restrict__ x, int nrhs, bool accumulate, const int* __restrict__ act) {
    const int nc = 2 * nv;
    const int nloc = B.bs * 6;
    const size_t total = (size_t)B.nb * 2 * nloc;
    const size_t fstride = (size_t)g.V * 12, cstride = (size_t)B.nb * nc;
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total; t += (size_t)gridDim.x * blockDim.x) {
        const int blk = (int)(t / (2 * nloc));
        const int chi = (int)((t / nloc) % 2);
        const int d = (int)(t % nloc);
        const Z* p = P + ((size_t)blk * 2 + chi) * nv * nloc + d;
        const int l = d / 6, sc = d % 6;
        const size_t idx = (size_t)block_fine_site(g, B, blk, l) * 12 + 6 * chi + sc;
        const Z* c0 = xc + (size_t)blk * nc + chi * nv;
        for (int j0 = 0; j0 < nrhs; j0 += kProlongRC) {
            Z acc[kProlongRC];
#pragma unroll
            for (int q = 0; q < kProlongRC; ++q) { acc[q].x = 0; acc[q].y = 0; }
            for (int i = 0; i < nv; ++i) {
                const Z pi = p[(size_t)i * nloc];
#pragma unroll
                for (int q = 0; q < kProlongRC; ++q)
                    if (j0 + q < nrhs) acc[q] += pi * c0[(size_t)(j0 + q) * cstride + i];
            }
#pragma unroll
            for (int q = 0; q < kProlongRC; ++q) {
                const int j = j0 + q;
                if (j >= nrhs || (act != nullptr && !act[j])) continue;
                Z o = acc[q];
                if (accumulate) o += x[(size_t)j * fstride + idx];
                x[(size_t)j * fstride + idx] = o;
            }
        }
    }
}

// ------------------------------------------------------------------ coarse build
// CTA (coarse site blk, direction d): column by column, h(l) = the part of
// (D P e_col)(y_l) that D couples from block blk + d (d = 0: site-diagonal and
// in-block hops), then A[blk][d][col][row] = P_blk[row]^H h.
template <typename R>
__device__ __forceinline__ void P_spinor(const cplx<R>* __restrict__ P, int nv, int nloc, int blk, int chi, int i, int l,
                                         Spinor<R>& s) {
#pragma unroll
    for (int k = 0; k < 12; ++k) s.c[k] = czero<R>();
    const cplx<R>* p = P + (((size_t)blk * 2 + chi) * nv + i) * nloc + (size_t)l * 6;
#pragma unroll
    for (int k = 0; k < 6; ++k) s.c[6 * chi + k] = p[k];
}

template <bool fwd, typename R>
__device__ __forceinline__ void hop_dispatch(int mu, const Spinor<R>& psi, const Link<R>& u, R sg, Spinor<R>& acc) {
    switch (mu) {
        case 0: hop_accumulate<R, 0, fwd>(psi, u, sg, acc); break;
        case 1: hop_accumulate<R, 1, fwd>(psi, u, sg, acc); break;
        case 2: hop_accumulate<R, 2, fwd>(psi, u, sg, acc); break;
        default: hop_accumulate<R, 3, fwd>(psi, u, sg, acc); break;
    }
}

// Sites of block blk that direction d draws from: all bs for d = 0, the
// sites on the face towards block blk + d otherwise (none when the block grid
// has extent 1 in that direction, whose hops wrap into d = 0).
__device__ __forceinline__ bool coarse_active(const Blocking& B, int d, const int o[4]) {
    if (d == 0) return true;
    const bool fw = d <= 4;
    const int mu = (d - 1) % 4;
    return (fw ? o[mu] == B.b[mu] - 1 : o[mu] == 0) && B.cd[mu] > 1;
}

// Columns col0 .. col0+nch-1 at a time: every thread takes (column, active
// site) tasks and leaves h in shared memory ([column][active site][12]);
// then one warp per (column, row) entry forms P_blk[row]^H h over the active
// sites only.
template <typename R>
__global__ void __launch_bounds__(256) build_coarse_kernel(Geom g, Blocking B, int nv, const cplx<R>* __restrict__ U,
                                                          const R* __restrict__ A, const cplx<R>* __restrict__ P,
                                                          cplx<R>* __restrict__ Ac, int chunk) {
    extern __shared__ __align__(16) unsigned char hraw[];
    cplx<R>* hsm = reinterpret_cast<cplx<R>*>(hraw);   // [chunk][na][12], then na ints
    int* lst = reinterpret_cast<int*>(hsm + (size_t)chunk * B.bs * 12);
    __shared__ int na_s;
    const int blk = blockIdx.x, d = blockIdx.y;
    const int nc = 2 * nv, nloc = B.bs * 6;
    int cb[4];
    block_coords(B, blk, cb);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
    if (threadIdx.x == 0) {
        int c = 0;
        for (int l = 0; l < B.bs; ++l) {
            int o[4];
            local_coords(B, l, o);
            if (coarse_active(B, d, o)) lst[c++] = l;
        }
        na_s = c;
    }
    __syncthreads();
    const int na = na_s;
    for (int col0 = 0; col0 < nc; col0 += chunk) {
        const int nch = min(chunk, nc - col0);
        for (int t = threadIdx.x; t < nch * na; t += blockDim.x) {
            const int cc = t / na, a = t % na;
            const int col = col0 + cc, l = lst[a];
            const int chic = col / nv, ic = col % nv;
            int o[4], x[4];
            local_coords(B, l, o);
            for (int mu = 0; mu < 4; ++mu) x[mu] = cb[mu] * B.b[mu] + o[mu];
            const int y = site_index(g, x);
            Spinor<R> acc;
#pragma unroll
            for (int k = 0; k < 12; ++k) acc.c[k] = czero<R>();
            if (d == 0) {
                Spinor<R> ps;
                P_spinor<R>(P, nv, nloc, blk, chic, ic, l, ps);
                clover_apply<R>(A + (size_t)y * 72, ps, acc);
            }
            for (int mu = 0; mu < 4; ++mu) {
                for (int dir = 0; dir < 2; ++dir) {
                    const bool fw = dir == 0;
                    const bool face = (fw ? (o[mu] == B.b[mu] - 1) : (o[mu] == 0)) && B.cd[mu] > 1;
                    const int want = face ? (fw ? 1 + mu : 5 + mu) : 0;
                    if (want != d) continue;
                    int neg;
                    const int yn = fw ? nb_fwd(g, x, y, mu, neg) : nb_bwd(g, x, y, mu, neg);
                    int xn[4];
                    site_coords(g, yn, xn);
                    int cn[4], on[4];
                    for (int k = 0; k < 4; ++k) { cn[k] = xn[k] / B.b[k]; on[k] = xn[k] % B.b[k]; }
                    Spinor<R> ps;
                    P_spinor<R>(P, nv, nloc, coarse_index(B, cn), chic, ic, local_index(B, on), ps);
                    Link<R> u;
                    load_link<R>(U + ((size_t)(fw ? y : yn) * 4 + mu) * 9, u);
                    if (fw) hop_dispatch<true, R>(mu, ps, u, neg ? R(-1) : R(1), acc);
                    else hop_dispatch<false, R>(mu, ps, u, neg ? R(-1) : R(1), acc);
                }
            }
            cplx<R>* h = hsm + ((size_t)cc * na + a) * 12;
#pragma unroll
            for (int k = 0; k < 12; ++k) h[k] = acc.c[k];
        }
        __syncthreads();
        for (int e = warp; e < nch * nc; e += nwarps) {
            const int cc = e / nc, row = e % nc;
            const int chir = row / nv, ir = row % nv;
            const cplx<R>* pr = P + (((size_t)blk * 2 + chir) * nv + ir) * nloc;
            const cplx<R>* h = hsm + (size_t)cc * na * 12 + 6 * chir;
            R re = 0, im = 0;
            for (int q = lane; q < na * 6; q += 32) {
                const int a = q / 6, sc = q % 6;
                const cplx<R> pv = pr[lst[a] * 6 + sc], hv = h[a * 12 + sc];
                re += pv.x * hv.x + pv.y * hv.y;
                im += pv.x * hv.y - pv.y * hv.x;
            }
            re = warp_sum(re);
            im = warp_sum(im);
            if (lane == 0) Ac[(((size_t)blk * 9 + d) * nc + col0 + cc) * nc + row] = mk<R>(re, im);
        }
        __syncthreads();
    }
}

__global__ void narrow_kernel(const double2* __restrict__ a, float2* __restrict__ b, size_t n) {
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x)
        b[t] = cvt<float2>(a[t]);
}

// ------------------------------------------------------------------ coarse apply
// Multi-right-hand-side coarse stencil: one CTA per (coarse site, chunk of
// up to kCoarseRC right-hand sides).  The 9 neighbour vectors of the chunk
// are staged in shared memory ([d][col][rhs]); every stencil block entry is
// then loaded once per chunk (coalesced: consecutive threads take consecutive
// rows of the column-major blocks) and multiplied into kCoarseRPT
// right-hand sides held in registers, so the (2 Nv)^2 x 9 blocks -- the bulk
// of the bytes -- are read once per chunk instead of once per right-hand side.
constexpr int kCoarseRC = 16;
constexpr int kCoarseRPT = 4;
template <typename Z, typename R>
__global__ void coarse_apply_mrhs_kernel(Geom gc, int nc, const Z* __restrict__ A, const Z* __restrict__ x,
                                         Z* __restrict__ y, int op, Shifts tau, int nrhs, int rc) {
    extern __shared__ __align__(16) unsigned char craw[];
    Z* xs = reinterpret_cast<Z*>(craw);                 // [9][nc][rc]
    __shared__ int nbr[9];
    const int s = blockIdx.x;
    const int j0 = blockIdx.y * rc;
    const size_t vstride = (size_t)gc.V * nc;
    if (threadIdx.x < 9) {
        const int d = threadIdx.x;
        int c[4];
        site_coords(gc, s, c);
        int sn = s;
        if (d > 0) {
            const int mu = (d - 1) & 3, step = d <= 4 ? 1 : -1;
            c[mu] = (c[mu] + step + gc.L[mu]) % gc.L[mu];
            sn = site_index(gc, c);
        }
        nbr[d] = sn;
    }
    __syncthreads();
    const int nstage = 9 * nc * rc;
    for (int e0 = threadIdx.x; e0 < nstage; e0 += 8 * blockDim.x) {
        Z v[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int e = e0 + q * blockDim.x;
            v[q].x = 0; v[q].y = 0;
            if (e < nstage) {
                const int col = e % nc, jj = (e / nc) % rc, d = e / (nc * rc);
                if (j0 + jj < nrhs) v[q] = __ldg(x + (size_t)(j0 + jj) * vstride + (size_t)nbr[d] * nc + col);
            }
        }
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int e = e0 + q * blockDim.x;
            if (e < nstage) {
                const int col = e % nc, jj = (e / nc) % rc, d = e / (nc * rc);
                xs[((size_t)d * nc + col) * rc + jj] = v[q];
            }
        }
    }
    __syncthreads();
    const int r = threadIdx.x % nc, grp = threadIdx.x / nc;
    if (grp * kCoarseRPT >= rc) return;
    Z acc[kCoarseRPT];
#pragma unroll
    for (int k = 0; k < kCoarseRPT; ++k) { acc[k].x = 0; acc[k].y = 0; }
    const Z* As = A + (size_t)s * 9 * nc * nc + r;
    for (int d = 0; d < 9; ++d) {
        const Z* Ad = As + (size_t)d * nc * nc;
        const Z* xd = xs + (size_t)d * nc * rc + grp * kCoarseRPT;
#pragma unroll 4
        for (int col = 0; col < nc; ++col) {
            const Z a = __ldg(Ad + (size_t)col * nc);
            const Z* xv = xd + (size_t)col * rc;
#pragma unroll
            for (int k = 0; k < kCoarseRPT; ++k) acc[k] += a * xv[k];
        }
    }
    const R sg = r < nc / 2 ? R(1) : R(-1);
#pragma unroll
    for (int k = 0; k < kCoarseRPT; ++k) {
        const int jj = grp * kCoarseRPT + k, j = j0 + jj;
        if (j >= nrhs) break;
        const R tj = (R)tau.t[j];
        const Z xv = xs[(size_t)r * rc + jj];        // direction 0 is the site itself
        Z o = acc[k];
        if (op == QCD_OP_D) { o -= (tj * sg) * xv; }
        else { o = sg * o; o -= tj * xv; }
        y[(size_t)j * vstride + (size_t)s * nc + r] = o;
    }
}

// ---- asynchronous bulk copies (TMA engine) into shared memory, completion
// tracked by an mbarrier.  Every wait is bounded in time: a wait that gives up
// counts itself in g_wait_timeouts and the caller skips its work.
__device__ unsigned long long g_wait_timeouts;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
// global -> shared copy of `bytes` (multiple of 16; both addresses 16-byte aligned)
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}
__device__ __forceinline__ bool mbar_try(uint64_t* bar, unsigned parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// wait for phase `parity` of the barrier, giving up after `limit` clocks
// (default 2^30, ~0.5 s)
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity, long long limit = 1ll << 30) {
    if (mbar_try(bar, parity)) return true;
    const long long t0 = clock64();
    while (!mbar_try(bar, parity)) {
        if (clock64() - t0 > limit) {
            atomicAdd(&g_wait_timeouts, 1ull);
            return false;
        }
    }
    return true;
}
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// Self-test of the bounded wait: one warp waits on an mbarrier that nothing
// arrives at, gives up after `limit` clocks, counts itself and returns.
__global__ void wait_probe_kernel(long long limit) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (threadIdx.x == 0) mbar_wait(&bar, 0, limit);
}

// FP32 coarse stencil on up to kBulkR right-hand sides per CTA, one coarse
// site per CTA.  The 9 stencil blocks A_d (nc x nc complex, contiguous) and
// the matching neighbour vectors (nc complex per right-hand side) stream
// through two shared-memory stages filled by bulk asynchronous copies, so
// each block is read from HBM exactly once while the previous one is
// multiplied.  Thread (row r, group q) accumulates row r of y for the 8
// right-hand sides 8q .. 8q+7: per column one block entry and eight
// broadcast vector entries feed 32 FMAs.
constexpr int kBulkR = 16;
constexpr int kBulkG = 8;   // right-hand sides per thread

// stage: block A_d, then the vectors of right-hand sides 0..7, 16 bytes of
// padding (the two thread groups' broadcast reads then fall in different
// banks), then right-hand sides 8..15
__host__ __device__ inline size_t coarse_bulk_stage_bytes(int nc) {
    return sizeof(float2) * ((size_t)nc * nc + (size_t)kBulkR * nc) + 16;
}
__host__ __device__ inline size_t coarse_bulk_xoff(int nc, int j) {
    return sizeof(float2) * ((size_t)nc * nc + (size_t)j * nc) + (j >= kBulkG ? 16 : 0);
}
size_t coarse_bulk_smem(int nc) { return 2 * coarse_bulk_stage_bytes(nc); }

__global__ void __launch_bounds__(128) coarse_apply_bulk_kernel(Geom gc, int nc, const float2* __restrict__ A,
                                                                const float2* __restrict__ x,
                                                                float2* __restrict__ y, int op, Shifts tau,
                                                                int nrhs) {
    extern __shared__ __align__(128) unsigned char bsm[];
    __shared__ __align__(8) uint64_t bar[2];
    __shared__ int nbr[9];
    __shared__ int fail;
    const int s = blockIdx.x, j0 = blockIdx.y * kBulkR;
    const int nr = min(kBulkR, nrhs - j0);
    const int tid = threadIdx.x;
    const size_t vstride = (size_t)gc.V * nc;
    const size_t stage = coarse_bulk_stage_bytes(nc);
    if (tid < 9) {
        int c[4];
        site_coords(gc, s, c);
        int sn = s;
        if (tid > 0) {
            const int mu = (tid - 1) & 3, step = tid <= 4 ? 1 : -1;
            c[mu] = (c[mu] + step + gc.L[mu]) % gc.L[mu];
            sn = site_index(gc, c);
        }
        nbr[tid] = sn;
    }
    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fail = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    const unsigned ablk = (unsigned)(sizeof(float2) * nc * nc), vseg = (unsigned)(sizeof(float2) * nc);
    // stage d: block A_d and the neighbour vectors x_j(nbr[d]), j < nr
    auto issue = [&](int d) {
        unsigned char* buf = bsm + (d & 1) * stage;
        if (tid == 0) {
            fence_async_smem();
            mbar_expect_tx(&bar[d & 1], ablk + (unsigned)nr * vseg);
        }
        __syncwarp();
        if (tid < 32) {
            if (tid == 0) bulk_g2s(buf, A + ((size_t)s * 9 + d) * nc * nc, ablk, &bar[d & 1]);
            for (int j = tid; j < nr; j += 32)
                bulk_g2s(buf + coarse_bulk_xoff(nc, j), x + (size_t)(j0 + j) * vstride + (size_t)nbr[d] * nc, vseg,
                         &bar[d & 1]);
        }
    };
    issue(0);
    issue(1);
    const int r = tid % nc, q = tid / nc;
    const bool active = q * kBulkG < nr;
    float2 acc[kBulkG], xself[kBulkG];
#pragma unroll
    for (int k = 0; k < kBulkG; ++k) { acc[k] = make_float2(0.f, 0.f); xself[k] = make_float2(0.f, 0.f); }
    for (int d = 0; d < 9; ++d) {
        const unsigned char* buf = bsm + (d & 1) * stage;
        if (!mbar_wait(&bar[d & 1], (unsigned)((d >> 1) & 1))) fail = 1;
        __syncthreads();
        if (fail) {
            // copies may still be in flight into this CTA's shared memory
            // (stages d and d + 1): wait for them once more, bounded, then
            // leave without writing y
            if (tid == 0) {
                mbar_wait(&bar[d & 1], (unsigned)((d >> 1) & 1));
                if (d + 1 < 9) mbar_wait(&bar[(d + 1) & 1], (unsigned)(((d + 1) >> 1) & 1));
            }
            __syncthreads();
            return;
        }
        const float2* As = reinterpret_cast<const float2*>(buf);
        const float2* Xs = reinterpret_cast<const float2*>(buf + coarse_bulk_xoff(nc, q * kBulkG));
        if (active) {
            if (d == 0) {
#pragma unroll
                for (int k = 0; k < kBulkG; ++k) xself[k] = Xs[(size_t)k * nc + r];
            }
            // two columns per step: one 16-byte broadcast load per right-hand side
#pragma unroll 2
            for (int col = 0; col < nc; col += 2) {
                const float2 a0 = As[(size_t)col * nc + r], a1 = As[(size_t)(col + 1) * nc + r];
#pragma unroll
                for (int k = 0; k < kBulkG; ++k) {
                    const float4 xv = *reinterpret_cast<const float4*>(Xs + (size_t)k * nc + col);
                    acc[k].x = fmaf(a0.x, xv.x, fmaf(-a0.y, xv.y, acc[k].x));
                    acc[k].y = fmaf(a0.x, xv.y, fmaf(a0.y, xv.x, acc[k].y));
                    acc[k].x = fmaf(a1.x, xv.z, fmaf(-a1.y, xv.w, acc[k].x));
                    acc[k].y = fmaf(a1.x, xv.w, fmaf(a1.y, xv.z, acc[k].y));
                }
            }
        }
        __syncthreads();   // stage d & 1 no longer read
        if (d + 2 < 9) issue(d + 2);
    }
    if (!active) return;
    const float sg = r < nc / 2 ? 1.f : -1.f;
#pragma unroll
    for (int k = 0; k < kBulkG; ++k) {
        const int j = j0 + q * kBulkG + k;
        if (j >= nrhs) break;
        const float tj = (float)tau.t[j];
        float2 o = acc[k];
        const float2 xv = xself[k];
        if (op == QCD_OP_D) { o -= (tj * sg) * xv; }
        else { o = sg * o; o -= tj * xv; }
        y[(size_t)j * vstride + (size_t)s * nc + r] = o;
    }
}

// Tensor-core coarse stencil (FP32 data, 3xTF32 products): per coarse site
// and chunk of kTcR right-hand sides, the stencil is one real GEMM
//   [Re y; Im y] (2nc x R) = sum_d [[Re A_d, -Im A_d], [Im A_d, Re A_d]] (2nc x 2nc)
//                            [Re x_d; Im x_d] (2nc x R),
// x_d the neighbour in direction d.  Each warp owns a 16-row tile of the
// result and runs mma.sync m16n8k8 (TF32 in, FP32 accumulate) over K = 9 x 2nc;
// every operand is split as big + small TF32 parts and the three products
// small*big + big*small + big*big keep FP32-level accuracy.  The neighbour
// vectors are staged once ([d][k][r], padded rows: conflict-free fragment
// loads); the blocks A_d one direction at a time.  Needs nc % 8 == 0.
constexpr int kTcR = 16;
constexpr int kTcXs = 24;   // padded row stride of the staged vectors (floats)
constexpr int kTcPre = 16;  // prefetched block entries per thread: nc^2 <= 16 x 32 (nc / 8)

__device__ __forceinline__ uint32_t tf32_of(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ void tf32_split(float x, uint32_t& big, uint32_t& small) {
    big = tf32_of(x);
    small = tf32_of(x - __uint_as_float(big));
}
__device__ __forceinline__ void mma_tf32(float (&c)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// column stride of the staged block (complex entries): 2 x stride = 16 mod 32
// words, so the four columns of a fragment load fall on disjoint bank halves
__host__ __device__ inline int tc_astride(int nc) { return nc + (24 - nc % 16) % 16; }

__global__ void coarse_apply_tc_kernel(Geom gc, int nc, const float2* __restrict__ A, const float2* __restrict__ x,
                                       float2* __restrict__ y, int op, Shifts tau, int nrhs) {
    extern __shared__ __align__(16) float tsm[];
    const int n2 = 2 * nc, astride = tc_astride(nc);
    float* Xs = tsm;                                               // [9][2nc][kTcXs]
    float2* As = reinterpret_cast<float2*>(Xs + (size_t)9 * n2 * kTcXs);   // [nc cols][astride]
    float* Ys = reinterpret_cast<float*>(As);                      // [2nc][kTcR], after the last direction
    __shared__ int nbr[9];
    const int s = blockIdx.x, j0 = blockIdx.y * kTcR;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int g = lane >> 2, t = lane & 3;
    const size_t vstride = (size_t)gc.V * nc;
    if (tid < 9) {
        int c[4];
        site_coords(gc, s, c);
        int sn = s;
        if (tid > 0) {
            const int mu = (tid - 1) & 3, step = tid <= 4 ? 1 : -1;
            c[mu] = (c[mu] + step + gc.L[mu]) % gc.L[mu];
            sn = site_index(gc, c);
        }
        nbr[tid] = sn;
    }
    __syncthreads();
    // stage the neighbour vectors: batches of 8 loads in flight per thread
    const int nstage = 9 * nc * kTcR;
    for (int e0 = tid; e0 < nstage; e0 += 8 * blockDim.x) {
        float2 v[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int e = e0 + q * blockDim.x;
            v[q] = make_float2(0.f, 0.f);
            if (e < nstage) {
                const int col = e % nc, r = (e / nc) % kTcR, d = e / (nc * kTcR);
                if (j0 + r < nrhs) v[q] = __ldg(x + (size_t)(j0 + r) * vstride + (size_t)nbr[d] * nc + col);
            }
        }
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int e = e0 + q * blockDim.x;
            if (e < nstage) {
                const int col = e % nc, r = (e / nc) % kTcR, d = e / (nc * kTcR);
                Xs[((size_t)d * n2 + col) * kTcXs + r] = v[q].x;
                Xs[((size_t)d * n2 + nc + col) * kTcXs + r] = v[q].y;
            }
        }
    }
    // the stencil block of the next direction is loaded into registers while
    // the current one is multiplied (up to kTcPre entries per thread)
    const int nblk = nc * nc;
    float2 pre[kTcPre];
    auto prefetch = [&](int d) {
        const float2* Ad = A + ((size_t)s * 9 + d) * nblk;
#pragma unroll
        for (int q = 0; q < kTcPre; ++q) {
            const int e = tid + q * blockDim.x;
            pre[q] = e < nblk ? __ldg(Ad + e) : make_float2(0.f, 0.f);
        }
    };
    prefetch(0);
    float acc[2][4] = {{0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}};
    const int row0 = 16 * warp;
    for (int d = 0; d < 9; ++d) {
        __syncthreads();   // staging done / previous block no longer read
#pragma unroll
        for (int q = 0; q < kTcPre; ++q) {
            const int e = tid + q * blockDim.x;
            if (e < nblk) As[(e / nc) * astride + (e % nc)] = pre[q];
        }
        __syncthreads();
        if (d + 1 < 9) prefetch(d + 1);
        const float* Xd = Xs + (size_t)d * n2 * kTcXs;
        for (int k0 = 0; k0 < n2; k0 += 8) {
            uint32_t ab[4], as_[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int rho = row0 + g + (i & 1) * 8, kap = k0 + t + (i >> 1) * 4;
                const bool rim = rho >= nc, kim = kap >= nc;
                const float2 v = As[(kim ? kap - nc : kap) * astride + (rim ? rho - nc : rho)];
                const float val = rim == kim ? v.x : (rim ? v.y : -v.y);
                tf32_split(val, ab[i], as_[i]);
            }
#pragma unroll
            for (int nt = 0; nt < 2; ++nt) {
                uint32_t bb0, bs0, bb1, bs1;
                tf32_split(Xd[(size_t)(k0 + t) * kTcXs + 8 * nt + g], bb0, bs0);
                tf32_split(Xd[(size_t)(k0 + t + 4) * kTcXs + 8 * nt + g], bb1, bs1);
                mma_tf32(acc[nt], as_, bb0, bb1);
                mma_tf32(acc[nt], ab, bs0, bs1);
                mma_tf32(acc[nt], ab, bb0, bb1);
            }
        }
    }
    __syncthreads();   // the last block is no longer read: Ys reuses its space
#pragma unroll
    for (int nt = 0; nt < 2; ++nt)
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int rho = row0 + g + (i >> 1) * 8, col = 8 * nt + 2 * t + (i & 1);
            Ys[rho * kTcR + col] = acc[nt][i];
        }
    __syncthreads();
    for (int e = tid; e < nc * kTcR; e += blockDim.x) {
        const int row = e % nc, r = e / nc, j = j0 + r;
        if (j >= nrhs) continue;
        float2 o = make_float2(Ys[row * kTcR + r], Ys[(row + nc) * kTcR + r]);
        const float2 xv = make_float2(Xs[(size_t)row * kTcXs + r], Xs[(size_t)(nc + row) * kTcXs + r]);
        const float sg = row < nc / 2 ? 1.f : -1.f;
        const float tj = (float)tau.t[j];
        if (op == QCD_OP_D) { o -= (tj * sg) * xv; }
        else { o = sg * o; o -= tj * xv; }
        y[(size_t)j * vstride + (size_t)s * nc + row] = o;
    }
}

size_t coarse_tc_smem(int nc) {
    // the block region also holds the 2nc x kTcR results at the end
    const size_t ablk = std::max(sizeof(float2) * (size_t)nc * tc_astride(nc), sizeof(float) * (size_t)2 * nc * kTcR);
    return sizeof(float) * (size_t)9 * 2 * nc * kTcXs + ablk;
}

// ------------------------------------------------------------------ SAP block solves
// One CTA per (block of one colour, rhs), one thread per block site; GMRES
// from zero on the Dirichlet block operator (hops leaving the block dropped),
// Arnoldi by modified Gram-Schmidt, Krylov vectors in global scratch.
template <typename R>
__device__ __forceinline__ void block_op(const Geom& g, const Blocking& B, const cplx<R>* __restrict__ U,
                                         const R* __restrict__ A, int y, int l, const int o[4],
                                         const cplx<R>* vsm, int op, R t, Spinor<R>& acc) {
    Spinor<R> psi;
#pragma unroll
    for (int k = 0; k < 12; ++k) psi.c[k] = vsm[l * 12 + k];
    clover_apply<R>(A + (size_t)y * 72, psi, acc);
    int lstride = 1;
#pragma unroll
    for (int mu = 3; mu >= 0; --mu) {
        Link<R> u;
        Spinor<R> nb;
        if (o[mu] < B.b[mu] - 1) {
            const int ln = l + lstride;
#pragma unroll
            for (int k = 0; k < 12; ++k) nb.c[k] = vsm[ln * 12 + k];
            load_link<R>(U + ((size_t)y * 4 + mu) * 9, u);
            switch (mu) {
                case 0: hop_accumulate<R, 0, true>(nb, u, R(1), acc); break;
                case 1: hop_accumulate<R, 1, true>(nb, u, R(1), acc); break;
                case 2: hop_accumulate<R, 2, true>(nb, u, R(1), acc); break;
                default: hop_accumulate<R, 3, true>(nb, u, R(1), acc); break;
            }
        }
        if (o[mu] > 0) {
            const int ln = l - lstride;
#pragma unroll
            for (int k = 0; k < 12; ++k) nb.c[k] = vsm[ln * 12 + k];
            int xb[4];
            site_coords(g, y, xb);
            xb[mu] -= 1;
            load_link<R>(U + ((size_t)site_index(g, xb) * 4 + mu) * 9, u);
            switch (mu) {
                case 0: hop_accumulate<R, 0, false>(nb, u, R(1), acc); break;
                case 1: hop_accumulate<R, 1, false>(nb, u, R(1), acc); break;
                case 2: hop_accumulate<R, 2, false>(nb, u, R(1), acc); break;
                default: hop_accumulate<R, 3, false>(nb, u, R(1), acc); break;
            }
        }
        lstride *= B.b[mu];
    }
    if (op == QCD_OP_D) {
#pragma unroll
        for (int k = 0; k < 6; ++k) acc.c[k] -= t * psi.c[k];
#pragma unroll
        for (int k = 6; k < 12; ++k) acc.c[k] += t * psi.c[k];
    } else {
#pragma unroll
        for (int k = 0; k < 6; ++k) acc.c[k] -= t * psi.c[k];
#pragma unroll
        for (int k = 6; k < 12; ++k) acc.c[k] = -acc.c[k] - t * psi.c[k];
    }
}

template <typename R>
__global__ void sap_block_kernel(Geom g, Blocking B, const cplx<R>* __restrict__ U, const R* __restrict__ A,
                                 const int* __restrict__ blocks, int op, Shifts tau, const cplx<R>* __restrict__ r,
                                 cplx<R>* __restrict__ x, int iters, double tol, cplx<R>* __restrict__ scratch,
                                 const int* __restrict__ act) {
    extern __shared__ double2 sm[];
    const int bs = B.bs;
    cplx<R>* vsm = reinterpret_cast<cplx<R>*>(sm);                       // [bs][12]
    double2* red = reinterpret_cast<double2*>(vsm + (size_t)bs * 12);    // [bs]
    double2* H = red + bs;                              // [(iters+1) * iters]
    double2* gv = H + (iters + 1) * iters;              // [iters + 1]
    double2* sn = gv + iters + 1;                       // [iters]
    double2* yv = sn + iters;                           // [iters]
    double* cs = reinterpret_cast<double*>(yv + iters); // [iters]
    int* flag = reinterpret_cast<int*>(cs + iters);     // [4]

    const int j = blockIdx.y;
    if (act != nullptr && !act[j]) return;
    const int blk = blocks[blockIdx.x];
    const int l = threadIdx.x;
    const size_t fstride = (size_t)g.V * 12;
    r += j * fstride;
    x += j * fstride;
    cplx<R>* kv = scratch + ((size_t)j * gridDim.x + blockIdx.x) * (size_t)(iters + 1) * bs * 12;
    const R t = (R)tau.t[j];

    int o[4];
    local_coords(B, l, o);
    const int y = block_fine_site(g, B, blk, l);

    Spinor<R> w;
    load_spinor<R>(r + (size_t)y * 12, w);
    double2 nn = make_double2(0, 0);
#pragma unroll
    for (int k = 0; k < 12; ++k) nn.x += (double)w.c[k].x * w.c[k].x + (double)w.c[k].y * w.c[k].y;
    nn = block_sum2(nn, red);
    const double beta = sqrt(nn.x);
    if (!(beta > 0.0)) return;
    {
        const R ib = (R)(1.0 / beta);
#pragma unroll
        for (int k = 0; k < 12; ++k) { w.c[k] = ib * w.c[k]; kv[(size_t)l * 12 + k] = w.c[k]; vsm[l * 12 + k] = w.c[k]; }
    }
    if (l == 0) { gv[0] = make_double2(beta, 0); flag[0] = 0; }
    int kdim = 0;
    for (int jj = 0; jj < iters; ++jj) {
        __syncthreads();
        block_op<R>(g, B, U, A, y, l, o, vsm, op, t, w);
        for (int i = 0; i <= jj; ++i) {
            const cplx<R>* vi = kv + (size_t)i * bs * 12 + (size_t)l * 12;
            double2 h = make_double2(0, 0);
#pragma unroll
            for (int k = 0; k < 12; ++k) {
                cplx<R> a = vi[k];
                h.x += (double)a.x * w.c[k].x + (double)a.y * w.c[k].y;
                h.y += (double)a.x * w.c[k].y - (double)a.y * w.c[k].x;
            }
            h = block_sum2(h, red);
            const cplx<R> hr = mk<R>((R)h.x, (R)h.y);
#pragma unroll
            for (int k = 0; k < 12; ++k) w.c[k] -= hr * vi[k];
            if (l == 0) H[i * iters + jj] = h;
        }
        double2 hn2 = make_double2(0, 0);
#pragma unroll
        for (int k = 0; k < 12; ++k) hn2.x += (double)w.c[k].x * w.c[k].x + (double)w.c[k].y * w.c[k].y;
        hn2 = block_sum2(hn2, red);
        const double hn = sqrt(hn2.x);
        {
            const R ih = hn > 0 ? (R)(1.0 / hn) : R(0);
#pragma unroll
            for (int k = 0; k < 12; ++k) {
                w.c[k] = ih * w.c[k];
                kv[(size_t)(jj + 1) * bs * 12 + (size_t)l * 12 + k] = w.c[k];
                vsm[l * 12 + k] = w.c[k];
            }
        }
        if (l == 0) {
            H[(jj + 1) * iters + jj] = make_double2(hn, 0);
            for (int i = 0; i < jj; ++i) {
                double2 a = H[i * iters + jj], c = H[(i + 1) * iters + jj];
                H[i * iters + jj] = cs[i] * a + sn[i] * c;
                H[(i + 1) * iters + jj] = cs[i] * c - conj(sn[i]) * a;
            }
            double2 a = H[jj * iters + jj];
            double2 c = H[(jj + 1) * iters + jj];
            double aa = sqrt(a.x * a.x + a.y * a.y), rr = sqrt(aa * aa + c.x * c.x + c.y * c.y);
            if (aa > 0) {
                cs[jj] = aa / rr;
                sn[jj] = (1.0 / aa) * a * conj(c);
                sn[jj] = (1.0 / rr) * sn[jj];
            } else {
                cs[jj] = 0.0;
                sn[jj] = make_double2(1, 0);
            }
            H[jj * iters + jj] = cs[jj] * a + sn[jj] * c;
            gv[jj + 1] = -1.0 * (conj(sn[jj]) * gv[jj]);
            gv[jj] = cs[jj] * gv[jj];
            const double res = sqrt(gv[jj + 1].x * gv[jj + 1].x + gv[jj + 1].y * gv[jj + 1].y);
            flag[0] = (tol >= 0.0 && res <= tol * beta) ? 1 : 0;
        }
        __syncthreads();
        kdim = jj + 1;
        if (flag[0]) break;
    }
    if (l == 0) {
        count_sap_work(bs, kdim);
        for (int i = kdim - 1; i >= 0; --i) {
            double2 s = gv[i];
            for (int k = i + 1; k < kdim; ++k) s -= H[i * iters + k] * yv[k];
            double2 dd = H[i * iters + i];
            double den = dd.x * dd.x + dd.y * dd.y;
            yv[i] = den > 0 ? (1.0 / den) * cmulc(dd, s) : make_double2(0, 0);
        }
    }
    __syncthreads();
    Spinor<R> e;
    load_spinor<R>(x + (size_t)y * 12, e);
    for (int i = 0; i < kdim; ++i) {
        const cplx<R> yi = mk<R>((R)yv[i].x, (R)yv[i].y);
        const cplx<R>* vi = kv + (size_t)i * bs * 12 + (size_t)l * 12;
#pragma unroll
        for (int k = 0; k < 12; ++k) e.c[k] += yi * vi[k];
    }
    store_spinor<R>(x + (size_t)y * 12, e);
}

// ------------------------------------------------------------------ SAP, small blocks
// Blocks of BS <= 32 sites: each SAP block is a BS-lane segment of one warp
// (32 / BS blocks per CTA of one warp).  The block's links and clover and the
// whole Krylov basis live in shared memory; inner products are reduced with
// xor-shuffles inside the segment; Arnoldi by modified Gram-Schmidt, as in the
// 256-site path.  Only __syncwarp() orders shared-memory traffic.
struct SapSmemLayout {
    size_t basis, links, clover, H, g, sn, y, cs, flag, total;
};
template <typename R>
__host__ __device__ inline SapSmemLayout sap_layout(int BS, int iters, size_t basis_elem = sizeof(cplx<R>)) {
    auto up = [](size_t v) { return (v + 15) & ~size_t(15); };
    SapSmemLayout L;
    size_t o = 0;
    L.basis = o;  o = up(o + (size_t)(iters + 1) * BS * 12 * basis_elem);
    L.links = o;  o = up(o + (size_t)BS * 36 * sizeof(cplx<R>));
    L.clover = o; o = up(o + (size_t)BS * 72 * sizeof(R));
    L.H = o;      o = up(o + (size_t)(iters + 1) * iters * sizeof(cplx<R>));
    L.g = o;      o = up(o + (size_t)(iters + 1) * sizeof(cplx<R>));
    L.sn = o;     o = up(o + (size_t)iters * sizeof(cplx<R>));
    L.y = o;      o = up(o + (size_t)iters * sizeof(cplx<R>));
    L.cs = o;     o = up(o + (size_t)iters * sizeof(R));
    L.flag = o;   o = up(o + 4 * sizeof(int));
    L.total = o;
    return L;
}

// Shared memory of the chirality-split kernel with rw right-hand sides per
// CTA: the block's links and clover once, then per warp its Krylov basis and
// GMRES scalars.
struct ChiLayout {
    size_t links, clover, shared, basis, H, g, sn, y, cs, flag, perwarp, total;
};
template <typename R>
__host__ __device__ inline ChiLayout chi_layout(int iters, size_t basis_elem, int rw) {
    auto up = [](size_t v) { return (v + 15) & ~size_t(15); };
    ChiLayout L;
    size_t o = 0;
    L.links = o;  o = up(o + (size_t)16 * 36 * sizeof(cplx<R>));
    L.clover = o; o = up(o + (size_t)16 * 72 * sizeof(R));
    L.shared = o;
    size_t w = 0;
    L.basis = w;  w = up(w + (size_t)(iters + 1) * 16 * 12 * basis_elem);
    L.H = w;      w = up(w + (size_t)(iters + 1) * iters * sizeof(cplx<R>));
    L.g = w;      w = up(w + (size_t)(iters + 1) * sizeof(cplx<R>));
    L.sn = w;     w = up(w + (size_t)iters * sizeof(cplx<R>));
    L.y = w;      w = up(w + (size_t)iters * sizeof(cplx<R>));
    L.cs = w;     w = up(w + (size_t)iters * sizeof(R));
    L.flag = w;   w = up(w + 4 * sizeof(int));
    L.perwarp = w;
    L.total = L.shared + (size_t)rw * w;
    return L;
}

template <int BS, typename T>
__device__ __forceinline__ T seg_sum(T v) {
#pragma unroll
    for (int o = BS / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

template <typename R, int BS>
__global__ void __launch_bounds__(32) sap_warp_kernel(Geom g, Blocking B, const cplx<R>* __restrict__ U,
                                                      const R* __restrict__ A, const int* __restrict__ blocks, int ncol,
                                                      int op, Shifts tau, const cplx<R>* __restrict__ r,
                                                      cplx<R>* __restrict__ x, int iters, double tol,
                                                      const int* __restrict__ act) {
    constexpr int SPW = 32 / BS;
    extern __shared__ __align__(16) unsigned char smraw[];
    const int lane = threadIdx.x;
    const int seg = lane / BS, l = lane % BS;
    const SapSmemLayout LY = sap_layout<R>(BS, iters);
    unsigned char* base = smraw + (size_t)seg * LY.total;
    cplx<R>* basis = reinterpret_cast<cplx<R>*>(base + LY.basis);
    cplx<R>* slink = reinterpret_cast<cplx<R>*>(base + LY.links);
    R* sclov = reinterpret_cast<R*>(base + LY.clover);
    // Hessenberg bookkeeping by lane 0 in the working precision (a dependent
    // FP64 chain is very slow on this part)
    cplx<R>* H = reinterpret_cast<cplx<R>*>(base + LY.H);
    cplx<R>* gv = reinterpret_cast<cplx<R>*>(base + LY.g);
    cplx<R>* sn = reinterpret_cast<cplx<R>*>(base + LY.sn);
    cplx<R>* yv = reinterpret_cast<cplx<R>*>(base + LY.y);
    R* cs = reinterpret_cast<R*>(base + LY.cs);
    int* flag = reinterpret_cast<int*>(base + LY.flag);

    const int j = blockIdx.y;
    if (act != nullptr && !act[j]) return;
    const int bidx = blockIdx.x * SPW + seg;
    const bool valid = bidx < ncol;
    const int blk = valid ? blocks[bidx] : blocks[0];
    const size_t fstride = (size_t)g.V * 12;
    r += j * fstride;
    x += j * fstride;
    const R t = (R)tau.t[j];
    int o[4];
    {
        int tt = l;
        o[3] = tt % B.b[3]; tt /= B.b[3];
        o[2] = tt % B.b[2]; tt /= B.b[2];
        o[1] = tt % B.b[1]; o[0] = tt / B.b[1];
    }
    const int y = block_fine_site(g, B, blk, l);
    // stage links (forward, this site) and clover
#pragma unroll
    for (int k = 0; k < 36; ++k) slink[l * 36 + k] = __ldg(U + (size_t)y * 36 + k);
#pragma unroll 8
    for (int k = 0; k < 72; ++k) sclov[l * 72 + k] = __ldg(A + (size_t)y * 72 + k);
    Spinor<R> w;
    load_spinor<R>(r + (size_t)y * 12, w);
    R nn = 0;
#pragma unroll
    for (int k = 0; k < 12; ++k) nn += w.c[k].x * w.c[k].x + w.c[k].y * w.c[k].y;
    nn = seg_sum<BS>(nn);
    const R beta = valid ? sqrt(nn) : R(0);
    {
        const R ib = beta > R(0) ? R(1) / beta : R(0);
#pragma unroll
        for (int k = 0; k < 12; ++k) basis[l * 12 + k] = ib * w.c[k];
    }
    if (l == 0) { gv[0] = mk<R>(beta, R(0)); flag[0] = beta > R(0) ? 0 : 1; flag[1] = 0; }
    __syncwarp();
    int lstride[4];
    lstride[3] = 1;
    lstride[2] = B.b[3];
    lstride[1] = B.b[3] * B.b[2];
    lstride[0] = B.b[3] * B.b[2] * B.b[1];
    for (int jj = 0; jj < iters; ++jj) {
        const bool active = flag[0] == 0;
        if (__all_sync(0xffffffffu, !active)) break;
        const cplx<R>* vj = basis + (size_t)jj * BS * 12;
        // w = A_block v_j
        Spinor<R> psi, acc;
#pragma unroll
        for (int k = 0; k < 12; ++k) psi.c[k] = vj[l * 12 + k];
        clover_apply_smem<R>(sclov + l * 72, psi, acc);
        // Dirichlet block: per mu one neighbour inside the block on the
        // forward side if there is one, else on the backward side (a 2-site
        // extent has exactly one), taken by all lanes together; interior
        // sites of wider blocks add their backward neighbour afterwards
#pragma unroll
        for (int mu = 0; mu < 4; ++mu) {
            Spinor<R> nb;
            Link<R> u;
            const bool fw = o[mu] < B.b[mu] - 1;
            if (fw || o[mu] > 0) {
                const int ln = fw ? l + lstride[mu] : l - lstride[mu];
#pragma unroll
                for (int k = 0; k < 12; ++k) nb.c[k] = vj[ln * 12 + k];
                const cplx<R>* lk = slink + (fw ? l : ln) * 36 + mu * 9;
#pragma unroll
                for (int k = 0; k < 9; ++k) u.e[k] = lk[k];
                switch (mu) {
                    case 0: hop_accumulate_dir<R, 0>(nb, u, R(1), fw, acc); break;
                    case 1: hop_accumulate_dir<R, 1>(nb, u, R(1), fw, acc); break;
                    case 2: hop_accumulate_dir<R, 2>(nb, u, R(1), fw, acc); break;
                    default: hop_accumulate_dir<R, 3>(nb, u, R(1), fw, acc); break;
                }
            }
            const bool both = fw && o[mu] > 0;
            if (__any_sync(0xffffffffu, both) && both) {
                const int ln = l - lstride[mu];
#pragma unroll
                for (int k = 0; k < 12; ++k) nb.c[k] = vj[ln * 12 + k];
#pragma unroll
                for (int k = 0; k < 9; ++k) u.e[k] = slink[ln * 36 + mu * 9 + k];
                switch (mu) {
                    case 0: hop_accumulate<R, 0, false>(nb, u, R(1), acc); break;
                    case 1: hop_accumulate<R, 1, false>(nb, u, R(1), acc); break;
                    case 2: hop_accumulate<R, 2, false>(nb, u, R(1), acc); break;
                    default: hop_accumulate<R, 3, false>(nb, u, R(1), acc); break;
                }
            }
        }
        if (op == QCD_OP_D) {
#pragma unroll
            for (int k = 0; k < 6; ++k) acc.c[k] -= t * psi.c[k];
#pragma unroll
            for (int k = 6; k < 12; ++k) acc.c[k] += t * psi.c[k];
        } else {
#pragma unroll
            for (int k = 0; k < 6; ++k) acc.c[k] -= t * psi.c[k];
#pragma unroll
            for (int k = 6; k < 12; ++k) acc.c[k] = -acc.c[k] - t * psi.c[k];
        }
        // modified Gram-Schmidt against v_0 .. v_jj
        for (int i = 0; i <= jj; ++i) {
            const cplx<R>* vi = basis + (size_t)i * BS * 12 + l * 12;
            R hr = 0, hi = 0;
#pragma unroll
            for (int k = 0; k < 12; ++k) {
                cplx<R> a = vi[k];
                hr += a.x * acc.c[k].x + a.y * acc.c[k].y;
                hi += a.x * acc.c[k].y - a.y * acc.c[k].x;
            }
            hr = seg_sum<BS>(hr);
            hi = seg_sum<BS>(hi);
            const cplx<R> h = mk<R>(hr, hi);
#pragma unroll
            for (int k = 0; k < 12; ++k) acc.c[k] -= h * vi[k];
            if (l == 0 && active) H[i * iters + jj] = mk<R>(hr, hi);
        }
        R hn2 = 0;
#pragma unroll
        for (int k = 0; k < 12; ++k) hn2 += acc.c[k].x * acc.c[k].x + acc.c[k].y * acc.c[k].y;
        hn2 = seg_sum<BS>(hn2);
        const R hn = sqrt(hn2);
        {
            const R ih = hn > R(0) ? R(1) / hn : R(0);
            cplx<R>* vn = basis + (size_t)(jj + 1) * BS * 12 + l * 12;
#pragma unroll
            for (int k = 0; k < 12; ++k) vn[k] = ih * acc.c[k];
        }
        if (l == 0 && active) {
            H[(jj + 1) * iters + jj] = mk<R>(hn, R(0));
            for (int i = 0; i < jj; ++i) {
                cplx<R> a = H[i * iters + jj], c = H[(i + 1) * iters + jj];
                H[i * iters + jj] = cs[i] * a + sn[i] * c;
                H[(i + 1) * iters + jj] = cs[i] * c - conj(sn[i]) * a;
            }
            cplx<R> a = H[jj * iters + jj];
            cplx<R> c = H[(jj + 1) * iters + jj];
            R aa = sqrt(a.x * a.x + a.y * a.y), rr = sqrt(aa * aa + c.x * c.x + c.y * c.y);
            if (aa > R(0)) {
                cs[jj] = aa / rr;
                sn[jj] = (R(1) / rr) * ((R(1) / aa) * a * conj(c));
            } else {
                cs[jj] = R(0);
                sn[jj] = mk<R>(R(1), R(0));
            }
            H[jj * iters + jj] = cs[jj] * a + sn[jj] * c;
            gv[jj + 1] = R(-1) * (conj(sn[jj]) * gv[jj]);
            gv[jj] = cs[jj] * gv[jj];
            const R res = sqrt(gv[jj + 1].x * gv[jj + 1].x + gv[jj + 1].y * gv[jj + 1].y);
            flag[1] = jj + 1;
            if (tol >= 0.0 && (double)res <= tol * (double)beta) flag[0] = 1;
        }
        __syncwarp();
    }
    const int kdim = flag[1];
    if (l == 0) {
        if (valid) count_sap_work(BS, kdim);
        for (int i = kdim - 1; i >= 0; --i) {
            cplx<R> sacc = gv[i];
            for (int k = i + 1; k < kdim; ++k) sacc -= H[i * iters + k] * yv[k];
            cplx<R> dd = H[i * iters + i];
            R den = dd.x * dd.x + dd.y * dd.y;
            yv[i] = den > R(0) ? (R(1) / den) * cmulc(dd, sacc) : mk<R>(R(0), R(0));
        }
    }
    __syncwarp();
    if (!valid || kdim == 0) return;
    Spinor<R> e;
    load_spinor<R>(x + (size_t)y * 12, e);
    for (int i = 0; i < kdim; ++i) {
        const cplx<R> yi = yv[i];
        const cplx<R>* vi = basis + (size_t)i * BS * 12 + l * 12;
#pragma unroll
        for (int k = 0; k < 12; ++k) e.c[k] += yi * vi[k];
    }
    store_spinor<R>(x + (size_t)y * 12, e);
}

// Storage of the SAP block Krylov basis: the working precision, or FP16
// pairs for FP32 solves (the basis then takes half the shared memory, so more
// block solves are resident per SM; the block solves only need a 1e-1
// reduction).
__device__ __forceinline__ float2 bload(const float2* p) { return *p; }
__device__ __forceinline__ double2 bload(const double2* p) { return *p; }
__device__ __forceinline__ float2 bload(const __half2* p) { return __half22float2(*p); }
__device__ __forceinline__ void bstore(float2* p, float2 v) { *p = v; }
__device__ __forceinline__ void bstore(double2* p, double2 v) { *p = v; }
__device__ __forceinline__ void bstore(__half2* p, float2 v) { *p = __float22half2_rn(v); }

// Copy N 16-byte words from global to shared memory with all N loads in
// flight before the first store (staging without a round trip per word).
template <int N>
__device__ __forceinline__ void stage16(void* __restrict__ dst, const void* __restrict__ src) {
    const int4* s4 = reinterpret_cast<const int4*>(src);
    int4* d4 = reinterpret_cast<int4*>(dst);
    int4 v[N];
#pragma unroll
    for (int q = 0; q < N; ++q) v[q] = __ldg(s4 + q);
#pragma unroll
    for (int q = 0; q < N; ++q) d4[q] = v[q];
}

// SAP block solve for 16-site blocks with two lanes per site: lane
// chi * 16 + l holds chirality half chi (spins 2chi, 2chi+1) of site l, so one
// warp solves one block.  The clover term is block diagonal in chirality; in a
// hop each lane forms the projected half-spinor h_s for s = chi, multiplies it
// by the link (9 complex products instead of 18) and takes the other s from
// the partner lane (lane ^ 16) before it reconstructs its own half.  Same
// GMRES as sap_warp_kernel (modified Gram-Schmidt, Givens by lane 0).
template <typename R, typename BT>
__global__ void __launch_bounds__(128) sap_chi_kernel(Geom g, Blocking B, const cplx<R>* __restrict__ U,
                                                      const R* __restrict__ A, const int* __restrict__ blocks,
                                                      int ncol, int op, Shifts tau, const cplx<R>* __restrict__ r,
                                                      cplx<R>* __restrict__ x, int iters, double tol,
                                                      const int* __restrict__ act, int nrhs) {
    constexpr int BS = 16;
    extern __shared__ __align__(16) unsigned char smraw[];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, rw = blockDim.x >> 5;
    const int chi = lane >> 4, l = lane & 15;
    const ChiLayout LY = chi_layout<R>(iters, sizeof(BT), rw);
    unsigned char* wbase = smraw + LY.shared + (size_t)wid * LY.perwarp;
    BT* basis = reinterpret_cast<BT*>(wbase + LY.basis);
    cplx<R>* slink = reinterpret_cast<cplx<R>*>(smraw + LY.links);
    R* sclov = reinterpret_cast<R*>(smraw + LY.clover);
    cplx<R>* H = reinterpret_cast<cplx<R>*>(wbase + LY.H);
    cplx<R>* gv = reinterpret_cast<cplx<R>*>(wbase + LY.g);
    cplx<R>* sn = reinterpret_cast<cplx<R>*>(wbase + LY.sn);
    cplx<R>* yv = reinterpret_cast<cplx<R>*>(wbase + LY.y);
    R* cs = reinterpret_cast<R*>(wbase + LY.cs);
    int* flag = reinterpret_cast<int*>(wbase + LY.flag);

    // warp w of the CTA solves the block for right-hand side blockIdx.y * rw + w;
    // the block's links and clover are staged once for all of them
    const int j = blockIdx.y * rw + wid;
    const int blk = blocks[blockIdx.x];
    int o[4];
    {
        int tt = l;
        o[3] = tt % B.b[3]; tt /= B.b[3];
        o[2] = tt % B.b[2]; tt /= B.b[2];
        o[1] = tt % B.b[1]; o[0] = tt / B.b[1];
    }
    const int y = block_fine_site(g, B, blk, l);
    // stage links and clover of the 16 sites (warp 0): lane chi copies half
    // of its site's links and its own chirality block of the clover term
    // (16-byte words, every load in flight at once)
    constexpr int kHalf = 18 * (int)sizeof(cplx<R>) / 16;   // 16-byte words in 18 complex / 36 reals
    if (wid == 0) {
        stage16<kHalf>(slink + l * 36 + 18 * chi, U + (size_t)y * 36 + 18 * chi);
        stage16<kHalf>(sclov + l * 72 + 36 * chi, A + (size_t)y * 72 + 36 * chi);
    }
    const bool mine = j < nrhs && (act == nullptr || act[j]);
    const size_t fstride = (size_t)g.V * 12;
    cplx<R> w[6];
    if (mine) {
        r += j * fstride;
        x += j * fstride;
#pragma unroll
        for (int k = 0; k < 6; ++k) w[k] = __ldg(r + (size_t)y * 12 + 6 * chi + k);
    }
    __syncthreads();
    if (!mine) return;
    const R t = (R)tau.t[j];
    R nn = 0;
#pragma unroll
    for (int k = 0; k < 6; ++k) nn += w[k].x * w[k].x + w[k].y * w[k].y;
    nn = warp_sum(nn);
    const R beta = sqrt(nn);
    {
        const R ib = beta > R(0) ? R(1) / beta : R(0);
#pragma unroll
        for (int k = 0; k < 6; ++k) bstore(basis + l * 12 + 6 * chi + k, ib * w[k]);
    }
    if (lane == 0) { gv[0] = mk<R>(beta, R(0)); flag[0] = beta > R(0) ? 0 : 1; flag[1] = 0; }
    __syncwarp();
    int lstride[4];
    lstride[3] = 1;
    lstride[2] = B.b[3];
    lstride[1] = B.b[3] * B.b[2];
    lstride[0] = B.b[3] * B.b[2] * B.b[1];
    for (int jj = 0; jj < iters; ++jj) {
        const bool active = flag[0] == 0;
        if (!active) break;   // flag is shared by the whole warp
        const BT* vj = basis + (size_t)jj * BS * 12;
        cplx<R> psi[6], acc[6];
#pragma unroll
        for (int k = 0; k < 6; ++k) psi[k] = bload(vj + l * 12 + 6 * chi + k);
        // clover block chi of site l
        {
            const R* a = sclov + l * 72 + 36 * chi;
#pragma unroll
            for (int i = 0; i < 6; ++i) acc[i] = a[i] * psi[i];
#pragma unroll
            for (int i = 0; i < 6; ++i) {
#pragma unroll
                for (int jc = i + 1; jc < 6; ++jc) {
                    const int oo = herm_off(i, jc);
                    const cplx<R> aij = mk<R>(a[oo], a[oo + 1]);
                    acc[i] += aij * psi[jc];
                    acc[jc] += cmulc(aij, psi[i]);
                }
            }
        }
        // hops inside the block (Dirichlet): per mu the forward neighbour if it
        // is inside, else the backward one; interior sites of wider blocks
        // add their backward neighbour in a second round
#pragma unroll
        for (int mu = 0; mu < 4; ++mu) {
            const SpinMono Bm = kB(mu), BHm = kBH(mu);
            for (int round = 0; round < 2; ++round) {
                const bool fw = round == 0 ? (o[mu] < B.b[mu] - 1) : false;
                const bool has = round == 0 ? (fw || o[mu] > 0) : (o[mu] < B.b[mu] - 1 && o[mu] > 0);
                if (round == 1 && !__any_sync(0xffffffffu, has)) break;
                const int ln = has ? (fw ? l + lstride[mu] : l - lstride[mu]) : l;
                const BT* nb = vj + ln * 12;
                const R pm = fw ? R(-1) : R(1);
                // h_s for s = chi: up_s + pm i^{ph_s} dn_{perm_s}
                const int sp = Bm.perm[chi], ph = Bm.ph[chi];
                cplx<R> h[3];
#pragma unroll
                for (int a = 0; a < 3; ++a) h[a] = bload(nb + chi * 3 + a) + pm * mul_ipow(bload(nb + (2 + sp) * 3 + a), ph);
                const cplx<R>* lk = slink + (fw ? l : ln) * 36 + mu * 9;
                cplx<R> os[3];
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    cplx<R> v = czero<R>();
#pragma unroll
                    for (int b = 0; b < 3; ++b) v += (fw ? lk[a * 3 + b] : conj(lk[b * 3 + a])) * h[b];
                    os[a] = has ? v : czero<R>();
                }
                cplx<R> ot[3];
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    ot[a].x = __shfl_xor_sync(0xffffffffu, os[a].x, 16);
                    ot[a].y = __shfl_xor_sync(0xffffffffu, os[a].y, 16);
                }
                // o[0], o[1] of the site; reconstruct this lane's half
                const R half = R(-0.5);
#pragma unroll
                for (int s2 = 0; s2 < 2; ++s2) {
                    const int src = chi ? BHm.perm[s2] : s2;
                    const int php = chi ? BHm.ph[s2] : 0;
                    const R c = chi ? pm * half : half;
                    const bool mine = src == chi;
#pragma unroll
                    for (int a = 0; a < 3; ++a) acc[s2 * 3 + a] += c * mul_ipow(mine ? os[a] : ot[a], php);
                }
            }
        }
        // shift: D - tau Gamma5 (op D) or Gamma5 D - tau (op Q)
        {
            const R g5 = chi ? R(-1) : R(1);
#pragma unroll
            for (int k = 0; k < 6; ++k) {
                if (op == QCD_OP_D) acc[k] -= (t * g5) * psi[k];
                else acc[k] = g5 * acc[k] - t * psi[k];
            }
        }
        // modified Gram-Schmidt against v_0 .. v_jj
        for (int i = 0; i <= jj; ++i) {
            const BT* vi = basis + (size_t)i * BS * 12 + l * 12 + 6 * chi;
            R hr = 0, hi = 0;
#pragma unroll
            for (int k = 0; k < 6; ++k) {
                const cplx<R> a = bload(vi + k);
                hr += a.x * acc[k].x + a.y * acc[k].y;
                hi += a.x * acc[k].y - a.y * acc[k].x;
            }
            hr = warp_sum(hr);
            hi = warp_sum(hi);
            const cplx<R> h = mk<R>(hr, hi);
#pragma unroll
            for (int k = 0; k < 6; ++k) acc[k] -= h * bload(vi + k);
            if (lane == 0) H[i * iters + jj] = h;
        }
        R hn2 = 0;
#pragma unroll
        for (int k = 0; k < 6; ++k) hn2 += acc[k].x * acc[k].x + acc[k].y * acc[k].y;
        hn2 = warp_sum(hn2);
        const R hn = sqrt(hn2);
        {
            const R ih = hn > R(0) ? R(1) / hn : R(0);
            BT* vn = basis + (size_t)(jj + 1) * BS * 12 + l * 12 + 6 * chi;
#pragma unroll
            for (int k = 0; k < 6; ++k) bstore(vn + k, ih * acc[k]);
        }
        if (lane == 0) {
            H[(jj + 1) * iters + jj] = mk<R>(hn, R(0));
            for (int i = 0; i < jj; ++i) {
                cplx<R> a = H[i * iters + jj], c = H[(i + 1) * iters + jj];
                H[i * iters + jj] = cs[i] * a + sn[i] * c;
                H[(i + 1) * iters + jj] = cs[i] * c - conj(sn[i]) * a;
            }
            cplx<R> a = H[jj * iters + jj];
            cplx<R> c = H[(jj + 1) * iters + jj];
            R aa = sqrt(a.x * a.x + a.y * a.y), rr = sqrt(aa * aa + c.x * c.x + c.y * c.y);
            if (aa > R(0)) {
                cs[jj] = aa / rr;
                sn[jj] = (R(1) / rr) * ((R(1) / aa) * a * conj(c));
            } else {
                cs[jj] = R(0);
                sn[jj] = mk<R>(R(1), R(0));
            }
            H[jj * iters + jj] = cs[jj] * a + sn[jj] * c;
            gv[jj + 1] = R(-1) * (conj(sn[jj]) * gv[jj]);
            gv[jj] = cs[jj] * gv[jj];
            const R res = sqrt(gv[jj + 1].x * gv[jj + 1].x + gv[jj + 1].y * gv[jj + 1].y);
            flag[1] = jj + 1;
            if (tol >= 0.0 && (double)res <= tol * (double)beta) flag[0] = 1;
        }
        __syncwarp();
    }
    const int kdim = flag[1];
    if (lane == 0) {
        count_sap_work(BS, kdim);
        for (int i = kdim - 1; i >= 0; --i) {
            cplx<R> sacc = gv[i];
            for (int k = i + 1; k < kdim; ++k) sacc -= H[i * iters + k] * yv[k];
            cplx<R> dd = H[i * iters + i];
            R den = dd.x * dd.x + dd.y * dd.y;
            yv[i] = den > R(0) ? (R(1) / den) * cmulc(dd, sacc) : mk<R>(R(0), R(0));
        }
    }
    __syncwarp();
    if (kdim == 0) return;
    cplx<R> e[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) e[k] = x[(size_t)y * 12 + 6 * chi + k];
    for (int i = 0; i < kdim; ++i) {
        const cplx<R> yi = yv[i];
        const BT* vi = basis + (size_t)i * BS * 12 + l * 12 + 6 * chi;
#pragma unroll
        for (int k = 0; k < 6; ++k) e[k] += yi * bload(vi + k);
    }
#pragma unroll
    for (int k = 0; k < 6; ++k) x[(size_t)y * 12 + 6 * chi + k] = e[k];
}

inline int grid_for(size_t n, int th = 256) {
    size_t gsz = (n + th - 1) / th;
    return (int)(gsz > 1048576 ? 1048576 : (gsz == 0 ? 1 : gsz));
}

}  // namespace

// ------------------------------------------------------------------ host launchers
void mg_build_P(const FineOp& f, Coarse& c, const double2* vecs, int nvec, cudaStream_t st) {
    dim3 grid(c.B.nb, 2);
    KTimer kt("build_P", 0.0, 0.0, st);
    build_P_kernel<<<grid, 256, 256 * sizeof(double2), st>>>(f.g, c.B, nvec, vecs, c.P64, c.P32);
}

void mg_build_coarse(const FineOp& f, Coarse& c, cudaStream_t st, bool fp32_only) {
    dim3 grid(c.B.nb, 9);
    // columns per pass: h of a pass within about 96 KB of shared memory
    const size_t es = fp32_only ? sizeof(float2) : sizeof(double2);
    const size_t per_col = (size_t)c.B.bs * 12 * es;
    const int chunk = (int)std::max<size_t>(1, std::min<size_t>(c.nc, (96u << 10) / per_col));
    const size_t sm = chunk * per_col + (size_t)c.B.bs * sizeof(int);
    if (fp32_only) {
        // the FP32 operator straight from P32, U32 and the FP32 clover; the
        // FP64 one is rebuilt on demand (Coarse::a64_stale)
        if (sm + 1024 > 48 * 1024)
            cudaFuncSetAttribute(build_coarse_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        KTimer kt("build_coarse_f32", 0.0, 0.0, st);
        build_coarse_kernel<float><<<grid, 256, sm, st>>>(f.g, c.B, c.nv, f.U32, f.A32, c.P32, c.A32, chunk);
        c.a64_stale = true;
        return;
    }
    if (sm + 1024 > 48 * 1024)
        cudaFuncSetAttribute(build_coarse_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    KTimer kt("build_coarse", 0.0, 0.0, st);
    build_coarse_kernel<double><<<grid, 256, sm, st>>>(f.g, c.B, c.nv, f.U64, f.A64, c.P64, c.A64, chunk);
    size_t n = (size_t)c.B.nb * 9 * c.nc * c.nc;
    KTimer kt2("narrow", (double)n * 24, 0.0, st);
    narrow_kernel<<<grid_for(n), 256, 0, st>>>(c.A64, c.A32, n);
    c.a64_stale = false;
}

void mg_restrict(const FineOp& f, const Coarse& c, int prec, int nrhs, const void* r, void* xc, cudaStream_t st,
                 const int* act) {
    size_t warps = (size_t)c.B.nb * c.nc;
    int grid = grid_for(warps * 32);
    const double es = prec == QCD_FP64 ? 16.0 : 8.0;
    const double nfine = (double)f.g.V * 12;
    const double chunks = (nrhs + (prec == QCD_FP64 ? 3 : 7)) / (prec == QCD_FP64 ? 4 : 8);
    KTimer kt(prec == QCD_FP64 ? "restrict_f64" : "restrict_f32",
              es * (nfine * c.nv * chunks + nrhs * (nfine + (double)c.gc.V * c.nc)), 8.0 * nfine * c.nv * nrhs, st);
    // aggregate kernel while one chunk of the gathered fine vectors fits
    // in shared memory (8 FP32 / 4 FP64 right-hand sides per chunk)
    const int nloc = c.B.bs * 6;
    const size_t sm = (size_t)nloc * 8 * sizeof(float2);
    if (sm <= 160 * 1024) {
        const int rcs = prec == QCD_FP64 ? 4 : 8;
        const dim3 ag(c.B.nb * 2, (nrhs + rcs - 1) / rcs);
        if (prec == QCD_FP64) {
            if (sm + 1024 > 48 * 1024)
                cudaFuncSetAttribute(restrict_agg_kernel<double2, double, 4>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
            restrict_agg_kernel<double2, double, 4><<<ag, 256, sm, st>>>(f.g, c.B, c.nv, c.P64, (const double2*)r,
                                                                        (double2*)xc, nrhs, act);
        } else {
            if (sm + 1024 > 48 * 1024)
                cudaFuncSetAttribute(restrict_agg_kernel<float2, float, 8>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
            restrict_agg_kernel<float2, float, 8><<<ag, 256, sm, st>>>(f.g, c.B, c.nv, c.P32, (const float2*)r,
                                                                      (float2*)xc, nrhs, act);
        }
        return;
    }
    if (prec == QCD_FP64)
        restrict_kernel<double2, double><<<grid, 256, 0, st>>>(f.g, c.B, c.nv, c.P64, (const double2*)r, (double2*)xc, nrhs, act);
    else
        restrict_kernel<float2, float><<<grid, 256, 0, st>>>(f.g, c.B, c.nv, c.P32, (const float2*)r, (float2*)xc, nrhs, act);
}

void mg_prolong(const FineOp& f, const Coarse& c, int prec, int nrhs, const void* xc, void* x, bool accumulate,
                cudaStream_t st, const int* act) {
    size_t n = (size_t)c.B.nb * 2 * c.B.bs * 6;
    const double es = prec == QCD_FP64 ? 16.0 : 8.0;
    const double nfine = (double)f.g.V * 12;
    const double chunks = (nrhs + kProlongRC - 1) / kProlongRC;
    KTimer kt(prec == QCD_FP64 ? "prolong_f64" : "prolong_f32",
              es * (nfine * c.nv * chunks + nrhs * (nfine * (accumulate ? 2 : 1) + (double)c.gc.V * c.nc)),
              8.0 * nfine * c.nv * nrhs, st);
    if (prec == QCD_FP64)
        prolong_kernel<double2><<<grid_for(n), 256, 0, st>>>(f.g, c.B, c.nv, c.P64, (const double2*)xc, (double2*)x, nrhs,
                                                             accumulate, act);
    else
        prolong_kernel<float2><<<grid_for(n), 256, 0, st>>>(f.g, c.B, c.nv, c.P32, (const float2*)xc, (float2*)x, nrhs,
                                                            accumulate, act);
}

void coarse_apply(const Coarse& c, int prec, int op, int nrhs, const void* x, void* y, const double* tau,
                  cudaStream_t st, bool tensor) {
    Shifts sh{};
    for (int j = 0; j < nrhs; ++j) sh.t[j] = tau ? tau[j] : 0.0;
    const double es = prec == QCD_FP64 ? 16.0 : 8.0;
    const bool tc = prec == QCD_FP32 && tensor && c.nc % 8 == 0 && c.nc <= 64;
    // bulk-copy kernel: FP32, 16-byte aligned vectors, 2 nc threads
    const bool bulk = prec == QCD_FP32 && !tc && c.nc <= 64 && ((uintptr_t)x & 15) == 0 &&
                      ((uintptr_t)c.A32 & 15) == 0;
    const int rchunk = bulk ? kBulkR : (tc ? kTcR : kCoarseRC);
    KTimer kt(prec == QCD_FP64 ? "coarse_apply_f64"
                               : (tc ? "coarse_apply_tc" : (bulk ? "coarse_apply_bulk" : "coarse_apply_f32")),
              es * ((double)c.gc.V * 9 * c.nc * c.nc * ((nrhs + rchunk - 1) / rchunk) +
                    2.0 * nrhs * c.gc.V * c.nc),
              8.0 * 9 * c.nc * c.nc * (double)c.gc.V * nrhs, st);
    if (bulk) {
        const size_t sm = coarse_bulk_smem(c.nc);
        if (sm + 1024 > 48 * 1024)
            cudaFuncSetAttribute(coarse_apply_bulk_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        const dim3 grid(c.gc.V, (nrhs + kBulkR - 1) / kBulkR);
        coarse_apply_bulk_kernel<<<grid, 2 * c.nc, sm, st>>>(c.gc, c.nc, c.A32, (const float2*)x, (float2*)y, op, sh,
                                                            nrhs);
        return;
    }
    if (prec == QCD_FP32 && tensor && c.nc % 8 == 0 && c.nc <= 64) {
        const size_t sm = coarse_tc_smem(c.nc);
        if (sm + 1024 > 48 * 1024)
            cudaFuncSetAttribute(coarse_apply_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        const dim3 grid(c.gc.V, (nrhs + kTcR - 1) / kTcR);
        coarse_apply_tc_kernel<<<grid, 32 * (c.nc / 8), sm, st>>>(c.gc, c.nc, c.A32, (const float2*)x, (float2*)y,
                                                                  op, sh, nrhs);
        return;
    }
    // right-hand sides per CTA: a multiple of kCoarseRPT, at most kCoarseRC
    const int rc = std::min(kCoarseRC, (nrhs + kCoarseRPT - 1) / kCoarseRPT * kCoarseRPT);
    const dim3 grid(c.gc.V, (nrhs + rc - 1) / rc);
    const int threads = c.nc * (rc / kCoarseRPT);
    const size_t ebytes = prec == QCD_FP64 ? sizeof(double2) : sizeof(float2);
    const size_t sm = (size_t)9 * c.nc * rc * ebytes;
    if (prec == QCD_FP64) {
        if (sm + 1024 > 48 * 1024)
            cudaFuncSetAttribute(coarse_apply_mrhs_kernel<double2, double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)sm);
        coarse_apply_mrhs_kernel<double2, double><<<grid, threads, sm, st>>>(c.gc, c.nc, c.A64, (const double2*)x,
                                                                            (double2*)y, op, sh, nrhs, rc);
    } else {
        if (sm + 1024 > 48 * 1024)
            cudaFuncSetAttribute(coarse_apply_mrhs_kernel<float2, float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)sm);
        coarse_apply_mrhs_kernel<float2, float><<<grid, threads, sm, st>>>(c.gc, c.nc, c.A32, (const float2*)x,
                                                                          (float2*)y, op, sh, nrhs, rc);
    }
}

bool sap_needs_scratch(const Blocking& B) { return B.bs != 16 && B.bs != 32; }

void sap_work_reset() {
    static const unsigned long long zero[2][64] = {};
    cudaMemcpyToSymbol(g_sap_work, zero, sizeof(zero));
}
void wait_probe(cudaStream_t st) {
    KTimer kt("wait_probe", 0.0, 0.0, st);
    wait_probe_kernel<<<1, 32, 0, st>>>(1ll << 21);
}

unsigned long long wait_timeouts_read() {
    unsigned long long h = 0;
    cudaMemcpyFromSymbol(&h, g_wait_timeouts, sizeof(h));
    return h;
}

void sap_work_read(double out[2]) {
    unsigned long long h[2][64];
    cudaMemcpyFromSymbol(h, g_sap_work, sizeof(h));
    out[0] = out[1] = 0.0;
    for (int i = 0; i < 64; ++i) {
        out[0] += (double)h[0][i];
        out[1] += (double)h[1][i];
    }
}

size_t sap_scratch_bytes(const SapPlan& sp, int prec, int nrhs, int iters) {
    if (!sap_needs_scratch(sp.B)) return 0;
    size_t per = (size_t)(iters + 1) * sp.B.bs * 12 * (prec == QCD_FP64 ? sizeof(double2) : sizeof(float2));
    int nmax = sp.ncol[0] > sp.ncol[1] ? sp.ncol[0] : sp.ncol[1];
    return per * nmax * nrhs;
}

void sap_blocks(const FineOp& f, const SapPlan& sp, int colour, int prec, int op, int nrhs, const void* r, void* x,
                const double* tau, int iters, double tol, void* scratch, cudaStream_t st, const int* act, bool half) {
    Shifts sh{};
    for (int j = 0; j < nrhs; ++j) sh.t[j] = tau ? tau[j] : 0.0;
    const int bs = sp.B.bs;
    const double rs = prec == QCD_FP64 ? 8.0 : 4.0;
    const double sites = (double)sp.ncol[colour] * bs;
    KTimer kt(prec == QCD_FP64 ? "sap_block_f64" : (half && bs == 16 ? "sap_block_f32h" : "sap_block_f32"),
              rs * sites * (nrhs * 72.0 + 144.0),
              1824.0 * sites * nrhs * iters, st);
    if (bs == 16) {
        // one warp per block solve; with four or more right-hand sides four
        // of them share a CTA (and one staged copy of the block's links and
        // clover), so more block solves fit in shared memory per SM
        const int rw = nrhs >= 4 ? 4 : 1;
        dim3 grid(sp.ncol[colour], (nrhs + rw - 1) / rw);
        if (prec == QCD_FP64) {
            const size_t sm = chi_layout<double>(iters, sizeof(double2), rw).total;
            if (sm + 1024 > 48 * 1024)
                cudaFuncSetAttribute(sap_chi_kernel<double, double2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)sm);
            sap_chi_kernel<double, double2><<<grid, 32 * rw, sm, st>>>(f.g, sp.B, f.U64, f.A64,
                sp.blocks_of_colour[colour], sp.ncol[colour], op, sh, (const double2*)r, (double2*)x, iters, tol,
                act, nrhs);
        } else if (half) {
            const size_t sm = chi_layout<float>(iters, sizeof(__half2), rw).total;
            if (sm + 1024 > 48 * 1024)
                cudaFuncSetAttribute(sap_chi_kernel<float, __half2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)sm);
            sap_chi_kernel<float, __half2><<<grid, 32 * rw, sm, st>>>(f.g, sp.B, f.U32, f.A32,
                sp.blocks_of_colour[colour], sp.ncol[colour], op, sh, (const float2*)r, (float2*)x, iters, tol,
                act, nrhs);
        } else {
            const size_t sm = chi_layout<float>(iters, sizeof(float2), rw).total;
            if (sm + 1024 > 48 * 1024)
                cudaFuncSetAttribute(sap_chi_kernel<float, float2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)sm);
            sap_chi_kernel<float, float2><<<grid, 32 * rw, sm, st>>>(f.g, sp.B, f.U32, f.A32,
                sp.blocks_of_colour[colour], sp.ncol[colour], op, sh, (const float2*)r, (float2*)x, iters, tol,
                act, nrhs);
        }
        return;
    }
    if (bs == 32) {
        // one 32-site block per single-warp CTA
        dim3 grid(sp.ncol[colour], nrhs);
        if (prec == QCD_FP64) {
            const size_t sm = sap_layout<double>(32, iters).total;
            if (sm + 1024 > 48 * 1024) cudaFuncSetAttribute(sap_warp_kernel<double, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
            sap_warp_kernel<double, 32><<<grid, 32, sm, st>>>(f.g, sp.B, f.U64, f.A64, sp.blocks_of_colour[colour],
                sp.ncol[colour], op, sh, (const double2*)r, (double2*)x, iters, tol, act);
        } else {
            const size_t sm = sap_layout<float>(32, iters).total;
            if (sm + 1024 > 48 * 1024) cudaFuncSetAttribute(sap_warp_kernel<float, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
            sap_warp_kernel<float, 32><<<grid, 32, sm, st>>>(f.g, sp.B, f.U32, f.A32, sp.blocks_of_colour[colour],
                sp.ncol[colour], op, sh, (const float2*)r, (float2*)x, iters, tol, act);
        }
        return;
    }
    // every other block size: one thread per block site, Krylov vectors in `scratch`
    dim3 grid(sp.ncol[colour], nrhs);
    size_t sm = sizeof(double2) * ((size_t)bs + (size_t)(iters + 1) * iters + (iters + 1) + 2 * iters) +
                sizeof(double) * iters + 4 * sizeof(int) +
                (size_t)bs * 12 * (prec == QCD_FP64 ? sizeof(double2) : sizeof(float2));
    if (prec == QCD_FP64) {
        if (sm + 1024 > 48 * 1024) cudaFuncSetAttribute(sap_block_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        sap_block_kernel<double><<<grid, bs, sm, st>>>(f.g, sp.B, f.U64, f.A64, sp.blocks_of_colour[colour], op, sh,
                                                       (const double2*)r, (double2*)x, iters, tol, (double2*)scratch, act);
    } else {
        if (sm + 1024 > 48 * 1024) cudaFuncSetAttribute(sap_block_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        sap_block_kernel<float><<<grid, bs, sm, st>>>(f.g, sp.B, f.U32, f.A32, sp.blocks_of_colour[colour], op, sh,
                                                      (const float2*)r, (float2*)x, iters, tol, (float2*)scratch, act);
    }
}

}  // namespace qcd
