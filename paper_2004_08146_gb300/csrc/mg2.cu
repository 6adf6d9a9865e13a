// Third level of the hierarchy: the aggregation of Sec. 2 applied to the
// coarse operator D_c.  Level-1 vectors are [site][chirality][i < Nv1]; a
// level-2 aggregate collects the level-1 sites of one block of the level-1
// lattice and splits them by the level-1 chirality index, so that
// Gamma5^c P2 = P2 Gamma5^cc.  The level-2 operator is the Galerkin product
// P2^H D_c P2, stored like D_c as a nine-direction stencil with column-major
// blocks [site][d][col][row].
#include <algorithm>

#include "internal.h"

namespace qcd {

namespace {

constexpr int kP2Threads = 128;
constexpr int kC2Threads = 64;   // >= 2 * Nv at every level (Nv <= 32)

// sum over the CTA (blockDim a power of two <= kP2Threads); every thread gets it
__device__ double2 cta_sum(double2 v, double2* red) {
    red[threadIdx.x] = v;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    const double2 r = red[0];
    __syncthreads();
    return r;
}

// lexicographic index (mu = 3 fastest) of coordinates c over extents L
__device__ __forceinline__ int lex4(const int c[4], const int L[4]) {
    return ((c[0] * L[1] + c[1]) * L[2] + c[2]) * L[3] + c[3];
}

}  // namespace

// CTA (b2, chi): copy the (aggregate, chirality) piece of the level-2 test
// vectors W [nv2][V1][2][nv1] into P2 [b2][chi][j][l][i], then modified
// Gram-Schmidt applied twice (each vector against the earlier ones, then
// normalised; the second pass repeats the first on its result).
__global__ void __launch_bounds__(kP2Threads) build_P2_kernel(Geom g1, Blocking B2, int nv1, int nv2,
                                                              const double2* __restrict__ W,
                                                              double2* __restrict__ P64, float2* __restrict__ P32) {
    __shared__ double2 red[kP2Threads];
    const int b2 = blockIdx.x, chi = blockIdx.y;
    const int L = B2.bs * nv1, nc1 = 2 * nv1;
    const size_t off = ((size_t)b2 * 2 + chi) * nv2 * L;
    double2* base = P64 + off;
    for (int j = 0; j < nv2; ++j)
        for (int e = threadIdx.x; e < L; e += blockDim.x) {
            const int l = e / nv1, i = e % nv1;
            const int site = block_fine_site(g1, B2, b2, l);
            base[(size_t)j * L + e] = W[(size_t)j * g1.V * nc1 + (size_t)site * nc1 + chi * nv1 + i];
        }
    __syncthreads();
    for (int pass = 0; pass < 2; ++pass)
        for (int j = 0; j < nv2; ++j) {
            double2* vj = base + (size_t)j * L;
            for (int k = 0; k < j; ++k) {
                const double2* vk = base + (size_t)k * L;
                double2 h = make_double2(0, 0);
                for (int e = threadIdx.x; e < L; e += blockDim.x) h += conj(vk[e]) * vj[e];
                h = cta_sum(h, red);
                for (int e = threadIdx.x; e < L; e += blockDim.x) vj[e] = vj[e] - h * vk[e];
            }
            double2 s = make_double2(0, 0);
            for (int e = threadIdx.x; e < L; e += blockDim.x) s.x += vj[e].x * vj[e].x + vj[e].y * vj[e].y;
            s = cta_sum(s, red);
            const double nrm = sqrt(s.x);
            const double inv = nrm > 0 ? 1.0 / nrm : 1.0;
            for (int e = threadIdx.x; e < L; e += blockDim.x) vj[e] = inv * vj[e];
            __syncthreads();
        }
    for (int e = threadIdx.x; e < nv2 * L; e += blockDim.x)
        P32[off + e] = make_float2((float)base[e].x, (float)base[e].y);
}

// xc[j][b2][chi][i2] = sum_{l, i} conj(P2[b2][chi][i2][l][i]) r[j][site(b2, l)][chi][i]; one warp per output
template <typename Z, typename R>
__global__ void restrict2_kernel(Geom g1, Blocking B2, int nv1, int nv2, const Z* __restrict__ P,
                                 const Z* __restrict__ r, Z* __restrict__ xc, int nrhs, const int* __restrict__ act) {
    const int nc2 = 2 * nv2, nc1 = 2 * nv1;
    const int nloc = B2.bs * nv1;
    const long total = (long)B2.nb * nc2 * nrhs;
    const int lane = threadIdx.x & 31;
    for (long w = (blockIdx.x * (long)blockDim.x + threadIdx.x) >> 5; w < total;
         w += ((long)gridDim.x * blockDim.x) >> 5) {
        const int j = (int)(w / ((long)B2.nb * nc2));
        if (act != nullptr && !act[j]) continue;
        const int rem = (int)(w - (long)j * B2.nb * nc2);
        const int blk = rem / nc2, ci = rem % nc2;
        const int chi = ci / nv2, i2 = ci % nv2;
        const Z* p = P + (((size_t)blk * 2 + chi) * nv2 + i2) * nloc;
        const Z* rr = r + (size_t)j * g1.V * nc1;
        R re = 0, im = 0;
        for (int d = lane; d < nloc; d += 32) {
            const int l = d / nv1, i = d % nv1;
            const int site = block_fine_site(g1, B2, blk, l);
            const Z a = p[d], b = rr[(size_t)site * nc1 + chi * nv1 + i];
            re += a.x * b.x + a.y * b.y;
            im += a.x * b.y - a.y * b.x;
        }
        re = warp_sum(re);
        im = warp_sum(im);
        if (lane == 0) {
            Z o;
            o.x = re;
            o.y = im;
            xc[(size_t)j * B2.nb * nc2 + (size_t)blk * nc2 + ci] = o;
        }
    }
}

// x[j][site(b2, l)][chi][i] = sum_i2 P2[b2][chi][i2][l][i] xc[j][b2][chi][i2] (overwrites x)
template <typename Z>
__global__ void prolong2_kernel(Geom g1, Blocking B2, int nv1, int nv2, const Z* __restrict__ P,
                                const Z* __restrict__ xc, Z* __restrict__ x, int nrhs, const int* __restrict__ act) {
    const int nc2 = 2 * nv2, nc1 = 2 * nv1;
    const int nloc = B2.bs * nv1;
    const size_t total = (size_t)nrhs * B2.nb * 2 * nloc;
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total; t += (size_t)gridDim.x * blockDim.x) {
        const int j = (int)(t / ((size_t)B2.nb * 2 * nloc));
        if (act != nullptr && !act[j]) continue;
        const size_t rem = t - (size_t)j * B2.nb * 2 * nloc;
        const int blk = (int)(rem / (2 * nloc));
        const int chi = (int)((rem / nloc) % 2);
        const int d = (int)(rem % nloc);
        const Z* p = P + ((size_t)blk * 2 + chi) * nv2 * nloc + d;
        const Z* c = xc + (size_t)j * B2.nb * nc2 + (size_t)blk * nc2 + chi * nv2;
        Z acc;
        acc.x = 0;
        acc.y = 0;
        for (int i2 = 0; i2 < nv2; ++i2) acc += p[(size_t)i2 * nloc] * c[i2];
        const int l = d / nv1, i = d % nv1;
        x[(size_t)j * g1.V * nc1 + (size_t)block_fine_site(g1, B2, blk, l) * nc1 + chi * nv1 + i] = acc;
    }
}

// CTA (b2, column (chi', j')): the column of P2 over all aggregates is pushed
// through the nine terms of the level-1 stencil from every level-1 site x of
// aggregate b2; a term that reads across the face of the aggregate in a
// direction with level-2 extent > 1 goes to that level-2 direction, every
// other term to the self term; each piece is restricted with P2_b2^H.  FP64
// arithmetic; the level-1 stencil is read in FP64, or in FP32 when only the
// FP32 operator of a mixed-precision hierarchy is current.
template <typename Z1>
__global__ void __launch_bounds__(kC2Threads) build_coarse2_kernel(Geom g1, Blocking B2, int nv1, int nv2,
                                                                   const Z1* __restrict__ A1,
                                                                   const double2* __restrict__ P2,
                                                                   double2* __restrict__ A2) {
    __shared__ double2 sv[32];
    __shared__ double2 h[64];
    __shared__ double2 acc[9][64];
    const int b2 = blockIdx.x, col = blockIdx.y;
    const int nc1 = 2 * nv1, nc2 = 2 * nv2, nloc = B2.bs * nv1;
    const int chic = col / nv2, jc = col % nv2;
    const int t = threadIdx.x;
    for (int d = 0; d < 9; ++d)
        if (t < nc2) acc[d][t] = make_double2(0, 0);
    __syncthreads();
    for (int l = 0; l < B2.bs; ++l) {
        const int x = block_fine_site(g1, B2, b2, l);
        int xc[4];
        site_coords(g1, x, xc);
        for (int d1 = 0; d1 < 9; ++d1) {
            int yc[4] = {xc[0], xc[1], xc[2], xc[3]};
            int d2 = 0;
            if (d1 > 0) {
                const int mu = (d1 - 1) % 4, sgn = d1 <= 4 ? 1 : -1;
                yc[mu] = (yc[mu] + sgn + g1.L[mu]) % g1.L[mu];
                const int o = xc[mu] % B2.b[mu];
                const bool face = (sgn > 0 ? o == B2.b[mu] - 1 : o == 0) && B2.cd[mu] > 1;
                d2 = face ? d1 : 0;
            }
            const int y = site_index(g1, yc);
            int cb[4], ob[4];
            for (int mu = 0; mu < 4; ++mu) {
                cb[mu] = yc[mu] / B2.b[mu];
                ob[mu] = yc[mu] % B2.b[mu];
            }
            const int b2y = lex4(cb, B2.cd), ly = lex4(ob, B2.b);
            if (t < nv1) sv[t] = P2[(((size_t)b2y * 2 + chic) * nv2 + jc) * nloc + (size_t)ly * nv1 + t];
            __syncthreads();
            if (t < nc1) {
                const Z1* a = A1 + ((size_t)x * 9 + d1) * nc1 * nc1 + (size_t)chic * nv1 * nc1 + t;
                double2 s = make_double2(0, 0);
                for (int i = 0; i < nv1; ++i) s += cvt<double2>(a[(size_t)i * nc1]) * sv[i];
                h[t] = s;
            }
            __syncthreads();
            if (t < nc2) {
                const int chi = t / nv2, j = t % nv2;
                const double2* p = P2 + (((size_t)b2 * 2 + chi) * nv2 + j) * nloc + (size_t)l * nv1;
                double2 s = make_double2(0, 0);
                for (int i = 0; i < nv1; ++i) s += conj(p[i]) * h[chi * nv1 + i];
                acc[d2][t] += s;
            }
            __syncthreads();
        }
    }
    if (t < nc2)
        for (int d = 0; d < 9; ++d) A2[(((size_t)b2 * 9 + d) * nc2 + col) * nc2 + t] = acc[d][t];
}

void mg2_build_P(const Coarse& c1, Coarse& c2, const double2* W, cudaStream_t st) {
    KTimer kt("build_P2", 0.0, 0.0, st);
    build_P2_kernel<<<dim3(c2.B.nb, 2), kP2Threads, 0, st>>>(c1.gc, c2.B, c1.nv, c2.nv, W, c2.P64, c2.P32);
}

void mg2_build_coarse(const Coarse& c1, Coarse& c2, cudaStream_t st) {
    {
        KTimer kt("build_coarse2", 0.0, 0.0, st);
        if (c1.a64_stale)
            build_coarse2_kernel<float2><<<dim3(c2.B.nb, c2.nc), kC2Threads, 0, st>>>(c1.gc, c2.B, c1.nv, c2.nv, c1.A32,
                                                                                     c2.P64, c2.A64);
        else
            build_coarse2_kernel<double2><<<dim3(c2.B.nb, c2.nc), kC2Threads, 0, st>>>(c1.gc, c2.B, c1.nv, c2.nv,
                                                                                      c1.A64, c2.P64, c2.A64);
    }
    blas_convert(QCD_FP64, c2.A64, QCD_FP32, c2.A32, (size_t)c2.B.nb * 9 * c2.nc * c2.nc, st);
    c2.a64_stale = false;
}

void mg2_restrict(const Coarse& c1, const Coarse& c2, int prec, int nrhs, const void* r, void* xc, cudaStream_t st,
                  const int* act) {
    const long warps = (long)c2.B.nb * c2.nc * nrhs;
    const int grid = (int)std::min<long>((warps * 32 + 255) / 256, 152L * 16);
    const double es = prec == QCD_FP64 ? 16.0 : 8.0, n1 = (double)c1.gc.V * c1.nc;
    KTimer kt(prec == QCD_FP64 ? "restrict2_f64" : "restrict2_f32",
              es * (n1 * c2.nv + nrhs * (n1 + (double)c2.gc.V * c2.nc)), 8.0 * n1 * c2.nv * nrhs, st);
    if (prec == QCD_FP64)
        restrict2_kernel<double2, double><<<grid, 256, 0, st>>>(c1.gc, c2.B, c1.nv, c2.nv, c2.P64, (const double2*)r,
                                                                (double2*)xc, nrhs, act);
    else
        restrict2_kernel<float2, float><<<grid, 256, 0, st>>>(c1.gc, c2.B, c1.nv, c2.nv, c2.P32, (const float2*)r,
                                                              (float2*)xc, nrhs, act);
}

void mg2_prolong(const Coarse& c1, const Coarse& c2, int prec, int nrhs, const void* xc, void* x, cudaStream_t st,
                 const int* act) {
    const size_t total = (size_t)nrhs * c2.B.nb * 2 * c2.B.bs * c1.nv;
    const int grid = (int)std::min<size_t>((total + 255) / 256, 152 * 16);
    const double es = prec == QCD_FP64 ? 16.0 : 8.0, n1 = (double)c1.gc.V * c1.nc;
    KTimer kt(prec == QCD_FP64 ? "prolong2_f64" : "prolong2_f32",
              es * (n1 * c2.nv + nrhs * (n1 + (double)c2.gc.V * c2.nc)), 8.0 * n1 * c2.nv * nrhs, st);
    if (prec == QCD_FP64)
        prolong2_kernel<double2><<<grid, 256, 0, st>>>(c1.gc, c2.B, c1.nv, c2.nv, c2.P64, (const double2*)xc,
                                                       (double2*)x, nrhs, act);
    else
        prolong2_kernel<float2><<<grid, 256, 0, st>>>(c1.gc, c2.B, c1.nv, c2.nv, c2.P32, (const float2*)xc,
                                                      (float2*)x, nrhs, act);
}

}  // namespace qcd
