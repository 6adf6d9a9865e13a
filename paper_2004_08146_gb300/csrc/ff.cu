// Double-float ("ff") vector kernels for the Davidson basis (Sec. 3,
// Algorithm 2: Gram-Schmidt against [V X], the basis combinations u = V s,
// W s, the thick-restart transform and the lock-time deflation).
//
// A complex number is stored as two FP32 pairs, hi + lo (16 bytes, the size
// of a complex128), good to about 2^-48 relative.  Products and sums use the
// error-free transformations of Dekker and Knuth on the FP32 units:
//   two_prod(a, b) = (a*b, fma(a, b, -a*b))        exact product,
//   two_sum(a, b)  = (a+b, rounding error of a+b)   exact sum (6 flops).
// On this part FP32 FMA throughput is about 60x the FP64 rate, so these
// operations run at HBM speed where the FP64 forms were bound by the FP64
// pipe.  Results of inner products are returned in FP64.
#include "internal.h"

namespace qcd {

namespace {

constexpr int kThreads = 256;

struct ffr {
    float h, l;
};

__device__ __forceinline__ ffr two_sum(float a, float b) {
    const float s = a + b;
    const float bb = s - a;
    const float e = (a - (s - bb)) + (b - bb);
    return {s, e};
}
__device__ __forceinline__ ffr fast_two_sum(float a, float b) {   // |a| >= |b| or a == 0
    const float s = a + b;
    return {s, b - (s - a)};
}
__device__ __forceinline__ ffr two_prod(float a, float b) {
    const float p = a * b;
    return {p, fmaf(a, b, -p)};
}
__device__ __forceinline__ ffr split(double d) {
    const float h = (float)d;
    return {h, (float)(d - (double)h)};
}
__device__ __forceinline__ double join(ffr a) { return (double)a.h + (double)a.l; }

// accumulator: acc += a * b with a = (ah, al), b = (bh, bl): the exact
// product of the high parts and the exact sum into the running high part,
// the rounding errors and cross terms into the low part, renormalised every
// step so that the low part stays below half an ulp of the high part
// (sums of a few thousand terms stay at ~1e-16 relative).
struct acc_t {
    float h = 0.f, l = 0.f;
    __device__ __forceinline__ void mac(float ah, float al, float bh, float bl) {
        const ffr p = two_prod(ah, bh);
        const ffr s = two_sum(h, p.h);
        const ffr r = fast_two_sum(s.h, l + (s.l + p.l + fmaf(ah, bl, al * bh)));
        h = r.h;
        l = r.l;
    }
    __device__ __forceinline__ void msub(float ah, float al, float bh, float bl) { mac(-ah, -al, bh, bl); }
    __device__ __forceinline__ ffr get() const { return fast_two_sum(h, l); }
};

__device__ __forceinline__ ffr ff_add(ffr a, ffr b) {
    const ffr s = two_sum(a.h, b.h);
    return fast_two_sum(s.h, s.l + a.l + b.l);
}

// ---- element access: float4 = (re.h, im.h, re.l, im.l)
__device__ __forceinline__ float4 pack(ffr re, ffr im) { return make_float4(re.h, im.h, re.l, im.l); }

__global__ void ff_from_fp64_kernel(const double2* __restrict__ x, float4* __restrict__ y, size_t n) {
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x) {
        const double2 v = x[t];
        y[t] = pack(split(v.x), split(v.y));
    }
}
__global__ void ff_to_fp64_kernel(const float4* __restrict__ x, double2* __restrict__ y, size_t n) {
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x) {
        const float4 v = x[t];
        y[t] = make_double2((double)v.x + (double)v.z, (double)v.y + (double)v.w);
    }
}
__global__ void ff_to_fp32_kernel(const float4* __restrict__ x, float2* __restrict__ y, size_t n) {
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x) {
        const float4 v = x[t];
        y[t] = make_float2(v.x + v.z, v.y + v.w);
    }
}
__global__ void ff_from_fp32_kernel(const float2* __restrict__ x, float4* __restrict__ y, size_t n) {
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x) {
        const float2 v = x[t];
        y[t] = make_float4(v.x, v.y, 0.f, 0.f);
    }
}

// dots[v] = <X_i, w_j> (v = i * nrhs + j), same split-reduction scheme as the
// FP64 kernel: per-thread double-float sums, FP64 across the CTA and across
// CTAs (the last CTA of each dot adds the partials in a fixed order).
// blockIdx.x runs over the dots so that CTAs reading the same chunk of w
// are scheduled together.
__global__ void ff_multidot_kernel(const float4* __restrict__ X, size_t xstride_vec, const float4* __restrict__ w,
                                   int nrhs, size_t n, int nsplit, double2* __restrict__ partial,
                                   unsigned* __restrict__ counters, double2* __restrict__ dots,
                                   const int* __restrict__ act) {
    const int v = blockIdx.x;
    const int i = v / nrhs, j = v % nrhs;
    if (act != nullptr && !act[j]) return;
    const float4* x = X + (size_t)i * xstride_vec + (size_t)j * n;
    const float4* y = w + (size_t)j * n;
    const size_t chunk = (n + nsplit - 1) / nsplit;
    const size_t lo = (size_t)blockIdx.y * chunk;
    const size_t hi = lo + chunk < n ? lo + chunk : n;
    // two independent accumulator pairs (even / odd strides): twice the
    // loads in flight and two interleaved error-free chains per thread
    acc_t re, im, re1, im1;
    const size_t bd = blockDim.x;
    size_t k = lo + threadIdx.x;
    for (; k + bd < hi; k += 2 * bd) {
        const float4 a = x[k], b = y[k], a1 = x[k + bd], b1 = y[k + bd];
        // conj(a) b: re = ar br + ai bi, im = ar bi - ai br
        re.mac(a.x, a.z, b.x, b.z);
        re1.mac(a1.x, a1.z, b1.x, b1.z);
        im.mac(a.x, a.z, b.y, b.w);
        im1.mac(a1.x, a1.z, b1.y, b1.w);
        re.mac(a.y, a.w, b.y, b.w);
        re1.mac(a1.y, a1.w, b1.y, b1.w);
        im.msub(a.y, a.w, b.x, b.z);
        im1.msub(a1.y, a1.w, b1.x, b1.z);
    }
    if (k < hi) {
        const float4 a = x[k], b = y[k];
        re.mac(a.x, a.z, b.x, b.z);
        re.mac(a.y, a.w, b.y, b.w);
        im.mac(a.x, a.z, b.y, b.w);
        im.msub(a.y, a.w, b.x, b.z);
    }
    double dr = join(re.get()) + join(re1.get()), di = join(im.get()) + join(im1.get());
    dr = warp_sum(dr);
    di = warp_sum(di);
    __shared__ double sre[32], sim[32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) { sre[wid] = dr; sim[wid] = di; }
    __syncthreads();
    if (wid == 0) {
        const int nw = blockDim.x >> 5;
        dr = lane < nw ? sre[lane] : 0.0;
        di = lane < nw ? sim[lane] : 0.0;
        dr = warp_sum(dr);
        di = warp_sum(di);
        if (lane == 0) partial[(size_t)v * nsplit + blockIdx.y] = make_double2(dr, di);
    }
    __shared__ bool last;
    if (threadIdx.x == 0) {
        __threadfence();
        last = atomicAdd(&counters[v], 1u) == (unsigned)nsplit - 1;
    }
    __syncthreads();
    if (!last || wid != 0) return;
    __threadfence();
    double sr = 0.0, si = 0.0;
    for (int k = lane; k < nsplit; k += 32) {
        const double2 q = __ldcg(&partial[(size_t)v * nsplit + k]);
        sr += q.x;
        si += q.y;
    }
    sr = warp_sum(sr);
    si = warp_sum(si);
    if (lane == 0) {
        dots[v] = make_double2(sr, si);
        counters[v] = 0u;
    }
}

constexpr int kFFCoef = 2048;   // coefficients staged per CTA (nvec * nrhs)

// w[j] += sign * sum_i c[i * nrhs + j] X[i][j] (coefficients FP64, split once per CTA)
__global__ void ff_multiaxpy_kernel(const float4* __restrict__ X, int nvec, size_t xstride_vec,
                                    const double2* __restrict__ c, double sign, float4* __restrict__ w, int nrhs,
                                    size_t n, const int* __restrict__ act) {
    __shared__ float4 cs[kFFCoef];
    const int nco = nvec * nrhs;
    const bool staged = nco <= kFFCoef;
    if (staged)
        for (int e = threadIdx.x; e < nco; e += blockDim.x) {
            const double2 v = c[e];
            cs[e] = pack(split(sign * v.x), split(sign * v.y));
        }
    __syncthreads();
    const size_t total = n * nrhs;
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total; t += (size_t)gridDim.x * blockDim.x) {
        const int j = (int)(t / n);
        if (act != nullptr && !act[j]) continue;
        const size_t k = t - (size_t)j * n;
        const float4 w0 = w[t];
        acc_t re, im;
        re.h = w0.x; re.l = w0.z;
        im.h = w0.y; im.l = w0.w;
        for (int i = 0; i < nvec; ++i) {
            float4 ci;
            if (staged) ci = cs[i * nrhs + j];
            else {
                const double2 v = c[i * nrhs + j];
                ci = pack(split(sign * v.x), split(sign * v.y));
            }
            if (ci.x == 0.f && ci.y == 0.f) continue;   // unused basis slots may hold stale data
            const float4 a = X[(size_t)i * xstride_vec + (size_t)j * n + k];
            // c a: re = cr ar - ci ai, im = cr ai + ci ar
            re.mac(ci.x, ci.z, a.x, a.z);
            re.msub(ci.y, ci.w, a.y, a.w);
            im.mac(ci.x, ci.z, a.y, a.w);
            im.mac(ci.y, ci.w, a.x, a.z);
        }
        w[t] = pack(re.get(), im.get());
    }
}

// y[j] = alpha_j x[j] (+ y[j]); alpha FP64 on the device
__global__ void ff_scale_kernel(const float4* __restrict__ x, float4* __restrict__ y, const double2* __restrict__ alpha,
                                int nrhs, size_t n, bool accumulate, const int* __restrict__ act) {
    const size_t total = n * nrhs;
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total; t += (size_t)gridDim.x * blockDim.x) {
        const int j = (int)(t / n);
        if (act != nullptr && !act[j]) continue;
        const double2 a = alpha[j];
        const ffr ar = split(a.x), ai = split(a.y);
        const float4 v = x[t];
        acc_t re, im;
        if (accumulate) {
            const float4 o = y[t];
            re.h = o.x; re.l = o.z;
            im.h = o.y; im.l = o.w;
        }
        re.mac(ar.h, ar.l, v.x, v.z);
        re.msub(ai.h, ai.l, v.y, v.w);
        im.mac(ar.h, ar.l, v.y, v.w);
        im.mac(ai.h, ai.l, v.x, v.z);
        y[t] = pack(re.get(), im.get());
    }
}

// y = a x + b y (host scalars)
__global__ void ff_axpby_kernel(double2 a, const float4* __restrict__ x, double2 b, float4* __restrict__ y, size_t n) {
    const ffr ar = split(a.x), ai = split(a.y), br = split(b.x), bi = split(b.y);
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x) {
        const float4 v = x[t], u = y[t];
        acc_t re, im;
        re.mac(ar.h, ar.l, v.x, v.z);
        re.msub(ai.h, ai.l, v.y, v.w);
        im.mac(ar.h, ar.l, v.y, v.w);
        im.mac(ai.h, ai.l, v.x, v.z);
        re.mac(br.h, br.l, u.x, u.z);
        re.msub(bi.h, bi.l, u.y, u.w);
        im.mac(br.h, br.l, u.y, u.w);
        im.mac(bi.h, bi.l, u.x, u.z);
        y[t] = pack(re.get(), im.get());
    }
}

__global__ void ff_gamma5_kernel(const float4* __restrict__ x, float4* __restrict__ y, size_t nsites) {
    const size_t total = nsites * 12;
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total; t += (size_t)gridDim.x * blockDim.x) {
        float4 v = x[t];
        if ((t % 12) >= 6) { v.x = -v.x; v.y = -v.y; v.z = -v.z; v.w = -v.w; }
        y[t] = v;
    }
}

// In-place tall-skinny transform A[j] <- sum_i C[i + j m] A[i], j < p <= m
// (thick restart): each CTA stages kTile rows of all m vectors in shared
// memory and overwrites them with the p new rows; a warp computes one output
// vector for the tile's rows (one row per lane), so each coefficient is a
// warp-wide broadcast.  Coefficients pre-split to double-float in Cf.
constexpr int kTile = 32;
__global__ void __launch_bounds__(256) ff_transform_kernel(float4* __restrict__ A, int m, const float4* __restrict__ Cf,
                                                           int p, size_t n) {
    extern __shared__ float4 tile[];   // [m][kTile]
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const size_t ntiles = (n + kTile - 1) / kTile;
    for (size_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const size_t k0 = t * kTile;
        const int rows = (int)min((size_t)kTile, n - k0);
        for (int e = threadIdx.x; e < m * kTile; e += blockDim.x) {
            const int i = e / kTile, r = e % kTile;
            tile[e] = r < rows ? A[(size_t)i * n + k0 + r] : make_float4(0.f, 0.f, 0.f, 0.f);
        }
        __syncthreads();
        for (int j = warp; j < p; j += nw) {
            acc_t re, im;
            for (int i = 0; i < m; ++i) {
                const float4 c = __ldg(&Cf[(size_t)j * m + i]);
                const float4 a = tile[i * kTile + lane];
                re.mac(c.x, c.z, a.x, a.z);
                re.msub(c.y, c.w, a.y, a.w);
                im.mac(c.x, c.z, a.y, a.w);
                im.mac(c.y, c.w, a.x, a.z);
            }
            if (lane < rows) A[(size_t)j * n + k0 + lane] = pack(re.get(), im.get());
        }
        __syncthreads();
    }
}

__global__ void ff_split_kernel(const double2* __restrict__ c, float4* __restrict__ cf, int cnt, double scale) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < cnt; e += gridDim.x * blockDim.x) {
        const double2 v = c[e];
        cf[e] = pack(split(scale * v.x), split(scale * v.y));
    }
}

// Lock-time deflation A[j-1] <- A[j] - conj(w_j) f (sum_i w_i A[i]), j = 1..m-1,
// for the pair (V, W) selected by blockIdx.y; w (m entries) and f = w[m].x
// pre-split in wf.  Row k of the result depends on row k of A only, so each
// thread finishes its rows in place.
__global__ void ff_deflate_kernel(float4* __restrict__ A0, float4* __restrict__ A1, int m, size_t n,
                                  const float4* __restrict__ wf) {
    __shared__ float4 w[kMaxBasis + 1];
    for (int i = threadIdx.x; i <= m; i += blockDim.x) w[i] = wf[i];
    __syncthreads();
    float4* A = blockIdx.y ? A1 : A0;
    const float4 f = w[m];
    for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n; k += (size_t)gridDim.x * blockDim.x) {
        acc_t yr, yi;
        for (int i = 0; i < m; ++i) {
            const float4 c = w[i], a = A[(size_t)i * n + k];
            yr.mac(c.x, c.z, a.x, a.z);
            yr.msub(c.y, c.w, a.y, a.w);
            yi.mac(c.x, c.z, a.y, a.w);
            yi.mac(c.y, c.w, a.x, a.z);
        }
        // y <- f y (f real)
        const ffr y0r = yr.get(), y0i = yi.get();
        acc_t fr, fi;
        fr.mac(f.x, f.z, y0r.h, y0r.l);
        fi.mac(f.x, f.z, y0i.h, y0i.l);
        const ffr yR = fr.get(), yI = fi.get();
        for (int j = 1; j < m; ++j) {
            const float4 c = w[j], a = A[(size_t)j * n + k];
            // a - conj(c) y: re = ar - (cr yr + ci yi), im = ai - (cr yi - ci yr)
            acc_t re, im;
            re.h = a.x; re.l = a.z;
            im.h = a.y; im.l = a.w;
            re.msub(c.x, c.z, yR.h, yR.l);
            re.msub(c.y, c.w, yI.h, yI.l);
            im.msub(c.x, c.z, yI.h, yI.l);
            im.mac(c.y, c.w, yR.h, yR.l);
            A[(size_t)(j - 1) * n + k] = pack(re.get(), im.get());
        }
    }
}

inline int grid_for(size_t n, int th = kThreads) {
    size_t g = (n + th - 1) / th;
    return (int)(g > 1048576 ? 1048576 : (g == 0 ? 1 : g));
}
int sm_count() {
    static int sms = 0;
    if (sms == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 1;
    }
    return sms;
}

}  // namespace

void ff_convert(int prec_in, const void* x, int prec_out, void* y, size_t n, cudaStream_t st) {
    KTimer kt("ff_convert", (double)n * 24, 0.0, st);
    if (prec_in == QCD_FP64 && prec_out == QCD_FF)
        ff_from_fp64_kernel<<<grid_for(n), kThreads, 0, st>>>((const double2*)x, (float4*)y, n);
    else if (prec_in == QCD_FF && prec_out == QCD_FP64)
        ff_to_fp64_kernel<<<grid_for(n), kThreads, 0, st>>>((const float4*)x, (double2*)y, n);
    else if (prec_in == QCD_FF && prec_out == QCD_FP32)
        ff_to_fp32_kernel<<<grid_for(n), kThreads, 0, st>>>((const float4*)x, (float2*)y, n);
    else
        ff_from_fp32_kernel<<<grid_for(n), kThreads, 0, st>>>((const float2*)x, (float4*)y, n);
}

void ff_multidot(const void* X, int nvec, size_t xstride_vec, const void* w, int nrhs, size_t n, double2* dots,
                 double2* partial, unsigned* counters, cudaStream_t st, const int* act) {
    if (nvec <= 0) return;
    int nsplit = 4 * sm_count() / (nvec * nrhs);
    if (nsplit > 64) nsplit = 64;
    if ((size_t)nsplit * 2048 > n) nsplit = (int)(n / 2048);
    if (nsplit < 1) nsplit = 1;
    dim3 grid(nvec * nrhs, nsplit);
    KTimer kt("multidot_ff", (double)(nvec + 1) * nrhs * n * 16, 8.0 * nvec * nrhs * n, st);
    ff_multidot_kernel<<<grid, kThreads, 0, st>>>((const float4*)X, xstride_vec, (const float4*)w, nrhs, n, nsplit,
                                                  partial, counters, dots, act);
}

void ff_multiaxpy(const void* X, int nvec, size_t xstride_vec, const double2* c, double sign, void* w, int nrhs,
                  size_t n, cudaStream_t st, const int* act) {
    if (nvec <= 0) return;
    const size_t total = n * nrhs;
    KTimer kt("multiaxpy_ff", (double)(nvec + 2) * nrhs * n * 16, 8.0 * nvec * nrhs * n, st);
    ff_multiaxpy_kernel<<<grid_for(total), kThreads, 0, st>>>((const float4*)X, nvec, xstride_vec, c, sign,
                                                              (float4*)w, nrhs, n, act);
}

void ff_scale_dev(const void* x, void* y, const double2* alpha, int nrhs, size_t n, bool accumulate, cudaStream_t st,
                  const int* act) {
    const size_t total = n * nrhs;
    KTimer kt("ff_scale", (double)total * (accumulate ? 3 : 2) * 16, 0.0, st);
    ff_scale_kernel<<<grid_for(total), kThreads, 0, st>>>((const float4*)x, (float4*)y, alpha, nrhs, n, accumulate,
                                                          act);
}

void ff_axpby(double2 a, const void* x, double2 b, void* y, size_t n, cudaStream_t st) {
    KTimer kt("ff_axpby", (double)n * 3 * 16, 0.0, st);
    ff_axpby_kernel<<<grid_for(n), kThreads, 0, st>>>(a, (const float4*)x, b, (float4*)y, n);
}

void ff_gamma5(const void* x, void* y, size_t nsites, cudaStream_t st) {
    const size_t total = nsites * 12;
    KTimer kt("ff_gamma5", (double)total * 2 * 16, 0.0, st);
    ff_gamma5_kernel<<<grid_for(total), kThreads, 0, st>>>((const float4*)x, (float4*)y, nsites);
}

void ff_transform_inplace(void* A, int m, const double2* C, int p, size_t n, void* cf_scratch, cudaStream_t st) {
    float4* Cf = (float4*)cf_scratch;
    ff_split_kernel<<<(m * p + 255) / 256, 256, 0, st>>>(C, Cf, m * p, 1.0);
    const size_t sm = (size_t)m * kTile * sizeof(float4);
    if (sm + 1024 > 48 * 1024)
        cudaFuncSetAttribute(ff_transform_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    const size_t ntiles = (n + kTile - 1) / kTile;
    const int grid = (int)std::min<size_t>(ntiles, (size_t)sm_count() * 4);
    KTimer kt("basis_transform_ff", (double)(m + p) * n * 16, 8.0 * m * p * n, st);
    ff_transform_kernel<<<grid, 256, sm, st>>>((float4*)A, m, Cf, p, n);
}

void ff_deflate(void* A0, void* A1, int m, size_t n, const double2* hw, void* wf_scratch, cudaStream_t st) {
    float4* wf = (float4*)wf_scratch;
    ff_split_kernel<<<1, 128, 0, st>>>(hw, wf, m + 1, 1.0);
    const int gx = (int)std::min<size_t>((n + 255) / 256, (size_t)sm_count() * 8);
    KTimer kt("householder_deflate_ff", (double)(4 * m - 2) * n * 16, 16.0 * m * n * 2, st);
    ff_deflate_kernel<<<dim3(gx, 2), 256, 0, st>>>((float4*)A0, (float4*)A1, m, n, wf);
}

}  // namespace qcd
