// Level-1 kernels on complex fields: copies, precision conversion, batched
// multi-dot products (deterministic two-pass reductions), multi-axpy for
// Gram-Schmidt (Algorithm 2, first line of the loop; FGMRES Arnoldi), Gamma5
// and a counter-based Gaussian generator for random start vectors.
#include "internal.h"

namespace qcd {

namespace {
constexpr int kThreads = 256;

inline size_t esz_of(int prec) { return prec == QCD_FP32 ? sizeof(float2) : sizeof(double2); }   // FF: 16 bytes

inline int grid_for(size_t n, int th = kThreads) {
    size_t g = (n + th - 1) / th;
    return (int)(g > 1048576 ? 1048576 : (g == 0 ? 1 : g));
}

template <typename Z>
__global__ void zero_kernel(Z* x, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        x[i] = Z{0, 0};
}
template <typename Zi, typename Zo>
__global__ void convert_kernel(const Zi* __restrict__ x, Zo* __restrict__ y, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        y[i] = cvt<Zo>(x[i]);
}

// partial[(v * nsplit) + split] = sum over this split of conj(X[i][j]) w[j]
template <typename Z>
__global__ void multidot_partial_kernel(const Z* __restrict__ X, size_t xstride_vec, const Z* __restrict__ w,
                                        int nrhs, size_t n, int nsplit, double2* __restrict__ partial,
                                        unsigned* __restrict__ counters, double2* __restrict__ dots,
                                        const int* __restrict__ act) {
    const int v = blockIdx.y;            // v = i * nrhs + j
    const int i = v / nrhs, j = v % nrhs;
    if (act != nullptr && !act[j]) return;
    const Z* x = X + (size_t)i * xstride_vec + (size_t)j * n;
    const Z* y = w + (size_t)j * n;
    const size_t chunk = (n + nsplit - 1) / nsplit;
    const size_t lo = (size_t)blockIdx.x * chunk;
    const size_t hi = lo + chunk < n ? lo + chunk : n;
    // per-thread and per-warp sums in the vector precision (FP64 arithmetic
    // is ~64x slower than FP32 on this part); the cross-warp sum in FP64
    using Rt = decltype(Z{}.x);
    Rt ret = 0, imt = 0;
    for (size_t k = lo + threadIdx.x; k < hi; k += blockDim.x) {
        Z a = x[k], b = y[k];
        ret += a.x * b.x + a.y * b.y;
        imt += a.x * b.y - a.y * b.x;
    }
    __shared__ double sre[32], sim[32];
    double re = (double)warp_sum(ret);
    double im = (double)warp_sum(imt);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) { sre[wid] = re; sim[wid] = im; }
    __syncthreads();
    if (wid == 0) {
        const int nw = blockDim.x >> 5;
        re = lane < nw ? sre[lane] : 0.0;
        im = lane < nw ? sim[lane] : 0.0;
        re = warp_sum(re);
        im = warp_sum(im);
        if (lane == 0) partial[(size_t)v * nsplit + blockIdx.x] = make_double2(re, im);
    }
    // the last CTA of dot v to finish adds the nsplit partials in a fixed
    // order and re-arms counters[v] (zero between launches)
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

constexpr int kAxpyCoef = 2048;   // coefficients staged per CTA (nvec * nrhs)

template <typename Z, typename R>
__global__ void multiaxpy_kernel(const Z* __restrict__ X, int nvec, size_t xstride_vec, const double2* __restrict__ c,
                                 double sign, Z* __restrict__ w, int nrhs, size_t n, const int* __restrict__ act) {
    // coefficients converted once per CTA to the working precision (a
    // conversion per element would run on the slow FP64 path)
    __shared__ Z cs[kAxpyCoef];
    const int nco = nvec * nrhs;
    const bool staged = nco <= kAxpyCoef;
    if (staged)
        for (int e = threadIdx.x; e < nco; e += blockDim.x) { cs[e].x = (R)c[e].x; cs[e].y = (R)c[e].y; }
    __syncthreads();
    const size_t total = n * nrhs;
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total; t += (size_t)gridDim.x * blockDim.x) {
        const int j = (int)(t / n);
        if (act != nullptr && !act[j]) continue;
        const size_t k = t - (size_t)j * n;
        Z acc; acc.x = 0; acc.y = 0;
        for (int i = 0; i < nvec; ++i) {
            Z ci;
            if (staged) ci = cs[i * nrhs + j];
            else { ci.x = (R)c[i * nrhs + j].x; ci.y = (R)c[i * nrhs + j].y; }
            if (ci.x == R(0) && ci.y == R(0)) continue;   // unused basis slots may hold stale data
            acc += ci * X[(size_t)i * xstride_vec + (size_t)j * n + k];
        }
        Z o = w[t];
        const R sg = (R)sign;
        o.x += sg * acc.x;
        o.y += sg * acc.y;
        w[t] = o;
    }
}

template <typename Z, typename R>
__global__ void scale_dev_kernel(const Z* __restrict__ x, Z* __restrict__ y, const double2* __restrict__ alpha,
                                 int nrhs, size_t n, bool invert_real, bool accumulate, const int* __restrict__ act) {
    const size_t total = n * nrhs;
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total; t += (size_t)gridDim.x * blockDim.x) {
        const int j = (int)(t / n);
        if (act != nullptr && !act[j]) continue;
        double2 a = alpha[j];
        if (invert_real) a = make_double2(a.x != 0.0 ? 1.0 / a.x : 0.0, 0.0);
        Z ar; ar.x = (R)a.x; ar.y = (R)a.y;
        Z o = ar * x[t];
        if (accumulate) o += y[t];
        y[t] = o;
    }
}

template <typename Z>
__global__ void gamma5_kernel(const Z* __restrict__ x, Z* __restrict__ y, size_t nsites) {
    const size_t total = nsites * 12;
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total; t += (size_t)gridDim.x * blockDim.x) {
        Z v = x[t];
        if ((t % 12) >= 6) { v.x = -v.x; v.y = -v.y; }
        y[t] = v;
    }
}

template <typename Z, typename R>
__global__ void axpby_kernel(double2 a, const Z* __restrict__ x, double2 b, Z* __restrict__ y, size_t n) {
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x) {
        Z ar, br;
        ar.x = (R)a.x; ar.y = (R)a.y;
        br.x = (R)b.x; br.y = (R)b.y;
        y[t] = ar * x[t] + br * y[t];
    }
}

// SplitMix64 (Steele, Lea, Flood 2014) as a counter-based hash.
__device__ __forceinline__ unsigned long long splitmix64(unsigned long long z) {
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
// Box-Muller: complex Gaussian with N(0,1) real and imaginary parts.
__global__ void gaussian_kernel(double2* x, size_t n, unsigned long long seed, unsigned long long offset) {
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x) {
        unsigned long long k = splitmix64(seed ^ splitmix64(offset + t));
        unsigned long long a = splitmix64(k), b = splitmix64(k + 1);
        double u1 = ((a >> 11) + 1.0) * (1.0 / 9007199254740993.0);   // (0, 1]
        double u2 = (b >> 11) * (1.0 / 9007199254740992.0);           // [0, 1)
        double r = sqrt(-2.0 * log(u1));
        double s, c;
        sincospi(2.0 * u2, &s, &c);
        x[t] = make_double2(r * c, r * s);
    }
}
}  // namespace

void blas_zero(int prec, void* x, size_t n, cudaStream_t st) {
    KTimer kt("blas_zero", (double)n * esz_of(prec), 0.0, st);
    if (prec != QCD_FP32) zero_kernel<double2><<<grid_for(n), kThreads, 0, st>>>((double2*)x, n);
    else zero_kernel<float2><<<grid_for(n), kThreads, 0, st>>>((float2*)x, n);
}
void blas_copy(int prec, const void* x, void* y, size_t n, cudaStream_t st) {
    cudaMemcpyAsync(y, x, n * esz_of(prec), cudaMemcpyDeviceToDevice, st);
}
void blas_convert(int prec_in, const void* x, int prec_out, void* y, size_t n, cudaStream_t st) {
    if (prec_in == prec_out) { blas_copy(prec_in, x, y, n, st); return; }
    if (prec_in == QCD_FF || prec_out == QCD_FF) { ff_convert(prec_in, x, prec_out, y, n, st); return; }
    KTimer kt("blas_convert", (double)n * (esz_of(prec_in) + esz_of(prec_out)), 0.0, st);
    if (prec_in == QCD_FP64)
        convert_kernel<double2, float2><<<grid_for(n), kThreads, 0, st>>>((const double2*)x, (float2*)y, n);
    else
        convert_kernel<float2, double2><<<grid_for(n), kThreads, 0, st>>>((const float2*)x, (double2*)y, n);
}
void blas_multidot(int prec, const void* X, int nvec, size_t xstride_vec, const void* w, int nrhs, size_t n,
                   double2* dots, double2* partial, unsigned* counters, cudaStream_t st, const int* act) {
    if (nvec <= 0) return;
    if (prec == QCD_FF) {
        ff_multidot(X, nvec, xstride_vec, w, nrhs, n, dots, partial, counters, st, act);
        return;
    }
    // enough CTAs to fill the GPU (about 4 per SM), at least 2048 elements each
    int nsplit = 608 / (nvec * nrhs);
    if (nsplit > 64) nsplit = 64;
    if ((size_t)nsplit * 2048 > n) nsplit = (int)(n / 2048);
    if (nsplit < 1) nsplit = 1;
    dim3 grid(nsplit, nvec * nrhs);
    KTimer kt(prec == QCD_FP64 ? "multidot_f64" : "multidot_f32", (double)(nvec + 1) * nrhs * n * esz_of(prec),
              8.0 * nvec * nrhs * n, st);
    if (prec == QCD_FP64)
        multidot_partial_kernel<double2><<<grid, kThreads, 0, st>>>((const double2*)X, xstride_vec, (const double2*)w,
                                                                   nrhs, n, nsplit, partial, counters, dots, act);
    else
        multidot_partial_kernel<float2><<<grid, kThreads, 0, st>>>((const float2*)X, xstride_vec, (const float2*)w,
                                                                  nrhs, n, nsplit, partial, counters, dots, act);
}
void blas_multiaxpy(int prec, const void* X, int nvec, size_t xstride_vec, const double2* c, double sign, void* w,
                    int nrhs, size_t n, cudaStream_t st, const int* act) {
    if (nvec <= 0) return;
    if (prec == QCD_FF) {
        ff_multiaxpy(X, nvec, xstride_vec, c, sign, w, nrhs, n, st, act);
        return;
    }
    size_t total = n * nrhs;
    KTimer kt(prec == QCD_FP64 ? "multiaxpy_f64" : "multiaxpy_f32", (double)(nvec + 2) * nrhs * n * esz_of(prec),
              8.0 * nvec * nrhs * n, st);
    if (prec == QCD_FP64)
        multiaxpy_kernel<double2, double><<<grid_for(total), kThreads, 0, st>>>((const double2*)X, nvec, xstride_vec, c,
                                                                              sign, (double2*)w, nrhs, n, act);
    else
        multiaxpy_kernel<float2, float><<<grid_for(total), kThreads, 0, st>>>((const float2*)X, nvec, xstride_vec, c,
                                                                            sign, (float2*)w, nrhs, n, act);
}
void blas_scale_dev(int prec, const void* x, void* y, const double2* alpha, int nrhs, size_t n, bool invert_real,
                    bool accumulate, cudaStream_t st, const int* act) {
    if (prec == QCD_FF) {
        if (invert_real) return;   // not used with double-float data
        ff_scale_dev(x, y, alpha, nrhs, n, accumulate, st, act);
        return;
    }
    size_t total = n * nrhs;
    KTimer kt("blas_scale", (double)total * (accumulate ? 3 : 2) * esz_of(prec), 0.0, st);
    if (prec == QCD_FP64)
        scale_dev_kernel<double2, double><<<grid_for(total), kThreads, 0, st>>>((const double2*)x, (double2*)y, alpha,
                                                                              nrhs, n, invert_real, accumulate, act);
    else
        scale_dev_kernel<float2, float><<<grid_for(total), kThreads, 0, st>>>((const float2*)x, (float2*)y, alpha,
                                                                            nrhs, n, invert_real, accumulate, act);
}
void blas_gamma5(int prec, const void* x, void* y, size_t nsites, cudaStream_t st) {
    if (prec == QCD_FF) { ff_gamma5(x, y, nsites, st); return; }
    size_t total = nsites * 12;
    KTimer kt("blas_gamma5", (double)total * 2 * esz_of(prec), 0.0, st);
    if (prec == QCD_FP64) gamma5_kernel<double2><<<grid_for(total), kThreads, 0, st>>>((const double2*)x, (double2*)y, nsites);
    else gamma5_kernel<float2><<<grid_for(total), kThreads, 0, st>>>((const float2*)x, (float2*)y, nsites);
}
void blas_gaussian(double2* x, size_t n, unsigned long long seed, unsigned long long offset, cudaStream_t st) {
    KTimer kt("gaussian", (double)n * 16, 0.0, st);
    gaussian_kernel<<<grid_for(n), kThreads, 0, st>>>(x, n, seed, offset);
}
void blas_axpby(int prec, double2 a, const void* x, double2 b, void* y, size_t n, cudaStream_t st) {
    if (prec == QCD_FF) { ff_axpby(a, x, b, y, n, st); return; }
    KTimer kt("blas_axpby", (double)n * 3 * esz_of(prec), 0.0, st);
    if (prec == QCD_FP64)
        axpby_kernel<double2, double><<<grid_for(n), kThreads, 0, st>>>(a, (const double2*)x, b, (double2*)y, n);
    else
        axpby_kernel<float2, float><<<grid_for(n), kThreads, 0, st>>>(a, (const float2*)x, b, (float2*)y, n);
}

}  // namespace qcd
