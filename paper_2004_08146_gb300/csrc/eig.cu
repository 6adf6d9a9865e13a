// Small dense FP64 kernels of the Davidson outer iteration (Sec. 3):
// the harmonic Ritz pencil of Theorem 1 / Eq. 3.5, (W^H V) s = mu (W^H W) s
// with mu = 1/theta, solved as Cholesky W^H W = L L^H, C = L^-1 (W^H V) L^-H
// and a parallel (round-robin) complex Jacobi eigensolver; the QR used for
// thick restarts and the orthogonal complement used for locking.  All run in
// one CTA on column-major matrices with m <= 64.
#include "internal.h"

namespace qcd {

namespace {
constexpr int kT = 256;
constexpr int kTE = 512;   // threads of the harmonic eigen kernel

__device__ __forceinline__ double cabs2(double2 a) { return a.x * a.x + a.y * a.y; }

__device__ double block_reduce_sum(double v, double* red) {
    v = warp_sum(v);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) red[w] = v;
    __syncthreads();
    if (w == 0) {
        v = lane < (int)(blockDim.x >> 5) ? red[lane] : 0.0;
        v = warp_sum(v);
        if (lane == 0) red[32] = v;
    }
    __syncthreads();
    double r = red[32];
    __syncthreads();
    return r;
}

// work layout: L, Li, T, C (m*m each, FP64, global, column-major ld = m);
// the Jacobi sweeps run on an FP32 copy of C and its rotations (2*m*m float2
// of shared memory)
__global__ void __launch_bounds__(kTE) harmonic_eig_kernel(const double2* __restrict__ G, const double2* __restrict__ Hm,
                                                          int m, int ld, double* __restrict__ mu,
                                                          double2* __restrict__ S, double2* __restrict__ work,
                                                          int* __restrict__ status) {
    __shared__ double red[33];
    __shared__ int pp[32], qq[32];
    __shared__ double pc[32], ps[32];
    __shared__ double2 pph[32];
    const int tid = threadIdx.x;
    extern __shared__ double2 shm[];
    double2* L = work;
    double2* Li = L + m * m;
    double2* T = Li + m * m;
    double2* C = T + m * m;      // L^-1 H L^-H (FP64)
#define IDX(i, j) ((j) * m + (i))
    for (int e = tid; e < m * m; e += blockDim.x) {
        int i = e % m, j = e / m;
        // Hermitian parts (symmetrise against round-off)
        double2 g = 0.5 * (G[j * ld + i] + conj(G[i * ld + j]));
        double2 h = 0.5 * (Hm[j * ld + i] + conj(Hm[i * ld + j]));
        L[IDX(i, j)] = g;
        C[IDX(i, j)] = h;
        Li[IDX(i, j)] = make_double2(i == j ? 1.0 : 0.0, 0.0);
    }
    __syncthreads();
    // Cholesky G = L L^H (lower triangle of L)
    for (int k = 0; k < m; ++k) {
        if (tid == 0) {
            double d = L[IDX(k, k)].x;
            if (!(d > 0.0)) { status[0] = 1; d = 1e-300; }
            L[IDX(k, k)] = make_double2(sqrt(d), 0.0);
        }
        __syncthreads();
        const double inv = 1.0 / L[IDX(k, k)].x;
        for (int i = k + 1 + tid; i < m; i += blockDim.x) L[IDX(i, k)] = inv * L[IDX(i, k)];
        __syncthreads();
        for (int e = tid; e < (m - k - 1) * (m - k - 1); e += blockDim.x) {
            int i = k + 1 + e % (m - k - 1), j = k + 1 + e / (m - k - 1);
            if (j <= i) L[IDX(i, j)] -= L[IDX(i, k)] * conj(L[IDX(j, k)]);
        }
        __syncthreads();
    }
    // Li = L^-1, one column per thread (forward substitution)
    for (int j = tid; j < m; j += blockDim.x) {
        for (int i = j; i < m; ++i) {
            double2 s = make_double2(i == j ? 1.0 : 0.0, 0.0);
            for (int k = j; k < i; ++k) s -= L[IDX(i, k)] * Li[IDX(k, j)];
            Li[IDX(i, j)] = (1.0 / L[IDX(i, i)].x) * s;
        }
    }
    __syncthreads();
    // T = Li * Hm ; C = T * Li^H
    for (int e = tid; e < m * m; e += blockDim.x) {
        int i = e % m, j = e / m;
        double2 s = make_double2(0, 0);
        for (int k = 0; k <= i; ++k) s += Li[IDX(i, k)] * C[IDX(k, j)];
        T[IDX(i, j)] = s;
    }
    __syncthreads();
    for (int e = tid; e < m * m; e += blockDim.x) {
        int i = e % m, j = e / m;
        double2 s = make_double2(0, 0);
        for (int k = 0; k <= j; ++k) s += T[IDX(i, k)] * conj(Li[IDX(j, k)]);
        C[IDX(i, j)] = s;
    }
    __syncthreads();
    // FP32 working copy for the Jacobi sweeps: the decomposition feeds target
    // selection and thick restarts, which need no more; the targeted pairs
    // are refined in FP64 afterwards (refine_targets_kernel)
    float2* Cf = reinterpret_cast<float2*>(shm);
    float2* Zf = Cf + m * m;
    for (int e = tid; e < m * m; e += blockDim.x) {
        Cf[e] = make_float2((float)C[e].x, (float)C[e].y);
        Zf[e] = make_float2((e % m) == (e / m) ? 1.f : 0.f, 0.f);
    }
    __syncthreads();
    const int mm = (m % 2) ? m + 1 : m;   // padded player count
    const int npair = mm / 2;
    float fro = 0.0f;
    for (int e = tid; e < m * m; e += blockDim.x) fro += Cf[e].x * Cf[e].x + Cf[e].y * Cf[e].y;
    fro = (float)block_reduce_sum((double)fro, red);
    for (int sweep = 0; sweep < 40; ++sweep) {
        float off = 0.0f;
        for (int e = tid; e < m * m; e += blockDim.x)
            if (e % m != e / m) off += Cf[e].x * Cf[e].x + Cf[e].y * Cf[e].y;
        off = (float)block_reduce_sum((double)off, red);
        if (off <= 1e-13f * fro || m < 2) break;
        for (int rnd = 0; rnd < mm - 1; ++rnd) {
            if (tid < npair) {
                int k = tid;
                auto player = [&](int pos) { return pos == 0 ? 0 : ((rnd + pos - 1) % (mm - 1)) + 1; };
                int p = player(k), q = player(mm - 1 - k);
                if (p > q) { int t = p; p = q; q = t; }
                float c = 1.f, sv = 0.f;
                float2 ph = make_float2(1.f, 0.f);
                if (q < m) {
                    float2 b = Cf[IDX(p, q)];
                    float ab = sqrtf(b.x * b.x + b.y * b.y);
                    if (ab > 1e-30f) {
                        ph = make_float2(b.x / ab, b.y / ab);
                        float a = Cf[IDX(p, p)].x, d = Cf[IDX(q, q)].x;
                        float zeta = (d - a) / (2.0f * ab);
                        float t = (zeta >= 0 ? 1.0f : -1.0f) / (fabsf(zeta) + sqrtf(1.0f + zeta * zeta));
                        c = 1.0f / sqrtf(1.0f + t * t);
                        sv = t * c;
                    }
                }
                pp[k] = p; qq[k] = q; pc[k] = c; ps[k] = sv; pph[k] = make_double2(ph.x, ph.y);
            }
            __syncthreads();
            for (int e = tid; e < npair * m; e += blockDim.x) {
                int k = e / m, r = e % m;
                int p = pp[k], q = qq[k];
                if (q >= m) continue;
                float c = (float)pc[k], sv = (float)ps[k];
                float2 em = make_float2((float)pph[k].x, -(float)pph[k].y);
                float2 ap = Cf[IDX(r, p)], aq = Cf[IDX(r, q)];
                Cf[IDX(r, p)] = c * ap - sv * (em * aq);
                Cf[IDX(r, q)] = sv * ap + c * (em * aq);
                float2 zp = Zf[IDX(r, p)], zq = Zf[IDX(r, q)];
                Zf[IDX(r, p)] = c * zp - sv * (em * zq);
                Zf[IDX(r, q)] = sv * zp + c * (em * zq);
            }
            __syncthreads();
            for (int e = tid; e < npair * m; e += blockDim.x) {
                int k = e / m, col = e % m;
                int p = pp[k], q = qq[k];
                if (q >= m) continue;
                float c = (float)pc[k], sv = (float)ps[k];
                float2 ep = make_float2((float)pph[k].x, (float)pph[k].y);
                float2 ap = Cf[IDX(p, col)], aq = Cf[IDX(q, col)];
                Cf[IDX(p, col)] = c * ap - sv * (ep * aq);
                Cf[IDX(q, col)] = sv * ap + c * (ep * aq);
            }
            __syncthreads();
        }
    }
    for (int i = tid; i < m; i += blockDim.x) mu[i] = (double)Cf[IDX(i, i)].x;
    // S = Li^H Z  (upper-triangular Li^H)
    for (int e = tid; e < m * m; e += blockDim.x) {
        int i = e % m, j = e / m;
        double2 sacc = make_double2(0, 0);
        for (int k = i; k < m; ++k) {
            float2 z = Zf[IDX(k, j)];
            sacc += conj(Li[IDX(k, i)]) * make_double2(z.x, z.y);
        }
        S[IDX(i, j)] = sacc;
    }
#undef IDX
}

// FP64 refinement of targeted harmonic Ritz pairs (one CTA per target):
// inverse iteration on the pencil H s = mu G s (mu = 1/theta), started from
// the FP32 pair, with the Rayleigh quotient of the pencil as the next shift:
// (H - mu G) z = G s by Gaussian elimination with partial pivoting, then
// s = z / ||z||, mu = (s^H H s) / (s^H G s).  Work: m*m + m per target.
__global__ void __launch_bounds__(kT) refine_targets_kernel(const double2* __restrict__ G, const double2* __restrict__ Hm,
                                                            int m, int ld, double2* __restrict__ S, double* __restrict__ mu,
                                                            const int* __restrict__ idx, double2* __restrict__ work,
                                                            int steps) {
    __shared__ double red[33];
    __shared__ int piv_s;
    __shared__ double2 sv[64], zv[64], yv[64];
    const int tid = threadIdx.x;
    const int col = idx[blockIdx.x];
    double2* M = work + (size_t)blockIdx.x * m * m;      // column-major, ld = m
    double2* s = S + (size_t)col * m;
    for (int i = tid; i < m; i += blockDim.x) sv[i] = s[i];
    double shift = mu[col];
    __syncthreads();
    for (int step = 0; step < steps; ++step) {
        // M = H - shift G (Hermitian parts), y = G s
        for (int e = tid; e < m * m; e += blockDim.x) {
            const int i = e % m, j = e / m;
            const double2 g = 0.5 * (G[j * ld + i] + conj(G[i * ld + j]));
            const double2 h = 0.5 * (Hm[j * ld + i] + conj(Hm[i * ld + j]));
            M[e] = h - shift * g;
        }
        for (int i = tid; i < m; i += blockDim.x) {
            double2 acc = make_double2(0, 0);
            for (int j = 0; j < m; ++j) acc += (0.5 * (G[j * ld + i] + conj(G[i * ld + j]))) * sv[j];
            yv[i] = acc;
        }
        __syncthreads();
        // Gaussian elimination with partial pivoting on [M | y]
        for (int k = 0; k < m; ++k) {
            if (tid < 32) {
                double best = -1.0;
                int bi = k;
                for (int i = k + tid; i < m; i += 32) {
                    const double a = M[k * m + i].x * M[k * m + i].x + M[k * m + i].y * M[k * m + i].y;
                    if (a > best) { best = a; bi = i; }
                }
                for (int o = 16; o > 0; o >>= 1) {
                    const double ob = __shfl_xor_sync(0xffffffffu, best, o);
                    const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
                    if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
                }
                if (tid == 0) piv_s = bi;
            }
            __syncthreads();
            const int pr = piv_s;
            if (pr != k) {
                for (int j = k + tid; j < m; j += blockDim.x) {
                    const double2 t = M[j * m + k];
                    M[j * m + k] = M[j * m + pr];
                    M[j * m + pr] = t;
                }
                if (tid == 0) { const double2 t = yv[k]; yv[k] = yv[pr]; yv[pr] = t; }
            }
            __syncthreads();
            double2 d = M[k * m + k];
            double dd = d.x * d.x + d.y * d.y;
            if (!(dd > 1e-300)) { d = make_double2(1e-150, 0.0); dd = 1e-300; }
            const double2 dinv = (1.0 / dd) * conj(d);
            const int rows = m - k - 1;
            for (int e = tid; e < rows * (m - k); e += blockDim.x) {
                const int i = k + 1 + e % rows, j = k + e / rows;
                const double2 f = M[k * m + i] * dinv;
                if (j == k) continue;
                M[j * m + i] -= f * M[j * m + k];
            }
            for (int i = k + 1 + tid; i < m; i += blockDim.x) yv[i] -= (M[k * m + i] * dinv) * yv[k];
            __syncthreads();
        }
        // back substitution
        if (tid == 0) {
            for (int i = m - 1; i >= 0; --i) {
                double2 acc = yv[i];
                for (int j = i + 1; j < m; ++j) acc -= M[j * m + i] * zv[j];
                double2 d = M[i * m + i];
                double dd = d.x * d.x + d.y * d.y;
                if (!(dd > 1e-300)) { d = make_double2(1e-150, 0.0); dd = 1e-300; }
                zv[i] = (1.0 / dd) * (conj(d) * acc);
            }
        }
        __syncthreads();
        double nz = 0.0;
        for (int i = tid; i < m; i += blockDim.x) nz += zv[i].x * zv[i].x + zv[i].y * zv[i].y;
        nz = block_reduce_sum(nz, red);
        const double inz = nz > 0 ? 1.0 / sqrt(nz) : 0.0;
        for (int i = tid; i < m; i += blockDim.x) sv[i] = inz * zv[i];
        __syncthreads();
        // Rayleigh quotient of the pencil
        double hr = 0.0, gr = 0.0;
        for (int i = tid; i < m; i += blockDim.x) {
            double2 hs = make_double2(0, 0), gs = make_double2(0, 0);
            for (int j = 0; j < m; ++j) {
                hs += (0.5 * (Hm[j * ld + i] + conj(Hm[i * ld + j]))) * sv[j];
                gs += (0.5 * (G[j * ld + i] + conj(G[i * ld + j]))) * sv[j];
            }
            hr += cmulc(sv[i], hs).x;
            gr += cmulc(sv[i], gs).x;
        }
        hr = block_reduce_sum(hr, red);
        gr = block_reduce_sum(gr, red);
        shift = gr > 0 ? hr / gr : shift;
    }
    for (int i = tid; i < m; i += blockDim.x) s[i] = sv[i];
    if (tid == 0) mu[col] = shift;
}

// Q = orthonormal basis of the columns of S (m x k): modified Gram-Schmidt, twice.
__global__ void __launch_bounds__(kT) small_qr_kernel(const double2* __restrict__ S, int m, int k, int lds,
                                                      double2* __restrict__ Q) {
    __shared__ double red[33];
    __shared__ double2 hsh;
    const int tid = threadIdx.x;
    for (int e = tid; e < m * k; e += blockDim.x) Q[e] = S[(e / m) * lds + e % m];
    __syncthreads();
    for (int pass = 0; pass < 2; ++pass) {
        for (int j = 0; j < k; ++j) {
            double2* qj = Q + (size_t)j * m;
            for (int i = 0; i < j; ++i) {
                const double2* qi = Q + (size_t)i * m;
                double hr = 0, hi = 0;
                for (int r = tid; r < m; r += blockDim.x) { double2 t = cmulc(qi[r], qj[r]); hr += t.x; hi += t.y; }
                hr = block_reduce_sum(hr, red);
                hi = block_reduce_sum(hi, red);
                if (tid == 0) hsh = make_double2(hr, hi);
                __syncthreads();
                double2 h = hsh;
                for (int r = tid; r < m; r += blockDim.x) qj[r] -= h * qi[r];
                __syncthreads();
            }
            double nn = 0;
            for (int r = tid; r < m; r += blockDim.x) nn += cabs2(qj[r]);
            nn = block_reduce_sum(nn, red);
            double inv = nn > 0 ? 1.0 / sqrt(nn) : 0.0;
            for (int r = tid; r < m; r += blockDim.x) qj[r] = inv * qj[r];
            __syncthreads();
        }
    }
}

// Householder complement of a unit vector s: H = I - 2 w w^H / (w^H w) with
// w = s + e^{i arg s_0} e_0; columns 1..m-1 of H are orthonormal and orthogonal to s.
__global__ void __launch_bounds__(kT) complement_kernel(const double2* __restrict__ s, int m, double2* __restrict__ Cm) {
    __shared__ double red[33];
    const int tid = threadIdx.x;
    double2 s0 = s[0];
    double a0 = sqrt(cabs2(s0));
    double2 ph = a0 > 0 ? (1.0 / a0) * s0 : make_double2(1, 0);
    double nn = 0;
    for (int r = tid; r < m; r += blockDim.x) {
        double2 w = s[r];
        if (r == 0) w += ph;
        nn += cabs2(w);
    }
    nn = block_reduce_sum(nn, red);
    const double f = nn > 0 ? 2.0 / nn : 0.0;
    for (int e = tid; e < m * (m - 1); e += blockDim.x) {
        int i = e % m, j = e / m + 1;
        double2 wi = s[i], wj = s[j];
        if (i == 0) wi += ph;
        if (j == 0) wj += ph;
        double2 v = make_double2(i == j ? 1.0 : 0.0, 0.0) - f * (wi * conj(wj));
        Cm[e] = v;
    }
}

// out (p x p) = C^H M C with M (m x m, ld ldm), C (m x p, ld m); work m*p.
__global__ void __launch_bounds__(kT) gram_transform_kernel(const double2* __restrict__ M, int m, int ldm,
                                                            const double2* __restrict__ C, int p,
                                                            double2* __restrict__ out, int ldo, double2* __restrict__ T) {
    const int tid = threadIdx.x;
    for (int e = tid; e < m * p; e += blockDim.x) {
        int i = e % m, j = e / m;
        double2 s = make_double2(0, 0);
        for (int k = 0; k < m; ++k) s += M[k * ldm + i] * C[j * m + k];
        T[j * m + i] = s;
    }
    __syncthreads();
    for (int e = tid; e < p * p; e += blockDim.x) {
        int i = e % p, j = e / p;
        double2 s = make_double2(0, 0);
        for (int k = 0; k < m; ++k) s += conj(C[i * m + k]) * T[j * m + k];
        out[j * ldo + i] = s;
    }
}
}  // namespace

void small_harmonic_eig(const double2* G, const double2* H, int m, int ld, double* mu, double2* S, double2* work,
                        int* status, cudaStream_t st) {
    KTimer kt("harmonic_eig", 0.0, 0.0, st);
    const size_t sm = (size_t)2 * m * m * sizeof(float2);
    if (sm > 48 * 1024) cudaFuncSetAttribute(harmonic_eig_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    harmonic_eig_kernel<<<1, kTE, sm, st>>>(G, H, m, ld, mu, S, work, status);
}
void small_refine_targets(const double2* G, const double2* H, int m, int ld, double2* S, double* mu, const int* idx,
                          int nb, double2* work, cudaStream_t st) {
    KTimer kt("refine_targets", 0.0, 0.0, st);
    refine_targets_kernel<<<nb, kT, 0, st>>>(G, H, m, ld, S, mu, idx, work, 1);
}
void small_qr(const double2* S, int m, int k, int lds, double2* Q, double2* work, cudaStream_t st) {
    (void)work;
    KTimer kt("small_qr", 0.0, 0.0, st);
    small_qr_kernel<<<1, kT, 0, st>>>(S, m, k, lds, Q);
}
void small_complement(const double2* s, int m, double2* C, double2* work, cudaStream_t st) {
    (void)work;
    KTimer kt("complement", 0.0, 0.0, st);
    complement_kernel<<<1, kT, 0, st>>>(s, m, C);
}
void small_gram_transform(const double2* M, int m, int ldm, const double2* C, int p, double2* out, int ldo,
                          double2* work, cudaStream_t st) {
    KTimer kt("gram_transform", 0.0, 0.0, st);
    gram_transform_kernel<<<1, kT, 0, st>>>(M, m, ldm, C, p, out, ldo, work);
}

}  // namespace qcd
