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

// work layout: L[m*m], Li[m*m], T[m*m] in global memory; C and Z (the Jacobi
// working matrix and its accumulated rotations) in 2*m*m double2 of shared
// memory (column-major, ld = m)
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
    double2* C = shm;            // working matrix and eigenvectors in shared memory
    double2* Z = shm + m * m;
#define IDX(i, j) ((j) * m + (i))
    for (int e = tid; e < m * m; e += blockDim.x) {
        int i = e % m, j = e / m;
        // Hermitian parts (symmetrise against round-off)
        double2 g = 0.5 * (G[j * ld + i] + conj(G[i * ld + j]));
        double2 h = 0.5 * (Hm[j * ld + i] + conj(Hm[i * ld + j]));
        L[IDX(i, j)] = g;
        C[IDX(i, j)] = h;
        Li[IDX(i, j)] = make_double2(i == j ? 1.0 : 0.0, 0.0);
        Z[IDX(i, j)] = make_double2(i == j ? 1.0 : 0.0, 0.0);
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
    // parallel cyclic Jacobi on the Hermitian C, round-robin pairs
    const int mm = (m % 2) ? m + 1 : m;   // padded player count
    const int npair = mm / 2;
    double fro = 0.0;
    for (int e = tid; e < m * m; e += blockDim.x) fro += cabs2(C[e]);
    fro = block_reduce_sum(fro, red);
    for (int sweep = 0; sweep < 60; ++sweep) {
        double off = 0.0;
        for (int e = tid; e < m * m; e += blockDim.x) if (e % m != e / m) off += cabs2(C[e]);
        off = block_reduce_sum(off, red);
        // stop at an off-diagonal norm of 1e-14 relative: the FP64 round-off
        // floor of m^2 entries sits near (m eps)^2 ~ 1e-28, so a stricter test
        // would never pass and would run every sweep
        if (off <= 1e-28 * fro || m < 2) break;
        for (int rnd = 0; rnd < mm - 1; ++rnd) {
            if (tid < npair) {
                int k = tid;
                auto player = [&](int pos) { return pos == 0 ? 0 : ((rnd + pos - 1) % (mm - 1)) + 1; };
                int p = player(k), q = player(mm - 1 - k);
                if (p > q) { int t = p; p = q; q = t; }
                double c = 1.0, s = 0.0;
                double2 ph = make_double2(1, 0);
                if (q < m) {
                    double2 b = C[IDX(p, q)];
                    double ab = sqrt(cabs2(b));
                    if (ab > 1e-300) {
                        ph = (1.0 / ab) * b;
                        double a = C[IDX(p, p)].x, d = C[IDX(q, q)].x;
                        double zeta = (d - a) / (2.0 * ab);
                        double t = (zeta >= 0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
                        c = 1.0 / sqrt(1.0 + t * t);
                        s = t * c;
                    }
                }
                pp[k] = p; qq[k] = q; pc[k] = c; ps[k] = s; pph[k] = ph;
            }
            __syncthreads();
            // columns: A <- A J, Z <- Z J ; J_pp = c, J_pq = s, J_qp = -s e^{-i phi}, J_qq = c e^{-i phi}
            for (int e = tid; e < npair * m; e += blockDim.x) {
                int k = e / m, r = e % m;
                int p = pp[k], q = qq[k];
                if (q >= m) continue;
                double c = pc[k], s = ps[k];
                double2 em = conj(pph[k]);
                double2 ap = C[IDX(r, p)], aq = C[IDX(r, q)];
                C[IDX(r, p)] = c * ap - s * (em * aq);
                C[IDX(r, q)] = s * ap + c * (em * aq);
                double2 zp = Z[IDX(r, p)], zq = Z[IDX(r, q)];
                Z[IDX(r, p)] = c * zp - s * (em * zq);
                Z[IDX(r, q)] = s * zp + c * (em * zq);
            }
            __syncthreads();
            // rows: A <- J^H A
            for (int e = tid; e < npair * m; e += blockDim.x) {
                int k = e / m, col = e % m;
                int p = pp[k], q = qq[k];
                if (q >= m) continue;
                double c = pc[k], s = ps[k];
                double2 ep = pph[k];
                double2 ap = C[IDX(p, col)], aq = C[IDX(q, col)];
                C[IDX(p, col)] = c * ap - s * (ep * aq);
                C[IDX(q, col)] = s * ap + c * (ep * aq);
            }
            __syncthreads();
        }
    }
    for (int i = tid; i < m; i += blockDim.x) mu[i] = C[IDX(i, i)].x;
    // S = Li^H Z  (upper-triangular Li^H)
    for (int e = tid; e < m * m; e += blockDim.x) {
        int i = e % m, j = e / m;
        double2 s = make_double2(0, 0);
        for (int k = i; k < m; ++k) s += conj(Li[IDX(k, i)]) * Z[IDX(k, j)];
        S[IDX(i, j)] = s;
    }
#undef IDX
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
    const size_t sm = (size_t)2 * m * m * sizeof(double2);
    if (sm > 48 * 1024) cudaFuncSetAttribute(harmonic_eig_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    harmonic_eig_kernel<<<1, kTE, sm, st>>>(G, H, m, ld, mu, S, work, status);
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
