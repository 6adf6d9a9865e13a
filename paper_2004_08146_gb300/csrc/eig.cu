// Small dense FP64 kernels of the Davidson outer iteration (Sec. 3):
// the harmonic Ritz pencil of Theorem 1 / Eq. 3.5, (W^H V) s = mu (W^H W) s
// with mu = 1/theta, solved as Cholesky W^H W = L L^H, C = L^-1 (W^H V) L^-H
// and a parallel (round-robin) complex Jacobi eigensolver, the FP64
// refinement of the targeted pairs and the QR used for thick restarts.  All
// run in one CTA (per target) on column-major matrices with m <= kMaxBasis.
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

// The pencil is reduced to the Hermitian C = Li H Li^H with Li = L^-1 and
// G = W^H W = L L^H (Cholesky).  `state` keeps, between calls, Li (row-major)
// and C (both FP64, leading dimension ld) and the FP32 eigenvectors Z of C
// (column-major, ld).  Appending basis vectors leaves the leading m0 x m0
// blocks of Li and C unchanged, so only rows m0..m-1 are computed, one row k
// at a time by matrix-vector products (one warp per output entry):
//   l = conj(Li[0:k,0:k] G[0:k,k])           (row k of L left of the diagonal)
//   L[k,k] = sqrt(G[k,k] - ||l||^2)
//   Li[k,j] = -(1/L[k,k]) sum_{j<=q<k} l[q] Li[q,j],  Li[k,k] = 1/L[k,k]
//   C[k,j] = (Li[k,:] H) Li[j,:]^H for j <= k,  C[j,k] = conj(C[k,j]).
// m0 = 0 recomputes everything.  C is then diagonalised by a parallel
// (round-robin) complex Jacobi eigensolver on an FP32 copy in shared memory:
// the decomposition feeds target selection and thick restarts, which need no
// more; the targeted pairs are refined in FP64 afterwards
// (refine_targets_kernel).  With m0 > 0 the sweeps start from the previous
// eigenvectors: in the basis Z0 (+) I the matrix is diag(mu_prev) bordered by
// Z0^H C[0:m0, m0:m] and C[m0:m, m0:m], which a few sweeps finish.  Each
// round applies the disjoint rotations J of its pairs as 2x2 blocks
// J_P^H A[P, Q] J_Q, one thread per block, so a round needs two barriers.
// The sweeps stop once the off-diagonal mass reaches the FP32 round-off
// floor, 4 m^2 u^2 ||C||_F^2 (u = 2^-24), or stops decreasing.  Outputs mu
// (eigenvalues of C, previous values read from mu when m0 > 0), S = Li^H Z
// (the pencil eigenvectors) and Z in `state`.
__global__ void __launch_bounds__(kTE) harmonic_eig_inc_kernel(const double2* __restrict__ G,
                                                              const double2* __restrict__ Hm, int m, int ld, int m0,
                                                              double* __restrict__ mu, double2* __restrict__ S,
                                                              double2* __restrict__ state, int* __restrict__ status) {
    constexpr int kPairs = kMaxBasis / 2 + 1;
    __shared__ double red[33];
    __shared__ int pp[kPairs], qq[kPairs];
    __shared__ float2 pj[kPairs][3];   // per pair: (c, s), e^{i phi}, unused
    __shared__ double2 rowv[kMaxBasis], rowt[kMaxBasis];
    __shared__ double lkk_s;
    extern __shared__ double2 shm[];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarp = blockDim.x >> 5;
    double2* Li = state;                          // row-major: Li[i * ld + j] = Li_ij
    double2* C = state + (size_t)ld * ld;         // Hermitian, both triangles stored
    float2* Zg = reinterpret_cast<float2*>(state + (size_t)2 * ld * ld);   // column-major
    auto Gh = [&](int i, int j) { return 0.5 * (G[(size_t)j * ld + i] + conj(G[(size_t)i * ld + j])); };
    auto Hh = [&](int i, int j) { return 0.5 * (Hm[(size_t)j * ld + i] + conj(Hm[(size_t)i * ld + j])); };
    auto wsum = [&](double2 v) {
        for (int o = 16; o > 0; o >>= 1) {
            v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
            v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
        }
        return v;
    };
    for (int k = m0; k < m; ++k) {
        // l = conj(Li[0:k,0:k] G[0:k,k])
        for (int i = warp; i < k; i += nwarp) {
            double2 acc = make_double2(0, 0);
            for (int l = lane; l <= i; l += 32) acc += Li[(size_t)i * ld + l] * Gh(l, k);
            acc = wsum(acc);
            if (lane == 0) rowv[i] = conj(acc);
        }
        __syncthreads();
        if (warp == 0) {
            double nn = 0.0;
            for (int i = lane; i < k; i += 32) nn += rowv[i].x * rowv[i].x + rowv[i].y * rowv[i].y;
            for (int o = 16; o > 0; o >>= 1) nn += __shfl_xor_sync(0xffffffffu, nn, o);
            if (lane == 0) {
                double d = Gh(k, k).x - nn;
                if (!(d > 0.0)) { status[0] = 1; d = 1e-300; }
                lkk_s = sqrt(d);
            }
        }
        __syncthreads();
        const double ilkk = 1.0 / lkk_s;
        // Li[k, j], j < k
        for (int j = warp; j < k; j += nwarp) {
            double2 acc = make_double2(0, 0);
            for (int l = j + lane; l < k; l += 32) acc += rowv[l] * Li[(size_t)l * ld + j];
            acc = wsum(acc);
            if (lane == 0) {
                Li[(size_t)k * ld + j] = (-ilkk) * acc;
                Li[(size_t)j * ld + k] = make_double2(0, 0);
            }
        }
        if (tid == 0) Li[(size_t)k * ld + k] = make_double2(ilkk, 0);
        __syncthreads();
        // t = Li[k,:] H
        for (int b = warp; b <= k; b += nwarp) {
            double2 acc = make_double2(0, 0);
            for (int a = lane; a <= k; a += 32) acc += Li[(size_t)k * ld + a] * Hh(a, b);
            acc = wsum(acc);
            if (lane == 0) rowt[b] = acc;
        }
        __syncthreads();
        // C[k, j] = t . conj(Li[j, :]), j <= k
        for (int j = warp; j <= k; j += nwarp) {
            double2 acc = make_double2(0, 0);
            for (int b = lane; b <= j; b += 32) acc += rowt[b] * conj(Li[(size_t)j * ld + b]);
            acc = wsum(acc);
            if (lane == 0) {
                if (j == k) acc.y = 0.0;
                C[(size_t)j * ld + k] = acc;
                C[(size_t)k * ld + j] = conj(acc);
            }
        }
        __syncthreads();
    }
    float2* Af = reinterpret_cast<float2*>(shm);   // m x m, column-major
    float2* Zf = Af + m * m;
#define IDX(i, j) ((j) * m + (i))
    const bool warm = m0 > 0;
    if (warm) {
        // A = (Z0 (+) I)^H C (Z0 (+) I) with its leading block taken as diag(mu_prev)
        for (int e = tid; e < m * m; e += blockDim.x) {
            const int i = e % m, j = e / m;
            Zf[e] = (i < m0 && j < m0) ? Zg[(size_t)j * ld + i] : make_float2(i == j ? 1.f : 0.f, 0.f);
            if (i < m0 && j < m0) Af[e] = make_float2(i == j ? (float)mu[i] : 0.f, 0.f);
            else if (i >= m0 && j >= m0) Af[e] = make_float2((float)C[(size_t)j * ld + i].x, (float)C[(size_t)j * ld + i].y);
        }
        __syncthreads();
        for (int e = tid; e < m0 * (m - m0); e += blockDim.x) {
            const int i = e % m0, j = m0 + e / m0;
            float2 acc = make_float2(0.f, 0.f);
            for (int q = 0; q < m0; ++q) {
                const float2 z = Zf[IDX(q, i)];
                const double2 c = C[(size_t)j * ld + q];
                acc += make_float2(z.x, -z.y) * make_float2((float)c.x, (float)c.y);
            }
            Af[IDX(i, j)] = acc;
            Af[IDX(j, i)] = make_float2(acc.x, -acc.y);
        }
    } else {
        for (int e = tid; e < m * m; e += blockDim.x) {
            const int i = e % m, j = e / m;
            const double2 c = C[(size_t)j * ld + i];
            Af[e] = make_float2((float)c.x, (float)c.y);
            Zf[e] = make_float2(i == j ? 1.f : 0.f, 0.f);
        }
    }
    __syncthreads();
    const int mm = (m % 2) ? m + 1 : m;   // players, padded with the empty index m
    const int npair = mm / 2;
    float fro = 0.0f;
    for (int e = tid; e < m * m; e += blockDim.x) fro += Af[e].x * Af[e].x + Af[e].y * Af[e].y;
    fro = (float)block_reduce_sum((double)fro, red);
    const float floor_off = 4.0f * (float)(m * m) * 3.5527137e-15f * fro;   // 4 m^2 (2^-24)^2 ||C||^2
    float prev_off = 3.0e38f;
    for (int sweep = 0; sweep < 40 && m > 1; ++sweep) {
        float off = 0.0f;
        for (int e = tid; e < m * m; e += blockDim.x)
            if (e % m != e / m) off += Af[e].x * Af[e].x + Af[e].y * Af[e].y;
        off = (float)block_reduce_sum((double)off, red);
        if (off <= floor_off || off >= prev_off) break;
        prev_off = off;
        for (int rnd = 0; rnd < mm - 1; ++rnd) {
            if (tid < npair) {
                auto player = [&](int pos) { return pos == 0 ? 0 : ((rnd + pos - 1) % (mm - 1)) + 1; };
                int p = player(tid), q = player(mm - 1 - tid);
                if (p > q) { int t = p; p = q; q = t; }
                float c = 1.f, sv = 0.f;
                float2 ph = make_float2(1.f, 0.f);
                if (q < m) {
                    const float2 b = Af[IDX(p, q)];
                    const float ab = sqrtf(b.x * b.x + b.y * b.y);
                    if (ab > 1e-30f) {
                        ph = make_float2(b.x / ab, b.y / ab);
                        const float zeta = (Af[IDX(q, q)].x - Af[IDX(p, p)].x) / (2.0f * ab);
                        const float t = (zeta >= 0 ? 1.0f : -1.0f) / (fabsf(zeta) + sqrtf(1.0f + zeta * zeta));
                        c = rsqrtf(1.0f + t * t);
                        sv = t * c;
                    }
                }
                pp[tid] = p; qq[tid] = q;
                pj[tid][0] = make_float2(c, sv);
                pj[tid][1] = ph;
            }
            __syncthreads();
            // J = [[c, s], [-s conj(ph), c conj(ph)]] on columns (p, q); rows get J^H
            for (int e = tid; e < npair * npair; e += blockDim.x) {
                const int P = e % npair, Q = e / npair;
                const int p1 = pp[P], q1 = qq[P], p2 = pp[Q], q2 = qq[Q];
                const bool v1 = q1 < m, v2 = q2 < m;
                const float2 cs1 = pj[P][0], e1 = pj[P][1], cs2 = pj[Q][0], e2 = pj[Q][1];
                const float2 a00 = Af[IDX(p1, p2)];
                const float2 a01 = v2 ? Af[IDX(p1, q2)] : make_float2(0.f, 0.f);
                const float2 a10 = v1 ? Af[IDX(q1, p2)] : make_float2(0.f, 0.f);
                const float2 a11 = (v1 && v2) ? Af[IDX(q1, q2)] : make_float2(0.f, 0.f);
                // columns: T = A J_Q
                const float2 f2 = make_float2(e2.x, -e2.y);   // conj(ph_Q)
                const float2 t00 = cs2.x * a00 - cs2.y * (f2 * a01), t01 = cs2.y * a00 + cs2.x * (f2 * a01);
                const float2 t10 = cs2.x * a10 - cs2.y * (f2 * a11), t11 = cs2.y * a10 + cs2.x * (f2 * a11);
                // rows: J_P^H T
                Af[IDX(p1, p2)] = cs1.x * t00 - cs1.y * (e1 * t10);
                if (v2) Af[IDX(p1, q2)] = cs1.x * t01 - cs1.y * (e1 * t11);
                if (v1) Af[IDX(q1, p2)] = cs1.y * t00 + cs1.x * (e1 * t10);
                if (v1 && v2) Af[IDX(q1, q2)] = cs1.y * t01 + cs1.x * (e1 * t11);
            }
            for (int e = tid; e < npair * m; e += blockDim.x) {
                const int r = e % m, Q = e / m;
                const int p = pp[Q], q = qq[Q];
                if (q >= m) continue;
                const float2 cs = pj[Q][0], ph = pj[Q][1];
                const float2 em = make_float2(ph.x, -ph.y);
                const float2 zp = Zf[IDX(r, p)], zq = Zf[IDX(r, q)];
                Zf[IDX(r, p)] = cs.x * zp - cs.y * (em * zq);
                Zf[IDX(r, q)] = cs.y * zp + cs.x * (em * zq);
            }
            __syncthreads();
        }
    }
    for (int i = tid; i < m; i += blockDim.x) mu[i] = (double)Af[IDX(i, i)].x;
    for (int e = tid; e < m * m; e += blockDim.x) Zg[(size_t)(e / m) * ld + (e % m)] = Zf[e];
    __syncthreads();
    // S = Li^H Z (upper-triangular Li^H) in FP32, Li staged in shared memory
    for (int e = tid; e < m * m; e += blockDim.x) {
        const int i = e / m, j = e % m;   // Li_ij, i >= j
        const double2 l = i >= j ? Li[(size_t)i * ld + j] : make_double2(0, 0);
        Af[IDX(i, j)] = make_float2((float)l.x, (float)l.y);
    }
    __syncthreads();
    for (int e = tid; e < m * m; e += blockDim.x) {
        const int i = e % m, j = e / m;
        float2 sacc = make_float2(0.f, 0.f);
        for (int k = i; k < m; ++k) {
            const float2 l = Af[IDX(k, i)];
            sacc += make_float2(l.x, -l.y) * Zf[IDX(k, j)];
        }
        S[IDX(i, j)] = make_double2(sacc.x, sacc.y);
    }
#undef IDX
}

// FP64 refinement of targeted harmonic Ritz pairs (one CTA per target).
// With C = Li H Li^H in FP64 and its FP32 eigenvectors Z (both left by
// harmonic_eig_inc_kernel), the target column z of Z is improved by
// first-order perturbation in the eigenbasis:
//   rho = z^H C z,  r = C z - rho z  (FP64),
//   z <- z - sum_{j != col} Z_j (Z_j^H r) / (mu_j - rho),  normalised,
// each step cutting the error by about the FP32 accuracy of Z; directions
// with |mu_j - rho| below 1e-6 max|mu| (an unresolved cluster) are left out.
// Then s = Li^H z (FP64) replaces column idx[b] of S and rho goes to
// mu_out[b] (mu itself is only read, so the CTAs do not race on it).
constexpr int kRefineThreads = 128;   // >= kMaxBasis
static_assert(kRefineThreads >= kMaxBasis, "one thread per pencil row");
__global__ void __launch_bounds__(kRefineThreads) refine_targets_kernel(const double2* __restrict__ state, int m, int ld,
                                                            double2* __restrict__ S, const double* __restrict__ mu,
                                                            double* __restrict__ mu_out, const int* __restrict__ idx,
                                                            int steps) {
    __shared__ double red[33];
    __shared__ double2 zv[kRefineThreads], rv[kRefineThreads];
    __shared__ float2 cf[kRefineThreads];
    __shared__ double muv[kRefineThreads];
    const int tid = threadIdx.x;   // one thread per row, m <= kRefineThreads
    const int col = idx[blockIdx.x];
    const double2* Li = state;
    const double2* C = state + (size_t)ld * ld;
    const float2* Z = reinterpret_cast<const float2*>(state + (size_t)2 * ld * ld);
    const bool row = tid < m;
    double amax = 0.0;
    if (row) {
        const float2 z = Z[(size_t)col * ld + tid];
        zv[tid] = make_double2(z.x, z.y);
        muv[tid] = mu[tid];
        amax = fabs(mu[tid]);
    }
    double nz = row ? cabs2(zv[tid]) : 0.0;
    nz = block_reduce_sum(nz, red);
    if (row) zv[tid] = (1.0 / sqrt(nz)) * zv[tid];
    // max |mu| (block_reduce_sum pattern with max)
    for (int o = 16; o > 0; o >>= 1) amax = fmax(amax, __shfl_xor_sync(0xffffffffu, amax, o));
    if ((tid & 31) == 0) red[tid >> 5] = amax;
    __syncthreads();
    amax = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) amax = fmax(amax, red[w]);
    __syncthreads();
    const double gap_min = 1e-6 * amax;
    double rho = 0.0;
    for (int step = 0; step <= steps; ++step) {
        double2 cz = make_double2(0, 0);
        if (row)
            for (int j = 0; j < m; ++j) cz += C[(size_t)j * ld + tid] * zv[j];
        double pr = row ? cmulc(zv[tid], cz).x : 0.0;
        rho = block_reduce_sum(pr, red);
        if (step == steps) break;
        if (row) rv[tid] = cz - rho * zv[tid];
        __syncthreads();
        // coefficients Z_j^H r / (mu_j - rho), FP32 (r is already small)
        if (row) {
            float2 acc = make_float2(0.f, 0.f);
            const float2* zj = Z + (size_t)tid * ld;
            for (int i = 0; i < m; ++i) {
                const float2 a = zj[i];
                const float2 b = make_float2((float)rv[i].x, (float)rv[i].y);
                acc += make_float2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
            }
            const double d = muv[tid] - rho;
            cf[tid] = (tid == col || fabs(d) < gap_min) ? make_float2(0.f, 0.f) : (float)(1.0 / d) * acc;
        }
        __syncthreads();
        if (row) {
            float2 dz = make_float2(0.f, 0.f);
            for (int j = 0; j < m; ++j) dz += Z[(size_t)j * ld + tid] * cf[j];
            zv[tid] -= make_double2(dz.x, dz.y);
        }
        __syncthreads();
        nz = row ? cabs2(zv[tid]) : 0.0;
        nz = block_reduce_sum(nz, red);
        if (row) zv[tid] = (1.0 / sqrt(nz)) * zv[tid];
        __syncthreads();
    }
    // s = Li^H z
    if (row) {
        double2 acc = make_double2(0, 0);
        for (int k = tid; k < m; ++k) acc += conj(Li[(size_t)k * ld + tid]) * zv[k];
        S[(size_t)col * m + tid] = acc;
    }
    if (tid == 0) mu_out[blockIdx.x] = rho;
}

// Q = orthonormal basis of the columns of S (m x k <= kMaxBasis): column by column,
// classical Gram-Schmidt twice against the previous columns (all inner
// products of a pass at once, one warp each), then normalisation.
__global__ void __launch_bounds__(kT) small_qr_kernel(const double2* __restrict__ S, int m, int k, int lds,
                                                      double2* __restrict__ Q) {
    __shared__ double red[33];
    __shared__ double2 h[kMaxBasis];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarp = blockDim.x >> 5;
    for (int e = tid; e < m * k; e += blockDim.x) Q[e] = S[(e / m) * lds + e % m];
    __syncthreads();
    for (int j = 0; j < k; ++j) {
        double2* qj = Q + (size_t)j * m;
        for (int pass = 0; pass < 2 && j > 0; ++pass) {
            // h_i = q_i^H q_j for all i < j at once, one warp per i
            for (int i = warp; i < j; i += nwarp) {
                const double2* qi = Q + (size_t)i * m;
                double2 acc = make_double2(0, 0);
                for (int r = lane; r < m; r += 32) acc += cmulc(qi[r], qj[r]);
                for (int o = 16; o > 0; o >>= 1) {
                    acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
                    acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
                }
                if (lane == 0) h[i] = acc;
            }
            __syncthreads();
            for (int r = tid; r < m; r += blockDim.x) {
                double2 v = qj[r];
                for (int i = 0; i < j; ++i) v -= h[i] * Q[(size_t)i * m + r];
                qj[r] = v;
            }
            __syncthreads();
        }
        double nn = 0;
        for (int r = tid; r < m; r += blockDim.x) nn += cabs2(qj[r]);
        nn = block_reduce_sum(nn, red);
        const double inv = nn > 0 ? 1.0 / sqrt(nn) : 0.0;
        for (int r = tid; r < m; r += blockDim.x) qj[r] = inv * qj[r];
        __syncthreads();
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

void small_harmonic_eig_inc(const double2* G, const double2* H, int m, int ld, int m0, double* mu, double2* S,
                            double2* state, int* status, cudaStream_t st) {
    KTimer kt(m0 == 0 ? "harmonic_eig_full" : "harmonic_eig_inc", 0.0, 0.0, st);
    const size_t sm = (size_t)2 * m * m * sizeof(float2);
    if (sm + 1024 > 48 * 1024) cudaFuncSetAttribute(harmonic_eig_inc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    harmonic_eig_inc_kernel<<<1, kTE, sm, st>>>(G, H, m, ld, m0, mu, S, state, status);
}
void small_refine_targets(const double2* state, int m, int ld, double2* S, const double* mu, double* mu_out,
                          const int* idx, int nb, cudaStream_t st) {
    KTimer kt("refine_targets", 0.0, 0.0, st);
    refine_targets_kernel<<<nb, kRefineThreads, 0, st>>>(state, m, ld, S, mu, mu_out, idx, 3);
}
void small_qr(const double2* S, int m, int k, int lds, double2* Q, double2* work, cudaStream_t st) {
    (void)work;
    KTimer kt("small_qr", 0.0, 0.0, st);
    small_qr_kernel<<<1, kT, 0, st>>>(S, m, k, lds, Q);
}
void small_gram_transform(const double2* M, int m, int ldm, const double2* C, int p, double2* out, int ldo,
                          double2* work, cudaStream_t st) {
    KTimer kt("gram_transform", 0.0, 0.0, st);
    gram_transform_kernel<<<1, kT, 0, st>>>(M, m, ldm, C, p, out, ldo, work);
}

}  // namespace qcd
