// Fine-lattice operator kernels: clover construction (Sec. 4, Table 1 clover
// term; Sheikholeslami-Wohlert) and the Wilson-clover stencil of Eq. 2.5 in
// the shifted forms D - tau Gamma5 (Eq. 3.7) and Q - tau (Eq. 3.6).
#include <algorithm>
#include <cstring>

#include "internal.h"
#include "dirac.cuh"

namespace qcd {

// ------------------------------------------------------------------ SU(3) helpers
template <typename R> struct M3 { cplx<R> e[3][3]; };
__device__ __forceinline__ M3<double> m3_load(const double2* p) {
    M3<double> m;
    for (int a = 0; a < 3; ++a) for (int b = 0; b < 3; ++b) m.e[a][b] = p[a * 3 + b];
    return m;
}
__device__ __forceinline__ M3<double> m3_mul(const M3<double>& x, const M3<double>& y) {
    M3<double> r;
    for (int a = 0; a < 3; ++a) for (int b = 0; b < 3; ++b) {
        double2 s = make_double2(0, 0);
        for (int c = 0; c < 3; ++c) s += x.e[a][c] * y.e[c][b];
        r.e[a][b] = s;
    }
    return r;
}
__device__ __forceinline__ M3<double> m3_dag(const M3<double>& x) {
    M3<double> r;
    for (int a = 0; a < 3; ++a) for (int b = 0; b < 3; ++b) r.e[a][b] = conj(x.e[b][a]);
    return r;
}

__device__ __forceinline__ int shifted(const Geom& g, const int x[4], int mu, int dmu, int nu, int dnu) {
    int y[4] = {x[0], x[1], x[2], x[3]};
    y[mu] = (y[mu] + dmu + g.L[mu]) % g.L[mu];
    y[nu] = (y[nu] + dnu + g.L[nu]) % g.L[nu];
    return site_index(g, y);
}

// sigma^chi_{mu nu} (2x2, chirality block chi) = (i/2)(B_mu B_nu^H - B_nu B_mu^H)
// for chi = 0 and (i/2)(B_mu^H B_nu - B_nu^H B_mu) for chi = 1.
__device__ void spin_block_dense(int mu, bool herm, double2 M[2][2]) {
    SpinMono m = herm ? kBH(mu) : kB(mu);
    for (int r = 0; r < 2; ++r) for (int c = 0; c < 2; ++c) M[r][c] = make_double2(0, 0);
    for (int r = 0; r < 2; ++r) M[r][m.perm[r]] = mul_ipow(make_double2(1, 0), m.ph[r]);
}
__device__ void sigma_block(int mu, int nu, int chi, double2 S[2][2]) {
    double2 A[2][2], Bh[2][2], Bn[2][2], Ah[2][2];
    // chi = 0: X_mu = B_mu, Y_nu = B_nu^H ; chi = 1: X_mu = B_mu^H, Y_nu = B_nu
    spin_block_dense(mu, chi == 1, A);
    spin_block_dense(nu, chi == 0, Bh);
    spin_block_dense(nu, chi == 1, Bn);
    spin_block_dense(mu, chi == 0, Ah);
    for (int r = 0; r < 2; ++r) for (int c = 0; c < 2; ++c) {
        double2 s = make_double2(0, 0);
        for (int k = 0; k < 2; ++k) s += A[r][k] * Bh[k][c] - Bn[r][k] * Ah[k][c];
        S[r][c] = mul_ipow(0.5 * s, 1);
    }
}

// One thread per site: the packed blocks A_chi = (m0 + 4) + C_chi with
// C = c_sw (i/2) sum_{mu<nu} sigma_{mu nu} (x) F_{mu nu},
// F_{mu nu} = (Q_{mu nu} - Q_{mu nu}^H)/8 from the four plaquette leaves.
__global__ void clover_build_kernel(const double2* __restrict__ U, Geom g, double m0, double csw,
                                    double* __restrict__ A64, float* __restrict__ A32) {
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= g.V) return;
    int x[4];
    site_coords(g, s, x);
    double2 C[2][6][6];
    for (int chi = 0; chi < 2; ++chi)
        for (int i = 0; i < 6; ++i) for (int j = 0; j < 6; ++j) C[chi][i][j] = make_double2(0, 0);
    if (csw != 0.0) {
        for (int mu = 0; mu < 4; ++mu) {
            for (int nu = mu + 1; nu < 4; ++nu) {
                auto L = [&](int site, int d) { return m3_load(U + ((size_t)site * 4 + d) * 9); };
                M3<double> Umu = L(s, mu), Unu = L(s, nu);
                M3<double> Umu_m = L(shifted(g, x, mu, -1, nu, 0), mu);
                M3<double> Unu_m = L(shifted(g, x, mu, 0, nu, -1), nu);
                M3<double> l1 = m3_mul(m3_mul(Umu, L(shifted(g, x, mu, 1, nu, 0), nu)),
                                       m3_mul(m3_dag(L(shifted(g, x, mu, 0, nu, 1), mu)), m3_dag(Unu)));
                M3<double> l2 = m3_mul(m3_mul(Unu, m3_dag(L(shifted(g, x, mu, -1, nu, 1), mu))),
                                       m3_mul(m3_dag(L(shifted(g, x, mu, -1, nu, 0), nu)), Umu_m));
                M3<double> l3 = m3_mul(m3_mul(m3_dag(Umu_m), m3_dag(L(shifted(g, x, mu, -1, nu, -1), nu))),
                                       m3_mul(L(shifted(g, x, mu, -1, nu, -1), mu), Unu_m));
                M3<double> l4 = m3_mul(m3_mul(m3_dag(Unu_m), L(shifted(g, x, mu, 0, nu, -1), mu)),
                                       m3_mul(L(shifted(g, x, mu, 1, nu, -1), nu), m3_dag(Umu)));
                double2 F[3][3];
                for (int a = 0; a < 3; ++a) for (int b = 0; b < 3; ++b) {
                    double2 q = l1.e[a][b] + l2.e[a][b] + l3.e[a][b] + l4.e[a][b];
                    double2 qh = conj(l1.e[b][a] + l2.e[b][a] + l3.e[b][a] + l4.e[b][a]);
                    F[a][b] = 0.125 * (q - qh);
                }
                for (int chi = 0; chi < 2; ++chi) {
                    double2 S[2][2];
                    sigma_block(mu, nu, chi, S);
                    for (int si = 0; si < 2; ++si) for (int sj = 0; sj < 2; ++sj)
                        for (int a = 0; a < 3; ++a) for (int b = 0; b < 3; ++b)
                            C[chi][si * 3 + a][sj * 3 + b] += S[si][sj] * F[a][b];
                }
            }
        }
    }
    // scale by c_sw * i/2 and add the diagonal m0 + 4
    for (int chi = 0; chi < 2; ++chi) {
        double* out = A64 + (size_t)s * 72 + 36 * chi;
        float* out32 = A32 + (size_t)s * 72 + 36 * chi;
        for (int i = 0; i < 6; ++i) {
            double2 d = mul_ipow(0.5 * csw * C[chi][i][i], 1);
            out[i] = m0 + 4.0 + d.x;
        }
        for (int i = 0; i < 6; ++i) for (int j = i + 1; j < 6; ++j) {
            double2 v = mul_ipow(0.5 * csw * C[chi][i][j], 1);
            int o = herm_off(i, j);
            out[o] = v.x;
            out[o + 1] = v.y;
        }
        for (int k = 0; k < 36; ++k) out32[k] = (float)out[k];
    }
}

// ------------------------------------------------------------------ derivative along a link direction
// Links move as U_mu(x) -> exp(i eps X_mu(x)) U_mu(x) (X traceless Hermitian),
// so dU/deps = i X U.  The operator is linear in the links of its hop terms, so
// their derivative is the stencil with dU; the clover leaves are four-link
// products, differentiated factor by factor below.
__global__ void link_tangent_kernel(const double2* __restrict__ U, const double2* __restrict__ X,
                                    double2* __restrict__ dU, int V) {
    const size_t nl = (size_t)V * 4;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < nl; e += (size_t)gridDim.x * blockDim.x) {
        const double2* u = U + e * 9;
        const double2* x = X + e * 9;
        for (int a = 0; a < 3; ++a)
            for (int c = 0; c < 3; ++c) {
                double2 acc = make_double2(0, 0);
                for (int b = 0; b < 3; ++b) acc += x[a * 3 + b] * u[b * 3 + c];
                dU[e * 9 + a * 3 + c] = make_double2(-acc.y, acc.x);   // i * acc
            }
    }
}

struct M3T { M3<double> m, d; };   // a matrix and its derivative
__device__ __forceinline__ M3T m3t_mul(const M3T& x, const M3T& y) {
    M3T r;
    r.m = m3_mul(x.m, y.m);
    const M3<double> a = m3_mul(x.d, y.m), b = m3_mul(x.m, y.d);
    for (int i = 0; i < 3; ++i) for (int j = 0; j < 3; ++j) r.d.e[i][j] = a.e[i][j] + b.e[i][j];
    return r;
}
__device__ __forceinline__ M3T m3t_dag(const M3T& x) { return M3T{m3_dag(x.m), m3_dag(x.d)}; }

// Packed derivative of the clover blocks (no constant diagonal), same layout
// and conventions as clover_build_kernel.
__global__ void clover_tangent_kernel(const double2* __restrict__ U, const double2* __restrict__ dU, Geom g,
                                      double csw, double* __restrict__ dA) {
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= g.V) return;
    int x[4];
    site_coords(g, s, x);
    double2 C[2][6][6];
    for (int chi = 0; chi < 2; ++chi)
        for (int i = 0; i < 6; ++i) for (int j = 0; j < 6; ++j) C[chi][i][j] = make_double2(0, 0);
    if (csw != 0.0) {
        for (int mu = 0; mu < 4; ++mu) {
            for (int nu = mu + 1; nu < 4; ++nu) {
                auto L = [&](int site, int d) {
                    return M3T{m3_load(U + ((size_t)site * 4 + d) * 9), m3_load(dU + ((size_t)site * 4 + d) * 9)};
                };
                const M3T Umu = L(s, mu), Unu = L(s, nu);
                const M3T Umu_m = L(shifted(g, x, mu, -1, nu, 0), mu);
                const M3T Unu_m = L(shifted(g, x, mu, 0, nu, -1), nu);
                const M3T l1 = m3t_mul(m3t_mul(Umu, L(shifted(g, x, mu, 1, nu, 0), nu)),
                                       m3t_mul(m3t_dag(L(shifted(g, x, mu, 0, nu, 1), mu)), m3t_dag(Unu)));
                const M3T l2 = m3t_mul(m3t_mul(Unu, m3t_dag(L(shifted(g, x, mu, -1, nu, 1), mu))),
                                       m3t_mul(m3t_dag(L(shifted(g, x, mu, -1, nu, 0), nu)), Umu_m));
                const M3T l3 = m3t_mul(m3t_mul(m3t_dag(Umu_m), m3t_dag(L(shifted(g, x, mu, -1, nu, -1), nu))),
                                       m3t_mul(L(shifted(g, x, mu, -1, nu, -1), mu), Unu_m));
                const M3T l4 = m3t_mul(m3t_mul(m3t_dag(Unu_m), L(shifted(g, x, mu, 0, nu, -1), mu)),
                                       m3t_mul(L(shifted(g, x, mu, 1, nu, -1), nu), m3t_dag(Umu)));
                double2 F[3][3];
                for (int a = 0; a < 3; ++a) for (int b = 0; b < 3; ++b) {
                    const double2 q = l1.d.e[a][b] + l2.d.e[a][b] + l3.d.e[a][b] + l4.d.e[a][b];
                    const double2 qh = conj(l1.d.e[b][a] + l2.d.e[b][a] + l3.d.e[b][a] + l4.d.e[b][a]);
                    F[a][b] = 0.125 * (q - qh);
                }
                for (int chi = 0; chi < 2; ++chi) {
                    double2 S[2][2];
                    sigma_block(mu, nu, chi, S);
                    for (int si = 0; si < 2; ++si) for (int sj = 0; sj < 2; ++sj)
                        for (int a = 0; a < 3; ++a) for (int b = 0; b < 3; ++b)
                            C[chi][si * 3 + a][sj * 3 + b] += S[si][sj] * F[a][b];
                }
            }
        }
    }
    for (int chi = 0; chi < 2; ++chi) {
        double* out = dA + (size_t)s * 72 + 36 * chi;
        for (int i = 0; i < 6; ++i) out[i] = mul_ipow(0.5 * csw * C[chi][i][i], 1).x;
        for (int i = 0; i < 6; ++i) for (int j = i + 1; j < 6; ++j) {
            const double2 v = mul_ipow(0.5 * csw * C[chi][i][j], 1);
            const int o = herm_off(i, j);
            out[o] = v.x;
            out[o + 1] = v.y;
        }
    }
}

// ------------------------------------------------------------------ force: the derivative per link
// F_rho(y) traceless Hermitian with d lambda / d eps = sum tr(X_rho(y) F_rho(y))
// for every direction field X (links moving as exp(i eps X) U).  With w =
// Gamma5 v, the hop terms give K = -i U A with the colour outer product
// A = sum_s ((1 - gamma_rho) v(y + rho))_s w_s(y)^H (the backward hop is its
// complex conjugate), and the clover term gives, per plane (rho, nu),
// (c_sw / 16) (below - above): the plaquettes above and below the link with the
// insertion Bt = B + B^H, B = sum_st sigma_{rho nu, st} v_t w_s^H, placed at
// each corner.  F is the traceless Hermitian part of K over v^H v.

__device__ __forceinline__ int plane_index(int mu, int nu) {   // mu < nu
    return mu == 0 ? nu - 1 : (mu == 1 ? nu + 1 : 5);
}

// Bt_{mu nu}(x) = B + B^H for the six planes mu < nu: [site][plane][3][3],
// B = sum_{st} sigma_st psi_t(x) (Gamma5 gv)_s(x)^H.  sigma is block diagonal
// in chirality and Gamma5 gv = +gv (spins 0, 1), -gv (spins 2, 3).
__global__ void clover_insertion_kernel(const double2* __restrict__ psi, const double2* __restrict__ gv, Geom g,
                                        double2* __restrict__ Bt) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= g.V) return;
    double2 p[12], q[12];
    for (int k = 0; k < 12; ++k) {
        p[k] = psi[(size_t)s * 12 + k];
        q[k] = gv[(size_t)s * 12 + k];
    }
    for (int mu = 0; mu < 4; ++mu)
        for (int nu = mu + 1; nu < 4; ++nu) {
            double2 B[3][3];
            for (int a = 0; a < 3; ++a) for (int b = 0; b < 3; ++b) B[a][b] = make_double2(0, 0);
            for (int chi = 0; chi < 2; ++chi) {
                double2 S[2][2];
                sigma_block(mu, nu, chi, S);
                const double sg = chi == 0 ? 1.0 : -1.0;
                for (int i = 0; i < 2; ++i) for (int j = 0; j < 2; ++j) {
                    const double2 c = sg * S[i][j];
                    for (int a = 0; a < 3; ++a) for (int b = 0; b < 3; ++b)
                        B[a][b] += c * (p[(2 * chi + j) * 3 + a] * conj(q[(2 * chi + i) * 3 + b]));
                }
            }
            double2* o = Bt + ((size_t)s * 6 + plane_index(mu, nu)) * 9;
            for (int a = 0; a < 3; ++a) for (int b = 0; b < 3; ++b) o[a * 3 + b] = B[a][b] + conj(B[b][a]);
        }
}

__device__ __forceinline__ M3<double> m3_add(const M3<double>& x, const M3<double>& y) {
    M3<double> r;
    for (int a = 0; a < 3; ++a) for (int b = 0; b < 3; ++b) r.e[a][b] = x.e[a][b] + y.e[a][b];
    return r;
}

// Forward-hop colour outer product A(a, b) = sum_{st} (I - gamma_rho)_{st}
// a_t(x + rho) (Gamma5 b)_s(x)^H: h = up - B dn of the projected neighbour,
// lower half -B^H h; A = sum_i h_i b_i^H + (B^H h)_i b_{2+i}^H (Gamma5 b
// flips the lower sign).  sg: boundary phase of the hop.
__device__ __forceinline__ M3<double> hop_outer(const double2* __restrict__ an, const double2* __restrict__ bs,
                                                int rho, double sg) {
    const SpinMono Bm = kB(rho), BHm = kBH(rho);
    double2 h[2][3], q[2][3];
    for (int i = 0; i < 2; ++i) for (int a = 0; a < 3; ++a)
        h[i][a] = sg * (an[i * 3 + a] - mul_ipow(an[(2 + Bm.perm[i]) * 3 + a], Bm.ph[i]));
    for (int i = 0; i < 2; ++i) for (int a = 0; a < 3; ++a) q[i][a] = mul_ipow(h[BHm.perm[i]][a], BHm.ph[i]);
    M3<double> A;
    for (int a = 0; a < 3; ++a) for (int b = 0; b < 3; ++b) {
        double2 t = make_double2(0, 0);
        for (int i = 0; i < 2; ++i) t += h[i][a] * conj(bs[i * 3 + b]) + q[i][a] * conj(bs[(2 + i) * 3 + b]);
        A.e[a][b] = t;
    }
    return A;
}

// One thread per link (site, rho): the force of Re <gv, Q' psi> (for
// psi = gv = v the eigenvalue force times v^H v).  Hop terms: Q' is
// Hermitian, so the real part is carried by the two forward terms
// -i/2 U (A(psi, gv) + A(gv, psi)); clover term through the insertions Bt.
// nrm: device v^H v dividing the result, or null.  grad = 1 writes the link
// gradient i F U instead of F.
__global__ void __launch_bounds__(128) link_force_kernel(const double2* __restrict__ U, const double2* __restrict__ psi,
                                                         const double2* __restrict__ gv, const double2* __restrict__ Bt,
                                                         const double2* __restrict__ nrm, Geom g, double csw, int grad,
                                                         double2* __restrict__ F) {
    const size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (e >= (size_t)g.V * 4) return;
    const int s = (int)(e >> 2), rho = (int)(e & 3);
    int x[4];
    site_coords(g, s, x);
    auto L = [&](int site, int d) { return m3_load(U + ((size_t)site * 4 + d) * 9); };
    const M3<double> u = L(s, rho);
    M3<double> K;
    {
        int neg;
        const int sf = nb_fwd(g, x, s, rho, neg);
        const double sg = neg ? -1.0 : 1.0;
        M3<double> A = hop_outer(psi + (size_t)sf * 12, gv + (size_t)s * 12, rho, sg);
        if (psi != gv) {
            const M3<double> A2 = hop_outer(gv + (size_t)sf * 12, psi + (size_t)s * 12, rho, sg);
            for (int a = 0; a < 3; ++a) for (int b = 0; b < 3; ++b) A.e[a][b] = 0.5 * (A.e[a][b] + A2.e[a][b]);
        }
        const M3<double> UA = m3_mul(u, A);
        for (int a = 0; a < 3; ++a) for (int b = 0; b < 3; ++b) K.e[a][b] = mul_ipow(UA.e[a][b], 3);   // -i U A
    }
    if (csw != 0.0) {
        const double c = csw / 16.0;
        for (int nu = 0; nu < 4; ++nu) {
            if (nu == rho) continue;
            const int pl = rho < nu ? plane_index(rho, nu) : plane_index(nu, rho);
            const double sg = rho < nu ? c : -c;   // Bt_{rho nu} = -Bt_{nu rho}
            auto Bx = [&](int site) { return m3_load(Bt + ((size_t)site * 6 + pl) * 9); };
            // plaquette above: a b c d from y, corners y, y+rho, y+rho+nu, y+nu
            M3<double> above;
            {
                const M3<double> b = L(shifted(g, x, rho, 1, nu, 0), nu);
                const M3<double> cm = m3_dag(L(shifted(g, x, rho, 0, nu, 1), rho));
                const M3<double> d = m3_dag(L(s, nu));
                const M3<double> cd = m3_mul(cm, d);
                const M3<double> t1 = m3_add(m3_mul(Bx(shifted(g, x, rho, 0, nu, 1)), d), m3_mul(d, Bx(s)));
                const M3<double> t2 = m3_add(m3_mul(Bx(shifted(g, x, rho, 1, nu, 1)), cd), m3_mul(cm, t1));
                const M3<double> t3 = m3_add(m3_mul(Bx(shifted(g, x, rho, 1, nu, 0)), m3_mul(b, cd)), m3_mul(b, t2));
                above = m3_mul(u, t3);
            }
            // plaquette below: path y -> y-nu -> y-nu+rho -> y+rho, then U_rho(y)^H
            M3<double> below;
            {
                const M3<double> dp = m3_dag(L(shifted(g, x, rho, 0, nu, -1), nu));
                const M3<double> ap = L(shifted(g, x, rho, 0, nu, -1), rho);
                const M3<double> bp = L(shifted(g, x, rho, 1, nu, -1), nu);
                const M3<double> apbp = m3_mul(ap, bp);
                const M3<double> t1 = m3_add(m3_mul(Bx(shifted(g, x, rho, 1, nu, -1)), bp),
                                             m3_mul(bp, Bx(shifted(g, x, rho, 1, nu, 0))));
                const M3<double> t2 = m3_add(m3_mul(Bx(shifted(g, x, rho, 0, nu, -1)), apbp), m3_mul(ap, t1));
                const M3<double> pre = m3_add(m3_mul(Bx(s), m3_mul(dp, apbp)), m3_mul(dp, t2));
                below = m3_mul(pre, m3_dag(u));
            }
            for (int a = 0; a < 3; ++a) for (int b = 0; b < 3; ++b)
                K.e[a][b] += sg * (below.e[a][b] - above.e[a][b]);
        }
    }
    double inv = 1.0;
    if (nrm != nullptr) {
        const double n = nrm[0].x;
        inv = n > 0 ? 1.0 / n : 0.0;
    }
    double2 H[3][3];
    for (int a = 0; a < 3; ++a) for (int b = 0; b < 3; ++b) H[a][b] = 0.5 * (K.e[a][b] + conj(K.e[b][a]));
    const double tr = (H[0][0].x + H[1][1].x + H[2][2].x) / 3.0;
    for (int a = 0; a < 3; ++a) H[a][a].x -= tr;
    if (!grad) {
        for (int a = 0; a < 3; ++a) for (int b = 0; b < 3; ++b) F[e * 9 + a * 3 + b] = inv * H[a][b];
        return;
    }
    // link gradient i F U: the tangent vector whose real inner product with
    // any dU = i X U is tr(X F)
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            double2 t = make_double2(0, 0);
            for (int c = 0; c < 3; ++c) t += H[a][c] * u.e[c][b];
            F[e * 9 + a * 3 + b] = inv * mul_ipow(t, 1);
        }
}

void eig_force(const FineOp& f, const double2* v, const double2* nrm, double2* Bt, double2* F, cudaStream_t st) {
    bilinear_force(f, v, v, nrm, 0, Bt, F, st);
}

void bilinear_force(const FineOp& f, const double2* gv, const double2* psi, const double2* nrm, int grad, double2* Bt,
                    double2* F, cudaStream_t st) {
    {
        KTimer kt("clover_insertion", 0.0, 0.0, st);
        clover_insertion_kernel<<<(f.g.V + 127) / 128, 128, 0, st>>>(psi, gv, f.g, Bt);
    }
    KTimer kt("link_force", 0.0, 0.0, st);
    const size_t nl = (size_t)f.g.V * 4;
    link_force_kernel<<<(unsigned)((nl + 127) / 128), 128, 0, st>>>(f.U64, psi, gv, Bt, nrm, f.g, f.csw, grad, F);
}

// ------------------------------------------------------------------ stencil
// out_j = op(tau_j) in_j, or out_j = b_j - op(tau_j) in_j when b != nullptr.
// op = QCD_OP_D: D - tau Gamma5 ; op = QCD_OP_Q: Gamma5 D - tau.
template <typename R>
__global__ void __launch_bounds__(128) wilson_clover_kernel(
    cplx<R>* __restrict__ out, const cplx<R>* __restrict__ in, const cplx<R>* __restrict__ b,
    const cplx<R>* __restrict__ U, const R* __restrict__ A, Geom g, int op, Shifts tau, size_t stride,
    const int* __restrict__ act) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= g.V) return;
    const int j = blockIdx.y;
    if (act != nullptr && !act[j]) return;
    in += j * stride;
    out += j * stride;
    int x[4];
    site_coords(g, s, x);
    Spinor<R> psi, acc;
    load_spinor<R>(in + (size_t)s * 12, psi);
    clover_apply<R>(A + (size_t)s * 72, psi, acc);
#pragma unroll
    for (int mu = 0; mu < 4; ++mu) {
        int neg;
        Spinor<R> nb;
        Link<R> u;
        int sf = nb_fwd(g, x, s, mu, neg);
        load_spinor<R>(in + (size_t)sf * 12, nb);
        load_link<R>(U + ((size_t)s * 4 + mu) * 9, u);
        R sg = neg ? R(-1) : R(1);
        switch (mu) {
            case 0: hop_accumulate<R, 0, true>(nb, u, sg, acc); break;
            case 1: hop_accumulate<R, 1, true>(nb, u, sg, acc); break;
            case 2: hop_accumulate<R, 2, true>(nb, u, sg, acc); break;
            default: hop_accumulate<R, 3, true>(nb, u, sg, acc); break;
        }
        int sb = nb_bwd(g, x, s, mu, neg);
        load_spinor<R>(in + (size_t)sb * 12, nb);
        load_link<R>(U + ((size_t)sb * 4 + mu) * 9, u);
        sg = neg ? R(-1) : R(1);
        switch (mu) {
            case 0: hop_accumulate<R, 0, false>(nb, u, sg, acc); break;
            case 1: hop_accumulate<R, 1, false>(nb, u, sg, acc); break;
            case 2: hop_accumulate<R, 2, false>(nb, u, sg, acc); break;
            default: hop_accumulate<R, 3, false>(nb, u, sg, acc); break;
        }
    }
    const R t = (R)tau.t[j];
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
    if (b != nullptr) {
        Spinor<R> bb;
        load_spinor<R>(b + j * stride + (size_t)s * 12, bb);
#pragma unroll
        for (int k = 0; k < 12; ++k) acc.c[k] = bb.c[k] - acc.c[k];
    }
    store_spinor<R>(out + (size_t)s * 12, acc);
}

// FP32 stencil with links and clover blocks in site-fastest (SoA) copies:
// Us[(mu * 9 + k) * V + site] (float2) and As[q * V + site] (float4, q < 18),
// so a warp's link and clover loads are contiguous; spinors keep the ABI
// layout.  Same arithmetic as wilson_clover_kernel<float>.  With several
// right-hand sides, consecutive CTAs take the same 128 sites for different
// right-hand sides (CTA index = site block x nrhs + rhs), so the CTAs that
// run together read the same links and clover blocks and all but the first
// find them in L2: the links and clover are read from HBM about once per
// site block instead of once per right-hand side.  With tb > 0 the site
// blocks are visited time-fastest within bricks of tb time slices
// (block u: t = (u / (tb ns)) tb + u % tb, spatial block (u / tb) % ns of
// ns = L1 L2 L3 / 128), so the neighbours of a block in every direction are
// read by CTAs a few hundred launches apart and still sit in L2; only the
// time neighbours across a brick face are fetched from DRAM again.  Four
// CTAs per SM (registers capped at 128, 8 bytes spilled): 16 warps in flight
// instead of 12 move the single-right-hand-side apply on 64 x 32^3 from 354 to
// 319 us (4.55 -> 5.05 TB/s).
__global__ void __launch_bounds__(128, 4) wilson_clover_soa_kernel(
    float2* __restrict__ out, const float2* __restrict__ in, const float2* __restrict__ b,
    const float2* __restrict__ Us, const float4* __restrict__ As, Geom g, int op, Shifts tau, size_t stride,
    const int* __restrict__ act, int nrhs, int tb) {
    const int j = (int)(blockIdx.x % nrhs);
    const unsigned u = blockIdx.x / nrhs;
    int s;
    if (tb > 0) {
        const unsigned vs = (unsigned)(g.L[1] * g.L[2] * g.L[3]), ns = vs / 128u;
        const unsigned t = (u / (tb * ns)) * tb + u % tb, sb = (u / tb) % ns;
        s = (int)(t * vs + sb * 128u + threadIdx.x);
    } else {
        s = (int)(u * blockDim.x + threadIdx.x);
    }
    if (s >= g.V) return;
    if (act != nullptr && !act[j]) return;
    in += j * stride;
    out += j * stride;
    const size_t V = (size_t)g.V;
    int x[4];
    site_coords(g, s, x);
    Spinor<float> psi, acc;
    load_spinor<float>(in + (size_t)s * 12, psi);
    {
        float ar[72];
#pragma unroll
        for (int q = 0; q < 18; ++q) {
            const float4 v = __ldg(As + (size_t)q * V + s);
            ar[4 * q] = v.x; ar[4 * q + 1] = v.y; ar[4 * q + 2] = v.z; ar[4 * q + 3] = v.w;
        }
        clover_apply_regs<float>(ar, psi, acc);
    }
    auto link = [&](int site, int mu, Link<float>& u) {
#pragma unroll
        for (int k = 0; k < 9; ++k) u.e[k] = __ldg(Us + (size_t)(mu * 9 + k) * V + site);
    };
#pragma unroll
    for (int mu = 0; mu < 4; ++mu) {
        int neg;
        Spinor<float> nb;
        Link<float> u;
        int sf = nb_fwd(g, x, s, mu, neg);
        load_spinor<float>(in + (size_t)sf * 12, nb);
        link(s, mu, u);
        float sg = neg ? -1.f : 1.f;
        switch (mu) {
            case 0: hop_accumulate<float, 0, true>(nb, u, sg, acc); break;
            case 1: hop_accumulate<float, 1, true>(nb, u, sg, acc); break;
            case 2: hop_accumulate<float, 2, true>(nb, u, sg, acc); break;
            default: hop_accumulate<float, 3, true>(nb, u, sg, acc); break;
        }
        int sb = nb_bwd(g, x, s, mu, neg);
        load_spinor<float>(in + (size_t)sb * 12, nb);
        link(sb, mu, u);
        sg = neg ? -1.f : 1.f;
        switch (mu) {
            case 0: hop_accumulate<float, 0, false>(nb, u, sg, acc); break;
            case 1: hop_accumulate<float, 1, false>(nb, u, sg, acc); break;
            case 2: hop_accumulate<float, 2, false>(nb, u, sg, acc); break;
            default: hop_accumulate<float, 3, false>(nb, u, sg, acc); break;
        }
    }
    const float t = (float)tau.t[j];
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
    if (b != nullptr) {
        Spinor<float> bb;
        load_spinor<float>(b + j * stride + (size_t)s * 12, bb);
#pragma unroll
        for (int k = 0; k < 12; ++k) acc.c[k] = bb.c[k] - acc.c[k];
    }
    store_spinor<float>(out + (size_t)s * 12, acc);
}

// site-fastest copies of the FP32 links and clover blocks
__global__ void soa_copies_kernel(const float2* __restrict__ U, const float* __restrict__ A, float2* __restrict__ Us,
                                  float4* __restrict__ As, int V) {
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < (size_t)V * 36; e += (size_t)gridDim.x * blockDim.x) {
        const size_t site = e % V;
        const int r = (int)(e / V);   // mu * 9 + k
        Us[e] = U[site * 36 + r];
    }
    const float4* A4 = reinterpret_cast<const float4*>(A);
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < (size_t)V * 18; e += (size_t)gridDim.x * blockDim.x) {
        const size_t site = e % V;
        const int q = (int)(e / V);
        As[e] = A4[site * 18 + q];
    }
}

// ------------------------------------------------------------------ host launchers
// Largest deviation of U U^H from the identity over all links, as the bit
// pattern of a non-negative double (which orders like the value); a
// non-finite entry records +inf.
__global__ void gauge_check_kernel(const double2* __restrict__ U, size_t nlinks, unsigned long long* __restrict__ dev) {
    double worst = 0.0;
    for (size_t l = blockIdx.x * (size_t)blockDim.x + threadIdx.x; l < nlinks; l += (size_t)gridDim.x * blockDim.x) {
        double2 u[9];
        bool fin = true;
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            u[k] = U[l * 9 + k];
            fin = fin && isfinite(u[k].x) && isfinite(u[k].y);
        }
        if (!fin) { worst = INFINITY; continue; }
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b) {
                double2 acc = make_double2(a == b ? -1.0 : 0.0, 0.0);
#pragma unroll
                for (int c = 0; c < 3; ++c) acc += u[a * 3 + c] * conj(u[b * 3 + c]);
                worst = fmax(worst, fmax(fabs(acc.x), fabs(acc.y)));
            }
    }
    for (int o = 16; o > 0; o >>= 1) worst = fmax(worst, __shfl_xor_sync(0xffffffffu, worst, o));
    if ((threadIdx.x & 31) == 0) atomicMax(dev, (unsigned long long)__double_as_longlong(worst));
}

double gauge_unitarity_deviation(const double2* U, size_t nlinks, unsigned long long* scratch, cudaStream_t st) {
    cudaMemsetAsync(scratch, 0, sizeof(unsigned long long), st);
    KTimer kt("gauge_check", (double)nlinks * 144, (double)nlinks * 27 * 8, st);
    const int grid = (int)std::min<size_t>((nlinks + 255) / 256, 4096);
    gauge_check_kernel<<<grid, 256, 0, st>>>(U, nlinks, scratch);
    unsigned long long h = 0;
    cudaMemcpyAsync(&h, scratch, sizeof(h), cudaMemcpyDeviceToHost, st);
    if (cudaStreamSynchronize(st) != cudaSuccess) return NAN;
    double d;
    memcpy(&d, &h, sizeof(d));
    return d;
}

void launch_clover_build(const FineOp& f, cudaStream_t st) {
    int th = 128;
    KTimer kt("clover_build", 0.0, 0.0, st);
    clover_build_kernel<<<(f.g.V + th - 1) / th, th, 0, st>>>(f.U64, f.g, f.m0, f.csw, f.A64, f.A32);
    if (f.U32s != nullptr && f.A32s != nullptr)
        soa_copies_kernel<<<1216, 256, 0, st>>>(f.U32, f.A32, f.U32s, f.A32s, f.g.V);
}

template <typename R>
void launch_dirac(const FineOp& f, int op, int nrhs, const void* in, void* out, const void* b,
                  const double* tau, const int* act, cudaStream_t st) {
    Shifts sh{};
    for (int j = 0; j < nrhs; ++j) sh.t[j] = tau ? tau[j] : 0.0;
    dim3 grid((f.g.V + 127) / 128, nrhs);
    const cplx<R>* U = std::is_same<R, double>::value ? (const cplx<R>*)f.U64 : (const cplx<R>*)f.U32;
    const R* A = std::is_same<R, double>::value ? (const R*)f.A64 : (const R*)f.A32;
    if (!std::is_same<R, double>::value && f.U32s != nullptr && f.A32s != nullptr) {
        const double bytes = (double)f.g.V * (nrhs * (b ? 72.0 : 48.0) + 144.0) * sizeof(R);
        KTimer kt("wilson_clover_f32", bytes, 1824.0 * f.g.V * nrhs, st);
        const unsigned gsoa = (unsigned)((f.g.V + 127) / 128) * (unsigned)nrhs;
        // several right-hand sides: time-fastest bricks of 8 time slices
        // (needs whole 128-site blocks per time slice and L0 a multiple of 8)
        const int vs = f.g.L[1] * f.g.L[2] * f.g.L[3];
        const int tb = (nrhs > 1 && vs % 128 == 0 && f.g.L[0] % 8 == 0) ? 8 : 0;
        wilson_clover_soa_kernel<<<gsoa, 128, 0, st>>>((float2*)out, (const float2*)in, (const float2*)b, f.U32s,
                                                       f.A32s, f.g, op, sh, (size_t)f.g.V * 12, act, nrhs, tb);
        return;
    }
    const double bytes = (double)f.g.V * (nrhs * (b ? 72.0 : 48.0) + 144.0) * sizeof(R);
    KTimer kt(std::is_same<R, double>::value ? "wilson_clover_f64" : "wilson_clover_f32", bytes,
              1824.0 * f.g.V * nrhs, st);
    wilson_clover_kernel<R><<<grid, 128, 0, st>>>((cplx<R>*)out, (const cplx<R>*)in, (const cplx<R>*)b,
                                                  U, A, f.g, op, sh, (size_t)f.g.V * 12, act);
}

void tangent_fields(const FineOp& f, const double2* X, double2* dU, double* dA, cudaStream_t st) {
    {
        KTimer kt("link_tangent", 0.0, 0.0, st);
        link_tangent_kernel<<<1216, 256, 0, st>>>(f.U64, X, dU, f.g.V);
    }
    KTimer kt("clover_tangent", 0.0, 0.0, st);
    clover_tangent_kernel<<<(f.g.V + 127) / 128, 128, 0, st>>>(f.U64, dU, f.g, f.csw, dA);
}

void apply_tangent(const FineOp& f, const double2* dU, const double* dA, int nrhs, const double2* in, double2* out,
                   cudaStream_t st) {
    // the hop terms with dU and the clover derivative: the stencil with these
    // fields in place of U and (m0 + 4) + C, shift 0
    Shifts sh{};
    dim3 grid((f.g.V + 127) / 128, nrhs);
    KTimer kt("wilson_tangent_f64", 0.0, 1824.0 * f.g.V * nrhs, st);
    wilson_clover_kernel<double><<<grid, 128, 0, st>>>(out, in, nullptr, dU, dA, f.g, QCD_OP_D, sh,
                                                       (size_t)f.g.V * 12, nullptr);
}

void apply_op(const FineOp& f, int prec, int op, int nrhs, const void* in, void* out,
              const double* tau, cudaStream_t st, const int* act) {
    if (prec == QCD_FP64) launch_dirac<double>(f, op, nrhs, in, out, nullptr, tau, act, st);
    else launch_dirac<float>(f, op, nrhs, in, out, nullptr, tau, act, st);
}

void residual_op(const FineOp& f, int prec, int op, int nrhs, const void* b, const void* x, void* r,
                 const double* tau, cudaStream_t st, const int* act) {
    if (prec == QCD_FP64) launch_dirac<double>(f, op, nrhs, x, r, b, tau, act, st);
    else launch_dirac<float>(f, op, nrhs, x, r, b, tau, act, st);
}

}  // namespace qcd
