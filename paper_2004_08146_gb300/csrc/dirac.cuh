// Device building blocks of the Wilson-clover operator (Eq. 2.5 plus the
// clover term): spinor loads/stores, SU(3) products, spin projection with
// the chiral-basis monomials of common.cuh and the packed clover apply.
#pragma once
#include "common.cuh"

namespace qcd {

template <typename R> struct Spinor { cplx<R> c[12]; };   // index = spin*3 + colour

template <typename R> __device__ __forceinline__ void load_spinor(const cplx<R>* __restrict__ p, Spinor<R>& s);
template <> __device__ __forceinline__ void load_spinor<double>(const double2* __restrict__ p, Spinor<double>& s) {
#pragma unroll
    for (int k = 0; k < 12; ++k) s.c[k] = __ldg(p + k);
}
template <> __device__ __forceinline__ void load_spinor<float>(const float2* __restrict__ p, Spinor<float>& s) {
    const float4* q = reinterpret_cast<const float4*>(p);
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        float4 v = __ldg(q + k);
        s.c[2 * k] = make_float2(v.x, v.y);
        s.c[2 * k + 1] = make_float2(v.z, v.w);
    }
}
template <typename R> __device__ __forceinline__ void store_spinor(cplx<R>* __restrict__ p, const Spinor<R>& s);
template <> __device__ __forceinline__ void store_spinor<double>(double2* __restrict__ p, const Spinor<double>& s) {
#pragma unroll
    for (int k = 0; k < 12; ++k) p[k] = s.c[k];
}
template <> __device__ __forceinline__ void store_spinor<float>(float2* __restrict__ p, const Spinor<float>& s) {
    float4* q = reinterpret_cast<float4*>(p);
#pragma unroll
    for (int k = 0; k < 6; ++k) q[k] = make_float4(s.c[2 * k].x, s.c[2 * k].y, s.c[2 * k + 1].x, s.c[2 * k + 1].y);
}

template <typename R> struct Link { cplx<R> e[9]; };
template <typename R> __device__ __forceinline__ void load_link(const cplx<R>* __restrict__ p, Link<R>& u) {
#pragma unroll
    for (int k = 0; k < 9; ++k) u.e[k] = __ldg(p + k);
}

// y = U h (dag = false) or U^H h (dag = true) on a 2-spinor h[2][3]
template <typename R, bool dag>
__device__ __forceinline__ void su3_mul_half(const Link<R>& u, const cplx<R> h[6], cplx<R> o[6]) {
#pragma unroll
    for (int s = 0; s < 2; ++s) {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            cplx<R> acc = czero<R>();
#pragma unroll
            for (int b = 0; b < 3; ++b) {
                if (dag) acc += cmulc(u.e[b * 3 + a], h[s * 3 + b]);
                else     acc += u.e[a * 3 + b] * h[s * 3 + b];
            }
            o[s * 3 + a] = acc;
        }
    }
}

// Hop contribution of direction mu: psi is the neighbour spinor (with the
// boundary sign already folded into `sgn`), U the link (U_mu(x) forward,
// U_mu(x-mu) backward, used daggered).  Adds
//   forward : -1/2 (1 - gamma_mu) U psi   -> up += -1/2 U h,  dn += +1/2 B^H U h,  h = up - B dn
//   backward: -1/2 (1 + gamma_mu) U^H psi -> up += -1/2 U^H h, dn += -1/2 B^H U^H h, h = up + B dn
template <typename R, int mu, bool fwd>
__device__ __forceinline__ void hop_accumulate(const Spinor<R>& psi, const Link<R>& u, R sgn, Spinor<R>& acc) {
    constexpr SpinMono B = kB(mu);
    constexpr SpinMono BH = kBH(mu);
    cplx<R> h[6], o[6];
#pragma unroll
    for (int s = 0; s < 2; ++s) {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            cplx<R> bd = mul_ipow(psi.c[(2 + B.perm[s]) * 3 + a], B.ph[s]);
            h[s * 3 + a] = fwd ? (psi.c[s * 3 + a] - bd) : (psi.c[s * 3 + a] + bd);
        }
    }
    su3_mul_half<R, !fwd>(u, h, o);
    const R half = R(-0.5) * sgn;
#pragma unroll
    for (int s = 0; s < 2; ++s) {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            acc.c[s * 3 + a] += half * o[s * 3 + a];
            cplx<R> bo = mul_ipow(o[BH.perm[s] * 3 + a], BH.ph[s]);
            if (fwd) acc.c[(2 + s) * 3 + a] -= half * bo;
            else     acc.c[(2 + s) * 3 + a] += half * bo;
        }
    }
}

// The same hop with the direction chosen at run time (fwd: U_mu(x) and
// 1 - gamma_mu; otherwise U_mu(x-mu)^H and 1 + gamma_mu), so that lanes with
// neighbours on different sides share one instruction stream.
template <typename R, int mu>
__device__ __forceinline__ void hop_accumulate_dir(const Spinor<R>& psi, const Link<R>& u, R sgn, bool fwd,
                                                   Spinor<R>& acc) {
    constexpr SpinMono B = kB(mu);
    constexpr SpinMono BH = kBH(mu);
    const R pm = fwd ? R(-1) : R(1);
    cplx<R> h[6], o[6];
#pragma unroll
    for (int s = 0; s < 2; ++s) {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const cplx<R> bd = mul_ipow(psi.c[(2 + B.perm[s]) * 3 + a], B.ph[s]);
            h[s * 3 + a] = psi.c[s * 3 + a] + pm * bd;
        }
    }
    cplx<R> e[9];   // U or U^H
#pragma unroll
    for (int a = 0; a < 3; ++a) {
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            const cplx<R> d = u.e[a * 3 + b], t = u.e[b * 3 + a];
            e[a * 3 + b] = fwd ? d : conj(t);
        }
    }
#pragma unroll
    for (int s = 0; s < 2; ++s) {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            cplx<R> accv = czero<R>();
#pragma unroll
            for (int b = 0; b < 3; ++b) accv += e[a * 3 + b] * h[s * 3 + b];
            o[s * 3 + a] = accv;
        }
    }
    const R half = R(-0.5) * sgn;
#pragma unroll
    for (int s = 0; s < 2; ++s) {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            acc.c[s * 3 + a] += half * o[s * 3 + a];
            const cplx<R> bo = mul_ipow(o[BH.perm[s] * 3 + a], BH.ph[s]);
            acc.c[(2 + s) * 3 + a] += (pm * half) * bo;
        }
    }
}

// y = A x for the two packed Hermitian 6x6 chirality blocks (diagonal reals,
// then the upper triangle as (re, im) pairs in herm_off order)
template <typename R>
__device__ __forceinline__ void clover_apply_regs(const R* a0, const Spinor<R>& x, Spinor<R>& y) {
#pragma unroll
    for (int chi = 0; chi < 2; ++chi) {
        const R* a = a0 + 36 * chi;
        const cplx<R>* xs = x.c + 6 * chi;
        cplx<R>* ys = y.c + 6 * chi;
#pragma unroll
        for (int i = 0; i < 6; ++i) ys[i] = a[i] * xs[i];
#pragma unroll
        for (int i = 0; i < 6; ++i) {
#pragma unroll
            for (int j = i + 1; j < 6; ++j) {
                const int o = herm_off(i, j);
                cplx<R> aij = mk<R>(a[o], a[o + 1]);
                ys[i] += aij * xs[j];
                ys[j] += cmulc(aij, xs[i]);
            }
        }
    }
}

template <typename R>
__device__ __forceinline__ void clover_apply(const R* __restrict__ A, const Spinor<R>& x, Spinor<R>& y) {
    // the 72 reals of the site (288 B in FP32, 576 B in FP64; 16-byte aligned)
    // in 16-byte loads
    if constexpr (sizeof(R) == 4) {
        R ar[72];
        const float4* q = reinterpret_cast<const float4*>(A);
#pragma unroll
        for (int k = 0; k < 18; ++k) {
            const float4 v = __ldg(q + k);
            ar[4 * k] = v.x; ar[4 * k + 1] = v.y; ar[4 * k + 2] = v.z; ar[4 * k + 3] = v.w;
        }
        clover_apply_regs<R>(ar, x, y);
    } else {
        // FP64: (re, im) pairs on demand (all pairs start at even offsets)
#pragma unroll
        for (int chi = 0; chi < 2; ++chi) {
            const double2* q = reinterpret_cast<const double2*>(A + 36 * chi);
            const cplx<R>* xs = x.c + 6 * chi;
            cplx<R>* ys = y.c + 6 * chi;
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                const double2 d = __ldg(q + i);
                ys[2 * i] = d.x * xs[2 * i];
                ys[2 * i + 1] = d.y * xs[2 * i + 1];
            }
#pragma unroll
            for (int i = 0; i < 6; ++i) {
#pragma unroll
                for (int j = i + 1; j < 6; ++j) {
                    const double2 aij = __ldg(q + herm_off(i, j) / 2);
                    ys[i] += aij * xs[j];
                    ys[j] += cmulc(aij, xs[i]);
                }
            }
        }
    }
}

// Same product with the packed blocks in shared memory.
template <typename R>
__device__ __forceinline__ void clover_apply_smem(const R* A, const Spinor<R>& x, Spinor<R>& y) {
    clover_apply_regs<R>(A, x, y);
}
// neighbour site and boundary sign
__device__ __forceinline__ int nb_fwd(const Geom& g, const int x[4], int s, int mu, int& sgn_neg) {
    int y[4] = {x[0], x[1], x[2], x[3]};
    y[mu] += 1;
    sgn_neg = 0;
    if (y[mu] == g.L[mu]) { y[mu] = 0; if (mu == 0 && g.antiperiodic) sgn_neg = 1; }
    return site_index(g, y);
}
__device__ __forceinline__ int nb_bwd(const Geom& g, const int x[4], int s, int mu, int& sgn_neg) {
    int y[4] = {x[0], x[1], x[2], x[3]};
    y[mu] -= 1;
    sgn_neg = 0;
    if (y[mu] < 0) { y[mu] = g.L[mu] - 1; if (mu == 0 && g.antiperiodic) sgn_neg = 1; }
    return site_index(g, y);
}

}  // namespace qcd
