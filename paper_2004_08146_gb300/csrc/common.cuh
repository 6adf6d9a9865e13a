// Shared device helpers for libqcd: complex arithmetic on float2/double2,
// lattice geometry, the chiral-basis spin tables, reductions and error codes.
#pragma once

#include <cuda_runtime.h>
#include <cstdint>
#include <cstddef>

#include "../../include/qcd.h"

namespace qcd {

// ------------------------------------------------------------------ complex
template <typename R> struct C2;
template <> struct C2<double> { using T = double2; };
template <> struct C2<float>  { using T = float2; };
template <typename R> using cplx = typename C2<R>::T;

template <typename R> __host__ __device__ __forceinline__ cplx<R> mk(R re, R im) {
    cplx<R> z; z.x = re; z.y = im; return z;
}
template <typename R> __host__ __device__ __forceinline__ cplx<R> czero() { return mk<R>(R(0), R(0)); }

#define QCD_HD __host__ __device__ __forceinline__
QCD_HD double2 operator+(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
QCD_HD double2 operator-(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
QCD_HD double2 operator-(double2 a) { return make_double2(-a.x, -a.y); }
QCD_HD double2 operator*(double2 a, double2 b) { return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
QCD_HD double2 operator*(double s, double2 a) { return make_double2(s * a.x, s * a.y); }
QCD_HD double2& operator+=(double2& a, double2 b) { a.x += b.x; a.y += b.y; return a; }
QCD_HD double2& operator-=(double2& a, double2 b) { a.x -= b.x; a.y -= b.y; return a; }
QCD_HD float2 operator+(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
QCD_HD float2 operator-(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
QCD_HD float2 operator-(float2 a) { return make_float2(-a.x, -a.y); }
QCD_HD float2 operator*(float2 a, float2 b) { return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
QCD_HD float2 operator*(float s, float2 a) { return make_float2(s * a.x, s * a.y); }
QCD_HD float2& operator+=(float2& a, float2 b) { a.x += b.x; a.y += b.y; return a; }
QCD_HD float2& operator-=(float2& a, float2 b) { a.x -= b.x; a.y -= b.y; return a; }

template <typename Z> QCD_HD Z conj(Z a) { a.y = -a.y; return a; }
// conj(a) * b
template <typename Z> QCD_HD Z cmulc(Z a, Z b) {
    Z r; r.x = a.x * b.x + a.y * b.y; r.y = a.x * b.y - a.y * b.x; return r;
}
// a * i^k (k = 0..3)
template <typename Z> QCD_HD Z mul_ipow(Z a, int k) {
    Z r;
    switch (k & 3) {
        case 0: r = a; break;
        case 1: r.x = -a.y; r.y = a.x; break;
        case 2: r.x = -a.x; r.y = -a.y; break;
        default: r.x = a.y; r.y = -a.x; break;
    }
    return r;
}
template <typename Zd, typename Zs> QCD_HD Zd cvt(Zs a) { Zd r; r.x = a.x; r.y = a.y; return r; }

// ------------------------------------------------------------------ geometry
struct Geom {
    int L[4];
    int V;
    int antiperiodic;
};

QCD_HD void site_coords(const Geom& g, int s, int x[4]) {
    x[3] = s % g.L[3]; s /= g.L[3];
    x[2] = s % g.L[2]; s /= g.L[2];
    x[1] = s % g.L[1];
    x[0] = s / g.L[1];
}
QCD_HD int site_index(const Geom& g, const int x[4]) {
    return ((x[0] * g.L[1] + x[1]) * g.L[2] + x[2]) * g.L[3] + x[3];
}

// ------------------------------------------------------------------ spin tables
// gamma_mu = [[0, B_mu], [B_mu^H, 0]] in 2x2 spin blocks (chiral basis,
// gamma5 = diag(1, 1, -1, -1)).  Each B_mu (and B_mu^H) has one non-zero per
// row: row r reads column perm[r] with phase i^ph[r].
//   B_0 = -I, B_1 = -i sigma_1, B_2 = -i sigma_2, B_3 = -i sigma_3.
struct SpinMono { int perm[2]; int ph[2]; };
__host__ __device__ constexpr SpinMono kB(int mu) {
    return mu == 0 ? SpinMono{{0, 1}, {2, 2}}
         : mu == 1 ? SpinMono{{1, 0}, {3, 3}}
         : mu == 2 ? SpinMono{{1, 0}, {2, 0}}
         :           SpinMono{{0, 1}, {3, 1}};
}
__host__ __device__ constexpr SpinMono kBH(int mu) {
    return mu == 0 ? SpinMono{{0, 1}, {2, 2}}
         : mu == 1 ? SpinMono{{1, 0}, {1, 1}}
         : mu == 2 ? SpinMono{{1, 0}, {0, 2}}
         :           SpinMono{{0, 1}, {1, 3}};
}

// ------------------------------------------------------------------ Hermitian 6x6 packed
// 36 reals: 6 real diagonal entries, then the 15 complex entries (i < j) of
// the upper triangle in row-major order.
QCD_HD int herm_off(int i, int j) {  // i < j
    return 6 + 2 * (i * 6 - i * (i + 1) / 2 + (j - i - 1));
}

// ------------------------------------------------------------------ shifts by value
constexpr int kMaxRhs = 64;
struct Shifts { double t[kMaxRhs]; };

// ------------------------------------------------------------------ reductions
template <typename R> __device__ __forceinline__ R warp_sum(R v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

}  // namespace qcd
