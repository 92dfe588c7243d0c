// Device-side building blocks of libpond: lattice tables, the one-dimensional Hermite
// re-centring matrices of the frame transformation, Lagrange weights, boundary maps and
// storage conversions.  Everything here is written for sm_103a (GB300).
//
// State representation.  After the collision every node's populations lie in the span of
// the reduced Grad basis (Eq. gradGeneralTransform, N = 3): the frame transformation
// projects onto it and both BGK equilibria lie in it.  So the 2Q populations of a node are
// kept, without loss, as (rho, u_x, u_y, T) in FP64 plus the non-equilibrium parts of the
// ten Hermite coefficients of f and of g of total order <= 3 in the node's own frame:
//     A_pq = sum_i f_i He_p(c_ia) He_q(c_ib),   B_pq = sum_i g_i He_p(c_ia) He_q(c_ib),
// f stores A_pq for (p,q) != (0,0) (A_00 = rho), g stores B_pq - B_pq^eq(rho, u, T).
// The populations are f_i = w_i sum_{p+q<=3} A_pq He_p(c_ia) He_q(c_ib) / (p! q!).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

namespace pond {

constexpr int NCOEF = 10;   // Hermite coefficients with p + q <= 3 in 2-D
constexpr int NNEQ = 19;    // stored per node: 9 for f (all but (0,0)), 10 for g
constexpr int NMAC = 4;     // rho, u_x, u_y, T (FP64)

// Coefficient slots: (p,q) = 00 10 01 20 11 02 30 21 12 03.
__host__ __device__ constexpr int slot(int p, int q)
{
    return (p + q == 0) ? 0 : (p + q == 1) ? 1 + q : (p + q == 2) ? 3 + q : 6 + q;
}

// Tables of the 1-D Gauss-Hermite rules of Table I (q1 = 4 or 5), in both precisions.
// Passed to every kernel by value, so that unrolled loops read them from the constant bank.
struct Lattice {
    int q1;
    double c[5], w[5];
    double he[5][4];     // He_p(c_a), p = 0..3 (probabilists' Hermite polynomials)
    double hn[5][4];     // He_p(c_a) / p!
    float cf[5], wf[5];
    float hef[5][4], hnf[5][4];
    double cmax;         // largest |c_a|
};

template <class R>
__device__ __forceinline__ R lat_c(const Lattice& L, int a)
{
    if constexpr (std::is_same<R, double>::value) return L.c[a]; else return L.cf[a];
}
template <class R>
__device__ __forceinline__ R lat_w(const Lattice& L, int a)
{
    if constexpr (std::is_same<R, double>::value) return L.w[a]; else return L.wf[a];
}
template <class R>
__device__ __forceinline__ R lat_he(const Lattice& L, int a, int p)
{
    if constexpr (std::is_same<R, double>::value) return L.he[a][p]; else return L.hef[a][p];
}
template <class R>
__device__ __forceinline__ R lat_hn(const Lattice& L, int a, int p)
{
    if constexpr (std::is_same<R, double>::value) return L.hn[a][p]; else return L.hnf[a][p];
}

// ---------------------------------------------------------------------------------------
// Re-centring of Hermite coefficients between frames.  For populations whose velocities
// are xi_old = (C - u_old)/sqrt(T_old), the new variable is xi_new = s xi_old + d with
// s = sqrt(T_old / T_new), d = (u_old - u_new)/sqrt(T_new).  He_n(s xi + d) expands in
// He_k(xi) with the lower-triangular matrix below (e = s^2 - 1 + d^2); in 2-D the map is
// the tensor product of one such matrix per axis.  Because it needs only coefficients of
// order <= n, it reproduces the frame transformation of Eq. (gradGeneralTransform) with
// N = 3 exactly.
// ---------------------------------------------------------------------------------------
template <class R>
struct Tau {
    R t10, t11, t20, t21, t22, t30, t31, t32, t33;   // t00 = 1
};

template <class R>
__device__ __forceinline__ Tau<R> make_tau(R s, R d)
{
    Tau<R> t;
    R s2 = s * s;
    R e = s2 - R(1) + d * d;
    t.t10 = d;
    t.t11 = s;
    t.t20 = e;
    t.t21 = R(2) * s * d;
    t.t22 = s2;
    t.t30 = d * (R(3) * e - R(2) * d * d);
    t.t31 = R(3) * s * e;
    t.t32 = R(3) * s2 * d;
    t.t33 = s2 * s;
    return t;
}

// B_pq = sum_{k<=p, l<=q} tx_pk ty_ql A_kl for p + q <= 3 (A may alias B).
template <class R>
__device__ __forceinline__ void retarget(const Tau<R>& x, const Tau<R>& y, const R* A, R* B)
{
    // x pass: X_{p,l} = sum_{k<=p} tx_pk A_{k,l}
    R a00 = A[slot(0, 0)], a10 = A[slot(1, 0)], a20 = A[slot(2, 0)], a30 = A[slot(3, 0)];
    R a01 = A[slot(0, 1)], a11 = A[slot(1, 1)], a21 = A[slot(2, 1)];
    R a02 = A[slot(0, 2)], a12 = A[slot(1, 2)];
    R a03 = A[slot(0, 3)];
    R x00 = a00;
    R x10 = x.t10 * a00 + x.t11 * a10;
    R x20 = x.t20 * a00 + x.t21 * a10 + x.t22 * a20;
    R x30 = x.t30 * a00 + x.t31 * a10 + x.t32 * a20 + x.t33 * a30;
    R x01 = a01;
    R x11 = x.t10 * a01 + x.t11 * a11;
    R x21 = x.t20 * a01 + x.t21 * a11 + x.t22 * a21;
    R x02 = a02;
    R x12 = x.t10 * a02 + x.t11 * a12;
    R x03 = a03;
    // y pass: B_{p,q} = sum_{l<=q} ty_ql X_{p,l}
    B[slot(0, 0)] = x00;
    B[slot(1, 0)] = x10;
    B[slot(2, 0)] = x20;
    B[slot(3, 0)] = x30;
    B[slot(0, 1)] = y.t10 * x00 + y.t11 * x01;
    B[slot(1, 1)] = y.t10 * x10 + y.t11 * x11;
    B[slot(2, 1)] = y.t10 * x20 + y.t11 * x21;
    B[slot(0, 2)] = y.t20 * x00 + y.t21 * x01 + y.t22 * x02;
    B[slot(1, 2)] = y.t20 * x10 + y.t21 * x11 + y.t22 * x12;
    B[slot(0, 3)] = y.t30 * x00 + y.t31 * x01 + y.t32 * x02 + y.t33 * x03;
}

// Entry (n, k) of a Tau matrix (k <= n <= 3).
template <class R>
__device__ __forceinline__ R tau_at(const Tau<R>& t, int n, int k)
{
    if (n == 0) return R(1);
    if (n == 1) return k == 0 ? t.t10 : t.t11;
    if (n == 2) return k == 0 ? t.t20 : (k == 1 ? t.t21 : t.t22);
    return k == 0 ? t.t30 : (k == 1 ? t.t31 : (k == 2 ? t.t32 : t.t33));
}

// ---------------------------------------------------------------------------------------
// Lagrange stencils (Sec. III.A.2).  off = departure point minus the node (cells).  Returns
// the offset of the first of the P taps; w receives their weights.
//   P = 4 (cubic): taps floor(off) - 1 .. floor(off) + 2, t = off - floor(off) in [0, 1);
//   P = 3 (quadratic): taps m - 1 .. m + 1, m = floor(off + 1/2), t = off - m in [-1/2, 1/2).
// ---------------------------------------------------------------------------------------
template <class R, int P>
__device__ __forceinline__ int lagrange(R off, R* w)
{
    if constexpr (P == 4) {
        R fl = floor(off);
        R t = off - fl;
        R tm1 = t - R(1), tm2 = t - R(2), tp1 = t + R(1);
        w[0] = -t * tm1 * tm2 * R(1.0 / 6.0);
        w[1] = tp1 * tm1 * tm2 * R(0.5);
        w[2] = -tp1 * t * tm2 * R(0.5);
        w[3] = tp1 * t * tm1 * R(1.0 / 6.0);
        return (int)fl - 1;
    } else {
        R m = floor(off + R(0.5));
        R t = off - m;
        w[0] = t * (t - R(1)) * R(0.5);
        w[1] = (R(1) - t) * (R(1) + t);
        w[2] = t * (t + R(1)) * R(0.5);
        return (int)m - 1;
    }
}

// Boundary maps: 0 periodic (index mod n), 1 outflow (clamp to the edge node).
__device__ __forceinline__ int bc_map(int j, int n, int bc)
{
    if (bc == 0) {
        int r = j % n;
        return r < 0 ? r + n : r;
    }
    return j < 0 ? 0 : (j > n - 1 ? n - 1 : j);
}

// ---------------------------------------------------------------------------------------
// Storage types of the non-equilibrium coefficients.
// ---------------------------------------------------------------------------------------
template <class S>
__device__ __forceinline__ double sto_load(const S* p)
{
    if constexpr (std::is_same<S, double>::value) return *p;
    else if constexpr (std::is_same<S, float>::value) return (double)*p;
    else if constexpr (std::is_same<S, __half>::value) return (double)__half2float(*p);
    else return (double)__bfloat162float(*p);
}
template <class S>
__device__ __forceinline__ float sto_loadf(const S* p)
{
    if constexpr (std::is_same<S, double>::value) return (float)*p;
    else if constexpr (std::is_same<S, float>::value) return *p;
    else if constexpr (std::is_same<S, __half>::value) return __half2float(*p);
    else return __bfloat162float(*p);
}
template <class S, class R>
__device__ __forceinline__ R sto_get(const S* p)
{
    if constexpr (std::is_same<R, double>::value) return sto_load<S>(p); else return sto_loadf<S>(p);
}
template <class S, class R>
__device__ __forceinline__ void sto_put(S* p, R v)
{
    if constexpr (std::is_same<S, double>::value) *p = (double)v;
    else if constexpr (std::is_same<S, float>::value) *p = (float)v;
    else if constexpr (std::is_same<S, __half>::value) *p = __float2half_rn((float)v);
    else *p = __float2bfloat16_rn((float)v);
}

// Equilibrium Hermite coefficients of g in its own frame (Sec. II g_eq, Sec. III.A lattice):
// total split    B_00 = rho (c_v T + |u|^2/2), B_10 = rho sqrt(T) u_x, B_01 = rho sqrt(T) u_y,
//                B_20 = B_02 = rho T, others 0;
// internal split B_00 = rho c_v T, B_20 = B_02 = rho T, others 0.
struct GEq {
    double b00, b10, b01, b20;   // b02 = b20
};
__device__ __forceinline__ GEq g_equilibrium(int split, double cv, double rho, double ux, double uy,
                                             double T, double sqrtT)
{
    GEq e;
    if (split == 0) {
        e.b00 = rho * (cv * T + 0.5 * (ux * ux + uy * uy));
        e.b10 = rho * sqrtT * ux;
        e.b01 = rho * sqrtT * uy;
    } else {
        e.b00 = rho * cv * T;
        e.b10 = 0.0;
        e.b01 = 0.0;
    }
    e.b20 = rho * T;
    return e;
}

// Kahan-Babuska compensated sum in working precision R (exact error term of each addition).
template <class R>
struct CompSum {
    R hi = R(0), lo = R(0);
    __device__ __forceinline__ void add(R x)
    {
        if constexpr (std::is_same<R, double>::value) {
            hi += x;
        } else {
            R s = hi + x;
            R bp = s - hi;
            lo += (hi - (s - bp)) + (x - bp);
            hi = s;
        }
    }
    __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};

// Sticky device status block (zeroed by pond_set_state*).
struct DevStatus {
    unsigned long long iters_total;
    unsigned long long nonconv;
    unsigned long long fallbacks;
    unsigned long long first_bad;    // atomicMin; ~0ull when none
    unsigned int iters_max;
    int flags;                        // bit 0 non-physical, bit 1 non-convergence
    unsigned long long steps;
    unsigned long long pad[2];
};

}  // namespace pond
