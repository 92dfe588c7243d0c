// Device-side building blocks of libpond: lattice tables, the one-dimensional Hermite
// re-centring matrices of the frame transformation, Lagrange weights, boundary maps and
// storage conversions.  Everything here is written for sm_103a (GB300).
//
// State representation.  After the collision every node's populations lie in the span of
// the reduced Grad basis of order N (Eq. gradGeneralTransform; N = 3 on D2Q16, 4 on D2Q25):
// the frame transformation projects onto it and both BGK equilibria lie in it.  So the 2Q
// populations of a node are kept, without loss, as (rho, u_x, u_y, T) in FP64 plus the
// non-equilibrium parts of the (N+1)(N+2)/2 Hermite coefficients of f and of g of total
// order <= N in the node's own frame:
//     A_pq = sum_i f_i He_p(c_ia) He_q(c_ib),   B_pq = sum_i g_i He_p(c_ia) He_q(c_ib),
// f stores A_pq for (p,q) != (0,0) (A_00 = rho), g stores B_pq - B_pq^eq(rho, u, T).
// The populations are f_i = w_i sum_{p+q<=N} A_pq He_p(c_ia) He_q(c_ib) / (p! q!).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

namespace pond {

// Hermite coefficients with p + q <= N in 2-D, and the planes stored per node (f without
// (0,0), g complete).
__host__ __device__ constexpr int ncoef(int N) { return (N + 1) * (N + 2) / 2; }
__host__ __device__ constexpr int nneq(int N) { return 2 * ncoef(N) - 1; }
constexpr int NCMAX = 15;   // N <= 4
constexpr int NMAC = 4;     // rho, u_x, u_y, T (FP64)

// The Grad order of a lattice: the total Hermite order its nodes carry (3 for D1Q4-based
// D2Q16, 4 for D1Q5-based D2Q25).
__host__ __device__ constexpr int grad_order_of_q1(int q1) { return q1 == 5 ? 4 : 3; }

// Coefficient slots by total order: (p,q) = 00 | 10 01 | 20 11 02 | 30 21 12 03 | 40 31 22 13 04.
__host__ __device__ constexpr int slot(int p, int q)
{
    return (p + q) * (p + q + 1) / 2 + q;
}

// Tables of the 1-D Gauss-Hermite rules of Table I (q1 = 4 or 5), in both precisions.
// Passed to every kernel by value, so that unrolled loops read them from the constant bank.
struct Lattice {
    int q1;
    double c[5], w[5];
    double he[5][5];     // He_p(c_a), p = 0..4 (probabilists' Hermite polynomials)
    double hn[5][5];     // He_p(c_a) / p!
    float cf[5], wf[5];
    float hef[5][5], hnf[5][5];
    double cmax;         // largest |c_a|
    float cmaxf;         // the same in FP32
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
// He_k(xi) with the lower-triangular matrix
//   t_nk = (n!/k!) s^k sum_j d^(n-k-2j) (sigma/2)^j / (j! (n-k-2j)!),   sigma = s^2 - 1,
// written out below for n <= 4 in terms of sigma (formed accurately by the caller) so that
// no s^2 - 1 cancels in FP32.  In 2-D the map is the tensor product of one matrix per axis.
// Because it needs only coefficients of order <= n, it reproduces the frame transformation
// of Eq. (gradGeneralTransform) with order N exactly.
// ---------------------------------------------------------------------------------------
template <class R, int N>
struct Tau {
    R t[N + 1][N + 1];   // t[n][k] for k <= n; t[0][0] = 1
    R u1[N + 1];         // t[n][1] / s (n >= 1)
    R u2[N + 1];         // t[n][2] / s^2 (n >= 2)
};

// Re-centring matrix from s, d and an accurately formed sigma = s^2 - 1.
template <class R, int N>
__device__ __forceinline__ Tau<R, N> make_tau_sig(R s, R d, R sig)
{
    Tau<R, N> t;
    const R e = sig + d * d;
    t.t[0][0] = R(1);
    t.t[1][0] = d;
    t.t[1][1] = s;
    t.t[2][0] = e;
    t.t[2][1] = R(2) * s * d;
    t.t[2][2] = R(1) + sig;
    t.t[3][0] = d * (R(3) * e - R(2) * d * d);
    t.t[3][1] = R(3) * s * e;
    t.t[3][2] = R(3) * (R(1) + sig) * d;
    t.t[3][3] = (R(1) + sig) * s;
    t.u1[1] = R(1);
    t.u1[2] = R(2) * d;
    t.u1[3] = R(3) * e;
    t.u2[2] = R(1);
    t.u2[3] = R(3) * d;
    if constexpr (N >= 4) {
        const R d2 = d * d;
        t.t[4][0] = d2 * d2 + R(6) * d2 * sig + R(3) * sig * sig;
        t.u1[4] = R(4) * d * (d2 + R(3) * sig);
        t.t[4][1] = s * t.u1[4];
        t.u2[4] = R(6) * e;
        t.t[4][2] = (R(1) + sig) * t.u2[4];
        t.t[4][3] = R(4) * (R(1) + sig) * s * d;
        t.t[4][4] = (R(1) + sig) * (R(1) + sig);
    }
    return t;
}

// B_pq = sum_{k<=p, l<=q} tx_pk ty_ql A_kl for p + q <= N (A may alias B).
template <class R, int N>
__device__ __forceinline__ void retarget(const Tau<R, N>& x, const Tau<R, N>& y, const R* A, R* B)
{
    constexpr int NC = ncoef(N);
    R X[NC];
    // x pass: X_{p,l} = sum_{k<=p} tx_pk A_{k,l}
#pragma unroll
    for (int l = 0; l <= N; ++l)
#pragma unroll
        for (int p = 0; p <= N - l; ++p) {
            R v = (p == 0) ? A[slot(0, l)] : x.t[p][0] * A[slot(0, l)];
#pragma unroll
            for (int k = 1; k <= p; ++k) v += x.t[p][k] * A[slot(k, l)];
            X[slot(p, l)] = v;
        }
    // y pass: B_{p,q} = sum_{l<=q} ty_ql X_{p,l}
#pragma unroll
    for (int p = 0; p <= N; ++p)
#pragma unroll
        for (int q = 0; q <= N - p; ++q) {
            R v = (q == 0) ? X[slot(p, 0)] : y.t[q][0] * X[slot(p, 0)];
#pragma unroll
            for (int l = 1; l <= q; ++l) v += y.t[q][l] * X[slot(p, l)];
            B[slot(p, q)] = v;
        }
}

// retarget of two coefficient vectors by the same matrices (f's and g's): B = M A and D = M C.
// FP32 pairs them through packed two-lane FMAs, each lane the operations of retarget in its
// order; other types call retarget twice.
template <class R, int N>
__device__ __forceinline__ void retarget2(const Tau<R, N>& x, const Tau<R, N>& y, const R* A, R* B, const R* C,
                                          R* D)
{
    if constexpr (std::is_same<R, float>::value) {
        constexpr int NC = ncoef(N);
        float2 X[NC];
#pragma unroll
        for (int l = 0; l <= N; ++l)
#pragma unroll
            for (int p = 0; p <= N - l; ++p) {
                const float2 a0 = make_float2(A[slot(0, l)], C[slot(0, l)]);
                float2 v = (p == 0) ? a0 : __fmul2_rn(make_float2(x.t[p][0], x.t[p][0]), a0);
#pragma unroll
                for (int k = 1; k <= p; ++k)
                    v = __ffma2_rn(make_float2(x.t[p][k], x.t[p][k]), make_float2(A[slot(k, l)], C[slot(k, l)]), v);
                X[slot(p, l)] = v;
            }
#pragma unroll
        for (int p = 0; p <= N; ++p)
#pragma unroll
            for (int q = 0; q <= N - p; ++q) {
                float2 v = (q == 0) ? X[slot(p, 0)] : __fmul2_rn(make_float2(y.t[q][0], y.t[q][0]), X[slot(p, 0)]);
#pragma unroll
                for (int l = 1; l <= q; ++l) v = __ffma2_rn(make_float2(y.t[q][l], y.t[q][l]), X[slot(p, l)], v);
                B[slot(p, q)] = v.x;
                D[slot(p, q)] = v.y;
            }
    } else {
        retarget<R, N>(x, y, A, B);
        retarget<R, N>(x, y, C, D);
    }
}

// Entry (n, k) of a re-centring matrix (k <= n <= N).
template <class R, int N>
__device__ __forceinline__ R tau_at(const Tau<R, N>& t, int n, int k)
{
    return n == 0 ? R(1) : t.t[n][k];
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

// Weights of the P-point stencil whose first tap is at offset base (as lagrange returned it for
// an earlier departure offset) at departure offset off: the same Lagrange polynomials, with
// t = off - (base + 1) possibly outside the range that lagrange would give.  The
// predictor-corrector keeps the stencils of its first iteration and moves only their weights.
template <class R, int P>
__device__ __forceinline__ void lagrange_at(R off, int base, R* w)
{
    const R t = off - R(base + 1);
    if constexpr (P == 4) {
        R tm1 = t - R(1), tm2 = t - R(2), tp1 = t + R(1);
        w[0] = -t * tm1 * tm2 * R(1.0 / 6.0);
        w[1] = tp1 * tm1 * tm2 * R(0.5);
        w[2] = -tp1 * t * tm2 * R(0.5);
        w[3] = tp1 * t * tm1 * R(1.0 / 6.0);
    } else {
        w[0] = t * (t - R(1)) * R(0.5);
        w[1] = (R(1) - t) * (R(1) + t);
        w[2] = t * (t + R(1)) * R(0.5);
    }
}

// Whether the P-point stencil whose first tap is at offset base still serves departure offset
// off: t = off - (base + 1) lies in the range the stencil was chosen for ([0, 1) for 4 taps,
// [-1/2, 1/2) for 3) widened by a quarter cell on each side.
template <class R, int P>
__device__ __forceinline__ bool stencil_holds(R off, int base)
{
    const R t = off - R(base + 1);
    return P == 4 ? (t >= R(-0.25) && t < R(1.25)) : (t >= R(-0.75) && t < R(0.75));
}

// v[a] for a runtime a < N, and v[a] = x, without indexing a register array dynamically.
template <int N>
__device__ __forceinline__ int sel_get(const int (&v)[N], int a)
{
    int r = v[0];
#pragma unroll
    for (int k = 1; k < N; ++k) r = (a == k) ? v[k] : r;
    return r;
}
template <int N>
__device__ __forceinline__ void sel_set(int (&v)[N], int a, int x)
{
#pragma unroll
    for (int k = 0; k < N; ++k) v[k] = (a == k) ? x : v[k];
}

// Boundary maps: 0 periodic (index mod n), 1 outflow (clamp to the edge node); positions
// beyond a wall (2) map to the edge node here and are replaced by the wall's ghost state by
// the callers that stream from them.
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
// internal split B_00 = rho c_v T, B_20 = B_02 = rho T, others 0;
// non-translational split B_00 = U' = rho (c_v - 1) T, others 0.
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
    } else if (split == 1) {
        e.b00 = rho * cv * T;
        e.b10 = 0.0;
        e.b01 = 0.0;
    } else {
        e.b00 = rho * (cv - 1.0) * T;
        e.b10 = 0.0;
        e.b01 = 0.0;
    }
    e.b20 = split == 2 ? 0.0 : rho * T;
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
// A double as a sum of two floats, hi + lo, formed with integer operations only (this part's
// FP64 pipe runs at 1/64 of the FP32 rate): hi holds the top 24 significant bits, truncated,
// lo the remaining 29 bits rounded to a float, so hi + lo is within 2^-48 of x.  Magnitudes
// below 2^-126 give (0, 0) and magnitudes beyond the float range an infinite hi.  The
// difference of two such pairs, (x.hi - r.hi) + (x.lo - r.lo), is x - r to FP32 rounding of
// the result plus 2^-47 max(|x|, |r|).
struct FloatPair {
    float hi, lo;
};

__device__ __forceinline__ FloatPair split_double(double x)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const unsigned int sign = (unsigned int)(b >> 32) & 0x80000000u;
    const int e = (int)((b >> 52) & 0x7ffull);                  // biased exponent
    FloatPair r;
    if (e < 1023 - 126) {                                        // zero, subnormal or below 2^-126
        r.hi = __int_as_float((int)sign);
        r.lo = 0.0f;
        return r;
    }
    if (e > 1023 + 127) {                                        // beyond the float range
        r.hi = __int_as_float((int)(sign | 0x7f800000u));
        r.lo = 0.0f;
        return r;
    }
    const unsigned long long m = b & 0x000fffffffffffffull;     // 52 fraction bits
    r.hi = __int_as_float((int)(sign | ((unsigned int)(e - 1023 + 127) << 23) | (unsigned int)(m >> 29)));
    // the low 29 bits are worth m_lo 2^(e - 1075)
    const float m_lo = __uint2float_rn((unsigned int)(m & 0x1fffffffull));
    const int k = e - 1075;
    const float scale = k >= -126 ? __int_as_float((k + 127) << 23) : 0.0f;
    r.lo = __int_as_float(__float_as_int(m_lo * scale) | (int)sign);
    return r;
}

// x truncated toward zero to FP32 precision (its top 24 significant bits), by integer
// operations: zero below the normal FP32 range, infinity above it, NaN for NaN.
__device__ __forceinline__ float double_hi(double x)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const unsigned int sign = (unsigned int)(b >> 32) & 0x80000000u;
    const int e = (int)((b >> 52) & 0x7ffull);
    const unsigned long long m = b & 0x000fffffffffffffull;
    if (e < 1023 - 126) return __int_as_float((int)sign);
    if (e == 0x7ff && m != 0) return __int_as_float(0x7fc00000);
    if (e > 1023 + 127) return __int_as_float((int)(sign | 0x7f800000u));
    return __int_as_float((int)(sign | ((unsigned int)(e - 1023 + 127) << 23) | (unsigned int)(m >> 29)));
}

// x > 0 (false for NaN), by integer operations on its bits.
__device__ __forceinline__ bool positive_double(double x)
{
    const long long b = __double_as_longlong(x);
    return b > 0 && b <= 0x7ff0000000000000ll;
}

__device__ __forceinline__ float pair_diff(const FloatPair& x, const FloatPair& r)
{
    return (x.hi - r.hi) + (x.lo - r.lo);
}

// Status flag of a rejected host input (bits 0 and 1 are the kernels' statuses, non-physical
// and non-convergence).
constexpr int kInputBad = 4;

struct DevStatus {
    unsigned long long iters_total;
    unsigned long long nonconv;
    unsigned long long fallbacks;
    unsigned long long first_bad;    // atomicMin; ~0ull when none
    unsigned int iters_max;
    int flags;                        // bit 0 non-physical, bit 1 non-convergence, bit 2 rejected host input
    unsigned long long steps;
    unsigned long long pad[2];
};

// Four [N] arrays (rho, u_x, u_y, T) for each member of a batched auxiliary launch over
// members [c0, c0 + count), count <= kAuxChunk, passed by value as a kernel argument.
constexpr int kAuxChunk = 64;
struct MemberFields {
    double* f[kAuxChunk][4];
};

}  // namespace pond
