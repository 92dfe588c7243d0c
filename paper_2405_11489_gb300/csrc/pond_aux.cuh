// Auxiliary kernels of libpond: equilibrium initialisation, population import/export,
// moments of the current state, and the internal-energy-split source pass.
#pragma once

#include "pond_device.cuh"
#include "pond_step.cuh"

namespace pond {

struct AuxParams {
    Lattice lat;
    int nx, ny, bc_x, bc_y, split;
    int nord;           // Grad order N of the state (3 or 4)
    long long N;
    double cv;
    double mu;          // dynamic viscosity (tau = mu / p)
    double* mac;        // [4][N] rho, u_x, u_y, T
    void* neq;          // [nneq(N)][N] storage type
    const double* mac_prev;  // internal source: frames before the step
    DevStatus* status;
    double wall[4][4];       // prescribed side states (u_x, u_y, T, rho), boundary types 2 and 3
    const double* prof[4];   // per side: null (uniform wall[side]) or [n][4] states along it
};

// Equilibrium state from rho, u, T (device-accessible arrays [N]): f_i = rho w_i, g_i = g_eq_i
// in the node's own frame (Sec. III.A) -> all non-equilibrium coefficients zero.
template <class S>
__device__ __forceinline__ void init_node(double* mac, void* neq, long long N, int nord, DevStatus* status,
                                          long long n, double r, double vx, double vy, double t)
{
    if (!(r > 0.0) || !(t > 0.0) || isnan(vx) || isnan(vy) || isinf(vx) || isinf(vy) || isinf(r) || isinf(t)) {
        atomicOr(&status->flags, 1);
        atomicMin(&status->first_bad, (unsigned long long)n);
    }
    mac[n] = r;
    mac[N + n] = vx;
    mac[2 * N + n] = vy;
    mac[3 * N + n] = t;
    S* q = reinterpret_cast<S*>(neq);
    for (int m = 0; m < nneq(nord); ++m) sto_put<S, double>(q + (long long)m * N + n, 0.0);
}

template <class S>
__device__ __forceinline__ void add_source_node(long long n, int x, int y, int nx, int ny, int bc_x, int bc_y,
                                                long long N, int nord, const double* vux, const double* vuy,
                                                const double (*wall)[4], const double* const* prof, double rho,
                                                double ux, double uy, double T, double dtux_d, double dtuy_d,
                                                double factor, void* neq);

// Internal split: the stored state is the post-collision g carried as g - (Omega + G)/2 (the
// trapezoidal rule of the source), which at equilibrium is g_eq + G/2, G with grad u of the
// given velocity fields and d_t u = 0.
template <class S>
__device__ __forceinline__ void init_internal_source(long long n, int nx, int ny, int bc_x, int bc_y, long long N,
                                                     int nord, const double* ux, const double* uy,
                                                     const double (*wall)[4], const double* const* prof,
                                                     double r, double t, void* neq)
{
    const int x = (int)(n % nx), y = (int)(n / nx);
    add_source_node<S>(n, x, y, nx, ny, bc_x, bc_y, N, nord, ux, uy, wall, prof, r, ux[n], uy[n], t, 0.0, 0.0, 0.5,
                       neq);
}

template <class S>
__global__ void init_kernel(AuxParams p, const double* rho, const double* ux, const double* uy,
                            const double* T)
{
    long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= p.N) return;
    if (p.status->flags & kInputBad) return;   // the input check before rejected it: state unchanged
    init_node<S>(p.mac, p.neq, p.N, p.nord, p.status, n, rho[n], ux[n], uy[n], T[n]);
    if (p.split == 1)
        init_internal_source<S>(n, p.nx, p.ny, p.bc_x, p.bc_y, p.N, p.nord, ux, uy, p.wall, p.prof, rho[n], T[n],
                                p.neq);
}

// Populations f, g [Q][N] in frames (ux, uy, T) -> Hermite coefficients of order <= N.
template <class S>
__global__ void set_pops_kernel(AuxParams p, const double* f, const double* g, const double* ux,
                                const double* uy, const double* T)
{
    long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= p.N) return;
    const Lattice& L = p.lat;
    const int q1 = L.q1, no = p.nord, nc = ncoef(no);
    double A[NCMAX] = {0}, B[NCMAX] = {0};
    for (int b = 0; b < q1; ++b)
        for (int a = 0; a < q1; ++a) {
            long long i = (long long)(b * q1 + a) * p.N + n;
            double fi = f[i], gi = g[i];
            for (int pp = 0; pp <= no; ++pp)
                for (int qq = 0; qq <= no - pp; ++qq) {
                    double h = L.he[a][pp] * L.he[b][qq];
                    A[slot(pp, qq)] += fi * h;
                    B[slot(pp, qq)] += gi * h;
                }
        }
    double vx = ux[n], vy = uy[n], t = T[n];
    double rho = A[0];
    if (!(rho > 0.0) || !(t > 0.0) || isnan(vx) || isnan(vy)) {
        atomicOr(&p.status->flags, 1);
        atomicMin(&p.status->first_bad, (unsigned long long)n);
    }
    p.mac[n] = rho;
    p.mac[p.N + n] = vx;
    p.mac[2 * p.N + n] = vy;
    p.mac[3 * p.N + n] = t;
    GEq e = g_equilibrium(p.split, p.cv, rho, vx, vy, t, sqrt(t));
    B[slot(0, 0)] -= e.b00;
    B[slot(1, 0)] -= e.b10;
    B[slot(0, 1)] -= e.b01;
    B[slot(2, 0)] -= e.b20;
    B[slot(0, 2)] -= e.b20;
    S* q = reinterpret_cast<S*>(p.neq);
    for (int m = 1; m < nc; ++m) sto_put<S, double>(q + (long long)(m - 1) * p.N + n, A[m]);
    for (int m = 0; m < nc; ++m) sto_put<S, double>(q + (long long)(nc - 1 + m) * p.N + n, B[m]);
}

// Full own-frame coefficients of node n (FP64).
template <class S>
__device__ __forceinline__ void node_coefficients(const double* mac, const void* neq, long long N, int nord,
                                                  int split, double cv, long long n, double* A, double* B,
                                                  double& rho, double& ux, double& uy, double& T)
{
    const S* q = reinterpret_cast<const S*>(neq);
    const int nc = ncoef(nord);
    rho = mac[n];
    ux = mac[N + n];
    uy = mac[2 * N + n];
    T = mac[3 * N + n];
    A[0] = rho;
    for (int m = 1; m < nc; ++m) A[m] = sto_load<S>(q + (long long)(m - 1) * N + n);
    for (int m = 0; m < nc; ++m) B[m] = sto_load<S>(q + (long long)(nc - 1 + m) * N + n);
    GEq e = g_equilibrium(split, cv, rho, ux, uy, T, sqrt(T));
    B[slot(0, 0)] += e.b00;
    B[slot(1, 0)] += e.b10;
    B[slot(0, 1)] += e.b01;
    B[slot(2, 0)] += e.b20;
    B[slot(0, 2)] += e.b20;
}

template <class S>
__device__ __forceinline__ void node_coefficients(const AuxParams& p, long long n, double* A, double* B,
                                                  double& rho, double& ux, double& uy, double& T)
{
    node_coefficients<S>(p.mac, p.neq, p.N, p.nord, p.split, p.cv, n, A, B, rho, ux, uy, T);
}

// Moments of the populations (Sec. II): rho = A_00, rho u = rho u_frame + sqrt(T) (A_10, A_01),
// total split E = B_00, T = (E/rho - |u|^2/2)/c_v; internal split: T of the frame, the
// temperature of the last collision (its stored B_00 holds U + (1/2) sum G, see the source);
// non-translational split E = B_00 + sum |C|^2/2 f with
// sum |C|^2/2 f = (T (A_20 + A_02 + 2 rho) + 2 sqrt(T) u_frame . (A_10, A_01) + |u_frame|^2 rho)/2.
// Written to out[0..3][n] (rho, u_x, u_y, T); null arrays are skipped.
//
// Mixed modes (storage S narrower than double): the same moments written relative to the
// stored frame (u_f, T_f), whose non-equilibrium coefficients are the only non-FP64 inputs:
// with d = u - u_f = sqrt(T_f) (A_10, A_01) / rho and b = B_00 - B_00^eq,
//   total split            T = T_f + (b / rho - u_f . d - |d|^2 / 2) / c_v,
//   internal split         T = T_f,
//   non-translational      T = T_f + (b / rho + T_f (A_20 + A_02) / (2 rho) - |d|^2 / 2) / c_v
// (B_00^eq = rho (c_v T_f + |u_f|^2/2), rho c_v T_f, rho (c_v - 1) T_f).  The corrections are
// formed in FP32 and added to the FP64 frame once: FP64 is slow on this part, and the
// coefficients carry FP32 (or narrower) precision in these modes anyway.
template <class S>
__device__ __forceinline__ void node_moments(const double* mac, const void* neq, long long N, int nord,
                                             int split, double cv, long long n, double* const* out)
{
    double rho, vx, vy, t;
    if constexpr (std::is_same<S, double>::value) {
        double A[NCMAX], B[NCMAX], ux, uy, T;
        node_coefficients<S>(mac, neq, N, nord, split, cv, n, A, B, rho, ux, uy, T);
        double sT = sqrt(T);
        vx = ux + sT * A[slot(1, 0)] / rho;
        vy = uy + sT * A[slot(0, 1)] / rho;
        double E = B[0];
        if (split == 2)
            E += 0.5 * (T * (A[slot(2, 0)] + A[slot(0, 2)] + 2.0 * rho) +
                        2.0 * sT * (ux * A[slot(1, 0)] + uy * A[slot(0, 1)]) + (ux * ux + uy * uy) * rho);
        t = (split == 1) ? T : (E / rho - 0.5 * (vx * vx + vy * vy)) / cv;
    } else {
        const S* q = reinterpret_cast<const S*>(neq);
        const int nc = ncoef(nord);
        rho = mac[n];
        const double ux = mac[N + n], uy = mac[2 * N + n], T = mac[3 * N + n];
        const float a10 = sto_loadf<S>(q + (long long)(slot(1, 0) - 1) * N + n);
        const float a01 = sto_loadf<S>(q + (long long)(slot(0, 1) - 1) * N + n);
        const float b = sto_loadf<S>(q + (long long)(nc - 1) * N + n);
        const float ir = 1.0f / (float)rho, Tf = (float)T, icv = 1.0f / (float)cv;
        const float sT = sqrtf(Tf);
        const float dx = sT * a10 * ir, dy = sT * a01 * ir;
        float e = split == 1 ? 0.0f : b * ir;
        if (split == 0) {
            e -= (float)ux * dx + (float)uy * dy + 0.5f * (dx * dx + dy * dy);
        } else if (split == 2) {
            const float a20 = sto_loadf<S>(q + (long long)(slot(2, 0) - 1) * N + n);
            const float a02 = sto_loadf<S>(q + (long long)(slot(0, 2) - 1) * N + n);
            e += 0.5f * Tf * (a20 + a02) * ir - 0.5f * (dx * dx + dy * dy);
        }
        vx = ux + (double)dx;
        vy = uy + (double)dy;
        t = T + (double)(e * icv);
    }
    if (out[0]) out[0][n] = rho;
    if (out[1]) out[1][n] = vx;
    if (out[2]) out[2][n] = vy;
    if (out[3]) out[3][n] = t;
}

template <class S>
__global__ void moments_kernel(AuxParams p, double* out_rho, double* out_ux, double* out_uy,
                               double* out_T)
{
    long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= p.N) return;
    double* const out[4] = {out_rho, out_ux, out_uy, out_T};
    node_moments<S>(p.mac, p.neq, p.N, p.nord, p.split, p.cv, n, out);
}

// Populations in each node's own frame: f_i = w_i sum A_pq He_p(c_a) He_q(c_b) / (p! q!).
template <class S>
__global__ void get_pops_kernel(AuxParams p, double* f, double* g, double* oux, double* ouy, double* oT)
{
    long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= p.N) return;
    const Lattice& L = p.lat;
    double A[NCMAX], B[NCMAX], rho, ux, uy, T;
    node_coefficients<S>(p, n, A, B, rho, ux, uy, T);
    const int q1 = L.q1, no = p.nord;
    for (int b = 0; b < q1; ++b)
        for (int a = 0; a < q1; ++a) {
            double sf = 0.0, sg = 0.0;
            for (int pp = 0; pp <= no; ++pp)
                for (int qq = 0; qq <= no - pp; ++qq) {
                    double h = L.hn[a][pp] * L.hn[b][qq];
                    sf += A[slot(pp, qq)] * h;
                    sg += B[slot(pp, qq)] * h;
                }
            long long i = (long long)(b * q1 + a) * p.N + n;
            double w = L.w[a] * L.w[b];
            if (f) f[i] = w * sf;
            if (g) g[i] = w * sg;
        }
    if (oux) oux[n] = ux;
    if (ouy) ouy[n] = uy;
    if (oT) oT[n] = T;
}

// Internal-energy split source (Eq. int_g_evolution; Appendix A, G term):
//   G_i = -rho w_i (C_i - u) . (d_t u + C_i . grad u)   (f -> f_eq inside the source),
// in Hermite coefficients of the node's frame G_00 = -rho T div u, G_10 = -rho sqrt(T) Du_x,
// G_01 = -rho sqrt(T) Du_y, G_20 = -2 rho T d_x u_x, G_11 = -rho T (d_y u_x + d_x u_y),
// G_02 = -2 rho T d_y u_y (Du = d_t u + u . grad u).  add_source_node adds factor * G to the
// stored g coefficients of node n = (x, y): grad u by central differences of the velocity
// fields vux, vuy (boundary-mapped; beyond a prescribed side its velocity), the node's own
// rho, u, T and d_t u given.
template <class S>
__device__ __forceinline__ void add_source_node(long long n, int x, int y, int nx, int ny, int bc_x, int bc_y,
                                                long long N, int nord, const double* vux, const double* vuy,
                                                const double (*wall)[4], const double* const* prof, double rho,
                                                double ux, double uy, double T, double dtux_d, double dtuy_d,
                                                double factor, void* neq)
{
    const int nb[4][2] = {{x + 1, y}, {x - 1, y}, {x, y + 1}, {x, y - 1}};
    double vx[4], vy[4];
    for (int k = 0; k < 4; ++k) {
        const int w = wall_of(bc_x, bc_y, nx, ny, nb[k][0], nb[k][1]);
        if (w >= 0) {
            const double* st = side_state(wall, prof, nx, ny, w, nb[k][0], nb[k][1]);
            vx[k] = st[0];
            vy[k] = st[1];
        } else {
            const long long m = (long long)bc_map(nb[k][1], ny, bc_y) * nx + bc_map(nb[k][0], nx, bc_x);
            vx[k] = vux[m];
            vy[k] = vuy[m];
        }
    }
    S* q = reinterpret_cast<S*>(neq);
    if constexpr (std::is_same<S, double>::value) {
        double dxux = 0.5 * (vx[0] - vx[1]), dyux = 0.5 * (vx[2] - vx[3]);
        double dxuy = 0.5 * (vy[0] - vy[1]), dyuy = 0.5 * (vy[2] - vy[3]);
        double Dux = dtux_d + ux * dxux + uy * dyux;
        double Duy = dtuy_d + ux * dxuy + uy * dyuy;
        double rT = rho * T, rsT = rho * sqrt(T);
        double G[6] = {-rT * (dxux + dyuy), -rsT * Dux, -rsT * Duy, -2.0 * rT * dxux,
                       -rT * (dyux + dxuy), -2.0 * rT * dyuy};
        for (int m = 0; m < 6; ++m) {
            S* a = q + (long long)(ncoef(nord) - 1 + m) * N + n;
            sto_put<S, double>(a, sto_load<S>(a) + factor * G[m]);
        }
    } else {
        // mixed modes: the velocity differences taken in FP64 (small against u), the source
        // formed in FP32 like the coefficients it is added to (FP64 is slow on this part)
        const float dxux = 0.5f * (float)(vx[0] - vx[1]), dyux = 0.5f * (float)(vx[2] - vx[3]);
        const float dxuy = 0.5f * (float)(vy[0] - vy[1]), dyuy = 0.5f * (float)(vy[2] - vy[3]);
        const float dtux = (float)dtux_d, dtuy = (float)dtuy_d;
        const float uxf = (float)ux, uyf = (float)uy, rf = (float)rho, Tf = (float)T, fac = (float)factor;
        const float Dux = dtux + uxf * dxux + uyf * dyux;
        const float Duy = dtuy + uxf * dxuy + uyf * dyuy;
        const float rT = rf * Tf, rsT = rf * sqrtf(Tf);
        const float G[6] = {-rT * (dxux + dyuy), -rsT * Dux, -rsT * Duy, -2.0f * rT * dxux,
                            -rT * (dyux + dxuy), -2.0f * rT * dyuy};
        for (int m = 0; m < 6; ++m) {
            S* a = q + (long long)(ncoef(nord) - 1 + m) * N + n;
            sto_put<S, float>(a, sto_loadf<S>(a) + fac * G[m]);
        }
    }
}

// The source of the step (trapezoidal rule along the characteristics): (1 - omega/2) G with
// the new state (mac), d_t u by the backward difference against the frame before the step
// (mac_prev), grad u of the new frames; omega = 1/(tau + 1/2), tau = mu/(rho T).
template <class S>
__device__ __forceinline__ void internal_source_node(long long n, int nx, int ny, int bc_x, int bc_y,
                                                     long long N, int nord, double mu, const double* mac,
                                                     const double* mac_prev, void* neq,
                                                     const double (*wall)[4], const double* const* prof)
{
    // 32-bit division where the grid allows it (64-bit division is a long software sequence)
    const int x = N <= 0x7fffffffll ? (int)n % nx : (int)(n % nx);
    const int y = N <= 0x7fffffffll ? (int)n / nx : (int)(n / nx);
    const double rho = mac[n], ux = mac[N + n], uy = mac[2 * N + n], T = mac[3 * N + n];
    double factor;
    if constexpr (std::is_same<S, double>::value) {
        factor = 1.0 - 0.5 / (mu / (rho * T) + 0.5);
    } else {   // FP32: FP64 divisions are slow on this part, and G is formed in FP32 here
        factor = (double)(1.0f - 0.5f / ((float)mu / ((float)rho * (float)T) + 0.5f));
    }
    add_source_node<S>(n, x, y, nx, ny, bc_x, bc_y, N, nord, mac + N, mac + 2 * N, wall, prof, rho, ux, uy, T,
                       ux - mac_prev[N + n], uy - mac_prev[2 * N + n], factor, neq);
}

template <class S>
__global__ void internal_source_kernel(AuxParams p)
{
    long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= p.N) return;
    internal_source_node<S>(n, p.nx, p.ny, p.bc_x, p.bc_y, p.N, p.nord, p.mu, p.mac, p.mac_prev, p.neq, p.wall,
                            p.prof);
}

// Batched auxiliary launches: block b works on nodes [256 (b - block_start[c]), ...) of member
// c, the last of members [c0, c1) with block_start[c] <= b.
__device__ __forceinline__ int member_of_block(const int* block_start, int c0, int c1, int b)
{
    int lo = c0, hi = c1 - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (block_start[mid] <= b) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Batched internal source; members of the total split return at once.
template <class S>
__global__ void internal_source_batch_kernel(const CaseDesc* cases, const int* block_start, int ncase,
                                             int flip)
{
    const int b = (int)blockIdx.x;
    const int lo = member_of_block(block_start, 0, ncase, b);
    const CaseDesc& c = cases[lo];
    if (c.split != 1) return;
    const long long n = (long long)(b - block_start[lo]) * blockDim.x + threadIdx.x;
    if (n >= c.N) return;
    const int in = c.cur ^ flip;          // the state before the step; the new one is in ^ 1
    internal_source_node<S>(n, c.nx, c.ny, c.bc_x, c.bc_y, c.N, c.nord, c.mu, c.mac[in ^ 1], c.mac[in],
                            c.neq[in ^ 1], c.wall, c.prof);
}

// Batched init and moments over members [c0, c1) of a batch (blocks from block_start[c0] = block0
// on): each member's current state is buffer cur ^ flip; the fields of member c are
// fld.f[c - c0].  Same per-node arithmetic as init_kernel and moments_kernel.
template <class S>
__global__ void init_batch_kernel(const CaseDesc* cases, const int* block_start, int c0, int c1, int block0,
                                  int flip, MemberFields fld)
{
    const int b = block0 + (int)blockIdx.x;
    const int c = member_of_block(block_start, c0, c1, b);
    const CaseDesc& d = cases[c];
    const long long n = (long long)(b - block_start[c]) * blockDim.x + threadIdx.x;
    if (n >= d.N) return;
    if (d.status->flags & kInputBad) return;   // the input check before rejected it: state unchanged
    const int cur = d.cur ^ flip;
    const double* const* in = fld.f[c - c0];
    init_node<S>(d.mac[cur], d.neq[cur], d.N, d.nord, d.status, n, in[0][n], in[1][n], in[2][n], in[3][n]);
    if (d.split == 1)
        init_internal_source<S>(n, d.nx, d.ny, d.bc_x, d.bc_y, d.N, d.nord, in[1], in[2], d.wall, d.prof, in[0][n],
                                in[3][n], d.neq[cur]);
}

template <class S>
__global__ void moments_batch_kernel(const CaseDesc* cases, const int* block_start, int c0, int c1, int block0,
                                     int flip, MemberFields fld)
{
    const int b = block0 + (int)blockIdx.x;
    const int c = member_of_block(block_start, c0, c1, b);
    const CaseDesc& d = cases[c];
    const long long n = (long long)(b - block_start[c]) * blockDim.x + threadIdx.x;
    if (n >= d.N) return;
    const int cur = d.cur ^ flip;
    node_moments<S>(d.mac[cur], d.neq[cur], d.N, d.nord, d.split, d.cv, n, fld.f[c - c0]);
}

}  // namespace pond
