// The fused PonD time step (Sec. III.A): one CUDA thread per target node, one CTA per tile.
//
// 1. Staging.  The CTA takes the frame lambda_r of its centre node as reference and, for every
//    source node of the tile's interpolation footprint (a box sized per tile from the
//    departure points of its nodes), moves that node's Hermite coefficients of order <= 3
//    into lambda_r (Eq. gradGeneralTransform, via the re-centring matrices) and stores, in
//    shared memory, their DEVIATION from the reference node's equilibrium coefficients
//    K = (rho_r, 0, ...) for f and B_eq(rho_r, u_r, T_r) for g.  Every large difference of
//    equilibrium-dominated quantities (rho_s - rho_r, E_s - E_r, p_s u_s - p_r u_r,
//    p_s T_s - p_r T_r) is formed in FP64; the rest are products of small shifts and are
//    formed in the working precision R.  So in mixed precision the FP32 values carry only
//    deviations, and the reference part is added back in FP64.
// 2. Predictor-corrector (frame lambda_bar, guess = the node's previous frame).  For each
//    population i = (a, b): departure point x - C_i(lambda_bar) dt, Lagrange weights,
//    interpolation of the staged deviations (Eq. propagationInterpolated; the transform is
//    linear, so interpolating coefficients in the common frame lambda_r and moving the
//    result into lambda_bar equals moving every stencil node first), then the population
//    deviation f'_i = gamma_i . D, where gamma_i folds the lambda_r -> lambda_bar move and the
//    Grad reconstruction of component i.  Since sum_i gamma_i . K = K_00 exactly, the moments
//    are rho = rho_r + sum f', E = E_r + sum g' and rho (u - u_bar) = rho_r (u_r - u_bar) +
//    sqrt(T_bar) sum c_i f'_i.  Iterate to the tolerance or the cap (or exactly K times).
// 3. Collision.  The streamed populations' Hermite coefficients are moved into the frame of
//    their moments lambda* (reference part analytically, deviation part by re-centring) and
//    relaxed there (BGK, tau = mu/p, omega = 1/(tau + 1/2)); rho, u*, T* (FP64) and the
//    non-equilibrium coefficients are written.
//
// A stencil that leaves the staged box (a frame far outside the per-tile estimate) is read
// from global memory instead, node by node, and counted.
#pragma once

#include "pond_device.cuh"

namespace pond {

struct StepParams {
    Lattice lat;
    int nx, ny, bc_x, bc_y, split, pc_max_iter, pc_fixed;
    int box_w, box_h;           // staged box capacity (nodes)
    long long N;                // nx * ny
    double cv, inv_cv, mu, pc_tol;
    const double* mac_in;       // [4][N]: rho, u_x, u_y, T at time n
    const void* neq_in;         // [19][N] storage type S
    double* mac_out;
    void* neq_out;
    DevStatus* status;
};

// Tile reference state: the centre node's frame and its equilibrium-derived scalars (FP64).
template <class R>
struct RefState {
    double rho, ux, uy, T, E, P, PT, Pux, Puy;   // P = rho T; E = B_00^eq
    double invT;                                 // 1 / T
    R isT, invTR;                                // 1/sqrt(T), 1/T in R
};

// 1-D re-centring matrix with an accurately formed sigma = s^2 - 1 (see make_tau).
template <class R>
__device__ __forceinline__ Tau<R> make_tau_sig(R s, R d, R sig)
{
    Tau<R> t;
    R e = sig + d * d;
    t.t10 = d;
    t.t11 = s;
    t.t20 = e;
    t.t21 = R(2) * s * d;
    t.t22 = R(1) + sig;
    t.t30 = d * (R(3) * e - R(2) * d * d);
    t.t31 = R(3) * s * e;
    t.t32 = R(3) * (R(1) + sig) * d;
    t.t33 = (R(1) + sig) * s;
    return t;
}

template <class R>
__device__ __forceinline__ R sqrt_r(R v)
{
    if constexpr (std::is_same<R, double>::value) return sqrt(v); else return sqrtf(v);
}

// 1/x for x > 0 to FP64 accuracy without a double division: FP32 estimate, two Newton steps.
__device__ __forceinline__ double rcp64(double x)
{
    double r = (double)(1.0f / (float)x);
    r = r * (2.0 - x * r);
    r = r * (2.0 - x * r);
    return r;
}

// Deviation of node nd's coefficients, moved into the reference frame, from the reference
// node's equilibrium coefficients.
template <class S, class R>
__device__ __forceinline__ void source_dev(const StepParams& p, const RefState<R>& rf, long long nd,
                                           R* Df, R* Dg)
{
    const long long N = p.N;
    const S* neq = reinterpret_cast<const S*>(p.neq_in);
    const double rho = p.mac_in[nd], ux = p.mac_in[N + nd], uy = p.mac_in[2 * N + nd];
    const double T = p.mac_in[3 * N + nd];
    // shifts of this node's frame relative to the reference frame
    const R dx = R(ux - rf.ux) * rf.isT;
    const R dy = R(uy - rf.uy) * rf.isT;
    const R sig = R(T - rf.T) * rf.invTR;            // T/T_r - 1
    const R s = sqrt_r<R>(R(1) + sig);               // sqrt(T/T_r)
    const Tau<R> tx = make_tau_sig<R>(s, dx, sig);
    const Tau<R> ty = make_tau_sig<R>(s, dy, sig);
    // non-equilibrium parts, moved (small numbers: working precision)
    R A[NCOEF], B[NCOEF];
    A[0] = R(0);
#pragma unroll
    for (int k = 1; k < NCOEF; ++k) A[k] = sto_get<S, R>(neq + (long long)(k - 1) * N + nd);
#pragma unroll
    for (int k = 0; k < NCOEF; ++k) B[k] = sto_get<S, R>(neq + (long long)(9 + k) * N + nd);
    retarget(tx, ty, A, Df);
    retarget(tx, ty, B, Dg);
    // f equilibrium: rho tx_p0 ty_q0, minus K_f = rho_r at (0,0)
    const R rr = R(rho);
    const R hx[4] = {R(1), tx.t10, tx.t20, tx.t30};
    const R hy[4] = {R(1), ty.t10, ty.t20, ty.t30};
    Df[0] += R(rho - rf.rho);
#pragma unroll
    for (int pp = 0; pp <= 3; ++pp)
#pragma unroll
        for (int q = 0; q <= 3 - pp; ++q)
            if (pp + q > 0) Df[slot(pp, q)] += rr * hx[pp] * hy[q];
    // g equilibrium (Sec. II g_eq in the node's frame), moved, minus K_g
    const double P = rho * T;
    const R PuxR = R(P * ux) * rf.isT, PuyR = R(P * uy) * rf.isT;   // rho sqrt(T) u * s (moved b10)
    const double dPT = P * T - rf.PT;
    if (p.split == 0) {
        const double E = rho * (p.cv * T + 0.5 * (ux * ux + uy * uy));
        const R Er = R(E);
        Dg[slot(0, 0)] += R(E - rf.E);
        Dg[slot(1, 0)] += dx * Er + R(P * ux - rf.Pux) * rf.isT;
        Dg[slot(0, 1)] += dy * Er + R(P * uy - rf.Puy) * rf.isT;
        Dg[slot(2, 0)] += tx.t20 * Er + R(2) * dx * PuxR + R(dPT * rf.invT);
        Dg[slot(0, 2)] += ty.t20 * Er + R(2) * dy * PuyR + R(dPT * rf.invT);
        Dg[slot(1, 1)] += dx * dy * Er + dx * PuyR + dy * PuxR;
        const R PsR = R(P) * (R(1) + sig);          // s^2 P
        Dg[slot(3, 0)] += tx.t30 * Er + R(3) * tx.t20 * PuxR + R(3) * dx * PsR;
        Dg[slot(0, 3)] += ty.t30 * Er + R(3) * ty.t20 * PuyR + R(3) * dy * PsR;
        Dg[slot(2, 1)] += tx.t20 * dy * Er + tx.t20 * PuyR + R(2) * dx * dy * PuxR + dy * PsR;
        Dg[slot(1, 2)] += ty.t20 * dx * Er + ty.t20 * PuxR + R(2) * dx * dy * PuyR + dx * PsR;
    } else {
        const R Ur = R(p.cv * P);
        const R PsR = R(P) * (R(1) + sig);
        Dg[slot(0, 0)] += R(p.cv * (P - rf.P));
        Dg[slot(1, 0)] += dx * Ur;
        Dg[slot(0, 1)] += dy * Ur;
        Dg[slot(2, 0)] += tx.t20 * Ur + R(dPT * rf.invT);
        Dg[slot(0, 2)] += ty.t20 * Ur + R(dPT * rf.invT);
        Dg[slot(1, 1)] += dx * dy * Ur;
        Dg[slot(3, 0)] += tx.t30 * Ur + R(3) * dx * PsR;
        Dg[slot(0, 3)] += ty.t30 * Ur + R(3) * dy * PsR;
        Dg[slot(2, 1)] += tx.t20 * dy * Ur + dy * PsR;
        Dg[slot(1, 2)] += ty.t20 * dx * Ur + dx * PsR;
    }
}

// Per-population lattice values, kept in shared memory so that the population loops can run
// without unrolling (the unrolled body would not fit the instruction cache).
template <class R>
struct LatRow {
    R c, w, he[4], hn[4];
};

// V_b(p, l) = sum_{q = l}^{3 - p} hn_b(q) ty_ql (shared by all a of one b).
template <class R>
__device__ __forceinline__ void make_V(const LatRow<R>& lb, const Tau<R>& ty, R* V)
{
#pragma unroll
    for (int pp = 0; pp <= 3; ++pp)
#pragma unroll
        for (int l = 0; l <= 3 - pp; ++l) {
            R v = R(0);
#pragma unroll
            for (int q = l; q <= 3 - pp; ++q) v += lb.hn[q] * tau_at(ty, q, l);
            V[slot(pp, l)] = v;
        }
}

// gamma_kl of population (a, b): f_ab = sum_kl gamma_kl R_kl for coefficients R in lambda_r,
//   gamma_kl = w_a w_b sum_{p >= k, q >= l, p + q <= 3} hn_a(p) tx_pk hn_b(q) ty_ql.
template <class R>
__device__ __forceinline__ void make_gamma(const LatRow<R>& la, R wab, const Tau<R>& tx, const R* V,
                                           R* gam)
{
    R U[4][4];
#pragma unroll
    for (int pp = 0; pp <= 3; ++pp)
#pragma unroll
        for (int k = 0; k <= pp; ++k) U[pp][k] = la.hn[pp] * tau_at(tx, pp, k);
#pragma unroll
    for (int k = 0; k <= 3; ++k)
#pragma unroll
        for (int l = 0; l <= 3 - k; ++l) {
            R g = R(0);
#pragma unroll
            for (int pp = k; pp <= 3 - l; ++pp) g += U[pp][k] * V[slot(pp, l)];
            gam[slot(k, l)] = wab * g;
        }
}

template <class S, class R, int Q1, int P, bool ONE_D, int TPB>
__global__ void __launch_bounds__(TPB, 1) step_kernel(const StepParams p)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    R* sm = reinterpret_cast<R*>(smem_raw);
    __shared__ float red[4][TPB / 32];
    __shared__ int box[4];
    __shared__ LatRow<R> lat[Q1];
    __shared__ RefState<R> srf;

    const int TX = blockDim.x, TY = blockDim.y;
    const int tid = threadIdx.y * TX + threadIdx.x;
    const int x = blockIdx.x * TX + threadIdx.x;
    const int y = blockIdx.y * TY + threadIdx.y;
    const bool active = (x < p.nx) && (y < p.ny);
    const long long N = p.N;
    const long long node = active ? (long long)y * p.nx + x : 0;
    const Lattice& L = p.lat;

    if (tid < Q1) {
        LatRow<R> r;
        r.c = lat_c<R>(L, tid);
        r.w = lat_w<R>(L, tid);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            r.he[k] = lat_he<R>(L, tid, k);
            r.hn[k] = lat_hn<R>(L, tid, k);
        }
        lat[tid] = r;
    }

    // ---- own frame (predictor) and the tile's reference state ------------------------------
    double ux0 = 0.0, uy0 = 0.0, T0 = 1.0;
    if (active) {
        ux0 = p.mac_in[N + node];
        uy0 = p.mac_in[2 * N + node];
        T0 = p.mac_in[3 * N + node];
    }
    if (tid == 0) {
        RefState<R> rf;
        const int cxn = min(blockIdx.x * TX + TX / 2, p.nx - 1);
        const int cyn = min(blockIdx.y * TY + TY / 2, p.ny - 1);
        const long long c = (long long)cyn * p.nx + cxn;
        rf.rho = p.mac_in[c];
        rf.ux = p.mac_in[N + c];
        rf.uy = p.mac_in[2 * N + c];
        rf.T = p.mac_in[3 * N + c];
        rf.P = rf.rho * rf.T;
        rf.PT = rf.P * rf.T;
        rf.Pux = rf.P * rf.ux;
        rf.Puy = rf.P * rf.uy;
        rf.E = (p.split == 0) ? rf.rho * (p.cv * rf.T + 0.5 * (rf.ux * rf.ux + rf.uy * rf.uy))
                              : p.cv * rf.P;
        rf.invT = rcp64(rf.T);
        rf.invTR = R(rf.invT);
        rf.isT = R(1) / sqrt_r<R>(R(rf.T));
        srf = rf;
    }
    __syncthreads();
    const RefState<R>& rf = srf;
    const R sTr = sqrt_r<R>(R(rf.T));

    // ---- per-tile interpolation footprint --------------------------------------------------
    {
        float cm = (float)L.cmax;
        float sT0 = sqrtf(fmaxf((float)T0, 0.f));
        float lx = active ? -(float)ux0 - cm * sT0 : 1e30f;
        float hx = active ? -(float)ux0 + cm * sT0 : -1e30f;
        float ly = active ? -(float)uy0 - cm * sT0 : 1e30f;
        float hy = active ? -(float)uy0 + cm * sT0 : -1e30f;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            lx = fminf(lx, __shfl_xor_sync(0xffffffffu, lx, o));
            hx = fmaxf(hx, __shfl_xor_sync(0xffffffffu, hx, o));
            ly = fminf(ly, __shfl_xor_sync(0xffffffffu, ly, o));
            hy = fmaxf(hy, __shfl_xor_sync(0xffffffffu, hy, o));
        }
        const int warp = tid >> 5, lane = tid & 31;
        if (lane == 0) {
            red[0][warp] = lx; red[1][warp] = hx; red[2][warp] = ly; red[3][warp] = hy;
        }
        __syncthreads();
        if (tid == 0) {
            for (int w = 1; w < TPB / 32; ++w) {
                lx = fminf(lx, red[0][w]); hx = fmaxf(hx, red[1][w]);
                ly = fminf(ly, red[2][w]); hy = fmaxf(hy, red[3][w]);
            }
            const float margin = 0.5f;   // room for the frame to move during the iterations
            // taps of a departure offset `off` lie in [floor(off) - 1, floor(off) + 2]
            int x_lo = (int)floorf(fmaxf(lx - margin, -1e6f)) - 1;
            int x_hi = (TX - 1) + (int)floorf(fminf(hx + margin, 1e6f)) + 2;
            int y_lo = (int)floorf(fmaxf(ly - margin, -1e6f)) - 1;
            int y_hi = (TY - 1) + (int)floorf(fminf(hy + margin, 1e6f)) + 2;
            box[0] = blockIdx.x * TX + x_lo;
            box[1] = ONE_D ? 0 : blockIdx.y * TY + y_lo;
            box[2] = min(x_hi - x_lo + 1, p.box_w);
            box[3] = ONE_D ? 1 : min(y_hi - y_lo + 1, p.box_h);
        }
        __syncthreads();
    }
    const int ox = box[0], oy = box[1], bw = box[2], bh = box[3];
    const int bn = bw * bh;

    // ---- staging: source deviations in the reference frame --------------------------------
    for (int i = tid; i < bn; i += TPB) {
        int lx = i % bw, ly = i / bw;
        int sx = bc_map(ox + lx, p.nx, p.bc_x);
        int sy = ONE_D ? 0 : bc_map(oy + ly, p.ny, p.bc_y);
        R Df[NCOEF], Dg[NCOEF];
        source_dev<S, R>(p, rf, (long long)sy * p.nx + sx, Df, Dg);
#pragma unroll
        for (int m = 0; m < NCOEF; ++m) {
            sm[m * bn + i] = Df[m];
            sm[(NCOEF + m) * bn + i] = Dg[m];
        }
    }
    __syncthreads();

    // ---- predictor-corrector ---------------------------------------------------------------
    int k = 0;
    bool bad = false, nonconv = false;
    unsigned int fallbacks = 0;
    double ubx = ux0, uby = uy0, Tb = T0;
    double rho = 1.0, unx = ux0, uny = uy0, Tn = T0;
    R Af[NCOEF], Ag[NCOEF];   // deviation coefficients of the streamed populations in lambda_bar

    if (active) {
        while (true) {
            const R sT = sqrt_r<R>(R(Tb));
            const R isT = R(1) / sT;
            const R sig_t = R(rf.T - Tb) * R(rcp64(Tb));      // T_r / T_bar - 1
            const R s_t = sTr * isT;
            const Tau<R> txr = make_tau_sig<R>(s_t, R(rf.ux - ubx) * isT, sig_t);
            const Tau<R> tyr = make_tau_sig<R>(s_t, R(rf.uy - uby) * isT, sig_t);
            const R ubxr = R(ubx), ubyr = R(uby);
#pragma unroll
            for (int m = 0; m < NCOEF; ++m) { Af[m] = R(0); Ag[m] = R(0); }

            if constexpr (!ONE_D) {
#pragma unroll 1
                for (int b = 0; b < Q1; ++b) {
                    const LatRow<R>& lb = lat[b];
                    R wy[P];
                    const int jy = lagrange<R, P>(-(sT * lb.c + ubyr), wy);
                    const int ty0 = y + jy - oy;
                    R V[NCOEF];
                    make_V<R>(lb, tyr, V);
                    R Sf[4] = {R(0), R(0), R(0), R(0)}, Sg[4] = {R(0), R(0), R(0), R(0)};
#pragma unroll 1
                    for (int a = 0; a < Q1; ++a) {
                        const LatRow<R>& la = lat[a];
                        R wx[P];
                        const int jx = lagrange<R, P>(-(sT * la.c + ubxr), wx);
                        const int tx0 = x + jx - ox;
                        R gam[NCOEF];
                        make_gamma<R>(la, la.w * lb.w, txr, V, gam);
                        R Ri[2 * NCOEF];
#pragma unroll
                        for (int m = 0; m < 2 * NCOEF; ++m) Ri[m] = R(0);
                        if (tx0 >= 0 && tx0 + P <= bw && ty0 >= 0 && ty0 + P <= bh) {
#pragma unroll
                            for (int j = 0; j < P; ++j) {
                                // one stencil row per fence: bounds the loads in flight
                                asm volatile("" ::: "memory");
#pragma unroll
                                for (int ii = 0; ii < P; ++ii) {
                                    const R W = wy[j] * wx[ii];
                                    const R* src = sm + (ty0 + j) * bw + tx0 + ii;
#pragma unroll
                                    for (int m = 0; m < 2 * NCOEF; ++m) Ri[m] += W * src[m * bn];
                                }
                            }
                        } else {
                            ++fallbacks;
                            for (int j = 0; j < P; ++j)
                                for (int ii = 0; ii < P; ++ii) {
                                    const R W = wy[j] * wx[ii];
                                    const int sx = bc_map(x + jx + ii, p.nx, p.bc_x);
                                    const int sy = bc_map(y + jy + j, p.ny, p.bc_y);
                                    R Df[NCOEF], Dg[NCOEF];
                                    source_dev<S, R>(p, rf, (long long)sy * p.nx + sx, Df, Dg);
#pragma unroll
                                    for (int m = 0; m < NCOEF; ++m) {
                                        Ri[m] += W * Df[m];
                                        Ri[NCOEF + m] += W * Dg[m];
                                    }
                                }
                        }
                        R f = R(0), g = R(0);
#pragma unroll
                        for (int m = 0; m < NCOEF; ++m) {
                            f += gam[m] * Ri[m];
                            g += gam[m] * Ri[NCOEF + m];
                        }
#pragma unroll
                        for (int pp = 0; pp < 4; ++pp) {
                            Sf[pp] += f * la.he[pp];
                            Sg[pp] += g * la.he[pp];
                        }
                    }
#pragma unroll
                    for (int pp = 0; pp <= 3; ++pp)
#pragma unroll
                        for (int q = 0; q <= 3 - pp; ++q) {
                            Af[slot(pp, q)] += Sf[pp] * lb.he[q];
                            Ag[slot(pp, q)] += Sg[pp] * lb.he[q];
                        }
                }
            } else {
                // quasi-1-D (ny = 1): every y tap reads row 0 and the y weights sum to one, so
                // the interpolated coefficients depend on a only.
#pragma unroll 1
                for (int a = 0; a < Q1; ++a) {
                    const LatRow<R>& la = lat[a];
                    R wx[P];
                    const int jx = lagrange<R, P>(-(sT * la.c + ubxr), wx);
                    const int tx0 = x + jx - ox;
                    R Ri[2 * NCOEF];
#pragma unroll
                    for (int m = 0; m < 2 * NCOEF; ++m) Ri[m] = R(0);
                    if (tx0 >= 0 && tx0 + P <= bw) {
#pragma unroll
                        for (int ii = 0; ii < P; ++ii) {
                            const R W = wx[ii];
                            const R* src = sm + tx0 + ii;
#pragma unroll
                            for (int m = 0; m < 2 * NCOEF; ++m) Ri[m] += W * src[m * bn];
                        }
                    } else {
                        ++fallbacks;
                        for (int ii = 0; ii < P; ++ii) {
                            const R W = wx[ii];
                            const int sx = bc_map(x + jx + ii, p.nx, p.bc_x);
                            R Df[NCOEF], Dg[NCOEF];
                            source_dev<S, R>(p, rf, (long long)sx, Df, Dg);
#pragma unroll
                            for (int m = 0; m < NCOEF; ++m) {
                                Ri[m] += W * Df[m];
                                Ri[NCOEF + m] += W * Dg[m];
                            }
                        }
                    }
                    R Sf[4] = {R(0), R(0), R(0), R(0)}, Sg[4] = {R(0), R(0), R(0), R(0)};
#pragma unroll 1
                    for (int b = 0; b < Q1; ++b) {
                        const LatRow<R>& lb = lat[b];
                        R V[NCOEF], gam[NCOEF];
                        make_V<R>(lb, tyr, V);
                        make_gamma<R>(la, la.w * lb.w, txr, V, gam);
                        R f = R(0), g = R(0);
#pragma unroll
                        for (int m = 0; m < NCOEF; ++m) {
                            f += gam[m] * Ri[m];
                            g += gam[m] * Ri[NCOEF + m];
                        }
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            Sf[q] += f * lb.he[q];
                            Sg[q] += g * lb.he[q];
                        }
                    }
#pragma unroll
                    for (int pp = 0; pp <= 3; ++pp)
#pragma unroll
                        for (int q = 0; q <= 3 - pp; ++q) {
                            Af[slot(pp, q)] += la.he[pp] * Sf[q];
                            Ag[slot(pp, q)] += la.he[pp] * Sg[q];
                        }
                }
            }

            // ---- moments of the streamed populations (Sec. II) --------------------------------
            // reference part exact in FP64, deviation part from the working precision
            rho = rf.rho + (double)Af[slot(0, 0)];
            const double E = rf.E + (double)Ag[slot(0, 0)];
            const double irho = rcp64(rho);
            const double sTd = (double)sT;
            // rho (u - u_bar) = rho_r (u_r - u_bar) + sqrt(T_bar) sum c f'
            unx = ubx + (rf.rho * (rf.ux - ubx) + sTd * (double)Af[slot(1, 0)]) * irho;
            uny = uby + (rf.rho * (rf.uy - uby) + sTd * (double)Af[slot(0, 1)]) * irho;
            if (p.split == 0) Tn = (E * irho - 0.5 * (unx * unx + uny * uny)) * p.inv_cv;
            else Tn = E * irho * p.inv_cv;
            ++k;
            if (!(rho > 0.0) || !(Tn > 0.0) || isnan(unx) || isnan(uny)) { bad = true; break; }
            const float du = sqrtf((float)((unx - ubx) * (unx - ubx) + (uny - uby) * (uny - uby)));
            const float change = fmaxf(du * rsqrtf((float)Tb), fabsf((float)(Tn - Tb) / (float)Tb));
            bool stop;
            if (p.pc_fixed > 0) stop = (k >= p.pc_fixed);
            else if (change <= (float)p.pc_tol) stop = true;
            else if (k >= p.pc_max_iter) { stop = true; nonconv = true; }
            else stop = false;
            if (stop) break;
            ubx = unx; uby = uny; Tb = Tn;                       // corrector
        }
    }

    // ---- collision in the frame of the final moments and write-back ---------------------------
    if (active) {
        S* nout = reinterpret_cast<S*>(p.neq_out);
        p.mac_out[node] = rho;
        p.mac_out[N + node] = unx;
        p.mac_out[2 * N + node] = uny;
        p.mac_out[3 * N + node] = Tn;
        if (!bad) {
            const double iTn = rcp64(Tn);
            const R isTn = R(1) / sqrt_r<R>(R(Tn));
            // deviation part: lambda_bar -> lambda*
            {
                const R sig = R(Tb - Tn) * R(iTn);
                const R s = sqrt_r<R>(R(1) + sig);
                const Tau<R> tx = make_tau_sig<R>(s, R(ubx - unx) * isTn, sig);
                const Tau<R> ty = make_tau_sig<R>(s, R(uby - uny) * isTn, sig);
                retarget(tx, ty, Af, Af);
                retarget(tx, ty, Ag, Ag);
            }
            // reference part: K moved lambda_r -> lambda*, minus the equilibrium in lambda*
            const R sig = R(rf.T - Tn) * R(iTn);                 // T_r/T* - 1
            const R s = sqrt_r<R>(R(1) + sig);
            const R dx = R(rf.ux - unx) * isTn, dy = R(rf.uy - uny) * isTn;
            const Tau<R> tx = make_tau_sig<R>(s, dx, sig);
            const Tau<R> ty = make_tau_sig<R>(s, dy, sig);
            const R rr = R(rf.rho);
            const R hx[4] = {R(1), tx.t10, tx.t20, tx.t30};
            const R hy[4] = {R(1), ty.t10, ty.t20, ty.t30};
#pragma unroll
            for (int pp = 0; pp <= 3; ++pp)
#pragma unroll
                for (int q = 0; q <= 3 - pp; ++q)
                    if (pp + q >= 2) Af[slot(pp, q)] += rr * hx[pp] * hy[q];
            // g: T_{r->*}(K_g) - B_eq(rho, u*, T*) for the slots with p + q >= 1 (00 is zero by
            // definition of T*); the large differences are formed in FP64.
            const double Pn = rho * Tn;
            const R PruxR = R(rf.Pux) * isTn, PruyR = R(rf.Puy) * isTn;   // s b10_r
            if (p.split == 0) {
                const R Er = R(rf.E);
                Ag[slot(1, 0)] += dx * Er + R(rf.Pux - Pn * unx) * isTn;
                Ag[slot(0, 1)] += dy * Er + R(rf.Puy - Pn * uny) * isTn;
                Ag[slot(2, 0)] += tx.t20 * Er + R(2) * dx * PruxR + R((rf.PT - Pn * Tn) * iTn);
                Ag[slot(0, 2)] += ty.t20 * Er + R(2) * dy * PruyR + R((rf.PT - Pn * Tn) * iTn);
                Ag[slot(1, 1)] += dx * dy * Er + dx * PruyR + dy * PruxR;
                const R PsR = R(rf.P) * (R(1) + sig);
                Ag[slot(3, 0)] += tx.t30 * Er + R(3) * tx.t20 * PruxR + R(3) * dx * PsR;
                Ag[slot(0, 3)] += ty.t30 * Er + R(3) * ty.t20 * PruyR + R(3) * dy * PsR;
                Ag[slot(2, 1)] += tx.t20 * dy * Er + tx.t20 * PruyR + R(2) * dx * dy * PruxR + dy * PsR;
                Ag[slot(1, 2)] += ty.t20 * dx * Er + ty.t20 * PruxR + R(2) * dx * dy * PruyR + dx * PsR;
            } else {
                const R Ur = R(rf.E);
                const R PsR = R(rf.P) * (R(1) + sig);
                Ag[slot(1, 0)] += dx * Ur;
                Ag[slot(0, 1)] += dy * Ur;
                Ag[slot(2, 0)] += tx.t20 * Ur + R((rf.PT - Pn * Tn) * iTn);
                Ag[slot(0, 2)] += ty.t20 * Ur + R((rf.PT - Pn * Tn) * iTn);
                Ag[slot(1, 1)] += dx * dy * Ur;
                Ag[slot(3, 0)] += tx.t30 * Ur + R(3) * dx * PsR;
                Ag[slot(0, 3)] += ty.t30 * Ur + R(3) * dy * PsR;
                Ag[slot(2, 1)] += tx.t20 * dy * Ur + dy * PsR;
                Ag[slot(1, 2)] += ty.t20 * dx * Ur + dx * PsR;
            }
            const double tau = p.mu * rcp64(rho) * iTn;            // tau = mu / (rho T)
            const R keep = R(1) - R(1) / (R(tau) + R(0.5));        // 1 - omega
            // f: A*_10 = A*_01 = 0 and B*_00 = B_00^eq hold by definition of lambda*.
            sto_put<S, R>(nout + 0 * N + node, R(0));
            sto_put<S, R>(nout + 1 * N + node, R(0));
#pragma unroll
            for (int m = 3; m < NCOEF; ++m) sto_put<S, R>(nout + (long long)(m - 1) * N + node, keep * Af[m]);
            sto_put<S, R>(nout + 9 * N + node, R(0));
#pragma unroll
            for (int m = 1; m < NCOEF; ++m) sto_put<S, R>(nout + (long long)(9 + m) * N + node, keep * Ag[m]);
        } else {
            for (int m = 0; m < NNEQ; ++m) sto_put<S, R>(nout + (long long)m * N + node, R(NAN));
        }
    }

    // ---- statistics (one atomic per warp) -----------------------------------------------------
    {
        unsigned int kk = active ? (unsigned int)k : 0u;
        unsigned int nc = (active && nonconv) ? 1u : 0u;
        unsigned int sum_k = __reduce_add_sync(0xffffffffu, kk);
        unsigned int max_k = __reduce_max_sync(0xffffffffu, kk);
        unsigned int sum_nc = __reduce_add_sync(0xffffffffu, nc);
        unsigned int sum_fb = __reduce_add_sync(0xffffffffu, fallbacks);
        if ((tid & 31) == 0) {
            atomicAdd(&p.status->iters_total, (unsigned long long)sum_k);
            atomicMax(&p.status->iters_max, max_k);
            if (sum_nc) {
                atomicAdd(&p.status->nonconv, (unsigned long long)sum_nc);
                atomicOr(&p.status->flags, 2);
            }
            if (sum_fb) atomicAdd(&p.status->fallbacks, (unsigned long long)sum_fb);
        }
        if (active && bad) {
            atomicOr(&p.status->flags, 1);
            atomicMin(&p.status->first_bad, (unsigned long long)node);
        }
    }
}

}  // namespace pond
