// The fused PonD time step (Sec. III.A): one CUDA thread per target node, one CTA per tile.
//
// 1. Staging.  The CTA takes the frame lambda_r of its centre node as reference and, for every
//    source node of the tile's interpolation footprint (a box sized per tile from the
//    departure points of its nodes), moves that node's Hermite coefficients of order <= 3
//    into lambda_r (Eq. gradGeneralTransform, via the re-centring matrices) and stores, in
//    shared memory, their DEVIATION from the reference node's equilibrium coefficients
//    K = (rho_r, 0, ...) for f and B_eq(rho_r, u_r, T_r) for g.
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
// Precision.  rho, u, T are FP64 in memory.  Only their differences from the reference
// (rho_s - rho_r, u_s - u_r, T_s - T_r) and the frame corrections are formed with FP64 adds;
// every other large difference (E_s - E_r, p_s u_s - p_r u_r, p_s T_s - p_r T_r, the new
// temperature) is expanded into products of those small differences with O(1) values and
// evaluated in the working precision R, so in mixed precision FP32 only ever carries
// deviations and no FP64 multiply, divide or square root is needed in the loops.
//
// Interpolation.  For each a, the x pass is done once per row of the union of the y stencils
// of all b and folded at once (make_phi / z_contract) into the four values that the
// populations (a, b) need along y, which are then added to the b's whose y stencil contains
// the row.  Quasi-1-D grids fold the single row once per a.
//
// A stencil that leaves the staged box (a frame far outside the per-tile estimate) is read
// from global memory instead, node by node, and counted.
#pragma once

#include "pond_device.cuh"
#include "pond_launch.h"

namespace pond {

// One simulation's parameters and state buffers.  A single launch carries one case by value;
// a batched launch carries a device table of cases and the first tile of each.
struct CaseDesc {
    int nx, ny, bc_x, bc_y, split, pc_max_iter, pc_fixed;
    int nord;                   // Grad order N of the state (3 or 4; the lattice's)
    int tiles_x;                // tiles along x (tile index -> tile coordinates)
    long long N;                // nx * ny
    double cv, inv_cv, mu, pc_tol;
    float cv_f, inv_cv_f, mu_f, pc_tol_f;   // the same rounded to FP32 by the host (on this part a
                                // conversion from FP64 holds the FP64 pipe for 64 cycles a warp)
    double* mac[2];             // [4][N]: rho, u_x, u_y, T
    void* neq[2];               // [nneq(N)][N] storage type S
    int cur;                    // buffer holding the state when flip = 0
    DevStatus* status;
    double wall[4][4];          // prescribed sides x-low, x-high, y-low, y-high: (u_x, u_y, T, rho)
    const double* prof[4];      // per side: null (uniform wall[side]) or [n][4] states along it
    double* upred;              // internal split: [2][N] predictor velocities (u_x, u_y), followed by the
                                // [2 ncoef][N] coefficients (arithmetic type) of its streamed f and g;
                                // else null
};

struct StepParams {
    Lattice lat;
    int box_w, box_h;           // staged box capacity (nodes)
    int flip;                   // the input state is buffer cur ^ flip, the output the other one
    int ncase;                  // 0: the single case `one`; > 0: `cases` (batched launch)
    int ahead;                  // blocks resident at once (one wave); 0: no L2 prefetch
    CaseDesc one;
    const CaseDesc* cases;
    const int* tile_start;      // [ncase + 1]: first tile of each case, total at the end
};

// The case of this block, resolved once per block (kept in shared memory).
struct CaseRun {
    int nx, ny, bc_x, bc_y, split, pc_max_iter, pc_fixed;
    int tile_x, tile_y;
    long long N;
    double cv, inv_cv, mu, pc_tol;
    float cv_f, inv_cv_f, mu_f, pc_tol_f;
    const double* mac_in;
    const void* neq_in;
    double* mac_out;
    void* neq_out;
    DevStatus* status;
    double wall[4][4];
    const double* prof[4];
    double* upred;
};

// A case scalar in the arithmetic type: the FP64 value, or its FP32 copy rounded on the host.
template <class R>
__device__ __forceinline__ R case_r(double d, float f)
{
    if constexpr (std::is_same<R, double>::value) return d; else return R(f);
}

// Resolves the block's case (warp 0 calls it).  In a batched launch every lane runs the same
// binary search over the tile prefix, the warp copies the case record into shared memory in
// one round of 8-byte loads, and lane 0 fills the block's CaseRun from that copy.
static_assert(sizeof(CaseDesc) % 8 == 0, "CaseDesc is copied in 8-byte words");

// The case of launch tile b in a batched launch: the last c with start[c] <= b (start[0] = 0,
// start strictly increasing).  The 32 lanes of a converged warp call it together: each round
// splits the candidate range into 32 parts and the lanes test one bound each, so 256 cases take
// two rounds of loads instead of eight.
__device__ __forceinline__ int find_case(const int* start, int ncase, int b, int lane)
{
    int lo = 0, hi = ncase - 1;
    while (hi - lo >= 32) {
        const int span = hi - lo + 1;
        const int c = lo + (int)((long long)span * lane / 32);
        const unsigned m = __ballot_sync(0xffffffffu, start[c] <= b);
        const int L = 31 - __clz(m);                  // bit 0 is set: start[lo] <= b
        const int nlo = lo + (int)((long long)span * L / 32);
        if (L < 31) hi = lo + (int)((long long)span * (L + 1) / 32) - 1;
        lo = nlo;
    }
    const int c = lo + lane;
    const unsigned m = __ballot_sync(0xffffffffu, c <= hi && start[c] <= b);
    return lo + 31 - __clz(m);
}

__device__ __forceinline__ void resolve_case(const StepParams& p, CaseRun& r, CaseDesc& sdesc, int lane)
{
    const CaseDesc* c = &p.one;
    int tile_x = blockIdx.x, tile_y = blockIdx.y;
    if (p.ncase > 0) {
        const int b = (int)blockIdx.x;
        const int lo = find_case(p.tile_start, p.ncase, b, lane);
        const unsigned long long* src = reinterpret_cast<const unsigned long long*>(p.cases + lo);
        unsigned long long* dst = reinterpret_cast<unsigned long long*>(&sdesc);
        for (int k = lane; k < (int)(sizeof(CaseDesc) / 8); k += 32) dst[k] = src[k];
        __syncwarp();
        c = &sdesc;
        const int tile = b - p.tile_start[lo];
        tile_x = tile % c->tiles_x;
        tile_y = tile / c->tiles_x;
    }
    if (lane != 0) return;
    // the record read whole before any field of r is written: r and the batched copy both lie
    // in shared memory, and field by field each read would wait for the write before it
    const CaseDesc d = *c;
    r.tile_x = tile_x;
    r.tile_y = tile_y;
    r.nx = d.nx; r.ny = d.ny; r.bc_x = d.bc_x; r.bc_y = d.bc_y; r.split = d.split;
    r.pc_max_iter = d.pc_max_iter; r.pc_fixed = d.pc_fixed;
    r.N = d.N; r.cv = d.cv; r.inv_cv = d.inv_cv; r.mu = d.mu; r.pc_tol = d.pc_tol;
    r.cv_f = d.cv_f; r.inv_cv_f = d.inv_cv_f; r.mu_f = d.mu_f; r.pc_tol_f = d.pc_tol_f;
    // (buffers chosen by selects: indexing d at run time would place it in local memory)
    const bool in1 = (d.cur ^ p.flip) != 0;
    r.mac_in = in1 ? d.mac[1] : d.mac[0];
    r.neq_in = in1 ? d.neq[1] : d.neq[0];
    r.mac_out = in1 ? d.mac[0] : d.mac[1];
    r.neq_out = in1 ? d.neq[0] : d.neq[1];
    r.status = d.status;
#pragma unroll
    for (int w = 0; w < 4; ++w) {
#pragma unroll
        for (int k = 0; k < 4; ++k) r.wall[w][k] = d.wall[w][k];
        r.prof[w] = d.prof[w];
    }
    r.upred = d.upred;
}

// Prescribed sides (the paper gives no discretisation for walls, nor for the prescribed
// inlet of the jet, Sec. III.C): every position beyond such a side holds the equilibrium at
// the side's state (rho_w, u_w, T_w), so the side lies half-way between the last node and the
// first position beyond it.  Walls (boundary type 2) prescribe both sides of the axis, inflow
// (type 3) the low side, with outflow at the high side.  Which prescribed side (0 x-low,
// 1 x-high, 2 y-low, 3 y-high) position (gx, gy) lies beyond, or -1; the y sides own the
// corners.
__device__ __forceinline__ int wall_of(int bc_x, int bc_y, int nx, int ny, int gx, int gy)
{
    if ((bc_y == 2 || bc_y == 3) && gy < 0) return 2;
    if (bc_y == 2 && gy > ny - 1) return 3;
    if ((bc_x == 2 || bc_x == 3) && gx < 0) return 0;
    if (bc_x == 2 && gx > nx - 1) return 1;
    return -1;
}

// The state (u_x, u_y, T, rho) prescribed at position (gx, gy) beyond side w: the side's
// profile entry at the position along the side (clamped to the grid), or its uniform state.
__device__ __forceinline__ const double* side_state(const double (*wall)[4], const double* const* prof,
                                                    int nx, int ny, int w, int gx, int gy)
{
    const double* pr = prof[w];
    if (!pr) return wall[w];
    const int n = w < 2 ? ny : nx;
    int along = w < 2 ? gy : gx;
    along = along < 0 ? 0 : (along > n - 1 ? n - 1 : along);
    return pr + 4 * (long long)along;
}

// Tile reference state: the centre node's frame (FP64) and derived values in R.
template <class R>
struct RefState {
    double rho, ux, uy, T;
    FloatPair rho2, ux2, uy2, T2;   // the same as float pairs (deviations of the mixed modes)
    R rhoR, uxR, uyR, TR;
    R ER;       // B_00^eq of the reference node: E_r (total), U_r (internal), U'_r (non-translational)
    R PR;       // p_r = rho_r T_r
    R eR;       // energy per mass whose balance gives T: E_r / rho_r (total, non-translational), c_v T_r (internal)
    R isT;      // 1 / sqrt(T_r)
    R invT;     // 1 / T_r
    R cvR;
};

// Base frame of a moved equilibrium (see add_g_eq_dev): its pressure and 1/sqrt(T), 1/T.
template <class R>
struct BaseFrame {
    R P, isT, invT;
};

template <class R>
__device__ __forceinline__ R sqrt_r(R v)
{
    if constexpr (std::is_same<R, double>::value) return sqrt(v); else return sqrtf(v);
}

// x and y factors of a moved equilibrium for order p: X0 = t_p0, X1 = t_p1/s, X2 = t_p2/s^2.
template <class R, int N>
__device__ __forceinline__ R tx0(const Tau<R, N>& t, int p) { return p == 0 ? R(1) : t.t[p][0]; }
template <class R, int N>
__device__ __forceinline__ R tx1(const Tau<R, N>& t, int p) { return p >= 1 ? t.u1[p] : R(0); }
template <class R, int N>
__device__ __forceinline__ R tx2(const Tau<R, N>& t, int p) { return p >= 2 ? t.u2[p] : R(0); }

// g equilibrium of a node (Sec. II g_eq in its own frame), moved into a base frame by tx, ty,
// minus the equilibrium of the base frame itself, for the slots (p,q) != (0,0) plus dE at
// (0,0).  Added into G.  Node values: B_00^eq (ES: E, U or U'), p (PS), u (uxS, uyS), T (TS);
// differences node - base: dP, dux, duy, dT; moving shifts dx, dy = (u - u_base)/sqrt(T_base)
// and sig = T/T_base - 1.  Every term is a product of small differences with O(1) values.
// Orders 0-2 carry the base equilibrium and are written out; orders >= 3 have none and follow
//   B_pq = ES X0_p Y0_q + s b10 X1_p Y0_q + s b01 X0_p Y1_q + s^2 p (X2_p Y0_q + X0_p Y2_q).
template <class R, int N>
__device__ __forceinline__ void add_g_eq_dev(int split, const BaseFrame<R>& bf, const Tau<R, N>& tx,
                                             const Tau<R, N>& ty, R dx, R dy, R sig, R ES, R dE, R PS,
                                             R uxS, R uyS, R dP, R dux, R duy, R TS, R dT, R* G)
{
    if (split == 2) {
        // non-translational: only B_00 = U' in the node's frame, moved like f's equilibrium
        G[slot(0, 0)] += dE;
#pragma unroll
        for (int pp = 0; pp <= N; ++pp)
#pragma unroll
            for (int q = 0; q <= N - pp; ++q)
                if (pp + q > 0) G[slot(pp, q)] += ES * tx0(tx, pp) * tx0(ty, q);
        return;
    }
    const R dPT = dP * TS + bf.P * dT;                    // p T - p_b T_b
    const R PsR = PS * (R(1) + sig);                      // s^2 p
    R PuxR = R(0), PuyR = R(0);                           // s b10, s b01 (total split)
    if (split == 0) {
        PuxR = PS * uxS * bf.isT;
        PuyR = PS * uyS * bf.isT;
        const R dPux = dP * uxS + bf.P * dux;             // p u - p_b u_b
        const R dPuy = dP * uyS + bf.P * duy;
        G[slot(0, 0)] += dE;
        G[slot(1, 0)] += dx * ES + dPux * bf.isT;
        G[slot(0, 1)] += dy * ES + dPuy * bf.isT;
        G[slot(2, 0)] += tx.t[2][0] * ES + R(2) * dx * PuxR + dPT * bf.invT;
        G[slot(0, 2)] += ty.t[2][0] * ES + R(2) * dy * PuyR + dPT * bf.invT;
        G[slot(1, 1)] += dx * dy * ES + dx * PuyR + dy * PuxR;
        G[slot(3, 0)] += tx.t[3][0] * ES + R(3) * tx.t[2][0] * PuxR + R(3) * dx * PsR;
        G[slot(0, 3)] += ty.t[3][0] * ES + R(3) * ty.t[2][0] * PuyR + R(3) * dy * PsR;
        G[slot(2, 1)] += tx.t[2][0] * dy * ES + tx.t[2][0] * PuyR + R(2) * dx * dy * PuxR + dy * PsR;
        G[slot(1, 2)] += ty.t[2][0] * dx * ES + ty.t[2][0] * PuxR + R(2) * dx * dy * PuyR + dx * PsR;
    } else {
        G[slot(0, 0)] += dE;
        G[slot(1, 0)] += dx * ES;
        G[slot(0, 1)] += dy * ES;
        G[slot(2, 0)] += tx.t[2][0] * ES + dPT * bf.invT;
        G[slot(0, 2)] += ty.t[2][0] * ES + dPT * bf.invT;
        G[slot(1, 1)] += dx * dy * ES;
        G[slot(3, 0)] += tx.t[3][0] * ES + R(3) * dx * PsR;
        G[slot(0, 3)] += ty.t[3][0] * ES + R(3) * dy * PsR;
        G[slot(2, 1)] += tx.t[2][0] * dy * ES + dy * PsR;
        G[slot(1, 2)] += ty.t[2][0] * dx * ES + dx * PsR;
    }
#pragma unroll
    for (int pp = 0; pp <= N; ++pp)
#pragma unroll
        for (int q = 0; q <= N - pp; ++q)
            if (pp + q >= 4)
                G[slot(pp, q)] += ES * tx0(tx, pp) * tx0(ty, q) + PuxR * tx1(tx, pp) * tx0(ty, q) +
                                  PuyR * tx0(tx, pp) * tx1(ty, q) +
                                  PsR * (tx2(tx, pp) * tx0(ty, q) + tx0(tx, pp) * tx2(ty, q));
}

// Deviation of a source's coefficients, moved into the reference frame, from the reference
// node's equilibrium coefficients (f into Df, g into Dg; ncoef(N) values each).  The source is
// the node whose non-equilibrium coefficient m is neq[m * stride + nd] (its planes in global
// memory, or values already loaded: stride 1) or, with neq = nullptr, the equilibrium at the
// primitive state (rho, ux, uy, T).
template <class S, class R, int N>
__device__ __forceinline__ void source_dev_state(const CaseRun& p, const RefState<R>& rf, double rho,
                                                 double ux, double uy, double T, const S* neq,
                                                 long long nd, long long stride, R* Df, R* Dg)
{
    constexpr int NC = ncoef(N);
    const long long Nn = stride;
    // differences of the primitive variables from the reference: FP64 in the FP64 mode, from
    // float pairs (integer splitting, no FP64 operation) in the mixed modes
    R drho, dux, duy, dT;
    if constexpr (std::is_same<R, double>::value) {
        drho = rho - rf.rho;
        dux = ux - rf.ux;
        duy = uy - rf.uy;
        dT = T - rf.T;
    } else {
        drho = pair_diff(split_double(rho), rf.rho2);
        dux = pair_diff(split_double(ux), rf.ux2);
        duy = pair_diff(split_double(uy), rf.uy2);
        dT = pair_diff(split_double(T), rf.T2);
    }
    const R rhoS = rf.rhoR + drho, uxS = rf.uxR + dux, uyS = rf.uyR + duy, TS = rf.TR + dT;
    const R dx = dux * rf.isT, dy = duy * rf.isT;
    const R sig = dT * rf.invT;                       // T/T_r - 1
    const R s = sqrt_r<R>(R(1) + sig);                // sqrt(T/T_r)
    const Tau<R, N> tx = make_tau_sig<R, N>(s, dx, sig);
    const Tau<R, N> ty = make_tau_sig<R, N>(s, dy, sig);
    // non-equilibrium parts, moved
    if (neq) {
        R A[NC], B[NC];
        A[0] = R(0);
#pragma unroll
        for (int k = 1; k < NC; ++k) A[k] = sto_get<S, R>(neq + (long long)(k - 1) * Nn + nd);
#pragma unroll
        for (int k = 0; k < NC; ++k) B[k] = sto_get<S, R>(neq + (long long)(NC - 1 + k) * Nn + nd);
        retarget2<R, N>(tx, ty, A, Df, B, Dg);
    } else {
#pragma unroll
        for (int k = 0; k < NC; ++k) { Df[k] = R(0); Dg[k] = R(0); }
    }
    // f equilibrium rho tx_p0 ty_q0 minus K_f = rho_r at (0,0)
    Df[0] += drho;
#pragma unroll
    for (int pp = 0; pp <= N; ++pp)
#pragma unroll
        for (int q = 0; q <= N - pp; ++q)
            if (pp + q > 0) Df[slot(pp, q)] += rhoS * tx0(tx, pp) * tx0(ty, q);
    // g equilibrium moved, minus K_g
    const R dP = drho * TS + rf.rhoR * dT;           // p - p_r
    const R PS = rf.PR + dP;
    R ES, dE;
    if (p.split == 0) {
        const R eS = rf.cvR * TS + R(0.5) * (uxS * uxS + uyS * uyS);
        ES = rhoS * eS;
        // E - E_r = (rho - rho_r) e + rho_r (c_v (T - T_r) + (u - u_r).(u + u_r)/2)
        dE = drho * eS + rf.rhoR * (rf.cvR * dT + R(0.5) * (dux * (R(2) * rf.uxR + dux) +
                                                              duy * (R(2) * rf.uyR + duy)));
    } else if (p.split == 1) {
        ES = rf.cvR * PS;
        dE = rf.cvR * dP;
    } else {
        ES = (rf.cvR - R(1)) * PS;                    // U' = rho (c_v - 1) T
        dE = (rf.cvR - R(1)) * dP;
    }
    const BaseFrame<R> bf = {rf.PR, rf.isT, rf.invT};
    add_g_eq_dev<R, N>(p.split, bf, tx, ty, dx, dy, sig, ES, dE, PS, uxS, uyS, dP, dux, duy, TS, dT, Dg);
}

template <class S, class R, int N>
__device__ __forceinline__ void source_dev(const CaseRun& p, const RefState<R>& rf, long long nd,
                                           R* Df, R* Dg)
{
    const long long Nn = p.N;
    source_dev_state<S, R, N>(p, rf, p.mac_in[nd], p.mac_in[Nn + nd], p.mac_in[2 * Nn + nd],
                              p.mac_in[3 * Nn + nd], reinterpret_cast<const S*>(p.neq_in), nd, Nn, Df, Dg);
}

// A staged source's inputs, read from global memory before any of its arithmetic so that the
// loads of several sources are in flight together.
template <class S, int N>
struct SourceLoad {
    double rho, ux, uy, T;
    S neq[nneq(N)];
    bool ghost;                 // beyond a prescribed side: the equilibrium at (rho, u, T)
};

template <class S, int N>
__device__ __forceinline__ void load_source(const CaseRun& p, int gx, int gy, SourceLoad<S, N>& L)
{
    const int w = wall_of(p.bc_x, p.bc_y, p.nx, p.ny, gx, gy);
    L.ghost = w >= 0;
    if (L.ghost) {
        const double* st = side_state(p.wall, p.prof, p.nx, p.ny, w, gx, gy);
        L.rho = st[3];
        L.ux = st[0];
        L.uy = st[1];
        L.T = st[2];
        return;
    }
    const long long Nn = p.N;
    const long long nd = (long long)bc_map(gy, p.ny, p.bc_y) * p.nx + bc_map(gx, p.nx, p.bc_x);
    L.rho = p.mac_in[nd];
    L.ux = p.mac_in[Nn + nd];
    L.uy = p.mac_in[2 * Nn + nd];
    L.T = p.mac_in[3 * Nn + nd];
    const S* q = reinterpret_cast<const S*>(p.neq_in);
#pragma unroll
    for (int m = 0; m < nneq(N); ++m) L.neq[m] = q[(long long)m * Nn + nd];
}

template <class S, class R, int N>
__device__ __forceinline__ void source_from_load(const CaseRun& p, const RefState<R>& rf, const SourceLoad<S, N>& L,
                                                 R* Df, R* Dg)
{
    source_dev_state<S, R, N>(p, rf, L.rho, L.ux, L.uy, L.T, L.ghost ? static_cast<const S*>(nullptr) : L.neq, 0,
                              1, Df, Dg);
}

// The source at position (gx, gy): the node the boundary maps it to, or a prescribed side's
// ghost.
template <class S, class R, int N>
__device__ __forceinline__ void source_at(const CaseRun& p, const RefState<R>& rf, int gx, int gy,
                                          R* Df, R* Dg)
{
    const int w = wall_of(p.bc_x, p.bc_y, p.nx, p.ny, gx, gy);
    if (w >= 0) {
        const double* st = side_state(p.wall, p.prof, p.nx, p.ny, w, gx, gy);
        source_dev_state<S, R, N>(p, rf, st[3], st[0], st[1], st[2], static_cast<const S*>(nullptr), 0, 1,
                                  Df, Dg);
    } else {
        const int sx = bc_map(gx, p.nx, p.bc_x), sy = bc_map(gy, p.ny, p.bc_y);
        source_dev<S, R, N>(p, rf, (long long)sy * p.nx + sx, Df, Dg);
    }
}

// Per-population lattice values, kept in shared memory so that the population loops can run
// without unrolling (the unrolled body would not fit the instruction cache).
template <class R>
struct LatRow {
    R c, w, he[5], hn[5];
};

// Folded x factors of population column a.  A population (a, b) of the target frame is
//   w_a w_b sum_q hn_b(q) sum_l ty_ql sum_{p <= N-q} hn_a(p) sum_{k <= p} tx_pk R_kl
// (the move lambda_r -> lambda_bar and the Grad reconstruction, R = interpolated coefficients
// in lambda_r).  Everything but hn_b(q) and the y interpolation is independent of b, so each
// x-interpolated row X (ncoef(N) values) is contracted at once into N + 1 values
//   Z_q = sum_{l <= q, k <= N-q} phi_q(k, l) X_kl,  phi_q(k, l) = ty_ql w_a sum_{p=k}^{N-q} hn_a(p) tx_pk,
// and only the Z_q are interpolated along y.  phi holds the factors in the order z_contract
// reads them: q = 0..N, then l = 0..q, then k = 0..N-q (20 for N = 3, 35 for N = 4).
__host__ __device__ constexpr int nphi(int N)
{
    int n = 0;
    for (int q = 0; q <= N; ++q) n += (q + 1) * (N - q + 1);
    return n;
}

template <class R, int N>
__device__ __forceinline__ void make_phi(const LatRow<R>& la, const Tau<R, N>& tx, const Tau<R, N>& ty, R* phi)
{
    int n = 0;
#pragma unroll
    for (int q = 0; q <= N; ++q) {
        R S[N + 1];
#pragma unroll
        for (int k = 0; k <= N - q; ++k) {
            R v = R(0);
#pragma unroll
            for (int p = k; p <= N - q; ++p) v += la.hn[p] * tau_at(tx, p, k);
            S[k] = la.w * v;
        }
#pragma unroll
        for (int l = 0; l <= q; ++l)
#pragma unroll
            for (int k = 0; k <= N - q; ++k) phi[n++] = tau_at(ty, q, l) * S[k];
    }
}

template <class R, int N>
__device__ __forceinline__ void z_contract(const R* phi, const R* X, R* Z)
{
    int n = 0;
#pragma unroll
    for (int q = 0; q <= N; ++q) {
        R z = R(0);
#pragma unroll
        for (int l = 0; l <= q; ++l)
#pragma unroll
            for (int k = 0; k <= N - q; ++k) z += phi[n++] * X[slot(k, l)];
        Z[q] = z;
    }
}

// z_contract for (f, g) pairs: Z[q] = (Z_q of the f half of X, Z_q of the g half), through
// packed two-lane FMAs (each lane the same fused operations, in the same order, as z_contract).
template <int N>
__device__ __forceinline__ void z_contract_pairs(const float* phi, const float2* X, float2* Z)
{
    int n = 0;
#pragma unroll
    for (int q = 0; q <= N; ++q) {
        float2 z = make_float2(0.f, 0.f);
#pragma unroll
        for (int l = 0; l <= q; ++l)
#pragma unroll
            for (int k = 0; k <= N - q; ++k) {
                z = __ffma2_rn(make_float2(phi[n], phi[n]), X[slot(k, l)], z);
                ++n;
            }
        Z[q] = z;
    }
}

// Node-interleaved shared-memory records.  N = 3: 20 values per node, f in 0..9 and g in
// 10..19.  N = 4, FP32: f in 0..14 and g in 16..30 (each distribution 16-byte aligned) in
// records of 36 floats; FP64: f in 0..14 and g in 15..29, records of 30 doubles (the box must
// fit shared memory).  Both strides (36 and 60 words) put the eight lanes of a 16-byte load
// phase on distinct banks.
template <class R, int N>
__host__ __device__ constexpr int rec_len() { return N == 3 ? 20 : (sizeof(R) == 4 ? 36 : 30); }
template <class R, int N>
__host__ __device__ constexpr int rec_goff() { return N == 3 ? 10 : (sizeof(R) == 4 ? 16 : 15); }

// FP32 arithmetic with N = 3 keeps (f_m, g_m) pairs: record = f_0 g_0 f_1 g_1 ... f_9 g_9, so
// that both distributions stream through packed two-lane FMAs (see stream_pairs).
template <class R, int N>
__host__ __device__ constexpr bool pair_records() { return sizeof(R) == 4 && N == 3; }

template <class R, int N>
__device__ __forceinline__ void store_rec(R* dst, const R* Df, const R* Dg)
{
    constexpr int NC = ncoef(N);
    if constexpr (N == 3) {
        R v[20];
#pragma unroll
        for (int m = 0; m < NC; ++m) { v[m] = Df[m]; v[NC + m] = Dg[m]; }
        if constexpr (std::is_same<R, float>::value) {
#pragma unroll
            for (int k = 0; k < 5; ++k)
                reinterpret_cast<float4*>(dst)[k] = make_float4(Df[2 * k], Dg[2 * k], Df[2 * k + 1], Dg[2 * k + 1]);
        } else {
#pragma unroll
            for (int k = 0; k < 10; ++k) reinterpret_cast<double2*>(dst)[k] = make_double2(v[2 * k], v[2 * k + 1]);
        }
    } else {
#pragma unroll
        for (int m = 0; m < NC; ++m) { dst[m] = Df[m]; dst[rec_goff<R, N>() + m] = Dg[m]; }
    }
}

// The ncoef(N) values of distribution D (0 = f, 1 = g) of one record.
template <class R, int N, int D>
__device__ __forceinline__ void load_one(const R* rec, R* v)
{
    if constexpr (N == 4) {
        const R* q = rec + D * rec_goff<R, 4>();
        if constexpr (std::is_same<R, float>::value) {
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const float4 t = reinterpret_cast<const float4*>(q)[k];
                v[4 * k] = t.x; v[4 * k + 1] = t.y; v[4 * k + 2] = t.z;
                if (k < 3) v[4 * k + 3] = t.w;
            }
        } else if constexpr (D == 0) {              // 0..13 in pairs, then 14
#pragma unroll
            for (int k = 0; k < 7; ++k) {
                const double2 t = reinterpret_cast<const double2*>(q)[k];
                v[2 * k] = t.x;
                v[2 * k + 1] = t.y;
            }
            v[14] = q[14];
        } else {                                    // 15, then 16..29 in pairs
            v[0] = q[0];
#pragma unroll
            for (int k = 0; k < 7; ++k) {
                const double2 t = reinterpret_cast<const double2*>(q + 1)[k];
                v[1 + 2 * k] = t.x;
                v[2 + 2 * k] = t.y;
            }
        }
    } else if constexpr (std::is_same<R, float>::value) {
        if constexpr (D == 0) {
            const float4 a = reinterpret_cast<const float4*>(rec)[0];
            const float4 b = reinterpret_cast<const float4*>(rec)[1];
            const float2 c = reinterpret_cast<const float2*>(rec)[4];
            v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
            v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
            v[8] = c.x; v[9] = c.y;
        } else {
            const float2 a = reinterpret_cast<const float2*>(rec)[5];
            const float4 b = reinterpret_cast<const float4*>(rec)[3];
            const float4 c = reinterpret_cast<const float4*>(rec)[4];
            v[0] = a.x; v[1] = a.y;
            v[2] = b.x; v[3] = b.y; v[4] = b.z; v[5] = b.w;
            v[6] = c.x; v[7] = c.y; v[8] = c.z; v[9] = c.w;
        }
    } else {
#pragma unroll
        for (int k = 0; k < 5; ++k) {
            const double2 t = reinterpret_cast<const double2*>(rec + D * 10)[k];
            v[2 * k] = t.x;
            v[2 * k + 1] = t.y;
        }
    }
}

// The values of ND distributions of one record starting at distribution d0 (ND = 2, N = 3:
// all 20 values with five or ten 16-byte loads).
template <class R, int N, int ND>
__device__ __forceinline__ void load_dist(const R* rec, int d0, R* v)
{
    if constexpr (ND == 2) {
        static_assert(N == 3, "both distributions in one pass only for N = 3");
        if constexpr (std::is_same<R, float>::value) {
#pragma unroll
            for (int k = 0; k < 5; ++k) {
                const float4 t = reinterpret_cast<const float4*>(rec)[k];
                v[4 * k] = t.x; v[4 * k + 1] = t.y; v[4 * k + 2] = t.z; v[4 * k + 3] = t.w;
            }
        } else {
#pragma unroll
            for (int k = 0; k < 10; ++k) {
                const double2 t = reinterpret_cast<const double2*>(rec)[k];
                v[2 * k] = t.x; v[2 * k + 1] = t.y;
            }
        }
    } else {
        if (d0 == 0) load_one<R, N, 0>(rec, v); else load_one<R, N, 1>(rec, v);
    }
}

// w[j] for a runtime j < n <= 4 without indexing the register array dynamically.
template <class R>
__device__ __forceinline__ R pick(const R* w, int j, int n)
{
    R v = w[0];
#pragma unroll
    for (int k = 1; k < 4; ++k)
        if (k < n) v = (j == k) ? w[k] : v;
    return v;
}

// Rows of the per-thread table of y-stencil weights of the FP32 D2Q16 2-D kernels: the weights
// of the four y stencils at each row of the warp's row range, so that the row loop reads the
// four weights of a row with one 16-byte load instead of selecting them (a warp whose range
// is longer streams through global gathers).
constexpr int kWtRows = 16;
__host__ __device__ constexpr bool weight_table(int rbytes, int q1, bool one_d)
{
    return rbytes == 4 && q1 == 4 && !one_d;
}

// Bytes of dynamic shared memory of the step kernel: the staged box, one record per node,
// then the weight table (kWtRows float4 per thread) where the kernel keeps one.
__host__ __device__ constexpr size_t step_smem_bytes(int rbytes, int q1, bool one_d, int box_w,
                                                     int box_h, int nodes)
{
    return (size_t)box_w * box_h * rbytes * (q1 == 5 ? (rbytes == 4 ? 36 : 30) : 20) +
           (weight_table(rbytes, q1, one_d) ? (size_t)kWtRows * nodes * 16 : 0);
}

template <class R>
__device__ __forceinline__ LatRow<R> lat_row(const Lattice& L, int a)
{
    LatRow<R> r;
    r.c = lat_c<R>(L, a);
    r.w = lat_w<R>(L, a);
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        r.he[k] = lat_he<R>(L, a, k);
        r.hn[k] = lat_hn<R>(L, a, k);
    }
    return r;
}

// The tile's reference state: the frame of its centre node (clamped into the grid).
template <class R>
__device__ __forceinline__ RefState<R> tile_reference(const CaseRun& p, int TX, int TY)
{
    RefState<R> rf;
    const long long N = p.N;
    const int cxn = min(p.tile_x * TX + TX / 2, p.nx - 1);
    const int cyn = min(p.tile_y * TY + TY / 2, p.ny - 1);
    const long long c = (long long)cyn * p.nx + cxn;
    rf.rho = p.mac_in[c];
    rf.ux = p.mac_in[N + c];
    rf.uy = p.mac_in[2 * N + c];
    rf.T = p.mac_in[3 * N + c];
    rf.rho2 = split_double(rf.rho);
    rf.ux2 = split_double(rf.ux);
    rf.uy2 = split_double(rf.uy);
    rf.T2 = split_double(rf.T);
    rf.rhoR = R(rf.rho);
    rf.uxR = R(rf.ux);
    rf.uyR = R(rf.uy);
    rf.TR = R(rf.T);
    rf.cvR = case_r<R>(p.cv, p.cv_f);
    // B_00 of g's equilibrium, and the energy per mass whose balance gives T.  One thread
    // computes these while the block waits, so the reduced precisions take them in R: at the
    // FP64 rate of this part a double division or square root costs the block about a
    // microsecond, and the values are rounded to R anyway.
    const R P = rf.rhoR * rf.TR;
    const R e_tot = rf.cvR * rf.TR + R(0.5) * (rf.uxR * rf.uxR + rf.uyR * rf.uyR);
    rf.ER = p.split == 0 ? rf.rhoR * e_tot : (p.split == 1 ? rf.cvR * P : (rf.cvR - R(1)) * P);
    rf.PR = P;
    rf.eR = p.split == 1 ? rf.cvR * rf.TR : e_tot;
    rf.isT = R(1) / sqrt_r<R>(rf.TR);
    rf.invT = R(1) / rf.TR;
    return rf;
}

// Interpolation footprint of the tile (all threads of the block call it; nodes may appear in
// several threads): the box of source nodes that covers the stencils of every node's departure
// points under its previous frame, plus a margin for the frame to move during the iterations.
// Writes box = {x0, y0, width, height} (each thread its own copy), the size clipped to the
// staged capacity.
template <bool ONE_D, int NW>
__device__ __forceinline__ void footprint_box(const CaseRun& p, const StepParams& pp, int TX, int TY,
                                              bool active, double ux0, double uy0, double T0,
                                              float (*red)[NW], int* box, int tid)
{
    // the frame to FP32 by truncation (integer operations, no FP64 conversion): the footprint
    // is an estimate with a margin
    const float cm = pp.lat.cmaxf;
    const float ux0f = double_hi(ux0), uy0f = double_hi(uy0);
    float sT0 = sqrtf(fmaxf(double_hi(T0), 0.f));
    float lx = active ? -ux0f - cm * sT0 : 1e30f;
    float hx = active ? -ux0f + cm * sT0 : -1e30f;
    float ly = active ? -uy0f - cm * sT0 : 1e30f;
    float hy = active ? -uy0f + cm * sT0 : -1e30f;
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
    // every thread combines the warps' extremes itself (broadcast reads; no second barrier)
    lx = red[0][0]; hx = red[1][0]; ly = red[2][0]; hy = red[3][0];
    for (int w = 1; w < NW; ++w) {
        lx = fminf(lx, red[0][w]); hx = fmaxf(hx, red[1][w]);
        ly = fminf(ly, red[2][w]); hy = fmaxf(hy, red[3][w]);
    }
    const float margin = 0.5f;   // room for the frame to move during the iterations
    // taps of a departure offset `off` lie in [floor(off) - 1, floor(off) + 2]
    const int x_lo = (int)floorf(fmaxf(lx - margin, -1e6f)) - 1;
    const int x_hi = (TX - 1) + (int)floorf(fminf(hx + margin, 1e6f)) + 2;
    const int y_lo = (int)floorf(fmaxf(ly - margin, -1e6f)) - 1;
    const int y_hi = (TY - 1) + (int)floorf(fminf(hy + margin, 1e6f)) + 2;
    box[0] = p.tile_x * TX + x_lo;
    box[1] = ONE_D ? 0 : p.tile_y * TY + y_lo;
    box[2] = min(x_hi - x_lo + 1, pp.box_w);
    box[3] = ONE_D ? 1 : min(y_hi - y_lo + 1, pp.box_h);
}

// Frame of the final moments lambda* and the maps of the collision (Sec. III.A, collision in the
// frame of the streamed populations' moments).  Inputs are the deviations of the last
// iteration: u - u_bar, T - T_bar, u - u_r, T - T_r, rho - rho_r.
template <class R, int N>
struct FinalFrame {
    Tau<R, N> dx, dy;       // lambda_bar -> lambda* (deviation part)
    Tau<R, N> rx, ry;       // lambda_r -> lambda* (reference part)
    R rdx, rdy, rsig;       // (u_r - u*)/sqrt(T*), T_r/T* - 1
    R isTn, iTn, TnR, rhoN, keep;
};

template <class R, int N>
__device__ __forceinline__ FinalFrame<R, N> final_frame(const RefState<R>& rf, R mu, R drho, R dubx,
                                                        R duby, R durx, R dury, R dTr, R dTb)
{
    FinalFrame<R, N> ff;
    ff.TnR = rf.TR + dTr;
    ff.isTn = R(1) / sqrt_r<R>(ff.TnR);
    ff.iTn = ff.isTn * ff.isTn;
    {
        const R sig = -dTb * ff.iTn;                          // T_bar/T* - 1
        const R s = sqrt_r<R>(R(1) + sig);
        ff.dx = make_tau_sig<R, N>(s, -dubx * ff.isTn, sig);
        ff.dy = make_tau_sig<R, N>(s, -duby * ff.isTn, sig);
    }
    ff.rsig = -dTr * ff.iTn;                                  // T_r/T* - 1
    const R s = sqrt_r<R>(R(1) + ff.rsig);
    ff.rdx = -durx * ff.isTn;                                 // (u_r - u*)/sqrt(T*)
    ff.rdy = -dury * ff.isTn;
    ff.rx = make_tau_sig<R, N>(s, ff.rdx, ff.rsig);
    ff.ry = make_tau_sig<R, N>(s, ff.rdy, ff.rsig);
    ff.rhoN = rf.rhoR + drho;
    const R tau = mu / (ff.rhoN * ff.TnR);                    // tau = mu / (rho T)
    ff.keep = R(1) - R(1) / (tau + R(0.5));                   // 1 - omega
    return ff;
}

// BGK relaxation of f in lambda*: the streamed deviation coefficients Af (in lambda_bar) are
// moved into lambda*, the reference part rho_r moved lambda_r -> lambda* is added (its order
// 0 and 1 terms are the equilibrium's), and the non-equilibrium part is relaxed and written.
// A*_10 = A*_01 = 0 hold by definition of lambda*.
// The arithmetic of collide_f without the writes: Af becomes the relaxed non-equilibrium
// coefficients of lambda* (slots 1, 2 zero; slot 0 unused).
// (Af has been moved into lambda* by the caller: retarget2 with Ag, or retarget.)
template <class R, int N>
__device__ __forceinline__ void relax_f(const FinalFrame<R, N>& ff, const RefState<R>& rf, R* Af)
{
    constexpr int NC = ncoef(N);
#pragma unroll
    for (int pp = 0; pp <= N; ++pp)
#pragma unroll
        for (int q = 0; q <= N - pp; ++q)
            if (pp + q >= 2) Af[slot(pp, q)] += rf.rhoR * tx0(ff.rx, pp) * tx0(ff.ry, q);
    Af[slot(1, 0)] = R(0);
    Af[slot(0, 1)] = R(0);
#pragma unroll
    for (int m = 3; m < NC; ++m) Af[m] = ff.keep * Af[m];
}

template <class S, class R, int N>
__device__ __forceinline__ void collide_f(const FinalFrame<R, N>& ff, const RefState<R>& rf, R* Af, S* nout,
                                          long long Nn, long long node)
{
    constexpr int NC = ncoef(N);
    relax_f<R, N>(ff, rf, Af);
#pragma unroll
    for (int m = 1; m < NC; ++m) sto_put<S, R>(nout + (long long)(m - 1) * Nn + node, Af[m]);
}

// BGK relaxation of g in lambda*: the reference equilibrium moved into lambda* minus the
// equilibrium of lambda* itself (the same expansion as for a staged node, with the reference as
// the node and lambda* as the base) is added.  Total split: B*_00 = B_00^eq by definition of
// T*.  Internal split: U* = B*_00 + (1/2) sum G, so B*_00 - U* = (1/2) rho* T* div u, relaxed
// like the other coefficients.  Non-translational split: T* also takes f's second moment, so
// B*_00 - U'* balances f's non-equilibrium A*_20 + A*_02 and is relaxed likewise.
// The arithmetic of collide_g without the writes (Ag already moved into lambda*): Ag becomes the
// relaxed non-equilibrium coefficients of lambda* (slot 0 zero for the total split).
template <class R, int N>
__device__ __forceinline__ void relax_g(int split, const FinalFrame<R, N>& ff, const RefState<R>& rf, R drho,
                                        R durx, R dury, R dTr, R* Ag)
{
    constexpr int NC = ncoef(N);
    const R dP = -(drho * ff.TnR + rf.rhoR * dTr);            // p_r - p*
    const BaseFrame<R> bf = {rf.PR - dP, ff.isTn, ff.iTn};    // p* = rho T*
    // U'_r - U'* (non-translational), U_r - U* (internal); unused by the total split
    const R dE = split == 2 ? (rf.cvR - R(1)) * dP : (split == 1 ? rf.cvR * dP : R(0));
    add_g_eq_dev<R, N>(split, bf, ff.rx, ff.ry, ff.rdx, ff.rdy, ff.rsig, rf.ER, dE, rf.PR, rf.uxR, rf.uyR,
                       dP, -durx, -dury, rf.TR, -dTr, Ag);
    Ag[0] = split != 0 ? ff.keep * Ag[0] : R(0);
#pragma unroll
    for (int m = 1; m < NC; ++m) Ag[m] = ff.keep * Ag[m];
}

template <class S, class R, int N>
__device__ __forceinline__ void collide_g(int split, const FinalFrame<R, N>& ff, const RefState<R>& rf,
                                          R drho, R durx, R dury, R dTr, R* Ag, S* nout, long long Nn,
                                          long long node)
{
    constexpr int NC = ncoef(N);
    relax_g<R, N>(split, ff, rf, drho, durx, dury, dTr, Ag);
#pragma unroll
    for (int m = 0; m < NC; ++m) sto_put<S, R>(nout + (long long)(NC - 1 + m) * Nn + node, Ag[m]);
}

// Per-warp sums of the step statistics, one atomic per warp (every lane of the warp calls it).
__device__ __forceinline__ void report_stats(DevStatus* st, int tid, unsigned int kk, unsigned int nc,
                                             unsigned int fb, bool bad, long long node)
{
    unsigned int sum_k = __reduce_add_sync(0xffffffffu, kk);
    unsigned int max_k = __reduce_max_sync(0xffffffffu, kk);
    unsigned int sum_nc = __reduce_add_sync(0xffffffffu, nc);
    unsigned int sum_fb = __reduce_add_sync(0xffffffffu, fb);
    if ((tid & 31) == 0) {
        atomicAdd(&st->iters_total, (unsigned long long)sum_k);
        atomicMax(&st->iters_max, max_k);
        if (sum_nc) {
            atomicAdd(&st->nonconv, (unsigned long long)sum_nc);
            atomicOr(&st->flags, 2);
        }
        if (sum_fb) atomicAdd(&st->fallbacks, (unsigned long long)sum_fb);
    }
    if (bad) {
        atomicOr(&st->flags, 1);
        atomicMin(&st->first_bad, (unsigned long long)node);
    }
}

// Warms L2 with the state that the block one wave later (pp.ahead launch positions on) will
// stage: the rows of the box capacity around its tile, clamped to its grid, in every frame and
// non-equilibrium plane.  A prefetch is a hint; every address lies inside the case's arrays.
template <class S, int NG, bool ONE_D>
__device__ __forceinline__ void prefetch_next_wave(const StepParams& pp, int TX, int TY, int tid, int nthreads)
{
    const long long b = (long long)blockIdx.y * gridDim.x + blockIdx.x + pp.ahead;
    const CaseDesc* c;
    long long tile;
    if (pp.ncase > 0) {
        if (b >= pp.tile_start[pp.ncase]) return;
        const int lo = find_case(pp.tile_start, pp.ncase, (int)b, tid & 31);
        c = pp.cases + lo;
        tile = b - pp.tile_start[lo];
    } else {
        if (b >= (long long)gridDim.x * gridDim.y) return;
        c = &pp.one;
        tile = b;
    }
    const int tiles_x = pp.ncase > 0 ? c->tiles_x : (int)gridDim.x;
    const int tx = (int)(tile % tiles_x), ty = (int)(tile / tiles_x);
    const int nx = c->nx, ny = c->ny;
    const long long N = c->N;
    const int in = c->cur ^ pp.flip;
    const char* mac = reinterpret_cast<const char*>(c->mac[in]);
    const char* neq = reinterpret_cast<const char*>(c->neq[in]);
    const int x0 = max(0, tx * TX - (pp.box_w - TX) / 2), x1 = min(nx - 1, tx * TX + TX - 1 + (pp.box_w - TX) / 2);
    const int y0 = ONE_D ? 0 : max(0, ty * TY - (pp.box_h - TY) / 2);
    const int y1 = ONE_D ? 0 : min(ny - 1, ty * TY + TY - 1 + (pp.box_h - TY) / 2);
    if (x0 > x1 || y0 > y1) return;
    const int rows = y1 - y0 + 1;
    const int planes = NMAC + nneq(NG);
    for (int k = tid; k < rows * planes; k += nthreads) {
        const int plane = k / rows;
        const long long first = (long long)(y0 + k % rows) * nx + x0;
        const bool is_mac = plane < NMAC;
        const size_t esz = is_mac ? sizeof(double) : sizeof(S);
        const char* row = is_mac ? mac + ((long long)plane * N + first) * sizeof(double)
                                 : neq + ((long long)(plane - NMAC) * N + first) * sizeof(S);
        const size_t bytes = (size_t)(x1 - x0 + 1) * esz;
        for (size_t off = 0; off < bytes; off += 128)
            asm volatile("prefetch.global.L2 [%0];" ::"l"(row + off));
    }
}

// Half the velocity divergence at node (x, y) of the internal split's predictor velocities
// (central differences; beyond a prescribed side its velocity): in FP64 for the FP64 kernels,
// from float pairs in the mixed modes.
template <class R>
__device__ __forceinline__ R half_predictor_divergence(const CaseRun& p, int x, int y)
{
    const int nb[4][2] = {{x + 1, y}, {x - 1, y}, {x, y + 1}, {x, y - 1}};
    double v[4];
    for (int k = 0; k < 4; ++k) {
        const int comp = k < 2 ? 0 : 1;                  // u_x along x, u_y along y
        const int w = wall_of(p.bc_x, p.bc_y, p.nx, p.ny, nb[k][0], nb[k][1]);
        if (w >= 0) {
            v[k] = side_state(p.wall, p.prof, p.nx, p.ny, w, nb[k][0], nb[k][1])[comp];
        } else {
            const long long m = (long long)bc_map(nb[k][1], p.ny, p.bc_y) * p.nx + bc_map(nb[k][0], p.nx, p.bc_x);
            v[k] = p.upred[comp * p.N + m];
        }
    }
    if constexpr (std::is_same<R, double>::value) {
        return 0.5 * (0.5 * (v[0] - v[1]) + 0.5 * (v[2] - v[3]));
    } else {
        // the differences from float pairs, without FP64 instructions (on this part one holds
        // the FP64 pipe for 64 cycles a warp): each to the FP32 rounding of the difference
        const float dx = pair_diff(split_double(v[0]), split_double(v[1]));
        const float dy = pair_diff(split_double(v[2]), split_double(v[3]));
        return R(0.25f * (dx + dy));
    }
}

// One thread per node, one CTA per tile of TPB nodes; CTAs resident per SM as
// step_blocks_per_sm says (the quasi-1-D D2Q16 kernel with FP32 arithmetic is held to three per
// SM).  PRED: the internal split's predictor pass instead of a step: each node streams f and g
// once in its previous frame and writes the velocity of f's result and the streamed
// coefficients to upred, where the step takes its first iteration from (other splits' blocks
// return at once; nothing else is written).
template <class S, class R, int Q1, int P, bool ONE_D, int TPB, bool PRED>
__global__ void __launch_bounds__(TPB, step_blocks_per_sm(ONE_D, Q1 == 5, std::is_same<R, double>::value))
    step_kernel(const StepParams pp)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    R* sm = reinterpret_cast<R*>(smem_raw);
    __shared__ float red[4][TPB / 32];
    __shared__ LatRow<R> lat[Q1];
    __shared__ RefState<R> srf;
    __shared__ CaseRun scase;
    const int TX = blockDim.x, TY = blockDim.y;
    const int tid = threadIdx.y * TX + threadIdx.x;
    __shared__ CaseDesc sdesc;
    if (tid < 32) resolve_case(pp, scase, sdesc, tid);
    __syncthreads();
    const CaseRun& p = scase;
    if constexpr (PRED) {
        if (p.split != 1) return;                             // the whole block: p is shared
    }
    // Node of this thread.  FP32 2-D grids: each warp covers a 16 x 2 block of the tile (a
    // TX x 32/TX block on tiles narrower than 16, 32 x 1 on one-row tiles), its consecutive
    // lanes running down a column (lane = x * rows + y), and its lanes stream the same
    // absolute rows together: the nodes of a column then read the same staged record in the
    // same load, and a 16-byte shared load merges equal addresses within each half warp.
    // Otherwise a warp covers 32 nodes of a row.  Tile sides are powers of two, TX * TY = 256.
    int lx = threadIdx.x, ly = threadIdx.y;
    if constexpr (!ONE_D && pair_records<R, grad_order_of_q1(Q1)>()) {
        const int wx = TX >= 16 ? (TY >= 2 ? 16 : 32) : TX, wy = 32 / wx, wpr = TX / wx;
        const int w = tid >> 5, l = tid & 31;
        lx = (w % wpr) * wx + l / wy;
        ly = (w / wpr) * wy + l % wy;
    }
    const int x = p.tile_x * TX + lx;
    const int y = p.tile_y * TY + ly;
    const bool active = (x < p.nx) && (y < p.ny);
    const long long N = p.N;
    const long long node = active ? (long long)y * p.nx + x : 0;
    constexpr int NG = grad_order_of_q1(Q1);                 // Grad order of the lattice
    constexpr int NC = ncoef(NG);
    constexpr int REC = rec_len<R, NG>();

    if (tid < Q1) lat[tid] = lat_row<R>(pp.lat, tid);
    // ---- own frame (predictor) and the tile's reference state ------------------------------
    double ux0 = 0.0, uy0 = 0.0, T0 = 1.0;
    if (active) {
        ux0 = p.mac_in[N + node];
        uy0 = p.mac_in[2 * N + node];
        T0 = p.mac_in[3 * N + node];
    }
    // quasi-1-D grids: the inputs of the box capacity centred on the tile are read before the
    // footprint is known, so that their latency overlaps the frames' and the reduction's; the
    // footprint box nearly always lies inside it (the capacity is then the staged box)
    constexpr int SC = ONE_D ? 2 : 1;
    SourceLoad<S, NG> Lc[SC];
    const int cx0 = p.tile_x * TX - (pp.box_w - TX) / 2;
    if constexpr (ONE_D) {
#pragma unroll
        for (int u = 0; u < SC; ++u) {
            const int i = tid + u * TPB;
            if (i < pp.box_w) load_source<S, NG>(p, cx0 + i, 0, Lc[u]);
        }
    }
    if (tid == 0) srf = tile_reference<R>(p, TX, TY);
    // the barrier inside footprint_box publishes srf and lat (the reference's loads overlap the
    // other warps' footprint reductions)
    int box[4];
    footprint_box<ONE_D, TPB / 32>(p, pp, TX, TY, active, ux0, uy0, T0, red, box, tid);
    bool centred = false;           // the footprint lies in the capacity read above (block-uniform)
    if constexpr (ONE_D) {
        centred = box[0] >= cx0 && box[0] + box[2] <= cx0 + pp.box_w && 2 * TPB >= pp.box_w;
        if (centred) {
            box[0] = cx0;
            box[2] = pp.box_w;
        }
    }
    const RefState<R>& rf = srf;
    const R sTr = R(1) / rf.isT;
    const int ox = box[0], oy = box[1], bw = box[2], bh = box[3];   // this thread's copy
    const int bn = bw * bh;

    // ---- staging: source deviations in the reference frame --------------------------------
    // Node-interleaved records (rec_len floats per box node).  Each thread reads the inputs of
    // SB box nodes before working on any of them, so that their global loads are in flight
    // together (the phase is bound by their latency).
    // (run once per tile, before the predictor-corrector's streaming iterations)
    auto stage_tile = [&]() {
        // (quasi-1-D boxes hold about one node per thread: nothing to batch)
        constexpr int SB = ONE_D ? 1 : ((sizeof(S) <= 4 && NG == 3) ? 4 : 2);
        if constexpr (ONE_D) {
            if (centred) {
#pragma unroll
                for (int u = 0; u < SC; ++u) {
                    const int i = tid + u * TPB;
                    if (i < bn) {
                        R D[2 * NC];
                        source_from_load<S, R, NG>(p, rf, Lc[u], D, D + NC);
                        store_rec<R, NG>(sm + (size_t)i * REC, D, D + NC);
                    }
                }
            }
        }
        for (int i0 = tid; i0 < (centred ? 0 : bn); i0 += SB * TPB) {
            SourceLoad<S, NG> L[SB];
#pragma unroll
            for (int u = 0; u < SB; ++u) {
                const int i = i0 + u * TPB;
                if (i < bn) load_source<S, NG>(p, ox + i % bw, ONE_D ? 0 : oy + i / bw, L[u]);
            }
#pragma unroll
            for (int u = 0; u < SB; ++u) {
                const int i = i0 + u * TPB;
                if (i < bn) {
                    R D[2 * NC];
                    source_from_load<S, R, NG>(p, rf, L[u], D, D + NC);
                    store_rec<R, NG>(sm + (size_t)i * REC, D, D + NC);
                }
            }
        }
        };

    // ---- predictor-corrector ---------------------------------------------------------------
    int k = 0;
    bool bad = false, nonconv = false;
    unsigned int fallbacks = 0;
    double unx = ux0, uny = uy0, Tn = T0;
    R drho = R(0), dubx = R(0), duby = R(0), durx = R(0), dury = R(0), dTr = R(0), dTb = R(0);
    R Af[NC], Ag[NC];         // deviation coefficients of the streamed populations in lambda_bar
    // internal split: half the velocity divergence at the new time level (from the predictor
    // velocities), for U = sum g + (1/2) sum G = sum g - (1/2) rho T div u
    R hD = R(0);
    if constexpr (!PRED) {
        if (active && p.split == 1) hD = half_predictor_divergence<R>(p, x, y);
    }
    // T - T_r = (c_v (T - T_r) from the energy balance - hD T_r) / (c_v + hD): the internal
    // split's rho (c_v + hD) T = U_s; hD = 0 for the others
    const R hDT = hD * rf.TR;
    const R icvD = p.split == 1 ? R(1) / (rf.cvR + hD) : case_r<R>(p.inv_cv, p.inv_cv_f);

    // frame of the iteration relative to the reference: the differences once (FP64, or from
    // float pairs in the mixed modes), then each corrector takes the new moments' deviations
    // (u - u_r, T - T_r) already in R; the frame's change over the iterations is summed in R
    // and added to the FP64 frame at the end, so the loop itself has no FP64 operation
    R rbx = R(0), rby = R(0), rbT = R(0);                      // u_r - u_bar, T_r - T_bar
    if (active) {
        if constexpr (std::is_same<R, double>::value) {
            rbx = rf.ux - ux0;
            rby = rf.uy - uy0;
            rbT = rf.T - T0;
        } else {
            rbx = pair_diff(rf.ux2, split_double(ux0));
            rby = pair_diff(rf.uy2, split_double(uy0));
            rbT = pair_diff(rf.T2, split_double(T0));
        }
    }
    R sum_dux = R(0), sum_duy = R(0);                          // u - u_bar, summed
    // first taps of the stencils, carried from one iteration to the next while the departure
    // point stays within a quarter cell of the range they were chosen for (a stencil chosen
    // again at every iteration makes the iteration map jump where a departure point crosses
    // its boundary, and the 3-point stencil's half-integer boundary then traps the iteration in
    // a cycle)
    int jy[Q1], jxk[Q1];
    // One predictor-corrector iteration of this node: streaming (or, from_predictor, the
    // predictor pass's streamed coefficients), moments, the stopping test and the corrector.
    // Returns true when the node stops (converged, iteration cap, non-physical, predictor).
    auto pc_iteration = [&](const bool from_predictor) -> bool {
            const R sT = sqrt_r<R>(rf.TR - rbT);                   // sqrt(T_bar)
            const R isT = R(1) / sT;
            const R iTb = isT * isT;
            const R sig_t = rbT * iTb;                             // T_r / T_bar - 1
            const R s_rb = sTr * isT, dx_rb = rbx * isT, dy_rb = rby * isT;   // lambda_r -> lambda_bar
            const Tau<R, NG> txr = make_tau_sig<R, NG>(s_rb, dx_rb, sig_t);
            const Tau<R, NG> tyr = make_tau_sig<R, NG>(s_rb, dy_rb, sig_t);
            const R ubxr = rf.uxR - rbx, ubyr = rf.uyR - rby;      // u_bar
#pragma unroll
            for (int m = 0; m < NC; ++m) { Af[m] = R(0); Ag[m] = R(0); }

            // internal split: the first iteration streams in the previous frame through the
            // same staged box and stencils as the predictor pass did, so its coefficients are
            // the predictor's (kept in the predictor buffer); only the stencil choice is redone
            if (from_predictor) {
                const R* first = reinterpret_cast<const R*>(p.upred + 2 * N);
#pragma unroll
                for (int m = 0; m < NC; ++m) {
                    Af[m] = first[(long long)m * N + node];
                    Ag[m] = first[(long long)(NC + m) * N + node];
                }
#pragma unroll
                for (int c = 0; c < Q1; ++c) {
                    R w[P];
                    if constexpr (!ONE_D) jy[c] = lagrange<R, P>(-(sT * lat[c].c + ubyr), w);
                    jxk[c] = lagrange<R, P>(-(sT * lat[c].c + ubxr), w);
                }
            } else if constexpr (!ONE_D) {
                // y stencils of all b (shared by every a and both distributions)
                R wy[Q1][P];
                int rmin = 1 << 30, rmax = -(1 << 30);
#pragma unroll
                for (int b = 0; b < Q1; ++b) {
                    const R off = -(sT * lat[b].c + ubyr);
                    if (k > 0 && stencil_holds<R, P>(off, jy[b])) lagrange_at<R, P>(off, jy[b], wy[b]);
                    else jy[b] = lagrange<R, P>(off, wy[b]);
                    rmin = min(rmin, jy[b]);
                    rmax = max(rmax, jy[b] + P - 1);
                }
                const bool rows_in = (y + rmin - oy >= 0) && (y + rmax - oy < bh);
                // FP32, N = 3: the warp's lanes whose y stencils lie in the box stream the union
                // of their rows [r_lo, r_hi] in one order; each lane's weights of the four y
                // stencils at every row of that range (0 outside its stencils) go into its
                // column of the weight table, once per iteration for all a
                int r_lo = 0, r_hi = -1;
                bool tab_ok = false;
                if constexpr (pair_records<R, NG>()) {
                    const unsigned rmask = __ballot_sync(__activemask(), rows_in);
                    if (rows_in) {
                        r_lo = __reduce_min_sync(rmask, y + rmin);
                        r_hi = __reduce_max_sync(rmask, y + rmax);
                        tab_ok = r_hi - r_lo < kWtRows;
                        if (tab_ok) {
                            float4* const wt = reinterpret_cast<float4*>(sm + (size_t)pp.box_w * pp.box_h * REC) + tid;
                            for (int i = 0; i <= r_hi - r_lo; ++i) wt[i * TPB] = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
                            for (int b = 0; b < Q1; ++b)
#pragma unroll
                                for (int j = 0; j < P; ++j)
                                    reinterpret_cast<float*>(wt + (y + jy[b] + j - r_lo) * TPB)[b] = wy[b][j];
                        }
                    }
                }
#pragma unroll 1
                for (int a = 0; a < Q1; ++a) {
                    const LatRow<R>& la = lat[a];
                    R wx[P];
                    const R offx = -(sT * la.c + ubxr);
                    int jx = k > 0 ? sel_get<Q1>(jxk, a) : 0;
                    if (k > 0 && stencil_holds<R, P>(offx, jx)) {
                        lagrange_at<R, P>(offx, jx, wx);
                    } else {
                        jx = lagrange<R, P>(offx, wx);
                        sel_set<Q1>(jxk, a, jx);
                    }
                    const int tx0 = x + jx - ox;
                    const bool cols_in = tx0 >= 0 && tx0 + P <= bw;
                    R phi[nphi(NG)];
                    {
                        // the iteration's moves, rebuilt here so that only four scalars stay live
                        const Tau<R, NG> tx = make_tau_sig<R, NG>(s_rb, dx_rb, sig_t);
                        const Tau<R, NG> ty = make_tau_sig<R, NG>(s_rb, dy_rb, sig_t);
                        make_phi<R, NG>(la, tx, ty, phi);
                    }
                  if constexpr (pair_records<R, NG>()) {
                    // FP32, N = 3: f and g stream together as (f_m, g_m) pairs through packed
                    // two-lane FMAs (the x pass, the fold and the row weights).  The
                    // warp's in-box lanes take the union of their rows in one order, rows
                    // outside a lane's y stencils adding with weight 0.
                    float2 acc[Q1][NG + 1];
#pragma unroll
                    for (int b = 0; b < Q1; ++b)
#pragma unroll
                        for (int q = 0; q <= NG; ++q) acc[b][q] = make_float2(0.f, 0.f);
                    const bool inbox = rows_in && cols_in && tab_ok;
                    if (inbox) {
                        float2 w2x[P];
#pragma unroll
                        for (int ii = 0; ii < P; ++ii) w2x[ii] = make_float2(wx[ii], wx[ii]);
                        const float* rowp = sm + ((size_t)(r_lo - oy) * bw + tx0) * REC;
                        const float4* wtp = reinterpret_cast<const float4*>(sm + (size_t)pp.box_w * pp.box_h * REC) + tid;
                        // two rows per trip on 4-point stencils (with the weight table; three or
                        // four were 1 % slower, one row 1-3 %)
                        constexpr int kRowUnroll = P == 4 ? 2 : 1;
#pragma unroll kRowUnroll
                        for (int r = r_lo; r <= r_hi; ++r, rowp += (size_t)bw * REC, wtp += TPB) {
                            float2 X[NC];
#pragma unroll
                            for (int ii = 0; ii < P; ++ii) {
                                const float4* q4 = reinterpret_cast<const float4*>(rowp + ii * REC);
#pragma unroll
                                for (int k = 0; k < NC / 2; ++k) {
                                    const float4 t = q4[k];
                                    const float2 lo = make_float2(t.x, t.y), hi = make_float2(t.z, t.w);
                                    if (ii == 0) {
                                        X[2 * k] = __fmul2_rn(w2x[0], lo);
                                        X[2 * k + 1] = __fmul2_rn(w2x[0], hi);
                                    } else {
                                        X[2 * k] = __ffma2_rn(w2x[ii], lo, X[2 * k]);
                                        X[2 * k + 1] = __ffma2_rn(w2x[ii], hi, X[2 * k + 1]);
                                    }
                                }
                            }
                            float2 Z[NG + 1];
                            z_contract_pairs<NG>(phi, X, Z);
                            const float4 w4 = *wtp;
                            const float wb[4] = {w4.x, w4.y, w4.z, w4.w};
#pragma unroll
                            for (int b = 0; b < Q1; ++b) {
                                const float2 w2 = make_float2(wb[b], wb[b]);
#pragma unroll
                                for (int q = 0; q <= NG; ++q) acc[b][q] = __ffma2_rn(w2, Z[q], acc[b][q]);
                            }
                        }
                    } else {
                        ++fallbacks;
                        // global gathers; indices into the register arrays stay static, and the
                        // y weights are formed again (the same stencils and offsets as above)
#pragma unroll
                        for (int b = 0; b < Q1; ++b) {
                            float wyb[P];
                            lagrange_at<float, P>(-(sT * lat[b].c + ubyr), jy[b], wyb);
#pragma unroll 1
                            for (int j = 0; j < P; ++j) {
                                const float wyj = pick<float>(wyb, j, P);
#pragma unroll 1
                                for (int ii = 0; ii < P; ++ii) {
                                    const float W = wyj * pick<float>(wx, ii, P);
                                    float D[2 * NC];
                                    source_at<S, float, NG>(p, rf, x + jx + ii, y + jy[b] + j, D, D + NC);
                                    float2 X[NC], Z[NG + 1];
#pragma unroll
                                    for (int m = 0; m < NC; ++m) X[m] = make_float2(D[m], D[NC + m]);
                                    z_contract_pairs<NG>(phi, X, Z);
                                    const float2 W2 = make_float2(W, W);
#pragma unroll
                                    for (int q = 0; q <= NG; ++q) acc[b][q] = __ffma2_rn(W2, Z[q], acc[b][q]);
                                }
                            }
                        }
                    }
                    // populations (a, b): f'_ab = w_b sum_q hn_b(q) acc_b(q); their moments
                    // (f, g) pairs through packed FMAs, each lane the same operations in the
                    // same order as the scalar form
                    float2 S2[NG + 1];
#pragma unroll
                    for (int q = 0; q <= NG; ++q) S2[q] = make_float2(0.f, 0.f);
#pragma unroll
                    for (int b = 0; b < Q1; ++b) {
                        const LatRow<R>& lb = lat[b];
                        float2 v = make_float2(0.f, 0.f);
#pragma unroll
                        for (int q = 0; q <= NG; ++q) v = __ffma2_rn(make_float2(lb.hn[q], lb.hn[q]), acc[b][q], v);
                        v = __fmul2_rn(v, make_float2(lb.w, lb.w));
#pragma unroll
                        for (int q = 0; q <= NG; ++q) S2[q] = __ffma2_rn(v, make_float2(lb.he[q], lb.he[q]), S2[q]);
                    }
#pragma unroll
                    for (int pq = 0; pq <= NG; ++pq)
#pragma unroll
                        for (int q = 0; q <= NG - pq; ++q) {
                            Af[slot(pq, q)] += la.he[pq] * S2[q].x;
                            Ag[slot(pq, q)] += la.he[pq] * S2[q].y;
                        }
                  } else {
                    // one pass per distribution (FP64; D2Q25)
                    constexpr int ND = 1;
                    constexpr int NDIST = 2;
                    // one pass each (ND = 1) share their code: unrolled, the two passes kept
                    // both sets of row temporaries live and spilled on D2Q25 (702 -> 534 us)
#pragma unroll 1
                    for (int d0 = 0; d0 < NDIST; d0 += ND) {
                        // x pass once per row of the union of the y stencils, folded into Z_q,
                        // then added to the b's whose y stencil contains the row
                        R acc[ND][Q1][NG + 1];
#pragma unroll
                        for (int e = 0; e < ND; ++e)
#pragma unroll
                            for (int b = 0; b < Q1; ++b)
#pragma unroll
                                for (int q = 0; q <= NG; ++q) acc[e][b][q] = R(0);
                        if (rows_in && cols_in) {
                            const R* rowp = sm + ((size_t)(y + rmin - oy) * bw + tx0) * REC;
                            // FP32, 4-point stencils: two rows per trip, so that one row's loads
                            // overlap the other's FMAs (260 -> 257.5 us; three or four rows were
                            // slower); FP64 had more spills with it, and 3-point stencils ran
                            // 2 % slower
                            constexpr int kRowUnroll = (std::is_same<R, float>::value && P == 4) ? 2 : 1;
#pragma unroll kRowUnroll
                            for (int r = rmin; r <= rmax; ++r, rowp += (size_t)bw * REC) {
                                R X[ND][NC];
#pragma unroll
                                for (int ii = 0; ii < P; ++ii) {
                                    R v[ND * NC];
                                    load_dist<R, NG, ND>(rowp + ii * REC, d0, v);
#pragma unroll
                                    for (int e = 0; e < ND; ++e)
#pragma unroll
                                        for (int m = 0; m < NC; ++m)
                                            X[e][m] = (ii == 0) ? wx[0] * v[e * NC + m]
                                                                : X[e][m] + wx[ii] * v[e * NC + m];
                                }
                                R Z[ND][NG + 1];
#pragma unroll
                                for (int e = 0; e < ND; ++e) z_contract<R, NG>(phi, X[e], Z[e]);
#pragma unroll
                                for (int b = 0; b < Q1; ++b) {
                                    const int j = r - jy[b];
                                    if constexpr (std::is_same<R, float>::value) {
                                        // FP32: no branch, a row outside b's stencil adds with weight
                                        // 0 (more FMAs, but resolving the branch cost more: 268 ->
                                        // 262 us); FP64 is bound by its pipe and keeps the branch
                                        const R w = ((unsigned)j < (unsigned)P) ? pick<R>(wy[b], j, P) : R(0);
#pragma unroll
                                        for (int e = 0; e < ND; ++e)
#pragma unroll
                                            for (int q = 0; q <= NG; ++q) acc[e][b][q] += w * Z[e][q];
                                    } else if ((unsigned)j < (unsigned)P) {
                                        const R w = pick<R>(wy[b], j, P);
#pragma unroll
                                        for (int e = 0; e < ND; ++e)
#pragma unroll
                                            for (int q = 0; q <= NG; ++q) acc[e][b][q] += w * Z[e][q];
                                    }
                                }
                            }
                        } else {
                            ++fallbacks;
                            // global gathers; indices into the register arrays stay static
#pragma unroll
                            for (int b = 0; b < Q1; ++b)
#pragma unroll 1
                                for (int j = 0; j < P; ++j) {
                                    const R wyj = pick<R>(wy[b], j, P);
#pragma unroll 1
                                    for (int ii = 0; ii < P; ++ii) {
                                        const R wxi = pick<R>(wx, ii, P);
                                        R D[2 * NC];
                                        source_at<S, R, NG>(p, rf, x + jx + ii, y + jy[b] + j, D, D + NC);
#pragma unroll
                                        for (int e = 0; e < ND; ++e) {
                                            R Z[NG + 1];
                                            z_contract<R, NG>(phi, D + (d0 + e) * NC, Z);
#pragma unroll
                                            for (int q = 0; q <= NG; ++q) acc[e][b][q] += wyj * wxi * Z[q];
                                        }
                                    }
                                }
                        }
                        // populations (a, b): f'_ab = w_b sum_q hn_b(q) acc_b(q); their moments
#pragma unroll
                        for (int e = 0; e < ND; ++e) {
                            R Sq[NG + 1];
#pragma unroll
                            for (int q = 0; q <= NG; ++q) Sq[q] = R(0);
#pragma unroll
                            for (int b = 0; b < Q1; ++b) {
                                const LatRow<R>& lb = lat[b];
                                R val = R(0);
#pragma unroll
                                for (int q = 0; q <= NG; ++q) val += lb.hn[q] * acc[e][b][q];
                                val *= lb.w;
#pragma unroll
                                for (int q = 0; q <= NG; ++q) Sq[q] += val * lb.he[q];
                            }
#pragma unroll
                            for (int pq = 0; pq <= NG; ++pq)
#pragma unroll
                                for (int q = 0; q <= NG - pq; ++q) {
                                    if (d0 + e == 0) Af[slot(pq, q)] += la.he[pq] * Sq[q];
                                    else Ag[slot(pq, q)] += la.he[pq] * Sq[q];
                                }
                        }
                    }
                  }
                }
            } else {
                // quasi-1-D (ny = 1): every y tap reads row 0 and the y weights sum to one, so
                // the interpolated coefficients depend on a only.
#pragma unroll 1
                for (int a = 0; a < Q1; ++a) {
                    const LatRow<R>& la = lat[a];
                    R wx[P];
                    const R offx = -(sT * la.c + ubxr);
                    int jx = k > 0 ? sel_get<Q1>(jxk, a) : 0;
                    if (k > 0 && stencil_holds<R, P>(offx, jx)) {
                        lagrange_at<R, P>(offx, jx, wx);
                    } else {
                        jx = lagrange<R, P>(offx, wx);
                        sel_set<Q1>(jxk, a, jx);
                    }
                    const int tx0 = x + jx - ox;
                    R Ri[2 * NC];
#pragma unroll
                    for (int m = 0; m < 2 * NC; ++m) Ri[m] = R(0);
                    if (tx0 >= 0 && tx0 + P <= bw) {
                        if constexpr (pair_records<R, NG>()) {
                            // (f_m, g_m) pairs through packed two-lane FMAs
                            float2 R2[NC];
#pragma unroll
                            for (int m = 0; m < NC; ++m) R2[m] = make_float2(0.f, 0.f);
#pragma unroll
                            for (int ii = 0; ii < P; ++ii) {
                                const float4* q4 = reinterpret_cast<const float4*>(sm + (size_t)(tx0 + ii) * REC);
                                const float2 w2 = make_float2(wx[ii], wx[ii]);
#pragma unroll
                                for (int k = 0; k < NC / 2; ++k) {
                                    const float4 t = q4[k];
                                    R2[2 * k] = __ffma2_rn(w2, make_float2(t.x, t.y), R2[2 * k]);
                                    R2[2 * k + 1] = __ffma2_rn(w2, make_float2(t.z, t.w), R2[2 * k + 1]);
                                }
                            }
#pragma unroll
                            for (int m = 0; m < NC; ++m) {
                                Ri[m] = R2[m].x;
                                Ri[NC + m] = R2[m].y;
                            }
                        } else {
#pragma unroll
                            for (int ii = 0; ii < P; ++ii) {
                                R v[NC];
                                load_one<R, NG, 0>(sm + (size_t)(tx0 + ii) * REC, v);
#pragma unroll
                                for (int m = 0; m < NC; ++m) Ri[m] += wx[ii] * v[m];
                                load_one<R, NG, 1>(sm + (size_t)(tx0 + ii) * REC, v);
#pragma unroll
                                for (int m = 0; m < NC; ++m) Ri[NC + m] += wx[ii] * v[m];
                            }
                        }
                    } else {
                        ++fallbacks;
#pragma unroll 1
                        for (int ii = 0; ii < P; ++ii) {
                            const R W = pick<R>(wx, ii, P);
                            R D[2 * NC];
                            source_at<S, R, NG>(p, rf, x + jx + ii, 0, D, D + NC);
#pragma unroll
                            for (int m = 0; m < 2 * NC; ++m) Ri[m] += W * D[m];
                        }
                    }
                    // the y taps all read row 0 with weights summing to one, so every b sees
                    // the same folded values Z (see make_phi)
                    R phi[nphi(NG)], Zf[NG + 1], Zg[NG + 1];
                    make_phi<R, NG>(la, txr, tyr, phi);
                  if constexpr (pair_records<R, NG>()) {
                    // FP32, N = 3: the fold and the populations' moments as (f, g) pairs through
                    // packed FMAs (each lane the scalar form's operations in its order)
                    float2 X2[NC], Z2[NG + 1], S2[NG + 1];
#pragma unroll
                    for (int m = 0; m < NC; ++m) X2[m] = make_float2(Ri[m], Ri[NC + m]);
                    z_contract_pairs<NG>(phi, X2, Z2);
#pragma unroll
                    for (int q = 0; q <= NG; ++q) S2[q] = make_float2(0.f, 0.f);
#pragma unroll
                    for (int b = 0; b < Q1; ++b) {
                        const LatRow<R>& lb = lat[b];
                        float2 v = make_float2(0.f, 0.f);
#pragma unroll
                        for (int q = 0; q <= NG; ++q) v = __ffma2_rn(make_float2(lb.hn[q], lb.hn[q]), Z2[q], v);
                        v = __fmul2_rn(v, make_float2(lb.w, lb.w));
#pragma unroll
                        for (int q = 0; q <= NG; ++q) S2[q] = __ffma2_rn(v, make_float2(lb.he[q], lb.he[q]), S2[q]);
                    }
#pragma unroll
                    for (int pp = 0; pp <= NG; ++pp)
#pragma unroll
                        for (int q = 0; q <= NG - pp; ++q) {
                            Af[slot(pp, q)] += la.he[pp] * S2[q].x;
                            Ag[slot(pp, q)] += la.he[pp] * S2[q].y;
                        }
                  } else {
                    z_contract<R, NG>(phi, Ri, Zf);
                    z_contract<R, NG>(phi, Ri + NC, Zg);
                    R Sf[NG + 1], Sg[NG + 1];
#pragma unroll
                    for (int q = 0; q <= NG; ++q) { Sf[q] = R(0); Sg[q] = R(0); }
#pragma unroll
                    for (int b = 0; b < Q1; ++b) {
                        const LatRow<R>& lb = lat[b];
                        R f = R(0), g = R(0);
#pragma unroll
                        for (int q = 0; q <= NG; ++q) {
                            f += lb.hn[q] * Zf[q];
                            g += lb.hn[q] * Zg[q];
                        }
                        f *= lb.w;
                        g *= lb.w;
#pragma unroll
                        for (int q = 0; q <= NG; ++q) {
                            Sf[q] += f * lb.he[q];
                            Sg[q] += g * lb.he[q];
                        }
                    }
#pragma unroll
                    for (int pp = 0; pp <= NG; ++pp)
#pragma unroll
                        for (int q = 0; q <= NG - pp; ++q) {
                            Af[slot(pp, q)] += la.he[pp] * Sf[q];
                            Ag[slot(pp, q)] += la.he[pp] * Sg[q];
                        }
                  }
                }
            }

            // ---- moments of the streamed populations (Sec. II), as deviations --------------
            drho = Af[slot(0, 0)];                                    // rho - rho_r
            const R rhoR = rf.rhoR + drho;
            const R irho = R(1) / rhoR;
            // rho (u - u_bar) = rho_r (u_r - u_bar) + sqrt(T_bar) sum_i c_i f'_i
            dubx = (rf.rhoR * rbx + sT * Af[slot(1, 0)]) * irho;      // u - u_bar
            duby = (rf.rhoR * rby + sT * Af[slot(0, 1)]) * irho;
            if constexpr (PRED) {
                ++k;
                return true;                                          // the predictor: u only
            }
            durx = dubx - rbx;                                        // u - u_r
            dury = duby - rby;
            // energy deviation: sum g' (total, internal), plus sum |C|^2/2 f' for the
            // non-translational split, |C|^2 = T_bar (He_2(c_x) + He_2(c_y) + 2) + 2 sqrt(T_bar) c.u_bar + u_bar^2
            R dEt = Ag[slot(0, 0)];
            if (p.split == 2)
                dEt += R(0.5) * (sT * sT * (Af[slot(2, 0)] + Af[slot(0, 2)] + R(2) * drho) +
                                 R(2) * sT * (ubxr * Af[slot(1, 0)] + ubyr * Af[slot(0, 1)]) +
                                 (ubxr * ubxr + ubyr * ubyr) * drho);
            // c_v (T - T_r) = (dE - e_r drho)/rho [- (u - u_r).(u + u_r)/2 unless internal split]
            R cvdT = (dEt - rf.eR * drho) * irho;
            if (p.split != 1)
                cvdT -= R(0.5) * (durx * (R(2) * rf.uxR + durx) + dury * (R(2) * rf.uyR + dury));
            dTr = (cvdT - hDT) * icvD;                                // T - T_r
            dTb = dTr + rbT;                                          // T - T_bar
            sum_dux += dubx;
            sum_duy += duby;
            ++k;
            if (!(rhoR > R(0)) || !(rf.TR + dTr > R(0)) || isnan(sum_dux) || isnan(sum_duy)) {
                bad = true;
                return true;
            }
            const float du = sqrtf((float)(dubx * dubx + duby * duby));
            const float change = fmaxf(du * (float)isT, fabsf((float)(dTb * iTb)));
            // the tolerance; in the mixed modes no smaller than the FP32 rounding of the
            // deviations the moments are formed from (16 ulps of their magnitudes against
            // sqrt(T_bar) and T_bar): a tile that spans a shock carries deviations far above the
            // local temperature on its cold side, and the change cannot fall below that floor
            float tol = p.pc_tol_f;
            if constexpr (!std::is_same<R, double>::value)
                tol = fmaxf(tol, 0x1p-20f * fmaxf((fabsf(rbx) + fabsf(rby) + fabsf(durx) + fabsf(dury)) * isT,
                                                  (fabsf(rbT) + fabsf(dTr)) * iTb));
            bool stop;
            if (p.pc_fixed > 0) stop = (k >= p.pc_fixed);
            else if (change <= tol) stop = true;
            else if (k >= p.pc_max_iter) { stop = true; nonconv = true; }
            else stop = false;
            if (stop) return true;
            rbx = -durx; rby = -dury; rbT = -dTr;                // corrector: lambda_bar <- lambda
            return false;
    };
    // internal split (the step, not its predictor pass) on 2-D grids in the mixed modes: the
    // first iteration takes the predictor's streamed coefficients and reads no staged record,
    // so it runs before the staging, and the box is staged only if some node of the tile
    // iterates on (the decision is the block's); a tile whose nodes all converge goes straight
    // to its collision.  (The FP64 kernel keeps the plain order: its registers are spent.)
    const bool lazy = !PRED && !ONE_D && !std::is_same<R, double>::value && p.split == 1;
    bool iterating = active;
    if (lazy && active) iterating = !pc_iteration(true);
    if (!lazy || __syncthreads_or(iterating)) {
        stage_tile();
        __syncthreads();
        if (pp.ahead > 0) prefetch_next_wave<S, NG, ONE_D>(pp, TX, TY, tid, TPB);
    }
    if (iterating)
        while (!pc_iteration(!PRED && k == 0 && p.split == 1)) {
        }
    if (active) {
        unx = ux0 + (double)sum_dux;
        uny = uy0 + (double)sum_duy;
        Tn = rf.T + (double)dTr;
        if (!positive_double(Tn)) bad = true;
    }
    if constexpr (PRED) {
        if (active) {
            p.upred[node] = ux0 + (double)dubx;                       // u of f streamed once
            p.upred[N + node] = uy0 + (double)duby;
            R* first = reinterpret_cast<R*>(p.upred + 2 * N);        // the step's first iteration
#pragma unroll
            for (int m = 0; m < NC; ++m) {
                first[(long long)m * N + node] = Af[m];
                first[(long long)(NC + m) * N + node] = Ag[m];
            }
        }
        return;
    }

    // ---- collision in the frame of the final moments and write-back ---------------------------
    if (active) {
        S* nout = reinterpret_cast<S*>(p.neq_out);
        p.mac_out[node] = rf.rho + (double)drho;
        p.mac_out[N + node] = unx;
        p.mac_out[2 * N + node] = uny;
        p.mac_out[3 * N + node] = Tn;
        if (!bad) {
            const FinalFrame<R, NG> ff = final_frame<R, NG>(rf, case_r<R>(p.mu, p.mu_f), drho, dubx, duby,
                                                            durx, dury, dTr, dTb);
            retarget2<R, NG>(ff.dx, ff.dy, Af, Af, Ag, Ag);        // lambda_bar -> lambda*
            collide_f<S, R, NG>(ff, rf, Af, nout, N, node);
            collide_g<S, R, NG>(p.split, ff, rf, drho, durx, dury, dTr, Ag, nout, N, node);
        } else {
            for (int m = 0; m < nneq(NG); ++m) sto_put<S, R>(nout + (long long)m * N + node, R(NAN));
        }
    }
    report_stats(p.status, tid, active ? (unsigned int)k : 0u, (active && nonconv) ? 1u : 0u, fallbacks,
                 active && bad, node);
}

}  // namespace pond
