/*
 * FP64 CPU oracle for the particles-on-demand (PonD) double-distribution BGK step
 * of Hosseini, Bhadauria & Karlin, "Probing double distribution function models in
 * the lattice Boltzmann method for highly compressible flows" (arXiv 2405.11489).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call this code; only the
 * tests, the smoke check and the CPU-baseline leg of the benchmark use it.  It shares
 * no code, header, table or constant with the CUDA library: the lattice, the Hermite
 * tensors and every formula are written out here again, in the paper's order.
 *
 * It is deliberately plain and slow: populations f_i, g_i are stored as they are
 * (Q values per node, each node in its own frame lambda = (u, T)), and streaming
 * applies the frame transformation to every stencil node separately before the
 * Lagrange interpolation, exactly as Eq. (propagationInterpolated) is written.
 * The only economy is a memo of the Grad coefficients of a source node in the current
 * target frame, which is the same computation repeated for every population i.
 *
 * Units: lattice units, r = 1, delta_x = delta_t = 1, T_L = 1 (Sec. III, Table I).
 * Build: gcc -O2 -ffp-contract=off (no fused multiply-add, so results are fixed by
 * the source order), optionally -fopenmp (the node loop is embarrassingly parallel
 * and each node's arithmetic is independent of the thread count).
 *
 * Readings taken where the paper is silent (each is listed with its reason in the
 * design notes of the repository):
 *   - discrete BGK: f* = f + omega (f_eq - f), omega = 1/(tau + 1/2), tau = mu/p;
 *   - Grad expansion order N = the Hermite order the lattice carries: N = 3 (all
 *     coefficients of total order <= 3) on D2Q16, N = 4 on D2Q25 (the non-translational
 *     split needs the fourth-order moments of f, Sec. III.A; and with N = 3 the D2Q25
 *     total split loses stability at Ma ~ 1.5-2); either can be forced by grad_order;
 *   - W(x - x_s) is evaluated at the departure point x - C_i(lambda_bar) dt;
 *   - cubic (4-point) Lagrange interpolation by default, 3-point as an option;
 *   - predictor-corrector: guess = previous frame of the node, metric
 *     max(|du|/sqrt(T_bar), |dT|/T_bar), stop at tolerance or iteration cap, or after
 *     exactly K iterations in fixed mode; from one iteration to the next the stencil nodes
 *     of each population are kept while the departure point stays within a quarter cell of
 *     the range they were chosen for, only their weights following the frame: choosing
 *     them again at every iteration makes the iteration map jump where a departure point
 *     crosses the 3-point stencil's half-integer boundary, and the iteration then cycles
 *     between two frames without a fixed point;
 *   - collision in the frame of the final moments, after projecting into it;
 *   - internal-energy split source (Eq. int_g_evolution), integrated along the
 *     characteristics by the trapezoidal rule, the same second-order rule that gives
 *     omega = 1/(tau + 1/2): with g carried as g - (Omega + G)/2, the internal energy of a
 *     node is U = sum g + (1/2) sum G and the collision adds (1 - omega/2) G.  Inside the
 *     source f -> f_eq, so sum G = -p div u exactly; d_t u is the backward difference
 *     against the frame before the step and grad u the central difference of the new
 *     velocities.  U needs div u at the new time level, which is non-local: it is taken
 *     from predictor velocities, the velocities of one streaming iteration of f in each
 *     node's previous frame, so that T = sum g / (rho (c_v + div u_pred / 2)).  (With
 *     div u of the previous step, the pdV work lags the compression by a step and sound
 *     waves grow instead of decaying at the bulk viscosity of Sec. II.)  The temperature
 *     of a node is its frame's;
 *   - non-translational split: E = sum g + sum |C|^2/2 f, g_eq = (U'/rho) f_eq;
 *   - walls (not in the paper): every position beyond a wall holds the equilibrium at the
 *     wall's state (rho_w, u_w, T_w), so the wall lies half-way between the last node and
 *     the first position beyond it; the internal-split gradients take the wall velocity;
 *   - inflow (the prescribed conditions of the jet, Sec. III.C; the paper gives no
 *     discretisation): the low side of the axis is a prescribed side treated like a wall,
 *     the high side is outflow;
 *   - a prescribed side's state may vary along it (a profile, one state per position along
 *     the side; positions beyond the grid's ends take the nearest entry); without one it is
 *     the side's uniform state.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_MAXQ1 5
#define OR_MAXQ (OR_MAXQ1 * OR_MAXQ1)

typedef struct {
    int32_t nx, ny;
    int32_t q1;            /* 4 -> D2Q16, 5 -> D2Q25 (Table I) */
    int32_t split;         /* 0 total, 1 internal, 2 non-translational energy split (Eq. Es) */
    int32_t interp_order;  /* 3 -> 4-point cubic Lagrange, 2 -> 3-point quadratic */
    int32_t bc_x, bc_y;    /* 0 periodic, 1 outflow (index clamp, zero gradient), 2 wall,
                              3 inflow at the low side and outflow at the high side */
    double gamma, mu;      /* adiabatic exponent (Eq. spec_heat), dynamic viscosity (Eq. kin_visc) */
    double pc_tol;
    int32_t pc_max_iter;
    int32_t pc_fixed_iters; /* > 0: exactly this many predictor-corrector iterations */
    int32_t grad_order;     /* Grad expansion order N: 3 or 4; 0 = the lattice's (3 on D2Q16, 4 on D2Q25) */
    double wall[4][4];      /* prescribed sides x-low, x-high, y-low, y-high: (u_x, u_y, T, rho) */
    const double *profile[4]; /* NULL, or per position along the side: [n][4] (u_x, u_y, T, rho),
                                 n = ny for the x sides, nx for the y sides */
} or_config;

static int grad_order_of(const or_config *cfg)
{
    if (cfg->grad_order == 3 || cfg->grad_order == 4) return cfg->grad_order;
    return cfg->q1 == 5 ? 4 : 3;
}

/* ---------------------------------------------------------------------------------- */
/* Table I: one-dimensional Gauss-Hermite quadratures with r T_L = 1.                  */
/* ---------------------------------------------------------------------------------- */
/* Threads of the node loops (OpenMP builds; 1 otherwise): n > 0 sets them; returns the count
 * in effect.  Timing only: a node's arithmetic does not depend on the thread count. */
int or_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}

int or_lattice_1d(int q1, double *c, double *w)
{
    if (q1 == 4) {
        /* D1Q4: c = {+-sqrt(3 - sqrt 6), +-sqrt(3 + sqrt 6)}, w = {(3 + sqrt 6)/12, (3 - sqrt 6)/12} */
        double cin = sqrt(3.0 - sqrt(6.0)), cout = sqrt(3.0 + sqrt(6.0));
        double win = (3.0 + sqrt(6.0)) / 12.0, wout = (3.0 - sqrt(6.0)) / 12.0;
        c[0] = -cout; c[1] = -cin; c[2] = cin; c[3] = cout;
        w[0] = wout;  w[1] = win;  w[2] = win; w[3] = wout;
        return 4;
    }
    if (q1 == 5) {
        /* D1Q5: c = {0, +-sqrt(5 - sqrt 10), +-sqrt(5 + sqrt 10)},
         *       w = {8/15, (7 + 2 sqrt 10)/60, (7 - 2 sqrt 10)/60} (larger weight on the inner node) */
        double cin = sqrt(5.0 - sqrt(10.0)), cout = sqrt(5.0 + sqrt(10.0));
        double w0 = 8.0 / 15.0, win = (7.0 + 2.0 * sqrt(10.0)) / 60.0, wout = (7.0 - 2.0 * sqrt(10.0)) / 60.0;
        c[0] = -cout; c[1] = -cin; c[2] = 0.0; c[3] = cin; c[4] = cout;
        w[0] = wout;  w[1] = win;  w[2] = w0;  w[3] = win; w[4] = wout;
        return 5;
    }
    return 0;
}

/* Tensor-product 2-D lattice: population i = b*q1 + a has c_i = (c_a, c_b), w_i = w_a w_b. */
typedef struct {
    int q1, Q;
    double cx[OR_MAXQ], cy[OR_MAXQ], w[OR_MAXQ];
} or_lattice;

static void make_lattice(int q1, or_lattice *L)
{
    double c[OR_MAXQ1], w[OR_MAXQ1];
    or_lattice_1d(q1, c, w);
    L->q1 = q1;
    L->Q = q1 * q1;
    for (int b = 0; b < q1; ++b)
        for (int a = 0; a < q1; ++a) {
            int i = b * q1 + a;
            L->cx[i] = c[a];
            L->cy[i] = c[b];
            L->w[i] = w[a] * w[b];
        }
}

/* ---------------------------------------------------------------------------------- */
/* Hermite tensors H^(n)(xi), n <= 3, in D = 2 (probabilists' normalisation, r T_L = 1) */
/* ---------------------------------------------------------------------------------- */
typedef struct {
    double h0, h1[2], h2[2][2], h3[2][2][2], h4[2][2][2][2];
} or_tensors;

static double kron(int a, int b) { return a == b ? 1.0 : 0.0; }

static void hermite_tensors(double xi_x, double xi_y, int order, or_tensors *H)
{
    double xi[2] = {xi_x, xi_y};
    H->h0 = 1.0;
    for (int a = 0; a < 2; ++a) H->h1[a] = xi[a];
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b) H->h2[a][b] = xi[a] * xi[b] - kron(a, b);
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b)
            for (int g = 0; g < 2; ++g)
                H->h3[a][b][g] = xi[a] * xi[b] * xi[g]
                               - xi[a] * kron(b, g) - xi[b] * kron(a, g) - xi[g] * kron(a, b);
    if (order < 4) return;                 /* rank 4 only for the order-4 transformation */
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b)
            for (int g = 0; g < 2; ++g)
                for (int d = 0; d < 2; ++d)
                    H->h4[a][b][g][d] = xi[a] * xi[b] * xi[g] * xi[d]
                        - xi[a] * xi[b] * kron(g, d) - xi[a] * xi[g] * kron(b, d)
                        - xi[a] * xi[d] * kron(b, g) - xi[b] * xi[g] * kron(a, d)
                        - xi[b] * xi[d] * kron(a, g) - xi[g] * xi[d] * kron(a, b)
                        + kron(a, b) * kron(g, d) + kron(a, g) * kron(b, d) + kron(a, d) * kron(b, g);
}

/* ---------------------------------------------------------------------------------- */
/* Frame transformation M_{lambda}^{lambda_bar}, Eq. (gradGeneralTransform), N = 3, 4. */
/* a_n = sum_j f_j H^(n)((C_j(lambda) - u_bar)/sqrt(T_bar)); the populations of the    */
/* target frame are f_i = w_i sum_n a_n : H^(n)(c_i) / n!.                             */
/* ---------------------------------------------------------------------------------- */
typedef struct { double ux, uy, T; } or_frame;

static void grad_coefficients(const or_lattice *L, const double *pops, int stride, int order,
                              or_frame src, or_frame dst, or_tensors *A)
{
    memset(A, 0, sizeof(*A));
    double sTs = sqrt(src.T), sTd = sqrt(dst.T);
    for (int j = 0; j < L->Q; ++j) {
        double Cx = sTs * L->cx[j] + src.ux;       /* C_j(lambda) = sqrt(T) c_j + u */
        double Cy = sTs * L->cy[j] + src.uy;
        double xix = (Cx - dst.ux) / sTd;
        double xiy = (Cy - dst.uy) / sTd;
        or_tensors H;
        hermite_tensors(xix, xiy, order, &H);
        double fj = pops[(size_t)j * stride];
        A->h0 += fj * H.h0;
        for (int a = 0; a < 2; ++a) A->h1[a] += fj * H.h1[a];
        for (int a = 0; a < 2; ++a)
            for (int b = 0; b < 2; ++b) A->h2[a][b] += fj * H.h2[a][b];
        for (int a = 0; a < 2; ++a)
            for (int b = 0; b < 2; ++b)
                for (int g = 0; g < 2; ++g) A->h3[a][b][g] += fj * H.h3[a][b][g];
        if (order >= 4)
            for (int a = 0; a < 2; ++a)
                for (int b = 0; b < 2; ++b)
                    for (int g = 0; g < 2; ++g)
                        for (int d = 0; d < 2; ++d) A->h4[a][b][g][d] += fj * H.h4[a][b][g][d];
    }
}

/* Full Frobenius contraction of every rank up to N (no symmetry shortcut), divided by n!. */
static double grad_population(const or_lattice *L, const or_tensors *A, int i, int order)
{
    or_tensors H;
    hermite_tensors(L->cx[i], L->cy[i], order, &H);
    double s0 = A->h0 * H.h0, s1 = 0.0, s2 = 0.0, s3 = 0.0, s4 = 0.0;
    for (int a = 0; a < 2; ++a) s1 += A->h1[a] * H.h1[a];
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b) s2 += A->h2[a][b] * H.h2[a][b];
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b)
            for (int g = 0; g < 2; ++g) s3 += A->h3[a][b][g] * H.h3[a][b][g];
    if (order >= 4)
        for (int a = 0; a < 2; ++a)
            for (int b = 0; b < 2; ++b)
                for (int g = 0; g < 2; ++g)
                    for (int d = 0; d < 2; ++d) s4 += A->h4[a][b][g][d] * H.h4[a][b][g][d];
    return L->w[i] * (s0 + s1 + s2 / 2.0 + s3 / 6.0 + s4 / 24.0);
}

/* Exported for the tests: transform Q populations from frame src to frame dst. */
void or_grad_transform(int q1, const double *pops_src, double sux, double suy, double sT,
                       double dux, double duy, double dT, double *pops_dst)
{
    or_lattice L;
    make_lattice(q1, &L);
    or_frame s = {sux, suy, sT}, d = {dux, duy, dT};
    or_tensors A;
    grad_coefficients(&L, pops_src, 1, 3, s, d, &A);
    for (int i = 0; i < L.Q; ++i) pops_dst[i] = grad_population(&L, &A, i, 3);
}

/* Exported for the tests: the same transformation with Grad order N (3 or 4). */
void or_grad_transform_n(int q1, int order, const double *pops_src, double sux, double suy, double sT,
                         double dux, double duy, double dT, double *pops_dst)
{
    or_lattice L;
    make_lattice(q1, &L);
    or_frame s = {sux, suy, sT}, d = {dux, duy, dT};
    or_tensors A;
    grad_coefficients(&L, pops_src, 1, order, s, d, &A);
    for (int i = 0; i < L.Q; ++i) pops_dst[i] = grad_population(&L, &A, i, order);
}

/* Exported for the tests: the Grad coefficient tensors in frame dst, flattened as
 * a0, a1[x,y], a2[xx,xy,yx,yy], a3[xxx,xxy,xyx,xyy,yxx,yxy,yyx,yyy] (15 values). */
void or_grad_coefficients(int q1, const double *pops_src, double sux, double suy, double sT,
                          double dux, double duy, double dT, double *out15)
{
    or_lattice L;
    make_lattice(q1, &L);
    or_frame s = {sux, suy, sT}, d = {dux, duy, dT};
    or_tensors A;
    grad_coefficients(&L, pops_src, 1, 3, s, d, &A);
    int k = 0;
    out15[k++] = A.h0;
    for (int a = 0; a < 2; ++a) out15[k++] = A.h1[a];
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b) out15[k++] = A.h2[a][b];
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b)
            for (int g = 0; g < 2; ++g) out15[k++] = A.h3[a][b][g];
}

/* ---------------------------------------------------------------------------------- */
/* Equilibria in the local frame (Sec. III.A, Eqs. f_eq and the g_eq of each split).   */
/* ---------------------------------------------------------------------------------- */
static double cv_of(double gamma) { return 1.0 / (gamma - 1.0); }   /* Eq. spec_heat, r = 1 */

/* f_eq_i = rho w_i in the frame lambda = (u, T) (Sec. III.A). */
static double feq_pop(const or_lattice *L, int i, double rho) { return rho * L->w[i]; }

/* g_eq_i = (U'/rho + |v|^2/2) f_eq (total split), (U'/rho + |v - u|^2/2) f_eq (internal
 * split) or (U'/rho) f_eq (non-translational split) at v = C_i(lambda);
 * U' = U - rho D T / 2 = rho (c_v - 1) T for D = 2. */
static double geq_pop(const or_lattice *L, int i, int split, double rho, or_frame fr, double cv)
{
    double sT = sqrt(fr.T);
    double Cx = sT * L->cx[i] + fr.ux, Cy = sT * L->cy[i] + fr.uy;
    double Uprime_over_rho = (cv - 1.0) * fr.T;
    double kin;
    if (split == 0)
        kin = 0.5 * (Cx * Cx + Cy * Cy);
    else if (split == 1)
        kin = 0.5 * ((Cx - fr.ux) * (Cx - fr.ux) + (Cy - fr.uy) * (Cy - fr.uy));
    else
        kin = 0.0;
    return (Uprime_over_rho + kin) * feq_pop(L, i, rho);
}

/* Exported: equilibrium populations for fields rho, u, T (the state set by set_state). */
static void node_source(const or_config *cfg, const or_lattice *L, double *g, int x, int y,
                        const double *ux1, const double *uy1, double T1, double rho1, double dtux,
                        double dtuy, double factor);

int or_init(const or_config *cfg, const double *rho, const double *ux, const double *uy,
            const double *T, double *f, double *g, double *fux, double *fuy, double *fT)
{
    or_lattice L;
    make_lattice(cfg->q1, &L);
    double cv = cv_of(cfg->gamma);
    size_t N = (size_t)cfg->nx * cfg->ny;
    for (size_t n = 0; n < N; ++n) {
        or_frame fr = {ux[n], uy[n], T[n]};
        for (int i = 0; i < L.Q; ++i) {
            f[(size_t)i * N + n] = feq_pop(&L, i, rho[n]);
            g[(size_t)i * N + n] = geq_pop(&L, i, cfg->split, rho[n], fr, cv);
        }
        fux[n] = ux[n];
        fuy[n] = uy[n];
        fT[n] = T[n];
    }
    /* internal split: g is carried as g - (Omega + G)/2 and the state is the post-collision
     * one, g - (Omega + G)/2 + Omega + G (see internal_source); at equilibrium (Omega = 0)
     * that is g_eq + G/2, with grad u of the initial fields and d_t u = 0 */
    if (cfg->split == 1)
        for (int y = 0; y < cfg->ny; ++y)
            for (int x = 0; x < cfg->nx; ++x) {
                size_t n = (size_t)y * cfg->nx + x;
                node_source(cfg, &L, g, x, y, ux, uy, T[n], rho[n], 0.0, 0.0, 0.5);
            }
    return 0;
}

/* ---------------------------------------------------------------------------------- */
/* Moments (Sec. II): rho = sum f, rho u = sum C f; total split E = sum g; internal     */
/* split U = sum g, E = U + rho u^2/2; non-translational split E = sum g + sum C^2/2 f. */
/* T from E = rho c_v T + rho u^2 / 2.                                                 */
/* ---------------------------------------------------------------------------------- */
typedef struct { double rho, ux, uy, T, E; } or_moments;

/* div: div u of the node at the new time level (internal split only; 0 elsewhere), for
 * U = sum g + (1/2) sum G = sum g - (1/2) rho T div u. */
static or_moments moments_of_div(const or_lattice *L, const double *f, const double *g, int stride,
                                 or_frame fr, int split, double cv, double div)
{
    double sT = sqrt(fr.T);
    double rho = 0.0, jx = 0.0, jy = 0.0, G = 0.0, K2 = 0.0;
    for (int i = 0; i < L->Q; ++i) {
        double fi = f[(size_t)i * stride], gi = g[(size_t)i * stride];
        double Cx = sT * L->cx[i] + fr.ux, Cy = sT * L->cy[i] + fr.uy;
        rho += fi;
        jx += Cx * fi;
        jy += Cy * fi;
        G += gi;
        K2 += 0.5 * (Cx * Cx + Cy * Cy) * fi;
    }
    or_moments m;
    m.rho = rho;
    m.ux = jx / rho;
    m.uy = jy / rho;
    double u2 = m.ux * m.ux + m.uy * m.uy;
    if (split == 0) {
        m.E = G;
        m.T = (G / rho - 0.5 * u2) / cv;
    } else if (split == 1) {
        m.T = G / (rho * (cv + 0.5 * div));          /* rho c_v T = sum g - (1/2) rho T div u */
        m.E = rho * cv * m.T + 0.5 * rho * u2;
    } else {
        m.E = G + K2;
        m.T = (m.E / rho - 0.5 * u2) / cv;
    }
    return m;
}

static or_moments moments_of(const or_lattice *L, const double *f, const double *g, int stride,
                             or_frame fr, int split, double cv)
{
    return moments_of_div(L, f, g, stride, fr, split, cv, 0.0);
}

/* Exported: rho, u, T of every node from its populations in its own frame (internal split:
 * the temperature is the frame's, the one its last collision relaxed to). */
int or_moments_field(const or_config *cfg, const double *f, const double *g, const double *fux,
                     const double *fuy, const double *fT, double *rho, double *ux, double *uy,
                     double *T, double *E)
{
    or_lattice L;
    make_lattice(cfg->q1, &L);
    double cv = cv_of(cfg->gamma);
    size_t N = (size_t)cfg->nx * cfg->ny;
    for (size_t n = 0; n < N; ++n) {
        or_frame fr = {fux[n], fuy[n], fT[n]};
        or_moments m = moments_of(&L, f + n, g + n, (int)N, fr, cfg->split, cv);
        if (cfg->split == 1) {
            m.T = fT[n];
            m.E = m.rho * cv * m.T + 0.5 * m.rho * (m.ux * m.ux + m.uy * m.uy);
        }
        rho[n] = m.rho;
        ux[n] = m.ux;
        uy[n] = m.uy;
        T[n] = m.T;
        if (E) E[n] = m.E;
    }
    return 0;
}

/* ---------------------------------------------------------------------------------- */
/* Boundaries and Lagrange interpolation kernels                                       */
/* ---------------------------------------------------------------------------------- */
static int bc_map(int j, int n, int bc)
{
    if (bc == 0) {              /* periodic */
        int r = j % n;
        return r < 0 ? r + n : r;
    }
    if (j < 0) return 0;        /* outflow: zero-gradient copy of the edge node; wall: edge node */
    if (j > n - 1) return n - 1;
    return j;
}

/* Which prescribed side (0 x-low, 1 x-high, 2 y-low, 3 y-high) a position lies beyond, or -1:
 * both sides of a wall axis (2), the low side of an inflow axis (3).  A position beyond both
 * a prescribed y side and a prescribed x side belongs to the y side. */
static int wall_of(const or_config *cfg, int gx, int gy)
{
    if ((cfg->bc_y == 2 || cfg->bc_y == 3) && gy < 0) return 2;
    if (cfg->bc_y == 2 && gy > cfg->ny - 1) return 3;
    if ((cfg->bc_x == 2 || cfg->bc_x == 3) && gx < 0) return 0;
    if (cfg->bc_x == 2 && gx > cfg->nx - 1) return 1;
    return -1;
}

/* The prescribed state (u_x, u_y, T, rho) at position (gx, gy) beyond side w: the profile's
 * entry at the position along the side, clamped to the grid, or the side's uniform state. */
static const double *side_state(const or_config *cfg, int w, int gx, int gy)
{
    if (!cfg->profile[w]) return cfg->wall[w];
    int along = w < 2 ? gy : gx, n = w < 2 ? cfg->ny : cfg->nx;
    if (along < 0) along = 0;
    if (along > n - 1) along = n - 1;
    return cfg->profile[w] + 4 * (size_t)along;
}

/* Weights of the stencil whose first node is base at departure point xd: the Lagrange
 * polynomials through the stencil's nodes, t = xd - (base + 1) the position relative to its
 * second node.  For the stencil that lagrange_stencil chooses t lies in [0, 1) (4-point) or
 * [-1/2, 1/2) (3-point); a stencil kept from an earlier departure point may give t slightly
 * outside. */
static void lagrange_weights_at(double xd, int order, int base, double *wts)
{
    double t = xd - (double)(base + 1);
    if (order == 3) {
        /* nodes at -1, 0, 1, 2 */
        wts[0] = -t * (t - 1.0) * (t - 2.0) / 6.0;
        wts[1] = (t + 1.0) * (t - 1.0) * (t - 2.0) / 2.0;
        wts[2] = -(t + 1.0) * t * (t - 2.0) / 2.0;
        wts[3] = (t + 1.0) * t * (t - 1.0) / 6.0;
    } else {
        /* nodes at -1, 0, 1 */
        wts[0] = t * (t - 1.0) / 2.0;
        wts[1] = (1.0 - t) * (1.0 + t);
        wts[2] = t * (t + 1.0) / 2.0;
    }
}

/* Whether the stencil whose first node is base still serves departure point xd: t lies in the
 * range the stencil was chosen for ([0, 1) for 4 points, [-1/2, 1/2) for 3) widened by a
 * quarter cell on each side, so that a kept stencil extrapolates by a quarter cell at most. */
static int stencil_holds(double xd, int order, int base)
{
    double t = xd - (double)(base + 1);
    return order == 3 ? (t >= -0.25 && t < 1.25) : (t >= -0.75 && t < 0.75);
}

/* The stencil of departure point xd: 4-point (order 3) on nodes floor(xd) - 1 .. + 2, or
 * 3-point (order 2) on nodes m - 1 .. m + 1, m = floor(xd + 1/2) (round half up).  Returns its
 * first node; wts receives the weights. */
static int lagrange_stencil(double xd, int order, double *wts)
{
    int base = order == 3 ? (int)floor(xd) - 1 : (int)floor(xd + 0.5) - 1;
    lagrange_weights_at(xd, order, base, wts);
    return base;
}

/* ---------------------------------------------------------------------------------- */
/* Semi-Lagrangian streaming at one node in a given target frame,                      */
/* Eq. (propagationInterpolated): {f_i, g_i}(x) = sum_s W(x - C_i dt - x_s) M{f,g}(x_s) */
/* ---------------------------------------------------------------------------------- */
#define OR_MEMO 1024
typedef struct {
    int64_t key[OR_MEMO];
    or_tensors Af[OR_MEMO], Ag[OR_MEMO];
} or_memo;

typedef struct {
    const or_config *cfg;
    const or_lattice *L;
    const double *f, *g, *fux, *fuy, *fT;   /* post-collision state of the previous step */
} or_src;

static void memo_clear(or_memo *M)
{
    for (int k = 0; k < OR_MEMO; ++k) M->key[k] = -1;
}

/* Grad coefficients, in the target frame, of the populations at position (gx, gy): the node
 * the boundaries map it to, or a wall's ghost equilibrium; memoised per target frame. */
static void source_coefficients(const or_src *S, or_memo *M, int gx, int gy, or_frame dst,
                                const or_tensors **Af, const or_tensors **Ag)
{
    const or_config *cfg = S->cfg;
    int nx = cfg->nx;
    size_t N = (size_t)nx * cfg->ny;
    int sx = bc_map(gx, nx, cfg->bc_x), sy = bc_map(gy, cfg->ny, cfg->bc_y);
    int wall = wall_of(cfg, gx, gy);
    int64_t key = wall < 0 ? (int64_t)sy * nx + sx : -1 - (((int64_t)(gy + 4096) << 20) + (gx + 4096));
    int slot = (int)(((gx & 1023) + 37 * (gy & 1023)) & (OR_MEMO - 1));
    if (M->key[slot] != key) {
        int64_t node = (int64_t)sy * nx + sx;
        if (wall < 0) {
            or_frame src = {S->fux[node], S->fuy[node], S->fT[node]};
            grad_coefficients(S->L, S->f + node, (int)N, grad_order_of(cfg), src, dst, &M->Af[slot]);
            grad_coefficients(S->L, S->g + node, (int)N, grad_order_of(cfg), src, dst, &M->Ag[slot]);
        } else {
            /* ghost: equilibrium at the prescribed state */
            const double *st = side_state(cfg, wall, gx, gy);
            or_frame wf = {st[0], st[1], st[2]};
            double rho_g = st[3];
            double fg[OR_MAXQ], gg[OR_MAXQ];
            for (int i = 0; i < S->L->Q; ++i) {
                fg[i] = feq_pop(S->L, i, rho_g);
                gg[i] = geq_pop(S->L, i, cfg->split, rho_g, wf, cv_of(cfg->gamma));
            }
            grad_coefficients(S->L, fg, 1, grad_order_of(cfg), wf, dst, &M->Af[slot]);
            grad_coefficients(S->L, gg, 1, grad_order_of(cfg), wf, dst, &M->Ag[slot]);
        }
        M->key[slot] = key;
    }
    *Af = &M->Af[slot];
    *Ag = &M->Ag[slot];
}

/* base (optional, 2 Q entries): the first stencil node of each population along x and y.
 * With keep = 0 the stencils are chosen from this frame's departure points and stored in
 * base; with keep = 1 a stored stencil is kept while it still serves the departure point
 * (stencil_holds), only its weights following the frame, and is chosen again and stored
 * otherwise.  The predictor-corrector carries its stencils this way from one iteration to the
 * next. */
static void stream_node_base(const or_src *S, or_memo *M, int x, int y, or_frame bar, int *base, int keep,
                             double *P, double *G)
{
    const or_config *cfg = S->cfg;
    const or_lattice *L = S->L;
    int p = cfg->interp_order == 3 ? 4 : 3;
    double sT = sqrt(bar.T);
    memo_clear(M);
    for (int i = 0; i < L->Q; ++i) {
        double Cx = sT * L->cx[i] + bar.ux, Cy = sT * L->cy[i] + bar.uy;
        double xd = (double)x - Cx * 1.0, yd = (double)y - Cy * 1.0;   /* delta_t = 1 */
        double wx[4], wy[4];
        int bx, by;
        if (base && keep && stencil_holds(xd, cfg->interp_order, base[i]))
            lagrange_weights_at(xd, cfg->interp_order, bx = base[i], wx);
        else
            bx = lagrange_stencil(xd, cfg->interp_order, wx);
        if (base && keep && stencil_holds(yd, cfg->interp_order, base[L->Q + i]))
            lagrange_weights_at(yd, cfg->interp_order, by = base[L->Q + i], wy);
        else
            by = lagrange_stencil(yd, cfg->interp_order, wy);
        if (base) {
            base[i] = bx;
            base[L->Q + i] = by;
        }
        double fi = 0.0, gi = 0.0;
        for (int ky = 0; ky < p; ++ky) {
            for (int kx = 0; kx < p; ++kx) {
                const or_tensors *Af, *Ag;
                source_coefficients(S, M, bx + kx, by + ky, bar, &Af, &Ag);
                double W = wx[kx] * wy[ky];
                fi += W * grad_population(L, Af, i, grad_order_of(cfg));
                gi += W * grad_population(L, Ag, i, grad_order_of(cfg));
            }
        }
        P[i] = fi;
        G[i] = gi;
    }
}

/* Streaming with the stencils of this frame's departure points. */
static void stream_node(const or_src *S, or_memo *M, int x, int y, or_frame bar, double *P, double *G)
{
    stream_node_base(S, M, x, y, bar, NULL, 0, P, G);
}

/* Exported for the tests: stream at node (x, y) in a prescribed frame. */
int or_stream_node(const or_config *cfg, const double *f, const double *g, const double *fux,
                   const double *fuy, const double *fT, int x, int y, double ux, double uy,
                   double T, double *P, double *G)
{
    or_lattice L;
    make_lattice(cfg->q1, &L);
    or_src S = {cfg, &L, f, g, fux, fuy, fT};
    or_memo *M = (or_memo *)malloc(sizeof(or_memo));
    if (!M) return -2;
    or_frame bar = {ux, uy, T};
    stream_node(&S, M, x, y, bar, P, G);
    free(M);
    return 0;
}

/* Exported for the tests: stream at node (x, y) in frame (ux, uy, T) with the stencils that
 * the departure points of frame (sux, suy, sT) select (as the predictor-corrector keeps the
 * stencils of its first iteration). */
int or_stream_node_kept(const or_config *cfg, const double *f, const double *g, const double *fux,
                        const double *fuy, const double *fT, int x, int y, double ux, double uy,
                        double T, double sux, double suy, double sT, double *P, double *G)
{
    or_lattice L;
    make_lattice(cfg->q1, &L);
    or_src S = {cfg, &L, f, g, fux, fuy, fT};
    or_memo *M = (or_memo *)malloc(sizeof(or_memo));
    if (!M) return -2;
    int base[2 * OR_MAXQ];
    or_frame sel = {sux, suy, sT}, bar = {ux, uy, T};
    stream_node_base(&S, M, x, y, sel, base, 0, P, G);   /* chooses the stencils */
    stream_node_base(&S, M, x, y, bar, base, 1, P, G);
    free(M);
    return 0;
}

/* ---------------------------------------------------------------------------------- */
/* BGK collision in the frame of the final moments (Eq. boltz_eq discretised).         */
/* ---------------------------------------------------------------------------------- */
static void collide_node(const or_lattice *L, const or_config *cfg, const double *P, const double *G,
                         or_frame bar, or_moments m, double *fo, double *go)
{
    double cv = cv_of(cfg->gamma);
    or_frame star = {m.ux, m.uy, m.T};
    or_tensors Af, Ag;
    grad_coefficients(L, P, 1, grad_order_of(cfg), bar, star, &Af);   /* project the streamed populations into lambda* */
    grad_coefficients(L, G, 1, grad_order_of(cfg), bar, star, &Ag);
    double rho = m.rho;
    double tau = cfg->mu / (rho * m.T);             /* Eq. kin_visc: tau = mu / p, p = rho T */
    double omega = 1.0 / (tau + 0.5);
    for (int i = 0; i < L->Q; ++i) {
        double fp = grad_population(L, &Af, i, grad_order_of(cfg));
        double gp = grad_population(L, &Ag, i, grad_order_of(cfg));
        double fe = feq_pop(L, i, rho);
        double ge = geq_pop(L, i, cfg->split, rho, star, cv);
        fo[i] = fp + omega * (fe - fp);
        go[i] = gp + omega * (ge - gp);
    }
}

static int nonphysical(or_moments m)
{
    return !(m.rho > 0.0) || !(m.T > 0.0) || isnan(m.ux) || isnan(m.uy) || isnan(m.E);
}

/* ---------------------------------------------------------------------------------- */
/* Internal-energy split source (Eq. int_g_evolution, Appendix A G term):              */
/*   G_i = -rho w_i (C_i - u) . (d_t u + C_i . grad u), f -> f_eq inside the source.   */
/* ---------------------------------------------------------------------------------- */
/* Velocity at position (gx, gy) of the fields ux, uy: the mapped node's, or the prescribed
 * velocity beyond a prescribed side. */
static void velocity_at(const or_config *cfg, const double *ux, const double *uy, int gx, int gy,
                        double *vx, double *vy)
{
    int w = wall_of(cfg, gx, gy);
    if (w >= 0) {
        const double *st = side_state(cfg, w, gx, gy);
        *vx = st[0];
        *vy = st[1];
    } else {
        size_t m = (size_t)bc_map(gy, cfg->ny, cfg->bc_y) * cfg->nx + bc_map(gx, cfg->nx, cfg->bc_x);
        *vx = ux[m];
        *vy = uy[m];
    }
}

/* Central differences of the velocity field at node (x, y): d_x u_x, d_y u_x, d_x u_y, d_y u_y. */
static void velocity_gradient(const or_config *cfg, const double *ux, const double *uy, int x, int y,
                              double grad[4])
{
    const int nb[4][2] = {{x + 1, y}, {x - 1, y}, {x, y + 1}, {x, y - 1}};
    double vx[4], vy[4];
    for (int k = 0; k < 4; ++k) velocity_at(cfg, ux, uy, nb[k][0], nb[k][1], &vx[k], &vy[k]);
    grad[0] = 0.5 * (vx[0] - vx[1]);
    grad[1] = 0.5 * (vx[2] - vx[3]);
    grad[2] = 0.5 * (vy[0] - vy[1]);
    grad[3] = 0.5 * (vy[2] - vy[3]);
}

/* Adds factor * G to the populations g of node (x, y) (n = its index), G at velocity field
 * ux1, uy1 (whose central differences give grad u), temperature T1, density rho1 and time
 * derivative (dtux, dtuy). */
static void node_source(const or_config *cfg, const or_lattice *L, double *g, int x, int y,
                        const double *ux1, const double *uy1, double T1, double rho1, double dtux,
                        double dtuy, double factor)
{
    size_t N = (size_t)cfg->nx * cfg->ny, n = (size_t)y * cfg->nx + x;
    double gr[4];
    velocity_gradient(cfg, ux1, uy1, x, y, gr);
    double dxux = gr[0], dyux = gr[1], dxuy = gr[2], dyuy = gr[3];
    double sT = sqrt(T1);
    for (int i = 0; i < L->Q; ++i) {
        double Cx = sT * L->cx[i] + ux1[n], Cy = sT * L->cy[i] + uy1[n];
        double ax = dtux + Cx * dxux + Cy * dyux;     /* d_t u_x + C . grad u_x */
        double ay = dtuy + Cx * dxuy + Cy * dyuy;
        double Gi = -rho1 * L->w[i] * ((Cx - ux1[n]) * ax + (Cy - uy1[n]) * ay);
        g[(size_t)i * N + n] += factor * Gi;
    }
}

/* Adds (1 - omega/2) G to the post-collision g of every node (the trapezoidal rule along the
 * characteristics), with u, T, rho of the new time level, d_t u = u^{n+1} - u^n (delta_t = 1). */
static void internal_source(const or_config *cfg, const or_lattice *L, double *g, const double *ux1,
                            const double *uy1, const double *T1, const double *rho1,
                            const double *ux0, const double *uy0)
{
    int nx = cfg->nx, ny = cfg->ny;
#pragma omp parallel for schedule(static)
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            size_t n = (size_t)y * nx + x;
            double tau = cfg->mu / (rho1[n] * T1[n]);
            double omega = 1.0 / (tau + 0.5);
            node_source(cfg, L, g, x, y, ux1, uy1, T1[n], rho1[n], ux1[n] - ux0[n], uy1[n] - uy0[n],
                        1.0 - 0.5 * omega);
        }
}

/* Predictor velocity of the internal split at node (x, y): rho u of the populations f
 * streamed once in the node's previous frame, over rho. */
static void predictor_velocity(const or_src *S, or_memo *M, int x, int y, double *upx, double *upy)
{
    const or_lattice *L = S->L;
    size_t n = (size_t)y * S->cfg->nx + x;
    or_frame bar = {S->fux[n], S->fuy[n], S->fT[n]};
    double P[OR_MAXQ], G[OR_MAXQ];
    stream_node(S, M, x, y, bar, P, G);
    double sT = sqrt(bar.T), rho = 0.0, jx = 0.0, jy = 0.0;
    for (int i = 0; i < L->Q; ++i) {
        rho += P[i];
        jx += (sT * L->cx[i] + bar.ux) * P[i];
        jy += (sT * L->cy[i] + bar.uy) * P[i];
    }
    *upx = jx / rho;
    *upy = jy / rho;
}

/* ---------------------------------------------------------------------------------- */
/* One time step.  Input state (f, g, frames) at time n, output state at n + 1.        */
/* iters (optional, per node): predictor-corrector iterations used.                    */
/* Returns: 0, or -4 if a non-physical state was met, or -5 if some node did not       */
/* converge within pc_max_iter (state still advanced).  first_bad receives the first   */
/* non-physical node (or -1).                                                          */
/* ---------------------------------------------------------------------------------- */
/* Predictor-corrector and collision at one node (x, y): streamed populations in successive
 * frames until the frame converges (or K iterations in fixed mode), then BGK in the frame of
 * the final moments.  div: div u of the node at the new time level (internal split).  Writes
 * the node's post-collision populations fo_n, go_n and its moments.  Returns the iteration
 * count; *badnode / *nonconv flag the outcomes. */
static int step_node(const or_src *S, or_memo *M, int x, int y, double div, double *fo_n, double *go_n,
                     or_moments *mout, int *badnode, int *nonconv)
{
    const or_config *cfg = S->cfg;
    const or_lattice *L = S->L;
    double cv = cv_of(cfg->gamma);
    size_t n = (size_t)y * cfg->nx + x;
    double P[OR_MAXQ], G[OR_MAXQ];
    or_frame bar = {S->fux[n], S->fuy[n], S->fT[n]};        /* predictor: previous frame */
    or_moments m;
    int k = 0, stop = 0;
    int base[2 * OR_MAXQ];                     /* stencils of the first iteration, kept */
    *badnode = 0;
    *nonconv = 0;
    while (!stop) {
        stream_node_base(S, M, x, y, bar, base, k > 0, P, G);
        m = moments_of_div(L, P, G, 1, bar, cfg->split, cv, div);
        ++k;
        if (nonphysical(m)) { *badnode = 1; break; }
        double du = sqrt((m.ux - bar.ux) * (m.ux - bar.ux) + (m.uy - bar.uy) * (m.uy - bar.uy));
        double change = fmax(du / sqrt(bar.T), fabs(m.T - bar.T) / bar.T);
        if (cfg->pc_fixed_iters > 0) {
            stop = (k >= cfg->pc_fixed_iters);
        } else if (change <= cfg->pc_tol) {
            stop = 1;
        } else if (k >= cfg->pc_max_iter) {
            stop = 1;
            *nonconv = 1;
        }
        if (!stop) {                                   /* corrector: frame of the moments */
            bar.ux = m.ux;
            bar.uy = m.uy;
            bar.T = m.T;
        }
    }
    *mout = m;
    if (*badnode) {
        for (int i = 0; i < L->Q; ++i) { fo_n[i] = NAN; go_n[i] = NAN; }
        return k;
    }
    collide_node(L, cfg, P, G, bar, m, fo_n, go_n);
    return k;
}

int or_step(const or_config *cfg, const double *f, const double *g, const double *fux,
            const double *fuy, const double *fT, double *fo, double *go, double *oux,
            double *ouy, double *oT, int32_t *iters, int64_t *first_bad)
{
    or_lattice L;
    make_lattice(cfg->q1, &L);
    int nx = cfg->nx, ny = cfg->ny;
    size_t N = (size_t)nx * ny;
    or_src S = {cfg, &L, f, g, fux, fuy, fT};
    int64_t nonconv = 0, bad = -1;
    double *rho1 = (double *)malloc(N * sizeof(double));
    if (!rho1) return -2;
    /* internal split: predictor velocities of every node (div u at the new time level) */
    double *upx = NULL, *upy = NULL;
    if (cfg->split == 1) {
        upx = (double *)malloc(N * sizeof(double));
        upy = (double *)malloc(N * sizeof(double));
        if (!upx || !upy) {
            free(rho1);
            free(upx);
            free(upy);
            return -2;
        }
#pragma omp parallel
        {
            or_memo *M = (or_memo *)malloc(sizeof(or_memo));
#pragma omp for schedule(static)
            for (int64_t n = 0; n < (int64_t)N; ++n)
                predictor_velocity(&S, M, (int)(n % nx), (int)(n / nx), &upx[n], &upy[n]);
            free(M);
        }
    }

#pragma omp parallel reduction(+ : nonconv)
    {
        or_memo *M = (or_memo *)malloc(sizeof(or_memo));
        double fo_n[OR_MAXQ], go_n[OR_MAXQ];
#pragma omp for schedule(static)
        for (int64_t n = 0; n < (int64_t)N; ++n) {
            int x = (int)(n % nx), y = (int)(n / nx);
            or_moments m;
            int badnode, nc;
            double div = 0.0;
            if (cfg->split == 1) {
                double gr[4];
                velocity_gradient(cfg, upx, upy, x, y, gr);
                div = gr[0] + gr[3];
            }
            int k = step_node(&S, M, x, y, div, fo_n, go_n, &m, &badnode, &nc);
            nonconv += nc;
            if (iters) iters[n] = k;
            if (badnode) {
#pragma omp critical
                { if (bad < 0 || n < bad) bad = n; }
            }
            for (int i = 0; i < L.Q; ++i) {
                fo[(size_t)i * N + n] = fo_n[i];
                go[(size_t)i * N + n] = go_n[i];
            }
            oux[n] = m.ux;
            ouy[n] = m.uy;
            oT[n] = m.T;
            rho1[n] = m.rho;
        }
        free(M);
    }
    if (cfg->split == 1 && bad < 0)
        internal_source(cfg, &L, go, oux, ouy, oT, rho1, fux, fuy);
    free(rho1);
    free(upx);
    free(upy);
    if (first_bad) *first_bad = bad;
    if (bad >= 0) return -4;
    if (nonconv > 0) return -5;
    return 0;
}

/* Exported for the tests: one time step at the nodes listed in xs, ys only (the internal
 * split before its source pass, with the predictor velocities of the four neighbours), from
 * the full state of the previous step: fo, go [Q][count], frame [3][count] (ux, uy, T),
 * iters [count]. */
int or_step_nodes(const or_config *cfg, const double *f, const double *g, const double *fux,
                  const double *fuy, const double *fT, int count, const int32_t *xs,
                  const int32_t *ys, double *fo, double *go, double *frame, int32_t *iters)
{
    for (int k = 0; k < count; ++k)          /* nodes outside the grid are an error */
        if (xs[k] < 0 || xs[k] >= cfg->nx || ys[k] < 0 || ys[k] >= cfg->ny) return -1;
    or_lattice L;
    make_lattice(cfg->q1, &L);
    or_src S = {cfg, &L, f, g, fux, fuy, fT};
    int rc = 0;
#pragma omp parallel
    {
        or_memo *M = (or_memo *)malloc(sizeof(or_memo));
        double fo_n[OR_MAXQ], go_n[OR_MAXQ];
#pragma omp for schedule(dynamic)
        for (int j = 0; j < count; ++j) {
            or_moments m;
            int badnode, nc;
            double div = 0.0;
            if (cfg->split == 1) {
                /* div u_pred by central differences; beyond a prescribed side its velocity */
                const int x = xs[j], y = ys[j];
                const int nb[4][2] = {{x + 1, y}, {x - 1, y}, {x, y + 1}, {x, y - 1}};
                double vx[4], vy[4];
                for (int q = 0; q < 4; ++q) {
                    int w = wall_of(cfg, nb[q][0], nb[q][1]);
                    if (w >= 0) {
                        const double *st = side_state(cfg, w, nb[q][0], nb[q][1]);
                        vx[q] = st[0];
                        vy[q] = st[1];
                    } else {
                        predictor_velocity(&S, M, bc_map(nb[q][0], cfg->nx, cfg->bc_x),
                                           bc_map(nb[q][1], cfg->ny, cfg->bc_y), &vx[q], &vy[q]);
                    }
                }
                div = 0.5 * (vx[0] - vx[1]) + 0.5 * (vy[2] - vy[3]);
            }
            int k = step_node(&S, M, xs[j], ys[j], div, fo_n, go_n, &m, &badnode, &nc);
            if (iters) iters[j] = k;
            if (badnode) rc = -4;
            for (int i = 0; i < L.Q; ++i) {
                fo[(size_t)i * count + j] = fo_n[i];
                go[(size_t)i * count + j] = go_n[i];
            }
            frame[j] = m.ux;
            frame[count + j] = m.uy;
            frame[2 * count + j] = m.T;
        }
        free(M);
    }
    return rc;
}

/* Exported for the tests: predictor-corrector-free collision of streamed populations P, G
 * living on the lattice of frame (bux, buy, bT): moments, projection into their frame,
 * BGK relaxation.  Writes the post-collision populations and their frame (ux, uy, T). */
int or_collide_node(const or_config *cfg, const double *P, const double *G, double bux,
                    double buy, double bT, double *fo, double *go, double *frame_out)
{
    or_lattice L;
    make_lattice(cfg->q1, &L);
    or_frame bar = {bux, buy, bT};
    or_moments m = moments_of(&L, P, G, 1, bar, cfg->split, cv_of(cfg->gamma));
    if (nonphysical(m)) return -4;
    collide_node(&L, cfg, P, G, bar, m, fo, go);
    frame_out[0] = m.ux;
    frame_out[1] = m.uy;
    frame_out[2] = m.T;
    return 0;
}
