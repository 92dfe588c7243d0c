"""A third implementation of the PonD step in 50-digit arithmetic (mpmath), for tiny periodic
grids: test infrastructure that pins the FP64 oracle's rounding.  It is written separately
from the oracle (no shared code) and follows the paper with the same readings:

- lattice: D1Q4 / D1Q5 Gauss-Hermite rules (Table I) in closed form, tensor products;
- frame transformation (Eq. gradGeneralTransform, N = 3 on D2Q16, 4 on D2Q25): Hermite
  coefficients of the source populations about the target frame,
  A_pq = sum_j f_j He_p(xi_jx) He_q(xi_jy) with xi_j = (C_j - u_bar)/sqrt(T_bar),
  p + q <= N, and the target populations w_i sum_{p+q<=N} A_pq He_p(c_ix) He_q(c_iy) / (p! q!);
- streaming (Eq. propagationInterpolated): cubic Lagrange interpolation at the departure
  point x - C_i(lambda_bar) of every stencil node's populations moved into lambda_bar;
- predictor-corrector: guess = previous frame, exactly K iterations, the stencil nodes of
  each population carried from one iteration to the next (their weights following the frame)
  while the departure point stays within a quarter cell of the range they were chosen for;
- collision: project into the frame of the final moments, BGK with omega = 1/(tau + 1/2),
  tau = mu/(rho T), f_eq = rho w_i, g_eq of the total, internal or non-translational split
  (Sec. II; the last with E = sum g + sum |C|^2/2 f);
- internal split: the source G_i = -rho w_i (C_i - u).(d_t u + C_i . grad u) by the
  trapezoidal rule along the characteristics: T from U = sum g + (1/2) sum G =
  sum g - (1/2) rho T div u, with div u from the predictor velocities (rho u of one streaming
  of f in each node's previous frame, central differences), and (1 - omega/2) G added after
  the collision, with d_t u = u^{n+1} - u^n and central differences of u^{n+1}.
"""
import mpmath as mp

mp.mp.dps = 50


def rule(q1):
    """Table I: nodes and weights of the 1-D Gauss-Hermite rule (ascending nodes)."""
    if q1 == 4:
        s6 = mp.sqrt(6)
        ci, co = mp.sqrt(3 - s6), mp.sqrt(3 + s6)
        wi, wo = (3 + s6) / 12, (3 - s6) / 12
        return [-co, -ci, ci, co], [wo, wi, wi, wo]
    s10 = mp.sqrt(10)
    ci, co = mp.sqrt(5 - s10), mp.sqrt(5 + s10)
    wi, wo = (7 + 2 * s10) / 60, (7 - 2 * s10) / 60
    return [-co, -ci, mp.mpf(0), ci, co], [wo, wi, mp.mpf(8) / 15, wi, wo]


def he(n, x):
    return (mp.mpf(1), x, x * x - 1, x * x * x - 3 * x, x ** 4 - 6 * x * x + 3)[n]


FACT = (1, 1, 2, 6, 24)


class Lattice:
    def __init__(self, q1, N=None):
        c, w = rule(q1)
        self.q1 = q1
        self.N = N if N else (4 if q1 == 5 else 3)
        self.orders = [(p, q) for p in range(self.N + 1) for q in range(self.N + 1 - p)]
        self.Q = q1 * q1
        self.cx = [c[i % q1] for i in range(self.Q)]      # population i = b q1 + a
        self.cy = [c[i // q1] for i in range(self.Q)]
        self.w = [w[i % q1] * w[i // q1] for i in range(self.Q)]


def coefficients(lat, pops, src, dst):
    """Hermite coefficients (p + q <= N) about frame dst of populations given in frame src."""
    sTs, sTd = mp.sqrt(src[2]), mp.sqrt(dst[2])
    A = {pq: mp.mpf(0) for pq in lat.orders}
    for j in range(lat.Q):
        xi_x = (sTs * lat.cx[j] + src[0] - dst[0]) / sTd
        xi_y = (sTs * lat.cy[j] + src[1] - dst[1]) / sTd
        hx = [he(n, xi_x) for n in range(lat.N + 1)]
        hy = [he(n, xi_y) for n in range(lat.N + 1)]
        for (p, q) in lat.orders:
            A[(p, q)] += pops[j] * hx[p] * hy[q]
    return A


def population(lat, A, i):
    s = mp.mpf(0)
    for (p, q) in lat.orders:
        s += A[(p, q)] * he(p, lat.cx[i]) * he(q, lat.cy[i]) / (FACT[p] * FACT[q])
    return lat.w[i] * s


def cubic_weights(t):
    return [-t * (t - 1) * (t - 2) / 6, (t + 1) * (t - 1) * (t - 2) / 2,
            -(t + 1) * t * (t - 2) / 2, (t + 1) * t * (t - 1) / 6]


def cubic(xd, first=None):
    """First node and weights of the 4-point stencil at departure point xd; with first given,
    the weights of that stencil (nodes first .. first + 3) at xd if xd lies within a quarter
    cell of the range it was chosen for, else the stencil xd selects."""
    if first is None or not (-mp.mpf(1) / 4 <= xd - (first + 1) < mp.mpf(5) / 4):
        first = int(mp.floor(xd)) - 1
    return first, cubic_weights(xd - (first + 1))


def g_eq(lat, i, split, rho, fr, cv):
    sT = mp.sqrt(fr[2])
    Cx, Cy = sT * lat.cx[i] + fr[0], sT * lat.cy[i] + fr[1]
    if split == "total":
        kin = (Cx * Cx + Cy * Cy) / 2
    elif split == "internal":
        kin = ((Cx - fr[0]) ** 2 + (Cy - fr[1]) ** 2) / 2
    else:
        kin = 0
    return ((cv - 1) * fr[2] + kin) * rho * lat.w[i]


def moments(lat, P, G, fr, split, cv, div=0):
    sT = mp.sqrt(fr[2])
    rho = sum(P)
    jx = sum((sT * lat.cx[i] + fr[0]) * P[i] for i in range(lat.Q))
    jy = sum((sT * lat.cy[i] + fr[1]) * P[i] for i in range(lat.Q))
    ux, uy = jx / rho, jy / rho
    if split == "total":
        T = (sum(G) / rho - (ux * ux + uy * uy) / 2) / cv
    elif split == "internal":
        T = sum(G) / (rho * (cv + div / 2))
    else:
        K2 = sum(((sT * lat.cx[i] + fr[0]) ** 2 + (sT * lat.cy[i] + fr[1]) ** 2) / 2 * P[i]
                 for i in range(lat.Q))
        T = ((sum(G) + K2) / rho - (ux * ux + uy * uy) / 2) / cv
    return rho, ux, uy, T


def init(lat, nx, ny, rho, ux, uy, T, split, gamma):
    """Equilibrium state from double fields [ny][nx]; pops [n][i], frames [n]."""
    cv = 1 / (mp.mpf(gamma) - 1)
    st = {"f": [], "g": [], "fr": []}
    for y in range(ny):
        for x in range(nx):
            r = mp.mpf(float(rho[y][x]))
            fr = (mp.mpf(float(ux[y][x])), mp.mpf(float(uy[y][x])), mp.mpf(float(T[y][x])))
            st["f"].append([r * lat.w[i] for i in range(lat.Q)])
            st["g"].append([g_eq(lat, i, split, r, fr, cv) for i in range(lat.Q)])
            st["fr"].append(fr)
    if split == "internal":
        # post-collision state of g carried as g - (Omega + G)/2: at equilibrium g_eq + G/2
        # (d_t u = 0 at the start)
        add_source(lat, st, st["fr"], [(0, 0)] * (nx * ny), nx, ny, lambda n: mp.mpf(1) / 2)
    return st


def stream(lat, st, nx, ny, x, y, bar, stencils=None):
    """Populations f, g streamed to node (x, y) on the lattice of frame bar.  stencils: a
    dict population -> (first x node, first y node), carried between calls (see cubic)."""
    cache = {}
    sT = mp.sqrt(bar[2])
    P, G = [], []
    for i in range(lat.Q):
        keep = stencils.get(i) if stencils is not None else None
        bx, wx = cubic(x - (sT * lat.cx[i] + bar[0]), keep[0] if keep else None)
        by, wy = cubic(y - (sT * lat.cy[i] + bar[1]), keep[1] if keep else None)
        if stencils is not None:
            stencils[i] = (bx, by)
        fi = gi = mp.mpf(0)
        for ky in range(4):
            for kx in range(4):
                s = ((by + ky) % ny) * nx + (bx + kx) % nx
                if s not in cache:
                    cache[s] = (coefficients(lat, st["f"][s], st["fr"][s], bar),
                                coefficients(lat, st["g"][s], st["fr"][s], bar))
                W = wx[kx] * wy[ky]
                fi += W * population(lat, cache[s][0], i)
                gi += W * population(lat, cache[s][1], i)
        P.append(fi)
        G.append(gi)
    return P, G


def divergence(lat, st, nx, ny):
    """Internal split: div u at the new time level from the predictor velocities (rho u / rho
    of f streamed once in each node's previous frame), central differences, periodic."""
    up = []
    for y in range(ny):
        for x in range(nx):
            bar = st["fr"][y * nx + x]
            P, _ = stream(lat, st, nx, ny, x, y, bar)
            sT = mp.sqrt(bar[2])
            rho = sum(P)
            up.append((sum((sT * lat.cx[i] + bar[0]) * P[i] for i in range(lat.Q)) / rho,
                       sum((sT * lat.cy[i] + bar[1]) * P[i] for i in range(lat.Q)) / rho))
    div = []
    for y in range(ny):
        for x in range(nx):
            xp, xm = y * nx + (x + 1) % nx, y * nx + (x - 1) % nx
            yp, ym = ((y + 1) % ny) * nx + x, ((y - 1) % ny) * nx + x
            div.append((up[xp][0] - up[xm][0]) / 2 + (up[yp][1] - up[ym][1]) / 2)
    return div


def step(lat, st, nx, ny, split, gamma, mu, K):
    """One time step of the whole (periodic) grid with exactly K PC iterations per node."""
    cv = 1 / (mp.mpf(gamma) - 1)
    mu = mp.mpf(mu)
    out = {"f": [], "g": [], "fr": []}
    div = divergence(lat, st, nx, ny) if split == "internal" else None
    for y in range(ny):
        for x in range(nx):
            bar = st["fr"][y * nx + x]
            stencils = {}
            for k in range(K):
                P, G = stream(lat, st, nx, ny, x, y, bar, stencils)
                m = moments(lat, P, G, bar, split, cv, div[y * nx + x] if div else 0)
                if k < K - 1:
                    bar = (m[1], m[2], m[3])
            rho, star = m[0], (m[1], m[2], m[3])
            Af = coefficients(lat, P, bar, star)
            Ag = coefficients(lat, G, bar, star)
            omega = 1 / (mu / (rho * star[2]) + mp.mpf(1) / 2)
            fo, go = [], []
            for i in range(lat.Q):
                fp, gp = population(lat, Af, i), population(lat, Ag, i)
                fo.append(fp + omega * (rho * lat.w[i] - fp))
                go.append(gp + omega * (g_eq(lat, i, split, rho, star, cv) - gp))
            out["f"].append(fo)
            out["g"].append(go)
            out["fr"].append(star)
    if split == "internal":
        internal_source(lat, st, out, nx, ny, mu)
    return out


def add_source(lat, st, frames, dtu, nx, ny, factor):
    """Adds factor(n) * G to st's g at every node n, G with the velocities and temperatures of
    frames (central differences, periodic), rho of st's f and time derivatives dtu[n]."""
    ux = [fr[0] for fr in frames]
    uy = [fr[1] for fr in frames]
    for y in range(ny):
        for x in range(nx):
            n = y * nx + x
            xp, xm = y * nx + (x + 1) % nx, y * nx + (x - 1) % nx
            yp, ym = ((y + 1) % ny) * nx + x, ((y - 1) % ny) * nx + x
            dxux, dyux = (ux[xp] - ux[xm]) / 2, (ux[yp] - ux[ym]) / 2
            dxuy, dyuy = (uy[xp] - uy[xm]) / 2, (uy[yp] - uy[ym]) / 2
            dtux, dtuy = dtu[n]
            rho = sum(st["f"][n])
            sT = mp.sqrt(frames[n][2])
            fac = factor(n)
            for i in range(lat.Q):
                Cx, Cy = sT * lat.cx[i] + ux[n], sT * lat.cy[i] + uy[n]
                ax = dtux + Cx * dxux + Cy * dyux
                ay = dtuy + Cx * dxuy + Cy * dyuy
                st["g"][n][i] += -fac * rho * lat.w[i] * ((Cx - ux[n]) * ax + (Cy - uy[n]) * ay)


def internal_source(lat, before, after, nx, ny, mu):
    """(1 - omega/2) G after the collision, d_t u = u^{n+1} - u^n."""
    fr1, fr0 = after["fr"], before["fr"]
    dtu = [(fr1[n][0] - fr0[n][0], fr1[n][1] - fr0[n][1]) for n in range(nx * ny)]

    def factor(n):
        omega = 1 / (mu / (sum(after["f"][n]) * fr1[n][2]) + mp.mpf(1) / 2)
        return 1 - omega / 2
    add_source(lat, after, fr1, dtu, nx, ny, factor)
