"""P-multigrid pseudo-time solver of one dual time step, in plain FP64
(test infrastructure).

Sec. 5 (application of the methods): the pseudo-iterations of each BDF2
physical step are accelerated by P-multigrid - the same mesh at the orders
p, p-1, ..., each level smoothed by pseudo-time steps, coarse levels
correcting the finer ones - in an asymmetric cycle given as (order,
iterations) pairs (Fig. pmg: (4,1), (3,1), (2,1), (1,4), (2,1), (3,1),
(4,7)), with the pseudo step multiplied by a constant factor (1.75) per
order below the finest.  The paper cites its multigrid and gives no
formulas; the readings taken here:

  * full approximation scheme (FAS).  With N(U) = R(U) - I_V (a0/dt) V the
    state-dependent part of the pseudo RHS and g a constant forcing, level q
    solves N_q(U_q) + g_q = 0.  The finest level's forcing is the constant
    BDF part -(a1 V^n + a2 V^{n-1})/dt on the velocity rows.  Going down
    from q to q-1: U0_{q-1} = I_r U_q, U_{q-1} = U0_{q-1},
    g_{q-1} = I_r (N_q(U_q) + g_q) - N_{q-1}(U0_{q-1}).  Going up from q-1
    to q: U_q += I_p (U_{q-1} - U0_{q-1});
  * the cycle's consecutive orders differ by one; each entry first moves to
    its order (down: restrict, up: prolong the correction), then smooths;
  * restriction I_r: per element and direction, the L2 projection onto
    polynomials of degree q-1, in nodal values at the coarse Gauss-Legendre
    points: I_r[i, k] = w^f_k l^c_i(x^f_k) / w^c_i (the fine rule integrates
    the products exactly; the coarse mass matrix is diag(w^c));
    prolongation I_p: evaluation of the coarse polynomial at the fine
    points, I_p[k, i] = l^c_i(x^f_k);
  * smoother: classical RK4 in pseudo time on dU/dtau = D (N(U) + g), D a
    constant diagonal scaling: 1 on the P rows, 1/(1 + dtau a0/dt) on the
    velocity rows, 1/(1 + dtau / T) on the gradient rows (a point-implicit
    treatment of the two linear stiff terms, -a0/dt V and -q/T; it is not in
    the paper, and it leaves the fixed point unchanged).  Without scaling,
    D = 1 and a level's smoothing is exactly timestep.pseudo_solve's RK4;
  * convergence: the finest level's velocity residual (RMS of N + g over
    the velocity rows), taken at the start of each cycle.

Anderson mixing over the cycles (Anderson class; not in the paper) is an
option of pseudo_solve.

Pins (tests/test_oracle_pmg.py): transfer operators exact on polynomials
(prolongation of degree <= q-1, restriction reproduces them, restriction
after prolongation is the identity, the projection error is orthogonal to
the coarse space); the scaled RK4 step on a pure relaxation equation is the
RK4 stability polynomial of -lambda dtau / (1 + lambda dtau); a converged
state is a fixed point of a cycle; cycles converge to the same state as
plain RK4 pseudo-stepping; Anderson mixing terminates on a linear map of
dimension n within n + 1 steps (its equivalence with GMRES) and is the plain
iteration for m = 0.
"""
import numpy as np

from . import fr, ops1d, timestep


def transfer_1d(order_f, order_c):
    """(I_r, I_p): restriction (m_c x m_f) and prolongation (m_f x m_c)."""
    xf, wf = ops1d.gauss_legendre(order_f + 1)
    xc, wc = ops1d.gauss_legendre(order_c + 1)
    Lc_at_f = ops1d.lagrange(xc, xf)          # [k, i] = l^c_i(x^f_k)
    Ip = Lc_at_f
    Ir = (Lc_at_f * wf[:, None]).T / wc[:, None]
    return Ir, Ip


def apply_tensor(A, U, d):
    """Apply the 1-D operator A (r x m) along every direction of each
    element: U [nv, m^d, ne] -> [nv, r^d, ne] (pt = i + m j + m^2 k)."""
    nv, npt, ne = U.shape
    m = A.shape[1]
    r = A.shape[0]
    G = U.reshape((nv,) + (m,) * d + (ne,))      # axes (v, [k,] j, i, e)
    for a in range(d):
        ax = d - a                                # direction a's axis
        G = np.moveaxis(np.tensordot(A, G, axes=([1], [ax])), 0, ax)
    return G.reshape(nv, r ** d, ne)


class Level:
    """One order of the hierarchy: the oracle's RHS at that order."""

    def __init__(self, mesh, order, params, correction="dg"):
        self.mesh, self.order, self.params, self.correction = mesh, order, params, correction
        self.ops = ops1d.Ops1D(order, correction)

    def N(self, U, a0dt):
        """R(U) - I_V (a0/dt) V."""
        R = fr.rhs(U, self.mesh, self.order, self.params, self.correction, ops=self.ops)
        d = self.mesh.d
        R[1:1 + d] -= a0dt * U[1:1 + d]
        return R


def scaling(d, nv, dtau, a0dt, T, implicit):
    """Diagonal D of the smoother, per variable."""
    D = np.ones(nv)
    if implicit:
        D[1:1 + d] = 1.0 / (1.0 + dtau * a0dt)
        D[1 + d:] = 1.0 / (1.0 + dtau / T)
    return D[:, None, None]


def smooth(level, U, g, a0dt, dtau, iters, implicit):
    """`iters` RK4 pseudo steps on dU/dtau = D (N(U) + g)."""
    d = level.mesh.d
    D = scaling(d, U.shape[0], dtau, a0dt, level.params.T, implicit)

    def f(X):
        return D * (level.N(X, a0dt) + g)

    for _ in range(iters):
        U = timestep.rk4_step(f, U, dtau)
    return U


def bdf_forcing(Un, Unm1, dt, bdf_order, d):
    """Finest-level forcing: -(a1 V^n + a2 V^{n-1}) / dt on the velocity rows."""
    a0, a1, a2 = timestep.bdf_coeffs(bdf_order)
    g = np.zeros_like(Un)
    g[1:1 + d] = -a1 * Un[1:1 + d] / dt
    if a2 != 0.0:
        g[1:1 + d] -= a2 * Unm1[1:1 + d] / dt
    return g, a0 / dt


def level_dtau(dtau, p, q, factor):
    """Pseudo step of order q: dtau factor^(p - q), or dtau factor[q] when
    factor maps orders to multipliers."""
    return dtau * (factor[q] if isinstance(factor, dict) else factor ** (p - q))


def cycle(levels, U, g_fine, a0dt, dtau, schedule, factor, implicit=True):
    """One P-multigrid cycle.  levels: {order: Level}; schedule: list of
    (order, iterations) starting at the finest order; factor: the pseudo
    step multiplier per order below the finest (or a map order ->
    multiplier); returns the new finest-level state."""
    p = schedule[0][0]
    d = levels[p].mesh.d
    state = {p: U}
    forcing = {p: g_fine}
    start = {}
    cur = p
    for order, iters in schedule:
        if order == cur - 1:              # restrict to the coarser level
            Ir, _ = transfer_1d(cur, order)
            r = levels[cur].N(state[cur], a0dt) + forcing[cur]
            start[order] = apply_tensor(Ir, state[cur], d)
            state[order] = start[order].copy()
            forcing[order] = apply_tensor(Ir, r, d) - levels[order].N(start[order], a0dt)
        elif order == cur + 1:            # prolong the coarse correction
            _, Ip = transfer_1d(order, cur)
            state[order] = state[order] + apply_tensor(Ip, state[cur] - start[cur], d)
        elif order != cur:
            raise ValueError("consecutive cycle orders must differ by one")
        cur = order
        state[cur] = smooth(levels[cur], state[cur], forcing[cur], a0dt,
                            level_dtau(dtau, p, cur, factor), iters, implicit)
    if cur != p:
        raise ValueError("the cycle must end on the finest order")
    return state[p]


def fine_residual(level, U, g, a0dt):
    d = level.mesh.d
    return timestep.velocity_residual(level.N(U, a0dt) + g, d)


class Anderson:
    """Anderson mixing of a fixed-point iteration x <- G(x) with memory m
    (Walker & Ni, SIAM J. Numer. Anal. 49, 2011, the undamped form; not in
    the paper): with f_j = G(x_j) - x_j over the last m + 1 iterates,
    gamma = argmin || f_k - dF gamma ||_2 (dF, dG the columns of successive
    differences of f and G), x_{k+1} = G(x_k) - dG gamma; with one iterate
    in the window, x_{k+1} = G(x_k).  m = 0 is the plain iteration."""

    def __init__(self, m):
        self.m, self.G, self.F = m, [], []

    def step(self, x, gx):
        if self.m == 0:
            return gx
        self.G.append(gx.copy())
        self.F.append(gx - x)
        self.G, self.F = self.G[-(self.m + 1):], self.F[-(self.m + 1):]
        if len(self.F) == 1:
            return gx
        dF = np.stack([(self.F[i + 1] - self.F[i]).ravel() for i in range(len(self.F) - 1)], 1)
        dG = np.stack([(self.G[i + 1] - self.G[i]).ravel() for i in range(len(self.G) - 1)], 1)
        gamma = np.linalg.lstsq(dF, self.F[-1].ravel(), rcond=None)[0]
        return (self.G[-1].ravel() - dG @ gamma).reshape(x.shape)


def pseudo_solve(levels, U0, Un, Unm1, dt, bdf_order, dtau, tol, max_cycles, schedule,
                 factor=1.75, implicit=True, anderson=0):
    """Cycles until the finest velocity residual (checked at the start of
    each cycle) is below tol, optionally with Anderson mixing of memory
    `anderson` over the cycles.  Returns (U, cycles, residual, converged)."""
    p = schedule[0][0]
    d = levels[p].mesh.d
    g, a0dt = bdf_forcing(Un, Unm1, dt, bdf_order, d)
    U = np.array(U0, dtype=np.float64, copy=True)
    mix = Anderson(anderson)
    n = 0
    res = fine_residual(levels[p], U, g, a0dt)
    while res >= tol and n < max_cycles:
        U = mix.step(U, cycle(levels, U, g, a0dt, dtau, schedule, factor, implicit))
        n += 1
        res = fine_residual(levels[p], U, g, a0dt)
    return U, n, res, res < tol


def paper_schedule(p, coarsest=1, down=1, bottom=4, up=1, top=7):
    """The paper's asymmetric cycle generalised to order p: one iteration on
    the way down, `bottom` on the coarsest order, one on the way up, `top`
    on the finest: for p = 4, (4,1) (3,1) (2,1) (1,4) (2,1) (3,1) (4,7)."""
    s = [(q, down) for q in range(p, coarsest, -1)] + [(coarsest, bottom)]
    s += [(q, up) for q in range(coarsest + 1, p)] + [(p, top)]
    return s
