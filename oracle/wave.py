"""The MFWH map, its iterations and the Helmholtz checks in plain FP64 numpy
(oracle; test infrastructure only).

Grid functions are numpy arrays over all grid points, boundary included,
indexed [j_y, j_x] in 2D and [j_z, j_y, j_x] in 3D (x fastest).  A stack of
N_f grid functions has shape (N_f, *grid).  Dirichlet data are zero
(the paper's examples), so boundary values of W and V are zero throughout.
"""

import math
from dataclasses import dataclass, field

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import filters


@dataclass
class Grid:
    """Uniform Cartesian grid on [0, L_1] x ... with n_i cells per axis (listed x first)."""
    n: tuple
    length: tuple

    @property
    def dim(self):
        return len(self.n)

    @property
    def h(self):
        return tuple(L / n for L, n in zip(self.length, self.n))

    @property
    def shape(self):
        # array shape: slowest axis first, x last
        return tuple(n + 1 for n in reversed(self.n))

    def interior(self):
        return tuple(slice(1, -1) for _ in range(self.dim))

    def coords(self):
        """Coordinate arrays (x, y[, z]) broadcast to the array shape."""
        axes = [np.arange(n + 1) * h for n, h in zip(self.n, self.h)]
        mesh = np.meshgrid(*reversed(axes), indexing="ij")
        return tuple(reversed(mesh))


def laplacian(W, grid, c2, order=2):
    """L_{ph} W = c^2 Delta_h W at interior points; zero on the boundary.  c2 is a scalar or
    a grid array.

    order = 2: second-order central differences, (W_{j-1} - 2 W_j + W_{j+1}) / h^2 per axis.
    order = 4: fourth-order central differences,
        (-W_{j-2} + 16 W_{j-1} - 30 W_j + 16 W_{j+1} - W_{j+2}) / (12 h^2) per axis,
    the p = 4 case of L_{ph} (Section "Discretizing the wave equation and filter").  At the
    points next to the boundary the stencil reaches one ghost point, whose value is the odd
    reflection W_{-1} = -W_1 (and W_{N+1} = -W_{N-1}) of homogeneous Dirichlet data.
    """
    out = np.zeros_like(W)
    inner = grid.interior()
    if order == 4:
        Wp = np.pad(W, 1, mode="reflect", reflect_type="odd")   # 2 W_0 - W_1 = -W_1
        core = tuple(slice(2, -2) for _ in range(grid.dim))
    acc = np.zeros_like(W[inner])
    for axis_x, h in enumerate(grid.h):          # axis_x = 0 is x, the last array axis
        ax = grid.dim - 1 - axis_x
        if order == 4:
            def sh(k):
                sl = list(core)
                sl[ax] = slice(2 + k, Wp.shape[ax] - 2 + k)
                return Wp[tuple(sl)]
            acc += (-sh(-2) + 16.0 * sh(-1) - 30.0 * sh(0) + 16.0 * sh(1) - sh(2)) / (12.0 * h * h)
        else:
            plus = [slice(1, -1)] * grid.dim
            minus = [slice(1, -1)] * grid.dim
            plus[ax] = slice(2, None)
            minus[ax] = slice(0, -2)
            acc += (W[tuple(plus)] - 2.0 * W[inner] + W[tuple(minus)]) / (h * h)
    c2 = c2 if np.isscalar(c2) else c2[inner]
    out[inner] = c2 * acc
    return out


@dataclass
class Problem:
    grid: Grid
    forcing: np.ndarray          # (N_f, *grid.shape), f^{(m)} at the grid points
    c2: object                   # scalar or grid array of c^2
    setup: filters.Setup = field(repr=False)
    order: int = 2               # order p of L_{ph}: 2 or 4
    explicit_filter: bool = False  # filter update with the current iterate (footnote to eq. filterII)

    @property
    def nf(self):
        return self.forcing.shape[0]


def make_problem(grid, omega, forcing, c2=1.0, cfl=0.5, n_p=1,
                 filter_mode=filters.FILTER_OPTIMIZED, user_params=None,
                 n_delta=20, c_delta=2.0, order=2, explicit_filter=False,
                 time_stepping="explicit", steps_per_period=10):
    c_max = math.sqrt(float(np.max(c2)))
    setup = filters.make_setup(omega, grid.h, c_max, cfl, n_p, filter_mode,
                               user_params, n_delta, c_delta, order,
                               time_stepping, steps_per_period)
    return Problem(grid, np.asarray(forcing, dtype=np.float64), c2, setup, order, explicit_filter)


def composite_forcing(prob, n):
    """F^n = sum_m f^{(m)} cos(omega~_m t^n) (beta + 2 alpha cos(omega~_m dt))
    (eq. WaveSchemeForcing), interior only; the last factor is 1 for the explicit scheme."""
    s = prob.setup
    alpha, beta = s.scheme
    t = n * s.dt
    F = np.zeros(prob.grid.shape)
    inner = prob.grid.interior()
    for m in range(prob.nf):
        factor = beta + 2.0 * alpha * math.cos(s.omega_t[m] * s.dt)
        F[inner] += prob.forcing[m][inner] * math.cos(s.omega_t[m] * t) * factor
    return F


def apply_Pi(prob, V, forced=True):
    """One application of the MFWH map (the loop body of Algorithm 1), explicit scheme.

    W^0 = sum_m V_m; W^1 = W^0 + dt^2/2 (L_h W^0 - F^0) (eq. implicitFirstStep with
    alpha = 0, beta = 1); W^{n+1} = 2 W^n - W^{n-1} + dt^2 (L_h W^n - F^n) for
    n = 1..N_t-1 (eq. WaveSchemeA); boundary values stay 0.  The filter sums
    q_m = sum_n w_{n,m} W^n (eq. pDefQ) accumulate while stepping, and the new
    iterate solves B V^{k+1} = q at every grid point (eq. waveHoltzMatrixIteration).
    With forced=False the forcing is dropped, which gives S V (eq. discreteMFWHmapping).
    With prob.explicit_filter the update is the explicit filter of the footnote to
    eq. filterII: B_mm V_m^{k+1} = q_m - sum_{j != m} B_mj V_j^k.
    """
    if prob.setup.scheme != filters.EXPLICIT:
        return _apply_Pi_implicit(prob, V, forced)
    s = prob.setup
    g = prob.grid
    inner = g.interior()
    dt2 = s.dt * s.dt
    W0 = np.sum(V, axis=0)
    W0 = W0.copy()
    zero_boundary(W0, g)

    def F(n):
        return composite_forcing(prob, n) if forced else 0.0

    q = np.zeros((prob.nf,) + g.shape)
    for m in range(prob.nf):
        q[m] += s.w[0, m] * W0

    W1 = np.zeros_like(W0)
    W1[inner] = (W0 + 0.5 * dt2 * (laplacian(W0, g, prob.c2, prob.order) - F(0)))[inner]
    for m in range(prob.nf):
        q[m] += s.w[1, m] * W1

    W_prev, W_cur = W0, W1
    for n in range(1, s.n_t):
        W_next = np.zeros_like(W_cur)
        W_next[inner] = (2.0 * W_cur - W_prev
                         + dt2 * (laplacian(W_cur, g, prob.c2, prob.order) - F(n)))[inner]
        for m in range(prob.nf):
            q[m] += s.w[n + 1, m] * W_next
        W_prev, W_cur = W_cur, W_next

    return _filter_update(prob, q, V)


def _apply_Pi_implicit(prob, V, forced=True):
    """One application of the MFWH map with an implicit scheme (alpha > 0), eq. WaveScheme.

    With A = I - alpha dt^2 L_h on the interior unknowns (Dirichlet data zero):
      first step (eq. implicitFirstStep):
        A W^1 = W^0 + (beta/2) dt^2 L_h W^0 - (dt^2/2) F^0,
      later steps (eq. WaveSchemeA solved for W^{n+1}):
        A W^{n+1} = 2 W^n - W^{n-1} + dt^2 L_h (beta W^n + alpha W^{n-1}) - dt^2 F^n,
    for n = 1..N_t-1, with F^n of eq. WaveSchemeForcing.  Each A-solve is a sparse
    LU solve (scipy's splu of the assembled matrix), which is the definition of the
    step; the filter sums and the update are those of the explicit map.
    """
    s = prob.setup
    g = prob.grid
    inner = g.interior()
    alpha, beta = s.scheme
    dt2 = s.dt * s.dt
    L = laplacian_matrix(g, prob.c2, prob.order).tocsc()
    A = (sp.identity(L.shape[0], format="csc") - alpha * dt2 * L).tocsc()
    lu = spla.splu(A)

    def solve(rhs_grid):
        out = np.zeros(g.shape)
        out[inner] = lu.solve(rhs_grid[inner].ravel()).reshape(out[inner].shape)
        return out

    def F(n):
        return composite_forcing(prob, n) if forced else np.zeros(g.shape)

    def Lh(W):
        return laplacian(W, g, prob.c2, prob.order)

    W0 = np.sum(V, axis=0).copy()
    zero_boundary(W0, g)
    q = np.zeros((prob.nf,) + g.shape)
    for m in range(prob.nf):
        q[m] += s.w[0, m] * W0

    W1 = solve(W0 + 0.5 * beta * dt2 * Lh(W0) - 0.5 * dt2 * F(0))
    for m in range(prob.nf):
        q[m] += s.w[1, m] * W1

    W_prev, W_cur = W0, W1
    for n in range(1, s.n_t):
        W_next = solve(2.0 * W_cur - W_prev + dt2 * Lh(beta * W_cur + alpha * W_prev)
                       - dt2 * F(n))
        for m in range(prob.nf):
            q[m] += s.w[n + 1, m] * W_next
        W_prev, W_cur = W_cur, W_next
    return _filter_update(prob, q, V)


def _filter_update(prob, q, V):
    """V^{k+1} from the filter sums: B V^{k+1} = q at every grid point (eq.
    waveHoltzMatrixIteration), or the explicit filter of the footnote to eq. filterII."""
    s = prob.setup
    g = prob.grid
    flat = q.reshape(prob.nf, -1)
    if prob.explicit_filter:
        # explicit filter: B_mm V_m^{k+1} = q_m - sum_{j != m} B_mj V_j^k, the variant with
        # v^{(j,k)} in place of v^{(j,k+1)} in the sum of eq. MFWHIteration / eq. filterII
        Vk = np.asarray(V, dtype=np.float64).reshape(prob.nf, -1).copy()
        Vk[:, ~_interior_mask(g).ravel()] = 0.0
        off = s.B - np.diag(np.diag(s.B))
        V_new = ((flat - off @ Vk) / np.diag(s.B)[:, None]).reshape(q.shape)
        return V_new
    V_new = np.linalg.solve(s.B, flat).reshape(q.shape)
    return V_new


def _interior_mask(grid):
    mask = np.zeros(grid.shape, dtype=bool)
    mask[grid.interior()] = True
    return mask


def zero_boundary(W, grid):
    for ax in range(grid.dim):
        idx = [slice(None)] * grid.dim
        idx[ax] = 0
        W[tuple(idx)] = 0.0
        idx[ax] = -1
        W[tuple(idx)] = 0.0


def fixed_point_iteration(prob, V0, iters):
    """Algorithm 1: V^{k+1} = Pi(V^k); returns the iterates V^1..V^iters."""
    out = []
    V = V0
    for _ in range(iters):
        V = apply_Pi(prob, V, forced=True)
        out.append(V)
    return out


def fpi_residual(V_new, V_old, grid):
    """r^{(k)} of eq. residual: RMS over interior points and frequencies of V^k - V^{k-1}."""
    inner = (slice(None),) + grid.interior()
    d = (V_new - V_old)[inner]
    return math.sqrt(float(np.mean(d * d)))


@dataclass
class GmresInfo:
    iterations: int = 0          # Arnoldi steps (each one application of S)
    pi_applications: int = 0     # forced + homogeneous applications of Pi
    history: list = field(default_factory=list)   # relative residual after each Arnoldi step
    rel_residual: float = float("nan")
    converged: bool = False


def gmres(prob, V0=None, restart=20, tol=1e-8, max_iters=500):
    """Restarted GMRES(restart) on A_h V = b_h with A_h = I - S_h and b_h = Pi(0)
    (eq. discreteMFWHmapping, eq. krylovSystem).

    Reading: no preconditioner, modified Gram-Schmidt Arnoldi, and the stopping
    test ||b - A x||_2 / ||b||_2 < tol on the stacked vector of all N_f grid
    functions.  The small least-squares problem min ||beta e_1 - Hbar y|| is
    solved afresh with numpy's lstsq after every Arnoldi step.
    """
    info = GmresInfo()
    b = apply_Pi(prob, np.zeros_like(prob.forcing), forced=True)
    info.pi_applications += 1

    def A(x):
        info.pi_applications += 1
        return x - apply_Pi(prob, x, forced=False)

    x = np.zeros_like(b) if V0 is None else np.array(V0, dtype=np.float64)
    bnorm = float(np.linalg.norm(b))
    if bnorm == 0.0:
        info.rel_residual = 0.0
        info.converged = True
        return x, info
    while info.iterations < max_iters:
        r = b - A(x) if np.any(x) else b.copy()
        beta = float(np.linalg.norm(r))
        info.rel_residual = beta / bnorm
        if info.rel_residual < tol:
            info.converged = True
            break
        basis = [r / beta]
        Hbar = np.zeros((restart + 1, restart))
        y = np.zeros(0)
        j_done = 0
        for j in range(restart):
            w = A(basis[j])
            info.iterations += 1
            for i in range(j + 1):                       # modified Gram-Schmidt
                Hbar[i, j] = float(np.vdot(basis[i], w))
                w = w - Hbar[i, j] * basis[i]
            Hbar[j + 1, j] = float(np.linalg.norm(w))
            rhs = np.zeros(j + 2)
            rhs[0] = beta
            y = np.linalg.lstsq(Hbar[:j + 2, :j + 1], rhs, rcond=None)[0]
            res = float(np.linalg.norm(rhs - Hbar[:j + 2, :j + 1] @ y))
            info.history.append(res / bnorm)
            j_done = j + 1
            if res / bnorm < tol or info.iterations >= max_iters or Hbar[j + 1, j] == 0.0:
                break
            basis.append(w / Hbar[j + 1, j])
        for i in range(j_done):
            x = x + y[i] * basis[i]
        info.rel_residual = info.history[-1]
        if info.rel_residual < tol:
            info.converged = True
            break
    return x, info


def helmholtz_residual(prob, V):
    """r_h^{(m)} = max_int |f_m - (L_h + omega_m^2) V_m| / max_int |f_m| (eq. errorAndResid).

    Reading: the paper prints L_{p,h} - omega_m^2 I inside the norm; the
    Helmholtz equation it solves is L u + omega^2 u = f, so the residual is
    taken with + omega_m^2.
    """
    inner = prob.grid.interior()
    out = np.zeros(prob.nf)
    for m in range(prob.nf):
        Hv = laplacian(V[m], prob.grid, prob.c2, prob.order) + prob.setup.omega[m] ** 2 * V[m]
        num = np.max(np.abs(prob.forcing[m][inner] - Hv[inner]))
        den = np.max(np.abs(prob.forcing[m][inner]))
        out[m] = num / den
    return out


# ---------------------------------------------------------------------------
# References used by the pins: sparse direct solve and the Dirichlet spectrum
# ---------------------------------------------------------------------------

def laplacian_matrix(grid, c2, order=2):
    """Sparse L_{ph} on interior unknowns (x fastest), Dirichlet zero boundary; for order 4
    the ghost value -W_1 folds into the first and last rows (-W_{-1} = +W_1)."""
    mats = []
    for n, h in zip(grid.n, grid.h):
        k = n - 1
        if order == 4:
            main = -30.0 * np.ones(k)
            main[0] += 1.0
            main[-1] += 1.0
            off1 = 16.0 * np.ones(k - 1)
            off2 = -np.ones(max(k - 2, 0))
            diags = [off2, off1, main, off1, off2] if k > 2 else [off1, main, off1]
            offs = [-2, -1, 0, 1, 2] if k > 2 else [-1, 0, 1]
            if k == 1:
                diags, offs = [main], [0]
            mats.append(sp.diags(diags, offs, shape=(k, k)) / (12.0 * h * h))
            continue
        main = -2.0 * np.ones(k)
        off = np.ones(k - 1)
        mats.append(sp.diags([off, main, off], [-1, 0, 1], shape=(k, k)) / (h * h))
    eyes = [sp.identity(n - 1) for n in grid.n]
    L = None
    for a in range(grid.dim):
        # Kronecker order: slowest axis (last in grid.n) first, x last
        factors = [mats[b] if b == a else eyes[b] for b in reversed(range(grid.dim))]
        term = factors[0]
        for fct in factors[1:]:
            term = sp.kron(term, fct)
        L = term if L is None else L + term
    c2v = c2 if np.isscalar(c2) else c2[grid.interior()].ravel()
    return sp.diags(np.broadcast_to(c2v, (L.shape[0],)).astype(np.float64)) @ L


def helmholtz_direct(prob):
    """U_m solving L_h U + omega_m^2 U = f_m at interior points (eq. discreteHelmholtz), U = 0 on the boundary."""
    L = laplacian_matrix(prob.grid, prob.c2, prob.order).tocsc()
    inner = prob.grid.interior()
    I = sp.identity(L.shape[0], format="csc")
    U = np.zeros_like(prob.forcing)
    for m in range(prob.nf):
        rhs = prob.forcing[m][inner].ravel()
        sol = spla.spsolve(L + prob.setup.omega[m] ** 2 * I, rhs)
        U[m][inner] = sol.reshape(U[m][inner].shape)
    return U


def dirichlet_mode(grid, k, order=2):
    """Discrete Dirichlet eigenfunction prod_i sin(k_i pi x_i / L_i) and its eigenvalue
    lambda^2 of -Delta_h (k listed x first): sum_i (4/h_i^2) sin^2(theta_i/2) for order 2 and
    sum_i (30 - 32 cos theta_i + 2 cos 2 theta_i) / (12 h_i^2) for order 4, theta_i = k_i pi / n_i
    (the sine modes satisfy the odd-reflection ghost values exactly)."""
    xs = grid.coords()
    phi = np.ones(grid.shape)
    lam2 = 0.0
    for x, kk, L, n, h in zip(xs, k, grid.length, grid.n, grid.h):
        phi = phi * np.sin(kk * math.pi * x / L)
        th = kk * math.pi / n
        if order == 4:
            lam2 += (30.0 - 32.0 * math.cos(th) + 2.0 * math.cos(2.0 * th)) / (12.0 * h * h)
        else:
            lam2 += 4.0 / (h * h) * math.sin(th / 2.0) ** 2
    zero_boundary(phi, grid)
    return phi, lam2
