"""MFWH set-up arithmetic in plain FP64 numpy (oracle; test infrastructure only).

Follows the paper's Sections "Governing equations", "Filter parameters from an
optimization problem" and "Discretizing the wave equation and filter".
Where the paper is silent the reading used is stated in the docstring.
"""

import math
from dataclasses import dataclass
from fractions import Fraction

import numpy as np

# ---------------------------------------------------------------------------
# Time discretisation
# ---------------------------------------------------------------------------

EXPLICIT = (0.0, 1.0)      # (alpha, beta) of eq. WaveSchemeA: leapfrog
TRAPEZOIDAL = (0.5, 0.0)   # (alpha, beta): implicit trapezoidal scheme


def adjusted_frequency(omega, dt, scheme=EXPLICIT):
    """eq. omegaImplicit: omega~ = acos((1 - (beta/2)(omega dt)^2) / (1 + alpha (omega dt)^2)) / dt."""
    alpha, beta = scheme
    x = np.asarray(omega, dtype=np.float64) * dt
    return np.arccos((1.0 - 0.5 * beta * x * x) / (1.0 + alpha * x * x)) / dt


def explicit_time_step(h, c_max, cfl, omega1, n_p, order=2):
    """Explicit time step and step count (Section "Time-step determination").

    Reading: the von Neumann limit of leapfrog with the second-order Laplacian
    is dt_stab = 1 / (c_max sqrt(sum_i 1/h_i^2)).  N_t is the smallest step
    count whose step fits under cfl*dt_stab over T_f = N_p 2 pi/omega_1, and dt
    is then chosen so that omega~_1 dt = 2 pi N_p / N_t exactly, which makes
    the adjusted final time N_p 2 pi / omega~_1 equal to N_t dt.  With the
    explicit omega~ that condition reads 1 - (omega_1 dt)^2/2 = cos(2 pi N_p/N_t),
    i.e. dt = 2 sin(pi N_p / N_t) / omega_1.

    For the fourth-order operator L_{4h} (order = 4) the spectral radius of -L_h is
    c_max^2 sum_i (16/3)/h_i^2 instead of c_max^2 sum_i 4/h_i^2, and leapfrog needs
    dt^2 rho(-L_h) <= 4, so dt_stab is smaller by the factor sqrt(3)/2.
    """
    h = np.atleast_1d(np.asarray(h, dtype=np.float64))
    dt_stab = 1.0 / (c_max * math.sqrt(float(np.sum(1.0 / (h * h)))))
    if order == 4:
        dt_stab *= math.sqrt(3.0) / 2.0
    t_final = n_p * 2.0 * math.pi / omega1
    n_t = max(2 * n_p + 1, int(math.ceil(t_final / (cfl * dt_stab))))
    dt = 2.0 * math.sin(math.pi * n_p / n_t) / omega1
    return dt, n_t


def implicit_time_step(omega1, omega_max, n_p, steps_per_period=10, scheme=TRAPEZOIDAL):
    """Implicit step count and step (Section "Time-step determination").

    Reading: N_t = ceil(steps_per_period * N_p * omega_Nf / omega_1) steps (10 per
    shortest period over N_p longest periods); dt solves omega~_1 dt = theta with
    theta = 2 pi N_p / N_t, i.e. (omega_1 dt)^2 = (1 - cos theta) / (beta/2 + alpha cos theta),
    so that the adjusted final time N_p 2 pi / omega~_1 is N_t dt.
    """
    alpha, beta = scheme
    n_t = int(math.ceil(steps_per_period * n_p * omega_max / omega1 - 1e-12))
    theta = 2.0 * math.pi * n_p / n_t
    x2 = (1.0 - math.cos(theta)) / (0.5 * beta + alpha * math.cos(theta))
    return math.sqrt(x2) / omega1, n_t


def period_counts(omega, n_p):
    """eq. TbarDef with periods T_m = 2 pi / omega_m.

    T_f = N_p T_1, N_{p,m} = floor(T_f / T_m) and T_{f,m} = N_{p,m} T_m.  The floor
    of T_f / T_m = N_p omega_m / omega_1 is taken in exact rational arithmetic on the
    given floating-point frequencies, so N_{p,1} = N_p and no count is lost when a
    ratio lies within rounding of an integer.
    """
    omega = np.asarray(omega, dtype=np.float64)
    w1 = Fraction(float(omega[0]))
    n_pm = np.array([math.floor(int(n_p) * Fraction(float(w)) / w1) for w in omega],
                    dtype=np.int64)
    t_fm = n_pm * (2.0 * math.pi / omega)
    t_f = n_p * 2.0 * math.pi / omega[0]
    return n_pm, t_fm, t_f


def trapezoid_weights(n_t, dt, t_fm):
    """Quadrature weights sigma_{n,m}, n = 0..N_t (eq. DefNI and the text after it).

    Composite trapezoid rule on [0, t_k], where t_k = k dt is the last grid time
    not beyond T_{f,m}; on the partial interval [t_k, T_{f,m}] the integrand is
    replaced by the straight line through (t_k, zeta_k), (t_{k+1}, zeta_{k+1}) and
    integrated exactly.  With r = T_{f,m}/dt - k in [0, 1) that line contributes
    dt (r - r^2/2) to sigma_k and dt r^2/2 to sigma_{k+1}; all later weights are 0.
    """
    t_fm = np.atleast_1d(np.asarray(t_fm, dtype=np.float64))
    sigma = np.zeros((n_t + 1, t_fm.size))
    for m, tm in enumerate(t_fm):
        k = int(math.floor(tm / dt))
        k = min(k, n_t)
        r = tm / dt - k
        for n in range(k + 1):                    # trapezoid on [0, t_k]
            sigma[n, m] = dt if 0 < n < k else 0.5 * dt
        if k == 0:
            sigma[0, m] = 0.0
        if k < n_t:                               # partial panel [t_k, T_{f,m}]
            sigma[k, m] += dt * (r - 0.5 * r * r)
            sigma[k + 1, m] += 0.5 * dt * r * r
    return sigma


# ---------------------------------------------------------------------------
# Filter kernel, traditional and least-squares parameters
# ---------------------------------------------------------------------------

def filter_kernel(tau, p):
    """eq. newFilterKernel: K(tau; a, c, s) = a + c cos(tau) + s sin(tau)."""
    a, c, s = p
    return a + c * np.cos(tau) + s * np.sin(tau)


def traditional_parameters(omega_t, dt):
    """eq. origParamAdjust: p_m = (a_m, 1, 0), a_m = -tan(omega~ dt/2) / (2 tan(omega~ dt))."""
    omega_t = np.asarray(omega_t, dtype=np.float64)
    a = -np.tan(0.5 * omega_t * dt) / (2.0 * np.tan(omega_t * dt))
    return np.stack([a, np.ones_like(a), np.zeros_like(a)], axis=1)


@dataclass
class OptResult:
    params: np.ndarray      # (N_f, 3): (a~_m, c~_m, s~_m)
    lam_max: float          # right end of Lambda (eq. LambdaRange)
    n_lambda: int           # number of midpoint quadrature points
    t_f: float              # N_p T_1
    n_pm: np.ndarray        # N_{p,m}
    cond_M: float = float("nan")   # 2-norm condition number of the least-squares matrix M


class _QuadratureBasis:
    """Component functions f_a, f_c, f_s of eq. compFuncs and their lambda-derivatives,
    each evaluated as (2/T_{f,m}) sum_i nu_{i,m} g(t_i) for a time rule (t_i, nu_{i,m}).

    The rule is either the trapezoid weights on the wave-solve time grid (the
    discrete form used for the computations, eq. betadDefA) or a Gauss-Legendre
    rule on [0, T_{f,m}] (the continuous integrals of eq. compFuncs).
    """

    def __init__(self, omega, t_fm, nodes, weights):
        self.omega = omega
        self.t_fm = t_fm
        self.nodes = nodes        # list per m of time nodes
        self.weights = weights    # list per m of weights

    def _eval(self, lam, m, kind, deriv):
        t = self.nodes[m]
        wt = self.weights[m] * (2.0 / self.t_fm[m])
        lam = np.atleast_1d(np.asarray(lam, dtype=np.float64))
        arg = np.outer(lam, t)
        base = {"a": np.ones_like(t),
                "c": np.cos(self.omega[m] * t),
                "s": np.sin(self.omega[m] * t)}[kind]
        if deriv:   # d/dlambda cos(lambda t) = -t sin(lambda t)
            return (-np.sin(arg) * t) @ (wt * base)
        return np.cos(arg) @ (wt * base)

    def f(self, kind, lam, m):
        return self._eval(lam, m, kind, False)

    def fp(self, kind, lam, m):
        return self._eval(lam, m, kind, True)


def _optimise(basis, omega, n_pm, n_delta, c_delta):
    """Algorithm 2 (optParameters) given a way to evaluate the component functions.

    Step order follows the algorithm: constraint matrices F_k, F'_k (eq.
    constraintsVec), G, H, z (eq. yt), the interval Lambda (eq. LambdaRange),
    midpoint points lambda_k, g_a and mu_0 (eq. muNice), the least-squares
    system M x_a = m_0, then y = G^{-1}(z - H x_a) (eq. yOpt).
    """
    nf = omega.size
    fk = {k: np.zeros((nf, nf)) for k in "acs"}
    fpk = {k: np.zeros((nf, nf)) for k in "acs"}
    for k in "acs":
        for j in range(nf):                       # column j: filter j
            fk[k][:, j] = basis.f(k, omega, j)    # row m: evaluated at omega_m
            fpk[k][:, j] = basis.fp(k, omega, j)
    G = np.block([[fk["c"], fk["s"]], [fpk["c"], fpk["s"]]])
    H = np.vstack([fk["a"], fpk["a"]])
    z = np.concatenate([np.ones(nf), np.zeros(nf)])

    delta_nf = omega[-1] / (2.0 * n_pm[-1])
    lam_max = omega[-1] + c_delta * nf * delta_nf
    n_lambda = int(math.ceil(n_delta * lam_max / delta_nf - 1e-9))
    lam = (np.arange(1, n_lambda + 1) - 0.5) * lam_max / n_lambda

    fa = np.stack([basis.f("a", lam, j) for j in range(nf)], axis=1)    # (N_lambda, N_f)
    fcs = np.hstack([np.stack([basis.f("c", lam, j) for j in range(nf)], axis=1),
                     np.stack([basis.f("s", lam, j) for j in range(nf)], axis=1)])
    ginv_h = np.linalg.solve(G, H)
    ginv_z = np.linalg.solve(G, z)
    M = fa - fcs @ ginv_h                # rows g_a(lambda_k)^T
    m0 = -(fcs @ ginv_z)                 # -mu_0(lambda_k)
    x_a = np.linalg.lstsq(M, m0, rcond=None)[0]
    y = np.linalg.solve(G, z - H @ x_a)
    params = np.stack([x_a, y[:nf], y[nf:]], axis=1)
    return params, lam_max, n_lambda, float(np.linalg.cond(M))


def opt_parameters_discrete(omega, n_p, n_t, n_delta=20, c_delta=2.0):
    """Least-squares filter parameters with the wave-solve quadrature (Algorithm 2,
    discrete form as used for the paper's computations, Appendix A).

    Inputs are the (adjusted) frequencies, N_p and N_t.  T_{f,m} follows eq.
    TbarDef, dt = max_m T_{f,m} / N_t, and the component functions are the
    trapezoid-rule sums of eq. betadDefA with cos(lambda t) or its derivative.
    """
    omega = np.asarray(omega, dtype=np.float64)
    n_pm, t_fm, _ = period_counts(omega, n_p)
    t_f = float(np.max(t_fm))
    dt = t_f / n_t
    sigma = trapezoid_weights(n_t, dt, t_fm)
    t = np.arange(n_t + 1) * dt
    basis = _QuadratureBasis(omega, t_fm, [t] * omega.size,
                             [sigma[:, m] for m in range(omega.size)])
    params, lam_max, n_lambda, cond_m = _optimise(basis, omega, n_pm, n_delta, c_delta)
    return OptResult(params, lam_max, n_lambda, t_f, n_pm, cond_m)


def opt_parameters_continuous(omega, n_p, n_delta=20, c_delta=2.0, n_gauss=512):
    """Least-squares filter parameters with the exact time integrals (Algorithm 2).

    The integrals of eq. compFuncs over [0, T_{f,m}] are evaluated with an
    n_gauss-point Gauss-Legendre rule, which is exact to rounding for the
    smooth, few-period integrands involved.
    """
    omega = np.asarray(omega, dtype=np.float64)
    n_pm, t_fm, t_f = period_counts(omega, n_p)
    x, wx = np.polynomial.legendre.leggauss(n_gauss)
    nodes = [0.5 * tm * (x + 1.0) for tm in t_fm]
    weights = [0.5 * tm * wx for tm in t_fm]
    basis = _QuadratureBasis(omega, t_fm, nodes, weights)
    params, lam_max, n_lambda, cond_m = _optimise(basis, omega, n_pm, n_delta, c_delta)
    return OptResult(params, lam_max, n_lambda, t_f, n_pm, cond_m)


# ---------------------------------------------------------------------------
# Discrete filter weights and B
# ---------------------------------------------------------------------------

def filter_weights(omega_t, dt, n_t, sigma, t_fm, params):
    """w_{n,m} = (2 / T~_{f,m}) sigma_{n,m} K(omega~_m t^n; p_m), t^n = n dt (eq. pDefQ)."""
    t = np.arange(n_t + 1) * dt
    w = np.zeros((n_t + 1, len(omega_t)))
    for m, om in enumerate(omega_t):
        w[:, m] = (2.0 / t_fm[m]) * sigma[:, m] * filter_kernel(om * t, params[m])
    return w


def filter_matrix(w, omega_t, dt):
    """Discrete B_omega (eq. filterA with eq. betadDefA): B_{mj} = sum_n w_{n,m} cos(omega~_j t^n).

    Reading: the discrete filter functions are evaluated at the adjusted
    frequencies omega~_j, the frequencies the composite forcing oscillates at in
    eq. WaveSchemeForcing; with this B the discrete Helmholtz solution is an
    exact fixed point of the discrete map.
    """
    n_t = w.shape[0] - 1
    t = np.arange(n_t + 1) * dt
    cos_tab = np.cos(np.outer(t, omega_t))         # (N_t+1, N_f): cos(omega~_j t^n)
    return w.T @ cos_tab


def discrete_beta(w, lam_tilde, dt):
    """beta_{d,m}(lambda) = sum_n w_{n,m} cos(lambda t^n) for each m (eq. betadDefA); shape (..., N_f)."""
    n_t = w.shape[0] - 1
    t = np.arange(n_t + 1) * dt
    lam_tilde = np.atleast_1d(np.asarray(lam_tilde, dtype=np.float64))
    return np.cos(np.outer(lam_tilde, t)) @ w


def mu_discrete(B, w, lam_tilde, dt):
    """mu_d(lambda) = sum_m gamma_m beta_{d,m}(lambda), gamma_m = column sums of B^{-1} (eq. MFWHmud)."""
    gamma = np.linalg.inv(B).sum(axis=0)
    return discrete_beta(w, lam_tilde, dt) @ gamma


# ---------------------------------------------------------------------------
# Complete set-up for a problem
# ---------------------------------------------------------------------------

FILTER_OPTIMIZED = "optimized"
FILTER_TRADITIONAL = "traditional"
FILTER_USER = "user"


@dataclass
class Setup:
    dt: float
    n_t: int
    omega: np.ndarray        # requested omega_m
    omega_t: np.ndarray      # adjusted omega~_m
    n_pm: np.ndarray
    t_fm: np.ndarray         # T~_{f,m}
    sigma: np.ndarray        # (N_t+1, N_f)
    params: np.ndarray       # (N_f, 3)
    w: np.ndarray            # (N_t+1, N_f) filter weights
    B: np.ndarray            # (N_f, N_f)
    cond_M: float = float("nan")   # conditioning of Algorithm 2's least-squares matrix (optimised mode)
    scheme: tuple = EXPLICIT       # (alpha, beta) of eq. WaveSchemeA


def make_setup(omega, h, c_max, cfl=0.5, n_p=1, filter_mode=FILTER_OPTIMIZED,
               user_params=None, n_delta=20, c_delta=2.0, order=2,
               time_stepping="explicit", steps_per_period=10):
    """Set-up of Algorithm 1 (its first two lines).

    Explicit scheme (alpha, beta) = (0, 1): time step per explicit_time_step.
    Implicit trapezoidal scheme (alpha, beta) = (1/2, 0) (time_stepping =
    "implicit"): time step per implicit_time_step with steps_per_period steps over
    the shortest period.  Then omega~ per eq. omegaImplicit with the scheme's
    (alpha, beta); N_{p,m} and T~_{f,m} per eq. TbarDef using omega~; sigma per
    eq. DefNI; parameters optimised (Algorithm 2 in its discrete form with inputs
    omega~, N_p, N_t, no further adjustment) or traditional (eq. origParamAdjust)
    or given; then w and B.
    """
    omega = np.asarray(omega, dtype=np.float64)
    if time_stepping == "implicit":
        scheme = TRAPEZOIDAL
        dt, n_t = implicit_time_step(float(omega[0]), float(omega[-1]), n_p,
                                     steps_per_period, scheme)
    elif time_stepping == "explicit":
        scheme = EXPLICIT
        dt, n_t = explicit_time_step(h, c_max, cfl, float(omega[0]), n_p, order)
    else:
        raise ValueError("time_stepping must be 'explicit' or 'implicit'")
    omega_t = adjusted_frequency(omega, dt, scheme)
    n_pm, t_fm, _ = period_counts(omega_t, n_p)
    sigma = trapezoid_weights(n_t, dt, t_fm)
    cond_m = float("nan")
    if filter_mode == FILTER_OPTIMIZED:
        opt = opt_parameters_discrete(omega_t, n_p, n_t, n_delta, c_delta)
        params, cond_m = opt.params, opt.cond_M
    elif filter_mode == FILTER_TRADITIONAL:
        params = traditional_parameters(omega_t, dt)
    else:
        params = np.asarray(user_params, dtype=np.float64).reshape(omega.size, 3)
    w = filter_weights(omega_t, dt, n_t, sigma, t_fm, params)
    B = filter_matrix(w, omega_t, dt)
    return Setup(dt, n_t, omega, omega_t, n_pm, t_fm, sigma, params, w, B, cond_m, scheme)
