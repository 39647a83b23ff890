"""Plausible mistakes planted in the oracle, one at a time (test infrastructure).

Each mutant rewrites one line of one oracle function, as a slip in transcribing the paper
would: a dropped factor, a wrong sign, a shifted index, a transposed operand, an unadjusted
frequency.  tests/test_oracle_mutants.py runs the oracle's pins once per mutant, in a fresh
process where conftest.py applies it (environment variable MFWH_ORACLE_MUTANT), and requires
a pin to fail: the pins, not the oracle's agreement with the library, catch each mistake.
Nothing here is imported by the library or by the oracle.
"""

import inspect
import textwrap

# name: (module, function or Class.method, text to replace, replacement, what it corrupts)
MUTANTS = {
    # --- the wave solve and filter sums (oracle/wave.py) --------------------------------------
    "forcing_sign": (
        "oracle.wave", "composite_forcing",
        "F[inner] += prob.forcing[m][inner]", "F[inner] -= prob.forcing[m][inner]",
        "sign of F^n, eq. WaveSchemeForcing"),
    "forcing_time_shift": (
        "oracle.wave", "composite_forcing", "t = n * s.dt", "t = (n + 1) * s.dt",
        "forcing at t^{n+1} instead of t^n, eq. WaveSchemeA"),
    "forcing_unadjusted_omega": (
        "oracle.wave", "composite_forcing", "math.cos(s.omega_t[m] * t)", "math.cos(s.omega[m] * t)",
        "omega instead of omega~ in the forcing, eq. WaveSchemeForcing"),
    "first_step_without_half": (
        "oracle.wave", "apply_Pi", "W1[inner] = (W0 + 0.5 * dt2 *", "W1[inner] = (W0 + dt2 *",
        "factor 1/2 of the first step, eq. implicitFirstStep"),
    "step_forcing_sign": (
        "oracle.wave", "apply_Pi", "- F(n)))[inner]", "+ F(n)))[inner]",
        "sign of F^n in the later steps, eq. WaveSchemeA"),
    "filter_weight_index": (
        "oracle.wave", "apply_Pi", "q[m] += s.w[n + 1, m] * W_next", "q[m] += s.w[n, m] * W_next",
        "weight w_{n+1} of W^{n+1} in q_m, eq. pDefQ"),
    "filter_weight_of_w0": (
        "oracle.wave", "apply_Pi", "q[m] += s.w[0, m] * W0", "q[m] += s.w[1, m] * W0",
        "weight w_0 of W^0 in q_m, eq. pDefQ"),
    "filter_solve_transposed": (
        "oracle.wave", "_filter_update", "np.linalg.solve(s.B, flat)", "np.linalg.solve(s.B.T, flat)",
        "B V = q solved with B^T, eq. waveHoltzMatrixIteration"),
    "explicit_filter_transposed": (
        "oracle.wave", "_filter_update", "off = s.B - np.diag(np.diag(s.B))",
        "off = s.B.T - np.diag(np.diag(s.B))", "off-diagonal B_mj of the explicit filter, "
        "footnote to eq. filterII"),
    "laplacian_one_spacing": (
        "oracle.wave", "laplacian", "acc += (W[tuple(plus)] - 2.0 * W[inner] + W[tuple(minus)]) / (h * h)",
        "acc += (W[tuple(plus)] - 2.0 * W[inner] + W[tuple(minus)]) / (grid.h[0] * grid.h[0])",
        "h_x used for every axis in Delta_h"),
    "laplacian_c_not_squared": (
        "oracle.wave", "laplacian", "out[inner] = c2 * acc", "out[inner] = np.sqrt(c2) * acc",
        "c instead of c^2 in L = c^2 Delta"),
    "laplacian4_centre": (
        "oracle.wave", "laplacian", "- 30.0 * sh(0)", "- 32.0 * sh(0)",
        "centre weight of the fourth-order stencil"),
    "laplacian4_even_ghost": (
        "oracle.wave", "laplacian", 'reflect_type="odd"', 'reflect_type="even"',
        "odd reflection of the Dirichlet ghost values, fourth order"),
    "implicit_lagged_level": (
        "oracle.wave", "_apply_Pi_implicit", "Lh(beta * W_cur + alpha * W_prev)",
        "Lh(beta * W_cur + alpha * W_cur)", "alpha L_h W^{n-1} term of eq. WaveSchemeA"),
    "residual_sign": (
        "oracle.wave", "helmholtz_residual", "+ prob.setup.omega[m] ** 2 * V[m]",
        "- prob.setup.omega[m] ** 2 * V[m]", "sign of omega^2, eq. errorAndResid"),
    "residual_unnormalised": (
        "oracle.wave", "helmholtz_residual", "den = np.max(np.abs(prob.forcing[m][inner]))",
        "den = 1.0", "normalisation by max|f_m|, eq. errorAndResid"),
    "gmres_projection_index": (
        "oracle.wave", "gmres", "w = w - Hbar[i, j] * basis[i]", "w = w - Hbar[i, j] * basis[j]",
        "Gram-Schmidt against basis vector i"),
    "gmres_update_index": (
        "oracle.wave", "gmres", "x = x + y[i] * basis[i]", "x = x + y[i] * basis[0]",
        "solution update x + V y"),
    "implicit_first_step_forcing_half": (
        "oracle.wave", "_apply_Pi_implicit", "- 0.5 * dt2 * F(0))", "- dt2 * F(0))",
        "factor 1/2 of F^0 in the implicit first step, eq. implicitFirstStep"),
    "implicit_forcing_factor_half": (
        "oracle.wave", "composite_forcing", "factor = beta + 2.0 * alpha * math.cos",
        "factor = beta + alpha * math.cos", "factor beta + 2 alpha cos(omega~ dt), "
        "eq. WaveSchemeForcing"),
    "direct_solve_sign": (
        "oracle.wave", "helmholtz_direct", "spla.spsolve(L + prob.setup.omega[m] ** 2 * I, rhs)",
        "spla.spsolve(L - prob.setup.omega[m] ** 2 * I, rhs)",
        "the direct reference solves L_h U + omega^2 U = f, eq. discreteHelmholtz"),
    "gmres_restart_residual_sign": (
        "oracle.wave", "gmres", "r = b - A(x) if np.any(x) else b.copy()",
        "r = b + A(x) if np.any(x) else b.copy()", "restart residual b - A x"),
    "gmres_initial_guess_ignored": (
        "oracle.wave", "gmres", "x = np.zeros_like(b) if V0 is None else np.array(V0, dtype=np.float64)",
        "x = np.zeros_like(b)", "GMRES from the given initial guess"),
    "fpi_residual_max_norm": (
        "oracle.wave", "fpi_residual", "return math.sqrt(float(np.mean(d * d)))",
        "return float(np.max(np.abs(d)))", "root mean square of V^k - V^{k-1}, eq. residual"),
    "fpi_restarts_from_initial": (
        "oracle.wave", "fixed_point_iteration", "V = apply_Pi(prob, V, forced=True)",
        "V = apply_Pi(prob, V0, forced=True)", "V^{k+1} = Pi(V^k), Algorithm 1"),
    "boundary_second_last_line": (
        "oracle.wave", "zero_boundary", "idx[ax] = -1", "idx[ax] = -2",
        "Dirichlet data on the last grid line"),
    "laplacian_matrix4_ghost_sign": (
        "oracle.wave", "laplacian_matrix", "main[0] += 1.0", "main[0] -= 1.0",
        "odd-reflection ghost value folded into the first row, fourth order"),
    "explicit_filter_no_diagonal_solve": (
        "oracle.wave", "_filter_update", "((flat - off @ Vk) / np.diag(s.B)[:, None])",
        "(flat - off @ Vk)", "division by B_mm in the explicit filter, footnote to eq. filterII"),
    # --- set-up (oracle/filters.py) -----------------------------------------------------------
    "adjusted_frequency_factor": (
        "oracle.filters", "adjusted_frequency", "(1.0 - 0.5 * beta * x * x)", "(1.0 - beta * x * x)",
        "factor beta/2 of eq. omegaImplicit"),
    "time_step_without_sqrt_d": (
        "oracle.filters", "explicit_time_step", "math.sqrt(float(np.sum(1.0 / (h * h))))",
        "math.sqrt(float(np.max(1.0 / (h * h))))", "von Neumann limit summed over the axes"),
    "time_step_unadjusted": (
        "oracle.filters", "explicit_time_step", "dt = 2.0 * math.sin(math.pi * n_p / n_t) / omega1",
        "dt = 2.0 * math.pi * n_p / n_t / omega1", "dt that makes omega~_1 N_t dt = 2 pi N_p"),
    "implicit_time_step_factor": (
        "oracle.filters", "implicit_time_step", "(0.5 * beta + alpha * math.cos(theta))",
        "(0.5 * beta + alpha)", "implicit dt from omega~_1 dt = theta"),
    "period_count_ceil": (
        "oracle.filters", "period_counts", "math.floor(int(n_p)", "math.ceil(int(n_p)",
        "floor in N_{p,m}, eq. TbarDef"),
    "trapezoid_interior_end": (
        "oracle.filters", "trapezoid_weights", "sigma[n, m] = dt if 0 < n < k else 0.5 * dt",
        "sigma[n, m] = dt if 0 < n <= k else 0.5 * dt", "half weight at t_k, eq. DefNI"),
    "trapezoid_partial_panel": (
        "oracle.filters", "trapezoid_weights", "sigma[k + 1, m] += 0.5 * dt * r * r",
        "sigma[k + 1, m] += dt * r * r", "partial panel [t_k, T_{f,m}], eq. DefNI"),
    "kernel_sine_sign": (
        "oracle.filters", "filter_kernel", "a + c * np.cos(tau) + s * np.sin(tau)",
        "a + c * np.cos(tau) - s * np.sin(tau)", "sign of the sine term, eq. newFilterKernel"),
    "traditional_factor": (
        "oracle.filters", "traditional_parameters", "(2.0 * np.tan(omega_t * dt))",
        "(np.tan(omega_t * dt))", "factor 2 of eq. origParamAdjust"),
    "weights_scale": (
        "oracle.filters", "filter_weights", "(2.0 / t_fm[m])", "(1.0 / t_fm[m])",
        "factor 2 / T~_{f,m} of eq. pDefQ"),
    "filter_matrix_transposed": (
        "oracle.filters", "filter_matrix", "return w.T @ cos_tab", "return cos_tab.T @ w",
        "B_{mj} with m and j exchanged, eq. filterA"),
    "lambda_range": (
        "oracle.filters", "_optimise", "lam_max = omega[-1] + c_delta * nf * delta_nf",
        "lam_max = omega[-1] + c_delta * delta_nf", "right end of Lambda, eq. LambdaRange"),
    "lambda_spacing": (
        "oracle.filters", "_optimise", "delta_nf = omega[-1] / (2.0 * n_pm[-1])",
        "delta_nf = omega[-1] / n_pm[-1]", "Delta_{N_f} of eq. LambdaRange"),
    "lambda_nodes_not_midpoints": (
        "oracle.filters", "_optimise", "(np.arange(1, n_lambda + 1) - 0.5)",
        "np.arange(1, n_lambda + 1)", "midpoint nodes lambda_k of Algorithm 2"),
    "parameters_c_s_exchanged": (
        "oracle.filters", "_optimise", "params = np.stack([x_a, y[:nf], y[nf:]], axis=1)",
        "params = np.stack([x_a, y[nf:], y[:nf]], axis=1)", "order (a, c, s) of y, eq. yOpt"),
    "derivative_sign": (
        "oracle.filters", "_QuadratureBasis._eval", "return (-np.sin(arg) * t) @ (wt * base)",
        "return (np.sin(arg) * t) @ (wt * base)", "d/dlambda cos(lambda t), eq. constraintsVec"),
    "mu_row_sums": (
        "oracle.filters", "mu_discrete", "np.linalg.inv(B).sum(axis=0)",
        "np.linalg.inv(B).sum(axis=1)", "gamma_m as column sums of B^{-1}, eq. MFWHmud"),
    "period_lengths_of_first_frequency": (
        "oracle.filters", "period_counts", "t_fm = n_pm * (2.0 * math.pi / omega)",
        "t_fm = n_pm * (2.0 * math.pi / omega[0])", "T~_{f,m} = N_{p,m} 2 pi / omega~_m, "
        "eq. TbarDef"),
    "weights_time_shift": (
        "oracle.filters", "filter_weights", "t = np.arange(n_t + 1) * dt",
        "t = np.arange(1, n_t + 2) * dt", "kernel evaluated at t^n, eq. pDefQ"),
    "beta_sine": (
        "oracle.filters", "discrete_beta", "np.cos(np.outer(lam_tilde, t)) @ w",
        "np.sin(np.outer(lam_tilde, t)) @ w", "cos(lambda t^n) in beta_d, eq. betadDefA"),
    "trapezoid_first_weight": (
        "oracle.filters", "trapezoid_weights", "if k == 0:\n            sigma[0, m] = 0.0",
        "if k == 0:\n            sigma[0, m] = 0.5 * dt", "no full panel when T_{f,m} < dt"),
    "setup_optimises_unadjusted_omega": (
        "oracle.filters", "make_setup", "opt = opt_parameters_discrete(omega_t, n_p, n_t",
        "opt = opt_parameters_discrete(omega, n_p, n_t", "Algorithm 2 with inputs omega~"),
    "step_count_floor": (
        "oracle.filters", "explicit_time_step",
        "int(math.ceil(t_final / (cfl * dt_stab)))", "int(math.floor(t_final / (cfl * dt_stab)))",
        "smallest N_t whose step fits under the CFL limit"),
    "gauss_nodes_unscaled": (
        "oracle.filters", "opt_parameters_continuous", "nodes = [0.5 * tm * (x + 1.0) for tm in t_fm]",
        "nodes = [tm * (x + 1.0) for tm in t_fm]", "Gauss-Legendre nodes mapped to [0, T_{f,m}]"),
    "component_scale": (
        "oracle.filters", "_QuadratureBasis._eval", "wt = self.weights[m] * (2.0 / self.t_fm[m])",
        "wt = self.weights[m] * (1.0 / self.t_fm[m])", "factor 2 / T_{f,m} of eq. compFuncs"),
    "discrete_basis_first_weights": (
        "oracle.filters", "opt_parameters_discrete", "[sigma[:, m] for m in range(omega.size)]",
        "[sigma[:, 0] for m in range(omega.size)]", "each filter's own quadrature weights, eq. betadDefA"),
    "gauss_weights_unscaled": (
        "oracle.filters", "opt_parameters_continuous", "weights = [0.5 * tm * wx for tm in t_fm]",
        "weights = [tm * wx for tm in t_fm]", "Gauss-Legendre weights mapped to [0, T_{f,m}]"),
    # --- warm-start network (oracle/cnn.py) ---------------------------------------------------
    "conv_flipped_kernel": (
        "oracle.cnn", "conv_same", 'np.einsum("oc,bchw->bohw", w[:, :, dy, dx], patch)',
        'np.einsum("oc,bchw->bohw", w[:, :, 2 - dy, 2 - dx], patch)',
        "convolution instead of cross-correlation"),
    "conv_backward_shift": (
        "oracle.cnn", "conv_same_backward", "gxp[:, :, dy:dy + H, dx:dx + W] +=",
        "gxp[:, :, 2 - dy:2 - dy + H, 2 - dx:2 - dx + W] +=", "input gradient scattered back"),
    "relu_derivative_dropped": (
        "oracle.cnn", "loss_and_grads", "g = gx * (acts[i] > 0.0)", "g = gx",
        "ReLU derivative in backpropagation"),
    "loss_gradient_factor": (
        "oracle.cnn", "loss_and_grads", "g = 2.0 * diff / count", "g = diff / count",
        "factor 2 of the squared-error gradient"),
    "adam_bias_power": (
        "oracle.cnn", "adam_step", "mhat = m / (1.0 - beta1 ** t)", "mhat = m / (1.0 - beta1)",
        "power t of Adam's bias correction"),
    "adam_eps_inside_sqrt": (
        "oracle.cnn", "adam_step", "(np.sqrt(vhat) + eps)", "np.sqrt(vhat + eps)",
        "epsilon added after the square root in Adam"),
    "relu_on_output": (
        "oracle.cnn", "forward", "if i + 1 < len(params):", "if i < len(params):",
        "no ReLU after the last layer"),
    "adam_first_moment_weight": (
        "oracle.cnn", "adam_step", "m = beta1 * m + (1.0 - beta1) * g", "m = beta1 * m + beta1 * g",
        "weight 1 - beta1 of the new gradient in Adam's first moment"),
    "adam_second_moment_linear": (
        "oracle.cnn", "adam_step", "v = beta2 * v + (1.0 - beta2) * g * g",
        "v = beta2 * v + (1.0 - beta2) * np.abs(g)", "squared gradient in Adam's second moment"),
    "conv_bias_dropped_in_gradient": (
        "oracle.cnn", "conv_same_backward", "gb = gout.sum(axis=(0, 2, 3))",
        "gb = gout.sum(axis=(0, 2, 3)) * 0.0", "bias gradient"),
}


def apply(name):
    """Replace the target function (or method) of mutant `name` by its mutated copy."""
    import importlib

    mod_name, target, old, new, _ = MUTANTS[name]
    mod = importlib.import_module(mod_name)
    owner, attr = mod, target
    if "." in target:
        cls, attr = target.split(".")
        owner = getattr(mod, cls)
    src = textwrap.dedent(inspect.getsource(getattr(owner, attr)))
    if src.count(old) != 1:
        raise ValueError(f"mutant {name}: expected the text once in {target}, found "
                         f"{src.count(old)} times")
    namespace = dict(mod.__dict__)
    exec(compile(src.replace(old, new), f"<mutant {name}>", "exec"), namespace)
    setattr(owner, attr, namespace[attr])
