"""Planted mistakes in the oracle, one at a time: each must make one of the
oracle's pins fail.

The pins (tests/test_oracle_pins.py, tests/test_integrators.py) tie the
oracle to closed forms, mpmath, scipy, exact eigenbases, quadrature exactness
and the paper's printed errors.  These tests show that they constrain the
arithmetic and not only the shapes: every plausible slip below (a dropped
term, a wrong sign, index or factorial, a transposed operand, a missing
scale, a wrong vec order) is planted on the CPU by recompiling one oracle
function with a one-line textual change (or by wrapping it), and the pin
named beside it must then fail.  The oracle's files are never modified.
"""
import inspect
import textwrap

import pytest

from oracle import dense, eig, expm, integrators, kron, params, phi_scalar, phiks_ref, quadrature
from oracle import taylor_action as ta

import test_complex_oracle as cpins
import test_integrators as ipins
import test_oracle_pins as pins


def plant(monkeypatch, module, name, old, new):
    """Replace module.name by its own source with `old` changed to `new`
    (exactly one occurrence), compiled in a copy of the module's globals."""
    src = textwrap.dedent(inspect.getsource(getattr(module, name)))
    assert src.count(old) == 1, (module.__name__, name, old)
    ns = dict(vars(module))
    exec(compile(src.replace(old, new), "<planted %s.%s>" % (module.__name__, name), "exec"), ns)
    monkeypatch.setattr(module, name, ns[name])
    return ns[name]


def fails(pin, *args):
    with pytest.raises(AssertionError):
        pin(*args)


# ------------------------------------------------------------------ phi_l(z)
def test_recurrence_factorial_index(monkeypatch):
    plant(monkeypatch, phi_scalar, "phi_recurrence", "math.factorial(j - 1)", "math.factorial(j)")
    fails(pins.test_phi_scalar_closed_form, 2, -4.5)


def test_series_term_index(monkeypatch):
    plant(monkeypatch, phi_scalar, "phi_series", "term * z / (k + l)", "term * z / (k + l - 1)")
    fails(pins.test_phi_scalar_closed_form, 2, 0.7)


# ------------------------------------------------------------------ expm, Kronecker algebra
def test_expm_one_squaring_short(monkeypatch):
    plant(monkeypatch, expm, "expm_taylor", "for _ in range(t):", "for _ in range(t - 1):")
    fails(pins.test_expm_vs_scipy)


def test_dense_oracle_with_a_short_expm(monkeypatch):
    bad = plant(monkeypatch, expm, "expm_taylor", "for _ in range(t):", "for _ in range(t - 1):")
    monkeypatch.setattr(dense.lincomb, "__defaults__", (1.0, bad))
    fails(pins.test_oracles_vs_mpmath_1d, 0.0, 10, 5e-3)


def test_expm_series_stopped_too_early(monkeypatch):
    plant(monkeypatch, expm, "expm_taylor", "2.0 ** -56 *", "2.0 ** -20 *")
    fails(pins.test_expm_vs_scipy)


def test_mode_product_transposed_operand(monkeypatch):
    plant(monkeypatch, kron, "mode_product", "axes=([1], [mu])", "axes=([0], [mu])")
    fails(pins.test_tucker_lemma_and_kron_exp)


def test_taylor_action_with_transposed_operators(monkeypatch):
    plant(monkeypatch, kron, "mode_product", "axes=([1], [mu])", "axes=([0], [mu])")
    fails(pins.test_oracles_vs_mpmath_1d, -20.0, 12, 5e-4)


def test_row_major_vec(monkeypatch):
    plant(monkeypatch, kron, "vec", 'order="F"', 'order="C"')
    plant(monkeypatch, kron, "unvec", 'order="F"', 'order="C"')
    fails(pins.test_tucker_lemma_and_kron_exp)


def test_kronecker_sum_factor_order(monkeypatch):
    plant(monkeypatch, kron, "kron_sum_dense", "for nu in reversed(range(d)):", "for nu in range(d):")
    fails(pins.test_tucker_lemma_and_kron_exp)


# ------------------------------------------------------------------ O1, O3
def test_augmented_shift_below_the_diagonal(monkeypatch):
    plant(monkeypatch, dense, "augmented", "B[N + k, N + k + 1] = 1.0", "B[N + k + 1, N + k] = 1.0")
    fails(pins.test_oracles_vs_mpmath_1d, 0.0, 10, 5e-3)


def test_augmented_columns_in_the_wrong_order(monkeypatch):
    plant(monkeypatch, dense, "lincomb", "vz[p + 1 - k] for k in range(1, p + 1)", "vz[k] for k in range(1, p + 1)")
    fails(pins.test_oracles_vs_mpmath_1d, 0.0, 10, 5e-3)


def test_dense_scale_applied_to_k_only(monkeypatch):
    plant(monkeypatch, dense, "lincomb", "E = expm(c * B)", "E = expm(augmented(c * tau * K, eta * W))")
    fails(pins.test_same_vs_lincomb_and_scales)


def test_taylor_action_ignores_the_scale(monkeypatch):
    plant(monkeypatch, ta, "lincomb", "h = c / sigma", "h = 1.0 / sigma")
    fails(pins.test_taylor_action_vs_dense_3d)


def test_taylor_action_drops_the_highest_vector(monkeypatch):
    plant(monkeypatch, ta, "lincomb", "W = [vz[p + 1 - k] for k in range(1, p + 1)]",
          "W = [None] + [vz[p + 1 - k] for k in range(2, p + 1)]")
    fails(pins.test_oracles_vs_mpmath_1d, 5.0, 9, 2e-3)


def test_taylor_action_shift_in_the_wrong_direction(monkeypatch):
    plant(monkeypatch, ta, "lincomb", "ybot[:-1] = y[1:]", "ybot[1:] = y[:-1]")
    fails(pins.test_oracles_vs_mpmath_1d, 0.0, 10, 5e-3)


def test_taylor_action_without_its_scaling(monkeypatch):
    plant(monkeypatch, ta, "lincomb", "sigma = max(1, int(math.ceil(abs(c) * normB)))", "sigma = 1")
    fails(pins.test_taylor_action_vs_eigenbasis_at_a_large_norm)


# ------------------------------------------------------------------ O2
def test_eigenbasis_with_n_in_place_of_n_plus_one(monkeypatch):
    plant(monkeypatch, eig, "eig_factors", "np.cos(k * pi / (n + 1))", "np.cos(k * pi / n)")
    fails(pins.test_sine_eigenbasis)


def test_eigenbasis_similarity_inverted(monkeypatch):
    plant(monkeypatch, eig, "eig_factors", "r = np.sqrt(a_ / c_)", "r = np.sqrt(c_ / a_)")
    fails(pins.test_sine_eigenbasis)


def test_complex_eigenbasis_with_zeta_conjugated(monkeypatch):
    plant(monkeypatch, eig, "scaled_phi_actions", "complex(c) * tau * complex(zeta) * Z",
          "complex(c) * tau * complex(zeta).conjugate() * Z")
    fails(cpins.test_eigenbasis_matches_dense_exponential)


def test_complex_eigenbasis_without_the_scale_power(monkeypatch):
    plant(monkeypatch, eig, "scaled_lincomb", "acc = acc + c ** l *", "acc = acc +")
    fails(cpins.test_eigenbasis_matches_taylor_action, 7, 2)


# ------------------------------------------------------------------ quadrature
def test_gll_weights_not_halved(monkeypatch):
    plant(monkeypatch, quadrature, "gll", "return (x + 1.0) / 2.0, w / 2.0", "return (x + 1.0) / 2.0, w")
    fails(pins.test_gll_exactness, 5)


def test_gll_interior_nodes_from_p_instead_of_its_derivative(monkeypatch):
    plant(monkeypatch, quadrature, "gll", "L.legroots(L.legder(c))", "L.legroots(c[:-1])")
    fails(pins.test_gll_exactness, 5)


def test_gl_nodes_left_on_minus_one_one(monkeypatch):
    plant(monkeypatch, quadrature, "gl", "return (x + 1.0) / 2.0, w / 2.0", "return x, w / 2.0")
    fails(pins.test_gl_exactness, 3)


# ------------------------------------------------------------------ the restated method
def test_small_exponentials_at_theta_instead_of_one_minus_theta(monkeypatch):
    plant(monkeypatch, phiks_ref, "_exps", "(1.0 - theta) * tau", "theta * tau")
    fails(pins.test_phiks_ref_scalar_squaring)


def test_same_vector_doubling_divides_by_the_wrong_power(monkeypatch):
    plant(monkeypatch, phiks_ref, "same", "acc[l - 1] = tot / 2.0 ** l", "acc[l - 1] = tot / 2.0 ** (l - 1)")
    fails(pins.test_phiks_ref_scalar_squaring)


def test_same_vector_node_weights_without_the_factorial(monkeypatch):
    plant(monkeypatch, phiks_ref, "same", "/ math.factorial(l - 1) * Y", "* Y")
    fails(pins.test_phiks_ref_scalar_squaring)


def test_linear_combination_doubling_with_the_wrong_level(monkeypatch):
    plant(monkeypatch, phiks_ref, "lincomb", "2.0 ** ((l - k) * j)", "2.0 ** ((l - k) * (j - 1))")
    fails(pins.test_phiks_ref_scales_match_fresh_calls)


def test_linear_combination_inputs_without_the_scaling(monkeypatch):
    plant(monkeypatch, phiks_ref, "lincomb", "/ 2.0 ** ((l - k + 1) * s)", "/ 2.0 ** ((l - k) * s)")
    fails(pins.test_phiks_ref_scales_match_fresh_calls)


# ------------------------------------------------------------------ parameter selection
def test_remainder_estimate_without_the_crouzeix_palencia_constant(monkeypatch):
    plant(monkeypatch, params, "remainder_bounds_all", "est.max() * (1.0 + math.sqrt(2.0)) / N_ZETA",
          "est.max() / N_ZETA")
    fails(pins.test_remainder_bound_is_the_crouzeix_palencia_constant_times_the_scalar_remainder, -5.0, "gll")


def test_remainder_estimate_without_the_scaling_by_two_to_the_s(monkeypatch):
    plant(monkeypatch, params, "remainder_bounds_all", "w = rect_boundary(rect) / (2.0 ** s)",
          "w = rect_boundary(rect)")
    fails(pins.test_remainder_bound_is_the_crouzeix_palencia_constant_times_the_scalar_remainder, -5.0, "gll")


def test_remainder_estimate_with_the_wrong_factorial(monkeypatch):
    plant(monkeypatch, params, "remainder_bounds_all", "/ math.factorial(l - 1) * dz", "/ math.factorial(l) * dz")
    fails(pins.test_remainder_bound_is_the_crouzeix_palencia_constant_times_the_scalar_remainder, -5.0, "gll")


def test_numerical_range_with_the_parts_swapped(monkeypatch):
    plant(monkeypatch, params, "numerical_range_rect", "eh = np.linalg.eigvalsh(H)", "eh = np.linalg.eigvalsh(S)")
    fails(pins.test_numerical_range_rectangle_contains_spectrum_and_range)


def test_tucker_count_without_the_scale_operators(monkeypatch):
    plant(monkeypatch, params, "tucker_count", "q + s * p + nscales if", "q + s * p if")
    fails(pins.test_tucker_count_is_the_operators_the_restatement_applies, "gl", monkeypatch)


# ------------------------------------------------------------------ integrators
def test_etd2rk_weight_halved(monkeypatch):
    monkeypatch.setitem(integrators.TABLEAUX, "etd2rk", ([(2, 1.0, {})], {2: [(0.5, 2, 1.0)]}))
    fails(ipins.test_oracle_reproduces_printed_errors, "etd2rk", 200, 1e-5)


def test_exponential_euler_without_the_nonlinear_term(monkeypatch):
    plant(monkeypatch, integrators, "exprk_step", "x = lc(blocks, tau, [u, tau * gn])", "x = lc(blocks, tau, [u])")
    fails(ipins.test_oracle_reproduces_printed_errors, "expeuler", 300, 1e-7)


def test_allen_cahn_nonlinearity_with_the_wrong_sign(monkeypatch):
    plant(monkeypatch, integrators, "ac_g", "return -(u * u * u) / (eps * eps)", "return (u * u * u) / (eps * eps)")
    fails(ipins.test_steady_states_are_kept, "etd2rk")


def test_brusselator_nonlinearity_with_the_species_swapped(monkeypatch):
    plant(monkeypatch, integrators, "bruss_g", "np.concatenate([a + uuv, b * u - uuv])",
          "np.concatenate([b * u - uuv, a + uuv])")
    fails(ipins.test_steady_states_are_kept, "exprk3")


def test_stages_without_the_phi_1_term(monkeypatch):
    plant(monkeypatch, integrators, "exprk_step", "x = lc(blocks, ci * tau, [u, ci * tau * gn])",
          "x = lc(blocks, ci * tau, [u])")
    fails(ipins.test_steady_states_are_kept, "exprk4s6")


def test_exprk3_with_the_sign_of_gamma_flipped(monkeypatch):
    bad = plant(monkeypatch, integrators, "_exprk3", "gam = (3 * c3 - 2) * c3", "gam = -(3 * c3 - 2) * c3")
    monkeypatch.setitem(integrators.TABLEAUX, "exprk3", bad())
    fails(ipins.test_orders_fourth_order_schemes_block_diagonal)
