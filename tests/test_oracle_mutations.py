"""Planted mistakes in the oracle must be caught by its pins.

Each case swaps one oracle function for a subtly wrong copy (a dropped
term, a wrong sign, a transposed operand, a wrong index order) and runs the
pins that should notice.  The mistake lives only in this CPU process.
"""

import numpy as np
import pytest
import scipy.linalg as la

import oracle.ams_oracle as O
import tests.test_oracle_pins as P


def _expect_some_pin_fails(pins):
    failed = []
    for pin in pins:
        try:
            pin()
        except (AssertionError, ValueError, la.LinAlgError, np.linalg.LinAlgError):
            failed.append(pin.__name__)
    assert failed, "no pin caught the planted mistake"


def _patch(monkeypatch, name, fn):
    monkeypatch.setattr(O, name, fn)
    if hasattr(P, name):
        monkeypatch.setattr(P, name, fn)


def test_mutation_hat_diagonal_kept(monkeypatch):
    """Forgetting to replace the diagonal (\\hat A_i = A_i)."""
    orig = O.local_matrices

    def bad(A, dofs):
        Ai, Ahat, s = orig(A, dofs)
        return Ai, Ai.copy(), np.diag(Ai).copy()

    _patch(monkeypatch, "local_matrices", bad)
    _expect_some_pin_fails([P.test_first_mode_is_constant,
                            lambda: P.test_path_subdomain_closed_form(9)])


def test_mutation_weight_from_a_not_ahat(monkeypatch):
    """S_i taken from diag(A_i) instead of diag(\\hat A_i)."""
    orig = O.local_matrices

    def bad(A, dofs):
        Ai, Ahat, s = orig(A, dofs)
        return Ai, Ahat, np.diag(Ai).copy()

    _patch(monkeypatch, "local_matrices", bad)
    _expect_some_pin_fails([lambda: P.test_path_subdomain_closed_form(9),
                            P.test_first_mode_is_constant])


def test_mutation_largest_instead_of_smallest_modes(monkeypatch):
    orig = O.local_eigenpairs

    def bad(Ahat, s, m, tie_rtol=1e-8, all_pairs=False, threshold=None):
        lam, V = la.eigh(Ahat, np.diag(s))
        mi = min(m, Ahat.shape[0])
        return lam[::-1], V[:, ::-1][:, :mi].copy(), mi

    _patch(monkeypatch, "local_eigenpairs", bad)
    _expect_some_pin_fails([P.test_first_mode_is_constant,
                            P.test_theorem2_local_approximation_bound,
                            P.test_iterations_do_not_grow_with_more_modes])


def test_mutation_descending_order_in_subdomain(monkeypatch):
    orig = O.index_maps

    def bad(part, nparts):
        perm, iperm, sub_ptr = orig(part, nparts)
        perm = perm.copy()
        for i in range(nparts):
            perm[sub_ptr[i]:sub_ptr[i + 1]] = perm[sub_ptr[i]:sub_ptr[i + 1]][::-1]
        iperm = np.empty_like(perm)
        iperm[perm] = np.arange(len(perm))
        return perm, iperm, sub_ptr

    _patch(monkeypatch, "index_maps", bad)
    _expect_some_pin_fails([P.test_index_maps_brute_force])


def test_mutation_coarse_term_dropped_in_apply(monkeypatch):
    monkeypatch.setattr(O.OracleAMS, "apply", lambda self, r: self.local_part(r))
    _expect_some_pin_fails([P.test_full_coarse_space_reproduces_inverse,
                            P.test_iterations_do_not_grow_with_more_modes])


def test_mutation_coarse_uses_transposed_restriction(monkeypatch):
    def bad(self, r):
        if self.Nc == 0:
            return np.zeros_like(r)
        rc = (self.R0T.T @ r)[::-1]
        ec = la.cho_solve(self.A0_chol, rc)
        return self.R0T @ ec

    monkeypatch.setattr(O.OracleAMS, "coarse_part", bad)
    _expect_some_pin_fails([P.test_full_coarse_space_reproduces_inverse,
                            P.test_preconditioner_symmetric_positive_definite])


def test_mutation_wrong_beta(monkeypatch):
    orig = O.pcg

    def bad(A, f, Minv, rtol=1e-8, maxit=10000, flexible=False):
        def Mbad(r):
            return Minv(r)
        res = orig(A, f, Mbad, rtol, maxit, flexible)
        res.betas = [b * 1.01 for b in res.betas]
        return res

    _patch(monkeypatch, "pcg", bad)
    _expect_some_pin_fails([P.test_lanczos_ritz_values_match_dense_spectrum])


def test_mutation_adjoint_sign(monkeypatch):
    orig = O.adjoint_gradient

    def bad(A, u, g, Minv, rtol=1e-8, maxit=10000):
        lam, dvals, res = orig(A, u, g, Minv, rtol, maxit)
        return lam, -dvals, res

    _patch(monkeypatch, "adjoint_gradient", bad)
    _expect_some_pin_fails([P.test_adjoint_matches_dense_and_closed_form_and_fd])


_TWO_GRID_PINS = [P.test_two_grid_cycle_is_symmetric_positive_definite,
                  P.test_two_grid_full_coarse_space_is_the_inverse,
                  P.test_two_grid_without_coarse_space_is_the_symmetrised_smoother,
                  P.test_two_grid_identity_of_the_abstract_theory]


@pytest.mark.parametrize("mistake", ["no_post_smoothing", "coarse_on_r", "post_residual_sign",
                                     "undamped_post_smoothing"])
def test_mutation_two_grid_cycle(monkeypatch, mistake):
    """A dropped post-smoothing step, a coarse correction of r instead of
    the residual, a wrong sign in the post-smoothing residual, or damping
    on one smoothing step only."""
    def bad(self, r, omega):
        x1 = omega * self.local_part(r)
        if mistake == "coarse_on_r":
            x2 = x1 + self.coarse_part(r)
        else:
            x2 = x1 + self.coarse_part(r - self.A @ x1)
        if mistake == "no_post_smoothing":
            return x2
        if mistake == "post_residual_sign":
            return x2 + omega * self.local_part(r + self.A @ x2)
        if mistake == "undamped_post_smoothing":
            return x2 + self.local_part(r - self.A @ x2)
        raise AssertionError(mistake)

    monkeypatch.setattr(O.OracleAMS, "apply_two_grid", bad)
    _expect_some_pin_fails(_TWO_GRID_PINS)


def test_mutation_coarse_matrix_without_a(monkeypatch):
    """A_0 = R_0 R_0^T: the operator dropped from the Galerkin product."""
    def bad(A, R0T):
        return (R0T.T @ R0T).toarray()

    _patch(monkeypatch, "coarse_matrix", bad)
    _expect_some_pin_fails([P.test_coarse_matrix_spd_and_galerkin_brute_force,
                            P.test_full_coarse_space_reproduces_inverse])


def test_mutation_local_solve_with_a_perturbed_block(monkeypatch):
    """The fine-level solves factor A_i with its diagonal scaled by 1.05."""
    orig = O.local_matrices

    def bad(A, dofs):
        Ai, Ahat, s = orig(A, dofs)
        Ai = Ai + 0.05 * np.diag(np.diag(Ai))
        return Ai, Ahat, s

    _patch(monkeypatch, "local_matrices", bad)
    _expect_some_pin_fails([P.test_single_subdomain_converges_in_one_iteration,
                            P.test_local_matrix_definitions_brute_force])


@pytest.mark.parametrize("mistake", ["loose_threshold", "off_by_one"])
def test_mutation_threshold_count(monkeypatch, mistake):
    """The adaptive count taken against 1.5 times the threshold, or one mode
    short (down to zero modes)."""
    orig = O.local_eigenpairs

    def bad(Ahat, s, m, tie_rtol=1e-8, all_pairs=False, threshold=None):
        lam, Psi, mi = orig(Ahat, s, m, tie_rtol, all_pairs, None)
        if threshold is None:
            return lam, Psi, mi
        cap = min(m, Ahat.shape[0])
        if mistake == "loose_threshold":
            k = max(1, int(np.count_nonzero(lam[:cap] <= threshold * 1.5)))
        else:
            k = int(np.count_nonzero(lam[:cap] < threshold)) - 1
            k = max(k, 0)
        Psi_all = orig(Ahat, s, max(k, 1), tie_rtol, all_pairs, None)[1]
        return lam, Psi_all[:, :k], k

    _patch(monkeypatch, "local_eigenpairs", bad)
    _expect_some_pin_fails([P.test_threshold_count_and_the_bound_it_buys])


def test_mutation_smoother_lambda_max_from_point_jacobi(monkeypatch):
    """lambda_max taken for the point-Jacobi pencil (A, diag A) instead of
    the block-diagonal one."""
    def bad(self):
        d = self.A.diagonal()
        return float(la.eigh(self.A.toarray(), np.diag(d), eigvals_only=True).max())

    monkeypatch.setattr(O.OracleAMS, "local_lambda_max", bad)
    _expect_some_pin_fails([P.test_two_grid_cycle_is_symmetric_positive_definite])


def _bf16_pins():
    return [P.test_bf16_rounding_hand_worked_values,
            P.test_bf16_rounding_matches_integer_rounding_and_torch_on_binary32_inputs]


@pytest.mark.parametrize("kind", ["seven_bits", "truncate", "half_away", "via_binary32", "no_subnormal"])
def test_mutation_bf16_rounding(monkeypatch, kind):
    """Plausible mistakes in the bfloat16 storage rounding: one bit short,
    truncation, ties away from zero, double rounding through binary32, and
    normal spacing carried below 2^-126."""
    orig = O.round_basis

    def bad(Psi, mode):
        if mode != "bf16":
            return orig(Psi, mode)
        Psi = np.asarray(Psi, dtype=np.float64)
        m, e = np.frexp(Psi)
        if kind == "seven_bits":
            return np.ldexp(np.rint(m * 128.0), e - 7)
        if kind == "truncate":
            return np.ldexp(np.trunc(m * 256.0), e - 8)
        if kind == "half_away":
            return np.ldexp(np.sign(m) * np.floor(np.abs(m) * 256.0 + 0.5), e - 8)
        if kind == "via_binary32":
            return orig(Psi.astype(np.float32).astype(np.float64), mode)
        return np.ldexp(np.rint(m * 256.0), e - 8)        # no_subnormal

    monkeypatch.setattr(O, "round_basis", bad)
    import oracle.ams_oracle as OA
    monkeypatch.setattr(OA, "round_basis", bad)
    _expect_some_pin_fails(_bf16_pins())


@pytest.mark.parametrize("mistake", ["residual_sign", "stop_relative_to_r0"])
def test_mutation_initial_guess(monkeypatch, mistake):
    """CG from x_0 with r_0 = f + A x_0, or with the stop taken relative to
    ||r_0|| instead of ||f||, must fail the initial-guess pin."""
    orig = O.pcg

    def bad(A, f, Minv, rtol=1e-8, maxit=10000, flexible=False, x0=None):
        if x0 is None:
            return orig(A, f, Minv, rtol, maxit, flexible)
        f = np.asarray(f, dtype=np.float64)
        nf = np.linalg.norm(f)
        if mistake == "residual_sign":       # (f + 2 A x_0) - A x_0 = f + A x_0
            return orig(A, f + 2.0 * (A @ x0), Minv, rtol, maxit, flexible, x0=x0)
        r0 = np.linalg.norm(f - A @ x0)
        return orig(A, f, Minv, rtol * r0 / nf if nf > 0 else rtol, maxit, flexible, x0=x0)

    _patch(monkeypatch, "pcg", bad)
    _expect_some_pin_fails([P.test_pcg_from_an_initial_guess])
