"""Multiplicative two-grid cycle (ams_options.two_grid_omega) against the
oracle's cycle (OracleAMS.apply_two_grid): the applied preconditioner
element by element for one and several right-hand sides (fused and
separate backward coarse substitution), and PCG iterations and solutions."""

import numpy as np
import pytest

from oracle import OracleAMS, csr_to_scipy, pcg
from workloads import make_small_2d, make_small_3d

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2606_04864_gb300 import AmsSolver  # noqa: E402

ROUND = {"fp64": None, "fp32": "fp32", "fp32_bf16": "bf16"}


def _case(kind):
    if kind == "2d":
        return make_small_2d(side=45, bs=10, m=3, std=2.0, sigma=3.0, seed=31, ny=37)
    return make_small_3d(side=16, bs=8, m=6, std=2.5, sigma=3.0, seed=32)


@pytest.mark.parametrize("kind", ["2d", "3d"])
@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("fp32", 5e-5), ("fp32_bf16", 5e-5)])
@pytest.mark.parametrize("nrhs", [1, 3, 6])
def test_two_grid_apply_matches_oracle(kind, prec, tol, nrhs):
    w = _case(kind)
    A = csr_to_scipy(w.rowptr, w.colind, w.vals)
    o = OracleAMS(A, w.part, w.nparts, w.m, basis_round=ROUND[prec])
    omega = 1.0 / o.local_lambda_max()
    s = AmsSolver(w.rowptr, w.colind, w.vals, w.part, w.nparts, w.m, precision=prec, two_grid_omega=omega)
    r = np.random.default_rng(5).standard_normal((nrhs, w.n))
    z = s.apply_preconditioner(r)
    for k in range(nrhs):
        zr = o.apply_two_grid(r[k], omega)
        assert np.linalg.norm(z[k] - zr) <= tol * np.linalg.norm(zr), (kind, prec, nrhs, k)


@pytest.mark.parametrize("kind", ["2d", "3d"])
def test_two_grid_pcg_matches_oracle(kind):
    w = _case(kind)
    A = csr_to_scipy(w.rowptr, w.colind, w.vals)
    o = OracleAMS(A, w.part, w.nparts, w.m)
    omega = 1.0 / o.local_lambda_max()
    ref = pcg(A, w.rhs[0], lambda r: o.apply_two_grid(r, omega), rtol=1e-8)
    s = AmsSolver(w.rowptr, w.colind, w.vals, w.part, w.nparts, w.m, precision="fp64", two_grid_omega=omega)
    u, its, rel = s.solve(w.rhs[0], rtol=1e-8)
    assert abs(int(its[0]) - ref.iters) <= 2
    assert np.linalg.norm(u - ref.u) <= 1e-10 * np.linalg.norm(ref.u)
    # the mixed path converges to the same solution; the cycle needs fewer
    # iterations than the additive preconditioner on the same coarse space
    m = AmsSolver(w.rowptr, w.colind, w.vals, w.part, w.nparts, w.m, precision="fp32_bf16",
                  two_grid_omega=omega)
    um, itm, relm = m.solve(w.rhs[0], rtol=1e-8)
    assert np.linalg.norm(w.rhs[0] - A @ um) <= 1e-6 * np.linalg.norm(w.rhs[0])
    # mixed path (flexible CG on the reduced-precision cycle): iterations
    # within 2 of the oracle's flexible CG on the FP64 cycle, solution within
    # max(1e-6, 10 x the oracle's own rtol-1e-8 error) of the oracle's
    ref_f = pcg(A, w.rhs[0], lambda r: o.apply_two_grid(r, omega), rtol=1e-8, flexible=True)
    tight = pcg(A, w.rhs[0], lambda r: o.apply_two_grid(r, omega), rtol=1e-13)
    assert abs(int(itm[0]) - ref_f.iters) <= 2, (itm, ref_f.iters)
    floor = np.linalg.norm(ref_f.u - tight.u) / np.linalg.norm(tight.u)
    err = np.linalg.norm(um - ref_f.u) / np.linalg.norm(ref_f.u)
    assert err <= max(1e-6, 10 * floor), (err, floor)
    add = pcg(A, w.rhs[0], o.apply, rtol=1e-8)
    assert ref.iters < add.iters


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("fp32", 5e-5)])
def test_two_grid_without_coarse_space_matches_oracle(prec, tol):
    """With no coarse space the cycle is the symmetrised smoother
    2 omega S - omega^2 S A S (not the plain local solves)."""
    w = _case("2d")
    A = csr_to_scipy(w.rowptr, w.colind, w.vals)
    o = OracleAMS(A, w.part, w.nparts, w.m, coarse=False)
    omega = 0.8 / o.local_lambda_max()
    s = AmsSolver(w.rowptr, w.colind, w.vals, w.part, w.nparts, w.m, precision=prec, coarse=False,
                  two_grid_omega=omega)
    r = np.random.default_rng(8).standard_normal((3, w.n))
    z = s.apply_preconditioner(r)
    for k in range(3):
        zr = o.apply_two_grid(r[k], omega)
        assert np.linalg.norm(z[k] - zr) <= tol * np.linalg.norm(zr), (prec, k)
        zplain = o.local_part(r[k])
        assert np.linalg.norm(z[k] - zplain) > 1e-3 * np.linalg.norm(zplain)
    if prec == "fp64":
        ref = pcg(A, w.rhs[0], lambda r: o.apply_two_grid(r, omega), rtol=1e-8)
        u, its, _ = s.solve(w.rhs[0], rtol=1e-8)
        assert abs(int(its[0]) - ref.iters) <= 2
        assert np.linalg.norm(u - ref.u) <= 1e-10 * np.linalg.norm(ref.u)


def test_two_grid_omega_is_validated():
    from paper_2606_04864_gb300._lib import AmsError
    w = _case("2d")
    for bad in (-2.0, float("nan"), float("inf")):
        with pytest.raises(AmsError):
            AmsSolver(w.rowptr, w.colind, w.vals, w.part, w.nparts, w.m, two_grid_omega=bad)


@pytest.mark.parametrize("prec", ["fp64", "fp32_bf16"])
def test_two_grid_damping_from_power_steps(prec):
    """two_grid_omega = -c: setup estimates lambda_max of the local solves
    times A by power steps (from below) and takes omega = c / lambda_max;
    the estimate agrees with the oracle's Lanczos value, and the solve with
    that omega matches the oracle's cycle with the same omega."""
    w = _case("3d")
    A = csr_to_scipy(w.rowptr, w.colind, w.vals)
    o = OracleAMS(A, w.part, w.nparts, w.m, basis_round=ROUND[prec])
    lam = o.local_lambda_max()
    s = AmsSolver(w.rowptr, w.colind, w.vals, w.part, w.nparts, w.m, precision=prec, two_grid_omega=-1.0)
    info = s.info()
    est = info["local_lambda_max"]
    assert 0.99 * lam <= est <= lam * (1 + (1e-6 if prec == "fp64" else 1e-4)), (est, lam)
    assert info["two_grid_omega"] == pytest.approx(1.0 / est, rel=1e-15)
    omega = info["two_grid_omega"]
    ref = pcg(A, w.rhs[0], lambda r: o.apply_two_grid(r, omega), rtol=1e-8, flexible=(prec != "fp64"))
    u, its, rel = s.solve(w.rhs[0], rtol=1e-8)
    assert abs(int(its[0]) - ref.iters) <= 2, (its, ref.iters)
    err = np.linalg.norm(u - ref.u) / np.linalg.norm(ref.u)
    if prec == "fp64":
        assert err <= 1e-10, err
    else:
        tight = pcg(A, w.rhs[0], lambda r: o.apply_two_grid(r, omega), rtol=1e-13)
        floor = np.linalg.norm(ref.u - tight.u) / np.linalg.norm(tight.u)
        assert err <= max(1e-6, 10 * floor), (err, floor)
    from paper_2606_04864_gb300._lib import AmsError
    with pytest.raises(AmsError):
        AmsSolver(w.rowptr, w.colind, w.vals, w.part, w.nparts, w.m, precision=prec, two_grid_omega=-2.5)


def test_oversized_omega_is_reported_as_breakdown():
    """omega = 10 / lambda_max makes the cycle indefinite (r^T B r < 0 for
    the first residual already, checked on the oracle's cycle): the solve
    stops with AMS_ERR_BREAKDOWN instead of iterating on."""
    from paper_2606_04864_gb300._lib import AmsError
    w = _case("3d")
    A = csr_to_scipy(w.rowptr, w.colind, w.vals)
    o = OracleAMS(A, w.part, w.nparts, w.m)
    omega = 10.0 / o.local_lambda_max()
    assert w.rhs[0] @ o.apply_two_grid(w.rhs[0], omega) < 0
    for prec in ("fp64", "fp32_bf16"):
        s = AmsSolver(w.rowptr, w.colind, w.vals, w.part, w.nparts, w.m, precision=prec, two_grid_omega=omega,
                      maxit=500)
        with pytest.raises(AmsError) as e:
            s.solve(w.rhs[0], rtol=1e-8)
        assert e.value.status == 3, prec
