"""Pins for the two bounds behind the FP64 CG head's exact <w,p>_c sum.

The head adds each thread's share of an element as a 128-bit fixed-point
integer at a scale 2^S chosen from <p,p>_c and an operator bound, so that no
sum can overflow.  Two facts carry that choice, and both are checked here with
the oracle alone:

* the element operator of Listing 1 (Sec. III) satisfies, pointwise,
  |A_e p| <= 9 |D|_1 |D|_inf max|G| max|p| (three derivatives, the 3x3
  geometric contraction, three transposed derivatives, each bounded by the
  triangle inequality);
* the CG recursion <p',p'>_c = rho' + beta^2 <p,p>_c (r' is orthogonal to p)
  follows the true <p,p>_c closely over a long run; the head allows a factor
  16 of error in it.
Measured here: max|A_e p| reaches 0.5-2.6 % of the operator bound (it is a
safe bound, which is the direction that matters), and the recursion matches
the true <p,p>_c to 2e-12 relative over 1500 iterations, through
convergence and 18 orders of magnitude of residual beyond it.
"""
import numpy as np
import pytest

from paper_2005_13425_gb300 import inputs


def operator_bound(D, gxyz):
    d1 = np.abs(D).sum(axis=0).max()      # max column sum
    dinf = np.abs(D).sum(axis=1).max()    # max row sum
    return 9.0 * d1 * dinf * np.abs(gxyz).max()


@pytest.mark.parametrize("n", [2, 4, 6, 10, 12])
def test_element_operator_bound(oracle, n):
    dims = (3, 2, 2)
    P = oracle.box_problem(*dims, n, 0.2, inputs.perturbation_coeffs(n))
    rng = np.random.default_rng(n)
    A = operator_bound(P["D"], P["gxyz"])
    for trial in range(4):
        # random, smooth and single-point inputs, the last ones the worst case
        # for cancellation-free growth
        if trial == 0:
            u = rng.uniform(-1, 1, (P["E"], n ** 3))
        elif trial == 1:
            u = np.sign(rng.uniform(-1, 1, (P["E"], n ** 3)))
        elif trial == 2:
            u = np.sin(3.0 * P["xyz"][:, 0]) * np.cos(2.0 * P["xyz"][:, 1])
        else:
            u = np.zeros((P["E"], n ** 3))
            u[np.arange(P["E"]), rng.integers(0, n ** 3, P["E"])] = 1.0
        w = oracle.ax_e(P["D"], P["gxyz"], u)
        assert np.abs(w).max() <= A * np.abs(u).max()


def test_search_direction_norm_recursion(oracle):
    """1500 CG iterations (oracle operator, weighted dot) on a problem that
    converges after about 600, so the run covers both the convergence phase
    and the round-off phase beyond it (relative residual down to ~1e-28): the
    recursion for <p,p>_c stays within 1 % of the true value (the head allows
    a factor 16).  Solves of the benchmark's problem take 850-1150
    iterations to 1e-10."""
    dims, n = (8, 8, 4), 10
    P = oracle.box_problem(*dims, n, inputs.PERTURB_AMP, inputs.perturbation_coeffs(0))
    f = oracle.apply_mask(P["mask"], oracle.scatter_unique(*dims, n, inputs.unique_field(*dims, n, 1)))
    dot = lambda a, b: oracle.dot_c(*dims, n, a, b)
    apply = lambda v: oracle.apply_A(*dims, n, P["D"], P["gxyz"], P["mask"], v)
    r = f.copy()
    p = np.zeros_like(f)
    rho_old, pn2 = 1.0, 0.0
    worst = 1.0
    f2 = dot(f, f)
    for it in range(1500):
        rho = dot(r, r)
        beta = 0.0 if it == 0 else rho / rho_old
        p = r + beta * p
        pn2 = rho if it == 0 else rho + beta * beta * pn2
        true = dot(p, p)
        worst = max(worst, pn2 / true, true / pn2)
        w = apply(p)
        alpha = rho / dot(w, p)
        r = r - alpha * w
        rho_old = rho
    assert np.sqrt(rho / f2) < 1e-20          # well past convergence
    assert worst <= 1.01
