"""Pins for the oracle's geometry and element operator ax_e (Listing 1).

Each check comes from mathematics, not from the oracle itself: the null
space and symmetry of the weak Laplacian, a dense element matrix assembled
from an independent Lagrange-basis formula, exact GLL stiffness on affine
elements, and the isoparametric identity x_c^T A x_a = delta_ca sum(w detJ).
"""
import numpy as np
import pytest

from paper_2005_13425_gb300 import inputs
from tests.test_oracle_gll import barycentric_dmat


def problem(oracle, dims, n, amp=0.05, seed=0):
    s = inputs.perturbation_coeffs(seed)
    return oracle.box_problem(*dims, n, amp, s)


@pytest.mark.parametrize("n", [2, 3, 5, 8, 10])
def test_ax_constant_nullspace_and_symmetry(oracle, n):
    P = problem(oracle, (2, 2, 1), n)
    E = P["E"]
    ones = np.ones((E, n ** 3))
    w1 = oracle.ax_e(P["D"], P["gxyz"], ones)
    rng = np.random.default_rng(5)
    x = rng.uniform(-1, 1, (E, n ** 3))
    y = rng.uniform(-1, 1, (E, n ** 3))
    Ax = oracle.ax_e(P["D"], P["gxyz"], x)
    Ay = oracle.ax_e(P["D"], P["gxyz"], y)
    scale = np.abs(Ax).max()
    assert np.abs(w1).max() < 1e-12 * scale
    for e in range(E):
        a, b = np.dot(y[e], Ax[e]), np.dot(x[e], Ay[e])
        assert abs(a - b) < 1e-12 * (abs(a) + np.abs(y[e] * Ax[e]).sum())
        assert np.dot(x[e], Ax[e]) > 0


def element_matrix_bruteforce(D, g6):
    """A = sum_ab Dab^T diag(G_ab) Dab with Kronecker gradient matrices built
    from an independent derivative matrix; g6 is one element's gxyz."""
    n = D.shape[0]
    I = np.eye(n)
    Dr = np.kron(I, np.kron(I, D))     # d/dr acts on i (fastest)
    Ds = np.kron(I, np.kron(D, I))     # d/ds acts on j
    Dt = np.kron(D, np.kron(I, I))     # d/dt acts on k
    Gd = [Dr, Ds, Dt]
    comp = {(0, 0): 0, (0, 1): 1, (0, 2): 2, (1, 1): 3, (1, 2): 4, (2, 2): 5}
    A = np.zeros((n ** 3, n ** 3))
    for a in range(3):
        for b in range(3):
            g = g6[comp[(min(a, b), max(a, b))]]
            A += Gd[a].T @ (g[:, None] * Gd[b])
    return A


@pytest.mark.parametrize("n", [2, 3, 4])
def test_ax_dense_element_matrix_bruteforce(oracle, n):
    P = problem(oracle, (2, 1, 1), n, amp=0.05, seed=3)
    Dind = barycentric_dmat(P["xi"])
    n3 = n ** 3
    for e in range(P["E"]):
        # element matrix by applying ax_e to unit vectors
        Aor = np.zeros((n3, n3))
        for q in range(n3):
            u = np.zeros((1, n3))
            u[0, q] = 1.0
            Aor[:, q] = oracle.ax_e(P["D"], P["gxyz"][e:e + 1], u)[0]
        Abf = element_matrix_bruteforce(Dind, P["gxyz"][e])
        assert np.abs(Aor - Abf).max() < 1e-12 * np.abs(Abf).max()
        ev = np.linalg.eigvalsh(0.5 * (Aor + Aor.T))
        # positive semi-definite with the constants as the only null space
        assert abs(ev[0]) < 1e-12 * ev[-1]
        assert ev[1] > 1e-6 * ev[-1]


def monomial_field(xyz, a, b, c):
    return xyz[:, 0] ** a * xyz[:, 1] ** b * xyz[:, 2] ** c


def exact_stiffness(a, b, c, d, e, f):
    """Closed form of int_[0,1]^3 grad(x^a y^b z^c) . grad(x^d y^e z^f)."""
    def I(p):
        return 1.0 / (p + 1)
    t = 0.0
    if a and d:
        t += a * d * I(a + d - 2) * I(b + e) * I(c + f)
    if b and e:
        t += b * e * I(a + d) * I(b + e - 2) * I(c + f)
    if c and f:
        t += c * f * I(a + d) * I(b + e) * I(c + f - 2)
    return t


@pytest.mark.parametrize("n", [3, 4, 6, 8])
def test_ax_exact_stiffness_affine(oracle, n):
    P = problem(oracle, (2, 3, 2), n, amp=0.0)
    N = n - 1
    rng = np.random.default_rng(n)
    for trial in range(6):
        ex1 = rng.integers(0, N, size=3)     # degree <= N - 1 per variable
        ex2 = rng.integers(0, N, size=3)
        u = monomial_field(P["xyz"], *ex1)
        v = monomial_field(P["xyz"], *ex2)
        Au = oracle.ax_e(P["D"], P["gxyz"], u)
        got = float(np.sum(v * Au))
        want = exact_stiffness(*ex1, *ex2)
        assert abs(got - want) < 1e-12 * max(1.0, abs(want)), (ex1, ex2, got, want)


def test_affine_gxyz_closed_form(oracle):
    n = 5
    dims = (2, 3, 4)
    P = problem(oracle, dims, n, amp=0.0)
    h = [1.0 / d for d in dims]
    w = P["w"]
    wq = np.einsum("k,j,i->kji", w, w, w).reshape(-1)
    vol = h[0] * h[1] * h[2] / 8.0
    g = P["gxyz"]
    np.testing.assert_allclose(g[:, 0], np.broadcast_to(wq * vol * (2 / h[0]) ** 2, g[:, 0].shape), rtol=1e-13)
    np.testing.assert_allclose(g[:, 3], np.broadcast_to(wq * vol * (2 / h[1]) ** 2, g[:, 3].shape), rtol=1e-13)
    np.testing.assert_allclose(g[:, 5], np.broadcast_to(wq * vol * (2 / h[2]) ** 2, g[:, 5].shape), rtol=1e-13)
    for c in (1, 2, 4):
        assert np.abs(g[:, c]).max() < 1e-13 * np.abs(g[:, 0]).max()


@pytest.mark.parametrize("n", [4, 8, 10])
def test_isoparametric_identity_perturbed(oracle, n):
    """For u = x_a (a nodal coordinate field) and v = x_c:
    x_c^T A_e x_a = delta_ca * sum_q w_q detJ_q, on any (curved) element."""
    P = problem(oracle, (2, 2, 2), n, amp=0.05, seed=11)
    xyz = P["xyz"]
    w = P["w"]
    wq = np.einsum("k,j,i->kji", w, w, w).reshape(-1)
    vol_e = (P["detJ"] * wq).sum(axis=1)
    for a in range(3):
        Axa = oracle.ax_e(P["D"], P["gxyz"], xyz[:, a])
        for c in range(3):
            got = np.einsum("eq,eq->e", xyz[:, c], Axa)
            want = vol_e if a == c else np.zeros_like(vol_e)
            assert np.abs(got - want).max() < 1e-12 * vol_e.max(), (a, c)
    # the perturbed map keeps the unit cube: quadrature volume ~ 1 (spectral)
    assert abs(vol_e.sum() - 1.0) < 1e-4
    assert P["detJ"].min() > 0


def test_perturbation_keeps_boundary(oracle):
    P = problem(oracle, (3, 2, 2), 6, amp=0.05, seed=4)
    Q = oracle.box_problem(3, 2, 2, 6, 0.0, (0, 0, 0))
    on_b = P["mask"] == 0
    for d in range(3):
        np.testing.assert_allclose(P["xyz"][:, d][on_b], Q["xyz"][:, d][on_b], atol=1e-15)
    assert np.abs(P["xyz"] - Q["xyz"]).max() > 1e-3
