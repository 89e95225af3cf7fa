"""Pins for the oracle's Jacobi preconditioner and PCG (preconditioned CG is
the paper's named future work, Sec. VII).

* The element-matrix diagonal equals the diagonal of the dense element
  matrix built by applying ax_e to unit vectors (brute force).
* PCG with the identity preconditioner reproduces plain CG bit for bit.
* Jacobi PCG converges to the dense library solve of the assembled system
  and, on a stretched mesh, needs fewer iterations than CG.
"""
import numpy as np
import pytest

from paper_2005_13425_gb300 import inputs
from tests.test_oracle_dssum_cg import assembled_interior_matrix


@pytest.mark.parametrize("n", [2, 3, 5])
def test_diag_matches_bruteforce_element_matrix(oracle, n):
    # 2x2x2 elements: interior element edges carry nonzero cross metric
    # terms g_rs, g_rt, g_st at the corner indices where D(i,i) != 0
    P = oracle.box_problem(2, 2, 2, n, 0.05, inputs.perturbation_coeffs(6))
    d = oracle.diag_e(P["D"], P["gxyz"])
    n3 = n ** 3
    for e in range(P["E"]):
        for q in range(n3):
            u = np.zeros((1, n3))
            u[0, q] = 1.0
            Aq = oracle.ax_e(P["D"], P["gxyz"][e:e + 1], u)[0]
            assert abs(Aq[q] - d[e, q]) <= 1e-13 * abs(Aq[q]), (e, q)


def test_pcg_identity_equals_cg(oracle):
    dims, n = (2, 2, 2), 5
    P = oracle.box_problem(*dims, n, 0.05, inputs.perturbation_coeffs(0))
    f = oracle.apply_mask(P["mask"], oracle.scatter_unique(*dims, n, inputs.unique_field(*dims, n)))
    ones = np.ones_like(f)
    x1, it1, rr1, h1, _ = oracle.cg(*dims, n, P["D"], P["gxyz"], P["mask"], f, tol=0.0, maxit=20)
    x2, it2, rr2, h2, _ = oracle.pcg(*dims, n, P["D"], P["gxyz"], P["mask"], ones, f, tol=0.0, maxit=20)
    assert it1 == it2 and np.array_equal(x1, x2) and np.array_equal(h1, h2) and rr1 == rr2


def test_jacobi_pcg_dense_solve_and_iterations(oracle):
    dims, n = (2, 2, 2), 4
    P = oracle.box_problem(*dims, n, 0.05, inputs.perturbation_coeffs(2))
    # stretch the mesh: scale the metric per element (a mesh of very
    # different element sizes) -- the diagonal then varies strongly
    scale = np.array([1.0, 30.0, 0.05, 8.0, 1.0, 0.2, 12.0, 0.5])[:, None, None]
    g = P["gxyz"] * scale
    P2 = dict(P, gxyz=g)
    A, idx = assembled_interior_matrix(oracle, P2)
    f_u = inputs.unique_field(*dims, n, seed=1)
    f = oracle.apply_mask(P["mask"], oracle.scatter_unique(*dims, n, f_u))
    minv = oracle.jacobi_inverse(*dims, n, P["D"], g, P["mask"])
    assert np.all(minv[P["mask"] == 0] == 0) and np.all(minv[P["mask"] == 1] > 0)
    x, it, rr, hist, st = oracle.pcg(*dims, n, P["D"], g, P["mask"], minv, f, tol=1e-12, maxit=2000)
    assert st == 0 and rr <= 1e-12
    NX, NY, NZ = inputs.unique_grid_shape(*dims, n)
    xg = np.zeros(NX * NY * NZ)
    xg[P["gid"].reshape(-1)] = x.reshape(-1)
    xd = np.linalg.solve(A, f_u[idx])
    assert np.abs(xg[idx] - xd).max() <= 10 * np.linalg.cond(A) * 1e-12 * np.abs(xd).max()
    _, it_cg, _, _, _ = oracle.cg(*dims, n, P["D"], g, P["mask"], f, tol=1e-12, maxit=2000)
    assert it < it_cg
