"""Pins for the oracle's numbering, dssum, mask, weighted dot and CG.

dssum is the paper's second step of Ax (Sec. III: the element results are
communicated to the neighbouring elements); the mask is Nekbone's boundary
condition (Sec. VI.B); CG solves Ax = f (Sec. III).  Checks use a
coordinate-based numbering, brute-force sums in canonical order, a dense
library solve and a manufactured solution.
"""
import numpy as np
import pytest

from paper_2005_13425_gb300 import inputs


def coord_classes(oracle, dims, n):
    """Independent numbering: group local points by their physical position
    on the unperturbed box, rank the groups lexicographically by (z, y, x)."""
    xyz = oracle.box_coords(*dims, n, 0.0, (0, 0, 0))
    pts = np.stack([xyz[:, 0], xyz[:, 1], xyz[:, 2]], axis=-1).reshape(-1, 3)
    key = np.round(pts * 2 ** 30).astype(np.int64)
    uniq, inv, counts = np.unique(key[:, ::-1], axis=0, return_inverse=True, return_counts=True)
    return uniq[:, ::-1], inv.reshape(-1), counts


@pytest.mark.parametrize("dims,n", [((2, 2, 2), 3), ((3, 2, 1), 4), ((2, 3, 2), 5), ((1, 1, 1), 2)])
def test_numbering_multiplicity_mask(oracle, dims, n):
    uniq, inv, counts = coord_classes(oracle, dims, n)
    gid = oracle.gid(*dims, n).reshape(-1)
    np.testing.assert_array_equal(gid, inv)                 # bit-exact ids
    NX, NY, NZ = inputs.unique_grid_shape(*dims, n)
    assert len(uniq) == NX * NY * NZ
    mult = oracle.multiplicity(*dims, n).reshape(-1)
    np.testing.assert_array_equal(mult, counts[inv])
    assert set(np.unique(mult)) <= {1, 2, 4, 8}
    assert abs((1.0 / mult).sum() - NX * NY * NZ) < 1e-9
    msk = oracle.mask(*dims, n).reshape(-1)
    on_b = np.any((uniq[inv] == 0) | (uniq[inv] == 2 ** 30), axis=1)
    np.testing.assert_array_equal(msk == 0, on_b)


@pytest.mark.parametrize("dims,n", [((2, 2, 2), 3), ((3, 2, 2), 4), ((2, 2, 3), 6)])
def test_dssum_canonical_order_bruteforce(oracle, dims, n):
    E = dims[0] * dims[1] * dims[2]
    rng = np.random.default_rng(9)
    w = rng.uniform(-1, 1, (E, n ** 3)) * 10.0 ** rng.uniform(-8, 8, (E, n ** 3))
    got = oracle.dssum(*dims, n, w)
    gid = oracle.gid(*dims, n)
    # brute force: per unique node, add copies from +0.0 in ascending
    # (element, local index) order with Python floats, write back.
    want = np.empty_like(w)
    groups = {}
    for e in range(E):
        for q in range(n ** 3):
            groups.setdefault(int(gid[e, q]), []).append((e, q))
    for g, copies in groups.items():
        s = 0.0
        for e, q in sorted(copies):
            s = s + float(w[e, q])
        for e, q in copies:
            want[e, q] = s
    assert np.array_equal(got.view(np.uint64), want.view(np.uint64))
    ones = np.ones_like(w)
    np.testing.assert_array_equal(oracle.dssum(*dims, n, ones), oracle.multiplicity(*dims, n))


def test_dot_c_equals_unique_dot(oracle):
    dims, n = (3, 2, 2), 5
    a_u = inputs.unique_field(*dims, n, seed=3)
    b_u = inputs.unique_field(*dims, n, seed=4)
    a = oracle.scatter_unique(*dims, n, a_u)
    b = oracle.scatter_unique(*dims, n, b_u)
    got = oracle.dot_c(*dims, n, a, b)
    assert abs(got - float(np.dot(a_u, b_u))) < 1e-12 * np.abs(a_u * b_u).sum()
    # a continuous field is an eigenvector of dssum with the multiplicity
    np.testing.assert_allclose(oracle.dssum(*dims, n, a), a * oracle.multiplicity(*dims, n), rtol=1e-15)


def assembled_interior_matrix(oracle, P):
    """Dense assembled operator on the interior unique nodes, one column per
    unit vector (scattered to local storage, then A = mask(dssum(ax_e)))."""
    dims = (P["Ex"], P["Ey"], P["Ez"])
    n = P["n"]
    NX, NY, NZ = inputs.unique_grid_shape(*dims, n)
    gx, gy, gz = np.meshgrid(np.arange(NX), np.arange(NY), np.arange(NZ), indexing="ij")
    gids = (gx + NX * (gy + NY * gz)).transpose(2, 1, 0).reshape(-1)
    interior = ((gx > 0) & (gx < NX - 1) & (gy > 0) & (gy < NY - 1)
                & (gz > 0) & (gz < NZ - 1)).transpose(2, 1, 0).reshape(-1)
    idx = gids[interior]
    gid = P["gid"]
    cols = []
    for g in idx:
        u = (gid == g).astype(float)
        Au = oracle.apply_A(*dims, n, P["D"], P["gxyz"], P["mask"], u)
        # read the assembled value at one copy of each interior node
        first = np.zeros(NX * NY * NZ)
        first[gid.reshape(-1)] = Au.reshape(-1)
        cols.append(first[idx])
    return np.array(cols).T, idx


@pytest.mark.parametrize("dims,n", [((2, 2, 2), 3), ((2, 1, 2), 4)])
def test_cg_matches_dense_solve(oracle, dims, n):
    P = oracle.box_problem(*dims, n, 0.05, inputs.perturbation_coeffs(2))
    A, idx = assembled_interior_matrix(oracle, P)
    np.testing.assert_allclose(A, A.T, atol=1e-12 * np.abs(A).max())
    NX, NY, NZ = inputs.unique_grid_shape(*dims, n)
    f_u = inputs.unique_field(*dims, n, seed=1)
    f = oracle.apply_mask(P["mask"], oracle.scatter_unique(*dims, n, f_u))
    x, iters, relres, hist, st = oracle.cg(*dims, n, P["D"], P["gxyz"], P["mask"], f,
                                           tol=1e-13, maxit=1000)
    assert st == 0 and relres <= 1e-13 and iters < 1000
    xd = np.linalg.solve(A, f_u[idx])
    kappa = np.linalg.cond(A)
    xg = np.zeros(NX * NY * NZ)
    xg[P["gid"].reshape(-1)] = x.reshape(-1)
    assert np.abs(xg[idx] - xd).max() <= 10 * kappa * 1e-13 * np.abs(xd).max()
    # masked nodes stay exactly zero
    assert np.all(x[P["mask"] == 0] == 0.0)


def test_cg_energy_error_decreases_and_fixed_iterations(oracle):
    dims, n = (2, 2, 2), 4
    P = oracle.box_problem(*dims, n, 0.05, inputs.perturbation_coeffs(0))
    f = oracle.apply_mask(P["mask"], oracle.scatter_unique(*dims, n, inputs.unique_field(*dims, n)))
    xs, _, _, _, _ = oracle.cg(*dims, n, P["D"], P["gxyz"], P["mask"], f, tol=1e-14, maxit=2000)
    errs = []
    for k in range(1, 12):
        x, iters, relres, hist, st = oracle.cg(*dims, n, P["D"], P["gxyz"], P["mask"], f, tol=0.0, maxit=k)
        assert iters == k and len(hist) == k + 1 and st == 0
        e = x - xs
        Ae = oracle.apply_A(*dims, n, P["D"], P["gxyz"], P["mask"], e)
        errs.append(oracle.dot_c(*dims, n, e, Ae))
        # the recursive residual agrees with the true residual f - A x
        r = f - oracle.apply_A(*dims, n, P["D"], P["gxyz"], P["mask"], x)
        true_rel = np.sqrt(oracle.dot_c(*dims, n, r, r) / oracle.dot_c(*dims, n, f, f))
        assert abs(true_rel - relres) < 1e-10
    assert all(b < a for a, b in zip(errs, errs[1:]))   # A-norm error is monotone


def test_cg_zero_rhs(oracle):
    dims, n = (1, 2, 1), 4
    P = oracle.box_problem(*dims, n, 0.05, inputs.perturbation_coeffs(0))
    f = np.zeros((P["E"], n ** 3))
    x, iters, relres, hist, st = oracle.cg(*dims, n, P["D"], P["gxyz"], P["mask"], f, tol=0.0, maxit=10)
    assert iters == 0 and relres == 0.0 and np.all(x == 0) and st == 0


@pytest.mark.parametrize("n", [5, 7])
def test_cg_manufactured_solution(oracle, n):
    """u* = sin(pi x) sin(pi y) sin(pi z) at the nodes, masked; f = A u*.
    The discrete solution is u* itself, so CG must return it."""
    dims = (2, 2, 2)
    P = oracle.box_problem(*dims, n, 0.05, inputs.perturbation_coeffs(1))
    xyz = P["xyz"]
    us = np.sin(np.pi * xyz[:, 0]) * np.sin(np.pi * xyz[:, 1]) * np.sin(np.pi * xyz[:, 2])
    us = oracle.apply_mask(P["mask"], us)
    f = oracle.apply_A(*dims, n, P["D"], P["gxyz"], P["mask"], us)
    x, iters, relres, hist, st = oracle.cg(*dims, n, P["D"], P["gxyz"], P["mask"], f,
                                           tol=1e-12, maxit=3000)
    assert st == 0 and relres <= 1e-12
    assert np.abs(x - us).max() < 1e-8
