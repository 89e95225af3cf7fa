"""GPU parity: the CUDA path through the C ABI against the CPU oracle.

Tolerances (derived from the arithmetic):
* ax_e, apply: max-norm relative error <= 1e-12 (FP64 contract) on identical
  inputs (the same D and gxyz on both sides), at every n, for data whose
  output is of the order of its terms (random u); for smooth data, whose
  output cancels 1e3-2e4 times, 1e-12 |w| + 2^-50 |D|^2 |G| |u| (48-bit
  double-float arithmetic); the absolute form 1e-12 |D|^2 |G| |u| for the
  near-null input A 1.
* device-built geometry against the oracle's: n eps kappa_J of max|G|, with
  kappa_J = |D|_inf max|x| / min|dx/dr| the condition number of the
  isoparametric Jacobian J = D x (absolute coordinates: two FP64
  constructions of J differ by about eps kappa_J relative).
* dssum, mask, numbering, multiplicity, scatter: exact (value equality).
* weighted dots: relative 1e-13 (reduction order differs).
* CG: rho history and final x relative <= 1e-8 after 100 fixed iterations
  (CG amplifies reduction-order differences).
"""
import numpy as np
import pytest

from paper_2005_13425_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

AX_TOL = 1e-12


@pytest.fixture(scope="module")
def nek():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2005_13425_gb300 import build as b
    b.build()
    from paper_2005_13425_gb300 import nekgb
    nekgb.load()
    s = torch.cuda.Stream()
    torch.cuda.set_stream(s)
    return nekgb


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host(t):
    torch.cuda.current_stream().synchronize()
    return t.cpu().numpy()


def rel_err(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def geometry_tol(D, dims, n, amp=0.05):
    """n eps kappa_J: the rounding bound of the isoparametric Jacobian
    J = D x on absolute coordinates (|x| <= 1 + amp), relative to its
    smallest diagonal entry (1/(2 max(dims)) less the perturbation's
    gradient, at most 3 pi amp of it)."""
    kappa = np.abs(D).sum(1).max() * (1.0 + amp) / (0.5 / max(dims) * (1.0 - 3.0 * np.pi * amp))
    return n * np.finfo(np.float64).eps * kappa


class Ctx:
    def __init__(self, nek, *args, box=False, **kw):
        self.nek = nek
        stream = torch.cuda.current_stream()
        if box:
            self.h = nek.nb_setup_box(*args, stream=stream, **kw)
        else:
            self.h = nek.nb_setup(*args, stream=stream, **kw)

    def __enter__(self):
        return self.h

    def __exit__(self, *a):
        self.nek.nb_destroy(self.h)


def oracle_problem(oracle, dims, n, seed=0, amp=0.05):
    return oracle.box_problem(*dims, n, amp, inputs.perturbation_coeffs(seed))


# ------------------------------------------------------------------ ax_e
AX_CASES = [((5, 3, 2), 2), ((5, 3, 2), 3), ((4, 3, 2), 4), ((3, 3, 2), 5), ((3, 2, 2), 6),
            ((3, 2, 2), 7), ((3, 2, 2), 8), ((2, 2, 2), 9), ((3, 2, 2), 10), ((2, 2, 1), 11),
            ((2, 2, 2), 12), ((2, 1, 1), 13), ((2, 1, 1), 14), ((1, 2, 1), 15), ((2, 1, 1), 16)]


@pytest.mark.parametrize("dims,n", AX_CASES)
@pytest.mark.parametrize("variant", [0, 1, 2])
def test_ax_parity(nek, oracle, dims, n, variant):
    P = oracle_problem(oracle, dims, n)
    u = inputs.local_field(P["E"], n, seed=n)
    want = oracle.ax_e(P["D"], P["gxyz"], u)
    with Ctx(nek, dims, n, P["D"], P["gxyz"]) as ctx:
        nek.nb_set_ax_variant(ctx, variant)
        w = torch.empty(P["E"], n ** 3, dtype=torch.float64, device="cuda")
        nek.nb_ax(ctx, dev(u), w)
        got = host(w)
    assert rel_err(got, want) <= AX_TOL


@pytest.mark.parametrize("scale_u,scale_g", [(1e-30, 1.0), (1e25, 1.0), (1.0, 1e-25), (1e-12, 1e20)])
def test_ax_double_float_scale_invariance(nek, oracle, scale_u, scale_g):
    """The FP32-pair kernel scales inputs by exact powers of two, so tiny or
    huge data keep the same relative accuracy as data of order one."""
    dims, n = (3, 2, 2), 10
    P = oracle_problem(oracle, dims, n, seed=5)
    g = P["gxyz"] * scale_g
    u = inputs.local_field(P["E"], n, seed=6) * scale_u
    u[1] *= 1e-6                           # elements of very different magnitude
    want = oracle.ax_e(P["D"], g, u)
    with Ctx(nek, dims, n, P["D"], g) as ctx:
        nek.nb_set_ax_variant(ctx, 2)
        w = torch.empty(P["E"], n ** 3, dtype=torch.float64, device="cuda")
        nek.nb_ax(ctx, dev(u), w)
        got = host(w)
    assert rel_err(got, want) <= AX_TOL
    # the small element is accurate relative to itself too
    assert rel_err(got[1], want[1]) <= 1e-11


@pytest.mark.parametrize("n", [5, 10])
def test_ax_general_derivative_matrix(nek, oracle, n):
    """A D without the GLL centro-antisymmetry takes the plain line
    products (the even-odd form needs D(i,l) = -D(n-1-i, n-1-l))."""
    dims = (3, 2, 2)
    P = oracle_problem(oracle, dims, n, seed=9)
    D = np.random.default_rng(n).uniform(-5, 5, (n, n))
    u = inputs.local_field(P["E"], n, seed=4)
    want = oracle.ax_e(D, P["gxyz"], u)
    with Ctx(nek, dims, n, D, P["gxyz"]) as ctx:
        for variant in (0, 1):
            nek.nb_set_ax_variant(ctx, variant)
            w = torch.empty(P["E"], n ** 3, dtype=torch.float64, device="cuda")
            nek.nb_ax(ctx, dev(u), w)
            assert rel_err(host(w), want) <= AX_TOL, variant


@pytest.mark.parametrize("n", [8, 10, 12])
def test_ax_smooth_input_error_bound(nek, oracle, n):
    """Smooth data (the manufactured solution sin(pi x) sin(pi y) sin(pi z)
    and sin(3x) cos(2y) + 0.3 z^2) cancel 3.5e3 to 1.9e4 times between the
    terms of ax_e and its output.  The double-float kernel carries 48-bit
    significands, so its error there is set by the term scale TS =
    |D|_inf^2 |G| |u| (emulated: about 2^-53 TS), and the bound is
    1e-12 |w| + 2^-50 TS: the relative contract where the output is of the
    order of its terms, 2^-50 of the terms where it is not."""
    dims = (4, 4, 4)
    P = oracle_problem(oracle, dims, n)
    X = P["xyz"]
    fields = [np.sin(np.pi * X[:, 0]) * np.sin(np.pi * X[:, 1]) * np.sin(np.pi * X[:, 2]),
              np.sin(3.0 * X[:, 0]) * np.cos(2.0 * X[:, 1]) + 0.3 * X[:, 2] ** 2]
    with Ctx(nek, dims, n, P["D"], P["gxyz"]) as ctx:
        for u in fields:
            want = oracle.ax_e(P["D"], P["gxyz"], u)
            w = torch.empty(P["E"], n ** 3, dtype=torch.float64, device="cuda")
            nek.nb_ax(ctx, dev(u), w)
            got = host(w)
            TS = np.abs(P["D"]).sum(1).max() ** 2 * np.abs(P["gxyz"]).max() * np.abs(u).max()
            assert TS / np.abs(want).max() > 1e3            # the inputs are the high-cancellation case
            assert np.abs(got - want).max() <= 1e-12 * np.abs(want).max() + 2.0 ** -50 * TS


def test_ax_ragged_many_elements(nek, oracle):
    """More elements than the grid holds at once, with a ragged last wave."""
    dims, n = (13, 11, 7), 6
    P = oracle_problem(oracle, dims, n, seed=4)
    u = inputs.local_field(P["E"], n, seed=3)
    want = oracle.ax_e(P["D"], P["gxyz"], u)
    with Ctx(nek, dims, n, P["D"], P["gxyz"]) as ctx:
        w = torch.empty(P["E"], n ** 3, dtype=torch.float64, device="cuda")
        nek.nb_ax(ctx, dev(u), w)
        assert rel_err(host(w), want) <= AX_TOL


def test_ax_constant_nullspace(nek, oracle):
    dims, n = (3, 3, 3), 10
    P = oracle_problem(oracle, dims, n, seed=7)
    with Ctx(nek, dims, n, P["D"], P["gxyz"]) as ctx:
        w = torch.empty(P["E"], n ** 3, dtype=torch.float64, device="cuda")
        nek.nb_ax(ctx, torch.ones(P["E"], n ** 3, dtype=torch.float64, device="cuda"), w)
        got = host(w)
    # absolute bound: 1e-12 * |G| |D|^2 |u|
    bound = 1e-12 * np.abs(P["gxyz"]).max() * np.abs(P["D"]).sum(1).max() ** 2
    assert np.abs(got).max() <= bound


def test_full_size_geometry_and_ax_sampled(nek, oracle):
    """E = 4096, n = 10 in the benchmark's configuration (device-built
    geometry, automatic kernel choice), checked on sampled elements."""
    dims, n = (16, 16, 16), 10
    s = inputs.perturbation_coeffs(inputs.SEED_MESH)
    P = oracle.box_problem(*dims, n, inputs.PERTURB_AMP, s)
    E = P["E"]
    u = inputs.local_field(E, n, seed=inputs.SEED_U)
    rng = np.random.default_rng(123)
    sample = np.unique(np.concatenate([[0, E - 1], rng.choice(E, 96, replace=False)]))
    want = oracle.ax_e(P["D"], P["gxyz"][sample], u[sample])
    with Ctx(nek, dims, n, inputs.PERTURB_AMP, s, box=True) as ctx:
        D = nek.nb_get_operator(ctx, n)
        g = torch.empty(E, 6, n ** 3, dtype=torch.float64, device="cuda")
        nek.nb_get_operator(ctx, n, g)
        w = torch.empty(E, n ** 3, dtype=torch.float64, device="cuda")
        nek.nb_ax(ctx, dev(u), w)
        got = host(w)[sample]
        gd = host(g)
    assert rel_err(D, P["D"]) <= 1e-13
    # max-norm of the whole metric tensor: the off-diagonal factors are
    # small differences of cofactor products and carry absolute, not
    # relative, rounding error
    gmax = np.abs(P["gxyz"]).max()
    for c in range(6):
        assert np.abs(gd[:, c] - P["gxyz"][:, c]).max() <= 1e-12 * gmax, c
    assert rel_err(got, want) <= AX_TOL


# ------------------------------------------------------------------ dssum/mask
GS_CASES = [((3, 2, 2), 4), ((4, 3, 5), 5), ((2, 2, 2), 2), ((1, 1, 1), 6), ((1, 3, 1), 3),
            ((5, 1, 2), 8), ((16, 16, 16), 10)]


@pytest.mark.parametrize("dims,n", GS_CASES)
def test_dssum_mask_tables_exact(nek, oracle, dims, n):
    E = dims[0] * dims[1] * dims[2]
    rng = np.random.default_rng(n)
    w = rng.uniform(-1, 1, (E, n ** 3)) * 10.0 ** rng.integers(-6, 6, (E, n ** 3))
    D = np.eye(n)
    g = np.zeros((E, 6, n ** 3))
    with Ctx(nek, dims, n, D, g) as ctx:
        wd = dev(w)
        nek.nb_dssum(ctx, wd)
        got = host(wd)
        nek.nb_mask(ctx, wd)
        got_m = host(wd)
        gid = torch.empty(E, n ** 3, dtype=torch.int64, device="cuda")
        mult = torch.empty(E, n ** 3, dtype=torch.int32, device="cuda")
        msk = torch.empty(E, n ** 3, dtype=torch.uint8, device="cuda")
        nek.nb_tables(ctx, gid, mult, msk)
        gid, mult, msk = host(gid), host(mult), host(msk)
    want = oracle.dssum(*dims, n, w)
    assert np.array_equal(got, want)
    omask = oracle.mask(*dims, n)
    assert np.array_equal(got_m, oracle.apply_mask(omask, want))
    assert np.array_equal(gid, oracle.gid(*dims, n))
    assert np.array_equal(mult, oracle.multiplicity(*dims, n))
    assert np.array_equal(msk, omask)


def test_custom_mask_and_scatter(nek, oracle):
    dims, n = (3, 2, 2), 5
    E = 12
    rng = np.random.default_rng(1)
    cm = (rng.uniform(size=(E, n ** 3)) > 0.3).astype(np.uint8)
    w = rng.uniform(-1, 1, (E, n ** 3))
    with Ctx(nek, dims, n, np.eye(n), np.zeros((E, 6, n ** 3)), mask=cm) as ctx:
        wd = dev(w)
        nek.nb_mask(ctx, wd)
        assert np.array_equal(host(wd), oracle.apply_mask(cm, w))
        fu = inputs.unique_field(*dims, n, seed=5)
        loc = torch.empty(E, n ** 3, dtype=torch.float64, device="cuda")
        nek.nb_scatter_unique(ctx, dev(fu), loc)
        assert np.array_equal(host(loc), oracle.scatter_unique(*dims, n, fu))
        msk = torch.empty(E, n ** 3, dtype=torch.uint8, device="cuda")
        nek.nb_tables(ctx, mask=msk)
        assert np.array_equal(host(msk), cm)


def test_apply_and_dot(nek, oracle):
    dims, n = (4, 3, 3), 8
    P = oracle_problem(oracle, dims, n, seed=2)
    u = inputs.local_field(P["E"], n, seed=8)
    want = oracle.apply_A(*dims, n, P["D"], P["gxyz"], P["mask"], u)
    with Ctx(nek, dims, n, P["D"], P["gxyz"]) as ctx:
        w = torch.empty_like(dev(u))
        ud = dev(u)
        nek.nb_apply(ctx, ud, w)
        got = host(w)
        d = nek.nb_dot_c(ctx, ud, w)
    assert rel_err(got, want) <= AX_TOL
    dw = oracle.dot_c(*dims, n, u, want)
    assert abs(d - dw) <= 1e-12 * abs(dw)


# ------------------------------------------------------------------ CG
def cg_inputs(oracle, dims, n, seed_mesh=0, seed_f=1):
    P = oracle_problem(oracle, dims, n, seed=seed_mesh)
    f = oracle.apply_mask(P["mask"], oracle.scatter_unique(*dims, n, inputs.unique_field(*dims, n, seed=seed_f)))
    return P, f


def test_cg_fixed_100_iterations_config1(nek, oracle):
    """4x4x4 elements, n = 8, 100 CG iterations (the paper's run length)."""
    dims, n = (4, 4, 4), 8
    P, f = cg_inputs(oracle, dims, n)
    x_ref, it_ref, rr_ref, hist_ref, st = oracle.cg(*dims, n, P["D"], P["gxyz"], P["mask"], f,
                                                    tol=0.0, maxit=100)
    assert st == 0 and it_ref == 100
    with Ctx(nek, dims, n, P["D"], P["gxyz"]) as ctx:
        x = torch.zeros(P["E"], n ** 3, dtype=torch.float64, device="cuda")
        st, it, rr = nek.nb_cg_solve(ctx, dev(f), x, tol=0.0, maxit=100)
        xg = host(x)
        hist = nek.nb_cg_history(ctx)
    assert it == 100
    assert np.abs(hist - hist_ref).max() / hist_ref.max() <= 1e-8
    assert np.all(np.abs(hist / hist_ref - 1) <= 1e-6)
    assert rel_err(xg, x_ref) <= 1e-8
    assert abs(rr - rr_ref) <= 1e-8 * max(rr_ref, 1e-300) + 1e-14


@pytest.mark.parametrize("dims,n", [((8, 6, 5), 2), ((4, 3, 2), 3), ((1, 1, 3), 7), ((2, 2, 2), 12),
                                    ((2, 1, 1), 16), ((5, 4, 3), 5)])
def test_cg_fixed_iterations_across_n(nek, oracle, dims, n):
    """30 fixed iterations of the two-kernel iteration (head + fused
    assemble/update) against the oracle's CG over the polynomial orders and
    thin meshes (a single element along some directions leaves the edge and
    vertex node ranges empty).  Every mesh has well over 30 unknowns, so the
    iteration never runs into round-off after exact convergence."""
    P, f = cg_inputs(oracle, dims, n, seed_mesh=n, seed_f=n + 1)
    x_ref, it_ref, rr_ref, hist_ref, st = oracle.cg(*dims, n, P["D"], P["gxyz"], P["mask"], f,
                                                    tol=0.0, maxit=30)
    with Ctx(nek, dims, n, P["D"], P["gxyz"]) as ctx:
        x = torch.zeros(P["E"], n ** 3, dtype=torch.float64, device="cuda")
        st, it, rr = nek.nb_cg_solve(ctx, dev(f), x, tol=0.0, maxit=30)
        xg = host(x)
        hist = nek.nb_cg_history(ctx)
    assert it == it_ref
    assert np.abs(hist - hist_ref).max() / hist_ref.max() <= 1e-8
    assert rel_err(xg, x_ref) <= 1e-8


def test_full_size_cg_in_bench_configuration(nek, oracle):
    """E = 4096, n = 10, the benchmark's problem and launch path (device-built
    geometry, graph-captured two-kernel iteration): 20 fixed CG iterations
    against the oracle's CG on the same mesh and right-hand side."""
    dims, n = (16, 16, 16), 10
    s = inputs.perturbation_coeffs(inputs.SEED_MESH)
    P = oracle.box_problem(*dims, n, inputs.PERTURB_AMP, s)
    f = oracle.apply_mask(P["mask"], oracle.scatter_unique(*dims, n, inputs.unique_field(*dims, n, inputs.SEED_F)))
    x_ref, it_ref, rr_ref, hist_ref, st = oracle.cg(*dims, n, P["D"], P["gxyz"], P["mask"], f, tol=0.0, maxit=20)
    with Ctx(nek, dims, n, inputs.PERTURB_AMP, s, box=True) as ctx:
        x = torch.zeros(P["E"], n ** 3, dtype=torch.float64, device="cuda")
        st, it, rr = nek.nb_cg_solve(ctx, dev(f), x, tol=0.0, maxit=20)
        xg = host(x)
        hist = nek.nb_cg_history(ctx)
    assert it == 20 == it_ref
    assert np.abs(hist - hist_ref).max() / hist_ref.max() <= 1e-8
    assert rel_err(xg, x_ref) <= 1e-8


def test_largest_served_size(nek, oracle):
    """The largest problem the served workload draws: 32 x 32 x 32 elements,
    n = 12 (56.6 M local points), device-built geometry.  ax_e on sampled
    elements against the oracle applied to the device's own D and gxyz
    (identical inputs, the 1e-12 relative contract), the device geometry
    against the oracle's (n eps kappa_J), dssum and mask over the whole mesh
    (bit-exact), and two fixed CG iterations of the graph-captured solver
    against the oracle's CG."""
    dims, n = (32, 32, 32), 12
    E = dims[0] * dims[1] * dims[2]
    s = inputs.perturbation_coeffs(inputs.SEED_MESH)
    xi, wq = oracle.gll(n)
    Dm = oracle.dmat(xi)
    xyz = oracle.box_coords(*dims, n, inputs.PERTURB_AMP, s)
    gxyz, _ = oracle.geom(n, xyz, Dm, wq)
    del xyz
    u = inputs.local_field(E, n, seed=inputs.SEED_U)
    rng = np.random.default_rng(7)
    sample = np.unique(np.concatenate([[0, E - 1], rng.choice(E, 64, replace=False)]))
    gs = gxyz[sample]
    msk = oracle.mask(*dims, n)
    f = oracle.apply_mask(msk, oracle.scatter_unique(*dims, n, inputs.unique_field(*dims, n, inputs.SEED_F)))
    x_ref, it_ref, _, hist_ref, _ = oracle.cg(*dims, n, Dm, gxyz, msk, f, tol=0.0, maxit=2)
    del gxyz
    with Ctx(nek, dims, n, inputs.PERTURB_AMP, s, box=True) as ctx:
        Dd = nek.nb_get_operator(ctx, n)
        g = torch.empty(E, 6, n ** 3, dtype=torch.float64, device="cuda")
        nek.nb_get_operator(ctx, n, g)
        gd = host(g[torch.from_numpy(sample).cuda()])
        del g
        ud = dev(u)
        w = torch.empty_like(ud)
        nek.nb_ax(ctx, ud, w)
        got_ax = host(w)[sample]
        wr = inputs.local_field(E, n, seed=11)
        wd = dev(wr)
        nek.nb_dssum(ctx, wd)
        got_ds = host(wd)
        nek.nb_mask(ctx, wd)
        got_m = host(wd)
        del ud, w, wd
        x = torch.zeros(E, n ** 3, dtype=torch.float64, device="cuda")
        st, it, rr = nek.nb_cg_solve(ctx, dev(f), x, tol=0.0, maxit=2)
        xg = host(x)
        hist = nek.nb_cg_history(ctx)
    assert rel_err(got_ax, oracle.ax_e(Dd, gd, u[sample])) <= AX_TOL
    assert rel_err(Dd, Dm) <= 1e-13
    assert np.abs(gd - gs).max() <= geometry_tol(Dm, dims, n) * np.abs(gs).max()
    want_ds = oracle.dssum(*dims, n, wr)
    assert np.array_equal(got_ds, want_ds)
    assert np.array_equal(got_m, oracle.apply_mask(msk, want_ds))
    assert st == nek.NB_OK and it == 2 == it_ref
    assert np.abs(hist - hist_ref).max() / hist_ref.max() <= 1e-10
    assert rel_err(xg, x_ref) <= 1e-10


@pytest.mark.parametrize("dims,n", [((32, 32, 32), 12), ((16, 16, 16), 16)])
def test_ax_full_size_identical_inputs(nek, oracle, dims, n):
    """The 1e-12 relative contract at the largest served degree (n = 12 on
    32^3 elements) and at the largest supported one (n = 16 on 16^3), with
    the oracle's own D and gxyz handed to nb_setup, checked on sampled
    elements of the whole-mesh launch."""
    E = dims[0] * dims[1] * dims[2]
    s = inputs.perturbation_coeffs(inputs.SEED_MESH)
    xi, wq = oracle.gll(n)
    Dm = oracle.dmat(xi)
    xyz = oracle.box_coords(*dims, n, inputs.PERTURB_AMP, s)
    gxyz, _ = oracle.geom(n, xyz, Dm, wq)
    del xyz
    u = inputs.local_field(E, n, seed=inputs.SEED_U + n)
    rng = np.random.default_rng(n)
    sample = np.unique(np.concatenate([[0, E - 1], rng.choice(E, 64, replace=False)]))
    want = oracle.ax_e(Dm, gxyz[sample], u[sample])
    with Ctx(nek, dims, n, Dm, gxyz) as ctx:
        del gxyz
        ud = dev(u)
        w = torch.empty_like(ud)
        nek.nb_ax(ctx, ud, w)
        got = host(w[torch.from_numpy(sample).cuda()])
    assert rel_err(got, want) <= AX_TOL


@pytest.mark.parametrize("k", [-90, 80])
def test_cg_scale_equivariance(nek, oracle, k):
    """Every step of the FP64-accurate CG commutes with scaling by a power of
    two: FP64 operations, the pair scales taken from exponents (per element
    for u, per iteration from <p,p>_c in the CG head) and <r,r>_c on the FP32
    pipes.  So f 2^k must give x 2^k bit for bit, and the same iteration
    history scaled by 2^2k."""
    dims, n = (4, 3, 3), 10
    P, f = cg_inputs(oracle, dims, n, seed_mesh=5, seed_f=6)
    out = []
    with Ctx(nek, dims, n, P["D"], P["gxyz"]) as ctx:
        for scale in (1.0, 2.0 ** k):
            x = torch.zeros(P["E"], n ** 3, dtype=torch.float64, device="cuda")
            st, it, rr = nek.nb_cg_solve(ctx, dev(f * scale), x, tol=0.0, maxit=40)
            out.append((host(x), nek.nb_cg_history(ctx), st, it))
    (x0, h0, s0, i0), (x1, h1, s1, i1) = out
    assert s0 == s1 == nek.NB_OK and i0 == i1 == 40
    assert np.array_equal(x1, x0 * 2.0 ** k)
    assert np.array_equal(h1, h0 * 2.0 ** (2 * k))


def test_cg_tolerance_and_determinism(nek, oracle):
    dims, n = (3, 2, 2), 6
    P, f = cg_inputs(oracle, dims, n, seed_mesh=3, seed_f=4)
    x_ref, it_ref, rr_ref, _, _ = oracle.cg(*dims, n, P["D"], P["gxyz"], P["mask"], f, tol=1e-10, maxit=5000)
    with Ctx(nek, dims, n, P["D"], P["gxyz"]) as ctx:
        outs = []
        for rep in range(2):
            x = torch.zeros(P["E"], n ** 3, dtype=torch.float64, device="cuda")
            st, it, rr = nek.nb_cg_solve(ctx, dev(f), x, tol=1e-10, maxit=5000)
            outs.append((host(x), it, rr, nek.nb_cg_history(ctx)))
    (x0, it0, rr0, h0), (x1, it1, rr1, h1) = outs
    assert np.array_equal(x0, x1) and it0 == it1 and np.array_equal(h0, h1)   # deterministic
    assert rr0 <= 1e-10 and abs(it0 - it_ref) <= 2
    assert rel_err(x0, x_ref) <= 1e-8


def test_cg_graph_and_plain_launch_agree(nek, oracle):
    """The default stream cannot be captured, so it runs plain launches;
    both paths must give bitwise-equal iterates."""
    dims, n = (2, 2, 3), 5
    P, f = cg_inputs(oracle, dims, n)
    res = []
    for stream in (torch.cuda.current_stream(), torch.cuda.default_stream()):
        with torch.cuda.stream(stream):
            h = nek.nb_setup(dims, n, P["D"], P["gxyz"], stream=stream)
            x = torch.zeros(P["E"], n ** 3, dtype=torch.float64, device="cuda")
            nek.nb_cg_solve(h, dev(f), x, tol=0.0, maxit=37)
            stream.synchronize()
            res.append(x.cpu().numpy())
            nek.nb_destroy(h)
    assert np.array_equal(res[0], res[1])


def test_cg_edge_cases(nek, oracle):
    dims, n = (2, 2, 2), 4
    P, f = cg_inputs(oracle, dims, n)
    E = P["E"]
    with Ctx(nek, dims, n, P["D"], P["gxyz"]) as ctx:
        x = torch.zeros(E, n ** 3, dtype=torch.float64, device="cuda")
        st, it, rr = nek.nb_cg_solve(ctx, dev(f), x, tol=0.0, maxit=0)
        assert it == 0 and torch.count_nonzero(x) == 0 and abs(rr - 1.0) < 1e-15
        st, it, rr = nek.nb_cg_solve(ctx, torch.zeros_like(x), x, tol=1e-8, maxit=10)
        assert it == 0 and rr == 0.0
        st, it, rr = nek.nb_cg_solve(ctx, dev(f), x, tol=1e-15, maxit=3, allow=(nek.NB_ERR_NOT_CONVERGED,))
        assert st == nek.NB_ERR_NOT_CONVERGED and it == 3
    # a negative-definite operator makes <Ap,p>_c < 0 in the first iteration
    with Ctx(nek, dims, n, P["D"], -P["gxyz"]) as ctx:
        x = torch.zeros(E, n ** 3, dtype=torch.float64, device="cuda")
        st, it, rr = nek.nb_cg_solve(ctx, dev(f), x, tol=0.0, maxit=10, allow=(nek.NB_ERR_BREAKDOWN,))
        assert st == nek.NB_ERR_BREAKDOWN and it == 0 and torch.count_nonzero(x) == 0


def test_cg_manufactured_solution(nek, oracle):
    dims, n = (2, 2, 2), 7
    P = oracle_problem(oracle, dims, n, seed=1)
    xyz = P["xyz"]
    us = np.sin(np.pi * xyz[:, 0]) * np.sin(np.pi * xyz[:, 1]) * np.sin(np.pi * xyz[:, 2])
    us = oracle.apply_mask(P["mask"], us)
    f = oracle.apply_A(*dims, n, P["D"], P["gxyz"], P["mask"], us)
    with Ctx(nek, dims, n, P["D"], P["gxyz"]) as ctx:
        x = torch.zeros_like(dev(f))
        st, it, rr = nek.nb_cg_solve(ctx, dev(f), x, tol=1e-12, maxit=3000)
        assert rr <= 1e-12
        assert np.abs(host(x) - us).max() < 1e-8


def test_cg_host_buffers_and_timing(nek, oracle):
    dims, n = (3, 3, 2), 6
    P, f = cg_inputs(oracle, dims, n)
    with Ctx(nek, dims, n, P["D"], P["gxyz"]) as ctx:
        x = torch.zeros(P["E"], n ** 3, dtype=torch.float64, device="cuda")
        nek.nb_cg_solve(ctx, dev(f), x, tol=0.0, maxit=20)
        xd = host(x)
        xh = np.zeros_like(f)
        nek.nb_timing_enable(ctx, True)
        st, it, rr = nek.nb_cg_solve_host(ctx, np.ascontiguousarray(f), xh, tol=0.0, maxit=20)
        ms, cnt = nek.nb_timing_read(ctx, nek.NB_K_AX)
        nek.nb_timing_enable(ctx, False)
    assert it == 20 and np.array_equal(xh, xd)
    assert cnt == 21 and ms > 0          # 20 iterations + the initial residual


def test_sampled_timing_keeps_the_solve_and_counts_launches(nek, oracle):
    """Sampled timing (nb_timing_enable(ctx, 2)) keeps the FP64 CG's graphs
    and event-times the first iteration of each chunk of 16: the solution and
    the rho history are bit-identical to an untimed solve, the timed launches
    are one iteration per chunk plus the once-per-solve kernels, and
    nb_launch_count counts every kernel, graph kernels included.  With every
    launch timed (1) the solve runs exactly maxit iterations of plain launches."""
    dims, n = (4, 3, 3), 10          # n = 10: the two-kernel iteration (head + assemble_update)
    P, f = cg_inputs(oracle, dims, n)
    maxit = 40                       # three chunks of 16 are launched; the last 8 iterations return at once
    with Ctx(nek, dims, n, P["D"], P["gxyz"]) as ctx:
        runs = {}
        for mode in (0, 2, 1):
            nek.nb_timing_enable(ctx, mode)
            x = torch.zeros_like(dev(f))
            st, it, rr = nek.nb_cg_solve(ctx, dev(f), x, tol=0.0, maxit=maxit)
            timed = {k: nek.nb_timing_read(ctx, k)[1] for k in range(nek.NB_K_COUNT)}
            runs[mode] = (host(x), nek.nb_cg_history(ctx), it, timed, nek.nb_launch_count(ctx))
        nek.nb_timing_enable(ctx, 0)
        with pytest.raises(nek.NekgbError) as ei:
            nek.nb_timing_enable(ctx, 3)
        assert ei.value.status == nek.NB_ERR_ARG
    x0, h0, it0, _, _ = runs[0]
    for mode in (1, 2):
        xm, hm, itm, _, _ = runs[mode]
        assert itm == it0 == maxit and np.array_equal(xm, x0) and np.array_equal(hm, h0)
    # setup: ax_e (w = A x0), dssum, mask, dot; then the iterations; then final x (other)
    _, _, _, t2, n2 = runs[2]
    chunks = -(-maxit // 16)
    assert n2 == 4 + 2 * 16 * chunks + 1
    assert t2[nek.NB_K_AX] == 1 + chunks and t2[nek.NB_K_UPDATE] == chunks
    assert t2[nek.NB_K_DSSUM] == 1 and t2[nek.NB_K_MASK] == 1 and t2[nek.NB_K_DOT] == 1
    assert t2[nek.NB_K_OTHER] == 1
    _, _, _, t1, n1 = runs[1]
    assert n1 == 4 + 2 * maxit + 1 == sum(t1.values())
    assert t1[nek.NB_K_AX] == 1 + maxit and t1[nek.NB_K_UPDATE] == maxit


def test_argument_errors_on_device(nek):
    dims, n = (2, 2, 2), 4
    with Ctx(nek, dims, n, np.eye(n), np.zeros((8, 6, n ** 3))) as ctx:
        u = torch.zeros(8 * n ** 3 + 1, dtype=torch.float64, device="cuda")
        with pytest.raises(nek.NekgbError) as ei:
            nek.nb_ax(ctx, u, u)
        assert ei.value.status == nek.NB_ERR_ARG
        with pytest.raises(nek.NekgbError):
            nek.nb_ax(ctx, u.data_ptr() + 4, u.data_ptr() + 8 * 4096)
