"""Pins for the FP64 CPU oracle: closed forms, invariants and brute force.

Each test ties the oracle to something other than itself, chosen so that a
plausible slip (a dropped term, a wrong sign or normal direction, a swapped
index, a transposed operand, a wrong quadrature weight) fails at least one:

* quadrature: exact integrals of monomials (degree <= 5) and the published
  table of the rule (tests/golden/stroud_t2_5_1.txt);
* K' on a sphere: K' 1 -> -1/2 and K' Y_1 -> -1/6 Y_1 (eigenvalues
  -1/(2(2l+1)) of the interior-limit operator), which fixes sign and scale;
* Born ion (Sec. 2.1 model, one central charge): closed form energy;
* Kirkwood series for off-centre charges (full solve) and its BIBEE
  counterparts (Eq. CFA, lambda = -1/2 and 0), with the ordering
  dG_P <= dG <= dG_CFA (CFA is an upper bound, Sec. 2.2);
* Gauss's law for the total induced charge;
* GMRES against dense LU (numpy.linalg.solve) on the assembled matrix;
* adjoint: dot-product identities for K'^T, B^T, C^T and central finite
  differences of the energy in the charge values and positions;
* rigid-motion invariance of the energy;
* exact flat-panel integrals: the normal field by closed-surface solid
  angles, refined quadrature and its unit jump; the single-layer potential by
  the equilateral centroid closed form, a polar integral on the panel's axis,
  refined quadrature, finite differences of its gradient, the jump of its
  normal derivative, and the uniform-shell potential R inside a sphere for
  charges just under the surface;
* the Galerkin form's transposes by dot-product identities and entry by
  entry, its adjoint gradients by central differences and q.(d dG/dq) = 2 dG.
"""
import os

import numpy as np
import pytest

import oracle
import synth
import sphere_series as ss

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def small3():
    m = synth.small_molecule(3)
    return m, oracle.Problem(m.panels, m.charges, m.eps_in, m.eps_out)


@pytest.fixture(scope="module")
def small4():
    m = synth.small_molecule(4)
    return m, oracle.Problem(m.panels, m.charges, m.eps_in, m.eps_out)


# ---------------------------------------------------------------- quadrature
def test_quad_rule_matches_published_table():
    rows = np.loadtxt(os.path.join(GOLDEN, "stroud_t2_5_1.txt"))
    bary, w = oracle.quad_rule(7)
    np.testing.assert_allclose(bary, rows[:, :3], atol=2e-15)
    np.testing.assert_allclose(w, rows[:, 3], atol=2e-15)
    assert abs(w.sum() - 1.0) < 1e-15


def _monomial_integral_ref(a, b):
    # int over {x>=0, y>=0, x+y<=1} of x^a y^b = a! b! / (a+b+2)!
    from math import factorial
    return factorial(a) * factorial(b) / factorial(a + b + 2)


@pytest.mark.parametrize("nq,degree", [(7, 5), (1, 1)])
def test_quad_rule_polynomial_exactness(nq, degree):
    # reference triangle embedded in z = 0, counter-clockwise seen from +z
    tri = np.array([[[0.0, 0.0, 0.0], [1.0, 0.0, 0.0], [0.0, 1.0, 0.0]]])
    P = oracle.Problem(tri, np.array([[0.3, 0.3, -1.0, 1.0]]), 1.0, 80.0, nq=nq)
    assert abs(P.area[0] - 0.5) < 1e-15
    np.testing.assert_allclose(P.nrm[0], [0.0, 0.0, 1.0], atol=1e-15)
    y = P.qp[0]
    for a in range(degree + 1):
        for b in range(degree + 1 - a):
            got = float(np.sum(P.qw[0] * y[:, 0] ** a * y[:, 1] ** b))
            assert abs(got - _monomial_integral_ref(a, b)) < 1e-14, (a, b)
    if nq == 7:
        # not exact one degree higher (so the table is not a higher-order rule)
        got = float(np.sum(P.qw[0] * y[:, 0] ** 6))
        assert abs(got - _monomial_integral_ref(6, 0)) > 1e-6


def test_quad_rule_exact_on_skewed_triangle():
    rng = np.random.default_rng(11)
    v = rng.normal(size=(3, 3))
    tri = v[None]
    P = oracle.Problem(tri, np.array([[9.0, 9.0, 9.0, 1.0]]), 1.0, 80.0)
    # barycentric monomials: int l1^a l2^b l3^c dA = 2 A a! b! c! / (a+b+c+2)!
    from math import factorial
    bary, _ = oracle.quad_rule(7)
    for a in range(6):
        for b in range(6 - a):
            for c in range(6 - a - b):
                exact = 2 * P.area[0] * factorial(a) * factorial(b) * factorial(c) / factorial(a + b + c + 2)
                got = float(np.sum(P.qw[0] * bary[:, 0] ** a * bary[:, 1] ** b * bary[:, 2] ** c))
                assert abs(got - exact) < 1e-13 * max(1.0, abs(exact))
    # the quadrature points really are those barycentric combinations
    np.testing.assert_allclose(P.qp[0], bary @ v, atol=1e-14)


def test_geometry_outward_and_area():
    m = synth.born(4)
    P = oracle.Problem(m.panels, m.charges, 1.0, 80.0)
    assert np.all(np.einsum("ij,ij->i", P.nrm, P.cen) > 0)  # normals point into the solvent
    np.testing.assert_allclose(np.linalg.norm(P.nrm, axis=1), 1.0, atol=1e-14)
    # inscribed polyhedron: area below, and close to, 4 pi R^2
    tot = P.area.sum()
    assert 0.99 * 4 * np.pi * 4.0 < tot < 4 * np.pi * 4.0


def test_degenerate_panel_rejected():
    tri = np.zeros((1, 3, 3))
    with pytest.raises(ValueError):
        oracle.Problem(tri, np.array([[0.0, 0.0, 1.0, 1.0]]), 1.0, 80.0)


# -------------------------------------------------------------- K' on a sphere
def test_kprime_sphere_eigenvalues(small3, small4):
    e0, e1 = [], []
    for m, P in (small3, small4):
        k1 = P.kprime(np.ones(P.n))
        e0.append(abs(k1.mean() + 0.5))          # eigenvalue -1/2 for l = 0
        z = P.cen[:, 2] / np.linalg.norm(P.cen, axis=1)
        kz = P.kprime(z)
        lam = float(kz @ z / (z @ z))            # eigenvalue -1/6 for l = 1
        e1.append(abs(lam + 1.0 / 6.0))
        assert np.linalg.norm(kz - lam * z) / np.linalg.norm(kz) < 0.05
    # first-order convergence (the fixed rule on near-singular neighbours)
    assert e0[1] < 0.015 and e0[1] < 0.6 * e0[0]
    assert e1[1] < 0.015 and e1[1] < 0.6 * e1[0]


def test_kprime_self_term_vanishes_on_flat_panel():
    # (c_i - y) . n_i = 0 for every y on a flat panel: refining the panel into
    # sub-triangles and summing the interior-limit-free contributions gives 0.
    tri = np.array([[0.0, 0.0, 0.0], [1.0, 0.1, 0.0], [0.2, 0.9, 0.0]])
    c = tri.mean(0)
    # the three corner children of the panel are coplanar with it: the
    # collocation point's kernel vanishes on each of them identically
    mids = [(tri[0] + tri[1]) / 2, (tri[1] + tri[2]) / 2, (tri[2] + tri[0]) / 2]
    kids = np.array([[tri[0], mids[0], mids[2]], [tri[1], mids[1], mids[0]],
                     [tri[2], mids[2], mids[1]]])
    P = oracle.Problem(np.concatenate([tri[None], kids]), np.array([[0, 0, 5.0, 1.0]]), 1, 80)
    K = P.kprime_dense()
    assert np.all(np.abs(K[0, 1:]) < 1e-14)
    assert K[0, 0] == 0.0


# ---------------------------------------------------------------- Born ion
def test_born_energy_converges_to_closed_form():
    exact = ss.born_energy(1.0, 2.0, 1.0, 80.0)
    assert abs(exact - (-81.97822593750)) < 1e-9
    errs = []
    for s in (2, 3, 4):
        m = synth.born(s)
        P = oracle.Problem(m.panels, m.charges, m.eps_in, m.eps_out)
        sig, info = P.solve(tol=1e-12)
        assert info["converged"]
        dg, _ = P.energy(sig)
        errs.append(abs(dg - exact) / abs(exact))
        # BIBEE/CFA is exact for a central charge (uniform normal field)
        _, dcfa = P.bibee("cfa")
        assert abs(dcfa - exact) / abs(exact) < 0.04 / 4 ** (s - 2)
    assert errs[0] < 0.07 and errs[1] < 0.03 and errs[2] < 0.015
    assert errs[1] / errs[0] < 0.6 and errs[2] / errs[1] < 0.6


def test_series_reduce_to_born():
    ch = np.array([[0.0, 0.0, 0.0, 1.3]])
    b = ss.born_energy(1.3, 5.0, 4.0, 80.0)
    for kind in ("full", "cfa"):
        assert abs(ss.sphere_energy(ch, 5.0, 4.0, 80.0, kind) - b) < 1e-12 * abs(b)


# ------------------------------------------------ Kirkwood and BIBEE series
def test_kirkwood_and_bibee_series(small3, small4):
    res = {}
    for tag, (m, P) in (("s3", small3), ("s4", small4)):
        sig, info = P.solve(tol=1e-11)
        assert info["converged"]
        dg, _ = P.energy(sig)
        _, dc = P.bibee("cfa")
        _, dp = P.bibee("p")
        ex = ss.sphere_energy(m.charges, m.radius, m.eps_in, m.eps_out, "full")
        exc = ss.sphere_energy(m.charges, m.radius, m.eps_in, m.eps_out, "cfa")
        exp_ = ss.sphere_energy(m.charges, m.radius, m.eps_in, m.eps_out, "p")
        res[tag] = (abs(dg - ex) / abs(ex), abs(dc - exc) / abs(exc), abs(dp - exp_) / abs(exp_))
        # ordering of the approximations (CFA upper bound, Sec. 2.2)
        assert dp < dg < dc
        assert exp_ < ex < exc
    assert res["s4"][0] < 0.025 and res["s4"][0] < 0.6 * res["s3"][0]
    assert res["s4"][1] < 0.004 and res["s4"][1] < 0.35 * res["s3"][1]
    assert res["s4"][2] < 0.004 and res["s4"][2] < 0.35 * res["s3"][2]


def test_bibee_lambda_variants_closed_form():
    e_in, e_out = 4.0, 80.0
    # lambda = -1/2: sigma_hat = (1 - eps_in/eps_out) E_n
    assert abs(oracle.bibee_factor(e_in, e_out, -0.5) - (1 - e_in / e_out)) < 1e-15
    # lambda = +1/2: sigma_hat = (eps_out - eps_in)/eps_in E_n
    assert abs(oracle.bibee_factor(e_in, e_out, 0.5) - (e_out - e_in) / e_in) < 1e-13


def test_gauss_law_total_induced_charge(small3, small4):
    errs = []
    for m, P in (small3, small4):
        sig, _ = P.solve(tol=1e-11)
        total = float(P.area @ sig)
        expect = -(1.0 - m.eps_in / m.eps_out) * m.charges[:, 3].sum()
        errs.append(abs(total - expect) / abs(expect))
    assert errs[1] < 0.02 and errs[1] < 0.6 * errs[0]


# --------------------------------------------------------------- GMRES vs LU
def test_gmres_matches_dense_lu():
    m = synth.small_molecule(3)
    P = oracle.Problem(m.panels, m.charges, m.eps_in, m.eps_out)
    A = np.eye(P.n) + P.ehat * P.kprime_dense()
    b = P.rhs()
    x_lu = np.linalg.solve(A, b)
    x, info = P.solve(tol=1e-12, restart=10)   # small restart exercises restarts
    assert info["converged"] and info["true_resid"] < 1e-11
    assert np.linalg.norm(x - x_lu) / np.linalg.norm(x_lu) < 1e-10
    # dense operator agrees with the matrix-free one
    v = np.random.default_rng(3).normal(size=P.n)
    np.testing.assert_allclose(A @ v, P.A(v), rtol=1e-12, atol=1e-12)


def test_gmres_textbook_on_known_system():
    rng = np.random.default_rng(0)
    n = 60
    M = np.eye(n) + 0.3 * rng.normal(size=(n, n)) / np.sqrt(n)
    b = rng.normal(size=n)
    x, info = oracle.gmres(lambda v: M @ v, b, tol=1e-13, restart=7, maxiter=2000)
    assert info["converged"]
    np.testing.assert_allclose(x, np.linalg.solve(M, b), rtol=1e-10, atol=1e-11)


# ---------------------------------------------------------------- adjoint
def test_transposes_by_dot_products(small3):
    m, P = small3
    rng = np.random.default_rng(5)
    x, y = rng.normal(size=P.n), rng.normal(size=P.n)
    assert abs(P.kprime(x) @ y - x @ P.kprime_t(y)) < 1e-12 * np.abs(P.kprime(x)).sum() * np.abs(y).max()
    K = P.kprime_dense()
    np.testing.assert_allclose(K @ x, P.kprime(x), rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(K.T @ y, P.kprime_t(y), rtol=1e-12, atol=1e-14)
    q, v = rng.normal(size=P.nc), rng.normal(size=P.n)
    assert abs(P.bq(q) @ v - q @ P.bt(v)) < 1e-12 * np.linalg.norm(P.bq(q)) * np.linalg.norm(v)
    s, u = rng.normal(size=P.n), rng.normal(size=P.nc)
    assert abs(P.c(s) @ u - s @ P.ct(u)) < 1e-12 * np.linalg.norm(P.c(s)) * np.linalg.norm(u)


def _energy_at(m, charges, tol=1e-13):
    P = oracle.Problem(m.panels, charges, m.eps_in, m.eps_out)
    sig, _ = P.solve(tol=tol, maxiter=2000)
    return P.energy(sig)[0]


def test_adjoint_gradients_match_central_differences():
    m = synth.small_molecule(2, n_charges=12)
    P = oracle.Problem(m.panels, m.charges, m.eps_in, m.eps_out)
    dg, dq, dx, _, _ = P.gradients(tol=1e-13)
    hq, hx = 1e-4, 1e-4
    for k in range(0, P.nc, 3):
        cp, cm = m.charges.copy(), m.charges.copy()
        cp[k, 3] += hq
        cm[k, 3] -= hq
        fd = (_energy_at(m, cp) - _energy_at(m, cm)) / (2 * hq)
        assert abs(fd - dq[k]) < 1e-7 * max(1.0, abs(dq[k])), (k, fd, dq[k])
        for d in range(3):
            cp, cm = m.charges.copy(), m.charges.copy()
            cp[k, d] += hx
            cm[k, d] -= hx
            fd = (_energy_at(m, cp) - _energy_at(m, cm)) / (2 * hx)
            assert abs(fd - dx[k, d]) < 1e-6 * max(1.0, np.abs(dx).max()), (k, d, fd, dx[k, d])


def test_energy_quadratic_in_charges(small3):
    # dG(q) = 1/2 q^T R q  =>  q . d dG/dq = 2 dG
    m, P = small3
    dg, dq, _, _, _ = P.gradients(tol=1e-13)
    assert abs(float(P.q @ dq) - 2.0 * dg) < 1e-9 * abs(dg)


# --------------------------------------------------------------- invariance
def test_energy_invariant_under_rigid_motion():
    m = synth.small_molecule(3)
    e0 = _energy_at(m, m.charges, tol=1e-12)
    R = synth.random_rotation(np.random.default_rng(9))
    t = np.array([3.0, -7.5, 12.25])
    pan = m.panels @ R.T + t
    ch = m.charges.copy()
    ch[:, :3] = ch[:, :3] @ R.T + t
    P = oracle.Problem(pan, ch, m.eps_in, m.eps_out)
    sig, _ = P.solve(tol=1e-12)
    e1 = P.energy(sig)[0]
    assert abs(e1 - e0) < 1e-9 * abs(e0)


def test_one_point_rule_variant_runs_and_converges():
    # the paper's centroid rule (Sec. 2.1): same model, coarser panel integrals
    m = synth.born(3)
    P = oracle.Problem(m.panels, m.charges, m.eps_in, m.eps_out, nq=1)
    sig, info = P.solve(tol=1e-10)
    assert info["converged"]
    dg, _ = P.energy(sig)
    assert abs(dg - ss.born_energy(1.0, 2.0, 1.0, 80.0)) / 81.978 < 0.05


# ------------------------------------------- exact flat-panel integrals
# The exact integral over a flat triangle of the normal field of a unit
# density (solid-angle term plus edge logarithms), used for the near-singular
# pairs in the higher-accuracy variant of the operator.
def _refined_7pt(t, n, tri, levels):
    import ctypes
    bary = np.zeros(21)
    w = np.zeros(7)
    oracle._load().oracle_quad_rule(7, bary.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                    w.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    bary = bary.reshape(7, 3)
    tris = [np.asarray(tri, dtype=np.float64)]
    for _ in range(levels):
        nxt = []
        for a, b, c in tris:
            ab, bc, ca = (a + b) / 2, (b + c) / 2, (c + a) / 2
            nxt += [np.array([a, ab, ca]), np.array([ab, b, bc]), np.array([ca, bc, c]),
                    np.array([ab, bc, ca])]
        tris = nxt
    acc = 0.0
    for tt in tris:
        A = 0.5 * np.linalg.norm(np.cross(tt[1] - tt[0], tt[2] - tt[0]))
        y = bary @ tt
        d = np.asarray(t) - y
        r = np.linalg.norm(d, axis=1)
        acc += float(np.sum(A * w * (-(d @ np.asarray(n))) / (4 * np.pi * r ** 3)))
    return acc


def test_solid_angles_of_a_closed_surface():
    pan = synth.icosphere(2, 1.0)
    inside = sum(oracle.solid_angle([0.1, 0.2, -0.3], p) for p in pan)
    outside = sum(oracle.solid_angle([2.0, 0.5, 0.1], p) for p in pan)
    assert abs(inside + 4 * np.pi) < 1e-10          # outward normals: -4 pi inside
    assert abs(outside) < 1e-10


def test_exact_panel_integral_matches_refined_quadrature():
    tri = np.array([[0.0, 0.0, 0.0], [1.0, 0.0, 0.0], [0.2, 0.9, 0.1]])
    n = np.array([0.2, -0.3, 0.93])
    n /= np.linalg.norm(n)
    # above the panel, and beyond the extension of an edge (the other log form)
    for t in ([0.3, 0.4, 0.35], [-0.7, 0.0, 0.05]):
        ex = oracle.panel_dn(t, n, tri)
        assert abs(_refined_7pt(t, n, tri, 5) - ex) < 1e-9 * max(1.0, abs(ex)), (t, ex)
        assert abs(_refined_7pt(t, n, tri, 0) - ex) > 1e-12   # the unrefined rule is not exact


def test_exact_panel_integral_jumps_by_one_across_the_sheet():
    # the normal field of a unit sheet density (G = 1/(4 pi r)) jumps by 1:
    # -1/2 just on the side the normal points to, +1/2 just behind
    tri = np.array([[0.0, 0.0, 0.0], [1.0, 0.0, 0.0], [0.0, 1.0, 0.0]])
    nu = np.array([0.0, 0.0, 1.0])
    c = tri.mean(axis=0)
    assert abs(oracle.panel_dn(c + 1e-9 * nu, nu, tri) + 0.5) < 1e-7
    assert abs(oracle.panel_dn(c - 1e-9 * nu, nu, tri) - 0.5) < 1e-7


def test_near_exact_rows_approach_the_exact_flat_panel_operator():
    # against K' integrated exactly for every pair, the 7-point rule errs at
    # the near-singular pairs; the near-exact variant keeps only the small
    # far-pair quadrature error
    pan = synth.icosphere(2, 1.0)
    P = oracle.Problem(pan, np.zeros((0, 4)), 1.0, 80.0)
    rng = np.random.default_rng(0)
    x = rng.standard_normal(P.n)
    rows = rng.choice(P.n, 40, replace=False)
    full = np.array([sum(oracle.panel_dn(P.cen[i], P.nrm[i], pan[j]) * x[j]
                         for j in range(P.n) if j != i) for i in rows])
    e_quad = np.linalg.norm(P.kprime_rows(x, rows) - full) / np.linalg.norm(full)
    e_near = np.linalg.norm(P.kprime_rows_near_exact(x, rows) - full) / np.linalg.norm(full)
    assert e_near < 3e-5 and e_quad > 1e-3, (e_near, e_quad)


# ------------------------------------------------------------- Galerkin
# Rows averaged over each panel by the rule, near-singular inner integrals
# exact (the Galerkin form of Sec. 2.1 with piecewise-constant functions).
def test_galerkin_with_one_point_rule_is_collocation():
    m = synth.small_molecule(2)
    P = oracle.Problem(m.panels, m.charges, m.eps_in, m.eps_out, nq=1)
    x = np.random.default_rng(0).standard_normal(P.n)
    rows = np.arange(P.n)
    a = P.kprime_rows_galerkin(x, rows)
    b = P.kprime_rows_near_exact(x, rows)
    assert np.abs(a - b).max() < 1e-12 * np.abs(b).max()


def test_galerkin_born_energy_and_gauss_law():
    # more accurate than collocation on the same mesh: the Born energy within
    # 1 % (collocation 2.8 %) and the total induced charge within 4e-3 of
    # -(1 - 1/eps_out) (collocation 2.4e-2) at 1,280 panels
    m = synth.born(3)
    P = oracle.Problem(m.panels, m.charges, m.eps_in, m.eps_out)
    born = ss.born_energy(1.0, 2.0, 1.0, 80.0)
    sg, info = P.solve_galerkin(tol=1e-11)
    assert info["converged"]
    eg = P.energy(sg)[0]
    sc, _ = P.solve(tol=1e-11)
    ec = P.energy(sc)[0]
    assert abs(eg - born) < 0.01 * abs(born)
    assert abs(eg - born) < 0.3 * abs(ec - born)
    gauss = 1.0 - 1.0 / 80.0
    assert abs((sg * P.area).sum() + gauss) < 4e-3
    assert abs((sg * P.area).sum() + gauss) < 0.2 * abs((sc * P.area).sum() + gauss)


# ------------------------------------------- sampled rows and arbitrary points
def test_normal_field_is_the_normal_derivative_of_the_potential():
    """oracle.normal_field(t, n, charges) = n . grad phi(t) with phi the
    Coulomb potential sum_k q_k / (4 pi |t - x_k|), checked by a central
    difference of that potential along n (computed here from its own
    definition, independent of the field's formula); a wrong sign, a missing
    4 pi or a swapped (t - x) fails."""
    rng = np.random.default_rng(11)
    ch = np.column_stack([rng.uniform(-2, 2, (30, 3)), rng.uniform(-1, 1, 30)])
    t = rng.uniform(3, 6, (50, 3)) * rng.choice([-1, 1], (50, 3))
    n = rng.standard_normal((50, 3))
    n /= np.linalg.norm(n, axis=1, keepdims=True)

    def phi(pts):
        d = np.linalg.norm(pts[:, None, :] - ch[None, :, :3], axis=2)
        return (ch[None, :, 3] / (4 * np.pi * d)).sum(axis=1)
    h = 1e-5
    fd = (phi(t + h * n) - phi(t - h * n)) / (2 * h)
    E = oracle.normal_field(t, n, ch)
    np.testing.assert_allclose(E, fd, rtol=1e-7, atol=1e-12)


def test_normal_field_of_a_central_charge_on_a_sphere():
    """A charge q at the centre of a sphere of radius R: at every point of the
    sphere the outward normal derivative of its potential is -q / (4 pi R^2)."""
    rng = np.random.default_rng(12)
    n = rng.standard_normal((40, 3))
    n /= np.linalg.norm(n, axis=1, keepdims=True)
    R, q = 3.0, -1.7
    E = oracle.normal_field(R * n, n, np.array([[0.0, 0.0, 0.0, q]]))
    np.testing.assert_allclose(E, -q / (4 * np.pi * R * R), rtol=1e-14)


def test_sampled_rows_match_the_full_products(small3):
    """bq_rows / c_rows are the full products restricted to a subset."""
    m, P = small3
    rows = np.random.default_rng(13).choice(m.n_p, 37, replace=False)
    np.testing.assert_array_equal(P.bq_rows(rows), P.bq()[rows])
    s = np.random.default_rng(14).standard_normal(m.n_p)
    ks = np.random.default_rng(15).choice(m.n_c, 9, replace=False)
    np.testing.assert_array_equal(P.c_rows(s, ks), P.c(s)[ks])
    np.testing.assert_array_equal(oracle.normal_field(P.cen, P.nrm, m.charges), P.bq())


# ------------------------------- exact single-layer integrals over a panel
# int_T dA / (4 pi |t - y|) over a flat triangle and its gradient, used for
# the charge-panel pairs closer than 2.5 sqrt(A_j) in the higher-accuracy
# charge products (C, C^T, grad C).
def _refined_7pt_phi(t, tri, levels):
    import ctypes
    bary = np.zeros(21)
    w = np.zeros(7)
    oracle._load().oracle_quad_rule(7, bary.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                    w.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    bary = bary.reshape(7, 3)
    tris = [np.asarray(tri, dtype=np.float64)]
    for _ in range(levels):
        nxt = []
        for a, b, c in tris:
            ab, bc, ca = (a + b) / 2, (b + c) / 2, (c + a) / 2
            nxt += [np.array([a, ab, ca]), np.array([ab, b, bc]), np.array([ca, bc, c]),
                    np.array([ab, bc, ca])]
        tris = nxt
    acc = 0.0
    for tt in tris:
        A = 0.5 * np.linalg.norm(np.cross(tt[1] - tt[0], tt[2] - tt[0]))
        r = np.linalg.norm(np.asarray(t) - bary @ tt, axis=1)
        acc += float(np.sum(A * w / (4 * np.pi * r)))
    return acc


def _equilateral(a=1.0):
    return np.array([[0.0, 0.0, 0.0], [a, 0.0, 0.0], [a / 2, a * np.sqrt(3) / 2, 0.0]])


def test_single_layer_at_the_centroid_of_an_equilateral_triangle():
    # in polar coordinates about the centroid each edge (inradius r) gives
    # r * 2 asinh(sqrt 3): int_T dA / R = sqrt(3) a ln(2 + sqrt 3)
    for a in (1.0, 0.37, 2.5):
        tri = _equilateral(a)
        ex = np.sqrt(3) * a * np.log(2 + np.sqrt(3)) / (4 * np.pi)
        assert abs(oracle.panel_phi(tri.mean(axis=0), tri) - ex) < 1e-14 * max(1.0, ex)


def test_single_layer_on_the_axis_of_an_equilateral_triangle():
    # t at height h above the centroid: int_T dA / R =
    # 3 int_{-pi/3}^{pi/3} (sqrt(r^2 sec^2 th + h^2) - |h|) dth, r the inradius
    from scipy.integrate import quad
    a = 1.3
    tri = _equilateral(a)
    r = a / (2 * np.sqrt(3))
    for h in (1e-4, 0.03, 0.5, 3.0, -0.2):
        f = lambda th: np.sqrt((r / np.cos(th)) ** 2 + h * h) - abs(h)
        ref = 3 * quad(f, -np.pi / 3, np.pi / 3, epsabs=1e-14, epsrel=1e-13, limit=200)[0] / (4 * np.pi)
        got = oracle.panel_phi(tri.mean(axis=0) + np.array([0.0, 0.0, h]), tri)
        assert abs(got - ref) < 1e-13, (h, got, ref)


def test_single_layer_matches_refined_quadrature():
    tri = np.array([[0.0, 0.0, 0.0], [1.0, 0.0, 0.0], [0.2, 0.9, 0.1]])
    # above the panel, behind it, in its plane beyond an edge and beyond a vertex
    for t in ([0.3, 0.4, 0.35], [0.5, 0.2, -0.4], [-0.7, 0.0, 0.0], [1.6, -0.5, 0.05]):
        ex = oracle.panel_phi(t, tri)
        assert abs(_refined_7pt_phi(t, tri, 5) - ex) < 1e-10 * abs(ex), (t, ex)
        assert abs(_refined_7pt_phi(t, tri, 0) - ex) > 1e-12   # the unrefined rule is not exact


def test_single_layer_gradient_is_the_derivative_of_the_potential():
    tri = np.array([[0.0, 0.0, 0.0], [1.0, 0.0, 0.0], [0.2, 0.9, 0.1]])
    eps = 1e-5
    for t in ([0.3, 0.4, 0.35], [0.4, 0.3, -0.02], [-0.7, 0.1, 0.05]):
        t = np.array(t)
        g = oracle.panel_grad_phi(t, tri)
        fd = np.array([(oracle.panel_phi(t + eps * e, tri) - oracle.panel_phi(t - eps * e, tri)) / (2 * eps)
                       for e in np.eye(3)])
        assert np.max(np.abs(g - fd)) < 1e-8 * max(1.0, np.max(np.abs(g))), (t, g, fd)


def test_single_layer_is_continuous_and_its_normal_derivative_jumps_by_one():
    # a unit sheet density: the potential is continuous through the panel and
    # its normal derivative drops by 1 from behind to the side the normal
    # points to; the tangential derivatives are continuous
    tri = np.array([[0.0, 0.0, 0.0], [1.0, 0.0, 0.0], [0.0, 1.0, 0.0]])
    nu = np.array([0.0, 0.0, 1.0])
    c = np.array([0.3, 0.25, 0.0])
    p_up, p_dn = oracle.panel_phi(c + 1e-9 * nu, tri), oracle.panel_phi(c - 1e-9 * nu, tri)
    assert abs(p_up - p_dn) < 1e-12
    g_up, g_dn = oracle.panel_grad_phi(c + 1e-9 * nu, tri), oracle.panel_grad_phi(c - 1e-9 * nu, tri)
    assert abs((g_up - g_dn) @ nu + 1.0) < 1e-7
    assert np.max(np.abs((g_up - g_dn)[:2])) < 1e-7


def _shell_problem(depth):
    # a uniform unit density on a sphere of radius R has potential R at every
    # interior point; charges just under three panel centroids and one deep
    m = synth.born(4, radius=2.0)
    P0 = oracle.Problem(m.panels, m.charges, m.eps_in, m.eps_out)
    ks = [0, 300, 2000]
    pts = [P0.cen[k] - depth * P0.nrm[k] for k in ks] + [[0.1, -0.2, 0.3]]
    ch = np.array([[*p, 1.0] for p in pts])
    return (oracle.Problem(m.panels, ch, m.eps_in, m.eps_out),
            oracle.Problem(m.panels, ch, m.eps_in, m.eps_out, exact_charge_near=True))


def test_exact_charge_near_pairs_recover_the_shell_potential():
    R = 2.0
    Pq, Pe = _shell_problem(0.01)
    one = np.ones(Pq.n)
    phi_q, phi_e = Pq.c(one), Pe.c(one)
    # the flat inscribed mesh (panel edge ~0.1 A) gives R to ~5e-4 everywhere
    # inside; the 7-point rule 0.01 A under a panel errs several times more
    assert np.max(np.abs(phi_e / R - 1)) < 1e-3, phi_e
    assert np.min(np.abs(phi_q[:3] / R - 1)) > 5 * np.max(np.abs(phi_e[:3] / R - 1)), (phi_q, phi_e)
    # far from the surface both variants coincide
    assert abs(phi_q[3] - phi_e[3]) < 1e-14


def test_exact_charge_near_transpose_and_gradient():
    Pq, Pe = _shell_problem(0.02)
    rng = np.random.default_rng(3)
    s, u = rng.standard_normal(Pe.n), rng.standard_normal(Pe.nc)
    # C^T is the transpose of C (dot-product identity), in both variants
    for P in (Pq, Pe):
        assert abs(u @ P.c(s) - P.ct(u) @ s) < 1e-12 * np.linalg.norm(u) * np.linalg.norm(P.ct(u)) * 10
    # the gradient at the charges is the derivative of C s (small steps keep
    # every pair on its side of the near/far threshold)
    g = Pe.grad_c(s)
    eps = 1e-6
    for k in range(Pe.nc):
        for c in range(3):
            xp, xm = Pe.xq.copy(), Pe.xq.copy()
            xp[k, c] += eps
            xm[k, c] -= eps
            chp = np.column_stack([xp, Pe.q])
            chm = np.column_stack([xm, Pe.q])
            fp = oracle.Problem(Pe.panels, chp, Pe.eps_in, Pe.eps_out, exact_charge_near=True).c(s)[k]
            fm = oracle.Problem(Pe.panels, chm, Pe.eps_in, Pe.eps_out, exact_charge_near=True).c(s)[k]
            fd = (fp - fm) / (2 * eps)
            assert abs(g[k, c] - fd) < 1e-6 * max(1.0, abs(fd)), (k, c, g[k, c], fd)


# ------------------------------------- Galerkin transposes and gradients
def test_galerkin_transposes_by_dot_products():
    m = synth.small_molecule(2, n_charges=12)
    P = oracle.Problem(m.panels, m.charges, m.eps_in, m.eps_out)
    rng = np.random.default_rng(8)
    x, y = rng.normal(size=P.n), rng.normal(size=P.n)
    kx = P.kprime_galerkin(x)
    assert abs(kx @ y - x @ P.kprime_t_galerkin(y)) < 1e-12 * np.abs(kx).sum() * np.abs(y).max()
    # entry for entry: K'_G^T e_j is row j of K'_G, (K'_G e_i)_j for every i
    eye = np.eye(P.n)
    for j in (0, 7, P.n - 1):
        row_j = np.array([P.kprime_rows_galerkin(eye[i], [j])[0] for i in range(P.n)])
        np.testing.assert_allclose(P.kprime_t_galerkin(eye[j]), row_j, rtol=1e-12, atol=1e-14)
    q, v = rng.normal(size=P.nc), rng.normal(size=P.n)
    bq = P.bq_galerkin(q)
    assert abs(bq @ v - q @ P.bt_galerkin(v)) < 1e-12 * np.linalg.norm(bq) * np.linalg.norm(v)


def _energy_galerkin_at(m, charges, tol=1e-13):
    P = oracle.Problem(m.panels, charges, m.eps_in, m.eps_out)
    sig, _ = P.solve_galerkin(tol=tol, maxiter=2000)
    return P.energy(sig)[0]


def test_galerkin_gradients_match_central_differences():
    m = synth.small_molecule(2, n_charges=9)
    P = oracle.Problem(m.panels, m.charges, m.eps_in, m.eps_out)
    dg, dq, dx, _, _ = P.gradients_galerkin(tol=1e-13)
    assert abs(P.q @ dq - 2 * dg) < 1e-8 * abs(dg)     # dG is quadratic in q
    hq, hx = 1e-4, 1e-4
    for k in range(0, P.nc, 4):
        cp, cm = m.charges.copy(), m.charges.copy()
        cp[k, 3] += hq
        cm[k, 3] -= hq
        fd = (_energy_galerkin_at(m, cp) - _energy_galerkin_at(m, cm)) / (2 * hq)
        assert abs(fd - dq[k]) < 1e-7 * max(1.0, abs(dq[k])), (k, fd, dq[k])
        for d in range(3):
            cp, cm = m.charges.copy(), m.charges.copy()
            cp[k, d] += hx
            cm[k, d] -= hx
            fd = (_energy_galerkin_at(m, cp) - _energy_galerkin_at(m, cm)) / (2 * hx)
            assert abs(fd - dx[k, d]) < 1e-6 * max(1.0, np.abs(dx).max()), (k, d, fd, dx[k, d])
