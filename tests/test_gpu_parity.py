"""GPU parity: the CUDA path through the C-ABI against the FP64 oracle.

Tolerances: relative L2 error of the operator product <= 1e-5 and of
solvation energies <= 1e-5 in the mixed FP32/FP64 mode; the FP64 mode
of the near field alone agrees with the dense FP64 sum to roundoff.
"""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import close, rel

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def pkg():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_1007_4591_gb300 as pkg
    pkg.load_library()
    return pkg


@pytest.fixture(scope="module")
def small4():
    m = synth.small_molecule(4)
    return m, oracle.Problem(m.panels, m.charges, m.eps_in, m.eps_out)


@pytest.fixture(scope="module")
def born3():
    m = synth.born(3)
    return m, oracle.Problem(m.panels, m.charges, m.eps_in, m.eps_out)


def _x(n, seed=0):
    return np.random.default_rng(seed).standard_normal(n)


@pytest.mark.parametrize("precision,tol", [(0, 2e-6), (1, 1e-12)])
def test_near_field_only_matches_dense(pkg, born3, precision, tol):
    m, P = born3
    x = _x(m.n_p)
    with pkg.Mesh(m.panels, m.charges, m.eps_in, m.eps_out, depth=-1, precision=precision) as g:
        y = g.matvec(torch.from_numpy(x).cuda()).cpu().numpy()
    close(y, P.A(x), tol)
    kx_ref = P.kprime(x)
    close((y - x) / P.ehat, kx_ref, 50 * tol)


@pytest.mark.parametrize("depth,p", [(2, 10), (3, 10), (3, 12), (4, 12), (4, 16)])
@pytest.mark.parametrize("m2l_mode", [1, 2, 3])
def test_fmm_matvec_matches_dense(pkg, small4, depth, p, m2l_mode):
    m, P = small4
    for x in (_x(m.n_p, 1), P.bq()):
        ref = P.A(x)
        with pkg.Mesh(m.panels, m.charges, m.eps_in, m.eps_out, depth=depth, p=p,
                      m2l_mode=m2l_mode) as g:
            y = g.matvec(torch.from_numpy(x).cuda()).cpu().numpy()
        close(y, ref, 1e-5)


@pytest.mark.parametrize("precision,tol", [(0, 2e-6), (1, 1e-11)])
@pytest.mark.parametrize("depth,p", [(3, 10), (4, 16)])
def test_p2m_from_panel_moments_matches_points(pkg, small4, precision, tol, depth, p):
    """P2M of the quadrature points from the per-panel moments built at mesh
    creation (the default) against the point P2M on every product
    (BEM_FLAG_P2M_FROM_POINTS): the far field alone (no near field) agrees to
    the precision's rounding, and both full products match the oracle."""
    m, P = small4
    x = _x(m.n_p, 3)
    far, full = [], []
    for flags in (0, pkg.BEM_FLAG_P2M_FROM_POINTS):
        with pkg.Mesh(m.panels, m.charges, m.eps_in, m.eps_out, depth=depth, p=p, precision=precision,
                      flags=flags | pkg.BEM_FLAG_NO_NEAR) as g:
            nseg = g.info()["p2m_segments"]
            if flags:
                assert nseg == 0
            else:
                # every panel has its points in one or a few leaves
                assert m.n_p <= nseg <= 7 * m.n_p, nseg
            far.append(g.matvec(torch.from_numpy(x).cuda()).cpu().numpy() - x)
        with pkg.Mesh(m.panels, m.charges, m.eps_in, m.eps_out, depth=depth, p=p, precision=precision,
                      flags=flags) as g:
            full.append(g.matvec(torch.from_numpy(x).cuda()).cpu().numpy())
    close(far[0], far[1], tol)
    ref = P.A(x)
    for y in full:
        close(y, ref, 1e-5)


def test_tensor_core_m2l_matches_simt(pkg, small4):
    """M2L on the tensor cores (3xTF32) against the SIMT FP32 operators."""
    m, P = small4
    x = P.bq()
    ys = []
    for mode in (1, 3):
        with pkg.Mesh(m.panels, m.charges, m.eps_in, m.eps_out, depth=4, p=10, m2l_mode=mode) as g:
            ys.append(g.matvec(torch.from_numpy(x).cuda()).cpu().numpy())
    close(ys[1] - x, ys[0] - x, 2e-6, inf=2e-5)


def test_tensor_core_m2l_repeats_to_summation_order(pkg, small4):
    """The tensor-core M2L adds every pair's row into its target with vector
    reductions (and BEM_FLAG_M2L_REDUCE, kept for compatibility, changes
    nothing): repeated products agree to the order of the FP32 additions, and
    both match the dense FP64 oracle."""
    m, P = small4
    x = np.random.default_rng(12).standard_normal(m.n_p)
    ref = P.A(x)
    ys = []
    for flags in (0, pkg.BEM_FLAG_M2L_REDUCE):
        with pkg.Mesh(m.panels, m.charges, m.eps_in, m.eps_out, depth=4, p=10, m2l_mode=3,
                      flags=flags) as g:
            ys.append(g.matvec(torch.from_numpy(x).cuda()).cpu().numpy())
            ys.append(g.matvec(torch.from_numpy(x).cuda()).cpu().numpy())
        close(ys[-1], ref, 1e-5)
    for y in ys[1:]:
        close(y - x, ys[0] - x, 1e-6, inf=1e-5)


@pytest.mark.parametrize("precision", [0, 1])
def test_translation_modes_agree(pkg, small4, precision):
    """The grouped dense operators and the per-target complex sums are the same
    linear maps: results agree to the working precision."""
    m, P = small4
    x = P.bq()
    ys = []
    for mode in (1, 2):
        with pkg.Mesh(m.panels, m.charges, m.eps_in, m.eps_out, depth=4, p=10,
                      m2l_mode=mode, precision=precision) as g:
            ys.append(g.matvec(torch.from_numpy(x).cuda()).cpu().numpy())
    kx = (ys[1] - x)
    tol = 2e-6 if precision == 0 else 1e-12
    close(ys[0] - x, kx, tol, inf=10 * tol)


@pytest.mark.parametrize("depth", [2, 3])
def test_fmm_matvec_fp64_mode(pkg, small4, depth):
    m, P = small4
    x = P.bq()
    with pkg.Mesh(m.panels, m.charges, m.eps_in, m.eps_out, depth=depth, p=12, precision=1) as g:
        y = g.matvec(torch.from_numpy(x).cuda()).cpu().numpy()
    close(y, P.A(x), 1e-6, inf=1e-5)  # p = 12 truncation: 3.5e-6 of the largest row


def test_ragged_open_surface(pkg):
    # a subset of panels (not a closed surface): ragged leaves and tails
    m = synth.small_molecule(4)
    pan = np.ascontiguousarray(m.panels[:3001])
    P = oracle.Problem(pan, m.charges, m.eps_in, m.eps_out)
    x = _x(3001, 4)
    with pkg.Mesh(pan, m.charges, m.eps_in, m.eps_out, depth=3, p=12) as g:
        y = g.matvec(torch.from_numpy(x).cuda()).cpu().numpy()
    close(y, P.A(x), 1e-5)


def test_rhs_matches_oracle(pkg, small4):
    m, P = small4
    with pkg.Mesh(m.panels, m.charges, m.eps_in, m.eps_out, depth=3, p=12) as g:
        b = g.rhs().cpu().numpy()
    close(b, P.rhs(), 1e-5)


@pytest.mark.parametrize("precision", [0, 1])
def test_energy_of_given_sigma(pkg, small4, precision):
    """dG from the dot product with C^T q (built once per charge set) and
    from phi = C sigma at the charges (the path taken when phi is asked for)
    both match the oracle, and each other to rounding."""
    m, P = small4
    sig = P.bq()
    dg_ref, phi_ref = P.energy(sig)
    with pkg.Mesh(m.panels, m.charges, m.eps_in, m.eps_out, depth=3, p=12, precision=precision) as g:
        dg_ctq = g.energy(torch.from_numpy(sig).cuda())
        dg, phi = g.energy(torch.from_numpy(sig).cuda(), want_phi=True)
    assert abs(dg - dg_ref) / abs(dg_ref) < 1e-5
    assert abs(dg_ctq - dg_ref) / abs(dg_ref) < 1e-5
    assert abs(dg_ctq - dg) / abs(dg_ref) < (1e-6 if precision == 0 else 1e-12), (dg_ctq, dg)
    close(phi.cpu().numpy(), phi_ref / m.eps_in, 1e-5)


def test_solve_and_energy_match_oracle(pkg, small4):
    m, P = small4
    sig_ref, _ = P.solve(tol=1e-11)
    dg_ref, _ = P.energy(sig_ref)
    with pkg.Mesh(m.panels, m.charges, m.eps_in, m.eps_out, depth=3, p=12, tol=1e-9) as g:
        sig, st = g.solve()
        dg = g.energy(sig)
    assert st["converged"] == 1
    close(sig.cpu().numpy(), sig_ref, 1e-5)
    assert abs(dg - dg_ref) / abs(dg_ref) < 1e-5


def test_born_solve(pkg, born3):
    m, P = born3
    sig_ref, _ = P.solve(tol=1e-11)
    dg_ref, _ = P.energy(sig_ref)
    with pkg.Mesh(m.panels, m.charges, m.eps_in, m.eps_out, p=10, leaf_size=64) as g:
        sig, st = g.solve()
        dg = g.energy(sig)
    assert abs(dg - dg_ref) / abs(dg_ref) < 1e-5


@pytest.mark.parametrize("variant,name", [(0, "cfa"), (1, "p"), (2, "plus_half")])
def test_bibee_matches_oracle(pkg, small4, variant, name):
    m, P = small4
    sh_ref, dg_ref = P.bibee(name)
    with pkg.Mesh(m.panels, m.charges, m.eps_in, m.eps_out, depth=3, p=12) as g:
        dg, sh = g.bibee(variant, want_sigma=True)
    close(sh.cpu().numpy(), sh_ref, 1e-5)
    assert abs(dg - dg_ref) / abs(dg_ref) < 1e-5


def test_host_and_device_arguments_agree(pkg, small4):
    m, P = small4
    x = _x(m.n_p, 7)
    h = pkg.bem_mesh_create(m.panels, m.charges, m.eps_in, m.eps_out, pkg.make_options(depth=3))
    try:
        y_host = np.empty(m.n_p)
        pkg.bem_matvec(h, x, y_host)
        xd = torch.from_numpy(x).cuda()
        yd = torch.empty_like(xd)
        pkg.bem_matvec(h, xd, yd)
        # atomically accumulated translations: equal up to summation order
        close(y_host, yd.cpu().numpy(), 1e-7, inf=1e-6)
    finally:
        pkg.bem_mesh_destroy(h)


def test_invalid_inputs_rejected(pkg):
    m = synth.born(2)
    bad = m.panels.copy()
    bad[3, 1] = np.nan
    with pytest.raises(pkg.BemError) as e:
        pkg.bem_mesh_create(bad, m.charges, 1.0, 80.0)
    assert e.value.code == pkg.BEM_EINVAL
    deg = m.panels.copy()
    deg[5, 2] = deg[5, 1]
    with pytest.raises(pkg.BemError) as e:
        pkg.bem_mesh_create(deg, m.charges, 1.0, 80.0)
    assert e.value.code == pkg.BEM_EINVAL
    with pytest.raises(pkg.BemError):
        pkg.bem_mesh_create(m.panels, m.charges, -1.0, 80.0)
    with pytest.raises(pkg.BemError):
        pkg.bem_mesh_create(m.panels, m.charges, 1.0, 80.0, pkg.make_options(p=0))


def test_full_size_sampled_rows(pkg):
    """The 81,920-panel globular molecule in the benchmark's launch
    configuration, checked on 256 sampled rows against the dense FP64 sum."""
    m = synth.globular(6)
    P = oracle.Problem(m.panels, m.charges, m.eps_in, m.eps_out)
    x = P.bq()
    rows = np.random.default_rng(3).choice(m.n_p, 256, replace=False)
    ref = x[rows] + P.ehat * P.kprime_rows(x, rows)
    with pkg.Mesh(m.panels, m.charges, m.eps_in, m.eps_out, p=12) as g:
        y = g.matvec(torch.from_numpy(x).cuda()).cpu().numpy()
        info = g.info()
    close(y[rows], ref, 1e-5)


@pytest.mark.parametrize("precision", [0, 1])
def test_exact_near_singular_integrals_match_oracle(pkg, precision):
    """near_table = BEM_NEAR_EXACT: the near-singular pairs take their exact
    flat-panel integral (oracle.kprime_rows_near_exact), a different operator
    from the 7-point one."""
    m = synth.small_molecule(4)
    P = oracle.Problem(m.panels, m.charges, m.eps_in, m.eps_out)
    x = np.random.default_rng(12).standard_normal(m.n_p)
    rows = np.random.default_rng(13).choice(m.n_p, 512, replace=False)
    ref = x[rows] + P.ehat * P.kprime_rows_near_exact(x, rows)
    quad = x[rows] + P.ehat * P.kprime_rows(x, rows)
    with pkg.Mesh(m.panels, m.charges, m.eps_in, m.eps_out, p=12, precision=precision,
                  near_table=pkg.BEM_NEAR_EXACT) as g:
        y = g.matvec(torch.from_numpy(x).cuda()).cpu().numpy()
        assert g.info()["near_table_nnz"] > 0
    err, _ = close(y[rows], ref, 1e-5)
    # the two operators really differ (4.5e-5 here), and the product follows
    # the exact one
    assert rel(quad, ref) > max(2e-5, 3 * err), (rel(quad, ref), err)


def test_exact_near_singular_integrals_full_size(pkg):
    m = synth.globular(6)
    P = oracle.Problem(m.panels, m.charges, m.eps_in, m.eps_out)
    x = P.bq()
    rows = np.random.default_rng(14).choice(m.n_p, 128, replace=False)
    ref = x[rows] + P.ehat * P.kprime_rows_near_exact(x, rows)
    with pkg.Mesh(m.panels, m.charges, m.eps_in, m.eps_out, p=10, leaf_size=64,
                  near_table=pkg.BEM_NEAR_EXACT) as g:
        y = g.matvec(torch.from_numpy(x).cuda()).cpu().numpy()
    close(y[rows], ref, 1e-5)
