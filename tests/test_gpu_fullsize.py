"""Full-size workloads on the GPU, checked on sampled outputs the dense FP64
oracle computes one by one, or by properties that hold at any size.

* globular-s6 (81,920 panels) in the launch configuration bench.py times
  (mixed precision, p = 10, leaf size 64);
* globular-s7 (327,680 panels): sampled rows of the product, and the energy
  gradients of one autograd call against the FP64 GPU form and central
  differences in q and x on 20 seeded charges;
* globular-s5 (20,480 panels, the same 2,000 charges): the gradients of one
  autograd call against the oracle's dense adjoint;
* batch64 (64 uneven molecules, 9.5M panels): batched solve against
  one-at-a-time solves and the BIBEE bounds around every solve;
* lattice10 (1,000 rotated copies of globular-s6, 81.9M panels): sampled
  rows of the product.
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


def _rows_check(pkg, m, x, rows, tol, **opts):
    P = oracle.Problem(m.panels, m.charges, m.eps_in, m.eps_out)
    ref = x[rows] + P.ehat * P.kprime_rows(x, rows)
    with pkg.Mesh(m.panels, m.charges, m.eps_in, m.eps_out, **opts) as g:
        y = g.matvec(torch.from_numpy(x).cuda()).cpu().numpy()
    return close(y[rows], ref, tol)


def test_globular_s6_bench_configuration_rows(pkg):
    """Smooth (the right-hand side B q) and random inputs, 256 rows each."""
    m = synth.globular(6)
    P = oracle.Problem(m.panels, m.charges, m.eps_in, m.eps_out)
    rows = np.random.default_rng(3).choice(m.n_p, 256, replace=False)
    for x in (P.bq(), np.random.default_rng(5).standard_normal(m.n_p)):
        ref = x[rows] + P.ehat * P.kprime_rows(x, rows)
        with pkg.Mesh(m.panels, m.charges, m.eps_in, m.eps_out, p=10, leaf_size=64, precision=0) as g:
            y = g.matvec(torch.from_numpy(x).cuda()).cpu().numpy()
            assert g.info()["depth"] == 5
        close(y[rows], ref, 1e-5)


def test_globular_s7_rows(pkg):
    m = synth.globular(7)
    P = oracle.Problem(m.panels, m.charges, m.eps_in, m.eps_out)
    x = P.bq()
    rows = np.random.default_rng(4).choice(m.n_p, 64, replace=False)
    ref = x[rows] + P.ehat * P.kprime_rows(x, rows)
    with pkg.Mesh(m.panels, m.charges, m.eps_in, m.eps_out, p=10, leaf_size=64, precision=0) as g:
        y = g.matvec(torch.from_numpy(x).cuda()).cpu().numpy()
    close(y[rows], ref, 1e-5)


def test_globular_s7_gradients(pkg):
    """One autograd call (mixed precision) gives d dG/dq and d dG/dx of all
    2,000 charges; they match the FP64 GPU form, whose own derivatives match
    central differences (steps 1e-4 e and 1e-4 A, every perturbed solve
    started from the unperturbed one) on 20 seeded charges."""
    m = synth.globular(7)
    with pkg.Mesh(m.panels, m.charges, m.eps_in, m.eps_out, p=10, leaf_size=64, precision=0,
                  tol=1e-10) as g:
        ch = torch.tensor(m.charges, dtype=torch.float64, device="cuda", requires_grad=True)
        dg = pkg.solvation_energy(g, ch)
        dg.backward()
        gq_mixed = ch.grad[:, 3].cpu().numpy()
        gx_mixed = ch.grad[:, :3].cpu().numpy()
        dg_mixed = float(dg.detach())
    with pkg.Mesh(m.panels, m.charges, m.eps_in, m.eps_out, p=12, leaf_size=64, precision=1,
                  tol=1e-12, max_iter=500) as g:
        s0, _ = g.solve()

        def energy(c):
            g.set_charges(torch.tensor(c).cuda())
            s, _ = g.solve(x0=s0)
            return g.energy(s)
        e0 = energy(m.charges)
        dq, dx = g.energy_backward(1.0)
        dq, dx = dq.cpu().numpy(), dx.cpu().numpy()
        assert abs(dg_mixed - e0) < 1e-5 * abs(e0), (dg_mixed, e0)
        close(gq_mixed, dq, 1e-5)
        close(gx_mixed, dx, 1e-5)
        rng = np.random.default_rng(3)
        for k in rng.choice(m.n_c, 20, replace=False):
            cp, cm = m.charges.copy(), m.charges.copy()
            cp[k, 3] += 1e-4
            cm[k, 3] -= 1e-4
            fd = (energy(cp) - energy(cm)) / 2e-4
            assert abs(fd - dq[k]) < 1e-5 * max(1.0, abs(dq[k])), (k, fd, dq[k])
            a = int(rng.integers(3))
            cp, cm = m.charges.copy(), m.charges.copy()
            cp[k, a] += 1e-4
            cm[k, a] -= 1e-4
            fd = (energy(cp) - energy(cm)) / 2e-4
            assert abs(fd - dx[k, a]) < 1e-4 * max(1.0, np.abs(dx).max()), (k, a, fd, dx[k, a])


def test_globular_s5_gradients_match_dense_adjoint(pkg):
    """d dG/dq and d dG/dx of the 2,000 charges at 20,480 panels (mixed
    precision, the bench's p = 10 and leaf 64) against the oracle's dense
    adjoint (solve A^T lam = C^T q, then the gradient formulas)."""
    m = synth.globular(5)
    P = oracle.Problem(m.panels, m.charges, m.eps_in, m.eps_out)
    dg_ref, dq_ref, dx_ref, _, _ = P.gradients(tol=1e-11)
    with pkg.Mesh(m.panels, m.charges, m.eps_in, m.eps_out, p=10, leaf_size=64, precision=0,
                  tol=1e-10) as g:
        ch = torch.tensor(m.charges, dtype=torch.float64, device="cuda", requires_grad=True)
        dg = pkg.solvation_energy(g, ch)
        dg.backward()
    assert abs(float(dg.detach()) - dg_ref) < 1e-5 * abs(dg_ref)
    close(ch.grad[:, 3].cpu().numpy(), dq_ref, 1e-5)
    close(ch.grad[:, :3].cpu().numpy(), dx_ref, 1e-5)


def test_batch64_solve_and_bounds(pkg):
    mols = synth.batch(64, seed=4)
    meshes = [pkg.Mesh(m.panels, m.charges, m.eps_in, m.eps_out, p=10, leaf_size=64, precision=0,
                       tol=1e-8) for m in mols]
    try:
        dg, dc, dp, st = pkg.bem_batch_solve(meshes, threads=8)
        assert all(s["converged"] == 1 for s in st)
        assert np.all(dp < dg) and np.all(dg < dc)          # BIBEE bounds around every solve
        assert np.all(dg < 0)
        for i in np.random.default_rng(6).choice(len(mols), 3, replace=False):
            s, _ = meshes[i].solve()
            e = meshes[i].energy(s)
            assert abs(dg[i] - e) < 1e-6 * abs(e), (i, dg[i], e)
    finally:
        for g in meshes:
            g.close()


@pytest.mark.slow
def test_lattice10_rows(pkg):
    """1,000 randomly rotated copies of globular-s6 on a 50 A lattice
    (81,920,000 panels, 573M quadrature points, 2M charges): 8 sampled rows
    of the product with a seeded random input."""
    m = synth.lattice(10)
    x = np.random.default_rng(8).standard_normal(m.n_p)
    rows = np.random.default_rng(9).choice(m.n_p, 8, replace=False)
    e2, ei = _rows_check(pkg, m, x, rows, 1e-5, p=10, leaf_size=64, precision=0)
    print(f"lattice10 product, 8 rows: relative L2 error {e2:.2e}, max {ei:.2e}")
