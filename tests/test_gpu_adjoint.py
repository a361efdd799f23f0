"""GPU adjoint: the transposed operator and the energy gradients against the
oracle's dense adjoint, the dot-product identity and central differences."""
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


@pytest.mark.parametrize("depth,precision", [(-1, 0), (-1, 1), (3, 0), (4, 0), (3, 1)])
def test_transposed_operator_matches_dense(pkg, small4, depth, precision):
    m, P = small4
    x = np.random.default_rng(2).standard_normal(m.n_p)
    ref = P.At(x)
    with pkg.Mesh(m.panels, m.charges, m.eps_in, m.eps_out, depth=depth, p=12,
                  precision=precision) as g:
        y = g.matvec_t(torch.from_numpy(x).cuda()).cpu().numpy()
    tol = 1e-12 if (precision == 1 and depth == -1) else 1e-5
    close(y, ref, tol)


def test_dot_product_identity_on_gpu(pkg, small4):
    m, P = small4
    rng = np.random.default_rng(8)
    x, y = rng.standard_normal(m.n_p), rng.standard_normal(m.n_p)
    with pkg.Mesh(m.panels, m.charges, m.eps_in, m.eps_out, depth=3, p=12) as g:
        ax = g.matvec(torch.from_numpy(x).cuda()).cpu().numpy()
        aty = g.matvec_t(torch.from_numpy(y).cuda()).cpu().numpy()
    lhs, rhs = float(ax @ y), float(x @ aty)
    assert abs(lhs - rhs) < 1e-6 * np.linalg.norm(ax) * np.linalg.norm(y)


def test_energy_gradients_match_dense_adjoint(pkg, small4):
    m, P = small4
    dg_ref, dq_ref, dx_ref, _, _ = P.gradients(tol=1e-12)
    with pkg.Mesh(m.panels, m.charges, m.eps_in, m.eps_out, depth=3, p=12, tol=1e-11) as g:
        sig, st = g.solve()
        dg = g.energy(sig)
        dq, dx = g.energy_backward(1.0)
    assert abs(dg - dg_ref) / abs(dg_ref) < 1e-5
    close(dq.cpu().numpy(), dq_ref, 1e-5)
    close(dx.cpu().numpy(), dx_ref, 1e-5)


def test_autograd_function_matches_backward(pkg):
    m = synth.small_molecule(3)
    with pkg.Mesh(m.panels, m.charges, m.eps_in, m.eps_out, depth=2, p=12, tol=1e-11) as g:
        ch = torch.tensor(m.charges, dtype=torch.float64, device="cuda", requires_grad=True)
        dg = pkg.solvation_energy(g, ch)
        dg.backward()
        dq, dx = g.energy_backward(1.0)
        # two backward solves: equal up to the solve tolerance and the order of
        # the FP32 atomic sums (repeated mixed-precision runs differ by ~1e-7 of
        # the largest entry, so the comparison is norm-wise)
        close(ch.grad[:, 3].cpu().numpy(), dq.cpu().numpy(), 1e-6, inf=1e-5)
        close(ch.grad[:, :3].cpu().numpy(), dx.cpu().numpy(), 1e-6, inf=1e-5)
        # quadratic in q: q . d dG/dq = 2 dG
        assert abs(float(ch.grad[:, 3] @ ch.detach()[:, 3]) - 2 * float(dg)) < 1e-6 * abs(float(dg))


def test_gradients_central_differences_fp64(pkg):
    """FP64 GPU path: d dG/dq and d dG/dx against central differences
    (steps 1e-4 e and 1e-4 A) on a few seeded charges."""
    m = synth.small_molecule(3)
    with pkg.Mesh(m.panels, m.charges, m.eps_in, m.eps_out, depth=2, p=14, precision=1,
                  tol=1e-13, max_iter=2000) as g:
        def energy(ch):
            g.set_charges(torch.tensor(ch).cuda())
            s, _ = g.solve()
            return g.energy(s)
        e0 = energy(m.charges)
        g.set_charges(torch.tensor(m.charges).cuda())
        s, _ = g.solve()
        dq, dx = g.energy_backward(1.0)
        dq, dx = dq.cpu().numpy(), dx.cpu().numpy()
        idx = np.random.default_rng(3).choice(m.n_c, 5, replace=False)
        for k in idx:
            cp, cm = m.charges.copy(), m.charges.copy()
            cp[k, 3] += 1e-4
            cm[k, 3] -= 1e-4
            fd = (energy(cp) - energy(cm)) / 2e-4
            assert abs(fd - dq[k]) < 1e-6 * max(1.0, abs(dq[k])), (k, fd, dq[k])
            for d in range(3):
                cp, cm = m.charges.copy(), m.charges.copy()
                cp[k, d] += 1e-4
                cm[k, d] -= 1e-4
                fd = (energy(cp) - energy(cm)) / 2e-4
                assert abs(fd - dx[k, d]) < 1e-5 * max(1.0, np.abs(dx).max()), (k, d, fd, dx[k, d])
    assert np.isfinite(e0)
