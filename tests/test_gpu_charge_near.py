"""GPU parity of the higher-accuracy charge products (BEM_FLAG_CHARGE_NEAR_EXACT):
C s, C^T q and grad_x C s with every charge-panel pair closer than
2.5 sqrt(A_j) integrated exactly over the flat panel (Sec. 2.1), against the
oracle's Problem(exact_charge_near=True).

The molecules carry charges 0.02 A under panel centroids, where the 7-point
rule errs visibly: each test also checks that the quadrature-only oracle is
farther from the exact one than the gate, so the comparison means something.
Both the direct charge sums and the fast multipole charge passes are
covered, in both precisions; the Born-sphere case finds its pairs over all
panels (its panels are wider than the charge tree's neighbour reach), the
larger molecule through the tree.
"""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import close

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def pkg():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_1007_4591_gb300 as pkg
    pkg.load_library()
    return pkg


def _near_surface(m, n_near, depth, seed):
    """m's panels with n_near charges `depth` under random panel centroids and
    two charges deep inside; values uniform in [-0.8, 0.8] e."""
    P0 = oracle.Problem(m.panels, m.charges[:1], m.eps_in, m.eps_out)
    rng = np.random.default_rng(seed)
    ks = rng.choice(P0.n, n_near, replace=False)
    pts = [P0.cen[k] - depth * P0.nrm[k] for k in ks] + [[0.1, -0.2, 0.3], [-0.4, 0.3, 0.2]]
    q = rng.uniform(-0.8, 0.8, len(pts))
    ch = np.column_stack([np.array(pts), q])
    return synth.Molecule(m.name + "-near", m.panels, ch, m.eps_in, m.eps_out, m.radius)


CASES = {
    "born3": (lambda: synth.born(3, radius=2.0, eps_in=4.0), 6, 1),
    "small4": (lambda: synth.small_molecule(4), 8, 2),
}

# Depth of the near charges under the surface, both precisions.  The
# mixed-precision direct sums carry each coordinate as an FP32 hi + lo pair
# about the root cube's centre (a difference (hi - hi) + (lo - lo) keeps
# 2^-24 of its own length; with a single FP32 coordinate a charge 0.02 A
# from a point lost |x| 2^-24 / 0.02 A ~ 1e-5 per pair term, measured up to
# 6e-5 in dx on the 6 A sphere); the multipole charge passes work in leaf
# frames.  At this depth the 7-point rule misses the exact pairs by 0.3 or
# more in the energy.
DEPTH = {0: 0.02, 1: 0.02}


@pytest.fixture(scope="module", params=sorted(CASES))
def case(request):
    make, n_near, seed = CASES[request.param]
    out = {}
    for precision, depth in DEPTH.items():
        m = _near_surface(make(), n_near, depth, seed)
        out[precision] = (m, oracle.Problem(m.panels, m.charges, m.eps_in, m.eps_out),
                          oracle.Problem(m.panels, m.charges, m.eps_in, m.eps_out, exact_charge_near=True))
    return request.param, out


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("mode", [1, 2])
def test_energy_and_phi_with_exact_charge_pairs(pkg, case, precision, mode):
    name, cs = case
    m, Pq, Pe = cs[precision]
    sig = Pe.bq()
    dg_ref, phi_ref = Pe.energy(sig)
    dg_q, phi_q = Pq.energy(sig)
    # the exact pairs move the result by far more than the gate
    assert abs(dg_q - dg_ref) > 5e-4 * abs(dg_ref), (dg_q, dg_ref)
    with pkg.Mesh(m.panels, m.charges, m.eps_in, m.eps_out, p=10, leaf_size=64, precision=precision,
                  charge_mode=mode, flags=pkg.BEM_FLAG_CHARGE_NEAR_EXACT) as g:
        s = torch.from_numpy(sig).cuda()
        dg_phi, phi = g.energy(s, want_phi=True)
        dg = g.energy(s)
    close(phi.cpu().numpy(), phi_ref / m.eps_in, 1e-5, what=f"{name} phi")
    assert abs(dg_phi - dg_ref) < 1e-5 * abs(dg_ref), (name, dg_phi, dg_ref)
    # without phi the energy is C^T q . sigma (the table's transpose)
    assert abs(dg - dg_ref) < 1e-5 * abs(dg_ref), (name, dg, dg_ref)


@pytest.mark.parametrize("precision", [0, 1])
def test_solve_and_gradients_with_exact_charge_pairs(pkg, case, precision):
    name, cs = case
    m, Pq, Pe = cs[precision]
    dg_ref, dq_ref, dx_ref, sig_ref, _ = Pe.gradients(tol=1e-12)
    _, _, dx_q, _, _ = Pq.gradients(tol=1e-12)
    assert np.abs(dx_q - dx_ref).max() > 1e-4 * np.abs(dx_ref).max()
    with pkg.Mesh(m.panels, m.charges, m.eps_in, m.eps_out, p=10, leaf_size=64, tol=1e-11,
                  precision=precision, flags=pkg.BEM_FLAG_CHARGE_NEAR_EXACT) as g:
        sig, st = g.solve()
        assert st["converged"] == 1
        dg = g.energy(sig)
        dq, dx = g.energy_backward(1.0)
    close(sig.cpu().numpy(), sig_ref, 1e-5, what=f"{name} sigma")
    assert abs(dg - dg_ref) < 1e-5 * abs(dg_ref), (name, dg, dg_ref)
    close(dq.cpu().numpy(), dq_ref, 1e-5, what=f"{name} dq")
    close(dx.cpu().numpy(), dx_ref, 1e-5, what=f"{name} dx")


def test_set_charges_rebuilds_the_exact_pairs(pkg, case):
    """A new charge set (bem_set_charges) gets its own exact pairs."""
    name, cs = case
    m, Pq, Pe = cs[1]
    sig = Pe.bq()
    ch2 = m.charges.copy()
    ch2[:, 3] *= -1.5
    Pe2 = oracle.Problem(m.panels, ch2, m.eps_in, m.eps_out, exact_charge_near=True)
    dg_ref, _ = Pe2.energy(sig)
    with pkg.Mesh(m.panels, m.charges, m.eps_in, m.eps_out, p=10, leaf_size=64, precision=1,
                  flags=pkg.BEM_FLAG_CHARGE_NEAR_EXACT) as g:
        g.set_charges(ch2)
        dg = g.energy(torch.from_numpy(sig).cuda())
    assert abs(dg - dg_ref) < 1e-5 * abs(dg_ref), (name, dg, dg_ref)
