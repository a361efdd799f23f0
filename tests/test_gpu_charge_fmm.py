"""GPU parity of the products between the charges and the surface when they
run as fast multipole passes on the charge tree (charge_mode = 1, the form
chosen automatically once n_c x n_p x 7 exceeds 4e10, e.g. the 81.9M-panel
lattice): the right-hand side -Ehat B q (Sec. 2.1, Eq. ASC), the reaction
potential C sigma at the charges (Eq. reac), the energies built on them
(solve, BIBEE) and the gradients, all against the dense FP64 oracle.

Point charges are the hard case for a fast multipole pass: a charge sits at
an arbitrary spot of its cell, so a one-cell separation converges only like
(sqrt(3)/2)^p.  The cases include a charge exactly on a cell corner (the
Born ion's central charge: the root cube is centred on it) and charges on a
leaf face and a leaf corner.
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


def _face_molecule():
    """small_molecule(4) with charge 0 moved onto a leaf face and charge 1
    onto a leaf corner (leaf level 3 of the root cube bem_mesh_create builds:
    the bounding cube of vertices and charges)."""
    m = synth.small_molecule(4)
    ch = m.charges.copy()
    pts = np.vstack([m.panels.reshape(-1, 3), ch[:, :3]])
    lo, hi = pts.min(0), pts.max(0)
    side = (hi - lo).max() * (1 + 1e-6) + 1e-12
    rmin = 0.5 * (lo + hi) - 0.5 * side
    h = side / 2 ** 3
    ix = np.floor((ch[0, :3] - rmin) / h)
    ch[0, :3] = rmin + h * np.array([ix[0] + 1.0, ix[1] + 0.5, ix[2] + 0.5])
    ch[1, :3] = rmin + h * (np.floor((ch[1, :3] - rmin) / h) + 1.0)
    # the moved charges stay inside the molecule (bounding box unchanged)
    assert np.all(np.linalg.norm(ch[:2, :3], axis=1) < 5.0)
    return synth.Molecule("small-s4-face", m.panels, ch, m.eps_in, m.eps_out, m.radius)


CASES = {
    "small4": lambda: synth.small_molecule(4),
    "born3": lambda: synth.born(3),
    "face": _face_molecule,
}


@pytest.fixture(scope="module", params=sorted(CASES))
def case(request):
    m = CASES[request.param]()
    return request.param, m, oracle.Problem(m.panels, m.charges, m.eps_in, m.eps_out)


@pytest.mark.parametrize("precision", [0, 1])
def test_rhs_bibee_and_phi_by_fmm(pkg, case, precision):
    name, m, P = case
    with pkg.Mesh(m.panels, m.charges, m.eps_in, m.eps_out, p=10, leaf_size=64, precision=precision,
                  charge_mode=pkg.BEM_CHARGE_FMM) as g:
        assert g.info()["depth"] >= 2
        close(g.rhs().cpu().numpy(), P.rhs(), 1e-5, what=f"{name} rhs")
        for v, nm in ((0, "cfa"), (1, "p"), (2, "plus_half")):
            sh_ref, dg_ref = P.bibee(nm)
            dg, sh = g.bibee(v, want_sigma=True)
            close(sh.cpu().numpy(), sh_ref, 1e-5, what=f"{name} bibee {nm}")
            assert abs(dg - dg_ref) < 1e-5 * abs(dg_ref), (name, nm, dg, dg_ref)
        sig = P.bq()
        dg_ref, phi_ref = P.energy(sig)
        dg, phi = g.energy(torch.from_numpy(sig).cuda(), want_phi=True)
        close(phi.cpu().numpy(), phi_ref / m.eps_in, 1e-5, what=f"{name} phi")
        assert abs(dg - dg_ref) < 1e-5 * abs(dg_ref)


def test_solve_energy_and_gradients_by_fmm(pkg, case):
    name, m, P = case
    dg_ref, dq_ref, dx_ref, sig_ref, _ = P.gradients(tol=1e-12)
    with pkg.Mesh(m.panels, m.charges, m.eps_in, m.eps_out, p=10, leaf_size=64, tol=1e-11,
                  charge_mode=pkg.BEM_CHARGE_FMM) as g:
        sig, st = g.solve()
        assert st["converged"] == 1
        dg, phi = g.energy(sig, want_phi=True)
        dq, dx = g.energy_backward(1.0)
    close(sig.cpu().numpy(), sig_ref, 1e-5, what=f"{name} sigma")
    assert abs(dg - dg_ref) < 1e-5 * abs(dg_ref), (name, dg, dg_ref)
    close(dq.cpu().numpy(), dq_ref, 1e-5, what=f"{name} dq")
    if np.abs(dx_ref).max() > 1e-8 * abs(dg_ref):
        close(dx.cpu().numpy(), dx_ref, 1e-5, what=f"{name} dx")
    else:  # the Born ion: a central charge feels no force (dx = 0 by symmetry)
        assert np.abs(dx.cpu().numpy()).max() < 1e-5 * abs(dg_ref) / m.radius


def test_fmm_and_direct_charge_sums_agree_on_globular_s6(pkg):
    """The two charge_mode forms on the benchmark molecule (81,920 panels,
    2,000 charges) give the same right-hand side and energies."""
    m = synth.globular(6)
    out = {}
    for mode in (1, 2):
        with pkg.Mesh(m.panels, m.charges, m.eps_in, m.eps_out, p=10, leaf_size=64, charge_mode=mode) as g:
            b = g.rhs().cpu().numpy()
            dg, phi = g.energy(torch.from_numpy(-b).cuda(), want_phi=True)
            out[mode] = (b, dg, phi.cpu().numpy())
    close(out[1][0], out[2][0], 1e-5, what="rhs")
    close(out[1][2], out[2][2], 1e-5, what="phi")
    assert abs(out[1][1] - out[2][1]) < 1e-5 * abs(out[2][1])


@pytest.mark.slow
def test_lattice10_rhs_rows(pkg):
    """The 81.9M-panel lattice (2M charges), where the automatic choice is the
    fast multipole pass: 16 sampled rows of the right-hand side against the
    oracle's rows of B q."""
    m = synth.lattice(10)
    P = oracle.Problem(m.panels, m.charges, m.eps_in, m.eps_out)
    rows = np.random.default_rng(10).choice(m.n_p, 16, replace=False)
    ref = -P.ehat * P.bq_rows(rows)
    with pkg.Mesh(m.panels, m.charges, m.eps_in, m.eps_out, p=10, leaf_size=64) as g:
        b = g.rhs().cpu().numpy()
    e2, ei = close(b[rows], ref, 1e-5, what="lattice10 rhs rows")
    print(f"lattice10 right-hand side, 16 rows: relative L2 error {e2:.2e}, max {ei:.2e}")
