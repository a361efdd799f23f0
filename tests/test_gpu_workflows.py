"""Workflows on top of the solver, against the dense FP64 oracle:
the binding free energy of a two-sphere complex (Eq. binding) and the
crowded-solution superposition heuristic next to the coupled solve (Sec. 5)."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def pkg():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_1007_4591_gb300 as pkg
    pkg.load_library()
    return pkg


def _oracle_energy(m, sigma=None):
    P = oracle.Problem(m.panels, m.charges, m.eps_in, m.eps_out)
    if sigma is None:
        sigma, _ = P.solve(tol=1e-11)
    e, _ = P.energy(sigma)
    return e, sigma


def test_binding_free_energy_matches_oracle(pkg):
    cpx, rec, lig = synth.complex_pair(s_rec=3, r_rec=10.0, n_rec=50, s_lig=2, r_lig=4.0, n_lig=20)
    dg_bind, (dc, dr, dl) = pkg.binding_free_energy(cpx, rec, lig, p=12, tol=1e-10)
    ref = [_oracle_energy(m)[0] for m in (cpx, rec, lig)]
    for got, want in zip((dc, dr, dl), ref):
        assert abs(got - want) < 1e-5 * abs(want), (got, want)
    bind_ref = ref[0] - ref[1] - ref[2]
    assert abs(dg_bind - bind_ref) < 1e-5 * abs(ref[0]), (dg_bind, bind_ref)
    # the complex is more than the sum of its parts: the surfaces interact
    assert abs(bind_ref) > 1e-3 * abs(ref[0])


def test_superposition_heuristic_matches_oracle(pkg):
    base = synth.small_molecule(2)
    system = synth.lattice(n_side=2, spacing=16.0, base=base)
    out = pkg.superposition_energy(base, system, copies=8, p=12, tol=1e-10)
    e_iso, s_iso = _oracle_energy(base)
    e_sup, _ = _oracle_energy(system, np.tile(s_iso, 8))
    e_cpl, _ = _oracle_energy(system)
    assert abs(out["dG_isolated"] - 8 * e_iso) < 1e-5 * abs(8 * e_iso)
    assert abs(out["dG_superposed"] - e_sup) < 1e-5 * abs(e_sup), (out["dG_superposed"], e_sup)
    assert abs(out["dG_coupled"] - e_cpl) < 1e-5 * abs(e_cpl), (out["dG_coupled"], e_cpl)
    # the copies polarise one another: the heuristic misses that by more than
    # the solves' tolerance (5e-5 relative at 16 A spacing)
    assert abs(e_sup - e_cpl) > 1e-6 * abs(e_cpl)
