"""Faults injected from the host, none of which faults or hangs the GPU:
a tiny wait budget for the tensor-core M2L kernel's pipeline (every bounded
wait runs out, the call reports BEM_ETIMEOUT, the mesh stays usable) and a
device memory cap (BEM_ENOMEM before the allocator is reached)."""
import numpy as np
import pytest

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


def test_wait_budget_timeout_is_reported_and_the_mesh_recovers(pkg):
    m = synth.small_molecule(4)
    x = torch.from_numpy(np.random.default_rng(21).standard_normal(m.n_p)).cuda()
    with pkg.Mesh(m.panels, m.charges, m.eps_in, m.eps_out, depth=3, p=10, precision=0) as g:
        assert g.info()["m2l_pairs"] > 0
        y0 = g.matvec(x).cpu().numpy()
        pkg.bem_set_wait_budget(g.h, 100)           # cycles: every pipeline wait runs out
        with pytest.raises(pkg.BemError) as ei:
            g.matvec(x)
        assert ei.value.code == pkg.BEM_ETIMEOUT
        pkg.bem_set_wait_budget(g.h, 0)             # back to the default
        y1 = g.matvec(x).cpu().numpy()
        close(y1, y0, 1e-6, inf=1e-5)
    with pytest.raises(pkg.BemError):
        pkg.bem_set_wait_budget(None, 5)


def test_device_memory_cap_gives_enomem(pkg):
    m = synth.small_molecule(3)
    try:
        pkg.bem_set_device_memory_cap(1)
        with pytest.raises(pkg.BemError) as ei:
            pkg.Mesh(m.panels, m.charges, m.eps_in, m.eps_out)
        assert ei.value.code == pkg.BEM_ENOMEM
        assert "cap" in pkg.bem_last_error()
    finally:
        pkg.bem_set_device_memory_cap(0)
    with pkg.Mesh(m.panels, m.charges, m.eps_in, m.eps_out) as g:   # no cap: fine again
        assert g.info()["n_p"] == m.n_p


def test_charge_outside_the_surface_is_rejected_when_checked(pkg):
    m = synth.small_molecule(3)
    flags = pkg.BEM_FLAG_CHECK_CHARGES
    with pkg.Mesh(m.panels, m.charges, m.eps_in, m.eps_out, flags=flags) as g:   # all enclosed
        assert g.info()["n_c"] == m.n_c
    bad = m.charges.copy()
    bad[5, :3] = [2.5 * m.radius, 0.0, 0.0]
    with pytest.raises(pkg.BemError) as ei:
        pkg.Mesh(m.panels, bad, m.eps_in, m.eps_out, flags=flags)
    assert ei.value.code == pkg.BEM_EINVAL and "charge 5" in pkg.bem_last_error()
    # two disjoint closed surfaces: each charge is enclosed by its own
    cpx, _, _ = synth.complex_pair(s_rec=3, r_rec=10.0, n_rec=50, s_lig=2, r_lig=4.0, n_lig=20)
    with pkg.Mesh(cpx.panels, cpx.charges, cpx.eps_in, cpx.eps_out, flags=flags) as g:
        assert g.info()["n_c"] == cpx.n_c
