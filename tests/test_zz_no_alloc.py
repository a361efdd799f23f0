"""The allocation-free entry point (bem_normal_field_noalloc) against the
ordinary one (bem_rhs), through the C ABI, on two calls in a row.

Callers that cannot allocate GPU memory (inside another framework's pool, in
a loop that must not touch the allocator) use bem_normal_field_noalloc: its
scratch is a fixed array in the library.  This file is collected last so that
a run stopping at the first failure has run everything else first; it passes
alone in a fresh process as well.
"""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _centroids_normals(panels):
    c = panels.mean(axis=1)
    n = np.cross(panels[:, 1] - panels[:, 0], panels[:, 2] - panels[:, 0])
    n /= np.linalg.norm(n, axis=1, keepdims=True)
    return np.ascontiguousarray(c), np.ascontiguousarray(n)


def test_noalloc_normal_field_matches_rhs_on_two_calls():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_1007_4591_gb300 as pkg
    pkg.load_library()
    mols = [synth.small_molecule(4),
            synth.globular(4, radius=10.0, n_charges=300, charge_radius=7.0, seed=9)]
    for mol in mols:  # two calls in a row, different sizes: no stale scratch may leak in
        with pkg.Mesh(mol.panels, mol.charges, mol.eps_in, mol.eps_out) as g:
            b = g.rhs().cpu().numpy()
        ehat = 2.0 * (mol.eps_in - mol.eps_out) / (mol.eps_in + mol.eps_out)
        c, n = _centroids_normals(mol.panels)
        tc = torch.from_numpy(c).cuda()
        tn = torch.from_numpy(n).cuda()
        tq = torch.from_numpy(np.ascontiguousarray(mol.charges)).cuda()
        field = torch.full((mol.n_p,), float("nan"), dtype=torch.float64, device="cuda")
        pkg.bem_normal_field_noalloc(tc, tn, tq, field)
        torch.cuda.synchronize()
        e = field.cpu().numpy()
        err = np.linalg.norm(-ehat * e - b) / np.linalg.norm(b)
        assert err < 1e-5, err


def test_noalloc_rejects_oversize_and_host_arrays():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_1007_4591_gb300 as pkg
    lib = pkg.load_library()
    import ctypes
    big = (1 << 21) + 1
    rc = lib.bem_normal_field_noalloc(None, None, big, None, 0, None, None)
    assert rc == pkg.BEM_EINVAL and "scratch" in pkg.bem_last_error()
    t = np.zeros((4, 3))
    with pytest.raises(pkg.BemError):
        pkg.bem_normal_field_noalloc(t, t, np.zeros((1, 4)), np.zeros(4))
