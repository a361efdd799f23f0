"""The allocation-free entry point (bem_normal_field_noalloc) against the
ordinary one (bem_rhs) and the oracle, through the C ABI.

Callers that cannot allocate GPU memory (code inside another framework's
memory pool, a loop that must not touch the allocator, a process whose device
memory is already handed out) use bem_normal_field_noalloc: its only scratch
is a fixed array in the library.  The calls here run back to back on that
shared array: two mesh-sized calls, then calls with one and with several
source splits, a larger call followed by a smaller one, a call without
charges and one at the largest accepted size, each compared element by
element.  This file is collected last so that a run stopping at the first
failure has run everything else first; it passes alone in a fresh process as
well.
"""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import close

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

MAX_TARGETS = 1 << 21  # BEM_NOALLOC_SCRATCH_FLOATS


@pytest.fixture(scope="module")
def pkg():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_1007_4591_gb300 as pkg
    pkg.load_library()
    return pkg


def _centroids_normals(panels):
    c = panels.mean(axis=1)
    n = np.cross(panels[:, 1] - panels[:, 0], panels[:, 2] - panels[:, 0])
    n /= np.linalg.norm(n, axis=1, keepdims=True)
    return np.ascontiguousarray(c), np.ascontiguousarray(n)


def _field(pkg, t, n, ch):
    tt = torch.from_numpy(np.ascontiguousarray(t)).cuda()
    tn = torch.from_numpy(np.ascontiguousarray(n)).cuda()
    tq = torch.from_numpy(np.ascontiguousarray(ch, dtype=np.float64).reshape(-1, 4)).cuda()
    field = torch.full((t.shape[0],), float("nan"), dtype=torch.float64, device="cuda")
    pkg.bem_normal_field_noalloc(tt, tn, tq, field)
    torch.cuda.synchronize()
    return field.cpu().numpy()


def _unit(rng, n):
    v = rng.standard_normal((n, 3))
    return v / np.linalg.norm(v, axis=1, keepdims=True)


def _points(n, seed):
    """n points in the shell 18 A <= r <= 25 A with random unit normals."""
    rng = np.random.default_rng(seed)
    t = _unit(rng, n) * rng.uniform(18.0, 25.0, (n, 1))
    return t, _unit(rng, n)


def _charges(n, seed):
    """n charges in the ball r <= 15 A (at least 3 A from every point)."""
    rng = np.random.default_rng(seed)
    x = _unit(rng, n) * (15.0 * rng.uniform(0.0, 1.0, (n, 1)) ** (1.0 / 3.0))
    return np.column_stack([x, rng.uniform(-1, 1, n)])


def test_noalloc_normal_field_matches_rhs_on_two_calls(pkg):
    mols = [synth.small_molecule(4),
            synth.globular(3, radius=10.0, n_charges=300, charge_radius=7.0, seed=9)]
    for mol in mols:  # two calls in a row, different sizes: no stale scratch may leak in
        with pkg.Mesh(mol.panels, mol.charges, mol.eps_in, mol.eps_out) as g:
            b = g.rhs().cpu().numpy()
        ehat = 2.0 * (mol.eps_in - mol.eps_out) / (mol.eps_in + mol.eps_out)
        c, n = _centroids_normals(mol.panels)
        e = _field(pkg, c, n, mol.charges)
        close(-ehat * e, b, 1e-5, what=mol.name)
        close(e, oracle.normal_field(c, n, mol.charges), 1e-5, what=mol.name + " vs oracle")


def test_noalloc_split_sizes_back_to_back(pkg):
    """Several source splits (20,000 charges over 2,000 points), then a
    larger single-split call, then a smaller one, then one without charges:
    each against the oracle element by element."""
    seq = [(2000, 20000), (60000, 300), (1000, 9000), (500, 0)]
    for i, (nt, nc) in enumerate(seq):
        t, nv = _points(nt, 100 + i)
        ch = _charges(nc, 200 + i)
        e = _field(pkg, t, nv, ch)
        if nc == 0:
            assert np.all(e == 0.0)
            continue
        rows = np.random.default_rng(300 + i).choice(nt, min(nt, 3000), replace=False)
        close(e[rows], oracle.normal_field(t[rows], nv[rows], ch), 1e-5, what=f"{nt} x {nc}")


def test_noalloc_far_from_the_origin(pkg):
    """A molecule 450 A from the origin (a corner of the 81.9M-panel
    lattice): the points' differences keep their precision."""
    mol = synth.small_molecule(4)
    shift = np.array([450.0, 440.0, 445.0])
    pan = mol.panels + shift
    ch = mol.charges.copy()
    ch[:, :3] += shift
    c, n = _centroids_normals(pan)
    e = _field(pkg, c, n, ch)
    close(e, oracle.normal_field(c, n, ch), 1e-5, what="shifted")


def test_noalloc_largest_size(pkg):
    """n_t = BEM_NOALLOC_SCRATCH_FLOATS, the largest accepted size."""
    t, nv = _points(MAX_TARGETS, 7)
    ch = _charges(5000, 8)
    e = _field(pkg, t, nv, ch)
    rows = np.random.default_rng(9).choice(MAX_TARGETS, 2000, replace=False)
    close(e[rows], oracle.normal_field(t[rows], nv[rows], ch), 1e-5, what="largest")


def test_noalloc_rejects_oversize_and_host_arrays(pkg):
    import ctypes
    lib = pkg.load_library()
    rc = lib.bem_normal_field_noalloc(None, None, MAX_TARGETS + 1, None, 0, None, None)
    assert rc == pkg.BEM_EINVAL and "scratch" in pkg.bem_last_error()
    t = np.zeros((4, 3))
    with pytest.raises(TypeError):
        pkg.bem_normal_field_noalloc(t, t, np.zeros((1, 4)), np.zeros(4))
    # host pointers straight through the C ABI
    q = np.zeros((1, 4))
    f = np.zeros(4)
    p = lambda a: ctypes.c_void_p(a.ctypes.data)
    rc = lib.bem_normal_field_noalloc(p(t), p(t), 4, p(q), 1, p(f), None)
    assert rc == pkg.BEM_EINVAL and "device memory" in pkg.bem_last_error()
    # wrong dtype or length is caught before the call
    td = torch.zeros((4, 3), dtype=torch.float32, device="cuda")
    with pytest.raises(TypeError):
        pkg.bem_normal_field_noalloc(td, td, torch.zeros((1, 4), dtype=torch.float64, device="cuda"),
                                     torch.zeros(4, dtype=torch.float64, device="cuda"))
    t64 = torch.zeros((4, 3), dtype=torch.float64, device="cuda")
    with pytest.raises(ValueError):
        pkg.bem_normal_field_noalloc(t64, t64, torch.zeros((1, 3), dtype=torch.float64, device="cuda"),
                                     torch.zeros(4, dtype=torch.float64, device="cuda"))
