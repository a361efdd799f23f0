"""Batching, graph replay, stream ordering and the autotuner on the GPU."""
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


def _mols():
    return synth.batch(n_molecules=5, seed=4, subdivisions=(3, 4), radius_range=(6.0, 12.0),
                       charge_range=(20, 80))


def test_batch_solve_equals_one_at_a_time(pkg):
    mols = _mols()
    meshes = [pkg.Mesh(m.panels, m.charges, m.eps_in, m.eps_out, p=10, tol=1e-10) for m in mols]
    dg, dc, dp, stats = pkg.bem_batch_solve(meshes, threads=3)
    for i, (m, g) in enumerate(zip(mols, meshes)):
        s, st = g.solve()
        e = g.energy(s)
        # atomically accumulated translations: equal to summation order
        assert abs(dg[i] - e) < 1e-6 * abs(e), (i, dg[i], e)
        assert abs(dc[i] - g.bibee(pkg.BEM_BIBEE_CFA)) < 1e-6 * abs(dc[i])
        assert abs(dp[i] - g.bibee(pkg.BEM_BIBEE_P)) < 1e-6 * abs(dp[i])
        assert dp[i] < dg[i] < dc[i]          # BIBEE bounds around the solve
        assert stats[i]["converged"] == 1
    for g in meshes:
        g.close()


def test_batch_solve_bitwise_in_the_deterministic_form(pkg):
    """With the translations as per-target gathers (m2l_mode = 2: M2M, M2L
    and L2L each summed by its output cell in a fixed order, no atomics) every
    kernel of the solve adds in a fixed order, so the batched solve
    reproduces one-at-a-time solves bit for bit (sigma, dG and both BIBEE
    bounds), and a repeated product is bitwise identical."""
    mols = _mols()
    meshes = [pkg.Mesh(m.panels, m.charges, m.eps_in, m.eps_out, p=10, tol=1e-10, m2l_mode=2) for m in mols]
    try:
        sig_b = [torch.empty(m.n_p, dtype=torch.float64, device="cuda") for m in mols]
        dg, dc, dp, stats = pkg.bem_batch_solve(meshes, threads=3, sigmas=sig_b)
        for i, g in enumerate(meshes):
            s, st = g.solve()
            assert torch.equal(s, sig_b[i]), i
            assert g.energy(s) == dg[i], i
            assert g.bibee(pkg.BEM_BIBEE_CFA) == dc[i] and g.bibee(pkg.BEM_BIBEE_P) == dp[i], i
            x = torch.from_numpy(np.random.default_rng(i).standard_normal(g.n_p)).cuda()
            assert torch.equal(g.matvec(x), g.matvec(x)), i
    finally:
        for g in meshes:
            g.close()


def test_batch_energies_match_oracle(pkg):
    mols = _mols()[:3]
    meshes = [pkg.Mesh(m.panels, m.charges, m.eps_in, m.eps_out, p=10, tol=1e-10) for m in mols]
    dg, dc, dp, _ = pkg.bem_batch_solve(meshes)
    for i, m in enumerate(mols):
        P = oracle.Problem(m.panels, m.charges, m.eps_in, m.eps_out)
        s, _ = P.solve(tol=1e-11)
        e, _ = P.energy(s)
        assert abs(dg[i] - e) / abs(e) < 1e-5
        assert abs(dc[i] - P.bibee("cfa")[1]) / abs(dc[i]) < 1e-5
    for g in meshes:
        g.close()


def test_graph_replay_matches_direct_launches(pkg):
    m = synth.small_molecule(4)
    x = np.random.default_rng(4).standard_normal(m.n_p)
    ys = []
    for graph in (0, 1):
        with pkg.Mesh(m.panels, m.charges, m.eps_in, m.eps_out, depth=3, graph=graph) as g:
            xt = torch.from_numpy(x).cuda()
            for _ in range(3):          # first call captures, later calls replay
                y = g.matvec(xt)
            ys.append(y.cpu().numpy())
            s, st = g.solve()
            ys.append(s.cpu().numpy())
    close(ys[2], ys[0], 1e-7, inf=1e-6)
    close(ys[3], ys[1], 1e-7, inf=1e-6)


def test_caller_stream_ordering(pkg):
    """Work queued on the caller's stream before a call is seen by the call."""
    m = synth.small_molecule(3)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        g = pkg.Mesh(m.panels, m.charges, m.eps_in, m.eps_out, depth=2)
        x = torch.zeros(m.n_p, dtype=torch.float64, device="cuda")
        torch.cuda._sleep(2_000_000)    # keep the stream busy, then fill x
        x.fill_(1.0)
        y = g.matvec(x)
    torch.cuda.synchronize()
    P = oracle.Problem(m.panels, m.charges, m.eps_in, m.eps_out)
    close(y.cpu().numpy(), P.A(np.ones(m.n_p)), 1e-5)
    g.close()


def test_autotune_meets_its_target(pkg):
    m = synth.small_molecule(4)
    opt = pkg.bem_autotune(m.panels, m.charges, m.eps_in, m.eps_out, target=1e-5)
    assert opt.p in (6, 8, 10) and opt.leaf_size in (32, 64, 128, 256)
    P = oracle.Problem(m.panels, m.charges, m.eps_in, m.eps_out)
    x = P.bq()
    with pkg.Mesh(m.panels, m.charges, m.eps_in, m.eps_out, p=opt.p, leaf_size=opt.leaf_size) as g:
        y = g.matvec(torch.from_numpy(x).cuda()).cpu().numpy()
    close(y, P.A(x), 3e-5)


def test_autotune_choice_is_cached(pkg, tmp_path):
    m = synth.small_molecule(3)
    cache = str(tmp_path / "tune.json")
    a = pkg.autotune_cached(m.panels, m.charges, m.eps_in, m.eps_out, cache=cache)
    assert not a["cached"] and a["p"] in (6, 8, 10)
    b = pkg.autotune_cached(m.panels, m.charges, m.eps_in, m.eps_out, cache=cache)
    assert b["cached"] and (b["leaf_size"], b["p"]) == (a["leaf_size"], a["p"])


def test_solve_resumes_from_a_saved_iterate(pkg):
    """A solve cut off after 3 iterations and resumed from its iterate (x0)
    needs fewer iterations than a fresh solve and ends at the same answer."""
    m = synth.small_molecule(4)
    with pkg.Mesh(m.panels, m.charges, m.eps_in, m.eps_out, tol=1e-8) as g:
        s_ref, st_ref = g.solve()
    with pkg.Mesh(m.panels, m.charges, m.eps_in, m.eps_out, tol=1e-8, max_iter=3) as g:
        s_cut, st_cut = g.solve(allow_noconv=True)
        assert st_cut["converged"] == 0
    with pkg.Mesh(m.panels, m.charges, m.eps_in, m.eps_out, tol=1e-8) as g:
        s_res, st_res = g.solve(x0=s_cut)
    assert st_res["converged"] == 1
    assert st_res["iterations"] < st_ref["iterations"], (st_res["iterations"], st_ref["iterations"])
    close(s_res.cpu().numpy(), s_ref.cpu().numpy(), 1e-6, inf=1e-5)
