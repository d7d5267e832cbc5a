"""Batched multi-device solve in one CUDA graph (hsc_solve_batch) and the autotuner (hsc_tune)."""
import numpy as np
import pytest

from paper_1702_05167_gb300 import hsc, workloads as W
from oracle import dense

pytestmark = pytest.mark.gpu
DIMS = [(6, 5, 4), (8, 6, 5), (5, 5, 7)]


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no GPU")
    return t


def _dev_tensor(torch, a):
    return torch.from_numpy(np.ascontiguousarray(a).view(np.float64)).cuda()


def test_batch_graph_matches_single_solves(torch):
    """Three cuboids with uneven separators and different energy counts in one graph launch give
    the same bits as three separate hsc_solve calls; the cached graph replays identically; every
    item matches the dense oracle."""
    solvers, items, refs = [], [], []
    for k, d in enumerate(DIMS):
        dev = W.cubic_device(d, W=1.0, seed=1000 + k)
        E = np.linspace(-3, 3, 3 + 2 * k) + 0.01 * k
        sr, sl = W.self_energies(dev, len(E))
        pairs = W.plane_pairs(dev, d[0] // 2)
        s = hsc.Solver(dev, 3)
        refs.append(s.solve(E, 0.05, sr, sl, pairs=pairs))
        solvers.append(s)
        n, npair = dev.n, len(pairs)
        items.append(dict(h=s.h, E=torch.from_numpy(E).cuda(), sigma_r=_dev_tensor(torch, sr),
                          sigma_less=_dev_tensor(torch, sl), pairs=pairs,
                          diag_gr=torch.zeros((len(E), 2 * n), dtype=torch.float64, device="cuda"),
                          diag_gl=torch.zeros((len(E), 2 * n), dtype=torch.float64, device="cuda"),
                          req_gr=torch.zeros((len(E), 2 * npair), dtype=torch.float64, device="cuda"),
                          req_gl=torch.zeros((len(E), 2 * npair), dtype=torch.float64, device="cuda")))
    stream = torch.cuda.current_stream().cuda_stream
    for use_graph, reps in ((True, 2), (False, 1)):
        for _ in range(reps):
            for it in items:
                for key in ("diag_gr", "diag_gl", "req_gr", "req_gl"):
                    it[key].zero_()
            hsc.hsc_solve_batch(items, 0.05, hsc.HSC_FP64, stream=stream, use_graph=use_graph)
            for it, ref in zip(items, refs):
                for key, r in zip(("diag_gr", "diag_gl", "req_gr", "req_gl"), ref):
                    got = it[key].cpu().numpy().view(np.complex128)
                    np.testing.assert_array_equal(got, r)
    # and every item against the dense definition (Eqs. 1-2) at 1e-10
    for k, (d, it) in enumerate(zip(DIMS, items)):
        dev = W.cubic_device(d, W=1.0, seed=1000 + k)
        E = it["E"].cpu().numpy()
        sr, sl = W.self_energies(dev, len(E))
        pairs = it["pairs"]
        Hd = dev.to_scipy().toarray()
        gr = it["diag_gr"].cpu().numpy().view(np.complex128)
        gl = it["diag_gl"].cpu().numpy().view(np.complex128)
        pg = it["req_gr"].cpu().numpy().view(np.complex128)
        for e in range(len(E)):
            G, Gl = dense.solve(Hd, E[e], 0.05, dev.contact_unknowns(), sr[e], sl[e])
            for x, ref in ((gr[e], np.diag(G)), (gl[e], np.diag(Gl)), (pg[e], G[pairs[:, 0], pairs[:, 1]])):
                assert np.abs(x - ref).max() <= 1e-10 * np.abs(ref).max()
    for s in solvers:
        s.close()


def test_autotuner_chooses_and_caches(torch, tmp_path):
    dev = W.cubic_device((12, 10, 9), W=1.0, seed=3)
    E = np.array([-1.0, 0.4])
    sr, sl = W.self_energies(dev, len(E))
    s = hsc.Solver(dev, 4)
    cache = tmp_path / "tune.jsonl"
    r = hsc.hsc_tune(s.h, E, 0.05, sr, sl, cache_path=cache)
    assert r["leaf_max"] in (4, 6, 8) and r["gj_panel"] in (16, 32, 64) and r["n_tried"] == 9
    assert not r["from_cache"] and r["ms_per_energy"] > 0
    assert hsc.hsc_get_option(s.h, hsc.HSC_OPT_LEAF) == r["leaf_max"]
    assert hsc.hsc_get_option(s.h, hsc.HSC_OPT_GJ_PANEL) == r["gj_panel"]
    r2 = hsc.hsc_tune(s.h, E, 0.05, sr, sl, cache_path=cache)
    assert r2["from_cache"] and r2["leaf_max"] == r["leaf_max"] and r2["gj_panel"] == r["gj_panel"]
    dgr, dgl, _, _ = s.solve(E, 0.05, sr, sl)
    Hd = dev.to_scipy().toarray()
    for k in range(len(E)):
        G, Gl = dense.solve(Hd, E[k], 0.05, dev.contact_unknowns(), sr[k], sl[k])
        assert np.abs(dgr[k] - np.diag(G)).max() / np.abs(np.diag(G)).max() <= 1e-10
        assert np.abs(dgl[k] - np.diag(Gl)).max() / np.abs(np.diag(Gl)).max() <= 1e-10
    s.close()


@pytest.mark.parametrize("nb", [1, 5, 32, 64])
def test_panel_width_option_keeps_results(torch, nb):
    dev = W.cubic_device((7, 6, 5), W=1.0, seed=2)
    E = np.array([0.7])
    sr, sl = W.self_energies(dev, 1)
    s = hsc.Solver(dev, 3)
    ref = s.solve(E, 0.05, sr, sl)
    hsc.hsc_set_option(s.h, hsc.HSC_OPT_GJ_PANEL, nb)
    got = s.solve(E, 0.05, sr, sl)
    s.close()
    for a, b in zip(got[:2], ref[:2]):
        assert np.abs(a - b).max() / np.abs(b).max() <= 1e-12


@pytest.mark.parametrize("nb,wide", [(32, 0), (32, 128), (16, 64), (8, 40), (5, 12)])
def test_nested_gauss_jordan_blocking_against_dense(torch, nb, wide):
    """Nested blocking of the cluster inversions (HSC_OPT_GJ_WIDE: panels of HSC_OPT_GJ_PANEL width
    reduced inside a wide panel, then one trailing product with K = the wide width): the same
    D_i^{-1} as unnested blocking, on leaves of 7 x 8 x 8 = 448 unknowns (a ragged last wide panel
    for every width) and separators of other sizes; against the dense definition at 1e-10."""
    dev = W.cubic_device((15, 16, 16), W=1.0, seed=4)
    E = np.array([-1.7, 0.35])
    sr, sl = W.self_energies(dev, len(E))
    s = hsc.Solver(dev, 8)
    assert hsc.hsc_get_option(s.h, hsc.HSC_OPT_TREE_FORM) == 1
    hsc.hsc_set_option(s.h, hsc.HSC_OPT_GJ_PANEL, nb)
    hsc.hsc_set_option(s.h, hsc.HSC_OPT_GJ_WIDE, wide)
    assert hsc.hsc_get_option(s.h, hsc.HSC_OPT_GJ_WIDE) == wide
    dgr, dgl, _, _ = s.solve(E, 0.05, sr, sl)
    s.close()
    Hd = dev.to_scipy().toarray()
    for k in range(len(E)):
        G, Gl = dense.solve(Hd, E[k], 0.05, dev.contact_unknowns(), sr[k], sl[k])
        assert np.abs(dgr[k] - np.diag(G)).max() / np.abs(np.diag(G)).max() <= 1e-10
        assert np.abs(dgl[k] - np.diag(Gl)).max() / np.abs(np.diag(Gl)).max() <= 1e-10
