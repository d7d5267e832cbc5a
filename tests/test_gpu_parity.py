"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle, element by element.

Tolerance (normwise relative error ||x - x_ref||_inf / ||x_ref||_inf of every output vector at
every energy: diag G^r, diag G^<, requested entries):

* TOL = 1e-10 for the complex128 path wherever the block elimination of Algorithm 1 keeps the
  contacts' broadening in every cluster block: the default tree (contact-connected dissection: x
  cut once, at the root, so every other cluster holds sites of an end plane) at any eta, and any
  tree at eta = 0.05 (every block then has Im D_i >= 0.05 I). Any indexing or sign mistake gives
  O(1) differences.
* The plain geometric tree (HSC_OPT_ORDERING = 2) at the workloads' eta = 1e-6 is the case the
  default tree exists for: its interior clusters carry no broadening but eta, and where one of them
  has a level within delta of E the downward step G_ii = D_i^{-1} + X G_UU X^T cancels terms of size
  ~1/delta^2, so any FP64 evaluation of those block steps (both engines, 3 or 4 real products, a
  numpy evaluation alike) loses digits: on the 32^3 workload 14 of 64 energies exceed 1e-4 and two
  reach 1e0 and 4e1. There the tests bound the error a posteriori by the solve's own residual
  of A G^r = I (hsc_residual): err <= RES_FACTOR x residual, RES_FACTOR = 1e2 (measured ratios
  1 to 30 on 32^3 with 8^3 leaves, up to 73 on 16^3), and by TOL_RESONANT = 1e-5 where the case was
  chosen for a mild resonance.
"""
import os

import numpy as np
import pytest

from paper_1702_05167_gb300 import hsc, workloads as W
from oracle import dense, rgf

pytestmark = pytest.mark.gpu
TOL = 1e-10
TOL_MID = 1e-8          # 32^3 at eta = 1e-6 on the default tree, any energy (measured worst 2.9e-9)
RES_MID = 1e-9          # largest residual of that solve after the default re-solve (measured 2.7e-10)
RES_CERT = 1e-11        # a residual at or below this certifies TOL on that workload
TOL_RESONANT = 1e-5
RES_FACTOR = 1e2
ETA_WELL = 0.05


def relerr(x, ref):
    return np.abs(x - ref).max() / np.abs(ref).max()


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    hsc.load()


def _dense_case(dev, leaf, energies, eta=ETA_WELL, f=(1.0, 0.0), pairs=None, tol=TOL, engine=None):
    sr, sl = W.self_energies(dev, len(energies), f)
    s = hsc.Solver(dev, leaf)
    if engine is not None:
        hsc.hsc_set_option(s.h, hsc.HSC_OPT_FP64_ENGINE, engine)
        hsc.hsc_profile(s.h, True)
    dgr, dgl, pgr, pgl = s.solve(energies, eta, sr, sl, pairs=pairs)
    if engine is not None:
        launches = {p["name"]: p["launches"] for p in hsc.hsc_profile_read(s.h)}
        emulated = sum(launches.get(c, 0) for c in ("gemm_z_ozaki", "schur_z_ozaki", "gj_update_ozaki"))
        # engine 2 runs every product list with K > 0 on the emulation, engine 1 none
        assert (emulated > 0) == (engine == 2), launches
    Hd = dev.to_scipy().toarray()
    for k, E in enumerate(energies):
        G, Gl = dense.solve(Hd, E, eta, dev.contact_unknowns(), sr[k], sl[k])
        assert relerr(dgr[k], np.diag(G)) <= tol
        assert relerr(dgl[k], np.diag(Gl)) <= tol
        if pairs is not None:
            assert relerr(pgr[k], G[pairs[:, 0], pairs[:, 1]]) <= tol
            assert relerr(pgl[k], Gl[pairs[:, 0], pairs[:, 1]]) <= tol
    s.close()


def test_tiny_8cube_matches_dense():
    cfg = W.tiny()
    _dense_case(cfg["dev"], cfg["leaf"], cfg["energies"], cfg["eta"], cfg["f"],
                pairs=W.plane_pairs(cfg["dev"], 3))


@pytest.mark.parametrize("dims,leaf,f", [((7, 5, 6), 2, (1.0, 0.3)), ((9, 4, 4), 3, (0.5, 1.0)),
                                         ((5, 5, 5), 5, (1.0, 0.0)), ((12, 3, 2), 1, (1.0, 0.0))])
def test_ragged_grids_several_energies(dims, leaf, f):
    dev = W.cubic_device(dims, W=1.0, seed=sum(dims))
    E = np.array([-2.9, -0.4, 0.0, 0.23, 1.3, 3.7])
    _dense_case(dev, leaf, E, f=f, pairs=W.plane_pairs(dev, dims[0] // 2))
    _dense_case(dev, leaf, E, eta=1e-6, f=f, pairs=W.plane_pairs(dev, dims[0] // 2))


def test_resonant_interior_block_on_the_plain_tree_and_the_default_tree():
    """At E = 0 the 7x5x6 grid (seed 18, leaves <= 2) has, on the plain geometric tree, a 4-site
    interior leaf whose local level sits within ~1e-4 of E; its block carries only eta, so no FP64
    evaluation of Algorithm 1 over that tree reaches 1e-10 (a LAPACK evaluation of the same block
    steps is off by 2.4e-7): the GPU result is bounded by TOL_RESONANT. With leaves of a few sites
    the residual does not bound it: the amplified rounding lies along the level's vector, which A
    nearly annihilates (measured: error 1.3e-7 at residual 1.5e-10). On the default
    contact-connected tree every block holds contact sites and the result meets TOL, with the
    residual at rounding level."""
    dev = W.cubic_device((7, 5, 6), W=1.0, seed=18)
    sr, sl = W.self_energies(dev, 1, (1.0, 0.3))
    G, Gl = dense.solve(dev.to_scipy().toarray(), 0.0, 1e-6, dev.contact_unknowns(), sr[0], sl[0])
    for ordering, tol in ((2, TOL_RESONANT), (0, TOL)):
        s = hsc.Solver(dev, 2, ordering=ordering)
        dgr, dgl, _, _ = s.solve(np.array([0.0]), 1e-6, sr, sl)
        res = hsc.hsc_residual(s.h, 1)[0]
        s.close()
        err = max(relerr(dgr[0], np.diag(G)), relerr(dgl[0], np.diag(Gl)))
        print(f"7x5x6 E=0 ordering {ordering}: error {err:.2e}, residual {res:.1e}")
        assert err <= tol
        if ordering == 0:
            assert relerr(dgr[0], np.diag(G)) <= RES_FACTOR * res + 1e-13


def test_multi_orbital_wire():
    dev = W.wire_device((6, 3, 2), orb=3, seed=2)
    _dense_case(dev, 2, np.array([-1.0, 0.1, 2.0]), pairs=W.plane_pairs(dev, 2))


def test_chain_degenerate_tree():
    """A 1D chain: every separator is one site; the tree degenerates towards RGF."""
    dev = W.chain_device(23, eps=np.linspace(-0.3, 0.3, 23))
    _dense_case(dev, 1, np.array([-1.5, 0.2, 1.9]), pairs=np.array([[4, 5], [11, 12], [0, 1]]))


def test_general_graph_bisection():
    dev = W.cubic_device((6, 5, 4), W=1.0, seed=11)
    sr, sl = W.self_energies(dev, 2)
    s = hsc.Solver(dev, 2, geometric=False)
    E = np.array([0.2, -1.1])
    dgr, dgl, _, _ = s.solve(E, ETA_WELL, sr, sl)
    Hd = dev.to_scipy().toarray()
    for k in range(2):
        G, Gl = dense.solve(Hd, E[k], ETA_WELL, dev.contact_unknowns(), sr[k], sl[k])
        assert relerr(dgr[k], np.diag(G)) <= TOL and relerr(dgl[k], np.diag(Gl)) <= TOL
    s.close()


def test_waves_and_device_io_agree():
    """Energies split into several workspace waves, and device-resident io, give the same bits as
    one host-io call."""
    import torch
    dev = W.cubic_device((8, 6, 5), W=1.0, seed=3)
    E = np.linspace(-3, 3, 11)
    sr, sl = W.self_energies(dev, len(E))
    free0 = torch.cuda.mem_get_info()[0]
    s = hsc.Solver(dev, 3)
    a = s.solve(E, 1e-6, sr, sl)
    # the device workspace one energy takes (block arrays, temporaries, operand images of the
    # emulated GEMMs): from the memory the first solve took, never below the analysis's block count
    per = max((free0 - torch.cuda.mem_get_info()[0]) / len(E), s.stats.bytes_per_energy)
    os.environ["HSC_WORKSPACE_GB"] = str(3.5 * per / 2**30)
    try:
        s2 = hsc.Solver(dev, 3)
        b = s2.solve(E, 1e-6, sr, sl)
        s2.close()
    finally:
        del os.environ["HSC_WORKSPACE_GB"]
    np.testing.assert_array_equal(a[0], b[0])
    np.testing.assert_array_equal(a[1], b[1])
    dv = torch.device("cuda:0")
    tE = torch.from_numpy(E).to(dv)
    tsr = torch.from_numpy(sr.view(np.float64)).to(dv)
    tsl = torch.from_numpy(sl.view(np.float64)).to(dv)
    ogr = torch.zeros((len(E), dev.n * 2), dtype=torch.float64, device=dv)
    ogl = torch.zeros_like(ogr)
    hsc.hsc_solve(s.h, tE, 1e-6, tsr, tsl, hsc.HSC_FP64, None, ogr, ogl, None, None,
                  stream=torch.cuda.current_stream().cuda_stream, io_on_device=True)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(ogr.cpu().numpy().view(np.complex128), a[0])
    np.testing.assert_array_equal(ogl.cpu().numpy().view(np.complex128), a[1])
    s.close()


def test_without_lesser_self_energy():
    dev = W.cubic_device((6, 6, 6), W=1.0, seed=4)
    E = np.array([0.7])
    sr, sl = W.self_energies(dev, 1)
    s = hsc.Solver(dev, 3)
    dgr, dgl, _, _ = s.solve(E, ETA_WELL, sr, None)
    assert dgl is None
    G, _ = dense.solve(dev.to_scipy().toarray(), E[0], ETA_WELL, dev.contact_unknowns(), sr[0], sl[0])
    assert relerr(dgr[0], np.diag(G)) <= TOL
    s.close()


def test_errors_are_reported():
    dev = W.cubic_device((4, 4, 4), seed=1)
    s = hsc.Solver(dev, 2)
    sr, sl = W.self_energies(dev, 1)
    with pytest.raises(hsc.HSCError) as ei:
        s.solve(np.array([0.1]), 1e-6, sr, sl, pairs=np.array([[0, 63]]))   # opposite corners
    assert ei.value.code == hsc.HSC_ERR_NOT_SELECTED
    s.close()


def _rgf_errors(dev, E, k, eta, sr, sl, dgr, dgl, pgr, pgl, pairs):
    Ls = dev.dims[1] * dev.dims[2] * dev.orb
    xc = (dev.dims[0] - 1) // 2
    out = rgf.sweep(dev.to_scipy(), Ls, E[k], eta, dev.contact_unknowns(), sr[k], sl[k], coupling_layers=(xc,))
    u, v = pairs[:, 0] - xc * Ls, pairs[:, 1] - (xc + 1) * Ls
    return [relerr(dgr[k], out["diag_gr"]), relerr(dgl[k], out["diag_gl"]),
            relerr(pgr[k], out["coupling_gr"][xc][u, v]), relerr(pgl[k], out["coupling_gl"][xc][u, v])]


def test_mid_32cube_sampled_against_rgf():
    """The 32^3 metric workload (eta = 1e-6, leaf_max 8, 64 energies) on the default
    contact-connected tree, against the RGF oracle at the energy with the largest residual and at
    E[26], E[27] (where the plain 8^3-leaf tree loses every digit: 3e-1 and 4e1) and E[40]:
    diag G^r, diag G^< and the x = 15/16 coupling blocks within TOL where the energy's residual is
    at most RES_CERT (the a-posteriori criterion: the errors run 1 to 30 x the residual), and
    within TOL_MID elsewhere; every energy's residual below RES_MID."""
    cfg = W.mid()
    dev = cfg["dev"]
    E = cfg["energies"]
    sr, sl = W.self_energies(dev, len(E), cfg["f"])
    s = hsc.Solver(dev, cfg["leaf"])
    assert hsc.hsc_get_option(s.h, hsc.HSC_OPT_TREE_FORM) == 1
    dgr, dgl, pgr, pgl = s.solve(E, cfg["eta"], sr, sl, pairs=cfg["pairs"])
    res = hsc.hsc_residual(s.h, len(E))
    s.close()
    print(f"32^3 residuals: median {np.median(res):.1e}, max {res.max():.1e} at E[{res.argmax()}]")
    assert res.max() <= RES_MID
    for k in sorted({int(res.argmax()), 26, 27, 40}):
        errs = _rgf_errors(dev, E, k, cfg["eta"], sr, sl, dgr, dgl, pgr, pgl, cfg["pairs"])
        print(f"32^3 E[{k}]={E[k]:+.4f} vs RGF: diag Gr {errs[0]:.2e} diag Gl {errs[1]:.2e} "
              f"Gr(15,16) {errs[2]:.2e} Gl(15,16) {errs[3]:.2e} residual {res[k]:.1e}")
        assert max(errs) <= (TOL if res[k] <= RES_CERT else TOL_MID)
    assert (res <= RES_CERT).sum() >= 16


def test_mid_32cube_plain_tree_is_bounded_by_its_residual():
    """The same workload on the plain geometric tree (8^3 leaves, HSC_OPT_ORDERING = 2, no re-solve):
    the resonant energies keep errors far above TOL, and the residual bounds them (E[26], E[27] and
    E[40] against RGF)."""
    cfg = W.mid()
    dev = cfg["dev"]
    E = cfg["energies"]
    sr, sl = W.self_energies(dev, len(E), cfg["f"])
    s = hsc.Solver(dev, cfg["leaf"], ordering=2)
    hsc.hsc_set_option(s.h, hsc.HSC_OPT_RESOLVE_DIGITS, 0)
    dgr, dgl, pgr, pgl = s.solve(E, cfg["eta"], sr, sl, pairs=cfg["pairs"])
    res = hsc.hsc_residual(s.h, len(E))
    s.close()
    for k in (26, 27, 40):
        errs = _rgf_errors(dev, E, k, cfg["eta"], sr, sl, dgr, dgl, pgr, pgl, cfg["pairs"])
        print(f"32^3 plain tree E[{k}]: diag Gr {errs[0]:.2e} diag Gl {errs[1]:.2e} residual {res[k]:.1e}")
        assert errs[0] <= RES_FACTOR * res[k] + 1e-13


def test_mid_32cube_well_conditioned_full_parity():
    """The 32^3 grid and leaves 8^3 at eta = 0.05 (bounded growth): full diag G^r, diag G^< and the
    plane-15/16 coupling blocks against the RGF oracle at 1e-10."""
    cfg = W.mid()
    dev = cfg["dev"]
    E = np.array([-3.3, 0.41])
    sr, sl = W.self_energies(dev, len(E), cfg["f"])
    s = hsc.Solver(dev, cfg["leaf"])
    dgr, dgl, pgr, pgl = s.solve(E, ETA_WELL, sr, sl, pairs=cfg["pairs"])
    s.close()
    Ls = 32 * 32
    u, v = cfg["pairs"][:, 0] - 15 * Ls, cfg["pairs"][:, 1] - 16 * Ls
    for k in range(len(E)):
        out = rgf.sweep(dev.to_scipy(), Ls, E[k], ETA_WELL, dev.contact_unknowns(), sr[k], sl[k],
                        coupling_layers=(15,))
        assert relerr(dgr[k], out["diag_gr"]) <= TOL
        assert relerr(dgl[k], out["diag_gl"]) <= TOL
        assert relerr(pgr[k], out["coupling_gr"][15][u, v]) <= TOL
        assert relerr(pgl[k], out["coupling_gl"][15][u, v]) <= TOL


def test_mixed_precision_bounded_growth():
    """HSC_MIXED (3xTF32 tensor-core products, FP32 accumulation, FP64 top levels) on a grid with
    bounded elimination growth (eta = 0.05): measured ~1e-5..1e-3 normwise; asserted at 5e-3. At
    the workloads' eta = 1e-6 the growth (~1e7) makes FP32-level products useless (see DESIGN)."""
    dev = W.cubic_device((12, 10, 8), W=1.0, seed=1)
    E = np.array([-2.1, 0.3, 1.7])
    sr, sl = W.self_energies(dev, len(E))
    s = hsc.Solver(dev, 3)
    dgr, dgl, _, _ = s.solve(E, ETA_WELL, sr, sl, precision=hsc.HSC_MIXED)
    s.close()
    Hd = dev.to_scipy().toarray()
    for k in range(len(E)):
        G, Gl = dense.solve(Hd, E[k], ETA_WELL, dev.contact_unknowns(), sr[k], sl[k])
        assert relerr(dgr[k], np.diag(G)) <= 5e-3
        assert relerr(dgl[k], np.diag(Gl)) <= 5e-3


def test_ten_orbital_wire_against_rgf():
    """The multi-orbital wire recipe (10 orbitals per site, random real-symmetric onsite blocks with
    eigenvalues in [-8, 8] eV, hopping blocks of Frobenius norm 2 eV, wide-band contacts on the end
    planes) on a 16 x 4 x 4 lattice (2560 unknowns) against the RGF oracle."""
    dev = W.wire_device((16, 4, 4), orb=10, seed=3, gamma=0.6)
    E = np.array([-1.5, 0.2, 1.9])
    sr, sl = W.self_energies(dev, len(E))
    pairs = W.plane_pairs(dev, 7)
    s = hsc.Solver(dev, 2)
    for eta, tol in ((ETA_WELL, TOL), (1e-6, TOL_RESONANT)):
        dgr, dgl, pgr, pgl = s.solve(E, eta, sr, sl, pairs=pairs)
        Ls = 4 * 4 * 10
        for k in range(len(E)):
            out = rgf.sweep(dev.to_scipy(), Ls, E[k], eta, dev.contact_unknowns(), sr[k], sl[k],
                            coupling_layers=(7,))
            assert relerr(dgr[k], out["diag_gr"]) <= tol
            assert relerr(dgl[k], out["diag_gl"]) <= tol
            u, v = pairs[:, 0] - 7 * Ls, pairs[:, 1] - 8 * Ls
            assert relerr(pgr[k], out["coupling_gr"][7][u, v]) <= tol
            assert relerr(pgl[k], out["coupling_gl"][7][u, v]) <= tol
    s.close()


def test_resonant_case_three_versus_four_products():
    """The resonant 9x4x4 case (eta = 1e-6, E = 0.23) on the plain geometric tree: with 3 or 4 real
    products per complex product (FP64 pipe) the error is the resonance's amplification of rounding,
    bounded by RES_FACTOR x the residual for both forms; on the default tree both meet TOL."""
    dev = W.cubic_device((9, 4, 4), W=1.0, seed=17)
    E = np.array([0.23])
    sr, sl = W.self_energies(dev, 1, (0.5, 1.0))
    G, Gl = dense.solve(dev.to_scipy().toarray(), 0.23, 1e-6, dev.contact_unknowns(), sr[0], sl[0])
    for ordering in (2, 0):
        for four in (0, 1):
            s = hsc.Solver(dev, 3, ordering=ordering)
            hsc.hsc_set_option(s.h, hsc.HSC_OPT_FP64_ENGINE, 1)
            hsc.hsc_set_option(s.h, hsc.HSC_OPT_COMPLEX_4M, four)
            dgr, dgl, _, _ = s.solve(E, 1e-6, sr, sl)
            res = hsc.hsc_residual(s.h, 1)[0]
            s.close()
            err = max(relerr(dgr[0], np.diag(G)), relerr(dgl[0], np.diag(Gl)))
            print(f"resonant 9x4x4 ordering {ordering}, {4 if four else 3} products: {err:.2e} (residual {res:.1e})")
            assert relerr(dgr[0], np.diag(G)) <= RES_FACTOR * res + 1e-13
            if ordering == 0:
                assert err <= TOL


@pytest.mark.parametrize("engine", [1, 2])
def test_fp64_engines_against_dense(engine):
    """Both FP64-accurate engines of the block products: the FP64 pipe (engine 1) and the FP64
    emulation on the BF16 tensor cores (engine 2, eight exact 7-bit slices per operand) must meet
    TOL on the tiny cube, a ragged grid, the multi-orbital wire and the degenerate chain, and
    TOL_RESONANT at eta = 1e-6."""
    cfg = W.tiny()
    _dense_case(cfg["dev"], cfg["leaf"], cfg["energies"], cfg["eta"], cfg["f"],
                pairs=W.plane_pairs(cfg["dev"], 3), engine=engine)
    dev = W.cubic_device((7, 5, 6), W=1.0, seed=18)
    E = np.array([-2.9, -0.4, 0.0, 0.23, 1.3, 3.7])
    _dense_case(dev, 2, E, f=(1.0, 0.3), pairs=W.plane_pairs(dev, 3), engine=engine)
    _dense_case(dev, 2, E, eta=1e-6, f=(1.0, 0.3), tol=TOL_RESONANT, engine=engine)
    wire = W.wire_device((6, 3, 2), orb=2, seed=5)
    _dense_case(wire, 3, np.array([-1.1, 0.4]), f=(1.0, 0.5), engine=engine)
    chain = W.chain_device(40, eps=np.linspace(-0.5, 0.5, 40))
    _dense_case(chain, 2, np.array([0.1, 0.9]), f=(0.2, 1.0), engine=engine)


def test_emulated_and_fp64_pipe_agree_on_mid_cube():
    """12^3 cube, leaves <= 4, 4 energies: the emulated and FP64-pipe solves agree to 1e-11 (both
    within rounding of the same block steps at eta = 0.05)."""
    dev = W.cubic_device((12, 12, 12), W=1.0, seed=3)
    E = np.array([-1.7, -0.2, 0.45, 2.2])
    sr, sl = W.self_energies(dev, len(E), (1.0, 0.0))
    out = {}
    for engine in (1, 2):
        s = hsc.Solver(dev, 4)
        hsc.hsc_set_option(s.h, hsc.HSC_OPT_FP64_ENGINE, engine)
        out[engine] = s.solve(E, ETA_WELL, sr, sl)
        s.close()
    for k in range(len(E)):
        assert relerr(out[2][0][k], out[1][0][k]) <= 1e-11
        assert relerr(out[2][1][k], out[1][1][k]) <= 1e-11


def test_growth_is_bounded_by_inverse_eta():
    """Im A = eta I + Gamma / 2 >= eta I (Eq. 1), and a Schur complement of a matrix with imaginary
    part >= eta I keeps that property, so every cluster block D_i of Algorithm 1 has
    ||D_i^{-1}||_2 <= 1 / eta: the recorded growth (largest |Re| + |Im| of an entry of D_i^{-1}) is
    positive and at most sqrt(2) / eta at every energy, for both the host and device io paths."""
    dev = W.cubic_device((9, 8, 7), W=1.0, seed=4)
    E = np.linspace(-4.0, 4.0, 17)
    sr, sl = W.self_energies(dev, len(E), (1.0, 0.5))
    for eta in (0.05, 1e-3, 1e-6):
        s = hsc.Solver(dev, 3)
        s.solve(E, eta, sr, sl)
        g = hsc.hsc_growth(s.h, len(E))
        s.close()
        assert np.all(g > 0) and np.all(g <= np.sqrt(2) / eta * (1 + 1e-6)), (eta, g.max())


def _cube16_resonant():
    """16^3 cube (W = 1, seed 0), leaves 4^3, 48 energies at eta = 1e-6: on the plain geometric
    tree some energies meet near-resonant interior clusters (error up to ~1e-2 at E = 0.1149)."""
    dev = W.cubic_device((16, 16, 16), t=-1.0, W=1.0, seed=0, gamma=0.5)
    E = np.linspace(-5.4, 5.4, 48)
    sr, sl = W.self_energies(dev, len(E), (1.0, 0.0))
    ref = np.array([rgf.sweep(dev.to_scipy(), 256, E[k], 1e-6, dev.contact_unknowns(), sr[k], sl[k])["diag_gr"]
                    for k in range(len(E))])
    return dev, E, sr, sl, ref


def test_residual_tracks_the_error():
    """hsc_residual (max |(A G^r - I)_uu| from the computed blocks) estimates the diag G^r error:
    against the RGF oracle the error stays within [1e-2, 1e2] x the residual on every energy of
    the resonant 16^3 set, and the residual is at rounding level where the growth is bounded."""
    dev, E, sr, sl, ref = _cube16_resonant()
    s = hsc.Solver(dev, 4, ordering=2)
    hsc.hsc_set_option(s.h, hsc.HSC_OPT_RESOLVE_DIGITS, 0)
    gr, _, _, _ = s.solve(E, 1e-6, sr, sl)
    r = hsc.hsc_residual(s.h, len(E))
    err = np.abs(gr - ref).max(axis=1) / np.abs(ref).max(axis=1)
    assert np.all(err <= 1e2 * r + 1e-13) and np.all(err >= 1e-2 * r - 1e-13)
    assert np.corrcoef(np.log10(err + 1e-16), np.log10(r + 1e-16))[0, 1] > 0.9
    s.solve(E[:4], ETA_WELL, sr[:4], sl[:4])
    assert np.all(hsc.hsc_residual(s.h, 4) <= 1e-12)
    s.close()


def test_resolve_on_alternate_trees():
    """HSC_OPT_RESOLVE_DIGITS = 6: energies whose residual exceeds 1e-6 are solved again on the
    alternate separator trees and the smallest-residual result is kept. No energy gets worse
    against the oracle, the worst one improves below 1e-4, the requested coupling entries stay
    available, and host and device io give identical results."""
    import torch
    dev, E, sr, sl, ref = _cube16_resonant()
    pairs = W.plane_pairs(dev, 7)
    out = {}
    for digits in (0, 6):
        s = hsc.Solver(dev, 4, ordering=2)
        hsc.hsc_set_option(s.h, hsc.HSC_OPT_RESOLVE_DIGITS, digits)
        hsc.hsc_set_option(s.h, hsc.HSC_OPT_GJ_PANEL, 16)   # the rounding this set was examined with
        out[digits] = s.solve(E, 1e-6, sr, sl, pairs=pairs)
        out[(digits, "r")] = hsc.hsc_residual(s.h, len(E))
        if digits:
            dv = torch.device("cuda")
            n, npair = dev.n, len(pairs)
            tE = torch.from_numpy(E).to(dv)
            tsr = torch.from_numpy(sr.view(np.float64)).to(dv)
            tsl = torch.from_numpy(sl.view(np.float64)).to(dv)
            ogr = torch.empty((len(E), 2 * n), dtype=torch.float64, device=dv)
            ogl, pgr, pgl = torch.empty_like(ogr), torch.empty((len(E), 2 * npair), dtype=torch.float64, device=dv), None
            pgl = torch.empty_like(pgr)
            hsc.hsc_solve(s.h, tE, 1e-6, tsr, tsl, hsc.HSC_FP64, pairs, ogr, ogl, pgr, pgl, io_on_device=True)
            torch.cuda.synchronize()
            assert np.array_equal(ogr.cpu().numpy().view(np.complex128), out[digits][0])
            assert np.array_equal(pgr.cpu().numpy().view(np.complex128), out[digits][2])
        s.close()
    e0 = np.abs(out[0][0] - ref).max(axis=1) / np.abs(ref).max(axis=1)
    e6 = np.abs(out[6][0] - ref).max(axis=1) / np.abs(ref).max(axis=1)
    assert np.all(e6 <= 1.01 * e0 + 1e-14)
    assert e0.max() > 1e-3 and e6.max() <= 1e-4
    assert np.all(out[(6, "r")] <= out[(0, "r")])
    # energies that were not re-solved are bit-identical
    same = out[(0, "r")] <= 1e-6
    assert np.array_equal(out[6][0][same], out[0][0][same])


@pytest.mark.parametrize("cluster", ["2", "4"])
def test_gauss_jordan_cluster_panels_are_bitwise_identical(cluster, monkeypatch):
    """The Gauss-Jordan panel step spread over a cluster of 2 or 4 CTAs per (matrix, energy) takes
    the same pivots and does the same arithmetic per row as the single-CTA kernel: the solve's
    outputs must be bit-identical (few energies, so the automatic choice would use clusters)."""
    dev = W.cubic_device((12, 11, 10), W=1.0, seed=6)
    E = np.array([-1.3, 0.2, 2.4])
    sr, sl = W.self_energies(dev, len(E), (1.0, 0.4))
    out = {}
    for c in ("1", cluster):
        monkeypatch.setenv("HSC_GJ_CLUSTER", c)
        s = hsc.Solver(dev, 5)
        hsc.hsc_set_option(s.h, hsc.HSC_OPT_GJ_PANEL, 16)
        out[c] = s.solve(E, ETA_WELL, sr, sl, pairs=W.plane_pairs(dev, 5))
        s.close()
    for a, b in zip(out["1"], out[cluster]):
        assert np.array_equal(a, b)
