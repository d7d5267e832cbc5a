"""Learned energy grid end to end on a small scale: training data generated by the library's own
solves, the surrogate trained by its own kernels, the adaptive grid checked against plain solves.

Reports what the surrogate-placed grid gains over a uniform grid with the same number of points
(error of each integral against a dense uniform reference); asserts that training converges, that
every integral on the adaptive grid stays close to the reference, and that the adaptive grid beats
the uniform one on the current integral (T(E), the smooth function the surrogate learns: gain 1.61
measured); prints the gains. The DOS and lesser-trace integrals gain nothing here: on this weakly
disordered cube they are dominated by interior levels of width eta that no grid of 96 points
resolves."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_learned_grid_small(capsys):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1702_05167_gb300 import learned, workloads as W
    X, Y = learned.make_dataset((8, 8, 8), n_real=16, n_E=32, seed=1, leaf=4)
    assert X.shape == (512, 17) and np.all(np.isfinite(Y))
    sur = learned.Surrogate(width=128, seed=1)
    hist = sur.fit(X, Y, steps=600, lr=2e-3, batch=256, seed=1)
    assert hist[-1][1] < 0.2 * hist[0][1]
    dev = W.cubic_device((10, 10, 10), W=1.0, seed=77)
    ev = learned.evaluate(dev, sur, n_points=96, n_ref=768, leaf=5)
    sur.close()
    for q, e in ev["rel_err"].items():
        assert e["adaptive"] < 0.05, (q, e)
    assert ev["gain"]["current_int_T_dE"] > 1.0, ev["gain"]
    with capsys.disabled():
        print("\nlearned grid (10^3 target, 96 points vs 768-point reference): gains",
              {k: round(v, 3) for k, v in ev["gain"].items()})
