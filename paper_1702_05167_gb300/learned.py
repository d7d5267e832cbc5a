"""Learned energy grid: an MLP surrogate of log10 T(E) and DOS(E) places an adaptive energy grid;
the plain selected-inversion solve is both its fallback and the arbiter of every integrated quantity.

* Training data: hsc_solve on disorder realisations of a cubic device (W uniform in a range),
  observables (DOS, transmission into the right contact, lesser trace) reduced on the GPU by
  hsc_observables.
* Network: input (E, 16 disorder features) -> 3 x 256 GELU -> (log10 T, DOS per site), trained on
  the GPU by the library's own forward/backward/Adam kernels (include/hsc_mlp.h), FP32 weights,
  BF16 inference.
* Grid: the surrogate's T(E) and DOS(E) on a fine grid give the trapezoid rule's local error
  densities |T''| h^2 and |DOS''| h^2; points are placed at equal quantiles of
  rho = |T''|^(1/3)/mean + |DOS''|^(1/3)/mean + floor (equidistributing those errors), then the real
  solve runs on them.
* Arbiter: integrals (current ~ int T dE, electron count ~ int sum Im G^< dE / 2 pi, int DOS dE) on the
  adaptive grid and on a uniform grid with the same number of points are compared with a dense
  uniform reference computed by the same solver.

Everything here is host orchestration over the C ABI; no step of the solve or of the network runs
outside the library's kernels.
"""
from __future__ import annotations

import json
import time

import numpy as np

from . import hsc, workloads as W

N_FEATURES = 16
WINDOW = (-6.0, 6.0)
_trap = getattr(np, "trapezoid", None) or getattr(np, "trapz")


def disorder_features(dev) -> np.ndarray:
    """Mean and central moments 2..8 of the onsite energies (as signed k-th roots), then the mean
    absolute value and central moments 2..8 of the nearest-neighbour onsite differences."""
    eps = np.asarray(dev.meta["onsite"], dtype=np.float64)
    mu = eps.mean()
    f = [mu]
    for k in range(2, 9):
        c = np.mean((eps - mu) ** k)
        f.append(np.sign(c) * np.abs(c) ** (1.0 / k))
    H = dev.to_scipy().tocoo()
    off = H.row != H.col
    d = eps[H.row[off]] - eps[H.col[off]]
    f.append(np.mean(np.abs(d)))
    md = d.mean()
    for k in range(2, 9):
        c = np.mean((d - md) ** k)
        f.append(np.sign(c) * np.abs(c) ** (1.0 / k))
    return np.asarray(f, dtype=np.float64)


def solve_observables(solver, E, eta=1e-6, f=(1.0, 0.0), precision=hsc.HSC_FP64):
    """DOS, T (into the right contact) and sum Im G^< at energies E, via hsc_solve + hsc_observables
    on device-resident buffers. Returns numpy arrays (dos, trans, lesser_trace)."""
    import torch
    dev = solver.dev
    E = np.ascontiguousarray(E, dtype=np.float64)
    sr, sl = W.self_energies(dev, len(E), f)
    tE = torch.from_numpy(E).cuda()
    tsr = torch.from_numpy(sr.view(np.float64)).cuda()
    tsl = torch.from_numpy(sl.view(np.float64)).cuda()
    gr = torch.empty((len(E), 2 * dev.n), dtype=torch.float64, device="cuda")
    gl = torch.empty_like(gr)
    out = torch.empty((len(E), 3), dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    hsc.hsc_solve(solver.h, tE, eta, tsr, tsl, precision, None, gr, gl, None, None, stream=stream,
                  io_on_device=True)
    hsc.hsc_observables(solver.h, gr, gl, tsr, 1, out, stream=stream)
    o = out.cpu().numpy()
    return o[:, 0], o[:, 1], o[:, 2]


def make_dataset(dims, n_real, n_E, W_range=(0.5, 2.0), seed=0, eta=1e-6, leaf=8):
    """Features/targets from n_real disorder realisations x n_E random energies each."""
    rng = np.random.default_rng(seed)
    X, Y = [], []
    n_sites = int(np.prod(dims))
    for r in range(n_real):
        Wr = rng.uniform(*W_range)
        dev = W.cubic_device(dims, W=Wr, seed=seed * 100003 + r)
        feats = disorder_features(dev)
        E = np.sort(rng.uniform(WINDOW[0], WINDOW[1], n_E))
        s = hsc.Solver(dev, leaf)
        dos, T, _ = solve_observables(s, E, eta)
        s.close()
        X.append(np.column_stack([E, np.tile(feats, (n_E, 1))]))
        Y.append(np.column_stack([np.log10(np.maximum(T, 1e-6)), dos / n_sites]))
    return np.concatenate(X), np.concatenate(Y)


class Surrogate:
    """MLP (E, 16 features) -> (log10 T, DOS per site) with input/target standardisation."""

    def __init__(self, width=256, hidden=3, max_batch=8192, seed=0):
        self.net = hsc.MLP(1 + N_FEATURES, width, hidden, 2, max_batch)
        self.max_batch = max_batch
        rng = np.random.default_rng(seed)
        p = []
        dims = [1 + N_FEATURES] + [width] * hidden + [2]
        for di, do in zip(dims[:-1], dims[1:]):
            p.append(rng.standard_normal(di * do) * np.sqrt(2.0 / di))
            p.append(np.zeros(do))
        self.net.set_params(np.concatenate(p).astype(np.float32))
        self.xm = self.xs = self.ym = self.ys = None

    def fit(self, X, Y, steps=3000, lr=1e-3, batch=1024, seed=0):
        import torch
        self.xm, self.xs = X.mean(0), X.std(0) + 1e-9
        self.ym, self.ys = Y.mean(0), Y.std(0) + 1e-9
        Xn = torch.from_numpy(((X - self.xm) / self.xs).astype(np.float32)).cuda()
        Yn = torch.from_numpy(((Y - self.ym) / self.ys).astype(np.float32)).cuda()
        rng = np.random.default_rng(seed)
        hist = []
        n = len(X)
        batch = min(batch, n, self.max_batch)
        for it in range(steps):
            idx = torch.from_numpy(rng.choice(n, batch, replace=False)).cuda()
            xb, yb = Xn[idx].contiguous(), Yn[idx].contiguous()
            step_lr = lr * 0.5 * (1 + np.cos(np.pi * it / steps))
            loss = self.net.loss_grad(xb, yb)
            self.net.adam(step_lr)
            if it % 100 == 0 or it == steps - 1:
                hist.append((it, loss))
        torch.cuda.synchronize()
        return hist

    def predict(self, X, bf16=True):
        import torch
        out = np.empty((len(X), 2))
        for a in range(0, len(X), self.max_batch):
            xb = torch.from_numpy(((X[a:a + self.max_batch] - self.xm) / self.xs).astype(np.float32)).cuda()
            yb = torch.empty((len(xb), 2), dtype=torch.float32, device="cuda")
            self.net.forward(xb, yb, bf16=bf16)
            out[a:a + len(xb)] = yb.cpu().numpy() * self.ys + self.ym
        return out

    def close(self):
        self.net.close()


def adaptive_grid(sur, feats, n_points, fine=8192, floor=1.0, window=WINDOW):
    """Energies at equal quantiles of rho = |T''|^(1/3)/s_T + |D''|^(1/3)/s_D + floor, with T and D
    the surrogate's transmission and DOS on a fine uniform grid (endpoints included). Each curvature
    term is normalised by s = max(its mean, (range / window^2)^(1/3)): the curvature a function of
    that range would have if it bent once over the window. A function with no curvature (constant
    or linear), whose discrete second derivative is rounding noise, then adds ~nothing instead of
    having its noise scaled to O(1) by its own tiny mean."""
    Ef = np.linspace(window[0], window[1], fine)
    pred = sur.predict(np.column_stack([Ef, np.tile(feats, (fine, 1))]))
    T = 10.0 ** pred[:, 0]
    Dn = pred[:, 1]
    h = Ef[1] - Ef[0]
    L = window[1] - window[0]
    d2 = lambda y: np.abs(np.gradient(np.gradient(y, h), h)) ** (1 / 3)
    scale = lambda c, y: max(c.mean(), (np.ptp(y) / (L * L)) ** (1 / 3), 1e-300)
    a, b = d2(T), d2(Dn)
    rho = a / scale(a, T) + b / scale(b, Dn) + floor
    cdf = np.concatenate([[0.0], np.cumsum(0.5 * (rho[1:] + rho[:-1]) * h)])
    cdf /= cdf[-1]
    return np.interp(np.linspace(0, 1, n_points), cdf, Ef)


def integrals(E, dos, T, ltr):
    return {"current_int_T_dE": float(_trap(T, E)),
            "electrons_int_ImGless_dE_over_2pi": float(_trap(ltr, E) / (2 * np.pi)),
            "int_DOS_dE": float(_trap(dos, E))}


def evaluate(dev, sur, n_points, n_ref, eta=1e-6, leaf=8, precision=hsc.HSC_FP64):
    """Integrals on the adaptive and on the uniform n_points grids against a uniform n_ref reference,
    all computed by hsc_solve (the arbiter)."""
    feats = disorder_features(dev)
    s = hsc.Solver(dev, leaf)
    res = {}
    grids = {"reference": np.linspace(WINDOW[0], WINDOW[1], n_ref),
             "uniform": np.linspace(WINDOW[0], WINDOW[1], n_points),
             "adaptive": adaptive_grid(sur, feats, n_points)}
    for name, E in grids.items():
        dos, T, ltr = solve_observables(s, E, eta, precision=precision)
        res[name] = integrals(E, dos, T, ltr)
    s.close()
    out = {"points": n_points, "reference_points": n_ref, "integrals": res, "rel_err": {}, "gain": {}}
    for q in res["reference"]:
        ref = res["reference"][q]
        eu = abs(res["uniform"][q] - ref) / abs(ref)
        ea = abs(res["adaptive"][q] - ref) / abs(ref)
        out["rel_err"][q] = {"uniform": eu, "adaptive": ea}
        out["gain"][q] = eu / ea if ea > 0 else float("inf")
    return out


def main(argv=None):
    import argparse
    import torch
    p = argparse.ArgumentParser(description="learned energy grid: train the surrogate, check the grid against plain solves")
    p.add_argument("--train-dims", type=int, default=16)
    p.add_argument("--n-real", type=int, default=64)
    p.add_argument("--n-e", type=int, default=64)
    p.add_argument("--steps", type=int, default=3000)
    p.add_argument("--target-dims", type=int, default=24)
    p.add_argument("--points", type=int, default=256)
    p.add_argument("--ref", type=int, default=2048)
    p.add_argument("--seed", type=int, default=0)
    a = p.parse_args(argv)
    torch.cuda.set_device(0)
    t0 = time.time()
    X, Y = make_dataset((a.train_dims,) * 3, a.n_real, a.n_e, seed=a.seed)
    t1 = time.time()
    sur = Surrogate(seed=a.seed)
    hist = sur.fit(X, Y, steps=a.steps, seed=a.seed)
    t2 = time.time()
    Xv, Yv = make_dataset((a.train_dims,) * 3, 4, a.n_e, seed=a.seed + 777)
    pv = sur.predict(Xv)
    val = {"rmse_log10T": float(np.sqrt(np.mean((pv[:, 0] - Yv[:, 0]) ** 2))),
           "rmse_dos_per_site": float(np.sqrt(np.mean((pv[:, 1] - Yv[:, 1]) ** 2))),
           "std_log10T": float(Yv[:, 0].std()), "std_dos_per_site": float(Yv[:, 1].std())}
    target = W.cubic_device((a.target_dims,) * 3, W=1.0, seed=a.seed + 4242)
    ev = evaluate(target, sur, a.points, a.ref)
    t3 = time.time()
    sur.close()
    print(json.dumps({"train": {"dims": [a.train_dims] * 3, "solves": len(X), "seconds_data": t1 - t0,
                                "seconds_fit": t2 - t1, "loss": hist[-1][1], "loss_first": hist[0][1]},
                      "validation": val, "target": {"dims": [a.target_dims] * 3, **ev},
                      "seconds_eval": t3 - t2}))


if __name__ == "__main__":
    main()
