"""Time the self-consistent dephasing loop (hsc_scba) on a cubic device whose interior is one
scattering contact, with device-resident inputs, and report the loop's cost against one plain
solve of the same device without dephasing:

    python -m paper_1702_05167_gb300.scba_bench --dims 16 16 16 --energies 16 --d0 0.1

Prints one JSON line: solves made, last delta, loop time, time per solve, the plain solve's time,
and the largest relative current imbalance |I_L + I_R + I_eta| / I_L over the energies.
"""
import argparse
import json

import numpy as np


def main():
    import torch
    from paper_1702_05167_gb300 import hsc, workloads as W
    p = argparse.ArgumentParser()
    p.add_argument("--dims", type=int, nargs=3, default=[16, 16, 16])
    p.add_argument("--energies", type=int, default=16)
    p.add_argument("--leaf", type=int, default=8)
    p.add_argument("--d0", type=float, default=0.1)
    p.add_argument("--mix", type=float, default=0.7)
    p.add_argument("--tol", type=float, default=1e-10)
    p.add_argument("--max-iter", type=int, default=200)
    p.add_argument("--eta", type=float, default=1e-6)
    a = p.parse_args()
    dv = torch.device("cuda")
    st = torch.cuda.current_stream()
    base = W.cubic_device(tuple(a.dims), seed=0)
    dev = W.with_scattering_contact(base)
    n_E, n = a.energies, dev.n
    E = np.linspace(-3.0, 3.0, n_E)

    def up(x):
        return torch.from_numpy(np.ascontiguousarray(x).view(np.float64)).to(dv)

    tE = torch.from_numpy(E).to(dv)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    # plain solve of the device without dephasing (contacts only), for scale
    sr0, sl0 = W.self_energies(base, n_E)
    s0 = hsc.Solver(base, a.leaf)
    o0 = torch.zeros((n_E, 2 * n), dtype=torch.float64, device=dv)
    o1 = torch.zeros_like(o0)
    t0r, t0l = up(sr0), up(sl0)
    for k in range(2):
        ev[0].record(st)
        hsc.hsc_solve(s0.h, tE, a.eta, t0r, t0l, hsc.HSC_FP64, None, o0, o1, None, None,
                      stream=st.cuda_stream, io_on_device=True)
        ev[1].record(st)
    torch.cuda.synchronize()
    plain_ms = ev[0].elapsed_time(ev[1])
    s0.close()
    sr, sl = W.self_energies(dev, n_E, f=(1.0, 0.0, 0.0))
    s = hsc.Solver(dev, a.leaf)
    ogr = torch.zeros((n_E, 2 * n), dtype=torch.float64, device=dv)
    ogl = torch.zeros_like(ogr)
    tsr, tsl = up(sr), up(sl)
    hsc.hsc_scba(s.h, tE, a.eta, tsr, tsl, a.d0, a.mix, a.tol, 1, hsc.HSC_FP64, ogr, ogl,
                 stream=st.cuda_stream, io_on_device=True)     # warm-up: workspace, schedule
    ev[2].record(st)
    it, dl = hsc.hsc_scba(s.h, tE, a.eta, tsr, tsl, a.d0, a.mix, a.tol, a.max_iter, hsc.HSC_FP64, ogr,
                          ogl, stream=st.cuda_stream, io_on_device=True)
    ev[3].record(st)
    torch.cuda.synchronize()
    loop_ms = ev[2].elapsed_time(ev[3])
    s.close()
    gr = ogr.cpu().numpy().view(np.complex128)
    gl = ogl.cpu().numpy().view(np.complex128)
    cid = base.contact_of_unknown()
    idx = base.contact_unknowns()
    g = base.gamma[cid]
    A = -2.0 * gr.imag
    gn = gl.imag
    i_l = (g * (A[:, idx] - gn[:, idx]))[:, cid == 0].sum(axis=1)
    i_r = -(g * gn[:, idx])[:, cid == 1].sum(axis=1)
    i_eta = -2.0 * a.eta * gn.sum(axis=1)
    imb = float((np.abs(i_l + i_r + i_eta) / np.abs(i_l)).max())
    print(json.dumps({"workload": f"cubic{a.dims[0]}x{a.dims[1]}x{a.dims[2]} dephasing d0={a.d0}",
                      "energies": n_E, "solves": it, "delta": dl, "loop_ms": round(loop_ms, 2),
                      "ms_per_solve": round(loop_ms / it, 2), "plain_solve_ms": round(plain_ms, 2),
                      "current_imbalance_max": imb}), flush=True)


if __name__ == "__main__":
    main()
