"""Time one complex128 GEMM C = A B (M x K times K x N, random normal entries) on the library's
block-product engines through the C ABI's debug entry (include/hsc_debug.h), and report the error
against torch's complex128 product:

    python -m paper_1702_05167_gb300.gemm_bench --m 2048 --n 2048 --k 2048 --engine 4 --reps 5

engine 0: FP64 tensor pipe (3 real products), 3: FP64 pipe with 4 real products, 4: FP64 emulation
on the BF16 tensor cores. Each call includes the engine's own allocation of its operand images;
the figure is the best of `reps` wall-clock calls.
"""
import argparse
import ctypes
import time


def main():
    import torch
    from paper_1702_05167_gb300 import hsc
    p = argparse.ArgumentParser()
    p.add_argument("--m", type=int, default=2048)
    p.add_argument("--n", type=int, default=2048)
    p.add_argument("--k", type=int, default=2048)
    p.add_argument("--engine", type=int, default=4, choices=[0, 3, 4])
    p.add_argument("--reps", type=int, default=5)
    a = p.parse_args()
    L = hsc.load()
    L.hsc_debug_gemm.argtypes = [ctypes.c_int32] * 6 + [ctypes.c_void_p, ctypes.c_int32] * 4 + \
        [ctypes.c_double] * 4 + [ctypes.c_void_p]
    L.hsc_debug_gemm.restype = ctypes.c_int
    dv = torch.device("cuda")
    g = torch.Generator(device=dv).manual_seed(0)
    A = torch.randn(a.m, 2 * a.k, dtype=torch.float64, device=dv, generator=g)
    B = torch.randn(a.k, 2 * a.n, dtype=torch.float64, device=dv, generator=g)
    C = torch.zeros(a.m, 2 * a.n, dtype=torch.float64, device=dv)
    best = float("inf")
    for _ in range(a.reps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rc = L.hsc_debug_gemm(a.engine, 0, 0, a.m, a.n, a.k, A.data_ptr(), a.k, B.data_ptr(), a.n,
                              C.data_ptr(), a.n, None, 0, 1.0, 0.0, 0.0, 0.0, None)
        torch.cuda.synchronize()
        if rc != 0:
            raise RuntimeError(hsc.hsc_last_error())
        best = min(best, time.perf_counter() - t0)
    ref = torch.view_as_complex(A.view(a.m, a.k, 2)) @ torch.view_as_complex(B.view(a.k, a.n, 2))
    err = ((torch.view_as_complex(C.view(a.m, a.n, 2)) - ref).abs().max() / ref.abs().max()).item()
    flops = 8.0 * a.m * a.n * a.k
    print(f"engine {a.engine} {a.m}x{a.n}x{a.k}: {best * 1e3:.3f} ms, {flops / best / 1e12:.2f} TFLOP/s "
          f"(8 flops per complex multiply-add), max |C - ref| / max |ref| = {err:.2e}")


if __name__ == "__main__":
    main()
