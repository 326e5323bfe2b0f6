"""Small, self-contained workloads for kernel profiling (ncu) and phase timing.

    python -m paper_2303_02156_gb300.profile_cases eval   --size 40 [--reps 10]
    python -m paper_2303_02156_gb300.profile_cases newton --size 40
    python -m paper_2303_02156_gb300.profile_cases tetho  --size 12 [--order 3]

`eval`: the SNH cube (size^3 cells, 6 tets per cell, jittered state, random
materials) evaluated with E+g+H+projection+assembly; prints the per-phase
milliseconds from the library's phase timer and the projection counters.
`newton`: one backward-Euler Newton step of the same cube from rest under
gravity (dt 5 ms), twice; prints Newton and PCG iteration counts.
`tetho`: 10- or 20-node Lagrange tets on a size^3 cube, a few E+g+H passes.

Each run holds well under a few GB on the device, so a capture of one or two
launches of its kernels ends within a minute or two.
"""
import argparse
import ctypes as C
import time

import numpy as np
import torch

from . import scenes, sx
from .scene import Context, Scene


def _snh_cube(ctx, n, gravity):
    m = scenes.kuhn_box(n, n, n, h=1.0 / n, seed=2)
    E, nu = scenes.material_random(m["tets"].shape[0], seed=2)
    s = Scene(ctx, m["X"])
    s.add_snh(m["tets"], E, nu, 1000.0)
    s.set_pinned(m["pinned"])
    if gravity:
        s.set_gravity((0.0, 0.0, -9.81))
    s.finalize()
    return s, m


def run_eval(n, reps):
    ctx = Context(0)
    s, m = _snh_cube(ctx, n, False)
    s.set_state(x=scenes.jitter_state(m["X"], 0.02 / n, seed=5))
    for _ in range(3):
        s.eval()
    ms = (C.c_double * 9)()
    ln = (C.c_int64 * 9)()
    sx.sx_profile(ctx.h, 1)
    sx.sx_profile_read(ctx.h, None, None, 1)
    for _ in range(reps):
        s.eval()
    sx.sx_profile_read(ctx.h, ms, ln, 1)
    sx.sx_profile(ctx.h, 0)
    print({sx.PHASES[i]: round(ms[i] / reps, 3) for i in range(5)}, s.stats(), flush=True)


def run_newton(n):
    ctx = Context(0)
    s, m = _snh_cube(ctx, n, True)
    for _ in range(2):
        s.set_state(x=m["X"], v=np.zeros_like(m["X"]))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rc, r = s.newton_step(0.005, raise_on_error=False, newton_tol=1e-8, pcg_tol=1e-10)
        torch.cuda.synchronize()
        print("rc", rc, "ms %.1f" % ((time.perf_counter() - t0) * 1e3),
              r["newton_iters"], r["pcg_iters"], flush=True)


def run_tetho(n, order):
    m = scenes.kuhn_box_ho(n, n, n, order, h=1.0 / n, seed=2)
    E, nu = scenes.material_random(m["tets"].shape[0], seed=2)
    ctx = Context(0)
    s = Scene(ctx, m["X"])
    rule = scenes.tet_rule_4point() if order == 2 else scenes.tet_rule_conical(3)
    s.add_tet_ho(order, m["tets"], E, nu, 1000.0, rule)
    s.set_pinned(m["pinned"])
    s.finalize()
    s.set_state(x=scenes.jitter_state(m["X"], 0.02 / n / order, seed=5))
    for _ in range(4):
        s.eval(sx.SX_EGH, False, sx.SX_FP64)
    torch.cuda.synchronize()
    print("ok", s.stats(), flush=True)


def main(argv=None):
    p = argparse.ArgumentParser()
    p.add_argument("case", choices=["eval", "newton", "tetho"])
    p.add_argument("--size", type=int, default=40)
    p.add_argument("--reps", type=int, default=10)
    p.add_argument("--order", type=int, default=3, choices=[2, 3])
    a = p.parse_args(argv)
    if a.case == "eval":
        run_eval(a.size, a.reps)
    elif a.case == "newton":
        run_newton(a.size)
    else:
        run_tetho(a.size, a.order)


if __name__ == "__main__":
    main()
