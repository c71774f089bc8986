"""Runs bench.run_sweep's incompressible part on the CPU with stand-ins for every device call (a
Problem that returns fixed statistics, CUDA tensor methods that stay on the host), so that the
benchmark's own Python (data preparation, rows, the JSON line) is exercised without a GPU. Used by
test_bench_dryrun.py in a subprocess, since it replaces module attributes."""
import argparse
import os
import sys
import types

import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


class _Stats:
    iters, grad_evals, obj_evals, pde_solves, converged = 3, 4, 3, 7, 1
    rel_grad_inf, mismatch = 1e-4, 0.1


class _Problem:
    def __init__(self, m0, m1, **kw):
        assert kw["model"] == "incompressible" and kw["reg_order"] == 3 and kw["prec"] == "fp64"
        assert tuple(m0.shape) == (256, 256) and m0.dtype == torch.float64

    def objective(self, v):
        return 1.0

    def solve(self, v):
        return _Stats(), 0

    def stats(self):
        return _Stats()

    def deformation(self, v, u, detj):
        detj.fill_(1.0)

    def close(self):
        pass


def main():
    fake = types.ModuleType("paper_2510_08782_gb300")
    fake.Problem, fake.GaError, fake.Stats = _Problem, RuntimeError, _Stats
    fake.ga_kernel_launches = lambda: 0
    fake_build = types.ModuleType("paper_2510_08782_gb300.build")
    fake_build.build = lambda *a, **k: None
    fake.build = fake_build
    sys.modules["paper_2510_08782_gb300"] = fake
    sys.modules["paper_2510_08782_gb300.build"] = fake_build
    torch.Tensor.cuda = lambda self, *a, **k: self
    torch.cuda.set_device = lambda *a, **k: None
    torch.cuda.synchronize = lambda *a, **k: None
    host = lambda f: (lambda *a, **k: f(*a, **{x: y for x, y in k.items() if x != "device"}))
    torch.zeros, torch.empty = host(torch.zeros), host(torch.empty)
    import bench

    bench.run_sweep(argparse.Namespace(sweep_parts="inc", sweep_tol=5e-2, sweep_max_n=512))


if __name__ == "__main__":
    main()
