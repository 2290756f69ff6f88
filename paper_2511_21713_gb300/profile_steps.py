"""Runs single steps of the solve a few times, for focused profiler captures.

  python -m paper_2511_21713_gb300.profile_steps --step farfield_f32 --reps 2
  steps: farfield_f32 | farfield_ff | farfield_f64 (V then K on Gamma_m and Gamma_s),
         assemble (HS Jacobian + load), omega (batched omega evaluation, 16 values),
         gmres (one block-preconditioned GMRES solve at 1e-6)

Workload: the multi-charge sphere of the bench (72,036 vertices, 408,000 tets,
8000 + 8000 triangles) or --workload small (the single-charge sphere).  Prints
the wall time of each repetition; under a profiler, capture with -k on the
kernel of interest.
"""
import argparse
import os
import sys
import time

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))


def main():
    import numpy as np
    import torch
    from paper_2511_21713_gb300 import build, inputs, pbfb
    ap = argparse.ArgumentParser()
    ap.add_argument("--step", default="farfield_f32")
    ap.add_argument("--reps", type=int, default=2)
    ap.add_argument("--workload", default="multi_charge_sphere", choices=["multi_charge_sphere", "small"])
    a = ap.parse_args()
    build.build()
    case = inputs.multi_charge_sphere() if a.workload == "multi_charge_sphere" else inputs.single_charge_sphere()
    m = pbfb.Mesh.from_case(case)
    m.charges_set(case.q_xyz, case.q_z)
    prec = {"farfield_f32": pbfb.MIXED, "farfield_ff": pbfb.FLOAT2, "farfield_f64": pbfb.FP64}.get(a.step, pbfb.MIXED)
    m.set_params(case.eps_in, case.eps_out, case.kappa, case.T, prec)
    dev = torch.device("cuda")
    r = np.linalg.norm(case.xyz, axis=1)
    u = torch.as_tensor(4.0 * np.exp(-0.2 * (r - r.min())), device=dev)
    for rep in range(a.reps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        if a.step.startswith("farfield"):
            for which, n in ((pbfb.GAMMA_M, m.n_m), (pbfb.GAMMA_S, m.n_s)):
                x = torch.ones(n, dtype=torch.float64, device=dev)
                y = torch.zeros_like(x)
                m.bem_apply(which, 0, x, y)
                m.bem_apply(which, 1, x, y)
        elif a.step == "assemble":
            N = torch.zeros(m.n_v, dtype=torch.float64, device=dev)
            m.assemble(pbfb.HS, u, N)
        elif a.step == "omega":
            du = 0.1 * u
            c = torch.ones(m.n, dtype=torch.float64, device=dev)
            m.omega_eval(pbfb.HS, u, du, c, c, np.linspace(0.25, 4.0, 16))
        elif a.step == "gmres":
            m.assemble(pbfb.HS, u)
            b = torch.ones(m.n, dtype=torch.float64, device=dev)
            x = torch.zeros_like(b)
            m.gmres(b, x, 1e-6, precond=pbfb.BLOCK, inner_iters=30)
        else:
            raise SystemExit(f"unknown step {a.step}")
        torch.cuda.synchronize()
        print(f"{a.step} rep {rep}: {1e3 * (time.perf_counter() - t0):.2f} ms", flush=True)
    m.close()


if __name__ == "__main__":
    main()
