"""Writes tests/golden/*.json from the CPU oracle only (never from the CUDA path).

multi_charge_sphere.json: the oracle's solve of the 200-charge sphere (radius 12,
shell to 24, nu = 20, 17 layers; 72,036 vertices, 408,000 tets, 8000 + 8000
triangles; eps 2/80, 0.1 M, 300 K) at the paper's default tolerances and at tight
ones: energies, iteration traces (Newton, GMRES and omega-evaluation counts), the
solution at a seeded sample of unknowns, and the oracle's own wall times (set-up
and each solve), which calibrate the bench's sampled CPU-baseline model.

Run: python tests/golden/make_golden.py   (about 10-20 minutes on 8 cores)
"""
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from paper_2511_21713_gb300 import inputs  # noqa: E402
from oracle import pb  # noqa: E402


def main():
    case = inputs.multi_charge_sphere()
    t0 = time.time()
    P = pb.Problem(case)
    t_setup = time.time() - t0
    out = dict(case=case.name, n_v=int(P.nv), n_m=int(P.nm), n_s=int(P.ns), n_t=int(case.n_t),
               kappa=case.kappa, setup_s=t_setup)
    rng = np.random.default_rng(12345)
    sample = np.sort(rng.choice(P.n, 64, replace=False))
    out['sample_index'] = sample.tolist()
    for name, opts in (('default', pb.Opts()),
                       ('tight', pb.Opts(tol_gmres0=1e-10, tol_gmres=1e-10, tol_nl=1e-7))):
        t = time.time()
        R = pb.solve(P, opts)
        out[name] = dict(total=R.total, LC=R.LC, NC=R.NC, dG_ion=R.dG_ion, newton_iters=R.newton_iters,
                         gmres=[int(g) for g in R.trace['gmres']], linear_gmres=int(R.trace['linear_gmres']),
                         omega=[float(w) for w in R.trace['omega']], e=[float(v) for v in R.trace['e']],
                         omega_evals=[int(v) for v in R.trace['omega_evals']],
                         tol_gmres=[float(v) for v in R.trace['tol_gmres']],
                         x_sample=R.x[sample].tolist(), x_norm=float(np.linalg.norm(R.x)),
                         u_norm=float(np.linalg.norm(R.x[:P.nv])), seconds=time.time() - t)
        print(name, out[name]['total'], out[name]['newton_iters'], out[name]['seconds'], flush=True)
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), 'multi_charge_sphere.json')
    with open(path, 'w') as f:
        json.dump(out, f, indent=1)
    print('wrote', path)


if __name__ == '__main__':
    main()
