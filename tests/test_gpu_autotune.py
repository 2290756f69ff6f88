"""The launch-shape autotuner (pbfb_autotune): valid shapes, applied to the mesh, cached in a
JSON file per GPU and size bucket, and results unchanged up to rounding."""
import json

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def dev(a):
    import torch
    return torch.as_tensor(np.ascontiguousarray(a, np.float64), device="cuda")


def test_autotune_shapes_cache_and_results(small_case, tmp_path):
    from paper_2511_21713_gb300 import pbfb
    c = small_case
    m = pbfb.Mesh.from_case(c)
    m.charges_set(c.q_xyz, c.q_z)
    m.set_params(c.eps_in, c.eps_out, c.kappa, c.T, pbfb.MIXED)
    x = dev(np.random.default_rng(2).standard_normal(m.n))
    y0 = dev(np.zeros(m.n))
    m.apply(x, y0)
    f0 = {}
    m.set_params(c.eps_in, c.eps_out, c.kappa, c.T, pbfb.FLOAT2)
    for which, n in ((pbfb.GAMMA_M, m.n_m), (pbfb.GAMMA_S, m.n_s)):
        f0[which] = dev(np.zeros(n))
        m.bem_apply(which, 0, x[:n].clone(), f0[which])
    _, r0 = m.solve(c.eps_in, c.eps_out, c.kappa, c.T, pbfb.default_opts(precision=pbfb.MIXED))
    m.set_params(c.eps_in, c.eps_out, c.kappa, c.T, pbfb.MIXED)

    cache = tmp_path / "tuning.json"
    shapes, ms = m.autotune(reps=2, cache_file=str(cache))
    assert shapes == m.get_tuning()
    assert shapes["nbody_targets_per_thread"] in (1, 2, 4) and shapes["nbody_blocks_per_sm"] in (0, 8, 16, 32, 64)
    assert shapes["nbody_packed"] in (0, 1, 2)
    assert shapes["ff_blocks_per_sm"] in (4, 8, 16, 24) and shapes["ff_kernel"] in (1, 2, 3, 4)
    assert shapes["spmv_lanes"] in (4, 8, 16) and shapes["spmv_block"] in (128, 256, 512)
    assert shapes["pcg_blocks_per_sm"] in (0, 1, 2, 4, 8) and shapes["pcg_lanes"] in (1, 2, 4, 8)
    assert shapes["treecode"] in (1, 2, 3)
    assert all(v > 0 for v in ms.values())
    stored = json.load(open(cache))
    assert len(stored) == 1 and list(stored.values())[0]["shapes"] == shapes

    y1 = dev(np.zeros(m.n))
    m.apply(x, y1)
    a, b = y1.cpu().numpy(), y0.cpu().numpy()
    assert np.abs(a - b).max() <= 3e-6 * np.abs(b).max()
    m.set_params(c.eps_in, c.eps_out, c.kappa, c.T, pbfb.FLOAT2)
    for which, n in ((pbfb.GAMMA_M, m.n_m), (pbfb.GAMMA_S, m.n_s)):
        f1 = dev(np.zeros(n))
        m.bem_apply(which, 0, x[:n].clone(), f1)
        a, b = f1.cpu().numpy(), f0[which].cpu().numpy()
        assert np.abs(a - b).max() <= 1e-13 * np.abs(b).max()
    _, r1 = m.solve(c.eps_in, c.eps_out, c.kappa, c.T, pbfb.default_opts(precision=pbfb.MIXED))
    assert abs(r1["total"] - r0["total"]) < 1e-8 * abs(r0["total"])

    # a second mesh of the same sizes takes the cached shapes without timing
    m2 = pbfb.Mesh.from_case(c)
    m2.set_params(c.eps_in, c.eps_out, c.kappa, c.T, pbfb.MIXED)
    s2, ms2 = m2.autotune(reps=2, cache_file=str(cache))
    assert s2 == shapes and m2.get_tuning() == shapes and ms2 == ms
    with pytest.raises(pbfb.PbfbError) as e:
        m2.apply_tuning(dict(shapes, spmv_lanes=3))
    assert e.value.code == 1
    m2.close()
    m.close()
