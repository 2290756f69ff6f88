"""pbfb_bem_apply_noalloc: the boundary-operator apply for callers that may not
allocate GPU memory while they run (a host whose device memory belongs to its own
pool, or a request loop that must avoid the device-wide synchronisation of
cudaMalloc/cudaFree).  Its working memory is the library's fixed device array.

Checked through the C ABI against pbfb_bem_apply (same float32 far field and
float64 near-field correction) on two calls in a row, so that the second call
also sees the scratch the first call left behind.  This file runs last and must
pass alone in a fresh process as well as after the other tests.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


# surfaces: 500 triangles (3,000 points: one-target unpacked kernel), 8,000 triangles (48,000
# points: the packed kernel, and more source splits than the fixed array's 8 in pbfb_bem_apply)
@pytest.fixture(scope="module", params=["tiny", "small", "bench"])
def mesh_case(request):
    from paper_2511_21713_gb300 import inputs, pbfb
    case = {"tiny": lambda: inputs.single_charge_sphere(nu=3, layers=5),
            "small": lambda: inputs.single_charge_sphere(nu=5, layers=13),
            "bench": lambda: inputs.sphere_case(nu=20, a=12.0, R=24.0, layers=2, eps_in=2.0,
                                                ionic=0.1)}[request.param]()
    m = pbfb.Mesh.from_case(case)
    m.set_params(case.eps_in, case.eps_out, case.kappa, case.T, pbfb.MIXED)
    yield case, m
    m.close()


def _compare(m, tol, seed):
    import torch
    from paper_2511_21713_gb300 import pbfb
    rng = np.random.default_rng(seed)
    for which, n in ((pbfb.GAMMA_M, m.n_m), (pbfb.GAMMA_S, m.n_s)):
        for op in (0, 1):
            xs = [torch.as_tensor(rng.standard_normal(n) + 1.0, device="cuda") for _ in range(2)]
            for x in xs:                                   # two calls in a row, different inputs
                ref = torch.zeros(n, dtype=torch.float64, device="cuda")
                got = torch.full((n,), np.nan, dtype=torch.float64, device="cuda")
                m.bem_apply(which, op, x, ref)
                m.bem_apply_noalloc(which, op, x, got)
                r, g = ref.cpu().numpy(), got.cpu().numpy()
                assert np.all(np.isfinite(g))
                assert np.linalg.norm(g - r) <= tol * np.linalg.norm(r), (which, op)


def test_noalloc_matches_bem_apply_on_consecutive_calls(mesh_case):
    """Built-in launch shapes: same kernels and split tiles, sums equal to float64 rounding."""
    _, m = mesh_case
    m.apply_tuning({})
    _compare(m, 1e-11, 21)


def test_noalloc_matches_bem_apply_under_tuned_shapes(mesh_case):
    """Shapes an autotuner picks: packed two targets per thread with the whole-wave split
    (blocks_per_sm 0) agrees to float64 rounding; a mesh tuned to the mutual-pair kernel runs the
    packed split kernel here, whose float32 sums run in another order (float32 rounding)."""
    _, m = mesh_case
    try:
        m.apply_tuning(dict(nbody_targets_per_thread=2, nbody_blocks_per_sm=0, nbody_packed=1))
        _compare(m, 1e-11, 22)
        m.apply_tuning(dict(nbody_targets_per_thread=4, nbody_blocks_per_sm=32, nbody_packed=2))
        _compare(m, 3e-6, 23)
    finally:
        m.apply_tuning({})


def test_noalloc_rejects_surfaces_beyond_its_limit():
    from paper_2511_21713_gb300 import inputs, pbfb
    import torch
    # nu = 24: 11,520 triangles = 69,120 quadrature points, just over the 65,536 the array holds
    case = inputs.sphere_case(nu=24, a=4.0, R=5.0, layers=1)
    m = pbfb.Mesh.from_case(case)
    m.set_params(case.eps_in, case.eps_out, case.kappa, case.T, pbfb.MIXED)
    x = torch.ones(m.n_m, dtype=torch.float64, device="cuda")
    y = torch.zeros_like(x)
    with pytest.raises(pbfb.PbfbError) as e:
        m.bem_apply_noalloc(pbfb.GAMMA_M, 0, x, y)
    assert e.value.code == 1 and "at most 65536" in str(e.value)
    m.close()
