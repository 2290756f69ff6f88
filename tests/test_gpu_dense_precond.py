"""Dense single-layer matrices and inverses (the surface block of the
PBFB_PRECOND_BLOCK_DENSE preconditioner), through the C ABI, against the oracle.

* V assembled on the GPU in float32 equals the oracle's Galerkin V (symmetrised)
  within 1e-5 of its largest entry (float32 sums of 36 x 36 kernel terms);
* the float32 sweep inverse satisfies |V^-1 V - I| < 2e-3 entrywise with the
  oracle's V (float32 rounding times the condition number of V);
* flexible GMRES with the dense block reaches the direct solution in fewer
  iterations than with the diagonal block, also after kappa changes.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def dev(a):
    import torch
    return torch.as_tensor(np.ascontiguousarray(a, np.float64), device="cuda")


def rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(b)


@pytest.fixture(scope="module", params=["tiny", "small"])
def pair(request, tiny_case, small_case, bem_cache):
    from paper_2511_21713_gb300 import pbfb
    from oracle import pb
    case = tiny_case if request.param == "tiny" else small_case
    m = pbfb.Mesh.from_case(case)
    m.charges_set(case.q_xyz, case.q_z)
    P = pb.Problem(case, bem_cache=bem_cache)
    yield case, m, P
    m.close()


def _dense(m, which, inverse, n):
    import torch
    out = torch.zeros((n, n), dtype=torch.float32, device="cuda")
    m.single_layer_dense(which, inverse, out)
    return out.cpu().numpy().astype(np.float64)


def test_dense_single_layer_matches_oracle(pair):
    from paper_2511_21713_gb300 import pbfb
    case, m, P = pair
    m.set_params(case.eps_in, case.eps_out, case.kappa, case.T)
    for which, V in ((pbfb.GAMMA_M, P.VL), (pbfb.GAMMA_S, P.VY)):
        G = _dense(m, which, 0, V.shape[0])
        Vs = 0.5 * (V + V.T)
        assert np.array_equal(G, G.T)
        assert np.abs(G - Vs).max() < 1e-5 * np.abs(Vs).max(), which


def test_dense_inverse(pair):
    from paper_2511_21713_gb300 import pbfb
    case, m, P = pair
    m.set_params(case.eps_in, case.eps_out, case.kappa, case.T)
    for which, V in ((pbfb.GAMMA_M, P.VL), (pbfb.GAMMA_S, P.VY)):
        Vs = 0.5 * (V + V.T)
        Gi = _dense(m, which, 1, V.shape[0])
        E = Gi @ Vs - np.eye(V.shape[0])
        assert np.abs(E).max() < 2e-3, (which, np.abs(E).max())
        # much closer to V^-1 than the diagonal scaling it replaces
        Ed = np.diag(1.0 / np.diag(Vs)) @ Vs - np.eye(V.shape[0])
        assert np.linalg.norm(E, 2) < 0.01 * np.linalg.norm(Ed, 2)


def test_dense_block_gmres(pair):
    from paper_2511_21713_gb300 import pbfb
    from oracle import pb
    case, m, P = pair
    m.set_params(case.eps_in, case.eps_out, case.kappa, case.T)
    u = 4.0 * np.exp(-0.3 * (np.linalg.norm(P.xyz, axis=1) - 4.0))
    m.assemble(pbfb.HS, dev(u))
    b = np.random.default_rng(12).standard_normal(P.n)
    xd = pb.linear_solve(P, P.J(u, "HS"), b, 0, pb.Opts(linear_solver="direct"))[0]
    xb, xs = dev(np.zeros(P.n)), dev(np.zeros(P.n))
    its_b, _ = m.gmres(dev(b), xb, 1e-11, precond=pbfb.BLOCK, inner_iters=20)
    its_d, rd = m.gmres(dev(b), xs, 1e-11, precond=pbfb.BLOCK_DENSE, inner_iters=20)
    assert rd <= 1e-11 and rel(xs.cpu().numpy(), xd) < 1e-8
    assert its_d < its_b, (its_d, its_b)


def test_dense_rebuilt_when_kappa_changes(tiny_case, bem_cache):
    from paper_2511_21713_gb300 import pbfb
    from oracle import pb
    c = tiny_case
    m = pbfb.Mesh.from_case(c)
    m.charges_set(c.q_xyz, c.q_z)
    b = np.random.default_rng(13).standard_normal(m.n)
    for kappa in (c.kappa, 2.5 * c.kappa):
        m.set_params(c.eps_in, c.eps_out, kappa, c.T)
        m.clear_jacobian()
        P = pb.Problem(c, kappa=kappa, bem_cache=bem_cache)
        x = dev(np.zeros(m.n))
        its, r = m.gmres(dev(b), x, 1e-11, precond=pbfb.BLOCK_DENSE, inner_iters=20)
        xd = pb.linear_solve(P, P.J(np.zeros(P.nv), "linear") * 0.0, b, 0, pb.Opts(linear_solver="direct"))[0]
        assert r <= 1e-11 and rel(x.cpu().numpy(), xd) < 1e-8, kappa
        Vs = 0.5 * (P.VY + P.VY.T)
        Gi = _dense(m, pbfb.GAMMA_S, 1, P.ns)
        assert np.abs(Gi @ Vs - np.eye(P.ns)).max() < 2e-3, kappa
    m.close()


def test_dense_errors(tiny_case):
    import torch
    from paper_2511_21713_gb300 import pbfb
    c = tiny_case
    m = pbfb.Mesh.from_case(c)
    out = torch.zeros((m.n_m, m.n_m), dtype=torch.float32, device="cuda")
    with pytest.raises(pbfb.PbfbError) as e:
        m.single_layer_dense(pbfb.GAMMA_M, 1, out)
    assert e.value.code == 8                       # STATE: parameters not set
    m.set_params(c.eps_in, c.eps_out, c.kappa, c.T)
    with pytest.raises(pbfb.PbfbError) as e:
        m.single_layer_dense(5, 1, out)
    assert e.value.code == 1
    with pytest.raises(pbfb.PbfbError) as e:
        m.single_layer_dense(pbfb.GAMMA_M, 1, out, ld=m.n_m - 1)
    assert e.value.code == 1
    m.single_layer_dense(pbfb.GAMMA_M, 1, out)
    assert torch.isfinite(out).all()
    m.close()


@pytest.mark.parametrize("lanes,prec", [(1, 0), (2, 1), (4, 1), (8, 1), (2, 2), (4, 2), (8, 2)])
def test_inner_pcg_lane_variants(pair, lanes, prec):
    """Every sparse-product form of the cooperative inner PCG (2, 4 or 8 lanes per CSR row, or one
    lane per row of the sliced-ELL copy, ragged last slice included), in float64 (1) and float32
    (2), gives a preconditioner with which flexible GMRES reaches the direct solution."""
    from paper_2511_21713_gb300 import pbfb
    from oracle import pb
    case, m, P = pair
    m.set_params(case.eps_in, case.eps_out, case.kappa, case.T)
    base = m.get_tuning()
    try:
        m.apply_tuning(dict(base, pcg_lanes=lanes, pcg_precision=prec))
        u = 3.0 * np.exp(-0.3 * (np.linalg.norm(P.xyz, axis=1) - 4.0))
        m.assemble(pbfb.HS, dev(u))
        b = np.random.default_rng(14).standard_normal(P.n)
        xd = pb.linear_solve(P, P.J(u, "HS"), b, 0, pb.Opts(linear_solver="direct"))[0]
        x = dev(np.zeros(P.n))
        its, r = m.gmres(dev(b), x, 1e-11, precond=pbfb.BLOCK_DENSE, inner_iters=30)
        assert r <= 1e-11 and rel(x.cpu().numpy(), xd) < 1e-8
    finally:
        m.apply_tuning(base)
