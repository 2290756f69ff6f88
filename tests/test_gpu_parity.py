"""Parity of every step of the CUDA path against the CPU oracle, through the C ABI.

Inputs are the seeded spheres of paper_2511_21713_gb300.inputs: the small
single-charge sphere (nu = 5, 13 layers: 3528 vertices, 19,500 tets, 500 + 500
triangles, several GPU tiles and ragged tails everywhere) and a tiny one
(nu = 3, 5 layers).  Tolerances: float64 path 1e-11 relative per step,
1e-8 relative L2 on the converged potentials and 1e-9 on the solvation energy;
the mixed path (float32 far field) 1e-5 on the energy.
"""
import numpy as np
import pytest
import scipy.sparse as sp

pytestmark = pytest.mark.gpu

TIGHT = dict(tol_gmres0=1e-12, tol_gmres=1e-12, tol_nl=1e-11)


def dev(a):
    import torch
    return torch.as_tensor(np.ascontiguousarray(a, np.float64), device="cuda")


def host(t):
    return t.detach().cpu().numpy()


def rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300)


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


def _u_field(P, seed=0):
    rng = np.random.default_rng(seed)
    r = np.linalg.norm(P.xyz, axis=1)
    return 4.0 * np.exp(-0.3 * (r - r.min())) + 0.2 * rng.standard_normal(P.nv)


def test_surface_vertex_order(pair):
    from paper_2511_21713_gb300 import pbfb
    _, m, P = pair
    assert np.array_equal(m.surface_vertices(pbfb.GAMMA_M), P.sm.verts)
    assert np.array_equal(m.surface_vertices(pbfb.GAMMA_S), P.ss.verts)
    assert (m.n_v, m.n_m, m.n_s, m.n) == (P.nv, P.nm, P.ns, P.n)


SCHEMES = {"linear": 0, "T3": 1, "HS": 2, "T5": 3, "T7": 4}


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("scheme", ["linear", "T3", "T5", "T7", "HS"])
def test_fem_rows_and_load(pair, scheme, precision):
    """FEM rows of A + J and the load N against the oracle; the mixed precision (1) takes sinh and
    cosh from the float-float exponential on the float32 pipes, the same tolerances."""
    case, m, P = pair
    m.set_params(case.eps_in, case.eps_out, case.kappa, case.T, precision)
    u = _u_field(P, 1)
    N_dev = dev(np.zeros(P.nv))
    m.assemble(SCHEMES[scheme], dev(u), N_dev)
    rp, col, val = m.fem_rows()
    G = sp.csr_matrix((val, col, rp), shape=(P.nv, P.n))
    O = sp.hstack([P.A + P.J(u, scheme), P.B_um, P.B_us]).tocsr()
    D = (G - O).toarray()
    assert np.abs(D).max() <= 1e-12 * np.abs(O).max()
    N_ref = P.N(u, scheme)
    assert rel(host(N_dev), N_ref) < 1e-13


@pytest.mark.parametrize("precision", [0, 1])
def test_sinh_rows_wide_range(pair, precision):
    """The sinh scheme with potentials from -75 to 75 (linear in x): the mixed precision's
    float-float kernels take the tets with all |u| <= 60 and the float64 sums the others, in the
    same launch.  Every FEM entry within 1e-12 of |A| + |J| (entrywise), every load within 1e-12
    of its row of J (cosh >= |sinh|), the omega dots within 1e-11 of the largest."""
    from paper_2511_21713_gb300 import pbfb
    from oracle import pb
    case, m, P = pair
    m.set_params(case.eps_in, case.eps_out, case.kappa, case.T, precision)
    x = P.xyz[:, 0]
    u = -75.0 + 150.0 * (x - x.min()) / (x.max() - x.min())
    assert (np.abs(u) > 60).any() and (np.abs(u) < 60).any()
    N_dev = dev(np.zeros(P.nv))
    m.assemble(SCHEMES["HS"], dev(u), N_dev)
    rp, col, val = m.fem_rows()
    G = sp.csr_matrix((val, col, rp), shape=(P.nv, P.n))
    Jm = P.J(u, "HS")
    O = sp.hstack([P.A + Jm, P.B_um, P.B_us]).tocsr()
    S = sp.hstack([abs(P.A) + abs(Jm), abs(P.B_um), abs(P.B_us)]).toarray()
    D = np.abs((G - O).toarray())
    assert (D <= 1e-12 * S).all()
    N_ref = P.N(u, "HS")
    row = np.asarray(abs(Jm).sum(axis=1)).ravel()
    assert (np.abs(host(N_dev) - N_ref) <= 1e-12 * row).all()
    rng = np.random.default_rng(3)
    du = 0.3 * rng.standard_normal(P.nv)
    c = rng.standard_normal(P.n)
    p = rng.standard_normal(P.n)
    oms = np.array([0.0, 1.0, -2.0])
    got = m.omega_eval(SCHEMES["HS"], dev(u), dev(du), dev(c), dev(p), oms)
    for o, om in enumerate(oms):
        Dd = pb.omega_dots(P, u, du, c, p, om, "HS")
        ref = [Dd["PR"], Dd["PP"], Dd["PRp"], Dd["RRpp"], Dd["PRpp"], Dd["RR"], Dd["pr"], Dd["pp"]]
        scale = max(abs(v) for v in ref)
        assert np.isfinite(got[o]).all() and np.abs(got[o] - ref).max() < 1e-11 * scale, om


@pytest.mark.parametrize("precision", [0, 1, 2])
def test_boundary_operators(pair, precision):
    """float64 (0) and float-float (2) far fields within 1e-11 of the oracle; float32 (1) 3e-6."""
    from paper_2511_21713_gb300 import pbfb
    case, m, P = pair
    m.set_params(case.eps_in, case.eps_out, case.kappa, case.T, precision)
    tol = 3e-6 if precision == pbfb.MIXED else 1e-11
    rng = np.random.default_rng(2)
    for which, Vo, Ko, n in ((pbfb.GAMMA_M, P.VL, P.KL, P.nm), (pbfb.GAMMA_S, P.VY, P.KY, P.ns)):
        for op, Mo in ((0, Vo), (1, Ko)):
            x = rng.standard_normal(n) + 1.0
            y = dev(np.zeros(n))
            m.bem_apply(which, op, dev(x), y)
            assert rel(host(y), Mo @ x) < tol, (which, op)


@pytest.mark.parametrize("shape", [dict(nbody_targets_per_thread=4, nbody_packed=2, nbody_blocks_per_sm=32),
                                   dict(nbody_targets_per_thread=1, nbody_packed=0, nbody_blocks_per_sm=16),
                                   dict(nbody_targets_per_thread=2, nbody_packed=1, nbody_blocks_per_sm=32),
                                   dict(treecode=2), dict(treecode=3)])
def test_float32_far_field_variants(pair, shape):
    """Every float32 far-field variant (mutual pairs, one target per thread, packed f32x2, the
    treecode: leaves of 256 points, ragged here) within 3e-6 of the oracle's operators, ragged
    tails included."""
    from paper_2511_21713_gb300 import pbfb
    case, m, P = pair
    m.set_params(case.eps_in, case.eps_out, case.kappa, case.T, pbfb.MIXED)
    base = m.get_tuning()
    rng = np.random.default_rng(8)
    try:
        m.apply_tuning(dict(base, **shape))
        for which, Vo, Ko, n in ((pbfb.GAMMA_M, P.VL, P.KL, P.nm), (pbfb.GAMMA_S, P.VY, P.KY, P.ns)):
            for op, Mo in ((0, Vo), (1, Ko)):
                x = rng.standard_normal(n) + 1.0
                y = dev(np.zeros(n))
                m.bem_apply(which, op, dev(x), y)
                assert rel(host(y), Mo @ x) < 3e-6, (which, op)
    finally:
        m.apply_tuning(base)


@pytest.mark.parametrize("precision", [0, 1, 2])
def test_coupled_apply(pair, precision):
    from paper_2511_21713_gb300 import pbfb
    case, m, P = pair
    m.set_params(case.eps_in, case.eps_out, case.kappa, case.T, precision)
    u = _u_field(P, 3)
    m.assemble(pbfb.HS, dev(u))
    x = np.random.default_rng(4).standard_normal(P.n)
    y = dev(np.zeros(P.n))
    m.apply(dev(x), y)
    ref = P.apply(x, P.J(u, "HS"))
    tol = 3e-6 if precision == pbfb.MIXED else 1e-11
    for a, b in zip(P.split(host(y)), P.split(ref)):
        assert rel(a, b) < tol
    m.clear_jacobian()
    m.apply(dev(x), y)
    assert rel(host(y), P.apply(x)) < tol


def test_gmres_against_direct_solve(pair):
    from paper_2511_21713_gb300 import pbfb
    from oracle import pb
    case, m, P = pair
    m.set_params(case.eps_in, case.eps_out, case.kappa, case.T)
    u = _u_field(P, 5)
    m.assemble(pbfb.T3, dev(u))
    b = np.random.default_rng(6).standard_normal(P.n)
    x = dev(np.zeros(P.n))
    its, r = m.gmres(dev(b), x, 1e-12)
    xd = pb.linear_solve(P, P.J(u, "T3"), b, 0, pb.Opts(linear_solver="direct"))[0]
    assert r <= 1e-12 and rel(host(x), xd) < 1e-9
    # same Krylov method, same preconditioner: iteration counts agree closely
    _, its_o, _ = pb.gmres(lambda v: P.apply(v, P.J(u, "T3")), b, 1e-12, 200, 2000, P.jacobi(P.J(u, "T3")))
    assert abs(its - its_o) <= max(2, its_o // 50)


def test_block_preconditioned_gmres(pair):
    """Flexible GMRES with the inner-PCG block preconditioner reaches the same solution
    in fewer outer iterations than Jacobi."""
    from paper_2511_21713_gb300 import pbfb
    from oracle import pb
    case, m, P = pair
    m.set_params(case.eps_in, case.eps_out, case.kappa, case.T)
    u = _u_field(P, 9)
    m.assemble(pbfb.HS, dev(u))
    b = np.random.default_rng(10).standard_normal(P.n)
    xd = pb.linear_solve(P, P.J(u, "HS"), b, 0, pb.Opts(linear_solver="direct"))[0]
    xj, xb = dev(np.zeros(P.n)), dev(np.zeros(P.n))
    its_j, _ = m.gmres(dev(b), xj, 1e-11, precond=pbfb.JACOBI)
    its_b, rb = m.gmres(dev(b), xb, 1e-11, precond=pbfb.BLOCK, inner_iters=30)
    assert rb <= 1e-11 and rel(host(xb), xd) < 1e-8
    assert its_b < its_j


@pytest.mark.parametrize("precision", [0, 1])
def test_omega_batch(pair, precision):
    """The batched omega dots against the oracle's, 1e-11 of the largest, in float64 and in the
    mixed precision (sinh / cosh from the float-float exponential); omega 3.9 puts the sinh
    arguments well beyond the table's central range."""
    from paper_2511_21713_gb300 import pbfb
    from oracle import pb
    case, m, P = pair
    m.set_params(case.eps_in, case.eps_out, case.kappa, case.T, precision)
    rng = np.random.default_rng(7)
    u = _u_field(P, 8)
    du = 0.3 * rng.standard_normal(P.nv)
    c = rng.standard_normal(P.n)
    p = rng.standard_normal(P.n)
    oms = np.array([0.0, 0.5, 1.0, 1.7, 2.0, 3.9])
    for sname in ("T3", "T5", "T7", "HS"):
        got = m.omega_eval(SCHEMES[sname], dev(u), dev(du), dev(c), dev(p), oms)
        for o, om in enumerate(oms):
            D = pb.omega_dots(P, u, du, c, p, om, sname)
            ref = [D["PR"], D["PP"], D["PRp"], D["RRpp"], D["PRpp"], D["RR"], D["pr"], D["pp"]]
            scale = max(abs(v) for v in ref)
            assert np.abs(got[o] - ref).max() < 1e-11 * scale, (sname, om)


def test_energy_of_oracle_solution(pair):
    from oracle import pb
    case, m, P = pair
    m.set_params(case.eps_in, case.eps_out, case.kappa, case.T)
    R = pb.solve(P, pb.Opts(**TIGHT))
    got = m.energy(dev(R.xL), dev(R.xNL))
    ref = [R.total, R.LC, R.NC, R.dG_ion]
    for g, r in zip(got, ref):
        assert abs(g - r) < 1e-11 * abs(R.total)


def test_full_solve_fp64_tight(pair):
    from paper_2511_21713_gb300 import pbfb
    from oracle import pb
    case, m, P = pair
    x, res = m.solve(case.eps_in, case.eps_out, case.kappa, case.T, pbfb.default_opts(**TIGHT))
    R = pb.solve(P, pb.Opts(**TIGHT))
    for a, b in zip(P.split(x), P.split(R.x)):
        assert rel(a, b) < 1e-8
    assert abs(res["total"] - R.total) < 1e-9 * abs(R.total)
    assert abs(res["LC"] - R.LC) < 1e-9 * abs(R.total)
    assert abs(res["dG_ion"] - R.dG_ion) < 1e-9 * abs(R.total)
    # at Tol_NL = 1e-11 the last step sits at rounding level: one more or less is allowed
    assert abs(res["newton_iters"] - R.newton_iters) <= 1


def test_full_solve_mixed(pair):
    """Float32 far field: its rounding noise floors the reachable relative residual near
    1e-8, so the tolerances sit above it; the energy must still be within 1e-5."""
    from paper_2511_21713_gb300 import pbfb
    from oracle import pb
    case, m, P = pair
    x, res = m.solve(case.eps_in, case.eps_out, case.kappa, case.T,
                     pbfb.default_opts(precision=pbfb.MIXED, tol_gmres0=1e-7, tol_gmres=1e-7, tol_nl=1e-6))
    R = pb.solve(P, pb.Opts(**TIGHT))
    assert abs(res["total"] - R.total) < 1e-5 * abs(R.total)
    assert rel(x, R.x) < 1e-4


def test_paper_default_trace(pair):
    """Paper tolerances with the oracle's Jacobi preconditioner: same Newton path."""
    from paper_2511_21713_gb300 import pbfb
    from oracle import pb
    case, m, P = pair
    _, res = m.solve(case.eps_in, case.eps_out, case.kappa, case.T, pbfb.default_opts(precond=pbfb.JACOBI))
    R = pb.solve(P, pb.Opts())
    assert res["newton_iters"] == R.newton_iters
    assert np.allclose(res["omega"], R.trace["omega"], rtol=1e-3, atol=1e-3)
    for g, o in zip(res["gmres"], R.trace["gmres"]):
        assert abs(g - o) <= 2
    assert abs(res["total"] - R.total) < 1e-4 * abs(R.total)


def test_picard_and_taylor_schedules(pair):
    """Picard (Sec. 2.4.1, direct-secant omega, R_e rule) and the T3-T5-T7-T7-HS schedule reach
    the oracle's discrete solution; at the paper's tolerances Picard follows the oracle's path."""
    from paper_2511_21713_gb300 import pbfb
    from oracle import pb
    case, m, P = pair
    ref = pb.solve(P, pb.Opts(**TIGHT))
    for gkw, okw in ((dict(method=pbfb.PICARD, omega0_first=0.5, omega0_rest=0.5),
                      dict(method="picard", omega0_first=0.5, omega0_rest=0.5)),
                     (dict(taylor=[pbfb.T3, pbfb.T5, pbfb.T7, pbfb.T7]), dict(taylor=("T3", "T5", "T7", "T7"))),
                     (dict(omega_warm_start=1), dict(omega_warm_start=True))):
        tight = dict(tol_gmres0=1e-12, tol_gmres=1e-12, tol_nl=1e-10)
        x, res = m.solve(case.eps_in, case.eps_out, case.kappa, case.T, pbfb.default_opts(**gkw, **tight))
        assert abs(res["total"] - ref.total) < 1e-9 * abs(ref.total)
        assert rel(x, ref.x) < 1e-8
        _, rp = m.solve(case.eps_in, case.eps_out, case.kappa, case.T,
                        pbfb.default_opts(precond=pbfb.JACOBI, **gkw))
        Ro = pb.solve(P, pb.Opts(**okw))
        assert rp["newton_iters"] == Ro.newton_iters
        assert np.allclose(rp["omega"], Ro.trace["omega"], rtol=1e-3, atol=1e-3)


def test_forced_fallback_and_picard_secant_follow_the_oracle(pair):
    """The omega search's scan-and-bisect fallback (forced: one Newton step on f_d, unreachable
    Tol_omega) for Newton and Picard, and Picard's direct secant (Eq. SEC_FD) with its R_e reuse
    rule, through pbfb_solve at tight GMRES tolerances: the oracle's omega sequence to 1e-9, the
    same number of fallbacks, and the same discrete solution (1e-8 L2, 1e-9 energy)."""
    from paper_2511_21713_gb300 import pbfb
    from oracle import pb
    case, m, P = pair
    tight = dict(tol_gmres0=1e-12, tol_gmres=1e-12, tol_nl=1e-10)
    forced = dict(max_omega_iters=1, tol_omega=1e-14)
    pic = dict(omega0_first=0.5, omega0_rest=0.5)
    for gkw, okw in ((forced, forced),
                     (dict(method=pbfb.PICARD, **pic, **forced), dict(method="picard", **pic, **forced)),
                     (dict(method=pbfb.PICARD, **pic), dict(method="picard", **pic))):
        x, res = m.solve(case.eps_in, case.eps_out, case.kappa, case.T, pbfb.default_opts(**gkw, **tight))
        R = pb.solve(P, pb.Opts(**okw, **tight))
        assert res["newton_iters"] == R.newton_iters, okw
        assert np.abs(np.array(res["omega"]) - np.array(R.trace["omega"])).max() < 1e-9, okw
        assert res["omega_fallbacks"] == R.trace.get("fallback", 0), okw
        if "max_omega_iters" in okw:
            assert res["omega_fallbacks"] >= 1
        assert abs(res["total"] - R.total) < 1e-9 * abs(R.total)
        assert rel(x, R.x) < 1e-8


def test_residual_update_option(pair):
    """Mixed solves with residual_update reach the oracle's energy within the mixed-path 1e-5
    (paper tolerances) and its solution at tight tolerances within 1e-6; the float64 path never
    updates (the option is ignored there)."""
    from paper_2511_21713_gb300 import pbfb
    from oracle import pb
    case, m, P = pair
    ref = pb.solve(P, pb.Opts(**TIGHT))
    _, r = m.solve(case.eps_in, case.eps_out, case.kappa, case.T,
                   pbfb.default_opts(precision=pbfb.MIXED, residual_update=0.5))
    assert r["residual_updates"] >= 1 and abs(r["total"] - ref.total) < 1e-5 * abs(ref.total)
    x, r = m.solve(case.eps_in, case.eps_out, case.kappa, case.T,
                   pbfb.default_opts(precision=pbfb.MIXED, residual_update=0.5, tol_gmres0=1e-10,
                                     tol_gmres=1e-10, tol_nl=1e-8))
    assert r["status"] == 0 and rel(x, ref.x) < 1e-6
    _, r = m.solve(case.eps_in, case.eps_out, case.kappa, case.T, pbfb.default_opts(residual_update=0.5))
    assert r["residual_updates"] == 0


@pytest.mark.parametrize("residual_update", [0.0, 0.5])
def test_residual_far_float32(pair, residual_update):
    """The Newton residual's full evaluations with the GMRES operator's float32 far field
    (residual_far = MIXED): the oracle's energy within the mixed-path 1e-5 at the paper's
    tolerances, with and without residual updates; ignored by the float64 path (bitwise the same
    solve)."""
    from paper_2511_21713_gb300 import pbfb
    from oracle import pb
    case, m, P = pair
    ref = pb.solve(P, pb.Opts(**TIGHT))
    _, r = m.solve(case.eps_in, case.eps_out, case.kappa, case.T,
                   pbfb.default_opts(precision=pbfb.MIXED, residual_update=residual_update,
                                     residual_far=pbfb.MIXED))
    assert r["status"] == 0 and abs(r["total"] - ref.total) < 1e-5 * abs(ref.total)
    x1, r1 = m.solve(case.eps_in, case.eps_out, case.kappa, case.T, pbfb.default_opts(residual_far=pbfb.MIXED))
    x2, r2 = m.solve(case.eps_in, case.eps_out, case.kappa, case.T, pbfb.default_opts())
    assert np.array_equal(x1, x2) and r1["total"] == r2["total"]


def test_deterministic(pair):
    from paper_2511_21713_gb300 import pbfb
    case, m, _ = pair
    o = pbfb.default_opts(**TIGHT)
    x1, r1 = m.solve(case.eps_in, case.eps_out, case.kappa, case.T, o)
    x2, r2 = m.solve(case.eps_in, case.eps_out, case.kappa, case.T, o)
    assert np.array_equal(x1, x2) and r1["total"] == r2["total"]


def test_kappa_zero_born_limit(tiny_case, bem_cache):
    from paper_2511_21713_gb300 import pbfb
    from oracle import pb
    c = tiny_case
    m = pbfb.Mesh.from_case(c)
    m.charges_set(c.q_xyz, c.q_z)
    x, res = m.solve(c.eps_in, c.eps_out, 0.0, c.T, pbfb.default_opts(**TIGHT))
    P = pb.Problem(c, kappa=0.0, bem_cache=bem_cache)
    R = pb.solve(P, pb.Opts(**TIGHT))
    assert abs(res["total"] - R.total) < 1e-9 * abs(R.total)
    assert res["dG_ion"] == 0.0
    m.close()


def test_zero_charges(tiny_case):
    """No charge: the solution is exactly zero, the first Newton residual is zero and the
    iteration stops there (e_0 = 0), every energy term zero, as in the oracle."""
    from paper_2511_21713_gb300 import pbfb
    c = tiny_case
    m = pbfb.Mesh.from_case(c)
    m.charges_set(c.q_xyz, 0.0 * c.q_z)
    for precision in (pbfb.FP64, pbfb.MIXED):
        x, res = m.solve(c.eps_in, c.eps_out, c.kappa, c.T, pbfb.default_opts(precision=precision))
        assert res["status"] == 0 and res["newton_iters"] == 1 and res["linear_gmres"] == 0
        assert not np.any(x) and res["e"][0] == 0.0
        assert (res["total"], res["LC"], res["NC"], res["dG_ion"]) == (0.0, 0.0, 0.0, 0.0)
    m.close()


def test_error_statuses(tiny_case):
    from paper_2511_21713_gb300 import pbfb
    c = tiny_case
    m = pbfb.Mesh.from_case(c)
    with pytest.raises(pbfb.PbfbError) as e:
        m.solve(c.eps_in, c.eps_out, c.kappa, c.T)
    assert e.value.code == 8                       # STATE: no charges yet
    with pytest.raises(pbfb.PbfbError) as e:
        m.charges_set(np.array([[0.0, np.nan, 0.0]]), np.array([1.0]))
    assert e.value.code == 1
    m.charges_set(c.q_xyz, c.q_z)
    with pytest.raises(pbfb.PbfbError) as e:
        m.solve(-1.0, c.eps_out, c.kappa, c.T)
    assert e.value.code == 1
    with pytest.raises(pbfb.PbfbError) as e:
        m.solve(c.eps_in, c.eps_out, c.kappa, c.T, pbfb.default_opts(max_newton=1, tol_nl=1e-12))
    assert e.value.code == 4                       # NEWTON_NOCONV
    with pytest.raises(pbfb.PbfbError) as e:
        m.solve(c.eps_in, c.eps_out, c.kappa, c.T, pbfb.default_opts(max_gmres=3, tol_gmres0=1e-12))
    assert e.value.code == 3                       # GMRES_NOCONV
    _, ref = m.solve(c.eps_in, c.eps_out, c.kappa, c.T)
    # no relaxation factor may be accepted (||d(omega)||^2 < 0 ||d(0)||^2): the search and its
    # fallback both refuse
    with pytest.raises(pbfb.PbfbError) as e:
        m.solve(c.eps_in, c.eps_out, c.kappa, c.T, pbfb.default_opts(accept_ratio=0.0))
    assert e.value.code == 5                       # OMEGA
    # a constant omega of 1e300 overflows the update or the next residual's sinh
    with pytest.raises(pbfb.PbfbError) as e:
        m.solve(c.eps_in, c.eps_out, c.kappa, c.T, pbfb.default_opts(omega_search=0, omega0_first=1e300))
    assert e.value.code == 6                       # NONFINITE
    for bad in (dict(omega_max=float("inf")), dict(accept_ratio=1.5), dict(accept_ratio=-0.1),
                dict(residual_far=0), dict(residual_far=3)):
        with pytest.raises(pbfb.PbfbError) as e:
            m.solve(c.eps_in, c.eps_out, c.kappa, c.T, pbfb.default_opts(**bad))
        assert e.value.code == 1, bad
    # a charge on Gamma_m or outside it: refused on the host, the mesh keeps its charges
    face = c.xyz[c.gm_tris[3]].mean(axis=0)
    for q in (np.vstack([c.q_xyz, face]), np.vstack([c.q_xyz, [0.0, 0.0, 7.0]])):
        with pytest.raises(pbfb.PbfbError) as e:
            m.charges_set(q, np.ones(q.shape[0]))
        assert e.value.code == 1 and "not strictly inside" in str(e.value)
    # the handle stays usable after errors, with the same result
    _, res = m.solve(c.eps_in, c.eps_out, c.kappa, c.T)
    assert res["status"] == 0 and res["total"] == ref["total"]
    m.close()


def test_float_float_kernels_agree(pair):
    """The float-float far-field variants -- one target per thread, two per thread on float2
    instructions, mutual pairs evaluated once for both directions, and mutual pairs with two
    targets per thread on float2 -- agree to float-float rounding (1e-13 of the largest entry),
    ragged tails included."""
    from paper_2511_21713_gb300 import pbfb
    case, m, P = pair
    m.set_params(case.eps_in, case.eps_out, case.kappa, case.T, pbfb.FLOAT2)
    rng = np.random.default_rng(21)
    base = m.get_tuning()
    try:
        for which, n in ((pbfb.GAMMA_M, P.nm), (pbfb.GAMMA_S, P.ns)):
            x = dev(rng.standard_normal(n) + 0.5)
            for op in (0, 1):
                ys = {}
                for kind in (1, 2, 3, 4):
                    m.apply_tuning(dict(base, ff_kernel=kind))
                    ys[kind] = dev(np.zeros(n))
                    m.bem_apply(which, op, x, ys[kind])
                b = host(ys[1])
                for kind in (2, 3, 4):
                    a = host(ys[kind])
                    assert np.abs(a - b).max() <= 1e-13 * np.abs(b).max(), (which, op, kind, np.abs(a - b).max())
    finally:
        m.apply_tuning(base)
